"""Seeded synthetic workloads: problem statements only.

This module is the one thing the CUDA path and the FP64 oracle both read.
It holds parameter records and seeded parameter draws, none of the method's
arithmetic (no propagation, moments, matching or Parareal step).

The model family is the scalar McKean-Vlasov SDE of Sec. 2.1
Eq. (SDE_class_1) with f(x) = x,

    dX = a(X, E[X]) dt + b(X, E[X]) dW,
    a(x, m) = -c3 x^3 + c1 x + kappa m + c0,
    b(x, m) = B x + BE m + B0,

which covers the linear SDE of Lemma 2.1 (c3 = 0), the cubic drift and the
double well V(x) = a x^4 - b x^2 of Sec. 5.3 Eq. (SDE_bimodal_first_time)
(c3 = 4a, the x coefficient 2b, plus the mean-field term kappa (E[X] - x)).

A second family (family = ROTATOR) is the plane rotator of Sec. 5 (Example
"Unimodal plane rotator", Eq. SDE_plane_rotator): drift
(K/P) sum_q sin(X_q - x) - g sin x, additive noise B0 = sqrt(2 k_B T), the
particles shifted modulo 2 pi into [-pi, pi] (centred on the stable point of
-sin x; the paper prints [0, 2 pi]).  Only the oracle propagates it so far;
the CUDA library refuses it.

The paper runs on synthetic SDEs only (no dataset, Sec. 5); the five
workloads below take the shapes of its unimodal and bimodal examples at the
sizes the project measures.
"""
from __future__ import annotations

import copy
from dataclasses import dataclass, replace

import numpy as np

UNIMODAL, MULTIMODAL, LEARNING = 0, 1, 2
CLOSURE, TAYLOR, SIGMA2, SIGMA3, TAYLOR1 = 0, 1, 2, 3, 4  # coarse moment models
POLY, ROTATOR = 0, 1  # drift families
SEED_BASE = 0x231011365


@dataclass
class Problem:
    c3: float = 0.0
    c1: float = 0.0
    kappa: float = 0.0
    c0: float = 0.0
    B: float = 0.0
    BE: float = 0.0
    B0: float = 0.0
    m0: float = 0.0
    s0: float = 0.0
    T: float = 1.0
    N: int = 1
    dt: float = 1e-3
    P: int = 1
    coarse_h: float = 0.25
    n_regions: int = 1
    threshold: float = 0.0
    variant: int = UNIMODAL
    seed: int = 0
    problem_tag: int = 0
    tol: float = 1e-8
    max_iter: int = 0          # 0 means N
    precision: str = "fp64"    # "fp64" or "mixed" (FP32 particles)
    coarse_model: int = 0      # CLOSURE, TAYLOR, SIGMA2 or SIGMA3
    threshold2: float = 0.0    # region boundaries t_2 < t_3 for n_regions 3 and 4
    threshold3: float = 0.0
    family: int = POLY         # POLY (the polynomial drift above) or ROTATOR
    K: float = 0.0             # plane rotator: coupling K and pinning g
    g: float = 0.0
    q2: float = 0.0            # second-moment coupling: the drift gets -q2 x E[X^2]

    def scaled(self, **kw) -> "Problem":
        return replace(copy.copy(self), **kw)


def linear(theta: float, kappa: float, sigma: float, **kw) -> Problem:
    """dX = (-theta X + kappa (E[X] - X)) dt + sigma dW (Lemma 2.1 form)."""
    return Problem(c3=0.0, c1=-(theta + kappa), kappa=kappa, c0=0.0, B0=sigma, **kw)


def cubic(kappa: float, sigma: float, **kw) -> Problem:
    """dX = (-X^3 + kappa (E[X] - X)) dt + sigma dW."""
    return Problem(c3=1.0, c1=-kappa, kappa=kappa, c0=0.0, B0=sigma, **kw)


def double_well(a: float, b: float, kappa: float, sigma: float, **kw) -> Problem:
    """dX = (-V'(X) + kappa (E[X] - X)) dt + sigma dW with V = a x^4 - b x^2."""
    return Problem(c3=4.0 * a, c1=2.0 * b - kappa, kappa=kappa, c0=0.0, B0=sigma, **kw)


def gbm(**kw) -> Problem:
    """The modified geometric Brownian motion of the paper's linear example
    (Sec. 5.1): dX = (alpha X + beta E[X] + a) dt + (sigma X + omega E[X] + b) dW
    with alpha = -1/2, beta = 4/5, a = 1/3, sigma = omega = sqrt(1/2)/2,
    b = 1/6, X0 ~ N(1, 1/4) and N = 10 slices.  T, dt and P are not given
    there; T = 1, dt = 1e-3, P = 1e5 here."""
    s = 0.5 * np.sqrt(0.5)
    p = Problem(c3=0.0, c1=-0.5, kappa=0.8, c0=1.0 / 3.0, B=s, BE=s, B0=1.0 / 6.0, m0=1.0, s0=0.5,
                T=1.0, N=10, dt=1e-3, P=100_000, coarse_h=0.25, seed=SEED_BASE + 6, tol=1e-8,
                precision="fp64")
    return p.scaled(**kw) if kw else p


def plane_rotator(K: float = 1.0, kT: float = 0.25, g: float = 1.0, **kw) -> Problem:
    """The unimodal plane rotator of Sec. 5: T = 10, dt = 1e-3 and
    X0 ~ N(pi/4, 3 pi/4) (read as mean and variance) as in the example, with
    the section's P = 1e5 particles and N = 10 slices; the coupling K and
    temperature k_B T are not given (K = 1, k_B T = 1/4 here, so
    B0 = sqrt(2 k_B T))."""
    p = Problem(family=ROTATOR, K=K, g=g, B0=float(np.sqrt(2.0 * kT)), m0=np.pi / 4,
                s0=float(np.sqrt(3.0 * np.pi / 4)), T=10.0, N=10, dt=1e-3, P=100_000, coarse_h=0.25,
                seed=SEED_BASE + 7, tol=1e-6, precision="fp64")
    return p.scaled(**kw) if kw else p


def polynomial_drift(alpha: float = -0.5, **kw) -> Problem:
    """The polynomial-drift example of App. C (after Son Doan et al.):
    dX = (alpha X + E[X] - X E[X^2]) dt + X dW, X(0) = 1, whose Taylor
    moment model is the exact moment system.  alpha is not given there
    (alpha = -1/2 here, as in the paper's linear example); T = 1, N = 10,
    dt = 1e-3 and P = 1e5 are chosen here."""
    p = Problem(c1=alpha, kappa=1.0, q2=1.0, B=1.0, m0=1.0, s0=0.0, T=1.0, N=10, dt=1e-3, P=100_000,
                coarse_h=0.25, coarse_model=TAYLOR, seed=SEED_BASE + 8, tol=1e-8, precision="fp64")
    return p.scaled(**kw) if kw else p


# --- the five measured workloads -----------------------------------------

def config1(**kw) -> Problem:
    """Linear MV SDE, theta=1, kappa=0.5, sigma=0.5, X0 ~ N(1, 0.1^2), T=4,
    N=16, dt=2e-3, P=2000, FP64, coarse step 0.25, tol 1e-8."""
    p = linear(1.0, 0.5, 0.5, m0=1.0, s0=0.1, T=4.0, N=16, dt=2e-3, P=2000, coarse_h=0.25,
               seed=SEED_BASE + 1, tol=1e-8, precision="fp64")
    return p.scaled(**kw) if kw else p


def config2(**kw) -> Problem:
    """Cubic unimodal, kappa=1, sigma=0.5, X0 ~ N(0.5, 0.2^2), T=8, N=64,
    dt=1e-3, P=1e6, Gaussian-closure coarse, tol 1e-6."""
    p = cubic(1.0, 0.5, m0=0.5, s0=0.2, T=8.0, N=64, dt=1e-3, P=1_000_000, coarse_h=0.25,
              seed=SEED_BASE + 2, tol=1e-6, precision="mixed")
    return p.scaled(**kw) if kw else p


def config3(**kw) -> Problem:
    """Double well a=1/4, b=1/2, kappa=0.1, sigma=0.7, X0 ~ N(0, 0.3^2),
    two regions split at 0, learning variant, T=20, N=128, dt=5e-4, P=4e6."""
    p = double_well(0.25, 0.5, 0.1, 0.7, m0=0.0, s0=0.3, T=20.0, N=128, dt=5e-4, P=4_000_000,
                    coarse_h=0.25, n_regions=2, threshold=0.0, variant=LEARNING,
                    seed=SEED_BASE + 3, tol=1e-6, precision="mixed")
    return p.scaled(**kw) if kw else p


def config4(**kw) -> Problem:
    """Adjoint workload: the double-well model at P=1e6, N=64, T=20, dt=1e-3."""
    p = double_well(0.25, 0.5, 0.1, 0.7, m0=0.0, s0=0.3, T=20.0, N=64, dt=1e-3, P=1_000_000,
                    coarse_h=0.25, n_regions=1, seed=SEED_BASE + 4, tol=1e-6, precision="mixed")
    return p.scaled(**kw) if kw else p


ADJOINT_TARGET_PARAMS = (0.15, 0.65, 0.25, 0.5)   # (kappa, sigma, a, b) of the target run
ADJOINT_EVAL_PARAMS = (0.1, 0.7, 0.25, 0.5)       # where the gradient is taken
ADJOINT_CKPT = 64


def config5(n_problems: int = 512, p_max: float = 2e6, **kw) -> list[Problem]:
    """Batch of seeded problems of the config-1 form (linear, unimodal) and
    the config-3 form (double well, two regions split at 0, learning
    variant): theta ~ U[0.5, 2], kappa ~ U[0, 1], sigma ~ U[0.3, 1],
    P log-uniform in [1e4, p_max], N uniform in 16..128, T=8, dt=1e-3."""
    rng = np.random.default_rng(SEED_BASE + 5)
    out = []
    for i in range(n_problems):
        theta = float(rng.uniform(0.5, 2.0))
        kappa = float(rng.uniform(0.0, 1.0))
        sigma = float(rng.uniform(0.3, 1.0))
        P = int(round(10 ** rng.uniform(4.0, np.log10(p_max))))
        N = int(rng.integers(16, 129))
        common = dict(T=8.0, N=N, dt=1e-3, P=P, coarse_h=0.25, seed=SEED_BASE + 5,
                      problem_tag=i, tol=1e-6, precision="mixed")
        if i % 2 == 0:
            p = linear(theta, kappa, sigma, m0=1.0, s0=0.1, **common)
        else:
            p = double_well(0.25, 0.5, kappa, sigma, m0=0.0, s0=0.3, n_regions=2, threshold=0.0,
                            variant=LEARNING, **common)
        out.append(p.scaled(**kw) if kw else p)
    return out
