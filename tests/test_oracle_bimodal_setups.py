"""The paper's five bimodal setups (Sec. 5.3, Table "Bimodal SDE: overview of
test setups", stored in tests/golden/bimodal_setups.txt) run through the
oracle's fine propagator, against what the text says of them at t = T:
setup 1 is bimodal; setup 3 is setup 2 with more diffusion; setup 4 is
weakly bimodal; in setup 5 the mean-field coupling makes the law unimodal.
The drift -(4 a X^3 - 2 gamma X - beta E[X]) is the polynomial family with
c3 = 4 a, c1 = 2 gamma, kappa = beta."""
import os

import numpy as np
import pytest

from paper_2310_11365_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "bimodal_setups.txt")


def _setups():
    rows = {}
    for line in open(GOLDEN):
        if line.strip() and not line.startswith("#"):
            name, a, gamma, beta, sigma, m0, sigma0, T = line.split()
            rows[int(name)] = dict(a=float(a), gamma=float(gamma), beta=float(beta), sigma=float(sigma),
                                   m0=float(m0), sigma0=float(sigma0), T=float(T))
    return rows


@pytest.fixture(scope="module")
def laws(orc):
    """Each setup's ensemble at t = T (P = 10^4, dt = 10^-2, one slice)."""
    out = {}
    for k, s in _setups().items():
        p = W.Problem(c3=4 * s["a"], c1=2 * s["gamma"], kappa=s["beta"], c0=0.0, B0=s["sigma"], m0=s["m0"],
                      s0=float(np.sqrt(s["sigma0"])), T=s["T"], N=1, dt=1e-2, P=10_000, seed=W.SEED_BASE + 20 + k)
        u = orc.fine(p, 0, orc.initial(p))
        hist, _ = np.histogram(u, bins=40, range=(-3.0, 3.0))
        c = len(hist) // 2
        out[k] = dict(left=float(np.mean(u < 0.0)), dip=float(hist[c - 1:c + 1].mean() / hist.max()),
                      var=float(u.var()))
    return out


def test_the_table_as_printed():
    s = _setups()
    assert sorted(s) == [1, 2, 3, 4, 5]
    assert all(r["a"] == 0.25 and r["gamma"] == 0.5 and r["m0"] == 1.0 for r in s.values())
    assert [s[k]["sigma"] for k in range(1, 6)] == [0.5, 0.5, 1.0, 2.0, 0.5]
    assert [s[k]["beta"] for k in range(1, 6)] == [0, 0, 0, 0, 1]
    assert [s[k]["T"] for k in range(1, 6)] == [20, 10, 10, 50, 10]


def test_setup_1_is_bimodal(laws):
    """Both wells hold a large share and the density dips deeply at the barrier."""
    assert 0.25 < laws[1]["left"] < 0.5
    assert laws[1]["dip"] < 0.3


def test_setup_3_has_more_diffusion_than_setup_2(laws):
    """The same start in the right well; more noise carries more particles over."""
    assert laws[3]["left"] > laws[2]["left"] + 0.1


def test_setup_4_is_weakly_bimodal(laws):
    """sigma = 2 at T = 50: the wells hold equal shares and the dip is shallow."""
    assert abs(laws[4]["left"] - 0.5) < 0.05
    assert 0.6 < laws[4]["dip"] < 1.0


def test_setup_5_mean_field_makes_it_unimodal(laws):
    """beta = 1: the mean field holds every particle in the right well,
    where setup 1 (the same but beta = 0) splits them."""
    assert laws[5]["left"] < 1e-3
    assert laws[5]["var"] < 0.1 < laws[1]["var"]
