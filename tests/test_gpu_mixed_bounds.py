"""Errors of the mixed form (FP32 particles and draws, FP64 moments) against
the FP64 oracle on the same draws, per result, for the config-1, -2 and -3
forms at test size, after a fixed number of sweeps:

  mean      max over slice ends of |dM| / max(|M|, sqrt(V))
  variance  max over slice ends of |dV| / V
  fraction  max over slice ends and regions of |dP| (two regions only)

Each measured error is printed (MIXED_ERROR lines) and must stay within its
bound, about twice the error measured on a GB300 (see the bounds below).
The bounds are three to four orders of magnitude below the Monte Carlo
error sqrt(V / P) of the moments (2e-3 to 6e-3 here), so the precision
split does not show at the method's accuracy."""
import json

import numpy as np
import pytest

from paper_2310_11365_gb300 import workloads as W

pytestmark = pytest.mark.gpu

CASES = {
    "config1": lambda: W.config1(precision="mixed", max_iter=4, tol=0.0),
    "config2": lambda: W.config2(P=20_000, N=8, T=1.0, precision="mixed", max_iter=3, tol=0.0),
    "config3": lambda: W.config3(P=20_001, N=8, T=4.0, dt=5e-3, precision="mixed", max_iter=4, tol=0.0),
}
# Bound on (mean, variance, fraction) per case: about twice the error
# measured on a GB300 (config 1: 5.4e-7, 1.46e-6; config 2: 5.3e-7,
# 1.15e-6; config 3: 2.8e-7, 1.5e-7; fractions equal in all three), the
# fraction bound two particles of P = 20001 (a particle within rounding of
# the region boundary may land on either side).
BOUNDS = {
    "config1": (1.2e-6, 3e-6, 0.0),
    "config2": (1.2e-6, 3e-6, 0.0),
    "config3": (6e-7, 4e-7, 1e-4),
}


def _errors(mom, ref, I):
    em = ev = ef = 0.0
    for n in range(mom.shape[0]):
        M, V = ref["hist"][-1][n]
        em = max(em, abs(mom[n, 6] - M) / max(abs(M), np.sqrt(V)))
        ev = max(ev, abs(mom[n, 7] - V) / V)
        if I > 1:
            for i in range(I):
                ef = max(ef, abs(mom[n, 3 * i] - ref["frac"][n][i]))
    return em, ev, ef


@pytest.mark.parametrize("name", sorted(CASES))
def test_mixed_errors_within_bounds(mmplib, orc, name):
    from paper_2310_11365_gb300.mmp import Solver

    p = CASES[name]()
    s = Solver(p)
    k = s.run()
    mom = s.moments()
    s.close()
    ref = orc.parareal(p.scaled(precision="fp64"))
    assert k == ref["sweeps"]
    em, ev, ef = _errors(mom, ref, p.n_regions)
    mc = float(np.sqrt(ref["hist"][-1][-1][1] / p.P))
    print("MIXED_ERROR " + json.dumps({"case": name, "mean": em, "var": ev, "frac": ef,
                                        "mc_sd_of_mean": mc, "P": p.P, "sweeps": k}))
    bm, bv, bf = BOUNDS[name]
    assert em <= bm and ev <= bv and ef <= bf, (name, em, ev, ef)
