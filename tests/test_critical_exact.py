"""The library's exact critical force of a periodic random-field sample (qew_critical_force_rf,
host code: runs without a GPU), against what fixes it.

Sec. III.B of arXiv:1211.7275: f_c^s is the largest drive at which the L x M sample (periodic in u
with period M) has a pinned configuration, and the critical configuration is that configuration.
The force values R(i, n mod M) are the oracle's (FP64), passed in as the sample.

  - L = 1 has no elasticity, and f_c^s = -min_n R(n) exactly (the minimum of a piecewise-linear
    force is at a node);
  - f_c^s lies in the oracle's bisection bracket (oracle.critical_force, the definition evaluated
    by relaxations, to 1e-6), for several sizes, periods and samples;
  - the critical configuration is static (every velocity vanishes at f_c^s) and stable (the line
    relaxed from it slightly below, at f_c^s - 1e-4, returns to it);
  - by no-passing the result does not depend on the pinned configuration the search starts from.
"""
import ctypes

import numpy as np
import pytest

from qew_workloads import SEED


def table(orc, L, M, s):
    i = np.repeat(np.arange(L), M)
    n = np.tile(np.arange(M), L)
    return orc.disorder_values(orc.KIND_RF, SEED, s, i, n).reshape(L, M)


@pytest.fixture(scope="module")
def crit():
    from paper_1211_7275_gb300 import critical
    return critical


@pytest.mark.parametrize("M,s", [(16, 0), (5, 2), (64, 3), (2, 1)])
def test_single_site_closed_form(orc, crit, M, s):
    R = table(orc, 1, M, s)
    # a single site pins for -max R <= f <= -min R; start inside that window (f_c^s < 0 when every
    # R(n) > 0, and a drive below -max R slides the site backwards for ever)
    r = crit.exact_critical_force(1, M, s, R=R, f_start=-0.5 * (R.max() + R.min()))
    assert abs(r["f_c"] - (-R.min())) <= 1e-12 * max(1.0, abs(R.min()))


@pytest.mark.parametrize("L,M,s", [(2, 16, 1), (3, 8, 0), (16, 16, 0), (48, 32, 0), (64, 64, 1), (100, 37, 4),
                                   (200, 300, 5)])
def test_inside_the_oracle_bracket(orc, crit, L, M, s):
    r = crit.exact_critical_force(L, M, s, R=table(orc, L, M, s))
    ref = orc.critical_force(L, M, orc.KIND_RF, SEED, s, tol=1e-6)
    lo, hi = ref["bracket"]
    assert lo - 1e-9 <= r["f_c"] <= hi + 1e-9, (r["f_c"], lo, hi)


def test_critical_configuration_is_static_and_stable(orc, crit):
    L, M, s = 48, 32, 0
    r = crit.exact_critical_force(L, M, s, R=table(orc, L, M, s))
    u, fc = r["u_c"], r["f_c"]
    F = orc.pinning_force(orc.KIND_RF, SEED, s, np.arange(L), u, period=M)
    vel = (np.roll(u, -1) + np.roll(u, 1) - 2 * u) + fc + F
    assert np.max(np.abs(vel)) < 1e-9
    # slightly below f_c the line started at u_c stays pinned next to it
    out = orc.run(L, fc - 1e-4, 0.1, orc.KIND_RF, SEED, [20000], s=[s], u0=u, want_state=True, period=M)
    assert abs(out["v"][0, 0]) < 1e-9 and np.max(np.abs(out["u"] - u)) < 0.05


def test_independent_of_the_start(orc, crit):
    R = table(orc, 64, 64, 1)
    a = crit.exact_critical_force(64, 64, 1, R=R)
    b = crit.exact_critical_force(64, 64, 1, R=R, f_start=0.3)
    assert abs(a["f_c"] - b["f_c"]) <= 1e-9


def test_argument_errors():
    import paper_1211_7275_gb300 as q
    lib = q.load()
    R = np.zeros(16)
    f = ctypes.c_double()
    P = R.ctypes.data_as(ctypes.c_void_p)
    assert lib.qew_critical_force_rf(0, 16, P, 0.1, 0.0, ctypes.byref(f), None, None, None) == -1
    assert lib.qew_critical_force_rf(1, 1, P, 0.1, 0.0, ctypes.byref(f), None, None, None) == -1
    assert lib.qew_critical_force_rf(1, 16, None, 0.1, 0.0, ctypes.byref(f), None, None, None) == -1
    assert lib.qew_critical_force_rf(1, 16, P, 0.6, 0.0, ctypes.byref(f), None, None, None) == -1
    # a drive at which the flat line cannot pin (R = 0 everywhere and f > 0)
    assert lib.qew_critical_force_rf(1, 16, P, 0.1, 0.5, ctypes.byref(f), None, None, None) == -6
