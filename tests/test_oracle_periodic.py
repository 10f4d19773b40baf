"""Pins of the oracle's periodic disorder: the L x M system of Sec. III.B of arXiv:1211.7275, where
the random values at the integer points repeat in u with period M (node index n taken mod M).

  - the values repeat with period M, also for negative n, and agree with the aperiodic values on
    the fundamental domain 0 <= n < M;
  - the dynamics commutes with a shift by M: the relaxation of u0 + M is the relaxation of u0
    shifted by M (true for periodic disorder only; the aperiodic control differs);
  - a relaxation whose cells stay inside [0, M) is the aperiodic relaxation, bit for bit.
"""
import numpy as np
import pytest

from qew_workloads import SEED, random_points, random_state

KINDS = [0, 1, 3, 4]   # RF, uniform RB cubic, Gaussian RB linear (Case 3), Gaussian RB cubic (Case 1)
FMOVE = {0: 1.2, 1: 2.2, 3: 2.2, 4: 2.6}


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("M", [1, 5, 64])
def test_values_repeat_with_period(orc, kind, M):
    i, n = random_points(5000, 1 << 20, -300, 300, seed=M)
    base = orc.disorder_values(kind, SEED, 3, i, n, period=M)
    for k in (-3, -1, 1, 2):
        np.testing.assert_array_equal(orc.disorder_values(kind, SEED, 3, i, n + k * M, period=M), base)
    inside = (n >= 0) & (n < M)
    np.testing.assert_array_equal(base[inside], orc.disorder_values(kind, SEED, 3, i[inside], n[inside]))
    np.testing.assert_array_equal(base, orc.disorder_values(kind, SEED, 3, i, np.mod(n, M)))


@pytest.mark.parametrize("kind", KINDS)
def test_dynamics_commutes_with_a_shift_by_the_period(orc, kind):
    L, M, steps = 97, 6, [0, 1, 40, 300]
    u0 = random_state(L, 0.8, seed=kind) + 2.3
    a = orc.run(L, FMOVE[kind], 0.1, kind, SEED, steps, u0=u0, want_state=True, period=M)
    b = orc.run(L, FMOVE[kind], 0.1, kind, SEED, steps, u0=u0 + M, want_state=True, period=M)
    np.testing.assert_allclose(b["u"] - M, a["u"], rtol=0, atol=1e-11)
    np.testing.assert_allclose(b["v"], a["v"], rtol=0, atol=1e-11)
    np.testing.assert_allclose(b["w2"], a["w2"], rtol=1e-10, atol=1e-12)
    c = orc.run(L, FMOVE[kind], 0.1, kind, SEED, steps, u0=u0 + M, want_state=True)
    assert np.max(np.abs(c["u"] - M - a["u"])) > 1e-3   # the aperiodic disorder differs


@pytest.mark.parametrize("kind", KINDS)
def test_fundamental_domain_is_the_aperiodic_system(orc, kind):
    L, M, steps = 64, 1000, [0, 10, 150]
    a = orc.run(L, FMOVE[kind], 0.1, kind, SEED, steps, u0=np.full(L, 500.0), want_state=True, period=M)
    b = orc.run(L, FMOVE[kind], 0.1, kind, SEED, steps, u0=np.full(L, 500.0), want_state=True)
    assert np.all((a["u"] > 0) & (a["u"] < M - 3))
    np.testing.assert_array_equal(a["u"], b["u"])
    np.testing.assert_array_equal(a["v"], b["v"])
