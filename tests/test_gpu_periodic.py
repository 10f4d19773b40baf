"""GPU parity of the periodic disorder (the L x M samples of Sec. III.B of arXiv:1211.7275): node
index n keys the generator as n mod M.

  - both GPU paths against the oracle with the same period, per site (FP64 to 1e-12 over 10^3
    steps; FP32-split to 1e-4, over 10^3 steps for the continuous forces and 100 steps for Cases
    1 and 3, as for the aperiodic disorder);
  - the split path commutes with a shift by M bit for bit: the cells move by M and every offset,
    cache value and force is the same;
  - period 0 is the aperiodic disorder.
"""
import numpy as np
import pytest

from qew_workloads import SEED, random_state

pytestmark = pytest.mark.gpu

RF, RB, NONE, RBG_LINEAR, RBG_CUBIC = 0, 1, 2, 3, 4
FP32, FP64 = 0, 1
FMOVE = {RF: 1.2, RB: 2.2, RBG_LINEAR: 2.2, RBG_CUBIC: 2.6}


@pytest.fixture(scope="module")
def qew():
    import paper_1211_7275_gb300 as q
    q.load()
    return q


def _run(qew, L, f, kind, steps, precision, period, u0=None, batch=2):
    with qew.Relaxation(L, f, kind, dt=0.1, seed=SEED, precision=precision, batch=batch) as r:
        r.set_disorder_period(period)
        if u0 is not None:
            r.set_state(u0)
        obs = r.observe(steps)
        u, _ = r.state()
    return obs, u


@pytest.mark.parametrize("kind", [RF, RB, RBG_LINEAR, RBG_CUBIC])
@pytest.mark.parametrize("M", [1, 5, 37])
def test_fp64_per_site(qew, orc, kind, M):
    L, steps = 777, np.array([0, 1, 100, 1000])
    obs, u = _run(qew, L, FMOVE[kind], kind, steps, FP64, M)
    ref = orc.run([L] * 2, FMOVE[kind], 0.1, kind, SEED, steps, want_state=True, period=M)
    assert np.max(np.abs(u - ref["u"]) / np.maximum(1.0, np.abs(ref["u"]))) <= 1e-12
    np.testing.assert_allclose(obs["v"], ref["v"], rtol=0, atol=1e-11)


@pytest.mark.parametrize("kind,n", [(RF, 1000), (RB, 1000), (RBG_LINEAR, 100), (RBG_CUBIC, 100)])
@pytest.mark.parametrize("M", [3, 8])
def test_split_per_site(qew, orc, kind, n, M):
    L, steps = 1500, np.array([0, 7, n])
    _, u = _run(qew, L, FMOVE[kind], kind, steps, FP32, M)
    ref = orc.run([L] * 2, FMOVE[kind], 0.1, kind, SEED, steps, want_state=True, period=M)
    assert np.max(np.abs(u - ref["u"])) <= 1e-4


@pytest.mark.parametrize("kind,n", [(RF, 400), (RB, 400), (RBG_CUBIC, 100)])
def test_negative_cells_per_site(qew, orc, kind, n):
    """A line far below zero: the node index n mod M must land in [0, M) for negative n as well
    (the generator is keyed by the wrapped index).  Both GPU paths per site against the oracle
    (Case 1 over 100 steps, as above)."""
    L, M, steps = 1500, 7, np.array([0, 9, n])
    u0 = -1000.3 + random_state(2 * L, 0.5, seed=31)
    ref = orc.run([L] * 2, FMOVE[kind], 0.1, kind, SEED, steps, u0=u0, want_state=True, period=M)
    _, u = _run(qew, L, FMOVE[kind], kind, steps, FP32, M, u0=u0)
    assert np.max(np.abs(u - ref["u"])) <= 1e-4
    obs, u64 = _run(qew, L, FMOVE[kind], kind, steps, FP64, M, u0=u0)
    assert np.max(np.abs(u64 - ref["u"]) / np.maximum(1.0, np.abs(ref["u"]))) <= 1e-12
    np.testing.assert_allclose(obs["v"], ref["v"], rtol=0, atol=1e-11)


@pytest.mark.parametrize("kind", [RF, RB, RBG_LINEAR, RBG_CUBIC])
def test_split_commutes_with_a_shift_by_the_period(qew, kind):
    L, M, steps = 2000, 6, np.array([0, 50, 700])
    u0 = np.round(random_state(2 * L, 0.6, seed=kind) * 64) / 64 + 3.0   # exact in FP32-split
    _, a = _run(qew, L, FMOVE[kind], kind, steps, FP32, M, u0=u0)
    _, b = _run(qew, L, FMOVE[kind], kind, steps, FP32, M, u0=u0 + M)
    np.testing.assert_array_equal(b - M, a)


def test_period_zero_is_aperiodic(qew):
    L, steps = 1024, np.array([0, 300])
    with qew.Relaxation(L, 1.0, RF, dt=0.1, seed=SEED, batch=2) as r:
        r.set_disorder_period(5)
        r.observe(steps)
        r.set_disorder_period(0)
        r.observe(steps)
        u, _ = r.state()
    with qew.Relaxation(L, 1.0, RF, dt=0.1, seed=SEED, batch=2) as r:
        r.observe(steps)
        u0, _ = r.state()
    np.testing.assert_array_equal(u, u0)


def test_bad_period(qew):
    with qew.Relaxation(100, 1.0, RF) as r:
        for bad in (-1, 1 << 31):
            with pytest.raises(qew.QewError) as e:
                r.set_disorder_period(bad)
            assert e.value.code == -1


def test_critical_force_matches_oracle(qew, orc):
    """f_c^s of periodic 64 x 64 random-field samples (Sec. III.B), bisected on the GPU's FP64 path
    and on the oracle: the two dynamics agree to rounding, so every trial takes the same decision
    and the brackets are equal."""
    from paper_1211_7275_gb300 import critical
    res = critical.critical_forces(64, 64, RF, 4, seed=SEED, tol=1e-4)
    for s in range(4):
        ref = orc.critical_force(64, 64, RF, SEED, s, tol=1e-4)
        assert res["lo"][s] == ref["bracket"][0] and res["hi"][s] == ref["bracket"][1], (s, res["f_c"][s], ref["f_c"])
        assert np.max(np.abs(res["u_c"][s] - ref["u_c"])) <= 1e-9


def test_critical_force_single_site_closed_form(qew, orc):
    from paper_1211_7275_gb300 import critical
    M = 16
    res = critical.critical_forces(1, M, RF, 6, seed=SEED, tol=1e-5)
    for s in range(6):
        R = orc.disorder_values(RF, SEED, s, np.zeros(M, np.int64), np.arange(M))
        assert res["lo"][s] <= -R.min() <= res["hi"][s]


def test_critical_force_mean_near_the_short_time_threshold(qew):
    """Sec. IV.A: the thermodynamic f_c of the critical configurations is the threshold of the
    short-time dynamics.  8 random-field samples of 512 x 512: the mean f_c^s within 5% of the
    GPU-bisected STD threshold of the 16 x 2^20 preset."""
    from paper_1211_7275_gb300 import critical
    from qew_workloads import preset_f
    res = critical.critical_forces(512, 512, RF, 8, seed=SEED, tol=1e-3)
    fc_std = preset_f("rf_16x2^20")
    print(f"mean f_c^s (512 x 512, 8 samples) = {np.mean(res['f_c']):.4f}, STD f_c^L = {fc_std:.4f}")
    assert abs(np.mean(res["f_c"]) - fc_std) < 0.05 * fc_std


def test_exact_critical_force_on_the_device_disorder(qew, orc):
    """The exact branch-following search (qew_critical_force_rf) on the device generator's FP64
    force values: for 64 x 64 random-field samples its f_c^s lies inside the GPU bisection's bracket
    (tol 1e-5), and its critical configuration is the bisection's pinned configuration at the
    bracket's lower end to within the distance that configuration can still move below f_c^s."""
    from paper_1211_7275_gb300 import critical
    res = critical.critical_forces(64, 64, RF, 4, seed=SEED, tol=1e-5)
    for s in range(4):
        ex = critical.exact_critical_force(64, 64, s, seed=SEED)
        assert res["lo"][s] - 1e-9 <= ex["f_c"] <= res["hi"][s] + 1e-9, (s, ex["f_c"], res["lo"][s], res["hi"][s])
        assert np.max(np.abs(ex["u_c"] - res["u_c"][s])) < 0.05


def test_exact_critical_forces_of_512_samples_match_the_short_time_threshold(qew):
    """Sec. IV.A with the exact search: the mean f_c^s of 16 random-field samples of 512 x 512 lies
    within 5% of the STD threshold of the 16 x 2^20 preset (finite L and M move it)."""
    from paper_1211_7275_gb300 import critical
    from qew_workloads import preset_f
    fcs = critical.exact_critical_forces(512, 512, 16, seed=SEED)["f_c"]
    print(f"exact mean f_c^s (512 x 512, 16 samples) = {np.mean(fcs):.5f} +- {np.std(fcs, ddof=1) / 4:.5f}")
    assert abs(np.mean(fcs) - preset_f("rf_16x2^20")) < 0.05 * preset_f("rf_16x2^20")
