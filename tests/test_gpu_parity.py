"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle on the same seeded inputs.

Bars (Sec. II-III of arXiv:1211.7275 define what is computed):
  - RNG words and integer cell indices: bit-exact (cells compared where the oracle's u is more
    than 1e-4 from an integer, where FP32 rounding cannot move the floor);
  - FP64 path: per site |du| <= 1e-12 max(1, |u|) over 10^3 steps;
  - FP32-split path: per site |du| <= 1e-4 over the first 10^3 steps;
  - ensemble v(t), w2(t): within 2 sigma of the oracle's sample error bars to t_max.
Sizes span several warp tiles and a ragged tail; degenerate lengths (L = 1, 2, 3, ...) make a
tile window wrap around the chain many times.
"""
import numpy as np
import pytest

from qew_workloads import SEED, cosine_profile, log_spaced_steps, positive_shift, random_points, random_state

pytestmark = pytest.mark.gpu

RF, RB, NONE, RBG_LINEAR, RBG_CUBIC = 0, 1, 2, 3, 4
FP32, FP64 = 0, 1


@pytest.fixture(scope="module")
def qew():
    import paper_1211_7275_gb300 as q
    q.load()
    return q


def gpu_run(qew, L, f, kind, steps, precision, *, tuning=None, u0=None, dt=0.1, seed=SEED):
    with qew.Relaxation(L, f, kind, dt=dt, seed=seed, precision=precision) as r:
        if tuning is not None:
            r.set_tuning(*tuning)
        if u0 is not None:
            r.set_state(u0)
        obs = r.observe(steps)
        u, step = r.state()
        cells = r.cells()
    assert step == steps[-1]
    return obs, u, cells


# ------------------------------------------------------------------------------------------
# generator
# ------------------------------------------------------------------------------------------
def test_philox_words_bitexact(qew, orc):
    rng = np.random.default_rng(5)
    ctr = rng.integers(0, 2 ** 32, size=(1 << 20, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2 ** 32, size=(1 << 20, 2), dtype=np.uint64).astype(np.uint32)
    assert np.array_equal(qew.philox_words(ctr, key), orc.philox4x32_10(ctr, key))


@pytest.mark.parametrize("kind", [RF, RB])
def test_disorder_values(qew, orc, kind):
    i, n = random_points(200_000, 1 << 25, -3000, 3000, seed=9)
    ref = orc.disorder_values(kind, SEED, 3, i, n)
    g64 = qew.disorder_values(kind, FP64, SEED, 3, i, n)
    g32 = qew.disorder_values(kind, FP32, SEED, 3, i, n)
    if kind == RB:
        assert np.array_equal(g64, ref)   # exact arithmetic on both sides
    else:
        assert np.max(np.abs(g64 - ref) / np.maximum(1.0, np.abs(ref))) < 4e-15
    assert np.max(np.abs(g32 - ref) / np.maximum(1.0, np.abs(ref))) < 6e-7


# ------------------------------------------------------------------------------------------
# FP64 path
# ------------------------------------------------------------------------------------------
@pytest.mark.parametrize("kind,L,f", [(RF, 1024, 1.0), (RB, 777, 1.9), (RF, 3, 0.8), (RB, 5, 2.0), (NONE, 64, 0.3)])
def test_fp64_per_site(qew, orc, kind, L, f):
    steps = np.array([0, 1, 2, 10, 100, 1000])
    obs, u, cells = gpu_run(qew, L, f, kind, steps, FP64)
    ref = orc.run(L, f, 0.1, kind, SEED, steps, want_state=True)
    err = np.abs(u - ref["u"]) / np.maximum(1.0, np.abs(ref["u"]))
    assert err.max() <= 1e-12, err.max()
    assert np.array_equal(cells, np.floor(ref["u"]).astype(np.int32))
    np.testing.assert_allclose(obs["v"], ref["v"], rtol=0, atol=1e-11)
    np.testing.assert_allclose(obs["ubar"], ref["ubar"], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(obs["w2"], ref["w2"], rtol=1e-9, atol=1e-12)


def test_fp64_closed_form(qew):
    L, k, A, B, f, dt = 128, 3, 0.7, 3.2, 0.37, 0.1
    u0 = cosine_profile(L, A, B, k)
    lam = 1.0 - 4.0 * dt * np.sin(np.pi * k / L) ** 2
    n = 300
    obs, u, _ = gpu_run(qew, L, f, NONE, [0, n], FP64, u0=u0)
    exact = B + f * n * dt + A * lam ** n * np.cos(2 * np.pi * k * np.arange(L) / L)
    assert np.max(np.abs(u - exact)) < 1e-12 * np.abs(exact).max()
    assert abs(obs["v"][1, 0] - f) < 1e-14
    assert abs(obs["w2"][1, 0] - A * A * lam ** (2 * n) / 2) < 1e-12


# ------------------------------------------------------------------------------------------
# FP32-split fused path
# ------------------------------------------------------------------------------------------
SHAPES = [(480, 16, 4), (224, 8, 2), (992, 32, 1), (736, 24, 8), (480, 13, 2), (1248, 32, 1), (1248, 9, 2)]


def _split_check(u, cells, ref_u, tol=1e-4):
    err = np.abs(u - ref_u)
    assert err.max() <= tol, err.max()
    far = np.abs(ref_u - np.round(ref_u)) > 1e-4
    assert np.array_equal(cells[far], np.floor(ref_u[far]).astype(np.int32))
    return err.max()


@pytest.mark.parametrize("L", [1, 2, 3, 5, 31, 33, 1024, 5000])
def test_split_rf_per_site(qew, orc, L):
    steps = np.array([0, 1, 7, 100, 1000])
    ref = orc.run(L, 1.0, 0.1, RF, SEED, steps, want_state=True)
    obs, u, cells = gpu_run(qew, L, 1.0, RF, steps, FP32)
    _split_check(u, cells, ref["u"])
    np.testing.assert_allclose(obs["ubar"], ref["ubar"], rtol=0, atol=2e-5)
    np.testing.assert_allclose(obs["v"], ref["v"], rtol=0, atol=2e-4)


@pytest.mark.parametrize("L", [3, 256, 4099])
def test_split_rb_per_site(qew, orc, L):
    steps = np.array([0, 3, 50, 1000])
    ref = orc.run(L, 1.9, 0.1, RB, SEED, steps, want_state=True)
    obs, u, cells = gpu_run(qew, L, 1.9, RB, steps, FP32)
    _split_check(u, cells, ref["u"])
    np.testing.assert_allclose(obs["v"], ref["v"], rtol=0, atol=2e-4)


@pytest.mark.parametrize("base", [2.0 ** 29 + 0.25, -(2.0 ** 29) - 0.75, -3.5])
@pytest.mark.parametrize("kind,f", [(RF, 1.0), (RB, 1.9)])
def test_far_from_zero_per_site(qew, orc, base, kind, f):
    """A rough line around u = +-2^29 or just below zero.  The disorder counter takes the cell as a
    two's-complement 32-bit word (negative cells included), the cells stay exact int32, the state
    read back is n + d, and the observables are summed relative to a chain reference at the
    line's rounded mean (so w2 of a line at 5e8 keeps its digits).  Per site against the oracle,
    FP32-split to 1e-4 and FP64 to 1e-6 absolute (1e-15 relative)."""
    L, steps = 3000, np.array([0, 10, 400])
    u0 = base + random_state(L, 0.5, seed=21)
    ref = orc.run(L, f, 0.1, kind, SEED, steps, u0=u0, want_state=True)
    obs, u, cells = gpu_run(qew, L, f, kind, steps, FP32, u0=u0)
    _split_check(u, cells, ref["u"])
    np.testing.assert_allclose(obs["ubar"], ref["ubar"], rtol=0, atol=2e-5)
    np.testing.assert_allclose(obs["v"], ref["v"], rtol=0, atol=2e-4)
    np.testing.assert_allclose(obs["w2"], ref["w2"], rtol=1e-4, atol=1e-6)
    obs64, u64, cells64 = gpu_run(qew, L, f, kind, steps, FP64, u0=u0)
    assert np.abs(u64 - ref["u"]).max() <= 1e-6
    assert np.array_equal(cells64, np.floor(u64).astype(np.int64).astype(np.int32))
    for k in ("v", "ubar", "w2"):
        np.testing.assert_allclose(obs64[k], ref[k], rtol=1e-9, atol=1e-9)


@pytest.mark.parametrize("kind,f", [(RF, 1.0), (RB, 1.9)])
def test_seed_with_a_high_word(qew, orc, kind, f):
    """A 64-bit seed whose high word is not zero: both Philox key words (the low and the high 32
    bits of the seed, reading A1) reach the fused kernel's precomputed key schedule and the FP64
    kernel.  Per site against the oracle."""
    seed, L, steps = 0xDEADBEEF12345678, 2048, np.array([0, 25, 600])
    ref = orc.run(L, f, 0.1, kind, seed, steps, want_state=True)
    obs, u, cells = gpu_run(qew, L, f, kind, steps, FP32, seed=seed)
    _split_check(u, cells, ref["u"])
    np.testing.assert_allclose(obs["v"], ref["v"], rtol=0, atol=2e-4)
    _, u64, _ = gpu_run(qew, L, f, kind, steps, FP64, seed=seed)
    assert np.max(np.abs(u64 - ref["u"]) / np.maximum(1.0, np.abs(ref["u"]))) <= 1e-12
    other = orc.run(L, f, 0.1, kind, seed & 0xFFFFFFFF, steps, want_state=True)
    assert np.abs(other["u"] - ref["u"]).max() > 1e-2   # the high word changes the disorder


@pytest.mark.parametrize("kind,f,dt", [(RF, 1.0, 0.01), (RF, 1.0, 0.25), (RB, 1.9, 0.01), (RB, 1.9, 0.2)])
def test_other_time_steps(qew, orc, kind, f, dt):
    """Euler steps other than the paper's dt = 0.1 (Sec. III.B), per site against the oracle in
    both precisions.  The larger steps are the largest at which the explicit Euler map still
    forgets a rounding-level difference: the map is monotone only while 1 - 2 dt + dt dF_p/du >= 0,
    and beyond that it is chaotic.  Measured on the oracle alone (2048 sites, 500 steps), a uniform
    1e-12 shift of the start ends at 1e-11 for the random field at dt = 0.25 but at 2e-7 at
    dt = 0.3 and 1.0 at dt = 0.37; for the random bond (steeper spline forces) at 1e-11 at
    dt = 0.2 and 1.5 at dt = 0.3.  There no two implementations agree per site."""
    L, steps = 2048, np.array([0, 30, 500])
    ref = orc.run(L, f, dt, kind, SEED, steps, want_state=True)
    obs, u, cells = gpu_run(qew, L, f, kind, steps, FP32, dt=dt)
    _split_check(u, cells, ref["u"])
    np.testing.assert_allclose(obs["v"], ref["v"], rtol=0, atol=2e-4)
    obs64, u64, _ = gpu_run(qew, L, f, kind, steps, FP64, dt=dt)
    assert np.max(np.abs(u64 - ref["u"]) / np.maximum(1.0, np.abs(ref["u"]))) <= 1e-12
    np.testing.assert_allclose(obs64["v"], ref["v"], rtol=0, atol=1e-11)


@pytest.mark.parametrize("shape", SHAPES)
def test_split_shapes_identical(qew, orc, shape):
    """Every launch shape performs the same per-site arithmetic: states agree bit for bit."""
    L, steps = 20000, np.array([0, 5, 333, 1000])
    _, u_ref, _ = gpu_run(qew, L, 1.0, RF, steps, FP32, tuning=SHAPES[0])
    obs, u, cells = gpu_run(qew, L, 1.0, RF, steps, FP32, tuning=shape)
    assert np.array_equal(u, u_ref)
    ref = orc.run(L, 1.0, 0.1, RF, SEED, steps, want_state=True)
    _split_check(u, cells, ref["u"])


def test_split_uneven_mixed_batch(qew, orc):
    # drives in the moving regime; the near-critical precision has its own test below
    L = np.array([1, 300, 4097, 1025, 77, 2048])
    kind = np.array([RF, RB, RF, RB, NONE, RF], dtype=np.int32)
    f = np.array([1.0, 1.9, 1.3, 2.0, 0.5, 1.1])
    steps = np.array([0, 10, 500])
    ref = orc.run(L, f, 0.1, kind, SEED, steps, want_state=True)
    for prec in (FP32, FP64):
        with qew.Relaxation(L, f, kind, dt=0.1, seed=SEED, precision=prec) as r:
            obs = r.observe(steps)
            u, _ = r.state()
        if prec == FP64:
            assert np.max(np.abs(u - ref["u"]) / np.maximum(1, np.abs(ref["u"]))) <= 1e-12
        else:
            assert np.max(np.abs(u - ref["u"])) <= 1e-4
        np.testing.assert_allclose(obs["v"], ref["v"], atol=2e-4)
        np.testing.assert_allclose(obs["w2"], ref["w2"], rtol=1e-4, atol=1e-6)


def test_split_near_critical_precision(qew, orc):
    """Random field at f = f_c^L (L = 4096, the oracle-bisected fixture), 16 chains, per site
    against the FP64 oracle.  Near the depinning threshold the dynamics amplifies any change of
    the force: the FP32 node model (the oracle's exact dynamics with each disorder value rounded
    to FP32, the floor of any FP32 store of the disorder) itself moves 28 of these 65536 sites by
    more than 1e-4 by step 1000 (max 5.0e-4), while through step 200 it stays below 2e-5.  So the
    per-site bar of 1e-4 is asked where the arithmetic can meet it:
      - through step 200, at every site;
      - at step 1000, at every site that the FP32 node model leaves within 1e-5 of the exact run
        (sites insensitive to the rounding at this horizon, 99.2% of them);
    and over all sites at step 1000 the distribution is bounded: rms <= 2e-5, at most 0.1% of
    sites above 1e-4, max <= 1e-3."""
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "fc_rf_L4096.json")) as fh:
        fc = json.load(fh)
    L, f, B = fc["L"], fc["f_c"], 16
    with qew.Relaxation(L, f, RF, dt=0.1, seed=SEED, precision=FP32, batch=B) as r:
        r.observe([200])
        u200, _ = r.state()
        r.observe([1000])
        u1000, _ = r.state()
    for n, u in ((200, u200), (1000, u1000)):
        ref = orc.run([L] * B, f, 0.1, RF, SEED, [n], want_state=True)["u"]
        floor = orc.run([L] * B, f, 0.1, RF, SEED, [n], want_state=True, node_f32=True)["u"]
        err, ef = np.abs(u - ref), np.abs(floor - ref)
        rms, frac, mx = float(np.sqrt(np.mean(err ** 2))), float(np.mean(err > 1e-4)), float(err.max())
        calm = ef <= 1e-5
        print(f"step {n}: FP32-split vs oracle rms {rms:.2e}, >1e-4: {frac:.1e}, max {mx:.2e}; FP32 node model "
              f"rms {np.sqrt(np.mean(ef ** 2)):.2e}, >1e-4: {np.mean(ef > 1e-4):.1e}, max {ef.max():.2e}; "
              f"max on the {calm.mean():.4f} insensitive sites {err[calm].max():.2e}")
        if n == 200:
            assert mx <= 1e-4, mx
        else:
            assert calm.mean() >= 0.98
            assert err[calm].max() <= 1e-4, err[calm].max()
            assert rms <= 2e-5 and frac <= 1e-3 and mx <= 1e-3, (rms, frac, mx)


def test_split_closed_form(qew):
    L, k, A, B, f, dt = 4096, 5, 0.7, 3.2, 0.37, 0.1
    u0 = cosine_profile(L, A, B, k)
    lam = 1.0 - 4.0 * dt * np.sin(np.pi * k / L) ** 2
    n = 1000
    obs, u, _ = gpu_run(qew, L, f, NONE, [0, n], FP32, u0=u0)
    exact = B + f * n * dt + A * lam ** n * np.cos(2 * np.pi * k * np.arange(L) / L)
    assert np.max(np.abs(u - exact)) < 1e-4
    assert abs(obs["ubar"][1, 0] - (B + f * n * dt)) < 1e-5


def test_split_no_passing(qew):
    L = 3000
    u0 = random_state(L, 0.5, seed=11)
    u1 = u0 + positive_shift(L, 0.3, seed=12)
    _, a, _ = gpu_run(qew, L, 1.0, RF, [0, 2000], FP32, u0=u0)
    _, b, _ = gpu_run(qew, L, 1.0, RF, [0, 2000], FP32, u0=u1)
    assert np.all(b >= a)


@pytest.mark.parametrize("precision", [FP32, FP64])
def test_mean_velocity_invariant(qew, precision):
    steps = np.array([0, 1, 2, 3, 50, 51, 400, 401])
    obs, _, _ = gpu_run(qew, 10007, 0.9, RF, steps, precision)
    ub, v = obs["ubar"][:, 0], obs["v"][:, 0]
    tol = 1e-12 if precision == FP64 else 2e-6
    for j in range(len(steps) - 1):
        if steps[j + 1] == steps[j] + 1:
            assert abs((ub[j + 1] - ub[j]) - 0.1 * v[j]) <= tol * max(1.0, abs(ub[j])), j


def test_resume_is_exact(qew):
    """state(2N) == set_state(state(N)) + N more steps: the disorder is a pure function of (i, n)."""
    L, N = 5000, 400
    for prec in (FP32, FP64):
        _, u_full, _ = gpu_run(qew, L, 1.0, RF, [2 * N], prec)
        _, u_half, _ = gpu_run(qew, L, 1.0, RF, [N], prec)
        _, u_res, _ = gpu_run(qew, L, 1.0, RF, [N], prec, u0=u_half)
        assert np.array_equal(u_full, u_res)


def test_deterministic_observables(qew):
    steps = log_spaced_steps(2000, 12)
    a, _, _ = gpu_run(qew, 70000, 1.0, RF, steps, FP32)
    b, _, _ = gpu_run(qew, 70000, 1.0, RF, steps, FP32)
    for k in ("v", "ubar", "w2"):
        assert np.array_equal(a[k], b[k])


def test_ensemble_within_two_sigma(qew, orc):
    """32 samples, L = 1024, 10^4 steps (the tiny preset's length and horizon): ensemble V(t),
    W2(t) of the fast path within 2 sigma of the oracle's, and the paired differences far
    smaller than sigma."""
    n_s, L = 32, 1024
    steps = log_spaced_steps(10_000, 40)
    ref = orc.run([L] * n_s, 1.0, 0.1, RF, SEED, steps)
    with qew.Relaxation(L, 1.0, RF, dt=0.1, seed=SEED, precision=FP32, batch=n_s) as r:
        obs = r.observe(steps)
    for key in ("v", "w2"):
        m_ref, m_gpu = ref[key].mean(1), obs[key].mean(1)
        sig = ref[key].std(1, ddof=1) / np.sqrt(n_s)
        sig[0] = max(sig[0], 1e-12)
        ok = np.abs(m_gpu - m_ref) <= 2 * sig + 1e-12
        assert ok.all(), (key, np.where(~ok))
        paired = np.abs(obs[key] - ref[key]).mean(1)
        assert np.all(paired[1:] <= 0.5 * np.maximum(ref[key].std(1, ddof=1)[1:], 1e-9)), key


# ------------------------------------------------------------------------------------------
# the benchmark's own launch configuration at full size: 4 chains of 2^25 sites
# ------------------------------------------------------------------------------------------
def test_full_size_sampled_sites(qew, orc):
    """Config of the bench: 4 x 2^25 sites.  After 1000 steps, sampled sites (tile edges, the
    periodic seam, random sites) against the oracle's light-cone evaluation of the same site;
    the invariant dubar = dt v at every chain."""
    from qew_workloads import preset_f
    L, batch, n = 1 << 25, 4, 1000
    f = preset_f("rf_4x2^25")
    steps = np.array([0, n - 1, n])
    with qew.Relaxation(L, f, RF, dt=0.1, seed=SEED, precision=FP32, batch=batch) as r:
        obs = r.observe(steps)
        u, _ = r.state()
        tile_w, K, _ = r.tuning()
    w_own = tile_w - 2 * K
    rng = np.random.default_rng(3)
    picks = []
    for c in range(batch):
        for i in [0, 1, L - 1, L - 2, w_own - 1, w_own, 5 * w_own + 1] + list(rng.integers(0, L, 3)):
            picks.append((c, int(i)))
    for c, i in picks:
        ref_u, _ = orc.lightcone(L, c, f, 0.1, RF, SEED, i, 1, n)
        assert abs(u[c * L + i] - ref_u[0]) <= 1e-4, (c, i)
    dub = obs["ubar"][2] - obs["ubar"][1]
    assert np.all(np.abs(dub - 0.1 * obs["v"][1]) <= 2e-6 * np.maximum(1, np.abs(obs["ubar"][1])))


def test_maximum_chain_length(qew, orc):
    """The longest chain the ABI accepts, L = 2^31 - 1 (int32 site index; 34 GB of FP32-split
    state in two buffers): odd, so every tile width leaves a ragged tail, and its last windows wrap
    around the seam at 2^31 - 1.  Sampled sites against the oracle's light-cone evaluation after
    70 steps (two full K = 32 launches and a ragged one in the largest shape), and the invariant
    dubar = dt v."""
    L, n, f = (1 << 31) - 1, 70, 1.2
    steps = np.array([0, n - 1, n])
    with qew.Relaxation(L, f, RF, dt=0.1, seed=SEED, precision=FP32) as r:
        r.set_tuning(1248, 32, 1)
        obs = r.observe(steps)
        u, _ = r.state()
    w_own = 1248 - 64
    rng = np.random.default_rng(5)
    picks = [0, 1, 2, w_own - 1, w_own, L // 2, L - w_own, L - 3, L - 2, L - 1] + list(rng.integers(0, L, 4))
    for i in picks:
        ref_u, _ = orc.lightcone(L, 0, f, 0.1, RF, SEED, int(i), 1, n)
        assert abs(u[i] - ref_u[0]) <= 1e-4, i
    del u
    dub = obs["ubar"][2] - obs["ubar"][1]
    assert np.all(np.abs(dub - 0.1 * obs["v"][1]) <= 2e-6 * np.maximum(1, np.abs(obs["ubar"][1])))


def test_maximum_chain_length_fp64(qew, orc):
    """The FP64 path on the same 2^31 - 1-site chain (one thread per site, neighbours wrapped at
    the seam): sampled sites to 1e-12 after 20 steps."""
    L, n, f = (1 << 31) - 1, 20, 1.2
    with qew.Relaxation(L, f, RF, dt=0.1, seed=SEED, precision=FP64) as r:
        r.observe([n])
        u, _ = r.state()
    for i in [0, 1, 1023, 1024, L // 2, L - 1025, L - 2, L - 1]:
        ref_u, _ = orc.lightcone(L, 0, f, 0.1, RF, SEED, i, 1, n)
        assert abs(u[i] - ref_u[0]) <= 1e-12 * max(1.0, abs(ref_u[0])), i


def test_rf_at_the_paper_size_has_the_printed_shape(qew):
    """The bench's 4 x 2^25 random-field chains at their f_c^L, 10^4 steps (t <= 10^3).
    - The corrected-form fit of V (procedure (a) of Sec. IV.E) gives beta/nu z near the printed
      0.128.
    - The effective slopes over the last decade match the long-time values of Sec. IV.B:
      -0.13 for v and 0.84 for w.
    - The slope of w over the decade before is near the short-time 0.67.
    - The amplitude is compared only in order of magnitude with the printed
      v = 0.53 t^-0.128 [1 + (t/0.382)^-0.927] (Sec. IV.D). The paper does not give its
      disorder strength, and the unit Gaussian here has a lower threshold (0.72 against 0.97).
    - The corrected fit of w is not asserted: within t <= 10^3 its exponent is poorly determined.
      The slope of w still rises through the window, and the fit extrapolates it (0.96 here, 1.02
      for the oracle at L = 8192).
    The oracle at L = 8192 (32 chains) gives -0.133 and 0.808 over the last decade."""
    from paper_1211_7275_gb300 import std
    from qew_workloads import preset_f
    steps = log_spaced_steps(10_000, 60)
    with qew.Relaxation(1 << 25, preset_f("rf_4x2^25"), RF, dt=0.1, seed=SEED, batch=4) as r:
        r.set_tuning(0, 0, 0)
        obs = r.observe(steps)
    t = steps * 0.1
    V, W = obs["v"].mean(1), np.sqrt(obs["w2"].mean(1))
    fv = std.fit_corrected(t, V, t_mic=2.0)

    def slope(y, a, b):
        sel = (t >= a) & (t <= b)
        return np.polyfit(np.log(t[sel]), np.log(y[sel]), 1)[0]

    sv, sw, sw_short = slope(V, 100, 1000), slope(W, 100, 1000), slope(W, 10, 100)
    sel = t >= 1.5
    ratio = V[sel] / std.corrected(t[sel], 0.53, -0.128, 0.382, 0.927)
    print(f"RF at 4 x 2^25: beta/nu z = {-fv['e']:.4f}; slopes over [100, 1000]: v {sv:.4f}, w {sw:.4f}; "
          f"w over [10, 100] {sw_short:.4f}; V / printed fit in [{ratio.min():.3f}, {ratio.max():.3f}]")
    assert 0.10 <= -fv["e"] <= 0.16
    assert -0.15 <= sv <= -0.115
    assert 0.74 <= sw <= 0.88
    assert 0.60 <= sw_short <= 0.75
    assert 0.3 <= ratio.min() and ratio.max() <= 3.0


def test_full_size_autotuned_shape_is_bitwise_identical(qew):
    """The bench's launch configuration: on its 4 x 2^25 chains the autotuner picks a shape at
    step 1024.  The state after 1100 steps in that shape is bit for bit the state in the default
    shape (the per-site arithmetic does not depend on the tiling), so the sampled-site parity
    above holds for the bench's shape too."""
    from qew_workloads import preset_f
    L, batch, n = 1 << 25, 4, 1100
    f = preset_f("rf_4x2^25")
    with qew.Relaxation(L, f, RF, dt=0.1, seed=SEED, precision=FP32, batch=batch) as r:
        r.set_tuning(0, 0, 0)
        r.observe([n])
        u_auto, _ = r.state()
        shape = r.tuning()
    with qew.Relaxation(L, f, RF, dt=0.1, seed=SEED, precision=FP32, batch=batch) as r:
        r.observe([n])
        u_default, _ = r.state()
        default = r.tuning()
    print(f"autotuned shape {shape}, default {default}")
    np.testing.assert_array_equal(u_auto, u_default)


def test_handles_on_concurrent_host_threads(qew):
    """Different handles may run at the same time from different host threads (ctypes releases
    the interpreter lock during each call): four threads with four tile shapes, whose first
    launches raise the kernels' shared-memory limits concurrently, give the states of sequential
    runs bit for bit."""
    import threading
    L, steps = 30000, np.array([0, 17, 400])
    shapes = [(1248, 32, 1), (224, 8, 8), (992, 32, 2), (736, 16, 4)]
    out, errs = [None] * len(shapes), []

    def work(k):
        try:
            out[k] = gpu_run(qew, L, 1.1, RF, steps, FP32, tuning=shapes[k], seed=SEED + k)[1]
        except Exception as e:  # pragma: no cover
            errs.append(e)

    ths = [threading.Thread(target=work, args=(k,)) for k in range(len(shapes))]
    for t in ths:
        t.start()
    for t in ths:
        t.join()
    assert not errs, errs
    for k, sh in enumerate(shapes):
        np.testing.assert_array_equal(out[k], gpu_run(qew, L, 1.1, RF, steps, FP32, tuning=sh, seed=SEED + k)[1])


# ------------------------------------------------------------------------------------------
# argument errors (need a device for handle creation)
# ------------------------------------------------------------------------------------------
def test_errors(qew):
    with qew.Relaxation(100, 1.0) as r:
        r.observe([10])
        with pytest.raises(qew.QewError) as e:
            r.observe([5])
        assert e.value.code == -1
        with pytest.raises(qew.QewError) as e:
            r.set_precision(FP64)
        assert e.value.code == -6
        with pytest.raises(qew.QewError):
            r.set_tuning(512, 8, 4)
        with pytest.raises(qew.QewError):
            r.set_tuning(480, 200, 4)
        r.observe([])
        r.advance(0)


# ------------------------------------------------------------------------------------------
# graph replay, failure path
# ------------------------------------------------------------------------------------------
def test_graph_replay_is_bitwise_identical(qew):
    steps = log_spaced_steps(3000, 15)
    with qew.Relaxation(30000, 0.72057, RF, dt=0.1, seed=SEED, batch=2) as r:
        first = r.observe(steps)            # captured
        r.reset()
        second = r.observe(steps)           # replayed
        u_replay, _ = r.state()
        r.reset()
        r.enable_stats(True)                # statistics switch graphs off: direct launches
        third = r.observe(steps)
        st = r.stats()
        u_direct, _ = r.state()
    for k in ("v", "ubar", "w2"):
        assert np.array_equal(first[k], second[k])
        assert np.array_equal(first[k], third[k])
    assert np.array_equal(u_replay, u_direct)
    assert st["fused_launches"] > 0


def test_bounded_wait_gives_up_and_reports(qew):
    lib = qew.load()
    with qew.Relaxation(1000, 1.0) as r:
        rc = lib.qew_selftest_bounded_wait(r._h, 4096)
        assert rc == -4, lib.qew_last_error(r._h)   # QEW_ETIMEOUT
        out = r.observe([0, 10])                      # the context and the handle still work
        assert np.all(np.isfinite(out["v"]))


# ------------------------------------------------------------------------------------------
# the other presets at full size (sampled sites; every launch shape computes the same states)
# ------------------------------------------------------------------------------------------
def _sampled_sites_check(qew, orc, L, f, kind, n_chains, n_steps, picks_per_chain, chains_to_check, tol=1e-4):
    Ls = np.atleast_1d(L)
    fs = np.broadcast_to(np.asarray(f, float), Ls.shape)
    ks = np.broadcast_to(np.asarray(kind, np.int32), Ls.shape)
    with qew.Relaxation(Ls, fs, ks, dt=0.1, seed=SEED) as r:
        r.set_tuning(0, 0, 0)
        obs = r.observe([0, n_steps - 1, n_steps])
        u, _ = r.state()
    off = np.concatenate([[0], np.cumsum(Ls)[:-1]])
    rng = np.random.default_rng(11)
    worst = 0.0
    for c in chains_to_check:
        Lc = int(Ls[c])
        sites = {0, Lc - 1} | set(int(x) for x in rng.integers(0, Lc, picks_per_chain))
        for i in sorted(sites):
            w = 1
            if 2 * n_steps + w > Lc:
                continue
            ref_u, _ = orc.lightcone(Lc, c, float(fs[c]), 0.1, int(ks[c]), SEED, i, w, n_steps)
            err = abs(u[off[c] + i] - ref_u[0])
            worst = max(worst, err)
            assert err <= tol, (c, i, err)
    dub = obs["ubar"][2] - obs["ubar"][1]
    assert np.all(np.abs(dub - 0.1 * obs["v"][1]) <= 2e-6 * np.maximum(1, np.abs(obs["ubar"][1])))
    return worst


def test_full_size_rf_16x2e20(qew, orc):
    from qew_workloads import PRESETS, preset_f
    p = PRESETS["rf_16x2^20"]
    _sampled_sites_check(qew, orc, [p["L"]] * p["batch"], preset_f("rf_16x2^20"), RF, p["batch"], 1000, 3,
                         chains_to_check=[0, 7, 15])


def test_full_size_rb_1024x2e16(qew, orc):
    from qew_workloads import PRESETS, preset_f
    p = PRESETS["rb_1024x2^16"]
    _sampled_sites_check(qew, orc, [p["L"]] * p["batch"], preset_f("rb_1024x2^16"), RB, p["batch"], 1000, 2,
                         chains_to_check=[0, 511, 1023])


def test_full_size_uneven_256(qew, orc):
    from qew_workloads import preset_f, sweep_offsets, uneven_kinds, uneven_lengths
    L = uneven_lengths(256)
    kinds = uneven_kinds(256)
    base = np.where(kinds == RF, preset_f("rf_16x2^20"), preset_f("rb_1024x2^16"))
    f = base * (1.0 + sweep_offsets(256))
    chains = [int(np.argmin(L)), int(np.argmax(L)), 5, 100, 255]
    _sampled_sites_check(qew, orc, L, f, kinds, 256, 600, 2, chains_to_check=chains)


@pytest.mark.parametrize("kind", [RF, RB, RBG_LINEAR, RBG_CUBIC])
def test_steep_state_within_the_exact_range(qew, orc, kind):
    """A valid but extreme state: a triangle wave rising by 4000 cells per site (below the 2^12
    limit on neighbouring displacements that qew_set_state enforces), so a tile window spans
    millions of cells.  The range guard at the end of each call checks the neighbour
    differences of such windows and must not raise; the cells relative to a tile's reference stay
    exact floats (below 2^24), and per site the FP32-split state follows the oracle over 100 steps
    to FP32 precision relative to u.  The Laplacian moves the peaks and valleys by hundreds of
    cells per step in both directions, so every disorder kind takes its multi-cell (all nodes
    drawn) and downward cache updates here, in every step."""
    L, f, n = 3000, 0.5, 100
    i = np.arange(L)
    tri = np.minimum(i % 600, 600 - i % 600)
    u0 = 4000.0 * tri + 0.25
    steps = np.array([0, 1, 10, n])
    obs, u, _ = gpu_run(qew, L, f, kind, steps, FP32, u0=u0)
    ref = orc.run(L, f, 0.1, kind, SEED, steps, u0=u0, want_state=True)
    # FP32 keeps the Laplacian's neighbour differences of ~4000 cells to 2^-24 relative, so the
    # per-site error scales with the local slope, not with 1e-4 cells
    rel = np.abs(u - ref["u"]) / np.maximum(1.0, np.abs(ref["u"]))
    bar = 1e-7
    if kind == RBG_LINEAR:
        # Case 3's force is piecewise constant: where the FP32 and the FP64 floor of a site
        # disagree, its force jumps by |G(n) - G(n+1)| = O(1).  Here the rounding scale of a step is
        # 4000 * 2^-24 = 2.4e-4 cells, and the exact dynamics itself moves by about 1e-5 relative
        # under a start perturbation of that size (1e-8 for the continuous forces), so that is the
        # bar.
        rng = np.random.default_rng(61)
        pert = orc.run(L, f, 0.1, kind, SEED, [n], u0=u0 + rng.uniform(-2.4e-4, 2.4e-4, L), want_state=True)["u"]
        bar = float(np.max(np.abs(pert - ref["u"]) / np.maximum(1.0, np.abs(ref["u"]))))
        print(f"Case 3: FP32-split vs oracle {rel.max():.2e}; the oracle under a 2.4e-4 start perturbation {bar:.2e}")
    assert rel.max() <= bar, (rel.max(), bar)
    # the fused sums are FP32 relative to a cell of each tile: error at most gamma_40 * D with D the
    # spread of a tile window (here 992 * 4000 cells; see tests/test_gpu_observables.py)
    D = 992 * 4000.0 + 1.0
    gamma = 40 * 2.0 ** -24 / (1 - 40 * 2.0 ** -24)
    assert np.all(np.abs(obs["ubar"][:, 0] - ref["ubar"][:, 0]) <= gamma * D)


def test_range_guard_reports_a_state_outside_the_exact_range(qew, orc):
    """A triangle wave rising 4095 cells per site is accepted (neighbours below 2^12 apart), but
    the pinning force pushes some neighbour differences to 4097-4098 cells within 50 steps (the
    oracle shows hundreds of such sites).  The range check at the end of the call must then report
    QEW_ESTATE instead of returning the observables; the next call starts clean."""
    L = 3000
    i = np.arange(L)
    tri = np.minimum(i % 600, 600 - i % 600)
    u0 = 4095.0 * tri + 0.25
    ref = orc.run(L, 0.5, 0.1, RF, SEED, [50], u0=u0, want_state=True)["u"]
    cells = np.floor(ref)
    assert np.abs(np.diff(np.r_[cells, cells[0]])).max() >= 4097   # the oracle crosses the bound
    with qew.Relaxation(L, 0.5, RF, dt=0.1, seed=SEED, precision=FP32) as r:
        r.set_state(u0)
        with pytest.raises(qew.QewError) as ei:
            r.observe([50])
        assert ei.value.code == -6 and b"2^12" in str(ei.value).encode()
        r.set_state(np.zeros(L))            # a valid state: the flag was cleared
        obs = r.observe([0, 10])
        assert np.all(np.isfinite(obs["v"]))


def test_creation_and_state_argument_errors(qew):
    """Every precondition of qew_create / qew_set_state is checked on the host and reported as
    QEW_EINVAL (-1); a batch larger than the device's memory is QEW_ENOMEM (-2), with nothing left
    allocated."""
    bad = [dict(L=0, f=1.0), dict(L=100, f=float("nan")), dict(L=100, f=4096.0), dict(L=100, f=1.0, dt=0.5),
           dict(L=100, f=1.0, dt=0.0), dict(L=100, f=1.0, kind=5), dict(L=1 << 31, f=1.0)]
    for kw in bad:
        with pytest.raises(qew.QewError) as e:
            qew.Relaxation(kw.pop("L"), kw.pop("f"), kw.pop("kind", RF), **kw)
        assert e.value.code == -1, kw
    with pytest.raises(qew.QewError) as e:   # 2^37 sites: the first state array alone exceeds the GPU
        qew.Relaxation((1 << 31) - 1, 1.0, RF, batch=64)
    assert e.value.code == -2
    with qew.Relaxation(100, 1.0) as r:
        for u in (np.r_[np.zeros(99), 5000.0], np.full(100, 2.0 ** 30), np.r_[np.zeros(99), np.inf]):
            with pytest.raises(qew.QewError) as e:
                r.set_state(u)
            assert e.value.code == -1
        obs = r.observe([0, 5])
        assert np.all(np.isfinite(obs["v"]))


def test_sample_indices_select_the_disorder(qew, orc):
    """qew_set_samples: a chain given sample index s relaxes on the disorder of sample s (the oracle
    with s), chains given the same index are identical, and resetting to 0..n-1 restores the default."""
    L, n = 777, 300
    with qew.Relaxation(L, 1.0, RF, dt=0.1, seed=SEED, precision=FP32, batch=3) as r:
        r.set_samples([5, 5, 9])
        r.observe([n])
        u, _ = r.state()
        r.set_samples([0, 1, 2])
        r.observe([n])
        u0, _ = r.state()
    u = u.reshape(3, L)
    assert np.array_equal(u[0], u[1]) and not np.array_equal(u[0], u[2])
    ref = orc.run([L] * 2, 1.0, 0.1, RF, SEED, [n], s=[5, 9], want_state=True)["u"].reshape(2, L)
    assert np.max(np.abs(u[0] - ref[0])) <= 1e-4 and np.max(np.abs(u[2] - ref[1])) <= 1e-4
    ref0 = orc.run([L] * 3, 1.0, 0.1, RF, SEED, [n], want_state=True)["u"]
    assert np.max(np.abs(u0 - ref0)) <= 1e-4


def test_fp64_per_site_at_the_critical_force(qew, orc):
    """The plain FP64 path at f_c^L (random field, 16 x 4096 sites, the oracle-bisected fixture):
    it evaluates the oracle's arithmetic in the oracle's order, so the near-threshold amplification
    acts only on the last-place differences of the transcendental functions (CUDA's log and cospi
    against the host libm's), and every site stays within 1e-12 relative over 10^3 steps (measured:
    1.6e-13, most sites bit for bit)."""
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "fc_rf_L4096.json")) as fh:
        fc = json.load(fh)
    L, f, B = fc["L"], fc["f_c"], 16
    with qew.Relaxation(L, f, RF, dt=0.1, seed=SEED, precision=FP64, batch=B) as r:
        r.observe([1000])
        u, _ = r.state()
    ref = orc.run([L] * B, f, 0.1, RF, SEED, [1000], want_state=True)["u"]
    err = np.abs(u - ref) / np.maximum(1.0, np.abs(ref))
    assert err.max() <= 1e-12, err.max()
