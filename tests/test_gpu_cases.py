"""GPU parity of the Gaussian random-bond kinds (Sec. IV.C): Case 3 (linear spline, the force
G(n) - G(n+1) constant in a cell and discontinuous at the integers) and Case 1 (Catmull-Rom
spline through the same G), through the C ABI against the CPU oracle.

Bars:
  - generator values G: FP64 to 4e-15 relative, FP32 to 6e-7 (the same transform as R);
  - FP64 path: per site |du| <= 1e-12 max(1, |u|) over 10^3 steps, for both kinds (the FP64 path
    takes the oracle's operations in the oracle's order, so even the discontinuous force is
    evaluated on the same side of every integer);
  - FP32-split, both kinds: per site |du| <= 1e-4 over the first 100 steps;
  - FP32-split, Case 1 over 10^3 steps: a distribution (rms <= 4e-5, at most 3% of sites above
    1e-4, max <= 3e-3).  The Gaussian nodes and the cubic's coefficients (up to ~20) make the FP32
    force error about ten times that of RF; a CPU model of the same FP32 arithmetic with correctly
    rounded nodes reaches max 1.1e-4 (L = 256) and 1.8e-4 (L = 4099) after 10^3 steps at f = 2.6,
    as the kernel does;
  - FP32-split, Case 3 over longer times: the force jumps by O(1) at the integers, so a site whose
    FP32 position lands on the other side of an integer than the FP64 one takes a different force
    for a step and the two trajectories part by O(dt) there.  Per-site parity stops being a
    meaningful bar once that has happened somewhere (a few hundred steps at L ~ 10^3), and the bar
    is the ensemble: V(t), W2(t) within 2 sigma of the oracle's;
  - every launch shape gives the same FP32-split state bit for bit (the per-site arithmetic does
    not depend on the tiling), which is checked exactly for both kinds.
"""
import json
import os

import numpy as np
import pytest

from qew_workloads import SEED, log_spaced_steps, random_points

pytestmark = pytest.mark.gpu

RF, RB, NONE, RBG_LINEAR, RBG_CUBIC = 0, 1, 2, 3, 4
FP32, FP64 = 0, 1
F_MOVING = {RBG_LINEAR: 2.2, RBG_CUBIC: 2.6, RB: 1.9}   # above f_c^L (about 1.55, 1.95, 0.91)


def _fc(name):
    with open(os.path.join(os.path.dirname(__file__), "golden", f"fc_{name}_L4096.json")) as fh:
        return json.load(fh)


@pytest.fixture(scope="module")
def qew():
    import paper_1211_7275_gb300 as q
    q.load()
    return q


def gpu_run(qew, L, f, kind, steps, precision, *, tuning=None, batch=1):
    with qew.Relaxation(L, f, kind, dt=0.1, seed=SEED, precision=precision, batch=batch) as r:
        if tuning is not None:
            r.set_tuning(*tuning)
        obs = r.observe(steps)
        u, step = r.state()
        cells = r.cells()
    assert step == steps[-1]
    return obs, u, cells


@pytest.mark.parametrize("kind", [RBG_LINEAR, RBG_CUBIC])
def test_gaussian_potential_values(qew, orc, kind):
    i, n = random_points(200_000, 1 << 25, -3000, 3000, seed=19)
    ref = orc.disorder_values(kind, SEED, 5, i, n)
    g64 = qew.disorder_values(kind, FP64, SEED, 5, i, n)
    g32 = qew.disorder_values(kind, FP32, SEED, 5, i, n)
    assert np.max(np.abs(g64 - ref) / np.maximum(1.0, np.abs(ref))) < 4e-15
    assert np.max(np.abs(g32 - ref) / np.maximum(1.0, np.abs(ref))) < 6e-7


@pytest.mark.parametrize("kind,L,f", [(RBG_LINEAR, 1024, 2.2), (RBG_LINEAR, 5, 3.0), (RBG_LINEAR, 4096, 1.5546),
                                      (RBG_CUBIC, 777, 2.6), (RBG_CUBIC, 3, 3.0)])
def test_fp64_per_site(qew, orc, kind, L, f):
    steps = np.array([0, 1, 2, 10, 100, 1000])
    obs, u, cells = gpu_run(qew, L, f, kind, steps, FP64)
    ref = orc.run(L, f, 0.1, kind, SEED, steps, want_state=True)
    err = np.abs(u - ref["u"]) / np.maximum(1.0, np.abs(ref["u"]))
    assert err.max() <= 1e-12, err.max()
    assert np.array_equal(cells, np.floor(ref["u"]).astype(np.int32))
    np.testing.assert_allclose(obs["v"], ref["v"], rtol=0, atol=1e-11)
    np.testing.assert_allclose(obs["w2"], ref["w2"], rtol=1e-9, atol=1e-12)


@pytest.mark.parametrize("L", [3, 256, 4099])
def test_split_case1_per_site(qew, orc, L):
    f = F_MOVING[RBG_CUBIC]
    steps = np.array([0, 3, 50, 100])
    ref = orc.run(L, f, 0.1, RBG_CUBIC, SEED, steps, want_state=True)
    obs, u, cells = gpu_run(qew, L, f, RBG_CUBIC, steps, FP32)
    err = np.abs(u - ref["u"])
    assert err.max() <= 1e-4, err.max()
    far = np.abs(ref["u"] - np.round(ref["u"])) > 1e-4
    assert np.array_equal(cells[far], np.floor(ref["u"][far]).astype(np.int32))
    np.testing.assert_allclose(obs["v"], ref["v"], rtol=0, atol=2e-4)
    # 10^3 steps: the FP32 deviation is a distribution
    ref = orc.run(L, f, 0.1, RBG_CUBIC, SEED, np.array([0, 1000]), want_state=True)
    _, u, _ = gpu_run(qew, L, f, RBG_CUBIC, np.array([0, 1000]), FP32)
    err = np.abs(u - ref["u"])
    rms, frac, mx = float(np.sqrt(np.mean(err ** 2))), float(np.mean(err > 1e-4)), float(err.max())
    print(f"Case 1 FP32-split vs oracle after 1000 steps, L={L}: rms {rms:.2e}, >1e-4: {frac:.1e}, max {mx:.2e}")
    assert rms <= 4e-5 and frac <= 3e-2 and mx <= 3e-3, (rms, frac, mx)


@pytest.mark.parametrize("L", [1, 3, 33, 1024, 5000])
def test_split_case3_per_site(qew, orc, L):
    """Every site within 1e-4 of the oracle after 7 steps; after 100 steps all but the few sites
    next to a step at which the FP32 and FP64 positions sat on opposite sides of an integer (at
    most 0.2% of 4 x 5000 sites: one such event moves a site by dt |dF| ~ 0.1-0.3 and its
    neighbours by less)."""
    f = F_MOVING[RBG_LINEAR]
    ref7 = orc.run([L] * 4, f, 0.1, RBG_LINEAR, SEED, np.array([0, 1, 7]), want_state=True)
    ref = orc.run([L] * 4, f, 0.1, RBG_LINEAR, SEED, np.array([0, 1, 7, 100]), want_state=True)
    with qew.Relaxation(L, f, RBG_LINEAR, dt=0.1, seed=SEED, precision=FP32, batch=4) as r:
        obs7 = r.observe(np.array([0, 1, 7]))
        u7, _ = r.state()
        cells7 = r.cells()
        r.observe(np.array([100]))
        u, _ = r.state()
    err7 = np.abs(u7 - ref7["u"])
    assert err7.max() <= 1e-4, err7.max()
    far = np.abs(ref7["u"] - np.round(ref7["u"])) > 1e-4
    assert np.array_equal(cells7[far], np.floor(ref7["u"][far]).astype(np.int32))
    np.testing.assert_allclose(obs7["v"], ref7["v"], rtol=0, atol=2e-4)
    np.testing.assert_allclose(obs7["ubar"], ref7["ubar"], rtol=0, atol=2e-5)
    err = np.abs(u - ref["u"])
    frac = float(np.mean(err > 1e-4))
    print(f"Case 3 FP32-split vs oracle after 100 steps, L={L}: max {err.max():.2e}, above 1e-4: {frac:.1e}")
    assert frac <= 2e-3, frac


@pytest.mark.parametrize("kind,shapes", [
    (RBG_LINEAR, [(480, 16, 4), (224, 8, 2), (992, 32, 1), (736, 24, 8), (480, 13, 2), (1248, 32, 1)]),
    (RBG_CUBIC, [(224, 16, 4), (480, 8, 2), (224, 13, 1), (480, 32, 8)]),
    (RB, [(224, 16, 4), (480, 8, 2), (224, 13, 1), (480, 32, 8)]),
])
def test_split_shapes_identical(qew, kind, shapes):
    """Every launch shape performs the same per-site arithmetic: states agree bit for bit, so the
    discontinuous Case 3 force is taken on the same side of every integer whatever the tiling, and
    the cubic coefficients (computed at tile load and at regeneration, in kernels instantiated per
    tile shape) round the same way everywhere."""
    L, steps = 20000, np.array([0, 5, 333, 1000])
    f = F_MOVING[kind]
    _, u_ref, c_ref = gpu_run(qew, L, f, kind, steps, FP32, tuning=shapes[0])
    for shape in shapes[1:]:
        _, u, c = gpu_run(qew, L, f, kind, steps, FP32, tuning=shape)
        assert np.array_equal(u, u_ref), shape
        assert np.array_equal(c, c_ref), shape


def test_mixed_batch_all_kinds(qew, orc):
    """One handle holding chains of all five kinds (the two-node cache array is shared by the RF
    and Case 3 chains, the four-node one by the two cubic random-bond kinds)."""
    L = np.array([300, 4097, 77, 1025, 2048, 5, 999])
    kind = np.array([RF, RB, NONE, RBG_LINEAR, RBG_CUBIC, RBG_LINEAR, RBG_CUBIC], dtype=np.int32)
    f = np.array([1.0, 1.9, 0.5, 2.2, 2.6, 3.0, 2.8])
    steps = np.array([0, 10, 100])
    ref = orc.run(L, f, 0.1, kind, SEED, steps, want_state=True)
    off = np.concatenate([[0], np.cumsum(L)])
    for prec in (FP32, FP64):
        with qew.Relaxation(L, f, kind, dt=0.1, seed=SEED, precision=prec) as r:
            obs = r.observe(steps)
            u, _ = r.state()
        if prec == FP64:
            assert np.max(np.abs(u - ref["u"]) / np.maximum(1, np.abs(ref["u"]))) <= 1e-12
            np.testing.assert_allclose(obs["v"], ref["v"], atol=1e-11)
            continue
        for c in range(len(L)):
            e = np.abs(u[off[c]:off[c + 1]] - ref["u"][off[c]:off[c + 1]])
            assert e.max() <= 1e-4, (c, e.max())
        np.testing.assert_allclose(obs["w2"], ref["w2"], rtol=2e-3, atol=1e-5)


def test_mixed_batch_per_kind_tile_widths(qew):
    """In a mixed batch each kind runs the widest tile it supports up to the requested one (cubic
    random-bond chains at most 480 sites, disorder-free chains at most 992): the states agree bit
    for bit with those of the narrowest common shape, and the reported width is the widest in use."""
    L = np.array([3000, 4097, 777, 5025, 2048, 9999])
    kind = np.array([RF, RB, NONE, RBG_LINEAR, RBG_CUBIC, RF], dtype=np.int32)
    f = np.array([1.0, 1.9, 0.5, 2.2, 2.6, 1.2])
    steps = np.array([0, 5, 333, 600])
    runs = []
    for shape, want_w in [((224, 8, 2), 224), ((1248, 32, 1), 1248), ((992, 16, 2), 992), ((736, 24, 4), 736)]:
        with qew.Relaxation(L, f, kind, dt=0.1, seed=SEED) as r:
            r.set_tuning(*shape)
            assert r.tuning()[0] == want_w
            r.observe(steps)
            runs.append((r.state()[0], r.cells()))
    for u, c in runs[1:]:
        assert np.array_equal(u, runs[0][0]) and np.array_equal(c, runs[0][1])
    with qew.Relaxation(L[1:2], f[1:2], kind[1:2], dt=0.1, seed=SEED) as r:
        r.set_tuning(1248, 32, 1)   # a cubic random-bond batch alone: 480-site tiles
        assert r.tuning()[0] == 480


@pytest.mark.parametrize("precision", [FP32, FP64])
def test_case3_mean_velocity_invariant(qew, precision):
    """dubar = dt v also with the discontinuous force: the periodic Laplacian sums to zero."""
    steps = np.array([0, 1, 2, 3, 50, 51, 400, 401])
    obs, _, _ = gpu_run(qew, 10007, 1.6, RBG_LINEAR, steps, precision)
    ub, v = obs["ubar"][:, 0], obs["v"][:, 0]
    tol = 1e-12 if precision == FP64 else 2e-6
    for j in range(len(steps) - 1):
        if steps[j + 1] == steps[j] + 1:
            assert abs((ub[j + 1] - ub[j]) - 0.1 * v[j]) <= tol * max(1.0, abs(ub[j])), j


@pytest.mark.parametrize("name,kind", [("rbg_linear", RBG_LINEAR), ("rbg_cubic", RBG_CUBIC)])
def test_ensemble_at_fc_within_two_sigma(qew, orc, name, kind):
    """At the oracle-bisected f_c^L (L = 4096 fixture; used here on L = 1024 chains), 32 samples to
    t = 10^3: the ensemble V(t), W2(t) of both GPU paths within 2 sigma of the oracle's, and the
    FP64 path equal to the oracle to rounding through step 100.

    Equality to rounding cannot hold to t_max at the critical force: there a chain can pass
    through strongly unstable stretches of the cubic Gaussian potential, which amplify a
    difference of one unit in the last place to an O(1) change in a site and a visible change in
    v.  The oracle shows this on its own: a perturbation of 1e-14 of sample 25's state at step 20
    changes its v by 0.4% at step 201."""
    fc = _fc(name)["f_c"]
    n_s, L = 32, 1024
    steps = log_spaced_steps(10_000, 30)
    early = steps <= 100
    ref = orc.run([L] * n_s, fc, 0.1, kind, SEED, steps)
    with qew.Relaxation(L, fc, kind, dt=0.1, seed=SEED, precision=FP32, batch=n_s) as r:
        obs = r.observe(steps)
    with qew.Relaxation(L, fc, kind, dt=0.1, seed=SEED, precision=FP64, batch=n_s) as r:
        obs64 = r.observe(steps)
    for key in ("v", "w2"):
        m_ref = ref[key].mean(1)
        sig = ref[key].std(1, ddof=1) / np.sqrt(n_s)
        sig[0] = max(sig[0], 1e-12)
        for label, o in (("FP32", obs), ("FP64", obs64)):
            ok = np.abs(o[key].mean(1) - m_ref) <= 2 * sig + 1e-12
            assert ok.all(), (label, key, np.where(~ok))
        paired = np.abs(obs[key] - ref[key]).mean(1)
        print(f"{name} {key}: paired |FP32 - oracle| / sample sd, max over t: "
              f"{np.max(paired[1:] / np.maximum(ref[key].std(1, ddof=1)[1:], 1e-12)):.2e}")
        np.testing.assert_allclose(obs64[key][early], ref[key][early], rtol=1e-9, atol=1e-11)


def test_full_size_case3_4x2e25(qew, orc):
    """The Case 3 preset at full size (4 x 2^25 sites, f = 1.5652, the paper's L = 2^25 value for
    this case) in the launch shape the autotuner picks: sampled sites (chain ends, tile edges,
    random sites) after 100 steps against the oracle's light-cone evaluation of the same site, and
    dubar = dt v on every chain."""
    from qew_workloads import PRESETS, preset_f
    p = PRESETS["rbg_linear_4x2^25"]
    L, batch, n = p["L"], p["batch"], 100
    f = preset_f("rbg_linear_4x2^25")
    with qew.Relaxation(L, f, RBG_LINEAR, dt=0.1, seed=SEED, precision=FP32, batch=batch) as r:
        r.set_tuning(0, 0, 0)
        obs = r.observe(np.array([0, n - 1, n]))
        u, _ = r.state()
        tile_w, K, _ = r.tuning()
    w_own = tile_w - 2 * K
    rng = np.random.default_rng(5)
    for c in range(batch):
        for i in [0, 1, L - 1, w_own - 1, w_own, 7 * w_own + 3] + [int(x) for x in rng.integers(0, L, 3)]:
            ref_u, _ = orc.lightcone(L, c, f, 0.1, RBG_LINEAR, SEED, i, 1, n)
            assert abs(u[c * L + i] - ref_u[0]) <= 1e-4, (c, i, u[c * L + i], ref_u[0])
    dub = obs["ubar"][2] - obs["ubar"][1]
    assert np.all(np.abs(dub - 0.1 * obs["v"][1]) <= 2e-6 * np.maximum(1, np.abs(obs["ubar"][1])))


def test_case3_at_the_paper_size_follows_the_printed_fits(qew):
    """Case 3 at the paper's largest run (4 x 2^25 sites, f_c = 1.5652, dt = 0.1, Sec. IV.D), 10^4
    steps: V(t) within 3% of the printed v = 0.721 t^-0.128 [1 + (t/0.110)^-0.715] for t >= 1.5,
    and the corrected-form fits of V and w (procedure (a) of Sec. IV.E, t_mic = 2) give exponents
    near the printed beta/nu z = 1 - zeta/z = 0.128."""
    from paper_1211_7275_gb300 import std
    steps = log_spaced_steps(10_000, 60)
    with qew.Relaxation(1 << 25, 1.5652, RBG_LINEAR, dt=0.1, seed=SEED, batch=4) as r:
        r.set_tuning(0, 0, 0)
        obs = r.observe(steps)
    t = steps * 0.1
    V, W2 = obs["v"].mean(1), obs["w2"].mean(1)
    sel = t >= 1.5
    ratio = V[sel] / std.corrected(t[sel], 0.721, -0.128, 0.110, 0.715)
    print(f"Case 3 at 4 x 2^25: V / printed fit in [{ratio.min():.4f}, {ratio.max():.4f}]")
    assert np.all(np.abs(ratio - 1) < 0.03)
    fv = std.fit_corrected(t, V, t_mic=2.0)
    fw = std.fit_corrected(t, np.sqrt(W2), t_mic=2.0)
    print(f"corrected fits: beta/nu z = {-fv['e']:.4f} (V0 {fv['A']:.3f}), zeta/z = {fw['e']:.4f}")
    assert 0.115 <= -fv["e"] <= 0.14
    assert 0.82 <= fw["e"] <= 0.95



@pytest.mark.parametrize("criterion", ["v", "gamma"])
def test_bisection_criteria_bracket_the_threshold(qew, criterion):
    """Both bisection criteria (the V t^0.128 slope and the gamma drift of Sec. IV.F) call a drive
    20% above the random-field f_c^L of the 16 x 2^20 preset "above" and 20% below "below"."""
    from paper_1211_7275_gb300 import bisect
    from qew_workloads import preset_f
    fc = preset_f("rf_16x2^20")
    up = bisect.drift(1.2 * fc, 1 << 16, 8, RF, 4096, criterion=criterion)
    down = bisect.drift(0.8 * fc, 1 << 16, 8, RF, 4096, criterion=criterion)
    assert up >= 0 > down, (up, down)


def test_std_command_line(qew):
    """python -m paper_1211_7275_gb300.std relaxes a batch on the GPU and prints its short-time
    analysis as one JSON line (Sec. IV.C-F): finite exponents near the class's values for random-
    field chains at their threshold."""
    import json
    import subprocess
    import sys
    out = subprocess.run([sys.executable, "-m", "paper_1211_7275_gb300.std", "--L", "65536", "--batch", "8",
                          "--f", "0.7206", "--kind", "0", "--steps", "20000", "--obs", "40"],
                         capture_output=True, text=True, check=True,
                         cwd=os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    d = json.loads(out.stdout.strip().splitlines()[-1])
    assert d["observations"] >= 30 and len(d["window_v"]) == len(d["window_t0"])
    assert 0.08 <= d["beta_over_nu_z"] <= 0.2
    assert 0.7 <= d["zeta_over_z"] <= 1.0
