"""Ensemble parity of the FP32-split path on the workloads' own shapes (Sec. II, Eqs. 3-5).

The observables the paper measures are sample averages: V(t) = <v_s(t)> and W2(t) = <w2_s(t)>
over independent disorder samples s.  Bar: V(t) and W2(t) of the fast path lie within 2 sigma of
the reference ensemble at every observation time, sigma = sample standard deviation / sqrt(N).
Both sides relax the same disorder samples (same seed and sample indices), so the paired
difference |x_fast - x_ref| of each sample is also reported and must stay well below the
sample-to-sample spread (a quarter of the standard deviation).

References: the CPU oracle itself on small chains; on the workloads' full sizes the FP64 GPU path
(itself equal to the oracle to 1e-12 per site over 10^3 steps, tests/test_gpu_parity.py), over the
horizon its run time allows:
  - 16 x 2^20 random field at f_c^L: the full 2^16 steps, 60 log-spaced observations;
  - 1024 x 2^16 uniform random bond at f_c^L: the first 2^13 of its 2^18 steps;
  - 4 x 2^25 random field at f_c^L: the first 2^11 of its 2^20 steps;
  - the uneven batch of 256 chains: the first 2^11 of its 2^17 steps, and a sample of its chains
    run one by one (FP64 and FP32-split), which must equal the batched chains bit for bit.
"""
import json
import os

import numpy as np
import pytest

from qew_workloads import (SEED, log_spaced_steps, preset_f, sweep_offsets, uneven_kinds,
                           uneven_lengths)

pytestmark = pytest.mark.gpu

RF, RB = 0, 1
FP32, FP64 = 0, 1


@pytest.fixture(scope="module")
def qew():
    import paper_1211_7275_gb300 as q
    q.load()
    return q


def fc_fixture(name):
    with open(os.path.join(os.path.dirname(__file__), "golden", name)) as fh:
        return json.load(fh)["f_c"]


def relax(qew, L, f, kind, steps, precision, batch=None, samples=None, tuning=None):
    with qew.Relaxation(L, f, kind, dt=0.1, seed=SEED, precision=precision, batch=batch) as r:
        if samples is not None:
            r.set_samples(samples)
        if tuning is not None:
            r.set_tuning(*tuning)
        obs = r.observe(steps)
        obs["tuning"] = r.tuning()
        return obs


def compare(fast, ref, label, keys=("v", "w2"), paired_frac=0.25):
    """V(t), W2(t) of ``fast`` within 2 sigma of ``ref``; paired differences below
    ``paired_frac`` of the sample standard deviation.  Returns the worst ratios, printed."""
    N = ref["v"].shape[1]
    worst = {}
    for key in keys:
        a, b = fast[key], ref[key]
        sd = b.std(1, ddof=1)
        sig = sd / np.sqrt(N)
        scale = np.maximum(np.abs(b).max(1), 1e-300)
        dm = np.abs(a.mean(1) - b.mean(1))
        ok = dm <= 2 * sig + 1e-12 * scale
        assert ok.all(), (label, key, np.where(~ok)[0], dm[~ok], sig[~ok])
        paired = np.abs(a - b).mean(1)
        live = sd > 1e-12 * scale
        okp = paired[live] <= paired_frac * sd[live]
        assert okp.all(), (label, key, paired[live][~okp], sd[live][~okp])
        worst[key] = (float(np.max(dm[live] / sig[live])) if live.any() else 0.0,
                      float(np.max(paired[live] / sd[live])) if live.any() else 0.0)
    print(f"{label}: max |dmean|/sigma, max paired/sd: " +
          ", ".join(f"{k} {z:.2e} {p:.2e}" for k, (z, p) in worst.items()))
    return worst


# ------------------------------------------------------------------------------------------
# small chains against the oracle itself, at the critical force
# ------------------------------------------------------------------------------------------
def test_rf_at_fc_small_chains_vs_oracle(qew, orc):
    """32 random-field samples of L = 1024 at the oracle-bisected f_c^L, 10^4 steps."""
    f, L, N = fc_fixture("fc_rf_L4096.json"), 1024, 32
    steps = log_spaced_steps(10_000, 40)
    ref = orc.run([L] * N, f, 0.1, RF, SEED, steps)
    compare(relax(qew, L, f, RF, steps, FP32, batch=N), ref, "RF f_c 32x1024 FP32-split vs oracle")
    compare(relax(qew, L, f, RF, steps, FP64, batch=N), ref, "RF f_c 32x1024 FP64 vs oracle")


def test_uniform_rb_at_fc_small_chains_vs_oracle(qew, orc):
    """32 uniform random-bond samples of L = 1024 at the preset's f_c^L, 10^4 steps."""
    f, L, N = preset_f("rb_1024x2^16"), 1024, 32
    steps = log_spaced_steps(10_000, 40)
    ref = orc.run([L] * N, f, 0.1, RB, SEED, steps)
    compare(relax(qew, L, f, RB, steps, FP32, batch=N), ref, "RB f_c 32x1024 FP32-split vs oracle")


# ------------------------------------------------------------------------------------------
# the workloads' full sizes against the FP64 GPU path
# ------------------------------------------------------------------------------------------
def test_rf_16x2e20_full_horizon_vs_fp64(qew):
    """16 x 2^20 random field at f_c^L, 2^16 steps, 60 log-spaced observations."""
    f = preset_f("rf_16x2^20")
    steps = log_spaced_steps(1 << 16, 60)
    fast = relax(qew, 1 << 20, f, RF, steps, FP32, batch=16)
    ref = relax(qew, 1 << 20, f, RF, steps, FP64, batch=16)
    compare(fast, ref, "RF 16x2^20 to 2^16 steps")


def test_rb_1024x2e16_prefix_vs_fp64(qew):
    """1024 x 2^16 uniform random bond at f_c^L, the first 2^13 steps, 40 observations."""
    f = preset_f("rb_1024x2^16")
    steps = log_spaced_steps(1 << 13, 40)
    fast = relax(qew, 1 << 16, f, RB, steps, FP32, batch=1024)
    ref = relax(qew, 1 << 16, f, RB, steps, FP64, batch=1024)
    compare(fast, ref, "RB 1024x2^16 to 2^13 steps")


def test_rf_4x2e25_prefix_vs_fp64(qew):
    """4 x 2^25 random field at f_c^L (the paper's largest chains), the first 2^11 steps."""
    f = preset_f("rf_4x2^25")
    steps = log_spaced_steps(1 << 11, 30)
    fast = relax(qew, 1 << 25, f, RF, steps, FP32, batch=4)
    ref = relax(qew, 1 << 25, f, RF, steps, FP64, batch=4)
    compare(fast, ref, "RF 4x2^25 to 2^11 steps")


def test_uneven_256_prefix_vs_fp64_and_one_by_one(qew):
    """The uneven batch (256 chains, L log-uniform in 2^12 .. 2^22, random field and uniform
    random bond 50/50, each at f_c^L of its kind times 1 + {-2, -1, 0, 1, 2}%), first 2^11 steps.
    Per (kind, drive) group the FP32-split ensemble is compared with the FP64 one; then six
    chains are relaxed on their own, in both precisions, with their sample index and the batch's
    launch shape, and must reproduce their batched observables bit for bit (no chain depends on
    its neighbours in the batch)."""
    n = 256
    L = uneven_lengths(n)
    kinds = uneven_kinds(n)
    off = sweep_offsets(n)
    f = np.where(kinds == RF, preset_f("rf_16x2^20"), preset_f("rb_1024x2^16")) * (1.0 + off)
    steps = log_spaced_steps(1 << 11, 20)
    fast = relax(qew, L, f, kinds, steps, FP32)
    ref = relax(qew, L, f, kinds, steps, FP64)
    for k in (RF, RB):
        for o in np.unique(off):
            sel = np.where((kinds == k) & (off == o))[0]
            sub = lambda obs: {key: obs[key][:, sel] for key in ("v", "w2")}  # noqa: E731
            compare(sub(fast), sub(ref), f"uneven kind {k} offset {o:+.2f} ({sel.size} chains)")
    pick = [int(np.argmin(L)), int(np.argmax(L)), 3, 77, 128, 250]
    for c in pick:
        for prec, batched in ((FP32, fast), (FP64, ref)):
            alone = relax(qew, [int(L[c])], [float(f[c])], [int(kinds[c])], steps, prec, samples=[c],
                          tuning=fast["tuning"] if prec == FP32 else None)
            for key in ("v", "ubar", "w2"):
                assert np.array_equal(alone[key][:, 0], batched[key][:, c]), (c, prec, key)
