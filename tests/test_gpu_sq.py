"""GPU parity of the structure factor S_q (Eq. 6, Sec. II of arXiv:1211.7275) through the C ABI.

The GPU evaluates S_q on its own state and the oracle on its own state after the same relaxation.
  - FP64 path: the states agree to ~1e-12, so S_q agrees to rtol 1e-9.
  - FP32-split path: with eps = max |u_gpu - u_oracle| <= 1e-4, each mode amplitude moves by
    at most eps (triangle inequality on the defining sum), and by Cauchy-Schwarz over the chains
    |S_gpu - S_ref| <= 2 eps sqrt(S_ref) + eps^2.
  - Parseval ties the spectrum to the width w2 that the fused reductions report (another code
    path): the sum over n = 1 .. L-1 of S_q equals the chain mean of w2.
  - Closed form: a disorder-free cosine mode decays by lambda_k per Euler step.
"""
import math

import numpy as np
import pytest

from qew_workloads import SEED, cosine_profile, random_state

pytestmark = pytest.mark.gpu

RF, RB, NONE = 0, 1, 2
FP32, FP64 = 0, 1


@pytest.fixture(scope="module")
def qew():
    import paper_1211_7275_gb300 as q
    q.load()
    return q


def _parseval(S, L):
    return 2.0 * S.sum() - (S[-1] if L % 2 == 0 else 0.0)


@pytest.mark.parametrize("L,kind,f", [(1024, RF, 1.0), (777, RB, 1.9), (4, RF, 0.8)])
def test_fp64_matches_oracle(qew, orc, L, kind, f):
    n_s, n = 8, 500
    ref = orc.run([L] * n_s, f, 0.1, kind, SEED, [n], want_state=True)
    with qew.Relaxation(L, f, kind, dt=0.1, seed=SEED, precision=FP64, batch=n_s) as r:
        r.observe([n])
        S = r.structure_factor()
    S_ref = orc.structure_factor(ref["u"], L)
    np.testing.assert_allclose(S, S_ref, rtol=1e-9, atol=1e-12 * S_ref.max())


@pytest.mark.parametrize("L,kind,f", [(1024, RF, 1.0), (4099, RF, 1.1), (1000, RB, 1.9)])
def test_split_matches_oracle_within_the_state_bound(qew, orc, L, kind, f):
    n_s, n = 4, 1000
    ref = orc.run([L] * n_s, f, 0.1, kind, SEED, [n], want_state=True)
    with qew.Relaxation(L, f, kind, dt=0.1, seed=SEED, precision=FP32, batch=n_s) as r:
        r.observe([n])
        u, _ = r.state()
        S = r.structure_factor()
    eps = 1e-4
    assert np.max(np.abs(u - ref["u"])) <= eps
    S_ref = orc.structure_factor(ref["u"], L)
    assert np.all(np.abs(S - S_ref) <= 2 * eps * np.sqrt(S_ref) + eps * eps)


# The fused reductions of the split path sum in FP32 within a warp tile (relative error of w2 up
# to ~1e-5); the FP64 path sums in FP64.
W2_RTOL = {FP32: 1e-4, FP64: 1e-9}


@pytest.mark.parametrize("precision", [FP32, FP64])
def test_parseval_against_the_fused_width(qew, precision):
    L, n_s = 2048, 6
    with qew.Relaxation(L, 0.9, RF, dt=0.1, seed=SEED, precision=precision, batch=n_s) as r:
        obs = r.observe([700])
        S = r.structure_factor()
    w2 = float(np.mean(obs["w2"][0]))
    assert abs(_parseval(S, L) - w2) <= W2_RTOL[precision] * w2


@pytest.mark.parametrize("precision", [FP32, FP64])
def test_invariant_under_a_lift_of_the_line(qew, precision):
    """S_q at q != 0 does not see the height of the line (Eq. 6): the same rough lines lifted or
    lowered by 2^29 cells give the same spectrum bit for bit, because each chain's rows are formed
    relative to the cell of its first site, exactly in FP64."""
    L, n_s = 1000, 3
    u = np.round(random_state(L * n_s, 0.7, seed=51) * 64) / 64   # exact in both layouts
    spectra = []
    for lift in (0.0, 2.0 ** 29, -(2.0 ** 29)):
        with qew.Relaxation(L, 0.5, NONE, precision=precision, batch=n_s) as r:
            r.set_state(u + lift)
            spectra.append(r.structure_factor())
    assert spectra[0].max() > 0
    np.testing.assert_array_equal(spectra[1], spectra[0])
    np.testing.assert_array_equal(spectra[2], spectra[0])


@pytest.mark.parametrize("precision,tol", [(FP64, 1e-12), (FP32, 1e-6)])
def test_disorder_free_mode_decay(qew, precision, tol):
    L, k, A, dt, n = 256, 7, 0.5, 0.1, 60
    with qew.Relaxation(L, 0.3, NONE, dt=dt, seed=SEED, precision=precision) as r:
        r.set_state(cosine_profile(L, A, 2.25, k))
        r.observe([n])
        S = r.structure_factor(32)
    lam = 1.0 - 4.0 * dt * math.sin(math.pi * k / L) ** 2
    expect = A * A * lam ** (2 * n) / 4
    assert abs(S[k - 1] - expect) <= tol * expect
    assert np.max(np.delete(S, k - 1)) <= (tol * A) ** 2


def test_many_chains_and_first_modes(qew):
    """1024 chains of 2^12 (more chains than one grid row): Parseval on the full spectrum, and a
    request for the first 10 modes returns the head of it."""
    L, n_s = 1 << 12, 1024
    with qew.Relaxation(L, 1.0, RB, dt=0.1, seed=SEED, batch=n_s) as r:
        obs = r.observe([300])
        S = r.structure_factor()
        head = r.structure_factor(10)
    w2 = float(np.mean(obs["w2"][0]))
    assert abs(_parseval(S, L) - w2) <= W2_RTOL[FP32] * w2
    np.testing.assert_array_equal(head, S[:10])


def test_full_size_bench_chains(qew):
    """The bench's 4 x 2^25 chains after 200 steps: Parseval against the fused width."""
    L, n_s = 1 << 25, 4
    with qew.Relaxation(L, 0.72057, RF, dt=0.1, seed=SEED, batch=n_s) as r:
        obs = r.observe([200])
        S = r.structure_factor()
    w2 = float(np.mean(obs["w2"][0]))
    assert abs(_parseval(S, L) - w2) <= W2_RTOL[FP32] * w2


def test_errors(qew):
    with qew.Relaxation([100, 101], 1.0, RF) as r:
        with pytest.raises(qew.QewError) as e:
            r.structure_factor(5)
        assert e.value.code == -1
    with qew.Relaxation(100, 1.0, RF, batch=2) as r:
        for bad in (0, 51, -3):
            with pytest.raises(qew.QewError) as e:
                r.structure_factor(bad)
            assert e.value.code == -1
        assert r.structure_factor(50).shape == (50,)
