"""Pins of the oracle's structure factor S_q (Eq. 6, Sec. II of arXiv:1211.7275):

    S_q(t) = mean over samples of |(1/L) sum_x u(x, t) e^{-iqx}|^2,  q = 2 pi n / L, n >= 1.

  - the double sum of Eq. 6 written out in plain Python on tiny chains (no FFT);
  - Parseval: sum over n = 1 .. L-1 of S_q equals the sample mean of w^2 (Eq. 5);
  - one cosine mode A cos(2 pi k x / L) has S = A^2 / 4 at n = k and nothing elsewhere;
  - disorder-free relaxation of that mode (the closed form of the Euler map) gives
    S = A^2 lambda_k^(2 n) / 4 after n steps, lambda_k = 1 - 4 dt sin^2(pi k / L);
  - physics: at the critical force the line becomes self-affine at short scales,
    S_q ~ q^-(1 + 2 zeta) with zeta = 1.25 (Sec. IV.A, Fig. 4), while the largest scales keep
    the memory of the flat start, a region that shrinks with time.
"""
import cmath
import json
import math
import os

import numpy as np
import pytest

from qew_workloads import SEED, cosine_profile, random_state

pytestmark = pytest.mark.filterwarnings("ignore")


def _direct(u, L):
    """Eq. 6 by its definition: for each n, (1/L) sum_x u(x) e^{-i 2 pi n x / L}, squared modulus,
    averaged over the chains."""
    rows = [u[c * L:(c + 1) * L] for c in range(len(u) // L)]
    out = []
    for n in range(1, L // 2 + 1):
        q = 2.0 * math.pi * n / L
        acc = 0.0
        for row in rows:
            z = sum(float(row[x]) * cmath.exp(-1j * q * x) for x in range(L)) / L
            acc += abs(z) ** 2
        out.append(acc / len(rows))
    return np.array(out)


@pytest.mark.parametrize("L", [2, 5, 8, 13])
def test_matches_the_defining_sum(orc, L):
    u = random_state(3 * L, 0.7, seed=L) + 40.0
    np.testing.assert_allclose(orc.structure_factor(u, L), _direct(u, L), rtol=1e-10, atol=1e-14)


@pytest.mark.parametrize("L", [64, 63])
def test_parseval_gives_the_width(orc, L):
    u = random_state(4 * L, 1.3, seed=7)
    S = orc.structure_factor(u, L)
    total = 2.0 * S.sum() - (S[-1] if L % 2 == 0 else 0.0)   # n = 1 .. L-1; n and L - n are equal
    w2 = np.mean(np.var(u.reshape(-1, L), axis=1))
    assert abs(total - w2) <= 1e-12 * max(1.0, w2)


def test_single_cosine_mode(orc):
    L, k, A = 128, 5, 0.8
    S = orc.structure_factor(cosine_profile(L, A, 3.0, k), L)
    assert abs(S[k - 1] - A * A / 4) < 1e-14
    others = np.delete(S, k - 1)
    assert np.max(others) < 1e-28


def test_disorder_free_mode_decay(orc):
    """kind NONE from a cosine profile: the mode decays by lambda_k per Euler step, so S at n = k
    is A^2 lambda_k^(2 n) / 4 (the other modes stay empty)."""
    L, k, A, dt, steps = 64, 3, 0.5, 0.1, 40
    u = orc.run(L, 0.3, dt, orc.KIND_NONE, SEED, [steps], u0=cosine_profile(L, A, 1.0, k), want_state=True)["u"]
    lam = 1.0 - 4.0 * dt * math.sin(math.pi * k / L) ** 2
    S = orc.structure_factor(u, L)
    assert abs(S[k - 1] - A * A * lam ** (2 * steps) / 4) <= 1e-13
    assert np.max(np.delete(S, k - 1)) < 1e-26


@pytest.fixture(scope="module")
def critical_spectra(orc):
    with open(os.path.join(os.path.dirname(__file__), "golden", "fc_rf_L4096.json")) as fh:
        fc = json.load(fh)["f_c"]
    L, n_s = 1024, 16
    out = {}
    for n in (500, 2000):
        u = orc.run([L] * n_s, fc, 0.1, orc.KIND_RF, SEED, [n], want_state=True)["u"]
        out[n] = orc.structure_factor(u, L)
    q = 2.0 * math.pi * np.arange(1, L // 2 + 1) / L
    return q, out


def _slope(q, S, lo, hi):
    return np.polyfit(np.log(q[lo:hi]), np.log(S[lo:hi]), 1)[0]


def test_self_affine_at_short_scales(critical_spectra):
    """1 + 2 zeta = 3.5 (Sec. IV.A): the local slope at n = 64 .. 200 after 2000 steps lies within
    the mesoscopic range the paper's effective exponents allow."""
    q, S = critical_spectra
    assert -4.0 <= _slope(q, S[2000], 64, 200) <= -2.8


def test_large_scales_remember_the_flat_start(critical_spectra):
    """Scales beyond the growing correlation length stay flat, and that region shrinks with time
    (Fig. 4): the small-q slope is shallow at 500 steps and steeper at 2000."""
    q, S = critical_spectra
    early, late = _slope(q, S[500], 4, 16), _slope(q, S[2000], 4, 16)
    assert early > -1.0
    assert late < early - 0.5
