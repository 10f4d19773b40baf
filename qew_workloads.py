"""Seeded synthetic inputs for the qEW relaxation: workload presets, observation schedules
and initial states.

This module holds no arithmetic of the method (no forces, no Euler step, no observables);
both the CUDA path's tests and bench and the CPU oracle take their inputs from here.

Workloads follow the shapes the paper simulates (arXiv:1211.7275): flat start (Sec. II),
dt = 0.1 (Figs. 12-13), periodic chains up to L = 2^25 with a handful of samples (Sec. IV.D),
random-field Gaussian and random-bond disorder (Sec. IV.C).  The paper uses no external
dataset: its inputs are the simulated chains themselves, generated here from fixed seeds.
"""
from __future__ import annotations

import math

import numpy as np

SEED = 12117275          # master disorder seed of every preset
LENGTH_SEED = 7275       # host PRNG seed of the uneven-batch chain lengths

RF = 0
RB = 1
NONE = 2
RBG_LINEAR = 3   # Gaussian random bond, linear spline (Case 3 of Sec. IV.C)
RBG_CUBIC = 4    # Gaussian random bond, Catmull-Rom spline (Case 1)

# f_c^L from ``python -m paper_1211_7275_gb300.bisect`` (short-time-dynamics criterion: sign of the
# log-log slope of V(t) t^0.128 over the last decade of a 2^14-step relaxation from the flat start,
# 14 halvings of [0.5, 3.0], seed SEED, the preset's own L and batch), run on a GB300.
# f_hint is the starting guess before a bisection exists (the paper's RF value, whose disorder
# normalisation differs).
PRESETS = {
    "tiny_rf_1x1024": dict(L=1024, batch=1, kind=RF, f=1.0, dt=0.1, n_steps=10_000, n_obs=40),
    "rf_16x2^20": dict(L=1 << 20, batch=16, kind=RF, f=0.72057, f_hint=0.9713, dt=0.1, n_steps=1 << 16,
                       n_obs=60),
    "rb_1024x2^16": dict(L=1 << 16, batch=1024, kind=RB, f=0.90749, f_hint=1.0, dt=0.1, n_steps=1 << 18,
                         n_obs=80),
    # f_c^L of the 2^25-site chains themselves: the root of the gamma drift (Sec. IV.F) over the
    # last decade of 2^19-step relaxations of this preset (drift +0.025 at 0.72057, +0.0009 at
    # 0.7209, -0.020 at 0.7212), run with ``python -m paper_1211_7275_gb300.std`` on a GB300.
    "rf_4x2^25": dict(L=1 << 25, batch=4, kind=RF, f=0.7209, f_hint=0.9713, dt=0.1, n_steps=1 << 20,
                      n_obs=100),
    "uneven_256": dict(n_chains=256, kind="mixed", dt=0.1, n_steps=1 << 17, n_obs=60),
    # Case 3 at the paper's largest size (Sec. IV.D runs it at L = 2^25 and finds f_c = 1.5652 for
    # this case; with N(0,1) potential values the L = 4096 threshold here matches Table I, so the
    # paper's value is used as the drive).
    "rbg_linear_4x2^25": dict(L=1 << 25, batch=4, kind=RBG_LINEAR, f=1.5652, dt=0.1, n_steps=1 << 20,
                              n_obs=100),
    # Disorder-free chains (F_p = 0) driven at f = 0.27, which gives the random-field preset's rate of
    # cell moves (about 0.027 per site and step): the fused kernel without disorder regeneration.
    "none_16x2^20": dict(L=1 << 20, batch=16, kind=NONE, f=0.27, dt=0.1, n_steps=1 << 16, n_obs=60),
}


def preset_f(name: str) -> float:
    """Drive f of a preset: its bisected f_c^L if recorded, else its starting hint."""
    p = PRESETS[name]
    return p["f"] if p.get("f") is not None else p["f_hint"]


def log_spaced_steps(n_steps: int, k: int, include_zero: bool = True) -> np.ndarray:
    """Observation steps round(n_steps^(j/(k-1))), j = 0..k-1, deduplicated and increasing,
    ending at n_steps; step 0 (the flat start) prepended when ``include_zero``."""
    if n_steps < 1 or k < 2:
        base = [n_steps] if n_steps >= 1 else []
    else:
        base = [int(round(n_steps ** (j / (k - 1)))) for j in range(k)]
        base[-1] = n_steps
    out = sorted(set(x for x in base if x >= 1))
    if include_zero:
        out = [0] + out
    return np.asarray(out, dtype=np.int64)


def uneven_lengths(n_chains: int = 256, lo_log2: float = 12.0, hi_log2: float = 22.0,
                   seed: int = LENGTH_SEED) -> np.ndarray:
    """Chain lengths drawn log-uniformly from 2^lo .. 2^hi with a fixed host PRNG."""
    rng = np.random.default_rng(seed)
    e = rng.uniform(lo_log2, hi_log2, size=n_chains)
    return np.floor(np.exp2(e)).astype(np.int64)


def uneven_kinds(n_chains: int = 256, seed: int = LENGTH_SEED) -> np.ndarray:
    """Disorder kind per chain, random field and random bond mixed 50/50."""
    rng = np.random.default_rng(seed + 1)
    k = np.array([RF] * (n_chains // 2) + [RB] * (n_chains - n_chains // 2), dtype=np.int32)
    rng.shuffle(k)
    return k


def sweep_offsets(n_chains: int) -> np.ndarray:
    """Relative drive offsets {-2%, -1%, 0, +1%, +2%} assigned round-robin to chains."""
    off = np.array([-0.02, -0.01, 0.0, 0.01, 0.02])
    return off[np.arange(n_chains) % 5]


def cosine_profile(L: int, amplitude: float, offset: float, mode: int) -> np.ndarray:
    """u_i = offset + amplitude * cos(2 pi mode i / L), an initial state for the
    disorder-free closed-form checks."""
    i = np.arange(L, dtype=np.float64)
    return offset + amplitude * np.cos(2.0 * math.pi * mode * i / L)


def random_state(total: int, spread: float, seed: int) -> np.ndarray:
    """A rough initial state: a random walk of step size ``spread`` (float64)."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.uniform(-spread, spread, size=total))


def positive_shift(total: int, scale: float, seed: int) -> np.ndarray:
    """Non-negative per-site shifts c_i in [0, scale) for the no-passing checks."""
    rng = np.random.default_rng(seed)
    return rng.uniform(0.0, scale, size=total)


def random_points(count: int, L: int, n_lo: int, n_hi: int, seed: int) -> tuple[np.ndarray, np.ndarray]:
    """Random integer points (i, n) with 0 <= i < L and n_lo <= n < n_hi."""
    rng = np.random.default_rng(seed)
    return (rng.integers(0, L, size=count, dtype=np.int64),
            rng.integers(n_lo, n_hi, size=count, dtype=np.int64))
