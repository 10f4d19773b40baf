"""Short-time-dynamics (STD) analysis of relaxation observables (arXiv:1211.7275, Sec. IV.B-E).

Host-side post-processing of the sample-averaged V(t) and W2(t) that a relaxation records:

  gamma(t)           gamma = w / (t v), w = sqrt(W2): constant in the critical scaling regime
                     (Sec. IV.C, from beta = nu (z - zeta)), decaying above f_c and growing
                     below it (Sec. IV.F).
  corrected          A t^e [1 + (t / t_c)^-alpha]: the corrected forms of w(t) (e = zeta/z) and
                     v(t) (e = -beta/nu z), and of gamma(t) with e = 0 (Sec. IV.D).
  fit_corrected      least-squares fit of that form to ln y for t >= t_mic (procedure (a) of
                     Sec. IV.E).
  fit_power          a pure power law A t^e on [t_lo, t_hi] (log-log least squares).
  plateau_fits       exponents of pure power laws fitted for t >= t_plat, for each t_plat
                     (procedure (b)).
  window_fits        exponents of pure power laws fitted on [t0, 4 t0], for each t0 (procedure (c)).
  gamma_drift        the log-log slope of gamma over the last decade of t: the sign of the
                     departure from f_c (gamma leaves its plateau downwards above f_c and upwards
                     below it, Sec. IV.F).

The functions take plain arrays (times t = step * dt, and V, W2 averaged over samples), so they
apply equally to the CUDA path's observables and to the oracle's.
"""
from __future__ import annotations

import math

import numpy as np


def gamma(t, V, W2) -> np.ndarray:
    """gamma(t) = w / (t v) with w = sqrt(W2) (Sec. IV.C)."""
    t, V, W2 = (np.asarray(a, dtype=np.float64) for a in (t, V, W2))
    return np.sqrt(W2) / (t * V)


def corrected(t, A: float, e: float, t_c: float, alpha: float) -> np.ndarray:
    """A t^e [1 + (t / t_c)^-alpha] (the corrected scaling forms of Sec. IV.D)."""
    t = np.asarray(t, dtype=np.float64)
    return A * t ** e * (1.0 + (t / t_c) ** (-alpha))


def fit_corrected(t, y, t_mic: float = 1.0, t_max: float | None = None, exponent: float | None = None,
                  p0: tuple | None = None) -> dict:
    """Fit A t^e [1 + (t/t_c)^-alpha] to y over t_mic <= t <= t_max (least squares on ln y).
    ``exponent`` fixes e (0 for gamma(t)).  Returns A, e, t_c, alpha and the rms residual of ln y."""
    from scipy.optimize import curve_fit

    t = np.asarray(t, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    sel = (t >= t_mic) & (y > 0) & np.isfinite(y)
    if t_max is not None:
        sel &= t <= t_max
    tt, ly = t[sel], np.log(y[sel])
    if tt.size < 5:
        raise ValueError("need at least 5 points in the fit range")
    slope = np.polyfit(np.log(tt), ly, 1)[0]

    def model(x, la, e, ltc, al):
        return la + e * np.log(x) + np.log1p((x / math.exp(ltc)) ** (-al))

    if exponent is None:
        f = model
        start = p0 or (ly[-1] - slope * math.log(tt[-1]), slope, math.log(max(t_mic, 0.1)), 0.7)
    else:
        def f(x, la, ltc, al):
            return model(x, la, exponent, ltc, al)
        start = p0 or (ly[-1] - exponent * math.log(tt[-1]), math.log(max(t_mic, 0.1)), 0.7)
    p, _ = curve_fit(f, tt, ly, p0=start, maxfev=50000)
    if exponent is None:
        la, e, ltc, al = p
    else:
        (la, ltc, al), e = p, exponent
    resid = ly - model(tt, la, e, ltc, al)
    return {"A": math.exp(la), "e": float(e), "t_c": math.exp(ltc), "alpha": float(al),
            "rms_log_residual": float(np.sqrt(np.mean(resid ** 2))), "t_range": [float(tt[0]), float(tt[-1])]}


def fit_power(t, y, t_lo: float, t_hi: float | None = None) -> tuple[float, float]:
    """A pure power law A t^e fitted to y on [t_lo, t_hi] by log-log least squares: (A, e)."""
    t = np.asarray(t, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    sel = (t >= t_lo) & (y > 0)
    if t_hi is not None:
        sel &= t <= t_hi
    if np.count_nonzero(sel) < 2:
        raise ValueError("need at least 2 points in the fit window")
    e, la = np.polyfit(np.log(t[sel]), np.log(y[sel]), 1)
    return math.exp(la), float(e)


def plateau_fits(t, y, t_plats) -> np.ndarray:
    """Exponent of the pure power law fitted for t >= t_plat, for each t_plat (Sec. IV.E (b))."""
    return np.array([fit_power(t, y, tp)[1] for tp in t_plats])


def window_fits(t, y, t0s) -> np.ndarray:
    """Exponent of the pure power law fitted on [t0, 4 t0], for each t0 (Sec. IV.E (c))."""
    return np.array([fit_power(t, y, t0, 4.0 * t0)[1] for t0 in t0s])


def gamma_drift(t, V, W2, decades: float = 1.0) -> float:
    """Log-log slope of gamma(t) over the last ``decades`` of t: negative above f_c (v saturates
    while w keeps growing slower than t), positive below it (v collapses)."""
    t = np.asarray(t, dtype=np.float64)
    g = gamma(t, V, W2)
    sel = (t >= t[-1] / 10.0 ** decades) & np.isfinite(g) & (g > 0)
    if np.count_nonzero(sel) < 2:
        raise ValueError("need at least 2 points in the last decade")
    return float(np.polyfit(np.log(t[sel]), np.log(g[sel]), 1)[0])


def _main() -> None:
    """Relax a batch on the GPU and print its STD analysis as one JSON line:
    python -m paper_1211_7275_gb300.std --L 33554432 --batch 4 --f 1.5652 --kind 3 --steps 1048576"""
    import argparse
    import json

    from . import relax

    p = argparse.ArgumentParser(description=_main.__doc__)
    p.add_argument("--L", type=int, required=True)
    p.add_argument("--batch", type=int, default=1)
    p.add_argument("--f", type=float, required=True)
    p.add_argument("--kind", type=int, default=0, help="0 RF, 1 uniform RB, 3 Gaussian RB linear, 4 Gaussian RB cubic")
    p.add_argument("--dt", type=float, default=0.1)
    p.add_argument("--seed", type=int, default=12117275)
    p.add_argument("--steps", type=int, required=True)
    p.add_argument("--obs", type=int, default=100, help="log-spaced observation steps")
    p.add_argument("--tuning", default="auto", help="'auto' or tile_w,K,tiles_per_cta")
    p.add_argument("--t-mic", type=float, default=2.0, help="lower end of the corrected fits (procedure (a))")
    a = p.parse_args()
    k = a.obs
    steps = sorted({0} | {int(round(a.steps ** (j / (k - 1)))) for j in range(k)} | {a.steps})
    steps = np.asarray([s for s in steps if s >= 1], dtype=np.int64)
    with relax.Relaxation(a.L, a.f, a.kind, dt=a.dt, seed=a.seed, batch=a.batch) as r:
        r.set_tuning(*([0, 0, 0] if a.tuning == "auto" else [int(x) for x in a.tuning.split(",")]))
        obs = r.observe(steps)
    t = steps * a.dt
    V, W2 = obs["v"].mean(1), obs["w2"].mean(1)
    W = np.sqrt(W2)
    t0s = [x for x in (10, 30, 100, 300, 1000, 3000, 10000, 25000) if 4 * x <= t[-1]]
    out = {"L": a.L, "batch": a.batch, "f": a.f, "kind": a.kind, "steps": a.steps, "observations": int(steps.size),
           "beta_over_nu_z": -fit_corrected(t, V, t_mic=a.t_mic)["e"],
           "zeta_over_z": fit_corrected(t, W, t_mic=a.t_mic)["e"],
           "window_t0": t0s, "window_v": window_fits(t, V, t0s).tolist(), "window_w": window_fits(t, W, t0s).tolist(),
           "gamma_drift_last_decade": gamma_drift(t, V, W2)}
    print(json.dumps(out))


if __name__ == "__main__":
    _main()
