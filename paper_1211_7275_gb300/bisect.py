"""Finite-size critical force f_c^L by bisection on the relaxation from the flat start.

Short-time dynamics criterion (arXiv:1211.7275, Sec. III.A): at f_c the velocity decays as a power
law v ~ t^{-beta/(nu z)}; above f_c it saturates, below it collapses.  Each trial relaxes a batch of
chains on the GPU and fits, over the last decade of t, either
  - "v" (default): the log-log slope of V(t) t^{beta/(nu z)} (beta/(nu z) = 0.128, Sec. IV.E); a
    slope >= 0 means f is above f_c^L; or
  - "gamma": the log-log slope of gamma = w / (t v) (Sec. IV.C, IV.F), which needs no exponent; a
    slope <= 0 means f is above f_c^L.
Ties count as above.  All the control is on the host; every trial is one GPU relaxation through
the C ABI.
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import relax as _relax
from . import std as _std

BETA_NU_Z = 0.128


def log_steps(n_steps: int, k: int = 30) -> np.ndarray:
    s = sorted(set(int(round(n_steps ** (j / (k - 1)))) for j in range(k)) | {n_steps})
    return np.asarray([x for x in s if x >= 1], dtype=np.int64)


def drift(f: float, L: int, batch: int, kind: int, n_steps: int, dt: float = 0.1, seed: int = 12117275,
          tuning=None, criterion: str = "v") -> float:
    """Positive (or zero) when f is above f_c^L, negative below, by the chosen criterion."""
    steps = log_steps(n_steps)
    with _relax.Relaxation(L, f, kind, dt=dt, seed=seed, batch=batch) as r:
        if tuning:
            r.set_tuning(*tuning)
        out = r.observe(steps)
    V = out["v"].mean(axis=1)
    t = steps * dt
    sel = t >= t[-1] / 10
    if np.any(V[sel] <= 0):
        return -math.inf
    if criterion == "gamma":
        return -_std.gamma_drift(t, V, out["w2"].mean(axis=1))
    return float(np.polyfit(np.log(t[sel]), np.log(V[sel] * t[sel] ** BETA_NU_Z), 1)[0])


def bisect(L: int, batch: int, kind: int, n_steps: int, lo: float = 0.5, hi: float = 3.0, iters: int = 15,
           **kw) -> dict:
    hist = []
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        d = drift(mid, L, batch, kind, n_steps, **kw)
        hist.append((mid, d))
        if d >= 0:
            hi = mid
        else:
            lo = mid
    return {"f_c": 0.5 * (lo + hi), "bracket": [lo, hi], "history": hist, "L": L, "batch": batch, "kind": kind,
            "n_steps": n_steps, "criterion": kw.get("criterion", "v"), "beta_over_nu_z": BETA_NU_Z}


def main() -> None:
    p = argparse.ArgumentParser(description=__doc__)
    p.add_argument("--L", type=int, required=True)
    p.add_argument("--batch", type=int, default=4)
    p.add_argument("--kind", type=int, default=0)
    p.add_argument("--n-steps", type=int, default=1 << 14)
    p.add_argument("--lo", type=float, default=0.5)
    p.add_argument("--hi", type=float, default=3.0)
    p.add_argument("--iters", type=int, default=15)
    p.add_argument("--criterion", choices=["v", "gamma"], default="v")
    a = p.parse_args()
    t0 = time.time()
    res = bisect(a.L, a.batch, a.kind, a.n_steps, a.lo, a.hi, a.iters, criterion=a.criterion)
    res["seconds"] = time.time() - t0
    print(json.dumps(res))


if __name__ == "__main__":
    main()
