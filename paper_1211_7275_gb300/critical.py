"""Critical force f_c^s and critical configuration of periodic L x M samples, on the GPU.

Sec. III.B of arXiv:1211.7275 defines them for a sample periodic in x (length L) and in u (period
M): the pinned configuration with the largest drive in the long-time dynamics.  This module
finds them by bisection on f, for a batch of samples at once; every relaxation runs in the
library (FP64 path by default, through the C ABI).  A trial force f starts from the pinned
configuration u_lo of the largest force known to pin.  There every velocity equals
f - f_lo > 0, and the Euler map keeps the order of configurations (Middleton's no-passing), so
the line only moves forward.  The trial then either
  - pins: the chain's mean velocity falls below ``v_tol``, so f <= f_c^s, and the state becomes
    the new u_lo; or
  - runs away: every site passes u_lo + M.  The disorder repeats with period M, so from there
    the motion repeats one period higher, forever: no pinned configuration exists, and
    f > f_c^s.
Each sample keeps its own bracket; chains that have decided keep moving until the batch has
decided, and their state at the decision is the one kept.

For the random field (linear interpolation, Case 4) ``exact_critical_force`` computes f_c^s
without bisection: the library follows the pinned configuration exactly while f grows (with the
cells fixed the static equation is linear) and the dynamics only through the avalanches where a
pinned branch ends (qew_critical_force_rf).

Run: python -m paper_1211_7275_gb300.critical --L 1024 --M 1024 --samples 16 [--exact]
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import relax as _relax

PINNED, MOVING = 1, 2


def _relax_batch(L: int, M: int, kind: int, f: np.ndarray, u0: np.ndarray, *, seed: int, dt: float, chunk: int,
                 max_steps: int, v_tol: float, precision: int):
    B = f.shape[0]
    status = np.zeros(B, dtype=np.int32)
    u = u0.copy()
    with _relax.Relaxation(np.full(B, L), f, kind, dt=dt, seed=seed, precision=precision) as r:
        r.set_disorder_period(M)
        r.set_state(u0.ravel())
        t = 0
        while t < max_steps and np.any(status == 0):
            t += chunk
            obs = r.observe([t])
            now, _ = r.state()
            now = now.reshape(B, L)
            open_ = status == 0
            moving = open_ & (np.min(now - u0, axis=1) >= M)
            pinned = open_ & ~moving & (np.abs(obs["v"][0]) < v_tol)
            status[moving] = MOVING
            status[pinned] = PINNED
            u[moving | pinned] = now[moving | pinned]
    return status, u


def critical_forces(L: int, M: int, kind: int, n_samples: int, *, seed: int = 12117275, f_start: float = 0.0,
                    f_hi: float = 3.0, tol: float = 1e-4, dt: float = 0.1, chunk: int = 2000,
                    max_steps: int = 1_000_000, v_tol: float = 1e-12, precision: int = _relax.FP64) -> dict:
    """f_c^s of samples 0 .. n_samples-1 (chain c uses sample index c) with their brackets and
    critical configurations [n_samples, L]."""
    B = int(n_samples)
    kw = dict(seed=seed, dt=dt, chunk=chunk, max_steps=max_steps, v_tol=v_tol, precision=precision)
    status, u_lo = _relax_batch(L, M, kind, np.full(B, float(f_start)), np.zeros((B, L)), **kw)
    if np.any(status != PINNED):
        raise RuntimeError(f"samples {np.where(status != PINNED)[0].tolist()} do not pin at f = {f_start}")
    lo = np.full(B, float(f_start))
    hi = np.full(B, float(f_hi))
    while np.any(hi - lo > tol):
        mid = 0.5 * (lo + hi)
        status, u = _relax_batch(L, M, kind, mid, u_lo, **kw)
        if np.any(status == 0):
            raise RuntimeError(f"no decision within {max_steps} steps for samples {np.where(status == 0)[0].tolist()}")
        active = hi - lo > tol
        up = active & (status == MOVING)
        down = active & (status == PINNED)
        hi[up] = mid[up]
        lo[down] = mid[down]
        u_lo[down] = u[down]
    return {"f_c": 0.5 * (lo + hi), "lo": lo, "hi": hi, "u_c": u_lo, "L": L, "M": M, "kind": kind, "tol": tol}


def exact_critical_force(L: int, M: int, s: int = 0, *, seed: int = 12117275, R: np.ndarray | None = None,
                         dt: float = 0.1, f_start: float = 0.0) -> dict:
    """f_c^s and the critical configuration of random-field sample ``s`` (L x M, periodic in u),
    by the library's exact branch-following search.  The force values R(i, n mod M) come from the
    device generator in FP64 (qew_disorder_values), unless ``R`` [L, M] is given."""
    import ctypes

    from . import _capi
    lib = _capi.load()
    if R is None:
        i = np.repeat(np.arange(L, dtype=np.int64), M)
        n = np.tile(np.arange(M, dtype=np.int64), L)
        R = _relax.disorder_values(_relax.RF_GAUSS_LINEAR, _relax.FP64, seed, s, i, n).reshape(L, M)
    R = np.ascontiguousarray(R, dtype=np.float64)
    if R.shape != (L, M):
        raise ValueError("R must have shape (L, M)")
    fc = ctypes.c_double()
    ev = ctypes.c_int64()
    steps = ctypes.c_int64()
    u = np.empty(L)
    rc = lib.qew_critical_force_rf(L, M, R.ctypes.data_as(ctypes.c_void_p), dt, f_start, ctypes.byref(fc),
                                   u.ctypes.data_as(ctypes.c_void_p), ctypes.byref(ev), ctypes.byref(steps))
    _capi.check(rc)
    return {"f_c": fc.value, "u_c": u, "events": ev.value, "dyn_steps": steps.value, "L": L, "M": M}


def exact_critical_forces(L: int, M: int, n_samples: int, *, seed: int = 12117275, dt: float = 0.1,
                          f_start: float = 0.0, threads: int | None = None) -> dict:
    """f_c^s and critical configurations of random-field samples 0 .. n_samples-1 by the exact
    search, one host thread per sample (the force tables come from the device generator first)."""
    import concurrent.futures as cf
    import os

    i = np.repeat(np.arange(L, dtype=np.int64), M)
    n = np.tile(np.arange(M, dtype=np.int64), L)
    tables = [_relax.disorder_values(_relax.RF_GAUSS_LINEAR, _relax.FP64, seed, s, i, n).reshape(L, M)
              for s in range(n_samples)]
    workers = threads or min(n_samples, os.cpu_count() or 1)
    with cf.ThreadPoolExecutor(max_workers=max(1, workers)) as ex:
        res = list(ex.map(lambda s: exact_critical_force(L, M, s, seed=seed, R=tables[s], dt=dt, f_start=f_start),
                          range(n_samples)))
    return {"f_c": np.array([r["f_c"] for r in res]), "u_c": np.stack([r["u_c"] for r in res]), "L": L, "M": M,
            "events": [r["events"] for r in res], "dyn_steps": [r["dyn_steps"] for r in res]}


def main() -> None:
    p = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    p.add_argument("--L", type=int, required=True)
    p.add_argument("--M", type=int, required=True)
    p.add_argument("--kind", type=int, default=0)
    p.add_argument("--samples", type=int, default=8)
    p.add_argument("--tol", type=float, default=1e-4)
    p.add_argument("--exact", action="store_true", help="exact branch-following search (random field only)")
    a = p.parse_args()
    t0 = time.time()
    if a.exact:
        if a.kind != 0:
            raise SystemExit("--exact needs the random field (kind 0)")
        fcs = exact_critical_forces(a.L, a.M, a.samples)["f_c"].tolist()
        out = {"f_c": fcs, "mean": float(np.mean(fcs)), "L": a.L, "M": a.M, "method": "exact",
               "sem": float(np.std(fcs, ddof=1) / np.sqrt(a.samples)) if a.samples > 1 else None,
               "seconds": time.time() - t0}
        print(json.dumps(out))
        return
    res = critical_forces(a.L, a.M, a.kind, a.samples, tol=a.tol)
    out = {k: (v.tolist() if isinstance(v, np.ndarray) and k != "u_c" else v) for k, v in res.items() if k != "u_c"}
    out["mean"] = float(np.mean(res["f_c"]))
    out["sem"] = float(np.std(res["f_c"], ddof=1) / np.sqrt(a.samples)) if a.samples > 1 else None
    out["seconds"] = time.time() - t0
    print(json.dumps(out))


if __name__ == "__main__":
    main()
