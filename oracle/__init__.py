"""FP64 CPU oracle for the qEW explicit-Euler relaxation (arXiv:1211.7275, Sec. II-III).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import this package.  The product library never loads it, and it
shares no code with the CUDA path: the arithmetic lives in ``qew_oracle.c`` (plain C, FP64,
no fused multiply-add) and this module marshals numpy arrays through ctypes, except for the
structure factor, which is numpy's FFT and a mean of squared moduli.

Functions and the passages they follow:
  philox4x32_10      Philox4x32-10 block function (Salmon et al., SC'11); the paper does not
                     name its generator (Sec. III.B), this is the reading used throughout.
  disorder_values    R(s,i,n) ~ N(0,1) (RF), V(s,i,n) ~ U(-1,1) (RB) or G(s,i,n) ~ N(0,1)
                     (Gaussian RB, Cases 1 and 3) drawn at integer (i,n), Sec. III.B and the
                     disorder cases of Sec. IV.C; optionally periodic in n with period M (the
                     L x M system of Sec. III.B).
  pinning_force      F_p(i,u): linear interpolation of R (RF), -dV/du of the Catmull-Rom
                     spline through V (RB) or G (Case 1), or -dV/du of the linear spline
                     through G (Case 3), Sec. III.B and Sec. IV.C.
  rb_potential       the RB spline potential itself (spline pins only).
  run                Euler integration of Eq. 1 (eta = c = 1, periodic in x, Sec. III.B) from
                     the flat start (Sec. II) or a given state, with v, ubar, w2 of Eqs. 3-5;
                     ``node_f32=True`` runs the same FP64 dynamics with every disorder value
                     rounded to FP32 (the floor of any FP32 store of the disorder).
  lightcone          the same dynamics evaluated on a window of 2n+w sites, exact for the
                     w central sites after n steps (stencil radius 1).
  structure_factor   S_q of Eq. 6 (Sec. II): the sample mean of |(1/L) sum_x u(x) e^{-iqx}|^2
                     at q = 2 pi n / L, n = 1 .. L/2, by a real FFT of each chain.
  critical_force     f_c^s of a periodic L x M sample (Sec. III.B): the largest drive with a
                     pinned configuration in the long-time dynamics, by bisection on f.

Parity of every function is pinned by ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

KIND_RF = 0
KIND_RB = 1
KIND_NONE = 2
KIND_RBG_LINEAR = 3   # Case 3: Gaussian potential, linear spline (force constant per cell)
KIND_RBG_CUBIC = 4    # Case 1: Gaussian potential, Catmull-Rom spline

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qew_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``qew_oracle.c`` into ``oracle/liboracle.so`` (gcc, FP64, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
               "-o", tmp, _SRC, "-lm", "-lpthread"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            lib.oracle_philox4x32_10.argtypes = [P, P, ctypes.c_int64, P]
            lib.oracle_philox4x32_10.restype = None
            lib.oracle_disorder_values.argtypes = [ctypes.c_int, ctypes.c_uint64, ctypes.c_uint32, P, P,
                                                   ctypes.c_int64, P, ctypes.c_int64]
            lib.oracle_disorder_values.restype = None
            lib.oracle_pinning_force.argtypes = [ctypes.c_int, ctypes.c_uint64, ctypes.c_uint32, P, P,
                                                 ctypes.c_int64, P, ctypes.c_int64]
            lib.oracle_pinning_force.restype = None
            lib.oracle_rb_potential.argtypes = [ctypes.c_int, ctypes.c_uint64, ctypes.c_uint32, P, P,
                                                ctypes.c_int64, P, ctypes.c_int64]
            lib.oracle_rb_potential.restype = None
            lib.oracle_run.argtypes = [ctypes.c_int32, P, P, P, P, ctypes.c_double, ctypes.c_uint64, P, P,
                                       ctypes.c_int32, P, P, P, P, ctypes.c_int32, ctypes.c_int64,
                                       ctypes.c_int32]
            lib.oracle_run.restype = ctypes.c_int
            lib.oracle_lightcone.argtypes = [ctypes.c_int64, ctypes.c_uint32, ctypes.c_double, ctypes.c_double,
                                             ctypes.c_int, ctypes.c_uint64, ctypes.c_int64, ctypes.c_int64,
                                             ctypes.c_int64, P, P, ctypes.c_int64]
            lib.oracle_lightcone.restype = ctypes.c_int
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def philox4x32_10(ctr, key) -> np.ndarray:
    """Philox4x32-10 blocks: ``ctr`` [n,4] uint32, ``key`` [n,2] uint32 -> [n,4] uint32."""
    ctr = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    key = np.ascontiguousarray(key, dtype=np.uint32).reshape(-1, 2)
    if key.shape[0] == 1 and ctr.shape[0] > 1:
        key = np.ascontiguousarray(np.broadcast_to(key, (ctr.shape[0], 2)))
    out = np.empty_like(ctr)
    _load().oracle_philox4x32_10(_p(ctr), _p(key), ctr.shape[0], _p(out))
    return out


def disorder_values(kind: int, seed: int, s: int, i, n, period: int = 0) -> np.ndarray:
    """R(s,i,n) for RF, V(s,i,n) for RB, G(s,i,n) for the Gaussian RB kinds, at integer (i, n)
    (n taken mod ``period`` when it is positive)."""
    i = np.ascontiguousarray(i, dtype=np.int64).ravel()
    n = np.ascontiguousarray(n, dtype=np.int64).ravel()
    out = np.empty(i.shape[0], np.float64)
    _load().oracle_disorder_values(kind, seed, s, _p(i), _p(n), i.shape[0], _p(out), period)
    return out


def pinning_force(kind: int, seed: int, s: int, i, u, period: int = 0) -> np.ndarray:
    """F_p(i, u) of chain ``s`` for each (i, u) pair."""
    i = np.ascontiguousarray(i, dtype=np.int64).ravel()
    u = np.ascontiguousarray(u, dtype=np.float64).ravel()
    out = np.empty(i.shape[0], np.float64)
    _load().oracle_pinning_force(kind, seed, s, _p(i), _p(u), i.shape[0], _p(out), period)
    return out


def rb_potential(seed: int, s: int, i, u, kind: int = KIND_RB, period: int = 0) -> np.ndarray:
    """RB potential V(i, u) of chain ``s``: Catmull-Rom (RB, Case 1) or linear (Case 3)."""
    i = np.ascontiguousarray(i, dtype=np.int64).ravel()
    u = np.ascontiguousarray(u, dtype=np.float64).ravel()
    out = np.empty(i.shape[0], np.float64)
    _load().oracle_rb_potential(kind, seed, s, _p(i), _p(u), i.shape[0], _p(out), period)
    return out


def run(L, f, dt: float, kind, seed: int, steps, *, s=None, u0=None, n_threads: int = 0,
        want_state: bool = False, period: int = 0, node_f32: bool = False) -> dict:
    """Relax independent periodic chains and observe them at ``steps``.

    ``L``, ``f``, ``kind`` and ``s`` are per-chain sequences (scalars broadcast); ``s``
    defaults to 0..n_chains-1.  ``u0`` is the concatenated initial state (default: flat).
    Returns ``v``, ``ubar``, ``w2`` as [n_times, n_chains] and, with ``want_state``, the
    concatenated final state ``u``.  ``period`` > 0 makes the disorder periodic in u with that
    period (the L x M system of Sec. III.B).  ``node_f32`` rounds every disorder value to FP32
    before it enters the force (the FP32 node model; the dynamics stays FP64).
    """
    L = np.atleast_1d(np.asarray(L, dtype=np.int64))
    n_chains = L.shape[0]
    f = np.ascontiguousarray(np.broadcast_to(np.asarray(f, np.float64), (n_chains,)))
    kind = np.ascontiguousarray(np.broadcast_to(np.asarray(kind, np.int32), (n_chains,)))
    s = np.arange(n_chains, dtype=np.uint32) if s is None else np.ascontiguousarray(
        np.broadcast_to(np.asarray(s, np.uint32), (n_chains,)))
    L = np.ascontiguousarray(L)
    steps = np.ascontiguousarray(np.asarray(steps, dtype=np.int64).ravel())
    nt = steps.shape[0]
    v = np.empty((nt, n_chains))
    ub = np.empty((nt, n_chains))
    w2 = np.empty((nt, n_chains))
    total = int(L.sum())
    u_in = None
    if u0 is not None:
        u_in = np.ascontiguousarray(np.asarray(u0, np.float64).ravel())
        if u_in.shape[0] != total:
            raise ValueError("u0 has the wrong length")
    u_out = np.empty(total) if want_state else None
    rc = _load().oracle_run(n_chains, _p(L), _p(s), _p(f), _p(kind), dt, seed,
                            _p(u_in) if u_in is not None else None, _p(steps), nt,
                            _p(v), _p(ub), _p(w2), _p(u_out) if u_out is not None else None, n_threads,
                            int(period), 1 if node_f32 else 0)
    if rc != 0:
        raise ValueError(f"oracle_run failed with status {rc}")
    out = {"v": v, "ubar": ub, "w2": w2}
    if want_state:
        out["u"] = u_out
    return out


def lightcone(L: int, s: int, f: float, dt: float, kind: int, seed: int, i0: int, w: int,
              n_steps: int, period: int = 0) -> tuple[np.ndarray, np.ndarray]:
    """u and F_p at sites i0..i0+w-1 (mod L) of chain ``s`` after ``n_steps`` from the flat start."""
    u = np.empty(w)
    F = np.empty(w)
    rc = _load().oracle_lightcone(L, s, f, dt, kind, seed, i0, w, n_steps, _p(u), _p(F), int(period))
    if rc != 0:
        raise ValueError(f"oracle_lightcone failed with status {rc}")
    return u, F


def structure_factor(u, L: int, n_modes: int | None = None) -> np.ndarray:
    """S_q of Eq. 6 for the chains of length ``L`` concatenated in ``u``: the mean over chains of
    |(1/L) sum_x u(x) e^{-iqx}|^2 at q = 2 pi n / L for n = 1 .. n_modes (default L // 2).  Modes
    n and L - n are equal for a real line, so n = 1 .. L/2 carry all of it."""
    u = np.asarray(u, dtype=np.float64).reshape(-1, L)
    m = L // 2 if n_modes is None else int(n_modes)
    if not 1 <= m <= L // 2:
        raise ValueError("n_modes must lie in [1, L/2]")
    z = np.fft.rfft(u, axis=1)[:, 1:m + 1] / L
    return np.mean(z.real ** 2 + z.imag ** 2, axis=0)


def critical_force(L: int, M: int, kind: int, seed: int, s: int = 0, *, f_hi: float = 3.0, tol: float = 1e-4,
                   dt: float = 0.1, chunk: int = 2000, max_steps: int = 1_000_000, v_tol: float = 1e-12,
                   f_start: float = 0.0) -> dict:
    """Critical force f_c^s and critical configuration of the periodic L x M sample ``s`` (Sec. III.B:
    the pinned configuration with the largest drive in the long-time dynamics), by bisection on f.

    A trial force f starts from the pinned configuration u_lo of the largest force f_lo known to
    pin.  There every velocity equals f - f_lo > 0, and the Euler map keeps the order of
    configurations (Middleton's no-passing), so the line only moves forward.  It either
      - pins: the mean velocity falls below ``v_tol``; f <= f_c^s and the pinned state becomes
        u_lo; or
      - runs away: every site passes u_lo + M.  The disorder repeats with period M, so from there
        the line repeats its motion one period higher, forever: no pinned configuration exists,
        and f > f_c^s.
    The first u_lo is the state the line relaxes to at f = f_start (below f_c^s) from the flat
    start.  Returns f_c^s (the bracket's midpoint), the bracket and the critical configuration u_lo.
    """
    def relax(f: float, u0: np.ndarray):
        u, t = u0.copy(), 0
        while t < max_steps:
            r = run([L], f, dt, kind, seed, [0, chunk], s=[s], u0=u, want_state=True, period=M)
            u, t = r["u"], t + chunk
            if np.min(u - u0) >= M:
                return "moving", u
            if abs(r["v"][-1, 0]) < v_tol:
                return "pinned", u
        return "undecided", u

    state, u_lo = relax(f_start, np.zeros(L))
    if state != "pinned":
        raise RuntimeError(f"the flat line does not pin at f = {f_start} ({state})")
    lo, hi = float(f_start), float(f_hi)
    while hi - lo > tol:
        mid = 0.5 * (lo + hi)
        state, u = relax(mid, u_lo)
        if state == "moving":
            hi = mid
        elif state == "pinned":
            lo, u_lo = mid, u
        else:
            raise RuntimeError(f"no decision at f = {mid} within {max_steps} steps")
    return {"f_c": 0.5 * (lo + hi), "bracket": [lo, hi], "u_c": u_lo}
