"""Python face of the qEW engine: a thin wrapper over the C ABI (include/qew.h).

``Relaxation`` holds one handle: a batch of periodic chains relaxing from the flat start under
explicit-Euler integration of Eq. 1 of arXiv:1211.7275 (Sec. II-III).  numpy arrays carry the
host-side arguments and results; the library owns the device state.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _capi
from ._capi import FP32_SPLIT, FP64, NONE, RB_GAUSS_CATMULLROM, RB_GAUSS_LINEAR, RB_UNIFORM_CATMULLROM, RF_GAUSS_LINEAR  # noqa: F401


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


class Relaxation:
    """A batch of chains: ``L`` (int or per-chain sequence), drive ``f`` and disorder ``kind``
    (scalars or per-chain), time step ``dt``, master ``seed``, ``precision`` (FP32_SPLIT or
    FP64).  Chain c uses sample index c unless ``set_samples`` says otherwise."""

    def __init__(self, L, f, kind=RF_GAUSS_LINEAR, dt: float = 0.1, seed: int = 12117275,
                 precision: int = FP32_SPLIT, batch: int | None = None, stream=None):
        lib = _capi.load()
        Ls = np.atleast_1d(np.asarray(L, dtype=np.int64))
        if batch is not None:
            if Ls.size != 1:
                raise ValueError("batch= needs a scalar L")
            Ls = np.full(batch, Ls[0], dtype=np.int64)
        n = Ls.size
        self.L = np.ascontiguousarray(Ls)
        self.f = np.ascontiguousarray(np.broadcast_to(np.asarray(f, np.float64), (n,)))
        self.kind = np.ascontiguousarray(np.broadcast_to(np.asarray(kind, np.int32), (n,)))
        self.dt = float(dt)
        self.seed = int(seed)
        self.precision = int(precision)
        self.n_chains = n
        h = ctypes.c_void_p()
        rc = lib.qew_create_batch(ctypes.byref(h), n, _ptr(self.L), _ptr(self.f), _ptr(self.kind), self.dt,
                                  self.seed, self.precision)
        _capi.check(rc, None)
        self._h = h
        self._lib = lib
        if stream is not None:
            self.set_stream(stream)

    # -- lifetime ------------------------------------------------------------------------------
    def close(self) -> None:
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.qew_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _check(self, rc: int) -> None:
        _capi.check(rc, self._h)

    # -- configuration -------------------------------------------------------------------------
    def set_stream(self, stream) -> None:
        """``stream``: a torch.cuda.Stream, a raw cudaStream_t integer, or None."""
        raw = getattr(stream, "cuda_stream", stream)
        self._check(self._lib.qew_set_stream(self._h, ctypes.c_void_p(raw or 0)))

    def set_precision(self, precision: int) -> None:
        self._check(self._lib.qew_set_precision(self._h, precision))
        self.precision = precision

    def set_disorder_period(self, period: int) -> None:
        """Disorder periodic in u with ``period`` (0: aperiodic); resets to the flat start."""
        self._check(self._lib.qew_set_disorder_period(self._h, int(period)))

    def set_samples(self, s) -> None:
        """Sample index (disorder realisation) of each chain; resets to the flat start."""
        s = np.ascontiguousarray(np.broadcast_to(np.asarray(s, np.uint32), (self.n_chains,)))
        self._check(self._lib.qew_set_samples(self._h, _ptr(s)))

    def set_tuning(self, tile_w: int = 0, K: int = 0, tiles_per_cta: int = 0) -> None:
        self._check(self._lib.qew_set_tuning(self._h, tile_w, K, tiles_per_cta))

    def tuning(self) -> tuple[int, int, int]:
        a, b, c = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        self._check(self._lib.qew_get_tuning(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        return a.value, b.value, c.value

    @property
    def n_sites(self) -> int:
        n = ctypes.c_int64()
        self._check(self._lib.qew_num_sites(self._h, ctypes.byref(n)))
        return n.value

    # -- dynamics ------------------------------------------------------------------------------
    def advance(self, n_steps: int) -> None:
        self._check(self._lib.qew_advance(self._h, int(n_steps)))

    def observe(self, steps) -> dict:
        """Advance through ``steps`` and return v, ubar, w2 as [n_times, n_chains] arrays."""
        st = np.ascontiguousarray(np.asarray(steps, dtype=np.int64).ravel())
        nt = st.size
        v = np.empty((nt, self.n_chains))
        ub = np.empty((nt, self.n_chains))
        w2 = np.empty((nt, self.n_chains))
        self._check(self._lib.qew_observe_ex(self._h, _ptr(st), nt, _ptr(v), _ptr(ub), _ptr(w2)))
        return {"steps": st, "v": v, "ubar": ub, "w2": w2}

    def reset(self) -> None:
        self._check(self._lib.qew_reset(self._h))

    def state(self) -> tuple[np.ndarray, int]:
        u = np.empty(self.n_sites)
        step = ctypes.c_int64()
        self._check(self._lib.qew_get_state(self._h, _ptr(u), ctypes.byref(step)))
        return u, step.value

    def cells(self) -> np.ndarray:
        c = np.empty(self.n_sites, dtype=np.int32)
        self._check(self._lib.qew_get_cells(self._h, _ptr(c)))
        return c

    def structure_factor(self, n_modes: int | None = None) -> np.ndarray:
        """S_q of Eq. 6 at q = 2 pi n / L, n = 1 .. n_modes (default L // 2), averaged over the
        chains (which must share one length)."""
        L = int(self.L[0])
        m = L // 2 if n_modes is None else int(n_modes)
        out = np.empty(max(m, 0))
        self._check(self._lib.qew_structure_factor(self._h, m, _ptr(out)))
        return out

    def enable_stats(self, on: bool = True) -> None:
        self._check(self._lib.qew_enable_stats(self._h, 1 if on else 0))

    def stats(self) -> dict:
        """Counters since the last call (see qew_get_stats); resets them."""
        a, b, d, e = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        ms = ctypes.c_double()
        self._check(self._lib.qew_get_stats(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(ms),
                                            ctypes.byref(d), ctypes.byref(e)))
        return {"launches": a.value, "fused_launches": b.value, "fused_ms": ms.value,
                "site_updates": d.value, "crossings": e.value}

    def set_state(self, u) -> None:
        u = np.ascontiguousarray(np.asarray(u, np.float64).ravel())
        if u.size != self.n_sites:
            raise ValueError("state has the wrong length")
        self._check(self._lib.qew_set_state(self._h, _ptr(u)))


def disorder_values(kind: int, precision: int, seed: int, s: int, i, n) -> np.ndarray:
    """The device generator's R(s,i,n) (RF) or V(s,i,n) (RB) in the given precision."""
    lib = _capi.load()
    i = np.ascontiguousarray(np.asarray(i, np.int64).ravel())
    n = np.ascontiguousarray(np.asarray(n, np.int64).ravel())
    out = np.empty(i.size)
    _capi.check(lib.qew_disorder_values(kind, precision, seed, s, _ptr(i), _ptr(n), i.size, _ptr(out)))
    return out


def philox_words(ctr, key) -> np.ndarray:
    """The device Philox4x32-10 block function on [n,4] counters and [n,2] keys."""
    lib = _capi.load()
    ctr = np.ascontiguousarray(np.asarray(ctr, np.uint32).reshape(-1, 4))
    key = np.ascontiguousarray(np.broadcast_to(np.asarray(key, np.uint32).reshape(-1, 2), (ctr.shape[0], 2)))
    out = np.empty_like(ctr)
    _capi.check(lib.qew_philox_words(_ptr(ctr), _ptr(key), ctr.shape[0], _ptr(out)))
    return out


def measure_alu_peaks() -> dict:
    """Measured lane-arithmetic rates of the current device (qew_measure_alu_peaks): FP32 and FP64
    FMAs per second over all lanes, Philox4x32-10 blocks per second, and the SM clock meanwhile."""
    lib = _capi.load()
    out = np.zeros(4)
    _capi.check(lib.qew_measure_alu_peaks(_ptr(out), 4))
    return {"fp32_fma_per_s": float(out[0]), "fp64_fma_per_s": float(out[1]), "philox_blocks_per_s": float(out[2]),
            "sm_mhz": float(out[3])}
