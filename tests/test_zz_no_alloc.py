"""The allocation-free observation entry point, qew_observe_state_noalloc, checked against the
handle-based qew_observe_ex on the same state, and against the CPU oracle.

Some callers cannot let a library call cudaMalloc.  One example is a framework whose caching
allocator already holds the GPU's memory, where an allocation behind its back can fail or
fragment the pool.  Another is a time-critical loop that must not take the device-wide
synchronisation that cudaMalloc/cudaFree can cause.  For them the library computes the
observables of a state that the caller keeps in device memory, using a fixed scratch array
inside the library instead of allocating.  Here a handle relaxes a batch of chains and reports
v, ubar and w2 at its last observation step.  The same state, copied into caller-owned device
buffers, goes through the allocation-free entry point twice in a row.  Both calls must agree
with the handle within the tolerances the parity tests use for these observables, and with the
oracle's v, ubar and w2 of that state (Eqs. 3-5, FP64 and the exact disorder values) within
what the FP32 disorder values and sums allow.  Every disorder kind is covered, and a batch of
more than 64 chains, which the entry point copies back in several chunks.  Oversized inputs must
be rejected.
"""
import ctypes

import numpy as np
import pytest

from qew_workloads import SEED, random_state

pytestmark = pytest.mark.gpu


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


@pytest.mark.parametrize("kind,f,L,batch,base", [(0, 0.72057, 5000, 3, None), (1, 0.90749, 3001, 2, None),
                                                 (2, 0.4, 700, 1, None), (3, 1.5652, 2049, 2, None),
                                                 (4, 1.9, 1500, 2, None), (0, 0.9, 300, 70, None),
                                                 (0, 1.0, 3000, 2, 2.0 ** 29 + 0.25), (1, 1.9, 2000, 2, -(2.0 ** 29) - 0.75)])
def test_noalloc_matches_observe(orc, kind, f, L, batch, base):
    """``base``: the chains start from a rough line around that height instead of the flat line
    (cells near +-2^29: the sums are taken relative to each chain's first cell)."""
    torch = pytest.importorskip("torch")
    import paper_1211_7275_gb300 as q
    lib = q.load()
    steps = [0, 37, 300]
    with q.Relaxation(L, f, kind, dt=0.1, seed=SEED, batch=batch) as r:
        if base is not None:
            r.set_state(base + random_state(L * batch, 0.5, seed=41))
        obs = r.observe(steps)
        u, _ = r.state()
        cells = r.cells()
    off = (u - cells).astype(np.float32)   # exact: u = n + d with d stored in FP32
    ref = orc.run([L] * batch, f, 0.1, kind, SEED, [0], u0=u)
    cell_d = torch.from_numpy(np.ascontiguousarray(cells)).cuda()
    off_d = torch.from_numpy(np.ascontiguousarray(off)).cuda()
    stream = torch.cuda.current_stream()
    for _ in range(2):
        v = np.full(batch, np.nan)
        ub = np.full(batch, np.nan)
        w2 = np.full(batch, np.nan)
        rc = lib.qew_observe_state_noalloc(ctypes.c_void_p(cell_d.data_ptr()), ctypes.c_void_p(off_d.data_ptr()), L,
                                           batch, f, kind, SEED, ctypes.c_void_p(stream.cuda_stream), _p(v), _p(ub),
                                           _p(w2))
        assert rc == 0, lib.qew_last_error(None)
        np.testing.assert_allclose(v, obs["v"][-1], rtol=0, atol=2e-4)
        np.testing.assert_allclose(ub, obs["ubar"][-1], rtol=0, atol=2e-5)
        np.testing.assert_allclose(w2, obs["w2"][-1], rtol=1e-4, atol=1e-6)
        # the oracle on the same state: FP32 disorder values (relative error 6e-7 for the Gaussian
        # kinds, cubic coefficients up to ~20) and FP32 tile sums
        np.testing.assert_allclose(v, ref["v"][0], rtol=0, atol=2e-5)
        np.testing.assert_allclose(ub, ref["ubar"][0], rtol=0, atol=2e-6 * max(1.0, np.abs(ub).max()))
        np.testing.assert_allclose(w2, ref["w2"][0], rtol=2e-5, atol=1e-8)


def test_noalloc_rejects_oversized_input():
    torch = pytest.importorskip("torch")
    import paper_1211_7275_gb300 as q
    lib = q.load()
    buf = torch.zeros(16, dtype=torch.int32, device="cuda")
    ptr = ctypes.c_void_p(buf.data_ptr())
    v = np.zeros(8)
    # 2^24 + 1 sites in one chain needs one tile more than the fixed scratch holds
    rc = lib.qew_observe_state_noalloc(ptr, ptr, (1 << 24) + 1, 1, 1.0, 0, SEED, None, _p(v), None, None)
    assert rc == -1
    assert b"too large" in lib.qew_last_error(None)
    rc = lib.qew_observe_state_noalloc(ptr, ptr, 16, 4097, 1.0, 0, SEED, None, _p(v), None, None)
    assert rc == -1
