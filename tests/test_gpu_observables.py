"""Error of the fused observables (Eqs. 3-5) of the FP32-split path against FP64 sums of the same
state, at the bench's chains (4 x 2^25 random field at f_c^L) after 10^4 Euler steps, when the
line is rough.

The fused epilogue sums, per warp tile, the FP32 values F_p, y = u - N0 and y^2 (N0: a cell of the
tile's window) sequentially over each lane's 31 sites and then over the 32 lanes in a shuffle tree;
lane 0 moves the tile's sums to the chain reference c in FP64, and the tiles are summed in FP64 in
a fixed order.  Each term therefore passes through at most 35 FP32 additions and 2 FP32 roundings of
its own (y = c + d and y^2), so with u = 2^-24 the classical bound of recursive summation gives
    |computed - exact| <= gamma * sum |terms|,  gamma = 40 u / (1 - 40 u)
for every tile sum.  With D = the largest spread of u over any two adjacent 992-site blocks plus
one cell (|y| <= D inside a tile) and R = |ubar - c| + D (the largest shift from a tile's N0 to the
chain reference), this bounds
    |d ubar| <= gamma D,   |d w2| <= gamma (D^2 + 2 R D) + 2 |ubar - c| gamma D,
    |d v| <= gamma max|F_p + f|  (F_p + f formed in FP32 and f removed again, two roundings),
with max|F_p + f| < 10 for N(0, 1) nodes and f < 1.
The FP64 reference: ubar and w2 are numpy's FP64 sums of the state (read through the C ABI, exact
n + d); v(t) is (ubar(t+1) - ubar(t)) / dt from the states at t and t + 1 (the periodic Laplacian
sums to zero, Eq. 3), which differs from f + <F_p> only by the FP32 rounding of each site's Euler
update (below 2^-25 per site, unbiased).
"""
import numpy as np
import pytest

from qew_workloads import SEED, preset_f

pytestmark = pytest.mark.gpu

RF, FP32 = 0, 0
GAMMA = 40 * 2.0 ** -24 / (1 - 40 * 2.0 ** -24)


def block_spread(u: np.ndarray, block: int = 992) -> float:
    """Largest max - min of u over two adjacent blocks of ``block`` sites (covers any tile window)."""
    n = (u.size // block) * block
    b = u[:n].reshape(-1, block)
    mx, mn = b.max(1), b.min(1)
    pair = np.maximum(mx[:-1], mx[1:]) - np.minimum(mn[:-1], mn[1:])
    return float(max(pair.max(), u.max() - u.min() if u.size < 2 * block else 0.0))


def test_observable_error_at_the_bench_size():
    import paper_1211_7275_gb300 as q
    q.load()
    L, B, t, dt = 1 << 25, 4, 10_000, 0.1
    f = preset_f("rf_4x2^25")
    with q.Relaxation(L, f, RF, dt=dt, seed=SEED, precision=FP32, batch=B) as r:
        obs = r.observe([t - 1, t])
        u0, _ = r.state()
        r.observe([t + 1])
        u1, _ = r.state()
    c_prev = np.floor(obs["ubar"][0] + 0.5)     # chain reference of the observation at t
    for s in range(B):
        a = u0[s * L:(s + 1) * L]
        b = u1[s * L:(s + 1) * L]
        ub64 = float(np.mean(a))
        w264 = float(np.mean((a - ub64) ** 2))
        v64 = float(np.mean(b - a)) / dt
        D = block_spread(a) + 1.0
        shift = abs(ub64 - c_prev[s])
        R = shift + D
        bound_ub = GAMMA * D
        bound_w2 = GAMMA * (D * D + 2 * R * D) + 2 * shift * GAMMA * D
        bound_v = GAMMA * 10.0 + 1e-9      # |F_p + f| < 10: N(0,1) nodes, f < 1 (a 9-sigma node has
                                           # probability 1e-19 per draw)
        e_ub = abs(obs["ubar"][1, s] - ub64)
        e_w2 = abs(obs["w2"][1, s] - w264)
        e_v = abs(obs["v"][1, s] - v64)
        print(f"chain {s}: ubar {ub64:.3f} w2 {w264:.4f} v {v64:.6f} (D {D:.1f}); errors: ubar {e_ub:.2e} "
              f"({e_ub / abs(ub64):.1e} rel, bound {bound_ub:.1e}), w2 {e_w2:.2e} ({e_w2 / w264:.1e} rel, bound "
              f"{bound_w2:.1e}), v {e_v:.2e} ({e_v / v64:.1e} rel, bound {bound_v:.1e})")
        assert e_ub <= bound_ub
        assert e_w2 <= bound_w2
        assert e_v <= bound_v
    # the sample spread the ensemble average is judged against (2 sigma bars)
    sig_w2 = np.std(obs["w2"][1], ddof=1) / np.sqrt(B)
    sig_v = np.std(obs["v"][1], ddof=1) / np.sqrt(B)
    print(f"sigma of the 4-sample means: w2 {sig_w2:.2e}, v {sig_v:.2e}")
