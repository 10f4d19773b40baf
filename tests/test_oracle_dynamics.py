"""Pins of the oracle's dynamics and observables against what the paper and the mathematics fix.

P2  disorder-free closed form: with F_p = 0 each Fourier mode of the periodic Euler map decays
    by lambda_k = 1 - 4 dt sin^2(pi k / L) per step and the centre of mass moves as f t
    (Eq. 1 discretised, Sec. III.B).
P3  the periodic Laplacian sums to zero, so ubar(step+1) - ubar(step) = dt v(step) with
    v = f + <F_p> (Eq. 3, Sec. II).
P4  Middleton no-passing (Sec. III.B): ordered initial states stay ordered while the Euler map
    is monotone, 1 - 2 dt + dt dF/du >= 0 at every site.  This needs a continuous force: for
    the linear-spline random bond (Case 3) the force jumps at the integers and the Euler map is
    not monotone there, so P4 is not asked of it.
P7  hand-computed single steps on tiny chains, the degenerate lengths L = 1, 2, 3.
Spline pins: the RF force interpolates R linearly between integers (Sec. III.B, Case 4 of
    Sec. IV.C); the RB force is minus the derivative of a C^1 cubic spline through V at the
    integers with the Catmull-Rom tangents (Cases 1-2); the Case 3 force is minus the slope of
    the linear spline through G, constant inside a cell, and equals the cell average of the
    Case 1 force through the same G (both potentials take the same values at the integers).
Observables: ubar, w2 against numpy's mean and population variance (Eqs. 4-5).
FP32 node model: the oracle's dynamics with every disorder value rounded to the nearest FP32
    number (the floor of any FP32 store of the disorder): one step from flat written out with
    numpy's float32 rounding, and 40 steps against a plain numpy restatement.
"""
import math

import numpy as np
import pytest

from qew_workloads import cosine_profile, positive_shift, random_points, random_state

SEED = 12117275


@pytest.mark.parametrize("L,k", [(64, 1), (64, 3), (63, 5), (17, 8)])
def test_closed_form_disorder_free(orc, L, k):
    A, B, f, dt = 0.7, 3.2, 0.37, 0.1
    u0 = cosine_profile(L, A, B, k)
    lam = 1.0 - 4.0 * dt * math.sin(math.pi * k / L) ** 2
    i = np.arange(L)
    for n in (1, 7, 50, 200):
        out = orc.run(L, f, dt, orc.KIND_NONE, SEED, [0, n], u0=u0, want_state=True)
        exact = B + f * n * dt + A * lam ** n * np.cos(2 * math.pi * k * i / L)
        assert np.max(np.abs(out["u"] - exact) / np.maximum(1.0, np.abs(exact))) < 1e-12
        assert abs(out["ubar"][1, 0] - (B + f * n * dt)) < 1e-12 * max(1.0, B + f * n * dt)
        assert abs(out["v"][1, 0] - f) < 1e-15
        if 2 * k != L:
            assert abs(out["w2"][1, 0] - A * A * lam ** (2 * n) / 2) < 1e-12
        assert abs(out["w2"][0, 0] - A * A / 2) < 1e-12


@pytest.mark.parametrize("kind,L,f", [(0, 257, 1.0), (1, 256, 1.9), (0, 5, 0.3), (1, 3, 2.5),
                                       (3, 256, 1.6), (3, 3, 3.0), (4, 255, 1.5)])
def test_mean_velocity_invariant(orc, kind, L, f):
    steps = list(range(0, 21)) + [100, 101, 500, 501]
    dt = 0.1
    out = orc.run([L, L], f, dt, kind, SEED, steps)
    ub, v = out["ubar"], out["v"]
    idx = [j for j in range(len(steps) - 1) if steps[j + 1] == steps[j] + 1]
    for j in idx:
        d = ub[j + 1] - ub[j]
        assert np.all(np.abs(d - dt * v[j]) <= 1e-12 * np.maximum(1.0, np.abs(ub[j + 1]))), j
    assert np.all(out["w2"][0] == 0.0)
    assert np.all(out["ubar"][0] == 0.0)


@pytest.mark.parametrize("kind,dt,f", [(0, 0.1, 1.0), (1, 0.02, 1.8), (4, 0.01, 1.5)])
def test_no_passing(orc, kind, dt, f):
    L = 300
    u0 = random_state(L, 0.5, seed=11)
    u1 = u0 + positive_shift(L, 0.3, seed=12)
    for n in (10, 200, 1000):
        a = orc.run(L, f, dt, kind, SEED, [n], u0=u0, want_state=True)["u"]
        b = orc.run(L, f, dt, kind, SEED, [n], u0=u1, want_state=True)["u"]
        assert np.all(b >= a), n


def test_one_step_by_hand_L3(orc):
    # u = (0, 1, 3), f = 0.5, dt = 0.1, no disorder:
    # lap = (1 + 3 - 0, 3 + 0 - 2, 0 + 1 - 6) = (4, 1, -5); u' = u + dt (lap + f)
    out = orc.run(3, 0.5, 0.1, orc.KIND_NONE, SEED, [1], u0=[0.0, 1.0, 3.0], want_state=True)
    assert np.allclose(out["u"], [0.45, 1.15, 2.55], rtol=0, atol=1e-15)


def test_degenerate_lengths(orc):
    # L = 1: the site is its own neighbour on both sides, lap = 0
    out = orc.run(1, 0.5, 0.1, orc.KIND_NONE, SEED, [3], u0=[2.0], want_state=True)
    assert abs(out["u"][0] - (2.0 + 3 * 0.05)) < 1e-15
    # L = 2: both neighbours of a site are the other site, lap_i = 2 (u_j - u_i)
    out = orc.run(2, 0.0, 0.1, orc.KIND_NONE, SEED, [1], u0=[0.0, 1.0], want_state=True)
    assert np.allclose(out["u"], [0.2, 0.8], rtol=0, atol=1e-15)


@pytest.mark.parametrize("kind", [0, 1, 3, 4])
def test_first_step_from_flat(orc, kind):
    """From the flat start lap = 0 and d = 0, so u_i(1) = dt (f + F_p(i, 0))."""
    L, f, dt = 97, 0.8, 0.1
    out = orc.run(L, f, dt, kind, SEED, [1], s=[4], want_state=True)
    i = np.arange(L)
    F0 = orc.pinning_force(kind, SEED, 4, i, np.zeros(L))
    assert np.allclose(out["u"], dt * (f + F0), rtol=0, atol=1e-15)
    if kind == 0:
        assert np.array_equal(F0, orc.disorder_values(0, SEED, 4, i, np.zeros(L)))
    if kind == 3:
        G0 = orc.disorder_values(3, SEED, 4, i, np.zeros(L))
        G1 = orc.disorder_values(3, SEED, 4, i, np.ones(L))
        assert np.array_equal(F0, G0 - G1)


def test_case3_two_steps_by_hand_L3(orc):
    """Case 3 on L = 3, written out: step 1 from flat, then step 2 with the cells floor(u(1))."""
    f, dt, s = 2.0, 0.1, 1
    i = np.arange(3)
    G = {k: orc.disorder_values(3, SEED, s, i, np.full(3, k)) for k in (-2, -1, 0, 1, 2)}
    u1 = dt * (f + (G[0] - G[1]))
    n1 = np.floor(u1).astype(int)
    F1 = np.array([G[n1[j]][j] - G[n1[j] + 1][j] for j in range(3)])
    lap = np.array([u1[1] + u1[2] - 2 * u1[0], u1[2] + u1[0] - 2 * u1[1], u1[0] + u1[1] - 2 * u1[2]])
    u2 = u1 + dt * (lap + f + F1)
    out = orc.run(3, f, dt, 3, SEED, [1, 2], s=[s], want_state=True)
    assert np.allclose(out["u"], u2, rtol=0, atol=1e-14)
    assert abs(out["v"][0, 0] - (f + np.mean(G[0] - G[1]))) < 1e-14


def test_rf_force_is_linear_interpolation(orc):
    i, n = random_points(2000, 1 << 20, -40, 40, seed=21)
    R0 = orc.disorder_values(0, SEED, 2, i, n)
    R1 = orc.disorder_values(0, SEED, 2, i, n + 1)
    # nodes
    assert np.array_equal(orc.pinning_force(0, SEED, 2, i, n.astype(float)), R0)
    # continuity at the upper node
    below = orc.pinning_force(0, SEED, 2, i, (n + 1).astype(float) - 1e-12)
    assert np.allclose(below, R1, atol=1e-10, rtol=0)
    # straight line in between: equal second differences vanish
    d = np.array([0.1, 0.35, 0.6, 0.85])
    F = np.stack([orc.pinning_force(0, SEED, 2, i, n + x) for x in d])
    assert np.allclose(F[1] - F[0], F[3] - F[2], atol=1e-12)
    assert np.allclose(F[2] - F[1], F[1] - F[0], atol=1e-12)
    # slope equals the node difference
    assert np.allclose((F[3] - F[0]) / 0.75, R1 - R0, atol=1e-11)


@pytest.mark.parametrize("kind", [1, 4])
def test_rb_spline_pins(orc, kind):
    i, n = random_points(2000, 1 << 18, -40, 40, seed=22)
    s = 6
    V = [orc.disorder_values(kind, SEED, s, i, n + k) for k in (-1, 0, 1, 2)]
    nf = n.astype(float)
    tol = 1.0 if kind == 1 else 4.0   # Gaussian values reach |G| ~ 4.5 on 8000 draws
    # the potential interpolates the drawn values at the integers
    assert np.allclose(orc.rb_potential(SEED, s, i, nf, kind), V[1], atol=1e-15 * tol, rtol=0)
    assert np.allclose(orc.rb_potential(SEED, s, i, nf + 1 - 1e-13, kind), V[2], atol=1e-11 * tol, rtol=0)
    # Catmull-Rom tangents: F(n) = -(V(n+1) - V(n-1)) / 2, F(n+1-) = -(V(n+2) - V(n)) / 2
    assert np.allclose(orc.pinning_force(kind, SEED, s, i, nf), -(V[2] - V[0]) / 2, atol=1e-15 * tol)
    assert np.allclose(orc.pinning_force(kind, SEED, s, i, nf + 1 - 1e-13), -(V[3] - V[1]) / 2,
                       atol=1e-11 * tol)
    # the force is quadratic in the cell: 3-point Gauss-Legendre integrates it exactly, and
    # its integral over the cell is -(V(n+1) - V(n))
    x, w = np.polynomial.legendre.leggauss(3)
    integral = sum(wk * orc.pinning_force(kind, SEED, s, i, nf + 0.5 + 0.5 * xk) for xk, wk in zip(x, w)) * 0.5
    assert np.allclose(integral, -(V[2] - V[1]), atol=1e-14 * tol)
    # F = -dV/du inside the cell (central difference of the potential)
    h = 1e-5
    for d in (0.2, 0.5, 0.77):
        Fd = orc.pinning_force(kind, SEED, s, i, nf + d)
        dV = (orc.rb_potential(SEED, s, i, nf + d + h, kind) - orc.rb_potential(SEED, s, i, nf + d - h, kind)) / (2 * h)
        assert np.allclose(Fd, -dV, atol=1e-8 * tol)


def test_case3_linear_spline_pins(orc):
    """Case 3: V is the straight line through G(n), G(n+1) on each cell, F = -dV/du."""
    i, n = random_points(2000, 1 << 18, -40, 40, seed=23)
    s = 2
    G0 = orc.disorder_values(3, SEED, s, i, n)
    G1 = orc.disorder_values(3, SEED, s, i, n + 1)
    nf = n.astype(float)
    # nodes, and the straight line in between
    assert np.array_equal(orc.rb_potential(SEED, s, i, nf, 3), G0)
    for d in (0.25, 0.5, 0.9):
        assert np.allclose(orc.rb_potential(SEED, s, i, nf + d, 3), G0 + d * (G1 - G0), atol=1e-14)
    # constant inside the cell (including the node itself: floor(n) = n)
    F = [orc.pinning_force(3, SEED, s, i, nf + d) for d in (0.0, 0.3, 0.75, 1 - 1e-12)]
    for Fd in F[1:]:
        assert np.array_equal(Fd, F[0])
    # minus the slope: the potential falls where the force is positive
    h = 1e-4
    dV = (orc.rb_potential(SEED, s, i, nf + 0.5 + h, 3) - orc.rb_potential(SEED, s, i, nf + 0.5 - h, 3)) / (2 * h)
    assert np.allclose(F[0], -dV, atol=1e-9)
    # the jump at the upper node is the next cell's force
    above = orc.pinning_force(3, SEED, s, i, nf + 1.0)
    G2 = orc.disorder_values(3, SEED, s, i, n + 2)
    assert np.array_equal(above, G1 - G2)


def test_case1_cell_average_is_case3_force(orc):
    """The cubic (Case 1) and linear (Case 3) splines through the same G agree at the integers,
    so the Case 1 force averaged over a cell equals the constant Case 3 force of that cell."""
    i, n = random_points(3000, 1 << 20, -60, 60, seed=24)
    s = 9
    nf = n.astype(float)
    x, w = np.polynomial.legendre.leggauss(3)
    avg = sum(wk * orc.pinning_force(4, SEED, s, i, nf + 0.5 + 0.5 * xk) for xk, wk in zip(x, w)) * 0.5
    F3 = orc.pinning_force(3, SEED, s, i, nf + 0.5)
    assert np.allclose(avg, F3, atol=1e-13, rtol=0)
    # and the two forces are different functions: the cubic one varies inside the cell
    assert np.mean(np.abs(orc.pinning_force(4, SEED, s, i, nf + 0.1) - F3) > 1e-3) > 0.9


def test_observables_match_numpy(orc):
    L = 1000
    u0 = random_state(L, 2.0, seed=31)
    f = 0.6
    out = orc.run(L, f, 0.1, 0, SEED, [0], u0=u0)
    assert abs(out["ubar"][0, 0] - np.mean(u0)) < 1e-12 * max(1, abs(np.mean(u0)))
    assert abs(out["w2"][0, 0] - np.var(u0)) < 1e-10 * np.var(u0)
    F = orc.pinning_force(0, SEED, 0, np.arange(L), u0)
    assert abs(out["v"][0, 0] - (f + np.mean(F))) < 1e-13


@pytest.mark.parametrize("kind", [0, 1, 3, 4])
def test_lightcone_equals_periodic_run(orc, kind):
    L, n, w = 101, 20, 7
    full = orc.run(L, 1.2, 0.1, kind, SEED, [n], s=[3], want_state=True)["u"]
    Ffull = orc.pinning_force(kind, SEED, 3, np.arange(L), full)
    for i0 in (0, 50, 97, L - 1):
        u, F = orc.lightcone(L, 3, 1.2, 0.1, kind, SEED, i0, w, n)
        idx = (i0 + np.arange(w)) % L
        assert np.array_equal(u, full[idx])
        assert np.array_equal(F, Ffull[idx])


def test_chains_are_independent_and_keyed_by_sample(orc):
    L = 64
    both = orc.run([L, L], 1.0, 0.1, 0, SEED, [100], s=[0, 1], want_state=True)["u"]
    one = orc.run(L, 1.0, 0.1, 0, SEED, [100], s=[1], want_state=True)["u"]
    assert np.array_equal(both[L:], one)
    assert not np.array_equal(both[:L], both[L:])


def test_rejects_bad_arguments(orc):
    with pytest.raises(ValueError):
        orc.run(8, 1.0, 0.1, 0, SEED, [5, 3])
    with pytest.raises(ValueError):
        orc.run(0, 1.0, 0.1, 0, SEED, [1])
    with pytest.raises(ValueError):
        orc.lightcone(10, 0, 1.0, 0.1, 0, SEED, 0, 3, 4)


# ------------------------------------------------------------------------------------------
# FP32 node model: the exact dynamics of the disorder rounded to FP32
# ------------------------------------------------------------------------------------------
@pytest.mark.parametrize("kind", [0, 1, 3, 4])
def test_fp32_node_model_first_step(orc, kind):
    """From the flat start (lap = 0, d = 0) one step of the FP32 node model is
    u_i(1) = dt ((0 + f) + F), with F formed from the disorder values rounded to the nearest
    FP32 number (numpy's float32 conversion, round to nearest even): R(0) for RF, G(0) - G(1)
    for Case 3, -(V(1) - V(-1)) / 2 for the Catmull-Rom kinds."""
    L, f, dt, s = 211, 0.8, 0.1, 2
    i = np.arange(L)

    def node(n):
        return orc.disorder_values(kind, SEED, s, i, np.full(L, n)).astype(np.float32).astype(np.float64)

    if kind == 0:
        F = node(0)
    elif kind == 3:
        F = node(0) - node(1)
    else:
        F = -0.5 * (node(1) - node(-1))
    out = orc.run(L, f, dt, kind, SEED, [1], s=[s], want_state=True, node_f32=True)
    assert np.array_equal(out["u"], dt * ((0.0 + f) + F))
    exact = orc.run(L, f, dt, kind, SEED, [1], s=[s], want_state=True)
    assert not np.array_equal(out["u"], exact["u"])          # the rounding is applied ...
    assert np.max(np.abs(out["u"] - exact["u"])) <= dt * 2.0 ** -23 * 8   # ... and is an FP32 rounding


def test_fp32_node_model_moves_cells(orc):
    """Later steps of the FP32 node model use the rounded values of the cell each site has moved
    to: after 40 steps the exact run's state and the node model agree to the size the rounding
    can explain, and the node model equals a plain numpy restatement with rounded nodes."""
    L, f, dt, s, n = 64, 1.3, 0.1, 5, 40
    out = orc.run(L, f, dt, 0, SEED, [n], s=[s], want_state=True, node_f32=True)["u"]
    u = np.zeros(L)
    i = np.arange(L)
    for _ in range(n):
        c = np.floor(u)
        d = u - c
        r0 = orc.disorder_values(0, SEED, s, i, c).astype(np.float32).astype(np.float64)
        r1 = orc.disorder_values(0, SEED, s, i, c + 1).astype(np.float32).astype(np.float64)
        F = (1.0 - d) * r0 + d * r1
        lap = (np.roll(u, -1) + np.roll(u, 1)) - 2.0 * u
        u = u + dt * ((lap + f) + F)
    assert np.array_equal(out, u)
    exact = orc.run(L, f, dt, 0, SEED, [n], s=[s], want_state=True)["u"]
    assert 0 < np.max(np.abs(out - exact)) < 1e-5
