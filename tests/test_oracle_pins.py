"""Pins of the oracle against what the paper and the mathematics fix.

Each test names the passage of arXiv 2601.02540 that fixes the checked value:
the printed SBP operators and SATs (Remark "Concrete SBP operators and SATs"),
the conservation theorems (Thm. 4.1, Thm. 4.2), the continuum system (eq.
(2D_hyperbolic_SGN)), the manufactured solution (Sec. 6.1.2), the
initialization (eq. (initialization)), the lambda = 0 reduction (Remark after
Thm. 4.1) and the 1D split form of Sec. 2.1.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle as orc
from oracle import Grid, PERIODIC, REFLECTING
from paper_2601_02540_b300 import inputs
import continuum as cont
import pins

O = orc.default()
GRIDS = [(3, 3), (5, 3), (7, 9), (16, 12), (33, 17)]


# ------------------------------------------------------------------ SBP operators
@pytest.mark.parametrize("bc,name", [(PERIODIC, "sbp_periodic_n5.txt"),
                                     (REFLECTING, "sbp_reflecting_n5.txt")])
@pytest.mark.parametrize("axis", ["x", "y"])
def test_operator_matches_printed_matrix(bc, name, axis):
    gold = pins.read_golden(name)
    D = pins.operator_matrix(O, bc, 5, axis)
    assert np.array_equal(2.0 * D, gold["2dx*D"])
    g = Grid(5, 5, 0.0, 5.0 if bc == PERIODIC else 4.0, 0.0, 5.0 if bc == PERIODIC else 4.0, bc)
    M = O.mass_weights(g)
    assert np.array_equal(M[2, :], gold["M/dx"][0])
    assert np.array_equal(M[:, 2], gold["M/dx"][0])


def test_sat_matches_printed_values():
    """SAT of eq. (semi_2D) on unit data: -2/dx at the first node, +2/dx at the
    last (Remark rem:concrete_sbp), isolated with h = 1 and a constant u."""
    gold = pins.read_golden("sbp_reflecting_n5.txt")["SAT*dx/2"][0]
    for dx in (1.0, 0.25):
        g = Grid(5, 4, 0.0, 4 * dx, 0.0, 3.0, REFLECTING)
        q = np.zeros((5, 4, 5))
        q[0] = 1.0
        q[4] = 1.0
        q[1] = 0.75
        dq = O.rhs(g, np.zeros((4, 5)), q)
        assert np.array_equal(dq[0] * dx / 2 / 0.75, np.tile(gold, (4, 1)))


@pytest.mark.parametrize("bc", [PERIODIC, REFLECTING])
@pytest.mark.parametrize("n", [3, 4, 5, 6, 7, 8])
def test_sbp_property_exact(bc, n):
    """M D + D^T M = e_R e_R^T - e_L e_L^T (reflecting) or 0 (periodic), exactly
    (dx = 1 makes all entries dyadic): Def. singledim_sbp and the remark."""
    D = pins.operator_matrix(O, bc, n)
    L = float(n) if bc == PERIODIC else float(n - 1)
    g = Grid(n, 3, 0.0, L, 0.0, 3.0 if bc == PERIODIC else 2.0, bc)
    M = np.diag(O.mass_weights(g)[1, :] / O.mass_weights(g)[1, 1])
    B = np.zeros((n, n))
    if bc == REFLECTING:
        B[0, 0], B[-1, -1] = -1.0, 1.0
    assert np.array_equal(M @ D + D.T @ M, B)
    assert np.all(np.diag(M) > 0)


@pytest.mark.parametrize("bc", [PERIODIC, REFLECTING])
def test_derivative_accuracy(bc):
    """D x^k = k x^(k-1) for k <= 1 everywhere and k = 2 on interior rows
    (Definition of a p-th order derivative matrix, Sec. 2.2)."""
    n = 9
    D = pins.operator_matrix(O, bc, n)
    xs = np.arange(n, dtype=float)
    assert np.array_equal(D @ np.ones(n), np.zeros(n))
    rows = slice(1, n - 1)
    assert np.allclose((D @ xs)[rows], 1.0, atol=0, rtol=0)
    assert np.allclose((D @ xs ** 2)[rows], 2 * xs[rows], rtol=0, atol=1e-14)
    if bc == REFLECTING:
        assert np.array_equal(D @ xs, np.ones(n))
        # boundary rows are only first-order: x^2 is not differentiated exactly
        assert (D @ xs ** 2)[0] != 0.0


@pytest.mark.parametrize("bc", [PERIODIC, REFLECTING])
def test_mass_matrix_quadrature(bc):
    """sum M = area, and the trapezoid/rectangle rule integrates x*y exactly on
    the closed (reflecting) grid."""
    g = Grid(7, 5, -1.0, 2.0, 0.5, 1.5, bc)
    M = O.mass_weights(g)
    assert np.isclose(M.sum(), 3.0 * 1.0, rtol=1e-15)
    if bc == REFLECTING:
        xs, ys = g.nodes()
        X, Y = np.meshgrid(xs, ys)
        exact = (2.0 ** 2 - 1.0) / 2 * (1.5 ** 2 - 0.5 ** 2) / 2
        assert np.isclose(np.sum(M * X * Y), exact, rtol=1e-14)


# ------------------------------------------------------------------ conservation
@pytest.mark.parametrize("bc", [PERIODIC, REFLECTING])
@pytest.mark.parametrize("nx,ny", GRIDS)
def test_mass_conserved_semidiscrete(bc, nx, ny):
    """Thm. 4.1/4.2 part 1: 1^T M h_t = 0 up to rounding."""
    for seed in (1, 2):
        p = inputs.smooth_state(nx, ny, bc, seed=seed)
        a, s = pins.mass_rate(O, p)
        assert a <= 1e-13 * s, (a, s)


@pytest.mark.parametrize("bc", [PERIODIC, REFLECTING])
@pytest.mark.parametrize("nx,ny", GRIDS)
def test_energy_conserved_semidiscrete(bc, nx, ny):
    """Thm. 4.1/4.2 part 2: <d_q E, q_t>_M = 0 up to rounding, both with the
    printed derivatives of E and by complex-step differentiation of E itself
    along the RHS (no derivative formula involved)."""
    for seed in (1, 2):
        p = inputs.smooth_state(nx, ny, bc, seed=seed)
        a, s = pins.energy_rate(O, p)
        assert a <= 1e-13 * s, (a, s)
        g = pins.grid_of(p)
        dq = O.rhs(g, p.b, p.q0)
        rate = O.energy_jvp(g, p.b, p.q0, dq)
        assert abs(rate) <= 1e-13 * s, (rate, s)


def test_energy_derivatives_match_energy():
    """The derivatives printed after eq. (splitcondition) are the gradient of
    the printed energy E (complex step on E along random directions)."""
    rng = np.random.default_rng(11)
    for bc in (PERIODIC, REFLECTING):
        p = inputs.smooth_state(9, 8, bc, seed=4)
        g = pins.grid_of(p)
        for _ in range(3):
            d = rng.standard_normal(p.q0.shape)
            a = O.energy_rate(g, p.b, p.q0, d)
            c = O.energy_jvp(g, p.b, p.q0, d)
            assert abs(a - c) <= 1e-13 * (abs(a) + 1.0), (a, c)


@pytest.mark.parametrize("bc", [PERIODIC, REFLECTING])
def test_energy_and_mass_closed_form(bc):
    """Flat b = -1, h = 1 at rest: E = g/2 h (h + 2b) = -g/2 per unit area,
    E' = E + g b^2/2 = 0; total mass = area."""
    g = Grid(6, 5, 0.0, 2.0, 0.0, 3.0, bc)
    b = np.full((5, 6), -1.0)
    q = np.zeros((5, 5, 6))
    q[0] = 1.0
    q[4] = 1.0
    d = O.diagnostics(g, b, q)
    assert np.isclose(d["mass"], 6.0, rtol=1e-15)
    assert np.isclose(d["energy"], -9.81 / 2 * 6.0, rtol=1e-15)
    assert abs(d["energy_shifted"]) <= 1e-15
    assert abs(d["dEdt"]) == 0.0


@pytest.mark.parametrize("bc", [PERIODIC, REFLECTING])
def test_lake_at_rest(bc):
    a, s = pins.lake_at_rest(O, bc)
    assert a <= 1e-14 * s, (a, s)


@pytest.mark.parametrize("bc", [PERIODIC, REFLECTING])
def test_relaxation_oscillator_closed_form(bc):
    err, tol = pins.relaxation_oscillator(O, bc, nsteps=200)
    assert err <= tol, err


@pytest.mark.parametrize("bc", [PERIODIC, REFLECTING])
def test_transpose_symmetry(bc):
    err, tol = pins.transpose_symmetry(O, bc)
    assert err <= tol, err


def test_y_uniform_reduces_to_1d_split_form():
    """Sec. 6: 1D problems run as y-uniform 2D data; all cross terms vanish.
    With lambda = 0 and b = 0 the (h, u) equations are the 1D split form of the
    shallow water equations printed in Sec. 2.1."""
    nx, ny = 24, 4
    g = Grid(nx, ny, 0.0, 3.0, 0.0, 1.0, PERIODIC, 9.81, 0.0)
    xs, _ = g.nodes()
    h1 = 1.0 + 0.2 * np.sin(2 * np.pi * xs / 3.0)
    u1 = 0.3 * np.cos(2 * np.pi * xs / 3.0 + 0.4)
    q = np.zeros((5, ny, nx))
    q[0], q[1], q[3], q[4] = h1, u1, 0.1, h1 * 1.01
    b = np.zeros((ny, nx))
    dq = O.rhs(g, b, q)
    assert np.all(dq[2] == 0.0)
    assert np.all(dq == dq[:, :1, :])
    dx = 3.0 / nx

    def D(f):
        return (np.roll(f, -1) - np.roll(f, 1)) / (2 * dx)

    ht = -(D(h1) * u1 + h1 * D(u1))
    hut = -(9.81 * D(h1 ** 2) - 9.81 * h1 * D(h1) + 0.5 * h1 * D(u1 ** 2) - 0.5 * D(h1) * u1 ** 2
            + 0.5 * D(h1 * u1) * u1 - 0.5 * h1 * u1 * D(u1))
    assert np.allclose(dq[0, 0], ht, rtol=0, atol=1e-13)
    assert np.allclose(dq[1, 0], hut / h1, rtol=0, atol=1e-12)


# ------------------------------------------------------------------ consistency
@pytest.mark.parametrize("bc", [PERIODIC, REFLECTING])
def test_consistency_with_continuum_system(bc):
    """The split-form RHS converges to the continuum RHS of eq.
    (2D_hyperbolic_SGN) (derived by sympy from the conservative form) at second
    order inside, first order on the one-sided boundary rows."""
    inner, edge, errs = pins.consistency_orders(O, bc)
    assert np.min(inner) > 1.8, inner
    if edge is not None:
        assert np.min(edge) > 0.85, edge


# ------------------------------------------------------------------ initialization
@pytest.mark.parametrize("bc", [PERIODIC, REFLECTING])
def test_init_aux(bc):
    """eq. (initialization): eta = h and w = -h (D_x u + D_y v) + 3/2 (u D_x b
    + v D_y b).  On a reflecting grid with linear u, v, b every SBP row is exact,
    so w equals the continuum formula."""
    p = inputs.smooth_state(10, 7, bc, seed=9)
    g = pins.grid_of(p)
    q = O.init_aux(g, p.b, p.q0)
    assert np.array_equal(q[4], q[0])
    assert np.array_equal(q[:3], p.q0[:3])
    if bc == REFLECTING:
        xs, ys = g.nodes()
        X, Y = np.meshgrid(xs, ys)
        u = 0.2 + 0.3 * X - 0.1 * Y
        v = -0.1 + 0.05 * X + 0.4 * Y
        b = -1.0 + 0.1 * X + 0.2 * Y
        q0 = p.q0.copy()
        q0[1], q0[2] = u, v
        q = O.init_aux(g, b, q0)
        w = -q0[0] * (0.3 + 0.4) + 1.5 * (u * 0.1 + v * 0.2)
        assert np.allclose(q[3], w, rtol=0, atol=1e-13)


# ------------------------------------------------------------------ time stepping
@pytest.mark.parametrize("bc", [PERIODIC, REFLECTING])
def test_rk4_preserves_mass(bc):
    """RK4 preserves the linear invariant 1^T M h (up to rounding)."""
    p = inputs.smooth_state(12, 10, bc, seed=3)
    g = pins.grid_of(p)
    q0 = O.init_aux(g, p.b, p.q0)
    m0 = O.diagnostics(g, p.b, q0)["mass"]
    q = O.rk4(g, p.b, q0, p.dt, 200)
    m1 = O.diagnostics(g, p.b, q)["mass"]
    assert abs(m1 - m0) <= 1e-13 * abs(m0)


def test_rk4_energy_drift_is_time_integration_error():
    """Sec. 6.2: with an energy-conserving semi-discretization, energy changes
    only through time integration; RK4 drift falls like dt^4 (here: halving dt
    reduces the drift by > 10x)."""
    p = inputs.smooth_state(16, 16, PERIODIC, seed=6)
    g = pins.grid_of(p)
    q0 = O.init_aux(g, p.b, p.q0)
    e0 = O.diagnostics(g, p.b, q0)["energy"]
    T = 40 * p.dt * 4
    drifts = []
    for k in (1, 2):
        q = O.rk4(g, p.b, q0, 4 * p.dt / k, 40 * k)
        drifts.append(abs(O.diagnostics(g, p.b, q)["energy"] - e0))
    assert drifts[1] < drifts[0] / 10, drifts
    assert T > 0


def test_complex_step_matches_finite_differences():
    """The complex build differentiates the real build: its JVP agrees with
    central differences of the real RHS."""
    rng = np.random.default_rng(2)
    for bc in (PERIODIC, REFLECTING):
        p = inputs.smooth_state(9, 7, bc, seed=8)
        g = pins.grid_of(p)
        dq = rng.standard_normal(p.q0.shape)
        db = rng.standard_normal(p.b.shape)
        jv = O.rhs_jvp(g, p.b, p.q0, db, dq)
        e = 1e-6
        fd = (O.rhs(g, p.b + e * db, p.q0 + e * dq) - O.rhs(g, p.b - e * db, p.q0 - e * dq)) / (2 * e)
        assert np.max(np.abs(jv - fd)) <= 1e-6 * np.max(np.abs(jv))


# ------------------------------------------------------------------ manufactured solution
def _mms_run(bc: int, n: int, t_end: float):
    (fb, fh, fu, fv, fw, feta), src = cont.manufactured()
    fns = cont.lambdify_fields((fb, fh, fu, fv, fw, feta) + tuple(src))
    g = Grid(n, n, -1.0, 1.0, -1.0, 1.0, bc, 9.81, 500.0)
    xs, ys = g.nodes()
    X, Y = np.meshgrid(xs, ys)
    b = cont.evaluate(fns[:1], X, Y, 0.0)[0]

    def exact(tt):
        return cont.evaluate(fns[1:6], X, Y, tt)

    def source(tt):
        return cont.evaluate(fns[6:], X, Y, tt)

    q = exact(0.0)
    dx, _ = g.spacing()
    c = 0.3 + np.sqrt(9.81 * 2.7 + 500.0 / 3.0)
    nsteps = int(np.ceil(t_end / (0.3 * dx / c)))
    dt = t_end / nsteps
    t = 0.0
    for _ in range(nsteps):
        k1 = O.rhs(g, b, q) + source(t)
        k2 = O.rhs(g, b, q + dt / 2 * k1) + source(t + dt / 2)
        k3 = O.rhs(g, b, q + dt / 2 * k2) + source(t + dt / 2)
        k4 = O.rhs(g, b, q + dt * k3) + source(t + dt)
        q = q + dt / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
        t += dt
    return np.max(np.abs(q - exact(t_end)), axis=(1, 2))


@pytest.mark.slow
@pytest.mark.parametrize("bc", [PERIODIC, REFLECTING])
def test_manufactured_solution_second_order(bc):
    """Sec. 6.1.2: the manufactured solution on [-1,1]^2 with lambda = 500
    converges at second order in all five variables, for both boundary
    treatments (here to t = 0.1 to keep the CPU suite short)."""
    errs = [_mms_run(bc, n, 0.1) for n in (16, 32, 64)]
    orders = np.log2(errs[1] / errs[2])
    assert np.all(orders > 1.7), (orders, errs)


# ------------------------------------------------------------------ gauge misfit
def test_gauge_loss_special_cases():
    """The misfit sum over observation times and gauges of (h - obs)^2 is 0
    against its own record, n c^2 against the record shifted by c, and its
    complex-step derivative agrees with central differences."""
    p = inputs.smooth_state(10, 9, REFLECTING, seed=12)
    g = pins.grid_of(p)
    q0 = O.init_aux(g, p.b, p.q0)
    gauges = np.array([11, 23, 47, 80], dtype=np.int64)
    rec = O.gauge_record(g, p.b, q0, p.dt, 12, 3, gauges)
    assert rec.shape == (4, 4)
    qa = O.rk4(g, p.b, q0, p.dt, 6)
    assert np.array_equal(rec[1], qa[0].ravel()[gauges])
    assert O.gauge_loss(g, p.b, q0, p.dt, 12, 3, gauges, rec) == 0.0
    c = 0.125
    assert np.isclose(O.gauge_loss(g, p.b, q0, p.dt, 12, 3, gauges, rec + c), 16 * c * c, rtol=1e-12)
    rng = np.random.default_rng(3)
    db = rng.standard_normal(p.b.shape)
    dq = np.zeros_like(q0)
    dq[0] = rng.standard_normal(p.b.shape)
    dq[4] = dq[0]
    obs = rec + 0.01
    jv = O.gauge_loss_jvp(g, p.b, q0, db, dq, p.dt, 12, 3, gauges, obs)
    e = 1e-6
    fd = (O.gauge_loss(g, p.b + e * db, q0 + e * dq, p.dt, 12, 3, gauges, obs)
          - O.gauge_loss(g, p.b - e * db, q0 - e * dq, p.dt, 12, 3, gauges, obs)) / (2 * e)
    assert abs(jv - fd) <= 1e-6 * abs(jv), (jv, fd)


@pytest.mark.parametrize("bc", [PERIODIC, REFLECTING])
@pytest.mark.parametrize("nx,ny", [(5, 3), (33, 17)])
def test_rhs_scale_bounds_the_rhs(bc, nx, ny):
    """The rounding scale S_f sums |coef| |D| |f| over the terms of the RHS
    value (and |pointwise terms|), so by the triangle inequality it bounds
    |k_f| at every node; it is what the parity tolerances multiply by u."""
    p = inputs.smooth_state(nx, ny, bc, seed=4, xmax=1.3, ymax=0.9)
    g = pins.grid_of(p)
    k = O.rhs(g, p.b, p.q0)
    S = O.rhs_scale(g, p.b, p.q0)
    assert np.all(S >= np.abs(k) * (1 - 1e-14))
    assert np.all(S > 0)


@pytest.mark.parametrize("bc", [PERIODIC, REFLECTING])
def test_rhs_scale_closed_form_on_constant_states(bc):
    """Pins the scale from above: on a constant state its value has a closed
    form (pins.rhs_scale_constant), which fixes the row sums of |D| (central
    and one-sided rows), the SAT terms, the count of (1 - eta/h) as
    1 + |eta/h| and the division of the u, v, w brackets by h; a scale that
    is too large anywhere would widen every parity bar that uses it."""
    dev, tol = pins.rhs_scale_constant(O, bc)
    assert dev <= tol, dev


# ------------------------------------------------------------------ solitary wave
@pytest.mark.slow
def test_soliton_second_order_against_sgn_solution():
    """Sec. 6.1.1 with lambda = 30000: the split-form scheme (RK4) converges at
    second order to the closed-form SGN solitary wave (eq.
    (solitary_wave_analytical)) of which the hyperbolic system is a close
    approximation; here over an eighth of a domain traversal."""
    errs = []
    for n in (64, 128, 256):
        p = inputs.soliton(n, ncross=3)
        g = pins.grid_of(p)
        q0 = O.init_aux(g, p.b, p.q0)
        k = p.nsteps // 8
        q = O.rk4(g, p.b, q0, p.dt, k)
        h, u = inputs.soliton_fields(p, k * p.dt)
        errs.append((np.max(np.abs(q[0] - h)), np.max(np.abs(q[1] - u))))
        assert np.max(np.abs(q[2])) <= 1e-12          # nothing moves across
    errs = np.array(errs)
    orders = np.log2(errs[-2] / errs[-1])
    assert np.all((orders > 1.85) & (orders < 2.2)), (orders, errs)


# ------------------------------------------------------------------ relaxation zones
@pytest.mark.parametrize("bc", [PERIODIC, REFLECTING])
def test_sponge_profile_and_rest_state(bc):
    """Relaxation zones (Sec. 6, wave-tank experiments): sigma is 0 away from
    the zones, reaches sigma_max where a reflecting wall node sits on the
    boundary, grows as the square of the depth into the zone, corners add
    both directions; a lake at rest equal to q0 is left unchanged."""
    g = Grid(41, 31, 0.0, 40.0, 0.0, 30.0, bc, 9.81, 500.0)
    wx, wy, smax = 5.0, 4.0, 5.0
    sg = O.sponge_sigma(g, wx, wy, smax)
    xs, ys = g.nodes()
    dxw = np.minimum(xs - g.xmin, g.xmax - xs)
    dyw = np.minimum(ys - g.ymin, g.ymax - ys)
    inner = np.outer(dyw >= wy, dxw >= wx)
    assert np.all(sg[inner] == 0.0) and np.all(sg >= 0.0)
    j = 15                                   # a row outside the y zones
    zx = dxw < wx
    prof = sg[j, zx] / smax
    depth = (wx - dxw[zx]) / wx
    assert np.allclose(prof, depth ** 2, rtol=1e-14, atol=0)
    if bc == REFLECTING:
        assert sg[j, 0] == smax and sg[j, -1] == smax and sg[0, 0] == 2 * smax
    # rest state
    b = -1.0 + 0.1 * np.outer(np.cos(ys / 5.0), np.sin(xs / 7.0))
    q0 = np.zeros((5, g.ny, g.nx))
    q0[0] = 0.3 - b
    q0[4] = q0[0]
    q = O.rk4_sponge(g, b, q0, 0.01, 20, q0, wx, wy, smax)
    assert np.max(np.abs(q - q0)) <= 1e-13
