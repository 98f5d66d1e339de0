"""Checks that pin the oracle to what the paper and the mathematics fix.

Each check takes an oracle object (``oracle.default()`` or a mutated build)
and returns the measured quantity together with the threshold it must meet, so
the same checks serve the pin tests and the mutation test.
"""
from __future__ import annotations

import functools
import os

import numpy as np
import sympy as sp

import oracle as orc
from oracle import Grid, PERIODIC, REFLECTING
from paper_2601_02540_b300 import inputs
import continuum as cont

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def grid_of(p: inputs.Problem) -> Grid:
    return Grid(p.nx, p.ny, p.xmin, p.xmax, p.ymin, p.ymax, p.bc, p.g, p.lam)


def read_golden(name: str) -> dict[str, np.ndarray]:
    blocks: dict[str, list[list[float]]] = {}
    cur = None
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            s = line.strip()
            if not s or s.startswith("#"):
                continue
            try:
                row = [float(t) for t in s.split()]
            except ValueError:
                cur = s
                blocks[cur] = []
                continue
            blocks[cur].append(row)
    return {k: np.array(v) for k, v in blocks.items()}


def operator_matrix(o, bc: int, n: int, axis: str = "x") -> np.ndarray:
    """Dense D (n x n) probed from the oracle with unit vectors, dx = 1."""
    L = float(n) if bc == PERIODIC else float(n - 1)
    if axis == "x":
        g = Grid(n, 3, 0.0, L, 0.0, 3.0 if bc == PERIODIC else 2.0, bc)
    else:
        g = Grid(3, n, 0.0, 3.0 if bc == PERIODIC else 2.0, 0.0, L, bc)
    D = np.zeros((n, n))
    for k in range(n):
        f = np.zeros((g.ny, g.nx))
        if axis == "x":
            f[:, k] = 1.0
            D[:, k] = o.dx_apply(g, f)[1, :]
        else:
            f[k, :] = 1.0
            D[:, k] = o.dy_apply(g, f)[:, 1]
    return D


# ------------------------------------------------------------------------ invariants
def mass_rate(o, p: inputs.Problem) -> tuple[float, float]:
    """|1^T M h_t| and its rounding scale (Thm. 4.1/4.2, part 1)."""
    g = grid_of(p)
    dq = o.rhs(g, p.b, p.q0)
    sc = o.rhs_scale(g, p.b, p.q0)
    M = o.mass_weights(g)
    return abs(float(np.sum(M * dq[0]))), float(np.sum(M * sc[0]))


def energy_rate(o, p: inputs.Problem) -> tuple[float, float]:
    """|<d_q E, RHS>_M| and its rounding scale (Thm. 4.1/4.2, part 2)."""
    d = o.diagnostics(grid_of(p), p.b, p.q0)
    return abs(d["dEdt"]), d["dEdt_scale"]


def lake_at_rest(o, bc: int, nx=9, ny=7, seed=3) -> tuple[float, float]:
    """h + b constant, u = v = w = 0, eta = h: the RHS vanishes (all the
    g-terms pair up; eta/h = 1 removes the lambda-terms)."""
    p = inputs.smooth_state(nx, ny, bc, seed=seed)
    h = 0.5 - p.b
    q = np.zeros_like(p.q0)
    q[0] = h
    q[4] = h
    g = grid_of(p)
    dq = o.rhs(g, p.b, q)
    sc = o.rhs_scale(g, p.b, q)
    return float(np.max(np.abs(dq))), float(np.max(sc))


def relaxation_oscillator(o, bc: int, H=0.7, delta=0.01, lam=500.0, nsteps=40) -> tuple[float, float]:
    """Flat b, uniform h = H, u = v = w = 0, uniform eta = H + delta.  All
    gradients vanish, h stays H, and (eta - H, w) obey y' = w, w' = -(lam/H^2) y
    exactly, so RK4 gives (y, w)_n = P^n (delta, 0) with
    P = I + Z + Z^2/2 + Z^3/6 + Z^4/24, Z = dt [[0, 1], [-lam/H^2, 0]]."""
    nx, ny = 6, 5
    L = 1.0
    g = Grid(nx, ny, 0.0, L, 0.0, L, bc, 9.81, lam)
    b = np.full((ny, nx), -2.0)
    q = np.zeros((5, ny, nx))
    q[0] = H
    q[4] = H + delta
    om2 = lam / H ** 2
    dt = 0.2 / np.sqrt(om2)
    qn = o.rk4(g, b, q, dt, nsteps)
    Z = dt * np.array([[0.0, 1.0], [-om2, 0.0]])
    P = np.eye(2) + Z + Z @ Z / 2 + Z @ Z @ Z / 6 + Z @ Z @ Z @ Z / 24
    ex = np.linalg.matrix_power(P, nsteps) @ np.array([delta, 0.0])
    err = max(float(np.max(np.abs(qn[4] - H - ex[0]))) / delta,
              float(np.max(np.abs(qn[3] - ex[1]))) / (delta * np.sqrt(om2)),
              float(np.max(np.abs(qn[0] - H))), float(np.max(np.abs(qn[1]))),
              float(np.max(np.abs(qn[2]))))
    return err, 1e-10


def transpose_symmetry(o, bc: int, nx=7, ny=5, seed=5) -> tuple[float, float]:
    """Swapping x and y (planes transposed, u <-> v, dx <-> dy) transposes the
    RHS with u_t <-> v_t (the scheme treats both directions alike)."""
    p = inputs.smooth_state(nx, ny, bc, seed=seed, xmax=1.3, ymax=0.9)
    g = grid_of(p)
    dq = o.rhs(g, p.b, p.q0)
    sc = o.rhs_scale(g, p.b, p.q0)
    qt = p.q0.transpose(0, 2, 1)[[0, 2, 1, 3, 4]]
    gt = Grid(ny, nx, p.ymin, p.ymax, p.xmin, p.xmax, bc, p.g, p.lam)
    dqt = o.rhs(gt, p.b.T, qt)
    back = dqt.transpose(0, 2, 1)[[0, 2, 1, 3, 4]]
    return float(np.max(np.abs(back - dq) / np.max(sc, axis=(1, 2), keepdims=True))), 1e-13


def rhs_scale_constant(o, bc: int, H=0.9, U=0.3, V=-0.2, W=0.15, E=1.1, B=-0.8) -> tuple[float, float]:
    """Closed form of the rounding-error scale on a constant state (every field
    and b constant, all active, eta != h).  Each split-form term coef * D f
    contributes |coef| |D| |f| = |coef| |f| kappa, where kappa is the row sum
    of |D|: 1/dx on central rows (|f|/(2dx) + |f|/(2dx)), 2/dx on the one-sided
    rows (f1 - f0)/dx of a reflecting wall.  Summing the terms of eqs.
    (sd_periodic_2D_SGN) / (semi_2D) by hand, with rho = E/H and the factor
    (1 - rho) counted as 1 + |rho|:
      S_h = 2H|U| kx + 2H|V| ky (+ (2/dx) H|U| at x-walls, (2/dy) H|V| at y-walls)
      S_u = [kx (2gH|H+B| + 2HU^2 + lam/6 rho^2 H + lam/3 |E| (1 + |rho|)
                + lam/6 E^2/H + lam/2 (1 + |rho|)|B|) + ky 2H|U||V|] / H
      S_v = the same with (x, U) and (y, V) exchanged
      S_w = [lam (1 + |rho|) + 2H|W| (|U| kx + |V| ky)] / H
      S_eta = |W| + |U| (|E| + 3/2 |B|) kx + |V| (|E| + 3/2 |B|) ky
    (the actual RHS of a constant state is lam (1 - rho)/H in w and W in eta,
    zero elsewhere).  Returns the largest relative deviation of the oracle's
    scale from this closed form over all nodes and fields."""
    nx, ny = 7, 6
    g = Grid(nx, ny, 0.0, 1.4, 0.0, 0.9, bc, 9.81, 500.0)
    dx, dy = g.spacing()
    b = np.full((ny, nx), B)
    q = np.empty((5, ny, nx))
    for f, val in enumerate((H, U, V, W, E)):
        q[f] = val
    S = o.rhs_scale(g, b, q)
    kx = np.full(nx, 1.0 / dx)
    ky = np.full(ny, 1.0 / dy)
    if bc == REFLECTING:
        kx[[0, -1]] = 2.0 / dx
        ky[[0, -1]] = 2.0 / dy
    KX, KY = np.meshgrid(kx, ky)
    gr, lam = g.g, g.lam
    rho = E / H
    aU, aV, aW, aE, aB = abs(U), abs(V), abs(W), abs(E), abs(B)
    lam_part = lam / 6 * rho ** 2 * H + lam / 3 * aE * (1 + abs(rho)) + lam / 6 * E ** 2 / H \
        + lam / 2 * (1 + abs(rho)) * aB
    ex = np.empty_like(S)
    ex[0] = 2 * H * aU * KX + 2 * H * aV * KY
    if bc == REFLECTING:
        ex[0][:, [0, -1]] += 2.0 / dx * H * aU
        ex[0][[0, -1], :] += 2.0 / dy * H * aV
    ex[1] = (KX * (2 * gr * H * abs(H + B) + 2 * H * U ** 2 + lam_part) + KY * 2 * H * aU * aV) / H
    ex[2] = (KY * (2 * gr * H * abs(H + B) + 2 * H * V ** 2 + lam_part) + KX * 2 * H * aU * aV) / H
    ex[3] = (lam * (1 + abs(rho)) + 2 * H * aW * (aU * KX + aV * KY)) / H
    ex[4] = aW + aU * (aE + 1.5 * aB) * KX + aV * (aE + 1.5 * aB) * KY
    return float(np.max(np.abs(S - ex) / ex)), 1e-14


# ------------------------------------------------------------------ consistency (sympy)
def _analytic_fields(bc: int):
    """Smooth analytic fields on [0,1]^2 with every variable active.  For the
    reflecting case u vanishes on x = 0, 1 and v on y = 0, 1 (wall condition),
    so the SATs vanish for the exact fields."""
    x, y = cont.x, cont.y
    pi = sp.pi
    b = -1 + sp.Rational(1, 10) * sp.cos(2 * pi * x) * sp.sin(2 * pi * y)
    h = 1 + sp.Rational(1, 5) * sp.sin(2 * pi * x) * sp.cos(2 * pi * y) - sp.Rational(1, 20) * sp.cos(2 * pi * y)
    if bc == PERIODIC:
        u = sp.Rational(3, 10) * sp.cos(2 * pi * x + sp.Rational(1, 2)) * sp.cos(2 * pi * y)
        v = sp.Rational(1, 5) * sp.sin(2 * pi * (x + y))
    else:
        u = sp.Rational(3, 10) * sp.sin(pi * x) * (1 + sp.cos(2 * pi * y) / 2)
        v = sp.Rational(1, 5) * sp.sin(pi * y) * sp.cos(2 * pi * x)
    w = sp.Rational(1, 10) * sp.cos(2 * pi * y) + sp.Rational(1, 20) * sp.sin(2 * pi * x)
    eta = h * (1 + sp.Rational(1, 20) * sp.sin(2 * pi * x) * sp.cos(4 * pi * y))
    return b, (h, u, v, w, eta)


@functools.lru_cache(maxsize=None)
def _continuum_fns(bc: int, lam: float):
    b, f = _analytic_fields(bc)
    rhs = cont.primitive_rhs(*f, b, 9.81, lam)
    return (cont.lambdify_fields((b,))[0], cont.lambdify_fields(f), cont.lambdify_fields(rhs))


def consistency_errors(o, bc: int, ns=(16, 32, 64), lam=500.0):
    """Max errors of the discrete RHS against the continuum RHS at the nodes,
    per field, split into interior and boundary nodes (boundary rows of the
    reflecting operator are first-order accurate)."""
    fb, ff, fr = _continuum_fns(bc, lam)
    res = []
    for n in ns:
        g = Grid(n, n, 0.0, 1.0, 0.0, 1.0, bc, 9.81, lam)
        xs, ys = g.nodes()
        X, Y = np.meshgrid(xs, ys)
        b = np.broadcast_to(np.asarray(fb(X, Y, 0.0), dtype=float), X.shape).copy()
        q = cont.evaluate(ff, X, Y)
        ex = cont.evaluate(fr, X, Y)
        dq = o.rhs(g, b, q)
        err = np.abs(dq - ex)
        inner = err[:, 1:-1, 1:-1] if bc == REFLECTING else err
        edge = err.copy()
        edge[:, 1:-1, 1:-1] = 0.0
        res.append((np.max(inner, axis=(1, 2)), np.max(edge, axis=(1, 2))))
    return res


def consistency_orders(o, bc: int, ns=(16, 32, 64)):
    errs = consistency_errors(o, bc, ns)
    inner = [np.log2(errs[k][0] / errs[k + 1][0]) for k in range(len(ns) - 1)]
    edge = [np.log2(errs[k][1] / errs[k + 1][1]) for k in range(len(ns) - 1)] if bc == REFLECTING else None
    return inner, edge, errs
