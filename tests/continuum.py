"""Continuum right-hand side of the 2D hyperbolized SGN system, derived with
sympy from its conservative form (eq. (2D_hyperbolic_SGN), Sec. 3.2), and the
manufactured solution of Sec. 6.1.2.

This is independent of the split form: the split-form semi-discretization must
reduce to these expressions as the grid is refined (consistency), and the
manufactured-solution source terms are built from them.

Conservative form (p = lambda/3 * eta/h * (1 - eta/h)):
  h_t    + (hu)_x + (hv)_y                                         = 0
  (hu)_t + (hu^2 + g h^2/2 + h p)_x + (huv)_y + (g h + 3/2 h/eta p) b_x = 0
  (hv)_t + (hvu)_x + (hv^2 + g h^2/2 + h p)_y + (g h + 3/2 h/eta p) b_y = 0
  (h eta)_t + (h eta u)_x + (h eta v)_y + 3/2 h (u b_x + v b_y)   = h w
  (hw)_t + (hwu)_x + (hwv)_y                                        = lambda (1 - eta/h)
The primitive derivatives follow from (h f)_t = h f_t + f h_t.
"""
from __future__ import annotations

import numpy as np
import sympy as sp

x, y, t = sp.symbols("x y t", real=True)
R = sp.Rational


def primitive_rhs(h, u, v, w, eta, b, g, lam):
    """(h_t, u_t, v_t, w_t, eta_t) as sympy expressions in x, y (and t)."""
    p = lam / 3 * eta / h * (1 - eta / h)
    ht = -(sp.diff(h * u, x) + sp.diff(h * v, y))
    hut = -(sp.diff(h * u ** 2 + g * h ** 2 / 2 + h * p, x) + sp.diff(h * u * v, y)
            + (g * h + R(3, 2) * h / eta * p) * sp.diff(b, x))
    hvt = -(sp.diff(h * v * u, x) + sp.diff(h * v ** 2 + g * h ** 2 / 2 + h * p, y)
            + (g * h + R(3, 2) * h / eta * p) * sp.diff(b, y))
    hetat = (h * w - sp.diff(h * eta * u, x) - sp.diff(h * eta * v, y)
             - R(3, 2) * h * (u * sp.diff(b, x) + v * sp.diff(b, y)))
    hwt = lam * (1 - eta / h) - sp.diff(h * w * u, x) - sp.diff(h * w * v, y)
    ut = (hut - u * ht) / h
    vt = (hvt - v * ht) / h
    wt = (hwt - w * ht) / h
    etat = (hetat - eta * ht) / h
    return ht, ut, vt, wt, etat


def lambdify_fields(exprs):
    """numpy callables f(X, Y, T) for a tuple of sympy expressions."""
    out = []
    for e in exprs:
        f = sp.lambdify((x, y, t), e, modules="numpy")
        out.append(f)
    return out


def evaluate(fns, X, Y, T=0.0):
    res = []
    for f in fns:
        val = f(X, Y, T)
        res.append(np.broadcast_to(np.asarray(val, dtype=np.float64), X.shape).copy())
    return np.stack(res)


# --------------------------------------------------------------- manufactured solution
def manufactured(g=9.81, lam=500):
    """The manufactured solution of Sec. 6.1.2 on [-1,1]^2 and its source terms
    S = q_t - RHS_continuum(q), so that q_t = RHS(q) + S holds exactly.
    Returns (fields (b, h, u, v, w, eta), sources (S_h, S_u, S_v, S_w, S_eta))
    as sympy expressions in x, y, t."""
    pi = sp.pi
    b = R(8, 100) * (sp.cos(2 * pi * x) * sp.cos(2 * pi * y)
                     + R(1, 2) * sp.cos(4 * pi * x) * sp.cos(4 * pi * y))
    h = 2 + R(1, 2) * sp.sin(2 * pi * x) * sp.sin(2 * pi * y) * sp.cos(2 * pi * t) - b
    u = R(3, 10) * sp.sin(2 * pi * x) * sp.sin(2 * pi * t)
    v = R(3, 10) * sp.sin(2 * pi * y) * sp.sin(2 * pi * t)
    eta = h
    w = -h * (sp.diff(u, x) + sp.diff(v, y)) + R(3, 2) * (u * sp.diff(b, x) + v * sp.diff(b, y))
    rhs = primitive_rhs(h, u, v, w, eta, b, g, lam)
    fields = (h, u, v, w, eta)
    src = tuple(sp.diff(f, t) - r for f, r in zip(fields, rhs))
    return (b, h, u, v, w, eta), src
