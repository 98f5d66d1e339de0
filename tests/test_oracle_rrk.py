"""Pins of the oracle's relaxation Runge-Kutta method (relaxed classical RK4:
q_{n+1} = q_n + gamma_n d, t_{n+1} = t_n + gamma_n dt, with gamma_n the root
near 1 of E(q_n + gamma d) = E(q_n); the paper names RRK as future work in its
conclusions and shows that standard RK does not conserve the energy of Thm.
4.1 / 4.2 in the fully discrete scheme).

What fixes the values:
  - the energy 1^T M E is conserved step by step to rounding (the defining
    property), while plain RK4 drifts; the mass (a linear invariant) stays
    conserved;
  - on the relaxation oscillator the energy is the quadratic form
    H/6 (omega^2 y^2 + w^2) + const, so gamma_n = -2 <x, d> / <d, d> in that
    inner product, with d = (P - I) x and P the RK4 propagator (closed form);
  - gamma_n - 1 = O(dt^3) at least (order p - 1 for RK4), and the relaxed
    method keeps order 4 at the relaxed times.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle as orc
from oracle import Grid, PERIODIC, REFLECTING
from paper_2601_02540_b300 import inputs
import pins

O = orc.default()


def _state(bc, nx=24, ny=16, seed=5):
    p = inputs.smooth_state(nx, ny, bc, seed=seed, xmax=4.0, ymax=3.0, lam=50.0)
    return p, pins.grid_of(p)


@pytest.mark.parametrize("bc", [PERIODIC, REFLECTING])
def test_rrk_conserves_energy_and_mass(bc):
    p, g = _state(bc)
    d0 = O.diagnostics(g, p.b, p.q0)
    q, gam, t = O.rrk4(g, p.b, p.q0, p.dt, 60)
    d1 = O.diagnostics(g, p.b, q)
    q4 = O.rk4(g, p.b, p.q0, p.dt, 60)
    d4 = O.diagnostics(g, p.b, q4)
    scale = abs(d0["energy"])
    assert abs(d1["energy"] - d0["energy"]) <= 1e-14 * scale
    assert abs(d4["energy"] - d0["energy"]) > 1e3 * abs(d1["energy"] - d0["energy"])
    assert abs(d1["mass"] - d0["mass"]) <= 1e-14 * abs(d0["mass"])
    assert abs(t - np.sum(gam) * p.dt) <= 1e-14 * t


@pytest.mark.parametrize("bc", [PERIODIC, REFLECTING])
def test_rrk_relaxation_oscillator_closed_form(bc):
    H, delta, lam = 0.7, 0.01, 500.0
    g = Grid(6, 5, 0.0, 1.0, 0.0, 1.0, bc, 9.81, lam)
    b = np.full((5, 6), -2.0)
    q = np.zeros((5, 5, 6))
    q[0] = H
    q[4] = H + delta
    om2 = lam / H ** 2
    dt = 0.4 / np.sqrt(om2)
    n = 25
    qn, gam, t = O.rrk4(g, b, q, dt, n)
    Z = dt * np.array([[0.0, 1.0], [-om2, 0.0]])
    P = np.eye(2) + Z + Z @ Z / 2 + Z @ Z @ Z / 6 + Z @ Z @ Z @ Z / 24
    W = np.diag([om2, 1.0])                       # energy inner product of (y, w)
    x = np.array([delta, 0.0])
    gams = []
    for _ in range(n):
        d = (P - np.eye(2)) @ x
        gm = -2.0 * (x @ W @ d) / (d @ W @ d)
        gams.append(gm)
        x = x + gm * d
    assert np.max(np.abs(gam - np.array(gams))) <= 1e-9
    assert np.max(np.abs(qn[4] - H - x[0])) <= 1e-10 * delta
    assert np.max(np.abs(qn[3] - x[1])) <= 1e-10 * delta * np.sqrt(om2)
    assert abs(t - dt * np.sum(gams)) <= 1e-9 * t


def test_rrk_gamma_minus_one_is_at_least_third_order():
    """gamma - 1 = O(dt^(p-1)) for an order-p method; here the RK4 energy error
    per step is O(dt^6) (as on skew linear problems), so it falls as dt^4."""
    p, g = _state(REFLECTING)
    dev = []
    for k in (1, 2, 4):
        _, gam, _ = O.rrk4(g, p.b, p.q0, p.dt / k, 1)
        dev.append(abs(gam[0] - 1.0))
    rates = np.log2(np.array(dev[:-1]) / np.array(dev[1:]))
    assert np.all((rates > 2.7) & (rates < 4.6)), (dev, rates)


def test_rrk_keeps_fourth_order_at_relaxed_times():
    p, g = _state(PERIODIC, nx=16, ny=12, seed=7)
    errs = []
    for k in (1, 2, 4):
        q, gam, t = O.rrk4(g, p.b, p.q0, 4 * p.dt / k, 10 * k)
        ref = O.rk4(g, p.b, p.q0, t / 800, 800)
        errs.append(np.max(np.abs(q - ref)))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all((rates > 3.6) & (rates < 4.4)), (errs, rates)
