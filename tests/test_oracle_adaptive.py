"""Pins of the oracle's adaptive time integrator (Sec. 6: an explicit
third-order Runge-Kutta pair with the first-same-as-last property, an embedded
error estimate and step-size control; the pair restated is Bogacki-Shampine
3(2), whose coefficients the paper does not print).

What fixes the values:
  - the relaxation oscillator (flat b, uniform h = H, u = v = w = 0,
    eta = H + delta) is an exact linear system for (eta - H, w) with
    Z = dt [[0, 1], [-lam/H^2, 0]].  Any three-stage third-order explicit
    method advances it by P = I + Z + Z^2/2 + Z^3/6; the pair's embedded
    second-order solution gives I + Z + Z^2/2 + 3 Z^3/16 + Z^4/48, so the error
    estimate of a step from y is e = -(Z^3 + Z^4)/48 y (closed forms of the
    published tableau on a linear problem);
  - third-order convergence on a nonlinear state;
  - the controller: step sizes scale as tol^(1/3) (an embedded estimate of
    order dt^3), growth is capped at 10x, a rejected attempt is retried from
    q_n and leaves no other trace, and the run lands exactly on t_end.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle as orc
from oracle import Grid, PERIODIC, REFLECTING
from paper_2601_02540_b300 import inputs
import pins

O = orc.default()


def _oscillator(bc, H=0.7, delta=0.01, lam=500.0):
    g = Grid(6, 5, 0.0, 1.0, 0.0, 1.0, bc, 9.81, lam)
    b = np.full((5, 6), -2.0)
    q = np.zeros((5, 5, 6))
    q[0] = H
    q[4] = H + delta
    om2 = lam / H ** 2
    return g, b, q, om2


@pytest.mark.parametrize("bc", [PERIODIC, REFLECTING])
def test_bs3_relaxation_oscillator_closed_form(bc):
    g, b, q, om2 = _oscillator(bc)
    H, delta = 0.7, 0.01
    dt = 0.2 / np.sqrt(om2)
    n = 30
    qn, e = O.bs3_fixed(g, b, q, dt, n)
    Z = dt * np.array([[0.0, 1.0], [-om2, 0.0]])
    P = np.eye(2) + Z + Z @ Z / 2 + Z @ Z @ Z / 6
    y = np.linalg.matrix_power(P, n) @ np.array([delta, 0.0])
    assert np.max(np.abs(qn[4] - H - y[0])) <= 1e-12 * delta
    assert np.max(np.abs(qn[3] - y[1])) <= 1e-12 * delta * np.sqrt(om2)
    assert np.max(np.abs(qn[0] - H)) == 0.0 and np.max(np.abs(qn[1])) == 0.0
    # error estimate of the last step, from y_{n-1}
    yp = np.linalg.matrix_power(P, n - 1) @ np.array([delta, 0.0])
    Z3 = Z @ Z @ Z
    ee = -(Z3 + Z3 @ Z) / 48.0 @ yp
    assert np.max(np.abs(e[4] - ee[0])) <= 1e-10 * abs(ee[0])
    assert np.max(np.abs(e[3] - ee[1])) <= 1e-10 * abs(ee[1])
    assert np.max(np.abs(e[0])) == 0.0


def test_bs3_third_order_convergence():
    p = inputs.smooth_state(16, 12, PERIODIC, seed=2, xmax=4.0, ymax=3.0, lam=50.0)
    g = pins.grid_of(p)
    T = 40 * p.dt
    ref = O.rk4(g, p.b, p.q0, T / 640, 640)
    errs = []
    for n in (20, 40, 80):
        qn, _ = O.bs3_fixed(g, p.b, p.q0, T / n, n)
        errs.append(np.max(np.abs(qn - ref)))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all((rates > 2.8) & (rates < 3.3)), (errs, rates)


def _adaptive_case():
    p = inputs.smooth_state(16, 12, REFLECTING, seed=3, xmax=4.0, ymax=3.0, lam=50.0)
    return p, pins.grid_of(p)


def test_adaptive_lands_on_t_end_and_counts():
    p, g = _adaptive_case()
    T = 30 * p.dt
    q, hist, st = O.rk_adaptive(g, p.b, p.q0, 0.0, T, p.dt, 1e-6, 1e-6)
    assert st["t"] == T
    assert st["accepted"] + st["rejected"] == len(hist)
    acc = hist[hist[:, 2] == 1]
    assert abs(np.sum(acc[:, 0]) - T) <= 1e-12 * T
    assert np.all((acc[:, 1] <= 1.0)) and np.all(hist[hist[:, 2] == 0][:, 1] > 1.0)


def test_adaptive_step_size_scales_as_tol_one_third():
    """err ~ C dt^3 per step, and the controller holds err near 0.9^3: the
    number of steps over a fixed interval grows by 8^(1/3) = 2 when the
    tolerances shrink by 8."""
    p, g = _adaptive_case()
    T = 60 * p.dt
    counts = []
    for tol in (1e-5, 1e-5 / 8, 1e-5 / 64):
        _, hist, st = O.rk_adaptive(g, p.b, p.q0, 0.0, T, p.dt / 50, tol, tol)
        counts.append(st["accepted"])
    ratios = np.array(counts[1:]) / np.array(counts[:-1])
    assert np.all((ratios > 1.7) & (ratios < 2.4)), (counts, ratios)


def test_adaptive_growth_capped_at_ten():
    p, g = _adaptive_case()
    dt0 = p.dt * 1e-5
    _, hist, _ = O.rk_adaptive(g, p.b, p.q0, 0.0, 10 * p.dt, dt0, 1e-6, 1e-6, max_attempts=3)
    # the first attempts are tiny: their error is far below the tolerance
    assert np.all(hist[:, 2] == 1)
    assert np.allclose(hist[:, 0], dt0 * 10.0 ** np.arange(3), rtol=1e-15, atol=0.0)


def test_adaptive_rejection_leaves_no_trace():
    p, g = _adaptive_case()
    T = 20 * p.dt
    q1, hist, st = O.rk_adaptive(g, p.b, p.q0, 0.0, T, 2.5 * p.dt, 1e-7, 1e-7)
    assert hist[0, 2] == 0 and st["rejected"] >= 1
    k = int(np.argmax(hist[:, 2] == 1))          # first accepted attempt
    q2, hist2, _ = O.rk_adaptive(g, p.b, p.q0, 0.0, T, hist[k, 0], 1e-7, 1e-7)
    assert np.array_equal(q1, q2)
    assert np.array_equal(hist[k:], hist2)
