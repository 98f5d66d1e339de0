"""Pins of the oracle's five-stage third-order FSAL pair (Sec. 6: an explicit
third-order, five-stage Runge-Kutta method with the first-same-as-last
property and an embedded error estimator, optimized for stability-limited
hyperbolic problems; the paper does not print its coefficients, and the pair
here was constructed to have those properties).

What fixes the values:
  - the design statement: third order (four conditions), the stability
    polynomial R(z) = 1 + z + z^2/2 + z^3/6 + 0.0324 z^4 + 0.006 z^5, which
    keeps |R(iy)| <= 1 up to |y| = 3.8798, the two-register structure
    a_ij = b_j (j < i - 1), an embedded second-order solution over the five
    stages and f(q_{n+1}) that is stable on the same interval;
  - the relaxation oscillator (flat b, uniform h = H, u = v = w = 0,
    eta = H + delta) is an exact linear system for (eta - H, w) with
    Z = dt [[0, 1], [-lam/H^2, 0]]: a step is R(Z), and the error estimate of
    a step from y is (R(Z) - Rhat(Z)) y with Rhat the embedded method's
    polynomial, formed here from the tableau by matrix powers (not by stages);
  - third-order convergence on a nonlinear state;
  - the controller: the step sizes of a run follow the PI rule with the
    atan limiter from the recorded errors, they scale as tol^(1/3), a rejected
    attempt is retried from q_n and leaves no other trace, the run lands
    exactly on t_end, and on a smooth problem it holds err near its target 0.9.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle as orc
from oracle import Grid, PERIODIC, REFLECTING
from paper_2601_02540_b300 import inputs
import pins

O = orc.default()
G4, G5 = 0.0324, 0.006
BETA = 3.8798


def _tableau():
    A, b, bh = O.p5_tableau()
    c = A.sum(axis=1)
    At = np.zeros((6, 6))
    At[:5, :5] = A
    At[5, :5] = b
    return A, b, bh, c, At, At.sum(axis=1)


def _R(y):
    z = 1j * np.asarray(y)
    return 1 + z + z ** 2 / 2 + z ** 3 / 6 + G4 * z ** 4 + G5 * z ** 5


def _series(M, w, n):
    """Coefficients w^T M^(k-1) 1, k = 1..n, of a method's stability polynomial."""
    one = np.ones(M.shape[0])
    return np.array([w @ np.linalg.matrix_power(M, k - 1) @ one for k in range(1, n + 1)])


def test_p5_tableau_order_structure_and_stability():
    A, b, bh, c, At, ct = _tableau()
    assert np.all(np.triu(A) == 0.0)                       # explicit
    for i in range(2, 5):                                  # two-register form
        assert np.all(A[i, : i - 1] == b[: i - 1])
    tol = 1e-15
    assert abs(b.sum() - 1) <= tol
    assert abs(b @ c - 1 / 2) <= tol
    assert abs(b @ c ** 2 - 1 / 3) <= tol
    assert abs(b @ A @ c - 1 / 6) <= tol
    m = _series(A, b, 5)
    assert np.allclose(m, [1, 1 / 2, 1 / 6, G4, G5], rtol=0, atol=1e-15), m
    # embedded: order 2 exactly (the third-order condition is missed by a clear margin)
    assert abs(bh.sum() - 1) <= tol and abs(bh @ ct - 1 / 2) <= tol
    assert abs(bh @ At @ ct - 1 / 6) > 0.05
    # imaginary-axis stability of the method and of its embedded solution
    y = np.linspace(0.0, BETA, 20001)
    assert np.all(np.abs(_R(y)) <= 1 + 1e-14)
    assert abs(_R(3.9)) > 1
    mh = _series(At, bh, 6)
    Rh = 1 + sum(mh[k] * (1j * y) ** (k + 1) for k in range(6))
    assert np.all(np.abs(Rh) <= 1 + 1e-14)
    # fourth-order error coefficients (accuracy of the design)
    t4 = [(b @ c ** 3 - 1 / 4) / 6, b @ (c * (A @ c)) - 1 / 8, (b @ A @ c ** 2 - 1 / 12) / 2, G4 - 1 / 24]
    assert np.sqrt(np.sum(np.square(t4))) < 0.0096


def _oscillator(bc, H=0.7, delta=0.01, lam=500.0):
    g = Grid(6, 5, 0.0, 1.0, 0.0, 1.0, bc, 9.81, lam)
    b = np.full((5, 6), -2.0)
    q = np.zeros((5, 5, 6))
    q[0] = H
    q[4] = H + delta
    return g, b, q, lam / H ** 2


def _poly(Z, coef):
    out = np.eye(2)
    Zk = np.eye(2)
    for a in coef:
        Zk = Zk @ Z
        out = out + a * Zk
    return out


@pytest.mark.parametrize("bc", [PERIODIC, REFLECTING])
@pytest.mark.parametrize("wdt", [0.3, 3.8])
def test_p5_relaxation_oscillator_closed_form(bc, wdt):
    """Steps of the pair on an exact linear system equal powers of R(Z), up to
    omega dt = 3.8 (near the edge of the stability interval), and the error
    estimate equals (R(Z) - Rhat(Z)) y."""
    A, b, bh, c, At, ct = _tableau()
    g, bb, q, om2 = _oscillator(bc)
    H, delta = 0.7, 0.01
    dt = wdt / np.sqrt(om2)
    n = 25
    qn, e = O.p5_fixed(g, bb, q, dt, n)
    Z = dt * np.array([[0.0, 1.0], [-om2, 0.0]])
    P = _poly(Z, [1, 1 / 2, 1 / 6, G4, G5])
    y = np.linalg.matrix_power(P, n) @ np.array([delta, 0.0])
    assert np.max(np.abs(qn[4] - H - y[0])) <= 1e-11 * delta
    assert np.max(np.abs(qn[3] - y[1])) <= 1e-11 * delta * np.sqrt(om2)
    assert np.max(np.abs(qn[0] - H)) == 0.0 and np.max(np.abs(qn[1])) == 0.0
    assert np.hypot(y[0], y[1] / np.sqrt(om2)) <= delta * (1 + 1e-12)      # |R| <= 1: no growth
    yp = np.linalg.matrix_power(P, n - 1) @ np.array([delta, 0.0])
    ee = (P - _poly(Z, _series(At, bh, 6))) @ yp
    assert np.max(np.abs(e[4] - ee[0])) <= 1e-9 * np.max(np.abs(ee))
    assert np.max(np.abs(e[3] - ee[1])) <= 1e-9 * np.max(np.abs(ee))


def test_p5_unstable_beyond_the_interval():
    """At omega dt = 4.0 (outside 3.8798) the oscillation grows as |R(4i)|^n."""
    g, bb, q, om2 = _oscillator(PERIODIC)
    dt = 4.0 / np.sqrt(om2)
    n = 40
    qn, _ = O.p5_fixed(g, bb, q, dt, n)
    amp = np.hypot(qn[4, 0, 0] - 0.7, qn[3, 0, 0] / np.sqrt(om2)) / 0.01
    assert amp > 0.5 * abs(_R(4.0)) ** n > 1e3


def test_p5_third_order_convergence():
    p = inputs.smooth_state(16, 12, PERIODIC, seed=2, xmax=4.0, ymax=3.0, lam=50.0)
    g = pins.grid_of(p)
    T = 40 * p.dt
    ref = O.rk4(g, p.b, p.q0, T / 640, 640)
    errs = []
    for n in (20, 40, 80):
        qn, _ = O.p5_fixed(g, p.b, p.q0, T / n, n)
        errs.append(np.max(np.abs(qn - ref)))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all((rates > 2.8) & (rates < 3.3)), (errs, rates)


def _adaptive_case():
    p = inputs.smooth_state(16, 12, REFLECTING, seed=3, xmax=4.0, ymax=3.0, lam=50.0)
    return p, pins.grid_of(p)


def _pi_factor(err, eps_prev):
    eps = 0.9 / max(err, 1e-10)
    x = eps ** (0.7 / 3.0) * eps_prev ** (-0.4 / 3.0) if err <= 1.0 else eps ** (1.0 / 3.0)
    return 1.0 + np.arctan(x - 1.0), eps


def test_p5_adaptive_follows_the_pi_rule_and_lands_on_t_end():
    p, g = _adaptive_case()
    T = 30 * p.dt
    q, hist, st = O.p5_adaptive(g, p.b, p.q0, 0.0, T, p.dt, 1e-6, 1e-6)
    # the controller aims at err = 0.9: the accepted attempts sit near it and
    # rejections (the local error varies from step to step) stay rare
    assert st["rejected"] <= 0.2 * len(hist), st
    assert abs(np.median(hist[hist[:, 2] == 1][:, 1]) - 0.9) < 0.1
    assert st["t"] == T
    assert st["accepted"] + st["rejected"] == len(hist)
    acc = hist[hist[:, 2] == 1]
    assert abs(np.sum(acc[:, 0]) - T) <= 1e-12 * T
    assert np.all(acc[:, 1] <= 1.0) and np.all(hist[hist[:, 2] == 0][:, 1] > 1.0)
    # every step size from the previous attempt's size and error (the last
    # accepted one cut to land on T is the only exception)
    eps_prev = 1.0
    t = 0.0
    dt_next = p.dt
    for h, err, ok in hist:
        if t + dt_next < T:
            assert h == dt_next or abs(h - dt_next) <= 1e-15 * dt_next, (h, dt_next)
        fac, eps = _pi_factor(err, eps_prev)
        dt_next = h * fac
        if ok:
            t += h
            eps_prev = eps
    assert abs(st["dt_next"] - dt_next) <= 1e-14 * dt_next


def test_p5_adaptive_step_size_scales_as_tol_one_third():
    p, g = _adaptive_case()
    T = 60 * p.dt
    counts = []
    for tol in (1e-5, 1e-5 / 8, 1e-5 / 64):
        _, hist, st = O.p5_adaptive(g, p.b, p.q0, 0.0, T, p.dt / 50, tol, tol)
        counts.append(st["accepted"])
    ratios = np.array(counts[1:]) / np.array(counts[:-1])
    assert np.all((ratios > 1.7) & (ratios < 2.4)), (counts, ratios)


def test_p5_adaptive_growth_is_limited():
    """Tiny first steps: err is below the 1e-10 floor, so the factor is
    1 + atan(x - 1) with x = (0.9e10)^(0.7/3) eps_prev^(-0.4/3): below 1 + pi/2."""
    p, g = _adaptive_case()
    dt0 = p.dt * 1e-6
    _, hist, _ = O.p5_adaptive(g, p.b, p.q0, 0.0, 10 * p.dt, dt0, 1e-6, 1e-6, max_attempts=3)
    assert np.all(hist[:, 2] == 1)
    eps_prev, h = 1.0, dt0
    for k in range(3):
        assert abs(hist[k, 0] - h) <= 1e-15 * h
        fac, eps_prev = _pi_factor(hist[k, 1], eps_prev)
        assert 1.0 < fac < 1 + np.pi / 2
        h *= fac


def test_p5_adaptive_rejection_leaves_no_trace():
    p, g = _adaptive_case()
    T = 20 * p.dt
    q1, hist, st = O.p5_adaptive(g, p.b, p.q0, 0.0, T, 6.0 * p.dt, 1e-7, 1e-7)
    assert hist[0, 2] == 0 and st["rejected"] >= 1
    k = int(np.argmax(hist[:, 2] == 1))          # first accepted attempt
    q2, hist2, _ = O.p5_adaptive(g, p.b, p.q0, 0.0, T, hist[k, 0], 1e-7, 1e-7)
    assert np.array_equal(q1, q2)
    assert np.array_equal(hist[k:], hist2)
