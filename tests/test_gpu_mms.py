"""The manufactured solution of Sec. 6.1.2 on the GPU.

The library evaluates the manufactured fields and their source terms by
forward-mode differentiation in CUDA; the tests compare them with sympy's
symbolic derivation (tests/continuum.py), run the forced RK4 against the
oracle's split-form RHS plus the sympy sources, and repeat the paper's
convergence study ([-1,1]^2, lambda = 500, t = 1, both boundary treatments):
second order in h, u, v, w and eta in the discrete L2 norm of the mass matrix
M (the max norm: second order when periodic, about 1.5 with reflecting walls,
whose one-sided boundary rows are first-order accurate).
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import continuum as cont
import oracle as orc
from oracle import Grid, PERIODIC, REFLECTING
from paper_2601_02540_b300 import sgn
import gpu_util as gu

pytestmark = pytest.mark.gpu

_FNS = None


def _fns():
    global _FNS
    if _FNS is None:
        fields, src = cont.manufactured()
        _FNS = cont.lambdify_fields(tuple(fields) + tuple(src))
    return _FNS


def _setup(bc, nx, ny):
    g = Grid(nx, ny, -1.0, 1.0, -1.0, 1.0, bc, 9.81, 500.0)
    xs, ys = g.nodes()
    X, Y = np.meshgrid(xs, ys)
    s = sgn.Solver(nx, ny, -1.0, 1.0, -1.0, 1.0, bc, torch.zeros((ny, nx), dtype=torch.float64, device="cuda"),
                   9.81, 500.0)
    q, b = s.mms_exact(0.0, with_b=True)
    s.set_bathymetry(b)
    return g, X, Y, s, q, b


@pytest.mark.parametrize("bc", [PERIODIC, REFLECTING])
def test_mms_fields_and_sources_match_sympy(bc):
    g, X, Y, s, q0, b = _setup(bc, 33, 17)
    fns = _fns()
    assert np.max(np.abs(gu.to_np(b) - cont.evaluate(fns[:1], X, Y, 0.0)[0])) <= 1e-15
    for t in (0.0, 0.3, 0.77):
        ex = cont.evaluate(fns[1:6], X, Y, t)
        got = gu.to_np(s.mms_exact(t))
        assert np.max(np.abs(got - ex)) <= 1e-13 * np.max(np.abs(ex))
        S = cont.evaluate(fns[6:], X, Y, t)
        Sg = gu.to_np(s.mms_source(t))
        err = np.max(np.abs(Sg - S), axis=(1, 2))
        assert np.all(err <= 1e-12 * np.max(np.abs(S), axis=(1, 2)) + 1e-12), (err, np.max(np.abs(S), axis=(1, 2)))
    s.close()


@pytest.mark.parametrize("bc", [PERIODIC, REFLECTING])
def test_mms_forced_steps_match_oracle(bc):
    """20 forced RK4 steps: GPU (fused stages, CUDA sources) against the
    oracle's RHS plus the sympy sources at the same stage times."""
    g, X, Y, s, q0, b = _setup(bc, 40, 23)
    fns = _fns()
    bn = gu.to_np(b)
    dt, n, t0 = 2e-3, 20, 0.1
    q = s.mms_exact(t0)
    qo = gu.to_np(q)
    s.step_mms(q, t0, dt, n)

    def src(tt):
        return cont.evaluate(fns[6:], X, Y, tt)

    t = t0
    for _ in range(n):
        k1 = orc.rhs(g, bn, qo) + src(t)
        k2 = orc.rhs(g, bn, qo + dt / 2 * k1) + src(t + dt / 2)
        k3 = orc.rhs(g, bn, qo + dt / 2 * k2) + src(t + dt / 2)
        k4 = orc.rhs(g, bn, qo + dt * k3) + src(t + dt)
        qo = qo + dt / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
        t += dt
    e = gu.state_errors(gu.to_np(q), qo)
    assert np.all(e <= gu.STEP_TOL), e
    s.close()


def _gpu_mms_error(bc, n, t_end=1.0):
    g, X, Y, s, q0, b = _setup(bc, n, n)
    dx, _ = g.spacing()
    c = 0.3 + np.sqrt(9.81 * 2.7 + 500.0 / 3.0)
    nsteps = int(np.ceil(t_end / (0.3 * dx / c)))
    dt = t_end / nsteps
    q = q0.clone()
    s.step_mms(q, 0.0, dt, nsteps)
    e = gu.to_np(q - s.mms_exact(t_end))
    s.close()
    M = orc.mass_weights(g)
    l2 = np.sqrt(np.sum(M * e * e, axis=(1, 2)) / np.sum(M))
    return l2, np.max(np.abs(e), axis=(1, 2))


@pytest.mark.parametrize("bc", [PERIODIC, REFLECTING])
def test_mms_second_order_convergence_to_t1(bc):
    """The paper's study (Sec. 6.1.2): second-order convergence in all five
    variables at t = 1 for both boundary treatments."""
    res = [_gpu_mms_error(bc, n) for n in (32, 64, 128, 256)]
    l2 = np.array([r[0] for r in res])
    mx = np.array([r[1] for r in res])
    orders = np.log2(l2[:-1] / l2[1:])
    assert np.all(orders[-1] > 1.8) and np.all(orders[-1] < 2.3), (orders, l2)
    # max norm: second order with periodic boundaries; the one-sided first-order
    # boundary rows of the reflecting operator leave O(dx^1.5) at the walls
    omax = np.log2(mx[-2] / mx[-1])
    assert np.all(omax > (1.8 if bc == PERIODIC else 1.4)), (omax, mx)


def test_mms_only_f64():
    s = sgn.Solver(16, 16, -1.0, 1.0, -1.0, 1.0, PERIODIC,
                   torch.zeros((16, 16), dtype=torch.float64, device="cuda"), prec="f32")
    q = torch.zeros((5, 16, 16), dtype=torch.float64, device="cuda")
    with pytest.raises(sgn.SgnError) as ei:
        s.step_mms(q, 0.0, 1e-3, 1)
    assert ei.value.status == 7      # SGN_E_UNSUPPORTED
    s.close()
