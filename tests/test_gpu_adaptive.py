"""The adaptive integrator (sgn_step_adaptive) against the oracle's
(Sec. 6: third-order FSAL pair with embedded error estimate and step-size
control): the five-stage pair (the paper's kind of integrator) against
oracle.p5_adaptive, and the Bogacki-Shampine pair against oracle.rk_adaptive.

Both sides take their accept/reject decisions and step sizes from their own
error norms, which differ only by rounding (the GPU sums the error in a
different order and evaluates the RHS with FMA); so the attempt histories must
agree: the same decisions, step sizes within 1e-9 relative, error norms within
1e-7 relative, and the final state within the step tolerance 1e-10.
"""
from __future__ import annotations

import ctypes

import numpy as np
import pytest
import torch

import oracle as orc
from oracle import PERIODIC, REFLECTING
from paper_2601_02540_b300 import inputs, sgn
import gpu_util as gu
import pins

pytestmark = pytest.mark.gpu


# Error norms are compared with an absolute floor beside the relative bar: e
# itself carries rounding of about u sum |b_i - bhat_i| |k_i| dt, i.e. up to
# ~1e-13 in units of the tolerance, which dominates a tiny norm (a short step
# cut to land on t_end).
ERR_FLOOR = 1e-12
# The five-stage pair's PI control carries the rounding of err (~1e-10
# relative) into every step size with a memory of the previous step, and the
# last step, cut to land on t_end, absorbs the accumulated time: over N ~ 200
# accepted steps the step sizes agree to ~N x 1e-11 ~ 1e-8 relative.
P5_BARS = dict(dt_tol=1e-8)


def _compare(p, q0, T, dt0, rtol=1e-6, atol=1e-6, prec="f64", dt_tol=1e-9, err_tol=1e-7, pair="bs3",
             state_tol=gu.STEP_TOL):
    g = pins.grid_of(p)
    oracle_run = orc.rk_adaptive if pair == "bs3" else orc.p5_adaptive
    qo, ho, so = oracle_run(g, p.b, q0, 0.0, T, dt0, rtol, atol)
    s = gu.solver(p, prec)
    q = s.state(q0)
    st, hist = s.step_adaptive(q, 0.0, T, dt0, rtol, atol, pair=pair)
    s.close()
    hg = np.array(hist)
    assert st["attempts"] == len(ho) and st["accepted"] == so["accepted"] and st["rejected"] == so["rejected"]
    assert st["t"] == so["t"] == T
    assert np.array_equal(hg[:, 2], ho[:, 2])
    assert np.all(np.abs(hg[:, 0] - ho[:, 0]) <= dt_tol * ho[:, 0])
    assert np.all(np.abs(hg[:, 1] - ho[:, 1]) <= err_tol * ho[:, 1] + ERR_FLOOR)
    e = gu.state_errors(gu.to_np(q), qo)
    assert np.all(e <= state_tol), e
    return st, hg


@pytest.mark.parametrize("bc", [PERIODIC, REFLECTING])
@pytest.mark.parametrize("nx,ny", [(33, 17), (100, 37)])
def test_adaptive_matches_oracle_generic(bc, nx, ny):
    p = inputs.smooth_state(nx, ny, bc, seed=11, xmax=4.0, ymax=3.0, lam=50.0)
    _compare(p, p.q0, 30 * p.dt, p.dt)


def test_adaptive_matches_oracle_workload1():
    """Periodic 64^2 hump (workload 1) over its whole run time, 200 RK4 steps
    of the fixed-step workload, paper tolerances rtol = atol = 1e-6."""
    p = inputs.workload1()
    g = pins.grid_of(p)
    q0 = orc.init_aux(g, p.b, p.q0)
    st, _ = _compare(p, q0, p.nsteps * p.dt, p.dt)
    assert st["accepted"] > 10


def test_adaptive_rejection_path_matches_oracle():
    """A first step far above the stable size is rejected on both sides."""
    p = inputs.smooth_state(40, 23, REFLECTING, seed=12, xmax=4.0, ymax=3.0, lam=50.0)
    st, hg = _compare(p, p.q0, 20 * p.dt, 2.5 * p.dt, 1e-7, 1e-7)
    assert hg[0, 2] == 0 and st["rejected"] >= 1


def test_adaptive_workload2_reduced_matches_oracle():
    p = inputs.workload2(200, 100)
    g = pins.grid_of(p)
    q0 = orc.init_aux(g, p.b, p.q0)
    _compare(p, q0, 40 * p.dt, p.dt)


def test_adaptive_only_f64_and_bad_arguments():
    p = inputs.smooth_state(16, 9, PERIODIC, seed=2)
    s = gu.solver(p, "f32")
    q = torch.as_tensor(p.q0, dtype=torch.float64, device="cuda")   # the library checks the context
    with pytest.raises(sgn.SgnError) as ei:
        s.step_adaptive(q, 0.0, 1.0, 0.1)
    assert ei.value.status == 7      # SGN_E_UNSUPPORTED
    s.close()
    s = gu.solver(p)
    q = s.state(p.q0)
    for args in ((1.0, 0.0, 0.1), (0.0, 1.0, 0.0), (0.0, 1.0, 0.1, 0.0, 0.0)):
        with pytest.raises(sgn.SgnError) as ei:
            s.step_adaptive(q, *args)
        assert ei.value.status == 1  # SGN_E_INVAL
    with pytest.raises(KeyError):
        s.step_adaptive(q, 0.0, 1.0, 0.1, pair="rk45")
    assert sgn.lib().sgn_step_adaptive(s.ctx, ctypes.c_void_p(q.data_ptr()), 0.0, 1.0, 0.1, 1e-6, 1e-6,
                                       10, 7, None, (ctypes.c_double * 5)(), None) == 1   # unknown pair
    st, hist = s.step_adaptive(q, 0.5, 0.5, 0.1)   # empty interval: no attempt
    assert st["attempts"] == 0 and torch.equal(q, s.state(p.q0))
    s.close()


def test_adaptive_nonpositive_initial_state_is_reported():
    p = inputs.smooth_state(16, 9, REFLECTING, seed=2)
    q0 = p.q0.copy()
    q0[0, 3, 4] = -0.5
    s = gu.solver(p)
    q = s.state(q0)
    with pytest.raises(sgn.SgnError) as ei:
        s.step_adaptive(q, 0.0, 1.0, 0.1)
    assert ei.value.status == 4      # SGN_E_NONPOSITIVE_H
    st, _ = s.step_adaptive(s.state(p.q0), 0.0, 2 * p.dt, p.dt)   # the context stays usable
    assert st["t"] == 2 * p.dt
    s.close()


# The float-pair RHS has the rounding unit 2^-48.  The error estimate e is a
# combination of the stage slopes that cancels to ~1e-6 of them, so its relative
# rounding is about 2^-48 |k| / |e| ~ 4e-9, and the step sizes, fed back
# through the controller, drift apart by up to ~1e-8 over a hundred attempts:
# the df64 bars are 1e-7 on the step sizes and 1e-5 on the error norms, with
# the same decisions and the df64 step bar on the final state.
DF64_BARS = dict(dt_tol=1e-7, err_tol=1e-5, state_tol=gu.STEP_TOL_DF64)


@pytest.mark.parametrize("bc", [PERIODIC, REFLECTING])
def test_adaptive_df64_matches_oracle(bc):
    p = inputs.smooth_state(100, 37, bc, seed=11, xmax=4.0, ymax=3.0, lam=50.0)
    _compare(p, p.q0, 30 * p.dt, p.dt, prec="df64", **DF64_BARS)


def test_adaptive_df64_workload1_matches_oracle():
    p = inputs.workload1()
    g = pins.grid_of(p)
    q0 = orc.init_aux(g, p.b, p.q0)
    _compare(p, q0, p.nsteps * p.dt, p.dt, prec="df64", **DF64_BARS)


# ------------------------------------------------------------------ the five-stage pair
@pytest.mark.parametrize("bc", [PERIODIC, REFLECTING])
@pytest.mark.parametrize("nx,ny", [(33, 17), (100, 37)])
def test_p5_matches_oracle_generic(bc, nx, ny):
    p = inputs.smooth_state(nx, ny, bc, seed=11, xmax=4.0, ymax=3.0, lam=50.0)
    _compare(p, p.q0, 30 * p.dt, p.dt, pair="p5s3", **P5_BARS)


def test_p5_matches_oracle_workload1():
    """Periodic 64^2 hump over the fixed-step workload's run time, paper
    tolerances rtol = atol = 1e-6."""
    p = inputs.workload1()
    g = pins.grid_of(p)
    q0 = orc.init_aux(g, p.b, p.q0)
    st, _ = _compare(p, q0, p.nsteps * p.dt, p.dt, pair="p5s3", **P5_BARS)
    assert st["accepted"] > 10


def test_p5_rejection_path_matches_oracle():
    p = inputs.smooth_state(40, 23, REFLECTING, seed=12, xmax=4.0, ymax=3.0, lam=50.0)
    st, hg = _compare(p, p.q0, 20 * p.dt, 6.0 * p.dt, 1e-7, 1e-7, pair="p5s3", **P5_BARS)
    assert hg[0, 2] == 0 and st["rejected"] >= 1


def test_p5_workload2_reduced_matches_oracle():
    p = inputs.workload2(200, 100)
    g = pins.grid_of(p)
    q0 = orc.init_aux(g, p.b, p.q0)
    _compare(p, q0, 40 * p.dt, p.dt, pair="p5s3", **P5_BARS)


@pytest.mark.parametrize("bc", [PERIODIC, REFLECTING])
def test_p5_df64_matches_oracle(bc):
    p = inputs.smooth_state(100, 37, bc, seed=11, xmax=4.0, ymax=3.0, lam=50.0)
    _compare(p, p.q0, 30 * p.dt, p.dt, prec="df64", pair="p5s3", **DF64_BARS)


def test_p5_df64_workload1_matches_oracle():
    p = inputs.workload1()
    g = pins.grid_of(p)
    q0 = orc.init_aux(g, p.b, p.q0)
    _compare(p, q0, p.nsteps * p.dt, p.dt, prec="df64", pair="p5s3", **DF64_BARS)
