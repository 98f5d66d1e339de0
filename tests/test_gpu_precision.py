"""The FP32 and mixed-precision paths against the FP64 oracle.

Both evaluate the same split-form RHS (eq. (sd_periodic_2D_SGN) / (semi_2D))
in float arithmetic, so their error is float rounding.  The bounds are stated
in units of u32 = 2^-24 and are evaluated at the float-rounded state and
bathymetry, so that the rounding of the inputs themselves is not counted:

  RHS     ||gpu_f - orc_f||_inf <= MULT u32 (||S_f||_inf + ||orc_f||_inf)
          with S_f the oracle's forward rounding-error scale of that RHS value
          (each term coef * D f counted as |coef| |D| |f|), MULT = 32: a few
          roundings per term plus the float-rounded grid constants.
  n steps (each step rounds the stage states, and in FP32 also q and the RK
          accumulator, to float; errors are summed without cancellation and
          given a factor 2 for their propagation over the short run)
          FP32:  ||dq_f|| <= 2 n (4 u32 ||q_f|| + dt MULT u32 (||S_f|| + ||k_f||))
          mixed: ||dq_f|| <= 2 n dt MULT u32 (||S_f|| + ||k_f||)
          (a stage state rounded to float, relative u32, moves the RHS by about
          u32 S: the same term as the float evaluation itself).
The mixed path keeps q_n and the accumulator in double, so its error carries
no n u32 ||q|| term: it is asserted to be well below the FP32 error.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle as orc
from oracle import PERIODIC, REFLECTING
from paper_2601_02540_b300 import inputs, sgn
import gpu_util as gu
import pins

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24
MULT = 32.0


def _f32(a: np.ndarray) -> np.ndarray:
    return a.astype(np.float32).astype(np.float64)


def _rounded(p: inputs.Problem) -> inputs.Problem:
    p.b = _f32(p.b)
    p.q0 = _f32(p.q0)
    return p


def _fieldmax(a: np.ndarray) -> np.ndarray:
    return np.max(np.abs(a), axis=(1, 2))


@pytest.mark.parametrize("prec", ["f32", "f32_f64acc"])
@pytest.mark.parametrize("bc", [PERIODIC, REFLECTING])
@pytest.mark.parametrize("nx,ny", [(5, 3), (33, 17), (100, 37)])
def test_rhs_within_float_rounding_bound(prec, bc, nx, ny):
    p = _rounded(inputs.smooth_state(nx, ny, bc, seed=3, xmax=1.3, ymax=0.9))
    s = gu.solver(p, prec)
    dq = gu.to_np(s.rhs(s.state(p.q0)))
    ref, sc = gu.oracle_rhs_and_scale(p, p.q0)
    err = _fieldmax(dq - ref)
    allow = MULT * U32 * (np.max(sc, axis=(1, 2)) + _fieldmax(ref))
    assert np.all(err <= allow), (err / allow)
    s.close()


@pytest.mark.parametrize("prec", ["f32", "f32_f64acc"])
def test_rhs_workload_state_within_float_rounding_bound(prec):
    """Reflecting bathymetry workload (1024x512 recipe at 200x100), at its
    initial state and after 5 oracle steps, h + b near 0 (still water)."""
    p = inputs.workload2(200, 100)
    g = pins.grid_of(p)
    p.b = _f32(p.b)
    q0 = orc.init_aux(g, p.b, _f32(p.q0))
    s = gu.solver(p, prec)
    for q in (_f32(q0), _f32(orc.rk4(g, p.b, q0, p.dt, 5))):
        dq = gu.to_np(s.rhs(s.state(q)))
        ref, sc = gu.oracle_rhs_and_scale(p, q)
        err = _fieldmax(dq - ref)
        allow = MULT * U32 * (np.max(sc, axis=(1, 2)) + _fieldmax(ref))
        assert np.all(err <= allow), (err / allow)
    s.close()


@pytest.mark.parametrize("bc", [PERIODIC, REFLECTING])
def test_steps_float_and_mixed_error_bounds(bc):
    p = _rounded(inputs.smooth_state(64, 48, bc, seed=5, xmax=1.3, ymax=0.9))
    g = pins.grid_of(p)
    n = 100
    ref = orc.rk4(g, p.b, p.q0, p.dt, n)
    # RHS scales at the start and the end of the run
    S = np.maximum(np.max(orc.rhs_scale(g, p.b, p.q0), axis=(1, 2)),
                   np.max(orc.rhs_scale(g, p.b, ref), axis=(1, 2)))
    K = np.maximum(_fieldmax(orc.rhs(g, p.b, p.q0)), _fieldmax(orc.rhs(g, p.b, ref)))
    Q = np.maximum(_fieldmax(p.q0), _fieldmax(ref))
    errs = {}
    for prec in ("f32", "f32_f64acc"):
        s = gu.solver(p, prec)
        q = s.state(p.q0)
        s.step(q, p.dt, n)
        errs[prec] = _fieldmax(gu.to_np(q) - ref)
        s.close()
    allow32 = 2 * n * (4 * U32 * Q + p.dt * MULT * U32 * (S + K))
    allow_mix = 2 * n * p.dt * MULT * U32 * (S + K)
    assert np.all(errs["f32"] <= allow32), errs["f32"] / allow32
    assert np.all(errs["f32_f64acc"] <= allow_mix), errs["f32_f64acc"] / allow_mix
    # the double accumulator removes the per-step rounding of q itself
    assert errs["f32_f64acc"][0] < 0.5 * errs["f32"][0], (errs["f32_f64acc"], errs["f32"])


def test_mixed_mass_drift_below_float():
    """Reflecting walls conserve 1^T M h exactly up to rounding (SAT, Thm.
    4.2): with q_n and the accumulator in double, the mixed path's mass drift
    is far below the FP32 path's."""
    p = _rounded(inputs.smooth_state(64, 48, REFLECTING, seed=6, xmax=1.3, ymax=0.9))
    drift = {}
    for prec in ("f32", "f32_f64acc", "f64"):
        s = gu.solver(p, prec)
        q = s.state(p.q0)
        m0 = s.mass_energy(q)["mass"]
        s.step(q, p.dt, 200)
        m1 = s.mass_energy(q)["mass"]
        drift[prec] = abs(m1 - m0) / abs(m0)
        s.close()
    assert drift["f64"] <= 1e-13, drift
    assert drift["f32_f64acc"] < 0.1 * drift["f32"] or drift["f32_f64acc"] <= 1e-10, drift


def test_workload2_2000_steps_float_and_mixed_vs_oracle():
    """The reflecting-wall workload as stated: 1024x512, 2000 RK4 steps in FP32
    (float state and RHS, FP64 reductions) and in the mixed mode (float RHS,
    q_n and the accumulator in double), against the FP64 oracle's stored run
    (tests/golden/workload2_2000.txt).  The errors at the sampled nodes are
    held to the a-priori bounds of the module docstring with n = 2000 and S,
    K, Q the larger of the oracle's initial and final values (the FP32 bound's
    n u32 ||q|| term also covers rounding the double initial state to float);
    the errors reached and the energy drift (E' = E + g b^2/2, whose constant
    offset is left out) of each run are reported beside the oracle's drift."""
    p = inputs.workload2()
    gd = gu.workload2_golden(p)
    n = p.nsteps
    S = np.maximum(gd["S_initial"], gd["S_final"])
    K = np.maximum(gd["k_initial"], gd["k_final"])
    Q = np.maximum(_fieldmax(gd["q0"]), gd["maxnorm"])
    den = np.maximum(gd["maxnorm"], 1e-3 * gd["maxnorm"][0])
    orc_drift = abs(gd["diag_final"][2] - gd["diag_initial"][2]) / abs(gd["diag_initial"][2])
    allow = {"f32": 2 * n * (4 * U32 * Q + p.dt * MULT * U32 * (S + K)),
             "f32_f64acc": 2 * n * p.dt * MULT * U32 * (S + K)}
    errs = {}
    for prec in ("f32", "f32_f64acc"):
        s = gu.solver(p, prec)
        q = s.state(gd["q0"])
        e0 = s.mass_energy(q)["energy_shifted"]
        s.step(q, p.dt, n)
        e1 = s.mass_energy(q)["energy_shifted"]
        out = gu.to_np(q)
        s.close()
        errs[prec] = np.max(np.abs(out[:, gd["j"], gd["i"]] - gd["values"]), axis=1)
        gu.report(f"{prec} steps workload2 1024x512 x2000 vs oracle (sampled)",
                  rel_err=errs[prec] / den, err_over_allow=errs[prec] / allow[prec],
                  energy_drift=abs(e1 - e0) / abs(e0), oracle_energy_drift=orc_drift)
    for prec in errs:
        assert np.all(errs[prec] <= allow[prec]), (prec, errs[prec] / allow[prec])
    assert errs["f32_f64acc"][0] < errs["f32"][0], errs


@pytest.mark.parametrize("bc", [PERIODIC, REFLECTING])
@pytest.mark.parametrize("nx,ny,nsteps", [(3, 3, 3), (5, 4, 2), (33, 17, 7), (100, 37, 4),
                                          (130, 70, 60), (1000, 515, 3)])
def test_fp32_stage_fusion_equals_one_stage_per_launch(bc, nx, ny, nsteps):
    """Two RK4 stages per launch (the first of each pair evaluated on the tile
    grown by one node, its result kept in shared memory) give the states of
    one launch per stage bit for bit: grids smaller than a tile, ragged tiles,
    odd step counts (the result copied back from the scratch state) and a
    50-step graph replay (130 x 70, 60 steps)."""
    p = inputs.smooth_state(nx, ny, bc, seed=41, xmax=1.3, ymax=0.9)
    s = gu.solver(p, "f32")
    s.set_stage_fusion(False)
    q1 = s.state(p.q0)
    s.step(q1, p.dt, nsteps)
    s.set_stage_fusion(True)
    q2 = s.state(p.q0)
    s.step(q2, p.dt, nsteps)
    assert torch.equal(q1, q2)
    q3 = s.state(p.q0)
    for _ in range(nsteps):
        s.step(q3, p.dt, 1)
    assert torch.equal(q1, q3)
    s.check()
    s.close()


def test_stage_fusion_is_for_fp32():
    p = inputs.smooth_state(16, 9, PERIODIC, seed=2)
    for prec in ("f64", "f32_f64acc", "df64"):
        s = gu.solver(p, prec)
        with pytest.raises(sgn.SgnError) as ei:
            s.set_stage_fusion(True)
        assert ei.value.status == 7          # SGN_E_UNSUPPORTED
        s.close()


@pytest.mark.parametrize("bc", [PERIODIC, REFLECTING])
@pytest.mark.parametrize("j,i", [(0, 0), (7, 31), (16, 32), (15, 63), (40, 77), (69, 129)])
def test_fp32_two_stage_step_reports_bad_water_height(bc, j, i):
    """The two-stage FP32 launches check h where they stage it: a negative or
    NaN water height at a grid corner, on a tile's edge or corner, or inside
    a tile is reported after one step (non-positive: status 4, non-finite:
    5), and the flag is cleared by the report."""
    p = inputs.smooth_state(130, 70, bc, seed=3)
    s = gu.solver(p, "f32")
    for val, status in ((-0.5, 4), (float("nan"), 5)):
        q = s.state(p.q0)
        q[0, j, i] = val
        s.step(q, p.dt, 1)
        with pytest.raises(sgn.SgnError) as ei:
            s.check()
        assert ei.value.status == status, (val, ei.value.status)
    q = s.state(p.q0)
    s.step(q, p.dt, 1)
    s.check()
    s.close()
