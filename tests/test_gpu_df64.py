"""The double-word (df64) precision mode against the FP64 oracle.

The RHS is evaluated in float-pair arithmetic with about 48 significant bits,
so its rounding unit is u_dw = 2^-48 instead of u = 2^-53, and the bar is the
FP64 parity bar with that unit:
  RHS    ||gpu_f - orc_f||_inf <= 1e-12 ||orc_f||_inf + 16 u_dw ||S_f||_inf
  steps  the FP64 step bar (1e-10 relative) on short runs, the state and the
         RK accumulator being double; on the 2000-step workload the bar scaled
         by the ratio of the rounding units, 2^5 (gpu_util.STEP_TOL_DF64), since
         rounding errors accumulated over a run scale with the unit
The diagnostics of a df64 context are those of its double state (equal to an
FP64 context's bit for bit).
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle as orc
from oracle import PERIODIC, REFLECTING
from paper_2601_02540_b300 import inputs
import gpu_util as gu
import pins

pytestmark = pytest.mark.gpu

U_DW = 2.0 ** -48


def _rhs_err(dq, ref, sc):
    err = np.max(np.abs(dq - ref), axis=(1, 2))
    allow = 1e-12 * np.max(np.abs(ref), axis=(1, 2)) + 16 * U_DW * np.max(sc, axis=(1, 2))
    allow = np.where(allow > 0, allow, np.finfo(float).tiny)     # a field whose RHS vanishes identically
    return err / allow


@pytest.mark.parametrize("bc", [PERIODIC, REFLECTING])
@pytest.mark.parametrize("nx,ny", [(3, 3), (5, 3), (33, 17), (100, 37), (130, 70)])
def test_df64_rhs_parity_generic(bc, nx, ny):
    for seed in (1, 2):
        p = inputs.smooth_state(nx, ny, bc, seed=seed, xmax=1.3, ymax=0.9)
        s = gu.solver(p, "df64")
        dq = gu.to_np(s.rhs(s.state(p.q0)))
        ref, sc = gu.oracle_rhs_and_scale(p, p.q0)
        e = _rhs_err(dq, ref, sc)
        assert np.all(e <= 1.0), e
        s.close()


def test_df64_rhs_parity_workload_states():
    for p in (inputs.workload1(), inputs.workload2(200, 100)):
        g = pins.grid_of(p)
        q0 = orc.init_aux(g, p.b, p.q0)
        q5 = orc.rk4(g, p.b, q0, p.dt, 5)
        s = gu.solver(p, "df64")
        for q in (q0, q5):
            dq = gu.to_np(s.rhs(s.state(q)))
            ref, sc = gu.oracle_rhs_and_scale(p, q)
            e = _rhs_err(dq, ref, sc)
            assert np.all(e <= 1.0), (p.name, e)
        s.close()


@pytest.mark.parametrize("bc", [PERIODIC, REFLECTING])
def test_df64_steps_parity(bc):
    p = inputs.smooth_state(100, 37, bc, seed=7, xmax=1.3, ymax=0.9)
    g = pins.grid_of(p)
    ref = orc.rk4(g, p.b, p.q0, p.dt, 50)
    s = gu.solver(p, "df64")
    q = s.state(p.q0)
    s.step(q, p.dt, 50)
    e = gu.state_errors(gu.to_np(q), ref)
    assert np.all(e <= gu.STEP_TOL), e
    s.close()


def test_df64_workload1_full_run():
    p = inputs.workload1()
    g = pins.grid_of(p)
    ref = orc.rk4(g, p.b, orc.init_aux(g, p.b, p.q0), p.dt, p.nsteps)
    s = gu.solver(p, "df64")
    q = gu.gpu_init(s, p.q0)
    s.step(q, p.dt, p.nsteps)
    e = gu.state_errors(gu.to_np(q), ref)
    assert np.all(e <= gu.STEP_TOL), e
    s.close()


@pytest.mark.parametrize("bc", [PERIODIC, REFLECTING])
def test_df64_diagnostics_are_those_of_the_double_state(bc):
    p = inputs.smooth_state(70, 45, bc, seed=33, xmax=1.3, ymax=0.9)
    s64, sdw = gu.solver(p, "f64"), gu.solver(p, "df64")
    q = s64.state(p.q0)
    a, b = s64.mass_energy(q), sdw.mass_energy(q)
    assert (a["mass"], a["energy"], a["energy_shifted"]) == (b["mass"], b["energy"], b["energy_shifted"])
    assert abs(a["dEdt"] - b["dEdt"]) <= 1e-10 * abs(a["energy"])
    s64.close()
    sdw.close()


def test_df64_workload2_2000_steps_vs_oracle():
    """The reflecting-wall workload at its stated length (1024x512, 2000 RK4
    steps) in df64 against the oracle's stored FP64 run: the df64 step bar
    on every sampled node and on the whole-state norms."""
    p = inputs.workload2()
    gd = gu.workload2_golden(p)
    s = gu.solver(p, "df64")
    q = s.state(gd["q0"])
    s.step(q, p.dt, p.nsteps)
    e = gu.golden_state_errors(gu.to_np(q), gd)
    s.close()
    gu.report("df64 steps workload2 1024x512 x2000 (sampled)", state_rel=e["samples"])
    assert np.all(e["samples"] <= gu.STEP_TOL_DF64), e
    assert np.all(e["norms"] <= gu.STEP_TOL_DF64), e
