"""Relaxation RK4 on the GPU (sgn_step_relaxed) against the oracle's relaxed
RK4 (energy-conserving fully discrete steps; the paper names relaxation RK as
future work).

gamma is the root near 1 of E(q + gamma d) = E(q).  The oracle brackets it by
bisection on the plain energy differences; the library solves a
cancellation-free form by Newton's method; both are exact up to rounding, whose
effect on gamma is about u |E| / |d^T E'' d| (~1e-12 here).  Bars: gamma per
step within 1e-9, time within n dt 1e-9, state within the step tolerance
1e-10, energy conserved to 1e-13 relative over the run.
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


def _compare(p, q0, dt, n):
    g = pins.grid_of(p)
    qo, go, to = orc.rrk4(g, p.b, q0, dt, n)
    s = gu.solver(p)
    q = s.state(q0)
    e0 = s.mass_energy(q)
    gam, t = s.step_relaxed(q, dt, n)
    e1 = s.mass_energy(q)
    s.close()
    assert np.max(np.abs(np.array(gam) - go)) <= 1e-9, np.max(np.abs(np.array(gam) - go))
    assert abs(t - to) <= 1e-9 * n * dt          # the per-step gamma bar, summed
    e = gu.state_errors(gu.to_np(q), qo)
    assert np.all(e <= gu.STEP_TOL), e
    assert abs(e1["energy"] - e0["energy"]) <= 1e-13 * abs(e0["energy"])
    assert abs(e1["mass"] - e0["mass"]) <= 1e-13 * abs(e0["mass"])
    return np.array(gam)


@pytest.mark.parametrize("bc", [PERIODIC, REFLECTING])
@pytest.mark.parametrize("nx,ny", [(33, 17), (100, 37)])
def test_relaxed_matches_oracle_generic(bc, nx, ny):
    p = inputs.smooth_state(nx, ny, bc, seed=13, xmax=4.0, ymax=3.0, lam=50.0)
    gam = _compare(p, p.q0, p.dt, 20)
    assert np.all(gam != 1.0)


def test_relaxed_matches_oracle_workload2_reduced():
    p = inputs.workload2(200, 100)
    g = pins.grid_of(p)
    q0 = orc.init_aux(g, p.b, p.q0)
    q0 = orc.rk4(g, p.b, q0, p.dt, 20)          # a state with moving water
    _compare(p, q0, p.dt, 20)


def test_relaxed_conserves_energy_where_rk4_drifts():
    p = inputs.workload1()
    s = gu.solver(p)
    q = gu.gpu_init(s, p.q0)
    q4 = q.clone()
    e0 = s.mass_energy(q)["energy"]
    s.step_relaxed(q, 4 * p.dt, 100)
    s.step(q4, 4 * p.dt, 100)
    er = abs(s.mass_energy(q)["energy"] - e0) / abs(e0)
    e4 = abs(s.mass_energy(q4)["energy"] - e0) / abs(e0)
    s.close()
    assert er <= 1e-13 and e4 > 1e3 * max(er, 1e-16), (er, e4)


def test_relaxed_only_f64():
    p = inputs.smooth_state(16, 9, PERIODIC, seed=2)
    s = gu.solver(p, "f32")
    q = torch.as_tensor(p.q0, dtype=torch.float64, device="cuda")
    with pytest.raises(sgn.SgnError) as ei:
        s.step_relaxed(q, 0.01, 1)
    assert ei.value.status == 7      # SGN_E_UNSUPPORTED
    s.close()
