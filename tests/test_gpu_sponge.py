"""Relaxation zones (sgn_step_sponge) against the oracle's RK4 with the same
source -sigma (q - q0) (Sec. 6, wave-tank experiments), and their effect: a
wave leaving the middle of a closed basin is absorbed."""
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


@pytest.mark.parametrize("bc", [PERIODIC, REFLECTING])
@pytest.mark.parametrize("wx,wy", [(0.8, 0.0), (0.7, 0.5)])
def test_sponge_matches_oracle(bc, wx, wy):
    p = inputs.smooth_state(65, 40, bc, seed=21, xmax=4.0, ymax=3.0, lam=50.0)
    q0 = inputs.smooth_state(65, 40, bc, seed=22, xmax=4.0, ymax=3.0, lam=50.0).q0
    g = pins.grid_of(p)
    ref = orc.rk4_sponge(g, p.b, p.q0, p.dt, 25, q0, wx, wy, 5.0)
    s = gu.solver(p)
    q = s.state(p.q0)
    s.step_sponge(q, p.dt, 25, s.state(q0), wx, wy, 5.0)
    e = gu.state_errors(gu.to_np(q), ref)
    assert np.all(e <= gu.STEP_TOL), e
    s.close()


def test_sponge_absorbs_outgoing_waves():
    """Workload 1's hump in a reflecting basin: with 15-wide zones at all four
    walls the wave energy (E' relative to the rest state) falls far below the
    closed basin's after the wave reaches the walls."""
    p = inputs.workload1()
    p.bc = REFLECTING
    s = gu.solver(p)
    q = gu.gpu_init(s, p.q0)
    rest = torch.zeros_like(q)
    rest[0] = 1.0
    rest[4] = 1.0
    qs = q.clone()
    e_rest = s.mass_energy(rest)["energy_shifted"]
    e0 = s.mass_energy(q)["energy_shifted"] - e_rest
    n = 8 * p.nsteps
    s.step(q, p.dt, n)
    s.step_sponge(qs, p.dt, n, rest, 15.0, 15.0, 5.0)
    e_closed = s.mass_energy(q)["energy_shifted"] - e_rest
    e_sponge = s.mass_energy(qs)["energy_shifted"] - e_rest
    s.close()
    assert e_closed > 0.9 * e0
    assert e_sponge < 0.2 * e0, (e0, e_closed, e_sponge)


def test_sponge_only_f64_and_arguments():
    p = inputs.smooth_state(16, 9, PERIODIC, seed=2)
    s = gu.solver(p)
    q = s.state(p.q0)
    with pytest.raises(sgn.SgnError) as ei:
        s.step_sponge(q, p.dt, 1, q, 1.0)
    assert ei.value.status == 1      # q0 overlapping q
    with pytest.raises(sgn.SgnError) as ei:
        s.step_sponge(q, p.dt, 1, q.clone(), -1.0)
    assert ei.value.status == 1
    s.close()
