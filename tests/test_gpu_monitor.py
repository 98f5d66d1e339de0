"""Per-step monitoring fused into the fourth RK4 stage (sgn_step_diag) and the
diagnostics of float-stage contexts.

- sgn_step_diag advances exactly as sgn_step and reports, after every step,
  the mass, energy and shifted energy that sgn_mass_energy reports for the new
  state, bit for bit (same per-node arithmetic on the stored state, same
  fixed-order reduction), in all three precisions and both boundary
  treatments.
- The diagnostics of a mixed-precision or df64 context (double q_n) are those
  of its double state: equal to an FP64 context's, bit for bit.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

from oracle import PERIODIC, REFLECTING
from paper_2601_02540_b300 import inputs
import gpu_util as gu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["f64", "f32", "f32_f64acc", "df64"])
@pytest.mark.parametrize("bc", [PERIODIC, REFLECTING])
def test_step_diag_equals_step_then_mass_energy(prec, bc):
    p = inputs.smooth_state(70, 45, bc, seed=31, xmax=1.3, ymax=0.9)
    s = gu.solver(p, prec)
    q1 = s.state(p.q0)
    q2 = s.state(p.q0)
    mon = s.step_diag(q1, p.dt, 6)
    for n in range(6):
        s.step(q2, p.dt, 1)
        d = s.mass_energy(q2)
        assert mon[n] == (d["mass"], d["energy"], d["energy_shifted"]), (n, mon[n], d)
    assert torch.equal(q1, q2)
    s.close()


@pytest.mark.parametrize("prec", ["f32_f64acc", "df64"])
@pytest.mark.parametrize("bc", [PERIODIC, REFLECTING])
def test_double_state_contexts_share_the_diagnostics(bc, prec):
    """Contexts with a double state (mixed: float stages; df64: float-pair
    stages and 32 x 8 tiles instead of the FP64 kernel's 32 x 24) report the
    mass and energies of the FP64 context bit for bit: the same per-node
    arithmetic on the stored state, summed per 32 x 8 band in band order."""
    p = inputs.smooth_state(70, 45, bc, seed=32, xmax=1.3, ymax=0.9)
    s64 = gu.solver(p, "f64")
    sx = gu.solver(p, prec)
    q = s64.state(p.q0)
    a = s64.mass_energy(q)
    b = sx.mass_energy(q)
    assert (a["mass"], a["energy"], a["energy_shifted"]) == (b["mass"], b["energy"], b["energy_shifted"])
    s64.close()
    sx.close()
