"""The solitary-wave convergence study of Sec. 6.1.1 on the GPU: the SGN
solitary wave (eq. (solitary_wave_analytical)) on [-30, 30], repeated in the
other direction (periodic), lambda = 30000, classical RK4 for one traversal of
the domain (t = 60 / C); second-order convergence of h and of the velocity
against the closed-form solution, propagating along x and along y (the two
must give the same errors: the scheme treats both directions alike)."""
from __future__ import annotations

import numpy as np
import pytest

from paper_2601_02540_b300 import inputs
import gpu_util as gu

pytestmark = pytest.mark.gpu


def _run(n, direction):
    p = inputs.soliton(n, direction=direction)
    s = gu.solver(p)
    q = gu.gpu_init(s, p.q0)
    s.step(q, p.dt, p.nsteps)
    qn = gu.to_np(q)
    s.close()
    h, vel = inputs.soliton_fields(p, p.nsteps * p.dt)
    k = 1 if direction == "x" else 2
    return np.array([np.max(np.abs(qn[0] - h)), np.max(np.abs(qn[k] - vel)), np.max(np.abs(qn[3 - k]))])


def test_soliton_second_order_one_traversal():
    ex = np.array([_run(n, "x") for n in (128, 256, 512, 1024)])
    ey = np.array([_run(n, "y") for n in (128, 256, 512, 1024)])
    assert np.allclose(ex, ey, rtol=1e-9, atol=1e-13), (ex, ey)
    assert np.all(ex[:, 2] <= 1e-12)              # the cross velocity stays zero
    orders = np.log2(ex[:-1, :2] / ex[1:, :2])
    assert np.all((orders[-1] > 1.85) & (orders[-1] < 2.2)), (orders, ex)
