"""sgn_step_host: a state in host memory, copied in and back by the library,
advances exactly as sgn_step / sgn_step_diag advance a device copy of it
(the same launches on the same values), from page-locked and from pageable
memory."""
from __future__ import annotations

import ctypes

import pytest
import torch

from paper_2601_02540_b300 import inputs, sgn

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["f64", "f32", "f32_f64acc"])
@pytest.mark.parametrize("pinned", [True, False])
def test_step_host_equals_device_steps(prec, pinned):
    p = inputs.workload2(160, 80)
    s = sgn.Solver.from_problem(p, prec=prec)
    q = s.init_aux(s.state(p.q0))
    qd = q.clone()
    ref = s.step_diag(qd, p.dt, 7)
    h = q.cpu().pin_memory() if pinned else q.cpu()
    got = s.step_host(h, p.dt, 7)
    assert torch.equal(h, qd.cpu())
    assert got == ref
    # without the monitor: the states of sgn_step
    h2 = q.cpu().pin_memory() if pinned else q.cpu()
    qd2 = q.clone()
    assert s.step_host(h2, p.dt, 5, monitor=False) is None
    s.step(qd2, p.dt, 5)
    assert torch.equal(h2, qd2.cpu())
    # zero steps leave the host state as it was
    h3 = h2.clone()
    assert s.step_host(h3, p.dt, 0) == []
    assert torch.equal(h3, h2)
    s.close()


def test_step_host_rejects_device_memory_and_bad_steps():
    p = inputs.workload2(64, 32)
    s = sgn.Solver.from_problem(p, prec="f64")
    q = s.init_aux(s.state(p.q0))
    with pytest.raises(ValueError):
        s.step_host(q, p.dt, 1)
    # the C ABI itself: a device pointer, a negative step count, dt <= 0
    lib = sgn.lib()
    assert lib.sgn_step_host(s.ctx, ctypes.c_void_p(q.data_ptr()), p.dt, 1, None, None) == 1
    h = q.cpu()
    assert lib.sgn_step_host(s.ctx, ctypes.c_void_p(h.data_ptr()), p.dt, -1, None, None) == 1
    assert lib.sgn_step_host(s.ctx, ctypes.c_void_p(h.data_ptr()), 0.0, 1, None, None) == 1
    assert torch.equal(h, q.cpu())
    s.close()
