"""sgn_mass_energy_noalloc: the diagnostics for callers that may not allocate
device memory (code inside a framework whose allocator owns the device,
latency-critical loops where cudaMalloc would synchronize the device, plugins
without allocation rights).  Called through the C ABI and checked against the
context-based sgn_mass_energy on two calls in a row, with the tolerances of
the other diagnostics tests.  Kept in its own file, collected last."""
from __future__ import annotations

import ctypes

import numpy as np
import pytest
import torch

import oracle as orc
from oracle import PERIODIC, REFLECTING
from paper_2601_02540_b300 import inputs, sgn
import pins

pytestmark = pytest.mark.gpu


def _noalloc(params: sgn.Params, b: torch.Tensor, q: torch.Tensor) -> tuple[int, list[float]]:
    out = (ctypes.c_double * 4)()
    st = sgn.lib().sgn_mass_energy_noalloc(ctypes.byref(params), ctypes.c_void_p(b.data_ptr()),
                                           ctypes.c_void_p(q.data_ptr()), out,
                                           ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st, list(out)


@pytest.mark.parametrize("bc", [PERIODIC, REFLECTING])
def test_noalloc_matches_context_diagnostics_twice(bc):
    assert torch.cuda.is_available()
    p = inputs.smooth_state(130, 70, bc, seed=5)
    s = sgn.Solver.from_problem(p, prec="f64")
    b = torch.as_tensor(p.b, dtype=torch.float64, device="cuda").contiguous()
    q = s.state(p.q0)
    scale = orc.diagnostics(pins.grid_of(p), p.b, p.q0)["dEdt_scale"]
    for call in range(2):   # two calls in a row, the second on a changed state
        ref = s.mass_energy(q)
        st, got = _noalloc(s.params, b, q)
        assert st == 0, sgn.lib().sgn_last_error().decode()
        for k, name in enumerate(("mass", "energy", "energy_shifted")):
            assert abs(got[k] - ref[name]) <= 1e-13 * abs(ref[name]), (call, name, got[k], ref[name])
        assert abs(got[3] - ref["dEdt"]) <= 1e-13 * scale, (call, got[3], ref["dEdt"])
        s.step(q, p.dt, 3)
    s.close()


def test_noalloc_rejects_grids_beyond_its_scratch():
    b = torch.zeros((8, 8), dtype=torch.float64, device="cuda")
    q = torch.ones((5, 8, 8), dtype=torch.float64, device="cuda")
    big = sgn.Params(8192, 8192, 0.0, 1.0, 0.0, 1.0, PERIODIC, 9.81, 500.0, sgn.F64)
    st, _ = _noalloc(big, b, q)
    assert st == 1
    assert "static scratch" in sgn.lib().sgn_last_error().decode()
    f32 = sgn.Params(8, 8, 0.0, 1.0, 0.0, 1.0, PERIODIC, 9.81, 500.0, sgn.F32)
    st, _ = _noalloc(f32, b, q)
    assert st == 7
