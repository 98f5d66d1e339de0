"""sgn_mass_energy_noalloc: the diagnostics for callers that may not allocate
device memory (code inside a framework whose allocator owns the device,
latency-critical loops where cudaMalloc would synchronize the device, plugins
without allocation rights).  Called through the C ABI and checked against the
context-based sgn_mass_energy on two calls in a row: the two run the same
kernels over the same bands in the same order, so the four results agree bit
for bit.  Kept in its own file, collected last."""
from __future__ import annotations

import ctypes

import numpy as np
import pytest
import torch

from oracle import PERIODIC, REFLECTING
from paper_2601_02540_b300 import inputs, sgn

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
    for call in range(2):   # two calls in a row, the second on a changed state
        ref = s.mass_energy(q)
        st, got = _noalloc(s.params, b, q)
        assert st == 0, sgn.lib().sgn_last_error().decode()
        for k, name in enumerate(("mass", "energy", "energy_shifted", "dEdt")):
            assert got[k] == ref[name], (call, name, got[k], ref[name])
        s.step(q, p.dt, 3)
    s.close()


def test_noalloc_largest_grid_matches_and_one_row_more_is_rejected():
    """The static scratch holds the band partials of 32768 blocks of 32x16
    nodes: 4096x4096 is the largest square grid it serves (accepted, equal to
    the context's diagnostics); 4096x4097 needs one more block row and is
    rejected before any launch."""
    n = 4096
    p = inputs.smooth_state(n, n, PERIODIC, seed=6)
    s = sgn.Solver.from_problem(p, prec="f64")
    b = torch.as_tensor(p.b, dtype=torch.float64, device="cuda").contiguous()
    q = s.state(p.q0)
    ref = s.mass_energy(q)
    st, got = _noalloc(s.params, b, q)
    assert st == 0, sgn.lib().sgn_last_error().decode()
    for k, name in enumerate(("mass", "energy", "energy_shifted", "dEdt")):
        assert got[k] == ref[name], (name, got[k], ref[name])
    s.close()
    over = sgn.Params(n, n + 1, 0.0, 1.0, 0.0, 1.0, PERIODIC, 9.81, 500.0, sgn.F64)
    st, _ = _noalloc(over, b, q)
    assert st == 1
    assert "static scratch" in sgn.lib().sgn_last_error().decode()


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
