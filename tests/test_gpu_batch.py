"""Ragged ensembles: one launch per RK4 stage over every instance must evolve
each instance exactly as the single-grid path does (same per-node arithmetic),
and match the oracle."""
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

SHAPES = [(33, 17, PERIODIC), (40, 23, REFLECTING), (64, 48, PERIODIC), (5, 3, REFLECTING),
          (100, 37, REFLECTING), (128, 128, PERIODIC), (3, 3, PERIODIC)]


def _ensemble():
    probs = []
    for k, (nx, ny, bc) in enumerate(SHAPES):
        p = inputs.smooth_state(nx, ny, bc, seed=20 + k, xmax=1.0 + 0.1 * k, ymax=0.8 + 0.05 * k,
                                lam=300.0 + 50 * k)
        probs.append(p)
    return probs


@pytest.mark.parametrize("prec", ["f64", "f32", "f32_f64acc"])
def test_batch_equals_single_grid_bitwise(prec):
    probs = _ensemble()
    bs = sgn.BatchSolver(probs, prec=prec)
    q = bs.pack([p.q0 for p in probs])
    bs.step(q, 30)          # one 26-step graph replay + 4 direct steps
    got = bs.unpack(q)
    for p, g in zip(probs, got):
        s = sgn.Solver.from_problem(p, prec=prec)
        qs = s.state(p.q0)
        s.step(qs, p.dt, 30)
        assert torch.equal(qs, g), p.name
        s.close()
    bs.close()


def test_batch_tile_heights_agree_and_autotune():
    probs = _ensemble()
    bs = sgn.BatchSolver(probs, prec="f64")
    ref = None
    for rows in (1, 2, 4):
        bs.set_rows(rows)
        q = bs.pack([p.q0 for p in probs])
        bs.step(q, 27)
        if ref is None:
            ref = q.clone()
        assert torch.equal(q, ref), rows
    q = bs.pack([p.q0 for p in probs])
    assert bs.autotune(q) in (1, 2, 4)
    assert torch.equal(q, bs.pack([p.q0 for p in probs]))   # autotune works on a copy
    bs.close()


def test_batch_diagnostics_do_not_depend_on_the_tile_height():
    """The diagnostics reduce per 32 x 8 band in band order: every tile height
    of the batched kernel and the single-grid FP64 kernel (32 x 24 tiles) give
    the same mass and energies bit for bit."""
    probs = _ensemble()
    bs = sgn.BatchSolver(probs, prec="f64")
    q = bs.pack([p.q0 for p in probs])
    bs.init_aux(q)
    bs.step(q, 5)
    ref = None
    for rows in (1, 2, 4):
        bs.set_rows(rows)
        d = bs.mass_energy(q)
        if ref is None:
            ref = d
        assert np.array_equal(d, ref), rows
    for k, (p, g) in enumerate(zip(probs, bs.unpack(q))):
        s = sgn.Solver.from_problem(p, prec="f64")
        d = s.mass_energy(g.clone())       # an aligned copy of the packed instance
        assert (ref[k, 0], ref[k, 1], ref[k, 2]) == (d["mass"], d["energy"], d["energy_shifted"]), p.name
        s.close()
    bs.close()


def test_batch_matches_oracle_and_diagnostics():
    probs = _ensemble()
    bs = sgn.BatchSolver(probs, prec="f64")
    q = bs.pack([p.q0 for p in probs])
    bs.init_aux(q)
    diag = bs.mass_energy(q)
    for k, (p, g) in enumerate(zip(probs, bs.unpack(q))):
        grid = pins.grid_of(p)
        q0 = orc.init_aux(grid, p.b, p.q0)
        assert np.array_equal(g.cpu().numpy()[4], q0[4])
        d = orc.diagnostics(grid, p.b, q0)
        assert abs(diag[k, 0] - d["mass"]) <= 1e-13 * abs(d["mass"])
        assert abs(diag[k, 1] - d["energy"]) <= 1e-13 * abs(d["energy"])
        assert abs(diag[k, 3]) <= 1e-13 * d["dEdt_scale"]
    bs.step(q, 20)
    for p, g in zip(probs, bs.unpack(q)):
        grid = pins.grid_of(p)
        ref = orc.rk4(grid, p.b, orc.init_aux(grid, p.b, p.q0), p.dt, 20)
        e = gu.state_errors(g.cpu().numpy(), ref)
        assert np.all(e <= gu.STEP_TOL), (p.name, e)
    bs.close()


def test_batch_workload_recipe_small():
    """The ensemble recipe (sizes, half periodic / half reflecting) at 8
    instances: per-instance diagnostics equal the single-grid diagnostics."""
    probs = inputs.workload5(ninst=8, nsteps=10, sizes=(128, 192))
    bs = sgn.BatchSolver(probs, prec="f32")
    q = bs.pack([p.q0 for p in probs])
    bs.init_aux(q)
    bs.step(q, 10)
    diag = bs.mass_energy(q)
    for k, p in enumerate(probs):
        s = sgn.Solver.from_problem(p, prec="f32")
        qs = s.state(p.q0)
        s.init_aux(qs)
        s.step(qs, p.dt, 10)
        assert torch.equal(qs, bs.unpack(q)[k])
        d = s.mass_energy(qs)
        assert diag[k, 0] == d["mass"] and diag[k, 1] == d["energy"]
        s.close()
    bs.close()


# ------------------------------------------------------------------ two stages per launch
@pytest.mark.parametrize("nsteps", [1, 31])
def test_fused_ensemble_equals_one_stage_per_launch_and_single_grids(nsteps):
    """FP32 ensembles advance two RK4 stages per launch by default, one
    launch per boundary class: the states equal one launch per stage and
    each instance's single-grid fused steps bit for bit (ragged grids down
    to 3x3, both boundary kinds; 31 steps: a 26-step graph replay and 5
    direct steps, the odd count ending with a copy back from the scratch
    state)."""
    probs = _ensemble()
    bs = sgn.BatchSolver(probs, prec="f32")
    assert bs.tiling()["fused"]
    q1 = bs.pack([p.q0 for p in probs])
    bs.step(q1, nsteps)
    bs.set_stage_fusion(False)
    assert not bs.tiling()["fused"]
    q2 = bs.pack([p.q0 for p in probs])
    bs.step(q2, nsteps)
    assert torch.equal(q1, q2)
    for p, g in zip(probs, bs.unpack(q1)):
        s = sgn.Solver.from_problem(p, prec="f32")
        qs = s.state(p.q0)
        s.step(qs, p.dt, nsteps)
        assert torch.equal(qs, g), p.name
        s.close()
    bs.close()


def test_fused_ensemble_unsupported_precisions_and_autotune():
    probs = _ensemble()
    for prec in ("f64", "f32_f64acc"):
        bs = sgn.BatchSolver(probs, prec=prec)
        assert not bs.tiling()["fused"]
        with pytest.raises(sgn.SgnError) as ei:
            bs.set_stage_fusion(True)
        assert ei.value.status == 7          # SGN_E_UNSUPPORTED
        bs.close()
    bs = sgn.BatchSolver(probs, prec="f32")
    q = bs.pack([p.q0 for p in probs])
    bs.autotune(q)
    q1 = q.clone()
    bs.step(q1, 7)
    bs.set_stage_fusion(not bs.tiling()["fused"])
    q2 = q.clone()
    bs.step(q2, 7)
    assert torch.equal(q1, q2)
    bs.close()


# ------------------------------------------------------------------ the persistent kernel
@pytest.mark.parametrize("prec", ["f32", "f32_f64acc"])
@pytest.mark.parametrize("rows", [1, 2])
def test_persistent_kernel_equals_per_tile_kernel_bitwise(prec, rows):
    """The persistent kernel (resident blocks walking the tile list, next tile
    prefetched with cp.async) runs the per-tile kernel's arithmetic: equal
    states bit for bit, through a graph replay and direct steps, on ragged
    grids of both boundary kinds."""
    probs = _ensemble()
    bs = sgn.BatchSolver(probs, prec=prec)
    bs.set_rows(rows)
    q1 = bs.pack([p.q0 for p in probs])
    bs.step(q1, 30)
    bs.set_persistent(True)
    t = bs.tiling()
    assert t["rows"] == rows and t["persistent"]
    q2 = bs.pack([p.q0 for p in probs])
    bs.step(q2, 30)
    assert torch.equal(q1, q2)
    bs.close()


def test_persistent_kernel_workload_recipe_equals_single_grid():
    probs = inputs.workload5(ninst=8, nsteps=10, sizes=(128, 192))
    bs = sgn.BatchSolver(probs, prec="f32")
    bs.set_persistent(True)
    q = bs.pack([p.q0 for p in probs])
    bs.init_aux(q)
    bs.step(q, 10)
    for k, p in enumerate(probs):
        s = sgn.Solver.from_problem(p, prec="f32")
        qs = s.state(p.q0)
        s.init_aux(qs)
        s.step(qs, p.dt, 10)
        assert torch.equal(qs, bs.unpack(q)[k]), p.name
        s.close()
    bs.close()


def test_persistent_kernel_unsupported_cases_and_autotune():
    probs = _ensemble()
    bs = sgn.BatchSolver(probs, prec="f64")
    with pytest.raises(sgn.SgnError) as ei:
        bs.set_persistent(True)
    assert ei.value.status == 7
    bs.close()
    bs = sgn.BatchSolver(probs, prec="f32")
    bs.set_rows(4)
    with pytest.raises(sgn.SgnError) as ei:
        bs.set_persistent(True)
    assert ei.value.status == 7
    bs.set_rows(2)
    bs.set_persistent(True)
    with pytest.raises(sgn.SgnError) as ei:
        bs.set_rows(4)
    assert ei.value.status == 7
    q = bs.pack([p.q0 for p in probs])
    rows = bs.autotune(q)
    t = bs.tiling()
    assert t["rows"] == rows and (rows in (1, 2) or not t["persistent"])
    assert torch.equal(q, bs.pack([p.q0 for p in probs]))   # autotune works on a copy
    bs.close()


def test_batch_create_rejects_instances_beyond_the_launch_limit():
    """An instance taller than 65535 rows of 8-node blocks is rejected before
    any of its data is read (a small bathymetry buffer suffices)."""
    import ctypes
    b = torch.zeros(16, dtype=torch.float64, device="cuda")
    for ny, ok in ((65535 * 8 + 1, False), (3, True)):
        inst = sgn.Instance(3, ny, 0.0, 1.0, 0.0, 1.0, 0, 9.81, 500.0, 1e-3)
        arr = (sgn.Instance * 1)(inst)
        h = ctypes.c_void_p()
        bb = torch.zeros(3 * ny, dtype=torch.float64, device="cuda") if ok else b
        st = sgn.lib().sgn_batch_create(arr, 1, 0, ctypes.c_void_p(bb.data_ptr()), ctypes.byref(h))
        if ok:
            assert st == 0
            sgn.lib().sgn_batch_destroy(h)
        else:
            assert st == 1 and h.value is None
            assert "invalid instance" in sgn.lib().sgn_last_error().decode()
