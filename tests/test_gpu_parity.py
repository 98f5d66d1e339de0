"""Parity of the CUDA path (through the C ABI) with the oracle.

Sizes span several stage tiles (32x24 FP64, 32x16 float, 32x8 df64) with
ragged tails, tiny odd grids, both boundary treatments, the workloads' own
initial states and generic states with every variable active; the full-size workloads are checked on the whole
grid where the oracle is fast enough (1024x512) and on sampled patches where it
is not (8192^2).  Tolerances are stated in gpu_util.
"""
from __future__ import annotations

import ctypes

import numpy as np
import pytest
import torch

import oracle as orc
from oracle import PERIODIC, REFLECTING
from paper_2601_02540_b300 import inputs, sgn
import gpu_util as gu
import pins

pytestmark = pytest.mark.gpu

GRIDS = [(3, 3), (5, 3), (7, 9), (33, 17), (65, 40), (100, 37), (130, 70)]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    sgn.lib()


# ------------------------------------------------------------------ right-hand side
@pytest.mark.parametrize("bc", [PERIODIC, REFLECTING])
@pytest.mark.parametrize("nx,ny", GRIDS)
def test_rhs_parity_generic_states(bc, nx, ny):
    for seed in (1, 2):
        p = inputs.smooth_state(nx, ny, bc, seed=seed, xmax=1.3, ymax=0.9)
        s = gu.solver(p)
        dq = gu.to_np(s.rhs(s.state(p.q0)))
        ref, sc = gu.oracle_rhs_and_scale(p, p.q0)
        gu.check_rhs(f"rhs {nx}x{ny} bc{bc} seed{seed}", dq, ref, sc)
        s.close()


@pytest.mark.parametrize("make", [lambda: inputs.workload1(),
                                  lambda: inputs.workload2(200, 100),
                                  lambda: inputs.workload2()],
                         ids=["workload1", "workload2_small", "workload2_full"])
def test_rhs_parity_workloads(make):
    """Workload initial states (after initialization) and the state after a few
    oracle steps, so that u, v, w are active; whole grid."""
    p = make()
    g = pins.grid_of(p)
    q0 = orc.init_aux(g, p.b, p.q0)
    q5 = orc.rk4(g, p.b, q0, p.dt, 5)
    s = gu.solver(p)
    for tag, q in (("q0", q0), ("q5", q5)):
        dq = gu.to_np(s.rhs(s.state(q)))
        ref, sc = gu.oracle_rhs_and_scale(p, q)
        gu.check_rhs(f"rhs {p.name} {p.nx}x{p.ny} {tag}", dq, ref, sc)
    s.close()


@pytest.mark.parametrize("bc", [PERIODIC, REFLECTING])
def test_init_aux_parity(bc):
    p = inputs.smooth_state(70, 45, bc, seed=3)
    s = gu.solver(p)
    q = gu.to_np(gu.gpu_init(s, p.q0))
    ref = orc.init_aux(pins.grid_of(p), p.b, p.q0)
    assert np.array_equal(q[4], ref[4])
    assert np.array_equal(q[:3], ref[:3])
    assert np.max(np.abs(q[3] - ref[3])) <= 1e-13 * np.max(np.abs(ref[3]))
    s.close()


# ------------------------------------------------------------------ time stepping
def _step_compare(p: inputs.Problem, nsteps: int):
    g = pins.grid_of(p)
    q0 = orc.init_aux(g, p.b, p.q0)
    ref = orc.rk4(g, p.b, q0, p.dt, nsteps)
    s = gu.solver(p)
    q = s.state(q0)
    s.step(q, p.dt, nsteps)
    out = gu.to_np(q)
    s.close()
    return gu.state_errors(out, ref), out, ref


def test_step_parity_workload1_full():
    """Periodic 64^2, 200 RK4 steps, FP64: within 1e-10 of the oracle."""
    p = inputs.workload1()
    e, out, ref = _step_compare(p, p.nsteps)
    gu.report("steps workload1 64^2 x200", state_rel=e)
    assert np.all(e <= gu.STEP_TOL), e


@pytest.mark.parametrize("bc", [PERIODIC, REFLECTING])
@pytest.mark.parametrize("nx,ny", [(5, 3), (33, 17), (100, 37)])
def test_step_parity_generic(bc, nx, ny):
    p = inputs.smooth_state(nx, ny, bc, seed=4, xmax=1.3, ymax=0.9)
    e, _, _ = _step_compare(p, 20)
    assert np.all(e <= gu.STEP_TOL), e


def test_step_parity_workload2_reduced():
    p = inputs.workload2(160, 80)
    e, _, _ = _step_compare(p, 300)
    assert np.all(e <= gu.STEP_TOL), e


def test_step_parity_workload2_full_size():
    """1024x512 reflecting, the launch configuration of the full workload,
    10 steps on the whole grid."""
    p = inputs.workload2()
    e, _, _ = _step_compare(p, 10)
    gu.report("steps workload2 1024x512 x10", state_rel=e)
    assert np.all(e <= gu.STEP_TOL), e


def test_step_parity_workload2_2000_steps():
    """The reflecting-wall workload at its stated length: 1024x512, 2000 FP64
    RK4 steps, against the oracle's final state stored by
    tests/golden/make_workload2_golden.py (sampled nodes on the walls and
    inside, per-field norms and the diagnostics of the whole state).  Every
    sampled value within 1e-10 max(||orc_f||, 1e-3 ||orc_h||) of the oracle."""
    p = inputs.workload2()
    gd = gu.workload2_golden(p)
    s = gu.solver(p)
    q = s.state(gd["q0"])
    s.step(q, p.dt, p.nsteps)
    out = gu.to_np(q)
    d = s.mass_energy(q)
    s.close()
    e = gu.golden_state_errors(out, gd)
    gu.report("steps workload2 1024x512 x2000 (sampled)", state_rel=e["samples"],
              norm_rel=e["norms"])
    assert np.all(e["samples"] <= gu.STEP_TOL), e
    assert np.all(e["norms"] <= gu.STEP_TOL), e
    for k, name in enumerate(("mass", "energy", "energy_shifted")):
        ref = gd["diag_final"][k]
        assert abs(d[name] - ref) <= 1e-12 * abs(ref), (name, d[name], ref)


def _patch(a: np.ndarray, j0: int, i0: int, m: int) -> np.ndarray:
    ny, nx = a.shape[-2:]
    jj = (np.arange(j0, j0 + m) % ny)[:, None]
    ii = (np.arange(i0, i0 + m) % nx)[None, :]
    return a[..., jj, ii]


def test_workload3_full_size_sampled_patches():
    """8192^2 periodic: RHS and one RK4 step on the whole grid; eight sampled
    patches recomputed by the oracle (with a halo of 1 for the RHS and 4 for a
    step, the domain of dependence), interiors compared."""
    p = inputs.workload3()
    dx, dy = p.spacing()
    q_host = orc.init_aux(pins.grid_of(p), p.b, p.q0)
    s = gu.solver(p)
    q = s.state(q_host)
    dq = gu.to_np(s.rhs(q))
    s.step(q, p.dt, 1)
    q1 = gu.to_np(q)
    s.close()
    # the plain relative error is reported against the whole grid's RHS
    # norm (a patch far from the humps has a near-zero RHS of its own)
    kmax = np.max(np.abs(dq), axis=(1, 2))
    rng = np.random.default_rng(7)
    m = 24
    for _ in range(8):
        j0, i0 = (int(v) for v in rng.integers(0, 8192, size=2))
        for halo, what in ((1, "rhs"), (4, "step")):
            n = m + 2 * halo
            g = orc.Grid(n, n, 0.0, n * dx, 0.0, n * dy, PERIODIC, p.g, p.lam)
            bp = _patch(p.b, j0 - halo, i0 - halo, n)
            qp = _patch(q_host, j0 - halo, i0 - halo, n)
            sl = (slice(None), slice(halo, halo + m), slice(halo, halo + m))
            if what == "rhs":
                ref = orc.rhs(g, bp, qp)[sl]
                sc = orc.rhs_scale(g, bp, qp)[sl]
                got = _patch(dq, j0, i0, m)
                gu.report(f"rhs workload3 8192^2 patch ({j0},{i0}) vs the grid's RHS norm",
                          rel_err_global=np.max(np.abs(got - ref), axis=(1, 2)) / kmax)
                gu.check_rhs(f"rhs workload3 8192^2 patch ({j0},{i0})", got, ref, sc)
            else:
                ref = orc.rk4(g, bp, qp, p.dt, 1)[sl]
                got = _patch(q1, j0, i0, m)
                e = gu.state_errors(got, ref)
                gu.report(f"step workload3 8192^2 patch ({j0},{i0})", state_rel=e)
                assert np.all(e <= gu.STEP_TOL), (what, e)


# ------------------------------------------------------------------ diagnostics
@pytest.mark.parametrize("bc", [PERIODIC, REFLECTING])
def test_mass_energy_parity(bc):
    p = inputs.smooth_state(130, 70, bc, seed=5)
    g = pins.grid_of(p)
    s = gu.solver(p)
    d = s.mass_energy(s.state(p.q0))
    ref = orc.diagnostics(g, p.b, p.q0)
    for k in ("mass", "energy", "energy_shifted"):
        assert abs(d[k] - ref[k]) <= 1e-13 * abs(ref[k]), (k, d[k], ref[k])
    # Thm. 4.1/4.2: the semi-discrete energy rate vanishes up to rounding
    assert abs(d["dEdt"]) <= 1e-13 * ref["dEdt_scale"], (d["dEdt"], ref["dEdt_scale"])
    s.close()


def test_mass_conserved_by_gpu_steps():
    p = inputs.workload2(256, 128)
    s = gu.solver(p)
    q = gu.gpu_init(s, p.q0)
    m0 = s.mass_energy(q)["mass"]
    s.step(q, p.dt, 200)
    m1 = s.mass_energy(q)["mass"]
    assert abs(m1 - m0) <= 1e-13 * abs(m0)
    s.close()


def test_diagnostics_and_steps_are_deterministic():
    p = inputs.smooth_state(100, 37, REFLECTING, seed=6)
    s = gu.solver(p)
    outs = []
    for _ in range(2):
        q = s.state(p.q0)
        s.step(q, p.dt, 7)
        outs.append((gu.to_np(q), s.mass_energy(q)))
    assert np.array_equal(outs[0][0], outs[1][0])
    assert outs[0][1] == outs[1][1]
    s.close()


# ------------------------------------------------------------------ errors (benign)
def test_nonfinite_and_nonpositive_h_are_reported():
    p = inputs.smooth_state(40, 20, PERIODIC, seed=1)
    s = gu.solver(p)
    q = s.state(p.q0)
    q[0, 3, 5] = float("nan")
    with pytest.raises(sgn.SgnError) as ei:
        s.mass_energy(q)
    assert ei.value.status == 5
    q = s.state(p.q0)
    q[0, 7, 9] = -0.5
    s.step(q, p.dt, 1)
    with pytest.raises(sgn.SgnError) as ei:
        s.check()
    assert ei.value.status == 4
    # the flag was cleared: a valid state passes again
    s.mass_energy(s.state(p.q0))
    s.close()


def test_invalid_pointers_rejected():
    p = inputs.smooth_state(16, 16, PERIODIC, seed=1)
    s = gu.solver(p)
    host = np.zeros((5, 16, 16))
    dev = s.state(p.q0)
    lib = sgn.lib()
    assert lib.sgn_rhs(s.ctx, ctypes.c_void_p(host.ctypes.data), ctypes.c_void_p(dev.data_ptr()), None) == 1
    assert lib.sgn_rhs(s.ctx, ctypes.c_void_p(dev.data_ptr()), ctypes.c_void_p(dev.data_ptr()), None) == 1
    assert lib.sgn_step(s.ctx, ctypes.c_void_p(dev.data_ptr()), float("nan"), 1, None) == 1
    assert lib.sgn_step(s.ctx, ctypes.c_void_p(dev.data_ptr() + 8), 0.1, 1, None) == 1
    s.close()


def test_zero_steps_is_identity():
    p = inputs.smooth_state(20, 12, REFLECTING, seed=2)
    s = gu.solver(p)
    q = s.state(p.q0)
    s.step(q, p.dt, 0)
    assert np.array_equal(gu.to_np(q), p.q0)
    s.close()


@pytest.mark.parametrize("prec", ["f64", "f32", "f32_f64acc", "df64"])
def test_graph_replay_equals_direct_steps(prec):
    """Small grids replay 50-step CUDA graphs inside sgn_step: 120 steps in one
    call (two replays + 20 direct steps) equal 120 single-step calls (direct
    launches) bit for bit, and a second call with another dt recaptures."""
    p = inputs.smooth_state(64, 40, REFLECTING, seed=9, xmax=1.3, ymax=0.9)
    s = gu.solver(p, prec)
    q1 = s.state(p.q0)
    s.step(q1, p.dt, 120)
    q2 = s.state(p.q0)
    for _ in range(120):
        s.step(q2, p.dt, 1)
    assert torch.equal(q1, q2)
    q3, q4 = s.state(p.q0), s.state(p.q0)
    s.step(q3, 0.5 * p.dt, 60)
    for _ in range(60):
        s.step(q4, 0.5 * p.dt, 1)
    assert torch.equal(q3, q4)
    s.close()


def test_fp64_fma_rate_measurement():
    n, sec = sgn.sgn_measure_fp64_fma(256)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert n == sms * 8 * 256 * 16 * 256 and sec > 0
    rate = n / sec
    assert 1e10 < rate < 2e12, rate          # FMA per second: B300 ~5e11


@pytest.mark.parametrize("bc", [PERIODIC, REFLECTING])
def test_fp64_tile_heights_agree_bitwise(bc):
    """Every FP64 stage tile height (32x8, 32x16, 32x24) gives the same states,
    RHS and diagnostics bit for bit: the per-node arithmetic and the 32x8 band
    sums do not depend on the tile (direct steps and graph replays, a ragged
    grid of several tiles of each height)."""
    p = inputs.smooth_state(100, 77, bc, seed=31, xmax=1.3, ymax=0.9)
    s = gu.solver(p, "f64")
    ref = None
    for rows in (1, 2, 3):
        s.set_tile_rows(rows)
        assert s.tile_rows() == rows
        q = s.state(p.q0)
        s.step(q, p.dt, 60)
        out = (q, s.rhs(q), s.mass_energy(q))
        if ref is None:
            ref = out
        else:
            assert torch.equal(out[0], ref[0]) and torch.equal(out[1], ref[1]), rows
            assert out[2] == ref[2], rows
    s.check()
    s.close()


@pytest.mark.parametrize("nx,ny", [(64, 64), (512, 512), (1024, 512), (8192, 512)])
def test_fp64_tile_height_choice(nx, ny):
    """sgn_create takes the height with the least FP64 work on the most
    loaded SM (blocks per SM rounded up x the operations of one tile:
    256 R x 68.75 + 34 (8 R + 2) x 15), a lower one only where it saves more
    than 2%; float precisions keep their own tile."""
    p = inputs.smooth_state(nx, ny, REFLECTING, seed=3)
    sms = torch.cuda.get_device_properties(0).multi_processor_count

    def cost(R):
        blocks = -(-nx // 32) * -(-ny // (8 * R))
        return -(-blocks // sms) * (256 * R * 68.75 + 34 * (8 * R + 2) * 15)

    want, best = 3, cost(3)
    for R in (2, 1):
        if cost(R) < 0.98 * best:
            want, best = R, cost(R)
    s = gu.solver(p, "f64")
    assert s.tile_rows() == want
    with pytest.raises(sgn.SgnError):
        s.set_tile_rows(4)
    s.close()
    s = gu.solver(p, "f32")
    with pytest.raises(sgn.SgnError) as ei:
        s.set_tile_rows(1)
    assert ei.value.status == 7          # SGN_E_UNSUPPORTED
    s.close()
