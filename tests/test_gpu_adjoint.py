"""The hand-written adjoint against the oracle's tangent-linear model (complex
step) and against finite differences.

- RHS: the full transposed Jacobian on tiny grids, element by element
  (GPU VJP of unit cotangents vs oracle JVP of unit directions), and dot-product
  tests <J d, a> = <d, J^T a> on multi-tile ragged grids, both boundaries.
- One RK4 step: dot-product test through sgn_step_record + sgn_step_vjp.
- The tape: sgn_step_record_tape advances and records exactly as
  sgn_step_record, its tape holds the RHS intermediates it names (checked
  against sgn_rhs and plain differences of the recorded states), and the VJP
  from the recorded tape equals the VJP that evaluates the tape itself, bit
  for bit (step and rollout).
- The gauge-misfit rollout gradient (checkpointing + recomputation) against the
  oracle's complex-step derivative of the whole rollout, and against central
  finite differences of the GPU loss (eps = 1e-6) on the inversion workload.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle as orc
from oracle import PERIODIC, REFLECTING
from paper_2601_02540_b300 import adjoint, inputs, sgn
import gpu_util as gu
import pins

pytestmark = pytest.mark.gpu


def _t(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("bc", [PERIODIC, REFLECTING])
@pytest.mark.parametrize("nx,ny", [(3, 3), (5, 4)])
def test_rhs_vjp_full_transpose_tiny(bc, nx, ny):
    p = inputs.smooth_state(nx, ny, bc, seed=3, xmax=1.3, ymax=0.9)
    g = pins.grid_of(p)
    n = 5 * nx * ny
    m = nx * ny
    # oracle Jacobian columns (state and bathymetry directions) by complex step
    Jq = np.zeros((n, n))
    Jb = np.zeros((n, m))
    zq = np.zeros_like(p.q0)
    zb = np.zeros_like(p.b)
    for k in range(n):
        d = np.zeros(n)
        d[k] = 1.0
        Jq[:, k] = orc.rhs_jvp(g, p.b, p.q0, zb, d.reshape(p.q0.shape)).ravel()
    for k in range(m):
        d = np.zeros(m)
        d[k] = 1.0
        Jb[:, k] = orc.rhs_jvp(g, p.b, p.q0, d.reshape(p.b.shape), zq).ravel()
    s = sgn.Solver.from_problem(p)
    q = _t(p.q0)
    JqT = np.zeros((n, n))
    JbT = np.zeros((m, n))
    for k in range(n):
        a = np.zeros(n)
        a[k] = 1.0
        qbar, bbar = s.rhs_vjp(q, _t(a.reshape(p.q0.shape)))
        JqT[:, k] = qbar.cpu().numpy().ravel()
        JbT[:, k] = bbar.cpu().numpy().ravel()
    s.check()           # latched flags (index bounds in the checked build)
    s.close()
    scale = np.max(np.abs(Jq))
    assert np.max(np.abs(JqT - Jq.T)) <= 1e-13 * scale, np.max(np.abs(JqT - Jq.T)) / scale
    assert np.max(np.abs(JbT - Jb.T)) <= 1e-13 * np.max(np.abs(Jb)), np.max(np.abs(JbT - Jb.T))


@pytest.mark.parametrize("bc", [PERIODIC, REFLECTING])
@pytest.mark.parametrize("nx,ny", [(33, 17), (100, 37)])
def test_rhs_vjp_dot_product(bc, nx, ny):
    p = inputs.smooth_state(nx, ny, bc, seed=8, xmax=1.3, ymax=0.9)
    g = pins.grid_of(p)
    rng = np.random.default_rng(4)
    s = sgn.Solver.from_problem(p)
    for _ in range(3):
        dq = rng.standard_normal(p.q0.shape)
        db = rng.standard_normal(p.b.shape)
        a = rng.standard_normal(p.q0.shape)
        jd = orc.rhs_jvp(g, p.b, p.q0, db, dq)
        qbar, bbar = s.rhs_vjp(_t(p.q0), _t(a))
        lhs = float(np.sum(jd * a))
        rhs = float(np.sum(dq * qbar.cpu().numpy()) + np.sum(db * bbar.cpu().numpy()))
        mag = float(np.sum(np.abs(jd * a)))
        assert abs(lhs - rhs) <= 1e-13 * mag, (lhs, rhs, mag)
    s.check()           # latched flags (index bounds in the checked build)
    s.close()


@pytest.mark.parametrize("bc", [PERIODIC, REFLECTING])
def test_step_vjp_dot_product(bc):
    p = inputs.smooth_state(40, 23, bc, seed=9, xmax=1.3, ymax=0.9)
    g = pins.grid_of(p)
    rng = np.random.default_rng(5)
    s = sgn.Solver.from_problem(p)
    stash = torch.empty((1, 20, p.ny, p.nx), dtype=torch.float64, device="cuda")
    for _ in range(2):
        dq = rng.standard_normal(p.q0.shape)
        db = rng.standard_normal(p.b.shape)
        a = rng.standard_normal(p.q0.shape)
        _, jd = orc.rk4_jvp(g, p.b, p.q0, db, dq, p.dt, 1)
        q = _t(p.q0)
        s.step_record(q, p.dt, 1, stash)
        qbar = _t(a)
        bbar = torch.zeros((p.ny, p.nx), dtype=torch.float64, device="cuda")
        s.step_vjp(stash[0], qbar, bbar, p.dt)
        lhs = float(np.sum(jd * a))
        rhs = float(np.sum(dq * qbar.cpu().numpy()) + np.sum(db * bbar.cpu().numpy()))
        mag = float(np.sum(np.abs(jd * a)))
        assert abs(lhs - rhs) <= 1e-13 * mag, (lhs, rhs, mag)
    s.check()           # latched flags (index bounds in the checked build)
    s.close()


def test_step_record_matches_step():
    p = inputs.smooth_state(40, 23, REFLECTING, seed=2)
    s = sgn.Solver.from_problem(p)
    q1 = _t(p.q0)
    s.step(q1, p.dt, 3)
    q2 = _t(p.q0)
    stash = torch.empty((3, 20, p.ny, p.nx), dtype=torch.float64, device="cuda")
    s.step_record(q2, p.dt, 3, stash)
    assert torch.equal(q1, q2)
    assert torch.equal(stash[0, :5], _t(p.q0))
    s.check()           # latched flags (index bounds in the checked build)
    s.close()


def _shift(f, axis, k, bc):
    """f at the neighbour k (+1 or -1) along `axis`; reflecting: the node
    itself past a wall (the one-sided end rows of the operator)."""
    if bc == PERIODIC:
        return torch.roll(f, -k, dims=axis)
    n = f.shape[axis]
    idx = torch.arange(n, device=f.device) + k
    idx = idx.clamp(0, n - 1)
    return f.index_select(axis, idx)


@pytest.mark.parametrize("bc", [PERIODIC, REFLECTING])
@pytest.mark.parametrize("nx,ny", [(40, 23), (1000, 515)])     # 32x8 and 32x24 stage tiles
def test_step_record_tape(bc, nx, ny):
    """The taped record advances and records bit for bit as sgn_step_record;
    its tape holds, for each stage state Q_s, k_u, k_v, k_w of sgn_rhs(Q_s)
    and the unscaled differences of h, u, v, w, eta + 3/2 b (bit for bit),
    1/h (to rounding of the reciprocal), and the continuity fluxes."""
    p = inputs.smooth_state(nx, ny, bc, seed=12, xmax=1.3, ymax=0.9)
    s = sgn.Solver.from_problem(p)
    n = 2
    q1, q2 = _t(p.q0), _t(p.q0)
    st1 = torch.empty((n, 20, ny, nx), dtype=torch.float64, device="cuda")
    st2 = torch.empty_like(st1)
    tape = torch.full((n, 4 * sgn.TAPE_PLANES, ny, nx), float("nan"), dtype=torch.float64, device="cuda")
    s.step_record(q1, p.dt, n, st1)
    s.step_record(q2, p.dt, n, st2, tape)
    assert torch.equal(q1, q2) and torch.equal(st1, st2)
    assert bool(torch.isfinite(tape).all())
    b = _t(p.b)
    T = sgn.TAPE_PLANES
    for m in range(n):
        for stage in range(4):
            X = st2[m, 5 * stage:5 * stage + 5].contiguous()
            tp = tape[m, T * stage:T * stage + T]
            k = s.rhs(X)
            for f, slot in ((1, 18), (2, 19), (3, 20)):              # TP_KU, TP_KV, TP_KW
                assert torch.equal(tp[slot], k[f])
            F = X[4] + 1.5 * b
            fields = [X[0], X[1], X[2], X[3], F]
            for f in range(5):                                       # TP_DXH .. TP_DYF
                dx = _shift(fields[f], 1, 1, bc) - _shift(fields[f], 1, -1, bc)
                dy = _shift(fields[f], 0, 1, bc) - _shift(fields[f], 0, -1, bc)
                tol = 0.0 if f < 4 else 1e-15 * float(F.abs().max())  # F is formed with one FMA
                assert float((tp[2 + 2 * f] - dx).abs().max()) <= tol
                assert float((tp[3 + 2 * f] - dy).abs().max()) <= tol
            assert float((tp[0] * X[0] - 1).abs().max()) <= 5e-16          # TP_R
            # A_x = u D_x h + h D_x u, A_y = v D_y h + h D_y v (one FMA each)
            for slot, t1, t2 in ((16, X[1] * tp[2], X[0] * tp[4]), (17, X[2] * tp[3], X[0] * tp[7])):
                err = (tp[slot] - (t1 + t2)).abs()
                assert bool((err <= 5e-16 * (t1.abs() + t2.abs()) + 1e-300).all())
    s.check()
    s.close()


@pytest.mark.parametrize("bc", [PERIODIC, REFLECTING])
@pytest.mark.parametrize("nx,ny", [(40, 23), (1000, 515)])
def test_step_vjp_tape_matches_step_vjp(bc, nx, ny):
    """The VJP of a recorded step from its recorded tapes equals the VJP that
    evaluates each stage's tape itself, bit for bit."""
    p = inputs.smooth_state(nx, ny, bc, seed=13, xmax=1.3, ymax=0.9)
    rng = np.random.default_rng(6)
    s = sgn.Solver.from_problem(p)
    q = _t(p.q0)
    stash = torch.empty((1, 20, ny, nx), dtype=torch.float64, device="cuda")
    tape = torch.empty((1, 4 * sgn.TAPE_PLANES, ny, nx), dtype=torch.float64, device="cuda")
    s.step_record(q, p.dt, 1, stash, tape)
    a = rng.standard_normal(p.q0.shape)
    b0 = rng.standard_normal(p.b.shape)
    qb1, bb1 = _t(a), _t(b0)
    qb2, bb2 = _t(a), _t(b0)
    s.step_vjp(stash[0], qb1, bb1, p.dt)
    s.step_vjp(stash[0], qb2, bb2, p.dt, tape[0])
    assert torch.equal(qb1, qb2) and torch.equal(bb1, bb2)
    s.check()
    s.close()


def _inversion_problem(n, nsteps, every, ngauges=16, seed=1004):
    p = inputs.workload4(n=n, nsteps=nsteps, every=every, ngauges=ngauges, ndirs=5, seed=seed)
    return p


def _gpu_loss_and_grad(p, obs, K, need_grad=True, tape=None):
    s = sgn.Solver.from_problem(p)
    gauges = torch.as_tensor(p.extra["gauges"], device="cuda")
    b = _t(p.b).requires_grad_(need_grad)
    h0 = _t(p.q0[0]).requires_grad_(need_grad)
    out = adjoint.gauge_rollout(b, h0, s, p.dt, p.nsteps, p.extra["every"], gauges, K, tape)
    loss = torch.sum((out - _t(obs)) ** 2)
    if need_grad:
        loss.backward()
        gb, gh = b.grad.cpu().numpy(), h0.grad.cpu().numpy()
    else:
        gb = gh = None
    s.check()           # latched flags (index bounds in the checked build)
    s.close()
    return float(loss.item()), gb, gh


def test_rollout_gradient_matches_oracle_tlm():
    """Small reflecting inversion problem: the checkpointed adjoint gradient
    along random directions equals the oracle's complex-step derivative of the
    whole rollout (checkpoint K = 7 does not divide the 40 steps)."""
    p = _inversion_problem(48, 40, 4, ngauges=6)
    g = pins.grid_of(p)
    gauges = p.extra["gauges"]
    # observations: the truth run (perturbed bathymetry), computed by the oracle
    qt = orc.init_aux(g, p.extra["b_true"], np.stack([p.extra["h_true0"]] + [np.zeros_like(p.b)] * 4))
    obs = orc.gauge_record(g, p.extra["b_true"], qt, p.dt, p.nsteps, p.extra["every"], gauges)
    loss, gb, gh = _gpu_loss_and_grad(p, obs, K=7)
    _, gb_all, gh_all = _gpu_loss_and_grad(p, obs, K=0)   # every stage kept, no recomputation
    assert np.array_equal(gb, gb_all) and np.array_equal(gh, gh_all)
    q0 = orc.init_aux(g, p.b, p.q0)
    loss_o = orc.gauge_loss(g, p.b, q0, p.dt, p.nsteps, p.extra["every"], gauges, obs)
    assert abs(loss - loss_o) <= 1e-10 * abs(loss_o)
    for d in p.extra["dirs"][:3]:
        db, dh = d[0], d[1]
        dq = np.zeros_like(p.q0)
        dq[0] = dh
        dq[4] = dh          # eta0 = h0
        tlm = orc.gauge_loss_jvp(g, p.b, q0, db, dq, p.dt, p.nsteps, p.extra["every"], gauges, obs)
        adj = float(np.sum(gb * db) + np.sum(gh * dh))
        assert abs(adj - tlm) <= 1e-10 * abs(tlm), (adj, tlm)


def test_rollout_gradient_matches_oracle_tlm_checkpointed():
    """The inversion recipe at 96^2, 200 steps, gauges every 10 steps,
    checkpoints every 100 steps (two segments, the first recomputed): the
    adjoint gradient along three of the workload's unit directions equals the
    oracle's complex-step derivative of the whole rollout within 1e-10."""
    p = _inversion_problem(96, 200, 10, ngauges=16)
    g = pins.grid_of(p)
    gauges = p.extra["gauges"]
    qt = orc.init_aux(g, p.extra["b_true"], np.stack([p.extra["h_true0"]] + [np.zeros_like(p.b)] * 4))
    obs = orc.gauge_record(g, p.extra["b_true"], qt, p.dt, p.nsteps, p.extra["every"], gauges)
    loss, gb, gh = _gpu_loss_and_grad(p, obs, K=100, tape=True)
    _, gb2, gh2 = _gpu_loss_and_grad(p, obs, K=100, tape=False)     # tapes evaluated by the VJP
    assert np.array_equal(gb, gb2) and np.array_equal(gh, gh2)
    q0 = orc.init_aux(g, p.b, p.q0)
    for d in p.extra["dirs"][:3]:
        dq = np.zeros_like(p.q0)
        dq[0] = d[1]
        dq[4] = d[1]          # eta0 = h0
        tlm = orc.gauge_loss_jvp(g, p.b, q0, d[0], dq, p.dt, p.nsteps, p.extra["every"], gauges, obs)
        adj = float(np.sum(gb * d[0]) + np.sum(gh * d[1]))
        assert abs(adj - tlm) <= 1e-10 * abs(tlm), (adj, tlm)


def _gpu_gauge_record(p, b, h0, K=100):
    """Gauge readings of a GPU rollout from (b, h0) (no gradient)."""
    s = sgn.Solver.from_problem(p)
    gauges = torch.as_tensor(p.extra["gauges"], device="cuda")
    with torch.no_grad():
        out = adjoint.gauge_rollout(_t(b), _t(h0), s, p.dt, p.nsteps, p.extra["every"], gauges, K)
    rec = out.cpu().numpy()
    s.check()
    s.close()
    return rec


def test_rollout_gradient_matches_finite_differences_full_size():
    """The inversion workload as stated: reflecting 512^2, 2000 RK4 steps, 16
    gauges read every 10 steps against the run with the perturbed (truth)
    bathymetry, checkpoints every 100 steps; the adjoint gradient along each
    of the 20 unit directions over (b, h0) against central differences of the
    GPU loss with eps = 1e-6, within 1e-5 relative."""
    p = inputs.workload4()
    assert (p.nx, p.nsteps, p.extra["every"], len(p.extra["dirs"])) == (512, 2000, 10, 20)
    obs = _gpu_gauge_record(p, p.extra["b_true"], p.extra["h_true0"])
    loss, gb, gh = _gpu_loss_and_grad(p, obs, K=100)
    eps = 1e-6
    b0, h00 = p.b.copy(), p.q0[0].copy()
    rel = []
    try:
        for d in p.extra["dirs"]:
            p.b = b0 + eps * d[0]
            p.q0[0] = h00 + eps * d[1]
            lp, _, _ = _gpu_loss_and_grad(p, obs, K=100, need_grad=False)
            p.b = b0 - eps * d[0]
            p.q0[0] = h00 - eps * d[1]
            lm, _, _ = _gpu_loss_and_grad(p, obs, K=100, need_grad=False)
            fd = (lp - lm) / (2 * eps)
            adj = float(np.sum(gb * d[0]) + np.sum(gh * d[1]))
            rel.append(abs(adj - fd) / abs(adj))
    finally:
        p.b, p.q0[0] = b0, h00
    gu.report("adjoint workload4 512^2 x2000 K=100 vs central FD (20 directions)", rel_err=rel)
    assert max(rel) <= 1e-5, rel


def test_rollout_gradient_matches_finite_differences():
    """Inversion workload recipe at 128^2, 300 steps, gauges every 10 steps:
    gradient vs central differences of the GPU loss, eps = 1e-6, 5 unit
    directions over (b, h0)."""
    p = _inversion_problem(128, 300, 10)
    g = pins.grid_of(p)
    qt = orc.init_aux(g, p.extra["b_true"], np.stack([p.extra["h_true0"]] + [np.zeros_like(p.b)] * 4))
    obs = orc.gauge_record(g, p.extra["b_true"], qt, p.dt, p.nsteps, p.extra["every"], p.extra["gauges"])
    loss, gb, gh = _gpu_loss_and_grad(p, obs, K=100)
    eps = 1e-6
    b0, h00 = p.b.copy(), p.q0[0].copy()
    for d in p.extra["dirs"]:
        p.b = b0 + eps * d[0]
        p.q0[0] = h00 + eps * d[1]
        lp, _, _ = _gpu_loss_and_grad(p, obs, K=100, need_grad=False)
        p.b = b0 - eps * d[0]
        p.q0[0] = h00 - eps * d[1]
        lm, _, _ = _gpu_loss_and_grad(p, obs, K=100, need_grad=False)
        fd = (lp - lm) / (2 * eps)
        adj = float(np.sum(gb * d[0]) + np.sum(gh * d[1]))
        assert abs(adj - fd) <= 1e-5 * abs(adj), (adj, fd)
    p.b, p.q0[0] = b0, h00


def test_step_vjp_rejects_dt_outside_scaled_range():
    """The stage cotangents carry the factor dt^4/24; a dt that underflows it is
    refused before any launch, and qbar is left untouched."""
    p = inputs.smooth_state(16, 9, PERIODIC, seed=2)
    s = sgn.Solver.from_problem(p)
    stash = torch.empty((1, 20, p.ny, p.nx), dtype=torch.float64, device="cuda")
    s.step_record(_t(p.q0), p.dt, 1, stash)
    qbar = _t(np.ones_like(p.q0))
    bbar = torch.zeros((p.ny, p.nx), dtype=torch.float64, device="cuda")
    with pytest.raises(sgn.SgnError) as ei:
        s.step_vjp(stash[0], qbar, bbar, 1e-90)
    assert ei.value.status == 1          # SGN_E_INVAL
    assert torch.equal(qbar, _t(np.ones_like(p.q0)))
    s.check()           # latched flags (index bounds in the checked build)
    s.close()
