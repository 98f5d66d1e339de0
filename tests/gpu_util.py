"""Helpers shared by the GPU parity tests: run a problem through the CUDA
library (C ABI via the ctypes binding) and through the oracle, and compare.

Tolerances (FP64 path):
  RHS    ||gpu_f - orc_f||_inf <= 1e-12 * ||orc_f||_inf + 16 u ||S_f||_inf
         per field f, u = 2^-53, where S_f is the oracle's forward rounding-error
         scale of that RHS value (each term coef * D f counted as
         |coef| |D| |f|, see oracle.rhs_scale).  The first part is the norm-wise
         relative bound of 1e-12 per RHS; the second is the rounding error any
         FP64 evaluation of the printed formula carries, which dominates only
         where the result is a near-cancellation of much larger terms (a state
         near rest, where the split-form differences of O(1) fields nearly
         cancel; a field whose RHS vanishes identically).
  steps  ||gpu_f - orc_f||_inf <= 1e-10 * max(||orc_f||_inf, 1e-3 * ||orc_h||_inf)
         per field after the run (same reading for fields that stay near 0).
"""
from __future__ import annotations

import json
import os

import numpy as np
import torch

import oracle as orc
from paper_2601_02540_b300 import inputs, sgn
import pins

RHS_TOL = 1e-12
STEP_TOL = 1e-10
# df64 (float-pair) evaluations round with the unit 2^-48, 32 times the FP64
# unit 2^-53; rounding errors accumulated over a run scale with the unit, so
# the after-steps bar of a df64 run is the FP64 bar times 32
STEP_TOL_DF64 = STEP_TOL * 2.0 ** 5
U64 = 2.0 ** -53
ROUNDING_MULT = 16.0


def solver(p: inputs.Problem, prec: str = "f64") -> sgn.Solver:
    return sgn.Solver.from_problem(p, prec=prec)


def gpu_init(s: sgn.Solver, q0: np.ndarray) -> torch.Tensor:
    q = s.state(q0)
    s.init_aux(q)
    return q


def to_np(t: torch.Tensor) -> np.ndarray:
    return t.detach().double().cpu().numpy()


def rhs_errors(gpu: np.ndarray, ref: np.ndarray, scale: np.ndarray) -> np.ndarray:
    """Per-field error divided by its allowance; <= 1 passes."""
    err = np.max(np.abs(gpu - ref), axis=(1, 2))
    allow = RHS_TOL * np.max(np.abs(ref), axis=(1, 2)) + ROUNDING_MULT * U64 * np.max(scale, axis=(1, 2))
    allow = np.where(allow > 0, allow, np.finfo(float).tiny)
    return err / allow


def rhs_rel(gpu: np.ndarray, ref: np.ndarray) -> np.ndarray:
    """Plain norm-wise relative error per field (reported, not asserted)."""
    err = np.max(np.abs(gpu - ref), axis=(1, 2))
    den = np.max(np.abs(ref), axis=(1, 2))
    return np.where(den > 0, err / np.where(den > 0, den, 1.0), err)


def state_errors(gpu: np.ndarray, ref: np.ndarray) -> np.ndarray:
    err = np.max(np.abs(gpu - ref), axis=(1, 2))
    floor = 1e-3 * np.max(np.abs(ref[0]))
    den = np.maximum(np.max(np.abs(ref), axis=(1, 2)), floor)
    return err / den


def oracle_rhs_and_scale(p: inputs.Problem, q: np.ndarray):
    g = pins.grid_of(p)
    return orc.rhs(g, p.b, q), orc.rhs_scale(g, p.b, q)


# ------------------------------------------------------------------ parity report
# Plain errors measured by the parity tests, printed at the end of the pytest
# run (tests/conftest.py) and, if SGN_PARITY_REPORT names a file, written there
# as JSON lines: what each bar allows is asserted, what was reached is reported.
REPORT: list[dict] = []


def report(test: str, **values) -> None:
    row = {"test": test}
    for k, v in values.items():
        row[k] = [float(x) for x in np.ravel(v)] if np.ndim(v) else float(v)
    REPORT.append(row)
    path = os.environ.get("SGN_PARITY_REPORT")
    if path:
        with open(path, "a") as fh:
            fh.write(json.dumps(row) + "\n")


def check_rhs(test: str, gpu: np.ndarray, ref: np.ndarray, scale: np.ndarray) -> np.ndarray:
    """Assert the RHS bar per field and report the plain relative error
    ||gpu_f - orc_f||_inf / ||orc_f||_inf beside err/allow."""
    e = rhs_errors(gpu, ref, scale)
    report(test, rhs_rel=rhs_rel(gpu, ref), err_over_allow=e)
    assert np.all(e <= 1.0), (e, rhs_rel(gpu, ref))
    return e


# ------------------------------------------------------------------ stored oracle runs
def workload2_golden(p: inputs.Problem) -> dict:
    """The oracle's 2000-step run of the reflecting-wall workload
    (tests/golden/workload2_2000.txt) with the initialized state it started
    from, recomputed here by the oracle's initialization and tied to the
    stored run by the per-field checksums."""
    gd = pins.read_golden("workload2_2000.txt")
    nx, ny, nsteps, dt = gd["meta"][0]
    assert (int(nx), int(ny), int(nsteps), dt) == (p.nx, p.ny, p.nsteps, p.dt), gd["meta"]
    q0 = orc.init_aux(pins.grid_of(p), p.b, p.q0)
    chk = q0.sum(axis=(1, 2))
    assert np.allclose(chk, gd["input"][0], rtol=1e-13, atol=1e-9), (chk, gd["input"][0])
    smp = gd["samples"]
    return dict(q0=q0, j=smp[:, 0].astype(np.int64), i=smp[:, 1].astype(np.int64),
                values=smp[:, 2:].T.copy(), maxnorm=gd["norms"][:, 1], l2=gd["norms"][:, 2],
                diag_initial=gd["diagnostics"][0], diag_final=gd["diagnostics"][1],
                k_initial=gd["rhs"][:5, 1], S_initial=gd["rhs"][:5, 2],
                k_final=gd["rhs"][5:, 1], S_final=gd["rhs"][5:, 2])


def golden_state_errors(out: np.ndarray, gd: dict) -> dict:
    """Errors of a final state against the stored oracle run, per field,
    relative to max(||orc_f||_inf, 1e-3 ||orc_h||_inf): over the sampled
    nodes, and of the whole-state max-norm."""
    den = np.maximum(gd["maxnorm"], 1e-3 * gd["maxnorm"][0])
    got = out[:, gd["j"], gd["i"]]
    samples = np.max(np.abs(got - gd["values"]), axis=1) / den
    norms = np.abs(np.max(np.abs(out), axis=(1, 2)) - gd["maxnorm"]) / den
    return dict(samples=samples, norms=norms)
