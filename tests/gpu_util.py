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

import numpy as np
import torch

import oracle as orc
from paper_2601_02540_b300 import inputs, sgn
import pins

RHS_TOL = 1e-12
STEP_TOL = 1e-10
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
