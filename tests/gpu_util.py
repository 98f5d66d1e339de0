"""Helpers shared by the GPU parity tests: run a problem through the CUDA
library (C ABI via the ctypes binding) and through the oracle, and compare.

Tolerances (FP64 path):
  RHS    ||gpu_f - orc_f||_inf <= 1e-12 * max(||orc_f||_inf, 1e-2 * ||S_f||_inf)
         per field f, where S_f is the oracle's sum of |terms| of that RHS value.
         This is the norm-wise relative bound of 1e-12 per RHS; the floor only
         matters for fields whose RHS vanishes identically (e.g. w_t of a state
         at rest), where a relative error has no meaning and the rounding level
         of the summed terms is the natural scale.
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


def solver(p: inputs.Problem, prec: str = "f64") -> sgn.Solver:
    return sgn.Solver.from_problem(p, prec=prec)


def gpu_init(s: sgn.Solver, q0: np.ndarray) -> torch.Tensor:
    q = s.state(q0)
    s.init_aux(q)
    return q


def to_np(t: torch.Tensor) -> np.ndarray:
    return t.detach().double().cpu().numpy()


def rhs_errors(gpu: np.ndarray, ref: np.ndarray, scale: np.ndarray) -> np.ndarray:
    """Per-field error normalized by the RHS tolerance denominator."""
    err = np.max(np.abs(gpu - ref), axis=(1, 2))
    den = np.maximum(np.max(np.abs(ref), axis=(1, 2)), 1e-2 * np.max(scale, axis=(1, 2)))
    den = np.where(den > 0, den, 1.0)
    return err / den


def state_errors(gpu: np.ndarray, ref: np.ndarray) -> np.ndarray:
    err = np.max(np.abs(gpu - ref), axis=(1, 2))
    floor = 1e-3 * np.max(np.abs(ref[0]))
    den = np.maximum(np.max(np.abs(ref), axis=(1, 2)), floor)
    return err / den


def oracle_rhs_and_scale(p: inputs.Problem, q: np.ndarray):
    g = pins.grid_of(p)
    return orc.rhs(g, p.b, q), orc.rhs_scale(g, p.b, q)
