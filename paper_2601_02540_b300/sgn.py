"""Thin ctypes binding of libsgn.so (include/sgn.h).

The functions below carry the C names and only marshal arguments: torch CUDA
tensors become device pointers, the current torch stream becomes the
``cudaStream_t``, and a non-OK status raises :class:`SgnError`.  Every step of
the computation runs in the library's CUDA kernels; there is no CPU path.
``Solver`` is a small convenience wrapper that owns a context.
"""
from __future__ import annotations

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
# SGN_LIBRARY=checked selects the checked build (poisoned tiles, index checks)
LIB_PATH = os.path.join(_HERE, "libsgn_checked.so" if os.environ.get("SGN_LIBRARY") == "checked"
                        else "libsgn.so")

SGN_OK = 0
STATUS = {0: "SGN_OK", 1: "SGN_E_INVAL", 2: "SGN_E_NOMEM", 3: "SGN_E_CUDA",
          4: "SGN_E_NONPOSITIVE_H", 5: "SGN_E_NONFINITE", 6: "SGN_E_TIMEOUT",
          7: "SGN_E_UNSUPPORTED"}
PERIODIC, REFLECTING = 0, 1
F64, F32, F32_F64ACC, DF64 = 0, 1, 2, 3
PREC = {"f64": F64, "f32": F32, "f32_f64acc": F32_F64ACC, "df64": DF64}

# every entry point the header declares: name -> (restype, argtypes)
_V = ctypes.c_void_p
_SIGNATURES = {
    "sgn_create": (ctypes.c_int, [_V, _V, _V]),
    "sgn_destroy": (ctypes.c_int, [_V]),
    "sgn_set_bathymetry": (ctypes.c_int, [_V, _V, _V]),
    "sgn_init_aux": (ctypes.c_int, [_V, _V, _V]),
    "sgn_rhs": (ctypes.c_int, [_V, _V, _V, _V]),
    "sgn_step": (ctypes.c_int, [_V, _V, ctypes.c_double, ctypes.c_int, _V]),
    "sgn_mms_exact": (ctypes.c_int, [_V, ctypes.c_double, _V, _V, _V]),
    "sgn_mms_source": (ctypes.c_int, [_V, ctypes.c_double, _V, _V]),
    "sgn_step_mms": (ctypes.c_int, [_V, _V, ctypes.c_double, ctypes.c_double, ctypes.c_int, _V]),
    "sgn_step_sponge": (ctypes.c_int, [_V, _V, ctypes.c_double, ctypes.c_int, _V, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_double, _V]),
    "sgn_step_relaxed": (ctypes.c_int, [_V, _V, ctypes.c_double, ctypes.c_int, _V, _V, _V]),
    "sgn_step_adaptive": (ctypes.c_int, [_V, _V, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                         _V, _V, _V]),
    "sgn_mass_energy": (ctypes.c_int, [_V, _V, _V, _V]),
    "sgn_step_diag": (ctypes.c_int, [_V, _V, ctypes.c_double, ctypes.c_int, _V, _V]),
    "sgn_step_host": (ctypes.c_int, [_V, _V, ctypes.c_double, ctypes.c_int, _V, _V]),
    "sgn_check": (ctypes.c_int, [_V, _V]),
    "sgn_mass_energy_noalloc": (ctypes.c_int, [_V, _V, _V, _V, _V]),
    "sgn_rhs_vjp": (ctypes.c_int, [_V, _V, _V, _V, _V, _V]),
    "sgn_step_record": (ctypes.c_int, [_V, _V, ctypes.c_double, ctypes.c_int, _V, _V]),
    "sgn_step_vjp": (ctypes.c_int, [_V, _V, _V, _V, ctypes.c_double, _V]),
    "sgn_set_tile_rows": (ctypes.c_int, [_V, ctypes.c_int]),
    "sgn_tile_rows": (ctypes.c_int, [_V, _V]),
    "sgn_set_stage_fusion": (ctypes.c_int, [_V, ctypes.c_int]),
    "sgn_step_record_tape": (ctypes.c_int, [_V, _V, ctypes.c_double, ctypes.c_int, _V, _V, _V]),
    "sgn_step_vjp_tape": (ctypes.c_int, [_V, _V, _V, _V, _V, ctypes.c_double, _V]),
    "sgn_batch_create": (ctypes.c_int, [_V, ctypes.c_int, ctypes.c_int, _V, _V]),
    "sgn_batch_destroy": (ctypes.c_int, [_V]),
    "sgn_batch_cells": (ctypes.c_longlong, [_V]),
    "sgn_batch_init_aux": (ctypes.c_int, [_V, _V, _V]),
    "sgn_batch_step": (ctypes.c_int, [_V, _V, ctypes.c_int, _V]),
    "sgn_batch_mass_energy": (ctypes.c_int, [_V, _V, _V, _V]),
    "sgn_batch_set_rows": (ctypes.c_int, [_V, ctypes.c_int]),
    "sgn_batch_autotune": (ctypes.c_int, [_V, _V, _V, _V]),
    "sgn_batch_set_persistent": (ctypes.c_int, [_V, ctypes.c_int]),
    "sgn_batch_tiling": (ctypes.c_int, [_V, _V, _V]),
    "sgn_batch_set_stage_fusion": (ctypes.c_int, [_V, ctypes.c_int]),
    "sgn_batch_stage_fusion": (ctypes.c_int, [_V, _V]),
    "sgn_status_str": (ctypes.c_char_p, [ctypes.c_int]),
    "sgn_last_error": (ctypes.c_char_p, []),
    "sgn_launch_count": (ctypes.c_ulonglong, []),
    "sgn_measure_fp64_fma": (ctypes.c_int, [ctypes.c_int, _V, _V, _V]),
}


class SgnError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {STATUS.get(status, status)}: {msg}")
        self.status = status


class Params(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("xmin", ctypes.c_double), ("xmax", ctypes.c_double),
                ("ymin", ctypes.c_double), ("ymax", ctypes.c_double),
                ("bc", ctypes.c_int), ("g", ctypes.c_double), ("lam", ctypes.c_double),
                ("prec", ctypes.c_int)]


class Instance(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("xmin", ctypes.c_double), ("xmax", ctypes.c_double),
                ("ymin", ctypes.c_double), ("ymax", ctypes.c_double),
                ("bc", ctypes.c_int), ("g", ctypes.c_double), ("lam", ctypes.c_double),
                ("dt", ctypes.c_double)]


_lib_handle = None


def lib() -> ctypes.CDLL:
    """Load libsgn.so (built in-tree).  Raises if it is missing: no fallback."""
    global _lib_handle
    if _lib_handle is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is not built; run `python -m paper_2601_02540_b300.build`")
        h = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGNATURES.items():
            fn = getattr(h, name)
            fn.restype = res
            fn.argtypes = args
        _lib_handle = h
    return _lib_handle


def _ok(status: int, where: str) -> None:
    if status != SGN_OK:
        raise SgnError(status, where, lib().sgn_last_error().decode())


def _stream(stream) -> ctypes.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dptr(t: torch.Tensor, dtype: torch.dtype, name: str) -> ctypes.c_void_p:
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


# ----------------------------------------------------------------------------- C names
def sgn_create(params: Params, b: torch.Tensor) -> ctypes.c_void_p:
    ctx = ctypes.c_void_p()
    _ok(lib().sgn_create(ctypes.byref(params), _dptr(b, torch.float64, "b"), ctypes.byref(ctx)),
        "sgn_create")
    return ctx


def sgn_destroy(ctx) -> None:
    _ok(lib().sgn_destroy(ctx), "sgn_destroy")


def sgn_set_bathymetry(ctx, b: torch.Tensor, stream=None) -> None:
    _ok(lib().sgn_set_bathymetry(ctx, _dptr(b, torch.float64, "b"), _stream(stream)),
        "sgn_set_bathymetry")


def sgn_init_aux(ctx, q: torch.Tensor, dtype: torch.dtype, stream=None) -> None:
    _ok(lib().sgn_init_aux(ctx, _dptr(q, dtype, "q"), _stream(stream)), "sgn_init_aux")


def sgn_rhs(ctx, q: torch.Tensor, dq: torch.Tensor, dtype: torch.dtype, stream=None) -> None:
    _ok(lib().sgn_rhs(ctx, _dptr(q, dtype, "q"), _dptr(dq, dtype, "dq"), _stream(stream)), "sgn_rhs")


def sgn_step(ctx, q: torch.Tensor, dt: float, nsteps: int, dtype: torch.dtype, stream=None) -> None:
    _ok(lib().sgn_step(ctx, _dptr(q, dtype, "q"), float(dt), int(nsteps), _stream(stream)), "sgn_step")


def sgn_mms_exact(ctx, t: float, q: torch.Tensor, b: torch.Tensor | None = None, stream=None) -> None:
    f = torch.float64
    _ok(lib().sgn_mms_exact(ctx, float(t), _dptr(q, f, "q"), None if b is None else _dptr(b, f, "b"),
                            _stream(stream)), "sgn_mms_exact")


def sgn_mms_source(ctx, t: float, s: torch.Tensor, stream=None) -> None:
    _ok(lib().sgn_mms_source(ctx, float(t), _dptr(s, torch.float64, "s"), _stream(stream)), "sgn_mms_source")


def sgn_step_mms(ctx, q: torch.Tensor, t0: float, dt: float, nsteps: int, stream=None) -> None:
    _ok(lib().sgn_step_mms(ctx, _dptr(q, torch.float64, "q"), float(t0), float(dt), int(nsteps),
                           _stream(stream)), "sgn_step_mms")


def sgn_step_sponge(ctx, q: torch.Tensor, dt: float, nsteps: int, q0: torch.Tensor, width_x: float,
                    width_y: float, sigma_max: float, stream=None) -> None:
    f = torch.float64
    _ok(lib().sgn_step_sponge(ctx, _dptr(q, f, "q"), float(dt), int(nsteps), _dptr(q0, f, "q0"), float(width_x),
                              float(width_y), float(sigma_max), _stream(stream)), "sgn_step_sponge")


def sgn_step_relaxed(ctx, q: torch.Tensor, dt: float, nsteps: int, stream=None):
    """Relaxation RK4 (FP64 contexts); returns (gammas, time advanced)."""
    gam = (ctypes.c_double * max(int(nsteps), 1))()
    t = ctypes.c_double(0.0)
    _ok(lib().sgn_step_relaxed(ctx, _dptr(q, torch.float64, "q"), float(dt), int(nsteps), gam,
                               ctypes.byref(t), _stream(stream)), "sgn_step_relaxed")
    return list(gam[:int(nsteps)]), t.value


PAIRS = {"p5s3": 0, "bs3": 1}


def sgn_step_adaptive(ctx, q: torch.Tensor, t0: float, t_end: float, dt0: float, rtol: float,
                      atol: float, max_attempts: int, want_history: bool = True, stream=None,
                      pair: str = "p5s3"):
    """Adaptive integration (FP64 / df64 contexts) with the pair `pair`
    ("p5s3": the five-stage third-order FSAL pair, "bs3": Bogacki-Shampine);
    returns (stats, history) with stats = {accepted, rejected, t, dt_next,
    attempts} and history an (attempts, 3) list of (dt, err, accepted) or None."""
    st = (ctypes.c_double * 5)()
    hist = (ctypes.c_double * (3 * max(int(max_attempts), 1)))() if want_history else None
    _ok(lib().sgn_step_adaptive(ctx, _dptr(q, torch.float64, "q"), float(t0), float(t_end), float(dt0),
                                float(rtol), float(atol), int(max_attempts), PAIRS[pair], hist, st,
                                _stream(stream)),
        "sgn_step_adaptive")
    n = int(st[4])
    stats = dict(accepted=int(st[0]), rejected=int(st[1]), t=float(st[2]), dt_next=float(st[3]), attempts=n)
    history = [tuple(hist[3 * k:3 * k + 3]) for k in range(n)] if want_history else None
    return stats, history


def sgn_step_diag(ctx, q: torch.Tensor, dt: float, nsteps: int, dtype: torch.dtype, stream=None) -> list:
    """RK4 steps with the mass, energy and shifted energy of every new state
    (fused into the fourth stage): a list of (mass, energy, energy_shifted)."""
    out = (ctypes.c_double * (3 * max(int(nsteps), 1)))()
    _ok(lib().sgn_step_diag(ctx, _dptr(q, dtype, "q"), float(dt), int(nsteps), out, _stream(stream)),
        "sgn_step_diag")
    return [tuple(out[3 * k:3 * k + 3]) for k in range(int(nsteps))]


def sgn_step_host(ctx, q_host: torch.Tensor, dt: float, nsteps: int, dtype: torch.dtype, monitor: bool = True,
                  stream=None):
    """RK4 steps of a state in host memory (copied in, advanced, copied back
    over q_host by the library); with monitor, the list of (mass, energy,
    energy_shifted) after each step, else None."""
    if q_host.is_cuda:
        raise ValueError("q_host must be a CPU tensor")
    if q_host.dtype != dtype:
        raise ValueError(f"q_host must be {dtype}, got {q_host.dtype}")
    if not q_host.is_contiguous():
        raise ValueError("q_host must be contiguous")
    out = (ctypes.c_double * (3 * max(int(nsteps), 1)))() if monitor else None
    _ok(lib().sgn_step_host(ctx, ctypes.c_void_p(q_host.data_ptr()), float(dt), int(nsteps), out,
                            _stream(stream)), "sgn_step_host")
    return [tuple(out[3 * k:3 * k + 3]) for k in range(int(nsteps))] if monitor else None


def sgn_mass_energy(ctx, q: torch.Tensor, dtype: torch.dtype, stream=None) -> list[float]:
    out = (ctypes.c_double * 4)()
    _ok(lib().sgn_mass_energy(ctx, _dptr(q, dtype, "q"), out, _stream(stream)), "sgn_mass_energy")
    return list(out)


def sgn_mass_energy_noalloc(params: Params, b: torch.Tensor, q: torch.Tensor, stream=None) -> list[float]:
    """Diagnostics without a context and without any device allocation (FP64
    only; grids up to 4096x4096); see include/sgn.h."""
    out = (ctypes.c_double * 4)()
    _ok(lib().sgn_mass_energy_noalloc(ctypes.byref(params), _dptr(b, torch.float64, "b"),
                                      _dptr(q, torch.float64, "q"), out, _stream(stream)),
        "sgn_mass_energy_noalloc")
    return list(out)


def sgn_rhs_vjp(ctx, q: torch.Tensor, abar: torch.Tensor, qbar: torch.Tensor, bbar: torch.Tensor,
                stream=None) -> None:
    f = torch.float64
    _ok(lib().sgn_rhs_vjp(ctx, _dptr(q, f, "q"), _dptr(abar, f, "abar"), _dptr(qbar, f, "qbar"),
                          _dptr(bbar, f, "bbar"), _stream(stream)), "sgn_rhs_vjp")


def sgn_step_record(ctx, q: torch.Tensor, dt: float, nsteps: int, stash: torch.Tensor, stream=None) -> None:
    f = torch.float64
    _ok(lib().sgn_step_record(ctx, _dptr(q, f, "q"), float(dt), int(nsteps), _dptr(stash, f, "stash"),
                              _stream(stream)), "sgn_step_record")


def sgn_step_vjp(ctx, stash_slot: torch.Tensor, qbar: torch.Tensor, bbar: torch.Tensor, dt: float,
                 stream=None) -> None:
    f = torch.float64
    _ok(lib().sgn_step_vjp(ctx, _dptr(stash_slot, f, "stash"), _dptr(qbar, f, "qbar"),
                           _dptr(bbar, f, "bbar"), float(dt), _stream(stream)), "sgn_step_vjp")


# planes of one RHS evaluation's tape (SGN_TAPE_PLANES); a step records four
TAPE_PLANES = 21


def sgn_step_record_tape(ctx, q: torch.Tensor, dt: float, nsteps: int, stash: torch.Tensor,
                         tape: torch.Tensor, stream=None) -> None:
    f = torch.float64
    _ok(lib().sgn_step_record_tape(ctx, _dptr(q, f, "q"), float(dt), int(nsteps), _dptr(stash, f, "stash"),
                                   _dptr(tape, f, "tape"), _stream(stream)), "sgn_step_record_tape")


def sgn_step_vjp_tape(ctx, stash_slot: torch.Tensor, tape_slot: torch.Tensor, qbar: torch.Tensor,
                      bbar: torch.Tensor, dt: float, stream=None) -> None:
    f = torch.float64
    _ok(lib().sgn_step_vjp_tape(ctx, _dptr(stash_slot, f, "stash"), _dptr(tape_slot, f, "tape"),
                                _dptr(qbar, f, "qbar"), _dptr(bbar, f, "bbar"), float(dt), _stream(stream)),
        "sgn_step_vjp_tape")


def sgn_check(ctx, stream=None) -> None:
    _ok(lib().sgn_check(ctx, _stream(stream)), "sgn_check")


def sgn_launch_count() -> int:
    return int(lib().sgn_launch_count())


def sgn_measure_fp64_fma(iters: int, stream=None) -> tuple[float, float]:
    """(FMAs executed, seconds) of one launch of the FP64 FMA-chain kernel."""
    n, sec = ctypes.c_double(0.0), ctypes.c_double(0.0)
    _ok(lib().sgn_measure_fp64_fma(int(iters), ctypes.byref(n), ctypes.byref(sec), _stream(stream)),
        "sgn_measure_fp64_fma")
    return n.value, sec.value


# ----------------------------------------------------------------------------- wrapper
class Solver:
    """One grid: owns a library context.  ``state_dtype`` is float64 except in
    pure f32 mode.  States are torch tensors of shape (5, ny, nx)."""

    def __init__(self, nx: int, ny: int, xmin: float, xmax: float, ymin: float, ymax: float,
                 bc: int, b: torch.Tensor, g: float = 9.81, lam: float = 500.0, prec: str = "f64"):
        self.prec = prec
        self.state_dtype = torch.float32 if prec == "f32" else torch.float64
        self.shape = (5, ny, nx)
        self.params = Params(nx, ny, xmin, xmax, ymin, ymax, bc, g, lam, PREC[prec])
        self.ctx = None
        self.ctx = sgn_create(self.params, b.to(torch.float64).contiguous())

    @classmethod
    def from_problem(cls, p, device="cuda", prec: str = "f64") -> "Solver":
        b = torch.as_tensor(p.b, dtype=torch.float64, device=device)
        return cls(p.nx, p.ny, p.xmin, p.xmax, p.ymin, p.ymax, p.bc, b, p.g, p.lam, prec)

    def state(self, q, device="cuda") -> torch.Tensor:
        return torch.as_tensor(q, device=device).to(self.state_dtype).contiguous()

    def set_bathymetry(self, b: torch.Tensor) -> None:
        sgn_set_bathymetry(self.ctx, b.to(torch.float64).contiguous())

    def init_aux(self, q: torch.Tensor) -> torch.Tensor:
        sgn_init_aux(self.ctx, q, self.state_dtype)
        return q

    def rhs(self, q: torch.Tensor, dq: torch.Tensor | None = None) -> torch.Tensor:
        if dq is None:
            dq = torch.empty_like(q)
        sgn_rhs(self.ctx, q, dq, self.state_dtype)
        return dq

    def step(self, q: torch.Tensor, dt: float, nsteps: int) -> torch.Tensor:
        sgn_step(self.ctx, q, dt, nsteps, self.state_dtype)
        return q

    def mms_exact(self, t: float, with_b: bool = False):
        """The manufactured state of Sec. 6.1.2 at time t on this grid (and b)."""
        q = torch.empty(self.shape, dtype=torch.float64, device="cuda")
        b = torch.empty(self.shape[1:], dtype=torch.float64, device="cuda") if with_b else None
        sgn_mms_exact(self.ctx, t, q, b)
        return (q, b) if with_b else q

    def mms_source(self, t: float) -> torch.Tensor:
        s = torch.empty(self.shape, dtype=torch.float64, device="cuda")
        sgn_mms_source(self.ctx, t, s)
        return s

    def step_mms(self, q: torch.Tensor, t0: float, dt: float, nsteps: int) -> torch.Tensor:
        """RK4 with the manufactured source (FP64 contexts), in place."""
        sgn_step_mms(self.ctx, q, t0, dt, nsteps)
        return q

    def step_sponge(self, q: torch.Tensor, dt: float, nsteps: int, q0: torch.Tensor, width_x: float,
                    width_y: float = 0.0, sigma_max: float = 5.0) -> torch.Tensor:
        """RK4 with relaxation zones toward the rest state q0 (FP64 contexts), in place."""
        sgn_step_sponge(self.ctx, q, dt, nsteps, q0, width_x, width_y, sigma_max)
        return q

    def step_relaxed(self, q: torch.Tensor, dt: float, nsteps: int):
        """Energy-conserving relaxation RK4 in place (FP64 contexts): (gammas, time advanced)."""
        return sgn_step_relaxed(self.ctx, q, dt, nsteps)

    def step_adaptive(self, q: torch.Tensor, t0: float, t_end: float, dt0: float, rtol: float = 1e-6,
                      atol: float = 1e-6, max_attempts: int = 100000, want_history: bool = True,
                      pair: str = "p5s3"):
        """Adaptive third-order FSAL integration from t0 to t_end in place
        (FP64 / df64 contexts); see sgn_step_adaptive."""
        return sgn_step_adaptive(self.ctx, q, t0, t_end, dt0, rtol, atol, max_attempts, want_history,
                                 pair=pair)

    def step_diag(self, q: torch.Tensor, dt: float, nsteps: int) -> list:
        """nsteps RK4 steps; (mass, energy, energy_shifted) after each."""
        return sgn_step_diag(self.ctx, q, dt, nsteps, self.state_dtype)

    def step_host(self, q_host: torch.Tensor, dt: float, nsteps: int, monitor: bool = True):
        """nsteps RK4 steps of a state in host memory (CPU tensor, updated in
        place through the library's own copies); see sgn_step_host."""
        return sgn_step_host(self.ctx, q_host, dt, nsteps, self.state_dtype, monitor)

    def mass_energy(self, q: torch.Tensor) -> dict:
        m, e, es, r = sgn_mass_energy(self.ctx, q, self.state_dtype)
        return dict(mass=m, energy=e, energy_shifted=es, dEdt=r)

    def rhs_vjp(self, q: torch.Tensor, abar: torch.Tensor, bbar: torch.Tensor | None = None):
        """(J(q)^T abar, bbar + (dRHS/db)^T abar); FP64 contexts only."""
        qbar = torch.empty_like(q)
        if bbar is None:
            bbar = torch.zeros(q.shape[1:], dtype=torch.float64, device=q.device)
        sgn_rhs_vjp(self.ctx, q, abar, qbar, bbar)
        return qbar, bbar

    def step_record(self, q: torch.Tensor, dt: float, nsteps: int, stash: torch.Tensor,
                    tape: torch.Tensor | None = None) -> torch.Tensor:
        """nsteps RK4 steps recording the stage states (stash: nsteps x 20
        planes) and, with `tape`, the tapes of the stage RHS evaluations
        (nsteps x 4 TAPE_PLANES planes)."""
        if tape is None:
            sgn_step_record(self.ctx, q, dt, nsteps, stash)
        else:
            sgn_step_record_tape(self.ctx, q, dt, nsteps, stash, tape)
        return q

    def step_vjp(self, stash_slot: torch.Tensor, qbar: torch.Tensor, bbar: torch.Tensor, dt: float,
                 tape_slot: torch.Tensor | None = None):
        if tape_slot is None:
            sgn_step_vjp(self.ctx, stash_slot, qbar, bbar, dt)
        else:
            sgn_step_vjp_tape(self.ctx, stash_slot, tape_slot, qbar, bbar, dt)
        return qbar, bbar

    def check(self) -> None:
        sgn_check(self.ctx)

    def set_tile_rows(self, rows: int) -> None:
        """Override the FP64 stage tile height (32 x 8 rows, rows in 1..3)."""
        _ok(lib().sgn_set_tile_rows(self.ctx, int(rows)), "sgn_set_tile_rows")

    def set_stage_fusion(self, on: bool) -> None:
        """FP32: two RK4 stages per launch (default) or one."""
        _ok(lib().sgn_set_stage_fusion(self.ctx, int(bool(on))), "sgn_set_stage_fusion")

    def tile_rows(self) -> int:
        r = ctypes.c_int()
        _ok(lib().sgn_tile_rows(self.ctx, ctypes.byref(r)), "sgn_tile_rows")
        return r.value

    def close(self) -> None:
        if self.ctx is not None and self.ctx.value:
            sgn_destroy(self.ctx)
        self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ----------------------------------------------------------------------------- ensembles
def sgn_batch_create(insts, prec: int, b_packed: torch.Tensor) -> ctypes.c_void_p:
    arr = (Instance * len(insts))(*insts)
    h = ctypes.c_void_p()
    _ok(lib().sgn_batch_create(arr, len(insts), prec, _dptr(b_packed, torch.float64, "b"), ctypes.byref(h)),
        "sgn_batch_create")
    return h


class BatchSolver:
    """A ragged ensemble packed into one state buffer (see include/sgn.h)."""

    def __init__(self, problems, prec: str = "f32", device: str = "cuda"):
        self.prec = prec
        self.state_dtype = torch.float32 if prec == "f32" else torch.float64
        self.problems = problems
        self.sizes = [p.nx * p.ny for p in problems]
        self.offsets = [0]
        for n in self.sizes:
            self.offsets.append(self.offsets[-1] + n)
        insts = [Instance(p.nx, p.ny, p.xmin, p.xmax, p.ymin, p.ymax, p.bc, p.g, p.lam, p.dt) for p in problems]
        b = torch.cat([torch.as_tensor(p.b, dtype=torch.float64).reshape(-1) for p in problems]).to(device)
        self.handle = None
        self.handle = sgn_batch_create(insts, PREC[prec], b.contiguous())
        self.cells = int(lib().sgn_batch_cells(self.handle))
        self.device = device

    def pack(self, states) -> torch.Tensor:
        parts = [torch.as_tensor(q, dtype=self.state_dtype).reshape(-1) for q in states]
        return torch.cat(parts).to(self.device).contiguous()

    def unpack(self, q: torch.Tensor):
        out = []
        for k, p in enumerate(self.problems):
            o = 5 * self.offsets[k]
            out.append(q[o:o + 5 * self.sizes[k]].view(5, p.ny, p.nx))
        return out

    def init_aux(self, q):
        _ok(lib().sgn_batch_init_aux(self.handle, _dptr(q, self.state_dtype, "q"), _stream(None)),
            "sgn_batch_init_aux")
        return q

    def step(self, q, nsteps: int):
        _ok(lib().sgn_batch_step(self.handle, _dptr(q, self.state_dtype, "q"), int(nsteps), _stream(None)),
            "sgn_batch_step")
        return q

    def mass_energy(self, q):
        out = (ctypes.c_double * (4 * len(self.problems)))()
        _ok(lib().sgn_batch_mass_energy(self.handle, _dptr(q, self.state_dtype, "q"), out, _stream(None)),
            "sgn_batch_mass_energy")
        import numpy as np
        return np.array(out[:]).reshape(len(self.problems), 4)

    def set_rows(self, rows: int):
        _ok(lib().sgn_batch_set_rows(self.handle, int(rows)), "sgn_batch_set_rows")

    def set_persistent(self, on: bool):
        _ok(lib().sgn_batch_set_persistent(self.handle, int(bool(on))), "sgn_batch_set_persistent")

    def set_stage_fusion(self, on: bool):
        _ok(lib().sgn_batch_set_stage_fusion(self.handle, int(bool(on))), "sgn_batch_set_stage_fusion")

    def tiling(self) -> dict:
        rows, pers, fuse = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _ok(lib().sgn_batch_tiling(self.handle, ctypes.byref(rows), ctypes.byref(pers)), "sgn_batch_tiling")
        _ok(lib().sgn_batch_stage_fusion(self.handle, ctypes.byref(fuse)), "sgn_batch_stage_fusion")
        return {"rows": rows.value, "persistent": bool(pers.value), "fused": bool(fuse.value)}

    def autotune(self, q) -> int:
        r = ctypes.c_int()
        _ok(lib().sgn_batch_autotune(self.handle, _dptr(q, self.state_dtype, "q"), ctypes.byref(r),
                                     _stream(None)), "sgn_batch_autotune")
        return r.value

    def close(self):
        if self.handle is not None and self.handle.value:
            lib().sgn_batch_destroy(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
