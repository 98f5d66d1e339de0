"""Oracle: plain FP64 CPU restatement of the split-form SBP semi-discretization
of the 2D hyperbolized Serre-Green-Naghdi equations (arXiv 2601.02540).

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA library; the two meet only through the seeded input generator
(``paper_2601_02540_b300.inputs``), which holds none of the method's
arithmetic.

The arithmetic lives in ``sgn_oracle.c`` (compiled without FMA contraction, so
every expression is evaluated as written).  It is compiled twice: with real
doubles (reference values) and with complex doubles, whose complex-step
derivative ``Im f(x + i eps d) / eps`` is the tangent-linear model used to
check the hand-written adjoint.

Functions and the passages they follow:
  dx_apply / dy_apply   1D SBP operators, Remark "Concrete SBP operators and SATs"
  mass_weights          diagonal mass matrix M of the same remark
  rhs                   eq. (sd_periodic_2D_SGN) (periodic), eq. (semi_2D) (reflecting)
  rhs_scale             forward rounding-error scale of each RHS value: every term
                        coef * D f counted as |coef| |D| |f|, the factor (1 - eta/h)
                        as 1 + |eta/h|, pointwise terms by |value| (tolerance scale)
  init_aux              eq. (initialization), Sec. 6
  rk4                   classical RK4 with fixed dt
  diagnostics           mass and energy of Thm. 4.1/4.2 and the rate of eq. (splitcondition)
  energy_total          1^T M E
  gauge_record / gauge_loss   gauge misfit of the inversion problem
  bs3_fixed, rk_adaptive     Bogacki-Shampine 3(2) FSAL pair, fixed / adaptive steps
  p5_tableau, p5_fixed, p5_adaptive   the five-stage third-order FSAL pair of Sec. 6
                        (coefficients constructed here; PI step-size control)
  *_jvp                 complex-step directional derivatives of the above
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sgn_oracle.c")
_LIB_REAL = os.path.join(_HERE, "liboracle.so")
_LIB_CPLX = os.path.join(_HERE, "liboracle_cplx.so")
_LIB_OMP = os.path.join(_HERE, "liboracle_omp.so")

PERIODIC = 0
REFLECTING = 1
FIELDS = ("h", "u", "v", "w", "eta")


def _compile(out: str, defines: list[str]) -> None:
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11", "-fPIC",
           "-shared", *defines, "-o", out + ".tmp", _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(out + ".tmp", out)


def build(force: bool = False) -> None:
    """Compile the oracle libraries with gcc (no FMA contraction): real, complex
    (complex step) and real with OpenMP (the all-core CPU baseline)."""
    for out, extra in ((_LIB_REAL, []), (_LIB_CPLX, ["-DORC_COMPLEX"]), (_LIB_OMP, ["-fopenmp"])):
        if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
            continue
        _compile(out, extra)


class _CGrid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("xmin", ctypes.c_double), ("xmax", ctypes.c_double),
                ("ymin", ctypes.c_double), ("ymax", ctypes.c_double),
                ("bc", ctypes.c_int), ("g", ctypes.c_double), ("lam", ctypes.c_double)]


@dataclass(frozen=True)
class Grid:
    nx: int
    ny: int
    xmin: float
    xmax: float
    ymin: float
    ymax: float
    bc: int
    g: float = 9.81
    lam: float = 500.0

    def c(self) -> _CGrid:
        return _CGrid(self.nx, self.ny, self.xmin, self.xmax, self.ymin, self.ymax,
                      self.bc, self.g, self.lam)

    def spacing(self) -> tuple[float, float]:
        """Node spacing: periodic grids exclude x_max, reflecting grids include it."""
        if self.bc == PERIODIC:
            return (self.xmax - self.xmin) / self.nx, (self.ymax - self.ymin) / self.ny
        return (self.xmax - self.xmin) / (self.nx - 1), (self.ymax - self.ymin) / (self.ny - 1)

    def nodes(self) -> tuple[np.ndarray, np.ndarray]:
        dx, dy = self.spacing()
        x = self.xmin + dx * np.arange(self.nx)
        y = self.ymin + dy * np.arange(self.ny)
        return x, y


_P = ctypes.c_void_p
EPS_CS = 1e-30


def _arr(a, dtype=np.float64) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=dtype)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _check(grid: Grid, b: np.ndarray, q: np.ndarray | None = None):
    assert b.shape == (grid.ny, grid.nx), (b.shape, grid)
    if q is not None:
        assert q.shape == (5, grid.ny, grid.nx), (q.shape, grid)


def _bind(lib: ctypes.CDLL, pre: str, real: bool) -> None:
    sig = [
        ("rhs", ctypes.c_int, [_P, _P, _P, _P]),
        ("init_aux", ctypes.c_int, [_P, _P, _P]),
        ("rk4", ctypes.c_int, [_P, _P, _P, ctypes.c_double, ctypes.c_int]),
        ("dx_apply", None, [_P, _P, _P]),
        ("dy_apply", None, [_P, _P, _P]),
        ("mass_weight", ctypes.c_double, [_P, ctypes.c_int, ctypes.c_int]),
        ("energy_total", None, [_P, _P, _P, _P]),
        ("energy_rate", None, [_P, _P, _P, _P, _P]),
        ("gauge_run", ctypes.c_int, [_P, _P, _P, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_int, _P, _P, _P, _P]),
    ]
    if real:
        sig += [("rhs_scale", ctypes.c_int, [_P, _P, _P, _P]),
                ("diagnostics", ctypes.c_int, [_P, _P, _P, _P]),
                ("bs3_fixed", ctypes.c_int, [_P, _P, _P, ctypes.c_double, ctypes.c_int, _P]),
                ("rrk4", ctypes.c_int, [_P, _P, _P, ctypes.c_double, ctypes.c_int, _P, _P]),
                ("sponge_sigma", ctypes.c_double, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                                   ctypes.c_double, ctypes.c_double]),
                ("rk4_sponge", ctypes.c_int, [_P, _P, _P, ctypes.c_double, ctypes.c_int, _P,
                                              ctypes.c_double, ctypes.c_double, ctypes.c_double]),
                ("rk_adaptive", ctypes.c_int, [_P, _P, _P, ctypes.c_double, ctypes.c_double,
                                               ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                               ctypes.c_int, _P, _P]),
                ("p5_tableau", None, [_P, _P, _P]),
                ("p5_fixed", ctypes.c_int, [_P, _P, _P, ctypes.c_double, ctypes.c_int, _P]),
                ("p5_adaptive", ctypes.c_int, [_P, _P, _P, ctypes.c_double, ctypes.c_double,
                                               ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                               ctypes.c_int, _P, _P])]
    for name, res, args in sig:
        fn = getattr(lib, pre + name)
        fn.restype = res
        fn.argtypes = args


class Oracle:
    """Bound pair of oracle libraries (real and complex builds)."""

    def __init__(self, real_path: str, cplx_path: str | None):
        self._r = ctypes.CDLL(real_path)
        _bind(self._r, "orc_", True)
        self._c = None
        if cplx_path is not None:
            self._c = ctypes.CDLL(cplx_path)
            _bind(self._c, "orcc_", False)

    @staticmethod
    def _ok(rc, name):
        if rc != 0:
            raise MemoryError(f"oracle {name} failed ({rc})")

    # ------------------------------------------------------------------ real
    def dx_apply(self, grid: Grid, f) -> np.ndarray:
        f = _arr(f)
        out = np.empty_like(f)
        g = grid.c()
        self._r.orc_dx_apply(ctypes.byref(g), _ptr(f), _ptr(out))
        return out

    def dy_apply(self, grid: Grid, f) -> np.ndarray:
        f = _arr(f)
        out = np.empty_like(f)
        g = grid.c()
        self._r.orc_dy_apply(ctypes.byref(g), _ptr(f), _ptr(out))
        return out

    def mass_weights(self, grid: Grid) -> np.ndarray:
        g = grid.c()
        return np.array([[self._r.orc_mass_weight(ctypes.byref(g), i, j) for i in range(grid.nx)]
                         for j in range(grid.ny)])

    def rhs(self, grid: Grid, b, q) -> np.ndarray:
        b, q = _arr(b), _arr(q)
        _check(grid, b, q)
        dq = np.empty_like(q)
        g = grid.c()
        self._ok(self._r.orc_rhs(ctypes.byref(g), _ptr(b), _ptr(q), _ptr(dq)), "rhs")
        return dq

    def rhs_scale(self, grid: Grid, b, q) -> np.ndarray:
        b, q = _arr(b), _arr(q)
        _check(grid, b, q)
        sc = np.empty_like(q)
        g = grid.c()
        self._ok(self._r.orc_rhs_scale(ctypes.byref(g), _ptr(b), _ptr(q), _ptr(sc)), "rhs_scale")
        return sc

    def init_aux(self, grid: Grid, b, q) -> np.ndarray:
        b = _arr(b)
        q = _arr(q).copy()
        _check(grid, b, q)
        g = grid.c()
        self._ok(self._r.orc_init_aux(ctypes.byref(g), _ptr(b), _ptr(q)), "init_aux")
        return q

    def bs3_fixed(self, grid: Grid, b, q, dt: float, nsteps: int):
        """The third-order FSAL pair of the adaptive integrator with a fixed
        step (every step accepted): (q after nsteps, error vector e of the
        last step)."""
        b = _arr(b)
        q = _arr(q).copy()
        _check(grid, b, q)
        e = np.zeros_like(q)
        g = grid.c()
        self._ok(self._r.orc_bs3_fixed(ctypes.byref(g), _ptr(b), _ptr(q), dt, nsteps, _ptr(e)),
                 "bs3_fixed")
        return q, e

    def rk_adaptive(self, grid: Grid, b, q, t0: float, t_end: float, dt0: float,
                    rtol: float = 1e-6, atol: float = 1e-6, max_attempts: int = 100000):
        """Adaptive integration from t0 to t_end (Sec. 6): (q, history, stats)
        with history[k] = (dt, err, accepted) of attempt k and stats =
        {accepted, rejected, t, dt_next}."""
        b = _arr(b)
        q = _arr(q).copy()
        _check(grid, b, q)
        hist = np.zeros((max_attempts, 3))
        st = np.zeros(4)
        g = grid.c()
        n = self._r.orc_rk_adaptive(ctypes.byref(g), _ptr(b), _ptr(q), t0, t_end, dt0, rtol, atol,
                                    max_attempts, _ptr(hist), _ptr(st))
        self._ok(0 if n >= 0 else n, "rk_adaptive")
        return q, hist[:n].copy(), dict(accepted=int(st[0]), rejected=int(st[1]), t=float(st[2]),
                                        dt_next=float(st[3]))

    def p5_tableau(self):
        """(A 5x5, b 5, bhat 6) of the five-stage third-order FSAL pair."""
        A, b, bh = np.zeros(25), np.zeros(5), np.zeros(6)
        self._r.orc_p5_tableau(_ptr(A), _ptr(b), _ptr(bh))
        return A.reshape(5, 5), b, bh

    def p5_fixed(self, grid: Grid, b, q, dt: float, nsteps: int):
        """The five-stage third-order FSAL pair with a fixed step (every step
        accepted): (q after nsteps, error vector e of the last step)."""
        b = _arr(b)
        q = _arr(q).copy()
        _check(grid, b, q)
        e = np.zeros_like(q)
        g = grid.c()
        self._ok(self._r.orc_p5_fixed(ctypes.byref(g), _ptr(b), _ptr(q), dt, nsteps, _ptr(e)), "p5_fixed")
        return q, e

    def p5_adaptive(self, grid: Grid, b, q, t0: float, t_end: float, dt0: float,
                    rtol: float = 1e-6, atol: float = 1e-6, max_attempts: int = 100000):
        """Adaptive integration with the five-stage pair and its PI controller
        (Sec. 6): (q, history, stats) as rk_adaptive."""
        b = _arr(b)
        q = _arr(q).copy()
        _check(grid, b, q)
        hist = np.zeros((max_attempts, 3))
        st = np.zeros(4)
        g = grid.c()
        n = self._r.orc_p5_adaptive(ctypes.byref(g), _ptr(b), _ptr(q), t0, t_end, dt0, rtol, atol,
                                    max_attempts, _ptr(hist), _ptr(st))
        self._ok(0 if n >= 0 else n, "p5_adaptive")
        return q, hist[:n].copy(), dict(accepted=int(st[0]), rejected=int(st[1]), t=float(st[2]),
                                        dt_next=float(st[3]))

    def sponge_sigma(self, grid: Grid, wx: float, wy: float, smax: float) -> np.ndarray:
        """Relaxation-zone damping coefficient sigma at every node."""
        g = grid.c()
        return np.array([[self._r.orc_sponge_sigma(ctypes.byref(g), i, j, wx, wy, smax)
                          for i in range(grid.nx)] for j in range(grid.ny)])

    def rk4_sponge(self, grid: Grid, b, q, dt: float, nsteps: int, q0, wx: float, wy: float,
                   smax: float) -> np.ndarray:
        """RK4 of q' = RHS(q) - sigma (q - q0) (relaxation zones)."""
        b, q0 = _arr(b), _arr(q0)
        q = _arr(q).copy()
        _check(grid, b, q)
        _check(grid, b, q0)
        g = grid.c()
        self._ok(self._r.orc_rk4_sponge(ctypes.byref(g), _ptr(b), _ptr(q), dt, nsteps, _ptr(q0), wx, wy, smax),
                 "rk4_sponge")
        return q

    def rrk4(self, grid: Grid, b, q, dt: float, nsteps: int):
        """Relaxation RK4 (energy-conserving): (q, gammas per step, time reached)."""
        b = _arr(b)
        q = _arr(q).copy()
        _check(grid, b, q)
        gam = np.zeros(max(nsteps, 1))
        t = ctypes.c_double(0.0)
        g = grid.c()
        rc = self._r.orc_rrk4(ctypes.byref(g), _ptr(b), _ptr(q), dt, nsteps, _ptr(gam), ctypes.byref(t))
        if rc == -2:
            raise ArithmeticError("relaxation: no sign change of the energy change on [1/2, 3/2]")
        self._ok(rc, "rrk4")
        return q, gam[:nsteps].copy(), t.value

    def rk4(self, grid: Grid, b, q, dt: float, nsteps: int) -> np.ndarray:
        b = _arr(b)
        q = _arr(q).copy()
        _check(grid, b, q)
        g = grid.c()
        self._ok(self._r.orc_rk4(ctypes.byref(g), _ptr(b), _ptr(q), float(dt), int(nsteps)), "rk4")
        return q

    def diagnostics(self, grid: Grid, b, q) -> dict:
        """mass, energy, energy_shifted (E + g b^2/2), dEdt, dEdt_scale."""
        b, q = _arr(b), _arr(q)
        _check(grid, b, q)
        out = np.zeros(5)
        g = grid.c()
        self._ok(self._r.orc_diagnostics(ctypes.byref(g), _ptr(b), _ptr(q), _ptr(out)), "diagnostics")
        return dict(mass=out[0], energy=out[1], energy_shifted=out[2], dEdt=out[3],
                    dEdt_scale=out[4])

    def energy_total(self, grid: Grid, b, q) -> float:
        b, q = _arr(b), _arr(q)
        _check(grid, b, q)
        out = np.zeros(1)
        g = grid.c()
        self._r.orc_energy_total(ctypes.byref(g), _ptr(b), _ptr(q), _ptr(out))
        return float(out[0])

    def energy_rate(self, grid: Grid, b, q, d) -> float:
        """sum M (d_q E . d) with the printed derivatives of E."""
        b, q, d = _arr(b), _arr(q), _arr(d)
        _check(grid, b, q)
        out = np.zeros(1)
        g = grid.c()
        self._r.orc_energy_rate(ctypes.byref(g), _ptr(b), _ptr(q), _ptr(d), _ptr(out))
        return float(out[0])

    def gauge_record(self, grid: Grid, b, q0, dt: float, nsteps: int, every: int, gauges):
        """h at the gauge nodes (flat indices j*nx+i) after every `every` steps."""
        b, q0 = _arr(b), _arr(q0)
        _check(grid, b, q0)
        gi = np.ascontiguousarray(gauges, dtype=np.int64)
        out = np.zeros((nsteps // every, gi.size))
        g = grid.c()
        self._ok(self._r.orc_gauge_run(ctypes.byref(g), _ptr(b), _ptr(q0), float(dt), int(nsteps),
                                       int(every), int(gi.size), _ptr(gi), None, _ptr(out), None),
                 "gauge_run")
        return out

    def gauge_loss(self, grid: Grid, b, q0, dt: float, nsteps: int, every: int, gauges, obs):
        """sum over observation times and gauges of (h - obs)^2."""
        b, q0 = _arr(b), _arr(q0)
        _check(grid, b, q0)
        gi = np.ascontiguousarray(gauges, dtype=np.int64)
        ob = _arr(obs)
        loss = np.zeros(1)
        g = grid.c()
        self._ok(self._r.orc_gauge_run(ctypes.byref(g), _ptr(b), _ptr(q0), float(dt), int(nsteps),
                                       int(every), int(gi.size), _ptr(gi), _ptr(ob), None,
                                       _ptr(loss)), "gauge_run")
        return float(loss[0])

    # ------------------------------------------------- complex step (tangent-linear model)
    @staticmethod
    def _cs(x, d, eps):
        return _arr(x, np.complex128) + 1j * eps * _arr(d, np.complex128)

    def rhs_jvp(self, grid: Grid, b, q, db, dqdir, eps: float = EPS_CS) -> np.ndarray:
        """Directional derivative of rhs at (b, q) along (db, dqdir)."""
        bc, qc = self._cs(b, db, eps), self._cs(q, dqdir, eps)
        _check(grid, bc, qc)
        out = np.empty_like(qc)
        g = grid.c()
        self._ok(self._c.orcc_rhs(ctypes.byref(g), _ptr(bc), _ptr(qc), _ptr(out)), "rhs")
        return out.imag / eps

    def rk4_jvp(self, grid: Grid, b, q, db, dqdir, dt: float, nsteps: int, eps: float = EPS_CS):
        """(state after nsteps, its directional derivative along (db, dqdir))."""
        bc, qc = self._cs(b, db, eps), self._cs(q, dqdir, eps)
        _check(grid, bc, qc)
        g = grid.c()
        self._ok(self._c.orcc_rk4(ctypes.byref(g), _ptr(bc), _ptr(qc), float(dt), int(nsteps)), "rk4")
        return qc.real.copy(), qc.imag / eps

    def energy_jvp(self, grid: Grid, b, q, dqdir, eps: float = EPS_CS) -> float:
        """Directional derivative of 1^T M E along dqdir (b fixed)."""
        bc = _arr(b, np.complex128)
        qc = self._cs(q, dqdir, eps)
        _check(grid, bc, qc)
        out = np.zeros(1, dtype=np.complex128)
        g = grid.c()
        self._c.orcc_energy_total(ctypes.byref(g), _ptr(bc), _ptr(qc), _ptr(out))
        return float(out[0].imag / eps)

    def gauge_loss_jvp(self, grid: Grid, b, q0, db, dq0, dt: float, nsteps: int, every: int,
                       gauges, obs, eps: float = EPS_CS) -> float:
        """Directional derivative of gauge_loss along (db, dq0)."""
        bc, qc = self._cs(b, db, eps), self._cs(q0, dq0, eps)
        _check(grid, bc, qc)
        gi = np.ascontiguousarray(gauges, dtype=np.int64)
        ob = _arr(obs)
        loss = np.zeros(1, dtype=np.complex128)
        g = grid.c()
        self._ok(self._c.orcc_gauge_run(ctypes.byref(g), _ptr(bc), _ptr(qc), float(dt), int(nsteps),
                                        int(every), int(gi.size), _ptr(gi), _ptr(ob), None,
                                        _ptr(loss)), "gauge_run")
        return float(loss[0].imag / eps)


_default: Oracle | None = None


def openmp() -> Oracle:
    """The real oracle built with OpenMP (threads from OMP_NUM_THREADS): the
    same results as default(), on all host cores."""
    build()
    return Oracle(_LIB_OMP, None)


def default() -> Oracle:
    global _default
    if _default is None:
        build()
        _default = Oracle(_LIB_REAL, _LIB_CPLX)
    return _default


class MutableOracle(Oracle):
    """Real-only build with the planted-mistake hooks compiled in
    (-DORC_MUTABLE).  Used only by the mutation test, which plants one known
    mistake at a time and checks that the pins detect it."""

    def mutate(self, f: int = -1, k: int = -1, kind: int = 0, op: int = 0) -> None:
        for name, val in (("orc_mut_f", f), ("orc_mut_k", k), ("orc_mut_kind", kind),
                          ("orc_mut_op", op)):
            ctypes.c_int.in_dll(self._r, name).value = val


def mutable(workdir: str) -> MutableOracle:
    path = os.path.join(workdir, "liboracle_mutable.so")
    _compile(path, ["-DORC_MUTABLE"])
    return MutableOracle(path, None)


def __getattr__(name):
    # module-level convenience: oracle.rhs(...) == oracle.default().rhs(...)
    if name.startswith("_"):
        raise AttributeError(name)
    return getattr(default(), name)
