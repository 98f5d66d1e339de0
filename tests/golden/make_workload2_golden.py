"""Write tests/golden/workload2_2000.txt: the oracle's state after the full
reflecting-wall workload (1024x512 on [0,200]x[0,100], eight seeded bathymetry
bumps, one hump of amplitude 0.05, lambda = 500, 2000 classical RK4 steps at
the fixed CFL step; closure of eq. (semi_2D) with the SATs of the SBP remark).

    python tests/golden/make_workload2_golden.py [--threads N]

Calls only the oracle (its OpenMP build: the same arithmetic as the serial
build, rows in parallel, so the same result) and the seeded input generator.
The full state is 21 MB, so the file keeps what a test needs to check a run of
the same workload at any precision against it:
  meta         nx ny nsteps dt
  input        checksums of the initialized state (sum of each field), which
               tie the stored values to this input recipe
  norms        per field: max |f| and sqrt(sum f^2) of the final state
  diagnostics  mass, energy, shifted energy of the initial and final states
  rhs          per field: max |k_f| and max S_f (the rounding-error scale of
               the RHS value, oracle.rhs_scale) at the initial and at the
               final state (first five rows initial, next five final)
  samples      j i h u v w eta at 2048 seeded nodes (512 on the walls, 1536
               inside), final state, all values printed with 17 digits
"""
from __future__ import annotations

import argparse
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

OUT = os.path.join(HERE, "workload2_2000.txt")
SAMPLE_SEED = 2002
N_WALL, N_INNER = 512, 1536


def sample_nodes(nx: int, ny: int) -> np.ndarray:
    """(j, i) of the sampled nodes: the four corners, the rest of the wall
    share spread over the four walls, the remainder inside; no repeats."""
    rng = np.random.Generator(np.random.PCG64(SAMPLE_SEED))
    picked: list[tuple[int, int]] = [(0, 0), (0, nx - 1), (ny - 1, 0), (ny - 1, nx - 1)]
    seen = set(picked)
    while len(picked) < N_WALL:
        wall = int(rng.integers(0, 4))
        if wall < 2:
            node = (0 if wall == 0 else ny - 1, int(rng.integers(0, nx)))
        else:
            node = (int(rng.integers(0, ny)), 0 if wall == 2 else nx - 1)
        if node not in seen:
            seen.add(node)
            picked.append(node)
    while len(picked) < N_WALL + N_INNER:
        node = (int(rng.integers(1, ny - 1)), int(rng.integers(1, nx - 1)))
        if node not in seen:
            seen.add(node)
            picked.append(node)
    return np.array(picked, dtype=np.int64)


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--threads", type=int, default=os.cpu_count())
    args = ap.parse_args()
    os.environ["OMP_NUM_THREADS"] = str(args.threads)

    import oracle as orc
    from paper_2601_02540_b300 import inputs

    p = inputs.workload2()
    g = orc.Grid(p.nx, p.ny, p.xmin, p.xmax, p.ymin, p.ymax, p.bc, p.g, p.lam)
    O = orc.openmp()
    q0 = O.init_aux(g, p.b, p.q0)
    d0 = O.diagnostics(g, p.b, q0)
    t0 = time.time()
    q = O.rk4(g, p.b, q0, p.dt, p.nsteps)
    wall = time.time() - t0
    d1 = O.diagnostics(g, p.b, q)
    nodes = sample_nodes(p.nx, p.ny)

    lines = [
        "# oracle state after the reflecting-wall workload: 1024x512, 2000 RK4 steps, FP64",
        "# written by tests/golden/make_workload2_golden.py (oracle only; "
        f"{args.threads} threads, {wall:.0f} s)",
        "meta",
        f"{p.nx} {p.ny} {p.nsteps} {float(p.dt)!r}",
        "input",
        " ".join(repr(float(np.sum(q0[f]))) for f in range(5)),
        "norms",
    ]
    for f in range(5):
        lines.append(f"{f} {float(np.max(np.abs(q[f])))!r} {float(np.sqrt(np.sum(q[f] ** 2)))!r}")
    lines.append("diagnostics")
    for d in (d0, d1):
        lines.append(f"{float(d['mass'])!r} {float(d['energy'])!r} {float(d['energy_shifted'])!r}")
    lines.append("rhs")
    for st in (q0, q):
        k = O.rhs(g, p.b, st)
        sc = O.rhs_scale(g, p.b, st)
        for f in range(5):
            lines.append(f"{f} {float(np.max(np.abs(k[f])))!r} {float(np.max(sc[f]))!r}")
    lines.append("samples")
    for j, i in nodes:
        lines.append(f"{j} {i} " + " ".join(repr(float(q[f, j, i])) for f in range(5)))
    with open(OUT + ".tmp", "w") as fh:
        fh.write("\n".join(lines) + "\n")
    os.replace(OUT + ".tmp", OUT)
    print(f"wrote {OUT} ({wall:.0f} s of oracle time)")


if __name__ == "__main__":
    main()
