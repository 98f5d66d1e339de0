"""Mutation test: plant one mistake at a time in the oracle (a dropped term, a
flipped sign, a wrong factor 1/2 in any term of any equation; a wrong boundary
row, periodic wrap, SAT weight or sign, or mass-matrix end weight; a wrong row
factor, (1 - eta/h) count, summation or division by h in the rounding-error
scale) and check that at least one of the pins detects it.  The planted mistakes live only in a
test build of the oracle (-DORC_MUTABLE)."""
from __future__ import annotations

import numpy as np
import pytest

import oracle as orc
from oracle import PERIODIC, REFLECTING
from paper_2601_02540_b300 import inputs
import pins

TERMS_PER_FIELD = [6, 15, 15, 9, 5]   # h (incl. the two SAT terms), u, v, w, eta


@pytest.fixture(scope="module")
def mutant(tmp_path_factory):
    return orc.mutable(str(tmp_path_factory.mktemp("mut")))


def _caught(M) -> list[str]:
    fails = []
    for bc in (PERIODIC, REFLECTING):
        st = inputs.smooth_state(11, 9, bc, seed=7)
        a, s = pins.mass_rate(M, st)
        if not a <= 1e-13 * s:
            fails.append(f"mass{bc}")
        a, s = pins.energy_rate(M, st)
        if not a <= 1e-13 * s:
            fails.append(f"energy{bc}")
        a, s = pins.lake_at_rest(M, bc)
        if not a <= 1e-13 * s:
            fails.append(f"lake{bc}")
        a, t = pins.relaxation_oscillator(M, bc)
        if not a <= t:
            fails.append(f"relax{bc}")
        a, t = pins.transpose_symmetry(M, bc)
        if not a <= t:
            fails.append(f"transpose{bc}")
        inner, edge, _ = pins.consistency_orders(M, bc, ns=(32, 64))
        if not np.all(np.isfinite(inner)) or np.min(inner) < 1.7:
            fails.append(f"consistency{bc}")
        if edge is not None and np.min(edge) < 0.8:
            fails.append(f"consistency_edge{bc}")
    return fails


def test_unmutated_build_passes(mutant):
    mutant.mutate()
    assert _caught(mutant) == []


def test_every_term_mistake_is_caught(mutant):
    survivors = []
    for f, nt in enumerate(TERMS_PER_FIELD):
        for k in range(nt):
            for kind in (0, 1, 2):
                mutant.mutate(f, k, kind, 0)
                if not _caught(mutant):
                    survivors.append((f, k, kind))
    mutant.mutate()
    assert survivors == []


@pytest.mark.parametrize("op", [1, 2, 3, 4, 5])
def test_operator_mistake_is_caught(mutant, op):
    mutant.mutate(-1, -1, 0, op)
    try:
        assert _caught(mutant) != []
    finally:
        mutant.mutate()


def _scale_caught(M) -> list[str]:
    fails = []
    for bc in (PERIODIC, REFLECTING):
        dev, tol = pins.rhs_scale_constant(M, bc)
        if not dev <= tol:
            fails.append(f"scale_constant{bc}")
        st = inputs.smooth_state(11, 9, bc, seed=4, xmax=1.3, ymax=0.9)
        g = pins.grid_of(st)
        k = M.rhs(g, st.b, st.q0)
        S = M.rhs_scale(g, st.b, st.q0)
        if not np.all(S >= np.abs(k) * (1 - 1e-14)):
            fails.append(f"scale_bound{bc}")
    return fails


def test_unmutated_scale_passes(mutant):
    mutant.mutate()
    assert _scale_caught(mutant) == []


@pytest.mark.parametrize("op", [6, 7, 8, 9, 10])
def test_rhs_scale_mistake_is_caught(mutant, op):
    """Mistakes that make the rounding-error scale too large (a row factor of
    |D| doubled, (1 - eta/h) counted twice, no division by h) or too small
    (a one-sided row factor halved, |sum| in place of the sum of |terms|)."""
    mutant.mutate(-1, -1, 0, op)
    try:
        assert _scale_caught(mutant) != []
    finally:
        mutant.mutate()
