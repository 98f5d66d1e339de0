"""Mutation test: plant one mistake at a time in the oracle (a dropped term, a
flipped sign, a wrong factor 1/2 in any term of any equation; a wrong boundary
row, periodic wrap, SAT weight or sign, or mass-matrix end weight) and check
that at least one of the pins detects it.  The planted mistakes live only in a
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
