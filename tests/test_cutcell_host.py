"""The library's cut-cell geometry (stk_cut_cells, host code: no device)
against the oracle's: the same pieces with the same phases, areas to 1e-13 of
a cell, the same merging (bit-exact element map) and the same greedy colours
of the merged elements, on three meshes of the embedded circle of radius 1/4;
the colours separate every pair of elements the coupling stencil joins."""
import numpy as np
import pytest

from paper_1911_05888_gb300 import build, native
from oracle import cutcell


@pytest.fixture(scope="module", autouse=True)
def lib():
    build.build()


@pytest.mark.parametrize("n,centre", [(16, (0.5, 0.5)), (32, (0.5, 0.5)), (40, (0.47, 0.53))])
def test_cut_cells_match_oracle(n, centre):
    g = native.cut_cells(n, centre, 0.25, q=8)
    m = cutcell.CutMesh(cutcell.Circle(centre, 0.25), n, q=8)
    assert len(g["area"]) == len(m.pieces)
    assert np.array_equal(g["cell"], np.array([p["cell"] for p in m.pieces]))
    assert np.array_equal(g["phase"], np.array([p["phase"] for p in m.pieces]))
    np.testing.assert_allclose(g["area"], [p["area"] for p in m.pieces], rtol=0, atol=1e-13 * m.cell_area)
    assert np.array_equal(g["element"], np.array(m.element))
    reps, col = cutcell.greedy_colours(m)
    cmap = dict(zip(reps, col))
    assert np.array_equal(g["colour"], np.array([cmap[e] for e in m.element]))
    perim = sum(w.sum() for (_, w, _) in m.interface.values())
    assert abs(g["interface_length"] - perim) <= 1e-13 and abs(perim - 2 * np.pi * 0.25) <= 1e-12


def test_cut_cell_colours_separate_coupled_elements():
    n = 24
    g = native.cut_cells(n, (0.5, 0.5), 0.25, q=6)
    cells_of = {}
    for (i, j), e in zip(g["cell"], g["element"]):
        cells_of.setdefault(int(e), []).append((int(i), int(j)))
    colour = {int(e): int(c) for e, c in zip(g["element"], g["colour"])}
    stencil = [(a, b) for a in (-1, 0, 1) for b in (-1, 0, 1)] + [(2, 0), (-2, 0), (0, 2), (0, -2)]
    owners = {}
    for e, cs in cells_of.items():
        for c in cs:
            owners.setdefault(c, set()).add(e)
    for e, cs in cells_of.items():
        for (i, j) in cs:
            for di, dj in stencil:
                for f in owners.get((i + di, j + dj), ()):
                    assert f == e or colour[f] != colour[e]


def test_cut_cells_rejects_bad_arguments():
    with pytest.raises(native.StkError):
        native.cut_cells(0, (0.5, 0.5), 0.25)
    with pytest.raises(native.StkError):
        native.cut_cells(8, (0.5, 0.5), -1.0)
