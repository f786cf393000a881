"""Pins of the oracle's patch detection (section 2, after Figure 1: cell-
restricted patches are the column sets of the rows with q (p+1)^d symbolic
nonzeros)."""
import numpy as np
import pytest

import problems as P
from oracle import psr_oracle as O


def as_set(a):
    return set(map(tuple, np.asarray(a)))


@pytest.mark.parametrize("case", ["poisson", "diff3d", "stokes", "stokes_graded"])
def test_recovers_the_generators_cells(case):
    """With the symbolic pattern kept (Dirichlet couplings stored as zeros),
    the detected patches are exactly the cells of the element DOF map the
    generator assembled from -- a construction independent of the matrix."""
    if case == "poisson":
        pr, q = P.poisson2d_q2(8, keep_pattern=True), 9
    elif case == "diff3d":
        pr, q = P.diffusion3d_q2(3, seed=1, keep_pattern=True), 27
    elif case == "stokes":
        pr, q = P.stokes2d_q2q1(8, keep_pattern=True), 22
    else:
        pr, q = P.stokes2d_q2q1(9, 1.05, keep_pattern=True), 22
    d = O.detect_patches(pr.rowptr, pr.colidx, pr.n, q)
    cells = np.sort(pr.dofs2d(), axis=1)
    assert d.shape == cells.shape and as_set(d) == as_set(cells)
    assert all(np.all(np.diff(row) > 0) for row in d)           # DOFs ascending


@pytest.mark.parametrize("N,d", [(8, 2), (6, 2), (4, 3)])
def test_eliminated_boundary_leaves_the_interior_cells(N, d):
    """With Dirichlet rows and columns removed, a boundary cell's rows lose
    entries, so exactly the (N-2)^d interior cells are found."""
    pr = P.poisson2d_q2(N) if d == 2 else P.diffusion3d_q2(N, seed=2)
    q = 9 if d == 2 else 27
    det = O.detect_patches(pr.rowptr, pr.colidx, pr.n, q)
    assert len(det) == (N - 2) ** d
    bnd = pr.meta["dirichlet"]
    interior = [tuple(sorted(c)) for c in pr.dofs2d() if not bnd[c].any()]
    assert as_set(det) == set(interior)


def test_hand_built_duplicates_order_and_empty():
    """Brute force on a 7-row pattern: rows 1, 4 and 6 share one 3-column
    set, row 2 has another 3-column set without its own diagonal, the rest
    have other counts; patches come in the order of their smallest row."""
    rows = [[0, 1], [1, 3, 5], [3, 4, 6], [0, 1, 2, 3], [1, 3, 5], [5], [1, 3, 5]]
    rowptr = np.cumsum([0] + [len(r) for r in rows]).astype(np.int32)
    colidx = np.array([c for r in rows for c in r], dtype=np.int32)
    det = O.detect_patches(rowptr, colidx, len(rows), 3)
    assert det.tolist() == [[1, 3, 5], [3, 4, 6]]
    assert O.detect_patches(rowptr, colidx, len(rows), 4).tolist() == [[0, 1, 2, 3]]
    none = O.detect_patches(rowptr, colidx, len(rows), 7)
    assert none.shape == (0, 7)
