"""Pins of the boundary partition of Alg. 2 (section 3.2: patches are split by
the rows that hold a boundary condition, each partition is clustered on its
own, clusters divided in proportion to the partition sizes)."""
import numpy as np
import pytest

import problems as P
from oracle import psr_oracle as O


def patches(pr):
    return O.extract_patches(pr.rowptr, pr.colidx, pr.vals, pr.n, pr.dofs2d())


@pytest.mark.parametrize("N,d", [(8, 2), (5, 2), (4, 3)])
def test_class_counts_and_sizes(N, d):
    """9 classes on a square, 27 on a cube; sizes: corners 1, edges N-2,
    faces (N-2)^2, interior (N-2)^d (closed forms of the cell counts)."""
    pr = P.poisson2d_q2(N) if d == 2 else P.diffusion3d_q2(N, seed=1)
    cls, k = O.boundary_classes(patches(pr))
    assert k == 3 ** d
    sizes = sorted(np.bincount(cls).tolist())
    if d == 2:
        want = [1] * 4 + [N - 2] * 4 + [(N - 2) ** 2]
    else:
        want = [1] * 8 + [N - 2] * 12 + [(N - 2) ** 2] * 6 + [(N - 2) ** 3]
    assert sizes == sorted(want)
    # the interior class is the one without boundary rows
    A = patches(pr)
    interior = [c for c in range(k) if not (np.count_nonzero(A[np.flatnonzero(cls == c)[0]], axis=1) == 1).any()]
    assert len(interior) == 1 and np.bincount(cls)[interior[0]] == (N - 2) ** d


def test_class_seeds_on_c1_reproduce_alg1():
    """On the uniform 2D Q2 Poisson problem the patches of one class are
    identical, so one seed per class gives Alg. 1's 9-entry database."""
    pr = P.poisson2d_q2(8)
    A = patches(pr)
    cls, k = O.boundary_classes(A)
    init = np.array([np.flatnonzero(cls == c)[0] for c in range(k)])
    r = O.kmeans_l1(A, init, classes=cls)
    a1 = O.alg1(A, 1e-12)
    assert len(a1["reps"]) == 9
    assert np.array_equal(r["phi"], cls) and r["sweeps"] == 2     # assign, then confirm
    for j in range(k):                      # the average of equal members: within a few ulps
        assert np.abs(r["means"][j] - A[init[j]]).max() <= 16 * 2.0 ** -53 * np.abs(A[init[j]]).max()


def test_partitioned_kmeans_is_a_fixed_point_within_classes():
    """Brute force: at the end every patch sits at its nearest mean among its
    own class's means and every mean is its members' average; no patch is
    ever assigned across classes."""
    pr = P.diffusion3d_q2(4, sigma=0.5, corr_len=3.0, seed=4)
    A = patches(pr)
    cls, k = O.boundary_classes(A)
    split = O.proportional_split(cls, 40)
    g = np.random.default_rng(3)
    init = np.concatenate([g.choice(np.flatnonzero(cls == c), split[c], replace=False) for c in range(k)])
    r = O.kmeans_l1(A, init, classes=cls)
    phi, B = r["phi"], r["means"]
    assert np.array_equal(cls[init][phi], cls)
    for i in range(A.shape[0]):
        mine = [j for j in range(len(init)) if cls[init[j]] == cls[i]]
        d = [np.abs(A[i] - B[j]).sum() for j in mine]
        assert mine[int(np.argmin(d))] == phi[i]
    for j in range(len(init)):
        mem = np.flatnonzero(phi == j)
        if mem.size:
            assert np.allclose(B[j], A[mem].mean(axis=0), rtol=1e-14, atol=0)


def test_proportional_split():
    cls = np.repeat(np.arange(3), [90, 9, 1])
    assert O.proportional_split(cls, 10).tolist() == [9, 1, 1]
    assert O.proportional_split(cls, 100).tolist() == [90, 9, 1]
    assert O.proportional_split(cls, 1).tolist() == [1, 1, 1]
