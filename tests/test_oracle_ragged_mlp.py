"""Pins of the oracle's ragged-size extraction and apply (the remark after
Eq. 1: patches of different sizes) and of the MLP forward pass, against
definitions written out independently of the oracle's own code paths."""
import numpy as np
import pytest

import problems
from oracle import psr_oracle as O


def _dense(pr):
    """Dense A from the CSR arrays by a plain double loop (no lookup code)."""
    A = np.zeros((pr.n, pr.n))
    for i in range(pr.n):
        for t in range(pr.rowptr[i], pr.rowptr[i + 1]):
            A[i, pr.colidx[t]] = pr.vals[t]
    return A


def _restriction(d, n):
    """The boolean V_k of section 2: (V_k)_{ij} = 1 iff global DOF j is local DOF i."""
    V = np.zeros((len(d), n))
    V[np.arange(len(d)), d] = 1.0
    return V


@pytest.fixture(scope="module")
def stokes3d_small():
    return problems.stokes3d_q2q1(3, seed=7)


def test_extract_ragged_is_the_principal_submatrix(stokes3d_small):
    pr = stokes3d_small
    A = _dense(pr)
    Ak = O.extract_patches_ragged(pr.rowptr, pr.colidx, pr.vals, pr.n, pr.patch_offsets, pr.patch_dofs)
    assert len(Ak) == pr.n_patches
    sizes = set()
    for k in range(pr.n_patches):
        d = pr.patch_dofs[pr.patch_offsets[k]:pr.patch_offsets[k + 1]]
        V = _restriction(d, pr.n)
        assert Ak[k].shape == (len(d), len(d))
        assert np.array_equal(Ak[k], V @ A @ V.T)
        sizes.add(len(d))
    assert len(sizes) > 1              # the case really has patches of several sizes


def test_extract_ragged_random_pattern():
    """Random sparse matrix, random ragged patches with repeated DOFs across
    patches and entries absent from the pattern (which must read as 0)."""
    g = np.random.default_rng(3)
    n = 40
    M = g.standard_normal((n, n)) * (g.random((n, n)) < 0.2)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    cols, vals = [], []
    for i in range(n):
        nz = np.flatnonzero(M[i])
        cols.extend(nz.tolist())
        vals.extend(M[i, nz].tolist())
        rowptr[i + 1] = len(cols)
    sizes = g.integers(1, 9, size=12)
    flat = np.concatenate([g.choice(n, size=s, replace=False) for s in sizes])
    offsets = np.concatenate([[0], np.cumsum(sizes)])
    Ak = O.extract_patches_ragged(rowptr, np.array(cols), np.array(vals), n, offsets, flat)
    for k, s in enumerate(sizes):
        d = flat[offsets[k]:offsets[k + 1]]
        assert np.array_equal(Ak[k], M[np.ix_(d, d)])


@pytest.mark.parametrize("weighting", ["left", "sym"])
def test_apply_ragged_equals_dense_sum(stokes3d_small, weighting):
    """apply_ragged(e_j) is column j of W sum_k V_k^T B_phi(k) V_k (LEFT) or
    W^1/2 (sum_k V_k^T B_phi(k) V_k) W^1/2 (SYM), formed with explicit V_k,
    for a map phi that sends patches to shared database entries of their size."""
    pr = stokes3d_small
    g = np.random.default_rng(11)
    sizes = pr.patch_sizes
    db, phi, first = [], np.empty(pr.n_patches, dtype=np.int64), {}
    for k, s in enumerate(sizes):           # one entry per size; the largest size alternates between two
        key = (int(s), k % 2 if s == sizes.max() else 0)
        if key not in first:
            first[key] = len(db)
            db.append(g.standard_normal((s, s)))
        phi[k] = first[key]
    mult = np.zeros(pr.n)
    S = np.zeros((pr.n, pr.n))
    for k in range(pr.n_patches):
        d = pr.patch_dofs[pr.patch_offsets[k]:pr.patch_offsets[k + 1]]
        V = _restriction(d, pr.n)
        S += V.T @ db[phi[k]] @ V
        mult += V.sum(axis=0)
    W = 1.0 / mult
    if weighting == "left":
        M = np.diag(W) @ S
    else:
        M = np.diag(np.sqrt(W)) @ S @ np.diag(np.sqrt(W))
    for j in g.choice(pr.n, size=25, replace=False):
        e = np.zeros(pr.n)
        e[j] = 1.0
        z = O.apply_ragged(e, pr.patch_offsets, pr.patch_dofs, db, phi, W, weighting)
        assert np.allclose(z, M[:, j], rtol=0, atol=1e-13 * np.abs(M).max())


@pytest.mark.parametrize("weighting", ["left", "sym"])
def test_apply_ragged_on_uniform_offsets_equals_apply(weighting):
    pr = problems.poisson2d_q2(4)
    st = O.setup(pr.rowptr, pr.colidx, pr.vals, pr.n, pr.dofs2d(), 1e-12)
    r = np.random.default_rng(2).uniform(-1, 1, pr.n)
    z1 = O.apply(r, pr.dofs2d(), st["Binv"], st["phi"], st["W"], weighting)
    z2 = O.apply_ragged(r, pr.patch_offsets, pr.patch_dofs, list(st["Binv"]), st["phi"], st["W"], weighting)
    assert np.allclose(z1, z2, rtol=0, atol=1e-14 * np.abs(z1).max())


def test_apply_ragged_block_jacobi_is_the_exact_inverse():
    """Disjoint patches of sizes 1..5 covering all DOFs of a block-diagonal A:
    W = I and Eq. (1) is blockdiag(A_k)^-1, so apply_ragged(A x) = x."""
    g = np.random.default_rng(5)
    sizes = [3, 1, 5, 2, 4, 5, 1]
    n = sum(sizes)
    perm = g.permutation(n)
    A = np.zeros((n, n))
    offsets = np.concatenate([[0], np.cumsum(sizes)])
    inv = []
    for k, s in enumerate(sizes):
        d = perm[offsets[k]:offsets[k + 1]]
        B = g.standard_normal((s, s)) + 2 * s * np.eye(s)
        A[np.ix_(d, d)] = B
        inv.append(np.linalg.inv(B))
    x = g.standard_normal(n)
    W = O.weights(O.multiplicity(n, perm))
    assert np.all(W == 1.0)
    z = O.apply_ragged(A @ x, offsets, perm, inv, np.arange(len(sizes)), W, "left")
    assert np.allclose(z, x, rtol=0, atol=1e-13 * np.abs(x).max())


def test_mlp_forward_hand_worked():
    """A 2-3-3-2 network worked by hand.  Row 1 closes some units of both hidden
    layers; row 2 closes every unit of the second layer, so its logits
    are the output bias alone.  A missing ReLU, a dropped bias or a
    transposed weight changes the numbers (or the shapes)."""
    W1 = np.array([[1.0, 0.0], [0.0, 1.0], [-1.0, -1.0]])
    b1 = np.array([0.5, -3.0, 1.0])
    W2 = np.array([[2.0, 1.0, 0.0], [0.0, 1.0, -1.0], [1.0, 1.0, 1.0]])
    b2 = np.array([0.0, 1.0, -2.0])
    W3 = np.array([[1.0, -1.0, 4.0], [0.5, 2.0, 1.0]])
    b3 = np.array([0.25, -1.0])
    X = np.array([[1.0, 2.0], [-1.0, 0.5]])
    logits, (X_, z1, h1, z2, h2) = O.mlp_forward((W1, b1, W2, b2, W3, b3), X)
    # row 1: z1 = (1.5, -1, -2) -> h1 = (1.5, 0, 0); z2 = (3, 1, -0.5) -> h2 = (3, 1, 0)
    # logits = (3 - 1 + 0 + 0.25, 1.5 + 2 + 0 - 1)
    # row 2: z1 = (-0.5, -2.5, 1.5) -> h1 = (0, 0, 1.5); z2 = (0, -0.5, -0.5) -> h2 = 0
    assert np.array_equal(z1, [[1.5, -1.0, -2.0], [-0.5, -2.5, 1.5]])
    assert np.array_equal(h1, [[1.5, 0.0, 0.0], [0.0, 0.0, 1.5]])
    assert np.array_equal(z2, [[3.0, 1.0, -0.5], [0.0, -0.5, -0.5]])
    assert np.array_equal(h2, [[3.0, 1.0, 0.0], [0.0, 0.0, 0.0]])
    assert np.array_equal(logits, [[2.25, 2.5], [0.25, -1.0]])
