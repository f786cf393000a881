"""Finite-element building blocks for the synthetic test problems.

This module produces the INPUT of the method (an assembled sparse matrix and a
cell -> DOF map).  It holds none of the patch-relaxation arithmetic: no patch
extraction, no inverse, no criterion, no sweep.  Both the CPU oracle and the
CUDA path consume what it produces.

Conventions
-----------
* Reference cell is [0,1]^d; tensor-product local numbering with x fastest,
  i.e. local node (a0, a1, a2) -> a0 + (p+1)*a1 + (p+1)^2*a2.
* Gauss-Legendre quadrature with `nq` points per direction.
* Rectilinear cells (sizes h = (hx, hy[, hz])) are integrated through scalar
  factors applied to reference matrices, so two cells with the same h and the
  same coefficient produce bitwise-identical element matrices (the property the
  paper relies on for regular meshes, section 3.1).
"""
from __future__ import annotations

import numpy as np


def gauss_legendre_01(nq: int):
    """nq-point Gauss-Legendre rule mapped to [0, 1]."""
    x, w = np.polynomial.legendre.leggauss(nq)
    return 0.5 * (x + 1.0), 0.5 * w


def lagrange_1d(p: int, x: np.ndarray):
    """Values V[i, q] and derivatives D[i, q] of the p+1 equispaced Lagrange
    polynomials on [0, 1] (nodes i/p) at the points x."""
    x = np.asarray(x, dtype=np.float64)
    nodes = np.linspace(0.0, 1.0, p + 1)
    V = np.zeros((p + 1, x.size))
    D = np.zeros((p + 1, x.size))
    for i in range(p + 1):
        others = [j for j in range(p + 1) if j != i]
        denom = 1.0
        for j in others:
            denom *= nodes[i] - nodes[j]
        val = np.ones_like(x)
        for j in others:
            val = val * (x - nodes[j])
        V[i] = val / denom
        der = np.zeros_like(x)
        for m in others:
            term = np.ones_like(x)
            for j in others:
                if j != m:
                    term = term * (x - nodes[j])
            der = der + term
        D[i] = der / denom
    return V, D


def tensor_basis(p: int, d: int, nq: int):
    """Tensor-product Lagrange basis of degree p on [0,1]^d at the tensor
    Gauss points.

    Returns (phi[a, q], dphi[k, a, q], w[q]) with local index a x-fastest and
    quadrature index q x-fastest.
    """
    xq, wq = gauss_legendre_01(nq)
    V, D = lagrange_1d(p, xq)
    n1 = p + 1
    nb = n1 ** d
    nqt = nq ** d
    phi = np.ones((nb, nqt))
    dphi = np.ones((d, nb, nqt))
    w = np.ones(nqt)
    for a in range(nb):
        ai = [(a // n1 ** k) % n1 for k in range(d)]
        for q in range(nqt):
            qi = [(q // nq ** k) % nq for k in range(d)]
            v = 1.0
            for k in range(d):
                v *= V[ai[k], qi[k]]
            phi[a, q] = v
            for kk in range(d):
                g = 1.0
                for k in range(d):
                    g *= D[ai[k], qi[k]] if k == kk else V[ai[k], qi[k]]
                dphi[kk, a, q] = g
    for q in range(nqt):
        qi = [(q // nq ** k) % nq for k in range(d)]
        for k in range(d):
            w[q] *= wq[qi[k]]
    return phi, dphi, w


def reference_matrices(p: int, d: int, nq: int):
    """Directional stiffness Kdir[k] = int dphi_k dphi_k and mass Mref on the
    unit reference cell."""
    phi, dphi, w = tensor_basis(p, d, nq)
    Kdir = np.einsum("q,kaq,kbq->kab", w, dphi, dphi)
    Mref = np.einsum("q,aq,bq->ab", w, phi, phi)
    # (w*x)*y and (w*y)*x may round differently: make the pair bitwise equal
    Kdir = 0.5 * (Kdir + np.transpose(Kdir, (0, 2, 1)))
    Mref = 0.5 * (Mref + Mref.T)
    return Kdir, Mref


def reference_divergence(pu: int, pp: int, d: int, nq: int):
    """Bref[k, c, a] = int psi_c d(phi_a)/dx_k on the unit cell, psi the degree
    pp pressure basis and phi the degree pu velocity basis."""
    _, dphi, w = tensor_basis(pu, d, nq)
    psi, _, w2 = tensor_basis(pp, d, nq)
    assert np.array_equal(w, w2)
    return np.einsum("q,cq,kaq->kca", w, psi, dphi)


def rect_diffusion_element(Kdir: np.ndarray, h: np.ndarray, rho: np.ndarray):
    """Element stiffness matrices rho_c * int grad phi_a . grad phi_b for
    rectilinear cells.

    h: (nc, d) cell sizes, rho: (nc,) coefficients.  Returns (nc, nb, nb).
    Every cell with equal (h, rho) gets a bitwise-equal matrix.
    """
    nc, d = h.shape
    vol = np.prod(h, axis=1)
    out = np.zeros((nc,) + Kdir.shape[1:])
    for k in range(d):
        s = rho * (vol / (h[:, k] * h[:, k]))
        out += s[:, None, None] * Kdir[k][None]
    return out


def assemble_csr(n: int, edofs: np.ndarray, Ke: np.ndarray, dirichlet: np.ndarray, keep_pattern: bool = False):
    """Assemble element matrices into CSR with symmetric Dirichlet identity
    rows.

    * edofs: (nc, ne) global DOF of each element DOF, cells in lexicographic
      order; Ke: (nc, ne, ne).
    * Each assembled entry is the sum of its element contributions taken in
      increasing cell order (so translation-equivalent cells give bitwise
      equal sums).
    * Rows and columns of Dirichlet DOFs are removed and a unit diagonal is
      put in their place ("a row with only one nonzero"); with keep_pattern
      their entries stay in the sparsity pattern as stored zeros (unit
      diagonal), so every row keeps the symbolic nonzeros of its cells.
    Returns (rowptr int32, colidx int32, vals float64); columns sorted and
    unique in every row.
    """
    nc, ne = edofs.shape
    e64 = edofs.astype(np.int64)
    rows = np.repeat(e64, ne, axis=1).reshape(-1)
    cols = np.tile(e64, (1, ne)).reshape(-1)
    vals = np.ascontiguousarray(Ke, dtype=np.float64).reshape(-1)
    drop = dirichlet[rows] | dirichlet[cols]
    if keep_pattern:
        vals = np.where(drop, 0.0, vals)
    else:
        keep = ~drop
        rows, cols, vals = rows[keep], cols[keep], vals[keep]
    key = rows * n + cols
    order = np.argsort(key, kind="stable")  # keeps cell order inside a key
    key = key[order]
    vals = vals[order]
    del order, rows, cols
    newgrp = np.empty(key.size, dtype=bool)
    if key.size:
        newgrp[0] = True
        np.not_equal(key[1:], key[:-1], out=newgrp[1:])
    starts = np.flatnonzero(newgrp)
    grp = np.cumsum(newgrp) - 1
    rank = np.arange(key.size) - starts[grp]
    sums = np.zeros(starts.size)
    for r in range(int(rank.max()) + 1 if key.size else 0):
        m = rank == r
        sums[grp[m]] += vals[m]  # one contribution per entry per pass
    ukey = key[starts]
    dd = np.flatnonzero(dirichlet).astype(np.int64)
    if keep_pattern:
        sums[np.isin(ukey, dd * n + dd)] = 1.0
    else:
        ukey = np.concatenate([ukey, dd * n + dd])
        sums = np.concatenate([sums, np.ones(dd.size)])
    o2 = np.argsort(ukey, kind="stable")
    ukey = ukey[o2]
    sums = sums[o2]
    r_all = ukey // n
    c_all = ukey - r_all * n
    counts = np.bincount(r_all, minlength=n)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    if rowptr[-1] >= 2 ** 31:
        raise ValueError("nnz exceeds int32 range")
    return rowptr.astype(np.int32), c_all.astype(np.int32), sums
