"""Pins of the Experiment 1 workload and of the two-level combination
preconditioner (Eq. 2) in the oracle: nodal convergence of the discrete
solution to the manufactured one, exact bilinear interpolation by P0, the
Galerkin coarse operator equal to the directly assembled Q1 stiffness on
interior vertices (Q1 is a subspace of Q_p and P0 injects it exactly), and
the P0 = I case of Eq. (2)."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spl

import problems as P
from problems import fem
from oracle import psr_oracle as O


def _P0(pr):
    prow, pcol, pval, n0 = pr.meta["P0"]
    return sp.csr_matrix((pval, pcol, prow), shape=(pr.n, n0))


def test_discrete_solution_converges_to_the_manufactured_one():
    errs = []
    for N in (8, 16):
        pr = P.smooth2d_qp(N, 2)
        x = spl.spsolve(pr.to_scipy().tocsc(), pr.meta["b"])
        errs.append(np.abs(x - pr.meta["u_nodes"]).max())
    assert errs[1] < errs[0] / 7.0            # at least O(h^3) at the nodes for Q2
    pr = P.smooth2d_qp(8, 3)
    x = spl.spsolve(pr.to_scipy().tocsc(), pr.meta["b"])
    assert np.abs(x - pr.meta["u_nodes"]).max() < errs[0] / 5.0    # Q3 beats Q2 on the same mesh


@pytest.mark.parametrize("p", [2, 3, 5])
def test_P0_interpolates_bilinear_functions_exactly(p):
    N = 4
    pr = P.smooth2d_qp(N, p)
    P0 = _P0(pr)
    nv, nn = N + 1, N * p + 1
    vx, vy = np.meshgrid(np.arange(nv) / N, np.arange(nv) / N, indexing="xy")
    fx, fy = np.meshgrid(np.arange(nn) / (N * p), np.arange(nn) / (N * p), indexing="xy")
    g = lambda x, y: 1.5 - 2.0 * x + 0.5 * y + 3.0 * x * y
    # within every cell a bilinear function is reproduced; globally the
    # piecewise bilinear interpolant of g is g itself
    assert np.abs(P0 @ g(vx, vy).reshape(-1) - g(fx, fy).reshape(-1)).max() < 1e-13
    assert np.abs(P0 @ np.ones(nv * nv) - 1.0).max() <= 4.0 * np.finfo(float).eps   # partition of unity


def test_galerkin_coarse_operator_is_the_q1_stiffness_inside():
    N, p = 6, 2
    pr = P.smooth2d_qp(N, p)
    A0 = O.coarse_operator(pr.rowptr, pr.colidx, pr.vals, pr.n, pr.meta["P0"])
    assert np.allclose(A0, A0.T, rtol=0, atol=1e-13 * np.abs(A0).max())
    assert np.linalg.eigvalsh(A0).min() > 0
    # Q1 stiffness with rho at the same quadrature points (nq = p + 2)
    nq = p + 2
    xq, _ = fem.gauss_legendre_01(nq)
    _, dphi1, w = fem.tensor_basis(1, 2, nq)
    h = 1.0 / N
    qx = np.array([xq[q % nq] for q in range(nq * nq)])
    qy = np.array([xq[q // nq] for q in range(nq * nq)])
    K1 = np.zeros(((N + 1) ** 2, (N + 1) ** 2))
    for cy in range(N):
        for cx in range(N):
            X, Y = (cx + qx) * h, (cy + qy) * h
            rho = np.sin(np.pi * X) ** 2 * np.sin(np.pi * Y) ** 2 + 0.1
            Ke = np.einsum("q,aq,bq->ab", rho * w, dphi1[0], dphi1[0]) + np.einsum("q,aq,bq->ab", rho * w, dphi1[1], dphi1[1])
            v = [cx + (N + 1) * cy, cx + 1 + (N + 1) * cy, cx + (N + 1) * (cy + 1), cx + 1 + (N + 1) * (cy + 1)]
            K1[np.ix_(v, v)] += Ke
    inner = [i + (N + 1) * j for j in range(2, N - 1) for i in range(2, N - 1)]   # away from Dirichlet nodes
    assert np.abs(A0[np.ix_(inner, inner)] - K1[np.ix_(inner, inner)]).max() <= 1e-12 * np.abs(K1).max()


def test_combo_with_identity_interpolation():
    pr = P.smooth2d_qp(4, 2)
    n = pr.n
    I0 = (np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32), np.ones(n), n)
    A = pr.to_scipy().toarray()
    A0 = O.coarse_operator(pr.rowptr, pr.colidx, pr.vals, n, I0)
    assert np.array_equal(A0, A)
    st = O.setup(pr.rowptr, pr.colidx, pr.vals, n, pr.dofs2d(), 0.0)
    W = O.weights(O.multiplicity(n, pr.patch_dofs))
    x = np.random.default_rng(1).standard_normal(n)
    r = A @ x
    z = O.combo_apply(r, pr.dofs2d(), st["Binv"], st["phi"], W, "left", I0, np.linalg.inv(A0))
    assert np.abs(z - (O.apply(r, pr.dofs2d(), st["Binv"], st["phi"], W, "left") + x)).max() < 1e-9 * np.abs(x).max()


def test_richardson_special_cases():
    # M^-1 = A^-1, omega = 1: one sweep solves A x = b from any x0
    pr = P.smooth2d_qp(4, 2)
    A = pr.to_scipy().toarray()
    b = pr.meta["b"]
    x0 = np.random.default_rng(2).standard_normal(pr.n)
    x1 = O.richardson(pr.rowptr, pr.colidx, pr.vals, pr.n, b, x0, lambda r: np.linalg.solve(A, r), 1.0, 1)
    assert np.abs(A @ x1 - b).max() < 1e-10 * np.abs(b).max()
    # damped Jacobi on [[2, -1], [-1, 2]]: the error contracts by the known
    # factors 1 - omega (1 +- 1/2) per sweep along the eigenvectors (1, +-1)
    rp = np.array([0, 2, 4], dtype=np.int32)
    ci = np.array([0, 1, 0, 1], dtype=np.int32)
    va = np.array([2.0, -1.0, -1.0, 2.0])
    xs = np.array([1.0, 2.0])
    b2 = np.array([0.0, 3.0])                              # A xs
    e0 = np.array([1.0, 1.0]) + np.array([1.0, -1.0])      # eigen-components 1 and 1
    w = 0.6
    x = O.richardson(rp, ci, va, 2, b2, xs + e0, lambda r: r / 2.0, w, 3)
    expect = xs + (1 - w * 0.5) ** 3 * np.array([1.0, 1.0]) + (1 - w * 1.5) ** 3 * np.array([1.0, -1.0])
    assert np.abs(x - expect).max() < 1e-14
