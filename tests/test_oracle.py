"""Pins for the CPU oracle against facts fixed by the paper and by mathematics
(not against the oracle itself).  CPU only."""
import os

import numpy as np
import pytest
import scipy.linalg as sla

import problems as P
from oracle import psr_oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rng(seed=0):
    return np.random.Generator(np.random.PCG64(seed))


# --------------------------------------------------------------------------- a1
def test_extract_matches_dense_submatrix():
    """A_k = V_k A V_k^T (section 2): the principal submatrix of the dense
    matrix (scipy's CSR -> dense conversion, a different route)."""
    pr = P.stokes2d_q2q1(4)
    Ad = pr.to_scipy().toarray()
    dofs = pr.dofs2d()
    Ak = O.extract_patches(pr.rowptr, pr.colidx, pr.vals, pr.n, dofs)
    for k in range(pr.n_patches):
        assert np.array_equal(Ak[k], Ad[np.ix_(dofs[k], dofs[k])])


def test_extract_with_boolean_restriction():
    """Same via explicit boolean V_k (p_s x n) and dense products."""
    pr = P.poisson2d_q2(3)
    Ad = pr.to_scipy().toarray()
    dofs = pr.dofs2d()
    Ak = O.extract_patches(pr.rowptr, pr.colidx, pr.vals, pr.n, dofs)
    for k in range(pr.n_patches):
        V = np.zeros((dofs.shape[1], pr.n))
        V[np.arange(dofs.shape[1]), dofs[k]] = 1.0
        assert np.array_equal(V @ Ad @ V.T, Ak[k])


def test_multiplicity_closed_form_q2():
    """Q2 on an N x N mesh: interior vertices lie in 4 cells, boundary
    (non-corner) vertices and interior edge midpoints in 2, corners, boundary
    edge midpoints and cell centres in 1."""
    N = 5
    pr = P.poisson2d_q2(N)
    mult = O.multiplicity(pr.n, pr.patch_dofs)
    m = 2 * N + 1
    ix, iy = np.meshgrid(np.arange(m), np.arange(m), indexing="xy")
    ix = ix.reshape(-1); iy = iy.reshape(-1)
    ex = np.where(ix % 2 == 1, 1, np.where((ix == 0) | (ix == m - 1), 1, 2))
    ey = np.where(iy % 2 == 1, 1, np.where((iy == 0) | (iy == m - 1), 1, 2))
    assert np.array_equal(mult, ex * ey)
    W = O.weights(mult)
    assert np.array_equal(W * mult, np.ones(pr.n))


def test_weights_reject_uncovered_dof():
    with pytest.raises(ValueError):
        O.weights(np.array([1, 0, 2]))


# --------------------------------------------------------------------------- a2
def test_lu_inverse_residual_bound():
    g = _rng(1)
    for p in (1, 5, 12, 22, 27):
        A = g.standard_normal((6, p, p)) + p * np.eye(p)
        X, sing = O.lu_inverse(A)
        assert not sing.any()
        for b in range(6):
            kappa = np.linalg.cond(A[b])
            err = np.linalg.norm(A[b] @ X[b] - np.eye(p), 2)
            assert err <= 10 * p * O.U_FP64 * kappa


def test_lu_pivots_match_lapack_getrf():
    """Partial pivoting choices equal LAPACK's GETRF (scipy lu_factor)."""
    g = _rng(2)
    for p in (3, 9, 22):
        A = g.standard_normal((p, p))
        L, U, perm, sing = O.lu_factor(A[None])
        lu, piv = sla.lu_factor(A)
        order = np.arange(p)
        for i, pi in enumerate(piv):
            order[[i, pi]] = order[[pi, i]]
        assert np.array_equal(perm[0], order)
        assert np.allclose(np.triu(lu), U[0], atol=1e-12 * np.abs(A).max())


def test_lu_tie_breaks_to_lowest_row():
    A = np.array([[1.0, 2.0], [-1.0, 5.0]])       # |1| == |-1|: keep row 0
    _, _, perm, _ = O.lu_factor(A[None])
    assert list(perm[0]) == [0, 1]
    A = np.array([[0.0, 1.0, 0.0], [2.0, 0.0, 0.0], [-2.0, 0.0, 1.0]])
    _, _, perm, _ = O.lu_factor(A[None])
    assert perm[0, 0] == 1


def test_lu_inverse_special_cases():
    d = np.array([2.0, -4.0, 0.5, 8.0])
    X, _ = O.lu_inverse(np.diag(d)[None])
    assert np.array_equal(X[0], np.diag(1.0 / d))          # exact
    Pm = np.eye(5)[[3, 0, 4, 1, 2]]
    X, _ = O.lu_inverse(Pm[None])
    assert np.array_equal(X[0], Pm.T)                       # exact
    n = 7                                                   # 1D Laplacian, closed form
    T = 2 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)
    i = np.arange(1, n + 1)
    Tinv = np.minimum.outer(i, i) * (n + 1 - np.maximum.outer(i, i)) / (n + 1)
    X, _ = O.lu_inverse(T[None])
    assert np.allclose(X[0], Tinv, rtol=0, atol=1e-14)


def test_lu_flags_singular():
    A = np.array([[1.0, 2.0, 3.0], [2.0, 4.0, 6.0], [1.0, 0.0, 1.0]])
    X, sing = O.lu_inverse(A[None])
    assert sing[0] and np.isnan(X[0]).all()


# --------------------------------------------------------------------------- a3
def test_criterion_identical_is_exactly_zero():
    g = _rng(3)
    A = g.standard_normal((9, 9)) + 9 * np.eye(9)
    X, _ = O.lu_inverse(A[None])
    assert O.criterion(A[None], A[None], X)[0] == 0.0


def test_criterion_scaled_patch():
    """A_i = s A_c  =>  I - A_i A_c^-1 = (1 - s) I, norm |1 - s|."""
    g = _rng(4)
    A = g.standard_normal((12, 12)) + 12 * np.eye(12)
    X, _ = O.lu_inverse(A[None])
    for s in (0.5, 0.999, 1.001, 3.0):
        d = O.criterion((s * A)[None], A[None], X)[0]
        assert abs(d - abs(1 - s)) <= 1e-12


def test_criterion_diagonal_closed_form():
    a = np.array([1.0, 2.0, 3.0, 4.0])
    c = np.array([1.5, 2.0, 2.0, 5.0])
    X, _ = O.lu_inverse(np.diag(c)[None])
    d = O.criterion(np.diag(a)[None], np.diag(c)[None], X)[0]
    assert abs(d - np.max(np.abs(1 - a / c))) <= 1e-15


def test_criterion_known_singular_values():
    """Build A_i so that (A_c - A_i) A_c^-1 = U diag(s) V^T with chosen s."""
    g = _rng(5)
    p = 22
    Ac = g.standard_normal((p, p)) + p * np.eye(p)
    U, _ = np.linalg.qr(g.standard_normal((p, p)))
    V, _ = np.linalg.qr(g.standard_normal((p, p)))
    s = np.sort(g.uniform(0, 0.3, p))[::-1]
    E = U @ np.diag(s) @ V.T
    Ai = Ac - E @ Ac
    X, _ = O.lu_inverse(Ac[None])
    d = O.criterion(Ai[None], Ac[None], X)[0]
    assert abs(d - s[0]) <= 1e-12
    # the paper's form ||I - A_i B^-1|| agrees up to u * kappa
    d2 = np.linalg.norm(np.eye(p) - Ai @ X[0], 2)
    assert abs(d - d2) <= 1e-12


# --------------------------------------------------------------------------- Alg. 1
def test_alg1_poisson2d_nine_classes():
    """Regular mesh, unit coefficient: 4 corner + 4 edge classes + 1
    interior (section 3.1 / section 3.2 boundary partitioning)."""
    pr = P.poisson2d_q2(16)
    st = O.setup(pr.rowptr, pr.colidx, pr.vals, pr.n, pr.dofs2d(), 1e-12)
    assert list(st["reps"]) == [0, 1, 15, 16, 17, 31, 240, 241, 255]
    counts = np.bincount(st["phi"])
    assert list(counts) == [1, 14, 1, 14, 196, 14, 1, 14, 1]
    assert st["near_ties"] == []
    # every patch of a class is bitwise identical to its representative
    A = st["A"]
    for k in range(pr.n_patches):
        assert np.array_equal(A[k], A[st["reps"][st["phi"][k]]])


def test_alg1_uniform_3d_27_classes():
    """rho = 1 on a cube: 27 boundary classes (Exp. 3 reports 27 entries)."""
    pr = P.diffusion3d_q2(4, uniform=True)
    A = O.extract_patches(pr.rowptr, pr.colidx, pr.vals, pr.n, pr.dofs2d())
    res = O.alg1(A, 1e-10)
    assert len(res["reps"]) == 27


def test_alg1_tol_zero_is_full_storage():
    """Strict '< eps' never holds for eps = 0: phi = identity."""
    pr = P.poisson2d_q2(4)
    A = O.extract_patches(pr.rowptr, pr.colidx, pr.vals, pr.n, pr.dofs2d())
    res = O.alg1(A, 0.0)
    assert np.array_equal(res["phi"], np.arange(pr.n_patches))
    assert np.array_equal(res["reps"], np.arange(pr.n_patches))


def test_alg1_recovers_planted_clusters():
    """Prototypes far apart (d >> tol), members perturbed by far less than
    tol: the database is the first occurrence of each prototype, in order."""
    g = _rng(6)
    p, K = 6, 5
    protos = [g.standard_normal((p, p)) + (3 + 2 * k) * np.eye(p) for k in range(K)]
    labels = g.integers(0, K, 60)
    A = np.stack([protos[l] * (1 + 1e-9 * g.standard_normal((p, p))) for l in labels])
    res = O.alg1(A, 1e-4)
    first = [int(np.flatnonzero(labels == l)[0]) for l in dict.fromkeys(labels)]
    assert list(res["reps"]) == first
    order = list(dict.fromkeys(labels))
    assert np.array_equal(res["phi"], [order.index(l) for l in labels])


def test_alg1_first_match_not_closest():
    """Two database entries both within tol: Alg. 1 takes the first."""
    p = 3
    A0 = np.diag([1.0, 1.0, 1.0])
    A1 = np.diag([1.0, 1.0, 1.3])       # d(A1, A0) = 0.3 > tol: new entry
    A2 = np.diag([1.0, 1.0, 1.2])       # d to A0 = 0.2, to A1 = 1/13 ~ 0.077
    res = O.alg1(np.stack([A0, A1, A2]), 0.25)
    assert list(res["reps"]) == [0, 1]
    assert res["phi"][2] == 0
    phi_c, _ = O.alg1_closest(np.stack([A0, A1, A2]), res["reps"], res["Binv"])
    assert phi_c[2] == 1


# --------------------------------------------------------------------------- a4
def _golden_apply():
    rows = {}
    with open(os.path.join(GOLDEN, "apply_3x3.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            k, *v = line.split()
            rows[k] = np.array([float(x) for x in v])
    return rows


def test_apply_hand_worked_3x3():
    gd = _golden_apply()
    A = gd["A"].reshape(3, 3)
    dofs = gd["patches"].astype(int).reshape(2, 2)
    Ak = np.stack([A[np.ix_(d, d)] for d in dofs])
    Binv, _ = O.lu_inverse(Ak)
    W = O.weights(O.multiplicity(3, dofs.reshape(-1)))
    for w in ("left", "sym"):
        M = np.stack([O.apply(e, dofs, Binv, np.arange(2), W, w) for e in np.eye(3)], axis=1)
        assert np.allclose(M, gd[w].reshape(3, 3), rtol=0, atol=1e-15)


def test_apply_identity_matrix_gives_identity():
    pr = P.poisson2d_q2(3)
    dofs = pr.dofs2d()
    p = dofs.shape[1]
    Binv = np.eye(p)[None]
    W = O.weights(O.multiplicity(pr.n, pr.patch_dofs))
    r = _rng(7).standard_normal(pr.n)
    for w in ("left", "sym"):
        z = O.apply(r, dofs, Binv, np.zeros(pr.n_patches, dtype=int), W, w)
        assert np.allclose(z, r, rtol=1e-15, atol=0)


def test_apply_block_jacobi_nonsymmetric():
    """Disjoint patches: W = I and M^-1 = blockdiag(A_k)^-1 exactly (section 2,
    block Jacobi); nonsymmetric blocks catch a transposed inverse."""
    g = _rng(8)
    p, npch = 4, 5
    n = p * npch
    perm = g.permutation(n)
    dofs = perm.reshape(npch, p)
    A = np.zeros((n, n))
    blocks = g.standard_normal((npch, p, p)) + 4 * np.eye(p)
    for k in range(npch):
        A[np.ix_(dofs[k], dofs[k])] = blocks[k]
    Binv, _ = O.lu_inverse(blocks)
    W = O.weights(O.multiplicity(n, dofs.reshape(-1)))
    assert np.array_equal(W, np.ones(n))
    x = g.standard_normal(n)
    z = O.apply(A @ x, dofs, Binv, np.arange(npch), W, "left")
    assert np.allclose(z, x, rtol=1e-12, atol=1e-12)


def test_apply_matches_dense_operator():
    """apply(e_j) = column j of the explicitly formed W sum V^T A^-1 V."""
    pr = P.stokes2d_q2q1(3)
    st = O.setup(pr.rowptr, pr.colidx, pr.vals, pr.n, pr.dofs2d(), 0.0)
    for w in ("left", "sym"):
        M = O.dense_preconditioner(pr.n, pr.dofs2d(), st["Binv"], st["phi"], st["W"], w)
        cols = np.stack([O.apply(e, pr.dofs2d(), st["Binv"], st["phi"], st["W"], w)
                         for e in np.eye(pr.n)], axis=1)
        assert np.allclose(cols, M, rtol=1e-13, atol=1e-13 * np.abs(M).max())


def test_apply_sym_weighting_is_symmetric():
    pr = P.poisson2d_q2(4)
    st = O.setup(pr.rowptr, pr.colidx, pr.vals, pr.n, pr.dofs2d(), 0.0)
    M = O.dense_preconditioner(pr.n, pr.dofs2d(), st["Binv"], st["phi"], st["W"], "sym")
    assert np.allclose(M, M.T, rtol=0, atol=1e-14 * np.abs(M).max())
    assert np.linalg.eigvalsh(0.5 * (M + M.T)).min() > 0


def test_tol_zero_and_exact_classes_reproduce_full_storage():
    """On C1 every class member is bitwise equal to its representative, so the
    tol = 1e-12 database applies bitwise the same operator as full storage."""
    pr = P.poisson2d_q2(16)
    s0 = O.setup(pr.rowptr, pr.colidx, pr.vals, pr.n, pr.dofs2d(), 0.0)
    s1 = O.setup(pr.rowptr, pr.colidx, pr.vals, pr.n, pr.dofs2d(), 1e-12)
    r = _rng(9).standard_normal(pr.n)
    for w in ("left", "sym"):
        z0 = O.apply(r, pr.dofs2d(), s0["Binv"], s0["phi"], s0["W"], w)
        z1 = O.apply(r, pr.dofs2d(), s1["Binv"], s1["phi"], s1["W"], w)
        assert np.array_equal(z0, z1)


# --------------------------------------------------------------------------- a5
def test_pcg_identity_preconditioner_distinct_eigenvalues():
    """CG on a matrix with k distinct eigenvalues terminates in k steps."""
    g = _rng(10)
    n, k = 40, 5
    Q, _ = np.linalg.qr(g.standard_normal((n, n)))
    lam = np.repeat(np.arange(1.0, k + 1), n // k)
    A = Q @ np.diag(lam) @ Q.T
    b = g.standard_normal(n)
    x, hist, it, conv = O.pcg(lambda v: A @ v, lambda v: v, b, rtol=1e-10)
    assert conv and it <= k
    assert np.allclose(x, np.linalg.solve(A, b), atol=1e-8)


def test_fgmres_exact_preconditioner_one_step():
    g = _rng(11)
    n = 30
    A = g.standard_normal((n, n)) + n * np.eye(n)
    Ainv = np.linalg.inv(A)
    b = g.standard_normal(n)
    x, hist, it, conv = O.fgmres(lambda v: A @ v, lambda v: Ainv @ v, b, rtol=1e-10)
    assert conv and it == 1


def test_fgmres_distinct_eigenvalues_and_monotone():
    g = _rng(12)
    n, k = 50, 7
    S = g.standard_normal((n, n)) + 5 * np.eye(n)
    lam = np.resize(np.arange(1.0, k + 1), n)
    A = S @ np.diag(lam) @ np.linalg.inv(S)
    b = g.standard_normal(n)
    x, hist, it, conv = O.fgmres(lambda v: A @ v, lambda v: v, b, restart=30, rtol=1e-9)
    assert conv and it <= k
    assert np.all(np.diff(hist) <= 1e-15)
    assert np.linalg.norm(b - A @ x) / np.linalg.norm(b) <= 1e-8


def test_fgmres_restart_and_true_residual():
    pr = P.poisson2d_q2(8)
    A = pr.to_scipy()
    b = pr.rhs(0)
    x, hist, it, conv = O.fgmres(lambda v: A @ v, lambda v: v, b, restart=5, rtol=1e-8, maxit=5000)
    assert conv and it > 5
    assert np.linalg.norm(b - A @ x) / np.linalg.norm(b) <= 2e-8


def test_c1_full_storage_pcg_converges():
    pr = P.poisson2d_q2(16)
    st = O.setup(pr.rowptr, pr.colidx, pr.vals, pr.n, pr.dofs2d(), 0.0)
    b = pr.rhs(0)
    x, hist, it, conv = O.solve(pr.rowptr, pr.colidx, pr.vals, pr.n, b, st, "cg", "sym")
    assert conv
    assert np.linalg.norm(b - pr.to_scipy() @ x) / np.linalg.norm(b) <= 1e-8 * 1.01
    # the preconditioner helps: plain CG needs more iterations
    _, _, it_plain, _ = O.pcg(lambda v: pr.to_scipy() @ v, lambda v: v, b)
    assert it < it_plain


# --------------------------------------------------------------------------- a6 (MLP)
def _mlp_params(g, d, h, m, scale=0.3):
    return [g.standard_normal((h, d)) * scale, g.standard_normal(h) * 0.1,
            g.standard_normal((h, h)) * scale, g.standard_normal(h) * 0.1,
            g.standard_normal((m, h)) * scale, g.standard_normal(m) * 0.1]


def test_mlp_gradient_matches_finite_differences():
    g = _rng(20)
    d, h, m, B = 7, 6, 4, 5
    params = _mlp_params(g, d, h, m)
    X = g.standard_normal((B, d))
    y = g.integers(0, m, B)
    loss, grads = O.mlp_loss_grad(params, X, y)
    eps = 1e-6
    for li, (Pm, Gm) in enumerate(zip(params, grads)):
        flat = Pm.reshape(-1)
        for idx in g.choice(flat.size, min(flat.size, 6), replace=False):
            old = flat[idx]
            flat[idx] = old + eps
            lp, _ = O.mlp_loss_grad(params, X, y)
            flat[idx] = old - eps
            lm, _ = O.mlp_loss_grad(params, X, y)
            flat[idx] = old
            fd = (lp - lm) / (2 * eps)
            assert abs(fd - Gm.reshape(-1)[idx]) <= 1e-6 * max(1.0, abs(fd)), (li, idx)


def test_softmax_xent_closed_forms():
    m = 7
    loss, G = O.softmax_xent(np.zeros((3, m)), np.array([0, 3, 6]))
    assert abs(loss - np.log(m)) < 1e-15
    assert np.allclose(G.sum(axis=1), 0.0)


def test_adam_first_step_is_signed_lr():
    """With zero state, the bias-corrected first Adam step is lr * sign(g)."""
    p = [np.array([1.0, -2.0, 3.0])]
    gr = [np.array([0.5, -4.0, 1e-3])]
    out, m, v = O.adam_step(p, gr, [np.zeros(3)], [np.zeros(3)], 1, 0.01, eps=0.0)
    assert np.allclose(out[0], p[0] - 0.01 * np.sign(gr[0]), atol=1e-15)


def test_features_scale_invariant_and_log_norm():
    g = _rng(21)
    A = g.standard_normal((3, 4, 4))
    X1 = O.patch_features(A, np.array([1.0, 2.0, 3.0]))
    X2 = O.patch_features(5.0 * A, np.array([1.0, 2.0, 3.0]))
    assert np.allclose(X1[:, :16], X2[:, :16])
    assert np.allclose(X2[:, 16] - X1[:, 16], np.log(5.0))
    assert np.allclose(X1[:, 17], np.log([1.0, 2.0, 3.0]))


def test_alg1_seeded_hints_keep_assignment_valid():
    """Seeded Alg. 1 without hints equals plain Alg. 1 when the seed is the
    plain run's database; correct hints cost one evaluation per patch, wrong
    hints fall back and still give a valid assignment."""
    pr = P.diffusion3d_q2(3, seed=4)
    A = O.extract_patches(pr.rowptr, pr.colidx, pr.vals, pr.n, pr.dofs2d())
    tol = 0.3
    base = O.alg1(A, tol)
    seed_A = A[base["reps"]]
    s0 = O.alg1_seeded(A, tol, seed_A)
    assert np.array_equal(s0["phi"], base["phi"])
    s1 = O.alg1_seeded(A, tol, seed_A, pred=base["phi"])
    assert s1["hits"] == A.shape[0] and s1["evals"] == A.shape[0]
    bad = (base["phi"] + 1) % len(base["reps"])
    s2 = O.alg1_seeded(A, tol, seed_A, pred=bad)
    d = O.criterion(A, A[base["reps"]][s2["phi"]], s2["Binv"][s2["phi"]])
    assert np.all(d < tol)


# ------------------------------------------------------------------ Alg. 2 (entrywise k-means)
def test_kmeans_from_class_representatives_recovers_alg1():
    """Started from the nine C1 class representatives, entrywise k-means
    assigns every patch to its class at once (class members are bitwise
    identical, so their distance to the class mean is rounding-small while
    other classes differ in whole entries), so phi equals Alg. 1's and the
    second sweep changes nothing."""
    pr = P.poisson2d_q2(16)
    A = O.extract_patches(pr.rowptr, pr.colidx, pr.vals, pr.n, pr.dofs2d())
    ref = O.alg1(A, 1e-12)
    km = O.kmeans_l1(A, ref["reps"])
    assert km["sweeps"] == 2
    assert np.array_equal(km["phi"], ref["phi"])
    assert km["near_ties"] == []


def test_kmeans_two_scaled_groups():
    """Patches s_k M with s in two separated groups: two clusters recovered
    from one seed in each, means = (average s) M."""
    g = np.random.default_rng(5)
    M = np.array([[4.0, 1.0, 0.0], [1.0, 3.0, 1.0], [0.0, 1.0, 2.0]])
    s = np.concatenate([1.0 + 0.05 * g.standard_normal(7), 5.0 + 0.05 * g.standard_normal(5)])
    order = g.permutation(12)
    s = s[order]
    A = s[:, None, None] * M
    grp = (s > 3.0).astype(int)
    init = [int(np.flatnonzero(grp == 0)[0]), int(np.flatnonzero(grp == 1)[0])]
    km = O.kmeans_l1(A, init)
    assert np.array_equal(km["phi"], grp)
    for j in range(2):
        assert np.allclose(km["means"][j], s[grp == j].mean() * M, rtol=1e-13, atol=0)
    assert np.allclose(km["Binv"][0] @ km["means"][0], np.eye(3), atol=1e-12)


def test_kmeans_fixed_point_properties():
    """At convergence (Lloyd's fixed point) every patch is assigned to its
    nearest mean and every nonempty mean is the average of its members;
    checked by brute force on random small patches."""
    g = np.random.default_rng(11)
    A = g.standard_normal((40, 3, 3)) + 3.0 * np.eye(3)
    init = g.choice(40, 5, replace=False)
    km = O.kmeans_l1(A, init, max_iter=200)
    assert km["sweeps"] < 200
    phi, B = km["phi"], km["means"]
    for i in range(40):
        d = [np.abs(A[i] - B[j]).sum() for j in range(5)]
        assert d[phi[i]] == min(d)
    for j in range(5):
        mem = np.flatnonzero(phi == j)
        if mem.size:
            assert np.allclose(B[j], A[mem].mean(axis=0), rtol=1e-14, atol=1e-14)


def test_kmeans_every_patch_its_own_mean():
    """m_p = n_p distinct patches as seeds: every patch is nearest to itself
    (distance 0), phi = identity after the first sweep."""
    g = np.random.default_rng(2)
    A = g.standard_normal((9, 4, 4)) + 4.0 * np.eye(4)
    km = O.kmeans_l1(A, np.arange(9))
    assert np.array_equal(km["phi"], np.arange(9)) and km["sweeps"] == 2


def test_alg1_l1_pins():
    """Alg. 1 with Experiment 3's entrywise l1 test: equal patches merge at any
    tol > 0, a scaled copy s A is within tol exactly when |1 - s| ||A||_l1 <
    tol, the first match in creation order wins, and on the uniform Q2 mesh
    the 9 boundary classes come out (Alg. 1's classes)."""
    g = np.random.default_rng(0)
    B = g.standard_normal((4, 4)) + 4 * np.eye(4)
    l1 = np.abs(B).sum()
    A = np.stack([B, 1.1 * B, B, 0.95 * B])
    r = O.alg1_l1(A, 0.08 * l1)                      # 1.1 B: 0.1 l1 > tol; 0.95 B: 0.05 l1 < tol
    assert list(r["phi"]) == [0, 1, 0, 0] and list(r["reps"]) == [0, 1]
    assert r["evals"] == 3                           # 1.1B vs B; B and 0.95B match entry 0 first
    r2 = O.alg1_l1(A, 0.06 * l1)                     # 0.95 B: 0.05 l1 < 0.06 l1 still matches entry 0
    assert list(r2["phi"]) == [0, 1, 0, 0]
    r3 = O.alg1_l1(A, 0.04 * l1)
    assert list(r3["phi"]) == [0, 1, 0, 2]
    pr = P.poisson2d_q2(16)
    Ap = O.extract_patches(pr.rowptr, pr.colidx, pr.vals, pr.n, pr.dofs2d())
    rc = O.alg1_l1(Ap, 1e-3)
    ra = O.alg1(Ap, 1e-3)
    assert len(rc["reps"]) == 9 and np.array_equal(rc["phi"], ra["phi"])
    assert np.allclose(np.einsum("kab,kbc->kac", rc["Binv"], Ap[rc["reps"]]), np.eye(9), atol=1e-12)


def test_kmeans_spectral_pins():
    """Spectral Alg. 2 (d = ||I - A_i B_j^-1||_2, B_j the cluster mean): class
    seeds on C1 reproduce Alg. 1; the final state is a Lloyd fixed point for
    the distance evaluated independently in its naive form (explicit inverse
    and ||I - A B^-1||_2 by SVD); for scaled copies d(sB, B) = |1 - s|, so the
    groups split as the closed form says; seeding with every patch gives
    phi = id (a second sweep confirms it)."""
    pr = P.poisson2d_q2(16)
    A = O.extract_patches(pr.rowptr, pr.colidx, pr.vals, pr.n, pr.dofs2d())
    seeds = np.array([0, 1, 15, 16, 17, 31, 240, 241, 255])
    r = O.kmeans_spectral(A, seeds)
    assert np.array_equal(r["phi"], O.alg1(A, 1e-3)["phi"]) and r["sweeps"] == 2   # assign, then no change
    g = np.random.default_rng(3)
    pd = P.diffusion3d_q2(4, sigma=0.5, corr_len=3.0, seed=1)
    A3 = O.extract_patches(pd.rowptr, pd.colidx, pd.vals, pd.n, pd.dofs2d())
    r3 = O.kmeans_spectral(A3, g.choice(len(A3), 6, replace=False))
    I = np.eye(A3.shape[1])
    dn = np.array([[np.linalg.svd(I - A3[i] @ np.linalg.inv(r3["means"][j]), compute_uv=False)[0]
                    for j in range(6)] for i in range(len(A3))])
    assert np.array_equal(np.argmin(dn, axis=1), r3["phi"])
    for j in range(6):
        mem = np.flatnonzero(r3["phi"] == j)
        if mem.size:
            assert np.allclose(r3["means"][j], A3[mem].mean(axis=0), rtol=0, atol=1e-14 * np.abs(A3).max())
    B = g.standard_normal((5, 5)) + 5 * np.eye(5)
    C = g.standard_normal((5, 5)) + 5 * np.eye(5)
    As = np.stack([B, 1.01 * B, C, 0.99 * C, 1.02 * B])
    assert abs(O.criterion(1.02 * B, B, np.linalg.inv(B)) - 0.02) < 1e-14
    rs = O.kmeans_spectral(As, np.array([0, 2]))
    assert list(rs["phi"]) == [0, 0, 1, 1, 0]
    ri = O.kmeans_spectral(As, np.arange(5))
    assert list(ri["phi"]) == [0, 1, 2, 3, 4] and ri["sweeps"] == 2


def test_kmeans_varmin_pins():
    """Variance-minimising Alg. 2: on C1 with class seeds the representatives
    stay the seeds (all members of a class are equal: every variance is 0 and
    the lowest index wins); for scaled copies d(s_k B, s_m B) = |1 - s_k/s_m|,
    so the medoid is the closed-form minimiser; the final state is a fixed
    point checked by brute force."""
    pr = P.poisson2d_q2(16)
    A = O.extract_patches(pr.rowptr, pr.colidx, pr.vals, pr.n, pr.dofs2d())
    seeds = np.array([0, 1, 15, 16, 17, 31, 240, 241, 255])
    r = O.kmeans_varmin(A, seeds)
    assert np.array_equal(r["phi"], O.alg1(A, 1e-3)["phi"]) and list(r["reps"]) == list(seeds)
    g = np.random.default_rng(4)
    B = g.standard_normal((5, 5)) + 5 * np.eye(5)
    C = g.standard_normal((5, 5)) + 5 * np.eye(5)
    s = np.array([1.0, 1.01, 1.03, 1.06])
    As = np.concatenate([s[:, None, None] * B[None], np.stack([C, 1.02 * C])])
    rs = O.kmeans_varmin(As, np.array([0, 4]))
    assert list(rs["phi"]) == [0, 0, 0, 0, 1, 1]
    V = [sum((1 - sk / sm) ** 2 for sk in s) for sm in s]
    assert rs["reps"][0] == int(np.argmin(V))
    pd = P.diffusion3d_q2(4, sigma=0.5, corr_len=3.0, seed=1)
    A3 = O.extract_patches(pd.rowptr, pd.colidx, pd.vals, pd.n, pd.dofs2d())
    r3 = O.kmeans_varmin(A3, np.random.default_rng(6).choice(len(A3), 5, replace=False))
    I = np.eye(A3.shape[1])
    dn = lambda i, m: np.linalg.svd(I - A3[i] @ np.linalg.inv(A3[m]), compute_uv=False)[0]
    for i in range(len(A3)):
        assert r3["phi"][i] == int(np.argmin([dn(i, m) for m in r3["reps"]]))
    for j, m in enumerate(r3["reps"]):
        mem = np.flatnonzero(r3["phi"] == j)
        if mem.size:
            Vm = [sum(dn(k, c) ** 2 for k in mem) for c in mem]
            assert m == mem[int(np.argmin(Vm))]
