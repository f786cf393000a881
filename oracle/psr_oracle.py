"""CPU oracle for compressed patch-based relaxation (Harper & Tuminaro,
"Compression and Reduced Representation Techniques for Patch-Based
Relaxation", arXiv 2306.10025).

TEST INFRASTRUCTURE.  This module is a plain, slow FP64 restatement of what
the method computes, written to check the CUDA library against.  Only the test
suite, the smoke check and the benchmark's CPU-baseline leg may import it; the
library never calls it and has no CPU fallback.  It shares no code with the
CUDA path: inputs come from ``problems`` (the seeded generators), everything
else is here.

Every function cites the passage it follows.  Readings adopted where the paper
is silent or ambiguous:

* Criterion form.  The paper writes d(A_i, B_j) = ||I - A_i B_j^{-1}||_2
  (Alg. 1, Eq. 4, Eq. 5).  With B_j the stored patch A_c this equals
  ||(A_c - A_i) B_c^{-1}||_2 exactly in real arithmetic; we evaluate that
  "difference form", which gives exactly 0 for identical patches.
* The 2-norm is "computed exactly by a small SVD" (section 3 remark): the
  largest singular value from LAPACK's SVD (a library primitive).
* Alg. 1: first match in database creation order, strict "< eps".
* Pivoting: partial pivoting, pivot = largest |entry| in the column, lowest
  row index on ties; a pivot with |u_kk| <= p_s * 2^-53 * max|A_k| marks the
  patch singular.
* Weighting: LEFT (the paper's W * sum V^T B^-1 V, Eq. 1 / Eq. 3) and SYM
  (W^1/2 (sum V^T B^-1 V) W^1/2, which is symmetric and used with CG).
* FGMRES residual history = |g_{j+1}| of the Givens-rotated least-squares
  problem (the recursively updated residual norm), divided by ||r_0||.
"""
from __future__ import annotations

import numpy as np

U_FP64 = 2.0 ** -53


# ---------------------------------------------------------------------------
# a1: patch extraction A_k = V_k A V_k^T   (section 2, definition of A_k)
# ---------------------------------------------------------------------------

def csr_lookup(rowptr, colidx, vals, n, rows, cols):
    """A(rows, cols) entrywise for a CSR matrix with sorted unique columns;
    entries absent from the pattern are 0.  Uses the row-major key
    row*n + col, which is sorted over the whole CSR array."""
    rowptr = np.asarray(rowptr, dtype=np.int64)
    r_of = np.repeat(np.arange(n, dtype=np.int64), np.diff(rowptr))
    keys = r_of * n + np.asarray(colidx, dtype=np.int64)
    q = np.asarray(rows, dtype=np.int64) * n + np.asarray(cols, dtype=np.int64)
    pos = np.searchsorted(keys, q)
    pos_c = np.minimum(pos, keys.size - 1)
    hit = (pos < keys.size) & (keys[pos_c] == q)
    out = np.where(hit, np.asarray(vals)[pos_c], 0.0)
    return out


def extract_patches(rowptr, colidx, vals, n, dofs):
    """A_k(i, j) = A(dofs[k, i], dofs[k, j]) for a (n_p, p_s) map of equal-size
    patches (section 2: A_k = V_k A V_k^T, (V_k)_{ij} = 1 iff global DOF j is
    local DOF i of patch k).  Returns (n_p, p_s, p_s)."""
    dofs = np.asarray(dofs, dtype=np.int64)
    npch, p = dofs.shape
    rows = np.repeat(dofs, p, axis=1)          # row index dofs[k, i]
    cols = np.tile(dofs, (1, p))               # col index dofs[k, j]
    return csr_lookup(rowptr, colidx, vals, n, rows, cols).reshape(npch, p, p)


def extract_patches_ragged(rowptr, colidx, vals, n, offsets, flat):
    """Patches of varying size: list of A_k in patch order (Remark after Eq. 1)."""
    out = []
    for k in range(len(offsets) - 1):
        d = np.asarray(flat[offsets[k]:offsets[k + 1]], dtype=np.int64)
        out.append(extract_patches(rowptr, colidx, vals, n, d[None])[0])
    return out


# ---------------------------------------------------------------------------
# a1': multiplicity and W = (sum_l V_l^T V_l)^{-1}   (section 2)
# ---------------------------------------------------------------------------

def multiplicity(n, flat_dofs):
    """mult[i] = number of patches containing global DOF i."""
    return np.bincount(np.asarray(flat_dofs, dtype=np.int64), minlength=n).astype(np.int64)


def weights(mult):
    """W_ii = 1 / mult[i]; a DOF in no patch makes W undefined."""
    if np.any(mult == 0):
        raise ValueError("a DOF belongs to no patch: W = (sum V^T V)^-1 does not exist")
    return 1.0 / mult.astype(np.float64)


# ---------------------------------------------------------------------------
# a2: LU with partial pivoting and the explicit inverse
#     (Eq. 1 needs A_k^{-1}; Exp. 3 factors with GETRF)
# ---------------------------------------------------------------------------

def lu_factor(A):
    """Batched LU with partial pivoting of A (B, p, p): P A = L U.

    Returns (L, U, perm, singular) with perm[b, i] = original row placed at
    row i, L unit lower, U upper, singular[b] True when some pivot satisfies
    |u_kk| <= p * 2^-53 * max|A_b|."""
    A = np.array(A, dtype=np.float64, copy=True)
    if A.ndim == 2:
        A = A[None]
    B, p, _ = A.shape
    U = A.copy()
    L = np.zeros_like(A)
    perm = np.tile(np.arange(p), (B, 1))
    bidx = np.arange(B)
    thresh = p * U_FP64 * np.max(np.abs(A).reshape(B, -1), axis=1)
    singular = np.zeros(B, dtype=bool)
    for k in range(p):
        piv = k + np.argmax(np.abs(U[:, k:, k]), axis=1)   # first max = lowest row
        # swap rows k <-> piv in U, in the computed part of L, and in perm
        rk = U[bidx, k, :].copy()
        U[bidx, k, :] = U[bidx, piv, :]
        U[bidx, piv, :] = rk
        lk = L[bidx, k, :k].copy()
        L[bidx, k, :k] = L[bidx, piv, :k]
        L[bidx, piv, :k] = lk
        pk = perm[bidx, k].copy()
        perm[bidx, k] = perm[bidx, piv]
        perm[bidx, piv] = pk
        pv = U[:, k, k]
        bad = np.abs(pv) <= thresh
        singular |= bad
        safe = np.where(bad, 1.0, pv)
        L[:, k, k] = 1.0
        if k + 1 < p:
            m = U[:, k + 1:, k] / safe[:, None]
            L[:, k + 1:, k] = m
            U[:, k + 1:, k:] -= m[:, :, None] * U[:, None, k, k:]
            U[:, k + 1:, k] = 0.0
    return L, U, perm, singular


def lu_inverse(A):
    """Explicit inverse by solving L U X = P (column by column, forward then
    back substitution).  Returns (Ainv (B,p,p), singular (B,))."""
    L, U, perm, singular = lu_factor(A)
    B, p, _ = U.shape
    # right-hand side P: row i of P is e_{perm[i]}^T
    P = np.zeros((B, p, p))
    P[np.arange(B)[:, None], np.arange(p)[None, :], perm] = 1.0
    Y = np.zeros_like(P)
    for i in range(p):                    # L Y = P, L unit lower
        Y[:, i, :] = P[:, i, :] - np.einsum("bk,bkj->bj", L[:, i, :i], Y[:, :i, :])
    X = np.zeros_like(P)
    diag = np.where(singular[:, None], 1.0, np.diagonal(U, axis1=1, axis2=2))
    for i in range(p - 1, -1, -1):        # U X = Y
        s = Y[:, i, :] - np.einsum("bk,bkj->bj", U[:, i, i + 1:], X[:, i + 1:, :])
        X[:, i, :] = s / diag[:, i, None]
    X[singular] = np.nan
    return X, singular


# ---------------------------------------------------------------------------
# a3: criterion d(A_i, B_c) = ||I - A_i B_c^{-1}||_2 and Alg. 1
# ---------------------------------------------------------------------------

def spectral_norm(E):
    """Largest singular value of each matrix of a (B, m, m) stack ("computed
    exactly by a small SVD", section 3 remark)."""
    E = np.asarray(E, dtype=np.float64)
    if E.ndim == 2:
        E = E[None]
    s = np.linalg.svd(E, compute_uv=False)
    return s[:, 0]


def criterion(A_i, A_c, Binv_c):
    """d(A_i, B_c) with B_c = A_c, evaluated as ||(A_c - A_i) B_c^{-1}||_2.

    Broadcasts: A_i (B,p,p) or (p,p); A_c/Binv_c likewise."""
    D = np.asarray(A_c, dtype=np.float64) - np.asarray(A_i, dtype=np.float64)
    E = np.matmul(D, Binv_c)
    return spectral_norm(E)


def alg1(A, tol, near_tie_rel=1e-6):
    """Alg. 1 (Patch Tolerance Construction) on equal-size patches A (n_p,p,p).

    For i = 1..n_p: compare A_i with the database entries in creation order;
    the first j with ||I - A_i B_j^{-1}||_2 < tol gives phi(i) = j; if none,
    A_i^{-1} is appended and phi(i) = |B|.

    Returns dict(phi, reps, Binv, evals, near_ties, singular) where reps are
    the patch indices whose inverses form the database (in creation order),
    evals counts the criterion evaluations of the printed loop (up to the
    first match), and near_ties lists (i, j, d) with |d - tol| <= near_tie_rel
    * tol among those evaluations.  (Evaluating patch i against all entries
    at once and keeping the first hit gives the same phi as the loop with
    its break.)
    """
    A = np.asarray(A, dtype=np.float64)
    npch, p, _ = A.shape
    phi = np.full(npch, -1, dtype=np.int64)
    reps: list[int] = []
    Binv = np.zeros((0, p, p))
    evals = 0
    near = []
    singular = []
    for i in range(npch):
        j_hit = -1
        if reps:
            d = criterion(A[i][None], A[reps], Binv)
            hits = np.flatnonzero(d < tol)
            j_hit = int(hits[0]) if hits.size else -1
            upto = j_hit + 1 if j_hit >= 0 else len(reps)
            evals += upto
            if tol > 0:
                close = np.flatnonzero(np.abs(d[:upto] - tol) <= near_tie_rel * tol)
                near.extend((i, int(j), float(d[j])) for j in close)
        if j_hit >= 0:
            phi[i] = j_hit
        else:
            inv, sing = lu_inverse(A[i][None])
            if sing[0]:
                singular.append(i)
            reps.append(i)
            Binv = np.concatenate([Binv, inv], axis=0)
            phi[i] = len(reps) - 1
    return {"phi": phi, "reps": np.array(reps, dtype=np.int64), "Binv": Binv,
            "evals": evals, "near_ties": near, "singular": singular}


def alg1_closest(A, reps, Binv):
    """Closest-match assignment (section 3.1, the variant that picks the
    closest of the database entries): argmin_j d(A_i, B_j), lowest j on ties.
    Returns (phi, dmin)."""
    A = np.asarray(A, dtype=np.float64)
    out = np.zeros(A.shape[0], dtype=np.int64)
    dmin = np.zeros(A.shape[0])
    for i in range(A.shape[0]):
        d = criterion(A[i][None], A[reps], Binv)
        out[i] = int(np.argmin(d))
        dmin[i] = d[out[i]]
    return out, dmin


# ---------------------------------------------------------------------------
# a4: apply z = W sum_k V_k^T B_{phi(k)}^{-1} V_k r   (Eq. 1, Eq. 3)
# ---------------------------------------------------------------------------

def apply(r, dofs, Binv, phi, W, weighting="left"):
    """Eq. (3) with equal-size patches dofs (n_p, p_s), database Binv
    (m_p, p_s, p_s), map phi (n_p,), weights W (n,).

    LEFT: z = W * sum_k V_k^T B^{-1} V_k r (the paper's form).
    SYM : z = W^1/2 * sum_k V_k^T B^{-1} V_k (W^1/2 r)."""
    r = np.asarray(r, dtype=np.float64)
    dofs = np.asarray(dofs, dtype=np.int64)
    if weighting == "sym":
        sw = np.sqrt(W)
        rk = (sw * r)[dofs]
    else:
        rk = r[dofs]
    yk = np.einsum("kab,kb->ka", Binv[phi], rk)
    acc = np.zeros_like(r)
    np.add.at(acc, dofs.reshape(-1), yk.reshape(-1))
    if weighting == "sym":
        return np.sqrt(W) * acc
    return W * acc


def apply_ragged(r, offsets, flat, Binv_list, phi, W, weighting="left"):
    """Eq. (3) for patches of varying size; Binv_list[j] is database entry j."""
    r = np.asarray(r, dtype=np.float64)
    sw = np.sqrt(W)
    x = sw * r if weighting == "sym" else r
    acc = np.zeros_like(r)
    for k in range(len(offsets) - 1):
        d = np.asarray(flat[offsets[k]:offsets[k + 1]], dtype=np.int64)
        y = Binv_list[phi[k]] @ x[d]
        np.add.at(acc, d, y)
    return sw * acc if weighting == "sym" else W * acc


def dense_preconditioner(n, dofs, Binv, phi, W, weighting="left"):
    """The n x n matrix W sum_k V_k^T B_{phi(k)}^{-1} V_k formed explicitly
    (tiny meshes only)."""
    M = np.zeros((n, n))
    dofs = np.asarray(dofs, dtype=np.int64)
    for k in range(dofs.shape[0]):
        d = dofs[k]
        M[np.ix_(d, d)] += Binv[phi[k]]
    if weighting == "sym":
        s = np.sqrt(W)
        return s[:, None] * M * s[None, :]
    return W[:, None] * M


# ---------------------------------------------------------------------------
# a5: outer Krylov solvers (x0 = 0, stop at ||r_k|| <= rtol ||r_0||)
# ---------------------------------------------------------------------------

def csr_matvec(rowptr, colidx, vals, x):
    rowptr = np.asarray(rowptr, dtype=np.int64)
    prod = np.asarray(vals) * x[np.asarray(colidx, dtype=np.int64)]
    out = np.add.reduceat(prod, rowptr[:-1]) if prod.size else np.zeros(len(rowptr) - 1)
    out[np.diff(rowptr) == 0] = 0.0
    return out


def pcg(matvec, prec, b, rtol=1e-8, maxit=10000):
    """Preconditioned conjugate gradients (Hestenes-Stiefel), x0 = 0.
    Returns (x, history of ||r_k||/||r_0||, iterations, converged)."""
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros_like(b)
    r = b.copy()
    r0 = np.linalg.norm(r)
    hist = [1.0]
    if r0 == 0.0:
        return x, hist, 0, True
    z = prec(r)
    p = z.copy()
    rz = r @ z
    for k in range(1, maxit + 1):
        q = matvec(p)
        alpha = rz / (p @ q)
        x += alpha * p
        r -= alpha * q
        rn = np.linalg.norm(r)
        hist.append(rn / r0)
        if rn <= rtol * r0:
            return x, hist, k, True
        z = prec(r)
        rz_new = r @ z
        beta = rz_new / rz
        rz = rz_new
        p = z + beta * p
    return x, hist, maxit, False


def fgmres(matvec, prec, b, restart=30, rtol=1e-8, maxit=10000):
    """Flexible GMRES(m) with right preconditioning (Saad 1993), modified
    Gram-Schmidt Arnoldi, Givens rotations, x0 = 0.

    history[k] = |g_{k+1}| / ||r_0|| after inner iteration k (history[0] = 1).
    At a restart x is updated and the true residual b - A x starts the next
    cycle.  Returns (x, history, iterations, converged)."""
    b = np.asarray(b, dtype=np.float64)
    n = b.size
    x = np.zeros(n)
    r = b.copy()
    r0 = np.linalg.norm(r)
    hist = [1.0]
    if r0 == 0.0:
        return x, hist, 0, True
    it = 0
    beta = r0
    m = restart
    while it < maxit:
        V = np.zeros((m + 1, n))
        Z = np.zeros((m, n))
        H = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[0] = r / beta
        j_done = 0
        converged = False
        for j in range(m):
            Z[j] = prec(V[j])
            w = matvec(Z[j])
            for i in range(j + 1):
                H[i, j] = w @ V[i]
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] != 0.0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = np.hypot(H[j, j], H[j + 1, j])
            cs[j] = H[j, j] / den
            sn[j] = H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            it += 1
            j_done = j + 1
            hist.append(abs(g[j + 1]) / r0)
            if abs(g[j + 1]) <= rtol * r0 or it >= maxit or H[j, j] == 0.0:
                converged = abs(g[j + 1]) <= rtol * r0
                break
        k = j_done
        y = np.zeros(k)
        for i in range(k - 1, -1, -1):
            y[i] = (g[i] - H[i, i + 1:k] @ y[i + 1:k]) / H[i, i]
        x = x + Z[:k].T @ y
        if converged:
            return x, hist, it, True
        r = b - matvec(x)
        beta = np.linalg.norm(r)
        if beta == 0.0:
            return x, hist, it, True
    return x, hist, it, False


# ---------------------------------------------------------------------------
# Whole setup (Alg. 1 + inverses) and solve, on equal-size patches
# ---------------------------------------------------------------------------

def setup(rowptr, colidx, vals, n, dofs, tol):
    """Setup of the approximate preconditioner (Eq. 3): extract the patches,
    run Alg. 1 with tolerance tol (tol = 0 never matches: full storage,
    Eq. 1), and compute W."""
    A = extract_patches(rowptr, colidx, vals, n, dofs)
    res = alg1(A, tol)
    mult = multiplicity(n, np.asarray(dofs).reshape(-1))
    res.update({"A": A, "W": weights(mult), "mult": mult, "dofs": np.asarray(dofs)})
    return res


def solve(rowptr, colidx, vals, n, b, st, krylov="cg", weighting="sym",
          restart=30, rtol=1e-8, maxit=10000):
    """Outer solve of A x = b preconditioned by Eq. (3)."""
    mv = lambda v: csr_matvec(rowptr, colidx, vals, v)
    pc = lambda v: apply(v, st["dofs"], st["Binv"], st["phi"], st["W"], weighting)
    if krylov == "cg":
        return pcg(mv, pc, b, rtol=rtol, maxit=maxit)
    return fgmres(mv, pc, b, restart=restart, rtol=rtol, maxit=maxit)


# ---------------------------------------------------------------------------
# a6: learned assignment (not in the paper; the paper leaves deep-learning
#     assisted clustering to future work at the end of section 3.2).
#     Features -> MLP (2 hidden ReLU layers) -> database entry; the exact
#     criterion verifies every prediction; misses run Alg. 1 against the
#     database (seed entries first, in creation order) and may append entries.
# ---------------------------------------------------------------------------

def patch_features(A, coef=None):
    """Per-patch feature vector: the patch entries divided by ||A_k||_F
    (row-major), log ||A_k||_F and log of the cell coefficient (0 when no
    coefficient is given).  A: (n_p, p, p)."""
    A = np.asarray(A, dtype=np.float64)
    npch, p, _ = A.shape
    fro = np.sqrt(np.einsum("kij,kij->k", A, A))
    X = np.zeros((npch, p * p + 2))
    X[:, :p * p] = A.reshape(npch, -1) / fro[:, None]
    X[:, p * p] = np.log(fro)
    X[:, p * p + 1] = 0.0 if coef is None else np.log(np.asarray(coef, dtype=np.float64))
    return X


def mlp_forward(params, X):
    """logits = W3 relu(W2 relu(W1 x + b1) + b2) + b3 for every row x of X.
    params = (W1, b1, W2, b2, W3, b3) with W_l of shape (out, in)."""
    W1, b1, W2, b2, W3, b3 = params
    z1 = X @ W1.T + b1
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2.T + b2
    h2 = np.maximum(z2, 0.0)
    logits = h2 @ W3.T + b3
    return logits, (X, z1, h1, z2, h2)


def softmax_xent(logits, y):
    """Mean cross-entropy of softmax(logits) against integer labels y and its
    gradient with respect to the logits."""
    B = logits.shape[0]
    s = logits - logits.max(axis=1, keepdims=True)
    e = np.exp(s)
    P = e / e.sum(axis=1, keepdims=True)
    loss = -np.mean(np.log(P[np.arange(B), y]))
    G = P.copy()
    G[np.arange(B), y] -= 1.0
    return loss, G / B


def mlp_loss_grad(params, X, y):
    """Loss and gradients (same order as params) by back-propagation."""
    W1, b1, W2, b2, W3, b3 = params
    logits, (X_, z1, h1, z2, h2) = mlp_forward(params, X)
    loss, G3 = softmax_xent(logits, y)
    gW3 = G3.T @ h2
    gb3 = G3.sum(axis=0)
    G2 = (G3 @ W3) * (z2 > 0)
    gW2 = G2.T @ h1
    gb2 = G2.sum(axis=0)
    G1 = (G2 @ W2) * (z1 > 0)
    gW1 = G1.T @ X_
    gb1 = G1.sum(axis=0)
    return loss, (gW1, gb1, gW2, gb2, gW3, gb3)


def adam_step(params, grads, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba), t = 1, 2, ...  Returns new (params, m, v)."""
    out_p, out_m, out_v = [], [], []
    for P_, G_, M_, V_ in zip(params, grads, m, v):
        M2 = beta1 * M_ + (1 - beta1) * G_
        V2 = beta2 * V_ + (1 - beta2) * G_ * G_
        mh = M2 / (1 - beta1 ** t)
        vh = V2 / (1 - beta2 ** t)
        out_p.append(P_ - lr * mh / (np.sqrt(vh) + eps))
        out_m.append(M2)
        out_v.append(V2)
    return out_p, out_m, out_v


def alg1_seeded(A, tol, A_seed, pred=None):
    """Alg. 1 started from a given database (the patches A_seed, inverted
    here) and optionally hinted: for patch i, when pred[i] >= 0 and
    d(A_i, B_pred[i]) < tol the prediction is taken (one evaluation);
    otherwise the database is searched in creation order (first match) and a
    new entry is appended when nothing matches.

    Returns dict(phi, reps (patch index of each new entry, -1 for seed
    entries), Binv, evals, hits)."""
    A = np.asarray(A, dtype=np.float64)
    npch, p, _ = A.shape
    Bs, sing = lu_inverse(A_seed)
    db_A = [a for a in np.asarray(A_seed, dtype=np.float64)]
    db_B = [b for b in Bs]
    reps = [-1] * len(db_A)
    phi = np.full(npch, -1, dtype=np.int64)
    evals = 0
    hits = 0
    for i in range(npch):
        if pred is not None and pred[i] >= 0:
            j = int(pred[i])
            evals += 1
            if criterion(A[i][None], db_A[j][None], db_B[j][None])[0] < tol:
                phi[i] = j
                hits += 1
                continue
        j_hit = -1
        if db_A:
            d = criterion(A[i][None], np.stack(db_A), np.stack(db_B))
            h = np.flatnonzero(d < tol)
            j_hit = int(h[0]) if h.size else -1
            evals += (j_hit + 1) if j_hit >= 0 else len(db_A)
        if j_hit >= 0:
            phi[i] = j_hit
        else:
            inv, _ = lu_inverse(A[i][None])
            db_A.append(A[i])
            db_B.append(inv[0])
            reps.append(i)
            phi[i] = len(db_A) - 1
    return {"phi": phi, "reps": np.array(reps), "Binv": np.stack(db_B), "evals": evals, "hits": hits}


# ---------------------------------------------------------------------------
# Alg. 2 (section 3.2), entrywise variant: a database of m_p entries fixed
# beforehand.  d(A_i, B_j) = ||A_i - B_j||_l1 entrywise; B_j the entrywise
# mean of its cluster (Eq. 6); the stored inverse is the inverse of that mean.
# The initial means are the patches init[0..m_p-1] (m_p distinct patches the
# caller drew at random: Alg. 2 draws them with randperm).  One sweep assigns
# every patch to its nearest mean (ties: the lowest j); when an assignment
# changed the means are recomputed (members summed in increasing patch index;
# a cluster left without members keeps its mean) and another sweep follows.
# ---------------------------------------------------------------------------

def kmeans_l1(A, init, max_iter=100, near_tie_rel=1e-9, classes=None):
    """Returns phi (n_p), means (m_p, p, p), Binv (inverses of the means),
    singular flags, the number of sweeps and the near ties of the last sweep:
    patches with another mean within near_tie_rel (relative) of the nearest,
    where the argmin could differ between two summation orders.
    classes (per patch, e.g. boundary_classes): each partition is clustered
    on its own -- a patch is assigned only to means seeded in its class."""
    A = np.asarray(A, dtype=np.float64)
    npch = A.shape[0]
    init = np.asarray(init, dtype=np.int64)
    m = init.size
    B = A[init].copy()
    phi = np.full(npch, -1, dtype=np.int64)
    flat = A.reshape(npch, -1)
    other = None
    if classes is not None:
        classes = np.asarray(classes)
        other = classes[:, None] != classes[init][None, :]
        assert not other.all(axis=1).any(), "a class without a seed"
    sweeps = 0
    near = []
    while sweeps < max_iter:
        sweeps += 1
        D = np.empty((npch, m))
        for j in range(m):
            D[:, j] = np.abs(flat - B[j].reshape(-1)).sum(axis=1)
        if other is not None:
            D[other] = np.inf
        new = np.argmin(D, axis=1)
        best = D[np.arange(npch), new]
        close = (D <= best[:, None] * (1.0 + near_tie_rel)) & (D > 0.0)
        close[np.arange(npch), new] = False
        # a mean bitwise equal to the nearest one gives a bitwise equal
        # distance in any summation order: that tie resolves to the lowest j
        # everywhere and is not reported
        for i in np.flatnonzero(close.any(axis=1)):
            for j in np.flatnonzero(close[i]):
                if np.array_equal(B[j], B[new[i]]):
                    close[i, j] = False
        near = [int(i) for i in np.flatnonzero(close.any(axis=1))]
        changed = bool(np.any(new != phi))
        phi = new
        if not changed:
            break
        for j in range(m):
            members = np.flatnonzero(phi == j)
            if members.size:
                acc = np.zeros(A.shape[1:])
                for k in members:
                    acc = acc + A[k]
                B[j] = acc / members.size
    Binv, singular = lu_inverse(B)
    return {"phi": phi, "means": B, "Binv": Binv, "singular": singular, "sweeps": sweeps, "near_ties": near}


# ---------------------------------------------------------------------------
# Two-level combination preconditioner (Eq. 2, Experiment 1):
#   M_combo^{-1} = M^{-1} + P0 A0^{-1} R0,  R0 = P0^T,  A0 = R0 A P0,
# M^{-1} the patch method of Eq. (3), P0 the interpolation from the
# low-order representation, and a direct solve with A0 in place of AMG (as
# in Experiment 1).  A0 is formed with library sparse products and inverted
# with LAPACK (np.linalg.inv) once; the apply follows Eq. (2) term by term.
# ---------------------------------------------------------------------------

def coarse_operator(rowptr, colidx, vals, n, P0):
    """A0 = P0^T A P0 (dense n0 x n0) with P0 = (rowptr, colidx, vals, n0)
    an n x n0 CSR."""
    import scipy.sparse as sp
    A = sp.csr_matrix((vals, colidx, rowptr), shape=(n, n))
    prow, pcol, pval, n0 = P0
    Pm = sp.csr_matrix((pval, pcol, prow), shape=(n, n0))
    return np.asarray((Pm.T @ (A @ Pm)).todense(), dtype=np.float64)


def combo_apply(r, dofs, Binv, phi, W, weighting, P0, A0inv):
    """Eq. (2): z = M^{-1} r + P0 (A0^{-1} (P0^T r))."""
    import scipy.sparse as sp
    prow, pcol, pval, n0 = P0
    Pm = sp.csr_matrix((pval, pcol, prow), shape=(len(r), n0))
    return apply(r, dofs, Binv, phi, W, weighting) + Pm @ (A0inv @ (Pm.T @ np.asarray(r, dtype=np.float64)))


# ---------------------------------------------------------------------------
# Smoothing iteration of Experiment 3: x <- x + omega M^{-1} (b - A x),
# repeated `sweeps` times (M^{-1} any preconditioner callable).
# ---------------------------------------------------------------------------

def richardson(rowptr, colidx, vals, n, b, x0, prec, omega, sweeps):
    import scipy.sparse as sp
    A = sp.csr_matrix((vals, colidx, rowptr), shape=(n, n))
    x = np.array(x0, dtype=np.float64, copy=True)
    for _ in range(sweeps):
        x = x + omega * prec(np.asarray(b, dtype=np.float64) - A @ x)
    return x


# ---------------------------------------------------------------------------
# Alg. 1 with the entrywise l1 test of Experiment 3: patch i takes the first
# entry j (creation order) with ||A_i - A_{rep_j}||_l1 < tol (sum of the
# absolute entrywise differences), else it becomes a new entry.  No inverse
# is needed to decide; the database holds the inverses of the entries.
# ---------------------------------------------------------------------------

def alg1_l1(A, tol, near_tie_rel=1e-9):
    A = np.asarray(A, dtype=np.float64)
    npch, p, _ = A.shape
    phi = np.full(npch, -1, dtype=np.int64)
    reps: list[int] = []
    evals = 0
    near = []
    for i in range(npch):
        j_hit = -1
        if reps:
            d = np.abs(A[reps] - A[i][None]).sum(axis=(1, 2))
            hits = np.flatnonzero(d < tol)
            j_hit = int(hits[0]) if hits.size else -1
            upto = j_hit + 1 if j_hit >= 0 else len(reps)
            evals += upto
            close = np.flatnonzero(np.abs(d[:upto] - tol) <= near_tie_rel * tol)
            near.extend((i, int(j), float(d[j])) for j in close)
        if j_hit >= 0:
            phi[i] = j_hit
        else:
            reps.append(i)
            phi[i] = len(reps) - 1
    Binv, singular = lu_inverse(A[reps]) if reps else (np.zeros((0, p, p)), np.zeros(0, dtype=bool))
    return {"phi": phi, "reps": np.array(reps, dtype=np.int64), "Binv": Binv, "evals": evals,
            "near_ties": near, "singular": [reps[k] for k in np.flatnonzero(singular)]}


# ---------------------------------------------------------------------------
# Alg. 2 (section 3.2), spectral variant: the same iteration as kmeans_l1
# with d(A_i, B_j) = ||I - A_i B_j^{-1}||_2, B_j^{-1} the inverse of the
# entrywise mean (recomputed after every update of the means), evaluated in
# the difference form of `criterion` (LAPACK SVD).  The means, their order of
# summation, the tie rule and the stopping rule are those of the entrywise
# variant.
# ---------------------------------------------------------------------------

def kmeans_spectral(A, init, max_iter=100, near_tie_rel=1e-9, classes=None):
    A = np.asarray(A, dtype=np.float64)
    npch = A.shape[0]
    init = np.asarray(init, dtype=np.int64)
    m = init.size
    B = A[init].copy()
    phi = np.full(npch, -1, dtype=np.int64)
    other = None
    if classes is not None:                  # boundary partition, as in kmeans_l1
        classes = np.asarray(classes)
        other = classes[:, None] != classes[init][None, :]
        assert not other.all(axis=1).any(), "a class without a seed"
    sweeps = 0
    near = []
    while sweeps < max_iter:
        sweeps += 1
        D = np.empty((npch, m))
        Bi, _ = lu_inverse(B)
        for j in range(m):
            D[:, j] = criterion(A, B[j][None], Bi[j][None])
        if other is not None:
            D[other] = np.inf
        new = np.argmin(D, axis=1)
        best = D[np.arange(npch), new]
        close = (D <= best[:, None] * (1.0 + near_tie_rel)) & (D > 0.0)
        close[np.arange(npch), new] = False
        for i in np.flatnonzero(close.any(axis=1)):
            for j in np.flatnonzero(close[i]):
                if np.array_equal(B[j], B[new[i]]):
                    close[i, j] = False
        near = [int(i) for i in np.flatnonzero(close.any(axis=1))]
        changed = bool(np.any(new != phi))
        phi = new
        if not changed:
            break
        for j in range(m):
            members = np.flatnonzero(phi == j)
            if members.size:
                acc = np.zeros(A.shape[1:])
                for k in members:
                    acc = acc + A[k]
                B[j] = acc / members.size
    Binv, singular = lu_inverse(B)
    return {"phi": phi, "means": B, "Binv": Binv, "singular": singular, "sweeps": sweeps, "near_ties": near}


# ---------------------------------------------------------------------------
# Alg. 2 (section 3.2), variance-minimising variant: d(A_i, B_j) =
# ||I - A_i B_j^{-1}||_2 as in the spectral variant, but B_j is a member of
# its cluster: the member m minimising the in-cluster variance
# sum_{k in C_j} d(A_k, A_m)^2 (sum in increasing k; the lowest m on ties);
# the stored inverse is that member's.  Starts from the patches init as the
# representatives; a cluster left empty keeps its representative.
# ---------------------------------------------------------------------------

def kmeans_varmin(A, init, max_iter=100, near_tie_rel=1e-9):
    A = np.asarray(A, dtype=np.float64)
    npch = A.shape[0]
    reps = np.asarray(init, dtype=np.int64).copy()
    m = reps.size
    Ainv, singular_all = lu_inverse(A)
    phi = np.full(npch, -1, dtype=np.int64)
    sweeps = 0
    near = []
    while sweeps < max_iter:
        sweeps += 1
        D = np.empty((npch, m))
        for j in range(m):
            D[:, j] = criterion(A, A[reps[j]][None], Ainv[reps[j]][None])
        new = np.argmin(D, axis=1)
        best = D[np.arange(npch), new]
        close = (D <= best[:, None] * (1.0 + near_tie_rel)) & (D > 0.0)
        close[np.arange(npch), new] = False
        near = [int(i) for i in np.flatnonzero(close.any(axis=1))]
        changed = bool(np.any(new != phi))
        phi = new
        if not changed:
            break
        for j in range(m):
            members = np.flatnonzero(phi == j)
            if members.size == 0:
                continue
            V = np.zeros(members.size)
            for t, mm in enumerate(members):
                d = criterion(A[members], A[mm][None], Ainv[mm][None])
                acc = 0.0
                for x in d:
                    acc = acc + x * x
                V[t] = acc
            t_best = int(np.argmin(V))
            vclose = np.flatnonzero((V <= V[t_best] * (1.0 + near_tie_rel) + 1e-300) & (np.arange(V.size) != t_best))
            near.extend(int(members[t]) for t in vclose)
            reps[j] = members[t_best]
    return {"phi": phi, "reps": reps, "Binv": Ainv[reps], "singular": singular_all[reps], "sweeps": sweeps,
            "near_ties": near}


# ---------------------------------------------------------------------------
# Patch detection from the matrix alone (section 2, after Figure 1: cell-
# restricted patches are found as the rows with q (p+1)^d stored entries)
# ---------------------------------------------------------------------------

def detect_patches(rowptr, colidx, n, row_nnz):
    """A row with exactly row_nnz = q (p+1)^d stored entries (q components,
    tensor-product cells of degree p in d dimensions) couples only with the
    DOFs of one cell, so its column set is that cell's DOF set.  Returns one
    patch per distinct column set, in the order of the smallest row that has
    it, each patch's DOFs ascending: an int32 array [patches, row_nnz]."""
    seen = set()
    out = []
    for r in range(n):
        a, b = int(rowptr[r]), int(rowptr[r + 1])
        if b - a != row_nnz:
            continue
        key = tuple(sorted(int(c) for c in colidx[a:b]))
        if key in seen:
            continue
        seen.add(key)
        out.append(key)
    return np.array(out, dtype=np.int32).reshape(-1, row_nnz)


# ---------------------------------------------------------------------------
# Boundary partition of the patch matrices (section 3.2, after the Alg. 2
# variants): boundary conditions show as patch rows with one nonzero entry
# ---------------------------------------------------------------------------

def boundary_classes(A):
    """Class of every patch: the set of its rows with exactly one nonzero
    entry (a boundary condition); patches with the same set form one
    partition.  Classes are numbered in the order of their first patch.
    Returns (class per patch, number of classes)."""
    A = np.asarray(A)
    ids = {}
    cls = np.empty(A.shape[0], dtype=np.int32)
    for k in range(A.shape[0]):
        key = tuple(np.flatnonzero(np.count_nonzero(A[k], axis=1) == 1))
        cls[k] = ids.setdefault(key, len(ids))
    return cls, len(ids)


def proportional_split(classes, m_total):
    """Clusters per class in proportion to the class sizes (section 3.2: the
    number of clusters divided between boundary types by patch count):
    round(m_total n_c / n), at least 1 and at most n_c."""
    sizes = np.bincount(np.asarray(classes))
    n = sizes.sum()
    return np.array([min(int(c), max(1, int(np.floor(m_total * c / n + 0.5)))) for c in sizes], dtype=np.int64)


# ---------------------------------------------------------------------------
# Faster / less order-sensitive forms of Alg. 1 (section 3.1, after Alg. 1)
# ---------------------------------------------------------------------------

def alg1_closest_match(A, tol, near_tie_rel=1e-9):
    """Alg. 1 in which A_i joins the closest of the entries that pass the
    test (d < tol) instead of the first one; lowest j on ties.  An entry is
    still created exactly when no entry passes, so the representatives are
    those of alg1; only phi can differ.  near_ties: patches whose two best
    passing distances lie within near_tie_rel of each other."""
    A = np.asarray(A, dtype=np.float64)
    npch, p, _ = A.shape
    phi = np.full(npch, -1, dtype=np.int64)
    reps: list[int] = []
    Binv = np.zeros((0, p, p))
    near = []
    for i in range(npch):
        j_hit = -1
        if reps:
            d = criterion(A[i][None], A[reps], Binv)
            ok = np.flatnonzero(d < tol)
            if ok.size:
                j_hit = int(ok[np.argmin(d[ok])])
                ds = np.sort(d[ok])
                if ds.size > 1 and ds[1] - ds[0] <= near_tie_rel * max(ds[1], 1e-300):
                    near.append(i)
        if j_hit >= 0:
            phi[i] = j_hit
        else:
            inv, _ = lu_inverse(A[i][None])
            reps.append(i)
            Binv = np.concatenate([Binv, inv], axis=0)
            phi[i] = len(reps) - 1
    return {"phi": phi, "reps": np.array(reps, dtype=np.int64), "Binv": Binv, "near_ties": near}


def alg1_sorted(A, tol):
    """Alg. 1 with the entries kept sorted by ||B_j||_2 (the O(n_p log m_p)
    search the paper suggests).  Since d = ||(B_j - A_i) B_j^{-1}||_2 >=
    ||B_j - A_i||_2 / ||B_j||_2 >= | ||B_j||_2 - ||A_i||_2 | / ||B_j||_2,
    an entry can pass only if ||A_i||_2 / (1 + tol) < ||B_j||_2 <
    ||A_i||_2 / (1 - tol) (tol < 1): a binary search finds that window and
    only its entries are tested, in creation order.  The result equals
    alg1's; evals counts the tests made."""
    A = np.asarray(A, dtype=np.float64)
    npch, p, _ = A.shape
    phi = np.full(npch, -1, dtype=np.int64)
    reps: list[int] = []
    Binv = np.zeros((0, p, p))
    norms = np.array([np.linalg.svd(A[k], compute_uv=False)[0] for k in range(npch)])
    keys: list[float] = []          # ||B_j||_2, sorted
    order: list[int] = []           # entry j of each sorted key
    evals = 0
    for i in range(npch):
        a = norms[i]
        lo = a / (1.0 + tol)
        hi = a / (1.0 - tol) if tol < 1.0 else np.inf
        # widened by the rounding of the norms (the window must not lose a match)
        s0 = np.searchsorted(keys, lo * (1 - 1e-12), side="left")
        s1 = np.searchsorted(keys, hi * (1 + 1e-12), side="right")
        cand = sorted(order[s0:s1])
        j_hit = -1
        if cand:
            d = criterion(A[i][None], A[[reps[j] for j in cand]], Binv[cand])
            for c, dj in zip(cand, d):
                evals += 1
                if dj < tol:
                    j_hit = c
                    break
        if j_hit >= 0:
            phi[i] = j_hit
        else:
            inv, _ = lu_inverse(A[i][None])
            reps.append(i)
            Binv = np.concatenate([Binv, inv], axis=0)
            phi[i] = len(reps) - 1
            pos = int(np.searchsorted(keys, norms[i], side="right"))
            keys.insert(pos, float(norms[i]))
            order.insert(pos, len(reps) - 1)
    return {"phi": phi, "reps": np.array(reps, dtype=np.int64), "Binv": Binv, "evals": evals}
