"""Alg. 1 and the criterion for patches of 33..128 DOFs (block-per-candidate
kernels): the Dirichlet-trimmed 3D Stokes Vanka groups (89 / 62 / 44 DOFs,
the 32-DOF corners take the warp kernels) and the Q5 cells of Experiment 1
(36 DOFs), against the oracle's Alg. 1 per size group (remark after Eq. 1)."""
import numpy as np
import pytest

import problems as P
from oracle import psr_oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    import paper_2306_10025_gb300 as L
    return L


def dev(a, dt):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")


def ctx_for(lib, pr, **kw):
    rp, ci, va = dev(pr.rowptr, torch.int32), dev(pr.colidx, torch.int32), dev(pr.vals, torch.float64)
    if pr.uniform_size:
        return lib.psr_setup(rp, ci, va, dev(pr.patch_dofs, torch.int32), uniform_size=pr.uniform_size,
                             opts=lib.make_opts(**kw))
    return lib.psr_setup(rp, ci, va, dev(pr.patch_dofs, torch.int32), offsets=dev(pr.patch_offsets, torch.int32),
                         opts=lib.make_opts(**kw))


@pytest.mark.parametrize("p", [36, 62, 89, 128])
def test_criterion_big_vs_exact_norm(lib, p):
    """psr_criterion at p > 32: the decision equals sigma_max(E) < tol (numpy
    SVD of the difference form) away from near ties; an accepted value bounds
    d from above, a rejected one from below."""
    g = np.random.default_rng(p)
    batch = 300
    Ac = g.standard_normal((p, p)) + p * np.eye(p)
    Binv = np.linalg.inv(Ac)
    scale = 10.0 ** g.uniform(-7, 0.5, (batch, 1, 1))
    Ai = Ac[None] + scale * g.standard_normal((batch, p, p))
    Ai[0] = Ac
    Ai[1] = 1.01 * Ac                                  # a scaled copy: d = 0.01 / 1.01
    d = np.linalg.norm(np.matmul(Ac[None] - Ai, Binv[None]), ord=2, axis=(1, 2))
    for tol in (float(np.median(d)), 1e-3, 0.05):
        acc = torch.full((batch,), -7, dtype=torch.int32, device="cuda")
        dv = torch.full((batch,), np.nan, dtype=torch.float64, device="cuda")
        lib.psr_criterion(dev(Ai, torch.float64), dev(Ac, torch.float64), dev(Binv, torch.float64), tol, acc, dv)
        a = acc.cpu().numpy().astype(bool)
        dvh = dv.cpu().numpy()
        far = np.abs(d - tol) > 1e-9 * tol
        assert np.array_equal(a[far], d[far] < tol), (p, tol)
        assert a[0] and dvh[0] == 0.0
        ok = far
        assert np.all(dvh[a & ok] >= d[a & ok] * (1 - 1e-12))
        assert np.all(dvh[~a & ok] <= d[~a & ok] * (1 + 1e-12))


def test_criterion_big_near_tie_goes_exact(lib):
    """tol equal to one candidate's sigma_max: no bound can decide it; the
    others still match the exact norm."""
    p, batch = 62, 64
    g = np.random.default_rng(3)
    Ac = g.standard_normal((p, p)) + p * np.eye(p)
    Binv = np.linalg.inv(Ac)
    Ai = Ac[None] + 10.0 ** g.uniform(-4, -1, (batch, 1, 1)) * g.standard_normal((batch, p, p))
    d = np.linalg.norm(np.matmul(Ac[None] - Ai, Binv[None]), ord=2, axis=(1, 2))
    tol = float(d[7])
    acc = torch.full((batch,), -7, dtype=torch.int32, device="cuda")
    lib.psr_criterion(dev(Ai, torch.float64), dev(Ac, torch.float64), dev(Binv, torch.float64), tol, acc)
    a = acc.cpu().numpy()
    assert a[7] in (0, 1)
    far = np.abs(d - tol) > 1e-9 * tol
    assert np.array_equal(a[far].astype(bool), d[far] < tol)


def _groups(pr):
    """Patch indices of each size group, larger sizes first (the library's
    group order), and the patch matrices of each group in patch order."""
    Alist = O.extract_patches_ragged(pr.rowptr, pr.colidx, pr.vals, pr.n, pr.patch_offsets, pr.patch_dofs)
    sizes = pr.patch_sizes
    out = []
    for s in sorted(set(sizes.tolist()), reverse=True):
        idx = np.flatnonzero(sizes == s)
        out.append((s, idx, np.stack([Alist[k] for k in idx])))
    return out


@pytest.mark.parametrize("case", ["jitter4", "jitter5", "uniform4"])
def test_alg1_big_groups_bit_exact(lib, case):
    """phi, the representatives and the evaluation counts of Alg. 1 per size
    group equal the oracle's (the GPU numbers entries group after group,
    larger patches first)."""
    if case == "jitter4":
        pr, tols = P.stokes3d_q2q1(4, seed=3), [15.0, 22.0, 40.0]
    elif case == "jitter5":
        pr, tols = P.stokes3d_q2q1(5, seed=1), [18.0, 30.0]
    else:
        pr, tols = P.stokes3d_q2q1(4, jitter=0.0), [1e-10, 0.5]
    groups = _groups(pr)
    for tol in tols:
        refs = [O.alg1(A, tol) for _, _, A in groups]
        for r in refs:
            assert r["near_ties"] == [], "oracle reports a near tie; pick another tol"
        ctx = ctx_for(lib, pr, tol=tol, weighting="left", krylov="fgmres")
        phi, reps, m = ctx.assignment()
        phi = phi.cpu().numpy()
        reps = reps.cpu().numpy()
        assert m == sum(len(r["reps"]) for r in refs), (case, tol)
        base = 0
        for (s, idx, _), r in zip(groups, refs):
            mg = len(r["reps"])
            assert np.array_equal(phi[idx] - base, r["phi"]), (case, tol, s)
            assert np.array_equal(reps[base:base + mg], idx[r["reps"]]), (case, tol, s)
            base += mg
        st = ctx.stats()
        assert st["criterion_evals"] == sum(r["evals"] for r in refs), (case, tol)
        ctx.destroy()


def test_alg1_big_uniform_classes():
    """Sanity of the uniform case itself: with no jitter the interior cells'
    patches are bitwise equal, so each size group keeps one entry per
    boundary class (interior 1, faces 6, edges 12, corners 8)."""
    pr = P.stokes3d_q2q1(4, jitter=0.0)
    counts = {s: len(O.alg1(A, 1e-10)["reps"]) for s, _, A in _groups(pr)}
    assert counts == {89: 1, 62: 6, 44: 12, 32: 8}


def test_exp1_q5_alg1_bit_exact(lib):
    """Q5 cells (36 DOFs) of Experiment 1's problem on a 10 x 10 mesh."""
    pr = P.smooth2d_qp(N=10, p=5)
    A = O.extract_patches(pr.rowptr, pr.colidx, pr.vals, pr.n, pr.dofs2d())
    for tol in (0.05, 0.2, 0.5, 2.0):
        ref = O.alg1(A, tol)
        assert ref["near_ties"] == []
        ctx = ctx_for(lib, pr, tol=tol, weighting="left", krylov="fgmres")
        phi, reps, m = ctx.assignment()
        assert m == len(ref["reps"])
        assert np.array_equal(phi.cpu().numpy(), ref["phi"])
        assert np.array_equal(reps.cpu().numpy(), ref["reps"])
        assert ctx.stats()["criterion_evals"] == ref["evals"]
        ctx.destroy()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_clustered_big_apply_vs_oracle(lib, prec):
    """Eq. 3 with the clustered 3D Stokes database (every group at tol 22):
    the apply equals the oracle's apply_ragged with the oracle's databases."""
    pr = P.stokes3d_q2q1(4, seed=3)
    tol = 22.0
    groups = _groups(pr)
    phi = np.empty(pr.n_patches, dtype=np.int64)
    db = []
    for s, idx, A in groups:
        r = O.alg1(A, tol)
        phi[idx] = len(db) + r["phi"]
        db.extend(list(r["Binv"]))
    W = O.weights(O.multiplicity(pr.n, pr.patch_dofs))
    ctx = ctx_for(lib, pr, tol=tol, store_prec=prec, weighting="left", krylov="fgmres")
    assert ctx.stats()["m_p"] < pr.n_patches
    g = np.random.default_rng(4)
    for _ in range(2):
        rv = g.standard_normal(pr.n)
        z = torch.empty(pr.n, dtype=torch.float64, device="cuda")
        ctx.apply(dev(rv, torch.float64), z)
        zr = O.apply_ragged(rv, pr.patch_offsets, pr.patch_dofs, db, phi, W, "left")
        err = np.abs(z.cpu().numpy() - zr).max() / np.abs(zr).max()
        assert err < (1e-12 if prec == "fp64" else 2e-5), err


CLOSEST_CASES = [("diff3d", lambda: P.diffusion3d_q2(4, sigma=0.5, corr_len=3.0, seed=1), 1.0),
                 ("diff3d_b", lambda: P.diffusion3d_q2(4, sigma=1.0, corr_len=2.0, seed=2), 0.8),
                 ("diff3d_b_tight", lambda: P.diffusion3d_q2(4, sigma=1.0, corr_len=2.0, seed=2), 0.3),
                 ("nedelec", lambda: P.nedelec3d(4, seed=5), 1.5),
                 ("stokes", lambda: P.stokes2d_q2q1(8, 1.05), 5.0),
                 ("poisson", lambda: P.poisson2d_q2(8), 1e-12)]


@pytest.mark.parametrize("name,make,tol", CLOSEST_CASES)
def test_closest_match_bit_exact(lib, name, make, tol):
    """opts.match = closest (section 3.1 variant): the representatives are
    Alg. 1's, phi the oracle's alg1_closest_match."""
    pr = make()
    A = O.extract_patches(pr.rowptr, pr.colidx, pr.vals, pr.n, pr.dofs2d())
    ref = O.alg1_closest_match(A, tol)
    assert ref["near_ties"] == []
    first = O.alg1(A, tol)
    ctx = ctx_for(lib, pr, tol=tol, weighting=pr.weighting, krylov=pr.krylov, match="closest")
    phi, reps, m = ctx.assignment()
    assert np.array_equal(reps.cpu().numpy(), ref["reps"])
    assert np.array_equal(phi.cpu().numpy(), ref["phi"])
    assert ctx.stats()["criterion_evals"] >= first["evals"]
    ctx.destroy()


def test_closest_match_differs_from_first_match_somewhere(lib):
    """The chosen cases are not vacuous: on them the two rules give
    different maps (12, 9, 1 and 10 patches move)."""
    moved = 0
    for name, make, tol in CLOSEST_CASES:
        pr = make()
        A = O.extract_patches(pr.rowptr, pr.colidx, pr.vals, pr.n, pr.dofs2d())
        moved += int((O.alg1(A, tol)["phi"] != O.alg1_closest_match(A, tol)["phi"]).sum())
    assert moved >= 30


def _window_clear(A, tol, reps, margin=1e-9):
    """No entry's ||A_c||_2 lies within `margin` (relative) of a patch's
    widened window edge, so that brackets of a few 1e-12 decide membership
    as the oracle's exact norms do.  An entry within 1e-13 of the patch's
    own norm (equal or mirrored patches) is inside on both sides for any
    tol >= 0, brackets included, and is left out of the check."""
    nrm = np.linalg.norm(A, ord=2, axis=(1, 2))
    keys = nrm[np.asarray(reps, dtype=np.int64)]
    same = np.abs(keys[None, :] - nrm[:, None]) <= 1e-13 * nrm[:, None]
    lo = nrm / (1.0 + tol) * (1 - 1e-12)
    gaps = [np.abs(keys[None, :] - lo[:, None]) / lo[:, None]]
    if tol < 1.0:
        hi = nrm / (1.0 - tol) * (1 + 1e-12)
        gaps.append(np.abs(keys[None, :] - hi[:, None]) / hi[:, None])
    return all(float(np.where(same, np.inf, g).min()) > margin for g in gaps)


SORTED_CASES = CLOSEST_CASES + [("diff3d_tight", lambda: P.diffusion3d_q2(4, sigma=1.0, corr_len=2.0, seed=2), 0.05)]


@pytest.mark.parametrize("name,make,tol", SORTED_CASES)
def test_norm_window_search_bit_exact(lib, name, make, tol):
    """opts.search = norm_window (the sorted search of section 3.1): phi,
    the representatives and the evaluation count equal the oracle's
    alg1_sorted, and no more tests are made than in creation order."""
    pr = make()
    A = O.extract_patches(pr.rowptr, pr.colidx, pr.vals, pr.n, pr.dofs2d())
    ref = O.alg1_sorted(A, tol)
    assert _window_clear(A, tol, ref["reps"])
    ctx = ctx_for(lib, pr, tol=tol, weighting=pr.weighting, krylov=pr.krylov, search="norm_window")
    phi, reps, m = ctx.assignment()
    assert np.array_equal(reps.cpu().numpy(), ref["reps"])
    assert np.array_equal(phi.cpu().numpy(), ref["phi"])
    assert ctx.stats()["criterion_evals"] == ref["evals"]
    assert ref["evals"] <= O.alg1(A, tol)["evals"]
    ctx.destroy()


@pytest.mark.parametrize("case", ["jitter4", "q5"])
def test_norm_window_search_big_groups(lib, case):
    """The norm-window search for patches of 33..128 DOFs (the block kernels)
    per size group, against alg1_sorted: phi, representatives, evaluations."""
    if case == "jitter4":
        pr, tols = P.stokes3d_q2q1(4, seed=3), [22.0, 0.9]
        groups = _groups(pr)
    else:
        pr, tols = P.smooth2d_qp(N=10, p=5), [0.2, 0.5]
        groups = [(36, np.arange(pr.n_patches), O.extract_patches(pr.rowptr, pr.colidx, pr.vals, pr.n,
                                                                   pr.dofs2d()))]
    for tol in tols:
        refs = [O.alg1_sorted(A, tol) for _, _, A in groups]
        for (_, _, A), r in zip(groups, refs):
            assert _window_clear(A, tol, r["reps"])
        ctx = ctx_for(lib, pr, tol=tol, weighting="left", krylov="fgmres", search="norm_window")
        phi, reps, m = ctx.assignment()
        phi = phi.cpu().numpy()
        reps = reps.cpu().numpy()
        base = 0
        for (s, idx, _), r in zip(groups, refs):
            mg = len(r["reps"])
            assert np.array_equal(phi[idx] - base, r["phi"]), (case, tol, s)
            assert np.array_equal(reps[base:base + mg], idx[r["reps"]]), (case, tol, s)
            base += mg
        assert m == base
        assert ctx.stats()["criterion_evals"] == sum(r["evals"] for r in refs), (case, tol)
        ctx.destroy()


def test_norm_window_search_rejects_unsupported(lib):
    """The norm-window search is a first-match search of the spectral
    criterion: with closest match or the l1 criterion setup fails."""
    pr = P.poisson2d_q2(4)
    for kw in (dict(match="closest"), dict(criterion="l1")):
        with pytest.raises(lib.PsrError):
            ctx_for(lib, pr, tol=0.1, search="norm_window", **kw)


@pytest.mark.parametrize("N", [64, 128])
def test_norm_window_search_bench_size(lib, N):
    """The norm-window search on the graded Stokes mesh at the benchmark
    sizes (4,096 and 16,384 patches of 22 DOFs, tol 1e-2): phi and the
    representatives of the creation-order search, the evaluation count of
    the oracle's alg1_sorted, below the creation-order count."""
    pr = P.stokes2d_q2q1(N, 1.05)
    tol = 1e-2
    A = O.extract_patches(pr.rowptr, pr.colidx, pr.vals, pr.n, pr.dofs2d())
    ref = O.alg1_sorted(A, tol)
    assert _window_clear(A, tol, ref["reps"])
    ctx = ctx_for(lib, pr, tol=tol, weighting="left", krylov="fgmres", search="norm_window")
    phi, reps, m = ctx.assignment()
    assert np.array_equal(phi.cpu().numpy(), ref["phi"])
    assert np.array_equal(reps.cpu().numpy(), ref["reps"])
    ev = ctx.stats()["criterion_evals"]
    ctx.destroy()
    assert ev == ref["evals"]
    ctx = ctx_for(lib, pr, tol=tol, weighting="left", krylov="fgmres")
    ev0 = ctx.stats()["criterion_evals"]
    ctx.destroy()
    assert ev < ev0


@pytest.mark.parametrize("search", ["creation", "norm_window"])
def test_split_rounds_path_bit_exact(lib, search):
    """The path the Alg. 1 rounds take without a cooperative launch (one
    entry per round, a screen and a decide launch each), forced by the
    rounds_split injection: phi, the entries and the evaluation count of the
    oracle (alg1, or alg1_sorted for the norm window), one round per entry."""
    cases = [("diff3d_b", P.diffusion3d_q2(4, sigma=1.0, corr_len=2.0, seed=2), 0.3),
             ("stokes", P.stokes2d_q2q1(8, 1.05), 5.0),
             ("poisson", P.poisson2d_q2(8), 1e-12)]
    lib.psr_debug_inject("rounds_split", 1)
    try:
        for name, pr, tol in cases:
            A = O.extract_patches(pr.rowptr, pr.colidx, pr.vals, pr.n, pr.dofs2d())
            ref = O.alg1_sorted(A, tol) if search == "norm_window" else O.alg1(A, tol)
            if search == "norm_window":
                assert _window_clear(A, tol, ref["reps"])
            ctx = ctx_for(lib, pr, tol=tol, weighting=pr.weighting, krylov=pr.krylov, search=search)
            phi, reps, m = ctx.assignment()
            st = ctx.stats()
            assert np.array_equal(reps.cpu().numpy(), ref["reps"]), name
            assert np.array_equal(phi.cpu().numpy(), ref["phi"]), name
            assert st["criterion_evals"] == ref["evals"], name
            assert st["rounds"] == m, name
            ctx.destroy()
    finally:
        lib.psr_debug_inject("rounds_split", 0)


@pytest.mark.parametrize("case", ["jitter5", "q5"])
def test_closest_match_big_groups(lib, case):
    """Closest match for patches of 33..128 DOFs (a block per patch after the
    rounds, sigma_max by a certified power iteration): the representatives
    are Alg. 1's and phi the oracle's alg1_closest_match, per size group; the
    cases move patches away from their first match."""
    if case == "jitter5":
        pr, tols = P.stokes3d_q2q1(5, seed=1), [15.0, 22.0]
        groups = _groups(pr)
    else:
        pr, tols = P.smooth2d_qp(N=10, p=5), [0.2, 2.0]
        groups = [(36, np.arange(pr.n_patches), O.extract_patches(pr.rowptr, pr.colidx, pr.vals, pr.n,
                                                                   pr.dofs2d()))]
    moved = 0
    for tol in tols:
        refs = [O.alg1_closest_match(A, tol) for _, _, A in groups]
        for r in refs:
            assert r["near_ties"] == []
        ctx = ctx_for(lib, pr, tol=tol, weighting="left", krylov="fgmres", match="closest")
        phi, reps, m = ctx.assignment()
        phi = phi.cpu().numpy()
        reps = reps.cpu().numpy()
        base = 0
        for (s, idx, A), r in zip(groups, refs):
            mg = len(r["reps"])
            assert np.array_equal(phi[idx] - base, r["phi"]), (case, tol, s)
            assert np.array_equal(reps[base:base + mg], idx[r["reps"]]), (case, tol, s)
            moved += int((r["phi"] != O.alg1(A, tol)["phi"]).sum())
            base += mg
        assert m == base
        ctx.destroy()
    assert moved >= 10
