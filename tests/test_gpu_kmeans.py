"""Alg. 2 (k-means, section 3.2; entrywise and spectral variants) on the GPU vs the CPU oracle:
assignment and sweep count bit-exact, means' inverses within rounding, the
preconditioner built from them equal to the oracle's Eq. (3) apply."""
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


def kmeans_ctx(lib, pr, init, max_iter=100, criterion="l1", patch_class=None, **kw):
    rp, ci, va = dev(pr.rowptr, torch.int32), dev(pr.colidx, torch.int32), dev(pr.vals, torch.float64)
    return lib.psr_setup_kmeans(rp, ci, va, dev(pr.patch_dofs, torch.int32), pr.uniform_size,
                                dev(np.asarray(init), torch.int32), max_iter=max_iter,
                                opts=lib.make_opts(criterion=criterion, **kw), patch_class=patch_class)


def seeds(n_p, m, seed):
    return np.random.default_rng(seed).choice(n_p, m, replace=False).astype(np.int32)


@pytest.mark.parametrize("case", ["c1_classes", "poisson_random", "stokes8", "diff3d", "nedelec"])
def test_kmeans_assignment_bit_exact(lib, case):
    if case == "c1_classes":
        pr = P.poisson2d_q2(16)
        init = np.array([0, 1, 15, 16, 17, 31, 240, 241, 255], dtype=np.int32)
    elif case == "poisson_random":
        pr = P.poisson2d_q2(12)
        init = seeds(pr.n_patches, 12, 1)
    elif case == "stokes8":
        pr = P.stokes2d_q2q1(8)
        init = seeds(pr.n_patches, 10, 2)
    elif case == "diff3d":
        pr = P.diffusion3d_q2(4, seed=3)
        init = seeds(pr.n_patches, 8, 3)
    else:
        pr = P.nedelec3d(4, seed=5)
        init = seeds(pr.n_patches, 16, 4)
    A = O.extract_patches(pr.rowptr, pr.colidx, pr.vals, pr.n, pr.dofs2d())
    ref = O.kmeans_l1(A, init)
    assert ref["near_ties"] == [], "oracle reports a near tie; pick other seeds"
    ctx = kmeans_ctx(lib, pr, init, weighting=pr.weighting, krylov=pr.krylov)
    phi, reps, m = ctx.assignment()
    assert m == len(init)
    assert np.array_equal(phi.cpu().numpy(), ref["phi"]), case
    assert ctx.stats()["rounds"] == ref["sweeps"], case
    # the preconditioner from the k-means database equals the oracle's Eq. (3)
    g = np.random.default_rng(7)
    r = g.standard_normal(pr.n)
    z = torch.empty(pr.n, dtype=torch.float64, device="cuda")
    ctx.apply(dev(r, torch.float64), z)
    W = O.weights(O.multiplicity(pr.n, pr.patch_dofs))
    zo = O.apply(r, pr.dofs2d(), ref["Binv"], ref["phi"], W, pr.weighting)
    assert np.abs(z.cpu().numpy() - zo).max() <= 1e-11 * np.abs(zo).max()
    ctx.destroy()


def test_kmeans_max_iter_and_errors(lib):
    pr = P.stokes2d_q2q1(8)
    A = O.extract_patches(pr.rowptr, pr.colidx, pr.vals, pr.n, pr.dofs2d())
    init = seeds(pr.n_patches, 10, 2)
    ref = O.kmeans_l1(A, init, max_iter=2)
    ctx = kmeans_ctx(lib, pr, init, max_iter=2, weighting="left", krylov="fgmres")
    assert ctx.stats()["rounds"] == 2 == ref["sweeps"]
    assert np.array_equal(ctx.assignment()[0].cpu().numpy(), ref["phi"])
    ctx.destroy()
    with pytest.raises(lib.PsrError):                      # repeated seed
        kmeans_ctx(lib, pr, np.array([3, 3], dtype=np.int32))
    with pytest.raises(lib.PsrError):                      # out of range
        kmeans_ctx(lib, pr, np.array([0, pr.n_patches], dtype=np.int32))


def test_kmeans_solve_converges(lib):
    """PCG with the k-means database (C1, 9 class seeds = the Alg. 1 classes)
    reaches 1e-8 with the iteration count of the Alg. 1 database."""
    pr = P.poisson2d_q2(16)
    b = dev(pr.rhs(0), torch.float64)
    init = np.array([0, 1, 15, 16, 17, 31, 240, 241, 255], dtype=np.int32)
    ctx = kmeans_ctx(lib, pr, init, weighting="sym", krylov="cg")
    x = torch.zeros(pr.n, dtype=torch.float64, device="cuda")
    info = ctx.solve(b, x)
    rp, ci, va = dev(pr.rowptr, torch.int32), dev(pr.colidx, torch.int32), dev(pr.vals, torch.float64)
    c1 = lib.psr_setup(rp, ci, va, dev(pr.patch_dofs, torch.int32), uniform_size=pr.uniform_size,
                       opts=lib.make_opts(tol=1e-12, weighting="sym", krylov="cg"))
    x1 = torch.zeros_like(x)
    info1 = c1.solve(b, x1)
    assert info["converged"] and abs(info["iterations"] - info1["iterations"]) <= 1


def test_kmeans_bootstrapped_from_alg1(lib):
    """Bootstrapping (section 3.2): the representatives of Alg. 1 are the
    initial means of Alg. 2; here 48 of 216 patches change cluster over
    three sweeps, bit for bit as in the oracle."""
    pr = P.diffusion3d_q2(6, sigma=0.5, corr_len=3.0, seed=3)
    A = O.extract_patches(pr.rowptr, pr.colidx, pr.vals, pr.n, pr.dofs2d())
    r1 = O.alg1(A, 0.2)
    assert r1["near_ties"] == []
    rp, ci, va = dev(pr.rowptr, torch.int32), dev(pr.colidx, torch.int32), dev(pr.vals, torch.float64)
    c1 = lib.psr_setup(rp, ci, va, dev(pr.patch_dofs, torch.int32), uniform_size=pr.uniform_size,
                       opts=lib.make_opts(tol=0.2, weighting="sym", krylov="cg"))
    _, reps, m = c1.assignment()
    assert np.array_equal(reps.cpu().numpy(), r1["reps"])
    ref = O.kmeans_l1(A, r1["reps"])
    assert ref["near_ties"] == [] and ref["sweeps"] == 3
    ctx = kmeans_ctx(lib, pr, reps.cpu().numpy().astype(np.int32), weighting="sym", krylov="cg")
    phi, _, mk = ctx.assignment()
    assert mk == m and np.array_equal(phi.cpu().numpy(), ref["phi"])
    assert ctx.stats()["rounds"] == ref["sweeps"]
    assert int((ref["phi"] != r1["phi"]).sum()) == 48
    for c in (c1, ctx):
        c.destroy()


@pytest.mark.parametrize("case", ["c1_classes", "diff3d_random"])
def test_kmeans_spectral_bit_exact(lib, case):
    """Spectral variant: d = ||A_i - B_j||_2 (Jacobi eigenvalues of D^T D on
    the GPU, LAPACK SVD in the oracle)."""
    if case == "c1_classes":
        pr = P.poisson2d_q2(16)
        init = np.array([0, 1, 15, 16, 17, 31, 240, 241, 255], dtype=np.int32)
    else:
        pr = P.diffusion3d_q2(4, sigma=0.5, corr_len=3.0, seed=1)
        init = seeds(pr.n_patches, 6, 5)
    A = O.extract_patches(pr.rowptr, pr.colidx, pr.vals, pr.n, pr.dofs2d())
    ref = O.kmeans_spectral(A, init)
    assert ref["near_ties"] == []
    ctx = kmeans_ctx(lib, pr, init, criterion="spectral", weighting=pr.weighting, krylov=pr.krylov)
    phi, _, m = ctx.assignment()
    assert np.array_equal(phi.cpu().numpy(), ref["phi"]) and ctx.stats()["rounds"] == ref["sweeps"]
    assert np.array_equal(ctx.export_database().cpu().numpy(), ref["means"])
    g = np.random.default_rng(9)
    r = g.standard_normal(pr.n)
    z = torch.empty(pr.n, dtype=torch.float64, device="cuda")
    ctx.apply(dev(r, torch.float64), z)
    W = O.weights(O.multiplicity(pr.n, pr.patch_dofs))
    zo = O.apply(r, pr.dofs2d(), ref["Binv"], ref["phi"], W, pr.weighting)
    assert np.abs(z.cpu().numpy() - zo).max() <= 1e-11 * np.abs(zo).max()
    ctx.destroy()


@pytest.mark.parametrize("case", ["c1_classes", "diff3d_random"])
def test_kmeans_varmin_bit_exact(lib, case):
    """Variance-minimising variant: representatives are the members of least
    in-cluster variance (spectral distance), stored with their own inverses."""
    if case == "c1_classes":
        pr = P.poisson2d_q2(16)
        init = np.array([0, 1, 15, 16, 17, 31, 240, 241, 255], dtype=np.int32)
    else:
        pr = P.diffusion3d_q2(4, sigma=0.5, corr_len=3.0, seed=1)
        init = np.random.default_rng(6).choice(pr.n_patches, 5, replace=False).astype(np.int32)
    A = O.extract_patches(pr.rowptr, pr.colidx, pr.vals, pr.n, pr.dofs2d())
    ref = O.kmeans_varmin(A, init)
    assert ref["near_ties"] == []
    ctx = kmeans_ctx(lib, pr, init, criterion="varmin", weighting=pr.weighting, krylov=pr.krylov)
    phi, reps, m = ctx.assignment()
    assert np.array_equal(phi.cpu().numpy(), ref["phi"]) and np.array_equal(reps.cpu().numpy(), ref["reps"])
    assert ctx.stats()["rounds"] == ref["sweeps"]
    assert np.array_equal(ctx.export_database().cpu().numpy(), A[ref["reps"]])
    r = np.random.default_rng(10).standard_normal(pr.n)
    z = torch.empty(pr.n, dtype=torch.float64, device="cuda")
    ctx.apply(dev(r, torch.float64), z)
    W = O.weights(O.multiplicity(pr.n, pr.patch_dofs))
    zo = O.apply(r, pr.dofs2d(), ref["Binv"], ref["phi"], W, pr.weighting)
    assert np.abs(z.cpu().numpy() - zo).max() <= 1e-11 * np.abs(zo).max()
    ctx.destroy()
    rp, ci, va = dev(pr.rowptr, torch.int32), dev(pr.colidx, torch.int32), dev(pr.vals, torch.float64)
    with pytest.raises(lib.PsrError):                      # Alg. 1 has no variance-minimising form
        lib.psr_setup(rp, ci, va, dev(pr.patch_dofs, torch.int32), uniform_size=pr.uniform_size,
                      opts=lib.make_opts(tol=0.1, criterion="varmin"))


@pytest.mark.parametrize("case,k", [("poisson", 9), ("diff3d", 27), ("stokes", 9)])
def test_boundary_classes_equal_oracle(lib, case, k):
    """The boundary partition (section 3.2): rows of a patch with one nonzero
    entry; 9 classes on a square, 27 on a cube; equal to the oracle's."""
    pr = {"poisson": lambda: P.poisson2d_q2(10), "diff3d": lambda: P.diffusion3d_q2(4, seed=2),
          "stokes": lambda: P.stokes2d_q2q1(8)}[case]()
    rp, ci, va = dev(pr.rowptr, torch.int32), dev(pr.colidx, torch.int32), dev(pr.vals, torch.float64)
    cls, kg = lib.psr_boundary_classes(rp, ci, va, dev(pr.patch_dofs, torch.int32), uniform_size=pr.uniform_size)
    ref, kr = O.boundary_classes(O.extract_patches(pr.rowptr, pr.colidx, pr.vals, pr.n, pr.dofs2d()))
    assert kg == kr == k and np.array_equal(cls.cpu().numpy(), ref)


@pytest.mark.parametrize("criterion", ["l1", "spectral"])
@pytest.mark.parametrize("partition", ["boundary", "mod3"])
def test_partitioned_kmeans_bit_exact(lib, criterion, partition):
    """Each partition clustered on its own: the assignment and sweep count
    equal the oracle's, and no patch leaves its class.  The boundary
    partition takes the proportional split (40 clusters over 27 classes);
    the arbitrary mod-3 partition moves 45 patches away from the
    unpartitioned result, so the class filter is exercised."""
    pr = P.diffusion3d_q2(4, sigma=0.5, corr_len=3.0, seed=4)
    A = O.extract_patches(pr.rowptr, pr.colidx, pr.vals, pr.n, pr.dofs2d())
    if partition == "boundary":
        cls, k = O.boundary_classes(A)
        split = O.proportional_split(cls, 40)
        g = np.random.default_rng(3)
        init = np.concatenate([g.choice(np.flatnonzero(cls == c), split[c], replace=False)
                               for c in range(k)]).astype(np.int32)
        rp, ci, va = dev(pr.rowptr, torch.int32), dev(pr.colidx, torch.int32), dev(pr.vals, torch.float64)
        cls_d, _ = lib.psr_boundary_classes(rp, ci, va, dev(pr.patch_dofs, torch.int32),
                                            uniform_size=pr.uniform_size)
    else:
        cls = (np.arange(pr.n_patches) % 3).astype(np.int32)
        init = np.random.default_rng(7).choice(pr.n_patches, 9, replace=False).astype(np.int32)
        cls_d = dev(cls, torch.int32)
    ref = (O.kmeans_l1 if criterion == "l1" else O.kmeans_spectral)(A, init, classes=cls)
    assert ref["near_ties"] == []
    ctx = kmeans_ctx(lib, pr, init, criterion=criterion, patch_class=cls_d, weighting=pr.weighting,
                     krylov=pr.krylov)
    phi = ctx.assignment()[0].cpu().numpy()
    assert np.array_equal(phi, ref["phi"]) and ctx.stats()["rounds"] == ref["sweeps"]
    assert np.array_equal(cls[init][phi], cls)
    ctx.destroy()


def test_partition_needs_a_seed_per_class(lib):
    pr = P.poisson2d_q2(8)
    cls = dev((np.arange(pr.n_patches) % 2).astype(np.int32), torch.int32)
    with pytest.raises(lib.PsrError):                      # every seed in class 0
        kmeans_ctx(lib, pr, np.array([0, 2, 4], dtype=np.int32), patch_class=cls)
