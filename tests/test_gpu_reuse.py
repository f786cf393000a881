"""Database reuse across a matrix sequence (section 3.2: for linear problem
sequences the database of the previous setup initialises the next one):
the database of a setup is exported (psr_export_database) and seeds the
setup of a perturbed matrix with the previous assignment as hints; the
result equals the oracle's seeded Alg. 1 bit for bit and needs fewer
criterion evaluations than a fresh setup."""
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


def csr(pr):
    return dev(pr.rowptr, torch.int32), dev(pr.colidx, torch.int32), dev(pr.vals, torch.float64)


def test_database_reuse_for_a_perturbed_matrix(lib):
    tol = 0.15
    # a "time step": the lognormal coefficient exp(sigma g) with sigma 1.0 -> 1.1
    p1 = P.diffusion3d_q2(5, sigma=1.0, corr_len=1.5, seed=3)
    p2 = P.diffusion3d_q2(5, sigma=1.1, corr_len=1.5, seed=3)
    A1 = O.extract_patches(p1.rowptr, p1.colidx, p1.vals, p1.n, p1.dofs2d())
    A2 = O.extract_patches(p2.rowptr, p2.colidx, p2.vals, p2.n, p2.dofs2d())
    r1 = O.alg1(A1, tol)
    assert r1["near_ties"] == []
    ref = O.alg1_seeded(A2, tol, A1[r1["reps"]], pred=r1["phi"])
    fresh = O.alg1(A2, tol)
    opts = lib.make_opts(tol=tol, weighting="sym", krylov="cg")
    ctx1 = lib.psr_setup(*csr(p1), dev(p1.patch_dofs, torch.int32), uniform_size=p1.uniform_size, opts=opts)
    phi1, reps1, m1 = ctx1.assignment()
    assert np.array_equal(phi1.cpu().numpy(), r1["phi"])
    entries = ctx1.export_database()
    assert tuple(entries.shape) == (m1, 27, 27)
    # the entries are the representatives' patch matrices, bit for bit
    assert np.array_equal(entries.cpu().numpy(), A1[r1["reps"]])
    ctx2 = lib.psr_setup_seeded(*csr(p2), dev(p2.patch_dofs, torch.int32), p2.uniform_size, entries, phi1,
                                opts=opts)
    phi2, _, m2 = ctx2.assignment()
    st = ctx2.stats()
    assert np.array_equal(phi2.cpu().numpy(), ref["phi"])
    assert m2 == len(ref["reps"]) and st["mlp_hits"] == ref["hits"] and st["criterion_evals"] == ref["evals"]
    assert st["criterion_evals"] < fresh["evals"] // 2
    # the second database: the seed entries first, then the new entries' patches of A2
    e2 = ctx2.export_database().cpu().numpy()
    assert np.array_equal(e2[:m1], A1[r1["reps"]])
    new = np.asarray(ref["reps"])[m1:]
    assert np.array_equal(e2[m1:], A2[new])
    # and the reused preconditioner applies like the oracle's Eq. (3)
    g = np.random.default_rng(5)
    r = g.standard_normal(p2.n)
    z = torch.empty(p2.n, dtype=torch.float64, device="cuda")
    ctx2.apply(dev(r, torch.float64), z)
    W = O.weights(O.multiplicity(p2.n, p2.patch_dofs))
    zo = O.apply(r, p2.dofs2d(), ref["Binv"], ref["phi"], W, "sym")
    assert np.abs(z.cpu().numpy() - zo).max() <= 1e-11 * np.abs(zo).max()
    for c in (ctx1, ctx2):
        c.destroy()


def test_export_after_kmeans_and_refusals(lib):
    pr = P.poisson2d_q2(16)
    init = np.array([0, 1, 15, 16, 17, 31, 240, 241, 255], dtype=np.int32)
    A = O.extract_patches(pr.rowptr, pr.colidx, pr.vals, pr.n, pr.dofs2d())
    ref = O.kmeans_l1(A, init)
    ctx = lib.psr_setup_kmeans(*csr(pr), dev(pr.patch_dofs, torch.int32), pr.uniform_size,
                               dev(init, torch.int32), opts=lib.make_opts(weighting="sym", krylov="cg", criterion="l1"))
    means = ctx.export_database().cpu().numpy()
    assert np.array_equal(means, ref["means"])        # Alg. 2 entries: the means
    ctx.destroy()
    # full storage keeps no database copy
    ctx0 = lib.psr_setup(*csr(pr), dev(pr.patch_dofs, torch.int32), uniform_size=pr.uniform_size,
                         opts=lib.make_opts(tol=0.0, weighting="sym", krylov="cg"))
    with pytest.raises(lib.PsrError):
        ctx0.export_database()
    ctx0.destroy()
