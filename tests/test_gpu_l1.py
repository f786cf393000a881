"""Alg. 1 with Experiment 3's entrywise l1 test (||A_i - A_c||_l1 < tol) on
the GPU against the oracle: assignment, entries and evaluation count bit for
bit (the l1 sums differ only in their order; the cases have no near ties),
and the preconditioner built from the entries' inverses equal to the
oracle's Eq. (3)."""
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


@pytest.mark.parametrize("case", ["c1", "diff3d_0.5", "diff3d_2", "stokes8_5"])
def test_alg1_l1_bit_exact(lib, case):
    if case == "c1":
        pr, tol, w, kr = P.poisson2d_q2(16), 1e-3, "sym", "cg"
    elif case.startswith("diff3d"):
        pr, tol, w, kr = P.diffusion3d_q2(6, sigma=0.5, corr_len=3.0, seed=3), float(case.split("_")[1]), "sym", "cg"
    else:
        pr, tol, w, kr = P.stokes2d_q2q1(8), 5.0, "left", "fgmres"
    A = O.extract_patches(pr.rowptr, pr.colidx, pr.vals, pr.n, pr.dofs2d())
    ref = O.alg1_l1(A, tol)
    assert ref["near_ties"] == []
    rp, ci, va = dev(pr.rowptr, torch.int32), dev(pr.colidx, torch.int32), dev(pr.vals, torch.float64)
    ctx = lib.psr_setup(rp, ci, va, dev(pr.patch_dofs, torch.int32), uniform_size=pr.uniform_size,
                        opts=lib.make_opts(tol=tol, weighting=w, krylov=kr, criterion="l1"))
    phi, reps, m = ctx.assignment()
    st = ctx.stats()
    assert np.array_equal(phi.cpu().numpy(), ref["phi"])
    assert np.array_equal(reps.cpu().numpy(), ref["reps"])
    assert st["criterion_evals"] == ref["evals"] and st["rounds"] == m == len(ref["reps"])
    assert np.array_equal(ctx.export_database().cpu().numpy(), A[ref["reps"]])
    r = np.random.default_rng(8).standard_normal(pr.n)
    z = torch.empty(pr.n, dtype=torch.float64, device="cuda")
    ctx.apply(dev(r, torch.float64), z)
    W = O.weights(O.multiplicity(pr.n, pr.patch_dofs))
    zo = O.apply(r, pr.dofs2d(), ref["Binv"], ref["phi"], W, w)
    assert np.abs(z.cpu().numpy() - zo).max() <= 1e-11 * np.abs(zo).max()
    ctx.destroy()


def test_l1_refuses_seeds(lib):
    pr = P.poisson2d_q2(8)
    A = O.extract_patches(pr.rowptr, pr.colidx, pr.vals, pr.n, pr.dofs2d())
    rp, ci, va = dev(pr.rowptr, torch.int32), dev(pr.colidx, torch.int32), dev(pr.vals, torch.float64)
    with pytest.raises(lib.PsrError):
        lib.psr_setup_seeded(rp, ci, va, dev(pr.patch_dofs, torch.int32), pr.uniform_size, dev(A[:2], torch.float64),
                             opts=lib.make_opts(tol=1e-3, criterion="l1"))
