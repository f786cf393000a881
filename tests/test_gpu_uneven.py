"""Patches of uneven size (Dirichlet-trimmed 3D Stokes cells: 89/62/44/32
DOFs): grouped persistent sweep vs per-group launches vs the oracle, with the
autotuner on, and the outer FGMRES history."""
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


@pytest.fixture(scope="module")
def stokes3d():
    pr = P.stokes3d_q2q1(4, seed=3)
    Alist = O.extract_patches_ragged(pr.rowptr, pr.colidx, pr.vals, pr.n, pr.patch_offsets, pr.patch_dofs)
    Binv = [O.lu_inverse(a[None])[0][0] for a in Alist]
    W = O.weights(O.multiplicity(pr.n, pr.patch_dofs))
    return pr, Binv, W


def dev(a, dt):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")


def ctx_for(lib, pr, **kw):
    rp, ci, va = dev(pr.rowptr, torch.int32), dev(pr.colidx, torch.int32), dev(pr.vals, torch.float64)
    return lib.psr_setup(rp, ci, va, dev(pr.patch_dofs, torch.int32), offsets=dev(pr.patch_offsets, torch.int32),
                         opts=lib.make_opts(**kw))


def test_sizes_present(stokes3d):
    pr, _, _ = stokes3d
    assert set(np.unique(pr.patch_sizes)) == {32, 44, 62, 89}


@pytest.mark.parametrize("kernel", ["grouped", "pergroup"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_uneven_apply_vs_oracle(lib, stokes3d, kernel, prec):
    pr, Binv, W = stokes3d
    ctx = ctx_for(lib, pr, tol=0.0, store_prec=prec, weighting="left", krylov="fgmres", sweep_kernel=kernel)
    st = ctx.stats()
    assert st["n_groups"] == 4 and st["m_p"] == pr.n_patches
    g = np.random.default_rng(5)
    for _ in range(2):
        r = g.standard_normal(pr.n)
        z = torch.empty(pr.n, dtype=torch.float64, device="cuda")
        ctx.apply(dev(r, torch.float64), z)
        zr = O.apply_ragged(r, pr.patch_offsets, pr.patch_dofs, Binv, np.arange(pr.n_patches), W, "left")
        err = np.abs(z.cpu().numpy() - zr).max() / np.abs(zr).max()
        assert err < (1e-12 if prec == "fp64" else 2e-5), err


def test_uneven_fgmres_history_vs_oracle(lib, stokes3d):
    pr, Binv, W = stokes3d
    A = pr.to_scipy()
    b = pr.rhs(2)
    pc = lambda v: O.apply_ragged(v, pr.patch_offsets, pr.patch_dofs, Binv, np.arange(pr.n_patches), W, "left")
    _, hist, it, conv = O.fgmres(lambda v: A @ v, pc, b, restart=30, rtol=1e-8, maxit=3000)
    assert conv
    ctx = ctx_for(lib, pr, tol=0.0, store_prec="fp64", weighting="left", krylov="fgmres", maxit=3000)
    x = torch.zeros(pr.n, dtype=torch.float64, device="cuda")
    info = ctx.solve(dev(b, torch.float64), x)
    assert info["converged"] and info["iterations"] == it
    h = np.asarray(ctx.history())
    hist = np.asarray(hist)
    assert np.max(np.abs(h - hist)) <= 1e-10
    big = hist >= 1e-4
    assert np.max(np.abs(h[big] - hist[big]) / hist[big]) <= 1e-10


def test_autotuner_keeps_results(lib, stokes3d):
    """Tuned and untuned layouts apply the same operator."""
    pr, _, _ = stokes3d
    r = dev(np.random.default_rng(6).standard_normal(pr.n), torch.float64)
    out = []
    for tune in (False, True):
        ctx = ctx_for(lib, pr, tol=0.0, store_prec="fp64", weighting="left", krylov="fgmres", autotune=tune)
        z = torch.empty(pr.n, dtype=torch.float64, device="cuda")
        ctx.apply(r, z)
        out.append(z.cpu().numpy())
    assert np.abs(out[0] - out[1]).max() <= 1e-13 * np.abs(out[0]).max()
