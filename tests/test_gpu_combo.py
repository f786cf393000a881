"""The two-level combination preconditioner of Eq. (2), M_combo^-1 = M^-1 +
P0 A0^-1 R0 (R0 = P0^T, A0 = R0 A P0, direct coarse solve as in Experiment
1), on the GPU against the oracle: the apply, the FGMRES(20) history, and
Experiment 1 itself (60 x 60 mesh, Q2, full storage), whose iteration count
is the paper's Table 1 value."""
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


def combo_ctx(lib, pr, tol, **kw):
    rp, ci, va = dev(pr.rowptr, torch.int32), dev(pr.colidx, torch.int32), dev(pr.vals, torch.float64)
    ctx = lib.psr_setup(rp, ci, va, dev(pr.patch_dofs, torch.int32), uniform_size=pr.uniform_size,
                        opts=lib.make_opts(tol=tol, weighting="left", krylov="fgmres", **kw))
    prow, pcol, pval, n0 = pr.meta["P0"]
    ctx.set_coarse(dev(prow, torch.int32), dev(pcol, torch.int32), dev(pval, torch.float64), n0)
    return ctx


@pytest.mark.parametrize("p,tol", [(2, 0.0), (2, 0.1), (3, 0.0), (3, 0.1)])
def test_combo_apply_vs_oracle(lib, p, tol):
    pr = P.smooth2d_qp(8, p)
    st = O.setup(pr.rowptr, pr.colidx, pr.vals, pr.n, pr.dofs2d(), tol)
    A0inv = np.linalg.inv(O.coarse_operator(pr.rowptr, pr.colidx, pr.vals, pr.n, pr.meta["P0"]))
    ctx = combo_ctx(lib, pr, tol)
    phi, _, m = ctx.assignment()
    assert np.array_equal(phi.cpu().numpy(), st["phi"])
    r = np.random.default_rng(3).standard_normal(pr.n)
    z = torch.empty(pr.n, dtype=torch.float64, device="cuda")
    ctx.apply(dev(r, torch.float64), z)
    zo = O.combo_apply(r, pr.dofs2d(), st["Binv"], st["phi"], st["W"], "left", pr.meta["P0"], A0inv)
    assert np.abs(z.cpu().numpy() - zo).max() <= 1e-11 * np.abs(zo).max()
    ctx.destroy()


def test_combo_fgmres20_history_vs_oracle(lib):
    pr = P.smooth2d_qp(12, 2)
    tol = 0.1
    st = O.setup(pr.rowptr, pr.colidx, pr.vals, pr.n, pr.dofs2d(), tol)
    A0inv = np.linalg.inv(O.coarse_operator(pr.rowptr, pr.colidx, pr.vals, pr.n, pr.meta["P0"]))
    A = pr.to_scipy()
    b = pr.meta["b"]
    pc = lambda v: O.combo_apply(v, pr.dofs2d(), st["Binv"], st["phi"], st["W"], "left", pr.meta["P0"], A0inv)
    _, hist, it, conv = O.fgmres(lambda v: A @ v, pc, b, restart=20, rtol=1e-8)
    assert conv
    ctx = combo_ctx(lib, pr, tol, restart=20, rtol=1e-8)
    x = torch.zeros(pr.n, dtype=torch.float64, device="cuda")
    info = ctx.solve(dev(b, torch.float64), x)
    assert info["converged"] and info["iterations"] == it
    h = ctx.history()
    assert h.shape == np.asarray(hist).shape and np.max(np.abs(h - hist)) <= 1e-10
    ctx.destroy()


def test_experiment1_iterations(lib):
    """60 x 60 mesh, Q2, full storage, FGMRES(20) + M_combo, x0 = 0, 1e-8:
    11 iterations, the paper's Table 1 count for this case (and the
    oracle's), and the discrete solution to the manufactured one."""
    pr = P.smooth2d_qp(60, 2)
    ctx = combo_ctx(lib, pr, 0.0, restart=20, rtol=1e-8)
    x = torch.zeros(pr.n, dtype=torch.float64, device="cuda")
    info = ctx.solve(dev(pr.meta["b"], torch.float64), x)
    assert info["converged"] and info["iterations"] == 11
    assert np.abs(x.cpu().numpy() - pr.meta["u_nodes"]).max() < 1e-7
    ctx.destroy()


def test_set_coarse_errors(lib):
    pr = P.smooth2d_qp(4, 2)
    rp, ci, va = dev(pr.rowptr, torch.int32), dev(pr.colidx, torch.int32), dev(pr.vals, torch.float64)
    ctx = lib.psr_setup(rp, ci, va, dev(pr.patch_dofs, torch.int32), uniform_size=pr.uniform_size,
                        opts=lib.make_opts(tol=0.0, weighting="left", krylov="fgmres"))
    prow, pcol, pval, n0 = pr.meta["P0"]
    bad = np.array(pcol)
    bad[0] = n0                                          # column out of range
    with pytest.raises(lib.PsrError):
        ctx.set_coarse(dev(prow, torch.int32), dev(bad, torch.int32), dev(pval, torch.float64), n0)
    with pytest.raises(lib.PsrError):
        ctx.set_coarse(dev(prow, torch.int32), dev(pcol, torch.int32), dev(pval, torch.float64), 20000)
    ctx.destroy()


@pytest.mark.parametrize("coarse", [False, True])
def test_smoothing_iteration_vs_oracle(lib, coarse):
    """Experiment 3's smoother x <- x + omega M^-1 (b - A x): three sweeps
    with the patch method (tol 0.1), and with M_combo."""
    pr = P.smooth2d_qp(8, 2)
    tol, omega, sweeps = 0.1, 0.8, 3
    st = O.setup(pr.rowptr, pr.colidx, pr.vals, pr.n, pr.dofs2d(), tol)
    if coarse:
        A0inv = np.linalg.inv(O.coarse_operator(pr.rowptr, pr.colidx, pr.vals, pr.n, pr.meta["P0"]))
        pc = lambda r: O.combo_apply(r, pr.dofs2d(), st["Binv"], st["phi"], st["W"], "left", pr.meta["P0"], A0inv)
        ctx = combo_ctx(lib, pr, tol)
    else:
        pc = lambda r: O.apply(r, pr.dofs2d(), st["Binv"], st["phi"], st["W"], "left")
        rp, ci, va = dev(pr.rowptr, torch.int32), dev(pr.colidx, torch.int32), dev(pr.vals, torch.float64)
        ctx = lib.psr_setup(rp, ci, va, dev(pr.patch_dofs, torch.int32), uniform_size=pr.uniform_size,
                            opts=lib.make_opts(tol=tol, weighting="left", krylov="fgmres"))
    b = pr.meta["b"]
    x0 = np.random.default_rng(4).standard_normal(pr.n)
    xo = O.richardson(pr.rowptr, pr.colidx, pr.vals, pr.n, b, x0, pc, omega, sweeps)
    x = dev(x0, torch.float64)
    ctx.smooth(dev(b, torch.float64), x, omega=omega, sweeps=sweeps)
    assert np.abs(x.cpu().numpy() - xo).max() <= 1e-11 * np.abs(xo).max()
    # the error against the discrete solution shrinks
    xs = np.linalg.solve(pr.to_scipy().toarray(), b)
    assert np.abs(x.cpu().numpy() - xs).max() < np.abs(x0 - xs).max()
    with pytest.raises(lib.PsrError):
        ctx.smooth(dev(b, torch.float64), x, sweeps=-1)
    ctx.destroy()
