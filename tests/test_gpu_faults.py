"""Failure paths made without a GPU fault: an injected allocation failure
(host side, in the library's caching allocator) must return PSR_ERR_OOM and
leave the library usable; a grid barrier of the Alg. 1 rounds kernel that
waits for a block that never arrives must give up after its bounded spin
and return PSR_ERR_TIMEOUT, with the next setup correct; a NaN in the matrix
must be reported as a singular patch."""
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
    yield L
    L.psr_debug_inject("alloc_fail", 0)
    L.psr_debug_inject("barrier_wait", 0)


def dev(a, dt):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")


def setup(lib, pr, vals=None, **kw):
    vals = pr.vals if vals is None else vals
    return lib.psr_setup(dev(pr.rowptr, torch.int32), dev(pr.colidx, torch.int32), dev(vals, torch.float64),
                         dev(pr.patch_dofs, torch.int32), uniform_size=pr.uniform_size, opts=lib.make_opts(**kw))


def check_correct(lib, pr, tol):
    st = O.setup(pr.rowptr, pr.colidx, pr.vals, pr.n, pr.dofs2d(), tol)
    ctx = setup(lib, pr, tol=tol, weighting="sym", krylov="cg")
    phi, reps, m = ctx.assignment()
    assert np.array_equal(phi.cpu().numpy(), st["phi"])
    r = np.random.default_rng(3).standard_normal(pr.n)
    z = torch.empty(pr.n, dtype=torch.float64, device="cuda")
    ctx.apply(dev(r, torch.float64), z)
    zr = O.apply(r, pr.dofs2d(), st["Binv"], st["phi"], st["W"], "sym")
    assert np.abs(z.cpu().numpy() - zr).max() <= 1e-12 * np.abs(zr).max()
    ctx.destroy()


@pytest.mark.parametrize("k", [1, 2, 3, 5, 8, 13, 21, 34])
def test_injected_allocation_failure(lib, k):
    """The failing setup returns PSR_ERR_OOM and gives back every block it
    had taken (the library's memory in use is what it was before)."""
    pr = P.poisson2d_q2(8)
    before = lib.psr_memory_in_use()
    lib.psr_debug_inject("alloc_fail", k)
    try:
        ctx = setup(lib, pr, tol=1e-12, weighting="sym", krylov="cg")
    except lib.PsrError as e:
        assert "PSR_ERR_OOM" in str(e)
    else:                                    # the setup needed fewer allocations than k
        ctx.destroy()
    lib.psr_debug_inject("alloc_fail", 0)
    assert lib.psr_memory_in_use() == before
    check_correct(lib, pr, 1e-12)


@pytest.mark.parametrize("k", [1, 4, 9, 16, 25, 36])
def test_injected_allocation_failure_large_patches(lib, k):
    """The same on the 3D Stokes patches (33..128 DOFs: the block kernels'
    own buffers) with the closest-match pass."""
    pr = P.stokes3d_q2q1(4, seed=3)
    t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")
    args = (t(pr.rowptr, torch.int32), t(pr.colidx, torch.int32), t(pr.vals, torch.float64),
            t(pr.patch_dofs, torch.int32))
    opts = lib.make_opts(tol=22.0, weighting="left", krylov="fgmres", match="closest")
    before = lib.psr_memory_in_use()
    lib.psr_debug_inject("alloc_fail", k)
    try:
        ctx = lib.psr_setup(*args, offsets=t(pr.patch_offsets, torch.int32), opts=opts)
    except lib.PsrError as e:
        assert "PSR_ERR_OOM" in str(e)
    else:
        ctx.destroy()
    lib.psr_debug_inject("alloc_fail", 0)
    assert lib.psr_memory_in_use() == before


def test_barrier_wait_runs_out(lib):
    """The rounds kernel's barriers wait for one block more than the grid
    holds: every block gives up after 2^14 spins, the setup returns
    PSR_ERR_TIMEOUT, and a setup after restoring the barrier is correct."""
    pr = P.stokes2d_q2q1(8)
    lib.psr_debug_inject("barrier_wait", 1 << 14)
    try:
        with pytest.raises(lib.PsrError) as e:
            setup(lib, pr, tol=1e-1, weighting="left", krylov="fgmres")
        assert "PSR_ERR_TIMEOUT" in str(e.value)
    finally:
        lib.psr_debug_inject("barrier_wait", 0)
    A = O.extract_patches(pr.rowptr, pr.colidx, pr.vals, pr.n, pr.dofs2d())
    ref = O.alg1(A, 1e-1)
    ctx = setup(lib, pr, tol=1e-1, weighting="left", krylov="fgmres")
    phi, reps, m = ctx.assignment()
    assert np.array_equal(phi.cpu().numpy(), ref["phi"])
    ctx.destroy()


def test_nan_in_matrix_is_a_singular_patch(lib):
    """A NaN entry makes the patches holding it fail the pivot test: the
    setup returns PSR_ERR_SINGULAR_PATCH and names one of them."""
    pr = P.poisson2d_q2(8)
    vals = pr.vals.copy()
    row = int(pr.patch_dofs[5 * 9 + 4])              # a DOF of patch 5
    t = int(pr.rowptr[row])
    vals[t] = np.nan
    with pytest.raises(lib.PsrError) as e:
        setup(lib, pr, vals=vals, tol=0.0, weighting="sym", krylov="cg")
    assert "PSR_ERR_SINGULAR_PATCH" in str(e.value)
    patches = [k for k in range(pr.n_patches) if row in pr.dofs2d()[k]]
    named = int(str(e.value).split("patch ")[1].split(" ")[0])
    assert named in patches
    check_correct(lib, pr, 1e-12)


@pytest.mark.parametrize("case", ["poisson", "stokes3d"])
def test_nan_with_norm_window_search(lib, case):
    """A NaN entry under the norm-window search (warp and block norm
    kernels): the NaN patch's norm bracket widens to [0, inf] instead of
    poisoning the window tests, and the setup reports a singular patch."""
    pr = P.poisson2d_q2(8) if case == "poisson" else P.stokes3d_q2q1(4, seed=3)
    vals = pr.vals.copy()
    row = int(pr.patch_dofs[5])
    vals[int(pr.rowptr[row])] = np.nan
    t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")
    args = (t(pr.rowptr, torch.int32), t(pr.colidx, torch.int32), t(vals, torch.float64),
            t(pr.patch_dofs, torch.int32))
    tol = 1e-12 if case == "poisson" else 22.0
    opts = lib.make_opts(tol=tol, weighting=pr.weighting, krylov=pr.krylov, search="norm_window")
    with pytest.raises(lib.PsrError) as e:
        if pr.uniform_size:
            lib.psr_setup(*args, uniform_size=pr.uniform_size, opts=opts)
        else:
            lib.psr_setup(*args, offsets=t(pr.patch_offsets, torch.int32), opts=opts)
    assert "PSR_ERR_SINGULAR_PATCH" in str(e.value)
