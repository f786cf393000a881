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
@pytest.mark.parametrize("prec", ["fp64", "fp64-native", "fp32"])
def test_uneven_apply_vs_oracle(lib, stokes3d, kernel, prec):
    """Full storage streams every group through k_sweep_stream; FP64 entries
    as FP32 pairs (default) or with FP64 FMAs, both within the FP64 bar."""
    pr, Binv, W = stokes3d
    arith = "native" if prec == "fp64-native" else "pairs"
    prec = prec.split("-")[0]
    ctx = ctx_for(lib, pr, tol=0.0, store_prec=prec, weighting="left", krylov="fgmres", sweep_kernel=kernel,
                  fp64_arith=arith)
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


def test_uneven_apply_bf16_vs_rounded_operator(lib, stokes3d):
    """BF16 full storage of the uneven groups: equal, up to FP32
    accumulation, to the exactly summed product of the symmetrised inverses
    rounded FP64 -> FP32 -> BF16 (nearest even) with x rounded to FP32."""
    pr, Binv, W = stokes3d

    def bf16(x):
        f = np.ascontiguousarray(np.asarray(x, dtype=np.float64).astype(np.float32))
        b = f.view(np.uint32).astype(np.uint64)
        b = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
        return b.astype(np.uint32).view(np.float32).astype(np.float64)

    Bq = [bf16(0.5 * (B + B.T)) for B in Binv]
    ctx = ctx_for(lib, pr, tol=0.0, store_prec="bf16", weighting="left", krylov="fgmres")
    g = np.random.default_rng(8)
    for _ in range(2):
        r = g.standard_normal(pr.n)
        z = torch.empty(pr.n, dtype=torch.float64, device="cuda")
        ctx.apply(dev(r, torch.float64), z)
        rq = r.astype(np.float32).astype(np.float64)
        zr = O.apply_ragged(rq, pr.patch_offsets, pr.patch_dofs, Bq, np.arange(pr.n_patches), W, "left")
        err = np.abs(z.cpu().numpy() - zr).max() / np.abs(zr).max()
        assert err < 2e-6, err


def test_uneven_apply_nan_propagates(lib, stokes3d):
    """A NaN in r reaches z at the DOFs of the patches holding it, and only
    through them: patches without it keep their values (FP64 pairs)."""
    pr, Binv, W = stokes3d
    ctx = ctx_for(lib, pr, tol=0.0, store_prec="fp64", weighting="left", krylov="fgmres")
    r = np.random.default_rng(9).standard_normal(pr.n)
    j = int(pr.patch_dofs[pr.patch_offsets[pr.n_patches // 2]])
    r_nan = r.copy()
    r_nan[j] = np.nan
    z = torch.empty(pr.n, dtype=torch.float64, device="cuda")
    ctx.apply(dev(r_nan, torch.float64), z)
    zc = z.cpu().numpy()
    touched = np.zeros(pr.n, dtype=bool)
    for k in range(pr.n_patches):
        d = pr.patch_dofs[pr.patch_offsets[k]:pr.patch_offsets[k + 1]]
        if j in d:
            touched[d] = True
    assert np.all(np.isnan(zc[touched]))
    zr = O.apply_ragged(np.where(np.isnan(r_nan), 0.0, r_nan), pr.patch_offsets, pr.patch_dofs, Binv,
                        np.arange(pr.n_patches), W, "left")
    # DOFs outside every patch holding j: unaffected by the NaN
    clean = np.ones(pr.n, dtype=bool)
    for k in range(pr.n_patches):
        d = pr.patch_dofs[pr.patch_offsets[k]:pr.patch_offsets[k + 1]]
        if touched[d].any():
            clean[d] = False
    assert clean.any()
    assert np.abs(zc[clean] - zr[clean]).max() <= 1e-12 * np.abs(zr).max()


@pytest.fixture(scope="module")
def stokes3d_8():
    pr = P.stokes3d_q2q1(8, seed=2)
    Alist = O.extract_patches_ragged(pr.rowptr, pr.colidx, pr.vals, pr.n, pr.patch_offsets, pr.patch_dofs)
    Binv = [O.lu_inverse(a[None])[0][0] for a in Alist]
    W = O.weights(O.multiplicity(pr.n, pr.patch_dofs))
    return pr, Binv, W


def test_sorted_sell_smoother_and_fgmres(lib, stokes3d_8):
    """3D Stokes 8^3 (10,854 rows, 69 % padding in slices of consecutive
    rows): the SpMV runs on length-sorted slices with a row map.  Two
    smoothing sweeps (residual b - A x on the sorted slices, Eq. 3 sweep)
    equal the oracle's Richardson iteration, and 40 FGMRES(30) iterations
    follow the oracle's history."""
    pr, Binv, W = stokes3d_8
    A = pr.to_scipy()
    b = pr.rhs(4)
    pc = lambda v: O.apply_ragged(v, pr.patch_offsets, pr.patch_dofs, Binv, np.arange(pr.n_patches), W, "left")
    ctx = ctx_for(lib, pr, tol=0.0, store_prec="fp64", weighting="left", krylov="fgmres", maxit=40)
    x = torch.zeros(pr.n, dtype=torch.float64, device="cuda")
    ctx.smooth(dev(b, torch.float64), x, omega=0.7, sweeps=2)
    xr = O.richardson(pr.rowptr, pr.colidx, pr.vals, pr.n, b, np.zeros(pr.n), pc, 0.7, 2)
    assert np.abs(x.cpu().numpy() - xr).max() <= 1e-11 * np.abs(xr).max()
    _, hist, it, conv = O.fgmres(lambda v: A @ v, pc, b, restart=30, rtol=1e-8, maxit=40)
    x.zero_()
    info = ctx.solve(dev(b, torch.float64), x)
    assert info["iterations"] == it == 40
    h = np.asarray(ctx.history())
    assert np.max(np.abs(h - np.asarray(hist))) <= 1e-10
