"""Per-kernel timing of the outer solve (instrumentation): it must not change
the solve's results, and it counts exactly the launches that did work, with
the algorithmic bytes stated in the header."""
import numpy as np
import pytest

import problems as P

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


def setup_ctx(lib, pr, **kw):
    rp, ci, va = (dev(pr.rowptr, torch.int32), dev(pr.colidx, torch.int32), dev(pr.vals, torch.float64))
    return lib.psr_setup(rp, ci, va, dev(pr.patch_dofs, torch.int32), uniform_size=pr.uniform_size,
                         opts=lib.make_opts(**kw))


@pytest.mark.parametrize("graph,ortho", [(True, "auto"), (False, "auto"), (True, "fp64"), (True, "split")])
def test_fgmres_timing_counts_and_bytes(lib, graph, ortho):
    pr = P.stokes2d_q2q1(8)
    maxit, m = 45, 30
    ctx = setup_ctx(lib, pr, tol=0.0, weighting="left", krylov="fgmres", restart=m, maxit=maxit, use_graph=graph,
                    ortho=ortho)
    b = dev(pr.rhs(0), torch.float64)
    x0 = torch.zeros(pr.n, dtype=torch.float64, device="cuda")
    i0 = ctx.solve(b, x0)
    h0 = ctx.history()
    ctx.set_kernel_timing(True)
    x1 = torch.zeros_like(x0)
    i1 = ctx.solve(b, x1)
    kt = ctx.kernel_timing()
    # the same results with the event marks in place (the sweep's scatter-add
    # uses atomics, so two solves agree to rounding, not bit for bit)
    assert i0["iterations"] == i1["iterations"] == maxit
    h1 = ctx.history()
    assert h1.shape == h0.shape and np.max(np.abs(h1 - h0)) <= 1e-10
    assert torch.allclose(x0, x1, rtol=1e-8, atol=1e-12)
    its = i1["iterations"]
    n = pr.n
    js = list(range(m)) + list(range(maxit - m))          # iterations j of each cycle
    assert kt["sweep"][1] == its and kt["spmv"][1] == its
    second = sum(8.0 * (j + 3) * n for j in js)            # bytes of the second passes, if all taken
    if ortho == "split":
        assert kt["maxpy"][1] > 0
    if kt["maxpy"][1] == 0:
        # fused Arnoldi step (cooperative launch): projection, update(s) and
        # normalisation in one kernel per step; on pairs it reads the pair
        # copy of the basis and keeps w as a pair between the passes
        assert kt["mdot"][1] == its and kt["vec"][1] == 0
        if ortho == "fp64":
            base = sum(8.0 * ((j + 2) + (j + 3) + 3) * n for j in js)
        else:
            # pairs: the last update fused with the normalisation
            base = sum(8.0 * ((j + 3) + (j + 4)) * n for j in js)
        assert base * (1 - 1e-12) <= kt["mdot"][2] <= (base + second) * (1 + 1e-12)
        classes = ("sweep", "spmv", "mdot")
    else:
        assert kt["mdot"][1] == its and kt["maxpy"][1] == 2 * its and kt["vec"][1] == its
        assert kt["mdot"][2] == pytest.approx(sum(8.0 * (j + 2) * n for j in js), rel=1e-12)
        # the second update moves bytes only on steps that reorthogonalise
        assert second * (1 - 1e-12) <= kt["maxpy"][2] <= 2 * second * (1 + 1e-12)
        classes = ("sweep", "spmv", "mdot", "maxpy", "vec")
    for name in classes:
        ms, cnt, by, fl = kt[name]
        assert ms > 0.0 and by > 0.0 and fl > 0.0, name
    # FP64 flops: SpMV 2 nnz per launch; the Gram-Schmidt step between its
    # single-pass and its two-pass count
    assert kt["spmv"][3] == pytest.approx(its * 2.0 * pr.nnz, rel=1e-12)
    if kt["maxpy"][1] == 0 and ortho == "fp64":
        lo = sum(4.0 * n * (j + 2) + 3.0 * n for j in js)
        hi = lo + sum(4.0 * n * (j + 1) for j in js)
        assert lo * (1 - 1e-12) <= kt["mdot"][3] <= hi * (1 + 1e-12)
    elif kt["maxpy"][1] == 0:
        # the fused step runs its dots and updates on FP32 pairs: 4 FP64
        # flops per entry (norm and split of w, FP64 copy of v)
        assert kt["mdot"][3] == pytest.approx(its * 4.0 * n, rel=1e-12)
    assert kt["spmv"][2] == pytest.approx(its * (12.0 * pr.nnz + 4.0 * (n + 1) + 16.0 * n), rel=1e-12)
    # disabling resets nothing but stops the marks; re-enabling resets
    ctx.set_kernel_timing(False)
    ctx.solve(b, x1)
    assert ctx.kernel_timing()["mdot"][1] == its
    ctx.set_kernel_timing(True)
    assert all(v[1] == 0 for v in ctx.kernel_timing().values())
    ctx.destroy()


def test_cg_timing_counts(lib):
    pr = P.poisson2d_q2(12)
    ctx = setup_ctx(lib, pr, tol=0.0, weighting="sym", krylov="cg")
    b = dev(pr.rhs(0), torch.float64)
    x = torch.zeros(pr.n, dtype=torch.float64, device="cuda")
    ctx.set_kernel_timing(True)
    info = ctx.solve(b, x)
    kt = ctx.kernel_timing()
    its = info["iterations"]
    assert info["converged"] and its > 8
    # every iteration runs its SpMV and x/r update; the convergence test in the
    # last one stops the sweep, dot and p update of that iteration early, but
    # they are still launched inside the last block and counted
    assert kt["spmv"][1] == its and kt["sweep"][1] == its and kt["vec"][1] == 3 * its
    assert kt["mdot"][1] == 0 and kt["maxpy"][1] == 0
    ctx.destroy()


def test_kernel_timing_rejects_bad_args(lib):
    pr = P.poisson2d_q2(4)
    ctx = setup_ctx(lib, pr, tol=0.0, weighting="sym", krylov="cg")
    L = lib.load()
    assert L.psr_get_kernel_timing(ctx.h, None, None, None, None, 0) == -1
    assert L.psr_get_kernel_timing(ctx.h, None, None, None, None, 6) == -1
    assert L.psr_set_kernel_timing(None, 1) == -1
    ctx.destroy()
