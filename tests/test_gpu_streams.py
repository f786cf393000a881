"""Stream ordering of the C ABI: every call runs on the stream it is given.
Setup, apply and solve on a side stream (created non-blocking by torch, so
the legacy default stream does not order it), with the inputs copied to the
device on that stream right before the setup, match the same calls on the
default stream: phi and the representatives bit for bit, the apply to
FP64 rounding, the solve to its iteration count and the iterate."""
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


def run(lib, pr, opts, r, b):
    """Inputs copied, setup, apply and solve, all on the current stream."""
    t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt).pin_memory().to("cuda", non_blocking=True)
    rp, ci, va = t(pr.rowptr, torch.int32), t(pr.colidx, torch.int32), t(pr.vals, torch.float64)
    dofs = t(pr.patch_dofs, torch.int32)
    ctx = lib.psr_setup(rp, ci, va, dofs, uniform_size=pr.uniform_size, opts=opts)
    rd, bd = t(r, torch.float64), t(b, torch.float64)
    z = torch.empty(pr.n, dtype=torch.float64, device="cuda")
    ctx.apply(rd, z)
    x = torch.zeros(pr.n, dtype=torch.float64, device="cuda")
    info = ctx.solve(bd, x)
    phi, reps, m = ctx.assignment()
    out = (phi.cpu().numpy(), reps[:m].cpu().numpy(), z.cpu().numpy(), x.cpu().numpy(), info)
    ctx.destroy()
    return out


@pytest.mark.parametrize("case", ["stokes2d", "diffusion3d"])
def test_side_stream_matches_default_stream(lib, case):
    if case == "stokes2d":
        pr, opts = P.stokes2d_q2q1(16, 1.05), lib.make_opts(tol=1e-2, weighting="left", krylov="fgmres", maxit=40)
    else:
        pr, opts = P.diffusion3d_q2(6, seed=1), lib.make_opts(tol=0.1, weighting="sym", krylov="cg", maxit=200)
    g = np.random.default_rng(5)
    r, b = g.standard_normal(pr.n), pr.rhs(0)
    ref = run(lib, pr, opts, r, b)
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        got = run(lib, pr, opts, r, b)
    side.synchronize()
    assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])
    assert np.max(np.abs(got[2] - ref[2])) <= 1e-12 * np.max(np.abs(ref[2]))
    assert abs(got[4]["iterations"] - ref[4]["iterations"]) <= 1 and got[4]["converged"] == ref[4]["converged"]
    assert np.max(np.abs(got[3] - ref[3])) <= 1e-6 * np.max(np.abs(ref[3]))
