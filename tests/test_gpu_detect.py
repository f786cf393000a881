"""Patch detection (section 2, after Figure 1) on the GPU against the CPU
oracle: the detected patch maps are equal element by element (integer work),
at small sizes and on the full 128 x 128 Stokes pattern."""
import ctypes as C

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


def detect(lib, rowptr, colidx, q):
    return lib.psr_detect_patches(dev(rowptr, torch.int32), dev(colidx, torch.int32), q).cpu().numpy()


@pytest.mark.parametrize("case", ["poisson", "diff3d", "stokes", "stokes_graded", "poisson_eliminated",
                                  "stokes_full"])
def test_detect_equals_oracle(lib, case):
    if case == "poisson":
        pr, q = P.poisson2d_q2(8, keep_pattern=True), 9
    elif case == "diff3d":
        pr, q = P.diffusion3d_q2(4, seed=1, keep_pattern=True), 27
    elif case == "stokes":
        pr, q = P.stokes2d_q2q1(8, keep_pattern=True), 22
    elif case == "stokes_graded":
        pr, q = P.stokes2d_q2q1(13, 1.05, keep_pattern=True), 22
    elif case == "poisson_eliminated":
        pr, q = P.poisson2d_q2(10), 9
    else:
        pr, q = P.stokes2d_q2q1(128, 1.05, keep_pattern=True), 22
    got = detect(lib, pr.rowptr, pr.colidx, q)
    ref = O.detect_patches(pr.rowptr, pr.colidx, pr.n, q)
    assert got.shape == ref.shape and np.array_equal(got, ref), case
    if case != "poisson_eliminated":
        assert got.shape[0] == pr.n_patches


def test_detected_map_drives_setup_and_solve(lib):
    """The detected map is a uniform-size patch map: Alg. 1 and PCG run on it."""
    pr = P.poisson2d_q2(12, keep_pattern=True)
    d = lib.psr_detect_patches(dev(pr.rowptr, torch.int32), dev(pr.colidx, torch.int32), 9)
    rp, ci, va = dev(pr.rowptr, torch.int32), dev(pr.colidx, torch.int32), dev(pr.vals, torch.float64)
    ctx = lib.psr_setup(rp, ci, va, d.reshape(-1).contiguous(), uniform_size=9,
                        opts=lib.make_opts(tol=1e-2, weighting="sym", krylov="cg", rtol=1e-8))
    x = torch.zeros(pr.n, dtype=torch.float64, device="cuda")
    info = ctx.solve(dev(pr.rhs(0), torch.float64), x)
    assert info["converged"]
    ctx.destroy()


def test_detect_edge_cases_and_errors(lib):
    rows = [[0, 1], [1, 3, 5], [3, 4, 6], [0, 1, 2, 3], [1, 3, 5], [5], [1, 3, 5]]
    rowptr = np.cumsum([0] + [len(r) for r in rows]).astype(np.int32)
    colidx = np.array([c for r in rows for c in r], dtype=np.int32)
    assert detect(lib, rowptr, colidx, 3).tolist() == [[1, 3, 5], [3, 4, 6]]
    assert detect(lib, rowptr, colidx, 7).shape == (0, 7)
    # too small an output: INVALID_ARG, with the count reported
    L = lib.binding
    rp, ci = dev(rowptr, torch.int32), dev(colidx, torch.int32)
    A = L.psr_csr(len(rows), len(colidx), rp.data_ptr(), ci.data_ptr(), 0)
    out = torch.empty(3, dtype=torch.int32, device="cuda")
    cnt = C.c_int32(0)
    rc = lib.load().psr_detect_patches(C.byref(A), 3, C.c_void_p(out.data_ptr()), 1, C.byref(cnt), None)
    assert rc == -1 and cnt.value == 2
    # a row of the requested length with unsorted or out-of-range columns
    for bad in ([[0, 2, 1], [1, 2, 0]], [[0, 1, 9], [0, 1, 2]]):
        rp2 = np.cumsum([0] + [len(r) for r in bad]).astype(np.int32)
        ci2 = np.array([c for r in bad for c in r], dtype=np.int32)
        with pytest.raises(lib.PsrError):
            lib.psr_detect_patches(dev(rp2, torch.int32), dev(ci2, torch.int32), 3)
