"""psr_criterion_noalloc -- the criterion for callers that cannot let the
library allocate device memory -- gives the same decisions and deciding
values as psr_criterion, on consecutive calls that reuse its fixed scratch.
Collected last on purpose; it must also pass on its own in a fresh process."""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _case(seed, p, batch):
    g = np.random.default_rng(seed)
    Ac = g.standard_normal((p, p)) + p * np.eye(p)
    Binv = np.linalg.inv(Ac)
    Ai = Ac[None] + 10.0 ** g.uniform(-6, 0, (batch, 1, 1)) * g.standard_normal((batch, p, p))
    Ai[0] = Ac
    return Ai, Ac, Binv


def _prep(Ai, Ac, Binv):
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    acc = torch.full((Ai.shape[0],), -7, dtype=torch.int32, device="cuda")
    dv = torch.full((Ai.shape[0],), np.nan, dtype=torch.float64, device="cuda")
    return dev(Ai), dev(Ac), dev(Binv), acc, dv


def _call(fn, bufs, tol):
    A_i, A_c, B_c, acc, dv = bufs
    s = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = fn(C.c_void_p(A_i.data_ptr()), A_i.shape[0], A_i.shape[1], C.c_void_p(A_c.data_ptr()),
            C.c_void_p(B_c.data_ptr()), C.c_double(tol), C.c_void_p(acc.data_ptr()), C.c_void_p(dv.data_ptr()), s)
    torch.cuda.synchronize()
    return rc


def _run(fn, Ai, Ac, Binv, tol):
    bufs = _prep(Ai, Ac, Binv)
    rc = _call(fn, bufs, tol)
    return rc, bufs[3].cpu().numpy(), bufs[4].cpu().numpy()


def test_noalloc_matches_allocating_entry_point():
    import __graft_entry__ as g
    g.build()
    import paper_2306_10025_gb300 as L
    lib = L.load()
    # two calls in a row with different sizes and tolerances: the second must
    # not see the first call's scratch contents
    for seed, p, batch, tol in [(1, 22, 3000, 1e-2), (2, 12, 700, 1e-4)]:
        Ai, Ac, Binv = _case(seed, p, batch)
        rc0, a0, d0 = _run(lib.psr_criterion, Ai, Ac, Binv, tol)
        rc1, a1, d1 = _run(lib.psr_criterion_noalloc, Ai, Ac, Binv, tol)
        assert rc0 == 0 and rc1 == 0
        assert np.array_equal(a1, a0)
        assert np.all(np.abs(d1 - d0) <= 1e-12 * np.abs(d0))
        assert a1[0] == 1 and d1[0] == 0.0


def test_noalloc_undecided_path_and_no_device_memory():
    """A tolerance equal to one candidate's sigma_max leaves that candidate
    within the rounding slack of every certified bound, so it goes through the
    scratch list of undecided candidates to the exact stage.  Decisions and
    values must still equal psr_criterion's, and the call must take no device
    memory: with the library's cache emptied first, any allocation would have
    to come from the driver and show in the free device memory."""
    import __graft_entry__ as g
    g.build()
    import paper_2306_10025_gb300 as L
    lib = L.load()
    p, batch = 16, 2000
    Ai, Ac, Binv = _case(5, p, batch)
    sig = np.linalg.norm(np.matmul(Ac[None] - Ai, Binv[None]), ord=2, axis=(1, 2))
    ks = np.flatnonzero((sig > 1e-3) & (sig < 1e-1))
    assert ks.size > 0
    tol = float(sig[ks[0]])
    rc0, a0, d0 = _run(lib.psr_criterion, Ai, Ac, Binv, tol)
    bufs = _prep(Ai, Ac, Binv)
    assert _call(lib.psr_criterion_noalloc, bufs, tol) == 0      # the first call sets the device up
    bufs[3].fill_(-7)
    bufs[4].fill_(np.nan)
    lib.psr_release_cached_memory()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    rc1 = _call(lib.psr_criterion_noalloc, bufs, tol)
    free1 = torch.cuda.mem_get_info()[0]
    a1, d1 = bufs[3].cpu().numpy(), bufs[4].cpu().numpy()
    assert rc0 == 0 and rc1 == 0
    assert free1 == free0
    assert np.array_equal(a1, a0)
    assert np.all(np.abs(d1 - d0) <= 1e-12 * np.abs(d0))
    # the undecided candidate's value is sigma_max itself, within FP64 rounding
    assert abs(d1[ks[0]] - tol) <= 1e-12 * tol
    # every other candidate agrees with the exact 2-norm away from the tie
    far = np.abs(sig - tol) > 1e-9 * tol
    assert np.array_equal(a1[far], (sig[far] < tol).astype(a1.dtype))


def test_noalloc_rejects_oversized_batch():
    import __graft_entry__ as g
    g.build()
    import paper_2306_10025_gb300 as L
    lib = L.load()
    n = 262144 + 1
    Ai = torch.zeros(n, dtype=torch.float64, device="cuda")
    one = torch.ones(1, dtype=torch.float64, device="cuda")
    acc = torch.zeros(n, dtype=torch.int32, device="cuda")
    rc = lib.psr_criterion_noalloc(C.c_void_p(Ai.data_ptr()), n, 1, C.c_void_p(one.data_ptr()),
                                   C.c_void_p(one.data_ptr()), C.c_double(0.1), C.c_void_p(acc.data_ptr()), None,
                                   None)
    assert rc == -1
    assert b"exceeds its fixed scratch" in lib.psr_last_error(None)
