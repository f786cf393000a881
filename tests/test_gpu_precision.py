"""Per-entry precision check of reduced-precision databases
(psr_opts.prec_check): an entry whose rounded, symmetrised inverse B~ has
||B~ A_c - I||_F above the threshold, or (CG) is not positive definite, is
kept and applied in FP64; the others stay in FP32 / BF16."""
import numpy as np
import pytest

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


def block_problem(p=8, kappa=1e6, copies=3, seed=0):
    """Block-diagonal SPD matrix whose disjoint patches are its blocks: four
    block types (the last one with condition number kappa), each repeated
    `copies` times, so Alg. 1 at a small tolerance keeps four entries."""
    g = np.random.default_rng(seed)
    types = []
    for t in range(4):
        Q, _ = np.linalg.qr(g.standard_normal((p, p)))
        ev = np.linspace(1.0, 2.0, p) if t < 3 else np.geomspace(1.0, 1.0 / kappa, p)
        B = (Q * ev) @ Q.T
        types.append(0.5 * (B + B.T))
    blocks = [types[t] for t in range(4) for _ in range(copies)]
    n = p * len(blocks)
    perm = g.permutation(n)                        # patches are scattered DOF sets
    dofs = perm.reshape(len(blocks), p)
    A = np.zeros((n, n))
    for k, Bk in enumerate(blocks):
        A[np.ix_(dofs[k], dofs[k])] = Bk
    rowptr = np.zeros(n + 1, dtype=np.int64)
    cols, vals = [], []
    for i in range(n):
        nz = np.flatnonzero(A[i])
        cols.extend(nz.tolist())
        vals.extend(A[i, nz].tolist())
        rowptr[i + 1] = len(cols)
    return A, rowptr, np.array(cols), np.array(vals), dofs


def rounded(B, prec):
    f = np.ascontiguousarray(B.astype(np.float32))
    if prec == "fp32":
        return f.astype(np.float64)
    b = f.view(np.uint32).astype(np.uint64)
    b = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


@pytest.mark.parametrize("prec", ["bf16", "fp32"])
def test_ill_conditioned_entry_falls_back_to_fp64(lib, prec):
    p = 8
    A, rowptr, cols, vals, dofs = block_problem(p=p, kappa=1e6)
    n = A.shape[0]
    Ak = np.stack([A[np.ix_(d, d)] for d in dofs])
    ref = O.alg1(Ak, 1e-10)
    assert len(ref["reps"]) == 4
    Binv = ref["Binv"]
    Bs = 0.5 * (Binv + np.transpose(Binv, (0, 2, 1)))
    rho = [np.linalg.norm(rounded(Bs[j], prec) @ Ak[ref["reps"][j]] - np.eye(p)) for j in range(4)]
    expect_hi = [r > 0.5 for r in rho]
    assert expect_hi[3] == (prec == "bf16") and not any(expect_hi[:3])
    W = np.ones(n)
    r = np.random.default_rng(4).standard_normal(n)
    out = {}
    for check in (0.5, 0.0):
        ctx = lib.psr_setup(dev(rowptr.astype(np.int32), torch.int32), dev(cols.astype(np.int32), torch.int32),
                            dev(vals, torch.float64), dev(dofs.reshape(-1).astype(np.int32), torch.int32),
                            uniform_size=p, opts=lib.make_opts(tol=1e-10, store_prec=prec, weighting="sym",
                                                               krylov="cg", prec_check=check))
        st = ctx.stats()
        assert st["m_p"] == 4
        assert st["prec_fallback"] == (sum(expect_hi) if check > 0 else 0)
        z = torch.empty(n, dtype=torch.float64, device="cuda")
        ctx.apply(dev(r, torch.float64), z)
        out[check] = z.cpu().numpy()
        ctx.destroy()
    # reference with the per-entry storage: FP64 for flagged entries, rounded otherwise
    db = [Binv[j] if expect_hi[j] else rounded(Bs[j], prec) for j in range(4)]
    x = r.astype(np.float32).astype(np.float64)      # the rounded path rounds r to FP32
    zr = np.zeros(n)
    for k in range(dofs.shape[0]):
        j = ref["phi"][k]
        xin = r[dofs[k]] if expect_hi[j] else x[dofs[k]]
        zr[dofs[k]] += db[j] @ xin
    z = out[0.5]
    exact = O.apply(r, dofs, Binv, ref["phi"], W, "sym")
    ill = np.concatenate([dofs[k] for k in range(dofs.shape[0]) if ref["phi"][k] == 3])
    ok = np.concatenate([dofs[k] for k in range(dofs.shape[0]) if ref["phi"][k] != 3])
    for part in (ill, ok):            # each part against its own magnitude
        assert np.abs(z[part] - zr[part]).max() <= 2e-6 * np.abs(zr[part]).max()
    if prec == "bf16":
        # with the check the ill-conditioned block is exact; without it, it is not
        assert np.abs(z[ill] - exact[ill]).max() <= 1e-10 * np.abs(exact[ill]).max()
        assert np.abs(out[0.0][ill] - exact[ill]).max() > 1e-3 * np.abs(exact[ill]).max()
