"""Learned assignment on the GPU vs the FP64 oracle: features, MLP loss and
gradients, Adam steps, predictions, and the hinted/seeded Alg. 1."""
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


def pack(params):
    return np.concatenate([p.reshape(-1) for p in params]).astype(np.float32)


def unpack(flat, d, h, m):
    shapes = [(h, d), (h,), (h, h), (h,), (m, h), (m,)]
    out, o = [], 0
    for s in shapes:
        k = int(np.prod(s))
        out.append(flat[o:o + k].reshape(s).astype(np.float64))
        o += k
    return out


def init_params(g, d, h, m):
    return [g.standard_normal((h, d)) / np.sqrt(d), np.zeros(h), g.standard_normal((h, h)) / np.sqrt(h),
            np.zeros(h), g.standard_normal((m, h)) / np.sqrt(h), np.zeros(m)]


def test_features_vs_oracle(lib):
    pr = P.diffusion3d_q2(4, seed=2)
    A = O.extract_patches(pr.rowptr, pr.colidx, pr.vals, pr.n, pr.dofs2d())
    X = torch.empty(pr.n_patches, 27 * 27 + 2, dtype=torch.float32, device="cuda")
    lib.psr_features(dev(A, torch.float64), dev(pr.cell_coef, torch.float64), X)
    Xo = O.patch_features(A, pr.cell_coef)
    np.testing.assert_allclose(X.cpu().numpy(), Xo, rtol=2e-7, atol=2e-7)


def test_loss_and_gradients_vs_oracle(lib):
    g = np.random.default_rng(30)
    d, h, m, B = 40, 32, 7, 300
    params = init_params(g, d, h, m)
    X = g.standard_normal((B, d))
    y = g.integers(0, m, B)
    net = lib.MLP(d, h, m)
    flat = pack(params)
    net.set_params(dev(flat, torch.float32))
    p32 = unpack(flat, d, h, m)                    # the FP32-rounded parameters
    X32 = X.astype(np.float32).astype(np.float64)
    loss, gr = net.loss_grad(dev(X32, torch.float32), dev(y, torch.int32))
    lo, go = O.mlp_loss_grad(p32, X32, y)
    assert abs(loss.item() - lo) <= 1e-5 * abs(lo)
    gg = unpack(gr.cpu().numpy(), d, h, m)
    for a, b_ in zip(gg, go):
        assert np.abs(a - b_).max() <= 1e-4 * max(np.abs(b_).max(), 1e-3)


def test_adam_steps_track_oracle(lib):
    g = np.random.default_rng(31)
    d, h, m, B = 24, 16, 5, 128
    params = init_params(g, d, h, m)
    X = g.standard_normal((B, d)).astype(np.float32).astype(np.float64)
    y = g.integers(0, m, B)
    net = lib.MLP(d, h, m)
    flat = pack(params)
    net.set_params(dev(flat, torch.float32))
    po = unpack(flat, d, h, m)
    mo = [np.zeros_like(p) for p in po]
    vo = [np.zeros_like(p) for p in po]
    Xd, yd = dev(X, torch.float32), dev(y, torch.int32)
    for t in range(1, 6):
        net.train_step(Xd, yd, 1e-2)
        _, go = O.mlp_loss_grad(po, X, y)
        po, mo, vo = O.adam_step(po, go, mo, vo, t, 1e-2)
    pg = unpack(net.get_params().cpu().numpy(), d, h, m)
    for a, b_ in zip(pg, po):
        assert np.abs(a - b_).max() <= 1e-3 * max(np.abs(b_).max(), 1e-2)


def test_training_reduces_loss_and_predicts(lib):
    """Separable synthetic classes: loss falls and predictions match labels."""
    g = np.random.default_rng(32)
    d, h, m, B = 16, 64, 4, 512
    centers = g.standard_normal((m, d)) * 3
    y = g.integers(0, m, B)
    X = centers[y] + 0.3 * g.standard_normal((B, d))
    net = lib.MLP(d, h, m)
    net.set_params(dev(pack(init_params(g, d, h, m)), torch.float32))
    Xd, yd = dev(X, torch.float32), dev(y, torch.int32)
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    net.train_step(Xd, yd, 1e-2, loss)
    l0 = loss.item()
    for _ in range(200):
        net.train_step(Xd, yd, 1e-2, loss)
    assert loss.item() < 0.1 * l0
    cls, lg = net.predict(Xd, logits=True)
    lgn = lg.cpu().numpy()
    assert np.array_equal(cls.cpu().numpy(), np.argmax(lgn, axis=1))
    assert np.mean(cls.cpu().numpy() == y) > 0.98


def _c4_small():
    pr = P.diffusion3d_q2(5, seed=7)
    A = O.extract_patches(pr.rowptr, pr.colidx, pr.vals, pr.n, pr.dofs2d())
    return pr, A


def _seeded(lib, pr, tol, seed_A, hints=None):
    rp, ci, va = dev(pr.rowptr, torch.int32), dev(pr.colidx, torch.int32), dev(pr.vals, torch.float64)
    ctx = lib.psr_setup_seeded(rp, ci, va, dev(pr.patch_dofs, torch.int32), pr.uniform_size,
                               dev(seed_A, torch.float64), None if hints is None else dev(hints, torch.int32),
                               opts=lib.make_opts(tol=tol, weighting="sym", krylov="cg"))
    return ctx


def test_seeded_alg1_bit_exact(lib):
    pr, A = _c4_small()
    tol = 0.3
    base = O.alg1(A, tol)
    half = base["reps"][: len(base["reps"]) // 2]
    seed_A = A[half]
    ref = O.alg1_seeded(A, tol, seed_A)
    ctx = _seeded(lib, pr, tol, seed_A)
    phi, reps, m = ctx.assignment()
    assert m == len(ref["reps"])
    assert np.array_equal(phi.cpu().numpy(), ref["phi"])
    assert np.array_equal(reps.cpu().numpy(), ref["reps"])
    assert ctx.stats()["criterion_evals"] == ref["evals"]


def test_hinted_alg1_bit_exact_and_gain(lib):
    """Hints = predictions of an MLP trained on the criterion's own labels
    for the first half of the patches; the oracle gets the same hints."""
    pr, A = _c4_small()
    tol = 0.3
    first = pr.n_patches // 2
    base = O.alg1(A[:first], tol)                         # database + labels from the first half
    seed_A = A[base["reps"]]
    d = 27 * 27 + 2
    X = torch.empty(pr.n_patches, d, dtype=torch.float32, device="cuda")
    lib.psr_features(dev(A, torch.float64), dev(pr.cell_coef, torch.float64), X)
    net = lib.MLP(d, 64, len(base["reps"]))
    g = np.random.default_rng(33)
    net.set_params(dev(pack(init_params(g, d, 64, len(base["reps"]))), torch.float32))
    yd = dev(base["phi"], torch.int32)
    for _ in range(300):
        net.train_step(X[:first].contiguous(), yd, 3e-3)
    hints = net.predict(X).cpu().numpy()
    ref = O.alg1_seeded(A, tol, seed_A, pred=hints)
    plain = O.alg1_seeded(A, tol, seed_A)
    ctx = _seeded(lib, pr, tol, seed_A, hints)
    phi, reps, m = ctx.assignment()
    st = ctx.stats()
    assert np.array_equal(phi.cpu().numpy(), ref["phi"])
    assert st["criterion_evals"] == ref["evals"] and st["mlp_hits"] == ref["hits"]
    assert ref["evals"] < plain["evals"]                  # the learned hints save evaluations
    # every assignment satisfies the criterion
    Bi = ref["Binv"][ref["phi"]]
    dbA = np.concatenate([seed_A, A[[r for r in ref["reps"] if r >= 0]]])
    dvals = O.criterion(A, dbA[ref["phi"]], Bi)
    assert np.all(dvals < tol)


def test_learned_setup_through_the_abi(lib):
    """psr_mlp_train + psr_setup_learned: a context built with closest-match
    labels trains its network on the GPU on the first half of its patches; a
    setup seeded with that context's database and hinted by its network
    (opts.use_mlp = 1) equals the oracle's hinted Alg. 1 given the same
    predictions, and needs fewer criterion evaluations than the same setup
    with use_mlp = 0 (which equals the unhinted oracle)."""
    pr, A = _c4_small()
    tol = 0.3
    p = pr.uniform_size
    rp, ci, va = dev(pr.rowptr, torch.int32), dev(pr.colidx, torch.int32), dev(pr.vals, torch.float64)
    dofs = dev(pr.patch_dofs, torch.int32)
    train = lib.psr_setup(rp, ci, va, dofs, uniform_size=p,
                          opts=lib.make_opts(tol=tol, weighting="sym", krylov="cg", match="closest"))
    closest = O.alg1_closest_match(A, tol)
    assert closest["near_ties"] == []
    phi_t, reps_t, m0 = train.assignment()
    assert np.array_equal(phi_t.cpu().numpy(), closest["phi"])
    info = train.mlp_train(hidden=64, epochs=300, lr=3e-3, train_fraction=0.5, seed=5)
    assert info["n_train"] == (pr.n_patches + 1) // 2 and info["classes"] == m0
    assert info["train_accuracy"] > 2.0 / m0                 # better than chance
    # the predictions the library uses: its network on its features (no coefficient)
    X = torch.empty(pr.n_patches, p * p + 2, dtype=torch.float32, device="cuda")
    lib.psr_features(dev(A, torch.float64), None, X)
    pred = train.mlp().predict(X).cpu().numpy()
    seed_A = train.export_database().cpu().numpy()
    assert np.array_equal(seed_A, A[closest["reps"]])
    out = {}
    for use in (False, True):
        ctx = lib.psr_setup_learned(rp, ci, va, dofs, p, train,
                                    opts=lib.make_opts(tol=tol, weighting="sym", krylov="cg", use_mlp=use))
        ref = O.alg1_seeded(A, tol, seed_A, pred=pred if use else None)
        phi, reps, m = ctx.assignment()
        st = ctx.stats()
        assert np.array_equal(phi.cpu().numpy(), ref["phi"]), use
        assert np.array_equal(reps.cpu().numpy(), ref["reps"]), use
        assert st["criterion_evals"] == ref["evals"] and st["mlp_hits"] == ref["hits"], use
        out[use] = st["criterion_evals"]
        ctx.destroy()
    assert out[True] < out[False]
    train.destroy()


def test_learned_setup_rejects_untrained_context(lib):
    pr, A = _c4_small()
    rp, ci, va = dev(pr.rowptr, torch.int32), dev(pr.colidx, torch.int32), dev(pr.vals, torch.float64)
    dofs = dev(pr.patch_dofs, torch.int32)
    ctx = lib.psr_setup(rp, ci, va, dofs, uniform_size=pr.uniform_size,
                        opts=lib.make_opts(tol=0.3, weighting="sym", krylov="cg"))
    with pytest.raises(lib.PsrError) as e:
        lib.psr_setup_learned(rp, ci, va, dofs, pr.uniform_size, ctx,
                              opts=lib.make_opts(tol=0.3, weighting="sym", krylov="cg", use_mlp=True))
    assert "PSR_ERR_INVALID_ARG" in str(e.value)
    ctx.destroy()
