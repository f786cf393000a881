"""ctypes binding of libpsr.so (include/psr.h).

Argument marshalling only: tensors are passed as raw device pointers plus
sizes, the current CUDA stream as a void*.  Every step of the method runs in
the library's CUDA kernels; there is no Python or CPU fallback and every call
raises when the library is missing or returns an error.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libpsr.so")

PSR_OK = 0
ERRORS = {
    -1: "PSR_ERR_INVALID_ARG", -2: "PSR_ERR_UNSORTED_CSR", -3: "PSR_ERR_SINGULAR_PATCH",
    -4: "PSR_ERR_NOT_CONVERGED", -5: "PSR_ERR_CUDA", -6: "PSR_ERR_OOM", -7: "PSR_ERR_TIMEOUT",
    -8: "PSR_ERR_UNCOVERED_DOF",
}
PREC = {"fp64": 0, "fp32": 1, "bf16": 2}
WEIGHT = {"left": 0, "sym": 1}
KRYLOV = {"cg": 0, "fgmres": 1}
SWEEP = {"auto": 0, "grouped": 1, "pergroup": 2, "tensor": 3}
ORTHO = {"auto": 0, "fp64": 1, "split": 2}
CRITERION = {"spectral": 0, "l1": 1, "varmin": 2}
FP64_ARITH = {"pairs": 0, "native": 1}
MATCH = {"first": 0, "closest": 1}
SEARCH = {"creation": 0, "norm_window": 1}

EXPORTS = ["psr_default_opts", "psr_setup", "psr_apply", "psr_solve", "psr_get_history",
           "psr_get_assignment", "psr_get_stats", "psr_last_error", "psr_destroy", "psr_extract",
           "psr_batched_inverse", "psr_criterion", "psr_spectral_norm", "psr_kernel_launches",
           "psr_setup_seeded", "psr_features", "psr_mlp_create", "psr_mlp_num_params", "psr_mlp_set_params",
           "psr_mlp_get_params", "psr_mlp_loss_grad", "psr_mlp_train_step", "psr_mlp_predict", "psr_mlp_destroy",
           "psr_criterion_noalloc", "psr_set_kernel_timing", "psr_get_kernel_timing", "psr_setup_kmeans",
           "psr_export_database", "psr_set_coarse", "psr_smooth", "psr_release_cached_memory", "psr_memory_in_use",
           "psr_detect_patches", "psr_boundary_classes", "psr_default_train_opts", "psr_mlp_train", "psr_ctx_mlp",
           "psr_setup_learned", "psr_debug_inject"]

KT_CLASSES = ("sweep", "spmv", "mdot", "maxpy", "vec")   # PSR_KT_* in order


class PsrError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class psr_csr(C.Structure):
    _fields_ = [("n", C.c_int32), ("nnz", C.c_int64), ("rowptr", C.c_void_p),
                ("colidx", C.c_void_p), ("vals", C.c_void_p)]


class psr_patches(C.Structure):
    _fields_ = [("n_patches", C.c_int32), ("uniform_size", C.c_int32),
                ("offsets", C.c_void_p), ("dofs", C.c_void_p)]


class psr_opts(C.Structure):
    _fields_ = [("tol", C.c_double), ("store_prec", C.c_int32), ("weighting", C.c_int32),
                ("krylov", C.c_int32), ("restart", C.c_int32), ("rtol", C.c_double),
                ("maxit", C.c_int32), ("use_graph", C.c_int32), ("sweep_kernel", C.c_int32),
                ("autotune", C.c_int32), ("symmetrize", C.c_int32), ("use_mlp", C.c_int32),
                ("ortho", C.c_int32), ("criterion", C.c_int32), ("fp64_arith", C.c_int32),
                ("match", C.c_int32), ("seed", C.c_uint64), ("prec_check", C.c_double),
                ("search", C.c_int32)]


class psr_train_opts(C.Structure):
    _fields_ = [("hidden", C.c_int32), ("epochs", C.c_int32), ("lr", C.c_float), ("train_fraction", C.c_float),
                ("seed", C.c_uint64)]


class psr_train_info(C.Structure):
    _fields_ = [("n_train", C.c_int32), ("classes", C.c_int32), ("final_loss", C.c_float),
                ("train_accuracy", C.c_float), ("seconds", C.c_double)]


class psr_csr_rect(C.Structure):
    _fields_ = [("n_rows", C.c_int32), ("n_cols", C.c_int32), ("nnz", C.c_int64), ("rowptr", C.c_void_p),
                ("colidx", C.c_void_p), ("vals", C.c_void_p)]


class psr_solve_info(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("converged", C.c_int32), ("relres", C.c_double),
                ("seconds", C.c_double)]


class psr_stats(C.Structure):
    _fields_ = [("n", C.c_int32), ("n_patches", C.c_int32), ("m_p", C.c_int32), ("n_groups", C.c_int32),
                ("criterion_evals", C.c_int64), ("criterion_exact", C.c_int64), ("mlp_hits", C.c_int64),
                ("factor_bytes", C.c_int64), ("index_bytes", C.c_int64),
                ("t_extract", C.c_double), ("t_rounds", C.c_double), ("t_invert", C.c_double),
                ("t_convert", C.c_double), ("t_autotune", C.c_double),
                ("first_singular", C.c_int32), ("rounds", C.c_int32), ("tc_groups", C.c_int32),
                ("prec_fallback", C.c_int32), ("criterion_screened", C.c_int64),
                ("criterion_decided", C.c_int64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib = None


def load(path: str = LIB_PATH):
    """Load libpsr.so; raises when it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libpsr.so not built ({path}); run __graft_entry__.build()")
    lib = C.CDLL(path)
    vp, i32, i64, d = C.c_void_p, C.c_int32, C.c_int64, C.c_double
    lib.psr_default_opts.argtypes = [C.POINTER(psr_opts)]
    lib.psr_default_opts.restype = None
    lib.psr_setup.argtypes = [C.POINTER(psr_csr), C.POINTER(psr_patches), C.POINTER(psr_opts), vp, C.POINTER(vp)]
    lib.psr_apply.argtypes = [vp, vp, vp, vp]
    lib.psr_solve.argtypes = [vp, vp, vp, vp, C.POINTER(psr_solve_info)]
    lib.psr_get_history.argtypes = [vp, vp, i32, C.POINTER(i32)]
    lib.psr_get_assignment.argtypes = [vp, vp, vp, C.POINTER(i32)]
    lib.psr_get_stats.argtypes = [vp, C.POINTER(psr_stats)]
    lib.psr_export_database.argtypes = [vp, vp, vp]
    lib.psr_set_coarse.argtypes = [vp, C.POINTER(psr_csr_rect), vp]
    lib.psr_smooth.argtypes = [vp, vp, vp, d, i32, vp]
    lib.psr_last_error.argtypes = [vp]
    lib.psr_last_error.restype = C.c_char_p
    lib.psr_destroy.argtypes = [vp]
    lib.psr_destroy.restype = None
    lib.psr_extract.argtypes = [C.POINTER(psr_csr), C.POINTER(psr_patches), vp, vp, vp, vp]
    lib.psr_batched_inverse.argtypes = [vp, i32, i32, vp, vp, vp]
    lib.psr_criterion.argtypes = [vp, i32, i32, vp, vp, d, vp, vp, vp]
    lib.psr_spectral_norm.argtypes = [vp, i32, i32, vp, vp]
    lib.psr_criterion_noalloc.argtypes = [vp, i32, i32, vp, vp, d, vp, vp, vp]
    lib.psr_kernel_launches.argtypes = []
    lib.psr_release_cached_memory.argtypes = []
    lib.psr_memory_in_use.argtypes = [vp, vp]
    lib.psr_detect_patches.argtypes = [C.POINTER(psr_csr), i32, vp, i32, C.POINTER(i32), vp]
    lib.psr_set_kernel_timing.argtypes = [vp, i32]
    lib.psr_get_kernel_timing.argtypes = [vp, vp, vp, vp, vp, i32]
    lib.psr_setup_seeded.argtypes = [C.POINTER(psr_csr), C.POINTER(psr_patches), C.POINTER(psr_opts), vp, i32, vp,
                                     vp, C.POINTER(vp)]
    lib.psr_features.argtypes = [vp, i32, i32, vp, vp, vp]
    lib.psr_setup_kmeans.argtypes = [C.POINTER(psr_csr), C.POINTER(psr_patches), C.POINTER(psr_opts), i32, vp, i32,
                                     vp, vp, C.POINTER(vp)]
    lib.psr_boundary_classes.argtypes = [C.POINTER(psr_csr), C.POINTER(psr_patches), vp, C.POINTER(i32), vp]
    lib.psr_mlp_create.argtypes = [i32, i32, i32, C.POINTER(vp)]
    lib.psr_mlp_num_params.argtypes = [vp]
    lib.psr_mlp_set_params.argtypes = [vp, vp, vp]
    lib.psr_mlp_get_params.argtypes = [vp, vp, vp]
    lib.psr_mlp_loss_grad.argtypes = [vp, vp, vp, i32, vp, vp, vp]
    lib.psr_mlp_train_step.argtypes = [vp, vp, vp, i32, C.c_float, vp, vp]
    lib.psr_mlp_predict.argtypes = [vp, vp, i32, vp, vp, vp]
    lib.psr_mlp_destroy.argtypes = [vp]
    lib.psr_default_train_opts.argtypes = [C.POINTER(psr_train_opts)]
    lib.psr_default_train_opts.restype = None
    lib.psr_mlp_train.argtypes = [vp, vp, C.POINTER(psr_train_opts), vp, C.POINTER(psr_train_info)]
    lib.psr_debug_inject.argtypes = [i32, i64]
    lib.psr_ctx_mlp.argtypes = [vp]
    lib.psr_ctx_mlp.restype = vp
    lib.psr_setup_learned.argtypes = [C.POINTER(psr_csr), C.POINTER(psr_patches), C.POINTER(psr_opts), vp, vp, vp,
                                      C.POINTER(vp)]
    void_ret = ("psr_default_opts", "psr_last_error", "psr_destroy", "psr_kernel_launches", "psr_mlp_num_params",
                "psr_mlp_destroy", "psr_default_train_opts", "psr_ctx_mlp")
    for name in EXPORTS:
        if name not in void_ret:
            getattr(lib, name).restype = C.c_int
    lib.psr_kernel_launches.restype = C.c_int64
    lib.psr_mlp_num_params.restype = C.c_int64
    lib.psr_mlp_destroy.restype = None
    _lib = lib
    return lib


def _check(rc: int, ctx=None):
    if rc != PSR_OK:
        msg = load().psr_last_error(ctx).decode(errors="replace")
        raise PsrError(rc, msg)


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _need(t, dtype, name):
    import torch
    if not (t.is_cuda and t.is_contiguous() and t.dtype == dtype):
        raise ValueError(f"{name} must be a contiguous CUDA tensor of {dtype}")


def make_opts(tol=0.0, store_prec="fp64", weighting="sym", krylov="cg", restart=30, rtol=1e-8,
              maxit=10000, use_graph=True, sweep_kernel="auto", autotune=True, symmetrize=True,
              use_mlp=False, ortho="auto", criterion="spectral", fp64_arith="pairs", match="first",
              seed=0, prec_check=0.5, search="creation") -> psr_opts:
    o = psr_opts()
    load().psr_default_opts(C.byref(o))
    o.tol = tol
    o.store_prec = PREC[store_prec]
    o.weighting = WEIGHT[weighting]
    o.krylov = KRYLOV[krylov]
    o.restart = restart
    o.rtol = rtol
    o.maxit = maxit
    o.use_graph = int(use_graph)
    o.sweep_kernel = SWEEP[sweep_kernel]
    o.autotune = int(autotune)
    o.symmetrize = int(symmetrize)
    o.use_mlp = int(use_mlp)
    o.ortho = ORTHO[ortho]
    o.criterion = CRITERION[criterion]
    o.fp64_arith = FP64_ARITH[fp64_arith]
    o.match = MATCH[match]
    o.seed = int(seed)
    o.prec_check = float(prec_check)
    o.search = SEARCH[search]
    return o


def _csr(rowptr, colidx, vals):
    import torch
    _need(rowptr, torch.int32, "rowptr")
    _need(colidx, torch.int32, "colidx")
    _need(vals, torch.float64, "vals")
    return psr_csr(rowptr.numel() - 1, colidx.numel(), rowptr.data_ptr(), colidx.data_ptr(), vals.data_ptr())


def _patches(dofs, offsets=None, uniform_size=0):
    import torch
    _need(dofs, torch.int32, "dofs")
    if offsets is not None:
        _need(offsets, torch.int32, "offsets")
        return psr_patches(offsets.numel() - 1, 0, offsets.data_ptr(), dofs.data_ptr())
    if uniform_size <= 0:
        raise ValueError("give offsets or uniform_size")
    return psr_patches(dofs.numel() // uniform_size, uniform_size, None, dofs.data_ptr())


# ------------------------------------------------------------- entry points
def psr_setup(rowptr, colidx, vals, dofs, offsets=None, uniform_size=0, opts: psr_opts | None = None,
              stream=None) -> "Context":
    lib = load()
    A = _csr(rowptr, colidx, vals)
    P = _patches(dofs, offsets, uniform_size)
    o = opts if opts is not None else make_opts()
    h = C.c_void_p()
    rc = lib.psr_setup(C.byref(A), C.byref(P), C.byref(o), _stream(stream), C.byref(h))
    _check(rc, None)
    return Context(h, A.n, P.n_patches, o, P.uniform_size)


class Context:
    """Owns a psr_ctx (library-owned device storage)."""

    def __init__(self, handle, n, n_patches, opts, p=0):
        self.h = handle
        self.n = n
        self.n_patches = n_patches
        self.opts = opts
        self.p = p                     # patch size when uniform, else 0

    def apply(self, r, z, stream=None):
        import torch
        _need(r, torch.float64, "r")
        _need(z, torch.float64, "z")
        _check(load().psr_apply(self.h, _ptr(r), _ptr(z), _stream(stream)), self.h)

    def solve(self, b, x, stream=None, raise_on_nonconvergence=False) -> dict:
        import torch
        _need(b, torch.float64, "b")
        _need(x, torch.float64, "x")
        info = psr_solve_info()
        rc = load().psr_solve(self.h, _ptr(b), _ptr(x), _stream(stream), C.byref(info))
        if rc != PSR_OK and not (rc == -4 and not raise_on_nonconvergence):
            _check(rc, self.h)
        return {"iterations": info.iterations, "converged": bool(info.converged),
                "relres": info.relres, "seconds": info.seconds}

    def history(self) -> np.ndarray:
        n = C.c_int32()
        _check(load().psr_get_history(self.h, None, 0, C.byref(n)), self.h)
        out = np.zeros(n.value)
        _check(load().psr_get_history(self.h, out.ctypes.data_as(C.c_void_p), n.value, C.byref(n)), self.h)
        return out

    def assignment(self):
        import torch
        m = C.c_int32()
        _check(load().psr_get_assignment(self.h, None, None, C.byref(m)), self.h)
        phi = torch.empty(self.n_patches, dtype=torch.int32, device="cuda")
        reps = torch.empty(max(m.value, 1), dtype=torch.int32, device="cuda")
        _check(load().psr_get_assignment(self.h, _ptr(phi), _ptr(reps), C.byref(m)), self.h)
        return phi, reps[: m.value], m.value

    def smooth(self, b, x, omega=1.0, sweeps=1, stream=None):
        """psr_smooth: sweeps of x <- x + omega M^-1 (b - A x), x in place."""
        import torch
        _need(b, torch.float64, "b")
        _need(x, torch.float64, "x")
        _check(load().psr_smooth(self.h, _ptr(b), _ptr(x), float(omega), int(sweeps), _stream(stream)), self.h)

    def set_coarse(self, rowptr, colidx, vals, n0, stream=None):
        """psr_set_coarse: the two-level term P0 A0^-1 P0^T of Eq. (2) with
        P0 an n x n0 CSR (device int32 rowptr / colidx, float64 vals)."""
        import torch
        _need(rowptr, torch.int32, "rowptr")
        _need(colidx, torch.int32, "colidx")
        _need(vals, torch.float64, "vals")
        P0 = psr_csr_rect(self.n, int(n0), colidx.numel(), _ptr(rowptr), _ptr(colidx), _ptr(vals))
        _check(load().psr_set_coarse(self.h, C.byref(P0), _stream(stream)), self.h)

    def export_database(self, stream=None):
        """psr_export_database: the entries' patch matrices (m_p x p x p, FP64)
        of a one-size setup, for psr_setup_seeded of a related matrix."""
        import torch
        m = C.c_int32()
        _check(load().psr_get_assignment(self.h, None, None, C.byref(m)), self.h)
        if self.p <= 0:
            raise ValueError("export_database needs patches of one size")
        out = torch.empty((m.value, self.p, self.p), dtype=torch.float64, device="cuda")
        _check(load().psr_export_database(self.h, _ptr(out), _stream(stream)), self.h)
        return out

    def mlp_train(self, features=None, hidden=256, epochs=300, lr=1e-3, train_fraction=1.0, seed=0,
                  stream=None) -> dict:
        """psr_mlp_train: a network owned by the context learns its phi."""
        t = psr_train_opts()
        load().psr_default_train_opts(C.byref(t))
        t.hidden, t.epochs, t.lr, t.train_fraction, t.seed = hidden, epochs, lr, train_fraction, seed
        info = psr_train_info()
        _check(load().psr_mlp_train(self.h, _ptr(features), C.byref(t), _stream(stream), C.byref(info)), self.h)
        return {f: getattr(info, f) for f, _ in info._fields_}

    def mlp(self) -> "MLP":
        """The context's trained network (not owned by the returned view)."""
        h = load().psr_ctx_mlp(self.h)
        if not h:
            raise ValueError("no trained network (psr_mlp_train)")
        return MLP.view_of(C.c_void_p(h), self)

    def stats(self) -> dict:
        st = psr_stats()
        _check(load().psr_get_stats(self.h, C.byref(st)), self.h)
        return st.as_dict()

    def set_kernel_timing(self, enable: bool):
        _check(load().psr_set_kernel_timing(self.h, int(bool(enable))), self.h)

    def kernel_timing(self) -> dict:
        """Per-class totals of psr_get_kernel_timing: {class: (ms, launches, bytes, fp64 flops)}."""
        k = len(KT_CLASSES)
        ms, nl, by, fl = (C.c_double * k)(), (C.c_int64 * k)(), (C.c_double * k)(), (C.c_double * k)()
        _check(load().psr_get_kernel_timing(self.h, C.cast(ms, C.c_void_p), C.cast(nl, C.c_void_p),
                                             C.cast(by, C.c_void_p), C.cast(fl, C.c_void_p), k), self.h)
        return {name: (ms[i], int(nl[i]), by[i], fl[i]) for i, name in enumerate(KT_CLASSES)}

    def destroy(self):
        if self.h:
            load().psr_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def psr_setup_seeded(rowptr, colidx, vals, dofs, uniform_size, seed_A, hints=None, opts: psr_opts | None = None,
                     stream=None) -> "Context":
    """Alg. 1 started from the database seed_A (m0 x p x p, device FP64) with
    optional per-patch hints (device int32, -1 = none)."""
    import torch
    lib = load()
    A = _csr(rowptr, colidx, vals)
    P = _patches(dofs, None, uniform_size)
    _need(seed_A, torch.float64, "seed_A")
    if hints is not None:
        _need(hints, torch.int32, "hints")
    o = opts if opts is not None else make_opts()
    h = C.c_void_p()
    rc = lib.psr_setup_seeded(C.byref(A), C.byref(P), C.byref(o), _ptr(seed_A), seed_A.shape[0], _ptr(hints),
                              _stream(stream), C.byref(h))
    _check(rc, None)
    return Context(h, A.n, P.n_patches, o, P.uniform_size)


def psr_setup_learned(rowptr, colidx, vals, dofs, uniform_size, trained: "Context", opts: psr_opts | None = None,
                      features=None, stream=None) -> "Context":
    """Setup seeded with trained's database and (opts.use_mlp) its network's
    predictions as hints."""
    lib = load()
    A = _csr(rowptr, colidx, vals)
    P = _patches(dofs, None, uniform_size)
    o = opts if opts is not None else make_opts()
    h = C.c_void_p()
    rc = lib.psr_setup_learned(C.byref(A), C.byref(P), C.byref(o), trained.h, _ptr(features), _stream(stream),
                               C.byref(h))
    _check(rc, None)
    return Context(h, A.n, P.n_patches, o, P.uniform_size)


def psr_setup_kmeans(rowptr, colidx, vals, dofs, uniform_size, init, max_iter=100, opts: psr_opts | None = None,
                     stream=None, patch_class=None) -> "Context":
    """Database by Alg. 2, entrywise k-means, seeded with the patches init
    (device int32, m_p distinct patch indices); patch_class (device int32 per
    patch, from psr_boundary_classes) restricts every patch to the means of
    its class."""
    import torch
    lib = load()
    A = _csr(rowptr, colidx, vals)
    P = _patches(dofs, None, uniform_size)
    _need(init, torch.int32, "init")
    if patch_class is not None:
        _need(patch_class, torch.int32, "patch_class")
    o = opts if opts is not None else make_opts()
    h = C.c_void_p()
    rc = lib.psr_setup_kmeans(C.byref(A), C.byref(P), C.byref(o), init.numel(), _ptr(init), max_iter,
                              _ptr(patch_class), _stream(stream), C.byref(h))
    _check(rc, None)
    return Context(h, A.n, P.n_patches, o, P.uniform_size)


def psr_features(A, coef, X, stream=None):
    import torch
    _need(A, torch.float64, "A")
    _need(X, torch.float32, "X")
    n, p, _ = A.shape
    _check(load().psr_features(_ptr(A), n, p, _ptr(coef), _ptr(X), _stream(stream)))


class MLP:
    """Owns a psr_mlp (d -> h -> h -> m ReLU network, FP32 parameters)."""

    def __init__(self, d, h, m):
        self.d, self.h, self.m = d, h, m
        self.ptr = C.c_void_p()
        self.owner = None
        _check(load().psr_mlp_create(d, h, m, C.byref(self.ptr)))
        self.num_params = int(load().psr_mlp_num_params(self.ptr))

    @classmethod
    def view_of(cls, ptr, owner):
        """A non-owning handle on a network that `owner` keeps alive."""
        self = cls.__new__(cls)
        self.ptr = ptr
        self.owner = owner
        self.num_params = int(load().psr_mlp_num_params(ptr))
        self.d = self.h = self.m = None
        return self

    def set_params(self, packed, stream=None):
        import torch
        _need(packed, torch.float32, "packed")
        _check(load().psr_mlp_set_params(self.ptr, _ptr(packed), _stream(stream)))

    def get_params(self, stream=None):
        import torch
        out = torch.empty(self.num_params, dtype=torch.float32, device="cuda")
        _check(load().psr_mlp_get_params(self.ptr, _ptr(out), _stream(stream)))
        return out

    def loss_grad(self, X, y, stream=None):
        import torch
        loss = torch.empty(1, dtype=torch.float32, device="cuda")
        g = torch.empty(self.num_params, dtype=torch.float32, device="cuda")
        _check(load().psr_mlp_loss_grad(self.ptr, _ptr(X), _ptr(y), X.shape[0], _ptr(loss), _ptr(g), _stream(stream)))
        return loss, g

    def train_step(self, X, y, lr, loss=None, stream=None):
        _check(load().psr_mlp_train_step(self.ptr, _ptr(X), _ptr(y), X.shape[0], float(lr), _ptr(loss),
                                         _stream(stream)))

    def predict(self, X, stream=None, logits=False):
        import torch
        cls = torch.empty(X.shape[0], dtype=torch.int32, device="cuda")
        lg = torch.empty(X.shape[0], self.m, dtype=torch.float32, device="cuda") if logits else None
        _check(load().psr_mlp_predict(self.ptr, _ptr(X), X.shape[0], _ptr(cls), _ptr(lg), _stream(stream)))
        return (cls, lg) if logits else cls

    def destroy(self):
        if self.ptr and self.owner is None:
            load().psr_mlp_destroy(self.ptr)
        self.ptr = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def psr_extract(rowptr, colidx, vals, dofs, offsets=None, uniform_size=0, A_out=None, mult_out=None,
                W_out=None, stream=None):
    A = _csr(rowptr, colidx, vals)
    P = _patches(dofs, offsets, uniform_size)
    _check(load().psr_extract(C.byref(A), C.byref(P), _ptr(A_out), _ptr(mult_out), _ptr(W_out), _stream(stream)))


def psr_batched_inverse(A, Ainv, singular=None, stream=None):
    import torch
    _need(A, torch.float64, "A")
    _need(Ainv, torch.float64, "Ainv")
    b, p, _ = A.shape
    _check(load().psr_batched_inverse(_ptr(A), b, p, _ptr(Ainv), _ptr(singular), _stream(stream)))


def psr_criterion(A_i, A_c, Binv_c, tol, accept, dval=None, stream=None):
    import torch
    _need(A_i, torch.float64, "A_i")
    b, p, _ = A_i.shape
    _check(load().psr_criterion(_ptr(A_i), b, p, _ptr(A_c), _ptr(Binv_c), float(tol), _ptr(accept),
                                _ptr(dval), _stream(stream)))


def psr_criterion_noalloc(A_i, A_c, Binv_c, tol, accept, dval=None, stream=None):
    """psr_criterion without any device allocation: for callers whose memory
    manager owns all device memory or who cannot afford an allocation's
    implicit synchronisation.  Its scratch is a fixed array in the library
    (batch <= PSR_CRITERION_NOALLOC_MAX); calls overlapping on the GPU race."""
    import torch
    _need(A_i, torch.float64, "A_i")
    b, p, _ = A_i.shape
    _check(load().psr_criterion_noalloc(_ptr(A_i), b, p, _ptr(A_c), _ptr(Binv_c), float(tol), _ptr(accept),
                                        _ptr(dval), _stream(stream)))


def psr_spectral_norm(E, sigma, stream=None):
    import torch
    _need(E, torch.float64, "E")
    b, p, _ = E.shape
    _check(load().psr_spectral_norm(_ptr(E), b, p, _ptr(sigma), _stream(stream)))


def psr_kernel_launches() -> int:
    return int(load().psr_kernel_launches())


def psr_detect_patches(rowptr, colidx, row_nnz: int, stream=None):
    """Cell-restricted patches of the rows with row_nnz stored entries:
    a device int32 tensor [patches, row_nnz], DOFs ascending, patches in the
    order of their smallest row (psr_detect_patches)."""
    import torch
    _need(rowptr, torch.int32, "rowptr")
    _need(colidx, torch.int32, "colidx")
    A = psr_csr(rowptr.numel() - 1, colidx.numel(), rowptr.data_ptr(), colidx.data_ptr(), 0)
    cnt = C.c_int32(0)
    _check(load().psr_detect_patches(C.byref(A), int(row_nnz), None, 0, C.byref(cnt), _stream(stream)))
    out = torch.empty((max(cnt.value, 0), int(row_nnz)), dtype=torch.int32, device=rowptr.device)
    if cnt.value > 0:
        got = C.c_int32(0)
        _check(load().psr_detect_patches(C.byref(A), int(row_nnz), _ptr(out), cnt.value, C.byref(got),
                                         _stream(stream)))
    return out


def psr_boundary_classes(rowptr, colidx, vals, dofs, offsets=None, uniform_size=0, stream=None):
    """Boundary partition of the patches (psr_boundary_classes): (device int32
    class per patch, number of classes)."""
    import torch
    A = _csr(rowptr, colidx, vals)
    P = _patches(dofs, offsets, uniform_size)
    out = torch.empty(P.n_patches, dtype=torch.int32, device=rowptr.device)
    k = C.c_int32(0)
    _check(load().psr_boundary_classes(C.byref(A), C.byref(P), _ptr(out), C.byref(k), _stream(stream)))
    return out, k.value


def psr_release_cached_memory() -> None:
    """Return the library's cached device and pinned host blocks to the driver."""
    _check(load().psr_release_cached_memory())


def psr_memory_in_use() -> tuple[int, int]:
    """(device bytes, pinned host bytes) the library's allocator has handed
    out and not taken back."""
    d, h = C.c_int64(), C.c_int64()
    _check(load().psr_memory_in_use(C.byref(d), C.byref(h)))
    return d.value, h.value


def exported_symbols(path: str = LIB_PATH) -> list[str]:
    """Names of the psr_* functions the shared library exports (via dlsym)."""
    lib = C.CDLL(path)
    found = []
    for name in EXPORTS:
        try:
            getattr(lib, name)
            found.append(name)
        except AttributeError:
            pass
    return found


INJECT = {"alloc_fail": 1, "barrier_wait": 2, "rounds_split": 3}


def psr_debug_inject(what: str, value: int) -> None:
    """Fault injection for tests (psr_debug_inject): "alloc_fail" makes the
    value-th next device allocation fail (0 disables); "barrier_wait" makes the
    Alg. 1 rounds barriers wait for a block that never arrives, giving up
    after value spins (0 restores); "rounds_split" (1 / 0) sends the Alg. 1
    rounds of patches of at most 32 DOFs down the one-entry-per-round path
    taken without a cooperative launch."""
    _check(load().psr_debug_inject(INJECT[what], int(value)))
