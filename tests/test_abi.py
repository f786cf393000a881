"""The C ABI library builds, loads and exports every symbol include/psr.h
declares (no compute calls: CPU only)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "psr.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(psr_[a-z_]+)\s*\(", src)))


def test_header_declares_boundary():
    names = declared_symbols()
    for need in ("psr_setup", "psr_apply", "psr_solve", "psr_destroy", "psr_extract",
                 "psr_batched_inverse", "psr_criterion"):
        assert need in names


def test_library_builds_and_exports_everything():
    import shutil
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("no nvcc")
    import __graft_entry__ as g
    g.build()
    import paper_2306_10025_gb300 as L
    exported = L.exported_symbols()
    missing = [n for n in declared_symbols() if n not in exported]
    assert not missing, missing
    # the binding names match the header
    assert set(L.binding.EXPORTS) == set(declared_symbols())


def test_compute_without_gpu_fails_loudly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    import __graft_entry__ as g
    g.build()
    import ctypes as C
    import paper_2306_10025_gb300 as L
    lib = L.load()
    h = C.c_void_p()
    A = L.binding.psr_csr(1, 1, 8, 8, 8)       # non-null pointers: never dereferenced
    P_ = L.binding.psr_patches(1, 1, None, 8)
    o = L.make_opts()
    rc = lib.psr_setup(C.byref(A), C.byref(P_), C.byref(o), None, C.byref(h))
    assert rc == -5 and not h.value
    assert b"CUDA" in lib.psr_last_error(None)
    # the allocator's release has nothing to return and reports the missing device
    assert lib.psr_release_cached_memory() == -5
    # argument checks come before any device work
    cnt = C.c_int32(7)
    assert lib.psr_detect_patches(None, 9, None, 0, C.byref(cnt), None) == -1
    assert lib.psr_detect_patches(C.byref(A), 0, None, 0, C.byref(cnt), None) == -1
    assert lib.psr_detect_patches(C.byref(A), 2000, None, 0, C.byref(cnt), None) == -1
    assert lib.psr_boundary_classes(None, C.byref(P_), None, C.byref(cnt), None) == -1
    big = L.binding.psr_patches(1, 65, None, 8)               # more than 64 DOFs per patch
    assert lib.psr_boundary_classes(C.byref(A), C.byref(big), C.c_void_p(8), C.byref(cnt), None) == -1


def test_debug_inject_arguments_without_device():
    """The allocation-failure injection is host state (accepted without a
    device); unknown kinds and negative values are rejected; the barrier
    injection needs a device."""
    import paper_2306_10025_gb300 as L
    lib = L.load()
    assert lib.psr_debug_inject(1, 3) == 0
    assert lib.psr_debug_inject(1, 0) == 0
    assert lib.psr_debug_inject(3, 1) == 0
    assert lib.psr_debug_inject(3, 0) == 0
    d, h = L.psr_memory_in_use()
    assert d >= 0 and h >= 0
    assert lib.psr_debug_inject(7, 1) == -1
    assert lib.psr_debug_inject(1, -1) == -1
    import torch
    if not torch.cuda.is_available():
        assert lib.psr_debug_inject(2, 100) == -5


def test_struct_layouts_match_header(tmp_path):
    """Every struct the binding marshals has the header's size and field
    offsets (a C program built against include/psr.h prints them)."""
    import ctypes as C
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    from paper_2306_10025_gb300 import binding as B
    structs = {n: c for n, c in vars(B).items()
               if n.startswith("psr_") and isinstance(c, type) and issubclass(c, C.Structure)}
    assert {"psr_opts", "psr_stats", "psr_csr", "psr_patches"} <= set(structs)
    body = ["#include <stdio.h>", "#include <stddef.h>", '#include "psr.h"', "int main(void) {"]
    want = []
    for n, c in sorted(structs.items()):
        body.append(f'printf("%zu\\n", sizeof({n}));')
        want.append(C.sizeof(c))
        for f, _ in c._fields_:
            body.append(f'printf("%zu\\n", offsetof({n}, {f}));')
            want.append(getattr(c, f).offset)
    body += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(body) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()]
    assert got == want


def test_option_constants_match_header(tmp_path):
    """The binding's option names map to the header's #define values (a C
    program built against include/psr.h prints them)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    from paper_2306_10025_gb300 import binding as B
    groups = {"PREC": ("PSR_PREC_", {"fp64": "FP64", "fp32": "FP32", "bf16": "BF16"}),
              "WEIGHT": ("PSR_WEIGHT_", {"left": "LEFT", "sym": "SYM"}),
              "KRYLOV": ("PSR_KRYLOV_", {"cg": "CG", "fgmres": "FGMRES"}),
              "SWEEP": ("PSR_SWEEP_", {"auto": "AUTO", "grouped": "GROUPED", "pergroup": "PERGROUP",
                                       "tensor": "TENSOR"}),
              "ORTHO": ("PSR_ORTHO_", {"auto": "AUTO", "fp64": "FP64", "split": "SPLIT"}),
              "CRITERION": ("PSR_CRITERION_", {"spectral": "SPECTRAL", "l1": "L1", "varmin": "VARMIN"}),
              "FP64_ARITH": ("PSR_FP64_", {"pairs": "PAIRS", "native": "NATIVE"}),
              "MATCH": ("PSR_MATCH_", {"first": "FIRST", "closest": "CLOSEST"}),
              "SEARCH": ("PSR_SEARCH_", {"creation": "CREATION", "norm_window": "NORM_WINDOW"}),
              "INJECT": ("PSR_INJECT_", {"alloc_fail": "ALLOC_FAIL", "barrier_wait": "BARRIER_WAIT",
                                         "rounds_split": "ROUNDS_SPLIT"})}
    body = ["#include <stdio.h>", '#include "psr.h"', "int main(void) {"]
    want = []
    for dict_name, (prefix, names) in groups.items():
        d = getattr(B, dict_name)
        assert set(d) == set(names), dict_name
        for key, suffix in names.items():
            body.append(f'printf("%d\\n", (int){prefix}{suffix});')
            want.append(d[key])
    for code, name in B.ERRORS.items():
        body.append(f'printf("%d\\n", (int){name});')
        want.append(code)
    for k, name in enumerate(B.KT_CLASSES):
        body.append(f'printf("%d\\n", (int)PSR_KT_{name.upper()});')
        want.append(k)
    body.append('printf("%d\\n", (int)PSR_KT_COUNT);')
    want.append(len(B.KT_CLASSES))
    body += ["return 0;", "}"]
    src = tmp_path / "consts.c"
    src.write_text("\n".join(body) + "\n")
    exe = tmp_path / "consts"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()]
    assert got == want


def test_plain_c_program_links_and_calls(tmp_path):
    """A C program built against include/psr.h and linked with libpsr.so
    (no Python, no torch): the defaults of psr_default_opts, argument
    checks before any device work, the error text, and the allocator's
    figures."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    import __graft_entry__ as g
    g.build()
    import paper_2306_10025_gb300 as L
    libdir = os.path.dirname(L.LIB_PATH)
    src = tmp_path / "use.c"
    src.write_text(r"""
#include <stdio.h>
#include <string.h>
#include "psr.h"
int main(void) {
    psr_opts o;
    memset(&o, 0xff, sizeof o);
    psr_default_opts(&o);
    printf("%g %d %d %d %d %g %d %d %d %d\n", o.tol, o.store_prec, o.weighting, o.krylov, o.restart, o.rtol,
           o.maxit, o.match, o.search, o.criterion);
    psr_ctx* ctx = (psr_ctx*)1;
    int rc = psr_setup(NULL, NULL, &o, NULL, &ctx);
    printf("%d %d %d\n", rc, ctx == NULL, psr_last_error(NULL) != NULL && strlen(psr_last_error(NULL)) > 0);
    int64_t d = -1, h = -1;
    rc = psr_memory_in_use(&d, &h);
    printf("%d %lld %lld\n", rc, (long long)d, (long long)h);
    return 0;
}
""")
    exe = tmp_path / "use"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-L", libdir, "-lpsr",
                    "-Wl,-rpath," + libdir, "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    tol, prec, w, kr, restart, rtol, maxit, match, search, crit = out[0].split()
    assert float(tol) == 0.0 and int(prec) == 0 and int(w) == 1 and int(kr) == 0 and int(restart) == 30
    assert float(rtol) == 1e-8 and int(maxit) == 10000 and int(match) == 0 and int(search) == 0 and int(crit) == 0
    assert out[1].split() == ["-1", "1", "1"]
    assert out[2].split() == ["0", "0", "0"]
