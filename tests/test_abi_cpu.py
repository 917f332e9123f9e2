"""CPU-side checks of the C ABI: the library loads without a GPU and exports every
entry point that include/helm.h declares, and the Python binding names them all."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", h) for h in ("helm.h", "helm_trace.h", "helm_server.h", "helm_blas.h")]
LIB = os.path.join(ROOT, "paper_2301_10762_gb300", "libhelm.so")


def declared_functions():
    src = "\n".join(open(h).read() for h in HEADERS)
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z_0-9]*\s*\*?\s*([A-Za-z_][A-Za-z_0-9]*)\s*\(", src, re.M)
    return sorted(set(n for n in names if n not in ("if", "while", "return")))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("helm_assemble", "helm_factor", "helm_solve", "helm_adjoint_solve", "fwi_misfit_grad",
              "bilevel_hypergrad", "helm_op_destroy", "helm_factor_destroy"):
        assert n in names


@pytest.mark.skipif(not os.path.exists(LIB), reason="libhelm.so not built (run __graft_entry__.build())")
def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(LIB)
    for n in declared_functions():
        assert hasattr(lib, n), n
    lib.helm_status_string.restype = ctypes.c_char_p
    assert lib.helm_status_string(5).startswith(b"HELM_ESINGULAR")


def test_binding_covers_the_header():
    from paper_2301_10762_gb300 import helm as hm
    assert sorted(hm.EXPORTED) == declared_functions()


def test_binding_struct_layouts_match_the_headers(tmp_path):
    """Every ctypes struct of the binding has the size and field offsets that a C compiler
    gives the struct of the same name in include/*.h (a drift would pass garbage across the
    boundary without any error)."""
    import shutil
    import subprocess
    from paper_2301_10762_gb300 import helm as hm
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = [v for v in vars(hm).values()
               if isinstance(v, type) and issubclass(v, ctypes.Structure) and v.__name__.startswith("helm_")]
    assert len(structs) >= 11
    lines = ["#include <stdio.h>", "#include <stddef.h>"] + [f'#include "{h}"' for h in HEADERS]
    lines.append("int main(void) {")
    expect = []
    for s in structs:
        lines.append(f'printf("%zu\\n", sizeof({s.__name__}));')
        expect.append(ctypes.sizeof(s))
        for name, *_ in s._fields_:
            lines.append(f'printf("%zu\\n", offsetof({s.__name__}, {name}));')
            expect.append(getattr(s, name).offset)
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-Wall", "-Werror", str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()]
    assert got == expect


@pytest.mark.skipif(not os.path.exists(LIB), reason="libhelm.so not built (run __graft_entry__.build())")
def test_invalid_arguments_return_einval_with_a_message():
    """Every entry point validates its arguments before any CUDA call: NULL or out-of-range
    arguments give HELM_EINVAL (no abort, no GPU needed) and a helm_last_error message naming
    the call."""
    lib = ctypes.CDLL(LIB)
    lib.helm_last_error.restype = ctypes.c_char_p
    d = ctypes.c_double
    calls = {
        "helm_assemble": lambda: lib.helm_assemble(None, None, None, 0, None, None),
        "helm_factor": lambda: lib.helm_factor(None, 0, None, None),
        "helm_solve": lambda: lib.helm_solve(None, 1, None, None, d(1e-10), 8, None),
        "helm_solve_noalloc": lambda: lib.helm_solve_noalloc(None, 1, None, None, d(1e-10), 8, 0, None),
        "helm_sources": lambda: lib.helm_sources(None, None, None),
        "helm_restrict": lambda: lib.helm_restrict(None, None, 1, None, None),
        "helm_restrict_adjoint": lambda: lib.helm_restrict_adjoint(None, None, 1, None, None),
        "helm_field_grad": lambda: lib.helm_field_grad(None, 1, None, None, None),
        "fwi_misfit_grad": lambda: lib.fwi_misfit_grad(None, None, None, d(0), d(0), d(1e-10), None, None, None,
                                                       None),
        "fwi_hessian_vec": lambda: lib.fwi_hessian_vec(None, None, None, None, None, d(0), d(0), d(1e-10), 0, None),
        "helm_gamma_solve": lambda: lib.helm_gamma_solve(None, d(1e-3), d(1e-6), 1, None, None, None),
        "bilevel_hypergrad": lambda: lib.bilevel_hypergrad(0, None, None, None, None, None, None, None, 0, d(0), d(0),
                                                           d(0), 0, None, None, None, None, None, None, None),
        "helm_zgemm_batched": lambda: lib.helm_zgemm_batched(1, 0, 1, 2, None, ctypes.c_int64(0), 2, None,
                                                             ctypes.c_int64(0), 2, ctypes.c_float(1.0), None, None,
                                                             ctypes.c_int64(0), 1, None),
        "helm_zinv_batched": lambda: lib.helm_zinv_batched(1, 0, None, ctypes.c_int64(0), 0, None, ctypes.c_int64(0),
                                                           0, None),
        "helm_server_create": lambda: lib.helm_server_create(None, None),
        "helm_server_add_model": lambda: lib.helm_server_add_model(None, None, None, None),
        "helm_server_submit": lambda: lib.helm_server_submit(None, None, None),
        "helm_server_wait": lambda: lib.helm_server_wait(None, ctypes.c_int64(0), None),
        "helm_server_stats": lambda: lib.helm_server_stats(None, None),
    }
    calls["helm_adjoint_solve"] = lambda: lib.helm_adjoint_solve(None, 1, None, None, d(1e-10), 8, None)
    for name, call in calls.items():
        assert call() == 1, name                        # HELM_EINVAL
        assert lib.helm_last_error().decode().startswith(name), (name, lib.helm_last_error())


@pytest.mark.skipif(not os.path.exists(LIB), reason="libhelm.so not built (run __graft_entry__.build())")
def test_fault_injection_words_are_parsed(monkeypatch):
    """HELM_FAULT (host-side fault injection) is read at every call: each word selects its bit,
    unknown words set HELM_FAULT_UNKNOWN, an unset or empty variable selects nothing.  A host
    function: no GPU needed."""
    lib = ctypes.CDLL(LIB)
    lib.helm_fault_mask.restype = ctypes.c_uint32
    cases = {"": 0, "alloc": 0x1, "pivot": 0x2, "timeout": 0x4, "nan_rhs": 0x8, "alloc,nan_rhs": 0x9,
             "pivot,timeout,alloc,nan_rhs": 0xF, "bogus": 0x80000000, "timeout,bogus,": 0x80000004,
             "allocx": 0x80000000}
    for value, bits in cases.items():
        monkeypatch.setenv("HELM_FAULT", value)
        assert lib.helm_fault_mask() == bits, value
    monkeypatch.delenv("HELM_FAULT")
    assert lib.helm_fault_mask() == 0


@pytest.mark.skipif(not os.path.exists(LIB), reason="libhelm.so not built (run __graft_entry__.build())")
def test_library_was_built_from_the_current_sources():
    """A build that failed after a source change leaves the previous libhelm.so behind, and the
    ABI checks above would then test stale code.  The build records a digest of the sources it
    compiled; it must match the sources as they are now."""
    from paper_2301_10762_gb300 import build as b
    if not os.path.exists(b.DIGEST):
        pytest.skip("library built without a source digest")
    with open(b.DIGEST) as fh:
        assert fh.read().strip() == b.source_digest(), "libhelm.so was built from other sources: rebuild"
