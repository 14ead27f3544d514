"""The C ABI library loads and exports every symbol the headers in include/
declare; the host-side argument checks run without a GPU (they return before
any CUDA call)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(bsm_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_1501_07800_gb300 import build
    build.build()
    import paper_1501_07800_gb300 as bsm
    return bsm.load()


def test_header_lists_the_api():
    names = declared_functions()
    for n in ["bsm_build", "bsm_multiply", "bsm_multiply_batched", "bsm_to_blocks", "bsm_info",
              "bsm_destroy", "bsm_status_string", "bsm_level_counts", "bsm_last_stats"]:
        assert n in names


def test_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_names_match_header():
    import paper_1501_07800_gb300 as bsm
    for name in declared_functions():
        assert callable(getattr(bsm, name)), name


def test_status_strings(lib):
    import paper_1501_07800_gb300 as bsm
    for code in bsm.STATUS:
        assert bsm.bsm_status_string(code) not in ("", "unknown status")
    assert bsm.bsm_status_string(12345) == "unknown status"


def test_argument_checks_before_any_device_work(lib):
    out = ctypes.c_void_p(1)
    # unsupported block size
    assert lib.bsm_build(64, 64, 17, 0, None, None, None, 0, None, ctypes.byref(out)) == -3
    assert out.value is None
    # negative sizes / missing buffers / NULL output
    assert lib.bsm_build(-1, 64, 32, 0, None, None, None, 0, None, ctypes.byref(out)) == -1
    assert lib.bsm_build(64, 64, 32, 3, None, None, None, 0, None, ctypes.byref(out)) == -1
    assert lib.bsm_build(64, 64, 32, 0, None, None, None, 0, None, None) == -1
    assert lib.bsm_build(64, 64, 32, 0, None, None, None, 2, None, ctypes.byref(out)) == -1
    # NULL handles
    assert lib.bsm_multiply(None, None, ctypes.byref(out), None, None) == -1
    assert lib.bsm_multiply(None, None, None, None, None) == -1
    assert lib.bsm_multiply_batched(-1, None, None, None, None, None) == -1
    assert lib.bsm_multiply_batched(0, None, None, None, None, None) == 0
    n = ctypes.c_int64(0)
    assert lib.bsm_to_blocks(None, ctypes.byref(n), None, None, None, 0, None) == -1
    assert lib.bsm_info(None, None, None, None, None) == -1
    assert lib.bsm_transpose(None, ctypes.byref(out), None) == -1
    assert lib.bsm_transpose(None, None, None) == -1
    assert lib.bsm_add(None, None, ctypes.byref(out), None) == -1
    assert lib.bsm_add(None, None, None, None) == -1
    assert lib.bsm_sym_square(None, ctypes.byref(out), None, None) == -1
    assert lib.bsm_sym_square(None, None, None, None) == -1
    assert lib.bsm_syrk(None, 0, ctypes.byref(out), None, None) == -1
    assert lib.bsm_sym_multiply(None, None, 0, ctypes.byref(out), None, None) == -1
    assert lib.bsm_sym_to_full(None, ctypes.byref(out), None) == -1
    assert lib.bsm_reblock(None, 32, ctypes.byref(out), None) == -1
    assert lib.bsm_multiply_range(None, None, 0, 1, ctypes.byref(out), None, None) == -1
    b = ctypes.c_int()
    assert lib.bsm_plan_block_size(None, ctypes.byref(b)) == -1
    assert lib.bsm_node_norms2(None, 0, None, None, None, ctypes.byref(n), 0, None) == -1
    assert lib.bsm_truncate(None, ctypes.c_double(1.0), ctypes.byref(out), None, None, None) == -1
    assert lib.bsm_destroy(None) == 0
    assert lib.bsm_memory_in_use(None) == -1
    assert lib.bsm_set_memory_limit(ctypes.c_uint64(0)) == 0
    # peak probes
    f, ms = ctypes.c_double(), ctypes.c_float()
    assert lib.bsm_probe_fp64(99, 1, ctypes.byref(f), ctypes.byref(ms), None) == -1
    assert lib.bsm_probe_fp64(0, 0, ctypes.byref(f), ctypes.byref(ms), None) == -1
    assert lib.bsm_probe_tcgen05(2, 64, 1, 1, 1, ctypes.byref(f), ctypes.byref(ms), None) == -1
    assert lib.bsm_probe_tcgen05(0, 40, 1, 1, 1, ctypes.byref(f), ctypes.byref(ms), None) == -1
    assert lib.bsm_probe_tcgen05(0, 64, 9, 1, 1, ctypes.byref(f), ctypes.byref(ms), None) == -1
    assert lib.bsm_probe_tcgen05(0, 128, 1, 3, 1, ctypes.byref(f), ctypes.byref(ms), None) == -1
    assert lib.bsm_probe_bulk_copy(1 << 20, 100, 4, ctypes.byref(f), ctypes.byref(ms),
                                   None) == -1
    assert lib.bsm_probe_bulk_copy(1 << 30, 65536, 8, ctypes.byref(f), ctypes.byref(ms),
                                   None) == -1


def test_misaligned_device_pointers_rejected_before_any_work(lib):
    """Device payloads are staged with 16-byte vector loads / bulk copies: a
    misaligned caller pointer is refused with INVALID_ARG (never dereferenced)."""
    out = ctypes.c_void_p(1)
    # vals at an address that is 8 (not 16) byte aligned; never touched
    assert lib.bsm_build(64, 64, 32, 1, 256, 512, 4104, 1, None, ctypes.byref(out)) == -1
    assert out.value is None
    assert lib.bsm_build(64, 64, 32, 1, 258, 512, 4096, 1, None, ctypes.byref(out)) == -1
    n = ctypes.c_int64(0)
    assert lib.bsm_block_products_fp64_noalloc(32, 1, 256, 256, 256, 4104, 1, 4096, 1, 4096,
                                               ctypes.byref(n), None) == -1


def test_header_is_plain_c_and_links_from_c(lib, tmp_path):
    """include/bsm.h compiles as strict C99 and a C program links against
    libbsm.so and calls it (calls that need no GPU)."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "use_bsm.c"
    src.write_text(
        '#include "bsm.h"\n#include "bsm_probe.h"\n#include <stdio.h>\n#include <string.h>\n'
        "int main(void) {\n"
        "  bsm_mult_opts o = {BSM_SPLIT_BF16, 7, 0, 32};\n"
        "  bsm_matrix m = NULL;\n"
        "  if (strcmp(bsm_status_string(BSM_OK), \"ok\") != 0) return 3;\n"
        "  if (o.bs != 32 || bsm_destroy(m) != BSM_OK) return 2;\n"
        "  return bsm_multiply(m, m, &m, &o, NULL) == BSM_ERR_INVALID_ARG ? 0 : 1;\n"
        "}\n")
    libdir = os.path.join(ROOT, "paper_1501_07800_gb300")
    inc = os.path.join(ROOT, "include")
    r = subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic",
                        "-fsyntax-only", "-I", inc, str(src)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    exe = tmp_path / "use_bsm"
    r = subprocess.run([gcc, "-std=c99", "-I", inc, str(src), "-L", libdir, "-lbsm",
                        f"-Wl,-rpath,{libdir}", "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    assert subprocess.run([str(exe)]).returncode == 0
