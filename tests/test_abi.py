"""CPU checks of the C-ABI library: it loads, exports every function that
include/bnedge.h declares, and its host-only entry points behave.  No compute
call is made (there is no GPU here)."""
import ctypes
import os
import re

import pytest

from oracle import oracle as orc
from paper_1408_1664_gb300 import binding as B
from paper_1408_1664_gb300 import build as Bld

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(bn_[a-z0-9_]+)\s*\(", txt))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    Bld.build()
    return B.load()


def test_library_exports_every_declared_function(lib):
    names = declared_functions()
    assert "bn_edge_posteriors" in names and "bn_submit" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert set(B.EXPORTS) <= set(names)


def test_test_hooks_only_in_the_testing_build(lib):
    """bn_debug_stage / bn_debug_counts sit in the header's BN_TESTING
    section; the release library does not export them, the testing one does."""
    txt = open(os.path.join(ROOT, "include", "bnedge.h")).read()
    guarded = txt[txt.index("#ifdef BN_TESTING"):txt.index("#endif /* BN_TESTING */")]
    for name in B.TEST_EXPORTS:
        assert name + "(" in guarded
        assert name + "(" not in txt.replace(guarded, "")
    release = ctypes.CDLL(Bld.LIB)
    testing = ctypes.CDLL(Bld.LIB_TESTING)
    for name in B.TEST_EXPORTS:
        assert not hasattr(release, name) and hasattr(testing, name)
    for name in B.EXPORTS:
        assert hasattr(release, name) and hasattr(testing, name)


def test_num_families_matches_oracle(lib):
    for n in range(1, 32):
        for d in range(0, 6):
            assert B.bn_num_families(n, d) == orc.num_families(n, d)
    assert B.bn_num_families(0, 1) == 0 and B.bn_num_families(5, -1) == 0


def test_strerror_names_codes(lib):
    assert B.bn_strerror(0) == "ok"
    for code in range(-8, 0):
        assert B.bn_strerror(code) not in ("", "unknown error")


def test_null_arguments_are_rejected(lib):
    assert lib.bn_ctx_create(None, None) == B.BN_EINVAL
    assert lib.bn_ctx_destroy(None) == B.BN_EINVAL
    assert lib.bn_edge_posteriors(None, None, None, None) == B.BN_EINVAL
    assert lib.bn_job_stats(None, 0, None) == B.BN_EINVAL
    assert lib.bn_feature_posterior(None, None, None, None, None) == B.BN_EINVAL


def test_structure_layouts_match_header(lib):
    # 4 int32 + 2 pointers + double + pointer + 2 int32 + 2 pointers on LP64
    assert ctypes.sizeof(B.bn_job_desc) == 16 + 16 + 8 + 8 + 8 + 16
    assert ctypes.sizeof(B.bn_ctx_opts) == 4 + 4 + 8 + 4 + 4
    assert ctypes.sizeof(B.bn_stats) == 10 * 8 + 8 + 8


def test_structure_sizes_match_a_c_compiler(tmp_path):
    """The ctypes mirrors have the sizes and field offsets the C compiler
    gives the header's structures."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "sz.c"
    src.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "bnedge.h"\n'
        "int main(void) { printf(\"%zu %zu %zu %zu %zu %zu %zu\\n\", sizeof(bn_job_desc), "
        "sizeof(bn_ctx_opts), sizeof(bn_stats), offsetof(bn_stats, kernels), "
        "offsetof(bn_stats, ms_upzeta_sums), offsetof(bn_job_desc, log_q), "
        "offsetof(bn_job_desc, log_w)); return 0; }\n")
    exe = tmp_path / "sz"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True,
                                          check=True).stdout.split()]
    assert got == [ctypes.sizeof(B.bn_job_desc), ctypes.sizeof(B.bn_ctx_opts),
                   ctypes.sizeof(B.bn_stats), B.bn_stats.kernels.offset,
                   B.bn_stats.ms_upzeta_sums.offset, B.bn_job_desc.log_q.offset,
                   B.bn_job_desc.log_w.offset]


def test_product_does_not_import_oracle():
    pkg = os.path.join(ROOT, "paper_1408_1664_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in re.sub(r"#.*|//.*", "", txt).lower() or f == "datagen.py", f
