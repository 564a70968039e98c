"""The C-ABI library builds, loads and exports every symbol its header declares.

These run without a GPU: no entry point here launches device work.
"""
import ctypes
import os
import re
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tucker_matern.h")


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(tk_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    sys.path.insert(0, ROOT)
    from paper_1711_06874_gb300 import build, binding

    build.build()
    return binding.load()


def test_header_declares_expected_entry_points():
    names = _declared_functions()
    for want in ["tk_create", "tk_tucker", "tk_reconstruct", "tk_rel_error", "tk_eval", "tk_gram",
                 "tk_sym_eig", "tk_ttm_core", "tk_result_free"]:
        assert want in names


def test_every_declared_symbol_is_exported(lib):
    from paper_1711_06874_gb300 import binding

    for name in _declared_functions():
        assert hasattr(lib, name), name
        assert name in binding.SIGNATURES, f"binding lacks {name}"


def test_struct_layouts_match_c(lib, tmp_path):
    """ctypes mirrors of tk_kernel / tk_grid / tk_opts have the C sizes and offsets."""
    from paper_1711_06874_gb300 import binding

    src = tmp_path / "layout.c"
    src.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "tucker_matern.h"\n'
        "int main(void){printf(\"%zu %zu %zu %zu %zu %zu %zu %zu\\n\", sizeof(tk_kernel), sizeof(tk_grid),"
        " sizeof(tk_opts), offsetof(tk_kernel, sigma2), offsetof(tk_grid, kind), offsetof(tk_opts, precision),"
        " offsetof(tk_opts, reflect_fold), offsetof(tk_opts, with_error)); return 0;}\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    want = [ctypes.sizeof(binding.Kernel), ctypes.sizeof(binding.Grid), ctypes.sizeof(binding.Opts),
            binding.Kernel.sigma2.offset, binding.Grid.kind.offset, binding.Opts.precision.offset,
            binding.Opts.reflect_fold.offset, binding.Opts.with_error.offset]
    assert got == want


def test_host_side_argument_handling_without_gpu(lib):
    from paper_1711_06874_gb300 import binding

    assert lib.tk_strerror(binding.TK_EINVAL) == b"invalid argument"
    assert lib.tk_version().startswith(b"tucker_matern")
    # NULL context / result arguments are rejected before any CUDA call
    assert lib.tk_tucker(None, None, None, None, None, None) == binding.TK_EINVAL
    r = (ctypes.c_int32 * 3)()
    assert lib.tk_ranks(None, r, None) == binding.TK_EINVAL
    o = binding.Opts()
    lib.tk_default_opts(ctypes.byref(o))
    assert abs(o.eps - 1e-6) < 1e-20 and list(o.rmax) == [32, 32, 32] and o.isotropic_shortcut == 1
    lib.tk_result_free(None)
    lib.tk_destroy(None)


def test_binding_fails_loudly_without_library(tmp_path):
    from paper_1711_06874_gb300 import binding

    saved = binding._lib
    try:
        binding._lib = None
        with pytest.raises(RuntimeError, match="not found"):
            binding.load(str(tmp_path / "missing.so"))
    finally:
        binding._lib = saved
