"""The C-ABI library: it builds for sm_103a, loads without a GPU, and exports every entry point that
include/comet_scan.h declares.  No compute call is made here."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "comet_scan.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(comet_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_1911_09340_gb300 import build
    return build.build()


def test_header_declares_the_scan_steps():
    names = declared_functions()
    for n in ("comet_scan_lattice", "comet_scan_propagate", "comet_scan_dca", "comet_scan_select",
              "comet_scan_classify", "comet_ctx_create", "comet_ctx_destroy", "comet_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    for name in declared_functions():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (comet_\w+)$", out, flags=re.M))
    assert set(declared_functions()) <= exported


def test_binding_signatures_cover_the_header():
    from paper_1911_09340_gb300 import binding
    assert set(binding.SIGNATURES) == set(declared_functions())


def test_library_is_built_for_sm_103a():
    """The build compiles every translation unit for sm_103a only (one -gencode)."""
    from paper_1911_09340_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    assert "-gencode" not in build.FLAGS and not any("arch" in f for f in build.FLAGS)


@pytest.mark.gpu
def test_kernels_report_sm_103():
    """The loaded library's kernels carry SM version 10.3 (read from a kernel's attributes)."""
    from paper_1911_09340_gb300 import binding
    assert binding.kernel_arch() == 103


def test_header_compiles_as_c(tmp_path):
    src = tmp_path / "t.c"
    src.write_text('#include "comet_scan.h"\nint main(void){ comet_scan_params p; (void)p; return 0; }\n')
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                    "-c", str(src), "-o", str(tmp_path / "t.o")], check=True)
