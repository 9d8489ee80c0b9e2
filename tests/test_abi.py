"""CPU checks of the C-ABI boundary: the library builds, loads, and exports every entry point
declared in include/*.h; the product library links nothing from the oracle."""
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def J():
    from paper_2604_22087_b300 import build
    build.build()
    from paper_2604_22087_b300 import jetsci
    return jetsci


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"^\s*(?:jetsci_status|const char\s*\*)\s*(jetsci_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_paper_calls():
    names = declared_functions()
    for n in ("jetsci_mesh_create", "jetsci_residual", "jetsci_tangent_csr", "jetsci_apply_tangent",
              "jetsci_material_grad", "jetsci_norm2"):
        assert n in names


def test_every_declared_symbol_is_exported(J):
    names = declared_functions()
    assert names
    for n in names:
        assert hasattr(J.lib, n), n
    assert sorted(J.EXPORTS) == names


def test_version_and_error_string_without_gpu(J):
    assert "sm_103a" in J.version()
    assert isinstance(J.lib.jetsci_last_error(), bytes)


def test_product_library_has_no_oracle_symbols(J):
    out = subprocess.run(["nm", "-D", "--defined-only", J.LIB_PATH], capture_output=True, text=True).stdout
    assert "or_element" not in out and "or_residual" not in out
    syms = set(re.findall(r"\b(jetsci_\w+)\b", out))
    assert set(declared_functions()) <= syms


def test_header_is_plain_c(tmp_path):
    """include/jetsci.h compiles as ISO C99 (pedantic, all warnings as errors) and as C++: the
    boundary needs no C++ or CUDA types from its callers."""
    src = tmp_path / "use_header.c"
    src.write_text('#include "jetsci.h"\nint main(void) { return (int)sizeof(jetsci_material); }\n')
    inc = os.path.join(ROOT, "include")
    for cmd in (["gcc", "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-fsyntax-only", "-I", inc, str(src)],
                ["g++", "-std=c++11", "-Wall", "-Werror", "-fsyntax-only", "-x", "c++", "-I", inc, str(src)]):
        out = subprocess.run(cmd, capture_output=True, text=True)
        assert out.returncode == 0, out.stderr


def test_plain_c_program_links_and_calls_the_library(J, tmp_path):
    """A C99 program linked against libjetsci.so calls the host-only entry points without a GPU:
    the version string, destroy(NULL) as a no-op, and argument validation of mesh creation
    (JETSCI_ERR_ARG with a message), so the boundary needs neither Python nor torch."""
    src = tmp_path / "use_lib.c"
    src.write_text(r'''#include <stdio.h>
#include <string.h>
#include "jetsci.h"
int main(void) {
    const char *v = jetsci_version();
    if (!v || !strstr(v, "sm_103a")) return 1;
    if (jetsci_mesh_destroy(NULL) != JETSCI_OK) return 2;
    double xyz[3] = {0, 0, 0};
    if (jetsci_mesh_create(xyz, 1, NULL, 0, NULL, NULL, 0, NULL, NULL) != JETSCI_ERR_ARG) return 3;
    if (strlen(jetsci_last_error()) == 0) return 4;
    return 0;
}
''')
    libdir = os.path.dirname(J.LIB_PATH)
    exe = tmp_path / "use_lib"
    cuda_lib = "/usr/local/cuda/lib64"
    out = subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src),
                          "-L" + libdir, "-ljetsci", "-Wl,-rpath," + libdir, "-L" + cuda_lib, "-Wl,-rpath," + cuda_lib,
                          "-o", str(exe)], capture_output=True, text=True)
    assert out.returncode == 0, out.stderr
    run = subprocess.run([str(exe)], capture_output=True, text=True)
    assert run.returncode == 0, (run.returncode, run.stderr)
