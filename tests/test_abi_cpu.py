"""CPU checks of the boundary: the CUDA library builds, loads without a GPU and
exports every entry point declared in include/mrhs.h; the Python binding
mirrors exactly those names; host-side argument validation rejects bad shapes
before any CUDA call."""
import ctypes
import os
import re

import pytest

import paper_1601_03184_gb300 as pkg
from paper_1601_03184_gb300 import build as libbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mrhs.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mrhs_[a-z_A-Z0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    libbuild.build()
    return ctypes.CDLL(libbuild.LIB)


def test_header_declares_the_setup_api():
    names = declared_functions()
    for required in ["mrhs_create", "mrhs_set_gauge", "mrhs_build_clover", "mrhs_setup_init", "mrhs_setup_refine",
                     "mrhs_apply_D", "mrhs_apply_Dc", "mrhs_destroy"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_mirrors_header():
    assert sorted(pkg.exported_symbols()) == declared_functions()
    for n in declared_functions():
        assert callable(getattr(pkg, n))


def test_host_side_shape_validation(lib):
    pkg.lib()
    out = ctypes.c_void_p()
    i4 = lambda v: (ctypes.c_int * 4)(*v)
    # 4 is not divisible by 3
    st = pkg.lib().mrhs_create(i4((4, 4, 4, 4)), i4((3, 2, 2, 2)), 4, 0, None, ctypes.byref(out))
    assert st == pkg.MRHS_ERR_SHAPE
    # odd number of aggregates along t
    st = pkg.lib().mrhs_create(i4((4, 4, 4, 6)), i4((2, 2, 2, 2)), 4, 0, None, ctypes.byref(out))
    assert st == pkg.MRHS_ERR_SHAPE
    assert b"even" in pkg.lib().mrhs_last_error(None)
    # bad precision enum
    st = pkg.lib().mrhs_create(i4((4, 4, 4, 4)), i4((2, 2, 2, 2)), 4, 9, None, ctypes.byref(out))
    assert st == pkg.MRHS_ERR_ARG
    # null output pointer
    st = pkg.lib().mrhs_create(i4((4, 4, 4, 4)), i4((2, 2, 2, 2)), 4, 0, None, None)
    assert st == pkg.MRHS_ERR_ARG


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    monkeypatch.setattr(pkg, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(pkg, "_lib", None)
    with pytest.raises(pkg.MrhsError):
        pkg.lib()


def test_checkpoint_calls_refuse_null_arguments(lib):
    # argument checks come before any device work, so they run without a GPU
    assert pkg.lib().mrhs_save_setup(None, b"setup.bin") == pkg.MRHS_ERR_ARG
    assert pkg.lib().mrhs_load_setup(None, b"setup.bin") == pkg.MRHS_ERR_ARG
    assert b"null" in pkg.lib().mrhs_last_error(None)


def test_header_is_plain_c_and_links(lib, tmp_path):
    """A C99 program that includes mrhs.h, takes the address of every declared
    entry point and links against libmrhs.so: the boundary needs no C++ or
    torch type. It then runs the argument checks that need no GPU."""
    import shutil
    import subprocess

    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    names = declared_functions()
    src = tmp_path / "use_abi.c"
    src.write_text(
        "#include <stdio.h>\n#include <string.h>\n#include \"mrhs.h\"\n"
        "typedef void (*any_fn)(void);\n"
        "static const any_fn table[] = {\n" + ",\n".join("  (any_fn)%s" % n for n in names) + "\n};\n"
        "int main(void) {\n"
        "  const int dims[4] = {4, 4, 4, 4}, bad_agg[4] = {3, 2, 2, 2};\n"
        "  mrhs_ctx ctx = NULL;\n"
        "  size_t i;\n"
        "  for (i = 0; i < sizeof table / sizeof table[0]; ++i)\n"
        "    if (!table[i]) return 10;\n"
        "  if (mrhs_create(dims, bad_agg, 4, MRHS_PREC_FP64, NULL, &ctx) != MRHS_ERR_SHAPE) return 11;\n"
        "  if (ctx != NULL || strlen(mrhs_last_error(NULL)) == 0) return 12;\n"
        "  if (mrhs_save_setup(NULL, \"setup.bin\") != MRHS_ERR_ARG) return 13;\n"
        "  if (mrhs_load_setup(NULL, \"setup.bin\") != MRHS_ERR_ARG) return 14;\n"
        "  mrhs_destroy(NULL);\n"
        "  printf(\"%u entry points\\n\", (unsigned)(sizeof table / sizeof table[0]));\n"
        "  return 0;\n"
        "}\n")
    exe = tmp_path / "use_abi"
    libdir = os.path.dirname(pkg.LIB_PATH)
    subprocess.check_call(["gcc", "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I",
                           os.path.join(ROOT, "include"), str(src), "-o", str(exe), "-L", libdir, "-lmrhs",
                           "-Wl,-rpath," + libdir])
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, (out.returncode, out.stderr)
    assert out.stdout.strip() == "%d entry points" % len(names)
