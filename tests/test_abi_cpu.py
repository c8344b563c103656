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


class FakeCudaTensor:
    """Stands in for a torch CUDA tensor on a CPU-only machine: the binding
    reads only these attributes of a device-field argument."""

    class _Dev:
        def __init__(self, index):
            self.index = index

    def __init__(self, nbytes, device=0, contiguous=True):
        self.nbytes_ = nbytes
        self.is_cuda = True
        self.device = self._Dev(device)
        self.contiguous = contiguous

    def data_ptr(self):
        return 1 << 20

    def is_contiguous(self):
        return self.contiguous

    def numel(self):
        return self.nbytes_

    def element_size(self):
        return 1


def _fake_library(monkeypatch, calls):
    class FakeLib:
        def __getattr__(self, name):
            return lambda *a: calls.append(name) or 0

    monkeypatch.setattr(pkg, "lib", lambda: FakeLib())
    monkeypatch.setattr(pkg, "mrhs_field_bytes", lambda ctx, nrhs, dtype, coarse=0: (2048 if coarse else 1024) * nrhs)
    monkeypatch.setattr(pkg, "mrhs_info", lambda ctx: [0, 0, 0, 2, 0, 0, 0, 0])  # ntv 2 on cuda:0


def _field_cases(np):
    F64 = pkg.MRHS_F64
    return [
        ("mrhs_apply_D", lambda f, c: pkg.mrhs_apply_D(1, f(2), f(2), 2, F64)),
        ("mrhs_apply_D_block", lambda f, c: pkg.mrhs_apply_D_block(1, f(2), f(2), 2, F64)),
        ("mrhs_sap", lambda f, c: pkg.mrhs_sap(1, f(2), f(2), 2, F64, 1, 1)),
        ("mrhs_restrict", lambda f, c: pkg.mrhs_restrict(1, f(2), c(2), 2, F64)),
        ("mrhs_prolong", lambda f, c: pkg.mrhs_prolong(1, c(2), f(2), 2, F64)),
        ("mrhs_apply_Dc", lambda f, c: pkg.mrhs_apply_Dc(1, c(2), c(2), 2, F64)),
        ("mrhs_coarse_solve", lambda f, c: pkg.mrhs_coarse_solve(1, c(2), c(2), 2, F64, 0.1, 4, 4)),
        ("mrhs_coarse_solve_noalloc", lambda f, c: pkg.mrhs_coarse_solve_noalloc(1, c(2), c(2), 2, F64, 0.1, 4, 4)),
        ("mrhs_pack", lambda f, c: pkg.mrhs_pack(1, np.zeros(1), F64, f(2), F64, 2)),
        ("mrhs_unpack", lambda f, c: pkg.mrhs_unpack(1, f(2), F64, np.zeros(1), F64, 2)),
        ("mrhs_pack_coarse", lambda f, c: pkg.mrhs_pack_coarse(1, np.zeros(1), F64, c(2), F64, 2)),
        ("mrhs_unpack_coarse", lambda f, c: pkg.mrhs_unpack_coarse(1, c(2), F64, np.zeros(1), F64, 2)),
        ("mrhs_set_tv", lambda f, c: pkg.mrhs_set_tv(1, f(2), F64)),
        ("mrhs_setup_init", lambda f, c: pkg.mrhs_setup_init(1, f(2), F64, 0, 1, 1)),
        ("mrhs_setup_init_learned", lambda f, c: pkg.mrhs_setup_init_learned(1, f(2), F64, 1, 1)),
    ]


def test_short_buffers_are_refused_before_the_library_is_called(monkeypatch):
    """The binding compares every torch tensor passed as a field with the
    library's size for that field and refuses a short one, so a kernel never
    reads or writes past the end of a caller's buffer."""
    import numpy as np

    calls = []
    _fake_library(monkeypatch, calls)
    fine = lambda n: FakeCudaTensor(1024 * n)
    coarse = lambda n: FakeCudaTensor(2048 * n)
    short_f = lambda n: FakeCudaTensor(1024 * n - 1)
    short_c = lambda n: FakeCudaTensor(2048 * n - 1)
    for name, call in _field_cases(np):
        calls.clear()
        call(fine, coarse)
        assert calls[-1] == name
        for f, c in ((short_f, coarse), (fine, short_c)):
            calls.clear()
            try:
                call(f, c)
            except pkg.MrhsError as e:
                assert e.status == pkg.MRHS_ERR_ARG and "needs" in str(e)
                assert calls == []
            else:
                # this call has no argument of the shortened kind
                assert calls == [name]
    # raw integer pointers are passed through (the library checks them);
    # non-contiguous tensors are refused
    calls.clear()
    pkg.mrhs_apply_D(1, 4096, 8192, 2, pkg.MRHS_F64)
    assert calls == ["mrhs_apply_D"]
    with pytest.raises(ValueError):
        pkg.mrhs_apply_D(1, FakeCudaTensor(2048, contiguous=False), fine(2), 2, pkg.MRHS_F64)


def test_host_memory_is_refused_as_a_device_field(monkeypatch):
    """A numpy array, a CPU tensor or a CUDA tensor of another GPU passed
    where the library expects a device field of the context's GPU is refused
    by the binding before any call: a host address handed to a kernel would
    fault the GPU. A CUDA tensor passed where a host array is expected is
    refused too."""
    import numpy as np
    import torch

    calls = []
    _fake_library(monkeypatch, calls)
    good_f = lambda n: FakeCudaTensor(1024 * n)
    good_c = lambda n: FakeCudaTensor(2048 * n)
    wrong = [lambda n, k=k: k(n) for k in (lambda n: np.zeros(1024 * n, np.uint8),
                                            lambda n: torch.zeros(1024 * n, dtype=torch.uint8),
                                            lambda n: FakeCudaTensor(4096 * n, device=1))]
    for name, call in _field_cases(np):
        for w in wrong:
            for f, c in ((w, good_c), (good_f, w)):
                calls.clear()
                try:
                    call(f, c)
                except pkg.MrhsError as e:
                    assert e.status == pkg.MRHS_ERR_ARG, (name, str(e))
                    assert calls == [], name
                else:
                    assert calls == [name]  # no argument of this kind
    for call in (lambda: pkg.mrhs_pack(1, FakeCudaTensor(64), pkg.MRHS_F64, good_f(2), pkg.MRHS_F64, 2),
                 lambda: pkg.mrhs_unpack(1, good_f(2), pkg.MRHS_F64, FakeCudaTensor(64), pkg.MRHS_F64, 2)):
        calls.clear()
        with pytest.raises(pkg.MrhsError):
            call()
        assert calls == []


def test_lattice_refuses_misshapen_host_arrays():
    """Host fields and the gauge field are read by the library with the
    lattice's own sizes, so the wrapper checks their shapes first."""
    import numpy as np

    from paper_1601_03184_gb300 import Lattice

    lat = object.__new__(Lattice)  # no device context: the checks come first
    lat.V, lat.nagg, lat.ntv, lat.ctx = 16, 1, 2, None
    with pytest.raises(ValueError):
        lat.to_device(np.zeros((2, 15, 12), np.complex128), pkg.MRHS_F64)
    with pytest.raises(ValueError):
        lat.to_device(np.zeros((16, 12), np.complex128), pkg.MRHS_F64)
    with pytest.raises(ValueError):
        lat.to_device(np.zeros((2, 1, 3), np.complex64), pkg.MRHS_F32, coarse=True)
    with pytest.raises(ValueError):
        lat.set_gauge(np.zeros((16, 4, 3, 2), np.complex128))


def test_create_refuses_empty_and_oversized_problems(lib):
    """Limits checked before any device work: ntv in 1..min(64, 6|aggregate|),
    volume below 2^30 sites (32-bit site indices with two flag bits), no
    empty lattice."""
    pkg.lib()
    out = ctypes.c_void_p()
    i4 = lambda v: (ctypes.c_int * 4)(*v)
    for dims, agg, ntv in [((4, 4, 4, 4), (2, 2, 2, 2), 0),          # no test vectors
                           ((8, 8, 8, 8), (4, 4, 4, 4), 65),         # above 64 test vectors
                           ((2, 2, 2, 2), (1, 1, 1, 1), 7),          # above 6 |aggregate|
                           ((1024, 1024, 1024, 2), (2, 2, 2, 1), 8),  # 2^31 sites
                           ((0, 4, 4, 4), (2, 2, 2, 2), 4),          # empty lattice
                           ((4, 4, 4, 4), (0, 2, 2, 2), 4)]:         # empty aggregate
        st = pkg.lib().mrhs_create(i4(dims), i4(agg), ntv, 0, None, ctypes.byref(out))
        assert st == pkg.MRHS_ERR_SHAPE, (dims, agg, ntv, st)
        assert out.value is None
