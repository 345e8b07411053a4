"""The C-ABI library builds, loads without a GPU, exports every entry point that
include/lns.h declares, and the Python binding's structures match the C layout."""
import ctypes as C
import os
import re
import subprocess
import tempfile

import numpy as np
import pytest

from paper_2008_01539_gb300 import build as B
from paper_2008_01539_gb300 import lns

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lns.h")


@pytest.fixture(scope="module")
def lib():
    B.build()
    return C.CDLL(B.LIB)


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lns_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary_calls():
    names = declared_functions()
    for required in ("lns_model_create", "lns_timestep", "lns_newton_iter", "lns_active_set", "lns_solve_local"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    assert sorted(lns.EXPORTS) == declared_functions()


def test_last_error_and_defaults_without_gpu(lib):
    lib.lns_last_error.restype = C.c_char_p
    assert isinstance(lib.lns_last_error(), bytes)
    o = lns.lns_options()
    lib.lns_options_default.argtypes = [C.POINTER(lns.lns_options)]
    assert lib.lns_options_default(C.byref(o)) == 0
    assert o.mode == lns.LNS_MODE_LOCAL and o.m_layers == 2
    assert abs(o.eps_p - 0.3 * lns.PSI) < 1e-9
    # invalid argument paths need no device
    lib.lns_options_default.argtypes = [C.c_void_p]
    assert lib.lns_options_default(None) == lns.LNS_EINVAL


def test_struct_layouts_match_c():
    structs = ["lns_fluid", "lns_model_desc", "lns_options", "lns_allocator", "lns_iter_stats", "lns_step_stats",
               "lns_kernel_time", "lns_server_options", "lns_completion", "lns_server_stats", "lns_dt_control",
               "lns_advance_stats", "lns_batch_stats", "lns_tuning", "lns_bo_fluid"]
    src = "#include <stdio.h>\n#include <stddef.h>\n#include \"lns.h\"\nint main(void){\n"
    for s in structs:
        src += f'  printf("{s} %zu\\n", sizeof({s}));\n'
    # every field of every mirrored structure: same name, same offset in C and in ctypes
    for s in structs:
        for name, _ in getattr(lns, s)._fields_:
            src += f'  printf("{s}.{name} %zu\\n", offsetof({s}, {name}));\n'
    src += "  return 0;\n}\n"
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        exe = os.path.join(d, "t")
        open(c, "w").write(src)
        subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {ln.split()[0]: int(ln.split()[1]) for ln in out if ln.strip()}
    for s in structs:
        st = getattr(lns, s)
        assert got[s] == C.sizeof(st), s
        for name, _ in st._fields_:
            assert got[f"{s}.{name}"] == getattr(st, name).offset, (s, name)


@pytest.mark.parametrize("n", [0, 1, 31, 32, 33, 1000])
def test_bitset_conversion_roundtrip(n):
    rng = np.random.default_rng(n)
    m = (rng.random(n) < 0.4).astype(np.uint8)
    bits = lns.mask_to_bits(m)
    assert bits.dtype == np.uint32 and bits.shape[0] == (n + 31) // 32
    assert np.array_equal(lns.bits_to_mask(bits, n), m)
    for i in np.flatnonzero(m):  # bit (i & 31) of word (i >> 5)
        assert (int(bits[i >> 5]) >> (i & 31)) & 1


def test_product_path_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_2008_01539_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "lns_oracle" not in text, f


def test_black_oil_entry_points_reject_bad_arguments_without_gpu(lib):
    """lns_bo_assemble / lns_bo_update check their arguments before touching the device."""
    L = lns.load()
    fl = lns.bo_fluid(__import__("paper_2008_01539_gb300.casegen", fromlist=["x"]).BlackOilFluid())
    args = lambda n, dt: [n, *([None] * 5), 0, *([None] * 13), dt, *([None] * 5)]  # noqa: E731
    assert L.lns_bo_assemble(None, *args(1, 1.0)) == lns.LNS_EINVAL          # no fluid
    assert L.lns_bo_assemble(C.byref(fl), *args(1, 1.0)) == lns.LNS_EINVAL   # NULL arrays
    assert L.lns_bo_assemble(C.byref(fl), *args(0, 0.0)) == lns.LNS_EINVAL   # dt <= 0
    assert L.lns_bo_assemble(C.byref(fl), *args(-1, 1.0)) == lns.LNS_EINVAL  # negative size
    assert L.lns_bo_assemble(C.byref(fl), *args(0, 1.0)) == lns.LNS_OK       # nothing to do
    bad = lns.bo_fluid(__import__("paper_2008_01539_gb300.casegen", fromlist=["x"]).BlackOilFluid(n_g=0))
    assert L.lns_bo_update(C.byref(fl), 4, 0.2, *([None] * 9)) == lns.LNS_EINVAL
    assert L.lns_bo_update(C.byref(fl), 0, 0.2, *([None] * 9)) == lns.LNS_OK
    assert L.lns_bo_assemble(C.byref(bad), *args(0, 1.0)) == lns.LNS_OK  # checked only with cells to assemble

