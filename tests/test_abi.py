"""Host-side checks of the C ABI (no GPU needed): the library builds, loads and
exports every entry point that include/hqmc.h declares; the binding covers them."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hqmc.h")


def declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hqmc_[A-Za-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2510_13866_gb300 import build

    return build.build()


def test_header_declares_the_path(libpath):
    names = declared()
    for required in ("hqmc_init_lattice", "hqmc_set_params", "hqmc_sweep", "hqmc_measure",
                     "hqmc_log_weight_grad", "hqmc_destroy", "hqmc_strerror"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    for name in declared():
        assert hasattr(lib, name), name


def test_binding_covers_every_symbol(libpath):
    from paper_2510_13866_gb300 import hqmc

    assert sorted(hqmc.SIGNATURES) == declared()


def test_strerror_and_supported_sizes(libpath):
    from paper_2510_13866_gb300 import hqmc

    lib = hqmc.lib()
    for code in range(-8, 1):
        assert lib.hqmc_strerror(code)
    assert 32 in hqmc.supported_L() and 16 in hqmc.supported_L()


def test_init_rejects_bad_arguments_without_a_gpu(libpath):
    """Argument checks happen before any device call."""
    from paper_2510_13866_gb300 import hqmc

    lib = hqmc.lib()
    ctx = ctypes.c_void_p()
    L = (ctypes.c_int * 1)(1)
    seeds = (ctypes.c_uint64 * 1)(0)
    assert lib.hqmc_init_lattice(ctypes.byref(ctx), 1, L, seeds, 0, 0) == -1  # L < 2
    L[0] = 5
    assert lib.hqmc_init_lattice(ctypes.byref(ctx), 1, L, seeds, 0, 0) == -6  # not built
    L[0] = 4
    assert lib.hqmc_init_lattice(ctypes.byref(ctx), 0, L, seeds, 0, 0) == -1
    assert lib.hqmc_init_lattice(ctypes.byref(ctx), 1, L, seeds, 7, 0) == -1
    out = ctypes.c_double(1.0)
    assert lib.hqmc_fp32_peak(0, 2, ctypes.byref(out)) == -1 and out.value == 1.0
    assert lib.hqmc_fp32_peak(0, 1, None) == -1
    assert lib.hqmc_fp64_peak(0, None) == -1


def test_product_path_does_not_reference_the_oracle():
    """The library sources and the binding never name the oracle."""
    pkg = os.path.join(ROOT, "paper_2510_13866_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "hqmc_oracle" not in text, f
