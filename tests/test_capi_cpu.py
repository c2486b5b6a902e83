"""CPU-only checks of the boundary: the CUDA library builds for sm_103a, loads, and
exports every function that include/amg.h declares (no GPU calls here)."""
import ctypes as C
import os
import subprocess

import pytest

from paper_1403_1649_gb300 import amg, build


@pytest.fixture(scope="module")
def built():
    return build.build()


def test_library_exports_every_header_symbol(built):
    names = amg.header_functions()
    assert "amg_setup" in names and "amg_solve" in names and len(names) >= 10
    lib = C.CDLL(built)
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", built], capture_output=True, text=True).stdout
    exported = {l.split()[-1] for l in out.splitlines() if " T " in l}
    assert set(names) <= exported


def test_default_params_host_only(built):
    p = amg.amg_default_params()
    assert p.alpha == 0.25 and p.coarse_max == 64 and p.kcycle_levels == 2 and p.kcycle_t == 0.25
    assert p.precision == amg.AMG_PREC_F64 and p.outer == 0 and p.restart == 30 and p.use_graph == 1
    assert amg.amg_last_error() == ""


def test_struct_layout_matches_header(built):
    # sizes of the ABI structs (x86_64 and aarch64 LP64 agree)
    assert C.sizeof(amg.amg_csr) == 40
    assert C.sizeof(amg.amg_params) == 104
    assert C.sizeof(amg.amg_level_info) == 40
    assert C.sizeof(amg.amg_solve_info) == 48


def test_null_arguments_rejected_without_gpu(built):
    L = amg.lib()
    h = C.c_void_p()
    assert L.amg_setup(None, None, None, C.byref(h)) == amg.AMG_ERR_BAD_INPUT
    assert "amg_setup" in amg.amg_last_error()
    assert L.amg_solve(None, None, None, 1e-8, None, None, None) == amg.AMG_ERR_BAD_INPUT
    L.amg_free(None)


def test_build_is_sm103a_only():
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    assert os.path.exists(os.path.join(build.CSRC, "setup.cu"))
