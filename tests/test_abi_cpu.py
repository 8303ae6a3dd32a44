"""C-ABI checks that need no GPU: the library builds and loads, exports
every function include/qcd.h declares, rejects bad lattice extents before
touching the device, and the ctypes structs mirror the C structs."""

import ctypes
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "qcd.h")


@pytest.fixture(scope="module")
def qcd():
    from paper_1411_5219_gb300 import _build, qcd
    _build.build()
    return qcd


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(qcd_[A-Za-z0-9_]+)\s*\(", text)))


def test_header_declares_the_hot_path_calls():
    names = declared_functions()
    for must in ["qcd_lattice_create", "qcd_gauge_create", "qcd_gauge_upload", "qcd_spinor_create",
                 "qcd_spinor_upload", "qcd_spinor_download", "qcd_apply_dslash", "qcd_apply_M", "qcd_solve_cg",
                 "qcd_status_string", "qcd_lattice_destroy", "qcd_gauge_destroy", "qcd_spinor_destroy"]:
        assert must in names


def test_library_exports_every_declared_symbol(qcd):
    lib = ctypes.CDLL(qcd.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    # and the binding knows them all
    assert set(declared_functions()) <= set(qcd._SIGS)


def test_status_strings_and_invalid_extents(qcd):
    lib = qcd.lib()
    assert lib.qcd_status_string(0) == b"QCD_OK"
    assert lib.qcd_status_string(4) == b"QCD_ERR_NOT_CONVERGED"
    for dims in [(3, 4, 4, 4), (4, 4, 4, 0), (4, 4, 1, 4)]:
        with pytest.raises(qcd.QcdError) as e:
            qcd.Lattice(dims)
        assert e.value.status == 1
    with pytest.raises(qcd.QcdError):
        qcd.Lattice((4, 4, 4, 4), t_bc=0)
    with pytest.raises(qcd.QcdError):  # 2^31 sites overflow 32-bit indices
        qcd.Lattice((2048, 1024, 1024, 2))


def test_ctypes_structs_match_c_layout(qcd):
    src = r"""
#include <stdio.h>
#include <stddef.h>
#include "qcd.h"
int main(void) {
  printf("%zu %zu %zu %zu\n", sizeof(qcd_solver_params), offsetof(qcd_solver_params, reliable_delta),
         offsetof(qcd_solver_params, inner_recon), sizeof(qcd_solver_stats));
  printf("%zu %zu\n", offsetof(qcd_solver_stats, true_rel_residual), offsetof(qcd_solver_stats, seconds));
  return 0;
}
"""
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        open(c, "w").write(src)
        exe = os.path.join(d, "t")
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()
    P, S = qcd.SolverParams, qcd.SolverStats
    assert [int(v) for v in out] == [ctypes.sizeof(P), P.reliable_delta.offset, P.inner_recon.offset,
                                     ctypes.sizeof(S), S.true_rel_residual.offset, S.seconds.offset]


def test_debug_inject_rejects_unknown_kinds(qcd):
    lib = qcd.lib()
    assert lib.qcd_debug_inject(99, 1) == 1
    assert lib.qcd_debug_inject(qcd.INJECT_SPINOR_CREATE, -1) == 1
    assert lib.qcd_debug_inject(qcd.INJECT_SPINOR_CREATE, 0) == 0
