"""The C-ABI library builds for sm_103a, loads, and exports every function include/rd_pdhg.h
declares (no compute calls: this runs without a GPU)."""
import ctypes
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "rd_pdhg.h")).read()
    return sorted(set(re.findall(r"RD_API\s+[\w\s\*]+?\b(rd_\w+)\s*\(", src)))


def test_header_declares_the_method_calls():
    names = _declared()
    for n in ("rd_pdhg_create", "rd_pdhg_step", "rd_pdhg_solve", "rd_pdhg_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2305_03945_gb300 import build, rd
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
    assert set(rd.EXPORTS) == set(_declared())


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_header_is_plain_c_and_links_against_the_library(tmp_path):
    """A C99 caller with every warning as an error: the header needs no C++ and no CUDA headers,
    and a program calling the method's entry points links against the built library."""
    from paper_2305_03945_gb300 import build
    lib = build.build()
    src = tmp_path / "caller.c"
    src.write_text("""
#include <stdio.h>
#include "rd_pdhg.h"
int run(double *d_u) {
  rd_grid g = {2, {64, 64, 1}, {1.0, 1.0, 1.0}};
  rd_reaction rx = {RD_RX_ALLEN_CAHN, 1, 0.1, 10.0, {0}};
  rd_precond pc = {RD_PC_STABILIZED, 2.0};
  rd_opts o;
  rd_pdhg *h = NULL;
  rd_step_info info;
  rd_opts_default(&o);
  o.precision = RD_PREC_FP32_DC;
  if (rd_pdhg_create(&h, &g, RD_BC_PERIODIC, RD_OP_LAPLACIAN, &rx, 1e-2, 1.0, 1.0, &pc, &o, NULL) != RD_OK) {
    fprintf(stderr, "%s\\n", rd_last_error());
    return 1;
  }
  rd_pdhg_step(h, d_u, d_u, &info);
  rd_pdhg_solve(h, d_u, 2, NULL);
  rd_pdhg_destroy(h);
  return info.status;
}
""")
    obj, so = tmp_path / "caller.o", tmp_path / "libcaller.so"
    inc = os.path.join(ROOT, "include")
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic", "-fPIC", "-I", inc, "-c",
                        str(src), "-o", str(obj)], stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
    assert r.returncode == 0, r.stdout.decode()
    r = subprocess.run(["gcc", "-shared", "-o", str(so), str(obj), "-L", os.path.dirname(lib), "-lrd_pdhg"],
                       stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
    assert r.returncode == 0, r.stdout.decode()


def test_status_strings_and_argument_checks_without_gpu():
    """Host-side validation runs before any CUDA call, so it is testable on a CPU machine."""
    from paper_2305_03945_gb300 import build, rd, workloads as WL
    build.build()
    lib = rd.load()
    assert lib.rd_status_string(rd.RD_ERR_DIVERGED) == b"RD_ERR_DIVERGED"
    pb = WL.config_allen_cahn_periodic(16, 1).problem
    g, rx, pc, o = rd.make_structs(pb)
    h = ctypes.c_void_p()
    # non-power-of-two side
    g.n[0] = 12
    s = lib.rd_pdhg_create(ctypes.byref(h), ctypes.byref(g), 0, 0, ctypes.byref(rx), pb.dt, 1.0, 1.0,
                           ctypes.byref(pc), ctypes.byref(o), None)
    assert s == rd.RD_ERR_UNSUPPORTED and not h.value
    g.n[0] = 16
    # wrong operator for Allen-Cahn
    s = lib.rd_pdhg_create(ctypes.byref(h), ctypes.byref(g), 0, 1, ctypes.byref(rx), pb.dt, 1.0, 1.0,
                           ctypes.byref(pc), ctypes.byref(o), None)
    assert s == rd.RD_ERR_INVALID_ARG and b"LAPLACIAN" in lib.rd_last_error()
    # non-positive step sizes and time step
    for dt, tau, sig in ((0.0, 1.0, 1.0), (0.01, -1.0, 1.0), (0.01, 1.0, 0.0)):
        s = lib.rd_pdhg_create(ctypes.byref(h), ctypes.byref(g), 0, 0, ctypes.byref(rx), dt, tau, sig,
                               ctypes.byref(pc), ctypes.byref(o), None)
        assert s == rd.RD_ERR_INVALID_ARG
    # ncomp must match the kind
    rx.ncomp = 2
    s = lib.rd_pdhg_create(ctypes.byref(h), ctypes.byref(g), 0, 0, ctypes.byref(rx), pb.dt, 1.0, 1.0,
                           ctypes.byref(pc), ctypes.byref(o), None)
    assert s == rd.RD_ERR_INVALID_ARG
    assert lib.rd_pdhg_step(None, None, None, None) == rd.RD_ERR_INVALID_ARG
    rx.ncomp = 1


def test_preconditioner_arguments_checked_without_gpu():
    """RD_PC_STABILIZED: s >= 0 and finite; the shift belongs to that kind alone; two-species
    systems refuse it (no scalar nonlinear factor); unknown kinds are invalid."""
    from paper_2305_03945_gb300 import build, rd, workloads as WL
    build.build()
    lib = rd.load()
    h = ctypes.c_void_p()

    def create(pb, kind, shift):
        g, rx, pc, o = rd.make_structs(pb)
        pc.kind, pc.s = kind, shift
        return lib.rd_pdhg_create(ctypes.byref(h), ctypes.byref(g), rd.BC[pb.bc], rd.OP[pb.op], ctypes.byref(rx),
                                  pb.dt, pb.tau_u, pb.tau_p, ctypes.byref(pc), ctypes.byref(o), None)

    ac = WL.config_allen_cahn_periodic(16, 1).problem
    for shift in (-1.0, float("nan"), float("inf")):
        assert create(ac, rd.PRECOND["stabilized"], shift) == rd.RD_ERR_INVALID_ARG and not h.value
        assert b"shift" in lib.rd_last_error()
    assert create(ac, rd.PRECOND["linear"], 2.0) == rd.RD_ERR_INVALID_ARG
    assert create(ac, rd.PRECOND["none"], 2.0) == rd.RD_ERR_INVALID_ARG
    assert create(ac, 3, 0.0) == rd.RD_ERR_INVALID_ARG and b"preconditioner kind" in lib.rd_last_error()
    gs = WL.Problem(nx=16, ny=16, lx=1.0, ly=1.0, bc="periodic", op="laplacian", kind="gray_scott",
                    p=(2e-3, 1e-3, 0.04, 0.06), dt=1.0)
    assert create(gs, rd.PRECOND["stabilized"], 2.0) == rd.RD_ERR_UNSUPPORTED and not h.value
