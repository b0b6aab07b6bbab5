"""The C++ oracle under AddressSanitizer and UndefinedBehaviorSanitizer, CPU only: every entry
point on every equation kind, both boundary conditions, 2-D and 3-D grids down to 2 x 2 (the
boundary mapping's degenerate cases) and the transform hooks at lengths 1..16, compiled with
-fsanitize=address,undefined into a temporary library and run in a child process; any report
fails the test."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r'''
import sys
from oracle import cpp_oracle as C
from paper_2305_03945_gb300 import workloads as WL
C.LIB = sys.argv[1]
C.up_to_date = lambda: True
C._lib = None
C.set_threads(1)
KINDS = [("none", "laplacian", ()), ("none", "neg_biharmonic", ()), ("allen_cahn", "laplacian", ()),
         ("ch_implicit", "neg_biharmonic", ()), ("ch_split", "neg_biharmonic", ()),
         ("gray_scott", "laplacian", (2e-3, 1e-3, 0.04, 0.06)),
         ("schnakenberg", "laplacian", (0.05, 1.0, 100.0, 0.1305, 0.7695)), ("fch", "functionalized", ())]
r = WL.rng(1)
n = 0
for bc in ("periodic", "neumann"):
    for kind, op, p in KINDS:
        for nz, ny, nx in [(1, 2, 2), (1, 2, 8), (1, 16, 4), (2, 4, 8), (4, 4, 4)]:
            if nz > 1 and kind in ("gray_scott", "schnakenberg", "fch"):
                continue
            ch = op != "laplacian"
            pb = WL.Problem(nx=nx, ny=ny, nz=nz, lx=1.0, ly=1.3, lz=0.7, bc=bc, op=op, kind=kind, p=p,
                            dt=1e-5 if ch else 2e-3, a=4e-4 if ch else 0.05, b=1.0, tau_u=0.9, tau_p=0.9,
                            tol=1e-12, tol_kind="f_rel", max_iter=50)
            if kind == "fch":
                pb = pb.replace(a=0.18 ** 2, dt=1e-6)
            U, W = r.uniform(0.1, 0.9, pb.shape), r.standard_normal(pb.shape)
            C.residual(pb, U, U)
            C.grad_F_T(pb, U, W)
            C.ghat(pb)
            C.apply_ginv(pb, W)
            C.pdhg_step(pb, U, history=True)
            C.pdhg_step(pb.replace(tol_kind="res_abs", tol=1e-9), U)
            if kind in ("allen_cahn", "ch_implicit", "ch_split"):
                C.apply_ginv(pb.replace(precond="stabilized", shift=2.0), W)
            n += 1
for m in (1, 2, 4, 8, 16):
    C.fft(r.standard_normal(m) + 1j * r.standard_normal(m))
    C.fft(r.standard_normal(m) + 0j, inverse=True)
    C.dct2(r.standard_normal(m))
    C.dct3(r.standard_normal(m))
print("sanitized-ok", n)
'''


def _asan_runtime():
    if shutil.which("g++") is None:
        return None
    r = subprocess.run(["g++", "-print-file-name=libasan.so"], stdout=subprocess.PIPE, text=True)
    p = r.stdout.strip()
    return p if os.path.isabs(p) and os.path.exists(p) else None


@pytest.mark.skipif(_asan_runtime() is None, reason="needs g++ with the AddressSanitizer runtime")
def test_cpp_oracle_is_clean_under_asan_and_ubsan(tmp_path):
    lib = tmp_path / "librd_oracle_sanitized.so"
    src = os.path.join(ROOT, "oracle", "rd_oracle_cpp.cpp")
    r = subprocess.run(["g++", "-O1", "-g", "-std=c++17", "-shared", "-fPIC", "-fno-omit-frame-pointer",
                        "-fsanitize=address,undefined", "-fno-sanitize-recover=undefined", "-o", str(lib), src],
                       stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
    assert r.returncode == 0, r.stdout.decode(errors="replace")
    env = dict(os.environ, LD_PRELOAD=_asan_runtime(), ASAN_OPTIONS="detect_leaks=0:abort_on_error=1",
               UBSAN_OPTIONS="print_stacktrace=1", PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, "-c", SCRIPT, str(lib)], cwd=ROOT, env=env, stdout=subprocess.PIPE,
                       stderr=subprocess.STDOUT, timeout=600)
    out = r.stdout.decode(errors="replace")
    assert r.returncode == 0 and "sanitized-ok" in out, out[-4000:]
    assert "runtime error" not in out and "AddressSanitizer" not in out, out[-4000:]
