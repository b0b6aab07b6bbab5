"""ctypes binding of the plain FP64 C++ oracle (oracle/rd_oracle_cpp.cpp).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``): imported by tests, smoke() and the
CPU-baseline / reference legs of bench.py, never by the product library.

The functions mirror ``rd_oracle``'s (``residual``, ``grad_F_T``, ``apply_ginv``, ``ghat``,
``measure`` is not needed, ``pdhg_step``, ``solve``) and take the same ``Problem`` records and
``[ncomp, ny, nx]`` float64 arrays.  ``build()`` compiles the library in place with g++ (-O2,
OpenMP when available); ``set_threads(n)`` sets the OpenMP thread count (timing only: results do
not depend on it).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "rd_oracle_cpp.cpp")
LIB = os.path.join(HERE, "librd_oracle.so")

OK, NOT_CONVERGED, DIVERGED = "ok", "not_converged", "diverged"
_STATUS = {0: OK, 1: NOT_CONVERGED, 2: DIVERGED}
_BC = {"periodic": 0, "neumann": 1}
_OP = {"laplacian": 0, "neg_biharmonic": 1, "functionalized": 2}
_KIND = {"none": 0, "allen_cahn": 1, "ch_implicit": 2, "ch_split": 3, "gray_scott": 4, "schnakenberg": 5, "fch": 6}
_PC = {"none": 0, "linear": 1, "stabilized": 2}
_TOL = {"res_abs": 0, "f_rel": 1}


class rdo_problem(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("lx", ctypes.c_double), ("ly", ctypes.c_double),
                ("bc", ctypes.c_int), ("op", ctypes.c_int), ("kind", ctypes.c_int),
                ("dt", ctypes.c_double), ("a", ctypes.c_double), ("b", ctypes.c_double),
                ("p", ctypes.c_double * 6), ("tau_u", ctypes.c_double), ("tau_p", ctypes.c_double),
                ("omega", ctypes.c_double), ("precond", ctypes.c_int), ("tol", ctypes.c_double),
                ("tol_kind", ctypes.c_int), ("max_iter", ctypes.c_int), ("nz", ctypes.c_int),
                ("lz", ctypes.c_double), ("shift", ctypes.c_double)]


def up_to_date() -> bool:
    return os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC)


def build(force: bool = False) -> str:
    """Compile librd_oracle.so next to its source (g++ -O2, with -fopenmp when it links)."""
    if not force and up_to_date():
        return LIB
    tmp = LIB + ".tmp"
    base = ["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-o", tmp, SRC]
    r = subprocess.run(base[:2] + ["-fopenmp"] + base[2:], stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
    if r.returncode != 0:
        r = subprocess.run(base, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
        if r.returncode != 0:
            raise RuntimeError("g++ failed:\n" + r.stdout.decode(errors="replace"))
    os.replace(tmp, LIB)
    return LIB


_lib = None


def load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(LIB)
        P = ctypes.POINTER
        d = P(ctypes.c_double)
        pp = P(rdo_problem)
        for name, args in (("rdo_residual", [pp, d, d, d]), ("rdo_grad_F_T", [pp, d, d, d]),
                           ("rdo_apply_ginv", [pp, d, d]), ("rdo_ghat", [pp, d])):
            getattr(lib, name).argtypes = args
            getattr(lib, name).restype = None
        lib.rdo_pdhg_step.argtypes = [pp, d, d, P(ctypes.c_int), P(ctypes.c_int), d, d, ctypes.c_int]
        lib.rdo_pdhg_step.restype = None
        lib.rdo_set_threads.argtypes = [ctypes.c_int]
        lib.rdo_set_threads.restype = ctypes.c_int
        lib.rdo_fft.argtypes = [d, ctypes.c_int, ctypes.c_int]
        lib.rdo_dct2.argtypes = [d, d, ctypes.c_int]
        lib.rdo_dct3.argtypes = [d, d, ctypes.c_int]
        for name in ("rdo_fft", "rdo_dct2", "rdo_dct3"):
            getattr(lib, name).restype = None
        _lib = lib
    return _lib


def set_threads(n: int) -> int:
    return load().rdo_set_threads(int(n))


def _transform_sides(pb):
    """The radix-2 FFT and the DCT through it take power-of-two lengths only."""
    if pb.precond == "none":
        return
    for n in (pb.nx, pb.ny) + ((pb.nz,) if pb.nz > 1 else ()):
        if n < 1 or n & (n - 1):
            raise ValueError("the C++ oracle's transforms need power-of-two grid sides, got %d" % n)


def _problem(pb) -> rdo_problem:
    s = rdo_problem()
    s.nx, s.ny, s.lx, s.ly = pb.nx, pb.ny, pb.lx, pb.ly
    s.bc, s.op, s.kind = _BC[pb.bc], _OP[pb.op], _KIND[pb.kind]
    s.dt, s.a, s.b = pb.dt, pb.a, pb.b
    for k, v in enumerate(pb.p):
        s.p[k] = v
    s.tau_u, s.tau_p, s.omega = pb.tau_u, pb.tau_p, pb.omega
    s.precond, s.tol, s.tol_kind, s.max_iter = _PC[pb.precond], pb.tol, _TOL[pb.tol_kind], pb.max_iter
    s.nz, s.lz = pb.nz, pb.lz
    s.shift = pb.shift
    return s


def _arr(x, pb=None):
    a = np.ascontiguousarray(x, dtype=np.float64)
    if pb is not None:
        a = a.reshape(pb.shape)
    return a


def _ptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def residual(pb, U, Uk):
    U, Uk = _arr(U, pb), _arr(Uk, pb)
    W = np.empty(pb.shape)
    load().rdo_residual(ctypes.byref(_problem(pb)), _ptr(U), _ptr(Uk), _ptr(W))
    return W


def grad_F_T(pb, U, Pt):
    U, Pt = _arr(U, pb), _arr(Pt, pb)
    g = np.empty(pb.shape)
    load().rdo_grad_F_T(ctypes.byref(_problem(pb)), _ptr(U), _ptr(Pt), _ptr(g))
    return g


def ghat(pb):
    g = np.empty(pb.shape)
    load().rdo_ghat(ctypes.byref(_problem(pb)), _ptr(g))
    return g


def apply_ginv(pb, W):
    _transform_sides(pb)
    W = _arr(W, pb)
    Y = np.empty(pb.shape)
    load().rdo_apply_ginv(ctypes.byref(_problem(pb)), _ptr(W), _ptr(Y))
    return Y


def pdhg_step(pb, Uk, history=False):
    """As rd_oracle.pdhg_step: (U, {iterations, status, residual[, history]})."""
    _transform_sides(pb)
    Uk = _arr(Uk, pb)
    U = np.empty(pb.shape)
    it, st, r = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
    cap = pb.max_iter + 1 if history else 0
    hist = np.empty(max(cap, 1))
    load().rdo_pdhg_step(ctypes.byref(_problem(pb)), _ptr(Uk), _ptr(U), ctypes.byref(it), ctypes.byref(st),
                         ctypes.byref(r), _ptr(hist) if history else None, cap)
    info = {"iterations": it.value, "status": _STATUS[st.value], "residual": r.value}
    if history:
        info["history"] = hist[:min(it.value + 1, cap)].copy()
    return U, info


def solve(pb, u0, nsteps, history=False):
    U = _arr(u0, pb).copy()
    infos = []
    for _ in range(nsteps):
        U, info = pdhg_step(pb, U, history=history)
        infos.append(info)
        if info["status"] != OK:
            break
    return U, infos


def fft(x, inverse=False):
    """Unnormalised complex DFT (testing hook of the C++ transform)."""
    z = np.ascontiguousarray(np.asarray(x, dtype=np.complex128)).copy()
    load().rdo_fft(z.view(np.float64).ctypes.data_as(ctypes.POINTER(ctypes.c_double)), len(z), 1 if inverse else -1)
    return z


def dct2(x):
    x = _arr(x)
    X = np.empty_like(x)
    load().rdo_dct2(_ptr(x), _ptr(X), len(x))
    return X


def dct3(X):
    X = _arr(X)
    x = np.empty_like(X)
    load().rdo_dct3(_ptr(X), _ptr(x), len(X))
    return x
