"""ctypes binding of ``librd_pdhg.so`` (argument marshalling only).

The functions carry the C names of ``include/rd_pdhg.h``.  ``Solver`` is a thin convenience
wrapper that maps a ``workloads.Problem`` record onto the C structs and passes torch tensors by
``data_ptr()`` together with torch's current CUDA stream; every step of the method runs in the
library's CUDA kernels.  Importing this module never falls back to any other implementation:
if the library is missing, ``load()`` raises.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librd_pdhg.so")

RD_OK, RD_ERR_INVALID_ARG, RD_ERR_UNSUPPORTED, RD_ERR_OOM, RD_ERR_CUDA = 0, 1, 2, 3, 4
RD_ERR_NOT_CONVERGED, RD_ERR_DIVERGED, RD_ERR_TIMEOUT, RD_ERR_BUSY = 5, 6, 7, 8
BC = {"periodic": 0, "neumann": 1}
OP = {"laplacian": 0, "neg_biharmonic": 1, "functionalized": 2}
KIND = {"none": 0, "allen_cahn": 1, "ch_implicit": 2, "ch_split": 3, "gray_scott": 4, "schnakenberg": 5,
        "fch": 6}
PRECOND = {"none": 0, "linear": 1, "stabilized": 2}
TOL = {"res_abs": 0, "f_rel": 1}
PREC = {"fp64": 0, "fp32_dc": 1}

EXPORTS = ("rd_opts_default", "rd_pdhg_create", "rd_pdhg_step", "rd_pdhg_solve", "rd_pdhg_solve_host",
           "rd_pdhg_residual", "rd_pdhg_apply_precond", "rd_pdhg_get_stats", "rd_pdhg_reset_stats",
           "rd_pdhg_destroy", "rd_status_string", "rd_last_error", "rd_apply_precond_static",
           "rd_pdhg_set_dt", "rd_pdhg_solve_adaptive",
           "rd_batch_create", "rd_batch_submit", "rd_batch_poll", "rd_batch_get_stats", "rd_batch_destroy")


class rd_grid(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int), ("n", ctypes.c_int * 3), ("length", ctypes.c_double * 3)]


class rd_reaction(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("ncomp", ctypes.c_int), ("a", ctypes.c_double),
                ("b", ctypes.c_double), ("p", ctypes.c_double * 6)]


class rd_precond(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("s", ctypes.c_double)]


class rd_opts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("tol_kind", ctypes.c_int), ("max_iter", ctypes.c_int),
                ("omega", ctypes.c_double), ("precision", ctypes.c_int),
                ("dc_inner_rtol", ctypes.c_double), ("dc_max_outer", ctypes.c_int),
                ("graph_k", ctypes.c_int), ("band_rows", ctypes.c_int), ("col_width", ctypes.c_int),
                ("upd_rows", ctypes.c_int),
                ("profile", ctypes.c_int), ("fft_buffers", ctypes.c_int), ("solve_loop", ctypes.c_int),
                ("fft_unrolled", ctypes.c_int), ("autotune", ctypes.c_int), ("dc_stall_window", ctypes.c_int),
                ("fused_update", ctypes.c_int), ("small_solve", ctypes.c_int)]


class rd_stats(ctypes.Structure):
    _fields_ = [("kernel_launches", ctypes.c_longlong), ("graph_launches", ctypes.c_longlong),
                ("pdhg_iterations", ctypes.c_longlong), ("residual_passes", ctypes.c_longlong),
                ("host_syncs", ctypes.c_longlong), ("kernel_ms", ctypes.c_double * 3),
                ("kernel_samples", ctypes.c_longlong * 3), ("plan_band_rows", ctypes.c_int),
                ("plan_col_width", ctypes.c_int), ("plan_upd_rows", ctypes.c_int),
                ("fused_update", ctypes.c_int), ("small_solve", ctypes.c_int), ("line_kernels", ctypes.c_int)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["kernel_ms"] = list(self.kernel_ms)
        d["kernel_samples"] = list(self.kernel_samples)
        return d


class rd_step_info(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("outer_rounds", ctypes.c_int), ("converged", ctypes.c_int),
                ("status", ctypes.c_int), ("residual", ctypes.c_double), ("mass", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class rd_adapt(ctypes.Structure):
    _fields_ = [("t_end", ctypes.c_double), ("n_hi", ctypes.c_int), ("n_lo", ctypes.c_int),
                ("eta", ctypes.c_double), ("max_attempts", ctypes.c_int)]


class rd_adapt_step(ctypes.Structure):
    _fields_ = [("t", ctypes.c_double), ("dt", ctypes.c_double), ("iterations", ctypes.c_int),
                ("outer_rounds", ctypes.c_int), ("status", ctypes.c_int), ("accepted", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class rd_request(ctypes.Structure):
    _fields_ = [("grid", rd_grid), ("bc", ctypes.c_int), ("op", ctypes.c_int), ("reaction", rd_reaction),
                ("dt", ctypes.c_double), ("tau", ctypes.c_double), ("sigma", ctypes.c_double),
                ("tol", ctypes.c_double), ("tol_kind", ctypes.c_int), ("nsteps", ctypes.c_int),
                ("u0_host", ctypes.c_void_p), ("tag", ctypes.c_uint64)]


class rd_result(ctypes.Structure):
    _fields_ = [("id", ctypes.c_uint64), ("tag", ctypes.c_uint64), ("status", ctypes.c_int),
                ("steps", ctypes.c_int), ("iterations", ctypes.c_longlong), ("outer_rounds", ctypes.c_int),
                ("residual", ctypes.c_double), ("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double),
                ("t_done", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class rd_batch_stats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_longlong) for k in ("submitted", "admitted", "completed", "graph_launches",
                                                  "queued", "arena_free_bytes")]


_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load the library (built by ``build.build()``) and declare the C signatures."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("librd_pdhg.so not built: run paper_2305_03945_gb300.build.build() (%s)" % path)
    lib = ctypes.CDLL(path)
    P = ctypes.POINTER
    vp = ctypes.c_void_p
    lib.rd_opts_default.argtypes = [P(rd_opts)]
    lib.rd_opts_default.restype = None
    lib.rd_pdhg_create.argtypes = [P(vp), P(rd_grid), ctypes.c_int, ctypes.c_int, P(rd_reaction),
                                   ctypes.c_double, ctypes.c_double, ctypes.c_double, P(rd_precond),
                                   P(rd_opts), vp]
    lib.rd_pdhg_create.restype = ctypes.c_int
    lib.rd_pdhg_step.argtypes = [vp, vp, vp, P(rd_step_info)]
    lib.rd_pdhg_step.restype = ctypes.c_int
    lib.rd_pdhg_solve.argtypes = [vp, vp, ctypes.c_int, P(rd_step_info)]
    lib.rd_pdhg_solve.restype = ctypes.c_int
    lib.rd_pdhg_solve_host.argtypes = [vp, vp, ctypes.c_int, P(rd_step_info)]
    lib.rd_pdhg_solve_host.restype = ctypes.c_int
    lib.rd_pdhg_residual.argtypes = [vp, vp, vp, vp]
    lib.rd_pdhg_residual.restype = ctypes.c_int
    lib.rd_pdhg_apply_precond.argtypes = [vp, vp, vp]
    lib.rd_pdhg_apply_precond.restype = ctypes.c_int
    lib.rd_pdhg_get_stats.argtypes = [vp, P(rd_stats)]
    lib.rd_pdhg_get_stats.restype = ctypes.c_int
    lib.rd_pdhg_reset_stats.argtypes = [vp]
    lib.rd_pdhg_reset_stats.restype = ctypes.c_int
    lib.rd_pdhg_set_dt.argtypes = [vp, ctypes.c_double]
    lib.rd_pdhg_set_dt.restype = ctypes.c_int
    lib.rd_pdhg_solve_adaptive.argtypes = [vp, vp, P(rd_adapt), P(rd_adapt_step), ctypes.c_int,
                                           P(ctypes.c_int), P(ctypes.c_double)]
    lib.rd_pdhg_solve_adaptive.restype = ctypes.c_int
    lib.rd_pdhg_destroy.argtypes = [vp]
    lib.rd_pdhg_destroy.restype = None
    lib.rd_apply_precond_static.argtypes = [P(rd_grid), ctypes.c_int, ctypes.c_int, P(rd_reaction),
                                            ctypes.c_double, vp, vp, vp]
    lib.rd_apply_precond_static.restype = ctypes.c_int
    lib.rd_batch_create.argtypes = [P(vp), ctypes.c_size_t, ctypes.c_int, P(rd_opts), vp]
    lib.rd_batch_create.restype = ctypes.c_int
    lib.rd_batch_submit.argtypes = [vp, P(rd_request), vp, P(ctypes.c_uint64)]
    lib.rd_batch_submit.restype = ctypes.c_int
    lib.rd_batch_poll.argtypes = [vp, P(rd_result), ctypes.c_int, P(ctypes.c_int), ctypes.c_double]
    lib.rd_batch_poll.restype = ctypes.c_int
    lib.rd_batch_get_stats.argtypes = [vp, P(rd_batch_stats)]
    lib.rd_batch_get_stats.restype = ctypes.c_int
    lib.rd_batch_destroy.argtypes = [vp]
    lib.rd_batch_destroy.restype = None
    lib.rd_status_string.argtypes = [ctypes.c_int]
    lib.rd_status_string.restype = ctypes.c_char_p
    lib.rd_last_error.argtypes = []
    lib.rd_last_error.restype = ctypes.c_char_p
    _lib = lib
    return lib


class RDError(RuntimeError):
    def __init__(self, status, detail):
        self.status = status
        super().__init__("%s: %s" % (load().rd_status_string(status).decode(), detail))


def _check(status, ok=(RD_OK,)):
    if status not in ok:
        raise RDError(status, load().rd_last_error().decode(errors="replace"))
    return status


def make_structs(pb, precision="fp64", graph_k=2, band_rows=0, col_width=0, dc_inner_rtol=None,
                 dc_max_outer=None, profile=0, fft_buffers=0, solve_loop="graph", fft_unrolled=1, autotune=0, upd_rows=0, dc_stall_window=None, fused_update=1,
                 small_solve=1):
    """C structs for a ``workloads.Problem``."""
    g = rd_grid()
    nz = getattr(pb, "nz", 1)
    g.ndim = 3 if nz > 1 else 2
    g.n[0], g.n[1], g.n[2] = pb.nx, pb.ny, nz
    g.length[0], g.length[1], g.length[2] = pb.lx, pb.ly, getattr(pb, "lz", 1.0)
    rx = rd_reaction()
    rx.kind = KIND[pb.kind]
    rx.ncomp = pb.ncomp
    rx.a, rx.b = pb.a, pb.b
    for k, v in enumerate(pb.p):
        rx.p[k] = v
    pc = rd_precond(PRECOND[pb.precond], getattr(pb, "shift", 0.0) if pb.precond == "stabilized" else 0.0)
    o = rd_opts()
    load().rd_opts_default(ctypes.byref(o))
    o.tol = pb.tol
    o.tol_kind = TOL[pb.tol_kind]
    o.max_iter = pb.max_iter
    o.omega = pb.omega
    o.precision = PREC[precision]
    o.graph_k = graph_k
    o.band_rows = band_rows
    o.col_width = col_width
    if dc_inner_rtol is not None:
        o.dc_inner_rtol = dc_inner_rtol
    if dc_max_outer is not None:
        o.dc_max_outer = dc_max_outer
    o.profile = profile
    o.fft_buffers = fft_buffers
    o.solve_loop = {"graph": 0, "host": 1}[solve_loop]
    o.fft_unrolled = fft_unrolled
    o.autotune = autotune
    o.upd_rows = upd_rows
    if dc_stall_window is not None:
        o.dc_stall_window = dc_stall_window
    o.fused_update = fused_update
    o.small_solve = small_solve
    return g, rx, pc, o


class Solver:
    """One ``rd_pdhg`` handle for a ``workloads.Problem``; tensors are float64 CUDA tensors of
    the problem's shape ([ncomp, ny, nx], or [ncomp, nz, ny, nx] on 3-D grids; contiguous)."""

    def __init__(self, pb, precision="fp64", stream=None, **opts):
        import torch
        lib = load()
        self.pb = pb
        self.precision = precision
        g, rx, pc, o = make_structs(pb, precision, **opts)
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        self._stream = stream
        h = ctypes.c_void_p()
        _check(lib.rd_pdhg_create(ctypes.byref(h), ctypes.byref(g), BC[pb.bc], OP[pb.op], ctypes.byref(rx),
                                  pb.dt, pb.tau_u, pb.tau_p, ctypes.byref(pc), ctypes.byref(o),
                                  ctypes.c_void_p(stream)))
        self.h = h

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            load().rd_pdhg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @staticmethod
    def _ptr(t):
        assert t.is_cuda and t.dtype.is_floating_point and t.is_contiguous()
        return ctypes.c_void_p(t.data_ptr())

    def step(self, u_n, u_np1, allow=(RD_OK,)):
        info = rd_step_info()
        s = load().rd_pdhg_step(self.h, self._ptr(u_n), self._ptr(u_np1), ctypes.byref(info))
        _check(s, allow)
        return info.as_dict()

    def solve(self, u, nsteps, allow=(RD_OK,)):
        infos = (rd_step_info * max(nsteps, 1))()
        s = load().rd_pdhg_solve(self.h, self._ptr(u), nsteps, infos)
        _check(s, allow)
        return [infos[k].as_dict() for k in range(nsteps)], s

    def solve_host(self, u_np, nsteps, allow=(RD_OK,)):
        """u_np: C-contiguous float64 numpy array (host); updated in place."""
        import numpy as np
        assert u_np.dtype == np.float64 and u_np.flags.c_contiguous
        infos = (rd_step_info * max(nsteps, 1))()
        s = load().rd_pdhg_solve_host(self.h, ctypes.c_void_p(u_np.ctypes.data), nsteps, infos)
        _check(s, allow)
        return [infos[k].as_dict() for k in range(nsteps)], s

    def set_dt(self, dt):
        _check(load().rd_pdhg_set_dt(self.h, dt))

    def solve_adaptive(self, u, t_end, n_hi, n_lo, eta, max_attempts=1000, allow=(RD_OK,)):
        """Adaptive time step size (Section 2.2) in place on u from t = 0 to t_end, with
        h_t^0 = the solver's dt.  Returns (log, t_reached, status)."""
        a = rd_adapt(t_end, n_hi, n_lo, eta, max_attempts)
        log = (rd_adapt_step * max_attempts)()
        n = ctypes.c_int()
        t = ctypes.c_double()
        s = load().rd_pdhg_solve_adaptive(self.h, self._ptr(u), ctypes.byref(a), log, max_attempts,
                                          ctypes.byref(n), ctypes.byref(t))
        _check(s, allow)
        return [log[k].as_dict() for k in range(min(n.value, max_attempts))], t.value, s

    def residual(self, u, uk, w):
        _check(load().rd_pdhg_residual(self.h, self._ptr(u), self._ptr(uk), self._ptr(w)))

    def stats(self):
        st = rd_stats()
        _check(load().rd_pdhg_get_stats(self.h, ctypes.byref(st)))
        return st.as_dict()

    def reset_stats(self):
        _check(load().rd_pdhg_reset_stats(self.h))

    def apply_precond(self, w, y):
        _check(load().rd_pdhg_apply_precond(self.h, self._ptr(w), self._ptr(y)))


class Batch:
    """Continuous-batching server of implicit-step runs (rd_batch_*).  Requests are
    ``workloads.Problem`` records plus a host float64 initial state and a step count; results
    come back through ``poll``, final states in the host arrays returned by ``submit``."""

    def __init__(self, hbm_budget_bytes, max_slots, graph_k=8, max_iter=10000, dc_inner_rtol=None,
                 dc_max_outer=None, stream=None, small_solve=1, autotune=1):
        import torch
        lib = load()
        o = rd_opts()
        lib.rd_opts_default(ctypes.byref(o))
        o.graph_k, o.max_iter = graph_k, max_iter
        o.small_solve = small_solve
        o.autotune = autotune
        if dc_max_outer is not None:
            o.dc_max_outer = dc_max_outer
        if dc_inner_rtol is not None:
            o.dc_inner_rtol = dc_inner_rtol
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        h = ctypes.c_void_p()
        _check(lib.rd_batch_create(ctypes.byref(h), int(hbm_budget_bytes), int(max_slots), ctypes.byref(o),
                                   ctypes.c_void_p(stream)))
        self.h = h
        self._keep = {}

    def submit(self, pb, u0, nsteps, tag=0):
        """Queue a run; returns (id, out) where out (host float64, the shape of u0) receives the
        final state when the run finishes."""
        import numpy as np
        g, rx, pc, o = make_structs(pb)
        r = rd_request()
        r.grid = g
        r.bc, r.op, r.reaction = BC[pb.bc], OP[pb.op], rx
        r.dt, r.tau, r.sigma = pb.dt, pb.tau_u, pb.tau_p
        r.tol, r.tol_kind, r.nsteps = pb.tol, TOL[pb.tol_kind], nsteps
        u0 = np.ascontiguousarray(u0, dtype=np.float64)
        out = np.empty_like(u0)
        r.u0_host = u0.ctypes.data
        r.tag = tag
        rid = ctypes.c_uint64()
        _check(load().rd_batch_submit(self.h, ctypes.byref(r), ctypes.c_void_p(out.ctypes.data), ctypes.byref(rid)))
        self._keep[rid.value] = out
        return rid.value, out

    def poll(self, cap=64, timeout=0.0):
        res = (rd_result * cap)()
        n = ctypes.c_int()
        _check(load().rd_batch_poll(self.h, res, cap, ctypes.byref(n), float(timeout)))
        out = [res[k].as_dict() for k in range(n.value)]
        for r in out:
            self._keep.pop(r["id"], None)
        return out

    def stats(self):
        st = rd_batch_stats()
        _check(load().rd_batch_get_stats(self.h, ctypes.byref(st)))
        return {k: getattr(st, k) for k, _ in st._fields_}

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            load().rd_batch_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
