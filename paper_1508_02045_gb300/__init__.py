"""Python binding of libhom (include/hom.h): argument marshalling only.

Every step of the method runs in the CUDA library; this module converts NumPy arrays and torch
CUDA tensors to the plain pointers and sizes of the C ABI, and raises on any non-zero status.
The library must have been built (``paper_1508_02045_gb300.build.build()``); importing this
module without it fails loudly: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhom.so")

HOM_OK, HOM_ERR_INVALID, HOM_ERR_OOM, HOM_ERR_UNSUPPORTED, HOM_ERR_NOT_CONVERGED, HOM_ERR_CUDA, \
    HOM_ERR_TIMEOUT, HOM_ERR_SCRATCH = range(8)
HOM_STATIC_SCRATCH_BYTES = 64 * 1024 * 1024
HOM_APPROX, HOM_EXACT = 0, 1
HOM_RICHARDSON, HOM_CG, HOM_CHEBYSHEV, HOM_EYRE_MILTON = range(4)
HOM_FP64, HOM_FP32_REFINED = 0, 1
HOM_A_PHASE, HOM_A_SCALAR, HOM_A_FOURIER, HOM_A_STIFFNESS = range(4)
HOM_STOP_DEFAULT, HOM_STOP_RESIDUAL, HOM_STOP_INCREMENT = range(3)
HOM_OP_AFFINE, HOM_OP_LINEAR, HOM_OP_PROJECT, HOM_OP_EM = range(4)
HOM_OP_FP32 = 16
HOM_OP_X_HOST, HOM_OP_Y_HOST = 32, 64
HOM_OUT_HOST, HOM_OUT_NGRID = 1, 2

SOLVERS = {"richardson": HOM_RICHARDSON, "cg": HOM_CG, "chebyshev": HOM_CHEBYSHEV,
           "eyre_milton": HOM_EYRE_MILTON}

EXPORTED = ["hom_create", "hom_grid", "hom_bounds", "hom_apply", "hom_solve", "hom_energy",
            "hom_prolongate", "hom_bound", "hom_destroy", "hom_strerror", "hom_kernel_launches",
            "hom_profile_enable", "hom_profile_read", "hom_solve_begin", "hom_solve_iterate",
            "hom_solve_end", "hom_apply_static", "hom_batch_create", "hom_batch_iterate",
            "hom_batch_destroy", "hom_server_create", "hom_server_submit", "hom_server_step",
            "hom_server_poll", "hom_server_status", "hom_server_destroy", "hom_autotune",
            "hom_solve_history", "hom_solve_current", "hom_solve_nonconformity", "hom_restrict",
            "hom_measure_fp64", "hom_debug_fail_alloc", "hom_debug_tma_stall", "hom_set_plan",
            "hom_solve_snapshot_size", "hom_solve_snapshot", "hom_solve_restore"]
PASS_KINDS = ["line_fwd", "strided", "proj", "line_inv", "vector", "pot_inv", "pot_line",
              "pot_fwd"]


class hom_material(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("data", ctypes.c_void_p), ("index_bytes", ctypes.c_int),
                ("table", ctypes.POINTER(ctypes.c_double)), ("nphase", ctypes.c_int),
                ("data_on_device", ctypes.c_int), ("cA", ctypes.c_double), ("CA", ctypes.c_double),
                ("M", ctypes.c_int * 3)]


class hom_opts(ctypes.Structure):
    _fields_ = [("maxit", ctypes.c_int), ("fixed_iters", ctypes.c_int), ("stop", ctypes.c_int),
                ("cA", ctypes.c_double), ("CA", ctypes.c_double), ("inner_tol", ctypes.c_double),
                ("check_every", ctypes.c_int), ("out_flags", ctypes.c_int),
                ("inner_form", ctypes.c_int)]


class hom_stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("matvecs", ctypes.c_int),
                ("inner_iterations", ctypes.c_int), ("converged", ctypes.c_int),
                ("residual", ctypes.c_double), ("true_residual", ctypes.c_double),
                ("time_ms", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class hom_request(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int), ("N", ctypes.c_int * 3), ("material", hom_material),
                ("integration", ctypes.c_int), ("precision", ctypes.c_int),
                ("E", ctypes.c_double * 6), ("solver", ctypes.c_int), ("tol", ctypes.c_double),
                ("opts", hom_opts)]


class hom_result(ctypes.Structure):
    _fields_ = [("id", ctypes.c_longlong), ("status", ctypes.c_int), ("AH_EE", ctypes.c_double),
                ("flux", ctypes.c_double * 6), ("stats", hom_stats),
                ("latency_ms", ctypes.c_double), ("queue_ms", ctypes.c_double)]


class hom_tune_report(ctypes.Structure):
    _fields_ = [("rmax64", ctypes.c_int), ("smem_kb64", ctypes.c_int), ("ms64", ctypes.c_double),
                ("rmax32", ctypes.c_int), ("smem_kb32", ctypes.c_int), ("ms32", ctypes.c_double),
                ("threads64", ctypes.c_int), ("threads32", ctypes.c_int), ("two_line32", ctypes.c_int)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libhom.so is not built ({LIB_PATH}); run paper_1508_02045_gb300.build.build()")
    lib = ctypes.CDLL(LIB_PATH)
    vp, ip, dp = ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_double)
    lib.hom_create.argtypes = [ip, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(hom_material), ip, ip,
                               vp, ctypes.POINTER(vp)]
    lib.hom_grid.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_longlong)]
    lib.hom_bounds.argtypes = [vp, dp, dp]
    lib.hom_apply.argtypes = [vp, ip, dp, vp, vp]
    lib.hom_solve.argtypes = [vp, dp, ip, ctypes.c_double, ctypes.POINTER(hom_opts), vp, dp, dp,
                              ctypes.POINTER(hom_stats)]
    lib.hom_energy.argtypes = [vp, dp, vp, dp, dp]
    lib.hom_apply_static.argtypes = [ip, ctypes.POINTER(ctypes.c_int), vp, ip, dp, ip, ip, dp, vp,
                                     vp, vp]
    lib.hom_autotune.argtypes = [vp, ip, ctypes.POINTER(hom_tune_report)]
    lib.hom_set_plan.argtypes = [vp, ctypes.POINTER(hom_tune_report)]
    lib.hom_batch_create.argtypes = [ctypes.POINTER(vp), ip, ctypes.POINTER(vp)]
    lib.hom_batch_iterate.argtypes = [vp, ip, ip, ctypes.POINTER(ctypes.c_int)]
    lib.hom_batch_destroy.argtypes = [vp]
    lib.hom_batch_destroy.restype = None
    lib.hom_server_create.argtypes = [ctypes.c_size_t, ip, vp, ctypes.POINTER(vp)]
    lib.hom_server_submit.argtypes = [vp, ctypes.POINTER(hom_request), ctypes.POINTER(ctypes.c_longlong)]
    lib.hom_server_step.argtypes = [vp, ip]
    lib.hom_server_poll.argtypes = [vp, ctypes.POINTER(hom_result), ip, ctypes.POINTER(ctypes.c_int)]
    lib.hom_server_status.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                      ctypes.POINTER(ctypes.c_size_t)]
    lib.hom_server_destroy.argtypes = [vp]
    lib.hom_server_destroy.restype = None
    lib.hom_solve_begin.argtypes = [vp, dp, ip, ctypes.c_double, ctypes.POINTER(hom_opts)]
    lib.hom_solve_iterate.argtypes = [vp, ip, ctypes.POINTER(ctypes.c_int)]
    lib.hom_solve_end.argtypes = [vp, vp, dp, dp, ctypes.POINTER(hom_stats)]
    lib.hom_solve_history.argtypes = [vp, dp, ip, ctypes.POINTER(ctypes.c_int)]
    lib.hom_solve_current.argtypes = [vp, vp]
    lib.hom_solve_nonconformity.argtypes = [vp, dp]
    lib.hom_solve_snapshot_size.argtypes = [vp, ctypes.POINTER(ctypes.c_size_t)]
    lib.hom_solve_snapshot.argtypes = [vp, vp, ctypes.c_size_t]
    lib.hom_solve_restore.argtypes = [vp, vp, ctypes.c_size_t]
    lib.hom_prolongate.argtypes = [vp, vp, vp, vp]
    lib.hom_restrict.argtypes = [vp, vp, vp]
    lib.hom_measure_fp64.argtypes = [ip, ip, vp, dp, dp]
    lib.hom_debug_fail_alloc.argtypes = [ip]
    lib.hom_debug_tma_stall.argtypes = [ip]
    lib.hom_bound.argtypes = [vp, vp, dp, vp, dp]
    lib.hom_destroy.argtypes = [vp]
    lib.hom_destroy.restype = None
    lib.hom_strerror.argtypes = [ip]
    lib.hom_strerror.restype = ctypes.c_char_p
    lib.hom_kernel_launches.argtypes = []
    lib.hom_kernel_launches.restype = ctypes.c_longlong
    lib.hom_profile_enable.argtypes = [ip]
    lib.hom_profile_read.argtypes = [dp, ctypes.POINTER(ctypes.c_longlong), ip]
    for name in EXPORTED:
        if name not in ("hom_destroy", "hom_strerror", "hom_kernel_launches", "hom_batch_destroy",
                        "hom_server_destroy"):
            getattr(lib, name).restype = ctypes.c_int
    return lib


_lib = _load()


class HomError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__(f"{where}: {hom_strerror(status)} (status {status})")


def _check(status, where):
    if status != HOM_OK:
        raise HomError(status, where)
    return status


def _dvec(values):
    arr = (ctypes.c_double * len(values))(*[float(v) for v in values])
    return arr


def _ptr(t):
    """Device pointer of a torch CUDA tensor (None -> NULL)."""
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def _host_or_dev(t):
    """(pointer, on_host) of a contiguous float64 torch tensor (CUDA or CPU, pinned or not) or
    NumPy array."""
    if isinstance(t, np.ndarray):
        if not t.flags["C_CONTIGUOUS"] or t.dtype != np.float64:
            raise ValueError("expected a C-contiguous float64 array")
        return ctypes.c_void_p(t.ctypes.data), True
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr()), not t.is_cuda


def _stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


# ------------------------------------------------------------------------------------------
# the C entry points under their own names
# ------------------------------------------------------------------------------------------

def hom_strerror(status: int) -> str:
    return _lib.hom_strerror(int(status)).decode()


def hom_kernel_launches() -> int:
    return int(_lib.hom_kernel_launches())


def hom_profile_enable(on: bool):
    return _check(_lib.hom_profile_enable(1 if on else 0), "hom_profile_enable")


def hom_profile_read():
    n = len(PASS_KINDS)
    ms = (ctypes.c_double * n)()
    cnt = (ctypes.c_longlong * n)()
    _check(_lib.hom_profile_read(ms, cnt, n), "hom_profile_read")
    return {k: (ms[i], cnt[i]) for i, k in enumerate(PASS_KINDS)}


def hom_create(d, N, material: hom_material, integration=HOM_APPROX, precision=HOM_FP64,
               stream=None):
    vals = [int(v) for v in N] + [1] * max(0, 3 - len(N))
    Narr = (ctypes.c_int * len(vals))(*vals)
    out = ctypes.c_void_p()
    st = _stream() if stream is None else ctypes.c_void_p(stream)
    _check(_lib.hom_create(int(d), Narr, ctypes.byref(material), int(integration), int(precision),
                           st, ctypes.byref(out)), "hom_create")
    return out


def hom_grid(P):
    M = (ctypes.c_int * 3)()
    n = ctypes.c_longlong()
    _check(_lib.hom_grid(P, M, ctypes.byref(n)), "hom_grid")
    return list(M), n.value


def hom_bounds(P):
    a, b = ctypes.c_double(), ctypes.c_double()
    _check(_lib.hom_bounds(P, ctypes.byref(a), ctypes.byref(b)), "hom_bounds")
    return a.value, b.value


def hom_apply(P, op, E, x, y):
    """x, y: CUDA tensors, or host tensors / arrays (flagged HOM_OP_X_HOST / HOM_OP_Y_HOST)."""
    Ep = _dvec(E) if E is not None else None
    xp, xh = _host_or_dev(x)
    yp, yh = _host_or_dev(y)
    flags = (HOM_OP_X_HOST if xh else 0) | (HOM_OP_Y_HOST if yh else 0)
    return _check(_lib.hom_apply(P, int(op) | flags, Ep, xp, yp), "hom_apply")


def hom_restrict(P, x, y):
    return _check(_lib.hom_restrict(P, _ptr(x), _ptr(y)), "hom_restrict")


def hom_measure_fp64(kind=0, iters=2000, stream=None):
    """(milliseconds, floating-point operations) of one timed FP64 throughput wave."""
    ms, ops = ctypes.c_double(), ctypes.c_double()
    st = _stream() if stream is None else ctypes.c_void_p(stream)
    _check(_lib.hom_measure_fp64(int(kind), int(iters), st, ctypes.byref(ms), ctypes.byref(ops)),
           "hom_measure_fp64")
    return ms.value, ops.value


def hom_debug_fail_alloc(n):
    return _check(_lib.hom_debug_fail_alloc(int(n)), "hom_debug_fail_alloc")


def hom_debug_tma_stall(on):
    return _check(_lib.hom_debug_tma_stall(int(bool(on))), "hom_debug_tma_stall")


def hom_solve(P, E, solver, tol, opts: hom_opts | None = None, x=None, allow_not_converged=False):
    AH = ctypes.c_double()
    d = len(E)
    flux = (ctypes.c_double * 6)()
    stats = hom_stats()
    xp = None
    if x is not None:
        xp, xh = _host_or_dev(x)
        if xh:  # a host corrector output is flagged in the options
            opts = make_opts() if opts is None else opts
            opts.out_flags |= HOM_OUT_HOST
    o = ctypes.byref(opts) if opts is not None else None
    st = _lib.hom_solve(P, _dvec(E), int(solver), float(tol), o, xp, ctypes.byref(AH), flux,
                        ctypes.byref(stats))
    if not (st == HOM_OK or (allow_not_converged and st == HOM_ERR_NOT_CONVERGED)):
        raise HomError(st, "hom_solve")
    return AH.value, [flux[i] for i in range(d)], stats.as_dict(), st


def hom_apply_static(d, N, phase_dev, table, op, E, x, y, stream=None):
    """Allocation-free operator application (see include/hom.h): phase_dev is a CUDA uint8 /
    uint16 tensor, table a host (nphase, d, d) array; x, y CUDA float64 fields."""
    vals = [int(v) for v in N] + [1] * max(0, 3 - len(N))
    Narr = (ctypes.c_int * len(vals))(*vals)
    table = np.ascontiguousarray(table, dtype=np.float64)
    Ep = _dvec(E) if E is not None else None
    st = _stream() if stream is None else ctypes.c_void_p(stream)
    return _check(_lib.hom_apply_static(int(d), Narr, _ptr(phase_dev), phase_dev.element_size(),
                                        table.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                        int(table.shape[0]), int(op), Ep, _ptr(x), _ptr(y), st),
                  "hom_apply_static")


def hom_solve_begin(P, E, solver, tol, opts: hom_opts | None = None):
    o = ctypes.byref(opts) if opts is not None else None
    return _check(_lib.hom_solve_begin(P, _dvec(E), int(solver), float(tol), o), "hom_solve_begin")


def hom_solve_iterate(P, iterations, poll=False):
    done = ctypes.c_int(0)
    _check(_lib.hom_solve_iterate(P, int(iterations), ctypes.byref(done) if poll else None),
           "hom_solve_iterate")
    return bool(done.value) if poll else None


def hom_solve_history(P, cap=1 << 20):
    """The per-iteration stopping quantity of the current or last solve (numpy array)."""
    import numpy as np
    count = ctypes.c_int(0)
    _check(_lib.hom_solve_history(P, None, 0, ctypes.byref(count)), "hom_solve_history")
    n = min(count.value, int(cap))
    buf = (ctypes.c_double * max(n, 1))()
    _check(_lib.hom_solve_history(P, buf, n, ctypes.byref(count)), "hom_solve_history")
    return np.array(buf[:n], dtype=np.float64)


def hom_solve_current(P, x):
    """Write the current iterate of the active session into the device tensor x."""
    return _check(_lib.hom_solve_current(P, _ptr(x)), "hom_solve_current")


def hom_solve_nonconformity(P):
    """Non-conformity of the current iterate of the active session (Section 4.4)."""
    v = ctypes.c_double()
    _check(_lib.hom_solve_nonconformity(P, ctypes.byref(v)), "hom_solve_nonconformity")
    return v.value


def hom_solve_snapshot(P):
    """The active FP64 session of P as host bytes (a numpy uint8 array)."""
    n = ctypes.c_size_t()
    _check(_lib.hom_solve_snapshot_size(P, ctypes.byref(n)), "hom_solve_snapshot_size")
    buf = np.empty(n.value, dtype=np.uint8)
    _check(_lib.hom_solve_snapshot(P, buf.ctypes.data, n.value), "hom_solve_snapshot")
    return buf


def hom_solve_restore(P, snapshot):
    """Restore a snapshot (from hom_solve_snapshot) into P's active session."""
    buf = np.ascontiguousarray(snapshot, dtype=np.uint8)
    return _check(_lib.hom_solve_restore(P, buf.ctypes.data, buf.nbytes), "hom_solve_restore")


def hom_solve_end(P, d, x=None, allow_not_converged=False):
    AH = ctypes.c_double()
    flux = (ctypes.c_double * 6)()
    stats = hom_stats()
    st = _lib.hom_solve_end(P, _ptr(x), ctypes.byref(AH), flux, ctypes.byref(stats))
    if not (st == HOM_OK or (allow_not_converged and st == HOM_ERR_NOT_CONVERGED)):
        raise HomError(st, "hom_solve_end")
    return AH.value, [flux[i] for i in range(d)], stats.as_dict(), st


def hom_autotune(P, reps=3):
    rep = hom_tune_report()
    _check(_lib.hom_autotune(P, int(reps), ctypes.byref(rep)), "hom_autotune")
    return {k: getattr(rep, k) for k, _ in rep._fields_}


def hom_set_plan(P, plan: dict):
    """Re-plan P with a launch plan given as hom_autotune's report (a dict of its fields)."""
    rep = hom_tune_report()
    for k, _ in rep._fields_:
        if k in plan:
            setattr(rep, k, type(getattr(rep, k))(plan[k]))
    return _check(_lib.hom_set_plan(P, ctypes.byref(rep)), "hom_set_plan")


def hom_batch_create(problems):
    arr = (ctypes.c_void_p * len(problems))(*[p.value if isinstance(p, ctypes.c_void_p) else p for p in problems])
    out = ctypes.c_void_p()
    _check(_lib.hom_batch_create(arr, len(problems), ctypes.byref(out)), "hom_batch_create")
    return out


def hom_batch_iterate(B, iterations, use_graph=True, poll=False):
    done = ctypes.c_int(0)
    _check(_lib.hom_batch_iterate(B, int(iterations), 1 if use_graph else 0,
                                  ctypes.byref(done) if poll else None), "hom_batch_iterate")
    return bool(done.value) if poll else None


def hom_batch_destroy(B):
    if B:
        _lib.hom_batch_destroy(B)


def hom_server_create(hbm_budget_bytes, max_batch=16, stream=0):
    out = ctypes.c_void_p()
    _check(_lib.hom_server_create(int(hbm_budget_bytes), int(max_batch), ctypes.c_void_p(stream),
                                  ctypes.byref(out)), "hom_server_create")
    return out


def make_request(d, N, material, E, solver, tol, integration=HOM_APPROX, precision=HOM_FP64,
                 opts=None):
    r = hom_request()
    r.d = d
    for i, v in enumerate(N):
        r.N[i] = int(v)
    r.material = material
    r.integration, r.precision = integration, precision
    for i, v in enumerate(E):
        r.E[i] = float(v)
    r.solver, r.tol = int(solver), float(tol)
    if opts is not None:
        r.opts = opts
    r._keep = material
    return r


def hom_server_submit(S, request):
    rid = ctypes.c_longlong()
    _check(_lib.hom_server_submit(S, ctypes.byref(request), ctypes.byref(rid)), "hom_server_submit")
    return rid.value


def hom_server_step(S, iterations):
    return _check(_lib.hom_server_step(S, int(iterations)), "hom_server_step")


def hom_server_poll(S, max_results=256):
    buf = (hom_result * max_results)()
    n = ctypes.c_int()
    _check(_lib.hom_server_poll(S, buf, max_results, ctypes.byref(n)), "hom_server_poll")
    out = []
    for i in range(n.value):
        r = buf[i]
        out.append({"id": r.id, "status": r.status, "AH_EE": r.AH_EE, "flux": list(r.flux),
                    "stats": r.stats.as_dict(), "latency_ms": r.latency_ms, "queue_ms": r.queue_ms})
    return out


def hom_server_status(S):
    a, q, b = ctypes.c_int(), ctypes.c_int(), ctypes.c_size_t()
    _check(_lib.hom_server_status(S, ctypes.byref(a), ctypes.byref(q), ctypes.byref(b)), "hom_server_status")
    return a.value, q.value, b.value


def hom_server_destroy(S):
    if S:
        _lib.hom_server_destroy(S)


def hom_energy(P, E, x=None):
    en = ctypes.c_double()
    flux = (ctypes.c_double * 6)()
    _check(_lib.hom_energy(P, _dvec(E), _ptr(x), ctypes.byref(en), flux), "hom_energy")
    return en.value, [flux[i] for i in range(len(E))]


def hom_prolongate(coarse, fine, x, y):
    return _check(_lib.hom_prolongate(coarse, fine, _ptr(x), _ptr(y)), "hom_prolongate")


def hom_bound(gani, ga, E, x):
    ue = ctypes.c_double()
    _check(_lib.hom_bound(gani, ga, _dvec(E), _ptr(x), ctypes.byref(ue)), "hom_bound")
    return ue.value


def hom_destroy(P):
    if P:
        _lib.hom_destroy(P)


# ------------------------------------------------------------------------------------------
# material descriptors (marshalling of host arrays; the arrays must outlive hom_create)
# ------------------------------------------------------------------------------------------

def phase_material(phase: np.ndarray, table: np.ndarray, cA=0.0, CA=0.0, M=None):
    """Phase image + table. With HOM_EXACT (scalar tables): the voxel-wise constant coefficient,
    integrated exactly on the grid M (default 2N - 1)."""
    phase = np.ascontiguousarray(phase)
    if phase.dtype not in (np.uint8, np.uint16):
        raise ValueError("phase image must be uint8 or uint16")
    table = np.ascontiguousarray(table, dtype=np.float64)
    m = hom_material()
    m.kind = HOM_A_PHASE
    m.data = phase.ctypes.data
    m.index_bytes = phase.dtype.itemsize
    m.table = table.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    m.nphase = table.shape[0]
    m.cA, m.CA = cA, CA
    if M is not None:
        for i, v in enumerate(M):
            m.M[i] = int(v)
    m._keep = (phase, table)
    return m


def stiffness_material(phase: np.ndarray, table: np.ndarray, cA=0.0, CA=0.0):
    """Linear elasticity: phase image + (nphase, nc, nc) Mandel stiffness matrices,
    nc = d (d + 1) / 2 (fields then have nc components, see include/hom.h)."""
    phase = np.ascontiguousarray(phase)
    if phase.dtype not in (np.uint8, np.uint16):
        raise ValueError("phase image must be uint8 or uint16")
    table = np.ascontiguousarray(table, dtype=np.float64)
    m = hom_material()
    m.kind = HOM_A_STIFFNESS
    m.data = phase.ctypes.data
    m.index_bytes = phase.dtype.itemsize
    m.table = table.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    m.nphase = table.shape[0]
    m.cA, m.CA = cA, CA
    m._keep = (phase, table)
    return m


def scalar_material(a: np.ndarray, cA=0.0, CA=0.0, M=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    m = hom_material()
    m.kind = HOM_A_SCALAR
    m.data = a.ctypes.data
    m.cA, m.CA = cA, CA
    if M is not None:
        for i, v in enumerate(M):
            m.M[i] = int(v)
    m._keep = (a,)
    return m


def fourier_material(Ahat: np.ndarray, cA, CA, M=None):
    c = np.ascontiguousarray(Ahat, dtype=np.complex128)
    m = hom_material()
    m.kind = HOM_A_FOURIER
    m.data = c.ctypes.data
    m.cA, m.CA = cA, CA
    if M is not None:
        for i, v in enumerate(M):
            m.M[i] = int(v)
    m._keep = (c,)
    return m


def make_opts(maxit=0, fixed_iters=0, stop=HOM_STOP_DEFAULT, cA=0.0, CA=0.0, inner_tol=0.0,
              check_every=0, out_flags=0, inner_form=0):
    o = hom_opts()
    o.maxit, o.fixed_iters, o.stop = maxit, fixed_iters, stop
    o.cA, o.CA, o.inner_tol, o.check_every = cA, CA, inner_tol, check_every
    o.out_flags, o.inner_form = out_flags, inner_form
    return o


class Problem:
    """Owning wrapper of a hom_problem handle."""

    def __init__(self, d, N, material, integration=HOM_APPROX, precision=HOM_FP64):
        self.d = d
        # components of a field: d, or d (d + 1) / 2 for strains (elasticity)
        self.nc = d * (d + 1) // 2 if material.kind == HOM_A_STIFFNESS else d
        self.N = tuple(N)
        self.material = material
        self.h = hom_create(d, N, material, integration, precision)
        self.grid, self.nodes = hom_grid(self.h)
        self.grid = tuple(self.grid[:d])

    def field(self, dtype=None):
        import torch
        return torch.zeros((self.nc,) + self.grid, dtype=dtype or torch.float64, device="cuda")

    def close(self):
        if self.h:
            hom_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
