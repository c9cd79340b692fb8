"""Python binding of libhubbard.so (include/hubbard.h): argument marshalling only.

Every computation runs in the CUDA library; this module converts torch
tensors to device pointers and the current torch stream to a cudaStream_t,
and raises HubError on a non-zero status.  There is no CPU fallback: if the
compiled library is missing, importing the binding's functions fails.
"""
import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libhubbard.so")

HUB_OK, HUB_EINVAL, HUB_ENOMEM, HUB_ECUDA, HUB_ENOTCONV, HUB_ETIMEOUT, HUB_EDEVICE, HUB_EPENDING = range(8)
HUB_F64, HUB_F32 = 0, 1
STATUS_NAMES = {0: "HUB_OK", 1: "HUB_EINVAL", 2: "HUB_ENOMEM", 3: "HUB_ECUDA", 4: "HUB_ENOTCONV",
                5: "HUB_ETIMEOUT", 6: "HUB_EDEVICE", 7: "HUB_EPENDING"}


class HubError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


class LanczosResult(ctypes.Structure):
    _fields_ = [("energy", ctypes.c_double), ("residual", ctypes.c_double), ("err_bound", ctypes.c_double),
                ("iters", ctypes.c_int32), ("status", ctypes.c_int32), ("breakdown", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class HubbardRequest(ctypes.Structure):
    _fields_ = [("ns", ctypes.c_int32), ("nup", ctypes.c_int32), ("ndn", ctypes.c_int32),
                ("n_bonds", ctypes.c_int32), ("bonds", ctypes.c_void_p), ("t", ctypes.c_double),
                ("U", ctypes.c_double), ("seed", ctypes.c_uint64)]


HOST_SOLVER = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_uint64, ctypes.POINTER(HubbardRequest),
                               ctypes.c_int, ctypes.POINTER(LanczosResult))


class ServerOpts(ctypes.Structure):
    _fields_ = [("hbm_budget", ctypes.c_double), ("small_lanes", ctypes.c_int32), ("big_lanes", ctypes.c_int32),
                ("small_max_dim", ctypes.c_int64), ("mid_max_dim", ctypes.c_int64), ("max_iters", ctypes.c_int32),
                ("batch_max", ctypes.c_int32), ("store_vectors", ctypes.c_int32), ("small_ctas", ctypes.c_int32),
                ("tol", ctypes.c_double), ("host_solver", HOST_SOLVER), ("host_ctx", ctypes.c_void_p)]


class Served(ctypes.Structure):
    _fields_ = [("result", LanczosResult), ("path", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double), ("t_done", ctypes.c_double)]


class ServerStats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in ("submitted", "completed", "failed", "verified", "running", "queued",
                                              "max_backlog", "batches", "batched_requests", "binary64_solves",
                                              "refined_solves")] + \
               [(n, ctypes.c_double) for n in ("budget_bytes", "peak_bytes", "free_bytes")]


_lib = None
P, I32, I64, D, SZ = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_size_t

# name -> (restype, argtypes); must match include/hubbard.h
SIGNATURES = {
    "hubbard_sector_create": (ctypes.c_int, [ctypes.c_int, P, ctypes.c_int, ctypes.c_int, ctypes.c_int, D, D, P]),
    "hubbard_sector_destroy": (None, [P]),
    "hubbard_sector_info": (ctypes.c_int, [P, P, P, P, P]),
    "hubbard_table_nnz": (I64, [P, ctypes.c_int]),
    "hubbard_export_tables": (ctypes.c_int, [P, ctypes.c_int, P, P, P, P]),
    "hubbard_apply": (ctypes.c_int, [P, P, P, ctypes.c_int, P]),
    "hubbard_apply_host": (ctypes.c_int, [P, P, P, ctypes.c_int, P]),
    "hubbard_apply_reference": (ctypes.c_int, [P, P, P, ctypes.c_int, P]),
    "hubbard_apply_noalloc": (ctypes.c_int, [P, P, P, P]),
    "hubbard_set_schedule": (ctypes.c_int, [P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "hubbard_vec_dot": (ctypes.c_int, [P, P, I64, ctypes.c_int, P, P]),
    "hubbard_vec_nrm2": (ctypes.c_int, [P, I64, ctypes.c_int, P, P]),
    "hubbard_vec_axpy": (ctypes.c_int, [D, P, P, I64, ctypes.c_int, P]),
    "hubbard_fill_start_vector": (ctypes.c_int, [P, I64, ctypes.c_uint64, I64, ctypes.c_int, P]),
    "hubbard_lanczos_step": (ctypes.c_int, [P, P, P, D, ctypes.c_int, P, P, P]),
    "lanczos_workspace_bytes": (SZ, [P, ctypes.c_int]),
    "lanczos_ground_state": (ctypes.c_int, [P, P, ctypes.c_int, D, ctypes.c_int, P, SZ, P, P, P, P, P]),
    "hubbard_host_spin_tables": (ctypes.c_int, [ctypes.c_int, P, ctypes.c_int, ctypes.c_int, P, P, P, P, P, P]),
    "hubbard_host_row_table": (ctypes.c_int, [ctypes.c_int, P, ctypes.c_int, ctypes.c_int, ctypes.c_int, P, P, P, P,
                                              P, P]),
    "hubbard_kernel_launches": (ctypes.c_uint64, []),
    "lanczos_refined_workspace_bytes": (SZ, [P]),
    "hubbard_batch_create": (ctypes.c_int, [P, ctypes.c_int, P]),
    "hubbard_batch_destroy": (None, [P]),
    "hubbard_batch_vector_offsets": (ctypes.c_int, [P, P]),
    "hubbard_batch_workspace_bytes": (SZ, [P, ctypes.c_int]),
    "hubbard_batch_set_schedule": (ctypes.c_int, [P, I64]),
    "hubbard_batch_solve_async": (ctypes.c_int, [P, P, ctypes.c_int, D, P, SZ, P]),
    "hubbard_batch_results": (ctypes.c_int, [P, P, ctypes.c_int, P, P]),
    "hubbard_batch_autotune": (ctypes.c_int, [P, P, ctypes.c_int, D, P, SZ, P, P]),
    "hubbard_batch_schedule_table": (ctypes.c_int, [P, P, ctypes.c_int, P]),
    "hubbard_queue_create": (ctypes.c_int, [ctypes.c_int, I64, ctypes.c_int, D, ctypes.c_int, P]),
    "hubbard_queue_post": (ctypes.c_int, [P, P, ctypes.c_uint64, P]),
    "hubbard_queue_poll": (ctypes.c_int, [P, I64, P]),
    "hubbard_queue_destroy": (None, [P]),
    "hubbard_queue_collect": (ctypes.c_int, [P, P, P, ctypes.c_int, P]),
    "hubbard_queue_prepare": (ctypes.c_int, [P, P]),
    "hubbard_batch_set_shape_mode": (ctypes.c_int, [P, ctypes.c_int, ctypes.c_int]),
    "hubbard_batch_set_task_ctas": (ctypes.c_int, [P, ctypes.c_int]),
    "hubbard_batch_get_schedule": (ctypes.c_int, [P, P, P]),
    "hubbard_selftest_wait_timeout": (ctypes.c_int, [P]),
    "hubbard_autotune_schedule": (ctypes.c_int, [P, P, P, ctypes.c_int, P, P]),
    "lanczos_ground_state_refined": (ctypes.c_int, [P, P, ctypes.c_int, D, P, SZ, P, P, P]),
    "hubbard_evolve_workspace_bytes": (SZ, [P, ctypes.c_int, ctypes.c_int]),
    "hubbard_time_evolve": (ctypes.c_int, [P, P, P, D, ctypes.c_int, D, P, SZ, P, P, P, P]),
    "hubbard_host_krylov_exp": (ctypes.c_int, [P, P, ctypes.c_int, D, P, P]),
    "hubbard_server_create": (ctypes.c_int, [P, P]),
    "hubbard_server_submit": (ctypes.c_int, [P, P, P]),
    "hubbard_server_poll": (ctypes.c_int, [P, ctypes.c_uint64, P]),
    "hubbard_server_wait": (ctypes.c_int, [P, ctypes.c_uint64, D, P]),
    "hubbard_server_stats_get": (ctypes.c_int, [P, P]),
    "hubbard_server_destroy": (None, [P]),
    "hubbard_last_error": (ctypes.c_char_p, []),
}


def load_library(path=LIB_PATH):
    """Load libhubbard.so; raises if it has not been built (no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with `python -m paper_1204_3425_gb300.build`")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(rc):
    if rc != HUB_OK:
        raise HubError(rc, _lib.hubbard_last_error().decode())


def _dtype_code(t):
    import torch
    if t.dtype == torch.float64:
        return HUB_F64
    if t.dtype == torch.float32:
        return HUB_F32
    raise TypeError(f"unsupported dtype {t.dtype}")


def _vec_pair(H, v, w, dtypes=None):
    """Checks that v and w are vectors of H.D elements of one supported dtype
    (the C entry points read and write exactly H.D elements of it)."""
    import torch
    allowed = dtypes if dtypes is not None else (torch.float64, torch.float32)
    if v.dtype not in allowed or w.dtype != v.dtype:
        raise TypeError(f"v and w must share one dtype of {allowed}, got {v.dtype} and {w.dtype}")
    if v.numel() != H.D or w.numel() != H.D:
        raise ValueError(f"v and w must hold D = {H.D} elements, got {v.numel()} and {w.numel()}")


def _ptr(t):
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


class Sector:
    """Owns one hubbard_t handle (device hopping tables of one sector)."""

    def __init__(self, handle, ns, bonds, nup, ndn, t, U):
        self.handle = handle
        self.ns, self.bonds, self.nup, self.ndn, self.t, self.U = ns, bonds, nup, ndn, t, U
        self.Dup, self.Ddn, self.Wup, self.Wdn = hubbard_sector_info(self)
        self.D = self.Dup * self.Ddn

    def close(self):
        if self.handle:
            _lib.hubbard_sector_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def hubbard_sector_create(ns, bonds, nup, ndn, t=1.0, U=0.0):
    lib = load_library()
    arr = np.ascontiguousarray(np.asarray(bonds, dtype=np.int32).reshape(-1))
    h = ctypes.c_void_p()
    _check(lib.hubbard_sector_create(int(ns), arr.ctypes.data if arr.size else None, arr.size // 2,
                                     int(nup), int(ndn), float(t), float(U), ctypes.byref(h)))
    return Sector(h, ns, bonds, nup, ndn, t, U)


def hubbard_sector_info(H):
    a, b, c, d = I64(), I64(), I32(), I32()
    _check(load_library().hubbard_sector_info(H.handle, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c),
                                              ctypes.byref(d)))
    return a.value, b.value, c.value, d.value


def hubbard_export_tables(H, spin):
    lib = load_library()
    D = H.Dup if spin == 0 else H.Ddn
    nnz = lib.hubbard_table_nnz(H.handle, spin)
    states = np.zeros(D, dtype=np.uint32)
    rowptr = np.zeros(D + 1, dtype=np.int32)
    tgt = np.zeros(max(nnz, 1), dtype=np.int32)
    sign = np.zeros(max(nnz, 1), dtype=np.int8)
    _check(lib.hubbard_export_tables(H.handle, spin, states.ctypes.data, rowptr.ctypes.data, tgt.ctypes.data,
                                     sign.ctypes.data))
    return states, rowptr, tgt[:nnz], sign[:nnz]


def hubbard_host_spin_tables(ns, bonds, n):
    """Host-only per-spin basis and hopping table (no GPU needed)."""
    lib = load_library()
    arr = np.ascontiguousarray(np.asarray(bonds, dtype=np.int32).reshape(-1))
    bp = arr.ctypes.data if arr.size else None
    D, nnz = I64(), I64()
    _check(lib.hubbard_host_spin_tables(int(ns), bp, arr.size // 2, int(n), ctypes.byref(D), ctypes.byref(nnz),
                                        None, None, None, None))
    states = np.zeros(D.value, dtype=np.uint32)
    rowptr = np.zeros(D.value + 1, dtype=np.int32)
    tgt = np.zeros(max(nnz.value, 1), dtype=np.int32)
    sign = np.zeros(max(nnz.value, 1), dtype=np.int8)
    _check(lib.hubbard_host_spin_tables(int(ns), bp, arr.size // 2, int(n), None, None, states.ctypes.data,
                                        rowptr.ctypes.data, tgt.ctypes.data, sign.ctypes.data))
    return states, rowptr, tgt[:nnz.value], sign[:nnz.value]


def hubbard_host_row_table(ns, bonds, n, elem_bytes):
    """Host-only row-phase hop table of one spin: (boff, bcnt, ent, narrow)."""
    lib = load_library()
    arr = np.ascontiguousarray(np.asarray(bonds, dtype=np.int32).reshape(-1))
    bp = arr.ctypes.data if arr.size else None
    G, E, nar = I64(), I64(), ctypes.c_int()
    _check(lib.hubbard_host_row_table(int(ns), bp, arr.size // 2, int(n), int(elem_bytes), ctypes.byref(G),
                                      ctypes.byref(E), ctypes.byref(nar), None, None, None))
    boff = np.zeros(max(G.value, 1), dtype=np.int64)
    bcnt = np.zeros(max(G.value, 1), dtype=np.int32)
    ent = np.zeros(max(E.value, 1), dtype=np.uint32)
    _check(lib.hubbard_host_row_table(int(ns), bp, arr.size // 2, int(n), int(elem_bytes), None, None, None,
                                      boff.ctypes.data, bcnt.ctypes.data, ent.ctypes.data))
    return boff[:G.value], bcnt[:G.value], ent[:E.value], bool(nar.value)


def hubbard_apply(H, v, w, stream=None):
    _vec_pair(H, v, w)
    _check(load_library().hubbard_apply(H.handle, _ptr(v), _ptr(w), _dtype_code(v), _stream(stream)))
    return w


def hubbard_apply_host(H, v, w, stream=None):
    """w = H v for CPU tensors (page-locked for overlap); asynchronous on `stream` (see hubbard.h)."""
    if v.device.type != "cpu" or w.device.type != "cpu":
        raise ValueError("hubbard_apply_host takes CPU tensors")
    if v.dtype != w.dtype:
        raise TypeError("v and w must have the same dtype")
    if v.numel() != H.D or w.numel() != H.D or not v.is_contiguous() or not w.is_contiguous():
        raise ValueError(f"v and w must be contiguous with {H.D} elements")
    _check(load_library().hubbard_apply_host(H.handle, ctypes.c_void_p(v.data_ptr()), ctypes.c_void_p(w.data_ptr()),
                                             _dtype_code(v), _stream(stream)))


def hubbard_apply_reference(H, v, w, stream=None):
    _vec_pair(H, v, w)
    _check(load_library().hubbard_apply_reference(H.handle, _ptr(v), _ptr(w), _dtype_code(v), _stream(stream)))
    return w


def hubbard_autotune_schedule(H, v, w, stream=None):
    """Times the H*v schedules on (v, w) and keeps the fastest; returns it as a tuple."""
    _vec_pair(H, v, w)
    out = (ctypes.c_int * 4)()
    _check(load_library().hubbard_autotune_schedule(H.handle, _ptr(v), _ptr(w), _dtype_code(v), _stream(stream), out))
    return tuple(out)


def hubbard_set_schedule(H, vec_rows=0, vec_cols=0, ctas_rows=0, ctas_cols=0):
    _check(load_library().hubbard_set_schedule(H.handle, int(vec_rows), int(vec_cols), int(ctas_rows),
                                               int(ctas_cols)))


HUBBARD_NOALLOC_MAX_ELEMS = 1 << 21


def hubbard_apply_noalloc(H, v, w, stream=None):
    """Binary64 w = H v through the entry point that allocates no device memory.

    For callers that cannot call cudaMalloc when they need H*v (another
    framework owns the allocator, a hard memory budget, or a hot loop that
    must not reach the allocator).  Its scratch is a fixed 16 MiB device array
    shared by all calls: sectors above HUBBARD_NOALLOC_MAX_ELEMS are rejected,
    and calls whose GPU work overlaps race on the array.
    """
    import torch
    _vec_pair(H, v, w, (torch.float64,))
    _check(load_library().hubbard_apply_noalloc(H.handle, _ptr(v), _ptr(w), _stream(stream)))
    return w


def hubbard_vec_dot(x, y, stream=None):
    out = D()
    _check(load_library().hubbard_vec_dot(_ptr(x), _ptr(y), x.numel(), _dtype_code(x), _stream(stream),
                                          ctypes.byref(out)))
    return out.value


def hubbard_vec_nrm2(x, stream=None):
    out = D()
    _check(load_library().hubbard_vec_nrm2(_ptr(x), x.numel(), _dtype_code(x), _stream(stream), ctypes.byref(out)))
    return out.value


def hubbard_vec_axpy(a, x, y, stream=None):
    _check(load_library().hubbard_vec_axpy(float(a), _ptr(x), _ptr(y), x.numel(), _dtype_code(x), _stream(stream)))
    return y


def hubbard_fill_start_vector(v, seed, start=0, stream=None):
    """Fill a device tensor with the seeded SplitMix64 start vector (entries start .. start+n-1)."""
    _check(load_library().hubbard_fill_start_vector(_ptr(v), v.numel(), int(seed), int(start), _dtype_code(v),
                                                    _stream(stream)))
    return v


def hubbard_lanczos_step(H, f, g, beta_j, stream=None):
    a, b = D(), D()
    _check(load_library().hubbard_lanczos_step(H.handle, _ptr(f), _ptr(g), float(beta_j), _dtype_code(f),
                                               _stream(stream), ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def lanczos_workspace_bytes(H, dtype=HUB_F64):
    return int(load_library().lanczos_workspace_bytes(H.handle, dtype))


def lanczos_ground_state(H, v0, max_iters, tol=0.0, workspace=None, stream=None, raise_on_notconv=False,
                         psi_out=None):
    """Returns dict(energy, residual, err_bound, iters, status, breakdown, alpha, beta).
    psi_out: optional float64 device tensor of D elements receiving the Ritz vector."""
    import torch
    lib = load_library()
    dt = _dtype_code(v0)
    if v0.numel() != H.D:
        raise ValueError(f"v0 must hold D = {H.D} elements, got {v0.numel()}")
    if psi_out is not None and (psi_out.dtype != torch.float64 or psi_out.numel() != H.D):
        raise ValueError("psi_out must be a float64 tensor of D elements")
    need = lanczos_workspace_bytes(H, dt)
    if workspace is None:
        workspace = torch.empty(need, dtype=torch.uint8, device=v0.device)
    a = np.zeros(max_iters)
    b = np.zeros(max_iters)
    res = LanczosResult()
    rc = lib.lanczos_ground_state(H.handle, _ptr(v0), int(max_iters), float(tol), dt, _ptr(workspace),
                                  workspace.numel() * workspace.element_size(),
                                  _ptr(psi_out) if psi_out is not None else None, _stream(stream),
                                  a.ctypes.data, b.ctypes.data, ctypes.byref(res))
    if rc != HUB_OK and not (rc == HUB_ENOTCONV and not raise_on_notconv):
        _check(rc)
    m = res.iters
    return dict(energy=res.energy, residual=res.residual, err_bound=res.err_bound, iters=m, status=res.status,
                breakdown=bool(res.breakdown), alpha=a[:m], beta=b[:m])


class RefinedResult(ctypes.Structure):
    _fields_ = [("energy", ctypes.c_double), ("residual", ctypes.c_double), ("error_bound", ctypes.c_double),
                ("energy_f32", ctypes.c_double), ("gap", ctypes.c_double), ("iters_f32", ctypes.c_int32),
                ("iters_f64", ctypes.c_int32), ("status", ctypes.c_int32), ("replayed", ctypes.c_int32)]


def lanczos_refined_workspace_bytes(H, store_vectors=0):
    """Minimum workspace, plus room for store_vectors binary32 Lanczos vectors
    (each stored vector saves one replayed step for the Ritz vector)."""
    slot = (H.D * 4 + 255) // 256 * 256
    return int(load_library().lanczos_refined_workspace_bytes(H.handle)) + int(store_vectors) * slot


def lanczos_ground_state_refined(H, v0, max_iters=1000, tol=1e-10, workspace=None, psi_out=None, stream=None,
                                 raise_on_notconv=False, store_vectors=0):
    """binary32 Lanczos + binary64 refinement; v0 binary64.  Returns a dict of the result fields.
    Without a workspace, one is allocated with room for store_vectors stored vectors."""
    import torch
    lib = load_library()
    need = lanczos_refined_workspace_bytes(H, store_vectors)
    if workspace is None:
        workspace = torch.empty(need, dtype=torch.uint8, device=v0.device)
    res = RefinedResult()
    rc = lib.lanczos_ground_state_refined(H.handle, _ptr(v0), int(max_iters), float(tol), _ptr(workspace),
                                          workspace.numel() * workspace.element_size(),
                                          _ptr(psi_out) if psi_out is not None else None, _stream(stream),
                                          ctypes.byref(res))
    if rc != HUB_OK and not (rc == HUB_ENOTCONV and not raise_on_notconv):
        _check(rc)
    return {f: getattr(res, f) for f, _ in RefinedResult._fields_}


class EvolveInfo(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int32), ("hv", ctypes.c_int32), ("krylov_dim", ctypes.c_int32),
                ("status", ctypes.c_int32), ("err_estimate", ctypes.c_double), ("norm", ctypes.c_double)]


def hubbard_evolve_workspace_bytes(H, krylov_max=40, store_basis=True):
    """Workspace of hubbard_time_evolve: 6 vectors, plus 2 * krylov_max stored
    Lanczos vectors when store_basis (else the recurrence is replayed)."""
    return int(load_library().hubbard_evolve_workspace_bytes(H.handle, int(krylov_max), 1 if store_basis else 0))


def hubbard_time_evolve(H, v_re, v_im, t, krylov_max=40, tol=1e-10, workspace=None, out_re=None, out_im=None,
                        store_basis=True, stream=None):
    """psi(t) = exp(-i H t) (v_re + i v_im) in binary64 (v_im may be None).
    Returns (out_re, out_im, info dict).  Without a workspace, one is allocated
    (with room for the Lanczos vectors when store_basis)."""
    import torch
    lib = load_library()
    _vec_pair(H, v_re, v_re, (torch.float64,))
    if v_im is not None:
        _vec_pair(H, v_im, v_im, (torch.float64,))
    if out_re is None:
        out_re = torch.empty_like(v_re)
    if out_im is None:
        out_im = torch.empty_like(v_re)
    _vec_pair(H, out_re, out_im, (torch.float64,))
    if workspace is None:
        workspace = torch.empty(hubbard_evolve_workspace_bytes(H, krylov_max, store_basis), dtype=torch.uint8,
                                device=v_re.device)
    info = EvolveInfo()
    rc = lib.hubbard_time_evolve(H.handle, _ptr(v_re), _ptr(v_im) if v_im is not None else None, float(t),
                                 int(krylov_max), float(tol), _ptr(workspace),
                                 workspace.numel() * workspace.element_size(), _ptr(out_re), _ptr(out_im),
                                 _stream(stream), ctypes.byref(info))
    _check(rc)
    return out_re, out_im, {f: getattr(info, f) for f, _ in EvolveInfo._fields_}


def hubbard_host_krylov_exp(a, b, tau):
    """Host helper: y = exp(-i T tau) e_1 for the tridiagonal T (diagonal a, off-diagonal b)."""
    import numpy as np
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    m = len(a)
    yr, yi = np.zeros(m), np.zeros(m)
    _check(load_library().hubbard_host_krylov_exp(a.ctypes.data, b.ctypes.data if len(b) else None, m, float(tau),
                                                  yr.ctypes.data, yi.ctypes.data))
    return yr + 1j * yi


def hubbard_selftest_wait_timeout(stream=None):
    """Runs the bounded-wait self-test; returns the status code (HUB_ETIMEOUT expected)."""
    rc = load_library().hubbard_selftest_wait_timeout(_stream(stream))
    return rc, load_library().hubbard_last_error().decode()


class SectorDesc(ctypes.Structure):
    _fields_ = [("ns", ctypes.c_int32), ("nup", ctypes.c_int32), ("ndn", ctypes.c_int32),
                ("n_bonds", ctypes.c_int32), ("bonds", ctypes.c_void_p), ("t", ctypes.c_double),
                ("U", ctypes.c_double)]


class Batch:
    """Owns a hubbard_batch_t: many sectors solved in one persistent launch."""

    def __init__(self, specs):
        """specs: list of (ns, bonds, nup, ndn, t, U)."""
        lib = load_library()
        self._bond_arrays = [np.ascontiguousarray(np.asarray(b, dtype=np.int32).reshape(-1)) for _, b, *_ in specs]
        descs = (SectorDesc * len(specs))()
        for i, ((ns, bonds, nup, ndn, t, U), arr) in enumerate(zip(specs, self._bond_arrays)):
            descs[i] = SectorDesc(int(ns), int(nup), int(ndn), arr.size // 2,
                                  arr.ctypes.data if arr.size else None, float(t), float(U))
        h = ctypes.c_void_p()
        _check(lib.hubbard_batch_create(descs, len(specs), ctypes.byref(h)))
        self.handle = h
        self.n = len(specs)
        off = np.zeros(self.n + 1, dtype=np.int64)
        _check(lib.hubbard_batch_vector_offsets(h, off.ctypes.data))
        self.offsets = off

    def workspace_bytes(self, max_iters):
        return int(load_library().hubbard_batch_workspace_bytes(self.handle, int(max_iters)))

    def set_schedule(self, elems_per_cta):
        _check(load_library().hubbard_batch_set_schedule(self.handle, int(elems_per_cta)))

    def solve_async(self, v0_all, max_iters, tol, workspace, stream=None):
        _check(load_library().hubbard_batch_solve_async(self.handle, _ptr(v0_all), int(max_iters), float(tol),
                                                        _ptr(workspace), workspace.numel(), _stream(stream)))

    def results(self, workspace, max_iters, stream=None):
        res = (LanczosResult * self.n)()
        _check(load_library().hubbard_batch_results(self.handle, _ptr(workspace), int(max_iters), _stream(stream),
                                                    res))
        return [dict(energy=r.energy, residual=r.residual, err_bound=r.err_bound, iters=r.iters, status=r.status,
                     breakdown=bool(r.breakdown)) for r in res]

    def autotune(self, v0_all, max_iters, tol, workspace, stream=None):
        chosen = I64()
        _check(load_library().hubbard_batch_autotune(self.handle, _ptr(v0_all), int(max_iters), float(tol),
                                                     _ptr(workspace), workspace.numel(), _stream(stream),
                                                     ctypes.byref(chosen)))
        return chosen.value

    def get_schedule(self):
        """(elems_per_cta, task_ctas) currently in use."""
        e, t = I64(), ctypes.c_int()
        _check(load_library().hubbard_batch_get_schedule(self.handle, ctypes.byref(e), ctypes.byref(t)))
        return e.value, t.value

    def set_task_ctas(self, n):
        _check(load_library().hubbard_batch_set_task_ctas(self.handle, int(n)))

    def set_shape_mode(self, shape, mode):
        _check(load_library().hubbard_batch_set_shape_mode(self.handle, int(shape), int(mode)))

    def schedule_table(self):
        """One dict per sector shape: D_up, D_dn, W, sectors, path ('task' / 'sweep'), mode bits."""
        lib = load_library()
        n = ctypes.c_int()
        _check(lib.hubbard_batch_schedule_table(self.handle, None, 0, ctypes.byref(n)))
        rows = (ctypes.c_int64 * (6 * max(n.value, 1)))()
        _check(lib.hubbard_batch_schedule_table(self.handle, rows, n.value, ctypes.byref(n)))
        return [dict(Dup=rows[6 * k], Ddn=rows[6 * k + 1], W=rows[6 * k + 2], sectors=rows[6 * k + 3],
                     path="sweep" if rows[6 * k + 4] == 2 else "task", mode=rows[6 * k + 5]) for k in range(n.value)]

    def close(self):
        if self.handle:
            load_library().hubbard_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def hubbard_kernel_launches():
    return int(load_library().hubbard_kernel_launches())


def hubbard_last_error():
    return load_library().hubbard_last_error().decode()


PATH_NAMES = {0: "batch", 1: "binary64", 2: "refined"}


class Queue:
    """Owns a hubbard_queue_t: sectors posted to a persistent solver while it runs."""

    def __init__(self, capacity=256, max_dim=20_000, max_iters=1000, tol=1e-10, ctas=0):
        h = ctypes.c_void_p()
        _check(load_library().hubbard_queue_create(int(capacity), int(max_dim), int(max_iters), float(tol), int(ctas),
                                                   ctypes.byref(h)))
        self.handle = h

    def post(self, ns, bonds, nup, ndn, t, U, seed):
        """Ticket of the posted sector, or None when the queue is full."""
        arr = np.ascontiguousarray(np.asarray(bonds, dtype=np.int32).reshape(-1))
        d = SectorDesc(int(ns), int(nup), int(ndn), arr.size // 2, arr.ctypes.data if arr.size else None, float(t),
                       float(U))
        tk = I64()
        rc = load_library().hubbard_queue_post(self.handle, ctypes.byref(d), int(seed), ctypes.byref(tk))
        if rc == HUB_EPENDING:
            return None
        _check(rc)
        return tk.value

    def poll(self, ticket):
        """The result dict once finished (returned once), else None."""
        r = LanczosResult()
        rc = load_library().hubbard_queue_poll(self.handle, int(ticket), ctypes.byref(r))
        if rc == HUB_EPENDING:
            return None
        _check(rc)
        return dict(energy=r.energy, residual=r.residual, err_bound=r.err_bound, iters=r.iters, status=r.status,
                    breakdown=bool(r.breakdown))

    def collect(self, cap=1024):
        """{ticket: result dict} of finished tasks not yet returned (each returned once)."""
        tk = (ctypes.c_int64 * max(cap, 1))()
        rs = (LanczosResult * max(cap, 1))()
        n = ctypes.c_int()
        _check(load_library().hubbard_queue_collect(self.handle, tk, rs, int(cap), ctypes.byref(n)))
        return {tk[i]: dict(energy=rs[i].energy, residual=rs[i].residual, err_bound=rs[i].err_bound,
                            iters=rs[i].iters, status=rs[i].status, breakdown=bool(rs[i].breakdown))
                for i in range(n.value)}

    def wait(self, ticket, timeout=60.0):
        import time
        end = time.perf_counter() + timeout
        while True:
            r = self.poll(ticket)
            if r is not None:
                return r
            if time.perf_counter() > end:
                raise TimeoutError(f"queue ticket {ticket} not finished after {timeout} s")
            time.sleep(0.0005)

    def close(self):
        if getattr(self, "handle", None):
            load_library().hubbard_queue_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Owns a hubbard_server_t: the native continuous-batching server.

    submit() queues one request (lattice bonds, fillings, t, U, seed) and
    returns its ticket; poll() / wait() return the result dict once it has
    finished.  host_solver (tests without a GPU): a Python callable
    (ticket, request_dict, path) -> dict(energy, residual, err_bound, iters,
    status) run by the lanes instead of the CUDA solvers."""

    def __init__(self, hbm_budget=0.0, small_lanes=2, big_lanes=8, small_max_dim=20_000, mid_max_dim=200_000,
                 max_iters=1000, batch_max=1024, store_vectors=128, tol=1e-10, host_solver=None, small_ctas=0):
        lib = load_library()
        self._cb = None
        cb = HOST_SOLVER()
        if host_solver is not None:
            def _solve(ctx, ticket, req, path, out):
                q = req.contents
                try:
                    r = host_solver(int(ticket), dict(ns=q.ns, nup=q.nup, ndn=q.ndn, t=q.t, U=q.U, seed=q.seed),
                                    int(path))
                except Exception:  # noqa: BLE001  (a failing request fails alone)
                    return HUB_EDEVICE
                o = out.contents
                o.energy, o.residual = float(r["energy"]), float(r.get("residual", 0.0))
                o.err_bound, o.iters = float(r.get("err_bound", 0.0)), int(r.get("iters", 1))
                o.status, o.breakdown = int(r.get("status", HUB_OK)), 0
                return int(r.get("status", HUB_OK))
            self._cb = cb = HOST_SOLVER(_solve)
        opts = ServerOpts(float(hbm_budget), int(small_lanes), int(big_lanes), int(small_max_dim), int(mid_max_dim),
                          int(max_iters), int(batch_max), int(store_vectors), int(small_ctas), float(tol), cb, None)
        h = ctypes.c_void_p()
        _check(lib.hubbard_server_create(ctypes.byref(opts), ctypes.byref(h)))
        self.handle = h
        self._bonds = {}

    def submit(self, ns, bonds, nup, ndn, t, U, seed):
        arr = np.ascontiguousarray(np.asarray(bonds, dtype=np.int32).reshape(-1))
        req = HubbardRequest(int(ns), int(nup), int(ndn), arr.size // 2, arr.ctypes.data if arr.size else None,
                             float(t), float(U), int(seed))
        tk = ctypes.c_uint64()
        _check(load_library().hubbard_server_submit(self.handle, ctypes.byref(req), ctypes.byref(tk)))
        return tk.value

    @staticmethod
    def _served(sv):
        r = sv.result
        return dict(energy=r.energy, residual=r.residual, err_bound=r.err_bound, iters=r.iters, status=r.status,
                    path=PATH_NAMES.get(sv.path, sv.path), t_submit=sv.t_submit, t_admit=sv.t_admit, t_done=sv.t_done)

    def poll(self, ticket):
        """The result dict once finished, else None."""
        sv = Served()
        rc = load_library().hubbard_server_poll(self.handle, int(ticket), ctypes.byref(sv))
        if rc == HUB_EPENDING:
            return None
        _check(rc)
        return self._served(sv)

    def wait(self, ticket, timeout=3600.0):
        sv = Served()
        _check(load_library().hubbard_server_wait(self.handle, int(ticket), float(timeout), ctypes.byref(sv)))
        return self._served(sv)

    def stats(self):
        st = ServerStats()
        _check(load_library().hubbard_server_stats_get(self.handle, ctypes.byref(st)))
        return {f: getattr(st, f) for f, _ in ServerStats._fields_}

    def close(self):
        if self.handle:
            load_library().hubbard_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
