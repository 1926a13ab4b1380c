"""Python binding of libddg, the B300 DDM-GNN Poisson solver (C ABI in include/ddg.h).

Argument marshalling only: every step runs in the library's CUDA kernels.
The functions keep the C names; handles are opaque ``ctypes.c_void_p`` values.
Host arrays are numpy arrays (copied by the library); device arrays are any
object with ``data_ptr()`` (a torch CUDA tensor) or a raw integer address.
A non-OK status raises ``DdgError`` (except ``ddg_fcg_solve``, which returns
its report so that NOT_CONVERGED can be inspected).

The shared library must exist (``paper_2402_08296_b300/libddg.so``, built by
``python paper_2402_08296_b300/build.py`` or ``__graft_entry__.build()``);
importing this package without it raises ``ImportError``.
"""
from __future__ import annotations

import ctypes
import os
import struct

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libddg.so")
if not os.path.exists(LIB_PATH):
    raise ImportError("libddg.so is not built; run `python paper_2402_08296_b300/build.py`")
lib = ctypes.CDLL(LIB_PATH)

DDG_OK = 0
DDG_INVALID_ARG = -1
DDG_OOM = -2
DDG_CUDA_ERROR = -3
DDG_NOT_CONVERGED = -4
DDG_BREAKDOWN = -5
DDG_BUSY = -6
DDG_TIMEOUT = -7
DDG_PENDING = -8
DDG_BAD_MESH = -9
DDG_TOO_LARGE = -10
DDG_INTERNAL = -11
STATUS_NAMES = {0: "OK", -1: "INVALID_ARG", -2: "OOM", -3: "CUDA_ERROR", -4: "NOT_CONVERGED",
                -5: "BREAKDOWN", -6: "BUSY", -7: "TIMEOUT", -8: "PENDING", -9: "BAD_MESH", -10: "TOO_LARGE",
                -11: "INTERNAL"}

DDG_NONE, DDG_DDM_LU, DDG_DDM_GNN = 0, 1, 2
DDG_COARSE, DDG_POU_PROLONG, DDG_BF16_WEIGHTS = 1, 2, 4

_p = ctypes.c_void_p
_i32 = ctypes.c_int32
_i64 = ctypes.c_int64
_u64 = ctypes.c_uint64
_sz = ctypes.c_size_t
_f32 = ctypes.c_float
_f64 = ctypes.c_double


class ddg_solve_report(ctypes.Structure):
    _fields_ = [("status", _i32), ("iterations", _i32), ("rel_residual", _f64),
                ("true_rel_residual", _f64), ("solve_ms", _f64), ("precond_ms", _f64),
                ("local_ms", _f64), ("local_launches", _i32), ("launches", _i32),
                ("local_applies", _i32), ("gnn_schedule", _i32), ("gnn_chunk_t", _i32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ddg_train_opts(ctypes.Structure):
    _fields_ = [("steps", _i32), ("batch", _i32), ("lr", _f32), ("clip", _f32), ("harvest_iters", _i32),
                ("seed", _u64)]


class ddg_train_report(ctypes.Structure):
    _fields_ = [("samples", _i32), ("steps", _i32), ("loss_first", _f64), ("loss_last", _f64), ("ms", _f64),
                ("lr_final", _f64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ddg_solve_opts(ctypes.Structure):
    _fields_ = [("kind", _i32), ("flags", ctypes.c_uint32), ("model", _p), ("K", _i32), ("overlap", _i32),
                ("rtol", _f64), ("max_iter", _i32), ("m_trunc", _i32)]


class ddg_serve_summary(ctypes.Structure):
    _fields_ = [("completed", _u64), ("failed", _u64), ("pending", _u64), ("active", _u64),
                ("reserved_bytes", _u64), ("device_bytes", _u64), ("p50_ms", _f64), ("p99_ms", _f64),
                ("solves_per_s", _f64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_SIGS = {
    "ddg_create": [_i32, _sz, ctypes.POINTER(_p)],
    "ddg_destroy": [_p],
    "ddg_memory_in_use": [_p, ctypes.POINTER(_sz)],
    "ddg_get_stream": [_p, ctypes.POINTER(_p)],
    "ddg_launch_count": [ctypes.POINTER(_u64)],
    "ddg_mesh_upload": [_p, _i32, _p, _i32, _p, _p, ctypes.POINTER(_p)],
    "ddg_problem_destroy": [_p],
    "ddg_assemble_poly": [_p, _p],
    "ddg_assemble_nodal": [_p, _p, _p],
    "ddg_problem_info": [_p, _p],
    "ddg_matrix_download": [_p, _p, _p, _p, _p],
    "ddg_partition": [_p, _i32, _i32, _p],
    "ddg_partition_download": [_p, _p, _p, _p, _p],
    "ddg_graph_download": [_p, _p, _p, _p, _p, _p],
    "ddg_coarse_download": [_p, _p, _p],
    "ddg_model_create": [_p, _i32, _i32, _f32, _p, _sz, _u64, ctypes.POINTER(_p)],
    "ddg_model_destroy": [_p],
    "ddg_model_get_weights": [_p, _p, _sz],
    "ddg_model_set_weights": [_p, _p, _sz],
    "ddg_setup_precond": [_p, _i32, _p, ctypes.c_uint32],
    "ddg_precondition": [_p, _p, _p, _p],
    "ddg_local_corrections": [_p, _p, _p, _p, _p],
    "ddg_apply_A": [_p, _p, _p, _p],
    "ddg_apply_A_dot_noalloc": [_p, _p, _p, _p, _p],
    "ddg_train_local_model": [_p, _p, ctypes.POINTER(ddg_train_opts), ctypes.POINTER(ddg_train_report)],
    "ddg_train_loss_grad": [_p, _p, _p, _p, _i32, ctypes.POINTER(_f64), _p],
    "ddg_submit": [_p, _i32, _p, _i32, _p, _p, ctypes.POINTER(ddg_solve_opts), ctypes.POINTER(_u64)],
    "ddg_poll": [_p, _u64, ctypes.POINTER(ddg_solve_report), _p],
    "ddg_serve_config": [_p, _i32, _i32, _i32],
    "ddg_serve_stats": [_p, ctypes.POINTER(ddg_serve_summary)],
    "ddg_fcg_solve": [_p, _p, _f64, _i32, _i32, _p, ctypes.POINTER(ddg_solve_report)],
    "ddg_fcg_history": [_p, _p, _i32, ctypes.POINTER(_i32)],
    "ddg_probe_fma_peaks": [_i32, ctypes.POINTER(_f64), ctypes.POINTER(_f64)],
}
for _name, _args in _SIGS.items():
    _fn = getattr(lib, _name)
    _fn.argtypes = _args
    _fn.restype = _i32
lib.ddg_last_error.argtypes = []
lib.ddg_last_error.restype = ctypes.c_char_p


class DdgError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = lib.ddg_last_error().decode(errors="replace")
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")


def _check(status: int, where: str) -> None:
    if status != DDG_OK:
        raise DdgError(status, where)


def _host(a, dtype):
    """Contiguous numpy copy/view of ``a`` with ``dtype`` and its address."""
    arr = np.ascontiguousarray(a, dtype=dtype)
    return arr, arr.ctypes.data_as(_p)


def _host_n(a, dtype, n: int, what: str):
    """_host with a length check: the library reads or writes exactly n values there."""
    arr, ptr = _host(a, dtype)
    if arr.size != n:
        raise ValueError(f"{what}: {arr.size} values, expected {n}")
    return arr, ptr


def _rows(a, dtype, width: int, what: str):
    """_host for an (n, width) array; returns (array, address, n)."""
    arr, ptr = _host(a, dtype)
    if arr.ndim != 2 or arr.shape[1] != width:
        raise ValueError(f"{what}: shape {arr.shape}, expected (n, {width})")
    return arr, ptr, arr.shape[0]


def _dev(x, n: int | None = None, what: str = "device array"):
    """Address of a device array: a contiguous CUDA torch tensor of float64 with at least n
    elements, or a raw device address (an int), which the caller vouches for."""
    if x is None:
        return None
    if isinstance(x, int):
        return _p(x)
    if not (hasattr(x, "data_ptr") and hasattr(x, "is_cuda") and hasattr(x, "dtype")):
        raise TypeError(f"{what}: expected a CUDA torch tensor or a device address, got {type(x).__name__}")
    import torch
    if x.dtype != torch.float64:
        raise TypeError(f"{what}: dtype {x.dtype}, expected torch.float64")
    if not x.is_cuda:
        raise ValueError(f"{what}: not on a CUDA device")
    if not x.is_contiguous():
        raise ValueError(f"{what}: not contiguous")
    if n is not None and x.numel() < n:
        raise ValueError(f"{what}: {x.numel()} elements, expected at least {n}")
    return _p(x.data_ptr())


def _devs(p, **arrays):
    """Checks the device arrays' types first (no library call), then their sizes against the
    problem: each keyword maps a name to (tensor, key of ddg_problem_info or a number)."""
    for name, (t, _) in arrays.items():
        _dev(t, None, name)
    info = ddg_problem_info(p)
    return [_dev(t, info[k] if isinstance(k, str) else k, name) for name, (t, k) in arrays.items()]


CUDA_STREAM_LEGACY = 1   # cudaStreamLegacy: the legacy default stream


def _stream(stream, *tensors):
    """The stream to launch on: the given one, else torch's current stream when torch tensors are passed.

    Handle 0 (torch's legacy default stream) is passed as cudaStreamLegacy, because the C ABI
    reads NULL as "the context's own stream", which does not synchronise with the default stream.
    """
    if stream is None:
        for t in tensors:
            if hasattr(t, "data_ptr") and hasattr(t, "device"):
                import torch
                stream = torch.cuda.current_stream(t.device)
                break
        else:
            return None
    h = stream if isinstance(stream, int) else stream.cuda_stream
    return _p(h if h else CUDA_STREAM_LEGACY)


def ddg_last_error() -> str:
    return lib.ddg_last_error().decode(errors="replace")


def ddg_create(device: int = 0, hbm_budget_bytes: int = 0):
    h = _p()
    _check(lib.ddg_create(device, hbm_budget_bytes, ctypes.byref(h)), "ddg_create")
    return h


def ddg_destroy(ctx) -> None:
    _check(lib.ddg_destroy(ctx), "ddg_destroy")


def ddg_memory_in_use(ctx) -> int:
    v = _sz()
    _check(lib.ddg_memory_in_use(ctx, ctypes.byref(v)), "ddg_memory_in_use")
    return int(v.value)


def ddg_get_stream(ctx) -> int:
    h = _p()
    _check(lib.ddg_get_stream(ctx, ctypes.byref(h)), "ddg_get_stream")
    return int(h.value or 0)


def ddg_launch_count() -> int:
    v = _u64()
    _check(lib.ddg_launch_count(ctypes.byref(v)), "ddg_launch_count")
    return int(v.value)


def ddg_mesh_upload(ctx, xy, tri, dirichlet=None):
    xy_a, xy_p, n = _rows(xy, np.float64, 2, "xy")
    tri_a, tri_p, t = _rows(tri, np.int32, 3, "tri")
    d_p = None
    if dirichlet is not None:
        d_a, d_p = _host_n(dirichlet, np.uint8, n, "dirichlet")
    h = _p()
    _check(lib.ddg_mesh_upload(ctx, n, xy_p, t, tri_p, d_p, ctypes.byref(h)), "ddg_mesh_upload")
    return h


def ddg_problem_destroy(p) -> None:
    _check(lib.ddg_problem_destroy(p), "ddg_problem_destroy")


def ddg_assemble_poly(p, r) -> None:
    r_a, r_p = _host_n(r, np.float64, 9, "r")
    _check(lib.ddg_assemble_poly(p, r_p), "ddg_assemble_poly")


def ddg_assemble_nodal(p, f, g) -> None:
    n = ddg_problem_info(p)["n_nodes"]
    f_a, f_p = _host_n(f, np.float64, n, "f")
    g_a, g_p = _host_n(g, np.float64, n, "g")
    _check(lib.ddg_assemble_nodal(p, f_p, g_p), "ddg_assemble_nodal")


def ddg_problem_info(p) -> dict:
    info = np.zeros(10, dtype=np.int64)
    _check(lib.ddg_problem_info(p, info.ctypes.data_as(_p)), "ddg_problem_info")
    keys = ["n_nodes", "n_tri", "n_free", "nnz", "K", "sum_k", "sum_loc", "sum_edges", "max_loc"]
    out = {k: int(v) for k, v in zip(keys, info[:9])}
    out["hbar"] = struct.unpack("<d", struct.pack("<q", int(info[9])))[0]
    return out


def ddg_matrix_download(p):
    info = ddg_problem_info(p)
    nf, nnz = info["n_free"], info["nnz"]
    rowptr = np.zeros(nf + 1, np.int32)
    col = np.zeros(nnz, np.int32)
    val = np.zeros(nnz, np.float64)
    b = np.zeros(nf, np.float64)
    _check(lib.ddg_matrix_download(p, rowptr.ctypes.data_as(_p), col.ctypes.data_as(_p), val.ctypes.data_as(_p),
                                   b.ctypes.data_as(_p)), "ddg_matrix_download")
    return rowptr, col, val, b


def ddg_partition(p, K: int, overlap_layers: int, part=None) -> None:
    pp = None
    if part is not None:
        part_a, pp = _host_n(part, np.int32, ddg_problem_info(p)["n_free"], "part")
    _check(lib.ddg_partition(p, K, overlap_layers, pp), "ddg_partition")


def ddg_partition_download(p):
    info = ddg_problem_info(p)
    nf, K, sk = info["n_free"], info["K"], info["sum_k"]
    part = np.zeros(nf, np.int32)
    sub_ptr = np.zeros(K + 1, np.int32)
    sub_idx = np.zeros(sk, np.int32)
    mult = np.zeros(nf, np.int32)
    _check(lib.ddg_partition_download(p, part.ctypes.data_as(_p), sub_ptr.ctypes.data_as(_p),
                                      sub_idx.ctypes.data_as(_p), mult.ctypes.data_as(_p)), "ddg_partition_download")
    return part, sub_ptr, sub_idx, mult


def ddg_graph_download(p):
    info = ddg_problem_info(p)
    K, sl, se = info["K"], info["sum_loc"], info["sum_edges"]
    loc_ptr = np.zeros(K + 1, np.int32)
    n_int = np.zeros(K, np.int32)
    loc_node = np.zeros(sl, np.int32)
    nbr_ptr = np.zeros(sl + K, np.int32)
    nbr = np.zeros(se, np.int32)
    _check(lib.ddg_graph_download(p, loc_ptr.ctypes.data_as(_p), n_int.ctypes.data_as(_p), loc_node.ctypes.data_as(_p),
                                  nbr_ptr.ctypes.data_as(_p), nbr.ctypes.data_as(_p)), "ddg_graph_download")
    return loc_ptr, n_int, loc_node, nbr_ptr, nbr


def ddg_coarse_download(p):
    K = ddg_problem_info(p)["K"]
    A0 = np.zeros((K, K))
    A0inv = np.zeros((K, K))
    _check(lib.ddg_coarse_download(p, A0.ctypes.data_as(_p), A0inv.ctypes.data_as(_p)), "ddg_coarse_download")
    return A0, A0inv


def ddg_model_create(ctx, kbar: int, d: int, alpha: float, w=None, seed: int = 0):
    n_w = kbar * (11 * d * d + 15 * d + 1)
    wp = None
    if w is not None:
        w_a, wp = _host_n(w, np.float32, n_w, "w")
    h = _p()
    _check(lib.ddg_model_create(ctx, kbar, d, alpha, wp, n_w, seed, ctypes.byref(h)), "ddg_model_create")
    return h


def ddg_model_destroy(m) -> None:
    _check(lib.ddg_model_destroy(m), "ddg_model_destroy")


def ddg_model_get_weights(m, n_w: int) -> np.ndarray:
    w = np.zeros(n_w, np.float32)
    _check(lib.ddg_model_get_weights(m, w.ctypes.data_as(_p), n_w), "ddg_model_get_weights")
    return w


def ddg_model_set_weights(m, w) -> None:
    w_a, w_p = _host(w, np.float32)
    _check(lib.ddg_model_set_weights(m, w_p, ctypes.c_size_t(w_a.size)), "ddg_model_set_weights")


def ddg_setup_precond(p, kind: int, model=None, flags: int = DDG_COARSE) -> None:
    _check(lib.ddg_setup_precond(p, kind, model, flags), "ddg_setup_precond")


def ddg_precondition(p, r_dev, z_dev, stream=None) -> None:
    r_p, z_p = _devs(p, r_dev=(r_dev, "n_free"), z_dev=(z_dev, "n_free"))
    _check(lib.ddg_precondition(p, r_p, z_p, _stream(stream, r_dev, z_dev)), "ddg_precondition")


def ddg_local_corrections(p, r_dev, corr_dev, s_dev, stream=None) -> None:
    r_p, c_p, s_p = _devs(p, r_dev=(r_dev, "n_free"), corr_dev=(corr_dev, "sum_k"), s_dev=(s_dev, "K"))
    _check(lib.ddg_local_corrections(p, r_p, c_p, s_p, _stream(stream, r_dev)), "ddg_local_corrections")


def ddg_apply_A(p, x_dev, y_dev, stream=None) -> None:
    x_p, y_p = _devs(p, x_dev=(x_dev, "n_free"), y_dev=(y_dev, "n_free"))
    _check(lib.ddg_apply_A(p, x_p, y_p, _stream(stream, x_dev, y_dev)), "ddg_apply_A")


def ddg_apply_A_dot_noalloc(p, x_dev, y_dev, xy_dev, stream=None) -> None:
    """y = A x and x . y into the one-element device tensor xy_dev, with no device allocation."""
    x_p, y_p, xy_p = _devs(p, x_dev=(x_dev, "n_free"), y_dev=(y_dev, "n_free"), xy_dev=(xy_dev, 1))
    _check(lib.ddg_apply_A_dot_noalloc(p, x_p, y_p, xy_p, _stream(stream, x_dev, y_dev)), "ddg_apply_A_dot_noalloc")


def ddg_train_local_model(p, m, steps: int, batch: int = 32, lr: float = 1e-2, clip: float = 1e-2,
                          harvest_iters: int = 60, seed: int = 0) -> dict:
    """Train model m on the local problems of p's decomposition (see include/ddg.h)."""
    o = ddg_train_opts(steps, batch, lr, clip, harvest_iters, seed)
    rep = ddg_train_report()
    _check(lib.ddg_train_local_model(p, m, ctypes.byref(o), ctypes.byref(rep)), "ddg_train_local_model")
    return rep.as_dict()


def ddg_train_loss_grad(p, m, r_dev, graphs, n_w: int):
    """(loss, flat gradient) of the training loss for the given local graphs with residual r_dev."""
    g_a, g_p = _host(graphs, np.int32)
    (r_p,) = _devs(p, r_dev=(r_dev, "n_free"))
    loss = _f64()
    grad = np.zeros(n_w, np.float32)
    _check(lib.ddg_train_loss_grad(p, m, r_p, g_p, g_a.size, ctypes.byref(loss), grad.ctypes.data_as(_p)),
           "ddg_train_loss_grad")
    return float(loss.value), grad


def ddg_fcg_solve(p, rtol: float, max_iter: int, m_trunc: int, x0=None, want_x: bool = True):
    """Returns (report dict, x over all mesh nodes or None)."""
    info = ddg_problem_info(p)
    x0p = None
    if x0 is not None:
        x0_a, x0p = _host_n(x0, np.float64, info["n_free"], "x0")
    x = np.zeros(info["n_nodes"], np.float64) if want_x else None
    rep = ddg_solve_report()
    st = lib.ddg_fcg_solve(p, x0p, rtol, max_iter, m_trunc, x.ctypes.data_as(_p) if want_x else None,
                           ctypes.byref(rep))
    if st not in (DDG_OK, DDG_NOT_CONVERGED, DDG_BREAKDOWN):
        raise DdgError(st, "ddg_fcg_solve")
    return rep.as_dict(), x


def ddg_fcg_history(p) -> np.ndarray:
    """|r| / |b| after every iteration of the problem's last ddg_fcg_solve."""
    cnt = _i32()
    _check(lib.ddg_fcg_history(p, None, 0, ctypes.byref(cnt)), "ddg_fcg_history")
    out = np.zeros(cnt.value, np.float64)
    if cnt.value:
        _check(lib.ddg_fcg_history(p, out.ctypes.data_as(_p), cnt.value, ctypes.byref(cnt)), "ddg_fcg_history")
    return out


def ddg_probe_fma_peaks(device: int = 0) -> dict:
    """FP32 and FP64 FMA rates (TFLOP/s) this GPU reaches (include/ddg_probe.h)."""
    f32, f64 = _f64(), _f64()
    _check(lib.ddg_probe_fma_peaks(device, ctypes.byref(f32), ctypes.byref(f64)), "ddg_probe_fma_peaks")
    return {"fp32_tflops": float(f32.value), "fp64_tflops": float(f64.value)}


_TICKET_NODES = {}  # (context address, ticket) -> nodes of the submitted mesh, until collected


def _addr(handle) -> int:
    return int(handle.value or 0) if hasattr(handle, "value") else int(handle or 0)


def ddg_submit(ctx, xy, tri, r, kind: int, model=None, flags: int = DDG_COARSE, K: int = 0, overlap: int = 2,
               rtol: float = 1e-6, max_iter: int = 2000, m_trunc: int = 10) -> int:
    """Queue a solve; returns its ticket."""
    xy_a, xy_p, n = _rows(xy, np.float64, 2, "xy")
    tri_a, tri_p, nt = _rows(tri, np.int32, 3, "tri")
    r_a, r_p = _host_n(r, np.float64, 9, "r")
    o = ddg_solve_opts(kind, flags, model, K, overlap, rtol, max_iter, m_trunc)
    t = _u64()
    _check(lib.ddg_submit(ctx, n, xy_p, nt, tri_p, r_p, ctypes.byref(o), ctypes.byref(t)), "ddg_submit")
    _TICKET_NODES[(_addr(ctx), int(t.value))] = n
    return int(t.value)


def ddg_poll(ctx, ticket: int, n_nodes: int | None = None):
    """(status, report dict, x or None); status DDG_PENDING while the request runs.

    With n_nodes given, x receives the solution; the buffer is sized from the mesh that
    ddg_submit sent, and a different n_nodes is refused (the library writes that many values)."""
    key = (_addr(ctx), int(ticket))
    known = _TICKET_NODES.get(key)
    if n_nodes and known is not None and n_nodes != known:
        raise ValueError(f"ddg_poll: n_nodes {n_nodes}, but ticket {ticket} was submitted with {known} nodes")
    rep = ddg_solve_report()
    x = np.zeros(known if known is not None else n_nodes, np.float64) if n_nodes else None
    st = lib.ddg_poll(ctx, ticket, ctypes.byref(rep), x.ctypes.data_as(_p) if x is not None else None)
    if st == DDG_PENDING:
        return st, None, None
    _TICKET_NODES.pop(key, None)
    if st == DDG_INVALID_ARG:
        raise DdgError(st, "ddg_poll")
    return st, rep.as_dict(), x


def ddg_serve_config(ctx, max_active: int, fuse_gnn: bool = False, max_pending: int = 65536) -> None:
    _check(lib.ddg_serve_config(ctx, max_active, 1 if fuse_gnn else 0, max_pending), "ddg_serve_config")


def ddg_serve_stats(ctx) -> dict:
    out = ddg_serve_summary()
    _check(lib.ddg_serve_stats(ctx, ctypes.byref(out)), "ddg_serve_stats")
    return out.as_dict()


_LOSS_FN = None


def dss_residual_loss(w, p, m, r_dev, graphs):
    """The training loss of Eq. 23 as a differentiable PyTorch function of the flat weights.

    Sets model m's weights to the float32 tensor ``w``, runs the library's forward kernel
    (saving every block's latents) and its hand-written backward kernel on the local graphs
    ``graphs`` of problem p with global residual ``r_dev``, and returns the loss as a 0-d
    FP64 tensor whose ``backward`` yields the gradient those kernels computed (a
    torch.autograd.Function; no PyTorch arithmetic is involved).
    """
    global _LOSS_FN
    if _LOSS_FN is None:
        import torch

        class _DssResidualLoss(torch.autograd.Function):
            @staticmethod
            def forward(ctx, w, p, m, r_dev, graphs):
                wh = w.detach().to("cpu", torch.float32).contiguous().numpy()
                ddg_model_set_weights(m, wh)
                loss, grad = ddg_train_loss_grad(p, m, r_dev, graphs, wh.size)
                ctx.save_for_backward(torch.as_tensor(grad).to(w.device))
                return torch.tensor(loss, dtype=torch.float64, device=w.device)

            @staticmethod
            def backward(ctx, g):
                (grad,) = ctx.saved_tensors
                return g.to(grad.dtype) * grad, None, None, None, None

        _LOSS_FN = _DssResidualLoss
    return _LOSS_FN.apply(w, p, m, r_dev, graphs)
