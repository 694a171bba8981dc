"""ctypes binding of libgbbc.so (include/gbbc.h), same names as the C ABI.

Argument marshalling only: every step of the computation runs in the CUDA
library.  Buffers may be numpy arrays (host) or torch tensors (host or CUDA);
streams are torch.cuda.Stream objects, raw cudaStream_t integers, or None
(the current torch stream when torch has CUDA, else the default stream).
A missing libgbbc.so raises ImportError at first use: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgbbc.so")
_lock = threading.Lock()
_lib = None

GBBC_OK, GBBC_ERR_INVALID, GBBC_ERR_OOM, GBBC_ERR_CUDA, GBBC_ERR_TIMEOUT, GBBC_ERR_CAPACITY, GBBC_ERR_STATE = range(7)
POLICY = {"auto": 0, "beamer": 1, "learned": 2, "push": 3, "pull": 4}
SCHEDULE = {"auto": 0, "grid": 1, "block": 2, "pair": 3}
GBBC_KEEP_STATE = 1
GBBC_TRACE = 2
GBBC_TRACE_BOTH = 4
GBBC_DEVICE_LOOP = 8
GBBC_SYNC_BACKWARD = 16

# every symbol include/gbbc.h declares
EXPORTS = ("bc_options_init", "bc_graph_create", "bc_graph_create_multi", "bc_graph_create_weighted", "bc_compute", "bc_compute_multi",
           "bc_read", "bc_read_source_state", "bc_reset", "bc_sync", "bc_graph_destroy", "bc_status_string",
           "bc_last_error_detail", "bc_get_stats", "bc_get_trace", "bc_clear_trace", "bc_get_profile",
           "bc_compute_noalloc", "bc_mlp_param_count", "bc_mlp_forward", "bc_mlp_loss_grad", "bc_mlp_adam_step",
           "bc_mlp_train", "bc_policy_eval", "bc_policy_load", "bc_read_fixed", "bc_source_features",
           "bc_grouping_load", "bc_grouping_scores", "bc_release_memory", "bc_add_fixed", "bc_partition",
           "bc_partition_info", "bc_read_border_matrix", "bc_compute_partitioned")
NOALLOC_MAX_VERTICES = 16384
MAX_WEIGHT = 64  # GBBC_MAX_WEIGHT


class gbbc_options(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_uint32), ("batch_width", ctypes.c_int32), ("policy", ctypes.c_int32),
                ("validate", ctypes.c_int32), ("timeout_spins", ctypes.c_int64), ("flags", ctypes.c_uint32),
                ("heavy_degree", ctypes.c_int32), ("mem_limit_bytes", ctypes.c_int64),
                ("schedule", ctypes.c_int32), ("streams", ctypes.c_int32)]


class gbbc_stats(ctypes.Structure):
    _fields_ = [("sources", ctypes.c_int64), ("batches", ctypes.c_int64), ("levels_fwd", ctypes.c_int64),
                ("levels_push", ctypes.c_int64), ("levels_pull", ctypes.c_int64), ("wide_batches", ctypes.c_int64),
                ("kernel_launches", ctypes.c_int64), ("device_bytes", ctypes.c_int64),
                ("batch_width", ctypes.c_int32), ("policy", ctypes.c_int32),
                ("schedule", ctypes.c_int32), ("block_slots", ctypes.c_int32),
                ("persist_launches", ctypes.c_int64), ("persist_ms", ctypes.c_double),
                ("persist_slots", ctypes.c_int32), ("persist_blocks", ctypes.c_int32),
                ("tuned_heavy_degree", ctypes.c_int32), ("tuned_device_loop", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class gbbc_level_trace(ctypes.Structure):
    _fields_ = [("batch", ctypes.c_int32), ("level", ctypes.c_int32), ("direction", ctypes.c_int32),
                ("active_lanes", ctypes.c_int32), ("n_range", ctypes.c_int64), ("nnz_range", ctypes.c_int64),
                ("frontier_vertices", ctypes.c_int64), ("frontier_edges", ctypes.c_int64),
                ("frontier_lanes", ctypes.c_int64), ("visited_lanes", ctypes.c_int64),
                ("visited_lane_edges", ctypes.c_int64), ("max_degree", ctypes.c_int64),
                ("next_vertices", ctypes.c_int64), ("next_edges", ctypes.c_int64),
                ("scanned_edges", ctypes.c_int64), ("ms_push", ctypes.c_float), ("ms_pull", ctypes.c_float),
                ("ms_gather", ctypes.c_float), ("ms_backward", ctypes.c_float),
                ("features", ctypes.c_float * 6)]


class gbbc_kernel_profile(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_int64), ("ms", ctypes.c_double),
                ("bytes", ctypes.c_double)]


class gbbc_partition_info(ctypes.Structure):
    _fields_ = [("parts", ctypes.c_int32), ("border_nodes", ctypes.c_int64), ("border_edges", ctypes.c_int64),
                ("intra_entries", ctypes.c_int64), ("matrix_entries", ctypes.c_int64),
                ("refinement_sweeps", ctypes.c_int64), ("backward_waits", ctypes.c_int64)]


class GbbcError(RuntimeError):
    def __init__(self, status, detail):
        super().__init__(f"{status_name(status)}: {detail}")
        self.status = status
        self.detail = detail


def load():
    """Load libgbbc.so (raises ImportError if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libgbbc.so not found at {LIB_PATH}: build it with __graft_entry__.build()")
        lib = ctypes.CDLL(LIB_PATH)
        vp, i32, i64, u32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32
        P = ctypes.POINTER
        sig = {
            "bc_options_init": (None, [P(gbbc_options)]),
            "bc_graph_create": (ctypes.c_int, [i32, i64, vp, vp, P(gbbc_options), vp, P(vp)]),
            "bc_graph_create_weighted": (ctypes.c_int, [i32, i64, vp, vp, vp, P(gbbc_options), vp, P(vp)]),
            "bc_graph_create_multi": (ctypes.c_int, [i32, vp, vp, vp, vp, P(gbbc_options), vp, P(vp)]),
            "bc_compute": (ctypes.c_int, [vp, vp, i64, vp]),
            "bc_compute_multi": (ctypes.c_int, [vp, vp, vp, i64, vp]),
            "bc_read": (ctypes.c_int, [vp, vp, i32, vp]),
            "bc_read_source_state": (ctypes.c_int, [vp, i64, vp, vp, vp]),
            "bc_read_fixed": (ctypes.c_int, [vp, vp, i32, vp]),
            "bc_add_fixed": (ctypes.c_int, [vp, vp, i32, vp]),
            "bc_partition": (ctypes.c_int, [vp, vp, i32, vp]),
            "bc_partition_info": (ctypes.c_int, [vp, P(gbbc_partition_info)]),
            "bc_read_border_matrix": (ctypes.c_int, [vp, i32, vp, vp, vp, vp, vp]),
            "bc_compute_partitioned": (ctypes.c_int, [vp, vp, i64, vp]),
            "bc_reset": (ctypes.c_int, [vp]),
            "bc_sync": (ctypes.c_int, [vp]),
            "bc_graph_destroy": (None, [vp]),
            "bc_status_string": (ctypes.c_char_p, [ctypes.c_int]),
            "bc_last_error_detail": (ctypes.c_int, [vp, ctypes.c_char_p, ctypes.c_size_t]),
            "bc_get_stats": (ctypes.c_int, [vp, P(gbbc_stats)]),
            "bc_get_trace": (ctypes.c_int, [vp, P(gbbc_level_trace), i64, P(i64)]),
            "bc_clear_trace": (ctypes.c_int, [vp]),
            "bc_get_profile": (ctypes.c_int, [vp, P(gbbc_kernel_profile), i32, P(i32)]),
            "bc_compute_noalloc": (ctypes.c_int, [i32, i64, vp, vp, vp, i64, vp, vp]),
            "bc_mlp_param_count": (i64, [i32]),
            "bc_mlp_forward": (ctypes.c_int, [vp, i32, vp, i64, vp, vp]),
            "bc_mlp_loss_grad": (ctypes.c_int, [vp, i32, vp, vp, vp, i64, i32, vp, vp, vp]),
            "bc_mlp_adam_step": (ctypes.c_int, [vp, vp, vp, vp, i64, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                                ctypes.c_float, i32, vp]),
            "bc_mlp_train": (ctypes.c_int, [vp, i32, vp, vp, vp, i64, i32, i32, ctypes.c_float, vp, vp]),
            "bc_policy_eval": (ctypes.c_int, [vp, vp, i64, vp, vp, vp]),
            "bc_policy_load": (ctypes.c_int, [vp, vp, ctypes.c_size_t]),
            "bc_grouping_load": (ctypes.c_int, [vp, vp, ctypes.c_size_t]),
            "bc_release_memory": (ctypes.c_int, [i32]),
            "bc_source_features": (ctypes.c_int, [vp, vp, i64, vp, vp]),
            "bc_grouping_scores": (ctypes.c_int, [vp, vp, i64, vp, vp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def status_name(status: int) -> str:
    try:
        return load().bc_status_string(int(status)).decode()
    except ImportError:
        return f"status {status}"


def last_error(handle=None) -> str:
    buf = ctypes.create_string_buffer(1024)
    load().bc_last_error_detail(handle, buf, len(buf))
    return buf.value.decode(errors="replace")


def _check(status, handle=None):
    if status != GBBC_OK:
        raise GbbcError(status, last_error(handle))


def _ptr(buf):
    """(pointer, keepalive) of a numpy array or torch tensor (contiguous)."""
    if buf is None:
        return None, None
    if hasattr(buf, "data_ptr"):
        if not buf.is_contiguous():
            buf = buf.contiguous()
        return buf.data_ptr(), buf
    arr = np.ascontiguousarray(buf)
    return arr.ctypes.data, arr


def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available() and torch.cuda.is_initialized():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return None
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


def _as_i32(buf):
    if hasattr(buf, "data_ptr"):
        import torch
        return buf.to(torch.int32).contiguous()
    return np.ascontiguousarray(buf, dtype=np.int32)


def options(batch_width=0, policy="auto", validate=False, flags=0, heavy_degree=0, mem_limit_bytes=0,
            timeout_spins=0, schedule="auto", streams=0) -> gbbc_options:
    o = gbbc_options()
    load().bc_options_init(ctypes.byref(o))
    o.batch_width = int(batch_width)
    o.policy = POLICY[policy] if isinstance(policy, str) else int(policy)
    o.validate = int(bool(validate))
    o.flags = int(flags)
    o.heavy_degree = int(heavy_degree)
    o.mem_limit_bytes = int(mem_limit_bytes)
    o.timeout_spins = int(timeout_spins)
    o.schedule = SCHEDULE[schedule] if isinstance(schedule, str) else int(schedule)
    o.streams = int(streams)
    return o


# ---- the C ABI, one wrapper per call ---------------------------------------

def bc_options_init() -> gbbc_options:
    return options()


def bc_graph_create(n, nnz, row_ptr, col, opt=None, stream=None):
    rp, k1 = _ptr(_as_i32(row_ptr))
    cl, k2 = _ptr(_as_i32(col))
    h = ctypes.c_void_p()
    st = load().bc_graph_create(int(n), int(nnz), rp, cl, ctypes.byref(opt) if opt is not None else None,
                                _stream(stream), ctypes.byref(h))
    _check(st)
    return h


def bc_graph_create_weighted(n, nnz, row_ptr, col, weight, opt=None, stream=None):
    rp, k1 = _ptr(_as_i32(row_ptr))
    cl, k2 = _ptr(_as_i32(col))
    wt, k3 = _ptr(_as_i32(weight))
    h = ctypes.c_void_p()
    st = load().bc_graph_create_weighted(int(n), int(nnz), rp, cl, wt,
                                         ctypes.byref(opt) if opt is not None else None, _stream(stream),
                                         ctypes.byref(h))
    _check(st)
    return h


def bc_graph_create_multi(ns, nnzs, row_ptrs, cols, opt=None, stream=None):
    count = len(ns)
    keep = []
    rps = (ctypes.c_void_p * max(count, 1))()
    cls = (ctypes.c_void_p * max(count, 1))()
    for i in range(count):
        a, ka = _ptr(_as_i32(row_ptrs[i]))
        b, kb = _ptr(_as_i32(cols[i]))
        rps[i], cls[i] = a, b
        keep += [ka, kb]
    n_arr = np.ascontiguousarray(ns, dtype=np.int32)
    m_arr = np.ascontiguousarray(nnzs, dtype=np.int64)
    h = ctypes.c_void_p()
    st = load().bc_graph_create_multi(count, n_arr.ctypes.data, m_arr.ctypes.data, ctypes.addressof(rps),
                                      ctypes.addressof(cls), ctypes.byref(opt) if opt is not None else None,
                                      _stream(stream), ctypes.byref(h))
    _check(st)
    return h


def bc_compute(handle, sources, k=None, stream=None):
    src = _as_i32(sources)
    p, keep = _ptr(src)
    k = len(src) if k is None else int(k)
    _check(load().bc_compute(handle, p, k, _stream(stream)), handle)


def bc_compute_multi(handle, graph_id, local_src, stream=None):
    gi = _as_i32(graph_id)
    ls = _as_i32(local_src)
    if len(gi) != len(ls):
        raise ValueError("graph_id and local_src differ in length")
    p1, k1 = _ptr(gi)
    p2, k2 = _ptr(ls)
    _check(load().bc_compute_multi(handle, p1, p2, len(gi), _stream(stream)), handle)


def bc_read(handle, n, out=None, graph_id=-1, stream=None):
    """Read BC into `out` (numpy float64 / torch float64, host or CUDA) or a
    new numpy array of n entries."""
    if out is None:
        out = np.zeros(int(n), np.float64)
    p, keep = _ptr(out)
    _check(load().bc_read(handle, p, int(graph_id), _stream(stream)), handle)
    return out


def bc_read_fixed(handle, n, graph_id=-1, stream=None):
    """Exact BC as uint64 [n, 2] (low, high words of 128-bit fixed point, units 2^-64)."""
    out = np.zeros((int(n), 2), np.uint64)
    _check(load().bc_read_fixed(handle, out.ctypes.data, int(graph_id), _stream(stream)), handle)
    return out


def bc_read_fixed_into(handle, out, graph_id=-1, stream=None):
    """bc_read_fixed into a caller buffer (numpy uint64 / torch int64 or
    uint64 [n, 2] or [2n], host or CUDA)."""
    p, keep = _ptr(out)
    _check(load().bc_read_fixed(handle, p, int(graph_id), _stream(stream)), handle)
    return out


def bc_add_fixed(handle, partial, graph_id=-1, stream=None):
    """Add an exact fixed-point BC vector ([n, 2] / [2n] uint64 or int64,
    host numpy or torch host/CUDA) into the handle's accumulated BC."""
    if hasattr(partial, "data_ptr"):
        p, keep = _ptr(partial)
    else:
        p, keep = _ptr(np.ascontiguousarray(partial, dtype=np.uint64))
    _check(load().bc_add_fixed(handle, p, int(graph_id), _stream(stream)), handle)


def bc_partition(handle, part=None, P=2, stream=None):
    """Split the handle's graph into P parts (part: int32[n] host/device, or
    None for P contiguous ranges) and build its border matrices."""
    if part is None:
        _check(load().bc_partition(handle, None, int(P), _stream(stream)), handle)
        return
    pp, keep = _ptr(_as_i32(part))
    _check(load().bc_partition(handle, pp, int(P), _stream(stream)), handle)


def bc_partition_info(handle) -> dict:
    s = gbbc_partition_info()
    _check(load().bc_partition_info(handle, ctypes.byref(s)), handle)
    return {k: getattr(s, k) for k, _ in s._fields_}


def bc_read_border_matrix(handle, p):
    """(border ids, BM [b, b] int32, sigmaM mod 2^64 [b, b] uint64, overflow [b, b] uint8) of part p."""
    lib = load()
    cnt = ctypes.c_int64()
    _check(lib.bc_read_border_matrix(handle, int(p), ctypes.byref(cnt), None, None, None, None), handle)
    b = cnt.value
    ids = np.zeros(max(b, 1), np.int32)
    bm = np.zeros((b, b), np.int32)
    sm = np.zeros((b, b), np.uint64)
    ov = np.zeros((b, b), np.uint8)
    if b:
        _check(lib.bc_read_border_matrix(handle, int(p), None, ids.ctypes.data, bm.ctypes.data, sm.ctypes.data,
                                         ov.ctypes.data), handle)
    return ids[:b].copy(), bm, sm, ov


def bc_compute_partitioned(handle, sources, stream=None):
    src = _as_i32(sources)
    p, keep = _ptr(src)
    _check(load().bc_compute_partitioned(handle, p, len(src), _stream(stream)), handle)


def bc_read_source_state(handle, source_index, n):
    dist = np.zeros(int(n), np.int32)
    sig = np.zeros(int(n), np.uint64)
    ovf = np.zeros(int(n), np.uint8)
    _check(load().bc_read_source_state(handle, int(source_index), dist.ctypes.data, sig.ctypes.data,
                                       ovf.ctypes.data), handle)
    return dist, sig, ovf


def bc_reset(handle):
    _check(load().bc_reset(handle), handle)


def bc_sync(handle):
    _check(load().bc_sync(handle), handle)


def bc_graph_destroy(handle):
    if handle:
        load().bc_graph_destroy(handle)


def bc_status_string(status):
    return status_name(status)


def bc_last_error_detail(handle=None):
    return last_error(handle)


def bc_get_stats(handle) -> dict:
    s = gbbc_stats()
    _check(load().bc_get_stats(handle, ctypes.byref(s)), handle)
    return s.as_dict()


TRACE_FIELDS = [f for f, _ in gbbc_level_trace._fields_]


def bc_get_trace(handle) -> dict:
    """Per-level trace records as a dict of numpy arrays (one entry per field;
    "features" is an [n, 6] float32 array)."""
    lib = load()
    cnt = ctypes.c_int64()
    _check(lib.bc_get_trace(handle, None, 0, ctypes.byref(cnt)), handle)
    arr = (gbbc_level_trace * max(cnt.value, 1))()
    _check(lib.bc_get_trace(handle, arr, cnt.value, ctypes.byref(cnt)), handle)
    recs = arr[: cnt.value]
    out = {f: np.array([getattr(r, f) for r in recs]) for f in TRACE_FIELDS if f != "features"}
    out["features"] = np.array([list(r.features) for r in recs], np.float32).reshape(-1, 6)
    return out


def bc_clear_trace(handle):
    _check(load().bc_clear_trace(handle), handle)


def bc_get_profile(handle) -> dict:
    """{kind: {"launches", "ms", "bytes"}} for the traced steps."""
    lib = load()
    arr = (gbbc_kernel_profile * 16)()
    cnt = ctypes.c_int32()
    _check(lib.bc_get_profile(handle, arr, 16, ctypes.byref(cnt)), handle)
    return {arr[i].name.decode(): {"launches": arr[i].launches, "ms": arr[i].ms, "bytes": arr[i].bytes}
            for i in range(cnt.value)}


# ---- learned direction policy ------------------------------------------------

def bc_mlp_param_count(k_out=2):
    return int(load().bc_mlp_param_count(int(k_out)))


def _dev_f32(t):
    import torch
    return torch.as_tensor(t, dtype=torch.float32).cuda().contiguous()


def bc_mlp_forward(params, x, k_out=2, stream=None):
    """Network outputs [n, k_out] (FP32) for device or host inputs; returns a CUDA tensor."""
    import torch
    p, xs = _dev_f32(params), _dev_f32(x).reshape(-1, 6)
    out = torch.zeros(xs.shape[0], k_out, dtype=torch.float32, device=xs.device)
    _check(load().bc_mlp_forward(p.data_ptr(), k_out, xs.data_ptr(), xs.shape[0], out.data_ptr(), _stream(stream)))
    return out


def bc_mlp_loss_grad(params, x, target, weight=None, k_out=2, loss_kind=0, stream=None):
    """(loss, grad) of the weighted loss over all samples."""
    import torch
    p, xs, ts = _dev_f32(params), _dev_f32(x).reshape(-1, 6), _dev_f32(target)
    ws = _dev_f32(weight) if weight is not None else None
    grad = torch.zeros_like(p)
    loss = torch.zeros(1, dtype=torch.float32, device=p.device)
    _check(load().bc_mlp_loss_grad(p.data_ptr(), k_out, xs.data_ptr(), ts.data_ptr(),
                                   ws.data_ptr() if ws is not None else None, xs.shape[0], loss_kind,
                                   grad.data_ptr(), loss.data_ptr(), _stream(stream)))
    return float(loss.item()), grad


def bc_mlp_adam_step(params, grad, m, v, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    """In-place Adam step on CUDA float32 tensors."""
    _check(load().bc_mlp_adam_step(params.data_ptr(), grad.data_ptr(), m.data_ptr(), v.data_ptr(), params.numel(),
                                   lr, beta1, beta2, eps, int(t), _stream(stream)))


def bc_mlp_train(params, x, target, weight=None, k_out=2, loss_kind=0, epochs=500, lr=3e-3, stream=None):
    """Train in place on the device; returns (params tensor, loss history)."""
    import torch
    p, xs, ts = _dev_f32(params), _dev_f32(x).reshape(-1, 6), _dev_f32(target)
    ws = _dev_f32(weight) if weight is not None else None
    hist = torch.zeros(max(int(epochs), 1), dtype=torch.float32, device=p.device)
    _check(load().bc_mlp_train(p.data_ptr(), k_out, xs.data_ptr(), ts.data_ptr(),
                               ws.data_ptr() if ws is not None else None, xs.shape[0], loss_kind, int(epochs),
                               float(lr), hist.data_ptr(), _stream(stream)))
    return p, hist[: int(epochs)].cpu().numpy()


def bc_policy_eval(params, x, stream=None):
    """Inference path of the level loop (FP16 weights, FP32 sums): (logits, choice)."""
    import torch
    p, xs = _dev_f32(params), _dev_f32(x).reshape(-1, 6)
    n = xs.shape[0]
    logits = torch.zeros(n, 2, dtype=torch.float32, device=p.device)
    choice = torch.zeros(n, dtype=torch.int32, device=p.device)
    _check(load().bc_policy_eval(p.data_ptr(), xs.data_ptr(), n, logits.data_ptr(), choice.data_ptr(),
                                 _stream(stream)))
    return logits.cpu().numpy(), choice.cpu().numpy()


def bc_policy_load(handle, params):
    """Load FP32 direction-network parameters (numpy or tensor) into a handle; None unloads."""
    if params is None:
        _check(load().bc_policy_load(handle, None, 0), handle)
        return
    if hasattr(params, "data_ptr"):
        t = params.to(dtype=__import__("torch").float32).contiguous()
        _check(load().bc_policy_load(handle, t.data_ptr(), t.numel() * 4), handle)
    else:
        a = np.ascontiguousarray(params, dtype=np.float32)
        _check(load().bc_policy_load(handle, a.ctypes.data, a.nbytes), handle)


def bc_source_features(handle, sources, stream=None):
    """Grouping features [k, 6] (float32) of the given sources."""
    src = np.ascontiguousarray(sources, dtype=np.int32)
    out = np.zeros((len(src), 6), np.float32)
    _check(load().bc_source_features(handle, src.ctypes.data, len(src), out.ctypes.data, _stream(stream)), handle)
    return out


def bc_grouping_scores(handle, sources, stream=None):
    """Scores [k] (float32) the loaded grouping network gives the sources."""
    src = np.ascontiguousarray(sources, dtype=np.int32)
    out = np.zeros(len(src), np.float32)
    _check(load().bc_grouping_scores(handle, src.ctypes.data, len(src), out.ctypes.data, _stream(stream)), handle)
    return out


def bc_release_memory(device=-1):
    """Return the library pool's unused device memory to the driver."""
    _check(load().bc_release_memory(int(device)))


def bc_grouping_load(handle, params):
    """Load FP32 grouping-network parameters (k_out = 1); None unloads."""
    if params is None:
        _check(load().bc_grouping_load(handle, None, 0), handle)
        return
    a = np.ascontiguousarray(params, dtype=np.float32)
    _check(load().bc_grouping_load(handle, a.ctypes.data, a.nbytes), handle)


def bc_compute_noalloc(n, nnz, row_ptr, col, sources, bc_out, stream=None):
    """Add the BC dependencies of `sources` (host int32) into bc_out (device
    float64[n]) for the CSR in device memory, without allocating anything
    in the library: for callers that may not allocate memory (see the C
    header for the shared static scratch and its limits)."""
    src = np.ascontiguousarray(sources, dtype=np.int32)
    rp, k1 = _ptr(row_ptr)
    cl, k2 = _ptr(col)
    out, k3 = _ptr(bc_out)
    st = load().bc_compute_noalloc(int(n), int(nnz), rp, cl, src.ctypes.data, len(src), out, _stream(stream))
    if st != GBBC_OK:
        raise GbbcError(st, "bc_compute_noalloc")


# ---- convenience object ------------------------------------------------------

class BC:
    """Owning wrapper of one handle.

        with BC.from_graph(g, batch_width=64) as bc:
            bc.compute(sources)
            scores = bc.read()
    """

    def __init__(self, handle, n, offsets=None):
        self.h = handle
        self.n = int(n)
        self.offsets = offsets

    @classmethod
    def from_csr(cls, n, row_ptr, col, stream=None, **opts):
        nnz = int(row_ptr[-1]) if len(row_ptr) else 0
        return cls(bc_graph_create(n, nnz, row_ptr, col, options(**opts), stream), n)

    @classmethod
    def from_graph(cls, g, stream=None, **opts):
        return cls.from_csr(g.n, g.row_ptr, g.col, stream=stream, **opts)

    @classmethod
    def from_weighted(cls, n, row_ptr, col, weight, stream=None, **opts):
        """A weighted graph: weight[p] is the length of CSR entry p's edge."""
        nnz = int(row_ptr[-1]) if len(row_ptr) else 0
        return cls(bc_graph_create_weighted(n, nnz, row_ptr, col, weight, options(**opts), stream), n)

    @classmethod
    def from_graphs(cls, graphs, stream=None, **opts):
        ns = [g.n for g in graphs]
        h = bc_graph_create_multi(ns, [g.nnz for g in graphs], [g.row_ptr for g in graphs],
                                  [g.col for g in graphs], options(**opts), stream)
        offs = np.concatenate([[0], np.cumsum(ns)]).astype(np.int64)
        return cls(h, int(offs[-1]), offs)

    def compute(self, sources, stream=None):
        bc_compute(self.h, sources, stream=stream)
        return self

    def compute_multi(self, graph_id, local_src, stream=None):
        bc_compute_multi(self.h, graph_id, local_src, stream=stream)
        return self

    def read(self, out=None, graph_id=-1, stream=None):
        n = self.n if graph_id < 0 else int(self.offsets[graph_id + 1] - self.offsets[graph_id])
        return bc_read(self.h, n, out, graph_id, stream)

    def read_fixed(self, graph_id=-1, stream=None):
        n = self.n if graph_id < 0 else int(self.offsets[graph_id + 1] - self.offsets[graph_id])
        return bc_read_fixed(self.h, n, graph_id, stream)

    def read_fixed_into(self, out, graph_id=-1, stream=None):
        return bc_read_fixed_into(self.h, out, graph_id, stream)

    def add_fixed(self, partial, graph_id=-1, stream=None):
        bc_add_fixed(self.h, partial, graph_id, stream)
        return self

    def partition(self, part=None, P=2, stream=None):
        bc_partition(self.h, part, P, stream)
        return self

    def partition_info(self):
        return bc_partition_info(self.h)

    def border_matrix(self, p):
        return bc_read_border_matrix(self.h, p)

    def compute_partitioned(self, sources, stream=None):
        bc_compute_partitioned(self.h, sources, stream=stream)
        return self

    def source_state(self, i):
        return bc_read_source_state(self.h, i, self.n)

    def reset(self):
        bc_reset(self.h)

    def sync(self):
        bc_sync(self.h)

    def stats(self):
        return bc_get_stats(self.h)

    def trace(self):
        return bc_get_trace(self.h)

    def profile(self):
        return bc_get_profile(self.h)

    def clear_trace(self):
        bc_clear_trace(self.h)

    def load_policy(self, params):
        bc_policy_load(self.h, params)
        return self

    def load_grouping(self, params):
        bc_grouping_load(self.h, params)
        return self

    def source_features(self, sources):
        return bc_source_features(self.h, sources)

    def grouping_scores(self, sources):
        return bc_grouping_scores(self.h, sources)

    def close(self):
        if self.h:
            bc_graph_destroy(self.h)
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
