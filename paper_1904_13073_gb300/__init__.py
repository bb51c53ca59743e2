"""Python binding of the SurfelWarp GB300 library (``include/surfelwarp.h``).

Argument marshalling only: every function here has the name of the C entry
point it calls, converts numpy arrays / torch tensors to pointers, and raises
``SwError`` with the library's message when a call returns an error.  All
computation runs in the CUDA library; if it cannot be loaded, every call
fails loudly (there is no fallback).
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# SW_BOUNDS_CHECK=1 selects the checked build (kernels range-check the
# indices they read or derive on the device; see build.py)
CHECKED_BUILD = os.environ.get("SW_BOUNDS_CHECK", "") == "1"
LIB_PATH = os.path.join(HERE, "libsurfelwarp_checked.so" if CHECKED_BUILD else "libsurfelwarp.so")

SW_MAX_GN_ITERS = 16
SW_MAX_PCG_ITERS = 128
SW_MAX_RIGID_ITERS = 16
SW_PRECISION_MIXED = 0           # FP32 solve, double-float PCG inner products, FP64 6x6 inverses
SW_PRECISION_FP64 = 1            # the whole solve in FP64
SW_PRECISION_MIXED_F64DOTS = 2   # FP32 solve, FP64 PCG inner products, FP64 6x6 inverses

STATUS = {0: "SW_OK", 1: "SW_ERR_INVALID_ARG", 2: "SW_ERR_NO_MEMORY", 3: "SW_ERR_NOT_INITIALIZED",
          4: "SW_ERR_SOLVER_BREAKDOWN", 5: "SW_ERR_TIMEOUT", 6: "SW_ERR_CUDA",
          7: "SW_ERR_BOUNDS"}


class SwError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class sw_params(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int), ("height", ctypes.c_int),
                ("fx", ctypes.c_float), ("fy", ctypes.c_float), ("cx", ctypes.c_float), ("cy", ctypes.c_float),
                ("max_surfels", ctypes.c_int), ("max_nodes", ctypes.c_int),
                ("lambda_", ctypes.c_float), ("fuse_dist", ctypes.c_float), ("fuse_normal", ctypes.c_float),
                ("corr_dist", ctypes.c_float), ("corr_normal", ctypes.c_float), ("stable_conf", ctypes.c_float),
                ("recent_frames", ctypes.c_int), ("precision", ctypes.c_int), ("visibility", ctypes.c_int),
                ("eps", ctypes.c_float), ("delta_nn", ctypes.c_float), ("fd_step", ctypes.c_float),
                ("t_low_confid", ctypes.c_int), ("extend_nodes", ctypes.c_int)]


class sw_solve_stats(ctypes.Structure):
    _fields_ = [("gn_iters", ctypes.c_int),
                ("e_depth", ctypes.c_double * SW_MAX_GN_ITERS),
                ("e_reg", ctypes.c_double * SW_MAX_GN_ITERS),
                ("n_corr", ctypes.c_int * SW_MAX_GN_ITERS),
                ("pcg_rz", ctypes.c_double * SW_MAX_GN_ITERS)]

    def as_dict(self):
        n = self.gn_iters
        return {"gn_iters": n, "e_depth": list(self.e_depth[:n]), "e_reg": list(self.e_reg[:n]),
                "n_corr": list(self.n_corr[:n]), "pcg_rz": list(self.pcg_rz[:n])}


class sw_append_stats(ctypes.Structure):
    _fields_ = [("candidates", ctypes.c_int), ("rejected_nn", ctypes.c_int), ("rejected_strain", ctypes.c_int),
                ("appended", ctypes.c_int), ("removed", ctypes.c_int), ("n_surfels", ctypes.c_int),
                ("kernel_ms", ctypes.c_double), ("rebuild_ms", ctypes.c_double), ("new_nodes", ctypes.c_int),
                ("resorted", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class sw_frame_result(ctypes.Structure):
    _fields_ = [("stream", ctypes.c_int), ("frame_id", ctypes.c_int), ("status", ctypes.c_int),
                ("batch_size", ctypes.c_int), ("submit_ms", ctypes.c_double), ("start_ms", ctypes.c_double),
                ("done_ms", ctypes.c_double), ("appended", ctypes.c_int), ("n_surfels", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class sw_server_stats(ctypes.Structure):
    _fields_ = [("admitted", ctypes.c_int), ("waiting", ctypes.c_int), ("steps", ctypes.c_longlong),
                ("frames", ctypes.c_longlong), ("busy_ms", ctypes.c_double), ("memory_in_use", ctypes.c_size_t),
                ("steps_alone", ctypes.c_longlong)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None

_P = ctypes.c_void_p
_I = ctypes.c_int
_SIGS = {
    "sw_params_default": [ctypes.POINTER(sw_params), _I, _I, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                          ctypes.c_float, _I, _I],
    "sw_create_stream": [ctypes.POINTER(sw_params), _P, ctypes.POINTER(_P)],
    "sw_destroy_stream": [_P],
    "sw_set_memory_budget": [ctypes.c_size_t],
    "sw_set_model": [_P, _P, _P, _P, _I, _P, _I],
    "sw_upload_depth": [_P, _P, _I, _I],
    "sw_solve_frame": [_P, _I, _I, ctypes.POINTER(sw_solve_stats)],
    "sw_fuse_frame": [_P],
    "sw_read_nodes": [_P, _P, _P, _I, ctypes.POINTER(_I)],
    "sw_read_surfels": [_P, _P, _P, _P, _I, ctypes.POINTER(_I)],
    "sw_read_live_surfels": [_P, _P, _P, _I, ctypes.POINTER(_I)],
    "sw_read_skinning": [_P, _P, _P, _I, ctypes.POINTER(_I)],
    "sw_read_graph": [_P, _P, _I],
    "sw_read_maps": [_P, _P, _P],
    "sw_debug_set_maps": [_P, _P, _P],
    "sw_set_node_dq": [_P, _P, _I],
    "sw_read_correspondence": [_P, _P, _I, ctypes.POINTER(_I)],
    "sw_debug_set_live": [_P, _P, _P, _I],
    "sw_debug_associate": [_P],
    "sw_debug_fusion_targets": [_P, _P, _P],
    "sw_debug_visibility": [_P, _P, _P],
    "sw_debug_assemble": [_P, ctypes.POINTER(_I), ctypes.POINTER(_I)],
    "sw_debug_read_jtj": [_P, _P, _P, _P, _P, _I],
    "sw_export_state": [_P, _P, ctypes.POINTER(ctypes.c_size_t)],
    "sw_import_state": [_P, _P, ctypes.c_size_t],
    "sw_fusion_targets_static": [_P, _P, _I, _P, _P, _I, _I, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                 ctypes.c_float, ctypes.c_float, ctypes.c_float, _P, _P],
    "sw_batch_create": [ctypes.POINTER(_P), _I, _P, ctypes.POINTER(_P)],
    "sw_batch_destroy": [_P],
    "sw_batch_set_active": [_P, ctypes.POINTER(_I)],
    "sw_batch_upload_depth": [_P, ctypes.POINTER(_P), _I, ctypes.POINTER(_I)],
    "sw_batch_solve": [_P, _I, _I, ctypes.POINTER(sw_solve_stats)],
    "sw_batch_fuse": [_P],
    "sw_set_profiling": [_P, _I],
    "sw_read_profile": [_P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_I)],
    "sw_batch_set_profiling": [_P, _I],
    "sw_batch_read_profile": [_P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_I)],
    "sw_debug_inject_wait_fault": [_I, _I],
    "sw_debug_set_pcg_mode": [_I],
    "sw_debug_pcg_mode": [_P, ctypes.POINTER(_I)],
    "sw_batch_debug_pcg_mode": [_P, ctypes.POINTER(_I)],
    "sw_read_visibility": [_P, _P, _I, ctypes.POINTER(_I)],
    "sw_debug_cluster_barrier_us": [_I, ctypes.POINTER(ctypes.c_double)],
    "sw_debug_pcg_cluster": [_P, _I, _I, ctypes.c_size_t, ctypes.POINTER(_I), ctypes.POINTER(ctypes.c_size_t),
                             ctypes.POINTER(_I)],
    "sw_debug_cluster_plan": [_I, _I, _P, _P, _P, ctypes.c_size_t, _P, ctypes.c_size_t,
                              ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_size_t)],
    "sw_debug_block_inverse": [_P, _I, _I, _P, _P],
    "sw_debug_scan": [_P, _I, _I, _P],
    "sw_debug_set_skin_node": [_P, _I, _I, _I],
    "sw_debug_record_correspondence": [_P, _I],
    "sw_read_correspondence_iter": [_P, _I, _P, _I, ctypes.POINTER(_I)],
    "sw_debug_radix_sort": [_I, _P, _P, _I, _I, _I, _P, _P],
    "sw_server_create": [ctypes.c_size_t, _I, _I, _I, ctypes.POINTER(_P)],
    "sw_server_destroy": [_P],
    "sw_server_open": [_P, ctypes.POINTER(sw_params), _P, _P, _P, _I, _P, _I, ctypes.POINTER(_I)],
    "sw_server_close": [_P, _I],
    "sw_server_is_admitted": [_P, _I, ctypes.POINTER(_I)],
    "sw_server_submit": [_P, _I, _P, _I],
    "sw_server_poll": [_P, ctypes.POINTER(sw_frame_result), _I, ctypes.POINTER(_I)],
    "sw_server_wait": [_P, _I],
    "sw_server_read_nodes": [_P, _I, _P, _P, _I, ctypes.POINTER(_I)],
    "sw_server_read_stats": [_P, ctypes.POINTER(sw_server_stats)],
    "sw_server_set_batch_window": [_P, ctypes.c_double],
    "sw_server_set_appending": [_P, _I],
    "sw_server_set_plain": [_P, _I],
    "sw_server_set_adaptive": [_P, _I],
    "sw_autotune": [_P, _I, ctypes.POINTER(_I), ctypes.POINTER(ctypes.c_double)],
    "sw_rigid_align": [_P, _I, ctypes.POINTER(_I), ctypes.POINTER(ctypes.c_double)],
    "sw_batch_rigid_align": [_P, _I],
    "sw_batch_autotune": [_P, _I, ctypes.POINTER(_I), ctypes.POINTER(ctypes.c_double)],
    "sw_append_frame": [_P, ctypes.POINTER(sw_append_stats)],
    "sw_debug_read_append": [_P, _P, _P, _P, _P, _P, _P, _P, _P, _I, ctypes.POINTER(_I)],
}

PROFILE_STAGES = ("depth", "reg_assembly", "data_assembly", "pcg", "fusion", "visibility")


def exported_symbols():
    """Names of every entry point declared in include/surfelwarp.h."""
    return sorted(list(_SIGS) + ["sw_memory_in_use", "sw_last_error", "sw_status_string"])


def lib():
    """Load the in-tree CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run paper_1904_13073_gb300.build.build() "
                               "(the CUDA library is required; there is no CPU path)")
        L = ctypes.CDLL(LIB_PATH)
        for name, args in _SIGS.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int
        L.sw_memory_in_use.argtypes = []
        L.sw_memory_in_use.restype = ctypes.c_size_t
        L.sw_last_error.argtypes = [_P]
        L.sw_last_error.restype = ctypes.c_char_p
        L.sw_status_string.argtypes = [_I]
        L.sw_status_string.restype = ctypes.c_char_p
        _lib = L
    return _lib


def _check(status, handle=None):
    if status != 0:
        msg = lib().sw_last_error(handle)
        raise SwError(status, msg.decode() if msg else "")


def _ptr(a, dtype=None, shape_last=None):
    """Pointer of a C-contiguous numpy array (copied to ``dtype`` if needed),
    or of a torch tensor (data_ptr); None stays None."""
    if a is None:
        return None, None
    if hasattr(a, "data_ptr"):
        return ctypes.c_void_p(a.data_ptr()), a
    arr = np.ascontiguousarray(a, dtype=dtype)
    if shape_last is not None and arr.shape[-1] != shape_last:
        raise ValueError(f"expected last dimension {shape_last}, got {arr.shape}")
    return arr.ctypes.data_as(ctypes.c_void_p), arr


def _pad4(a, w):
    a = np.asarray(a, dtype=np.float32)
    if a.ndim == 1:
        a = a[:, None]
    out = np.empty((a.shape[0], 4), dtype=np.float32)
    out[:, :3] = a[:, :3]
    out[:, 3] = w
    return out


# --------------------------------------------------------------------------- calls

def sw_params_default(width, height, fx, fy, cx, cy, max_surfels, max_nodes):
    p = sw_params()
    _check(lib().sw_params_default(ctypes.byref(p), width, height, fx, fy, cx, cy, max_surfels, max_nodes))
    return p


def sw_set_memory_budget(nbytes):
    _check(lib().sw_set_memory_budget(nbytes))


def sw_memory_in_use():
    return int(lib().sw_memory_in_use())


def sw_create_stream(params, cuda_stream=None):
    """Returns an opaque handle (int).  ``cuda_stream``: a raw cudaStream_t
    (int), a torch.cuda.Stream, or None for a library-owned stream."""
    if cuda_stream is not None and hasattr(cuda_stream, "cuda_stream"):
        cuda_stream = cuda_stream.cuda_stream
    h = ctypes.c_void_p()
    _check(lib().sw_create_stream(ctypes.byref(params), ctypes.c_void_p(cuda_stream or 0), ctypes.byref(h)))
    return h.value


def sw_destroy_stream(h):
    _check(lib().sw_destroy_stream(h), h)


def sw_set_model(h, v4, n4, t2, node4):
    """v4 [n,4] x y z r; n4 [n,4] nx ny nz c; t2 [n,2] int32 or None; node4 [m,4] x y z σ."""
    pv, v4a = _ptr(v4, np.float32, 4)
    pn, n4a = _ptr(n4, np.float32, 4)
    pt, t2a = _ptr(t2, np.int32, 2)
    pnode, nodea = _ptr(node4, np.float32, 4)
    n = 0 if v4a is None else v4a.shape[0]
    _check(lib().sw_set_model(h, pv, pn, pt, n, pnode, nodea.shape[0]), h)


def sw_upload_depth(h, depth, frame_id):
    """depth: numpy (host) or a CUDA torch tensor (device), [H, W] float32."""
    on_device = hasattr(depth, "is_cuda") and depth.is_cuda
    if hasattr(depth, "data_ptr") and not on_device:
        depth = depth.numpy()
    p, keep = _ptr(depth, np.float32)
    _check(lib().sw_upload_depth(h, p, int(on_device), int(frame_id)), h)
    return keep


def sw_solve_frame(h, gn_iters, pcg_iters, want_stats=True):
    st = sw_solve_stats() if want_stats else None
    _check(lib().sw_solve_frame(h, gn_iters, pcg_iters, ctypes.byref(st) if st is not None else None), h)
    return st.as_dict() if st is not None else None


def sw_fuse_frame(h):
    _check(lib().sw_fuse_frame(h), h)


def _count_nodes(h):
    n = ctypes.c_int()
    _check(lib().sw_read_nodes(h, None, None, 0, ctypes.byref(n)), h)
    return n.value


def sw_read_nodes(h):
    """(pos4 [n,4], dq8 [n,8]) float32."""
    n = _count_nodes(h)
    pos = np.empty((n, 4), np.float32)
    dq = np.empty((n, 8), np.float32)
    cnt = ctypes.c_int()
    _check(lib().sw_read_nodes(h, pos.ctypes.data_as(_P), dq.ctypes.data_as(_P), n, ctypes.byref(cnt)), h)
    return pos, dq


def _count_surfels(h):
    n = ctypes.c_int()
    _check(lib().sw_read_surfels(h, None, None, None, 1 << 30, ctypes.byref(n)), h)
    return n.value


def sw_read_surfels(h):
    n = _count_surfels(h)
    v = np.empty((n, 4), np.float32)
    nn = np.empty((n, 4), np.float32)
    t = np.empty((n, 2), np.int32)
    _check(lib().sw_read_surfels(h, v.ctypes.data_as(_P), nn.ctypes.data_as(_P), t.ctypes.data_as(_P), n, None), h)
    return v, nn, t


def sw_read_live_surfels(h):
    n = _count_surfels(h)
    v = np.empty((n, 4), np.float32)
    nn = np.empty((n, 4), np.float32)
    _check(lib().sw_read_live_surfels(h, v.ctypes.data_as(_P), nn.ctypes.data_as(_P), n, None), h)
    return v, nn


def sw_read_skinning(h):
    n = _count_surfels(h)
    k = np.empty((n, 4), np.int32)
    w = np.empty((n, 4), np.float32)
    _check(lib().sw_read_skinning(h, k.ctypes.data_as(_P), w.ctypes.data_as(_P), n, None), h)
    return k, w


def sw_read_graph(h):
    m = _count_nodes(h)
    g = np.empty((m, 8), np.int32)
    _check(lib().sw_read_graph(h, g.ctypes.data_as(_P), m), h)
    return g


def sw_read_maps(h, height, width):
    V = np.empty((height, width, 4), np.float32)
    N = np.empty((height, width, 4), np.float32)
    _check(lib().sw_read_maps(h, V.ctypes.data_as(_P), N.ctypes.data_as(_P)), h)
    return V, N


def sw_debug_set_maps(h, V4, N4):
    pV, a = _ptr(V4, np.float32)
    pN, b = _ptr(N4, np.float32)
    _check(lib().sw_debug_set_maps(h, pV, pN), h)


def sw_set_node_dq(h, dq8):
    p, a = _ptr(dq8, np.float32, 8)
    _check(lib().sw_set_node_dq(h, p, a.shape[0]), h)


def sw_read_correspondence(h):
    n = _count_surfels(h)
    pix = np.empty(n, np.int32)
    _check(lib().sw_read_correspondence(h, pix.ctypes.data_as(_P), n, None), h)
    return pix


def sw_debug_record_correspondence(h, enable):
    _check(lib().sw_debug_record_correspondence(h, int(bool(enable))), h)


def sw_read_correspondence_iter(h, gn_iter):
    """The association of Gauss-Newton iteration gn_iter of the last solve (recording on)."""
    n = _count_surfels(h)
    pix = np.empty(n, np.int32)
    _check(lib().sw_read_correspondence_iter(h, int(gn_iter), pix.ctypes.data_as(_P), n, None), h)
    return pix


def sw_debug_set_live(h, v, n):
    pv, a = _ptr(_pad4(v, 0.0))
    pn, b = _ptr(_pad4(n, 0.0))
    _check(lib().sw_debug_set_live(h, pv, pn, a.shape[0]), h)


def sw_debug_visibility(h, height, width):
    """(vis_map (H, W) caller ids or -1, visible (n,) bool) of the stored live surfels."""
    n = _count_surfels(h)
    vm = np.empty((height, width), np.int32)
    vis = np.empty(max(1, n), np.int32)
    _check(lib().sw_debug_visibility(h, vm.ctypes.data_as(_P), vis.ctypes.data_as(_P)), h)
    return vm, vis[:n].astype(bool)


def sw_debug_associate(h):
    _check(lib().sw_debug_associate(h), h)


def sw_debug_fusion_targets(h, height, width):
    t = np.empty(height * width, np.int32)
    im = np.empty((4 * height, 4 * width), np.int32)
    _check(lib().sw_debug_fusion_targets(h, t.ctypes.data_as(_P), im.ctypes.data_as(_P)), h)
    return t, im


def sw_debug_assemble(h):
    nb, nc = ctypes.c_int(), ctypes.c_int()
    _check(lib().sw_debug_assemble(h, ctypes.byref(nb), ctypes.byref(nc)), h)
    return nb.value, nc.value


def sw_debug_read_jtj(h, nnzb, n_nodes):
    rows = np.empty(nnzb, np.int32)
    cols = np.empty(nnzb, np.int32)
    vals = np.empty((nnzb, 6, 6), np.float32)
    g = np.empty(6 * n_nodes, np.float32)
    _check(lib().sw_debug_read_jtj(h, rows.ctypes.data_as(_P), cols.ctypes.data_as(_P), vals.ctypes.data_as(_P),
                                   g.ctypes.data_as(_P), nnzb), h)
    return rows, cols, vals, g


def sw_export_state(h):
    n = ctypes.c_size_t()
    _check(lib().sw_export_state(h, None, ctypes.byref(n)), h)
    buf = np.empty(n.value, np.uint8)
    _check(lib().sw_export_state(h, buf.ctypes.data_as(_P), ctypes.byref(n)), h)
    return buf


def sw_import_state(h, buf):
    buf = np.ascontiguousarray(buf, dtype=np.uint8)
    _check(lib().sw_import_state(h, buf.ctypes.data_as(_P), buf.size), h)


def sw_fusion_targets_static(v_live4, n_live4, vmap4, nmap4, width, height, fx, fy, cx, cy,
                             fuse_dist, fuse_normal, target, cuda_stream=None):
    """Fusion targets with no device allocation (all arguments CUDA tensors
    the caller owns; see include/surfelwarp.h for the size limit and the rule
    that overlapping calls race).  Enqueued on ``cuda_stream``; no wait."""
    if cuda_stream is not None and hasattr(cuda_stream, "cuda_stream"):
        cuda_stream = cuda_stream.cuda_stream
    n = 0 if v_live4 is None else int(v_live4.shape[0])
    ptr = (lambda t: None if t is None else ctypes.c_void_p(t.data_ptr()))
    _check(lib().sw_fusion_targets_static(ptr(v_live4), ptr(n_live4), n, ptr(vmap4), ptr(nmap4), width, height,
                                          fx, fy, cx, cy, fuse_dist, fuse_normal, ptr(target),
                                          ctypes.c_void_p(cuda_stream or 0)))


_batch_sizes = {}


def sw_batch_create(handles, cuda_stream=None):
    if cuda_stream is not None and hasattr(cuda_stream, "cuda_stream"):
        cuda_stream = cuda_stream.cuda_stream
    arr = (_P * len(handles))(*handles)
    b = ctypes.c_void_p()
    _check(lib().sw_batch_create(arr, len(handles), ctypes.c_void_p(cuda_stream or 0), ctypes.byref(b)))
    _batch_sizes[b.value] = len(handles)
    return b.value


def sw_batch_destroy(b):
    _check(lib().sw_batch_destroy(b))
    _batch_sizes.pop(b, None)


def sw_batch_set_active(b, active):
    arr = (_I * len(active))(*[int(bool(a)) for a in active])
    _check(lib().sw_batch_set_active(b, arr))


def sw_batch_upload_depth(b, depths, frame_ids):
    """depths: list of numpy arrays (host), CUDA tensors (device) or None."""
    on_device = any(hasattr(d, "is_cuda") and d.is_cuda for d in depths if d is not None)
    keep, ptrs = [], []
    for d in depths:
        if d is None:
            ptrs.append(None)
            continue
        if hasattr(d, "data_ptr") and not on_device:
            d = d.numpy()
        p, k = _ptr(d, np.float32)
        keep.append(k)
        ptrs.append(p.value if p is not None else None)
    arr = (_P * len(depths))(*ptrs)
    ids = (_I * len(frame_ids))(*[int(f) for f in frame_ids])
    _check(lib().sw_batch_upload_depth(b, arr, int(on_device), ids))
    return keep


def sw_batch_solve(b, gn_iters, pcg_iters, want_stats=True):
    st = (sw_solve_stats * _batch_sizes[b])() if want_stats else None
    _check(lib().sw_batch_solve(b, gn_iters, pcg_iters, st))
    return [x.as_dict() for x in st] if st is not None else None


def sw_batch_fuse(b):
    _check(lib().sw_batch_fuse(b))


def sw_set_profiling(h, enable):
    _check(lib().sw_set_profiling(h, int(bool(enable))), h)


def _profile(fn, h, handle_for_error):
    ms = (ctypes.c_double * len(PROFILE_STAGES))()
    n = (_I * len(PROFILE_STAGES))()
    _check(fn(h, ms, n), handle_for_error)
    return {k: (ms[i], n[i]) for i, k in enumerate(PROFILE_STAGES)}


def sw_read_profile(h):
    """{stage: (milliseconds, launches)} of the last upload, solve and fusion."""
    return _profile(lib().sw_read_profile, h, h)


def sw_batch_set_profiling(b, enable):
    _check(lib().sw_batch_set_profiling(b, int(bool(enable))))


def sw_batch_read_profile(b):
    return _profile(lib().sw_batch_read_profile, b, None)


def sw_debug_block_inverse(blocks, fp64=False, mode=None):
    """(inverses (n, 21) packed lower, ok (n,) bool) of the PCG's block inverse on (n, 6, 6) blocks.
    mode 0: FP32 blocks, double-float arithmetic (the default precision); 1: FP64; 2: FP32 blocks,
    FP64 arithmetic.  Without mode, fp64 picks 1 or 0."""
    mode = (1 if fp64 else 0) if mode is None else int(mode)
    dt = np.float64 if mode == 1 else np.float32
    b = np.ascontiguousarray(np.asarray(blocks, dt).reshape(-1, 36))
    n = b.shape[0]
    out = np.empty((max(1, n), 21), dt)
    ok = np.empty(max(1, n), np.int32)
    _check(lib().sw_debug_block_inverse(b.ctypes.data_as(_P), n, mode, out.ctypes.data_as(_P),
                                        ok.ctypes.data_as(_P)), None)
    return out[:n], ok[:n].astype(bool)


def sw_debug_set_skin_node(h, surfel, slot, node):
    """Write one skinning node id of an internal-order surfel (checked-build test hook)."""
    _check(lib().sw_debug_set_skin_node(h, int(surfel), int(slot), int(node)), h)


def sw_debug_scan(values, inclusive=False):
    """The library's device prefix sum of an int32 array (exclusive unless inclusive)."""
    v = np.ascontiguousarray(np.asarray(values, np.int32).reshape(-1))
    out = np.empty(max(1, v.size), np.int32)
    _check(lib().sw_debug_scan(v.ctypes.data_as(_P), v.size, int(bool(inclusive)), out.ctypes.data_as(_P)), None)
    return out[:v.size]


def sw_debug_radix_sort(keys, values=None, begin_bit=0, end_bit=None):
    """The library's stable device radix sort of uint32 or uint64 keys by bits
    [begin_bit, end_bit); returns (sorted keys, their values or None)."""
    k = np.asarray(keys)
    if k.dtype not in (np.uint32, np.uint64):
        raise TypeError("keys must be uint32 or uint64")
    k = np.ascontiguousarray(k.reshape(-1))
    kb = k.dtype.itemsize
    end_bit = 8 * kb if end_bit is None else end_bit
    out = np.empty(max(1, k.size), k.dtype)
    vp, vout = None, None
    if values is not None:
        v = np.ascontiguousarray(np.asarray(values, np.int32).reshape(-1))
        if v.size != k.size:
            raise ValueError("values and keys differ in length")
        vout = np.empty(max(1, v.size), np.int32)
        vp = v.ctypes.data_as(_P)
    _check(lib().sw_debug_radix_sort(kb, k.ctypes.data_as(_P), vp, k.size, begin_bit, end_bit,
                                     out.ctypes.data_as(_P), None if vout is None else vout.ctypes.data_as(_P)),
           None)
    return out[:k.size], (None if vout is None else vout[:k.size])


# failure kinds of sw_debug_inject_wait_fault
SW_FAULT_NONE, SW_FAULT_PCG_PARTIAL, SW_FAULT_PCG_VECTOR, SW_FAULT_DEPTH_TMA = 0, 1, 2, 3


def sw_debug_inject_wait_fault(kind, spin_limit=0):
    """Make the product's bounded device waits run out (kind 0 turns it off)."""
    _check(lib().sw_debug_inject_wait_fault(int(kind), int(spin_limit)), None)


def sw_debug_set_pcg_mode(max_mode):
    """Cap the PCG's SpMV staging mode (2 = no cap) for launch plans built afterwards."""
    _check(lib().sw_debug_set_pcg_mode(int(max_mode)), None)


def sw_debug_pcg_mode(h):
    m = _I()
    _check(lib().sw_debug_pcg_mode(h, ctypes.byref(m)), h)
    return m.value


def sw_batch_debug_pcg_mode(b):
    m = _I()
    _check(lib().sw_batch_debug_pcg_mode(b, ctypes.byref(m)), None)
    return m.value


def sw_debug_cluster_plan(ctas, row_ptr, col, node4, smem_limit):
    """(plan int32 array, shared-memory bytes per CTA) of the cluster PCG for
    an upper block pattern (host code; raises SwError if it does not fit)."""
    rp = np.ascontiguousarray(row_ptr, np.int32)
    cl = np.ascontiguousarray(col, np.int32)
    nd = np.ascontiguousarray(node4, np.float32).reshape(-1, 4)
    n = len(rp) - 1
    size, smem = ctypes.c_size_t(), ctypes.c_size_t()
    args = (int(ctas), n, rp.ctypes.data_as(_P), cl.ctypes.data_as(_P), nd.ctypes.data_as(_P),
            int(smem_limit))
    _check(lib().sw_debug_cluster_plan(*args, None, 0, ctypes.byref(size), ctypes.byref(smem)), None)
    out = np.empty(max(1, size.value), np.int32)
    _check(lib().sw_debug_cluster_plan(*args, out.ctypes.data_as(_P), size.value, None, None), None)
    return out[:size.value], smem.value


def sw_debug_pcg_cluster(h=None, precision=0, ctas=16, smem=0):
    """(plan cluster size, plan shared memory per CTA, clusters of `ctas`
    CTAs with `smem` bytes that the device runs at once)."""
    c, b, a = _I(), ctypes.c_size_t(), _I()
    _check(lib().sw_debug_pcg_cluster(h, int(precision), int(ctas), int(smem), ctypes.byref(c), ctypes.byref(b),
                                      ctypes.byref(a)), h)
    return c.value, b.value, a.value


def sw_debug_cluster_barrier_us(ctas=16):
    """Microseconds of one cluster barrier of `ctas` CTAs of the cluster PCG's size."""
    us = ctypes.c_double()
    _check(lib().sw_debug_cluster_barrier_us(int(ctas), ctypes.byref(us)), None)
    return us.value


def sw_read_visibility(h):
    """Per surfel (caller order) 1 if the last solve's visibility prediction kept it."""
    n = _count_surfels(h)
    out = np.empty(max(1, n), np.int32)
    got = _I()
    _check(lib().sw_read_visibility(h, out.ctypes.data_as(_P), max(1, n), ctypes.byref(got)), h)
    return out[:got.value]


def sw_last_error(h=None):
    m = lib().sw_last_error(h)
    return m.decode() if m else ""


def sw_status_string(status):
    return lib().sw_status_string(status).decode()


# --------------------------------------------------------------------------- helpers

def params_for(cam, n_surfels, n_nodes, **over):
    """sw_params for a synth.Camera-like object with Table 1 defaults."""
    p = sw_params_default(cam.width, cam.height, cam.fx, cam.fy, cam.cx, cam.cy, max(1, n_surfels), n_nodes)
    for k, v in over.items():
        setattr(p, "lambda_" if k == "lam" else k, v)
    return p


def model_arrays(scene):
    """(v4, n4, t2, node4) of a synth.Scene in the library's layout."""
    return (_pad4(scene.surfel_v, scene.surfel_r), _pad4(scene.surfel_n, scene.surfel_c),
            np.ascontiguousarray(scene.surfel_t, dtype=np.int32), _pad4(scene.node_p, scene.node_sigma))


# ---------------------------------------------------------------- serving

def sw_server_create(memory_budget, gn_iters, pcg_iters, queue_depth=4):
    out = ctypes.c_void_p()
    _check(lib().sw_server_create(int(memory_budget), gn_iters, pcg_iters, queue_depth, ctypes.byref(out)))
    return out.value


def sw_server_destroy(srv):
    _check(lib().sw_server_destroy(srv))


def sw_server_open(srv, params, v4, n4, t2, node4):
    """Open a stream on the server; returns its id (admission happens later)."""
    v4 = np.ascontiguousarray(v4, np.float32)
    n4 = np.ascontiguousarray(n4, np.float32)
    node4 = np.ascontiguousarray(node4, np.float32)
    t2p = None
    if t2 is not None:
        t2 = np.ascontiguousarray(t2, np.int32)
        t2p = t2.ctypes.data_as(_P)
    sid = ctypes.c_int()
    _check(lib().sw_server_open(srv, ctypes.byref(params), v4.ctypes.data_as(_P), n4.ctypes.data_as(_P), t2p,
                                len(v4), node4.ctypes.data_as(_P), len(node4), ctypes.byref(sid)))
    return sid.value


def sw_server_close(srv, stream_id):
    _check(lib().sw_server_close(srv, stream_id))


def sw_server_is_admitted(srv, stream_id):
    a = ctypes.c_int()
    _check(lib().sw_server_is_admitted(srv, stream_id, ctypes.byref(a)))
    return bool(a.value)


def sw_server_submit(srv, stream_id, depth, frame_id):
    """Queue a frame; returns the sw_status (0 = queued, 2 = queue full,
    3 = not admitted yet) instead of raising for those two."""
    d = np.ascontiguousarray(depth, np.float32)
    st = lib().sw_server_submit(srv, stream_id, d.ctypes.data_as(_P), frame_id)
    if st not in (0, 2, 3):
        _check(st)
    return st


def sw_server_poll(srv, cap=4096):
    buf = (sw_frame_result * cap)()
    n = ctypes.c_int()
    _check(lib().sw_server_poll(srv, buf, cap, ctypes.byref(n)))
    return [buf[k].as_dict() for k in range(n.value)]


def sw_server_wait(srv, timeout_ms):
    return lib().sw_server_wait(srv, int(timeout_ms)) == 0


def sw_server_read_nodes(srv, stream_id, n_nodes):
    pos = np.empty((n_nodes, 4), np.float32)
    dq = np.empty((n_nodes, 8), np.float32)
    cnt = ctypes.c_int()
    _check(lib().sw_server_read_nodes(srv, stream_id, pos.ctypes.data_as(_P), dq.ctypes.data_as(_P), n_nodes,
                                      ctypes.byref(cnt)))
    return pos[:cnt.value], dq[:cnt.value]


def sw_server_set_batch_window(srv, window_ms):
    _check(lib().sw_server_set_batch_window(srv, float(window_ms)))


def sw_server_set_appending(s, enable):
    _check(lib().sw_server_set_appending(s, int(bool(enable))))


def sw_server_set_plain(s, enable):
    _check(lib().sw_server_set_plain(s, int(bool(enable))), None)


def sw_server_set_adaptive(s, enable):
    _check(lib().sw_server_set_adaptive(s, int(bool(enable))), None)


def sw_server_read_stats(srv):
    st = sw_server_stats()
    _check(lib().sw_server_read_stats(srv, ctypes.byref(st)))
    return st.as_dict()


# ---------------------------------------------------------------- autotuning

def sw_autotune(h, pcg_iters):
    """(rows per PCG CTA chosen, PCG microseconds per launch)."""
    r, us = ctypes.c_int(), ctypes.c_double()
    _check(lib().sw_autotune(h, pcg_iters, ctypes.byref(r), ctypes.byref(us)), h)
    return r.value, us.value


def sw_batch_autotune(b, pcg_iters):
    r, us = ctypes.c_int(), ctypes.c_double()
    _check(lib().sw_batch_autotune(b, pcg_iters, ctypes.byref(r), ctypes.byref(us)))
    return r.value, us.value


# ---------------------------------------------------------------- rigid pre-alignment

def sw_rigid_align(h, iters, want_stats=True):
    """Per iteration (correspondences, sum of squared residuals) before its
    update; without want_stats returns None and does not wait for the GPU."""
    if not want_stats:
        _check(lib().sw_rigid_align(h, iters, None, None), h)
        return None
    n = (_I * max(1, iters))()
    e = (ctypes.c_double * max(1, iters))()
    _check(lib().sw_rigid_align(h, iters, n, e), h)
    return [(n[k], e[k]) for k in range(iters)]


def sw_append_frame(h):
    """Appending and removal after fusion; returns the counts as a dict."""
    st = sw_append_stats()
    _check(lib().sw_append_frame(h, ctypes.byref(st)), h)
    return st.as_dict()


def sw_debug_read_append(h):
    """The per-candidate record of the last sw_append_frame (candidate order)."""
    n = _I(0)
    _check(lib().sw_debug_read_append(h, None, None, None, None, None, None, None, None, 0, ctypes.byref(n)), h)
    m = n.value
    out = {"pix": np.zeros(m, np.int32), "knn": np.zeros((m, 4), np.int32), "flags": np.zeros(m, np.int32),
           "wsum": np.zeros(m, np.float64), "strain": np.zeros((m, 3, 3), np.float64),
           "w": np.zeros((m, 4), np.float32), "v4": np.zeros((m, 4), np.float32), "n4": np.zeros((m, 4), np.float32)}
    if m:
        ptrs = [out[k].ctypes.data_as(ctypes.c_void_p) for k in ("pix", "knn", "flags", "wsum", "strain", "w", "v4", "n4")]
        _check(lib().sw_debug_read_append(h, *ptrs, m, ctypes.byref(n)), h)
    return out


def sw_batch_rigid_align(b, iters):
    _check(lib().sw_batch_rigid_align(b, iters))
