"""Python binding of the C ABI in include/heff.h (ctypes; argument marshalling only).

Every function named ``heff_*`` here calls the C function of the same name in the
in-tree ``libheff.so``; device buffers are passed as ``torch.Tensor`` (their
``data_ptr()``) and streams as ``torch.cuda.Stream`` (default: the current
stream).  If the library has not been built this module raises ImportError: there is
no fallback implementation.

``Layout`` and ``Plan`` are small owners of the C handles with helpers to move block
tensors between a per-block description and the flat buffer layout.
"""
import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBPATH = os.path.join(_HERE, "libheff.so")
if not os.path.exists(_LIBPATH):
    raise ImportError(f"{_LIBPATH} is missing: build it with "
                      "`python -c 'import __graft_entry__ as g; g.build()'`")
_lib = C.CDLL(_LIBPATH)

HEFF_OK = 0
PREC = {"fp64": 0, "bf16x3": 1, "tf32x3": 2}
DTYPE = {"f64": 0, "f32": 1}
ERRORS = {-1: "INVALID_ARG", -2: "CHARGE_MISMATCH", -3: "UNSUPPORTED", -4: "OOM", -5: "CUDA",
          -6: "TIMEOUT", -7: "WORKSPACE"}


class HeffError(RuntimeError):
    def __init__(self, code, what):
        self.code = code
        super().__init__(f"{what} failed with {ERRORS.get(code, code)}: "
                         f"{_lib.heff_last_error().decode()}")


class _Index(C.Structure):
    _fields_ = [("nsec", C.c_int32), ("nq", C.c_int32), ("charges", C.POINTER(C.c_int32)),
                ("dims", C.POINTER(C.c_int32)), ("flow", C.c_int32)]


class _Opts(C.Structure):
    _fields_ = [("precision", C.c_int32), ("io_dtype", C.c_int32), ("max_batch", C.c_int32),
                ("shard_count", C.c_int32), ("shard_index", C.c_int32), ("reserved", C.c_int32 * 3)]


_vp, _i32, _i64, _sz = C.c_void_p, C.c_int32, C.c_int64, C.c_size_t
_P = C.POINTER
_sig = {
    "heff_qn_block_layout": (C.c_int, [_P(_Index), _i32, _P(_i32), _P(_vp)]),
    "heff_layout_info": (C.c_int, [_vp, _P(_i64), _P(_i64), _P(_i32)]),
    "heff_layout_blocks": (C.c_int, [_vp, _P(_i32), _P(_i64)]),
    "heff_layout_destroy": (None, [_vp]),
    "heff_plan_create": (C.c_int, [_vp, _vp, _vp, _vp, _vp, _P(C.c_double), _P(C.c_double),
                                   _P(_Opts), _P(_vp)]),
    "heff_plan_workspace_size": (C.c_int, [_vp, _P(_sz)]),
    "heff_plan_shard_sectors": (C.c_int, [_vp, _P(C.c_int32), _P(C.c_int32)]),
    "heff_plan_select_tiles": (C.c_int, [_vp, C.c_int32, C.c_int32]),
    "heff_two_site_create": (C.c_int, [_vp, _vp, _vp, _P(_vp)]),
    "heff_svd_info": (C.c_int, [_vp, _P(C.c_int32), _P(C.c_int32)]),
    "heff_davidson_workspace_size": (C.c_int, [_vp, C.c_int32, _P(_sz)]),
    "heff_apply_host_staging_size": (C.c_int, [_vp, _P(_sz)]),
    "heff_apply_host": (C.c_int, [_vp] * 8 + [_sz, _vp, _sz, _vp]),
    "heff_davidson": (C.c_int, [_vp] * 7 + [C.c_int32, C.c_double, _vp, _vp, _vp, _sz, _vp, _sz, _vp]),
    "heff_two_site_apply": (C.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "heff_two_site_destroy": (None, [_vp]),
    "heff_plan_flops": (C.c_int, [_vp, _P(C.c_double), _P(C.c_double)]),
    "heff_plan_stats": (C.c_int, [_vp, _P(_i64)]),
    "heff_plan_export": (C.c_int, [_vp, _i32, _vp, _P(_i64)]),
    "heff_plan_destroy": (None, [_vp]),
    "heff_prepare": (C.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, _sz, _vp]),
    "heff_apply_prepared": (C.c_int, [_vp, _vp, _vp, _vp, _sz, _vp]),
    "heff_apply": (C.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _sz, _vp]),
    "heff_apply_batched": (C.c_int, [_vp, _vp, _vp, _vp, _vp, _P(_vp), _P(_vp), _i32, _vp, _sz, _vp]),
    "heff_apply_noalloc": (C.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "heff_apply_noalloc_status": (C.c_int, [_vp, _vp]),
    "heff_svd_create": (C.c_int, [_vp, _P(_vp)]),
    "heff_svd_workspace_size": (C.c_int, [_vp, _P(_sz)]),
    "heff_svd_compute": (C.c_int, [_vp, _vp, _vp, _sz, _vp, _P(_i32)]),
    "heff_svd_truncate": (C.c_int, [_vp, _i32, C.c_double, _P(_i32), _P(_i32), _P(_i32), _P(C.c_double),
                                    _P(C.c_double)]),
    "heff_svd_singular_values": (C.c_int, [_vp, _P(C.c_double)]),
    "heff_svd_write": (C.c_int, [_vp, _vp, _vp, _vp, _vp, _i32, _vp, _sz, _vp]),
    "heff_svd_destroy": (None, [_vp]),
    "heff_grad_plan_create": (C.c_int, [_vp, _vp, _vp, _vp, _vp, _P(C.c_double), _P(C.c_double), _sz, _P(_vp)]),
    "heff_grad_chunks": (C.c_int, [_vp, _P(C.c_int32)]),
    "heff_grad_workspace_size": (C.c_int, [_vp, _P(_sz)]),
    "heff_backward": (C.c_int, [_vp] * 13 + [_vp, _sz, _vp, _sz, _vp]),
    "heff_grad_plan_destroy": (None, [_vp]),
    "heff_grad_plan_set_precision": (C.c_int, [_vp, _i32]),
    "heff_grad_status": (C.c_int, [_vp, _vp, _sz, _vp]),
    "heff_env_plan_create": (C.c_int, [_vp, _vp, _vp, _vp, _P(C.c_double), _i32, _P(_vp)]),
    "heff_env_workspace_size": (C.c_int, [_vp, _P(_sz)]),
    "heff_env_flops": (C.c_int, [_vp, _P(C.c_double)]),
    "heff_env_update": (C.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, _sz, _vp]),
    "heff_env_plan_destroy": (None, [_vp]),
    "heff_env_plan_set_precision": (C.c_int, [_vp, _i32]),
    "heff_env_status": (C.c_int, [_vp, _vp, _sz, _vp]),
    "heff_lanczos_workspace_size": (C.c_int, [_vp, _i32, _P(_sz)]),
    "heff_ground_state_workspace_size": (C.c_int, [_vp, _i32, _P(_sz)]),
    "heff_ground_state": (C.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _i32, _i32, C.c_double, _vp,
                                     _P(C.c_double), _vp, _sz, _vp, _sz, _vp, _sz, _vp]),
    "heff_lanczos": (C.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, _i32, _vp, _vp, _vp, _sz, _vp, _sz, _vp]),
    "heff_plan_autotune": (C.c_int, [_vp] * 8 + [_sz, _vp, _P(_i32), _P(C.c_float)]),
    "heff_plan_set_timing": (C.c_int, [_vp, _i32]),
    "heff_plan_check_mpo": (C.c_int, [_vp, _vp, _vp, _vp, _P(_i64)]),
    "heff_plan_timings": (C.c_int, [_vp, _P(C.c_float)]),
    "heff_workspace_status": (C.c_int, [_vp, _vp, _sz, _vp]),
    "heff_wait_selftest": (C.c_int, [_vp, _vp, _sz, _i32, _vp, _P(C.c_float)]),
    "heff_last_error": (C.c_char_p, []),
    "heff_launch_count": (C.c_int64, []),
    "heff_version": (C.c_char_p, []),
}
for _name, (_res, _args) in _sig.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args

EXPORTED = tuple(_sig)


def _check(rc, what):
    if rc != HEFF_OK:
        raise HeffError(rc, what)


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _nbytes(t):
    return t.numel() * t.element_size()


def _stream(s):
    if s is None:
        import torch
        s = torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


# ------------------------------------------------------------------ C-named functions
def heff_qn_block_layout(indices, target=None):
    """indices: list of (charges [nsec, nq] int, dims [nsec] int, flow +-1)."""
    keep = []
    arr = (_Index * len(indices))()
    nq = None
    for k, (q, d, flow) in enumerate(indices):
        q = np.ascontiguousarray(np.asarray(q, dtype=np.int32).reshape(len(d), -1))
        d = np.ascontiguousarray(np.asarray(d, dtype=np.int32))
        nq = q.shape[1]
        keep += [q, d]
        arr[k] = _Index(len(d), nq, q.ctypes.data_as(_P(_i32)), d.ctypes.data_as(_P(_i32)), int(flow))
    tgt = None
    if target is not None:
        t = np.ascontiguousarray(np.asarray(target, dtype=np.int32).reshape(-1))
        keep.append(t)
        tgt = t.ctypes.data_as(_P(_i32))
    out = _vp()
    _check(_lib.heff_qn_block_layout(arr, len(indices), tgt, C.byref(out)), "heff_qn_block_layout")
    return out


def heff_layout_info(lay):
    nb, ne, ni = _i64(), _i64(), _i32()
    _check(_lib.heff_layout_info(lay, C.byref(nb), C.byref(ne), C.byref(ni)), "heff_layout_info")
    return nb.value, ne.value, ni.value


def heff_layout_blocks(lay):
    nb, ne, ni = heff_layout_info(lay)
    keys = np.zeros((nb, ni), dtype=np.int32)
    offs = np.zeros(nb, dtype=np.int64)
    _check(_lib.heff_layout_blocks(lay, keys.ctypes.data_as(_P(_i32)), offs.ctypes.data_as(_P(_i64))),
           "heff_layout_blocks")
    return keys, offs


def heff_layout_destroy(lay):
    _lib.heff_layout_destroy(lay)


def heff_plan_create(L, W1, W2, R, x, W1_host, W2_host, precision="bf16x3", io_dtype="f32",
                     max_batch=1, shard=None):
    """shard = (index, count) builds the plan of one row shard (left sectors of y)."""
    w1 = np.ascontiguousarray(W1_host, dtype=np.float64)
    w2 = np.ascontiguousarray(W2_host, dtype=np.float64)
    si, sc = (0, 0) if shard is None else (int(shard[0]), int(shard[1]))
    opts = _Opts(PREC[precision], DTYPE[io_dtype], int(max_batch), sc, si)
    out = _vp()
    _check(_lib.heff_plan_create(L, W1, W2, R, x, w1.ctypes.data_as(_P(C.c_double)),
                                 w2.ctypes.data_as(_P(C.c_double)), C.byref(opts), C.byref(out)),
           "heff_plan_create")
    return out


def heff_plan_shard_sectors(plan):
    n = C.c_int32()
    _check(_lib.heff_plan_shard_sectors(plan, None, C.byref(n)), "heff_plan_shard_sectors")
    out = np.zeros(n.value, dtype=np.int32)
    if n.value:
        _check(_lib.heff_plan_shard_sectors(plan, out.ctypes.data_as(_P(C.c_int32)), C.byref(n)),
               "heff_plan_shard_sectors")
    return out


def heff_plan_select_tiles(plan, tn1=0, tn2=0):
    _check(_lib.heff_plan_select_tiles(plan, int(tn1), int(tn2)), "heff_plan_select_tiles")


def heff_plan_workspace_size(plan):
    b = _sz()
    _check(_lib.heff_plan_workspace_size(plan, C.byref(b)), "heff_plan_workspace_size")
    return b.value


def heff_plan_flops(plan):
    c, e = C.c_double(), C.c_double()
    _check(_lib.heff_plan_flops(plan, C.byref(c), C.byref(e)), "heff_plan_flops")
    return c.value, e.value


def heff_plan_stats(plan):
    s = np.zeros(24, dtype=np.int64)
    _check(_lib.heff_plan_stats(plan, s.ctypes.data_as(_P(_i64))), "heff_plan_stats")
    return s


def heff_plan_destroy(plan):
    _lib.heff_plan_destroy(plan)


# record formats of the schedule tables (match csrc/internal.h)
TABLE_DTYPES = {
    0: np.dtype([("x_off", "<i8"), ("xt_row0", "<i8"), ("xt_col0", "<i4"), ("m_a", "<i4"),
                 ("m_b", "<i4"), ("a_pad", "<i4"), ("a0", "<i4"), ("b0", "<i4")]),
    1: np.dtype([("dst_row0", "<i8"), ("dst_col0", "<i4"), ("rows", "<i4"), ("cols", "<i4"),
                 ("cols_pad", "<i4"), ("r0", "<i4"), ("nrows", "<i4"), ("term_begin", "<i4"),
                 ("term_count", "<i4"), ("which", "<i4"), ("_pad", "<i4")]),
    2: np.dtype([("src_off", "<i8"), ("w_idx", "<i4"), ("_pad", "<i4")]),
    3: np.dtype([("a_row", "<i8"), ("b_row", "<i8"), ("c_off", "<i8"), ("m", "<i4"), ("n", "<i4"),
                 ("ldc", "<i4"), ("n_zero", "<i4"), ("seg_begin", "<i4"), ("seg_count", "<i4"),
                 ("ktotal", "<i4"), ("_pad", "<i4")]),
    4: np.dtype([("k0", "<i4"), ("klen", "<i4")]),
}
TABLE_DTYPES[5] = TABLE_DTYPES[3]
TABLE_DTYPES[6] = TABLE_DTYPES[4]


def heff_plan_export(plan, table):
    """The plan's schedule table as a numpy structured array."""
    n = _i64()
    _check(_lib.heff_plan_export(plan, int(table), None, C.byref(n)), "heff_plan_export")
    dt = TABLE_DTYPES[int(table)]
    if n.value % dt.itemsize:
        raise HeffError(-1, f"heff_plan_export: record size mismatch for table {table}")
    out = np.zeros(n.value // dt.itemsize, dtype=dt)
    if n.value:
        _check(_lib.heff_plan_export(plan, int(table), C.c_void_p(out.ctypes.data), C.byref(n)),
               "heff_plan_export")
    return out


def heff_prepare(plan, L, W1, W2, R, ws, stream=None):
    _check(_lib.heff_prepare(plan, _ptr(L), _ptr(W1), _ptr(W2), _ptr(R), _ptr(ws), _nbytes(ws),
                             _stream(stream)), "heff_prepare")


def heff_apply_prepared(plan, x, y, ws, stream=None):
    _check(_lib.heff_apply_prepared(plan, _ptr(x), _ptr(y), _ptr(ws), _nbytes(ws), _stream(stream)),
           "heff_apply_prepared")


def heff_apply(plan, L, W1, W2, R, x, y, ws, stream=None):
    _check(_lib.heff_apply(plan, _ptr(L), _ptr(W1), _ptr(W2), _ptr(R), _ptr(x), _ptr(y), _ptr(ws),
                           _nbytes(ws), _stream(stream)), "heff_apply")


def heff_apply_host_staging_size(plan):
    b = _sz()
    _check(_lib.heff_apply_host_staging_size(plan, C.byref(b)), "heff_apply_host_staging_size")
    return b.value


def heff_apply_host(plan, L, W1, W2, R, x, y, staging, ws, stream=None):
    """heff_apply on host (CPU, ideally pinned) tensors through a device staging buffer."""
    _check(_lib.heff_apply_host(plan, _ptr(L), _ptr(W1), _ptr(W2), _ptr(R), _ptr(x), _ptr(y), _ptr(staging),
                                _nbytes(staging), _ptr(ws), _nbytes(ws), _stream(stream)), "heff_apply_host")


def heff_apply_batched(plan, L, W1, W2, R, xs, ys, ws, stream=None):
    n = len(xs)
    xa = (_vp * n)(*[t.data_ptr() for t in xs])
    ya = (_vp * n)(*[t.data_ptr() for t in ys])
    _check(_lib.heff_apply_batched(plan, _ptr(L), _ptr(W1), _ptr(W2), _ptr(R), xa, ya, n, _ptr(ws),
                                   _nbytes(ws), _stream(stream)), "heff_apply_batched")


def heff_svd_create(x_layout):
    out = _vp()
    _check(_lib.heff_svd_create(x_layout, C.byref(out)), "heff_svd_create")
    return out


def heff_svd_workspace_size(s):
    b = _sz()
    _check(_lib.heff_svd_workspace_size(s, C.byref(b)), "heff_svd_workspace_size")
    return b.value


def heff_svd_compute(s, x, ws, stream=None):
    sw = _i32()
    _check(_lib.heff_svd_compute(s, _ptr(x), _ptr(ws), _nbytes(ws), _stream(stream), C.byref(sw)),
           "heff_svd_compute")
    return sw.value


def heff_svd_truncate(s, m_max, cutoff, nq, max_sectors):
    """Returns (charges [nsec, nq], dims [nsec], discarded weight, ||x||)."""
    ns = _i32()
    q = np.zeros(max_sectors * nq, dtype=np.int32)
    d = np.zeros(max_sectors, dtype=np.int32)
    disc, nrm = C.c_double(), C.c_double()
    _check(_lib.heff_svd_truncate(s, int(m_max), float(cutoff), C.byref(ns), q.ctypes.data_as(_P(_i32)),
                                  d.ctypes.data_as(_P(_i32)), C.byref(disc), C.byref(nrm)), "heff_svd_truncate")
    n = ns.value
    return q[:n * nq].reshape(n, nq), d[:n], disc.value, nrm.value


def heff_svd_info(s):
    """(FP32 preconditioning sweeps, FP64 sweeps) of the last heff_svd_compute."""
    a, b = C.c_int32(), C.c_int32()
    _check(_lib.heff_svd_info(s, C.byref(a), C.byref(b)), "heff_svd_info")
    return a.value, b.value


def heff_svd_singular_values(s, n):
    out = np.zeros(n, dtype=np.float64)
    _check(_lib.heff_svd_singular_values(s, out.ctypes.data_as(_P(C.c_double))), "heff_svd_singular_values")
    return out


def heff_svd_write(s, A_layout, B_layout, A, B, absorb_right, ws, stream=None):
    _check(_lib.heff_svd_write(s, A_layout, B_layout, _ptr(A), _ptr(B), 1 if absorb_right else 0, _ptr(ws),
                               _nbytes(ws), _stream(stream)), "heff_svd_write")


def heff_svd_destroy(s):
    _lib.heff_svd_destroy(s)


def heff_two_site_create(A, B, x):
    out = _vp()
    _check(_lib.heff_two_site_create(A, B, x, C.byref(out)), "heff_two_site_create")
    return out


def heff_two_site_apply(plan, A, B, x, stream=None):
    _check(_lib.heff_two_site_apply(plan, _ptr(A), _ptr(B), _ptr(x), _stream(stream)), "heff_two_site_apply")


def heff_two_site_destroy(plan):
    _lib.heff_two_site_destroy(plan)


def heff_grad_plan_create(L, W1, W2, R, x, W1_host, W2_host, ws_limit=0):
    """Gradient plan; ws_limit > 0 bounds the workspace by streaming left-sector chunks."""
    w1 = np.ascontiguousarray(W1_host, dtype=np.float64)
    w2 = np.ascontiguousarray(W2_host, dtype=np.float64)
    out = _vp()
    _check(_lib.heff_grad_plan_create(L, W1, W2, R, x, w1.ctypes.data_as(_P(C.c_double)),
                                      w2.ctypes.data_as(_P(C.c_double)), int(ws_limit), C.byref(out)),
           "heff_grad_plan_create")
    return out


def heff_grad_chunks(g):
    n = C.c_int32()
    _check(_lib.heff_grad_chunks(g, C.byref(n)), "heff_grad_chunks")
    return n.value


def heff_grad_workspace_size(g):
    b = _sz()
    _check(_lib.heff_grad_workspace_size(g, C.byref(b)), "heff_grad_workspace_size")
    return b.value


def heff_backward(g, plan, L, W1, W2, R, x, rho, dx, dL, dR, dW1, dW2, apply_ws, grad_ws, stream=None):
    """rho = <x|K|x>/<x|x> (device scalar) and its gradients (device float64 buffers)."""
    _check(_lib.heff_backward(g, plan, _ptr(L), _ptr(W1), _ptr(W2), _ptr(R), _ptr(x), _ptr(rho), _ptr(dx),
                              _ptr(dL), _ptr(dR), _ptr(dW1), _ptr(dW2), _ptr(apply_ws), _nbytes(apply_ws),
                              _ptr(grad_ws), _nbytes(grad_ws), _stream(stream)), "heff_backward")


def heff_grad_plan_destroy(g):
    _lib.heff_grad_plan_destroy(g)


def heff_grad_plan_set_precision(g, precision):
    """"fp64" (default) or "bf16x3" (tensor-core block products; FP64 buffers)."""
    _check(_lib.heff_grad_plan_set_precision(g, PREC[precision]), "heff_grad_plan_set_precision")


def heff_grad_status(g, grad_ws, stream=None):
    """Read and clear the gradient workspace's error flag; returns the status code (0 or -6)."""
    return int(_lib.heff_grad_status(g, _ptr(grad_ws), _nbytes(grad_ws), _stream(stream)))


def heff_env_plan_create(env_old, site, W, env_new, W_host, side):
    w = np.ascontiguousarray(W_host, dtype=np.float64)
    out = _vp()
    _check(_lib.heff_env_plan_create(env_old, site, W, env_new, w.ctypes.data_as(_P(C.c_double)),
                                     0 if side in (0, "left") else 1, C.byref(out)), "heff_env_plan_create")
    return out


def heff_env_workspace_size(plan):
    b = _sz()
    _check(_lib.heff_env_workspace_size(plan, C.byref(b)), "heff_env_workspace_size")
    return b.value


def heff_env_flops(plan):
    f = C.c_double()
    _check(_lib.heff_env_flops(plan, C.byref(f)), "heff_env_flops")
    return f.value


def heff_env_update(plan, env_old, site, W, env_new, ws, stream=None):
    _check(_lib.heff_env_update(plan, _ptr(env_old), _ptr(site), _ptr(W), _ptr(env_new), _ptr(ws),
                                _nbytes(ws), _stream(stream)), "heff_env_update")


def heff_env_plan_destroy(plan):
    _lib.heff_env_plan_destroy(plan)


def heff_env_plan_set_precision(plan, precision):
    """"fp64" (default) or "bf16x3" (tensor-core block products; FP64 buffers)."""
    _check(_lib.heff_env_plan_set_precision(plan, PREC[precision]), "heff_env_plan_set_precision")


def heff_env_status(plan, ws, stream=None):
    """Read and clear the env workspace's error flag; returns the status code (0 or -6)."""
    return int(_lib.heff_env_status(plan, _ptr(ws), _nbytes(ws), _stream(stream)))


def heff_davidson_workspace_size(plan, max_vecs):
    b = _sz()
    _check(_lib.heff_davidson_workspace_size(plan, int(max_vecs), C.byref(b)), "heff_davidson_workspace_size")
    return b.value


def heff_davidson(plan, L, W1, W2, R, x0, rnd, max_vecs, tol, x_out, result, apply_ws, dav_ws, stream=None):
    """Algorithm 1 (Davidson); result (device, 3 doubles): [lambda, ||q||, vectors used]."""
    _check(_lib.heff_davidson(plan, _ptr(L), _ptr(W1), _ptr(W2), _ptr(R), _ptr(x0), _ptr(rnd), int(max_vecs),
                              float(tol), _ptr(x_out), _ptr(result), _ptr(apply_ws), _nbytes(apply_ws),
                              _ptr(dav_ws), _nbytes(dav_ws), _stream(stream)), "heff_davidson")


def heff_lanczos_workspace_size(plan, n_iter):
    b = _sz()
    _check(_lib.heff_lanczos_workspace_size(plan, int(n_iter), C.byref(b)), "heff_lanczos_workspace_size")
    return b.value


def heff_lanczos(plan, L, W1, W2, R, x0, n_iter, x_out, result, apply_ws, lz_ws, stream=None):
    """Lowest Ritz pair after n_iter FP64 Lanczos steps; result (device, float64) receives
    [theta, residual estimate, Krylov dimension, alpha..., beta...]."""
    _check(_lib.heff_lanczos(plan, _ptr(L), _ptr(W1), _ptr(W2), _ptr(R), _ptr(x0), int(n_iter),
                             _ptr(x_out), _ptr(result), _ptr(apply_ws), _nbytes(apply_ws), _ptr(lz_ws),
                             _nbytes(lz_ws), _stream(stream)), "heff_lanczos")


def heff_ground_state_workspace_size(plan, n_iter):
    b = _sz()
    _check(_lib.heff_ground_state_workspace_size(plan, int(n_iter), C.byref(b)),
           "heff_ground_state_workspace_size")
    return b.value


def heff_ground_state(plan, plan64, L, W1, W2, R, x0, n_iter, max_cycles, tol, x_out, apply_ws, apply_ws64,
                      gs_ws, stream=None):
    """Restarted Lanczos to a residual tolerance, energy by an FP64 Rayleigh quotient
    (plan64, or None).  Returns dict(energy, ritz, residual_estimate, cycles, matvecs,
    residual_fp64)."""
    r = (C.c_double * 6)()
    _check(_lib.heff_ground_state(plan, plan64, _ptr(L), _ptr(W1), _ptr(W2), _ptr(R), _ptr(x0), int(n_iter),
                                  int(max_cycles), float(tol), _ptr(x_out), r, _ptr(apply_ws), _nbytes(apply_ws),
                                  _ptr(apply_ws64), 0 if apply_ws64 is None else _nbytes(apply_ws64), _ptr(gs_ws),
                                  _nbytes(gs_ws), _stream(stream)), "heff_ground_state")
    return {"energy": r[0], "ritz": r[1], "residual_estimate": r[2], "cycles": int(r[3]), "matvecs": int(r[4]),
            "residual_fp64": r[5]}


NOALLOC_WORKSPACE_BYTES = 128 << 20   # HEFF_NOALLOC_WORKSPACE_BYTES in include/heff.h


def heff_apply_noalloc(plan, L, W1, W2, R, x, y, stream=None):
    """heff_apply with the library's built-in workspace (no device allocation anywhere);
    calls that overlap on the GPU race on that shared workspace."""
    _check(_lib.heff_apply_noalloc(plan, _ptr(L), _ptr(W1), _ptr(W2), _ptr(R), _ptr(x), _ptr(y),
                                   _stream(stream)), "heff_apply_noalloc")


def heff_apply_noalloc_status(plan, stream=None):
    """Read and clear the built-in workspace's error flag; returns the status (0 or -6)."""
    return int(_lib.heff_apply_noalloc_status(plan, _stream(stream)))


TILE_256, TILE_128, TILE_PAIR_256, TILE_VARIANTS = 256, 128, 512, 3


def heff_plan_autotune(plan, L, W1, W2, R, x, y, ws, stream=None, times=None):
    """Pick the fastest tile variant (TILE_256, TILE_128, TILE_PAIR_256) per GEMM on these
    inputs; returns (variant of GEMM 1, variant of GEMM 2).  If `times` is a list, the
    median times {GEMM 1: 256, 128, pairs; GEMM 2: 256, 128, pairs} (ms) are appended."""
    tn = (_i32 * 2)()
    ms = (C.c_float * (2 * TILE_VARIANTS))()
    _check(_lib.heff_plan_autotune(plan, _ptr(L), _ptr(W1), _ptr(W2), _ptr(R), _ptr(x), _ptr(y), _ptr(ws),
                                   _nbytes(ws), _stream(stream), tn, ms), "heff_plan_autotune")
    if times is not None:
        times.extend(float(v) for v in ms)
    return int(tn[0]), int(tn[1])


def heff_plan_set_timing(plan, enable=True):
    _check(_lib.heff_plan_set_timing(plan, 1 if enable else 0), "heff_plan_set_timing")


def heff_plan_check_mpo(plan, W1, W2, stream=None):
    """Entries of the device MPO tensors that are nonzero where the plan's host copies were
    zero (0: the tensors fit the plan)."""
    v = _i64()
    _check(_lib.heff_plan_check_mpo(plan, _ptr(W1), _ptr(W2), _stream(stream), C.byref(v)), "heff_plan_check_mpo")
    return int(v.value)


def heff_plan_timings(plan):
    """Milliseconds of (prepare, pack, GEMM 1, GEMM 2) of the last call."""
    ms = (C.c_float * 4)()
    _check(_lib.heff_plan_timings(plan, ms), "heff_plan_timings")
    return [float(v) for v in ms]


def heff_workspace_status(plan, ws, stream=None):
    """Read and clear the workspace's sticky device error flag; returns the status code
    (0, or -6 when a bounded device-side wait expired) without raising."""
    return int(_lib.heff_workspace_status(plan, _ptr(ws), _nbytes(ws), _stream(stream)))


def heff_wait_selftest(plan, ws, kind, stream=None):
    """Run one device-side bounded wait that nothing completes (kind 0: the GEMM kernels'
    mbarrier wait, kind 1: the SVD sweeps' grid barrier); returns its duration in ms.  The
    expired wait leaves the workspace's error flag set."""
    ms = C.c_float(0.0)
    _check(_lib.heff_wait_selftest(plan, _ptr(ws), _nbytes(ws), int(kind), _stream(stream), C.byref(ms)),
           "heff_wait_selftest")
    return float(ms.value)


def heff_last_error():
    return _lib.heff_last_error().decode()


def heff_launch_count():
    return int(_lib.heff_launch_count())


def heff_version():
    return _lib.heff_version().decode()


# ------------------------------------------------------------------ owners
class Layout:
    """Owner of a heff_layout with the block list as numpy arrays."""

    def __init__(self, indices, target=None):
        self.indices = [(np.asarray(q, dtype=np.int32).reshape(len(d), -1),
                         np.asarray(d, dtype=np.int32), int(f)) for q, d, f in indices]
        self.handle = heff_qn_block_layout(self.indices, target)
        self.nblocks, self.nelem, self.nidx = heff_layout_info(self.handle)
        self.keys, self.offsets = heff_layout_blocks(self.handle)
        dims = [d for _, d, _ in self.indices]
        self.sizes = np.ones(self.nblocks, dtype=np.int64)
        for k in range(self.nidx):
            self.sizes *= dims[k][self.keys[:, k]]

    def blocks(self):
        """Iterate (key tuple, offset, size)."""
        for b in range(self.nblocks):
            yield tuple(int(v) for v in self.keys[b]), int(self.offsets[b]), int(self.sizes[b])

    def assemble(self, fill, dtype=np.float64):
        """Flat buffer with fill(key) (an array of the block's size) at each block."""
        out = np.zeros(self.nelem, dtype=dtype)
        for key, off, size in self.blocks():
            v = np.asarray(fill(key), dtype=np.float64).reshape(-1)
            if v.size != size:
                raise ValueError(f"block {key}: got {v.size} values, layout wants {size}")
            out[off:off + size] = v
        return out

    def split(self, flat):
        """Dict key -> block view (1-D) of a flat buffer."""
        return {key: flat[off:off + size] for key, off, size in self.blocks()}

    def __del__(self):
        if getattr(self, "handle", None):
            heff_layout_destroy(self.handle)
            self.handle = None


def heff_layouts(alpha, beta, phys, ql, qm, qr, target=None):
    """Layouts of (L, W1, W2, R, x) for a two-site problem in the library's conventions.

    alpha/beta: (charges, dims) of the left/right bond; phys: site charges [d, nq];
    ql/qm/qr: MPO channel charges of the three MPO bonds.
    """
    aq, ad = alpha
    bq, bd = beta
    ph = np.asarray(phys, dtype=np.int32)
    ones = lambda n: np.ones(n, dtype=np.int32)
    A = lambda f: (aq, ad, f)
    B = lambda f: (bq, bd, f)
    S = lambda f: (ph, ones(len(ph)), f)
    ch = lambda q, f: (np.asarray(q, dtype=np.int32), ones(len(q)), f)
    Ll = Layout([A(-1), ch(ql, 1), A(1)])
    W1l = Layout([ch(ql, 1), S(1), S(-1), ch(qm, -1)])
    W2l = Layout([ch(qm, 1), S(1), S(-1), ch(qr, -1)])
    Rl = Layout([B(-1), ch(qr, 1), B(1)])
    xl = Layout([A(1), S(1), S(1), B(-1)], target)
    return Ll, W1l, W2l, Rl, xl


class Plan:
    """Owner of a heff_plan built from the five layouts and host MPO values."""

    def __init__(self, L, W1, W2, R, x, W1_host, W2_host, precision="bf16x3", io_dtype="f32",
                 max_batch=1, shard=None):
        self.layouts = (L, W1, W2, R, x)
        self.precision, self.io_dtype, self.max_batch = precision, io_dtype, max_batch
        self.handle = heff_plan_create(L.handle, W1.handle, W2.handle, R.handle, x.handle,
                                       W1_host, W2_host, precision, io_dtype, max_batch, shard)
        self.workspace_bytes = heff_plan_workspace_size(self.handle)
        self.flops_canonical, self.flops_executed = heff_plan_flops(self.handle)
        self.stats = heff_plan_stats(self.handle)

    def workspace(self, device="cuda"):
        import torch
        return torch.empty(max(self.workspace_bytes, 256), dtype=torch.uint8, device=device)

    def __del__(self):
        if getattr(self, "handle", None):
            heff_plan_destroy(self.handle)
            self.handle = None


class RayleighQuotient:
    """torch.autograd.Function for rho(x, L, W1, W2, R) = <x|K|x> / <x|x>.

    ``RayleighQuotient.apply(ctx_obj, x, L, W1, W2, R)`` returns rho as a 0-d tensor; the
    forward pass runs heff_backward (one apply plus the closed-form gradients, all on the
    GPU) and the backward pass scales the stored gradients by the incoming gradient.
    ``ctx_obj`` holds the plans and workspaces: ``(grad_plan, apply_plan, apply_ws, grad_ws)``.
    """

    _fn = None

    @classmethod
    def apply(cls, ctx_obj, x, L, W1, W2, R):
        if cls._fn is None:
            import torch

            class _F(torch.autograd.Function):
                @staticmethod
                def forward(ctx, x, L, W1, W2, R, holder):
                    g, plan, aws, gws = holder
                    rho = torch.empty((), dtype=torch.float64, device=x.device)
                    grads = [torch.empty_like(t) for t in (x, L, R, W1, W2)]
                    heff_backward(g, plan, L, W1, W2, R, x, rho, grads[0], grads[1], grads[2], grads[3],
                                  grads[4], aws, gws)
                    ctx.save_for_backward(*grads)
                    return rho

                @staticmethod
                def backward(ctx, go):
                    dx, dL, dR, dW1, dW2 = ctx.saved_tensors
                    return go * dx, go * dL, go * dW1, go * dW2, go * dR, None

            cls._fn = _F
        return cls._fn.apply(x, L, W1, W2, R, ctx_obj)
