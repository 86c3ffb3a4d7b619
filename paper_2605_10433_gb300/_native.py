"""ctypes binding of libsagms.so (include/sagms.h): argument marshalling only.

Every function named ``sagms_*`` here is the C entry point of the same name; the helpers
below them take PyTorch tensors for device memory and streams and pass raw pointers.
If the library has not been built, importing the binding raises instead of falling
back to anything else.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsagms.so")

SAGMS_MS, SAGMS_SMS, SAGMS_SAGMS, SAGMS_BP = 0, 1, 2, 3
SAGMS_FLAG_L0_PER_QUBIT = 1
SAGMS_FLAG_NO_EARLY_STOP = 2
SAGMS_FLAG_GENERIC_KERNEL = 4
SAGMS_OK = 0
ERRORS = {-1: "ERR_ARG", -2: "ERR_CSR", -3: "ERR_DEGREE", -4: "ERR_PARAM", -5: "ERR_OOM", -6: "ERR_CUDA",
          -7: "ERR_TIMEOUT", -8: "ERR_BUSY", -9: "ERR_SIZE", -10: "ERR_CANCELLED"}
SAGMS_SERVE_CONTINUOUS, SAGMS_SERVE_PLAIN = 0, 1
MODES = {"ms": SAGMS_MS, "sms": SAGMS_SMS, "sagms": SAGMS_SAGMS, "bp": SAGMS_BP}


class SagmsError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class sagms_params(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("alpha", ctypes.c_float), ("alpha_min", ctypes.c_float),
                ("alpha_max", ctypes.c_float), ("eta_unsat", ctypes.c_float), ("max_iter", ctypes.c_int32),
                ("flags", ctypes.c_uint32)]


class sagms_job(ctypes.Structure):
    _fields_ = [("code", ctypes.c_void_p), ("params", sagms_params), ("shots", ctypes.c_int64),
                ("d_syn", ctypes.c_void_p), ("d_L0", ctypes.c_void_p), ("d_err", ctypes.c_void_p),
                ("d_conv", ctypes.c_void_p), ("d_iters", ctypes.c_void_p)]


class sagms_mc_counts(ctypes.Structure):
    _fields_ = [("shots", ctypes.c_int64), ("failures", ctypes.c_int64), ("not_converged", ctypes.c_int64),
                ("logical", ctypes.c_int64), ("iters_sum", ctypes.c_int64)]

    def as_dict(self):
        return {f: int(getattr(self, f)) for f, _ in self._fields_}


def _load_library():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libsagms.so is not built ({LIB_PATH}); run __graft_entry__.build() "
                          "or python -m paper_2605_10433_gb300.build")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    P = ctypes.POINTER
    sig = {
        "sagms_load_code": (ctypes.c_int, [i32, i32, i64, P(i32), P(i32), P(vp)]),
        "sagms_free_code": (None, [vp]),
        "sagms_code_info": (ctypes.c_int, [vp, P(i32), P(i32), P(i32), P(i32)]),
        "sagms_code_kernels": (ctypes.c_int, [vp, P(ctypes.c_uint32)]),
        "sagms_phi": (ctypes.c_int, [vp, vp, i64, i32, vp]),
        "sagms_check_layers": (ctypes.c_int, [i32, i32, i64, P(i32), P(i32), P(i32), P(i32)]),
        "sagms_column_slots": (ctypes.c_int, [i32, i32, i64, P(i32), P(i32), i32, P(i32)]),
        "sagms_check_params": (ctypes.c_int, [P(sagms_params)]),
        "sagms_decode": (ctypes.c_int, [vp, P(sagms_params), i64, vp, vp, vp, vp, vp, vp]),
        "sagms_decode_trace": (ctypes.c_int, [vp, P(sagms_params), i64, vp, vp, vp, vp, vp, vp, vp]),
        "sagms_decode_host": (ctypes.c_int, [vp, P(sagms_params), i64, vp, vp, vp, vp, vp]),
        "sagms_decode_noalloc": (ctypes.c_int, [vp, P(sagms_params), i64, vp, vp, vp, vp, vp, vp]),
        "sagms_decode_multi": (ctypes.c_int, [P(sagms_job), i32, vp]),
        "sagms_graph_create": (ctypes.c_int, [P(sagms_job), i32, P(vp)]),
        "sagms_graph_launch": (ctypes.c_int, [vp, vp]),
        "sagms_graph_destroy": (None, [vp]),
        "sagms_autotune": (ctypes.c_int, [vp, P(sagms_params), i64, vp, vp, vp, vp, vp, P(i32),
                                          P(ctypes.c_float), vp]),
        "sagms_set_plan": (ctypes.c_int, [vp, i32]),
        "sagms_set_launch_limit": (ctypes.c_int, [vp, i64]),
        "sagms_gf4_load_code": (ctypes.c_int, [i32, i32, i64, P(i32), P(i32), P(ctypes.c_uint8), P(vp)]),
        "sagms_gf4_free_code": (None, [vp]),
        "sagms_gf4_layout": (ctypes.c_int, [vp]),
        "sagms_gf4_decode": (ctypes.c_int, [vp, P(sagms_params), i64, vp, vp, vp, vp, vp, vp]),
        "sagms_gf4_decode_trace": (ctypes.c_int, [vp, P(sagms_params), i64, vp, vp, vp, vp, vp, vp, vp]),
        "sagms_server_create": (ctypes.c_int, [ctypes.c_size_t, i32, i32, i32, P(vp)]),
        "sagms_server_add_code": (ctypes.c_int, [vp, vp, P(sagms_params), P(i32)]),
        "sagms_server_submit": (ctypes.c_int, [vp, i32, i64, vp, vp, vp, vp, vp, P(ctypes.c_uint64)]),
        "sagms_server_poll": (ctypes.c_int, [vp, ctypes.c_uint64, i64]),
        "sagms_server_cancel": (ctypes.c_int, [vp, ctypes.c_uint64]),
        "sagms_server_times": (ctypes.c_int, [vp, ctypes.c_uint64, P(i64), P(i64)]),
        "sagms_server_release": (ctypes.c_int, [vp, ctypes.c_uint64]),
        "sagms_server_destroy": (ctypes.c_int, [vp]),
        "sagms_server_replay": (ctypes.c_int, [vp, i32, P(i32), P(i64), P(i64), P(vp), P(vp), P(vp), P(vp),
                                               P(vp), P(ctypes.c_uint64)]),
        "sagms_alpha_star": (ctypes.c_double, [ctypes.c_double, i32]),
        "sagms_last_error_string": (ctypes.c_char_p, []),
        "sagms_version": (ctypes.c_char_p, []),
        "sagms_x_logicals": (ctypes.c_int, [i32, i32, P(i32), P(i32), i32, P(i32), P(i32), i32, vp, P(i32)]),
        "sagms_mc_set_logicals": (ctypes.c_int, [vp, i32, vp]),
        "sagms_mc_sample": (ctypes.c_int, [vp, ctypes.c_uint64, ctypes.c_double, ctypes.c_float, i64, i64,
                                           vp, vp, vp, vp]),
        "sagms_mc_check": (ctypes.c_int, [vp, i64, vp, vp, vp, vp, vp, vp, vp]),
        "sagms_mc_run": (ctypes.c_int, [vp, P(sagms_params), ctypes.c_uint64, ctypes.c_double, ctypes.c_float,
                                        i64, i64, i64, P(sagms_mc_counts)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


_lib = _load_library()


def lib():
    return _lib


def _check(rc: int):
    if rc != SAGMS_OK:
        raise SagmsError(rc, _lib.sagms_last_error_string().decode())


# ----------------------------------------------------------------------- C entry points
def sagms_load_code(m, n, row_ptr, col_idx):
    """Returns an opaque handle (int).  row_ptr / col_idx: int32 numpy arrays (host)."""
    import numpy as np
    rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
    ci = np.ascontiguousarray(col_idx, dtype=np.int32)
    h = ctypes.c_void_p()
    _check(_lib.sagms_load_code(int(m), int(n), int(rp[-1]) if len(rp) else 0,
                                rp.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                ci.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), ctypes.byref(h)))
    return h.value


def sagms_free_code(handle):
    _lib.sagms_free_code(handle)


def sagms_code_info(handle):
    v = [ctypes.c_int32() for _ in range(4)]
    _check(_lib.sagms_code_info(handle, *[ctypes.byref(x) for x in v]))
    return tuple(x.value for x in v)


def sagms_code_kernels(handle):
    """Bit mask of the plan kernels (1-4) that have a layout for the code."""
    v = ctypes.c_uint32()
    _check(_lib.sagms_code_kernels(handle, ctypes.byref(v)))
    return v.value


def sagms_phi(x, form=0, stream=None):
    """phi(x) = -ln tanh(x/2) on the GPU for a float32 CUDA tensor x (form 0: the decoder's
    evaluation, form 1: log1pf(2 / expm1f(x)))."""
    import torch
    y = torch.empty_like(x)
    _check(_lib.sagms_phi(x.data_ptr(), y.data_ptr(), int(x.numel()), int(form),
                          stream.cuda_stream if stream is not None else None))
    return y


def sagms_check_layers(m, n, row_ptr, col_idx):
    """First-fit layer of every check (int32 numpy array) and the layer count."""
    import numpy as np
    rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
    ci = np.ascontiguousarray(col_idx, dtype=np.int32)
    out = np.zeros(int(m), dtype=np.int32)
    L = ctypes.c_int32()
    _check(_lib.sagms_check_layers(int(m), int(n), int(rp[-1]) if len(rp) else 0,
                                   rp.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                   ci.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                   out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), ctypes.byref(L)))
    return out, L.value


def sagms_column_slots(m, n, row_ptr, col_idx, D):
    """Column-indexed slot of every edge (int32 numpy array, CSR order) for D message rows."""
    import numpy as np
    rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
    ci = np.ascontiguousarray(col_idx, dtype=np.int32)
    out = np.zeros(len(ci), dtype=np.int32)
    _check(_lib.sagms_column_slots(int(m), int(n), int(rp[-1]) if len(rp) else 0,
                                   rp.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                   ci.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), int(D),
                                   out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))))
    return out


def sagms_check_params(params: sagms_params) -> int:
    return _lib.sagms_check_params(ctypes.byref(params))


def sagms_decode(handle, params, shots, syn_ptr, L0_ptr, err_ptr, conv_ptr, iters_ptr, stream_ptr):
    _check(_lib.sagms_decode(handle, ctypes.byref(params), int(shots), syn_ptr, L0_ptr, err_ptr, conv_ptr,
                             iters_ptr, stream_ptr))


def sagms_decode_trace(handle, params, shots, syn_ptr, L0_ptr, err_ptr, conv_ptr, iters_ptr, trace_ptr, stream_ptr):
    _check(_lib.sagms_decode_trace(handle, ctypes.byref(params), int(shots), syn_ptr, L0_ptr, err_ptr, conv_ptr,
                                   iters_ptr, trace_ptr, stream_ptr))


def sagms_decode_host(handle, params, shots, syn_ptr, L0_ptr, err_ptr, conv_ptr, iters_ptr):
    _check(_lib.sagms_decode_host(handle, ctypes.byref(params), int(shots), syn_ptr, L0_ptr, err_ptr, conv_ptr,
                                  iters_ptr))


def sagms_decode_noalloc(handle, params, shots, syn_ptr, L0_ptr, err_ptr, conv_ptr, iters_ptr, stream_ptr):
    """sagms_decode for callers that cannot allocate device memory (fixed library scratch)."""
    _check(_lib.sagms_decode_noalloc(handle, ctypes.byref(params), int(shots), syn_ptr, L0_ptr, err_ptr, conv_ptr,
                                     iters_ptr, stream_ptr))


def sagms_decode_multi(jobs, stream_ptr):
    arr = (sagms_job * len(jobs))(*jobs)
    _check(_lib.sagms_decode_multi(arr, len(jobs), stream_ptr))


def sagms_graph_create(jobs):
    arr = (sagms_job * len(jobs))(*jobs)
    g = ctypes.c_void_p()
    _check(_lib.sagms_graph_create(arr, len(jobs), ctypes.byref(g)))
    return g.value


def sagms_graph_launch(graph, stream_ptr):
    _check(_lib.sagms_graph_launch(graph, stream_ptr))


def sagms_graph_destroy(graph):
    _lib.sagms_graph_destroy(graph)


def sagms_autotune(handle, params, shots, syn_ptr, L0_ptr, err_ptr, conv_ptr, iters_ptr, stream_ptr):
    plan = ctypes.c_int32()
    rate = ctypes.c_float()
    _check(_lib.sagms_autotune(handle, ctypes.byref(params), int(shots), syn_ptr, L0_ptr, err_ptr, conv_ptr,
                               iters_ptr, ctypes.byref(plan), ctypes.byref(rate), stream_ptr))
    return plan.value, rate.value


def sagms_set_plan(handle, plan):
    _check(_lib.sagms_set_plan(handle, int(plan)))


def sagms_set_launch_limit(handle, shots):
    _check(_lib.sagms_set_launch_limit(handle, int(shots)))


def sagms_gf4_load_code(m, n, row_ptr, col_idx, pauli):
    """Returns an opaque handle (int).  Host arrays: row_ptr int32, col_idx int32, pauli uint8."""
    import numpy as np
    rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
    ci = np.ascontiguousarray(col_idx, dtype=np.int32)
    pa = np.ascontiguousarray(pauli, dtype=np.uint8)
    if rp.shape != (int(m) + 1,) or ci.shape != pa.shape or ci.shape[0] != int(rp[-1]):
        raise ValueError("sagms_gf4_load_code: row_ptr must have m + 1 entries and col_idx / pauli nnz each")
    out = ctypes.c_void_p()
    _check(_lib.sagms_gf4_load_code(int(m), int(n), int(rp[-1]), rp.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                    ci.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                    pa.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), ctypes.byref(out)))
    return out.value


def sagms_gf4_layout(handle):
    """1 when the loaded GF(4) code takes the column-indexed CSS kernel, 0 for the generic one."""
    rc = _lib.sagms_gf4_layout(handle)
    _check(min(rc, 0))
    return rc


def sagms_gf4_free_code(handle):
    _lib.sagms_gf4_free_code(handle)


def sagms_gf4_decode(handle, params, shots, syn_ptr, L0_ptr, err_ptr, conv_ptr, iters_ptr, stream_ptr, trace_ptr=None):
    if trace_ptr is None:
        _check(_lib.sagms_gf4_decode(handle, ctypes.byref(params), shots, syn_ptr, L0_ptr, err_ptr, conv_ptr, iters_ptr,
                                     stream_ptr))
    else:
        _check(_lib.sagms_gf4_decode_trace(handle, ctypes.byref(params), shots, syn_ptr, L0_ptr, err_ptr, conv_ptr,
                                           iters_ptr, trace_ptr, stream_ptr))


def sagms_alpha_star(L0: float, dc: int) -> float:
    return _lib.sagms_alpha_star(float(L0), int(dc))


def sagms_version() -> str:
    return _lib.sagms_version().decode()


def sagms_last_error_string() -> str:
    return _lib.sagms_last_error_string().decode()


def _i32(a):
    import numpy as np
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def sagms_x_logicals(n, hx_row_ptr, hx_col_idx, hz_row_ptr, hz_col_idx):
    """Basis of X-logical operators (ker H_Z modulo rowspace H_X) as uint32 [k][ceil(n/32)]."""
    import numpy as np
    keep = [_i32(a) for a in (hx_row_ptr, hx_col_idx, hz_row_ptr, hz_col_idx)]
    (hxr, hxr_p), (hxc, hxc_p), (hzr, hzr_p), (hzc, hzc_p) = keep
    k = ctypes.c_int32(0)
    _check(_lib.sagms_x_logicals(int(n), len(hxr) - 1, hxr_p, hxc_p, len(hzr) - 1, hzr_p, hzc_p, 0, None,
                                 ctypes.byref(k)))
    out = np.zeros((k.value, (int(n) + 31) // 32), dtype=np.uint32)
    _check(_lib.sagms_x_logicals(int(n), len(hxr) - 1, hxr_p, hxc_p, len(hzr) - 1, hzr_p, hzc_p, k.value,
                                 out.ctypes.data_as(ctypes.c_void_p), ctypes.byref(k)))
    return out


def sagms_mc_set_logicals(handle, logicals):
    import numpy as np
    L = np.ascontiguousarray(logicals, dtype=np.uint32)
    _check(_lib.sagms_mc_set_logicals(handle, L.shape[0], L.ctypes.data_as(ctypes.c_void_p) if L.size else None))


def sagms_mc_sample(handle, seed, q, L0, shot0, shots, err_ptr, syn_ptr, L0_ptr, stream_ptr):
    _check(_lib.sagms_mc_sample(handle, int(seed) & 0xFFFFFFFFFFFFFFFF, float(q), float(L0), int(shot0), int(shots),
                                err_ptr, syn_ptr, L0_ptr, stream_ptr))


def sagms_mc_check(handle, shots, err_ptr, ehat_ptr, conv_ptr, iters_ptr, fail_ptr, counts_ptr, stream_ptr):
    _check(_lib.sagms_mc_check(handle, int(shots), err_ptr, ehat_ptr, conv_ptr, iters_ptr, fail_ptr, counts_ptr,
                               stream_ptr))


def sagms_mc_run(handle, params, seed, q, L0, target_failures, max_shots, batch, counts):
    _check(_lib.sagms_mc_run(handle, ctypes.byref(params), int(seed) & 0xFFFFFFFFFFFFFFFF, float(q), float(L0),
                             int(target_failures), int(max_shots), int(batch), ctypes.byref(counts)))
