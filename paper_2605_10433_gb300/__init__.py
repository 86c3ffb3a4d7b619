"""GB300-native batched SAGMS / SMS / MS / BP syndrome decoding of quantum LDPC codes.

The decoder runs in ``libsagms.so`` (hand-written CUDA for sm_103a, C ABI in
``include/sagms.h``).  This package adds the thin Python layer: ``_native`` binds the C
entry points by name, and :class:`DeviceCode` / :func:`decode` pass PyTorch tensors (device
memory and streams only) to them.  ``inputs`` builds seeded codes and syndromes.
"""
from __future__ import annotations

from dataclasses import dataclass

MODES = {"ms": 0, "sms": 1, "sagms": 2, "bp": 3}
FLAG_L0_PER_QUBIT = 1
FLAG_NO_EARLY_STOP = 2
FLAG_GENERIC_KERNEL = 4
FLAG_AUTO_CEILING = 16
FLAG_LAYERED = 32


@dataclass
class Params:
    """Decoder parameters (defaults: the SAGMS values of the paper's experiments, Sec. V-B)."""
    mode: str = "sagms"
    alpha: float = 0.75
    alpha_min: float = 0.30
    alpha_max: float = 0.50
    eta_unsat: float = 1.10
    max_iter: int = 100
    flags: int = 0

    def to_c(self):
        from . import _native
        return _native.sagms_params(MODES[self.mode] if isinstance(self.mode, str) else int(self.mode),
                                    self.alpha, self.alpha_min, self.alpha_max, self.eta_unsat,
                                    self.max_iter, self.flags)


class DeviceCode:
    """A parity-check matrix loaded on the current CUDA device (owns the C handle)."""

    def __init__(self, m, n, row_ptr, col_idx):
        from . import _native
        self._native = _native
        self.m, self.n = int(m), int(n)
        import torch
        self.device = torch.cuda.current_device()   # sagms_load_code uploads to the current device
        self.handle = _native.sagms_load_code(m, n, row_ptr, col_idx)
        _, _, self.dc_max, self.dv_max = _native.sagms_code_info(self.handle)

    @classmethod
    def from_code(cls, code):
        return cls(code.m, code.n, code.row_ptr, code.col_idx)

    @property
    def mw(self):
        return (self.m + 31) // 32

    @property
    def nw(self):
        return (self.n + 31) // 32

    @property
    def kernels(self):
        """Names of the kernels with a layout for this code (decode_plan's names)."""
        mask = self._native.sagms_code_kernels(self.handle)
        return [KERNEL_NAMES[k] for k in range(1, 6) if mask >> k & 1]

    def set_logicals(self, logicals):
        """Attach logical operators (uint32 [k][ceil(n/32)]) for the Monte Carlo check."""
        self._native.sagms_mc_set_logicals(self.handle, logicals)

    def close(self):
        if getattr(self, "handle", None):
            self._native.sagms_free_code(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Gf4DeviceCode:
    """A stabilizer matrix with Pauli entries (GF(4), Sec. II) loaded on the current CUDA device
    for the quaternary decoder (owns the C handle).  ``gcode``: inputs.gf4.Gf4Code or any
    object with m, n, row_ptr, col_idx and pauli (1 X, 2 Z, 3 Y)."""

    def __init__(self, gcode):
        from . import _native
        import torch
        self._native = _native
        self.m, self.n = int(gcode.m), int(gcode.n)
        self.device = torch.cuda.current_device()
        self.handle = _native.sagms_gf4_load_code(self.m, self.n, gcode.row_ptr, gcode.col_idx, gcode.pauli)

    @property
    def mw(self):
        return (self.m + 31) // 32

    @property
    def nw(self):
        return (self.n + 31) // 32

    @property
    def css_layout(self) -> bool:
        """True when the code takes the column-indexed CSS kernel (a CSS matrix with a slot
        assignment per row type), False for the generic kernel."""
        return self._native.sagms_gf4_layout(self.handle) == 1

    def close(self):
        if getattr(self, "handle", None):
            self._native.sagms_gf4_free_code(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def gf4_decode(code: Gf4DeviceCode, syn, L0, params: Params | None = None, stream=None, trace=False):
    """Decode on the GPU with the quaternary decoder.  ``syn``: int32 CUDA tensor [shots, mw];
    ``L0``: float32 CUDA tensor [shots] (one prior LLR per shot, ln((1 - eps0)/(eps0/3))).
    Returns (err [shots, 2, nw] int32: x bits then z bits of e_hat, conv [shots] uint8,
    iters [shots] int32[, trace [shots, max_iter+1, n, 3] float32: Lambda(X, Z, Y)])."""
    import torch
    from . import _native
    p = params or Params()
    if p.flags & ~(FLAG_NO_EARLY_STOP | FLAG_GENERIC_KERNEL):
        raise ValueError("the GF(4) decoder takes one prior per shot and no flag but FLAG_NO_EARLY_STOP "
                         "and FLAG_GENERIC_KERNEL")
    dev = f"cuda:{code.device}"
    for name, a, dt in (("syn", syn, (torch.int32, torch.uint32) if hasattr(torch, "uint32") else (torch.int32,)),
                        ("L0", L0, (torch.float32,))):
        if not hasattr(a, "data_ptr") or str(a.device) != dev or a.dtype not in dt or not a.is_contiguous():
            raise ValueError(f"{name}: need a contiguous {dt[0]} tensor on {dev}")
    if syn.dim() != 2 or syn.shape[1] != code.mw:
        raise ValueError(f"syn: shape {list(syn.shape)}, need [shots, {code.mw}]")
    shots = int(syn.shape[0])
    if tuple(L0.shape) != (shots,):
        raise ValueError(f"L0: shape {list(L0.shape)}, need [{shots}]")
    err = torch.empty((shots, 2, code.nw), dtype=torch.int32, device=dev)
    conv = torch.empty((shots,), dtype=torch.uint8, device=dev)
    iters = torch.empty((shots,), dtype=torch.int32, device=dev)
    tr = torch.empty((shots, p.max_iter + 1, code.n, 3), dtype=torch.float32, device=dev) if trace else None
    _native.sagms_gf4_decode(code.handle, p.to_c(), shots, syn.data_ptr(), L0.data_ptr(), err.data_ptr(),
                             conv.data_ptr(), iters.data_ptr(), _stream_ptr(stream),
                             tr.data_ptr() if tr is not None else None)
    return (err, conv, iters, tr) if trace else (err, conv, iters)


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes_void(stream.cuda_stream)


def ctypes_void(x):
    import ctypes
    return ctypes.c_void_p(int(x))


# Element kinds and sizes of the decode buffers: (name, numpy kinds, itemsize).
_BUFFERS = (("syn", "iu", 4), ("L0", "f", 4), ("err", "iu", 4), ("conv", "u", 1), ("iters", "i", 4))


def _buffer_facts(a):
    """(numpy dtype, shape, C-contiguous, device) of a torch tensor or numpy array; device is
    'cpu' or 'cuda:<index>'."""
    import numpy as np
    if hasattr(a, "data_ptr"):
        try:
            dt = np.dtype(str(a.dtype).replace("torch.", ""))
        except TypeError:   # a torch type numpy does not have (bfloat16, ...)
            raise TypeError(f"unsupported buffer dtype {a.dtype}") from None
        dev = f"cuda:{a.device.index}" if a.is_cuda else "cpu"
        return dt, tuple(a.shape), a.is_contiguous(), dev
    a = np.asarray(a)
    return a.dtype, a.shape, a.flags.c_contiguous, "cpu"


def _check_buffers(code: "DeviceCode", params: "Params", bufs, host: bool):
    """Check the caller's buffers against the code before their pointers reach the library:
    a wrong dtype or shape would let a kernel or a copy run past a buffer's end.  ``bufs`` are
    (syn, L0, err, conv, iters); syn's rows give the shot count.  Output buffers may hold more
    rows than shots (only the first rows are written); row widths and L0's length must match.
    Raises TypeError or ValueError; returns the shot count."""
    facts = [_buffer_facts(a) for a in bufs]
    shots = facts[0][1][0] if len(facts[0][1]) == 2 else -1
    per_qubit = bool(params.flags & FLAG_L0_PER_QUBIT)
    for (name, kinds, size), (dt, shape, contig, dev) in zip(_BUFFERS, facts):
        if dt.kind not in kinds or dt.itemsize != size:
            raise TypeError(f"{name}: dtype {dt} (need a {size}-byte {'/'.join(kinds)} type)")
        if not contig:
            raise ValueError(f"{name}: not contiguous")
        if host and dev != "cpu":
            raise ValueError(f"{name}: must be in host memory (numpy or a CPU tensor), got {dev}")
        if not host and dev != f"cuda:{code.device}":
            raise ValueError(f"{name}: must be a CUDA tensor on cuda:{code.device} (the code's device), got {dev}")
        if name == "syn":
            ok = len(shape) == 2 and shape[1] == code.mw
            want = f"[shots, {code.mw}]"
        elif name == "L0":
            want_len = code.n if per_qubit else shots
            ok = shape == (want_len,)
            want = f"[{want_len}]" + (" (one prior per qubit)" if per_qubit else " (one prior per shot)")
        elif name == "err":
            ok = len(shape) == 2 and shape[1] == code.nw and shape[0] >= shots
            want = f"[>= {shots}, {code.nw}]"
        else:
            ok = len(shape) == 1 and shape[0] >= shots
            want = f"[>= {shots}]"
        if not ok:
            raise ValueError(f"{name}: shape {list(shape)}, need {want}")
    return shots


def decode(code: DeviceCode, syn, L0, params: Params | None = None, out=None, stream=None, trace=False):
    """Decode packed syndromes on the GPU.

    syn: int32 CUDA tensor [shots, ceil(m/32)] (uint32 bit patterns); L0: float32 CUDA tensor
    [shots] (or [n] with FLAG_L0_PER_QUBIT).  Returns (err [shots, ceil(n/32)] int32,
    conv [shots] uint8, iters [shots] int32[, trace [shots, max_iter+1, n] float32]).
    Asynchronous on ``stream`` (default: torch's current stream)."""
    import torch
    from . import _native
    params = params or Params()
    shots = syn.shape[0]
    dev = syn.device
    if out is None:
        err = torch.empty((shots, code.nw), dtype=torch.int32, device=dev)
        conv = torch.empty((shots,), dtype=torch.uint8, device=dev)
        iters = torch.empty((shots,), dtype=torch.int32, device=dev)
    else:
        err, conv, iters = out
    _check_buffers(code, params, (syn, L0, err, conv, iters), host=False)
    p = params.to_c()
    sp = _stream_ptr(stream)
    if trace:
        tr = torch.full((shots, params.max_iter + 1, code.n), float("nan"), dtype=torch.float32, device=dev)
        _native.sagms_decode_trace(code.handle, p, shots, syn.data_ptr(), L0.data_ptr(), err.data_ptr(),
                                   conv.data_ptr(), iters.data_ptr(), tr.data_ptr(), sp)
        return err, conv, iters, tr
    _native.sagms_decode(code.handle, p, shots, syn.data_ptr(), L0.data_ptr(), err.data_ptr(), conv.data_ptr(),
                         iters.data_ptr(), sp)
    return err, conv, iters


def decode_host(code: DeviceCode, syn, L0, params: Params | None = None, out=None):
    """End-to-end decode from host memory (numpy or CPU torch tensors, ideally pinned):
    the library copies in, decodes and copies back with overlapped chunks.  Synchronous."""
    import numpy as np
    from . import _native
    params = params or Params()
    shots = syn.shape[0]

    def ptr(a):
        return a.data_ptr() if hasattr(a, "data_ptr") else a.ctypes.data

    if out is None:
        err = np.empty((shots, code.nw), dtype=np.uint32)
        conv = np.empty((shots,), dtype=np.uint8)
        iters = np.empty((shots,), dtype=np.int32)
    else:
        err, conv, iters = out
    _check_buffers(code, params, (syn, L0, err, conv, iters), host=True)
    _native.sagms_decode_host(code.handle, params.to_c(), shots, ptr(syn), ptr(L0), ptr(err), ptr(conv), ptr(iters))
    return err, conv, iters


KERNEL_NAMES = {0: "auto", 1: "one-shot-per-CTA", 2: "two-slot", 3: "two-group", 4: "two-group-qc",
                5: "two-group-qc-bp"}


def decode_plan(plan: int) -> dict:
    """Unpack a launch plan returned by sagms_autotune."""
    return {"kernel": KERNEL_NAMES[plan & 7],
            "ctas_per_sm": (plan >> 8) & 0xff, "chunk_lg": (plan >> 16) & 0xf}


class Job:
    """One batch of a mixed-code launch (sagms_decode_multi / sagms_graph_*): a loaded code,
    parameters and device tensors (outputs allocated here unless given)."""

    def __init__(self, code: DeviceCode, syn, L0, params: Params | None = None, out=None):
        import torch
        self.code, self.syn, self.L0 = code, syn, L0
        self.params = params or Params()
        shots = syn.shape[0]
        if out is None:
            out = (torch.empty((shots, code.nw), dtype=torch.int32, device=syn.device),
                   torch.empty((shots,), dtype=torch.uint8, device=syn.device),
                   torch.empty((shots,), dtype=torch.int32, device=syn.device))
        self.err, self.conv, self.iters = out
        _check_buffers(code, self.params, (syn, L0, self.err, self.conv, self.iters), host=False)

    def to_c(self):
        from . import _native
        return _native.sagms_job(self.code.handle, self.params.to_c(), self.syn.shape[0], self.syn.data_ptr(),
                                 self.L0.data_ptr(), self.err.data_ptr(), self.conv.data_ptr(), self.iters.data_ptr())


def decode_multi(jobs, stream=None):
    """Run all jobs in one call (overlapping on the GPU); asynchronous on ``stream``."""
    from . import _native
    _native.sagms_decode_multi([j.to_c() for j in jobs], _stream_ptr(stream))


class Graph:
    """A CUDA graph of one decode_multi over the jobs' fixed buffers; launch() replays it."""

    def __init__(self, jobs):
        from . import _native
        self._native = _native
        self.jobs = list(jobs)
        self.handle = _native.sagms_graph_create([j.to_c() for j in self.jobs])

    def launch(self, stream=None):
        self._native.sagms_graph_launch(self.handle, _stream_ptr(stream))

    def close(self):
        if getattr(self, "handle", None):
            self._native.sagms_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def autotune(code: DeviceCode, syn, L0, params: Params | None = None, stream=None):
    """Pick and store the fastest launch plan for this code on a sample batch; returns
    (plan, shots/s)."""
    import torch
    from . import _native
    params = params or Params()
    shots = syn.shape[0]
    err = torch.empty((shots, code.nw), dtype=torch.int32, device=syn.device)
    conv = torch.empty((shots,), dtype=torch.uint8, device=syn.device)
    iters = torch.empty((shots,), dtype=torch.int32, device=syn.device)
    _check_buffers(code, params, (syn, L0, err, conv, iters), host=False)
    return _native.sagms_autotune(code.handle, params.to_c(), shots, syn.data_ptr(), L0.data_ptr(), err.data_ptr(),
                                  conv.data_ptr(), iters.data_ptr(), _stream_ptr(stream))


class Server:
    """Continuous-batching decode server (sagms_server_*).  Requests carry host buffers
    (numpy arrays or CPU torch tensors; page-locked memory copies fastest) that the server
    keeps referenced until the request is released."""

    MODES = {"continuous": 0, "plain": 1}

    def __init__(self, mem_budget=1 << 30, max_inflight=16, mode="continuous", shots_per_cta=16):
        import ctypes
        from . import _native
        self._native = _native
        h = ctypes.c_void_p()
        _native._check(_native.lib().sagms_server_create(int(mem_budget), int(max_inflight), self.MODES[mode],
                                                         int(shots_per_cta), ctypes.byref(h)))
        self.handle = h.value
        self._bufs = {}
        self._codes = {}   # code id -> (DeviceCode, Params), to check request buffers

    def add_code(self, code: DeviceCode, params: Params | None = None) -> int:
        import ctypes
        cid = ctypes.c_int32()
        params = params or Params()
        p = params.to_c()
        self._native._check(self._native.lib().sagms_server_add_code(self.handle, code.handle, ctypes.byref(p),
                                                                     ctypes.byref(cid)))
        self._codes[cid.value] = (code, params)
        return cid.value

    def _check_request(self, code_id, bufs):
        # an unknown id is left to the library, which refuses it
        if int(code_id) in self._codes:
            code, params = self._codes[int(code_id)]
            _check_buffers(code, params, bufs, host=True)

    @staticmethod
    def _ptr(a):
        return a.data_ptr() if hasattr(a, "data_ptr") else a.ctypes.data

    def submit(self, code_id, syn, L0, err, conv, iters) -> int:
        import ctypes
        t = ctypes.c_uint64()
        shots = syn.shape[0]
        self._check_request(code_id, (syn, L0, err, conv, iters))
        self._native._check(self._native.lib().sagms_server_submit(
            self.handle, int(code_id), shots, self._ptr(syn), self._ptr(L0), self._ptr(err), self._ptr(conv),
            self._ptr(iters), ctypes.byref(t)))
        self._bufs[t.value] = (syn, L0, err, conv, iters)
        return t.value

    def poll(self, ticket, timeout_us=0) -> int:
        return self._native.lib().sagms_server_poll(self.handle, ticket, int(timeout_us))

    def wait(self, ticket, timeout_s=60.0):
        rc = self.poll(ticket, int(timeout_s * 1e6))
        self._native._check(rc)

    def cancel(self, ticket) -> int:
        return self._native.lib().sagms_server_cancel(self.handle, ticket)

    def times(self, ticket):
        import ctypes
        a, b = ctypes.c_int64(), ctypes.c_int64()
        self._native._check(self._native.lib().sagms_server_times(self.handle, ticket, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def release(self, ticket):
        rc = self._native.lib().sagms_server_release(self.handle, ticket)
        if rc == 0:
            self._bufs.pop(ticket, None)
        return rc

    def replay(self, code_ids, requests, arrival_ns):
        """Submit requests[i] = (syn, L0, err, conv, iters) at arrival_ns[i] after the call
        starts (native pacing); returns the tickets."""
        import ctypes
        import numpy as np
        n = len(requests)
        for cid, r in zip(code_ids, requests):
            self._check_request(cid, r)
        VP = ctypes.c_void_p * n
        cols = list(zip(*requests)) if n else [[]] * 5
        ptrs = [VP(*[self._ptr(a) for a in col]) for col in cols]
        ids = np.ascontiguousarray(code_ids, dtype=np.int32)
        shots = np.ascontiguousarray([r[0].shape[0] for r in requests], dtype=np.int64)
        arr = np.ascontiguousarray(arrival_ns, dtype=np.int64)
        tickets = np.zeros(n, dtype=np.uint64)
        P = ctypes.POINTER
        self._native._check(self._native.lib().sagms_server_replay(
            self.handle, n, ids.ctypes.data_as(P(ctypes.c_int32)), shots.ctypes.data_as(P(ctypes.c_int64)),
            arr.ctypes.data_as(P(ctypes.c_int64)), ptrs[0], ptrs[1], ptrs[2], ptrs[3], ptrs[4],
            tickets.ctypes.data_as(P(ctypes.c_uint64))))
        for t, r in zip(tickets, requests):
            self._bufs[int(t)] = r
        return [int(t) for t in tickets]

    def close(self):
        if getattr(self, "handle", None):
            self._native.lib().sagms_server_destroy(self.handle)
            self.handle = None
            self._bufs.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# --------------------------------------------------------------------------- Monte Carlo
def x_logicals(code):
    """X-logical operators of a CSS code object with ``hz_rows`` (H_Z rows as Python-int
    bitsets, as the GB generator provides): uint32 [k][ceil(n/32)] (computed in the library)."""
    import numpy as np
    from . import _native
    rows = [[j for j in range(code.n) if (r >> j) & 1] for r in code.hz_rows]
    hz_rp = np.concatenate([[0], np.cumsum([len(r) for r in rows])]).astype(np.int32)
    hz_ci = np.asarray([j for r in rows for j in r], dtype=np.int32)
    return _native.sagms_x_logicals(code.n, code.row_ptr, code.col_idx, hz_rp, hz_ci)


def llr(q: float) -> float:
    """The channel prior of a flip probability: ln((1 - q) / q) (Sec. II), for 0 < q < 1."""
    import math
    if not 0.0 < q < 1.0:
        raise ValueError(f"no finite prior for flip probability {q}: pass L0 explicitly")
    return math.log((1.0 - q) / q)


def mc_sample(code: DeviceCode, seed: int, q: float, shot0: int, shots: int, L0: float | None = None, stream=None):
    """Frames shot0 .. shot0 + shots - 1 of the on-device generator: (err int32 [shots, nw],
    syn int32 [shots, mw], L0 float32 [shots]) CUDA tensors.  Asynchronous on ``stream``."""
    import torch
    from . import _native
    err = torch.empty((shots, code.nw), dtype=torch.int32, device="cuda")
    syn = torch.empty((shots, code.mw), dtype=torch.int32, device="cuda")
    l0 = torch.empty((shots,), dtype=torch.float32, device="cuda")
    _native.sagms_mc_sample(code.handle, seed, q, llr(q) if L0 is None else L0, shot0, shots, err.data_ptr(),
                            syn.data_ptr(), l0.data_ptr(), _stream_ptr(stream))
    return err, syn, l0


def _check_mc_frames(code, name, a, shots, tail, kinds, size):
    dt, shape, contig, dev = _buffer_facts(a)
    if dt.kind not in kinds or dt.itemsize != size:
        raise TypeError(f"{name}: dtype {dt} (need a {size}-byte {'/'.join(kinds)} type)")
    if not contig or dev != f"cuda:{code.device}" or shape != (shots, *tail):
        raise ValueError(f"{name}: need a contiguous CUDA tensor on cuda:{code.device} of shape "
                         f"{[shots, *tail]}, got {list(shape)} on {dev}")


def mc_check(code: DeviceCode, err, err_hat, conv, iters, stream=None):
    """Logical check of decoded frames (logicals attached): (fail uint8 [shots] with 0 success,
    1 not converged, 2 logical error; counts dict).  Synchronises ``stream``."""
    import torch
    from . import _native
    shots = err.shape[0]
    for name, a in (("err", err), ("err_hat", err_hat)):
        _check_mc_frames(code, name, a, shots, (code.nw,), "iu", 4)
    _check_mc_frames(code, "conv", conv, shots, (), "u", 1)
    _check_mc_frames(code, "iters", iters, shots, (), "i", 4)
    fail = torch.empty((shots,), dtype=torch.uint8, device="cuda")
    counts = torch.zeros((5,), dtype=torch.int64, device="cuda")
    _native.sagms_mc_check(code.handle, shots, err.data_ptr(), err_hat.data_ptr(), conv.data_ptr(), iters.data_ptr(),
                           fail.data_ptr(), counts.data_ptr(), _stream_ptr(stream))
    c = counts.cpu().tolist()
    return fail, dict(zip(("shots", "failures", "not_converged", "logical", "iters_sum"), c))


def mc_run(code: DeviceCode, params: Params, seed: int, q: float, L0: float | None = None,
           target_failures: int = 500, max_shots: int = 20_000_000, batch: int = 1 << 22, counts=None):
    """The frame-error protocol of Sec. V (setup) for one noise level, entirely on the GPU:
    sample, decode and check batches until ``target_failures`` failures or ``max_shots``
    frames.  ``counts`` (a dict from an earlier call) continues the same frame sequence.
    Returns the counts dict."""
    from . import _native
    c = _native.sagms_mc_counts(**(counts or {}))
    _native.sagms_mc_run(code.handle, params.to_c(), seed, q, llr(q) if L0 is None else L0, target_failures,
                         max_shots, batch, c)
    return c.as_dict()
