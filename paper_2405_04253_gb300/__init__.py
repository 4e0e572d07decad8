"""GB300 (sm_103a) FNT-CDC / FNT-AEQ: Python binding of libfnt.

Argument marshalling only: every step of the path runs in the CUDA kernels of
libfnt.so (built in-tree by :func:`build`).  PyTorch supplies device memory and
streams; tensors are passed to the C ABI (include/fnt.h) as raw pointers.
There is no CPU fallback: without the library or a GPU every call raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .build import LIB, build  # noqa: F401

FNT_OK, FNT_ERR_INVALID, FNT_ERR_BOUND, FNT_ERR_NOMEM, FNT_ERR_BUSY, FNT_ERR_TIMEOUT, FNT_ERR_CUDA, \
    FNT_ERR_NOT_FOUND, FNT_ERR_CANCELLED = range(9)
OP_CDC, OP_AEQ, OP_CHAIN = 0, 1, 2

_STATUS = {0: "FNT_OK", 1: "FNT_ERR_INVALID", 2: "FNT_ERR_BOUND", 3: "FNT_ERR_NOMEM", 4: "FNT_ERR_BUSY",
           5: "FNT_ERR_TIMEOUT", 6: "FNT_ERR_CUDA", 7: "FNT_ERR_NOT_FOUND", 8: "FNT_ERR_CANCELLED"}


class FntError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class PlanDesc(ctypes.Structure):
    _fields_ = [("n_cdc", ctypes.c_int32), ("alpha_cdc", ctypes.c_int32), ("cdc_step", ctypes.c_int32),
                ("n_aeq", ctypes.c_int32), ("alpha_aeq", ctypes.c_int32), ("aeq_taps", ctypes.c_int32),
                ("mu_shift", ctypes.c_int32), ("rde_a", ctypes.c_int32), ("tap_init", ctypes.c_int32),
                ("aeq_update_period", ctypes.c_int32), ("aeq_segment", ctypes.c_int64), ("aeq_warmup", ctypes.c_int64),
                ("aeq_freq_sum", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class FrameC(ctypes.Structure):
    _fields_ = [("in_", ctypes.c_void_p), ("out", ctypes.c_void_p), ("cd_taps", ctypes.c_void_p),
                ("aeq_state", ctypes.c_void_p), ("n", ctypes.c_int64), ("n_pol", ctypes.c_int32),
                ("cd_len", ctypes.c_int32)]


class BatchC(ctypes.Structure):
    _fields_ = [("n_frames", ctypes.c_int32), ("host_buffers", ctypes.c_int32),
                ("frames", ctypes.POINTER(FrameC))]


class OpCounts(ctypes.Structure):
    _fields_ = [("cdc_mults_per_symbol", ctypes.c_double), ("aeq_mults_per_symbol", ctypes.c_double),
                ("cdc_butterflies_per_symbol", ctypes.c_double), ("aeq_cta_mults_per_symbol", ctypes.c_double)]


class Completion(ctypes.Structure):
    _fields_ = [("ticket", ctypes.c_uint64), ("link", ctypes.c_int32), ("status", ctypes.c_int32),
                ("n_sym", ctypes.c_int64), ("submit_us", ctypes.c_double), ("start_us", ctypes.c_double),
                ("done_us", ctypes.c_double)]


class SessionStats(ctypes.Structure):
    _fields_ = [("admitted", ctypes.c_uint64), ("completed", ctypes.c_uint64), ("failed", ctypes.c_uint64),
                ("cancelled", ctypes.c_uint64), ("waves", ctypes.c_uint64), ("chained_waves", ctypes.c_uint64),
                ("wave_frames", ctypes.c_uint64), ("max_wave", ctypes.c_uint64), ("arena_used", ctypes.c_uint64),
                ("arena_peak", ctypes.c_uint64), ("queued", ctypes.c_int32), ("in_flight", ctypes.c_int32)]


# fnt_request (batched session admission) and fnt_completion as numpy records
REQUEST_DTYPE = np.dtype([("link", np.int32), ("reserved", np.int32), ("in_", np.uint64), ("n", np.int64),
                          ("out", np.uint64)], align=True)
COMPLETION_DTYPE = np.dtype([("ticket", np.uint64), ("link", np.int32), ("status", np.int32), ("n_sym", np.int64),
                             ("submit_us", np.float64), ("start_us", np.float64), ("done_us", np.float64)],
                            align=True)
assert REQUEST_DTYPE.itemsize == 32 and COMPLETION_DTYPE.itemsize == ctypes.sizeof(Completion)


# Every symbol include/fnt.h declares, with (restype, argtypes).
_VP, _I32, _I64, _SZ = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
SIGNATURES = {
    "fnt_last_error": (_SZ, [ctypes.c_char_p, _SZ]),
    "fnt_version": (ctypes.c_char_p, []),
    "fnt_plan_desc_default": (None, [ctypes.POINTER(PlanDesc)]),
    "fnt_plan_create": (_I32, [ctypes.POINTER(PlanDesc), ctypes.POINTER(_VP)]),
    "fnt_plan_destroy": (_I32, [_VP]),
    "fnt_plan_set_launch": (_I32, [_VP, _I32, _I32]),
    "fnt_plan_set_pipeline": (_I32, [_VP, _I32]),
    "fnt_plan_set_tensor_gradient": (_I32, [_VP, _I32]),
    "fnt_plan_set_cdc_items": (_I32, [_VP, _I32]),
    "fnt_plan_initial_taps": (_I32, [_VP, _VP]),
    "fnt_plan_set_aeq_occupancy": (_I32, [_VP, _I32]),
    "fnt_plan_set_aeq_kernel": (_I32, [_VP, _I32]),
    "fnt_plan_set_cdc_kernel": (_I32, [_VP, _I32]),
    "fnt_plan_cdc_kernel_for": (_I32, [_VP, _I64]),
    "fnt_plan_set_test_inject": (_I32, [_VP, _I32]),
    "fnt_device_faults": (_I32, [_I32, ctypes.POINTER(ctypes.c_uint32)]),
    "fnt_plan_aeq_kernel_for": (_I32, [_VP, _I64, _I64]),
    "fnt_op_counts_for": (_I32, [ctypes.POINTER(PlanDesc), _I32, ctypes.POINTER(OpCounts)]),
    "fnt_cdc_run": (_I32, [_VP, ctypes.POINTER(BatchC), _VP]),
    "fnt_aeq_run": (_I32, [_VP, ctypes.POINTER(BatchC), _VP]),
    "fnt_cdc_aeq_run": (_I32, [_VP, ctypes.POINTER(BatchC), _VP]),
    "fnt_batch_create": (_I32, [_VP, ctypes.POINTER(BatchC), _I32, _I32, ctypes.POINTER(_VP)]),
    "fnt_batch_launch": (_I32, [_VP, _VP]),
    "fnt_batch_launch_stage": (_I32, [_VP, _I32, _VP]),
    "fnt_batch_set_input_copy": (_I32, [_VP, _I32]),
    "fnt_batch_kernel_count": (_I32, [_VP]),
    "fnt_batch_destroy": (_I32, [_VP]),
    "fnt_cdc_aeq_run_noalloc": (_I32, [_VP, ctypes.POINTER(FrameC), _VP]),
    "fnt_session_create": (_I32, [_VP, _I32, _SZ, _I32, ctypes.POINTER(_VP)]),
    "fnt_session_set_link": (_I32, [_VP, _I32, _VP, _I32]),
    "fnt_session_submit": (_I32, [_VP, _I32, _VP, _I64, _VP, ctypes.POINTER(ctypes.c_uint64)]),
    "fnt_session_submit_many": (_I32, [_VP, _VP, _I32, _VP, ctypes.POINTER(_I32)]),
    "fnt_session_cancel": (_I32, [_VP, ctypes.c_uint64]),
    "fnt_session_get_stats": (_I32, [_VP, ctypes.POINTER(SessionStats)]),
    "fnt_session_poll": (_I32, [_VP, _I32, ctypes.POINTER(Completion), _I32, ctypes.POINTER(_I32)]),
    "fnt_session_pending": (_I32, [_VP]),
    "fnt_session_get_link_state": (_I32, [_VP, _I32, _VP]),
    "fnt_session_set_link_state": (_I32, [_VP, _I32, _VP]),
    "fnt_session_inject_failures": (_I32, [_VP, _I32]),
    "fnt_session_destroy": (_I32, [_VP]),
}

_lib = None


def lib(path: str | None = None):
    """Loads libfnt.so (building it first if needed).  Raises if it cannot."""
    global _lib
    if _lib is None:
        p = path or os.environ.get("FNT_LIB") or build()
        L = ctypes.CDLL(p)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


FAULT_CDC_WINDOW_WAIT = 1


def device_faults(clear: bool = False) -> int:
    """The current device's fault word (bits set by bounded waits that ran out)."""
    v = ctypes.c_uint32()
    check(lib().fnt_device_faults(int(bool(clear)), ctypes.byref(v)))
    return int(v.value)


def last_error() -> str:
    buf = ctypes.create_string_buffer(1024)
    lib().fnt_last_error(buf, 1024)
    return buf.value.decode()


def check(status: int) -> None:
    if status != FNT_OK:
        raise FntError(status, last_error())


def _ptr(t) -> int | None:
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return t.data_ptr()


def _stream_handle(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def default_desc(**over) -> PlanDesc:
    d = PlanDesc()
    lib().fnt_plan_desc_default(ctypes.byref(d))
    for k, v in over.items():
        setattr(d, k, v)
    return d


def op_counts(cd_len: int, **over) -> dict:
    """Tab. 1 multiplication counts of the kernels for a plan description."""
    d = default_desc(**over)
    oc = OpCounts()
    check(lib().fnt_op_counts_for(ctypes.byref(d), cd_len, ctypes.byref(oc)))
    return {f: getattr(oc, f) for f, _ in OpCounts._fields_}


class Plan:
    """A validated CDC / AEQ configuration (fnt_plan)."""

    def __init__(self, **over):
        self.desc = default_desc(**over)
        h = ctypes.c_void_p()
        check(lib().fnt_plan_create(ctypes.byref(self.desc), ctypes.byref(h)))
        self.handle = h

    def close(self):
        if self.handle:
            lib().fnt_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_launch(self, cdc_warps: int = 0, aeq_warps: int = 0):
        check(lib().fnt_plan_set_launch(self.handle, cdc_warps, aeq_warps))

    def set_pipeline(self, chunks: int):
        check(lib().fnt_plan_set_pipeline(self.handle, chunks))

    def set_aeq_occupancy(self, max_warps_per_sm: int):
        """Caps the AEQ warps resident per SM (0 = no cap); same results."""
        check(lib().fnt_plan_set_aeq_occupancy(self.handle, int(max_warps_per_sm)))

    def set_aeq_kernel(self, kind: int):
        """AEQ kernel: 1 a warp per (chain, polarisation), 2 a CTA per one,
        0 automatic; same results."""
        check(lib().fnt_plan_set_aeq_kernel(self.handle, int(kind)))

    def set_cdc_kernel(self, kind: int):
        """CDC kernel: 1 a block per lane, 2 a block per 8 threads, 0
        automatic; same results."""
        check(lib().fnt_plan_set_cdc_kernel(self.handle, int(kind)))

    def set_test_inject(self, mode: int):
        """Test hook: 1 makes the CDC's bulk-copy window waits run out (see
        fnt_plan_set_test_inject); 0 is normal operation."""
        check(lib().fnt_plan_set_test_inject(self.handle, int(mode)))

    def cdc_kernel_for(self, n_items: int) -> int:
        """The CDC kernel (1 or 2) a launch of n_items 32-block work items takes."""
        return int(lib().fnt_plan_cdc_kernel_for(self.handle, int(n_items)))

    def aeq_kernel_for(self, n_chains: int, longest_symbols: int) -> int:
        """The AEQ kernel (1 or 2) a launch of n_chains chains, the longest of
        longest_symbols symbols, takes."""
        return int(lib().fnt_plan_aeq_kernel_for(self.handle, int(n_chains), int(longest_symbols)))

    def initial_state(self) -> np.ndarray:
        """The plan's initial AEQ taps, int32 [4 (S2)][4 (S1)][16]."""
        st = np.zeros((4, 4, 16), np.int32)
        check(lib().fnt_plan_initial_taps(self.handle, st.ctypes.data))
        return st

    def set_cdc_items(self, pols: int):
        """CDC items of one (1) or both (2) polarisations; 0 = automatic."""
        check(lib().fnt_plan_set_cdc_items(self.handle, pols))

    def set_tensor_gradient(self, on: bool):
        """AEQ gradient on the tensor cores (exact; same results)."""
        check(lib().fnt_plan_set_tensor_gradient(self.handle, int(bool(on))))


class Frame:
    """One frame: `x` input, `out` result, `taps` int8 [L, 2] numpy (host),
    `state` int32 [4, 4, 16] device tensor or None.  `n` is the sample (or,
    for the AEQ alone, symbol) count; it defaults to x.shape[0]."""

    def __init__(self, x, out, taps=None, state=None, n: int | None = None, n_pol: int = 2):
        self.x, self.out, self.state = x, out, state
        self.taps = None if taps is None else np.ascontiguousarray(taps, dtype=np.int8)
        self.n = int(x.shape[0]) if n is None else int(n)
        self.n_pol = n_pol

    def c(self) -> FrameC:
        return FrameC(_ptr(self.x), _ptr(self.out), _ptr(self.taps), _ptr(self.state), self.n, self.n_pol,
                      0 if self.taps is None else self.taps.shape[0])


def _batch(frames, host: bool):
    arr = (FrameC * max(1, len(frames)))(*[f.c() for f in frames])
    return BatchC(len(frames), 1 if host else 0, arr), arr


def cdc_run(plan: Plan, frames, stream=None, host: bool = False):
    b, keep = _batch(frames, host)
    check(lib().fnt_cdc_run(plan.handle, ctypes.byref(b), None if host and stream is None else _stream_handle(stream)))


def aeq_run(plan: Plan, frames, stream=None, host: bool = False):
    b, keep = _batch(frames, host)
    check(lib().fnt_aeq_run(plan.handle, ctypes.byref(b), None if host and stream is None else _stream_handle(stream)))


def cdc_aeq_run(plan: Plan, frames, stream=None, host: bool = False):
    b, keep = _batch(frames, host)
    check(lib().fnt_cdc_aeq_run(plan.handle, ctypes.byref(b),
                                None if host and stream is None else _stream_handle(stream)))


NOALLOC_MAX_SAMPLES = 1 << 21


def cdc_aeq_run_noalloc(plan: Plan, frame: Frame, stream=None):
    """The chain for one frame through fnt_cdc_aeq_run_noalloc: no memory is
    allocated; its scratch is a fixed device array inside libfnt shared by all
    calls on the device (see include/fnt.h)."""
    fc = frame.c()
    check(lib().fnt_cdc_aeq_run_noalloc(plan.handle, ctypes.byref(fc), _stream_handle(stream)))


class Batch:
    """A prepared batch (fnt_batch): work lists built and uploaded once."""

    def __init__(self, plan: Plan, frames, op: int, use_graph: bool = True, host: bool = False):
        """host: the frames' buffers are page-locked host memory, used in place."""
        self.plan, self.frames = plan, frames
        b, keep = _batch(frames, host)
        h = ctypes.c_void_p()
        check(lib().fnt_batch_create(plan.handle, ctypes.byref(b), op, 1 if use_graph else 0, ctypes.byref(h)))
        self.handle = h

    def launch(self, stream=None):
        check(lib().fnt_batch_launch(self.handle, _stream_handle(stream)))

    def set_input_copy(self, on: bool):
        """Host-buffer batches: copy the inputs to the device by DMA on the
        batch's own stream, started at launch() without waiting for `stream`
        (the input must hold its data when launch() is called)."""
        check(lib().fnt_batch_set_input_copy(self.handle, int(bool(on))))

    def launch_stage(self, stage: int, stream=None):
        check(lib().fnt_batch_launch_stage(self.handle, stage, _stream_handle(stream)))

    def kernel_count(self) -> int:
        return int(lib().fnt_batch_kernel_count(self.handle))

    def close(self):
        if self.handle:
            lib().fnt_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def chain_nsym(n: int, L: int) -> int:
    """Symbols the chain writes for n samples and L CD taps."""
    phase = ((L - 1) // 2) & 1
    return max(0, (n - phase + 1) // 2)


class Requests:
    """Prepared fnt_request records for fnt_session_submit_many: frame i goes to
    links[i] with input xs[i] and output outs[i] (tensors or page-locked arrays,
    kept alive here)."""

    def __init__(self, links, xs, outs, ns=None):
        self.rec = np.zeros(len(xs), REQUEST_DTYPE)
        self.rec["link"] = np.asarray(links, dtype=np.int32)
        self.rec["in_"] = [_ptr(x) or 0 for x in xs]
        self.rec["n"] = [int(x.shape[0]) for x in xs] if ns is None else np.asarray(ns, dtype=np.int64)
        self.rec["out"] = [_ptr(o) or 0 for o in outs]
        self.bufs = list(zip(xs, outs))

    def __len__(self) -> int:
        return len(self.rec)


class Session:
    """Continuous-batching serving session (fnt_session)."""

    def __init__(self, plan: Plan, n_links: int, mem_cap_bytes: int, n_streams: int = 4):
        self.plan = plan
        h = ctypes.c_void_p()
        check(lib().fnt_session_create(plan.handle, n_links, mem_cap_bytes, n_streams, ctypes.byref(h)))
        self.handle = h
        self._keep = {}
        self._done = np.zeros(0, COMPLETION_DTYPE)

    def set_link(self, link: int, taps):
        t = np.ascontiguousarray(taps, dtype=np.int8)
        check(lib().fnt_session_set_link(self.handle, link, t.ctypes.data, t.shape[0]))

    def submit(self, link: int, x, out, n: int | None = None) -> int:
        """Returns the ticket; raises FntError (status FNT_ERR_BUSY) when the
        memory cap refuses admission."""
        tk = ctypes.c_uint64()
        check(lib().fnt_session_submit(self.handle, link, _ptr(x), int(x.shape[0]) if n is None else int(n),
                                       _ptr(out), ctypes.byref(tk)))
        self._keep[tk.value] = (x, out)
        return tk.value

    def try_submit(self, link: int, x, out, n: int | None = None) -> int | None:
        tk = ctypes.c_uint64()
        st = lib().fnt_session_submit(self.handle, link, _ptr(x), int(x.shape[0]) if n is None else int(n),
                                      _ptr(out), ctypes.byref(tk))
        if st == FNT_ERR_BUSY:
            return None
        check(st)
        self._keep[tk.value] = (x, out)
        return tk.value

    def submit_many(self, reqs: Requests, start: int = 0, count: int | None = None) -> list[int]:
        """Admits reqs[start:start+count] in order with one call; returns the
        tickets of those admitted (a prefix: admission stops where the memory
        cap refuses a request).  Other errors raise FntError."""
        n = len(reqs) - start if count is None else int(count)
        if n <= 0:
            return []
        tk = np.zeros(n, np.uint64)
        na = ctypes.c_int32()
        st = lib().fnt_session_submit_many(self.handle, reqs.rec.ctypes.data + start * REQUEST_DTYPE.itemsize, n,
                                           tk.ctypes.data, ctypes.byref(na))
        out = tk[:na.value].tolist()
        for i, t in enumerate(out):
            self._keep[t] = reqs.bufs[start + i]
        if st != FNT_ERR_BUSY:
            check(st)
        return out

    def poll_array(self, timeout_us: int = 0, max_done: int = 4096) -> np.ndarray:
        """As :meth:`poll`, returning the completions as a COMPLETION_DTYPE array."""
        if self._done.shape[0] < max_done:
            self._done = np.zeros(max_done, COMPLETION_DTYPE)
        nd = ctypes.c_int32()
        st = lib().fnt_session_poll(self.handle, timeout_us, self._done.ctypes.data_as(ctypes.POINTER(Completion)),
                                    max_done, ctypes.byref(nd))
        if st == FNT_ERR_TIMEOUT:
            return self._done[:0].copy()
        check(st)
        got = self._done[:nd.value].copy()
        for t in got["ticket"].tolist():
            self._keep.pop(t, None)
        return got

    def poll(self, timeout_us: int = 0, max_done: int = 1024):
        arr = (Completion * max_done)()
        nd = ctypes.c_int32()
        st = lib().fnt_session_poll(self.handle, timeout_us, arr, max_done, ctypes.byref(nd))
        if st == FNT_ERR_TIMEOUT:
            return []
        check(st)
        out = []
        for i in range(nd.value):
            c = arr[i]
            self._keep.pop(c.ticket, None)
            out.append(dict(ticket=c.ticket, link=c.link, status=c.status, n_sym=c.n_sym, submit_us=c.submit_us,
                            start_us=c.start_us, done_us=c.done_us))
        return out

    def cancel(self, ticket: int) -> bool:
        """Cancels a request not launched yet (it completes as FNT_ERR_CANCELLED);
        False when it is already launched, complete or unknown."""
        st = lib().fnt_session_cancel(self.handle, int(ticket))
        if st == FNT_ERR_NOT_FOUND:
            return False
        check(st)
        return True

    def stats(self) -> dict:
        st = SessionStats()
        check(lib().fnt_session_get_stats(self.handle, ctypes.byref(st)))
        return {f: getattr(st, f) for f, _ in SessionStats._fields_}

    def pending(self) -> int:
        return int(lib().fnt_session_pending(self.handle))

    def get_link_state(self, link: int) -> np.ndarray:
        st = np.zeros((4, 4, 16), np.int32)
        check(lib().fnt_session_get_link_state(self.handle, link, st.ctypes.data))
        return st

    def set_link_state(self, link: int, state):
        st = np.ascontiguousarray(state, dtype=np.int32)
        check(lib().fnt_session_set_link_state(self.handle, link, st.ctypes.data))

    def inject_failures(self, n_waves: int):
        check(lib().fnt_session_inject_failures(self.handle, n_waves))

    def close(self):
        if self.handle:
            lib().fnt_session_destroy(self.handle)
            self.handle = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
