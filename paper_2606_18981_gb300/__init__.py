"""qftfft: GB300 QFT->FFT library -- thin ctypes binding over libqftfft.so.

Every step of the transform runs in the library's CUDA kernels; this module
only marshals arguments (device pointers from torch tensors, CUDA stream
handles, sizes) into the C ABI declared in ``include/qftfft.h``.  There is no
CPU fallback: importing the package fails loudly if ``libqftfft.so`` has not
been built (``python paper_2606_18981_gb300/build.py``).

Conventions (Markidis et al., Sec. 2-3): qubit q_j is bit j of the array index;
FORWARD uses omega_N = e^{-2 pi i / N}; the circuit is U = DFT_N / sqrt(N);
scale modes STATE / UNITARY / UNNORM / INV_N are the decode rules of Sec. 3
step 4; order NATURAL applies the qubit-reversal swaps, BITREV leaves them to
the caller (out[i] holds frequency bitrev_n(i)).
"""
from __future__ import annotations

import ctypes
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libqftfft.so")

C64, C128 = 0, 1
FORWARD, INVERSE = -1, +1
SCALE_STATE, SCALE_UNITARY, SCALE_UNNORM, SCALE_INV_N = 0, 1, 2, 3
ORDER_NATURAL, ORDER_BITREV = 0, 1
PREC_NATIVE, PREC_TF32, PREC_BF16, PREC_BF16X3, PREC_FP16, PREC_FP16X3, PREC_FP64 = 0, 1, 2, 3, 4, 5, 6
OK, ERR_BAD_ARG, ERR_SIZE, ERR_BUDGET, ERR_CUDA, ERR_TIMEOUT, ERR_NOMEM, ERR_UNSUPPORTED, ERR_STATE, ERR_CANCELED = \
    0, -1, -2, -3, -4, -5, -6, -7, -8, -9

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build the CUDA library first "
                      "(python paper_2606_18981_gb300/build.py)")

_lib = ctypes.CDLL(LIB_PATH)


class QftError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        msg = _lib.qft_strerror(code).decode()
        if code == ERR_CUDA:
            msg += f" (cudaError {_lib.qft_last_cuda_error()})"
        super().__init__(f"{what}: {msg} [{code}]" if what else f"{msg} [{code}]")


class PlanInfo(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("k_eff", ctypes.c_int), ("direction", ctypes.c_int),
                ("dtype", ctypes.c_int), ("order", ctypes.c_int),
                ("n_h", ctypes.c_longlong), ("n_cp", ctypes.c_longlong), ("n_swap", ctypes.c_longlong),
                ("passes", ctypes.c_int), ("wires_per_pass", ctypes.c_int * 8),
                ("stages_per_pass", ctypes.c_int * 8), ("tile_bits", ctypes.c_int * 8),
                ("coalesce_bits", ctypes.c_int * 8), ("workspace_bytes", ctypes.c_size_t),
                ("bytes_per_execute", ctypes.c_longlong), ("n_addr", ctypes.c_int), ("w0", ctypes.c_int),
                ("fused_blocks", ctypes.c_int), ("max_fused_size", ctypes.c_int)]


class Opts(ctypes.Structure):
    _fields_ = [("order", ctypes.c_int), ("tile_bits", ctypes.c_int), ("coalesce_bits", ctypes.c_int),
                ("max_stage_bits", ctypes.c_int), ("wait_limit_ms", ctypes.c_int),
                ("test_skip_first_load", ctypes.c_int), ("threads", ctypes.c_int),
                ("precision", ctypes.c_int), ("paired", ctypes.c_int), ("pass_split", ctypes.c_int)]


_vp = ctypes.c_void_p
_lib.qft_version.restype = ctypes.c_int
_lib.qft_strerror.restype = ctypes.c_char_p
_lib.qft_strerror.argtypes = [ctypes.c_int]
_lib.qft_last_cuda_error.restype = ctypes.c_int
_lib.qft_plan_create.argtypes = [ctypes.POINTER(_vp), ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                 ctypes.POINTER(Opts)]
_lib.qft_plan_destroy.argtypes = [_vp]
_lib.qft_plan_create_subset.argtypes = [ctypes.POINTER(_vp), ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_int, ctypes.c_int, ctypes.POINTER(Opts)]
_lib.qft_plan_get_info.argtypes = [_vp, ctypes.POINTER(PlanInfo)]
_lib.qft_workspace_size.argtypes = [_vp]
_lib.qft_workspace_size.restype = ctypes.c_size_t
_lib.qft_load.argtypes = [_vp, _vp, _vp, ctypes.c_size_t, ctypes.c_int, _vp]
_lib.qft_load_padded.argtypes = [_vp, _vp, _vp, ctypes.c_size_t, ctypes.c_int, _vp]
_lib.qft_execute.argtypes = [_vp, _vp, _vp, _vp, ctypes.c_int, _vp]
_lib.qft_execute_pass.argtypes = [_vp, ctypes.c_int, _vp, _vp, _vp, ctypes.c_int, _vp]
_lib.qft_read.argtypes = [_vp, _vp, _vp, ctypes.c_int, _vp]
_lib.qft_execute_noalloc.argtypes = [_vp, _vp, _vp, ctypes.c_int, _vp]
_lib.qft_noalloc_status.argtypes = [_vp]
_lib.qft_noalloc_status.restype = ctypes.c_int
_lib.qft_execute_oop.argtypes = [_vp, _vp, _vp, _vp, _vp, ctypes.c_int, _vp]
_lib.qft_qpe_workspace_size.argtypes = [ctypes.c_int, ctypes.c_int]
_lib.qft_qpe_workspace_size.restype = ctypes.c_size_t
_lib.qft_qpe_prepare.argtypes = [_vp, ctypes.c_int, ctypes.c_int, _vp, _vp, ctypes.c_int, _vp, _vp]
_lib.qft_qpe_probabilities.argtypes = [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp, _vp]
_lib.qft_mc_workspace_size.argtypes = [ctypes.c_int]
_lib.qft_mc_workspace_size.restype = ctypes.c_size_t
_lib.qft_mc_prepare.argtypes = [ctypes.c_int, ctypes.c_int, _vp, _vp, _vp]
_lib.qft_mc_sample.argtypes = [ctypes.c_int, ctypes.c_int, _vp, _vp, _vp, ctypes.c_int64, _vp, _vp, _vp]
_lib.qft_mc_bins.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp, _vp, ctypes.c_int64, _vp, ctypes.c_int,
                             _vp, _vp, _vp]
_lib.qft_mc_sparse_workspace_size.argtypes = [ctypes.c_int64]
_lib.qft_mc_sparse_workspace_size.restype = ctypes.c_size_t
_lib.qft_mc_prepare_sparse.argtypes = [ctypes.c_int64, ctypes.c_int, _vp, _vp, _vp]
_lib.qft_mc_sample_sparse.argtypes = [ctypes.c_int64, ctypes.c_int, _vp, _vp, _vp, _vp, ctypes.c_int64, _vp, _vp, _vp]
_lib.qft_rplan_create.argtypes = [ctypes.POINTER(_vp), ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(Opts)]
_lib.qft_rplan_destroy.argtypes = [_vp]
_lib.qft_rplan_workspace_size.argtypes = [_vp]
_lib.qft_rplan_workspace_size.restype = ctypes.c_size_t
_lib.qft_rplan_execute.argtypes = [_vp, _vp, _vp, _vp, ctypes.c_int, _vp]
_lib.qft_get_scale_in.argtypes = [_vp, _vp, ctypes.POINTER(ctypes.c_double), _vp]
_lib.qft_check_status.argtypes = [_vp, _vp, _vp]
_lib.qft_plan_describe_pass.argtypes = [_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_longlong), ctypes.c_int]

_lib.qft_batch_workspace_size.argtypes = [ctypes.POINTER(_vp), ctypes.c_int]
_lib.qft_batch_workspace_size.restype = ctypes.c_size_t
_lib.qft_batch_create.argtypes = [ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.c_int, _vp,
                                  ctypes.c_size_t, _vp, ctypes.c_int]
_lib.qft_batch_execute.argtypes = [_vp, _vp]
_lib.qft_batch_status.argtypes = [_vp, _vp]


class BatchInfo(ctypes.Structure):
    _fields_ = [("transforms", ctypes.c_int), ("wide_groups", ctypes.c_int), ("wide_transforms", ctypes.c_int),
                ("persistent_items", ctypes.c_int), ("kernel_launches", ctypes.c_int), ("side_streams", ctypes.c_int)]


_lib.qft_batch_get_info.argtypes = [_vp, ctypes.POINTER(BatchInfo)]
_lib.qft_batch_destroy.argtypes = [_vp]

class Request(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("k", ctypes.c_int), ("direction", ctypes.c_int), ("dtype", ctypes.c_int),
                ("order", ctypes.c_int), ("scale_mode", ctypes.c_int), ("input", _vp), ("input_on_device", ctypes.c_int),
                ("output", _vp), ("output_on_device", ctypes.c_int), ("scale_in_out", ctypes.POINTER(ctypes.c_double))]


class ServerStats(ctypes.Structure):
    _fields_ = [("completed", ctypes.c_longlong), ("failed", ctypes.c_longlong), ("pending", ctypes.c_longlong),
                ("in_flight", ctypes.c_longlong), ("bytes_in_use", ctypes.c_size_t), ("bytes_pooled", ctypes.c_size_t),
                ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double), ("max_ms", ctypes.c_double),
                ("requests_per_s", ctypes.c_double), ("batches", ctypes.c_longlong),
                ("batched_requests", ctypes.c_longlong)]


_lib.qft_server_create.argtypes = [ctypes.POINTER(_vp), ctypes.c_size_t, ctypes.c_int, ctypes.c_int]
_lib.qft_server_submit.argtypes = [_vp, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_uint64)]
_lib.qft_server_poll.argtypes = [_vp, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int)]
_lib.qft_server_wait.argtypes = [_vp, ctypes.c_uint64, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
_lib.qft_server_get_stats.argtypes = [_vp, ctypes.POINTER(ServerStats)]
_lib.qft_server_reset_stats.argtypes = [_vp]
_lib.qft_server_destroy.argtypes = [_vp]
_lib.qft_server_cancel.argtypes = [_vp, ctypes.c_uint64]
_lib.qft_server_inject_alloc_failures.argtypes = [_vp, ctypes.c_int]
_lib.qft_server_set_batching.argtypes = [_vp, ctypes.c_int]

lib = _lib  # the raw ctypes handle (tests call the C ABI through it)


def _check(rc: int, what: str) -> int:
    if rc < 0:
        raise QftError(rc, what)
    return rc


def _dtype_code(dtype) -> int:
    if dtype in (C64, "c64", "complex64"):
        return C64
    if dtype in (C128, "c128", "complex128"):
        return C128
    s = str(dtype)
    if s.endswith("complex64"):
        return C64
    if s.endswith("complex128"):
        return C128
    raise ValueError(f"unsupported dtype {dtype!r}")


def _stream_handle(stream) -> int | None:
    if stream is None:
        import torch

        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _ptr(t) -> int:
    return t if isinstance(t, int) else t.data_ptr()


class Plan:
    """A planned (A)QFT: n qubits, cutoff k (-1 or >= n-1: exact), direction, dtype, order."""

    def __init__(self, n: int, k: int = -1, direction: int = FORWARD, dtype="c64", order: int = ORDER_NATURAL,
                 tile_bits: int = 0, coalesce_bits: int = 0, max_stage_bits: int = 0,
                 wait_limit_ms: int = 0, test_skip_first_load: int = 0, threads: int = 0, precision: int = 0,
                 paired: int = 0, pass_split: int = 0, tuned: bool = False, n_addr: int | None = None,
                 w0: int = 0):
        """n_addr / w0: a QFT on index bits [w0, w0 + n) of 2^n_addr amplitudes (qft_plan_create_subset)."""
        self._h = _vp()
        self.n, self.k, self.direction = int(n), int(k), int(direction)
        self.n_addr = int(n) if n_addr is None else int(n_addr)
        self.w0 = int(w0)
        subset = self.n_addr != self.n or self.w0 != 0
        self.dtype = _dtype_code(dtype)
        self.order = int(order)
        if tuned and precision == 0 and not subset:  # plan shape from the autotuner's cache, where it has one
            from .autotune import best_opts

            t = best_opts(self.n, "c64" if self.dtype == C64 else "c128")
            tile_bits = tile_bits or t.get("tile_bits", 0)
            coalesce_bits = coalesce_bits or t.get("coalesce_bits", 0)
            max_stage_bits = max_stage_bits or t.get("max_stage_bits", 0)
            threads = threads or t.get("threads", 0)
            paired = paired or t.get("paired", 0)
            pass_split = pass_split or t.get("pass_split", 0)
        opts = Opts(order, tile_bits, coalesce_bits, max_stage_bits, wait_limit_ms, test_skip_first_load, threads,
                    precision, paired, pass_split)
        if subset:
            _check(_lib.qft_plan_create_subset(ctypes.byref(self._h), self.n_addr, self.w0, self.n, self.k,
                                               self.direction, self.dtype, ctypes.byref(opts)),
                   "qft_plan_create_subset")
        else:
            _check(_lib.qft_plan_create(ctypes.byref(self._h), self.n, self.k, self.direction, self.dtype,
                                        ctypes.byref(opts)), "qft_plan_create")

    @property
    def handle(self) -> int:
        return self._h.value

    @property
    def N(self) -> int:
        """Amplitudes of the state buffer (2^n_addr)."""
        return 1 << self.n_addr

    @property
    def elem_bytes(self) -> int:
        return 8 if self.dtype == C64 else 16

    def info(self) -> PlanInfo:
        inf = PlanInfo()
        _check(_lib.qft_plan_get_info(self._h, ctypes.byref(inf)), "qft_plan_get_info")
        return inf

    def workspace_size(self) -> int:
        return int(_lib.qft_workspace_size(self._h))

    def describe_pass(self, i: int) -> list[int]:
        buf = (ctypes.c_longlong * 1024)()
        m = _check(_lib.qft_plan_describe_pass(self._h, i, buf, 1024), "qft_plan_describe_pass")
        return list(buf[:m])

    def alloc_workspace(self, device="cuda"):
        import torch

        return torch.empty(self.workspace_size(), dtype=torch.uint8, device=device)

    def load(self, state, src, stream=None, pad: bool = False) -> None:
        """Copy src (host or device tensor / numpy array) into the device state buffer.
        pad=True: src may be shorter than 2^n; the rest of the state is zeroed."""
        on_dev = 1
        if hasattr(src, "is_cuda"):
            on_dev = 1 if src.is_cuda else 0
            ptr, ln = src.data_ptr(), src.numel()
        else:  # numpy
            on_dev, ptr, ln = 0, src.ctypes.data, src.size
        fn = _lib.qft_load_padded if pad else _lib.qft_load
        _check(fn(self._h, _ptr(state), ptr, ln, on_dev, _stream_handle(stream)), "qft_load")

    def execute(self, state, workspace, scale_mode: int = SCALE_STATE, scale_out=None, stream=None) -> None:
        """Run the transform in place on the device state tensor (async on stream)."""
        _check(_lib.qft_execute(self._h, _ptr(state), _ptr(workspace),
                                _ptr(scale_out) if scale_out is not None else None,
                                int(scale_mode), _stream_handle(stream)), "qft_execute")

    def execute_oop(self, inp, out, workspace, scale_mode: int = SCALE_STATE, scale_out=None, stream=None) -> None:
        """Run the transform out of place: reads inp (unchanged), writes out."""
        _check(_lib.qft_execute_oop(self._h, _ptr(inp), _ptr(out), _ptr(workspace),
                                    _ptr(scale_out) if scale_out is not None else None,
                                    int(scale_mode), _stream_handle(stream)), "qft_execute_oop")

    def execute_pass(self, i: int, state, workspace, scale_mode: int = SCALE_STATE, scale_out=None,
                     stream=None) -> None:
        """Launch pass i only (passes 0..P-1 in order on one stream == execute)."""
        _check(_lib.qft_execute_pass(self._h, int(i), _ptr(state), _ptr(workspace),
                                     _ptr(scale_out) if scale_out is not None else None,
                                     int(scale_mode), _stream_handle(stream)), "qft_execute_pass")

    def execute_noalloc(self, state, scale_mode: int = SCALE_STATE, scale_out=None, stream=None) -> None:
        """Run the transform with the library's fixed device scratch (no allocation)."""
        _check(_lib.qft_execute_noalloc(self._h, _ptr(state), _ptr(scale_out) if scale_out is not None else None,
                                        int(scale_mode), _stream_handle(stream)), "qft_execute_noalloc")

    def read(self, state, dst, stream=None) -> None:
        on_dev = 1 if getattr(dst, "is_cuda", False) else 0
        ptr = dst.data_ptr() if hasattr(dst, "data_ptr") else dst.ctypes.data
        _check(_lib.qft_read(self._h, _ptr(state), ptr, on_dev, _stream_handle(stream)), "qft_read")

    def scale_in(self, workspace, stream=None) -> float:
        out = ctypes.c_double()
        _check(_lib.qft_get_scale_in(self._h, _ptr(workspace), ctypes.byref(out), _stream_handle(stream)),
               "qft_get_scale_in")
        return out.value

    def status(self, workspace, stream=None) -> int:
        return _lib.qft_check_status(self._h, _ptr(workspace), _stream_handle(stream))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            _lib.qft_plan_destroy(h)
            self._h = _vp()


class RealPlan:
    """Real-input transform of N = 2^n real samples: FORWARD = R2C (numpy.fft.rfft
    with SCALE_UNNORM), INVERSE = C2R (numpy.fft.irfft with SCALE_INV_N).
    dtype "c64" works on float32 data, "c128" on float64 data."""

    def __init__(self, n: int, direction: int = FORWARD, dtype="c64", tuned: bool = True, **opts):
        """tuned: the inner (n-1)-qubit plan takes the autotuner's shape for its size
        (explicit opts win)."""
        self._h = _vp()
        self.n, self.direction = int(n), int(direction)
        self.dtype = _dtype_code(dtype)
        if tuned and not opts.get("precision", 0):
            from .autotune import best_opts

            for key, v in best_opts(self.n - 1, "c64" if self.dtype == C64 else "c128").items():
                if key != "paired":
                    opts.setdefault(key, v)
        o = Opts(0, opts.get("tile_bits", 0), opts.get("coalesce_bits", 0), opts.get("max_stage_bits", 0),
                 opts.get("wait_limit_ms", 0), 0, opts.get("threads", 0), opts.get("precision", 0), 0,
                 opts.get("pass_split", 0))
        _check(_lib.qft_rplan_create(ctypes.byref(self._h), self.n, self.direction, self.dtype, ctypes.byref(o)),
               "qft_rplan_create")

    def workspace_size(self) -> int:
        return int(_lib.qft_rplan_workspace_size(self._h))

    def alloc_workspace(self, device="cuda"):
        import torch

        return torch.empty(self.workspace_size(), dtype=torch.uint8, device=device)

    def execute(self, inp, out, workspace, scale_mode: int = SCALE_UNNORM, stream=None) -> None:
        _check(_lib.qft_rplan_execute(self._h, _ptr(inp), _ptr(out), _ptr(workspace), int(scale_mode),
                                      _stream_handle(stream)), "qft_rplan_execute")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            _lib.qft_rplan_destroy(h)
            self._h = _vp()


class Batch:
    """Many transforms (plans[i] on device tensors states[i]) in one call: wide groups plus one persistent launch."""

    def __init__(self, plans, states, scale_mode: int = SCALE_STATE, scale_out=None, device="cuda"):
        import torch

        n = len(plans)
        self.plans = list(plans)  # keep the plans alive
        self.states = list(states)
        parr = (_vp * n)(*[p.handle for p in plans])
        sarr = (_vp * n)(*[_ptr(s) for s in states])
        size = int(_lib.qft_batch_workspace_size(parr, n))
        if size == 0:
            raise QftError(ERR_BAD_ARG, "qft_batch_workspace_size")
        self.workspace = torch.empty(size, dtype=torch.uint8, device=device)
        self._h = _vp()
        _check(_lib.qft_batch_create(ctypes.byref(self._h), parr, sarr, n, self.workspace.data_ptr(), size,
                                     _ptr(scale_out) if scale_out is not None else None, int(scale_mode)),
               "qft_batch_create")

    def execute(self, stream=None) -> None:
        _check(_lib.qft_batch_execute(self._h, _stream_handle(stream)), "qft_batch_execute")

    def status(self, stream=None) -> int:
        return _lib.qft_batch_status(self._h, _stream_handle(stream))

    def info(self) -> BatchInfo:
        out = BatchInfo()
        _check(_lib.qft_batch_get_info(self._h, ctypes.byref(out)), "qft_batch_get_info")
        return out

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            _lib.qft_batch_destroy(h)
            self._h = _vp()


class Server:
    """Continuous-batching request loop (C++ worker thread inside the library)."""

    def __init__(self, hbm_budget_bytes: int, streams: int = 0, max_inflight: int = 0):
        self._h = _vp()
        _check(_lib.qft_server_create(ctypes.byref(self._h), int(hbm_budget_bytes), int(streams), int(max_inflight)),
               "qft_server_create")
        self._keep = {}

    def submit(self, x, out, n: int, k: int = -1, direction: int = FORWARD, dtype="c64", order: int = ORDER_NATURAL,
               scale_mode: int = SCALE_STATE) -> int:
        """Queue a transform of x into out (torch tensors or numpy arrays; keep them alive)."""
        def ptr_loc(t):
            if hasattr(t, "data_ptr"):
                return t.data_ptr(), 1 if t.is_cuda else 0
            return t.ctypes.data, 0
        ip, il = ptr_loc(x)
        op, ol = ptr_loc(out)
        scale = ctypes.c_double(0.0)
        req = Request(int(n), int(k), int(direction), _dtype_code(dtype), int(order), int(scale_mode), ip, il, op, ol,
                      ctypes.pointer(scale))
        t = ctypes.c_uint64()
        _check(_lib.qft_server_submit(self._h, ctypes.byref(req), ctypes.byref(t)), "qft_server_submit")
        self._keep[t.value] = (x, out, scale)
        return t.value

    def wait(self, ticket: int, timeout_ms: int = -1):
        """Returns (status, latency_ms, scale_in)."""
        lat = ctypes.c_double()
        rc = _lib.qft_server_wait(self._h, ctypes.c_uint64(ticket), int(timeout_ms), ctypes.byref(lat))
        keep = self._keep.pop(ticket, None)
        return rc, lat.value, keep[2].value if keep else None

    def cancel(self, ticket: int) -> int:
        """Withdraw a request not yet admitted (0); QFT_ERR_STATE if it already runs or ran."""
        return _lib.qft_server_cancel(self._h, ctypes.c_uint64(ticket))

    def set_batching(self, max_n: int) -> None:
        """Batch requests with n <= max_n (0: none; default 18)."""
        _check(_lib.qft_server_set_batching(self._h, int(max_n)), "qft_server_set_batching")

    def inject_alloc_failures(self, count: int) -> None:
        """Test hook: the next `count` device allocations of the server fail."""
        _check(_lib.qft_server_inject_alloc_failures(self._h, int(count)), "qft_server_inject_alloc_failures")

    def stats(self) -> ServerStats:
        st = ServerStats()
        _check(_lib.qft_server_get_stats(self._h, ctypes.byref(st)), "qft_server_get_stats")
        return st

    def reset_stats(self) -> None:
        _lib.qft_server_reset_stats(self._h)

    def close(self) -> None:
        if self._h.value:
            _lib.qft_server_destroy(self._h)
            self._h = _vp()

    def __del__(self):
        self.close()


_plan_cache: dict = {}


def fft(x, k: int | None = None, inverse: bool = False, norm: str = "backward", order: str = "natural"):
    """numpy.fft-style convenience on a CUDA complex tensor (length 2^n), out of place.

    norm="backward": forward unscaled, inverse 1/N (numpy's default);
    "ortho": 1/sqrt(N) both ways; "forward": forward 1/N, inverse unscaled;
    "state": the normalised simulator state psi' (Sec. 3 step 4).
    k: AQFT cutoff (None = exact).
    """
    import torch

    if not x.is_cuda:
        raise ValueError("fft expects a CUDA tensor")
    N = x.numel()
    n = N.bit_length() - 1
    if N < 2 or (1 << n) != N:
        raise QftError(ERR_SIZE, "fft")
    direction = INVERSE if inverse else FORWARD
    modes = {("backward", False): SCALE_UNNORM, ("backward", True): SCALE_INV_N,
             ("ortho", False): SCALE_UNITARY, ("ortho", True): SCALE_UNITARY,
             ("forward", False): SCALE_INV_N, ("forward", True): SCALE_UNNORM,
             ("state", False): SCALE_STATE, ("state", True): SCALE_STATE}
    mode = modes[(norm, bool(inverse))]
    ordc = ORDER_NATURAL if order == "natural" else ORDER_BITREV
    key = (n, -1 if k is None else int(k), direction, _dtype_code(x.dtype), ordc)
    p = _plan_cache.get(key)
    if p is None:
        p = _plan_cache[key] = Plan(n, key[1], direction, key[3], ordc, tuned=True)
    out = torch.empty_like(x)
    ws = p.alloc_workspace(x.device)
    p.execute_oop(x.contiguous(), out, ws, mode)
    return out


def fft2(x, inverse: bool = False, norm: str = "backward"):
    """numpy.fft.fft2 / ifft2 of a CUDA complex (2^a, 2^b) tensor: the QFT on the
    column-index qubits (each row) and then on the row-index qubits (each
    column), as two subset plans of the a + b qubit register."""
    import torch

    if not x.is_cuda or x.dim() != 2:
        raise ValueError("fft2 expects a 2-D CUDA tensor")
    R, C = x.shape
    a, b = R.bit_length() - 1, C.bit_length() - 1
    if R < 2 or C < 2 or (1 << a) != R or (1 << b) != C:
        raise QftError(ERR_SIZE, "fft2")
    direction = INVERSE if inverse else FORWARD
    mode = {("backward", False): SCALE_UNNORM, ("backward", True): SCALE_INV_N,
            ("ortho", False): SCALE_UNITARY, ("ortho", True): SCALE_UNITARY,
            ("forward", False): SCALE_INV_N, ("forward", True): SCALE_UNNORM}[(norm, bool(inverse))]
    dt = _dtype_code(x.dtype)
    rows = Plan(b, -1, direction, dt, n_addr=a + b, w0=0)
    cols = Plan(a, -1, direction, dt, n_addr=a + b, w0=b)
    out = torch.empty_like(x)
    ws = torch.empty(max(rows.workspace_size(), cols.workspace_size()), dtype=torch.uint8, device=x.device)
    rows.execute_oop(x.contiguous(), out, ws, mode)
    cols.execute(out, ws, mode)
    return out


def qpe(thetas, coefs, m: int, k: int = -1, dtype="c128", device="cuda"):
    """Quantum phase estimation of an operator given by its eigenphases (turns)
    and the input's overlaps with its eigenvectors: prepare the state after the
    controlled evolutions, run the Fourier readout of the m counting qubits
    (omega = e^{-2 pi i / 2^m}: FORWARD here, the textbook inverse QFT; AQFT
    cutoff k), and return the counting register's distribution P(x), x < 2^m,
    as a CUDA float64 tensor (it peaks at x ~ theta_j 2^m)."""
    import torch

    th = torch.as_tensor(thetas, dtype=torch.float64).reshape(-1).to(device)
    c = torch.as_tensor(coefs, dtype=torch.complex128).reshape(-1).to(device)
    d = th.numel()
    db = d.bit_length() - 1
    if d < 1 or (1 << db) != d or c.numel() != d:
        raise QftError(ERR_SIZE, "qpe")
    dt = _dtype_code(dtype)
    state = torch.empty(d << m, dtype=torch.complex64 if dt == C64 else torch.complex128, device=device)
    scratch = torch.empty(max(8, int(_lib.qft_qpe_workspace_size(m, db))), dtype=torch.uint8, device=device)
    _check(_lib.qft_qpe_prepare(state.data_ptr(), m, db, th.data_ptr(), c.data_ptr(), dt, scratch.data_ptr(),
                                _stream_handle(None)), "qft_qpe_prepare")
    p = Plan(m, k, FORWARD, dt, n_addr=m + db, w0=0)
    p.execute(state, p.alloc_workspace(device), SCALE_UNITARY)
    prob = torch.empty(1 << m, dtype=torch.float64, device=device)
    _check(_lib.qft_qpe_probabilities(state.data_ptr(), m, db, dt, prob.data_ptr(), _stream_handle(None)),
           "qft_qpe_probabilities")
    return prob


class MonteCarlo:
    """Monte Carlo estimates of single output bins (Sec. 6, sum over histories)
    of the range-k transform of one input x (a CUDA complex64 / complex128
    tensor of length 2^n): prepare once, then draw samples from caller-given
    uniforms and evaluate any bins (qft_mc_prepare / qft_mc_sample /
    qft_mc_bins)."""

    def __init__(self, x, pos=None, n: int | None = None):
        """x: the dense input (length 2^n), or with pos (CUDA int64 input
        indices < 2^n) and n the K nonzero amplitudes of a sparse input of an
        n-wire register (n <= 62)."""
        import torch

        if not x.is_cuda or x.dtype not in (torch.complex64, torch.complex128):
            raise ValueError("MonteCarlo expects a CUDA complex64 or complex128 tensor")
        self.dtype = C64 if x.dtype == torch.complex64 else C128
        self.x = x.contiguous()
        self.pos = None
        if pos is None:
            N = x.numel()
            n = N.bit_length() - 1
            if (1 << n) != N:
                raise QftError(ERR_SIZE, "MonteCarlo")
            self.n = n
            self.ws = torch.empty(int(_lib.qft_mc_workspace_size(n)), dtype=torch.uint8, device=x.device)
            _check(_lib.qft_mc_prepare(n, self.dtype, self.x.data_ptr(), self.ws.data_ptr(), _stream_handle(None)),
                   "qft_mc_prepare")
        else:
            self.pos = pos.to(torch.int64).contiguous()
            if n is None or self.pos.numel() != self.x.numel():
                raise QftError(ERR_BAD_ARG, "MonteCarlo")
            self.n = int(n)
            K = self.x.numel()
            self.ws = torch.empty(int(_lib.qft_mc_sparse_workspace_size(K)), dtype=torch.uint8, device=x.device)
            _check(_lib.qft_mc_prepare_sparse(K, self.dtype, self.x.data_ptr(), self.ws.data_ptr(),
                                              _stream_handle(None)), "qft_mc_prepare_sparse")

    def sample(self, u, stream=None):
        """Input indices (int64) and weights (complex128) for the uniforms u (CUDA float64)."""
        import torch

        u = u.contiguous()
        m = u.numel()
        idx = torch.empty(m, dtype=torch.int64, device=u.device)
        w = torch.empty(m, dtype=torch.complex128, device=u.device)
        if self.pos is None:
            rc = _lib.qft_mc_sample(self.n, self.dtype, self.x.data_ptr(), self.ws.data_ptr(), u.data_ptr(), m,
                                    idx.data_ptr(), w.data_ptr(), _stream_handle(stream))
        else:
            rc = _lib.qft_mc_sample_sparse(self.x.numel(), self.dtype, self.pos.data_ptr(), self.x.data_ptr(),
                                           self.ws.data_ptr(), u.data_ptr(), m, idx.data_ptr(), w.data_ptr(),
                                           _stream_handle(stream))
        _check(rc, "qft_mc_sample")
        return idx, w

    def bins(self, idx, w, ys, k: int = -1, direction: int = FORWARD, stream=None):
        """(mean complex128, power float64, standard error float64) per bin of ys."""
        import torch

        ys = torch.as_tensor(ys, dtype=torch.int64, device=idx.device).contiguous()
        out = torch.empty(4 * max(1, ys.numel()), dtype=torch.float64, device=idx.device)
        _check(_lib.qft_mc_bins(self.n, int(k), int(direction), idx.data_ptr(), w.data_ptr(), idx.numel(),
                                ys.data_ptr(), ys.numel(), self.ws.data_ptr(), out.data_ptr(), _stream_handle(stream)),
               "qft_mc_bins")
        o = out[:4 * ys.numel()].view(-1, 4)
        return torch.complex(o[:, 0], o[:, 1]), o[:, 2], o[:, 3]


_rplan_cache: dict = {}


def rfft(x, norm: str = "backward"):
    """numpy.fft.rfft on a CUDA float32 / float64 tensor of length 2^n (n >= 2)."""
    import torch

    if not x.is_cuda or x.dtype not in (torch.float32, torch.float64):
        raise ValueError("rfft expects a CUDA float32 or float64 tensor")
    N = x.numel()
    n = N.bit_length() - 1
    if N < 4 or (1 << n) != N:
        raise QftError(ERR_SIZE, "rfft")
    dt = C64 if x.dtype == torch.float32 else C128
    mode = {"backward": SCALE_UNNORM, "ortho": SCALE_UNITARY, "forward": SCALE_INV_N}[norm]
    key = (n, FORWARD, dt)
    p = _rplan_cache.get(key) or _rplan_cache.setdefault(key, RealPlan(n, FORWARD, dt))
    out = torch.empty(N // 2 + 1, dtype=torch.complex64 if dt == C64 else torch.complex128, device=x.device)
    p.execute(x.contiguous(), out, p.alloc_workspace(x.device), mode)
    return out


def irfft(X, n: int | None = None, norm: str = "backward"):
    """numpy.fft.irfft of a CUDA half spectrum X (N/2 + 1 complex values, N = 2^n)."""
    import torch

    if not X.is_cuda or X.dtype not in (torch.complex64, torch.complex128):
        raise ValueError("irfft expects a CUDA complex64 or complex128 tensor")
    N = 2 * (X.numel() - 1) if n is None else int(n)
    nb = N.bit_length() - 1
    if N < 4 or (1 << nb) != N or X.numel() != N // 2 + 1:
        raise QftError(ERR_SIZE, "irfft")
    dt = C64 if X.dtype == torch.complex64 else C128
    mode = {"backward": SCALE_INV_N, "ortho": SCALE_UNITARY, "forward": SCALE_UNNORM}[norm]
    key = (nb, INVERSE, dt)
    p = _rplan_cache.get(key) or _rplan_cache.setdefault(key, RealPlan(nb, INVERSE, dt))
    out = torch.empty(N, dtype=torch.float32 if dt == C64 else torch.float64, device=X.device)
    p.execute(X.contiguous(), out, p.alloc_workspace(X.device), mode)
    return out


__all__ = ["Plan", "RealPlan", "Batch", "Server", "PlanInfo", "QftError", "fft", "fft2", "rfft", "irfft", "qpe", "lib", "C64", "C128", "FORWARD", "INVERSE",
           "SCALE_STATE", "SCALE_UNITARY", "SCALE_UNNORM", "SCALE_INV_N", "ORDER_NATURAL", "ORDER_BITREV"]
