"""GB300 (sm_103a) FFT-based continuous wavelet transform.

Thin ctypes binding of the C ABI in include/cwt.h (libcwt_gb300.so): the
functions below carry the ABI's names and only marshal arguments; every step
of the transform runs in the library's CUDA kernels.  torch tensors supply
device memory and streams.  There is no CPU fallback: if the library cannot be
built or loaded, the call raises.

Transform (Wang & He, RASTI 2023, arXiv:2302.03909, Sec. 3.1, Eqs. 8-10):
W[s, n] = sqrt(dx / w~_s) / M * sum_m F(m) psi_hat(2 pi m~ / (M w~_s)) e^{-2 pi i m n / M},
F(m) = sum_n f(n) e^{+2 pi i m n / M}; power spectrum Eq. 42.
"""
from __future__ import annotations

import ctypes
import threading

import numpy as np

from . import build as _build

__all__ = [
    "CwtError", "Plan", "cwt_plan_create", "cwt_plan_destroy", "cwt_plan_info", "cwt_exec",
    "cwt_exec_with_power", "cwt_wavelet_power", "cwt_env_power", "cwt_icwt", "cwt_exec_host",
    "cwt_scales_paper_grid",
    "cwt_status_string", "cwt_wavelet_power_noalloc", "cwt_plan_set_timing", "cwt_plan_get_timing", "load_library",
    "Batch", "cwt_batch_create", "cwt_batch_exec", "cwt_batch_info", "cwt_batch_destroy", "cwt_plan_get_opts",
    "cwt_plan_scratch_bytes", "cwt_exec_scratch", "ABI_FUNCTIONS", "KERNEL_CLASSES",
]

WAVELETS = {"gdw": 0, "mexhat": 0, "morlet": 1, "cbsw": 2, "cwgdw": 3}
BOUNDARIES = {"periodic": 0, "zero": 1}
SCALE_UNITS = {"dilation": 0, "w_tilde": 1}
INPUT_DTYPES = {"f32": 0, "f64": 1}
PRECISIONS = {"fp32": 0, "fp16": 1, "bf16": 2, "fp16x3": 3, "bf16x3": 4}

# every symbol include/cwt.h declares
ABI_FUNCTIONS = [
    "cwt_plan_opts_default", "cwt_plan_create", "cwt_plan_create_ex", "cwt_plan_destroy",
    "cwt_plan_info", "cwt_exec", "cwt_exec_with_power", "cwt_wavelet_power", "cwt_exec_host",
    "cwt_scales_paper_grid", "cwt_status_string", "cwt_plan_last_error", "cwt_plan_set_timing",
    "cwt_plan_get_timing", "cwt_wavelet_power_noalloc", "cwt_env_power", "cwt_icwt",
    "cwt_batch_create", "cwt_batch_exec", "cwt_batch_info", "cwt_batch_destroy", "cwt_plan_get_opts",
    "cwt_plan_scratch_bytes", "cwt_exec_scratch",
]
NOALLOC_MAX_PARTIALS = 65536
NOALLOC_CHUNK = 32768
KERNEL_CLASSES = {"forward": 0, "band": 1, "wide1": 2, "wide2": 3, "power": 4}


class _Opts(ctypes.Structure):
    _fields_ = [("omega0", ctypes.c_double), ("dx", ctypes.c_double),
                ("scale_unit", ctypes.c_int32), ("input_dtype", ctypes.c_int32),
                ("fft_len", ctypes.c_int64), ("eps_trunc", ctypes.c_double),
                ("min_ctas", ctypes.c_int32), ("tune", ctypes.c_int32),
                ("wide_batch_bytes", ctypes.c_int64), ("precision", ctypes.c_int32),
                ("band_depth", ctypes.c_int32), ("wide2_kernel", ctypes.c_int32),
                ("scratch", ctypes.c_int32)]

SCRATCH_MODES = {"plan": 0, "caller": 1}


class CwtError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{msg} (status {status})")
        self.status = status


_lock = threading.Lock()
_lib = None


def load_library(build_if_needed: bool = True) -> ctypes.CDLL:
    """Load libcwt_gb300.so (compiling it with nvcc first if it is stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.build() if build_if_needed else _build.LIB_PATH
        lib = ctypes.CDLL(path)
        vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
        pd = ctypes.POINTER(ctypes.c_double)
        lib.cwt_plan_opts_default.restype = None
        lib.cwt_plan_opts_default.argtypes = [ctypes.POINTER(_Opts)]
        lib.cwt_plan_create.restype = ctypes.c_int
        lib.cwt_plan_create.argtypes = [ctypes.POINTER(vp), i64, pd, i32, i32, i32]
        lib.cwt_plan_create_ex.restype = ctypes.c_int
        lib.cwt_plan_create_ex.argtypes = [ctypes.POINTER(vp), i64, pd, i32, i32, i32,
                                           ctypes.POINTER(_Opts)]
        lib.cwt_plan_destroy.restype = ctypes.c_int
        lib.cwt_plan_destroy.argtypes = [vp]
        lib.cwt_plan_info.restype = ctypes.c_int
        lib.cwt_plan_info.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(ctypes.c_size_t),
                                      ctypes.POINTER(i32)]
        lib.cwt_exec.restype = ctypes.c_int
        lib.cwt_exec.argtypes = [vp, vp, vp, vp]
        lib.cwt_exec_with_power.restype = ctypes.c_int
        lib.cwt_exec_with_power.argtypes = [vp, vp, vp, vp, vp]
        lib.cwt_wavelet_power.restype = ctypes.c_int
        lib.cwt_wavelet_power.argtypes = [vp, vp, vp, vp]
        lib.cwt_exec_host.restype = ctypes.c_int
        lib.cwt_exec_host.argtypes = [vp, vp, vp, vp, vp]
        lib.cwt_scales_paper_grid.restype = ctypes.c_int
        lib.cwt_scales_paper_grid.argtypes = [i64, i32, dbl, i32, pd, ctypes.POINTER(i32)]
        lib.cwt_status_string.restype = ctypes.c_char_p
        lib.cwt_status_string.argtypes = [ctypes.c_int]
        lib.cwt_plan_last_error.restype = ctypes.c_char_p
        lib.cwt_plan_last_error.argtypes = [vp]
        lib.cwt_plan_set_timing.restype = ctypes.c_int
        lib.cwt_plan_set_timing.argtypes = [vp, i32]
        lib.cwt_plan_get_timing.restype = ctypes.c_int
        lib.cwt_plan_get_timing.argtypes = [vp, i32, pd, ctypes.POINTER(i64), pd]
        lib.cwt_wavelet_power_noalloc.restype = ctypes.c_int
        lib.cwt_wavelet_power_noalloc.argtypes = [vp, i64, i32, i32, vp, vp]
        lib.cwt_env_power.restype = ctypes.c_int
        lib.cwt_env_power.argtypes = [vp, vp, vp, vp, vp, vp, vp]
        lib.cwt_icwt.restype = ctypes.c_int
        lib.cwt_icwt.argtypes = [vp, vp, vp, vp]
        pvp = ctypes.POINTER(vp)
        lib.cwt_batch_create.restype = ctypes.c_int
        lib.cwt_batch_create.argtypes = [ctypes.POINTER(vp), pvp, pvp, pvp, pvp, i32, i32]
        lib.cwt_batch_exec.restype = ctypes.c_int
        lib.cwt_batch_exec.argtypes = [vp, vp]
        lib.cwt_batch_info.restype = ctypes.c_int
        lib.cwt_batch_info.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i64),
                                       ctypes.POINTER(i64)]
        lib.cwt_batch_destroy.restype = ctypes.c_int
        lib.cwt_batch_destroy.argtypes = [vp]
        lib.cwt_plan_get_opts.restype = ctypes.c_int
        lib.cwt_plan_get_opts.argtypes = [vp, ctypes.POINTER(_Opts)]
        lib.cwt_plan_scratch_bytes.restype = ctypes.c_int
        lib.cwt_plan_scratch_bytes.argtypes = [vp, ctypes.POINTER(ctypes.c_size_t)]
        lib.cwt_exec_scratch.restype = ctypes.c_int
        lib.cwt_exec_scratch.argtypes = [vp, vp, vp, vp, vp, ctypes.c_size_t, vp]
        _lib = lib
        return lib


def cwt_status_string(status: int) -> str:
    return load_library().cwt_status_string(status).decode()


def _check(status: int, plan=None):
    if status != 0:
        msg = cwt_status_string(status)
        if plan is not None and plan._h:
            detail = load_library().cwt_plan_last_error(plan._h).decode()
            if detail:
                msg = f"{msg}: {detail}"
        raise CwtError(status, msg)


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


class Plan:
    """A cwt_plan handle plus the parameters it was made with."""

    def __init__(self, handle, N, n_scales, wavelet, boundary, opts):
        self._h = handle
        self.N = N
        self.n_scales = n_scales
        self.wavelet = wavelet
        self.boundary = boundary
        self.opts = opts
        M, ws, cplx = cwt_plan_info(self)
        self.M = M
        self.workspace_bytes = ws
        self.is_complex = bool(cplx)

    @property
    def out_shape(self):
        return (self.n_scales, self.N)

    def empty_output(self, device="cuda"):
        import torch
        dt = torch.complex64 if self.is_complex else torch.float32
        return torch.empty(self.out_shape, dtype=dt, device=device)

    def close(self):
        if self._h:
            cwt_plan_destroy(self)

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def cwt_plan_create(N: int, scales, wavelet: str = "gdw", boundary: str = "periodic", *,
                    omega0: float = 6.0, dx: float = 1.0, scale_unit: str = "dilation",
                    input_dtype: str = "f32", fft_len: int = 0, eps_trunc: float = 1e-10,
                    min_ctas: int = 0, tune: bool = False, wide_batch_bytes: int = 0,
                    precision: str = "fp32", band_depth: int = 0, wide2_kernel: int = 0,
                    scratch: str = "plan") -> Plan:
    lib = load_library()
    sc = np.ascontiguousarray(scales, dtype=np.float64)
    opts = _Opts()
    lib.cwt_plan_opts_default(ctypes.byref(opts))
    opts.omega0, opts.dx = float(omega0), float(dx)
    opts.scale_unit = SCALE_UNITS[scale_unit]
    opts.input_dtype = INPUT_DTYPES[input_dtype]
    opts.fft_len = int(fft_len)
    opts.eps_trunc = float(eps_trunc)
    opts.min_ctas = int(min_ctas)
    opts.tune = 1 if tune else 0
    opts.wide_batch_bytes = int(wide_batch_bytes)
    opts.precision = PRECISIONS[precision]
    opts.band_depth = int(band_depth)
    opts.wide2_kernel = int(wide2_kernel)
    opts.scratch = SCRATCH_MODES[scratch]
    h = ctypes.c_void_p()
    st = lib.cwt_plan_create_ex(ctypes.byref(h), int(N),
                                sc.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), len(sc),
                                WAVELETS[wavelet], BOUNDARIES[boundary], ctypes.byref(opts))
    _check(st)
    return Plan(h, int(N), len(sc), wavelet, boundary,
                dict(omega0=omega0, dx=dx, scale_unit=scale_unit, input_dtype=input_dtype,
                     fft_len=fft_len, eps_trunc=eps_trunc, precision=precision, scratch=scratch))


def cwt_plan_get_opts(plan: Plan) -> dict:
    """The options the plan was made with (launch shape as used, after tuning)."""
    o = _Opts()
    _check(load_library().cwt_plan_get_opts(plan._h, ctypes.byref(o)), plan)
    return {name: getattr(o, name) for name, _ in _Opts._fields_}


def cwt_plan_destroy(plan: Plan):
    if plan._h:
        h, plan._h = plan._h, None
        _check(load_library().cwt_plan_destroy(h))


def cwt_plan_info(plan: Plan):
    M = ctypes.c_int64()
    ws = ctypes.c_size_t()
    c = ctypes.c_int32()
    _check(load_library().cwt_plan_info(plan._h, ctypes.byref(M), ctypes.byref(ws), ctypes.byref(c)),
           plan)
    return M.value, ws.value, c.value


def _dev_ptr(t, name):
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def _check_signal(plan: Plan, signal):
    import torch
    want = torch.float64 if plan.opts["input_dtype"] == "f64" else torch.float32
    if signal.dtype != want or signal.numel() != plan.N:
        raise ValueError(f"signal must hold {plan.N} values of {want}")


def _check_W(plan: Plan, W):
    import torch
    want = torch.complex64 if plan.is_complex else torch.float32
    if W.dtype != want or tuple(W.shape) != plan.out_shape:
        raise ValueError(f"W must be {want} of shape {plan.out_shape}")


def cwt_exec(plan: Plan, signal, W=None, stream=None):
    """W (n_scales x N) of one device signal; allocates W if not given."""
    _check_signal(plan, signal)
    if W is None:
        W = plan.empty_output(signal.device)
    _check_W(plan, W)
    _check(load_library().cwt_exec(plan._h, _dev_ptr(signal, "signal"), _dev_ptr(W, "W"),
                                   _stream_ptr(stream)), plan)
    return W


def cwt_exec_with_power(plan: Plan, signal, W=None, spectrum=None, stream=None):
    import torch
    _check_signal(plan, signal)
    if W is None:
        W = plan.empty_output(signal.device)
    if spectrum is None:
        spectrum = torch.empty(plan.n_scales, dtype=torch.float64, device=signal.device)
    _check_W(plan, W)
    if spectrum.dtype != torch.float64 or spectrum.numel() != plan.n_scales:
        raise ValueError("spectrum must hold n_scales float64 values")
    _check(load_library().cwt_exec_with_power(plan._h, _dev_ptr(signal, "signal"), _dev_ptr(W, "W"),
                                              _dev_ptr(spectrum, "spectrum"), _stream_ptr(stream)),
           plan)
    return W, spectrum


def cwt_plan_scratch_bytes(plan: Plan) -> int:
    """Bytes of caller scratch a plan made with scratch="caller" needs per call (0 otherwise)."""
    n = ctypes.c_size_t()
    _check(load_library().cwt_plan_scratch_bytes(plan._h, ctypes.byref(n)), plan)
    return n.value


def cwt_exec_scratch(plan: Plan, signal, W, spectrum, scratch, stream=None):
    """cwt_exec_with_power for a plan made with scratch="caller": its per-call
    buffers are carved from ``scratch`` (a contiguous CUDA tensor of at least
    cwt_plan_scratch_bytes bytes, 256 B aligned).  spectrum may be None."""
    import torch
    _check_signal(plan, signal)
    _check_W(plan, W)
    if spectrum is not None and (spectrum.dtype != torch.float64 or spectrum.numel() != plan.n_scales):
        raise ValueError("spectrum must hold n_scales float64 values")
    nbytes = scratch.numel() * scratch.element_size()
    sp = _dev_ptr(spectrum, "spectrum") if spectrum is not None else None
    _check(load_library().cwt_exec_scratch(plan._h, _dev_ptr(signal, "signal"), _dev_ptr(W, "W"), sp,
                                           _dev_ptr(scratch, "scratch"), nbytes, _stream_ptr(stream)), plan)
    return W, spectrum


def cwt_wavelet_power(plan: Plan, W, spectrum=None, stream=None):
    import torch
    _check_W(plan, W)
    if spectrum is None:
        spectrum = torch.empty(plan.n_scales, dtype=torch.float64, device=W.device)
    _check(load_library().cwt_wavelet_power(plan._h, _dev_ptr(W, "W"), _dev_ptr(spectrum, "spectrum"),
                                            _stream_ptr(stream)), plan)
    return spectrum


def cwt_env_power(plan: Plan, W, delta, stream=None):
    """Eqs. 41 and 43: (p_pos, p_neg, frac) -- the power spectrum of W over the
    positions with delta > 0 and with delta < 0, and the two environments'
    fractions of the N positions.  delta: N values on the device, in the plan's
    input dtype."""
    import torch
    _check_W(plan, W)
    want = torch.float64 if plan.opts["input_dtype"] == "f64" else torch.float32
    if delta.dtype != want or delta.numel() != plan.N or not delta.is_contiguous():
        raise ValueError(f"delta must be {plan.N} contiguous {want} values")
    p_pos = torch.empty(plan.n_scales, dtype=torch.float64, device=W.device)
    p_neg = torch.empty_like(p_pos)
    frac = torch.empty(2, dtype=torch.float64, device=W.device)
    _check(load_library().cwt_env_power(plan._h, _dev_ptr(W, "W"), _dev_ptr(delta, "delta"),
                                        _dev_ptr(p_pos, "p_pos"), _dev_ptr(p_neg, "p_neg"),
                                        _dev_ptr(frac, "frac"), _stream_ptr(stream)), plan)
    return p_pos, p_neg, frac


def cwt_icwt(plan: Plan, W, out=None, stream=None):
    """Inverse CWT over the plan's scales (Eq. 6; Eq. 5 for the Morlet): the
    signal minus its mean, as N float32 values on the device."""
    import torch
    _check_W(plan, W)
    if out is None:
        out = torch.empty(plan.N, dtype=torch.float32, device=W.device)
    elif out.dtype != torch.float32 or out.numel() != plan.N or not out.is_contiguous():
        raise ValueError(f"out must be {plan.N} contiguous float32 values")
    _check(load_library().cwt_icwt(plan._h, _dev_ptr(W, "W"), _dev_ptr(out, "out"),
                                   _stream_ptr(stream)), plan)
    return out


def cwt_exec_host(plan: Plan, signal, W, spectrum=None, stream=None):
    """Host-buffer transform: signal and W (and spectrum) are host arrays or CPU tensors."""
    def hptr(a):
        if isinstance(a, np.ndarray):
            if not a.flags["C_CONTIGUOUS"]:
                raise ValueError("host arrays must be C-contiguous")
            return ctypes.c_void_p(a.ctypes.data)
        if a.is_cuda or not a.is_contiguous():
            raise ValueError("host tensors must be contiguous CPU tensors")
        return ctypes.c_void_p(a.data_ptr())
    sp = hptr(spectrum) if spectrum is not None else ctypes.c_void_p(0)
    _check(load_library().cwt_exec_host(plan._h, hptr(signal), hptr(W), sp, _stream_ptr(stream)),
           plan)
    return W, spectrum


def cwt_wavelet_power_noalloc(W, spectrum, stream=None):
    """Power spectrum of W (rows = scales) with no plan and no device allocation:
    the library keeps its partial sums in a fixed device array, so the caller
    must pre-allocate `spectrum` (n_scales float64) and serialise calls that
    could overlap on the GPU.  Rejects n_scales * ceil(N / 32768) > 65536."""
    import torch
    if W.dim() != 2 or W.dtype not in (torch.float32, torch.complex64):
        raise ValueError("W must be a 2-D float32 or complex64 CUDA tensor")
    S, N = W.shape
    if spectrum.dtype != torch.float64 or spectrum.numel() != S:
        raise ValueError("spectrum must hold n_scales float64 values")
    if W.device != spectrum.device:
        raise ValueError(f"W is on {W.device}, spectrum on {spectrum.device}: both must be on one device")
    with torch.cuda.device(W.device):
        st = load_library().cwt_wavelet_power_noalloc(_dev_ptr(W, "W"), N, S, int(W.dtype == torch.complex64),
                                                      _dev_ptr(spectrum, "spectrum"), _stream_ptr(stream))
    if st == 2:
        need = S * -(-N // NOALLOC_CHUNK)
        raise CwtError(st, f"{need} partial sums needed, the static scratch holds {NOALLOC_MAX_PARTIALS}")
    _check(st)
    return spectrum


def cwt_plan_set_timing(plan: Plan, enable=True):
    """Record a CUDA event pair around each kernel launch of the following calls.

    enable: False/0 off; True/1 events on each launch's own stream; 2 or
    "serial" also runs every launch on the call's stream, one after another, so
    that each event pair times one kernel alone."""
    mode = 2 if enable == "serial" else int(enable)
    _check(load_library().cwt_plan_set_timing(plan._h, mode), plan)


def cwt_plan_get_timing(plan: Plan) -> dict:
    """{class: (total_ms, launches, algorithmic_bytes)} since cwt_plan_set_timing."""
    lib = load_library()
    out = {}
    for name, c in KERNEL_CLASSES.items():
        ms, n, b = ctypes.c_double(), ctypes.c_int64(), ctypes.c_double()
        _check(lib.cwt_plan_get_timing(plan._h, c, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(b)),
               plan)
        out[name] = (ms.value, n.value, b.value)
    return out


def cwt_scales_paper_grid(N: int, wavelet: str = "gdw", omega0: float = 6.0,
                          n_subs: int = 4) -> np.ndarray:
    lib = load_library()
    n = ctypes.c_int32()
    _check(lib.cwt_scales_paper_grid(int(N), WAVELETS[wavelet], float(omega0), int(n_subs), None,
                                     ctypes.byref(n)))
    out = np.empty(n.value, dtype=np.float64)
    _check(lib.cwt_scales_paper_grid(int(N), WAVELETS[wavelet], float(omega0), int(n_subs),
                                     out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                     ctypes.byref(n)))
    return out


class Batch:
    """A cwt_batch handle.  Keeps the plans and tensors it was bound to alive."""

    def __init__(self, handle, keep):
        self._h = handle
        self._keep = keep

    def exec(self, stream=None):
        cwt_batch_exec(self, stream)

    def info(self) -> dict:
        return cwt_batch_info(self)

    def close(self):
        cwt_batch_destroy(self)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def cwt_batch_create(items, n_streams: int = 4) -> Batch:
    """One batch over items = [(plan, signal, W, spectrum or None), ...]: each
    plan bound to its own device tensors, as cwt_exec_with_power takes them."""
    n = len(items)
    if n < 1:
        raise ValueError("a batch needs at least one item")
    plans = (ctypes.c_void_p * n)()
    sigs = (ctypes.c_void_p * n)()
    Ws = (ctypes.c_void_p * n)()
    sps = (ctypes.c_void_p * n)()
    for i, (plan, signal, W, spectrum) in enumerate(items):
        _check_signal(plan, signal)
        _check_W(plan, W)
        plans[i] = plan._h
        sigs[i] = _dev_ptr(signal, "signal").value
        Ws[i] = _dev_ptr(W, "W").value
        if spectrum is not None:
            import torch
            if spectrum.dtype != torch.float64 or spectrum.numel() != plan.n_scales:
                raise ValueError(f"spectrum must hold {plan.n_scales} float64 values")
            sps[i] = _dev_ptr(spectrum, "spectrum").value
    h = ctypes.c_void_p()
    st = load_library().cwt_batch_create(ctypes.byref(h), plans, sigs, Ws, sps, n, int(n_streams))
    _check(st, items[0][0] if st not in (0,) else None)
    return Batch(h, list(items))


def cwt_batch_exec(batch: Batch, stream=None):
    if not batch._h:
        raise ValueError("batch is closed")
    _check(load_library().cwt_batch_exec(batch._h, _stream_ptr(stream)))


def cwt_batch_info(batch: Batch) -> dict:
    lv, nl = ctypes.c_int32(), ctypes.c_int32()
    ct, rec = ctypes.c_int64(), ctypes.c_int64()
    _check(load_library().cwt_batch_info(batch._h, ctypes.byref(lv), ctypes.byref(nl), ctypes.byref(ct),
                                         ctypes.byref(rec)))
    return {"levels": lv.value, "launches": nl.value, "ctas": ct.value, "plan_launches": rec.value}


def cwt_batch_destroy(batch: Batch):
    if batch._h:
        load_library().cwt_batch_destroy(batch._h)
        batch._h = None
        batch._keep = None
