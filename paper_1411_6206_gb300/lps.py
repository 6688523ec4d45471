"""Thin Python binding of liblps.so (include/lps_api.h): argument marshalling only.

Every function here has the name of the C entry point without the ``lps_`` prefix and
forwards to it; array arguments may be torch tensors (CUDA or CPU) or numpy arrays and are
passed as raw pointers (the library accepts host or device memory). Every step of the
reconstruction runs in the library's CUDA kernels; a missing library raises ImportError
and there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "liblps.so")

OK = 0
ERR_INVALID_ARG = -1
ERR_OOM = -2
ERR_CUDA = -3
ERR_TIMEOUT = -4
ERR_NONFINITE = -5
ERR_ADMISSION = -6
ERR_STATE = -7
ERR_UNSUPPORTED = -8

LAYOUT_SLICES, LAYOUT_FRAMES = 0, 1
COILS_FP32, COILS_FP16 = 0, 1
DATA_FP32, DATA_FP16 = 0, 1
EIG_FP32, EIG_FP64 = 0, 1
FP32, TF32_REFINE, BF16_REFINE = 0, 1, 2
KERNEL_CLASSES = 6
SUPPORT_THRESHOLD, SUPPORT_NONZERO = 0, 1
MAX_NC = 32
NOALLOC_SCRATCH_BYTES = 16 << 20


class Params(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("ncoil", C.c_int),
                ("layout", C.c_int), ("fft_z", C.c_int), ("wavelet_levels", C.c_int),
                ("max_iters", C.c_int),
                ("lambda_L_rel", C.c_double), ("lambda_S_rel", C.c_double),
                ("lambda_p", C.c_double), ("rank_tau", C.c_double), ("tol", C.c_double),
                ("precision", C.c_int), ("eig_precision", C.c_int), ("support_rule", C.c_int),
                ("recursive", C.c_int), ("coil_format", C.c_int), ("nx_total", C.c_int), ("x0", C.c_int),
                ("wavelet_dims", C.c_int), ("frame_slices", C.c_int), ("data_format", C.c_int),
                ("reserved", C.c_int * 2)]


class Stats(C.Structure):
    _fields_ = [("iters", C.c_int), ("rank", C.c_int), ("support_count", C.c_longlong),
                ("lambda_L", C.c_double), ("lambda_S", C.c_double), ("sigma_max", C.c_double),
                ("resid_norm2", C.c_double), ("nuclear", C.c_double),
                ("l1_off_support", C.c_double), ("objective", C.c_double),
                ("rel_change", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class IterRecord(C.Structure):
    _fields_ = [("resid_norm2", C.c_double), ("nuclear", C.c_double),
                ("l1_off_support", C.c_double), ("objective", C.c_double),
                ("rel_change", C.c_double), ("rank", C.c_int), ("eig_sweeps", C.c_int)]


class KernelTimes(C.Structure):
    _fields_ = [("launches", C.c_int * KERNEL_CLASSES), ("ms", C.c_double * KERNEL_CLASSES)]

    CLASSES = ("data_consistency", "sparse_step", "eig_svt", "init", "gram_tc", "reproj_tc")

    def as_dict(self):
        return {n: {"launches": self.launches[i], "ms": self.ms[i]} for i, n in enumerate(self.CLASSES)}


class TuneResult(C.Structure):
    _fields_ = [("dc_variant", C.c_int), ("radix_y", C.c_int * 8), ("radix_z", C.c_int * 8),
                ("lrs_tiles", C.c_int), ("candidates", C.c_int), ("cached", C.c_int),
                ("dc_us", C.c_double), ("lrs_us", C.c_double)]

    def as_dict(self):
        return {"dc_variant": self.dc_variant, "radix_y": [r for r in self.radix_y if r],
                "radix_z": [r for r in self.radix_z if r], "lrs_tiles": self.lrs_tiles,
                "candidates": self.candidates, "cached": self.cached,
                "dc_us": self.dc_us, "lrs_us": self.lrs_us}


class ServerConfig(C.Structure):
    _fields_ = [("hbm_budget_bytes", C.c_size_t), ("max_inflight", C.c_int), ("single_stream", C.c_int),
                ("autotune", C.c_int), ("reserved", C.c_int * 5)]


class LpsError(RuntimeError):
    def __init__(self, code: int, where: str, msg: str):
        super().__init__(f"{where}: {status_string(code)} ({code}): {msg}")
        self.code = code


_lib = None
_VP = C.c_void_p
_SIGS = {
    "lps_version": ([], C.c_int),
    "lps_last_error": ([], C.c_char_p),
    "lps_status_string": ([C.c_int], C.c_char_p),
    "lps_params_init": ([C.POINTER(Params)], C.c_int),
    "lps_support_words": ([C.POINTER(Params)], C.c_size_t),
    "lps_estimate_device_bytes": ([C.POINTER(Params), C.POINTER(C.c_size_t)], C.c_int),
    "lps_plan_create": ([C.POINTER(Params), _VP, C.POINTER(_VP)], C.c_int),
    "lps_plan_destroy": ([_VP], C.c_int),
    "lps_set_stream": ([_VP, _VP], C.c_int),
    "lps_plan_device_bytes": ([_VP, C.POINTER(C.c_size_t)], C.c_int),
    "lps_set_mask": ([_VP, _VP, C.POINTER(C.c_int)], C.c_int),
    "lps_set_coils": ([_VP, _VP], C.c_int),
    "lps_set_data": ([_VP, _VP, C.c_int], C.c_int),
    "lps_set_prior": ([_VP, _VP, _VP], C.c_int),
    "lps_clear_prior": ([_VP], C.c_int),
    "lps_iterate": ([_VP, C.c_int, C.POINTER(Stats)], C.c_int),
    "lps_reconstruct_frame": ([_VP, _VP, _VP, _VP, _VP, _VP, C.POINTER(Stats)], C.c_int),
    "lps_get_history": ([_VP, C.POINTER(IterRecord), C.c_int, C.POINTER(C.c_int)], C.c_int),
    "lps_get_state": ([_VP, _VP, _VP, _VP], C.c_int),
    "lps_get_support": ([_VP, _VP, _VP], C.c_int),
    "lps_set_state": ([_VP, _VP, _VP, _VP, C.c_double, C.c_double, C.c_int], C.c_int),
    "lps_forward": ([_VP, _VP, _VP], C.c_int),
    "lps_adjoint": ([_VP, _VP, _VP], C.c_int),
    "lps_casorati_gram": ([_VP, _VP, _VP, _VP], C.c_int),
    "lps_lowrank_reproject": ([_VP, _VP, _VP, _VP, _VP], C.c_int),
    "lps_data_consistency": ([_VP, _VP, _VP, C.POINTER(C.c_double)], C.c_int),
    "lps_test_stall_wait": ([_VP, C.c_int], C.c_int),
    "lps_batch_data_consistency": ([_VP, C.POINTER(_VP), C.POINTER(_VP), C.c_int, C.POINTER(C.c_float)], C.c_int),
    "lps_set_profiling": ([_VP, C.c_int], C.c_int),
    "lps_get_kernel_times": ([_VP, C.POINTER(KernelTimes)], C.c_int),
    "lps_shift_prior_columns": ([_VP, C.c_int], C.c_int),
    "lps_slab_reduction_size": ([_VP, C.POINTER(C.c_size_t), C.POINTER(C.c_size_t)], C.c_int),
    "lps_slab_begin": ([_VP, _VP], C.c_int),
    "lps_slab_iterate": ([_VP, _VP, C.c_int], C.c_int),
    "lps_slab_end": ([_VP, _VP, C.POINTER(Stats)], C.c_int),
    "lps_adjoint_noalloc": ([C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, _VP, _VP, _VP, C.c_int, _VP, _VP],
                            C.c_int),
    "lps_get_recon": ([_VP, _VP], C.c_int),
    "lps_autotune": ([_VP, _VP], C.c_int),
    "lps_autotune_clear_cache": ([], C.c_int),
    "lps_apply_tune": ([_VP, C.POINTER(TuneResult)], C.c_int),
    "lps_batch_create": ([C.POINTER(Params), C.c_int, _VP, C.POINTER(_VP)], C.c_int),
    "lps_batch_destroy": ([_VP], C.c_int),
    "lps_batch_size": ([_VP], C.c_int),
    "lps_batch_plan": ([_VP, C.c_int, C.POINTER(_VP)], C.c_int),
    "lps_batch_set_active": ([_VP, C.c_int, C.c_int], C.c_int),
    "lps_batch_autotune": ([_VP], C.c_int),
    "lps_batch_reconstruct": ([_VP], C.c_int),
    "lps_server_create": ([C.POINTER(ServerConfig), C.POINTER(_VP)], C.c_int),
    "lps_server_destroy": ([_VP], C.c_int),
    "lps_server_now": ([_VP], C.c_double),
    "lps_server_open": ([_VP, C.POINTER(Params), _VP, C.POINTER(C.c_int)], C.c_int),
    "lps_server_close": ([_VP, C.c_int], C.c_int),
    "lps_server_plan": ([_VP, C.c_int, C.POINTER(_VP)], C.c_int),
    "lps_server_bytes_in_use": ([_VP], C.c_size_t),
    "lps_server_submit": ([_VP, C.c_int, _VP, _VP, C.c_double, C.POINTER(C.c_longlong)], C.c_int),
    "lps_server_poll": ([_VP, C.c_longlong, C.POINTER(C.c_double), C.POINTER(C.c_double)], C.c_int),
    "lps_server_wait": ([_VP, C.c_longlong, C.POINTER(C.c_double), C.POINTER(C.c_double)], C.c_int),
    "lps_server_release": ([_VP, C.c_longlong], C.c_int),
    "lps_server_result": ([_VP, C.c_int, _VP], C.c_int),
    "lps_session_export": ([_VP, _VP, C.POINTER(C.c_size_t)], C.c_int),
    "lps_session_import": ([_VP, _VP, C.c_size_t], C.c_int),
}


def load(path: str = LIB_PATH):
    """Load liblps.so (built by paper_1411_6206_gb300.build) and declare its signatures."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with `python -m paper_1411_6206_gb300.build`")
    lib = C.CDLL(path)
    for name, (args, res) in _SIGS.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def exported_symbols():
    return list(_SIGS)


def status_string(code: int) -> str:
    return load().lps_status_string(code).decode()


def last_error() -> str:
    return load().lps_last_error().decode()


def _check(rc: int, where: str):
    if rc != OK:
        raise LpsError(rc, where, last_error())
    return rc


def ptr(a) -> Optional[int]:
    """Raw address of a contiguous torch tensor / numpy array (None passes NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    if isinstance(a, int):
        return a
    raise TypeError(f"unsupported array type {type(a)}")


def _stream(stream) -> Optional[int]:
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


# ---- entry points -------------------------------------------------------------------

def version() -> int:
    return load().lps_version()


def params_init(**kw) -> Params:
    p = Params()
    _check(load().lps_params_init(C.byref(p)), "params_init")
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def support_words(p: Params) -> int:
    return load().lps_support_words(C.byref(p))


def estimate_device_bytes(p: Params) -> int:
    b = C.c_size_t()
    _check(load().lps_estimate_device_bytes(C.byref(p), C.byref(b)), "estimate_device_bytes")
    return b.value


def plan_create(p: Params, stream=None) -> int:
    h = _VP()
    _check(load().lps_plan_create(C.byref(p), _stream(stream), C.byref(h)), "plan_create")
    return h.value


def plan_destroy(plan: int):
    _check(load().lps_plan_destroy(plan), "plan_destroy")


def set_stream(plan: int, stream):
    _check(load().lps_set_stream(plan, _stream(stream)), "set_stream")


def plan_device_bytes(plan: int) -> int:
    b = C.c_size_t()
    _check(load().lps_plan_device_bytes(plan, C.byref(b)), "plan_device_bytes")
    return b.value


def set_mask(plan: int, mask) -> int:
    n = C.c_int()
    _check(load().lps_set_mask(plan, ptr(mask), C.byref(n)), "set_mask")
    return n.value


def set_coils(plan: int, coils):
    _check(load().lps_set_coils(plan, ptr(coils)), "set_coils")


def set_data(plan: int, kdata, nlines: int):
    _check(load().lps_set_data(plan, ptr(kdata), nlines), "set_data")


def set_prior(plan: int, support=None, sigma=None):
    _check(load().lps_set_prior(plan, ptr(support), ptr(sigma)), "set_prior")


def clear_prior(plan: int):
    _check(load().lps_clear_prior(plan), "clear_prior")


def iterate(plan: int, n_iters: int) -> Stats:
    s = Stats()
    _check(load().lps_iterate(plan, n_iters, C.byref(s)), "iterate")
    return s


def reconstruct_frame(plan: int, recon=None, L=None, S=None, support=None, sigma=None,
                      stats: bool = True) -> Optional[Stats]:
    s = Stats() if stats else None
    _check(load().lps_reconstruct_frame(plan, ptr(recon), ptr(L), ptr(S), ptr(support), ptr(sigma),
                                        C.byref(s) if s is not None else None),
           "reconstruct_frame")
    return s


def get_history(plan: int, max_records: int = 4096):
    buf = (IterRecord * max_records)()
    n = C.c_int()
    _check(load().lps_get_history(plan, buf, max_records, C.byref(n)), "get_history")
    return [{k: getattr(buf[i], k) for k, _ in IterRecord._fields_}
            for i in range(n.value)]


def get_state(plan: int, X=None, L=None, S=None):
    _check(load().lps_get_state(plan, ptr(X), ptr(L), ptr(S)), "get_state")


def get_support(plan: int, support=None, sigma=None):
    _check(load().lps_get_support(plan, ptr(support), ptr(sigma)), "get_support")


def set_state(plan: int, X, S, L_prev, lambda_L: float, lambda_S: float, iters_done: int = 0):
    _check(load().lps_set_state(plan, ptr(X), ptr(S), ptr(L_prev), lambda_L, lambda_S, iters_done),
           "set_state")


def forward(plan: int, image, kdata):
    _check(load().lps_forward(plan, ptr(image), ptr(kdata)), "forward")


def adjoint(plan: int, kdata, image):
    _check(load().lps_adjoint(plan, ptr(kdata), ptr(image)), "adjoint")


def casorati_gram(plan: int, X, S, G):
    """G = (X - S)^H (X - S) over the Casorati columns (S may be None), plan precision."""
    _check(load().lps_casorati_gram(plan, ptr(X), ptr(S), ptr(G)), "casorati_gram")


def lowrank_reproject(plan: int, X, S, W, L):
    """L = (X - S) W over the Casorati columns (S may be None), plan precision."""
    _check(load().lps_lowrank_reproject(plan, ptr(X), ptr(S), ptr(W), ptr(L)), "lowrank_reproject")


def test_stall_wait(plan: int, polls: int):
    """Test hook: the next data_consistency call on the staged-coil kernel waits, once, on an
    mbarrier that nothing completes (polls polls) and returns LPS_ERR_TIMEOUT."""
    _check(load().lps_test_stall_wait(plan, polls), "test_stall_wait")


def data_consistency(plan: int, Z, X) -> float:
    r = C.c_double()
    _check(load().lps_data_consistency(plan, ptr(Z), ptr(X), C.byref(r)), "data_consistency")
    return r.value


def set_profiling(plan: int, on: bool):
    _check(load().lps_set_profiling(plan, int(bool(on))), "set_profiling")


def get_kernel_times(plan: int) -> KernelTimes:
    t = KernelTimes()
    _check(load().lps_get_kernel_times(plan, C.byref(t)), "get_kernel_times")
    return t


def adjoint_noalloc(nx: int, ny: int, nz: int, ncoil: int, mask, coils, kdata, nlines: int, image,
                    fft_z: int = 1, stream=None):
    """E^H without any device allocation (scratch in a fixed device array of the library);
    for callers that cannot allocate device memory at the point of use."""
    _check(load().lps_adjoint_noalloc(nx, ny, nz, ncoil, fft_z, ptr(mask), ptr(coils), ptr(kdata), nlines,
                                      ptr(image), _stream(stream)), "adjoint_noalloc")


def shift_prior_columns(plan: int, shift: int = 1):
    _check(load().lps_shift_prior_columns(plan, shift), "shift_prior_columns")


def slab_reduction_size(plan: int):
    """(sum_floats, max_floats) of the reduction record of an x-slab plan."""
    a, b = C.c_size_t(), C.c_size_t()
    _check(load().lps_slab_reduction_size(plan, C.byref(a), C.byref(b)), "slab_reduction_size")
    return a.value, b.value


def slab_begin(plan: int, rec):
    _check(load().lps_slab_begin(plan, ptr(rec)), "slab_begin")


def slab_iterate(plan: int, rec, k: int):
    _check(load().lps_slab_iterate(plan, ptr(rec), k), "slab_iterate")


def slab_end(plan: int, rec) -> "Stats":
    st = Stats()
    _check(load().lps_slab_end(plan, ptr(rec), C.byref(st)), "slab_end")
    return st


def get_recon(plan: int, out):
    _check(load().lps_get_recon(plan, ptr(out)), "get_recon")


def autotune(plan: int) -> TuneResult:
    r = TuneResult()
    _check(load().lps_autotune(plan, C.byref(r)), "autotune")
    return r


def apply_tune(plan: int, dc_variant: int, radix_y=(), radix_z=(), lrs_tiles: int = 1):
    t = TuneResult()
    t.dc_variant = dc_variant
    for i, r in enumerate(radix_y):
        t.radix_y[i] = r
    for i, r in enumerate(radix_z):
        t.radix_z[i] = r
    t.lrs_tiles = lrs_tiles
    _check(load().lps_apply_tune(plan, C.byref(t)), "apply_tune")


def autotune_clear_cache():
    _check(load().lps_autotune_clear_cache(), "autotune_clear_cache")


def session_export(plan: int) -> bytes:
    n = C.c_size_t()
    _check(load().lps_session_export(plan, None, C.byref(n)), "session_export")
    buf = C.create_string_buffer(n.value)
    _check(load().lps_session_export(plan, buf, C.byref(n)), "session_export")
    return buf.raw[: n.value]


def session_import(plan: int, blob: bytes):
    buf = C.create_string_buffer(blob, len(blob))
    _check(load().lps_session_import(plan, buf, len(blob)), "session_import")


class Plan:
    """Owning handle over lps_plan with the same calls as methods."""

    def __init__(self, nx, ny, nz, ncoil, stream=None, **kw):
        self.params = params_init(nx=nx, ny=ny, nz=nz, ncoil=ncoil, **kw)
        self.handle = plan_create(self.params, stream)
        self.nlines = 0

    @property
    def shape(self):
        return (self.params.nz, self.params.nx, self.params.ny)

    def close(self):
        if self.handle:
            plan_destroy(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_mask(self, mask):
        self.nlines = set_mask(self.handle, mask)
        return self.nlines

    def set_coils(self, coils):
        set_coils(self.handle, coils)

    def set_data(self, kdata):
        set_data(self.handle, kdata, self.nlines)

    def set_prior(self, support=None, sigma=None):
        set_prior(self.handle, support, sigma)

    def clear_prior(self):
        clear_prior(self.handle)

    def iterate(self, n):
        return iterate(self.handle, n)

    def reconstruct_frame(self, **kw):
        return reconstruct_frame(self.handle, **kw)

    def history(self):
        return get_history(self.handle)

    def support_words(self):
        return support_words(self.params)

    def autotune(self):
        return autotune(self.handle)

    def recon(self, out):
        get_recon(self.handle, out)
        return out


class _MemberPlan(Plan):
    """A plan owned by a batch: the same calls as Plan, never destroyed by Python."""

    def __init__(self, handle, params):
        self.params = params
        self.handle = handle
        self.nlines = 0

    def close(self):
        self.handle = None


class Batch:
    """Owning handle over lps_batch: independent problems reconstructed by one graph launch
    per frame step."""

    def __init__(self, params_list, stream=None):
        n = len(params_list)
        arr = (Params * n)(*params_list)
        h = _VP()
        _check(load().lps_batch_create(arr, n, _stream(stream), C.byref(h)), "batch_create")
        self.handle = h.value
        self.members = []
        for i, p in enumerate(params_list):
            ph = _VP()
            _check(load().lps_batch_plan(self.handle, i, C.byref(ph)), "batch_plan")
            self.members.append(_MemberPlan(ph.value, p))

    def __len__(self):
        return len(self.members)

    def __getitem__(self, i):
        return self.members[i]

    def set_active(self, i, active: bool):
        _check(load().lps_batch_set_active(self.handle, i, int(bool(active))), "batch_set_active")

    def autotune(self):
        _check(load().lps_batch_autotune(self.handle), "batch_autotune")

    def reconstruct(self):
        _check(load().lps_batch_reconstruct(self.handle), "batch_reconstruct")

    def data_consistency(self, Z, X, persistent: bool = False) -> float:
        """Step (4) alone on every active member (Z[i], X[i] device images, None for inactive
        members): each member's own kernel (graph branches) or one persistent launch over the
        batch's descriptor table. Returns the launch's device time in ms."""
        n = len(self.members)
        zs = (_VP * n)(*[ptr(z) if z is not None else None for z in Z])
        xs = (_VP * n)(*[ptr(x) if x is not None else None for x in X])
        ms = C.c_float()
        _check(load().lps_batch_data_consistency(self.handle, zs, xs, int(bool(persistent)), C.byref(ms)),
               "batch_data_consistency")
        return ms.value

    def close(self):
        if self.handle:
            for m in self.members:
                m.close()
            load().lps_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Owning handle over lps_server: admission by device-memory budget, per-session streams,
    frames issued as slots free up (max_inflight = 0: no limit); single_stream runs every frame
    in arrival order on one stream (the plain frame-by-frame path)."""

    def __init__(self, hbm_budget_bytes: int, max_inflight: int = 0, single_stream: bool = False,
                 autotune: bool = False):
        cfg = ServerConfig(hbm_budget_bytes=int(hbm_budget_bytes), max_inflight=int(max_inflight),
                           single_stream=int(bool(single_stream)), autotune=int(bool(autotune)))
        h = _VP()
        _check(load().lps_server_create(C.byref(cfg), C.byref(h)), "server_create")
        self.handle = h.value
        self._keep = {}

    def now(self) -> float:
        return load().lps_server_now(self.handle)

    def bytes_in_use(self) -> int:
        return load().lps_server_bytes_in_use(self.handle)

    def open(self, params: Params, coils) -> int:
        sid = C.c_int()
        _check(load().lps_server_open(self.handle, C.byref(params), ptr(coils), C.byref(sid)), "server_open")
        return sid.value

    def close_session(self, sid: int):
        _check(load().lps_server_close(self.handle, sid), "server_close")

    def submit(self, sid: int, mask, kdata, arrival: float) -> int:
        import numpy as np
        m = np.ascontiguousarray(mask, dtype=np.uint8)
        t = C.c_longlong()
        _check(load().lps_server_submit(self.handle, sid, m.ctypes.data, ptr(kdata), float(arrival), C.byref(t)),
               "server_submit")
        self._keep[t.value] = (m, kdata)       # alive until the frame is released
        return t.value

    def poll(self, ticket: int):
        lat, comp = C.c_double(), C.c_double()
        rc = load().lps_server_poll(self.handle, ticket, C.byref(lat), C.byref(comp))
        if rc < 0:
            _check(rc, "server_poll")
        return (lat.value, comp.value) if rc == 1 else None

    def wait(self, ticket: int):
        lat, comp = C.c_double(), C.c_double()
        _check(load().lps_server_wait(self.handle, ticket, C.byref(lat), C.byref(comp)), "server_wait")
        return lat.value, comp.value

    def release(self, ticket: int):
        _check(load().lps_server_release(self.handle, ticket), "server_release")
        self._keep.pop(ticket, None)

    def result(self, sid: int, out):
        _check(load().lps_server_result(self.handle, sid, ptr(out)), "server_result")
        return out

    def close(self):
        if self.handle:
            load().lps_server_destroy(self.handle)
            self.handle = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
