"""Python binding of liblsd (include/lsd.h): argument marshalling only.

Every decoding step runs in the library's CUDA kernels.  PyTorch provides the device
memory and the stream; numpy arrays are accepted for host-side inputs.  If the
compiled library is missing this module raises instead of falling back to anything.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib", "liblsd.so")

LSD_OK = 0
LSD_ERR_INVALID_ARG = -1
LSD_ERR_CUDA = -2
LSD_ERR_OOM = -3
LSD_ERR_ADMISSION = -4
LSD_ERR_TIMEOUT = -5
LSD_ERR_UNSUPPORTED = -6
SHOT_OK_BP = 1
SHOT_OK_LSD = 2
SHOT_UNSOLVABLE = 3

# Every entry point declared in include/lsd.h.
EXPORTS = ("lsd_create", "lsd_decode_batch", "lsd_decode_batch_host", "lsd_bp_batch",
           "lsd_postprocess_batch", "lsd_get_stats", "lsd_get_priors", "lsd_workspace_bytes",
           "lsd_kernel_launches", "lsd_destroy", "lsd_status_string",
           "lsd_decode_batch_static", "lsd_prior_num_params", "lsd_prior_create",
           "lsd_prior_set_params", "lsd_prior_get_params", "lsd_prior_forward",
           "lsd_prior_gradient", "lsd_prior_train_step", "lsd_decode_learned",
           "lsd_prior_destroy", "lsd_sample", "lsd_server_create", "lsd_server_submit",
           "lsd_server_wait_all", "lsd_server_get_report", "lsd_server_run_poisson",
           "lsd_server_destroy", "lsd_autotune", "lsd_last_error", "lsd_window_create",
           "lsd_window_decode", "lsd_window_kernel_launches", "lsd_window_destroy",
           "lsd_window_stream_reset", "lsd_window_stream_push", "lsd_giant_create",
           "lsd_giant_decode", "lsd_giant_postprocess", "lsd_giant_kernel_launches",
           "lsd_giant_destroy", "lsd_giant_test_hold_barrier", "lsd_bp_variant_name",
           "lsd_server_create_with_windows", "lsd_server_submit_round",
           "lsd_server_get_code_report", "lsd_prior_set_kernel", "lsd_prior_get_kernel",
           "lsd_decode_batch_packed", "lsd_decode_batch_host_packed")


class LsdError(RuntimeError):
    def __init__(self, code: int, what: str):
        detail = ""
        if code in (LSD_ERR_CUDA, LSD_ERR_OOM):
            detail = lib().lsd_last_error().decode()
            detail = f" [{detail}]" if detail else ""
        super().__init__(f"{what}: {status_string(code)} ({code}){detail}")
        self.code = code


class Options(C.Structure):
    _fields_ = [("ms_scaling", C.c_float), ("bp_method", C.c_int32),
                ("no_early_exit", C.c_int32), ("single_cluster", C.c_int32),
                ("bp_lanes", C.c_int32), ("lsd_warps", C.c_int32),
                ("bp_kernel", C.c_int32), ("lsd_kernel", C.c_int32),
                ("osd_method", C.c_int32), ("osd_cs_order", C.c_int32),
                ("reserved", C.c_int32),
                ("mem_budget", C.c_size_t),
                ("stream", C.c_void_p)]


class TuneReport(C.Structure):
    _fields_ = [("bp_variant", C.c_int32), ("bp_candidates", C.c_int32),
                ("lsd_warps", C.c_int32), ("lsd_candidates", C.c_int32),
                ("ms_bp_best", C.c_float), ("ms_bp_first", C.c_float),
                ("ms_lsd_best", C.c_float), ("ms_lsd_first", C.c_float)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Stats(C.Structure):
    _fields_ = [("shots", C.c_int64), ("bp_converged", C.c_int64), ("lsd_shots", C.c_int64),
                ("unsolvable", C.c_int64), ("bp_iterations", C.c_int64),
                ("lsd_steps", C.c_int64), ("kappa_max", C.c_int32), ("nu_max", C.c_int32),
                ("ms_bp", C.c_float), ("ms_lsd", C.c_float), ("lsd_spilled", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


class GiantInfo(C.Structure):
    _fields_ = [("status", C.c_int32), ("bp_iterations", C.c_int32), ("nu", C.c_int32),
                ("kappa", C.c_int32), ("steps", C.c_int32), ("reserved", C.c_int32),
                ("arena_bytes_used", C.c_int64), ("ms_bp", C.c_float), ("ms_lsd", C.c_float)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


def lib():
    """Load liblsd.so (built in-tree by ``paper_2406_18655_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is not built; run __graft_entry__.build() first")
    L = C.CDLL(LIB_PATH)
    P = C.c_void_p
    L.lsd_create.argtypes = [C.POINTER(P), C.c_int32, C.c_int32, C.c_int64, P, P, P, C.c_int32,
                             C.c_int32, C.POINTER(Options)]
    L.lsd_decode_batch.argtypes = [P, C.c_int64, P, P, P, P, C.POINTER(Stats)]
    L.lsd_decode_batch_host.argtypes = [P, C.c_int64, P, P, P, C.POINTER(Stats)]
    L.lsd_decode_batch_packed.argtypes = [P, C.c_int64, P, P, P, C.POINTER(Stats)]
    L.lsd_decode_batch_host_packed.argtypes = [P, C.c_int64, P, P, P, C.POINTER(Stats)]
    L.lsd_bp_batch.argtypes = [P, C.c_int64, P, P, P, P]
    L.lsd_postprocess_batch.argtypes = [P, C.c_int64, P, P, P, P, P]
    L.lsd_get_stats.argtypes = [P, C.POINTER(Stats)]
    L.lsd_get_priors.argtypes = [P, P]
    L.lsd_workspace_bytes.argtypes = [P, C.POINTER(C.c_size_t)]
    L.lsd_kernel_launches.argtypes = [P, C.POINTER(C.c_int64)]
    L.lsd_destroy.argtypes = [P]
    L.lsd_decode_batch_static.argtypes = [P, C.c_int64, P, P, P]
    L.lsd_prior_num_params.argtypes = []
    L.lsd_prior_create.argtypes = [C.POINTER(P), P, C.c_int32, P]
    L.lsd_prior_set_params.argtypes = [P, P]
    L.lsd_prior_get_params.argtypes = [P, P]
    L.lsd_prior_forward.argtypes = [P, C.c_int64, P, P]
    L.lsd_prior_set_kernel.argtypes = [P, C.c_int32]
    L.lsd_prior_get_kernel.argtypes = [P, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]
    L.lsd_prior_gradient.argtypes = [P, C.c_int64, P, P, C.POINTER(C.c_double), P]
    L.lsd_prior_train_step.argtypes = [P, C.c_int64, P, P, C.c_float, C.POINTER(C.c_double)]
    L.lsd_decode_learned.argtypes = [P, P, C.c_int64, P, P, P, C.POINTER(Stats)]
    L.lsd_prior_destroy.argtypes = [P]
    L.lsd_sample.argtypes = [P, C.c_uint64, C.c_int64, C.c_int64, P, P]
    L.lsd_autotune.argtypes = [P, C.c_int64, P, C.POINTER(TuneReport)]
    L.lsd_window_create.argtypes = [C.POINTER(P), C.c_int32, C.c_int32, C.c_int64, P, P, P, P,
                                     C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_int32,
                                     C.POINTER(Options)]
    L.lsd_window_decode.argtypes = [P, C.c_int64, P, P, P, C.POINTER(Stats)]
    L.lsd_window_kernel_launches.argtypes = [P, C.POINTER(C.c_int64)]
    L.lsd_window_destroy.argtypes = [P]
    L.lsd_giant_create.argtypes = [C.POINTER(P), C.c_int32, C.c_int32, C.c_int64, P, P, P,
                                    C.c_int32, C.c_int32, C.c_size_t, C.POINTER(Options)]
    L.lsd_giant_decode.argtypes = [P, P, P, P, C.POINTER(GiantInfo)]
    L.lsd_giant_postprocess.argtypes = [P, P, P, P, C.POINTER(GiantInfo)]
    L.lsd_giant_kernel_launches.argtypes = [P, C.POINTER(C.c_int64)]
    L.lsd_giant_destroy.argtypes = [P]
    L.lsd_giant_test_hold_barrier.argtypes = [P, C.c_int32, C.c_int64]
    L.lsd_window_stream_reset.argtypes = [P, C.c_int64]
    L.lsd_window_stream_push.argtypes = [P, P, P, P, C.POINTER(C.c_int32),
                                         C.POINTER(C.c_int32)]
    L.lsd_status_string.argtypes = [C.c_int]
    L.lsd_bp_variant_name.argtypes = [C.c_int32]
    for name in EXPORTS:
        getattr(L, name).restype = (C.c_char_p if name in ("lsd_status_string", "lsd_last_error",
                                                           "lsd_bp_variant_name")
                                    else C.c_int)
    _lib = L
    return L


def status_string(code: int) -> str:
    return lib().lsd_status_string(int(code)).decode()


def pack_bits(rows) -> np.ndarray:
    """[k][L] 0/1 bytes -> [k][ceil(L/32)] uint32: element i is bit i & 31 of word i >> 5."""
    a = np.ascontiguousarray(np.asarray(rows, dtype=np.uint8))
    k, L = a.shape
    W = (L + 31) // 32
    pad = np.zeros((k, 32 * W), np.uint8)
    pad[:, :L] = a
    return np.ascontiguousarray(np.packbits(pad, axis=1, bitorder="little")).view("<u4")


def unpack_bits(words, L: int) -> np.ndarray:
    """Inverse of pack_bits: [k][W] uint32 -> [k][L] 0/1 bytes."""
    w = np.ascontiguousarray(np.asarray(words, dtype="<u4"))
    return np.unpackbits(w.view(np.uint8), axis=1, bitorder="little")[:, :L]


def bp_variant_name(variant: int) -> str:
    """Kernel and template shape of a BP variant id (``Decoder.autotune()['bp_variant']``)."""
    return lib().lsd_bp_variant_name(int(variant)).decode()


def _check(code: int, what: str):
    if code != LSD_OK:
        raise LsdError(code, what)


def _ptr(t):
    """Device pointer of a CUDA tensor (or None)."""
    if t is None:
        return None
    return C.c_void_p(t.data_ptr())


def _dev_tensor(t, dtype, shape, name):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype or tuple(t.shape) != tuple(shape) or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous {dtype} tensor of shape {tuple(shape)}")
    return t


class Decoder:
    """BP + LSD decoder of one check matrix (``lsd_create``).

    ``h`` is a dense 0/1 matrix (numpy or torch, m x n).  ``stream`` is a
    ``torch.cuda.Stream`` (default: the current stream at construction); all work of
    this decoder runs on it.  ``osd_cs = None`` reprocesses LSD-mu's clusters with OSD-E of
    order mu, ``osd_cs = w`` with the combination sweep OSD-CS-w (then lsd_order may exceed
    12: it only counts growth steps).
    """

    def __init__(self, h, channel_probs, bp_iters: int, lsd_order: int = 0, *,
                 ms_scaling: float = 0.0, bp_method: int = 0, no_early_exit: bool = False,
                 single_cluster: bool = False, bp_lanes: int = 0, lsd_warps: int = 0,
                 bp_kernel: int = 0, lsd_kernel: int = 0, mem_budget: int = 0, stream=None,
                 osd_cs: int | None = None):
        import torch
        h = np.asarray(h.cpu() if isinstance(h, torch.Tensor) else h, dtype=np.uint8)
        self.m, self.n = h.shape
        rows, cols = np.nonzero(h)
        rows = np.ascontiguousarray(rows, np.int32)
        cols = np.ascontiguousarray(cols, np.int32)
        p = np.asarray(channel_probs, dtype=np.float32)
        if p.ndim == 0:
            p = np.full(self.n, float(p), np.float32)
        p = np.ascontiguousarray(p)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        opt = Options()
        opt.ms_scaling = ms_scaling
        opt.bp_method = bp_method
        opt.no_early_exit = int(no_early_exit)
        opt.single_cluster = int(single_cluster)
        opt.bp_lanes = bp_lanes
        opt.lsd_warps = lsd_warps
        opt.bp_kernel = bp_kernel
        opt.lsd_kernel = lsd_kernel
        opt.osd_method = 0 if osd_cs is None else 1
        opt.osd_cs_order = 0 if osd_cs is None else osd_cs
        opt.mem_budget = mem_budget
        opt.stream = C.c_void_p(self.stream.cuda_stream)
        self._opt = opt
        handle = C.c_void_p()
        _check(lib().lsd_create(C.byref(handle), self.m, self.n, rows.size,
                                rows.ctypes.data_as(C.c_void_p), cols.ctypes.data_as(C.c_void_p),
                                p.ctypes.data_as(C.c_void_p), bp_iters, lsd_order, C.byref(opt)),
               "lsd_create")
        self._h = handle
        self.bp_iters = bp_iters
        self.lsd_order = lsd_order
        self.osd_cs = osd_cs

    # -- lifetime ---------------------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            lib().lsd_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- entry points -----------------------------------------------------------------
    def decode(self, syndromes, corrections=None, status=None, posteriors=None,
               want_stats: bool = False):
        """BP then LSD on device syndromes [shots][m] (uint8).  Returns (corrections, status[, stats])."""
        import torch
        shots = syndromes.shape[0]
        _dev_tensor(syndromes, torch.uint8, (shots, self.m), "syndromes")
        dev = syndromes.device
        if corrections is None:
            corrections = torch.empty((shots, self.n), dtype=torch.uint8, device=dev)
        if status is None:
            status = torch.empty(shots, dtype=torch.uint8, device=dev)
        _dev_tensor(corrections, torch.uint8, (shots, self.n), "corrections")
        _dev_tensor(status, torch.uint8, (shots,), "status")
        if posteriors is not None:
            _dev_tensor(posteriors, torch.float32, (shots, self.n), "posteriors")
        st = Stats() if want_stats else None
        _check(lib().lsd_decode_batch(self._h, shots, _ptr(syndromes), _ptr(corrections),
                                      _ptr(status), _ptr(posteriors),
                                      C.byref(st) if st is not None else None),
               "lsd_decode_batch")
        if want_stats:
            return corrections, status, st.as_dict()
        return corrections, status

    def decode_packed(self, syndromes, corrections=None, status=None, want_stats: bool = False):
        """BP then LSD on bit-packed device syndromes [shots][ceil(m/32)] (int32 tensor holding
        the uint32 words).  Returns (packed corrections [shots][ceil(n/32)], status[, stats])."""
        import torch
        shots = syndromes.shape[0]
        wm, wn = (self.m + 31) // 32, (self.n + 31) // 32
        _dev_tensor(syndromes, torch.int32, (shots, wm), "syndromes")
        dev = syndromes.device
        if corrections is None:
            corrections = torch.empty((shots, wn), dtype=torch.int32, device=dev)
        if status is None:
            status = torch.empty(shots, dtype=torch.uint8, device=dev)
        _dev_tensor(corrections, torch.int32, (shots, wn), "corrections")
        _dev_tensor(status, torch.uint8, (shots,), "status")
        st = Stats() if want_stats else None
        _check(lib().lsd_decode_batch_packed(self._h, shots, _ptr(syndromes), _ptr(corrections),
                                             _ptr(status), C.byref(st) if st is not None else None),
               "lsd_decode_batch_packed")
        if want_stats:
            return corrections, status, st.as_dict()
        return corrections, status

    def decode_host_packed(self, syndromes, corrections=None, status=None):
        """Host-buffer packed decode: syndromes [shots][ceil(m/32)] uint32 (numpy, or CPU int32
        tensors); returns (corrections [shots][ceil(n/32)], status)."""
        shots = syndromes.shape[0]
        wm, wn = (self.m + 31) // 32, (self.n + 31) // 32
        if corrections is None:
            corrections = np.empty((shots, wn), np.uint32)
        if status is None:
            status = np.empty(shots, np.uint8)

        def hp(a, shape, name):
            if hasattr(a, "data_ptr"):
                if a.is_cuda or not a.is_contiguous() or tuple(a.shape) != tuple(shape):
                    raise ValueError(f"{name} must be a contiguous CPU tensor of shape {shape}")
                return C.c_void_p(a.data_ptr())
            if a.dtype.itemsize != 4 and name != "status" or not a.flags.c_contiguous \
                    or a.shape != tuple(shape):
                raise ValueError(f"{name} must be a contiguous array of shape {shape}")
            return a.ctypes.data_as(C.c_void_p)

        _check(lib().lsd_decode_batch_host_packed(
            self._h, shots, hp(syndromes, (shots, wm), "syndromes"),
            hp(corrections, (shots, wn), "corrections"), hp(status, (shots,), "status"), None),
            "lsd_decode_batch_host_packed")
        return corrections, status

    def decode_host(self, syndromes, corrections=None, status=None, want_stats: bool = False):
        """Host-buffer entry point: syndromes and outputs in host memory (numpy or CPU tensors)."""
        s = syndromes
        shots = s.shape[0]
        if corrections is None:
            corrections = np.empty((shots, self.n), np.uint8)
        if status is None:
            status = np.empty(shots, np.uint8)

        def hp(a, shape, name):
            if hasattr(a, "data_ptr"):
                if a.is_cuda or not a.is_contiguous() or tuple(a.shape) != tuple(shape):
                    raise ValueError(f"{name} must be a contiguous CPU tensor of shape {shape}")
                return C.c_void_p(a.data_ptr())
            if a.dtype != np.uint8 or not a.flags.c_contiguous or a.shape != tuple(shape):
                raise ValueError(f"{name} must be a contiguous uint8 array of shape {shape}")
            return a.ctypes.data_as(C.c_void_p)

        st = Stats() if want_stats else None
        _check(lib().lsd_decode_batch_host(self._h, shots, hp(s, (shots, self.m), "syndromes"),
                                           hp(corrections, (shots, self.n), "corrections"),
                                           hp(status, (shots,), "status"),
                                           C.byref(st) if st is not None else None),
               "lsd_decode_batch_host")
        if want_stats:
            return corrections, status, st.as_dict()
        return corrections, status

    def bp(self, syndromes):
        """BP only.  Returns (posteriors [shots][n] f32, converged [shots] u8, iterations [shots] i32)."""
        import torch
        shots = syndromes.shape[0]
        _dev_tensor(syndromes, torch.uint8, (shots, self.m), "syndromes")
        dev = syndromes.device
        post = torch.empty((shots, self.n), dtype=torch.float32, device=dev)
        conv = torch.empty(shots, dtype=torch.uint8, device=dev)
        iters = torch.empty(shots, dtype=torch.int32, device=dev)
        _check(lib().lsd_bp_batch(self._h, shots, _ptr(syndromes), _ptr(post), _ptr(conv),
                                  _ptr(iters)), "lsd_bp_batch")
        return post, conv, iters

    def postprocess(self, llrs, syndromes):
        """LSD only on device soft information.  Returns (corrections, status, info[nu, kappa, steps])."""
        import torch
        shots = syndromes.shape[0]
        _dev_tensor(syndromes, torch.uint8, (shots, self.m), "syndromes")
        _dev_tensor(llrs, torch.float32, (shots, self.n), "llrs")
        dev = syndromes.device
        corr = torch.empty((shots, self.n), dtype=torch.uint8, device=dev)
        status = torch.empty(shots, dtype=torch.uint8, device=dev)
        info = torch.empty((shots, 3), dtype=torch.int32, device=dev)
        _check(lib().lsd_postprocess_batch(self._h, shots, _ptr(llrs), _ptr(syndromes),
                                           _ptr(corr), _ptr(status), _ptr(info)),
               "lsd_postprocess_batch")
        return corr, status, info

    def stats(self) -> dict:
        """Counters and kernel times of the last call (synchronizes the decoder's stream)."""
        st = Stats()
        _check(lib().lsd_get_stats(self._h, C.byref(st)), "lsd_get_stats")
        return st.as_dict()

    def sample(self, seed: int, shots: int, first_shot: int = 0):
        """Seeded i.i.d. pairs on the device: (errors [shots][n], syndromes [shots][m]) uint8."""
        import torch
        e = torch.empty((shots, self.n), dtype=torch.uint8, device="cuda")
        s = torch.empty((shots, self.m), dtype=torch.uint8, device="cuda")
        _check(lib().lsd_sample(self._h, seed & 0xFFFFFFFFFFFFFFFF, first_shot, shots, _ptr(e),
                                _ptr(s)), "lsd_sample")
        return e, s

    def autotune(self, syndromes) -> dict:
        """Times the launch variants on a sample batch (device syndromes) and keeps the fastest."""
        import torch
        shots = syndromes.shape[0]
        _dev_tensor(syndromes, torch.uint8, (shots, self.m), "syndromes")
        r = TuneReport()
        _check(lib().lsd_autotune(self._h, shots, _ptr(syndromes), C.byref(r)), "lsd_autotune")
        return r.as_dict()

    def decode_learned(self, prior, syndromes, want_stats: bool = False):
        """Learned prior + LSD (BP + LSD as the fallback).  Returns (corrections, status[, stats])."""
        import torch
        shots = syndromes.shape[0]
        _dev_tensor(syndromes, torch.uint8, (shots, self.m), "syndromes")
        corr = torch.empty((shots, self.n), dtype=torch.uint8, device=syndromes.device)
        status = torch.empty(shots, dtype=torch.uint8, device=syndromes.device)
        st = Stats()
        _check(lib().lsd_decode_learned(self._h, prior._h, shots, _ptr(syndromes), _ptr(corr),
                                        _ptr(status), C.byref(st)), "lsd_decode_learned")
        if want_stats:
            return corr, status, st.as_dict()
        return corr, status

    def priors(self):
        out = np.empty(self.n, np.float32)
        _check(lib().lsd_get_priors(self._h, out.ctypes.data_as(C.c_void_p)), "lsd_get_priors")
        return out

    def workspace_bytes(self) -> int:
        v = C.c_size_t()
        _check(lib().lsd_workspace_bytes(self._h, C.byref(v)), "lsd_workspace_bytes")
        return v.value

    def kernel_launches(self) -> int:
        v = C.c_int64()
        _check(lib().lsd_kernel_launches(self._h, C.byref(v)), "lsd_kernel_launches")
        return v.value


class WindowDecoder:
    """(w, c) overlapping-window decoder of d noisy syndrome rounds of ``h`` plus a noiseless
    one (``lsd_window_create``; Methods 4.3 uses w = 3, c = 1).  ``p_data`` (n) and
    ``q_meas`` (m) are the per-round fault probabilities; the remaining keywords are those
    of :class:`Decoder`, applied to every window."""

    def __init__(self, h, p_data, q_meas, rounds: int, window: int = 3, commit: int = 1,
                 bp_iters: int = 30, lsd_order: int = 0, *, osd_cs: int | None = None,
                 bp_kernel: int = 0, lsd_kernel: int = 0, stream=None):
        import torch
        h = np.asarray(h.cpu() if isinstance(h, torch.Tensor) else h, dtype=np.uint8)
        self.m, self.n = h.shape
        self.d = rounds
        rows, cols = np.nonzero(h)
        rows = np.ascontiguousarray(rows, np.int32)
        cols = np.ascontiguousarray(cols, np.int32)

        def probs(v, k):
            v = np.asarray(v, dtype=np.float32)
            return np.ascontiguousarray(np.full(k, float(v), np.float32) if v.ndim == 0 else v)
        p = probs(p_data, self.n)
        q = probs(q_meas, self.m)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        opt = Options()
        opt.bp_kernel = bp_kernel
        opt.lsd_kernel = lsd_kernel
        opt.osd_method = 0 if osd_cs is None else 1
        opt.osd_cs_order = 0 if osd_cs is None else osd_cs
        opt.stream = C.c_void_p(self.stream.cuda_stream)
        handle = C.c_void_p()
        _check(lib().lsd_window_create(C.byref(handle), self.m, self.n, rows.size,
                                       rows.ctypes.data_as(C.c_void_p),
                                       cols.ctypes.data_as(C.c_void_p),
                                       p.ctypes.data_as(C.c_void_p), q.ctypes.data_as(C.c_void_p),
                                       rounds, window, commit, bp_iters, lsd_order, C.byref(opt)),
               "lsd_window_create")
        self._h = handle

    @property
    def syndrome_len(self) -> int:
        return (self.d + 1) * self.m

    @property
    def fault_len(self) -> int:
        return self.d * (self.n + self.m)

    def close(self):
        if getattr(self, "_h", None):
            lib().lsd_window_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def decode(self, syndromes, corrections=None, status=None, want_stats: bool = False):
        """Device syndromes [shots][(d+1) m] -> (corrections [shots][d (n+m)], status[, stats])."""
        import torch
        shots = syndromes.shape[0]
        _dev_tensor(syndromes, torch.uint8, (shots, self.syndrome_len), "syndromes")
        dev = syndromes.device
        if corrections is None:
            corrections = torch.empty((shots, self.fault_len), dtype=torch.uint8, device=dev)
        if status is None:
            status = torch.empty(shots, dtype=torch.uint8, device=dev)
        _dev_tensor(corrections, torch.uint8, (shots, self.fault_len), "corrections")
        _dev_tensor(status, torch.uint8, (shots,), "status")
        st = Stats() if want_stats else None
        _check(lib().lsd_window_decode(self._h, shots, _ptr(syndromes), _ptr(corrections),
                                       _ptr(status), C.byref(st) if st is not None else None),
               "lsd_window_decode")
        if want_stats:
            return corrections, status, st.as_dict()
        return corrections, status

    def stream_reset(self, shots: int):
        """Start `shots` concurrent streams whose detector blocks arrive one push at a time."""
        _check(lib().lsd_window_stream_reset(self._h, shots), "lsd_window_stream_reset")
        self._stream_shots = shots

    def stream_push(self, block, corrections, status=None):
        """Next detector block [shots][m] of every stream; returns (first_round, count) of the
        rounds committed into `corrections` [shots][d (n+m)] (count 0: no window completed)."""
        import torch
        shots = self._stream_shots
        _dev_tensor(block, torch.uint8, (shots, self.m), "block")
        _dev_tensor(corrections, torch.uint8, (shots, self.fault_len), "corrections")
        if status is not None:
            _dev_tensor(status, torch.uint8, (shots,), "status")
        first, count = C.c_int32(), C.c_int32()
        _check(lib().lsd_window_stream_push(self._h, _ptr(block), _ptr(corrections),
                                            _ptr(status), C.byref(first), C.byref(count)),
               "lsd_window_stream_push")
        return first.value, count.value

    def kernel_launches(self) -> int:
        v = C.c_int64()
        _check(lib().lsd_window_kernel_launches(self._h, C.byref(v)),
               "lsd_window_kernel_launches")
        return v.value


class GiantDecoder:
    """One large shot on the whole GPU (``lsd_giant_create``): BP with a thread per check
    and per variable, then P-LSD (Alg. 2).  ``rows``, ``cols`` are the COO list of H (no
    dense matrix is needed); :meth:`from_dense` takes a 0/1 matrix."""

    def __init__(self, m: int, n: int, rows, cols, channel_probs, bp_iters: int,
                 lsd_order: int = 0, *, osd_cs: int | None = None, arena_bytes: int = 0,
                 ms_scaling: float = 0.0, stream=None):
        import torch
        self.m, self.n = int(m), int(n)
        rows = np.ascontiguousarray(rows, np.int32)
        cols = np.ascontiguousarray(cols, np.int32)
        p = np.asarray(channel_probs, dtype=np.float32)
        if p.ndim == 0:
            p = np.full(self.n, float(p), np.float32)
        p = np.ascontiguousarray(p)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        opt = Options()
        opt.ms_scaling = ms_scaling
        opt.osd_method = 0 if osd_cs is None else 1
        opt.osd_cs_order = 0 if osd_cs is None else osd_cs
        opt.stream = C.c_void_p(self.stream.cuda_stream)
        handle = C.c_void_p()
        _check(lib().lsd_giant_create(C.byref(handle), self.m, self.n, rows.size,
                                      rows.ctypes.data_as(C.c_void_p),
                                      cols.ctypes.data_as(C.c_void_p),
                                      p.ctypes.data_as(C.c_void_p), bp_iters, lsd_order,
                                      arena_bytes, C.byref(opt)),
               "lsd_giant_create")
        self._h = handle

    @classmethod
    def from_dense(cls, h, channel_probs, bp_iters: int, lsd_order: int = 0, **kw):
        h = np.asarray(h, dtype=np.uint8)
        r, c = np.nonzero(h)
        return cls(h.shape[0], h.shape[1], r, c, channel_probs, bp_iters, lsd_order, **kw)

    def close(self):
        if getattr(self, "_h", None):
            lib().lsd_giant_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def decode(self, syndrome, correction=None, posteriors=None):
        """Device syndrome [m] (uint8) -> (correction [n], info dict)."""
        import torch
        _dev_tensor(syndrome, torch.uint8, (self.m,), "syndrome")
        if correction is None:
            correction = torch.empty(self.n, dtype=torch.uint8, device=syndrome.device)
        _dev_tensor(correction, torch.uint8, (self.n,), "correction")
        if posteriors is not None:
            _dev_tensor(posteriors, torch.float32, (self.n,), "posteriors")
        info = GiantInfo()
        _check(lib().lsd_giant_decode(self._h, _ptr(syndrome), _ptr(correction),
                                      _ptr(posteriors), C.byref(info)), "lsd_giant_decode")
        return correction, info.as_dict()

    def postprocess(self, llr, syndrome, correction=None):
        """P-LSD on device soft information llr [n] (float32) -> (correction, info dict)."""
        import torch
        _dev_tensor(llr, torch.float32, (self.n,), "llr")
        _dev_tensor(syndrome, torch.uint8, (self.m,), "syndrome")
        if correction is None:
            correction = torch.empty(self.n, dtype=torch.uint8, device=syndrome.device)
        _dev_tensor(correction, torch.uint8, (self.n,), "correction")
        info = GiantInfo()
        _check(lib().lsd_giant_postprocess(self._h, _ptr(llr), _ptr(syndrome),
                                           _ptr(correction), C.byref(info)),
               "lsd_giant_postprocess")
        return correction, info.as_dict()

    def kernel_launches(self) -> int:
        v = C.c_int64()
        _check(lib().lsd_giant_kernel_launches(self._h, C.byref(v)), "lsd_giant_kernel_launches")
        return v.value

    def test_hold_barrier(self, hold: bool, limit_ns: int = 20_000_000):
        """Timeout-path test facility (lsd_giant_test_hold_barrier)."""
        _check(lib().lsd_giant_test_hold_barrier(self._h, int(hold), limit_ns),
               "lsd_giant_test_hold_barrier")


class Prior:
    """Learned edge-MLP prior of a decoder (lsd_prior_create)."""

    def __init__(self, decoder: Decoder, rounds: int = 4, params=None):
        self.decoder = decoder
        self.np = int(lib().lsd_prior_num_params())
        handle = C.c_void_p()
        buf = None
        if params is not None:
            buf = np.ascontiguousarray(params, dtype=np.float32)
            assert buf.size == self.np
        _check(lib().lsd_prior_create(C.byref(handle), decoder._h, rounds,
                                      None if buf is None else buf.ctypes.data_as(C.c_void_p)),
               "lsd_prior_create")
        self._h = handle
        self.rounds = rounds

    def close(self):
        if getattr(self, "_h", None):
            lib().lsd_prior_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get_params(self):
        out = np.empty(self.np, np.float32)
        _check(lib().lsd_prior_get_params(self._h, out.ctypes.data_as(C.c_void_p)),
               "lsd_prior_get_params")
        return out

    def set_params(self, params):
        buf = np.ascontiguousarray(params, dtype=np.float32)
        assert buf.size == self.np
        _check(lib().lsd_prior_set_params(self._h, buf.ctypes.data_as(C.c_void_p)),
               "lsd_prior_set_params")

    def set_kernel(self, kernel: str):
        """Inference kernel: "auto", "mma_sync" (per-node kernel) or "tcgen05"
        (tensor-memory kernel)."""
        code = {"auto": 0, "mma_sync": 1, "tcgen05": 2}[kernel]
        _check(lib().lsd_prior_set_kernel(self._h, code), "lsd_prior_set_kernel")

    def kernel(self) -> dict:
        """The inference kernel in use and its grid (CTAs)."""
        k, g = C.c_int32(), C.c_int32()
        _check(lib().lsd_prior_get_kernel(self._h, C.byref(k), C.byref(g)), "lsd_prior_get_kernel")
        return {"kernel": {1: "mma_sync", 2: "tcgen05"}[k.value], "grid": g.value}

    def forward(self, syndromes):
        import torch
        d = self.decoder
        shots = syndromes.shape[0]
        _dev_tensor(syndromes, torch.uint8, (shots, d.m), "syndromes")
        llr = torch.empty((shots, d.n), dtype=torch.float32, device=syndromes.device)
        _check(lib().lsd_prior_forward(self._h, shots, _ptr(syndromes), _ptr(llr)),
               "lsd_prior_forward")
        return llr

    def gradient(self, syndromes, errors):
        """(mean loss, gradient as a numpy float32 vector) of a batch; no update."""
        shots = syndromes.shape[0]
        loss = C.c_double()
        g = np.empty(self.np, np.float32)
        _check(lib().lsd_prior_gradient(self._h, shots, _ptr(syndromes), _ptr(errors),
                                        C.byref(loss), g.ctypes.data_as(C.c_void_p)),
               "lsd_prior_gradient")
        return loss.value, g

    def train_step(self, syndromes, errors, lr: float, want_loss: bool = False):
        shots = syndromes.shape[0]
        loss = C.c_double()
        _check(lib().lsd_prior_train_step(self._h, shots, _ptr(syndromes), _ptr(errors), lr,
                                          C.byref(loss) if want_loss else None),
               "lsd_prior_train_step")
        return loss.value if want_loss else None


class ServerCode(C.Structure):
    _fields_ = [("m", C.c_int32), ("n", C.c_int32), ("nnz", C.c_int64), ("rows", C.c_void_p),
                ("cols", C.c_void_p), ("channel_probs", C.c_void_p), ("bp_iters", C.c_int32),
                ("lsd_order", C.c_int32)]


class ServerWindowCode(C.Structure):
    _fields_ = [("m", C.c_int32), ("n", C.c_int32), ("nnz", C.c_int64), ("rows", C.c_void_p),
                ("cols", C.c_void_p), ("p_data", C.c_void_p), ("q_meas", C.c_void_p),
                ("rounds", C.c_int32), ("window", C.c_int32), ("commit", C.c_int32),
                ("bp_iters", C.c_int32), ("lsd_order", C.c_int32), ("streams", C.c_int32)]


class ServerOptions(C.Structure):
    _fields_ = [("slots_per_code", C.c_int32), ("max_batch", C.c_int32),
                ("max_wait_us", C.c_int32), ("use_graphs", C.c_int32), ("mem_budget", C.c_size_t)]


class ServerReport(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("completed", C.c_int64), ("batches", C.c_int64),
                ("admission_waits", C.c_int64), ("peak_inflight_bytes", C.c_int64),
                ("generated", C.c_int64), ("mean_batch", C.c_double), ("seconds", C.c_double),
                ("shots_per_s", C.c_double), ("p50_us", C.c_double), ("p99_us", C.c_double),
                ("mean_us", C.c_double), ("max_us", C.c_double), ("offered_rate", C.c_double),
                ("p99_lag_us", C.c_double), ("p99_queue_us", C.c_double),
                ("p99_service_us", C.c_double), ("p99_batch_gpu_us", C.c_double),
                ("p99_launch_call_us", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def _server_lib():
    L = lib()
    if not getattr(L, "_server_ready", False):
        P = C.c_void_p
        L.lsd_server_create.argtypes = [C.POINTER(P), C.c_int32, P, C.POINTER(ServerOptions)]
        L.lsd_server_submit.argtypes = [P, C.c_int32, P, P, P, C.POINTER(C.c_int64)]
        L.lsd_server_wait_all.argtypes = [P]
        L.lsd_server_get_report.argtypes = [P, C.POINTER(ServerReport), C.c_int32]
        L.lsd_server_run_poisson.argtypes = [P, C.c_double, C.c_double, P, P, P, C.c_uint64,
                                             C.POINTER(ServerReport)]
        L.lsd_server_destroy.argtypes = [P]
        L.lsd_server_create_with_windows.argtypes = [C.POINTER(P), C.c_int32, P, C.c_int32, P,
                                                     C.POINTER(ServerOptions)]
        L.lsd_server_submit_round.argtypes = [P, C.c_int32, C.c_int32, P, P, P,
                                              C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                              C.POINTER(C.c_int64)]
        L.lsd_server_get_code_report.argtypes = [P, C.c_int32, C.POINTER(ServerReport)]
        for name in ("lsd_server_create", "lsd_server_submit", "lsd_server_wait_all",
                     "lsd_server_get_report", "lsd_server_run_poisson", "lsd_server_destroy",
                     "lsd_server_create_with_windows", "lsd_server_submit_round",
                     "lsd_server_get_code_report"):
            getattr(L, name).restype = C.c_int
        L._server_ready = True
    return L


class Server:
    """Continuous-batching decode server over several codes (lsd_server_*).

    ``codes`` is a list of (h, channel_probs, bp_iters, lsd_order).  ``window_codes`` is a
    list of dicts (h, p, q, rounds, window, commit, bp_iters, lsd_order, streams): streams of
    syndrome rounds of h decoded in (window, commit) windows; their code ids follow the shot
    codes'.  Request buffers must be pinned host tensors (``pin_memory()``) or CUDA tensors;
    the blocks of ``submit_round`` may be any host tensors.
    """

    def __init__(self, codes, slots_per_code: int = 0, max_batch: int = 0, max_wait_us: int = 0,
                 mem_budget: int = 0, graphs: bool = True, window_codes=()):
        L = _server_lib()
        keep = []
        arr = (ServerCode * max(1, len(codes)))()
        self.shapes = []
        for k, (h, probs, iters, order) in enumerate(codes):
            h = np.asarray(h, dtype=np.uint8)
            r, c = np.nonzero(h)
            r = np.ascontiguousarray(r, np.int32)
            c = np.ascontiguousarray(c, np.int32)
            p = np.asarray(probs, np.float32)
            if p.ndim == 0:
                p = np.full(h.shape[1], float(p), np.float32)
            p = np.ascontiguousarray(p)
            keep += [r, c, p]
            arr[k] = ServerCode(h.shape[0], h.shape[1], r.size, r.ctypes.data, c.ctypes.data,
                                p.ctypes.data, iters, order)
            self.shapes.append(h.shape)
        warr = (ServerWindowCode * max(1, len(window_codes)))()
        self.window_shapes = []
        for k, wc in enumerate(window_codes):
            h = np.asarray(wc["h"], dtype=np.uint8)
            m, n = h.shape
            r, c = np.nonzero(h)
            r = np.ascontiguousarray(r, np.int32)
            c = np.ascontiguousarray(c, np.int32)
            pd = np.ascontiguousarray(np.broadcast_to(np.asarray(wc["p"], np.float32), (n,)))
            qm = np.ascontiguousarray(np.broadcast_to(np.asarray(wc["q"], np.float32), (m,)))
            keep += [r, c, pd, qm]
            warr[k] = ServerWindowCode(m, n, r.size, r.ctypes.data, c.ctypes.data, pd.ctypes.data,
                                       qm.ctypes.data, wc["rounds"], wc.get("window", 3),
                                       wc.get("commit", 1), wc.get("bp_iters", 30),
                                       wc.get("lsd_order", 0), wc["streams"])
            self.window_shapes.append((m, n, wc["rounds"]))
        opt = ServerOptions(slots_per_code, max_batch, max_wait_us, 0 if graphs else -1, mem_budget)
        handle = C.c_void_p()
        _check(L.lsd_server_create_with_windows(
            C.byref(handle), len(codes), C.cast(arr, C.c_void_p), len(window_codes),
            C.cast(warr, C.c_void_p), C.byref(opt)), "lsd_server_create_with_windows")
        self._h = handle

    def submit(self, code: int, syndrome, correction=None, status=None) -> int:
        """syndrome / correction / status: 1-D uint8 tensors (pinned host or CUDA)."""
        rid = C.c_int64()
        _check(_server_lib().lsd_server_submit(
            self._h, code, C.c_void_p(syndrome.data_ptr()),
            None if correction is None else C.c_void_p(correction.data_ptr()),
            None if status is None else C.c_void_p(status.data_ptr()), C.byref(rid)),
            "lsd_server_submit")
        return rid.value

    def submit_round(self, code: int, stream: int, block, correction=None, status=None):
        """Next detector block (1-D uint8 host tensor or array) of a stream of a window code.
        Returns (first_round, rounds) of the window it completes, or (-1, 0)."""
        first, rounds, rid = C.c_int32(), C.c_int32(), C.c_int64()
        ptr = block.data_ptr() if hasattr(block, "data_ptr") else block.ctypes.data
        _check(_server_lib().lsd_server_submit_round(
            self._h, code, stream, C.c_void_p(ptr),
            None if correction is None else C.c_void_p(correction.data_ptr()),
            None if status is None else C.c_void_p(status.data_ptr()), C.byref(first),
            C.byref(rounds), C.byref(rid)), "lsd_server_submit_round")
        return first.value, rounds.value

    def code_report(self, code: int) -> dict:
        r = ServerReport()
        _check(_server_lib().lsd_server_get_code_report(self._h, code, C.byref(r)),
               "lsd_server_get_code_report")
        return r.as_dict()

    def wait_all(self):
        _check(_server_lib().lsd_server_wait_all(self._h), "lsd_server_wait_all")

    def report(self, reset: bool = False) -> dict:
        r = ServerReport()
        _check(_server_lib().lsd_server_get_report(self._h, C.byref(r), int(reset)),
               "lsd_server_get_report")
        return r.as_dict()

    def run_poisson(self, rate: float, seconds: float, mix, pools, seed: int = 1) -> dict:
        """Poisson load test; pools[c] is a pinned uint8 tensor [k][m_c] of syndromes, or for
        a window code a host tensor [k][(d+1) m] of block sequences."""
        nc = len(self.shapes) + len(self.window_shapes)
        mixa = (C.c_double * nc)(*[float(x) for x in mix])
        ptrs = (C.c_void_p * nc)(*[C.c_void_p(t.data_ptr()) for t in pools])
        sizes = (C.c_int64 * nc)(*[int(t.shape[0]) for t in pools])
        r = ServerReport()
        _check(_server_lib().lsd_server_run_poisson(self._h, rate, seconds, mixa, ptrs, sizes,
                                                    seed, C.byref(r)), "lsd_server_run_poisson")
        return r.as_dict()

    def close(self):
        if getattr(self, "_h", None):
            _server_lib().lsd_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
