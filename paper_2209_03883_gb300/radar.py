"""Thin ctypes binding of libofdm_radar.so (include/ofdm_radar.h).

Argument marshalling only: every step of the receive chain runs in the CUDA
library.  Functions keep the C names; device buffers are torch CUDA tensors
passed by data_ptr(), the stream is torch's current stream unless given.
If the library is missing the import of this module raises -- there is no
fallback path.
"""
from __future__ import annotations

import ctypes
import os
import re

PKG = os.path.dirname(os.path.abspath(__file__))
# OFDM_RADAR_LIB may name another build of the same library (same ABI).
LIB_PATH = os.environ.get("OFDM_RADAR_LIB") or os.path.join(PKG, "libofdm_radar.so")
HEADER = os.path.join(os.path.dirname(PKG), "include", "ofdm_radar.h")

OFDM_OK = 0
ERRORS = {-1: "INVALID_ARG", -2: "UNSUPPORTED_SIZE", -3: "CUDA", -4: "TIMEOUT", -5: "NO_MEMORY"}
WINDOW_RECT, WINDOW_HANN, WINDOW_HAMMING = 0, 1, 2
DETECT_TOPK, DETECT_THRESHOLD, DETECT_CFAR = 0, 1, 2
PREC_FP32, PREC_SPLIT_BF16, PREC_SPLIT_FP16 = 0, 1, 2
STATUS_ZERO_X, STATUS_NONFINITE, STATUS_OVERFLOW, STATUS_FEW_PEAKS = 1, 2, 4, 8
STATUS_UNREFINED, STATUS_TIMEOUT = 32, 64


class Params(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int32), ("M", ctypes.c_int32),
                ("N_pad", ctypes.c_int32), ("M_pad", ctypes.c_int32),
                ("L_cp", ctypes.c_int32), ("n_cp", ctypes.c_int32),
                ("zc_root", ctypes.c_int32), ("zc_q", ctypes.c_int32),
                ("x_is_precoded", ctypes.c_int32), ("window", ctypes.c_int32),
                ("detect_mode", ctypes.c_int32), ("max_targets", ctypes.c_int32),
                ("max_frames", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("pfa", ctypes.c_float), ("noise_var", ctypes.c_float),
                ("fc_hz", ctypes.c_double), ("df_hz", ctypes.c_double),
                ("cfar_guard", ctypes.c_int32), ("cfar_train", ctypes.c_int32)]


class Target(ctypes.Structure):
    _fields_ = [("r", ctypes.c_int32), ("s", ctypes.c_int32), ("power", ctypes.c_float),
                ("range_m", ctypes.c_float), ("vel_mps", ctypes.c_float)]


TARGET_BYTES = ctypes.sizeof(Target)   # 20


class FrameDesc(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int32), ("M", ctypes.c_int32), ("L_cp", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("yx_offset", ctypes.c_int64), ("map_offset", ctypes.c_int64)]


BATCH_NO_GRAPH, BATCH_NO_TUNE = 1, 2


class FpsParams(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("offsets", ctypes.c_int32),
                ("max_recover", ctypes.c_int32), ("bin_pfa", ctypes.c_float),
                ("coherence_min", ctypes.c_float), ("dynamic_range", ctypes.c_float)]


class OfdmError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        msg = _lib.ofdm_radar_strerror(code).decode() if _lib else ERRORS.get(code, str(code))
        super().__init__(f"{where}: {ERRORS.get(code, code)} ({msg})")


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is not built; run __graft_entry__.build()")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i32 = ctypes.c_void_p, ctypes.c_int32
    P = ctypes.POINTER
    lib.ofdm_radar_default_params.argtypes = [P(Params)]
    lib.ofdm_radar_default_params.restype = None
    lib.ofdm_radar_plan_create.argtypes = [P(Params), P(vp)]
    lib.ofdm_radar_plan_destroy.argtypes = [vp]
    lib.ofdm_radar_plan_destroy.restype = None
    lib.ofdm_radar_workspace_intact.argtypes = []
    lib.ofdm_radar_support_rows.argtypes = [vp, vp]
    lib.ofdm_radar_process.argtypes = [vp, vp, vp, i32, vp, vp, vp, vp, vp]
    lib.ofdm_radar_process_host.argtypes = [vp, vp, vp, i32, vp, vp, vp, vp, vp]
    lib.ofdm_zc_precode.argtypes = [vp, vp, vp, i32, i32, vp]
    lib.ofdm_radar_range_profile.argtypes = [vp, vp, vp, i32, vp, vp]
    lib.ofdm_radar_doppler.argtypes = [vp, vp, i32, vp, vp]
    lib.ofdm_radar_detect.argtypes = [vp, vp, i32, vp, vp, vp, vp]
    lib.ofdm_radar_last_launch_count.argtypes = [vp]
    lib.ofdm_radar_timing_enable.argtypes = [vp, i32]
    lib.ofdm_radar_timing_read.argtypes = [vp, vp, vp, i32]
    lib.ofdm_radar_process_noalloc.argtypes = [P(Params), vp, vp, i32, vp, vp, vp, vp, vp]
    lib.ofdm_radar_process_noalloc.restype = ctypes.c_int
    lib.ofdm_fps_default_params.argtypes = [P(FpsParams)]
    lib.ofdm_fps_default_params.restype = None
    lib.ofdm_fps_sft.argtypes = [vp, vp, vp, i32, P(FpsParams), vp, vp, vp, vp]
    lib.ofdm_fps_sft.restype = ctypes.c_int
    lib.ofdm_tx_amplifier.argtypes = [vp, vp, i32, i32, ctypes.c_float, vp, vp, vp]
    lib.ofdm_tx_amplifier.restype = ctypes.c_int
    lib.ofdm_radar_batch_create.argtypes = [P(Params), vp, i32, ctypes.c_uint32, P(vp)]
    lib.ofdm_radar_batch_create.restype = ctypes.c_int
    lib.ofdm_radar_batch_process.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp]
    lib.ofdm_radar_batch_process.restype = ctypes.c_int
    lib.ofdm_radar_batch_groups.argtypes = [vp, vp]
    lib.ofdm_radar_batch_groups.restype = ctypes.c_int
    lib.ofdm_radar_batch_used_graph.argtypes = [vp]
    lib.ofdm_radar_batch_used_graph.restype = ctypes.c_int
    lib.ofdm_radar_batch_destroy.argtypes = [vp]
    lib.ofdm_radar_batch_destroy.restype = None
    f32 = ctypes.c_float
    lib.ofdm_radar_learned_prepare.argtypes = [vp]
    lib.ofdm_radar_coarse_shape.argtypes = [vp, vp, vp]
    lib.ofdm_radar_coarse_map.argtypes = [vp, vp, vp, i32, vp, vp]
    lib.ofdm_radar_process_learned.argtypes = [vp, vp, vp, vp, i32, f32, i32, vp, vp, vp, vp]
    lib.ofdm_cnn_param_count.argtypes = []
    lib.ofdm_cnn_forward.argtypes = [vp, i32, vp, i32, i32, i32, vp, vp, vp, vp]
    lib.ofdm_cnn_backward.argtypes = [vp, i32, vp, vp, vp, vp, i32, i32, i32, vp, vp, vp, vp]
    lib.ofdm_cnn_bce.argtypes = [vp, vp, i32, f32, vp, vp, vp]
    lib.ofdm_cnn_adam.argtypes = [vp, vp, vp, vp, i32, i32, f32, f32, f32, f32, vp]
    for name in ("ofdm_radar_learned_prepare", "ofdm_radar_coarse_shape", "ofdm_radar_coarse_map",
                 "ofdm_radar_process_learned", "ofdm_cnn_param_count", "ofdm_cnn_forward",
                 "ofdm_cnn_backward", "ofdm_cnn_bce", "ofdm_cnn_adam"):
        getattr(lib, name).restype = ctypes.c_int
    lib.ofdm_radar_strerror.argtypes = [ctypes.c_int]
    lib.ofdm_radar_strerror.restype = ctypes.c_char_p
    for name in ("ofdm_radar_plan_create", "ofdm_radar_support_rows", "ofdm_radar_process",
                 "ofdm_radar_process_host", "ofdm_zc_precode", "ofdm_radar_range_profile",
                 "ofdm_radar_doppler", "ofdm_radar_detect", "ofdm_radar_last_launch_count",
                 "ofdm_radar_timing_enable", "ofdm_radar_timing_read"):
        getattr(lib, name).restype = ctypes.c_int
    return lib


_lib = _load()


def lib():
    return _lib


def declared_functions(header: str = HEADER):
    """Names of the functions declared in the public header."""
    text = open(header).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ofdm_[a-z0-9_]+)\s*\(", text)))


def default_params(**kw) -> Params:
    p = Params()
    _lib.ofdm_radar_default_params(ctypes.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise AttributeError(k)
        setattr(p, k, v)
    return p


def _check(code, where):
    if code < 0:
        raise OfdmError(code, where)
    return code


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


_DTYPES = {"c64": ("complex64",), "f32": ("float32",), "i32": ("int32", "uint32"), "u8": ("uint8",)}


def _buf(t, kind, need, where, name, host=False):
    """Pointer of tensor `t` after checking it against what the C call reads
    or writes: dtype, contiguity, device (CUDA, or host memory for the *_host
    entry point) and at least `need` elements.  None passes as NULL."""
    if t is None:
        return None
    dt = str(t.dtype).replace("torch.", "")
    if dt not in _DTYPES[kind]:
        raise TypeError(f"{where}: {name} must be {_DTYPES[kind][0]}, got {dt}")
    if not t.is_contiguous():
        raise ValueError(f"{where}: {name} must be contiguous")
    if host == bool(t.is_cuda):
        raise ValueError(f"{where}: {name} must be a {'host' if host else 'CUDA'} tensor")
    if t.numel() < need:
        raise ValueError(f"{where}: {name} has {t.numel()} elements, the call needs {need}")
    return ctypes.c_void_p(t.data_ptr())


def _frames(frames, where, cap=None):
    """The frame count, rejected (as the library does, INVALID_ARG) outside
    [1, cap] before any buffer is looked at."""
    frames = int(frames)
    if frames < 1 or (cap is not None and frames > cap):
        raise OfdmError(-1, f"{where}: frames = {frames} outside [1, {cap}]")
    return frames


def _chain_ptrs(where, frames, N, M, Np, Mp, K, Y, X, out_map, out_targets, n_targets, status, host=False):
    g = frames * M * N
    return (_buf(Y, "c64", g, where, "Y", host), _buf(X, "c64", g, where, "X", host),
            _buf(out_map, "f32", frames * Np * Mp, where, "out_map", host),
            _buf(out_targets, "u8", frames * K * TARGET_BYTES, where, "out_targets", host),
            _buf(n_targets, "i32", frames, where, "n_targets", host),
            _buf(status, "i32", frames, where, "status", host))


def _stream(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(getattr(stream, "cuda_stream", stream))


class Plan:
    """Owns an ofdm_radar_plan (tables + workspace on the current device)."""

    def __init__(self, params: Params | None = None, **kw):
        self.params = params if params is not None else default_params(**kw)
        h = ctypes.c_void_p()
        _check(_lib.ofdm_radar_plan_create(ctypes.byref(self.params), ctypes.byref(h)),
               "ofdm_radar_plan_create")
        self._h = h
        p = self.params
        self.N, self.M = p.N, p.M
        self.Np, self.Mp = p.N_pad or p.N, p.M_pad or p.M
        self.max_targets, self.max_frames = p.max_targets, p.max_frames
        self.n_rows = _check(_lib.ofdm_radar_support_rows(self._h, None), "ofdm_radar_support_rows")

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            _lib.ofdm_radar_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def support_rows(self):
        n = _check(_lib.ofdm_radar_support_rows(self._h, None), "ofdm_radar_support_rows")
        arr = (ctypes.c_int32 * n)()
        _lib.ofdm_radar_support_rows(self._h, ctypes.cast(arr, ctypes.c_void_p))
        return list(arr)

    def last_launch_count(self):
        return _lib.ofdm_radar_last_launch_count(self._h)

    KERNEL_KINDS = ("column", "zero_rows", "doppler", "detect", "zct", "coarse", "cnn", "refine")

    def timing_enable(self, on=True):
        _check(_lib.ofdm_radar_timing_enable(self._h, int(bool(on))), "ofdm_radar_timing_enable")

    def timing_read(self):
        """{kind: (total_ms, launches)} of the launches recorded since the last read."""
        n = len(self.KERNEL_KINDS)
        ms = (ctypes.c_float * n)()
        cnt = (ctypes.c_int32 * n)()
        m = _check(_lib.ofdm_radar_timing_read(self._h, ctypes.cast(ms, ctypes.c_void_p),
                                                ctypes.cast(cnt, ctypes.c_void_p), n),
                   "ofdm_radar_timing_read")
        return {self.KERNEL_KINDS[k]: (float(ms[k]), int(cnt[k])) for k in range(m)}


def ofdm_radar_process(plan: Plan, Y, X, frames, out_map=None, out_targets=None, n_targets=None,
                       status=None, stream=None):
    w = "ofdm_radar_process"
    frames = _frames(frames, w, plan.max_frames)
    ptrs = _chain_ptrs(w, frames, plan.N, plan.M, plan.Np, plan.Mp, plan.max_targets, Y, X, out_map,
                       out_targets, n_targets, status)
    return _check(_lib.ofdm_radar_process(plan.handle, ptrs[0], ptrs[1], frames, *ptrs[2:], _stream(stream)), w)


def ofdm_radar_process_host(plan: Plan, Y_host, X_host, frames, map_host=None, targets_host=None,
                            n_targets_host=None, status_host=None, stream=None):
    w = "ofdm_radar_process_host"
    frames = _frames(frames, w, plan.max_frames)
    ptrs = _chain_ptrs(w, frames, plan.N, plan.M, plan.Np, plan.Mp, plan.max_targets, Y_host, X_host, map_host,
                       targets_host, n_targets_host, status_host, host=True)
    return _check(_lib.ofdm_radar_process_host(plan.handle, ptrs[0], ptrs[1], frames, *ptrs[2:], _stream(stream)),
                  w)


def ofdm_radar_process_noalloc(params: Params, Y, X, frames, out_map=None, out_targets=None,
                               n_targets=None, status=None, stream=None):
    """The chain without any device allocation (no plan; fixed in-library scratch)."""
    w = "ofdm_radar_process_noalloc"
    frames = _frames(frames, w)
    # Requests beyond the library's fixed array are rejected by the library
    # before it reads anything; the buffers are checked for what it accepts.
    N, M, Mp = params.N, params.M, params.M_pad or params.M
    spread = 0 if params.window == WINDOW_RECT else 2
    rows = N if params.L_cp + spread >= N else params.L_cp + spread
    checked = frames if frames <= 4096 and frames * rows * max(M, Mp) <= (1 << 20) else 1
    ptrs = _chain_ptrs(w, checked, N, M, params.N_pad or N, Mp, params.max_targets, Y, X, out_map, out_targets,
                       n_targets, status)
    return _check(_lib.ofdm_radar_process_noalloc(ctypes.byref(params), ptrs[0], ptrs[1], frames, *ptrs[2:],
                                                  _stream(stream)), w)


def ofdm_zc_precode(plan: Plan, inp, out, frames, inverse=False, stream=None):
    w = "ofdm_zc_precode"
    frames = _frames(frames, w)
    g = frames * plan.M * plan.N
    return _check(_lib.ofdm_zc_precode(plan.handle, _buf(inp, "c64", g, w, "in"), _buf(out, "c64", g, w, "out"),
                                       frames, int(bool(inverse)), _stream(stream)), w)


def ofdm_radar_range_profile(plan: Plan, Y, X, frames, strip, stream=None):
    w = "ofdm_radar_range_profile"
    frames = _frames(frames, w, plan.max_frames)
    g = frames * plan.M * plan.N
    return _check(_lib.ofdm_radar_range_profile(plan.handle, _buf(Y, "c64", g, w, "Y"), _buf(X, "c64", g, w, "X"),
                                                frames, _buf(strip, "c64", frames * plan.n_rows * plan.M, w, "strip"),
                                                _stream(stream)), w)


def ofdm_radar_doppler(plan: Plan, strip, frames, out_map, stream=None):
    w = "ofdm_radar_doppler"
    frames = _frames(frames, w, plan.max_frames)
    return _check(_lib.ofdm_radar_doppler(plan.handle, _buf(strip, "c64", frames * plan.n_rows * plan.M, w, "strip"),
                                          frames, _buf(out_map, "f32", frames * plan.Np * plan.Mp, w, "out_map"),
                                          _stream(stream)), w)


def ofdm_radar_detect(plan: Plan, map_, frames, out_targets=None, n_targets=None, status=None,
                      stream=None):
    w = "ofdm_radar_detect"
    frames = _frames(frames, w, plan.max_frames)
    return _check(_lib.ofdm_radar_detect(plan.handle, _buf(map_, "f32", frames * plan.Np * plan.Mp, w, "map"), frames,
                                         _buf(out_targets, "u8", frames * plan.max_targets * TARGET_BYTES, w,
                                              "out_targets"),
                                         _buf(n_targets, "i32", frames, w, "n_targets"),
                                         _buf(status, "i32", frames, w, "status"), _stream(stream)), w)


def targets_view(raw, frames, max_targets):
    """Decode a uint8 tensor/array of [frames][max_targets] ofdm_target records
    into numpy arrays (r, s, power, range_m, vel_mps)."""
    import numpy as np
    dt = np.dtype([("r", "<i4"), ("s", "<i4"), ("power", "<f4"), ("range_m", "<f4"),
                   ("vel_mps", "<f4")])
    a = raw.cpu().numpy() if hasattr(raw, "cpu") else np.asarray(raw)
    return a.view(dt).reshape(frames, max_targets)


# ------------------------------------------------------------- torch helpers
def ofdm_radar_workspace_intact() -> bool:
    """True if no launch wrote past the end of any device buffer the library
    allocated on the current device (the 256-byte canaries behind every plan
    and batch buffer).  Waits for all work on the current device."""
    return _check(_lib.ofdm_radar_workspace_intact(), "ofdm_radar_workspace_intact") == 1


def alloc_outputs(plan: Plan, frames: int, device="cuda", with_map=True):
    import torch
    out = {
        "map": torch.empty((frames, plan.Np, plan.Mp), dtype=torch.float32, device=device)
        if with_map else None,
        "targets": torch.zeros((frames * plan.max_targets * TARGET_BYTES,), dtype=torch.uint8,
                               device=device),
        "n_targets": torch.zeros((frames,), dtype=torch.int32, device=device),
        "status": torch.zeros((frames,), dtype=torch.int32, device=device),
    }
    return out


def process(plan: Plan, Y, X, frames=None, with_map=True, stream=None):
    """Run the chain on complex64 CUDA tensors [frames, M, N]; returns the outputs dict."""
    frames = Y.shape[0] if frames is None else frames
    out = alloc_outputs(plan, frames, Y.device, with_map)
    ofdm_radar_process(plan, Y, X, frames, out["map"], out["targets"], out["n_targets"],
                       out["status"], stream)
    return out


def fps_default_params(**kw) -> FpsParams:
    fp = FpsParams()
    _lib.ofdm_fps_default_params(ctypes.byref(fp))
    for k, v in kw.items():
        setattr(fp, k, v)
    return fp


def ofdm_fps_sft(plan: Plan, Y, X, frames, fp: FpsParams, slices, out_targets=None, n_targets=None,
                 stream=None):
    """FPS-SFT; `slices` is a device int32 tensor [frames][iterations][2 + 2 * offsets]."""
    w = "ofdm_fps_sft"
    frames = _frames(frames, w, plan.max_frames)
    g = frames * plan.M * plan.N
    return _check(_lib.ofdm_fps_sft(plan.handle, _buf(Y, "c64", g, w, "Y"), _buf(X, "c64", g, w, "X"), frames,
                                    ctypes.byref(fp),
                                    _buf(slices, "i32", frames * fp.iterations * (2 + 2 * fp.offsets), w, "slices"),
                                    _buf(out_targets, "u8", frames * plan.max_targets * TARGET_BYTES, w,
                                         "out_targets"),
                                    _buf(n_targets, "i32", frames, w, "n_targets"), _stream(stream)), w)


class Batch:
    """Frames of uneven shape processed together (ofdm_radar_batch_*)."""

    def __init__(self, params: Params, descs, flags=0):
        arr = (FrameDesc * len(descs))()
        for i, d in enumerate(descs):
            arr[i] = FrameDesc(*d[:3], 0, d[3], d[4])
        self.nframes = len(descs)
        self.max_targets = params.max_targets
        self.yx_extent = max(int(d[3]) + int(d[0]) * int(d[1]) for d in descs)
        self.map_extent = max(int(d[4]) + int(d[0]) * int(d[1]) for d in descs)
        h = ctypes.c_void_p()
        _check(_lib.ofdm_radar_batch_create(ctypes.byref(params), ctypes.cast(arr, ctypes.c_void_p),
                                            len(descs), flags, ctypes.byref(h)), "ofdm_radar_batch_create")
        self._h = h

    def groups(self):
        n = _check(_lib.ofdm_radar_batch_groups(self._h, None), "ofdm_radar_batch_groups")
        arr = (ctypes.c_int32 * (5 * n))()
        _lib.ofdm_radar_batch_groups(self._h, ctypes.cast(arr, ctypes.c_void_p))
        return [tuple(arr[5 * i:5 * i + 5]) for i in range(n)]

    def used_graph(self):
        return bool(_lib.ofdm_radar_batch_used_graph(self._h))

    def process(self, Y, X, out_map, targets, n_targets, status, stream=None):
        w, n = "ofdm_radar_batch_process", self.nframes
        return _check(_lib.ofdm_radar_batch_process(self._h, _buf(Y, "c64", self.yx_extent, w, "Y"),
                                                    _buf(X, "c64", self.yx_extent, w, "X"),
                                                    _buf(out_map, "f32", self.map_extent, w, "out_map"),
                                                    _buf(targets, "u8", n * self.max_targets * TARGET_BYTES, w,
                                                         "targets"),
                                                    _buf(n_targets, "i32", n, w, "n_targets"),
                                                    _buf(status, "i32", n, w, "status"), _stream(stream)), w)

    def close(self):
        if getattr(self, "_h", None):
            _lib.ofdm_radar_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------- learned proposal
STATUS_FALLBACK = 16


def ofdm_radar_learned_prepare(plan: Plan):
    _check(_lib.ofdm_radar_learned_prepare(plan.handle), "ofdm_radar_learned_prepare")
    h, w = ctypes.c_int32(), ctypes.c_int32()
    _check(_lib.ofdm_radar_coarse_shape(plan.handle, ctypes.byref(h), ctypes.byref(w)),
           "ofdm_radar_coarse_shape")
    return h.value, w.value


def ofdm_radar_coarse_map(plan: Plan, Y, X, frames, x_out=None, stream=None):
    w = "ofdm_radar_coarse_map"
    frames = _frames(frames, w, plan.max_frames)
    g = frames * plan.M * plan.N
    h, wd = ctypes.c_int32(), ctypes.c_int32()
    _check(_lib.ofdm_radar_coarse_shape(plan.handle, ctypes.byref(h), ctypes.byref(wd)), "ofdm_radar_coarse_shape")
    return _check(_lib.ofdm_radar_coarse_map(plan.handle, _buf(Y, "c64", g, w, "Y"), _buf(X, "c64", g, w, "X"),
                                             frames, _buf(x_out, "f32", frames * h.value * wd.value, w, "x_out"),
                                             _stream(stream)), w)


def ofdm_radar_process_learned(plan: Plan, theta, Y, X, frames, logit_threshold, max_candidates,
                               out_targets=None, n_targets=None, status=None, stream=None):
    w = "ofdm_radar_process_learned"
    frames = _frames(frames, w, plan.max_frames)
    g = frames * plan.M * plan.N
    return _check(_lib.ofdm_radar_process_learned(plan.handle, _buf(theta, "f32", ofdm_cnn_param_count(), w, "theta"),
                                                  _buf(Y, "c64", g, w, "Y"), _buf(X, "c64", g, w, "X"), frames,
                                                  float(logit_threshold), int(max_candidates),
                                                  _buf(out_targets, "u8", frames * plan.max_targets * TARGET_BYTES,
                                                       w, "out_targets"),
                                                  _buf(n_targets, "i32", frames, w, "n_targets"),
                                                  _buf(status, "i32", frames, w, "status"), _stream(stream)), w)


def ofdm_cnn_param_count():
    return _lib.ofdm_cnn_param_count()


def ofdm_cnn_forward(theta, bf16, x, B, H, W, a1, a2, logits, stream=None):
    w, c, a = "ofdm_cnn_forward", B * H * W, 16 * B * H * W
    return _check(_lib.ofdm_cnn_forward(_buf(theta, "f32", ofdm_cnn_param_count(), w, "theta"), int(bf16),
                                        _buf(x, "f32", c, w, "x"), B, H, W, _buf(a1, "f32", a, w, "a1"),
                                        _buf(a2, "f32", a, w, "a2"), _buf(logits, "f32", c, w, "logits"),
                                        _stream(stream)), w)


def ofdm_cnn_backward(theta, bf16, x, a1, a2, glogits, B, H, W, ga1, ga2, gtheta, stream=None):
    w, c, a, n = "ofdm_cnn_backward", B * H * W, 16 * B * H * W, ofdm_cnn_param_count()
    return _check(_lib.ofdm_cnn_backward(_buf(theta, "f32", n, w, "theta"), int(bf16), _buf(x, "f32", c, w, "x"),
                                         _buf(a1, "f32", a, w, "a1"), _buf(a2, "f32", a, w, "a2"),
                                         _buf(glogits, "f32", c, w, "glogits"), B, H, W,
                                         _buf(ga1, "f32", a, w, "ga1"), _buf(ga2, "f32", a, w, "ga2"),
                                         _buf(gtheta, "f32", n, w, "gtheta"), _stream(stream)), w)


def ofdm_cnn_bce(logits, labels, n, pos_weight, loss, glogits, stream=None):
    w = "ofdm_cnn_bce"
    return _check(_lib.ofdm_cnn_bce(_buf(logits, "f32", n, w, "logits"), _buf(labels, "f32", n, w, "labels"), n,
                                    float(pos_weight), _buf(loss, "f32", 1, w, "loss"),
                                    _buf(glogits, "f32", n, w, "glogits"), _stream(stream)), w)


def ofdm_cnn_adam(theta, grad, m, v, n, step, lr, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    w = "ofdm_cnn_adam"
    return _check(_lib.ofdm_cnn_adam(_buf(theta, "f32", n, w, "theta"), _buf(grad, "f32", n, w, "grad"),
                                     _buf(m, "f32", n, w, "m"), _buf(v, "f32", n, w, "v"), n, step, float(lr),
                                     float(beta1), float(beta2), float(eps), _stream(stream)), w)


# ------------------------------------------------------------- transmit side
def ofdm_tx_amplifier(plan: Plan, S, frames, oversample=4, q=2.0, papr=None, aci=None, stream=None):
    """PAPR and amplifier out-of-band power of each OFDM symbol of the
    transmitted grid S ([frames][M][N] complex64): papr, aci [frames][M] float32."""
    w = "ofdm_tx_amplifier"
    frames = _frames(frames, w, plan.max_frames)
    n = frames * plan.M
    return _check(_lib.ofdm_tx_amplifier(plan.handle, _buf(S, "c64", n * plan.N, w, "S"), frames, int(oversample),
                                         float(q), _buf(papr, "f32", n, w, "papr"), _buf(aci, "f32", n, w, "aci"),
                                         _stream(stream)), w)
