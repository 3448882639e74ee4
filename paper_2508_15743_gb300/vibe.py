"""ctypes binding of libvibe.so (include/vibe.h), with the C names, plus a small Decoder wrapper.

Argument marshalling only: every decoding step runs in the CUDA library. Device buffers are torch
tensors (their data pointers are passed through); the stream is torch's current CUDA stream unless
one is given. Importing this module loads the library and raises if it has not been built -- there
is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

VIBE_OK = 0
VIBE_ERR_INVALID = -1
VIBE_ERR_NOMEM = -2
VIBE_ERR_CUDA = -3
VIBE_ERR_UNSUPPORTED = -4
VIBE_NUM_COUNTERS = 8
CNT_SHOTS, CNT_FAILURES, CNT_LSD, CNT_PAIR_ITERS, CNT_UNSOLVABLE, CNT_BAD_PROBLEM, CNT_RESCANS = 0, 1, 2, 3, 4, 5, 6
CNT_LSD_WORDOPS = 7
VIBE_STATUS_OK, VIBE_STATUS_UNSOLVABLE, VIBE_STATUS_BAD_PROBLEM, VIBE_STATUS_CLUSTER_LIMIT = 0, 1, 2, 3

STATS_DTYPE = np.dtype([("status", "u1"), ("lsd_invoked", "u1"), ("n_converged", "u1"),
                        ("chosen_member", "u1"), ("iters", "<u2"), ("largest_cluster", "<u2"),
                        ("n_clusters", "<u4")])
assert STATS_DTYPE.itemsize == 12


class VibeError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"vibe error {code}: {msg}")
        self.code = code


class vibe_csr(ctypes.Structure):
    _fields_ = [("nrows", ctypes.c_int32), ("ncols", ctypes.c_int32),
                ("rowptr", ctypes.c_void_p), ("colidx", ctypes.c_void_p)]


class vibe_params(ctypes.Structure):
    _fields_ = [("max_iter", ctypes.c_int32), ("alpha", ctypes.c_float), ("M", ctypes.c_int32),
                ("lsd_order", ctypes.c_int32), ("msg_fp16", ctypes.c_int32), ("seed", ctypes.c_uint64),
                ("bp_engine", ctypes.c_int32), ("n_flood", ctypes.c_int32),
                ("member_alpha", ctypes.c_void_p), ("pair_mode", ctypes.c_int32), ("n_layered", ctypes.c_int32)]


ENGINE_AUTO, ENGINE_IMAGE, ENGINE_SUMMARY = 0, 1, 2


def _load():
    path = _build.LIB
    if not os.path.exists(path):
        raise ImportError(f"libvibe.so is not built ({path}); run paper_2508_15743_gb300.build.build_library()")
    lib = ctypes.CDLL(path)
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    lib.vibe_create.argtypes = [vp, vp, vp, i32, vp, vp, ctypes.POINTER(vp)]
    lib.vibe_create.restype = ctypes.c_int
    lib.vibe_decode.argtypes = [vp, vp, i64, vp, vp, vp, vp, vp, vp, vp]
    lib.vibe_decode.restype = ctypes.c_int
    lib.vibe_decode_host.argtypes = [vp, vp, i64, vp, vp, vp, vp, vp, vp]
    lib.vibe_decode_host.restype = ctypes.c_int
    lib.vibe_decode_noalloc.argtypes = [vp, vp, i64, vp, vp, vp, vp]
    lib.vibe_decode_noalloc.restype = ctypes.c_int
    lib.vibe_get_wavefronts.argtypes = [vp, i32, vp, vp, vp]
    lib.vibe_get_wavefronts.restype = ctypes.c_int
    lib.vibe_get_layers.argtypes = [vp, vp, vp]
    lib.vibe_get_layers.restype = ctypes.c_int
    lib.vibe_profile.argtypes = [vp, i32]
    lib.vibe_profile.restype = ctypes.c_int
    lib.vibe_profile_read.argtypes = [vp, vp, vp, vp, vp]
    lib.vibe_profile_read.restype = ctypes.c_int
    lib.vibe_autotune.argtypes = [vp, vp, i64, vp, vp, vp, vp, vp]
    lib.vibe_autotune.restype = ctypes.c_int
    lib.vibe_batch_create.argtypes = [vp, i32, ctypes.POINTER(vp)]
    lib.vibe_batch_create.restype = ctypes.c_int
    lib.vibe_batch_decode.argtypes = [vp, vp, vp, i32, i64, vp, i32, vp, i32, vp, vp, vp, vp]
    lib.vibe_batch_decode.restype = ctypes.c_int
    lib.vibe_batch_autotune.argtypes = [vp, vp, vp, i32, i64, vp]
    lib.vibe_batch_autotune.restype = ctypes.c_int
    lib.vibe_get_launch.argtypes = [vp, vp, vp]
    lib.vibe_get_launch.restype = ctypes.c_int
    lib.vibe_batch_destroy.argtypes = [vp]
    lib.vibe_batch_destroy.restype = ctypes.c_int
    lib.vibe_destroy.argtypes = [vp]
    lib.vibe_destroy.restype = ctypes.c_int
    lib.vibe_last_error.argtypes = []
    lib.vibe_last_error.restype = ctypes.c_char_p
    return lib


_lib = _load()
LIBRARY_PATH = _build.LIB


def vibe_last_error() -> str:
    return _lib.vibe_last_error().decode()


def _check(rc):
    if rc != VIBE_OK:
        raise VibeError(rc, vibe_last_error())


def _ptr(x):
    """Raw address of a torch tensor, a numpy array, an int, or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    return x.ctypes.data


def _stream_ptr(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# ---------------------------------------------------------------------------------------------
# The C entry points, same names, same argument order
# ---------------------------------------------------------------------------------------------

def vibe_create(H, L, priors, K, schedules, params):
    """H, L: objects with nrows/ncols/rowptr/colidx (int32 numpy); priors float64[n];
    schedules uint32 [K, n] or None; params: vibe_params. Returns an opaque handle (int)."""
    keep = []

    def csr(A):
        rp = np.ascontiguousarray(A.rowptr, dtype=np.int32)
        ci = np.ascontiguousarray(A.colidx, dtype=np.int32)
        keep.extend([rp, ci])
        return vibe_csr(A.nrows, A.ncols, rp.ctypes.data, ci.ctypes.data)

    Hc, Lc = csr(H), csr(L)
    pr = np.ascontiguousarray(priors, dtype=np.float64)
    sc = None if schedules is None else np.ascontiguousarray(schedules, dtype=np.uint32)
    out = ctypes.c_void_p()
    rc = _lib.vibe_create(ctypes.byref(Hc), ctypes.byref(Lc), pr.ctypes.data, int(K), _ptr(sc),
                          ctypes.byref(params), ctypes.byref(out))
    _check(rc)
    return out.value


def vibe_decode(h, d_syndromes, B, d_corrections, d_logical=None, d_stats=None, d_soft=None,
                d_observables=None, d_counters=None, stream=None):
    _check(_lib.vibe_decode(h, _ptr(d_syndromes), int(B), _ptr(d_corrections), _ptr(d_logical), _ptr(d_stats),
                            _ptr(d_soft), _ptr(d_observables), _ptr(d_counters), _stream_ptr(stream)))


def vibe_decode_host(h, h_syndromes, B, h_corrections, h_logical=None, h_stats=None, h_observables=None,
                     h_counters=None, stream=None):
    _check(_lib.vibe_decode_host(h, _ptr(h_syndromes), int(B), _ptr(h_corrections), _ptr(h_logical),
                                 _ptr(h_stats), _ptr(h_observables), _ptr(h_counters), _stream_ptr(stream)))


def vibe_decode_noalloc(h, d_syndromes, B, d_corrections, d_logical=None, d_stats=None, stream=None):
    """vibe_decode with the library's static device scratch instead of a per-handle workspace."""
    _check(_lib.vibe_decode_noalloc(h, _ptr(d_syndromes), int(B), _ptr(d_corrections), _ptr(d_logical),
                                    _ptr(d_stats), _stream_ptr(stream)))


def vibe_get_wavefronts(h, member, n):
    order = np.zeros(n, np.uint32)
    offs = np.zeros(n + 1, np.uint32)
    nl = ctypes.c_int32(0)
    _check(_lib.vibe_get_wavefronts(h, int(member), order.ctypes.data, offs.ctypes.data, ctypes.addressof(nl)))
    return order, offs[:nl.value + 1].copy(), nl.value


def vibe_get_layers(h, m):
    """(layer of each of the m checks as int32 [m], number of layers) of a handle with layered members."""
    layer = np.zeros(m, np.int32)
    nl = ctypes.c_int32(0)
    _check(_lib.vibe_get_layers(h, layer.ctypes.data, ctypes.addressof(nl)))
    return layer, nl.value


def vibe_profile(h, enable):
    _check(_lib.vibe_profile(h, int(bool(enable))))


def vibe_profile_read(h):
    bp, lsd = ctypes.c_double(0), ctypes.c_double(0)
    nb, nl = ctypes.c_int64(0), ctypes.c_int64(0)
    _check(_lib.vibe_profile_read(h, ctypes.addressof(bp), ctypes.addressof(lsd), ctypes.addressof(nb),
                                  ctypes.addressof(nl)))
    return dict(bp_ms=bp.value, lsd_ms=lsd.value, bp_launches=nb.value, lsd_launches=nl.value)


def vibe_autotune(h, d_syndromes, B, stream=None):
    """Returns the (engine, BP CTAs per SM, LSD CTAs per SM, LSD threads per CTA) the tuner kept."""
    eng, bp, lsd, nt = ctypes.c_int32(0), ctypes.c_int32(0), ctypes.c_int32(0), ctypes.c_int32(0)
    _check(_lib.vibe_autotune(h, _ptr(d_syndromes), int(B), _stream_ptr(stream), ctypes.addressof(eng),
                              ctypes.addressof(bp), ctypes.addressof(lsd), ctypes.addressof(nt)))
    return eng.value, bp.value, lsd.value, nt.value


def vibe_destroy(h):
    if h:
        _check(_lib.vibe_destroy(h))


def vibe_batch_create(handles):
    arr = (ctypes.c_void_p * len(handles))(*handles)
    out = ctypes.c_void_p()
    _check(_lib.vibe_batch_create(arr, len(handles), ctypes.byref(out)))
    return out.value


def vibe_batch_decode(b, d_problem, d_syndromes, syn_stride, B, d_corrections, corr_stride, d_logical=None,
                      log_stride=0, d_stats=None, d_observables=None, d_counters=None, stream=None):
    _check(_lib.vibe_batch_decode(b, _ptr(d_problem), _ptr(d_syndromes), int(syn_stride), int(B),
                                  _ptr(d_corrections), int(corr_stride), _ptr(d_logical), int(log_stride),
                                  _ptr(d_stats), _ptr(d_observables), _ptr(d_counters), _stream_ptr(stream)))


def vibe_batch_autotune(b, d_problem, d_syndromes, syn_stride, B, stream=None):
    _check(_lib.vibe_batch_autotune(b, _ptr(d_problem), _ptr(d_syndromes), int(syn_stride), int(B),
                                    _stream_ptr(stream)))


class vibe_launch(ctypes.Structure):
    _fields_ = [("engines", ctypes.c_int32), ("pair_mode", ctypes.c_int32), ("bp_blocks_per_sm", ctypes.c_int32),
                ("bpx_blocks_per_sm", ctypes.c_int32), ("lsd_blocks_per_sm", ctypes.c_int32),
                ("lsd_threads", ctypes.c_int32), ("num_sms", ctypes.c_int32)]


def vibe_get_launch(h=None, b=None):
    """The launch configuration of a handle or a batch, as a dict."""
    out = vibe_launch()
    _check(_lib.vibe_get_launch(h, b, ctypes.byref(out)))
    return {f: getattr(out, f) for f, _ in vibe_launch._fields_}


def vibe_batch_destroy(b):
    if b:
        _check(_lib.vibe_batch_destroy(b))


# ---------------------------------------------------------------------------------------------
# Convenience wrapper
# ---------------------------------------------------------------------------------------------

class Decoder:
    """One resident decoding problem: vibe_create at construction, vibe_destroy on close()."""

    def __init__(self, dem, K, schedules=None, T=30, alpha=0.625, M=None, lsd_order=0, msg_fp16=False, seed=0,
                 engine=ENGINE_AUTO, n_flood=0, member_alpha=None, pair_mode=False, n_layered=0):
        if M is None:
            M = 1 if K == 1 else min(5, K)
        self.dem = dem
        self.m, self.n, self.k = dem.m, dem.n, dem.k
        self.mw, self.nw, self.kw = (self.m + 31) // 32, (self.n + 31) // 32, (self.k + 31) // 32
        self.K, self.T, self.M = K, T, M
        ma = None if member_alpha is None else np.ascontiguousarray(member_alpha, dtype=np.float32)
        if ma is not None and ma.shape != (K,):
            raise ValueError("member_alpha needs one factor per member")
        self.params = vibe_params(int(T), float(alpha), int(M), int(lsd_order), int(bool(msg_fp16)), int(seed),
                                  int(engine), int(n_flood), None if ma is None else ma.ctypes.data,
                                  int(bool(pair_mode)), int(n_layered))
        self.handle = vibe_create(dem.H, dem.L, dem.priors, K, schedules, self.params)
        self.params.member_alpha = None   # vibe_create copied the factors

    def close(self):
        if self.handle:
            vibe_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def decode(self, syndromes, observables=None, want_soft=False, counters=None, stream=None, out=None):
        """syndromes: int32/uint32 CUDA tensor [B, ceil(m/32)]. Returns a dict of CUDA tensors."""
        import torch
        B = int(syndromes.shape[0])
        dev = syndromes.device
        if out is None:
            out = dict(corrections=torch.empty((B, self.nw), dtype=torch.int32, device=dev),
                       logical=torch.empty((B, self.kw), dtype=torch.int32, device=dev),
                       stats=torch.empty((B, 12), dtype=torch.uint8, device=dev),
                       soft=torch.empty((B, self.n), dtype=torch.float32, device=dev) if want_soft else None)
        vibe_decode(self.handle, syndromes, B, out["corrections"], out["logical"], out["stats"], out.get("soft"),
                    observables, counters, stream)
        return out

    def decode_host(self, syndromes, observables=None, stream=None):
        """Host (numpy) buffers through vibe_decode_host; returns numpy outputs and this call's counters."""
        syn = np.ascontiguousarray(syndromes, dtype=np.uint32)
        B = syn.shape[0]
        corr = np.zeros((B, self.nw), np.uint32)
        logi = np.zeros((B, self.kw), np.uint32)
        stats = np.zeros(B, STATS_DTYPE)
        cnt = np.zeros(VIBE_NUM_COUNTERS, np.uint64)
        obs = None if observables is None else np.ascontiguousarray(observables, dtype=np.uint32)
        vibe_decode_host(self.handle, syn, B, corr, logi, stats, obs, cnt, stream)
        return dict(corrections=corr, logical=logi, stats=stats, counters=cnt)

    def wavefronts(self, member):
        return vibe_get_wavefronts(self.handle, member, self.n)

    def layers(self):
        return vibe_get_layers(self.handle, self.m)

    def profile(self, enable=True):
        vibe_profile(self.handle, enable)

    def profile_read(self):
        return vibe_profile_read(self.handle)

    def autotune(self, syndromes, stream=None):
        return vibe_autotune(self.handle, syndromes, int(syndromes.shape[0]), stream)

    def launch(self):
        return vibe_get_launch(h=self.handle)


class MixedBatch:
    """Several Decoders decoded by one launch pair (vibe_batch_*); shot b uses decoders[problem[b]]."""

    def __init__(self, decoders):
        self.decoders = list(decoders)
        self.mw = max(d.mw for d in self.decoders)
        self.nw = max(d.nw for d in self.decoders)
        self.kw = max(d.kw for d in self.decoders)
        self.handle = vibe_batch_create([d.handle for d in self.decoders])

    def close(self):
        if self.handle:
            vibe_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def decode(self, problem, syndromes, observables=None, counters=None, stream=None, out=None):
        """problem: int32 CUDA tensor [B]; syndromes: int32 CUDA tensor [B, >= max ceil(m/32)]."""
        import torch
        B = int(syndromes.shape[0])
        dev = syndromes.device
        if out is None:
            out = dict(corrections=torch.zeros((B, self.nw), dtype=torch.int32, device=dev),
                       logical=torch.zeros((B, self.kw), dtype=torch.int32, device=dev),
                       stats=torch.empty((B, 12), dtype=torch.uint8, device=dev))
        vibe_batch_decode(self.handle, problem, syndromes, syndromes.shape[1], B, out["corrections"],
                          out["corrections"].shape[1], out["logical"], out["logical"].shape[1], out["stats"],
                          observables, counters, stream)
        return out

    def autotune(self, problem, syndromes, stream=None):
        """Times a sample of mixed shots and keeps the fastest launch; returns it (see launch())."""
        vibe_batch_autotune(self.handle, problem, syndromes, syndromes.shape[1], int(syndromes.shape[0]), stream)
        return self.launch()

    def launch(self):
        return vibe_get_launch(b=self.handle)


def stats_to_numpy(stats_tensor):
    """uint8 [B, 12] tensor/array of per-shot records -> numpy structured array."""
    a = stats_tensor.cpu().numpy() if hasattr(stats_tensor, "cpu") else np.asarray(stats_tensor)
    return np.ascontiguousarray(a).view(STATS_DTYPE).reshape(-1)
