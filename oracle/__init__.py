"""CPU oracle for the VibeLSD decoding path -- test infrastructure only.

A plain, slow C implementation (vibe_oracle.c) of serial min-sum BP (Algorithm 1), the K-member
ensemble with correction limit M and likelihood ranking, the normalised LLR average, and LSD
(Sec. III.C-III.D), wrapped here with ctypes. Only the tests, the smoke check and the benchmark's
CPU-baseline leg import this package; the CUDA library never does, and the two share no code.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_SRC = os.path.join(_HERE, "vibe_oracle.c")
_lock = threading.Lock()
_lib = None

FP32, FP16MSG, FP64 = 0, 1, 2

STATS_DTYPE = np.dtype([("status", "u1"), ("lsd_invoked", "u1"), ("n_converged", "u1"),
                        ("chosen_member", "u1"), ("iters", "<u2"), ("largest_cluster", "<u2"),
                        ("n_clusters", "<u4")])


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no contraction, no fast-math) into oracle/_build/liboracle.so."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "vibe_oracle.h"))):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
               "-pthread", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Problem(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int32), ("n", ctypes.c_int32), ("k", ctypes.c_int32),
                ("rowptr", ctypes.c_void_p), ("colidx", ctypes.c_void_p),
                ("lrowptr", ctypes.c_void_p), ("lcolidx", ctypes.c_void_p),
                ("priors", ctypes.c_void_p)]


class _Params(ctypes.Structure):
    _fields_ = [("T", ctypes.c_int32), ("alpha", ctypes.c_float), ("M", ctypes.c_int32),
                ("lsd_order", ctypes.c_int32), ("mode", ctypes.c_int32), ("n_flood", ctypes.c_int32),
                ("member_alpha", ctypes.c_void_p), ("n_layered", ctypes.c_int32)]


def _bind(path):
    lib = ctypes.CDLL(path)
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    lib.or_prior_llr.argtypes = [i32, vp, vp, vp]
    lib.or_bp_member.argtypes = [vp, vp, vp, i32, ctypes.c_float, i32, i32, vp, vp]
    lib.or_bp_member.restype = i32
    lib.or_bp_member_flood.argtypes = [vp, vp, i32, ctypes.c_float, i32, i32, vp, vp]
    lib.or_bp_member_flood.restype = i32
    lib.or_bp_member_layered.argtypes = [vp, vp, i32, ctypes.c_float, i32, i32, vp, vp, vp]
    lib.or_bp_member_layered.restype = i32
    lib.or_check_layers.argtypes = [vp, vp]
    lib.or_check_layers.restype = i32
    lib.or_decode.argtypes = [vp, i32, vp, vp, i64, vp, vp, vp, vp, vp, i32]
    lib.or_decode.restype = i32
    lib.or_lsd.argtypes = [vp, vp, vp, i32, vp, vp, vp, vp, vp, vp]
    lib.or_lsd.restype = i32
    lib.or_seeded_schedules.argtypes = [i32, i32, ctypes.c_uint64, vp]
    return lib


def _load():
    """Bind the oracle library; VIBE_ORACLE_LIB selects another build (used to plant mistakes)."""
    global _lib
    with _lock:
        if _lib is None:
            alt = os.environ.get("VIBE_ORACLE_LIB")
            _lib = _bind(alt if alt else build())
    return _lib


def use_library(path):
    """Point this module at another build of vibe_oracle.c (tests that plant mistakes use this).

    Returns the previous library handle so the caller can restore it with restore_library()."""
    global _lib
    with _lock:
        prev = _lib
        _lib = _bind(path)
    return prev


def restore_library(prev):
    global _lib
    with _lock:
        _lib = prev


def compile_variant(src_text, out_path):
    """Compile a variant of the oracle source (same flags as build()) into out_path."""
    src_path = out_path + ".c"
    with open(src_path, "w") as f:
        f.write(src_text)
    cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
           "-pthread", "-I", _HERE, "-o", out_path, src_path, "-lm"]
    subprocess.run(cmd, check=True)
    return out_path


def source_text():
    with open(_SRC) as f:
        return f.read()


def _ptr(a):
    return None if a is None else a.ctypes.data


class Problem:
    """Holds contiguous copies of a DEM's arrays and the C struct pointing at them."""

    def __init__(self, dem):
        self.dem = dem
        self.rowptr = np.ascontiguousarray(dem.H.rowptr, dtype=np.int32)
        self.colidx = np.ascontiguousarray(dem.H.colidx, dtype=np.int32)
        self.lrowptr = np.ascontiguousarray(dem.L.rowptr, dtype=np.int32)
        self.lcolidx = np.ascontiguousarray(dem.L.colidx, dtype=np.int32)
        self.priors = np.ascontiguousarray(dem.priors, dtype=np.float64)
        self.m, self.n, self.k = dem.H.nrows, dem.H.ncols, dem.L.nrows
        self.c = _Problem(self.m, self.n, self.k, _ptr(self.rowptr), _ptr(self.colidx),
                          _ptr(self.lrowptr), _ptr(self.lcolidx), _ptr(self.priors))


def prior_llr(priors):
    lib = _load()
    priors = np.ascontiguousarray(priors, dtype=np.float64)
    l32 = np.zeros(len(priors), np.float32)
    l64 = np.zeros(len(priors), np.float64)
    lib.or_prior_llr(len(priors), _ptr(priors), _ptr(l32), _ptr(l64))
    return l32, l64


def bp_member(dem, syndrome_bits, perm, T, alpha, mode=FP32, early_stop=True):
    """One serial BP member. syndrome_bits uint8[m]. Returns (t_conv, posterior f64[n], ebits u8[n])."""
    lib = _load()
    P = Problem(dem)
    s = np.ascontiguousarray(syndrome_bits, dtype=np.uint8)
    perm = np.ascontiguousarray(perm, dtype=np.uint32)
    post = np.zeros(P.n, np.float64)
    eb = np.zeros(P.n, np.uint8)
    t = lib.or_bp_member(ctypes.byref(P.c), _ptr(s), _ptr(perm), int(T), float(alpha), int(mode),
                         int(bool(early_stop)), _ptr(post), _ptr(eb))
    return int(t), post, eb


def decode(dem, perms, syndromes, T, alpha, M, lsd_order=0, mode=FP32, nthreads=1, want_soft=True, n_flood=0,
           member_alpha=None, n_layered=0):
    """Full VibeLSD on packed syndromes uint32 [B, ceil(m/32)] with schedules uint32 [K, n].

    member_alpha: None, or K scaling factors, member i using member_alpha[i] instead of alpha.
    n_flood, n_layered: members 0 .. n_flood-1 run the flooding schedule, the next n_layered members
    the layered one, the rest their serial schedules.

    Returns dict(corrections uint32 [B, ceil(n/32)], logical uint32 [B, ceil(k/32)], stats, soft f64 [B, n]).
    """
    lib = _load()
    P = Problem(dem)
    perms = np.ascontiguousarray(perms, dtype=np.uint32)
    K = perms.shape[0]
    syn = np.ascontiguousarray(syndromes, dtype=np.uint32)
    B = syn.shape[0]
    corr = np.zeros((B, (P.n + 31) // 32), np.uint32)
    logi = np.zeros((B, (P.k + 31) // 32), np.uint32)
    stats = np.zeros(B, STATS_DTYPE)
    soft = np.zeros((B, P.n), np.float64) if want_soft else None
    ma = None if member_alpha is None else np.ascontiguousarray(member_alpha, dtype=np.float32)
    if ma is not None and ma.shape != (K,):
        raise ValueError("member_alpha needs one factor per member")
    prm = _Params(int(T), float(alpha), int(M), int(lsd_order), int(mode), int(n_flood),
                  None if ma is None else ma.ctypes.data, int(n_layered))
    rc = lib.or_decode(ctypes.byref(P.c), K, _ptr(perms), ctypes.byref(prm), B, _ptr(syn), _ptr(corr),
                       _ptr(logi), _ptr(stats), _ptr(soft), int(nthreads))
    if rc != 0:
        raise ValueError("oracle rejected the arguments")
    return dict(corrections=corr, logical=logi, stats=stats, soft=soft)


def bp_member_flood(dem, syndrome_bits, T, alpha, mode=FP32, early_stop=True):
    """One parallel-schedule (flooding) BP member, Algorithm 1's other branch.
    Returns (t_conv, posterior f64[n], ebits u8[n])."""
    lib = _load()
    P = Problem(dem)
    s = np.ascontiguousarray(syndrome_bits, dtype=np.uint8)
    post = np.zeros(P.n, np.float64)
    eb = np.zeros(P.n, np.uint8)
    t = lib.or_bp_member_flood(ctypes.byref(P.c), _ptr(s), int(T), float(alpha), int(mode),
                               int(bool(early_stop)), _ptr(post), _ptr(eb))
    return int(t), post, eb


def bp_member_layered(dem, syndrome_bits, T, alpha, mode=FP32, early_stop=True, return_layers=False):
    """One layered-schedule BP member (reading R10). Returns (t_conv, posterior f64[n], ebits u8[n]),
    plus the number of check layers when return_layers is set."""
    lib = _load()
    P = Problem(dem)
    s = np.ascontiguousarray(syndrome_bits, dtype=np.uint8)
    post = np.zeros(P.n, np.float64)
    eb = np.zeros(P.n, np.uint8)
    nl = np.zeros(1, np.int32)
    t = lib.or_bp_member_layered(ctypes.byref(P.c), _ptr(s), int(T), float(alpha), int(mode),
                                 int(bool(early_stop)), _ptr(post), _ptr(eb), _ptr(nl))
    return (int(t), post, eb, int(nl[0])) if return_layers else (int(t), post, eb)


def check_layers(dem):
    """The check layers of reading R10: (layer of each check int32[m], number of layers)."""
    lib = _load()
    P = Problem(dem)
    lay = np.zeros(max(P.m, 1), np.int32)
    nl = lib.or_check_layers(ctypes.byref(P.c), _ptr(lay))
    return lay[:P.m], int(nl)


def lsd(dem, soft, syndrome_bits, order=0, mode=FP32):
    """LSD alone. Returns (status, ebits u8[n], cluster_of_col i32[n], n_clusters, largest)."""
    lib = _load()
    P = Problem(dem)
    soft = np.ascontiguousarray(soft, dtype=np.float64)
    s = np.ascontiguousarray(syndrome_bits, dtype=np.uint8)
    l32, l64 = prior_llr(dem.priors)
    eb = np.zeros(P.n, np.uint8)
    cl = np.zeros(P.n, np.int32)
    ncl = ctypes.c_int32(0)
    big = ctypes.c_int32(0)
    st = lib.or_lsd(ctypes.byref(P.c), _ptr(soft), _ptr(s), int(order), _ptr(l32),
                    _ptr(l64) if mode == FP64 else None, _ptr(eb), _ptr(cl), ctypes.byref(ncl),
                    ctypes.byref(big))
    return int(st), eb, cl, int(ncl.value), int(big.value)


def seeded_schedules(n, K, seed):
    lib = _load()
    out = np.zeros((K, n), np.uint32)
    lib.or_seeded_schedules(int(n), int(K), ctypes.c_uint64(seed), _ptr(out))
    return out
