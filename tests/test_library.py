"""CPU checks of the C-ABI library: it builds, loads, exports every entry point of include/vibe.h,
and rejects malformed input on the host before any device work (no GPU needed)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2508_15743_gb300 import build as B
from paper_2508_15743_gb300 import dem as D

HEADER = os.path.join(B.INCLUDE, "vibe.h")


@pytest.fixture(scope="module")
def V():
    B.build_library()
    from paper_2508_15743_gb300 import vibe
    return vibe


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(vibe_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["vibe_create", "vibe_decode", "vibe_decode_host", "vibe_destroy", "vibe_last_error",
                     "vibe_get_wavefronts", "vibe_profile", "vibe_profile_read"]:
        assert required in names


def test_library_exports_every_declared_symbol(V):
    lib = ctypes.CDLL(V.LIBRARY_PATH)
    for name in declared_functions():
        assert hasattr(lib, name), f"{name} declared in vibe.h but not exported"


def test_library_is_sm103a_only():
    # the build compiles exactly one target: sm_103a
    assert B.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def _params(V, **kw):
    p = dict(max_iter=20, alpha=0.625, M=1, lsd_order=0, msg_fp16=0, seed=0, bp_engine=0, n_flood=0,
             member_alpha=None, pair_mode=0, n_layered=0)
    p.update(kw)
    ma = p["member_alpha"]
    return V.vibe_params(p["max_iter"], p["alpha"], p["M"], p["lsd_order"], p["msg_fp16"], p["seed"],
                         p["bp_engine"], p["n_flood"], None if ma is None else ma.ctypes.data, p["pair_mode"],
                         p["n_layered"])


def _err(V, H, L, priors, K, sched, params):
    with pytest.raises(V.VibeError) as ei:
        V.vibe_create(H, L, priors, K, sched, params)
    return ei.value.code, V.vibe_last_error()


def test_host_validation_rejects_bad_input(V):
    dm = D.build_workload("cc666_d5_codecap")
    H, L, pr = dm.H, dm.L, dm.priors
    ok = _params(V)
    # malformed CSR: descending columns
    bad = D.CSR(H.nrows, H.ncols, H.rowptr.copy(), H.colidx.copy())
    bad.colidx[0], bad.colidx[1] = bad.colidx[1], bad.colidx[0]
    code, msg = _err(V, bad, L, pr, 1, None, ok)
    assert code == V.VIBE_ERR_INVALID and "ascending" in msg
    # column index out of range
    bad = D.CSR(H.nrows, H.ncols, H.rowptr.copy(), H.colidx.copy())
    bad.colidx[-1] = H.ncols
    assert _err(V, bad, L, pr, 1, None, ok)[0] == V.VIBE_ERR_INVALID
    # empty row
    rows = [list(H.row(r)) for r in range(H.nrows)] + [[]]
    assert _err(V, D.CSR.from_rows(rows, H.ncols), L, pr, 1, None, ok)[0] == V.VIBE_ERR_INVALID
    # priors outside (0, 0.5)
    for bad_p in [0.0, 0.5, -0.1, np.nan]:
        p2 = pr.copy()
        p2[3] = bad_p
        assert _err(V, H, L, p2, 1, None, ok)[0] == V.VIBE_ERR_INVALID
    # parameters
    assert _err(V, H, L, pr, 0, None, ok)[0] == V.VIBE_ERR_INVALID
    assert _err(V, H, L, pr, 4, None, _params(V, M=5))[0] == V.VIBE_ERR_INVALID
    assert _err(V, H, L, pr, 1, None, _params(V, max_iter=0))[0] == V.VIBE_ERR_INVALID
    assert _err(V, H, L, pr, 1, None, _params(V, alpha=0.0))[0] == V.VIBE_ERR_INVALID
    assert _err(V, H, L, pr, 1, None, _params(V, msg_fp16=2))[0] == V.VIBE_ERR_INVALID
    assert _err(V, H, L, pr, 1, None, _params(V, bp_engine=3))[0] == V.VIBE_ERR_INVALID
    assert _err(V, H, L, pr, 1, None, _params(V, bp_engine=-1))[0] == V.VIBE_ERR_INVALID
    assert _err(V, H, L, pr, 1, None, _params(V, pair_mode=2))[0] == V.VIBE_ERR_INVALID
    # flooding and layered members: n_flood + n_layered <= K, the image engine only
    assert _err(V, H, L, pr, 1, None, _params(V, n_flood=2))[0] == V.VIBE_ERR_INVALID
    assert _err(V, H, L, pr, 1, None, _params(V, n_layered=2))[0] == V.VIBE_ERR_INVALID
    assert _err(V, H, L, pr, 1, None, _params(V, n_flood=1, n_layered=1))[0] == V.VIBE_ERR_INVALID
    assert _err(V, H, L, pr, 1, None, _params(V, n_layered=-1))[0] == V.VIBE_ERR_INVALID
    assert _err(V, H, L, pr, 1, None, _params(V, n_flood=1, bp_engine=2))[0] == V.VIBE_ERR_UNSUPPORTED
    assert _err(V, H, L, pr, 1, None, _params(V, n_layered=1, bp_engine=2))[0] == V.VIBE_ERR_UNSUPPORTED
    # per-member scaling factors: one per member (checked by the binding), each in (0, 1] (the library)
    with pytest.raises(ValueError):
        V.Decoder(dm, 2, None, T=5, M=1, member_alpha=np.array([0.5, 0.5, 0.5], np.float32))
    for bad_a in [0.0, 1.5, -0.5, np.nan]:
        ma = np.array([0.625, bad_a], np.float32)
        code, msg = _err(V, H, L, pr, 2, None, _params(V, member_alpha=ma))
        assert code == V.VIBE_ERR_INVALID and "member_alpha[1]" in msg
    # schedules must be permutations
    sched = np.tile(np.arange(H.ncols, dtype=np.uint32), (2, 1))
    sched[1, 0] = sched[1, 1]
    assert _err(V, H, L, pr, 2, sched, _params(V, M=1))[0] == V.VIBE_ERR_INVALID
    # L shape
    Lbad = D.CSR.from_rows([[0]], H.ncols + 1)
    assert _err(V, H, Lbad, pr, 1, None, ok)[0] == V.VIBE_ERR_INVALID


def test_column_degree_limit_is_reported(V):
    # a column in 33 checks
    rows = [[0, j] for j in range(1, 34)]
    H = D.CSR.from_rows(rows, 34)
    L = D.CSR.from_rows([[0]], 34)
    code, msg = _err(V, H, L, np.full(34, 0.1), 1, None, _params(V))
    assert code == V.VIBE_ERR_UNSUPPORTED and "32" in msg


def test_get_launch_wants_exactly_one_object(V):
    import ctypes
    out = V.vibe_launch()
    assert V._lib.vibe_get_launch(None, None, ctypes.byref(out)) == V.VIBE_ERR_INVALID
    assert V._lib.vibe_batch_autotune(None, None, None, 1, 1, None) == V.VIBE_ERR_INVALID


def test_decode_rejects_null_handle(V):
    with pytest.raises(V.VibeError) as ei:
        V.vibe_decode(None, 0, 1, 0, stream=0)
    assert ei.value.code == V.VIBE_ERR_INVALID
    with pytest.raises(V.VibeError):
        V.vibe_decode_host(None, np.zeros((1, 1), np.uint32), 1, np.zeros((1, 1), np.uint32), stream=0)
