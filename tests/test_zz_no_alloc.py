"""vibe_decode_noalloc against vibe_decode, through the C ABI, on two calls in a row.

The no-allocation entry point serves callers that cannot allocate device memory once they are
decoding; it must give exactly what vibe_decode gives, and after its zero-shot set-up call the
device's free memory must not change across a call. This file runs last (collection order) so that
a failure here does not hide the other GPU tests; it must also pass alone in a fresh process.
"""
import numpy as np
import pytest

from paper_2508_15743_gb300 import dem as D

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def V():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2508_15743_gb300 import build
    build.build_library()
    from paper_2508_15743_gb300 import vibe
    return vibe


@pytest.mark.parametrize("fp16", [False, True])
def test_noalloc_matches_decode_on_two_calls(V, fp16):
    w = D.WORKLOADS["cc666_d9_pheno"]
    dm = D.build_workload("cc666_d9_pheno")
    perms = D.schedules(dm.n, w["K"], w["seed"])
    dec = V.Decoder(dm, w["K"], perms, T=w["T"], alpha=w["alpha"], M=w["M"], msg_fp16=fp16)
    V.vibe_decode_noalloc(dec.handle, None, 0, None)   # set-up: places the static array on this device
    for call, (B, seed) in enumerate([(3000, 501), (1777, 502)]):
        syn, _ = D.sample(dm, B, seed)
        syn_t = torch.from_numpy(syn.view(np.int32)).cuda()
        ref = dec.decode(syn_t)
        corr = torch.full((B, dec.nw), -1, dtype=torch.int32, device="cuda")
        logi = torch.full((B, dec.kw), -1, dtype=torch.int32, device="cuda")
        stats = torch.full((B, 12), 255, dtype=torch.uint8, device="cuda")
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        V.vibe_decode_noalloc(dec.handle, syn_t, B, corr, logi, stats)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0, f"call {call}: device memory was allocated"
        assert torch.equal(corr, ref["corrections"]), f"call {call}: corrections differ"
        assert torch.equal(logi, ref["logical"]), f"call {call}: logical flips differ"
        assert torch.equal(stats, ref["stats"]), f"call {call}: per-shot records differ"
        assert int(V.stats_to_numpy(stats)["lsd_invoked"].sum()) > 100
    dec.close()


def test_noalloc_rejects_oversized_batch(V):
    dm = D.build_workload("cc666_d9_pheno")
    dec = V.Decoder(dm, 4, D.schedules(dm.n, 4, 1), T=10, M=2)
    B = 200_000
    syn_t = torch.zeros((B, dec.mw), dtype=torch.int32, device="cuda")
    corr = torch.empty((B, dec.nw), dtype=torch.int32, device="cuda")
    with pytest.raises(V.VibeError) as ei:
        V.vibe_decode_noalloc(dec.handle, syn_t, B, corr)
    assert ei.value.code == V.VIBE_ERR_UNSUPPORTED
    assert "at most" in V.vibe_last_error()
    dec.close()
