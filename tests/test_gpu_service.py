"""The streaming service on the GPU: every request's output equals a direct decode of the same
syndrome with its problem's handle (batching changes nothing per shot), a sample matches the oracle,
and the device-memory budget sizes the micro-batches."""
import numpy as np
import pytest

import oracle
from paper_2508_15743_gb300 import dem as D
from paper_2508_15743_gb300 import service as S

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


def test_service_outputs_equal_direct_decodes_and_oracle(V):
    names = ["codecap_d5", "pheno_d9"]
    svc, backend, decs, dems = S.build_service(names, 2 << 30, fp16=False, max_batch=4096, seed=11)
    arrivals, problems, syn, obs = S.make_requests(dems, 30_000, 150_000.0, seed=12)
    rep, corr, logi, stats = svc.run(arrivals, problems, syn, observables=obs)
    assert rep.requests == 30_000 and rep.batches >= 30_000 / 4096
    assert rep.max_inflight <= rep.capacity
    lat = rep.latency_ms
    assert 0 < lat["p50"] <= lat["p99"] <= lat["p999"] <= lat["max"]
    for i, d in enumerate(decs):
        rows = np.nonzero(problems == i)[0]
        one = d.decode(torch.from_numpy(np.ascontiguousarray(syn[rows][:, :d.mw]).view(np.int32)).cuda())
        assert np.array_equal(corr[rows][:, :d.nw], one["corrections"].cpu().numpy().view(np.uint32)), names[i]
        assert np.array_equal(stats[rows], V.stats_to_numpy(one["stats"])), names[i]
    # a sample against the oracle, per problem
    specs = S._problem_specs()
    for i, dm in enumerate(dems):
        _, K, T, M, natural = specs[names[i]]
        rows = np.nonzero(problems == i)[0][:400]
        perms = D.schedules(dm.n, K, 11 + i, natural=natural)
        r = oracle.decode(dm, perms, syn[rows][:, :D.words(dm.m)], T, 0.625, M, nthreads=8, want_soft=False)
        assert np.array_equal(corr[rows][:, :D.words(dm.n)], r["corrections"]), names[i]
    fails = sum(int((logi[problems == i][:, :1] != obs[problems == i][:, :1]).any(axis=1).sum())
                for i in range(len(dems)))
    assert rep.failures == fails
    backend.close()
    for d in decs:
        d.close()


def test_budget_limits_the_batch(V):
    svc, backend, decs, dems = S.build_service(["pheno_d9"], 1 << 30, fp16=True, max_batch=1 << 22, seed=3)
    b = svc.budget
    assert b["max_batch"] < 1 << 22
    assert b["fixed_bytes"] + b["pipelines"] * b["max_batch"] * b["per_shot_bytes"] <= 1 << 30
    backend.close()
    for d in decs:
        d.close()
    with pytest.raises(MemoryError):
        S.build_service(["pheno_d9"], 1 << 20, fp16=True, max_batch=1024, seed=3)
