"""Serving: request recipe, memory estimate (CPU) and continuous batching
that leaves every result unchanged (GPU)."""
import numpy as np
import pytest


def test_request_stream_recipe():
    from paper_1005_5312_gb300.serve import make_requests
    reqs = make_requests(64, rate_hz=50.0, log2_np=(12, 14), seed=3)
    assert len(reqs) == 64
    t = np.array([r.t_arrive for r in reqs])
    assert np.all(np.diff(t) > 0)
    assert 0.01 < t[-1] / 64 < 0.04                       # mean 20 ms
    for r in reqs:
        assert 2 ** 12 - 1 <= r.n_p <= 2 ** 14 + 1 and 1 <= r.n_s <= r.n_p
        assert r.theta in (0.5, 1.0)
        assert r.pos.shape == (3, r.n_p) and r.pos.dtype == np.float32
        assert r.pos.min() >= 0 and r.pos.max() <= 6.6


def test_memory_estimate_is_monotone_and_capped():
    from paper_1005_5312_gb300.serve import list_length_estimate, memory_estimate
    assert abs(list_length_estimate(1024, 0.5) - 321) < 0.1 * 321
    assert abs(list_length_estimate(1024, 1.0) - 146) < 0.1 * 146
    assert list_length_estimate(3, 0.5) == 3
    a = memory_estimate(1 << 16, 100, 0.5, 1 << 27)
    b = memory_estimate(1 << 18, 100, 0.5, 1 << 27)
    c = memory_estimate(1 << 18, 10000, 0.5, 1 << 27)
    d = memory_estimate(1 << 21, 1 << 20, 0.5, 1 << 27)
    assert a < b < c < d
    assert d < memory_estimate(1 << 21, 1 << 20, 0.5, 1 << 40)   # the pair budget caps it


def test_request_knobs_policy():
    """Resident chains only for requests of several coupled steps (unless
    fixed by the server); the tuner's knobs of the request's class on top."""
    from paper_1005_5312_gb300.autotune import Tuner, problem_class
    from paper_1005_5312_gb300.serve import make_requests, request_knobs
    one, two = make_requests(2, log2_np=(12, 13), seed=5, steps=1)[0], \
        make_requests(1, log2_np=(12, 13), seed=6, steps=2)[0]
    assert request_knobs(one) == {"reuse_chains": 0}
    assert request_knobs(two) == {"reuse_chains": 1}
    assert request_knobs(two, reuse_fixed=True) == {}
    t = Tuner()
    t.cache[problem_class(one.n_p, one.n_s, one.theta)] = {"march_group": 4, "row_bins": 6}
    k = request_knobs(one, tuner=t)
    assert k["reuse_chains"] == 0 and k["march_group"] == 4 and k["row_bins"] == 6


@pytest.mark.gpu
def test_results_identical_alone_and_in_a_mix():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1005_5312_gb300 as S
    from paper_1005_5312_gb300.serve import Server, make_requests, summarize
    S.build()
    reqs = make_requests(8, rate_hz=200.0, log2_np=(12, 14.5), seed=11, steps=2)
    alone = Server(workers=1)
    r1 = alone.serve(reqs, realtime=False)
    alone.close()
    mixed = Server(workers=4)
    r2 = mixed.serve(reqs, realtime=True)
    mixed.close()
    for a, b in zip(r1, r2):
        assert a.rid == b.rid
        assert np.array_equal(a.gamma, b.gamma)
        assert np.array_equal(a.y, b.y)
        assert a.rays == b.rays > 0
    s = summarize(r2)
    assert s["n"] == 8 and s["solves_per_s"] > 0 and s["p99_ms"] >= s["p50_ms"]
    # a budget smaller than any request still serves them, one at a time
    tight = Server(workers=3, budget_bytes=1.0)
    r3 = tight.serve(reqs[:3], realtime=False)
    tight.close()
    for a, b in zip(r1[:3], r3):
        assert np.array_equal(a.gamma, b.gamma)
    # workers whose contexts are recreated after every request (trim threshold 0)
    trimmed = Server(workers=2, trim_bytes=0.0)
    r4 = trimmed.serve(reqs, realtime=False)
    assert trimmed.trims == len(reqs)
    trimmed.close()
    for a, b in zip(r1, r4):
        assert np.array_equal(a.gamma, b.gamma) and np.array_equal(a.y, b.y)


@pytest.mark.gpu
def test_batched_small_requests_identical_to_alone():
    """Small requests that have arrived together are solved as one batch
    (start_build_batch): every request's Gamma and y are bitwise those of
    solving it alone, over two coupled steps (full solves each step: a batch
    keeps no resident chains)."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1005_5312_gb300 as S
    from paper_1005_5312_gb300.serve import Server, make_requests
    S.build()
    reqs = make_requests(24, rate_hz=1e6, log2_np=(9, 13), seed=12, steps=2)
    alone = Server(workers=1, reuse_chains=0)
    r1 = alone.serve(reqs, realtime=False)
    alone.close()
    batched = Server(workers=2, batch_small=8, small_n_p=1 << 13, reuse_chains=0)
    r2 = batched.serve(reqs, realtime=True)
    assert batched.batches > 0
    batched.close()
    for a, b in zip(r1, r2):
        assert a.rid == b.rid
        assert np.array_equal(a.gamma, b.gamma)
        assert np.array_equal(a.y, b.y)
