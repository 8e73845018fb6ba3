"""The serving engine (continuous batching under a device-memory budget):
each request's result is the same alone and in a concurrent mix, and equal
to the oracle; admission waits for memory; latencies are reported."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

P = synth.CompassParams()


@pytest.fixture(scope="module")
def g():
    import paper_2002_11529_gb300 as g
    g.build.build()
    return g


def make_requests(sizes, seed0=500):
    out = []
    for i, n in enumerate(sizes):
        b = synth.generate(n_events=n, n_sectors=256, tracks=200, hits=4000, seed=seed0 + i)
        out.append(b)
    return out


def test_same_result_alone_and_in_the_mix(g):
    from paper_2002_11529_gb300 import serve
    batches = make_requests([64, 300, 128, 700, 64, 256, 1000, 90, 500, 64, 200, 400])
    geom = batches[0].geom
    alone = []
    with serve.Server(geom, P, budget_bytes=4 << 30, n_slots=1) as sv:
        for b in batches:
            req = serve.HostRequest.from_batch(b)
            sv.submit(req)
            res = sv.drain()
            assert len(res) == 1 and res[0]["status"] == 0
            alone.append(req.outputs())
    reqs = [serve.HostRequest.from_batch(b) for b in batches]
    with serve.Server(geom, P, budget_bytes=4 << 30, n_slots=4) as sv:
        summary, res = serve.run_closed_loop(sv, reqs)
        assert not summary["errors"]
        slots = {r["slot"] for r in res}
        assert len(slots) > 1                      # work ran on several streams
    for req, ref in zip(reqs, alone):
        out = req.outputs()
        for k in ref:
            assert np.array_equal(out[k], ref[k]), k
    # and the oracle agrees on two of them
    for i in (0, 3):
        _, ot = oracle.run_batch(batches[i], P)
        out = reqs[i].outputs()
        assert np.array_equal(out["hit"], ot.hit)
        assert np.array_equal(out["qop"].view(np.uint32), ot.qop.view(np.uint32))


def test_admission_waits_for_memory(g):
    from paper_2002_11529_gb300 import serve
    batches = make_requests([400] * 6, seed0=900)
    reqs = [serve.HostRequest.from_batch(b) for b in batches]
    with serve.Server(batches[0].geom, P, budget_bytes=1 << 30, n_slots=8) as probe:
        need = probe.request_bytes(reqs[0])
    budget = int(2.5 * need)                       # room for two at a time
    with serve.Server(batches[0].geom, P, budget_bytes=budget, n_slots=8) as sv:
        summary, res = serve.run_closed_loop(sv, reqs)
        st = sv.stats()
        assert not summary["errors"]
        assert st["arena_peak"] <= budget and st["arena_peak"] >= 2 * need
        assert max(r["queue_s"] for r in res) > 0   # later requests waited
    alone = serve.HostRequest.from_batch(batches[5])
    with serve.Server(batches[0].geom, P, budget_bytes=budget, n_slots=1) as sv:
        sv.submit(alone)
        sv.drain()
    for k in alone.out:
        assert np.array_equal(alone.outputs()[k], reqs[5].outputs()[k])


def test_request_larger_than_budget_is_refused(g):
    from paper_2002_11529_gb300 import serve
    b = make_requests([200], seed0=1200)[0]
    with serve.Server(b.geom, P, budget_bytes=1 << 20, n_slots=2) as sv:
        with pytest.raises(Exception):
            sv.submit(serve.HostRequest.from_batch(b))


def test_open_loop_reports_latency(g):
    from paper_2002_11529_gb300 import serve
    rng = np.random.default_rng(4)
    sizes = np.exp(rng.uniform(np.log(64), np.log(4096), 10)).astype(int)
    reqs = [serve.HostRequest.from_batch(b) for b in make_requests(list(sizes), seed0=1300)]
    with serve.Server(reqs and synth.Geometry(n_sectors=256), P, budget_bytes=8 << 30, n_slots=4) as sv:
        summary, res = serve.run_open_loop(sv, reqs, events_per_s=200_000.0)
    assert not summary["errors"] and summary["requests"] == 10
    assert summary["p99_ms"] >= summary["p50_ms"] > 0
