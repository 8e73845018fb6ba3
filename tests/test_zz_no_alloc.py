"""ut_decode_noalloc: the allocation-free decode entry point.

Some callers cannot allocate device memory (a host framework that keeps
all device memory in its own pool, or a processing loop that must not pay
cudaMalloc's implicit synchronisation).  This entry point takes no
workspace and no context: its scratch is a static device array of the
library.  These tests call it through the C ABI and compare its output with
ut_decode's, bit for bit, on two calls in a row (the second on a smaller
batch, so stale scratch from the first call must not leak into it), and
with the CPU oracle's decode.
"""
import ctypes

import numpy as np
import pytest

import oracle
import synth


def test_rejects_too_many_events_without_touching_the_gpu():
    import paper_2002_11529_gb300 as g
    g.build.build()
    geom = g.geometry_struct(synth.Geometry(n_sectors=4))
    h = g.UtHits()
    h.hit_off = 16
    rc = g.lib().ut_decode_noalloc(ctypes.byref(geom), None, 0, None, 65537, ctypes.byref(h), 1,
                                   ctypes.c_void_p(8), None)
    assert rc == g.UT_ERR_ARG


@pytest.mark.gpu
def test_noalloc_decode_matches_ut_decode_twice():
    import torch
    import paper_2002_11529_gb300 as g
    g.build.build()
    big = synth.generate_config("plain", n_events=300)
    small = synth.generate_config("plain", n_events=120, seed=77)
    geom = big.geom
    ctx = g.Context(geom)
    status = torch.empty(1, dtype=torch.int64, device="cuda")
    for b in (big, small):
        raw, ev = g.upload_raw(b.raw, b.ev_off)
        nw = int(b.ev_off[-1])
        for sorted_ in (True, False):
            ref = g.HitBuffers.allocate(2 * nw, b.n_events, geom.n_sectors)
            ctx.reset()
            g.ut_decode(ctx, raw, nw, ev, b.n_events, ref, sorted_)
            assert ctx.status()[0] == 0
            got = g.HitBuffers.allocate(2 * nw, b.n_events, geom.n_sectors)
            g.ut_decode_noalloc(geom, raw, nw, ev, b.n_events, got, status, sorted_)
            torch.cuda.synchronize()
            assert g.decode_status_key(int(status.item())) == (0, -1, -1)
            r, o = g.hits_to_numpy(ref), g.hits_to_numpy(got)
            assert np.array_equal(r["hit_off"], o["hit_off"])
            n = int(r["hit_off"][-1])
            assert n == b.n_hits
            for k in ("x", "z", "sector", "layer", "id"):
                assert np.array_equal(r[k][:n].view(np.uint8), o[k][:n].view(np.uint8)), k
            # and the oracle's decode, directly
            rc, oh, _ = oracle.decode(b.raw, b.ev_off, b.n_events, geom, sorted_)
            assert rc == 0
            assert np.array_equal(o["hit_off"], oh.hit_off)
            assert np.array_equal(o["x"][:n].view(np.uint32), oh.x[:n].view(np.uint32))
            assert np.array_equal(o["id"][:n], oh.id[:n])
    ctx.close()


@pytest.mark.gpu
def test_noalloc_argument_error_enqueues_nothing():
    """A call refused by a host check (a null output array) returns
    UT_ERR_ARG without writing the caller's status word."""
    import torch
    import paper_2002_11529_gb300 as g
    g.build.build()
    b = synth.generate_config("tiny")
    raw, ev = g.upload_raw(b.raw, b.ev_off)
    nw = int(b.ev_off[-1])
    out = g.HitBuffers.allocate(2 * nw, b.n_events, b.geom.n_sectors)
    h = out.struct()
    h.z = None
    status = torch.full((1,), 1234, dtype=torch.int64, device="cuda")
    geo = g.geometry_struct(b.geom)
    rc = g.lib().ut_decode_noalloc(ctypes.byref(geo), ctypes.c_void_p(raw.data_ptr()), nw,
                                   ctypes.c_void_p(ev.data_ptr()), b.n_events, ctypes.byref(h), 1,
                                   ctypes.c_void_p(status.data_ptr()), None)
    assert rc == g.UT_ERR_ARG
    torch.cuda.synchronize()
    assert int(status.item()) == 1234


@pytest.mark.gpu
def test_noalloc_reports_errors_in_caller_status():
    import torch
    import paper_2002_11529_gb300 as g
    g.build.build()
    b = synth.generate_config("tiny")
    bad = b.raw.copy()
    base = int(b.ev_off[5])
    d = base + int(bad[base + 7])
    bad[d] = (bad[d] & 0xFFFF) | (9 << 16)
    raw, ev = g.upload_raw(bad, b.ev_off)
    nw = int(b.ev_off[-1])
    out = g.HitBuffers.allocate(2 * nw, b.n_events, b.geom.n_sectors)
    status = torch.empty(1, dtype=torch.int64, device="cuda")
    g.ut_decode_noalloc(b.geom, raw, nw, ev, b.n_events, out, status, True)
    torch.cuda.synchronize()
    assert g.decode_status_key(int(status.item())) == (g.UT_ERR_HEADER, 5, 7)
