"""The bounds-checked build (UT_CHECKED=1: -DUT_CHECKED, the library that
compares every checked index with its array's extent).

Run the whole GPU suite under it with `UT_CHECKED=1 python -m pytest tests
-m gpu`: every parity test then also shows that no checked access left its
array (the tests read the status word).  The test below gives the alignment
kernels a hit index beyond the capacity the caller declares; the arrays
behind it are larger, so the plain build reads valid memory, and the
checked build must refuse the access and record UT_ERR_BOUNDS (site 601)."""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    import paper_2002_11529_gb300 as g
    g.build.build()
    assert torch.cuda.is_available()
    return g


def test_checked_build_reports_an_index_beyond_the_declared_capacity(g):
    a = synth.generate_alignment(2000, 64, seed=9)
    b = a.batch
    ctx = g.Context(b.geom)
    raw, ev = g.upload_raw(b.raw, b.ev_off)
    nw = int(b.ev_off[-1])
    hits = g.HitBuffers.allocate(2 * nw, b.n_events, b.geom.n_sectors)
    g.ut_decode(ctx, raw, nw, ev, b.n_events, hits, sorted_=False)
    ctx.check(what="decode")
    n = int(hits.hit_off[-1].item())
    th = np.ascontiguousarray(a.track_hits).copy()
    th[7, 0] = n + 3                       # inside the allocation, beyond `capacity` below
    for arr in (hits.x, hits.z, hits.sector, hits.layer, hits.id):
        arr[n:n + 4].zero_()               # a valid hit (layer 0, sector 0) for the plain build
    hits.capacity = n                      # the caller declares exactly n hits
    t = lambda arr, dt: torch.from_numpy(np.ascontiguousarray(arr).view(dt)).cuda()
    velo = g.VeloBuffers(t(a.x, np.float32), t(a.y, np.float32), t(a.tx, np.float32), t(a.ty, np.float32),
                         torch.zeros(a.n_tracks, dtype=torch.uint8, device="cuda"),
                         torch.zeros(2, dtype=torch.int32, device="cuda"))
    from paper_2002_11529_gb300 import align
    prob = align.AlignmentProblem(ctx, hits, t(th, np.int32), velo, synth.CompassParams())
    ctx.reset()
    prob.refit(torch.zeros((4 * b.geom.n_sectors, 3), dtype=torch.float32, device="cuda"))
    code, where_a, where_b = ctx.status()
    if g.build.checked():
        assert (code, where_a, where_b) == (g.UT_ERR_BOUNDS, -1, 601)
    else:
        assert code == g.UT_OK              # the plain build does not look
    ctx.close()
