"""The sector-group layout (ut_sector_groups, Sec. IV and Table I) against
the oracle, bit for bit: x, z, y range, weight, id and group offsets."""
import numpy as np
import pytest
import torch

import oracle
from synth.grouped import GroupGeometry, generate_grouped

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    import paper_2002_11529_gb300 as g
    g.build.build()
    assert torch.cuda.is_available()
    return g


CASES = {
    "default": dict(n_events=16),
    "rows3_groups10": dict(n_events=12, n_columns=8, rows=3, n_groups=10, seed=3),
    "one_row": dict(n_events=8, rows=1, n_groups=6, seed=4),
    "busy": dict(n_events=200, tracks=150, hits=3000, seed=9),
    "max_groups": dict(n_events=6, n_columns=32, rows=7, n_groups=128, tracks=100, hits=2500, seed=10),
    # 4 x 128 x 8 keys: the most the layout takes (fewer warp tables fit)
    "max_keys": dict(n_events=5, n_columns=31, rows=8, n_groups=128, tracks=100, hits=3000, seed=12),
    "one_event_dense": dict(n_events=1, tracks=200, hits=6000, seed=13),
    # events with fewer hits than warps (empty and short chunks), and empty events
    "sparse": dict(n_events=6, tracks=1, hits=5, seed=21),
    "empty": dict(n_events=6, tracks=0, hits=0, seed=22),
}


@pytest.mark.parametrize("name", list(CASES))
def test_sector_groups_match_oracle(g, name):
    b = generate_grouped(**CASES[name])
    ref = oracle.decode_groups(b.raw, b.ev_off, b.n_events, b.geom)
    ctx, out = g.decode_groups(b.raw, b.ev_off, b.n_events, b.geom)
    got = g.group_hits_to_numpy(out)
    assert np.array_equal(got["group_off"], ref.group_off)
    assert np.array_equal(got["id"], ref.id)
    for k, r in (("x", ref.x), ("z", ref.z), ("y_begin", ref.y_begin), ("y_end", ref.y_end),
                 ("weight", ref.weight)):
        assert np.array_equal(got[k].view(np.uint32), r.view(np.uint32)), k
    ctx.close()


def test_refused_geometries(g):
    """A group geometry whose sensors are not the context's (host check,
    nothing launched)."""
    b = generate_grouped(4)
    ctx, out = g.decode_groups(b.raw, b.ev_off, b.n_events, b.geom)
    raw_d, ev_d = g.upload_raw(b.raw, b.ev_off)
    nw = int(b.ev_off[-1])
    hits = g.HitBuffers.allocate(2 * nw + 8, b.n_events, b.geom.n_columns * b.geom.rows)
    g.ut_decode(ctx, raw_d, nw, ev_d, b.n_events, hits, False)
    bad = GroupGeometry(b.geom.n_columns, rows=b.geom.rows + 1)
    with pytest.raises(g.UtError) as err:
        g.ut_sector_groups(ctx, hits, b.n_events, bad, out)
    assert err.value.code == g.UT_ERR_ARG
    ctx.check(what="refused geometry")
    ctx.close()
