"""The physics-performance bookkeeping (CPU): truth mapping and the
reconstructed / fake / reconstructible rules on hand-made track slots."""
import numpy as np

import oracle
import synth
from paper_2002_11529_gb300 import physics


def _batch():
    return synth.generate(n_events=6, n_sectors=16, tracks=40, hits=700, seed=21)


def test_sorted_to_raw_matches_the_decoded_order():
    b = _batch()
    _, hits, _ = oracle.decode(b.raw, b.ev_off, b.n_events, b.geom, sorted_=True)
    perm = physics.sorted_to_raw(b)
    # the decoded id carries (layer, sector, word): the raw word of perm[i]
    word = (b.truth_h.astype(np.int64) >> 1) | ((b.truth_h.astype(np.int64) & 1) << 10) | \
           (b.truth_flags.astype(np.int64) << 11)
    raw_id = (b.truth_layer.astype(np.int64) << 24) | (b.truth_sector.astype(np.int64) << 16) | word
    assert np.array_equal(raw_id[perm], hits.id[: hits.n].astype(np.int64))


def _truth_hits(b, perm):
    """Sorted-hit indices of every generated track's own hits, per layer."""
    inv = np.empty_like(perm)
    inv[perm] = np.arange(perm.size)
    T = b.n_tracks
    own = np.full((T, 4), -1, np.int64)
    sig = np.nonzero(b.truth_track >= 0)[0]
    own[b.truth_track[sig], b.truth_layer[sig].astype(np.int64)] = inv[sig]
    return own


def test_truth_tracks_are_all_reconstructed_and_no_fakes():
    b = _batch()
    own = _truth_hits(b, physics.sorted_to_raw(b))
    nh = (own >= 0).sum(1)
    tracks = {"hit": own, "found": (nh >= 3).astype(np.uint8)}
    r = physics.evaluate(b, tracks)
    assert r["efficiency"] == 1.0 and r["fakes"] == 0 and r["clones"] == 0
    assert r["reconstructible"] == int((nh >= 3).sum())


def test_seventy_percent_rule_and_foreign_hits():
    b = _batch()
    own = _truth_hits(b, physics.sorted_to_raw(b))
    full = np.nonzero((own >= 0).all(1))[0]
    t0, t1, t2 = full[:3]
    hit = np.full((b.n_tracks, 4), -1, np.int64)
    found = np.zeros(b.n_tracks, np.uint8)
    noise = int(np.nonzero(b.truth_track[physics.sorted_to_raw(b)] < 0)[0][0])
    hit[t0] = own[t0]
    hit[t0, 3] = noise                   # 3 of 4 own hits: 75 %, reconstructed
    hit[t1, :3] = own[t1, :3]
    hit[t1, 2] = noise                   # 2 of 3: 67 %, fake
    hit[t2] = own[t1]                    # another particle's hits: fake
    found[[t0, t1, t2]] = 1
    r = physics.evaluate(b, {"hit": hit, "found": found})
    assert r["found"] == 3 and r["fakes"] == 2
    assert r["reconstructed_and_reconstructible"] == 1
