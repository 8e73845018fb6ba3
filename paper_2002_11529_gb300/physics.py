"""Physics performance of the found tracks on synthetic truth (Sec. II-C).

A particle is reconstructible when its hits lie in at least three of the
four UT layers (and its VELO track is a forward one).  A found track is
reconstructed when at least 70 % of its UT hits come from one particle;
here every VELO track is one generated particle, so a found track counts as
reconstructed when that particle is its own, and as a fake otherwise (its
UT hits belong to no particle, or to another particle than its VELO part).
Efficiency = reconstructed and reconstructible / reconstructible; fake rate
= fakes / found tracks.  A clone needs two found tracks of one particle,
which one output slot per VELO track excludes: the clone rate is 0 here.

Hit indices of the found tracks refer to the x-sorted hits; the generator's
truth is in raw (bank, word) order, and the sort is stable by half-strip
inside each bank, so the same stable order maps one to the other.
"""
from __future__ import annotations

import numpy as np

RECONSTRUCTED_FRACTION = 0.7


def sorted_to_raw(batch) -> np.ndarray:
    """Raw (bank, word) index of every hit of the x-sorted order."""
    bank = np.repeat(np.arange(batch.bank_n.size), batch.bank_n.astype(np.int64))
    return np.lexsort((batch.truth_h.astype(np.int64), bank))


def own_track(batch, tracks: dict) -> np.ndarray:
    """Per track slot: found, and at least 70 % of its UT hits come from the
    particle of its own VELO track (reconstructed)."""
    T = batch.n_tracks
    hit = np.asarray(tracks["hit"])[:T]
    found = np.asarray(tracks["found"])[:T].astype(bool)
    owner_raw = np.asarray(batch.truth_track, np.int64)
    perm = sorted_to_raw(batch)
    present = hit >= 0
    owner = np.full(hit.shape, -1, np.int64)
    owner[present] = owner_raw[perm[hit[present]]]
    nh = present.sum(axis=1)
    own = (present & (owner == np.arange(T)[:, None])).sum(axis=1)
    return found & (nh > 0) & (own >= RECONSTRUCTED_FRACTION * np.maximum(nh, 1))


def evaluate(batch, tracks: dict) -> dict:
    """tracks: the track slots (numpy: hit [T,4] sorted-hit indices or -1,
    found [T]) of `batch`.  Returns counts and rates."""
    T = batch.n_tracks
    found = np.asarray(tracks["found"])[:T].astype(bool)
    owner_raw = np.asarray(batch.truth_track, np.int64)
    correct = own_track(batch, tracks)
    fake = found & ~correct
    # reconstructible: true hits in >= 3 layers, forward VELO track
    sig = owner_raw >= 0
    layers = np.zeros((T, 4), bool)
    layers[owner_raw[sig], np.asarray(batch.truth_layer)[sig].astype(np.int64)] = True
    forward = (np.asarray(batch.velo_flags)[:T] & 1) == 0
    reconstructible = forward & (layers.sum(axis=1) >= 3)
    n_rec = int(reconstructible.sum())
    n_found = int(found.sum())
    return {"tracks": T, "reconstructible": n_rec, "found": n_found,
            "reconstructed_and_reconstructible": int((correct & reconstructible).sum()),
            "fakes": int(fake.sum()), "clones": 0,
            "efficiency": float((correct & reconstructible).sum() / n_rec) if n_rec else None,
            "fake_rate": float(fake.sum() / n_found) if n_found else None,
            "clone_rate": 0.0 if n_found else None}
