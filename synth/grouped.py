"""Seeded synthetic events for the sector-group decoding (Sec. IV): sensors
of finite strip length and pre-defined x regions ("sector groups").

A plane is tiled along x by `n_columns` columns of 96 mm (as in the base
detector) and along y by `rows` rows of `sensor_height` mm centred on y = 0;
sensor (c, r) is raw bank s = c * rows + r of its layer (bank b = l *
n_columns * rows + s), so the raw format is the base one with
n_columns * rows sectors.  A hit's strips span its sensor's y range.  The
sector groups of a plane are `n_groups` x regions over the plane, narrower
in the centre: group j from the centre (on either side) is j + 1 times the
central width.

Hits are made with the base generator (same tracks, kick and noise) and
placed in the row their track crosses at the plane (noise in a random
row); hits outside the rows are lost.  This module holds no decoding
arithmetic of the method.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from .generator import Geometry, encode, generate, SECTOR_PITCH, STRIP_PITCH, Z_LAYERS, Z_VELO


@dataclasses.dataclass
class GroupGeometry:
    n_columns: int
    rows: int = 4
    sensor_height: float = 250.0
    n_groups: int = 24
    base: Geometry = None
    edges: np.ndarray = None    # optional explicit group edges (float32[n_groups + 1])

    def __post_init__(self):
        if self.base is None:
            self.base = Geometry(n_sectors=self.n_columns)

    @property
    def x_min(self) -> float:
        return self.base.x_min

    @property
    def y_min(self) -> float:
        return float(np.float32(-self.rows * self.sensor_height / 2.0))

    @property
    def n_banks(self) -> int:
        return 4 * self.n_columns * self.rows

    def group_edges(self) -> np.ndarray:
        """float32[n_groups + 1]: x edges of the groups (x_min ... x_max)."""
        if self.edges is not None:
            return np.asarray(self.edges, np.float32)
        half = self.n_groups // 2
        span = self.n_columns * SECTOR_PITCH / 2.0
        w0 = span / (half * (half + 1) / 2.0)
        right = np.cumsum(w0 * np.arange(1, half + 1, dtype=np.float64))
        e = np.concatenate([-right[::-1], [0.0], right])
        e[0], e[-1] = -span, span
        return e.astype(np.float32)

    def raw_geometry(self) -> Geometry:
        """The base geometry with one sector per sensor (validates the raw banks)."""
        return Geometry(n_sectors=self.n_columns * self.rows)


@dataclasses.dataclass
class GroupedBatch:
    geom: GroupGeometry
    n_events: int
    raw: np.ndarray
    ev_off: np.ndarray
    bank_n: np.ndarray          # u32[E * n_banks]
    truth_event: np.ndarray     # per raw hit word, raw (bank) order
    truth_layer: np.ndarray
    truth_column: np.ndarray
    truth_row: np.ndarray
    truth_h: np.ndarray
    truth_flags: np.ndarray
    truth_track: np.ndarray
    truth_y: np.ndarray         # float64: the track's y at the plane (NaN for noise)
    velo_x: np.ndarray = None   # the VELO tracks of the base batch (as synth.Batch)
    velo_y: np.ndarray = None
    velo_tx: np.ndarray = None
    velo_ty: np.ndarray = None
    velo_flags: np.ndarray = None
    trk_off: np.ndarray = None
    qop_true: np.ndarray = None

    @property
    def n_tracks(self) -> int:
        return int(self.trk_off[-1])


def generate_grouped(n_events: int, n_columns: int = 16, rows: int = 4, sensor_height: float = 250.0,
                     n_groups: int = 24, tracks=60, hits=1200, seed: int = 1, edges=None, **kw) -> GroupedBatch:
    """kw: further arguments of the base generator (noise_frac, efficiency, ...)."""
    gg = GroupGeometry(n_columns, rows, sensor_height, n_groups, edges=edges)
    b = generate(n_events=n_events, n_sectors=n_columns, tracks=tracks, hits=hits, seed=seed, **kw)
    rng = np.random.Generator(np.random.Philox(key=seed + 7919))
    tr = b.truth_track
    sig = tr >= 0
    z = np.asarray(Z_LAYERS, np.float64)[b.truth_layer.astype(np.int64)]
    y = np.full(tr.size, np.nan)
    y[sig] = b.velo_y[tr[sig]].astype(np.float64) + b.velo_ty[tr[sig]].astype(np.float64) * (z[sig] - Z_VELO)
    row = np.empty(tr.size, np.int64)
    row[sig] = np.floor((y[sig] - gg.y_min) / sensor_height).astype(np.int64)
    row[~sig] = rng.integers(0, rows, int((~sig).sum()))
    keep = (row >= 0) & (row < rows)
    ev = b.truth_event[keep].astype(np.int64)
    ly = b.truth_layer[keep].astype(np.int64)
    col = b.truth_sector[keep].astype(np.int64)
    rw = row[keep]
    S2 = n_columns * rows
    B = 4 * S2
    gbank = ev * B + ly * S2 + col * rows + rw
    order = np.argsort(gbank, kind="stable")   # keeps each base bank's shuffled order
    cols = [a[order] for a in (ev, ly, col, rw, b.truth_h[keep].astype(np.int64),
                               b.truth_flags[keep].astype(np.int64), tr[keep], y[keep], gbank)]
    ev, ly, col, rw, hv, fl, trk, yy, gbank = cols
    bank_n = np.bincount(gbank, minlength=n_events * B).astype(np.int64)
    raw, ev_off = encode(bank_n.reshape(n_events, B), hv, fl, S2)
    return GroupedBatch(gg, n_events, raw, ev_off, bank_n.astype(np.uint32), ev.astype(np.int32),
                        ly.astype(np.int8), col.astype(np.int16), rw.astype(np.int16), hv.astype(np.int16),
                        fl.astype(np.int8), trk.astype(np.int64), yy, b.velo_x, b.velo_y, b.velo_tx, b.velo_ty,
                        b.velo_flags, b.trk_off, b.qop_true)
