"""Seeded synthetic UT events: VELO tracks, UT hits and their raw banks.

This module is the input generator that the CUDA path, the oracle, the tests
and the benchmark all share.  It simulates a detector and encodes raw data;
it holds none of the decoding or tracking arithmetic of the method.

Detector (the four UT planes UTaX, UTaU, UTbV, UTbX of Sec. III-A; the z
positions and the sector tiling are synthetic stand-ins, the paper gives
neither):

* plane l at z_l = 2327 / 2372 / 2597 / 2642 mm, strip stereo angle
  0 / +5 / -5 / 0 degrees.  A strip of plane l is the line x = u + y*tan(a_l);
  u is the coordinate the plane measures ("x at y = 0", Sec. IV).
* each plane is tiled along u by S sectors, 96 mm wide, starting at
  x_min = -S*96/2.  Sector s carries 512 strips of 0.187 mm pitch starting at
  its left edge; a hit records the half-strip index h = 2*strip + frac.

Trajectories (the magnet kick as a kink, Sec. III-C): a VELO track is a
straight line given at z = 770 mm by (x, y, tx, ty); in the UT the true
position is x(z) = x + tx*(z-770) + 1.2*qop*(z-2500), y(z) = y + ty*(z-770),
with qop = charge/p in 1/GeV.  With `field_fn` (the "fieldmap" workload)
the kick 1.2 is replaced by field_fn(tx, ty), a direction-dependent field
integral (`field_kick`); the tracking is given that field only as a map
sampled on a grid (`kick_map`), as the paper's look-up tables.

Raw bank layout (the paper calls it a "highly compact format" without a bit
layout; this layout is this project's):

* an event is a run of u32 words: first a directory dir[B] (B = 4*S banks,
  bank b = l*S + s), each entry the word offset of bank b's header counted
  from the event's first word; then the banks in order b = 0..B-1;
* a bank is a header word (bits 0-15: hit count n, bits 16-31: source id b)
  followed by n 16-bit hit words packed two per u32, low half first, with a
  zero half-word of padding when n is odd;
* a hit word holds strip (bits 0-9), frac (bit 10) and 5 flag bits (11-15).

`ev_off[e]` is the u32 word offset of event e in the batch's raw buffer; the
buffer is padded with zero words to a multiple of 4 words (16 bytes).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

Z_LAYERS = (2327.0, 2372.0, 2597.0, 2642.0)
STEREO_DEG = (0.0, 5.0, -5.0, 0.0)
SECTOR_PITCH = 96.0
STRIP_PITCH = 0.187
N_STRIPS = 512
Z_VELO = 770.0
Z_KINK = 2500.0
KICK_K = 1.2           # mm of x per mm of z per GeV^-1 (1.2e3 mm*GeV/1000)


def field_kick(tx, ty) -> np.ndarray:
    """Kick of the synthetic magnet per unit q/p (mm of x per mm of z per
    GeV^-1) for a track of direction (tx, ty): KICK_K scaled by a smooth
    field integral, larger for tracks at large |ty| and smaller at large |tx|
    (up to +40 % and -20 % over the VELO acceptance).  A property of the
    simulated detector; the tracking only sees it sampled by `kick_map`."""
    tx = np.asarray(tx, np.float64)
    ty = np.asarray(ty, np.float64)
    return KICK_K * (1.0 + 0.4 * (ty / 0.25) ** 2) * (1.0 - 0.2 * (tx / 0.3) ** 2)


@dataclasses.dataclass
class KickMap:
    """A field map of the kick: values[j, i] is the kick at tx_i = -tx_max +
    i * 2 tx_max / (nx - 1), ty_j = -ty_max + j * 2 ty_max / (ny - 1)."""
    nx: int
    ny: int
    tx_max: float
    ty_max: float
    values: np.ndarray  # float32 [ny, nx]


def kick_map(nx: int = 17, ny: int = 17, tx_max: float = 0.3, ty_max: float = 0.25, fn=None) -> KickMap:
    """`fn` (default field_kick) sampled on the grid, rounded to float32."""
    fn = field_kick if fn is None else fn
    tx = -tx_max + np.arange(nx, dtype=np.float64) * (2.0 * tx_max / (nx - 1))
    ty = -ty_max + np.arange(ny, dtype=np.float64) * (2.0 * ty_max / (ny - 1))
    v = fn(tx[None, :], ty[:, None]).astype(np.float32)
    return KickMap(nx, ny, tx_max, ty_max, np.ascontiguousarray(v))


def tan_stereo_f32() -> np.ndarray:
    """tan of the four stereo angles, rounded to float32 (geometry constants)."""
    return np.tan(np.deg2rad(np.asarray(STEREO_DEG, dtype=np.float64))).astype(np.float32)


@dataclasses.dataclass
class Geometry:
    n_sectors: int
    z: np.ndarray = dataclasses.field(default_factory=lambda: np.asarray(Z_LAYERS, np.float32))
    tan_stereo: np.ndarray = dataclasses.field(default_factory=tan_stereo_f32)
    sector_pitch: float = SECTOR_PITCH
    strip_pitch: float = STRIP_PITCH
    strips: int = N_STRIPS
    z_velo: float = Z_VELO

    @property
    def x_min(self) -> float:
        return float(np.float32(-self.n_sectors * self.sector_pitch / 2.0))

    @property
    def n_banks(self) -> int:
        return 4 * self.n_sectors


@dataclasses.dataclass
class Batch:
    """One batch of events.

    raw        u32[n_words]   all events' raw data (layout in the module doc)
    ev_off     u64[E+1]       event start offsets in u32 words
    velo_*     f32[T_total]   VELO state at z=770 for all tracks, event-major
    velo_flags u8[T_total]    bit 0 = backward
    trk_off    u32[E+1]       track offsets per event
    truth_*    per raw hit word, in raw (bank) order: event, layer, sector,
               half-strip h, flags and the generating track (-1 = noise,
               else the global track index)
    qop_true   f32[T_total]   generating charge/p of each track
    """
    geom: Geometry
    n_events: int
    raw: np.ndarray
    ev_off: np.ndarray
    velo_x: np.ndarray
    velo_y: np.ndarray
    velo_tx: np.ndarray
    velo_ty: np.ndarray
    velo_flags: np.ndarray
    trk_off: np.ndarray
    qop_true: np.ndarray
    bank_n: np.ndarray          # u32[E*B] hits per bank
    truth_event: np.ndarray
    truth_layer: np.ndarray
    truth_sector: np.ndarray
    truth_h: np.ndarray
    truth_flags: np.ndarray
    truth_track: np.ndarray

    @property
    def n_tracks(self) -> int:
        return int(self.trk_off[-1])

    @property
    def n_hits(self) -> int:
        return int(self.bank_n.sum())


# Named workloads (the paper's LHCb minbias samples are not available; these
# seeded synthetic sets stand in for them).
CONFIGS = {
    "tiny": dict(n_events=16, n_sectors=64, tracks=100, hits=1500, seed=1),
    "plain": dict(n_events=1000, n_sectors=256, tracks=200, hits=4000, seed=2),
    "batched": dict(n_events=20000, n_sectors=256, tracks=None, hits="lognormal", seed=3),
    # the plain workload's shapes, hits made with the direction-dependent field
    "fieldmap": dict(n_events=1000, n_sectors=256, tracks=200, hits=4000, seed=6, field_fn=field_kick),
}


def _event_sizes(rng, n_events, tracks, hits):
    if hits == "lognormal":
        h = np.exp(rng.normal(math.log(3000.0), 0.6, size=n_events))
        h = np.clip(np.rint(h), 500, 15000).astype(np.int64)
        t = np.maximum(np.rint(0.05 * h), 1).astype(np.int64)
        return t, h
    t = np.full(n_events, int(tracks), dtype=np.int64)
    if hits is None:
        return t, None
    return t, np.full(n_events, int(hits), dtype=np.int64)


def generate(n_events: int, n_sectors: int, tracks=100, hits=1500, seed: int = 1,
             noise_frac: float | None = None, efficiency: float = 0.95,
             backward_frac: float = 0.0, field: float = KICK_K,
             smear: bool = True, plane_covering: bool = False,
             p_range=(1.5, 100.0), flags_random: bool = True, misalign=None, field_fn=None) -> Batch:
    """Generate a seeded batch.

    hits: target hits per event (noise = target - signal, at least 0), or
    "lognormal" (median 3000, sigma_ln 0.6, clipped to [500, 15000], with
    tracks = round(0.05*hits)), or None together with noise_frac (noise hits
    = noise_frac/(1-noise_frac) * signal hits).
    field: kick constant used to make the hits (0 gives straight tracks).
    field_fn: optional f(tx, ty) -> kick per track (float64), replacing field.
    plane_covering: VELO x at z=770 drawn so that the tracks cover the plane
    (used by the alignment workload) instead of coming from the beam line.
    misalign: optional (dx, dz, gamma), each [4, S]: sector (l, s) sits at
    z_l + dz, shifted by dx along x and its strips rotated by gamma in the
    plane (strip line x = u + dx + y tan(a_l + gamma)).
    """
    geom = Geometry(n_sectors=n_sectors)
    rng = np.random.Generator(np.random.Philox(key=seed))
    S = n_sectors
    B = 4 * S
    n_trk, n_target = _event_sizes(rng, n_events, tracks, hits)
    T = int(n_trk.sum())
    trk_off = np.zeros(n_events + 1, dtype=np.uint32)
    trk_off[1:] = np.cumsum(n_trk)
    trk_event = np.repeat(np.arange(n_events), n_trk)

    # VELO states at z = 770 mm.
    tx = rng.uniform(-0.3, 0.3, T)
    ty = rng.uniform(-0.25, 0.25, T)
    charge = np.where(rng.random(T) < 0.5, -1.0, 1.0)
    lp = rng.uniform(math.log(p_range[0]), math.log(p_range[1]), T)
    qop = charge / np.exp(lp)
    x_pv = rng.normal(0.0, 0.05, T)
    y_pv = rng.normal(0.0, 0.05, T)
    if plane_covering:
        half = -geom.x_min
        # x at z=770 such that the straight line at z_0 covers the plane.
        x = rng.uniform(-half, half, T) - tx * (Z_LAYERS[0] - Z_VELO)
        x = x + 0.0 * x_pv
    else:
        x = x_pv + Z_VELO * tx
    y = y_pv + Z_VELO * ty
    backward = rng.random(T) < backward_frac
    # the state is stored in float32; the hits are made from those values
    vx = x.astype(np.float32)
    vy = y.astype(np.float32)
    vtx = tx.astype(np.float32)
    vty = ty.astype(np.float32)
    qop32 = qop.astype(np.float32)
    kick = (np.full(T, float(field)) if field_fn is None
            else np.asarray(field_fn(vtx.astype(np.float64), vty.astype(np.float64)), np.float64))

    z = np.asarray(Z_LAYERS, dtype=np.float64)
    tan_a = tan_stereo_f32().astype(np.float64)
    sigma = STRIP_PITCH / math.sqrt(12.0)
    x_min = geom.x_min
    half_pitch = STRIP_PITCH / 2.0
    active = N_STRIPS * STRIP_PITCH

    # Signal hits: one per (track, layer) with probability `efficiency`.
    tl_t = np.repeat(np.arange(T), 4)
    tl_l = np.tile(np.arange(4), T)
    keep = rng.random(4 * T) < efficiency
    smear_v = rng.normal(0.0, sigma, 4 * T) if smear else np.zeros(4 * T)
    flag_v = rng.integers(0, 32, 4 * T) if flags_random else np.zeros(4 * T, np.int64)
    def measure(zz, dxs, gam):
        dz = zz - Z_VELO
        xt = vx[tl_t].astype(np.float64) + vtx[tl_t] * dz + kick[tl_t] * qop32[tl_t].astype(np.float64) * (zz - Z_KINK)
        yt = vy[tl_t].astype(np.float64) + vty[tl_t] * dz
        ta = (tan_a[tl_l] + np.tan(gam)) / (1.0 - tan_a[tl_l] * np.tan(gam))
        return xt - dxs - yt * ta + smear_v

    zz = z[tl_l]
    u = measure(zz, 0.0, 0.0)
    sec = np.floor((u - x_min) / SECTOR_PITCH).astype(np.int64)
    if misalign is not None:
        mdx, mdz, mg = (np.asarray(a, np.float64) for a in misalign)
        for _ in range(2):   # the sector crossed depends on the sector's own offsets
            sc = np.clip(sec, 0, S - 1)
            u = measure(zz + mdz[tl_l, sc], mdx[tl_l, sc], mg[tl_l, sc])
            sec = np.floor((u - x_min) / SECTOR_PITCH).astype(np.int64)
    inside = (sec >= 0) & (sec < S)
    loc = u - (x_min + SECTOR_PITCH * np.clip(sec, 0, S - 1))
    inside &= (loc >= 0.0) & (loc < active)
    keep &= inside & ~backward[tl_t]
    hh = np.clip(np.floor(loc / half_pitch), 0, 2 * N_STRIPS - 1).astype(np.int64)
    sig_event = trk_event[tl_t[keep]]
    sig_layer = tl_l[keep]
    sig_sector = sec[keep]
    sig_h = hh[keep]
    sig_flags = flag_v[keep]
    sig_track = tl_t[keep]

    # Noise hits, uniform over (layer, sector, h).
    sig_count = np.bincount(sig_event, minlength=n_events)
    if n_target is not None:
        n_noise = np.maximum(n_target - sig_count, 0)
    else:
        nf = 0.3 if noise_frac is None else float(noise_frac)
        n_noise = np.rint(sig_count * nf / (1.0 - nf)).astype(np.int64)
    NN = int(n_noise.sum())
    nz_event = np.repeat(np.arange(n_events), n_noise)
    nz_layer = rng.integers(0, 4, NN)
    nz_sector = rng.integers(0, S, NN)
    nz_h = rng.integers(0, 2 * N_STRIPS, NN)
    nz_flags = rng.integers(0, 32, NN) if flags_random else np.zeros(NN, np.int64)

    ev = np.concatenate([sig_event, nz_event]).astype(np.int64)
    ly = np.concatenate([sig_layer, nz_layer]).astype(np.int64)
    sc = np.concatenate([sig_sector, nz_sector]).astype(np.int64)
    hv = np.concatenate([sig_h, nz_h]).astype(np.int64)
    fl = np.concatenate([sig_flags, nz_flags]).astype(np.int64)
    tr = np.concatenate([sig_track, np.full(NN, -1)]).astype(np.int64)

    # Order: by (event, bank), shuffled inside each bank.
    gbank = ev * B + ly * S + sc
    key = (gbank << 32) | rng.integers(0, 1 << 32, gbank.size, dtype=np.int64)
    order = np.argsort(key, kind="stable")
    ev, ly, sc, hv, fl, tr, gbank = (a[order] for a in (ev, ly, sc, hv, fl, tr, gbank))

    bank_n = np.bincount(gbank, minlength=n_events * B).astype(np.int64)
    raw, ev_off = encode(bank_n.reshape(n_events, B), hv, fl, S)
    return Batch(
        geom=geom, n_events=n_events, raw=raw, ev_off=ev_off,
        velo_x=vx, velo_y=vy, velo_tx=vtx, velo_ty=vty,
        velo_flags=backward.astype(np.uint8), trk_off=trk_off, qop_true=qop32,
        bank_n=bank_n.astype(np.uint32),
        truth_event=ev.astype(np.int32), truth_layer=ly.astype(np.int8),
        truth_sector=sc.astype(np.int16), truth_h=hv.astype(np.int16),
        truth_flags=fl.astype(np.int8), truth_track=tr.astype(np.int64))


def encode(bank_n: np.ndarray, h: np.ndarray, flags: np.ndarray, n_sectors: int):
    """Pack hits (already in (event, bank) order) into raw banks.

    bank_n: [E, B] hit counts; h, flags: per hit.  Returns (raw u32, ev_off u64).
    """
    E, B = bank_n.shape
    bank_words = 1 + (bank_n + 1) // 2                      # header + packed words
    ev_words = B + bank_words.sum(axis=1)
    ev_off = np.zeros(E + 1, dtype=np.uint64)
    ev_off[1:] = np.cumsum(ev_words)
    n_words = int(ev_off[-1])
    n_words_pad = (n_words + 3) // 4 * 4
    raw = np.zeros(n_words_pad, dtype=np.uint32)
    # directory: offset of each bank header within the event
    dirs = B + np.concatenate([np.zeros((E, 1), np.int64), np.cumsum(bank_words, axis=1)[:, :-1]], axis=1)
    ev_start = ev_off[:-1].astype(np.int64)
    didx = (ev_start[:, None] + np.arange(B)[None, :]).ravel()
    raw[didx] = dirs.ravel().astype(np.uint32)
    hdr_pos = (ev_start[:, None] + dirs).ravel()
    src = np.tile(np.arange(B, dtype=np.int64), E)
    nflat = bank_n.ravel()
    raw[hdr_pos] = (nflat | (src << 16)).astype(np.uint32)
    # hit words
    nh = int(nflat.sum())
    if nh:
        first = np.zeros(nflat.size, np.int64)
        first[1:] = np.cumsum(nflat)[:-1]
        bank_of_hit = np.repeat(np.arange(nflat.size), nflat)
        k = np.arange(nh) - first[bank_of_hit]
        half_idx = 2 * (hdr_pos[bank_of_hit] + 1) + k
        words = ((h >> 1) & 0x3FF) | ((h & 1) << 10) | ((flags & 0x1F) << 11)
        raw16 = raw.view("<u2")
        raw16[half_idx] = words.astype(np.uint16)
    return raw, ev_off


def generate_config(name: str, n_events: int | None = None, **kw) -> Batch:
    """Generate one of the named workloads ("tiny", "plain", "batched")."""
    c = dict(CONFIGS[name])
    if n_events is not None:
        c["n_events"] = n_events
    c.update(kw)
    return generate(**c)


def subset(b: Batch, e0: int, e1: int) -> Batch:
    """Events [e0, e1) of a batch as a batch of their own (raw re-based)."""
    w0, w1 = int(b.ev_off[e0]), int(b.ev_off[e1])
    nw = w1 - w0
    raw = np.zeros((nw + 3) // 4 * 4, np.uint32)
    raw[:nw] = b.raw[w0:w1]
    t0, t1 = int(b.trk_off[e0]), int(b.trk_off[e1])
    B = b.geom.n_banks
    hb = b.bank_n[: e0 * B].sum(dtype=np.int64)
    he = hb + b.bank_n[e0 * B: e1 * B].sum(dtype=np.int64)
    tsl = slice(int(hb), int(he))
    tt = b.truth_track[tsl].copy()
    tt[tt >= 0] -= t0
    return Batch(
        geom=b.geom, n_events=e1 - e0, raw=raw, ev_off=(b.ev_off[e0:e1 + 1] - b.ev_off[e0]),
        velo_x=b.velo_x[t0:t1], velo_y=b.velo_y[t0:t1], velo_tx=b.velo_tx[t0:t1],
        velo_ty=b.velo_ty[t0:t1], velo_flags=b.velo_flags[t0:t1],
        trk_off=(b.trk_off[e0:e1 + 1] - b.trk_off[e0]), qop_true=b.qop_true[t0:t1],
        bank_n=b.bank_n[e0 * B: e1 * B], truth_event=b.truth_event[tsl] - e0,
        truth_layer=b.truth_layer[tsl], truth_sector=b.truth_sector[tsl],
        truth_h=b.truth_h[tsl], truth_flags=b.truth_flags[tsl], truth_track=tt)


@dataclasses.dataclass
class AlignmentSet:
    """Tracks with 3 or 4 true hits in a misaligned detector.

    batch holds the raw banks of all generated tracks; the alignment tracks
    are the first n_tracks generated tracks with at least 3 hits, given by
    their VELO state and the raw-order index of their hit in each layer."""
    batch: Batch
    dx: np.ndarray          # [4, S] injected offsets (mm)
    dz: np.ndarray          # [4, S] (mm)
    gamma: np.ndarray       # [4, S] in-plane rotation (rad)
    track_hits: np.ndarray  # [T, 4] raw-order hit index per layer, -1 none
    x: np.ndarray           # [T] VELO state of the alignment tracks
    y: np.ndarray
    tx: np.ndarray
    ty: np.ndarray
    qop_true: np.ndarray

    @property
    def n_tracks(self) -> int:
        return int(self.track_hits.shape[0])

    def align_true(self) -> np.ndarray:
        """[4S, 3] (dx, dz, gamma) per global sector l*S + s."""
        return np.stack([self.dx.ravel(), self.dz.ravel(), self.gamma.ravel()], 1)


def generate_alignment(n_tracks: int = 100_000, n_sectors: int = 256, seed: int = 4,
                       sigmas=(0.05, 0.2, 1e-4), tracks_per_event: int = 1000,
                       plane_covering: bool = True) -> AlignmentSet:
    """Misaligned-detector workload: per-sector (dx, dz, gamma) drawn from
    N(0, sigmas); noise-free events of plane-covering tracks; the selected
    hits of each track are its generated hits (held fixed)."""
    rng = np.random.Generator(np.random.Philox(key=seed + 7919))
    dx = rng.normal(0.0, sigmas[0], (4, n_sectors))
    dz = rng.normal(0.0, sigmas[1], (4, n_sectors))
    gm = rng.normal(0.0, sigmas[2], (4, n_sectors))
    n_gen = int(n_tracks / 0.95) + tracks_per_event
    n_events = max(1, (n_gen + tracks_per_event - 1) // tracks_per_event)
    b = generate(n_events=n_events, n_sectors=n_sectors, tracks=tracks_per_event, hits=None,
                 noise_frac=0.0, seed=seed, plane_covering=plane_covering,
                 misalign=(dx, dz, gm))
    T = b.n_tracks
    th = np.full((T, 4), -1, np.int64)
    idx = np.nonzero(b.truth_track >= 0)[0]
    th[b.truth_track[idx], b.truth_layer[idx].astype(np.int64)] = idx
    keep = np.nonzero((th >= 0).sum(axis=1) >= 3)[0][:n_tracks]
    return AlignmentSet(b, dx, dz, gm, th[keep].astype(np.int32), b.velo_x[keep], b.velo_y[keep],
                        b.velo_tx[keep], b.velo_ty[keep], b.qop_true[keep])
