"""CPU oracle for UT decoding and Compass (test infrastructure).

Only the tests, the smoke check and the benchmark's CPU-baseline leg use
this package.  It is a ctypes wrapper around `oracle.c`, a plain C
statement of the method (see that file's header for the passages of the
paper each function follows), built with gcc -O2 -ffp-contract=off.
It imports nothing from the GPU package.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

ERR_NAMES = {0: "OK", -1: "ARG", -2: "DIR", -3: "HEADER", -4: "STRIP", -5: "CAPACITY", -6: "WIN16"}


def build(force: bool = False) -> str:
    """Compile oracle.c into a shared library (idempotent)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
               "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Geom(ctypes.Structure):
    _fields_ = [("S", ctypes.c_int), ("z", ctypes.c_float * 4), ("tan_a", ctypes.c_float * 4),
                ("pitch", ctypes.c_float), ("x_min", ctypes.c_float), ("z_velo", ctypes.c_float)]


class _Params(ctypes.Structure):
    _fields_ = [("n_sectors", ctypes.c_int), ("n_candidates", ctypes.c_int)] + [
        (n, ctypes.c_float) for n in ("qop_max", "tol_win", "tol_kink", "tol_col", "tol_slope",
                                      "chi2ndof_max", "sigma_hit", "sigma_x_prior",
                                      "sigma_tx_prior", "z_kink", "kick_k")] + [("gec_max_hits", ctypes.c_int)] + [
        ("kmap_nx", ctypes.c_int), ("kmap_ny", ctypes.c_int), ("kmap_tx_max", ctypes.c_float),
        ("kmap_ty_max", ctypes.c_float), ("kmap_v", ctypes.c_void_p)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            _lib.orc_decode.restype = ctypes.c_int
            _lib.orc_decode.argtypes = [P, ctypes.c_uint64, P, ctypes.c_int, ctypes.c_int, P, ctypes.c_float,
                                        ctypes.c_float, ctypes.c_int, ctypes.c_float, ctypes.c_int,
                                        ctypes.c_uint64, P, P, P, P, P, P, P, P, ctypes.c_int]
            _lib.orc_sort_hits.restype = ctypes.c_int
            _lib.orc_sort_hits.argtypes = [ctypes.c_size_t] + [P] * 12
            _lib.orc_compass.restype = ctypes.c_int
            _lib.orc_compass.argtypes = [P, P, ctypes.c_int, P, P, P, P, P, P, P, P,
                                         P, P, P, P, P, P, P, P, P, P, P, P, ctypes.c_int]
            _lib.orc_fit_tracks.restype = ctypes.c_int
            _lib.orc_fit_tracks.argtypes = [P, P, P, P, P, P, ctypes.c_uint32, P, P,
                                            P, P, P, P, P, P, P]
            _lib.orc_fit64_d.restype = ctypes.c_int
            _lib.orc_fit64_d.argtypes = [P, P, P, P, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_double, P, P]
            _lib.orc_fit32_d.restype = ctypes.c_int
            _lib.orc_fit32_d.argtypes = [P, P, P, P, ctypes.c_float, ctypes.c_float,
                                         ctypes.c_float, P]
            _lib.orc_max_threads.restype = ctypes.c_int
            _lib.orc_compass_groups.restype = ctypes.c_int
            _lib.orc_compass_groups.argtypes = [P, P, P, P, ctypes.c_int, P, ctypes.c_int, P, P, P, P, P, P, P,
                                                P, ctypes.c_float, P, P, P, P, P, P, P, P, P, ctypes.c_int]
            _lib.orc_group_candidates.restype = ctypes.c_int
            _lib.orc_group_candidates.argtypes = [P, P, P, P, ctypes.c_int, P, ctypes.c_int, P, P, P, P, P, P, P,
                                                  P, ctypes.c_float, ctypes.c_int, P, P]
            _lib.orc_extrapolate.restype = None
            _lib.orc_extrapolate.argtypes = [P, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float, P, P]
            _lib.orc_kick_at.restype = ctypes.c_float
            _lib.orc_kick_at.argtypes = [P, ctypes.c_float, ctypes.c_float]
            _lib.orc_align_chi2.restype = ctypes.c_int
            _lib.orc_align_chi2.argtypes = [P, P, P, P, ctypes.c_uint32, P, P, P, P, P, P, P, P,
                                            P, P, P, P]
            _lib.orc_align_refit.restype = ctypes.c_int
            _lib.orc_align_refit.argtypes = [P, P, P, P, ctypes.c_uint32, P, P, P, P, P, P, P, P]
        return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def max_threads() -> int:
    return int(lib().orc_max_threads())


@dataclasses.dataclass
class Hits:
    x: np.ndarray
    z: np.ndarray
    sector: np.ndarray
    layer: np.ndarray
    id: np.ndarray
    hit_off: np.ndarray

    @property
    def n(self) -> int:
        return int(self.hit_off[-1])


class OracleError(RuntimeError):
    def __init__(self, code, where):
        super().__init__(f"oracle error {ERR_NAMES.get(code, code)} at {where}")
        self.code = code
        self.where = where


def geom_struct(geom) -> _Geom:
    g = _Geom()
    g.S = int(geom.n_sectors)
    for l in range(4):
        g.z[l] = float(geom.z[l])
        g.tan_a[l] = float(geom.tan_stereo[l])
    g.pitch = float(geom.sector_pitch)
    g.x_min = float(geom.x_min)
    g.z_velo = float(geom.z_velo)
    return g


def params_struct(p, kick_map=None) -> _Params:
    """kick_map: None (the constant kick_k) or an object with nx, ny, tx_max,
    ty_max and values (float32 [ny, nx]) -- the field map of Sec. III-C."""
    s = _Params()
    for f in dataclasses.fields(p):
        setattr(s, f.name, getattr(p, f.name))
    if kick_map is not None:
        v = np.ascontiguousarray(kick_map.values, np.float32)
        assert v.shape == (kick_map.ny, kick_map.nx)
        s.kmap_nx, s.kmap_ny = int(kick_map.nx), int(kick_map.ny)
        s.kmap_tx_max, s.kmap_ty_max = float(kick_map.tx_max), float(kick_map.ty_max)
        s.kmap_v = v.ctypes.data
        s._keep = v  # the values must outlive the call
    return s


def kick_at(params, kick_map, tx, ty):
    """The kick map evaluated at track directions (tx, ty) (float32 arrays)."""
    pp = params_struct(params, kick_map)
    tx = np.asarray(tx, np.float32).ravel()
    ty = np.asarray(ty, np.float32).ravel()
    return np.array([lib().orc_kick_at(ctypes.byref(pp), ctypes.c_float(a), ctypes.c_float(b))
                     for a, b in zip(tx, ty)], np.float32)


def decode(raw, ev_off, n_events, geom, sorted_=True, capacity=None, n_threads=0,
           raise_on_error=True, n_words=None):
    """Decode a batch's raw banks (Sec. IV).  Returns (code, Hits, (event, bank))."""
    raw = np.ascontiguousarray(raw, dtype=np.uint32)
    ev_off = np.ascontiguousarray(ev_off, dtype=np.uint64)
    if capacity is None:
        capacity = 2 * int(ev_off[n_events])
    cap = max(int(capacity), 1)
    B = 4 * geom.n_sectors
    x = np.zeros(cap, np.float32)
    z = np.zeros(cap, np.float32)
    sector = np.zeros(cap, np.uint16)
    layer = np.zeros(cap, np.uint8)
    hid = np.zeros(cap, np.uint32)
    hit_off = np.zeros(n_events * B + 1, np.uint32)
    ee = np.zeros(1, np.int64)
    eb = np.zeros(1, np.int64)
    zl = np.ascontiguousarray(geom.z, dtype=np.float32)
    nwords = raw.size if n_words is None else int(n_words)
    rc = lib().orc_decode(_p(raw), nwords, _p(ev_off), n_events, geom.n_sectors, _p(zl),
                          geom.sector_pitch, geom.strip_pitch, geom.strips, geom.x_min,
                          1 if sorted_ else 0, int(capacity), _p(x), _p(z), _p(sector),
                          _p(layer), _p(hid), _p(hit_off), _p(ee), _p(eb), n_threads)
    if rc != 0 and raise_on_error:
        raise OracleError(rc, (int(ee[0]), int(eb[0])))
    n = int(hit_off[-1]) if rc == 0 else 0
    hits = Hits(x[:n], z[:n], sector[:n], layer[:n], hid[:n], hit_off)
    return rc, hits, (int(ee[0]), int(eb[0]))


def sort_hits(h: Hits):
    """Stable per-bank sort of decoded hits by half-strip (Table I permutation)."""
    n = h.n
    out = Hits(np.zeros(n, np.float32), np.zeros(n, np.float32), np.zeros(n, np.uint16),
               np.zeros(n, np.uint8), np.zeros(n, np.uint32), h.hit_off.copy())
    perm = np.zeros(n, np.uint32)
    lib().orc_sort_hits(h.hit_off.size - 1, _p(h.hit_off), _p(h.x), _p(h.z), _p(h.sector),
                        _p(h.layer), _p(h.id), _p(out.x), _p(out.z), _p(out.sector),
                        _p(out.layer), _p(out.id), _p(perm))
    return out, perm


@dataclasses.dataclass
class Tracks:
    hit: np.ndarray       # i32 [T, 4]
    qop: np.ndarray
    chi2: np.ndarray
    x: np.ndarray
    tx: np.ndarray
    nhits: np.ndarray
    found: np.ndarray
    win: np.ndarray | None
    near: np.ndarray      # min decision margin per track
    qop64: np.ndarray
    chi2_64: np.ndarray


def compass(hx, hit_off, n_events, geom, velo, params, want_windows=False, n_threads=0,
            raise_on_error=True, kick_map=None):
    """Windows + tracklet search + selection (Sec. V) for every VELO track.

    velo: object with x, y, tx, ty (f32), flags (u8), trk_off (u32[E+1]).
    kick_map: see params_struct.
    """
    hx = np.ascontiguousarray(hx, dtype=np.float32)
    hit_off = np.ascontiguousarray(hit_off, dtype=np.uint32)
    T = int(velo.trk_off[n_events])
    vx = np.ascontiguousarray(velo.x[:T], np.float32)
    vy = np.ascontiguousarray(velo.y[:T], np.float32)
    vtx = np.ascontiguousarray(velo.tx[:T], np.float32)
    vty = np.ascontiguousarray(velo.ty[:T], np.float32)
    vfl = np.ascontiguousarray(velo.flags[:T], np.uint8)
    toff = np.ascontiguousarray(velo.trk_off[: n_events + 1], np.uint32)
    Tn = max(T, 1)
    out = Tracks(np.full((Tn, 4), -1, np.int32), np.zeros(Tn, np.float32), np.zeros(Tn, np.float32),
                 np.zeros(Tn, np.float32), np.zeros(Tn, np.float32), np.zeros(Tn, np.uint8),
                 np.zeros(Tn, np.uint8),
                 np.full((Tn, 4, params.n_sectors, 2), -1, np.int16) if want_windows else None,
                 np.zeros(Tn, np.float64), np.zeros(Tn, np.float64), np.zeros(Tn, np.float64))
    g = geom_struct(geom)
    pp = params_struct(params, kick_map)
    et = np.zeros(1, np.int64)
    rc = lib().orc_compass(_p(hx), _p(hit_off), n_events, ctypes.byref(g), _p(vx), _p(vy), _p(vtx),
                           _p(vty), _p(vfl), _p(toff), ctypes.byref(pp), _p(out.hit), _p(out.qop),
                           _p(out.chi2), _p(out.x), _p(out.tx), _p(out.nhits), _p(out.found),
                           _p(out.win) if want_windows else None, _p(out.near), _p(out.qop64),
                           _p(out.chi2_64), _p(et), n_threads)
    if rc != 0 and raise_on_error:
        raise OracleError(rc, int(et[0]))
    if T == 0:
        out = Tracks(*(a[:0] if isinstance(a, np.ndarray) else a for a in dataclasses.astuple(out)))
    return out


def fit_tracks(hx, geom, velo, hit, params, kick_map=None):
    """Refit given hit sets (float and double).  Returns dict of arrays."""
    hx = np.ascontiguousarray(hx, dtype=np.float32)
    hit = np.ascontiguousarray(hit, dtype=np.int32)
    T = hit.shape[0]
    vx = np.ascontiguousarray(velo.x[:T], np.float32)
    vy = np.ascontiguousarray(velo.y[:T], np.float32)
    vtx = np.ascontiguousarray(velo.tx[:T], np.float32)
    vty = np.ascontiguousarray(velo.ty[:T], np.float32)
    o = {k: np.zeros(max(T, 1), np.float32) for k in ("qop", "chi2", "x", "tx")}
    o["ok"] = np.zeros(max(T, 1), np.uint8)
    o["qop64"] = np.zeros(max(T, 1), np.float64)
    o["chi2_64"] = np.zeros(max(T, 1), np.float64)
    g = geom_struct(geom)
    pp = params_struct(params, kick_map)
    lib().orc_fit_tracks(_p(hx), ctypes.byref(g), _p(vx), _p(vy), _p(vtx), _p(vty), T, _p(hit),
                         ctypes.byref(pp), _p(o["qop"]), _p(o["chi2"]), _p(o["x"]), _p(o["tx"]),
                         _p(o["ok"]), _p(o["qop64"]), _p(o["chi2_64"]))
    return {k: v[:T] for k, v in o.items()}


def fit64_d(d, present, t, f, w, px, ptx):
    """Double-precision p-kick least squares on explicit residuals (Sec. III-C)."""
    d = np.ascontiguousarray(d, np.float64)
    pr = np.ascontiguousarray(present, np.int32)
    t = np.ascontiguousarray(t, np.float64)
    f = np.ascontiguousarray(f, np.float64)
    delta = np.zeros(3, np.float64)
    c2 = np.zeros(1, np.float64)
    ok = lib().orc_fit64_d(_p(d), _p(pr), _p(t), _p(f), w, px, ptx, _p(delta), _p(c2))
    return bool(ok), delta, float(c2[0])


def fit32_d(d, present, t, f, w, px, ptx):
    """The float fit on explicit residuals: returns ok, (a, b, q, chi2)."""
    d = np.ascontiguousarray(d, np.float32)
    pr = np.ascontiguousarray(present, np.int32)
    t = np.ascontiguousarray(t, np.float32)
    f = np.ascontiguousarray(f, np.float32)
    out = np.zeros(4, np.float32)
    ok = lib().orc_fit32_d(_p(d), _p(pr), _p(t), _p(f), np.float32(w), np.float32(px),
                           np.float32(ptx), _p(out))
    return bool(ok), out


class Velo:
    """VELO tracks view of a synthetic batch."""

    def __init__(self, batch):
        self.x, self.y, self.tx, self.ty = batch.velo_x, batch.velo_y, batch.velo_tx, batch.velo_ty
        self.flags = batch.velo_flags
        self.trk_off = batch.trk_off


def run_batch(batch, params, n_threads=0, want_windows=False, kick_map=None):
    """Decode (sorted) + Compass for a whole batch: (Hits, Tracks)."""
    _, hits, _ = decode(batch.raw, batch.ev_off, batch.n_events, batch.geom, True, n_threads=n_threads)
    tr = compass(hits.x, hits.hit_off, batch.n_events, batch.geom, Velo(batch), params,
                 want_windows=want_windows, n_threads=n_threads, kick_map=kick_map)
    return hits, tr


def consolidate(tracks, trk_off):
    """Prefix sum and consolidation (Sec. VI): the found tracks, in (event,
    VELO track) order, and the first row of every event.  Written out by
    its definition: the found tracks' indices, and the count of found
    tracks before each event's first track."""
    found = np.asarray(tracks["found"] if isinstance(tracks, dict) else tracks.found).astype(bool)
    get = (lambda k: tracks[k]) if isinstance(tracks, dict) else (lambda k: getattr(tracks, k))
    idx = np.nonzero(found)[0]
    before = np.concatenate([[0], np.cumsum(found, dtype=np.int64)])
    out = {k: np.asarray(get(k))[idx] for k in ("hit", "qop", "chi2", "x", "tx", "nhits")}
    out["velo"] = idx.astype(np.uint32)
    return out, before[np.asarray(trk_off, np.int64)].astype(np.uint32)


def align_chi2(hits, track_hits, geom, velo, params, align, theta, grads=True):
    """Alignment chi2 (double) with its gradient with respect to the track
    states theta [T,3] = (x, tx, qop) and the per-sector alignment
    align [4S,3] = (dx, dz, gamma), and the per-sector Gauss-Newton blocks
    [4S,6].  hits: Hits (decoded, any order); track_hits [T,4] hit indices."""
    th = np.ascontiguousarray(track_hits, np.int32)
    T = th.shape[0]
    al = np.ascontiguousarray(align, np.float64)
    tt = np.ascontiguousarray(theta, np.float64)
    c2 = np.zeros(1, np.float64)
    gt = np.zeros((max(T, 1), 3), np.float64) if grads else None
    ga = np.zeros((4 * geom.n_sectors, 3), np.float64) if grads else None
    ha = np.zeros((4 * geom.n_sectors, 6), np.float64) if grads else None
    g = geom_struct(geom)
    pp = params_struct(params)
    vel = [np.ascontiguousarray(a[:T], np.float32) for a in (velo.x, velo.y, velo.tx, velo.ty)]
    lib().orc_align_chi2(_p(hits.x), _p(hits.sector), _p(hits.layer), _p(th), T, ctypes.byref(g),
                         *(_p(v) for v in vel), ctypes.byref(pp), _p(al), _p(tt), _p(c2),
                         _p(gt) if grads else None, _p(ga) if grads else None,
                         _p(ha) if grads else None)
    if not grads:
        return float(c2[0])
    return float(c2[0]), gt[:T], ga, ha


def align_refit(hits, track_hits, geom, velo, params, align):
    """Per-track refit (double) in the aligned detector: theta [T,3]."""
    th = np.ascontiguousarray(track_hits, np.int32)
    T = th.shape[0]
    out = np.zeros((max(T, 1), 3), np.float64)
    g = geom_struct(geom)
    pp = params_struct(params)
    vel = [np.ascontiguousarray(a[:T], np.float32) for a in (velo.x, velo.y, velo.tx, velo.ty)]
    lib().orc_align_refit(_p(hits.x), _p(hits.sector), _p(hits.layer), _p(th), T, ctypes.byref(g),
                          *(_p(v) for v in vel), ctypes.byref(pp), _p(np.ascontiguousarray(align, np.float64)),
                          _p(out))
    return out[:T]


@dataclasses.dataclass
class GroupHits:
    """Hits of the sector-group decoding, in output order (event, layer,
    group, then yBegin, then raw order)."""
    x: np.ndarray         # f32, x at y = 0
    z: np.ndarray         # f32, z of the plane
    y_begin: np.ndarray   # f32
    y_end: np.ndarray     # f32
    weight: np.ndarray    # f32, 1 / sigma^2 of the position
    id: np.ndarray        # u32, (layer << 24) | (sensor << 16) | word
    group_off: np.ndarray  # u32[E * 4 * n_groups + 1]
    src: np.ndarray       # i64, index of each output hit in the bank-order decode


def decode_groups(raw, ev_off, n_events, gg, n_threads=0):
    """Sector-group decoding (Sec. IV; Table I's pre-decode, find permutation
    and decode-in-order kernels): every hit's x at y = 0 and z, its strip's
    y range [yBegin, yEnd] (its sensor's rows), its weight, and its sector
    group (the x region holding x); hits stored by (event, layer, group)
    with offsets, sorted by yBegin inside a group (stable: ties keep the raw
    order).  `gg`: synth.grouped.GroupGeometry.  The raw banks are checked
    and read by the bank-order decode (one sector per sensor); the rest is
    written out here in float32, each operation as stated."""
    rg = gg.raw_geometry()
    code, h, where = decode(raw, ev_off, n_events, rg, sorted_=False, n_threads=n_threads)
    if code != 0:
        raise OracleError(code, where)
    n = int(h.n)
    ids = h.id[:n].astype(np.int64)
    R = int(gg.rows)
    S2 = int(gg.n_columns) * R
    NG = int(gg.n_groups)
    layer = ids >> 24
    sensor = (ids >> 16) & 0xFF
    word = ids & 0xFFFF
    col = sensor // R
    row = sensor % R
    half = 2 * (word & 0x3FF) + ((word >> 10) & 1)
    f32 = np.float32
    # x at y = 0 (as the base decode, per column): x0 = c * pitch + x_min; x = x0 + (h + 1/2) * (pitch/2)
    x0 = col.astype(f32) * f32(gg.base.sector_pitch) + f32(gg.x_min)
    hp = f32(gg.base.strip_pitch) * f32(0.5)
    x = x0 + (half.astype(f32) + f32(0.5)) * hp
    z = np.asarray(gg.base.z, f32)[layer]
    H = f32(gg.sensor_height)
    yb = f32(gg.y_min) + row.astype(f32) * H
    ye = yb + H
    sig = f32(np.float64(f32(gg.base.strip_pitch)) / np.sqrt(12.0))   # the float pitch, / sqrt(12) in double
    w = np.full(n, f32(1.0) / (sig * sig), f32)
    edges = gg.group_edges()
    grp = np.searchsorted(edges[1:-1], x, side="right").astype(np.int64)   # interior edges <= x
    B = 4 * S2
    bank_first = h.hit_off[: n_events * B : B].astype(np.int64)           # first hit of each event
    event = np.searchsorted(bank_first, np.arange(n), side="right") - 1 if n else np.zeros(0, np.int64)
    order = np.lexsort((np.arange(n), yb, grp, layer, event))
    cell = (event * 4 + layer) * NG + grp
    counts = np.bincount(cell, minlength=n_events * 4 * NG)
    goff = np.zeros(n_events * 4 * NG + 1, np.int64)
    goff[1:] = np.cumsum(counts)
    return GroupHits(x[order], z[order], yb[order], ye[order], w[order], h.id[:n][order],
                     goff.astype(np.uint32), order.astype(np.int64))


def compass_groups(gh, batch, params, tol_y=10.0, kick_map=None, n_threads=0, vy=None, vty=None):
    """Compass on the sector-group layout (row f2; orc_compass_groups):
    windows over groups with y windows by two binary searches, then the
    same tracklet search and selection.  gh: GroupHits of decode_groups;
    batch: synth.grouped.GroupedBatch (its VELO tracks; vy, vty optionally
    replace their y and ty).  Hit indices refer to gh's output order."""
    gg = batch.geom
    E = batch.n_events
    T = int(batch.trk_off[E])
    geo = geom_struct(gg.base)
    pp = params_struct(params, kick_map)
    edges = np.ascontiguousarray(gg.group_edges(), np.float32)
    vy = batch.velo_y if vy is None else vy
    vty = batch.velo_ty if vty is None else vty
    v = [np.ascontiguousarray(a[:T], np.float32) for a in (batch.velo_x, vy, batch.velo_tx, vty)]
    vfl = np.ascontiguousarray(batch.velo_flags[:T], np.uint8)
    toff = np.ascontiguousarray(batch.trk_off[: E + 1], np.uint32)
    Tn = max(T, 1)
    out = Tracks(np.full((Tn, 4), -1, np.int32), np.zeros(Tn, np.float32), np.zeros(Tn, np.float32),
                 np.zeros(Tn, np.float32), np.zeros(Tn, np.float32), np.zeros(Tn, np.uint8), np.zeros(Tn, np.uint8),
                 None, np.zeros(Tn, np.float64), np.zeros(Tn, np.float64), np.zeros(Tn, np.float64))
    gx = np.ascontiguousarray(gh.x, np.float32)
    gyb = np.ascontiguousarray(gh.y_begin, np.float32)
    gye = np.ascontiguousarray(gh.y_end, np.float32)
    goff = np.ascontiguousarray(gh.group_off, np.uint32)
    rc = lib().orc_compass_groups(_p(gx), _p(gyb), _p(gye), _p(goff), E, ctypes.byref(geo), int(gg.n_groups),
                                  _p(edges), _p(v[0]), _p(v[1]), _p(v[2]), _p(v[3]), _p(vfl), _p(toff),
                                  ctypes.byref(pp), float(tol_y), _p(out.hit), _p(out.qop), _p(out.chi2),
                                  _p(out.x), _p(out.tx), _p(out.nhits), _p(out.found), _p(out.near),
                                  _p(out.qop64), n_threads)
    if rc != 0:
        raise OracleError(rc, -1)
    if T == 0:
        out = Tracks(*(a[:0] if isinstance(a, np.ndarray) else a for a in dataclasses.astuple(out)))
    return out


def group_candidates(gh, batch, params, tol_y=10.0, kick_map=None, max_cand=4096, vy=None, vty=None):
    """The candidates of every track of the group search
    (orc_group_candidates): int32 [T, 4, max_cand] group-layout indices in
    the search's order and int32 [T, 4] counts.  vy, vty (optional) replace
    the batch's VELO y and ty."""
    gg = batch.geom
    E = batch.n_events
    T = int(batch.trk_off[E])
    geo = geom_struct(gg.base)
    pp = params_struct(params, kick_map)
    edges = np.ascontiguousarray(gg.group_edges(), np.float32)
    vy = batch.velo_y if vy is None else vy
    vty = batch.velo_ty if vty is None else vty
    v = [np.ascontiguousarray(a[:T], np.float32) for a in (batch.velo_x, vy, batch.velo_tx, vty)]
    vfl = np.ascontiguousarray(batch.velo_flags[:T], np.uint8)
    toff = np.ascontiguousarray(batch.trk_off[: E + 1], np.uint32)
    cand = np.full((max(T, 1), 4, max_cand), -1, np.int32)
    n = np.zeros((max(T, 1), 4), np.int32)
    rc = lib().orc_group_candidates(_p(np.ascontiguousarray(gh.x, np.float32)),
                                    _p(np.ascontiguousarray(gh.y_begin, np.float32)),
                                    _p(np.ascontiguousarray(gh.y_end, np.float32)),
                                    _p(np.ascontiguousarray(gh.group_off, np.uint32)), E, ctypes.byref(geo),
                                    int(gg.n_groups), _p(edges), _p(v[0]), _p(v[1]), _p(v[2]), _p(v[3]), _p(vfl),
                                    _p(toff), ctypes.byref(pp), float(tol_y), int(max_cand), _p(cand), _p(n))
    if rc != 0:
        raise OracleError(rc, -1)
    return cand[:T], n[:T]


def extrapolate(geom, vx, vy, vtx, vty):
    """The oracle's prediction of a VELO track in the four layers
    (orc_extrapolate): float32 arrays hi[4], lo[4]."""
    g = geom_struct(geom)
    hi = np.zeros(4, np.float32)
    lo = np.zeros(4, np.float32)
    lib().orc_extrapolate(ctypes.byref(g), ctypes.c_float(vx), ctypes.c_float(vy), ctypes.c_float(vtx),
                          ctypes.c_float(vty), _p(hi), _p(lo))
    return hi, lo
