"""GB300-native UT raw-bank decoding and Compass track following.

Thin Python binding of the C ABI in include/ut_compass.h: it marshals torch
device tensors into the ABI structs and calls the CUDA library; every step
of the computation runs in the library's kernels.  PyTorch provides device
memory and streams only.  The library must be built first
(`paper_2002_11529_gb300.build.build()`); without it every call raises.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import threading

import numpy as np
import torch

from . import build as _build

UT_OK, UT_ERR_ARG, UT_ERR_DIR, UT_ERR_HEADER, UT_ERR_STRIP = 0, -1, -2, -3, -4
UT_ERR_CAPACITY, UT_ERR_WIN16, UT_ERR_TIMEOUT, UT_ERR_CUDA, UT_ERR_BOUNDS = -5, -6, -7, -8, -9
ERR_NAMES = {0: "OK", -1: "ARG", -2: "DIR", -3: "HEADER", -4: "STRIP", -5: "CAPACITY",
             -6: "WIN16", -7: "TIMEOUT", -8: "CUDA", -9: "BOUNDS"}

EXPORTS = ("ut_ctx_create", "ut_ctx_destroy", "ut_ctx_set_kick_map", "ut_ctx_set_wait_limit",
           "ut_ctx_set_first_ticket", "ut_status", "ut_status_reset",
           "ut_decode_workspace_size", "ut_decode", "ut_sort_hits", "compass_find", "compass_fit",
           "ut_decode_noalloc", "ut_run_batched", "ut_align_workspace_size", "ut_align_chi2",
           "ut_align_refit", "ut_align_hvp", "ut_align_solve_workspace_size", "ut_align_solve",
           "ut_consolidate_workspace_size", "ut_consolidate",
           "ut_sector_groups", "compass_find_groups")


class UtGeometry(ctypes.Structure):
    _fields_ = [("n_sectors", ctypes.c_int), ("z", ctypes.c_float * 4),
                ("tan_stereo", ctypes.c_float * 4), ("sector_pitch", ctypes.c_float),
                ("strip_pitch", ctypes.c_float), ("strips", ctypes.c_int),
                ("x_min", ctypes.c_float), ("z_velo", ctypes.c_float)]


class UtHits(ctypes.Structure):
    _fields_ = [("x", ctypes.c_void_p), ("z", ctypes.c_void_p), ("sector", ctypes.c_void_p),
                ("layer", ctypes.c_void_p), ("id", ctypes.c_void_p), ("hit_off", ctypes.c_void_p),
                ("capacity", ctypes.c_uint32)]


class UtGroupGeometry(ctypes.Structure):
    _fields_ = [("n_columns", ctypes.c_int), ("rows", ctypes.c_int), ("n_groups", ctypes.c_int),
                ("sector_pitch", ctypes.c_float), ("strip_pitch", ctypes.c_float), ("x_min", ctypes.c_float),
                ("y_min", ctypes.c_float), ("sensor_height", ctypes.c_float), ("z", ctypes.c_float * 4),
                ("edges", ctypes.c_float * 129)]


class UtGroupHits(ctypes.Structure):
    _fields_ = [(n, ctypes.c_void_p) for n in ("x", "z", "y_begin", "y_end", "weight", "id", "group_off")] + [
        ("capacity", ctypes.c_uint32)]


class VeloTracks(ctypes.Structure):
    _fields_ = [(n, ctypes.c_void_p) for n in ("x", "y", "tx", "ty", "flags", "trk_off")]


class CompassParamsC(ctypes.Structure):
    _fields_ = [("n_sectors", ctypes.c_int), ("n_candidates", ctypes.c_int)] + [
        (n, ctypes.c_float) for n in ("qop_max", "tol_win", "tol_kink", "tol_col", "tol_slope",
                                      "chi2ndof_max", "sigma_hit", "sigma_x_prior",
                                      "sigma_tx_prior", "z_kink", "kick_k")] + [("gec_max_hits", ctypes.c_int),
                                                                                ("output_order", ctypes.c_int)]


class CompassTracksC(ctypes.Structure):
    _fields_ = [(n, ctypes.c_void_p) for n in ("hit", "qop", "chi2", "x", "tx", "nhits", "found", "velo",
                                               "n_found")]


class UtTracksCompactC(ctypes.Structure):
    _fields_ = [(n, ctypes.c_void_p) for n in ("hit", "qop", "chi2", "x", "tx", "nhits", "velo")] + [
        ("capacity", ctypes.c_uint32)]


class LaunchConfigC(ctypes.Structure):
    _fields_ = [("tracks_per_warp", ctypes.c_int), ("block", ctypes.c_int), ("x_cap", ctypes.c_int),
                ("stage_words", ctypes.c_int)]


@dataclasses.dataclass(frozen=True)
class LaunchConfig:
    """Launch shape of the batched form (0 = library default)."""
    tracks_per_warp: int = 4
    block: int = 256
    x_cap: int = 8192
    stage_words: int = 8192

    def struct(self) -> LaunchConfigC:
        return LaunchConfigC(self.tracks_per_warp, self.block, self.x_cap, self.stage_words)


_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.lib_path()


def lib():
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.lib_path()
            if not os.path.exists(path):
                raise RuntimeError(f"CUDA library not built ({path}); run paper_2002_11529_gb300.build.build()")
            L = ctypes.CDLL(path)
            P, I, U32, U64, SZ = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_size_t
            sig = {
                "ut_ctx_create": ([P, P], I),
                "ut_ctx_destroy": ([P], I),
                "ut_ctx_set_kick_map": ([P, I, I, ctypes.c_float, ctypes.c_float, P], I),
                "ut_ctx_set_wait_limit": ([P, ctypes.c_longlong], I),
                "ut_ctx_set_first_ticket": ([P, I], I),
                "ut_status": ([P, P, P, P, P], I),
                "ut_status_reset": ([P, P], I),
                "ut_decode_workspace_size": ([I], SZ),
                "ut_decode": ([P, P, U64, P, I, P, I, P, SZ, P], I),
                "ut_sort_hits": ([P, P, P, P, I, P], I),
                "compass_find": ([P, P, P, I, U32, P, P, P, I, I, P], I),
                "compass_fit": ([P, P, P, U32, P, P, P], I),
                "ut_decode_noalloc": ([P, P, U64, P, I, P, I, P, P], I),
                "ut_run_batched": ([P, P, U64, P, I, P, U32, P, P, P, P, P, SZ, P], I),
                "ut_align_workspace_size": ([I], SZ),
                "ut_consolidate_workspace_size": ([I], SZ),
                "ut_consolidate": ([P, P, I, P, P, P, P, SZ, P], I),
                "ut_sector_groups": ([P, P, I, P, P, P], I),
                "compass_find_groups": ([P, P, P, P, I, U32, P, ctypes.c_float, P, P], I),
                "ut_align_chi2": ([P, P, P, P, U32, P, P, P, P, P, P, P, P, SZ, P], I),
                "ut_align_refit": ([P, P, P, P, U32, P, P, P, P], I),
                "ut_align_hvp": ([P, P, P, P, U32, P, P, P, P, P, P], I),
                "ut_align_solve_workspace_size": ([I, U32], SZ),
                "ut_align_solve": ([P, P, P, P, U32, P, P, I, I, P, P, SZ, P], I),
            }
            for name, (args, res) in sig.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = res
            _lib = L
        return _lib


class UtError(RuntimeError):
    def __init__(self, code, where=None, what=""):
        super().__init__(f"{what}: {ERR_NAMES.get(code, code)}" + (f" at {where}" if where else ""))
        self.code = code
        self.where = where


def _check(rc, what):
    if rc != UT_OK:
        raise UtError(rc, what=what)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _stream(stream):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def geometry_struct(geom) -> UtGeometry:
    g = UtGeometry()
    g.n_sectors = int(geom.n_sectors)
    for l in range(4):
        g.z[l] = float(geom.z[l])
        g.tan_stereo[l] = float(geom.tan_stereo[l])
    g.sector_pitch = float(geom.sector_pitch)
    g.strip_pitch = float(geom.strip_pitch)
    g.strips = int(geom.strips)
    g.x_min = float(geom.x_min)
    g.z_velo = float(geom.z_velo)
    return g


def params_struct(p) -> CompassParamsC:
    s = CompassParamsC()
    for f in dataclasses.fields(p):
        setattr(s, f.name, getattr(p, f.name))
    return s


class Context:
    """ut_ctx wrapper (one per geometry and device)."""

    def __init__(self, geom):
        self.geom = geom
        self._g = geometry_struct(geom)
        h = ctypes.c_void_p()
        _check(lib().ut_ctx_create(ctypes.byref(h), ctypes.byref(self._g)), "ut_ctx_create")
        self.handle = h

    def close(self):
        if self.handle:
            lib().ut_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def status(self, stream=None):
        code = ctypes.c_int()
        a = ctypes.c_int64()
        b = ctypes.c_int64()
        _check(lib().ut_status(self.handle, _stream(stream), ctypes.byref(code), ctypes.byref(a),
                               ctypes.byref(b)), "ut_status")
        return code.value, a.value, b.value

    def reset(self, stream=None):
        _check(lib().ut_status_reset(self.handle, _stream(stream)), "ut_status_reset")

    def set_kick_map(self, kick_map=None):
        """Field look-up table of the kick (ut_ctx_set_kick_map): an object with
        nx, ny, tx_max, ty_max and values (float32 [ny, nx]); None removes it."""
        if kick_map is None:
            _check(lib().ut_ctx_set_kick_map(self.handle, 0, 0, 0.0, 0.0, None), "ut_ctx_set_kick_map")
            return
        v = np.ascontiguousarray(kick_map.values, dtype=np.float32)
        if v.shape != (int(kick_map.ny), int(kick_map.nx)):
            raise ValueError("kick map values must have shape (ny, nx)")
        _check(lib().ut_ctx_set_kick_map(self.handle, int(kick_map.nx), int(kick_map.ny),
                                         float(kick_map.tx_max), float(kick_map.ty_max),
                                         v.ctypes.data_as(ctypes.c_void_p)), "ut_ctx_set_kick_map")

    def set_wait_limit(self, spins=0):
        """Polls of a bounded device wait before UT_ERR_TIMEOUT (0 = default)."""
        _check(lib().ut_ctx_set_wait_limit(self.handle, int(spins)), "ut_ctx_set_wait_limit")

    def set_first_ticket(self, first=0):
        """Test facility: the decodes skip events [0, first) (ut_ctx_set_first_ticket)."""
        _check(lib().ut_ctx_set_first_ticket(self.handle, int(first)), "ut_ctx_set_first_ticket")

    def check(self, stream=None, what="device"):
        code, a, b = self.status(stream)
        if code != UT_OK:
            raise UtError(code, (a, b), what)


@dataclasses.dataclass
class HitBuffers:
    """Device SoA hits (ut_hits) with `capacity` entries and n_events*B+1 offsets."""
    x: torch.Tensor
    z: torch.Tensor
    sector: torch.Tensor
    layer: torch.Tensor
    id: torch.Tensor
    hit_off: torch.Tensor
    capacity: int

    @staticmethod
    def allocate(capacity, n_events, n_sectors, device="cuda"):
        cap = max(int(capacity), 1)
        return HitBuffers(torch.empty(cap, dtype=torch.float32, device=device),
                          torch.empty(cap, dtype=torch.float32, device=device),
                          torch.empty(cap, dtype=torch.int16, device=device),
                          torch.empty(cap, dtype=torch.uint8, device=device),
                          torch.empty(cap, dtype=torch.int32, device=device),
                          torch.empty(n_events * 4 * n_sectors + 1, dtype=torch.int32, device=device),
                          int(capacity))

    def struct(self) -> UtHits:
        h = UtHits()
        h.x, h.z, h.sector, h.layer = (t.data_ptr() for t in (self.x, self.z, self.sector, self.layer))
        h.id, h.hit_off = self.id.data_ptr(), self.hit_off.data_ptr()
        h.capacity = min(int(self.capacity), 0xFFFFFFFF)
        return h


@dataclasses.dataclass
class VeloBuffers:
    x: torch.Tensor
    y: torch.Tensor
    tx: torch.Tensor
    ty: torch.Tensor
    flags: torch.Tensor
    trk_off: torch.Tensor

    @property
    def n_tracks(self):
        return int(self.x.numel())

    def struct(self) -> VeloTracks:
        v = VeloTracks()
        for n in ("x", "y", "tx", "ty", "flags", "trk_off"):
            setattr(v, n, getattr(self, n).data_ptr())
        return v


@dataclasses.dataclass
class TrackBuffers:
    """Track outputs (compass_tracks).  velo and n_found (int32 [rows] and
    [n_events]) are only used by the paper's atomic output order
    (compass_params.output_order = 1)."""
    hit: torch.Tensor
    qop: torch.Tensor
    chi2: torch.Tensor
    x: torch.Tensor
    tx: torch.Tensor
    nhits: torch.Tensor
    found: torch.Tensor
    velo: torch.Tensor | None = None
    n_found: torch.Tensor | None = None

    @staticmethod
    def allocate(n_tracks, device="cuda", n_events=None):
        T = max(int(n_tracks), 1)
        f = lambda: torch.empty(T, dtype=torch.float32, device=device)
        tb = TrackBuffers(torch.empty((T, 4), dtype=torch.int32, device=device), f(), f(), f(), f(),
                          torch.empty(T, dtype=torch.uint8, device=device),
                          torch.empty(T, dtype=torch.uint8, device=device))
        if n_events is not None:
            tb.velo = torch.empty(T, dtype=torch.int32, device=device)
            tb.n_found = torch.empty(max(int(n_events), 1), dtype=torch.int32, device=device)
        return tb

    def struct(self) -> CompassTracksC:
        c = CompassTracksC()
        for n in ("hit", "qop", "chi2", "x", "tx", "nhits", "found", "velo", "n_found"):
            t = getattr(self, n)
            setattr(c, n, t.data_ptr() if t is not None else None)
        return c


@dataclasses.dataclass
class CompactTracks:
    """Consolidated found tracks (rows in (event, VELO track) order)."""
    hit: torch.Tensor
    qop: torch.Tensor
    chi2: torch.Tensor
    x: torch.Tensor
    tx: torch.Tensor
    nhits: torch.Tensor
    velo: torch.Tensor
    capacity: int

    @staticmethod
    def allocate(capacity, device="cuda"):
        n = max(int(capacity), 1)
        f = lambda: torch.empty(n, dtype=torch.float32, device=device)
        return CompactTracks(torch.empty((n, 4), dtype=torch.int32, device=device), f(), f(), f(), f(),
                             torch.empty(n, dtype=torch.uint8, device=device),
                             torch.empty(n, dtype=torch.int32, device=device), int(capacity))

    def struct(self) -> UtTracksCompactC:
        c = UtTracksCompactC()
        for n in ("hit", "qop", "chi2", "x", "tx", "nhits", "velo"):
            setattr(c, n, getattr(self, n).data_ptr())
        c.capacity = self.capacity
        return c


def decode_workspace_size(n_events: int) -> int:
    return int(lib().ut_decode_workspace_size(int(n_events)))


def ut_decode(ctx, raw, n_raw_words, ev_off, n_events, out: HitBuffers, sorted_=True,
              workspace=None, stream=None):
    """Raw banks -> hits (one kernel).  raw: int32 device tensor (u32 words,
    length a multiple of 4); ev_off: int64 device tensor (n_events + 1)."""
    ws_bytes = decode_workspace_size(n_events)
    if workspace is None:
        workspace = torch.empty((ws_bytes + 15) // 16 * 4, dtype=torch.int32, device=raw.device)
    h = out.struct()
    rc = lib().ut_decode(ctx.handle, _ptr(raw), int(n_raw_words), _ptr(ev_off), int(n_events),
                         ctypes.byref(h), 1 if sorted_ else 0, _ptr(workspace),
                         workspace.numel() * workspace.element_size(), _stream(stream))
    _check(rc, "ut_decode")
    return workspace


def ut_decode_noalloc(geom, raw, n_raw_words, ev_off, n_events, out: HitBuffers, status,
                      sorted_=True, stream=None):
    """ut_decode without allocations: scratch in the library's static device
    array, errors in `status` (int64 device tensor of one element)."""
    g = geometry_struct(geom)
    h = out.struct()
    rc = lib().ut_decode_noalloc(ctypes.byref(g), _ptr(raw), int(n_raw_words), _ptr(ev_off),
                                 int(n_events), ctypes.byref(h), 1 if sorted_ else 0, _ptr(status),
                                 _stream(stream))
    _check(rc, "ut_decode_noalloc")


def decode_status_key(key: int):
    """(code, event, bank) of a status key (all ones = no error)."""
    key &= 0xFFFFFFFFFFFFFFFF
    if key == 0xFFFFFFFFFFFFFFFF:
        return UT_OK, -1, -1
    a, b = key >> 32, (key >> 8) & 0xFFFFFF
    return -(key & 0xFF), (-1 if a == 0xFFFFFFFF else a), (-1 if b == 0xFFFFFF else b)


def ut_sort_hits(ctx, hits_in: HitBuffers, hits_out: HitBuffers, n_events, perm=None, stream=None):
    hi, ho = hits_in.struct(), hits_out.struct()
    _check(lib().ut_sort_hits(ctx.handle, ctypes.byref(hi), ctypes.byref(ho), _ptr(perm),
                              int(n_events), _stream(stream)), "ut_sort_hits")


def compass_find(ctx, hits: HitBuffers, velo: VeloBuffers, n_events, params, out: TrackBuffers,
                 win=None, tracks_per_warp=1, block=256, stream=None):
    h, v, p, o = hits.struct(), velo.struct(), params_struct(params), out.struct()
    _check(lib().compass_find(ctx.handle, ctypes.byref(h), ctypes.byref(v), int(n_events),
                              velo.n_tracks, ctypes.byref(p), ctypes.byref(o), _ptr(win),
                              int(tracks_per_warp), int(block), _stream(stream)), "compass_find")


def ut_run_batched(ctx, raw, n_raw_words, ev_off, n_events, velo: VeloBuffers, params,
                   hits_out: HitBuffers, tracks_out: TrackBuffers, cfg: LaunchConfig | None = None,
                   workspace=None, stream=None):
    """The whole path for a batch in one persistent launch (decode, sort,
    windows, tracklets, fit)."""
    ws_bytes = decode_workspace_size(n_events)
    if workspace is None:
        workspace = torch.empty((ws_bytes + 15) // 16 * 4, dtype=torch.int32, device=raw.device)
    h, v, p, o = hits_out.struct(), velo.struct(), params_struct(params), tracks_out.struct()
    c = (cfg or LaunchConfig()).struct()
    _check(lib().ut_run_batched(ctx.handle, _ptr(raw), int(n_raw_words), _ptr(ev_off), int(n_events),
                                ctypes.byref(v), velo.n_tracks, ctypes.byref(p), ctypes.byref(h),
                                ctypes.byref(o), ctypes.byref(c), _ptr(workspace),
                                workspace.numel() * workspace.element_size(), _stream(stream)),
           "ut_run_batched")
    return workspace


def compass_fit(ctx, hits: HitBuffers, velo: VeloBuffers, params, inout: TrackBuffers, stream=None):
    h, v, p, o = hits.struct(), velo.struct(), params_struct(params), inout.struct()
    _check(lib().compass_fit(ctx.handle, ctypes.byref(h), ctypes.byref(v), velo.n_tracks,
                             ctypes.byref(p), ctypes.byref(o), _stream(stream)), "compass_fit")


# ---------------------------------------------------------------------------
# Host <-> device helpers for a batch of events.
# ---------------------------------------------------------------------------

def upload_raw(raw_np: np.ndarray, ev_off_np: np.ndarray, device="cuda"):
    """Copy raw words (u32, padded to a multiple of 4) and event offsets."""
    n = raw_np.size
    padded = (n + 3) // 4 * 4
    buf = np.zeros(max(padded, 4), dtype=np.uint32)
    buf[:n] = raw_np
    raw = torch.from_numpy(buf.view(np.int32)).to(device)
    ev = torch.from_numpy(np.ascontiguousarray(ev_off_np, dtype=np.uint64).view(np.int64)).to(device)
    return raw, ev


def upload_velo(batch, device="cuda") -> VeloBuffers:
    t = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a).view(dt)).to(device)
    return VeloBuffers(t(batch.velo_x, np.float32), t(batch.velo_y, np.float32),
                       t(batch.velo_tx, np.float32), t(batch.velo_ty, np.float32),
                       t(batch.velo_flags.astype(np.uint8), np.uint8),
                       t(batch.trk_off.astype(np.uint32), np.int32))


def hits_to_numpy(h: HitBuffers, n=None):
    off = h.hit_off.cpu().numpy().view(np.uint32)
    n = int(off[-1]) if n is None else n
    return dict(x=h.x[:n].cpu().numpy(), z=h.z[:n].cpu().numpy(),
                sector=h.sector[:n].cpu().numpy().view(np.uint16),
                layer=h.layer[:n].cpu().numpy(), id=h.id[:n].cpu().numpy().view(np.uint32),
                hit_off=off)


def consolidate_workspace_size(n_events: int) -> int:
    return int(lib().ut_consolidate_workspace_size(int(n_events)))


def ut_consolidate(ctx, trk_off, n_events, tracks: TrackBuffers, out: CompactTracks, out_off,
                   workspace=None, stream=None):
    """Found tracks of `tracks` -> consecutive rows of `out`, in (event, VELO
    track) order; out_off (int32 device tensor, n_events + 1) = first row of
    each event, then the total."""
    ws_bytes = consolidate_workspace_size(n_events)
    if workspace is None:
        workspace = torch.empty((ws_bytes + 15) // 16 * 4, dtype=torch.int32, device=out_off.device)
    tin = tracks.struct()
    tout = out.struct()
    _check(lib().ut_consolidate(ctx.handle, _ptr(trk_off), int(n_events), ctypes.byref(tin), ctypes.byref(tout),
                                _ptr(out_off), _ptr(workspace), workspace.numel() * workspace.element_size(),
                                _stream(stream)), "ut_consolidate")
    return workspace


def compact_to_numpy(c: CompactTracks, n):
    return dict(hit=c.hit[:n].cpu().numpy(), qop=c.qop[:n].cpu().numpy(), chi2=c.chi2[:n].cpu().numpy(),
                x=c.x[:n].cpu().numpy(), tx=c.tx[:n].cpu().numpy(), nhits=c.nhits[:n].cpu().numpy(),
                velo=c.velo[:n].cpu().numpy().view(np.uint32))


def tracks_to_numpy(t: TrackBuffers, n):
    return dict(hit=t.hit[:n].cpu().numpy(), qop=t.qop[:n].cpu().numpy(),
                chi2=t.chi2[:n].cpu().numpy(), x=t.x[:n].cpu().numpy(), tx=t.tx[:n].cpu().numpy(),
                nhits=t.nhits[:n].cpu().numpy(), found=t.found[:n].cpu().numpy())


class Pipeline:
    """Device-resident buffers for one batch and the two launch forms:

    plain:  ut_decode(sorted=0) -> ut_sort_hits -> compass_find -> compass_fit
            (four kernels, the per-step form);
    fused:  ut_decode(sorted=1) -> compass_find (decode, sort and the
            tracklet fit in two kernels).
    """

    def __init__(self, ctx, batch, params, device="cuda", capacity=None):
        self.ctx = ctx
        self.params = params
        self.n_events = batch.n_events
        self.n_words = int(batch.ev_off[-1])
        self.raw, self.ev_off = upload_raw(batch.raw, batch.ev_off, device)
        self.velo = upload_velo(batch, device)
        S = batch.geom.n_sectors
        cap = int(capacity) if capacity is not None else 2 * self.n_words
        self.hits_a = HitBuffers.allocate(cap, self.n_events, S, device)
        self.hits_b = HitBuffers.allocate(cap, self.n_events, S, device)
        self.tracks = TrackBuffers.allocate(self.velo.n_tracks, device)
        ws = decode_workspace_size(self.n_events)
        self.workspace = torch.empty((ws + 15) // 16 * 4, dtype=torch.int32, device=device)

    def run_plain(self, stream=None, tracks_per_warp=1, block=256):
        ut_decode(self.ctx, self.raw, self.n_words, self.ev_off, self.n_events, self.hits_a, False,
                  self.workspace, stream)
        ut_sort_hits(self.ctx, self.hits_a, self.hits_b, self.n_events, stream=stream)
        self.hits_b.hit_off = self.hits_a.hit_off
        compass_find(self.ctx, self.hits_b, self.velo, self.n_events, self.params, self.tracks,
                     tracks_per_warp=tracks_per_warp, block=block, stream=stream)
        compass_fit(self.ctx, self.hits_b, self.velo, self.params, self.tracks, stream=stream)
        return self.hits_b

    def run_batched(self, cfg: LaunchConfig | None = None, stream=None):
        ut_run_batched(self.ctx, self.raw, self.n_words, self.ev_off, self.n_events, self.velo,
                       self.params, self.hits_a, self.tracks, cfg, self.workspace, stream)
        return self.hits_a

    def run_fused(self, stream=None, tracks_per_warp=1, block=256):
        ut_decode(self.ctx, self.raw, self.n_words, self.ev_off, self.n_events, self.hits_a, True,
                  self.workspace, stream)
        compass_find(self.ctx, self.hits_a, self.velo, self.n_events, self.params, self.tracks,
                     tracks_per_warp=tracks_per_warp, block=block, stream=stream)
        return self.hits_a


class GraphRunner:
    """The batched form of a Pipeline captured once in a CUDA graph and
    replayed (one graph launch per pass over the batch)."""

    def __init__(self, pipe: Pipeline, cfg: LaunchConfig | None = None):
        self.pipe = pipe
        self.cfg = cfg
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            pipe.run_batched(cfg)          # warm-up outside the capture
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            pipe.run_batched(cfg)

    def replay(self):
        self.graph.replay()


def group_geometry_struct(gg) -> UtGroupGeometry:
    """ut_group_geometry of a synth.grouped.GroupGeometry."""
    s = UtGroupGeometry()
    s.n_columns, s.rows, s.n_groups = int(gg.n_columns), int(gg.rows), int(gg.n_groups)
    s.sector_pitch = float(gg.base.sector_pitch)
    s.strip_pitch = float(gg.base.strip_pitch)
    s.x_min, s.y_min, s.sensor_height = float(gg.x_min), float(gg.y_min), float(gg.sensor_height)
    for l in range(4):
        s.z[l] = float(gg.base.z[l])
    e = np.asarray(gg.group_edges(), np.float32)
    for k, v in enumerate(e):
        s.edges[k] = float(v)
    return s


@dataclasses.dataclass
class GroupHitBuffers:
    """Device SoA of the sector-group layout (ut_group_hits)."""
    x: torch.Tensor
    z: torch.Tensor
    y_begin: torch.Tensor
    y_end: torch.Tensor
    weight: torch.Tensor
    id: torch.Tensor
    group_off: torch.Tensor
    capacity: int

    @staticmethod
    def allocate(capacity, n_events, n_groups, device="cuda"):
        cap = max(int(capacity), 1)
        f = lambda: torch.empty(cap, dtype=torch.float32, device=device)
        return GroupHitBuffers(f(), f(), f(), f(), f(), torch.empty(cap, dtype=torch.int32, device=device),
                               torch.empty(n_events * 4 * n_groups + 1, dtype=torch.int32, device=device),
                               int(capacity))

    def struct(self) -> UtGroupHits:
        h = UtGroupHits()
        for n in ("x", "z", "y_begin", "y_end", "weight", "id", "group_off"):
            setattr(h, n, getattr(self, n).data_ptr())
        h.capacity = min(int(self.capacity), 0xFFFFFFFF)
        return h


def ut_sector_groups(ctx, bank_order: HitBuffers, n_events, gg, out: GroupHitBuffers, stream=None):
    """The sector-group layout from a bank-order decode (ut_sector_groups)."""
    h, g, o = bank_order.struct(), group_geometry_struct(gg), out.struct()
    _check(lib().ut_sector_groups(ctx.handle, ctypes.byref(h), int(n_events), ctypes.byref(g), ctypes.byref(o),
                                  _stream(stream)), "ut_sector_groups")


def decode_groups(raw, ev_off, n_events, gg, stream=None):
    """Raw banks of a grouped detector -> (Context, GroupHitBuffers): the
    bank-order decode on a context with one sector per sensor, then
    ut_sector_groups.  The context's status is checked."""
    ctx = Context(gg.raw_geometry())
    raw_d, ev_d = upload_raw(raw, ev_off)
    nw = int(ev_off[n_events]) if n_events else 0
    hits = HitBuffers.allocate(2 * nw + 8, n_events, gg.n_columns * gg.rows)
    ut_decode(ctx, raw_d, nw, ev_d, n_events, hits, False, stream=stream)
    out = GroupHitBuffers.allocate(2 * nw + 8, n_events, gg.n_groups)
    ut_sector_groups(ctx, hits, n_events, gg, out, stream)
    ctx.check(stream, "decode_groups")
    return ctx, out


def group_hits_to_numpy(gh: GroupHitBuffers):
    off = gh.group_off.cpu().numpy().view(np.uint32)
    n = int(off[-1])
    return dict(x=gh.x[:n].cpu().numpy(), z=gh.z[:n].cpu().numpy(), y_begin=gh.y_begin[:n].cpu().numpy(),
                y_end=gh.y_end[:n].cpu().numpy(), weight=gh.weight[:n].cpu().numpy(),
                id=gh.id[:n].cpu().numpy().view(np.uint32), group_off=off)


def compass_find_groups(ctx, hits: GroupHitBuffers, gg, velo: VeloBuffers, n_events, params, out: TrackBuffers,
                        tol_y=10.0, stream=None):
    """Compass on the sector-group layout (compass_find_groups): windows over
    the groups with y windows, then compass_find's tracklet search; hit
    indices refer to the group layout."""
    h, g, v, p, o = hits.struct(), group_geometry_struct(gg), velo.struct(), params_struct(params), out.struct()
    _check(lib().compass_find_groups(ctx.handle, ctypes.byref(h), ctypes.byref(g), ctypes.byref(v), int(n_events),
                                     velo.n_tracks, ctypes.byref(p), float(tol_y), ctypes.byref(o), _stream(stream)),
           "compass_find_groups")
