"""Serving: continuous batching of decode + Compass requests.

Server wraps the library's native engine (ut_server_*): one device arena of
a fixed byte budget, a pool of stream slots and a worker thread that admits
waiting requests in arrival order as soon as a slot and arena memory are
free, so that requests arriving while others run overlap on the device.

HostRequest packs one batch of events into page-locked host buffers (inputs
and the track-slot outputs).  run_open_loop replays Poisson arrivals at a
given event rate; run_closed_loop submits everything at once to measure the
sustained peak.  Both report p50/p99 request latency and events/s.
"""
from __future__ import annotations

import ctypes
import dataclasses
import threading
import time

import numpy as np
import torch

from . import (UT_OK, ERR_NAMES, UtError, _build, geometry_struct, params_struct, lib, LaunchConfig)


class ServerRequestC(ctypes.Structure):
    _fields_ = [("raw", ctypes.c_void_p), ("n_raw_words", ctypes.c_uint64), ("ev_off", ctypes.c_void_p),
                ("n_events", ctypes.c_int), ("vx", ctypes.c_void_p), ("vy", ctypes.c_void_p),
                ("vtx", ctypes.c_void_p), ("vty", ctypes.c_void_p), ("flags", ctypes.c_void_p),
                ("trk_off", ctypes.c_void_p), ("n_tracks", ctypes.c_uint32), ("out_hit", ctypes.c_void_p),
                ("out_qop", ctypes.c_void_p), ("out_chi2", ctypes.c_void_p), ("out_x", ctypes.c_void_p),
                ("out_tx", ctypes.c_void_p), ("out_nhits", ctypes.c_void_p), ("out_found", ctypes.c_void_p)]


class ServerResultC(ctypes.Structure):
    _fields_ = [("id", ctypes.c_int64), ("status", ctypes.c_int), ("where_a", ctypes.c_int64),
                ("where_b", ctypes.c_int64), ("queue_s", ctypes.c_double), ("latency_s", ctypes.c_double),
                ("slot", ctypes.c_int)]


_sigs_done = False


def _sigs():
    global _sigs_done
    if _sigs_done:
        return lib()
    L = lib()
    P = ctypes.c_void_p
    L.ut_server_create.argtypes = [P, P, P, ctypes.c_size_t, ctypes.c_int, P]
    L.ut_server_create.restype = ctypes.c_int
    L.ut_server_submit.argtypes = [P, P]
    L.ut_server_submit.restype = ctypes.c_int64
    L.ut_server_poll.argtypes = [P, P, ctypes.c_int, ctypes.c_int]
    L.ut_server_poll.restype = ctypes.c_int
    L.ut_server_stats.argtypes = [P, P, P, P]
    L.ut_server_stats.restype = ctypes.c_int
    L.ut_server_destroy.argtypes = [P]
    L.ut_server_destroy.restype = ctypes.c_int
    L.ut_server_request_bytes.argtypes = [P, P]
    L.ut_server_request_bytes.restype = ctypes.c_size_t
    _sigs_done = True
    return L


def _pinned(a: np.ndarray, dtype) -> torch.Tensor:
    t = torch.from_numpy(np.ascontiguousarray(a).view(dtype)).pin_memory()
    return t


@dataclasses.dataclass
class HostRequest:
    """One batch of events in page-locked host memory, with its outputs."""
    n_events: int
    n_tracks: int
    n_raw_words: int
    bufs: dict
    out: dict

    @staticmethod
    def from_batch(batch) -> "HostRequest":
        n = int(batch.ev_off[-1])
        raw = np.zeros((n + 3) // 4 * 4, np.uint32)
        raw[:n] = batch.raw[:n]
        T = batch.n_tracks
        bufs = {"raw": _pinned(raw, np.int32), "ev_off": _pinned(batch.ev_off.astype(np.uint64), np.int64),
                "vx": _pinned(batch.velo_x, np.float32), "vy": _pinned(batch.velo_y, np.float32),
                "vtx": _pinned(batch.velo_tx, np.float32), "vty": _pinned(batch.velo_ty, np.float32),
                "flags": _pinned(batch.velo_flags.astype(np.uint8), np.uint8),
                "trk_off": _pinned(batch.trk_off.astype(np.uint32), np.int32)}
        Tn = max(T, 1)
        out = {"hit": torch.empty((Tn, 4), dtype=torch.int32).pin_memory(),
               "qop": torch.empty(Tn, dtype=torch.float32).pin_memory(),
               "chi2": torch.empty(Tn, dtype=torch.float32).pin_memory(),
               "x": torch.empty(Tn, dtype=torch.float32).pin_memory(),
               "tx": torch.empty(Tn, dtype=torch.float32).pin_memory(),
               "nhits": torch.empty(Tn, dtype=torch.uint8).pin_memory(),
               "found": torch.empty(Tn, dtype=torch.uint8).pin_memory()}
        return HostRequest(batch.n_events, T, n, bufs, out)

    def struct(self) -> ServerRequestC:
        b, o = self.bufs, self.out
        p = lambda t: t.data_ptr()
        return ServerRequestC(p(b["raw"]), self.n_raw_words, p(b["ev_off"]), self.n_events, p(b["vx"]),
                              p(b["vy"]), p(b["vtx"]), p(b["vty"]), p(b["flags"]), p(b["trk_off"]),
                              self.n_tracks, p(o["hit"]), p(o["qop"]), p(o["chi2"]), p(o["x"]), p(o["tx"]),
                              p(o["nhits"]), p(o["found"]))

    def outputs(self) -> dict:
        T = self.n_tracks
        return {k: v[:T].numpy().copy() for k, v in self.out.items()}


class Server:
    """The native serving engine on the current device."""

    def __init__(self, geom, params, budget_bytes: int = 40 << 30, n_slots: int = 8,
                 cfg: LaunchConfig | None = None):
        L = _sigs()
        self._g = geometry_struct(geom)
        self._p = params_struct(params)
        self._cfg = cfg.struct() if cfg is not None else None
        h = ctypes.c_void_p()
        rc = L.ut_server_create(ctypes.byref(h), ctypes.byref(self._g), ctypes.byref(self._p),
                                int(budget_bytes), int(n_slots),
                                ctypes.byref(self._cfg) if self._cfg is not None else None)
        if rc != UT_OK:
            raise UtError(rc, what="ut_server_create")
        self.handle = h
        self.live = {}       # id -> (HostRequest, struct) kept alive until done
        self.lock = threading.Lock()

    def request_bytes(self, req: HostRequest) -> int:
        s = req.struct()
        return int(_sigs().ut_server_request_bytes(ctypes.byref(self._g), ctypes.byref(s)))

    def submit(self, req: HostRequest) -> int:
        s = req.struct()
        rid = int(_sigs().ut_server_submit(self.handle, ctypes.byref(s)))
        if rid < 0:
            raise UtError(rid, what="ut_server_submit")
        with self.lock:
            self.live[rid] = (req, s)
        return rid

    def poll(self, wait=False, max_results=256):
        arr = (ServerResultC * max_results)()
        n = _sigs().ut_server_poll(self.handle, arr, max_results, 1 if wait else 0)
        out = []
        for i in range(n):
            r = arr[i]
            with self.lock:
                req, _ = self.live.pop(r.id)
            out.append({"id": r.id, "status": r.status, "where": (r.where_a, r.where_b),
                        "queue_s": r.queue_s, "latency_s": r.latency_s, "slot": r.slot,
                        "request": req})
        return out

    def stats(self):
        n = ctypes.c_int64()
        used = ctypes.c_size_t()
        peak = ctypes.c_size_t()
        _sigs().ut_server_stats(self.handle, ctypes.byref(n), ctypes.byref(used), ctypes.byref(peak))
        return {"in_flight": n.value, "arena_used": used.value, "arena_peak": peak.value}

    def drain(self):
        done = []
        while True:
            if self.stats()["in_flight"] == 0 and not self.live:
                break
            done += self.poll(wait=True)
        return done

    def close(self):
        if self.handle:
            _sigs().ut_server_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def _summary(results, n_events_total, wall_s):
    lat = np.array([r["latency_s"] for r in results]) * 1e3
    q = np.array([r["queue_s"] for r in results]) * 1e3
    bad = [r for r in results if r["status"] != UT_OK]
    return {"requests": len(results), "events": int(n_events_total), "wall_s": wall_s,
            "events_per_s": n_events_total / wall_s if wall_s > 0 else 0.0,
            "p50_ms": float(np.percentile(lat, 50)) if len(lat) else None,
            "p99_ms": float(np.percentile(lat, 99)) if len(lat) else None,
            "queue_p50_ms": float(np.percentile(q, 50)) if len(q) else None,
            "errors": [(r["id"], ERR_NAMES.get(r["status"], r["status"])) for r in bad]}


def run_closed_loop(server: Server, requests):
    """Submit every request at once; sustained events/s and latencies."""
    t0 = time.perf_counter()
    for r in requests:
        server.submit(r)
    res = server.drain()
    wall = time.perf_counter() - t0
    return _summary(res, sum(r.n_events for r in requests), wall), res


def run_open_loop(server: Server, requests, events_per_s: float, seed: int = 0):
    """Poisson arrivals: request i arrives after exponential gaps whose mean
    is its event count / events_per_s.  Completed requests are collected
    while later ones arrive (continuous batching)."""
    rng = np.random.default_rng(seed)
    gaps = [rng.exponential(r.n_events / events_per_s) for r in requests]
    done = []
    t0 = time.perf_counter()
    t_next = t0
    for r, gap in zip(requests, gaps):
        t_next += gap
        while True:
            now = time.perf_counter()
            if now >= t_next:
                break
            done += server.poll(wait=False)
            time.sleep(min(2e-4, t_next - now))
        server.submit(r)
    done += server.drain()
    wall = time.perf_counter() - t0
    return _summary(done, sum(r.n_events for r in requests), wall), done
