"""Streaming reconstruction: concurrent scan sessions with frame-to-render
latency.

The paper images in real time by reconstructing only the newly acquired
frames and re-processing only the regions that changed, with acquisition,
reconstruction and display running concurrently (Sec. II.C).  Here each
scan session owns a resident volume and a CUDA stream; frames arrive from
the probe in bursts, and each burst is

    host->device copy -> usv_insert_frames -> usv_fill_holes_region
    -> usv_project_depth_band_region

on the session's stream, the region being the voxel box the burst's frames
touch plus the one-voxel neighbourhood the 3x3x3 fill reads.  A burst's
frame-to-render latency is the time from its arrival on the host to the
moment its refreshed projection is complete on the device, observed from
the host.  Sessions are admitted only while their device memory fits a
budget; every volume stays resident.

Two dispatch modes.  Per-session streams: each burst is enqueued on its
session's stream as it arrives.  Batched: one engine stream; whenever it
dispatches, it takes every session's oldest waiting burst, inserts all the
nearest-neighbour ones with one usv_insert_frames_multi call (one set-up and
one persistent insertion launch over all volumes), then refreshes each
session's region.  Either mode can also replay the scans as fast as the GPU
takes them (no real-time pacing) to measure serving throughput.

All GPU work is the library's kernels (through the C ABI); this module only
schedules.
"""
from __future__ import annotations

import threading
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import usvol

MAX_BURST = 32


class AdmissionError(RuntimeError):
    """A session does not fit the device-memory budget."""


def session_bytes(w) -> int:
    """Device bytes a session holds: volume, frame staging, projection."""
    nx, ny, nz = w.grid
    frame = w.H * w.W * (4 if w.images.dtype == np.float32 else 1)
    return (usvol.volume_bytes(w.grid, w.mode) + MAX_BURST * (frame + 128) +
            nx * ny * 6)


@dataclass
class SessionStats:
    name: str
    fps: float
    frames: int = 0
    bursts: int = 0
    latencies_ms: list = field(default_factory=list)   # one entry per frame

    def percentile(self, p):
        return float(np.percentile(self.latencies_ms, p)) if self.latencies_ms else None


class Session:
    """One scan: a resident volume fed by bursts of frames."""

    def __init__(self, name: str, w, fps: float, device, seed: int = 0):
        self.name = name
        self.w = w
        self.fps = float(fps)
        self.device = torch.device(device)
        self.stream = torch.cuda.Stream(self.device)
        self.vol = usvol.Volume(w.grid, w.spacing, w.origin, w.mode, device=self.device)
        self.cal = usvol.calibration_of(w)
        nx, ny, nz = w.grid
        with torch.cuda.stream(self.stream):
            self.vol.reset(self.stream)
            self.vol.fill(self.stream)
        self.h_imgs = torch.from_numpy(np.ascontiguousarray(w.images)).pin_memory()
        self.h_poses = torch.from_numpy(np.ascontiguousarray(w.poses)).pin_memory()
        self.d_imgs = torch.empty((MAX_BURST,) + tuple(w.images.shape[1:]),
                                  dtype=self.h_imgs.dtype, device=self.device)
        self.d_poses = torch.empty((MAX_BURST, 4, 4), dtype=torch.float64, device=self.device)
        self.out = torch.zeros((ny, nx), dtype=torch.float32, device=self.device)
        self.cnt = torch.zeros((ny, nx), dtype=torch.int16, device=self.device)
        rng = np.random.default_rng(seed)
        self.sizes = []
        total = 0
        while total < w.n:
            b = int(rng.integers(1, MAX_BURST + 1))
            b = min(b, w.n - total)
            self.sizes.append(b)
            total += b
        self.stats = SessionStats(name, self.fps)

    def arrivals(self, t0: float):
        """(time, first frame, count) of each burst: a burst arrives when
        its last frame has been acquired at the session's frame rate."""
        f = 0
        for b in self.sizes:
            yield t0 + (f + b) / self.fps, f, b
            f += b

    def stage(self, f0: int, b: int, st, poses: bool = False):
        """Host->device copy of burst [f0, f0 + b) into the staging buffers
        (the frames; the poses too if `poses`, for the multi-volume call)."""
        self.d_imgs[:b].copy_(self.h_imgs[f0:f0 + b], non_blocking=True)
        if poses:
            self.d_poses[:b].copy_(self.h_poses[f0:f0 + b], non_blocking=True)

    def refresh(self, f0: int, b: int, st):
        """Fill + projection of the region burst [f0, f0 + b) touched: the
        library's voxel box of the burst, widened by the fill's one-voxel
        neighbourhood."""
        w = self.w
        lo, hi = self.vol.voxel_box(self.h_poses[f0:f0 + b], w.H, w.W, self.cal, margin=1)
        usvol.fill_holes_region(self.vol.handle, lo, hi, 1, st)
        usvol.project_depth_band_region(self.vol.handle, w.band[0], w.band[1], lo[:2], hi[:2],
                                        self.out.data_ptr(), self.cnt.data_ptr(), st)

    def dispatch(self, f0: int, b: int):
        """Enqueue one burst on the session's stream; returns its done-event."""
        st = self.stream
        with torch.cuda.stream(st):
            self.stage(f0, b, st)
            # host poses: the library stages them (usv_insert_frames)
            self.vol.insert(self.d_imgs[:b], self.h_poses[f0:f0 + b], self.cal, st)
            self.refresh(f0, b, st)
            ev = torch.cuda.Event()
            ev.record(st)
        return ev


class Scheduler:
    """Admits sessions by device memory and runs them concurrently in real
    time (one dispatcher, one completion watcher per session)."""

    def __init__(self, device="cuda", memory_budget: int | None = None):
        self.device = torch.device(device)
        if memory_budget is None:
            free, _ = torch.cuda.mem_get_info(self.device)
            memory_budget = int(free * 0.9)
        self.budget = int(memory_budget)
        self.used = 0
        self.sessions: list[Session] = []

    def admit(self, name: str, w, fps: float, seed: int = 0) -> Session:
        need = session_bytes(w)
        if self.used + need > self.budget:
            raise AdmissionError(f"session {name} needs {need} B; {self.budget - self.used} B "
                                 f"of the {self.budget} B budget left")
        s = Session(name, w, fps, self.device, seed)
        self.used += need
        self.sessions.append(s)
        return s

    def _events(self, t0: float, seconds, realtime: bool):
        events = []
        for si, s in enumerate(self.sessions):
            for t, f0, b in s.arrivals(t0):
                if seconds is not None and t - t0 > seconds:
                    break
                events.append((t if realtime else t0, si, f0, b))
        events.sort(key=lambda e: (e[0], e[2], e[1]))
        return events

    def dispatch_batch(self, bursts, st):
        """One engine dispatch: bursts = [(session index, f0, b)], at most one
        per session.  Returns the done-event."""
        with torch.cuda.stream(st):
            for si, f0, b in bursts:
                self.sessions[si].stage(f0, b, st, poses=self.sessions[si].w.mode == "pnn")
            pnn = [(si, b) for si, _, b in bursts if self.sessions[si].w.mode == "pnn"]
            if pnn:
                usvol.insert_frames_multi(
                    [(self.sessions[si].vol, self.sessions[si].d_imgs[:b],
                      self.sessions[si].d_poses[:b], self.sessions[si].cal) for si, b in pnn], st)
            for si, f0, b in bursts:
                s = self.sessions[si]
                if s.w.mode != "pnn":
                    s.vol.insert(s.d_imgs[:b], s.h_poses[f0:f0 + b], s.cal, st)
            for si, f0, b in bursts:
                self.sessions[si].refresh(f0, b, st)
            ev = torch.cuda.Event()
            ev.record(st)
        return ev

    def run(self, seconds: float | None = None, batched: bool = False, realtime: bool = True):
        """Stream every session's frames at its frame rate (for at most
        `seconds` of scan time); returns the per-session stats.  batched:
        one engine stream with multi-volume insertion; realtime=False: every
        burst is available at once and the GPU takes them as fast as it can
        (latencies then measure queueing, use wall_s for throughput)."""
        if batched:
            return self._run_batched(seconds, realtime)
        torch.cuda.synchronize(self.device)
        t0 = time.perf_counter() + 0.05
        events = self._events(t0, seconds, realtime)
        queues = [[] for _ in self.sessions]
        conds = [threading.Condition() for _ in self.sessions]
        done = [False] * len(self.sessions)

        def watch(si):
            s = self.sessions[si]
            while True:
                with conds[si]:
                    while not queues[si] and not done[si]:
                        conds[si].wait()
                    if not queues[si]:
                        return
                    ev, t_arr, b = queues[si].pop(0)
                ev.synchronize()
                lat = (time.perf_counter() - t_arr) * 1e3
                s.stats.latencies_ms.extend([lat] * b)
                s.stats.frames += b
                s.stats.bursts += 1

        threads = [threading.Thread(target=watch, args=(i,), daemon=True)
                   for i in range(len(self.sessions))]
        for th in threads:
            th.start()
        for t, si, f0, b in events:
            delay = t - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            ev = self.sessions[si].dispatch(f0, b)
            with conds[si]:
                queues[si].append((ev, t, b))
                conds[si].notify()
        for si in range(len(self.sessions)):
            with conds[si]:
                done[si] = True
                conds[si].notify()
        for th in threads:
            th.join()
        self.wall_s = time.perf_counter() - t0
        return [s.stats for s in self.sessions]

    def _run_batched(self, seconds, realtime: bool):
        torch.cuda.synchronize(self.device)
        engine = torch.cuda.Stream(self.device)
        t0 = time.perf_counter() + 0.05
        pending = self._events(t0, seconds, realtime)
        queue, cond, state = [], threading.Condition(), {"done": False}
        self.dispatches = 0

        def watch():
            while True:
                with cond:
                    while not queue and not state["done"]:
                        cond.wait()
                    if not queue:
                        return
                    ev, members = queue.pop(0)
                ev.synchronize()
                now = time.perf_counter()
                for si, t_arr, b in members:
                    st = self.sessions[si].stats
                    st.latencies_ms.extend([(now - t_arr) * 1e3] * b)
                    st.frames += b
                    st.bursts += 1

        th = threading.Thread(target=watch, daemon=True)
        th.start()
        i = 0
        while i < len(pending):
            delay = pending[i][0] - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            now = time.perf_counter()
            # every session's oldest burst that has arrived (one per session:
            # its staging buffers hold one burst)
            take, seen, rest = [], set(), []
            for e in pending[i:]:
                if e[0] > now:
                    rest.append(e)
                elif e[1] in seen:
                    rest.append(e)
                else:
                    seen.add(e[1])
                    take.append(e)
            ev = self.dispatch_batch([(si, f0, b) for _, si, f0, b in take], engine)
            self.dispatches += 1
            with cond:
                queue.append((ev, [(si, t, b) for t, si, f0, b in take]))
                cond.notify()
            pending = sorted(rest, key=lambda e: (e[0], e[2], e[1]))
            i = 0
        with cond:
            state["done"] = True
            cond.notify()
        th.join()
        self.wall_s = time.perf_counter() - t0
        return [s.stats for s in self.sessions]


def summary(stats) -> dict:
    lat = [x for s in stats for x in s.latencies_ms]
    return {
        "frames": int(sum(s.frames for s in stats)),
        "bursts": int(sum(s.bursts for s in stats)),
        "p50_ms": float(np.percentile(lat, 50)) if lat else None,
        "p99_ms": float(np.percentile(lat, 99)) if lat else None,
        "max_ms": float(np.max(lat)) if lat else None,
        "sessions": [{"name": s.name, "fps": s.fps, "frames": s.frames, "bursts": s.bursts,
                      "p50_ms": s.percentile(50), "p99_ms": s.percentile(99)} for s in stats],
    }
