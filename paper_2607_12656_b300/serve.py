"""Continuous-batching decode server on one GPU.

Requests (scene bitstreams with arrival times) are admitted as soon as a slot and HBM budget
are free.  Each slot owns a CUDA stream and a library context whose decode scratch, sized for
the pool's largest scene, is allocated once when the server is built; the slots' scratch is
charged against the HBM budget then, and each request is charged its own device buffers
(bitstream + decoded outputs) at admission, in arrival order.  A request that cannot fit
even with every other slot idle is answered at once with E_NOMEM instead of holding up the
queue.  Admitted decodes overlap on the device while the host loop keeps admitting and
retiring.  Latency = completion - arrival, with the completion taken from the device: the
admission time plus the CUDA-event time from the slot's first enqueued operation to the end
of its decode (the loop's polling delay is not counted).

Only orchestration lives here; every decode runs in the library's kernels through
``scene_decode``.
"""
from __future__ import annotations

import collections
import dataclasses
import time

import numpy as np

from . import sgs


@dataclasses.dataclass
class Scene:
    """A coded scene held in pinned host memory."""
    bits: bytes
    info: sgs.SceneInfo = None
    host: object = None  # pinned uint8 tensor

    def __post_init__(self):
        import torch
        if self.info is None:
            self.info = sgs.scene_query(self.bits)
        if self.host is None:
            self.host = torch.frombuffer(bytearray(self.bits), dtype=torch.uint8).pin_memory()

    @property
    def n_rows(self) -> int:
        return int(self.info.n_rows)

    def buffers(self) -> int:
        """Device bytes a request allocates: the bitstream and the decoded outputs."""
        return int(self.info.total_len) + 4 * 59 * self.n_rows

    def footprint(self) -> int:
        """Device bytes of one decode of this scene: its buffers plus its decode scratch."""
        return self.buffers() + int(self.info.scratch_bytes)


@dataclasses.dataclass
class Result:
    req: int
    scene: int
    arrival: float
    admitted: float
    done: float
    status: int
    attr: object = None
    pos: object = None
    digest: tuple = None  # (sha256 of attr bytes, sha256 of pos bytes) with keep_outputs="digest"

    @property
    def latency(self) -> float:
        return self.done - self.arrival


class _Slot:
    def __init__(self, device: int, scratch: int):
        import torch
        self.stream = torch.cuda.Stream(device=device)
        self.ctx = sgs.Context(device, scratch)
        self.busy = None  # (req, scene_id, arrival, admitted, ev_start, ev_end, bufs)


class DecodeServer:
    def __init__(self, scenes: list[Scene], *, slots: int = 8, hbm_budget: int = 120 << 30,
                 device: int = 0, keep_outputs=False):
        """keep_outputs: False, True (results carry host copies of the outputs) or "digest"
        (results carry SHA-256 digests of the outputs' bytes, for scenes too large to keep)."""
        self.scenes = scenes
        self.device = device
        self.budget = hbm_budget
        self.keep = keep_outputs
        scratch = max(s.info.scratch_bytes for s in scenes)
        self.slot_scratch = slots * int(scratch)  # allocated now, charged once
        self.slots = self._make_slots(slots, scratch)
        self.in_use = self.slot_scratch

    # ---- device side: one stream and one library context per slot
    def _make_slots(self, n: int, scratch: int) -> list:
        return [_Slot(self.device, scratch) for _ in range(n)]

    def _launch(self, slot: _Slot, req: int, sid: int, arrival: float, now: float):
        import torch
        sc = self.scenes[sid]
        dev = torch.device("cuda", self.device)
        with torch.cuda.stream(slot.stream):
            bits = torch.empty(len(sc.bits), dtype=torch.uint8, device=dev)
            attr = torch.empty((56, max(sc.n_rows, 1)), device=dev)
            pos = torch.empty((3, max(sc.n_rows, 1)), device=dev)
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record(slot.stream)
            bits.copy_(sc.host, non_blocking=True)
            sgs.scene_decode(slot.ctx, bits, sc.info, attr, pos, None, None, slot.stream)
            ev1.record(slot.stream)
        slot.busy = (req, sid, arrival, now, ev0, ev1, (bits, attr, pos))

    def _finished(self, slot: _Slot) -> bool:
        return slot.busy[5].query()

    def _retire(self, slot: _Slot, t0: float) -> Result:
        req, sid, arr, adm, ev0, ev1, bufs = slot.busy
        st = slot.ctx.sync(slot.stream)
        r = Result(req, sid, arr, adm, adm + ev0.elapsed_time(ev1) / 1e3, st)
        if self.keep:
            n = self.scenes[sid].n_rows
            a, p = bufs[1][:, :n].cpu(), bufs[2][:, :n].cpu()
            if self.keep == "digest":
                import hashlib
                r.digest = (hashlib.sha256(a.numpy().tobytes()).hexdigest(),
                            hashlib.sha256(p.numpy().tobytes()).hexdigest())
            else:
                r.attr, r.pos = a, p
        return r

    # ---- host loop: arrivals, retirement, admission
    def run(self, requests: list[tuple[float, int]]) -> list[Result]:
        """requests: (arrival offset in s, scene index), sorted by arrival.  Returns results in
        completion order."""
        pending = collections.deque((i, t, s) for i, (t, s) in enumerate(requests))
        queue = collections.deque()
        results = []
        t0 = time.perf_counter()
        while pending or queue or any(sl.busy for sl in self.slots):
            now = time.perf_counter() - t0
            while pending and pending[0][1] <= now:
                queue.append(pending.popleft())
            for sl in self.slots:
                if sl.busy and self._finished(sl):
                    sid = sl.busy[1]
                    results.append(self._retire(sl, t0))
                    self.in_use -= self.scenes[sid].buffers()
                    sl.busy = None
            # admit in arrival order while a slot and memory are free
            while queue:
                req, arr, sid = queue[0]
                fp = self.scenes[sid].buffers()
                if fp + self.slot_scratch > self.budget:  # can never fit: answer now, do not block
                    queue.popleft()
                    t = time.perf_counter() - t0
                    results.append(Result(req, sid, arr, t, t, sgs.E_NOMEM))
                    continue
                free = [sl for sl in self.slots if sl.busy is None]
                if not free or self.in_use + fp > self.budget:
                    break
                queue.popleft()
                self.in_use += fp
                self._launch(free[0], req, sid, arr, time.perf_counter() - t0)
            if not queue and pending:
                wait = pending[0][1] - (time.perf_counter() - t0)
                if wait > 0 and not any(sl.busy for sl in self.slots):
                    time.sleep(min(wait, 0.002))
        return results

    def close(self):
        for sl in self.slots:
            sl.ctx.close()


def poisson_arrivals(rate: float, n: int, n_scenes: int, seed: int) -> list[tuple[float, int]]:
    rng = np.random.Generator(np.random.PCG64(seed))
    gaps = rng.exponential(1.0 / rate, size=n)
    t = np.cumsum(gaps)
    which = rng.integers(0, n_scenes, size=n)
    return [(float(a), int(b)) for a, b in zip(t, which)]


def poisson_arrivals_modes(rate: float, n: int, modes: dict, seed: int) -> list[tuple[float, int]]:
    """Poisson arrivals; each request draws a coding mode uniformly, then a scene of that mode
    uniformly (scene ids from modes: name -> list of ids)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = np.cumsum(rng.exponential(1.0 / rate, size=n))
    groups = [ids for ids in modes.values() if ids]
    m = rng.integers(0, len(groups), size=n)
    out = []
    for a, g in zip(t, m):
        ids = groups[int(g)]
        out.append((float(a), int(ids[int(rng.integers(0, len(ids)))])))
    return out


def summarize(results: list[Result], scenes: list[Scene], modes: dict | None = None) -> dict:
    lat = np.array([r.latency for r in results]) * 1e3
    span = max(r.done for r in results) - min(r.arrival for r in results)
    out = {"requests": len(results), "p50_ms": float(np.percentile(lat, 50)),
           "p99_ms": float(np.percentile(lat, 99)),
           "gaussians_per_s": sum(scenes[r.scene].n_rows for r in results) / span,
           "bad_status": sum(1 for r in results if r.status != sgs.OK)}
    if modes:
        for name, ids in modes.items():
            sel = [r for r in results if r.scene in ids]
            if sel:
                l2 = np.array([r.latency for r in sel]) * 1e3
                out[name] = {"requests": len(sel), "p50_ms": float(np.percentile(l2, 50)),
                             "p99_ms": float(np.percentile(l2, 99))}
    return out
