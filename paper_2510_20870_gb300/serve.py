"""Continuous-batching server for opacity cross-section requests (the serving path).

Requests ask for a window of the 0.01 cm^-1 lattice on one of several resident line lists at
one (P,T). The server keeps the lists prepared on the device (rox_prepare), admits requests as
they arrive while in-flight slots and the device-memory budget allow, packs everything queued
into one persistent launch (rox_xsec_jobs) on a free stream -- so batches launched while
others are still running overlap on the GPU -- and returns each result to pinned host memory.
Each request's result does not depend on what it was batched with (same lines, same
summation order), which the tests check bit for bit.
"""
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import _binding as rb
from .partition import PartitionFunction


@dataclass
class Request:
    rid: int
    t_arrival: float      # s, relative to the start of the run
    list_id: int
    p_bar: float
    t_k: float
    first: int            # lattice index of the window start
    n: int                # window points


@dataclass
class Result:
    rid: int
    sigma: np.ndarray
    t_arrival: float
    t_launch: float
    t_done: float

    @property
    def latency(self):
        return self.t_done - self.t_arrival


@dataclass
class _Batch:
    stream: object
    event: object
    reqs: list
    outs: list
    host: list
    ws: object
    t_launch: float
    nbytes: int


class Server:
    def __init__(self, lists, lattice, cutoff, mass_amu, q_spec, max_inflight=3, max_batch=64,
                 mem_budget=16 << 30):
        """lists: dicts of nu0-sorted device columns (see paper_2510_20870_gb300._binding.lines_struct)."""
        self.prepared = [rb.Prepared(L, lattice, cutoff) for L in lists]
        for p in self.prepared:
            rc, _ = p.status()
            if rc != 0:
                raise rb.RoxError(rc, "line list is not sorted by nu0")
        self.lattice = lattice
        self.mass = float(mass_amu)
        self.Q = PartitionFunction(q_spec)
        self.Q_ref = self.Q(296.0)
        self.streams = [torch.cuda.Stream() for _ in range(max_inflight)]
        self.max_batch = max_batch
        self.mem_budget = mem_budget
        self.evals = 0
        self.launches = 0
        self.max_inflight_seen = 0
        self.max_batch_seen = 0

    def _job(self, r, out):
        return rb.make_job(self.prepared[r.list_id], r.list_id, r.first, r.n, r.p_bar, r.t_k, self.Q(r.t_k),
                           self.Q_ref, self.mass, out)

    def _bytes(self, r):
        l0, cnt = self.prepared[r.list_id].line_range(r.first, r.n)
        return cnt * 12 + r.n * 8 + 4096

    def _launch(self, reqs, stream, t0):
        with torch.cuda.stream(stream):
            outs = [torch.empty(r.n, dtype=torch.float32, device="cuda") for r in reqs]
            jobs = [self._job(r, o) for r, o in zip(reqs, outs)]
            ws = torch.empty(rb.rox_jobs_workspace_size(jobs), dtype=torch.uint8, device="cuda")
            rb.rox_xsec_jobs(self.prepared, jobs, ws, stream)
            host = [torch.empty(r.n, dtype=torch.float32, pin_memory=True) for r in reqs]
            for h, o in zip(host, outs):
                h.copy_(o, non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(stream)
        self.launches += 1
        return _Batch(stream, ev, reqs, outs, host, ws, time.perf_counter() - t0, sum(self._bytes(r) for r in reqs))

    def run(self, requests, realtime=True, one_per_launch=False):
        """Serve `requests` (arrival times in s). realtime: arrivals follow the wall clock;
        otherwise everything is queued at once. one_per_launch: the plain baseline, each
        request alone in its own launch, one at a time. Returns a list of Result."""
        pending = sorted(requests, key=lambda r: r.t_arrival)
        queue, inflight, results = [], [], []
        max_batch = 1 if one_per_launch else self.max_batch
        slots = 1 if one_per_launch else len(self.streams)
        used = 0
        k = 0
        t0 = time.perf_counter()
        while k < len(pending) or queue or inflight:
            now = time.perf_counter() - t0
            while k < len(pending) and (not realtime or pending[k].t_arrival <= now):
                queue.append(pending[k])
                k += 1
            still = []
            for b in inflight:
                if b.event.query():
                    t_done = time.perf_counter() - t0
                    rc, ev = rb.rox_ws_status(b.ws, b.stream)
                    if rc != 0:
                        raise rb.RoxError(rc, rb.lib.rox_last_error().decode())
                    self.evals += ev
                    for r, h in zip(b.reqs, b.host):
                        results.append(Result(r.rid, h.numpy(), r.t_arrival, b.t_launch, t_done))
                    used -= b.nbytes
                else:
                    still.append(b)
            inflight = still
            if queue and len(inflight) < slots:
                batch, nb = [], 0
                while queue and len(batch) < max_batch and (not batch or used + nb + self._bytes(queue[0]) <= self.mem_budget):
                    nb += self._bytes(queue[0])
                    batch.append(queue.pop(0))
                busy = {id(b.stream) for b in inflight}
                stream = next(s for s in self.streams if id(s) not in busy)
                inflight.append(self._launch(batch, stream, t0))
                used += nb
                self.max_inflight_seen = max(self.max_inflight_seen, len(inflight))
                self.max_batch_seen = max(self.max_batch_seen, len(batch))
                continue
            if not queue and not inflight and k < len(pending):
                time.sleep(max(0.0, min(pending[k].t_arrival - (time.perf_counter() - t0), 0.002)))
            else:
                time.sleep(0.0002)
        return sorted(results, key=lambda r: r.rid)


def requests_from_stream(reqs, lattice):
    """Server requests from rox_synth's request stream (windows given by their start wavenumber
    on the lattice)."""
    nu_min, dnu, _ = lattice
    return [Request(r.rid, r.t_arrival, r.list_id, r.p_bar, r.t_k, int(round((r.nu_min - nu_min) / dnu)), r.n)
            for r in reqs]


def latency_stats(results):
    lat = np.array([r.latency for r in results])
    return {"p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "mean_ms": float(lat.mean() * 1e3), "n": int(lat.size)}
