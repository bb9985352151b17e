"""Continuous-batching server for opacity cross-section requests (the serving path).

Requests ask for a window of the 0.01 cm^-1 lattice on one of several resident line lists at
one (P,T). The server keeps the lists prepared on the device (rox_prepare), admits requests as
they arrive while in-flight slots and the device-memory budget allow, packs what is queued into
one persistent launch (rox_xsec_jobs) on a free stream -- so batches launched while others are
still running overlap on the GPU -- and returns each result to pinned host memory.

Packing is size-aware: the queue is served shortest job first (estimated evaluations; a request
that has waited `promote_s` goes ahead in arrival order, so long ones are not starved), a batch
holds at most `batch_evals` estimated evaluations (a request larger than that runs alone), so
a long request occupies one slot while short ones keep flowing through the others. A request
that has waited longer than `max_wait_s` is rejected instead of served (the overload policy).
Device memory: a batch holds its outputs and its rox_xsec_jobs workspace (counted exactly with
rox_jobs_workspace_size); batches are admitted while the bytes of all in-flight batches stay
within the budget, by default 80% of the device memory free when the server starts
(cudaMemGetInfo). A request that would not fit even alone is rejected.
Each request's result does not depend on what it was batched with (same lines, same
summation order), which the tests check bit for bit.
"""
import time
from dataclasses import dataclass

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
                 mem_budget=None, batch_evals=6e10, max_wait_s=None, promote_s=0.25):
        """lists: dicts of nu0-sorted device columns (see paper_2510_20870_gb300._binding.lines_struct).
        mem_budget: device bytes the in-flight batches may hold (None: 80% of the free memory now).
        batch_evals: estimated evaluations per batch (a larger request runs alone).
        max_wait_s: queueing time after which a request is rejected (None: never).
        promote_s: queueing time after which a request goes ahead of shorter ones (no starvation)."""
        self.prepared = [rb.Prepared(L, lattice, cutoff) for L in lists]
        for p in self.prepared:
            rc, _ = p.status()
            if rc != 0:
                raise rb.RoxError(rc, "line list is not sorted by nu0")
        self.lattice = lattice
        self.cutoff = float(cutoff)
        self.win_pts = int(2.0 * cutoff / lattice[1]) + 1
        self.mass = float(mass_amu)
        self.Q = PartitionFunction(q_spec)
        self.Q_ref = self.Q(296.0)
        self.streams = [torch.cuda.Stream() for _ in range(max_inflight)]
        self.max_batch = max_batch
        if mem_budget is None:
            free, _ = torch.cuda.mem_get_info()
            mem_budget = int(0.8 * free)
        self.mem_budget = int(mem_budget)
        self.batch_evals = float(batch_evals)
        self.max_wait_s = max_wait_s
        self.promote_s = promote_s
        self.evals = 0
        self.launches = 0
        self.rejected = []
        self.max_inflight_seen = 0
        self.max_batch_seen = 0
        self.max_bytes_seen = 0
        self.max_queue_seen = 0

    def _job(self, r, out_ptr):
        l0, cnt = self.prepared[r.list_id].line_range(r.first, r.n)
        return rb.RoxJob(list=r.list_id, flags=0, first=r.first, n=r.n, line_first=l0, line_count=cnt, P_bar=r.p_bar,
                         T=r.t_k, Q_T=self.Q(r.t_k), Q_ref=self.Q_ref, mass_amu=self.mass, sigma_out=out_ptr)

    def work(self, r):
        """Estimated evaluations of a request: the lines that can reach its window times the
        points each covers at most."""
        _, cnt = self.prepared[r.list_id].line_range(r.first, r.n)
        return cnt * min(r.n, self.win_pts)

    def batch_bytes(self, reqs):
        """Device bytes a batch holds while in flight: its outputs and its rox_xsec_jobs workspace."""
        jobs = [self._job(r, 0) for r in reqs]
        return int(rb.rox_jobs_workspace_size(jobs)) + sum(4 * r.n for r in reqs)

    def _launch(self, reqs, stream, t0, nbytes):
        with torch.cuda.stream(stream):
            outs = [torch.empty(r.n, dtype=torch.float32, device="cuda") for r in reqs]
            jobs = [self._job(r, o.data_ptr()) for r, o in zip(reqs, outs)]
            ws = torch.empty(rb.rox_jobs_workspace_size(jobs), dtype=torch.uint8, device="cuda")
            rb.rox_xsec_jobs(self.prepared, jobs, ws, stream)
            host = [torch.empty(r.n, dtype=torch.float32, pin_memory=True) for r in reqs]
            for h, o in zip(host, outs):
                h.copy_(o, non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(stream)
        self.launches += 1
        return _Batch(stream, ev, reqs, outs, host, ws, time.perf_counter() - t0, nbytes)

    def _form_batch(self, queue, used, max_batch, work_of):
        """Requests for the next launch from the queue (sorted shortest first), within the work
        bound and the memory budget; [] if even the first does not fit next to the batches in
        flight."""
        batch, work = [], 0.0
        for r in list(queue):
            if len(batch) >= max_batch:
                break
            wr = work_of[id(r)]
            if batch and work + wr > self.batch_evals:
                break
            if used + self.batch_bytes(batch + [r]) > self.mem_budget:
                break
            batch.append(r)
            work += wr
        return batch

    def run(self, requests, realtime=True, one_per_launch=False):
        """Serve `requests` (arrival times in s). realtime: arrivals follow the wall clock;
        otherwise everything is queued at once. one_per_launch: the plain baseline, each
        request alone in its own launch (with as many launches in flight as the server has
        slots). Returns a list of Result; rejected requests are listed in self.rejected."""
        pending = sorted(requests, key=lambda r: r.t_arrival)
        work_of = {id(r): self.work(r) for r in pending}
        queue, inflight, results = [], [], []
        max_batch = 1 if one_per_launch else self.max_batch
        self.rejected = []
        used = 0
        k = 0
        t0 = time.perf_counter()
        while k < len(pending) or queue or inflight:
            now = time.perf_counter() - t0
            while k < len(pending) and (not realtime or pending[k].t_arrival <= now):
                r = pending[k]
                k += 1
                if self.batch_bytes([r]) > self.mem_budget:
                    self.rejected.append(r)          # can never fit, even alone
                    continue
                queue.append(r)
            if queue and not one_per_launch:
                # shortest job first; a request that has waited promote_s goes ahead (arrival order)
                queue.sort(key=lambda r: (0, r.t_arrival) if now - r.t_arrival > self.promote_s else (1, work_of[id(r)]))
            self.max_queue_seen = max(self.max_queue_seen, len(queue))
            if self.max_wait_s is not None:
                keep = []
                for r in queue:
                    (self.rejected if now - r.t_arrival > self.max_wait_s else keep).append(r)
                queue = keep
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
            if queue and len(inflight) < len(self.streams):
                batch = self._form_batch(queue, used, max_batch, work_of)
                if batch:
                    for r in batch:
                        queue.remove(r)
                    nb = self.batch_bytes(batch)
                    busy = {id(b.stream) for b in inflight}
                    stream = next(s for s in self.streams if id(s) not in busy)
                    inflight.append(self._launch(batch, stream, t0, nb))
                    used += nb
                    self.max_inflight_seen = max(self.max_inflight_seen, len(inflight))
                    self.max_batch_seen = max(self.max_batch_seen, len(batch))
                    self.max_bytes_seen = max(self.max_bytes_seen, used)
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
    if not results:
        return {"p50_ms": None, "p99_ms": None, "mean_ms": None, "n": 0}
    lat = np.array([r.latency for r in results])
    return {"p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "mean_ms": float(lat.mean() * 1e3), "n": int(lat.size)}
