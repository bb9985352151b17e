#!/usr/bin/env python
"""Throughput of the line-by-line opacity cross-section hot path on GB300.

Workload (default): the large-list case -- 1e9 synthetic HITRAN-style lines (half-precision
widths, 20 B per line) held on the device as ten nu0-sorted chunks of 1e8, nu0 uniform
500-10000 cm^-1, grid 500-10000 cm^-1 at 0.01 cm^-1 (950,001 points), 100 cm^-1 wing cutoff,
(P,T) = (10 bar, 3000 K). One step = one cross-section of the whole list through the C ABI:
rox_xsec_batch on each chunk in turn, the chunks after the first added into sigma
(ROX_ACCUMULATE); each call computes strengths and widths, windows and span ranges, and runs the
Voigt kernel. Metric: Voigt line-profile evaluations per second, one evaluation being a (line,
grid point) pair inside the cutoff, counted exactly. (The 300-point batch case, 1e8 lines at
15 P x 20 T, takes about a minute per step; it runs with --config 3.)

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl rox|reference] [--config 1..4]

--impl reference times the FP64 CPU oracle (scipy.special.wofz) on a bounded sample of
the same workload on the host cores. Under torchrun (N > 1) every rank runs one replica
of the workload on its own GPU (the path has no exchange step).
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import rox_synth as rs  # noqa: E402

FLOPS_PER_EVAL = 11.0   # far-wing pair formula: 10 FFMA + 2 FMUL per 2 evaluations (+ 1 MUFU rcp)
# DRAM bytes per Voigt launch on the full exomol workload: ncu dram__bytes_read + write of the
# 2e6-line case (151.3 MB + 43.4 MB, profiles/k_voigt_exomol_2e6lines.md), scaled by evaluations
# (x5.0); most of the writes are L2 write-backs of the per-line constants k_line_params wrote
VOIGT_TRAFFIC_BYTES = 9.737e8
# DRAM bytes of one k_cia_grid launch on the CIA workload (ncu dram__bytes_read + write,
# profiles/k_cia_grid_40T_2970001pts.md; part of the 950 MB output is still in L2 at the end)
CIA_TRAFFIC_BYTES = 8.955e8
# DRAM bytes per evaluation of k_voigt on the large list: ncu dram__bytes_read + write on one
# 1e7-line chunk of it (4.170 GB for 1.989e11 evaluations, profiles/k_voigt_large_1e7_chunk.md)
VOIGT_TRAFFIC_LARGE = 4.1697e9 / 1.98948e11
FP32_LANES_PER_SM = 128
SM_MAX_MHZ = 2070.0
METRIC = "Voigt line-profile evals/s"
UNIT = "evals/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="rox", choices=["rox", "reference"])
    ap.add_argument("--config", type=int, default=4)
    ap.add_argument("--chunk", type=int, default=100_000_000, help="lines per resident chunk (large list)")
    ap.add_argument("--no-config2", action="store_true", help="skip the single-(P,T) exomol summary of the large run")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="target CPU time of the oracle sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end leg (profiling runs)")
    ap.add_argument("--lines", type=int, default=None,
                    help="use only the first N lines of the workload (smaller profiling case)")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving (request-latency) leg")
    ap.add_argument("--select", type=float, default=None, metavar="REL",
                    help="main-contributor selection: keep lines with S >= REL x the largest S of their nu0 bin "
                         "(rox_xsec_select_batch)")
    ap.add_argument("--select-bin", type=float, default=1.0, help="selection bin width (cm^-1)")
    ap.add_argument("--cia", action="store_true",
                    help="CIA restructuring: 40 synthetic temperatures of coefficient blocks onto config 2's grid "
                         "(rox_cia_regrid); prints its own JSON line")
    ap.add_argument("--broadening", action="store_true",
                    help="broadener mixture and natural broadening (rox_xsec_broadened_batch): 0.85 H2 from per-line "
                         "columns + 0.15 He from a J table, plus A/(4 pi c)")
    ap.add_argument("--nodes", action="store_true",
                    help="user-provided grid: the workload's lines on nodes of fixed resolving power R = %g over the "
                         "same wavenumber range (rox_xsec_nodes_batch)" % rs.FIXED_R)
    ap.add_argument("--serve-rates", default="50,100,200,500", help="Poisson request rates (req/s) of the serving leg")
    ap.add_argument("--serve-seconds", type=float, default=4.0, help="arrival window per rate (s)")
    ap.add_argument("--autotune", action="store_true",
                    help="sweep the Voigt launch configuration (paper_2510_20870_gb300/autotune.py) on the large "
                         "list's 1e8-line chunk and on the exomol list, write the cache and print the results")
    ap.add_argument("--probes", action="store_true",
                    help="print the FP32 probes only: the FMA peak and the Voigt pair loop's standalone rate")
    return ap.parse_args()


def workload(cid):
    w = rs.CONFIGS[cid]
    grid = rs.grid_of(w)
    (P, T), = w.pts
    q = rs.q_table(w)
    return w, grid, P, T, q


def q_of(q, T):
    """Q(T) for the GPU arm (the library's host-side helper)."""
    from paper_2510_20870_gb300.partition import PartitionFunction
    return PartitionFunction(q)(T)


def q_oracle(q, T):
    """Q(T) for the CPU oracle arm."""
    import oracle
    return float(oracle.partition_function(q, T))


# ------------------------------------------------------------------ CPU oracle (baseline / reference arm)
def _oracle_window(args):
    sub, grid, j0, j1, P, T, Qt, Qr, mass, cutoff = args
    import oracle
    if isinstance(grid, np.ndarray):           # user-provided nodes: grid holds the window's nodes
        s = oracle.xsec_nodes(sub, grid, P, T, Qt, Qr, mass, cutoff)
        jlo, jhi = oracle.node_windows(sub["nu0"], grid, cutoff)
        return int(np.sum(np.maximum(jhi - jlo + 1, 0))), float(s.sum())
    s = oracle.xsec_window(sub, grid, j0, j1, P, T, Qt, Qr, mass, cutoff)
    jlo, jhi = oracle.window_indices(sub["nu0"], *grid, cutoff)
    ev = int(np.sum(np.maximum(np.minimum(jhi, j1 - 1) - np.maximum(jlo, j0) + 1, 0)))
    return ev, float(s.sum())


def oracle_sample_tasks(Ls, grid, P, T, Qt, Qr, mass, cutoff, n_windows, width, seed):
    rng = np.random.default_rng(seed)
    tasks = []
    nu0 = Ls["nu0"]
    nodes = isinstance(grid, np.ndarray)
    n = grid.size if nodes else grid[2]
    for s in rng.integers(0, n - width, n_windows):
        if nodes:
            lo, hi = grid[s] - cutoff - 1.0, grid[s + width - 1] + cutoff + 1.0
        else:
            lo = grid[0] + grid[1] * s - cutoff - 1.0
            hi = grid[0] + grid[1] * (s + width) + cutoff + 1.0
        a, b = np.searchsorted(nu0, lo), np.searchsorted(nu0, hi)
        sub = {k: (v[a:b] if isinstance(v, np.ndarray) else v) for k, v in Ls.items()}
        g = grid[s:s + width].copy() if nodes else grid
        tasks.append((sub, g, int(s), int(s) + width, P, T, Qt, Qr, mass, cutoff))
    return tasks


def time_oracle(tasks, cores):
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        pool.map(_oracle_window, tasks[:cores])          # warm the workers (imports)
        t0 = time.perf_counter()
        res = pool.map(_oracle_window, tasks, chunksize=1)
        dt = time.perf_counter() - t0
    return sum(r[0] for r in res), dt


def sorted_host_lines(w):
    import oracle
    return oracle.sort_lines(rs.make_lines(w))


def cpu_baseline(w, grid, P, T, q, Ls, target_s):
    cores = len(os.sched_getaffinity(0))
    Qt, Qr = q_oracle(q, T), q_oracle(q, 296.0)
    width = 256
    probe = oracle_sample_tasks(Ls, grid, P, T, Qt, Qr, w.mass_amu, w.cutoff, cores, width, 7)
    ev, dt = time_oracle(probe, cores)
    rate = ev / dt
    n_win = max(cores, int(target_s * rate / (ev / len(probe))))
    tasks = oracle_sample_tasks(Ls, grid, P, T, Qt, Qr, w.mass_amu, w.cutoff, n_win, width, 8)
    ev, dt = time_oracle(tasks, cores)
    return {"value": ev / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "%d random windows of %d %s of the %s workload (all lines within the cutoff "
                      "of each window), FP64 scipy.special.wofz, %d evals in %.1f s" % (
                          n_win, width, "nodes" if isinstance(grid, np.ndarray) else "grid points", w.name, ev, dt)}


def run_reference(args):
    """The reference arm: the FP64 oracle as it stands, on this host's cores (one spawned pool for
    the whole run), each step a bounded sample of random 256-point windows of the workload sized
    to about 4 s of oracle work, so that per-task overheads do not dominate. Lists above 1e7 lines
    are represented by their first 1e6 lines (the subsample the large list's accuracy is stated
    on); workloads with several (P,T) points draw one per window."""
    import multiprocessing as mp
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w = rs.CONFIGS[args.config]
    grid = rs.grid_of(w)
    q = rs.q_table(w)
    Ls, n_sub = oracle_subsample(w)
    cores = len(os.sched_getaffinity(0))
    Qr = q_oracle(q, 296.0)
    pts = list(w.pts)
    rng = np.random.default_rng(12)

    def tasks_for(count, seed):
        out = []
        for k in range(count):
            P, T = pts[int(rng.integers(0, len(pts)))]
            out += oracle_sample_tasks(Ls, grid, P, T, q_oracle(q, T), Qr, w.mass_amu, w.cutoff, 1, 256, seed * 100003 + k)
        return out

    total_ev, total_t = 0, 0.0
    with mp.get_context("spawn").Pool(cores) as pool:
        probe = tasks_for(cores, 99)
        pool.map(_oracle_window, probe)                  # warm the workers (imports)
        t0 = time.perf_counter()
        pool.map(_oracle_window, probe, chunksize=1)
        per_window = (time.perf_counter() - t0) * cores / len(probe)   # core-seconds per window
        per_step = cores * max(2, int(round(4.0 / max(per_window, 1e-6))))
        for step in range(args.warmup + args.steps):
            tasks = tasks_for(per_step, 100 + step)
            t0 = time.perf_counter()
            res = pool.map(_oracle_window, tasks, chunksize=1)
            dt = time.perf_counter() - t0
            if step >= args.warmup:
                total_ev += sum(r[0] for r in res)
                total_t += dt
    value = total_ev / total_t
    lines_note = "all %d lines" % w.n_lines if n_sub == w.n_lines else "its first %d lines (of %d)" % (n_sub, w.n_lines)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "%s: %d lines, grid %d points, cutoff %g cm^-1, %d (P,T) point(s)" % (
                w.name, w.n_lines, grid[2], w.cutoff, len(pts)),
                "sample_per_step": "%d windows x 256 points on %s" % (per_step, lines_note)},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "%d steps of %d random 256-point windows of the %s workload on %s (all of "
                                       "them within the cutoff of each window), FP64 scipy.special.wofz, one pool "
                                       "of %d processes" % (args.steps, per_step, w.name, lines_note, cores)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ------------------------------------------------------------------ serving leg (request latency)
def serving_leg(rates, seconds, max_wait_s=2.0):
    """Four resident lists (1e5..1e8 lines, exomol distributions) on the 0.01 cm^-1 lattice of
    300-30000 cm^-1; Poisson requests (list, P, T, window of 10-5000 cm^-1) arriving for `seconds`
    at each rate. Continuous batching against the plain one-request-per-launch loop, same request
    stream, same number of launches in flight (3); requests queued longer than max_wait_s are
    rejected (counted, not in the latency figures)."""
    import torch
    import paper_2510_20870_gb300 as rox
    from paper_2510_20870_gb300 import serve
    from rox_synth.device import make_lines_device

    lattice = (300.0, 0.01, 2970001)
    lists = []
    for w in rs.SERVE_LISTS:
        raw = make_lines_device(w, 0, w.n_lines)
        out = {k: (torch.empty_like(v) if isinstance(v, torch.Tensor) else v) for k, v in raw.items()}
        ws = torch.empty(rox.rox_sort_workspace_size(w.n_lines), dtype=torch.uint8, device="cuda")
        rox.rox_sort_lines(raw, out, None, ws)
        del raw, ws
        lists.append(out)
    w0 = rs.SERVE_LISTS[0]
    srv = serve.Server(lists, lattice, w0.cutoff, w0.mass_amu, rs.q_table(w0), max_inflight=3, max_batch=32,
                       max_wait_s=max_wait_s)
    srv.run(serve.requests_from_stream(rs.serve_requests(200.0, 16, seed=99), lattice), realtime=False)  # warm-up
    out = {}
    for rate in rates:
        reqs = serve.requests_from_stream(rs.serve_requests(rate, max(8, int(rate * seconds)), seed=5), lattice)
        demand = sum(srv.work(r) for r in reqs) / max(r.t_arrival for r in reqs)
        legs = {}
        for name, opl in (("batched", False), ("one_per_launch", True)):
            srv.evals, srv.launches, srv.max_queue_seen = 0, 0, 0
            t = time.perf_counter()
            res = srv.run(reqs, realtime=True, one_per_launch=opl)
            wall = time.perf_counter() - t
            st = serve.latency_stats(res)
            st.update({"served": len(res), "rejected": len(srv.rejected), "max_queued": srv.max_queue_seen,
                       "evals_per_s": srv.evals / wall, "launches": srv.launches, "wall_s": wall})
            legs[name] = st
        legs["requests"] = len(reqs)
        legs["demand_evals_per_s"] = demand
        out["%g" % rate] = legs
    budget = srv.mem_budget
    del srv, lists
    torch.cuda.empty_cache()
    return {"workload": "4 resident lists (1e5, 1e6, 1e7, 1e8 lines), Poisson arrivals for %g s per rate, list uniform, "
                        "P log-uniform 1e-5..1e2 bar, T uniform 300..3000 K, window 10..5000 cm^-1 at 0.01 cm^-1, "
                        "cutoff 25" % seconds,
            "policy": "continuous batching: 3 launches in flight, shortest job first (requests waiting over 0.25 s "
                      "first), at most 6e10 estimated evaluations per batch, device-memory budget %.1f GB (80%% of "
                      "free memory), requests queued over %g s rejected; one_per_launch: one request per launch, "
                      "3 in flight, same rejection rule" % (budget / 1e9, max_wait_s),
            "rates_req_per_s": out}


# ------------------------------------------------------------------ GPU arm
class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for k, name in enumerate(names):
                if f[5 + k].lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def run_gpu(args):
    import torch
    import paper_2510_20870_gb300 as rox

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)

    w, grid, P, T, q = workload(args.config)
    Qt, Qr = q_of(q, T), q_of(q, 296.0)
    from paper_2510_20870_gb300 import autotune
    launch_cfg, tuned = autotune.apply("exomol" if args.config == 2 else w.name)
    host = rs.make_lines(w, 0, args.lines)     # unsorted, generation order
    cols = ["nu0", "s_or_a", "g_up", "e_lower", "gamma_ref", "n_t"]
    pinned = {k: torch.from_numpy(host[k]).pin_memory() for k in cols if host[k] is not None}
    raw = {k: torch.empty_like(v, device=dev) for k, v in pinned.items()}
    raw["convention"] = host["convention"]
    lines = {k: torch.empty_like(v) for k, v in raw.items() if k != "convention"}
    lines["convention"] = host["convention"]
    raw.setdefault("g_up", None)
    lines.setdefault("g_up", None)
    n = len(host["nu0"])
    h2d_bytes = sum(v.numel() * v.element_size() for v in pinned.values())
    sort_ws = torch.empty(rox.rox_sort_workspace_size(n), dtype=torch.uint8, device=dev)
    if sum([args.nodes, args.select is not None, args.broadening]) > 1:
        raise SystemExit("--nodes, --select and --broadening are separate modes")
    if args.broadening:
        # broadener columns and J of the lines in nu0 order (the device sort is stable on nu0, like this one)
        order = np.argsort(host["nu0"], kind="stable")
        jl = rs.j_lower_of(w, 0, n)[order]
        tab_j = np.arange(60)
        extra_pin = {"j": torch.from_numpy(np.ascontiguousarray(jl)).pin_memory(),
                     "g_h2": torch.from_numpy((host["gamma_ref"][order].astype(np.float64) * 1.3)
                                              .astype(host["gamma_ref"].dtype)).pin_memory(),
                     "n_h2": torch.from_numpy((host["n_t"][order].astype(np.float64) - 0.1)
                                              .astype(host["n_t"].dtype)).pin_memory(),
                     "tg": torch.from_numpy((0.09 * np.exp(-tab_j / 40.0) + 0.01).astype(np.float32)).pin_memory(),
                     "tn": torch.from_numpy((0.45 + 0.004 * tab_j).astype(np.float32)).pin_memory()}
        extra = {k: v.to(dev) for k, v in extra_pin.items()}
        h2d_bytes += sum(v.numel() * v.element_size() for v in extra_pin.values())
        bro = {"vmr": [0.85, 0.15], "gamma_ref": [extra["g_h2"], None], "n_t": [extra["n_h2"], None],
               "table_gamma": [None, extra["tg"]], "table_n": [None, extra["tn"]], "j_lower": extra["j"],
               "natural": True}
    if args.nodes:
        nodes_np = rs.fixed_resolution_grid(w.grid_lo, w.grid_hi, rs.FIXED_R)
        nodes_pin = torch.from_numpy(nodes_np).pin_memory()
        nodes_dev = torch.empty_like(nodes_pin, device=dev)
        nodes_dev.copy_(nodes_pin)
        n_grid = nodes_np.size
        h2d_bytes += n_grid * 8
        ws = torch.empty(rox.rox_xsec_nodes_workspace_size(n, n_grid, 1), dtype=torch.uint8, device=dev)
    elif args.select is not None:
        n_grid = grid[2]
        ws = torch.empty(rox.rox_xsec_select_workspace_size(n, grid, 1, w.cutoff, args.select, args.select_bin),
                         dtype=torch.uint8, device=dev)
    elif args.broadening:
        n_grid = grid[2]
        ws = torch.empty(rox.rox_xsec_broadened_workspace_size(n, grid, 1), dtype=torch.uint8, device=dev)
    else:
        n_grid = grid[2]
        ws = torch.empty(rox.rox_xsec_workspace_size(n, grid, 1), dtype=torch.uint8, device=dev)
    sigma = torch.empty((1, n_grid), dtype=torch.float32, device=dev)
    sigma_host = torch.empty((1, n_grid), dtype=torch.float32).pin_memory()
    stream = torch.cuda.current_stream()

    def upload_and_sort():
        for k, v in pinned.items():
            raw[k].copy_(v, non_blocking=True)
        if args.nodes:
            nodes_dev.copy_(nodes_pin, non_blocking=True)
        if args.broadening:
            for k, v in extra_pin.items():
                extra[k].copy_(v, non_blocking=True)
        rox.rox_sort_lines(raw, lines, None, sort_ws)

    def step():
        if args.nodes:
            rox.rox_xsec_nodes_batch(lines, nodes_dev, [P], [T], [Qt], Qr, w.mass_amu, w.cutoff, sigma, ws)
        elif args.select is not None:
            rox.rox_xsec_select_batch(lines, grid, [P], [T], [Qt], Qr, w.mass_amu, w.cutoff, args.select,
                                      args.select_bin, sigma, ws)
        elif args.broadening:
            rox.rox_xsec_broadened_batch(lines, grid, bro, [P], [T], [Qt], Qr, w.mass_amu, w.cutoff, sigma, ws)
        else:
            rox.rox_xsec(lines, grid, P, T, Qt, Qr, w.mass_amu, w.cutoff, sigma, ws)

    upload_and_sort()
    step()
    rc, evals = rox.rox_ws_status(ws)
    if rc != 0:
        raise RuntimeError(rox.lib.rox_last_error().decode())

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    # ---- device-resident throughput, with the Voigt kernel timed by events around its launch
    for _ in range(args.warmup):
        step()
    ev_pairs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for a, b in ev_pairs:
        a.record()
        b.record()
    barrier()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clocks:
        time.sleep(0.3)
        barrier()
        t0.record()
        for a, b in ev_pairs:
            rox.rox_set_profile_events(a, b)
            step()
        rox.rox_set_profile_events(None, None)
        t1.record()
        barrier()
    ms = t0.elapsed_time(t1)
    voigt_ms = [a.elapsed_time(b) for a, b in ev_pairs]
    if dist is not None:
        tt = torch.tensor([ms], device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        ms = float(tt.item())
    ms_per_step = ms / args.steps
    value = world * evals * args.steps / (ms * 1e-3)

    # ---- end to end through the public API: pinned host -> device, sort, xsec, sigma -> host
    e2e_steps = 0 if args.no_e2e else args.steps
    pipelined = e2e_steps > 0 and not (args.nodes or args.broadening or args.select is not None)
    if pipelined:
        # every step uploads and sorts its own list and reads its own sigma back; step k+1's upload
        # and sort (copy stream) overlap step k's cross-section (main stream), the read-back runs on
        # a third stream; a buffer is refilled once its previous cross-section is done and sigma is
        # overwritten once its read-back is done
        def twin(d):
            return {k: (torch.empty_like(v) if isinstance(v, torch.Tensor) else v) for k, v in d.items()}
        raw_b, lines_b = [raw, twin(raw)], [lines, twin(lines)]
        sort_b = [sort_ws, torch.empty_like(sort_ws)]
        sigma_b = [sigma, torch.empty_like(sigma)]
        host_b = [sigma_host, torch.empty_like(sigma_host).pin_memory()]
        main_s, copy_s, d2h_s = torch.cuda.current_stream(), torch.cuda.Stream(), torch.cuda.Stream()
        up_ev = [torch.cuda.Event() for _ in range(2)]
        comp_ev = [torch.cuda.Event() for _ in range(2)]
        d2h_ev = [torch.cuda.Event() for _ in range(2)]

        def upload(b):
            copy_s.wait_event(comp_ev[b])
            with torch.cuda.stream(copy_s):
                for k, v in pinned.items():
                    raw_b[b][k].copy_(v, non_blocking=True)
                rox.rox_sort_lines(raw_b[b], lines_b[b], None, sort_b[b], stream=copy_s)
            up_ev[b].record(copy_s)

        def compute(b):
            main_s.wait_event(up_ev[b])
            main_s.wait_event(d2h_ev[b])
            rox.rox_xsec(lines_b[b], grid, P, T, Qt, Qr, w.mass_amu, w.cutoff, sigma_b[b], ws)
            comp_ev[b].record(main_s)
            d2h_s.wait_event(comp_ev[b])
            with torch.cuda.stream(d2h_s):
                host_b[b].copy_(sigma_b[b], non_blocking=True)
            d2h_ev[b].record(d2h_s)

        def e2e_run(k_steps):
            upload(0)
            for i in range(k_steps):
                if i + 1 < k_steps:
                    upload((i + 1) % 2)
                compute(i % 2)
            main_s.wait_event(d2h_ev[(k_steps - 1) % 2])

        for b in range(2):
            comp_ev[b].record(main_s)
            d2h_ev[b].record(main_s)
        e2e_run(max(2, args.warmup))
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(main_s)
        copy_s.wait_event(e0)
        e2e_run(e2e_steps)
        e1.record(main_s)
        barrier()
        e2e_ms = e0.elapsed_time(e1)
    else:
        for _ in range(max(1, args.warmup // 2) if e2e_steps else 0):
            upload_and_sort()
            step()
            sigma_host.copy_(sigma, non_blocking=True)
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(e2e_steps):
            upload_and_sort()
            step()
            sigma_host.copy_(sigma, non_blocking=True)
        e1.record()
        barrier()
        e2e_ms = e0.elapsed_time(e1)
    if dist is not None:
        tt = torch.tensor([e2e_ms], device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        e2e_ms = float(tt.item())
    e2e_value = world * evals * e2e_steps / (e2e_ms * 1e-3) if e2e_steps else None
    if e2e_steps:
        assert np.isfinite(sigma_host.numpy()).all()

    csum = clocks.summary()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peak = sms * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12
    v_ms = statistics.mean(voigt_ms)
    achieved = evals * FLOPS_PER_EVAL / (v_ms * 1e-3) / 1e12
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": VOIGT_TRAFFIC_BYTES if (args.config == 2 and args.lines is None and not args.nodes) else None,
            "traffic_note": "ncu capture of the 2e6-line case scaled by evaluations", "kernel": "k_voigt",
            "kernel_ms": v_ms,
            "peak_basis": "%d SMs x 128 FP32 lanes x 2 flop x %.0f MHz (max SM clock)" % (sms, SM_MAX_MHZ),
            "flops_per_eval": FLOPS_PER_EVAL}
    if csum.get("sm_mhz"):
        roof["frac_at_median_clock"] = achieved / (sms * FP32_LANES_PER_SM * 2 * csum["sm_mhz"] * 1e6 / 1e12)

    ws_mb = ws.numel() / 1e6
    sigma_bytes = sigma.numel() * 4
    serving = None
    if rank == 0 and world == 1 and not args.no_serve:
        del lines, raw, ws, sort_ws
        torch.cuda.empty_cache()
        serving = serving_leg([float(r) for r in args.serve_rates.split(",")], args.serve_seconds)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        Ls = oracle.sort_lines(host)
        cpu = cpu_baseline(w, nodes_np if args.nodes else grid, P, T, q, Ls, args.cpu_seconds)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": (("%s: %d lines (%s-style), grid %g-%g cm^-1 at %g (%d points), cutoff %g "
                                         "cm^-1, (P,T)=(%g bar, %g K)") % (
                                             w.name, n, "ExoMol" if w.convention == 1 else "HITRAN", w.grid_lo, w.grid_hi,
                                             w.dnu, grid[2], w.cutoff, P, T)) if not args.nodes else (
                                   ("%s lines on user-provided nodes: %d lines (%s-style), fixed resolving power "
                                    "R = %g over %g-%g cm^-1 (%d nodes), cutoff %g cm^-1, (P,T)=(%g bar, %g K)") % (
                                       w.name, n, "ExoMol" if w.convention == 1 else "HITRAN", rs.FIXED_R, w.grid_lo,
                                       w.grid_hi, n_grid, w.cutoff, P, T)),
                           "evals_per_step": evals, "xsecs_per_s": world * args.steps / (ms * 1e-3),
                           "selection": None if args.select is None else {
                               "rel": args.select, "bin_width_cm": args.select_bin,
                               "note": "value counts the kept (line, point) pairs; xsecs_per_s is the like-for-like "
                                       "speed against the unselected run"},
                           "broadening": None if not args.broadening else (
                               "0.85 H2 (per-line columns 1.3 x gamma_ref, n_T - 0.1) + 0.15 He (table by J'' of "
                               "60 entries) + natural A/(4 pi c)"),
                           "step": ("rox_xsec_nodes_batch" if args.nodes else
                                    "rox_xsec_select_batch" if args.select is not None else
                                    "rox_xsec_broadened_batch" if args.broadening else "rox_xsec") +
                                   " on the resident nu0-sorted list (strengths, widths, windows, tile "
                                   "ranges, Voigt accumulate); the once-per-list sort is inside e2e",
                           "l2": "inputs larger than L2 (line list %.0f MB, workspace %.0f MB)" % (
                               h2d_bytes / 1e6, ws_mb),
                           "parallelism": "replicas" if world > 1 else "single GPU",
                           "launch_config": launch_cfg, "launch_config_tuned": tuned},
                "roofline": roof, "cpu_baseline": cpu, "serving": serving,
                "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d_bytes,
                        "d2h_bytes_per_step": sigma_bytes,
                        "ms_per_step": e2e_ms / e2e_steps if e2e_steps else None,
                        "includes": "H2D of the unsorted list%s, rox_sort_lines, %s, D2H of sigma%s" % (
                            " and the nodes" if args.nodes else "", "rox_xsec_nodes_batch" if args.nodes else "rox_xsec",
                            "; two list buffers, step k+1's upload and sort overlap step k's cross-section"
                            if pipelined else "")},
                "gpu_launches": args.steps * 6 if args.select is None else args.steps * 9,
                "gpu_launches_note": (
                    "per step: windows, strengths, line bins, bin maxima, FP64 fix-up of the bin maxima, "
                    "selection and scaling, kept flags, span ranges over the kept lines, Voigt kernel (+ CUB's "
                    "two select kernels and memsets)" if args.select is not None else
                    "per step: %swindows, strengths, strength scaling, %stile ranges, %sVoigt kernel "
                    "(+ memsets)" % ("node offsets, " if args.nodes else "", "broadening, " if args.broadening else "",
                                     "" if args.nodes or args.broadening else "per-line constants, ")),
                "clocks": csum}
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


# ------------------------------------------------------------------ roofline helpers
def fp32_peaks(dev_index, sms):
    """The Voigt kernel's roofline denominators: the formula peak (SMs x 128 FP32 lanes x 2 flop x
    the maximum SM clock) and the FMA rate the probe kernel (include/rox.h rox_fp32_probe) sustains on
    this GPU, timed with CUDA events while nvidia-smi samples the SM clock."""
    import torch
    from paper_2510_20870_gb300 import _binding as rb
    nb = sms * 4
    out = torch.empty(rb.rox_fp32_probe_out_size(nb) // 4, dtype=torch.float32, device="cuda")
    rb.rox_fp32_probe(nb, 100, out)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(dev_index) as clk:
        time.sleep(0.25)
        e0.record()
        fma = sum(rb.rox_fp32_probe(nb, 200_000, out) for _ in range(6))
        e1.record()
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    c = clk.summary()
    meas = 2.0 * fma / (ms * 1e-3) / 1e12
    res = {"formula_tflops": sms * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12,
           "formula_basis": "%d SMs x 128 FP32 lanes x 2 flop x %.0f MHz (max SM clock)" % (sms, SM_MAX_MHZ),
           "measured_tflops": meas, "measured_ms": ms, "measured_sm_mhz": c.get("sm_mhz"),
           "measured_basis": "rox_fp32_probe: %d blocks x 256 threads x 16 FMA chains, %.3g FMAs in %.1f ms "
                             "(CUDA events)" % (nb, fma, ms)}
    if c.get("sm_mhz"):
        res["measured_fma_per_sm_clock"] = fma / (ms * 1e-3) / (sms * c["sm_mhz"] * 1e6)
    res.update(loop_ceilings(dev_index, sms, out))
    return res


def loop_ceilings(dev_index, sms, out):
    """The attainable rate of the Voigt kernel's inner loop: its pass-1 pair loop run alone
    (rox_pair_loop_probe), timed with CUDA events while nvidia-smi samples the SM clock."""
    import torch
    from paper_2510_20870_gb300 import _binding as rb
    nb = sms * 3
    rb.rox_pair_loop_probe(nb, 10, out)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(dev_index) as clk:
        time.sleep(0.1)
        e0.record()
        ev = sum(rb.rox_pair_loop_probe(nb, 1_000, out) for _ in range(20))
        e1.record()
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    mhz = clk.summary().get("sm_mhz")
    res = {"pair_loop_evals_s": ev / (ms * 1e-3),
           "pair_loop_basis": "rox_pair_loop_probe: %d blocks x 256 threads, %.3g evaluations in %.1f ms (CUDA "
                              "events), SM clock %s MHz" % (nb, ev, ms, mhz)}
    if mhz:
        res["pair_loop_evals_per_sm_clock"] = ev / (ms * 1e-3) / (sms * mhz * 1e6)
    return res


def voigt_roofline(evals, kernel_ms, peaks, traffic, traffic_note, clocks):
    achieved = evals * FLOPS_PER_EVAL / (kernel_ms * 1e-3) / 1e12
    peak = peaks["formula_tflops"]
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": traffic, "traffic_note": traffic_note, "kernel": "k_voigt", "kernel_ms": kernel_ms,
            "peak_basis": peaks["formula_basis"], "flops_per_eval": FLOPS_PER_EVAL,
            "peak_measured": peaks["measured_tflops"], "frac_of_measured": achieved / peaks["measured_tflops"],
            "peak_measured_basis": peaks["measured_basis"], "peak_measured_sm_mhz": peaks.get("measured_sm_mhz")}
    if peaks.get("pair_loop_evals_s"):
        roof["pair_loop_ceiling_evals_s"] = peaks["pair_loop_evals_s"]
        roof["frac_of_pair_loop"] = evals / (kernel_ms * 1e-3) / peaks["pair_loop_evals_s"]
        roof["pair_loop_basis"] = peaks["pair_loop_basis"]
    if clocks.get("sm_mhz"):
        roof["frac_at_median_clock"] = achieved / (peak * clocks["sm_mhz"] / SM_MAX_MHZ)
    return roof


def oracle_subsample(w, n_sub=1_000_000):
    """Host lines for the oracle legs: the whole list up to 1e7 lines, else its first n_sub lines
    (generation indices 0..n_sub-1, regenerated on the host), sorted by nu0."""
    import oracle
    n = w.n_lines if w.n_lines <= 10_000_000 else n_sub
    return oracle.sort_lines(rs.make_lines(w, 0, n)), n


# ------------------------------------------------------------------ the large list (default workload)
def run_large(args):
    """Config 4: 1e9 lines held on the device as nu0-sorted chunks, one cross-section per step."""
    import torch
    import paper_2510_20870_gb300 as rox
    from rox_synth.device import alloc_lines, make_lines_device

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count

    w = rs.CONFIGS[4]
    grid = rs.grid_of(w)
    (P, T), = w.pts
    q = rs.q_table(w)
    Qt, Qr = q_of(q, T), q_of(q, 296.0)
    n = args.lines or w.n_lines
    chunk = min(n, args.chunk)
    starts = list(range(0, n, chunk))
    cols = ["nu0", "s_or_a", "e_lower", "gamma_ref", "n_t"]
    do_e2e = not args.no_e2e

    # resident sorted chunks (the timed step's input) and, for the end-to-end leg, the unsorted
    # chunks in pinned host memory
    sort_ws = torch.empty(rox.rox_sort_workspace_size(chunk), dtype=torch.uint8, device=dev)
    resident, host = [], []
    for s0 in starts:
        cnt = min(chunk, n - s0)
        raw = make_lines_device(w, s0, cnt)
        if do_e2e:
            hp = {k: torch.empty(raw[k].shape, dtype=raw[k].dtype, pin_memory=True) for k in cols}
            for k in cols:
                hp[k].copy_(raw[k])
            host.append(hp)
        out = {k: torch.empty_like(raw[k]) for k in cols}
        out["g_up"], out["convention"] = None, w.convention
        rox.rox_sort_lines(raw, out, None, sort_ws)
        resident.append(out)
        del raw
    torch.cuda.synchronize()
    line_bytes = sum(v.numel() * v.element_size() for L in resident for k, v in L.items() if k in cols)
    ws = torch.empty(rox.rox_xsec_workspace_size(chunk, grid, 1), dtype=torch.uint8, device=dev)
    sigma = torch.empty((1, grid[2]), dtype=torch.float32, device=dev)
    from paper_2510_20870_gb300 import autotune
    launch_cfg, tuned = autotune.apply("large")

    def step(evs=None, lines=resident, stream=None):
        for c, L in enumerate(lines):
            if evs is not None:
                rox.rox_set_profile_events(*evs[c])
            rox.rox_xsec_batch(L, grid, [P], [T], [Qt], Qr, w.mass_amu, w.cutoff, sigma, ws,
                               flags=(rox.ROX_ACCUMULATE if c else 0) | rox.ROX_KAHAN, stream=stream)
        if evs is not None:
            rox.rox_set_profile_events(None, None)

    # exact evaluation count of one step (the status call synchronises, so outside the timing)
    evals = 0
    for c, L in enumerate(resident):
        rox.rox_xsec_batch(L, grid, [P], [T], [Qt], Qr, w.mass_amu, w.cutoff, sigma, ws,
                           flags=(rox.ROX_ACCUMULATE if c else 0) | rox.ROX_KAHAN)
        rc, ev = rox.rox_ws_status(ws)
        if rc != 0:
            raise RuntimeError(rox.lib.rox_last_error().decode())
        evals += ev

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        step()
    ev_pairs = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in starts]
                for _ in range(args.steps)]
    for pairs in ev_pairs:
        for a, b in pairs:
            a.record()
            b.record()
    barrier()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clocks:
        time.sleep(0.3)
        barrier()
        t0.record()
        for pairs in ev_pairs:
            step(pairs)
        t1.record()
        barrier()
    ms = t0.elapsed_time(t1)
    voigt_ms = [sum(a.elapsed_time(b) for a, b in pairs) for pairs in ev_pairs]
    if dist is not None:
        tt = torch.tensor([ms], device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        ms = float(tt.item())
    value = world * evals * args.steps / (ms * 1e-3)
    sig_max = float(sigma.max())
    csum = clocks.summary()

    # ---- end to end through the public API: every step uploads the unsorted chunks from pinned
    # host memory (chunk c+1's upload and sort on a copy stream overlap chunk c's cross-section),
    # sorts them (rox_sort_lines), adds each chunk's cross-section into sigma and reads sigma back
    e2e = None
    if do_e2e:
        bufs = [alloc_lines(w, chunk, device=dev) for _ in range(2)]
        sbufs = [{k: torch.empty_like(b[k]) for k in cols} for b in bufs]
        for sb in sbufs:
            sb["g_up"], sb["convention"] = None, w.convention
        sort_b = [sort_ws, torch.empty_like(sort_ws)]
        sigma_h = torch.empty((1, grid[2]), dtype=torch.float32, pin_memory=True)
        main_s, copy_s = torch.cuda.current_stream(), torch.cuda.Stream()
        up_ev = [torch.cuda.Event() for _ in range(2)]
        comp_ev = [torch.cuda.Event() for _ in range(2)]
        for b in range(2):
            comp_ev[b].record(main_s)

        def upload(c):
            b = c % 2
            cnt = min(chunk, n - starts[c])
            copy_s.wait_event(comp_ev[b])
            with torch.cuda.stream(copy_s):
                raw = {k: bufs[b][k][:cnt] for k in cols}
                for k in cols:
                    raw[k].copy_(host[c][k], non_blocking=True)
                raw["g_up"], raw["convention"] = None, w.convention
                out = {k: sbufs[b][k][:cnt] for k in cols}
                out["g_up"], out["convention"] = None, w.convention
                rox.rox_sort_lines(raw, out, None, sort_b[b], stream=copy_s)
            up_ev[b].record(copy_s)
            return out

        def e2e_step():
            cur = upload(0)
            for c in range(len(starts)):
                nxt = upload(c + 1) if c + 1 < len(starts) else None
                main_s.wait_event(up_ev[c % 2])
                rox.rox_xsec_batch(cur, grid, [P], [T], [Qt], Qr, w.mass_amu, w.cutoff, sigma, ws,
                                   flags=(rox.ROX_ACCUMULATE if c else 0) | rox.ROX_KAHAN)
                comp_ev[c % 2].record(main_s)
                cur = nxt
            sigma_h.copy_(sigma, non_blocking=True)

        e2e_step()
        barrier()
        n_e2e = max(1, min(args.steps, 3))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(main_s)
        copy_s.wait_event(e0)
        for _ in range(n_e2e):
            e2e_step()
        e1.record(main_s)
        barrier()
        e2e_ms = e0.elapsed_time(e1)
        if dist is not None:
            tt = torch.tensor([e2e_ms], device=dev)
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
            e2e_ms = float(tt.item())
        assert np.isfinite(sigma_h.numpy()).all()
        h2d = sum(v.numel() * v.element_size() for hp in host for v in hp.values())
        e2e = {"value": world * evals * n_e2e / (e2e_ms * 1e-3), "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": sigma_h.numel() * 4, "ms_per_step": e2e_ms / n_e2e, "steps": n_e2e,
               "includes": "per step: H2D of the %d unsorted chunks from pinned host memory, rox_sort_lines and "
                           "rox_xsec_batch (ROX_ACCUMULATE) per chunk, D2H of sigma; chunk c+1's upload and sort "
                           "overlap chunk c's cross-section" % len(starts)}
        del bufs, sbufs, sort_b, host
    del resident, ws, sort_ws
    torch.cuda.empty_cache()

    peaks = fp32_peaks(local, sms)
    roof = voigt_roofline(evals, statistics.mean(voigt_ms), peaks,
                          VOIGT_TRAFFIC_LARGE * evals if VOIGT_TRAFFIC_LARGE else None,
                          "ncu dram__bytes_read + write of k_voigt on one 1e7-line chunk of this workload, per "
                          "evaluation, times this step's evaluations (the kernel reads each line once per span it "
                          "reaches; the traffic grows with the evaluations)", csum)
    roof["kernel_ms_note"] = "sum over the %d chunk launches of one step (CUDA events around each launch)" % len(starts)

    extra2 = None
    if rank == 0 and world == 1 and not args.no_config2:
        extra2 = config2_summary(args, peaks)
    serving = None
    if rank == 0 and world == 1 and not args.no_serve:
        serving = serving_leg([float(r) for r in args.serve_rates.split(",")], args.serve_seconds)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        Ls, n_sub = oracle_subsample(w)
        cpu = cpu_baseline(w, grid, P, T, q, Ls, args.cpu_seconds)
        cpu["sample"] = "lines 0..%d of the large list (its 1e6-line subsample, all of them within the cutoff of " \
                        "each window); " % (n_sub - 1) + cpu["sample"]

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": "large: %d HITRAN-style lines (f16 widths, 20 B per line) as %d device-resident "
                                       "nu0-sorted chunks, grid %g-%g cm^-1 at %g (%d points), cutoff %g cm^-1, "
                                       "(P,T)=(%g bar, %g K)" % (n, len(starts), w.grid_lo, w.grid_hi, w.dnu, grid[2],
                                                                 w.cutoff, P, T),
                           "evals_per_step": evals, "xsecs_per_s": world * args.steps / (ms * 1e-3),
                           "step": "rox_xsec_batch per chunk (strengths, windows, span ranges, per-line constants, "
                                   "Voigt accumulate), flags ROX_KAHAN, chunks after the first also ROX_ACCUMULATE",
                           "l2": "inputs larger than L2 (line list %.1f GB)" % (line_bytes / 1e9),
                           "sigma_max": sig_max, "parallelism": "replicas" if world > 1 else "single GPU",
                           "launch_config": launch_cfg,
                           "launch_config_source": "autotuner cache (paper_2510_20870_gb300/tuning.json)" if tuned
                                                   else "library default (no cache entry for this GPU)"},
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "config2": extra2, "serving": serving,
                "gpu_launches": args.steps * 6 * len(starts),
                "gpu_launches_note": "per chunk: windows, strengths, strength scaling, span ranges, per-line "
                                     "constants, Voigt kernel (+ memsets)",
                "clocks": csum}
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


def config2_summary(args, peaks):
    """The single-(P,T) exomol workload (1e7 lines, 2,970,001 points), timed like the main run, as a
    second figure beside the large list."""
    import torch
    import paper_2510_20870_gb300 as rox
    from rox_synth.device import make_lines_device
    from paper_2510_20870_gb300 import autotune
    w, grid, P, T, q = workload(2)
    Qt, Qr = q_of(q, T), q_of(q, 296.0)
    launch_cfg, tuned = autotune.apply("exomol")
    raw = make_lines_device(w, 0, w.n_lines)
    lines = {k: (torch.empty_like(v) if isinstance(v, torch.Tensor) else v) for k, v in raw.items()}
    sws = torch.empty(rox.rox_sort_workspace_size(w.n_lines), dtype=torch.uint8, device="cuda")
    rox.rox_sort_lines(raw, lines, None, sws)
    del raw, sws
    ws = torch.empty(rox.rox_xsec_workspace_size(w.n_lines, grid, 1), dtype=torch.uint8, device="cuda")
    sigma = torch.empty((1, grid[2]), dtype=torch.float32, device="cuda")
    rox.rox_xsec(lines, grid, P, T, Qt, Qr, w.mass_amu, w.cutoff, sigma, ws)
    rc, evals = rox.rox_ws_status(ws)
    for _ in range(args.warmup):
        rox.rox_xsec(lines, grid, P, T, Qt, Qr, w.mass_amu, w.cutoff, sigma, ws)
    steps = max(args.steps, 10)
    pairs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for a, b in pairs:
        a.record()
        b.record()
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record()
    for a, b in pairs:
        rox.rox_set_profile_events(a, b)
        rox.rox_xsec(lines, grid, P, T, Qt, Qr, w.mass_amu, w.cutoff, sigma, ws)
    rox.rox_set_profile_events(None, None)
    t1.record()
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1) / steps
    kms = statistics.mean(a.elapsed_time(b) for a, b in pairs)
    # the same step with plain (uncompensated) summation of the partial sums
    t0.record()
    for _ in range(steps):
        rox.rox_xsec_batch(lines, grid, [P], [T], [Qt], Qr, w.mass_amu, w.cutoff, sigma, ws, flags=0)
    t1.record()
    torch.cuda.synchronize()
    ms_plain = t0.elapsed_time(t1) / steps
    del lines, ws, sigma
    torch.cuda.empty_cache()
    return {"workload": "exomol: %d lines, grid %d points, cutoff %g cm^-1, (P,T)=(%g bar, %g K)" % (
                w.n_lines, grid[2], w.cutoff, P, T),
            "value": evals / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms, "steps": steps, "status": rc,
            "kernel_ms": kms, "xsecs_per_s": 1e3 / ms, "summation": "compensated (ROX_KAHAN)",
            "ms_per_step_plain_sum": ms_plain, "launch_config": launch_cfg, "launch_config_tuned": tuned,
            "roofline_frac": evals * FLOPS_PER_EVAL / (kms * 1e-3) / 1e12 / peaks["formula_tflops"]}


# ------------------------------------------------------------------ other workloads (documentation runs)
def _sorted_device_lines(w, start, count, stream=None):
    import torch
    import paper_2510_20870_gb300 as rox
    from rox_synth.device import make_lines_device
    raw = make_lines_device(w, start, count, stream=stream)
    out = {k: (torch.empty_like(v) if isinstance(v, torch.Tensor) else v) for k, v in raw.items()}
    ws = torch.empty(rox.rox_sort_workspace_size(count), dtype=torch.uint8, device="cuda")
    rox.rox_sort_lines(raw, out, None, ws, stream=stream)
    return out, (raw, ws)


def run_batch_config(args):
    """Config 3: 1e8 lines, 15 P x 20 T = 300 cross-sections in one persistent launch (about 52 s
    a step on GB300, so not the default workload: the default K = 20, W = 5 would hold the GPU for
    about 20 minutes). Same keys as the default line; the end-to-end leg uploads the unsorted list
    from pinned memory, sorts it, computes the 300 cross-sections and reads the 3.56 GB back."""
    import torch
    import paper_2510_20870_gb300 as rox
    from paper_2510_20870_gb300 import autotune
    from rox_synth.device import make_lines_device
    w = rs.CONFIGS[3]
    grid = rs.grid_of(w)
    pts = rs.pt_points(w)
    n = args.lines or w.n_lines
    q = rs.q_table(w)
    Qr = q_of(q, 296.0)
    launch_cfg, tuned = autotune.apply("batch")
    raw = make_lines_device(w, 0, n)
    cols = [k for k in ("nu0", "s_or_a", "g_up", "e_lower", "gamma_ref", "n_t") if raw.get(k) is not None]
    host = {k: torch.empty(raw[k].shape, dtype=raw[k].dtype, pin_memory=True) for k in cols}
    for k in cols:
        host[k].copy_(raw[k])
    lines = {k: (torch.empty_like(v) if isinstance(v, torch.Tensor) else v) for k, v in raw.items()}
    sort_ws = torch.empty(rox.rox_sort_workspace_size(n), dtype=torch.uint8, device="cuda")
    rox.rox_sort_lines(raw, lines, None, sort_ws)
    n_temps = len(set(T for _, T in pts))
    ws = torch.empty(rox.rox_xsec_workspace_size(n, grid, n_temps), dtype=torch.uint8, device="cuda")
    sigma = torch.empty((len(pts), grid[2]), dtype=torch.float32, device="cuda")
    P = [p for p, _ in pts]
    T = [t for _, t in pts]
    Q = [q_of(q, t) for t in T]

    def step(L=lines):
        rox.rox_xsec_batch(L, grid, P, T, Q, Qr, w.mass_amu, w.cutoff, sigma, ws, flags=rox.ROX_KAHAN)
    step()
    rc, evals = rox.rox_ws_status(ws)
    for _ in range(args.warmup):
        step()
    pairs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for a_, b_ in pairs:
        a_.record()
        b_.record()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(0) as clocks:
        e0.record()
        for a_, b_ in pairs:
            rox.rox_set_profile_events(a_, b_)
            step()
        rox.rox_set_profile_events(None, None)
        e1.record()
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    kms = statistics.mean(a_.elapsed_time(b_) for a_, b_ in pairs)
    csum = clocks.summary()
    e2e = None
    if not args.no_e2e:
        sigma_h = torch.empty(sigma.shape, dtype=torch.float32, pin_memory=True)
        e0.record()
        for k in cols:
            raw[k].copy_(host[k], non_blocking=True)
        rox.rox_sort_lines(raw, lines, None, sort_ws)
        step()
        sigma_h.copy_(sigma, non_blocking=True)
        e1.record()
        torch.cuda.synchronize()
        ms_e = e0.elapsed_time(e1)
        e2e = {"value": evals / (ms_e * 1e-3), "unit": UNIT, "ms_per_step": ms_e, "steps": 1,
               "h2d_bytes_per_step": int(sum(v.numel() * v.element_size() for v in host.values())),
               "d2h_bytes_per_step": int(sigma_h.numel() * 4),
               "includes": "H2D of the unsorted list from pinned memory, rox_sort_lines, rox_xsec_batch at 300 (P,T), "
                           "D2H of all 300 cross-sections"}
    del raw, lines, ws, sigma, sort_ws
    torch.cuda.empty_cache()
    peaks = fp32_peaks(0, torch.cuda.get_device_properties(0).multi_processor_count)
    roof = voigt_roofline(evals, kms, peaks, None, "not captured for this workload", csum)
    cpu = None
    if not args.no_cpu_baseline:
        import multiprocessing as mp
        Ls, n_sub = oracle_subsample(w)
        cores = len(os.sched_getaffinity(0))
        rng = np.random.default_rng(13)
        tasks = []
        for k in range(8 * cores):
            Pk, Tk = pts[int(rng.integers(0, len(pts)))]
            tasks += oracle_sample_tasks(Ls, grid, Pk, Tk, q_oracle(q, Tk), q_oracle(q, 296.0), w.mass_amu, w.cutoff,
                                         1, 256, 1000 + k)
        ev, dt = time_oracle(tasks, cores)
        cpu = {"value": ev / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": "%d random 256-point windows, each at one of the 300 (P,T) points drawn at random, on the "
                         "first %d lines of the batch list (all of them within the cutoff of each window), FP64 "
                         "scipy.special.wofz, %d evals in %.1f s" % (len(tasks), n_sub, ev, dt)}
    print(json.dumps({"metric": METRIC, "value": evals / (ms * 1e-3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
                      "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                      "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                      "config": {"workload": "batch: %d lines (ExoMol-style), %d (P,T) points (15 P x 20 T) in one "
                                             "persistent launch, grid %d points, cutoff %g" % (n, len(pts), grid[2],
                                                                                              w.cutoff),
                                 "evals_per_step": evals, "xsecs_per_s": len(pts) / (ms * 1e-3), "status": rc,
                                 "launch_config": launch_cfg, "launch_config_tuned": tuned,
                                 "l2": "inputs larger than L2 (line list %.1f GB, output 3.56 GB)" % (n * 28 / 1e9)},
                      "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": args.steps * 5,
                      "gpu_launches_note": "per step: windows, strengths (20 temperatures), strength scaling, span "
                                           "ranges, Voigt kernel over 300 (P,T) (+ memsets)",
                      "clocks": csum}))


def run_cia(args):
    """CIA restructuring: synthetic coefficient blocks of 40 temperatures (1-3 blocks each, 4000
    samples per temperature over 20-10000 cm^-1) onto config 2's grid, 2,970,001 points per row."""
    import torch
    import paper_2510_20870_gb300 as rox
    grid = rs.grid_of(rs.CONFIGS[2])
    temps = list(np.linspace(200.0, 3000.0, 40))
    Tb, off, nu_h, k_h = rs.cia_blocks(60, temps, samples=4000)
    nu, k = torch.from_numpy(nu_h).cuda(), torch.from_numpy(k_h).cuda()
    out = torch.empty((len(temps), grid[2]), dtype=torch.float64, device="cuda")
    ws = torch.empty(rox.rox_cia_workspace_size(len(Tb), nu_h.size), dtype=torch.uint8, device="cuda")
    for _ in range(args.warmup):
        rox.rox_cia_regrid(Tb, off, nu, k, grid, temps, out, ws)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(0) as clocks:
        e0.record()
        for _ in range(args.steps):
            rox.rox_cia_regrid(Tb, off, nu, k, grid, temps, out, ws)
        e1.record()
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    points = len(temps) * grid[2]
    out_bytes = points * 8
    e2e = None
    if not args.no_e2e:
        # through the public call from pinned host memory: the blocks in, the rows out, every step
        nu_p = torch.from_numpy(nu_h).pin_memory()
        k_p = torch.from_numpy(k_h).pin_memory()
        out_p = torch.empty(out.shape, dtype=torch.float64).pin_memory()
        n_e2e = max(3, min(args.steps, 50))

        def e2e_step():
            nu.copy_(nu_p, non_blocking=True)
            k.copy_(k_p, non_blocking=True)
            rox.rox_cia_regrid(Tb, off, nu, k, grid, temps, out, ws)
            out_p.copy_(out, non_blocking=True)
        e2e_step()
        torch.cuda.synchronize()
        e0.record()
        for _ in range(n_e2e):
            e2e_step()
        e1.record()
        torch.cuda.synchronize()
        ms_e = e0.elapsed_time(e1) / n_e2e
        assert np.array_equal(out_p.numpy(), out.cpu().numpy())
        e2e = {"value": points / (ms_e * 1e-3), "unit": "points/s", "h2d_bytes_per_step": int(nu_h.nbytes + k_h.nbytes),
               "d2h_bytes_per_step": int(out_bytes), "ms_per_step": ms_e, "steps": n_e2e,
               "includes": "H2D of the blocks from pinned memory, rox_cia_regrid, D2H of all rows to pinned memory"}
    cpu = None
    if not args.no_cpu_baseline:
        # the oracle (numpy, one thread): the whole workload, repeated for about 10 s
        import oracle
        nodes = oracle.grid_nodes(*grid)
        per_nu = [nu_h[off[b]:off[b + 1]] for b in range(len(Tb))]
        per_k = [k_h[off[b]:off[b + 1]] for b in range(len(Tb))]
        reps, t0 = 0, time.perf_counter()
        while reps == 0 or time.perf_counter() - t0 < 10.0:
            oracle.cia_regrid(Tb, per_nu, per_k, temps, nodes)
            reps += 1
        dt = time.perf_counter() - t0
        cpu = {"value": reps * points / dt, "unit": "points/s", "cores": 1, "kind": "oracle",
               "sample": "the whole workload (%d temperatures x %d points) %d times (numpy, one thread), %.1f s" % (
                   len(temps), grid[2], reps, dt)}
    peak = json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")))["hbm_gbs"] \
        if os.path.exists(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")) else 6800.0
    achieved = out_bytes / (ms * 1e-3) / 1e9
    print(json.dumps({"metric": "CIA grid points/s", "value": points / (ms * 1e-3), "unit": "points/s", "n_gpus": 1,
                      "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
                      "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                      "config": {"workload": "CIA restructuring: %d temperatures (%d blocks, %d samples) onto %d "
                                             "points (300-30000 cm^-1 at 0.01)" % (len(temps), len(Tb), nu_h.size,
                                                                                   grid[2]),
                                 "l2": "output %.0f MB per step, larger than L2" % (out_bytes / 1e6)},
                      "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                                   "frac": achieved / peak, "traffic": CIA_TRAFFIC_BYTES, "kernel": "k_cia_grid",
                                   "peak_basis": "measured copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
                                   "note": "algorithmic bytes: the float64 output written once (inputs %.1f MB, "
                                           "L2-resident), over the whole step (per-sample interval pass + "
                                           "grid kernel)" % ((nu_h.size * 16) / 1e6)},
                      "gpu_launches": 2 * args.steps, "clocks": clocks.summary(), "cpu_baseline": cpu, "e2e": e2e}))


def run_autotune(args):
    """Sweeps the launch configuration on one 1e8-line chunk of the large list, on the exomol
    list and on the batch list (1e8 lines; every eleventh of its 300 (P,T) points, so one candidate
    takes seconds, with the same line density and the same mix of widths), writes the cache
    (paper_2510_20870_gb300/tuning.json) and prints the results."""
    import torch
    import paper_2510_20870_gb300 as rox
    from paper_2510_20870_gb300 import autotune
    from rox_synth.device import make_lines_device
    out = {}
    for cls, cid, n in (("large", 4, 100_000_000), ("exomol", 2, None), ("batch", 3, None)):
        w = rs.CONFIGS[cid]
        grid = rs.grid_of(w)
        pts = rs.pt_points(w)[::11]
        P, T = [p for p, _ in pts], [t for _, t in pts]
        q = rs.q_table(w)
        Qt, Qr = [q_of(q, t) for t in T], q_of(q, 296.0)
        n = n or w.n_lines
        raw = make_lines_device(w, 0, n)
        lines = {k: (torch.empty_like(v) if isinstance(v, torch.Tensor) else v) for k, v in raw.items()}
        sws = torch.empty(rox.rox_sort_workspace_size(n), dtype=torch.uint8, device="cuda")
        rox.rox_sort_lines(raw, lines, None, sws)
        del raw, sws
        ws = torch.empty(rox.rox_xsec_workspace_size(n, grid, len(set(T))), dtype=torch.uint8, device="cuda")
        sigma = torch.empty((len(pts), grid[2]), dtype=torch.float32, device="cuda")

        def step():
            rox.rox_xsec_batch(lines, grid, P, T, Qt, Qr, w.mass_amu, w.cutoff, sigma, ws, flags=rox.ROX_KAHAN)
        res = autotune.sweep(step, reps=5 if cid == 2 else (1 if cid == 3 else 2))
        best = autotune.save(cls, res, note="%s: %d lines, %d (P,T) point(s), one rox_xsec_batch call" % (
            w.name, n, len(pts)))
        out[autotune.key(cls)] = {"best": best, "results": [{"config": c, "ms": ms} for c, ms in res]}
        del lines, ws, sigma
        torch.cuda.empty_cache()
    print(json.dumps({"autotune": out, "cache": autotune.CACHE}))


def main():
    args = parse()
    if args.autotune:
        run_autotune(args)
        return
    if args.probes:
        import torch
        torch.cuda.set_device(0)
        sms = torch.cuda.get_device_properties(0).multi_processor_count
        print(json.dumps({"probes": fp32_peaks(0, sms), "device": torch.cuda.get_device_name(0)}))
        return
    if args.impl == "reference":
        run_reference(args)
    elif args.cia:
        run_cia(args)
    elif args.config == 3:
        run_batch_config(args)
    elif args.config == 4:
        run_large(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
