"""Benchmark: the Pregel superstep hot path on the billion-edge workload.

One step = PageRank (10 supersteps, FP32, pull) + SSSP from the max-out-degree vertex
(u32 weights in [1,255], push with a min combiner) on a directed R-MAT graph of scale
26 and edge factor 28 (1.84e9 edges after self-loop and duplicate removal, seed 1),
synthetic input standing in for the paper's billion-edge Friendster graph.

value      edges traversed per second (PageRank: 10 m; SSSP: messages sent), graph
           resident in HBM, timed with CUDA events on the library's stream.
e2e        the same metric through the host-buffer C ABI: ipg_graph_create from a host
           CSR in page-locked ipg_host_alloc memory (upload + in-edge build),
           ipg_pagerank and ipg_sssp into host arrays, ipg_graph_destroy, every step.
roofline   the dominant kernel's algorithmic bytes per launch / its mean CUDA-event
           duration, against the measured HBM copy bandwidth (frac) and the nominal
           7.9 TB/s (frac_of_nominal).
cpu_baseline  the CPU oracle (single thread) on a bounded sample of the same graph.
cpu_parallel  the paper's final design on all host cores (cpu_baseline/, OpenMP) on the
           same kind of sample, sized to about 10 s of wall time; reported, not targeted.

Multi-GPU: the path does not shard here; with --gpus N every rank runs its own replica
(scaling "weak"), value = all ranks' edges / the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "GTEPS (edges traversed per second: PageRank 10 supersteps + SSSP), per superstep roofline"
UNIT = "GTEPS"
PR_UPDATES = 10


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", choices=["billion", "pagerank16", "hashmin20", "batch", "cc-batch", "serve",
                                          "combiner"],
                   default="billion",
                   help="billion: the default bench line; pagerank16: PageRank on directed R-MAT 16/16; "
                        "hashmin20: Hashmin components on undirected R-MAT 20/16; "
                        "batch: 256-source batched SSSP vs one at a time; "
                        "cc-batch: 64 uneven Hashmin graphs in one object vs one at a time; "
                        "serve: Poisson stream of mixed queries on 32 resident graphs; "
                        "combiner: wide-message programs and the combination step alone")
    p.add_argument("--rate", type=float, default=2000.0, help="serve: mean arrivals per second")
    p.add_argument("--requests", type=int, default=10000, help="serve: measured requests (after 10%% warm-up)")
    p.add_argument("--batch-sources", type=int, default=256)
    p.add_argument("--min-sssp-batch", type=int, default=0,
                   help="serve: fewest queued SSSP queries that start a lane session (0: the library default, per graph)")
    p.add_argument("--scale", type=int, default=26)
    p.add_argument("--edge-factor", type=int, default=28)
    p.add_argument("--seed", type=int, default=1)
    p.add_argument("--e2e-steps", type=int, default=2)
    p.add_argument("--cpu-seconds", type=float, default=30.0,
                   help="calibration target for the oracle sample; the sample's SSSP part grows faster than "
                        "its size, so the measured time comes out at about half of it")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-other-configs", action="store_true",
                   help="default run: skip the compact lines of the other workloads after the timed region")
    p.add_argument("--pull-divisor", type=int, default=None,
                   help="Hashmin/SSSP direction knob (library default if omitted; 0 = always push)")
    p.add_argument("--no-autotune", action="store_true",
                   help="skip ipg_autotune (the graph then runs with the process-wide knobs)")
    p.add_argument("--tuning", action="append", default=[], metavar="NAME=VALUE",
                   help="set a library knob (ipg_set_tuning) before the run, e.g. batch_loop=0 for a "
                        "launch list in which every kernel of the batched loop is visible; repeatable")
    return p.parse_args()


def apply_tuning(a):
    """--tuning NAME=VALUE: process-wide library knobs, set before anything runs."""
    if not a.tuning:
        return
    import paper_2010_01542_gb300 as ipg

    ipg.load_library()
    for item in a.tuning:
        name, _, value = item.partition("=")
        ipg.ipg_set_tuning(name.strip(), int(value))


_CAPTURE = None  # a list while the default run collects the other workloads' lines


def emit(line):
    """Print a workload's JSON line, or keep it when the default run collects it."""
    if _CAPTURE is not None:
        _CAPTURE.append(line)
    else:
        print(json.dumps(line), flush=True)


def workload_name(a):
    return (f"rmat{a.scale}-ef{a.edge_factor} directed weighted[1,255] seed {a.seed}: "
            f"PageRank {PR_UPDATES} supersteps + SSSP from the max-out-degree vertex")


# ---------------------------------------------------------------------------------------
# distributed plumbing


def dist_init(a):
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch
        import torch.distributed as dist

        dist.barrier()
        if torch.cuda.is_available():
            torch.cuda.synchronize()


def all_max(x, world):
    """Max of x over the ranks (the slowest rank's time); works on nccl (CUDA tensor) and gloo."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(units_per_rank, ms_local, world):
    """Whole-job rate for replicas (weak scaling, no data-path collective): every rank
    processes units_per_rank; the job takes as long as its slowest rank."""
    ms = all_max(ms_local, world)
    return world * units_per_rank / (ms / 1e3), ms


# ---------------------------------------------------------------------------------------
# clocks


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix="clocks", suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------------------
# oracle sample (CPU baseline and the reference arm)


SAMPLE_BLOCK = 1024  # rows per sampled block


def strided_subgraph(g, edges):
    """A sample of g's source rows holding about `edges` edges, over all n vertices: blocks of
    SAMPLE_BLOCK consecutive rows, one block in every `stride`.  R-MAT puts its hubs at the
    lowest ids, so a prefix of rows would be all hubs; strided blocks take hub, middle and
    tail rows in their proportions.  Returns (rows kept, edges kept, offsets, columns, weights,
    description)."""
    n, m = g.n, g.m
    stride = max(1, int(round(m / max(edges, 1))))
    deg = np.diff(g.offsets.astype(np.int64))
    keep = (np.arange(n, dtype=np.int64) // SAMPLE_BLOCK) % stride == 0
    deg_s = np.where(keep, deg, 0)
    off = np.zeros(n + 1, dtype=np.uint64)
    np.cumsum(deg_s, out=off[1:])
    starts = np.arange(0, n, SAMPLE_BLOCK * stride, dtype=np.int64)
    ends = np.minimum(starts + SAMPLE_BLOCK, n)
    pieces = [(int(g.offsets[b]), int(g.offsets[e])) for b, e in zip(starts, ends)]
    cols = np.concatenate([g.cols[b:e] for b, e in pieces]) if pieces else g.cols[:0]
    w = None if g.weights is None else np.concatenate([g.weights[b:e] for b, e in pieces])
    rows = int(keep.sum())
    desc = (f"{rows} source rows ({int(off[-1])} edges) in blocks of {SAMPLE_BLOCK} rows, one block in every "
            f"{stride}, of the same graph, all n vertices")
    return rows, int(off[-1]), off, cols, w, desc


def sample_source(off, src):
    """SSSP source in the sample: src if its row was kept, else the kept row of most out-edges."""
    deg = np.diff(off.astype(np.int64))
    return src if deg[src] > 0 else int(np.argmax(deg))


def oracle_sample(g, src, edges):
    """Oracle PageRank (one update) + SSSP on the strided row sample; returns (edges traversed,
    seconds, description)."""
    import oracle

    _, _, off, cols, w, desc = strided_subgraph(g, edges)
    s0 = sample_source(off, src)
    t0 = time.perf_counter()
    pr = oracle.pagerank(g.n, off, cols, 1)
    ss = oracle.sssp(g.n, off, cols, w, s0)
    t = time.perf_counter() - t0
    traversed = sum(s.messages_sent for s in pr.stats) + sum(s.messages_sent for s in ss.stats)
    return traversed, t, desc


def calibrate_sample(g, src, seconds):
    edges = 20_000_000
    tr, t, _ = oracle_sample(g, src, edges)
    rate = tr / max(t, 1e-6)  # edges traversed per second
    per_edge = tr / max(edges, 1)
    return int(min(g.m, max(1_000_000, seconds * rate / max(per_edge, 1e-9))))


def cpu_baseline(g, src, seconds):
    edges = calibrate_sample(g, src, seconds)
    tr, t, desc = oracle_sample(g, src, edges)
    return {"value": tr / t / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"oracle PageRank (1 update) + SSSP to quiescence on {desc}; {tr} edges traversed "
                      f"in {t:.1f} s"}


def parallel_sample(g, src, edges):
    """The OpenMP baseline (cpu_baseline/) on the same kind of strided row sample as the oracle's:
    PageRank (one update, pull) + SSSP (push); returns (edges traversed, superstep seconds,
    edges kept, wall seconds, description)."""
    import cpu_baseline as omp_baseline

    _, mS, off, cols, w, desc = strided_subgraph(g, edges)
    t0 = time.perf_counter()
    pr = omp_baseline.pagerank(g.n, off, cols, 1)
    ss = omp_baseline.sssp(g.n, off, cols, w, sample_source(off, src))
    wall = time.perf_counter() - t0  # also the untimed in-edge build: it sizes the sample
    return pr.messages + ss.messages, pr.seconds + ss.seconds, mS, wall, desc


def cpu_parallel_baseline(g, src, seconds):
    """The paper's final design (pull PageRank, SSSP pushed from the active list into CAS
    mailboxes, OpenMP dynamic,256) on all host cores: a reported comparison point beside the
    single-threaded oracle.  Never fails the bench: any error becomes an `unavailable` entry."""
    try:
        import cpu_baseline as omp_baseline

        probe = 20_000_000
        _, _, mS, wall, _ = parallel_sample(g, src, probe)
        # size the sample so that its whole run (in-edge build + supersteps) takes about `seconds`
        edges = int(min(g.m, max(1_000_000, seconds * max(mS, 1) / max(wall, 1e-6))))
        tr, t, mS, _, desc = parallel_sample(g, src, edges)
        return {"value": tr / t / 1e9, "unit": UNIT, "cores": omp_baseline.threads(),
                "kind": "paper design: OpenMP, pull PageRank, push SSSP with CAS mailboxes, dynamic 256",
                "sample": f"PageRank (1 update) + SSSP to quiescence on {desc}; {tr} edges traversed in "
                          f"{t:.2f} s of supersteps"}
    except Exception as e:  # noqa: BLE001 - a baseline must not take the bench down
        return {"unavailable": f"{type(e).__name__}: {e}"[:300]}


def cpu_parallel_whole(g, pagerank: bool):
    """The OpenMP baseline on the whole graph: PageRank (10 updates) or Hashmin to quiescence."""
    try:
        import cpu_baseline as omp_baseline

        r = (omp_baseline.pagerank(g.n, g.offsets, g.cols, PR_UPDATES) if pagerank
             else omp_baseline.hashmin(g.n, g.offsets, g.cols))
        return {"value": round(r.messages / r.seconds / 1e9, 4), "unit": UNIT, "cores": omp_baseline.threads(),
                "kind": "paper design: OpenMP, pull " + ("PageRank" if pagerank else "Hashmin") + ", dynamic 256",
                "sample": f"the whole graph: {r.messages} messages in {r.seconds:.3f} s of supersteps, "
                          f"{r.supersteps} supersteps"}
    except Exception as e:  # noqa: BLE001 - a baseline must not take the bench down
        return {"unavailable": f"{type(e).__name__}: {e}"[:300]}


# ---------------------------------------------------------------------------------------
# roofline helpers


def kernel_hash(files):
    h = hashlib.sha256()
    for f in files:
        h.update(open(os.path.join(ROOT, f), "rb").read())
    return h.hexdigest()[:16]


_CSRC = "paper_2010_01542_gb300/csrc/"
KERNEL_FILES = {  # the files that define each kernel's code
    "pr_pull_kernel": [_CSRC + "ipg_pagerank.cu", _CSRC + "ipg_mergepath.cuh"],
    "pull_min_kernel": [_CSRC + "ipg_pull_min.cu", _CSRC + "ipg_mergepath.cuh"],
    "push_relax_kernel": [_CSRC + "ipg_push.cu"],
}


def measured_traffic(kernel, workload):
    """DRAM bytes per launch from the committed ncu record (profiles/traffic.json), if it
    was taken on this workload and on the current kernel source; else None."""
    try:
        d = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))[kernel]
    except Exception:
        return None
    if d.get("source_hash") != kernel_hash(KERNEL_FILES[kernel]) or d.get("workload") != workload:
        return None
    return d["dram_bytes_per_launch"]


NOMINAL_HBM_GBS = 7900.0  # GB300 HBM3e, nominal


def host_huge_fraction(arrays):
    """Fraction of the bytes of these host arrays that the kernel backs with transparent huge
    pages (AnonHugePages of the mappings holding them, from /proc/self/smaps); None if unknown."""
    try:
        spans = [(a.ctypes.data, a.ctypes.data + a.nbytes) for a in arrays if a is not None and a.nbytes]
        total = sum(e - b for b, e in spans)
        huge = 0
        cur = None
        for line in open("/proc/self/smaps"):
            head = line.split()
            if head and "-" in head[0] and len(head) >= 5 and all(c in "0123456789abcdef-" for c in head[0]):
                lo, hi = (int(x, 16) for x in head[0].split("-"))
                cur = (lo, hi) if any(b < hi and e > lo for b, e in spans) else None
            elif cur and line.startswith("AnonHugePages:"):
                kb = int(line.split()[1])
                lo, hi = cur
                inside = sum(max(0, min(e, hi) - max(b, lo)) for b, e in spans)
                huge += min(kb * 1024, inside)
        return round(huge / total, 4) if total else None
    except Exception:  # noqa: BLE001 - a diagnostic only
        return None


def peak_hbm():
    try:
        pk = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ---------------------------------------------------------------------------------------


def run_ours(a):
    import torch

    import gen
    import paper_2010_01542_gb300 as ipg

    world, rank, local = dist_init(a)
    ipg.load_library()
    if a.pull_divisor is not None:
        ipg.ipg_set_tuning("pull_divisor", a.pull_divisor)

    dg = gen.rmat_device(a.scale, a.edge_factor, seed=a.seed, weighted=True, device=local)
    n, m = dg.n, dg.m
    stream = torch.cuda.Stream()
    h = ipg.ipg_graph_create_dev(dg.offsets, dg.cols, dg.weights, n, m, True, stream=stream)
    host = dg.to_host(alloc=ipg.host_empty)  # page-locked, huge-page backed: the e2e leg uploads from it
    del dg
    torch.cuda.empty_cache()
    src = gen.max_out_degree_vertex(host)
    ranks = torch.empty(n, dtype=torch.float32, device="cuda")
    dist = torch.empty(n, dtype=torch.int32, device="cuda")
    flags = ipg.IPG_STAT_TIMING
    tune = None
    if not a.no_autotune and a.pull_divisor is None:  # untimed: picks this graph's launch shape
        t0 = time.perf_counter()
        tune = ipg.ipg_autotune(h, ipg.IPG_TUNE_PAGERANK | ipg.IPG_TUNE_SSSP, src, stream=stream)
        tune = {k: (round(v, 3) if isinstance(v, float) else v) for k, v in tune.items()}
        tune["seconds"] = round(time.perf_counter() - t0, 2)

    def step():
        c1, pst = ipg.ipg_pagerank_dev(h, PR_UPDATES, ranks, stats_flags=flags, stream=stream)
        c2, sst = ipg.ipg_sssp_dev(h, src, dist, stats_flags=flags, stream=stream)
        return pst, sst

    for _ in range(max(a.warmup, 0)):
        step()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    barrier(world)
    torch.cuda.synchronize()
    sampler.start()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    all_stats = [step() for _ in range(a.steps)]
    t_end.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clocks = sampler.stop()
    ms = t_start.elapsed_time(t_end)

    pr_edges = PR_UPDATES * m
    sssp_edges = [sum(s.messages_sent for s in sst) for _, sst in all_stats]
    edges_per_step = pr_edges + statistics.mean(sssp_edges)
    rate, ms_max = replica_throughput(edges_per_step * a.steps, ms, world)
    value = rate / 1e9
    pr_kernel_ms = [s.kernel_ms for pst, _ in all_stats for s in pst[:PR_UPDATES]]
    pr_step_ms = [s.superstep_ms for pst, _ in all_stats for s in pst[:PR_UPDATES]]
    sssp_kernel_ms = [sum(s.kernel_ms for s in sst) for _, sst in all_stats]
    sssp_ms = [sum(s.superstep_ms for s in sst) for _, sst in all_stats]
    sssp_supersteps = [len(sst) for _, sst in all_stats]
    # kernels of one step: PageRank init, (pull, fix-up) per superstep, unpermute; SSSP init,
    # per superstep 3 frontier passes + (partition, relax) in push form or (scatter, pull,
    # fix-up) in pull form, unpermute
    launches_per_step = (2 + 2 * PR_UPDATES) + statistics.mean(
        2 + sum(3 + (3 if s.flags & ipg.IPG_STAT_PULL else 2) for s in sst if s.senders > 0)
        for _, sst in all_stats)

    # roofline for the kernel that dominates the step (by CUDA-event time in the timed region)
    peak, peak_kind = peak_hbm()
    wl = f"rmat{a.scale}-ef{a.edge_factor}"
    pr_bytes = 8 * m + 24 * n  # per pull superstep
    pr_total_ms = sum(pr_kernel_ms)
    # SSSP supersteps ran either as push relax or as pull-min (IPG_STAT_PULL); both are
    # credited with the SSSP superstep's algorithmic bytes: 12 B per message + 16 B per sender
    sssp_recs = [s for _, sst in all_stats for s in sst if s.senders]
    kernels = {
        "pr_pull_kernel": {"launches": len(pr_kernel_ms), "total_ms": round(pr_total_ms, 3),
                           "algorithmic_bytes_per_launch": pr_bytes,
                           "achieved_gbs": round(pr_bytes * len(pr_kernel_ms) / (pr_total_ms / 1e3) / 1e9, 1),
                           "traffic_per_launch": measured_traffic("pr_pull_kernel", wl),
                           "bytes_rule": "8 m + 24 n per launch"},
    }
    for name, want_pull in (("push_relax_kernel", False), ("pull_min_kernel", True)):
        recs = [s for s in sssp_recs if bool(s.flags & ipg.IPG_STAT_PULL) == want_pull]
        if not recs:
            continue
        byts = [12 * s.messages_sent + 16 * s.senders for s in recs]
        ms = sum(s.kernel_ms for s in recs)
        kernels[name] = {"launches": len(recs), "total_ms": round(ms, 3),
                         "algorithmic_bytes_per_launch": int(statistics.mean(byts)),
                         "achieved_gbs": round(sum(byts) / (ms / 1e3) / 1e9, 1),
                         "traffic_per_launch": measured_traffic(name, wl) if name in KERNEL_FILES else None,
                         "bytes_rule": "12 B per message + 16 B per sender (the SSSP superstep's)"}
    dom = max(kernels, key=lambda k: kernels[k]["total_ms"])
    kd = kernels[dom]
    share = kd["total_ms"] / sum(k["total_ms"] for k in kernels.values())
    roofline = {"bound": "hbm", "kernel": dom, "achieved": kd["achieved_gbs"], "peak": peak,
                "peak_source": peak_kind, "unit": "GB/s", "frac": round(kd["achieved_gbs"] / peak, 4),
                "frac_of_nominal": round(kd["achieved_gbs"] / NOMINAL_HBM_GBS, 4),
                "traffic": None if kd["traffic_per_launch"] is None else int(kd["traffic_per_launch"]),
                "algorithmic_bytes_per_launch": kd["algorithmic_bytes_per_launch"],
                "share_of_kernel_time": round(share, 3)}
    if roofline["traffic"] is None:
        roofline["traffic_note"] = ("no ncu DRAM capture on this workload's size and the current kernel source; "
                                    "profiles/dram_rmat24_ef28_pull_kernels.md has the scale-24 figures")
    pr_mean = statistics.mean(pr_kernel_ms)

    # end to end through the host-buffer C ABI
    e2e = None
    if a.e2e_steps > 0:
        out_r = ipg.host_empty(n, np.float32)
        out_d = ipg.host_empty(n, np.uint32)
        times, e2e_edges = [], []
        phases = {"create": [], "pagerank": [], "sssp": [], "destroy": []}  # host calls return when done
        create_parts = []
        for i in range(a.e2e_steps + 1):  # the first round is a warm-up
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            g2 = ipg.ipg_graph_create(host.offsets, host.cols, host.weights, n, m, True)
            prof = ipg.ipg_graph_create_profile(g2)
            if tune:  # an identical graph: the tuning comes from the process-wide cache
                ipg.ipg_autotune(g2, ipg.IPG_TUNE_PAGERANK | ipg.IPG_TUNE_SSSP, src)
            t1 = time.perf_counter()
            _, c1, _ = ipg.ipg_pagerank(g2, PR_UPDATES, out_r)
            t2 = time.perf_counter()
            _, c2, sst = ipg.ipg_sssp(g2, src, out_d, stats_flags=0)
            t3 = time.perf_counter()
            ipg.ipg_graph_destroy(g2)
            t4 = time.perf_counter()
            dt = t4 - t0
            if i > 0:
                times.append(dt)
                e2e_edges.append(pr_edges + statistics.mean(sssp_edges))
                for k, v in zip(phases, (t1 - t0, t2 - t1, t3 - t2, t4 - t3)):
                    phases[k].append(v)
                create_parts.append(prof)
        t_e2e = all_max(statistics.mean(times), world)
        e2e = {"value": round(world * statistics.mean(e2e_edges) / t_e2e / 1e9, 3), "unit": UNIT,
               "h2d_bytes_per_step": int(host.offsets.nbytes + host.cols.nbytes + host.weights.nbytes),
               "d2h_bytes_per_step": int(out_r.nbytes + out_d.nbytes), "ms_per_step": round(t_e2e * 1e3, 2),
               "phases_ms": {k: round(statistics.mean(v) * 1e3, 1) for k, v in phases.items()},
               "create_ms": {k: round(statistics.mean(p[k] for p in create_parts), 1) for k in create_parts[0]},
               "host_huge_page_fraction": host_huge_fraction([host.offsets, host.cols, host.weights]),
               "api": "ipg_graph_create + ipg_autotune (cached) + ipg_pagerank + ipg_sssp + ipg_graph_destroy, "
                      "host buffers"}

    cpu = cpu_par = None
    if rank == 0 and not a.no_cpu_baseline:
        cpu = cpu_baseline(host, src, a.cpu_seconds)
        cpu_par = cpu_parallel_baseline(host, src, 10.0)

    l2_note = "inputs larger than L2 (graph %.1f GB resident)" % ((host.offsets.nbytes + 2 * host.cols.nbytes) / 1e9)
    h.destroy()
    del host
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": round(ms_max / a.steps, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+u32", "data": "synthetic",
            "config": {"workload": workload_name(a), "scale": a.scale, "edge_factor": a.edge_factor, "n": n, "m": m,
                       "sssp_source": src, "l2": l2_note,
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "roofline": roofline, "kernels": kernels, "cpu_baseline": cpu, "cpu_parallel": cpu_par, "e2e": e2e,
            "gpu_launches": int(round(launches_per_step * a.steps)), "clocks": clocks,
            "pagerank": {"edges_per_step": pr_edges, "ms_per_superstep": round(statistics.mean(pr_step_ms), 4),
                         "kernel_ms": round(pr_mean, 4),
                         "gteps": round(m / (statistics.mean(pr_step_ms) / 1e3) / 1e9, 2)},
            "autotune": tune,
            "sssp": {"edges_per_step": int(statistics.mean(sssp_edges)), "supersteps": sssp_supersteps[0],
                     "pull_divisor": tune["sssp_pull_divisor"] if tune else ipg.ipg_get_tuning("pull_divisor"),
                     "kernel_ms_per_superstep": [round(s.kernel_ms, 3) for s in all_stats[-1][1]],
                     "messages_per_superstep": [s.messages_sent for s in all_stats[-1][1]],
                     "ms": round(statistics.mean(sssp_ms), 3), "kernel_ms": round(statistics.mean(sssp_kernel_ms), 3),
                     "gteps": round(statistics.mean(sssp_edges) / (statistics.mean(sssp_ms) / 1e3) / 1e9, 2),
                     "graph500_gteps": round(m / (statistics.mean(sssp_ms) / 1e3) / 1e9, 2)},  # m / run time
        }
        if world == 1 and not a.no_other_configs:
            line["other_configs"] = run_other_configs(a)
        emit(line)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


def _compact(name, line):
    if name in ("pagerank16", "hashmin20"):
        r = line["roofline"]
        return {"workload": line["config"]["workload"], "gteps": line["value"], "ms_per_step": line["ms_per_step"],
                "roofline": {"kernel": r["kernel"], "achieved_gbs": r["achieved"], "frac": r["frac"]}}
    if name in ("batch", "cc_batch"):
        return {"workload": line["config"]["workload"], "unit": line["unit"], "value": line["value"],
                "one_at_a_time": line["one_at_a_time"]["value"], "speedup": line["speedup"],
                "results_equal": line["results_equal"]}
    if name == "serve":
        cb = line["continuous_batching"]
        return {"workload": line["config"]["workload"], "offered_per_s": cb["offered_per_s"],
                "queries_per_s": cb["queries_per_s"], "p50_ms": cb["p50_ms"], "p99_ms": cb["p99_ms"],
                "joined_running_batch": cb.get("joined_running_batch"),
                "one_at_a_time_queries_per_s": line["one_at_a_time"]["queries_per_s"],
                "at_75pct_rate": {k: line["continuous_batching_at_75pct_rate"][k]
                                  for k in ("queries_per_s", "p50_ms", "p99_ms")}}
    c = line["combine"]
    return {"workload": line["config"]["workload"],
            "sssp_tree_u64_gteps": line["programs"]["sssp_tree_u64"]["gteps"],
            "bfs_paths_u128_gteps": line["programs"]["bfs_paths_u128"]["gteps"],
            "sssp_min_u32_gteps": line["programs"]["sssp_min_u32"]["gteps"],
            "combine_g_messages_per_s": {k: v["g_messages_per_s"] for k, v in c.items() if isinstance(v, dict)},
            "combine_call_overhead_ms": {k: v["call_overhead_ms"] for k, v in c.items() if isinstance(v, dict)}}


def run_other_configs(a):
    """The other workloads, each run once after the default run's timed region (never inside
    it) with a few steps, reported as compact summaries; `bench.py --workload X` prints each
    one's full line."""
    global _CAPTURE
    out = {}
    jobs = (("pagerank16", lambda b: run_small_config(b, "pagerank16"), dict(steps=20, warmup=3)),
            ("hashmin20", lambda b: run_small_config(b, "hashmin20"), dict(steps=20, warmup=3)),
            ("batch", run_batch, dict(steps=5, warmup=2)),
            ("cc_batch", run_cc_batch, dict(steps=5, warmup=2)),
            ("serve", run_serve, dict(requests=6000)),
            ("combiner", run_combiner, dict(steps=5, warmup=2)))
    for name, fn, over in jobs:
        b = argparse.Namespace(**vars(a))
        b.no_cpu_baseline = True
        for k, v in over.items():
            setattr(b, k, v)
        _CAPTURE = []
        t0 = time.perf_counter()
        try:
            fn(b)
            out[name] = _compact(name, _CAPTURE[-1]) if _CAPTURE else {"unavailable": "no line"}
        except Exception as e:  # noqa: BLE001 - one workload must not take the headline line down
            out[name] = {"unavailable": f"{type(e).__name__}: {e}"[:300]}
        finally:
            _CAPTURE = None
        out[name]["seconds"] = round(time.perf_counter() - t0, 1)
        import torch

        torch.cuda.synchronize()
        torch.cuda.empty_cache()
    return out


def run_reference(a):
    """The oracle, as it stands, on the host cores: each step is a bounded sample of the
    same workload (strided row sample, PageRank one update + SSSP)."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import gen

    import torch

    if torch.cuda.is_available():
        g = gen.rmat_device(a.scale, a.edge_factor, seed=a.seed, weighted=True).to_host()
    else:
        g = gen.rmat(a.scale, a.edge_factor, seed=a.seed, weighted=True)
    src = gen.max_out_degree_vertex(g)
    budget = 150.0 / max(1, a.steps + a.warmup)
    edges = calibrate_sample(g, src, budget)
    for _ in range(a.warmup):
        oracle_sample(g, src, edges)
    trav, secs = 0, 0.0
    desc = None
    for _ in range(a.steps):
        tr, t, d = oracle_sample(g, src, edges)
        trav += tr
        secs += t
        desc = f"oracle PageRank (1 update) + SSSP to quiescence on {d}, 1 thread"
    value = trav / secs / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": world,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": round(secs / a.steps * 1e3, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64+u32",
            "data": "synthetic", "config": {"workload": workload_name(a), "scale": a.scale,
                                            "edge_factor": a.edge_factor, "n": g.n, "m": g.m},
            "cpu_baseline": {"value": round(value, 4), "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc},
            "e2e": {"value": round(value, 4), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    emit(line)


def run_batch(a):
    """Batched SSSP: k seeded uniform-random sources on a directed weighted R-MAT graph
    (default scale 22, EF 16), one ipg_sssp_batch_dev call per step, against the same k
    sources run one at a time with ipg_sssp_dev; results compared on the device."""
    import torch

    import gen
    import paper_2010_01542_gb300 as ipg

    world, rank, local = dist_init(a)
    ipg.load_library()
    scale = a.scale if a.scale != 26 else 22
    ef = a.edge_factor if a.edge_factor != 28 else 16
    dg = gen.rmat_device(scale, ef, seed=a.seed, weighted=True, device=local)
    n, m = dg.n, dg.m
    stream = torch.cuda.Stream()
    h = ipg.ipg_graph_create_dev(dg.offsets, dg.cols, dg.weights, n, m, True, stream=stream)
    del dg
    k = a.batch_sources
    sources = gen.batch_sources(n, k, a.seed)
    out = torch.empty(k * n, dtype=torch.int32, device="cuda")
    single = torch.empty(n, dtype=torch.int32, device="cuda")
    for _ in range(max(a.warmup, 1)):
        ipg.ipg_sssp_batch_dev(h, sources, out, stream=stream)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier(world)
    e0.record(stream)
    for _ in range(a.steps):
        steps_b = ipg.ipg_sssp_batch_dev(h, sources, out, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    t_batch = all_max(e0.elapsed_time(e1) / a.steps, world)
    binfo = ipg.ipg_sssp_batch_info(h)
    # one at a time, same sources, checked against the batch rows
    ipg.ipg_sssp_dev(h, int(sources[0]), single, stream=stream)
    torch.cuda.synchronize()
    e0.record(stream)
    counts = []
    for i, s in enumerate(sources):
        c, _ = ipg.ipg_sssp_dev(h, int(s), single, stream=stream)
        counts.append(c)
    e1.record(stream)
    torch.cuda.synchronize()
    t_single = all_max(e0.elapsed_time(e1), world)
    equal = True
    for i, s in enumerate(sources):
        ipg.ipg_sssp_dev(h, int(s), single, stream=stream)
        torch.cuda.synchronize()
        equal &= bool(torch.equal(out[i * n:(i + 1) * n], single)) and counts[i] == int(steps_b[i])
    if rank == 0:
        line = {"metric": "SSSP queries/s, batched (k sources per call) vs one at a time", "unit": "queries/s",
                "value": round(world * k / (t_batch / 1e3), 1), "n_gpus": world, "steps": a.steps,
                "warmup": a.warmup, "ms_per_step": round(t_batch, 3), "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "u32", "data": "synthetic",
                "config": {"workload": f"rmat{scale}-ef{ef} directed weighted[1,255] seed {a.seed}, "
                                       f"{k} uniform random sources (seed {a.seed})", "n": n, "m": m, "k": k},
                "one_at_a_time": {"value": round(world * k / (t_single / 1e3), 1), "unit": "queries/s",
                                  "ms_total": round(t_single, 2)},
                "speedup": round(t_single / t_batch, 2), "results_equal": equal,
                "supersteps": {"min": int(steps_b.min()), "max": int(steps_b.max()),
                               "sum_over_queries": int(steps_b.sum())},
                "lane_loop": binfo,
                "ms_per_lane_superstep": round(t_batch / max(binfo["supersteps"], 1), 3)}
        emit(line)
    h.destroy()


def run_combiner(a):
    """The general (hybrid) combiner on one GPU, graph resident.
    Programs with wide messages on a directed weighted R-MAT graph (default scale 22, EF 16),
    from the max-out-degree vertex: the shortest-path tree ((distance, parent) messages) and
    shortest-path counting ((level, count) messages), beside plain SSSP (32-bit min) on the
    same graph; messages/s each, distances checked equal on the device.
    The combination step alone (ipg_combine_dev): 2^26 messages to uniform random vertices
    among 2^22 mailboxes, for every message kind; messages/s and streamed GB/s."""
    import torch

    import gen
    import paper_2010_01542_gb300 as ipg

    world, rank, local = dist_init(a)
    ipg.load_library()
    scale = a.scale if a.scale != 26 else 22
    ef = a.edge_factor if a.edge_factor != 28 else 16
    dg = gen.rmat_device(scale, ef, seed=a.seed, weighted=True, device=local)
    n, m = dg.n, dg.m
    stream = torch.cuda.Stream()
    h = ipg.ipg_graph_create_dev(dg.offsets, dg.cols, dg.weights, n, m, True, stream=stream)
    src = gen.max_out_degree_vertex(dg.to_host())
    del dg
    d0 = torch.empty(n, dtype=torch.int32, device="cuda")
    d1 = torch.empty(n, dtype=torch.int32, device="cuda")
    par = torch.empty(n, dtype=torch.int32, device="cuda")
    lvl = torch.empty(n, dtype=torch.int32, device="cuda")
    cnt = torch.empty(n, dtype=torch.int64, device="cuda")
    progs = {
        "sssp_min_u32": lambda: ipg.ipg_sssp_dev(h, src, d0, stream=stream),
        "sssp_tree_u64": lambda: ipg.ipg_sssp_tree_dev(h, src, d1, par, stream=stream),
        "bfs_paths_u128": lambda: ipg.ipg_bfs_paths_dev(h, src, lvl, cnt, stream=stream),
    }
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    results = {}
    for name, run in progs.items():
        for _ in range(max(a.warmup, 1)):
            count, st = run()
        msgs = sum(s.messages_sent for s in st)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(a.steps):
            run()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = all_max(e0.elapsed_time(e1) / a.steps, world)
        results[name] = {"ms": round(ms, 3), "supersteps": count, "messages": msgs,
                         "gteps": round(msgs / (ms / 1e3) / 1e9, 2)}
    same_dist = bool(torch.equal(d0, d1))
    # the combination step alone
    k, nm = 1 << 26, 1 << 22
    rng = np.random.default_rng(a.seed)
    dst = torch.from_numpy(rng.integers(0, nm, size=k).astype(np.uint32).view(np.int32)).cuda()
    kinds = {"xor_u32": (ipg.IPG_COMBINE_XOR_U32, 4, 0), "min_u64": (ipg.IPG_COMBINE_MIN_U64, 8, 0),
             "min_u64_native_atomic": (ipg.IPG_COMBINE_MIN_U64, 8, ipg.IPG_COMBINE_NATIVE),
             "sum_u64": (ipg.IPG_COMBINE_SUM_U64, 8, 0), "mincount_u128": (ipg.IPG_COMBINE_MINCOUNT_U128, 16, 0)}
    combine = {}
    for name, (kind, size, opt) in kinds.items():
        if size == 4:
            msgs_t = torch.from_numpy(rng.integers(0, 1 << 32, size=k, dtype=np.uint64).astype(np.uint32)
                                      .view(np.int32)).cuda()
            mail = torch.zeros(nm, dtype=torch.int32, device="cuda")
        elif size == 8:
            msgs_t = torch.from_numpy(rng.integers(0, 1 << 62, size=k, dtype=np.int64)).cuda()
            mail = torch.zeros(nm, dtype=torch.int64, device="cuda")
        else:
            keys = rng.integers(0, 3, size=k, dtype=np.int64)
            msgs_t = torch.from_numpy(np.stack([keys, np.ones(k, dtype=np.int64)], axis=1)).cuda()
            mail = torch.zeros((nm, 2), dtype=torch.int64, device="cuda")
        flags = torch.zeros(nm, dtype=torch.int32, device="cuda")
        for _ in range(max(a.warmup, 1)):
            recv = ipg.ipg_combine_dev(kind, nm, dst, msgs_t, flags, mail, opt, stream=stream)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(a.steps):
            ipg.ipg_combine_dev(kind, nm, dst, msgs_t, flags, mail, opt, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = all_max(e0.elapsed_time(e1) / a.steps, world)
        # the call's fixed cost (counter allocation, the flag clear, the copy back and the
        # host synchronisation), timed as a call with no messages and the same options
        e0.record(stream)
        for _ in range(a.steps):
            ipg.ipg_combine_dev(kind, nm, dst[:0], msgs_t[:0], flags, mail, opt, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        fixed = all_max(e0.elapsed_time(e1) / a.steps, world)
        net = max(ms - fixed, 1e-6)
        combine[name] = {"ms": round(ms, 3), "call_overhead_ms": round(fixed, 3),
                         "g_messages_per_s": round(k / (net / 1e3) / 1e9, 2),
                         "g_messages_per_s_whole_call": round(k / (ms / 1e3) / 1e9, 2),
                         "streamed_gbs": round(k * (4 + size) / (net / 1e3) / 1e9, 1), "receivers": recv}
        del msgs_t, mail, flags
    if rank == 0:
        tree = results["sssp_tree_u64"]
        line = {"metric": "GTEPS, shortest-path tree (hybrid combiner, 64-bit messages)", "unit": UNIT,
                "value": round(world * tree["messages"] / (tree["ms"] / 1e3) / 1e9, 3), "n_gpus": world,
                "steps": a.steps, "warmup": a.warmup, "ms_per_step": tree["ms"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "u64/u128", "data": "synthetic",
                "config": {"workload": f"rmat{scale}-ef{ef} directed weighted[1,255] seed {a.seed}, source = "
                                       f"max-out-degree vertex; combine step: 2^26 messages into 2^22 mailboxes",
                           "n": n, "m": m, "source": int(src)},
                "programs": results, "tree_distances_equal_sssp": same_dist, "combine": combine}
        emit(line)
    h.destroy()


def run_small_config(a, kind):
    """One small configuration on one GPU, graph resident:
    pagerank16  PageRank, 10 supersteps, directed R-MAT scale 16 EF 16 (value: GTEPS = 10 m / t);
    hashmin20   Hashmin components to quiescence, undirected R-MAT scale 20 EF 16
                (value: GTEPS = messages sent / t).
    Per-superstep CUDA events give the dominant kernel's roofline; the oracle runs on the
    whole graph on one host core for the CPU baseline.  With several ranks every rank runs
    a replica."""
    import torch

    import gen
    import oracle
    import paper_2010_01542_gb300 as ipg

    world, rank, local = dist_init(a)
    ipg.load_library()
    pr = kind == "pagerank16"
    scale, ef = (16, 16) if pr else (20, 16)
    g = gen.rmat(scale, ef, seed=a.seed, undirected=not pr)
    h = ipg.ipg_graph_create(g.offsets, g.cols, None, g.n, g.m, pr)
    stream = torch.cuda.Stream()
    out = torch.empty(g.n, dtype=torch.float32 if pr else torch.int32, device="cuda")
    tune = None
    if not a.no_autotune:
        tune = ipg.ipg_autotune(h, ipg.IPG_TUNE_PAGERANK if pr else ipg.IPG_TUNE_HASHMIN, stream=stream)
        tune = {k: (round(v, 3) if isinstance(v, float) else v) for k, v in tune.items()}

    # the timed steps run without per-superstep events, so that the superstep loop runs
    # as a captured CUDA graph; separate runs with events give the kernels' times for
    # the roofline
    def step(timing=False):
        flags = ipg.IPG_STAT_TIMING if timing else 0
        if pr:
            return ipg.ipg_pagerank_dev(h, PR_UPDATES, out, stats_flags=flags, stream=stream)
        return ipg.ipg_hashmin_cc_dev(h, out, stats_flags=flags, stream=stream)

    for _ in range(max(a.warmup, 3)):
        step()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    barrier(world)
    sampler.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    runs = [step() for _ in range(a.steps)]
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1)
    count, st = runs[-1]
    edges = PR_UPDATES * g.m if pr else sum(s.messages_sent for s in st)
    assert all(c == count for c, _ in runs)
    rate, ms_max = replica_throughput(edges * a.steps, ms, world)
    # roofline of the step's dominant kernel (PageRank pull / pull-min or push relax)
    peak, peak_kind = peak_hbm()
    timed_runs = [step(timing=True) for _ in range(3)]
    recs = [s for _, sts in timed_runs for s in sts if s.flags & ipg.IPG_STAT_TIMING]
    if pr:
        byts = 8 * g.m + 24 * g.n
        kern = {"pr_pull_kernel": (len(recs), sum(s.kernel_ms for s in recs), byts)}
        rule = "8 m + 24 n per launch"
    else:
        kern = {}
        for name, want in (("push_relax_kernel", False), ("pull_min_kernel", True)):
            rr = [s for s in recs if s.senders and bool(s.flags & ipg.IPG_STAT_PULL) == want]
            if rr:
                kern[name] = (len(rr), sum(s.kernel_ms for s in rr),
                              statistics.mean(8 * s.messages_sent + 16 * s.senders for s in rr))
        rule = "8 B per message (4 B column + 4 B value RMW) + 16 B per sender"
    dom = max(kern, key=lambda k: kern[k][1])
    nl, kms, bpl = kern[dom]
    achieved = bpl * nl / (kms / 1e3) / 1e9
    cpu = cpu_par = None
    if rank == 0 and not a.no_cpu_baseline:
        cpu_par = cpu_parallel_whole(g, pr)
        t0 = time.perf_counter()
        ref = oracle.pagerank(g.n, g.offsets, g.cols, PR_UPDATES) if pr else oracle.hashmin(g.n, g.offsets, g.cols)
        t = time.perf_counter() - t0
        host = out.cpu().numpy()
        if pr:
            ok = float(np.max(np.abs(host.astype(np.float64) - ref.values)) / ref.values.max()) <= 1e-5
        else:
            ok = bool(np.array_equal(host.view(np.uint32), ref.values))
        ok = ok and ref.supersteps == count
        cpu_edges = sum(s.messages_sent for s in ref.stats)
        cpu = {"value": round(cpu_edges / t / 1e9, 5), "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"the whole graph: oracle {'PageRank 10 updates' if pr else 'Hashmin to quiescence'}, "
                         f"{cpu_edges} messages in {t:.2f} s; GPU result matches the oracle: {ok}"}
    if rank == 0:
        line = {"metric": ("GTEPS, PageRank 10 supersteps" if pr else "GTEPS, Hashmin components to quiescence"),
                "value": round(rate / 1e9, 3), "unit": UNIT, "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
                "ms_per_step": round(ms_max / a.steps, 4), "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32+u32" if pr else "u32", "data": "synthetic",
                "config": {"workload": (f"rmat{scale}-ef{ef} {'directed' if pr else 'undirected'} seed {a.seed}: "
                                        + ("PageRank 10 supersteps" if pr else "Hashmin components")),
                           "n": g.n, "m": g.m, "supersteps": count,
                           "l2": "graph L2-resident: latency- and launch-bound at this size"},
                "roofline": {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1), "peak": peak,
                             "peak_source": peak_kind, "unit": "GB/s", "frac": round(achieved / peak, 4),
                             "frac_of_nominal": round(achieved / NOMINAL_HBM_GBS, 4),
                             "traffic": None, "algorithmic_bytes_per_launch": int(bpl), "bytes_rule": rule},
                "cpu_baseline": cpu, "cpu_parallel": cpu_par, "autotune": tune, "clocks": clocks,
                "gpu_launches": ((1 + 2 * PR_UPDATES + 1) if pr else
                                 (1 + 5 * sum(1 for s in st if s.senders) + 1)) * a.steps,
                "messages_per_superstep": [s.messages_sent for s in st]}
        emit(line)
    h.destroy()


def run_cc_batch(a, count=64):
    """Hashmin on 64 undirected R-MAT graphs (EF 16, uneven scales 10..20, seeds 1..64) held in
    one batch graph, one ipg_hashmin_cc_batch_dev call per step, against 64 separate graphs run
    one at a time with ipg_hashmin_cc_dev; labels and superstep counts compared."""
    import torch

    import gen
    import paper_2010_01542_gb300 as ipg

    world, rank, local = dist_init(a)
    ipg.load_library()
    scales = gen.cc_batch_scales(count, a.seed)
    graphs = [gen.rmat_device(sc, 16, seed=i + 1, undirected=True, device=local).to_host()
              for i, sc in enumerate(scales)]
    hb = ipg.ipg_graph_create_batch(graphs, directed=False)
    _, bases = ipg.ipg_graph_instances(hb)
    total_n = int(bases[-1])
    total_m = sum(g.m for g in graphs)
    stream = torch.cuda.Stream()
    labels = torch.empty(total_n, dtype=torch.int32, device="cuda")
    for _ in range(max(a.warmup, 1)):
        steps_b = ipg.ipg_hashmin_cc_batch_dev(hb, labels, stream=stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(a.steps):
        steps_b = ipg.ipg_hashmin_cc_batch_dev(hb, labels, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    t_batch = all_max(e0.elapsed_time(e1) / a.steps, world)
    singles = [ipg.ipg_graph_create(g.offsets, g.cols, None, g.n, g.m, False) for g in graphs]
    outs = [torch.empty(g.n, dtype=torch.int32, device="cuda") for g in graphs]
    for h, o in zip(singles, outs):
        ipg.ipg_hashmin_cc_dev(h, o, stream=stream)
    torch.cuda.synchronize()
    e0.record(stream)
    counts = [ipg.ipg_hashmin_cc_dev(h, o, stream=stream)[0] for h, o in zip(singles, outs)]
    e1.record(stream)
    torch.cuda.synchronize()
    t_single = all_max(e0.elapsed_time(e1), world)
    equal = all(bool(torch.equal(labels[int(bases[i]):int(bases[i + 1])], outs[i])) and counts[i] == int(steps_b[i])
                for i in range(count))
    if rank == 0:
        line = {"metric": "Hashmin CC graphs/s, many graphs in one batch vs one at a time", "unit": "graphs/s",
                "value": round(world * count / (t_batch / 1e3), 1), "n_gpus": world, "steps": a.steps,
                "warmup": a.warmup, "ms_per_step": round(t_batch, 3), "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "u32", "data": "synthetic",
                "config": {"workload": f"{count} undirected R-MAT graphs, EF 16, scales 10..20 "
                                       f"(scale_i from splitmix64, seed {a.seed}), graph seeds 1..{count}",
                           "scales": scales, "total_n": total_n, "total_m": total_m},
                "one_at_a_time": {"value": round(world * count / (t_single / 1e3), 1), "unit": "graphs/s",
                                  "ms_total": round(t_single, 2)},
                "speedup": round(t_single / t_batch, 2), "results_equal": equal,
                "gteps": round(sum(int(x) for x in [total_m]) / (t_batch / 1e3) / 1e9, 2)}
        emit(line)


def serve_stream(srv, graphs, requests, rate, seed, warm):
    """Drive one server with a seeded Poisson stream; returns per-request records of the
    measured part (latency from the scheduled arrival)."""
    import paper_2010_01542_gb300 as ipg

    rng = np.random.default_rng(seed)
    total = requests + warm
    gaps = rng.exponential(1.0 / rate, size=total)
    arrivals = np.cumsum(gaps)
    gsel = rng.integers(0, len(graphs), size=total)
    kinds = rng.random(size=total)
    srcs = rng.random(size=total)
    pools = [[np.empty(g.n, dtype=np.uint32) for _ in range(24)] for g in graphs]
    free = {i: list(range(24)) for i in range(len(graphs))}
    owner = {}
    recs = {}

    def collect(wait_ms):
        for c in srv.poll(wait_ms):
            gi, slot, t_arr, kind, batch = owner.pop(c.user)
            free[gi].append(slot)
            if c.status != 0:
                raise RuntimeError(f"query {c.user} failed with status {c.status}")
            recs[c.user] = (t_arr, c.t_done, kind, c.batch, c.joined)

    t0 = srv.now() + 0.05
    for i in range(total):
        gi = int(gsel[i])
        kind = ipg.IPG_Q_SSSP if kinds[i] < 0.6 else (ipg.IPG_Q_HASHMIN if kinds[i] < 0.9 else ipg.IPG_Q_PAGERANK)
        while not free[gi]:
            collect(1)
        t_arr = t0 + arrivals[i]
        while srv.now() < t_arr:
            collect(0)
        slot = free[gi].pop()
        out = pools[gi][slot]
        if kind == ipg.IPG_Q_PAGERANK:
            out = out.view(np.float32)
        owner[i] = (gi, slot, t_arr, kind, 0)
        srv.submit(gi, kind, out, source=int(srcs[i] * graphs[gi].n), updates=10, user=i)
        collect(0)
    srv.drain()
    collect(0)
    return {u: r for u, r in recs.items() if u >= warm}


def serve_summary(recs):
    lat = np.array([(r[1] - r[0]) * 1e3 for r in recs.values()])
    t_first = min(r[0] for r in recs.values())
    t_last = max(r[1] for r in recs.values())
    sssp = [r for r in recs.values() if r[2] == 0]
    batches = np.array([r[3] for r in sssp])
    shared = np.array([r[3] for r in recs.values() if r[2] != 0])
    return {"queries_per_s": round(len(recs) / (t_last - t_first), 1), "p50_ms": round(float(np.percentile(lat, 50)), 3),
            "p99_ms": round(float(np.percentile(lat, 99)), 3), "mean_ms": round(float(lat.mean()), 3),
            "sssp_batch_mean": round(float(batches.mean()), 2) if batches.size else None,
            "joined_running_batch": int(sum(r[4] for r in sssp)), "sssp_queries": len(sssp),
            "cc_pr_shared_run_mean": round(float(shared.mean()), 2) if shared.size else None}


def run_serve(a, count=32):
    """Config: 32 undirected weighted R-MAT graphs (EF 16, scale_i = 12 + splitmix64(splitmix64(seed)
    + i) % 11, graph seeds 101..132) resident on the GPU; a seeded Poisson stream of --rate requests/s:
    60% SSSP from a uniform random source, 30% Hashmin, 10% PageRank (10 supersteps).  The
    continuous-batching server (8 workers, SSSP batches up to 256) against one worker without
    batching, on the same stream.  Each server runs every program once per graph at
    creation (IPG_SERVER_PREPARE), so no workspace is allocated while queries wait."""
    import gen
    import paper_2010_01542_gb300 as ipg

    world, rank, local = dist_init(a)
    ipg.load_library()
    scales = gen.serve_scales(count, a.seed)
    graphs = [gen.rmat_device(sc, 16, seed=101 + i, undirected=True, weighted=True, device=local).to_host()
              for i, sc in enumerate(scales)]
    handles = [ipg.ipg_graph_create(g.offsets, g.cols, g.weights, g.n, g.m, False) for g in graphs]
    warm = max(a.requests // 10, 100)
    res = {}
    # every server prepares the graphs' workspaces before the stream starts
    msb = a.min_sssp_batch
    for name, kw, rate in (("continuous_batching", dict(workers=8, max_batch=256, prepare=True, min_sssp_batch=msb),
                            a.rate),
                           ("one_at_a_time", dict(workers=1, max_batch=1, prepare=True), a.rate),
                           ("continuous_batching_at_75pct_rate",
                            dict(workers=8, max_batch=256, prepare=True, min_sssp_batch=msb),
                            0.75 * a.rate)):
        srv = ipg.Server(handles, **kw)
        recs = serve_stream(srv, graphs, a.requests, rate, a.seed, warm)
        srv.close()
        res[name] = serve_summary(recs)
        res[name]["offered_per_s"] = rate
    if rank == 0:
        cb = res["continuous_batching"]
        line = {"metric": "served queries/s with p50/p99 latency (Poisson arrivals, mixed SSSP/CC/PageRank)",
                "unit": "queries/s", "value": cb["queries_per_s"], "n_gpus": world, "steps": a.requests,
                "warmup": warm, "ms_per_step": cb["mean_ms"], "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "u32+f32", "data": "synthetic",
                "config": {"workload": f"{count} undirected weighted R-MAT graphs, EF 16, scales 12..22, "
                                       f"Poisson {a.rate:g} req/s, 60% SSSP / 30% Hashmin / 10% PageRank, "
                                       f"seed {a.seed}", "scales": scales,
                           "total_m": int(sum(g.m for g in graphs))},
                "p50_ms": cb["p50_ms"], "p99_ms": cb["p99_ms"], "continuous_batching": cb,
                "one_at_a_time": res["one_at_a_time"],
                "continuous_batching_at_75pct_rate": res["continuous_batching_at_75pct_rate"]}
        emit(line)


def main():
    a = parse()
    if a.impl == "reference":
        run_reference(a)
        return
    apply_tuning(a)
    if a.workload in ("pagerank16", "hashmin20"):
        run_small_config(a, a.workload)
    elif a.workload == "batch":
        run_batch(a)
    elif a.workload == "cc-batch":
        run_cc_batch(a)
    elif a.workload == "serve":
        run_serve(a)
    elif a.workload == "combiner":
        run_combiner(a)
    else:
        run_ours(a)


if __name__ == "__main__":
    main()
