#!/usr/bin/env python
"""Benchmark of the extremum-graph path on GB300.

One step = one full extremum graph of one field (classification, path
resolution, arcs and CSR assembly: every step of the hot path), computed by
libeg.so through its C ABI.  Default workload: the 3D 512^3 float32 Gaussian
random field with P(k) ~ k^-11/3 (seed 2), the single-field roofline
configuration.  The field (537 MB) is larger than L2 (129 MB), so no flush is
needed between timed steps.

Output: ONE JSON line on rank 0 (see the keys below).  Multi-GPU runs (torchrun)
are replicas: each rank computes its own copy of the workload, no collective
touches the data path ("scaling": "weak").

--impl reference times the CPU oracle (test infrastructure, sequential C) on
a bounded slab of the same workload.
"""
from __future__ import annotations

import argparse
import contextlib
import gc
import json
import os
import platform
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    "grf512": ("3D 512^3 float32 Gaussian random field, P(k)~k^-11/3, zero mean, unit variance, seed 2; "
               "Freudenthal 14-neighbour; plain single-field path"),
    "gauss3d256": ("3D 256^3 float32, 64 anisotropic Gaussians (sigma U[6,30], amplitude U[0.3,1]) + "
                   "U(-1e-3,1e-3) noise, seed 1; plain single-field path"),
    "gauss2d256": ("2D 256x256 float32, 16 isotropic Gaussians (sigma U[4,16], amplitude U[0.5,1]) + "
                   "N(0,0.01) noise, seed 0"),
    "grf384": ("3D 384^3 float32 Gaussian random field, P(k)~k^-11/3, seed 2 (profiling case: larger than "
               "L2, a few GB on the device)"),
    "schwefel4d128": ("4D 128^4 float32 Schwefel function sum_i -x_i sin(sqrt|x_i|) sampled on [-500,500]^4 "
                      "(window shifted by seed 5); Freudenthal 30-neighbour; plain single-field path "
                      "(the shape of Table 3's largest 4D row)"),
    "schwefel4d96": ("4D 96^4 float32 Schwefel function on [-500,500]^4 (seed 5) (profiling case: larger than "
                     "L2, a few GB on the device)"),
    "schwefel4d64": ("4D 64^4 float32 Schwefel function on [-500,500]^4 (seed 5); Freudenthal 30-neighbour; "
                     "plain single-field path (the shape of a Table 3 row)"),
    "schwefel5d32": ("5D 32^5 float32 Schwefel function on [-500,500]^5 (seed 5); Freudenthal 62-neighbour; "
                     "plain single-field path (the shape of a Table 3 row)"),
    "schwefel5d64": ("5D 64^5 float32 Schwefel function on [-500,500]^5 (seed 5); Freudenthal 62-neighbour; "
                     "plain single-field path (1.07 G vertices: the shape of Table 3's largest 5D row)"),
    "serve": ("Served stream: requests with Poisson arrivals, each a float32 2D/3D/4D field (vertex count "
              "log-uniform 1e4..1e7, sums of U{4..64} Gaussians + 1e-3 uniform noise), seed 4; admission by "
              "free HBM, continuous batching on three engines, results kept in device memory"),
    "batch": ("Batched: 256 float32 fields, 2D (side log-uniform 64..2048) or 3D (side log-uniform 32..256) "
              "50/50, sums of U{4..64} Gaussians + 1e-3 uniform noise, seed 3; one submission (persistent "
              "work-queue classifier, captured CUDA graphs, knobs autotuned on the batch) vs per-field plain "
              "launches"),
}


def make_field(name):
    from paper_2303_02724_gb300 import fields as F
    if name == "grf512":
        return F.config_3d_512()
    if name == "gauss3d256":
        return F.config_3d_256()
    if name == "gauss2d256":
        return F.config_2d_256()
    if name == "grf384":
        return F.config_3d_512(side=384)
    if name == "schwefel4d128":
        return F.schwefel((128, 128, 128, 128))
    if name == "schwefel4d96":
        return F.schwefel((96, 96, 96, 96))
    if name == "schwefel5d32":
        return F.schwefel((32,) * 5)
    if name == "schwefel5d64":
        return F.schwefel((64,) * 5)
    if name == "schwefel4d64":
        return F.schwefel((64, 64, 64, 64))
    raise ValueError(name)


def oracle_slab(field, max_vertices):
    """Bounded sample of a field for the CPU oracle: its first slabs along the
    slowest axis (whole rows/planes), about max_vertices vertices."""
    v = field.values
    per = int(v[0].size)
    k = max(1, min(v.shape[0], max_vertices // per))
    return v[:k], f"first {k} of {v.shape[0]} slabs along the slowest axis ({k * per} vertices)"


def host_cpu():
    """Model and core count of the host CPU (for the CPU baseline)."""
    model = platform.processor() or platform.machine()
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.lower().startswith(("model name", "cpu part")):
                    model = ln.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    return {"model": model, "machine": platform.machine(), "cores": os.cpu_count()}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples during the timed region (SM clock, throttle reasons)."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.p = None
        # raw samples go to $EG_CLOCKS_DIR when set (kept for inspection), else a temporary file
        out = os.environ.get("EG_CLOCKS_DIR")
        self.path = os.path.join(out, f"clocks_rank{device}.csv") if out and os.path.isdir(out) \
            else os.path.join(tempfile.gettempdir(), f"eg_clocks_{os.getpid()}_{device}.csv")

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.close()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = max(mx, float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def path_bytes(c, es=4):
    """Algorithmic bytes of one field: read f, write labels, the graph and its
    value copies (maxima, saddles, beta0+, row_ptr as uint64, col).  es: bytes
    per value of the field's element type."""
    N, M, S, A = c["n_vertices"], c["n_maxima"], c["n_saddles"], c["n_arcs"]
    geometry = 4 * c["n_path_vertices"] + 8 * (c["n_paths"] + 1) if "n_path_vertices" in c else 0
    return es * N + 4 * N + (4 + es) * M + (5 + es) * S + 8 * (S + 1) + 4 * A + geometry


def kernel_bytes(c, es=4):
    """Compulsory bytes of each step's own contract (inputs read once, outputs
    written once).  classify: f, gradient pointers, critical records (12 B),
    counts; resolve: pointers in, labels out; emit: records in, graph out."""
    N, M, S, P, A = c["n_vertices"], c["n_maxima"], c["n_saddles"], c["n_paths"], c["n_arcs"]
    rec = 12 * (M + S)
    return {"classify": es * N + 4 * N + rec,
            "resolve": 4 * N + 4 * N,
            "emit": rec + 4 * P + (4 + es) * M + (5 + es) * S + 8 * (S + 1) + 4 * A}


SHORT_DTYPE = {"float32": "f32", "float64": "f64", "int8": "i8", "uint8": "u8", "int16": "i16",
               "uint16": "u16", "int32": "i32", "uint32": "u32", "int64": "i64", "uint64": "u64"}


def graph_d2h_bytes(c):
    M, S, A = c["n_maxima"], c["n_saddles"], c["n_arcs"]
    return 8 * M + 9 * S + 8 * (S + 1) + 4 * A


@contextlib.contextmanager
def quiet_gc():
    """Keep the interpreter's cyclic collector out of a timed region (as
    timeit does): this process holds many objects (fields, arrays, results),
    and a collection walking them in the middle of a run stalls the host loop
    that feeds the GPU.  Collect once, then exempt the existing objects."""
    gc.collect()
    gc.freeze()
    try:
        yield
    finally:
        gc.unfreeze()


def traffic_from_profiles(step, workload):
    """DRAM bytes per launch of `step`'s kernels on `workload` from the
    committed ncu summary, if it was taken on the kernels' current source
    (else None)."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(p):
        return None
    try:
        from paper_2303_02724_gb300 import _build
        e = json.load(open(p)).get("steps", {}).get(step, {}).get(workload)
        if not e or e.get("source_fingerprint") != _build.kernel_fingerprint(e.get("source", "")):
            return None
        return e.get("dram_bytes_per_launch")
    except Exception:
        return None


def dist_setup(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch
        import torch.distributed as dist
        if args.impl == "reference":
            return ws, rank, local
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    return ws, rank, local


# vertices of oracle work a reference-arm run may take in all (warm-up and
# timed steps): about three minutes on one host core
REF_BUDGET_VERTICES = 300_000_000


def ref_sample_cap(steps, warmup, requested):
    """Vertices per step of the reference arm: the requested sample (the
    cpu_baseline leg's), unless that many steps of it would take more than a
    few minutes (then proportionally fewer, at least 65,536)."""
    return min(requested, max(65536, REF_BUDGET_VERTICES // max(1, steps + warmup)))


def run_reference(args, ws, rank):
    if rank != 0:
        return
    import numpy as np
    import oracle
    sample_cap = ref_sample_cap(args.steps, args.warmup, args.ref_sample_vertices)
    if args.workload == "batch":
        from paper_2303_02724_gb300 import fields as F
        samples, n = [], 0
        for (e, sd, g) in F.batch_specs(3, args.batch_count):
            if n + int(np.prod(e)) > sample_cap:
                continue
            samples.append(F.batch_field(e, sd, g).values)
            n += int(np.prod(e))
        desc = f"{len(samples)} fields of the batch mix ({n} vertices)"
    elif args.workload == "serve":
        samples, n = [], 0
        for v in serve_fields(64):
            if n + int(v.size) > sample_cap:
                continue
            samples.append(v)
            n += int(v.size)
        desc = f"{len(samples)} requests of the served stream ({n} vertices)"
    else:
        fld = make_field(args.workload)
        sample, desc = oracle_slab(fld, sample_cap)
        samples, n = [sample], int(sample.size)
    for _ in range(args.warmup):
        for smp in samples:
            oracle.compute(smp)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        for smp in samples:
            oracle.compute(smp)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = n * args.steps / total / 1e6
    line = {
        "impl": "reference", "metric": "Mvertices/s full extremum graph (bit-exact)", "value": value,
        "unit": "Mvertices/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload], "sample": desc},
        "cpu_baseline": {"value": value, "unit": "Mvertices/s", "cores": 1, "kind": "oracle",
                         "sample": desc},
        "e2e": {"value": value, "unit": "Mvertices/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def batch_leg(args, ws, rank, local, steps, warmup):
    """Batched submission of the uneven 256-field mix vs per-field plain
    launches, both arms on the knobs the autotuner picked for the batch (and
    the plain arm once more on the library defaults).  Returns a dict."""
    import numpy as np
    import torch
    from paper_2303_02724_gb300 import _build, eg, fields as F
    from paper_2303_02724_gb300 import replicas
    _build.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    specs = F.batch_specs(3, args.batch_count)
    sizes = [int(np.prod(e)) for (e, _, _) in specs]
    mine = replicas.my_share(sizes, rank, ws)  # fields are independent: no data exchange
    flds = [F.batch_field(*specs[i]) for i in mine]
    ts = [torch.from_numpy(x.values).to(dev) for x in flds]
    nv_mine = sum(sizes[i] for i in mine)
    del flds
    stream = torch.cuda.current_stream(dev)
    h = eg.Handle(local)
    tuned = h.autotune(ts, stream)
    knobs = {k: tuned[k] for k in ["classify_rows", "classify_planes", "resolve_walks", "persistent_ctas"]}
    hp = eg.Handle(local, config=eg.EGConfig(**knobs))  # plain arm, same knobs
    hd = eg.Handle(local)  # plain arm, library defaults
    h.set_timing(True)
    bsteps = []

    def batched():
        ids = h.batch_submit(ts, stream)
        for rid in ids:
            h.get_graph_device(rid)
        bsteps.append(h.step_times(ids[0]))  # the batch's step times
        for rid in ids:
            h.release(rid)

    def plain_on(hh):
        def run():
            for t in ts:
                rid = hh.compute(t, stream)
                hh.get_graph_device(rid)
                hh.release(rid)
        return run

    out = {}
    for name, fn, hh in [("batched", batched, h), ("plain", plain_on(hp), hp), ("plain_default", plain_on(hd), hd)]:
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize(dev)
        if ws > 1:
            import torch.distributed as tdist
            tdist.barrier()
        l0 = hh.launch_count()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        with quiet_gc():
            e0.record(stream)
            for _ in range(steps):
                fn()
            e1.record(stream)
            torch.cuda.synchronize(dev)
        ms = replicas.reduce_max(e0.elapsed_time(e1) / steps, device=dev)
        out[name] = {"ms_per_step": ms, "value": sum(sizes) / (ms / 1e3) / 1e6,
                     "gpu_launches": int(hh.launch_count() - l0)}
    for hh in (h, hp, hd):
        hh.close()
    return {"workload": WORKLOADS["batch"], "fields": len(specs), "vertices": sum(sizes),
            "fields_this_rank": len(mine), "vertices_this_rank": nv_mine, "steps": steps, "warmup": warmup,
            "timing": "CUDA events on the launching stream around all steps; one step = every field of the "
                      "batch through the full path (results read back as device buffers)",
            "batched": out["batched"], "plain": out["plain"], "plain_default": out["plain_default"],
            "speedup_vs_plain": out["batched"]["value"] / out["plain"]["value"],
            "speedup_vs_plain_default": out["batched"]["value"] / out["plain_default"]["value"],
            "autotuned": knobs,
            "step_ms": {nm: statistics.mean(x[i] for x in bsteps[-steps:])
                        for i, nm in enumerate(["classify", "resolve", "emit"])}}


def run_batch(args, ws, rank, local):
    b = batch_leg(args, ws, rank, local, args.steps, args.warmup)
    if rank == 0:
        line = {"metric": "Mvertices/s full extremum graph (bit-exact), batched vs plain",
                "value": b["batched"]["value"], "unit": "Mvertices/s", "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": b["batched"]["ms_per_step"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": WORKLOADS["batch"], "fields": b["fields"], "vertices": b["vertices"],
                           "parallelism": f"fields sharded over {ws} ranks"},
                "batch": b, "gpu_launches": b["batched"]["gpu_launches"]}
        print(json.dumps(line), flush=True)


def serve_fields(count, seed=4):
    """Request fields: the seeded request shapes, values cropped at seeded
    offsets from a few large sum-of-Gaussian fields per dimension."""
    import numpy as np
    from paper_2303_02724_gb300 import fields as F
    specs = F.serve_requests(seed, count)
    rng = np.random.default_rng(seed + 1000)
    pools = {}
    out = []
    for (ext, fseed, ng) in specs:
        d = len(ext)
        if d not in pools:
            side = int(round(1e7 ** (1.0 / d))) + 2
            pools[d] = [F.serve_field((side,) * d, int(rng.integers(1 << 31)), 48).values for _ in range(3)]
        src = pools[d][fseed % 3]
        sl = tuple(slice(int(o), int(o) + int(e)) for o, e in
                   zip([rng.integers(0, src.shape[k] - e + 1) for k, e in enumerate(reversed(ext))], reversed(ext)))
        out.append(np.ascontiguousarray(src[sl]))
    return out


def serve_leg(args, ws, rank, local, n_requests, fractions):
    """Served stream: capacity (every request queued at once) and Poisson
    arrivals at fractions of it, through the continuous-batching loop; the
    client consumes each result as it completes (releases it), and the same
    requests one by one through the plain path for comparison."""
    import numpy as np
    import torch
    from paper_2303_02724_gb300 import _build, eg, serve
    _build.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    vals = serve_fields(n_requests)
    nv = sum(int(v.size) for v in vals)
    # requests arrive in page-locked host buffers (where a network receive
    # path would place them); the engines copy them straight to the device
    vals = [torch.from_numpy(v).pin_memory() for v in vals]
    free, _total = torch.cuda.mem_get_info(local)
    # results stay in device memory until the client, called as each request
    # completes, releases them
    # three engines (host threads with a handle and stream each) so that one's
    # host work overlaps the others' GPU work; batches of at most 32 requests
    # and 64 M vertices keep the tail short under streaming arrivals
    engines = [serve.GpuEngine(local, results="device") for _ in range(3)]
    budget = int(free * 0.6)

    def consume(r):
        if r.result is not None:
            r.result.release()

    def run(offsets):
        srv = serve.Server(engines, budget_bytes=budget, max_batch=32, max_batch_vertices=1 << 26,
                           on_done=consume)
        serve.replay(srv, vals[:len(offsets)], offsets)
        srv.drain(3600)
        srv.close()
        return srv.stats()

    run(np.zeros(len(vals)))  # warm-up: pools and staging buffers reach their steady size
    # everything queued at once: capacity, the median of three runs (a run
    # lasts a tenth of a second, and single runs differ by about 10%)
    caps = []
    for _ in range(3):
        with quiet_gc():
            caps.append(run(np.zeros(len(vals))))
    caps.sort(key=lambda c: c["throughput_mvps"])
    cap = dict(caps[1], runs_mvps=[c["throughput_mvps"] for c in caps], of_runs=3)
    rate_v = cap["throughput_mvps"] * 1e6
    mean_n = nv / len(vals)
    res = {}
    for frac in fractions:
        offs = serve.poisson_arrivals(frac * rate_v / mean_n, len(vals), 4)
        with quiet_gc():
            res[str(frac)] = run(offs)
    for e in engines:
        e.close()
    # the same requests one at a time through the plain path (upload, compute,
    # wait, release), for comparison with the served throughput
    hp = eg.Handle(local)
    for v in vals[:16]:
        rid = hp.compute(v.to(dev, non_blocking=True))
        hp.get_graph_device(rid)
        hp.release(rid)
    torch.cuda.synchronize(dev)
    with quiet_gc():
        t0 = time.perf_counter()
        for v in vals:
            rid = hp.compute(v.to(dev, non_blocking=True))
            hp.get_graph_device(rid)
            hp.release(rid)
        torch.cuda.synchronize(dev)
        plain_s = time.perf_counter() - t0
    hp.close()
    plain = {"throughput_mvps": nv / plain_s / 1e6, "seconds": plain_s,
             "mode": "each request alone: upload, eg_compute, wait, release"}
    return {"workload": WORKLOADS["serve"], "requests": len(vals), "vertices": nv, "budget_bytes": budget,
            "engines": len(engines), "timing": "host wall clock from the first arrival to the last completion",
            "requests_in": "page-locked host tensors, copied straight to the device",
            "capacity": cap, "poisson": res, "plain_one_by_one": plain,
            "speedup_vs_plain": cap["throughput_mvps"] / plain["throughput_mvps"]}


def run_serve(args, ws, rank, local):
    sv = serve_leg(args, ws, rank, local, args.serve_requests, args.serve_fractions)
    if rank == 0:
        line = {"metric": "served throughput (Mvertices/s) and latency", "value": sv["capacity"]["throughput_mvps"],
                "unit": "Mvertices/s", "n_gpus": ws, "steps": len(args.serve_fractions) + 1, "warmup": 1,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic",
                "config": {"workload": WORKLOADS["serve"], "requests": sv["requests"], "vertices": sv["vertices"],
                           "budget_bytes": sv["budget_bytes"], "engines": sv["engines"]},
                "serve": sv}
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="grf512", choices=sorted(WORKLOADS))
    ap.add_argument("--cpu-sample-vertices", type=int, default=4 * 1024 * 1024)
    ap.add_argument("--ref-sample-vertices", type=int, default=4 * 1024 * 1024,
                    help="oracle sample per step of the reference arm (the same slabs as the cpu_baseline leg; "
                         "fewer when the steps asked for would take the oracle more than a few minutes)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-threads", type=int, default=4,
                    help="host threads (one library handle each) taking turns in the end-to-end loop")
    ap.add_argument("--bundle", action="store_true",
                    help="also time arc bundling (eg_get_bundled) on one result of the workload")
    ap.add_argument("--cancel", type=float, nargs="*", default=None,
                    help="also time persistence-directed cancellation (eg_get_cancelled) on one result of the "
                         "workload at these thresholds (fractions of the range of maximum values; the rounds, "
                         "and so the time, grow steeply with the threshold on large fields)")
    ap.add_argument("--paths", action="store_true",
                    help="also gather the arc geometry (EG_FLAG_PATHS) in every timed step")
    ap.add_argument("--dtype", default="float32", choices=list(SHORT_DTYPE),
                    help="element type of the single-field workload: the field quantised onto the "
                         "integer type's range (plateaus for narrow types) or widened to float64")
    ap.add_argument("--batch-count", type=int, default=256)
    ap.add_argument("--serve-requests", type=int, default=4096)
    ap.add_argument("--serve-fractions", type=float, nargs="+", default=[0.5, 0.8, 0.95])
    ap.add_argument("--no-legs", action="store_true",
                    help="default workload only: skip the batched-vs-plain and served legs of the line")
    ap.add_argument("--leg-steps", type=int, default=10, help="timed passes of the batched-vs-plain leg")
    ap.add_argument("--leg-requests", type=int, default=1024, help="requests of the served leg")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)

    ws, rank, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, ws, rank)
        return
    if args.workload == "batch":
        run_batch(args, ws, rank, local)
        return
    if args.workload == "serve":
        run_serve(args, ws, rank, local)
        return

    import numpy as np
    import torch
    from paper_2303_02724_gb300 import _build, eg

    _build.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    fld = make_field(args.workload)
    typed = args.dtype != "float32"
    if typed:
        from paper_2303_02724_gb300 import fields as F
        fld = F.quantise(fld, args.dtype)
    es = fld.values.dtype.itemsize
    N = fld.n
    t_field = eg.device_array(fld.values, local)
    stream = torch.cuda.current_stream(dev)
    h = eg.Handle(local, paths=args.paths)
    h.set_timing(True)

    def step():
        rid = h.compute(t_field, stream, dtype=fld.values.dtype if typed else None)
        g = h.get_graph_device(rid)  # waits for the result (counts only)
        return rid, g

    L2_BYTES = 129 * 1024 * 1024
    flush = None if es * N > 2 * L2_BYTES else torch.empty(64 << 20, dtype=torch.int32, device=dev)
    counts = None
    for _ in range(args.warmup):
        rid, g = step()
        counts = dict(n_vertices=g.n_vertices, n_maxima=g.n_maxima, n_saddles=g.n_saddles,
                      n_paths=g.n_paths, n_arcs=g.n_arcs)
        if args.paths:
            counts["n_path_vertices"] = h.path_count(rid)
        h.release(rid)

    clocks = ClockSampler(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize(dev)
    clocks.start()
    launches0 = h.launch_count()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize(dev)
    step_ms = []
    with quiet_gc():
        if flush is None:
            e0.record(stream)
            for _ in range(args.steps):
                rid, g = step()
                step_ms.append(h.step_times(rid))
                h.release(rid)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            ms_total = e0.elapsed_time(e1)
        else:
            # field smaller than L2: overwrite L2 before every step, outside
            # the timed spans
            ms_total = 0.0
            for _ in range(args.steps):
                flush.add_(1)
                e0.record(stream)
                rid, g = step()
                e1.record(stream)
                torch.cuda.synchronize(dev)
                ms_total += e0.elapsed_time(e1)
                step_ms.append(h.step_times(rid))
                h.release(rid)
    if dist is not None:
        dist.barrier()
    launches = h.launch_count() - launches0
    clk = clocks.stop()
    if dist is not None:
        t = torch.tensor([ms_total], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_total = float(t.item())
    value = N * args.steps * ws / (ms_total / 1e3) / 1e6

    # roofline of the dominant step (device time from the library's events)
    names = ["classify", "resolve", "emit"]
    mean_ms = {nm: statistics.mean(s[i] for s in step_ms) for i, nm in enumerate(names)}
    dom = max(mean_ms, key=mean_ms.get)
    kb = kernel_bytes(counts, es)
    peak, peak_kind = peaks()
    achieved = kb[dom] / (mean_ms[dom] / 1e3) / 1e9
    mean_step_ms = statistics.mean(s[3] for s in step_ms)
    pb = path_bytes(counts, es)
    path_achieved = pb / (mean_step_ms / 1e3) / 1e9

    bundle = None
    if args.bundle:
        rid, g = step()
        h.get_bundled(rid)  # warm-up
        torch.cuda.synchronize(dev)
        reps = 5
        t0 = time.perf_counter()
        for _ in range(reps):
            keep = h.get_bundled(rid)
        bms = (time.perf_counter() - t0) / reps * 1e3
        h.release(rid)
        bundle = {"ms": bms, "timing": "host wall clock per eg_get_bundled call (device work, two waits, "
                  "copy of the keep mask)", "saddles": int(keep.size), "kept": int(keep.sum())}

    cancel = None
    if args.cancel is not None:
        rid, g = step()
        gh = h.get_graph(rid, labels=False)
        spread = float(np.float32(gh.max_val.max()) - np.float32(gh.max_val.min()))
        cancel = []
        for frac in (args.cancel or [0.0005, 0.001]):
            tau = float(np.float32(spread * frac)) if np.isfinite(frac) else float("inf")
            h.get_cancelled(rid, tau)  # warm-up
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            alive, surv, n, rounds = h.get_cancelled(rid, tau)
            cancel.append({"tau_fraction_of_range": frac, "tau": tau, "ms": (time.perf_counter() - t0) * 1e3,
                           "cancelled": n, "rounds": rounds, "saddles": int(alive.size),
                           "surviving_maxima": int(np.unique(surv).size)})
        h.release(rid)

    # end to end through the C ABI with host buffers: H2D of the field and
    # D2H of the graph inside the timed region
    e2e = None
    if not args.no_e2e and not args.paths and not typed:
        host = torch.from_numpy(fld.values).pin_memory().numpy()
        # two host threads, each with its own handle, stream and page-locked
        # output buffers (allocated once, reused), take alternate steps, so one
        # step's upload and kernels overlap the other's kernels and download
        import threading
        nw = max(1, args.e2e_threads)
        hs = [h] + [eg.Handle(local) for _ in range(nw - 1)]
        sts = [stream] + [torch.cuda.Stream(device=dev) for _ in range(nw - 1)]
        outbs = [eg.GraphBuffers(counts["n_maxima"], counts["n_saddles"], counts["n_arcs"], pinned=True)
                 for _ in hs]

        def e2e_worker(w, k_steps, errs):
            try:
                torch.cuda.set_device(dev)
                for _ in range(w, k_steps, nw):
                    rid = hs[w].compute_host(host, sts[w])
                    hs[w].get_graph(rid, labels=False, buffers=outbs[w])
                    hs[w].release(rid)
            except Exception as ex:  # reported after the join
                errs.append(ex)

        def e2e_run(k_steps):
            errs = []
            th = [threading.Thread(target=e2e_worker, args=(w, k_steps, errs)) for w in range(nw)]
            for t in th:
                t.start()
            for t in th:
                t.join()
            if errs:
                raise errs[0]

        e2e_run(2 * nw)
        torch.cuda.synchronize(dev)
        if dist is not None:
            dist.barrier()
        with quiet_gc():
            t0 = time.perf_counter()
            e2e_run(args.steps)
            torch.cuda.synchronize(dev)
            e2e_s = time.perf_counter() - t0
        for hx in hs[1:]:
            hx.close()
        if dist is not None:
            t = torch.tensor([e2e_s], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            e2e_s = float(t.item())
        e2e_value = N * args.steps * ws / e2e_s / 1e6

        e2e = {"value": e2e_value, "unit": "Mvertices/s", "h2d_bytes_per_step": 4 * N,
               "d2h_bytes_per_step": graph_d2h_bytes(counts),
               "mode": "eg_compute_host + eg_get_graph + eg_release per step, pinned host buffers; "
                       f"{nw} host threads with a handle each take turns, so uploads, kernels and downloads "
                       "of consecutive steps overlap"}

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        import oracle
        sample, desc = oracle_slab(fld, args.cpu_sample_vertices)
        # 7 runs, the best and the worst dropped, the other 5 averaged
        runs = []
        for _ in range(7):
            t0 = time.perf_counter()
            oracle.compute(sample, dtype=sample.dtype)
            runs.append(time.perf_counter() - t0)
        dt = statistics.mean(sorted(runs)[1:-1])
        cpu = {"value": sample.size / dt / 1e6, "unit": "Mvertices/s", "cores": 1, "kind": "oracle",
               "sample": desc + f", mean of 5 of 7 runs (best and worst dropped), {dt:.2f} s per run",
               "host": host_cpu()}

    # the metric's second half on the default line: the batched form against
    # per-field plain launches on the uneven mix, and a short served stream
    legs = {}
    if args.workload == "grf512" and not args.no_legs and not args.paths and not typed:
        h.close()
        torch.cuda.empty_cache()
        legs["batch"] = batch_leg(args, ws, rank, local, args.leg_steps, args.warmup)
        torch.cuda.empty_cache()
        if ws == 1:
            legs["serve"] = serve_leg(args, ws, rank, local, args.leg_requests, [0.8])

    if rank == 0:
        line = {
            "metric": "Mvertices/s full extremum graph (bit-exact)", "value": value, "unit": "Mvertices/s",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": SHORT_DTYPE[args.dtype],
            "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload] + ("; with the arc geometry (EG_FLAG_PATHS)"
                                                               if args.paths else "")
                       + (f"; quantised to {args.dtype}" if typed and fld.values.dtype.kind in "iu" else "")
                       + ("; widened to float64" if args.dtype == "float64" else ""),
                       "vertices": N, "l2": "inputs larger than L2"
                       if flush is None else "L2 flushed before every step (256 MB written)",
                       "parallelism": f"replicas x{ws}", **{k: v for k, v in counts.items() if k != "n_vertices"}},
            "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_kind": peak_kind,
                         "traffic": None if typed else traffic_from_profiles(dom, args.workload),
                         "algorithmic_bytes": kb[dom], "ms": mean_ms[dom]},
            "path_roofline": {"achieved": path_achieved, "frac": path_achieved / peak,
                              "algorithmic_bytes": pb, "ms": mean_step_ms},
            "step_ms": mean_ms,
            "e2e": e2e,
            "gpu_launches": int(launches),
            "clocks": clk,
            "cpu_baseline": cpu,
        }
        if bundle is not None:
            line["bundle"] = bundle
        if cancel is not None:
            line["cancel"] = {"timing": "host wall clock per eg_get_cancelled call (setup, all rounds in one "
                                        "cooperative launch, copies of the results)", "runs": cancel}
        line.update(legs)
        print(json.dumps(line), flush=True)
    h.close()
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
