"""Throughput benchmark of the Downstream tracking + two-track vertexing path.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

One step = ds_reconstruct + ds_vertex over one batch of 1000 synthetic events
shaped like the paper's minimum-bias workload (Poisson(300) SciFi seeds, 40 %
true, 5000 UT hits per event, 16-32-32-1 ghost killer in FP32, opposite-charge
vertexing with DOCA < 2 mm), inputs resident in HBM.  Inputs rotate over
replicas totalling more than three times the L2, so every step reads cold
inputs.  Steps are issued round-robin on STREAMS CUDA streams, each with its
own library context (workspaces and outputs), so consecutive batches overlap
(the whole-job throughput a production loop gets); the same steps on one
stream are reported as `single_stream`.  Prints one JSON line (rank 0).

Under torchrun each rank processes its own batch (weak scaling, no
collective on the data path); value = all events / max-over-ranks time.
--impl reference times the FP64 CPU oracle on the host cores instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

L2_BYTES = 126 * 2 ** 20
N_EVENTS = 1000
WORKLOAD = ("c2: 1000 events/step, Poisson(300) SciFi seeds (40% true), 5000 UT hits/event, "
            "16-32-32-1 ghost killer FP32, opposite-charge vertexing DOCA<2mm")
STREAMS = 4             # concurrent batches in the headline measurement


def dist_info():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def aggregate(elapsed_s: list, events_per_rank: int, steps: int) -> dict:
    """Whole-job throughput: every rank's events over the slowest rank's time."""
    t = max(elapsed_s)
    n = len(elapsed_s) * events_per_rank * steps
    return dict(value=n / t, ms_per_step=1e3 * t / steps, events=n)


def max_over_ranks(x: float) -> float:
    """The largest x over all ranks (the job's time is its slowest rank's)."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return x
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6400.0), d.get("sm_max_mhz", 2032.0), "measured"
    return 6400.0, 2032.0, "fallback"


class Clocks:
    """nvidia-smi sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, out_path: str | None):
        self.p = None
        self.path = out_path
        try:
            self.f = open(out_path, "w") if out_path else subprocess.DEVNULL
            self.p = subprocess.Popen(["nvidia-smi", f"--id={gpu_index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None

    def stop(self) -> dict:
        if self.p is None:
            return dict(sm_mhz=None, sm_max_mhz=None, reasons=["nvidia-smi unavailable"])
        self.p.terminate()
        out, _ = self.p.communicate(timeout=10)
        if self.path:
            with open(self.path, "w") as f:
                f.write(out)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            c = [x.strip() for x in line.split(",")]
            if len(c) < 9:
                continue
            try:
                sm.append(float(c[1])); smax.append(float(c[2]))
            except ValueError:
                continue
            for n, v in zip(names, c[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return dict(sm_mhz=None, sm_max_mhz=None, reasons=["no samples"])
        return dict(sm_mhz=float(np.median(sm)), sm_max_mhz=float(max(smax)), reasons=sorted(reasons),
                    samples=len(sm))


MLP_FLOP = 2 * (16 * 32 + 32 * 32 + 32)          # 16-32-32-1 network: multiply-adds x 2


def algorithmic(E, S, H, n_t, n_v, n_cand, n_pairs, table_stride, fused=True):
    """Bytes each kernel of a step moves through HBM, this design's
    workspaces included (each read once, each write once), and FLOPs.  C =
    candidates, T = tracks, V = vertices, P = opposite-charge pairs."""
    tb = 2 * table_stride * E                    # per-event bin tables
    mlp_flop = MLP_FLOP
    # seeds (24 B), staged x0 + index map (6 B/hit), tables; fused: the pick
    # key + hit ids (24 B) and rank (4 B) per seed and one record per track;
    # unfused: candidates (64 B inputs + 48 B fit) + per-seed range and rank
    search = (24 * S + 6 * H + tb + 28 * S + 64 * n_t) if fused else (24 * S + 6 * H + tb + 112 * n_cand + 20 * S)
    return {
        # hits in (13 B) -> sorted x0 (4 B) + index inside the event (2 B) + tables
        "k_bucket": dict(bytes=13 * H + 6 * H + tb),
        "k_search": dict(bytes=search, flop=mlp_flop * n_cand if fused else 0),
        "k_mlp": dict(bytes=68 * n_cand, flop=mlp_flop * n_cand),
        "k_pick": dict(bytes=16 * S + 20 * n_cand + 48 * n_t + 88 * S),
        "k_clone": dict(bytes=28 * S + 8 * E),
        "k_scatter_tracks": dict(bytes=4 * S + 128 * n_t),
        "k_vertex_small": dict(bytes=20 * n_t + 36 * n_v),
        "k_vertex_large": dict(bytes=0),
        "k_scatter_vertices": dict(bytes=68 * n_v),
    }


def method_bytes(S, H, n_t, n_v):
    """Algorithmic bytes per launch in the method's own units (each input read
    once, each output written once: seeds 24 B, UT hits 13 B, tracks 64 B,
    vertices 32 B), assigned to the kernels that read or write them.  Kernels
    that only move this design's intermediates (candidates, winners, ranks)
    have none."""
    return {
        "k_bucket": 13 * H,
        "k_search": 24 * S + 13 * H,
        "k_scatter_tracks": 64 * n_t,
        "k_vertex_small": 64 * n_t + 32 * n_v,
        "k_scatter_vertices": 32 * n_v,
    }


def traffic_for(kernel: str):
    """Per-launch DRAM bytes from the committed ncu summary, if the kernel's
    source has not changed since it was taken."""
    import hashlib
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    e = d.get(kernel)
    if not e:
        return None
    src = os.path.join(ROOT, "paper_2503_13092_b300", "csrc", e["source"])
    if not os.path.exists(src) or hashlib.sha256(open(src, "rb").read()).hexdigest()[:16] != e["sha"]:
        return None
    return e["bytes_per_launch"]


def step_traffic():
    """Per-step DRAM bytes (read + write) summed over the kernels of the
    committed ncu capture, if every kernel's source is unchanged since."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    tot = 0.0
    for k, e in d.items():
        if not isinstance(e, dict) or "bytes_per_launch" not in e:
            continue
        b = traffic_for(k)
        if b is None:
            return None
        tot += b * e.get("launches_per_step", 1)
    return tot


def h2d_ceiling(torch, arrays, reps=5, d2h_bytes=0):
    """Upload rate of the e2e step's own pinned host arrays with nothing else
    running: one cudaMemcpyAsync per array (as the serving path issues them)
    on one stream, and the same copies spread over two streams; with
    d2h_bytes, also the rate of one download of that size into pinned host
    memory with nothing else running."""
    from cuda.bindings import runtime as rt
    nbytes = sum(a.nbytes for a in arrays)
    dst = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    h2d = rt.cudaMemcpyKind.cudaMemcpyHostToDevice

    def issue(n_streams):
        off = 0
        for k, a in enumerate(arrays):
            st = streams[k % n_streams]
            err, = rt.cudaMemcpyAsync(dst.data_ptr() + off, a.ctypes.data, a.nbytes, h2d, st.cuda_stream)
            assert err == rt.cudaError_t.cudaSuccess, err
            off += a.nbytes

    def timed(fn, st):
        fn()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        streams[1].wait_stream(streams[0])
        for _ in range(reps):
            fn()
        streams[0].wait_stream(streams[1])
        e1.record(st)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) * 1e-3

    res = dict(bytes=nbytes, copies=len(arrays))
    for name, ns in (("one_stream", 1), ("two_streams", 2)):
        res[name + "_gbs"] = nbytes * reps / timed(lambda: issue(ns), streams[0]) / 1e9
    if d2h_bytes:
        src = torch.empty(d2h_bytes, dtype=torch.uint8, device="cuda")
        host = torch.empty(d2h_bytes, dtype=torch.uint8).pin_memory()
        d2h = rt.cudaMemcpyKind.cudaMemcpyDeviceToHost

        def down():
            err, = rt.cudaMemcpyAsync(host.data_ptr(), src.data_ptr(), d2h_bytes, d2h, streams[0].cuda_stream)
            assert err == rt.cudaError_t.cudaSuccess, err

        res["d2h_bytes"] = d2h_bytes
        res["d2h_gbs"] = d2h_bytes * reps / timed(down, streams[0]) / 1e9
        # both directions at once: the uploads on one stream, the download on
        # another; time until both are done
        s3 = torch.cuda.Stream()

        def both():
            issue(1)
            err, = rt.cudaMemcpyAsync(host.data_ptr(), src.data_ptr(), d2h_bytes, d2h, s3.cuda_stream)
            assert err == rt.cudaError_t.cudaSuccess, err

        both()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        e0.record(streams[0])
        s3.wait_stream(streams[0])
        for _ in range(reps):
            both()
        streams[0].wait_stream(s3)
        e1.record(streams[0])
        torch.cuda.synchronize()
        res["up_and_down_concurrent_ms"] = e0.elapsed_time(e1) / reps
    return res


def run_cpu_baseline(batch, cfg, w, target_s=12.0):
    import oracle
    cores = os.cpu_count() or 1
    E = batch["n_events"]
    n = 16
    while True:
        ev = list(range(min(n, E)))
        sb = _sub(batch, ev)
        t0 = time.perf_counter()
        r = oracle.reconstruct(sb, cfg, w, n_threads=cores)
        tk = oracle.tracks_from(r, sb["seed_off"])
        st = tk["state"].astype(np.float32)
        oracle.vertex(cfg, tk["trk_off"], st[:, 0], st[:, 1], st[:, 2], st[:, 3], st[:, 4])
        dt = time.perf_counter() - t0
        if dt > 0.25 * target_s or n >= E:
            break
        n = min(E, int(n * max(2.0, 0.5 * target_s / max(dt, 1e-3))))
    # the same oracle on one thread (a smaller sample of the same events)
    n1 = min(16, E)
    sb1 = _sub(batch, list(range(n1)))
    t1 = time.perf_counter()
    r1 = oracle.reconstruct(sb1, cfg, w, n_threads=1)
    tk1 = oracle.tracks_from(r1, sb1["seed_off"])
    st1 = tk1["state"].astype(np.float32)
    oracle.vertex(cfg, tk1["trk_off"], st1[:, 0], st1[:, 1], st1[:, 2], st1[:, 3], st1[:, 4])
    dt1 = time.perf_counter() - t1
    return dict(value=len(ev) / dt, unit="events/s", cores=cores, kind="oracle", cpu_model=cpu_model(),
                sample=f"first {len(ev)} events of the step's batch, reconstruct + vertex, "
                       f"{cores} threads (one event per thread), {dt:.2f} s",
                single_thread=dict(value=n1 / dt1, unit="events/s", sample=f"first {n1} events, one thread, {dt1:.2f} s"))


def cpu_model():
    """The host CPU's model name (Linux /proc/cpuinfo), or None."""
    try:
        for line in open("/proc/cpuinfo"):
            if line.startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return None


def _sub(b, events):
    out = dict(n_events=len(events))
    so, ho, si, hi = [0], [0], [], []
    for e in events:
        s0, s1, h0, h1 = int(b["seed_off"][e]), int(b["seed_off"][e + 1]), int(b["hit_off"][e]), int(b["hit_off"][e + 1])
        si.append(np.arange(s0, s1)); hi.append(np.arange(h0, h1))
        so.append(so[-1] + s1 - s0); ho.append(ho[-1] + h1 - h0)
    si, hi = np.concatenate(si), np.concatenate(hi)
    out["seed_off"] = np.array(so, np.int32); out["hit_off"] = np.array(ho, np.int32)
    for k in ("seed_x", "seed_y", "seed_tx", "seed_ty", "seed_qop", "seed_chi2"):
        out[k] = b[k][si]
    for k in ("hit_x0", "hit_ybeg", "hit_yend", "hit_layer"):
        out[k] = b[k][hi]
    return out


def replicas_for(E, S, H):
    """Input replicas the timed steps rotate over, so that every step reads
    inputs that are not in L2 (more than three L2s of inputs in all)."""
    in_bytes = 24 * S + 13 * H + 8 * (E + 1)
    R = max(2, math.ceil(3 * L2_BYTES / in_bytes))
    return STREAMS * math.ceil(R / STREAMS), in_bytes    # replica k % R belongs to stream k % STREAMS


def workload_config(E, S, H, ws):
    """The `config` of both arms' JSON lines: the workload and how L2 is kept
    out of the timing (run statistics go to `step_stats`)."""
    R, in_bytes = replicas_for(E, S, H)
    return dict(workload=WORKLOAD, n_events=E, n_seeds=S, n_hits=H, mlp="fp32",
                l2=f"inputs rotate over {R} replicas ({R * in_bytes / 2**20:.0f} MB > 3x L2)",
                parallelism=f"replicas x{ws}" if ws > 1 else "single GPU")


def bench_reference(args):
    """FP64 CPU oracle, as it stands, on the host cores (rank 0 only)."""
    ws, rank, _ = dist_info()
    if rank != 0:
        return 0
    import oracle
    from paper_2503_13092_b300 import synth
    batch = synth.config_batch("c2")
    cfg = synth.default_config()
    w = synth.nn_weights()
    cores = os.cpu_count() or 1
    per_step = max(8, min(N_EVENTS, 4 * cores))
    times = []
    for k in range(args.warmup + args.steps):
        ev = [(k * per_step + i) % N_EVENTS for i in range(per_step)]
        sb = _sub(batch, ev)
        t0 = time.perf_counter()
        r = oracle.reconstruct(sb, cfg, w, n_threads=cores)
        tk = oracle.tracks_from(r, sb["seed_off"])
        st = tk["state"].astype(np.float32)
        oracle.vertex(cfg, tk["trk_off"], st[:, 0], st[:, 1], st[:, 2], st[:, 3], st[:, 4])
        if k >= args.warmup:
            times.append(time.perf_counter() - t0)
    t = sum(times)
    val = per_step * args.steps / t
    line = dict(metric="events/s per B300 (Downstream+vertexing)", value=val, unit="events/s", n_gpus=args.gpus,
                steps=args.steps, warmup=args.warmup, ms_per_step=1e3 * t / args.steps, higher_is_better=True,
                scaling="weak", vs_baseline=None, dtype="f64", data="synthetic", impl="reference",
                config=workload_config(int(batch["n_events"]), int(batch["seed_off"][-1]), int(batch["hit_off"][-1]), ws),
                cpu_baseline=dict(value=val, unit="events/s", cores=cores, kind="oracle",
                                  sample=f"{per_step} events per step of the same batch, {cores} threads",
                                  sample_events_per_step=per_step),
                e2e=dict(value=val, unit="events/s", h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line), flush=True)
    return 0


def selection(batch, g):
    """Truth efficiency (true seeds whose track has >= 3 hits of their own
    track) and ghost rate (tracks that do not) of one reconstruction."""
    t = g["tracks"]
    st = batch["seed_track"][t["seed"]]
    h = t["hit"]
    own = ((h >= 0) & (batch["hit_track"][np.clip(h, 0, None)] == st[:, None])).sum(1)
    good = (st >= 0) & (own >= 3)
    return dict(efficiency=float(good.sum() / max((batch["seed_track"] >= 0).sum(), 1)),
                ghost_rate=float(1.0 - good.mean()) if len(t) else 0.0, tracks=int(len(t)))


def reduced_precision_forms(d, ds, torch, batch, devs, ref, step, n_prof, stream, kernels, n_cand):
    """The ghost-killer network on the tensor cores (BF16, FP8) against the FP32
    network on the same batch (the weights loaded in d): k_mlp time, share of
    seeds whose selected track changes, the response change on tracks both
    keep, and the selection's truth efficiency and ghost rate.  Also
    ds_mlp_eval alone on 2^20 feature rows (kernel throughput without the rest
    of the step)."""
    S = int(batch["seed_off"][-1])

    def per_seed(g):
        t = g["tracks"]
        has = np.zeros(S, bool); hits = np.full((S, 4), -1, np.int64); nn = np.zeros(S)
        has[t["seed"]] = True; hits[t["seed"]] = t["hit"]; nn[t["seed"]] = t["nn"]
        return has, hits, nn

    h32, k32, n32 = per_seed(ref)
    rng = np.random.default_rng(17)
    n_rows = 1 << 20
    feats = torch.from_numpy(rng.standard_normal((n_rows, 16)).astype(np.float32)).cuda()
    logit = torch.empty(n_rows, dtype=torch.float32, device="cuda")
    forms = {}
    for name, prec in (("fp32", ds.DS_MLP_FP32), ("bf16", ds.DS_MLP_BF16), ("fp8_e4m3", ds.DS_MLP_FP8)):
        d.set_params(mlp_precision=prec)
        f = {}
        if prec != ds.DS_MLP_FP32:
            for k in range(3):      # first launches of this kernel variant load it
                step(k)
            d.sync(stream)
            ds.ds_profile_enable(d.ctx, True)
            for k in range(n_prof):
                step(k)
            pr = ds.ds_profile_read(d.ctx)
            ds.ds_profile_enable(d.ctx, False)
            d.sync(stream)
            f["k_mlp_us"] = 1e3 * pr["k_mlp"][1] / max(pr["k_mlp"][0], 1)
            g = d.run(batch, dev=devs[0])
            hl, kl, nl = per_seed(g)
            flip = (h32 != hl) | (h32 & hl & np.any(k32 != kl, axis=1))
            both = h32 & hl & ~flip
            dn = np.abs(nl[both] - n32[both])
            f.update(seed_flip_rate=float(flip.mean()),
                     response_err_max=float(dn.max()) if dn.size else 0.0,
                     response_err_mean=float(dn.mean()) if dn.size else 0.0, **selection(batch, g))
        elif "k_mlp" in kernels:
            f["k_mlp_us"] = kernels["k_mlp"]["avg_us"]
            f.update(selection(batch, ref))
        else:       # the FP32 network runs inside k_search (no separate launch)
            f["k_mlp_us"] = None
            f["network"] = "fused into k_search"
            f["k_search_us"] = kernels["k_search"]["avg_us"]
            f.update(selection(batch, ref))
        if f["k_mlp_us"]:
            f["k_mlp_candidates_per_s"] = n_cand / (f["k_mlp_us"] * 1e-6)
        for _ in range(3):
            ds.ds_mlp_eval(d.ctx, feats, logit, prec, stream)
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(10):
            ds.ds_mlp_eval(d.ctx, feats, logit, prec, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        us = e0.elapsed_time(e1) * 1e3 / 10
        f["eval_1M_us"] = us
        f["eval_rows_per_s"] = n_rows / (us * 1e-6)
        f["eval_tflops"] = MLP_FLOP * n_rows / (us * 1e-6) / 1e12
        f["eval_gbs"] = 68 * n_rows / (us * 1e-6) / 1e9
        forms[name] = f
    d.set_params(mlp_precision=ds.DS_MLP_FP32)
    d.sync(stream)
    return forms


def bench_c3(ds, torch, cfg, w, steps, warmup, dev_index):
    """Config 3: 10000 events of log-normal occupancy in one graph-captured step;
    the search launch shape is first left at its default, then chosen by the
    autotuner on the same batch."""
    from paper_2503_13092_b300 import synth
    t_gen = time.perf_counter()
    b = synth.config_batch("c3", seed=3)
    t_gen = time.perf_counter() - t_gen
    E, S, H = b["n_events"], int(b["seed_off"][-1]), int(b["hit_off"][-1])
    d = ds.Downstream(cfg, w, device=dev_index)
    ds.ds_reserve(d.ctx, E, S, H)
    dv = d.to_device(b)
    probe = d.run(b, dev=dv)
    n_t, n_v = probe["n_tracks"], probe["n_vertices"]
    out = d.alloc_tracks(E, S)
    vout = d.alloc_vertices(E, 2 * n_v + 4096)
    stream = torch.cuda.current_stream()

    def timed(label):
        for _ in range(warmup):
            d.reconstruct(dv, out, stream); d.vertex(out, vout, stream)
        d.sync(stream)
        g = torch.cuda.CUDAGraph()
        cap = torch.cuda.Stream()
        with torch.cuda.graph(g, stream=cap):
            cs = torch.cuda.current_stream()
            d.reconstruct(dv, out, cs)
            d.vertex(out, vout, cs)
        for _ in range(2):
            g.replay()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            g.replay()
        e1.record(stream)
        torch.cuda.synchronize()
        st = d.sync(stream)
        assert st["status"] == 0, st
        ms = e0.elapsed_time(e1) / steps
        return dict(value=E / (ms * 1e-3), ms_per_step=ms, tuning=ds.ds_get_tuning(d.ctx).as_dict())

    default = timed("default")
    # per-kernel CUDA-event times of one profiled (eager) step
    d.sync(stream)
    ds.ds_profile_enable(d.ctx, True)
    for _ in range(2):
        d.reconstruct(dv, out, stream); d.vertex(out, vout, stream)
    pr = ds.ds_profile_read(d.ctx)
    ds.ds_profile_enable(d.ctx, False)
    d.sync(stream)
    c3_kernels = {k: dict(launches=v[0], avg_us=1e3 * v[1] / max(v[0], 1)) for k, v in pr.items()}
    t_tune = time.perf_counter()
    best, entries = ds.ds_autotune(d.ctx, dv, out, reps=2)
    t_tune = time.perf_counter() - t_tune
    tuned = timed("tuned")
    hits = np.diff(b["hit_off"]); seeds = np.diff(b["seed_off"])
    res = dict(workload="C3: 10000 events, occupancy LogNormal(0, 0.77): seeds 20-2000, UT hits 300-30000 per event",
               unit="events/s", n_events=E, n_seeds=S, n_hits=H, tracks=n_t, vertices=n_v,
               seeds_per_event=[int(seeds.min()), int(seeds.max())], hits_per_event=[int(hits.min()), int(hits.max())],
               default=default, autotuned=tuned, autotune_s=t_tune, autotune_configs=len(entries),
               kernels=c3_kernels,
               generate_s=t_gen, inputs_mb=(24 * S + 13 * H) / 2**20,
               step="one CUDA graph replay: ds_reconstruct + ds_vertex over all 10000 events")
    d.close()
    return res


def bench_c5(ds, torch, cfg, w, dev_index, n_requests=1000):
    """Config 5: the serving loop under Poisson arrivals of requests of 1-500
    events of config-1 occupancy, latency counted from each request's arrival
    to its results on the host (uploads and downloads included).  The batched
    form (continuous batching, 4 slots, BF16 tensor-core ghost killer) is set
    against the plain form (one request at a time, one event per launch,
    FP32) on the same requests."""
    from paper_2503_13092_b300 import synth
    pool = synth.c5_pool(4000, seed=5)
    for k in ("seed_x", "seed_y", "seed_tx", "seed_ty", "seed_qop", "seed_chi2", "hit_x0", "hit_ybeg", "hit_yend",
              "hit_layer"):
        pool[k] = torch.from_numpy(np.ascontiguousarray(pool[k])).pin_memory().numpy()
    sizes, starts, gaps = synth.c5_trace(n_requests, 1.0, pool["n_events"], seed=5)
    reqs = [synth.slice_events(pool, int(a), int(a + k)) for k, a in zip(sizes, starts)]
    ev = np.array([r["n_events"] for r in reqs])

    def truth(res, r):
        """(true seeds, found with >= 3 hits of their own track, tracks kept)."""
        st = r["seed_track"]; ht = r["hit_track"]
        t = res["tracks"]
        tid = st[t["seed"]]
        h = t["hit"]
        own = (h >= 0) & (ht[np.clip(h, 0, None)] == tid[:, None])
        good = int(np.sum((tid >= 0) & (own.sum(1) >= 3)))
        return int(np.sum(st >= 0)), good, len(t)

    def pinned(n, dtype):
        t = torch.empty(n * np.dtype(dtype).itemsize, dtype=torch.uint8, pin_memory=True)
        return t.numpy().view(dtype)

    # every request's output buffers (a track per seed, a vertex per seed + 4096)
    # carved from two pinned blocks allocated once, so that no pinned allocation
    # happens while requests are in flight however many are outstanding
    n_seeds = np.array([int(r["seed_off"][-1]) for r in reqs])
    n_vcap = n_seeds + 4096
    slab_t, slab_v = pinned(int(n_seeds.sum()) + 1, ds.TRACK_DTYPE), pinned(int(n_vcap.sum()), ds.VERTEX_DTYPE)
    t_at, v_at = np.concatenate([[0], np.cumsum(n_seeds)]), np.concatenate([[0], np.cumsum(n_vcap)])
    out_views = [dict(tracks=slab_t[t_at[i]:t_at[i] + max(1, n_seeds[i])], vertices=slab_v[v_at[i]:v_at[i + 1]])
                 for i in range(len(reqs))]

    def serve(config, idx, arrivals=None, window=64, accuracy=False):
        """arrivals None: closed loop, `window` requests outstanding (capacity);
        else open loop: each request is submitted at its arrival time by a
        submitter thread."""
        import threading
        srv = ds.Server(cfg, w, device=dev_index, **config)
        ids, got, acc = {}, {}, []
        peak = [0]                             # most requests outstanding at a submission
        lock = threading.Lock()

        def submit(i, arrival=0.0):
            o = dict(out_views[i])
            E = int(reqs[i]["n_events"])
            o["trk_off"] = np.zeros(E + 1, np.int32)
            o["vtx_off"] = np.zeros(E + 1, np.int32)
            rid = srv.submit(reqs[i], arrival=arrival, out=o)
            ids[rid] = i
            peak[0] = max(peak[0], len(ids) - len(got))

        def take(cs):
            for c in cs:
                i = ids[c["id"]]
                if accuracy:
                    acc.append(truth(c, reqs[i]))
                c.pop("tracks"); c.pop("vertices")
                got[c["id"]] = c

        t_start = srv.now()
        client_s = 0.0                      # client time between polls (scoring, resubmission)
        if arrivals is None:
            todo = list(idx)
            with lock:
                for i in todo[:window]:
                    submit(i)
            todo = todo[window:]
            while len(got) < len(idx):
                cs = srv.poll(timeout=1.0)
                tc = time.perf_counter()
                with lock:
                    take(cs)
                    for _ in cs:
                        if todo:
                            submit(todo.pop(0))
                client_s += time.perf_counter() - tc
            t_first = t_start
        else:
            t0 = srv.now() + 0.05
            t_first = t0 + float(arrivals[0])

            def submitter():
                for i, a in zip(idx, arrivals):
                    wait = t0 + a - 1e-3 - srv.now()
                    if wait > 0:
                        time.sleep(wait)
                    with lock:
                        submit(i, arrival=t0 + a)

            th = threading.Thread(target=submitter)
            th.start()
            while len(got) < len(idx):
                cs = srv.poll(timeout=1.0)
                with lock:
                    take(cs)
            th.join()
        st = srv.stats()
        srv.close()
        lat = np.array([got[k]["t_done"] - got[k]["t_arrival"] for k in ids])
        n_ev = int(sum(ev[i] for i in idx))
        span = max(c["t_done"] for c in got.values()) - t_first
        ev_lat = np.repeat(lat, [ev[ids[k]] for k in ids])
        res = dict(requests=len(idx), events=n_ev, events_per_s=n_ev / span,
                   p50_ms=1e3 * float(np.percentile(lat, 50)), p99_ms=1e3 * float(np.percentile(lat, 99)),
                   event_p50_ms=1e3 * float(np.percentile(ev_lat, 50)),
                   event_p99_ms=1e3 * float(np.percentile(ev_lat, 99)),
                   batches=st["batches"], peak_inflight=st["peak_inflight"], hbm_peak_mb=st["hbm_peak"] / 2**20,
                   worker_busy=(st["worker_launch_s"] + st["worker_finish_s"]) / max(st["worker_wall_s"], 1e-9),
                   gathered_frac=st["bytes_gathered"] / max(1, st["bytes_gathered"] + st["bytes_copied"]),
                   peak_outstanding=peak[0],
                   status_ok=all(c["status"] == 0 for c in got.values()))
        if arrivals is None:
            res["outstanding"] = window
            res["client_busy"] = client_s / max(span, 1e-9)
        if accuracy:
            tot = np.array(acc).sum(0)
            res.update(efficiency=tot[1] / max(tot[0], 1), true_track_fraction=tot[1] / max(tot[2], 1))
        return res

    batched_cfg = dict(n_slots=4, max_batch_events=1024, max_batch_seeds=1024 * 200, max_batch_hits=1024 * 1500,
                       mlp_precision=ds.DS_MLP_BF16)
    plain_cfg = dict(n_slots=1, max_batch_events=1, max_batch_seeds=4096, max_batch_hits=65535, events_per_launch=1,
                     mlp_precision=ds.DS_MLP_FP32)
    all_idx = np.arange(n_requests)
    # capacity without per-request scoring in the client loop (scoring there
    # took longer per request than the server, so it measured the client);
    # the physics scores come from a second, scored pass over the same requests
    burst = serve(batched_cfg, all_idx)
    scored = serve(batched_cfg, all_idx, accuracy=True)
    burst.update(efficiency=scored["efficiency"], true_track_fraction=scored["true_track_fraction"],
                 scored_pass_events_per_s=scored["events_per_s"], scored_pass_client_busy=scored["client_busy"])
    cap = burst["events_per_s"]
    mean_ev = float(ev.mean())
    loads = {}
    for f in (0.15, 0.3, 0.6, 0.9):
        rate = f * cap / mean_ev
        loads[f"{f:.1f}"] = dict(offered_events_per_s=f * cap, **serve(batched_cfg, all_idx, gaps / rate))
    n_plain = 24
    p_idx = all_idx[:n_plain]
    plain_burst = serve(plain_cfg, p_idx, window=4, accuracy=True)
    pcap = plain_burst["events_per_s"]
    mean_p = float(ev[p_idx].mean())
    plain_loaded = dict(offered_events_per_s=0.6 * pcap,
                        **serve(plain_cfg, p_idx, gaps[:n_plain] / (0.6 * pcap / mean_p)))
    batched_same = dict(offered_events_per_s=0.6 * pcap,
                        **serve(batched_cfg, p_idx, gaps[:n_plain] / (0.6 * pcap / mean_p)))
    return dict(workload="C5: Poisson arrivals, requests of 1-500 events of config-1 occupancy "
                         "(200 seeds, ~1500 UT hits per event), pinned host inputs",
                input_bytes_per_event=float(sum(24 * int(r["seed_off"][-1]) + 13 * int(r["hit_off"][-1])
                                                for r in reqs) / ev.sum()),
                batched=dict(form="continuous batching, 4 slots, batches <= 1024 events, BF16 tensor-core ghost killer, "
                                  "request arrays below 1 MiB read from pinned host memory by the gather kernel, "
                                  "larger ones by cudaMemcpyAsync",
                             capacity=burst, loads=loads, at_plain_load=batched_same),
                plain=dict(form="one request at a time, one event per launch, FP32",
                           capacity=plain_burst, load_0_6=plain_loaded),
                note="latency = results on the host minus the request's arrival; capacity from a closed loop "
                     "with a fixed number of requests outstanding; loads (open loop, Poisson) as fractions of it")


def e2e_pipelined(ds, torch, cfg, w, pin, E, S, H, dev_index, n_steps=10, slots=3):
    """End to end through the serving API: each step is one request carrying
    the whole batch from pinned host memory, results copied back into pinned
    host buffers; `slots` requests are outstanding, so one step's upload
    overlaps another's compute and download (a closed loop)."""
    srv = ds.Server(cfg, w, device=dev_index, n_slots=slots, max_batch_events=E, max_batch_seeds=S,
                    max_batch_hits=H, vertices_per_seed=2)
    outs = [srv.alloc_outputs(pin, vtx_capacity=2 * S + 4096) for _ in range(slots)]
    free = list(range(slots))
    held = {}

    def submit():
        k = free.pop()
        o = dict(outs[k])
        held[srv.submit(pin, out=o)] = k

    for _ in range(slots):                   # warm-up round
        submit()
    got = 0
    while got < slots:
        for c in srv.poll(timeout=1.0):
            free.append(held.pop(c["id"]))
            got += 1
    t0 = time.perf_counter()
    for _ in range(slots):
        submit()
    sent, done, last = slots, 0, None
    while done < n_steps:
        for c in srv.poll(timeout=1.0):
            free.append(held.pop(c["id"]))
            done += 1
            last = c
            assert c["status"] == 0, c
            if sent < n_steps:
                submit()
                sent += 1
    el = time.perf_counter() - t0
    srv.close()
    return dict(value=n_steps * E / el, unit="events/s", ms_per_step=1e3 * el / n_steps,
                h2d_bytes_per_step=24 * S + 13 * H + 8 * (E + 1),
                d2h_bytes_per_step=64 * last["n_tracks"] + 32 * last["n_vertices"] + 8 * (E + 1),
                steps=n_steps, outstanding=slots,
                note="serving API (ds_server_*): one request per step with the whole batch, pinned host "
                     "buffers, uploads, compute and downloads of consecutive steps overlapped")


def vertex_physics_leg(d, ds, torch, synth, dv, out, vout, stream, n_v, reps=10):
    """ds_vertex_physics on one step's vertices (four fixed-seed line networks,
    FP32 on the CUDA cores and BF16 on the tensor cores): kernel time,
    vertices/s and the algorithmic bytes rate (vertex record + two track
    records read, one 64-byte record written)."""
    ds.ds_load_line_weights(d.ctx, synth.line_weights())
    d.reconstruct(dv, out, stream)
    d.vertex(out, vout, stream)
    info = torch.zeros((max(n_v, 1), 64), dtype=torch.uint8, device="cuda")
    res = dict(vertices=int(n_v), lines=4,
               note="per vertex: daughter momenta at the vertex, three mass hypotheses, parent P, P_T, impact "
                    "parameter, 16 inputs, four 16-32-1 line networks")
    for name, prec in (("fp32", ds.DS_MLP_FP32), ("bf16_tensor_cores", ds.DS_MLP_BF16)):
        d.set_params(mlp_precision=prec)
        for _ in range(3):
            ds.ds_vertex_physics(d.ctx, out, vout, info, stream)
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            ds.ds_vertex_physics(d.ctx, out, vout, info, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        us = e0.elapsed_time(e1) * 1e3 / reps
        d.sync(stream)
        res[name] = dict(us=us, vertices_per_s=n_v / (us * 1e-6), gbs=224.0 * n_v / (us * 1e-6) / 1e9)
    d.set_params(mlp_precision=ds.DS_MLP_FP32)
    rec = info.cpu().numpy().view(ds.VINFO_DTYPE).reshape(-1)[:n_v]
    res["k0s_window_fraction"] = float((np.abs(rec["m_pipi"] - 497.611) < 20.0).mean()) if n_v else 0.0
    return res


def dv1_leg(ds, torch, cfg, w, batch, dv, dev_index, reps=10):
    """The paper's two variants on the step's batch: Dv0 (momentum window in
    UTbX) and Dv1 (triplet search in UTaX x UTbX), with Dv0's origin-pointing
    window (the paper's first version) beside them; device time of
    ds_reconstruct + ds_vertex and the chi2-pick selection against truth."""
    res = {}
    for name, over in (("dv0_kick", dict(variant=0)), ("dv0_origin", dict(variant=0, first_window_origin=1)),
                       ("dv1", dict(variant=1))):
        c = dict(cfg, pick_chi2=1, nn_threshold=2.0, **over)
        d = ds.Downstream(c, w, device=dev_index)
        g = d.run(batch, dev=dv)
        out = d.alloc_tracks(dv["n_events"], dv["n_seeds"])
        vout = d.alloc_vertices(dv["n_events"], 2 * int(g["n_vertices"]) + 4096)
        st = torch.cuda.current_stream()
        for _ in range(3):
            d.reconstruct(dv, out, st); d.vertex(out, vout, st)
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(reps):
            d.reconstruct(dv, out, st); d.vertex(out, vout, st)
        e1.record(st)
        torch.cuda.synchronize()
        d.sync(st)
        ms = e0.elapsed_time(e1) / reps
        res[name] = dict(ms_per_step=ms, events_per_s=dv["n_events"] / (ms * 1e-3), **selection(batch, g))
        d.close()
    res["note"] = ("chi2 pick (the paper's distance score) so that the variants are compared without a trained "
                   "network; eager launches")
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--plain-events", type=int, default=200)
    ap.add_argument("--clocks-log", default=None)
    ap.add_argument("--ncu", action="store_true",
                    help="profiling run: warmup + steps eager steps on one batch, nothing else")
    ap.add_argument("--events", type=int, default=N_EVENTS)
    ap.add_argument("--no-c3", action="store_true", help="skip the config-3 (log-normal, 10000 events) leg")
    ap.add_argument("--no-c5", action="store_true", help="skip the config-5 (serving loop) leg")
    ap.add_argument("--mlp-precision", default="fp32", choices=["fp32", "bf16", "fp8"],
                    help="network arithmetic (ghost killer and trigger lines) in the --ncu profiling run")
    ap.add_argument("--physics", action="store_true", help="--ncu run: add ds_vertex_physics to every step")
    ap.add_argument("--variant", type=int, default=0, choices=[0, 1], help="--ncu run: 1 = Dv1 triplet search")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return bench_reference(args)

    import torch
    from paper_2503_13092_b300 import build, ds, synth
    build.build()
    ws, rank, local = dist_info()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev_index = local if ws > 1 else 0
    torch.cuda.set_device(dev_index)

    batch = synth.config_batch("c2", seed=2 + rank, n_events=args.events)
    cfg = synth.default_config()
    w = synth.nn_weights()
    E, S, H = batch["n_events"], int(batch["seed_off"][-1]), int(batch["hit_off"][-1])
    d = ds.Downstream(cfg, w, device=dev_index)
    ds.ds_reserve(d.ctx, E, S, H)
    if args.ncu:
        d.set_params(mlp_precision={"fp32": ds.DS_MLP_FP32, "bf16": ds.DS_MLP_BF16, "fp8": ds.DS_MLP_FP8}[
            args.mlp_precision])
        if args.variant:
            d.set_params(variant=1)
        dv = d.to_device(batch)
        out = d.alloc_tracks(E, S)
        vout = d.alloc_vertices(E, 16 * S + 4096)
        info = None
        if args.physics:
            ds.ds_load_line_weights(d.ctx, synth.line_weights())
            info = torch.zeros((16 * S + 4096, 64), dtype=torch.uint8, device="cuda")
        for _ in range(args.warmup + args.steps):
            d.reconstruct(dv, out)
            d.vertex(out, vout)
            if info is not None:
                ds.ds_vertex_physics(d.ctx, out, vout, info)
        st = d.sync()
        print(json.dumps(dict(ncu_run=True, steps=args.warmup + args.steps, status=st["status"],
                              tracks=st["n_tracks"], vertices=st["n_vertices"])), flush=True)
        d.close()
        return 0
    R, in_bytes = replicas_for(E, S, H)
    devs = [d.to_device(batch) for _ in range(R)]
    out = d.alloc_tracks(E, S)
    # size the vertex output from one run
    probe = d.run(batch, dev=devs[0])
    n_t, n_v = probe["n_tracks"], probe["n_vertices"]
    vcap = 2 * n_v + 4096
    vout = d.alloc_vertices(E, vcap)
    stream = torch.cuda.current_stream()

    def step(k):
        dv = devs[k % R]
        d.reconstruct(dv, out, stream)
        d.vertex(out, vout, stream)

    for k in range(args.warmup):
        step(k)
    st = d.sync(stream)
    n_cand, n_pairs, n_fp64 = st["n_candidates"] // args.warmup, st["n_pairs"] // args.warmup, \
        st["n_pairs_fp64"] // args.warmup

    # eager timing (Python + ctypes enqueue per step) for reference
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(args.steps):
        step(k)
    e1.record(stream)
    torch.cuda.synchronize()
    eager_s = e0.elapsed_time(e1) / 1e3
    d.sync(stream)

    # one CUDA graph per input replica: a step is one graph launch
    graphs = []
    cap_stream = torch.cuda.Stream()
    for r in range(R):
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=cap_stream):
            cs = torch.cuda.current_stream()
            d.reconstruct(devs[r], out, cs)
            d.vertex(out, vout, cs)
        graphs.append(g)
    for k in range(args.warmup):
        graphs[k % R].replay()
    d.sync(stream)

    def step_graph(k):
        graphs[k % R].replay()

    # one stream, one context: the same steps in sequence
    torch.cuda.synchronize()
    s0e = torch.cuda.Event(enable_timing=True)
    s1e = torch.cuda.Event(enable_timing=True)
    s0e.record(stream)
    for k in range(args.steps):
        step_graph(k)
    s1e.record(stream)
    torch.cuda.synchronize()
    single_s = s0e.elapsed_time(s1e) / 1e3
    st = d.sync(stream)
    assert st["status"] == 0, st

    # STREAMS lanes (context + outputs + stream); lane l replays the graphs of
    # replicas l, l + STREAMS, ...  The lanes' buffers stay referenced here for
    # as long as their graphs exist.
    lanes = [dict(d=d, out=out, vout=vout, stream=torch.cuda.Stream(), graphs={})]
    for _ in range(1, STREAMS):
        dl = ds.Downstream(cfg, w, device=dev_index)
        ds.ds_reserve(dl.ctx, E, S, H)
        dl.run(batch, dev=devs[0])            # sizes its vertex workspace
        lanes.append(dict(d=dl, out=dl.alloc_tracks(E, S), vout=dl.alloc_vertices(E, vcap),
                          stream=torch.cuda.Stream(), graphs={}))
    for r in range(R):
        ln = lanes[r % STREAMS]
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=cap_stream):
            cs = torch.cuda.current_stream()
            ln["d"].reconstruct(devs[r], ln["out"], cs)
            ln["d"].vertex(ln["out"], ln["vout"], cs)
        ln["graphs"][r] = g

    def steps_lanes(k0, n):
        for k in range(k0, k0 + n):
            ln = lanes[k % STREAMS]
            with torch.cuda.stream(ln["stream"]):
                ln["graphs"][k % R].replay()

    torch.cuda.synchronize()
    steps_lanes(0, max(args.warmup, STREAMS))
    torch.cuda.synchronize()

    # ------------------------------------------------------------- timed
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    clk = Clocks(dev_index, args.clocks_log)
    time.sleep(0.3)
    t0e = torch.cuda.Event(enable_timing=True)
    t1e = torch.cuda.Event(enable_timing=True)
    t0e.record(stream)
    for ln in lanes:
        ln["stream"].wait_event(t0e)
    steps_lanes(0, args.steps)
    for ln in lanes:
        ev = torch.cuda.Event()
        ev.record(ln["stream"])
        stream.wait_event(ev)
    t1e.record(stream)
    torch.cuda.synchronize()
    clocks = clk.stop()
    if ws > 1:
        dist.barrier()
    elapsed = t0e.elapsed_time(t1e) / 1e3
    for ln in lanes:
        st = ln["d"].sync(ln["stream"])
        assert st["status"] == 0, st
    for ln in lanes[1:]:                  # graphs first, then the contexts they point into
        ln["graphs"].clear()
        ln["d"].close()
    lanes[0]["graphs"].clear()
    times = [max_over_ranks(elapsed)] * ws
    agg = aggregate(times, E, args.steps)
    single = dict(value=ws * E * args.steps / max_over_ranks(single_s), unit="events/s",
                  ms_per_step=1e3 * max_over_ranks(single_s) / args.steps,
                  note="the same graph steps on one stream and one context, in sequence")

    # ------------------------------------------------- per-kernel roofline
    ds.ds_profile_enable(d.ctx, True)
    n_prof = min(args.steps, 10)
    for k in range(n_prof):
        step(k)
    prof = ds.ds_profile_read(d.ctx)
    ds.ds_profile_enable(d.ctx, False)
    d.sync(stream)
    # per-event table (uint16 entries): offsets padded to 8 entries, then 16 bytes of row flags
    table_stride = (((4 * cfg["n_sectors"] * 64 + 1) + 7) & ~7) + 8
    alg = algorithmic(E, S, H, n_t, n_v, n_cand, n_pairs, table_stride, fused="k_mlp" not in prof)
    kernels = {k: dict(launches=v[0], avg_us=1e3 * v[1] / max(v[0], 1)) for k, v in prof.items()}
    launches_per_step = sum(v["launches"] for v in kernels.values()) / n_prof
    step_us = sum(v["avg_us"] * v["launches"] for v in kernels.values()) / n_prof
    for k, v in kernels.items():
        v["share"] = v["avg_us"] * v["launches"] / n_prof / step_us
        a = alg.get(k, {})
        v["gbs"] = a.get("bytes", 0) / (v["avg_us"] * 1e-6) / 1e9 if v["avg_us"] > 0 else 0.0
        if a.get("flop"):
            v["tflops"] = a["flop"] / (v["avg_us"] * 1e-6) / 1e12
    mb = method_bytes(S, H, n_t, n_v)
    for k, v in kernels.items():
        v["method_gbs"] = mb.get(k, 0) / (v["avg_us"] * 1e-6) / 1e9 if v["avg_us"] > 0 else 0.0
    # the network scored inside the search kernel instead (fuse_network = 1)
    d.set_params(fuse_network=1)
    for k in range(3):
        step(k)
    d.sync(stream)
    ds.ds_profile_enable(d.ctx, True)
    for k in range(n_prof):
        step(k)
    prf = ds.ds_profile_read(d.ctx)
    ds.ds_profile_enable(d.ctx, False)
    d.set_params(fuse_network=0)
    d.sync(stream)
    fused_form = {k: 1e3 * v[1] / max(v[0], 1) for k, v in prf.items()}
    fused_form = dict(kernels_us=fused_form, step_us=sum(1e3 * v[1] for v in prf.values()) / n_prof,
                      separate_step_us=step_us,
                      note="network + pick inside k_search (fuse_network = 1) against the separate k_mlp and "
                           "k_pick (default), CUDA-event time per kernel, same steps")
    dom = max(kernels, key=lambda k: kernels[k]["share"])
    hbm, sm_mhz, src = peaks()
    kd = kernels[dom]
    # achieved: the method's bytes (seeds 24 B + hits 13 B for the search)
    # over the kernel's CUDA-event time; the bytes this design moves through
    # its own workspaces (candidates, staged x0, bin tables) beside it
    roof = dict(kernel=dom, bound="hbm", achieved=kd["method_gbs"], peak=hbm, unit="GB/s",
                frac=kd["method_gbs"] / hbm, avg_us=kd["avg_us"], method_bytes_per_launch=mb.get(dom, 0),
                peak_source=f"{src} (MEASURED_PEAKS.json hbm_gbs)" if src == "measured" else "fallback",
                traffic=traffic_for(dom),
                with_workspace=dict(bytes_per_launch=alg.get(dom, {}).get("bytes", 0), gbs=kd["gbs"],
                                    frac=kd["gbs"] / hbm))
    variants = dv1_leg(ds, torch, cfg, w, batch, devs[0], dev_index)

    # vertex-level physics + trigger-line networks on the step's vertices
    vphys = vertex_physics_leg(d, ds, torch, synth, devs[0], out, vout, stream, n_v)

    # ghost killer trained on separate synthetic events (training mode, BCE +
    # Adam in FP64); the reduced-precision forms are compared with it loaded
    from paper_2503_13092_b300 import train
    t_tr = time.perf_counter()
    tb = synth.config_batch("c2", seed=21, n_events=80)
    x_tr, y_tr, _ = train.training_set(cfg, tb, w, device=dev_index)
    hist = []
    w_tr = train.train(x_tr, y_tr, epochs=12, seed=0, history=hist)
    t_tr = time.perf_counter() - t_tr
    sel_fixed = selection(batch, probe)
    ds.ds_load_nn_weights(d.ctx, w_tr)
    probe_tr = d.run(batch, dev=devs[0])
    mlp_forms = reduced_precision_forms(d, ds, torch, batch, devs, probe_tr, step, n_prof, stream, kernels, n_cand)
    ds.ds_load_nn_weights(d.ctx, w)
    trained = dict(events=80, candidates=int(len(y_tr)), ghost_fraction=float(y_tr.mean()), epochs=12,
                   loss_first=hist[0], loss_last=hist[-1], seconds=t_tr,
                   selection_fixed_seed_fp32=sel_fixed, selection_trained_fp32=selection(batch, probe_tr),
                   note="trained on 80 other C2 events in training mode (100/10 mm windows, no clone "
                        "killing); mlp_forms use these weights; the headline step uses the fixed-seed ones")

    path_bytes = 24 * S + 13 * H + 64 * n_t + 32 * n_v
    path = dict(bytes_per_step=path_bytes, gbs=path_bytes * args.steps / max(times) / 1e9,
                frac_of_hbm=path_bytes * args.steps / max(times) / 1e9 / hbm)
    tr = step_traffic()
    if tr is not None:
        path.update(dram_bytes_per_step=tr, dram_over_method_bytes=tr / path_bytes)

    # ---------------------------------------------------------- end to end
    pin = {}
    for k in ("seed_x", "seed_y", "seed_tx", "seed_ty", "seed_qop", "seed_chi2", "hit_x0", "hit_ybeg", "hit_yend",
              "hit_layer", "seed_off", "hit_off"):
        t = torch.from_numpy(np.ascontiguousarray(batch[k])).pin_memory()
        pin[k] = t.numpy()
    pin["n_events"] = E
    host_out = dict(tracks=torch.zeros((S, 64), dtype=torch.uint8).pin_memory().numpy().view(ds.TRACK_DTYPE).reshape(-1),
                    trk_off=torch.zeros(E + 1, dtype=torch.int32).pin_memory().numpy(),
                    vertices=torch.zeros((vcap, 32), dtype=torch.uint8).pin_memory().numpy().view(ds.VERTEX_DTYPE).reshape(-1),
                    vtx_off=torch.zeros(E + 1, dtype=torch.int32).pin_memory().numpy())
    n_e2e = min(args.steps, 10)
    for _ in range(2):
        ds.ds_process_host(d.ctx, pin, S, vcap, stream, host_out)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(n_e2e):
        h = ds.ds_process_host(d.ctx, pin, S, vcap, stream, host_out)
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / n_e2e
    e2e_single = dict(value=ws * E / e2e_s, unit="events/s", h2d_bytes_per_step=in_bytes,
                      d2h_bytes_per_step=64 * h["n_tracks"] + 32 * h["n_vertices"] + 8 * (E + 1) + 8,
                      ms_per_step=1e3 * e2e_s,
                      note="ds_process_host: one call per step, upload, compute and download in sequence")
    e2e = e2e_pipelined(ds, torch, cfg, w, pin, E, S, H, dev_index, n_steps=max(args.steps, 10))
    e2e["value"] *= ws
    ceil = h2d_ceiling(torch, [pin[k] for k in ("seed_off", "hit_off", "seed_x", "seed_y", "seed_tx", "seed_ty",
                                                "seed_qop", "seed_chi2", "hit_x0", "hit_ybeg", "hit_yend",
                                                "hit_layer")], d2h_bytes=e2e["d2h_bytes_per_step"])
    best = max(ceil["one_stream_gbs"], ceil["two_streams_gbs"])
    e2e["h2d_ceiling_gbs"] = best
    e2e["h2d_ceiling"] = ceil
    # the rate the upload alone allows, and e2e as a fraction of it
    e2e["upload_bound_events_per_s"] = ws * E / (e2e["h2d_bytes_per_step"] / (best * 1e9))
    e2e["frac_of_upload_bound"] = e2e["value"] / e2e["upload_bound_events_per_s"]
    # the rate with each step's upload and download in sequence at their
    # measured rates (no overlap of the two directions)
    t_serial = e2e["h2d_bytes_per_step"] / (best * 1e9) + e2e["d2h_bytes_per_step"] / (ceil["d2h_gbs"] * 1e9)
    e2e["serial_copy_bound_events_per_s"] = ws * E / t_serial
    e2e["frac_of_serial_copy_bound"] = e2e["value"] / e2e["serial_copy_bound_events_per_s"]
    # and with the step's upload and download issued together
    e2e["concurrent_copy_bound_events_per_s"] = ws * E / (ceil["up_and_down_concurrent_ms"] * 1e-3)
    e2e["frac_of_concurrent_copy_bound"] = e2e["value"] / e2e["concurrent_copy_bound_events_per_s"]

    # ------------------------------------------------ plain form (1 event/launch)
    n_plain = min(args.plain_events, E)
    dv = devs[0]
    per_event = []
    for e in range(n_plain):
        s0, s1 = int(batch["seed_off"][e]), int(batch["seed_off"][e + 1])
        h0, h1 = int(batch["hit_off"][e]), int(batch["hit_off"][e + 1])
        pe = dict(n_events=1, n_seeds=s1 - s0, n_hits=h1 - h0,
                  seed_off=torch.tensor([0, s1 - s0], dtype=torch.int32, device="cuda"),
                  hit_off=torch.tensor([0, h1 - h0], dtype=torch.int32, device="cuda"))
        for k in ("seed_x", "seed_y", "seed_tx", "seed_ty", "seed_qop", "seed_chi2"):
            pe[k] = dv[k][s0:s1]
        for k in ("hit_x0", "hit_ybeg", "hit_yend", "hit_layer"):
            pe[k] = dv[k][h0:h1]
        per_event.append(pe)
    pout = d.alloc_tracks(1, 4096)
    pvout = d.alloc_vertices(1, 1 << 16)
    for pe in per_event[:5]:
        d.reconstruct(pe, pout, stream); d.vertex(pout, pvout, stream)
    torch.cuda.synchronize()
    p0 = torch.cuda.Event(enable_timing=True); p1 = torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    for pe in per_event:
        d.reconstruct(pe, pout, stream)
        d.vertex(pout, pvout, stream)
    p1.record(stream)
    torch.cuda.synchronize()
    plain_s = p0.elapsed_time(p1) / 1e3
    d.sync(stream)

    c3 = None
    if not args.no_c3:
        c3 = bench_c3(ds, torch, cfg, w, min(args.steps, 10), args.warmup, dev_index)

    c5 = None
    if not args.no_c5:
        c5 = bench_c5(ds, torch, cfg, w_tr, dev_index)
        cap = c5["batched"]["capacity"]
        cap["upload_bound_events_per_s"] = e2e["h2d_ceiling_gbs"] * 1e9 / c5["input_bytes_per_event"]
        cap["frac_of_upload_bound"] = cap["events_per_s"] / cap["upload_bound_events_per_s"]

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = run_cpu_baseline(batch, cfg, w)

    if rank == 0:
        line = dict(
            metric="events/s per B300 (Downstream+vertexing)", value=agg["value"], unit="events/s", n_gpus=ws,
            steps=args.steps, warmup=args.warmup, ms_per_step=agg["ms_per_step"], higher_is_better=True,
            scaling="weak", vs_baseline=None, dtype="f32", data="synthetic",
            config=workload_config(E, S, H, ws),
            step_stats=dict(tracks=n_t, vertices=n_v, candidates=n_cand, pairs=n_pairs, pairs_fp64=n_fp64,
                            streams=STREAMS),
            single_stream=single,
            roofline=roof, path_roofline=path, kernels=kernels, clocks=clocks, e2e=e2e, e2e_single_call=e2e_single,
            mlp_forms=mlp_forms, network_in_search=fused_form, ghost_killer_training=trained, vertex_physics=vphys, variants=variants,
            c3=c3, c5=c5,
            plain_form=dict(value=n_plain / plain_s, unit="events/s",
                            note="one event per ds_reconstruct + ds_vertex call, FP32", events=n_plain),
            eager=dict(value=ws * E * args.steps / eager_s, unit="events/s",
                       note="same steps launched from Python without CUDA graphs"),
            gpu_launches=int(round(launches_per_step * args.steps)), kernels_per_step=launches_per_step,
            cpu_baseline=cpu)
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    d.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
