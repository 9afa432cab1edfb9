"""Throughput of the Haar-domain phase shift + double product on GB300.

One step = one frame of the RGB 128x256 lat-long lighting workload: 16
fractional translations of the lighting map's Haar coefficients
(haar_shift, coefficient-major output) followed by the top-256 CSR FP32
double product for 50 000 torus vertices (shade_vertices): 800 000
vertex-rotations per step.  Inputs are synthetic (seeded scene: lognormal
lighting with hot spots, torus vertices, occluder spheres) and resident in
HBM before timing; L2 is flushed (256 MiB write) between timed steps.

Prints one JSON line (rank 0).  ``--impl reference`` times the CPU FP64
oracle on a bounded sample of the same frame instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "M vertex-rotations/s and % of HBM/tensor roofline; BF16+surrogate vs FP32 plain"
UNIT = "M vertex-rotations/s"
WORKLOAD = ("RGB 128x256 lat-long lighting (32768 Haar coefficients per channel), 16 fractional "
            "shifts per frame, 50000 torus vertices (8 occluders), top-256 CSR FP32 transport")
FLUSH_BYTES = 256 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample", type=int, default=2000, help="vertices in the oracle's timed sample")
    return ap.parse_args()


# ----------------------------------------------------------------- oracle timing

def oracle_frame_sample(n_vertices: int, seed_stream: int = 0):
    """Time the CPU oracle on one c1 frame: the full 16-shift phase shift and
    the brute-force double product of a sample of vertices.  Returns
    (seconds for the shift, seconds per vertex of shading, vertices)."""
    import numpy as np
    import synth
    from oracle import haar, shade, shift, transport
    sc = synth.scene(1, V=n_vertices)
    H, W = sc["H"], sc["W"]
    w = synth.transport_weights(sc["pos"], sc["nrm"], sc["occ_c"], sc["occ_r"], H, W).numpy()
    T = transport.project(w)
    vals, idx, rowptr = transport.topk_csr(T, 256)
    dense = transport.csr_dense(vals, idx, rowptr, H * W)
    L = haar.forward(sc["light"])
    t0 = time.perf_counter()
    Ls = shift.haar_shift(L, H, W, shift.TRANSLATE, sc["params"])
    t1 = time.perf_counter()
    shade.radiance(Ls, dense, H, W)
    t2 = time.perf_counter()
    return t1 - t0, (t2 - t1) / n_vertices, n_vertices


def cpu_baseline(sample: int):
    t_shift, t_vert, n = oracle_frame_sample(sample)
    V, S = 50000, 16
    frame = t_shift + t_vert * V
    return {"value": V * S / frame / 1e6, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"one frame's 16-shift phase shift (full map) + brute-force pixel-space shading of "
                      f"{n} of the 50000 vertices, scaled to the frame: shift {t_shift:.2f} s, "
                      f"{t_vert * 1e3:.2f} ms per vertex (numpy FP64, single process)"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    per_step_vertices = max(50, args.cpu_sample // 10)
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        t_shift, t_vert, n = oracle_frame_sample(per_step_vertices)
        dt = t_shift + t_vert * 50000
        if i >= args.warmup:
            times.append(dt)
    frame = statistics.mean(times)
    value = 50000 * 16 / frame / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": frame * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"each step: the full 16-shift phase shift + brute-force shading of "
                                       f"{per_step_vertices} vertices, scaled to the 50000-vertex frame"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------- GPU workload

def prepare_c1(hs, dev, rank: int):
    """Device-resident c1 frame: lighting coefficients, shifts, CSR transport."""
    import numpy as np
    import torch
    import synth
    sc = synth.scene(1)
    if rank:
        rg = synth.rng_for(1, 100 + rank)
        sc["pos"], sc["nrm"] = synth.torus_vertices(rg, sc["V"])
    H, W, C, S, V = sc["H"], sc["W"], sc["C"], sc["S"], sc["V"]
    light = torch.tensor(sc["light"], dtype=torch.float32, device=dev)
    L = hs.haar_forward(light).contiguous()                                    # [3, 32768]
    K = 256
    vals = torch.empty((V, K), dtype=torch.float32, device=dev)
    idx = torch.empty((V, K), dtype=torch.int64, device=dev)
    chunk = 4096
    for v0 in range(0, V, chunk):
        v1 = min(V, v0 + chunk)
        w = synth.transport_weights(sc["pos"][v0:v1], sc["nrm"][v0:v1], sc["occ_c"], sc["occ_r"], H, W,
                                    device=dev, dtype=torch.float32).contiguous()
        T = hs.haar_forward(w)
        top = torch.topk(T.abs(), K, dim=1).indices
        top, _ = torch.sort(top, dim=1)
        idx[v0:v1] = top
        vals[v0:v1] = torch.gather(T, 1, top)
        del w, T
    rowptr = (torch.arange(V + 1, device=dev, dtype=torch.int64) * K).to(torch.int32)
    idx16 = idx.to(torch.int32).to(torch.int16).contiguous()
    params = torch.tensor(sc["params"], dtype=torch.float64, device=dev)
    plan = hs.Plan(H, W, C, kind=hs.HAAR_SHIFT_TRANSLATE, max_shifts=S, out_layout=hs.HAAR_LAYOUT_KSC)
    tr = hs.Transport(hs.HAAR_T_CSR_F32_U16, V, 0, vals.reshape(-1).contiguous(), idx16.reshape(-1), rowptr)
    lighting = torch.empty((H * W, S, C), dtype=torch.float32, device=dev)
    radiance = torch.empty((V, S, C), dtype=torch.float32, device=dev)
    torch.cuda.synchronize()
    return dict(sc=sc, H=H, W=W, C=C, S=S, V=V, K=K, L=L, params=params, plan=plan, tr=tr,
                lighting=lighting, radiance=radiance)


def algorithmic_bytes(wl):
    """Bytes a kernel must move at least, per launch."""
    V, K, S, C, N = wl["V"], wl["K"], wl["S"], wl["C"], wl["H"] * wl["W"]
    shade = V * K * 4 + V * K * 2 + (V + 1) * 4 + N * S * C * 4 + V * S * C * 4
    shift = C * N * 4 + S * C * N * 4
    return {"k_shade_csr_f32": shade, "k_shift": shift}


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join(ROOT, "gpurun_out", f"clocks_rank{index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(self.index), "-lms", "200"], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def traffic_record(kernel: str):
    """DRAM bytes per launch from the committed ncu capture, if the kernel's
    source is unchanged since it was taken."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        rec = json.load(open(path))[kernel]
    except Exception:
        return None
    src = os.path.join(ROOT, "paper_1705_07272_gb300", "csrc", rec["source"])
    try:
        h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    except OSError:
        return None
    if h != rec.get("source_sha256_16"):
        return None
    return rec["dram_bytes_per_launch"]


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args.cpu_sample)

    import torch
    import paper_1705_07272_gb300 as hs
    from paper_1705_07272_gb300 import build as _build
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    _build.build()
    hs.lib()

    wl = prepare_c1(hs, dev, rank)
    plan, tr = wl["plan"], wl["tr"]
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def step():
        hs.haar_shift(plan, wl["L"], wl["params"], wl["lighting"])
        hs.shade_vertices(plan, tr, wl["lighting"], wl["S"], wl["radiance"])

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()

    def timed(fn, k):
        evs = []
        for _ in range(k):
            flush.fill_(1.0)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            evs.append((a, b))
        torch.cuda.synchronize()
        return [a.elapsed_time(b) for a, b in evs]

    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    step_ms = timed(step, args.steps)
    clk = clocks.stop()
    total_ms = sum(step_ms)
    if world > 1:
        t = torch.tensor([total_ms], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(t.item())
    ms_per_step = total_ms / args.steps
    units = wl["V"] * wl["S"] * world
    value = units / (ms_per_step * 1e-3) / 1e6

    # per-kernel durations for the roofline (same stream, same flush discipline)
    shade_ms = timed(lambda: hs.shade_vertices(plan, tr, wl["lighting"], wl["S"], wl["radiance"]), args.steps)
    shift_ms = timed(lambda: hs.haar_shift(plan, wl["L"], wl["params"], wl["lighting"]), args.steps)
    shade_avg, shift_avg = statistics.mean(shade_ms), statistics.mean(shift_ms)
    ab = algorithmic_bytes(wl)
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    hbm = peaks.get("hbm_gbs", 6800.0)
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
    if shade_avg >= shift_avg:
        kname, kms = "k_shade_csr_f32", shade_avg
    else:
        kname, kms = "k_shift", shift_avg
    achieved = ab[kname] / (kms * 1e-3) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                "traffic": traffic_record(kname), "kernel": kname, "peak_source": peak_src,
                "algorithmic_bytes": ab[kname], "kernel_ms": kms,
                "other_kernels_ms": {"k_setup+k_shift": shift_avg} if kname != "k_shift" else
                {"k_shade_csr_f32": shade_avg}}

    # end to end through the public API with host buffers
    L_host = wl["L"].cpu().pin_memory()
    p_host = wl["params"].cpu().pin_memory()
    R_host = torch.empty(wl["radiance"].shape, dtype=torch.float32).pin_memory()
    L_dev = torch.empty_like(wl["L"])
    p_dev = torch.empty_like(wl["params"])

    def e2e_step():
        L_dev.copy_(L_host, non_blocking=True)
        p_dev.copy_(p_host, non_blocking=True)
        hs.shade_batch(plan, L_dev, p_dev, tr, wl["radiance"])
        R_host.copy_(wl["radiance"], non_blocking=True)

    for _ in range(3):
        e2e_step()
    e2e_ms = timed(e2e_step, args.steps)
    e2e_tot = sum(e2e_ms)
    if world > 1:
        t = torch.tensor([e2e_tot], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        e2e_tot = float(t.item())
    e2e_value = units / (e2e_tot / args.steps * 1e-3) / 1e6
    h2d = L_host.numel() * 4 + p_host.numel() * 8
    d2h = R_host.numel() * 4

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": WORKLOAD, "H": wl["H"], "W": wl["W"], "channels": wl["C"],
                           "shifts_per_step": wl["S"], "vertices_per_gpu": wl["V"], "topk": wl["K"],
                           "l2": "flushed between timed steps (256 MiB write)",
                           "parallelism": f"{world} independent vertex shards (no collective)"},
                "roofline": roofline, "cpu_baseline": cpu,
                "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
                "gpu_launches": 3 * args.steps, "clocks": clk}
        print(json.dumps(line), flush=True)
    plan.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
