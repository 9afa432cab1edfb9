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
            "shifts per frame, 50000 torus vertices (8 occluders), top-256 CSR FP32 transport "
            "(repacked as 4-vertex group CSR)")
FLUSH_BYTES = 256 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-rows", action="store_true", help="skip the per-row measurements of the other configs")
    ap.add_argument("--only", default=None,
                    help="comma-separated rows to run alone (no c1 frame), for profiling one kernel")
    ap.add_argument("--batch-shifts", type=int, default=4096,
                    help="shifts of the translation_shift_batch row (a smaller batch for profiling)")
    ap.add_argument("--cpu-sample", type=int, default=128,
                    help="vertices per host process in the oracle's timed frame sample")
    return ap.parse_args()


# ----------------------------------------------------------------- oracle timing

def _oracle_worker(conn, cid, verts, shm_name, shape):
    """One host process of the oracle's timed frame.  Before timing it builds
    the stored top-256 transport of its vertices (oracle projection); then, on
    command, it computes oracle shifts into the shared lighting buffer or
    shades its vertices from that buffer (brute force through pixel space)."""
    os.environ["OPENBLAS_NUM_THREADS"] = "1"
    os.environ["OMP_NUM_THREADS"] = "1"
    import numpy as np
    import torch
    from multiprocessing import shared_memory
    torch.set_num_threads(1)
    import synth
    from oracle import haar, shade, shift, transport
    sc = synth.scene(cid)
    H, W = sc["H"], sc["W"]
    L = haar.forward(sc["light"])
    T = None
    if len(verts):
        w = synth.transport_weights(sc["pos"][verts], sc["nrm"][verts], sc["occ_c"], sc["occ_r"], H, W).numpy()
        vals, idx, rowptr = transport.topk_csr(transport.project(w), 256)
        T = transport.csr_dense(vals, idx, rowptr, H * W)
        del w
    shm = shared_memory.SharedMemory(name=shm_name)
    Ls = np.ndarray(shape, dtype=np.float64, buffer=shm.buf)
    conn.send("ready")
    while True:
        msg = conn.recv()
        if msg[0] == "shift":
            for s in msg[1]:
                Ls[s] = shift.haar_shift(L, H, W, shift.TRANSLATE, sc["params"][s:s + 1])[0]
            conn.send("done")
        elif msg[0] == "shade":
            r = shade.radiance(Ls, T, H, W) if T is not None else np.zeros((0, shape[0], shape[1]))
            conn.send(r.shape[0])
        else:
            break
    del Ls
    shm.close()


class OracleFrame:
    """The CPU FP64 oracle (unmodified) on a bounded sample of the headline
    frame, spread over `procs` host processes: a step is the frame's 16-shift
    phase shift of the full RGB 128x256 map (shifts divided among the
    processes) followed by the brute-force shading of `n` of its vertices
    (evenly spaced over the 50 000; divided among the processes).  Each
    process is single-threaded; the pool is started with `spawn`."""

    def __init__(self, procs: int, n: int):
        import multiprocessing as mp
        import numpy as np
        from multiprocessing import shared_memory
        import synth
        self.procs, self.n = procs, n
        wl = synth.WORKLOADS[1]
        self.S = wl.S
        shape = (wl.S, wl.C, wl.H * wl.W)
        self.shm = shared_memory.SharedMemory(create=True, size=int(np.prod(shape)) * 8)
        verts = np.linspace(0, wl.V - 1, n).astype(np.int64)
        ctx = mp.get_context("spawn")
        self.conns, self.workers = [], []
        for k, part in enumerate(np.array_split(verts, procs)):
            a, b = ctx.Pipe()
            pr = ctx.Process(target=_oracle_worker, args=(b, 1, part, self.shm.name, shape), daemon=True)
            pr.start()
            self.conns.append(a)
            self.workers.append(pr)
        for c in self.conns:
            assert c.recv() == "ready"

    def step(self) -> float:
        """Seconds of one frame sample (wall clock)."""
        t0 = time.perf_counter()
        for k, c in enumerate(self.conns):
            c.send(("shift", list(range(k, self.S, self.procs))))
        for c in self.conns:
            c.recv()
        for c in self.conns:
            c.send(("shade",))
        done = sum(c.recv() for c in self.conns)
        assert done == self.n
        return time.perf_counter() - t0

    def close(self):
        for c in self.conns:
            c.send(("stop",))
        for w in self.workers:
            w.join(timeout=30)
        self.shm.close()
        self.shm.unlink()

    def sample_text(self) -> str:
        return (f"each step: the frame's 16-shift phase shift of the full RGB 128x256 map and the brute-force "
                f"pixel-space shading of {self.n} of its 50000 vertices (evenly spaced), numpy FP64 oracle in "
                f"{self.procs} single-threaded host processes; value = {self.n} x 16 vertex-rotations / measured "
                f"step time")


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_baseline(per_proc: int):
    """The oracle on all host cores (2 timed steps after one warm-up) and in
    one process, each on a bounded sample of the frame."""
    P = host_cores()
    fr = OracleFrame(P, P * per_proc)
    fr.step()
    t = statistics.mean(fr.step() for _ in range(2))
    out = {"value": fr.n * 16 / t / 1e6, "unit": UNIT, "cores": P, "kind": "oracle", "step_s": t,
           "sample": fr.sample_text()}
    fr.close()
    one = OracleFrame(1, per_proc)
    t1 = one.step()
    out["single_thread"] = {"value": one.n * 16 / t1 / 1e6, "unit": UNIT, "cores": 1, "step_s": t1,
                            "sample": one.sample_text()}
    one.close()
    return out


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    P = host_cores()
    fr = OracleFrame(P, P * args.cpu_sample)
    times = []
    for i in range(args.warmup + args.steps):
        dt = fr.step()
        if i >= args.warmup:
            times.append(dt)
    fr.close()
    step_s = statistics.mean(times)
    value = fr.n * 16 / step_s / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_s * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": bench_config(),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": P, "kind": "oracle",
                             "sample": fr.sample_text()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def bench_config(world: int = 1):
    return {"workload": WORKLOAD, "H": 128, "W": 256, "channels": 3, "shifts_per_step": 16,
            "vertices_per_gpu": 50000, "topk": 256, "l2": "flushed between timed steps (256 MiB write)",
            "parallelism": f"{world} independent vertex shards (no collective)"}


# ----------------------------------------------------------------- oracle checks

CHECK_VERTS = {"c1": 48, "c2": 64, "c3": 24}


def oracle_checks():
    """Sampled FP64-oracle results for the bench rows, computed on the host
    (the CPU-baseline leg) before any GPU work.  Every input is built by the
    oracle from the seeded scenes (lighting coefficients, stored transports,
    view bins); the GPU side re-runs each row's launches on these inputs and
    states the relative L2 error of the sampled outputs."""
    import numpy as np
    import synth
    from oracle import haar, shade, shift, transport
    f32 = lambda x: np.asarray(x, dtype=np.float32).astype(np.float64)
    out = {}

    def weights(sc, vs, Ht, Wt, **kw):
        return synth.transport_weights(sc["pos"][vs], sc["nrm"][vs], sc["occ_c"], sc["occ_r"], Ht, Wt,
                                       **kw).numpy()

    # c0: the whole frame (1 shift of the 32x32 map, 1000 vertices, dense FP32)
    sc = synth.scene(0)
    L = f32(haar.forward(sc["light"]))
    T = f32(transport.project(weights(sc, slice(None), 32, 32)))
    ref = shade.radiance(shift.haar_shift(L, 32, 32, shift.TRANSLATE, sc["params"]), T, 32, 32)
    out["c0"] = dict(L=L, T=T, params=sc["params"], ref=ref)
    # c1: the frame's 16 shifts; shading of evenly spaced vertices (top-256 FP32 CSR)
    sc = synth.scene(1)
    H, W, N = sc["H"], sc["W"], sc["H"] * sc["W"]
    L1 = f32(haar.forward(sc["light"]))
    vs = np.linspace(0, sc["V"] - 1, CHECK_VERTS["c1"]).astype(np.int64)
    vals, idx, rowptr = transport.topk_csr(transport.project(weights(sc, vs, H, W)), 256)
    vals = f32(vals)
    Ls = shift.haar_shift(L1, H, W, shift.TRANSLATE, sc["params"])
    out["c1"] = dict(L=L1, vals=vals, idx=idx, rowptr=rowptr, params=sc["params"], lighting=Ls,
                     ref=shade.radiance(Ls, transport.csr_dense(vals, idx, rowptr, N), H, W))
    # translation batch: sampled shifts of the 4096
    prm = synth.translations(synth.rng_for(1, 7), 4096, 256.0, 256.0)
    smp = [0, 2048, 4095]
    out["translation_shift_batch"] = dict(L=L1, params=prm, sample=smp,
                                          ref=shift.haar_shift(L1, H, W, shift.TRANSLATE, prm[smp]))
    # rotation batch: sampled rotations of the 512
    sc2 = synth.scene(2)
    L2 = f32(haar.forward(sc2["light"]))
    eul = synth.euler_angles(synth.rng_for(2, 7), 512)
    smp = [0, 511]
    out["rotation_shift_batch"] = dict(L=L2, params=eul, sample=smp,
                                       ref=shift.haar_shift(L2, 256, 512, shift.ROTATE_EULER, eul[smp]))
    # c2: the 64 rotations (bf16 hi + lo of the lowest 4096), sampled vertices and rotations;
    # stored transport = the lowest 4096 coefficients in bf16
    vs = np.linspace(0, sc2["V"] - 1, CHECK_VERTS["c2"]).astype(np.int64)
    Tb = transport.to_bf16(transport.project(weights(sc2, vs, 64, 128), 256, 512)[:, :4096])
    smp = [0, 21, 42, 63]
    Ls = shift.haar_shift(L2, 256, 512, shift.ROTATE_EULER, sc2["params"][smp], out_coeffs=4096)
    out["c2_dense_tc"] = dict(L=L2, T=Tb, params=sc2["params"], sample=smp,
                              ref=shade.radiance(Ls, Tb, 256, 512))
    # c3: view bins of sampled vertices for the 32 cameras, 16 bins x top-512 FP16 glossy transport,
    # sampled (rotation, view) pairs
    sc3 = synth.scene(3)
    L3 = f32(haar.forward(sc3["light"]))
    nv = CHECK_VERTS["c3"]
    vs = np.linspace(0, sc3["V"] - 1, nv).astype(np.int64)
    dirs = synth.view_bin_dirs(16)
    view = synth.bin_view_world(sc3["nrm"][vs], 16).reshape(-1, 3)
    rep = np.repeat(vs, 16)
    w = synth.transport_weights(sc3["pos"][rep], sc3["nrm"][rep], sc3["occ_c"], sc3["occ_r"], 64, 128,
                                view=view, expo=sc3["expo"][rep]).numpy()
    vals, idx, _ = transport.topk_csr(transport.project(w, 256, 512)[:, :8192], 512)
    vals = transport.to_f16(vals).reshape(nv, 16, 512)
    idx = idx.reshape(nv, 16, 512)
    pos, nrm, cams = f32(sc3["pos"][vs]), f32(sc3["nrm"][vs]), f32(sc3["cams"])
    bins, margin = transport.view_bins(pos, nrm, cams, f32(dirs))
    smp = [0, 11, 22, 31]
    Ls = shift.haar_shift(L3, 256, 512, shift.ROTATE_EULER, sc3["params"][smp])
    ref = np.zeros((nv, len(smp), 3))
    for k, s in enumerate(smp):
        for v in range(nv):
            Tv = np.zeros((1, 256 * 512))
            Tv[0, idx[v, bins[s, v]]] = vals[v, bins[s, v]]
            ref[v, k] = shade.radiance(Ls[k:k + 1], Tv, 256, 512)[0, 0]
    out["c3_bincsr"] = dict(L=L3, vals=vals, idx=idx, pos=pos, nrm=nrm, cams=cams, dirs=dirs, bins=bins,
                            margin=margin, params=sc3["params"], sample=smp, ref=ref)
    return out


def _rel(a, b):
    import numpy as np
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def gpu_checks(hs, dev, chk):
    """The rows' launches on the oracle's inputs; relative L2 error of the
    sampled outputs against the oracle (max over the sampled shifts or
    rotations where there are several)."""
    import numpy as np
    import torch
    t = lambda x, dt=torch.float32: torch.tensor(np.ascontiguousarray(x), dtype=dt, device=dev)
    res = {}
    c = chk["c0"]
    plan = hs.Plan(32, 32, 1, max_shifts=1)
    tr = hs.Transport(hs.HAAR_T_DENSE_F32, c["T"].shape[0], c["T"].shape[1], t(c["T"]))
    R = hs.shade_batch(plan, t(c["L"]), t(c["params"], torch.float64), tr).cpu().numpy()
    res["c0"] = {"rel_l2_vs_oracle": _rel(R, c["ref"]), "checked": "the whole frame (1000 vertices)"}
    plan.close()

    c = chk["c1"]
    plan = hs.Plan(128, 256, 3, max_shifts=16, out_layout=hs.HAAR_LAYOUT_KSC)
    lit = hs.haar_shift(plan, t(c["L"]), t(c["params"], torch.float64))
    V = len(c["rowptr"]) - 1
    g = hs.haar_transport_group(V, 128 * 256, t(c["rowptr"], torch.int32), t(c["idx"].astype(np.int16), torch.int16),
                                t(c["vals"]))
    R = hs.shade_vertices(plan, g, lit, 16).cpu().numpy()
    lk = lit.double().cpu().numpy().transpose(1, 2, 0)                     # KSC -> [S][C][K]
    res["c1"] = {"rel_l2_vs_oracle": _rel(R, c["ref"]), "shift_rel_l2_vs_oracle": _rel(lk, c["lighting"]),
                 "checked": f"the frame's 16 shifts (all coefficients) and the shading of {V} of the 50000 vertices"}
    plan.close()

    for name, H, W, kind in (("translation_shift_batch", 128, 256, hs.HAAR_SHIFT_TRANSLATE),
                             ("rotation_shift_batch", 256, 512, hs.HAAR_SHIFT_ROTATE_EULER)):
        c = chk[name]
        S = len(c["params"])
        plan = hs.Plan(H, W, 3, kind=kind, max_shifts=S)
        o = hs.haar_shift(plan, t(c["L"]), t(c["params"], torch.float64))
        got = o[torch.tensor(c["sample"], device=dev)].double().cpu().numpy()
        res[name] = {"rel_l2_vs_oracle": max(_rel(got[k], c["ref"][k]) for k in range(len(c["sample"]))),
                     "checked": f"shifts {c['sample']} of the {S}-shift launch"}
        plan.close()
        del o

    c = chk["c2_dense_tc"]
    plan = hs.Plan(256, 512, 3, kind=hs.HAAR_SHIFT_ROTATE_EULER, max_shifts=64, out_coeffs=4096,
                   out_type=hs.HAAR_OUT_BF16_HILO)
    lit = hs.haar_shift(plan, t(c["L"]), t(c["params"], torch.float64))
    V = c["T"].shape[0]
    tr = hs.Transport(hs.HAAR_T_DENSE_BF16, V, 4096, t(c["T"], torch.bfloat16))
    R = hs.shade_vertices(plan, tr, lit, 64)[:, c["sample"]].cpu().numpy()
    res["c2_dense_tc"] = {"rel_l2_vs_oracle": max(_rel(R[:, k], c["ref"][:, k]) for k in range(len(c["sample"]))),
                          "checked": f"rotations {c['sample']} of the 64 (bf16 hi + lo lighting) for {V} of the "
                                     f"200000 vertices; error of the hi/lo lighting and the tensor-core "
                                     f"accumulation against the FP64 double product of the stored bf16 transport"}
    plan.close()

    c = chk["c3_bincsr"]
    plan = hs.Plan(256, 512, 3, kind=hs.HAAR_SHIFT_ROTATE_EULER, max_shifts=32, out_layout=hs.HAAR_LAYOUT_SKC4)
    lit = hs.haar_shift(plan, t(c["L"]), t(c["params"], torch.float64))
    bins = hs.haar_view_bins(t(c["pos"]), t(c["nrm"]), t(c["cams"]), t(c["dirs"]))
    b = bins.cpu().numpy().astype(np.int64)
    ok = c["margin"] > 1e-5
    V = c["vals"].shape[0]
    tr = hs.Transport(hs.HAAR_T_BINCSR_F16_U32, V, 512, t(c["vals"], torch.float16),
                      t(c["idx"].astype(np.int32), torch.int32), bins=16, bin_of=bins)
    R = hs.shade_vertices(plan, tr, lit, 32)[:, c["sample"]].cpu().numpy()
    okp = ok[c["sample"]].T
    res["c3_bincsr"] = {"rel_l2_vs_oracle": max(_rel(R[:, k][okp[:, k]], c["ref"][:, k][okp[:, k]])
                                                for k in range(len(c["sample"]))),
                        "view_bins_equal": bool(np.array_equal(b[ok], c["bins"][ok])),
                        "checked": f"pairs {c['sample']} of the 32 for {V} of the 100000 vertices (view bins away "
                                   f"from near-ties); FP16 transport summed in FP32"}
    plan.close()
    return res


# ----------------------------------------------------------------- GPU workload

def shard_vertices(cid: int, rank: int, V: int):
    """Vertex shard of a rank: rank 0 uses the workload's own vertices, rank r
    an independent draw of the same surface (weak scaling, no overlap)."""
    import synth
    sc = synth.scene(cid, V=V)
    if rank == 0:
        return sc["pos"], sc["nrm"]
    rg = synth.rng_for(cid, 100 + rank)
    if synth.WORKLOADS[cid].surface == "sphere":
        return synth.sphere_vertices(rg, V)
    return synth.torus_vertices(rg, V)


def max_over_ranks(x: float, dev) -> float:
    """The largest value over all ranks (the slowest rank's time)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(units_per_rank: int, ms: float, world: int) -> float:
    """Units of all ranks per second, in millions."""
    return units_per_rank * world / (ms * 1e-3) / 1e6


def prepare_c1(hs, dev, rank: int):
    """Device-resident c1 frame: lighting coefficients, shifts, CSR transport."""
    import numpy as np
    import torch
    import synth
    sc = synth.scene(1)
    sc["pos"], sc["nrm"] = shard_vertices(1, rank, sc["V"])
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
                                    device=dev, dtype=torch.float32, chunk=2048).contiguous()
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
    csr = hs.Transport(hs.HAAR_T_CSR_F32_U16, V, 0, vals.reshape(-1).contiguous(), idx16.reshape(-1), rowptr)
    tr = hs.haar_transport_group(V, H * W, rowptr, idx16.reshape(-1), vals.reshape(-1).contiguous())
    del vals, idx
    lighting = torch.empty((H * W, S, C), dtype=torch.float32, device=dev)
    radiance = torch.empty((V, S, C), dtype=torch.float32, device=dev)
    torch.cuda.synchronize()
    return dict(sc=sc, H=H, W=W, C=C, S=S, V=V, K=K, L=L, params=params, plan=plan, tr=tr, csr=csr,
                union=int(tr.rowptr[-1].item()), lighting=lighting, radiance=radiance)


def algorithmic_bytes(wl):
    """Bytes a kernel must move at least, per launch: its stored input read
    once, the lighting read once, its output written once."""
    V, K, S, C, N = wl["V"], wl["K"], wl["S"], wl["C"], wl["H"] * wl["W"]
    import paper_1705_07272_gb300 as hs
    U, G = wl["union"], (wl["V"] + hs.GROUP - 1) // hs.GROUP
    gcsr = U * (4 * hs.GROUP + 2) + (G + 1) * 4 + N * S * C * 4 + V * S * C * 4
    csr = V * K * 4 + V * K * 2 + (V + 1) * 4 + N * S * C * 4 + V * S * C * 4
    shift = C * N * 4 + S * C * N * 4
    return {"k_shade_gcsr48": gcsr, "k_shade_csr_f32": csr, "k_shift": shift}


# ----------------------------------------------------------------- other §8 rows

def _timeit(fn, reps, flush, stream):
    import torch
    for _ in range(2):
        fn()
    torch.cuda.synchronize()
    evs = []
    for _ in range(reps):
        flush.fill_(1.0)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        evs.append((a, b))
    torch.cuda.synchronize()
    return statistics.median([a.elapsed_time(b) for a, b in evs])


def _bf16_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    d = json.load(open(p)) if os.path.exists(p) else {}
    return d.get("bf16_tflops", 1900.0), d.get("hbm_gbs", 6800.0)


def _glossy_transport(hs, sc, dev, bins=16, K=512, chunk=8192, expo=None, by_magnitude=False):
    """View-binned top-K glossy transport of every (vertex, bin) on the GPU:
    Phong transfer on the 64x128 grid, projected by haar_forward (the lowest
    8192 coefficients of the 256x512 map), top-K per row, sorted by index (or
    by decreasing magnitude); `expo` overrides every vertex's Phong exponent."""
    import numpy as np
    import torch
    import synth
    V = sc["V"]
    view = synth.bin_view_world(sc["nrm"], bins).reshape(-1, 3)
    rows = V * bins
    vals = torch.empty((rows, K), dtype=torch.float16, device=dev)
    idx = torch.empty((rows, K), dtype=torch.int32, device=dev)
    absum = torch.zeros(8192, dtype=torch.float64, device=dev)
    for a in range(0, rows, chunk):
        b = min(rows, a + chunk)
        vi = np.arange(a, b) // bins
        ex = sc["expo"][vi] if expo is None else np.full(b - a, float(expo))
        w = synth.transport_weights(sc["pos"][vi], sc["nrm"][vi], sc["occ_c"], sc["occ_r"], 64, 128,
                                    view=view[a:b], expo=ex, device=dev, dtype=torch.float32,
                                    chunk=chunk)
        T = hs.haar_forward(w.contiguous(), scale=0.25)
        absum += T.abs().sum(0).double()
        top = torch.topk(T.abs(), K, dim=1, sorted=by_magnitude).indices
        if not by_magnitude:
            top, _ = torch.sort(top, dim=1)
        idx[a:b] = top.to(torch.int32)
        vals[a:b] = torch.gather(T, 1, top).to(torch.float16)
        del w, T
    return vals.reshape(V, bins, K), idx.reshape(V, bins, K), absum


def _init_params(rng):
    """He-initialised weights, zero biases, in the flat order haar_mlp_set_params takes."""
    import numpy as np
    flat = []
    for fi, fo in ((320, 256), (256, 256), (256, 256), (256, 256), (256, 512)):
        flat += [rng.standard_normal(fo * fi) * math.sqrt(2.0 / fi), np.zeros(fo)]
    return np.concatenate(flat)


def _glossy_pairs(rng, sc, n):
    """n random (vertex, camera) pairs of the glossy scene: the surrogate's
    raw inputs [n, 9] (position, normal, view direction) and the transfer
    parameters of each pair."""
    import numpy as np
    import synth
    vid = rng.integers(0, sc["V"], n)
    cams = synth.cameras(rng, n)
    pos, nrm, expo = sc["pos"][vid], sc["nrm"][vid], sc["expo"][vid]
    view = cams - pos
    view /= np.linalg.norm(view, axis=1, keepdims=True)
    raw = np.concatenate([pos, nrm, view], axis=1).astype(np.float32)
    return raw, (pos, nrm, view, expo)


def _glossy_rows(hs, sc, dev, gen, fn, chunk=8192):
    """The lowest 8192 coefficients of every pair's transport (Phong transfer
    on the 64x128 grid, projected by haar_forward; finer levels of the
    256x512 map are zero), handed to fn(a, b, T[b - a, 8192]) chunk by chunk."""
    import torch
    import synth
    pos, nrm, view, expo = gen
    n = len(pos)
    for a in range(0, n, chunk):
        b = min(n, a + chunk)
        w = synth.transport_weights(pos[a:b], nrm[a:b], sc["occ_c"], sc["occ_r"], 64, 128, view=view[a:b],
                                    expo=expo[a:b], device=dev, dtype=torch.float32, chunk=chunk)
        fn(a, b, hs.haar_forward(w.contiguous(), scale=0.25))
        del w


def _surrogate_accuracy(hs, net, sc, dev, lit, bins, vals, idx, isel, mu, sg, absum, n_eval=8192):
    """Radiance of sampled (vertex, pair) of the c4 frame from (a) the trained
    surrogate, (b) the view-binned stored transport of the c3 frame (the plain
    method), (c) the transport at the exact view, untruncated, and (d) that
    transport restricted to the surrogate's index set; relative L2 errors, and
    the index-set truncation error for larger index sets."""
    import numpy as np
    import torch
    V, S = sc["V"], sc["S"]
    rng = np.random.default_rng(43)
    vid = rng.integers(0, V, n_eval)
    sid = rng.integers(0, S, n_eval)
    pos, nrm, expo = sc["pos"][vid], sc["nrm"][vid], sc["expo"][vid]
    view = sc["cams"][sid] - pos
    view /= np.linalg.norm(view, axis=1, keepdims=True)
    raw = torch.tensor(np.concatenate([pos, nrm, view], axis=1), dtype=torch.float32, device=dev)
    Lk = lit.reshape(S, -1, 4)[:, :8192, :3].double()                   # SKC4 -> [S][8192][3]
    s_t = torch.tensor(sid, device=dev)
    v_t = torch.tensor(vid, device=dev)
    Te = torch.empty((n_eval, 8192), dtype=torch.float64, device=dev)

    def put(a, b, T):
        Te[a:b] = T.double()
    _glossy_rows(hs, sc, dev, (pos, nrm, view, expo), put)
    b = bins[s_t, v_t].long()
    sv = vals[v_t, b].double()                                           # [n, 512] stored bin rows
    si = idx[v_t, b].long()
    Tsur = mu[None] + sg * net.forward(raw).double()                     # [n, 512] at isel
    curves = (512, 1024, 2048, 4096, 8192)
    sets = [torch.topk(absum, kk).indices for kk in curves]
    exact = torch.zeros((n_eval, 3), dtype=torch.float64, device=dev)
    plain, sur, trunc = torch.zeros_like(exact), torch.zeros_like(exact), torch.zeros_like(exact)
    tk = [torch.zeros_like(exact) for _ in curves]
    for s in range(S):
        m = s_t == s
        if not bool(m.any()):
            continue
        L = Lk[s]                                                        # [8192, 3]
        exact[m] = Te[m] @ L
        plain[m] = torch.einsum("nj,njc->nc", sv[m], L[si[m]])
        sur[m] = Tsur[m] @ L[isel]
        trunc[m] = Te[m][:, isel] @ L[isel]
        for q, ik in enumerate(sets):
            tk[q][m] = Te[m][:, ik] @ L[ik]
    rel = lambda x, y: float((x - y).norm() / y.norm())
    curve = [{"index_set": kk, "rel_l2_vs_untruncated": rel(t, exact)} for kk, t in zip(curves, tk)]
    return {"samples": f"{n_eval} random (vertex, pair) of the 100000 x 32 frame",
            "rel_l2_vs_plain": rel(sur, plain), "rel_l2_vs_untruncated": rel(sur, exact),
            "plain_vs_untruncated": rel(plain, exact),
            "index_set_floor_vs_untruncated": rel(trunc, exact),
            "index_set_curve": curve}


def measure_rows(hs, dev, flush, only=None, batch_shifts=4096):
    """Per-row measurements of the rest of the hot path; ``only`` restricts
    them to the named rows (for profiling one kernel); ``batch_shifts`` sizes
    the translation batch."""
    import numpy as np
    import torch
    import synth
    stream = torch.cuda.current_stream(dev)
    bf16_peak, hbm = _bf16_peak()
    rows = {}

    def want(name):
        return only is None or name in only

    # c0: one fractional shift of a one-channel 32x32 map + dense FP32 shading of 1000 sphere
    # vertices (1024 coefficients each): a launch-bound frame
    if want("c0"):
        sc0 = synth.scene(0)
        L0 = hs.haar_forward(torch.tensor(sc0["light"], dtype=torch.float32, device=dev))
        w = synth.transport_weights(sc0["pos"], sc0["nrm"], sc0["occ_c"], sc0["occ_r"], 32, 32, device=dev,
                                    dtype=torch.float32).contiguous()
        T0 = hs.haar_forward(w)
        prm0 = torch.tensor(sc0["params"], dtype=torch.float64, device=dev)
        plan = hs.Plan(32, 32, 1, max_shifts=1)
        tr = hs.Transport(hs.HAAR_T_DENSE_F32, 1000, 1024, T0)
        R0 = torch.empty((1000, 1, 1), dtype=torch.float32, device=dev)
        ms = _timeit(lambda: hs.shade_batch(plan, L0, prm0, tr, R0), 20, flush, stream)
        rows["c0"] = {"what": "c0 frame: 1 shift of a 1-channel 32x32 map + dense FP32 shading of 1000 vertices "
                              "(shade_batch: set-up, shift, shade)", "frame_ms": ms,
                      "value": 1000 / ms / 1e3, "unit": UNIT, "bound": "launch latency (4 KB map, 4 MB transport)"}
        plan.close()

    # S2 / S4 roofline: 4096 translations of the RGB 128x256 map, full FP32 output (1.6 GB)
    if want("translation_shift_batch"):
        sc1 = synth.scene(1, V=1)
        L1 = hs.haar_forward(torch.tensor(sc1["light"], dtype=torch.float32, device=dev))
        S = batch_shifts
        prm = torch.tensor(synth.translations(synth.rng_for(1, 7), S, 256.0, 256.0), dtype=torch.float64, device=dev)
        plan = hs.Plan(128, 256, 3, max_shifts=S)
        out = torch.empty(plan.out_shape(S), dtype=torch.float32, device=dev)
        ms = _timeit(lambda: hs.haar_shift(plan, L1, prm, out), 5, flush, stream)
        byt = 4 * 3 * 32768 * (S + 1)
        rows["translation_shift_batch"] = {"what": f"haar_shift, {S} fractional shifts of RGB 128x256, FP32 SCK",
                                           "ms": ms, "achieved_gbs": byt / ms / 1e6, "frac_hbm": byt / ms / 1e6 / hbm,
                                           "bound": "hbm", "algorithmic_bytes": byt}
        plan.close()
        del out

    # S3 roofline: 512 rotations of the RGB 256x512 map, full FP32 output (805 MB)
    if want("rotation_shift_batch"):
        sc2 = synth.scene(2, V=1)
        L2 = hs.haar_forward(torch.tensor(sc2["light"], dtype=torch.float32, device=dev))
        S = 512
        eul = torch.tensor(synth.euler_angles(synth.rng_for(2, 7), S), dtype=torch.float64, device=dev)
        plan = hs.Plan(256, 512, 3, kind=hs.HAAR_SHIFT_ROTATE_EULER, max_shifts=S)
        out = torch.empty(plan.out_shape(S), dtype=torch.float32, device=dev)
        ms = _timeit(lambda: hs.haar_shift(plan, L2, eul, out), 5, flush, stream)
        byt = 4 * 3 * 131072 * (S + 1)
        rows["rotation_shift_batch"] = {"what": "haar_shift, 512 rotations of RGB 256x512, FP32 SCK",
                                        "ms": ms, "achieved_gbs": byt / ms / 1e6, "frac_hbm": byt / ms / 1e6 / hbm,
                                        "bound": "alu (atan2 coordinates) / hbm", "algorithmic_bytes": byt}
        plan.close()
        del out

    # coefficient-count sweep (the paper's other accuracy / cost knob): the c1
    # frame shaded from the top-K transport, K = 4 .. 256 (group CSR), time and
    # rel-L2 of the radiance against the untruncated double product on 512
    # sampled vertices
    if want("coefficient_count_sweep"):
        sc1 = synth.scene(1)
        H, W, C, S, V = sc1["H"], sc1["W"], sc1["C"], sc1["S"], sc1["V"]
        Lc = hs.haar_forward(torch.tensor(sc1["light"], dtype=torch.float32, device=dev)).contiguous()
        prm = torch.tensor(sc1["params"], dtype=torch.float64, device=dev)
        Kmax = 256
        order = torch.empty((V, Kmax), dtype=torch.int64, device=dev)      # by decreasing |T|
        ordv = torch.empty((V, Kmax), dtype=torch.float32, device=dev)
        pick = torch.tensor(np.sort(np.random.default_rng(11).choice(V, 512, replace=False)), device=dev)
        dense_pick = torch.empty((512, H * W), dtype=torch.float64, device=dev)
        for v0 in range(0, V, 4096):
            v1 = min(V, v0 + 4096)
            w = synth.transport_weights(sc1["pos"][v0:v1], sc1["nrm"][v0:v1], sc1["occ_c"], sc1["occ_r"], H, W,
                                        device=dev, dtype=torch.float32, chunk=2048).contiguous()
            T = hs.haar_forward(w)
            top = torch.topk(T.abs(), Kmax, dim=1, sorted=True).indices
            order[v0:v1] = top
            ordv[v0:v1] = torch.gather(T, 1, top)
            sel = (pick >= v0) & (pick < v1)
            if bool(sel.any()):
                dense_pick[sel] = T[pick[sel] - v0].double()
            del w, T
        plan = hs.Plan(H, W, C, max_shifts=S, out_layout=hs.HAAR_LAYOUT_KSC)
        lit = torch.empty(plan.out_shape(S), dtype=torch.float32, device=dev)
        hs.haar_shift(plan, Lc, prm, lit)
        Ld = lit.double().reshape(H * W, S * C)
        exact = (dense_pick @ Ld).reshape(512, S, C)
        R = torch.empty((V, S, C), dtype=torch.float32, device=dev)
        sweep = []
        for K in (4, 8, 16, 32, 64, 128, 256):
            idx, perm = torch.sort(order[:, :K], dim=1)
            vals = torch.gather(ordv[:, :K], 1, perm).reshape(-1).contiguous()
            rowptr = (torch.arange(V + 1, device=dev, dtype=torch.int64) * K).to(torch.int32)
            idx16 = idx.to(torch.int32).to(torch.int16).reshape(-1).contiguous()
            tr = hs.haar_transport_group(V, H * W, rowptr, idx16, vals)
            ms = _timeit(lambda: hs.shade_vertices(plan, tr, lit, S, R), 10, flush, stream)
            err = float(((R[pick].double() - exact).norm() / exact.norm()).item())
            sweep.append({"K": K, "shade_ms": ms, "rel_l2_vs_untruncated": err})
            del tr, vals, idx16
        rows["coefficient_count_sweep"] = {"what": "c1 frame shaded from top-K transport (4-vertex group CSR), "
                                                   "error against the untruncated double product (512 vertices)",
                                           "levels": sweep}
        plan.close()
        del order, ordv, dense_pick

    # start-level sweep (the paper's accuracy / cost knob): the 64 c2 rotations of
    # RGB 256x512 started at level k = 0..3, time and rel-L2 of the N/4^k
    # coarsest coefficients against the full-map shift's
    if want("start_level_sweep"):
        sc2 = synth.scene(2, V=1)
        L2 = hs.haar_forward(torch.tensor(sc2["light"], dtype=torch.float32, device=dev))
        eul = torch.tensor(sc2["params"], dtype=torch.float64, device=dev)
        S = eul.shape[0]
        sweep, exact = [], None
        for k in range(4):
            plan = hs.Plan(256, 512, 3, kind=hs.HAAR_SHIFT_ROTATE_EULER, max_shifts=S, start_level=k)
            out = torch.empty(plan.out_shape(S), dtype=torch.float32, device=dev)
            ms = _timeit(lambda: hs.haar_shift(plan, L2, eul, out), 10, flush, stream)
            if k == 0:
                exact = out.clone()
            n = out.shape[-1]
            ref = exact[..., :n]
            err = float(((out - ref).norm() / ref.norm()).item())
            sweep.append({"start_level": k, "coeffs": n, "ms": ms, "rel_l2_vs_full_map": err})
            plan.close()
        rows["start_level_sweep"] = {"what": "64 rotations of RGB 256x512 started at level k (Sec. Algorithmic "
                                             "optimization), FP32", "levels": sweep}

    # the paper's own rotation route (chain rule on the finest derivative fields,
    # Eq. pde1-pde3, then Eq. conv/tker/sker) beside the exact operator: time for
    # the 64 c2 rotations of RGB 256x512, and its accuracy as PSNR against the
    # exact rotation (the synthetic analogue of Tables 1-4, at the paper's
    # levels 5 and 6 and at 256x512) on two kinds of map: a band-limited one
    # (smooth at the poles, like a measured environment's low frequencies) and
    # the per-pixel lognormal map of the c2 scene.  PSNR = 10 log10(peak^2 /
    # MSE) with the source map's peak and the per-pixel MSE (the transform is
    # orthonormal, so it is the coefficient MSE), averaged over the rotations
    if want("chain_rule_rotation"):
        sc2 = synth.scene(2, V=1)
        eul = torch.tensor(sc2["params"], dtype=torch.float64, device=dev)
        S = eul.shape[0]
        acc = []
        for lvl, (H, W), kind in ((5, (32, 64), "smooth"), (6, (64, 128), "smooth"), (8, (256, 512), "smooth"),
                                  (5, (32, 64), "lognormal"), (6, (64, 128), "lognormal"),
                                  (8, (256, 512), "lognormal")):
            if kind == "smooth":
                light = synth.smooth_lighting(synth.rng_for(2, 30 + lvl), 3, H, W)
            elif H != 256:
                light = synth.lighting_pixels(synth.rng_for(2, 20 + lvl), 3, H, W)
            else:
                light = sc2["light"]
            Lm = hs.haar_forward(torch.tensor(light, dtype=torch.float32, device=dev))
            pe = hs.Plan(H, W, 3, kind=hs.HAAR_SHIFT_ROTATE_EULER, max_shifts=S)
            pc = hs.Plan(H, W, 3, kind=hs.HAAR_SHIFT_ROTATE_CHAIN, max_shifts=S)
            oe = torch.empty(pe.out_shape(S), dtype=torch.float32, device=dev)
            oc = torch.empty(pc.out_shape(S), dtype=torch.float32, device=dev)
            hs.haar_shift(pe, Lm, eul, oe)
            hs.haar_shift(pc, Lm, eul, oc)
            mse = ((oc.double() - oe.double()) ** 2).mean(dim=(1, 2))
            peak = float(np.max(light))
            psnr = (10.0 * torch.log10(peak * peak / mse)).cpu().numpy()
            rel = ((oc.double() - oe.double()).norm(dim=(1, 2)) / oe.double().norm(dim=(1, 2))).cpu().numpy()
            row = {"level": lvl, "map": f"{H}x{W} {kind}", "psnr_db_mean": float(psnr.mean()),
                   "psnr_db_min": float(psnr.min()), "rel_l2_mean": float(rel.mean()), "rel_l2_max": float(rel.max())}
            if H == 256 and kind == "lognormal":
                row["chain_ms"] = _timeit(lambda: hs.haar_shift(pc, Lm, eul, oc), 10, flush, stream)
                row["exact_ms"] = _timeit(lambda: hs.haar_shift(pe, Lm, eul, oe), 10, flush, stream)
            acc.append(row)
            pe.close()
            pc.close()
            del oe, oc
        rows["chain_rule_rotation"] = {"what": "64 rotations of RGB maps by the paper's chain-rule route "
                                               "(HAAR_SHIFT_ROTATE_CHAIN) against the exact operator, FP32",
                                       "levels": acc}

    # the paper's shading loop (N2): rotation input pass (normal -> record),
    # rotation pass (each vertex's BRDF map rotated onto its normal by
    # haar_shift) and triple integral pass (Tripling Coefficient Theorem) for
    # the 50 000 c1 torus vertices, at the paper's levels 5 (32x64) and 6
    # (64x128); the triple kernel is bound by reading each vertex's two rows
    if want("triple_product_loop"):
        sc1 = synth.scene(1)
        V = sc1["V"]
        nrm = torch.tensor(sc1["nrm"], dtype=torch.float32, device=dev)
        levels = []
        for lvl, (H, W) in ((5, (32, 64)), (6, (64, 128))):
            N = H * W
            light = hs.haar_forward(torch.tensor(synth.lighting_pixels(synth.rng_for(1, 40 + lvl), 3, H, W),
                                                 dtype=torch.float32, device=dev))
            brdf = hs.haar_forward(torch.tensor(synth.local_brdf_map(H, W)[None], dtype=torch.float32, device=dev))
            vis = torch.empty((V, N), dtype=torch.float32, device=dev)
            for v0 in range(0, V, 8192):
                v1 = min(V, v0 + 8192)
                w = synth.transport_weights(sc1["pos"][v0:v1], sc1["nrm"][v0:v1], sc1["occ_c"], sc1["occ_r"], H, W,
                                            device=dev, dtype=torch.float32, chunk=4096, cosine=False).contiguous()
                vis[v0:v1] = hs.haar_forward(w)
                del w
            plan = hs.Plan(H, W, 1, kind=hs.HAAR_SHIFT_ROTATE, max_shifts=V)
            prm = torch.empty((V, 9), dtype=torch.float64, device=dev)
            rot = torch.empty(plan.out_shape(V), dtype=torch.float32, device=dev)
            out = torch.empty((V, 3), dtype=torch.float32, device=dev)
            work = torch.empty(hs.haar_triple_work_floats(H, W, 3), dtype=torch.float32, device=dev)

            work2 = torch.empty(hs.haar_shade_triple_work_floats(H, W, 3), dtype=torch.float32, device=dev)
            brdf_l = brdf[0].contiguous()

            def unfused():
                hs.haar_normal_rotations(nrm, prm)
                hs.haar_shift(plan, brdf, prm, rot)
                hs.haar_triple_product(H, W, light, rot[:, 0, :], vis, out, work)

            def fused():
                hs.haar_normal_rotations(nrm, prm)
                hs.haar_shade_triple(H, W, light, brdf_l, prm, vis, out, work2)

            unfused()
            ref_out = out.clone()
            fused()
            agree = float(((out - ref_out).norm() / ref_out.norm()).item())
            ms_frame = _timeit(fused, 10, flush, stream)
            ms_fused = _timeit(lambda: hs.haar_shade_triple(H, W, light, brdf_l, prm, vis, out, work2), 10, flush,
                               stream)
            ms_unfused = _timeit(unfused, 10, flush, stream)
            ms_rot = _timeit(lambda: hs.haar_shift(plan, brdf, prm, rot), 10, flush, stream)
            ms_tri = _timeit(lambda: hs.haar_triple_product(H, W, light, rot[:, 0, :], vis, out, work), 10, flush,
                             stream)
            byt = V * (2 * N + 3) * 4
            byt_fused = V * (N + 3) * 4
            levels.append({"level": lvl, "map": f"{H}x{W}", "frame_ms": ms_frame, "vertices_per_s": V / ms_frame * 1e3,
                           "fused_kernel_ms": ms_fused, "fused_achieved_gbs": byt_fused / ms_fused / 1e6,
                           "fused_bound": "alu (per-pixel rotation coordinates)",
                           "unfused_frame_ms": ms_unfused, "unfused_rotation_ms": ms_rot, "triple_ms": ms_tri,
                           "triple_achieved_gbs": byt / ms_tri / 1e6, "triple_frac_hbm": byt / ms_tri / 1e6 / hbm,
                           "triple_algorithmic_bytes": byt, "fused_vs_unfused_rel_l2": agree})
            plan.close()
            del vis, rot
        rows["triple_product_loop"] = {"what": "shading loop of 50 000 torus vertices: normal -> rotation record, "
                                               "Lambertian BRDF map rotated per vertex, RGB triple product with "
                                               "per-vertex visibility, FP32; frame = the fused kernel "
                                               "(haar_shade_triple), unfused = haar_shift + haar_triple_product",
                                       "levels": levels}

    # the paper's whole frame with a headless rasteriser in place of its Cg pass
    # (N4): a 50 176-vertex torus mesh shaded per vertex by the fused shading
    # loop (level 5, Lambertian, c1 occluders), rasterised at 1920x1080
    # (triangle id + perspective-correct barycentrics per pixel) and shaded
    # per pixel by interpolating the vertex radiance
    if want("raster_frame"):
        sc1 = synth.scene(1, V=1)
        pos_np, nrm_np, tris_np = synth.torus_mesh(256, 196)
        V, T = len(pos_np), len(tris_np)
        H, W = 32, 64
        Wi, Hi = 1920, 1080
        pos = torch.tensor(pos_np, device=dev)
        nrm = torch.tensor(nrm_np, device=dev)
        tris = torch.tensor(tris_np, device=dev)
        M = torch.tensor(synth.view_projection((0.4, 1.6, 2.6), (0.0, 0.0, 0.0), aspect=Wi / Hi).reshape(-1),
                         device=dev)
        light = hs.haar_forward(torch.tensor(synth.lighting_pixels(synth.rng_for(1, 45), 3, H, W),
                                             dtype=torch.float32, device=dev))
        brdf = hs.haar_forward(torch.tensor(synth.local_brdf_map(H, W), dtype=torch.float32, device=dev)[None])[0]
        w = synth.transport_weights(pos_np, nrm_np, sc1["occ_c"], sc1["occ_r"], H, W, device=dev,
                                    dtype=torch.float32, chunk=4096, cosine=False).contiguous()
        vis = hs.haar_forward(w)
        del w
        prm = torch.empty((V, 9), dtype=torch.float64, device=dev)
        rad = torch.empty((V, 3), dtype=torch.float32, device=dev)
        work = torch.empty(hs.haar_shade_triple_work_floats(H, W, 3), dtype=torch.float32, device=dev)
        rs = hs.Raster(Wi, Hi, V)
        bg = torch.zeros(3, dtype=torch.float32, device=dev)
        img = torch.empty((Hi, Wi, 3), dtype=torch.float32, device=dev)

        def frame():
            hs.haar_normal_rotations(nrm, prm)
            hs.haar_shade_triple(H, W, light, brdf, prm, vis, rad, work)
            rs.rasterize(pos, tris, M)
            rs.shade(tris, rad, bg, img)

        frame()
        covered = int((rs.tri_id >= 0).sum().item())
        ms_frame = _timeit(frame, 10, flush, stream)
        ms_raster = _timeit(lambda: rs.rasterize(pos, tris, M), 10, flush, stream)
        ms_pix = _timeit(lambda: rs.shade(tris, rad, bg, img), 10, flush, stream)
        rows["raster_frame"] = {"what": "torus mesh of 50 176 vertices / 100 352 triangles: fused per-vertex "
                                        "shading loop (32x64, RGB) + headless rasterisation at 1920x1080 + "
                                        "per-pixel interpolation", "frame_ms": ms_frame,
                                "frames_per_s": 1e3 / ms_frame, "raster_ms": ms_raster, "pixel_shade_ms": ms_pix,
                                "covered_pixels": covered, "triangles": T, "vertices": V}

    # c2 frame: 64 rotations -> bf16 hi/lo lowest 4096 -> tcgen05 contraction for 200k vertices
    if want("c2_dense_tc"):
        sc2 = synth.scene(2)
        V, K, S = sc2["V"], 4096, 64
        T = torch.empty((V, K), dtype=torch.bfloat16, device=dev)
        for a in range(0, V, 16384):
            b = min(V, a + 16384)
            w = synth.transport_weights(sc2["pos"][a:b], sc2["nrm"][a:b], sc2["occ_c"], sc2["occ_r"], 64, 128,
                                        device=dev, dtype=torch.float32, chunk=8192).contiguous()
            T[a:b] = hs.haar_forward(w, scale=0.25)[:, :K].to(torch.bfloat16)
            del w
        L2 = hs.haar_forward(torch.tensor(sc2["light"], dtype=torch.float32, device=dev))
        eul = torch.tensor(sc2["params"], dtype=torch.float64, device=dev)
        plan = hs.Plan(256, 512, 3, kind=hs.HAAR_SHIFT_ROTATE_EULER, max_shifts=S, out_coeffs=K,
                       out_type=hs.HAAR_OUT_BF16_HILO)
        lit = torch.empty(plan.out_shape(S), dtype=torch.bfloat16, device=dev)
        tr = hs.Transport(hs.HAAR_T_DENSE_BF16, V, K, T)
        R = torch.empty((V, S, 3), dtype=torch.float32, device=dev)
        hs.haar_shift(plan, L2, eul, lit)
        ms_gemm = _timeit(lambda: hs.shade_vertices(plan, tr, lit, S, R), 10, flush, stream)
        ms_frame = _timeit(lambda: (hs.haar_shift(plan, L2, eul, lit), hs.shade_vertices(plan, tr, lit, S, R)), 10,
                           flush, stream)
        flops = 2.0 * 2.0 * V * K * S * 3
        gbytes = (2.0 * V * K + 4.0 * V * S * 3 + 2 * 2.0 * S * 3 * K)
        rows["c2_dense_tc"] = {"what": "c2 frame: 64 rotations + tcgen05 bf16 contraction T[200000x4096] x (Lhi+Llo)[4096x192]",
                               "frame_ms": ms_frame, "value": V * S / ms_frame / 1e3, "unit": UNIT,
                               "kernel": "k_dense_bf16", "kernel_ms": ms_gemm,
                               "achieved_tflops": flops / ms_gemm / 1e9, "peak_tflops": bf16_peak,
                               "frac_tensor": flops / ms_gemm / 1e9 / bf16_peak,
                               "achieved_gbs": gbytes / ms_gemm / 1e6, "frac_hbm": gbytes / ms_gemm / 1e6 / hbm,
                               "flops_counted": "2 x (2 V K S C): hi and lo products"}
        plan.close()
        del T, lit, R, tr

    # c3 frame: view bins + 32 rotations (FP32 SKC4) + view-binned top-512 FP16 shading
    c3 = None
    if want("c3_bincsr") or want("c4_surrogate") or want("surrogate_training") or want("glossy_coefficient_sweep"):
        sc3 = synth.scene(3)
        V, S = sc3["V"], sc3["S"]
        vals, idx, absum = _glossy_transport(hs, sc3, dev)
        f = lambda x: torch.tensor(x, dtype=torch.float32, device=dev)
        pos, nrm, cams, dirs = f(sc3["pos"]), f(sc3["nrm"]), f(sc3["cams"]), f(synth.view_bin_dirs(16))
        eul3 = torch.tensor(sc3["params"], dtype=torch.float64, device=dev)
        L3 = hs.haar_forward(torch.tensor(sc3["light"], dtype=torch.float32, device=dev))
        plan = hs.Plan(256, 512, 3, kind=hs.HAAR_SHIFT_ROTATE_EULER, max_shifts=S, out_layout=hs.HAAR_LAYOUT_SKC4)
        lit = torch.empty(plan.out_shape(S), dtype=torch.float32, device=dev)
        bins = torch.empty((S, V), dtype=torch.uint8, device=dev)
        R = torch.empty((V, S, 3), dtype=torch.float32, device=dev)
        tr = hs.Transport(hs.HAAR_T_BINCSR_F16_U32, V, 512, vals, idx, bins=16, bin_of=bins)

        def c3_frame():
            hs.haar_view_bins(pos, nrm, cams, dirs, bins)
            hs.haar_shift(plan, L3, eul3, lit)
            hs.shade_vertices(plan, tr, lit, S, R)
        ms_frame = _timeit(c3_frame, 10, flush, stream)
        plain_c3 = V * S / ms_frame / 1e3
        if want("c3_bincsr"):
            ms_shade = _timeit(lambda: hs.shade_vertices(plan, tr, lit, S, R), 10, flush, stream)
            distinct = int(torch.unique(bins.to(torch.int64) + 16 * torch.arange(V, device=dev)[None, :]).numel())
            byt = distinct * 512 * 6 + V * S * 3 * 4 + S * 8192 * 3 * 4
            rows["c3_bincsr"] = {"what": "c3 frame: view bins + 32 rotations + top-512 FP16 view-binned shading, 100k vertices",
                                 "frame_ms": ms_frame, "value": plain_c3, "unit": UNIT,
                                 "kernel": "k_shade_bincsr_f16", "kernel_ms": ms_shade,
                                 "achieved_gbs": byt / ms_shade / 1e6, "frac_hbm": byt / ms_shade / 1e6 / hbm,
                                 "distinct_vertex_bins": distinct,
                                 "transport": "per (vertex, bin) the top 512 of the lowest 8192 coefficients (Phong "
                                              "transfer integrated on the 64x128 grid: levels 1-2 of the 256x512 map "
                                              "are zero, so no stored index is finer than level 3)"}
        del tr, R
        c3 = True

    # N3 with glossiness: the c3 frame's view-binned shading from the top-K of
    # each stored row, K = 16 .. 512, for Phong exponents 8, 32 and 128 (every
    # vertex at that exponent); time of the shading kernel and rel-L2 of the
    # radiance against the untruncated product (all 8192 coefficients of the
    # same bin's transport) on sampled (vertex, pair)
    if c3 and want("glossy_coefficient_sweep"):
        sweep = []
        rng = np.random.default_rng(47)
        ns = 4096
        vs_ = torch.tensor(rng.integers(0, V, ns), device=dev)
        ss_ = torch.tensor(rng.integers(0, S, ns), device=dev)
        Lk = lit.reshape(S, -1, 4)[:, :8192, :3].double()
        Rk = torch.empty((V, S, 3), dtype=torch.float32, device=dev)
        for ex in (8.0, 32.0, 128.0):
            gv, gi, _ = _glossy_transport(hs, sc3, dev, K=512, expo=ex, by_magnitude=True)
            b_ = bins[ss_, vs_].long()
            vsn, bsn = vs_.cpu().numpy(), b_.cpu().numpy()
            view = synth.bin_view_world(sc3["nrm"][vsn], 16)[np.arange(ns), bsn]
            Tf = torch.empty((ns, 8192), dtype=torch.float64, device=dev)

            def putf(a, b, T):
                Tf[a:b] = T.double()
            _glossy_rows(hs, sc3, dev, (sc3["pos"][vsn], sc3["nrm"][vsn], view, np.full(ns, ex)), putf)
            full = torch.zeros((ns, 3), dtype=torch.float64, device=dev)
            for s_ in range(S):
                m = ss_ == s_
                if bool(m.any()):
                    full[m] = Tf[m] @ Lk[s_]
            levels = []
            for K in (16, 32, 64, 128, 256, 512):
                ik, perm = torch.sort(gi[..., :K], dim=2)
                vk = torch.gather(gv[..., :K], 2, perm).contiguous()
                trk = hs.Transport(hs.HAAR_T_BINCSR_F16_U32, V, K, vk, ik.contiguous(), bins=16, bin_of=bins)
                ms = _timeit(lambda: hs.shade_vertices(plan, trk, lit, S, Rk), 5, flush, stream)
                got = Rk[vs_, ss_].double()
                levels.append({"K": K, "shade_ms": ms,
                               "rel_l2_vs_untruncated": float((got - full).norm() / full.norm())})
                del trk, vk, ik, perm
            sweep.append({"phong_exponent": ex, "levels": levels})
            del gv, gi, Tf
        rows["glossy_coefficient_sweep"] = {"what": "c3 frame shaded from the top-K of each view-binned row "
                                                    "(every vertex at one Phong exponent), shading kernel time "
                                                    "and error against the bin's untruncated transport "
                                                    f"({ns} sampled (vertex, pair))", "exponents": sweep}

    if c3 and (want("c4_surrogate") or want("surrogate_training")):
        # S8 + c4: train the surrogate on transports of the glossy scene (random
        # (vertex, camera) pairs, Phong transfer on the 64x128 grid projected by
        # haar_forward), index set = the 512 largest mean |T|; then the c4 frame:
        # the same 32 rotations, transport from the trained surrogate fused with
        # the shading, and its accuracy against the stored-transport frame
        from paper_1705_07272_gb300 import training
        K = 512
        n_train = int(os.environ.get("HAAR_SURROGATE_SAMPLES", "2000000"))
        rng = np.random.default_rng(41)
        raw_tr, gen_tr = _glossy_pairs(rng, sc3, n_train)
        nt = 8192
        s1 = torch.zeros(nt, dtype=torch.float64, device=dev)
        s2 = torch.zeros(nt, dtype=torch.float64, device=dev)
        sa = torch.zeros(nt, dtype=torch.float64, device=dev)

        def acc_moments(a, b, T):
            s1.add_(T.sum(0).double())
            s2.add_((T.double() ** 2).sum(0))
            sa.add_(T.abs().sum(0).double())
        t0 = time.perf_counter()
        _glossy_rows(hs, sc3, dev, gen_tr, acc_moments)
        isel = torch.sort(torch.topk(sa, K).indices).values
        mu64 = s1[isel] / n_train
        sg64 = torch.sqrt(torch.clamp((s2[isel] / n_train - mu64 ** 2).mean(), min=1e-30))
        Y = torch.empty((n_train, K), dtype=torch.float32, device=dev)

        def targets(a, b, T):
            Y[a:b] = ((T[:, isel].double() - mu64) / sg64).float()
        _glossy_rows(hs, sc3, dev, gen_tr, targets)
        torch.cuda.synchronize()
        t_data = time.perf_counter() - t0
        raw_g = torch.tensor(raw_tr, dtype=torch.float32, device=dev)
        net = hs.Surrogate(max_batch=8192, max_rows=262144, max_groups=S)
        net.set_params(torch.tensor(_init_params(np.random.default_rng(4)), dtype=torch.float32, device=dev))
        epochs = int(os.environ.get("HAAR_SURROGATE_EPOCHS", "30"))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        last_loss = training.fit(net, raw_g, Y, epochs=epochs, batch=8192, lr=(2e-3, 6e-4, 2e-4))
        torch.cuda.synchronize()
        t_train = time.perf_counter() - t0
        del Y, raw_g
        mu = mu64.float().contiguous()
        sg = sg64.float().expand(K).contiguous()
        isel32 = isel.to(torch.int32)
        R4 = torch.empty((V, S, 3), dtype=torch.float32, device=dev)
        N3 = 131072
        strides = (N3 * 4, 1, 4)                    # SKC4 lighting
        hs.haar_shift(plan, L3, eul3, lit)
        acc = _surrogate_accuracy(hs, net, sc3, dev, lit, bins, vals, idx, isel, mu64, sg64, sa)
        if want("c4_surrogate"):
            def c4_frame():
                hs.haar_shift(plan, L3, eul3, lit)
                net.shade(pos, nrm, cams, mu, sg, isel32, lit, 3, strides, R4)
            ms_frame = _timeit(c4_frame, 5, flush, stream)
            ms_mlp = _timeit(lambda: net.shade(pos, nrm, cams, mu, sg, isel32, lit, 3, strides, R4), 5, flush, stream)
            mlp_flops = 2.0 * V * S * (320 * 256 + 3 * 256 * 256 + 256 * 3)
            rows["c4_surrogate"] = {"what": "c4 frame: 32 rotations + surrogate transport (4x256 GELU MLP, bf16 tcgen05) "
                                            "fused with shading, trained weights",
                                    "frame_ms": ms_frame, "value": V * S / ms_frame / 1e3, "unit": UNIT,
                                    "kernel": "haar_mlp_shade", "kernel_ms": ms_mlp,
                                    "achieved_tflops": mlp_flops / ms_mlp / 1e9,
                                    "frac_tensor": mlp_flops / ms_mlp / 1e9 / bf16_peak,
                                    "vs_plain_c3_frame": (V * S / ms_frame / 1e3) / plain_c3,
                                    "weights": f"trained: {n_train} transports, {epochs} epochs of batch 8192, "
                                               f"last-epoch loss {last_loss:.4f}",
                                    "accuracy": acc,
                                    "storage_bytes": {"surrogate_weights_bf16": int(net.n_params) * 2,
                                                      "view_binned_transport": V * 16 * 512 * 6}}
        if want("surrogate_training"):
            # S8: one Adam training step on a batch of 8192, and the whole training run above
            B = 8192
            raw = torch.randn((B, 9), dtype=torch.float32, device=dev)
            tgt = torch.randn((B, 512), dtype=torch.float32, device=dev)
            ms_eager = _timeit(lambda: net.train_step(raw, tgt, 1e-7), 10, flush, stream)
            graph, _ = net.capture_train_step(raw, tgt, 1e-7)
            ms_train = _timeit(graph.replay, 10, flush, stream)
            tflops = 3.0 * 2.0 * B * (320 * 256 + 3 * 256 * 256 + 256 * 512) / ms_train / 1e9
            rows["surrogate_training"] = {"what": "haar_mlp_train_step, batch 8192 (forward, backward, Adam), "
                                                  "replayed from a CUDA graph; and the c4 training run",
                                          "ms": ms_train, "eager_ms": ms_eager, "samples_per_s": B / ms_train * 1e3,
                                          "achieved_tflops": tflops, "frac_tensor": tflops / bf16_peak,
                                          "training_run": {"samples": n_train, "epochs": epochs,
                                                           "data_s": t_data, "train_s": t_train,
                                                           "last_epoch_loss": last_loss}}
        net.close()
    if c3:
        del vals, idx
        plan.close()
    return rows


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        out_dir = os.environ.get("HAAR_CLOCKS_DIR", os.path.join(ROOT, "clocks"))
        self.path = os.path.join(out_dir, f"clocks_rank{index}.csv")

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
    cpu, checks = None, None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # the host-side leg: the oracle's timed frame sample and the oracle's
        # results for the rows' accuracy checks, all before any GPU work
        cpu = cpu_baseline(args.cpu_sample)
        checks = oracle_checks()

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

    if args.only:
        flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
        print(json.dumps({"rows": measure_rows(hs, dev, flush, set(args.only.split(",")), args.batch_shifts)}),
              flush=True)
        return 0
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
    total_ms = max_over_ranks(sum(step_ms), dev)
    ms_per_step = total_ms / args.steps
    units = wl["V"] * wl["S"] * world
    value = whole_job_value(wl["V"] * wl["S"], ms_per_step, world)

    # per-kernel durations for the roofline: the same frames (same stream, same
    # flush discipline) with an event between the shift and the shading, so the
    # shading kernel is timed as it runs in the frame (lighting just written)
    def timed_split(shade_tr, k):
        evs = []
        for _ in range(k):
            flush.fill_(1.0)
            a, m, b = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            a.record(stream)
            hs.haar_shift(plan, wl["L"], wl["params"], wl["lighting"])
            m.record(stream)
            hs.shade_vertices(plan, shade_tr, wl["lighting"], wl["S"], wl["radiance"])
            b.record(stream)
            evs.append((a, m, b))
        torch.cuda.synchronize()
        return [a.elapsed_time(m) for a, m, b in evs], [m.elapsed_time(b) for a, m, b in evs]

    shift_ms, shade_ms = timed_split(tr, args.steps)
    shade_avg, shift_avg = statistics.mean(shade_ms), statistics.mean(shift_ms)
    ab = algorithmic_bytes(wl)
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    hbm = peaks.get("hbm_gbs", 6800.0)
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
    csr_avg = statistics.mean(timed_split(wl["csr"], args.steps)[1])
    if shade_avg >= shift_avg:
        kname, kms = "k_shade_gcsr48", shade_avg
    else:
        kname, kms = "k_shift", shift_avg
    achieved = ab[kname] / (kms * 1e-3) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                "traffic": traffic_record(kname), "kernel": kname, "peak_source": peak_src,
                "algorithmic_bytes": ab[kname], "kernel_ms": kms,
                "other_kernels_ms": {"k_setup+k_shift": shift_avg, "k_shade_gcsr48": shade_avg},
                "plain_csr_kernel": {"kernel": "k_shade_csr_f32", "ms": csr_avg,
                                     "achieved_gbs": ab["k_shade_csr_f32"] / (csr_avg * 1e-3) / 1e9}}
    if kname == "k_shade_gcsr48":
        # what binds it: every group-CSR entry gathers one lighting row (S C
        # floats) from the L2-resident lighting
        gb = wl["union"] * wl["S"] * wl["C"] * 4
        roofline["l2_row_gather_bytes"] = gb
        roofline["l2_row_gather_gbs"] = gb / (kms * 1e-3) / 1e9

    # end to end through the public API with host buffers
    L_host = wl["L"].cpu().pin_memory()
    p_host = wl["params"].cpu().pin_memory()
    R_host = torch.empty(wl["radiance"].shape, dtype=torch.float32).pin_memory()
    L_dev = torch.empty_like(wl["L"])
    p_dev = torch.empty_like(wl["params"])

    # the inputs are copied host -> device every step; the shading kernel
    # writes the radiance straight into pinned host memory (NVLink-C2C), which
    # measured 0.135 ms per step against 0.191 ms for a device buffer plus a
    # separate device -> host copy
    def e2e_step():
        L_dev.copy_(L_host, non_blocking=True)
        p_dev.copy_(p_host, non_blocking=True)
        hs.shade_batch(plan, L_dev, p_dev, tr, R_host)

    for _ in range(3):
        e2e_step()
    e2e_ms = timed(e2e_step, args.steps)
    e2e_tot = max_over_ranks(sum(e2e_ms), dev)
    e2e_value = whole_job_value(wl["V"] * wl["S"], e2e_tot / args.steps, world)
    h2d = L_host.numel() * 4 + p_host.numel() * 8
    d2h = R_host.numel() * 4

    rows = None
    if rank == 0 and not args.no_rows:
        rows = measure_rows(hs, dev, flush)
    acc = gpu_checks(hs, dev, checks) if checks is not None else None
    if acc is not None and rows is not None:
        for name, r in acc.items():
            if name in rows:
                rows[name]["accuracy"] = r

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": bench_config(world),
                "roofline": roofline, "cpu_baseline": cpu,
                "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                        "d2h": "radiance written by the shading kernel into pinned host memory"},
                "gpu_launches": 3 * args.steps, "clocks": clk,
                "accuracy": None if acc is None else acc["c1"], "rows": rows}
        print(json.dumps(line), flush=True)
    plan.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
