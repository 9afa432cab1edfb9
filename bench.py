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
    return {"k_shade_gcsr_f32": gcsr, "k_shade_csr_f32": csr, "k_shift": shift}


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


def _glossy_transport(hs, sc, dev, bins=16, K=512, chunk=8192):
    """View-binned top-K glossy transport of every (vertex, bin) on the GPU:
    Phong transfer on the 64x128 grid, projected by haar_forward (the lowest
    8192 coefficients of the 256x512 map), top-K per row, sorted by index."""
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
        w = synth.transport_weights(sc["pos"][vi], sc["nrm"][vi], sc["occ_c"], sc["occ_r"], 64, 128,
                                    view=view[a:b], expo=sc["expo"][vi], device=dev, dtype=torch.float32,
                                    chunk=chunk)
        T = hs.haar_forward(w.contiguous(), scale=0.25)
        absum += T.abs().sum(0).double()
        top = torch.topk(T.abs(), K, dim=1).indices
        top, _ = torch.sort(top, dim=1)
        idx[a:b] = top.to(torch.int32)
        vals[a:b] = torch.gather(T, 1, top).to(torch.float16)
        del w, T
    return vals.reshape(V, bins, K), idx.reshape(V, bins, K), absum


def measure_rows(hs, dev, flush, only=None):
    """Per-row measurements of the rest of the hot path; ``only`` restricts
    them to the named rows (for profiling one kernel)."""
    import numpy as np
    import torch
    import synth
    stream = torch.cuda.current_stream(dev)
    bf16_peak, hbm = _bf16_peak()
    rows = {}

    def want(name):
        return only is None or name in only

    # S2 / S4 roofline: 4096 translations of the RGB 128x256 map, full FP32 output (1.6 GB)
    if want("translation_shift_batch"):
        sc1 = synth.scene(1, V=1)
        L1 = hs.haar_forward(torch.tensor(sc1["light"], dtype=torch.float32, device=dev))
        S = 4096
        prm = torch.tensor(synth.translations(synth.rng_for(1, 7), S, 256.0, 256.0), dtype=torch.float64, device=dev)
        plan = hs.Plan(128, 256, 3, max_shifts=S)
        out = torch.empty(plan.out_shape(S), dtype=torch.float32, device=dev)
        ms = _timeit(lambda: hs.haar_shift(plan, L1, prm, out), 5, flush, stream)
        byt = 4 * 3 * 32768 * (S + 1)
        rows["translation_shift_batch"] = {"what": "haar_shift, 4096 fractional shifts of RGB 128x256, FP32 SCK",
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
    if want("c3_bincsr") or want("c4_surrogate") or want("surrogate_training"):
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
                                 "distinct_vertex_bins": distinct}
        del vals, idx, tr, R
        c3 = True

    if c3 and (want("c4_surrogate") or want("surrogate_training")):
        # c4 frame: the same 32 rotations, transport from the surrogate (random-init
        # weights, index set = 512 largest mean |T| of the c3 transports), fused shading
        K = 512
        isel = torch.sort(torch.topk(absum, K).indices).values.to(torch.int32)
        mu = torch.zeros(K, dtype=torch.float32, device=dev)
        sg = torch.full((K,), 1e-3, dtype=torch.float32, device=dev)
        net = hs.Surrogate(max_batch=8192, max_rows=262144, max_groups=S)
        rng = np.random.default_rng(4)
        flat = []
        for fi, fo in ((320, 256), (256, 256), (256, 256), (256, 256), (256, 512)):
            flat += [rng.standard_normal(fo * fi) * math.sqrt(2.0 / fi), np.zeros(fo)]
        net.set_params(torch.tensor(np.concatenate(flat), dtype=torch.float32, device=dev))
        R4 = torch.empty((V, S, 3), dtype=torch.float32, device=dev)
        N3 = 131072
        strides = (N3 * 4, 1, 4)                    # SKC4 lighting
        if want("c4_surrogate"):
            def c4_frame():
                hs.haar_shift(plan, L3, eul3, lit)
                net.shade(pos, nrm, cams, mu, sg, isel, lit, 3, strides, R4)
            ms_frame = _timeit(c4_frame, 5, flush, stream)
            ms_mlp = _timeit(lambda: net.shade(pos, nrm, cams, mu, sg, isel, lit, 3, strides, R4), 5, flush, stream)
            mlp_flops = 2.0 * V * S * (320 * 256 + 3 * 256 * 256 + 256 * 3)
            rows["c4_surrogate"] = {"what": "c4 frame: 32 rotations + surrogate transport (4x256 GELU MLP, bf16 tcgen05) "
                                            "fused with shading",
                                    "frame_ms": ms_frame, "value": V * S / ms_frame / 1e3, "unit": UNIT,
                                    "kernel": "haar_mlp_shade", "kernel_ms": ms_mlp,
                                    "achieved_tflops": mlp_flops / ms_mlp / 1e9,
                                    "frac_tensor": mlp_flops / ms_mlp / 1e9 / bf16_peak,
                                    "vs_plain_c3_frame": (V * S / ms_frame / 1e3) / plain_c3,
                                    "weights": "random init (throughput only)"}
        if want("surrogate_training"):
            # S8: one Adam training step on a batch of 8192
            B = 8192
            raw = torch.randn((B, 9), dtype=torch.float32, device=dev)
            tgt = torch.randn((B, 512), dtype=torch.float32, device=dev)
            ms_eager = _timeit(lambda: net.train_step(raw, tgt, 1e-4), 10, flush, stream)
            graph, _ = net.capture_train_step(raw, tgt, 1e-4)
            ms_train = _timeit(graph.replay, 10, flush, stream)
            tflops = 3.0 * 2.0 * B * (320 * 256 + 3 * 256 * 256 + 256 * 512) / ms_train / 1e9
            rows["surrogate_training"] = {"what": "haar_mlp_train_step, batch 8192 (forward, backward, Adam), "
                                                  "replayed from a CUDA graph",
                                          "ms": ms_train, "eager_ms": ms_eager, "samples_per_s": B / ms_train * 1e3,
                                          "achieved_tflops": tflops, "frac_tensor": tflops / bf16_peak}
        net.close()
    if c3:
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

    if args.only:
        flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
        print(json.dumps({"rows": measure_rows(hs, dev, flush, set(args.only.split(",")))}), flush=True)
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

    # per-kernel durations for the roofline (same stream, same flush discipline)
    shade_ms = timed(lambda: hs.shade_vertices(plan, tr, wl["lighting"], wl["S"], wl["radiance"]), args.steps)
    shift_ms = timed(lambda: hs.haar_shift(plan, wl["L"], wl["params"], wl["lighting"]), args.steps)
    shade_avg, shift_avg = statistics.mean(shade_ms), statistics.mean(shift_ms)
    ab = algorithmic_bytes(wl)
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    hbm = peaks.get("hbm_gbs", 6800.0)
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
    csr_ms = timed(lambda: hs.shade_vertices(plan, wl["csr"], wl["lighting"], wl["S"], wl["radiance"]), args.steps)
    csr_avg = statistics.mean(csr_ms)
    if shade_avg >= shift_avg:
        kname, kms = "k_shade_gcsr_f32", shade_avg
    else:
        kname, kms = "k_shift", shift_avg
    achieved = ab[kname] / (kms * 1e-3) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                "traffic": traffic_record(kname), "kernel": kname, "peak_source": peak_src,
                "algorithmic_bytes": ab[kname], "kernel_ms": kms,
                "other_kernels_ms": {"k_setup+k_shift": shift_avg, "k_shade_gcsr_f32": shade_avg},
                "plain_csr_kernel": {"kernel": "k_shade_csr_f32", "ms": csr_avg,
                                     "achieved_gbs": ab["k_shade_csr_f32"] / (csr_avg * 1e-3) / 1e9}}
    if kname == "k_shade_gcsr_f32":
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

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": WORKLOAD, "H": wl["H"], "W": wl["W"], "channels": wl["C"],
                           "shifts_per_step": wl["S"], "vertices_per_gpu": wl["V"], "topk": wl["K"],
                           "l2": "flushed between timed steps (256 MiB write)",
                           "parallelism": f"{world} independent vertex shards (no collective)"},
                "roofline": roofline, "cpu_baseline": cpu,
                "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                        "d2h": "radiance written by the shading kernel into pinned host memory"},
                "gpu_launches": 3 * args.steps, "clocks": clk, "rows": rows}
        print(json.dumps(line), flush=True)
    plan.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
