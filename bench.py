"""Shadow-ray throughput of the NIF query vs the exact BVH cast on one GB300.

Workload (default, --workload full): 480 displaced icospheres of 62,720
triangles (30.1M) on a jittered lattice in a 12-triangle room, 1920x1080
pixel-centre primary hits, a 4 x 4 ceiling area light sampled 4 times per
pixel -> 8,294,400 shadow rays; dense 8-level x 2-feature FP16 grids (R 4..64)
per object, shared outer/inner 3x64 networks in FP16 on the tensor cores,
trained online on 64 shadow samples per pixel before timing (FP16 forward and
backward on the tensor cores with FP32 masters and a dynamic loss scale;
--train-precision f32 trains in FP32 on the CUDA cores).  --workload room
is the 1.0M-triangle scene with hashed 16-level grids and one point light
(2,073,600 shadow rays); the other workloads are listed in WORKLOADS.

One step = one full visibility query of all shadow rays: exact cast of the
non-NIF geometry (the room), the top-level front end (pairs binned by
network) and the fused encode + MLP + visibility kernel.  The exact BVH cast
of the same rays is timed the same way for comparison.  Inputs are resident
in HBM; L2 is flushed (256 MB write) before every timed step.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

SCHED_NAME = {0: "auto", 1: "serial", 2: "pipelined"}
METRIC = "shadow rays/sec NIF vs own GPU BVH at <=1% visibility error; tensor-pipe util"
UNIT = "shadow rays/s"
WORKLOADS = {
    "paper": ("paper's encoding on the room scene: 64 displaced icospheres (1,003,520 tris) + 12-tri "
              "room, 1920x1080 primary hits, 1 point light -> 2,073,600 shadow rays; per object spherical "
              "2D grids (outer R 256 N 3; inner R 128 N 5 + 1D R 128 N 3) FP16; outer 2x64 and inner "
              "3x48 leaky-ReLU networks (inner padded to 64 for the tensor cores), trained 64 Adam "
              "steps x 262,144 pairs"),
    "room": ("room: 64 displaced icospheres (1,003,520 tris) + 12-tri room, 1920x1080 primary hits, "
             "1 point light -> 2,073,600 shadow rays; hashed 16x2 FP16 grids (2^19/level) per object; "
             "shared outer/inner MLP 3x64 FP16 trained 64 Adam steps x 262,144 pairs"),
    "full": ("full scale: 480 displaced icospheres x 62,720 tris (30.1M) on a jittered lattice + room, "
             "1920x1080 primary hits, 4x4 area light x 4 samples -> 8,294,400 shadow rays; dense 8x2 "
             "FP16 grids (R 4..64) per object; outer/inner MLP 3x64 FP16 trained on 64 shadow "
             "samples/pixel"),
    "grouped": ("grouped per-object networks: 32 displaced icospheres with 10k-500k tris (log-uniform), "
                "rays aimed at each object's box, power-law (alpha 1.5) pair counts totalling 8M; one "
                "3x64 FP16 network and dense 8x2 FP16 grid per object; one persistent grouped launch "
                "replayed from a CUDA graph"),
    "mixed": ("mixed NIF/BVH scene: 32 displaced icospheres (radius 1.5) with 10k-500k tris "
              "(log-uniform) + 12-tri room, 1920x1080 primary hits, 1 point light -> 2,073,600 shadow "
              "rays; NIF (hashed 16x2 FP16 grids, 3x64 FP16 networks, trained 64 Adam steps x 262,144 "
              "pairs) only for objects above 100k tris, the exact BVH for the rest and the room; "
              "compared with the exact BVH over every triangle"),
    "primary": ("primary rays (NIF outputs occupancy, shading normal and depth, Sec. 6.1): the room "
                "scene (64 displaced icospheres, 1,003,520 tris, + 12-tri room), 1920x1080 pixel-centre "
                "camera rays -> 2,073,600 primary rays; hashed 16x2 FP16 grids per object, outer/inner 3x64 "
                "FP16 networks with 5 outputs trained 64 Adam steps x 262,144 pairs from 4 jittered "
                "samples per pixel; compared with the exact closest-hit BVH cast over every triangle"),
    "render": ("direct-lighting frame (Sec. 5, Sec. 6.2): the room scene (64 displaced icospheres + room) "
               "under 8 ceiling quad lights (fluxes over 200x), 1920x1080 primary hits, 4 light samples per "
               "pixel picked by flux from a tabulated CDF -> 8,294,400 shadow rays; the paper's encoding and "
               "networks (FP16), trained on 4 jittered samples per pixel with importance-sampled lights; one "
               "step = primary cast, light sampling, shadow query, shading"),
    "mlp": ("the inference stage alone (nif_mlp_infer, the tcgen05 MLP over encoded inputs): 1,048,576 "
            "rows of synthetic FP16 inputs, U(-1, 1), in two groups (2/3 outer, 1/3 inner), class networks "
            "3x64 FP16 with Xavier weights; shapes K = 96 (the room's hashed 16x2 encoding) and K = 48 "
            "(the full-scale 8x2 encoding); L2 flushed before every launch"),
    "mma": ("the tensor-core instruction rate (nif_tc_mma_rate): SM cycles per tcgen05.mma (kind::f16, "
            "K = 16, one CTA per SM on every SM, zero operands) at the shapes the MLP kernels issue "
            "(M = 128 x N = 64, M = 64 x N = 256) and at the widest (M = 128 x N = 256); 64 back-to-back "
            "MMAs per commit, and 4 per commit as in a hidden layer"),
    "precision": ("precision sweep: small-configuration object (20,480 tris) in the room, 4 point "
                  "lights -> 8,294,400 shadow rays; dense 8x2 FP32 grids (R 4..64), MLP 3x64 trained "
                  "in FP32, inferred in FP32 / BF16 / FP16 / FP8-E4M3"),
}


# DRAM bytes (read + write) of one step's fused-kernel launches, from the ncu
# captures summarised under profiles/, keyed by (workload, schedule, CTAs per
# SM, round-1 rule) of the kernel as it stands; a configuration without an
# entry reports null.
FUSED_TRAFFIC_BYTES = {
    ("full", "pipelined", 0, "nearest"): 761_019_136,   # fused_ws_full_dram.md
    ("room", "serial", 4, "outer"): 1_720_619_776,      # fused_tm_room_dram.md
}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), float(p["bf16_tflops"]), "measured"
    except Exception:
        return 6800.0, 1900.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
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
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def reduce_max(x: float, world: int, device) -> float:
    """Max of a per-rank value over all ranks (the slowest replica's time)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ---------------------------------------------------------------- oracle arm
class OracleFrame:
    """The CPU oracle's own view of a workload's evaluation frame: the scene
    from the seeded generator, the oracle's BVH over it, and the FP64 oracle
    model with the seeded initial latents and weights.  Imports only the
    oracle and the seeded input generators (no CUDA library)."""

    def __init__(self, name: str):
        import numpy as np

        import oracle
        from oracle import nif as onif
        from paper_2306_07191_gb300 import synth, workloads

        f = workloads.FRAMES[name]
        self.f = f
        self.ws = workloads.room_scene(f.n_obj, f.n, f.width, f.height, f.seed, layout=f.layout)
        sc = self.ws.scene
        self.bvh = oracle.OracleBVH(sc.verts, sc.tris)
        npix = self.ws.camera.shape[0]
        self.light = (workloads.area_light_samples(np.random.default_rng(workloads.EVAL_LIGHT_SEED), npix,
                                                   f.samples).reshape(npix, f.samples, 3)
                      if f.area_light else None)
        _, _, off = onif.level_layout(list(f.res), f.log2_table)
        V = int(off[-1])
        rng = np.random.default_rng(f.seed + 101)
        nets = [[np.asarray(w, np.float64) for w in synth.mlp_init(rng, f.K, f.width_mlp, f.n_hidden)]
                for _ in range(2)]
        self.model = onif.Model(res=list(f.res), F=f.n_features, log2_table=f.log2_table,
                                obj_aabb=sc.obj_aabb,
                                grids=synth.SplitMixGrids(V * f.n_features, workloads.GRID_SEED,
                                                          workloads.GRID_SCALE),
                                nets=nets, net_mode="class")

    def rays(self, n_pixels: int | None = None, seed: int = 5):
        """Shadow rays of n_pixels sampled pixels (all if None), derived by
        the oracle from the camera rays, its own closest hits and the light."""
        import numpy as np

        from oracle import frames
        npix = self.ws.camera.shape[0]
        pix = (np.arange(npix) if n_pixels is None else
               np.sort(np.random.default_rng(seed).choice(npix, n_pixels, replace=False)))
        pts = self.light[pix].reshape(-1, 3) if self.light is not None else self.ws.light
        return frames.frame_rays(self.bvh, self.ws.camera[pix], pts, self.f.tmin, self.f.samples)


# pixels of the CPU-baseline sample (x the workload's shadow rays per pixel)
CPU_BASELINE_PIXELS = {"room": 1 << 20, "full": 1 << 19}
# pixels per step of the reference arm
REFERENCE_PIXELS = {"room": 1 << 18, "full": 1 << 16}


def cpu_baseline(name: str):
    """The FP64 oracle's visibility query (box tests, encoding, MLP,
    threshold) timed on a sample of the workload's frame, on every host core
    (one worker process per core, chunks of rays)."""
    from oracle import frames
    npix = CPU_BASELINE_PIXELS[name]
    fr = OracleFrame(name)
    rays = fr.rays(npix)
    pool = frames.QueryPool(fr.model)
    try:
        v, dt, nq, _ = pool.timed_query(rays)
    finally:
        pool.close()
    return {"value": v, "unit": UNIT, "cores": pool.processes, "kind": "oracle",
            "sample": f"{rays.shape[0]} shadow rays of {npix} sampled pixels of the {name} frame "
                      f"({nq} pairs), FP64 NIF query on the initial latents, {pool.processes} worker "
                      f"processes, {dt:.1f} s"}


def run_reference(args):
    """The oracle arm: the FP64 CPU oracle's query of a bounded sample of
    the same workload per step, on every host core."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    from oracle import frames
    from paper_2306_07191_gb300 import workloads
    name = args.workload if args.workload in workloads.FRAMES else "full"
    f = workloads.FRAMES[name]
    npix = REFERENCE_PIXELS[name]
    fr = OracleFrame(name)
    pool = frames.QueryPool(fr.model)
    times = []
    n = 0
    try:
        for s in range(args.warmup + args.steps):
            rays = fr.rays(npix, seed=100 + s)
            n = int(rays.shape[0])
            _, dt, _, _ = pool.timed_query(rays)
            if s >= args.warmup:
                times.append(dt)
    finally:
        pool.close()
    med = statistics.median(times)
    val = n / med
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": med * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOADS[name], "rays": f.width * f.height * f.samples,
                       "sample_rays_per_step": n},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": pool.processes, "kind": "oracle",
                             "sample": f"{n} shadow rays of {npix} sampled pixels per step, FP64 oracle "
                                       f"NIF query, {pool.processes} worker processes"},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- our arm
def precision_sweep(pipe, log, steps: int = 10, warmup: int = 3):
    """The trained FP32 network inferred with FP32 / BF16 / FP16 / FP8-E4M3
    operands (FP32 accumulation): time per query of all shadow rays,
    disagreement with BVH truth and with the FP32 decisions."""
    import statistics as st

    import torch

    from paper_2306_07191_gb300 import _lib as L
    from paper_2306_07191_gb300 import nif

    model = pipe.model
    n = pipe.n_rays
    ref = nif.empty_bits(n)
    pipe.bvh_query(ref)
    truth = nif.bits_to_bool(ref, n)
    q8, sc8 = pipe.calibrate_e4m3(pipe.pairs)
    w32 = pipe.trainer.w_master.clone()
    variants = [("f32", L.NIF_F32, w32, None), ("bf16", L.NIF_BF16, w32.bfloat16(), None),
                ("f16", L.NIF_F16, w32.half(), None), ("e4m3", L.NIF_E4M3, q8, sc8)]
    out = {}
    dec32 = None
    saved = (model.cfg.mlp_dtype, model.weights, model.scales)
    for name, dt, w, sc in variants:
        model.cfg.mlp_dtype, model.weights, model.scales = dt, w.contiguous(), sc
        bits = nif.empty_bits(n)
        pipe.nif_query(bits)
        torch.cuda.synchronize()
        dec = nif.bits_to_bool(bits, n)
        if dec32 is None:
            dec32 = dec
        times = []
        for i in range(warmup + steps):
            bits.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            pipe.nif_query(bits)
            e1.record()
            torch.cuda.synchronize()
            if i >= warmup:
                times.append(e0.elapsed_time(e1))
        ms = st.median(times)
        out[name] = {"ms_per_query": ms, "rays_per_s": n / (ms * 1e-3),
                     "disagreement_vs_bvh": float((dec != truth).float().mean()),
                     "disagreement_vs_f32": float((dec != dec32).float().mean())}
        log(f"precision {name}: {out[name]}")
    model.cfg.mlp_dtype, model.weights, model.scales = saved
    return out


def mlp_alone_stats(pipe, bits, steps: int, warmup: int, flush):
    """Time nif_mlp_infer (the tcgen05 MLP over encoded FP16 inputs) on the
    frame's round-1 pairs; returns its tensor-pipe rate or None when the
    model is not an FP16 width-64 network over 16-bit-aligned inputs."""
    import ctypes

    import torch

    from paper_2306_07191_gb300 import _lib as L
    from paper_2306_07191_gb300 import nif
    model = pipe.front_model()
    c = model.cfg
    if (c.mlp_dtype != L.NIF_F16 or c.width != 64 or model.n_nets > 2 or c.K % 8 != 0
            or c.encoding != L.NIF_ENC_MULTIRES):
        return None
    b = pipe._query_buffers()
    pipe.query_step(bits)
    torch.cuda.synchronize()
    nq = int(b["count"][0].item())
    x = model.encode(pipe.rays, b["ray_id"], b["qobj"], nq, dtype=L.NIF_F16)
    goff = b["goff1"].clone()
    z = torch.empty(nq, dtype=torch.float32, device=x.device)
    ws = torch.zeros(256, dtype=torch.uint8, device=x.device)
    d = model.desc()
    vp = ctypes.c_void_p

    def run():
        L.call("nif_mlp_infer", ctypes.byref(d), vp(x.data_ptr()), vp(goff.data_ptr()), nq, vp(z.data_ptr()),
               vp(ws.data_ptr()), ws.numel(), nif._stream())

    out = {"rows": nq, "K": c.K, "input_bytes": nq * c.K * 2, "per_tile_m": {}}
    _, bf16_peak, src = _peaks()
    flops = nq * 2 * (c.K * 64 + (c.n_hidden - 1) * 64 * 64 + 64)
    # both tile shapes of nif_mlp_infer: 256 rows as the MMA's N, 128 rows as its M
    for tile_m in (256, 128):
        d.tile_m = tile_m
        res = {}
        for mode in ("hbm", "l2"):
            ts = []
            for i in range(warmup + steps):
                if mode == "hbm":
                    flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                run()
                e1.record()
                torch.cuda.synchronize()
                if i >= warmup:
                    ts.append(e0.elapsed_time(e1))
            ms = statistics.median(ts)
            tf = flops / (ms * 1e-3) / 1e12
            res[mode] = {"ms": ms, "tensor_tflops": tf, "tensor_frac": tf / bf16_peak,
                         "input_gbs": nq * c.K * 2 / (ms * 1e-3) / 1e9}
        out["per_tile_m"][tile_m] = res
    best = min(out["per_tile_m"], key=lambda m: out["per_tile_m"][m]["hbm"]["ms"])
    out["tile_m"] = best
    out["hbm"], out["l2"] = out["per_tile_m"][best]["hbm"], out["per_tile_m"][best]["l2"]
    out["tensor_peak_tflops"] = bf16_peak
    out["peak_source"] = src
    model.check(ws)
    return out


def run_mlp(args):
    """The inference stage alone on synthetic encoded inputs: nif_mlp_infer's
    rows per second and tensor-pipe rate for the room-shaped (K = 96) and the
    full-scale-shaped (K = 48) network inputs, with L2 flushed before every
    launch (inputs from HBM).  The timed launches are the only ones inside
    the profiler range, so an ncu capture with --profile-from-start off sees
    only them."""
    import ctypes

    import numpy as np
    import torch

    from paper_2306_07191_gb300 import _lib as L
    from paper_2306_07191_gb300 import nif, synth, workloads
    world, rank, local = dist_env()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    rows = (1 << 17) if args.small else (1 << 20)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    _, bf16_peak, src = _peaks()
    vp = ctypes.c_void_p
    shapes = {}
    gpu_warm(flush)
    with ClockSampler(local) as clk:
        for name, res in (("room K=96", workloads.ROOM_RES), ("full K=48", workloads.TINY_RES)):
            rng = np.random.default_rng(len(res))
            cfg = nif.NifConfig(res=list(res), n_features=2, log2_table=19, grid_dtype=L.NIF_F16, n_hidden=3,
                                width=64, mlp_dtype=L.NIF_F16, net_mode=L.NIF_NETS_CLASS)
            K = cfg.K
            flat = np.concatenate([synth.flatten_mlp(synth.mlp_init(rng, K, 64, 3)) for _ in range(2)])
            V = nif.NifModel.grid_vertices(cfg)
            model = nif.NifModel(cfg, torch.zeros((1, 6), device=dev),
                                 torch.zeros(2 * V * 2, dtype=torch.float16, device=dev),
                                 torch.from_numpy(flat).half().to(dev))
            x = torch.from_numpy(rng.uniform(-1, 1, size=(rows, K)).astype(np.float16)).to(dev)
            goff = torch.tensor([0, 2 * rows // 3, rows], dtype=torch.int64, device=dev)
            ws = torch.zeros(256, dtype=torch.uint8, device=dev)
            st = nif._stream()
            stream = torch.cuda.current_stream(dev)
            flops = rows * 2 * (K * 64 + 2 * 64 * 64 + 64)
            per_tile = {}
            outs = {}
            # both tile shapes: 128 rows as the MMA's M, 256 rows as its N
            for tile_m in (256, 128):
                model.cfg.tile_m = tile_m
                d = model.desc()
                z = torch.empty(rows, dtype=torch.float32, device=dev)

                def run():
                    L.call("nif_mlp_infer", ctypes.byref(d), vp(x.data_ptr()), vp(goff.data_ptr()), rows,
                           vp(z.data_ptr()), vp(ws.data_ptr()), ws.numel(), st)

                for _ in range(args.warmup):
                    flush.zero_()
                    run()
                torch.cuda.synchronize()
                ts = []
                torch.cuda.profiler.start()
                for _ in range(args.steps):
                    flush.zero_()
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    run()
                    e1.record(stream)
                    ts.append((e0, e1))
                torch.cuda.profiler.stop()
                torch.cuda.synchronize()
                model.check(ws)
                assert torch.isfinite(z).all()
                ms = statistics.median(a.elapsed_time(b) for a, b in ts)
                tf = flops / (ms * 1e-3) / 1e12
                per_tile[tile_m] = {"ms": ms, "rows_per_s": rows / (ms * 1e-3), "tensor_tflops": tf,
                                    "tensor_frac": tf / bf16_peak}
                outs[tile_m] = z
            # the two tile shapes round the last hidden layer differently
            # (FP32 dot, or FP16 operands of one more MMA): logits agree to
            # the FP16 rounding of that layer
            diff = float((outs[128] - outs[256]).abs().max())
            best = min(per_tile, key=lambda m: per_tile[m]["ms"])
            ms = per_tile[best]["ms"]
            tf = flops / (ms * 1e-3) / 1e12
            shapes[name] = {"K": K, "ms": ms, "rows_per_s": rows / (ms * 1e-3), "tensor_tflops": tf,
                            "tensor_frac": tf / bf16_peak, "input_gbs": rows * K * 2 / (ms * 1e-3) / 1e9,
                            "flops_per_row": flops // rows, "tile_m": best, "per_tile_m": per_tile,
                            "max_logit_diff_between_tiles": diff}
    clocks = clk.summary()
    head = shapes["room K=96"]
    line = {
        "metric": "MLP rows/s, inference stage alone (tcgen05); tensor-pipe util", "value": head["rows_per_s"],
        "unit": "rows/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": head["ms"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f16", "data": "synthetic",
        "config": {"workload": WORKLOADS["mlp"], "rows": rows, "l2": "flushed (256 MB write) before every launch",
                   "parallelism": "single GPU"},
        "shapes": shapes,
        "roofline": {"kernel": ("k_mlp_rows" if head["tile_m"] == 256 else "k_mlp_pipe") + " (room K=96)", "bound": "tensor", "achieved": head["tensor_tflops"],
                     "peak": bf16_peak, "unit": "TFLOP/s", "frac": head["tensor_frac"], "traffic": None,
                     "peak_source": src},
        "gpu_launches": 4 * args.steps,
        "clocks": clocks,
        "cpu_baseline": None,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


def gpu_warm(buf, seconds: float = 0.5):
    """Keep the GPU busy for a moment before a short timed run, so that its
    memory and SM clocks have left their idle states (the MLP and rate
    workloads time a few milliseconds in all)."""
    import time

    import torch
    t0 = time.time()
    while time.time() - t0 < seconds:
        for _ in range(20):
            buf.zero_()
        torch.cuda.synchronize()


def run_mma(args):
    """SM cycles per tcgen05.mma at the MLP kernels' shapes (nif_tc_mma_rate)
    and the tensor-pipe rate each implies at the sampled SM clock against the
    measured bf16 peak: the ceiling of an MLP kernel that issues MMAs of that
    shape back to back."""
    import ctypes

    import torch

    from paper_2306_07191_gb300 import _lib as L
    from paper_2306_07191_gb300 import nif
    world, rank, local = dist_env()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    _, bf16_peak, src = _peaks()
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    ws = torch.zeros(256, dtype=torch.uint8, device=dev)
    vp = ctypes.c_void_p
    gpu_warm(torch.empty(256 << 20, dtype=torch.uint8, device=dev))
    # (M, N, A in TMEM, CTAs per SM)
    shapes = [(128, 64, 0, 1), (128, 64, 1, 1), (64, 256, 0, 1), (128, 128, 0, 1), (128, 256, 0, 1),
              (128, 256, 1, 1), (128, 64, 0, 2), (128, 64, 1, 2), (128, 128, 0, 2)]
    cyc = torch.zeros(2 * n_sm, dtype=torch.int64, device=dev)
    rows = []
    with ClockSampler(local) as clk:
        for _ in range(max(1, args.steps // 5)):
            for m, n, a_tmem, per_sm in shapes:
                for chain, reps in ((64, 40), (4, 400)):
                    nc = per_sm * n_sm
                    L.call("nif_tc_mma_rate", m, n, a_tmem, chain, reps, nc, vp(cyc.data_ptr()), vp(ws.data_ptr()),
                           ws.numel(), nif._stream())
                    torch.cuda.synchronize()
                    c = cyc[:nc].double()
                    assert bool((c > 0).all()), "an MMA wait timed out"
                    # cycles per MMA of one SM: each CTA's own rate divided by the CTAs sharing the SM
                    rows.append((m, n, a_tmem, per_sm, chain, float(c.mean()) / (reps * chain) / per_sm))
    clocks = clk.summary()
    det = ctypes.c_int64()
    L.call("nif_check", vp(ws.data_ptr()), ctypes.byref(det), nif._stream())
    mhz = clocks.get("sm_mhz") or 2070.0
    out = {}
    for m, n, a_tmem, per_sm, chain, per in rows:
        key = f"M{m}xN{n}" + ("_A_tmem" if a_tmem else "") + (f"_{per_sm}cta_per_sm" if per_sm > 1 else "") + \
            f"_chain{chain}"
        out.setdefault(key, []).append(per)
    table = {}
    for key, v in out.items():
        per = statistics.median(v)
        m = int(key.split("x")[0][1:])
        n = int(key.split("N")[1].split("_")[0])
        fma_clk = m * n * 16 / per
        tf = 2 * fma_clk * n_sm * mhz * 1e6 / 1e12
        table[key] = {"cycles_per_mma": per, "fma_per_clk_per_sm": fma_clk, "tflops_at_clock": tf,
                      "frac_of_bf16_peak": tf / bf16_peak}
    head = table["M128xN64_chain64"]
    line = {
        "metric": "SM cycles per tcgen05.mma (kind::f16) at the MLP's shape", "value": head["cycles_per_mma"],
        "unit": "cycles", "n_gpus": 1, "steps": args.steps, "warmup": 0, "ms_per_step": None,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f16", "data": "synthetic",
        "config": {"workload": WORKLOADS["mma"], "ctas": n_sm, "sm_mhz_for_rates": mhz, "parallelism": "single GPU"},
        "shapes": table, "tensor_peak_tflops": bf16_peak, "peak_source": src,
        "gpu_launches": len(rows), "clocks": clocks, "cpu_baseline": None,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


def r_sweep(log, steps: int = 5, warmup: int = 3):
    """The paper's resolution sweep (Fig. 4: outer grid R = 64 / 256 / 1024)
    on the paper-encoding workload: per R a freshly trained pipeline, its
    visibility disagreement with the BVH and the device time of the query
    step (L2 flushed before each)."""
    import statistics

    import torch

    from paper_2306_07191_gb300 import nif
    from paper_2306_07191_gb300.pipeline import PaperEncodingConfig, PaperEncodingPipeline
    out = {}
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    for R in (64, 256, 1024):
        pipe = PaperEncodingPipeline(PaperEncodingConfig(outer_res=R), log=log)
        train_s = pipe.train()
        dis = pipe.disagreement()
        pipe.release_training_state()
        for m, _ in pipe.forward_models():
            m.cfg.ctas_per_sm, m.cfg.schedule = 4, 1
        bits = nif.empty_bits(pipe.n_rays)
        ts = []
        for k in range(warmup + steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            pipe.query_step(bits)
            e1.record()
            torch.cuda.synchronize()
            if k >= warmup:
                ts.append(e0.elapsed_time(e1))
        pipe.check()
        ms = statistics.median(ts)
        out[R] = {"ms_per_step": ms, "rays_per_s": pipe.n_rays / (ms * 1e-3),
                  "disagreement": dis["all"], "disagreement_queried": dis["queried"],
                  "outer_grid_latents": int(pipe.cls["outer"]["model"].grids.numel()), "train_s": train_s}
        log(f"R {R}: {out[R]}")
        del pipe
        torch.cuda.empty_cache()
    return out


def run_ours(args):
    import ctypes

    import torch
    import torch.distributed as dist

    from paper_2306_07191_gb300 import _lib as L
    from paper_2306_07191_gb300 import nif
    from paper_2306_07191_gb300.pipeline import RoomConfig, RoomPipeline

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    log = (lambda *a: print(*a, file=sys.stderr, flush=True)) if rank == 0 else (lambda *a: None)
    from paper_2306_07191_gb300.pipeline import (PaperEncodingConfig, PaperEncodingPipeline,
                                                 full_scale_config, mixed_scene_config,
                                                 small_object_precision_config)
    pipe_cls = RoomPipeline
    if args.workload == "paper":
        cfg = PaperEncodingConfig()
        pipe_cls = PaperEncodingPipeline
    elif args.workload == "full":
        cfg = full_scale_config()
    elif args.workload == "precision":
        cfg = small_object_precision_config()
    elif args.workload == "mixed":
        cfg = mixed_scene_config()
    else:
        cfg = RoomConfig()
    if args.small:
        cfg.width, cfg.height, cfg.train_steps, cfg.batch = 640, 360, 8, 65536
        cfg.train_spp = min(cfg.train_spp, 2)
        if cfg.layout == "random":
            cfg.n_obj = 16
    if args.ctas_per_sm:
        cfg.ctas_per_sm = args.ctas_per_sm
        cfg.schedule = L.NIF_SCHED_SERIAL
    if args.schedule:
        cfg.schedule = {"serial": L.NIF_SCHED_SERIAL, "pipelined": L.NIF_SCHED_PIPELINED}[args.schedule]
    if args.exact_cast:
        cfg.exact_cast = args.exact_cast
    if args.tlas:
        cfg.tlas_builder = args.tlas
    # half-precision training needs a 16-bit network over the multi-resolution
    # encoding (the precision sweep trains its FP32 network in FP32 and
    # quantises it afterwards; the paper's spherical encoding trains in FP32)
    if (args.train_precision == "f16" and pipe_cls is RoomPipeline
            and cfg.mlp_dtype in (L.NIF_F16, L.NIF_BF16)):
        cfg.half_precision_train = True
    pipe = pipe_cls(cfg, log=log)
    train_s = pipe.train()
    n_par = pipe.param_count()
    tms = sorted(pipe.train_step_ms[1:]) or pipe.train_step_ms
    train_stats = {
        "steps": len(pipe.train_step_ms), "batch_pairs": min(cfg.batch, int(pipe.pairs[1].shape[0])),
        "gpu_ms_per_step_median": tms[len(tms) // 2], "params": n_par,
        # dense Adam reads master, grad, m, v and writes master, m, v, the
        # 16-bit copy and the zeroed grad: 34 B per parameter per step
        "adam_bytes_per_step": 34 * n_par,
        "adam_floor_ms": 34 * n_par / (_peaks()[0] * 1e9) * 1e3,
        "wall_includes": "host-side batch draw (numpy) and copies",
        "precision": "f16" if getattr(cfg, "half_precision_train", False) else "f32",
        # batch loss every 8 steps and at the last one
        "loss_curve": [round(v, 6) for v in pipe.losses[::8] + pipe.losses[-1:]]}
    dis = pipe.disagreement()
    abl = pipe.ablations()
    log(f"disagreement {dis}  ablations {abl}")
    sweep = None
    if args.workload == "precision":
        sweep = precision_sweep(pipe, log)
    pipe.release_training_state()
    torch.cuda.empty_cache()
    tune_ms = None
    if not (args.ctas_per_sm or args.schedule) and pipe.model.cfg.mlp_dtype != L.NIF_F32:
        tbits = nif.empty_bits(pipe.n_rays)
        fwd = [m for m, _ in pipe.forward_models()]
        # the spherical encodings run the serial schedule only
        cands = nif.SCHEDULE_CANDIDATES if args.workload != "paper" else \
            tuple(c for c in nif.SCHEDULE_CANDIDATES if c[0] == L.NIF_SCHED_SERIAL)
        sched, occ, tune_ms = nif.autotune(fwd[0], lambda: pipe.query_step(tbits), also=fwd[1:],
                                           candidates=cands, key_extra=(pipe.n_rays, args.workload))
        log(f"autotuned fused kernel: schedule {sched}, {occ} CTAs/SM ({tune_ms})")
    # the round-1 rule that queries fewer pairs on this frame
    round1_pairs = pipe.tune_round1()
    from paper_2306_07191_gb300.pipeline import ROUND1_NAME
    round1 = ROUND1_NAME[pipe.front_model().cfg.round1]
    log(f"round 1 takes each ray's {round1} pair ({round1_pairs})")
    n = pipe.n_rays
    rays = pipe.rays
    model = pipe.model
    dev = rays.device
    stream = torch.cuda.current_stream()
    # explicit sub-steps so CUDA events bracket each kernel group
    max_q = cfg.max_pairs_per_ray * n + 1024
    ws = model.workspace(max_q, n)
    ray_id = torch.empty(max_q, dtype=torch.int32, device=dev)
    qobj = torch.empty(max_q, dtype=torch.int32, device=dev)
    count = torch.empty(2, dtype=torch.int64, device=dev)
    goff1 = torch.empty(model.n_nets + 1, dtype=torch.int64, device=dev)
    bits = nif.empty_bits(n, dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    sp = nif._stream()
    vp = ctypes.c_void_p

    def nif_step(ev=None):
        # the calls nif_infer makes, with events between them: nearest pair
        # per ray, its forward, the other pairs of still-unoccluded rays, theirs
        pipe.query_step(bits, ev=ev)

    def timed(fn, K, W, sub=False):
        for _ in range(W):
            flush.zero_()
            fn()
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        tot, parts = [], []
        for _ in range(K):
            flush.zero_()
            e = [torch.cuda.Event(enable_timing=True) for _ in range(7)]
            e[0].record(stream)
            if sub:
                fn(e[1:6])
            else:
                fn()
            e[6].record(stream)
            parts.append(e)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        for e in parts:
            tot.append(e[0].elapsed_time(e[6]))
        subs = None
        if sub:
            def m(a, b):
                return statistics.median(e[a].elapsed_time(e[b]) for e in parts)
            subs = {"room_cast_ms": m(0, 1), "frontend_nearest_ms": m(1, 2), "fused_round1_ms": m(2, 3),
                    "frontend_rest_ms": m(3, 4), "fused_round2_ms": m(4, 5)}
            if cfg.exact_cast == "after":
                # the first interval clears the mask; the exact cast follows
                # the round-2 forward
                subs["mask_clear_ms"] = m(0, 1)
                subs["room_cast_ms"] = m(5, 6)
            elif cfg.exact_cast == "overlap":
                # the exact cast runs beside the NIF calls on a second
                # stream; the last interval is the wait for it
                subs["mask_clear_ms"] = subs.pop("room_cast_ms")
                subs["exact_join_ms"] = m(5, 6)
            subs["frontend_ms"] = subs["frontend_nearest_ms"] + subs["frontend_rest_ms"]
            subs["fused_ms"] = subs["fused_round1_ms"] + subs["fused_round2_ms"]
        return tot, subs

    # the whole step captured once in a CUDA graph and replayed: no host
    # launch overhead between its kernels (the stage split comes from an
    # eager run with events between the calls)
    graphs = {}

    def capture(fn):
        g = torch.cuda.CUDAGraph()
        gs = torch.cuda.Stream()
        gs.wait_stream(stream)
        with torch.cuda.stream(gs):
            fn()
            torch.cuda.synchronize()
            with torch.cuda.graph(g, stream=gs):
                fn()
        stream.wait_stream(gs)
        torch.cuda.synchronize()
        return g

    # the comparison trees over every triangle: the LBVH the pipeline built
    # and a PLOC tree (locally-ordered clustering, lower surface-area cost),
    # built untimed; the NIF step is compared with the faster cast
    trees = {"lbvh": pipe.bvh, "ploc": nif.BVH(pipe.verts, pipe.tris, pipe.tags, builder="ploc")}
    if not args.no_graph:
        graphs["nif"] = capture(nif_step)
        for name, tree in trees.items():
            graphs[name] = capture(lambda t=tree: t.cast_shadow(rays, out=bits))
    with ClockSampler(local) as clk:
        torch.cuda.profiler.start()
        eager_ms, subs = timed(nif_step, args.steps, args.warmup, sub=True)
        nif_ms = timed(graphs["nif"].replay, args.steps, args.warmup)[0] if graphs else eager_ms
        tree_ms = {name: timed(graphs[name].replay if graphs else (lambda t=tree: t.cast_shadow(rays, out=bits)),
                               args.steps, args.warmup)[0] for name, tree in trees.items()}
        torch.cuda.profiler.stop()
    tree_med = {name: statistics.median(v) for name, v in tree_ms.items()}
    best_tree = min(tree_med, key=tree_med.get)
    bvh_ms = tree_ms[best_tree]
    tree_stats = {}
    for name, tree in trees.items():
        st_ = tree.stats(rays)
        st_["ms_per_step"] = reduce_max(tree_med[name], world, dev)
        st_["rays_per_s"] = world * n / (st_["ms_per_step"] * 1e-3)
        tree_stats[name] = st_
        tree.check()
    log(f"comparison trees: {tree_stats}")
    clocks = clk.summary()
    nq1, nq = pipe.last_query_counts()
    pipe.check()
    # pairs of the single-round query (every pair of every ray), for reference
    d = model.desc()
    L.call("nif_frontend", ctypes.byref(d), vp(pipe.tlas.buf.data_ptr()), vp(rays.data_ptr()), n,
           vp(ray_id.data_ptr()), vp(qobj.data_ptr()), max_q, vp(goff1.data_ptr()),
           vp(count.data_ptr()), vp(ws.data_ptr()), ws.numel(), sp)
    nq_all = int(count[0].item())

    # end to end through the C ABI with host buffers: every frame's rays go
    # up from pinned memory and its mask comes back.  Two frames are in
    # flight (frame k + 1's rays go up while frame k is queried, its mask
    # comes back while k + 1 is queried); the L2 flush before every frame's
    # query is inside the timed span.  The per-frame latency (rays up,
    # query, mask back, one frame at a time) is reported beside it.
    host_rays = torch.empty((n, 8), dtype=torch.float32, pin_memory=True)
    host_rays.copy_(rays.cpu())
    host_bits = [torch.empty(bits.numel(), dtype=torch.int32, pin_memory=True) for _ in range(2)]
    dev_rays2 = [torch.empty_like(rays) for _ in range(2)]
    bits2 = [nif.empty_bits(n, dev) for _ in range(2)]

    def e2e_frames(K):
        frames = [(host_rays, host_bits[k % 2]) for k in range(K)]
        pipe.nif_query_host_frames(frames, dev_rays2, bits2, on_frame=lambda k: flush.zero_())

    e2e_frames(args.warmup)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    e_a, e_b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e_a.record(stream)
    e2e_frames(args.steps)
    e_b.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    e2e_ms = [e_a.elapsed_time(e_b) / args.steps]

    def e2e_one():
        pipe.nif_query_host(host_rays, host_bits[0], dev_rays2[0], bits2[0], n_chunks=1)

    lat_ms, _ = timed(e2e_one, args.steps, args.warmup)

    # the inference stage alone (the paper's separate Inference kernel):
    # nif_mlp_infer over the round-1 pairs, their inputs encoded once in
    # FP16 (nif_encode), timed with L2 flushed before each launch (inputs
    # from HBM) and back to back (inputs left in L2 when they fit)
    mlp_alone = mlp_alone_stats(pipe, bits, args.steps, args.warmup, flush)
    # medians of the timed steps (the e2e figure is one span over all steps)
    ms = reduce_max(statistics.median(nif_ms), world, dev)
    ms_eager = reduce_max(statistics.median(eager_ms), world, dev)
    bms = reduce_max(statistics.median(bvh_ms), world, dev)
    ems = reduce_max(statistics.mean(e2e_ms), world, dev)
    value = world * n / (ms * 1e-3)
    hbm, tflops, src = _peaks()
    fused_s = subs["fused_ms"] * 1e-3
    alg_bytes, flops_q = pipe.query_cost()
    ach_gbs = nq * alg_bytes / fused_s / 1e9
    tc_tflops = nq * flops_q / fused_s / 1e12
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {0: "f32", 1: "f16", 2: "bf16", 3: "e4m3"}[cfg.mlp_dtype],
        "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload], "rays": n, "queries": nq,
                   "queries_round1": nq1, "queries_all_pairs": nq_all, "triangles": pipe.n_tris,
                   "objects": cfg.n_obj, "nif_objects": pipe.n_obj, "triangles_nif": pipe.n_tris_nif,
                   "l2": "flushed (256 MB write) before every timed step",
                   "exact_cast": cfg.exact_cast, "tlas": cfg.tlas_builder, "cuda_graph": bool(graphs),
                   "round1": round1, "round1_pairs": round1_pairs,
                   "fused_schedule": SCHED_NAME[pipe.forward_models()[0][0].cfg.schedule],
                   "fused_ctas_per_sm": pipe.forward_models()[0][0].cfg.ctas_per_sm,
                   "fused_tile_m": pipe.forward_models()[0][0].cfg.tile_m or 128, "autotune_ms": tune_ms,
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "ms_per_step_eager": ms_eager,
        "bvh_rays_per_s": world * n / (bms * 1e-3), "bvh_ms_per_step": bms,
        "speedup_vs_bvh": bms / ms, "bvh_compared": best_tree, "bvh_trees": tree_stats,
        "visibility_disagreement": dis, "ablations": abl, "train_s": train_s,
        "train": train_stats,
        "stages_ms": subs,
        "roofline": {"kernel": "nif fused encode+MLP (tcgen05), both rounds", "bound": "hbm",
                     "achieved": ach_gbs, "peak": hbm, "unit": "GB/s", "frac": ach_gbs / hbm,
                     "traffic": FUSED_TRAFFIC_BYTES.get(
                         (args.workload, SCHED_NAME[pipe.forward_models()[0][0].cfg.schedule],
                          pipe.forward_models()[0][0].cfg.ctas_per_sm, round1)),
                     "traffic_source": ("ncu dram__bytes_read.sum + dram__bytes_write.sum summed "
                                        "over the step's two fused launches"),
                     "peak_source": src,
                     "tensor_tflops": tc_tflops, "tensor_peak_tflops": tflops,
                     "tensor_frac": tc_tflops / tflops,
                     "alg_bytes_per_query": alg_bytes, "flops_per_query": flops_q},
        "e2e": {"value": world * n / (ems * 1e-3), "unit": UNIT,
                "h2d_bytes_per_step": n * 32, "d2h_bytes_per_step": bits.numel() * 4,
                "frames_in_flight": 2, "l2": "flushed before every frame's query, inside the timed span",
                "latency_ms_per_frame": reduce_max(statistics.median(lat_ms), world, dev)},
        # per step: the exact cast (and the mask clear when it does not come
        # first), 3 + 3 front-end kernels, one fused forward per network
        # model and round
        "gpu_launches": (7 + (cfg.exact_cast != "first") + 2 * len(pipe.forward_models())) * args.steps,
        "clocks": clocks,
    }
    if mlp_alone is not None:
        line["mlp_alone"] = mlp_alone
    if sweep is not None:
        line["precision_sweep"] = sweep
    if args.r_sweep and args.workload == "paper" and rank == 0:
        line["r_sweep"] = r_sweep(log)
    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.workload in ("room", "full"):
        line["cpu_baseline"] = cpu_baseline(args.workload)
    elif rank == 0:
        line["cpu_baseline"] = None
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_grouped(args):
    """Per-object networks (one per object, uneven pair counts) in one
    persistent grouped launch captured in a CUDA graph, against the BVH cast
    of the same rays (objects are far apart, so the any-hit cast answers each
    ray's own object)."""
    import ctypes

    import numpy as np
    import torch

    from paper_2306_07191_gb300 import _lib as L
    from paper_2306_07191_gb300 import nif, synth, workloads
    from paper_2306_07191_gb300.pipeline import GRID_SCALE, GRID_SEED

    log = lambda *a: print(*a, file=sys.stderr, flush=True)
    t0 = time.time()
    gw = workloads.grouped_objects(total_rays=8_000_000 if not args.small else 400_000)
    sc = gw.scene
    n_obj = sc.n_obj
    dev = torch.device("cuda")
    verts, tris = torch.from_numpy(sc.verts).to(dev), torch.from_numpy(sc.tris).to(dev)
    bvh = nif.BVH(verts, tris)
    rays = torch.from_numpy(gw.rays).to(dev)
    n = int(rays.shape[0])
    cfg = nif.NifConfig(res=list(workloads.TINY_RES), n_features=2, log2_table=19, grid_dtype=L.NIF_F16,
                        n_hidden=3, width=64, mlp_dtype=L.NIF_F16, net_mode=L.NIF_NETS_OBJECT)
    V = nif.NifModel.grid_vertices(cfg)
    g32 = torch.empty(n_obj * 2 * V * 2, dtype=torch.float32, device=dev)
    L.call("nif_fill_uniform", ctypes.c_void_p(g32.data_ptr()), g32.numel(), GRID_SEED, GRID_SCALE, nif._stream())
    rng = np.random.default_rng(5)
    flat = np.concatenate([synth.flatten_mlp(synth.mlp_init(rng, cfg.K, 64, 3)) for _ in range(n_obj)])
    model = nif.NifModel(cfg, torch.from_numpy(sc.obj_aabb).to(dev), g32.half(), torch.from_numpy(flat).half().to(dev))
    del g32
    obj = np.repeat(np.arange(n_obj, dtype=np.int32), gw.counts)
    ray_id = torch.arange(n, dtype=torch.int32, device=dev)
    qobj = torch.from_numpy(obj).to(dev)
    goff = torch.from_numpy(np.concatenate([[0], np.cumsum(gw.counts)]).astype(np.int64)).to(dev)
    bits = nif.empty_bits(n, dev)
    ws = model.workspace(0)
    log(f"grouped workload ready: {n_obj} objects, {sc.tris.shape[0]} triangles, {n} pairs "
        f"({time.time() - t0:.1f}s)")

    def query():
        d = model.desc()
        L.call("nif_infer_queries", ctypes.byref(d), ctypes.c_void_p(rays.data_ptr()), n,
               ctypes.c_void_p(ray_id.data_ptr()), ctypes.c_void_p(qobj.data_ptr()),
               ctypes.c_void_p(goff.data_ptr()), n, ctypes.c_void_p(bits.data_ptr()), None,
               ctypes.c_void_p(ws.data_ptr()), ws.numel(), nif._stream())

    def time_fn(fn, K, W):
        for _ in range(W):
            fn()
        torch.cuda.synchronize()
        out = []
        for _ in range(K):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            out.append(e0.elapsed_time(e1))
        return statistics.median(out)

    # project autotuner: schedule and CTAs per SM of the persistent grouped launch
    if args.ctas_per_sm or args.schedule:
        model.cfg.ctas_per_sm = args.ctas_per_sm
        model.cfg.schedule = (L.NIF_SCHED_SERIAL if args.ctas_per_sm else
                              {"serial": L.NIF_SCHED_SERIAL, "pipelined": L.NIF_SCHED_PIPELINED}[args.schedule])
        sched, best, sweep = model.cfg.schedule, model.cfg.ctas_per_sm, None
    else:
        sched, best, sweep = nif.autotune(model, query, key_extra=(n, "grouped"))
    query()
    torch.cuda.synchronize()
    # one persistent grouped launch captured in a CUDA graph
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        query()
        torch.cuda.synchronize()
        with torch.cuda.graph(g, stream=s):
            query()
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    nif_ms = time_fn(g.replay, args.steps, args.warmup)
    model.check(ws)
    bvh_bits = nif.empty_bits(n, dev)
    # the comparison: the faster of the LBVH and PLOC casts of the same rays
    trees = {"lbvh": bvh, "ploc": nif.BVH(verts, tris, builder="ploc")}
    tree_ms = {name: time_fn(lambda t=t: t.cast_shadow(rays, out=bvh_bits), args.steps, args.warmup)
               for name, t in trees.items()}
    best_tree = min(tree_ms, key=tree_ms.get)
    bvh_ms = tree_ms[best_tree]
    tree_stats = {name: {**t.stats(rays), "ms_per_step": tree_ms[name]} for name, t in trees.items()}
    alg_bytes, flops_q = 3 * 8 * 8 * 2 * 2, 2 * (48 * 64 + 2 * 64 * 64 + 64)
    hbm, tflops, src = _peaks()
    line = {"metric": METRIC, "value": n / (nif_ms * 1e-3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": nif_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f16", "data": "synthetic",
            "config": {"workload": WORKLOADS["grouped"], "rays": n, "objects": n_obj,
                       "triangles": int(sc.tris.shape[0]), "pairs_per_object": gw.counts.tolist(),
                       "fused_schedule": SCHED_NAME[sched], "fused_ctas_per_sm": best,
                       "fused_tile_m": model.cfg.tile_m or 128,
                       "autotune_ms": sweep, "cuda_graph": True},
            "bvh_rays_per_s": n / (bvh_ms * 1e-3), "bvh_ms_per_step": bvh_ms, "speedup_vs_bvh": bvh_ms / nif_ms,
            "bvh_compared": best_tree, "bvh_trees": tree_stats,
            "roofline": {"kernel": "nif fused encode+MLP (tcgen05), grouped", "bound": "hbm",
                         "achieved": n * alg_bytes / (nif_ms * 1e-3) / 1e9, "peak": hbm, "unit": "GB/s",
                         "frac": n * alg_bytes / (nif_ms * 1e-3) / 1e9 / hbm, "traffic": None,
                         "peak_source": src, "tensor_tflops": n * flops_q / (nif_ms * 1e-3) / 1e12}}
    print(json.dumps(line), flush=True)


PRIMARY_METRIC = "primary rays/sec NIF (hit, normal, depth) vs own GPU BVH closest hit"


def run_primary(args):
    """NIF for primary rays on the room frame: one step = the exact
    closest-hit cast of the room, the front end (every pair), the fused
    five-output network and the closest-hit resolution, against the exact
    closest-hit cast over every triangle."""
    import torch

    from paper_2306_07191_gb300 import _lib as L
    from paper_2306_07191_gb300 import nif
    from paper_2306_07191_gb300.pipeline import PrimaryPipeline, primary_config

    log = lambda *a: print(*a, file=sys.stderr, flush=True)
    cfg = primary_config()
    if args.small:
        cfg.width, cfg.height, cfg.train_steps, cfg.batch, cfg.train_spp, cfg.n_obj = 640, 360, 8, 65536, 2, 16
    if args.ctas_per_sm:
        cfg.ctas_per_sm = args.ctas_per_sm
    pipe = PrimaryPipeline(cfg, log=log)
    pipe.two_rounds = args.primary_two_rounds
    train_s = pipe.train()
    tms = sorted(pipe.train_step_ms[1:]) or pipe.train_step_ms
    acc = pipe.disagreement()
    abl = pipe.ablations()
    log(f"primary accuracy {acc}  ablations {abl}")
    pipe.release_training_state()
    torch.cuda.empty_cache()
    tune_ms = None
    if not args.ctas_per_sm:
        cands = tuple(c for c in nif.SCHEDULE_CANDIDATES if c[0] == L.NIF_SCHED_SERIAL)
        sched, occ, tune_ms = nif.autotune(pipe.model, lambda: pipe.primary_step(), candidates=cands,
                                           key_extra=(pipe.n_rays, "primary"))
        log(f"autotuned fused kernel: {occ} CTAs/SM ({tune_ms})")
    n = pipe.n_rays
    rays = pipe.rays
    dev = rays.device
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def timed(fn, sub=False):
        for _ in range(args.warmup):
            flush.zero_()
            fn()
        torch.cuda.synchronize()
        parts = []
        for _ in range(args.steps):
            flush.zero_()
            e = [torch.cuda.Event(enable_timing=True) for _ in range(7)]
            if sub:
                fn(e[0:6])
                if not pipe.two_rounds:  # events 4 and 5 are not recorded
                    e[4].record(stream)
                    e[5].record(stream)
            else:
                e[0].record(stream)
                fn()
            e[6].record(stream)
            parts.append(e)
        torch.cuda.synchronize()
        tot = statistics.median(e[0].elapsed_time(e[6]) for e in parts)
        subs = None
        if sub:
            def m(a, b):
                return statistics.median(e[a].elapsed_time(e[b]) for e in parts)
            if pipe.two_rounds:
                # start, exact cast, front end 1, fused 1, resolve 1 + front
                # end 2, fused 2, resolve 2 (end)
                subs = {"room_cast_ms": m(0, 1), "frontend_nearest_ms": m(1, 2), "fused_round1_ms": m(2, 3),
                        "resolve1_frontend_rest_ms": m(3, 4), "fused_round2_ms": m(4, 5),
                        "resolve2_ms": m(5, 6)}
                subs["fused_ms"] = subs["fused_round1_ms"] + subs["fused_round2_ms"]
            else:
                subs = {"room_cast_ms": m(0, 1), "frontend_ms": m(1, 2), "fused_ms": m(2, 3),
                        "resolve_ms": m(3, 6)}
        return tot, subs

    with ClockSampler(0) as clk:
        torch.cuda.profiler.start()
        nif_ms, subs = timed(lambda ev=None: pipe.primary_step(ev=ev), sub=True)
        bvh_ms, _ = timed(lambda: pipe.bvh_step())
        torch.cuda.profiler.stop()
    clocks = clk.summary()
    pipe.check()
    nq = int(pipe._primary_buffers()["count"][1 if pipe.two_rounds else 0].item())
    host_rays = torch.empty((n, 8), dtype=torch.float32, pin_memory=True)
    host_rays.copy_(rays.cpu())
    host_t = torch.empty(n, dtype=torch.float32, pin_memory=True)
    host_n = torch.empty((n, 3), dtype=torch.float32, pin_memory=True)
    dev_rays = torch.empty_like(rays)

    def e2e_step():
        dev_rays.copy_(host_rays, non_blocking=True)
        t, nrm, _ = pipe.primary_step(dev_rays)
        host_t.copy_(t, non_blocking=True)
        host_n.copy_(nrm, non_blocking=True)

    e2e_ms, _ = timed(e2e_step)
    hbm, tflops, src = _peaks()
    alg_bytes, flops_q = pipe.query_cost()
    fused_s = subs["fused_ms"] * 1e-3
    ach = nq * alg_bytes / fused_s / 1e9
    line = {
        "metric": PRIMARY_METRIC, "value": n / (nif_ms * 1e-3), "unit": "primary rays/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": nif_ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f16", "data": "synthetic",
        "config": {"workload": WORKLOADS["primary"], "rays": n, "queries": nq, "triangles": pipe.n_tris,
                   "objects": pipe.n_obj, "outputs": pipe.n_outputs,
                   "l2": "flushed (256 MB write) before every timed step", "fused_schedule": "serial",
                   "fused_ctas_per_sm": pipe.model.cfg.ctas_per_sm, "autotune_ms": tune_ms,
                   "parallelism": "single GPU"},
        "bvh_rays_per_s": n / (bvh_ms * 1e-3), "bvh_ms_per_step": bvh_ms, "speedup_vs_bvh": bvh_ms / nif_ms,
        "accuracy": acc, "ablations": abl, "train_s": train_s,
        "train": {"steps": len(pipe.train_step_ms), "gpu_ms_per_step_median": tms[len(tms) // 2],
                  "loss_curve": [round(v, 6) for v in pipe.losses[::8] + pipe.losses[-1:]]},
        "stages_ms": subs,
        "roofline": {"kernel": "nif fused encode+MLP (tcgen05), 5 outputs", "bound": "hbm", "achieved": ach,
                     "peak": hbm, "unit": "GB/s", "frac": ach / hbm, "traffic": None, "peak_source": src,
                     "tensor_tflops": nq * flops_q / fused_s / 1e12, "tensor_peak_tflops": tflops,
                     "alg_bytes_per_query": alg_bytes, "flops_per_query": flops_q},
        "e2e": {"value": n / (e2e_ms * 1e-3), "unit": "primary rays/s", "h2d_bytes_per_step": n * 32,
                "d2h_bytes_per_step": n * 16},
        # per step: room cast; per round 3 front-end kernels, the fused
        # forward and 2 resolution kernels
        "gpu_launches": (13 if pipe.two_rounds else 7) * args.steps,
        "clocks": clocks,
        "cpu_baseline": None,
    }
    print(json.dumps(line), flush=True)


def run_render(args):
    """A direct-lighting frame with NIF shadows against the same frame with
    exact BVH shadows, and the PSNR of NIF frames trained on importance- or
    uniformly-sampled light rays at 1, 4 and 16 training samples per pixel
    (the comparison of Sec. 6.2)."""
    import ctypes

    import torch

    from paper_2306_07191_gb300 import _lib as L
    from paper_2306_07191_gb300 import nif
    from paper_2306_07191_gb300.pipeline import RenderPipeline, render_config

    log = lambda *a: print(*a, file=sys.stderr, flush=True)

    def make(sampling, spp):
        cfg = render_config(sampling, spp)
        if args.small:
            cfg.width, cfg.height, cfg.train_steps, cfg.batch, cfg.n_obj = 640, 360, 8, 65536, 16
        return RenderPipeline(cfg, log=log)

    sweep = {"importance": {}, "uniform": {}}
    main_pipe = None
    for sampling in ("importance", "uniform"):
        for spp in ((1, 4) if args.small else (1, 4, 16)):
            pipe = make(sampling, spp)
            pipe.train()
            sweep[sampling][spp] = pipe.psnr()
            log(f"{sampling} training rays, {spp} spp: PSNR {sweep[sampling][spp]:.2f} dB")
            if sampling == "importance" and spp == 4:
                main_pipe = pipe
            else:
                del pipe
                torch.cuda.empty_cache()
    pipe = main_pipe
    dis = pipe.disagreement()
    pipe.release_training_state()
    torch.cuda.empty_cache()
    fwd = [m for m, _ in pipe.forward_models()]
    tbits = nif.empty_bits(pipe.n_rays)
    cands = tuple(c for c in nif.SCHEDULE_CANDIDATES if c[0] == L.NIF_SCHED_SERIAL)
    sched, occ, tune_ms = nif.autotune(fwd[0], lambda: pipe.query_step(tbits), also=fwd[1:], candidates=cands,
                                       key_extra=(pipe.n_rays, "render"))
    round1_pairs = pipe.tune_round1()
    from paper_2306_07191_gb300.pipeline import ROUND1_NAME
    round1 = ROUND1_NAME[pipe.front_model().cfg.round1]
    cam, u, spp = pipe.eval_camera, pipe.eval_u, pipe.cfg.render_spp
    n_pix, n = pipe.n_pix, pipe.n_rays
    lights, cdf = pipe._light_setup(), pipe._cdf["importance"]
    dev = cam.device
    t = torch.empty(n_pix, dtype=torch.float32, device=dev)
    prim = torch.empty(n_pix, dtype=torch.int32, device=dev)
    rays = torch.empty((n, 8), dtype=torch.float32, device=dev)
    f = torch.empty(n, dtype=torch.float32, device=dev)
    bits = nif.empty_bits(n)
    radiance = torch.empty(n_pix, dtype=torch.float32, device=dev)
    vp, sp = ctypes.c_void_p, nif._stream()
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def frame(nif_vis, ev=None):
        L.call("bvh_cast_closest", vp(pipe.bvh.buf.data_ptr()), vp(cam.data_ptr()), n_pix, vp(t.data_ptr()),
               vp(prim.data_ptr()), sp)
        L.call("nif_light_samples", vp(cam.data_ptr()), vp(t.data_ptr()), vp(prim.data_ptr()),
               vp(pipe.verts.data_ptr()), vp(pipe.tris.data_ptr()), n_pix, spp, vp(lights.data_ptr()),
               vp(cdf.data_ptr()), int(lights.shape[0]), vp(u.data_ptr()), pipe.cfg.tmin, pipe.cfg.albedo,
               vp(rays.data_ptr()), vp(f.data_ptr()), sp)
        if ev is not None:
            ev[0].record(stream)
        if nif_vis:
            pipe.query_step(bits, rays=rays)
        else:
            pipe.bvh.cast_shadow(rays, out=bits)
        if ev is not None:
            ev[1].record(stream)
        L.call("nif_shade", vp(f.data_ptr()), vp(bits.data_ptr()), n_pix, spp, vp(radiance.data_ptr()), sp)

    def timed(nif_vis):
        for _ in range(args.warmup):
            flush.zero_()
            frame(nif_vis)
        torch.cuda.synchronize()
        parts = []
        for _ in range(args.steps):
            flush.zero_()
            e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
            e[0].record(stream)
            frame(nif_vis, e[1:3])
            e[3].record(stream)
            parts.append(e)
        torch.cuda.synchronize()
        return (statistics.median(e[0].elapsed_time(e[3]) for e in parts),
                statistics.median(e[1].elapsed_time(e[2]) for e in parts))

    with ClockSampler(0) as clk:
        torch.cuda.profiler.start()
        nif_ms, nif_shadow_ms = timed(True)
        bvh_ms, bvh_shadow_ms = timed(False)
        torch.cuda.profiler.stop()
    clocks = clk.summary()
    pipe.check()
    line = {
        "metric": METRIC, "value": n / (nif_shadow_ms * 1e-3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": nif_shadow_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f16", "data": "synthetic",
        "config": {"workload": WORKLOADS["render"], "rays": n, "pixels": n_pix, "light_spp": spp,
                   "objects": pipe.n_obj, "triangles": pipe.n_tris,
                   "l2": "flushed (256 MB write) before every timed step", "fused_schedule": "serial",
                   "fused_ctas_per_sm": occ, "autotune_ms": tune_ms, "round1": round1,
                   "round1_pairs": round1_pairs, "parallelism": "single GPU"},
        "bvh_rays_per_s": n / (bvh_shadow_ms * 1e-3), "bvh_ms_per_step": bvh_shadow_ms,
        "speedup_vs_bvh": bvh_shadow_ms / nif_shadow_ms,
        "frame_ms": {"nif": nif_ms, "bvh": bvh_ms},
        "visibility_disagreement": dis,
        "psnr_db": {k: {str(s_): v for s_, v in d.items()} for k, d in sweep.items()},
        # per step: primary cast, light sampling, the shadow query (room cast,
        # 3 + 3 front-end kernels, 4 fused forwards), shading
        "gpu_launches": 14 * args.steps,
        "clocks": clocks,
        "cpu_baseline": None,
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--small", action="store_true", help="reduced workload for quick checks")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ctas-per-sm", type=int, default=0,
                    help="fix the serial schedule's CTAs per SM (skips the autotuner)")
    ap.add_argument("--r-sweep", action="store_true",
                    help="paper workload: also sweep the outer grid resolution R = 64, 256, 1024")
    ap.add_argument("--schedule", default="", choices=["", "serial", "pipelined"],
                    help="fix the fused kernel's schedule (skips the autotuner)")
    ap.add_argument("--workload", default="full", choices=sorted(WORKLOADS))
    ap.add_argument("--primary-two-rounds", action="store_true",
                    help="primary workload: nearest pair first, then only pairs entered before the nearest hit")
    ap.add_argument("--train-precision", choices=("f32", "f16"), default="f16",
                    help="online training: FP32 on the CUDA cores, or FP16 operands on the tensor cores with a "
                         "dynamic loss scale")
    ap.add_argument("--no-graph", action="store_true",
                    help="time the step's calls one by one instead of replaying a CUDA graph of them")
    ap.add_argument("--exact-cast", choices=("first", "after", "overlap"), default=None,
                    help="when the non-NIF geometry is cast: before the NIF query (default), after it, "
                         "or beside it on a second stream")
    ap.add_argument("--tlas", choices=("lbvh", "ploc"), default=None,
                    help="builder of the top level over the object boxes (default: the workload's)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "grouped":
        run_grouped(args)
    elif args.workload == "mlp":
        run_mlp(args)
    elif args.workload == "mma":
        run_mma(args)
    elif args.workload == "primary":
        run_primary(args)
    elif args.workload == "render":
        run_render(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
