"""Benchmark of the hot path on GB300.

One step = one FP32 training step of the ellipsoid-union workload (64^3
voxels, 16 hash levels x 2 features, T = 2^19, MLP 576-64-64-64-16):
16 poses drawn on the device, rays sampled per pose until 2^18 ray/voxel
segments are filled, then segments -> linearization -> labels -> encoding ->
MLP -> losses -> backward -> Adam, all in the library's kernels. `value` is
train samples (segments) per second over all ranks.

Next to it, `query` reports neural intersection queries per second of the
inference path (torus at 128^3, 2^22 rays, network of the 16^3 torus
workload) in FP32 and, where built, mixed precision.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun every rank runs the same per-GPU work (weak scaling, no
collective on the data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "neural intersection queries/s and train samples/s on 1 GB300, mixed vs FP32, at stated error"
TRAIN_WORKLOAD = "ellipsoids64_train"
QUERY_WORKLOAD = "torus128_query"
N_SEG = 1 << 18
N_POSES = 16
# DRAM bytes (read + write) per launch from one ncu capture (--set full) of
# the current kernel of a stage on this workload (the encoding backward with
# a term's levels split over two tasks); a stage missing here reports
# traffic null.
NCU_TRAFFIC = {"encode_bwd": 701.4e6}
# stages the library runs beside the main stream's work (weight gradients and
# the weights' update on its second stream, the next step's batch on its
# third): their event intervals include the overlap, so they are not the
# step's critical path
OVERLAPPED = {"mlp_dw_fp32", "mlp_dw_tc", "adam_weights", "sample_rays", "refit", "seg_traverse", "scan",
              "seg_scatter", "seg_emit", "linearize", "labels"}


def _emit(line, args):
    """Prints the run's JSON line and, with --log, appends it to a JSON-lines
    file (one record per run, kept beside the profiles of the same build)."""
    text = json.dumps(line)
    print(text, flush=True)
    if getattr(args, "log", None):
        with open(args.log, "a") as f:
            f.write(text + "\n")


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), d.get("bf16_tflops", 1900.0), d.get("bf16_tflops_sustained", 1700.0), "measured"
    return 6800.0, 1900.0, 1700.0, "fallback"


class Clocks:
    """nvidia-smi sampler during the timed region (clocks and throttle reasons)."""

    def __init__(self, index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={index}", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                       "-lms", "50"], stdout=self.f, stderr=subprocess.DEVNULL)
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
        self.f.flush()
        rows = [r.split(",") for r in open(self.f.name).read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
                for k, nm in enumerate(names):
                    if r[5 + k].strip().lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def _max_over_ranks(x, ws):
    """Max of a host float over ranks (NCCL on GPUs, gloo on CPU)."""
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------
# Oracle timing (the CPU baseline and the reference arm)
# ---------------------------------------------------------------------------
_ORACLE_SETUP = {}


def _oracle_setup():
    """The training workload's mesh, voxelization and initial parameters for
    the oracle, built once per process (outside every timed interval)."""
    if not _ORACLE_SETUP:
        import oracle as O
        from paper_2604_24666_gb300 import synth as S
        net = S.WORKLOADS[TRAIN_WORKLOAD]["net"]
        mesh = S.make_mesh(S.WORKLOADS[TRAIN_WORKLOAD]["shape"])
        occ, ptr, idx = O.voxelize(net.voxel_res, mesh)
        _ORACLE_SETUP["v"] = (net, mesh, occ, ptr, idx) + tuple(S.init_params(net))
    return _ORACLE_SETUP["v"]


def oracle_train_sample(n_rays=384, seed=0):
    """One oracle training step on a bounded sample of the training workload.

    Returns (segments processed, seconds, threads)."""
    import oracle as O
    from paper_2604_24666_gb300 import synth as S
    net, mesh, occ, ptr, idx, tables, ws, s = _oracle_setup()
    pose = S.poses(1, seed=100 + seed)[0]
    rays = S.sphere_rays(n_rays, seed=200 + seed)
    t0 = time.perf_counter()
    seg = O.segments(net.voxel_res, occ, pose, rays)
    p0, p1, ld, lr = O.linearize(pose, rays, seg)
    lab = O.labels(mesh, ptr, idx, seg.vox, p0, p1)
    x = O.encode_segments(net, tables, p0, p1)
    out, acts = O.mlp_forward(ws, x)
    tot, parts, dout, ds = O.loss(net, out, lab, s, lr)
    dws, dx = O.mlp_backward(ws, acts, dout)
    half = net.in_dim // 2
    dt0, _ = O.encode_points_backward(net, tables, p0, dx[:, :half])
    dt1, _ = O.encode_points_backward(net, tables, p1, dx[:, half:])
    z = np.zeros_like(tables, dtype=np.float64)
    O.adam(tables.astype(np.float64), z, z, dt0 + dt1, 1, 1e-2)
    for wi, gi in zip(ws, dws):
        O.adam(wi.astype(np.float64), 0 * gi, 0 * gi, gi, 1, 1e-3)
    return len(seg), time.perf_counter() - t0, O.num_threads()


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    import oracle as O
    O.build()
    # each step a bounded sample: 384 rays (about 1 s of oracle work on 16
    # Arm cores, the sample of the CPU-baseline leg) for up to 100 steps, fewer
    # rays per step beyond, so a run stays within about two minutes (a step
    # also pays a fixed cost for Adam over the whole tables, so fewer rays per
    # step lower the segments/s)
    n_rays = 384 if args.steps <= 100 else max(48, 384 * 100 // args.steps)
    for i in range(args.warmup):
        oracle_train_sample(n_rays=n_rays, seed=i)
    segs, secs = 0, 0.0
    thr = 1
    for i in range(args.steps):
        n, t, thr = oracle_train_sample(n_rays=n_rays, seed=1000 + i)
        segs += n
        secs += t
    v = segs / secs
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "segments/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": TRAIN_WORKLOAD, "note": "FP64 oracle on the host cores; each step a bounded "
                       f"sample of {n_rays} rays of the workload (one pose)"},
            "cpu_baseline": {"value": v, "unit": "segments/s", "cores": thr, "kind": "oracle",
                             "sample": f"{args.steps} steps x {n_rays} rays (~{segs // max(args.steps, 1)} segments/step)"},
            "e2e": {"value": v, "unit": "segments/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    _emit(line, args)
    return 0


# ---------------------------------------------------------------------------
# Our arm
# ---------------------------------------------------------------------------
def _stage_work(net, stage, n_seg):
    """Algorithmic bytes or flops of one stage over n_seg segments: (amount, unit, bound)."""
    P, L = net.n_terms, net.levels
    gathers = 2 * P * L * 8                       # corner reads per segment
    if stage == "encode_fwd":
        return n_seg * (gathers * 8 + 32 + net.in_dim * 4), "bytes", "hbm"
    if stage == "encode_bwd":
        return n_seg * (gathers * 8 + 32 + net.in_dim * 4), "bytes", "hbm"
    # FP32 MLP on the tensor cores (split TF32): bound by the rows it streams
    W, H = net.mlp_width, net.mlp_depth
    if stage == "mlp_fwd_fp32":     # features read; outputs and activations written
        return n_seg * (net.in_dim * 4 + 64 + H * W * 4), "bytes", "hbm"
    if stage == "mlp_bwd_fp32":     # output gradients and activations read; dY_l written
        return n_seg * (64 + 2 * H * W * 4), "bytes", "hbm"
    if stage == "mlp_dx_fp32":      # dY_0 read; feature gradients written
        return n_seg * (W * 4 + net.in_dim * 4), "bytes", "hbm"
    if stage == "mlp_dw_fp32":      # features, activations and every dY_l read
        return n_seg * (net.in_dim * 4 + 2 * H * W * 4 + 64), "bytes", "hbm"
    return None


def _l2_probe(nif, h, dev):
    """Measured ceilings of the encoding kernels' memory patterns (library
    probes, CUDA events): 8- and 16-byte FP32 reductions into a 64 MiB buffer
    held in L2 (the table gradient's size) and random 8-byte rows of 64 MiB /
    4-byte rows of 32 MiB and 1 MiB (the FP32 and FP16 tables)."""
    import torch
    out = {}
    buf = torch.zeros((16 << 20,), dtype=torch.float32, device=dev)          # 64 MiB
    for name, kind, nbytes in (("red8_64MiB", nif.NIF_PROBE_RED8, 64 << 20), ("red16_64MiB", nif.NIF_PROBE_RED16, 64 << 20),
                               ("load8_64MiB", nif.NIF_PROBE_LOAD8, 64 << 20), ("load4_32MiB", nif.NIF_PROBE_LOAD4, 32 << 20),
                               ("load4_1MiB", nif.NIF_PROBE_LOAD4, 1 << 20),
                               ("red8_64MiB_warp", nif.NIF_PROBE_RED8_WARP, 64 << 20),
                               ("red16_64MiB_warp", nif.NIF_PROBE_RED16_WARP, 64 << 20),
                               ("load8_64MiB_warp", nif.NIF_PROBE_LOAD8_WARP, 64 << 20),
                               ("load4_32MiB_warp", nif.NIF_PROBE_LOAD4_WARP, 32 << 20)):
        gbs, ms = nif.nif_probe_memory(h.h, kind, buf[:nbytes // 4], iters=128)
        out[name] = {"GB/s": gbs, "ms_per_launch": ms}
    # the ceilings: whole sectors (every fetched byte used); the random rows
    # (one sector per 8-byte access) are the floor of the same pattern
    out["ceiling_red"] = max(out["red8_64MiB_warp"]["GB/s"], out["red16_64MiB_warp"]["GB/s"])
    out["ceiling_load8"] = out["load8_64MiB_warp"]["GB/s"]
    del buf
    return out


def _hashed_levels(net):
    """Levels whose rows are the spatial hash ((N_l + 1)^3 > T): there every
    corner row of a point is its own 32-byte sector."""
    T = 1 << net.log2_table
    return sum(1 for l in range(net.levels) if (int(math.floor(net.base_res * net.growth ** l)) + 1) ** 3 > T)


def _l2_work(net, stage, n_pts):
    """Payload bytes of the encoding's L2-bound accesses over the step's
    distinct end points: one 8-byte FP32 corner row per (point, gamma term,
    level, corner), gathered (forward) or reduced (backward)."""
    if stage in ("encode_fwd", "encode_bwd"):
        return n_pts * net.n_terms * net.levels * 8 * 8
    return None


def _scatter_ops(net, stage, n_pts):
    """Scattered L2 accesses of the hashed levels over the step's distinct
    end points (one sector each): the forward loads 8 corner rows per
    (point, term, level); the backward issues 6 reductions on average (the
    two corners of an x-edge share one 16-byte reduction when the cell's x is
    even, which the hash leaves adjacent: 4 x-edges, half of them paired)."""
    per = {"encode_fwd": 8, "encode_bwd": 6}.get(stage)
    return None if per is None else n_pts * net.n_terms * _hashed_levels(net) * per


def run_ours(args):
    import torch
    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
    torch.cuda.set_device(local)
    dev = torch.device(f"cuda:{local}")
    from paper_2604_24666_gb300 import build as B
    B.build()
    from paper_2604_24666_gb300 import nif, synth as S
    hbm, bf16, bf16s, peak_src = _peaks()
    w = S.WORKLOADS[TRAIN_WORKLOAD]
    net = w["net"]
    mesh = S.make_mesh(w["shape"])
    h = nif.Nif(net, mesh, seed=1234 + rank)
    stream = torch.cuda.current_stream()

    # ---- device-resident training steps -------------------------------
    seed0 = 77 + 1000003 * rank
    # K steps in one call: each step's batch (sampling, segments, linearization,
    # labels) is built on the library's third stream beside the previous step
    nif.nif_train_steps(h.h, args.warmup, N_SEG, N_POSES, seed0, lr_grid=1e-2, lr_mlp=1e-3)
    torch.cuda.synchronize()

    def timed_steps(k, seed, stages=None):
        """k steps in one call, CUDA events on the stream around them, the
        library's per-stage events on (only for `stages` if given)."""
        nif.nif_profile_filter(h.h, stages)
        nif.nif_profile(h.h, 1)
        _barrier(ws)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        nif.nif_train_steps(h.h, k, N_SEG, N_POSES, seed, lr_grid=1e-2, lr_mlp=1e-3)
        b.record(stream)
        torch.cuda.synchronize()
        _barrier(ws)
        p = nif.nif_profile_read(h.h)
        nif.nif_profile(h.h, 0)
        nif.nif_profile_filter(h.h, None)
        return a.elapsed_time(b), p

    # every stage timed (two events each): the per-kernel split and the
    # dominant kernel; then the measured interval, with only the dominant
    # kernel's events in it
    ms_all, prof = timed_steps(args.steps, seed0 + args.warmup)
    dom = max((k for k in prof if k not in OVERLAPPED), key=lambda k: prof[k][0])
    clk = Clocks(local) if rank == 0 else None
    launches0 = nif.nif_kernel_launches()
    ms, prof_dom = timed_steps(args.steps, seed0 + args.warmup + args.steps, [dom])
    launches = nif.nif_kernel_launches() - launches0
    clocks = clk.stop() if clk else None
    ms_max = _max_over_ranks(ms, ws)
    value = ws * args.steps * N_SEG / (ms_max / 1e3)
    # the default one-launch FP32 forward on part of the SMs beside the
    # alternatives: on every SM (NIF_KNOB_STEP_FWD_CTAS = -1) and one launch
    # per layer (NIF_KNOB_FP32_FUSED = 0)
    nif.nif_set_knob(h.h, nif.NIF_KNOB_STEP_FWD_CTAS, -1)
    ms_all_sms, prof_all_sms = timed_steps(args.steps, seed0 + args.warmup + 2 * args.steps)
    nif.nif_set_knob(h.h, nif.NIF_KNOB_STEP_FWD_CTAS, 0)
    nif.nif_set_knob(h.h, nif.NIF_KNOB_FP32_FUSED, 0)
    ms_layer, prof_layer = timed_steps(args.steps, seed0 + args.warmup + 3 * args.steps)
    nif.nif_set_knob(h.h, nif.NIF_KNOB_FP32_FUSED, 1)
    fused_fwd = {"ms_per_step": ms_all / args.steps,
                 "mlp_fwd_fp32_ms": prof["mlp_fwd_fp32"][0] / args.steps,
                 "one_launch_every_sm": {"ms_per_step": ms_all_sms / args.steps,
                                         "mlp_fwd_fp32_ms": prof_all_sms["mlp_fwd_fp32"][0] / args.steps},
                 "per_layer": {"ms_per_step": ms_layer / args.steps,
                               "mlp_fwd_fp32_ms": prof_layer["mlp_fwd_fp32"][0] / args.steps},
                 "note": "all with every stage's events on; the one-launch forward keeps hidden activations in "
                         "shared memory and still writes those the backward reads; by default it runs on 3/4 of "
                         "the SMs (tile-balanced) while the next batch is built beside it"}
    loss, _ = nif.nif_train_step(h.h, N_SEG, N_POSES, seed0 + 99999, want_loss=True)

    # ---- dominant stage and its roofline -------------------------------
    # The encoding kernels are bound by L2 (gathers from and reductions into
    # 64 MiB tables that stay in L2), not by HBM: their fraction is taken
    # against the library's measured L2 ceilings over the payload of the
    # step's distinct end points; the HBM fraction over all end points is
    # kept beside it.
    n_pts, n_segs_enc = nif.nif_encoder_points(h.h)
    l2 = _l2_probe(nif, h, dev) if rank == 0 else None
    l2_peak = {"encode_bwd": ("ceiling_red", "red8_64MiB", "FP32 vector reductions into 64 MiB held in L2, whole "
                              "sectors per warp (the better of 8- and 16-byte)"),
               "encode_fwd": ("ceiling_load8", "load8_64MiB", "8-byte row loads from 64 MiB held in L2, whole sectors "
                              "per warp")}
    # scattered-access rate of the L2 (random rows, one sector each), G accesses / s
    l2_ops = {"encode_bwd": l2["red8_64MiB"]["GB/s"] / 8.0, "encode_fwd": l2["load8_64MiB"]["GB/s"] / 8.0} if l2 else None
    stages = {k: v for k, v in prof.items()}
    tot_ms = sum(v[0] for v in stages.values())
    roof = None
    work = _stage_work(net, dom, N_SEG)
    if work is not None:
        amount, unit, bound = work
        avg_ms = prof_dom[dom][0] / max(args.steps, 1)      # per step (one launch), inside the measured interval
        ach = amount / (avg_ms / 1e3) / 1e9
        hbm_roof = {"bound": bound, "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                    "peak_source": f"{peak_src} hbm_gbs", "algorithmic_bytes": amount,
                    "per": "segment: 2 end points x P terms x L levels x 8 corners x 8 B + 32 B + in_dim x 4 B"}
        roof = dict(hbm_roof, kernel=dom, traffic=NCU_TRAFFIC.get(dom))
        lw = _l2_work(net, dom, n_pts)
        ops = _scatter_ops(net, dom, n_pts)
        if lw is not None and l2 is not None and dom in l2_peak and ops is not None:
            key, floor_key, what = l2_peak[dom]
            ach2 = lw / (avg_ms / 1e3) / 1e9
            # the binding resource: the L2's rate for scattered accesses, which
            # the hashed levels' corner rows are (one sector each); payload of
            # those accesses per second against the probe's payload rate for
            # the same access mix (the coarse, dense levels counted as free)
            pay = ops * (64.0 / 6.0 if dom == "encode_bwd" else 8.0)      # bytes the scattered accesses carry
            peak_pay = l2_ops[dom] * (64.0 / 6.0 if dom == "encode_bwd" else 8.0)
            ach3 = pay / (avg_ms / 1e3) / 1e9
            roof = {"bound": "l2", "kernel": dom, "achieved": ach3, "peak": peak_pay, "unit": "GB/s",
                    "frac": ach3 / peak_pay,
                    "peak_source": "measured: the L2's rate for scattered accesses (nif_probe_memory " + floor_key +
                                   ", one 32-byte sector per access), at the kernel's mix of 8- and 16-byte accesses",
                    "scattered_accesses": ops,
                    "per": f"distinct end point: P terms x {_hashed_levels(net)} hashed levels x "
                           f"{'6 reductions (64 B)' if dom == 'encode_bwd' else '8 loads (64 B)'} "
                           f"({n_pts} distinct end points of {n_segs_enc} segments)",
                    "traffic": NCU_TRAFFIC.get(dom), "algorithmic_bytes": pay,
                    "all_levels": {"achieved": ach2, "algorithmic_bytes": lw, "ceiling": l2[key],
                                   "frac_of_ceiling": ach2 / l2[key],
                                   "ceiling_source": f"measured: {what} (nif_probe_memory)"},
                    "hbm": hbm_roof}
    kernels = {}
    for k, (kms, cnt) in sorted(stages.items(), key=lambda kv: -kv[1][0]):
        ent = {"ms_per_step": kms / max(args.steps, 1), "share": kms / tot_ms if tot_ms else None}
        if k in OVERLAPPED:
            ent["overlapped"] = True
        wk = _stage_work(net, k, N_SEG)
        if wk is not None:
            amount, unit, bound = wk
            ent["GB/s"] = amount / (ent["ms_per_step"] / 1e3) / 1e9
            ent["frac_hbm"] = ent["GB/s"] / hbm
        lw = _l2_work(net, k, n_pts)
        if lw is not None and l2 is not None and k in l2_peak:
            ent["l2_GB/s"] = lw / (ent["ms_per_step"] / 1e3) / 1e9
            ent["frac_l2_ceiling"] = ent["l2_GB/s"] / l2[l2_peak[k][0]]
            ops = _scatter_ops(net, k, n_pts)
            ent["scattered_G_per_s"] = ops / (ent["ms_per_step"] / 1e3) / 1e9
            ent["frac_l2_scatter"] = ent["scattered_G_per_s"] / l2_ops[k]          # l2_ops: G accesses / s
        kernels[k] = ent

    # ---- end to end through the public API, host buffers ----------------
    # The same workload (N_POSES poses U[-1,1]^3 per step, rays of the training
    # distribution per pose) given as host data: every step's rays are copied
    # from pinned host memory and every step's loss is read back to the host,
    # inside the timed region, by nif_train_steps_rays.
    per = int(math.ceil(N_SEG / N_POSES / max(h_seg_per_ray(h, nif), 0.05) * 1.2)) + 1
    n_rays_e2e = per * N_POSES
    inst_e2e = torch.arange(0, n_rays_e2e + 1, per, dtype=torch.int32, device=dev)

    def host_steps(k, seed):
        rays = np.stack([S.sphere_rays(n_rays_e2e, seed=seed + 7919 * i) for i in range(k)])
        poses = np.stack([S.poses(N_POSES, seed=seed + 104729 * i + 1) for i in range(k)])
        return torch.from_numpy(rays).pin_memory(), poses

    rays_w, poses_w = host_steps(args.warmup, 500 + 1000 * rank)
    rays_t, poses_t = host_steps(args.steps, 900 + 1000 * rank)
    nif.nif_train_steps_rays(h.h, poses_w, rays_w, N_SEG, inst_offsets=inst_e2e, lr_grid=1e-2, lr_mlp=1e-3)
    torch.cuda.synchronize()
    _barrier(ws)
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    loss_e2e = nif.nif_train_steps_rays(h.h, poses_t, rays_t, N_SEG, inst_offsets=inst_e2e, lr_grid=1e-2,
                                        lr_mlp=1e-3)       # every step's loss parts, read back as it ends
    f1.record(stream)
    torch.cuda.synchronize()
    assert np.isfinite(loss_e2e).all()
    e2e_ms = _max_over_ranks(f0.elapsed_time(f1), ws)
    e2e = {"value": ws * args.steps * N_SEG / (e2e_ms / 1e3), "unit": "segments/s",
           "h2d_bytes_per_step": int(n_rays_e2e * 32), "d2h_bytes_per_step": 48,
           "call": "nif_train_steps_rays", "input": "host rays (pinned) and poses per step"}
    h.close()

    # ---- mixed-precision training, same workload ---------------------------
    mixed = run_train_mixed(args, nif, S, dev, rank, hbm) if not args.no_mixed else None
    det = run_train_det(args, nif, S, dev, rank) if not args.no_det else None

    # ---- inference queries ------------------------------------------------
    query = run_query(args, nif, S, dev, rank) if not args.no_query else None
    batch = run_batch(args, nif, S, dev, rank) if not args.no_batch else None
    precision = run_precision(args, nif, S, dev) if (not args.no_precision and rank == 0) else None
    frame = run_frame(args, nif, S, dev) if (not args.no_frame and rank == 0) else None
    trav = run_traversal(args, nif, S, dev) if (not args.no_traversal and rank == 0) else None
    field = run_field(args, nif, S, dev, rank) if not args.no_field else None

    if rank != 0:
        return 0
    cpu = None
    if ws == 1 and not args.no_cpu:
        import oracle as O
        O.build()
        n, t, thr = oracle_train_sample(seed=0)
        segs_s, secs = n, t
        while secs < 10.0:
            n, t, thr = oracle_train_sample(seed=int(secs * 100) + 1)
            segs_s += n
            secs += t
        cpu = {"value": segs_s / secs, "unit": "segments/s", "cores": thr, "kind": "oracle",
               "sample": f"{segs_s} segments of the training workload in {secs:.1f} s (384 rays per sample)"}
    line = {"metric": METRIC, "value": value, "unit": "segments/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": TRAIN_WORKLOAD, "segments_per_step": N_SEG, "poses_per_step": N_POSES,
                       "voxels": "64^3", "levels": net.levels, "table": f"2^{net.log2_table}",
                       "mlp": "-".join(str(x) for x in [net.in_dim] + [net.mlp_width] * net.mlp_depth + [16]),
                       "l2": "working set larger than L2 (tables, gradients, Adam state 256 MB; features 604 MB)"},
            "profile": {"measured_interval": f"events of {dom} only", "all_stages_ms_per_step": ms_all / args.steps},
            "fp32_fused_forward": fused_fwd,
            "roofline": roof, "kernels": kernels, "l2_probe": l2, "encoder_points": {"distinct": n_pts, "segments": n_segs_enc},
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
            "clocks": clocks, "loss": list(loss) if loss is not None else None, "train_mixed": mixed,
            "train_deterministic": det, "query": query, "batch": batch, "frame_loop": frame, "traversal": trav, "field": field,
            "precision": precision}
    _emit(line, args)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def run_train_mixed(args, nif, S, dev, rank, hbm):
    """The training step of the same workload on the mixed-precision path
    (FP16 / BF16 tensor-core MLP forward and backward, FP16 table copy,
    FP32 masters, loss scaling): segments/s and the per-stage split."""
    import torch
    w = S.WORKLOADS[TRAIN_WORKLOAD]
    net = w["net"]
    mesh = S.make_mesh(w["shape"])
    res = {}
    for name, prec in (("fp16", nif.NIF_FP16), ("bf16", nif.NIF_BF16)):
        h = nif.Nif(net, mesh, precision=prec, seed=1234 + rank, flags=nif.NIF_FLAG_MIXED_TRAINING)
        stream = torch.cuda.current_stream()
        seed0 = 91 + 1000003 * rank
        nif.nif_train_steps(h.h, args.warmup, N_SEG, N_POSES, seed0, lr_grid=1e-2, lr_mlp=1e-3)
        torch.cuda.synchronize()
        nif.nif_profile(h.h, 1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        nif.nif_train_steps(h.h, args.steps, N_SEG, N_POSES, seed0 + args.warmup, lr_grid=1e-2, lr_mlp=1e-3)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        prof = nif.nif_profile_read(h.h)
        nif.nif_profile(h.h, 0)
        loss, _ = nif.nif_train_step(h.h, N_SEG, N_POSES, seed0 + 99999, want_loss=True)
        scale, skipped = nif.nif_loss_scale(h.h)
        tot = sum(v[0] for v in prof.values())
        stages = {k: {"ms_per_step": v[0] / max(args.steps, 1), "share": v[0] / tot if tot else None,
                      **({"overlapped": True} if k in OVERLAPPED else {})}
                  for k, v in sorted(prof.items(), key=lambda kv: -kv[1][0])}
        for k in ("encode_fwd", "encode_bwd"):
            if k in stages:
                amount = _stage_work(net, k, N_SEG)[0]
                if k == "encode_fwd":       # FP16 table corners, 16-bit feature rows
                    P, L = net.n_terms, net.levels
                    amount = N_SEG * (2 * P * L * 8 * 4 + 32 + net.in_dim * 2)
                stages[k]["GB/s"] = amount / (stages[k]["ms_per_step"] / 1e3) / 1e9
                stages[k]["frac_hbm"] = stages[k]["GB/s"] / hbm
        res[name] = {"value": args.steps * N_SEG / (ms / 1e3), "unit": "segments/s", "ms_per_step": ms / args.steps,
                     "loss_scale": scale, "skipped_steps": skipped, "loss": list(loss), "kernels": stages}
        h.close()
    return res


def run_train_det(args, nif, S, dev, rank):
    """The FP32 training step of the same workload with NIF_KNOB_DETERMINISTIC
    (order-free gradient sums: 64-bit fixed-point table gradient, per-range
    weight gradients added in order): segments/s, ms per step and the
    encoding backward's share, over at most 20 steps."""
    import torch
    w = S.WORKLOADS[TRAIN_WORKLOAD]
    h = nif.Nif(w["net"], S.make_mesh(w["shape"]), seed=1234 + rank)
    nif.nif_set_knob(h.h, nif.NIF_KNOB_DETERMINISTIC, 1)
    stream = torch.cuda.current_stream()
    k = max(1, min(args.steps, 20))
    seed0 = 77 + 1000003 * rank
    nif.nif_train_steps(h.h, args.warmup, N_SEG, N_POSES, seed0, lr_grid=1e-2, lr_mlp=1e-3)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    nif.nif_train_steps(h.h, k, N_SEG, N_POSES, seed0 + args.warmup, lr_grid=1e-2, lr_mlp=1e-3)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    nif.nif_profile(h.h, 1)
    nif.nif_profile_filter(h.h, ["encode_bwd"])
    nif.nif_train_steps(h.h, k, N_SEG, N_POSES, seed0 + args.warmup + k, lr_grid=1e-2, lr_mlp=1e-3)
    torch.cuda.synchronize()
    prof = nif.nif_profile_read(h.h)
    nif.nif_profile(h.h, 0)
    h.close()
    bwd = prof.get("encode_bwd", (0.0,))[0] / k
    return {"value": k * N_SEG / (ms / 1e3), "unit": "segments/s", "ms_per_step": ms / k, "steps": k,
            "encode_bwd_ms_per_step": bwd}


def h_seg_per_ray(h, nif):
    """Segments per ray of the training ray distribution (count through the C ABI)."""
    rays = nif.nif_sample_rays(h.h, 4242, 0, 8192)
    _, segs = nif.nif_segments(h.h, [(0.0, 0.0, 0.0)], rays)
    return segs.shape[0] / 8192


def run_traversal(args, nif, S, dev):
    """Segment generation two ways on the same rays and pose: the library's
    enumeration of every occupied hull through the octree, and the paper's
    traversal (Sec. 2.1: BVH first hit, then the walk through the exit faces of
    the deformed voxels, a new BVH query after leaving the grid); plus the
    walk's first BVH query alone, the BVH part the paper quotes at 2-3 % of its
    cost (Sec. 3.2). Count passes only (per-ray counts, which the segment lists
    are written from), GPU time of each stage from the library's profile."""
    import ctypes
    import torch
    out = {}
    for wname, n in ((QUERY_WORKLOAD, 1 << 22), (TRAIN_WORKLOAD, 1 << 20)):
        w = S.WORKLOADS[wname]
        mesh = S.make_mesh(w["shape"])
        rays = torch.from_numpy(S.sphere_rays(n, seed=950)).to(dev)
        p, n_inst = nif._poses(S.poses(1, seed=951))
        h = nif.Nif(w["net"], mesh, seed=31)
        offs = torch.zeros(n + 1, dtype=torch.int32, device=dev)
        total = nif._i64()
        L = nif.lib()

        def enumerate_():
            nif._check(h.h, L.nif_segments(h.h, p, n_inst, nif._ptr(rays), None, n, nif._ptr(offs), None, 0,
                                           ctypes.byref(total), None))

        def walk(flags):
            nif._check(h.h, L.nif_segments_walk(h.h, p, n_inst, nif._ptr(rays), None, n, nif._ptr(offs), None, 0,
                                                ctypes.byref(total), flags, None))

        enumerate_()
        n_seg = total.value
        walk(0)
        n_seg_walk = total.value          # equal to n_seg but for rays through tied hull decisions
        walk(nif.NIF_WALK_FIRST_HIT)
        reps = 3
        nif.nif_profile(h.h, 1)
        for _ in range(reps):
            enumerate_()
            walk(0)
            walk(nif.NIF_WALK_FIRST_HIT)
        prof = nif.nif_profile_read(h.h)
        nif.nif_profile(h.h, 0)
        h.close()
        # the same enumeration with the faces read as bilinear patches
        import dataclasses
        hb = nif.Nif(dataclasses.replace(w["net"], faces="bilinear"), mesh, seed=31)
        nif._check(hb.h, L.nif_segments(hb.h, p, n_inst, nif._ptr(rays), None, n, nif._ptr(offs), None, 0,
                                        ctypes.byref(total), None))
        n_seg_bil = total.value
        nif.nif_profile(hb.h, 1)
        for _ in range(reps):
            nif._check(hb.h, L.nif_segments(hb.h, p, n_inst, nif._ptr(rays), None, n, nif._ptr(offs), None, 0,
                                            ctypes.byref(total), None))
        prof_b = nif.nif_profile_read(hb.h)
        nif.nif_profile(hb.h, 0)
        hb.close()
        ms = {k: v[0] / reps for k, v in prof.items()}
        e, wk, lt, f = ms.get("seg_count", 0.0), ms.get("walk_count", 0.0), ms.get("walk_lattice", 0.0), ms.get(
            "walk_first", 0.0)
        eb = prof_b.get("seg_count", (0.0,))[0] / reps
        out[wname] = {"rays": n, "segments": n_seg, "segments_walk": n_seg_walk, "enumerate_ms": e, "walk_ms": wk, "walk_lattice_ms": lt,
                      "bvh_first_hit_ms": f, "walk_over_enumerate": (wk + lt) / e if e else None,
                      "bvh_share_of_walk": f / (wk + lt) if wk else None,
                      "segments_bilinear_faces": n_seg_bil, "enumerate_bilinear_faces_ms": eb}
    return out


def run_query(args, nif, S, dev, rank):
    import torch
    w = S.WORKLOADS[QUERY_WORKLOAD]
    net = w["net"]
    mesh = S.make_mesh(w["shape"])
    n = args.query_rays or w["n_rays"]
    rays = torch.from_numpy(S.sphere_rays(n, seed=900 + rank)).to(dev)
    pose = S.poses(1, seed=901 + rank)
    res = {"workload": QUERY_WORKLOAD, "rays_per_step": n}
    hbm = _peaks()[0]
    precs = [(nm, {"fp32": nif.NIF_FP32, "bf16": nif.NIF_BF16, "fp16": nif.NIF_FP16}[nm])
             for nm in args.query_prec.split(",")]
    # the BF16 query also as two kernels per chunk (encoding, then the MLP
    # from a global feature buffer) beside the fused default
    if "bf16" in args.query_prec.split(","):
        precs.append(("bf16_two_kernels", nif.NIF_BF16))
    for name, prec in precs:
        try:
            h = nif.Nif(net, mesh, precision=prec, seed=31)
            if name.endswith("_two_kernels"):
                nif.nif_set_knob(h.h, nif.NIF_KNOB_QUERY_FUSED, 0)
            ws_, s_ = S.init_params(net, seed=32)[1:]
            ws_[-1][0, :] *= 4.0
            h.set_params(S.init_params(net, seed=32)[0], ws_, s_)
            hits = torch.zeros((n, 8), dtype=torch.float32, device=dev)
            for i in range(max(args.warmup, 1)):
                nif.nif_query(h.h, pose, rays, hits=hits)
            torch.cuda.synchronize()
            nif.nif_profile(h.h, 1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            k = max(2, args.steps // 2)
            e0.record()
            for i in range(k):
                nif.nif_query(h.h, pose, rays, hits=hits)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / k
            prof = nif.nif_profile_read(h.h)
            nif.nif_profile(h.h, 0)
            _, segs = nif.nif_segments(h.h, pose, rays)
            n_seg = int(segs.shape[0])
            del segs
            st = {kk: v[0] / k for kk, v in prof.items()}
            res["segments_per_step"] = n_seg
            res[name] = {"queries_per_s": n / (ms / 1e3), "ms_per_query_batch": ms, "stages_ms": st,
                         "hit_rate": float((hits[:, 7].view(torch.int32) & 0xff).ne(0).float().mean().item())}
            if "encode_mlp_tc" in st:
                # fused kernel: per segment 2 P L 8 corner rows gathered (repeated
                # entry points once), 32 B of segment read, 64 B of outputs written
                gat = n_seg * 2 * net.n_terms * net.levels * 8
                res[name]["encode_mlp"] = {"ms": st["encode_mlp_tc"], "corner_gathers_G_per_s":
                                           gat / (st["encode_mlp_tc"] / 1e3) / 1e9,
                                           "hbm_bytes_per_segment": 96, "feature_bytes_to_hbm": 0}
            if "mlp_fwd_tc" in st:
                by = n_seg * (net.in_dim * 2 + 16 * 4)          # 16-bit features in, FP32 outputs out
                gbs = by / (st["mlp_fwd_tc"] / 1e3) / 1e9
                res[name]["mlp_roofline"] = {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s",
                                             "frac": gbs / hbm, "bytes_per_segment": net.in_dim * 2 + 64}
            h.close()
        except nif.NifError as e:
            res[name] = {"unavailable": str(e)}
    return res


def run_field(args, nif, S, dev, rank):
    """The learned deformation field: (1) fitting steps (nif_field_step) on the
    training workload's network and shape, 4 instances with their own 9^3
    lattices under half of their target poses, 2^18 segments per step;
    (2) the BF16 query of the 128^3 torus (2^22 rays) through a 9^3 lattice,
    beside the same query without it."""
    import torch
    out = {}
    w = S.WORKLOADS[TRAIN_WORKLOAD]
    net = w["net"]
    h = nif.Nif(net, S.make_mesh(w["shape"]), seed=55)
    n_inst, G = 4, 9
    nif.nif_set_field(h.h, np.zeros((n_inst, G, G, G, 3), np.float32))
    target = S.poses(n_inst, seed=56)
    pose = (0.5 * target).astype(np.float32)
    per = int(N_SEG / n_inst / 4.0 * 1.3)
    rays = torch.from_numpy(S.sphere_rays(per * n_inst, seed=57 + rank)).to(dev)
    inst = torch.arange(0, per * n_inst + 1, per, dtype=torch.int32, device=dev)
    for i in range(max(args.warmup, 1)):
        nif.nif_field_step(h.h, pose, rays, N_SEG, target, inst_offsets=inst, lr_field=1e-3, want_loss=False)
    torch.cuda.synchronize()
    k = max(3, args.steps // 4)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for i in range(k):
        nif.nif_field_step(h.h, pose, rays, N_SEG, target, inst_offsets=inst, lr_field=1e-3, want_loss=False)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / k
    out["fit"] = {"workload": TRAIN_WORKLOAD, "instances": n_inst, "lattice": G, "segments_per_step": N_SEG,
                  "ms_per_step": ms, "segments_per_s": N_SEG / (ms / 1e3), "network": "frozen"}
    h.close()
    wq = S.WORKLOADS[QUERY_WORKLOAD]
    netq = wq["net"]
    n = args.query_rays or wq["n_rays"]
    rq = torch.from_numpy(S.sphere_rays(n, seed=900 + rank)).to(dev)
    pq = S.poses(1, seed=901 + rank)
    fld = np.random.default_rng(58).normal(size=(1, G, G, G, 3))
    res = {}
    for with_field in (False, True):
        hq = nif.Nif(netq, S.make_mesh(wq["shape"]), precision=nif.NIF_BF16, seed=31)
        if with_field:
            f = fld[0]
            lip = _field_lipschitz(f)
            nif.nif_set_field(hq.h, (fld * (0.5 / lip)).astype(np.float32))
        hits = torch.zeros((n, 8), dtype=torch.float32, device=dev)
        for i in range(max(args.warmup, 1)):
            nif.nif_query(hq.h, pq, rq, hits=hits)
        torch.cuda.synchronize()
        kq = max(2, args.steps // 4)
        e0.record()
        for i in range(kq):
            nif.nif_query(hq.h, pq, rq, hits=hits)
        e1.record()
        torch.cuda.synchronize()
        msq = e0.elapsed_time(e1) / kq
        res["with_field" if with_field else "without_field"] = {"ms_per_query_batch": msq,
                                                                "queries_per_s": n / (msq / 1e3)}
        nif.nif_sync_status(hq.h)
        hq.close()
    out["query_bf16"] = dict(res, workload=QUERY_WORKLOAD, rays=n, lattice=G, lipschitz=0.5)
    return out


def _field_lipschitz(f):
    """Lipschitz bound of a [G,G,G,3] lattice as the library defines it (for
    scaling a random benchmark field to a chosen bound)."""
    G = f.shape[0]
    m = []
    for ax in (2, 1, 0):
        e = np.linalg.norm(np.diff(f, axis=ax), axis=-1) * (G - 1)
        for o in [o for o in (0, 1, 2) if o != ax]:
            e = np.maximum(np.take(e, range(0, e.shape[o] - 1), axis=o), np.take(e, range(1, e.shape[o]), axis=o))
        m.append(e)
    return float(np.sqrt(sum(x ** 2 for x in m)).max())


BATCH_WORKLOAD = "torus16x64_batch"
FRAME_WORKLOAD = "ellipsoids256_frame"


def run_batch(args, nif, S, dev, rank):
    """Batched queries of 64 deforming instances with Zipf ray counts (about
    2^22 rays), one autotuned CUDA-graph replay per step: mixed precision
    (BF16 MLP, FP16 tables; the encoding inside the MLP kernel, and as two
    kernels per chunk) and, on the same rays and poses, FP32."""
    import torch
    w = S.WORKLOADS[BATCH_WORKLOAD]
    net = w["net"]
    mesh = S.make_mesh(w["shape"])
    counts = S.zipf_ray_counts(w["n_inst"], seed=700 + rank)
    rays_np = np.concatenate([S.sphere_rays(int(c), seed=1000 * rank + 710 + i) for i, c in enumerate(counts)])
    inst = np.concatenate([[0], np.cumsum(counts)]).astype(np.int32)
    n = len(rays_np)
    rays = torch.from_numpy(rays_np).to(dev)
    it = torch.from_numpy(inst).to(dev)
    rng = np.random.default_rng(720 + rank)
    poses = [rng.uniform(-1, 1, (w["n_inst"], 3)).astype(np.float32) for _ in range(args.steps + args.warmup)]
    res = None
    for name, prec in (("bf16", nif.NIF_BF16), ("bf16_two_kernels", nif.NIF_BF16), ("fp32", nif.NIF_FP32)):
        h = nif.Nif(net, mesh, precision=prec, seed=41)
        if name.endswith("_two_kernels"):           # encoding and MLP as two kernels per chunk
            nif.nif_set_knob(h.h, nif.NIF_KNOB_QUERY_FUSED, 0)
        hits = torch.zeros((n, 8), dtype=torch.float32, device=dev)
        t0 = time.perf_counter()
        plan = nif.QueryPlan(h.h, poses[0], rays, hits, inst_offsets=it, autotune=True)
        tune_s = time.perf_counter() - t0
        for i in range(args.warmup):
            plan.run(poses[i])
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for i in range(args.steps):
            plan.run(poses[args.warmup + i])
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        nif.nif_sync_status(h.h)
        ent = {"queries_per_s": n / (ms / 1e3), "ms_per_batch": ms, "knobs": plan.info(), "autotune_s": tune_s,
               "hit_rate": float((hits[:, 7].view(torch.int32) & 0xff).ne(0).float().mean().item())}
        if res is None:
            offs = torch.zeros(n + 1, dtype=torch.int32, device=dev)
            total = nif._i64()
            p_, n_inst = nif._poses(poses[args.warmup])
            nif._check(h.h, nif.lib().nif_segments(h.h, p_, n_inst, nif._ptr(rays), nif._ptr(it), n, nif._ptr(offs),
                                                   None, 0, nif.ctypes.byref(total), None))
            res = {"workload": BATCH_WORKLOAD, "instances": int(w["n_inst"]), "rays_per_step": int(n),
                   "segments_per_step": int(total.value),
                   "rays_per_instance_min_max": [int(counts.min()), int(counts.max())], "precision": "bf16",
                   "queries_per_s": ent["queries_per_s"], "ms_per_batch": ms, "graph": True, "knobs": ent["knobs"],
                   "autotune_s": tune_s, "hit_rate": ent["hit_rate"]}
        res[name] = ent
        plan.close()
        h.close()
    res["mixed_over_fp32"] = res["bf16"]["queries_per_s"] / res["fp32"]["queries_per_s"]
    return res


def run_frame(args, nif, S, dev):
    """Animated frame loop: 16 deforming ellipsoid-union instances at 256^3
    (T = 2^21, MLP 4 x 64, BF16 mixed precision) on a 4 x 4 screen grid.
    Per frame: new sinusoidal poses, 1920x1080 primary rays (one CUDA-graph
    query plan), shadow rays toward a directional light from the primary hits
    and an occlusion-only query plan, and one pose-fitting gradient step of
    all 16 pose estimates on every 32nd primary ray (the task-loss gradient
    w.r.t. the deformation parameters). Before the loop the network trains
    for 20k steps of 2^18 segments, as the workload states (timed as train
    samples/s)."""
    import torch
    w = S.WORKLOADS[FRAME_WORKLOAD]
    net = w["net"]
    t_setup = time.perf_counter()
    mesh = S.make_mesh(w["shape"])
    h = nif.Nif(net, mesh, precision=nif.NIF_BF16, seed=51, flags=nif.NIF_FLAG_MIXED_TRAINING)
    setup_s = time.perf_counter() - t_setup
    n_inst, frames = w["n_inst"], args.frames
    stream = torch.cuda.current_stream()
    # ---- pre-training (mixed BF16, 2^18 segments, 16 poses) ----
    for i in range(2):
        nif.nif_train_step(h.h, N_SEG, N_POSES, 9000 + i, lr_grid=1e-2, lr_mlp=5e-3, want_loss=False)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    done = 0
    while done < args.frame_pretrain:       # pipelined steps, 1000 per call
        k = min(1000, args.frame_pretrain - done)
        nif.nif_train_steps(h.h, k, N_SEG, N_POSES, 9100 + done, lr_grid=1e-2, lr_mlp=5e-3)
        done += k
    e1.record(stream)
    torch.cuda.synchronize()
    train_ms = e0.elapsed_time(e1) / max(args.frame_pretrain, 1)
    loss, _ = nif.nif_train_step(h.h, N_SEG, N_POSES, 9999, lr_grid=1e-2, lr_mlp=5e-3, want_loss=True)
    # ---- frame inputs ----
    rays_np, offs_np = S.camera_rays(w["width"], w["height"], grid=4)
    n = len(rays_np)
    prim = torch.from_numpy(rays_np).to(dev)
    it = torch.from_numpy(offs_np).to(dev)
    prim_hits = torch.zeros((n, 8), dtype=torch.float32, device=dev)
    shadow = torch.zeros_like(prim)
    shadow_hits = torch.zeros((n, 8), dtype=torch.float32, device=dev)
    per = n // n_inst
    fit_idx = np.concatenate([np.arange(i * per, (i + 1) * per, 32) for i in range(n_inst)])
    fit_rays = prim[torch.from_numpy(fit_idx).to(dev)].contiguous()
    fit_off = torch.from_numpy((np.arange(n_inst + 1) * (len(fit_idx) // n_inst)).astype(np.int32)).to(dev)
    poses = S.animated_poses(n_inst, max(frames, 1) + args.warmup, seed=1301)
    light = (0.4, 0.3, 0.87)
    t0 = time.perf_counter()
    plan_p = nif.QueryPlan(h.h, poses[0], prim, prim_hits, inst_offsets=it, autotune=True)
    nif.nif_shadow_rays(h.h, prim, prim_hits, light, eps=1e-3, tmax=4.0, out=shadow)
    plan_s = nif.QueryPlan(h.h, poses[0], shadow, shadow_hits, inst_offsets=it, flags=nif.NIF_SHADOW_ONLY,
                           autotune=False)
    plan_s_ms = (time.perf_counter() - t0) * 1e3
    lim = np.array([1.0, 4.0, 1.0], np.float32)          # |bend|, |twist|, |taper| bounds of the deformation
    est = np.clip(0.8 * poses[0] + 0.1, -lim, lim)       # pose estimates start off the animation
    dposes = torch.zeros((n_inst, 3), dtype=torch.float32, device=dev)
    fit_seg = 1 << 17

    def frame(f):
        nonlocal est
        plan_p.run(poses[f])
        nif.nif_shadow_rays(h.h, prim, prim_hits, light, eps=1e-3, tmax=4.0, out=shadow)
        plan_s.run(poses[f])
        nif.nif_pose_step(h.h, est, fit_rays, fit_seg, inst_offsets=fit_off, dposes=dposes)
        est = np.clip(est - 0.05 * dposes.cpu().numpy(), -lim, lim)     # host update of the 48 estimates

    for f in range(args.warmup):
        frame(f)
    torch.cuda.synchronize()
    nif.nif_profile(h.h, 1)
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    for f in range(frames):
        frame(args.warmup + f)
    f1.record(stream)
    torch.cuda.synchronize()
    ms = f0.elapsed_time(f1)
    prof = nif.nif_profile_read(h.h)
    nif.nif_profile(h.h, 0)
    nif.nif_sync_status(h.h)
    hit_rate = float((prim_hits[:, 7].view(torch.int32) & 0xff).ne(0).float().mean().item())
    shadow_rate = float((shadow_hits[:, 7].view(torch.int32) & 0xff).ne(0).float().mean().item())
    res = {"workload": FRAME_WORKLOAD, "instances": n_inst, "resolution": [w["width"], w["height"]],
           "frames": frames, "precision": "bf16", "frames_per_s": frames / (ms / 1e3), "ms_per_frame": ms / frames,
           "queries_per_s": frames * 2 * n / (ms / 1e3), "rays_per_frame": 2 * n,
           "pose_fit_rays_per_frame": int(len(fit_idx)), "primary_hit_rate": hit_rate,
           "shadowed_fraction": shadow_rate,
           "stages_ms_per_frame": {k: v[0] / max(frames, 1) for k, v in
                                   sorted(prof.items(), key=lambda kv: -kv[1][0])},
           "pretrain": {"steps": args.frame_pretrain, "segments_per_step": N_SEG, "ms_per_step": train_ms,
                        "train_samples_per_s": N_SEG / (train_ms / 1e3), "loss": list(loss)},
           "setup_s": setup_s, "plans_ms": plan_s_ms}
    if args.frame_pretrain < 20000:
        res["note"] = "pre-training is shortened from 20k steps; query and fitting cost do not depend on it"
    plan_s.close()
    plan_p.close()
    h.close()
    return res


def run_precision(args, nif, S, dev, workloads=("torus16_fwd", "torus128_query")):
    """Per-output error of the BF16 / FP16 query paths against the FP32 GPU
    path on a trained network: the config-1 torus network (L = 8, T = 2^14,
    MLP 288-32-32-16) trained on the GPU at 16^3 voxels (FP32, 4000 steps of
    2^16 segments, poses U[-1,1]^3), then queried with 2^22 rays on each
    workload's voxel grid: 16^3, and the 128^3 of the precision workload
    (the same encoding and MLP; a network trained at 128^3 predicts no hit,
    because its finest level has 68 cells per axis). The comparison with the
    FP64 oracle is tests/test_gpu_precision.py."""
    import torch
    w = S.WORKLOADS["torus16_fwd"]
    mesh = S.make_mesh(w["shape"])
    t0 = time.perf_counter()
    h32 = nif.Nif(w["net"], mesh, precision=nif.NIF_FP32, seed=51)
    for step in range(4000):
        loss, _ = nif.nif_train_step(h32.h, 1 << 16, 16, 5000 + step, lr_grid=1e-2, lr_mlp=5e-3,
                                     want_loss=(step == 3999))
    train_s = time.perf_counter() - t0
    tables, ws, s = h32.get_params()
    h32.close()
    pose = S.poses(1, seed=52)[0]          # U[-1,1]^3, the training distribution

    def fields(hits):
        a = hits.cpu().numpy().view(nif.HIT_DTYPE).reshape(-1)
        return (a["hit"] > 0, a["D"].astype(np.float64), a["n"].astype(np.float64), a["albedo"].astype(np.float64),
                a["material"])

    def errs(ref, got, N):
        # outputs compared where both first hits lie in the same segment
        # (|dD| < half a voxel); a flip on an earlier segment moves the hit by
        # about a voxel and is counted in same_first_segment instead
        h0, d0, n0, a0, m0 = ref
        h1, d1, n1, a1, m1 = got
        both = h0 & h1
        same = both.copy()
        same[both] = np.abs(d0[both] - d1[both]) < 0.5 / N
        ang = np.degrees(np.arccos(np.clip((n0[same] * n1[same]).sum(1), -1, 1)))
        dd = np.abs(d0[same] - d1[same])
        da = np.abs(a0[same] - a1[same]).max(1)
        return {"hit_iou": float((h0 & h1).sum() / max(1, (h0 | h1).sum())),
                "same_first_segment": float(same.sum() / max(1, (h0 & h1).sum())),
                "D_abs_median": float(np.median(dd)) if same.any() else None,
                "D_abs_p99": float(np.percentile(dd, 99)) if same.any() else None,
                "normal_deg_median": float(np.median(ang)) if same.any() else None,
                "normal_deg_p99": float(np.percentile(ang, 99)) if same.any() else None,
                "albedo_abs_p99": float(np.percentile(da, 99)) if same.any() else None,
                "material_acc": float((m0[same] == m1[same]).mean()) if same.any() else None}

    rays_np = S.sphere_rays(1 << 22, seed=53)
    rays = torch.from_numpy(rays_np).to(dev)
    res = {"network": "torus16_fwd trained at 16^3", "train_steps": 4000, "train_s": train_s,
           "train_loss": [float(x) for x in loss], "rays": 1 << 22}
    for wname in workloads:
        net = S.WORKLOADS[wname]["net"]
        hs = {}
        for name, p in (("fp32", nif.NIF_FP32), ("bf16", nif.NIF_BF16), ("fp16", nif.NIF_FP16)):
            hs[name] = nif.Nif(net, mesh, precision=p, seed=51)
            hs[name].set_params(tables, ws, s)
        got = {k: fields(nif.nif_query(hh.h, [pose], rays)) for k, hh in hs.items()}
        for hh in hs.values():
            hh.close()
        res[wname] = {"voxels": f"{net.voxel_res}^3", "hit_rate_fp32": float(got["fp32"][0].mean()),
                      "vs_fp32_gpu_all_rays": {k: errs(got["fp32"], got[k], net.voxel_res) for k in ("bf16", "fp16")}}
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline leg")
    ap.add_argument("--no-query", action="store_true", help="skip the inference-query measurement")
    ap.add_argument("--only-query", action="store_true", help="measure only the inference queries (profiling aid)")
    ap.add_argument("--query-rays", type=int, default=0, help="rays per query batch (default: the workload's 2^22)")
    ap.add_argument("--query-prec", default="fp32,bf16,fp16", help="comma list of query precisions")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched 64-instance query measurement")
    ap.add_argument("--no-precision", action="store_true", help="skip the per-output precision study")
    ap.add_argument("--no-mixed", action="store_true", help="skip the mixed-precision training measurement")
    ap.add_argument("--no-det", action="store_true", help="skip the deterministic-gradient training measurement")
    ap.add_argument("--no-frame", action="store_true", help="skip the animated frame loop")
    ap.add_argument("--no-traversal", action="store_true", help="skip the enumeration vs exit-face walk comparison")
    ap.add_argument("--no-field", action="store_true", help="skip the learned deformation field measurement")
    ap.add_argument("--only-field", action="store_true", help="measure only the learned deformation field (profiling aid)")
    ap.add_argument("--only-batch", action="store_true", help="measure only the batched query (profiling aid)")
    ap.add_argument("--only-traversal", action="store_true", help="measure only the traversal comparison (profiling aid)")
    ap.add_argument("--log", default="", help="also append the JSON line to this JSON-lines file")
    ap.add_argument("--frames", type=int, default=120, help="frames of the animated frame loop")
    ap.add_argument("--frame-pretrain", type=int, default=20000, help="training steps before the frame loop")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.only_query:
        import torch
        torch.cuda.set_device(0)
        from paper_2604_24666_gb300 import build as B
        B.build()
        from paper_2604_24666_gb300 import nif, synth as S
        print(json.dumps({"query": run_query(args, nif, S, torch.device("cuda:0"), 0)}), flush=True)
        return 0
    if args.only_batch:
        import torch
        torch.cuda.set_device(0)
        from paper_2604_24666_gb300 import build as B
        B.build()
        from paper_2604_24666_gb300 import nif, synth as S
        print(json.dumps({"batch": run_batch(args, nif, S, torch.device("cuda:0"), 0)}), flush=True)
        return 0
    if args.only_field:
        import torch
        torch.cuda.set_device(0)
        from paper_2604_24666_gb300 import build as B
        B.build()
        from paper_2604_24666_gb300 import nif, synth as S
        print(json.dumps({"field": run_field(args, nif, S, torch.device("cuda:0"), 0)}), flush=True)
        return 0
    if args.only_traversal:
        import torch
        torch.cuda.set_device(0)
        from paper_2604_24666_gb300 import build as B
        B.build()
        from paper_2604_24666_gb300 import nif, synth as S
        print(json.dumps({"traversal": run_traversal(args, nif, S, torch.device("cuda:0"))}), flush=True)
        return 0
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
