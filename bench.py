#!/usr/bin/env python3
"""Benchmark: voxel-samples/s of batched partial objective evaluation.

One step = one GOMEA generation of partial evaluations (Sec. 2.2) of the
dual simplex-mesh registration objectives (Sec. 2.3) over the whole
population: for every wave of independent FOS groups, propose, evaluate the
touched tetrahedra of every (group, candidate) trial, accept-if-improves and
commit -- one CUDA-graph launch.  One voxel-sample is one (candidate,
direction, voxel) squared-difference term.

Default workload (batch64): 64 independent registration problems of uneven
size (edge 32..128 voxels, meshes 4^3..9^3 points, populations 64..512),
one generation of single-point FOS partial evaluations over all of them per
step, one CUDA graph.  Secondary workloads: --workload ellipsoid64 | ct |
ct_coarse | sphere16 (single problems), learned, mlp_forward, cube_multires.

Besides the counted samples the line reports the samples the raster kernels
actually mapped and sampled (executed); the rest were settled exactly without
sampling (rows of 0 against an all-0 partner region), and the roofline
fraction is taken on the executed ones.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank runs an independent replica (its own
population; there is no data-path exchange) and rank 0 prints one JSON line
with the whole-job throughput.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "voxel-samples/s of batched partial objective eval"
UNIT = "voxel-samples/s"
# Minimal FP32 lane operations one voxel-sample needs by definition (affine
# map 9, floor/fraction 6, cell index 2, trilinear 7 lerps = 14, difference
# and square 2, black test 3, accumulate 1).
ALG_OPS_PER_SAMPLE = 37
FALLBACK_HBM_GBS = 6800.0
# DRAM bytes (read + write) of one fast raster-pass launch (one wave of the
# generation, the mean over the 4 waves), from the full-size ncu capture of
# the current kernel (1-pass metrics, caches not flushed) summarised under
# profiles/, per (workload, storage); None for workloads without one.
FAST_PASS_DRAM_BYTES = {("batch64", "f32"): 23.94e9, ("ct", "f32"): 2.498e9, ("ellipsoid64", "f32"): 5.3e6}
# Instruction-issue utilisation of the fast raster pass (smsp__issue_active,
# share of cycles in which a warp instruction issued), from the ncu captures
# of the current kernel summarised under profiles/: the resource that binds
# it (its ALU fraction counts only the 37 sampling operations per executed
# sample, not the rasterisation instructions).
FAST_PASS_ISSUE_ACTIVE = {("batch64", "f32"): 0.798, ("ct", "f32"): 0.782}


def reduce_over_ranks(total_s, samples, dist, device):
    """Whole-job figures over the replicas: the slowest rank's time and the
    summed samples (each rank evaluates its own independent population)."""
    if dist is None:
        return float(total_s), float(samples)
    import torch

    t = torch.tensor([float(total_s)], dtype=torch.float64, device=device)
    n = torch.tensor([float(samples)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(n, op=dist.ReduceOp.SUM)
    return float(t.item()), float(n.item())


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def workload(name, seed):
    from paper_2202_11001_gb300 import synth

    if name == "ellipsoid64":
        pr = synth.ellipsoid_pair(seed=1 + seed, C=128)
        pr["sigma"] = 1.5
        pr["desc"] = ("ellipsoid64: 64^3 float32 pair (3 ellipsoids 0.3/0.6/1.0 on 0, target warped by 4 "
                      "Gaussian bumps <= 6 vox), 5^3-point meshes (384 tets), 20 guidance pairs, population 128, "
                      "one generation over 125 single-point FOS groups")
    elif name == "ct":
        pr = synth.ct_phantom(seed=3 + seed, C=512)
        pr["sigma"] = 2.0
        pr["desc"] = ("ct256: 256x256x96 CT phantom mapped to [0,1], spacing 1x1x3 mm, 10^3-point meshes "
                      "(4374 tets), 200 guidance pairs, population 512, one generation over 1000 single-point groups")
    elif name == "ct_coarse":
        pr = synth.ct_phantom(seed=3 + seed, C=512, level="coarse")
        pr["sigma"] = 0.5
        pr["desc"] = "ct64 coarse level: 64x64x24, spacing 4x4x12 mm, 10^3-point meshes, population 512"
    elif name == "sphere16":
        pr = synth.sphere_pair(seed=seed, C=10)
        pr["sigma"] = 0.4
        pr["desc"] = "sphere16: 16^3 float32 pair, 3^3-point meshes (48 tets), 5 guidance pairs, population 10"
    else:
        raise SystemExit("unknown workload " + name)
    return pr


BATCH_DESC = ("batch64: 64 independent problems built like the mid ellipsoid configuration (edge U{32..128} "
              "voxels, meshes U{4..9}^3 points, populations U{64..512}, 8 guidance pairs each), one generation of "
              "single-point FOS partial evaluations, one persistent launch per kernel and wave, one CUDA graph "
              "per generation")


def batch_inputs(seed, n_problems=0):
    """The 64 seeded problems, their FOS groups and per-problem proposal
    offsets of one generation."""
    from paper_2202_11001_gb300 import synth

    probs = synth.batch_problems(seed=seed)
    if n_problems:
        probs = probs[:n_problems]
    groups, dels = [], []
    for i, pr in enumerate(probs):
        C = pr["coords"].shape[0]
        pr["sigma"] = 0.1 * pr["img"][0].shape[0] / (pr["mesh"][0] - 1)
        gr = synth.single_point_fos(pr["mesh"])
        groups.append(gr)
        dels.append(deltas_for(pr, gr, C, np.random.default_rng(500 + i)))
    return probs, groups, dels


def build_batch(probs, groups, storage, stream):
    import torch

    from paper_2202_11001_gb300 import dmr

    gs = []
    for pr, gr in zip(probs, groups):
        C = pr["coords"].shape[0]
        g = dmr.Problem(pr["img"][0], pr["img"][1], *pr["spacing"], pr["mesh"], guide=pr["guide"],
                        model=dmr.LINEAR, storage=storage, max_candidates=C, stream=stream)
        g.eval_full(torch.from_numpy(pr["coords"]).cuda())
        g.set_fos(gr)
        gs.append(g)
    return gs


def batch_tile(gs, probs, tile):
    """The raster tile of a batch plan: fixed (--tile) or autotuned on the
    problem with the most work; plans take the first problem's tile."""
    if tile:
        w, v = (int(x) for x in tile.lower().split("x"))
        table = {}
    else:
        big = max(range(len(gs)), key=lambda i: probs[i]["coords"].shape[0] * gs[i].ntet)
        w, v, table = gs[big].autotune()
    gs[0].set_tile(w, v)
    return w, v, table


def time_plan(plan, steps, flush, ev0, ev1):
    """Device time of `steps` plan runs (L2 flushed before each, outside the
    event bracket): per-step ms and summed raster-kernel ms."""
    import torch

    step_ms, raster_ms = [], 0.0
    for _ in range(steps):
        flush.zero_()
        ev0.record()
        plan.run()
        ev1.record()
        torch.cuda.synchronize()
        step_ms.append(ev0.elapsed_time(ev1))
        raster_ms += plan.kernel_ms()[1]
    return step_ms, raster_ms


def batch_counts(gs):
    c = e = 0
    for g in gs:
        a, b = g.sample_counts(reset=True)
        c += a
        e += b
    return c, e


def cpu_baseline_batch(probs, groups, min_s=10.0, max_s=30.0, n_probs=4, n_cand=16):
    """The FP64 oracle as it stands, on the host cores, on a bounded sample of
    the batch workload: for n_probs problems spread over the batch, one wave of
    partial evaluations of its first n_cand candidates, cycled until about
    min_s of oracle time; samples = the oracle's own coverage counts."""
    from oracle import oracle as orc
    from paper_2202_11001_gb300 import synth

    cores = os.cpu_count() or 1
    orc.set_threads(cores)
    pick = [int(round(k * (len(probs) - 1) / max(1, n_probs - 1))) for k in range(n_probs)]
    work = []
    rng = np.random.default_rng(7)
    for q in pick:
        pr, gr = probs[q], groups[q]
        o = orc.Oracle(pr["img"][0], pr["img"][1], *pr["spacing"], pr["mesh"], guide=pr["guide"],
                       model=orc.LINEAR)
        nc = min(n_cand, pr["coords"].shape[0])
        o.eval_full(pr["coords"][:nc])
        m = pr["mesh"]
        # a wave of independent groups: points of one coordinate parity class
        w = np.array([g for g in range(len(gr)) if (g % m[0]) % 2 == 0 and ((g // m[0]) % m[1]) % 2 == 0
                      and (g // (m[0] * m[1])) % 2 == 0])
        gids = np.repeat(w, nc)
        cids = np.tile(np.arange(nc), len(w))
        cur = np.stack([o.coords(c) for c in range(nc)])
        tc = synth.trial_coords(cur, gr, gids, cids, pr["sigma"], m, rng)
        work.append((o, gr, gids, cids, tc))
    samples, secs, it, ntr = 0, 0.0, 0, 0
    cov = []
    while secs < min_s and secs < max_s:
        o, gr, gids, cids, tc = work[it % len(work)]
        t0 = time.perf_counter()
        o.eval_partial(gr, gids, cids, tc)
        secs += time.perf_counter() - t0
        if it < len(work):
            cov.append(sum(int(o.trial(k, cap=256)["cov"].sum()) for k in range(len(gids))))
        samples += cov[it % len(work)]
        ntr += len(gids)
        it += 1
    return {"value": samples / secs, "unit": UNIT, "cores": orc.max_threads(), "kind": "oracle",
            "sample": "%d wave evaluations over problems %s of the batch (one wave of single-point groups x the "
                      "first %d candidates each, cycled; %d trials, %d voxel-samples), FP64 C oracle, OpenMP over "
                      "trials, %.1f s" % (it, pick, n_cand, ntr, samples, secs)}


def run_batch(args):
    """--workload batch64 (the default): 64 independent problems of uneven
    size, one CUDA-graph generation over all of them per step."""
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2202_11001_gb300 import dmr

    # every replica its own seeded batch (independent populations, no exchange)
    probs, groups, dels = batch_inputs(2 + rank, args.problems)
    stream = torch.cuda.current_stream().cuda_stream
    cands = [np.arange(pr["coords"].shape[0], dtype=np.int32) for pr in probs]
    gs = build_batch(probs, groups, args.storage, stream)
    w, v, table = batch_tile(gs, probs, args.tile)
    bt = dmr.Batch(gs)
    plan = bt.plan_generation(cands, dels)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(args.warmup):
        plan.run()
    torch.cuda.synchronize()
    batch_counts(gs)
    sampler = ClockSampler(local)
    sampler.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    step_ms, raster_ms = time_plan(plan, args.steps, flush, ev0, ev1)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    counted, executed = batch_counts(gs)
    total_s = sum(step_ms) / 1e3
    total_s, all_samples = reduce_over_ranks(total_s, counted, dist, "cuda")
    value = all_samples / total_s
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count

    # e2e through the public API with host buffers: every step uploads each
    # problem's proposal offsets from pinned host memory into the plan
    # (dmr_plan_update), runs it (dmr_plan_run) and reads every problem's
    # objectives back (dmr_objectives_out)
    e2e = None
    if args.e2e_steps > 0:
        pins = [torch.from_numpy(np.ascontiguousarray(d)).pin_memory() for d in dels]
        plan.update(pins)
        plan.run()
        for g in gs:
            g.objectives()
        torch.cuda.synchronize()
        batch_counts(gs)
        d2h = 0
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            plan.update(pins)
            plan.run()
            d2h = 0
            for g in gs:
                d2h += g.objectives().nbytes
        dt = time.perf_counter() - t0
        ec, _ = batch_counts(gs)
        e2e = {"value": ec / dt, "unit": UNIT, "h2d_bytes_per_step": int(sum(p.numel() * 8 for p in pins)),
               "d2h_bytes_per_step": int(d2h), "steps": args.e2e_steps,
               "path": "dmr_plan_update (pinned host offsets of all 64 problems) + dmr_plan_run + "
                       "dmr_objectives_out per problem, per generation"}

    peaks, peak_kind = measured_peaks()
    clock_max = clocks.get("sm_max_mhz") or 2070.0
    alu_peak = n_sm * 128 * clock_max * 1e6 / 1e12
    raster_s = raster_ms / 1e3 / args.steps
    counted_step, executed_step = counted / args.steps, executed / args.steps
    bpv = 4 if args.storage == "f32" else 2
    hbm = float(peaks.get("hbm_gbs", FALLBACK_HBM_GBS))
    achieved = executed_step * ALG_OPS_PER_SAMPLE / raster_s / 1e12
    roofline = {"bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "T lane-op/s",
                "frac": achieved / alu_peak, "traffic": FAST_PASS_DRAM_BYTES.get(("batch64", args.storage)),
                "traffic_unit": "DRAM bytes per fast raster-pass launch (one wave), ncu",
                "kernel": "k_raster (rasterise + map + trilinear sample + SSD), fast and full-logic passes",
                "ops_per_sample": ALG_OPS_PER_SAMPLE, "basis": "executed samples",
                "peak_basis": "%d SMs x 128 FP32 lanes x %.0f MHz (max SM clock)" % (n_sm, clock_max),
                "raster_ms_per_step": raster_s * 1e3,
                "counted_samples_per_step": counted_step, "executed_samples_per_step": executed_step,
                "executed_frac": executed_step / max(counted_step, 1.0),
                "executed_samples_per_s_raster": executed_step / raster_s,
                "frac_on_counted_samples": counted_step * ALG_OPS_PER_SAMPLE / raster_s / 1e12 / alu_peak,
                "touched_bytes_frac_of_hbm": value * 2 * bpv / 1e9 / hbm,
                "touched_bytes_frac_of_hbm_executed": executed_step / (total_s / args.steps) * 2 * bpv / 1e9 / hbm,
                "hbm_peak_gbs": hbm, "hbm_peak_kind": peak_kind,
                "issue_active_ncu": FAST_PASS_ISSUE_ACTIVE.get(("batch64", args.storage))}
    launches = plan.launches
    plan.close()
    bt.close()

    variants = {}
    if not args.no_variants and world == 1:
        for st in ("f32", "bf16", "f16"):
            if st == args.storage:
                variants[st] = {"value": value, "executed_per_s": executed / (sum(step_ms) / 1e3)}
                continue
            gv = build_batch(probs, groups, st, stream)
            batch_tile(gv, probs, args.tile)
            bv = dmr.Batch(gv)
            pv = bv.plan_generation(cands, dels)
            for _ in range(3):
                pv.run()
            torch.cuda.synchronize()
            batch_counts(gv)
            ms, _ = time_plan(pv, max(3, args.steps // 2), flush, ev0, ev1)
            c, e = batch_counts(gv)
            variants[st] = {"value": c / (sum(ms) / 1e3), "executed_per_s": e / (sum(ms) / 1e3)}
            pv.close()
            bv.close()
            for g in gv:
                g.close()

    precision = None
    if not args.no_variants and rank == 0 and world == 1:
        # the first problem of the batch with an edge of at most 64 voxels
        q = next(i for i, pr in enumerate(probs) if pr["img"][0].shape[0] <= 64)
        precision = precision_report(probs[q], stream)
        precision["problem"] = probs[q]["name"]

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_batch(probs, groups)

    for g in gs:
        g.close()
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": args.storage,
                "data": "synthetic (64 seeded ellipsoid problems per replica)",
                "config": {"workload": BATCH_DESC, "storage": args.storage, "problems": len(probs),
                           "population_total": int(sum(len(c) for c in cands)),
                           "samples_per_step": counted_step, "executed_samples_per_step": executed_step,
                           "tile": {"warps_per_cta": w, "voxels_per_warp": v,
                                    "autotune_ms": {"%dx%d" % k: round(t, 4) for k, t in table.items()}},
                           "l2": "flushed before every timed step (256 MiB write outside the event bracket)",
                           "parallelism": "replicas" if world > 1 else "single GPU"},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
                "gpu_launches": launches * args.steps, "variants_samples_per_s": variants,
                "precision": precision}
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def run_learned(args):
    """--workload learned: the learned proposal on the coarse CT level (64x64x24,
    10^3-point meshes, population 512): collect elites from plain runs, train
    the network on the tensor cores, then compare hypervolume against
    evaluations with and without the learned sampler.  Also times the fused
    network forward over one generation's 512 x 1000 rows."""
    import torch

    from paper_2202_11001_gb300 import dmr, learned, synth

    pr = synth.ct_phantom(seed=3, C=512, level="coarse")
    rng = np.random.default_rng(0)
    t0 = time.time()
    X, Y = learned.collect(pr, seeds=[11, 12], generations=args.steps, sigma0=0.5, n_samples=100000, rng=rng)
    t_collect = time.time() - t0
    net = dmr.MLP(seed=1)
    t0 = time.time()
    losses = learned.train(net, X, Y, steps=600, batch=4096, lr=1e-3, rng=rng)
    torch.cuda.synchronize()
    t_train = time.time() - t0
    # inference throughput: features + fused forward for 512 x 1000 rows
    prob = learned.make_problem(pr)
    coords = torch.from_numpy(pr["coords"]).cuda()
    Xi = dmr.MLP.features(prob, coords)
    for _ in range(3):
        net.forward(Xi)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    reps = 10
    for _ in range(reps):
        net.forward(Xi)
    e1.record()
    torch.cuda.synchronize()
    fwd_ms = e0.elapsed_time(e1) / reps
    rows = Xi.shape[0]
    flop = rows * 2.0 * (256 * 128 + 128 * 128 * 2 + 128 * 16)
    peaks, kind = measured_peaks()
    peak = float(peaks.get("bf16_tflops", 1900.0)) if kind == "measured" else 1900.0
    ref, cmp_rows = learned.compare(pr, net, seeds=[21, 22, 23, 24, 25], generations=args.steps, sigma0=0.5,
                                    alpha=0.25)
    fin = lambda v: None if v is None or not np.isfinite(v) else float(v)  # None: the plain final HV is not reached
    for r in cmp_rows:
        r["plain_evals"], r["learned_evals"] = fin(r["plain_evals"]), fin(r["learned_evals"])
    pe = [r["plain_evals"] for r in cmp_rows]
    le = [r["learned_evals"] for r in cmp_rows]
    line = {"metric": "HV at fixed eval budget", "workload": "ct64 coarse level (64x64x24, 4x4x12 mm), 10^3-point "
            "meshes, population 512, 1000 single-point groups, learned sampler alpha 0.25",
            "generations": args.steps, "reference_point": ref.tolist(),
            "per_seed": [{k: v for k, v in r.items() if k != "curves"} for r in cmp_rows],
            "evals_to_plain_final_hv": {"plain": pe, "learned": le},
            "train": {"samples": int(X.shape[0]), "steps": 600, "batch": 4096, "loss_first": losses[0],
                      "loss_last": losses[-1], "seconds": t_train, "collect_seconds": t_collect},
            "forward": {"rows": rows, "ms": fwd_ms, "tflops": flop / fwd_ms / 1e9,
                        "roofline": {"bound": "tensor", "achieved": flop / fwd_ms / 1e9, "peak": peak,
                                     "unit": "TFLOP/s", "frac": flop / fwd_ms / 1e9 / peak,
                                     "peak_kind": kind}},
            "curves": {str(r["seed"]): {a: r["curves"][a] for a in ("plain", "learned")} for r in cmp_rows}}
    print(json.dumps(line), flush=True)
    return 0


def run_mlp_forward(args):
    """--workload mlp_forward: the fused tensor-core forward of the learned
    proposal network over one generation's rows (population 512 x 1000 points
    of the ct64 coarse level), features gathered on the GPU beforehand."""
    import torch

    from paper_2202_11001_gb300 import dmr, learned, synth

    pr = synth.ct_phantom(seed=3, C=512, level="coarse")
    net = dmr.MLP(seed=1)
    prob = learned.make_problem(pr)
    Xi = dmr.MLP.features(prob, torch.from_numpy(pr["coords"]).cuda())
    for _ in range(args.warmup):
        net.forward(Xi)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        net.forward(Xi)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    rows = Xi.shape[0]
    flop = rows * 2.0 * (256 * 128 + 128 * 128 * 2 + 128 * 16)
    peaks, kind = measured_peaks()
    peak = float(peaks.get("bf16_tflops", 1900.0)) if kind == "measured" else 1900.0
    # one training step (forward with saved activations, backward on the
    # tensor cores, Adam) at batch 4096, device time per step
    nb = 4096
    Xb = Xi[:nb].contiguous()
    Yb = torch.randn(nb, 3, device="cuda") * 0.5
    for _ in range(3):
        net.train_step(Xb, Yb, 1e-4, want_loss=False)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(args.steps):
        net.train_step(Xb, Yb, 1e-4, want_loss=False)
    e1.record()
    torch.cuda.synchronize()
    train_ms = e0.elapsed_time(e1) / args.steps
    train_flop = 3 * nb * 2.0 * (256 * 128 + 128 * 128 * 2 + 128 * 16)
    line = {"metric": "fused MLP forward throughput", "value": flop / ms / 1e9, "unit": "TFLOP/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic (ct64 coarse features)",
            "config": {"workload": "learned-proposal forward, %d rows x 256 features" % rows},
            "roofline": {"bound": "tensor", "achieved": flop / ms / 1e9, "peak": peak, "unit": "TFLOP/s",
                         "frac": flop / ms / 1e9 / peak, "traffic": None, "peak_kind": kind},
            "train_step": {"batch": nb, "ms": train_ms, "tflops": train_flop / train_ms / 1e9,
                           "note": "forward + backward + Adam, enqueued back to back (no loss read back), device time "
                                   "per step; flop counted as 3x the forward"},
            "gpu_launches": args.steps}
    print(json.dumps(line), flush=True)
    return 0


def run_multires(args):
    """--workload cube_multires: the paper's synthetic cube problem through the
    grid multi-resolution scheme with the paper's settings (Sec. 2.4, 2.5):
    6^3-point meshes, population 250, 300 generations; then 11^3-point meshes
    seeded by refining a random sample of the approximation set, population
    500, 600 generations.  Reports the hypervolume per level and the run time
    (the minimal GOMEA scaffold, not the full RV-GOMEA model building)."""
    import torch

    from paper_2202_11001_gb300 import dmr, gomea, synth

    gens = [int(g) for g in args.generations.split(",")]
    pr = synth.cube_pair(seed=0, n=50, mesh=6, C=250)
    src, tgt = pr["img"]

    def build(mesh, C):
        return dmr.Problem(src, tgt, *pr["spacing"], mesh, guide=pr["guide"], model=dmr.LINEAR, storage="f32",
                           max_candidates=C)

    p0 = build(pr["mesh"], 250)
    o0 = np.asarray(p0.eval_full(pr["coords"]))
    p0.close()
    feas = o0[:, 3] == 0
    ref = 1.1 * np.max(o0[feas, :3], axis=0)
    rng = np.random.default_rng(1)
    levels = [{"mesh": (6, 6, 6), "C": 250, "generations": gens[0], "sigma0": 1.0},
              {"mesh": (11, 11, 11), "C": 500, "generations": gens[1], "sigma0": 0.5}]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    res = gomea.multi_resolution(build, pr["coords"], levels, ref, rng)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    per = []
    for r in res:
        g = r.pop("gomea")
        per.append({k: v for k, v in r.items() if k != "curve"} | {
            "hv_curve": [(round(e, 1), h) for e, h in r["curve"][:: max(1, len(r["curve"]) // 20)]],
            "evaluations": g.evals, "voxel_samples": g.prob.samples()})
        g.prob.close()
    line = {"metric": "HV of the final approximation set (grid multi-resolution run)", "value": res[-1]["final_hv"],
            "unit": "normalised HV", "n_gpus": 1, "higher_is_better": True, "data": "synthetic (paper's cube problem, "
            "50^3 reading)", "config": {"workload": "cube50: cube with parabolic side intrusions and a shrinking "
                                        "sphere, 20 guidance pairs; 6^3 -> 11^3 points; populations 250 / 500; "
                                        "generations %d / %d" % tuple(gens), "reference_point": ref.tolist()},
            "levels": per, "wall_seconds": wall}
    print(json.dumps(line), flush=True)
    return 0


def deltas_for(pr, groups, C, rng):
    from paper_2202_11001_gb300 import synth

    fix = synth.fixed_axes(pr["mesh"])
    d = rng.normal(0.0, pr.get("sigma", 1.0), size=(len(groups), C, 2, 3, 1))
    for gi, grp in enumerate(groups):
        for ax in range(3):
            if (fix[grp[0]] >> ax) & 1:
                d[gi, :, :, ax, 0] = 0.0
    return d


class ClockSampler:
    """nvidia-smi clocks and throttle reasons while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        # raw samples: BENCH_CLOCKS_DIR if set, else the system temporary directory
        out_dir = os.environ.get("BENCH_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(out_dir, "clocks_bench_%d.csv" % os.getpid())

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception as e:  # pragma: no cover
            log("clock sampling unavailable:", e)
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            d = json.load(open(p))
            return d, "measured"
        except Exception:
            pass
    return {"hbm_gbs": FALLBACK_HBM_GBS}, "fallback"


def cpu_baseline(pr, groups, waves, C, rng_seed, min_s=10.0, max_s=30.0):
    """The FP64 oracle as it stands, on the host cores, on a bounded sample:
    partial evaluations of the generation's waves (repeated until about
    min_s of work), then a single-thread timing on part of the first wave."""
    from oracle import oracle as orc
    from paper_2202_11001_gb300 import synth

    cores = os.cpu_count() or 1
    orc.set_threads(cores)
    src, tgt = pr["img"]
    o = orc.Oracle(src, tgt, *pr["spacing"], pr["mesh"], guide=pr["guide"], model=orc.LINEAR)
    o.eval_full(pr["coords"])
    rng = np.random.default_rng(rng_seed)
    cur = np.stack([o.coords(c) for c in range(C)])
    batches = []
    for w in waves:
        gids = np.repeat(w, C)
        cids = np.tile(np.arange(C), len(w))
        tc = synth.trial_coords(cur, groups, gids, cids, pr["sigma"], pr["mesh"], rng)
        batches.append((gids, cids, tc))
    samples, secs, nw, ntr, it = 0, 0.0, 0, 0, 0
    cov_of = []
    while secs < min_s and secs < max_s:
        gids, cids, tc = batches[it % len(batches)]
        t0 = time.perf_counter()
        o.eval_partial(groups, gids, cids, tc)
        secs += time.perf_counter() - t0
        if it < len(batches):
            cov_of.append(sum(int(o.trial(k, cap=256)["cov"].sum()) for k in range(len(gids))))
        samples += cov_of[it % len(batches)]
        nw += 1
        ntr += len(gids)
        it += 1
    value = samples / secs
    # single thread: the first trials of the first wave
    gids, cids, tc = batches[0]
    n1 = min(len(gids), 400)
    orc.set_threads(1)
    t0 = time.perf_counter()
    o.eval_partial(groups, gids[:n1], cids[:n1], tc[:n1])
    s1 = time.perf_counter() - t0
    c1 = sum(int(o.trial(k, cap=256)["cov"].sum()) for k in range(n1))
    orc.set_threads(cores)
    return {"value": value, "unit": UNIT, "cores": orc.max_threads() if cores > 1 else 1,
            "kind": "oracle", "single_thread_value": c1 / s1,
            "sample": "%d wave evaluations (%d of %d waves, repeated; %d trials, %d voxel-samples), FP64 C oracle, "
                      "OpenMP over trials, %.1f s; single thread: %d trials of the first wave, %.1f s"
                      % (nw, min(nw, len(waves)), len(waves), ntr, samples, secs, n1, s1)}


def precision_report(pr, stream, n_cand=8):
    """Objective errors of the reduced-precision image storage (Sec. 2.3.2
    dissimilarity with FP32 sampling): against the oracle fed the same
    quantised images (arithmetic error) and against the oracle fed the FP32
    images (quantisation error); max relative error per objective over the
    first n_cand candidates of a full evaluation."""
    import torch
    from oracle import oracle as orc
    from paper_2202_11001_gb300 import dmr

    orc.set_threads(os.cpu_count() or 1)
    src, tgt = pr["img"]
    coords = np.ascontiguousarray(pr["coords"][:n_cand])

    def quant(img, st):
        if st == "f32":
            return np.asarray(img, np.float32)
        dt = torch.bfloat16 if st == "bf16" else torch.float16
        return torch.from_numpy(np.asarray(img, np.float32)).to(dt).to(torch.float32).numpy()

    def oracle_obj(s_img, t_img):
        o = orc.Oracle(s_img, t_img, *pr["spacing"], pr["mesh"], guide=pr["guide"], model=orc.LINEAR)
        return np.asarray(o.eval_full(coords))

    def rel(a, b):
        a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
        return [float(np.max(np.abs(a[:, q] - b[:, q]) / np.maximum(np.abs(b[:, q]), 1e-300))) for q in range(3)]

    ref32 = oracle_obj(quant(src, "f32"), quant(tgt, "f32"))
    out = {"objectives": ["f_sim", "f_def", "f_guid"], "candidates": n_cand}
    for st in ("f32", "bf16", "f16"):
        g = dmr.Problem(src, tgt, *pr["spacing"], pr["mesh"], guide=pr["guide"], model=dmr.LINEAR, storage=st,
                        max_candidates=n_cand, stream=stream)
        gpu = np.asarray(g.eval_full(coords))
        g.close()
        refq = ref32 if st == "f32" else oracle_obj(quant(src, st), quant(tgt, st))
        out[st] = {"arith_rel_err": rel(gpu, refq), "quant_rel_err": rel(gpu, ref32)}
    return out


def _parity_waves(m, n_groups):
    """Waves of independent single-point groups: points of equal coordinate
    parity have disjoint stars."""
    par = [((p % m[0]) & 1) + 2 * (((p // m[0]) % m[1]) & 1) + 4 * ((p // (m[0] * m[1])) & 1)
           for p in range(n_groups)]
    return [np.array([g for g in range(n_groups) if par[g] == c]) for c in range(8)]


def run_reference(args):
    """--impl reference: the FP64 oracle, timed on the host cores, on bounded
    samples of the same workload.  batch64: each step is one wave of partial
    evaluations of 8 candidates of one of 4 problems spread over the batch
    (cycled); single problems: one wave of a quarter of the population."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from oracle import oracle as orc
    from paper_2202_11001_gb300 import synth

    cores = os.cpu_count() or 1
    orc.set_threads(cores)
    units = []  # (oracle, groups, waves, candidates, sigma, mesh)
    if args.workload == "batch64":
        probs, groups, _ = batch_inputs(2)
        pick = [0, 21, 42, 63]
        ncand = 8
        for q in pick:
            pr = probs[q]
            o = orc.Oracle(pr["img"][0], pr["img"][1], *pr["spacing"], pr["mesh"], guide=pr["guide"],
                           model=orc.LINEAR)
            o.eval_full(pr["coords"][:ncand])
            units.append((o, groups[q], _parity_waves(pr["mesh"], len(groups[q])), pr["sigma"], pr["mesh"]))
        desc = BATCH_DESC
        step_desc = "one wave of partial evaluations of %d candidates of one of problems %s (cycled)" % (ncand, pick)
    else:
        pr = workload(args.workload, 0)
        C = pr["coords"].shape[0]
        groups = synth.single_point_fos(pr["mesh"])
        o = orc.Oracle(pr["img"][0], pr["img"][1], *pr["spacing"], pr["mesh"], guide=pr["guide"], model=orc.LINEAR)
        o.eval_full(pr["coords"])
        ncand = max(8, C // 4)
        units.append((o, groups, _parity_waves(pr["mesh"], len(groups)), pr["sigma"], pr["mesh"]))
        desc = pr["desc"]
        step_desc = "one wave of partial evaluations for %d candidates (bounded sample)" % ncand
    rng = np.random.default_rng(11)
    tot_s, tot_n = 0.0, 0
    for step in range(args.warmup + args.steps):
        o, groups, waves, sigma, m = units[step % len(units)]
        w = waves[(step // len(units)) % 8]
        gids = np.repeat(w, ncand)
        cids = np.tile(np.arange(ncand), len(w))
        cur = np.stack([o.coords(c) for c in range(ncand)])
        tc = synth.trial_coords(cur, groups, gids, cids, sigma, m, rng)
        t0 = time.perf_counter()
        o.eval_partial(groups, gids, cids, tc)
        dt = time.perf_counter() - t0
        n = sum(int(o.trial(k, cap=256)["cov"].sum()) for k in range(len(gids)))
        if step >= args.warmup:
            tot_s += dt
            tot_n += n
    value = tot_n / tot_s
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_s / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": desc, "step": step_desc},
            "cpu_baseline": {"value": value, "unit": UNIT, "kind": "oracle", "cores": orc.max_threads(),
                             "sample": step_desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="batch64")
    ap.add_argument("--storage", default="f32", choices=["f32", "bf16", "f16"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--generations", default="300,600", help="cube_multires: generations per level")
    ap.add_argument("--tile", default="", help="fixed raster tile WARPSxVOXELS (e.g. 4x32) instead of autotuning")
    ap.add_argument("--problems", type=int, default=0,
                    help="batch64: only the first N problems (small profiling captures; not a bench line)")
    ap.add_argument("--population", type=int, default=0,
                    help="single-problem workloads: only the first N candidates (small profiling captures)")
    args = ap.parse_args()
    if args.warmup < 3:
        log("warm-up raised to 3")
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch64":
        return run_batch(args)
    if args.workload == "learned":
        return run_learned(args)
    if args.workload == "mlp_forward":
        return run_mlp_forward(args)
    if args.workload == "cube_multires":
        return run_multires(args)

    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2202_11001_gb300 import dmr, synth

    pr = workload(args.workload, rank)
    if args.population:
        pr["coords"] = np.ascontiguousarray(pr["coords"][: args.population])
    C = pr["coords"].shape[0]
    src, tgt = pr["img"]
    stream = torch.cuda.current_stream().cuda_stream

    def build(storage):
        g = dmr.Problem(src, tgt, *pr["spacing"], pr["mesh"], guide=pr["guide"], model=dmr.LINEAR,
                        storage=storage, max_candidates=C, stream=stream)
        g.eval_full(torch.from_numpy(pr["coords"]).cuda())
        groups = synth.single_point_fos(pr["mesh"])
        g.set_fos(groups)
        return g, groups

    g, groups = build(args.storage)
    if args.tile:
        # a fixed tile (no autotuning): reproducible profiling of one kernel instance
        tile_w, tile_v = (int(v) for v in args.tile.lower().split("x"))
        g.set_tile(tile_w, tile_v)
        tile_table = {}
    else:
        tile_w, tile_v, tile_table = g.autotune()
    waves = g.waves()
    rng = np.random.default_rng(100 + rank)
    deltas = deltas_for(pr, groups, C, rng)
    plan = g.plan_generation(np.arange(C, dtype=np.int32), deltas)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    for _ in range(args.warmup):
        plan.run()
    torch.cuda.synchronize()
    g.sample_counts(reset=True)
    sampler = ClockSampler(local)
    sampler.start()
    step_ms, raster_ms = [], 0.0
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    for _ in range(args.steps):
        flush.zero_()  # L2 flush outside the timed step
        ev0.record()
        plan.run()
        ev1.record()
        torch.cuda.synchronize()
        step_ms.append(ev0.elapsed_time(ev1))
        _, ra = plan.kernel_ms()
        raster_ms += ra
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    samples, executed = g.sample_counts(reset=True)
    total_s = sum(step_ms) / 1e3
    total_s, all_samples = reduce_over_ranks(total_s, samples, dist, "cuda")
    value = all_samples / total_s
    samples_per_step = samples / args.steps
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count

    # e2e: the public API with host (pinned) buffers, copies inside the timed
    # region.  Primary: the generation plan fed each step's proposal offsets
    # from pinned host memory (dmr_plan_update), run, objectives read back
    # (dmr_objectives_out).  Also: one dmr_eval_partial + dmr_commit_improving
    # call per wave.
    e2e = None
    if args.e2e_steps > 0:
        pin_d = torch.from_numpy(np.ascontiguousarray(deltas)).pin_memory()
        obj_h = np.zeros((C, 4))
        plan.update(pin_d)
        plan.run()
        g.objectives()
        g.samples(reset=True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            plan.update(pin_d)
            plan.run()
            obj_h = g.objectives()
        dt = time.perf_counter() - t0
        e2e = {"value": g.samples(reset=True) / dt, "unit": UNIT, "h2d_bytes_per_step": int(pin_d.numel() * 8),
               "d2h_bytes_per_step": int(obj_h.size * 8),
               "path": "dmr_plan_update (pinned host deltas) + dmr_plan_run + dmr_objectives_out per generation"}
    if args.e2e_steps > 0:
        cur0 = pr["coords"]
        per_wave = []
        h2d = d2h = 0
        for w in waves:
            cids = np.repeat(np.arange(C), len(w)).astype(np.int32)
            gids = np.tile(w, C).astype(np.int32)
            tc = np.stack([cur0[c][:, :, groups[gg]] + deltas[gg, c] for gg, c in zip(gids, cids)])
            pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
            per_wave.append((pin(gids), pin(cids), pin(tc), torch.empty((len(gids), 4), dtype=torch.float64,
                                                                        pin_memory=True)))
            h2d += tc.nbytes  # group / candidate ids repeat: the library keeps their layout on the device
            d2h += len(gids) * 4 * 8 + len(gids)
        g.samples(reset=True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            for gi, ci, tc, ob in per_wave:
                g.eval_partial(gi, ci, tc, out=ob)
                g.commit_improving()
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        e2e["per_wave_api"] = {"value": g.samples(reset=True) / dt, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                               "d2h_bytes_per_step": int(d2h),
                               "path": "dmr_eval_partial + dmr_commit_improving per wave, pinned host buffers; "
                                       "trial layouts cached by the library after the first generation"}

    peaks, peak_kind = measured_peaks()
    clock_max = clocks.get("sm_max_mhz") or 2070.0
    alu_peak = n_sm * 128 * clock_max * 1e6 / 1e12  # T lane-ops/s
    raster_s_per_step = raster_ms / 1e3 / args.steps
    executed_per_step = executed / args.steps
    achieved = executed_per_step * ALG_OPS_PER_SAMPLE / raster_s_per_step / 1e12
    bpv = 4 if args.storage == "f32" else 2
    hbm = float(peaks.get("hbm_gbs", FALLBACK_HBM_GBS))
    traffic = FAST_PASS_DRAM_BYTES.get((args.workload, args.storage))
    roofline = {"bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "T lane-op/s",
                "frac": achieved / alu_peak, "traffic": traffic,
                "issue_active_ncu": FAST_PASS_ISSUE_ACTIVE.get((args.workload, args.storage)),
                "traffic_unit": "DRAM bytes per fast raster-pass launch (one wave), ncu",
                "kernel": "k_raster (rasterise + map + trilinear sample + SSD)",
                "ops_per_sample": ALG_OPS_PER_SAMPLE, "basis": "executed samples",
                "peak_basis": "%d SMs x 128 FP32 lanes x %.0f MHz (max SM clock)" % (n_sm, clock_max),
                "raster_ms_per_step": raster_s_per_step * 1e3,
                "counted_samples_per_step": samples_per_step, "executed_samples_per_step": executed_per_step,
                "executed_frac": executed_per_step / max(samples_per_step, 1.0),
                "touched_bytes_frac_of_hbm": value * 2 * bpv / 1e9 / hbm,
                "hbm_peak_gbs": hbm, "hbm_peak_kind": peak_kind}

    variants = {}
    if not args.no_variants and world == 1:
        for st in ("f32", "bf16", "f16"):
            if st == args.storage:
                variants[st] = value
                continue
            gv, _ = build(st)
            gv.autotune()
            pv = gv.plan_generation(np.arange(C, dtype=np.int32), deltas)
            for _ in range(3):
                pv.run()
            torch.cuda.synchronize()
            gv.samples(reset=True)
            tt = 0.0
            for _ in range(max(3, args.steps // 2)):
                flush.zero_()
                ev0.record()
                pv.run()
                ev1.record()
                torch.cuda.synchronize()
                tt += ev0.elapsed_time(ev1)
            variants[st] = gv.samples(reset=True) / (tt / 1e3)
            pv.close()
            gv.close()

    precision = None
    if not args.no_variants and rank == 0 and world == 1 and args.workload != "ct":
        precision = precision_report(pr, stream)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(pr, groups, waves, C, 7)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": args.storage,
                "data": "synthetic (seeded phantom, %s)" % pr["name"],
                "config": {"workload": pr["desc"], "storage": args.storage, "population": C,
                           "fos_groups": len(groups), "waves": len(waves), "mesh_pts": list(pr["mesh"]),
                           "deform_model": "linear_elastic", "samples_per_step": samples_per_step,
                           "executed_samples_per_step": executed_per_step,
                           "tile": {"warps_per_cta": tile_w, "voxels_per_warp": tile_v,
                                    "autotune_ms": {"%dx%d" % k: round(v, 4) for k, v in tile_table.items()}},
                           "l2": "flushed before every timed step (256 MiB write outside the event bracket)",
                           "parallelism": "replicas" if world > 1 else "single GPU"},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
                "gpu_launches": plan.launches * args.steps, "variants_samples_per_s": variants,
                "precision": precision}
        print(json.dumps(line), flush=True)
    plan.close()
    g.close()
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
