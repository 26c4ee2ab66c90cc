#!/usr/bin/env python3
"""Benchmark of the vector navigator step (distance to the next boundary for a
basket of tracks in one mother volume, Fig. 1 of the paper) on the GPU.

Workload: the toy detector (tube mother r 1000 mm, half-z 1500 mm, 40
daughters: 8 coaxial tube shells, 24 rotated boxes, 8 endcap cones), a basket
of 2^20 tracks uniform in the mother's exclusive part with isotropic
directions.  One step = one geo_dist_to_boundary call over the basket in
GEO_FP32_REFINE mode; the plain FP64 mode is timed beside it.

Prints one JSON line (rank 0).  Run `python bench.py --impl reference` for the
CPU oracle timed on the host cores (the reference arm).
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

N_TRACKS = 1 << 20
N_COPIES = 8          # rotating basket copies: 8 x 60 MB > 2 x 129 MB L2
E2E_COPIES = 4        # pinned host copies for the end-to-end timing: 4 x 60 MB > L2
METRIC = "tracks/s dist-to-boundary, FP32+FP64-refine vs plain FP64 on GPU; % roofline"
WORKLOAD = "toy detector: tube mother r0-1000 half-z 1500 mm, 40 daughters (8 tube shells, 24 rotated boxes, " \
           "8 cones), 2^20 tracks uniform in the mother's exclusive part, isotropic, seed 1"

# Nominal peaks derived from unit counts and clocks (GB300: 152 SMs at a
# 2070 MHz maximum SM clock): FP32 = 128 FMA lanes per SM; FP64 = 2 DFMA
# lanes per SM (ncu: sm__sass_thread_inst_executed_op_dfma_pred_on peak
# sustained = 2 per cycle per SM).  Flops count an FMA as 2.
SM_COUNT, SM_HZ = 152, 2.07e9
PEAK_FP32_TFLOPS = SM_COUNT * 128 * 2 * SM_HZ / 1e12
PEAK_FP64_TFLOPS = SM_COUNT * 2 * 2 * SM_HZ / 1e12

# FP64-pipe instructions of one evaluation of each routine in shapes64.cuh
# (comparisons run on the integer ALU and are not counted):
# (plain FP64 instructions, square roots, divisions).
FP64_OPS = {
    ("out", 0): (30, 0, 1), ("out", 1): (23, 2, 3), ("out", 2): (33, 2, 3),
    ("in", 0): (3, 0, 3), ("in", 1): (12, 1, 2), ("in", 2): (17, 1, 2),
}
FP64_TRANSFORM = 21          # rotated placement: 3 subtractions + 18 multiply/FMA
FP64_TRANSFORM_IDENTITY = 3  # identity rotation: the 3 subtractions alone
FP64_BPOINT = 3
# FP32 instructions of the filter per daughter: bounding-sphere test,
# transform, and the bound of each kind (MUFU reciprocal / square root
# counted as 4)
FP32_SPHERE, FP32_TRANSFORM = 16, 18   # the rotation is skipped for identity placements
FP32_SHAPE = {0: 45, 1: 90, 2: 110}
FP32_DDA_STEP = 12     # one grid step: pick the axis, advance index and boundary, test the range
FP32_MOTHER = 100      # the mother's two FP32 exits (shrunk and grown copy)
KERNEL_SOURCES = ("nav_refine.cu", "refine_kernel.cuh", "nav_refine.cuh", "shapes32.cuh", "shapes64.cuh", "nav_common.cuh",
                  "stage.cuh", "geo_internal.h")


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def dist_env():
    from paper_1312_0816_gb300 import replicas

    return replicas.env()


class Clocks:
    """nvidia-smi sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.path = tempfile.mktemp(suffix=".csv")
        self.proc = None
        self.gpu = gpu_index

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def mark(self):
        """Samples before this point (idle pre-roll) are not counted."""
        try:
            self.fh.flush()
            self.skip = sum(1 for _ in open(self.path))
        except Exception:
            self.skip = 0

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = []
        for k, line in enumerate(open(self.path)):
            f = [c.strip() for c in line.split(",")]
            if len(f) >= 9 and k >= getattr(self, "skip", 0):
                rows.append(f)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(v):
            try:
                return float(v)
            except ValueError:
                return None

        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows),
                "power_w_max": max((num(r[3]) or 0.0) for r in rows)}


def algorithmic_ops(sc, hit):
    """Share of the tracks whose winner is the mother, and per (kind, identity
    placement) the share whose winner is such a daughter."""
    kinds = sc.kinds
    eye = sc.identity_mask()
    w = hit[hit >= -1]
    m = (w == -1).mean()
    ops_d = {}
    wd = np.maximum(w, 0)
    for k in (0, 1, 2):
        for ident in (False, True):
            ops_d[(k, ident)] = ((w >= 0) & (kinds[wd] == k) & (eye[wd] == ident)).mean()
    return m, ops_d


def fp64_ops_per_track(sc, frac_mother, frac_kind, q_sqrt, q_div):
    """Algorithmic FP64 work of the filter+refine step per track, in DFMA
    equivalents: the mother's DistFromInside (always), the transform (3
    operations for an identity rotation, 21 otherwise) and DistFromOutside of
    the winning daughter, and the boundary point."""
    def cost(key):
        a, s, d = FP64_OPS[key]
        return a + s * q_sqrt + d * q_div

    ops = cost(("in", sc.mother_kind))
    for (k, ident), f in frac_kind.items():
        ops += f * ((FP64_TRANSFORM_IDENTITY if ident else FP64_TRANSFORM) + cost(("out", k)))
    return ops + FP64_BPOINT


def fp64_cost_per_track(sc, hit, q_sqrt, q_div, with_mother=True):
    """Per-track algorithmic FP64 work (DFMA equivalents) of a step in scene
    sc given its winners `hit`: the mother's DistFromInside (always, with
    with_mother), the winning daughter's transform (3 or 21) and
    DistFromOutside, and the boundary point.  Tracks outside the mother or
    invalid count 0."""
    def cost(key):
        a, s_, d = FP64_OPS[key]
        return a + s_ * q_sqrt + d * q_div

    eye = sc.identity_mask()
    per_d = np.array([(FP64_TRANSFORM_IDENTITY if e else FP64_TRANSFORM) + cost(("out", int(k)))
                      for k, e in zip(sc.kinds, eye)] + [0.0])
    hit = np.asarray(hit)
    c = np.where(hit >= 0, per_d[np.maximum(hit, 0)], 0.0)
    if with_mother:
        c = c + np.where(hit >= -1, cost(("in", sc.mother_kind)) + FP64_BPOINT, 0.0)
    return c


def fp32_ops_per_track(sc):
    """Algorithmic FP32 work: every daughter bounded in FP32 (the rotation
    only for rotated placements)."""
    eye = sc.identity_mask()
    return float(sum(FP32_SPHERE + (0 if e else FP32_TRANSFORM) + FP32_SHAPE[int(k)] for k, e in zip(sc.kinds, eye)))


def code_only(text: str) -> str:
    """A source file without its comments and with its blank space collapsed,
    so that an edit of comments alone keeps the kernel's captured counters."""
    import re

    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return " ".join(text.split())


def sources_sha(read=None):
    """Hash of the refine kernel's code (comments excluded); read(name) gives
    a source's text (default: the file in the package)."""
    import hashlib

    if read is None:
        def read(f):
            return open(os.path.join(ROOT, "paper_1312_0816_gb300", "csrc", f)).read()
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        h.update(code_only(read(f)).encode())
    return h.hexdigest()[:16]


def captured_traffic():
    """DRAM bytes per launch of the refine kernel from the committed ncu
    summary, only if the kernel sources are those that were captured."""
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "k_dist_refine_toy40_2p20.json")))
    except Exception:
        return None, None
    if rec.get("sources_sha") != sources_sha():
        return None, rec.get("sources_sha")
    return rec.get("dram_bytes_per_launch"), rec.get("sources_sha")


def run_reference(args):
    """The CPU oracle, as it stands, on the host cores (reference arm)."""
    import oracle
    from paper_1312_0816_gb300 import scenes

    ws, rank, _ = dist_env()
    if rank != 0:
        return
    cores = len(os.sched_getaffinity(0))
    sc = scenes.toy40(1)
    sample = args.n
    tr = scenes.sample_tracks(sc, sample, 1)   # the GPU arm's basket (rank 0)
    for _ in range(args.warmup):
        oracle.navigate(sc, tr.slice(0, 1024), nthreads=cores)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.navigate(sc, tr, nthreads=cores)
    dt = (time.perf_counter() - t0) / args.steps
    value = sample / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "tracks/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "tracks_per_gpu": sample, "mode": "the FP64 oracle",
                       "same_config": sample == N_TRACKS},
            "cpu_baseline": {"value": value, "unit": "tracks/s", "cores": cores, "kind": "oracle",
                             "sample": f"the whole {sample}-track toy-detector basket per step"},
            "e2e": {"value": value, "unit": "tracks/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# Samples of the side legs' GPU answers, checked against the oracle in the
# CPU-baseline leg (the one place the benchmark runs the oracle).
SAMPLES = {}
SAMPLES_WORLD = {}
Q_RATES = [8.6, 5.7]       # sqrt, div in DFMA equivalents (the probe's values replace these)
PEAK_HBM = [6760.9]        # GB/s (MEASURED_PEAKS.json replaces this)
MOVE = 1e-9   # mm: a start-point move that defines "decided by rounding"


def _moved(scenes, tr, k, sign):
    f = [tr.x.copy(), tr.y.copy(), tr.z.copy()]
    f[k] = f[k] + sign * MOVE
    return scenes.Tracks(*f, tr.dx, tr.dy, tr.dz)


def accuracy(oracle, scenes, sc, tr, ref, step, hit, cores):
    """Per-result error of GPU answers against the FP64 oracle, every track:
    |dstep| within max(1e-9 mm, err) (err the oracle's a-priori FP64 bound),
    hit equal outside the tie band; a track outside that counts as decided by
    rounding if its answer is the oracle's for a start moved by 1e-9 mm, else
    as a violation (must be 0)."""
    dn = np.sqrt(tr.dx ** 2 + tr.dy ** 2 + tr.dz ** 2)
    ok = ~np.isnan(ref["step"])
    tol = np.maximum(1e-9 / dn, ref["err"])
    d = np.where(ok, np.abs(step - ref["step"]), 0.0)
    tie = ok & ((ref["second"] - ref["step"]) < tol)
    cond = ok & (ref["err"] > 1e-9)
    nan_mismatch = int((np.isnan(step) != ~ok).sum())
    off = ok & (~(d <= tol) | (~tie & (hit != ref["hit"])))
    graze = np.zeros(tr.n, dtype=bool)
    idx = np.nonzero(off)[0]
    if idx.size:
        sub = scenes.Tracks(*(f[idx] for f in tr.fields()))
        m = np.zeros(idx.size, dtype=bool)
        for k in range(3):
            for sg in (-1.0, 1.0):
                r = oracle.navigate(sc, _moved(scenes, sub, k, sg), nthreads=cores)
                t2 = np.maximum(1e-6 / dn[idx], r["err"])
                m |= (np.abs(step[idx] - r["step"]) <= t2) & ((hit[idx] == r["hit"]) | (r["second"] - r["step"] < t2))
        graze[idx] = m
    viol = off & ~graze
    return {"tracks": int(ok.sum()), "max_abs_dstep_mm": float((d * dn)[ok & ~cond & ~graze].max(initial=0.0)),
            "max_abs_dstep_cond_band_mm": float((d * dn)[cond & ~graze].max(initial=0.0)),
            "tie_banded": int(tie.sum()), "cond_banded": int(cond.sum()),
            "hit_mismatch_outside_tie_band": int((ok & ~tie & (hit != ref["hit"]) & ~graze).sum()),
            "rounding_decided": int(graze.sum()), "violations": int(viol.sum()) + nan_mismatch,
            "bar": "|dstep| <= max(1e-9 mm, err) on every track; hit exact outside the tie band"}


def cpu_baseline(sc, tr, step, hit):
    """The oracle as it stands on all host cores, over the whole basket (about
    1 s wall on 16 cores), plus a single-thread rate on its first 8192 tracks;
    then, untimed, the per-result error of the GPU answers on that basket and
    on the side legs' samples against the oracle's."""
    import oracle
    from paper_1312_0816_gb300 import scenes

    cores = len(os.sched_getaffinity(0))
    t0 = time.perf_counter()
    ref = oracle.navigate(sc, tr, nthreads=cores)
    dt = time.perf_counter() - t0
    one = tr.slice(0, 8192)
    t1 = time.perf_counter()
    oracle.navigate(sc, one, nthreads=1)
    dt1 = time.perf_counter() - t1
    acc = {"headline": accuracy(oracle, scenes, sc, tr, ref, step, hit, cores)}
    for name, (ssc, str_, sstep, shit) in SAMPLES.items():
        if isinstance(ssc, list):   # batched: one scene per track
            parts = []
            for v in sorted(set(id(x) for x in ssc)):
                sel = np.array([id(x) == v for x in ssc])
                vs = next(x for x in ssc if id(x) == v)
                sub = scenes.Tracks(*(f[sel] for f in str_.fields()))
                r = oracle.navigate(vs, sub, nthreads=cores)
                parts.append(accuracy(oracle, scenes, vs, sub, r, sstep[sel], shit[sel], cores))
            agg = {k: sum(p_[k] for p_ in parts) for k in ("tracks", "tie_banded", "cond_banded",
                                                             "hit_mismatch_outside_tie_band", "rounding_decided",
                                                             "violations")}
            agg["max_abs_dstep_mm"] = max(p_["max_abs_dstep_mm"] for p_ in parts)
            agg["max_abs_dstep_cond_band_mm"] = max(p_["max_abs_dstep_cond_band_mm"] for p_ in parts)
            acc[name] = agg
        else:
            r = oracle.navigate(ssc, str_, nthreads=cores)
            acc[name] = accuracy(oracle, scenes, ssc, str_, r, sstep, shit, cores)
    for name, (w, wt, nd, fl, wstep, wnode, wflag) in SAMPLES_WORLD.items():
        acc[name] = world_accuracy(oracle, scenes, w, wt, nd, fl, wstep, wnode, wflag)
    return {"value": tr.n / dt, "unit": "tracks/s", "cores": cores, "kind": "oracle",
            "sample": f"the whole {tr.n}-track basket once, {cores} threads ({dt:.2f} s wall)",
            "single_thread_value": 8192 / dt1}, acc


def world_accuracy(oracle, scenes, w, tr, node, flag, step, node_out, flag_out):
    """The tree step against the oracle's: |dstep| within max(1e-9 mm, err)
    (err with the placements' rounding), node and flag equal unless the
    oracle's own answer changes for a start moved by 1e-9 mm."""
    s, nn, ff, info = oracle.world_step(w, tr, node, flag, info=True)
    alive = node >= 0
    tol = np.maximum(1e-9, info["err"])
    d = np.where(alive, np.abs(step - s), 0.0)
    diff = alive & ((node_out != nn) | (flag_out != ff))
    unstable = np.zeros(tr.n, dtype=bool)
    if diff.any():
        for k in range(3):
            for sg in (-1.0, 1.0):
                _, n2, f2 = oracle.world_step(w, _moved(scenes, tr, k, sg), node, flag)
                unstable |= (n2 != nn) | (f2 != ff)
    cond = alive & (info["err"] > 1e-9)
    return {"tracks": int(alive.sum()), "max_abs_dstep_mm": float(d[alive & ~cond].max(initial=0.0)),
            "max_abs_dstep_cond_band_mm": float(d[cond].max(initial=0.0)), "cond_banded": int(cond.sum()),
            "node_or_flag_differs": int(diff.sum()), "of_which_rounding_decided": int((diff & unstable).sum()),
            "violations": int((alive & ~(d <= tol)).sum() + (diff & ~unstable).sum()),
            "bar": "|dstep| <= max(1e-9 mm, err); node and flag exact unless a 1e-9 mm move changes the oracle's"}


def roof_block(fp64_dfma, fp32_instr, hbm_bytes, seconds, kernel, note, peak_hbm_gbs):
    """Binding roofline of a launch from its algorithmic work: T_roof =
    max(HBM bytes / measured copy bandwidth, FP32 / nominal FP32, FP64 /
    nominal FP64); frac = T_roof / measured time, reported against the
    binding term's own peak."""
    t = {"hbm": hbm_bytes / (peak_hbm_gbs * 1e9), "fp64": fp64_dfma * 2 / (PEAK_FP64_TFLOPS * 1e12),
         "fp32": fp32_instr * 2 / (PEAK_FP32_TFLOPS * 1e12)}
    bind = max(t, key=t.get)
    if bind == "hbm":
        ach, peak, unit, bound = hbm_bytes / seconds / 1e9, peak_hbm_gbs, "GB/s", "hbm"
    else:
        work = fp64_dfma if bind == "fp64" else fp32_instr
        peak = PEAK_FP64_TFLOPS if bind == "fp64" else PEAK_FP32_TFLOPS
        ach, unit, bound = work * 2 / seconds / 1e12, "TFLOP/s", "alu"
    return {"bound": bound, "pipe": bind, "achieved": ach, "peak": peak, "unit": unit, "frac": ach / peak,
            "t_roof_us": {k: v * 1e6 for k, v in t.items()}, "kernel": kernel, "algorithmic": note,
            "peak_source": "FP32/FP64 nominal from unit counts x 2.07 GHz; HBM measured copy bandwidth"}


def batched_leg(pkg, scenes, rank, steps):
    """64 logical volumes (4..200 daughters), 561 baskets of 16..65536 tracks
    (2^22 tracks): one persistent launch per step, replayed as a CUDA graph,
    schedule chosen by the autotuner."""
    import torch

    from paper_1312_0816_gb300 import autotune

    vols, baskets = scenes.batched64(seed=3)
    tr, rows = scenes.batched_tracks(vols, baskets, 3 + 1000 * rank)
    volh = [pkg.geo_build_volume(v) for v in vols]
    x = [torch.from_numpy(f).cuda() for f in tr.fields()]
    step = torch.empty(tr.n, dtype=torch.float64, device="cuda")
    hit = torch.empty(tr.n, dtype=torch.int32, device="cuda")
    order, bps, tile, timings = autotune.tune_batch(volh, rows, x, step, hit)
    batch = pkg.geo_build_batch(volh, rows, tile_order=order, blocks_per_sm=bps, tile_tracks=tile)
    ms = autotune.time_graph(batch, x, step, hit, reps=steps)
    batch.close()
    # a sample of the last launch's answers for the accuracy check
    owner = np.repeat(np.arange(len(rows)), rows[:, 2].astype(np.int64))
    idx = np.sort(np.random.default_rng(31).choice(tr.n, 20000, replace=False))
    s_np, h_np = step.cpu().numpy(), hit.cpu().numpy()
    SAMPLES["batched"] = ([vols[int(rows[owner[i], 0])] for i in idx], scenes.Tracks(*(f[idx] for f in tr.fields())),
                          s_np[idx], h_np[idx])
    # algorithmic work of the launch: per basket, its volume's mother, winner
    # and FP32 bounds of every daughter
    f64 = f32 = 0.0
    for v, off, cnt in rows:
        sc_v = vols[int(v)]
        f64 += float(fp64_cost_per_track(sc_v, h_np[off:off + cnt], Q_RATES[0], Q_RATES[1]).sum())
        f32 += fp32_ops_per_track(sc_v) * int(cnt)
    roof = roof_block(f64, f32, 60.0 * tr.n, ms * 1e-3, "k_dist_batched (one launch per step)",
                      "per track: its volume's mother exit, winning daughter and boundary point in FP64; "
                      "every daughter bounded in FP32; 60 B of HBM", PEAK_HBM[0])
    return {"workload": "64 volumes (box/tube mothers, 4..200 mixed daughters), %d baskets of 16..65536 "
                        "tracks, %d tracks, FP32+refine, one persistent launch per step as a CUDA graph"
                        % (len(rows), tr.n),
            "value": tr.n / (ms * 1e-3), "unit": "tracks/s", "ms_per_launch": ms, "steps": steps,
            "schedule": {"tile_order": order, "blocks_per_sm": bps, "tile_tracks": tile,
                         "warps": "12 producer + 4 consumer" if tile == 384 else "8 producer + 4 consumer"},
            "autotune_ms": timings, "roofline": roof}


def voxel_counts(sc, grid, tr, step):
    """Instrumented walk of the uniform grid (counting only; not the
    navigator): for each track, the distinct daughters listed in the cells
    its line crosses from its start up to its step, and the grid steps taken.
    The cells list the daughters whose world bounding box overlaps them, as
    the library's grid does.  Returns (candidates, dda_steps) per track."""
    mp = sc.mother_params
    half = np.array(mp[:3], dtype=float)
    g = np.array(grid, dtype=int)
    lo, cell = -half, 2.0 * half / g
    lists = [[] for _ in range(int(g.prod()))]
    for j in range(sc.n_daughters):
        k, p = int(sc.kinds[j]), sc.params[j]
        he = np.array(p[:3]) if k == 0 else np.array([p[1], p[1], p[2]])
        R = sc.rot[j].reshape(3, 3)
        ext = np.abs(R) @ he
        a = np.clip(np.floor((sc.trans[j] - ext - lo) / cell), 0, g - 1).astype(int)
        b = np.clip(np.floor((sc.trans[j] + ext - lo) / cell), 0, g - 1).astype(int)
        for i0 in range(a[0], b[0] + 1):
            for i1 in range(a[1], b[1] + 1):
                for i2 in range(a[2], b[2] + 1):
                    lists[(i0 * g[1] + i1) * g[2] + i2].append(j)
    cand, steps = np.zeros(tr.n, dtype=int), np.zeros(tr.n, dtype=int)
    for t in range(tr.n):
        p = np.array([tr.x[t], tr.y[t], tr.z[t]])
        d = np.array([tr.dx[t], tr.dy[t], tr.dz[t]])
        ii = np.clip(np.floor((p - lo) / cell).astype(int), 0, g - 1)
        st = np.sign(d).astype(int)
        with np.errstate(divide="ignore", invalid="ignore"):
            nxt = np.where(d > 0, lo + (ii + 1) * cell, lo + ii * cell)
            tm = np.where(d != 0, (nxt - p) / d, np.inf)
            te = np.where(d != 0, cell / np.abs(d), np.inf)
        seen = set()
        n = 0
        while True:
            seen.update(lists[(ii[0] * g[1] + ii[1]) * g[2] + ii[2]])
            k = int(np.argmin(tm))
            if not tm[k] <= step[t]:
                break
            ii[k] += st[k]
            if ii[k] < 0 or ii[k] >= g[k]:
                break
            tm[k] += te[k]
            n += 1
        cand[t], steps[t] = len(seen), n
    return cand, steps


def voxel_leg(pkg, scenes, rank, steps, n=1 << 24):
    """512 daughters (boxes and tubes, rotated, on an 8x8x8 grid) in a box
    mother with the uniform-grid candidate list; n = 2^24 tracks (fewer only
    for a profiler capture); FP32+refine vs plain FP64, both walking the
    grid."""
    import torch

    sc = scenes.grid512(5)
    tr = scenes.sample_tracks(sc, n, 5 + 1000 * rank)
    vol = pkg.geo_build_volume(sc, voxelize=True)
    x = [torch.from_numpy(f).cuda() for f in tr.fields()]
    step = torch.empty(tr.n, dtype=torch.float64, device="cuda")
    hit = torch.empty(tr.n, dtype=torch.int32, device="cuda")
    out = {}
    for mode, name, k in ((1, "fp32_refine", steps), (0, "fp64_plain", max(3, steps // 4))):
        for _ in range(3):
            pkg.geo_dist_to_boundary(vol, *x, mode=mode, step=step, hit=hit)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(k):
            pkg.geo_dist_to_boundary(vol, *x, mode=mode, step=step, hit=hit)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / k
        out[name] = {"value": tr.n / (ms * 1e-3), "unit": "tracks/s", "ms_per_step": ms, "steps": k}
        if mode == 1:   # a sample of the answers for the accuracy check and the work count
            idx = np.sort(np.random.default_rng(37).choice(tr.n, 20000, replace=False))
            s_np, h_np = step.cpu().numpy(), hit.cpu().numpy()
            SAMPLES["voxel_512"] = (sc, scenes.Tracks(*(f[idx] for f in tr.fields())), s_np[idx], h_np[idx])
            sub = idx[:4000]
            cand, dda = voxel_counts(sc, pkg.geo_volume_info(vol)["grid"], scenes.Tracks(*(f[sub] for f in tr.fields())),
                                     s_np[sub])
            eye = sc.identity_mask()
            per_cand = np.mean([FP32_SPHERE + (0 if e else FP32_TRANSFORM) + FP32_SHAPE[int(k)]
                                for k, e in zip(sc.kinds, eye)])
            f32_track = float(cand.mean() * per_cand + dda.mean() * FP32_DDA_STEP + FP32_MOTHER)
            f64_track = float(fp64_cost_per_track(sc, h_np, Q_RATES[0], Q_RATES[1]).mean())
            out["roofline"] = roof_block(f64_track * tr.n, f32_track * tr.n, 60.0 * tr.n, ms * 1e-3,
                                         "k_dist_refine, grid traversal (one launch per step)",
                                         "per track: FP32 bounds of the distinct daughters listed in the cells "
                                         "the line crosses up to its step (%.2f on average, instrumented walk of "
                                         "4000 tracks) and %.2f grid steps; FP64 mother, winner and boundary point"
                                         % (cand.mean(), dda.mean()), PEAK_HBM[0])
    info = pkg.geo_volume_info(vol)
    vol.close()
    out["workload"] = ("box mother half 800 mm, 512 rotated boxes/tubes on an 8x8x8 grid, uniform grid %s, "
                       "%d tracks (inputs %d MB > L2)" % ("x".join(str(g) for g in info["grid"]), n, n * 48 // 10**6))
    out["speedup_of_refine"] = out["fp64_plain"]["ms_per_step"] / out["fp32_refine"]["ms_per_step"]
    return out


def segments_leg(pkg, scenes, rank, steps):
    """The navigator step (Fig. 1) in volumes holding tube segments and
    polycones (Sec. 3.1's segmented and multi-section shapes): seg4 (box
    mother, four tube segments), pcon4 (box mother, four polycones) and pconm
    (a polycone mother with a waist holding a tube, two boxes and a cone
    segment); 2^20 tracks, 4 rotating copies (201 MB > L2), both modes."""
    import torch

    out = {}
    n = 1 << 20
    for name in ("seg4", "pcon4", "pconm"):
        sc = scenes.SCENES[name]()
        tr = scenes.sample_tracks(sc, n, 61 + 1000 * rank)
        vol = pkg.geo_build_volume(sc)
        base = [torch.from_numpy(np.ascontiguousarray(f)).cuda() for f in tr.fields()]
        g = torch.Generator(device="cuda")
        g.manual_seed(13)
        copies = [base] + [[f[p].contiguous() for f in base]
                           for p in (torch.randperm(n, device="cuda", generator=g) for _ in range(3))]
        step = torch.empty(n, dtype=torch.float64, device="cuda")
        hit = torch.empty(n, dtype=torch.int32, device="cuda")
        row = {}
        for mode, key, k in ((1, "fp32_refine", steps), (0, "fp64_plain", max(3, steps // 4))):
            ms = _event_time(lambda it: pkg.geo_dist_to_boundary(vol, *copies[it % 4], mode=mode, step=step, hit=hit), k)
            row[key] = {"value": n / (ms * 1e-3), "unit": "tracks/s", "ms_per_step": ms, "steps": k}
        row["speedup_of_refine"] = row["fp64_plain"]["ms_per_step"] / row["fp32_refine"]["ms_per_step"]
        out[name] = row
        vol.close()
    out["workload"] = "2^20 tracks uniform in the mother's exclusive part, isotropic, 4 rotating copies (201 MB > L2)"
    return out


SWEEP_SIZES = (16, 64, 256, 1024, 4096, 65536, 1 << 20)


def sweep_leg(pkg, scenes, rank, steps, vol, base, sizes=SWEEP_SIZES):
    """Fig. 3's axis, time per track against basket size, on the toy detector:
    baskets of N = 16 .. 2^20 consecutive tracks of the 2^20-track basket;
    per N the tracks/s of one geo_dist_to_boundary call per basket (32 calls
    at different offsets captured in a CUDA graph, so the time is the
    device's: launch-bound for small N; the basket is L2-resident, 50 MB) and
    of 2^22 tracks as 2^22/N baskets in one batched launch replayed as a CUDA
    graph (four copies of the basket, 201 MB > L2).  Also the paper's
    1024-track basket of four boxes in a box (microseconds per call, stream
    launch and graph replay, both modes) and the paper's own 8-daughter toy
    detector at 2^20 tracks (both modes)."""
    import torch

    from paper_1312_0816_gb300 import autotune

    n = int(base[0].numel())
    out = {"workload": "toy detector (40 daughters); basket sizes 16..2^20; the 1024-track box4 basket; "
                       "toy8 at 2^20 tracks"}
    step = torch.empty(n, dtype=torch.float64, device="cuda")
    hit = torch.empty(n, dtype=torch.int32, device="cuda")
    rng = np.random.default_rng(7 + rank)
    big = [torch.cat([f] * 4) for f in base]
    nb = int(big[0].numel())
    bstep = torch.empty(nb, dtype=torch.float64, device="cuda")
    bhit = torch.empty(nb, dtype=torch.int32, device="cuda")
    sweep = {}
    for N in sizes:
        offs = rng.integers(0, n - N + 1, size=32)
        calls = 32 if N < (1 << 20) else 1
        args = [[f[int(o): int(o) + N] for f in base] for o in offs[:calls]]
        pkg.geo_dist_to_boundary(vol, *args[0], mode=1, step=step[:N], hit=hit[:N])
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        st = torch.cuda.Stream()
        with torch.cuda.stream(st):
            with torch.cuda.graph(g, stream=st):
                for a in args:
                    pkg.geo_dist_to_boundary(vol, *a, mode=1, step=step[:N], hit=hit[:N])
        ms = _event_time(lambda it: g.replay(), max(5, min(100, (1 << 22) // (N * calls)))) / calls
        rows = np.array([(0, j * N, N) for j in range(nb // N)], dtype=np.int64)
        batch = pkg.geo_build_batch([vol], rows, tile_order=1)
        msb = autotune.time_graph(batch, big, bstep, bhit, reps=max(3, steps // 4))
        batch.close()
        sweep[str(N)] = {"per_call": {"value": N / (ms * 1e-3), "unit": "tracks/s", "us_per_call": ms * 1e3},
                         "batched_2p22": {"value": nb / (msb * 1e-3), "unit": "tracks/s", "ms_per_launch": msb,
                                          "baskets": int(len(rows))}}
    out["basket_sizes"] = sweep
    # the paper's 1024-track basket (box mother, four boxes)
    sc1 = scenes.box4(0)
    t1 = scenes.sample_tracks(sc1, 1024, 0)
    v1 = pkg.geo_build_volume(sc1)
    x1 = [torch.from_numpy(f).cuda() for f in t1.fields()]
    s1 = torch.empty(1024, dtype=torch.float64, device="cuda")
    h1 = torch.empty(1024, dtype=torch.int32, device="cuda")
    box4 = {}
    for mode, key in ((0, "fp64_plain"), (1, "fp32_refine")):
        ms = _event_time(lambda it: pkg.geo_dist_to_boundary(v1, *x1, mode=mode, step=s1, hit=h1), 200)
        box4[key] = {"us_per_call": ms * 1e3, "value": 1024 / (ms * 1e-3), "unit": "tracks/s"}
        try:
            pkg.geo_dist_to_boundary(v1, *x1, mode=mode, step=s1, hit=h1)
            torch.cuda.synchronize()
            g = torch.cuda.CUDAGraph()
            st = torch.cuda.Stream()
            with torch.cuda.stream(st):
                with torch.cuda.graph(g, stream=st):
                    pkg.geo_dist_to_boundary(v1, *x1, mode=mode, step=s1, hit=h1)
            box4[key]["us_per_graph_replay"] = _event_time(lambda it: g.replay(), 200) * 1e3
        except RuntimeError as e:
            torch.cuda.synchronize()
            box4[key]["us_per_graph_replay"] = None
            box4[key]["graph_error"] = str(e).splitlines()[0][:200]
    v1.close()
    out["box4_1024"] = box4
    # the paper's own toy detector composition (8 daughters)
    sc8 = scenes.toy8(1)
    t8 = scenes.sample_tracks(sc8, 1 << 20, 8 + 1000 * rank)
    v8 = pkg.geo_build_volume(sc8)
    x8 = [torch.from_numpy(f).cuda() for f in t8.fields()]
    g8 = torch.Generator(device="cuda")
    g8.manual_seed(21)
    c8 = [x8] + [[f[p].contiguous() for f in x8] for p in (torch.randperm(1 << 20, device="cuda", generator=g8)
                                                          for _ in range(3))]
    toy8 = {}
    for mode, key, kk in ((1, "fp32_refine", steps), (0, "fp64_plain", max(3, steps // 4))):
        ms = _event_time(lambda it: pkg.geo_dist_to_boundary(v8, *c8[it % 4], mode=mode, step=step, hit=hit), kk)
        toy8[key] = {"value": (1 << 20) / (ms * 1e-3), "unit": "tracks/s", "ms_per_step": ms}
    v8.close()
    out["toy8_2p20"] = toy8
    return out


def _event_time(fn, k):
    import torch

    for _ in range(3):
        fn(0)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for it in range(k):
        fn(it)
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / k


def adjoint_leg(pkg, scenes, rank, steps):
    """Gradients of the summed step: box mother with four boxes and the
    box/tube/cone scene, 2^18 tracks; the adjoint alone (per-track gradients
    plus the deterministic geometry reduction) and forward + adjoint.  Eight
    rotating basket copies keep the inputs out of L2."""
    import torch

    out = {}
    n = 1 << 18
    for name, sc in (("box4", scenes.box4(0)), ("diff3", scenes.diff3())):
        tr = scenes.sample_tracks(sc, n, 4 + 1000 * rank)
        vol = pkg.geo_build_volume(sc)
        base = [torch.from_numpy(f).cuda() for f in tr.fields()]
        g = torch.Generator(device="cuda")
        g.manual_seed(77 + rank)
        copies = [base] + [[f[p].contiguous() for f in base]
                           for p in (torch.randperm(n, device="cuda", generator=g) for _ in range(7))]
        hits = [pkg.geo_dist_to_boundary(vol, *c, mode=0)[1] for c in copies]
        w = torch.ones(n, dtype=torch.float64, device="cuda")
        ms_adj = _event_time(lambda it: pkg.geo_dist_to_boundary_adjoint(vol, *copies[it % 8], hits[it % 8], w),
                             steps)

        def fwd_bwd(it):
            c = copies[it % 8]
            _, h = pkg.geo_dist_to_boundary(vol, *c, mode=1)
            pkg.geo_dist_to_boundary_adjoint(vol, *c, h, w)

        ms_fb = _event_time(fwd_bwd, steps)
        h0 = hits[0].cpu().numpy()
        eye = sc.identity_mask()
        rot = np.where(h0 >= 0, ~eye[np.maximum(h0, 0)], False)
        # the winner's routine again, then the gradient: crossing point 3, surface
        # gradient 8, g.u 5, R g 9 (rotated placements), one division, the per-track
        # outputs 17, the owner sums 8
        f64 = fp64_cost_per_track(sc, h0, Q_RATES[0], Q_RATES[1], with_mother=False)
        f64 = f64 + np.where(h0 == -1, fp64_cost_per_track(sc, np.full_like(h0, -1), Q_RATES[0], Q_RATES[1])
                             - FP64_BPOINT, 0.0)
        f64 = f64 + np.where(h0 >= -1, 3 + 8 + 5 + 17 + 8 + Q_RATES[1] + 9 * rot, 0.0)
        roof = roof_block(float(f64.sum()), 0.0, 108.0 * n, ms_adj * 1e-3, "k_adjoint + k_adjoint_reduce",
                          "per track: the winning surface's routine again (transform, distance with its face) "
                          "and the implicit-function gradient, in FP64", PEAK_HBM[0])
        vol.close()
        # algorithmic bytes of the adjoint: p, d, hit, dL/dstep in; dL/dp, dL/dd out
        gbs = 108.0 * n / (ms_adj * 1e-3) / 1e9
        out[name] = {"adjoint": {"value": n / (ms_adj * 1e-3), "unit": "tracks/s", "ms_per_step": ms_adj,
                                 "algorithmic_gb_s": gbs, "roofline": roof},
                     "forward_plus_adjoint": {"value": n / (ms_fb * 1e-3), "unit": "tracks/s",
                                              "ms_per_step": ms_fb}}
    out["workload"] = ("2^18 tracks; box mother half 100 mm with 4 boxes, and box mother with one rotated box, "
                       "tube and cone; dL/dstep = 1; 8 rotating copies (226 MB > L2); steps %d" % steps)
    out["bytes_per_track"] = 108
    return out


def queries_leg(pkg, scenes, rank, steps, sc):
    """Contains and Safety over the toy detector, 2^22 points (inputs 100 MB,
    4 rotating copies > L2); Safety exact in both modes and the cheaper
    under-estimate (GEO_SAFETY_ESTIMATE)."""
    import torch

    n = 1 << 22
    tr = scenes.sample_tracks(sc, n, 9 + 1000 * rank, exclusive=False)
    vol = pkg.geo_build_volume(sc)
    base = [torch.from_numpy(f).cuda() for f in tr.fields()[:3]]
    g = torch.Generator(device="cuda")
    g.manual_seed(99 + rank)
    copies = [base] + [[f[p].contiguous() for f in base]
                       for p in (torch.randperm(n, device="cuda", generator=g) for _ in range(3))]
    where = torch.empty(n, dtype=torch.int32, device="cuda")
    saf = torch.empty(n, dtype=torch.float64, device="cuda")
    out = {"workload": "toy detector (40 daughters), 2^22 points uniform in the mother (daughters included), "
                       "4 rotating copies; steps %d" % steps}
    for mode, key in ((0, "contains_fp64"), (1, "contains_fp32_refine")):
        ms = _event_time(lambda it: pkg.geo_contains(vol, *copies[it % 4], mode=mode, where=where), steps)
        out[key] = {"value": n / (ms * 1e-3), "unit": "points/s", "ms_per_step": ms,
                    "algorithmic_gb_s": 28.0 * n / (ms * 1e-3) / 1e9}
    for mode, key in ((0, "safety_fp64"), (1, "safety_fp32_refine"), (2, "safety_estimate")):
        ms = _event_time(lambda it: pkg.geo_safety(vol, *copies[it % 4], mode=mode, safety=saf), steps)
        out[key] = {"value": n / (ms * 1e-3), "unit": "points/s", "ms_per_step": ms,
                    "algorithmic_gb_s": 32.0 * n / (ms * 1e-3) / 1e9}
    vol.close()
    return out


def shapes_leg(pkg, steps, q_sqrt, q_div):
    """Each solid's queries on their own (the per-shape algorithms of Sec. 3.1
    that Fig. 2 times per shape): DistFromOutside and DistFromInside of a box,
    a tube shell, a hollow cone, a tube segment and polycones (a cone segment
    and a six-plane bobbin), for baskets of 1024 tracks (launch-bound:
    microseconds per call) and 2^20 tracks (8 rotating copies, 403 MB > L2);
    for box, tube and cone the FP64 work per track from the routines'
    instruction mix (the identity placement's 3 subtractions included), as a
    fraction of the FP64 peak."""
    import torch
    from paper_1312_0816_gb300.scenes import Pcon

    solids = {"box": (0, (10.0, 20.0, 30.0)), "tube": (1, (5.0, 20.0, 30.0)),
              "cone": (2, (30.0, 5.0, 10.0, 8.0, 20.0)), "tube_segment": (3, (5.0, 20.0, 30.0, 0.4, 4.0)),
              "cone_segment": (4, Pcon((-30.0, 30.0), (5.0, 8.0), (10.0, 20.0), 0.4, 4.0)),
              "polycone_6": (4, Pcon((-30.0, -25.0, -20.0, 20.0, 25.0, 30.0), (0.0,) * 6,
                                     (25.0, 25.0, 10.0, 10.0, 25.0, 25.0)))}
    out = {"workload": "points uniform in 1.5x the solid's extent (inside and outside), isotropic directions; "
                       "identity placement; steps %d" % steps}
    rng = np.random.default_rng(5)
    for name, (kind, prm) in solids.items():
        if kind == 4:
            ext = np.array([max(prm.rmax)] * 2 + [max(abs(prm.z[0]), abs(prm.z[-1]))])
        else:
            ext = np.array(prm[:3]) if kind == 0 else (np.array([prm[1], prm[1], prm[2]]) if kind in (1, 3)
                                                       else np.array([max(prm[2], prm[4])] * 2 + [prm[0]]))
        row = {}
        for n in (1024, 1 << 20):
            x = rng.uniform(-1.5, 1.5, size=(n, 3)) * ext
            v = rng.normal(size=(n, 3))
            v /= np.linalg.norm(v, axis=1, keepdims=True)
            base = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (*x.T, *v.T)]
            ncp = 8 if n > 1024 else 1
            g = torch.Generator(device="cuda")
            g.manual_seed(11)
            copies = [base] + [[f[p].contiguous() for f in base]
                               for p in (torch.randperm(n, device="cuda", generator=g) for _ in range(ncp - 1))]
            res = torch.empty(n, dtype=torch.float64, device="cuda")
            for what, key in ((pkg.GEO_Q_DIST_OUT, "out"), (pkg.GEO_Q_DIST_IN, "in")):
                ms = _event_time(lambda it: pkg.geo_shape_query(kind, prm, what, *copies[it % ncp], out=res), steps)
                rec = {"value": n / (ms * 1e-3), "unit": "tracks/s", "us_per_call": ms * 1e3}
                if (key, kind) in FP64_OPS:   # instruction mixes are counted for box, tube, cone
                    a, sq, dv = FP64_OPS[(key, kind)]
                    ops = FP64_TRANSFORM_IDENTITY + a + sq * q_sqrt + dv * q_div
                    rec["fp64_dfma_equiv_per_track"] = ops
                    rec["fp64_frac"] = n * ops * 2 / (ms * 1e-3) / 1e12 / PEAK_FP64_TFLOPS
                row[f"dist_{key}_{n}"] = rec
        out[name] = row
    return out


def world_leg(pkg, scenes, rank, steps):
    """Transport steps in a tree of logical volumes (the toy detector in a
    hall with racks; 162 placed volumes, 3 levels): the step of Fig. 1 in
    each track's node followed by final localisation.  2^20 tracks; the
    states after 0..3 transport steps (flags and nodes of every kind) are
    prepared once and the timed steps rotate over them."""
    import torch

    w = scenes.world_toy()
    vols = [pkg.geo_build_volume(v) for v in w.volumes]
    W = pkg.geo_build_world(vols, w.child, w.root)
    n = 1 << 20
    tr = scenes.world_points(w, n, 11 + 1000 * rank)
    x = [torch.from_numpy(f).cuda() for f in tr.fields()]
    node = pkg.geo_world_locate(W, *x[:3])
    flag = torch.full_like(node, -1)
    states = []
    for _ in range(4):
        states.append(([t.clone() for t in x], node.clone(), flag.clone()))
        s, nn, ff = pkg.geo_world_step(W, *x, node, flag, mode=1)
        alive = node >= 0
        s = torch.where(alive, s, torch.zeros_like(s))
        for k in range(3):
            x[k] = x[k] + s * x[3 + k]
        node = torch.where(alive, nn, torch.full_like(nn, -1))
        flag = torch.where(alive, ff, torch.full_like(ff, -1))
    alive_frac = [float((st[1] >= 0).float().mean()) for st in states]
    step = torch.empty(n, dtype=torch.float64, device="cuda")
    no = torch.empty(n, dtype=torch.int32, device="cuda")
    fo = torch.empty(n, dtype=torch.int32, device="cuda")
    out = {"workload": "toy world: hall > detector (40 daughters) > shells with 8 sensors / boxes with 2 sub-boxes, "
                       "racks > tube; 162 placed volumes; 2^20 tracks uniform in the hall, states after 0..3 "
                       "transport steps in rotation (alive fractions %s); steps %d"
                       % ([round(a, 3) for a in alive_frac], steps)}
    for mode, key in ((1, "fp32_refine"), (0, "fp64_plain")):
        k = steps if mode == 1 else max(3, steps // 4)
        ms = _event_time(lambda it: pkg.geo_world_step(W, *states[it % 4][0], states[it % 4][1], states[it % 4][2],
                                                       mode=mode, step=step, node_out=no, flag_out=fo), k)
        out[key] = {"value": n / (ms * 1e-3), "unit": "tracks/s", "ms_per_step": ms, "steps": k}
    out["speedup_of_refine"] = out["fp64_plain"]["ms_per_step"] / out["fp32_refine"]["ms_per_step"]
    # a sample of the answers (state after one transport step) for the accuracy check
    xs, nd, fl = states[1]
    pkg.geo_world_step(W, *xs, nd, fl, mode=1, step=step, node_out=no, flag_out=fo)
    idx = np.sort(np.random.default_rng(41).choice(n, 20000, replace=False))
    pick = lambda t: t.cpu().numpy()[idx]
    SAMPLES_WORLD["world"] = (w, scenes.Tracks(*(pick(t) for t in xs)), pick(nd), pick(fl), pick(step), pick(no),
                              pick(fo))
    W.close()
    for v in vols:
        v.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=N_TRACKS)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-voxel", action="store_true")
    ap.add_argument("--voxel-n", type=int, default=1 << 24, help="tracks of the voxel leg (a smaller case for ncu)")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-queries", action="store_true")
    ap.add_argument("--no-shapes", action="store_true")
    ap.add_argument("--no-world", action="store_true")
    ap.add_argument("--no-segments", action="store_true")
    ap.add_argument("--no-sweep", action="store_true")
    ap.add_argument("--sweep-sizes", default=",".join(str(v) for v in SWEEP_SIZES),
                    help="basket sizes of the sweep leg, comma-separated (one size for an ncu capture)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        run_reference(args)
        return

    import torch
    import torch.distributed as tdist

    import paper_1312_0816_gb300 as pkg
    from paper_1312_0816_gb300 import scenes

    from paper_1312_0816_gb300 import replicas

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    replicas.init("nccl", device=torch.device("cuda", local))
    barrier = replicas.barrier

    def max_over_ranks(v):
        return replicas.max_over_ranks(v, device="cuda")

    sc = scenes.toy40(1)
    n = args.n
    tr = scenes.sample_tracks(sc, n, 1 + rank)
    vol = pkg.geo_build_volume(sc)
    base = [torch.from_numpy(f).cuda() for f in tr.fields()]
    copies = [base]
    g = torch.Generator(device="cuda")
    g.manual_seed(1234 + rank)
    for _ in range(N_COPIES - 1):
        perm = torch.randperm(n, device="cuda", generator=g)
        copies.append([f[perm].contiguous() for f in base])
    outs = [(torch.empty(n, dtype=torch.float64, device="cuda"), torch.empty(n, dtype=torch.int32, device="cuda"))
            for _ in range(N_COPIES)]
    stream = torch.cuda.current_stream()

    def step(k, mode):
        c = copies[k % N_COPIES]
        o = outs[k % N_COPIES]
        pkg.geo_dist_to_boundary(vol, *c, mode=mode, step=o[0], hit=o[1])

    def timed(mode, steps, warmup, clocks=None):
        """K steps bracketed by a barrier and synchronisation, timed with CUDA
        events on the launching stream (the mean over the K steps).  With clocks, nvidia-smi
        samples the timed region and, so that a short region still has its
        samples, one more second of the same launches right after it."""
        for k in range(warmup):
            step(k, mode)
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        if clocks:
            clocks.start()
            time.sleep(0.5)
            clocks.mark()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        # a spin of about a millisecond ahead of the first event, so that the
        # timed launches are queued before the device reaches it: the events
        # then bracket device time, not the host's latency to the first launch
        torch.cuda._sleep(2_000_000)
        e0.record(stream)
        for k in range(steps):
            step(k, mode)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        ms = e0.elapsed_time(e1) / steps
        clk = None
        if clocks:
            t_end, k = time.time() + 1.0, 0
            while time.time() < t_end:
                step(k, mode)
                k += 1
                if k % 64 == 0:
                    torch.cuda.synchronize()
            torch.cuda.synchronize()
            clk = clocks.stop()
            clk["sampled_over"] = "the timed region and 1 s of the same launches right after it"
        return max_over_ranks(ms), clk

    def median_ms(mode, reps):
        """Median over `reps` launches, each between its own pair of events."""
        per = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
        for k in range(reps):
            per[k][0].record(stream)
            step(k, mode)
            per[k][1].record(stream)
        torch.cuda.synchronize()
        return statistics.median(a.elapsed_time(b) for a, b in per)

    # correctness guard: both modes agree before anything is timed
    step(0, 1)
    s1, h1 = outs[0][0].clone(), outs[0][1].clone()
    step(0, 0)
    torch.cuda.synchronize()
    agree = bool(torch.equal(s1, outs[0][0]) and torch.equal(h1, outs[0][1]))
    pkg.geo_check_device_status(vol)

    clocks = Clocks(local)
    ms_ref, clk = timed(1, args.steps, args.warmup, clocks)
    # the median of at least 30 launches, each between its own events, after
    # the timed region (events between the timed launches would perturb them)
    n_med = max(30, min(args.steps, 400))
    ms_median = median_ms(1, n_med)
    ms_f64, _ = timed(0, max(3, args.steps // 20), 3)
    pkg.geo_check_device_status(vol)

    # statistics of the refine stage
    st_s, st_h, nref = pkg.geo_dist_to_boundary_stats(vol, *copies[0])
    torch.cuda.synchronize()
    nref = nref.cpu().numpy()
    hit = st_h.cpu().numpy()
    fallback = int((nref >= 1000).sum())
    evals = float(np.where(nref >= 1000, nref - 1000, nref).mean())

    # pipe rates for the roofline (measured) and the nominal peaks
    r_f32 = pkg.geo_probe_pipe(0, 1 << 15)
    r_f64 = pkg.geo_probe_pipe(1, 1 << 12)
    r_div = pkg.geo_probe_pipe(2, 1 << 9)
    r_sqrt = pkg.geo_probe_pipe(3, 1 << 9)
    q_div, q_sqrt = r_f64 / r_div, r_f64 / r_sqrt

    hit0 = np.asarray(hit)
    fm, fk = algorithmic_ops(sc, hit0)
    ops64 = fp64_ops_per_track(sc, fm, fk, q_sqrt, q_div)        # DFMA equivalents per track
    # the kernel evaluates the mother in FP64 only where its bound does not
    # lose to the winning daughter's: the work it must do is the winner's alone
    a_m, s_m, d_m = FP64_OPS[("in", sc.mother_kind)]
    ops64_winner = ops64 - (1.0 - fm) * (a_m + s_m * q_sqrt + d_m * q_div)
    Q_RATES[0], Q_RATES[1] = q_sqrt, q_div
    ops32 = fp32_ops_per_track(sc)                                # FP32 instructions per track
    hbm_bytes = 60.0
    peak_hbm = 6760.9
    try:
        peak_hbm = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"]
    except Exception:
        pass
    PEAK_HBM[0] = peak_hbm
    t_hbm = n * hbm_bytes / (peak_hbm * 1e9)
    t_f64 = n * ops64 * 2 / (PEAK_FP64_TFLOPS * 1e12)
    t_f32 = n * ops32 * 2 / (PEAK_FP32_TFLOPS * 1e12)
    t_roof = max(t_hbm, t_f64, t_f32)
    launch_s = ms_ref * 1e-3
    achieved64 = n * ops64 * 2 / launch_s / 1e12
    traffic, sha = captured_traffic()
    roof = {"bound": "alu", "achieved": achieved64, "peak": PEAK_FP64_TFLOPS, "unit": "TFLOP/s",
            "frac": achieved64 / PEAK_FP64_TFLOPS, "traffic": traffic,
            "pipe": "fp64",
            "peak_source": "nominal: 152 SMs x 2 DFMA/cycle x 2 flop x 2.07 GHz (unit counts and clock); "
                           "the probe measured %.3f TFLOP/s" % (2 * r_f64 / 1e12),
            "kernel": "k_dist_refine (one launch per step)", "kernel_sources_sha": sources_sha(),
            "algorithmic_per_track": {"hbm_bytes": hbm_bytes, "fp64_dfma_equiv": ops64, "fp32_instr": ops32},
            "fp64_count": "the mother's exit on every track, the winning daughter's transform and "
                          "DistFromOutside, the boundary point",
            "winner_only": {"fp64_dfma_equiv": ops64_winner,
                            "frac": n * ops64_winner * 2 / launch_s / 1e12 / PEAK_FP64_TFLOPS,
                            "note": "the FP64 work the filter leaves: the winner's evaluation alone "
                                    "(the mother's only where it wins) and the boundary point"},
            "t_roof_us": {"hbm": t_hbm * 1e6, "fp64": t_f64 * 1e6, "fp32": t_f32 * 1e6},
            "measured_rates": {"fp32_fma_tflops": 2 * r_f32 / 1e12, "fp64_fma_tflops": 2 * r_f64 / 1e12,
                               "fp64_div_per_s": r_div, "fp64_sqrt_per_s": r_sqrt,
                               "div_in_dfma": q_div, "sqrt_in_dfma": q_sqrt}}

    # end to end through the host-memory entry point: pinned host buffers,
    # which the step reads and writes in place over the host link; E2E_COPIES
    # permuted copies in rotation (more than L2 holds), each with its outputs
    pinned, houts = [], []
    for c in range(E2E_COPIES):
        perm = np.random.default_rng(1000 + c).permutation(n)
        pinned.append([torch.from_numpy(np.ascontiguousarray(f[perm])).pin_memory() for f in tr.fields()])
        houts.append((torch.empty(n, dtype=torch.float64).pin_memory(), torch.empty(n, dtype=torch.int32).pin_memory()))
    for c in range(E2E_COPIES):
        pkg.geo_dist_to_boundary_host(vol, *pinned[c], mode=1, step=houts[c][0], hit=houts[c][1])
    k_e2e = max(3, args.steps // 40)
    barrier()
    t0 = time.perf_counter()
    for it in range(k_e2e):
        c = it % E2E_COPIES
        pkg.geo_dist_to_boundary_host(vol, *pinned[c], mode=1, step=houts[c][0], hit=houts[c][1])
    e2e_s = max_over_ranks((time.perf_counter() - t0) / k_e2e)

    batched = None if args.no_batched else batched_leg(pkg, scenes, rank, max(10, args.steps // 40))
    voxel = None if args.no_voxel else voxel_leg(pkg, scenes, rank, max(5, args.steps // 200), args.voxel_n)
    adjoint = None if args.no_adjoint else adjoint_leg(pkg, scenes, rank, max(10, args.steps // 40))
    queries = None if args.no_queries else queries_leg(pkg, scenes, rank, max(10, args.steps // 100), sc)
    shapes = None if args.no_shapes else shapes_leg(pkg, max(10, args.steps // 100), q_sqrt, q_div)
    world = None if args.no_world else world_leg(pkg, scenes, rank, max(10, args.steps // 100))
    segments = None if args.no_segments else segments_leg(pkg, scenes, rank, max(10, args.steps // 100))
    sizes = tuple(int(v) for v in args.sweep_sizes.split(",") if v)
    sweep = None if args.no_sweep else sweep_leg(pkg, scenes, rank, max(10, args.steps // 100), vol, base, sizes)

    cpu, acc = None, None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu, acc = cpu_baseline(sc, tr, st_s.cpu().numpy(), hit0)

    if rank == 0:
        line = {
            "metric": METRIC, "value": ws * n / (ms_ref * 1e-3), "unit": "tracks/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_ref,
            "ms_median": {"value": ms_median, "launches": n_med,
                          "of": "per-launch CUDA events around each of these launches, after the timed region"},
            "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "tracks_per_gpu": n, "mode": "GEO_FP32_REFINE",
                       "l2": f"{N_COPIES} rotating basket copies ({N_COPIES * n * 60 / 1e6:.0f} MB > L2)",
                       "parallelism": f"replicas x{ws}"},
            "fp64_plain": {"value": ws * n / (ms_f64 * 1e-3), "unit": "tracks/s", "ms_per_step": ms_f64,
                           "speedup_of_refine": ms_f64 / ms_ref},
            "modes_bit_identical": agree,
            "refine": {"fp64_evals_per_track": evals, "fallback_tracks": fallback},
            "roofline": roof,
            "accuracy": acc,
            "e2e": {"value": ws * n / e2e_s, "unit": "tracks/s", "h2d_bytes_per_step": 48 * n,
                    "d2h_bytes_per_step": 12 * n,
                    "api": "geo_dist_to_boundary_host on pinned host buffers (the step reads the tracks and writes "
                           "the results in place over the host link; %d permuted copies in rotation, %.0f MB > L2; "
                           "synchronised every call)" % (E2E_COPIES, E2E_COPIES * n * 60 / 1e6)},
            "gpu_launches": args.steps,
            "clocks": clk,
            "cpu_baseline": cpu,
            "batched": batched,
            "voxel_512": voxel,
            "adjoint": adjoint,
            "contains_safety": queries,
            "shapes": shapes,
            "world": world,
            "segments": segments,
            "sweep": sweep,
        }
        print(json.dumps(line), flush=True)
    vol.close()
    if ws > 1:
        tdist.destroy_process_group()


if __name__ == "__main__":
    main()
