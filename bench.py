#!/usr/bin/env python3
"""Throughput benchmark of the GB300 Parthenon-hydro hot path.

Workload (one "step" = one full cycle: two RK stages, two ghost exchanges,
the dt reduction): a uniform 256^3-zone periodic mesh carrying a seeded
linear sound wave of amplitude 1e-4 on rho=1, p=0.6 (gamma=5/3), travelling
along the (1,1,1) diagonal, split into
blocks of 16^3, 32^3 or 64^3 zones.  The headline is FP64 with 32^3 blocks;
the other block sizes and the FP32 variant are reported under "variants".

Metric: zone-cycles/s = zones x cycles / device time (CUDA events on the
mesh's stream around K replays of the captured cycle graph, after W warm-up
cycles).  The state (671 MB in FP64, 335 MB in FP32) is larger than the
129 MB L2, so no flush is needed between cycles.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle (written from the paper; there is
no reference program to run) on a bounded sample of the same workload, on
the host cores.
Under torchrun each rank runs an independent replica (replicas only: the
single-GPU path has no exchange step between meshes); value sums the ranks.
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

import workloads as W  # noqa: E402

METRIC = "zone-cycles/s on 1 GB300 (FP64 plain vs batched/FP32) and % of HBM roofline"
MESH = 256
GAMMA = 5.0 / 3.0
PEAKS_PATH = os.path.join(ROOT, "MEASURED_PEAKS.json")
# FP64 pipe: 2 DFMA per clock per SM (measured 1.20 TFLOP/s at ~1.98 GHz on
# 152 SMs); FP32: 128 FFMA per clock per SM.
SMS = 152
SM_MAX_MHZ = 2070.0
# Algorithmic work per zone and stage launch:
#  bytes: stage 1 reads U0 and writes U1 (10 words), stage 2 reads U1 and U0
#  and writes U0 (15 words): 25 words per zone-cycle, 12.5 per launch.
WORDS_PER_ZONE_LAUNCH = 12.5
#  With the exchange inside the stage (periodic meshes), each launch also
#  writes the ghost shell of its output: 5 words per ghost cell, i.e.
#  5 ((n+4)^3 - n^3) / n^3 words per zone for blocks of n^3.


def ghost_words_per_zone(block):
    return 5.0 * ((block + 4) ** 3 - block ** 3) / block ** 3
#  flops: counted from the method, one flop per add/sub/mul/div/sqrt.
FLOPS_PER_ZONE_CYCLE = 1078.0


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def peaks():
    try:
        with open(PEAKS_PATH) as f:
            p = json.load(f)
        return p, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class Clocks:
    """nvidia-smi sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index=0):
        self.dev = device_index
        self.p = None
        self.path = os.path.join(tempfile.gettempdir(), "ph_clocks_%d.csv" % os.getpid())

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        try:
            os.remove(self.path)
        except OSError:
            pass
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def build_mesh(ph, block, precision, nbfac=1, bc=None):
    n = MESH // nbfac
    nb = n // block
    cfg = ph.make_config((block,) * 3, (nb,) * 3, precision=precision, bc=bc)
    m = ph.Mesh(cfg)
    geo = W.Geometry((block,) * 3, (nb,) * 3)
    return m, geo


# Oblique wave vector: every variable varies along every axis, so no slope is
# trivially zero (a wave along x1 leaves v2, v3 and every x2/x3 difference
# exactly 0, which skips most limiter divisions).
WAVE_K = (1, 1, 1)


def wave_state(geo, leaves, dtype, kvec=WAVE_K):
    return W.linear_wave(geo, leaves, gamma=GAMMA, seed=0, amp=1e-4, kvec=kvec).astype(dtype)


def time_variant(ph, torch, block, precision, steps, warmup, kvec=WAVE_K, bc=None, barrier=None):
    """Device-timed cycles of one variant; returns a dict.  barrier (if given)
    is called right before and right after the timed cycles, with the device
    synchronised on both sides (all ranks start and end the timed region
    together)."""
    m, geo = build_mesh(ph, block, precision, bc=bc)
    dtype = np.float32 if precision == "fp32" else np.float64
    U = wave_state(geo, m.tree(), dtype, kvec)
    m.set_state(U)
    zones = MESH ** 3
    stream = torch.cuda.current_stream()
    m.step(warmup)
    torch.cuda.synchronize()
    if barrier:
        barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    m.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    if barrier:
        barrier()
    ms = e0.elapsed_time(e1)
    # per-launch device times over the same number of cycles (events between launches)
    prof = m.profile(steps)
    rc, floors, nonfinite = m.status()
    res = {
        "block": block, "precision": precision, "nblocks": m.nblocks, "tile": list(m.tile()),
        "wave_k": list(kvec),
        "ms_per_cycle": ms / steps, "zone_cycles_per_s": zones * steps / (ms / 1e3),
        "launches_per_cycle": m.launches_per_cycle(),
        "stage_ms_avg": float((prof[0] + prof[2]) / (2 * steps)),
        "ghost_ms_avg": float((prof[1] + prof[3]) / (2 * steps)),
        "launch_ms": [float(x / steps) for x in prof],
        "floors": floors, "nonfinite": nonfinite,
    }
    m.close()
    return res


STAGE_SOURCES = ("ph_stage.cuh", "ph_stage_pair.cuh", "ph_device.cuh", "ph_tma.cuh")


def kernel_source_hash():
    """SHA-256 of the stage kernels' source with comments and whitespace
    removed: a change of the code, not of its comments, retires a traffic
    capture."""
    import hashlib
    import re
    h = hashlib.sha256()
    for f in STAGE_SOURCES:
        text = open(os.path.join(ROOT, "paper_2202_12309_gb300", "csrc", f)).read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        text = re.sub(r"//[^\n]*", " ", text)
        h.update(" ".join(text.split()).encode())
    return h.hexdigest()


def measured_traffic(precision, block):
    """DRAM bytes of one stage launch at this mesh size, from the committed ncu
    capture (profiles/stage_kernel_traffic.json: mean of the stage-1 and stage-2
    launches, per zone, scaled by zones), or None when the kernel source changed
    since the capture or the block size differs from the captured one."""
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "stage_kernel_traffic.json")))
        if kernel_source_hash() != rec["kernel_source_sha256"] or rec[precision]["block"] != block:
            return None
        return rec[precision]["bytes_per_zone"] * MESH ** 3
    except Exception:
        return None


def fma_peak(ph, torch, kind="fp64", reps=10, warm=5):
    """Measured peak of one arithmetic pipe: the best of `reps` CUDA-event
    timings of ph_debug_fma_rate (8 independent multiply-add chains per
    thread, 8 CTAs of 256 threads per SM, ~16 ms a launch) on the current
    stream, after `warm` untimed launches, in TFLOP/s.  Run after the
    headline, on a GPU already at its working clocks."""
    ctas = SMS * 8
    iters = 4096 if kind == "fp64" else 4096 * 64
    out = torch.empty(ctas * 256, dtype=torch.float64 if kind == "fp64" else torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    for _ in range(warm):
        flops = ph.debug_fma_rate(kind, ctas, iters, out)
    best = float("inf")
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ph.debug_fma_rate(kind, ctas, iters, out)
        e1.record(stream)
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1) / 1e3)
    return flops / best / 1e12


def roofline_for(v, pk, peak_kind, fp64_measured=None):
    """Roofline of the stage kernel: the binding roof (FP32: HBM; FP64: the
    FP64 pipe), with the other roof's fraction beside it.  Algorithmic bytes
    are the streaming model's 12.5 words per zone and launch (100 B per
    zone-cycle FP32, 200 B FP64); the ghost shell a periodic stage also
    writes is overhead, reported separately."""
    zones = MESH ** 3
    traffic = measured_traffic(v["precision"], v["block"])
    word = 4 if v["precision"] == "fp32" else 8
    words = WORDS_PER_ZONE_LAUNCH
    ghost = ghost_words_per_zone(v["block"]) * word if v.get("launches_per_cycle") == 3 else 0.0
    secs = v["stage_ms_avg"] / 1e3
    gbs = words * word * zones / secs / 1e9
    hbm_peak = pk.get("hbm_gbs", 6800.0)
    tflops = FLOPS_PER_ZONE_CYCLE * 0.5 * zones / secs / 1e12
    hbm = {"achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak,
           "algorithmic_bytes_per_zone_launch": words * word,
           "ghost_bytes_per_zone_launch": ghost,
           "peak_source": peak_kind + " hbm_gbs (copy bandwidth)"}
    if v["precision"] == "fp32":
        out = {"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s",
               "frac": gbs / hbm_peak, "traffic": traffic,
               "traffic_launch": "mean of stage 1 and 2 (ncu)",
               "peak_source": peak_kind + " hbm_gbs (copy bandwidth)",
               "algorithmic_bytes_per_zone_launch": words * word,
               "ghost_bytes_per_zone_launch": ghost}
        # the other roof: FP32 arithmetic (128 lanes per SM, fma = 2 flops)
        fp32_peak = SMS * 128 * 2 * SM_MAX_MHZ * 1e6 / 1e12
        out["alu"] = {"achieved": tflops, "peak": fp32_peak, "unit": "TFLOP/s", "frac": tflops / fp32_peak,
                      "flops_per_zone_launch": FLOPS_PER_ZONE_CYCLE * 0.5,
                      "peak_source": "FP32 pipe: 152 SMs x 128 lanes x 2 flop x 2070 MHz (derived)"}
        return out
    # FP64: bound by the FP64 pipe
    peak = SMS * 2 * 2 * SM_MAX_MHZ * 1e6 / 1e12
    out = {"bound": "alu", "achieved": tflops, "peak": peak, "unit": "TFLOP/s",
           "frac": tflops / peak, "traffic": traffic, "traffic_launch": "mean of stage 1 and 2 (ncu)",
           "peak_source": "FP64 pipe: 152 SMs x 2 DFMA/clk x 2 flop x 2070 MHz (derived)",
           "flops_per_zone_launch": FLOPS_PER_ZONE_CYCLE * 0.5,
           "hbm": hbm}
    if fp64_measured:
        out["peak_measured"] = fp64_measured
        out["frac_of_measured"] = tflops / fp64_measured
        out["peak_measured_source"] = ("measured in this run: ph_debug_fma_rate, FP64 DFMA chains, "
                                       "%d CTAs x 256 threads, best of 10" % (SMS * 8))
    return out


def batch_variant(ph, torch, precision, steps, warmup, nsim=64, seed=0, launch=None):
    """64 independent blast-wave meshes, sizes 32^3..128^3 zones in 16^3 or
    32^3 blocks (seeded), one persistent launch per cycle; autotuned."""
    members = W.batch_members(seed=seed, nsim=nsim)
    dtype = np.float32 if precision == "fp32" else np.float64
    cfgs, states, zones = [], [], 0
    for mb in members:
        nb = mb.n // mb.block
        cfg = ph.make_config((mb.block,) * 3, (nb,) * 3, precision=precision)
        cfgs.append(cfg)
        geo = W.Geometry((mb.block,) * 3, (nb,) * 3)
        m = ph.Mesh(cfg)
        states.append(W.blast(geo, m.tree(), seed=mb.seed, center=mb.center, p_in=mb.p_in).astype(dtype))
        m.close()
        zones += mb.n ** 3
    B = ph.Batch(cfgs)
    for s, U in enumerate(states):
        B.set_state(s, U)
    t0 = time.perf_counter()
    if launch:
        B.set_launch(launch)
        choice = B.launch()
    else:
        choice = B.autotune(1)
    tune_s = time.perf_counter() - t0
    B.step(warmup)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    stream = torch.cuda.current_stream()
    e0.record(stream)
    B.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    rc, floors, nonfinite = B.status()
    B.close()
    return {"workload": "batched: %d independent blast-wave meshes (sizes 32^3-128^3, blocks 16^3/32^3), "
                        "one persistent launch per cycle" % nsim,
            "precision": precision, "zones": zones, "ms_per_cycle": ms / steps,
            "zone_cycles_per_s": zones * steps / (ms / 1e3), "launch": list(choice),
            "autotune_s": tune_s, "status": rc, "floors": floors, "nonfinite": nonfinite}


def scalar_variant(ph, torch, steps, warmup, precision="fp64", nscalars=2, block=32):
    """The 256^3 wave with passive scalars carried along (two smooth
    concentrations): the cost of advecting extra conserved variables."""
    nb = MESH // block
    cfg = ph.make_config((block,) * 3, (nb,) * 3, precision=precision, nscalars=nscalars)
    m = ph.Mesh(cfg)
    geo = W.Geometry((block,) * 3, (nb,) * 3)
    dtype = np.float32 if precision == "fp32" else np.float64
    U = wave_state(geo, m.tree(), np.float64)
    conc = [W.smooth_random_density(geo, m.tree(), seed=30 + s)[:, 0:1] - 0.5 for s in range(nscalars)]
    m.set_state(np.concatenate([U] + [U[:, 0:1] * c for c in conc], axis=1).astype(dtype))
    stream = torch.cuda.current_stream()
    m.step(warmup)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    m.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    tile = list(m.tile())
    m.close()
    return {"workload": "%d^3 wave with %d passive scalars, %d blocks of %d^3" % (MESH, nscalars, nb ** 3, block),
            "precision": precision, "tile": tile, "ms_per_cycle": ms / steps,
            "zone_cycles_per_s": MESH ** 3 * steps / (ms / 1e3)}


def shard_variant(ph, torch, steps, warmup, nshards=2, precision="fp64", block=32):
    """The 256^3 wave as `nshards` shards of one process on this GPU
    (ph_shards_step): the decomposed cycle with its pack / copy / unpack
    exchange and the dt reduction over shards, against the same mesh in one
    piece.  Wall-clock around the cycles (the shards run on their own
    streams), synchronised on both sides."""
    nb = MESH // block
    cfg = ph.make_config((block,) * 3, (nb,) * 3, precision=precision)
    sm = ph.ShardedMesh(cfg, nshards)
    geo = W.Geometry((block,) * 3, (nb,) * 3)
    dtype = np.float32 if precision == "fp32" else np.float64
    sm.set_state(wave_state(geo, sm.tree(), dtype))
    sm.step(warmup)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sm.step(steps)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    halo = sum(sh.halo(p)[0][2] for sh in sm.shards for p in range(nshards) if p != sh.shard)
    rcs = [sh.status()[0] for sh in sm.shards]
    sm.close()
    return {"workload": "%d^3 wave as %d shards of one process on one GPU (%d blocks of %d^3), "
                        "pack / device copy / unpack exchange, dt reduced over shards" % (MESH, nshards, nb ** 3, block),
            "precision": precision, "nshards": nshards, "ms_per_cycle": dt / steps * 1e3,
            "zone_cycles_per_s": MESH ** 3 * steps / dt, "halo_cells_per_exchange": int(halo),
            "status": max(rcs)}


def restart_variant(ph, torch, block=32):
    """Write and read a restart file of the 256^3 FP64 benchmark mesh (state,
    tree, scalars) in the system's temporary directory: GB/s of file bytes,
    each direction timed once after one untimed round."""
    m, geo = build_mesh(ph, block, "fp64")
    m.set_state(wave_state(geo, m.tree(), np.float64))
    m.step(1)
    path = os.path.join(tempfile.gettempdir(), "ph_restart_%d.phr" % os.getpid())
    try:
        m.save(path)
        r = ph.Mesh.load(path)
        r.close()
        t0 = time.perf_counter()
        m.save(path)
        t1 = time.perf_counter()
        r = ph.Mesh.load(path)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        same = bool(np.array_equal(r.get_state(), m.get_state()))
        r.close()
        nbytes = os.path.getsize(path)
    finally:
        if os.path.exists(path):
            os.remove(path)
    m.close()
    return {"workload": "restart file of the %d^3 FP64 mesh (%d blocks of %d^3)" % (MESH, (MESH // block) ** 3, block),
            "bytes": nbytes, "save_s": t1 - t0, "load_s": t2 - t1,
            "save_gbs": nbytes / (t1 - t0) / 1e9, "load_gbs": nbytes / (t2 - t1) / 1e9,
            "bitwise_state": same}


def two_level_variant(ph, torch, steps, warmup):
    """Blast wave on a two-level mesh: root 128^3 zones in 16^3 blocks, the
    central cube of side 0.4 refined (static) plus adaptive refinement at a
    density-gradient threshold of 0.05; FP64.  Each cycle reads the refinement
    flags on the host, so the time is wall-clock around the cycles."""
    nx, nb = (16, 16, 16), (8, 8, 8)
    cfg = ph.make_config(nx, nb, max_level=1, static_region=1, adaptive=1)
    m = ph.Mesh(cfg)
    geo = W.Geometry(nx, nb)
    m.set_state(W.blast(geo, m.tree(), seed=0))
    m.step(warmup)
    torch.cuda.synchronize()
    zones = 0
    t0 = time.perf_counter()
    for _ in range(steps):
        zones += m.nblocks * 16 ** 3
        m.step(1)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    rc, floors, nonfinite = m.status()
    nblocks = m.nblocks
    m.close()
    return {"workload": "two-level blast: root 128^3 in 16^3 blocks, static cube 0.4 + adaptive (0.05)",
            "precision": "fp64", "leaves": nblocks, "zone_cycles_per_s": zones / dt,
            "ms_per_cycle": dt / steps * 1e3, "status": rc, "floors": floors}


def multilevel_variant(ph, torch, steps, warmup, max_level=2, precision="fp64"):
    """Kelvin-Helmholtz shear layers on an adaptive tree of max_level+1
    levels: root 128 x 128 x 32 zones in 16^3 blocks, refinement at a
    density-gradient threshold of 0.05 (the layers refine to the finest
    level, touching blocks within one level).  Each cycle reads the
    refinement flags on the host, so the time is wall-clock around the
    cycles; zones are counted per cycle over the leaves of that cycle."""
    nx, nb = (16, 16, 16), (8, 8, 2)
    cfg = ph.make_config(nx, nb, max_level=max_level, adaptive=1, gamma=1.4, precision=precision,
                         xmin=(-0.5, -0.5, -0.125), xmax=(0.5, 0.5, 0.125))
    m = ph.Mesh(cfg)
    geo = W.Geometry(nx, nb, tuple(cfg.xmin), tuple(cfg.xmax))
    dtype = np.float32 if precision == "fp32" else np.float64
    m.set_state(W.kelvin_helmholtz(geo, m.tree(), seed=0).astype(dtype))
    m.step(warmup)
    torch.cuda.synchronize()
    zones = 0
    t0 = time.perf_counter()
    for _ in range(steps):
        zones += m.nblocks * 16 ** 3
        m.step(1)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    rc, floors, nonfinite = m.status()
    tree = m.tree()
    m.close()
    return {"workload": "adaptive Kelvin-Helmholtz, %d levels: root 128x128x32 in 16^3 blocks" % (max_level + 1),
            "precision": precision, "leaves": int(len(tree)),
            "leaves_per_level": [int((tree[:, 0] == l).sum()) for l in range(max_level + 1)],
            "zone_cycles_per_s": zones / dt, "ms_per_cycle": dt / steps * 1e3,
            "status": rc, "floors": floors}


def adjoint_variant(ph, torch, precision, cycles=20, ckpt=5):
    """Gradient of the L2 density loss after 20 cycles on 64^3 zones (8 blocks
    of 32^3), checkpoint every 5: forward + recompute + reverse time."""
    nx, nb = (32, 32, 32), (2, 2, 2)
    dtype = np.float32 if precision == "fp32" else np.float64
    cfg = ph.make_config(nx, nb, precision=precision)
    geo = W.Geometry(nx, nb)
    m = ph.Mesh(cfg)
    U0 = W.smooth_random_density(geo, m.tree(), seed=21).astype(dtype)
    target = W.density_target(geo, m.tree(), seed=22)
    m.set_state(U0)
    m.step(cycles)
    Uf = m.get_state()
    dLdU = np.zeros_like(U0)
    dLdU[:, 0] = 2.0 * (Uf[:, 0] - target)
    m.adjoint(U0, dLdU, cycles, ckpt)  # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    m.adjoint(U0, dLdU, cycles, ckpt)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    # the same with U0, dL/dU and the gradient resident in device memory
    U0d = torch.from_numpy(U0).cuda()
    dLdUd = torch.from_numpy(dLdU).cuda()
    m.adjoint(U0d, dLdUd, cycles, ckpt)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    m.adjoint(U0d, dLdUd, cycles, ckpt)
    torch.cuda.synchronize()
    dtd = time.perf_counter() - t0
    m.close()
    zones = 64 ** 3
    return {"workload": "adjoint: 64^3 zones (8 blocks of 32^3), %d cycles, checkpoint every %d" % (cycles, ckpt),
            "precision": precision, "seconds_per_gradient": dt,
            "seconds_per_gradient_device": dtd,
            "zone_cycles_per_s": zones * cycles / dt,
            "note": "forward + recomputation + reverse; seconds_per_gradient with host arrays in and out "
                    "(copies inside), _device with device tensors"}


def e2e_variant(ph, torch, block, precision, steps, warmup, nbuf=3):
    """Same metric through the public API with pinned host buffers: every step
    copies a state in from the host (ph_set_state_async), runs one cycle and
    reads the new state back to the host (ph_get_state_async).  Steps rotate
    over `nbuf` meshes on as many streams; each step's cycle waits for the
    previous step's cycle (an event), so the cycles run one after the other
    at full speed while the other meshes' transfers (the read-back of the
    state before and the copy-in of the state after) overlap it.  The timed
    region ends when every stream has drained."""
    streams = [torch.cuda.Stream() for _ in range(nbuf)]
    meshes = []
    for st in streams:
        n = MESH
        nb = n // block
        cfg = ph.make_config((block,) * 3, (nb,) * 3, precision=precision)
        meshes.append(ph.Mesh(cfg, stream=st.cuda_stream))
    geo = W.Geometry((block,) * 3, (MESH // block,) * 3)
    dtype = np.float32 if precision == "fp32" else np.float64
    U = wave_state(geo, meshes[0].tree(), dtype)
    host_in = [torch.from_numpy(U.copy()).pin_memory() for _ in range(nbuf)]
    host_out = [torch.empty_like(host_in[0]).pin_memory() for _ in range(nbuf)]

    def run(nsteps):
        done = None
        for k in range(nsteps):
            m, st = meshes[k % nbuf], streams[k % nbuf]
            m.set_state(host_in[k % nbuf].numpy(), sync=False)
            if done is not None:
                st.wait_event(done)
            m.step(1)
            done = torch.cuda.Event()
            done.record(st)
            m.get_state(host_out[k % nbuf].numpy(), sync=False)

    run(max(2, warmup))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    run(steps)
    for st in streams:
        st.synchronize()
    dt = time.perf_counter() - t0
    nbytes = host_in[0].numel() * host_in[0].element_size()
    for m in meshes:
        m.close()
    return {"value": MESH ** 3 * steps / dt, "unit": "zone-cycles/s",
            "h2d_bytes_per_step": int(nbytes), "d2h_bytes_per_step": int(nbytes),
            "note": "%d meshes on %d streams, cycles in sequence, the other meshes' transfers "
                    "overlapping each cycle" % (nbuf, nbuf)}


def oracle_rate(block, n_sample, cycles, warmup=0):
    """FP64 oracle zone-cycles/s on an n_sample^3 mesh of the same workload,
    in this process (one core)."""
    import oracle as O
    nb = max(1, n_sample // block)
    blk = min(block, n_sample)
    cfg = O.make_config((blk,) * 3, (nb,) * 3)
    om = O.OracleMesh(cfg)
    geo = W.Geometry((blk,) * 3, (nb,) * 3)
    om.set_state(wave_state(geo, om.tree(), np.float64))
    if warmup:
        om.step(warmup)
    t0 = time.perf_counter()
    om.step(cycles)
    dt = time.perf_counter() - t0
    return (blk * nb) ** 3 * cycles / dt, (blk * nb), dt


def _oracle_worker(a):
    block, n_sample, cycles, warmup = a
    rate, n, secs = oracle_rate(block, n_sample, cycles, warmup)
    return n ** 3 * cycles, n, secs


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def host_cpu():
    """The host CPU as /proc/cpuinfo names it (model name, or the Arm
    implementer / part numbers), and the machine type."""
    import platform
    name = ""
    try:
        info = open("/proc/cpuinfo").read().splitlines()
        fields = dict(l.split(":", 1) for l in info if ":" in l)
        fields = {k.strip(): v.strip() for k, v in fields.items()}
        name = fields.get("model name") or ("Arm implementer %s part %s" % (
            fields.get("CPU implementer", "?"), fields.get("CPU part", "?")))
    except OSError:
        pass
    return "%s (%s)" % (name or "unknown", platform.machine())


def oracle_rate_all_cores(block, n_sample, cycles, warmup=0):
    """The same oracle run as one independent process per host core (each on
    its own copy of the sample, as replicas): aggregate zone-cycles/s over the
    slowest process's time.  Processes are spawned, never forked."""
    import multiprocessing as mp
    import oracle as O
    O.build()  # once, before the workers load it
    n = host_cores()
    with mp.get_context("spawn").Pool(n) as pool:
        res = pool.map(_oracle_worker, [(block, n_sample, cycles, warmup)] * n, chunksize=1)
    work = sum(r[0] for r in res)
    secs = max(r[2] for r in res)
    return work / secs, res[0][1], secs, n


def rank_reduce(x, op, world, device):
    """max or min of x over the ranks of the default process group (x when
    there is one rank)."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.MIN)
    return float(t.item())


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def headline_config(block, precision, nb, world=1):
    """The `config` of the benchmark line: the workload both arms report on."""
    cfg = {"workload": "uniform %d^3-zone periodic linear sound wave (A=1e-4, k=2pi(1,1,1)), "
                       "%d blocks of %d^3, 2 ghost zones, %s, 1 cycle per step"
                       % (MESH, nb, block, precision.upper()),
           "zones": MESH ** 3, "block": block, "nblocks": nb,
           "l2": "state %.0f MB > 129 MB L2: no flush needed"
                 % (MESH ** 3 * 5 * (8 if precision == "fp64" else 4) / 1e6 * (1 + 4.0 / block) ** 3),
           "parallelism": "replicas" if world > 1 else "single GPU"}
    return cfg


def run_reference(args):
    """The reference arm: the FP64 CPU oracle (written from the paper; there is
    no reference program) on the host cores, on the headline's config and
    metric.  Each step is one oracle cycle of a bounded sample of that
    workload (a 64^3-zone piece, 8 blocks of 32^3, in one process per core);
    value = zone-cycles/s over all cores."""
    world, rank, _ = dist_setup(args)
    if rank != 0:
        return 0
    block, n_sample = 32, 64
    value, n, secs, cores = oracle_rate_all_cores(block, n_sample, args.steps, args.warmup)
    nb = (MESH // args.block) ** 3
    sample = ("%d processes, each a 64^3-zone sample of the workload (8 blocks of 32^3), "
              "%d cycles after %d warm-up, %.1f s" % (cores, args.steps, args.warmup, secs))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "zone-cycles/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": secs / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": headline_config(args.block, args.precision, nb, world=1),
        "cpu_baseline": {"value": value, "unit": "zone-cycles/s", "cores": cores, "kind": "oracle",
                         "cpu": host_cpu(), "sample": sample},
        "e2e": {"value": value, "unit": "zone-cycles/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--block", type=int, default=32)
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32"])
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--quick", action="store_true", help="headline only: no variants, e2e, CPU leg")
    ap.add_argument("--mesh", type=int, default=256, help="zones per dimension (profiling runs)")
    ap.add_argument("--batch-launch", help="TX,TY,KC,CTAS: skip the batch autotuner (profiling runs)")
    ap.add_argument("--only", choices=["batch", "two_level", "multilevel", "adjoint", "restart", "scalars", "e2e",
                                       "shards"],
                    help="run one variant workload only and print its record (profiling runs)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    global MESH
    MESH = args.mesh
    if args.quick:
        args.no_variants = args.no_cpu = True
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import paper_2202_12309_gb300 as ph
    from paper_2202_12309_gb300 import build as B

    world, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    if rank == 0 or not os.path.exists(ph.LIB_PATH):
        B.build()
    if world > 1:
        torch.distributed.barrier()
    ph.use_torch_allocator()
    pk, peak_kind = peaks()
    if args.only:
        if args.only == "batch":
            launch = [int(x) for x in args.batch_launch.split(",")] if args.batch_launch else None
            rec = batch_variant(ph, torch, args.precision, args.steps, args.warmup, launch=launch)
        elif args.only == "two_level":
            rec = two_level_variant(ph, torch, args.steps, args.warmup)
        elif args.only == "restart":
            rec = restart_variant(ph, torch)
        elif args.only == "multilevel":
            rec = multilevel_variant(ph, torch, args.steps, args.warmup)
        elif args.only == "scalars":
            rec = scalar_variant(ph, torch, args.steps, args.warmup, precision=args.precision)
        elif args.only == "e2e":
            rec = e2e_variant(ph, torch, args.block, args.precision, args.steps, args.warmup)
        elif args.only == "shards":
            rec = shard_variant(ph, torch, args.steps, args.warmup, precision=args.precision)
        else:
            rec = adjoint_variant(ph, torch, args.precision)
        if rank == 0:
            print(json.dumps(rec), flush=True)
        return 0

    # headline: timed with clocks sampled; barrier + max over ranks
    clocks = Clocks(local)
    barrier = torch.distributed.barrier if world > 1 else None
    torch.cuda.synchronize()
    clocks.start()
    head = time_variant(ph, torch, args.block, args.precision, args.steps, args.warmup, barrier=barrier)
    ck = clocks.stop()
    fp64_peak = fma_peak(ph, torch, "fp64")
    ms = rank_reduce(head["ms_per_cycle"] * args.steps, "max", world, "cuda")
    value = world * MESH ** 3 * args.steps / (ms / 1e3)

    # end to end through the public API, right after the headline (before the
    # variants, whose restart leg writes and reads a state file on the host)
    e2e = None
    if not args.quick:
        e2e = e2e_variant(ph, torch, args.block, args.precision, args.steps, args.warmup)
    if world > 1 and e2e is not None:
        e2e["value"] = rank_reduce(e2e["value"], "min", world, "cuda") * world

    variants = []
    if not args.no_variants:
        for prec in ("fp64", "fp32"):
            for block in (16, 32, 64):
                if prec == args.precision and block == args.block:
                    continue
                v = time_variant(ph, torch, block, prec, args.steps, args.warmup)
                v["roofline"] = roofline_for(v, pk, peak_kind, fp64_peak)
                variants.append(v)
                log("variant %s block %d: %.3e zone-cycles/s" % (prec, block, v["zone_cycles_per_s"]))
        for prec in ("fp64", "fp32"):
            v = time_variant(ph, torch, args.block, prec, args.steps, args.warmup, kvec=(1, 0, 0))
            v["roofline"] = roofline_for(v, pk, peak_kind, fp64_peak)
            v["workload"] = "wave along x1 only (v2, v3 and all x2/x3 differences exactly 0)"
            variants.append(v)
            log("variant %s x1-wave: %.3e zone-cycles/s" % (prec, v["zone_cycles_per_s"]))
        for prec in ("fp64", "fp32"):
            v = time_variant(ph, torch, args.block, prec, args.steps, args.warmup,
                             bc=("reflect",) * 6)
            v["roofline"] = roofline_for(v, pk, peak_kind, fp64_peak)
            v["workload"] = "closed box: reflecting walls on all six faces"
            variants.append(v)
            log("variant %s reflecting box: %.3e zone-cycles/s" % (prec, v["zone_cycles_per_s"]))
        for prec in ("fp32", "fp64"):
            v = batch_variant(ph, torch, prec, args.steps, args.warmup)
            variants.append(v)
            log("batched %s: %.3e zone-cycles/s, launch %s" % (prec, v["zone_cycles_per_s"], v["launch"]))
        v = two_level_variant(ph, torch, args.steps, args.warmup)
        variants.append(v)
        log("two-level: %.3e zone-cycles/s (%d leaves)" % (v["zone_cycles_per_s"], v["leaves"]))
        for ml in (2, 3):
            v = multilevel_variant(ph, torch, args.steps, args.warmup, max_level=ml)
            variants.append(v)
            log("KH %d levels: %.3e zone-cycles/s (leaves per level %s)"
                % (ml + 1, v["zone_cycles_per_s"], v["leaves_per_level"]))
        for prec in ("fp64", "fp32"):
            v = adjoint_variant(ph, torch, prec)
            variants.append(v)
            log("adjoint %s: %.4f s per gradient (%.4f s with device-resident inputs)"
                % (prec, v["seconds_per_gradient"], v["seconds_per_gradient_device"]))
        for prec in ("fp64", "fp32"):
            v = scalar_variant(ph, torch, args.steps, args.warmup, precision=prec)
            variants.append(v)
            log("%s with 2 passive scalars: %.3e zone-cycles/s" % (prec, v["zone_cycles_per_s"]))
        for ns in (2, 4):
            v = shard_variant(ph, torch, args.steps, args.warmup, nshards=ns)
            variants.append(v)
            log("fp64 in %d shards: %.3e zone-cycles/s (%d halo cells per exchange)"
                % (ns, v["zone_cycles_per_s"], v["halo_cells_per_exchange"]))
        v = restart_variant(ph, torch)
        variants.append(v)
        log("restart: save %.2f GB/s, load %.2f GB/s (%.0f MB)" % (v["save_gbs"], v["load_gbs"], v["bytes"] / 1e6))

    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return 0

    cpu = None
    if not args.no_cpu:
        # about 10 s of oracle work per host core: 8 cycles of a 128^3 sample in
        # one process per core
        ncyc = 8
        rate, n, secs, cores = oracle_rate_all_cores(args.block, 128, ncyc)
        cpu = {"value": rate, "unit": "zone-cycles/s", "cores": cores, "kind": "oracle", "cpu": host_cpu(),
               "sample": "%d processes, each %d^3 zones of the same workload (blocks of %d^3), "
                         "%d cycles, %.1f s; %.3g zone-cycles/s per core"
                         % (cores, n, min(args.block, n), ncyc, secs, rate / cores)}

    roof = roofline_for(head, pk, peak_kind, fp64_peak)
    nb = (MESH // args.block) ** 3
    line = {
        "metric": METRIC, "value": value, "unit": "zone-cycles/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": head["ms_per_cycle"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if args.precision == "fp64" else "f32", "data": "synthetic",
        "config": headline_config(args.block, args.precision, nb, world=world),
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": head["launches_per_cycle"] * args.steps,
        "clocks": ck,
        "kernel_ms": {"tile": head["tile"], "stage_avg": head["stage_ms_avg"], "ghost_avg": head["ghost_ms_avg"],
                      "per_launch": head["launch_ms"]},
        "variants": variants,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
