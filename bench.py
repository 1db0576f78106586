#!/usr/bin/env python
"""Benchmark of the DysonNet / ABACUS local estimator on GB300.

Workload (one step): the long-range transverse-field Ising chain N = 128
(H = sum_{i<j} r^-3 sz sz + sum sx, open), a DysonNet of 4 layers x 32
channels x 32 S4 modes (w = 2) in FP32, 4096 uniform random configurations:
the local energy of every configuration, i.e. one forward pass, the output
and interlayer link tensors, and the ABACUS log-amplitude ratio of all 128
single flips of every configuration (524,288 ratios per step).

Reported: flip ratios/s of the whole step (value), the same through the C ABI
with host buffers (e2e), the ABACUS kernel alone, the full-forward recompute of
every flipped configuration on the GPU, per-kernel device time from the
library's CUDA-event tracing, the roofline of the dominant kernel, and the
CPU FP64 oracle on a bounded sample (cpu_baseline).  `--impl reference` times
the oracle alone on the host cores.
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

METRIC = "ABACUS flip ratios/s vs full-forward recompute on GB300; p50/p99 serve latency"
WORKLOAD = "lr-TFIM N=128 open, DysonNet L=4 d=32 s=32 w=2 FP32, 4096 samples x 128 single flips"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")


def _peaks():
    try:
        with open(PEAKS_FILE) as f:
            p = json.load(f)
        return p, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}, \
            "fallback"


# FP32 FFMA issue rate of GB300: 152 SMs x 128 FP32 lanes x 2 flop per FMA per clock.
SMS, FP32_LANES = 152, 128


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ["index", "clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.active",
              "clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
              "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap"]

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={','.join(self.FIELDS)}",
                                          "--format=csv,noheader,nounits", "-lms", "200", "-i", str(self.gpu)],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.th = threading.Thread(target=self._read, daemon=True)
        self.th.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == len(self.FIELDS):
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4) if r[5 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(self.rows)}


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def cpu_baseline(cfg, params, spins_np, n_samples: int):
    """The FP64 oracle (full recompute per flip) on the first n_samples configurations."""
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    os.environ.setdefault("OMP_NUM_THREADS", str(cores))
    import oracle
    oracle.build()
    sub = spins_np[:n_samples]
    oracle.eloc(cfg["desc"], params, cfg["ham"], sub[:1])       # warm (kernel taps, page-in)
    t0 = time.perf_counter()
    oracle.eloc(cfg["desc"], params, cfg["ham"], sub)
    dt = time.perf_counter() - t0
    flips = n_samples * cfg["N"]
    return {"value": flips / dt, "unit": "flip ratios/s", "cores": int(os.environ["OMP_NUM_THREADS"]),
            "kind": "oracle", "sample": f"local energy of the first {n_samples} configurations of the workload "
                                        f"({flips} ratios, full FP64 recompute per flip, OpenMP over samples)",
            "seconds": dt}


def run_reference(args):
    world, rank, _ = _dist()
    if rank != 0:
        return 0
    import synth
    cfg = synth.CONFIGS["lrtfim_n128"]
    params = synth.make_params(cfg)
    spins_np = synth.make_spins(cfg, B=max(args.ref_samples, 1))
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    os.environ.setdefault("OMP_NUM_THREADS", str(cores))
    import oracle
    oracle.build()
    sub = spins_np[:args.ref_samples]
    for _ in range(args.warmup):
        oracle.eloc(cfg["desc"], params, cfg["ham"], sub)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.eloc(cfg["desc"], params, cfg["ham"], sub)
    dt = (time.perf_counter() - t0) / max(args.steps, 1)
    flips = args.ref_samples * cfg["N"]
    value = flips / dt
    sample = (f"each step: local energy of the first {args.ref_samples} configurations of the workload "
              f"({flips} ratios, FP64 full recompute per flip)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "flip ratios/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD + " (bounded sample on the host cores)"},
            "cpu_baseline": {"value": value, "unit": "flip ratios/s", "cores": int(os.environ["OMP_NUM_THREADS"]),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "flip ratios/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def link_conv_flops(N, L, d, B):
    """FLOPs of the full-field convolutions of the link build in one step:
    a probe from source layer m crosses full convolutions at layers m+2..L-1."""
    total = 0
    for m in range(0, L - 1):
        probes = B * N * (1 if m == 0 else d)
        hops = max(0, (L - 1) - (m + 2) + 1)
        total += probes * hops * 2 * N * N * d
    return total


def dhop_bytes(N, L, d, B, fused=False):
    """HBM bytes of the vertex hops of one step: every hop reads the probe field of
    one layer and writes it back mixed (d N P values each way; P = N probes for the
    embedding chain, N d for a source chain from layer m, which makes L - 2 - m hops).
    With the fused chain ends the last hop of every source chain with a full hop
    (m <= L - 3) runs inside k_dband instead."""
    per = (L - 2) * 2 * d * N * N * 4
    per += sum((L - 2 - m - (1 if fused and m <= L - 3 else 0)) * 2 * d * N * (N * d) * 4 for m in range(1, L - 1))
    return B * per


def dband_bytes(N, L, d, w, B, WF=None):
    """HBM bytes of the fused chain ends (k_dband) of one step: for every source chain
    with a full hop (m = 1 .. L - 3) the hop output read once, the vertex matrices of
    layer L - 1 and the band of G^(L) written."""
    W = 2 * w + 1
    WF = W if WF is None else WF
    Rk = WF - 1
    chains = max(0, L - 3)
    return B * chains * (d * N * (N * d) * 4 + N * d * d * 4 + N * (2 * Rk + 1) * d * d * 4)


def bandconv_gen_flops(N, L, d, w, B, WF=None):
    """FLOPs of the band convolutions whose operand is generated in-kernel (the chain from
    layer L-2, one hop): (2R+1) band sums over N sites for each of the N d sources and d
    channels, 2 flops each."""
    if L < 3:
        return 0
    W = 2 * w + 1
    WF = W if WF is None else WF
    Rk = WF - 1
    return B * 2 * (2 * Rk + 1) * N * (N * d) * d


def bandconv_bytes(N, L, d, w, B, WF=None, fused=False):
    """HBM bytes of the last-layer band convolutions that read their operand (k_bandconv) in
    one step: the probe field read once (the embedding chain and every source chain with
    a full hop, unless its end is fused into k_dband) plus the band entries written.  The
    chain from layer L-2 generates its operand from D0 and the taps (k_bandconv_gen,
    counted in flops)."""
    W = 2 * w + 1
    WF = W if WF is None else WF
    Rk, Rl = WF - 1, WF - 1 - w
    per = d * N * N * 4 + N * (2 * Rl + 1) * d * 4
    if not fused:
        for m in range(1, L - 2):
            per += d * N * (N * d) * 4 + N * (2 * Rk + 1) * d * d * 4
    return B * per


def abacus_unique_bytes(N, L, d, dout, w, P, B, tb=4):
    """Algorithmic bytes of one ABACUS launch over all single flips of B samples:
    every cache value the flips read, counted once (per-sample caches are
    shared by that sample's N flips), plus the float64 outputs."""
    W = 2 * w + 1
    Rk, Rl = W - 1, w
    per_sample = (2 * L * N * d                 # y, chi
                  + L * dout * N * d            # rho
                  + N * dout                    # t
                  + (L - 1) * N * (2 * Rl + 1) * d   # ell
                  + P * N * (2 * Rk + 1) * d * d)    # K
    return B * (per_sample * tb + N) + B * N * 8


def measure_n1024(dn, synth, torch, barrier, lib, chains, recompute_flips=128, L=6):
    """ABACUS ratios/s given caches, cache-build time and the GPU full-forward recompute
    at N = 1024 for the L-layer, 64-channel, 64-mode model (FP32, long-range TFIM
    chains, all N single flips per chain; the recompute is timed on a sample of
    `recompute_flips` flips per chain and scaled per ratio).  The ABACUS roofline: the
    cache bytes the flips need, once, over the layer kernels' device time (a separate
    traced pass) and over the whole ABACUS call."""
    Nn = 1024
    torch.cuda.empty_cache()          # the caches get fresh allocations, not the earlier workloads' pieces
    desc = synth.ModelDesc(L=L, d=64, s=64, w=2, dh=64, dout=2, periodic=0)
    params = synth.init_params(desc, 1005, a_scale=10.0)
    spins_np = synth.spins_uniform(chains, Nn, 2005)
    model = dn.Model(desc, params)
    spins = torch.from_numpy(spins_np).cuda()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    # Warm-up: weights, taps and kernels for this N (one chain).
    model.forward_cache(spins[:1], prec="fp32").destroy()
    barrier()
    ev0.record()
    cache = model.forward_cache(spins, prec="fp32")
    ev1.record()
    barrier()
    build_ms = ev0.elapsed_time(ev1)
    torch.cuda.empty_cache()          # hand the link-construction scratch back to the driver
    out = cache.single_flip_ratios()
    barrier()
    reps = 3
    ev0.record()
    for _ in range(reps):
        cache.single_flip_ratios(out=out)
    ev1.record()
    barrier()
    ab_ms = ev0.elapsed_time(ev1) / reps
    lib.dn_profile_enable(1)
    for _ in range(reps):
        cache.single_flip_ratios(out=out)
    barrier()
    prof = read_profile(lib)
    lib.dn_profile_enable(0)
    cache_bytes = model.cache_bytes(Nn, 1, "fp32")
    cache.destroy()
    P = (L - 1) * (L - 2) // 2
    ab_bytes = abacus_unique_bytes(Nn, L, 64, 2, 2, P, chains)
    peaks, src = _peaks()
    lay = [v for k, v in prof.items() if k.endswith("k_ab_layer")]
    lay_ms = sum(v[1] for v in lay) / reps
    split = {k.split("/")[-1]: round(v[1] / reps, 4) for k, v in prof.items()}
    roof = {"kernel": "k_ab_layer", "bound": "hbm", "achieved": ab_bytes / (lay_ms / 1e3) / 1e9,
            "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": ab_bytes / (lay_ms / 1e3) / 1e9 / peaks["hbm_gbs"],
            "launches": sum(v[0] for v in lay) // reps, "ms": lay_ms,
            "whole_call_frac": ab_bytes / (ab_ms / 1e3) / 1e9 / peaks["hbm_gbs"],
            "algorithmic_bytes": ab_bytes, "kernels_ms": split,
            "peak_source": f"{src} (MEASURED_PEAKS hbm_gbs)"} if lay_ms > 0 else None
    sample_np, sites_np = synth.random_flips(chains, Nn, chains * recompute_flips, seed=3005)
    s_t = torch.from_numpy(sample_np).cuda()
    x_t = torch.from_numpy(sites_np).cuda()
    r = model.recompute_flip_ratios(spins, s_t, x_t, prec="fp32")
    barrier()
    ev0.record()
    model.recompute_flip_ratios(spins, s_t, x_t, prec="fp32", out=r)
    ev1.record()
    barrier()
    rc_ms = ev0.elapsed_time(ev1)
    model.close()
    ratios = chains * Nn
    ab_rate = ratios / (ab_ms / 1e3)
    rc_rate = chains * recompute_flips / (rc_ms / 1e3)
    e2e_rate = ratios / ((ab_ms + build_ms) / 1e3)
    return {"workload": "lr-TFIM N=1024 open, DysonNet L=%d d=64 s=64 w=2 FP32, %d chains x 1024 single flips"
                        % (L, chains),
            "abacus_given_caches": {"value": ab_rate, "unit": "flip ratios/s", "ms": ab_ms},
            "abacus_roofline": roof,
            "cache_build_ms": build_ms, "cache_bytes_per_chain": cache_bytes,
            "recompute": {"value": rc_rate, "unit": "flip ratios/s", "ms": rc_ms,
                          "sample": "%d random single flips per chain" % recompute_flips},
            "abacus_incl_cache_build": {"value": e2e_rate, "unit": "flip ratios/s"},
            "speedup_abacus_given_caches_over_recompute": ab_rate / rc_rate,
            "speedup_incl_cache_build_over_recompute": e2e_rate / rc_rate}


def measure_grad(dn, synth, torch, barrier, lib, B=4096, reps=2):
    """Forward + backward of the N = 256, 6-layer, 64-channel, 64-mode long-range TFIM
    model (FP32, open chain): per-configuration log-derivatives O [B][P] of B configurations
    (dn_logpsi_grad), then the sample-space SR matrix Oc Oc^T / B (dn_sr_matrices).
    Per-kernel device times from the library's tracing."""
    N = 256
    desc = synth.ModelDesc(L=6, d=64, s=64, w=2, dh=64, dout=2, periodic=0)
    params = synth.init_params(desc, 1004, a_scale=10.0)
    model = dn.Model(desc, params)
    spins = torch.from_numpy(synth.spins_uniform(B, N, 2004)).cuda()
    P = model.nparams
    O = torch.empty((B, P), dtype=torch.float32, device="cuda")
    G = torch.empty((B, B), dtype=torch.float64, device="cuda")
    lp = torch.empty(B, dtype=torch.float64, device="cuda")
    ev0, ev1, ev2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    st = torch.cuda.current_stream().cuda_stream

    def step():
        dn._check(lib.dn_logpsi_grad(model._h, N, dn._ptr(spins), B, dn.PRECISIONS["fp32"], st, dn._ptr(lp),
                                     dn._ptr(O), None, None), "dn_logpsi_grad")
        ev1.record()
        dn._check(lib.dn_sr_matrices(dn._ptr(O), B, P, dn.PRECISIONS["fp32"], st, dn._ptr(G), 0, 0, None),
                  "dn_sr_matrices")

    step()
    torch.cuda.synchronize()
    barrier()
    grad_ms = gram_ms = 0.0
    for _ in range(reps):
        ev0.record()
        step()
        ev2.record()
        torch.cuda.synchronize()
        grad_ms += ev0.elapsed_time(ev1) / reps
        gram_ms += ev1.elapsed_time(ev2) / reps
    # kernel split from separate traced passes
    lib.dn_profile_enable(1)
    for _ in range(reps):
        step()
    prof = read_profile(lib)
    lib.dn_profile_enable(0)
    barrier()
    model.close()
    tot = sum(v[1] for v in prof.values()) or 1.0
    kern = sorted(({"name": k, "launches": v[0] // reps, "ms_per_step": v[1] / reps, "share": v[1] / tot}
                   for k, v in prof.items()), key=lambda r: -r["ms_per_step"])
    gram_flop = 2.0 * B * B * P / 2            # symmetric half
    return {"workload": "lr-TFIM N=256 open, DysonNet L=6 d=64 s=64 w=2 FP32, %d configurations, %d parameters"
                        % (B, P),
            "grad": {"value": B / (grad_ms / 1e3), "unit": "configurations/s (forward + all %d log-derivatives)" % P,
                     "ms": grad_ms},
            "sr_gram": {"ms": gram_ms, "tflops": gram_flop / (gram_ms / 1e3) / 1e12,
                        "note": "Oc Oc^T / B on tcgen05, FP32 values as 3 BF16 planes (6 products), FP32 accumulation in tensor memory folded into FP32 totals every 1024 terms, K splits of <= 16384 terms summed in FP64; flops counted once per FP32 product"},
            "kernels": kern[:12]}


def measure_sampler(dn, synth, torch, barrier, C=4096, s=8, eps=0.01, sweeps=2):
    """Screened typewriter sampler (Alg. 2) on C chains of the N = 128 benchmark model (FP32):
    full sweeps (even then odd blocks of width s, one proposal per block), ambiguous window
    eps; against sequential exact Metropolis on the GPU (every proposal by a full forward
    pass of the flipped configurations, dn_recompute_flip_ratios), both on the same
    proposals and uniforms."""
    N = 128
    desc = synth.ModelDesc(L=4, d=32, s=32, w=2, dh=32, dout=2, periodic=0)
    params = synth.init_params(desc, 1002, a_scale=8.0)
    model = dn.Model(desc, params)
    spins0 = synth.spins_uniform(C, N, 2002)
    batches = []
    for sw in range(sweeps + 1):
        for parity in (0, 1):
            sites = synth.typewriter_sites(C, N, s, parity, 3000 + 2 * sw + parity)
            u = synth.uniforms(C, sites.shape[1], 5000 + 2 * sw + parity)
            batches.append((torch.from_numpy(sites).cuda(), torch.from_numpy(u).cuda()))
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    # screened sampler: warm-up sweep, then timed sweeps
    sp = torch.from_numpy(spins0).cuda()
    for sites, u in batches[:2]:
        model.sampler_batch(sp, sites, u, eps, prec="fp32")
    barrier()
    tot = {"proposals": 0, "accepted": 0, "refreshes": 0}
    ev0.record()
    for sites, u in batches[2:]:
        _, st = model.sampler_batch(sp, sites, u, eps, prec="fp32")
        for k in tot:
            tot[k] += st[k]
    ev1.record()
    barrier()
    scr_ms = ev0.elapsed_time(ev1)
    # exact sequential Metropolis, one proposal index at a time over all chains
    sp2 = torch.from_numpy(spins0).cuda()
    sample = torch.arange(C, dtype=torch.int32, device="cuda")
    fl = torch.full((C, 2), -1, dtype=torch.int32, device="cuda")
    out = torch.empty(C, dtype=torch.float64, device="cuda")

    def exact(batch):
        sites, u = batch
        for k in range(sites.shape[1]):
            fl[:, 0] = sites[:, k]
            model.recompute_flip_ratios(sp2, sample, fl, prec="fp32", out=out)
            take = u[:, k] < torch.clamp(torch.exp(2.0 * out), max=1.0)
            rows = torch.nonzero(take).flatten()
            cols = sites[rows, k].long()
            sp2[rows, cols] = -sp2[rows, cols]

    for b in batches[:2]:
        exact(b)
    barrier()
    ev0.record()
    for b in batches[2:]:
        exact(b)
    ev1.record()
    barrier()
    ex_ms = ev0.elapsed_time(ev1)
    model.close()
    props = tot["proposals"]
    return {"workload": "lr-TFIM N=128 open, DysonNet L=4 d=32 s=32 w=2 FP32, %d chains, typewriter blocks of "
                        "%d sites, eps=%g, %d sweeps" % (C, s, eps, sweeps),
            "screened": {"value": props / (scr_ms / 1e3), "unit": "proposals/s", "ms_per_sweep": scr_ms / sweeps,
                         "accepted": tot["accepted"], "refreshes": tot["refreshes"], "proposals": props},
            "exact_recompute": {"value": props / (ex_ms / 1e3), "unit": "proposals/s", "ms_per_sweep": ex_ms / sweeps},
            "speedup": ex_ms / scr_ms}


def measure_bf16_forward(dn, synth, torch, barrier, lib, B=2048, reps=3):
    """Full forward passes (log psi) of the N = 256, 6-layer, 64-channel, 64-mode model in BF16
    on the tensor cores (S4 convolutions as Toeplitz GEMMs with the configurations as columns,
    channel mixing and gate as two chained MMAs) and in FP32 on the FMA kernels, B configurations
    each; the BF16 result's largest deviation from FP32 is reported beside the timings."""
    N = 256
    desc = synth.ModelDesc(L=6, d=64, s=64, w=2, dh=64, dout=2, periodic=1)
    params = synth.init_params(desc, 1003, a_scale=10.0)
    model = dn.Model(desc, params)
    spins = torch.from_numpy(synth.spins_uniform(B, N, 2003)).cuda()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = {}
    lps = {}
    for prec in ("bf16", "fp32"):
        lps[prec] = model.full_forward(spins, prec=prec)
        barrier()
        ev0.record()
        for _ in range(reps):
            model.full_forward(spins, prec=prec)
        ev1.record()
        barrier()
        ms = ev0.elapsed_time(ev1) / reps
        lib.dn_profile_enable(1)   # kernel split from a separate traced pass
        for _ in range(reps):
            model.full_forward(spins, prec=prec)
        prof = read_profile(lib)
        lib.dn_profile_enable(0)
        out[prec] = {"value": B / (ms / 1e3), "unit": "configurations/s", "ms": ms,
                     "kernels": {k: round(v[1] / reps, 3) for k, v in sorted(prof.items(), key=lambda kv: -kv[1][1])[:6]}}
    # tensor-core work of the BF16 forward: convolution 2 N^2 d and mixing 2 x 2 N d^2 flops per layer
    flops = 6 * B * (2.0 * N * N * 64 + 4.0 * N * 64 * 64)
    out["bf16"]["tflops"] = flops / (out["bf16"]["ms"] / 1e3) / 1e12
    dev = (lps["bf16"] - lps["fp32"]).abs() / lps["fp32"].abs().clamp(min=1.0)
    out["bf16_vs_fp32_max_rel"] = float(dev.max())
    model.close()
    return {"workload": "J1-J2 ring N=256, DysonNet L=6 d=64 s=64 w=2, %d configurations, full forward" % B, **out}


def measure_bf16_j1j2(dn, synth, torch, barrier, lib, B=64):
    """Local energies of the J1-J2 ring workload model (N = 256, L = 6, d = 64, s = 64,
    zero-magnetisation configurations, connected configurations from antialigned NN and
    NNN pairs) in BF16 (tensor-core forward; links, adjoint and ABACUS at FP32 accuracy)
    and in FP32, on B configurations: pair ratios/s including the cache build, the split
    into forward, link construction and ABACUS, the BF16 deviation from FP32, and the GPU
    full-forward recompute of the same pairs.  The error against the FP64 oracle is
    measured by the GPU tests (tests/test_gpu_tc_forward.py)."""
    import numpy as np
    cfg = synth.CONFIGS["j1j2_n256"]
    desc, N = cfg["desc"], cfg["N"]
    model = dn.Model(desc, synth.make_params(cfg))
    spins_np = synth.make_spins(cfg, B)
    spins = torch.from_numpy(spins_np).cuda()
    pairs = [(b, i, (i + sep) % N) for b in range(B) for sep in (1, 2) for i in range(N)
             if spins_np[b, i] != spins_np[b, (i + sep) % N]]
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out, el = {}, {}
    for prec in ("bf16", "fp32"):
        el[prec] = torch.empty(B, dtype=torch.float64, device="cuda")
        model.local_energy(cfg["ham"], spins, prec=prec, out=el[prec])
        barrier()
        ev0.record()
        model.local_energy(cfg["ham"], spins, prec=prec, out=el[prec])
        ev1.record()
        barrier()
        ms = ev0.elapsed_time(ev1)
        lib.dn_profile_enable(1)   # split from a separate traced pass
        model.local_energy(cfg["ham"], spins, prec=prec, out=el[prec])
        prof = read_profile(lib)
        lib.dn_profile_enable(0)
        part = lambda key: sum(v[1] for k, v in prof.items() if ("/" + key + "/") in ("/" + k))
        out[prec] = {"value": len(pairs) / (ms / 1e3), "unit": "pair ratios/s (local energy incl. cache build)",
                     "ms": ms, "forward_ms": part("forward"), "adjoint_ms": part("adjoint"),
                     "links_ms": part("links"), "abacus_ms": part("abacus")}
    e16, e32 = el["bf16"].cpu().numpy(), el["fp32"].cpu().numpy()
    out["bf16_vs_fp32_eloc_max_rel"] = float(np.max(np.abs(e16 - e32) / np.maximum(1.0, np.abs(e32))))
    sample = torch.tensor([p[0] for p in pairs], dtype=torch.int32, device="cuda")
    sites = torch.tensor([[p[1], p[2]] for p in pairs], dtype=torch.int32, device="cuda")
    # ABACUS alone on one FP32 cache: every pair of both bonds grouped by site (what the
    # local energy runs) against the flip-list kernel on the antialigned pairs only.
    cache = model.forward_cache(spins, prec="fp32", max_cluster=3)
    grp = cache.pair_flip_ratios((1, 2))
    fl = cache.flip_ratios(sample, sites)
    timings = {}
    for name, fn in (("grouped", lambda: cache.pair_flip_ratios((1, 2), out=grp)),
                     ("flip_list", lambda: cache.flip_ratios(sample, sites, out=fl))):
        barrier()
        ev0.record()
        fn()
        ev1.record()
        barrier()
        timings[name] = ev0.elapsed_time(ev1)
    g_np = grp.cpu().numpy()
    g_sel = np.array([g_np[b, (j2 - j1) % N - 1, j1] for b, j1, j2 in pairs])
    f_np = fl.cpu().numpy()
    out["pair_abacus"] = {
        "grouped_ms": timings["grouped"], "flip_list_ms": timings["flip_list"],
        "grouped_pairs_evaluated": int(B * 2 * N), "antialigned_pairs": len(pairs),
        "value_grouped": len(pairs) / (timings["grouped"] / 1e3),
        "value_flip_list": len(pairs) / (timings["flip_list"] / 1e3), "unit": "pair ratios/s (caches built)",
        "max_abs_diff_grouped_vs_flip_list": float(np.max(np.abs(g_sel - f_np)))}
    cache.destroy()
    r = model.recompute_flip_ratios(spins, sample, sites, prec="fp32")
    barrier()
    ev0.record()
    model.recompute_flip_ratios(spins, sample, sites, prec="fp32", out=r)
    ev1.record()
    barrier()
    rc_ms = ev0.elapsed_time(ev1)
    out["recompute"] = {"value": len(pairs) / (rc_ms / 1e3), "unit": "pair ratios/s", "ms": rc_ms}
    model.close()
    return {"workload": "J1-J2 ring N=256 (J2/J1 = 0.5), DysonNet L=6 d=64 s=64 w=2, %d zero-magnetisation "
                        "configurations, %d antialigned NN/NNN pairs" % (B, len(pairs)), **out}


def measure_serving(dn, synth, n_req=160, rate=20.0, seed=4005):
    """Serving workload: Markov chains with N in {64, 128, 256, 512, 1024} (two each) of
    the 6-layer, 64-channel, 64-mode model (FP32), requests of 1-512 random single-flip
    proposals for a random chain.  For the ABACUS server (one launch per batch), the
    persistent ABACUS server (one resident kernel fed through a work queue) and the
    per-request full-forward recompute server: throughput with every request queued at
    once, and p50/p99 latency (submission to result in host memory) under Poisson
    arrivals at `rate` requests/s."""
    import numpy as np
    import time
    desc = synth.ModelDesc(L=6, d=64, s=64, w=2, dh=64, dout=2, periodic=0)
    params = synth.init_params(desc, 1005, a_scale=10.0)
    Ns = [64, 128, 256, 512, 1024] * 2
    chains = [synth.spins_uniform(1, N, 2005 + k)[0] for k, N in enumerate(Ns)]
    rng = np.random.default_rng(seed)
    reqs = []
    for _ in range(n_req):
        c = int(rng.integers(len(Ns)))
        F = int(rng.integers(1, 513))
        reqs.append((c, rng.integers(0, Ns[c], size=F).astype(np.int32)))
    gaps = rng.exponential(1.0 / rate, size=n_req)
    flips = sum(len(s_) for _, s_ in reqs)
    model = dn.Model(desc, params)
    res = {"workload": "chains N in {64,128,256,512,1024} x 2, DysonNet L=6 d=64 s=64 w=2 FP32, %d requests of "
                       "1-512 random single flips (%d flips)" % (n_req, flips),
           "rate_per_s": rate}
    for mode in ("abacus", "persistent", "recompute"):
        srv = dn.Server(model, prec="fp32", mode=mode, hbm_budget_bytes=24 << 30, max_batch_flips=4096,
                        max_batch_chains=16)
        t0 = time.perf_counter()
        for k, sp in enumerate(chains):
            srv.set_chain(k, sp, build_now=True)
        build_s = time.perf_counter() - t0
        for t in [srv.submit(k, np.array([0], dtype=np.int32)) for k in range(len(Ns))]:
            srv.wait(t)
        t0 = time.perf_counter()
        tickets = [srv.submit(c, s_) for c, s_ in reqs]
        for t in tickets:
            srv.wait(t)
        sat_s = time.perf_counter() - t0
        lat = []
        t_next = time.perf_counter()
        tickets = []
        for (c, s_), gap in zip(reqs, gaps):
            t_next += gap
            while time.perf_counter() < t_next:
                time.sleep(min(1e-4, max(0.0, t_next - time.perf_counter())))
            tickets.append(srv.submit(c, s_))
        for t in tickets:
            lat.append(srv.wait(t)[1])
        st = srv.stats()
        srv.close()
        lat = np.array(lat) * 1e3
        res[mode] = {"saturation": {"value": flips / sat_s, "unit": "flip ratios/s", "requests_per_s": n_req / sat_s},
                     "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                     "mean_ms": float(lat.mean()), "batches": st["batches"],
                     "cache_build_s": build_s if mode != "recompute" else None,
                     "resident_cache_bytes": st["resident_bytes"]}
    model.close()
    res["speedup_saturation"] = res["abacus"]["saturation"]["value"] / res["recompute"]["saturation"]["value"]
    res["speedup_saturation_persistent"] = (res["persistent"]["saturation"]["value"] /
                                            res["recompute"]["saturation"]["value"])
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--samples", type=int, default=4096)
    ap.add_argument("--ref-samples", type=int, default=8)
    ap.add_argument("--cpu-samples", type=int, default=512)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-recompute", action="store_true")
    ap.add_argument("--no-n1024", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-grad", action="store_true")
    ap.add_argument("--no-sampler", action="store_true")
    ap.add_argument("--no-bf16-forward", action="store_true")
    ap.add_argument("--bf16-samples", type=int, default=2048)
    ap.add_argument("--j1j2-samples", type=int, default=64)
    ap.add_argument("--grad-samples", type=int, default=4096)
    ap.add_argument("--n1024-chains", type=int, default=4)
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch
    import torch.distributed as tdist

    world, rank, local = _dist()
    torch.cuda.set_device(local)
    # Replicas: every rank runs the whole workload on its own GPU (no data-path collective).
    if world > 1:
        tdist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2603_11189_gb300 import build as B_
    if rank == 0 and B_.needs_build():
        import __graft_entry__
        __graft_entry__.build()
    if world > 1:
        tdist.barrier()
    from paper_2603_11189_gb300 import dysonnet as dn
    from paper_2603_11189_gb300 import replicas
    import synth

    lib = dn._lib()
    lib.dn_launch_count.restype = ctypes_ll()

    def barrier():
        if world > 1:
            tdist.barrier()
        torch.cuda.synchronize()

    # The long-chain lines run first, before the headline workload has allocated and freed
    # its tens of GB of caches: after that, the same N = 1024 layer kernels measured 0.65
    # instead of 0.81 of HBM (a 60 GB allocate-and-free alone does the same), an effect of
    # where the caches land in device memory, not of the kernels.
    n1024 = None if args.no_n1024 else measure_n1024(dn, synth, torch, barrier, lib, args.n1024_chains)
    # The same at depths whose exact links need no full N x N hop beyond the embedding chain
    # (L = 2: the paper's own depth; L = 3: one interlayer pair, built directly).
    n1024_shallow = None if args.no_n1024 else {
        "L%d" % Ls: measure_n1024(dn, synth, torch, barrier, lib, 16, L=Ls) for Ls in (3, 2)}
    torch.cuda.empty_cache()

    cfg = synth.CONFIGS["lrtfim_n128"]
    desc = cfg["desc"]
    N, Bs = cfg["N"], args.samples
    params = synth.make_params(cfg)
    spins_np = synth.make_spins(cfg, B=Bs)
    model = dn.Model(desc, params)
    spins = torch.from_numpy(spins_np).cuda()
    eloc = torch.empty(Bs, dtype=torch.float64, device="cuda")
    ham = cfg["ham"]

    def step():
        model.local_energy(ham, spins, prec="fp32", out=eloc)

    for _ in range(args.warmup):
        step()
    barrier()
    sampler = ClockSampler(int(os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[0])
                           if os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",")[0].isdigit() else local)
    sampler.start()
    # Timed region: tracing off (the launch counter is always on).
    launches0 = lib.dn_launch_count()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    for _ in range(args.steps):
        step()
    ev1.record()
    barrier()
    launches = lib.dn_launch_count() - launches0
    clocks = sampler.stop()
    ms = ev0.elapsed_time(ev1) / args.steps
    flips_step = Bs * N
    value, ms_max = replicas.throughput(flips_step, ms, device="cuda")

    # Per-kernel device times from a separate traced pass of the same steps (an event
    # pair around every launch); its wall time is reported beside the untraced one.
    lib.dn_profile_enable(1)
    ev0.record()
    for _ in range(args.steps):
        step()
    ev1.record()
    barrier()
    lib.dn_profile_enable(0)
    traced_ms = ev0.elapsed_time(ev1) / args.steps
    prof = read_profile(lib)
    assert np.all(np.isfinite(eloc.cpu().numpy())), "non-finite local energies"

    # End to end through the C ABI with host buffers (pinned): H2D spins, D2H energies.
    spins_host = torch.from_numpy(spins_np).pin_memory()
    eloc_host = torch.empty(Bs, dtype=torch.float64).pin_memory()
    spins_dev2 = torch.empty_like(spins)

    def e2e_step():
        spins_dev2.copy_(spins_host, non_blocking=True)
        model.local_energy(ham, spins_dev2, prec="fp32", out=eloc)
        eloc_host.copy_(eloc, non_blocking=True)

    e2e_step()
    barrier()
    ev0.record()
    for _ in range(args.steps):
        e2e_step()
    ev1.record()
    barrier()
    e2e_ms = ev0.elapsed_time(ev1) / args.steps
    e2e_value, _ = replicas.throughput(flips_step, e2e_ms, device="cuda")

    # ABACUS kernel alone and the GPU full-forward recompute of every flipped configuration.
    ab_ms = sum(v[1] for k, v in prof.items() if "/abacus/" in "/" + k) / args.steps
    build_ms = sum(v[1] for k, v in prof.items() if "/forward/" in k + "/" or "/adjoint/" in k or "/links/" in k) \
        / args.steps
    recompute = None
    if not args.no_recompute:
        sample_np, sites_np = synth.single_flips(Bs, N)
        sample, sites = torch.from_numpy(sample_np).cuda(), torch.from_numpy(sites_np).cuda()
        out = torch.empty(Bs * N, dtype=torch.float64, device="cuda")
        model.recompute_flip_ratios(spins, sample, sites, prec="fp32", out=out)
        barrier()
        ev0.record()
        reps = 2
        for _ in range(reps):
            model.recompute_flip_ratios(spins, sample, sites, prec="fp32", out=out)
        ev1.record()
        barrier()
        rms = ev0.elapsed_time(ev1) / reps
        recompute = {"value": flips_step / (rms / 1e3), "unit": "flip ratios/s", "ms": rms,
                     "speedup_of_abacus_step": (flips_step / (ms / 1e3)) / (flips_step / (rms / 1e3))}

    serving = None if args.no_serving else measure_serving(dn, synth)
    grad = None if args.no_grad else measure_grad(dn, synth, torch, barrier, lib, B=args.grad_samples)
    sampler = None if args.no_sampler else measure_sampler(dn, synth, torch, barrier)
    bf16_forward = None if args.no_bf16_forward else measure_bf16_forward(dn, synth, torch, barrier, lib,
                                                                           B=args.bf16_samples)
    bf16_j1j2 = None if args.no_bf16_forward else measure_bf16_j1j2(dn, synth, torch, barrier, lib, B=args.j1j2_samples)

    peaks, src = _peaks()
    roof, families = roofline(prof, args.steps, desc, N, Bs, peaks, src, clocks)
    kernels = sorted(((k, v[0], v[1]) for k, v in prof.items()), key=lambda x: -x[2])
    total_k = sum(k[2] for k in kernels) or 1.0
    line = {
        "metric": METRIC, "value": value, "unit": "flip ratios/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded splitmix64 weights and spins)",
        "config": {"workload": WORKLOAD, "N": N, "L": desc.L, "d": desc.d, "s": desc.s, "w": desc.w,
                   "samples_per_gpu": Bs, "flips_per_sample": N, "precision": "fp32", "parallelism": f"replicas{world}",
                   "l2": "working set > L2: the per-step caches (tens of GB) are written and read once per step"},
        "roofline": roof,
        "rooflines": families,
        "e2e": {"value": e2e_value, "unit": "flip ratios/s", "h2d_bytes_per_step": int(spins_np.nbytes),
                "d2h_bytes_per_step": int(Bs * 8)},
        "gpu_launches": int(launches),
        "clocks": clocks,
        "traced_pass_ms_per_step": traced_ms,
        "abacus_kernel": {"value": flips_step / (ab_ms / 1e3) if ab_ms else None, "unit": "flip ratios/s",
                          "ms_per_step": ab_ms},
        "cache_build_ms_per_step": build_ms,
        "recompute": recompute,
        "n1024": n1024,
        "n1024_shallow": n1024_shallow,
        "grad": grad,
        "sampler": sampler,
        "bf16_forward": bf16_forward,
        "bf16_j1j2_local_energy": bf16_j1j2,
        "serving": serving,
        "kernels": [{"name": k, "launches": n // args.steps, "ms_per_step": v / args.steps,
                     "share": v / total_k} for k, n, v in kernels[:16]],
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(cfg, params, spins_np, args.cpu_samples)
    if rank == 0:
        print(json.dumps(line), flush=True)
    model.close()
    if world > 1:
        tdist.barrier()
        tdist.destroy_process_group()
    return 0


def ctypes_ll():
    import ctypes
    return ctypes.c_longlong


def read_profile(lib):
    import ctypes
    lib.dn_profile_count.restype = ctypes.c_int
    out = {}
    buf = ctypes.create_string_buffer(256)
    n_l, ms = ctypes.c_longlong(), ctypes.c_double()
    for i in range(lib.dn_profile_count()):
        if lib.dn_profile_get(i, buf, 256, ctypes.byref(n_l), ctypes.byref(ms)) == 0 and n_l.value > 0:
            out[buf.value.decode()] = (n_l.value, ms.value)
    return out


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per algorithmic unit of each
# family (byte for the HBM-bound ones, flop for the others), from one ncu capture of every
# launch of those kernels over four steps of this workload at 64 configurations.  The
# launches have the same per-launch shapes at 64 and 4096 configurations (link sub-batches
# of at most 47 configurations; ABACUS traffic proportional to the configurations), so a
# full-size launch's traffic is the ratio times its algorithmic units.  Valid for the
# kernels as captured: a family whose kernel changes is reported with traffic null until
# it is captured again.
DRAM_PER_UNIT = {"abacus": 1.076, "links_dhop": 0.857, "links_bandconv": 0.964, "links_dband": 0.994,
                 "links_bandconv_gen": 0.0105, "links_tgemm_tc": 0.01665}


def traffic_per_launch(fam, units_per_launch):
    r = DRAM_PER_UNIT.get(fam)
    return None if r is None else r * units_per_launch


def kernel_rooflines(prof, steps, desc, N, Bs, peaks, src):
    """Rooflines of the kernel families that carry the step: the ABACUS layer
    kernels (HBM-bound: algorithmic bytes = every cache value the flips need, once
    per configuration), the Toeplitz GEMM of the link build (2 N^2 d flops per
    source column per full hop) and its vertex hops and band convolutions
    (HBM-bound: probe fields read and written once)."""
    out = {}
    P = (desc.L - 1) * (desc.L - 2) // 2
    ab = [(k, v) for k, v in prof.items() if k.endswith("/k_ab_layer")]
    if ab:
        launches = sum(v[0] for _, v in ab)
        tot_s = sum(v[1] for _, v in ab) / 1e3
        byts = abacus_unique_bytes(N, desc.L, desc.d, desc.dout, desc.w, P, Bs) * steps
        ach = byts / tot_s / 1e9
        peak = peaks["hbm_gbs"]
        out["abacus"] = {"kernel": "k_ab_layer", "bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
                         "frac": ach / peak, "traffic": traffic_per_launch("abacus", byts / launches),
                         "launches": launches,
                         "ms_per_launch": tot_s * 1e3 / launches, "peak_source": f"{src} (MEASURED_PEAKS hbm_gbs)"}
    tg = [(k, v) for k, v in prof.items() if k.endswith("links/k_tgemm")]
    if tg:
        launches = sum(v[0] for _, v in tg)
        tot_s = sum(v[1] for _, v in tg) / 1e3
        flops = link_conv_flops(N, desc.L, desc.d, Bs) * steps
        ach = flops / tot_s / 1e12
        mhz = peaks.get("sm_max_mhz", 2070.0)
        peak = SMS * FP32_LANES * 2 * mhz * 1e6 / 1e12
        out["links_tgemm"] = {"kernel": "k_tgemm", "bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                              "frac": ach / peak, "traffic": None, "launches": launches,
                              "ms_per_launch": tot_s * 1e3 / launches,
                              "peak_source": f"FP32 FMA issue rate: 152 SMs x 128 lanes x 2 flop x {mhz:.0f} MHz"}
    fused = any(k.endswith("links/k_dband") for k in prof)
    for fam_name, kname, byts in (("links_dhop", "k_dhop", dhop_bytes(N, desc.L, desc.d, Bs, fused)),
                                  ("links_bandconv", "k_bandconv",
                                   bandconv_bytes(N, desc.L, desc.d, desc.w, Bs, fused=fused)),
                                  ("links_dband", "k_dband", dband_bytes(N, desc.L, desc.d, desc.w, Bs))):
        ks = [(k, v) for k, v in prof.items() if k.endswith("links/" + kname)]
        if ks:
            launches = sum(v[0] for _, v in ks)
            tot_s = sum(v[1] for _, v in ks) / 1e3
            ach = byts * steps / tot_s / 1e9
            peak = peaks["hbm_gbs"]
            out[fam_name] = {"kernel": kname, "bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
                             "frac": ach / peak, "traffic": traffic_per_launch(fam_name, byts * steps / launches),
                             "launches": launches,
                             "ms_per_launch": tot_s * 1e3 / launches,
                             "peak_source": f"{src} (MEASURED_PEAKS hbm_gbs)"}
    gen = [(k, v) for k, v in prof.items() if k.endswith("links/k_bandconv_gen")]
    if gen:
        launches = sum(v[0] for _, v in gen)
        tot_s = sum(v[1] for _, v in gen) / 1e3
        gflops = bandconv_gen_flops(N, desc.L, desc.d, desc.w, Bs) * steps
        ach = gflops / tot_s / 1e12
        mhz = peaks.get("sm_max_mhz", 2070.0)
        peak = SMS * FP32_LANES * 2 * mhz * 1e6 / 1e12
        out["links_bandconv_gen"] = {"kernel": "k_bandconv_gen", "bound": "alu", "achieved": ach, "peak": peak,
                                     "unit": "TFLOP/s", "frac": ach / peak,
                                     "traffic": traffic_per_launch("links_bandconv_gen", gflops / launches),
                                     "launches": launches,
                                     "ms_per_launch": tot_s * 1e3 / launches,
                                     "peak_source": f"FP32 FMA issue rate: 152 SMs x 128 lanes x 2 flop x {mhz:.0f} MHz"}
    tc = [(k, v) for k, v in prof.items() if k.endswith("links/k_tgemm_tc")]
    if tc:
        launches = sum(v[0] for _, v in tc)
        tot_s = sum(v[1] for _, v in tc) / 1e3
        flops = link_conv_flops(N, desc.L, desc.d, Bs) * steps
        ach = flops / tot_s / 1e12
        # Each FP32 product is carried by three BF16 tensor-core products
        # (hi*hi + hi*lo + lo*hi), so the FP32-equivalent peak is a third of the
        # BF16 dense rate; the kernel runs inside a long step, hence the
        # sustained figure.
        bf16 = peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops"))
        peak = bf16 / 3.0
        out["links_tgemm_tc"] = {"kernel": "k_tgemm_tc", "bound": "tensor", "achieved": ach, "peak": peak,
                                 "unit": "TFLOP/s", "frac": ach / peak,
                                 "traffic": traffic_per_launch("links_tgemm_tc", flops / launches),
                                 "launches": launches,
                                 "ms_per_launch": tot_s * 1e3 / launches,
                                 "peak_source": f"{src} bf16_tflops_sustained / 3 (3-product BF16 split of FP32)"}
    return out


def roofline(prof, steps, desc, N, Bs, peaks, src, clocks):
    """Roofline of the kernel family with the largest device time in the step."""
    if not prof:
        return None, {}
    fam = kernel_rooflines(prof, steps, desc, N, Bs, peaks, src)
    name, (launches, tot_ms) = max(prof.items(), key=lambda kv: kv[1][1])
    if name.endswith("/k_ab_layer") and "abacus" in fam:
        return fam["abacus"], fam
    if name.endswith("links/k_tgemm") and "links_tgemm" in fam:
        return fam["links_tgemm"], fam
    if name.endswith("links/k_dhop") and "links_dhop" in fam:
        return fam["links_dhop"], fam
    if name.endswith("links/k_bandconv") and "links_bandconv" in fam:
        return fam["links_bandconv"], fam
    if name.endswith("links/k_dband") and "links_dband" in fam:
        return fam["links_dband"], fam
    if name.endswith("links/k_bandconv_gen") and "links_bandconv_gen" in fam:
        return fam["links_bandconv_gen"], fam
    if name.endswith("links/k_tgemm_tc") and "links_tgemm_tc" in fam:
        return fam["links_tgemm_tc"], fam
    return {"kernel": name, "bound": None, "achieved": None, "peak": None, "unit": None, "frac": None,
            "traffic": None, "ms_per_launch": tot_ms / launches}, fam


if __name__ == "__main__":
    sys.exit(main())
