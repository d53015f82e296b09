"""Benchmark: eps^-1 (q, w) blocks per second of the mixed-precision path.

One step = the whole hot path over the mid-size workload (diamond cell,
12 sp shells per atom -> N_b = 96, 8x8x8 k, N_v = 4, N_c = 32, N_t = 65536,
N_G = 181, 50 q x 200 w = 10000 blocks): per q the pair densities, the
tcgen05 chi0 with the Dyson step, the batched inverse and the loss tables;
then the |q+G| binning of both loss functions and the FP64 halo rate and
recoil spectrum.  Inputs (states) are resident in HBM before the timed
region; the per-q R planes (150 MB) and states (1.3 GB) exceed the 129 MB
L2, so no separate L2 flush is done.

Usage:  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun (N > 1) every rank processes its own 50-q shard (weak scaling);
the |q+G| bins of the loss tables are summed over the ranks by one all-reduce
(the path's only exchange) and rank 0 evaluates the rate; the timing is the
max over ranks.  Run without a launcher, --gpus N starts the N ranks itself.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# DRAM bytes (read + write) of one k_chi0_tc launch over 1 q x 200 w of the mid workload, from one ncu capture
# of `bench.py --profile-case mid200` (dram__bytes_read.sum + dram__bytes_write.sum), and the commit of the kernel
# source it was taken at; None once the kernel has changed since.
CHI0_TRAFFIC = {"bytes": 719207680 + 182851072, "commit": "1fa000c"}
# Executed FP32 flops of one k_pair_density_fused launch over 1 q of the mid workload (512 k x 181 G), from the
# ncu thread-instruction counters of `bench.py --profile-case mid` (2 FFMA + FADD + FMUL,
# smsp__sass_thread_inst_executed_op_{ffma,fadd,fmul}_pred_on.sum), and the commit of the kernel source.
PD_FP32_FLOPS = {"flops": 2 * 26974224384 + 3570466816 + 10942709760, "commit": "1fa000c"}
METRIC = "eps^-1 (q,w) blocks/s vs FP64 plain GPU path at <=1e-4 rel err; tensor-pipe %"
WORKLOAD = ("mid: diamond a=5.43 A, 12 sp shells/atom (N_b=96), 8x8x8 k, N_v=4, N_c=32 (N_t=65536), "
            "N_G=181, 50 q x 200 w on 0-60 eV, eta=0.1 eV")


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "fallback": True}


def device_uuid(local):
    """nvidia-smi's id of the CUDA device in use ("GPU-<uuid>"): nvidia-smi
    ignores CUDA_VISIBLE_DEVICES, so a CUDA ordinal may name another GPU."""
    try:
        import torch
        u = str(torch.cuda.get_device_properties(local).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms on the GPU
    given by its UUID (or index when the UUID is unknown)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        sm = [float(r[1]) for r in self.rows if len(r) > 8 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) > 8 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            if len(r) > 8:
                for i, n in enumerate(names):
                    if r[5 + i].lower().startswith("active"):
                        reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm), "gpu": str(self.device)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _barrier_max(ws, value):
    if ws == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _config(ws, precision, blocks_per_step=10000):
    """The workload both arms report (the reference arm adds its own precision)."""
    return {"workload": WORKLOAD, "blocks_per_step": blocks_per_step, "l2": "inputs larger than L2 (no flush)",
            "precision": precision, "parallelism": f"q shards x {ws}"}


def _weak_value(nq, nw, steps, ws, ms_max):
    """Whole-job blocks/s: every rank processes its own nq x nw blocks per step;
    the time is the slowest rank's."""
    return nq * nw * steps * ws / (ms_max / 1e3)


def _barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


# --------------------------------------------------------------- oracle arm
def oracle_sample(prob, Ck, Ckq0, nk_sub=128, nw_sub=4):
    """Time the CPU oracle on a bounded sample of one q: pair densities for
    nk_sub of the k points and chi0 + eps + inverse + loss for nw_sub
    frequencies over those transitions.  Returns (blocks/s extrapolated to
    the full q, seconds spent, description)."""
    from oracle import rpa
    c, b = prob.cell, prob.basis
    kap = prob.qpts[0][None, :] + prob.G_int @ c.recip
    t0 = time.perf_counter()
    rho = rpa.pair_density_lean(c.lattice, c.atoms, b.shell_atom, b.shell_l, b.shell_exp, prob.kpts[:nk_sub], kap,
                                Ck[:nk_sub], Ckq0[:nk_sub])
    t1 = time.perf_counter()
    dE = rpa.transition_energies(prob.Ek[:nk_sub], prob.Ekq[0][:nk_sub])
    ws = prob.w[np.linspace(1, len(prob.w) - 1, nw_sub).astype(int)]
    W = rpa.transition_weights(dE, ws, prob.eta)
    chi = rpa.chi0(rho, W, prob.nk, c.volume)
    eps = rpa.dielectric_matrix(chi, rpa.coulomb_sqrt(prob.qpts[0], prob.G_int @ c.recip))
    rpa.loss_functions(eps)
    t2 = time.perf_counter()
    scale = prob.nk / nk_sub
    per_block = (t1 - t0) * scale / len(prob.w) + (t2 - t1) * scale / nw_sub
    desc = (f"1 q of the mid workload: pair densities for {nk_sub}/{prob.nk} k points and chi0+eps+inverse+loss "
            f"for {nw_sub}/{len(prob.w)} w over those transitions; time scaled linearly in k to all "
            f"{prob.nk} k, pair densities amortised over {len(prob.w)} w")
    return 1.0 / per_block, t2 - t0, desc


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count()


def run_reference(args, ws, rank):
    """Reference arm: the CPU oracle (the only implementation the paper gives
    a definition for), timed on the host cores."""
    if rank != 0:
        return
    import synth
    from oracle import rpa
    prob = synth.make_mid(nq=1)
    Ck = rpa.orthonormalise(rpa.overlap(prob.cell.lattice, prob.cell.atoms, prob.basis.shell_atom,
                                        prob.basis.shell_l, prob.basis.shell_exp, prob.kpts[:128]), prob.Zk[:128])
    kq = prob.kpts[:128] + prob.qpts[0][None, :]
    Ckq = rpa.orthonormalise(rpa.overlap(prob.cell.lattice, prob.cell.atoms, prob.basis.shell_atom,
                                         prob.basis.shell_l, prob.basis.shell_exp, kq), prob.zkq(0)[:128])
    vals = []
    for i in range(args.warmup + args.steps):
        v, _, desc = oracle_sample(prob, Ck, Ckq)
        if i >= args.warmup:
            vals.append(v)
    v = float(np.median(vals))
    out = {"metric": METRIC, "value": v, "unit": "blocks/s", "impl": "reference", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * 10000 / v / 1.0,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic",
           "config": _config(1, "the FP64 oracle (plain numpy, complex128) on a bounded sample of the workload"),
           "cpu_baseline": {"value": v, "unit": "blocks/s", "cores": cpu_cores(), "kind": "oracle", "sample": desc},
           "e2e": {"value": v, "unit": "blocks/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ----------------------------------------------------------------- our arm
def run_ours(args, ws, rank, local):
    import torch

    import synth
    from paper_2603_12326_gb300 import QCX_FP64, QCX_MIXED, qcx, shards, states
    from paper_2603_12326_gb300.build import build

    build()
    torch.cuda.set_device(local)
    stream = torch.cuda.Stream()
    ctx = qcx.Context(local, stream=stream.cuda_stream)
    prob = synth.make_mid()
    if ws > 1:   # weak scaling: each rank a different 50-q shard of the same distribution
        prob = synth.make_mid_shard(rank)
    nq, nw, ng = prob.nq, len(prob.w), prob.ng
    Ck, Ckq = states.load_problem(ctx, prob)
    G = prob.G_int
    w = prob.w
    eta = prob.eta
    edges = np.linspace(0.0, 12.0, 121)          # |q+G| bins, bohr^-1
    halo = qcx.halo_params()
    nt = prob.nt
    pref_flops = 8.0 * nt * ng * ng * nw          # algorithmic chi0 flops per q (one launch)

    chi_events = []
    pd_events = []
    # algorithmic bytes of one pair-density launch: the FP32 coefficients read once, the three BF16 planes of
    # rho written once
    pd_bytes = 8.0 * prob.nk * prob.basis.nbasis * (prob.nv + prob.nc) + 12.0 * nt * ng

    def step(record=False):
        for iq in range(nq):
            if record:
                p0 = torch.cuda.Event(enable_timing=True)
                p1 = torch.cuda.Event(enable_timing=True)
                p0.record(stream)
            ctx.pair_density(iq, G, QCX_MIXED)
            if record:
                p1.record(stream)
                pd_events.append((p0, p1))
            if record:
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
            ctx.chi0(iq, w, eta, QCX_MIXED)
            if record:
                e1.record(stream)
                chi_events.append((e0, e1))
            ctx.invert_eps(iq, QCX_MIXED, want=False)
        Lb, cnt = ctx.bin_loss(list(range(nq)), 0, edges, nw)
        Lb2, cnt2 = ctx.bin_loss(list(range(nq)), 1, edges, nw)
        if ws > 1:
            # the one exchange of the path: the |q+G| bins of every rank's q, summed over the ranks
            Lb, cnt = shards.combine_bins(Lb, cnt, device=f"cuda:{local}")
            Lb2, _ = shards.combine_bins(Lb2, cnt2, device=f"cuda:{local}")
            if rank != 0:
                return None, None
        nz = cnt > 0
        qb = 0.5 * (edges[1:] + edges[:-1])[nz]
        dR, dQ = ctx.rate(qb, w, Lb[nz], halo, nQ=10)
        dR2, dQ2 = ctx.rate(qb, w, Lb2[nz], halo, nQ=10)
        return dQ, dQ2

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    sampler = ClockSampler(device_uuid(local) or local)
    sampler.start()
    _barrier(ws)
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        step(record=True)
    ev1.record(stream)
    torch.cuda.synchronize()
    _barrier(ws)
    clocks = sampler.stop()
    ms = ev0.elapsed_time(ev1)
    ms = _barrier_max(ws, ms)
    value = _weak_value(nq, nw, args.steps, ws, ms)
    chi_ms = [a.elapsed_time(b) for a, b in chi_events]
    chi_avg = float(np.mean(chi_ms))
    pd_avg = float(np.mean([a.elapsed_time(b) for a, b in pd_events]))
    peaks = _peaks()
    achieved = pref_flops / (chi_avg / 1e3) / 1e12
    peak = peaks.get("bf16_tflops_sustained", 1700.0)

    # ------------------------------------------------------ end to end (host buffers)
    import ctypes as ct
    pin = {}
    for name, arr in (("kpts", prob.kpts), ("Ck", Ck), ("Ek", prob.Ek), ("qpts", prob.qpts), ("Ckq", Ckq),
                      ("Ekq", prob.Ekq)):
        t = torch.from_numpy(np.ascontiguousarray(arr)).pin_memory()
        pin[name] = t
    outL = torch.empty((nq, 2, nw, ng), dtype=torch.float64).pin_memory()
    # each q's loss tables go to device memory (no per-q synchronisation: a host destination makes the
    # library wait for the stream) and all q come back to the pinned host buffer in one copy per step
    outL_dev = torch.empty((nq, 2, nw, ng), dtype=torch.float64, device=f"cuda:{local}")
    h2d = sum(t.numel() * t.element_size() for t in pin.values())
    d2h = outL.numel() * outL.element_size() + 2 * 10 * 8

    def e2e_step():
        st = qcx.qcx_set_states(ctx.h, prob.nk, qcx.P(pin["kpts"].data_ptr()), prob.nv, qcx.P(pin["Ck"].data_ptr()),
                                qcx.P(pin["Ek"].data_ptr()), nq, qcx.P(pin["qpts"].data_ptr()), prob.nc,
                                qcx.P(pin["Ckq"].data_ptr()), qcx.P(pin["Ekq"].data_ptr()))
        ctx._check(st)
        for iq in range(nq):
            ctx.pair_density(iq, G, QCX_MIXED)
            ctx.chi0(iq, w, eta, QCX_MIXED)
            ctx.invert_eps(iq, QCX_MIXED, want=False)
            ctx.loss_function(iq, QCX_MIXED, out_lfe=outL_dev[iq, 0], out_nolfe=outL_dev[iq, 1])
        with torch.cuda.stream(stream):
            outL.copy_(outL_dev, non_blocking=True)
        Lb, cnt = ctx.bin_loss(list(range(nq)), 0, edges, nw)
        if ws > 1:
            Lb, cnt = shards.combine_bins(Lb, cnt, device=f"cuda:{local}")
            if rank != 0:
                return
        nz = cnt > 0
        ctx.rate(0.5 * (edges[1:] + edges[:-1])[nz], w, Lb[nz], halo, nQ=10)

    e2e_step()
    torch.cuda.synchronize()
    _barrier(ws)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    n_e2e = max(1, min(args.steps, 2))
    for _ in range(n_e2e):
        e2e_step()
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = _barrier_max(ws, e0.elapsed_time(e1) / n_e2e)

    # ------------------------------------------ rate end on the mixed tables of every q (rank 0)
    rate_end = rate_end_leg(ctx, prob, w) if rank == 0 and ws == 1 else None

    # ------------------------------------ accuracy over every q: mixed vs the FP64 GPU path
    # The e2e step left the mixed loss tables of all q in the context; each q is then recomputed by the
    # FP64 path (pinned to the oracle at 1e-10) at eight frequencies.
    accuracy = accuracy_sweep(ctx, prob, G, w, eta, outL) if not args.no_sweep else None

    # -------------------------------------------------- FP64 plain GPU path (sample)
    nw64 = 40
    w64 = w[np.linspace(1, nw - 1, nw64).astype(int)]
    ctx.pair_density(0, G, QCX_FP64)
    ctx.chi0(0, w64, eta, QCX_FP64)
    ctx.invert_eps(0, QCX_FP64, want=False)
    torch.cuda.synchronize()
    t = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    t[0].record(stream)
    ctx.pair_density(0, G, QCX_FP64)
    t[1].record(stream)
    ctx.chi0(0, w64, eta, QCX_FP64)
    t[2].record(stream)
    ctx.invert_eps(0, QCX_FP64, want=False)
    t[3].record(stream)
    torch.cuda.synchronize()
    per_block64 = (t[0].elapsed_time(t[1]) / nw + t[1].elapsed_time(t[3]) / nw64) / 1e3
    fp64_value = 1.0 / per_block64
    chi64_ms = t[1].elapsed_time(t[2])
    chi64_tflops = 8.0 * nt * ng * ng * nw64 / (chi64_ms / 1e3) / 1e12
    fma = fma_peaks(local)

    # ------------------------------------ spectral route (binned spectral function + Kramers-Kronig)
    spec = spectral_leg(ctx, prob, G, w, eta, stream, fma) if (rank == 0 and ws == 1 and not args.no_spectral) else None
    optic = optical_leg(stream) if (rank == 0 and ws == 1 and not args.no_spectral) else None

    # ------------------------------------------- batched uneven instances (rank 0, N=1)
    batched = batched_leg(stream) if (rank == 0 and ws == 1) else None
    large = large_leg(stream) if (rank == 0 and ws == 1 and not args.no_large) else None
    surro = surrogate_leg(stream) if (rank == 0 and ws == 1 and not args.no_surrogate) else None

    # -------------------------------------------------------- CPU oracle (rank 0, N=1)
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        v, secs, desc = oracle_sample(prob, Ck, Ckq[0])
        cpu = {"value": v, "unit": "blocks/s", "cores": cpu_cores(), "kind": "oracle", "sample": desc,
               "seconds": round(secs, 2)}

    if rank == 0:
        # per q: G setup, the two pair-density tables, pair densities, W table, chi0, chi0 diagonal without
        # cancellation (two kernels), Gauss-Jordan, FP64 diagonal correction, loss by the quadratic form, |q+G|,
        # the dielectric values kept for 3-D binning; per step two binnings and two rate + recoil pairs
        launches_per_step = nq * 13 + 2 + 4
        out = {"metric": METRIC, "value": value, "unit": "blocks/s", "n_gpus": ws, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
               "vs_baseline": None, "dtype": "bf16",
               "data": "synthetic (seeded states shaped like the paper's workloads)",
               "config": _config(ws, "chi0 as split-BF16 tcgen05 products: rho~ (two BF16 terms of the FP32 "
                                     "pair densities) against W rho~ in three terms, five products, FP32 "
                                     "accumulation restarted every 20 MMAs and FP64 partial sums, diagonal summed "
                                     "again in FP32; inverse FP32 + FP64 diagonal correction; rate FP64", nq * nw),
               "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                            "frac": achieved / peak,
                            "traffic": CHI0_TRAFFIC["bytes"] if CHI0_TRAFFIC else None,
                            "traffic_source": (f"ncu dram__bytes_read.sum + dram__bytes_write.sum of one k_chi0_tc "
                                               f"launch of 1 q x 200 w at commit {CHI0_TRAFFIC['commit']}"
                                               if CHI0_TRAFFIC else "not retaken since the kernel changed"),
                            "kernel": "k_chi0_tc", "flops_per_launch": pref_flops,
                            "avg_launch_ms": chi_avg,
                            "peak_source": "bf16_tflops_sustained of measured (MEASURED_PEAKS.json)"},
               "pair_density": {"kernel": "k_pair_density_fused", "avg_launch_ms": pd_avg, "bound": "alu",
                                "fp32_flops_per_launch": PD_FP32_FLOPS["flops"] if PD_FP32_FLOPS else None,
                                "fp32_flops_source": (f"ncu FFMA/FADD/FMUL thread-instruction counts of one launch "
                                                      f"(1 q), kernel at commit {PD_FP32_FLOPS['commit']}"
                                                      if PD_FP32_FLOPS else "not recounted since the kernel changed"),
                                "achieved_tflops": (PD_FP32_FLOPS["flops"] / (pd_avg / 1e3) / 1e12
                                                    if PD_FP32_FLOPS else None),
                                "fp32_peak_tflops": fma.get("fp32_tflops"),
                                "frac": (PD_FP32_FLOPS["flops"] / (pd_avg / 1e3) / 1e12 / fma["fp32_tflops"]
                                         if fma.get("fp32_tflops") and PD_FP32_FLOPS else None),
                                "peak_source": "FFMA microbenchmark measured in this run (libqcx_peaks)",
                                "algorithmic_bytes": pd_bytes, "achieved_GBs": pd_bytes / (pd_avg / 1e3) / 1e9,
                                "hbm_peak_GBs": peaks.get("hbm_gbs", 6800.0),
                                "hbm_frac": pd_bytes / (pd_avg / 1e3) / 1e9 / peaks.get("hbm_gbs", 6800.0),
                                "note": "FP32 block assembly and contractions with the coefficients bound it, not HBM"},
               "e2e": {"value": nq * nw * ws / (e2e_ms / 1e3), "unit": "blocks/s", "h2d_bytes_per_step": h2d,
                       "d2h_bytes_per_step": d2h},
               "fp64_gpu": {"value": fp64_value, "unit": "blocks/s",
                            "sample": f"1 q: FP64 pair densities amortised over {nw} w + FP64 chi0/inverse "
                                      f"for {nw64} w",
                            "chi0_kernel": "k_chi0_fp64", "chi0_ms": chi64_ms, "chi0_tflops": chi64_tflops,
                            "fp64_peak_tflops": fma.get("fp64_tflops"),
                            "chi0_frac_of_fp64_peak": (chi64_tflops / fma["fp64_tflops"]
                                                       if fma.get("fp64_tflops") else None),
                            "peak_source": "DFMA microbenchmark measured in this run (libqcx_peaks)"},
               "fma_peaks": fma,
               "speedup_vs_fp64_gpu": value / fp64_value,
               "gpu_launches": launches_per_step * args.steps,
               "clocks": clocks}
        if accuracy:
            out["accuracy"] = accuracy
        if rate_end:
            out["rate_end"] = rate_end
        if spec:
            out["spectral"] = spec
        if optic:
            out["optical_limit"] = optic
        if cpu:
            out["cpu_baseline"] = cpu
        if batched:
            out["batched"] = batched
        if large:
            out["large"] = large
        if surro:
            out["surrogate"] = surro
        print(json.dumps(out), flush=True)
    ctx.close()


def rate_end_leg(ctx, prob, w, q_lfe=8.0, dq=0.02, nth=9, nph=16, nshell=640):
    """The composite function of the timed workload's 50 q (mixed tables, 200 w)
    in the paper's 3-D bins (dq = 0.02 alpha m_e, 9 x 16 angular cells, q_LFE = 8
    alpha m_e), filled, reduced to the isotropic loss under four screening
    choices, and the general rate of the halo flux (vector and scalar heavy
    mediators) with recoil spectrum and reach; wall-clock times of the calls
    (host outputs, so copies included)."""
    import synth
    from paper_2603_12326_gb300 import qcx
    nq, nw = prob.nq, len(w)
    t = {}
    t0 = time.perf_counter()
    eps, cnt = ctx.bin_eps3d(list(range(nq)), q_lfe, nshell, dq, nth, nph, nw, fill=True)
    t["bin_eps3d_ms"] = 1e3 * (time.perf_counter() - t0)
    ne = 8.0 / prob.cell.volume
    L = {}
    for name, model in (("self", qcx.SCREEN_SELF), ("none", qcx.SCREEN_NONE), ("mtf", qcx.SCREEN_MTF),
                        ("lindhard", qcx.SCREEN_LINDHARD)):
        t0 = time.perf_counter()
        L[name], ncell = ctx.loss_isotropic(eps, cnt, w, dq, qcx.screening(model, ne_bohr3=ne, fp=0.1))
        t[f"loss_isotropic_{name}_ms"] = 1e3 * (time.perf_counter() - t0)
    used = ncell > 0
    qs = (np.arange(nshell) + 0.5)[used] * dq
    v = np.linspace(1e-6, 3e-3, 2000)
    flux = synth.halo_flux(v)
    rates = {}
    for name, kind in (("vector", 0), ("scalar", 1)):
        t0 = time.perf_counter()
        dR, dQ, reach = ctx.rate_general(qs, w, L["self"][used], v, flux, qcx.rate_params(mediator=kind), nQ=10,
                                         want_reach=True)
        t[f"rate_general_{name}_ms"] = 1e3 * (time.perf_counter() - t0)
        rates[name] = {"recoil_spectrum_events_per_kg_yr": [float(x) for x in dQ],
                       "reach_cm2_1kg_yr": [float(x) for x in reach]}
    return {"bins": {"shells": nshell, "dq_bohr": dq, "n_theta": nth, "n_phi": nph, "q_lfe_bohr": q_lfe,
                     "filled": int(np.sum(cnt > 0)), "interpolated": int(np.sum(cnt < 0)),
                     "shells_used": int(used.sum())},
            "times": t, "rates": rates,
            "flux": "standard halo, m_chi = 1 GeV, 2000 speeds to 3e-3 c"}


def fma_peaks(device):
    """Measured FP64 (DFMA) and FP32 (FFMA) peaks of the CUDA cores."""
    import ctypes as ct
    from paper_2603_12326_gb300 import build as b
    try:
        lib = ct.CDLL(b.PEAKS_LIB)
    except OSError:
        return {}
    f = lib.qcx_peak_fma
    f.restype = ct.c_int
    f.argtypes = [ct.c_int, ct.c_int, ct.c_int, ct.c_int, ct.c_int, ct.POINTER(ct.c_double), ct.POINTER(ct.c_double)]
    out = {}
    for name, fp64, iters in (("fp64", 1, 6000), ("fp32", 0, 200000)):
        tf, ms = ct.c_double(), ct.c_double()
        if f(device, fp64, 4, iters, 5, ct.byref(tf), ct.byref(ms)) == 0:
            out[f"{name}_tflops"] = tf.value
            out[f"{name}_ms"] = ms.value
    out["method"] = ("8 independent FMA chains per thread, 4 CTAs of 256 threads per SM, best of 5 launches "
                     "timed with CUDA events")
    return out


def _masked_err(a, b, frac=1e-3):
    """Worst relative error of a against b per spectrum (fixed G, column of [w][G]) where
    |b| exceeds frac of the spectrum's maximum."""
    top = np.max(np.abs(b), axis=0, keepdims=True)
    m = np.abs(b) > frac * top
    return float(np.max(np.abs(a[m] - b[m]) / np.abs(b[m])))


def spectral_leg(ctx, prob, G, w, eta, stream, fma, nq_spec=10, frac=20, nsample=8):
    """The spectral route to chi0 (spectral function on a uniform energy grid of
    step eta/frac, principal part by the Kramers-Kronig relations) on the first
    nq_spec q of the timed workload, all 200 w: the mixed route timed per q with
    CUDA events (pair densities, chi0, inverse), its contraction kernel's FP32
    roofline from the stage times the library records, the FP64 route on q 0,
    and the loss of both routes against the FP64 direct sum at nsample
    frequencies of q 0 (the route's discretisation in energy, second order in
    the step)."""
    import torch
    from paper_2603_12326_gb300 import QCX_FP64, QCX_MIXED
    nw, ng = len(w), prob.ng
    step = eta / frac
    grids = [ctx.spectral_grid(iq, step) for iq in range(nq_spec)]
    ctx.pair_density(0, G, QCX_MIXED)                         # warm-up
    ctx.chi0_spectral(0, w, eta, grids[0][0], step, grids[0][1], QCX_MIXED)
    ctx.invert_eps(0, QCX_MIXED, want=False)
    torch.cuda.synchronize()
    kk_ms, wt_ms, flops = [], [], 0.0
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for iq in range(nq_spec):
        E0, nbin = grids[iq]
        ctx.pair_density(iq, G, QCX_MIXED)
        ctx.chi0_spectral(iq, w, eta, E0, step, nbin, QCX_MIXED)
        tm = ctx.spectral_timings()
        kk_ms.append(tm["contraction"])
        wt_ms.append(tm["weights"])
        flops += 4.0 * nw * nbin * ng * (ng + 1)             # 4 FMA per (w, grid point, G <= G') pair
        ctx.invert_eps(iq, QCX_MIXED, want=False)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    # q 0 again for its tables (the loop ended on the last q); then the same contraction on the
    # CUDA cores in FP32 for comparison
    ctx.pair_density(0, G, QCX_MIXED)
    ctx.chi0_spectral(0, w, eta, grids[0][0], step, grids[0][1], QCX_MIXED)
    ctx.invert_eps(0, QCX_MIXED, want=False)
    Lm = ctx.loss_function(0, QCX_MIXED)
    ctx.set_spectral_engine(True)
    ctx.chi0_spectral(0, w, eta, grids[0][0], step, grids[0][1], QCX_MIXED)
    cc_ms = ctx.spectral_timings()["contraction"]
    ctx.set_spectral_engine(False)
    # FP64 route, q 0
    ctx.pair_density(0, G, QCX_FP64)
    torch.cuda.synchronize()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    ctx.chi0_spectral(0, w, eta, grids[0][0], step, grids[0][1], QCX_FP64)
    ctx.invert_eps(0, QCX_FP64, want=False)
    f1.record(stream)
    torch.cuda.synchronize()
    ms64 = f0.elapsed_time(f1)
    tm64 = ctx.spectral_timings()
    L64 = ctx.loss_function(0, QCX_FP64)
    # the direct sum in FP64 at nsample frequencies of q 0
    sample = np.linspace(1, nw - 1, nsample).astype(int)
    ctx.chi0(0, w[sample], eta, QCX_FP64)
    ctx.invert_eps(0, QCX_FP64, want=False)
    Ld = ctx.loss_function(0, QCX_FP64)
    kk = float(np.sum(kk_ms))
    achieved = flops / (kk / 1e3) / 1e12
    flops64 = 4.0 * nw * grids[0][1] * ng * (ng + 1)
    ach64 = flops64 / (tm64["contraction"] / 1e3) / 1e12
    return {"workload": f"first {nq_spec} q of the timed workload x {nw} w, grid step eta/{frac} "
                        f"({grids[0][1]} points at q 0)",
            "value": nq_spec * nw / (ms / 1e3), "unit": "blocks/s",
            "ms_per_q": ms / nq_spec,
            "precision": "FP32 pair densities and weights; contraction on tcgen05 in three-term split BF16 "
                         "(FP32 sums restarted every 24 MMAs, chunks added in FP64); grid and K in FP64; inverse as "
                         "the mixed direct path",
            "contraction": {"kernel": "k_spec_kk_tc (with the K-major split of the weights, k_spec_s_split)",
                            "bound": "tensor", "ms_per_q": kk / nq_spec,
                            "weights_ms_per_q": float(np.sum(wt_ms)) / nq_spec,
                            "flops": "4 FMA per (w, grid point, G <= G') pair",
                            "achieved_tflops": achieved,
                            "peak_tflops": _peaks().get("bf16_tflops_sustained"),
                            "frac": achieved / _peaks().get("bf16_tflops_sustained", 1700.0),
                            "peak_source": "bf16_tflops_sustained of measured (MEASURED_PEAKS.json)",
                            "cuda_cores_fp32": {"kernel": "k_spec_kk<float>", "ms_q0": cc_ms,
                                                "achieved_tflops": 4.0 * nw * grids[0][1] * ng * (ng + 1) / (cc_ms / 1e3)
                                                / 1e12,
                                                "fp32_peak_tflops": fma.get("fp32_tflops")}},
            "fp64": {"value": nw / (ms64 / 1e3), "unit": "blocks/s", "sample": "q 0 (chi0 + inverse; pair "
                     "densities excluded)", "contraction_ms": tm64["contraction"], "weights_ms": tm64["weights"],
                     "contraction_tflops": ach64,
                     "frac_of_fp64_peak": ach64 / fma["fp64_tflops"] if fma.get("fp64_tflops") else None},
            "vs_direct_sum": {"mixed_L_lfe": _masked_err(Lm[0][sample], Ld[0]),
                              "mixed_L_nolfe": _masked_err(Lm[1][sample], Ld[1]),
                              "fp64_L_lfe": _masked_err(L64[0][sample], Ld[0]),
                              "fp64_L_nolfe": _masked_err(L64[1][sample], Ld[1]),
                              "mixed_vs_fp64_route_L_lfe": _masked_err(Lm[0], L64[0]),
                              "sample": f"q 0, {nsample} w, every G; per spectrum where L > 1e-3 of its maximum "
                                        f"over the sampled w"}}


def optical_leg(stream):
    """The optical limit q -> 0 on the mid workload's cell, basis, k grid and G set
    (a single q = 0 with conduction states at k, orthonormal together with the
    valence states): for the three Cartesian directions, the pair densities with
    the G = 0 row from the momentum matrix elements, chi0 over 200 w, inverse and
    losses on the mixed path, timed with CUDA events; the head's loss peak."""
    import torch

    import synth
    from paper_2603_12326_gb300 import QCX_MIXED, qcx, states

    ctx = qcx.Context(torch.cuda.current_device(), stream=stream.cuda_stream)
    p = synth.make_optical("mid")
    states.load_optical(ctx, p)
    G, w = p.G_int, p.w
    g0 = int(np.flatnonzero(np.all(G == 0, axis=1))[0])
    ctx.pair_density_optical(0, G, [1.0, 0.0, 0.0], QCX_MIXED)       # warm-up (momentum matrix, buffers)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    heads = {}
    e0.record(stream)
    for name, d in (("x", [1.0, 0.0, 0.0]), ("y", [0.0, 1.0, 0.0]), ("z", [0.0, 0.0, 1.0])):
        ctx.pair_density_optical(0, G, d, QCX_MIXED)
        ctx.chi0(0, w, p.eta, QCX_MIXED)
        ctx.invert_eps(0, QCX_MIXED, want=False)
        L1, L2 = ctx.loss_function(0, QCX_MIXED)
        heads[name] = (L1[:, g0], L2[:, g0])
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    ctx.close()
    wev = w * 27.211386245988
    out = {"workload": "mid workload's cell, basis, 8x8x8 k, N_v=4, N_c=32, N_G=181, q -> 0 along x, y, z, 200 w",
           "value": 3 * len(w) / (ms / 1e3), "unit": "blocks/s", "ms_per_direction": ms / 3}
    for name, (a, b) in heads.items():
        out[f"head_{name}"] = {"L_lfe_peak_eV": float(wev[int(np.argmax(a))]), "L_lfe_max": float(np.max(a)),
                               "L_nolfe_peak_eV": float(wev[int(np.argmax(b))]), "L_nolfe_max": float(np.max(b))}
    return out


def accuracy_sweep(ctx, prob, G, w, eta, outL, nsample=8):
    """Worst relative error of the mixed loss tables (outL[q][0|1][w][G], all
    200 w) against the FP64 GPU path at nsample frequencies of every q, per
    spectrum where L > 1e-3 of its maximum over all frequencies."""
    from paper_2603_12326_gb300 import QCX_FP64
    sample = np.linspace(1, len(w) - 1, nsample).astype(int)
    worst = [0.0, 0.0]
    for iq in range(prob.nq):
        ctx.pair_density(iq, G, QCX_FP64)
        ctx.chi0(iq, w[sample], eta, QCX_FP64)
        ctx.invert_eps(iq, QCX_FP64, want=False)
        d = ctx.loss_function(iq, QCX_FP64)
        for j in range(2):
            m = outL[iq, j].numpy()
            top = np.max(np.abs(m), axis=0, keepdims=True)
            mask = np.abs(d[j]) > 1e-3 * top
            worst[j] = max(worst[j], float(np.max(np.abs(m[sample][mask] - d[j][mask]) / np.abs(d[j][mask]))))
    return {"L_lfe_max_rel_err": worst[0], "L_nolfe_max_rel_err": worst[1], "bar": 1e-4,
            "vs": "FP64 GPU path (held to 1e-10 of the oracle)",
            "sample": f"all {prob.nq} q x {nsample} w of the timed workload, every G; per spectrum where "
                      f"L > 1e-3 of its maximum over the {len(w)} w"}


def large_leg(stream, nq=2, nk_oracle=8):
    """The large all-electron workload (18 sp shells per atom up to 5000 bohr^-2,
    12^3 k, N_v = 14, N_c = 64: N_t = 1 548 288, N_G = 531, 400 w on 0-100 eV,
    eta = 0.05 eV) through the mixed path for its first nq q (every q costs the
    same): blocks/s over the per-q path (pair densities, chi0 with the Dyson
    step, inverse and loss tables), the chi0 launch's algorithmic rate against
    the sustained peak, the FP64 recoil spectrum of those q, and the oracle on
    a bounded sample (nk_oracle of the 1728 k points, 1 q x 4 w)."""
    import torch

    import synth
    from paper_2603_12326_gb300 import QCX_MIXED, qcx, states

    ctx = qcx.Context(torch.cuda.current_device(), stream=stream.cuda_stream)
    p = synth.make_large(nq=nq)
    Ck, Ckq = states.load_problem(ctx, p)
    G, w = p.G_int, p.w
    ng, nw, nt = p.ng, len(w), p.nt
    ctx.pair_density(0, G, QCX_MIXED)                      # warm-up (kernel attributes, buffers)
    ctx.chi0(0, w[:8], p.eta, QCX_MIXED)
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * nq + 2)]
    chi = []
    ev[0].record(stream)
    for iq in range(nq):
        ctx.pair_density(iq, G, QCX_MIXED)
        c0 = torch.cuda.Event(enable_timing=True)
        c1 = torch.cuda.Event(enable_timing=True)
        c0.record(stream)
        ctx.chi0(iq, w, p.eta, QCX_MIXED)
        c1.record(stream)
        chi.append((c0, c1))
        ctx.invert_eps(iq, QCX_MIXED, want=False)
    ev[1].record(stream)
    torch.cuda.synchronize()
    ms = ev[0].elapsed_time(ev[1])
    chi_ms = float(np.mean([a.elapsed_time(b) for a, b in chi]))
    flops = 8.0 * nt * ng * ng * nw
    peak = _peaks().get("bf16_tflops_sustained", 1700.0)
    edges = np.linspace(0.0, 16.0, 161)
    halo = qcx.halo_params()
    Lb, cnt = ctx.bin_loss(list(range(nq)), 0, edges, nw)
    nz = cnt > 0
    dR, dQ = ctx.rate(0.5 * (edges[1:] + edges[:-1])[nz], w, Lb[nz], halo, nQ=10)
    L1, L2 = ctx.loss_function(0, QCX_MIXED)
    spec = _large_spectral(ctx, p, G, w, nq, stream, L1, L2)
    ctx.close()
    # the oracle on a bounded sample of the same workload
    from oracle import rpa
    c, b = p.cell, p.basis
    kap = p.qpts[0][None, :] + G @ c.recip
    ws_ = w[np.linspace(1, nw - 1, 4).astype(int)]
    t0 = time.perf_counter()
    rho = rpa.pair_density_lean(c.lattice, c.atoms, b.shell_atom, b.shell_l, b.shell_exp, p.kpts[:nk_oracle], kap,
                                Ck[:nk_oracle], Ckq[0][:nk_oracle])
    t1 = time.perf_counter()
    W = rpa.transition_weights(rpa.transition_energies(p.Ek[:nk_oracle], p.Ekq[0][:nk_oracle]), ws_, p.eta)
    eps = rpa.dielectric_matrix(rpa.chi0(rho, W, p.nk, c.volume), rpa.coulomb_sqrt(p.qpts[0], G @ c.recip))
    rpa.loss_functions(eps)
    t2 = time.perf_counter()
    scale = p.nk / nk_oracle
    per_block = (t1 - t0) * scale / nw + (t2 - t1) * scale / len(ws_)
    return {"workload": "large: diamond a=5.43 A, 18 sp shells/atom up to 5000 bohr^-2 (N_b=144), 12x12x12 k, "
                        "N_v=14, N_c=64 (N_t=1548288), N_G=531, 400 w on 0-100 eV, eta=0.05 eV",
            "q_timed": nq, "value": nq * nw / (ms / 1e3), "unit": "blocks/s", "ms_per_q": ms / nq,
            "chi0": {"kernel": "k_chi0_tc", "avg_launch_ms": chi_ms, "flops_per_launch": flops,
                     "achieved_tflops": flops / (chi_ms / 1e3) / 1e12, "peak": peak,
                     "frac": flops / (chi_ms / 1e3) / 1e12 / peak,
                     "peak_source": "bf16_tflops_sustained of measured (MEASURED_PEAKS.json)"},
            "recoil_spectrum_events_per_kg_yr": [float(x) for x in dQ],
            "recoil_spectrum_note": f"FP64 rate over the |q+G| bins of the {nq} timed q (heavy mediator, "
                                    f"m_chi = 1 GeV)",
            "loss_table_finite": bool(np.all(np.isfinite(L1))),
            "spectral": spec,
            "cpu_baseline": {"value": 1.0 / per_block, "unit": "blocks/s", "cores": cpu_cores(), "kind": "oracle",
                             "sample": f"1 q: pair densities for {nk_oracle}/{p.nk} k and chi0+eps+inverse+loss for "
                                       f"4/{nw} w over those transitions, scaled linearly in k",
                             "seconds": round(t2 - t0, 2)}}


def _large_spectral(ctx, p, G, w, nq, stream, L1, L2, frac=40):
    """The spectral route on the same q of the large workload (grid step eta/frac):
    blocks/s over the per-q path with chi0 from the spectral function, the FP32
    contraction's rate, and the loss of q 0 against the direct route's (L1, L2)
    over all frequencies."""
    import torch
    from paper_2603_12326_gb300 import QCX_MIXED
    nw, ng = len(w), p.ng
    step = p.eta / frac
    grids = [ctx.spectral_grid(iq, step) for iq in range(nq)]
    ctx.pair_density(0, G, QCX_MIXED)                      # warm-up (buffers)
    ctx.chi0_spectral(0, w, p.eta, grids[0][0], step, grids[0][1], QCX_MIXED)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    kk, wt, flops = 0.0, 0.0, 0.0
    e0.record(stream)
    for iq in range(nq):
        E0, nbin = grids[iq]
        ctx.pair_density(iq, G, QCX_MIXED)
        ctx.chi0_spectral(iq, w, p.eta, E0, step, nbin, QCX_MIXED)
        tm = ctx.spectral_timings()
        kk += tm["contraction"]
        wt += tm["weights"]
        flops += 4.0 * nw * nbin * ng * (ng + 1)
        ctx.invert_eps(iq, QCX_MIXED, want=False)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    S1, S2 = ctx.loss_function(0, QCX_MIXED)
    # reference for both mixed routes over all frequencies: the FP64 spectral route of q 0 (its
    # discretisation against the FP64 direct sum is far below the bar at this step)
    from paper_2603_12326_gb300 import QCX_FP64
    ctx.pair_density(0, G, QCX_FP64)
    ctx.chi0_spectral(0, w, p.eta, grids[0][0], step, grids[0][1], QCX_FP64)
    ctx.invert_eps(0, QCX_FP64, want=False)
    F1, F2 = ctx.loss_function(0, QCX_FP64)
    return {"grid": f"step eta/{frac}, {grids[0][1]} points at q 0", "value": nq * nw / (ms / 1e3),
            "unit": "blocks/s", "ms_per_q": ms / nq,
            "contraction": {"kernel": "k_spec_kk_tc", "ms_per_q": kk / nq,
                            "achieved_tflops": flops / (kk / 1e3) / 1e12},
            "weights_ms_per_q": wt / nq,
            "vs_fp64_spectral_route": {"spectral_mixed_L_lfe": _masked_err(S1, F1),
                                       "spectral_mixed_L_nolfe": _masked_err(S2, F2),
                                       "direct_mixed_L_lfe": _masked_err(L1, F1),
                                       "direct_mixed_L_nolfe": _masked_err(L2, F2),
                                       "sample": "q 0, all 400 w, every G; per spectrum where L > 1e-3 of its "
                                                 "maximum"}}


def batched_leg(stream, reps=10):
    """The uneven workload (256 (q, w) instances, N_G 19-339, one call =
    one captured-graph replay) through qcx_solve_batch, mixed and FP64."""
    import torch

    import synth
    from paper_2603_12326_gb300 import QCX_FP64, QCX_MIXED, qcx, states

    ctx = qcx.Context(torch.cuda.current_device(), stream=stream.cuda_stream)
    p = synth.make_uneven()
    states.load_problem(ctx, p)
    e = p.extra
    q, w, g = e["inst_q"], e["inst_w"], e["inst_gmax"]
    n = len(q)
    flops = 8.0 * p.nk * p.nv * p.nc * float((e["inst_ng"].astype(float) ** 2).sum())
    res = {}
    for name, prec, k in (("mixed", QCX_MIXED, reps), ("fp64", QCX_FP64, 2)):
        ctx.solve_batch(q, w, g, p.eta, prec)          # plan, autotune, capture
        for _ in range(3):
            ctx.solve_batch(q, w, g, p.eta, prec)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(k):
            ctx.solve_batch(q, w, g, p.eta, prec)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / k
        res[name] = (ms, ctx.batch_info())
    ctx.close()
    ms, info = res["mixed"]
    ms64, info64 = res["fp64"]
    return {"workload": "uneven: 256 (q,w) instances on the small workload's states (8 sp shells/atom, 4x4x4 k, "
                        "N_v=4, N_c=12, N_t=3072), G sets |q+G| < G_max with N_G 19-339, eta=0.1 eV",
            "value": n / (ms / 1e3), "unit": "blocks/s", "ms_per_batch": ms,
            "fp64_gpu": {"value": n / (ms64 / 1e3), "unit": "blocks/s", "ms_per_batch": ms64},
            "speedup_vs_fp64_gpu": ms64 / ms,
            "chi0_algorithmic_tflops_over_whole_batch": flops / (ms / 1e3) / 1e12,
            "timing": "CUDA events around qcx_solve_batch calls (graph replay, frequency upload, head copy-out)",
            "plan": info, "gpu_launches_per_batch": info["kernels_per_replay"]}


def surrogate_leg(stream):
    """The learned correction on its own workload (110 q of the mid workload,
    200 w each): heads by the mixed Dyson route, training on 100 q, evaluated on
    the 10 others; then the surrogate route (accept where sigma < 1e-2, 5 %
    spot check, Dyson fallback) on the held-out q."""
    import torch

    import synth
    from paper_2603_12326_gb300 import QCX_MIXED, qcx, states, surrogate

    ctx = qcx.Context(torch.cuda.current_device(), stream=stream.cuda_stream)
    p = synth.make_surrogate_set()
    L1, L2 = surrogate.head_table(ctx, p, range(p.nq))
    unit = 2.0 * np.pi / p.cell.a
    qmax, wmax = 4.0 * unit, float(p.w[-1])
    ntr = 100
    X, y, _ = surrogate.dataset(ctx, p, range(ntr), L1[:ntr], L2[:ntr], qmax, wmax)
    Xt, yt, _ = surrogate.dataset(ctx, p, range(ntr, p.nq), L1[ntr:], L2[ntr:], qmax, wmax)
    ctx.mlp_set_params(synth.mlp_init(2024))
    epochs = 200
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    curve = ctx.mlp_train(X, y, qcx.mlp_opts(epochs=epochs, batch=256, lr=1e-3, seed=5))
    e1.record(stream)
    torch.cuda.synchronize()
    train_ms = e0.elapsed_time(e1)
    mu, lv = ctx.mlp_predict(Xt)
    Xbig = np.tile(Xt, (max(1, 1000000 // len(Xt)), 1))
    ctx.mlp_predict(Xbig)
    torch.cuda.synchronize()
    e0.record(stream)
    ctx.mlp_predict(Xbig)
    e1.record(stream)
    torch.cuda.synchronize()
    pred_ms = e0.elapsed_time(e1)
    te = list(range(ntr, p.nq))
    states.load_problem(ctx, p, te)
    opts = qcx.SurrogateOpts(qmax, wmax, 1e-2, 0.05, 1e-2, 7)
    w = p.w[1:]
    ctx.surrogate_heads(range(len(te)), p.G_int, w, p.eta, opts, QCX_MIXED)
    torch.cuda.synchronize()
    e0.record(stream)
    _, _, src, chk = ctx.surrogate_heads(range(len(te)), p.G_int, w, p.eta, opts, QCX_MIXED)
    e1.record(stream)
    torch.cuda.synchronize()
    route_ms = e0.elapsed_time(e1)
    ctx.close()
    return {"workload": "110 q of the mid workload x 200 w (heads), 100 q train / 10 q held out",
            "train": {"samples": int(len(y)), "epochs": epochs, "ms": train_ms,
                      "samples_per_s": len(y) * epochs / (train_ms / 1e3), "loss_first_last": [float(curve[0]),
                                                                                               float(curve[-1])]},
            "predict_samples_per_s": len(Xbig) / (pred_ms / 1e3),
            "held_out": {"samples": int(len(yt)), "mae_log_ratio_network": float(np.mean(np.abs(mu - yt))),
                         "mae_log_ratio_no_lfe": float(np.mean(np.abs(yt)))},
            "route": {"value": len(te) * len(w) / (route_ms / 1e3), "unit": "blocks/s",
                      "accepted_fraction": float(np.mean(src == 0)), "spot_checked": int(np.sum(src == 2)),
                      "largest_spot_check_miss": chk,
                      "note": "accept where sigma < 1e-2; the rest falls back to the mixed Dyson route"}}


def run_profile_case_batch():
    """The uneven workload once through qcx_solve_batch (mixed, no autotuning:
    one capture, one replay) - every batch kernel launches once or twice."""
    import torch

    import synth
    from paper_2603_12326_gb300 import QCX_MIXED, qcx, states
    from paper_2603_12326_gb300.build import build
    build()
    ctx = qcx.Context(0)
    p = synth.make_uneven()
    states.load_problem(ctx, p)
    ctx.batch_autotune(False)
    e = p.extra
    ctx.solve_batch(e["inst_q"], e["inst_w"], e["inst_gmax"], p.eta, QCX_MIXED)
    torch.cuda.synchronize()
    ctx.close()
    print("profile case done")


def run_profile_case_mlp():
    """One training step's gradient on 256 samples and a 20000-sample prediction."""
    import synth
    from paper_2603_12326_gb300 import qcx
    from paper_2603_12326_gb300.build import build
    build()
    ctx = qcx.Context(0)
    rng = np.random.default_rng(3)
    X = rng.standard_normal((20000, 6)).astype(np.float32)
    y = rng.standard_normal(20000).astype(np.float32)
    ctx.mlp_set_params(synth.mlp_init(1))
    ctx.mlp_grad(X[:256], y[:256])
    ctx.mlp_predict(X)
    ctx.close()
    print("profile case done")


def run_profile_case(nw=50):
    """1 q x nw w of the mid workload through the mixed path, twice (nw = 200 is the
    launch configuration the benchmark step times)."""
    import torch

    import synth
    from paper_2603_12326_gb300 import QCX_MIXED, qcx, states
    from paper_2603_12326_gb300.build import build
    build()
    ctx = qcx.Context(0)
    prob = synth.make_mid(nq=1, nw=nw)
    states.load_problem(ctx, prob)
    for _ in range(2):
        ctx.pair_density(0, prob.G_int, QCX_MIXED)
        ctx.chi0(0, prob.w, prob.eta, QCX_MIXED)
        ctx.invert_eps(0, QCX_MIXED, want=False)
    ctx.sync()
    torch.cuda.synchronize()
    ctx.close()
    print("profile case done")


def run_profile_case_spectral(frac=20):
    """q 0 of the mid workload through the mixed spectral route (grid step eta/frac,
    all 200 w), twice: the launch configuration of the bench's spectral leg."""
    import torch

    import synth
    from paper_2603_12326_gb300 import QCX_MIXED, qcx, states
    from paper_2603_12326_gb300.build import build
    build()
    ctx = qcx.Context(0)
    prob = synth.make_mid(nq=1)
    states.load_problem(ctx, prob)
    step = prob.eta / frac
    E0, nbin = ctx.spectral_grid(0, step)
    for _ in range(2):
        ctx.pair_density(0, prob.G_int, QCX_MIXED)
        ctx.chi0_spectral(0, prob.w, prob.eta, E0, step, nbin, QCX_MIXED)
    ctx.sync()
    torch.cuda.synchronize()
    ctx.close()
    print("profile case done")


def _relaunch(n):
    """Re-run this command as n ranks (torch.distributed.run, 127.0.0.1)."""
    import socket
    with socket.socket() as so:
        so.bind(("127.0.0.1", 0))
        port = so.getsockname()[1]
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={n}",
           "--master-addr=127.0.0.1", f"--master-port={port}", os.path.abspath(__file__), *sys.argv[1:]]
    os.execv(sys.executable, cmd)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle sample")
    ap.add_argument("--no-surrogate", action="store_true", help="skip the learned-correction leg")
    ap.add_argument("--no-sweep", action="store_true", help="skip the accuracy sweep over every q")
    ap.add_argument("--no-large", action="store_true", help="skip the large-workload leg")
    ap.add_argument("--no-spectral", action="store_true", help="skip the spectral-route leg")
    ap.add_argument("--profile-case", nargs="?", const="mid", choices=["mid", "mid200", "batch", "mlp", "spectral"],
                    help="small case for profilers, no report: mid = 1 q x 50 w of the mid workload, 2 passes; "
                         "batch = the uneven workload once; mlp = one gradient and one prediction")
    args = ap.parse_args()
    ws, rank, local = _dist()
    if "WORLD_SIZE" not in os.environ and args.gpus > 1:
        # started without a launcher: start the N ranks here, one process per GPU
        _relaunch(args.gpus)
    if ws != args.gpus:
        sys.exit(f"bench.py: --gpus {args.gpus} but the launcher started {ws} rank(s)")
    if ws > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    if args.profile_case == "mid":
        run_profile_case()
    elif args.profile_case == "mid200":
        run_profile_case(200)
    elif args.profile_case == "batch":
        run_profile_case_batch()
    elif args.profile_case == "mlp":
        run_profile_case_mlp()
    elif args.profile_case == "spectral":
        run_profile_case_spectral()
    elif args.impl == "reference":
        run_reference(args, ws, rank)
    else:
        run_ours(args, ws, rank, local)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
