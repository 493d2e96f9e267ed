#!/usr/bin/env python
"""Benchmark: site-frequencies/s of diag(H(i w_k)^-1) by the Lanczos-based
low-rank correction method on one GB300 (per GPU: one replica of the workload).

Workload (default, the largest single-GPU configuration): 512x512 open square
lattice, t = -1, mu = 0, trap V_i = 0.01 r_i^2, Sigma_i = a_i - i b_i sign(w_k)
(a ~ U[-1,1], b ~ U[0,0.5]), 32 Matsubara frequencies at beta = 10, p = 16
strip subdomains, Lanczos rank cap k = 64, mixed precision; all 32 frequencies
in one batched, graph-replayed launch sequence.  Side measurements on the
128x128, 64-frequency workload (p = 4, k = 32): its own throughput, one
frequency per launch against the batch, the exact p = 1 diagonal, block
Lanczos and the stencil SpMV.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--form mixed|fp64]
    python bench.py --impl reference      # the FP64 CPU oracle on the host cores

Prints ONE JSON line (rank 0).  A "step" is one full solve of all frequencies
with inputs resident on the device; `e2e` repeats it through the C ABI with
pinned host buffers, host<->device copies inside the timed region.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "site-frequencies/s for diag(H^-1) at ≤1e-6 rel err vs plain; p50/p99 solve latency"
UNIT = "site-frequencies/s"
DEFAULT_WORKLOAD = "square512_K32_p16_k64"
SIDE_WORKLOAD = "square128_K64_p4_k32"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_source_hash():
    """Hash of every kernel source (any change invalidates recorded ncu traffic)."""
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1102_3137_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        if f.endswith(".cuh") or (f.startswith("k_") and f.endswith(".cu")):
            with open(os.path.join(csrc, f), "rb") as fh:
                h.update(fh.read())
    return h.hexdigest()[:16]


def lanczos_algorithmic_bytes(steps, N, reads):
    """Algorithmic DRAM bytes of the Lanczos steps of one solve: a frequency that ran n
    steps read the basis `reads` times at step j (j vectors of N complex entries of 16 B)
    plus ~6 N-vectors per step: sum over j = 1..n of (reads j + 6) N 16 B."""
    return float(sum((reads * n * (n + 1) / 2 + 6.0 * n) * N * 16.0 for n in steps))


def union_ms(starts, ends):
    """Total length of the union of intervals [starts[k], ends[k]]."""
    tot, cur_a, cur_b = 0.0, None, None
    for a_, b_ in sorted(zip(starts, ends)):
        if cur_b is None or a_ > cur_b:
            if cur_b is not None:
                tot += cur_b - cur_a
            cur_a, cur_b = a_, b_
        else:
            cur_b = max(cur_b, b_)
    if cur_b is not None:
        tot += cur_b - cur_a
    return float(tot)


def recorded_traffic(kernel, workload):
    """DRAM bytes per step (all launches of the kernel) from the last ncu capture, if the
    kernel has not changed since."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            d = json.load(f)
        e = d.get(kernel, {}).get(workload, {})
        if e.get("source_hash") == kernel_source_hash():
            return float(e["dram_bytes_per_step"])
    except Exception:
        pass
    return None


# FP64 peak of GB300: 152 SMs x 2 FP64 FMA/clk/SM x 2 flop x 2.07 GHz (the
# nominal 1.25 TFLOP/s of the part).
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


# ----------------------------------------------------------------- oracle timing
def _oracle_freq(args):
    name, k, threads = args
    for v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = str(threads)
    from oracle import dyson_oracle as O
    from paper_1102_3137_gb300 import inputs as I
    w = I.WORKLOADS[name]
    omega, V, sigma, q1 = I.make_inputs(w)
    t0 = time.perf_counter()
    O.lowrank_diag(w.L, (False,) * 3, w.t, w.mu, V, sigma[k], omega[k], q1, w.p, w.k)
    return time.perf_counter() - t0


def oracle_sample(name, n_freq, cores, offset=0):
    """The seeded frequency sample of one oracle measurement: n_freq frequencies spread
    over the grid (k = 0, the lowest and worst conditioned, always first), rotated by
    `offset` steps of the spread."""
    from paper_1102_3137_gb300 import inputs as I
    w = I.WORKLOADS[name]
    n = max(1, min(n_freq, w.K))
    ks = sorted({int(round(x)) for x in [i * (w.K - 1) / max(1, n - 1) for i in range(n)]}) if n > 1 else [0]
    if offset:
        ks = sorted({(k + offset * max(1, w.K // max(1, n))) % w.K for k in ks})
    return ks


def oracle_rate(name, n_freq, cores, offset=0):
    return oracle_rate_ks(name, oracle_sample(name, n_freq, cores, offset), cores)


def oracle_rate_ks(name, ks, cores):
    """Time the FP64 oracle on the frequencies ks of a workload, on `cores`
    host cores: one spawned worker per frequency (one BLAS thread each) when the sample
    has at least as many frequencies as cores, else one worker per frequency with the
    cores shared out as BLAS threads."""
    import multiprocessing as mp
    from paper_1102_3137_gb300 import inputs as I
    w = I.WORKLOADS[name]
    procs = max(1, min(len(ks), cores))
    threads = max(1, cores // procs)
    ctx = mp.get_context("spawn")
    t0 = time.perf_counter()
    with ctx.Pool(processes=procs) as pool:
        per = pool.map(_oracle_freq, [(name, k, threads) for k in ks])
    wall = time.perf_counter() - t0
    value = len(ks) * w.N / wall
    return dict(value=value, unit=UNIT, cores=procs * threads, kind="oracle",
                sample=f"{len(ks)} of {w.K} frequencies (k = {','.join(map(str, ks))}), full "
                       f"{'x'.join(map(str, w.L))} lattice, {procs} worker(s) x {threads} BLAS thread(s), "
                       f"wall {wall:.2f} s, per-frequency {statistics.mean(per):.2f} s; time for all K = {w.K} "
                       f"at this rate (extrapolated, not measured): {wall * w.K / len(ks):.1f} s",
                wall_s=wall)


# ----------------------------------------------------------------- clocks
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.idx = gpu_index
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
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
        rows = []
        with open(self.f.name) as f:
            for line in f:
                c = [x.strip() for x in line.split(",")]
                if len(c) >= 9:
                    rows.append(c)
        os.unlink(self.f.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = max(float(r[2]) for r in rows if r[2].replace(".", "").isdigit())
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return dict(sm_mhz=statistics.median(sm) if sm else None, sm_max_mhz=mx, reasons=reasons,
                    samples=len(rows),
                    power_w_max=max(float(r[3]) for r in rows if r[3].replace(".", "").isdigit()))


REC_MIN_SITES = 1024


def side_measurements(a, dev, stream):
    """The 128x128, 64-frequency workload (p = 4, k = 32) beside the headline: its own
    batched throughput in the headline's form and in plain FP64 (with the error between
    them), one frequency per launch against the batch, the exact diagonal (p = 1) and
    the low-rank truncation error against it, block Lanczos, the recursive
    decomposition, and the complex64 stencil SpMV on a batch far larger than L2."""
    import numpy as np
    import torch
    from paper_1102_3137_gb300 import dyson as D
    from paper_1102_3137_gb300 import inputs as I
    w = I.WORKLOADS[SIDE_WORKLOAD]
    omega, V, sigma, q1 = I.make_inputs(w)
    t = lambda x: torch.from_numpy(x).to(dev)
    om, Vd, sg, qd = t(omega), t(V), t(sigma), t(q1)
    ss = stream.cuda_stream
    prec = D.DYSON_MIXED if a.form == "mixed" else D.DYSON_FP64
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    nrep = 3

    def timed(plan, K, *args, nb=1):
        D.dyson_solve(plan.handle, K, *args, ss, nb)           # warm-up (autotune, capture)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(nrep):
            D.dyson_solve(plan.handle, K, *args, ss, nb)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / nrep

    side = dict(workload=SIDE_WORKLOAD, lattice="x".join(map(str, w.L)), K=w.K, p=w.p, k=w.k)
    out = torch.zeros((w.K, w.N), dtype=torch.complex128, device=dev)
    st = torch.zeros(w.K, dtype=torch.int32, device=dev)
    pm = D.Plan(w.L, w.t, w.mu, w.p, w.k, prec, max_freqs=w.K)
    ms = timed(pm, w.K, om, Vd, sg, qd, out, st)
    res = out.cpu().numpy()
    side["batched"] = dict(form=a.form, value=w.K * w.N / (ms / 1e3), ms_per_step=ms)
    pm.close()
    pf = D.Plan(w.L, w.t, w.mu, w.p, w.k, D.DYSON_FP64, max_freqs=w.K)
    outf = torch.zeros_like(out)
    ms_f = timed(pf, w.K, om, Vd, sg, qd, outf, st)
    plain = outf.cpu().numpy()
    rel = np.abs(res - plain) / np.abs(plain)
    side["fp64_plain"] = dict(value=w.K * w.N / (ms_f / 1e3), ms_per_step=ms_f)
    side["err_vs_plain"] = dict(max=float(rel.max()), median=float(np.median(rel)),
                                sites_above_1e_6=int((rel > 1e-6).sum()))
    pf.close()
    # one frequency per launch vs all frequencies in one batch (same form)
    p1 = D.Plan(w.L, w.t, w.mu, w.p, w.k, prec, max_freqs=1)
    o1 = torch.zeros((1, w.N), dtype=torch.complex128, device=dev)
    s1 = torch.zeros(1, dtype=torch.int32, device=dev)
    D.dyson_solve(p1.handle, 1, om[:1], Vd, sg[:1], qd, o1, s1, ss)
    torch.cuda.synchronize()
    e0.record(stream)
    for k in range(w.K):
        D.dyson_solve(p1.handle, 1, om[k:k + 1], Vd, sg[k:k + 1], qd, o1, s1, ss)
    e1.record(stream)
    torch.cuda.synchronize()
    ms1 = e0.elapsed_time(e1)
    side["one_frequency_per_launch"] = dict(value=w.K * w.N / (ms1 / 1e3), ms_all=ms1)
    p1.close()
    # exact diagonal as its own mode: one subdomain, so diag(H^-1) = diag(B^-1) from the
    # slice recursion alone (no interface, no Lanczos), FP64; its throughput, and the
    # truncation error of the low-rank result against it
    pe = D.Plan(w.L, w.t, w.mu, 1, 1, D.DYSON_FP64, max_freqs=w.K)
    oute = torch.zeros_like(out)
    ms_e = timed(pe, w.K, om, Vd, sg, qd, oute, st)
    exact = oute.cpu().numpy()
    tr = np.abs(res - exact) / np.abs(exact)
    side["exact_p1"] = dict(value=w.K * w.N / (ms_e / 1e3), ms_per_step=ms_e, form="fp64",
                            lowrank_truncation_error=dict(max=float(tr.max()), median=float(np.median(tr))))
    pe.close()
    # block Lanczos (block size 2, the same rank cap k: k/2 block steps) in the
    # headline form: throughput and truncation error against the exact diagonal
    nbb = 2
    pb = D.Plan(w.L, w.t, w.mu, w.p, w.k, prec, max_freqs=w.K, block_size=nbb)
    qb = t(I.start_block(q1, nbb))
    outb = torch.zeros_like(out)
    stb = torch.zeros_like(st)
    ms_b = timed(pb, w.K, om, Vd, sg, qb, outb, stb, nb=nbb)
    tb = np.abs(outb.cpu().numpy() - exact) / np.abs(exact)
    side["block_lanczos"] = dict(block_size=nbb, value=w.K * w.N / (ms_b / 1e3), ms_per_step=ms_b,
                                 form=a.form, status_flags=sorted(set(stb.cpu().tolist())),
                                 truncation_error=dict(max=float(tb.max()), median=float(np.median(tb))))
    pb.close()
    # the recursive decomposition (Sec. 2.3, last paragraph; domains alternating
    # (2,1), (1,2), ...) down to boxes of 1024 sites, the same rank cap in every
    # box, in the headline form: throughput and truncation error against the exact
    # diagonal
    rp = D.RecursivePlan(w.L, w.t, w.mu, w.k, prec, max_freqs=w.K, min_sites=REC_MIN_SITES,
                         first_cut=D.DYSON_CUT_X)
    outr = torch.zeros_like(out)
    str_ = torch.zeros_like(st)
    D.dyson_recursive_solve(rp.handle, w.K, w.N, om, Vd, sg, qd, outr, str_, ss)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(nrep):
        D.dyson_recursive_solve(rp.handle, w.K, w.N, om, Vd, sg, qd, outr, str_, ss)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_r = e0.elapsed_time(e1) / nrep
    trr = np.abs(outr.cpu().numpy() - exact) / np.abs(exact)
    info = rp.info()
    side["recursive"] = dict(min_sites=REC_MIN_SITES, levels=info["levels"], boxes=info["boxes"],
                             leaves=info["leaves"], value=w.K * w.N / (ms_r / 1e3), ms_per_step=ms_r,
                             form=a.form, status_flags=sorted(set(str_.cpu().tolist())),
                             truncation_error=dict(max=float(trr.max()), median=float(np.median(trr))))
    rp.close()
    # the complex64 stencil SpMV (row a1, y = H(i w_k) x) on a batch far larger than L2:
    # algorithmic 32 B per site-frequency (x c64 8 + y c64 8 + Sigma c128 16; V stays in L2)
    Ks = 4096
    hbm_peak, _ = peaks()
    ps = D.Plan(w.L, w.t, w.mu, w.p, 1, D.DYSON_FP64, max_freqs=1)   # device buffers: no plan storage used
    om_s = torch.from_numpy(I.matsubara(w.beta, Ks)).to(dev)
    sg_s = sg[:1].repeat(Ks, 1).contiguous()
    xs = torch.randn((Ks, w.N), dtype=torch.complex64, device=dev)
    ysp = torch.empty_like(xs)
    for _ in range(3):
        D.dyson_apply_H_c64(ps.handle, Ks, om_s, Vd, sg_s, xs, ysp, ss)
    reps = 10
    e0.record(stream)
    for _ in range(reps):
        D.dyson_apply_H_c64(ps.handle, Ks, om_s, Vd, sg_s, xs, ysp, ss)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_k = e0.elapsed_time(e1) / reps
    gbs = 32.0 * Ks * w.N / (ms_k / 1e3) / 1e9
    side["spmv_c64"] = dict(bound="hbm", achieved=gbs, peak=hbm_peak, unit="GB/s",
                            frac=gbs / hbm_peak, ms_per_launch=ms_k,
                            work=f"{Ks} frequencies x {w.N} sites, 32 B algorithmic per site-frequency")
    ps.close()
    del sg_s, xs, ysp
    return side


# ----------------------------------------------------------------- our arm
def aggregate_ranks(total_ms, units_per_step, steps, world, device="cpu"):
    """(ms per step, whole-job units/s) of `world` replicas that each processed
    units_per_step units per step for `steps` steps in total_ms: the job's time is
    the slowest rank's (MAX over ranks), its work the sum over ranks."""
    if world > 1:
        import torch
        tt = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
        torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(tt.item())
    ms_per_step = total_ms / steps
    return ms_per_step, world * units_per_step / (ms_per_step / 1e3)


def run_ours(a, rank, world, local_rank):
    import numpy as np
    import torch
    from paper_1102_3137_gb300 import build as B
    from paper_1102_3137_gb300 import dyson as D
    from paper_1102_3137_gb300 import inputs as I

    if rank == 0:
        B.build()
    if world > 1:
        torch.distributed.barrier()
    D.load()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    w = I.WORKLOADS[a.workload]
    omega, V, sigma, q1 = I.make_inputs(w, seed=w.seed + rank)
    t = lambda x: torch.from_numpy(x).to(dev)
    om, Vd, sg, qd = t(omega), t(V), t(sigma), t(q1)
    prec = D.DYSON_MIXED if a.form == "mixed" else D.DYSON_FP64
    stream = torch.cuda.current_stream(dev)
    ss = stream.cuda_stream

    # CPU baseline first (spawned pool, before the first CUDA call of the workload)
    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        cpu = oracle_rate(a.workload, cpu_freqs(a, w), os.cpu_count() or 1)

    plan = D.Plan(w.L, w.t, w.mu, w.p, w.k, prec, max_freqs=w.K)
    D.dyson_plan_set_profiling(plan.handle, 1)
    out = torch.zeros((w.K, w.N), dtype=torch.complex128, device=dev)
    st = torch.zeros(w.K, dtype=torch.int32, device=dev)

    def step():
        D.dyson_solve(plan.handle, w.K, om, Vd, sg, qd, out, st, ss)

    for _ in range(a.warmup):
        step()
    torch.cuda.synchronize()
    clocks = Clocks(local_rank) if rank == 0 else None
    if clocks:
        clocks.start()
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(a.steps + 1)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    evs[0].record(stream)
    for i in range(a.steps):
        step()
        evs[i + 1].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop() if clocks else None
    step_ms = [evs[i].elapsed_time(evs[i + 1]) for i in range(a.steps)]
    total_ms = evs[0].elapsed_time(evs[-1])
    ms_per_step, value = aggregate_ranks(total_ms, w.K * w.N, a.steps, world, dev)

    # kernel profile of the last timed step (events captured inside the graph)
    kinds, kms = D.dyson_profile_read(plan.handle)
    n_launch = len(kinds)
    sweeps = D.dyson_work_counters(plan.handle, w.K, w.p)
    info = plan.info(w.K)
    status = st.cpu().numpy()
    res = out.cpu().numpy()
    xm = kms[kinds == 3]
    heights, _, _ = D.dyson_partition(plan.geom)
    T = 1 if len(w.L) == 2 else w.L[1]
    wi = np.array([T * h for h in heights], dtype=np.float64)
    cs = 8 if prec == D.DYSON_MIXED else 16
    # algorithmic work of one sweep of subdomain i: g_s read twice (forward, back),
    # Lx blocks of w_i x w_i complex entries; 8 real flops per complex multiply-add.
    sw_bytes = float((sweeps.astype(np.float64) * (2 * w.L[0] * wi * wi * cs)[None, :]).sum())
    sw_flops = float((sweeps.astype(np.float64) * (2 * w.L[0] * wi * wi * 8)[None, :]).sum())
    n_xm = max(1, len(xm))
    hbm_peak, peak_src = peaks()
    xm_avg_ms = float(xm.mean()) if len(xm) else float("nan")
    # the frequency groups' X-matvec launches overlap in time: the kernel's time
    # in the step is the union of its launch intervals (CUDA events on each
    # launch's own stream, inside the replayed graph)
    t0, t1 = D.dyson_profile_spans(plan.handle)
    xm_union_ms = union_ms(t0[kinds == 3], t1[kinds == 3])
    if prec == D.DYSON_MIXED:
        ach = sw_bytes / (xm_union_ms / 1e3) / 1e9
        roof = dict(bound="hbm", achieved=ach, peak=hbm_peak, unit="GB/s", frac=ach / hbm_peak,
                    traffic=recorded_traffic("k_xmatvec<float>", a.workload),
                    kernel="k_xmatvec<float>", peak_source=peak_src,
                    per_step_algorithmic_bytes=sw_bytes,
                    per_launch_algorithmic_bytes=sw_bytes / n_xm,
                    per_launch_achieved=sw_bytes / n_xm / (xm_avg_ms / 1e3) / 1e9)
    else:
        ach = sw_flops / (xm_union_ms / 1e3) / 1e12
        roof = dict(bound="alu", achieved=ach, peak=FP64_PEAK_TFLOPS, unit="TFLOP/s",
                    frac=ach / FP64_PEAK_TFLOPS,
                    traffic=recorded_traffic("k_xmatvec<double>", a.workload),
                    kernel="k_xmatvec<double>",
                    peak_source="derived: 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz",
                    per_step_algorithmic_flops=sw_flops,
                    per_launch_algorithmic_flops=sw_flops / n_xm,
                    per_launch_achieved=sw_flops / n_xm / (xm_avg_ms / 1e3) / 1e12)
    roof.update(launches_per_step=int(len(xm)), union_ms_per_step=xm_union_ms,
                mean_launch_ms=xm_avg_ms,
                basis="achieved = algorithmic bytes (flops) of all X-matvec launches of a step / "
                      "the union of their intervals; traffic = ncu DRAM bytes of those launches per step")
    roof["share_of_step"] = float(xm_union_ms / ms_per_step) if ms_per_step > 0 else None
    # the Lanczos step (row a7/a8), complex128-sized entries of 16 B per site.  The
    # FP64 form's CGS2 reads the basis three times per step (g = Q^T u; r1 = u - Q g
    # with h = Q^T r1 in the same pass; r = r1 - Q h); the mixed form's takes h from
    # the Gram matrix of the basis and reads it twice (g = Q^T u; r = u - Q (g + h)
    # with the next Gram column Q^T r in the same pass).  Plus ~6 vectors (u, q_j,
    # q_{j-1}, r written, the running diagonal read and written).  A frequency that
    # ran n steps moves sum_{j=1..n} (reads j + 6) N 16 B.
    lz = kms[kinds == 4]
    steps_k = np.asarray(info["steps"], dtype=np.float64)
    lz_reads = 2 if (prec == D.DYSON_MIXED and w.k <= 64) else 3
    lz_bytes = lanczos_algorithmic_bytes(steps_k, w.N, lz_reads)
    lz_union = union_ms(t0[kinds == 4], t1[kinds == 4])
    lz_ach = lz_bytes / (lz_union / 1e3) / 1e9 if lz_union > 0 else float("nan")
    roof_lz = dict(bound="hbm", achieved=lz_ach, peak=hbm_peak, unit="GB/s", frac=lz_ach / hbm_peak,
                   traffic=recorded_traffic("k_lanczos", a.workload),
                   kernel="k_lanczos_dd" if prec == D.DYSON_MIXED else "k_lanczos", peak_source=peak_src,
                   per_step_algorithmic_bytes=lz_bytes, launches_per_step=int(len(lz)),
                   union_ms_per_step=lz_union, mean_launch_ms=float(lz.mean()) if len(lz) else None,
                   basis=("two reads of the basis per Lanczos step (CGS2, second-pass coefficients "
                          "from the Gram matrix)" if lz_reads == 2 else
                          "three reads of the basis per Lanczos step (CGS2)") +
                         " + 6 vectors, complex128, over the union of the step's Lanczos launch intervals")
    phases = {D.KERNEL_NAMES[int(k)]: round(float(kms[kinds == k].sum()), 3) for k in sorted(set(kinds))}
    tuning = D.dyson_plan_tuning(plan.handle)

    extra = {}
    if rank == 0 and world == 1 and not a.quick:
        # error vs the plain FP64 GPU method (the metric's condition) and its throughput
        pf = D.Plan(w.L, w.t, w.mu, w.p, w.k, D.DYSON_FP64, max_freqs=w.K)
        outf = torch.zeros_like(out)
        stf = torch.zeros_like(st)
        D.dyson_solve(pf.handle, w.K, om, Vd, sg, qd, outf, stf, ss)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        nf = 2
        e0.record(stream)
        for _ in range(nf):
            D.dyson_solve(pf.handle, w.K, om, Vd, sg, qd, outf, stf, ss)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_f = e0.elapsed_time(e1) / nf
        plain = outf.cpu().numpy()
        rel = np.abs(res - plain) / np.abs(plain)
        extra["err_vs_plain"] = dict(max=float(rel.max()), median=float(np.median(rel)),
                                     sites_above_1e_6=int((rel > 1e-6).sum()))
        extra["fp64_plain"] = dict(value=w.K * w.N / (ms_f / 1e3), ms_per_step=ms_f,
                                   autotuner=D.dyson_plan_tuning(pf.handle))
        pf.close()
        del outf, stf
        if a.workload != SIDE_WORKLOAD:
            extra["side_" + SIDE_WORKLOAD] = side_measurements(a, dev, stream)
        torch.cuda.empty_cache()
        if not a.no_serving_sample:
            extra["serving"] = serving_stream(SAMPLE_SIZES, 16, 48, 12, [0.8, 2.0], 8)
            extra["serving"]["sample"] = ("bounded sample of the serving stream: 12 requests over "
                                          "64^2, 128^2, 256^2 and 24^3, K in 16..48 (the full stream, "
                                          "with 48^3 and K up to 256: bench.py --serving)")
            torch.cuda.empty_cache()

    e2e = None
    if True:
        pin = lambda x: torch.from_numpy(x).pin_memory().numpy()
        h_om, h_V, h_sg, h_q = pin(omega), pin(V), pin(sigma), pin(q1)
        h_out = torch.zeros((w.K, w.N), dtype=torch.complex128).pin_memory().numpy()
        h_st = torch.zeros(w.K, dtype=torch.int32).pin_memory().numpy()
        D.dyson_solve(plan.handle, w.K, h_om, h_V, h_sg, h_q, h_out, h_st, ss)
        n_e2e = max(2, a.steps // 2)
        if world > 1:
            torch.distributed.barrier()
        t0 = time.perf_counter()
        for _ in range(n_e2e):
            D.dyson_solve(plan.handle, w.K, h_om, h_V, h_sg, h_q, h_out, h_st, ss)
        e2e_ms, e2e_value = aggregate_ranks((time.perf_counter() - t0) * 1e3, w.K * w.N, n_e2e, world, dev)
        e2e_s = e2e_ms / 1e3
        e2e = dict(value=e2e_value, unit=UNIT,
                   h2d_bytes_per_step=int(h_om.nbytes + h_V.nbytes + h_sg.nbytes + h_q.nbytes),
                   d2h_bytes_per_step=int(h_out.nbytes + h_st.nbytes), ms_per_step=e2e_s * 1e3)
    plan.close()
    if rank != 0:
        return None
    sl = sorted(step_ms)
    pct = lambda q: sl[min(len(sl) - 1, int(math.ceil(q * len(sl))) - 1)]
    line = dict(
        metric=METRIC, value=value, unit=UNIT, n_gpus=world, steps=a.steps, warmup=a.warmup,
        ms_per_step=ms_per_step, higher_is_better=True, scaling="weak", vs_baseline=None,
        dtype="mixed c64/f64 (c64 sweeps, 2xf32 slice recursion, f64 Lanczos and refinement)" if prec == D.DYSON_MIXED else "c128 (f64)",
        data="synthetic",
        config=dict(workload=a.workload, lattice="x".join(map(str, w.L)), K=w.K, p=w.p, k=w.k,
                    form=a.form, N=w.N, beta=w.beta,
                    l2="per-step working set > L2: factors + Lanczos basis ~1 GB, no flush",
                    parallelism=f"replicas x{world}"),
        latency_ms=dict(p50=pct(0.50), p99=pct(0.99)),
        roofline=roof, roofline_lanczos=roof_lz, phases_ms_last_step=phases, autotuner=tuning,
        interface_iterations_per_xmatvec=float(np.mean(info["iters"]) / max(1, w.k)),
        status_flags=sorted({int(x) for x in status}),
        cpu_baseline=({k: v for k, v in cpu.items() if k != "wall_s"} if cpu else None),
        e2e=e2e, gpu_launches=int(n_launch * a.steps), clocks=clk,
        **extra)
    return line


# ----------------------------------------------------------------- reference arm
def cpu_freqs(a, w):
    """Frequencies per bounded oracle sample: about 10-30 s of host work.  One oracle
    frequency of the 512^2 workload (its full-lattice factorisation dominates) takes
    ~14 s on 16 cores, one of the 128^2 workload under a second on one core."""
    if a.cpu_freqs:
        return a.cpu_freqs
    return 1 if w.N >= 100000 else 16


def run_reference(a, rank, world):
    """The FP64 CPU oracle as the reference arm, on the host cores: every step a bounded
    sample of the workload's frequencies (rotating through a seeded subset that holds
    k = 0), timed per step; the value is the site-frequencies of the samples over their
    time."""
    if rank != 0:
        return None
    from paper_1102_3137_gb300 import inputs as I
    w = I.WORKLOADS[a.workload]
    cores = os.cpu_count() or 1
    n = cpu_freqs(a, w)
    if a.warmup > 0:                      # page numpy and the oracle in, on a tiny lattice
        oracle_rate("square16_K8_p2_k16", 1, 1)
    subset = oracle_sample(a.workload, max(4, n), cores)
    vals = []
    for i in range(a.steps):
        if n >= len(subset):
            vals.append(oracle_rate(a.workload, n, cores))
        else:
            vals.append(oracle_rate_ks(a.workload, [subset[(i * n + c) % len(subset)] for c in range(n)], cores))
    wall = sum(v["wall_s"] for v in vals)
    value = n * w.N * a.steps / wall
    ms = wall / a.steps * 1e3
    c = vals[-1]
    return dict(
        impl="reference", metric=METRIC, value=value, unit=UNIT, n_gpus=world, steps=a.steps,
        warmup=a.warmup, ms_per_step=ms, higher_is_better=True, scaling="weak", vs_baseline=None,
        dtype="c128 (f64)", data="synthetic",
        config=dict(workload=a.workload, lattice="x".join(map(str, w.L)), K=w.K, p=w.p, k=w.k,
                    form="fp64 oracle", N=w.N, beta=w.beta,
                    step=f"{n} of {w.K} frequencies per step (bounded CPU sample), rotating through "
                         f"k = {','.join(map(str, subset))}"),
        cpu_baseline=dict(value=value, unit=UNIT, cores=c["cores"], kind="oracle", sample=c["sample"]),
        e2e=dict(value=value, unit=UNIT, h2d_bytes_per_step=0, d2h_bytes_per_step=0),
        gpu_launches=0)


# ----------------------------------------------------------------- serving stream
# lattices of the serving stream: (L, p, k, frequencies a resident plan holds; a request
# with more runs as consecutive chunks on its plan).  48^3 takes p = 16 (slice width 144),
# so both forms run it (p = 8 gives W = 288, complex64 form only).
SERVE_SIZES = [((64, 64), 4, 32, 128), ((128, 128), 4, 32, 128), ((256, 256), 8, 48, 64),
               ((24, 24, 24), 4, 48, 64), ((48, 48, 48), 16, 64, 16)]
# the bounded sample in the bench line: the 2D lattices and 24^3 (a 48^3 request alone
# takes ~17 s mixed and ~50 s in FP64 at K = 16), K in 16..48, 12 requests
SAMPLE_SIZES = SERVE_SIZES[:4]


def serving_stream(sizes, kmin, kmax, nreq, rate_fracs, inflight, seed=5):
    """Open-loop Poisson arrivals of Dyson solves from simulated IDMFT loops.

    Lattices drawn uniformly from `sizes`, K uniform in [kmin, kmax], a fresh seeded
    self-energy per request (seed 1000 + request index).  The plain-FP64 capacity is
    measured first by solving every request alone, one after the other (each submitted
    after the previous one finished, so none is fused; after one untimed pass that
    creates the plans and captures their graphs); the stream then
    arrives at rate_frac x that capacity and is served by the continuous-batching server
    (mixed form, plans resident and reused).  Reports delivered site-frequencies/s,
    p50/p99 latency from submission, and the served results' error against the plain
    FP64 per-request results.
    """
    import numpy as np
    import torch
    from paper_1102_3137_gb300 import dyson as D
    from paper_1102_3137_gb300 import inputs as I
    rng = np.random.default_rng(seed)
    reqs = []
    pin = lambda x: torch.from_numpy(np.ascontiguousarray(x)).pin_memory().numpy()
    # one simulated IDMFT client per lattice: its trap V and Lanczos start vector stay
    # fixed over its iterations (seeded 5000 + lattice index), Sigma is fresh per request
    client = {}
    for n in range(nreq):
        li = int(rng.integers(len(sizes)))
        L, p, k, cap = sizes[li]
        K = int(rng.integers(kmin, kmax + 1))
        w = I.Workload("serve", L, -1.0, 0.0, 0.01, 0.5, 20.0, K, p, k, 1000 + n)
        omega, _, sigma, _ = I.make_inputs(w)
        if li not in client:
            wc = I.Workload("client", L, -1.0, 0.0, 0.01, 0.5, 20.0, 1, p, k, 5000 + li)
            _, Vc, _, qc = I.make_inputs(wc)
            client[li] = (pin(Vc), pin(qc))
        V, q1 = client[li]
        zero = lambda: torch.zeros((K, w.N), dtype=torch.complex128).pin_memory().numpy()
        reqs.append(dict(w=w, cap=cap, omega=pin(omega), V=V, sigma=pin(sigma), q1=q1,
                         out=zero(), plain=zero()))
    work = sum(r["w"].N * r["w"].K for r in reqs)

    def serve(prec, arrivals, nflight, key, one_by_one=False):
        srv = D.dyson_server_create(96 << 30, max_inflight=nflight)
        t0 = time.perf_counter()
        tickets, lat = [], []
        for r, ta in zip(reqs, arrivals):
            dt = ta - (time.perf_counter() - t0)
            if dt > 0:
                time.sleep(dt)
            w = r["w"]
            geom = D.make_geometry(w.L, w.t, w.mu, w.p, w.k, prec, max_freqs=r["cap"])
            tickets.append(D.dyson_submit(srv, geom, w.K, r["omega"], r["V"], r["sigma"], r["q1"], r[key]))
            if one_by_one:                   # per-request solves: nothing queues, nothing fuses
                lat.append(D.dyson_wait(srv, tickets.pop())[0])
        lat += [D.dyson_wait(srv, t)[0] for t in tickets]
        wall = time.perf_counter() - t0
        st = D.dyson_server_stats(srv)
        D.dyson_server_destroy(srv)
        return wall, lat, st

    serve(D.DYSON_FP64, [0.0] * len(reqs), 1, "plain", True)          # plans and graphs
    wall_plain, _, _ = serve(D.DYSON_FP64, [0.0] * len(reqs), 1, "plain", True)
    capacity = work / wall_plain
    mean_work = work / len(reqs)
    out = dict(unit="site-frequencies/s", requests=len(reqs), site_frequencies=work,
               config=dict(lattices=" | ".join(f"{'x'.join(map(str, L))} p={p} k={k} plan={c}"
                                               for L, p, k, c in sizes),
                           K=f"uniform {kmin}..{kmax}", arrivals=f"open-loop Poisson, seed {seed}",
                           served_form="mixed", max_inflight=inflight, hbm_budget_gb=96),
               plain_fp64_capacity=capacity, plain_fp64_sequential_wall_s=wall_plain, rates=[])
    serve(D.DYSON_MIXED, [0.0] * len(reqs), inflight, "out")         # mixed plans and graphs
    for frac in rate_fracs:
        lam = frac * capacity / mean_work                              # requests per second
        gaps = np.random.default_rng(int(frac * 1000)).exponential(1.0 / lam, len(reqs))
        arrivals = np.cumsum(gaps) - gaps[0]
        wall, lat, st = serve(D.DYSON_MIXED, list(arrivals), inflight, "out")
        sl = sorted(lat)
        out["rates"].append(dict(rate_frac=frac, offered=frac * capacity, value=work / wall,
                                 p50_ms=sl[len(sl) // 2], p99_ms=sl[min(len(sl) - 1, int(0.99 * len(sl)))],
                                 peak_running=st["peak_running"], plans_created=st["plans_created"],
                                 plans_evicted=st["plans_evicted"], fused_requests=st["fused"]))
    # served (mixed) against the plain FP64 per-request results, per lattice: the truncated
    # rank-k diagonal of the 3D slabs is not reproducible at 1e-6 even between two FP64
    # runs (its rounding amplification), so the lattices are reported apart
    per = {}
    for r in reqs:
        name = "x".join(map(str, r["w"].L))
        rel = (np.abs(r["out"] - r["plain"]) / np.abs(r["plain"])).ravel()
        e = per.setdefault(name, dict(requests=0, max=0.0, sites=0, sites_above_1e_6=0, med=[]))
        e["requests"] += 1
        e["max"] = max(e["max"], float(rel.max()))
        e["sites"] += int(rel.size)
        e["sites_above_1e_6"] += int((rel > 1e-6).sum())
        e["med"].append(float(np.median(rel)))
    for e in per.values():
        e["median"] = float(np.median(e.pop("med")))
    out["err_vs_plain"] = per
    return out


def run_serving(a):
    """The serving stream on all five lattices (`--serving`): K in 16..256, --requests."""
    import torch
    from paper_1102_3137_gb300 import build as B
    from paper_1102_3137_gb300 import dyson as D
    B.build()
    D.load()
    torch.cuda.set_device(0)
    out = serving_stream(SERVE_SIZES, 16, 256, a.requests, a.rate_fracs, a.inflight)
    out["metric"] = "serving: site-frequencies/s and p50/p99 request latency (continuous batching)"
    return out


def run_profile_case(a):
    """A small case of a workload for ncu: its first --freqs frequencies in --groups
    frequency groups; one solve (autotuning, graph capture), then one more solve between
    cudaProfilerStart and cudaProfilerStop (profile with --profile-from-start off)."""
    import numpy as np
    import torch
    from paper_1102_3137_gb300 import build as B
    from paper_1102_3137_gb300 import dyson as D
    from paper_1102_3137_gb300 import inputs as I
    B.build()
    D.load()
    dev = torch.device("cuda", 0)
    w = I.WORKLOADS[a.workload]
    K = a.freqs or w.K
    omega, V, sigma, q1 = I.make_inputs(w)
    t = lambda x: torch.from_numpy(np.ascontiguousarray(x)).to(dev)
    om, Vd, sg, qd = t(omega[:K]), t(V), t(sigma[:K]), t(q1)
    prec = D.DYSON_MIXED if a.form == "mixed" else D.DYSON_FP64
    plan = D.Plan(w.L, w.t, w.mu, w.p, w.k, prec, max_freqs=K, freq_groups=a.groups)
    out = torch.zeros((K, w.N), dtype=torch.complex128, device=dev)
    st = torch.zeros(K, dtype=torch.int32, device=dev)
    ss = torch.cuda.current_stream(dev).cuda_stream
    D.dyson_solve(plan.handle, K, om, Vd, sg, qd, out, st, ss)
    torch.cuda.synchronize()
    torch.cuda.profiler.start()
    D.dyson_solve(plan.handle, K, om, Vd, sg, qd, out, st, ss)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    flags = sorted({int(x) for x in st.cpu().numpy()})
    plan.close()
    return dict(profile_case=a.workload, form=a.form, K=K, groups=a.groups, status_flags=flags)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--form", choices=["mixed", "fp64"], default="mixed")
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--cpu-freqs", type=int, default=0,
                    help="frequencies per oracle sample (0: 1 for the 512^2 workload, 16 otherwise)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--quick", action="store_true", help="skip the plain-FP64 and per-launch extras")
    ap.add_argument("--no-serving-sample", action="store_true", help="skip the bounded serving sample")
    ap.add_argument("--serving", action="store_true", help="run the continuous-batching serving stream")
    ap.add_argument("--requests", type=int, default=48)
    ap.add_argument("--inflight", type=int, default=8)
    ap.add_argument("--rate-fracs", type=float, nargs="+", default=[0.5, 0.8, 0.95, 2.0, 4.0])
    ap.add_argument("--profile-case", action="store_true",
                    help="run a small case for ncu (--freqs, --groups) and print no bench line")
    ap.add_argument("--freqs", type=int, default=0, help="--profile-case: first K frequencies (0: all)")
    ap.add_argument("--groups", type=int, default=1, help="--profile-case: frequency groups")
    a = ap.parse_args()
    if a.profile_case:
        print(json.dumps(run_profile_case(a)), flush=True)
        return
    if a.serving:
        print(json.dumps(run_serving(a)), flush=True)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if a.impl == "reference":
        line = run_reference(a, rank, world)
    else:
        if world > 1:
            import torch
            torch.cuda.set_device(local_rank)
            torch.distributed.init_process_group("nccl")
        line = run_ours(a, rank, world, local_rank)
        if world > 1:
            import torch
            torch.distributed.destroy_process_group()
    if line is not None:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
