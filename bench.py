#!/usr/bin/env python
"""Block CUR benchmark on GB300: decompositions per second (one JSON line).

A *step* is one whole Block CUR decomposition of one synthetic matrix held in
HBM: randomized range finder + block leverage scores, block sampling, C/R
gather + U = C^+ A R^+, and the fused residual ||A - CUR||_F.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
                    [--sketch-prec P] [--fit-prec P] [--impl native|reference]

Under torchrun (N > 1) every rank decomposes its own matrix (independent
problems, weak scaling, no collective on the data path); the max over ranks
of the timed region sets the throughput.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import bcur_inputs as bi  # noqa: E402

METRIC = "Block CUR decomps/sec and p50/p99 latency at rel-Frobenius err <= oracle+1e-3"
UNIT = "decomp/s"


def workload(name: str, rank: int = 0) -> bi.Problem:
    if name == "fp32_32768":
        return bi.fp32_32768(seed=1 + 1000 * rank)
    if name == "precision_32768":
        return bi.precision_32768(seed=1 + 1000 * rank)
    if name == "plain_fp64_512x1024":
        return bi.plain_fp64_512x1024(seed=rank)
    if name.startswith("haar_"):   # haar_<n>: the fp32_32768 recipe at n x n
        n = int(name.split("_")[1])
        s = max(16, n // 64)
        return bi.scaled_haar(n, n, s, k=50, p=10, q=2, g_col=16, g_row=16, seed=1 + 1000 * rank,
                              rank=200, noise=1e-4)
    raise SystemExit(f"unknown workload {name}")


# ---------------------------------------------------------------------------
# Clock sampling during the timed region
# ---------------------------------------------------------------------------
class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.proc is None:
            return out
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
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
        os.unlink(self.path)
        if sm:
            out.update(sm_mhz=statistics.median(sm), sm_max_mhz=max(mx), samples=len(sm))
        out["reasons"] = sorted(reasons)
        return out


# ---------------------------------------------------------------------------
# Oracle timing (CPU baseline and the reference arm)
# ---------------------------------------------------------------------------
def oracle_flops(m, n, c, r, l, q):
    """FLOP model of the FP64 oracle's dominant steps, used only when no
    measured full-size / sample ratio is stored: range finder 2(2q+2) m n l;
    SVD-based pinv of C and R ~ 4 m c^2 + 8 c^3 and 4 n r^2 + 8 r^3;
    C^+ A R^+ 2 c m n + 2 c n r; C U R 2 m c r + 2 m r n."""
    return (2 * (2 * q + 2) * m * n * l + 4 * m * c * c + 8 * c ** 3 + 4 * n * r * r + 8 * r ** 3
            + 2 * c * m * n + 2 * c * n * r + 2 * m * c * r + 2 * m * r * n)


def oracle_scale(full: bi.Problem, p: bi.Problem):
    """(factor, how) that turns the oracle's time on the bounded sample p into
    its time on the full problem.  Preferred: the ratio of the two times the
    committed golden script measured in one process on the same host
    (tests/golden/<workload>_oracle.json, seconds_oracle / seconds_sample);
    otherwise the FLOP model above."""
    if p is full:
        return 1.0, "the full problem itself"
    ref_path = os.path.join(ROOT, "tests", "golden", f"{full.name}_oracle.json")
    if os.path.exists(ref_path):
        ref = json.load(open(ref_path))
        if ref.get("seconds_sample") and ref.get("seed") == full.seed and ref.get("k") == full.k:
            f = float(ref["seconds_oracle"]) / float(ref["seconds_sample"])
            return f, (f"measured ratio x{f:.1f}: full-size oracle {ref['seconds_oracle']} s vs "
                       f"this sample {ref['seconds_sample']} s, one process on "
                       f"{ref.get('cores', '?')} host cores (tests/golden/"
                       f"{os.path.basename(ref_path)})")
    c_full = int(np.sum(np.sort(np.diff(full.col_off))[::-1][:full.g_col]))
    r_full = int(np.sum(np.sort(np.diff(full.row_off))[::-1][:full.g_row]))
    cs = int(np.sum(np.sort(np.diff(p.col_off))[::-1][:p.g_col]))
    rs = int(np.sum(np.sort(np.diff(p.row_off))[::-1][:p.g_row]))
    f = oracle_flops(full.m, full.n, c_full, r_full, full.l, full.q) / oracle_flops(
        p.m, p.n, cs, rs, p.l, p.q)
    return f, f"oracle FLOP model x{f:.1f} (no measured ratio stored)"


def time_oracle(full: bi.Problem, steps: int, warmup: int = 0):
    """Time the FP64 oracle on a bounded sample of the workload.  Returns
    (full-size decompositions/s, description, mean seconds per sample run)."""
    import oracle as orc

    p = bi.host_sample(full)
    scale, how = oracle_scale(full, p)
    A = p.matrix()
    om, uc, ur = p.omega(), p.u_col(), p.u_row()
    times = []
    for i in range(warmup + steps):
        t0 = time.perf_counter()
        orc.block_cur(A, p.col_off, p.row_off, p.k, p.q, p.g_col, p.g_row, om, uc, ur)
        dt = time.perf_counter() - t0
        if i >= warmup:
            times.append(dt)
    t = float(np.mean(times))
    sample = (f"FP64 NumPy oracle, whole pipeline on a {p.m}x{p.n} matrix of the same recipe "
              f"({len(p.col_off) - 1}+{len(p.row_off) - 1} blocks of {int(p.col_off[1])}, "
              f"{p.g_col}+{p.g_row} drawn, k={p.k}, p={p.p}, q={p.q}); mean of {steps} runs "
              f"{t:.3f} s; " + (f"the sample is the {full.m}x{full.n} workload itself (no scaling)"
                                if p is full else
                                f"decomps/s of the {full.m}x{full.n} workload by the {how}"))
    return 1.0 / (t * scale), sample, t


# ---------------------------------------------------------------------------
# Native arm
# ---------------------------------------------------------------------------
def roofline_peak(prec: str, peaks: dict, sm_mhz):
    """(bound, peak, unit, source) of the dominant kernel for its precision."""
    if prec == "bf16":
        return "tensor", peaks.get("bf16_tflops_sustained", 1700.0), "TFLOP/s", "measured bf16 sustained"
    if prec == "tf32":
        return ("tensor", peaks.get("bf16_tflops_sustained", 1700.0) / 2.0, "TFLOP/s",
                "measured bf16 sustained x 1/2 (nominal tf32:bf16 ratio)")
    # FP32 FMA on CUDA cores: 152 SMs x 128 lanes x 2 flop x SM clock.
    mhz = peaks.get("sm_max_mhz", 2070.0) if not sm_mhz else sm_mhz
    if prec == "f32":
        return "alu", 152 * 128 * 2 * mhz * 1e6 / 1e12, "TFLOP/s", f"FP32 FMA peak at {mhz:.0f} MHz"
    return "alu", 152 * 2 * 2 * mhz * 1e6 / 1e12, "TFLOP/s", f"FP64 FMA estimate at {mhz:.0f} MHz"


def main_native(args):
    import torch

    import paper_1703_06065_gb300 as pkg

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
    pkg.load()
    p = workload(args.workload, rank)
    # FP32 data: BF16 sketch (re-orthonormalised after every product) and the
    # adaptive split-BF16 fit on tensor cores (split Cholesky-QR; one-term core
    # products and residual, redone with three terms on the device when the
    # error is small); FP64 data stays FP64.
    sp = args.sketch_prec or ("f64" if p.storage == "f64" else "bf16")
    fp = args.fit_prec or ("f64" if p.storage == "f64" else "bf16x3a")
    tdt = torch.float64 if p.storage == "f64" else torch.float32

    # inputs resident in HBM before the timed region; the host draws exactly the
    # matrix the FP64 oracle's stored reference was computed on
    t_gen = time.perf_counter()
    A = torch.from_numpy(p.matrix()).to(dev, tdt)
    t_gen = time.perf_counter() - t_gen
    om = torch.from_numpy(np.ascontiguousarray(p.omega().T)).to(dev, tdt)
    uc = torch.from_numpy(p.u_col()).to(dev)
    ur = torch.from_numpy(p.u_row()).to(dev)
    plan = pkg.Plan(p.m, p.n, p.k, p.p, p.q, p.col_off, p.row_off, p.g_col, p.g_row,
                    dtype=p.storage, sketch_prec=sp, fit_prec=fp)
    Ubuf = torch.empty(plan.c_max, plan.r_max, dtype=tdt, device=dev)
    ebuf = torch.empty(3, dtype=torch.float64, device=dev)

    def step(Ain):
        cs, rs = plan.scores(Ain, om)
        ci, ri, _, _ = plan.sample(cs, rs, uc, ur)
        plan.fit(Ain, ci, ri, U=Ubuf)
        plan.error(Ain, out=ebuf)
        return cs, rs, ci, ri

    def barrier():
        if world > 1:
            import torch.distributed as dist

            dist.barrier()

    for _ in range(args.warmup):
        step(A)
    torch.cuda.synchronize()
    plan.sync_status()
    barrier()
    torch.cuda.synchronize()

    L = pkg.load()
    launches0 = L.bcur_launch_count()
    clocks = Clocks(local)
    clocks.start()
    s = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("bench_timed")  # lets a profiler select the timed steps
    ev0.record(s)
    for _ in range(args.steps):
        step(A)
    ev1.record(s)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    clk = clocks.stop()
    launches = (L.bcur_launch_count() - launches0) // max(args.steps, 1)
    plan.sync_status()
    ms = ev0.elapsed_time(ev1) / args.steps
    e = ebuf.cpu().numpy()
    fit_terms = plan.fit_terms()[0]   # BF16 terms of the fit's core products
    if world > 1:
        import torch.distributed as dist

        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    value = world * 1000.0 / ms

    # -- end to end: inputs from pinned host memory, results read back --------
    e2e = None
    if not args.no_e2e:
        A_h = A.cpu().pin_memory()
        om_h = om.cpu().pin_memory()
        uc_h, ur_h = uc.cpu().pin_memory(), ur.cpu().pin_memory()
        outs = plan.decompose_host(A_h, om_h, uc_h, ur_h)   # allocates the pinned outputs

        def e2e_step():
            # one C-ABI call: H2D of A, Omega and the uniforms, the whole method,
            # D2H of the scores, indices, U and the error
            plan.decompose_host(A_h, om_h, uc_h, ur_h, out=outs)

        torch.cuda.synchronize()
        barrier()
        k2 = max(1, min(args.steps, 3))
        ev0.record(s)
        for _ in range(k2):
            e2e_step()
        ev1.record(s)
        torch.cuda.synchronize()
        plan.sync_status()
        ms2 = ev0.elapsed_time(ev1) / k2
        if world > 1:
            import torch.distributed as dist

            t = torch.tensor([ms2], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms2 = float(t.item())
        h2d = sum(x.numel() * x.element_size() for x in (A_h, om_h, uc_h, ur_h))
        d2h = sum(x.numel() * x.element_size() for x in outs.values())
        e2e = {"value": world * 1000.0 / ms2, "unit": UNIT, "ms_per_step": ms2,
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "api": "bcur_decompose_host (host buffers in, host results out; copies on the "
                      "plan's stream inside the timed region)",
               "matches_device_run": bool(abs(float(outs["err"][1]) - float(e[1])) == 0.0)}
        del A_h, outs

    # -- dominant kernel, timed live ---------------------------------------
    # The tensor-core GEMM's store variant takes most of the step; its largest
    # launch is W = A Q_R of the fit (m x n times n x r).  It is re-run here
    # on the resident A through the C ABI and timed with CUDA events.  The
    # fused residual (sum (A - P Q)^2, one BF16 term) is reported beside it.
    roof = None
    if rank == 0:
        peaks = {}
        try:
            peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        except Exception:
            pass
        r = plan.r_max
        nrep = 3
        if fp.startswith("bf16"):
            # W = A Q_R as the fit ran it: three split terms, or one BF16 term
            # when the adaptive fit kept one
            terms = 1 if fit_terms == 1 else 3
            Ah = A.to(torch.bfloat16)
            Al = (A - Ah.float()).to(torch.bfloat16)
            Q = torch.randn(r, p.n, device=dev, dtype=torch.float32) / float(np.sqrt(p.n))
            Qh = Q.to(torch.bfloat16)
            Ql = (Q - Qh.float()).to(torch.bfloat16)
            Wd = torch.empty(p.m, r, device=dev, dtype=torch.float32)

            def wgemm():
                if terms == 3:
                    pkg.gemm_split(Ah, Al, Qh, Ql, False, True, out=Wd)
                else:
                    pkg.gemm(Ah, Qh, False, True, prec="bf16", out=Wd)

            wgemm()
            torch.cuda.synchronize()
            ev0.record(s)
            for _ in range(nrep):
                wgemm()
            ev1.record(s)
            torch.cuda.synchronize()
            kms = ev0.elapsed_time(ev1) / nrep
            alg = 2.0 * p.m * p.n * r              # the method's flops for W = A Q_R
            mma = terms * alg                      # issued BF16 MMA flops
            achieved = alg / (kms * 1e-3) / 1e12
            peak = peaks.get("bf16_tflops", 1968.0)
            what = "split BF16 (3 terms)" if terms == 3 else "one BF16 term (adaptive fit)"
            roof = {"kernel": f"tc_gemm_kernel<256, BF16, store>: W = A Q_R, {what}",
                    "bound": "tensor", "achieved": round(achieved, 3), "peak": round(peak, 3),
                    "unit": "TFLOP/s", "frac": round(achieved / peak, 4), "traffic": None,
                    "ms": round(kms, 4),
                    "algorithmic": f"2*m*n*r = {alg:.4g} flop per launch (m={p.m}, n={p.n}, "
                                   f"r={r}): the product the method needs, counted once",
                    "tensor_pipe_frac": round(mma / (kms * 1e-3) / 1e12 / peak, 4),
                    "tensor_pipe_note": f"issued BF16 MMA work {terms} x 2*m*n*r = {mma:.4g} "
                                        f"flop ({mma / (kms * 1e-3) / 1e12:.1f} TFLOP/s)",
                    "peak_source": "MEASURED_PEAKS bf16_tflops (burst; kernel timed alone)"}
            del Ah, Al, Q, Qh, Ql, Wd
            Pm = (torch.randn(p.m, r, device=dev) / float(np.sqrt(r))).to(torch.bfloat16)
            Qm = (torch.randn(r, p.n, device=dev) / float(np.sqrt(p.n))).to(torch.bfloat16)
            pkg.residual(A, Pm, Qm, "bf16")
            torch.cuda.synchronize()
            ev0.record(s)
            for _ in range(nrep):
                pkg.residual(A, Pm, Qm, "bf16")
            ev1.record(s)
            torch.cuda.synchronize()
            rms = ev0.elapsed_time(ev1) / nrep
            rfl = 2.0 * p.m * p.n * r
            roof["residual"] = {"kernel": "tc_gemm_kernel<256, BF16, residual>", "ms": round(rms, 4),
                                "achieved": round(rfl / (rms * 1e-3) / 1e12, 3),
                                "frac": round(rfl / (rms * 1e-3) / 1e12 / peak, 4),
                                "algorithmic": f"2*m*n*r = {rfl:.4g} flop per launch"}
            del Pm, Qm
        else:
            Pm = torch.randn(p.m, r, device=dev, dtype=tdt) / float(np.sqrt(r))
            Qm = torch.randn(r, p.n, device=dev, dtype=tdt) / float(np.sqrt(p.n))
            pkg.residual(A, Pm, Qm, fp)
            torch.cuda.synchronize()
            ev0.record(s)
            for _ in range(nrep):
                pkg.residual(A, Pm, Qm, fp)
            ev1.record(s)
            torch.cuda.synchronize()
            kms = ev0.elapsed_time(ev1) / nrep
            flops = 2.0 * p.m * p.n * r
            achieved = flops / (kms * 1e-3) / 1e12
            bound, peak, unit, src = roofline_peak(fp, peaks, clk.get("sm_mhz"))
            roof = {"kernel": "gemm_simt_kernel residual  sum (A - P Q)^2", "bound": bound,
                    "achieved": round(achieved, 3), "peak": round(peak, 3), "unit": unit,
                    "frac": round(achieved / peak, 4), "traffic": None, "ms": round(kms, 4),
                    "algorithmic": f"2*m*n*r = {flops:.4g} flop per launch (m={p.m}, n={p.n}, r={r})",
                    "peak_source": src}
            del Pm, Qm

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, sample, _ = time_oracle(p, steps=1)
        cpu = {"value": v, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
               "sample": sample}

    # per-stage times of one extra step (events between the C-ABI calls)
    stage_ms = None
    if rank == 0:
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
        evs[0].record(s)
        cs_t, rs_t = plan.scores(A, om)
        evs[1].record(s)
        ci_t, ri_t, _, _ = plan.sample(cs_t, rs_t, uc, ur)
        evs[2].record(s)
        plan.fit(A, ci_t, ri_t, U=Ubuf)
        evs[3].record(s)
        plan.error(A, out=ebuf)
        evs[4].record(s)
        torch.cuda.synchronize()
        stage_ms = {nm: round(evs[i].elapsed_time(evs[i + 1]), 3)
                    for i, nm in enumerate(["scores", "sample", "fit", "error"])}

    # accuracy gate against the stored FP64 oracle result for this workload
    gate = None
    ref_path = os.path.join(ROOT, "tests", "golden", f"{p.name}_oracle.json")
    if rank == 0 and os.path.exists(ref_path):
        ref = json.load(open(ref_path))
        if ref.get("seed") == p.seed and ref.get("m") == p.m and ref.get("k") == p.k:
            cs_l, rs_l, ci_l, ri_l = step(A)
            torch.cuda.synchronize()
            ci_l, ri_l = ci_l.cpu().tolist(), ri_l.cpu().tolist()
            csd = np.abs(cs_l.cpu().numpy() - np.asarray(ref["col_scores"]))
            rsd = np.abs(rs_l.cpu().numpy() - np.asarray(ref["row_scores"]))
            gate = {"oracle_rel_err": ref["rel"], "rel_err": float(ebuf[1].item()),
                    "abs_diff": abs(float(ebuf[1].item()) - ref["rel"]),
                    "within_1e-3": abs(float(ebuf[1].item()) - ref["rel"]) <= 1e-3,
                    "col_idx_match": ci_l == ref["col_idx"], "row_idx_match": ri_l == ref["row_idx"],
                    "score_max_rel_diff": float(max(csd.max() / max(ref["col_scores"]),
                                                    rsd.max() / max(ref["row_scores"]))),
                    "source": "tests/golden/" + os.path.basename(ref_path)}

    # DRAM traffic of the roofline kernel from its committed ncu capture, if
    # the kernel source is unchanged since the capture
    if roof is not None:
        tpath = os.path.join(ROOT, "profiles", "tc_gemm_traffic.json")
        if os.path.exists(tpath) and fp.startswith("bf16"):
            import hashlib

            src = open(os.path.join(ROOT, "paper_1703_06065_gb300", "csrc", "gemm_tc.cu"), "rb").read()
            sha = hashlib.sha256(src).hexdigest()
            terms = 1 if fit_terms == 1 else 3
            for tr in json.load(open(tpath)).get("records", []):
                if (tr.get("source_sha256") == sha and tr.get("terms") == terms
                        and tr.get("m") == p.m and tr.get("n") == p.n and tr.get("r") == plan.r_max):
                    roof["traffic"] = tr["dram_bytes_read"] + tr["dram_bytes_write"]
                    roof["traffic_source"] = f"profiles/tc_gemm_traffic.json ({terms} term(s))"

    study = None
    if rank == 0 and p.name == "precision_32768" and not args.no_cpu_baseline:
        study = precision_study(p, dev)

    if rank == 0:
        dtype = sp if sp == fp else f"{sp}/{fp}"
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": dtype, "data": "synthetic",
            "config": single_config(p, sp, fp, world),
            "rel_err": float(e[1]), "fro_err": float(e[0]),
            "accuracy_gate": gate, "stage_ms": stage_ms, "input_generation_s": round(t_gen, 1),
            "clocks": clk, "e2e": e2e, "gpu_launches": int(launches),
            "roofline": roof, "cpu_baseline": cpu,
        }
        if fp.startswith("bf16"):
            line["config"]["fit_terms"] = fit_terms
        if study is not None:
            line["precision_study"] = study
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


def main_reference_batched(args, world):
    """The oracle on random members of the batch (bounded sample per step)."""
    import oracle as orc

    probs = batch_problems(0)
    # W untimed warm-up members, then two timed members per step
    w = max(0, args.warmup)
    idx = batch_oracle_sample(probs, w + 2 * max(1, args.steps))
    times = []
    for j, i in enumerate(idx[: w + 2 * args.steps]):
        p = probs[i]
        A = p.matrix()
        t0 = time.perf_counter()
        orc.block_cur(A, p.col_off, p.row_off, p.k, p.q, p.g_col, p.g_row, p.omega(), p.u_col(),
                      p.u_row())
        if j >= w:
            times.append(time.perf_counter() - t0)
    v = len(times) / sum(times)
    timed = idx[w: w + 2 * args.steps]
    sample = (f"FP64 NumPy oracle, whole pipeline on {len(times)} random members {timed} of the "
              f"512-matrix batch (host-drawn, same recipe; {w} more members as untimed warm-up); "
              f"decomps/s = members / time")
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 / v,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": "batched_biometric", "matrices": BATCH_COUNT},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def precision_study(full: bi.Problem, dev):
    """Per-stage error of each sketch precision (BF16, FP8 with per-row and with
    per-128x128-block scales, split BF16, FP32) and of the adaptive fit against
    the FP64 oracle, on the bounded sample of the workload that the oracle
    decomposes in seconds (bcur_inputs.host_sample: the same recipe at 1/4 the
    size per side, k, p, q unchanged), with the split-BF16 fit:
      - subspace: sin of the largest principal angle between the GPU's top-k
        right (and left) singular subspace and the oracle's;
      - scores: max |l_gpu - l_orc| / max l_orc over both sides;
      - indices: draws equal to the oracle's (per side, in draw order);
      - U: ||U_gpu - U_orc||_F / ||U_orc||_F with the oracle's blocks forced;
      - e: |e_gpu - e_orc| (e = ||A - CUR||_F / ||A||_F)."""
    import torch

    import oracle as orc
    import paper_1703_06065_gb300 as pkg

    p = bi.host_sample(full)
    A = p.matrix()
    om, uc, ur = p.omega(), p.u_col(), p.u_row()
    t0 = time.perf_counter()
    ref = orc.block_cur(A, p.col_off, p.row_off, p.k, p.q, p.g_col, p.g_row, om, uc, ur)
    t_orc = time.perf_counter() - t0
    At = torch.from_numpy(A).to(dev)
    omt = torch.from_numpy(np.ascontiguousarray(om.T)).to(dev, torch.float32)
    uct, urt = torch.from_numpy(uc).to(dev), torch.from_numpy(ur).to(dev)
    ci_o = torch.tensor(ref["col_idx"], dtype=torch.int32, device=dev)
    ri_o = torch.tensor(ref["row_idx"], dtype=torch.int32, device=dev)

    def sin_angle(Xg, Xo):
        q, _ = np.linalg.qr(Xg)
        d = q - Xo @ (Xo.T @ q)
        return float(np.linalg.norm(d, 2))

    out = {"sample": f"{p.m}x{p.n}, k={p.k}, p={p.p}, q={p.q}, {p.g_col}+{p.g_row} blocks of "
                     f"{int(p.col_off[1])}", "oracle_s": round(t_orc, 2),
           "fit": "bf16x3 (keys: sketch precision), bf16x3a for the key sketch/fit"}
    for sp, fp in (("bf16", "bf16x3"), ("fp8", "bf16x3"), ("fp8b", "bf16x3"), ("bf16x3", "bf16x3"),
                   ("f32", "bf16x3"), ("bf16", "bf16x3a")):
        plan = pkg.Plan(p.m, p.n, p.k, p.p, p.q, p.col_off, p.row_off, p.g_col, p.g_row,
                        dtype="f32", sketch_prec=sp, fit_prec=fp)
        cs, rs = plan.scores(At, omt)
        Vt, Ut, _ = plan.factors()
        ci, ri, _, _ = plan.sample(cs, rs, uct, urt)
        U = plan.fit(At, ci_o, ri_o)
        e = plan.error(At)
        plan.sync_status()
        lmax = max(ref["col_scores"].max(), ref["row_scores"].max())
        sd = max(np.abs(cs.cpu().numpy() - ref["col_scores"]).max(),
                 np.abs(rs.cpu().numpy() - ref["row_scores"]).max()) / lmax
        cig, rig = ci.cpu().tolist(), ri.cpu().tolist()
        c, r = ref["U"].shape
        Ug = U.double().cpu().numpy()[:c, :r]
        key = sp if fp == "bf16x3" else f"{sp}/{fp}"
        out[key] = {
            "sin_angle_V": sin_angle(Vt.double().cpu().numpy().T, ref["V_k"]),
            "sin_angle_U": sin_angle(Ut.double().cpu().numpy().T, ref["U_k"]),
            "score_max_rel": float(sd),
            "col_idx_equal": sum(a == b for a, b in zip(cig, ref["col_idx"])),
            "row_idx_equal": sum(a == b for a, b in zip(rig, ref["row_idx"])),
            "U_rel_fro": float(np.linalg.norm(Ug - ref["U"]) / np.linalg.norm(ref["U"])),
            "e_abs_diff": abs(float(e[1].item()) - ref["rel"]),
        }
        if fp == "bf16x3a":
            out[key]["fit_terms"] = plan.fit_terms()[0]
        del plan
    return out


def single_config(p, sp, fp, world):
    """The config object of a single-matrix workload, shared by both arms."""
    a_bytes = p.m * p.n * (8 if p.storage == "f64" else 4)
    return {"workload": p.name, "m": p.m, "n": p.n, "k": p.k, "p": p.p, "q": p.q,
            "block": int(p.col_off[1]), "G_col": int(p.col_off.size - 1),
            "G_row": int(p.row_off.size - 1), "g_col": p.g_col, "g_row": p.g_row,
            "storage": p.storage, "sketch_prec": sp, "fit_prec": fp,
            "l2": (f"inputs larger than L2 (A = {a_bytes / 1e9:.2f} GB)" if a_bytes > 129e6 else
                   f"A = {a_bytes / 1e6:.1f} MB fits in L2 and is not flushed between steps: a "
                   f"latency figure for the small case"),
            "parallelism": f"replicas x{world}"}


def main_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    if args.workload in ("batched_biometric", "serving"):
        main_reference_batched(args, world)
        return
    p = workload(args.workload, 0)
    steps = args.steps
    v, sample, t = time_oracle(p, steps=steps, warmup=args.warmup)
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
        "steps": steps, "warmup": args.warmup, "ms_per_step": 1000.0 * t,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": single_config(p, args.sketch_prec or ("f64" if p.storage == "f64" else "bf16"),
                                args.fit_prec or ("f64" if p.storage == "f64" else "bf16x3a"), world),
        "step_note": "each timed step is one oracle decomposition of the bounded sample named in "
                     "cpu_baseline.sample (ms_per_step is its measured time); value is in "
                     "decompositions/s of the full workload, scaled as that sample states",
        "full_size_ms_per_decomp": 1000.0 / v,
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# Batched workload: 512 uneven biometric-like matrices, every stage one launch
# over the whole batch, the launch sequence replayed from a CUDA graph
# ---------------------------------------------------------------------------
BATCH_COUNT = 512


def batch_problems(rank: int, count: int = BATCH_COUNT):
    """The first `count` matrices of the 512-matrix batch (all of it by default)."""
    return bi.batched_biometric(BATCH_COUNT, seed=3 + 1000 * rank)[:count]


def batch_item(p):
    return dict(m=p.m, n=p.n, k=p.k, p=p.p, block=int(p.col_off[1] - p.col_off[0]),
                g_col=p.g_col, g_row=p.g_row)


def batch_oracle_sample(probs, count: int, seed: int = 7):
    """Indices of a uniform random sample of the batch (fixed seed)."""
    g = np.random.default_rng(seed)
    return sorted(int(i) for i in g.choice(len(probs), size=count, replace=False))


def batch_kernel_model(label: str, probs, items, lp: int = 64):
    """(bound, algorithmic amount per launch, unit) of a batched kernel kind."""
    mn = sum(p.m * p.n for p in probs)
    if label == "sketch_gemm":
        # A_hi read once (2 B), the skinny panel read (2 B) and the FP32 panel
        # written (4 B), averaged over Y = A Omega and Z = A^T Q launches
        byt = sum(2 * p.m * p.n + (2 * lp * (p.m + p.n) + 4 * lp * (p.m + p.n)) / 2 for p in probs)
        return "hbm", byt, "bytes"
    if label == "split":
        return "hbm", 8.0 * mn + sum(4 * p.n * p.l + 2 * 64 * p.n for p in probs), "bytes"
    if label == "w_gemm":
        fl = sum(3 * 2.0 * p.m * p.n * (-(-it["g_row"] * it["block"] // 64) * 64)
                 for p, it in zip(probs, items))
        return "tensor", fl, "flop"
    if label == "residual":
        # one BF16 term (the refinement launch exits at once at these errors):
        # A read once in FP32 is the bound
        return "hbm", 4.0 * mn, "bytes"
    return None, None, None


def main_batched(args):
    import torch

    import paper_1703_06065_gb300 as pkg
    import oracle as orc

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
    pkg.load()
    probs = batch_problems(rank, args.count)
    items = [batch_item(p) for p in probs]
    t_gen = time.perf_counter()
    As = [p.matrix_device(dev) for p in probs]
    oms = [torch.from_numpy(np.ascontiguousarray(p.omega().T)).to(dev, torch.float32) for p in probs]
    ucs = [torch.from_numpy(p.u_col()).to(dev) for p in probs]
    urs = [torch.from_numpy(p.u_row()).to(dev) for p in probs]
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t_gen
    bfp = args.fit_prec or "bf16x3a"
    batch = pkg.Batch(items, q=2, fit_prec=bfp)
    graph = not args.no_graph

    def barrier():
        if world > 1:
            import torch.distributed as dist

            dist.barrier()

    for _ in range(args.warmup):
        out = batch.run(As, oms, ucs, urs, want_u=True, use_graph=graph)
    torch.cuda.synchronize()
    batch.sync_status()
    barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    s = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("bench_timed")
    ev0.record(s)
    for _ in range(args.steps):
        out = batch.run(As, oms, ucs, urs, want_u=True, use_graph=graph)
    ev1.record(s)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    clk = clocks.stop()
    batch.sync_status()
    ms = ev0.elapsed_time(ev1) / args.steps
    if world > 1:
        import torch.distributed as dist

        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    B = len(probs)
    value = world * B * 1000.0 / ms
    launches = batch.launches_per_run
    terms1 = sum(1 for t in batch.fit_terms() if t == 1)  # items that kept one BF16 term

    # -- end to end: every matrix from pinned host memory, results read back ---
    e2e = None
    if not args.no_e2e:
        try:
            A_h = [a.cpu().pin_memory() for a in As]
            A_d = [torch.empty_like(a) for a in As]
            res_h = {k: [torch.empty(v.shape, dtype=v.dtype).pin_memory() for v in out[k]]
                     for k in ("col_scores", "row_scores", "col_idx", "row_idx", "err", "U")}

            def e2e_step():
                for d, h in zip(A_d, A_h):
                    d.copy_(h, non_blocking=True)
                o = batch.run(A_d, oms, ucs, urs, want_u=True, use_graph=False)
                for k, lst in res_h.items():
                    for h, d in zip(lst, o[k]):
                        h.copy_(d, non_blocking=True)

            e2e_step()
            torch.cuda.synchronize()
            barrier()
            k2 = max(1, min(args.steps, 2))
            ev0.record(s)
            for _ in range(k2):
                e2e_step()
            ev1.record(s)
            torch.cuda.synchronize()
            ms2 = ev0.elapsed_time(ev1) / k2
            h2d = sum(x.numel() * x.element_size() for x in A_h)
            d2h = sum(x.numel() * x.element_size() for lst in res_h.values() for x in lst)
            e2e = {"value": world * B * 1000.0 / ms2, "unit": UNIT, "ms_per_step": ms2,
                   "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                   "note": "A of all 512 matrices copied from pinned host memory each step; "
                           "Omega and the uniforms stay resident"}
            del A_h, A_d, res_h
        except RuntimeError as exc:  # host memory for the pinned copies
            e2e = {"value": None, "unit": UNIT, "h2d_bytes_per_step": None,
                   "d2h_bytes_per_step": None, "skipped": str(exc)[:200]}

    # -- per-kernel times from one profiled eager run, dominant kernel ------
    roof, stages = None, None
    if rank == 0:
        peaks = {}
        try:
            peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        except Exception:
            pass
        batch.profile(True)
        batch.run(As, oms, ucs, urs, want_u=True, use_graph=False)
        torch.cuda.synchronize()
        steps = batch.profile_steps()
        batch.profile(False)
        stages, counts = {}, {}
        for lab, t in steps:
            stages[lab] = stages.get(lab, 0.0) + t
            counts[lab] = counts.get(lab, 0) + 1
        stages = {k: round(v, 3) for k, v in sorted(stages.items(), key=lambda kv: -kv[1])}
        dom = next(iter(stages))
        bound, amount, unit = batch_kernel_model(dom, probs, items)
        if bound is not None:
            per_launch_ms = stages[dom] / counts[dom]
            if bound == "hbm":
                achieved = amount / (per_launch_ms * 1e-3) / 1e9
                peak = peaks.get("hbm_gbs", 6789.0)
                roof = {"bound": "hbm", "unit": "GB/s", "peak_source": "MEASURED_PEAKS hbm_gbs"}
            else:
                achieved = amount / (per_launch_ms * 1e-3) / 1e12
                peak = peaks.get("bf16_tflops_sustained", 1721.0)
                roof = {"bound": "tensor", "unit": "TFLOP/s",
                        "peak_source": "MEASURED_PEAKS bf16_tflops_sustained (timed inside the step)"}
            roof.update(kernel=f"{dom} ({counts[dom]} launches per step)",
                        achieved=round(achieved, 3), peak=round(peak, 3),
                        frac=round(achieved / peak, 4), traffic=None, ms=round(per_launch_ms, 4),
                        algorithmic=f"{amount:.4g} {unit} per launch (model in bench.py)")
            # DRAM traffic of this kernel kind from its committed ncu capture,
            # valid while the kernel sources are the ones it was taken on
            tpath = os.path.join(ROOT, "profiles", f"batched_{dom}_traffic.json")
            if os.path.exists(tpath) and len(probs) == BATCH_COUNT:
                tr = json.load(open(tpath))
                if all(tr.get("sha256", {}).get(f) == _sha(f) for f in tr.get("sha256", {})):
                    roof["traffic"] = tr["bytes_per_launch"]
                    roof["traffic_source"] = os.path.relpath(tpath, ROOT)

    # -- sampled accuracy gate: the FP64 oracle on random members ---------
    gate, cpu = None, None
    if rank == 0:
        idx = batch_oracle_sample(probs, 3 if args.no_cpu_baseline else 4)
        diffs, ok_idx, t_orc = [], True, []
        for i in idx:
            p = probs[i]
            A64 = As[i].double().cpu().numpy()
            t0 = time.perf_counter()
            ref = orc.block_cur(A64, p.col_off, p.row_off, p.k, p.q, p.g_col, p.g_row, p.omega(),
                                p.u_col(), p.u_row())
            t_orc.append(time.perf_counter() - t0)
            e_gpu = float(out["err"][i][1].item())
            diffs.append(abs(e_gpu - ref["rel"]))
            ok_idx &= (out["col_idx"][i].cpu().tolist() == list(ref["col_idx"])
                       and out["row_idx"][i].cpu().tolist() == list(ref["row_idx"]))
        gate = {"members": idx, "max_abs_diff_rel_err": max(diffs),
                "within_1e-3": max(diffs) <= 1e-3, "indices_match": bool(ok_idx),
                "source": "FP64 oracle run on the same device-drawn matrices (host copies)"}
        if world == 1 and not args.no_cpu_baseline:
            v = len(t_orc) / sum(t_orc)
            cpu = {"value": v, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                   "sample": f"FP64 NumPy oracle, whole pipeline on {len(idx)} random members "
                             f"{idx} of the 512-matrix batch; {sum(t_orc):.2f} s in total, "
                             f"decomps/s = members / time"}

    if rank == 0:
        mn = sum(p.m * p.n for p in probs)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": f"bf16/{bfp}", "data": "synthetic",
            "config": {"workload": "batched_biometric" if B == BATCH_COUNT
                       else f"batched_biometric[:{B}]", "matrices": B,
                       "sum_mn": mn, "storage": "f32", "sketch_prec": "bf16", "fit_prec": bfp,
                       "fit_terms_1": terms1,
                       "q": 2, "cuda_graph": graph,
                       "l2": f"inputs larger than L2 (A total {4 * mn / 1e9:.1f} GB)",
                       "parallelism": f"replicas x{world}"},
            "ms_per_decomp": ms / B, "accuracy_gate": gate, "stage_ms": stages,
            "input_generation_s": round(t_gen, 1), "clocks": clk, "e2e": e2e,
            "gpu_launches": int(launches), "roofline": roof, "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


# ---------------------------------------------------------------------------
# Serving workload: Poisson arrivals, continuous batching on several streams
# ---------------------------------------------------------------------------
def main_serving(args):
    import torch

    import paper_1703_06065_gb300 as pkg
    from paper_1703_06065_gb300 import serve

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pkg.load()
    reqs = bi.serving_requests(args.rate, args.duration, seed=4 + 1000 * rank)
    sfp = args.fit_prec or "bf16x3a"
    srv = serve.Server(hbm_budget=args.hbm_budget, lanes=3, max_batch=128, heavy_lanes=2,
                       max_heavy_batch=16, draw=bi.generators.request_inputs_device,
                       fit_prec=sfp)
    # warm-up: the kernels, the allocator and the plan builders on the first requests
    warm = bi.serving_requests(args.rate, 0.05, seed=99)
    srv.run(warm, realtime=False)
    # tile widths of shape classes first met during the timed run are the
    # fixed ones: no autotuner measurements inside the timed region
    os.environ["BCUR_AUTOTUNE"] = "0"
    clocks = Clocks(local)
    clocks.start()
    t0 = time.perf_counter()
    done = srv.run(reqs, realtime=True, timeout=max(600.0, 20 * args.duration))
    wall = time.perf_counter() - t0
    clk = clocks.stop()
    st = serve.latency_stats(done)
    jobs = {}
    for kind, nreq, a, b in srv.jobs:
        j = jobs.setdefault(kind, {"groups": 0, "requests": 0, "gpu_s": 0.0})
        j["groups"] += 1
        j["requests"] += nreq
        j["gpu_s"] += b - a
    for j in jobs.values():
        j["gpu_s"] = round(j["gpu_s"], 3)
        j["mean_group"] = round(j["requests"] / max(1, j["groups"]), 1)

    # baseline: the plain one-at-a-time FP32 path (CUDA cores) on a sample of
    # the same request stream, each request alone on the GPU
    base = None
    if not args.no_cpu_baseline:
        sample = [r for r in reqs if not r.heavy][:40] + [r for r in reqs if r.heavy][:4]
        times = []
        for r in sample:
            p = r.problem
            A, om, uc, ur = bi.generators.request_inputs_device(p, dev)
            plan = pkg.Plan(p.m, p.n, p.k, p.p, p.q, p.col_off, p.row_off, p.g_col, p.g_row,
                            dtype="f32", sketch_prec="f32", fit_prec="f32")
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            pkg.decompose(plan, A, om, uc, ur)
            torch.cuda.synchronize()
            times.append(time.perf_counter() - t1)
            del plan, A
        nl = sum(1 for r in sample if not r.heavy)
        tl, th = float(np.mean(times[:nl])), float(np.mean(times[nl:]))
        frac_h = sum(r.heavy for r in reqs) / len(reqs)
        cap = 1.0 / ((1 - frac_h) * tl + frac_h * th)
        base = {"path": "plain FP32 plan, one request at a time (CUDA cores)",
                "light_ms": round(1e3 * tl, 2), "heavy_ms": round(1e3 * th, 2),
                "capacity_decomps_per_s": round(cap, 1),
                "sample": f"{nl} light + {len(sample) - nl} heavy requests of the stream"}
    if rank == 0:
        line = {
            "metric": METRIC, "value": st["decomps_per_s"], "unit": UNIT, "n_gpus": world,
            "steps": 1, "warmup": 1, "ms_per_step": 1e3 * wall, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": f"bf16/{sfp}", "data": "synthetic",
            "config": {"workload": "serving", "rate_per_s": args.rate, "duration_s": args.duration,
                       "fit_prec": sfp,
                       "requests": len(reqs), "heavy": int(sum(r.heavy for r in reqs)),
                       "lanes": "3 light + 2 heavy streams, batched groups (up to 128 "
                                "light, 16 heavy)",
                       "hbm_budget_gb": args.hbm_budget / 1e9},
            "latency": {k: round(v, 3) for k, v in st.items() if k.endswith("_ms")},
            "completed": st["requests"], "wall_s": round(wall, 2), "groups": jobs,
            "clocks": clk, "baseline_one_at_a_time": base,
        }
        print(json.dumps(line), flush=True)


def _sha(rel: str) -> str:
    import hashlib

    return hashlib.sha256(open(os.path.join(ROOT, rel), "rb").read()).hexdigest()


# ---------------------------------------------------------------------------
# Kernel-only mode: one tensor-core GEMM of the fit, for profiling
# ---------------------------------------------------------------------------
def main_kernel(args):
    """W = A Q_R as the fit computes it (split BF16, three terms, or one BF16
    term as the adaptive fit keeps it: --terms) on random operands of the
    given shape, timed with CUDA events; prints one JSON line."""
    import torch

    import paper_1703_06065_gb300 as pkg

    m, n, r = (int(x) for x in args.shape.split(","))
    dev = torch.device("cuda", 0)
    g = torch.Generator(device=dev)
    g.manual_seed(5)
    A = torch.randn(m, n, device=dev, generator=g)
    Ah = A.to(torch.bfloat16)
    Al = (A - Ah.float()).to(torch.bfloat16)
    del A
    Q = torch.randn(r, n, device=dev, generator=g) / float(np.sqrt(n))
    Qh = Q.to(torch.bfloat16)
    Ql = (Q - Qh.float()).to(torch.bfloat16)
    del Q
    W = torch.empty(m, r, device=dev)
    terms = 1 if args.terms == 1 else 3

    def run():
        if terms == 3:
            pkg.gemm_split(Ah, Al, Qh, Ql, False, True, out=W)
        else:
            pkg.gemm(Ah, Qh, False, True, prec="bf16", out=W)

    for _ in range(args.warmup):
        run()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("bench_timed")
    e0.record()
    for _ in range(args.steps):
        run()
    e1.record()
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    what = "split BF16 (3 terms)" if terms == 3 else "one BF16 term"
    print(json.dumps({"kernel": f"tc_gemm_kernel<256, BF16, store> {what}",
                      "m": m, "n": n, "r": r, "terms": terms, "ms": ms,
                      "bf16_mma_tflops": terms * 2.0 * m * n * r / (ms * 1e-3) / 1e12}),
          flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default="fp32_32768")
    ap.add_argument("--sketch-prec", default=None)
    ap.add_argument("--fit-prec", default=None)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--count", type=int, default=BATCH_COUNT,
                    help="batched workload: decompose only the first COUNT matrices (profiling)")
    ap.add_argument("--rate", type=float, default=2000.0, help="serving: arrivals per second")
    ap.add_argument("--duration", type=float, default=60.0,
                    help="serving: seconds of arrivals")
    ap.add_argument("--hbm-budget", type=float, default=160e9, help="serving: admission budget")
    ap.add_argument("--kernel", default=None, choices=["wgemm"],
                    help="time one kernel instead of the workload (profiling)")
    ap.add_argument("--shape", default="32768,32768,8192", help="kernel mode: m,n,r")
    ap.add_argument("--terms", type=int, default=3, choices=[1, 3],
                    help="kernel mode: BF16 terms of W = A Q_R")
    ap.add_argument("--no-graph", action="store_true",
                    help="batched workload: launch eagerly instead of replaying a CUDA graph")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "native":
        args.warmup = 3
    if args.kernel:
        main_kernel(args)
    elif args.impl == "reference":
        main_reference(args)
    elif args.workload == "batched_biometric":
        main_batched(args)
    elif args.workload == "serving":
        main_serving(args)
    else:
        main_native(args)


if __name__ == "__main__":
    main()
