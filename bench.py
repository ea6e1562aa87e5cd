"""Benchmark of the sFISTA hot path on one GB300 (or N replicas).

Workload (one "step"): one full structured-FISTA solve (Alg. 2) of the
512 x 512 problem with a 31 x 31 rotated anisotropic Gaussian PSF
(sigma_x 3, sigma_y 1, 30 deg), reflective boundary, r = 3 Kronecker terms,
lambda = 0.005, 1 % noise, 200 iterations, on seeded synthetic data that
stands in for the paper's IR-Tools test images.  The metric is sFISTA
iterations per second; the result of each measured form is checked against
the FP64 oracle (relative Frobenius error) in the same run.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line.  For N > 1 launch under torch.distributed.run: every
rank solves its own copy (replicas, no collective) and the value is the
total over ranks divided by the slowest rank's time.
"""
import argparse
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "sFISTA iters/s and op TFLOP/s, mixed vs FP32 form, at <=1e-4 rel err vs FP64"
WORKLOAD = "512x512 reflexive, 31x31 rotated Gaussian PSF (3,1,30deg), r=3, lambda=0.005, 1% noise, 200 its"
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12   # 152 SMs x 128 FP32 lanes x FMA x 2.07 GHz
# Kernels per sFISTA iteration by operator form (a solve adds an input
# check, the state initialisation and the output conversion).
# Kernel launches per iteration (the persistent form: one launch per solve).
KERNELS_PER_ITER = {"banded": 4, "banded_fused": 2, "gemm_band": 4, "gemm_dense": 4}
# DRAM bytes (read + write) per launch of a form's dominant kernel, from an
# ncu capture of the current kernel code on this workload (the summary in
# profiles/ gives the command); forms without one report null.
TRAFFIC = {
    # one 200-iteration solve (one launch) of band_solve_fused, 64-row tiles on 512-thread blocks, cold L2
    "fp32:banded_persistent:0": {"bytes": 7209472 + 9216,
                                 "source": "profiles/solve_fused_fp32_cfg2_512_r3.md (ncu dram__bytes_read.sum + "
                                           "dram__bytes_write.sum, one 200-iteration launch)"},
}


def one_launch_fused(m, n):
    """The library's rule for the persistent form: the fused one-launch solver
    when m, n are multiples of 4 and every 32 x 32 tile has one of the two
    co-resident blocks per SM, else the two-pass persistent solver."""
    import torch
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    return m % 4 == 0 and n % 4 == 0 and -(-m // 32) * -(-n // 32) <= 2 * sms
# Stated tolerances against the FP64 oracle: relative Frobenius error, and for
# the split-precision forms also |PSNR - PSNR_oracle| <= 0.01 dB.  The
# single-product BF16 / TF32 forms have no stated tolerance: they are reported
# with their error and meets_tol = None.
TOL = {"fp32": 1e-5, "bf16x3": 1e-4, "tf32x3": 1e-4}
DPSNR_TOL = {"bf16x3": 0.01, "tf32x3": 0.01}


def meets_tol(prec, err, dpsnr=None):
    """True / False against the form's stated tolerance, None where it has none."""
    if prec not in TOL:
        return None
    ok = err <= TOL[prec]
    if prec in DPSNR_TOL:
        ok = ok and dpsnr is not None and abs(dpsnr) <= DPSNR_TOL[prec]
    return bool(ok)
DTYPE = {"fp32": "f32", "bf16x3": "bf16", "tf32x3": "tf32", "bf16": "bf16", "tf32": "tf32"}
NPROD = {"bf16x3": 3, "tf32x3": 3, "bf16": 1, "tf32": 1}
STAGES = ["fwd_right", "fwd_left+residual", "adj_right", "adj_left+prox+momentum"]


def _form(f):
    """'prec:op[+tune][+refN]' -> (prec, op, tune)."""
    prec, op = f.split(":") if ":" in f else (f, "auto")
    return prec, op.split("+")[0], "+tune" in op


def _refine(f):
    """The k_ref of a 'prec:op+refN' form (FP32 residual every N-th iteration), else 0."""
    m = re.search(r"\+ref(\d+)", f)
    return int(m.group(1)) if m else 0


def mma_flops_per_stage(info, m, n, r, prec, op):
    """Tensor-core flops each GEMM stage issues: 128 x 128 tiles, K blocks of 128 bytes,
    K range per M tile [m0 + lo, m0 + 127 + hi] (band) or [0, K) (dense); x3 for split."""
    kb = 64 if prec.startswith("bf16") else 32
    align = 8 if prec.startswith("bf16") else 4
    lo = info["lo"]
    wA, wB = info["band_right"], info["band_left"]

    def nkb(m0, K, lo_, w):
        if op == "gemm_dense":
            return (K + kb - 1) // kb
        klo = max(0, m0 + lo_) // align * align
        khi = min(K, m0 + 128 + lo_ + w - 1)
        return (khi - klo + kb - 1) // kb if khi > klo else 0

    tile = 2.0 * 128 * 128 * kb * NPROD[prec]
    mt_n, mt_m = (n + 127) // 128, (m + 127) // 128
    st0 = sum(nkb(t * 128, n, lo["A"], wA) for t in range(mt_n)) * r * ((m + 127) // 128) * tile
    st1 = sum(nkb(t * 128, m, lo["B"], wB) for t in range(mt_m)) * r * ((n + 127) // 128) * tile
    st2 = sum(nkb(t * 128, n, lo["AT"], wA) for t in range(mt_n)) * r * ((m + 127) // 128) * tile
    st3 = sum(nkb(t * 128, m, lo["BT"], wB) for t in range(mt_m)) * r * ((n + 127) // 128) * tile
    return [st0, st1, st2, st3]


def replica_throughput(local_ms, iters, steps, world, device="cpu"):
    """Replicas, no data-path collective: every rank solved `steps` problems of `iters`
    iterations in local_ms.  Returns (whole-job iterations/s, slowest rank's ms) using a
    MAX all-reduce of the times (the only collective, outside the timed region)."""
    ms = float(local_ms)
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return world * iters * steps / (ms / 1e3), ms


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def _problem():
    from paper_1901_00913_gb300 import workloads as W
    return W.config2()


def _observation_gpu(pr, torch):
    """b = exact blur (library kernel) + scaled noise draw, on the device."""
    from paper_1901_00913_gb300 import api, workloads as W
    x = torch.from_numpy(pr.x_true.astype(np.float32)).cuda()
    bx = api.sfista_blur(pr.psf, x, pr.bc)
    bxn = bx.double().cpu().numpy()
    b = bxn + W.noise_scale(bxn, pr.noise, pr.noise_level)
    return torch.from_numpy(b.astype(np.float32)).cuda()


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev):
        self.dev = dev
        self.proc = None
        # Raw samples: $SFISTA_CLOCKS_DIR if set, else the temp directory.
        self.path = os.path.join(os.environ.get("SFISTA_CLOCKS_DIR") or tempfile.gettempdir(),
                                 "clocks_bench_%d.csv" % os.getpid())

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            self.proc.wait()
            self.f.close()

    def summary(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [t.strip() for t in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo), or None."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return None


def oracle_reference(pr, b32, iters, L, single_thread_iters=10):
    """FP64 oracle solve on the host cores; returns (X, seconds, threads, one-thread s/iteration)."""
    import oracle
    from oracle import kron, _native
    cr, cc = pr.centre
    ka = kron.kron_approx(pr.psf, cr, cc, pr.x_true.shape[0], pr.x_true.shape[1], pr.bc, pr.r)
    t0 = time.perf_counter()
    X = oracle.sfista(b32.astype(np.float64), ka, L, pr.lam, iters)
    dt = time.perf_counter() - t0
    nthreads = _native.threads()
    one = None
    if single_thread_iters > 0:
        _native.set_threads(1)
        t0 = time.perf_counter()
        oracle.sfista(b32.astype(np.float64), ka, L, pr.lam, single_thread_iters)
        one = (time.perf_counter() - t0) / single_thread_iters
        _native.set_threads(nthreads)
    return X, dt, nthreads, one


def run_reference(args):
    """--impl reference: the FP64 oracle as the reference arm, on the host cores."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import kron, _native
    import oracle
    pr = _problem()
    cr, cc = pr.centre
    bx = oracle.blur(pr.x_true, pr.psf, cr, cc, pr.bc)
    from paper_1901_00913_gb300 import workloads as W
    b = (bx + W.noise_scale(bx, pr.noise, pr.noise_level)).astype(np.float32).astype(np.float64)
    n = pr.x_true.shape[0]
    ka = kron.kron_approx(pr.psf, cr, cc, n, n, pr.bc, pr.r)
    L = 1.0
    sample = 20   # iterations of the 200-iteration solve per step
    for _ in range(args.warmup):
        oracle.sfista(b, ka, L, pr.lam, sample)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.sfista(b, ka, L, pr.lam, sample)
    dt = time.perf_counter() - t0
    v = sample * args.steps / dt
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "iters/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "form": "FP64 CPU oracle",
                                            "global_batch": 1, "seq_len": 0, "parallelism": "replicas"},
            "cpu_baseline": {"value": v, "unit": "iters/s", "cores": _native.threads(), "kind": "oracle",
                             "sample": "%d of the 200 iterations per step" % sample},
            "e2e": {"value": v, "unit": "iters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_large(args, torch):
    """--workload cfg3: 2048^2, r=5, 63x63 PSF, 300 iterations per step; every form is
    checked against the FP64 oracle on the first `--check-iters` iterations."""
    from paper_1901_00913_gb300 import api, build, workloads as W
    import oracle
    from oracle import kron
    build.build()
    pr = W.config3()
    n, iters, r = pr.x_true.shape[0], pr.iters, pr.r
    db = _observation_gpu(pr, torch)
    b_host = db.cpu().numpy()
    s0 = api.Sfista(pr.psf, (n, n), pr.bc, r, prec="fp32", op="banded", lipschitz_tol=1e-8, lipschitz_maxit=300)
    L = s0.info()["lipschitz"]
    s0.close()
    cr, cc = pr.centre
    ka = kron.kron_approx(pr.psf, cr, cc, n, n, pr.bc, r)
    t0 = time.perf_counter()
    Xref = oracle.sfista(b_host.astype(np.float64), ka, L, pr.lam, args.check_iters)
    cpu_s = time.perf_counter() - t0
    peaks, peak_src_name = _peaks()
    forms = {}
    for f in args.forms.split(","):
        prec, op, tune = _form(f)
        s = api.Sfista(pr.psf, (n, n), pr.bc, r, prec=prec, op=op, lipschitz=L)
        tuned = s.tune(iters=5) if tune else None
        Xc = s.solve_device(db, pr.lam, args.check_iters).cpu().numpy()
        err = oracle.rel_fro(Xc, Xref)
        out = torch.empty_like(db)
        for _ in range(args.warmup):
            s.solve_device(db, pr.lam, iters, out=out)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ms = 0.0
        with Clocks(0) as clk:
            for _ in range(args.steps):
                ev0.record()
                s.solve_device(db, pr.lam, iters, out=out, sync=False)
                ev1.record()
                torch.cuda.synchronize()
                ms += ev0.elapsed_time(ev1)
        api.sfista_sync(s.ctx)
        info = s.info()
        op = info["op"]
        sm = [float(x) for x in api.sfista_time_stages(s.ctx, db, pr.lam, 5)]
        v = iters * args.steps / (ms / 1e3)
        wA, wB = info["band_right"], info["band_left"]
        alg = [2.0 * wA * r * n * n, 2.0 * wB * r * n * n] * 2
        if op.startswith("gemm"):
            work = mma_flops_per_stage(info, n, n, r, prec, op)
            bf16 = peaks.get("bf16_tflops", 1900.0)
            peak = bf16 if prec.startswith("bf16") else bf16 * (1.1 / 2.25)
            bound = "tensor"
        else:
            work = {"banded": alg, "banded_fused": [alg[0] + alg[1], 0, alg[2] + alg[3], 0]}.get(op, [sum(alg), 0, 0, 0])
            peak, bound = FP32_PEAK_TFLOPS, "alu"
        dom = int(np.argmax(sm))
        dur_ms = ms / (args.steps * iters) * sm[dom] / sum(sm)   # in-region share, as in the main workload
        ach = work[dom] / (dur_ms / 1e3) / 1e12
        forms[f] = {
            "resolved_op": op, "tuned": tuned,
            "iters_per_s": v, "rel_err_vs_oracle_first_%d_its" % args.check_iters: err, "stage_ms": sm,
            "dominant_stage": STAGES[dom], "roofline": {"bound": bound, "achieved_tflops": ach, "peak": peak,
                                                        "frac": ach / peak, "duration_us": dur_ms * 1e3},
            "op_tflops_executed": sum(work) * v / 1e12, "op_tflops_algorithmic": sum(alg) * v / 1e12,
            "dense_equiv_tflops": 8.0 * r * n ** 3 * v / 1e12, "clocks": clk.summary()}
        s.close()
    line = {"metric": METRIC, "workload": "2048x2048 reflexive, 63x63 mixture+Moffat PSF, r=5, lambda=0.002, "
            "0.5% noise, 300 its", "unit": "iters/s", "steps": args.steps, "warmup": args.warmup,
            "forms": forms, "cpu_baseline": {"value": args.check_iters / cpu_s, "unit": "iters/s",
                                             "kind": "oracle", "sample": "%d iterations" % args.check_iters},
            "peaks": {"source": peak_src_name, "bf16_tflops": peaks.get("bf16_tflops")}}
    print(json.dumps(line), flush=True)


def run_batched(args, torch):
    """--workload cfg4: 64 problems of uneven size / PSF / rank, 150 iterations, grouped launches."""
    from paper_1901_00913_gb300 import api, build, workloads as W
    import oracle
    from oracle import kron
    build.build()
    probs = W.config4()
    iters = probs[0].iters
    d_bs, Ls = [], []
    for pr in probs:
        db = _observation_gpu(pr, torch)
        d_bs.append(db)
        s0 = api.Sfista(pr.psf, pr.x_true.shape, pr.bc, pr.r, prec="fp32", op="banded", lipschitz_tol=1e-7,
                        lipschitz_maxit=200)
        Ls.append(s0.info()["lipschitz"])
        s0.close()
    lams = [pr.lam for pr in probs]
    # oracle on a sample: the three smallest problems and the largest
    order = sorted(range(len(probs)), key=lambda k: probs[k].x_true.size * probs[k].r)
    sample = order[:3] + order[-1:]
    refs = {}
    t0 = time.perf_counter()
    for k in sample:
        pr = probs[k]
        cr, cc = pr.centre
        ka = kron.kron_approx(pr.psf, cr, cc, pr.x_true.shape[0], pr.x_true.shape[1], pr.bc, pr.r)
        refs[k] = oracle.sfista(d_bs[k].double().cpu().numpy(), ka, Ls[k], lams[k], iters)
    cpu_s = time.perf_counter() - t0
    total_px = sum(pr.x_true.size for pr in probs)
    forms = {}
    for f in args.forms.split(","):
        prec, op, _ = _form(f)
        solvers = [api.Sfista(pr.psf, pr.x_true.shape, pr.bc, pr.r, prec=prec, op=op, lipschitz=L)
                   for pr, L in zip(probs, Ls)]
        # autotuned tiles: each problem's term chunking (and, for op auto, its form)
        t_tune = time.perf_counter()
        for sv in solvers:
            sv.tune(iters=3)
        t_tune = time.perf_counter() - t_tune
        batch = api.Batch(solvers)
        t_bt = time.perf_counter()
        batch_tuning = batch.tune(iters=5)     # the grouped launches' shared-memory plan
        t_tune += time.perf_counter() - t_bt
        outs = [torch.empty_like(d) for d in d_bs]
        for _ in range(args.warmup):
            batch.solve(d_bs, lams, iters, outs=outs)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ms = 0.0
        with Clocks(0) as clk:
            for _ in range(args.steps):
                ev0.record()
                batch.solve(d_bs, lams, iters, outs=outs, sync=False)
                ev1.record()
                torch.cuda.synchronize()
                ms += ev0.elapsed_time(ev1)
        api.sfista_batch_sync(batch.handle)
        errs = {probs[k].name: oracle.rel_fro(outs[k].cpu().numpy(), refs[k]) for k in sample}
        # the same problems one at a time (no grouping), for comparison
        t_single = 0.0
        for sv, db, lam in zip(solvers, d_bs, lams):
            sv.solve_device(db, lam, iters)
        ev0.record()
        for sv, db, lam in zip(solvers, d_bs, lams):
            sv.solve_device(db, lam, iters, sync=False)
        ev1.record()
        torch.cuda.synchronize()
        t_single = ev0.elapsed_time(ev1)
        v = len(probs) * iters * args.steps / (ms / 1e3)
        forms[prec + ":" + op] = {"problem_iters_per_s": v, "batch_iters_per_s": v / len(probs),
                                  "megapixel_iters_per_s": total_px * iters * args.steps / (ms / 1e3) / 1e6,
                                  "sequential_problem_iters_per_s": len(probs) * iters / (t_single / 1e3),
                                  "max_rel_err_sample": max(errs.values()), "rel_err_sample": errs,
                                  "autotune_s": t_tune, "batch_tuning": batch_tuning,
                                  "clocks": clk.summary()}
        batch.close()
        for sv in solvers:
            sv.close()
    line = {"metric": METRIC, "workload": "64 problems, n in {256..1024}, PSF 15-41 px mixtures, r in 1..4, "
            "reflexive, lambda 0.005, 1% noise, 150 its, grouped launches + CUDA graph, autotuned term chunks",
            "unit": "problem-iters/s",
            "steps": args.steps, "warmup": args.warmup, "forms": forms,
            "cpu_baseline": {"value": len(sample) * iters / cpu_s, "unit": "problem-iters/s", "kind": "oracle",
                             "sample": "4 problems (3 smallest, largest), full 150 its"}}
    print(json.dumps(line), flush=True)


def run_unrolled(args, torch):
    """--workload cfg5: reverse mode of the unrolled 50-iteration solve (512^2, r=3, checkpoint every 10).

    One step = sfista_unrolled_fwd (forward with checkpoints) + the loss gradient
    2 (X_50 - X_true) + sfista_unrolled_bwd (gradients for b, lambda, A_i, B_i).
    Parity: the GPU backward is fed the oracle's dl/dX_50 and compared with the
    oracle's FP64 reverse mode (dense factors).
    """
    from paper_1901_00913_gb300 import api, build, workloads as W
    from oracle import adjoint, kron
    build.build()
    pr = W.config5()
    K, ck = pr.iters, pr.extra["ckpt_every"]
    m, n = pr.x_true.shape
    r = pr.r
    db = _observation_gpu(pr, torch)
    s0 = api.Sfista(pr.psf, (m, n), pr.bc, r, prec="fp32", op="banded")
    L = s0.info()["lipschitz"]
    s0.close()
    xt = torch.from_numpy(pr.x_true.astype(np.float32)).cuda()
    cr, cc = pr.centre
    ka = kron.kron_approx(pr.psf, cr, cc, m, n, pr.bc, r)
    Bf, Af = kron.dense_factors(ka)
    b64 = db.double().cpu().numpy()
    t0 = time.perf_counter()
    Xo = adjoint.unrolled_forward(b64, Af, Bf, L, pr.lam, K)[0]
    gXo = 2.0 * (Xo - pr.x_true)
    ob, ol, oA, oB = adjoint.unrolled_grad(b64, Af, Bf, L, pr.lam, K, gXo)
    cpu_s = time.perf_counter() - t0

    def rel(a, b):
        return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))

    nseg = (K + ck - 1) // ck
    forms = {}
    for f in args.forms.split(","):
        prec, op, _ = _form(f)
        s = api.Sfista(pr.psf, (m, n), pr.bc, r, prec=prec, op=op, lipschitz=L)
        ckpt = torch.empty(2 * nseg, m, n, dtype=torch.float64, device="cuda")
        X = torch.empty_like(db)
        gX = torch.empty_like(db)
        gb = torch.empty_like(db)
        gA = torch.empty(r, n, n, device="cuda")
        gB = torch.empty(r, m, m, device="cuda")
        # parity against the oracle's reverse mode, on the oracle's dl/dX
        api.sfista_unrolled_fwd(s.ctx, db, pr.lam, K, ck, ckpt, X)
        gl = api.sfista_unrolled_bwd(s.ctx, db, pr.lam, K, ck, ckpt,
                                     torch.from_numpy(gXo.astype(np.float32)).cuda(), gb, gA, gB)
        torch.cuda.synchronize()
        errs = {"X": rel(X.cpu().numpy(), Xo), "g_b": rel(gb.cpu().numpy(), ob),
                "g_lambda": abs(gl - ol) / abs(ol), "g_A": rel(gA.cpu().numpy(), oA), "g_B": rel(gB.cpu().numpy(), oB)}
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        fwd_ms = bwd_ms = 0.0
        for it in range(args.warmup + args.steps):
            ev[0].record()
            api.sfista_unrolled_fwd(s.ctx, db, pr.lam, K, ck, ckpt, X)
            ev[1].record()
            torch.sub(X, xt, out=gX).mul_(2.0)
            api.sfista_unrolled_bwd(s.ctx, db, pr.lam, K, ck, ckpt, gX, gb, gA, gB)
            ev[2].record()
            torch.cuda.synchronize()
            if it >= args.warmup:
                fwd_ms += ev[0].elapsed_time(ev[1])
                bwd_ms += ev[1].elapsed_time(ev[2])
        with Clocks(0) as clk:
            for _ in range(2):
                api.sfista_unrolled_fwd(s.ctx, db, pr.lam, K, ck, ckpt, X)
                torch.sub(X, xt, out=gX).mul_(2.0)
                api.sfista_unrolled_bwd(s.ctx, db, pr.lam, K, ck, ckpt, gX, gb, gA, gB)
            torch.cuda.synchronize()
        step_ms = (fwd_ms + bwd_ms) / args.steps
        forms[prec + ":" + op] = {"unrolled_iters_per_s": K / (step_ms / 1e3), "ms_per_step": step_ms,
                                  "fwd_ms": fwd_ms / args.steps, "bwd_ms": bwd_ms / args.steps,
                                  "rel_err_vs_oracle_reverse_mode": errs,
                                  "meets_tol": errs["X"] <= 1e-5 and max(errs[k] for k in errs if k != "X") <= 1e-4,
                                  "clocks": clk.summary()}
        s.close()
    line = {"metric": METRIC, "workload": "512x512 reflexive, 31x31 rotated Gaussian PSF, r=3, lambda=0.005, 50 "
            "unrolled its, checkpoint every 10; forward + backward for b, lambda, A_i, B_i",
            "unit": "unrolled iters/s (forward + backward)", "steps": args.steps, "warmup": args.warmup,
            "forms": forms,
            "cpu_baseline": {"value": K / cpu_s, "unit": "unrolled iters/s (forward + backward)", "kind": "oracle",
                             "cores": os.cpu_count(), "sample": "one full 50-iteration FP64 forward + reverse mode "
                             "(numpy BLAS, dense factors)"}}
    print(json.dumps(line), flush=True)


def run_example2(args, torch):
    """--workload ex2: the Example 2 stand-in set (defocus and shake blur at three
    levels, Gaussian / Laplace / multiplicative noise), 18 problems of 256^2,
    r = 5, 50 iterations each.  Per case and form: iterations/s, the error
    against the FP64 oracle on the first --check-iters iterations, the
    restoration error eta = ||X - x|| / ||x|| and residual gamma = ||A X - b|| /
    ||b|| (exact blur) of Sec. 4, and the singular-value decay of P and P_bar."""
    from paper_1901_00913_gb300 import api, build, diagnostics as D, workloads as W
    import oracle
    from oracle import kron, _native
    build.build()
    cases = W.example2_cases()
    forms = {}
    cpu_s, cpu_its = 0.0, 0
    decay = {}
    for f in args.forms.split(","):
        prec, op, tune = _form(f)
        rows = {}
        rates = []
        for pr in cases:
            n = pr.x_true.shape[0]
            xt = torch.from_numpy(pr.x_true.astype(np.float32)).cuda()
            bx = api.sfista_blur(pr.psf, xt, pr.bc).double().cpu().numpy()
            b = (bx + W.noise_of_kind(pr.extra["noise"], bx, pr.noise, pr.noise_level)).astype(np.float32)
            db = torch.from_numpy(b).cuda()
            s = api.Sfista(pr.psf, (n, n), pr.bc, pr.r, prec=prec, op=op)
            if tune:
                s.tune(iters=5)
            info = s.info()
            L = info["lipschitz"]
            Xc = s.solve_device(db, pr.lam, args.check_iters).cpu().numpy()
            if pr.name not in decay:
                cr, cc = pr.centre
                ka = kron.kron_approx(pr.psf, cr, cc, n, n, pr.bc, pr.r)
                t0 = time.perf_counter()
                Xo = oracle.sfista(b.astype(np.float64), ka, L, pr.lam, args.check_iters)
                cpu_s += time.perf_counter() - t0
                cpu_its += args.check_iters
                decay[pr.name] = {"P": D.decay_ratios(D.psf_singular_values(pr.psf)),
                                  "P_bar": D.decay_ratios(info["sigma"]), "ref": Xo}
            err = oracle.rel_fro(Xc, decay[pr.name]["ref"])
            out = torch.empty_like(db)
            for _ in range(args.warmup):
                s.solve_device(db, pr.lam, pr.iters, out=out)
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record()
            for _ in range(args.steps):
                s.solve_device(db, pr.lam, pr.iters, out=out, sync=False)
            ev1.record()
            torch.cuda.synchronize()
            v = pr.iters * args.steps / (ev0.elapsed_time(ev1) / 1e3)
            rates.append(v)
            res = api.sfista_blur(pr.psf, out, pr.bc) - db
            eta = float(torch.linalg.norm(out.double() - xt.double()) / torch.linalg.norm(xt.double()))
            gamma = float(torch.linalg.norm(res.double()) / torch.linalg.norm(db.double()))
            rows[pr.name] = {"op": info["op"], "iters_per_s": v,
                             "rel_err_vs_oracle_first_%d_its" % args.check_iters: err,
                             "eta": eta, "gamma": gamma, "psf": list(pr.psf.shape),
                             "sigma_decay": {"P": decay[pr.name]["P"], "P_bar": decay[pr.name]["P_bar"]}}
            s.close()
        forms[f] = {"mean_iters_per_s": float(np.mean(rates)), "min_iters_per_s": float(np.min(rates)),
                    "max_rel_err": max(r["rel_err_vs_oracle_first_%d_its" % args.check_iters]
                                       for r in rows.values()), "cases": rows}
    # The same 18 problems as FP32 batches, two ways: all 18 in one batch (its
    # tiles outnumber the co-resident blocks: grouped launches), and groups
    # whose tiles fit as co-resident blocks (one launch of the fused solver
    # each); plus the batch tuner's own comparison of the two plans on one
    # such group.
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    solvers, dbs, lams, tiles = [], [], [], []
    for pr in cases:
        n = pr.x_true.shape[0]
        xt = torch.from_numpy(pr.x_true.astype(np.float32)).cuda()
        bx = api.sfista_blur(pr.psf, xt, pr.bc).double().cpu().numpy()
        b = (bx + W.noise_of_kind(pr.extra["noise"], bx, pr.noise, pr.noise_level)).astype(np.float32)
        dbs.append(torch.from_numpy(b).cuda())
        solvers.append(api.Sfista(pr.psf, (n, n), pr.bc, pr.r, prec="fp32", op="banded"))
        lams.append(pr.lam)
        tiles.append((-(-n // 32)) ** 2)
    fit_groups, cur, used = [], [], 0
    for i, t in enumerate(tiles):
        if cur and used + t > 2 * sms:
            fit_groups.append(cur)
            cur, used = [], 0
        cur.append(i)
        used += t
    fit_groups.append(cur)
    iters = cases[0].iters
    singles = [sv.solve_device(db, lam, iters) for sv, db, lam in zip(solvers, dbs, lams)]
    for name, groups in (("fp32:batched_all", [list(range(len(cases)))]), ("fp32:batched_one_launch", fit_groups)):
        batches = [api.Batch([solvers[i] for i in g]) for g in groups]
        outs = []
        for _ in range(args.warmup):
            outs = [bt.solve([dbs[i] for i in g], [lams[i] for i in g], iters) for bt, g in zip(batches, groups)]
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        for _ in range(args.steps):
            for bt, g, og in zip(batches, groups, outs):
                bt.solve([dbs[i] for i in g], [lams[i] for i in g], iters, outs=og, sync=False)
        ev1.record()
        torch.cuda.synchronize()
        diff = max(float(torch.max(torch.abs(X - singles[i]))) for g, og in zip(groups, outs) for i, X in zip(g, og))
        forms[name] = {"problem_iters_per_s": len(cases) * iters * args.steps / (ev0.elapsed_time(ev1) / 1e3),
                       "groups": [len(g) for g in groups],
                       "one_launch": all(sum(tiles[i] for i in g) <= 2 * sms for g in groups),
                       "max_abs_diff_vs_single_solves": diff}
        if name == "fp32:batched_one_launch":
            forms[name]["batch_tune_first_group"] = batches[0].tune(iters=10)
        for bt in batches:
            bt.close()
    for sv in solvers:
        sv.close()
    line = {"metric": METRIC, "workload": "Example 2 stand-in: 18 problems 256x256, defocus / shake blur x 3 levels "
            "x gauss / laplace / multiplicative noise (1%), reflexive, r=5, lambda=0.005, 50 its",
            "unit": "iters/s", "steps": args.steps, "warmup": args.warmup, "forms": forms,
            "cpu_baseline": {"value": cpu_its / cpu_s, "unit": "iters/s", "kind": "oracle",
                             "cores": _native.threads(), "sample": "%d iterations of each of the 18 problems"
                             % args.check_iters}}
    print(json.dumps(line), flush=True)


def _fft_len(L):
    """Smallest 2^a 3^b 5^c >= L (sizes cuFFT handles with its fast radices)."""
    best = 1 << (L - 1).bit_length()
    a = 1
    while a < 2 * L:
        b = a
        while b < 2 * L:
            c = b
            while c < best:
                if c >= L:
                    best = c
                c *= 5
            b *= 3
        a *= 2
    return best


def _corr_lines(torch, X, T, lo, bc, summed):
    """1-D factor applications along the last axis of X (lines of length n):
    out_k[.., c] = sum_j T[k, j] * ext(X)[.., c + lo + j], ext the zero (bc 0) or
    half-sample reflected (bc 1) extension, as circular correlations of length
    N >= n + w - 1 (so no wrap-around) by real FFTs.  summed: the sum over k,
    else one output per k."""
    n, (r, w) = X.shape[-1], T.shape
    L = n + w - 1
    N = _fft_len(L)
    t = torch.arange(L, device=X.device) + lo
    if bc == 1:
        t = torch.where(t < 0, -1 - t, torch.where(t >= n, 2 * n - 1 - t, t))
    ok = (t >= 0) & (t < n)
    E = torch.index_select(X, -1, t.clamp(0, n - 1)) * ok.to(X.dtype)
    Tf = torch.fft.rfft(T.to(X.dtype), n=N).conj()
    shape = (r,) + (1,) * (X.dim() - (2 if summed else 1)) + (Tf.shape[-1],)
    prod = torch.fft.rfft(E, n=N) * Tf.reshape(shape)
    if summed:
        prod = prod.sum(0)
    return torch.fft.irfft(prod, n=N)[..., :n]


def fft_kron_apply(torch, Y, C, cr, D, cc, bc):
    """sum_k B_k Y A_k^T (Sec. 2's matrix form of the Kronecker sum) with every
    1-D factor applied as the paper's structured product: toep (bc 0) or
    toep + hank (bc 1) of the profile, i.e. a correlation of the extended line
    with the reversed profile, computed by FFT.  Y (m, n); C (r, p) column
    profiles (left factors B_k, centre cr); D (r, q) row profiles (right
    factors A_k, centre cc)."""
    p, q = C.shape[1], D.shape[1]
    Z = _corr_lines(torch, Y, D.flip(-1), cc - (q - 1), bc, False)               # (r, m, n): Y A_k^T
    out = _corr_lines(torch, Z.transpose(-1, -2), C.flip(-1), cr - (p - 1), bc, True)   # (n, m)
    return out.transpose(-1, -2)


def run_fft(args, torch):
    """The operator A_s applied once, three ways: the library's banded FP32 form
    (the automatic FP32 choice), its BF16x3 tensor-core form, and the FFT
    structured product (cuFFT through torch.fft, FP32, unfused, replayed as a
    CUDA graph).  Timed with CUDA events over back-to-back applications; error
    of each against the FP64 oracle's operator on the same input."""
    from paper_1901_00913_gb300 import api, build, workloads as W
    import oracle
    from oracle import kron
    build.build()
    api.load()
    res = {}
    for name, cfg in (("cfg2", W.config2), ("cfg3", W.config3)):
        pr = cfg()
        n = pr.x_true.shape[0]
        cr, cc = pr.centre
        X = torch.from_numpy(pr.x_true.astype(np.float32)).cuda()
        ka = kron.kron_approx(pr.psf, cr, cc, n, n, pr.bc, pr.r)
        t0 = time.perf_counter()
        Yo = oracle.kron_apply(pr.x_true, ka)
        cpu_s = time.perf_counter() - t0
        forms = {}
        s32 = api.Sfista(pr.psf, (n, n), pr.bc, pr.r, prec="fp32", op="auto", lipschitz=1.0)
        C, D = s32.profiles()
        Cd, Dd = torch.from_numpy(C).float().cuda(), torch.from_numpy(D).float().cuda()

        # The FFT form's ~14 torch operations replayed as one CUDA graph, so
        # its time is device time (no per-operation host dispatch).
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            for _ in range(3):
                fft_kron_apply(torch, X, Cd, cr, Dd, cc, pr.bc)
        torch.cuda.current_stream().wait_stream(side)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            Yfft = fft_kron_apply(torch, X, Cd, cr, Dd, cc, pr.bc)

        def fft_form():
            graph.replay()
            return Yfft

        sbf = api.Sfista(pr.psf, (n, n), pr.bc, pr.r, prec="bf16x3", op="gemm_band", lipschitz=1.0)
        out = torch.empty_like(X)
        cands = [("fp32 banded (%s)" % s32.info()["op"], lambda: s32.apply(X, out=out, sync=False)),
                 ("bf16x3 tcgen05 gemm_band", lambda: sbf.apply(X, out=out, sync=False)),
                 ("fp32 FFT structured product (cuFFT, one CUDA graph)", fft_form)]
        for label, fn in cands:
            for _ in range(3):
                Yg = fn()
            torch.cuda.synchronize()
            reps = 50 if n <= 512 else 10
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                Yg = fn()
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            Yg = fn()
            torch.cuda.synchronize()
            forms[label] = {"us_per_application": 1e3 * ms, "applications_per_s": 1e3 / ms,
                            "rel_err_vs_fp64_oracle": oracle.rel_fro(Yg.double().cpu().numpy(), Yo)}
        s32.close()
        sbf.close()
        res[name] = {"workload": "%s: %dx%d, %dx%d PSF, r=%d, reflexive" % (pr.name, n, n, pr.psf.shape[0],
                                                                              pr.psf.shape[1], pr.r),
                     "forms": forms, "oracle_cpu_s": cpu_s}
    print(json.dumps({"metric": "operator applications/s (A_s once) by form", "workload": "fft",
                      "unit": "applications/s", "data": "synthetic", "timing": "CUDA events, back-to-back, warm L2",
                      "configs": res}), flush=True)


GOLDEN = os.path.join(ROOT, "tests", "golden")


def _summary_errors(X, ref, sfx=""):
    """Relative errors of X against a stored oracle summary (tests/golden): over the seeded sampled
    pixels, and the CountSketch estimate of the whole image's relative Frobenius error."""
    from paper_1901_00913_gb300 import workloads as W
    X = np.asarray(X, dtype=np.float64)
    idx, vals = ref["idx" + sfx], ref["vals" + sfx]
    d = X.ravel()[idx] - vals
    sampled = float(np.sqrt(np.mean(d * d)) / np.sqrt(np.mean(vals * vals)))
    seed = int(ref["sketch_seed"]) + (int(ref["k" + sfx]) if sfx else 0)
    est = float(np.linalg.norm(W.count_sketch(X, len(ref["sketch" + sfx]), seed) - ref["sketch" + sfx])
                / float(ref["x_norm" + sfx]))
    return sampled, est


def _solve_rate(s, db, lam, iters, steps, warmup, torch):
    out = torch.empty_like(db)
    for _ in range(warmup):
        s.solve_device(db, lam, iters, out=out)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    for _ in range(steps):
        s.solve_device(db, lam, iters, out=out, sync=False)
    ev1.record()
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    return iters * steps / (ms / 1e3), ms / steps, out


def _even_smooth(need):
    """The FFT form's transform length: the smallest even 2^a 3^b 5^c >= need."""
    best = None
    a = 2
    while a < 4 * need:
        b = a
        while b < 4 * need:
            c = b
            while c < 4 * need:
                if c >= need and (best is None or c < best):
                    best = c
                c *= 5
            b *= 3
        a *= 2
    return best


def fft_bytes_per_iter(info_fft, m, n):
    """Algorithmic DRAM bytes of one FFT-form iteration (two operator applications, three passes
    each): pass A reads the (extended) rows and writes their half spectra, pass B reads them and the
    kernel spectrum and writes the filtered half spectra, pass C reads those and writes the output
    with its epilogue (residual: B read; Step 1 + 3: Y_k, X_{k-1} read, X_k, Y_{k+1} written as
    double-float pairs, the FP32 operand copy written)."""
    N1, N2, er = info_fft["N1"], info_fft["N2"], info_fft["ext_rows"]
    H2 = N2 // 2 + 1
    spec = 8.0 * H2
    fwd = 4.0 * er * n + spec * er + spec * er + spec * N1 + spec * m + spec * m + (4 + 4) * m * n
    adj = 4.0 * m * n + spec * m + spec * m + spec * N1 + spec * m + spec * m + (16 + 16 + 4) * m * n
    return fwd + adj


def config3_section(args, torch, peaks):
    """The 2048^2 workload (r = 5, 63 x 63 mixture + Moffat PSF, 300 iterations): every form's
    iterations/s and its error against the stored 300-iteration FP64 oracle result
    (tests/golden/config3_oracle_300.npz).  The CPU-baseline leg forms the observation with the
    oracle's exact blur (the stored result was computed from that b) and times one oracle iteration."""
    import oracle
    from oracle import kron
    from paper_1901_00913_gb300 import api, workloads as W
    ref = np.load(os.path.join(GOLDEN, "config3_oracle_300.npz"))
    pr = W.config3()
    n, r, iters = 2048, pr.r, int(ref["iters"])
    cr, cc = pr.centre
    t0 = time.perf_counter()
    bx = oracle.blur(pr.x_true, pr.psf, cr, cc, pr.bc)
    b = (bx + W.noise_scale(bx, pr.noise, pr.noise_level)).astype(np.float32)
    ka = kron.kron_approx(pr.psf, cr, cc, n, n, pr.bc, r)
    t1 = time.perf_counter()
    oracle.sfista(b.astype(np.float64), ka, float(ref["L"]), pr.lam, 1)
    cpu_it_s = 1.0 / (time.perf_counter() - t1)
    blur_s = t1 - t0
    db = torch.from_numpy(b).cuda()
    L = float(ref["L"])
    steps = max(1, min(args.steps, 3))
    sus = peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops", 1700.0))
    forms = {}
    for f in ("fp32:auto+tune", "fp32:fft", "bf16x3:gemm_band", "bf16x3:gemm_dense", "tf32x3:gemm_band"):
        prec, op, tune = _form(f)
        s = api.Sfista(pr.psf, (n, n), pr.bc, r, prec=prec, op=op, lipschitz=L)
        tuned = s.tune(iters=3) if tune else None
        v, ms, out = _solve_rate(s, db, pr.lam, iters, steps, 2, torch)
        X = out.cpu().numpy()
        sampled, est = _summary_errors(X, ref)
        dpsnr = oracle.psnr(X, pr.x_true) - float(ref["psnr"])
        info = s.info()
        rop = info["op"]
        sm = [float(x) for x in api.sfista_time_stages(s.ctx, db, pr.lam, 3)]
        dom = int(np.argmax(sm))
        dur_ms = ms / iters * sm[dom] / sum(sm)
        wA, wB = info["band_right"], info["band_left"]
        alg = 4.0 * r * (wA + wB) * n * n
        row = {"resolved_op": rop, "iters_per_s": v, "rel_err_sampled": sampled, "rel_err_sketch": est,
               "dpsnr_db": dpsnr, "meets_tol": meets_tol(prec, max(sampled, est), dpsnr),
               "op_tflops_algorithmic": alg * v / 1e12, "stage_ms": sm}
        if rop.startswith("gemm"):
            work = mma_flops_per_stage(info, n, n, r, prec, rop)
            peak = sus if prec.startswith("bf16") else sus * (1.1 / 2.25)
            ach = work[dom] / (dur_ms / 1e3) / 1e12
            row["roofline"] = {"bound": "tensor", "stage": STAGES[dom], "achieved": ach, "peak": peak,
                               "frac": ach / peak, "unit": "TFLOP/s",
                               "peak_source": "bf16_tflops_sustained of MEASURED_PEAKS.json" +
                               ("" if prec.startswith("bf16") else " x 1.1/2.25")}
            row["dense_equiv_tflops"] = 8.0 * r * n ** 3 * v / 1e12
        elif rop == "fft":
            fi = {"N1": _even_smooth(n + pr.psf.shape[0] - 1), "N2": _even_smooth(n + pr.psf.shape[1] - 1),
                  "ext_rows": n + pr.psf.shape[0] - 1}
            row["roofline"] = {"bound": "hbm", "achieved": fft_bytes_per_iter(fi, n, n) * v / 1e9,
                               "peak": peaks.get("hbm_gbs"), "unit": "GB/s (whole iteration, algorithmic bytes)"}
            row["roofline"]["frac"] = row["roofline"]["achieved"] / row["roofline"]["peak"]
        else:
            row["roofline"] = {"bound": "alu", "achieved": alg * v / 1e12, "peak": FP32_PEAK_TFLOPS,
                               "frac": alg * v / 1e12 / FP32_PEAK_TFLOPS, "unit": "TFLOP/s (whole iteration)"}
        if tuned is not None:
            row["tuned"] = tuned
        forms[f] = row
        s.close()
    # Alg. 1 on the exact blur (the paper's comparison system): its rate and the ratio
    # t(sFISTA) / t(FISTA) of Sec. 4's tables for the fastest sFISTA form that holds its tolerance.
    se = api.Sfista(pr.psf, (n, n), pr.bc, r, exact=True, lipschitz_tol=1e-6, lipschitz_maxit=200)
    ve, _, _ = _solve_rate(se, db, pr.lam, iters, steps, 2, torch)
    se.close()
    held = [k for k, v in forms.items() if v["meets_tol"] is True]
    best = max(held or list(forms), key=lambda k: forms[k]["iters_per_s"])
    return {"workload": "2048x2048 reflexive, 63x63 mixture+Moffat PSF, r=5, lambda=0.002, 0.5% noise, 300 its",
            "unit": "iters/s", "steps": steps, "forms": forms, "best_form": best,
            "exact_blur_fista": {"iters_per_s": ve, "tratio": ve / forms[best]["iters_per_s"],
                                 "note": "tratio = t(sFISTA) / t(FISTA on the exact blur), Sec. 4"},
            "reference": "stored 300-iteration FP64 oracle result (tests/golden/config3_oracle_300.npz)",
            "cpu_baseline": {"value": cpu_it_s, "unit": "iters/s", "kind": "oracle", "cores": _cores(),
                             "sample": "1 of the 300 iterations (the oracle's exact blur of b: %.1f s)" % blur_s}}


def config4_section(args, torch):
    """The batched workload (64 problems 256^2..1024^2, PSF 15-41 px, r 1..4, 150 iterations) as one
    batch per form; the checked problem of every size class against the stored FP64 oracle results
    (tests/golden/config4_oracle_150.npz), whose observations the CPU-baseline leg forms with the
    oracle's exact blur."""
    import oracle
    from paper_1901_00913_gb300 import api, workloads as W
    ref = np.load(os.path.join(GOLDEN, "config4_oracle_150.npz"))
    probs = W.config4()
    iters = probs[0].iters
    checked = {int(ref["k%d" % j]): j for j in range(int(ref["count"]))}
    d_bs, Ls = [], []
    t0 = time.perf_counter()
    for k, pr in enumerate(probs):
        if k in checked:
            cr, cc = pr.centre
            bx = oracle.blur(pr.x_true, pr.psf, cr, cc, pr.bc)
            d_bs.append(torch.from_numpy((bx + W.noise_scale(bx, pr.noise, pr.noise_level)).astype(np.float32)).cuda())
            Ls.append(float(ref["L%d" % checked[k]]))
        else:
            xt = torch.from_numpy(pr.x_true.astype(np.float32)).cuda()
            bx = api.sfista_blur(pr.psf, xt, pr.bc).double().cpu().numpy()
            d_bs.append(torch.from_numpy((bx + W.noise_scale(bx, pr.noise, pr.noise_level)).astype(np.float32)).cuda())
            s0 = api.Sfista(pr.psf, pr.x_true.shape, pr.bc, pr.r, prec="fp32", op="banded", lipschitz_tol=1e-7,
                            lipschitz_maxit=200)
            Ls.append(s0.info()["lipschitz"])
            s0.close()
    prep_s = time.perf_counter() - t0
    lams = [pr.lam for pr in probs]
    steps = max(1, min(args.steps, 3))
    forms = {}
    for f in ("fp32:banded", "bf16x3:gemm_band"):
        prec, op, _ = _form(f)
        solvers = [api.Sfista(pr.psf, pr.x_true.shape, pr.bc, pr.r, prec=prec, op=op, lipschitz=L)
                   for pr, L in zip(probs, Ls)]
        for sv in solvers:
            sv.tune(iters=2)
        batch = api.Batch(solvers)
        batch.tune(iters=3)
        outs = [torch.empty_like(d) for d in d_bs]
        for _ in range(2):
            batch.solve(d_bs, lams, iters, outs=outs)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        for _ in range(steps):
            batch.solve(d_bs, lams, iters, outs=outs, sync=False)
        ev1.record()
        torch.cuda.synchronize()
        api.sfista_batch_sync(batch.handle)
        v = len(probs) * iters * steps / (ev0.elapsed_time(ev1) / 1e3)
        errs = {}
        for k, j in checked.items():
            sampled, est = _summary_errors(outs[k].cpu().numpy(), ref, str(j))
            errs[probs[k].name] = max(sampled, est)
        worst = max(errs.values())
        forms[f] = {"problem_iters_per_s": v, "max_rel_err_checked": worst, "rel_err_checked": errs,
                    "meets_tol": meets_tol(prec, worst, 0.0)}
        batch.close()
        for sv in solvers:
            sv.close()
    a, b = forms["bf16x3:gemm_band"], forms["fp32:banded"]
    return {"workload": "64 problems, n in {256..1024}, PSF 15-41 px mixtures, r in 1..4, reflexive, "
            "lambda 0.005, 1% noise, 150 its, one batch per form", "unit": "problem-iters/s", "steps": steps,
            "forms": forms,
            "mixed_beats_fp32_at_tolerance": bool(a["meets_tol"] and b["meets_tol"] and
                                                  a["problem_iters_per_s"] > b["problem_iters_per_s"]),
            "reference": "stored 150-iteration FP64 oracle results of one problem per size class "
                         "(tests/golden/config4_oracle_150.npz); errors are max(sampled, sketched)",
            "prep_s": prep_s}


def wide_section(args, torch, peaks):
    """512^2 with a 127 x 127 PSF (p about n / 4), r = 3, 200 iterations: the regime where the FFT
    form's cost (independent of the PSF width) beats the band forms'.  Each form's error against
    the FP64 oracle on the first 10 iterations; the CPU-baseline leg forms the observation with the
    oracle's exact blur and runs those 10 oracle iterations."""
    import oracle
    from oracle import kron
    from paper_1901_00913_gb300 import api, workloads as W
    pr = W.wide_psf()
    n, r, iters, check = 512, pr.r, pr.iters, 10
    cr, cc = pr.centre
    bx = oracle.blur(pr.x_true, pr.psf, cr, cc, pr.bc)
    b = (bx + W.noise_scale(bx, pr.noise, pr.noise_level)).astype(np.float32)
    ka = kron.kron_approx(pr.psf, cr, cc, n, n, pr.bc, r)
    db = torch.from_numpy(b).cuda()
    s0 = api.Sfista(pr.psf, (n, n), pr.bc, r, prec="fp32", op="banded", lipschitz_tol=1e-8, lipschitz_maxit=300)
    L = s0.info()["lipschitz"]
    s0.close()
    t0 = time.perf_counter()
    Xo = oracle.sfista(b.astype(np.float64), ka, L, pr.lam, check)
    cpu_s = time.perf_counter() - t0
    steps = max(1, min(args.steps, 5))
    forms = {}
    for f in ("fp32:auto+tune", "fp32:banded", "fp32:fft", "bf16x3:gemm_band"):
        prec, op, tune = _form(f)
        s = api.Sfista(pr.psf, (n, n), pr.bc, r, prec=prec, op=op, lipschitz=L)
        tuned = s.tune(iters=5) if tune else None
        err = oracle.rel_fro(s.solve_device(db, pr.lam, check).cpu().numpy(), Xo)
        v, _, _ = _solve_rate(s, db, pr.lam, iters, steps, 3, torch)
        forms[f] = {"resolved_op": s.info()["op"], "iters_per_s": v,
                    "rel_err_vs_oracle_first_%d_its" % check: err}
        if tuned is not None:
            forms[f]["tuned_whole_iteration_ms"] = {e["op"] + ("" if not e["chunk"] else ":%d" % e["chunk"]): e["ms"]
                                                    for e in tuned if e["stage"] == -1}
        s.close()
    return {"workload": "512x512 reflexive, 127x127 mixture+Moffat PSF, r=3, lambda=0.005, 1% noise, 200 its",
            "unit": "iters/s", "steps": steps, "forms": forms,
            "cpu_baseline": {"value": check / cpu_s, "unit": "iters/s", "kind": "oracle", "cores": _cores(),
                             "sample": "%d of the 200 iterations" % check}}


def _cores():
    from oracle import _native
    return _native.threads()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--forms", default="fp32:auto+tune,fp32:banded_fused,fp32:banded,fp32:banded_persistent,bf16x3:gemm_band,bf16x3:gemm_band+tune,tf32x3:gemm_band,bf16:gemm_band,tf32:gemm_band,bf16x3:gemm_band+ref1,bf16:gemm_band+ref1",
                    help="comma list of prec:op forms to measure")
    ap.add_argument("--workload", default="cfg2", choices=["cfg2", "cfg3", "cfg4", "cfg5", "ex2", "fft"])
    ap.add_argument("--check-iters", type=int, default=10)
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the 2048^2, batched and wide-PSF sections of the default line")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload != "cfg2":
        import torch
        if args.workload == "fft":
            return run_fft(args, torch)
        if args.forms.startswith("fp32:auto+tune,fp32:banded_fused,fp32:banded,fp32:banded_persistent"):
            args.forms = {"cfg3": "fp32:auto+tune,fp32:banded_fused,fp32:banded,bf16x3:auto+tune,bf16x3:gemm_band,"
                                  "tf32x3:gemm_band,bf16x3:gemm_dense",
                          "cfg4": "fp32:banded,bf16x3:gemm_band,tf32x3:gemm_band",
                          "cfg5": "fp32:banded_fused,fp32:banded",
                          "ex2": "fp32:auto,bf16x3:auto"}[args.workload]
        run = {"cfg3": run_large, "cfg4": run_batched, "cfg5": run_unrolled, "ex2": run_example2}[args.workload]
        return run(args, torch)

    import torch
    from paper_1901_00913_gb300 import api, build
    import oracle

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    if rank == 0 or world == 1:
        build.build()
    if world > 1:
        dist.barrier()
    api.load()

    pr = _problem()
    n = pr.x_true.shape[0]
    iters = pr.iters
    db = _observation_gpu(pr, torch)
    b_host = db.cpu().numpy()

    # L once, in FP64 on the device (the library's own estimate); all forms share it.
    s0 = api.Sfista(pr.psf, (n, n), pr.bc, pr.r, prec="fp32", op="banded")
    L = s0.info()["lipschitz"]
    s0.close()

    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")   # 256 MB > L2
    forms = [(f,) + _form(f) for f in args.forms.split(",")]
    results = {}
    peaks, peak_src_name = _peaks()
    for form, prec, op, tune in forms:
        s = api.Sfista(pr.psf, (n, n), pr.bc, pr.r, prec=prec, op=op, lipschitz=L, refine_every=_refine(form))
        tuned = s.tune(iters=10) if tune else None
        out = torch.empty_like(db)
        for _ in range(args.warmup):
            s.solve_device(db, pr.lam, iters, out=out)
        torch.cuda.synchronize()
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        with Clocks(local) as clk:
            for i in range(args.steps):
                flush.fill_(float(i))
                starts[i].record()
                s.solve_device(db, pr.lam, iters, out=out, sync=False)
                ends[i].record()
            torch.cuda.synchronize()
        api.sfista_sync(s.ctx)
        ms = sum(a.elapsed_time(b) for a, b in zip(starts, ends))
        _, ms = replica_throughput(ms, iters, args.steps, world, "cuda")
        X = out.cpu().numpy()
        stage_ms = api.sfista_time_stages(s.ctx, db, pr.lam, 50)
        info = s.info()
        # e2e: host buffers (pinned), H2D + solve + D2H inside the timed region.
        bh = torch.from_numpy(b_host).pin_memory()
        xh = torch.empty_like(bh).pin_memory()
        bnp, xnp = bh.numpy(), xh.numpy()
        for _ in range(2):
            api.sfista_solve(s.ctx, bnp, pr.lam, iters, xnp)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            api.sfista_solve(s.ctx, bnp, pr.lam, iters, xnp)
        e2e_s = time.perf_counter() - t0
        results[form] = dict(ms_total=ms, X=X, stage_ms=stage_ms, info=info, tuned=tuned,
                                                 clocks=clk.summary(), e2e_s=e2e_s)
        s.close()

    if rank != 0:
        if world > 1:
            dist.barrier()
            dist.destroy_process_group()
        return

    # CPU baseline: the FP64 oracle on the same b and L (also the parity reference).
    Xref, cpu_s, cores, one_s = oracle_reference(pr, b_host, iters, L)
    r = pr.r
    lines = {}
    for key, res in results.items():
        info = res["info"]
        prec, op = info["prec"], info["op"]
        err = oracle.rel_fro(res["X"], Xref)
        dpsnr = oracle.psnr(res["X"], pr.x_true) - oracle.psnr(Xref, pr.x_true)
        v = world * iters * args.steps / (res["ms_total"] / 1e3)
        wA, wB = info["band_right"], info["band_left"]
        alg = [2.0 * wA * r * n * n, 2.0 * wB * r * n * n, 2.0 * wA * r * n * n, 2.0 * wB * r * n * n]
        sm = [float(x) for x in res["stage_ms"]]
        dom = int(np.argmax(sm))
        if op in ("banded", "banded_fused", "banded_persistent"):
            if op == "banded_persistent":
                work = [sum(alg), 0.0, 0.0, 0.0]   # one persistent launch: all four stages per iteration
            elif op == "banded_fused":
                work = [alg[0] + alg[1], 0.0, alg[2] + alg[3], 0.0]   # one kernel per operator application
            else:
                work = alg
            bound, peak, unit = "alu", FP32_PEAK_TFLOPS, "TFLOP/s"
            peak_src = "152 SM x 128 FP32 lanes x 2 x 2070 MHz (derived)"
        else:
            work = mma_flops_per_stage(info, n, n, r, prec, op)
            bound, unit = "tensor", "TFLOP/s"
            bf16 = peaks.get("bf16_tflops", 1900.0)
            peak = bf16 if prec.startswith("bf16") else bf16 * (1.1 / 2.25)
            peak_src = ("%s bf16 burst" % peak_src_name) + ("" if prec.startswith("bf16") else " x 1.1/2.25 (tf32 nominal ratio)")
        # Duration of the dominant kernel inside the timed region: the
        # per-iteration time of the timed graph runs, split over the stages in
        # proportion to their standalone event timings.
        iter_ms = res["ms_total"] / (args.steps * iters)
        dur_ms = iter_ms * sm[dom] / sum(sm)
        achieved = work[dom] / (dur_ms / 1e3) / 1e12
        ok = meets_tol(prec, err, dpsnr)
        kname = {"banded_persistent": ("band_solve_fused (whole solve, one launch)" if one_launch_fused(n, n)
                                       else "band_solve_persistent (whole solve, one launch)"),
                 "banded_fused": ["band_op_fused_kernel (forward + residual)", "",
                                  "band_op_fused_kernel (adjoint + shrink + momentum)", ""][dom]}.get(op, STAGES[dom])
        launches = 1 + 3 if op == "banded_persistent" else KERNELS_PER_ITER.get(op, 4) * iters + 3
        kref = _refine(key) if op.startswith("gemm") else 0
        if kref:
            # Refined iterations: rows + columns + split (+ FP32 copy of a
            # double-float Y) in place of stages 0 and 1; the stage split of
            # the standalone timings no longer describes the iteration.
            launches += (iters // kref) * (1 + (prec == "tf32x3"))
            achieved = None
        lines[key] = dict(kernel=kname, value=v, err=err, dpsnr=dpsnr, stage_ms=sm, dom=dom, achieved=achieved, ok=ok,
                          dur_us=dur_ms * 1e3, launches=launches,
                          traffic=TRAFFIC.get("%s:%s:%d" % (prec, op, dom)),
                          bound=bound, peak=peak, unit=unit, peak_src=peak_src, prec=prec,
                          op_tflops_alg=sum(alg) * v / world / 1e12,
                          op_tflops_exec=(sum(work) - (work[0] + work[1]) * (iters // kref if kref else 0) / iters)
                          * v / world / 1e12,
                          e2e=iters * args.steps / res["e2e_s"], clocks=res["clocks"],
                          ms_per_step=res["ms_total"] / args.steps, resolved_op=op, tuned=res["tuned"],
                          refine_every=kref)
    held = [k for k in lines if lines[k]["ok"] is True and lines[k]["achieved"] is not None]
    key0 = max(held or list(lines), key=lambda k: lines[k]["value"])
    L0 = lines[key0]
    line = {
        "metric": METRIC, "value": L0["value"], "unit": "iters/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": L0["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": DTYPE[L0["prec"]], "data": "synthetic",
        "config": {"workload": WORKLOAD, "form": key0, "resolved_op": L0["resolved_op"], "iters_per_step": iters,
                   "m": n, "n": n, "r": r,
                   "psf": "31x31", "global_batch": 1, "seq_len": 0, "parallelism": "replicas",
                   "l2": "flushed between steps (256 MB write); the solve's working set is L2-resident"},
        "rel_err_vs_fp64_oracle": L0["err"], "dpsnr_db_vs_oracle": L0["dpsnr"],
        "op_tflops_algorithmic": L0["op_tflops_alg"], "op_tflops_executed": L0["op_tflops_exec"],
        "roofline": {"bound": L0["bound"], "kernel": L0["kernel"], "achieved": L0["achieved"],
                     "peak": L0["peak"], "unit": L0["unit"], "frac": L0["achieved"] / L0["peak"],
                     "traffic": L0["traffic"]["bytes"] if L0["traffic"] else None,
                     "traffic_source": L0["traffic"]["source"] if L0["traffic"] else None,
                     "duration_us": L0["dur_us"], "peak_source": L0["peak_src"]},
        "stage_ms": dict(zip(STAGES, L0["stage_ms"])),
        "cpu_baseline": {"value": iters / cpu_s, "unit": "iters/s", "cores": cores, "kind": "oracle",
                         "sample": "one full 200-iteration FP64 solve of the same problem",
                         "single_thread_iters_per_s": 1.0 / one_s if one_s else None,
                         "cpu_model": cpu_model()},
        "e2e": {"value": L0["e2e"], "unit": "iters/s", "h2d_bytes_per_step": 4 * n * n,
                "d2h_bytes_per_step": 4 * n * n},
        "gpu_launches": L0["launches"] * args.steps,
        "clocks": L0["clocks"],
        "forms": {k: {"iters_per_s": v["value"], "rel_err": v["err"], "dpsnr_db": v["dpsnr"],
                      "meets_tol": v["ok"], "stage_ms": v["stage_ms"],
                      "roofline_frac": v["achieved"] / v["peak"] if v["achieved"] is not None else None,
                      "bound": v["bound"], "op_tflops_executed": v["op_tflops_exec"],
                      "resolved_op": v["resolved_op"], "tuned": v["tuned"], "refine_every": v["refine_every"]}
                  for k, v in lines.items()},
        "peaks": {"source": peak_src_name, "hbm_gbs": peaks.get("hbm_gbs"), "bf16_tflops": peaks.get("bf16_tflops"),
                  "bf16_tflops_sustained": peaks.get("bf16_tflops_sustained")},
    }
    if world == 1 and not args.no_extra:
        # The other two single-GPU workloads, measured after the headline (not part of its
        # timed region): where the tensor-core and batched targets are stated.
        line["config3"] = config3_section(args, torch, peaks)
        line["config4"] = config4_section(args, torch)
        line["wide_psf"] = wide_section(args, torch, peaks)
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
