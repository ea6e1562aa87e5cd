"""Run one workload's solve a few times, for profilers (ncu) and quick timing.

  python -m paper_1901_00913_gb300.profile_case --config 2 --prec fp32 --op banded --iters 20 --reps 2

Uses L = 1 (no power iteration), so the first kernels launched are the
solve's own: per solve, one input check, one state initialisation, then
4 kernels per iteration, then one output conversion.  --config 4 solves the
batched workload (64 problems) as one batch with default tile shapes (no
tuning), so the launches are the batch's own.
"""
import argparse
import time

import numpy as np


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--config", type=int, default=2, choices=[1, 2, 3, 4])
    ap.add_argument("--prec", default="fp32")
    ap.add_argument("--op", default="auto")
    ap.add_argument("--iters", type=int, default=20)
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--graph", type=int, default=0)
    args = ap.parse_args()
    import torch
    from . import api, build, workloads as W
    build.build()
    if args.config == 4:
        probs = W.config4()
        solvers, bs = [], []
        for q in probs:
            n = q.x_true.shape[0]
            bq = api.sfista_blur(q.psf, torch.from_numpy(q.x_true.astype(np.float32)).cuda(), q.bc)
            bs.append(bq)
            solvers.append(api.Sfista(q.psf, (n, n), q.bc, q.r, prec=args.prec, op=args.op, lipschitz=1.0,
                                      use_graph=bool(args.graph)))
        batch = api.Batch(solvers)
        outs = [torch.empty_like(bq) for bq in bs]
        for _ in range(args.reps):
            t0 = time.perf_counter()
            batch.solve(bs, [q.lam for q in probs], args.iters, outs=outs)
            torch.cuda.synchronize()
            print("config 4 batch (%d problems): %d iters in %.3f ms" % (len(probs), args.iters,
                                                                    1e3 * (time.perf_counter() - t0)))
        batch.close()
        for sv in solvers:
            sv.close()
        return
    pr = {1: W.config1, 2: W.config2, 3: W.config3}[args.config]()
    n = pr.x_true.shape[0]
    b = torch.from_numpy(pr.x_true.astype(np.float32)).cuda()
    b = api.sfista_blur(pr.psf, b, pr.bc)
    s = api.Sfista(pr.psf, (n, n), pr.bc, pr.r, prec=args.prec, op=args.op, lipschitz=1.0,
                   use_graph=bool(args.graph))
    out = torch.empty_like(b)
    for _ in range(args.reps):
        t0 = time.perf_counter()
        s.solve_device(b, pr.lam, args.iters, out=out)
        torch.cuda.synchronize()
        print("%s %s: %d iters in %.3f ms" % (pr.name, s.info()["op"], args.iters,
                                             1e3 * (time.perf_counter() - t0)))
    s.close()


if __name__ == "__main__":
    main()
