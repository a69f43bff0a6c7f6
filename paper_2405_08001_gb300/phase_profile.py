"""Phase timings of the persistent time step, block by block.

Runs a scene for a few warm-up steps, then asks the library (sim_profile_barriers) for every block's arrival and
departure time at every grid barrier of one more step, and prints per phase: the time from the release of the
previous barrier to the last block's arrival, the median and largest per-block work, the release latency of the
barrier (last arrival to first departure) and how late the last block arrives after the median one.

    python -m paper_2405_08001_gb300.phase_profile [--scene twisted_bar|cube_drop] [--precision fp32|fp64] [--steps K]
"""
import argparse
import collections

import numpy as np


def phase_table(arrive, depart, kinds):
    a = arrive.astype(np.int64)
    d = depart.astype(np.int64)
    rows = collections.defaultdict(list)
    for i in range(1, a.shape[0]):
        work = a[i] - d[i - 1]
        rows[kinds[i]].append((a[i].max() - d[i - 1].min(), np.median(work), work.max(), d[i].min() - a[i].max(),
                               a[i].max() - np.median(a[i])))
    return {k: np.array(v, dtype=np.float64) for k, v in rows.items()}


def main():
    import torch
    from . import binding as B, build, scenes as S
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--scene", default="twisted_bar", choices=("twisted_bar", "cube_drop"))
    ap.add_argument("--precision", default="fp32", choices=("fp32", "fp64"))
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--steps", type=int, default=3)
    args = ap.parse_args()
    build.build()
    B.load()
    sc = S.twisted_bar() if args.scene == "twisted_bar" else S.cube_drop()
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    prec = B.SIM_FP32_MIXED if args.precision == "fp32" else B.SIM_FP64
    sim = B.Sim(sc, precision=prec, cuda_stream=stream.cuda_stream, persistent=1)
    tg = sc.all_targets(args.warmup + args.steps)
    for s in range(args.warmup):
        B.sim_step(sim.h, 1, tg[s])
    acc = collections.defaultdict(list)
    nblocks = 0
    spans = []
    for s in range(args.warmup, args.warmup + args.steps):
        a, d, kinds = B.sim_profile_barriers(sim.h, tg[s])
        nblocks = a.shape[1]
        spans.append(float(a[-1].astype(np.int64).max() - d[0].astype(np.int64).min()))
        for k, v in phase_table(a, d, kinds).items():
            acc[k].append(v)
    sim.close()
    print(f"{args.scene} {args.precision}: {args.steps} steps after {args.warmup} warm-up steps, {nblocks} blocks; "
          f"times in microseconds, per phase instance")
    print(f"{'phase':12s} {'per step':>8s} {'span':>8s} {'median':>8s} {'max':>8s} {'release':>8s} {'late':>8s}")
    print(f"step span (first barrier's release to the last arrival): {np.mean(spans) / 1e3:.1f} us")
    for k, parts in acc.items():
        v = np.concatenate(parts)
        print(f"{k:12s} {len(v) / args.steps:8.1f} {v[:, 0].mean() / 1e3:8.2f} {v[:, 1].mean() / 1e3:8.2f} "
              f"{v[:, 2].mean() / 1e3:8.2f} {v[:, 3].mean() / 1e3:8.2f} {v[:, 4].mean() / 1e3:8.2f}")


if __name__ == "__main__":
    main()
