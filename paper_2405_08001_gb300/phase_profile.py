"""Diagnostic command line of the library: runs one of the benchmark workloads for some steps and reports where a
persistent time step spends its time, block by block.

After `--warmup` untimed steps it asks the library (sim_profile_barriers) for every block's arrival and departure
time at every grid barrier of `--steps` more steps and prints, per phase: the time from the release of the previous
barrier to the last block's arrival, the median and largest per-block work, the release latency of the barrier
(last arrival to first departure) and how late the last block arrives after the median one.  With `--plain` it only
runs the steps (no barrier recording): a fixed, countable sequence of launches for an external profiler, e.g.
`ncu -k regex:k_persistent -s W -c 1` captures the first step after W warm-up steps.

    python -m paper_2405_08001_gb300.phase_profile [--scene twisted_bar|cube_drop|large_pile|contact_stack|batched]
        [--precision fp32|fp64] [--warmup W] [--steps K] [--phases] [--plain] [--block-shape S] [--scatter C]
"""
import argparse
import collections

import numpy as np

SCENES = ("twisted_bar", "cube_drop", "large_pile", "contact_stack", "batched")


def make_scene(name):
    from . import scenes as S
    if name == "twisted_bar":
        return S.twisted_bar()
    if name == "cube_drop":
        return S.cube_drop()
    if name == "large_pile":
        return S.pile()
    if name == "contact_stack":
        return S.pile(gap=0.5, jitter=False, steps=20)
    return S.batched()


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
    from . import binding as B, build
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--scene", default="twisted_bar", choices=SCENES)
    ap.add_argument("--precision", default="fp32", choices=("fp32", "fp64"))
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--phases", action="store_true", help="one kernel per phase instead of the persistent step")
    ap.add_argument("--plain", action="store_true", help="only run the steps (for an external profiler)")
    ap.add_argument("--block-shape", type=int, default=0, help="sim_options.block_shape (0-4; -1 = autotuned)")
    ap.add_argument("--scatter", type=int, default=0, help="sim_options.scatter (0 atomic, 1 segmented, 2 block, 3 colour)")
    args = ap.parse_args()
    build.build()
    B.load()
    sc = make_scene(args.scene)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    prec = B.SIM_FP32_MIXED if args.precision == "fp32" else B.SIM_FP64
    sim = B.Sim(sc, precision=prec, cuda_stream=stream.cuda_stream, persistent=0 if args.phases else 1,
                block_shape=args.block_shape, scatter=args.scatter)
    n = args.warmup + args.steps
    tg = sc.all_targets(n)
    for s in range(args.warmup):
        B.sim_step(sim.h, 1, None if tg is None else tg[s])
    if args.plain or args.phases:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for s in range(args.warmup, n):
            B.sim_step(sim.h, 1, None if tg is None else tg[s])
        e1.record(stream)
        torch.cuda.synchronize()
        _, _, st = B.sim_get_state(sim.h, want_x=False, want_v=False)
        sim.close()
        print(f"{args.scene} {args.precision}: {n} steps, {e0.elapsed_time(e1) / max(1, args.steps):.3f} ms per step "
              f"after the warm-up (CUDA events); last step: {st['n_candidates']} candidates, "
              f"{st['n_active']} active pairs, {st['n_rebuilds']} candidate builds; block shape "
              f"{st['block_threads']} x {st['blocks_per_sm']}; scatter {args.scatter}, {st['n_colors']} colours")
        return
    acc = collections.defaultdict(list)
    nblocks = 0
    spans = []
    for s in range(args.warmup, n):
        a, d, kinds = B.sim_profile_barriers(sim.h, None if tg is None else tg[s])
        nblocks = a.shape[1]
        spans.append(float(a[-1].astype(np.int64).max() - d[0].astype(np.int64).min()))
        for k, v in phase_table(a, d, kinds).items():
            acc[k].append(v)
    _, _, st = B.sim_get_state(sim.h, want_x=False, want_v=False)
    sim.close()
    print(f"{args.scene} {args.precision}: {args.steps} steps after {args.warmup} warm-up steps, {nblocks} blocks of "
          f"{st['block_threads']} threads; {st['n_candidates']} candidates, {st['n_active']} active pairs; times in "
          f"microseconds, per phase instance")
    print(f"{'phase':12s} {'per step':>8s} {'span':>8s} {'median':>8s} {'max':>8s} {'release':>8s} {'late':>8s}")
    print(f"step span (first barrier's release to the last arrival): {np.mean(spans) / 1e3:.1f} us")
    for k, parts in acc.items():
        v = np.concatenate(parts)
        print(f"{k:12s} {len(v) / args.steps:8.1f} {v[:, 0].mean() / 1e3:8.2f} {v[:, 1].mean() / 1e3:8.2f} "
              f"{v[:, 2].mean() / 1e3:8.2f} {v[:, 3].mean() / 1e3:8.2f} {v[:, 4].mean() / 1e3:8.2f}")


if __name__ == "__main__":
    main()
