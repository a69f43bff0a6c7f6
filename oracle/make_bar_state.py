"""Writes oracle/data/twisted_bar_step100.npz: the state (x, v) of the 98,304-tet twisted bar at the start of time
step 100, computed by the FP64 oracle alone (100 time steps of 50 PNCG iterations from the rest pose).

The benchmark's CPU timings start from it, so that the oracle is timed on the same time steps as the GPU's timed
window (steps 100-119, where the twist has brought tens of thousands of surface pairs within reach) without
spending ten minutes re-running the lead-in.  Test infrastructure: only the benchmark's CPU legs read the file.

    python -m oracle.make_bar_state [--steps 100]
"""
import argparse
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))


def main():
    import oracle
    from paper_2405_08001_gb300 import scenes as S
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--steps", type=int, default=100)
    args = ap.parse_args()
    sc = S.twisted_bar()
    o = oracle.Oracle.from_scene(sc)
    x, v = sc.x0.copy(), sc.v0.copy()
    t0 = time.time()
    for s in range(args.steps):
        o.step(x, v, sc.targets(s), iters=sc.iters)
        print(f"step {s} done at {time.time() - t0:.0f} s", flush=True)
    out = os.path.join(HERE, "data", f"twisted_bar_step{args.steps}.npz")
    np.savez_compressed(out, x=x, v=v, step=args.steps, iters=sc.iters)
    print("wrote", out)


if __name__ == "__main__":
    main()
