"""Conditioning of the interface matrices W = I - R33b R33a (Sec. 2.2) of the
benchmark workloads, from the oracle: per merge level from the root down, the
largest 1-norm condition number over the level's merges.  Two correct FP64
builds can differ by about cond(W) times the unit roundoff at the top levels,
so these figures go beside the GPU-vs-oracle errors.

    python -m oracle.cond_report [16] [64]
"""
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_1812_07167_gb300 import workloads as W  # noqa: E402


def report(m: int) -> None:
    if m == 16:
        wl = W.point_sources()
    else:
        wl = W.random_medium_sources(m, 16, {64: 300.0, 128: 600.0}.get(m, 300.0))
    pr = O.Problem(wl.m, wl.p, wl.kappa, wl.eta)
    lxy, bxy = O.nodes(pr)
    c, _, _ = wl.sample(lxy, bxy)
    t0 = time.perf_counter()
    with O.Tree(pr, c, nthreads=os.cpu_count() or 1) as T:
        cond = T.cond_W()
    print(f"{wl.name} {m}x{m} p={wl.p} kappa={wl.kappa:g}: cond_1(W) per level from the root "
          + ", ".join(f"{v:.3g}" for v in cond) + f"  ({time.perf_counter() - t0:.0f} s)", flush=True)


if __name__ == "__main__":
    for a in sys.argv[1:] or ["16"]:
        report(int(a))
