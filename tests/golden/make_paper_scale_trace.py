"""Write paper_scale_trace.npz: the oracle's full trace of the 1e6-pair workload.

Workload `lowp_n1e6_128L3` of the seeded generator (1e6 unit pairs, 99%
uniform outliers, inlier noise 0.005, delta = 0.03, 128^3 coarse grid plus
three refinement levels of the top 16 cells; the paper's largest synthetic
setting, Sec. 5.3.1).  Everything stored comes from `oracle.solve` (the FP64
C oracle, threads over cells; counts are integers, so the thread count does
not change them):

  input_sha256       SHA-256 of a.tobytes() + b.tobytes() (float32 [n, 3])
  l0_count, l0_amb   per coarse cell, in table order (increasing linear index):
                     the vote count and the number of ambiguous tests
                     (|v - tau| <= 1e-6 in FP64)
  l{k}_idx, l{k}_count, l{k}_amb   the same for refinement level k = 1..3
  topk{k}            linear indices of the kept cells of level k, rank order
  q, best_cell, best_count, inliers, status, ambiguous, tests   the result

The coarse cell indices and thresholds are not stored: the oracle's level
enumeration and its cell geometry reproduce them in a second.

Run from the repository root:  python tests/golden/make_paper_scale_trace.py
(about 20 minutes on 8 cores).  Nothing here calls the CUDA library.
"""
import hashlib
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2506_11547_gb300 import synth  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_scale_trace.npz")


def main() -> None:
    p, grid_n, levels = synth.config_problem("lowp_n1e6_128L3")
    h = hashlib.sha256(p.a.tobytes() + p.b.tobytes()).hexdigest()
    t0 = time.time()
    o = oracle.solve(p.a, p.b, float(np.float32(p.delta)), grid_n=grid_n, levels=levels,
                     nthreads=max(1, os.cpu_count() or 1), trace=True)
    dt = time.time() - t0
    out = dict(input_sha256=np.array(h), q=o.q, best_cell=np.int64(o.best_cell),
               best_count=np.int32(o.best_count), inliers=np.int32(o.inliers), status=np.int32(o.status),
               ambiguous=np.int64(o.ambiguous), tests=np.int64(o.tests))
    lv0 = o.levels[0]
    out["l0_count"] = lv0["count"].astype(np.int32)
    out["l0_amb"] = lv0["amb"].astype(np.int32)
    out["topk0"] = lv0["topk_idx"].astype(np.int64)
    for k in range(1, levels + 1):
        lv = o.levels[k]
        out[f"l{k}_idx"] = lv["idx"].astype(np.int64)
        out[f"l{k}_count"] = lv["count"].astype(np.int32)
        out[f"l{k}_amb"] = lv["amb"].astype(np.int32)
        out[f"topk{k}"] = lv["topk_idx"].astype(np.int64)
    np.savez_compressed(OUT, **out)
    print(f"wrote {OUT}: {len(lv0['count'])} coarse cells, ambiguous {o.ambiguous}, "
          f"{dt:.0f} s on {max(1, os.cpu_count() or 1)} threads, {os.path.getsize(OUT)} bytes")


if __name__ == "__main__":
    main()
