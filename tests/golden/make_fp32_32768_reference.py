"""Write the FP64 oracle's result for a 32768 x 32768 workload.

Runs only the oracle (host, NumPy/LAPACK) on the stored FP32 matrix that
``bcur_inputs.fp32_32768()`` (or ``precision_32768()``, k = 100, p = 20,
q = 3) draws, and stores block scores, block indices, the top singular values
and the residual in ``<workload>_oracle.json`` next to this file.  It also
times the oracle on the bounded sample that the benchmark times
(``bcur_inputs.host_sample``: the same recipe at 1/4 the size per side), in
the same process on the same host cores, so that the benchmark can scale its
sample's time to the full size by a measured ratio.  Needs about 45 GB of
host memory and a few minutes on 16 cores.

    python tests/golden/make_fp32_32768_reference.py [fp32_32768 | precision_32768]
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import bcur_inputs as bi  # noqa: E402
import oracle as orc  # noqa: E402


def main():
    name = sys.argv[1] if len(sys.argv) > 1 else "fp32_32768"
    t0 = time.time()
    p = {"fp32_32768": bi.fp32_32768, "precision_32768": bi.precision_32768}[name]()
    A = p.matrix()                      # FP32 storage, as the GPU reads it
    t1 = time.time()
    r = orc.block_cur(A, p.col_off, p.row_off, p.k, p.q, p.g_col, p.g_row, p.omega(), p.u_col(),
                      p.u_row())
    t2 = time.time()
    out = dict(workload=p.name, m=p.m, n=p.n, k=p.k, p=p.p, q=p.q, seed=p.seed,
               col_scores=[float(x) for x in r["col_scores"]],
               row_scores=[float(x) for x in r["row_scores"]],
               col_idx=[int(x) for x in r["col_idx"]], row_idx=[int(x) for x in r["row_idx"]],
               sigma=[float(x) for x in r["sigma"]], err=float(r["err"]), rel=float(r["rel"]),
               norm_a=float(np.linalg.norm(A.astype(np.float64))),
               seconds_generate=round(t1 - t0, 1), seconds_oracle=round(t2 - t1, 1))
    ps = bi.host_sample(p)
    As = ps.matrix()
    t3 = time.time()
    orc.block_cur(As, ps.col_off, ps.row_off, ps.k, ps.q, ps.g_col, ps.g_row, ps.omega(),
                  ps.u_col(), ps.u_row())
    t4 = time.time()
    out.update(seconds_sample=round(t4 - t3, 2), sample=f"{ps.m}x{ps.n}, g {ps.g_col}+{ps.g_row}",
               cores=os.cpu_count())
    path = os.path.join(HERE, f"{p.name}_oracle.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps({k: out[k] for k in ("rel", "err", "col_idx", "row_idx", "seconds_generate",
                                          "seconds_oracle", "seconds_sample", "cores")}))


if __name__ == "__main__":
    main()
