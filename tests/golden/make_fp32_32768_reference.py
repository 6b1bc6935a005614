"""Write the FP64 oracle's result for the 32768 x 32768 benchmark workload.

Runs only the oracle (host, NumPy/LAPACK) on the stored FP32 matrix that
``bcur_inputs.fp32_32768()`` draws, and stores block scores, block indices,
the top singular values and the residual in ``fp32_32768_oracle.json`` next
to this file.  Needs about 45 GB of host memory and a few minutes on 16 cores.

    python tests/golden/make_fp32_32768_reference.py
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
    t0 = time.time()
    p = bi.fp32_32768()
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
    path = os.path.join(HERE, "fp32_32768_oracle.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps({k: out[k] for k in ("rel", "err", "col_idx", "row_idx",
                                          "seconds_generate", "seconds_oracle")}))


if __name__ == "__main__":
    main()
