"""Write tests/golden/oracle_fixed_256.json: the FP64 oracle on the 256^3 7-point Poisson
workload (x_true ~ U[-1,1) seed 0, b = A x_true, Jacobi, lambda_max from 20 power iterations
with start vector seed 1, lambda_min = Gershgorin bound = 0) run for a FIXED number of outer
iterations (rtol = 0), so that the CUDA path can be compared with it at the full size:

* the relative residual history ||r^(k)|| / ||b||, k = 0..K;
* x at 4096 sampled indices (SplitMix64 seed 11, mod n), in index order of the sample;
* two functionals of the whole x: ||x||_2 and w^T x with w ~ U[-1,1) (SplitMix64 seed 12),
  which move if any entry of x is wrong.

Calls only the oracle (and the seeded input module).  Slow: about 3 s of one CPU core per
PCG-S outer iteration, 0.4 s per PCG iteration.  Usage:
    python tests/golden/make_oracle_fixed_256.py [config ...]
config: "pcg_K<k>" or "<literal|onesync>_s<S>nu<NU>_K<k>" (default: literal_s4nu3_K32
literal_s4nu3_K40 literal_s4nu30_K131 pcg_K520).
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_2603_09790_gb300 import inputs as I  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_fixed_256.json")
N = 256
NSAMPLE = 4096


def sample_indices(n):
    """Sorted, distinct sample indices from the SplitMix64 stream with seed 11."""
    idx = np.unique(I.splitmix64(11, 2 * NSAMPLE) % np.uint64(n)).astype(np.int64)
    return idx[:NSAMPLE]


def weights(n):
    return I.uniform_pm1(12, n)


def main(configs):
    dims = (N, N, N)
    A = O.CSR(*I.poisson_csr(dims, 7))
    xt, b = I.poisson_problem(dims, 7)
    v0 = I.power_start(A.n)
    lam, _ = O.power(A, "jacobi", v0, 20, 0.0)
    lmin = O.gershgorin_lower(A, "jacobi")
    idx = sample_indices(A.n)
    w = weights(A.n)
    for cfg in configs:
        t = time.time()
        head, k = cfg.rsplit("_K", 1)
        K = int(k)
        if head == "pcg":
            r = O.pcg(A, b, rtol=0.0, max_iters=K, history=True)
        else:
            algo, rest = head.split("_")
            s, nu = rest[1:].split("nu")
            r = O.pcgs(A, b, s=int(s), nu=int(nu), rtol=0.0, max_outer=K, algo=algo,
                       lambda_min=lmin, lambda_max=lam, history=True)
        assert r.iters == K, (cfg, r.iters, r.status)
        rec = dict(K=K, lambda_max=lam, lambda_min=lmin, hist=[float(v) for v in r.hist[:K + 1]],
                   sample_index=[int(i) for i in idx], x_sample=[float(v) for v in r.x[idx]],
                   x_norm=float(np.linalg.norm(r.x)), wx=float(w @ r.x),
                   w_norm=float(np.linalg.norm(w)), seconds_1core=time.time() - t)
        data = json.load(open(OUT)) if os.path.exists(OUT) else {}
        data[cfg] = rec
        json.dump(data, open(OUT + ".tmp", "w"), indent=0, sort_keys=True)
        os.replace(OUT + ".tmp", OUT)
        print(cfg, {k_: v for k_, v in rec.items() if k_ not in ("hist", "sample_index", "x_sample")},
              flush=True)


if __name__ == "__main__":
    main(sys.argv[1:] or ["literal_s4nu3_K32", "literal_s4nu3_K40", "literal_s4nu30_K131", "pcg_K520"])
