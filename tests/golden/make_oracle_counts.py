"""Write tests/golden/oracle_counts_256.json: iteration counts of the FP64 oracle on the
256^3 7-point Poisson workload (x_true ~ U[-1,1) seed 0, b = A x_true, Jacobi, rtol 1e-8,
lambda_max from 20 power iterations with start vector seed 1, Gershgorin lower bound = 0).

Calls only the oracle (and the seeded input module).  Slow: tens of minutes of one CPU core
per configuration.  Usage: python tests/golden/make_oracle_counts.py [config ...]
where config is "pcg" or "<literal|onesync>_s<S>nu<NU>"
(default: pcg literal_s4nu3 literal_s4nu30).
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_2603_09790_gb300 import inputs as I  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_counts_256.json")


def main(configs):
    dims = (256, 256, 256)
    A = O.CSR(*I.poisson_csr(dims, 7))
    xt, b = I.poisson_problem(dims, 7)
    v0 = I.power_start(A.n)
    lam, _ = O.power(A, "jacobi", v0, 20, 0.0)
    lmin = O.gershgorin_lower(A, "jacobi")
    for cfg in configs:
        t = time.time()
        if cfg == "pcg":
            r = O.pcg(A, b, rtol=1e-8)
        else:
            algo, rest = cfg.split("_")
            s, nu = rest[1:].split("nu")
            r = O.pcgs(A, b, s=int(s), nu=int(nu), rtol=1e-8, algo=algo, lambda_min=lmin,
                       lambda_max=lam)
        rec = dict(iters=r.iters, status=r.status, relres=r.relres, relres_true=r.relres_true,
                   lambda_max=lam, lambda_min=lmin, seconds_1core=time.time() - t)
        data = json.load(open(OUT)) if os.path.exists(OUT) else {}
        data[cfg] = rec
        json.dump(data, open(OUT + ".tmp", "w"), indent=1, sort_keys=True)
        os.replace(OUT + ".tmp", OUT)
        print(cfg, rec, flush=True)


if __name__ == "__main__":
    main(sys.argv[1:] or ["pcg", "literal_s4nu3", "literal_s4nu30"])
