"""Write the dense-oracle solution of a named workload to tests/golden/<name>_x.npy.

The stored values come from oracle/ only: the oracle's dense CBIE/MFIE matrix
(Eq. 20: Nystrom far rule with independently integrated self/near entries, the
1/2 identity term of the jump relation, Eq. 5) and its plane-wave right-hand
sides (Eq. 22), solved by dense LU with partial pivoting.  The LU step is the
library routine LAPACK zgesv (numpy.linalg.solve): at 19,200 unknowns the
oracle's plain right-looking LU streams the trailing matrix once per column and
would run for hours on a workstation; zgesv computes the same factorisation
(partial pivoting; the oracle's LU is checked against it in the oracle pins).

Also written: <name>_x.json with the residual of the stored solution against the
oracle's matrix, the bound sqrt(|A|_1 |A|_inf) >= |A|_2 and the power-iteration value of
|A|_2 (either turns a solution error into a bound on the full residual:
|A x - b| <= |A|_2 |x - x_o| + |A x_o - b|), and the wall times of the fill and of the
solve on this machine.

  python tests/golden/make_dense_solution.py sphere_d8_m4_nc10
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_2408_17116_gb300 import workloads  # noqa: E402


def main(name):
    wl = workloads.workload(name)
    o = oracle.Oracle(wl["bodies"], wl["ms"], wl["nc"], wl["k"])
    b = o.rhs(wl["kdirs"], wl["pols"])
    t = time.perf_counter()
    A = o.dense()
    t_fill = time.perf_counter() - t
    t = time.perf_counter()
    X = np.linalg.solve(A, b.T).T
    t_solve = time.perf_counter() - t
    res = [float(np.linalg.norm(A @ X[r] - b[r]) / np.linalg.norm(b[r])) for r in range(b.shape[0])]
    a1 = float(np.abs(A).sum(axis=0).max())
    ainf = float(np.abs(A).sum(axis=1).max())
    # the largest singular value by power iteration on A^H A (seeded start vector), run
    # until the estimate changes by less than 1e-9 relative
    v = np.random.default_rng(1).standard_normal(o.N) + 0j
    v /= np.linalg.norm(v)
    smax = 0.0
    for it in range(500):
        w = np.conj(A.T @ np.conj(A @ v))  # A^H (A v) without forming A^H
        s_new = float(np.sqrt(np.linalg.norm(w)))
        v = w / np.linalg.norm(w)
        if abs(s_new - smax) <= 1e-9 * s_new:
            smax = s_new
            break
        smax = s_new
    power_iters = it + 1
    np.save(os.path.join(HERE, name + "_x.npy"), np.ascontiguousarray(X.astype(np.complex128)))
    meta = {"workload": name, "unknowns": int(o.N), "rhs": int(b.shape[0]), "residual": res,
            "norm2_bound": float(np.sqrt(a1 * ainf)), "norm2_power": smax, "power_iters": power_iters,
            "bnorm": [float(np.linalg.norm(b[r])) for r in range(b.shape[0])],
            "fill_s": t_fill, "solve_s": t_solve, "host_threads": os.cpu_count(),
            "script": "tests/golden/make_dense_solution.py"}
    with open(os.path.join(HERE, name + "_x.json"), "w") as f:
        json.dump(meta, f, indent=1)
    print(json.dumps(meta))


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else "sphere_d8_m4_nc10")
