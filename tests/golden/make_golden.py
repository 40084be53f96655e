"""Writes c1_mu_oracle.txt beside this script.

The stored values are the FP64 oracle's (oracle/, test infrastructure) full
MU solve (Algorithm 1: tol 1e-4, up to 10 outer and 10 inner iterations) of
the 100 x 80 x 60 workload with 10,000 uniformly drawn nonzeros, counts
Poisson(1)+1 and rank 10, from the seeded initial model lambda = 1 and U(0,1)
factors (seed 1001 + 17).  Only oracle/ computes them; synth supplies the
seeded inputs.  Rerun after a change to the oracle's arithmetic that a
passage of the paper justifies:

    python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

OUT = os.path.join(HERE, "c1_mu_oracle.txt")


def solve():
    import oracle
    from paper_2307_03276_gb300 import synth
    oracle.build()
    spec = synth.C1
    T = synth.generate(spec)
    lam = np.ones(T.rank)
    fs = synth.random_factors(T.dims, T.rank, spec.seed + 17)
    return oracle.mu_solve(T.dims, T.idx, T.vals, lam, fs, tol=1e-4, max_outer=10, max_inner=10)


def write(path=OUT):
    r = solve()
    with open(path, "w") as f:
        f.write("# FP64 oracle, Algorithm 1 on the 100x80x60 / 1e4-nonzero / R=10 workload; see make_golden.py\n")
        f.write(f"outer_iters {r['outer_iters']}\n")
        f.write(f"converged {int(r['converged'])}\n")
        for k in range(r["outer_iters"]):
            f.write(f"outer {k + 1} inner {' '.join(str(int(x)) for x in r['inner'][k])} "
                    f"kkt {r['kkt'][k]:.17e} loglik {r['loglik'][k]:.17e}\n")
        f.write("lambda " + " ".join(f"{x:.17e}" for x in r["lambda"]) + "\n")


def read(path=OUT):
    out = {"outer": []}
    with open(path) as f:
        for line in f:
            if line.startswith("#"):
                continue
            w = line.split()
            if w[0] == "outer_iters":
                out["outer_iters"] = int(w[1])
            elif w[0] == "converged":
                out["converged"] = bool(int(w[1]))
            elif w[0] == "outer":
                i = w.index("inner")
                kk = w.index("kkt")
                out["outer"].append(([int(x) for x in w[i + 1:kk]], float(w[kk + 1]), float(w[kk + 3])))
            elif w[0] == "lambda":
                out["lambda"] = np.array([float(x) for x in w[1:]])
    return out


if __name__ == "__main__":
    write()
    print("wrote", OUT)
