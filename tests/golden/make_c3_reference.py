"""Write tests/golden/c3_reference.npz: the FP64 oracle's solution of the 3D workload
(unit cube, Q1 on 128^3 cells, k = 40, delta = 0, u = 0 on z = 0 and Sommerfeld on the other
faces, Gaussian source sigma = 0.05 at the centre, b = M f), sampled at every 11th node.

Only the oracle and the seeded input generators are called: hh_oracle assembles the matrices
(element by element, CSR) and the plain-C oracle (hss_omp, OpenMP) runs FGMRES with the
shifted-HSS preconditioner of Def. 4.1 to a relative residual of 1e-11; the residual is then
recomputed with the Python oracle's own B.  The solution of B_0 u = b is unique, so any
delta_hat serves; the one that needs the fewest oracle steps is used.  The file also holds a
hash of the inputs, so that a test fails loudly when the workload it solves is not this one.

    python tests/golden/make_c3_reference.py [delta_hat] [cycles_per_hss]
    python tests/golden/make_c3_reference.py --rekey     (recompute only the inputs' key)
"""
import hashlib
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import hh_oracle as O  # noqa: E402
from oracle import hss_omp as C  # noqa: E402
from paper_2506_18694_gb300 import inputs  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "c3_reference.npz")
STRIDE = 11
TOL = 1e-11


def input_key(w, f):
    """sha1 over the workload's parameters and a fingerprint of the nodal source (its sum and the
    sum of its magnitudes to 10 significant digits: the last bits of exp differ between
    machines, so the raw bytes would not give the same key everywhere)."""
    f = np.asarray(f, dtype=np.complex128)
    fp = "%.10e %.10e %.10e" % (f.sum().real, f.sum().imag, np.abs(f).sum())
    meta = json.dumps({"dim": w.dim, "n": w.n, "k": w.k, "delta": w.delta, "bc": list(w.bc),
                       "centre": list(w.centre), "sigma": w.sigma, "source": fp}, sort_keys=True)
    return hashlib.sha1(meta.encode()).hexdigest()


def rekey():
    """Rewrite the key of the stored file with input_key (the solution is left as it is)."""
    w = inputs.workload("3d_n128_k40")
    f = inputs.gaussian_source(w.dim, w.n, w.centre, w.sigma)
    d = dict(np.load(OUT))
    d["key"] = input_key(w, f)
    np.savez_compressed(OUT, **d)
    print("rekeyed", OUT, d["key"])


def main():
    dh = sys.argv[1] if len(sys.argv) > 1 else "k"
    cycles = int(sys.argv[2]) if len(sys.argv) > 2 else 1
    w = inputs.workload("3d_n128_k40", dh)
    g = O.Grid(w.dim, w.n, w.bc)
    f = inputs.gaussian_source(w.dim, w.n, w.centre, w.sigma)
    t0 = time.perf_counter()
    prob = O.Problem(g, w.k, w.delta, w.delta_hat, O.Options(cycles_per_hss=cycles, restart=60))
    b = prob.mats[0][1] @ f
    c = C.COracle(prob)
    x, its, rr = c.fgmres(b, TOL, restart=60, max_it=5000)
    res = np.linalg.norm(b - prob.B @ x) / np.linalg.norm(b)
    dt = time.perf_counter() - t0
    print(f"delta_hat={w.delta_hat} cycles={cycles}: {its} iterations, residual {rr:.3e} "
          f"(recomputed {res:.3e}) in {dt:.0f} s, {C.COracle.threads()} threads", flush=True)
    if not res <= 2 * TOL:
        raise SystemExit("the oracle did not reach the tolerance")
    np.savez_compressed(OUT, key=input_key(w, f), stride=STRIDE, u=x[::STRIDE], norm_u=np.linalg.norm(x),
                        rel_residual=res, iterations=its, delta_hat=w.delta_hat, cycles_per_hss=cycles, tol=TOL)
    print("wrote", OUT)


if __name__ == "__main__":
    rekey() if sys.argv[1:] == ["--rekey"] else main()
