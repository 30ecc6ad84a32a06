"""The stored 3D oracle solution (tests/golden/c3_reference.npz) is the oracle's answer for the
3D workload: its key matches these inputs, its recorded residual meets its tolerance, and on
the sampled nodes it satisfies the discrete problem's structure (zero on the Dirichlet face)."""
import importlib.util
import os

import numpy as np

from oracle import hh_oracle as O
from paper_2506_18694_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def test_c3_reference_matches_its_inputs():
    spec = importlib.util.spec_from_file_location("make_c3_reference", os.path.join(GOLDEN, "make_c3_reference.py"))
    mk = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mk)
    w = inputs.workload("3d_n128_k40")
    f = inputs.gaussian_source(w.dim, w.n, w.centre, w.sigma)
    ref = np.load(os.path.join(GOLDEN, "c3_reference.npz"))
    assert str(ref["key"]) == mk.input_key(w, f)
    assert float(ref["rel_residual"]) <= 2 * float(ref["tol"]) <= 2e-11
    g = O.Grid(w.dim, w.n, w.bc)
    stride = int(ref["stride"])
    u = ref["u"]
    assert u.size == len(range(0, g.N, stride))
    free = g.free()[::stride]
    assert np.all(u[~free] == 0) and np.all(np.isfinite(u)) and np.abs(u[free]).max() > 0
