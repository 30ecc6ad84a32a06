"""Element-by-element comparison of a GPU result with the oracle's.

rel(a, ref) is the larger of two relative errors:
  norm-wise      ||a - ref||_2 / ||ref||_2
  per node       max_i |a_i - ref_i| / max_i |ref_i|
so that one node that is wrong by far more than rounding fails even in a large vector,
where its share of the norm would be small.  Where the oracle's value is an exact zero
(Dirichlet nodes, whose unknowns are eliminated) the GPU value must be an exact zero too;
otherwise rel returns inf.
"""
import numpy as np


def rel(a, ref):
    a = np.asarray(a).reshape(-1)
    ref = np.asarray(ref).reshape(-1)
    assert a.shape == ref.shape, (a.shape, ref.shape)
    zero = ref == 0
    if np.any(a[zero] != 0):
        return float("inf")
    d = np.abs(a - ref)
    nref = np.linalg.norm(ref)
    mref = np.abs(ref).max() if ref.size else 0.0
    normwise = np.linalg.norm(d) / (nref if nref > 0 else 1.0)
    pernode = (d.max() if d.size else 0.0) / (mref if mref > 0 else 1.0)
    return float(max(normwise, pernode))
