"""Comparison helpers shared by the GPU parity tests (not a test module).

rel: ||got - want||_2 / ||want||_2 over the whole result.
partition_max: the worst partition's max |got - want| / max |want| (per
  right-hand side column), so an error confined to one partition (its tip
  rows, say) is measured against that partition's own scale.  Every parity
  test checks both: the 2-norm bound of the path, and the per-partition
  max-norm at ten times that bound.  A localized defect that keeps the
  global 2-norm within bound (one partition of n_i rows contributes only
  sqrt(n_i / n) of the norm) exceeds the per-partition bound.
"""
import numpy as np

from oracle import lrspike_oracle as O


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def partition_max(got, want, n, p):
    """max over partitions i and columns c of max_rows |got - want| / max_rows |want|."""
    g = np.asarray(got).reshape(n, -1)
    w = np.asarray(want).reshape(n, -1)
    offs = O.partition_offsets(n, p)
    worst = 0.0
    for i in range(p):
        s, e = int(offs[i]), int(offs[i + 1])
        scale = np.abs(w[s:e]).max(axis=0)
        scale[scale == 0.0] = 1.0
        worst = max(worst, float((np.abs(g[s:e] - w[s:e]).max(axis=0) / scale).max()))
    return worst


def check(got, want, n, p, tol):
    """2-norm within tol and every partition's max-norm within 10 tol."""
    r = rel(got, want)
    m = partition_max(got, want, n, p)
    assert r <= tol, f"relative 2-norm error {r:.3e} > {tol:.1e}"
    assert m <= 10 * tol, f"per-partition max-norm error {m:.3e} > {10 * tol:.1e}"
