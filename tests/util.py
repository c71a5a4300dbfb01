"""Shared test helpers (matching of eigenvalue sets)."""
import numpy as np
from scipy.optimize import linear_sum_assignment


def match_eigs(ref, got):
    """Optimal assignment between two eigenvalue sets; returns the max
    relative distance over matched pairs (inf if the counts differ)."""
    ref = np.asarray(ref, dtype=np.complex128)
    got = np.asarray(got, dtype=np.complex128)
    if len(ref) != len(got):
        return np.inf
    if len(ref) == 0:
        return 0.0
    C = np.abs(ref[:, None] - got[None, :])
    r, c = linear_sum_assignment(C)
    return float(np.max(C[r, c] / np.maximum(np.abs(ref[r]), 1e-300)))
