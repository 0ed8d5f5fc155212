"""Shared helpers for the parity tests (no method arithmetic here)."""
import numpy as np

FP64_TOL = 1e-12     # FP64 path vs FP64 oracle, normwise per field
MIXED_TOL = 1e-5     # mixed path vs FP64 oracle, normwise per conserved field


def normwise(a, b, axis_fields=0, floor=None):
    """Per-field max |a - b| / max |b| over the cells (array layout [var, ...])."""
    a = np.asarray(a)
    b = np.asarray(b)
    out = []
    for q in range(a.shape[axis_fields]):
        d = np.max(np.abs(a[q] - b[q]))
        s = np.max(np.abs(b[q]))
        if floor is not None:
            s = max(s, floor)
        out.append(d / s if s > 0 else d)
    return np.array(out)


def interior(arr, ng):
    return arr[(slice(None),) + tuple(slice(ng, s - ng) for s in arr.shape[1:])]
