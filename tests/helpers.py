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


def vector_normwise(a, b):
    """Per-field error of the 8 conserved fields [D, S_x, S_y, S_z, tau, B^x,
    B^y, B^z]: max |a - b| over the cells, divided by max |b| for the scalars
    D and tau, and by the largest Euclidean length of the vector (S_i or B^i)
    over the cells for its components.  A component far smaller than its
    vector (a transverse momentum driven only by a 1% perturbation) is then
    held to the vector's scale, as a rotation of the axes would demand."""
    a = np.asarray(a)
    b = np.asarray(b)
    vec = {1: slice(1, 4), 2: slice(1, 4), 3: slice(1, 4), 5: slice(5, 8), 6: slice(5, 8), 7: slice(5, 8)}
    out = []
    for q in range(8):
        d = np.max(np.abs(a[q] - b[q]))
        s = np.max(np.sqrt(np.sum(b[vec[q]] ** 2, axis=0))) if q in vec else np.max(np.abs(b[q]))
        out.append(d / s if s > 0 else d)
    return np.array(out)


def interior(arr, ng):
    return arr[(slice(None),) + tuple(slice(ng, s - ng) for s in arr.shape[1:])]
