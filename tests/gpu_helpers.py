"""Shared helpers of the GPU parity tests (no PSF arithmetic here)."""
import numpy as np

from oracle.optics import Optics


def oracle_optics(d):
    return Optics.from_dict(d)


def max_rel(x, ref):
    """max |x - ref| / max |ref| over the whole stack (the 1e-5 metric)."""
    x = np.asarray(x)
    ref = np.asarray(ref)
    return float(np.max(np.abs(x - ref)) / np.max(np.abs(ref)))


def rel_l2(x, ref):
    x = np.asarray(x)
    ref = np.asarray(ref)
    return float(np.linalg.norm((x - ref).ravel()) / np.linalg.norm(ref.ravel()))
