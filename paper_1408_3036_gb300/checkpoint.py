"""Checkpoint files of the Lanczos recursion (host side; no GPU work).

A checkpoint holds the state after k steps of gw_lanczos: the basis Q
[k][N^3], alpha [k], beta [k-1] and the frequency.  Resuming recomputes step
k - 1 from Q and continues (gw_lanczos_resume), so a checkpoint is exactly the
output of a gw_lanczos call with its basis.

File: a NumPy .npz with the arrays and a SHA-256 digest over their bytes;
load_lanczos raises CheckpointError when the file cannot be read, misses an
array, has inconsistent shapes or a digest that does not match (a damaged
file).  The library then checks the state itself (finite coefficients,
beta > 0, orthonormal vectors) before any step.
"""
from __future__ import annotations

import hashlib
import os

import numpy as np


class CheckpointError(ValueError):
    pass


def _digest(Q, alpha, beta, omega):
    h = hashlib.sha256()
    for x in (Q, alpha, beta, np.asarray([omega], np.float64)):
        x = np.ascontiguousarray(x)
        h.update(str(x.dtype).encode())
        h.update(str(x.shape).encode())
        h.update(x.tobytes())
    return h.hexdigest()


def save_lanczos(path, Q, alpha, beta, omega):
    """Write the state atomically (a temporary file, then a rename)."""
    Q = np.ascontiguousarray(np.asarray(Q, np.float64))
    k = Q.shape[0]
    alpha = np.ascontiguousarray(np.asarray(alpha, np.float64)[:k])
    beta = np.ascontiguousarray(np.asarray(beta, np.float64)[:max(k - 1, 0)])
    tmp = str(path) + ".tmp.npz"
    np.savez(tmp, Q=Q, alpha=alpha, beta=beta, omega=np.float64(omega),
             sha256=np.array(_digest(Q, alpha, beta, float(omega))))
    os.replace(tmp, path)


def load_lanczos(path):
    """(Q, alpha, beta, omega) from a checkpoint file, after its checks."""
    try:
        with np.load(path, allow_pickle=False) as f:
            Q, alpha, beta = f["Q"], f["alpha"], f["beta"]
            omega = float(f["omega"])
            digest = str(f["sha256"])
    except Exception as e:          # unreadable, truncated, missing arrays
        raise CheckpointError(f"unreadable checkpoint {path}: {e}") from e
    if Q.ndim != 2 or alpha.shape != (Q.shape[0],) or beta.shape != (max(Q.shape[0] - 1, 0),):
        raise CheckpointError(f"inconsistent checkpoint shapes in {path}")
    if _digest(Q, alpha, beta, omega) != digest:
        raise CheckpointError(f"checkpoint {path} does not match its digest (damaged)")
    return Q, alpha, beta, omega
