"""The oracle's Sternheimer route of Eq. P1 with its per-state solves spread
over a process pool (test infrastructure; spawn start method, one BLAS thread
per worker).  The arithmetic is the oracle's own (response.chi0_sternheimer
restricted to one occupied state per task); only the sum over states is
distributed."""
import multiprocessing as mp
import os

import numpy as np

_ST = {}


def _init(L, N, ecut, vloc, C, eps, gaps):
    from oracle import pw
    sph = pw.Sphere(L, N, ecut)
    _ST["gs"] = pw.GroundState(sph, vloc, len(eps), eps, C)
    _ST["gaps"] = gaps


def _term(args):
    y, v, tol = args
    from oracle import response
    return response.chi0_sternheimer(_ST["gs"], y, 0.0, tol, _ST["gaps"], states=[v])


class Chi0Pool:
    """chi0(0) f = sum over occupied states, one state per task."""

    def __init__(self, cell, gs, gaps, workers=None):
        self.n_occ = gs.n_occ
        n = workers or max(1, min(os.cpu_count() or 1, gs.n_occ))
        saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS")}
        os.environ.update({k: "1" for k in saved})
        try:
            self.pool = mp.get_context("spawn").Pool(
                n, initializer=_init, initargs=(cell.L, cell.N, cell.ecut, cell.vloc, gs.C, gs.eps, gaps))
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v

    def chi0(self, y, tol=1e-14):
        parts = self.pool.map(_term, [(np.asarray(y), v, tol) for v in range(self.n_occ)])
        return sum(parts)

    def close(self):
        self.pool.terminate()
