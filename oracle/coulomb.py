"""Square root of the Coulomb kernel, diagonal in G.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Sec. Results: isolated systems use a spherical truncation of the Coulomb
potential with radius half the cubic cell edge.  The truncated kernel is
    v(G) = 4 pi (1 - cos(|G| R_c)) / |G|^2,   v(0) = 2 pi R_c^2,  R_c = L/2,
and the bare kernel (option) is v(G) = 4 pi / |G|^2, v(0) = 0.
The symmetric dielectric operator (Eq. epsilon and its footnote) uses v^1/2,
which has only non-negative eigenvalues (Sec. Lanczos, below Eq. epsilon_nonp).
"""
from __future__ import annotations

import numpy as np

TRUNCATED, BARE = 0, 1


def vcoul(sph, kind=TRUNCATED):
    """v(G) on the full grid (FFT order), flattened."""
    G = sph.gvec_norm()
    G2 = G * G
    v = np.zeros_like(G)
    nz = G2 > 0
    if kind == TRUNCATED:
        Rc = 0.5 * sph.L
        v[nz] = 4.0 * np.pi * (1.0 - np.cos(G[nz] * Rc)) / G2[nz]
        v[~nz] = 2.0 * np.pi * Rc * Rc
    elif kind == BARE:
        v[nz] = 4.0 * np.pi / G2[nz]
    else:
        raise ValueError(kind)
    return v


def sqrt_v_apply(sph, sqv, x):
    """v^1/2 x: multiply the forward transform by sqrt(v(G)), transform back."""
    return sph.inv(sqv * sph.fwd(x))
