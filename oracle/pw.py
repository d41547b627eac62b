"""Plane-wave sphere, real-space grid and the Kohn-Sham-like Hamiltonian.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Conventions (atomic units; cubic cell of edge L, volume Omega = L^3, FFT grid
N^3 with N_g = N^3 points, C order [i0][i1][i2]):

* G = 2 pi n / L with n in FFT order (n = i for i < N/2, else i - N).
* The plane-wave basis is the sphere {n : |G|^2 / 2 <= E_cut} (Sec. Scaling:
  N_PW components per wavefunction).  Canonical order: ascending linear grid
  index (i0 N + i1) N + i2.
* Forward transform F[k] = N_g^-1 sum_r f(r) exp(-i G_k r); inverse
  f(r) = sum_k F[k] exp(i G_k r).
* A wavefunction with sphere coefficients c is psi(r) = Omega^-1/2 u(r),
  u(r) = sum_G c_G exp(i G r).  Grid inner product <f|g> = (Omega/N_g) sum f* g.
* H_{GG'} = |G|^2/2 delta_{GG'} + V~[(n - n') mod N], V~ the forward
  transform of the sampled V_loc: exactly the operator that an FFT
  application of the local potential realises on this grid (aliasing included).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg
import scipy.sparse.linalg


def fft_n(N):
    """Integer frequencies n in FFT order."""
    return (np.fft.fftfreq(N) * N).round().astype(np.int64)


class Sphere:
    """The plane-wave sphere of a cell (Sec. Scaling: N_PW; Sec. Results)."""

    def __init__(self, L, N, ecut):
        self.L, self.N, self.ecut = float(L), int(N), float(ecut)
        n = fft_n(N)
        n0, n1, n2 = np.meshgrid(n, n, n, indexing="ij")
        nn = (n0 * n0 + n1 * n1 + n2 * n2).reshape(-1)
        g = 2.0 * np.pi / self.L
        kin = 0.5 * (g * g) * nn.astype(np.float64)
        mask = kin <= self.ecut
        self.index = np.nonzero(mask)[0]                     # linear grid index
        self.miller = np.stack([n0.reshape(-1), n1.reshape(-1), n2.reshape(-1)],
                               axis=1)[self.index]
        self.kin = kin[self.index]                           # |G|^2 / 2
        self.npw = len(self.index)
        self.ng = N ** 3
        self.omega_vol = self.L ** 3
        if np.abs(self.miller).max(initial=0) * 2 >= N:
            raise ValueError("sphere does not fit in the FFT grid")

    # -- transforms --------------------------------------------------------
    def to_grid(self, c):
        """u(r) = sum_G c_G exp(iGr) on the grid; c: (..., npw)."""
        c = np.asarray(c)
        lead = c.shape[:-1]
        g = np.zeros(lead + (self.ng,), dtype=np.complex128)
        g[..., self.index] = c
        g = g.reshape(lead + (self.N,) * 3)
        u = np.fft.ifftn(g, axes=(-3, -2, -1)) * self.ng
        return u.reshape(lead + (self.ng,))

    def fwd(self, f):
        """Full forward transform F[k] = N_g^-1 sum_r f(r) e^{-iG_k r}."""
        f = np.asarray(f)
        lead = f.shape[:-1]
        F = np.fft.fftn(f.reshape(lead + (self.N,) * 3), axes=(-3, -2, -1))
        return F.reshape(lead + (self.ng,)) / self.ng

    def inv(self, F):
        F = np.asarray(F)
        lead = F.shape[:-1]
        f = np.fft.ifftn(F.reshape(lead + (self.N,) * 3), axes=(-3, -2, -1))
        return f.reshape(lead + (self.ng,)) * self.ng

    def to_sphere(self, f):
        """Sphere components of a grid field: F[G] for G in the sphere.
        For g = u* f this is <G|psi* f> with |G> = Omega^-1/2 e^{iGr}."""
        return self.fwd(f)[..., self.index]

    def gvec_norm(self):
        """|G| on the full grid (FFT order), flattened."""
        n = fft_n(self.N)
        n0, n1, n2 = np.meshgrid(n, n, n, indexing="ij")
        g = 2.0 * np.pi / self.L
        return g * np.sqrt((n0 * n0 + n1 * n1 + n2 * n2).reshape(-1).astype(float))


def vtilde(sph: Sphere, vloc):
    """V~[m] = N_g^-1 sum_r V(r) exp(-i G_m r), as an (N,N,N) array."""
    return np.fft.fftn(np.asarray(vloc, float).reshape((sph.N,) * 3)) / sph.ng


def dense_h(sph: Sphere, vloc):
    """Dense Hermitian H_{GG'} = |G|^2/2 delta + V~[(n - n') mod N]."""
    vt = vtilde(sph, vloc)
    m = sph.miller
    H = np.empty((sph.npw, sph.npw), dtype=np.complex128)
    step = max(1, 4_000_000 // max(1, sph.npw))
    for a in range(0, sph.npw, step):
        d = (m[a:a + step, None, :] - m[None, :, :]) % sph.N
        H[a:a + step] = vt[d[..., 0], d[..., 1], d[..., 2]]
    H[np.arange(sph.npw), np.arange(sph.npw)] += sph.kin
    return H


def h_apply(sph: Sphere, vloc, c):
    """H c through the grid: kinetic diagonal plus V_loc multiplied in real
    space (Sec. Scaling: one H application costs N_FFT ln N_FFT)."""
    u = sph.to_grid(c)
    return sph.kin * c + sph.to_sphere(np.asarray(vloc, float) * u)


class GroundState:
    """Eigenpairs standing in for the DFT input (Sec. Results: DFT states
    converged to squared residual < 1e-12 Ha^2; exact diagonalisation here)."""

    def __init__(self, sph, vloc, n_occ, eps, C, eps_all=None, C_all=None):
        self.sph, self.vloc, self.n_occ = sph, np.asarray(vloc, float), n_occ
        self.eps = eps            # (n_occ,)
        self.C = C                # (n_occ, npw)  rows = occupied coefficients
        self.eps_all = eps_all    # all eigenvalues (dense route) or None
        self.C_all = C_all        # (nstates, npw) or None

    @property
    def u(self):
        """u_v(r) = Omega^1/2 psi_v(r) on the grid, (n_occ, N_g)."""
        return self.sph.to_grid(self.C)

    def gap(self):
        if self.eps_all is None:
            return None
        return self.eps_all[self.n_occ] - self.eps_all[self.n_occ - 1]


def ground_state_dense(sph, vloc, n_occ):
    H = dense_h(sph, vloc)
    e, V = np.linalg.eigh(H)
    C_all = V.T.copy()
    return GroundState(sph, vloc, n_occ, e[:n_occ].copy(), C_all[:n_occ].copy(),
                       e, C_all)


def ground_state_iterative(sph, vloc, n_occ, tol=1e-11, seed=7, maxiter=2000):
    """Lowest n_occ eigenpairs by LOBPCG (library routine) on the FFT
    H application, then a final Rayleigh-Ritz.  For cells too large for a
    dense eigensolver."""
    rng = np.random.default_rng(seed)
    nb = n_occ + max(4, n_occ // 4)
    X = rng.standard_normal((sph.npw, nb)) + 1j * rng.standard_normal((sph.npw, nb))
    X *= 1.0 / (1.0 + sph.kin)[:, None]

    def mv(Y):
        Y = np.asarray(Y)
        return h_apply(sph, vloc, Y.T).T

    A = scipy.sparse.linalg.LinearOperator((sph.npw, sph.npw), matvec=mv,
                                           matmat=mv, dtype=np.complex128)
    vt0 = vtilde(sph, vloc).reshape(-1)[0].real
    pre = 1.0 / (sph.kin + abs(vt0) + 1.0)
    M = scipy.sparse.linalg.LinearOperator(
        (sph.npw, sph.npw), matvec=lambda y: pre * np.asarray(y).reshape(-1),
        matmat=lambda Y: pre[:, None] * np.asarray(Y), dtype=np.complex128)
    e, V = scipy.sparse.linalg.lobpcg(A, X, M=M, largest=False, tol=tol,
                                      maxiter=maxiter)
    # Rayleigh-Ritz polish
    Q, _ = np.linalg.qr(V)
    HQ = mv(Q)
    h = Q.conj().T @ HQ
    w, U = np.linalg.eigh(0.5 * (h + h.conj().T))
    V = Q @ U
    order = np.argsort(w)
    w, V = w[order], V[:, order]
    return GroundState(sph, vloc, n_occ, w[:n_occ].copy(), V[:, :n_occ].T.copy(),
                       None, None), w, V.T


def residuals(sph, vloc, eps, C):
    """|(H - eps_n) psi_n| for each row of C."""
    HC = h_apply(sph, vloc, C)
    return np.linalg.norm(HC - eps[:, None] * C, axis=1)
