"""Lanczos recursion on the dielectric operator and its inverse in the
Lanczos basis.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Sec. Lanczos: the Krylov space of eps - 1 (Eq. krylov) is built by the Lanczos
procedure, which tridiagonalises the operator; each residual is
re-orthogonalised by Gram-Schmidt against all previous Lanczos vectors (the
paper's vectors lose orthogonality in about ten steps without it); the
tridiagonal matrix is then inverted (cost ~ N^2 for a tridiagonal matrix).

Readings:
* The recursion runs on eps~ itself; alpha(eps~ - 1) = alpha - 1 and beta is
  unchanged.
* "Gram-Schmidt" is classical Gram-Schmidt applied twice (CGS2).
* Inner product on grid fields: <f|g> = (Omega/N_g) sum_r f* g (Hermitian), or
  the bilinear form (Omega/N_g) sum_r f g for complex-symmetric operators
  (complex frequency).
* Step k: w = A q_k - beta_{k-1} q_{k-1}; alpha_k = <q_k|w>; w -= alpha_k q_k;
  w -= Q (Q^H w) twice; beta_k = |w|; q_{k+1} = w / beta_k.
* The inverse dielectric matrix in the Lanczos basis is T_K^-1 (dense solve);
  for a start vector phi, <phi|eps^-1|phi> ~ |phi|^2 (T_K^-1)_11.
* Sec. Dielectric model (Eq. subs_epsilon): eps^-1 - 1 is split into
  (eps^-1 - eps_m^-1), taken in the exact Lanczos basis, and (eps_m^-1 - 1),
  taken in the Lanczos basis of the model operator (``epsinv_split``).
"""
from __future__ import annotations

import numpy as np


def _ip(weight, bilinear):
    if bilinear:
        return lambda a, b: weight * np.sum(a * b)
    return lambda a, b: weight * np.vdot(a, b)


def lanczos(apply, x0, K, weight=1.0, reorth=2, bilinear=False, breakdown=None):
    """Single-vector Lanczos.  Returns (alpha[K], beta[K-1], Q (K, n)).
    With ``breakdown`` set, the recursion stops after step k when
    |beta_k| <= breakdown |alpha_k| (an invariant subspace: alpha, beta and Q
    then have k + 1, k and k + 1 entries)."""
    ip = _ip(weight, bilinear)
    x0 = np.asarray(x0)
    nrm = np.sqrt(ip(x0, x0))
    q = x0 / nrm
    Q = [q]
    alpha, beta = [], []
    for k in range(K):
        w = apply(Q[k])
        if k > 0:
            w = w - beta[k - 1] * Q[k - 1]
        a = ip(Q[k], w)
        w = w - a * Q[k]
        for _ in range(reorth):
            Qm = np.array(Q)
            if bilinear:
                h = weight * (Qm @ w)
            else:
                h = weight * (np.conj(Qm) @ w)
            w = w - h @ Qm
        alpha.append(a)
        if k == K - 1:
            break
        b = np.sqrt(ip(w, w))
        if breakdown is not None and abs(b) <= breakdown * abs(a):
            break
        beta.append(b)
        Q.append(w / b)
    return np.array(alpha), np.array(beta), np.array(Q)


def tridiag(alpha, beta):
    T = np.diag(np.asarray(alpha)).astype(np.result_type(alpha, beta, float))
    b = np.asarray(beta)
    if len(b):
        T = T + np.diag(b, 1) + np.diag(b, -1)
    return T


def block_lanczos(apply, X0, K, weight=1.0, bilinear=False):
    """Block Lanczos with full (CGS2, block) re-orthogonalisation.

    Q_{k+1} B_k = A Q_k - Q_k A_k - Q_{k-1} B_{k-1}^T   (bilinear: ^T)
    or ... - Q_{k-1} B_{k-1}^H (Hermitian).  Blocks are rows: Q_k is (b, n).
    Normalisation of a block W: Hermitian case, Householder QR with positive
    R diagonal (Cholesky of the Gram matrix, same factor); bilinear case,
    complex Cholesky of W W^T with principal square roots.
    In row form (rows are vectors) the recursion reads
        W = A(Q_k) - A_k^T Q_k - B_{k-1}^(*) Q_{k-1},
    with A_k[i, j] = <q_i|A q_j> and ^(*) complex conjugation in the
    Hermitian case.
    Returns (A: (K, b, b), B: (K-1, b, b), Q: (K*b, n)).
    """
    X0 = np.atleast_2d(np.asarray(X0))
    b = X0.shape[0]
    def gram(Y, Z):
        return weight * ((Y if bilinear else np.conj(Y)) @ Z.T)

    def normalise(W):
        G = gram(W, W)
        R = _chol_upper(G, bilinear)       # G = R^T R (bilinear) or R^H R
        Q = np.linalg.solve(R.T, W)            # rows of W R^-1
        return Q, R

    Qk, _ = normalise(X0)
    Qs = [Qk]
    As, Bs = [], []
    for k in range(K):
        W = apply(Qs[k])                       # rows
        if k > 0:
            Bp = Bs[k - 1] if bilinear else np.conj(Bs[k - 1])
            W = W - Bp @ Qs[k - 1]             # rows of Q_{k-1} B_{k-1}^{T/H}
        Ak = gram(Qs[k], W)                    # b x b: <q_i|w_j>
        W = W - Ak.T @ Qs[k]
        for _ in range(2):
            Qm = np.concatenate(Qs, axis=0)
            H = gram(Qm, W)
            W = W - H.T @ Qm
        As.append(Ak)
        if k == K - 1:
            break
        Qn, Bk = normalise(W)
        Bs.append(Bk)
        Qs.append(Qn)
    return np.array(As), np.array(Bs), np.concatenate(Qs, axis=0)


def _chol_upper(G, bilinear):
    """Upper factor R with G = R^H R (Hermitian) or G = R^T R (bilinear,
    complex symmetric; principal square roots on the diagonal)."""
    n = G.shape[0]
    R = np.zeros_like(G, dtype=np.result_type(G, complex if bilinear else G.dtype))
    for i in range(n):
        if bilinear:
            s = G[i, i] - np.sum(R[:i, i] * R[:i, i])
            R[i, i] = np.sqrt(s + 0j)
            for j in range(i + 1, n):
                R[i, j] = (G[i, j] - np.sum(R[:i, i] * R[:i, j])) / R[i, i]
        else:
            s = (G[i, i] - np.sum(np.conj(R[:i, i]) * R[:i, i])).real
            if s <= 0:
                raise np.linalg.LinAlgError("block Lanczos breakdown")
            R[i, i] = np.sqrt(s)
            for j in range(i + 1, n):
                R[i, j] = (G[i, j] - np.sum(np.conj(R[:i, i]) * R[:i, j])) / R[i, i]
    return R


def block_tridiag(As, Bs, bilinear=False):
    """Assemble the (K b) x (K b) block tridiagonal T = Q^H A Q (or Q^T A Q)
    with diagonal blocks A_k, B_k below and B_k^H (bilinear: B_k^T) above."""
    K, b = len(As), As[0].shape[0]
    T = np.zeros((K * b, K * b), dtype=np.result_type(As[0], float))
    for k in range(K):
        T[k * b:(k + 1) * b, k * b:(k + 1) * b] = As[k]
    for k in range(K - 1):
        T[(k + 1) * b:(k + 2) * b, k * b:(k + 1) * b] = Bs[k]
        T[k * b:(k + 1) * b, (k + 1) * b:(k + 2) * b] = (
            Bs[k].T if bilinear else np.conj(Bs[k]).T)
    return T


def epsinv_lanczos(alpha, beta):
    """T_K^-1: the inverse dielectric matrix in the Lanczos basis (dense)."""
    return np.linalg.inv(tridiag(alpha, beta))


def quad_s(alpha, beta, phi_norm2):
    """s_K = |phi|^2 (T_K^-1)_11 (Gauss quadrature estimate of <phi|A^-1|phi>)."""
    Ti = epsinv_lanczos(alpha, beta)
    return phi_norm2 * Ti[0, 0]


# ---------------------------------------------------------------------------
# Sec. Dielectric model, Eq. subs_epsilon: eps^-1 - 1 split over two bases
# ---------------------------------------------------------------------------
def compress(apply, Q, weight=1.0):
    """<Q|A Q>: the operator A in the orthonormal basis Q (rows), one
    application per basis vector; M[i][j] = weight sum_r Q_i(r) (A Q_j)(r)."""
    Q = np.asarray(Q)
    AQ = np.array([apply(q) for q in Q])
    return weight * (np.conj(Q) @ AQ.T)


def epsinv_split(a, T, M, a_m, T_m):
    """<phi_i|eps^-1 - 1|phi_j> by Eq. subs_epsilon,
        eps^-1 - 1 = (eps^-1 - eps_m^-1) + (eps_m^-1 - 1),
    the first part in the basis {l} of the exact operator, the second in the
    basis {l~} of the model operator:
        a_i^T (T^-1 - M^-1) a_j + a~_i^T (T~^-1 - 1) a~_j,
    with T = <l|eps l'> (the Lanczos matrix), M = <l|eps_m l'> (the model in
    the exact basis, from ``compress``), T~ = <l~|eps_m l~'> and the fields'
    coefficients a = <l|phi> (m x k), a~ = <l~|phi> (m x k~).  Reading: in the
    exact basis the model operator is compressed and then inverted, the same
    way T^-1 stands for eps^-1 there."""
    a, a_m = np.atleast_2d(a), np.atleast_2d(a_m)
    D = np.linalg.inv(T) - np.linalg.inv(M)
    D_m = np.linalg.inv(T_m) - np.eye(len(T_m))
    return a @ D @ a.T + a_m @ D_m @ a_m.T
