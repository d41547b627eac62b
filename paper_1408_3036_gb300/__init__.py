"""GB300-native Lanczos-basis dielectric matrix for Sternheimer G0W0.

Thin ctypes binding of ``libgw.so`` (C ABI in ``include/gw.h``): the functions
below carry the C names and only marshal arguments.  Every step of the path
runs in the library's CUDA kernels; there is no CPU fallback.  If the library
is missing the import succeeds but every call raises ``GwError``.

Arrays: numpy arrays are host buffers (``device_ptrs = 0``); CUDA torch
tensors are device buffers (``device_ptrs = 1``).  Complex values are
complex128 (interleaved re/im doubles).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libgw.so")

GW_FP64, GW_MIXED = 0, 1
GW_COULOMB_TRUNCATED, GW_COULOMB_BARE = 0, 1
GW_OP_STERNHEIMER, GW_OP_MODEL = 0, 1
GW_CG_PERSISTENT, GW_CG_MULTI_LAUNCH, GW_CG_CLUSTER = 0, 1, 2
GW_IMAG_SQMR, GW_IMAG_SQUARED = 0, 1
STATUS = {0: "GW_OK", 1: "GW_E_ARG", 2: "GW_E_CUDA", 3: "GW_E_NOMEM", 4: "GW_E_NOCONV",
          5: "GW_E_BREAKDOWN", 6: "GW_E_TIMEOUT", 7: "GW_E_NONFINITE", 8: "GW_E_UNSUPPORTED"}
EXPORTS = ("gw_setup", "gw_npw", "gw_sphere", "gw_set_occupied", "gw_apply_h", "gw_apply_chi0",
           "gw_apply_eps", "gw_lanczos", "gw_epsinv_elements", "gw_grad_vloc", "gw_stats",
           "gw_set_solver", "gw_set_precond", "gw_set_deflation", "gw_profile", "gw_profile_read", "gw_last_error", "gw_destroy",
           "gw_epsinv_elements_noalloc", "gw_apply_chi0_c", "gw_apply_eps_c", "gw_block_lanczos",
           "gw_epsinv_block", "gw_batch_setup", "gw_batch_size", "gw_batch_cell", "gw_batch_lanczos",
           "gw_batch_last_error", "gw_batch_destroy", "gw_set_operator", "gw_epsinv_split", "gw_sigma_p", "gw_recycle_eps", "gw_sigma_c",
           "gw_set_cg_kernel", "gw_grad_vloc_basis", "gw_set_graphs", "gw_set_imaginary_route",
           "gw_set_recycle_augment", "gw_proj_coef", "gw_set_tensor_cores",
           "gw_set_autotune", "gw_lanczos_resume")
PROFILE_CLASSES = ("z_scatter_inv", "y_inv", "x_h", "y_fwd", "z_gather_h", "proj", "cg_update",
                   "refine_fp64", "persistent_cg", "pcg_tasks", "pcg_A_busy", "pcg_A_wait", "pcg_B_busy",
                   "pcg_B_wait", "pcg_C_busy", "pcg_C_wait", "pcg_A_load", "pcg_A_sums", "pcg_A_update",
                   "pcg_A_fft", "pcg_B_load", "pcg_B_fft", "pcg_B_store", "pcg_B_unused", "pcg_C_load",
                   "pcg_C_fft", "pcg_C_dots", "pcg_C_sums")


class GwError(RuntimeError):
    def __init__(self, status, msg=""):
        self.status = status
        super().__init__(f"{STATUS.get(status, status)}: {msg}")


_lib = None


def load(path=LIB_PATH):
    """Load libgw.so (build it first with ``paper_1408_3036_gb300._build``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise GwError(2, f"libgw.so not built at {path}; the CUDA path has no fallback")
    lib = ctypes.CDLL(path)
    P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    sig = {
        "gw_setup": (I, [ctypes.POINTER(P), D, I, D, P, I, P]),
        "gw_npw": (I, [P]),
        "gw_sphere": (I, [P, P]),
        "gw_set_occupied": (I, [P, I, P, P]),
        "gw_apply_h": (I, [P, P, I, P, I, I]),
        "gw_apply_chi0": (I, [P, P, I, P, I, P, I, I]),
        "gw_apply_eps": (I, [P, P, I, P, I, P, I, I]),
        "gw_apply_chi0_c": (I, [P, P, I, P, I, P, I, I]),
        "gw_apply_eps_c": (I, [P, P, I, P, I, P, I, I]),
        "gw_lanczos": (I, [P, P, I, I, P, P, P, P, I, I]),
        "gw_lanczos_resume": (I, [P, P, P, P, I, I, P, P, P, P, I, I]),
        "gw_epsinv_elements": (I, [P, P, P, I, I, P, I]),
        "gw_epsinv_elements_noalloc": (I, [P, P, I, P, P]),
        "gw_block_lanczos": (I, [P, P, I, I, P, P, P, P, I, I]),
        "gw_epsinv_block": (I, [P, P, P, I, I, I, P, I]),
        "gw_grad_vloc": (I, [P, P, I, P, P, I, I]),
        "gw_grad_vloc_basis": (I, [P, P, P, P, P, I, P, P, I, I]),
        "gw_stats": (I, [P, P, I]),
        "gw_set_solver": (I, [P, D, D, I, I]),
        "gw_set_precond": (I, [P, I]),
        "gw_set_cg_kernel": (I, [P, I, ctypes.c_longlong]),
        "gw_set_graphs": (I, [P, I]),
        "gw_set_imaginary_route": (I, [P, I]),
        "gw_set_recycle_augment": (I, [P, D]),
        "gw_proj_coef": (I, [P, P, I, P, I]),
        "gw_set_tensor_cores": (I, [P, I]),
        "gw_set_autotune": (I, [P, I]),
        "gw_set_operator": (I, [P, I]),
        "gw_epsinv_split": (I, [P, P, I, P, P, P, I, P, P, P, I, D, P, I]),
        "gw_sigma_p": (I, [P, P, D, D, I, P, P, P, I, P, P, I, I]),
        "gw_recycle_eps": (I, [P, P, I, P, I, D, P, P, I, I]),
        "gw_sigma_c": (I, [P, I, D, D, I, P, I, I, I, P, I, I]),
        "gw_set_deflation": (I, [P, I, P, P]),
        "gw_profile": (I, [P, ctypes.c_uint]),
        "gw_profile_read": (I, [P, P, P, I]),
        "gw_last_error": (ctypes.c_char_p, [P]),
        "gw_destroy": (None, [P]),
        "gw_batch_setup": (I, [ctypes.POINTER(P), I, P, P, P, P, I, I]),
        "gw_batch_size": (I, [P]),
        "gw_batch_cell": (P, [P, I]),
        "gw_batch_lanczos": (I, [P, P, I, I, P, P, P, I, P]),
        "gw_batch_last_error": (ctypes.c_char_p, [P]),
        "gw_batch_destroy": (None, [P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _ptr(a):
    """(pointer, is_device) for a numpy array or a torch tensor."""
    if a is None:
        return None, 0
    if isinstance(a, np.ndarray):
        if not a.flags.c_contiguous:
            raise ValueError("arrays must be C contiguous")
        return a.ctypes.data, 0
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return a.data_ptr(), 1 if a.is_cuda else 0
    raise TypeError(type(a))


def _check(ctx, st):
    if st != 0:
        msg = load().gw_last_error(ctx).decode() if ctx else ""
        raise GwError(st, msg)


def _omega_buf(omegas):
    om = np.ascontiguousarray(np.asarray(omegas, dtype=np.complex128).reshape(-1))
    return om


def gw_setup(L, n_grid, ecut, vloc, coulomb=GW_COULOMB_TRUNCATED, cuda_stream=None):
    lib = load()
    v = np.ascontiguousarray(np.asarray(vloc, dtype=np.float64).reshape(-1))
    if v.size != n_grid ** 3:
        raise ValueError("vloc must hold n_grid^3 values")
    out = ctypes.c_void_p()
    st = lib.gw_setup(ctypes.byref(out), float(L), int(n_grid), float(ecut), v.ctypes.data, int(coulomb),
                      cuda_stream)
    _check(None, st)
    return out


def gw_npw(ctx):
    return load().gw_npw(ctx)


def gw_sphere(ctx):
    m = np.zeros((gw_npw(ctx), 3), dtype=np.int32)
    _check(ctx, load().gw_sphere(ctx, m.ctypes.data))
    return m


def gw_set_occupied(ctx, psi, eps):
    psi = np.ascontiguousarray(np.asarray(psi, dtype=np.complex128))
    eps = np.ascontiguousarray(np.asarray(eps, dtype=np.float64))
    _check(ctx, load().gw_set_occupied(ctx, len(eps), psi.ctypes.data, eps.ctypes.data))


def gw_apply_h(ctx, x, y, prec=GW_FP64):
    px, dx = _ptr(x)
    py, dy = _ptr(y)
    if dx != dy:
        raise ValueError("x and y must both be host or both device")
    nb = x.shape[0] if x.ndim == 2 else 1
    _check(ctx, load().gw_apply_h(ctx, px, nb, py, int(prec), dx))
    return y


def gw_apply_chi0(ctx, dV, omegas, dn, prec=GW_FP64):
    om = _omega_buf(omegas)
    p, d = _ptr(dV)
    q, e = _ptr(dn)
    if d != e:
        raise ValueError("mixed host/device buffers")
    nb = dV.shape[0] if dV.ndim == 2 else 1
    _check(ctx, load().gw_apply_chi0(ctx, p, nb, om.ctypes.data, len(om), q, int(prec), d))
    return dn


def gw_apply_eps(ctx, x, omegas, out, prec=GW_FP64):
    om = _omega_buf(omegas)
    p, d = _ptr(x)
    q, e = _ptr(out)
    if d != e:
        raise ValueError("mixed host/device buffers")
    nb = x.shape[0] if x.ndim == 2 else 1
    _check(ctx, load().gw_apply_eps(ctx, p, nb, om.ctypes.data, len(om), q, int(prec), d))
    return out


def gw_apply_chi0_c(ctx, dV, omegas, dn, prec=GW_FP64):
    om = _omega_buf(omegas)
    p, d = _ptr(dV)
    q, e = _ptr(dn)
    if d != e:
        raise ValueError("mixed host/device buffers")
    nb = dV.shape[0] if dV.ndim == 2 else 1
    _check(ctx, load().gw_apply_chi0_c(ctx, p, nb, om.ctypes.data, len(om), q, int(prec), d))
    return dn


def gw_apply_eps_c(ctx, x, omegas, out, prec=GW_FP64):
    om = _omega_buf(omegas)
    p, d = _ptr(x)
    q, e = _ptr(out)
    if d != e:
        raise ValueError("mixed host/device buffers")
    nb = x.shape[0] if x.ndim == 2 else 1
    _check(ctx, load().gw_apply_eps_c(ctx, p, nb, om.ctypes.data, len(om), q, int(prec), d))
    return out


def gw_lanczos(ctx, start, k, omega, alpha, beta, basis=None, prec=GW_FP64, blk=1):
    om = _omega_buf([omega])
    ps, d = _ptr(start)
    pa, _ = _ptr(alpha)
    pb, _ = _ptr(beta)
    pq, _ = _ptr(basis)
    _check(ctx, load().gw_lanczos(ctx, ps, int(blk), int(k), om.ctypes.data, pa, pb, pq, int(prec), d))
    return alpha, beta, basis


def gw_lanczos_resume(ctx, basis_in, alpha_in, beta_in, k0, k, omega, alpha, beta, basis=None, prec=GW_FP64):
    om = _omega_buf([omega])
    pqi, d = _ptr(basis_in)
    pai, _ = _ptr(alpha_in)
    pbi, _ = _ptr(beta_in)
    pa, _ = _ptr(alpha)
    pb, _ = _ptr(beta)
    pq, _ = _ptr(basis)
    _check(ctx, load().gw_lanczos_resume(ctx, pqi, pai, pbi, int(k0), int(k), om.ctypes.data, pa, pb, pq,
                                         int(prec), d))
    return alpha, beta, basis


def gw_block_lanczos(ctx, start, k, omega, A, B, basis=None, prec=GW_FP64):
    om = _omega_buf([omega])
    ps, d = _ptr(start)
    pa, _ = _ptr(A)
    pb, _ = _ptr(B)
    pq, _ = _ptr(basis)
    blk = start.shape[0] if start.ndim == 2 else 1
    _check(ctx, load().gw_block_lanczos(ctx, ps, int(blk), int(k), om.ctypes.data, pa, pb, pq, int(prec), d))
    return A, B, basis


def gw_epsinv_block(ctx, A, B, k, blk, bilinear, out):
    pa, d = _ptr(A)
    pb, _ = _ptr(B)
    po, _ = _ptr(out)
    _check(ctx, load().gw_epsinv_block(ctx, pa, pb, int(k), int(blk), int(bilinear), po, d))
    return out


def gw_epsinv_elements(ctx, alpha, beta, k, out, blk=1):
    pa, d = _ptr(alpha)
    pb, _ = _ptr(beta)
    po, _ = _ptr(out)
    _check(ctx, load().gw_epsinv_elements(ctx, pa, pb, int(k), int(blk), po, d))
    return out


def gw_epsinv_elements_noalloc(alpha, beta, k, out, cuda_stream=None):
    """T_K^-1 without a context or any device allocation (device tensors only);
    see include/gw.h for the shared fixed scratch and its limits.

    The kernel reads k + (k - 1) doubles and writes k * k doubles through raw
    pointers, so every buffer is checked here first: contiguous float64 CUDA
    tensors on the current device, alpha with at least k entries, beta with at
    least k - 1 (it may be None only when k == 1), out with at least k * k."""
    import torch
    k = int(k)
    if k < 1:
        raise ValueError("k must be >= 1")
    cur = torch.cuda.current_device()

    def need(name, t, n):
        if not isinstance(t, torch.Tensor) or not t.is_cuda:
            raise ValueError(f"{name} must be a CUDA tensor")
        if t.dtype != torch.float64:
            raise ValueError(f"{name} must be float64")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
        if t.device.index != cur:
            raise ValueError(f"{name} is on cuda:{t.device.index}, the current device is cuda:{cur}")
        if t.numel() < n:
            raise ValueError(f"{name} holds {t.numel()} values, {n} needed")
        return t.data_ptr()

    pa = need("alpha", alpha, k)
    if beta is None:
        if k > 1:
            raise ValueError("beta is required for k > 1")
        pb = None
    else:
        pb = need("beta", beta, k - 1)
    po = need("out", out, k * k)
    _check(None, load().gw_epsinv_elements_noalloc(pa, pb, k, po, cuda_stream))
    return out


def gw_grad_vloc(ctx, phi, k, s, grad, prec=GW_FP64):
    pp, d = _ptr(phi)
    ps, _ = _ptr(s)
    pg, _ = _ptr(grad)
    _check(ctx, load().gw_grad_vloc(ctx, pp, int(k), ps, pg, int(prec), d))
    return s, grad


def gw_grad_vloc_basis(ctx, phi, basis, alpha, beta, k, s, grad, prec=GW_FP64):
    """s and ds/dV_loc from a kept Lanczos basis (gw_lanczos at omega = 0 from phi)."""
    pp, d = _ptr(phi)
    pq, d2 = _ptr(basis)
    pa, d3 = _ptr(alpha)
    pb, d4 = _ptr(beta)
    ps, d5 = _ptr(s)
    pg, d6 = _ptr(grad)
    if len({d, d2, d3, d5, d6} | ({d4} if beta is not None else set())) != 1:
        raise ValueError("mixed host/device buffers")
    _check(ctx, load().gw_grad_vloc_basis(ctx, pp, pq, pa, pb, int(k), ps, pg, int(prec), d))
    return s, grad


def gw_stats(ctx):
    out = np.zeros(12)
    _check(ctx, load().gw_stats(ctx, out.ctypes.data, 12))
    return dict(columns=out[0], max_iter=out[1], mean_iter=out[2], outer=out[3], max_residual=out[4],
                h_columns=out[5], launches=int(out[6]), launch_iterations=int(out[7]), launch_ctas=int(out[8]),
                cluster=int(out[9]), graph_replays=int(out[10]), cta_threads=int(out[11]))


def gw_set_autotune(ctx, on):
    _check(ctx, load().gw_set_autotune(ctx, int(on)))


def gw_proj_coef(ctx, y, coef, kernel=1):
    """coef [n_proj][ncol] complex128 = <C_v|y_j> for y [ncol][N_PW] complex64 (both CUDA tensors)."""
    py, d = _ptr(y)
    pc, d2 = _ptr(coef)
    if not (d and d2):
        raise ValueError("device buffers required")
    _check(ctx, load().gw_proj_coef(ctx, py, int(y.shape[0]), pc, int(kernel)))
    return coef


def gw_set_tensor_cores(ctx, on):
    _check(ctx, load().gw_set_tensor_cores(ctx, int(on)))


def gw_set_recycle_augment(ctx, w0):
    """Recycled bases augmented with x(i w0) (w0 > 0), or not (0)."""
    _check(ctx, load().gw_set_recycle_augment(ctx, float(w0)))


def gw_set_imaginary_route(ctx, route):
    """GW_IMAG_SQMR (default) or GW_IMAG_SQUARED (Eq. P2+) at purely imaginary frequencies."""
    _check(ctx, load().gw_set_imaginary_route(ctx, int(route)))


def gw_set_graphs(ctx, on):
    """SQMR iterations replayed from a captured CUDA graph (1, default) or launched one by one (0)."""
    _check(ctx, load().gw_set_graphs(ctx, int(on)))


def gw_set_solver(ctx, tol=0.0, tol_inner=0.0, max_iter=0, max_outer=0):
    _check(ctx, load().gw_set_solver(ctx, float(tol), float(tol_inner), int(max_iter), int(max_outer)))


def gw_set_deflation(ctx, psi, eps):
    """Lowest conduction states (rows of psi, sphere order) as a deflation block."""
    psi = np.ascontiguousarray(np.asarray(psi, np.complex128))
    eps = np.ascontiguousarray(np.asarray(eps, np.float64))
    n = len(eps)
    _check(ctx, load().gw_set_deflation(ctx, n, psi.ctypes.data if n else None, eps.ctypes.data if n else None))


def gw_set_precond(ctx, kind):
    _check(ctx, load().gw_set_precond(ctx, int(kind)))


def gw_set_cg_kernel(ctx, kind, wait_limit=0):
    """GW_CG_PERSISTENT, GW_CG_MULTI_LAUNCH or GW_CG_CLUSTER, and the bound on the
    persistent kernel's device waits (0 keeps it)."""
    _check(ctx, load().gw_set_cg_kernel(ctx, int(kind), int(wait_limit)))


def gw_set_operator(ctx, op):
    """GW_OP_STERNHEIMER (Eqs. P1, P2) or GW_OP_MODEL (Eq. model_eq)."""
    _check(ctx, load().gw_set_operator(ctx, int(op)))


def gw_epsinv_split(ctx, phi, basis, alpha, beta, basis_m, alpha_m, beta_m, omega, out):
    """<phi_i|eps~^-1 - 1|phi_j> from the Sternheimer basis (basis, alpha, beta)
    and the model basis (basis_m, alpha_m, beta_m), Eq. subs_epsilon."""
    pp, d = _ptr(phi)
    m = phi.shape[0] if phi.ndim == 2 else 1
    k, km = len(alpha), len(alpha_m)
    pq, _ = _ptr(basis)
    pa, _ = _ptr(alpha)
    pb, _ = _ptr(beta)
    pqm, _ = _ptr(basis_m)
    pam, _ = _ptr(alpha_m)
    pbm, _ = _ptr(beta_m)
    po, e = _ptr(out)
    if d != e:
        raise ValueError("mixed host/device buffers")
    _check(ctx, load().gw_epsinv_split(ctx, pp, int(m), pq, pa, pb, int(k), pqm, pam, pbm, int(km),
                                       float(omega), po, d))
    return out


def gw_sigma_p(ctx, psi_e, eps_e, delta, psi, eps, occ, k, sigma, terms=None, prec=GW_FP64):
    """Sigma^P_e(delta) of Eq. pe (one k-step Lanczos per pole); see include/gw.h."""
    pe, d = _ptr(psi_e)
    n = len(eps)
    pp, _ = _ptr(psi)
    pe2, _ = _ptr(eps)
    po, _ = _ptr(occ)
    ps, e = _ptr(sigma)
    pt, _ = _ptr(terms)
    if d != e:
        raise ValueError("mixed host/device buffers")
    _check(ctx, load().gw_sigma_p(ctx, pe, float(eps_e), float(delta), int(n), pp, pe2, po, int(k), ps, pt,
                                  int(prec), d))
    return sigma, terms


def gw_recycle_eps(ctx, fields, w, out, rtol=0.0, prec=GW_FP64):
    """<l|eps~(i w) - 1|l'> for every w from recycled per-state bases (Eq. recy_eq).
    Returns the smallest number of recycled directions kept over the states."""
    pf, d = _ptr(fields)
    nl = fields.shape[0] if fields.ndim == 2 else 1
    pw_, _ = _ptr(w)
    po, e = _ptr(out)
    if d != e:
        raise ValueError("mixed host/device buffers")
    kept = ctypes.c_int(0)
    _check(ctx, load().gw_recycle_eps(ctx, pf, int(nl), pw_, int(len(w)), float(rtol), po, ctypes.byref(kept),
                                      int(prec), d))
    return kept.value


def gw_sigma_c(ctx, e, delta, alpha, n_freq, fields, k_h, k_p, out, prec=GW_FP64):
    """Sigma^c of occupied state e (Eq. e_c): out[4] = total, integral, Sigma^A, Sigma^P."""
    pf, d = _ptr(fields)
    nl = fields.shape[0] if fields.ndim == 2 else 1
    po, e2 = _ptr(out)
    if d != e2:
        raise ValueError("mixed host/device buffers")
    _check(ctx, load().gw_sigma_c(ctx, int(e), float(delta), float(alpha), int(n_freq), pf, int(nl), int(k_h),
                                  int(k_p), po, int(prec), d))
    return out


def gw_profile(ctx, mask):
    _check(ctx, load().gw_profile(ctx, int(mask)))


def gw_profile_read(ctx):
    n = len(PROFILE_CLASSES)
    ms = np.zeros(n)
    cnt = np.zeros(n, dtype=np.int64)
    _check(ctx, load().gw_profile_read(ctx, ms.ctypes.data, cnt.ctypes.data, n))
    return {k: (float(ms[i]), int(cnt[i])) for i, k in enumerate(PROFILE_CLASSES)}


def gw_last_error(ctx):
    return load().gw_last_error(ctx).decode()


def gw_destroy(ctx):
    if ctx:
        load().gw_destroy(ctx)


class Cell:
    """Convenience owner of one context (setup ... destroy)."""

    def __init__(self, L, n_grid, ecut, vloc, coulomb=GW_COULOMB_TRUNCATED, cuda_stream=None, _ctx=None):
        self.L, self.N, self.ecut = float(L), int(n_grid), float(ecut)
        self.owned = _ctx is None
        self.ctx = gw_setup(L, n_grid, ecut, vloc, coulomb, cuda_stream) if _ctx is None else _ctx
        self.npw = gw_npw(self.ctx)
        self.ng = self.N ** 3

    def close(self):
        if self.ctx and self.owned:
            gw_destroy(self.ctx)
        self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sphere(self):
        return gw_sphere(self.ctx)

    def set_occupied(self, psi, eps):
        gw_set_occupied(self.ctx, psi, eps)
        self.n_occ = len(eps)

    def apply_h(self, x, prec=GW_FP64):
        x = np.ascontiguousarray(np.atleast_2d(np.asarray(x, np.complex128)))
        y = np.empty_like(x)
        return gw_apply_h(self.ctx, x, y, prec)

    def apply_chi0(self, dV, omegas=(0.0,), prec=GW_FP64):
        cplx_out = bool(np.any(np.imag(np.asarray(omegas, complex)) != 0))
        if np.iscomplexobj(dV):
            dV = np.ascontiguousarray(np.atleast_2d(np.asarray(dV, np.complex128)))
            dn = np.empty((len(omegas), dV.shape[0], self.ng), np.complex128)
            return gw_apply_chi0_c(self.ctx, dV, omegas, dn, prec)
        dV = np.ascontiguousarray(np.atleast_2d(np.asarray(dV, np.float64)))
        dn = np.empty((len(omegas), dV.shape[0], self.ng), np.complex128 if cplx_out else np.float64)
        return gw_apply_chi0(self.ctx, dV, omegas, dn, prec)

    def apply_eps(self, x, omegas=(0.0,), prec=GW_FP64):
        cplx_out = bool(np.any(np.imag(np.asarray(omegas, complex)) != 0))
        if np.iscomplexobj(x):
            x = np.ascontiguousarray(np.atleast_2d(np.asarray(x, np.complex128)))
            out = np.empty((len(omegas), x.shape[0], self.ng), np.complex128)
            return gw_apply_eps_c(self.ctx, x, omegas, out, prec)
        x = np.ascontiguousarray(np.atleast_2d(np.asarray(x, np.float64)))
        out = np.empty((len(omegas), x.shape[0], self.ng), np.complex128 if cplx_out else np.float64)
        return gw_apply_eps(self.ctx, x, omegas, out, prec)

    def lanczos(self, start, k, omega=0.0, prec=GW_FP64, basis=False):
        start = np.ascontiguousarray(np.asarray(start, np.float64).reshape(-1))
        a = np.empty(k)
        b = np.empty(max(k - 1, 1))
        Q = np.empty((k, self.ng)) if basis else None
        gw_lanczos(self.ctx, start, k, omega, a, b, Q, prec)
        return a, b[:k - 1], Q

    def lanczos_resume(self, Q, alpha, beta, k, omega=0.0, prec=GW_FP64):
        """Continue a recursion from a saved state: Q rows q_1 .. q_{k0+1},
        alpha[:k0], beta[:k0] (k0 = len(Q) - 1); returns alpha [k], beta [k-1]
        and the basis [k][N^3] of the k-step recursion."""
        Q = np.ascontiguousarray(np.asarray(Q, np.float64))
        k0 = Q.shape[0] - 1
        ai = np.ascontiguousarray(np.asarray(alpha, np.float64)[:k0])
        bi = np.ascontiguousarray(np.asarray(beta, np.float64)[:k0])
        if ai.size != k0 or bi.size != k0:
            raise ValueError("a saved state with k0 + 1 vectors needs k0 alpha and k0 beta values")
        a = np.empty(k)
        b = np.empty(max(k - 1, 1))
        Qo = np.empty((k, self.ng))
        gw_lanczos_resume(self.ctx, Q, ai, bi, k0, k, omega, a, b, Qo, prec)
        return a, b[:k - 1], Qo

    def lanczos_checkpointed(self, start, k, path, every, omega=0.0, prec=GW_FP64):
        """k Lanczos steps in segments of ``every`` steps, the state written to
        ``path`` (checkpoint.save_lanczos) after each segment; returns alpha,
        beta, basis as ``lanczos``."""
        from .checkpoint import save_lanczos
        k1 = min(max(int(every), 2), k)
        a, b, Q = self.lanczos(start, k1, omega, prec, basis=True)
        save_lanczos(path, Q, a, b, omega)
        while k1 < k:
            k2 = min(k1 + every, k)
            a, b, Q = self.lanczos_resume(Q, a[:k1 - 1], b[:k1 - 1], k2, omega, prec)
            save_lanczos(path, Q, a, b, omega)
            k1 = k2
        return a, b, Q

    def lanczos_from_checkpoint(self, path, k, prec=GW_FP64):
        """Continue to k steps from a checkpoint file (checked: checksum in
        load_lanczos, then the state itself in gw_lanczos_resume)."""
        from .checkpoint import load_lanczos
        Q, a, b, omega = load_lanczos(path)
        k1 = Q.shape[0]
        return self.lanczos_resume(Q, a[:k1 - 1], b[:k1 - 1], k, omega, prec)

    def block_lanczos(self, start, k, omega=0.0, prec=GW_FP64, basis=False):
        start = np.ascontiguousarray(np.atleast_2d(np.asarray(start, np.float64)))
        blk = start.shape[0]
        A = np.empty((k, blk, blk), np.complex128)
        B = np.zeros((max(k - 1, 1), blk, blk), np.complex128)
        Q = np.empty((k * blk, self.ng), np.complex128) if basis else None
        gw_block_lanczos(self.ctx, start, k, omega, A, B, Q, prec)
        return A, B[:k - 1], Q

    def epsinv_block(self, A, B, bilinear=False):
        k, blk = A.shape[0], A.shape[1]
        out = np.empty((k * blk, k * blk), np.complex128)
        Bb = np.ascontiguousarray(B if len(B) else np.zeros((1, blk, blk), np.complex128), np.complex128)
        return gw_epsinv_block(self.ctx, np.ascontiguousarray(A, np.complex128), Bb, k, blk, bilinear, out)

    def epsinv(self, alpha, beta):
        k = len(alpha)
        out = np.empty((k, k))
        a = np.ascontiguousarray(alpha, np.float64)
        b = np.ascontiguousarray(beta if len(beta) else np.zeros(1), np.float64)
        return gw_epsinv_elements(self.ctx, a, b, k, out)

    def grad_vloc(self, phi, k, prec=GW_FP64):
        phi = np.ascontiguousarray(np.asarray(phi, np.float64).reshape(-1))
        s = np.zeros(1)
        g = np.empty(self.ng)
        gw_grad_vloc(self.ctx, phi, k, s, g, prec)
        return s[0], g

    def stats(self):
        return gw_stats(self.ctx)

    def set_solver(self, **kw):
        gw_set_solver(self.ctx, **kw)

    def set_precond(self, kind):
        gw_set_precond(self.ctx, kind)

    def set_autotune(self, on):
        gw_set_autotune(self.ctx, on)

    def set_tensor_cores(self, on):
        gw_set_tensor_cores(self.ctx, on)

    def set_recycle_augment(self, w0):
        gw_set_recycle_augment(self.ctx, w0)

    def set_imaginary_route(self, route):
        gw_set_imaginary_route(self.ctx, route)

    def set_graphs(self, on):
        gw_set_graphs(self.ctx, on)

    def set_cg_kernel(self, kind, wait_limit=0):
        gw_set_cg_kernel(self.ctx, kind, wait_limit)

    def set_operator(self, op):
        gw_set_operator(self.ctx, op)

    def sigma_p(self, psi_e, eps_e, delta, psi, eps, occ, k=4, prec=GW_FP64):
        """Sigma^P_e(delta) and the term of every candidate state (host arrays)."""
        pe = np.ascontiguousarray(np.asarray(psi_e, np.complex128).reshape(-1))
        pp = np.ascontiguousarray(np.atleast_2d(np.asarray(psi, np.complex128)))
        ee = np.ascontiguousarray(np.asarray(eps, np.float64).reshape(-1))
        oo = np.ascontiguousarray(np.asarray(occ, np.int32).reshape(-1))
        sg = np.zeros(1)
        tt = np.zeros(len(ee))
        gw_sigma_p(self.ctx, pe, eps_e, delta, pp, ee, oo, k, sg, tt, prec)
        return float(sg[0]), tt

    def recycle_eps(self, fields, w, rtol=0.0, prec=GW_FP64):
        """(out [nw][nl][nl], kept) for imaginary frequencies w (host arrays)."""
        F = np.ascontiguousarray(np.atleast_2d(np.asarray(fields, np.float64)))
        ww = np.ascontiguousarray(np.asarray(w, np.float64).reshape(-1))
        out = np.zeros((len(ww), F.shape[0], F.shape[0]))
        kept = gw_recycle_eps(self.ctx, F, ww, out, rtol, prec)
        return out, kept

    def sigma_c(self, e, delta, fields, alpha=1.0, n_freq=8, k_h=8, k_p=4, prec=GW_FP64):
        """dict(total, integral, SA, SP) of Eq. e_c for occupied state e (host arrays)."""
        F = np.ascontiguousarray(np.atleast_2d(np.asarray(fields, np.float64)))
        out = np.zeros(4)
        gw_sigma_c(self.ctx, e, delta, alpha, n_freq, F, k_h, k_p, out, prec)
        return dict(total=out[0], integral=out[1], SA=out[2], SP=out[3])

    def epsinv_split(self, phi, lz, lz_model, omega=0.0):
        """Eq. subs_epsilon from two host Lanczos results (alpha, beta, basis)."""
        phi = np.ascontiguousarray(np.atleast_2d(np.asarray(phi, np.float64)))
        a, b, Q = (np.ascontiguousarray(np.asarray(x, np.float64)) for x in lz)
        am, bm, Qm = (np.ascontiguousarray(np.asarray(x, np.float64)) for x in lz_model)
        out = np.zeros((phi.shape[0], phi.shape[0]))
        return gw_epsinv_split(self.ctx, phi, Q, a, b, Qm, am, bm, omega, out)

    def set_deflation(self, psi, eps):
        gw_set_deflation(self.ctx, psi, eps)


def _check_batch(b, st):
    if st != 0:
        msg = load().gw_batch_last_error(b).decode() if b else ""
        raise GwError(st, msg)


def gw_batch_setup(cells, coulomb=GW_COULOMB_TRUNCATED, workers=0):
    """cells: list of (L, n_grid, ecut, vloc).  Returns the batch handle."""
    lib = load()
    vs = [np.ascontiguousarray(np.asarray(c[3], np.float64).reshape(-1)) for c in cells]
    for c, v in zip(cells, vs):
        if v.size != int(c[1]) ** 3:
            raise ValueError("vloc must hold n_grid^3 values")
    n = len(cells)
    L = np.array([c[0] for c in cells], np.float64)
    N = np.array([c[1] for c in cells], np.int32)
    E = np.array([c[2] for c in cells], np.float64)
    vp = (ctypes.c_void_p * n)(*[v.ctypes.data for v in vs])
    out = ctypes.c_void_p()
    _check_batch(None, lib.gw_batch_setup(ctypes.byref(out), n, L.ctypes.data, N.ctypes.data, E.ctypes.data,
                                          ctypes.cast(vp, ctypes.c_void_p), int(coulomb), int(workers)))
    return out.value


def gw_batch_size(b):
    return load().gw_batch_size(b)


def gw_batch_cell(b, i):
    return load().gw_batch_cell(b, int(i))


def gw_batch_lanczos(b, starts, k, omegas, alpha, beta, prec=GW_FP64, status=None):
    """omegas: (n_cells, n_omega) complex, or (n_omega,) shared by all cells."""
    n = len(starts)
    sp = (ctypes.c_void_p * n)(*[x.ctypes.data for x in starts])
    om = np.asarray(omegas, np.complex128)
    om = np.ascontiguousarray(np.broadcast_to(om, (n, om.shape[-1])))
    ps = status.ctypes.data if status is not None else None
    _check_batch(b, load().gw_batch_lanczos(b, ctypes.cast(sp, ctypes.c_void_p), int(k), int(om.shape[1]),
                                            om.ctypes.data, alpha.ctypes.data, beta.ctypes.data, int(prec), ps))
    return alpha, beta


def gw_batch_last_error(b):
    return load().gw_batch_last_error(b).decode()


def gw_batch_destroy(b):
    load().gw_batch_destroy(b)


class Batch:
    """Independent cells run concurrently (gw_batch_*).  ``cells`` is a list of
    (L, n_grid, ecut, vloc); ``cell(i)`` is a non-owning Cell view of cell i."""

    def __init__(self, cells, coulomb=GW_COULOMB_TRUNCATED, workers=0):
        self.b = gw_batch_setup(cells, coulomb, workers)
        self.cells = [Cell(c[0], c[1], c[2], None, _ctx=gw_batch_cell(self.b, i)) for i, c in enumerate(cells)]

    def __len__(self):
        return gw_batch_size(self.b)

    def cell(self, i):
        return self.cells[i]

    def lanczos(self, starts, k, omegas, prec=GW_FP64):
        """alpha [n_cells][n_omega][k], beta [..][k-1] (complex), per-cell status.
        A failing cell raises GwError after all cells ran; see ``last_status``."""
        n = len(self.cells)
        st = [np.ascontiguousarray(np.asarray(x, np.float64).reshape(-1)) for x in starts]
        if len(st) != n:
            raise ValueError("one start field per cell")
        for c, x in zip(self.cells, st):
            if x.size != c.ng:
                raise ValueError("start field size does not match its cell")
        n_om = np.asarray(omegas).shape[-1]
        A = np.empty((n, n_om, k), np.complex128)
        B = np.empty((n, n_om, max(k - 1, 0)), np.complex128)
        self.last_status = np.zeros(n, np.int32)
        gw_batch_lanczos(self.b, st, k, omegas, A, B, prec, self.last_status)
        return A, B

    def close(self):
        if getattr(self, "b", None):
            for c in self.cells:
                c.ctx = None
            gw_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
