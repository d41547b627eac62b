"""Benchmark: eps~ applications per second on one GB300 (mixed vs FP64).

Workload (molecule-sized static screening, the configuration the headline
metric is quoted on): cubic cell L = 20 bohr, 48^3 grid, 10 Ha cutoff
(~12k plane waves), 8 seeded Gaussian wells (D = -3 Ha, sigma = 0.8 bohr),
16 occupied states, omega = 0, 100 Lanczos steps with full
re-orthogonalisation.  One step = one complete 100-step Lanczos run = 100 eps~
applications (unit of work: one eps~ application to one column at one omega).

Inputs are synthetic (workloads.py); the occupied states come from the
library's own H application inside a block LOBPCG (input preparation, not
timed).  Inside a step the 16-column working set (~14 MB) stays in L2; L2 is
flushed between timed steps by writing a 512 MB buffer.

Beside the headline, ``model_operator`` times the same Lanczos run on the
model dielectric operator of Sec. Dielectric model (Eq. model_eq, H -> T:
one kinetic division per Sternheimer solve) on the same cell and start
vector (``--model-k 0`` skips it), and ``sigma_p`` times the residue term of
Eq. pe for the highest occupied state, one four-step Lanczos per pole at its
real frequency (``--sigma-p-k 0`` skips it), and ``recycle`` builds
eps~(i w) - 1 in the first Lanczos vectors at many imaginary frequencies from
one recycled basis per occupied state (Eq. recy_eq; ``--recycle-nl 0`` skips
it), against one direct application at w = 0.5i; ``sigma_c`` times the
correlation self-energy of the highest occupied state (Eq. e_c) in the first
eight Lanczos vectors (``--sigma-c-nl 0`` skips it).

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle
instead, on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "eps~ applies/sec & % HBM roofline, mixed vs FP64 GPU at <=1e-6 rel err"
UNIT = "applies/s"
WORKLOAD = ("molecule static screening: L=20 bohr, grid 48^3, ecut 10 Ha (12053 PW), 8 Gaussian wells "
            "(D=-3 Ha, sigma=0.8 bohr), N_occ=16, omega=0, K=100 Lanczos steps, CGS2")


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ---------------------------------------------------------------------------
# oracle timing (reported baseline; runs before any CUDA call)
# ---------------------------------------------------------------------------
_ORC = {}


def _oracle_worker_init(L, N, ecut, vloc, C, eps, gaps):
    """Worker of the oracle pool: the cell's sphere and ground state, once."""
    from oracle import pw
    sph = pw.Sphere(L, N, ecut)
    _ORC["gs"] = pw.GroundState(sph, vloc, len(eps), eps, C)
    _ORC["gaps"] = gaps


def _oracle_state_term(args):
    """One occupied state's term of Eq. P1 by the oracle's Sternheimer route
    (Eq. P2, plain CG to 1e-14): the partial sum over states {v}."""
    y, v = args
    from oracle import response
    return response.chi0_sternheimer(_ORC["gs"], y, 0.0, 1e-14, _ORC["gaps"], states=[v])


class OracleTimer:
    """eps~ applications of the molecule workload by the FP64 oracle on the
    host cores: v^1/2, the sum over all occupied states of Eq. P1 (each state's
    Sternheimer solve in its own process of a spawn pool, one thread each),
    v^1/2.  The ground state (oracle LOBPCG) is prepared once, untimed."""

    def __init__(self, wl):
        import multiprocessing as mp
        from oracle import pw, response
        c = wl.cells[0]
        self.n_occ = c.n_occ
        sph = pw.Sphere(c.L, c.N, c.ecut)
        t0 = time.perf_counter()
        gs, w, _ = pw.ground_state_iterative(sph, c.vloc, c.n_occ, tol=1e-9, maxiter=500)
        self.t_gs = time.perf_counter() - t0
        gaps = w[c.n_occ] - gs.eps
        self.D = response.Dielectric(gs, 0.0, route="sternheimer", gaps=gaps)
        self.x = wl.starts[0][0]
        self.cores = max(1, min(os.cpu_count() or 1, c.n_occ))
        # one BLAS/OpenMP thread per worker: the environment is read when a
        # spawned worker first imports numpy, so it is set around the spawn
        saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS")}
        os.environ.update({k: "1" for k in saved})
        try:
            self.pool = mp.get_context("spawn").Pool(self.cores, initializer=_oracle_worker_init,
                                                     initargs=(c.L, c.N, c.ecut, c.vloc, gs.C, gs.eps, gaps))
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v
        self.pool.map(abs, range(self.cores))          # workers up before any timing

    def apply_once(self):
        """Seconds for one eps~ application (all occupied states)."""
        t0 = time.perf_counter()
        y = self.D.sqrtv(self.x).real
        parts = self.pool.map(_oracle_state_term, [(y, v) for v in range(self.n_occ)])
        self.D.sqrtv(sum(parts))
        return time.perf_counter() - t0

    def sample(self):
        return (f"one eps~ application of the molecule workload (start vector of the bench): v^1/2, Eq. P1 over "
                f"all {self.n_occ} occupied states with the oracle's FP64 Sternheimer route (plain CG to 1e-14, one "
                f"process per state on {self.cores} host cores, one thread each), v^1/2; ground state (oracle "
                f"LOBPCG, {self.t_gs:.1f} s) prepared once, not timed")

    def close(self):
        self.pool.terminate()


def oracle_baseline(wl, reps=2):
    """cpu_baseline of the GPU arm: the same sample as the reference arm."""
    ot = OracleTimer(wl)
    ot.apply_once()                                    # warm-up (imports, first FFT plans)
    ts = [ot.apply_once() for _ in range(reps)]
    ot.close()
    t = float(np.median(ts))
    return dict(value=1.0 / t, unit=UNIT, cores=ot.cores, kind="oracle", sample=ot.sample())


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    wl = W.molecule()
    ot = OracleTimer(wl)
    for _ in range(args.warmup):
        ot.apply_once()
    ts = [ot.apply_once() for _ in range(max(1, args.steps))]
    ot.close()
    v = len(ts) / sum(ts)                  # one step = one eps~ application, timed
    line = dict(metric=METRIC, value=v, unit=UNIT, n_gpus=args.gpus, steps=len(ts), warmup=args.warmup,
                ms_per_step=1e3 * sum(ts) / len(ts), higher_is_better=True, scaling="weak", vs_baseline=None,
                dtype="f64", data="synthetic", impl="reference",
                config=dict(workload=WORKLOAD, step="one eps~ application (the GPU arm's step is a 100-step "
                            "Lanczos run: 100 applications)", l2="n/a (CPU)"),
                cpu_baseline=dict(value=v, unit=UNIT, cores=ot.cores, kind="oracle", sample=ot.sample()),
                e2e=dict(value=v, unit=UNIT, h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------
# replicas: one independent copy of the workload per rank (the path does not
# shard: one Lanczos recursion is sequential), no data-path collective
# ---------------------------------------------------------------------------
def replica_rate(local_ms, steps, k, world, group_max):
    """Whole-job applications/s of `world` replicas: the applications of all
    ranks over the slowest rank's time.  ``group_max(x)`` returns the maximum of
    x over the ranks (identity for one rank).  Returns (rate, max_ms)."""
    total = float(group_max(float(local_ms)))
    return world * steps * k / (total / 1e3), total


def torch_group_max(device=None):
    """group_max over the default torch.distributed process group (any backend)."""
    import torch
    import torch.distributed as dist

    def f(x):
        t = torch.tensor([x], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())
    return f


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.p = None
        return self

    def _read(self):
        for line in self.p.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.p:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except Exception:
                self.p.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
                for n, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(n)
            except Exception:
                continue
        if not sm:
            return dict(sm_mhz=None, sm_max_mhz=None, reasons=["unavailable"], samples=0)
        return dict(sm_mhz=float(np.median(sm)), sm_max_mhz=float(max(mx)), reasons=sorted(reasons),
                    samples=len(sm))


# ---------------------------------------------------------------------------
# algorithmic bytes per column-iteration of each kernel class
# ---------------------------------------------------------------------------
def class_bytes(miller, N, npw, nocc, s):
    """Algorithmic bytes of the inner CG kernels per column-iteration, and per
    launch-iteration for data shared by all columns; s = bytes per complex value.

    persistent_cg (one launch = one CG pass, four phases per iteration):
      A  read r, p, write p (3 N_PW s); write the planes of the sphere (P0 N^2 s)
      B  read + write those planes (2 P0 N^2 s); V shared (N^3 real)
      C  read the planes (P0 N^2 s); read p, write Ap (2 N_PW s); C_v shared (n_occ N_PW s)
      E  read Ap, p, x, r, write x, r (6 N_PW s); C_v shared again
    """
    n = np.mod(miller, N)
    D = len({(a, b) for a, b in zip(n[:, 0], n[:, 1])})        # disc pencils
    P0 = len(set(n[:, 0]))                                     # planes cut by the sphere
    real = s // 2
    col = {
        "persistent_cg": 11 * npw * s + 4 * P0 * N * N * s,
        "z_scatter_inv": 3 * npw * s + D * N * s,
        "y_inv": D * N * s + P0 * N * N * s,
        "x_h": 2 * P0 * N * N * s,
        "y_fwd": P0 * N * N * s + D * N * s,
        "z_gather_h": D * N * s + 2 * npw * s,
        "proj": 4 * npw * s,
        "cg_update": 6 * npw * s,
    }
    shared = {
        "persistent_cg": N ** 3 * real + 2 * nocc * npw * s,
        "z_scatter_inv": 8 * npw, "y_inv": 0, "x_h": N ** 3 * real, "y_fwd": 0,
        "z_gather_h": 8 * npw + npw * real, "proj": 2 * nocc * npw * s, "cg_update": 0,
    }
    return col, shared, dict(D=D, P0=P0)


def cg_bytes_per_col_iter(N, npw, s):
    """Algorithmic bytes of one Sternheimer iteration of one column (the byte
    model of the measurement plan): s (11 N_PW + 4 N_g), s = bytes per complex
    value -- p in / Hp out in the sphere, one grid round trip for each of the
    two transforms, about seven sphere vectors for the CG update, the P_c
    column read and write.  V_loc and the occupied states are amortised over
    the columns and not counted."""
    return s * (11 * npw + 4 * N ** 3)


def model_bytes(N, npw, nocc, s):
    """Algorithmic bytes of one model eps~ application (Eq. model_eq) to one
    field, s = bytes per complex value: the occupied grids u_v read twice (the
    products psi_v* y before the projector, the reduction sum_v u_v f_v after
    it), the occupied coefficients read four times (two projectors, each a
    Gram pass and an update), the field read and eps~ y written (FP64)."""
    return 2 * nocc * N ** 3 * s + 4 * nocc * npw * s + 2 * N ** 3 * 8


def src_hash():
    h = hashlib.sha256()
    for f in ("fft.cuh", "kernels_fft.cu", "kernels_linalg.cu", "gw_common.cuh", "kernels_cg.cu", "pcg.cuh"):
        with open(os.path.join(ROOT, "paper_1408_3036_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel_class):
    """DRAM bytes per column-iteration of the persistent CG kernel from the
    committed ncu summary, if it was taken on the current kernel sources."""
    if kernel_class != "persistent_cg":
        return None
    p = os.path.join(ROOT, "profiles", "k_cg_persistent_molecule.md")
    try:
        with open(p) as f:
            for line in f:
                if line.startswith("traffic-per-column-iteration:"):
                    parts = line.split()
                    if parts[3] == src_hash():
                        return {"dram_bytes_per_col_iter": float(parts[1])}
    except (OSError, IndexError, ValueError):
        pass
    return None


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def run_gpu(args):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    wl = W.molecule()
    K = args.lanczos_k
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = oracle_baseline(wl)          # before any CUDA call in this process

    import torch
    import paper_1408_3036_gb300 as gw
    from paper_1408_3036_gb300 import _build
    from paper_1408_3036_gb300.groundstate import lowest_states
    _build.build()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    c = wl.cells[0]
    attempt = 0
    while True:
        cell = gw.Cell(c.L, c.N, c.ecut, c.vloc, 0, stream.cuda_stream)
        eps, psi, res = lowest_states(cell, c.n_occ + args.deflation, tol=1e-10)
        if res > 1e-8:
            raise RuntimeError(f"ground state did not converge (residual {res:.2e})")
        if eps[c.n_occ] - eps[c.n_occ - 1] > 1e-3 or attempt >= 5:
            break
        attempt += 1
        wl = W.molecule(attempt)
        c = wl.cells[0]
    cell.set_occupied(psi[:c.n_occ], eps[:c.n_occ])
    ndef = args.deflation
    while ndef > 0 and eps[c.n_occ + ndef] - eps[c.n_occ + ndef - 1] <= 1e-3:   # keep shells whole
        ndef -= 1
    if ndef > 0:
        cell.set_deflation(psi[c.n_occ:c.n_occ + ndef], eps[c.n_occ:c.n_occ + ndef])
    ng = cell.ng
    dev = torch.device("cuda", local)
    start = torch.tensor(wl.starts[0][0], dtype=torch.float64, device=dev)
    alpha = torch.empty(K, dtype=torch.float64, device=dev)
    beta = torch.empty(max(K - 1, 1), dtype=torch.float64, device=dev)
    Q = torch.empty((K, ng), dtype=torch.float64, device=dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def step(prec):
        gw.gw_lanczos(cell.ctx, start, K, 0.0, alpha, beta, Q, prec)

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
            torch.cuda.synchronize()

    prec = gw.GW_MIXED if args.prec == "mixed" else gw.GW_FP64
    for _ in range(args.warmup):
        step(prec)
    # --- timed region: K steps, CUDA events on the work stream, L2 flushed between steps
    launches0 = gw.gw_stats(cell.ctx)["launches"]
    times = []
    it_cols = 0.0
    cols = 0.0
    it_launch = 0
    dominant = args.profile_class
    gw.gw_profile(cell.ctx, 1 << gw.PROFILE_CLASSES.index(dominant))
    barrier()
    with Clocks(local) as clk:
        for _ in range(args.steps):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.nvtx.range_push("timed")
            e0.record(stream)
            step(prec)
            e1.record(stream)
            torch.cuda.nvtx.range_pop()
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
            st = gw.gw_stats(cell.ctx)
            it_cols += st["columns"] * st["mean_iter"]
            cols += st["columns"]
            it_launch += st["launch_iterations"]
    barrier()
    prof = gw.gw_profile_read(cell.ctx)
    gw.gw_profile(cell.ctx, 0)
    launches = gw.gw_stats(cell.ctx)["launches"] - launches0
    stats_last = gw.gw_stats(cell.ctx)
    value, total_ms = replica_rate(float(sum(times)), args.steps, K, world,
                                   torch_group_max(dev) if world > 1 else (lambda x: x))
    alpha_mixed = alpha.cpu().numpy().copy()
    beta_mixed = beta[:K - 1].cpu().numpy().copy()

    # --- roofline of the dominant inner-loop kernel (measured live above)
    miller = cell.sphere()
    s = 8 if prec == gw.GW_MIXED else 16
    colb, shared, geo = class_bytes(miller, c.N, cell.npw, c.n_occ, s)
    b_it = cg_bytes_per_col_iter(c.N, cell.npw, s)
    ms_dom, n_dom = prof[dominant]
    hbm, hbm_kind = peaks()
    alg_bytes = it_cols * b_it
    achieved = alg_bytes / (ms_dom / 1e3) / 1e9 if ms_dom > 0 else None
    per_launch_units = it_launch if dominant == "persistent_cg" else n_dom
    pruned_bytes = it_cols * colb[dominant] + per_launch_units * shared[dominant]
    tr = ncu_traffic(dominant)
    traffic = None
    if tr is not None and n_dom > 0:
        traffic = tr["dram_bytes_per_col_iter"] * it_cols / n_dom
    roofline = dict(bound="hbm", kernel=dominant, achieved=achieved, peak=hbm, unit="GB/s",
                    frac=(achieved / hbm if achieved else None), peak_kind=hbm_kind,
                    traffic=traffic, alg_bytes_per_launch=alg_bytes / max(n_dom, 1),
                    alg_bytes_per_col_iter=b_it,
                    byte_model="s (11 N_PW + 4 N_g) per column-iteration, s = bytes per complex value",
                    achieved_pruned_model=(pruned_bytes / (ms_dom / 1e3) / 1e9 if ms_dom > 0 else None),
                    kernel_ms_share=ms_dom / total_ms, launches=n_dom, column_iterations=it_cols,
                    launch_iterations=it_launch)

    # --- FP64 path: the same K-step Lanczos run, timed over the same number of steps
    fp64 = None
    if not args.no_fp64:
        a64 = torch.empty(K, dtype=torch.float64, device=dev)
        b64 = torch.empty(max(K - 1, 1), dtype=torch.float64, device=dev)
        Q64 = torch.empty((K, ng), dtype=torch.float64, device=dev)
        gw.gw_lanczos(cell.ctx, start, K, 0.0, a64, b64, Q64, gw.GW_FP64)   # warm-up
        t64 = []
        for _ in range(args.steps):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            gw.gw_lanczos(cell.ctx, start, K, 0.0, a64, b64, Q64, gw.GW_FP64)
            e1.record(stream)
            e1.synchronize()
            t64.append(e0.elapsed_time(e1))
        a64h, b64h = a64.cpu().numpy(), b64[:K - 1].cpu().numpy()
        st64 = gw.gw_stats(cell.ctx)
        err_a = float(np.abs(alpha_mixed - a64h).max() / np.abs(a64h).max())
        err_b = float(np.abs(beta_mixed - b64h).max() / np.abs(b64h).max()) if K > 1 else 0.0
        v64, _ = replica_rate(float(sum(t64)), args.steps, K, world,
                              torch_group_max(dev) if world > 1 else (lambda x: x))
        fp64 = dict(value=v64, unit=UNIT, lanczos_steps=K, steps=args.steps, ms_per_step=float(sum(t64)) / args.steps,
                    mean_iter=st64["mean_iter"], max_iter=st64["max_iter"], mixed_speedup=value / v64,
                    mixed_vs_fp64_rel_err=dict(alpha=err_a, beta=err_b))

    # --- end to end through the C ABI with host buffers (pinned), copies inside the region
    h_start = torch.tensor(wl.starts[0][0], dtype=torch.float64).pin_memory()
    h_alpha = torch.empty(K, dtype=torch.float64).pin_memory()
    h_beta = torch.empty(max(K - 1, 1), dtype=torch.float64).pin_memory()
    gw.gw_lanczos(cell.ctx, h_start, K, 0.0, h_alpha, h_beta, None, prec)   # warm-up of this path
    barrier()
    te2e = 0.0
    for _ in range(args.steps):              # the same number of steps as the device-timed region
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        gw.gw_lanczos(cell.ctx, h_start, K, 0.0, h_alpha, h_beta, None, prec)
        e1.record(stream)
        e1.synchronize()
        te2e += e0.elapsed_time(e1)
    e2e = dict(value=world * K * args.steps / (te2e / 1e3), unit=UNIT, h2d_bytes_per_step=ng * 8,
               d2h_bytes_per_step=(2 * K - 1) * 8)

    # --- eps~(i w) - 1 in the first Lanczos vectors from recycled per-state bases (Eq. recy_eq)
    rec = None
    if args.recycle_nl > 0:
        nl = min(args.recycle_nl, K)
        Fq = Q[:nl].contiguous()
        w8 = np.array([0.05, 0.1, 0.2, 0.5, 1.0, 2.0, 5.0, 10.0])
        w64 = np.geomspace(0.01, 100.0, 64)
        o8 = torch.empty((len(w8), nl, nl), dtype=torch.float64, device=dev)
        o64 = torch.empty((len(w64), nl, nl), dtype=torch.float64, device=dev)
        tw8 = torch.tensor(w8, device=dev)
        tw64 = torch.tensor(w64, device=dev)
        kept = gw.gw_recycle_eps(cell.ctx, Fq, tw8, o8, 0.0, prec)      # warm-up
        rt = []
        for tw, oo in ((tw8, o8), (tw64, o64)):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            kept = gw.gw_recycle_eps(cell.ctx, Fq, tw, oo, 0.0, prec)
            e1.record(stream)
            e1.synchronize()
            rt.append(e0.elapsed_time(e1))
        # direct: nl eps~ applications at w = 0.5i (SQMR), then <l|.>
        yd = torch.empty((1, nl, ng), dtype=torch.complex128, device=dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        gw.gw_apply_eps(cell.ctx, Fq, [0.5j], torch.view_as_real(yd), prec)
        e1.record(stream)
        e1.synchronize()
        t_dir = e0.elapsed_time(e1)
        wgt = c.L ** 3 / ng
        Ed = (wgt * (Fq @ (yd[0].real - Fq).T)).cpu().numpy()
        Er = o8[3].cpu().numpy()
        # the basis augmented with the solutions at a third frequency (w0 = 1 Ha, the paper's choice)
        cell.set_recycle_augment(1.0)
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        kept_a = gw.gw_recycle_eps(cell.ctx, Fq, tw8, o8, 0.0, prec)
        e1.record(stream)
        e1.synchronize()
        t_aug = e0.elapsed_time(e1)
        cell.set_recycle_augment(0.0)
        Era = o8[3].cpu().numpy()
        rec = dict(fields=nl, precision=args.prec, kept_min=int(kept), ms_8_frequencies=rt[0],
                   ms_64_frequencies=rt[1], ms_per_extra_frequency=(rt[1] - rt[0]) / 56.0,
                   direct_ms_one_frequency=t_dir,
                   rel_err_vs_direct_at_0p5i=float(np.abs(Er - Ed).max() / np.abs(Ed).max()),
                   augmented_w0_1ha=dict(kept_min=int(kept_a), ms_8_frequencies=t_aug,
                                         rel_err_vs_direct_at_0p5i=float(np.abs(Era - Ed).max()
                                                                         / np.abs(Ed).max())))

    # --- Sigma^c of the highest occupied state (Eq. e_c) in the first Lanczos vectors
    sigc = None
    if args.sigma_c_nl > 0:
        nl = min(args.sigma_c_nl, K, 16)
        Fq = Q[:nl].contiguous()
        so = torch.zeros(4, dtype=torch.float64, device=dev)
        gw.gw_sigma_c(cell.ctx, c.n_occ - 1, 0.0, 1.0, 8, Fq, 8, 4, so, prec)    # warm-up
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.nvtx.range_push("sigma_c")
        e0.record(stream)
        gw.gw_sigma_c(cell.ctx, c.n_occ - 1, 0.0, 1.0, 8, Fq, 8, 4, so, prec)
        e1.record(stream)
        e1.synchronize()
        torch.cuda.nvtx.range_pop()
        sv = so.cpu().numpy()
        sigc = dict(state="HOMO", delta=0.0, alpha=1.0, frequencies=8, fields=nl, lanczos_h_steps=8,
                    precision=args.prec, ms=e0.elapsed_time(e1), sigma_c=float(sv[0]), integral=float(sv[1]),
                    sigma_a=float(sv[2]), sigma_p=float(sv[3]))

    # --- model operator (Eq. model_eq) on the same cell and start vector
    model = None
    if args.model_k > 0:
        Km = min(args.model_k, K)
        cell.set_operator(gw.GW_OP_MODEL)

        def mstep(pr, k=Km):
            gw.gw_lanczos(cell.ctx, start, k, 0.0, alpha, beta, Q, pr)

        for _ in range(args.warmup):
            mstep(prec)
        mtimes = []
        for _ in range(args.steps):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.nvtx.range_push("model")
            e0.record(stream)
            mstep(prec)
            e1.record(stream)
            torch.cuda.nvtx.range_pop()
            e1.synchronize()
            mtimes.append(e0.elapsed_time(e1))
        am = alpha[:Km].cpu().numpy().copy()
        bm = beta[:Km - 1].cpu().numpy().copy()
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        mstep(gw.GW_FP64)
        e1.record(stream)
        e1.synchronize()
        tm64 = e0.elapsed_time(e1)
        a64m = alpha[:Km].cpu().numpy()
        b64m = beta[:Km - 1].cpu().numpy()
        # one application to one field, alone (no Lanczos), for the roofline
        xf = Q[:1].clone()
        yf = torch.empty((1, 1, ng), dtype=torch.float64, device=dev)
        gw.gw_apply_eps(cell.ctx, xf, [0.0], yf, prec)
        napp = 20
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(napp):
            gw.gw_apply_eps(cell.ctx, xf, [0.0], yf, prec)
        e1.record(stream)
        e1.synchronize()
        t_app = e0.elapsed_time(e1) / napp
        cell.set_operator(gw.GW_OP_STERNHEIMER)
        mb = model_bytes(c.N, cell.npw, c.n_occ, s)
        ach = mb / (t_app / 1e3) / 1e9
        mval, _ = replica_rate(float(sum(mtimes)), args.steps, Km, world,
                               torch_group_max(dev) if world > 1 else (lambda x: x))
        model = dict(
            value=mval, unit=UNIT, lanczos_steps=Km, ms_per_step=float(sum(mtimes)) / args.steps,
            precision=args.prec, speedup_vs_sternheimer=mval / value, fp64_value=Km / (tm64 / 1e3),
            mixed_vs_fp64_rel_err=dict(alpha=float(np.abs(am - a64m).max() / np.abs(a64m).max()),
                                       beta=float(np.abs(bm - b64m).max() / np.abs(b64m).max()) if Km > 1 else 0.0),
            occupied_energies_above_zero=int((eps[:c.n_occ] > 0).sum()),
            roofline=dict(bound="hbm", kernel="one model eps~ application (all its kernels)", achieved=ach,
                          peak=hbm, unit="GB/s", frac=ach / hbm, peak_kind=hbm_kind, traffic=None,
                          alg_bytes_per_apply=mb, ms_per_apply=t_app))

    # --- residue term Sigma^P_e(delta) of Eq. pe for e = HOMO (k-step Lanczos per pole at real w)
    sigp = None
    if args.sigma_p_k > 0:
        ok = False
        try:
            eps_c, psi_c, res_c = lowest_states(cell, c.n_occ + 4, tol=1e-10)
            ok = float(res_c) <= 1e-8
        except Exception as exc:            # input preparation only; the leg is skipped
            res_c = str(exc)
        if ok:
            cand = np.ascontiguousarray(psi_c[:c.n_occ + 4])
            ce = np.ascontiguousarray(eps_c[:c.n_occ + 4])
            oc = np.array([1] * c.n_occ + [0] * 4, np.int32)
            gap = float(ce[c.n_occ] - ce[c.n_occ - 1])
            e_h = float(ce[c.n_occ - 1])
            rows = []
            for delta in (-0.5 * gap, 1.5 * gap):
                sg = np.zeros(1)
                tt = np.zeros(len(ce))
                gw.gw_sigma_p(cell.ctx, cand[c.n_occ - 1], e_h, delta, cand, ce, oc, args.sigma_p_k, sg, tt, prec)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                gw.gw_sigma_p(cell.ctx, cand[c.n_occ - 1], e_h, delta, cand, ce, oc, args.sigma_p_k, sg, tt, prec)
                e1.record(stream)
                e1.synchronize()
                rows.append(dict(delta=delta, poles=int(np.count_nonzero(tt)), sigma=float(sg[0]),
                                 ms=e0.elapsed_time(e1)))
            sigp = dict(state="HOMO", k=args.sigma_p_k, precision=args.prec, candidates="16 occupied + 4 conduction",
                        runs=rows)
        else:
            sigp = dict(skipped=f"conduction states not converged: {res_c}")

    # --- block complex-frequency workload at full size (64^3, 38401 PW, 64 occupied, blocks of 8)
    bfl = None
    if args.block_freq_steps > 0:
        bw = W.block_freq()
        bc = bw.cells[0]
        bcell = gw.Cell(bc.L, bc.N, bc.ecut, bc.vloc, 0, stream.cuda_stream)
        beps, bpsi, bres = lowest_states(bcell, bc.n_occ, tol=1e-10)
        if bres <= 1e-8 and beps[bc.n_occ] - beps[bc.n_occ - 1] > 1e-3:
            bcell.set_occupied(bpsi, beps[:bc.n_occ])
            om = complex(bw.omegas[0])
            X0 = bw.starts[0]
            kb = args.block_freq_steps
            rows = []
            for tc_on in (0, 1):
                bcell.set_tensor_cores(tc_on)
                flush.fill_(1.0)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                A, B, _ = bcell.block_lanczos(X0, kb, om, prec)
                e1.record(stream)
                e1.synchronize()
                stb = gw.gw_stats(bcell.ctx)
                rows.append(dict(tensor_core_projector=bool(tc_on), ms=e0.elapsed_time(e1),
                                 applies_per_s=kb * X0.shape[0] / (e0.elapsed_time(e1) / 1e3),
                                 sqmr_mean_iter=stb["mean_iter"], sqmr_max_iter=stb["max_iter"],
                                 sqmr_columns=stb["columns"], graph_replays=stb["graph_replays"]))
            bcell.set_tensor_cores(0)
            bfl = dict(workload="L=24 bohr, 64^3, 15 Ha (%d PW), 24 wells, N_occ=64, block 8, omega=%.4f+0.1i"
                       % (bcell.npw, om.real), block_steps=kb, precision=args.prec, runs=rows,
                       unit="eps~ applications (block columns) per second")
        else:
            bfl = dict(skipped=f"ground state not converged or gap too small (residual {bres:.2e})")
        bcell.close()

    # --- many uneven cells at once (32 cells, K = 40, four real frequencies each)
    bat = None
    if args.batch_cells > 0:
        from paper_1408_3036_gb300.groundstate import levels_below
        bw = W.batch(n_cells=args.batch_cells)
        bt = gw.Batch([(x.L, x.N, x.ecut, x.vloc) for x in bw.cells], workers=8)
        bom = np.tile(np.array(bw.omegas, complex), (len(bw.cells), 1))
        t_prep = time.perf_counter()
        nredraw = 0
        for i, x in enumerate(bw.cells):
            # input preparation on a context of its own on the bench stream (a
            # batch cell's context works on the batch's stream)
            prep = gw.Cell(x.L, x.N, x.ecut, x.vloc, 0, stream.cuda_stream)
            e_occ, p_occ, _ = lowest_states(prep, x.n_occ, tol=1e-10)
            bt.cell(i).set_occupied(p_occ, e_occ[:x.n_occ])
            lev = levels_below(prep, e_occ[x.n_occ - 1] + 1.01, x.n_occ + 32, tol=1e-4)
            prep.close()
            tr = np.subtract.outer(lev[x.n_occ:], lev[:x.n_occ]).ravel()
            for w in range(bom.shape[1]):
                att = 0
                while tr.size and np.abs(tr - bom[i, w].real).min() <= 1e-3:   # re-drawn per cell
                    att += 1
                    nredraw += 1
                    bom[i, w] = W.redraw_omega(W.BASE_SEED + 3 + 1000 * att + 100 * i + w, 0.0, 1.0)
        t_prep = time.perf_counter() - t_prep
        bst = [x[0] for x in bw.starts]
        rows = []
        for graphs in (1, 0):
            for i in range(len(bw.cells)):
                bt.cell(i).set_graphs(graphs)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            bt.lanczos(bst, args.batch_k, bom, prec)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            replays = sum(gw.gw_stats(bt.cell(i).ctx)["graph_replays"] for i in range(len(bw.cells)))
            rows.append(dict(cuda_graphs=bool(graphs), s=dt,
                             applies_per_s=len(bw.cells) * bom.shape[1] * args.batch_k / dt,
                             status_ok=int((bt.last_status == 0).sum()),
                             graph_replays_last_solve=int(replays)))
        bat = dict(workload="%d uneven cells (L 8-16 bohr, N 24-48, 5-10 Ha, N_occ 4-32), K=%d Lanczos steps "
                   "(the configuration's 40 with --batch-k 40), 4 real omega in [0,1] per cell"
                   % (len(bw.cells), args.batch_k),
                   precision=args.prec, frequencies_redrawn=nredraw, prep_s=t_prep, runs=rows,
                   timing="host wall clock around the whole batch call (all cells, all frequencies)",
                   unit="eps~ applications per second (all cells)")
        bt.close()

    if rank == 0:
        line = dict(
            metric=METRIC, value=value, unit=UNIT, n_gpus=world, steps=args.steps, warmup=args.warmup,
            ms_per_step=total_ms / args.steps, higher_is_better=True, scaling="weak", vs_baseline=None,
            dtype="f32+f64-refine" if prec == gw.GW_MIXED else "f64", data="synthetic",
            config=dict(workload=WORKLOAD, parallelism=("replicas" if world > 1 else "single"),
                        precision=args.prec, lanczos_steps=K,
                        l2="working set (~14 MB) L2-resident inside a step; L2 flushed (512 MB write) "
                           "between timed steps",
                        ground_state_residual=res, gap_homo_lumo=float(eps[c.n_occ] - eps[c.n_occ - 1]),
                        deflation_states=ndef,
                        sternheimer_mean_iter=stats_last["mean_iter"], sternheimer_max_iter=stats_last["max_iter"],
                        column_iterations_per_step=it_cols / args.steps, geometry=geo),
            roofline=roofline, cpu_baseline=cpu, e2e=e2e, gpu_launches=int(launches),
            clocks=clk.summary(), fp64=fp64, profile_ms={k: v[0] for k, v in prof.items() if v[1]},
            model_operator=model, sigma_p=sigp, recycle=rec, sigma_c=sigc, block_freq=bfl,
            batch=bat,
        )
        print(json.dumps(line))
    cell.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--prec", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--lanczos-k", type=int, default=100)
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile-class", default="persistent_cg")
    ap.add_argument("--model-k", type=int, default=100,
                    help="Lanczos steps timed on the model operator of Eq. model_eq (0: skip)")
    ap.add_argument("--sigma-c-nl", type=int, default=8,
                    help="Lanczos vectors of the Sigma^c leg (Eq. e_c, HOMO, 8 frequencies; 0: skip)")
    ap.add_argument("--recycle-nl", type=int, default=20,
                    help="Lanczos vectors in which eps~(i w) - 1 is built from recycled bases (Eq. recy_eq; 0: skip)")
    ap.add_argument("--sigma-p-k", type=int, default=4,
                    help="Lanczos steps per pole of the Sigma^P leg (Eq. pe; 0: skip)")
    ap.add_argument("--block-freq-steps", type=int, default=1,
                    help="block Lanczos steps timed on the full block complex-frequency workload (0: skip)")
    ap.add_argument("--batch-cells", type=int, default=32,
                    help="cells of the many-cell leg (0: skip)")
    ap.add_argument("--batch-k", type=int, default=10,
                    help="Lanczos steps per cell and frequency in the many-cell leg")
    ap.add_argument("--deflation", type=int, default=0,
                    help="lowest conduction states handed to the solvers as a deflation block (0: none)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
