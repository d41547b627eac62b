"""Seeded synthetic inputs for the Lanczos/Sternheimer dielectric-matrix path.

This module draws random numbers and samples the synthetic local potential; it
holds none of the method's arithmetic (no Hamiltonian, no FFT, no response).
Both the oracle-based tests and the GPU bench take their inputs from here.

The paper's workloads are pseudopotential molecules in a vacuum box
(Sec. Results, Table conv_par).  Those DFT states and pseudopotentials are not
available, so localised attractive Gaussian wells in a periodic cubic box stand
in for them: a handful to 64 bound occupied states, the same shape of problem.

Well shape (reading of "depth D, width sigma"):
    V(r) = D * sum_a sum_{m in {-1,0,1}^3} exp(-|r - R_a - L m|^2 / (2 sigma^2))
sampled at r = L * (i0, i1, i2) / N, C order [i0][i1][i2].

Seeds: numpy PCG64, seed = 14083036 + config index + 1000 * attempt.
Draw order: centres, then (for the batch config) per-cell sizes, then start
vectors, then frequencies.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

BASE_SEED = 14083036


@dataclasses.dataclass
class Cell:
    L: float                 # cubic box edge (bohr)
    N: int                   # FFT grid points per edge
    ecut: float              # plane-wave cutoff (Ha): |G|^2/2 <= ecut
    n_occ: int               # occupied (doubly occupied) states
    centres: np.ndarray      # (n_wells, 3) bohr
    depth: float             # Ha (negative = attractive)
    sigma: float             # bohr
    coulomb: int = 0         # 0 = spherical truncation R_c = L/2, 1 = bare

    @property
    def vloc(self) -> np.ndarray:
        return gaussian_wells(self.L, self.N, self.centres, self.depth, self.sigma)

    @property
    def ng(self) -> int:
        return self.N ** 3

    @property
    def sphere_radius(self) -> float:
        """R = sqrt(2 ecut) L / (2 pi): largest |n| in the sphere."""
        return math.sqrt(2.0 * self.ecut) * self.L / (2.0 * math.pi)


@dataclasses.dataclass
class Workload:
    name: str
    cells: list
    omegas: np.ndarray       # complex frequencies (Ha)
    starts: list             # per cell: (blk, N^3) real start block
    k: int                   # Lanczos steps (blocks)
    blk: int = 1
    phi: np.ndarray | None = None   # differentiation config: Gaussian phi


def gaussian_wells(L, N, centres, depth, sigma):
    x = np.arange(N) * (L / N)
    X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
    v = np.zeros((N, N, N))
    for c in np.atleast_2d(centres):
        for m0 in (-1, 0, 1):
            for m1 in (-1, 0, 1):
                for m2 in (-1, 0, 1):
                    d2 = ((X - c[0] - L * m0) ** 2 + (Y - c[1] - L * m1) ** 2
                          + (Z - c[2] - L * m2) ** 2)
                    v += np.exp(-d2 / (2.0 * sigma * sigma))
    return (depth * v).reshape(-1)


def gaussian_phi(L, N, centre, sigma=1.5):
    """Seeded Gaussian test field phi (same periodic images as the wells)."""
    return gaussian_wells(L, N, np.atleast_2d(centre), 1.0, sigma)


def _rng(idx, attempt):
    return np.random.Generator(np.random.PCG64(BASE_SEED + idx + 1000 * attempt))


def _starts(rng, n, blk):
    return rng.standard_normal((blk, n))


def tiny(attempt=0, N=16, L=10.0, ecut=5.0, n_wells=4, n_occ=4, k=20):
    """Tiny plain-method case: L=10, 16^3 grid, 5 Ha, 4 wells, N_occ=4, K=20."""
    rng = _rng(0, attempt)
    centres = rng.uniform(0.0, L, size=(n_wells, 3))
    cell = Cell(L, N, ecut, n_occ, centres, -2.0, 1.0)
    return Workload("tiny", [cell], np.array([0.0 + 0.0j]),
                    [_starts(rng, cell.ng, 1)], k)


def molecule(attempt=0):
    """Molecule-sized static screening: L=20, 48^3, 10 Ha, 8 wells (D=-3,
    sigma=0.8), N_occ=16, omega=0, K=100 with full re-orthogonalisation."""
    rng = _rng(1, attempt)
    L = 20.0
    centres = rng.uniform(0.0, L, size=(8, 3))
    cell = Cell(L, 48, 10.0, 16, centres, -3.0, 0.8)
    return Workload("molecule", [cell], np.array([0.0 + 0.0j]),
                    [_starts(rng, cell.ng, 1)], 100)


def block_freq(attempt=0):
    """Frequency-dependent block Lanczos: L=24, 64^3, 15 Ha, 24 wells,
    N_occ=64, block 8, 60 block steps, 16 omega = U(0,2) + 0.1i."""
    rng = _rng(2, attempt)
    L = 24.0
    centres = rng.uniform(0.0, L, size=(24, 3))
    cell = Cell(L, 64, 15.0, 64, centres, -3.0, 0.8)
    starts = [_starts(rng, cell.ng, 8)]
    omegas = rng.uniform(0.0, 2.0, size=16) + 0.1j
    return Workload("block_freq", [cell], omegas, starts, 60, blk=8)


def block_freq_slice(attempt=0):
    """Reduced slice of the block complex-frequency workload for oracle
    parity: its structure (24 wells, D=-3, sigma=0.8; N_occ=64; blocks of 8;
    omega = U(0,2) + 0.1i) on a cell the oracle diagonalises densely --
    L=16, 32^3, 5 Ha (2109 plane waves); 2 frequencies, 2 block steps."""
    rng = _rng(7, attempt)
    L = 16.0
    centres = rng.uniform(0.0, L, size=(24, 3))
    cell = Cell(L, 32, 5.0, 64, centres, -3.0, 0.8)
    starts = [_starts(rng, cell.ng, 8)]
    omegas = rng.uniform(0.0, 2.0, size=2) + 0.1j
    return Workload("block_freq_slice", [cell], omegas, starts, 2, blk=8)


ALLOWED_N = (24, 30, 32, 36, 40, 45, 48)


def batch(attempt=0, n_cells=32):
    """32 uneven cells: L~U[8,16], N in {24..48} (>= 2R+1), ecut~U[5,10],
    N_occ~U{4..32} (capped below N_PW/4), wells U{4..12}, K=40, 4 real omega
    in [0,1].  Frequencies near a transition are re-drawn by the caller, who
    knows the spectrum (the generator holds no method arithmetic)."""
    rng = _rng(3, attempt)
    cells = []
    for _ in range(n_cells):
        L = rng.uniform(8.0, 16.0)
        ecut = rng.uniform(5.0, 10.0)
        R = math.sqrt(2.0 * ecut) * L / (2.0 * math.pi)
        okN = [n for n in ALLOWED_N if n >= 2 * math.floor(R) + 1]
        if not okN:
            # shrink the cutoff until the largest grid holds the sphere
            ecut = 0.5 * (2.0 * math.pi * (ALLOWED_N[-1] - 1) / 2 / L) ** 2
            okN = [ALLOWED_N[-1]]
        N = int(rng.choice(okN))
        n_wells = int(rng.integers(4, 13))
        centres = rng.uniform(0.0, L, size=(n_wells, 3))
        npw_est = 4.0 / 3.0 * math.pi * R ** 3
        n_occ = int(min(rng.integers(4, 33), max(4, int(npw_est / 4) - 1)))
        cells.append(Cell(L, N, ecut, n_occ, centres, -2.0, 1.0))
    starts = [_starts(rng, c.ng, 1) for c in cells]
    omegas = rng.uniform(0.0, 1.0, size=4) + 0.0j
    return Workload("batch", cells, omegas, starts, 40)


SMALL_N = (12, 15, 16, 18, 20)


def batch_small(attempt=0, n_cells=5):
    """The uneven-batch recipe scaled down to sizes the oracle finishes in
    seconds: L~U[6,9], N in {12..20} (>= 2R+1), ecut~U[2,4], N_occ~U{2..6},
    wells U{2..5} (D=-2, sigma=1), K=8; frequencies 0, two real in [0,1] and
    one complex."""
    rng = _rng(13, attempt)
    cells = []
    for _ in range(n_cells):
        L = rng.uniform(6.0, 9.0)
        ecut = rng.uniform(2.0, 4.0)
        R = math.sqrt(2.0 * ecut) * L / (2.0 * math.pi)
        okN = [n for n in SMALL_N if n >= 2 * math.floor(R) + 1]
        if not okN:
            ecut = 0.5 * (2.0 * math.pi * (SMALL_N[-1] - 1) / 2 / L) ** 2
            okN = [SMALL_N[-1]]
        N = int(rng.choice(okN))
        n_wells = int(rng.integers(2, 6))
        centres = rng.uniform(0.0, L, size=(n_wells, 3))
        n_occ = int(rng.integers(2, 7))
        cells.append(Cell(L, N, ecut, n_occ, centres, -2.0, 1.0))
    starts = [_starts(rng, c.ng, 1) for c in cells]
    omegas = np.concatenate([[0.0], rng.uniform(0.0, 1.0, size=2), [0.3 + 0.1j]]).astype(complex)
    return Workload("batch_small", cells, omegas, starts, 8)


def redraw_omega(attempt_rng_seed, lo, hi):
    """Fresh frequency draw for the batch config when one lands within 1e-3 Ha
    of a transition (the caller decides; this only draws)."""
    rng = np.random.Generator(np.random.PCG64(attempt_rng_seed))
    return rng.uniform(lo, hi)


def differentiation(attempt=0):
    """s = <phi|eps^-1(0)|phi>, phi Gaussian sigma=1.5: L=14, 32^3, 8 Ha,
    N_occ=8, 6 wells (D=-2, sigma=1), K=40."""
    rng = _rng(4, attempt)
    L = 14.0
    centres = rng.uniform(0.0, L, size=(6, 3))
    cell = Cell(L, 32, 8.0, 8, centres, -2.0, 1.0)
    centre = rng.uniform(0.0, L, size=3)
    phi = gaussian_phi(L, 32, centre, 1.5)
    return Workload("differentiation", [cell], np.array([0.0 + 0.0j]),
                    [phi[None, :]], 40, phi=phi)


def small(attempt=0, N=12, L=8.0, ecut=3.0, n_wells=2, n_occ=2, k=8, seed_idx=10):
    """Very small case for brute-force pins and finite differences."""
    rng = _rng(seed_idx, attempt)
    centres = rng.uniform(0.0, L, size=(n_wells, 3))
    cell = Cell(L, N, ecut, n_occ, centres, -2.0, 1.0)
    return Workload("small", [cell], np.array([0.0 + 0.0j]),
                    [_starts(rng, cell.ng, 1)], k)


def random_fields(seed, n, ng, complex_=False):
    rng = np.random.Generator(np.random.PCG64(seed))
    x = rng.standard_normal((n, ng))
    if complex_:
        x = x + 1j * rng.standard_normal((n, ng))
    return x


CONFIGS = {
    "tiny": tiny,
    "molecule": molecule,
    "block_freq": block_freq,
    "batch": batch,
    "differentiation": differentiation,
}
