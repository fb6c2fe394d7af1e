"""Seeded synthetic inputs for the FEAST eigensolver.

This module builds the *inputs* of the generalized problem A x = lambda B x
(Polizzi, arXiv:0901.2665, Sec. III.A, Eq. 2): Q1 trilinear finite-element
operators on layered interior grids, smooth Gaussian potentials, random start
blocks Y and the table of synthetic workloads.  It performs no step of the
eigensolver (no contour quadrature, no linear solve, no Rayleigh-Ritz); both the
CPU oracle and the CUDA path receive their inputs from here and from nowhere
else.

Operator layout (shared by every consumer): grid node id = ix + nx*(iy + ny*iz)
with 0 <= ix < nx, 0 <= iy < ny, 0 <= iz < nz; a z-layer holds n = nx*ny
consecutive unknowns.  A and B are stored as ``[27][N]`` float64 arrays of
row-wise stencil coefficients; stencil slot s = (dz+1)*9 + (dy+1)*3 + (dx+1)
couples node i to node i + dx + nx*(dy + ny*dz); slots whose neighbour lies
outside the grid (homogeneous Dirichlet boundary) hold 0.
"""

from __future__ import annotations

import dataclasses
import math

import numpy as np

# ----------------------------------------------------------------------------
# Stencil geometry
# ----------------------------------------------------------------------------

STENCIL_OFFSETS = [(dx, dy, dz) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
"""Slot s -> (dx, dy, dz); slot 13 is the centre."""


def slot(dx: int, dy: int, dz: int) -> int:
    return (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1)


def grid_index(nx: int, ny: int, nz: int):
    """(ix, iy, iz) integer arrays of every node, in node-id order."""
    N = nx * ny * nz
    idx = np.arange(N, dtype=np.int64)
    return idx % nx, (idx // nx) % ny, idx // (nx * ny)


# ----------------------------------------------------------------------------
# Counter-based random numbers: SplitMix64 (Steele, Lea & Flood, OOPSLA 2014)
# ----------------------------------------------------------------------------

SPLITMIX_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_MIX1 = np.uint64(0xBF58476D1CE4E5B9)
_MIX2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, counter: np.ndarray) -> np.ndarray:
    """k-th SplitMix64 output of a generator seeded with ``seed`` (k = counter).

    The generator advances its state by the golden-ratio increment and returns
    the mixed state, so output k is mix(seed + (k + 1) * GAMMA) (mod 2**64)."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (counter.astype(np.uint64) + np.uint64(1)) * SPLITMIX_GAMMA
        z = (z ^ (z >> np.uint64(30))) * _MIX1
        z = (z ^ (z >> np.uint64(27))) * _MIX2
        return z ^ (z >> np.uint64(31))


def uniform_pm1(seed: int, counter: np.ndarray) -> np.ndarray:
    """Uniform doubles in [-1, 1) from the top 53 bits of SplitMix64."""
    u = (splitmix64(seed, counter) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    return 2.0 * u - 1.0


def random_Y(N: int, M0: int, seed: int) -> np.ndarray:
    """Random start block Y (N x M0, Fig. 2 step 1), column-major order.

    Entry (row, col) is uniform_pm1(seed, col*N + row); returned as a Fortran
    ordered array so ``Y.ravel(order='F')`` is the device layout."""
    k = np.arange(N * M0, dtype=np.uint64)
    return uniform_pm1(seed, k).reshape((M0, N)).T.copy(order="F").astype(np.float64)


# ----------------------------------------------------------------------------
# Smooth potential: a sum of Gaussians
# ----------------------------------------------------------------------------

@dataclasses.dataclass
class Potential:
    centres: np.ndarray   # (G, 3)
    sigmas: np.ndarray    # (G,)
    amps: np.ndarray      # (G,)

    def __call__(self, x, y, z):
        V = np.zeros_like(x, dtype=np.float64)
        for c, s, a in zip(self.centres, self.sigmas, self.amps):
            r2 = (x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2
            V += a * np.exp(-r2 / (2.0 * s * s))
        return V

    def scalars(self) -> np.ndarray:
        """Per-Gaussian (c_z, width, amplitude): 3 scalars each."""
        return np.stack([self.centres[:, 2], self.sigmas, self.amps], axis=1).ravel()


def box_lengths(nx: int, ny: int, nz: int):
    h = 1.0 / (nx + 1)
    return h, 1.0, (ny + 1) * h, (nz + 1) * h


def gaussian_potential(G: int, seed: int, nx: int, ny: int, nz: int,
                       fixed_xy_seed: int | None = None) -> Potential:
    """G Gaussians: centres uniform in the box, widths 0.1-0.3 of the box's x
    length, amplitudes U[-2, 0].  With ``fixed_xy_seed`` the (x, y) centres are
    drawn from that seed instead (shared by a family of instances) and only
    (c_z, width, amplitude) vary with ``seed``."""
    _, Lx, Ly, Lz = box_lengths(nx, ny, nz)
    rng = np.random.default_rng(np.random.PCG64(seed))
    cz = rng.uniform(0.0, Lz, G)
    cx = rng.uniform(0.0, Lx, G)
    cy = rng.uniform(0.0, Ly, G)
    w = rng.uniform(0.1, 0.3, G)
    a = rng.uniform(-2.0, 0.0, G)
    if fixed_xy_seed is not None:
        rxy = np.random.default_rng(np.random.PCG64(fixed_xy_seed))
        cx = rxy.uniform(0.0, Lx, G)
        cy = rxy.uniform(0.0, Ly, G)
    return Potential(np.stack([cx, cy, cz], axis=1), w * Lx, a)


# ----------------------------------------------------------------------------
# Q1 trilinear finite-element operator on the layered grid
# ----------------------------------------------------------------------------

@dataclasses.dataclass
class Operator:
    nx: int
    ny: int
    nz: int
    A27: np.ndarray   # (27, N) float64, C-contiguous
    B27: np.ndarray   # (27, N)

    @property
    def N(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def n(self) -> int:
        return self.nx * self.ny


def q1_operator(nx: int, ny: int, nz: int, potential: Potential | None = None) -> Operator:
    """A = 1/2 K + M_V and B = M for Q1 elements with uniform spacing
    h = 1/(nx+1) on every axis and a homogeneous Dirichlet boundary.

    The 1-D linear-element matrices are K1 = (1/h) tridiag(-1, 2, -1) and
    M1 = (h/6) tridiag(1, 4, 1); the trilinear ones are their tensor products
    K = K1(x)M1(x)M1 + M1(x)K1(x)M1 + M1(x)M1(x)K1 and M = M1(x)M1(x)M1.
    The potential enters mass-weighted: (M_V)_ij = M_ij (V(r_i) + V(r_j)) / 2,
    which keeps the 27-point pattern and the symmetry."""
    h = 1.0 / (nx + 1)
    k1 = {-1: -1.0 / h, 0: 2.0 / h, 1: -1.0 / h}
    m1 = {-1: h / 6.0, 0: 4.0 * h / 6.0, 1: h / 6.0}
    N = nx * ny * nz
    ix, iy, iz = grid_index(nx, ny, nz)
    if potential is not None:
        V = potential((ix + 1) * h, (iy + 1) * h, (iz + 1) * h)
    else:
        V = np.zeros(N)
    A27 = np.zeros((27, N))
    B27 = np.zeros((27, N))
    idx = np.arange(N, dtype=np.int64)
    for s, (dx, dy, dz) in enumerate(STENCIL_OFFSETS):
        valid = ((ix + dx >= 0) & (ix + dx < nx) & (iy + dy >= 0) & (iy + dy < ny)
                 & (iz + dz >= 0) & (iz + dz < nz))
        m = m1[dx] * m1[dy] * m1[dz]
        kk = k1[dx] * m1[dy] * m1[dz] + m1[dx] * k1[dy] * m1[dz] + m1[dx] * m1[dy] * k1[dz]
        j = np.where(valid, idx + dx + nx * (dy + ny * dz), 0)
        vavg = 0.5 * (V + V[j])
        A27[s] = np.where(valid, 0.5 * kk + m * vavg, 0.0)
        B27[s] = np.where(valid, m, 0.0)
    return Operator(nx, ny, nz, np.ascontiguousarray(A27), np.ascontiguousarray(B27))


def peierls_operator(op: Operator, flux: float = 0.0, gauge_seed: int | None = None,
                     gauge_B: bool = False) -> Operator:
    """A Hermitian operator from a real one: every coupling A_ij (i != j) gets
    the phase exp(i phi_ij) with phi_ji = -phi_ij, so that A_ji = conj(A_ij).
    phi_ij = flux * (x_i + x_j)/2 * (y_j - y_i) in grid units (a uniform field
    along z in the Landau gauge) plus chi_j - chi_i for a seeded uniform chi in
    [0, 2 pi) when gauge_seed is given.  With gauge_B the couplings of B get
    the gauge part exp(i (chi_j - chi_i)) too: the pencil is then D^H (A, B) D
    for D = diag(exp(i chi)) (at flux 0), with the eigenvalues of (A, B).
    A27 (and then B27) is complex128."""
    nx, ny, nz = op.nx, op.ny, op.nz
    ix, iy, iz = grid_index(nx, ny, nz)
    N = op.N
    chi = np.zeros(N)
    if gauge_seed is not None:
        chi = 2.0 * np.pi * np.random.default_rng(gauge_seed).random(N)
    idx = np.arange(N, dtype=np.int64)
    A27 = np.zeros((27, N), dtype=np.complex128)
    B27 = np.zeros((27, N), dtype=np.complex128)
    for s, (dx, dy, dz) in enumerate(STENCIL_OFFSETS):
        valid = ((ix + dx >= 0) & (ix + dx < nx) & (iy + dy >= 0) & (iy + dy < ny)
                 & (iz + dz >= 0) & (iz + dz < nz))
        j = np.where(valid, idx + dx + nx * (dy + ny * dz), idx)
        phi = flux * (ix + 0.5 * dx) * dy + chi[j] - chi
        A27[s] = np.where(valid, op.A27[s] * np.exp(1j * phi), 0.0)
        if gauge_B:
            B27[s] = np.where(valid, op.B27[s] * np.exp(1j * (chi[j] - chi)), 0.0)
    return Operator(nx, ny, nz, np.ascontiguousarray(A27), B27 if gauge_B else op.B27.copy())


def random_Y_complex(N: int, M0: int, seed: int) -> np.ndarray:
    """Complex start block: real part random_Y(seed), imaginary part
    random_Y(seed + 1) (the same counter-based generator)."""
    return random_Y(N, M0, seed) + 1j * random_Y(N, M0, seed + 1)


def decouple_layers(op: Operator, cut_layers) -> Operator:
    """Zero the couplings across the z-interfaces just below each layer in
    ``cut_layers``: the matrices become block diagonal with one block per slab
    (the k(N, M) replica construction of Sec. IV.B uses equal slabs)."""
    A27 = op.A27.copy()
    B27 = op.B27.copy()
    n = op.n
    for L in cut_layers:
        lo = slice((L - 1) * n, L * n)   # rows of layer L-1: drop dz=+1
        hi = slice(L * n, (L + 1) * n)   # rows of layer L: drop dz=-1
        for s, (dx, dy, dz) in enumerate(STENCIL_OFFSETS):
            if dz == 1:
                A27[s, lo] = 0.0
                B27[s, lo] = 0.0
            if dz == -1:
                A27[s, hi] = 0.0
                B27[s, hi] = 0.0
    return Operator(op.nx, op.ny, op.nz, A27, B27)


def replicate_z(op_block: Operator, k: int) -> Operator:
    """k uncoupled copies of a block operator stacked along z (block diagonal)."""
    A27 = np.concatenate([op_block.A27] * k, axis=1)
    B27 = np.concatenate([op_block.B27] * k, axis=1)
    rep = Operator(op_block.nx, op_block.ny, op_block.nz * k,
                   np.ascontiguousarray(A27), np.ascontiguousarray(B27))
    # the copies were built with Dirichlet walls at their own z ends, so the
    # dz=+-1 slots at the seams are already zero
    return rep


# ----------------------------------------------------------------------------
# Workload table: the five synthetic configurations
# ----------------------------------------------------------------------------

@dataclasses.dataclass
class Workload:
    name: str
    nx: int
    ny: int
    nz: int
    gaussians: int
    M: int
    M0: int
    Ne: int = 8
    tol: float = 1e-12
    precision: str = "fp64"

    @property
    def N(self) -> int:
        return self.nx * self.ny * self.nz

    def operator(self, seed: int, zero_potential: bool = False) -> Operator:
        pot = None if zero_potential else gaussian_potential(self.gaussians, seed, self.nx, self.ny, self.nz)
        return q1_operator(self.nx, self.ny, self.nz, pot)


WORKLOADS = {
    # 10x10x20 grid, n=100, 20 layers; lowest 10 eigenpairs, M0=16
    "q1_10x10x20_fp64": Workload("q1_10x10x20_fp64", 10, 10, 20, 8, 10, 16),
    # 32x32x400 grid, n=1024, 400 layers; lowest 100 eigenpairs, M0=128
    "q1_32x32x400_fp64": Workload("q1_32x32x400_fp64", 32, 32, 400, 32, 100, 128),
    # same operator, complex64 tensor-core factors + FP64 iterative refinement
    "q1_32x32x400_mixed": Workload("q1_32x32x400_mixed", 32, 32, 400, 32, 100, 128, precision="mixed"),
    # 24x24x100 grid, n=576; lowest 40 eigenpairs, M0=64 (learned-start family)
    "q1_24x24x100_fp64": Workload("q1_24x24x100_fp64", 24, 24, 100, 16, 40, 64),
}


# ----------------------------------------------------------------------------
# Batched workload: 64 independent instances of uneven size
# ----------------------------------------------------------------------------

@dataclasses.dataclass
class BatchInstance:
    index: int
    nx: int
    ny: int
    nz: int
    M0: int
    potential_seed: int
    gaussians: int = 8

    def operator(self) -> Operator:
        pot = gaussian_potential(self.gaussians, self.potential_seed, self.nx, self.ny, self.nz)
        return q1_operator(self.nx, self.ny, self.nz, pot)


def batch_instances(count: int = 64, master_seed: int = 3, nz_range=(50, 400), sides=(16, 24, 32),
                    m0_choices=(32, 64, 128)):
    """Instance i draws its cross-section side from `sides` (block sizes
    256/576/1024), its layer count uniformly in `nz_range` and M0 from
    `m0_choices`, from the stream PCG64([master_seed, i]); its potential uses
    8 Gaussians with seed 1000*master_seed + i."""
    out = []
    for i in range(count):
        rng = np.random.default_rng(np.random.PCG64([master_seed, i]))
        side = int(rng.choice(sides))
        nz = int(rng.integers(nz_range[0], nz_range[1] + 1))
        M0 = int(rng.choice(m0_choices))
        out.append(BatchInstance(i, side, side, nz, M0, 1000 * master_seed + i))
    return out
