"""Seeded synthetic inputs for the Dyson-equation diagonal solve.

This module only draws numbers: lattice shapes, the trap potential V_i, the
self-energy samples Sigma_i(i w_k), the Matsubara grid and the Lanczos start
vector.  It holds none of the method's arithmetic (no H assembly, no solve),
so both the CUDA path and the CPU oracle can take their inputs from it.

Workloads stand in for the paper's Falicov-Kimball IDMFT data (Sec. 3: a
101x101 square lattice, 63 Matsubara frequencies), whose self-energies are not
available: Sigma_i(i w_k) = a_i - i b_i sign(w_k) with a_i ~ U[-1, 1] and
b_i ~ U[0, b_max] drawn per site, V_i = c r_i^2 measured from the lattice
centre, w_k = (2k + 1) pi / beta (Sec. 1, Eq. 1 and the text after it).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass(frozen=True)
class Workload:
    """One lattice problem: geometry, physics parameters and method sizes."""

    name: str
    L: tuple            # (Lx, Ly) or (Lx, Ly, Lz); x is the fastest site index
    t: float            # nearest-neighbour hopping
    mu: float           # chemical potential
    trap: float         # V_i = trap * r_i^2
    b_max: float        # b_i ~ U[0, b_max]
    beta: float         # inverse temperature of the Matsubara grid
    K: int              # number of Matsubara frequencies
    p: int              # subdomains along the slowest axis
    k: int              # Lanczos rank cap
    seed: int
    periodic: tuple = field(default=(False, False, False))

    @property
    def N(self) -> int:
        return int(np.prod(self.L))

    @property
    def dim(self) -> int:
        return len(self.L)


# Lattice workloads shaped like the paper's 2D run and its 3D outlook (Sec. 3, Sec. 4).
WORKLOADS = {
    "square16_K8_p2_k16": Workload("square16_K8_p2_k16", (16, 16), -1.0, 0.0, 0.01, 0.5,
                                   10.0, 8, 2, 16, 1),
    "square128_K64_p4_k32": Workload("square128_K64_p4_k32", (128, 128), -1.0, 0.0, 0.01, 0.5,
                                     20.0, 64, 4, 32, 2),
    "cubic32_K128_p8_k48": Workload("cubic32_K128_p8_k48", (32, 32, 32), -1.0, 0.0, 0.005, 1.0,
                                    40.0, 128, 8, 48, 3),
    "square512_K32_p16_k64": Workload("square512_K32_p16_k64", (512, 512), -1.0, 0.0, 0.01, 0.5,
                                      10.0, 32, 16, 64, 4),
}


def matsubara(beta: float, K: int) -> np.ndarray:
    """Fermionic Matsubara frequencies w_k = (2k+1) pi / beta, k = 0..K-1."""
    return (2.0 * np.arange(K) + 1.0) * math.pi / beta


def trap_potential(L: tuple, c: float) -> np.ndarray:
    """V_i = c r_i^2 with r measured from the centre ((L_d - 1)/2 per axis), natural order."""
    axes = [np.arange(n, dtype=np.float64) - (n - 1) / 2.0 for n in L]
    grids = np.meshgrid(*axes, indexing="ij")          # grids[d][x, y, (z)]
    r2 = sum(g * g for g in grids)
    # natural order: x fastest -> transpose so that ravel() runs x fastest
    return np.ascontiguousarray(np.transpose(r2)).ravel() * c


def real_grid(t: float, K: int) -> np.ndarray:
    """K real frequencies spanning the band of the lattice and a margin: [-(4|t|+1), 4|t|+1]
    (the 2D band edge is 4|t|; in 3D, 6|t|, the grid then stops inside the band)."""
    e = 4.0 * abs(t) + 1.0
    return np.linspace(-e, e, K) if K > 1 else np.zeros(1)


def make_inputs(w: Workload, K: int | None = None, seed: int | None = None, axis: str = "matsubara"):
    """Draw (omega[K], V[N], sigma[K, N] complex128, q1[N] real) for a workload.

    The self-energy samples a_i, b_i and the start vector q1 come from one
    numpy Generator seeded with the workload's seed, in that order, so every
    consumer of the same (workload, seed) sees identical arrays.
    axis = "matsubara": omega are the fermionic Matsubara frequencies and
    Sigma_i(i w_k) = a_i - i b_i sign(w_k).  axis = "real": omega is a real
    grid across the band and Sigma_i(w) = a_i - i b_i, the retarded form
    (Im Sigma <= 0 for every w).
    """
    K = w.K if K is None else K
    seed = w.seed if seed is None else seed
    rng = np.random.default_rng(seed)
    N = w.N
    a = rng.uniform(-1.0, 1.0, N)
    b = rng.uniform(0.0, w.b_max, N)
    q1 = rng.uniform(-1.0, 1.0, N)
    if axis not in ("matsubara", "real"):
        raise ValueError("axis must be 'matsubara' or 'real'")
    omega = matsubara(w.beta, K) if axis == "matsubara" else real_grid(w.t, K)
    V = trap_potential(w.L, w.trap)
    sign = np.sign(omega)[:, None] if axis == "matsubara" else np.ones((K, 1))
    sigma = a[None, :] - 1j * b[None, :] * sign
    return omega, V, np.ascontiguousarray(sigma.astype(np.complex128)), q1


def homogeneous_inputs(L: tuple, omega: np.ndarray, sigma0: complex, q_seed: int = 7):
    """Constant self-energy, no trap: the case with a closed-form lattice Green's function."""
    N = int(np.prod(L))
    V = np.zeros(N)
    sigma = np.full((len(omega), N), sigma0, dtype=np.complex128)
    q1 = np.random.default_rng(q_seed).uniform(-1.0, 1.0, N)
    return np.asarray(omega, dtype=np.float64), V, sigma, q1


def start_block(q1: np.ndarray, nb: int, seed: int = 97) -> np.ndarray:
    """A real start block [nb][N] for block Lanczos: row 0 is q1, rows 1..nb-1
    are uniform(-1, 1) draws from generators seeded (seed, row)."""
    N = q1.shape[0]
    rows = [np.asarray(q1, dtype=np.float64)]
    for c in range(1, nb):
        rows.append(np.random.default_rng((seed, c)).uniform(-1.0, 1.0, N))
    return np.ascontiguousarray(np.stack(rows))
