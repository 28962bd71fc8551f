"""Seeded synthetic inputs for the block multishift RHMC path.

This module only draws random numbers and lays them out; it contains none of
the method's arithmetic (no Dirac operator, no solver, no force).  Both the
CUDA path and the CPU oracle consume what it produces.

Workload recipe (stands in for the thermalised 8^4, beta=5.12 ensembles of
the paper's Sec. IV, which are not available):

* gauge links U_mu(x) = exp(i * eps * H_mu(x)),  H = sum_a h^a lambda^a / 2,
  h^a ~ N(0, 1), lambda^a the Gell-Mann matrices; the exponential is taken
  through an FP64 eigendecomposition of the Hermitian H, so every link is
  unitary with unit determinant to rounding (SU(3));
* pseudofermions phi_i with complex Gaussian entries, Re and Im ~ N(0, 1/2),
  i.e. weight exp(-phi^dagger phi) as in the pseudofermion integral of Sec. II;
* random gauge transformations g(x) in SU(3) drawn like the links with eps=pi.

Layouts (shared convention of the C ABI):

* lattice site lex index  = x + Lx*(y + Ly*(z + Lz*t)), x fastest;
* gauge field  U[t][z][y][x][mu][a][b] complex128, mu = 0..3 = x, y, z, t;
* even (odd) sites have x+y+z+t even (odd); because Lx is even, the rank of a
  site among the sites of its parity is lex // 2;
* a pseudofermion block ("pencil") on one parity is [V/2][3][n] complex128,
  the n right-hand sides fastest.

Seeds: gauge field 1000 + k, pseudofermions 2000 + k, gauge transform 3000,
where k is the index of the workload (0-based).
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "gell_mann",
    "random_su3",
    "random_links",
    "unit_links",
    "gaussian_pseudofermions",
    "random_gauge_transform",
    "volume",
    "seed_gauge",
    "seed_phi",
    "SEED_GAUGE_TRANSFORM",
]

SEED_GAUGE_TRANSFORM = 3000


def seed_gauge(k: int) -> int:
    return 1000 + int(k)


def seed_phi(k: int) -> int:
    return 2000 + int(k)


def volume(dims) -> int:
    lx, ly, lz, lt = (int(d) for d in dims)
    return lx * ly * lz * lt


def _check_dims(dims):
    dims = tuple(int(d) for d in dims)
    if len(dims) != 4 or any(d < 2 or d % 2 for d in dims):
        raise ValueError(f"lattice extents must be four even integers >= 2, got {dims}")
    return dims


def gell_mann() -> np.ndarray:
    """The eight Gell-Mann matrices, shape (8, 3, 3) complex128."""
    lam = np.zeros((8, 3, 3), dtype=np.complex128)
    lam[0, 0, 1] = lam[0, 1, 0] = 1
    lam[1, 0, 1] = -1j
    lam[1, 1, 0] = 1j
    lam[2, 0, 0] = 1
    lam[2, 1, 1] = -1
    lam[3, 0, 2] = lam[3, 2, 0] = 1
    lam[4, 0, 2] = -1j
    lam[4, 2, 0] = 1j
    lam[5, 1, 2] = lam[5, 2, 1] = 1
    lam[6, 1, 2] = -1j
    lam[6, 2, 1] = 1j
    lam[7, 0, 0] = lam[7, 1, 1] = 1 / np.sqrt(3)
    lam[7, 2, 2] = -2 / np.sqrt(3)
    return lam


def random_su3(shape, eps: float, rng: np.random.Generator) -> np.ndarray:
    """exp(i eps H) for H = sum_a h^a lambda^a/2, h^a ~ N(0,1); shape + (3, 3)."""
    shape = tuple(shape)
    h = rng.standard_normal(shape + (8,))
    H = np.einsum("...a,aij->...ij", h, gell_mann()) * 0.5
    w, v = np.linalg.eigh(H)
    ph = np.exp(1j * eps * w)
    return np.einsum("...ij,...j,...kj->...ik", v, ph, v.conj())


def random_links(dims, eps: float, seed: int) -> np.ndarray:
    """Random SU(3) gauge field, shape (Lt, Lz, Ly, Lx, 4, 3, 3) complex128."""
    lx, ly, lz, lt = _check_dims(dims)
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.ascontiguousarray(random_su3((lt, lz, ly, lx, 4), eps, rng))


def unit_links(dims) -> np.ndarray:
    """Free field U = 1, shape (Lt, Lz, Ly, Lx, 4, 3, 3) complex128."""
    lx, ly, lz, lt = _check_dims(dims)
    U = np.zeros((lt, lz, ly, lx, 4, 3, 3), dtype=np.complex128)
    U[..., 0, 0] = U[..., 1, 1] = U[..., 2, 2] = 1
    return U


def gaussian_pseudofermions(dims, n: int, seed: int) -> np.ndarray:
    """n complex Gaussian fields on one parity, shape (V/2, 3, n) complex128."""
    _check_dims(dims)
    vh = volume(dims) // 2
    rng = np.random.Generator(np.random.PCG64(seed))
    z = rng.standard_normal((vh, 3, n, 2)) * np.sqrt(0.5)
    return np.ascontiguousarray(z[..., 0] + 1j * z[..., 1])


def momentum_normals(dims, seed: int) -> np.ndarray:
    """Standard normals p^a of the momentum heatbath, shape (Lt, Lz, Ly, Lx, 4, 8) float64."""
    lx, ly, lz, lt = _check_dims(dims)
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.standard_normal((lt, lz, ly, lx, 4, 8))


def random_gauge_transform(dims, seed: int = SEED_GAUGE_TRANSFORM) -> np.ndarray:
    """Random g(x) in SU(3), shape (Lt, Lz, Ly, Lx, 3, 3) complex128."""
    lx, ly, lz, lt = _check_dims(dims)
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.ascontiguousarray(random_su3((lt, lz, ly, lx), np.pi, rng))
