"""Independent dense numpy brute force for tiny lattices (2^4, 4^4).

TEST INFRASTRUCTURE ONLY.  Shares no code with ``oracle.cpp``: the staggered
operator is written here on the *full* lattice with ``np.roll`` shifts,
M = 2m + D is formed as a dense matrix, and the even-odd operator is read off
as the even-even block of M^dagger M (the even-odd preconditioning of Sec. IV),
instead of being composed from two hops.  Solves are dense LU, spectra dense
eigendecompositions, and derivatives central finite differences.  The
Lie-algebra components of the force, F^a = Re tr(G^dagger T^a U) with the
Gell-Mann generators written out here, give the force norm of Sec. II.

Normalisation (the paper fixes none; this is the reading used throughout):
(D psi)(x) = sum_mu eta_mu(x) [b_mu(x) U_mu(x) psi(x+mu) - b_mu(x-mu) U_mu(x-mu)^dagger psi(x-mu)],
eta_mu(x) = (-1)^(x_0 + ... + x_{mu-1}), b = -1 on t-links wrapping Lt-1 -> 0 when bc_t = -1.
"""
from __future__ import annotations

import numpy as np

# array axis of direction mu in a (Lt, Lz, Ly, Lx, ...) field
_AX = {0: 3, 1: 2, 2: 1, 3: 0}


def _grid(dims):
    lx, ly, lz, lt = dims
    t, z, y, x = np.meshgrid(np.arange(lt), np.arange(lz), np.arange(ly), np.arange(lx), indexing="ij")
    return (x, y, z, t)


def eta(dims, mu):
    xs = _grid(dims)
    s = sum(xs[nu] for nu in range(mu)) if mu > 0 else np.zeros_like(xs[0])
    return np.where(s % 2 == 0, 1.0, -1.0)


def bsign(dims, mu, bc_t):
    xs = _grid(dims)
    b = np.ones(xs[0].shape)
    if mu == 3 and bc_t == -1:
        b[xs[3] == dims[3] - 1] = -1.0
    return b


def apply_D(dims, U, psi, bc_t=-1):
    """Full-lattice D psi; psi shape (Lt, Lz, Ly, Lx, 3)."""
    out = np.zeros_like(psi)
    for mu in range(4):
        ax = _AX[mu]
        Ub = U[..., mu, :, :] * bsign(dims, mu, bc_t)[..., None, None]
        fwd = np.einsum("...ab,...b->...a", Ub, np.roll(psi, -1, axis=ax))
        bwd = np.roll(np.einsum("...ba,...b->...a", Ub.conj(), psi), 1, axis=ax)
        out += eta(dims, mu)[..., None] * (fwd - bwd)
    return out


def dense_D(dims, U, bc_t=-1):
    """Dense matrix of D on the full lattice, index lex*3 + colour."""
    lx, ly, lz, lt = dims
    V = lx * ly * lz * lt
    Dm = np.zeros((3 * V, 3 * V), dtype=np.complex128)
    for k in range(3 * V):
        e = np.zeros(3 * V, dtype=np.complex128)
        e[k] = 1.0
        Dm[:, k] = apply_D(dims, U, e.reshape(lt, lz, ly, lx, 3), bc_t).reshape(-1)
    return Dm


def parity_lex(dims, p):
    """Lex indices of the sites of parity p, in rank order."""
    x, y, z, t = (a.reshape(-1) for a in _grid(dims))
    return np.nonzero((x + y + z + t) % 2 == p)[0]


def _rows(dims, p):
    lex = parity_lex(dims, p)
    return (lex[:, None] * 3 + np.arange(3)[None, :]).reshape(-1)


def dense_A(dims, mass, U, bc_t=-1):
    """Even-even block of M^dagger M, M = 2m + D (dense, 3V/2 x 3V/2)."""
    Dm = dense_D(dims, U, bc_t)
    M = 2.0 * mass * np.eye(Dm.shape[0]) + Dm
    MdM = M.conj().T @ M
    e = _rows(dims, 0)
    return MdM[np.ix_(e, e)]


def dense_blocks(dims, U, bc_t=-1):
    """(D_eo, D_oe) as dense matrices."""
    Dm = dense_D(dims, U, bc_t)
    e, o = _rows(dims, 0), _rows(dims, 1)
    return Dm[np.ix_(e, o)], Dm[np.ix_(o, e)]


def field_to_vec(F):
    """[Vh][3][n] parity field -> (3Vh, n) dense vectors in the same row order."""
    vh, _, n = F.shape
    return F.reshape(vh * 3, n)


def vec_to_field(v, n):
    return v.reshape(-1, 3, n)


def free_field_spectrum(dims, mass, bc_t=-1):
    """Closed form: even-sublattice eigenvalues of A at U = 1, ascending.

    Plane waves diagonalise -D^2 with eigenvalue 4 sum_mu sin^2 p_mu;
    p_mu = 2 pi k / L_mu, or (2k+1) pi / L_t in t when antiperiodic.  Each
    value has colour multiplicity 3, and p and p + (pi,pi,pi,pi) share it, one
    combination living on each parity, so the even spectrum is every other
    element of the sorted full spectrum.
    """
    lx, ly, lz, lt = dims
    ps = []
    for mu, L in enumerate(dims):
        k = np.arange(L)
        if mu == 3 and bc_t == -1:
            ps.append((2 * k + 1) * np.pi / L)
        else:
            ps.append(2 * k * np.pi / L)
    s = (np.sin(ps[0])[:, None, None, None] ** 2 + np.sin(ps[1])[None, :, None, None] ** 2
         + np.sin(ps[2])[None, None, :, None] ** 2 + np.sin(ps[3])[None, None, None, :] ** 2)
    lam = 4.0 * mass ** 2 + 4.0 * s.reshape(-1)
    full = np.sort(np.repeat(lam, 3))
    return full[::2]


def solve(Adense, B, sigma):
    """(A + sigma)^-1 B by dense LU; B (rows, n)."""
    return np.linalg.solve(Adense + sigma * np.eye(Adense.shape[0]), B)


def action(dims, mass, U, Phi, alpha0, alpha, beta, bc_t=-1):
    """S = sum_i phi_i^dagger [alpha_0 + sum_s alpha_s (A + beta_s)^-1] phi_i, dense."""
    A = dense_A(dims, mass, U, bc_t)
    B = field_to_vec(Phi)
    S = alpha0 * np.vdot(B, B).real
    for a, b in zip(alpha, beta):
        S += a * np.vdot(B, solve(A, B, b)).real
    return float(S)


def action_rational(dims, mass, U, Phi, alpha0, alpha, beta, bc_t=-1):
    """Same action through the eigendecomposition: sum_i phi^dagger R(A) phi, R(x) = a0 + sum a/(x+b)."""
    A = dense_A(dims, mass, U, bc_t)
    w, v = np.linalg.eigh(A)
    B = v.conj().T @ field_to_vec(Phi)
    R = alpha0 + sum(a / (w + b) for a, b in zip(alpha, beta))
    return float(np.sum(R[:, None] * np.abs(B) ** 2))


def fd_directional(dims, mass, U, Phi, alpha0, alpha, beta, V, h=1e-5, bc_t=-1):
    """Central difference (S(U + hV) - S(U - hV)) / 2h with dense solves."""
    Sp = action(dims, mass, U + h * V, Phi, alpha0, alpha, beta, bc_t)
    Sm = action(dims, mass, U - h * V, Phi, alpha0, alpha, beta, bc_t)
    return (Sp - Sm) / (2 * h)


def matrix_power_apply(dims, mass, U, Phi, r, bc_t=-1):
    """A^r Phi by dense eigendecomposition."""
    A = dense_A(dims, mass, U, bc_t)
    w, v = np.linalg.eigh(A)
    B = field_to_vec(Phi)
    return vec_to_field(v @ ((w ** r)[:, None] * (v.conj().T @ B)), Phi.shape[-1])


# ---------------------------------------------------------------- Lie-algebra force (Sec. II)
def gell_mann_matrices():
    """The eight Gell-Mann matrices lambda^a (Hermitian, traceless, tr(l^a l^b) = 2 delta_ab)."""
    L = np.zeros((8, 3, 3), dtype=np.complex128)
    L[0][0, 1] = L[0][1, 0] = 1
    L[1][0, 1], L[1][1, 0] = -1j, 1j
    L[2][0, 0], L[2][1, 1] = 1, -1
    L[3][0, 2] = L[3][2, 0] = 1
    L[4][0, 2], L[4][2, 0] = -1j, 1j
    L[5][1, 2] = L[5][2, 1] = 1
    L[6][1, 2], L[6][2, 1] = -1j, 1j
    L[7] = np.diag([1, 1, -2]) / np.sqrt(3)
    return L


def lie_components(U, G):
    """F^a = d S / d w along U -> exp(w T^a) U at every link, T^a = i lambda^a / 2.
    With G = dS/dRe U + i dS/dIm U, dS = Re tr(G^dagger dU), so F^a = Re tr(G^dagger T^a U).
    U, G (..., 3, 3); returns (..., 8)."""
    T = 0.5j * gell_mann_matrices()
    return np.einsum("...ji,ajk,...ki->...a", G.conj(), T, U).real


def force_norm2(U, G):
    """sum over links and a of (F^a)^2 / 2 (the summand of the force norm F^2, Sec. II)."""
    return float(0.5 * np.sum(lie_components(U, G) ** 2))


def ta_project(M):
    """Traceless anti-Hermitian part: (M - M^dagger)/2 - tr(M - M^dagger)/6."""
    A = 0.5 * (M - np.swapaxes(M.conj(), -1, -2))
    tr = np.trace(A, axis1=-2, axis2=-1)
    return A - (tr / 3.0)[..., None, None] * np.eye(3)


def force_lie(U, G):
    """F = TA(U G^dagger) per link."""
    return ta_project(U @ np.swapaxes(G.conj(), -1, -2))
