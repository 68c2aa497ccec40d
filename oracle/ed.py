"""Exact references that pin the TTN oracle (test infrastructure only).

Nothing in the library's product path may import or run this module.

* Lattice Hamiltonians built spin by spin from their definitions (Eq. (H2D) for
  the thin torus; the periodic Ising and Heisenberg chains), independently of
  the factorised one-site / product-term form the sweep uses.
* Ground energies by sparse exact diagonalisation (small lattices) and the
  closed form of the periodic transverse-field Ising chain.
* The full state vector of a small TTN, contracted node by node from the top
  tensor down, and brute-force expectation values and reduced density
  matrices computed from it.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

_SX = np.array([[0.0, 1.0], [1.0, 0.0]])
_SZ = np.array([[1.0, 0.0], [0.0, -1.0]])
_SY = np.array([[0.0, -1.0j], [1.0j, 0.0]])


def _op_on(ops: dict, n: int):
    """Sparse Kronecker product over n spins with ``ops[i]`` on spin i."""
    out = sp.identity(1, format="csr", dtype=complex)
    for i in range(n):
        m = ops.get(i)
        out = sp.kron(out, sp.csr_matrix(m) if m is not None else sp.identity(2, format="csr"),
                      format="csr")
    return out


def tfim_chain_hamiltonian(L: int, h: float):
    """-sum_i Z_i Z_{i+1} - h sum_i X_i with periodic boundary, as a sparse matrix."""
    H = sp.csr_matrix((2 ** L, 2 ** L), dtype=complex)
    for i in range(L):
        H = H - _op_on({i: _SZ, (i + 1) % L: _SZ}, L) - h * _op_on({i: _SX}, L)
    return H.real.tocsr()


def heisenberg_hamiltonian(L: int):
    """sum_i (X_i X_{i+1} + Y_i Y_{i+1} + Z_i Z_{i+1}), periodic, with complex Y."""
    H = sp.csr_matrix((2 ** L, 2 ** L), dtype=complex)
    for i in range(L):
        j = (i + 1) % L
        for s in (_SX, _SY, _SZ):
            H = H + _op_on({i: s, j: s}, L)
    assert abs(H.imag).max() < 1e-14
    return H.real.tocsr()


def torus_hamiltonian(Lx: int, Ly: int, h: float):
    """Eq. (H2D) on an Lx x Ly torus; spin (m, n) has index m * Ly + n.

    sum_{m,n} ( -X_(m,n) X_(m+1,n) - X_(m,n) X_(m,n+1) + h Z_(m,n) ), both
    directions periodic.  Vertical bonds are taken for Ly >= 2 only; for
    Ly = 2 the sum over n counts the single vertical pair twice (literal sum).
    """
    N = Lx * Ly
    H = sp.csr_matrix((2 ** N, 2 ** N), dtype=complex)
    idx = lambda m, n: (m % Lx) * Ly + (n % Ly)
    for m in range(Lx):
        for n in range(Ly):
            H = H - _op_on({idx(m, n): _SX, idx(m + 1, n): _SX}, N)
            if Ly >= 2:
                H = H - _op_on({idx(m, n): _SX, idx(m, n + 1): _SX}, N)
            H = H + h * _op_on({idx(m, n): _SZ}, N)
    return H.real.tocsr()


def ground_energy(H) -> float:
    """Lowest eigenvalue of a sparse symmetric matrix."""
    if H.shape[0] <= 4096:
        return float(np.linalg.eigvalsh(H.toarray())[0])
    return float(spla.eigsh(H, k=1, which="SA", tol=1e-14)[0][0])


def tfim_closed_form(L: int, h: float) -> float:
    """Ground energy of the periodic TFIM chain -sum ZZ - h sum X (Jordan-Wigner).

    E0 = -sum_{n=0}^{L-1} sqrt(1 + h^2 - 2 h cos((2n+1) pi / L)); the ground
    state lies in the even-parity sector with antiperiodic fermion momenta.
    At h = 1 this is -2 / sin(pi / (2L)).
    """
    k = (2 * np.arange(L) + 1) * math.pi / L
    return float(-np.sum(np.sqrt(1.0 + h * h - 2.0 * h * np.cos(k))))


# ---------------------------------------------------------------------------
# Brute-force state vector of a TTN.
# ---------------------------------------------------------------------------


def state_vector(ws, V, per_node=False, stop_layer=0):
    """Contract the tree into the amplitudes on site layer ``stop_layer``.

    Start from the two top legs of V; replace every leg of site layer t+1 by
    its two children through w_t (w[p, l, r]: parent p -> children (l, r)),
    down to site layer ``stop_layer``.  Returns a vector of length
    prod_j chi_{stop_layer}, sites ordered left to right, the leftmost most
    significant.
    """
    psi = np.array(V, dtype=np.float64)       # shape (c, c)
    T = len(ws)
    for t in range(T - 1, stop_layer - 1, -1):
        N_parent = psi.ndim
        for J in range(N_parent - 1, -1, -1):
            w = ws[t][J] if per_node else ws[t]
            # contract leg J of psi with w's parent leg; children take its place
            psi = np.tensordot(psi, w, axes=([J], [0]))        # legs: others..., l, r
            psi = np.moveaxis(psi, [-2, -1], [J, J + 1])
    return psi.reshape(-1)


def expectation(psi, H) -> float:
    return float(psi @ (H @ psi)) / float(psi @ psi)


def site_density_matrix(psi, n_sites, d, j):
    """rho_j[a, a'] = sum over the other sites of psi psi^T."""
    t = psi.reshape((d,) * n_sites)
    t = np.moveaxis(t, j, 0).reshape(d, -1)
    return t @ t.T


def pair_density_matrix(psi, n_sites, d, j):
    """Two-site density matrix of sites j, j+1 (periodic), as (d, d, d, d)
    indexed [a, b, a', b'] for site j (a) and j+1 (b)."""
    t = psi.reshape((d,) * n_sites)
    k = (j + 1) % n_sites
    t = np.moveaxis(t, [j, k], [0, 1]).reshape(d * d, -1)
    return (t @ t.T).reshape(d, d, d, d)
