"""Seeded synthetic inputs shared by the FP64 oracle and the CUDA path.

This module holds input data only and none of the sweep's arithmetic:

* the one-site Pauli matrices and the factorised nearest-neighbour Hamiltonians
  ``H = sum_m [ o_m + sum_k A_k,m B_k,m+1 ]`` that the library takes as its
  "H terms" (Sec. II.A-B, Eqs. (H2D), (H1D), (1)-(5));
* the seeded initial isometries and top tensor (Gaussian matrices made
  orthonormal by QR; the paper does not state an initialisation);
* the recipes of the five synthetic workloads (chain, Heisenberg, thin torus,
  batched chains) with their seeds.

Neither the oracle nor the CUDA path imports the other; both import this.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# Pauli matrices, all real.  iY = [[0, 1], [-1, 0]] is i times Pauli Y, so that
# Y (x) Y = -(iY) (x) (iY) keeps the Heisenberg chain real.
I2 = np.eye(2)
X = np.array([[0.0, 1.0], [1.0, 0.0]])
Z = np.array([[1.0, 0.0], [0.0, -1.0]])
IY = np.array([[0.0, 1.0], [-1.0, 0.0]])


@dataclasses.dataclass
class Model:
    """A translation-invariant chain Hamiltonian in factorised form.

    ``o`` is the one-site term (d0 x d0); ``A[k]`` and ``B[k]`` (K x d0 x d0) are
    the factors of the K product terms on each bond (m, m+1):
    ``H = sum_m [ o_m + sum_k A[k]_m B[k]_{m+1} ]`` on a periodic chain of
    ``Lx`` effective sites.  For a thin torus each effective site is one column
    of ``Ly`` spins, ``d0 = 2**Ly``.
    """
    name: str
    Lx: int
    Ly: int
    o: np.ndarray
    A: np.ndarray
    B: np.ndarray
    params: dict

    @property
    def d0(self) -> int:
        return self.o.shape[0]

    @property
    def K(self) -> int:
        return self.A.shape[0]

    @property
    def n_spins(self) -> int:
        return self.Lx * self.Ly


def tfim_chain(L: int, h: float) -> Model:
    """Periodic transverse-field Ising chain ``H = -sum Z_i Z_{i+1} - h sum X_i``.

    The paper's form ``-XX + hZ`` (Eq. (H2D) with Ly = 1) is unitarily equivalent
    (Hadamard on every site, then conjugation by the string of Z), so it has the
    same spectrum.  One product term: A = -Z, B = Z.
    """
    return Model("tfim_chain", L, 1, -h * X, np.stack([-Z]), np.stack([Z]), {"h": h})


def heisenberg_xxx(L: int) -> Model:
    """Periodic antiferromagnetic Heisenberg chain ``H = sum (XX + YY + ZZ)``.

    Three product terms (X, X), (iY, -iY), (Z, Z); the middle one equals Y (x) Y.
    The iY factors are antisymmetric, so no product factor may be assumed
    symmetric.
    """
    return Model("heisenberg_xxx", L, 1, np.zeros((2, 2)),
                 np.stack([X, IY, Z]), np.stack([X, -IY, Z]), {})


def _site_op(op: np.ndarray, n: int, Ly: int) -> np.ndarray:
    """``op`` on spin n (0-based) of a column of Ly spins, as a 2**Ly matrix."""
    out = np.ones((1, 1))
    for j in range(Ly):
        out = np.kron(out, op if j == n else I2)
    return out


def tfim_torus(Lx: int, Ly: int, h: float) -> Model:
    """2D transverse-field Ising model on an Lx x Ly thin torus, Eq. (H2D).

    ``H = sum_{m,n} ( -X_(m,n) X_(m+1,n) - X_(m,n) X_(m,n+1) + h Z_(m,n) )``.
    Each column of Ly spins is one effective site of dimension d0 = 2**Ly
    (Sec. II.B).  The one-site term ``o`` is the whole column Hamiltonian: the
    vertical bonds (periodic in y) and the fields, without the 1/2 that Eqs.
    (2)-(5) use to share it between the two bonds touching the column.  The
    horizontal bonds are K = Ly product terms A_n = -X_(n), B_n = X_(n).
    For Ly = 1 there are no vertical bonds; for Ly = 2 the periodic sum over n
    visits the single vertical pair twice, as Eq. (H2D) written literally does.
    """
    d0 = 2 ** Ly
    o = np.zeros((d0, d0))
    if Ly >= 2:
        for n in range(Ly):
            o -= _site_op(X, n, Ly) @ _site_op(X, (n + 1) % Ly, Ly)
    for n in range(Ly):
        o += h * _site_op(Z, n, Ly)
    A = np.stack([-_site_op(X, n, Ly) for n in range(Ly)])
    B = np.stack([_site_op(X, n, Ly) for n in range(Ly)])
    return Model("tfim_torus", Lx, Ly, o, A, B, {"h": h})


def chi_schedule(L: int, d0: int, chi: int) -> list[int]:
    """Bond dimensions chi_0..chi_T of site layers 0..T, T = log2(L) - 1.

    chi_0 = d0 and chi_{t+1} = min(chi, chi_t**2): the bond cap
    min(chi, d0**(2**t)) of the regular binary tree (Sec. II.C).
    """
    n = int(round(math.log2(L)))
    if 2 ** n != L or L < 4:
        raise ValueError("L must be a power of two >= 4")
    chis = [d0]
    for _ in range(n - 1):
        chis.append(min(chi, chis[-1] ** 2))
    return chis


def _random_isometry(rng: np.random.Generator, P: int, n: int) -> np.ndarray:
    """Gaussian n^2 x P matrix, QR, column signs with diag(R) > 0, W = Q^T."""
    G = rng.standard_normal((n * n, P))
    Q, R = np.linalg.qr(G)
    Q = Q * np.sign(np.diag(R))[None, :]
    return np.ascontiguousarray(Q.T.reshape(P, n, n))


def initial_tensors(L: int, d0: int, chi: int, seed: int, per_node: bool = False):
    """Seeded initial isometries and top tensor.

    Returns ``(ws, V)``.  ``ws[t]`` has shape (P, n, n) with P = chi_{t+1} and
    n = chi_t (one shared isometry per layer), or (N_{t+1}, P, n, n) with one
    isometry per node when ``per_node``.  Draw order: layer 0 first; within a
    layer, node 0 first; then V.  Each isometry is the transpose of the Q of a
    Gaussian n^2 x P matrix (signs fixed so diag R > 0); V is Gaussian with
    unit Frobenius norm (Eqs. (constraint), (normalization)).
    """
    rng = np.random.default_rng(seed)
    chis = chi_schedule(L, d0, chi)
    ws = []
    for t in range(len(chis) - 1):
        n, P = chis[t], chis[t + 1]
        if per_node:
            nodes = L >> (t + 1)
            ws.append(np.stack([_random_isometry(rng, P, n) for _ in range(nodes)]))
        else:
            ws.append(_random_isometry(rng, P, n))
    cT = chis[-1]
    V = rng.standard_normal((cT, cT))
    V /= np.linalg.norm(V)
    return ws, V


# ---------------------------------------------------------------------------
# The five workloads, named by what they are.
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class Workload:
    name: str
    model: Model
    chi: int
    seed: int
    sweeps: int
    per_node: bool = False


def tfim_l16_pernode() -> Workload:
    """TFIM chain L=16, h=1, chi=8, one isometry per node, seed 0, 30 sweeps."""
    return Workload("tfim_L16_chi8_pernode", tfim_chain(16, 1.0), 8, 0, 30, True)


def tfim_l1024(chi: int = 128, sweeps: int = 200) -> Workload:
    """Critical TFIM chain L=1024, h=1, chi in {32, 64, 128}, seed 1, 200 sweeps."""
    return Workload(f"tfim_L1024_chi{chi}", tfim_chain(1024, 1.0), chi, 1, sweeps)


def heisenberg_l256(chi: int = 256, sweeps: int = 100) -> Workload:
    """Heisenberg XXX chain L=256, chi=256, K=3, seed 2, 100 sweeps."""
    return Workload(f"heisenberg_L256_chi{chi}", heisenberg_xxx(256), chi, 2, sweeps)


def torus_64x4(chi: int = 128, sweeps: int = 100) -> Workload:
    """TFIM on a 64 x 4 thin torus, h=3.04, d0=16, K=4, chi=128, seed 3."""
    return Workload(f"torus_64x4_chi{chi}", tfim_torus(64, 4, 3.04), chi, 3, sweeps)


def batched_chains(count: int = 64, seed: int = 4, sweeps: int = 100):
    """Independent TFIM chains: per instance, in order, h ~ U[0.5, 1.5],
    L ~ {64, 128, 256, 512}, chi ~ {32, 64, 128}; then that instance's
    isometries are drawn from a seed taken from the same generator."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        h = float(rng.uniform(0.5, 1.5))
        L = int(rng.choice([64, 128, 256, 512]))
        chi = int(rng.choice([32, 64, 128]))
        iseed = int(rng.integers(0, 2**31 - 1))
        out.append(Workload(f"batch{i}_tfim_L{L}_chi{chi}", tfim_chain(L, h), chi, iseed, sweeps))
    return out
