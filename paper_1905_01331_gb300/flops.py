"""Algorithmic floating-point work of one TTN sweep.

Counts 2*m*n*k for every matrix product the method needs (Sec. III.A: each
environment contribution reduces to products of cost at most O(chi^4); Sec. V:
the whole sweep costs O(chi^4)).  Products that the isometric constraint
removes (w w^dagger = I, Fig. 3) cost nothing and are not counted.  The
iterative parts -- the top eigensolver's matrix-vector products and the
polynomial iterations of the polar factor -- are counted separately, since
their count depends on the data; ``sweep_flops`` is the fixed part.

Units for an isometry layer with P = chi_{t+1}, n = chi_t:
  u1 = 2 P n^3  -- one one-site operator applied to one child leg of w
  u2 = 2 P^2 n^2 -- one product over both child legs, or of a P x P matrix with w
Per layer, K product terms:
  ascend   (2+4K) u1 + (1+2K) u2
  env      G W products: (2+4K) u2, new one-leg products (2+4K) u1; when every
           operator factor is symmetric the pairs (G, X) and (G^T, X^T) coincide
           and the environment needs (1+2K) u2 and no new one-leg product
  polar    one Gram and one apply: 2 u2 (one polynomial step)
  descend  (1+2K) u2 + 2K u1 (one-leg products with the new w) + (2+4K) u1 (traces)
Top (chi_T): adjoints (2+8K) products of 2 chi_T^3, energy (2+4K) of 2 chi_T^3.
"""
from __future__ import annotations


def layer_flops(P: int, n: int, K: int, symmetric: bool) -> float:
    u1 = 2.0 * P * n ** 3
    u2 = 2.0 * P * P * n * n
    f = (2 + 4 * K) * u1 + (1 + 2 * K) * u2                # ascend
    if symmetric:
        f += (1 + 2 * K) * u2                              # environment
    else:
        f += (2 + 4 * K) * u2 + (2 + 4 * K) * u1
    f += 2 * u2                                            # polar: Gram + apply
    f += (1 + 2 * K) * u2 + 2 * K * u1 + (2 + 4 * K) * u1  # descend
    return f


def top_flops(cT: int, K: int) -> float:
    return (2 + 8 * K) * 2.0 * cT ** 3 + (2 + 4 * K) * 2.0 * cT ** 3


def sweep_flops(L: int, chis, K: int, per_node: bool = False, symmetric: bool = True) -> float:
    """Fixed algorithmic flops of one sweep over a tree with bond dimensions
    ``chis`` (chi_0 .. chi_T).  Per-node trees repeat every layer's work on each
    of its L / 2^(t+1) nodes."""
    total = 0.0
    for t in range(len(chis) - 1):
        f = layer_flops(chis[t + 1], chis[t], K, symmetric)
        total += f * ((L >> (t + 1)) if per_node else 1)
    return total + top_flops(chis[-1], K)


def polar_step_flops(P: int, n: int) -> float:
    """One polynomial step of the polar iteration on a P x n^2 matrix: a Gram
    matrix and one application, 2 u2."""
    return 2 * 2.0 * P * P * n * n


def top_matvec_flops(cT: int, K: int) -> float:
    """One application of the two-site top Hamiltonian: (2+4K) products of
    chi_T x chi_T matrices."""
    return (2 + 4 * K) * 2.0 * cT ** 3
