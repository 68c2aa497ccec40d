"""FP64 CPU oracle of the tree-tensor-network (TTN) energy-minimisation sweep.

TEST INFRASTRUCTURE ONLY.  Nothing in the library's product path may import,
call or run this module; only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use it.  It shares no code with the CUDA path.

It is a plain, slow, direct transcription of the method of arXiv 1905.01331:

* a regular binary tree of isometries w (Sec. II.C, Eq. (constraint)) under a
  normalised top tensor v (Eq. (normalization));
* the environment E of each isometry as a sum of contributions of all
  Hamiltonian terms, contracted at O(chi^4) (Sec. III.A, Figs. 3, 4b);
* the update w <- from the SVD of the environment (Sec. III.B, Fig. 4c-d);
* one shared isometry per layer for translation-invariant H (Sec. III), or one
  isometry per node (the general labels w^(tau,m) of Sec. II.C).

Notation.  Site layer t has N_t = L / 2**t sites of dimension chi_t.  Isometry
layer t maps two site-t legs (left child l, right child r) to one site-(t+1)
leg p: ``w[p, l, r]``, or as a matrix W (P x n^2) with P = chi_{t+1}, n = chi_t.
The Hamiltonian is kept as ``sum_m [ o_m + sum_k A_k,m B_k,m+1 ]``; its bond
index has dimension K, not chi (Fig. 2b).  The pairing of two matrices is
``<X, Y> = sum_ij X_ij Y_ij``; ``d E / d X`` is meant in that pairing.

Readings of points the paper leaves open (each is stated where it is used):

* the sweep schedule -- "standard energy minimisation" (Sec. III): ascend all
  layers, solve the top, then update layers top-down, descending the density
  matrices with each freshly updated isometry;
* the update sign -- w = -(polar factor of dE/dw), with the Hamiltonian shifted
  by c per bond so that every bond term is negative semidefinite (Sec. III.B
  writes w = V U^dagger for the environment E = U S V^dagger without a sign);
* the top update "similarly" (Sec. III.B) -- the exact lowest eigenvector of
  the two-site top Hamiltonian;
* energy "per site" (Sec. IV) -- per spin, E / (Lx * Ly).
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.sparse.linalg as spla

# ---------------------------------------------------------------------------
# Small helpers.  ``w`` is an isometry (P, n, n) indexed [p, l, r].
# ---------------------------------------------------------------------------


def apply_pair(w, X1=None, X2=None):
    """W (X1 (x) X2): result[p, l', r'] = sum_{l,r} w[p,l,r] X1[l,l'] X2[r,r'].

    ``None`` stands for the identity on that child leg.
    """
    out = w
    if X1 is not None:
        out = np.einsum("plr,lm->pmr", out, X1, optimize=True)
    if X2 is not None:
        out = np.einsum("plr,rs->pls", out, X2, optimize=True)
    return out


def left_product(G, t):
    """G acting on the parent leg: result[p, l, r] = sum_q G[p,q] t[q,l,r]."""
    P = t.shape[0]
    return (G @ t.reshape(P, -1)).reshape(t.shape)


def close(a, b):
    """<a|b> over both child legs: result[p, q] = sum_{l,r} a[p,l,r] b[q,l,r]."""
    P, Q = a.shape[0], b.shape[0]
    return a.reshape(P, -1) @ b.reshape(Q, -1).T


def d_left(w, Gw, X2=None):
    """d/dX1 of <G, W (X1 (x) X2) W^T>, given Gw = G W.

    D[l, l'] = sum_{p,r,r'} w[p,l,r] X2[r,r'] (G W)[p,l',r'].
    """
    t = w if X2 is None else apply_pair(w, None, X2)
    return np.einsum("plr,pmr->lm", t, Gw, optimize=True)


def d_right(w, Gw, X1=None):
    """d/dX2 of <G, W (X1 (x) X2) W^T>, given Gw = G W.

    D[r, r'] = sum_{p,l,l'} w[p,l,r] X1[l,l'] (G W)[p,l',r'].
    """
    t = w if X1 is None else apply_pair(w, X1, None)
    return np.einsum("plr,pls->rs", t, Gw, optimize=True)


def bond_shift(o, A, B):
    """c = largest eigenvalue of the bond term 1/2 (o(x)I + I(x)o) + sum_k A_k (x) B_k.

    Subtracting c from o on every site makes each bond term negative
    semidefinite, so that the update w = -polar(dE/dw) cannot raise the energy.
    """
    d = o.shape[0]
    I = np.eye(d)
    h = 0.5 * (np.kron(o, I) + np.kron(I, o))
    for a, b in zip(A, B):
        h = h + np.kron(a, b)
    h = 0.5 * (h + h.T)
    return float(np.linalg.eigvalsh(h)[-1])


# Proximal weight of the update (a reading, see ``polar_update``).
POLAR_DAMPING = 1e-7


def polar_update(gamma, w_old, damping=POLAR_DAMPING):
    """Sec. III.B / Fig. 4c-d: from the SVD of the environment, the new isometry.

    ``gamma`` is dE/dw as a P x n^2 matrix (the paper's E flattened to
    n^2 x P is its transpose).  With gamma = U S V^T (thin SVD), the paper's
    w = V U^dagger of E = gamma^T is U V^T here; the update takes its negative.

    Reading: when E is numerically rank deficient (the top tensor's singular
    values fall to ~1e-13 of the largest), U and V are arbitrary on the null
    directions and any two SVD routines give different isometries there, which
    changes later sweeps at the 1e-5 level.  The update therefore takes the SVD
    of gamma - damping * ||gamma||_F * w_old: the null directions keep the old
    isometry, the fixed points w = -polar(gamma) are unchanged, and the energy
    still cannot rise (the added term is a proximal penalty).  The weight 1e-7
    is the smallest decade value at which two LAPACK SVD drivers (gesdd and
    gesvd) keep the per-sweep energies of the chain workloads within the FP64
    tolerance 1e-10 of each other (measured by oracle/damping_study.py:
    1.6e-11 on the 16-site per-node chain, 3e-14 on L=1024 at chi=32; at
    1e-8 already 1.6e-10, undamped 2.2e-5).
    """
    P = gamma.shape[0]
    g = gamma.reshape(P, -1)
    g = g - damping * np.linalg.norm(g) * w_old.reshape(P, -1)
    U, _, Vt = np.linalg.svd(g, full_matrices=False)
    return -(U @ Vt).reshape(gamma.shape)


# ---------------------------------------------------------------------------
# Translation-invariant (one shared isometry per layer) steps.
# Operators at a site layer: o (n x n), A, B (K x n x n).
# Adjoints (dE/d of those operators, summed over the sites): R, P, Q.
# ---------------------------------------------------------------------------


def ascend(w, o, A, B):
    """Coarse-grain the Hamiltonian through one layer (Fig. 3 pushed upward).

    o'   = W [o(x)I + I(x)o + sum_k A_k(x)B_k] W^T      (bond inside the block)
    A'_k = W (I(x)A_k) W^T                             (A on the right child)
    B'_k = W (B_k(x)I) W^T                             (B on the left child)
    """
    inner = apply_pair(w, o, None) + apply_pair(w, None, o)
    for a, b in zip(A, B):
        inner = inner + apply_pair(w, a, b)
    o_up = close(inner, w)
    A_up = np.stack([close(apply_pair(w, None, a), w) for a in A])
    B_up = np.stack([close(apply_pair(w, b, None), w) for b in B])
    return o_up, A_up, B_up


def top_apply(V, o, A, B):
    """Two-site top Hamiltonian on V: both bonds (1,2) and (2,1) of the ring.

    H_top V = o V + V o^T + sum_k (A_k V B_k^T + B_k V A_k^T).
    """
    out = o @ V + V @ o.T
    for a, b in zip(A, B):
        out = out + a @ V @ b.T + b @ V @ a.T
    return out


def top_matrix(o, A, B):
    """H_top as a dense (chi^2 x chi^2) matrix acting on vec(V) (row-major)."""
    c = o.shape[0]
    I = np.eye(c)
    H = np.kron(o, I) + np.kron(I, o)
    for a, b in zip(A, B):
        H = H + np.kron(a, b) + np.kron(b, a)
    return 0.5 * (H + H.T)


def top_ground(o, A, B, V_prev=None, dense_max=4096, tol=1e-13):
    """Lowest eigenvector of H_top ("the top tensor v is updated similarly").

    Dense symmetric eigensolver when chi^2 <= dense_max, else Lanczos (ARPACK)
    started from the previous V.  Sign: <V, V_prev> >= 0, or, without V_prev,
    the entry of largest magnitude positive.
    """
    c = o.shape[0]
    if c * c <= dense_max:
        evals, evecs = np.linalg.eigh(top_matrix(o, A, B))
        V = evecs[:, 0].reshape(c, c)
    else:
        op = spla.LinearOperator((c * c, c * c), dtype=np.float64,
                                 matvec=lambda x: top_apply(x.reshape(c, c), o, A, B).ravel())
        v0 = None if V_prev is None else V_prev.ravel()
        evals, evecs = spla.eigsh(op, k=1, which="SA", v0=v0, tol=tol, ncv=min(c * c, 40))
        V = evecs[:, 0].reshape(c, c)
    V = V / np.linalg.norm(V)
    if V_prev is not None:
        if np.sum(V * V_prev) < 0:
            V = -V
    else:
        i = np.argmax(np.abs(V))
        if V.flat[i] < 0:
            V = -V
    return V


def top_adjoints(V, A, B):
    """dE/d(top operators) for E = <V, H_top V>.

    R = V V^T + V^T V;  P_k = V B_k V^T + V^T B_k V;  Q_k = V^T A_k V + V A_k V^T.
    """
    R = V @ V.T + V.T @ V
    P = np.stack([V @ b @ V.T + V.T @ b @ V for b in B])
    Q = np.stack([V.T @ a @ V + V @ a @ V.T for a in A])
    return R, P, Q


def _env_terms(o, A, B):
    """(adjoint index, X1, X2) for every product operator that W is sandwiched
    around in ``ascend``; index 0 is R, 1+k is P_k, 1+K+k is Q_k."""
    K = len(A)
    terms = [(0, o, None), (0, None, o)]
    terms += [(0, A[k], B[k]) for k in range(K)]
    terms += [(1 + k, None, A[k]) for k in range(K)]
    terms += [(1 + K + k, B[k], None) for k in range(K)]
    return terms


def environment(w, o, A, B, R, P, Q):
    """Environment dE/dw of one isometry layer (Sec. III.A, Figs. 2b, 3).

    The energy is sum_(G, X) <G, W X W^T> over the pairs (R, o(x)I), (R, I(x)o),
    (R, A_k(x)B_k), (P_k, I(x)A_k), (Q_k, B_k(x)I); its derivative is
    Gamma = sum (G W X^T + G^T W X), a P x n x n tensor.  No assumption of
    symmetry is made on G or X.
    """
    G_all = [R] + list(P) + list(Q)
    gamma = np.zeros_like(w)
    for gi, X1, X2 in _env_terms(o, A, B):
        G = G_all[gi]
        X1t = None if X1 is None else X1.T
        X2t = None if X2 is None else X2.T
        gamma += left_product(G, apply_pair(w, X1t, X2t))
        gamma += left_product(G.T, apply_pair(w, X1, X2))
    return gamma


def descend(w, o, A, B, R, P, Q):
    """Adjoints one layer down: the derivatives of the energy with respect to
    the operators of site layer t, through ``ascend`` with isometry ``w``.

    With M = W^T R W (indexed (l,r),(l',r'), never formed):
    R-   = Tr_r M + Tr_l M
    P_k- = [sum_{r,r'} M(l,r,l',r') B_k(r,r')] + Tr_l(W^T P_k W)
    Q_k- = [sum_{l,l'} M(l,r,l',r') A_k(l,l')] + Tr_r(W^T Q_k W)
    These are summed density matrices of the lower layer (descending, Sec. IV).
    """
    Rw = left_product(R, w)
    R_dn = d_left(w, Rw) + d_right(w, Rw)
    P_dn = np.stack([d_left(w, Rw, B[k]) + d_right(w, left_product(P[k], w))
                     for k in range(len(A))])
    Q_dn = np.stack([d_right(w, Rw, A[k]) + d_left(w, left_product(Q[k], w))
                     for k in range(len(A))])
    return R_dn, P_dn, Q_dn


# ---------------------------------------------------------------------------
# One-isometry-per-node steps.  Site j of layer t carries its own o_j, the left
# factors A_k,j of bond (j, j+1) and the right factors B_k,j of bond (j-1, j);
# node J of isometry layer t has children 2J (left) and 2J+1 (right).
# ---------------------------------------------------------------------------


def ascend_nodes(ws, o, A, B):
    """``ascend`` node by node.  o: (N, n, n); A, B: (N, K, n, n)."""
    o_up, A_up, B_up = [], [], []
    for J, w in enumerate(ws):
        l, r = 2 * J, 2 * J + 1
        inner = apply_pair(w, o[l], None) + apply_pair(w, None, o[r])
        for k in range(A.shape[1]):
            inner = inner + apply_pair(w, A[l, k], B[r, k])
        o_up.append(close(inner, w))
        A_up.append(np.stack([close(apply_pair(w, None, A[r, k]), w) for k in range(A.shape[1])]))
        B_up.append(np.stack([close(apply_pair(w, B[l, k], None), w) for k in range(A.shape[1])]))
    return np.stack(o_up), np.stack(A_up), np.stack(B_up)


def top_apply_nodes(V, o, A, B):
    """Top Hamiltonian with site-dependent operators of the two top sites."""
    out = o[0] @ V + V @ o[1].T
    for k in range(A.shape[1]):
        out = out + A[0, k] @ V @ B[1, k].T + B[0, k] @ V @ A[1, k].T
    return out


def top_matrix_nodes(o, A, B):
    c = o.shape[1]
    I = np.eye(c)
    H = np.kron(o[0], I) + np.kron(I, o[1])
    for k in range(A.shape[1]):
        H = H + np.kron(A[0, k], B[1, k]) + np.kron(B[0, k], A[1, k])
    return 0.5 * (H + H.T)


def top_adjoints_nodes(V, A, B):
    """Site-resolved top adjoints (shape (2, ...))."""
    R = np.stack([V @ V.T, V.T @ V])
    K = A.shape[1]
    P = np.stack([np.stack([V @ B[1, k] @ V.T for k in range(K)]),
                  np.stack([V.T @ B[0, k] @ V for k in range(K)])])
    Q = np.stack([np.stack([V @ A[1, k] @ V.T for k in range(K)]),
                  np.stack([V.T @ A[0, k] @ V for k in range(K)])])
    return R, P, Q


def environment_nodes(ws, o, A, B, R, P, Q):
    """Per-node environments: node J sees only its own adjoints and children."""
    out = []
    K = A.shape[1]
    for J, w in enumerate(ws):
        l, r = 2 * J, 2 * J + 1
        terms = [(R[J], o[l], None), (R[J], None, o[r])]
        terms += [(R[J], A[l, k], B[r, k]) for k in range(K)]
        terms += [(P[J, k], None, A[r, k]) for k in range(K)]
        terms += [(Q[J, k], B[l, k], None) for k in range(K)]
        g = np.zeros_like(w)
        for G, X1, X2 in terms:
            X1t = None if X1 is None else X1.T
            X2t = None if X2 is None else X2.T
            g += left_product(G, apply_pair(w, X1t, X2t))
            g += left_product(G.T, apply_pair(w, X1, X2))
        out.append(g)
    return np.stack(out)


def descend_nodes(ws, o, A, B, R, P, Q):
    """Per-node ``descend``: children 2J, 2J+1 of node J get their own adjoints."""
    N = 2 * len(ws)
    K = A.shape[1]
    n = ws.shape[2]
    R_dn = np.zeros((N, n, n))
    P_dn = np.zeros((N, K, n, n))
    Q_dn = np.zeros((N, K, n, n))
    for J, w in enumerate(ws):
        l, r = 2 * J, 2 * J + 1
        Rw = left_product(R[J], w)
        R_dn[l] = d_left(w, Rw)
        R_dn[r] = d_right(w, Rw)
        for k in range(K):
            P_dn[l, k] = d_left(w, Rw, B[r, k])             # intra bond, A on the left child
            P_dn[r, k] = d_right(w, left_product(P[J, k], w))  # straddling bond, A on the right child
            Q_dn[r, k] = d_right(w, Rw, A[l, k])            # intra bond, B on the right child
            Q_dn[l, k] = d_left(w, left_product(Q[J, k], w))   # straddling bond, B on the left child
    return R_dn, P_dn, Q_dn


# ---------------------------------------------------------------------------
# The sweep.
# ---------------------------------------------------------------------------


@dataclasses.dataclass
class State:
    """A TTN for a periodic chain of L effective sites."""
    L: int
    n_spins: int
    o: np.ndarray          # shifted one-site term at layer 0 (d0 x d0)
    A: np.ndarray          # (K, d0, d0)
    B: np.ndarray
    c: float               # bond shift
    ws: list               # per layer (P, n, n) or (N, P, n, n)
    V: np.ndarray
    per_node: bool = False
    sweeps_done: int = 0


def make_state(model, ws, V, c=None, per_node=False):
    """Set up a state from a factorised model and initial tensors (step a0)."""
    if c is None:
        c = bond_shift(model.o, model.A, model.B)
    o = model.o - c * np.eye(model.d0)
    return State(model.Lx, model.n_spins, o, model.A.copy(), model.B.copy(), float(c),
                 [np.array(w, dtype=np.float64) for w in ws], np.array(V, dtype=np.float64),
                 per_node)


def layer0_operators(st):
    """Operators at site layer 0, site-resolved when the tree is per-node."""
    if not st.per_node:
        return st.o, st.A, st.B
    L = st.L
    K = st.A.shape[0]
    return (np.broadcast_to(st.o, (L,) + st.o.shape).copy(),
            np.broadcast_to(st.A, (L, K) + st.A.shape[1:]).copy(),
            np.broadcast_to(st.B, (L, K) + st.B.shape[1:]).copy())


def ascend_all(st):
    """Operators of every site layer 0..T (forward half of the sweep)."""
    Fs = [layer0_operators(st)]
    for w in st.ws:
        f = ascend_nodes if st.per_node else ascend
        Fs.append(f(w, *Fs[-1]))
    return Fs


def top_energy(st, V, F_top):
    """<V, H_top V> + c L: the energy of the state, restoring the shift."""
    f = top_apply_nodes if st.per_node else top_apply
    return float(np.sum(V * f(V, *F_top))) + st.c * st.L


def solve_top(st, F_top):
    """New top tensor: lowest eigenvector of H_top, sign aligned with the old V."""
    if st.per_node:
        c = F_top[0].shape[1]
        if c * c <= 4096:
            V = np.linalg.eigh(top_matrix_nodes(*F_top))[1][:, 0].reshape(c, c)
        else:
            op = spla.LinearOperator((c * c, c * c), dtype=np.float64,
                                     matvec=lambda x: top_apply_nodes(x.reshape(c, c), *F_top).ravel())
            V = spla.eigsh(op, k=1, which="SA", v0=st.V.ravel(), tol=1e-13)[1][:, 0].reshape(c, c)
        V = V / np.linalg.norm(V)
        if np.sum(V * st.V) < 0:
            V = -V
        return V
    return top_ground(*F_top, V_prev=st.V)


def top_polar_step(st, F_top):
    """The literal reading of "the top tensor v is updated similarly" (Sec.
    III.B): v <- minus the polar factor of its environment.  The environment of
    v is H_top v (dE/dv = 2 H_top v); the polar factor of a single vector is
    the vector normalised, so v <- -H_top v / |H_top v|.  With the shifted
    (negative semidefinite) Hamiltonian this is one power-iteration step toward
    the lowest eigenvector."""
    f = top_apply_nodes if st.per_node else top_apply
    g = f(st.V, *F_top)
    return -g / np.linalg.norm(g)


def sweep(st, top_mode=0):
    """One sweep (Sec. III): ascend, top solve, then top-down updates.

    Returns the energy found by the top solve (the energy of the state made of
    the isometries at the start of the sweep and the new top tensor).
    top_mode 0: the top tensor is the lowest eigenvector of H_top; 1: one
    polar step of its environment (``top_polar_step``).
    """
    Fs = ascend_all(st)
    T = len(st.ws)
    V = solve_top(st, Fs[T]) if top_mode == 0 else top_polar_step(st, Fs[T])
    E = top_energy(st, V, Fs[T])
    st.V = V
    if st.per_node:
        D = top_adjoints_nodes(V, Fs[T][1], Fs[T][2])
    else:
        D = top_adjoints(V, Fs[T][1], Fs[T][2])
    for t in range(T - 1, -1, -1):
        o, A, B = Fs[t]
        if st.per_node:
            gam = environment_nodes(st.ws[t], o, A, B, *D)
            st.ws[t] = np.stack([polar_update(g, w) for g, w in zip(gam, st.ws[t])])
            D = descend_nodes(st.ws[t], o, A, B, *D)
        else:
            gam = environment(st.ws[t], o, A, B, *D)
            st.ws[t] = polar_update(gam, st.ws[t])
            D = descend(st.ws[t], o, A, B, *D)
    st.sweeps_done += 1
    return E


def energy(st):
    """Energy <psi|H|psi> of the stored tensors (no re-optimisation)."""
    Fs = ascend_all(st)
    return top_energy(st, st.V, Fs[-1])


def run(model, chi, seed, sweeps, per_node=False):
    """Initial tensors from the shared seeded generator, then ``sweeps`` sweeps.
    Returns (state, energies)."""
    from ttn_inputs import initial_tensors
    ws, V = initial_tensors(model.Lx, model.d0, chi, seed, per_node)
    st = make_state(model, ws, V, per_node=per_node)
    Es = [sweep(st) for _ in range(sweeps)]
    return st, Es


# ---------------------------------------------------------------------------
# Analysis: density matrices, entanglement (Sec. IV.B), layer diagnostics.
# ---------------------------------------------------------------------------


def adjoints_all(st):
    """Adjoints (R, P, Q) of every site layer for the stored tensors, without
    updating anything.  Index t is site layer t; index T is the top."""
    Fs = ascend_all(st)
    T = len(st.ws)
    if st.per_node:
        D = top_adjoints_nodes(st.V, Fs[T][1], Fs[T][2])
    else:
        D = top_adjoints(st.V, Fs[T][1], Fs[T][2])
    Ds = [None] * (T + 1)
    Ds[T] = D
    for t in range(T - 1, -1, -1):
        f = descend_nodes if st.per_node else descend
        D = f(st.ws[t], *Fs[t], *D)
        Ds[t] = D
    return Fs, Ds


def rdm(st, site_layer, which=0):
    """Reduced density matrix on one bond of site layer ``site_layer``.

    which=0: the site average R / N_t; which=1: the leftmost site's density
    matrix, V V^T at the top, then Tr_r(W^T rho W) down the left spine.
    """
    T = len(st.ws)
    if which == 0:
        _, Ds = adjoints_all(st)
        R = Ds[site_layer][0]
        if st.per_node:
            R = R.sum(axis=0)
        return R / (st.L >> site_layer)
    rho = st.V @ st.V.T
    for t in range(T - 1, site_layer - 1, -1):
        w = st.ws[t][0] if st.per_node else st.ws[t]
        rho = d_left(w, left_product(rho, w))
    return rho


def entanglement(rho):
    """Entanglement spectrum lambda_a = -log2 p_a and entropy S = -sum p log2 p
    of a density matrix (Sec. IV.B)."""
    p = np.linalg.eigvalsh(0.5 * (rho + rho.T))[::-1]
    p = p[p > 0]
    return -np.log2(p), float(-np.sum(p * np.log2(p)))


def env_layer(st, layer):
    """dE/dw of isometry layer ``layer`` at the stored tensors (no update)."""
    Fs, Ds = adjoints_all(st)
    f = environment_nodes if st.per_node else environment
    return f(st.ws[layer], *Fs[layer], *Ds[layer + 1])
