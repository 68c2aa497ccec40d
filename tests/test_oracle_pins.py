"""Pins of the FP64 oracle against things other than itself (CPU only).

Each test checks the oracle against a closed form, an exact diagonalisation
built spin by spin, a brute-force contraction of the whole tree, finite
differences, or an invariant the paper states (Eqs. (constraint),
(normalization); density matrices; the variational bound).
"""
import json
import math
import os

import numpy as np
import pytest

import ttn_inputs as ti
from oracle import ed, ttn
from paper_1905_01331_gb300 import flops

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _state(model, chi, seed, per_node=False):
    ws, V = ti.initial_tensors(model.Lx, model.d0, chi, seed, per_node)
    return ttn.make_state(model, ws, V, per_node=per_node)


# --- closed form and exact diagonalisation -----------------------------------

def test_closed_form_golden_values():
    """TFIM closed form at h = 1 reduces to -2 / sin(pi / (2L))."""
    with open(os.path.join(GOLDEN, "tfim_closed_form.json")) as f:
        g = json.load(f)
    for case in g["cases"]:
        L, h, E = case["L"], case["h"], case["E0"]
        assert abs(ed.tfim_closed_form(L, h) - E) < 1e-12 * abs(E)
        if h == 1.0:
            assert abs(E + 2.0 / math.sin(math.pi / (2 * L))) < 1e-12 * abs(E)


@pytest.mark.parametrize("L,h", [(6, 0.5), (8, 1.0), (10, 1.5), (12, 1.0)])
def test_closed_form_matches_sparse_ed(L, h):
    E_ed = ed.ground_energy(ed.tfim_chain_hamiltonian(L, h))
    assert abs(E_ed - ed.tfim_closed_form(L, h)) < 1e-11 * abs(E_ed)


def test_heisenberg_ed_limit():
    """Heisenberg ring: ED per site approaches 1 - 4 ln 2 (Bethe ansatz) from
    below as L grows; L = 4 has the exact value -8 (singlet, E = -2 L)."""
    assert abs(ed.ground_energy(ed.heisenberg_hamiltonian(4)) + 8.0) < 1e-12
    e12 = ed.ground_energy(ed.heisenberg_hamiltonian(12)) / 12
    assert -1.80 < e12 < 1 - 4 * math.log(2) + 0.0


# --- factorised model = lattice definition -----------------------------------

@pytest.mark.parametrize("per_node", [False, True])
@pytest.mark.parametrize("which", ["tfim", "heis", "torus"])
def test_energy_equals_brute_force_expectation(which, per_node):
    """Ascend + top energy equals <psi|H|psi> of the contracted state vector,
    with H built spin by spin from its definition (shift restored)."""
    if which == "tfim":
        m, H, chi = ti.tfim_chain(8, 0.7), ed.tfim_chain_hamiltonian(8, 0.7), 3
    elif which == "heis":
        m, H, chi = ti.heisenberg_xxx(8), ed.heisenberg_hamiltonian(8), 3
    else:
        m, H, chi = ti.tfim_torus(4, 3, 2.9), ed.torus_hamiltonian(4, 3, 2.9), 5
    st = _state(m, chi, 11, per_node)
    psi = ed.state_vector(st.ws, st.V, per_node=per_node)
    assert abs(np.linalg.norm(psi) - 1.0) < 1e-13
    E_brute = ed.expectation(psi, H)
    assert abs(ttn.energy(st) - E_brute) < 1e-12 * max(1.0, abs(E_brute))


@pytest.mark.parametrize("which", ["tfim", "heis", "torus"])
def test_full_chi_top_solve_is_exact(which):
    """With chi at the full Hilbert-space dimension every w is unitary and one
    top solve gives the exact ground energy, for any isometries."""
    if which == "tfim":
        m, E0, chi = ti.tfim_chain(8, 1.0), ed.tfim_closed_form(8, 1.0), 16
    elif which == "heis":
        m, E0, chi = ti.heisenberg_xxx(8), ed.ground_energy(ed.heisenberg_hamiltonian(8)), 16
    else:
        m, E0, chi = ti.tfim_torus(4, 3, 3.04), ed.ground_energy(ed.torus_hamiltonian(4, 3, 3.04)), 64
    st = _state(m, chi, 3)
    E = ttn.sweep(st)
    assert abs(E - E0) < 1e-11 * abs(E0)


def test_variational_and_monotone_l16_per_node():
    """TFIM L=16, chi=8, per node: energies never rise and stay above E0."""
    m = ti.tfim_chain(16, 1.0)
    st = _state(m, 8, 0, per_node=True)
    E0 = ed.tfim_closed_form(16, 1.0)
    Es = [ttn.sweep(st) for _ in range(30)]
    assert all(b <= a + 1e-11 * abs(a) for a, b in zip(Es, Es[1:]))
    assert min(Es) >= E0 - 1e-10
    assert Es[-1] - E0 < 2e-2


# --- isometries, top tensor, density matrices --------------------------------

def test_isometries_and_top_after_sweeps():
    st = _state(ti.heisenberg_xxx(32), 6, 5)
    for _ in range(4):
        ttn.sweep(st)
    for w in st.ws:
        W = w.reshape(w.shape[0], -1)
        assert np.abs(W @ W.T - np.eye(W.shape[0])).max() < 1e-13
    assert abs(np.linalg.norm(st.V) - 1.0) < 1e-14


def test_density_matrix_invariants():
    st = _state(ti.tfim_chain(64, 1.0), 8, 9)
    for _ in range(3):
        ttn.sweep(st)
    Fs, Ds = ttn.adjoints_all(st)
    for t, (R, _, _) in enumerate(Ds):
        assert abs(np.trace(R) - (st.L >> t)) < 1e-11 * (st.L >> t)
        assert np.abs(R - R.T).max() < 1e-12
        assert np.linalg.eigvalsh(R).min() > -1e-12
    rho = ttn.rdm(st, 2, which=1)
    assert abs(np.trace(rho) - 1) < 1e-13


def test_descended_density_matrices_match_brute_force():
    """Per node at L=8: descended R, P, Q equal the one- and two-site density
    matrices of the state vector expressed in the basis of site layer t."""
    m = ti.heisenberg_xxx(8)
    st = _state(m, 3, 21, per_node=True)
    Fs, Ds = ttn.adjoints_all(st)
    for t in range(len(st.ws)):
        psi = ed.state_vector(st.ws, st.V, per_node=True, stop_layer=t)
        N = st.L >> t
        d = Fs[t][0].shape[1]
        R, P, Q = Ds[t]
        for j in range(N):
            rho = ed.site_density_matrix(psi, N, d, j)
            assert np.abs(R[j] - rho).max() < 1e-12
            rho2 = ed.pair_density_matrix(psi, N, d, j)   # sites j, j+1
            A, B = Fs[t][1], Fs[t][2]
            jn = (j + 1) % N
            for k in range(m.K):
                # dE/dA_{k,j} over bond (j, j+1): sum_{b b'} rho2[a,b,a',b'] B_{k,j+1}[b,b']
                Pj = np.einsum("abcd,bd->ac", rho2, B[jn, k])
                Qjn = np.einsum("abcd,ac->bd", rho2, A[j, k])
                assert np.abs(P[j, k] - Pj).max() < 1e-12
                assert np.abs(Q[jn, k] - Qjn).max() < 1e-12


def test_top_reduced_density_matrices_share_spectrum():
    """Schmidt decomposition of V: rho_left = V V^T and rho_right = V^T V."""
    st = _state(ti.tfim_chain(32, 1.0), 6, 4)
    ttn.sweep(st)
    a = np.linalg.eigvalsh(st.V @ st.V.T)
    b = np.linalg.eigvalsh(st.V.T @ st.V)
    assert np.abs(a - b).max() < 1e-14
    lam, S = ttn.entanglement(st.V @ st.V.T)
    p = 2.0 ** (-lam)
    assert abs(p.sum() - 1) < 1e-12 and S >= 0


# --- environment (the derivative) and the layer identity ---------------------

@pytest.mark.parametrize("per_node", [False, True])
def test_environment_matches_finite_differences(per_node):
    """Gamma = dE/dw at fixed other tensors; Heisenberg has antisymmetric
    factors, so a transposition slip would show."""
    st = _state(ti.heisenberg_xxx(16), 4, 13, per_node)
    ttn.sweep(st)
    rng = np.random.default_rng(0)
    for layer in range(len(st.ws)):
        g = ttn.env_layer(st, layer)
        D = rng.standard_normal(st.ws[layer].shape)
        eps = 1e-6
        base = [w.copy() for w in st.ws]
        st.ws[layer] = base[layer] + eps * D
        Ep = ttn.energy(st)
        st.ws[layer] = base[layer] - eps * D
        Em = ttn.energy(st)
        st.ws[layer] = base[layer]
        fd = (Ep - Em) / (2 * eps)
        an = float(np.sum(g * D))
        assert abs(fd - an) < 1e-7 * max(1.0, abs(an))


def test_layer_identity():
    """E is linear in o_t and in each of {A_k,t}, {B_k,t}: by Euler,
    <R,o> + sum <P,A> = <R,o> + sum <Q,B> = E - cL at every site layer."""
    st = _state(ti.heisenberg_xxx(32), 5, 2)
    ttn.sweep(st)
    Fs, Ds = ttn.adjoints_all(st)
    E = ttn.energy(st) - st.c * st.L
    for (o, A, B), (R, P, Q) in zip(Fs, Ds):
        a = np.sum(R * o) + np.sum(P * A)
        b = np.sum(R * o) + np.sum(Q * B)
        assert abs(a - E) < 1e-12 * abs(E)
        assert abs(b - E) < 1e-12 * abs(E)


def test_translation_invariant_equals_uniform_per_node():
    """One shared w per layer is the per-node tree with identical nodes: same
    energy, and the shared environment is the sum of the node environments."""
    m = ti.tfim_chain(16, 0.9)
    ws, V = ti.initial_tensors(16, 2, 4, 8)
    ws_n = [np.stack([w] * (16 >> (t + 1))) for t, w in enumerate(ws)]
    a = ttn.make_state(m, ws, V)
    b = ttn.make_state(m, ws_n, V, per_node=True)
    assert abs(ttn.energy(a) - ttn.energy(b)) < 1e-12 * abs(ttn.energy(a))
    for layer in range(len(ws)):
        ga = ttn.env_layer(a, layer)
        gb = ttn.env_layer(b, layer).sum(axis=0)
        assert np.abs(ga - gb).max() < 1e-11 * np.abs(ga).max()


# --- shift and update ---------------------------------------------------------

@pytest.mark.parametrize("model", [ti.tfim_chain(8, 1.3), ti.heisenberg_xxx(8), ti.tfim_torus(8, 3, 2.9)])
def test_shift_makes_bond_terms_negative_semidefinite(model):
    c = ttn.bond_shift(model.o, model.A, model.B)
    d = model.d0
    I = np.eye(d)
    h = 0.5 * (np.kron(model.o, I) + np.kron(I, model.o))
    for a, b in zip(model.A, model.B):
        h = h + np.kron(a, b)
    ev = np.linalg.eigvalsh(0.5 * (h + h.T) - c * np.eye(d * d))
    assert ev.max() < 1e-12 and ev.max() > -1e-12


def test_polar_update_closed_form_and_fixed_point():
    """For gamma = -S Q (S symmetric positive definite, Q isometric) the update
    returns Q, with and without the proximal term, and Q is a fixed point."""
    rng = np.random.default_rng(1)
    P, n = 6, 3
    Q = np.linalg.qr(rng.standard_normal((n * n, P)))[0].T
    X = rng.standard_normal((P, P))
    S = X @ X.T + P * np.eye(P)
    gamma = (-S @ Q).reshape(P, n, n)
    other = np.linalg.qr(rng.standard_normal((n * n, P)))[0].T.reshape(P, n, n)
    w = ttn.polar_update(gamma, other, damping=0.0)
    assert np.abs(w.reshape(P, -1) - Q).max() < 1e-13
    w = ttn.polar_update(gamma, Q.reshape(P, n, n), damping=1e-3)
    assert np.abs(w.reshape(P, -1) - Q).max() < 1e-13


def test_flop_counter_scales_as_chi4():
    """Sec. V: cost O(chi^4); full layers of a doubled chi cost 16 times more."""
    r = flops.layer_flops(256, 256, 1, True) / flops.layer_flops(128, 128, 1, True)
    assert abs(r - 16.0) < 1e-12
    chis = ti.chi_schedule(1024, 2, 128)
    assert chis == [2, 4, 16, 128, 128, 128, 128, 128, 128, 128]
    f = flops.sweep_flops(1024, chis, 1)
    assert 5e10 < f < 2e11


# --- planted mistakes: each must be caught by a pin above ---------------------

def test_planted_mistakes_are_caught(monkeypatch):
    m, H = ti.tfim_chain(8, 0.7), ed.tfim_chain_hamiltonian(8, 0.7)
    ws, V = ti.initial_tensors(8, 2, 3, 4)
    E_ref = ed.expectation(ed.state_vector(ws, V), H)

    def energy_with(ascend_fn):
        monkeypatch.setattr(ttn, "ascend", ascend_fn)
        st = ttn.make_state(m, ws, V)
        return ttn.energy(st)

    good = ttn.ascend

    def drop_right_term(w, o, A, B):           # forget I (x) o
        inner = ttn.apply_pair(w, o, None)
        for a, b in zip(A, B):
            inner = inner + ttn.apply_pair(w, a, b)
        return ttn.close(inner, w), good(w, o, A, B)[1], good(w, o, A, B)[2]

    def swap_children(w, o, A, B):             # A' on the left child instead of the right
        o_up, _, B_up = good(w, o, A, B)
        A_up = np.stack([ttn.close(ttn.apply_pair(w, a, None), w) for a in A])
        return o_up, A_up, B_up

    for bad in (drop_right_term, swap_children):
        assert abs(energy_with(bad) - E_ref) > 1e-6
    assert abs(energy_with(good) - E_ref) < 1e-12


def test_top_polar_step_is_a_power_step_and_monotone():
    """top_mode = 1: v <- -H v/|H v| with the shifted, negative semidefinite
    top Hamiltonian never raises <v, H v> (power iteration), and the sweep
    energies never rise."""
    m = ti.tfim_chain(32, 0.8)
    st = _state(m, 6, 12)
    Fs = ttn.ascend_all(st)
    H = ttn.top_matrix(*Fs[-1])
    assert np.linalg.eigvalsh(H).max() < 1e-10          # shifted: NSD
    v0 = st.V.ravel()
    v1 = ttn.top_polar_step(st, Fs[-1]).ravel()
    assert abs(np.linalg.norm(v1) - 1) < 1e-14
    assert v1 @ H @ v1 <= v0 @ H @ v0 + 1e-12
    Es = [ttn.sweep(st, top_mode=1) for _ in range(6)]
    assert all(b <= a + 1e-11 * abs(a) for a, b in zip(Es, Es[1:]))


# --- pins added for the leftmost density matrix, the damping sign, entropy ----

@pytest.mark.parametrize("per_node", [False, True])
@pytest.mark.parametrize("which", ["tfim", "heis"])
def test_leftmost_density_matrix_matches_brute_force(which, per_node):
    """rdm(which=1) is the one-site density matrix of the leftmost site of
    each site layer, traced out of the contracted state vector.  The right
    spine (the other child at every level) gives another site's matrix and
    must fail the same comparison on some layer."""
    m = ti.tfim_chain(16, 0.8) if which == "tfim" else ti.heisenberg_xxx(16)
    st = _state(m, 3, 31, per_node)
    for _ in range(2):
        ttn.sweep(st)
    T = len(st.ws)
    right_spine_differs = False
    for t in range(T + 1):
        psi = ed.state_vector(st.ws, st.V, per_node=per_node, stop_layer=t)
        N, d = st.L >> t, (st.V.shape[0] if t == T else st.ws[t].shape[-1])
        brute = ed.site_density_matrix(psi, N, d, 0)
        rho = ttn.rdm(st, t, which=1)
        assert np.abs(rho - brute).max() < 1e-13
        # planted mistake: walk down through the right child instead
        wrong = st.V @ st.V.T
        for u in range(T - 1, t - 1, -1):
            w = st.ws[u][0] if per_node else st.ws[u]
            wrong = ttn.d_right(w, ttn.left_product(wrong, w))
        if np.abs(wrong - brute).max() > 1e-6:
            right_spine_differs = True
    assert right_spine_differs


def test_damping_keeps_old_isometry_on_null_directions():
    """Rank-deficient environment gamma = -S Q (S positive semidefinite of rank
    2 < P, Q isometric) with w_old = Q: on the null directions of S only the
    proximal term -mu |gamma| w_old is left, so the update must return w_old
    there, i.e. exactly Q.  With the opposite sign of the damping term the null
    directions flip and the result differs from Q by O(1)."""
    rng = np.random.default_rng(5)
    P, n = 5, 3
    Q = np.linalg.qr(rng.standard_normal((n * n, P)))[0].T
    U = np.linalg.qr(rng.standard_normal((P, P)))[0]
    S = U @ np.diag([3.0, 1.5, 0.0, 0.0, 0.0]) @ U.T
    gamma = (-S @ Q).reshape(P, n, n)
    w = ttn.polar_update(gamma, Q.reshape(P, n, n), damping=1e-7)
    assert np.abs(w.reshape(P, -1) - Q).max() < 1e-9
    g = gamma.reshape(P, -1) + 1e-7 * np.linalg.norm(gamma) * Q   # wrong sign
    Uw, _, Vt = np.linalg.svd(g, full_matrices=False)
    assert np.abs(-(Uw @ Vt) - Q).max() > 0.5


def test_entanglement_of_hand_computed_spectra():
    """Sec. IV.B: lambda = -log2 p, S = -sum p log2 p.  A density matrix with
    eigenvalues (1/2, 1/4, 1/4) in a random basis: lambda = (1, 2, 2) and
    S = 1.5 bits; the maximally mixed state of dimension 8: S = 3; a pure
    state: S = 0."""
    rng = np.random.default_rng(2)
    O = np.linalg.qr(rng.standard_normal((3, 3)))[0]
    lam, S = ttn.entanglement(O @ np.diag([0.25, 0.5, 0.25]) @ O.T)
    assert np.abs(np.sort(lam) - np.array([1.0, 2.0, 2.0])).max() < 1e-12
    assert abs(S - 1.5) < 1e-12
    lam, S = ttn.entanglement(np.eye(8) / 8)
    assert np.abs(lam - 3.0).max() < 1e-12 and abs(S - 3.0) < 1e-12
    v = rng.standard_normal(6)
    v /= np.linalg.norm(v)
    lam, S = ttn.entanglement(np.outer(v, v))
    assert abs(S) < 1e-12 and abs(lam[0]) < 1e-12
