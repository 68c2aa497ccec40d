"""The paper's workload shape (Sec. IV): the thin-torus transverse-field Ising
model at h = 2.9 with columns of Ly = 5 spins (d0 = 32, K = 5 product terms),
here 16 x 5 at chi = 32.  After FP64 sweeps on the GPU, the leftmost site's
density matrix of every site layer (the rho of Sec. IV.B's entanglement
spectrum, the upper bond of the leftmost isometry) matches the oracle's on
the same tensors element by element, and so do its entanglement spectrum and
entropy.  Exact diagonalisation of 80 spins is out of reach, so the energy
is checked against the oracle's energy of the same tensors, and the sweeps
must not raise it."""
import numpy as np
import pytest

import ttn_inputs as ti
from oracle import ttn as oracle

pytestmark = pytest.mark.gpu


def test_paper_torus_16x5_leftmost_density_matrices_and_entanglement():
    from paper_1905_01331_gb300 import Sweeper
    m = ti.tfim_torus(16, 5, 2.9)
    ws, V = ti.initial_tensors(16, m.d0, 32, 5)
    s = Sweeper(m, 32)
    s.set_isometries(0, ws, V)
    E = s.sweep(20)[:, 0]
    assert np.all(np.diff(E) <= 1e-9 * np.abs(E[1:]))          # monotone (variational steps)
    ws2, V2 = s.get_isometries(0)
    st = oracle.make_state(m, ws2, V2)
    e = s.energy(0)
    assert abs(e - oracle.energy(st)) < 1e-12 * abs(e)
    T = len(ws2)
    for t in range(T + 1):
        r = s.rdm(0, t, which=1)
        ref = oracle.rdm(st, t, which=1)
        assert np.abs(r - ref).max() < 1e-12, t
        lam, S = oracle.entanglement(r)
        lam_ref, S_ref = oracle.entanglement(ref)
        k = min(len(lam), len(lam_ref), 30)
        big = lam_ref[:k] < 30          # eigenvalues above 1e-9: resolved spectrum
        assert np.abs(lam[:k][big] - lam_ref[:k][big]).max() < 1e-8
        assert abs(S - S_ref) < 1e-10
    print("16x5 torus, chi 32, 20 sweeps: energy per spin", e / m.n_spins)
    s.close()
