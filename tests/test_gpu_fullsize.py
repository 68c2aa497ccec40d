"""Parity at the workloads' full sizes, through the C ABI in the launch
configuration the benchmark uses (graph-captured sweeps).

Oracle values at these sizes are stored trajectories written by
oracle/make_golden.py (energies of every sweep from the seeded start); the
FP64 GPU path must reproduce them to 1e-10 relative.  The batched workload is
checked on sampled instances against the oracle's first sweep.
"""
import json
import os

import numpy as np
import pytest

import ttn_inputs as ti
from oracle import ttn as oracle

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    with open(os.path.join(GOLDEN, f"oracle_{name}.json")) as f:
        return json.load(f)


def _trajectory(wl, n, prec="fp64"):
    from paper_1905_01331_gb300 import Sweeper
    ws, V = ti.initial_tensors(wl.model.Lx, wl.model.d0, wl.chi, wl.seed, wl.per_node)
    s = Sweeper(wl.model, wl.chi, per_node=wl.per_node, prec=prec)
    s.set_isometries(0, ws, V)
    E = s.sweep(n)[:, 0]
    Ef = s.energy(0)
    s.close()
    return E, Ef


@pytest.mark.parametrize("chi", [32, 128])
def test_tfim_l1024_fp64_trajectory(chi):
    g = _golden(f"tfim_L1024_chi{chi}")
    E, Ef = _trajectory(ti.tfim_l1024(chi), g["sweeps"])
    rel = np.abs(E - np.array(g["energies"])) / np.abs(np.array(g["energies"]))
    print("chi", chi, "max rel deviation over", g["sweeps"], "sweeps:", rel.max())
    assert rel.max() < 1e-10
    assert abs(Ef - g["final_energy"]) < 1e-10 * abs(g["final_energy"])


def test_heisenberg_l256_chi256_fp64_trajectory():
    g = _golden("heisenberg_L256_chi256")
    E, Ef = _trajectory(ti.heisenberg_l256(256), g["sweeps"])
    rel = np.abs(E - np.array(g["energies"])) / np.abs(np.array(g["energies"]))
    print("heisenberg chi=256 rel deviation", rel)
    assert rel.max() < 1e-10
    assert abs(Ef - g["final_energy"]) < 1e-10 * abs(g["final_energy"])


def test_torus_64x4_chi128_fp64_trajectory():
    g = _golden("torus_64x4_chi128")
    E, Ef = _trajectory(ti.torus_64x4(128), g["sweeps"])
    rel = np.abs(E - np.array(g["energies"])) / np.abs(np.array(g["energies"]))
    print("torus chi=128 max rel deviation", rel.max())
    assert rel.max() < 1e-10
    assert abs(Ef - g["final_energy"]) < 1e-10 * abs(g["final_energy"])


def test_batched_64_chains_sampled():
    """All 64 instances advance together; sampled small instances match the
    oracle's first sweep, and every energy is finite and above the closed form."""
    from oracle import ed
    from paper_1905_01331_gb300 import Sweeper
    wls = ti.batched_chains()
    s = Sweeper([w.model for w in wls], [w.chi for w in wls])
    inits = []
    for i, w in enumerate(wls):
        ws, V = ti.initial_tensors(w.model.Lx, 2, w.chi, w.seed)
        s.set_isometries(i, ws, V)
        inits.append((ws, V))
    E = s.sweep(1)[0]
    assert np.all(np.isfinite(E))
    for i, w in enumerate(wls):
        assert E[i] >= ed.tfim_closed_form(w.model.Lx, w.model.params["h"]) - 1e-9
    small = [i for i, w in enumerate(wls) if w.model.Lx <= 128 and w.chi <= 64][:3]
    for i in small:
        st = oracle.make_state(wls[i].model, *inits[i])
        E_ref = oracle.sweep(st)
        assert abs(E[i] - E_ref) < 1e-10 * abs(E_ref), (i, E[i], E_ref)
    s.close()
