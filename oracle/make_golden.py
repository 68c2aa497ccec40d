"""Write the oracle's reference energies to tests/golden/ (test infrastructure).

Calls only ``oracle`` and the shared seeded inputs.  Usage:
    python -m oracle.make_golden [name ...]
Each file records the workload, its seed, the bond shift and the energy found
by the top solve of every sweep, plus the energy of the final tensors.
"""
from __future__ import annotations

import json
import os
import sys
import time

import ttn_inputs as ti
from oracle import ttn

OUT = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "tests", "golden")


def workloads():
    return {
        "tfim_L16_chi8_pernode": (ti.tfim_l16_pernode(), None),
        "tfim_L1024_chi32": (ti.tfim_l1024(32), None),
        "tfim_L1024_chi64": (ti.tfim_l1024(64), None),
        "tfim_L1024_chi128": (ti.tfim_l1024(128), None),
        "torus_64x4_chi128": (ti.torus_64x4(128), 20),
        "heisenberg_L256_chi256": (ti.heisenberg_l256(256), 4),
    }


def run_one(name, wl, sweeps=None):
    n = wl.sweeps if sweeps is None else sweeps
    ws, V = ti.initial_tensors(wl.model.Lx, wl.model.d0, wl.chi, wl.seed, wl.per_node)
    st = ttn.make_state(wl.model, ws, V, per_node=wl.per_node)
    t0 = time.time()
    Es = []
    for i in range(n):
        Es.append(ttn.sweep(st))
        print(name, i, Es[-1], f"{time.time() - t0:.1f}s", flush=True)
    rec = {
        "workload": name, "model": wl.model.name, "params": wl.model.params,
        "Lx": wl.model.Lx, "Ly": wl.model.Ly, "chi": wl.chi, "seed": wl.seed,
        "per_node": wl.per_node, "sweeps": n, "polar_damping": ttn.POLAR_DAMPING,
        "shift": st.c, "energies": Es, "final_energy": ttn.energy(st),
        "n_spins": wl.model.n_spins,
        "source": "oracle/ttn.py (FP64, numpy/LAPACK), written by oracle/make_golden.py",
    }
    with open(os.path.join(OUT, f"oracle_{name}.json"), "w") as f:
        json.dump(rec, f, indent=0)


def run_batched_first_sweep(name="batched64_first_sweep"):
    """The 64 independent chains of the batched workload: for every instance,
    the energy found by the top solve of its first sweep from the seeded
    start, and the energy of its tensors after that sweep."""
    out = []
    t0 = time.time()
    for i, wl in enumerate(ti.batched_chains()):
        ws, V = ti.initial_tensors(wl.model.Lx, wl.model.d0, wl.chi, wl.seed)
        st = ttn.make_state(wl.model, ws, V)
        E1 = ttn.sweep(st)
        out.append({"instance": i, "L": wl.model.Lx, "chi": wl.chi, "h": wl.model.params["h"],
                    "seed": wl.seed, "shift": st.c, "first_sweep_energy": E1,
                    "energy_after_first_sweep": ttn.energy(st)})
        print(name, i, E1, f"{time.time() - t0:.1f}s", flush=True)
    rec = {"workload": name, "count": len(out), "polar_damping": ttn.POLAR_DAMPING,
           "instances": out,
           "source": "oracle/ttn.py (FP64, numpy/LAPACK), written by oracle/make_golden.py"}
    with open(os.path.join(OUT, f"oracle_{name}.json"), "w") as f:
        json.dump(rec, f, indent=0)


if __name__ == "__main__":
    wls = workloads()
    names = sys.argv[1:] or list(wls) + ["batched64_first_sweep"]
    for nm in names:
        if nm == "batched64_first_sweep":
            run_batched_first_sweep()
            continue
        wl, n = wls[nm]
        run_one(nm, wl, n)
