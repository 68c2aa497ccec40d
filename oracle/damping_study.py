"""Spread of the FP64 sweep between two LAPACK SVD drivers as a function of
the proximal weight mu of the update (test infrastructure: calls only the
oracle and the shared seeded inputs).

The update of Sec. III.B takes the polar factor (from an SVD) of the
environment.  When the environment is numerically rank deficient the SVD's
singular vectors are arbitrary on the null directions, so two correct FP64
implementations (LAPACK's divide-and-conquer gesdd and QR-iteration gesvd)
follow different trajectories.  The oracle therefore takes the polar factor of
Gamma - mu |Gamma|_F w_old; this script measures, for mu on a decade grid,
the largest relative difference of the per-sweep energies of the two drivers
from the same seeded start.  The oracle's mu is the smallest grid value at
which the two stay within the FP64 tolerance 1e-10 at every sweep of every
workload run.

    python -m oracle.damping_study [workload ...]    (c1, c2_32, c2_64)
"""
from __future__ import annotations

import json
import sys

import numpy as np
import scipy.linalg as sla

import ttn_inputs as ti
from oracle import ttn

MUS = (0.0, 1e-10, 1e-9, 1e-8, 1e-7)
WORKLOADS = {"c1": (ti.tfim_l16_pernode, 30), "c2_32": (lambda: ti.tfim_l1024(32), 200),
             "c2_64": (lambda: ti.tfim_l1024(64), 200)}


def update_with(mu, driver):
    """The oracle's update with weight mu and the given LAPACK SVD driver."""
    def upd(gamma, w_old, damping=None):
        P = gamma.shape[0]
        g = gamma.reshape(P, -1) - mu * np.linalg.norm(gamma) * w_old.reshape(P, -1)
        U, _, Vt = sla.svd(g, full_matrices=False, lapack_driver=driver)
        return -(U @ Vt).reshape(gamma.shape)
    return upd


def energies(wl, sweeps, mu, driver):
    saved = ttn.polar_update
    ttn.polar_update = update_with(mu, driver)
    try:
        ws, V = ti.initial_tensors(wl.model.Lx, wl.model.d0, wl.chi, wl.seed, wl.per_node)
        st = ttn.make_state(wl.model, ws, V, per_node=wl.per_node)
        return np.array([ttn.sweep(st) for _ in range(sweeps)])
    finally:
        ttn.polar_update = saved


def main(names):
    out = {}
    for nm in names:
        make, sweeps = WORKLOADS[nm]
        wl = make()
        for mu in MUS:
            a = energies(wl, sweeps, mu, "gesdd")
            b = energies(wl, sweeps, mu, "gesvd")
            spread = float(np.max(np.abs(a - b) / np.abs(a)))
            out[f"{nm} mu={mu:g}"] = {"final_energy_gesdd": float(a[-1]), "max_rel_spread": spread}
            print(nm, f"mu={mu:g}", "E_last %.10f" % a[-1], "max rel spread %.1e" % spread, flush=True)
    return out


if __name__ == "__main__":
    print(json.dumps(main(sys.argv[1:] or ["c1", "c2_32"]), indent=1))
