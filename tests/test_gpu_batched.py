"""Many independent Hamiltonians (different couplings, L and chi) advanced
together in one context: every instance equals its own single-instance run
bit for bit, and the first sweep of each equals the oracle's."""
import numpy as np
import pytest

import ttn_inputs as ti
from oracle import ttn as oracle

pytestmark = pytest.mark.gpu


def test_batched_instances_match_single_runs_and_oracle():
    from paper_1905_01331_gb300 import Sweeper
    wls = ti.batched_chains(count=5, seed=4, sweeps=3)
    wls = [w for w in wls if w.model.Lx <= 256 and w.chi <= 64][:3] or wls[:2]
    models = [w.model for w in wls]
    chis = [w.chi for w in wls]
    multi = Sweeper(models, chis)
    inits = []
    for i, w in enumerate(wls):
        ws, V = ti.initial_tensors(w.model.Lx, 2, w.chi, w.seed)
        multi.set_isometries(i, ws, V)
        inits.append((ws, V))
    E_multi = multi.sweep(3)
    for i, w in enumerate(wls):
        one = Sweeper(w.model, w.chi)
        one.set_isometries(0, *inits[i])
        E_one = one.sweep(3)[:, 0]
        assert np.array_equal(E_multi[:, i], E_one)
        one.close()
        st = oracle.make_state(w.model, *inits[i])
        E_ref = oracle.sweep(st)
        assert abs(E_multi[0, i] - E_ref) < 1e-10 * abs(E_ref)
    multi.close()
