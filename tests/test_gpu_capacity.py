"""Edge capacity overflow and its retry.  The asynchronous neighbour build writes
into preallocated edge arrays (64 per atom at first) and reports on the device
when a structure needs more; the evaluation then runs again with the count the
device reported, and a serving batch reruns through the same path.  A dense
cell (about 95 neighbours per atom within 5 A) forces both."""

import time

import numpy as np
import pytest

import oracle
from synth import MODEL_SEVENNET0, normal_weights, random_structure
from gpu_common import errors

pytestmark = pytest.mark.gpu


def _dense():
    s = random_structure({"Si": 20, "O": 40}, 6.0, 1.0, seed=71)
    dst, _, _ = oracle.neighbor_list(s.pos, s.cell, MODEL_SEVENNET0.r_cut)
    assert len(dst) / s.n_atoms > 64          # beyond the first capacity
    return s


def test_dense_cell_is_retried_with_more_edge_room():
    import paper_2402_03789_gb300 as sn
    spec = MODEL_SEVENNET0
    w = normal_weights(oracle.n_params(spec))
    s = _dense()
    model = sn.SevenNet(spec, w)              # a fresh workspace
    E, F, W = model.evaluate(s.pos, s.cell, s.species, "fp32")
    Eo, Fo, Wo, *_ = oracle.energy_forces_virial(spec, w, s.species, s.pos, s.cell)
    e_pa, f_rel, w_rel = errors(E, F, W, Eo, Fo, Wo, s.n_atoms)
    assert e_pa <= 1e-6 and f_rel <= 1e-5 and w_rel <= 1e-5, (e_pa, f_rel, w_rel)
    model.close()


def test_server_reruns_a_batch_beyond_its_slot_capacity():
    import paper_2402_03789_gb300 as sn
    spec = MODEL_SEVENNET0
    w = normal_weights(oracle.n_params(spec))
    s = _dense()
    model = sn.SevenNet(spec, w)
    E, F, W = model.evaluate(s.pos, s.cell, s.species, "fp32")
    # a slot of 64 atoms (about 51 KB each for this model): its 4,096 edges are fewer than the cell needs
    srv = sn.Server(model, hbm_budget_bytes=3_300_000, n_streams=1, max_batch_structs=4, precision="fp32")
    t = srv.submit(s.pos, s.cell, s.species)
    r, t0 = None, time.time()
    while r is None and time.time() - t0 < 60:
        r = srv.poll(t)
        time.sleep(0.001)
    assert r is not None
    assert r["energy"] == E and np.array_equal(r["forces"], F) and np.array_equal(r["virial"], W)
    srv.close()
    model.close()
