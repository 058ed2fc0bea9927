"""MD (velocity Verlet on the device) against the oracle integrator, NVE
drift on the 3,000-atom SiO2 cell, and the continuous-batching server:
results equal to single evaluations, batches formed and overlapping, and
admission by device-memory budget."""

import dataclasses
import time

import numpy as np
import pytest

import oracle
from synth import (MODEL_SEVENNET0, MODEL_TINY, make_workload, maxwell_boltzmann, normal_weights,
                   random_structure)
from gpu_common import get_model

pytestmark = pytest.mark.gpu


def test_md_tracks_oracle_trajectory():
    import paper_2402_03789_gb300 as sn
    s, spec = make_workload("sio2_192")
    spec = dataclasses.replace(spec, scale=200.0)
    w = normal_weights(oracle.n_params(spec))
    model = sn.SevenNet(spec, w)
    m = s.masses()
    v = maxwell_boltzmann(m, 3000.0, seed=3)
    masses = np.array([14.0067, 15.999, 28.0855])
    md = sn.MD(model, s.pos, v, s.species, masses, s.cell, "fp32")
    ep, ek = md.step(10, 1.0)
    p, vv, f = md.state()
    po, vo, fo, epo, eko = oracle.velocity_verlet(spec, w, s.species, s.pos, v, m, s.cell, 1.0, 10)
    # FP32-path tolerances; energies carry the x200 energy scale of this model
    assert np.abs(p - po).max() < 1e-6
    assert np.abs(vv - vo).max() < 1e-7
    assert np.abs(ep - epo).max() / s.n_atoms < 1e-6 * spec.scale
    assert np.abs(ek - eko).max() / s.n_atoms < 1e-6 * spec.scale
    md.close()
    model.close()


def test_md_nve_drift_sio2_3000():
    import paper_2402_03789_gb300 as sn
    s, spec = make_workload("sio2_3000")
    model = get_model(spec)
    m = s.masses()
    v = maxwell_boltzmann(m, 3000.0, seed=3)
    md = sn.MD(model, s.pos, v, s.species, np.array([14.0067, 15.999, 28.0855]), s.cell, "fp32")
    ep, ek = md.step(100, 1.0)
    E0, _, _ = model.evaluate(s.pos, s.cell, s.species)
    etot0 = E0 + oracle.kinetic_energy(v, m)
    drift = np.abs(ep + ek - etot0).max() / s.n_atoms
    print(f"NVE drift over 100 fs: {drift:.2e} eV/atom")
    assert drift < 1e-5
    md.close()


def test_server_results_equal_single_evaluations():
    import paper_2402_03789_gb300 as sn
    spec = MODEL_SEVENNET0
    model = get_model(spec)
    rng = np.random.default_rng(5)
    structs = []
    for k in range(24):
        n = int(rng.integers(16, 300))
        el = rng.integers(0, 3, n)
        counts = {name: int((el == i).sum()) for i, name in enumerate(("N", "O", "Si")) if (el == i).sum()}
        structs.append(random_structure(counts, float(rng.uniform(2.2, 3.1)), 1.5, seed=100 + k))
    srv = sn.Server(model, hbm_budget_bytes=2 << 30, n_streams=3, max_batch_structs=8, precision="fp32")
    tickets = []
    # a burst (queued faster than one evaluation takes, so later batches carry
    # several structures), then arrivals spread out while batches are running
    for i, s in enumerate(structs):
        tickets.append(srv.submit(s.pos, s.cell, s.species))
        if i >= 16:
            time.sleep(0.002)
    results = {}
    t0 = time.time()
    while len(results) < len(tickets) and time.time() - t0 < 120:
        for t in tickets:
            if t not in results:
                r = srv.poll(t)
                if r is not None:
                    results[t] = r
        time.sleep(0.001)
    assert len(results) == len(tickets)
    # each result equals its evaluation alone bit for bit: in FP32 every sum of a
    # structure has a fixed order whatever batch it runs in
    for t, s in zip(tickets, structs):
        E, F, W = model.evaluate(s.pos, s.cell, s.species, "fp32")
        r = results[t]
        assert r["energy"] == E and np.array_equal(r["forces"], F) and np.array_equal(r["virial"], W)
    batches = {}
    for r in results.values():
        batches.setdefault(r["batch_id"], (r["start_s"], r["done_s"], r["batch_structs"]))
    assert max(b[2] for b in batches.values()) > 1            # requests were batched
    spans = sorted((b[0], b[1]) for b in batches.values())
    overlap = any(spans[i + 1][0] < spans[i][1] for i in range(len(spans) - 1))
    assert overlap                                           # a batch launched while another ran
    srv.close()


def test_server_admission_refuses_oversized_request():
    import paper_2402_03789_gb300 as sn
    model = get_model(MODEL_SEVENNET0)
    srv = sn.Server(model, hbm_budget_bytes=1 << 20, n_streams=1, max_batch_structs=4)
    s = random_structure({"Si": 100, "O": 200}, 2.2, 1.6, seed=7)
    with pytest.raises(sn.SevenNetError) as ei:
        srv.submit(s.pos, s.cell, s.species)
    assert ei.value.status == -6
    srv.close()
