"""The MD options on the device: Nose-Hoover NVT against the oracle's NVT
integrator (trajectory, thermostat state and extended-energy conservation),
and the Verlet skin against rebuilding every step (same trajectory, fewer
builds, the refreshed edge set equal to a full build's)."""

import dataclasses

import numpy as np
import pytest

import oracle
from synth import make_workload, maxwell_boltzmann, normal_weights
from gpu_common import get_model

pytestmark = pytest.mark.gpu

MASSES = np.array([14.0067, 15.999, 28.0855])


def _tiny(scale):
    import paper_2402_03789_gb300 as sn
    s, spec = make_workload("sio2_192")
    spec = dataclasses.replace(spec, scale=scale)
    w = normal_weights(oracle.n_params(spec))
    return sn, s, spec, w, sn.SevenNet(spec, w)


def test_nose_hoover_tracks_oracle():
    sn, s, spec, w, model = _tiny(200.0)
    m = s.masses()
    v = maxwell_boltzmann(m, 1000.0, seed=3)
    md = sn.MD(model, s.pos, v, s.species, MASSES, s.cell, "fp32")
    md.set_nose_hoover(3000.0, 10.0)
    ep, ek = md.step(10, 1.0)
    p, vv, _ = md.state()
    xi, eta = md.nose_hoover()
    po, vo, _, xio, etao, epo, eko, exo = oracle.nose_hoover_nvt(spec, w, s.species, s.pos, v, m, s.cell,
                                                                1.0, 10, 3000.0, 10.0)
    assert abs(xio) > 1e-3                         # the thermostat is working
    # FP32-path tolerances (as for NVE), energies on the x200 scale of this model
    assert np.abs(p - po).max() < 1e-6
    assert np.abs(vv - vo).max() < 1e-7
    assert abs(xi - xio) < 1e-6 * abs(xio) + 1e-9
    assert abs(eta - etao) < 1e-6 * abs(etao) + 1e-9
    assert np.abs(ek - eko).max() / s.n_atoms < 1e-6 * spec.scale
    assert np.abs(ep - epo).max() / s.n_atoms < 1e-6 * spec.scale
    md.close()
    model.close()


def test_nose_hoover_ramp_tracks_oracle():
    # a melt-quench-style schedule: a 6-step ramp split over two md_step calls,
    # then a hold at its end value; trajectory and thermostat against the oracle
    sn, s, spec, w, model = _tiny(200.0)
    m = s.masses()
    v = maxwell_boltzmann(m, 1500.0, seed=7)
    md = sn.MD(model, s.pos, v, s.species, MASSES, s.cell, "fp32")
    md.set_nose_hoover_ramp(3000.0, 600.0, 6, 10.0)
    ep1, ek1 = md.step(4, 1.0)
    ep2, ek2 = md.step(6, 1.0)                     # 2 ramp steps, then 4 at 600 K
    ep, ek = np.concatenate([ep1, ep2]), np.concatenate([ek1, ek2])
    p, vv, _ = md.state()
    xi, eta = md.nose_hoover()
    po, vo, _, xio, etao, epo, eko, _ = oracle.nose_hoover_nvt(spec, w, s.species, s.pos, v, m, s.cell, 1.0, 10,
                                                               3000.0, 10.0, t_end_k=600.0, ramp_steps=6)
    assert abs(xio) > 1e-3
    assert np.abs(p - po).max() < 1e-6
    assert np.abs(vv - vo).max() < 1e-7
    assert abs(xi - xio) < 1e-6 * abs(xio) + 1e-9
    assert abs(eta - etao) < 1e-6 * abs(etao) + 1e-9
    assert np.abs(ek - eko).max() / s.n_atoms < 1e-6 * spec.scale
    assert np.abs(ep - epo).max() / s.n_atoms < 1e-6 * spec.scale
    # the schedule helper runs the same sequence
    md2 = sn.MD(model, s.pos, v, s.species, MASSES, s.cell, "fp32")
    ep3, ek3 = md2.run_schedule([("ramp", 3000.0, 600.0, 6), ("hold", 600.0, 4)], 1.0, 10.0)
    assert ep3.shape == (10,)
    assert np.abs(md2.state()[0] - po).max() < 1e-6
    with pytest.raises(sn.SevenNetError):
        md2.set_nose_hoover_ramp(3000.0, 600.0, 0, 10.0)
    md.close()
    md2.close()
    model.close()


def test_nose_hoover_heats_and_conserves_extended_energy():
    sn, s, spec, w, model = _tiny(1.0)
    m = s.masses()
    n = s.n_atoms
    v = maxwell_boltzmann(m, 300.0, seed=4)
    md = sn.MD(model, s.pos, v, s.species, MASSES, s.cell, "fp32")
    t0k, tau = 3000.0, 20.0
    md.set_nose_hoover(t0k, tau)
    E0, _, _ = model.evaluate(s.pos, s.cell, s.species, "fp32")
    ex0 = E0 + oracle.kinetic_energy(v, m)
    ep, ek = md.step(200, 1.0)
    xi, eta = md.nose_hoover()
    nf, kt0 = 3 * n - 3, oracle.md.KB * t0k
    q = oracle.nose_hoover_q(n, t0k, tau)
    ex = ep[-1] + ek[-1] + 0.5 * q * xi * xi + nf * kt0 * eta
    temps = 2 * ek / (nf * oracle.md.KB)
    assert temps.max() > 2000.0                    # driven from 300 K towards 3000 K
    assert abs(ex - ex0) / n < 1e-5, (ex, ex0)     # the extended energy is conserved
    md.close()
    model.close()


def test_skin_matches_rebuild_every_step():
    import paper_2402_03789_gb300 as sn
    s, spec = make_workload("sio2_192_l2")
    model = get_model(spec)
    m = s.masses()
    v = maxwell_boltzmann(m, 3000.0, seed=5)
    a = sn.MD(model, s.pos, v, s.species, MASSES, s.cell, "fp32")
    b = sn.MD(model, s.pos, v, s.species, MASSES, s.cell, "fp32")
    b.set_skin(0.5)
    epa, eka = a.step(40, 1.0)
    epb, ekb = b.step(40, 1.0)
    pa, va, fa = a.state()
    pb, vb, fb = b.state()
    builds, n_edges = b.stats()
    # atoms move ~0.5 A in 40 fs at 3000 K: the list is rebuilt a few times, not every step
    assert 2 <= builds < 20, builds
    assert np.abs(pa - pb).max() < 1e-8
    assert np.abs(fa - fb).max() < 1e-5 * np.sqrt((fa ** 2).mean()) + 1e-9
    assert np.abs(epa - epb).max() / s.n_atoms < 1e-7
    # the refreshed list has exactly the edges of a full build at the final positions
    dst, src, shift = model.neighbors(pb, s.cell)
    assert n_edges == len(dst)
    a.close()
    b.close()


def test_skin_across_calls_matches_rebuild_every_step():
    # each md_step call sizes the edge capacity from the last count and grows it
    # when the count rose, which reallocates the stored Verlet list: the next step
    # must then build a new list rather than filter the old arrays
    import paper_2402_03789_gb300 as sn
    s, spec = make_workload("sio2_192_l2")
    model = get_model(spec)
    m = s.masses()
    v = maxwell_boltzmann(m, 3000.0, seed=5)
    a = sn.MD(model, s.pos, v, s.species, MASSES, s.cell, "fp32")
    b = sn.MD(model, s.pos, v, s.species, MASSES, s.cell, "fp32")
    b.set_skin(0.5)
    a.step(40, 1.0)
    counts = [b.stats()[1]]
    for _ in range(8):
        b.step(5, 1.0)
        counts.append(b.stats()[1])
    # a count above all earlier ones before the last call: the next call grew the capacity
    assert any(counts[k] > max(counts[:k]) for k in range(1, 8)), counts
    pa, va, fa = a.state()
    pb, vb, fb = b.state()
    assert np.abs(pa - pb).max() < 1e-8
    assert np.abs(fa - fb).max() < 1e-5 * np.sqrt((fa ** 2).mean()) + 1e-9
    a.close()
    b.close()


def test_skin_rejects_negative():
    import paper_2402_03789_gb300 as sn
    s, spec = make_workload("sio2_192_l2")
    model = get_model(spec)
    m = s.masses()
    md = sn.MD(model, s.pos, maxwell_boltzmann(m, 300.0, seed=5), s.species, MASSES, s.cell, "fp32")
    with pytest.raises(sn.SevenNetError):
        md.set_skin(-0.1)
    with pytest.raises(sn.SevenNetError):
        md.set_nose_hoover(-5.0, 10.0)
    md.close()
