"""Pins of the oracle potential: parameter count (Sec. 5.1), invariances,
zero net force, finite differences of energy (Eq. 2 and the strain
derivative), extensivity, closed-form messages on one edge (Eq. 3),
the linear layout, and continuity at the cutoff."""

import dataclasses
import json
import math
import os

import numpy as np
import pytest
import torch
from scipy.spatial.transform import Rotation

import oracle
from oracle.model import (ModelLayout, layer_specs, conv_layer, edge_features,
                          radial_mlp, _lin)
from synth import (MODEL_SEVENNET0, MODEL_SEVENNET0_89, MODEL_TINY, make_workload,
                   normal_weights, random_structure, Structure)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def efv(spec, w, s, pos=None, cell=None):
    return oracle.energy_forces_virial(spec, w, s.species,
                                       s.pos if pos is None else pos,
                                       s.cell if cell is None else cell)


def test_parameter_count_matches_paper():
    ref = json.load(open(os.path.join(GOLDEN, "sevennet0_param_count.json")))
    n = oracle.n_params(MODEL_SEVENNET0_89)
    assert round(n / 1e6, 2) == ref["paper_value_millions"]
    assert n == ref["derived_exact_under_readings"]


def test_path_sets():
    L = layer_specs(MODEL_SEVENNET0)
    assert len(L[0].paths) == 3 and sum(L[0].path_mul) == 384
    assert len(L[1].paths) == 15 and sum(L[1].path_mul) == 960
    assert L[1].msg_muls == {0: 224, 1: 384, 2: 352}
    assert L[4].paths == [(0, 0, 0), (1, 1, 0), (2, 2, 0)] and sum(L[4].path_mul) == 224
    T = layer_specs(MODEL_TINY)
    assert [sum(x.path_mul) for x in T] == [64, 160, 64]


def test_invariances_and_net_force(tiny_case):
    s, spec, w = tiny_case
    E, F, W, ea, _ = efv(spec, w, s)
    assert abs(F.sum(0)).max() < 1e-14 * max(1.0, abs(F).max() * len(F))
    assert np.abs(W - W.T).max() < 1e-12 * np.abs(W).max()
    R = Rotation.random(random_state=5).as_matrix()
    E2, F2, W2, *_ = efv(spec, w, s, pos=s.pos @ R.T, cell=s.cell @ R.T)
    assert abs(E2 - E) < 1e-11 * abs(E)
    assert np.abs(F2 - F @ R.T).max() < 1e-11
    assert np.abs(W2 - R @ W @ R.T).max() < 1e-11
    E3, F3, *_ = efv(spec, w, s, pos=s.pos + np.array([0.3, -1.7, 2.2]))
    assert abs(E3 - E) < 1e-11 * abs(E) and np.abs(F3 - F).max() < 1e-12
    perm = np.random.default_rng(1).permutation(s.n_atoms)
    sp = Structure(pos=s.pos[perm], species=s.species[perm], cell=s.cell)
    E4, F4, *_ = efv(spec, w, sp)
    assert abs(E4 - E) < 1e-11 * abs(E) and np.abs(F4 - F[perm]).max() < 1e-12


def test_forces_equal_central_differences(tiny_case):
    s, spec, w = tiny_case
    E, F, *_ = efv(spec, w, s)
    h = 1e-4
    scale = np.abs(F).max()
    for (i, a) in [(0, 0), (17, 1), (101, 2), (191, 0)]:
        p = s.pos.copy(); p[i, a] += h
        Ep = efv(spec, w, s, pos=p)[0]
        p[i, a] -= 2 * h
        Em = efv(spec, w, s, pos=p)[0]
        fd = -(Ep - Em) / (2 * h)
        assert abs(fd - F[i, a]) <= 1e-6 * scale, (i, a, fd, F[i, a])


def test_virial_equals_strain_differences(tiny_case):
    s, spec, w = tiny_case
    E, F, W, *_ = efv(spec, w, s)
    h = 1e-5
    for (a, b) in [(0, 0), (1, 2), (2, 1), (0, 2)]:
        vals = []
        for sgn in (+1, -1):
            eps = np.zeros((3, 3)); eps[a, b] = sgn * h
            M = np.eye(3) + eps
            vals.append(efv(spec, w, s, pos=s.pos @ M.T, cell=s.cell @ M.T)[0])
        fd = -(vals[0] - vals[1]) / (2 * h)
        assert abs(fd - W[a, b]) <= 1e-6 * np.abs(W).max(), (a, b, fd, W[a, b])


def test_extensivity_supercell(tiny_case):
    s, spec, w = tiny_case
    E = efv(spec, w, s)[0]
    shifts = np.array([(i, j, k) for i in range(2) for j in range(2) for k in range(2)])
    pos2 = np.concatenate([s.pos + sh @ s.cell for sh in shifts])
    sp2 = np.concatenate([s.species] * 8)
    E2 = oracle.energy_forces_virial(spec, w, sp2, pos2, 2 * s.cell)[0]
    assert abs(E2 - 8 * E) < 1e-10 * abs(E2)


def _one_edge_setup(spec, t):
    layout = ModelLayout(spec)
    Wd = layout.unpack(normal_weights(layout.size))
    L = layer_specs(spec)[t]
    pos = torch.tensor([[0.0, 0.0, 0.0], [1.3, 0.4, -0.9]], dtype=torch.float64)
    dst = torch.tensor([0, 1]); src = torch.tensor([1, 0])
    d = pos[src] - pos[dst]
    Y, B = edge_features(spec, d)
    w = radial_mlp(spec, Wd, t, B)
    g = torch.Generator().manual_seed(3)
    x = {l: torch.randn((2, 2 * l + 1, mu), generator=g, dtype=torch.float64)
         for l, mu in L.in_muls.items()}
    return L, x, Y, w, dst, src


def _closed_form_messages(spec, L, x, Y, w, recv, send, edge):
    """Explicit m for the paths whose CG is identity, dot or cross product."""
    a = spec.avg_num_neigh
    out = {}
    col = 0
    perm = [1, 2, 0]
    inv = [2, 0, 1]
    for (l1, l2, l3), mu in zip(L.paths, L.path_mul):
        we = w[edge, col:col + mu]
        xs = x[l1][send]
        if l1 == 0 and l2 == l3:
            out[(l1, l2, l3)] = xs[0][None, :] * Y[l2][edge][:, None] * we / a
        elif l2 == 0 and l1 == l3:
            out[(l1, l2, l3)] = xs * we / a
        elif (l1, l2, l3) == (1, 1, 0):
            out[(l1, l2, l3)] = ((xs * Y[1][edge][:, None]).sum(0) / math.sqrt(3) * we)[None] / a
        elif (l1, l2, l3) == (1, 1, 1):
            xv = xs[inv].T                             # [mu, 3] as (x, y, z)
            yv = Y[1][edge][inv]
            cr = torch.linalg.cross(xv, yv.expand_as(xv))[:, perm].T
            out[(l1, l2, l3)] = cr / math.sqrt(2) * we / a
        col += mu
    return out


@pytest.mark.parametrize("t", [0, 1, 4])
def test_one_edge_messages_closed_form(t):
    spec = MODEL_SEVENNET0
    L, x, Y, w, dst, src = _one_edge_setup(spec, t)
    m = conv_layer(spec, L, x, Y, w, dst, src, 2)
    ref = _closed_form_messages(spec, L, x, Y, w, recv=0, send=1, edge=0)
    offs = {}
    checked = 0
    for p, mu in zip(L.paths, L.path_mul):
        o = offs.get(p[2], 0)
        offs[p[2]] = o + mu
        if p in ref:
            assert torch.allclose(m[p[2]][0, :, o:o + mu], ref[p], atol=1e-13), p
            checked += 1
    assert checked >= 2


def test_planted_gather_mistake_is_caught():
    spec = MODEL_SEVENNET0
    L, x, Y, w, dst, src = _one_edge_setup(spec, 1)
    bad = conv_layer(spec, L, x, Y, w, dst, dst, 2)      # gathers the receiver
    ref = _closed_form_messages(spec, L, x, Y, w, recv=0, send=1, edge=0)
    o = L.path_mul[0]
    p = L.paths[1]
    assert not torch.allclose(bad[p[2]][0, :, :L.path_mul[1]], ref[p], atol=1e-6)


def test_linear_layout_row_is_input_channel():
    W = torch.zeros((4, 3), dtype=torch.float64)
    W[2, 1] = 1.0
    x = torch.zeros((1, 3, 4), dtype=torch.float64)
    x[0, :, 2] = torch.tensor([1.0, 2.0, 3.0])
    y = _lin(x, W)
    assert torch.allclose(y[0, :, 1], torch.tensor([1.0, 2.0, 3.0], dtype=torch.float64) / 2.0)
    assert float(y[0, :, 0].abs().sum()) == 0.0


def test_energy_continuous_at_cutoff():
    spec = MODEL_TINY
    w = normal_weights(oracle.n_params(spec))
    cell = np.eye(3) * 30.0
    far = oracle.energy_forces_virial(spec, w, np.array([2, 1]),
                                      np.array([[0, 0, 0], [9.0, 0, 0]]), cell)[0]
    diffs = []
    for dlt in (1e-2, 1e-3):
        e = oracle.energy_forces_virial(spec, w, np.array([2, 1]),
                                        np.array([[0, 0, 0], [spec.r_cut - dlt, 0, 0]]), cell)[0]
        diffs.append(abs(e - far))
    assert diffs[1] < 1e-9 and diffs[0] > 0
    assert diffs[1] < diffs[0] * 1e-2


def test_five_layer_model_gradients_and_rotation():
    s, spec = make_workload("sio2_192_l2")
    w = normal_weights(oracle.n_params(spec))
    E, F, W, *_ = efv(spec, w, s)
    assert abs(F.sum(0)).max() < 1e-14 * max(1.0, abs(F).max() * len(F))
    R = Rotation.random(random_state=8).as_matrix()
    E2, F2, *_ = efv(spec, w, s, pos=s.pos @ R.T, cell=s.cell @ R.T)
    assert abs(E2 - E) < 1e-11 * abs(E) and np.abs(F2 - F @ R.T).max() < 1e-12
    h = 1e-4
    i, a = 42, 1
    p = s.pos.copy(); p[i, a] += h
    Ep = efv(spec, w, s, pos=p)[0]
    p[i, a] -= 2 * h
    Em = efv(spec, w, s, pos=p)[0]
    assert abs(-(Ep - Em) / (2 * h) - F[i, a]) <= 1e-6 * np.abs(F).max()


def test_lmax3_model_invariances_and_forces():
    # the paper's benchmark models have lmax 3 (Sec. 4): rotation and translation
    # invariance, zero net force and central differences of the forces
    from synth import benchmark_model, make_quartz
    spec = benchmark_model(2, 32, lmax=3)
    s = make_quartz("quartz_216")
    w = normal_weights(oracle.n_params(spec))
    E, F, W, *_ = efv(spec, w, s)
    R = Rotation.random(random_state=3).as_matrix()
    E2, F2, *_ = efv(spec, w, s, pos=s.pos @ R.T, cell=s.cell @ R.T)
    assert abs(E2 - E) < 1e-10 * max(1.0, abs(E))
    assert np.abs(F2 - F @ R.T).max() < 1e-10
    assert np.abs(F.sum(0)).max() < 1e-10
    h = 1e-4
    for i, a in ((3, 0), (50, 2)):
        p = s.pos.copy(); p[i, a] += h
        Ep = efv(spec, w, s, pos=p)[0]
        p[i, a] -= 2 * h
        Em = efv(spec, w, s, pos=p)[0]
        fd = -(Ep - Em) / (2 * h)
        assert abs(fd - F[i, a]) <= 1e-6 * max(1.0, abs(F[i, a])) + 1e-9, (fd, F[i, a])
