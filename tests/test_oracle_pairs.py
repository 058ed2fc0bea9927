"""Pins of the identities behind the adjoint over unordered edge pairs.

The GPU adjoint handles an edge e (receiver v, sender w, displacement d) and its
reverse (receiver w, sender v, -d) together.  It relies on four facts, each
checked here on the oracle's FP64 functions, with the plausible mistake planted
to show that the check catches it:
- forces and the virial depend on the edge gradients only through
  dE/dd_e - dE/dd_rev(e) (Eqs. 5-7), so the pair's whole gradient may sit on e;
- Y_l(-d) = (-1)^l Y_l(d) for the real harmonics, so the reverse edge's G matrix
  of path (l1, l2, l3) is (-1)^l2 times that of e;
- the radial basis, hence the radial weights, depend on |d| only;
- through the tensor product (Eq. 3), the reverse direction's share of dE/dw and
  of dE/dY(d) is that of a message with dE/dm of w taken times (-1)^l2.
"""

import numpy as np
import pytest
import torch

import oracle
from oracle.model import ModelLayout, conv_layer, edge_features, layer_specs, model_energy
from oracle.neighbors import neighbor_list
from oracle.so3 import real_cg, real_sh
from synth import MODEL_TINY, normal_weights, random_structure


def _reverse_index(dst, src, shift):
    key = {(int(v), int(w), tuple(int(c) for c in s)): i for i, (v, w, s) in enumerate(zip(dst, src, shift))}
    return np.array([key[(int(w), int(v), tuple(-int(c) for c in s))] for v, w, s in zip(dst, src, shift)])


def _edge_gradients(spec, s, weights):
    """dE/dd of every edge by autograd through the oracle model, with the edges."""
    Wd = ModelLayout(spec).unpack(weights)
    dst, src, shift = neighbor_list(s.pos, s.cell, spec.r_cut)
    d = torch.tensor(s.pos[src] - s.pos[dst] + shift @ s.cell, requires_grad=True)
    E = model_energy(spec, Wd, s.species, d, torch.as_tensor(dst, dtype=torch.long),
                     torch.as_tensor(src, dtype=torch.long), s.n_atoms).sum()
    (g,) = torch.autograd.grad(E, d)
    return dst, src, shift, d.detach().numpy(), g.numpy()


def _forces_virial(n, dst, rev, d, g):
    """F_v = sum over edges into v of (g_e - g_rev(e)) (Eq. 6), W_ab = -sum_e g_a d_b."""
    F = np.zeros((n, 3))
    np.add.at(F, dst, g - g[rev])
    return F, -(g.T @ d)


@pytest.fixture(scope="module")
def small_cell():
    spec = MODEL_TINY
    s = random_structure({"Si": 4, "O": 8}, 2.2, 1.6, seed=41)
    w = normal_weights(oracle.n_params(spec))
    E, F, W, *_ = oracle.energy_forces_virial(spec, w, s.species, s.pos, s.cell)
    dst, src, shift, d, g = _edge_gradients(spec, s, w)
    return s, dst, _reverse_index(dst, src, shift), d, g, F, W


def test_edge_gradients_give_the_oracle_forces_and_virial(small_cell):
    s, dst, rev, d, g, F, W = small_cell
    F1, W1 = _forces_virial(s.n_atoms, dst, rev, d, g)
    assert np.allclose(F1, F, rtol=0, atol=1e-10 * np.abs(F).max())
    assert np.allclose(W1, W, rtol=0, atol=1e-10 * np.abs(W).max())


def test_pair_gradient_on_one_edge_keeps_forces_and_virial(small_cell):
    s, dst, rev, d, g, F, W = small_cell
    canon = np.arange(len(dst)) < rev
    assert canon.sum() * 2 == len(dst) and np.all(rev[rev] == np.arange(len(dst)))
    assert np.allclose(d[rev], -d, rtol=0, atol=1e-12)
    g2 = np.zeros_like(g)
    g2[canon] = g[canon] - g[rev[canon]]
    F2, W2 = _forces_virial(s.n_atoms, dst, rev, d, g2)
    assert np.allclose(F2, F, rtol=0, atol=1e-10 * np.abs(F).max())
    assert np.allclose(W2, W, rtol=0, atol=1e-10 * np.abs(W).max())
    # planted: the reverse's gradient added instead of subtracted
    g3 = np.zeros_like(g)
    g3[canon] = g[canon] + g[rev[canon]]
    F3, _ = _forces_virial(s.n_atoms, dst, rev, d, g3)
    assert not np.allclose(F3, F, rtol=0, atol=1e-6 * np.abs(F).max())


def _couplings(lmax):
    return [(l1, l2, l3) for l1 in range(lmax + 1) for l2 in range(lmax + 1)
            for l3 in range(abs(l1 - l2), min(l1 + l2, lmax) + 1)]


def test_reverse_edge_g_matrix_sign():
    gen = torch.Generator().manual_seed(3)
    d = torch.randn((5, 3), generator=gen, dtype=torch.float64)
    Yp, Ym = real_sh(3, d), real_sh(3, -d)
    for l in range(4):
        assert torch.allclose(Ym[l], (-1) ** l * Yp[l], rtol=0, atol=1e-14)
    wrong = 0
    for l1, l2, l3 in _couplings(3):
        C = torch.as_tensor(real_cg(l1, l2, l3))
        Gp = torch.einsum("abc,eb->eac", C, Yp[l2])
        Gm = torch.einsum("abc,eb->eac", C, Ym[l2])
        assert torch.allclose(Gm, (-1) ** l2 * Gp, rtol=0, atol=1e-13)
        # planted: the sign taken from l3 (or l1) instead of l2
        wrong += not torch.allclose(Gm, (-1) ** l3 * Gp, rtol=0, atol=1e-13)
    assert wrong > 0


def test_radial_basis_depends_on_length_only():
    gen = torch.Generator().manual_seed(5)
    d = 1.0 + 3.0 * torch.rand((7, 3), generator=gen, dtype=torch.float64)
    _, Bp = edge_features(MODEL_TINY, d)
    _, Bm = edge_features(MODEL_TINY, -d)
    assert torch.equal(Bp, Bm)


def _pair_adjoint(spec, L, x, gm, w, Yd, v, wv, sign_b):
    """dE/dw, dE/dY(d) and dE/dx of E = <gm, m> for the two directed edges of one
    pair, by the pair formulas: direction a is e (receiver v, sender wv, Y(d)),
    direction b its reverse, with dE/dm of wv times sign_b(l2)."""
    dw, gY = [], {l: torch.zeros_like(y) for l, y in enumerate(Yd)}
    gx = {l: torch.zeros_like(t) for l, t in x.items()}
    m_off = {}
    for (l1, l2, l3), mu in zip(L.paths, L.path_mul):
        C = torch.as_tensor(real_cg(l1, l2, l3))
        G = torch.einsum("abc,b->ac", C, Yd[l2])                     # [N1, N3]
        o = m_off.get(l3, 0)
        m_off[l3] = o + mu
        ga = gm[l3][v, :, o:o + mu] / spec.avg_num_neigh              # [N3, mu]
        gb = sign_b(l2) * gm[l3][wv, :, o:o + mu] / spec.avg_num_neigh
        col = sum(len(dw_i) for dw_i in dw)
        ww = w[col:col + mu]
        xa, xb = x[l1][wv], x[l1][v]                                   # senders of a and b, [N1, mu]
        qa, qb = G @ ga, G @ gb                                        # [N1, mu]
        dw.append((xa * qa).sum(0) + (xb * qb).sum(0))
        gx[l1][wv] += ww * qa
        gx[l1][v] += ww * qb
        gY[l2] += torch.einsum("abc,au,cu->b", C, ww * xa, ga) + torch.einsum("abc,au,cu->b", C, ww * xb, gb)
    return torch.cat(dw), gY, gx


@pytest.mark.parametrize("planted", [False, True])
def test_pair_adjoint_of_the_tensor_product(planted):
    spec = MODEL_TINY
    L = layer_specs(spec)[1]                                           # a middle block: l1, l2, l3 <= 1
    gen = torch.Generator().manual_seed(9)
    n, v, wv = 3, 0, 2
    x = {l: torch.randn((n, 2 * l + 1, mu), generator=gen, dtype=torch.float64, requires_grad=True)
         for l, mu in L.in_muls.items()}
    W = sum(L.path_mul)
    w = torch.randn(W, generator=gen, dtype=torch.float64, requires_grad=True)
    d = torch.tensor([1.1, -0.7, 2.3], dtype=torch.float64)
    Yd = [y[0].detach().clone().requires_grad_(True) for y in real_sh(spec.lmax, d[None])]
    # the two directed edges: e = (v <- wv, d) and its reverse (wv <- v, -d)
    Y = [torch.stack([Yd[l], (-1) ** l * Yd[l]]) for l in range(spec.lmax + 1)]
    dst = torch.tensor([v, wv])
    src = torch.tensor([wv, v])
    m = conv_layer(spec, L, x, Y, torch.stack([w, w]), dst, src, n)
    gm = {l: torch.randn(t.shape, generator=gen, dtype=torch.float64) for l, t in m.items()}
    E = sum((gm[l] * m[l]).sum() for l in m)
    g_w, *g_Y = torch.autograd.grad(E, [w] + Yd, retain_graph=True)
    g_x = torch.autograd.grad(E, [x[l] for l in sorted(x)])
    sign_b = (lambda l2: 1.0) if planted else (lambda l2: (-1.0) ** l2)
    dw, gY, gx = _pair_adjoint(spec, L, {l: t.detach() for l, t in x.items()}, gm, w.detach(),
                               [y.detach() for y in Yd], v, wv, sign_b)
    ok = torch.allclose(dw, g_w, rtol=1e-12, atol=1e-12) and all(
        torch.allclose(gY[l], g_Y[l], rtol=1e-12, atol=1e-12) for l in range(spec.lmax + 1)) and all(
        torch.allclose(gx[l], g, rtol=1e-12, atol=1e-12) for l, g in zip(sorted(x), g_x))
    assert ok != planted
