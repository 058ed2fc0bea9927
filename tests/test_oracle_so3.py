"""Pins of the oracle's spherical harmonics and Clebsch-Gordan tensors.

Independent checks: scipy's complex spherical harmonics (a library routine),
the addition theorem, rotation equivariance with D-matrices fitted from the
harmonics themselves, CG orthogonality, the closed-form special cases
(identity, dot product, cross product) and the Gaunt-type projection
Y_l1(u) (x) Y_l2(u) -> Y_l1+l2(u).
"""

import math

import numpy as np
import pytest
import torch
from scipy.spatial.transform import Rotation
from scipy.special import sph_harm_y

from oracle.so3 import real_sh, real_cg

PATHS = [(l1, l2, l3) for l1 in range(4) for l2 in range(4)
         for l3 in range(abs(l1 - l2), min(l1 + l2, 3) + 1)]


def _pts(n, seed):
    return np.random.default_rng(seed).normal(size=(n, 3))


def _fit_D(R):
    a, b = _pts(300, 11), _pts(300, 12)
    Ya = real_sh(3, torch.tensor(a))
    Yr = real_sh(3, torch.tensor(a @ R.T))
    Ds = []
    for l in range(4):
        Dl, *_ = np.linalg.lstsq(Ya[l].numpy(), Yr[l].numpy(), rcond=None)
        Ds.append(Dl.T)
    # validate on other points: the fit must hold there too
    Yb = real_sh(3, torch.tensor(b))
    Ybr = real_sh(3, torch.tensor(b @ R.T))
    for l in range(4):
        assert np.abs(Yb[l].numpy() @ Ds[l].T - Ybr[l].numpy()).max() < 1e-12
    return Ds


def test_sh_matches_scipy_textbook_real_form():
    p = _pts(100, 1)
    u = p / np.linalg.norm(p, axis=1, keepdims=True)
    theta = np.arccos(np.clip(u[:, 2], -1, 1))
    phi = np.arctan2(u[:, 1], u[:, 0])
    Y = real_sh(3, torch.tensor(p))
    for l in range(4):
        ref = np.zeros((p.shape[0], 2 * l + 1))
        for m in range(-l, l + 1):
            c = sph_harm_y(l, abs(m), theta, phi)
            if m > 0:
                val = math.sqrt(2) * (-1) ** m * c.real
            elif m < 0:
                val = math.sqrt(2) * (-1) ** m * c.imag
            else:
                val = c.real
            ref[:, m + l] = val * math.sqrt(4 * math.pi)
        assert np.abs(Y[l].numpy() - ref).max() < 1e-12


def test_sh_addition_theorem_and_scale_invariance():
    p = torch.tensor(_pts(50, 2))
    Y = real_sh(3, p)
    Y2 = real_sh(3, 3.7 * p)
    for l in range(4):
        assert torch.allclose((Y[l] ** 2).sum(-1), torch.full((50,), 2.0 * l + 1, dtype=torch.float64), atol=1e-12)
        assert torch.allclose(Y[l], Y2[l], atol=1e-14)


def test_sh_closed_form_values():
    # along +z: Y1 = sqrt3 (0, 1, 0); Y2 = (0, 0, sqrt5, 0, 0)
    Y = real_sh(2, torch.tensor([[0.0, 0.0, 2.0]]))
    assert np.allclose(Y[1].numpy(), [[0, math.sqrt(3), 0]])
    assert np.allclose(Y[2].numpy(), [[0, 0, math.sqrt(5), 0, 0]])
    # along +x: Y1 = sqrt3 (0, 0, 1); Y2 = (0, 0, -sqrt5/2, 0, sqrt15/2)
    Y = real_sh(2, torch.tensor([[1.0, 0.0, 0.0]]))
    assert np.allclose(Y[1].numpy(), [[0, 0, math.sqrt(3)]])
    assert np.allclose(Y[2].numpy(), [[0, 0, -math.sqrt(5) / 2, 0, math.sqrt(15) / 2]])


@pytest.mark.parametrize("path", PATHS)
def test_cg_orthogonality(path):
    C = real_cg(*path)
    G = np.einsum("abc,abd->cd", C, C)
    assert np.abs(G - np.eye(2 * path[2] + 1)).max() < 1e-12


@pytest.mark.parametrize("seed", [1, 2])
def test_cg_equivariance(seed):
    R = Rotation.random(random_state=seed).as_matrix()
    D = _fit_D(R)
    for (l1, l2, l3) in PATHS:
        C = real_cg(l1, l2, l3)
        lhs = np.einsum("abc,ai,bj->ijc", C, D[l1], D[l2])
        rhs = np.einsum("ck,ijk->ijc", D[l3], C)
        assert np.abs(lhs - rhs).max() < 1e-12, (l1, l2, l3)


def test_cg_special_cases():
    for l in range(4):
        assert np.allclose(real_cg(0, l, l)[0], np.eye(2 * l + 1))
        assert np.allclose(real_cg(l, 0, l)[:, 0, :], np.eye(2 * l + 1))
    # 1 x 1 -> 0 is the dot product / sqrt(3)
    assert np.allclose(real_cg(1, 1, 0)[:, :, 0], np.eye(3) / math.sqrt(3))
    # 1 x 1 -> 1 is the cross product / sqrt(2) (components ordered y, z, x)
    a, b = _pts(1, 3)[0], _pts(1, 4)[0]
    perm = [1, 2, 0]                       # (x, y, z) -> (y, z, x)
    f = np.einsum("abc,a,b->c", real_cg(1, 1, 1), a[perm], b[perm])
    assert np.allclose(f, np.cross(a, b)[perm] / math.sqrt(2))


@pytest.mark.parametrize("l1,l2", [(1, 1), (0, 2), (1, 0), (1, 2), (2, 1), (0, 3)])
def test_cg_projects_products_of_harmonics(l1, l2):
    # sum_ab C[a,b,c] Y_l1(u)_a Y_l2(u)_b is proportional to Y_{l1+l2}(u)_c
    p = torch.tensor(_pts(40, 5))
    Y = real_sh(3, p)
    C = real_cg(l1, l2, l1 + l2)
    f = np.einsum("abc,na,nb->nc", C, Y[l1].numpy(), Y[l2].numpy())
    ratio = f / Y[l1 + l2].numpy()
    assert np.abs(ratio - ratio.flat[0]).max() < 1e-10
    assert abs(ratio.flat[0]) > 0.5      # sign is the convention's, size is not


def test_planted_cg_sign_error_is_caught():
    R = Rotation.random(random_state=7).as_matrix()
    D = _fit_D(R)
    C = real_cg(2, 1, 2).copy()
    nz = np.argwhere(np.abs(C) > 1e-9)[3]
    C[tuple(nz)] *= -1.0
    lhs = np.einsum("abc,ai,bj->ijc", C, D[2], D[1])
    rhs = np.einsum("ck,ijk->ijc", D[2], C)
    assert np.abs(lhs - rhs).max() > 1e-3
