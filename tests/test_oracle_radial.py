"""Pins of the radial basis and the cutoff envelope (Sec. 5.1, NequIP forms)."""

import math

import numpy as np
import torch
from scipy.integrate import quad

from oracle.radial import bessel_basis, poly_envelope


def test_bessel_orthogonality_fixes_frequencies_and_prefactor():
    rc, n = 5.0, 8
    # int_0^rc r^2 b_n b_m dr = (2/rc) delta_nm for b_n = 2/rc sin(n pi r/rc)/r
    G = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            f = lambda r: r * r * float(bessel_basis(torch.tensor([r], dtype=torch.float64), rc, n)[0, i] *
                                          bessel_basis(torch.tensor([r], dtype=torch.float64), rc, n)[0, j])
            G[i, j] = quad(f, 1e-9, rc, limit=200)[0]
    assert np.abs(G - (2.0 / rc) * np.eye(n)).max() < 1e-8


def test_bessel_small_r_limit():
    rc, n = 5.0, 8
    b = bessel_basis(torch.tensor([1e-7], dtype=torch.float64), rc, n)[0].numpy()
    ref = 2.0 / rc * np.arange(1, n + 1) * math.pi / rc
    assert np.allclose(b, ref, rtol=1e-10)


def test_envelope_smoothness_at_cutoff():
    rc, p = 5.0, 6
    r = torch.tensor([rc * (1 - 1e-12)], dtype=torch.float64, requires_grad=True)
    u = poly_envelope(r, rc, p)
    (du,) = torch.autograd.grad(u.sum(), r, create_graph=True)
    (d2u,) = torch.autograd.grad(du.sum(), r)
    assert abs(float(u)) < 1e-9 and abs(float(du)) < 1e-9 and abs(float(d2u)) < 1e-8
    assert float(poly_envelope(torch.tensor([0.0], dtype=torch.float64), rc, p)) == 1.0
    beyond = poly_envelope(torch.tensor([rc, rc + 0.1], dtype=torch.float64), rc, p)
    assert torch.all(beyond == 0)


def test_envelope_p6_coefficients():
    x = np.linspace(0, 0.99, 7)
    u = poly_envelope(torch.tensor(x * 5.0), 5.0, 6).numpy()
    assert np.allclose(u, 1 - 28 * x ** 6 + 48 * x ** 7 - 21 * x ** 8, atol=1e-14)
