"""Radial basis of the edge embedding (FP64).

Sec. 5.1: "8 radial Bessel functions"; the NequIP form is used (the paper is
silent on the exact form, read as in NequIP):
    b_n(r) = (2 / r_c) sin(n pi r / r_c) / r,   n = 1..n_basis,
multiplied by the polynomial cutoff envelope of order p (NequIP's
PolynomialCutoff), with x = r / r_c:
    u(x) = 1 - (p+1)(p+2)/2 x^p + p(p+2) x^(p+1) - p(p+1)/2 x^(p+2)  for x < 1,
    u(x) = 0 for x >= 1.
For p = 6: u(x) = 1 - 28 x^6 + 48 x^7 - 21 x^8.
"""

import math

import torch


def bessel_basis(r: torch.Tensor, r_cut: float, n_basis: int) -> torch.Tensor:
    """[..., n_basis] Bessel functions of the distances r (> 0)."""
    n = torch.arange(1, n_basis + 1, dtype=r.dtype, device=r.device)
    return (2.0 / r_cut) * torch.sin(n * math.pi * r[..., None] / r_cut) / r[..., None]


def poly_envelope(r: torch.Tensor, r_cut: float, p: int) -> torch.Tensor:
    """Polynomial cutoff u(r / r_c), zero at and beyond r_c."""
    x = r / r_cut
    a = (p + 1.0) * (p + 2.0) / 2.0
    b = p * (p + 2.0)
    c = p * (p + 1.0) / 2.0
    u = 1.0 - a * x ** p + b * x ** (p + 1) - c * x ** (p + 2)
    return torch.where(x < 1.0, u, torch.zeros_like(u))
