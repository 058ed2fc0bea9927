"""Real spherical harmonics and real-basis Clebsch-Gordan tensors (FP64).

Conventions (the paper defers to NequIP/e3nn, Sec. 3.2, and states only
"spherical harmonics up to l = 2", Sec. 5.1):

* Real spherical harmonics with z as the polar axis, ordered m = -l..l, in
  "component" normalisation: sum_m Y_lm(u)^2 = 2l + 1 on the unit sphere.
      l = 0: 1
      l = 1: sqrt(3) (y, z, x)
      l = 2: sqrt(15) xy, sqrt(15) yz, sqrt(5)/2 (3z^2 - 1), sqrt(15) xz,
             sqrt(15)/2 (x^2 - y^2)
* Real CG tensor C[a, b, c] of the coupling l1 (x) l2 -> l3: the complex
  Clebsch-Gordan coefficients <l1 m1 l2 m2 | l3 m3> (sympy, exact) carried to
  the real basis above by the unitary map U_l (real = U_l complex), i.e.
      C = sum U3[c, m3] <l1 m1 l2 m2|l3 m3> conj(U1[a, m1]) conj(U2[b, m2]),
  which is purely real or purely imaginary; the non-zero part is kept,
  scaled to sum C^2 = 2 l3 + 1, and its sign fixed so that the first entry in
  (a, b, c) order with |C| > 1e-9 is positive.
"""

from functools import lru_cache
import math

import numpy as np
import torch


def real_sh(lmax: int, vec: torch.Tensor) -> list:
    """Y_l(vec / |vec|) for l = 0..lmax; returns a list of [..., 2l+1] tensors."""
    r = torch.linalg.norm(vec, dim=-1, keepdim=True)
    u = vec / r
    x, y, z = u[..., 0], u[..., 1], u[..., 2]
    out = [torch.ones_like(x)[..., None]]
    if lmax >= 1:
        s3 = math.sqrt(3.0)
        out.append(torch.stack([s3 * y, s3 * z, s3 * x], dim=-1))
    if lmax >= 2:
        s15 = math.sqrt(15.0)
        s5 = math.sqrt(5.0)
        out.append(torch.stack([
            s15 * x * y,
            s15 * y * z,
            0.5 * s5 * (3.0 * z * z - 1.0),
            s15 * x * z,
            0.5 * s15 * (x * x - y * y),
        ], dim=-1))
    if lmax >= 3:
        # the standard real harmonics of degree 3 times sqrt(4 pi), m = -3..3
        a, b, c, d = math.sqrt(70.0) / 4.0, math.sqrt(105.0), math.sqrt(42.0) / 4.0, math.sqrt(7.0) / 2.0
        out.append(torch.stack([
            a * y * (3.0 * x * x - y * y),
            b * x * y * z,
            c * y * (5.0 * z * z - 1.0),
            d * z * (5.0 * z * z - 3.0),
            c * x * (5.0 * z * z - 1.0),
            0.5 * b * z * (x * x - y * y),
            a * x * (x * x - 3.0 * y * y),
        ], dim=-1))
    if lmax > 3:
        raise NotImplementedError("real_sh: lmax <= 3")
    return out


def complex_to_real(l: int) -> np.ndarray:
    """U_l with Y_real[m] = sum_m' U_l[m, m'] Y_complex[m'] (rows/cols m = -l..l).

    Real SH defined from Condon-Shortley complex SH as
      m > 0: sqrt(2) (-1)^m Re Y_l^m,   m = 0: Y_l^0,   m < 0: sqrt(2) (-1)^m Im Y_l^|m|;
    with Y_l^{-m} = (-1)^m conj(Y_l^m) these are the entries below.
    """
    U = np.zeros((2 * l + 1, 2 * l + 1), dtype=np.complex128)
    s = 1.0 / math.sqrt(2.0)
    for m in range(-l, l + 1):
        i = m + l
        if m == 0:
            U[i, l] = 1.0
        elif m > 0:
            U[i, m + l] = (-1) ** m * s
            U[i, -m + l] = s
        else:
            mu = -m
            U[i, -mu + l] = 1j * s
            U[i, mu + l] = -1j * (-1) ** mu * s
    return U


@lru_cache(maxsize=None)
def complex_cg(l1: int, l2: int, l3: int) -> np.ndarray:
    """<l1 m1 l2 m2 | l3 m3> as a dense [2l1+1, 2l2+1, 2l3+1] array (sympy, exact)."""
    from sympy.physics.quantum.cg import CG
    from sympy import S
    T = np.zeros((2 * l1 + 1, 2 * l2 + 1, 2 * l3 + 1))
    for m1 in range(-l1, l1 + 1):
        for m2 in range(-l2, l2 + 1):
            m3 = m1 + m2
            if abs(m3) <= l3:
                T[m1 + l1, m2 + l2, m3 + l3] = float(
                    CG(S(l1), S(m1), S(l2), S(m2), S(l3), S(m3)).doit())
    return T


@lru_cache(maxsize=None)
def real_cg(l1: int, l2: int, l3: int) -> np.ndarray:
    """Real-basis coupling tensor C[a, b, c] (see module docstring)."""
    if not (abs(l1 - l2) <= l3 <= l1 + l2):
        raise ValueError("real_cg: triangle condition violated")
    Cc = complex_cg(l1, l2, l3)
    U1, U2, U3 = complex_to_real(l1), complex_to_real(l2), complex_to_real(l3)
    C = np.einsum("cz,xyz,ax,by->abc", U3, Cc, U1.conj(), U2.conj())
    re, im = np.abs(C.real).max(), np.abs(C.imag).max()
    C = C.real if re >= im else C.imag
    if min(re, im) > 1e-12 * max(re, im):
        raise AssertionError("real_cg: tensor neither real nor imaginary")
    C = C * math.sqrt((2 * l3 + 1) / (C * C).sum())
    flat = C.reshape(-1)
    first = flat[np.nonzero(np.abs(flat) > 1e-9)[0][0]]
    if first < 0:
        C = -C
    C[np.abs(C) < 1e-15] = 0.0
    return C
