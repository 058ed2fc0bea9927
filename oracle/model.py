"""The NequIP-style potential of SevenNet, evaluated plainly in FP64 on the CPU.

Paper: Sec. 2 (Eqs. 1-4, Figure 2), Sec. 3.1 (Eqs. 5-8 for forces), Sec. 3.2
("identical to NequIP"), Sec. 5.1 (SevenNet-0: 5 blocks, 128x0e+64x1e+32x2e,
r_c = 5 A, 8 Bessel bases, SH to l = 2, messages / average neighbour count,
self-connection as a linear, last block keeps scalar-output paths only).

Model definition (readings of the points the paper leaves open):

  h^(1)_v = W_emb[Z_v]                                        (mul0 x 0e)
  per block t = 1..T, with input irreps In and gate-input irreps Y:
    sc  = LinSC(h)        x = Lin1(h)
    w_e = MLP(B(r_e))     B = Bessel(r) * envelope(r),  MLP = n_basis -> H -> H -> W,
                          SiLU after the hidden layers, no biases, 1/sqrt(fan_in)
    m_v[p][m3, u] = 1/avg_nn * sum_{e: recv v} w_e[p, u] *
                    sum_{m1, m2} C_p[m1, m2, m3] x_{src e}[l1][m1, u] Y_{l2}(d_e)[m2]
                    (uvu tensor product, Figure 2b; paths p = (l1, l2, l3) with
                     |l1 - l2| <= l3 <= min(l1 + l2, lmax), SO(3) only; last block: l3 = 0)
    y   = Lin2(m) + sc
    h'  = Gate(y): SiLU on the mul0 scalars, SiLU(gate_{l,u}) * y_l[:, u] for l >= 1
          (last block: h' = SiLU(y), mul0 x 0e)
  E_v = scale * R2(R1(h^(T+1)_0e)) + shift[Z_v]              (Eq. 1: E = sum_v E_v)
  Linears act per irrep l on the channel index, out = in @ W / sqrt(mul_in).

Pins (tests/test_oracle_*.py): parameter count 842,432 = "0.84 million"
(Sec. 5.1); rotation / translation / permutation invariance; extensivity;
zero net force; forces and virial against central finite differences;
closed-form messages of one edge for the identity / dot / cross couplings.
The readings of points the paper leaves open are pinned structurally in
tests/test_oracle_readings.py: gate() (SiLU scalars, SiLU gates in the order
[scalars | gates of l = 1 | gates of l = 2 ...], one open gate lets exactly its
channel through), radial_mlp() (one-hot basis through unit weights gives
SiLU(SiLU(1/sqrt(n_basis))/sqrt(H))/sqrt(H); no biases), the message sum over
the constant avg_num_neigh = 34.0, and the readout's two plain linears; each
pin fails under the planted alternatives (no SiLU, sigmoid gates, swapped gate
blocks, 1/fan_in, an output activation, biases, 1/sqrt(avg_num_neigh), a
per-structure degree).  What no test can pin is agreement with the trained
SevenNet's own numbers: no reference weights or printed values exist.

Canonical weight order (one flat FP64 vector): embed [n_species, mul0]; then per
block: sc[l] [mul_in, mul_y] for l in Y and In (ascending l), lin1[l] [mul, mul]
for l in In, mlp0 [n_basis, H], mlp1 [H, H], mlp2 [H, W] (columns: path-major,
channel-minor), lin2[l] [mul_msg, mul_y] for l in Y with messages; finally
readout0 [mul0, hid], readout1 [hid, 1].  Row index = input channel.
"""

from dataclasses import dataclass
import math

import numpy as np
import torch

from .so3 import real_sh, real_cg
from .radial import bessel_basis, poly_envelope
from .neighbors import neighbor_list


@dataclass
class LayerSpec:
    first: bool
    last: bool
    in_muls: dict      # l -> multiplicity of the block input h
    paths: list        # [(l1, l2, l3)]
    path_mul: list     # multiplicity of each path (= in_muls[l1])
    msg_muls: dict     # l3 -> total multiplicity of the messages
    y_muls: dict       # l -> multiplicity of the gate input y
    out_muls: dict     # l -> multiplicity of h'


def layer_specs(spec) -> list:
    lmax = spec.lmax
    full = {l: spec.mul[l] for l in range(lmax + 1)}
    out = []
    for t in range(spec.n_layers):
        first, last = t == 0, t == spec.n_layers - 1
        in_muls = {0: spec.mul[0]} if first else dict(full)
        paths = []
        for l1 in sorted(in_muls):
            for l2 in range(lmax + 1):
                for l3 in range(abs(l1 - l2), min(l1 + l2, lmax) + 1):
                    if last and l3 != 0:
                        continue
                    paths.append((l1, l2, l3))
        path_mul = [in_muls[p[0]] for p in paths]
        msg_muls = {}
        for p, mu in zip(paths, path_mul):
            msg_muls[p[2]] = msg_muls.get(p[2], 0) + mu
        if last:
            y_muls = {0: spec.mul[0]}
            out_muls = {0: spec.mul[0]}
        else:
            y_muls = {0: spec.mul[0] + sum(spec.mul[1:])}
            y_muls.update({l: spec.mul[l] for l in range(1, lmax + 1)})
            out_muls = dict(full)
        out.append(LayerSpec(first, last, in_muls, paths, path_mul,
                             dict(sorted(msg_muls.items())), y_muls, out_muls))
    return out


class ModelLayout:
    """Names, shapes and offsets of the canonical flat weight vector."""

    def __init__(self, spec):
        self.spec = spec
        self.layers = layer_specs(spec)
        entries = [("embed", (spec.n_species, spec.mul[0]))]
        H = spec.mlp_hidden
        for t, L in enumerate(self.layers):
            for l in sorted(L.y_muls):
                if l in L.in_muls:
                    entries.append((f"L{t}.sc.{l}", (L.in_muls[l], L.y_muls[l])))
            for l in sorted(L.in_muls):
                entries.append((f"L{t}.lin1.{l}", (L.in_muls[l], L.in_muls[l])))
            entries.append((f"L{t}.mlp0", (spec.n_basis, H)))
            entries.append((f"L{t}.mlp1", (H, H)))
            entries.append((f"L{t}.mlp2", (H, sum(L.path_mul))))
            for l in sorted(L.y_muls):
                if l in L.msg_muls:
                    entries.append((f"L{t}.lin2.{l}", (L.msg_muls[l], L.y_muls[l])))
        entries.append(("readout0", (spec.mul[0], spec.readout_hidden)))
        entries.append(("readout1", (spec.readout_hidden, 1)))
        self.entries = entries
        self.offsets = {}
        off = 0
        for name, shape in entries:
            self.offsets[name] = (off, shape)
            off += int(np.prod(shape))
        self.size = off

    def unpack(self, flat) -> dict:
        flat = torch.as_tensor(np.asarray(flat, dtype=np.float64))
        if flat.numel() < self.size:
            raise ValueError("weight vector too short")
        return {n: flat[o:o + int(np.prod(s))].reshape(s)
                for n, (o, s) in self.offsets.items()}


def param_layout(spec) -> ModelLayout:
    return ModelLayout(spec)


def n_params(spec) -> int:
    return ModelLayout(spec).size


def _lin(x, W):
    """Per-irrep linear: x [N, 2l+1, mul_in] @ W [mul_in, mul_out] / sqrt(mul_in)."""
    return torch.matmul(x, W) / math.sqrt(W.shape[0])


def radial_mlp(spec, Wd, t, basis):
    a1 = basis @ Wd[f"L{t}.mlp0"] / math.sqrt(spec.n_basis)
    h1 = torch.nn.functional.silu(a1)
    a2 = h1 @ Wd[f"L{t}.mlp1"] / math.sqrt(spec.mlp_hidden)
    h2 = torch.nn.functional.silu(a2)
    return h2 @ Wd[f"L{t}.mlp2"] / math.sqrt(spec.mlp_hidden)


def edge_features(spec, d):
    """Y_l(d) for l <= lmax and the enveloped Bessel basis of |d| (Sec. 2, 5.1)."""
    r = torch.linalg.norm(d, dim=-1)
    Y = real_sh(spec.lmax, d)
    B = bessel_basis(r, spec.r_cut, spec.n_basis) * \
        poly_envelope(r, spec.r_cut, spec.poly_p)[..., None]
    return Y, B


def conv_layer(spec, L, x, Y, w, dst, src, n_atoms):
    """Messages of Eq. 3: uvu CG tensor product summed over each receiver.

    x: dict l1 -> [N, 2l1+1, mul];  Y: list of [E, 2l2+1];  w: [E, W].
    Returns dict l3 -> [N, 2l3+1, msg_mul] with paths concatenated in order.
    """
    parts = {}
    col = 0
    for (l1, l2, l3), mu in zip(L.paths, L.path_mul):
        C = torch.as_tensor(real_cg(l1, l2, l3))
        xw = x[l1][src]                                     # [E, 2l1+1, mu]
        if xw.shape[0] == 0:                                # no edges: no messages
            t = torch.zeros((0, 2 * l3 + 1, mu), dtype=xw.dtype)
        else:
            t = torch.einsum("abc,eau,eb->ecu", C, xw, Y[l2])   # [E, 2l3+1, mu]
        t = t * w[:, None, col:col + mu]
        col += mu
        m = torch.zeros((n_atoms, 2 * l3 + 1, mu), dtype=t.dtype)
        m = m.index_add(0, dst, t)
        parts.setdefault(l3, []).append(m / spec.avg_num_neigh)
    return {l3: torch.cat(v, dim=-1) for l3, v in sorted(parts.items())}


def gate(spec, L, y):
    if L.last:
        return {0: torch.nn.functional.silu(y[0])}
    m0 = spec.mul[0]
    s = y[0][..., :m0]
    g = torch.nn.functional.silu(y[0][..., m0:])
    out = {0: torch.nn.functional.silu(s)}
    off = 0
    for l in range(1, spec.lmax + 1):
        mu = spec.mul[l]
        out[l] = y[l] * g[..., off:off + mu]
        off += mu
    return out


def model_energy(spec, Wd, species, d, dst, src, n_atoms, return_layers=False):
    """Per-atom energies from edge displacement vectors d (Eq. 1)."""
    layers = layer_specs(spec)
    Y, B = edge_features(spec, d)
    species = torch.as_tensor(species, dtype=torch.long)
    h = {0: Wd["embed"][species][:, None, :]}
    trace = []
    for t, L in enumerate(layers):
        sc = {l: _lin(h[l], Wd[f"L{t}.sc.{l}"]) for l in L.y_muls if l in h}
        x = {l: _lin(h[l], Wd[f"L{t}.lin1.{l}"]) for l in L.in_muls}
        w = radial_mlp(spec, Wd, t, B)
        m = conv_layer(spec, L, x, Y, w, dst, src, n_atoms)
        y = {}
        for l, mu in L.y_muls.items():
            acc = sc.get(l)
            if l in m:
                z = _lin(m[l], Wd[f"L{t}.lin2.{l}"])
                acc = z if acc is None else acc + z
            if acc is None:
                acc = torch.zeros((n_atoms, 2 * l + 1, mu), dtype=d.dtype)
            y[l] = acc
        h = gate(spec, L, y)
        trace.append(dict(x=x, m=m, y=y, h=h))
    h0 = h[0][:, 0, :]
    z = h0 @ Wd["readout0"] / math.sqrt(spec.mul[0])
    e = (z @ Wd["readout1"])[:, 0] / math.sqrt(spec.readout_hidden)
    shift = torch.as_tensor(spec.shifts(), dtype=d.dtype)
    e_atom = spec.scale * e + shift[species]
    if return_layers:
        return e_atom, trace
    return e_atom


def energy_forces_virial(spec, weights, species, pos, cell, pbc=(True, True, True),
                         edges=None):
    """E (Eq. 1), F = -dE/dr (Eq. 2) and W = -dE/d(strain) in FP64.

    weights: flat canonical FP64 vector; pos [N, 3] A; cell [3, 3] rows.
    Returns (E, F [N, 3], W [3, 3], e_atom [N], (dst, src, shift)).
    Strain eps maps r -> (I + eps) r and the cell rows likewise; W_ab = -dE/deps_ab.
    """
    layout = ModelLayout(spec)
    Wd = layout.unpack(weights)
    pos = np.asarray(pos, np.float64)
    cell = np.asarray(cell, np.float64)
    if edges is None:
        edges = neighbor_list(pos, cell, spec.r_cut, pbc)
    dst, src, shift = edges
    n = pos.shape[0]
    P = torch.tensor(pos, requires_grad=True)
    eps = torch.zeros((3, 3), dtype=torch.float64, requires_grad=True)
    F_ = torch.eye(3, dtype=torch.float64) + eps
    Ps = P @ F_.T
    Cs = torch.as_tensor(cell) @ F_.T
    dst_t = torch.as_tensor(dst, dtype=torch.long)
    src_t = torch.as_tensor(src, dtype=torch.long)
    d = Ps[src_t] - Ps[dst_t] + torch.as_tensor(shift, dtype=torch.float64) @ Cs
    e_atom = model_energy(spec, Wd, species, d, dst_t, src_t, n)
    E = e_atom.sum()
    gP, gE = torch.autograd.grad(E, (P, eps))
    return (float(E.detach()), (-gP).numpy(), (-gE).numpy(), e_atom.detach().numpy(),
            (dst, src, shift))
