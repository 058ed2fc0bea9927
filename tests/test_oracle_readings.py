"""Pins of the oracle's readings of points the paper leaves open.

The paper says the architecture is NequIP's (Sec. 3.2) and gives SevenNet-0's
sizes (Sec. 5.1) but not the gate wiring, the radial MLP's activations and
scales, or how the message sum is normalised.  The oracle takes one reading of
each (SiLU gates in the order [scalars, gates of l = 1, gates of l = 2, ...];
an MLP n_basis -> H -> H -> W with SiLU after the two hidden layers, no biases
and 1/sqrt(fan_in) per layer; the sum of messages divided by the average
neighbour count, a model constant).  Each test below feeds a structured input
whose output under the written reading has a closed form computed here by hand
(math.exp, no torch activation), and plants the plausible mistakes in a copy of
the function to show that the pin catches each one.
"""

import dataclasses
import math

import pytest
import torch

from oracle.model import ModelLayout, conv_layer, gate, layer_specs, radial_mlp
from synth import MODEL_SEVENNET0, MODEL_TINY, normal_weights


def _silu(z):
    return z / (1.0 + math.exp(-z))


def _sigmoid(z):
    return 1.0 / (1.0 + math.exp(-z))


# ------------------------------------------------------------------ gate (Sec. 5.1, Figure 2b)
def _gate_input(spec, seed=4):
    """y of a middle block: y[0] = [mul0 scalars | gates of l = 1 | gates of l = 2 | ...]."""
    g = torch.Generator().manual_seed(seed)
    L = layer_specs(spec)[1]
    return L, {l: torch.randn((1, 2 * l + 1, mu), generator=g, dtype=torch.float64)
               for l, mu in L.y_muls.items()}


def _gate_pin_holds(spec, gate_fn):
    """Every output against the written reading, element by element."""
    L, y = _gate_input(spec)
    out = gate_fn(spec, L, y)
    m0 = spec.mul[0]
    y0 = y[0][0, 0]
    for c in range(m0):
        if abs(float(out[0][0, 0, c]) - _silu(float(y0[c]))) > 1e-14:
            return False
    off = m0
    for l in range(1, spec.lmax + 1):
        for u in range(spec.mul[l]):
            s = _silu(float(y0[off + u]))
            for m in range(2 * l + 1):
                if abs(float(out[l][0, m, u]) - float(y[l][0, m, u]) * s) > 1e-14:
                    return False
        off += spec.mul[l]
    return True


def _gate_one_open(spec, gate_fn, l_open, u_open):
    """All gates zero except channel u_open of irrep l_open: only that channel survives."""
    L, y = _gate_input(spec, seed=9)
    m0 = spec.mul[0]
    y[0][0, 0, m0:] = 0.0
    off = m0 + sum(spec.mul[1:l_open])
    y[0][0, 0, off + u_open] = 0.7
    out = gate_fn(spec, L, y)
    for l in range(1, spec.lmax + 1):
        for u in range(spec.mul[l]):
            nz = float(out[l][0, :, u].abs().max()) > 0.0
            if nz != (l == l_open and u == u_open):
                return False
    ref = y[l_open][0, :, u_open] * _silu(0.7)
    return bool(torch.allclose(out[l_open][0, :, u_open], ref, rtol=0, atol=1e-14))


def _gate_swapped_blocks(spec, L, y):          # planted: gates of l = 2 read first
    m0 = spec.mul[0]
    g = torch.nn.functional.silu(y[0][..., m0:])
    out = {0: torch.nn.functional.silu(y[0][..., :m0])}
    off = 0
    for l in range(spec.lmax, 0, -1):
        out[l] = y[l] * g[..., off:off + spec.mul[l]]
        off += spec.mul[l]
    return out


def _gate_no_silu(spec, L, y):                 # planted: raw gate values
    m0 = spec.mul[0]
    out = {0: torch.nn.functional.silu(y[0][..., :m0])}
    off = m0
    for l in range(1, spec.lmax + 1):
        out[l] = y[l] * y[0][..., off:off + spec.mul[l]]
        off += spec.mul[l]
    return out


def _gate_sigmoid(spec, L, y):                 # planted: sigmoid gates (e3nn's odd-parity habit)
    m0 = spec.mul[0]
    out = {0: torch.nn.functional.silu(y[0][..., :m0])}
    off = m0
    for l in range(1, spec.lmax + 1):
        out[l] = y[l] * torch.sigmoid(y[0][..., off:off + spec.mul[l]])
        off += spec.mul[l]
    return out


def _gate_linear_scalars(spec, L, y):          # planted: scalars pass without SiLU
    out = gate(spec, L, y)
    out[0] = y[0][..., :spec.mul[0]].clone()
    return out


def test_gate_reading_pinned():
    spec = MODEL_SEVENNET0
    assert _gate_pin_holds(spec, gate)
    assert _gate_one_open(spec, gate, 1, 17)
    assert _gate_one_open(spec, gate, 2, 5)


@pytest.mark.parametrize("mutant", [_gate_swapped_blocks, _gate_no_silu, _gate_sigmoid, _gate_linear_scalars])
def test_gate_pin_catches_planted_mistakes(mutant):
    spec = MODEL_SEVENNET0
    caught = not _gate_pin_holds(spec, mutant)
    caught = caught or not _gate_one_open(spec, mutant, 1, 17) or not _gate_one_open(spec, mutant, 2, 5)
    assert caught


def test_gate_last_block_is_silu_of_scalars():
    spec = MODEL_SEVENNET0
    L = layer_specs(spec)[-1]
    y = {0: torch.linspace(-3.0, 3.0, spec.mul[0], dtype=torch.float64).reshape(1, 1, -1)}
    out = gate(spec, L, y)
    assert set(out) == {0}
    for c in range(spec.mul[0]):
        assert abs(float(out[0][0, 0, c]) - _silu(float(y[0][0, 0, c]))) <= 1e-15


# ------------------------------------------------------------------ radial MLP (Sec. 5.1)
def _unit_mlp_weights(spec, t, sign=1.0):
    """mlp0 passes basis function 0 to hidden unit 0, mlp1 is the identity, mlp2
    sends hidden unit 0 to every output column with weight `sign`."""
    layout = ModelLayout(spec)
    Wd = layout.unpack(torch.zeros(layout.size, dtype=torch.float64).numpy())
    Wd = {k: v.clone() for k, v in Wd.items()}
    Wd[f"L{t}.mlp0"][0, 0] = 1.0
    Wd[f"L{t}.mlp1"].copy_(torch.eye(spec.mlp_hidden, dtype=torch.float64))
    Wd[f"L{t}.mlp2"][0, :] = sign
    return Wd


def _mlp_pin_holds(spec, mlp_fn):
    t = 1
    H, nb = spec.mlp_hidden, spec.n_basis
    B = torch.zeros((1, nb), dtype=torch.float64)
    B[0, 0] = 1.0
    for sign in (1.0, -1.0):
        Wd = _unit_mlp_weights(spec, t, sign)
        w = mlp_fn(spec, Wd, t, B)
        # hidden 1: SiLU(1/sqrt(n_basis)); hidden 2: SiLU(that / sqrt(H)); output: sign * that / sqrt(H)
        want = sign * _silu(_silu(1.0 / math.sqrt(nb)) / math.sqrt(H)) / math.sqrt(H)
        if float((w - want).abs().max()) > 1e-15:
            return False
    # no biases: a zero basis vector gives zero weights for any weight matrices
    layout = ModelLayout(spec)
    Wd = layout.unpack(normal_weights(layout.size))
    w0 = mlp_fn(spec, Wd, t, torch.zeros((1, nb), dtype=torch.float64))
    return float(w0.abs().max()) == 0.0


def _mlp_no_silu(spec, Wd, t, B):              # planted: linear MLP
    a1 = B @ Wd[f"L{t}.mlp0"] / math.sqrt(spec.n_basis)
    a2 = a1 @ Wd[f"L{t}.mlp1"] / math.sqrt(spec.mlp_hidden)
    return a2 @ Wd[f"L{t}.mlp2"] / math.sqrt(spec.mlp_hidden)


def _mlp_fan_in(spec, Wd, t, B):               # planted: 1/fan_in instead of 1/sqrt(fan_in)
    h1 = torch.nn.functional.silu(B @ Wd[f"L{t}.mlp0"] / spec.n_basis)
    h2 = torch.nn.functional.silu(h1 @ Wd[f"L{t}.mlp1"] / spec.mlp_hidden)
    return h2 @ Wd[f"L{t}.mlp2"] / spec.mlp_hidden


def _mlp_output_silu(spec, Wd, t, B):          # planted: an activation after the last layer
    return torch.nn.functional.silu(radial_mlp(spec, Wd, t, B))


def _mlp_bias(spec, Wd, t, B):                 # planted: a constant bias on the hidden layers
    a1 = B @ Wd[f"L{t}.mlp0"] / math.sqrt(spec.n_basis) + 0.1
    h1 = torch.nn.functional.silu(a1)
    h2 = torch.nn.functional.silu(h1 @ Wd[f"L{t}.mlp1"] / math.sqrt(spec.mlp_hidden))
    return h2 @ Wd[f"L{t}.mlp2"] / math.sqrt(spec.mlp_hidden)


def test_radial_mlp_reading_pinned():
    assert _mlp_pin_holds(MODEL_SEVENNET0, radial_mlp)
    assert _mlp_pin_holds(MODEL_TINY, radial_mlp)


@pytest.mark.parametrize("mutant", [_mlp_no_silu, _mlp_fan_in, _mlp_output_silu, _mlp_bias])
def test_radial_mlp_pin_catches_planted_mistakes(mutant):
    assert not _mlp_pin_holds(MODEL_SEVENNET0, mutant)


# ------------------------------------------------------------------ message normalisation (Sec. 5.1)
def _one_edge(spec):
    """Receiver 0 with a single sender 1; x, Y and w chosen so that path (0, 0, 0)
    has the closed form m = x * Y_0 * w / avg_num_neigh (C(0,0,0) = 1, Y_0 = 1)."""
    L = layer_specs(spec)[0]
    mu = spec.mul[0]
    x = {0: torch.zeros((2, 1, mu), dtype=torch.float64)}
    x[0][1, 0, :] = torch.arange(1, mu + 1, dtype=torch.float64)
    Y = [torch.ones((1, 1), dtype=torch.float64)] + \
        [torch.zeros((1, 2 * l + 1), dtype=torch.float64) for l in range(1, spec.lmax + 1)]
    w = torch.zeros((1, sum(L.path_mul)), dtype=torch.float64)
    w[0, :mu] = 0.5
    return L, x, Y, w, torch.tensor([0]), torch.tensor([1])


def _norm_pin_holds(spec, conv_fn):
    L, x, Y, w, dst, src = _one_edge(spec)
    m = conv_fn(spec, L, x, Y, w, dst, src, 2)
    mu = spec.mul[0]
    for u in range(mu):
        want = (u + 1) * 1.0 * 0.5 / 34.0          # SevenNet-0's average neighbour count, a constant
        if abs(float(m[0][0, 0, u]) - want) > 1e-15:
            return False
    if float(m[0][1].abs().max()) != 0.0:          # the sender receives nothing
        return False
    # a model constant: the same factor however many edges the structure has
    dst2, src2 = torch.tensor([0, 0]), torch.tensor([1, 1])
    m2 = conv_fn(spec, L, x, Y, torch.cat([w, w]), dst2, src2, 2)
    return bool(torch.allclose(m2[0][0], 2 * m[0][0], rtol=1e-15, atol=0))


def _conv_sqrt_norm(spec, L, x, Y, w, dst, src, n):    # planted: 1/sqrt(avg_num_neigh)
    s = dataclasses.replace(spec, avg_num_neigh=math.sqrt(spec.avg_num_neigh))
    return conv_layer(s, L, x, Y, w, dst, src, n)


def _conv_per_structure(spec, L, x, Y, w, dst, src, n):  # planted: divide by this structure's mean degree
    s = dataclasses.replace(spec, avg_num_neigh=len(dst) / n)
    return conv_layer(s, L, x, Y, w, dst, src, n)


def _conv_unnormalised(spec, L, x, Y, w, dst, src, n):   # planted: no normalisation
    s = dataclasses.replace(spec, avg_num_neigh=1.0)
    return conv_layer(s, L, x, Y, w, dst, src, n)


def test_message_normalisation_pinned():
    assert MODEL_SEVENNET0.avg_num_neigh == 34.0
    assert _norm_pin_holds(MODEL_SEVENNET0, conv_layer)


@pytest.mark.parametrize("mutant", [_conv_sqrt_norm, _conv_per_structure, _conv_unnormalised])
def test_message_normalisation_pin_catches_planted_mistakes(mutant):
    assert not _norm_pin_holds(MODEL_SEVENNET0, mutant)


# ------------------------------------------------------------------ readout (Eq. 1; NequIP's two linears)
def _readout_model():
    """Weights: embedding row of species 2 = 0.3 + 0.01 c, every self-connection of
    the scalars the identity, all else zero (so x, w and the messages vanish and
    each block maps the scalars h -> SiLU(h / sqrt(128))); readout0 sends every
    channel to hidden unit 0, readout1 = 1."""
    spec = MODEL_SEVENNET0
    layout = ModelLayout(spec)
    Wd = {k: v.clone() for k, v in layout.unpack(torch.zeros(layout.size).numpy()).items()}
    m0 = spec.mul[0]
    Wd["embed"][2] = 0.3 + 0.01 * torch.arange(m0, dtype=torch.float64)
    for t in range(spec.n_layers):
        Wd[f"L{t}.sc.0"][:, :m0] = torch.eye(m0, dtype=torch.float64)
    Wd["readout0"][:, 0] = 1.0
    Wd["readout1"][0, 0] = 1.0
    return spec, Wd


def _readout_hand(spec, act_between=False, fan_in=True):
    m0, hid = spec.mul[0], spec.readout_hidden
    h = [0.3 + 0.01 * c for c in range(m0)]
    for _ in range(spec.n_layers):
        h = [_silu(v / math.sqrt(m0)) for v in h]
    z = sum(h) / (math.sqrt(m0) if fan_in else 1.0)
    if act_between:
        z = _silu(z)
    return z / (math.sqrt(hid) if fan_in else 1.0)


def test_readout_reading_pinned():
    from oracle.model import model_energy
    spec, Wd = _readout_model()
    d = torch.zeros((0, 3), dtype=torch.float64)
    e = model_energy(spec, Wd, [2], d, torch.zeros(0, dtype=torch.long), torch.zeros(0, dtype=torch.long), 1)
    want = _readout_hand(spec)
    assert abs(float(e[0]) - want) <= 1e-14 * abs(want)
    # the readings it excludes: an activation between the two readout linears, no 1/sqrt(fan_in)
    for alt in (_readout_hand(spec, act_between=True), _readout_hand(spec, fan_in=False)):
        assert abs(alt - want) > 1e-3 * abs(want)
