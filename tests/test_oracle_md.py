"""Pins of the oracle integrators: NVE energy conservation of velocity Verlet
and its second-order error (halving dt quarters the energy error); the
Nose-Hoover NVT splitting against velocity Verlet (tau -> infinity), its
extended-energy conservation and second-order error, and the zero-force case
against an independent ODE solution (scipy)."""

import dataclasses

import numpy as np

import oracle
from synth import make_workload, normal_weights, maxwell_boltzmann

KB = 8.617333262e-5


def _setup(scale):
    s, spec = make_workload("sio2_192")
    spec = dataclasses.replace(spec, scale=scale)
    w = normal_weights(oracle.n_params(spec))
    m = s.masses()
    v = maxwell_boltzmann(m, 3000.0, seed=3)
    return s, spec, w, m, v


def test_initial_velocities():
    s, spec, w, m, v = _setup(1.0)
    assert abs(oracle.kinetic_energy(v, m) - 0.5 * (3 * len(m) - 3) * KB * 3000) < 1e-9
    assert np.abs((m[:, None] * v).sum(0)).max() < 1e-12


def test_nve_drift_small():
    s, spec, w, m, v = _setup(1.0)
    E0, F0, *_ = oracle.energy_forces_virial(spec, w, s.species, s.pos, s.cell)
    etot0 = E0 + oracle.kinetic_energy(v, m)
    _, _, _, ep, ek = oracle.velocity_verlet(spec, w, s.species, s.pos, v, m, s.cell, 1.0, 100)
    drift = np.abs(ep + ek - etot0).max() / len(m)
    assert drift < 1e-5, drift


def test_verlet_error_is_second_order():
    # an energy scale of 200 gives O(0.1) eV/A forces, so the error is measurable
    s, spec, w, m, v = _setup(200.0)
    E0, F0, *_ = oracle.energy_forces_virial(spec, w, s.species, s.pos, s.cell)
    assert np.sqrt((F0 ** 2).mean()) > 0.05
    etot0 = E0 + oracle.kinetic_energy(v, m)
    errs = []
    for dt, n in ((1.0, 8), (0.5, 16)):
        _, _, _, ep, ek = oracle.velocity_verlet(spec, w, s.species, s.pos, v, m, s.cell, dt, n)
        errs.append(abs(ep[-1] + ek[-1] - etot0))
    ratio = errs[0] / errs[1]
    assert 2.5 < ratio < 6.0, (errs, ratio)


def test_nose_hoover_reduces_to_verlet_for_infinite_tau():
    s, spec, w, m, v = _setup(200.0)
    p1, v1, *_ = oracle.velocity_verlet(spec, w, s.species, s.pos, v, m, s.cell, 1.0, 6)
    out = oracle.nose_hoover_nvt(spec, w, s.species, s.pos, v, m, s.cell, 1.0, 6, 3000.0, 1e12)
    assert np.abs(out[0] - p1).max() < 1e-10
    assert np.abs(out[1] - v1).max() < 1e-12
    assert abs(out[3]) < 1e-20 and abs(out[4]) < 1e-18          # xi, eta stay zero


def test_nose_hoover_extended_energy_second_order():
    s, spec, w, m, v = _setup(200.0)
    errs = []
    for dt, n in ((1.0, 8), (0.5, 16)):
        out = oracle.nose_hoover_nvt(spec, w, s.species, s.pos, v, m, s.cell, dt, n, 1500.0, 10.0)
        ex = out[7]
        E0, *_ = oracle.energy_forces_virial(spec, w, s.species, s.pos, s.cell)
        ex0 = E0 + oracle.kinetic_energy(v, m)
        errs.append(abs(ex[-1] - ex0))
        assert abs(out[3]) > 1e-4           # the thermostat acts (T0 != T)
    ratio = errs[0] / errs[1]
    assert 2.5 < ratio < 6.0, (errs, ratio)


def test_nose_hoover_zero_forces_matches_ode():
    # With F = 0 every velocity scales by exp(-eta), so K = K0 exp(-2 eta) and
    # the thermostat obeys eta' = xi, xi' = (2 K0 exp(-2 eta) - N_f k T0) / Q.
    from scipy.integrate import solve_ivp
    rng = np.random.default_rng(11)
    n = 64
    m = rng.uniform(10.0, 30.0, n)
    v = maxwell_boltzmann(m, 1000.0, seed=12)
    pos = rng.uniform(0, 10, (n, 3))
    t0k, tau, t_end = 3000.0, 10.0, 20.0
    q = oracle.nose_hoover_q(n, t0k, tau)
    nf, kt0 = 3 * n - 3, KB * t0k
    k0 = oracle.kinetic_energy(v, m)

    def rhs(_, y):
        return [y[1], (2.0 * k0 * np.exp(-2.0 * y[0]) - nf * kt0) / q]
    ref = solve_ivp(rhs, (0.0, t_end), [0.0, 0.0], rtol=1e-12, atol=1e-14).y[:, -1]
    zero = lambda p: (0.0, np.zeros_like(p))
    errs = []
    for dt in (0.2, 0.1):
        out = oracle.nose_hoover_steps(zero, pos, v, m, dt, int(round(t_end / dt)), t0k, tau)
        errs.append(abs(out[4] - ref[0]))
        assert abs(out[6][-1] - k0 * np.exp(-2.0 * ref[0])) < 1e-3 * k0
        assert abs(out[3] - ref[1]) < 1e-3 * abs(ref[1]) + 1e-9
    assert errs[1] < 1e-4 * abs(ref[0]) + 1e-9
    assert 3.0 < errs[0] / errs[1] < 5.0, errs


def test_nose_hoover_flat_ramp_equals_constant_target():
    # a ramp from T to T is the constant-target thermostat, bit for bit
    rng = np.random.default_rng(21)
    n = 40
    m = rng.uniform(10.0, 30.0, n)
    v = maxwell_boltzmann(m, 800.0, seed=22)
    pos = rng.uniform(0, 10, (n, 3))
    spring = lambda p: (0.5 * float((p * p).sum()), -p)
    a = oracle.nose_hoover_steps(spring, pos, v, m, 0.5, 30, 1200.0, 20.0)
    b = oracle.nose_hoover_steps(spring, pos, v, m, 0.5, 30, 1200.0, 20.0, t_end_k=1200.0, ramp_steps=17)
    for x, y in zip(a, b):
        assert np.array_equal(np.asarray(x), np.asarray(y))


def test_ramp_target_midpoints():
    # step k of an n-step ramp sits at the ramp's value at k + 1/2; afterwards the end value
    vals = [oracle.ramp_target(3000.0, 2000.0, 4, k) for k in range(6)]
    assert np.allclose(vals, [2875.0, 2625.0, 2375.0, 2125.0, 2000.0, 2000.0], rtol=0, atol=1e-12)
    assert oracle.ramp_target(300.0, 5000.0, 0, 7) == 300.0


def test_nose_hoover_ramp_zero_forces_matches_ode():
    # F = 0 under a continuously ramped target T0(t) = T_s + (T_e - T_s) t / t_r and
    # Q(t) = N_f k_B T0(t) tau^2: eta' = xi, xi' = (2 K0 exp(-2 eta) - N_f k_B T0(t)) / Q(t).
    # The stepped schedule (target at each step's middle) converges to it at second order.
    from scipy.integrate import solve_ivp
    rng = np.random.default_rng(23)
    n = 64
    m = rng.uniform(10.0, 30.0, n)
    v = maxwell_boltzmann(m, 1000.0, seed=24)
    pos = rng.uniform(0, 10, (n, 3))
    ts, te, tau, t_r = 1000.0, 3000.0, 10.0, 20.0
    nf = 3 * n - 3
    k0 = oracle.kinetic_energy(v, m)

    def rhs(t, y):
        t0 = ts + (te - ts) * t / t_r
        return [y[1], (2.0 * k0 * np.exp(-2.0 * y[0]) - nf * KB * t0) / (nf * KB * t0 * tau * tau)]
    ref = solve_ivp(rhs, (0.0, t_r), [0.0, 0.0], rtol=1e-12, atol=1e-14).y[:, -1]
    zero = lambda p: (0.0, np.zeros_like(p))
    errs = []
    for dt in (0.2, 0.1):
        steps = int(round(t_r / dt))
        out = oracle.nose_hoover_steps(zero, pos, v, m, dt, steps, ts, tau, t_end_k=te, ramp_steps=steps)
        errs.append(abs(out[4] - ref[0]))
        assert abs(out[3] - ref[1]) < 1e-3 * abs(ref[1]) + 1e-9
    assert errs[1] < 1e-4 * abs(ref[0]) + 1e-9
    assert 3.0 < errs[0] / errs[1] < 5.0, errs
