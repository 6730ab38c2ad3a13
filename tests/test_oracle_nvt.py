"""Pins of the oracle's Nose-Hoover NVT step (oracle/md.py) against the
mathematics, not against itself:

  * an infinitely heavy thermostat (Q = inf) leaves xi at 0, and the step is
    then exactly the NVE velocity-Verlet step;
  * the split is time reversible: n steps, then v, L_b and xi negated, n
    steps, return to the start;
  * with a smooth pair energy the extended energy H' = E + K + Q xi^2/2 +
    g kT eta is conserved to second order in dt;
  * for free bodies (no forces, spherical tops) the total kinetic energy,
    xi and eta follow the thermostat's own ODE system
      dK/dt = -2 xi K,  dxi/dt = (2K - g kT)/Q,  deta/dt = xi,
    solved independently to 1e-12 by scipy, with O(dt^2) error.
No GPU.
"""
import numpy as np
import pytest

import oracle
from oracle import bodies, md, nn
from paper_2402_12199_gb300 import inputs

CUBE = bodies.cube_template()


def _cube_system(n=8, seed=3, phi=0.12, kT=1.0):
    M, I = bodies.mass_and_inertia(CUBE)
    st, L = inputs.system_state(n, phi, kT, seed, M, np.diag(I))
    box = np.array([L] * 3)
    state = {"pos": st["pos"][:, :3].astype(np.float64), "quat": st["quat"].astype(np.float64),
             "vel": st["vel"][:, :3].astype(np.float64),
             "angmom": st["angmom"][:, :3].astype(np.float64)}
    return state, M, np.diag(I), box


def _bead_forces(box):
    Rc = bodies.pair_cutoff(CUBE)

    def force_fn(pos, quat):
        pairs = oracle.pairs_bruteforce(pos, box, Rc)
        F, tau, E, _ = oracle.forces_beads(pos, quat, box, CUBE, pairs)
        return F, tau, E

    return force_fn


def test_infinite_thermostat_mass_is_nve():
    state, M, I, box = _cube_system()
    force_fn = _bead_forces(box)
    F, tau, _ = force_fn(state["pos"], state["quat"])
    st = dict(state, F=F, tau=tau)
    th = dict(md.thermostat(8, 1.0, 1.0), Q=np.inf)
    a, Ea = md.step(st, force_fn, M, I, box, 0.004)
    b, Eb, th2 = md.step_nvt(st, force_fn, M, I, box, 0.004, th)
    assert th2["xi"] == 0.0 and th2["eta"] == 0.0
    for k in ("pos", "quat", "vel", "angmom"):
        np.testing.assert_array_equal(a[k], b[k])
    assert Ea == Eb


def test_nvt_time_reversibility():
    state, M, I, box = _cube_system(seed=4)
    force_fn = _bead_forces(box)
    th = md.thermostat(8, 1.5, 0.2, xi=0.3)
    st, th1, _ = md.run_nvt(state, force_fn, M, I, box, 0.004, 12, th)
    assert abs(th1["xi"] - 0.3) > 1e-3
    back = dict(st, vel=-st["vel"], angmom=-st["angmom"])
    st2, th2, _ = md.run_nvt(back, force_fn, M, I, box, 0.004, 12, dict(th1, xi=-th1["xi"]))
    np.testing.assert_allclose(st2["pos"], state["pos"], atol=1e-9)
    np.testing.assert_allclose(np.abs((st2["quat"] * state["quat"]).sum(1)), 1.0, atol=1e-12)
    np.testing.assert_allclose(-st2["vel"], state["vel"], atol=1e-10)
    np.testing.assert_allclose(-st2["angmom"], state["angmom"], atol=1e-8)
    assert -th2["xi"] == pytest.approx(0.3, abs=1e-10)
    assert th2["eta"] == pytest.approx(0.0, abs=1e-10)


def test_extended_energy_is_conserved_to_second_order():
    rng = np.random.default_rng(7)
    mu, isd = inputs.feature_normalisation(5.0, 9.4)
    flat = inputs.mlp_params(16, 3, 7, mu=mu, inv_sd=isd, e_scale=2.0, e_shift=-0.3)
    p = nn.unpack(flat.astype(np.float64), 16)
    state, M, I, box = _cube_system(n=8, seed=6)
    Rc = bodies.pair_cutoff(CUBE)

    def force_fn(pos, quat):
        pairs = oracle.pairs_bruteforce(pos, box, Rc)
        F, tau, E, _ = nn.forces_nn(p, pos, quat, box, pairs)
        return F, tau, E

    state = dict(state, vel=state["vel"] * 20, angmom=state["angmom"] * 20)
    th = md.thermostat(8, 2.0, 0.05)
    _, t1, h1 = md.run_nvt(state, force_fn, M, I, box, 0.004, 10, th)
    _, t2, h2 = md.run_nvt(state, force_fn, M, I, box, 0.002, 20, th)
    assert abs(t1["xi"]) > 1e-2  # the thermostat acts
    d1 = np.abs(h1 - h1[0]).max()
    d2 = np.abs(h2 - h2[0]).max()
    assert d1 > 1e-12
    assert 2.5 < d1 / d2 < 6.0, (d1, d2)


def test_free_bodies_follow_the_thermostat_ode():
    from scipy.integrate import solve_ivp

    n = 27
    state, M, I, box = _cube_system(n=n, seed=8, phi=0.01)
    zero = lambda pos, quat: (np.zeros_like(pos), np.zeros_like(pos), 0.0)
    kT, tau, T_end = 2.0, 0.3, 0.6
    th0 = md.thermostat(n, kT, tau, xi=0.5)
    kt, kr = md.kinetic(state["vel"], state["angmom"], M, I)
    K0 = kt + kr
    g_kT, Q = th0["g"] * kT, th0["Q"]

    def rhs(_, y):
        K, xi, _eta = y
        return [-2.0 * xi * K, (2.0 * K - g_kT) / Q, xi]

    ref = solve_ivp(rhs, (0.0, T_end), [K0, 0.5, 0.0], method="DOP853", rtol=1e-12, atol=1e-12)
    K_ref, xi_ref, eta_ref = ref.y[:, -1]
    errs = []
    for dt in (0.01, 0.005):
        st, th, _ = md.run_nvt(state, zero, M, I, box, dt, int(round(T_end / dt)), th0)
        kt, kr = md.kinetic(st["vel"], st["angmom"], M, I)
        e = np.array([(kt + kr - K_ref) / K_ref, th["xi"] - xi_ref, th["eta"] - eta_ref])
        assert np.abs(e).max() < 5e-3
        errs.append(np.abs(e).max())
    assert 2.5 < errs[0] / errs[1] < 6.0, errs
