"""Oracle: rigid-body NVE velocity Verlet (numpy FP64).

TEST INFRASTRUCTURE (see the package docstring).

The paper integrates the rigid bodies' equations of motion with the forces and
torques of either method (Results; HOOMD-blue for the bead form, an in-house
code for the network form) but gives no integrator.  The reading used here is
velocity Verlet for the centre of mass and the NO_SQUISH symmetric free-rotor
splitting for the orientation (Miller, Eleftheriou, Pattnaik, Ndirango, Newns,
Martyna, J. Chem. Phys. 116, 8649 (2002)), with the angular momentum kept in
the body frame, principal axes along the template axes:

  1. v += dt/2 F/M;  L_b += dt/2 R(q)^T tau
  2. p += dt v, wrapped into [0, L)
  3. free rotation about body axes 3, 2, 1, 2, 3 for dt/2, dt/2, dt, dt/2,
     dt/2: phi = h L_b,k / I_k;  q <- q (x) (cos phi/2, sin phi/2 e_k);
     L_b <- Rot_k(-phi) L_b;  then q <- q/|q|
  4. F, tau at the new configuration
  5. v += dt/2 F/M;  L_b += dt/2 R(q)^T tau

Nose-Hoover NVT (paper, Results: the bead-form runs keep the temperature with
a Nose-Hoover thermostat at dt = 0.005; no equations are given).  Reading:
one thermostat variable xi acts on every translational and rotational
degree of freedom,
  dv/dt = F/M - xi v,   dL_b/dt = tau_b - w x L_b - xi L_b,
  dxi/dt = (2K - g kT) / Q,   d eta/dt = xi,
with K the total (translational + rotational) kinetic energy, g = 6N - 3
(the centre-of-mass momentum stays zero), Q = g kT tau_T^2 for a thermostat
period tau_T.  H' = E_pot + K + Q xi^2/2 + g kT eta is conserved.  The step
is the time-reversible Trotter split
  T(dt/2) . [steps 1-5 above] . T(dt/2),
  T(h): xi += h/2 G(K);  s = exp(-xi h);  v, L_b *= s;  K *= s^2;
        eta += xi h;  xi += h/2 G(K),       G(K) = (2K - g kT) / Q.
Image counters (whole box lengths crossed, for unwrapped positions) are kept
when the state carries them.
"""
from __future__ import annotations

import numpy as np

from . import bodies


def rotate_free(q, Lb, inertia, dt):
    """Step 3: the NO_SQUISH free-rotor sequence for one full step."""
    q = np.array(q, dtype=np.float64)
    Lb = np.array(Lb, dtype=np.float64)
    I = np.asarray(inertia, dtype=np.float64)
    for k, h in ((2, 0.5 * dt), (1, 0.5 * dt), (0, dt), (1, 0.5 * dt), (2, 0.5 * dt)):
        phi = h * Lb[:, k] / I[k]
        rq = np.zeros((len(q), 4))
        rq[:, 0] = np.cos(0.5 * phi)
        rq[:, 1 + k] = np.sin(0.5 * phi)
        q = bodies.qmul(q, rq)
        # L_b rotates by -phi about body axis k
        a, b = [(1, 2), (2, 0), (0, 1)][k]
        c, s = np.cos(phi), np.sin(phi)
        La, Lbb = Lb[:, a].copy(), Lb[:, b].copy()
        Lb[:, a] = c * La + s * Lbb
        Lb[:, b] = -s * La + c * Lbb
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q, Lb


def half_kick(vel, Lb, q, F, tau, mass, dt):
    R = bodies.qmatrix(q)
    vel = vel + 0.5 * dt * F / mass
    Lb = Lb + 0.5 * dt * np.einsum("nab,na->nb", R, tau)
    return vel, Lb


def kinetic(vel, Lb, mass, inertia):
    """(translational, rotational) kinetic energy."""
    ke_t = 0.5 * mass * float(np.sum(vel * vel))
    ke_r = float(np.sum(0.5 * Lb * Lb / np.asarray(inertia)[None, :]))
    return ke_t, ke_r


def step(state, force_fn, mass, inertia, box, dt):
    """One velocity-Verlet step.  state = dict(pos, quat, vel, angmom, F, tau
    [, image]); force_fn(pos, quat) -> (F, tau, E_pot).  Returns the new state
    and E_pot."""
    box = np.asarray(box, dtype=np.float64)
    vel, Lb = half_kick(state["vel"], state["angmom"], state["quat"], state["F"], state["tau"],
                        mass, dt)
    pos = state["pos"] + dt * vel
    shift = np.floor(pos / box)
    pos = pos - box * shift
    quat, Lb = rotate_free(state["quat"], Lb, inertia, dt)
    F, tau, E = force_fn(pos, quat)
    vel, Lb = half_kick(vel, Lb, quat, F, tau, mass, dt)
    out = {"pos": pos, "quat": quat, "vel": vel, "angmom": Lb, "F": F, "tau": tau}
    if "image" in state:
        out["image"] = state["image"] + shift
    return out, E


def thermostat_half(vel, Lb, thermo, K, h):
    """T(h) of the Nose-Hoover split: returns scaled vel, L_b, the new
    thermostat dict and the scaled kinetic energy."""
    g_kT = thermo["g"] * thermo["kT"]
    Q = thermo["Q"]
    xi = thermo["xi"] + 0.5 * h * (2.0 * K - g_kT) / Q
    s = np.exp(-xi * h)
    K = K * s * s
    eta = thermo["eta"] + xi * h
    xi = xi + 0.5 * h * (2.0 * K - g_kT) / Q
    return vel * s, Lb * s, dict(thermo, xi=xi, eta=eta), K


def step_nvt(state, force_fn, mass, inertia, box, dt, thermo):
    """One Nose-Hoover NVT step: T(dt/2), the velocity-Verlet step, T(dt/2).
    thermo = dict(xi, eta, kT, Q, g).  Returns the new state, E_pot and the
    new thermostat dict."""
    kt, kr = kinetic(state["vel"], state["angmom"], mass, inertia)
    vel, Lb, thermo, _ = thermostat_half(state["vel"], state["angmom"], thermo, kt + kr, 0.5 * dt)
    st, E = step(dict(state, vel=vel, angmom=Lb), force_fn, mass, inertia, box, dt)
    kt, kr = kinetic(st["vel"], st["angmom"], mass, inertia)
    vel, Lb, thermo, _ = thermostat_half(st["vel"], st["angmom"], thermo, kt + kr, 0.5 * dt)
    return dict(st, vel=vel, angmom=Lb), E, thermo


def thermostat(n_bodies: int, kT: float, tau: float, xi: float = 0.0, eta: float = 0.0):
    """Thermostat dict for n_bodies rigid bodies: g = 6N - 3, Q = g kT tau^2."""
    g = 6.0 * n_bodies - 3.0
    return {"xi": xi, "eta": eta, "kT": kT, "g": g, "Q": g * kT * tau * tau}


def conserved_nvt(E_pot, K, thermo):
    """H' = E_pot + K + Q xi^2 / 2 + g kT eta."""
    return E_pot + K + 0.5 * thermo["Q"] * thermo["xi"] ** 2 + thermo["g"] * thermo["kT"] * thermo["eta"]


def run_nvt(state, force_fn, mass, inertia, box, dt, n_steps, thermo):
    """n_steps of NVT; returns the final state, the thermostat dict and H'
    after each step (index 0 = before the first step)."""
    F, tau, E = force_fn(state["pos"], state["quat"])
    st = dict(state, F=F, tau=tau)
    kt, kr = kinetic(st["vel"], st["angmom"], mass, inertia)
    h = [conserved_nvt(E, kt + kr, thermo)]
    for _ in range(n_steps):
        st, E, thermo = step_nvt(st, force_fn, mass, inertia, box, dt, thermo)
        kt, kr = kinetic(st["vel"], st["angmom"], mass, inertia)
        h.append(conserved_nvt(E, kt + kr, thermo))
    return st, thermo, np.array(h)


def run(state, force_fn, mass, inertia, box, dt, n_steps):
    """n_steps of NVE; returns final state and the total energy after each step
    (index 0 = before the first step)."""
    F, tau, E = force_fn(state["pos"], state["quat"])
    st = dict(state, F=F, tau=tau)
    kt, kr = kinetic(st["vel"], st["angmom"], mass, inertia)
    energies = [E + kt + kr]
    for _ in range(n_steps):
        st, E = step(st, force_fn, mass, inertia, box, dt)
        kt, kr = kinetic(st["vel"], st["angmom"], mass, inertia)
        energies.append(E + kt + kr)
    return st, np.array(energies)
