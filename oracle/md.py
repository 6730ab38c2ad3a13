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
    """One velocity-Verlet step.  state = dict(pos, quat, vel, angmom, F, tau);
    force_fn(pos, quat) -> (F, tau, E_pot).  Returns the new state and E_pot."""
    box = np.asarray(box, dtype=np.float64)
    vel, Lb = half_kick(state["vel"], state["angmom"], state["quat"], state["F"], state["tau"],
                        mass, dt)
    pos = state["pos"] + dt * vel
    pos = pos - box * np.floor(pos / box)
    quat, Lb = rotate_free(state["quat"], Lb, inertia, dt)
    F, tau, E = force_fn(pos, quat)
    vel, Lb = half_kick(vel, Lb, quat, F, tau, mass, dt)
    return {"pos": pos, "quat": quat, "vel": vel, "angmom": Lb, "F": F, "tau": tau}, E


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
