"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module draws inputs only.  It holds none of the method's arithmetic (no
bead potential, no rotation of bead templates, no network, no integrator), so
that the CUDA library and the independent oracle can both consume the same
draws without sharing any of the computation they are checked on.

Workload recipe (readings of the paper's set-up; the paper states the packing
fraction phi = N V_particle / V but not V_particle):
  * cube: 5 x 5 x 5 beads at 1 sigma, V_particle = (5 sigma)^3 = 125 sigma^3,
    bead-centre circumradius 2 sqrt(3) sigma;
  * cylinder: 8 layers of 19 hexagonally packed beads (152), bead-centre
    radius 2 sigma and length 8 sigma, V_particle = pi 2.5^2 9 sigma^3,
    bead-centre circumradius sqrt(20) sigma;
  * cubic periodic box of side L = (N V_particle / phi)^(1/3);
  * centres on a simple-cubic lattice (face-centred cubic when the simple-cubic
    spacing is too tight) in a seeded shuffled order, jittered so that no two
    circumscribed spheres plus 1 sigma overlap, i.e. no two beads of
    different bodies start closer than 1 sigma;
  * orientations uniform (normalised 4-D Gaussians);
  * velocities Maxwell at kT: v ~ N(0, kT/M) per component with the total
    momentum removed, body-frame angular momentum L_k ~ N(0, kT I_k).
"""
from __future__ import annotations

import math

import numpy as np

SHAPES = {
    "cube": {"v_particle": 125.0, "r_circ": 2.0 * math.sqrt(3.0), "n_beads": 125},
    "cylinder": {"v_particle": math.pi * 2.5 ** 2 * 9.0, "r_circ": math.sqrt(20.0),
                 "n_beads": 152},
}


# The paper's half-power half-cosine bead parameters (Eq. 1 and the text
# after it; units eps, sigma): well depth 2A, minimum at b, cosine rate c,
# repulsive power p.  Its cube workload runs at phi = 0.16 with a
# Nose-Hoover thermostat and dt = 0.005.
HPHC_PAPER = {"A": 0.00035, "b": 1.46375, "c": 3.3833, "p": 2.5}


def box_length(n_bodies: int, phi: float, shape: str = "cube") -> float:
    return (n_bodies * SHAPES[shape]["v_particle"] / phi) ** (1.0 / 3.0)


def _lattice(n: int, L: float, d_min: float):
    m = int(math.ceil(n ** (1.0 / 3.0) - 1e-9))
    a = L / m
    if a >= d_min:
        g = (np.arange(m) + 0.5) * a
        sites = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
        return sites, a
    m = int(math.ceil((n / 4.0) ** (1.0 / 3.0) - 1e-9))
    a = L / m
    base = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]]) + 0.25
    g = np.arange(m)
    cells = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    sites = ((cells[:, None, :] + base[None, :, :]) * a).reshape(-1, 3)
    return sites, a / math.sqrt(2.0)


def place_bodies(n: int, L: float, r_circ: float, rng: np.random.Generator,
                 gap: float = 1.0) -> np.ndarray:
    d_min = 2.0 * r_circ + gap
    sites, spacing = _lattice(n, L, d_min)
    if spacing < d_min:
        raise ValueError(f"cannot place {n} bodies of circumradius {r_circ} in a box of "
                         f"side {L:.3f} with a {gap} sigma gap (lattice spacing {spacing:.3f})")
    order = rng.permutation(len(sites))[:n]
    pos = sites[order]
    delta = max(0.0, 0.5 * (spacing - d_min))
    pos = pos + rng.uniform(-delta, delta, size=pos.shape)
    return np.mod(pos, L)


def random_quaternions(n: int, rng: np.random.Generator) -> np.ndarray:
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q


def velocities(n: int, mass: float, inertia, kT: float, rng: np.random.Generator):
    v = rng.standard_normal((n, 3)) * math.sqrt(kT / mass)
    if n > 1:
        v -= v.mean(axis=0, keepdims=True)
    I = np.asarray(inertia, dtype=np.float64).reshape(3)
    Lb = rng.standard_normal((n, 3)) * np.sqrt(kT * I)[None, :]
    return v, Lb


def system_state(n: int, phi: float, kT: float, seed: int, mass: float, inertia,
                 shape: str = "cube"):
    """Initial state of one system as float32 float4 rows (N, 4):
    pos (x, y, z, 0), quat (s, i, j, k), vel (vx, vy, vz, 0),
    angmom (body-frame L, 0); plus the box side."""
    rng = np.random.default_rng(seed)
    L = box_length(n, phi, shape)
    pos = place_bodies(n, L, SHAPES[shape]["r_circ"], rng)
    q = random_quaternions(n, rng)
    v, Lb = velocities(n, mass, inertia, kT, rng)
    f4 = lambda a3: np.concatenate([a3, np.zeros((n, 1))], 1).astype(np.float32)
    st = {"pos": f4(pos), "quat": q.astype(np.float32), "vel": f4(v), "angmom": f4(Lb)}
    # positions are wrapped into [0, L) in float32 as well
    st["pos"][:, :3] = np.where(st["pos"][:, :3] >= np.float32(L), np.float32(0.0),
                                st["pos"][:, :3])
    return st, float(np.float32(L))


def sampler_uniforms(n: int, seed: int) -> np.ndarray:
    """Six uniforms in [0, 1) per training sample (direction, orientation,
    separation), float32."""
    rng = np.random.default_rng(seed)
    return rng.random((n, 6), dtype=np.float32)


def pair_configs(n: int, seed: int, rho_min: float, rho_max: float) -> np.ndarray:
    """Random pair configurations (s, q_rel) in the frame of body i: separation
    uniform in [rho_min, rho_max) along a uniform direction, uniform q_rel."""
    rng = np.random.default_rng(seed)
    d = rng.standard_normal((n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    rho = rng.uniform(rho_min, rho_max, size=(n, 1))
    q = random_quaternions(n, rng)
    return np.concatenate([d * rho, q], 1).astype(np.float32)


def mlp_params(width: int, depth: int = 3, seed: int = 0, n_in: int = 10,
               mu=None, inv_sd=None, e_scale: float = 1.0, e_shift: float = 0.0,
               gain: float = 1.0) -> np.ndarray:
    """Random flat parameter vector (float32) in the library's layout:
    mu, inv_sd, W1, b1, (W_l, b_l) for l = 2..depth, w_o, b_o, e_scale,
    e_shift.  Weights ~ N(0, gain^2 / fan_in); biases ~ N(0, 0.1^2)."""
    rng = np.random.default_rng(seed)
    mu = np.zeros(n_in) if mu is None else np.asarray(mu, dtype=np.float64)
    inv_sd = np.ones(n_in) if inv_sd is None else np.asarray(inv_sd, dtype=np.float64)
    parts = [mu, inv_sd]
    fan = n_in
    for _ in range(depth):
        parts.append(rng.standard_normal(width * fan) * gain / math.sqrt(fan))
        parts.append(rng.standard_normal(width) * 0.1)
        fan = width
    parts.append(rng.standard_normal(width) * gain / math.sqrt(width))
    parts.append(rng.standard_normal(1) * 0.1)
    parts.append([e_scale, e_shift])
    return np.concatenate([np.asarray(p, dtype=np.float64).ravel() for p in parts]).astype(
        np.float32)


def feature_normalisation(rho_min: float, rho_max: float):
    """Fixed (mu, inv_sd) for the 10 features when pairs are drawn with rho
    uniform in [rho_min, rho_max): s components and quaternion components
    centred on 0 (q_s on 0.5), rho terms on their uniform-distribution moments."""
    r = np.linspace(rho_min, rho_max, 4097)
    feats = [r, 1.0 / r, r * r]
    mu = [0.0, 0.0, 0.0, 0.5, 0.0, 0.0, 0.0] + [float(f.mean()) for f in feats]
    sd = [rho_max / math.sqrt(5.0)] * 3 + [0.3, 0.5, 0.5, 0.5] + [float(f.std()) for f in feats]
    return np.array(mu), 1.0 / np.array(sd)
