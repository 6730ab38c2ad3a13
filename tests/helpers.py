"""Shared test helpers: build systems from the seeded inputs, run the oracle,
and compute the error metrics: the aggregate relative L2 norm over bodies
(e_F, e_tau) and the element-wise error max_i |a_i - b_i| / max(rms, |b_i|),
which a single wrong body cannot hide under."""
from __future__ import annotations

import numpy as np

import oracle
from oracle import bodies, nn
from paper_2402_12199_gb300 import inputs

TOL_F32 = 1e-5   # FP32 bead and FP32 network paths vs FP64
TOL_BF16 = 2e-2  # BF16 tensor-core network path vs FP64


def rel_err(a, b) -> float:
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / den) if den > 0 else float(np.linalg.norm(a - b))


def max_body_err(a, b) -> float:
    """max_i |a_i - b_i| / max(rms, |b_i|) over the rows i (bodies or pairs) of
    (n, k) arrays, rms = sqrt(mean_i |b_i|^2); a 1-D array is taken as n rows
    of one value.  Rows far larger than the rms (a body in hard contact among
    many in soft contact: the bead forces and torques are heavy-tailed) are
    held to their own magnitude, the others to the rms."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    if a.ndim == 1:
        a, b = a[:, None], b[:, None]
    if len(a) == 0:
        return 0.0
    d = np.sqrt(np.sum((a - b) ** 2, axis=1))
    nb = np.sqrt(np.sum(b * b, axis=1))
    rms = float(np.sqrt(np.mean(nb * nb)))
    if rms == 0.0:
        return float(d.max())
    return float(np.max(d / np.maximum(nb, rms)))


PER_BODY_FACTOR = 10.0  # element-wise bound: max_i |error_i| / max(rms, |ref_i|) <= 10 x tolerance


def assert_parity(got, ref, tol, what=""):
    """Aggregate relative error below `tol` and no row worse than
    PER_BODY_FACTOR x tol relative to max(rms of the reference rows, its own
    reference magnitude)."""
    e = rel_err(got, ref)
    m = max_body_err(got, ref)
    assert e < tol and m < PER_BODY_FACTOR * tol, (what, e, m, tol)
    return e, m


def template(shape: str):
    return bodies.cube_template() if shape == "cube" else bodies.cylinder_template()


def make_state(n, phi, seed, shape="cube", kT=1.0):
    tmpl = template(shape)
    M, I = bodies.mass_and_inertia(tmpl)
    st, L = inputs.system_state(n, phi, kT, seed, M, np.diag(I), shape)
    return st, L, tmpl


def gpu_system(st, L, shape="cube", max_neighbors=0):
    import torch

    from paper_2402_12199_gb300 import api

    s = api.System(len(st["pos"]), [L] * 3, shape, max_neighbors=max_neighbors)
    s.set_state(*(torch.from_numpy(np.ascontiguousarray(st[k])).cuda()
                  for k in ("pos", "quat", "vel", "angmom")))
    return s


def oracle_beads(st, L, tmpl, pairs=None):
    pos = st["pos"][:, :3].astype(np.float64)
    quat = st["quat"].astype(np.float64)
    box = np.array([L] * 3, dtype=np.float64)
    if pairs is None:
        pairs = oracle.pairs_bruteforce(pos, box, bodies.pair_cutoff(tmpl))
    F, T, E, vir = oracle.forces_beads(pos, quat, box, tmpl, pairs)
    return F, T, E, vir, pairs


def oracle_nn(st, L, tmpl, flat, width, depth=3, pairs=None):
    pos = st["pos"][:, :3].astype(np.float64)
    quat = st["quat"].astype(np.float64)
    box = np.array([L] * 3, dtype=np.float64)
    if pairs is None:
        pairs = oracle.pairs_bruteforce(pos, box, bodies.pair_cutoff(tmpl))
    p = nn.unpack(np.asarray(flat, dtype=np.float64), width, depth)
    F, T, E, per = nn.forces_nn(p, pos, quat, box, pairs)
    return F, T, E, per, pairs


def canonical_margin(st, pairs):
    """Smallest |scalar part| of q_i^* q_j over the pairs (FP64), used to skip
    pairs whose canonical sign could flip between FP32 and FP64."""
    if len(pairs) == 0:
        return np.inf
    q = st["quat"].astype(np.float64)
    qr = bodies.qmul(bodies.qconj(q[pairs[:, 0]]), q[pairs[:, 1]])
    return float(np.abs(qr[:, 0]).min())
