"""Bead-sum pairs whose interacting bead pairs sit just inside (or just outside)
the bead cutoff r_c, in the orientations where the bead kernel's column test
is tightest: the farthest bead of body j pointing straight at the end bead of
one of body i's columns (corner to corner for the cube, rim to rim for the
cylinder), plus random orientations at the same smallest bead distance.

The kernel scans only the columns of body i whose segment comes within
r_c + r_circ of body j's centre; a column dropped by mistake removes the whole
interaction of such a pair, so every pair is compared on its own with the FP64
oracle's bead double sum (paper, Methods: U = sum over bead pairs of u), and a
pair just outside r_c must give exactly zero."""
import numpy as np
import pytest

import oracle
from oracle import bodies
from tests.helpers import TOL_F32, assert_parity, template

pytestmark = pytest.mark.gpu
RC = 2.5
DELTA = 2e-3
SPACING = 40.0  # between configurations: far beyond the body-pair cutoff


@pytest.fixture(scope="module", autouse=True)
def _built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()


def _separation(q_i, q_j, direction, target, tmpl, box):
    """Distance t along `direction` at which the smallest bead-bead distance of
    the two bodies is `target` (bisection on the oracle's minimum)."""
    r_circ = float(np.sqrt((tmpl ** 2).sum(1)).max())
    p0 = np.zeros(3) + 0.5 * box
    lo, hi = 0.0, 2.0 * r_circ + RC + 1.0
    f = lambda t: oracle.min_bead_distance(p0, q_i, p0 + t * direction, q_j, box, tmpl)
    assert f(hi) > target
    while f(lo) >= target:  # start inside
        lo -= 1.0
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        if f(mid) < target:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def _configs(shape, seed):
    """(q_i, q_j, direction, target) of every configuration."""
    tmpl = template(shape)
    r = np.sqrt((tmpl ** 2).sum(1))
    far = tmpl[r > r.max() - 1e-9]  # corners / rim beads of the end layers
    ident = np.array([1.0, 0.0, 0.0, 0.0])
    out = []
    for t_a in far:  # bead t_a of i faces bead -t_a of j (the template is centrosymmetric)
        out.append((ident, ident, t_a / np.linalg.norm(t_a), RC - DELTA))
    # (aligned just outside r_c the centres are beyond the pair cutoff: never listed)
    rng = np.random.default_rng(seed)
    for target in (RC - DELTA, RC + DELTA):
        for _ in range(24):
            qi = rng.standard_normal(4)
            qj = rng.standard_normal(4)
            d = rng.standard_normal(3)
            out.append((qi / np.linalg.norm(qi), qj / np.linalg.norm(qj), d / np.linalg.norm(d),
                        target))
    return out


@pytest.mark.parametrize("shape", ["cube", "cylinder"])
def test_pairs_at_the_bead_cutoff(shape):
    import torch

    from paper_2402_12199_gb300 import api

    tmpl = template(shape)
    cfgs = _configs(shape, 11 if shape == "cube" else 12)
    K = len(cfgs)
    g = int(np.ceil(K ** (1 / 3)))
    L = SPACING * g
    box = np.array([L] * 3)
    pos = np.zeros((2 * K, 4), np.float32)
    quat = np.zeros((2 * K, 4), np.float32)
    for k, (qi, qj, d, target) in enumerate(cfgs):
        c = SPACING * (np.array([k % g, (k // g) % g, k // (g * g)]) + 0.25)
        t = _separation(qi, qj, d, target, tmpl, box)
        pos[2 * k, :3] = c
        pos[2 * k + 1, :3] = c + t * d
        quat[2 * k], quat[2 * k + 1] = qi, qj
    pos64 = pos[:, :3].astype(np.float64)
    q64 = quat.astype(np.float64)
    pairs = np.array([[2 * k, 2 * k + 1] for k in range(K)])
    # the FP32 positions the GPU sees keep every configuration on its side of r_c
    inside = np.array([oracle.min_bead_distance(pos64[2 * k], q64[2 * k], pos64[2 * k + 1],
                                                q64[2 * k + 1], box, tmpl) < RC
                       for k in range(K)])
    assert np.array_equal(inside, np.array([c[3] < RC for c in cfgs]))
    F, T, E, _ = oracle.forces_beads(pos64, q64, box, tmpl, pairs)
    s = api.System(2 * K, [L] * 3, shape)
    zeros = torch.zeros((2 * K, 4), dtype=torch.float32, device="cuda")
    s.set_state(torch.from_numpy(pos).cuda(), torch.from_numpy(quat).cuda(), zeros, zeros)
    listed = np.linalg.norm(pos64[1::2] - pos64[0::2], axis=1) < bodies.pair_cutoff(tmpl)
    assert np.all(listed[inside]) and listed[~inside].sum() >= 12  # the outside cases run too
    assert s.build_pairs() == int(listed.sum())
    r = s.forces_beads()
    s.sync()
    got_F = r["force"][:, :3].double().cpu().numpy()
    got_T = r["torque"][:, :3].double().cpu().numpy()
    body_in = np.repeat(inside, 2)
    assert np.all(np.linalg.norm(F[body_in], axis=1) > 1e-3)  # every inside pair interacts
    assert_parity(got_F[body_in], F[body_in], TOL_F32, "force")
    assert_parity(got_T[body_in], T[body_in], TOL_F32, "torque")
    assert np.all(got_F[~body_in] == 0.0) and np.all(got_T[~body_in] == 0.0)
    assert np.all(F[~body_in] == 0.0)
