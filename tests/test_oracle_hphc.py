"""Pins of the oracle's half-power half-cosine bead potential (paper, Eq. 1)
and of the bead double sum with it, against facts fixed by the mathematics:

  * closed-form values at special arguments (cosine at 0, pi/3, pi/2;
    (b - r)^p at b - r = 1 and 1/4 with p = 5/2);
  * -u'(r)/r equal to central differences of u in both branches;
  * the continuous reading is C1 (value and slope match at r = b and vanish
    at the cutoff b + pi/c); the printed reading jumps by exactly A at r = b
    and ends at the first zero of its cosine, b + pi/(2c);
  * two aligned cubes face to face: the 15625-term double sum collapses to
    729 offset classes with multiplicities (structurally different sum);
  * forces and torques of cube pairs are central differences of the double
    sum's energy, and obey Newton's third law and angular-momentum balance.
No GPU.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import bodies, sampler
from paper_2402_12199_gb300 import inputs

H = inputs.HPHC_PAPER
A, B, C, P = H["A"], H["b"], H["c"], H["p"]
CUBE = bodies.cube_template()
NOBOX = np.zeros(3)
ID = np.array([1.0, 0, 0, 0])


def rand_q(rng):
    q = rng.standard_normal(4)
    return q / np.linalg.norm(q)


@pytest.mark.parametrize("printed", [False, True])
def test_special_values(printed):
    # repulsive branch: (b - r)^p - 2A; 1^p = 1 and (1/4)^(5/2) = 1/32
    assert oracle.hphc(B - 1.0, A, B, C, P, printed)[0] == pytest.approx(1.0 - 2 * A, abs=1e-15)
    assert oracle.hphc(B - 0.25, A, B, C, P, printed)[0] == pytest.approx(1 / 32 - 2 * A, abs=1e-15)
    assert oracle.hphc(B, A, B, C, P, printed)[0] == pytest.approx(-2 * A, abs=1e-18)
    third = B + math.pi / (3 * C)
    if printed:
        # -A cos(pi/3) = -A/2; cut at b + pi/(2c)
        assert oracle.hphc(third, A, B, C, P, True)[0] == pytest.approx(-0.5 * A, rel=1e-12)
        assert oracle.hphc_cutoff(B, C, True) == pytest.approx(B + math.pi / (2 * C), rel=1e-15)
    else:
        # -A (1 + cos(pi/3)) = -3A/2 and -A (1 + cos(pi/2)) = -A; cut at b + pi/c
        assert oracle.hphc(third, A, B, C, P)[0] == pytest.approx(-1.5 * A, rel=1e-12)
        assert oracle.hphc(B + math.pi / (2 * C), A, B, C, P)[0] == pytest.approx(-A, rel=1e-12)
        assert oracle.hphc_cutoff(B, C) == pytest.approx(B + math.pi / C, rel=1e-15)
    rc = oracle.hphc_cutoff(B, C, printed)
    assert oracle.hphc(rc, A, B, C, P, printed) == (0.0, 0.0)
    assert oracle.hphc(rc + 0.3, A, B, C, P, printed) == (0.0, 0.0)


@pytest.mark.parametrize("printed", [False, True])
def test_force_is_minus_derivative(printed):
    rc = oracle.hphc_cutoff(B, C, printed)
    h = 1e-6
    for r in [0.6, 0.9, 1.2, 1.4, B + 0.05, B + 0.3, 0.5 * (B + rc), rc - 0.05]:
        fd = -(oracle.hphc(r + h, A, B, C, P, printed)[0]
               - oracle.hphc(r - h, A, B, C, P, printed)[0]) / (2 * h)
        assert oracle.hphc(r, A, B, C, P, printed)[1] * r == pytest.approx(fd, rel=1e-7, abs=1e-12)


def test_continuous_reading_is_c1():
    rc = oracle.hphc_cutoff(B, C)
    e = 1e-9
    for x in (B, rc):
        lo = oracle.hphc(x - e, A, B, C, P)
        hi = oracle.hphc(x + e, A, B, C, P)
        assert abs(lo[0] - hi[0]) < 1e-12
        # slope vanishes at both joins
        assert abs(lo[1] * x) < 1e-8 and abs(hi[1] * x) < 1e-8
    # a well: decreasing to -2A on (0, b], increasing to 0 on (b, rc)
    r = np.linspace(0.3, rc - 1e-6, 4001)
    u = np.array([oracle.hphc(x, A, B, C, P)[0] for x in r])
    k = np.searchsorted(r, B)
    assert np.all(np.diff(u[:k]) < 0) and np.all(np.diff(u[k + 1:]) > 0)
    assert u.min() >= -2 * A - 1e-15


def test_printed_reading_jumps_by_A():
    e = 1e-12
    below = oracle.hphc(B, A, B, C, P, True)[0]
    above = oracle.hphc(B + e, A, B, C, P, True)[0]
    assert below == pytest.approx(-2 * A, abs=1e-18)
    assert above - below == pytest.approx(A, rel=1e-6)


def test_one_bead_bodies_reduce_to_the_bead_potential():
    one = np.zeros((1, 3))
    pot = oracle.pot_hphc(A, B, C, P)
    rng = np.random.default_rng(0)
    for r in [0.8, 1.3, 1.7, 2.2]:
        d = rng.standard_normal(3)
        d /= np.linalg.norm(d)
        res = oracle.bead_pair(np.zeros(3), rand_q(rng), r * d, rand_q(rng), NOBOX, one, pot=pot)
        u, fr = oracle.hphc(r, A, B, C, P)
        assert res["E"] == pytest.approx(u, abs=1e-16)
        np.testing.assert_allclose(res["F_j"], fr * r * d, atol=1e-15)
        np.testing.assert_allclose(res["tau_i"], 0, atol=1e-16)
        np.testing.assert_allclose(res["tau_j"], 0, atol=1e-16)


def _face_sum(D, printed):
    """Aligned 5x5x5 cubes D apart along x: 729 offset classes with
    multiplicities (5-|dx|)(5-|dy|)(5-|dz|)."""
    rc = oracle.hphc_cutoff(B, C, printed)
    E = Fx = 0.0
    for dx in range(-4, 5):
        for dy in range(-4, 5):
            for dz in range(-4, 5):
                m = (5 - abs(dx)) * (5 - abs(dy)) * (5 - abs(dz))
                x = D + dx
                r = math.sqrt(x * x + dy * dy + dz * dz)
                if r < rc:
                    u, fr = oracle.hphc(r, A, B, C, P, printed)
                    E += m * u
                    Fx += m * fr * x
    return E, Fx


@pytest.mark.parametrize("D,printed", [(5.4, False), (5.9, False), (6.3, False), (5.7, True)])
def test_face_to_face_cubes_lattice_sum(D, printed):
    pot = oracle.pot_hphc(A, B, C, P, printed)
    res = oracle.bead_pair(np.zeros(3), ID, np.array([D, 0, 0]), ID, NOBOX, CUBE, pot=pot)
    E, Fx = _face_sum(D, printed)
    assert res["n_in"] > 0
    assert res["E"] == pytest.approx(E, rel=1e-12, abs=1e-15)
    assert res["F_j"][0] == pytest.approx(Fx, rel=1e-11, abs=1e-15)
    np.testing.assert_allclose(res["F_j"][1:], 0, atol=1e-13)


def test_forces_torques_are_energy_gradients_and_balance():
    pot = oracle.pot_hphc(A, B, C, P)
    rc = oracle.pot_cutoff(pot)
    rng = np.random.default_rng(5)
    for _ in range(3):
        q_i, q_j = rand_q(rng), rand_q(rng)
        d = rng.standard_normal(3)
        d /= np.linalg.norm(d)
        # just outside contact at one sigma, well inside the attraction
        rho = sampler.contact_distance(d, bodies.qmul(bodies.qconj(q_i), q_j), CUBE,
                                       bodies.pair_cutoff(CUBE, rc))
        R = bodies.qrotate(q_i, (rho + 0.2) * d)
        res = oracle.bead_pair(np.zeros(3), q_i, R, q_j, NOBOX, CUBE, pot=pot)
        assert res["n_in"] > 0
        E = lambda pi, qi, pj, qj: oracle.bead_pair(pi, qi, pj, qj, NOBOX, CUBE, pot=pot)["E"]
        h = 1e-5
        scale = max(np.abs(res["F_j"]).max(), np.abs(res["tau_j"]).max(), 1e-6)
        for k in range(3):
            e = np.eye(3)[k]
            fd = -(E(np.zeros(3), q_i, R + h * e, q_j) - E(np.zeros(3), q_i, R - h * e, q_j)) / (2 * h)
            assert res["F_j"][k] == pytest.approx(fd, abs=1e-6 * scale)
            rp, rm = bodies.qexp(h * e), bodies.qexp(-h * e)
            fd_j = -(E(np.zeros(3), q_i, R, bodies.qmul(rp, q_j))
                     - E(np.zeros(3), q_i, R, bodies.qmul(rm, q_j))) / (2 * h)
            fd_i = -(E(np.zeros(3), bodies.qmul(rp, q_i), R, q_j)
                     - E(np.zeros(3), bodies.qmul(rm, q_i), R, q_j)) / (2 * h)
            assert res["tau_j"][k] == pytest.approx(fd_j, abs=1e-6 * scale)
            assert res["tau_i"][k] == pytest.approx(fd_i, abs=1e-6 * scale)
        np.testing.assert_allclose(res["F_i"] + res["F_j"], 0, atol=1e-14 * scale + 1e-18)
        L = res["tau_i"] + res["tau_j"] + np.cross(R, res["F_j"])
        np.testing.assert_allclose(L, 0, atol=1e-12 * scale + 1e-18)
