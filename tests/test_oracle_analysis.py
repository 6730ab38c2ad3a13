"""Pins of the oracle's analyses (oracle/analysis.py) against closed forms:

  * g(r) counts of a periodic simple cubic lattice: N z / 2 pairs in the bins
    of the first four shells (z = 6, 12, 8, 6 at a, sqrt2 a, sqrt3 a, 2a) and
    none elsewhere;
  * g(r) of uniformly scattered centres (ideal gas) is 1 within its
    statistical error, which pins the normalisation;
  * MSD of free ballistic flight across the periodic boundaries is
    <|v|^2> t^2 (pins the image counting of the integrator and the
    unwrapping);
  * MSR of bodies turned by known angles |theta| is <sin^2(|theta| / 2)>,
    the SI Sec. 5 distance of q0 and q0 exp(theta); d is blind to the sign
    of a quaternion, symmetric, 0 for equal and 1 for half-turned bodies.
No GPU.
"""
import numpy as np
import pytest

from oracle import analysis, bodies, md
from paper_2402_12199_gb300 import inputs

CUBE = bodies.cube_template()


def test_gr_counts_simple_cubic_lattice():
    m, a = 6, 3.0
    g = (np.arange(m) + 0.5) * a
    pos = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    N = len(pos)
    rng = np.random.default_rng(1)
    pos = pos[rng.permutation(N)]  # order does not matter
    c = analysis.gr_counts(pos, [m * a] * 3, 6.5, 65)
    expect = np.zeros(65, dtype=np.int64)
    for r, z in ((a, 6), (np.sqrt(2) * a, 12), (np.sqrt(3) * a, 8), (2 * a, 6)):
        expect[int(r * 10)] += N * z // 2
    np.testing.assert_array_equal(c, expect)


def test_gr_edge_counts_find_shells_on_bin_edges():
    """dr = 0.5 puts the lattice's first shell (a = 3) and fourth (2a = 6) on
    bin edges 6 and 12; the second and third (4.24, 5.20) lie 0.24 and 0.20
    from the nearest edges.  A pair exactly on an edge belongs to the bin
    above it."""
    m, a = 6, 3.0
    g = (np.arange(m) + 0.5) * a
    pos = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    N = len(pos)
    e = analysis.gr_edge_counts(pos, [m * a] * 3, 6.5, 13, 1e-6)
    expect = np.zeros(14, dtype=np.int64)
    expect[6] = N * 6 // 2
    expect[12] = N * 6 // 2
    np.testing.assert_array_equal(e, expect)
    assert analysis.gr_edge_counts(pos, [m * a] * 3, 6.5, 13, 0.21)[10] == N * 8 // 2
    c = analysis.gr_counts(pos, [m * a] * 3, 6.5, 13)
    assert c[6] == N * 6 // 2 and c[5] == 0 and c[12] == N * 6 // 2


def test_gr_of_ideal_gas_is_one():
    rng = np.random.default_rng(2)
    N, L = 3000, 40.0
    pos = rng.uniform(0, L, (N, 3))
    r_max, n_bins = 8.0, 32
    c = analysis.gr_counts(pos, [L] * 3, r_max, n_bins)
    g = analysis.gr_normalise(c, r_max, 1, N, L ** 3)
    # shells beyond r = 2 hold hundreds of pairs or more: Poisson error < 7 %
    sel = g[8:]
    assert np.abs(sel - 1).max() < 0.15
    assert abs(np.average(sel, weights=c[8:]) - 1) < 0.02


def _free_state(n, seed, scale_v=1.0, scale_L=1.0):
    M, I = bodies.mass_and_inertia(CUBE)
    st, L = inputs.system_state(n, 0.01, 1.0, seed, M, np.diag(I))
    q = st["quat"].astype(np.float64)
    q /= np.linalg.norm(q, axis=1, keepdims=True)  # exactly unit in FP64
    state = {"pos": st["pos"][:, :3].astype(np.float64), "quat": q,
             "vel": st["vel"][:, :3].astype(np.float64) * scale_v,
             "angmom": st["angmom"][:, :3].astype(np.float64) * scale_L,
             "image": np.zeros((n, 3))}
    return state, M, np.diag(I), np.array([L] * 3)


def test_msd_of_ballistic_flight_across_boundaries():
    state, M, I, box = _free_state(64, 3, scale_v=400.0)
    zero = lambda pos, quat: (np.zeros_like(pos), np.zeros_like(pos), 0.0)
    dt, n = 0.01, 60
    st, _ = md.run(state, zero, M, I, box, dt, n)
    assert np.abs(st["image"]).max() >= 1  # bodies crossed the box
    t = dt * n
    expect = np.mean(np.sum(state["vel"] ** 2, axis=1)) * t * t
    got = analysis.msd(st["pos"], st["image"], state["pos"], state["image"], box)
    assert got == pytest.approx(expect, rel=1e-10)


def test_msr_of_rotations_with_known_angles():
    """Body i turned by the angle |theta_i| about any axis: q = q0 exp(theta),
    so <q0, q> = cos(|theta|/2) and d = sin^2(|theta|/2)."""
    rng = np.random.default_rng(4)
    n = 50
    q0 = rng.standard_normal((n, 4))
    q0 /= np.linalg.norm(q0, axis=1, keepdims=True)
    theta = rng.standard_normal((n, 3)) * 0.8
    q = bodies.qmul(q0, bodies.qexp(theta))
    expect = np.mean(np.sin(0.5 * np.linalg.norm(theta, axis=1)) ** 2)
    assert 0.05 < expect < 0.95
    assert analysis.msr(q, q0) == pytest.approx(expect, rel=1e-12)
    # q and -q are the same orientation; the distance is symmetric
    assert analysis.msr(-q, q0) == pytest.approx(expect, rel=1e-12)
    assert analysis.msr(q0, q) == pytest.approx(expect, rel=1e-12)
    np.testing.assert_allclose(analysis.orientational_distance(q0, q0), 0, atol=1e-15)
    # a half turn gives the largest distance, 1
    assert analysis.orientational_distance(q0[:1], bodies.qmul(q0[:1], bodies.qexp(np.array([[np.pi, 0, 0]]))))[0] == pytest.approx(1.0, abs=1e-15)
