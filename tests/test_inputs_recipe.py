"""The synthetic input recipe (the generator shared by the oracle and the
GPU tests, holding none of the method's arithmetic) against what it
promises: the packing fraction sets the box, no two bodies start with beads
closer than one bead diameter, orientations are unit quaternions, and the
total momentum is zero.  CPU only."""
import numpy as np
import pytest

import oracle
from oracle import bodies
from paper_2402_12199_gb300 import inputs


@pytest.mark.parametrize("shape,n,phi", [("cube", 64, 0.20), ("cube", 125, 0.25),
                                         ("cylinder", 64, 0.15)])
def test_placement_keeps_beads_apart_and_fills_the_box(shape, n, phi):
    tmpl = bodies.cube_template() if shape == "cube" else bodies.cylinder_template()
    M, I = bodies.mass_and_inertia(tmpl)
    st, L = inputs.system_state(n, phi, 1.0, 7, M, np.diag(I), shape)
    assert L == pytest.approx(inputs.box_length(n, phi, shape))
    pos = st["pos"][:, :3].astype(np.float64)
    quat = st["quat"].astype(np.float64)
    box = np.array([L] * 3)
    assert np.all((pos >= 0) & (pos < L))
    np.testing.assert_allclose(np.linalg.norm(quat, axis=1), 1.0, atol=1e-6)
    pairs = oracle.pairs_bruteforce(pos, box, bodies.pair_cutoff(tmpl))
    dmin = min(oracle.min_bead_distance(pos[i], quat[i], pos[j], quat[j], box, tmpl) for i, j in pairs)
    assert dmin >= 1.0 - 1e-6, dmin


def test_velocities_have_zero_total_momentum_and_the_set_temperature():
    tmpl = bodies.cube_template()
    M, I = bodies.mass_and_inertia(tmpl)
    st, L = inputs.system_state(4096, 0.05, 1.3, 8, M, np.diag(I))
    v = st["vel"][:, :3].astype(np.float64)
    np.testing.assert_allclose(v.sum(0), 0.0, atol=1e-3 * np.abs(v).sum() / len(v))
    kT = M * (v ** 2).sum() / (3 * (len(v) - 1))
    assert kT == pytest.approx(1.3, rel=0.05)
