"""GPU parity of the half-power half-cosine bead potential (paper, Eq. 1; both
readings) against the FP64 oracle: whole-system forces, torques, energy and
virial for the cube (column path), the cylinder (column path, three packed
slot pairs) and a template without columns (generic path), at the paper's
packing fraction 0.16; energy conservation of an NVE run with the
continuous reading."""
import numpy as np
import pytest

import oracle
from oracle import bodies
from paper_2402_12199_gb300 import inputs
from tests.helpers import TOL_F32, assert_parity, make_state, rel_err

pytestmark = pytest.mark.gpu
H = inputs.HPHC_PAPER


@pytest.fixture(scope="module", autouse=True)
def _built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()


def _gpu(st, L, shape, potential, template=None):
    import torch

    from paper_2402_12199_gb300 import api

    s = api.System(len(st["pos"]), [L] * 3, shape, potential=potential, hphc=H, template=template)
    s.set_state(*(torch.from_numpy(np.ascontiguousarray(st[k])).cuda()
                  for k in ("pos", "quat", "vel", "angmom")))
    return s


def _oracle(st, L, tmpl, printed):
    pot = oracle.pot_hphc(H["A"], H["b"], H["c"], H["p"], printed)
    pos = st["pos"][:, :3].astype(np.float64)
    quat = st["quat"].astype(np.float64)
    box = np.array([L] * 3)
    pairs = oracle.pairs_bruteforce(pos, box, bodies.pair_cutoff(tmpl, oracle.pot_cutoff(pot)))
    return oracle.forces_beads(pos, quat, box, tmpl, pairs, pot=pot)


# at phi = 0.16 few bead pairs reach the repulsive branch and the forces are
# sums of small attractive terms that largely cancel; phi = 0.25 (bodies one
# bead gap apart at the start) gives contact forces as well
@pytest.mark.parametrize("shape,n,printed,phi", [("cube", 1000, False, 0.16), ("cube", 1000, False, 0.25),
                                                 ("cube", 1000, True, 0.25),
                                                 ("cylinder", 400, False, 0.16)])
def test_hphc_system_parity(shape, n, printed, phi):
    st, L, tmpl = make_state(n, phi, 21 + n, shape)
    s = _gpu(st, L, shape, "hphc_printed" if printed else "hphc")
    rc = oracle.hphc_cutoff(H["b"], H["c"], printed)
    assert s.pair_cutoff == pytest.approx(2 * bodies.circumradius(tmpl) + rc, rel=1e-6)
    res = s.forces_beads(energy=True, virial=True)
    s.sync()
    F, T, E, vir = _oracle(st, L, tmpl, printed)
    assert np.abs(F).max() > 0
    assert_parity(res["force"][:, :3].double().cpu().numpy(), F, TOL_F32)
    assert_parity(res["torque"][:, :3].double().cpu().numpy(), T, TOL_F32)
    assert res["energy"] == pytest.approx(E, rel=TOL_F32)
    assert rel_err(res["virial"], vir) < TOL_F32


def test_hphc_generic_template_parity():
    """A 3 x 4 x 6 box of beads has no 5- or 8-bead columns: the generic path."""
    box_t = np.stack(np.meshgrid(np.arange(3) - 1.0, np.arange(4) - 1.5, np.arange(6) - 2.5,
                                 indexing="ij"), -1).reshape(-1, 3)
    M, I = bodies.mass_and_inertia(box_t)
    rc_box = bodies.circumradius(box_t)
    n, phi = 300, 0.16
    L = (n * 72.0 / phi) ** (1 / 3)
    rng = np.random.default_rng(5)
    pos = inputs.place_bodies(n, L, rc_box, rng)
    st = {"pos": np.concatenate([pos, np.zeros((n, 1))], 1).astype(np.float32),
          "quat": inputs.random_quaternions(n, rng).astype(np.float32),
          "vel": np.zeros((n, 4), np.float32), "angmom": np.zeros((n, 4), np.float32)}
    s = _gpu(st, L, "custom", "hphc", template=box_t)
    res = s.forces_beads(energy=True)
    s.sync()
    F, T, E, _ = _oracle(st, L, box_t, False)
    assert np.abs(F).max() > 0
    assert_parity(res["force"][:, :3].double().cpu().numpy(), F, TOL_F32)
    assert_parity(res["torque"][:, :3].double().cpu().numpy(), T, TOL_F32)
    assert res["energy"] == pytest.approx(E, rel=TOL_F32)


def test_hphc_nve_conserves_energy():
    from paper_2402_12199_gb300 import api

    st, L, tmpl = make_state(512, 0.16, 9, "cube", kT=0.5)
    s = _gpu(st, L, "cube", "hphc")
    s.forces_beads()
    e0 = sum(s.energy())
    s.step(400, 0.005, path=api.RB_PATH_BEADS)
    e1 = sum(s.energy())
    s.sync()
    assert np.isfinite(e1) and abs(e1 - e0) < 1e-3 * 512 * 0.5, (e0, e1)
