"""A client that keeps the whole velocity-Verlet state on the host (centres,
orientations, momenta and the forces at the current centres: rb_get_state /
rb_get_forces out, rb_set_state / rb_set_forces back in, every step) runs the
same trajectory bit for bit as an uninterrupted rb_step loop; the forces
given back are the ones the next half kick uses, and forces given for
another path or precision are ignored (evaluated again)."""
import numpy as np
import pytest

from tests.helpers import make_state

pytestmark = pytest.mark.gpu
DT = 0.002


@pytest.fixture(scope="module", autouse=True)
def _built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()


def _system(st, L):
    import torch

    from paper_2402_12199_gb300 import api

    s = api.System(len(st["pos"]), [L] * 3, "cube", skin=0.4)
    s.set_state(*(torch.from_numpy(np.ascontiguousarray(st[k])).cuda()
                  for k in ("pos", "quat", "vel", "angmom")))
    return s


def _cfg(kind):
    from paper_2402_12199_gb300 import api, inputs
    from oracle import bodies, symmetry

    if kind == "beads":
        return dict(path=api.RB_PATH_BEADS)
    mu, isd = inputs.feature_normalisation(5.0, 9.43)
    m = api.MLP(128, 3)
    m.set_params(inputs.mlp_params(128, 3, 9, mu=mu, inv_sd=isd, e_scale=0.5))
    q, inv = symmetry.point_group(bodies.cube_template())
    m.set_symmetry(q.astype(np.float32), inv)
    m.set_cutoff(8.43, 9.43)
    return dict(path=api.RB_PATH_NN, mlp=m, precision=kind)


def _host_round_trip(s, cfg, forces=None):
    st = s.get_state(to_host=True)
    F, T = s.get_forces(to_host=True)
    s.set_state(*(st[k] for k in ("pos", "quat", "vel", "angmom")))
    if forces is not None:
        F, T = forces
    s.set_forces(F, T, **cfg)


@pytest.mark.parametrize("kind", ["beads", "bf16", "f16x3"])
def test_round_trip_is_bit_identical(kind):
    import torch

    st, L, _ = make_state(1500, 0.20, 31)
    cfg = _cfg(kind)
    a, b = _system(st, L), _system(st, L)
    a.step(4, DT, **cfg)
    b.step(1, DT, **cfg)
    for _ in range(3):
        _host_round_trip(b, cfg)
        b.step(1, DT, **cfg)
    sa, sb = a.get_state(), b.get_state()
    for k in ("pos", "quat", "vel", "angmom"):
        assert torch.equal(sa[k], sb[k]), k
    fa, fb = a.get_forces(), b.get_forces()
    assert torch.equal(fa[0], fb[0]) and torch.equal(fa[1], fb[1])


def test_given_forces_are_used_and_others_ignored():
    import torch

    st, L, _ = make_state(1500, 0.20, 32)
    cfg = _cfg("bf16")
    ref = _system(st, L)
    ref.step(2, DT, **cfg)
    zero = (torch.zeros((1500, 4)), torch.zeros((1500, 4)))
    # zero forces for this path: the first half kick uses them, so the velocities differ
    b = _system(st, L)
    b.step(1, DT, **cfg)
    _host_round_trip(b, cfg, forces=zero)
    b.step(1, DT, **cfg)
    assert not torch.equal(ref.get_state()["vel"], b.get_state()["vel"])
    # the same zeros given for another precision are evaluated again: same as the reference
    c = _system(st, L)
    c.step(1, DT, **cfg)
    st_c = c.get_state(to_host=True)
    c.set_state(*(st_c[k] for k in ("pos", "quat", "vel", "angmom")))
    c.set_forces(*zero, path=cfg["path"], mlp=cfg["mlp"], precision="f16x3")
    c.step(1, DT, **cfg)
    for k in ("pos", "quat", "vel", "angmom"):
        assert torch.equal(ref.get_state()[k], c.get_state()[k]), k


def test_set_forces_refuses_bad_arguments():
    import torch

    from paper_2402_12199_gb300 import api

    st, L, _ = make_state(64, 0.10, 33)
    s = _system(st, L)
    F = torch.zeros((64, 4), device="cuda")
    with pytest.raises(api.RBError):
        s.set_forces(F, F, path=7)
    with pytest.raises(api.RBError):
        s.set_forces(F, F, path=api.RB_PATH_NN, mlp=None, precision="bf16")
    with pytest.raises(ValueError):
        s.set_forces(F, torch.zeros((64, 4)))


@pytest.mark.parametrize("copies", [False, True])
@pytest.mark.parametrize("kind", ["beads", "bf16"])
def test_step_host_state_matches_the_uninterrupted_run(kind, copies):
    import torch

    keys = ("pos", "quat", "vel", "angmom")
    st, L, _ = make_state(1500, 0.20, 34)
    cfg = _cfg(kind)
    a, b = _system(st, L), _system(st, L)
    a.step(4, DT, **cfg)
    b.step(1, DT, **cfg)
    blk = torch.empty((6, 1500, 4), dtype=torch.float32).pin_memory()
    b.get_state(to_host=True, out={k: blk[i] for i, k in enumerate(keys)})
    b.get_forces(to_host=True, out=(blk[4], blk[5]))
    for _ in range(3):
        b.step_host_state(blk, 1, DT, copies=copies, **cfg)
    sa = a.get_state()
    fa = a.get_forces()
    for i, k in enumerate(keys):
        assert torch.equal(sa[k].cpu(), blk[i]), k
    assert torch.equal(fa[0].cpu(), blk[4]) and torch.equal(fa[1].cpu(), blk[5])
    # the device side holds the same state and forces as the block
    sb, fb = b.get_state(), b.get_forces()
    for i, k in enumerate(keys):
        assert torch.equal(sb[k].cpu(), blk[i]), k
    assert torch.equal(fb[0].cpu(), blk[4]) and torch.equal(fb[1].cpu(), blk[5])
    with pytest.raises(ValueError):
        b.step_host_state(blk[:5], 1, DT, **cfg)


def test_step_host_state_with_thermostat_matches_the_uninterrupted_run():
    """With a thermostat the call takes the copy form (the direct form is for
    NVE steps); the trajectory is that of rb_step to rounding: handing the
    momenta back makes the thermostat take the kinetic energy from them again
    (an FP64 sum of the FP32 momenta, where the uninterrupted run carries the
    value its last half step scaled), which may differ in the last bits."""
    import torch

    keys = ("pos", "quat", "vel", "angmom")
    st, L, _ = make_state(1200, 0.18, 35)
    cfg = _cfg("beads")
    a, b = _system(st, L), _system(st, L)
    for s in (a, b):
        s.set_thermostat(1.0, 0.5)
    a.step(4, DT, **cfg)
    b.step(1, DT, **cfg)
    blk = torch.empty((6, 1200, 4), dtype=torch.float32).pin_memory()
    b.get_state(to_host=True, out={k: blk[i] for i, k in enumerate(keys)})
    b.get_forces(to_host=True, out=(blk[4], blk[5]))
    for _ in range(3):
        b.step_host_state(blk, 1, DT, **cfg)
    sa = a.get_state()
    for i, k in enumerate(keys):
        ref = sa[k].cpu().double()
        d = float((blk[i].double() - ref).abs().max())
        assert d <= 1e-5 * float(ref.abs().max()), (k, d)
