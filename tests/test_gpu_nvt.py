"""GPU Nose-Hoover NVT (rb_set_thermostat) against the FP64 oracle and its
invariants: each GPU step matches one oracle NVT step started from the GPU's
previous state and thermostat variables; the extended energy H' is conserved
while the plain total energy is not; the temperature settles at the bath's;
an extremely slow thermostat reproduces NVE bit for bit, and switching it off
restores NVE."""
import numpy as np
import pytest

import oracle
from oracle import bodies, md
from paper_2402_12199_gb300 import inputs
from tests.helpers import gpu_system, make_state, rel_err

pytestmark = pytest.mark.gpu
H = inputs.HPHC_PAPER


@pytest.fixture(scope="module", autouse=True)
def _built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()


def test_nvt_shadow_20_steps_64_cubes():
    n, kT, tau, dt = 64, 1.5, 0.05, 0.002
    st, L, tmpl = make_state(n, 0.10, 1, kT=0.6)
    M, I = bodies.mass_and_inertia(tmpl)
    I = np.diag(I)
    box = np.array([L] * 3)
    Rc = bodies.pair_cutoff(tmpl)
    s = gpu_system(st, L)
    s.set_thermostat(kT, tau)
    th = s.thermostat()
    g = 6 * n - 3
    assert th["xi"] == 0.0 and th["eta"] == 0.0
    assert th["Q"] == pytest.approx(g * kT * tau * tau, rel=1e-6)
    assert th["g_kT"] == pytest.approx(g * kT, rel=1e-6)

    def force_fn(pos, quat):
        pairs = oracle.pairs_bruteforce(pos, box, Rc)
        F, T, E, _ = oracle.forces_beads(pos, quat, box, tmpl, pairs)
        return F, T, E

    prev = s.get_state(to_host=True)
    s.forces_beads()
    worst = {"pos": 0.0, "quat": 0.0, "vel": 0.0, "angmom": 0.0, "xi": 0.0, "eta": 0.0}
    for _ in range(20):
        th_prev = s.thermostat()
        s.step(1, dt)
        cur = s.get_state(to_host=True)
        th_cur = s.thermostat()
        st64 = {"pos": prev["pos"][:, :3].astype(np.float64), "quat": prev["quat"].astype(np.float64),
                "vel": prev["vel"][:, :3].astype(np.float64),
                "angmom": prev["angmom"][:, :3].astype(np.float64)}
        F, T, _ = force_fn(st64["pos"], st64["quat"])
        thermo = md.thermostat(n, kT, tau, xi=th_prev["xi"], eta=th_prev["eta"])
        nxt, _, th_o = md.step_nvt(dict(st64, F=F, tau=T), force_fn, M, I, box, dt, thermo)
        dp = cur["pos"][:, :3] - nxt["pos"]
        dp -= L * np.rint(dp / L)
        worst["pos"] = max(worst["pos"], np.abs(dp).max())
        worst["quat"] = max(worst["quat"], np.abs(cur["quat"] - nxt["quat"]).max())
        worst["vel"] = max(worst["vel"], rel_err(cur["vel"][:, :3], nxt["vel"]))
        worst["angmom"] = max(worst["angmom"], rel_err(cur["angmom"][:, :3], nxt["angmom"]))
        worst["xi"] = max(worst["xi"], abs(th_cur["xi"] - th_o["xi"]) / (abs(th_o["xi"]) + 1e-3))
        worst["eta"] = max(worst["eta"], abs(th_cur["eta"] - th_o["eta"]) / (abs(th_o["eta"]) + 1e-5))
        prev = cur
    s.sync()
    assert abs(s.thermostat()["xi"]) > 1e-2  # the thermostat acted
    assert worst["pos"] < 2e-5 and worst["quat"] < 2e-6, worst
    assert worst["vel"] < 1e-5 and worst["angmom"] < 1e-5, worst
    assert worst["xi"] < 1e-5 and worst["eta"] < 1e-5, worst


def _hphc_system(n, kT_start, seed):
    import torch

    from paper_2402_12199_gb300 import api

    st, L, tmpl = make_state(n, 0.16, seed, kT=kT_start)
    s = api.System(n, [L] * 3, "cube", potential="hphc", hphc=H)
    s.set_state(*(torch.from_numpy(np.ascontiguousarray(st[k])).cuda()
                  for k in ("pos", "quat", "vel", "angmom")))
    return s


def test_nvt_conserves_extended_energy_paper_workload():
    """The paper's set-up: half-power half-cosine cubes at phi = 0.16, dt = 0.005."""
    n, kT = 512, 0.5
    s = _hphc_system(n, 1.0, 31)
    s.set_thermostat(kT, 0.5)
    s.forces_beads()

    def extended():
        e, kt, kr = s.energy()
        th = s.thermostat()
        return e + kt + kr, e + kt + kr + 0.5 * th["Q"] * th["xi"] ** 2 + th["g_kT"] * th["eta"]

    e0, h0 = extended()
    s.step(400, 0.005)
    e1, h1 = extended()
    s.sync()
    assert abs(e1 - e0) > 0.05 * abs(e0)  # the bath takes energy out
    assert abs(h1 - h0) < 2e-4 * abs(h0), (h0, h1, e0, e1)


def test_nvt_reaches_the_bath_temperature():
    n, kT = 512, 0.5
    s = _hphc_system(n, 0.25, 32)
    s.set_thermostat(kT, 0.1)
    s.step(1000, 0.005)
    temps = []
    for _ in range(200):
        s.step(10, 0.005)
        _, kt, kr = s.energy()
        temps.append(2 * (kt + kr) / (6 * n - 3))
    s.sync()
    assert np.mean(temps) == pytest.approx(kT, rel=0.05), np.mean(temps)


def test_slow_thermostat_is_nve_bit_for_bit_and_off_restores_nve():
    st, L, tmpl = make_state(300, 0.15, 33)
    a, b, c = gpu_system(st, L), gpu_system(st, L), gpu_system(st, L)
    b.set_thermostat(1.0, 1e6)   # Q so large that exp(-xi h) rounds to 1 in FP32
    c.set_thermostat(1.0, 0.1)
    c.step(5, 0.002)
    c.set_thermostat(1.0, 0.0)   # off
    c.set_state(*(a.get_state()[k] for k in ("pos", "quat", "vel", "angmom")))
    for sys in (a, b, c):
        sys.step(50, 0.002)
    ra, rb, rc = (x.get_state(to_host=True) for x in (a, b, c))
    for k in ("pos", "quat", "vel", "angmom"):
        assert np.array_equal(ra[k], rb[k]), k
        assert np.array_equal(ra[k], rc[k]), k
    assert c.thermostat() == {"xi": 0.0, "eta": 0.0, "Q": 0.0, "g_kT": 0.0}


def test_nvt_checkpoint_restore_continues_bit_for_bit(tmp_path):
    from paper_2402_12199_gb300 import api

    st, L, tmpl = make_state(500, 0.15, 34)
    st = dict(st)
    st["vel"] = st["vel"] * 30.0  # some centres cross the box
    a = gpu_system(st, L)
    a.set_skin(0.3)
    a.set_thermostat(1.2, 0.2)
    a.step(25, 0.002)
    path = tmp_path / "nvt.rbck"
    a.checkpoint(path)
    img_ck = a.images()
    a.step(30, 0.002)
    ref, th_ref, img_ref = a.get_state(to_host=True), a.thermostat(), a.images()
    b = api.System(500, [L] * 3, "cube")
    b.restore(path)
    assert np.array_equal(b.images(), img_ck)
    b.step(30, 0.002)
    got = b.get_state(to_host=True)
    for k in ("pos", "quat", "vel", "angmom"):
        assert np.array_equal(ref[k], got[k]), k
    assert b.thermostat() == th_ref
    assert np.array_equal(b.images(), img_ref)
