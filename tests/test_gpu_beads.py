"""GPU parity of the bead-sum path (cell list, pair list, bead kernel,
reduction) and the integrator against the FP64 oracle, through the C ABI."""
import numpy as np
import pytest

import oracle
from oracle import bodies, md
from tests.helpers import (TOL_F32, assert_parity, gpu_system, make_state, oracle_beads, rel_err,
                           template)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()


@pytest.mark.parametrize("shape", ["cube", "cylinder"])
def test_body_template_and_inertia_match_oracle(shape):
    st, L, tmpl = make_state(8, 0.05, 1, shape)
    s = gpu_system(st, L, shape)
    got = s.template().astype(np.float64)
    key = lambda a: a[np.lexsort(np.round(a, 5).T[::-1])]
    np.testing.assert_allclose(key(got), key(tmpl), atol=1e-6)
    M, I = bodies.mass_and_inertia(tmpl)
    assert s.mass == pytest.approx(M)
    np.testing.assert_allclose(s.inertia, np.diag(I), rtol=1e-6)
    assert s.pair_cutoff == pytest.approx(bodies.pair_cutoff(tmpl), rel=1e-6)


@pytest.mark.parametrize("n,phi,seed", [(64, 0.10, 1), (4096, 0.20, 7), (1000, 0.25, 8)])
def test_pair_list_matches_bruteforce(n, phi, seed):
    st, L, tmpl = make_state(n, phi, seed)
    s = gpu_system(st, L)
    m = s.build_pairs()
    got = {tuple(p) for p in s.pairs().tolist()}
    assert len(got) == m
    pos = st["pos"][:, :3].astype(np.float64)
    Rc = bodies.pair_cutoff(tmpl)
    ref = {tuple(p) for p in oracle.pairs_bruteforce(pos, [L] * 3, Rc).tolist()}
    # pairs within FP32 rounding of the cutoff may legitimately differ
    diff = got ^ ref
    for i, j in diff:
        d = pos[j] - pos[i]
        d -= L * np.rint(d / L)
        assert abs(np.linalg.norm(d) - Rc) < 1e-4, (i, j, np.linalg.norm(d))
    assert all(i < j for i, j in got)
    assert len(ref) > 0


def _parity(st, L, tmpl, shape, tol=TOL_F32):
    s = gpu_system(st, L, shape)
    res = s.forces_beads(energy=True, virial=True)
    s.sync()
    F, T, E, vir, pairs = oracle_beads(st, L, tmpl)
    Fg = res["force"][:, :3].double().cpu().numpy()
    Tg = res["torque"][:, :3].double().cpu().numpy()
    eF, _ = assert_parity(Fg, F, tol, "force")
    eT, _ = assert_parity(Tg, T, tol, "torque")
    # energy: relative to the sum of |pair energies|
    pp = oracle.forces_beads(st["pos"][:, :3], st["quat"], [L] * 3, tmpl, pairs,
                             per_pair=True)[4]
    scale = np.abs(pp[:, 0]).sum()
    assert abs(res["energy"] - E) <= tol * max(scale, 1e-12), (res["energy"], E)
    assert rel_err(res["virial"], vir) < tol
    # per-body energy halves sum to the total
    assert abs(res["force"][:, 3].double().sum().item() - E) <= 1e-4 * max(scale, 1.0)
    return eF, eT, len(pairs)


def test_bead_forces_parity_64_cubes():
    st, L, tmpl = make_state(64, 0.10, 1)
    eF, eT, m = _parity(st, L, tmpl, "cube")
    assert m >= 20


def test_bead_forces_parity_ragged_dense_cubes():
    st, L, tmpl = make_state(777, 0.25, 9)
    _parity(st, L, tmpl, "cube")


def test_bead_forces_parity_cylinders():
    st, L, tmpl = make_state(300, 0.15, 4, "cylinder")
    _parity(st, L, tmpl, "cylinder")


def test_bead_forces_parity_custom_template():
    """A 3 x 4 x 6 box of beads: its (x, y) columns hold 6 beads, so the pair
    kernel takes its any-template path (the cube and cylinder take the
    column-shared test)."""
    import torch

    from paper_2402_12199_gb300 import api

    g = np.stack(np.meshgrid(np.arange(3) - 1.0, np.arange(4) - 1.5, np.arange(6) - 2.5,
                             indexing="ij"), -1).reshape(-1, 3)
    st, L, _ = make_state(300, 0.20, 31)
    s = api.System(300, [L] * 3, "custom", template=g)
    s.set_state(*(torch.from_numpy(np.ascontiguousarray(st[k])).cuda()
                  for k in ("pos", "quat", "vel", "angmom")))
    res = s.forces_beads(energy=True)
    s.sync()
    F, T, E, _, pairs = oracle_beads(st, L, g)
    assert len(pairs) > 50
    assert_parity(res["force"][:, :3].double().cpu().numpy(), F, TOL_F32, "force")
    assert_parity(res["torque"][:, :3].double().cpu().numpy(), T, TOL_F32, "torque")


def test_bead_forces_sampled_32768_cubes():
    """Full bench size (32768 cubes, phi = 0.20): every pair of 40 sampled
    bodies recomputed by the oracle; forces/torques on those bodies compared."""
    st, L, tmpl = make_state(32768, 0.20, 3)
    s = gpu_system(st, L)
    res = s.forces_beads()
    s.sync()
    rng = np.random.default_rng(0)
    idx = rng.choice(32768, 40, replace=False)
    pos = st["pos"][:, :3].astype(np.float64)
    Rc = bodies.pair_cutoff(tmpl)
    pairs = set()
    for i in idx:
        d = pos - pos[i]
        d -= L * np.rint(d / L)
        for j in np.nonzero((d ** 2).sum(1) < Rc * Rc)[0]:
            if j != i:
                pairs.add((min(i, j), max(i, j)))
    pairs = np.array(sorted(pairs), dtype=np.int64)
    F, T, E, _ = oracle.forces_beads(pos, st["quat"], [L] * 3, tmpl, pairs)
    Fg = res["force"][:, :3].double().cpu().numpy()[idx]
    Tg = res["torque"][:, :3].double().cpu().numpy()[idx]
    assert_parity(Fg, F[idx], TOL_F32, "force")
    assert_parity(Tg, T[idx], TOL_F32, "torque")
    n_pairs = s.build_pairs()
    assert 60000 < n_pairs < 200000


@pytest.mark.parametrize("shape,n,phi,seed", [("cube", 4096, 0.20, 13), ("cylinder", 1500, 0.15, 14)])
def test_kinetic_energies_match_oracle(shape, n, phi, seed):
    """rb_energy's translational and rotational kinetic energies (FP64 sums on
    the device) equal the oracle's sum(M |v|^2 / 2) and sum(L_b,k^2 / 2 I_k)
    on the same state, after a few steps so that v and L_b are not the
    initial draw; FP64 sums in different orders agree to ~N x 1e-16.  The
    system holds its principal moments in FP32 (the cylinder's are not
    representable exactly), so the oracle takes the same FP32 values, the
    moments the dynamics run with."""
    st, L, tmpl = make_state(n, phi, seed, shape)
    M, I = bodies.mass_and_inertia(tmpl)
    s = gpu_system(st, L, shape)
    s.step(5, 0.002)
    _, ke_t, ke_r = s.energy()
    cur = s.get_state(to_host=True)
    s.sync()
    I32 = np.diag(I).astype(np.float32).astype(np.float64)
    ref_t, ref_r = md.kinetic(cur["vel"][:, :3].astype(np.float64),
                              cur["angmom"][:, :3].astype(np.float64), M, I32)
    assert ke_t == pytest.approx(ref_t, rel=1e-12)
    assert ke_r == pytest.approx(ref_r, rel=1e-12)
    assert ref_t > 0 and ref_r > 0


def test_edge_cases():
    from paper_2402_12199_gb300 import api

    tmpl = template("cube")
    M, I = bodies.mass_and_inertia(tmpl)
    # one body: no pairs, zero force
    st = {"pos": np.array([[5.0, 5, 5, 0]], np.float32), "quat": np.array([[1.0, 0, 0, 0]], np.float32),
          "vel": np.zeros((1, 4), np.float32), "angmom": np.zeros((1, 4), np.float32)}
    s = gpu_system(st, 30.0)
    r = s.forces_beads(energy=True)
    assert r["energy"] == 0.0 and float(r["force"].abs().max()) == 0.0
    assert s.build_pairs() == 0
    # two bodies, far apart (periodic image included): no pair
    st2 = {k: np.repeat(v, 2, axis=0) for k, v in st.items()}
    st2["pos"][1, :3] = [5.0 + 15.0, 5.0, 5.0]
    s = gpu_system(st2, 30.0)
    r = s.forces_beads(energy=True)
    assert r["energy"] == 0.0
    # two bodies in face contact across the periodic boundary
    st2["pos"][0, :3] = [0.5, 5.0, 5.0]
    st2["pos"][1, :3] = [30.0 - 5.3, 5.0, 5.0]
    s = gpu_system(st2, 30.0)
    r = s.forces_beads(energy=True)
    F, T, E, _, pairs = oracle_beads(st2, 30.0, tmpl)
    assert len(pairs) == 1 and E != 0.0
    assert_parity(r["force"][:, :3].double().cpu().numpy(), F, TOL_F32)
    assert r["energy"] == pytest.approx(E, rel=TOL_F32)
    # invalid box: smaller than 2 Rc
    with pytest.raises(api.RBError) as ei:
        api.System(2, [10.0] * 3, "cube")
    assert ei.value.status == 1
    # neighbour capacity overflow is reported, not silently truncated
    st3, L3, _ = make_state(512, 0.25, 2)
    s = gpu_system(st3, L3, max_neighbors=2)
    with pytest.raises(api.RBError) as ei:
        s.build_pairs()
    assert ei.value.status == 4


def test_bead_forces_are_deterministic():
    st, L, tmpl = make_state(2000, 0.2, 5)
    s = gpu_system(st, L)
    a = s.forces_beads(energy=True)
    b = s.forces_beads(energy=True)
    s.sync()
    assert bool((a["force"] == b["force"]).all()) and bool((a["torque"] == b["torque"]).all())
    assert a["energy"] == b["energy"]


def test_nve_shadow_20_steps_64_cubes():
    """Each GPU step is compared with one oracle step started from the GPU's
    previous state; the FP64 total energy stays within the drift bound."""
    st, L, tmpl = make_state(64, 0.10, 1)
    M, I = bodies.mass_and_inertia(tmpl)
    I = np.diag(I)
    box = np.array([L] * 3)
    Rc = bodies.pair_cutoff(tmpl)
    s = gpu_system(st, L)
    dt = 0.002

    def force_fn(pos, quat):
        pairs = oracle.pairs_bruteforce(pos, box, Rc)
        F, T, E, _ = oracle.forces_beads(pos, quat, box, tmpl, pairs)
        return F, T, E

    prev = s.get_state(to_host=True)
    s.forces_beads()
    e0 = sum(s.energy())
    worst = {"pos": 0.0, "quat": 0.0, "vel": 0.0, "angmom": 0.0}
    for _ in range(20):
        s.step(1, dt)
        cur = s.get_state(to_host=True)
        st64 = {"pos": prev["pos"][:, :3].astype(np.float64), "quat": prev["quat"].astype(np.float64),
                "vel": prev["vel"][:, :3].astype(np.float64), "angmom": prev["angmom"][:, :3].astype(np.float64)}
        F, T, _ = force_fn(st64["pos"], st64["quat"])
        nxt, _ = md.step(dict(st64, F=F, tau=T), force_fn, M, I, box, dt)
        dp = cur["pos"][:, :3] - nxt["pos"]
        dp -= L * np.rint(dp / L)
        worst["pos"] = max(worst["pos"], np.abs(dp).max())
        worst["quat"] = max(worst["quat"], np.abs(cur["quat"] - nxt["quat"]).max())
        worst["vel"] = max(worst["vel"], rel_err(cur["vel"][:, :3], nxt["vel"]))
        worst["angmom"] = max(worst["angmom"], rel_err(cur["angmom"][:, :3], nxt["angmom"]))
        prev = cur
    assert worst["pos"] < 2e-5 and worst["quat"] < 2e-6, worst
    assert worst["vel"] < 1e-5 and worst["angmom"] < 1e-5, worst
    e1 = sum(s.energy())
    assert abs(e1 - e0) < 1e-3 * 64, (e0, e1)


def test_verlet_skin_gives_identical_forces_and_trajectories():
    """With a skin the list holds pairs within Rc + skin and is rebuilt only
    after a centre moves more than skin/2; pairs beyond Rc give exactly zero,
    so forces and whole trajectories equal those of a list rebuilt every step."""
    from paper_2402_12199_gb300 import api

    st, L, tmpl = make_state(3000, 0.1, 71)
    st = dict(st)
    st["vel"] = st["vel"] * 40.0  # hot: centres cross the skin within a few steps
    a = gpu_system(st, L)
    b = gpu_system(st, L)
    b.set_skin(0.4)
    fa, fb = a.forces_beads(), b.forces_beads()
    assert b.build_pairs() > a.build_pairs()
    assert bool((fa["force"] == fb["force"]).all()) and bool((fa["torque"] == fb["torque"]).all())
    for path, mlp, prec in [(api.RB_PATH_BEADS, None, "fp32")]:
        a.step(60, 0.004, path=path, mlp=mlp, precision=prec)
        b.step(60, 0.004, path=path, mlp=mlp, precision=prec)
        sa, sb = a.get_state(to_host=True), b.get_state(to_host=True)
        for k in ("pos", "quat", "vel", "angmom"):
            assert np.array_equal(sa[k], sb[k]), k
    a.sync()
    b.sync()


def test_checkpoint_restore_continues_bit_for_bit(tmp_path):
    from paper_2402_12199_gb300 import api

    st, L, tmpl = make_state(1000, 0.15, 81)
    a = gpu_system(st, L)
    a.set_skin(0.3)
    a.step(20, 0.002)
    path = tmp_path / "ck.rbck"
    a.checkpoint(path)
    a.step(30, 0.002)
    ref = a.get_state(to_host=True)
    b = api.System(1000, [L] * 3, "cube")
    b.restore(path)
    assert b.step_count == 20
    b.step(30, 0.002)
    got = b.get_state(to_host=True)
    for k in ("pos", "quat", "vel", "angmom"):
        assert np.array_equal(ref[k], got[k]), k
    assert b.step_count == 50
    c = api.System(999, [L] * 3, "cube")
    with pytest.raises(api.RBError):
        c.restore(path)


def test_state_read_back_asynchronously_into_pinned_memory():
    """rb_get_state with to_host = 2 queues the copies; after a stream
    synchronisation the page-locked buffers hold the same state as a
    synchronous read."""
    import torch

    from paper_2402_12199_gb300 import api

    st, L, tmpl = make_state(300, 0.15, 61)
    s = gpu_system(st, L)
    s.forces_beads()
    s.step(3, 0.002, path=api.RB_PATH_BEADS)
    out = {k: torch.full((300, 4), float("nan")).pin_memory() for k in ("pos", "quat", "vel", "angmom")}
    s.get_state(to_host=True, out=out, sync=False)
    torch.cuda.synchronize()
    ref = s.get_state(to_host=True)
    for k in out:
        np.testing.assert_array_equal(out[k].numpy(), ref[k])


def test_contiguous_state_block_moves_in_one_copy_and_round_trips():
    """State given as one page-locked block (pos | quat | vel | angmom) takes the
    single-copy path in and out and round-trips exactly; separate arrays and
    the block give the same state."""
    import torch

    st, L, tmpl = make_state(777, 0.1, 91)
    a = gpu_system(st, L)
    blk = torch.from_numpy(np.stack([st[k] for k in ("pos", "quat", "vel", "angmom")])).pin_memory()
    b = gpu_system(st, L)
    b.set_state(blk[0], blk[1], blk[2], blk[3])
    out = torch.empty((4, 777, 4), dtype=torch.float32).pin_memory()
    b.get_state(to_host=True, out={k: out[i] for i, k in enumerate(("pos", "quat", "vel", "angmom"))})
    for i, k in enumerate(("pos", "quat", "vel", "angmom")):
        assert np.array_equal(out[i].numpy(), st[k]), k
    a.step(10, 0.002)
    b.step(10, 0.002)
    ra, rb = a.get_state(to_host=True), b.get_state(to_host=True)
    for k in ("pos", "quat", "vel", "angmom"):
        assert np.array_equal(ra[k], rb[k]), k
