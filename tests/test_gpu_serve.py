"""Serving: continuous batching of independent MD replicas.  A request's
result is the same alone and in a mix; admission respects the memory budget;
waits time out; a network that produces non-finite forces falls back to the
bead path."""
import time

import numpy as np
import pytest

from paper_2402_12199_gb300 import inputs
from tests.helpers import make_state

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()


def net(seed=3):
    from paper_2402_12199_gb300 import api

    mu, isd = inputs.feature_normalisation(5.0, 9.43)
    m = api.MLP(128, 3)
    m.set_params(inputs.mlp_params(128, 3, seed, mu=mu, inv_sd=isd))
    return m


def test_result_is_identical_alone_and_in_a_mix():
    from paper_2402_12199_gb300 import api

    m = net()
    A = make_state(512, 0.20, 41)
    B = make_state(900, 0.15, 42, "cylinder")
    C = make_state(2000, 0.10, 43)
    s1 = api.Server(4 << 30, 1, m, steps_per_tick=5)
    ta = s1.submit(A[0], [A[1]] * 3, "cube", api.RB_PATH_NN, "bf16", 30)
    ra = s1.wait(ta)
    alone = s1.fetch_state(ta)
    s1.close()
    assert ra["status"] == 0 and ra["steps_done"] == 30
    s2 = api.Server(4 << 30, 4, m, steps_per_tick=3)
    tb = s2.submit(B[0], [B[1]] * 3, "cylinder", api.RB_PATH_BEADS, "fp32", 25)
    tc = s2.submit(C[0], [C[1]] * 3, "cube", api.RB_PATH_NN, "fp32", 20)
    ta2 = s2.submit(A[0], [A[1]] * 3, "cube", api.RB_PATH_NN, "bf16", 30)
    for t in (tb, tc, ta2):
        r = s2.wait(t)
        assert r["status"] == 0, r
    mixed = s2.fetch_state(ta2)
    st = s2.stats()
    s2.close()
    for k in ("pos", "quat", "vel", "angmom"):
        assert np.array_equal(alone[k], mixed[k]), k
    assert st["peak_resident"] >= 2 and st["steps"] == 75


def test_admission_respects_memory_budget():
    from paper_2402_12199_gb300 import api

    st, L, _ = make_state(1000, 0.2, 44)
    fp = api.footprint(1000, [L] * 3)
    srv = api.Server(int(2.5 * fp), 8, None, steps_per_tick=4)
    tickets = [srv.submit(st, [L] * 3, n_steps=12) for _ in range(6)]
    res = [srv.wait(t) for t in tickets]
    stats = srv.stats()
    srv.close()
    assert all(r["status"] == 0 and r["steps_done"] == 12 for r in res)
    assert 1 <= stats["peak_resident"] <= 2
    # identical requests give identical results whatever their admission order
    assert len({round(r["e_end"], 12) for r in res}) == 1
    with pytest.raises(api.RBError) as ei:
        api.Server(fp // 2, 2).submit(st, [L] * 3)
    assert ei.value.status == 2


def test_wait_times_out_and_poll_is_nonblocking():
    from paper_2402_12199_gb300 import api

    st, L, _ = make_state(8000, 0.2, 45)
    srv = api.Server(8 << 30, 2, None, steps_per_tick=8)
    t = srv.submit(st, [L] * 3, n_steps=3000)
    t0 = time.perf_counter()
    assert srv.poll(t) is None
    with pytest.raises(api.RBError) as ei:
        srv.wait(t, timeout_ms=5)
    assert ei.value.status == 6
    assert time.perf_counter() - t0 < 2.0
    srv.close()  # the unfinished request is drained, not leaked


def test_non_finite_network_falls_back_to_beads():
    from paper_2402_12199_gb300 import api

    m = api.MLP(128, 3)
    flat = inputs.mlp_params(128, 3, 9)
    flat[100] = np.nan
    m.set_params(flat)
    st, L, _ = make_state(512, 0.2, 46)
    srv = api.Server(4 << 30, 2, m, steps_per_tick=4)
    t = srv.submit(st, [L] * 3, path=api.RB_PATH_NN, precision="bf16", n_steps=16)
    tb = srv.submit(st, [L] * 3, path=api.RB_PATH_BEADS, n_steps=16)
    r = srv.wait(t)
    rb = srv.wait(tb)
    fin = srv.fetch_state(t)
    finb = srv.fetch_state(tb)
    srv.close()
    assert r["status"] == 0 and r["fell_back"] == 1 and r["steps_done"] == 16
    assert np.isfinite(fin["pos"]).all()
    # the fallback replica followed the bead path from its start
    for k in ("pos", "quat", "vel", "angmom"):
        assert np.array_equal(fin[k], finb[k]), k


def test_batched_replicas_match_their_own_runs():
    """Resident replicas step together (one launch per phase for all of them,
    the pair kernels over their concatenated lists); each ends where its own
    rb_step run ends, to rounding: the batched kernels do the same arithmetic
    but are separate kernels, whose fused multiply-adds the compiler may form
    differently (a * b + c * d), so the last bit may differ.  A wrong system,
    box or pair slot for any pair would be far outside the bound.  The mix
    covers both batched pair kernels (BF16 network, bead sum of the cube and
    of the cylinder), a precision launched per replica inside the batch
    (F16X3), skin and no skin, and ticks of 4 and 2 steps."""
    import torch

    from paper_2402_12199_gb300 import api

    m = net()
    cases = [
        (make_state(600, 0.20, 51), "cube", api.RB_PATH_NN, "bf16", 0.4),
        (make_state(700, 0.15, 52, "cylinder"), "cylinder", api.RB_PATH_BEADS, "fp32", 0.4),
        (make_state(500, 0.20, 53), "cube", api.RB_PATH_BEADS, "fp32", 0.0),
        (make_state(800, 0.20, 54), "cube", api.RB_PATH_NN, "bf16", 0.0),
        (make_state(400, 0.20, 55), "cube", api.RB_PATH_NN, "f16x3", 0.4),
        (make_state(300, 0.10, 56), "cube", api.RB_PATH_BEADS, "fp32", 0.4),
    ]
    steps = 14
    srv = api.Server(8 << 30, 8, m, steps_per_tick=4)
    tickets = [srv.submit(st, [L] * 3, shape, path, prec, steps, skin=skin)
               for (st, L, _), shape, path, prec, skin in cases]
    results = [srv.wait(t) for t in tickets]
    finals = [srv.fetch_state(t) for t in tickets]
    stats = srv.stats()
    srv.close()
    assert stats["peak_resident"] == len(cases)
    keys = ("pos", "quat", "vel", "angmom")
    for ((st, L, _), shape, path, prec, skin), r, fin in zip(cases, results, finals):
        assert r["status"] == 0 and r["steps_done"] == steps and r["fell_back"] == 0, r
        s = api.System(len(st["pos"]), [L] * 3, shape, skin=skin)
        s.set_state(*(torch.from_numpy(np.ascontiguousarray(st[k])).cuda() for k in keys))
        cfg = dict(path=path) if path == api.RB_PATH_BEADS else dict(path=path, mlp=m, precision=prec)
        s.step(steps, 0.002, **cfg)
        own = s.get_state(to_host=True)
        for k in keys:
            a, b = np.asarray(fin[k], np.float64), np.asarray(own[k], np.float64)
            d = float(np.max(np.abs(a - b)))
            assert d <= 1e-5 * float(np.max(np.abs(b))), (shape, path, prec, skin, k, d)


def test_lanes_do_not_change_results():
    """The same requests spread over one lane, three lanes or eight end bit for
    bit alike: a replica's arithmetic does not depend on which batch it is in."""
    from paper_2402_12199_gb300 import api

    m = net()
    reqs = [(make_state(400 + 150 * k, (0.10 if k % 2 else 0.15) + 0.01 * (k % 3), 60 + k,
                        "cylinder" if k % 2 else "cube"), k % 2) for k in range(6)]
    finals = []
    for lanes in (1, 3, 8):
        srv = api.Server(8 << 30, 6, m, steps_per_tick=3, lanes=lanes)
        tickets = [srv.submit(st, [L] * 3, "cylinder" if cyl else "cube",
                              api.RB_PATH_BEADS if cyl else api.RB_PATH_NN, "bf16", 10, skin=0.4)
                   for (st, L, _), cyl in reqs]
        res = [srv.wait(t) for t in tickets]
        assert all(r["status"] == 0 and r["steps_done"] == 10 for r in res), res
        finals.append([srv.fetch_state(t) for t in tickets])
        srv.close()
    for other in finals[1:]:
        for a, b in zip(finals[0], other):
            for k in ("pos", "quat", "vel", "angmom"):
                assert np.array_equal(a[k], b[k]), k
    with pytest.raises(api.RBError):
        api.Server(1 << 30, 2, m, lanes=9)


def test_networks_per_body_shape():
    """Network-path requests use the network set for their body shape (with
    its bead-fallback radius): each replica ends where its own rb_step run
    with that network and fallback ends (to rounding, as above).  The cube
    network's radius, 8.5 sigma, sends the closer pairs to the bead sum inside
    the batched step."""
    import torch

    from paper_2402_12199_gb300 import api

    m_cube = net(3)
    m_cyl = api.MLP(256, 3)  # width 256: the batched width-256 kernel for the cylinders
    mu, isd = inputs.feature_normalisation(5.0, 4 * 3 ** 0.5 + 2.5)
    m_cyl.set_params(inputs.mlp_params(256, 3, 5, mu=mu, inv_sd=isd))
    A = make_state(600, 0.20, 71)
    B = make_state(500, 0.12, 72, "cylinder")
    C = make_state(700, 0.10, 73, "cylinder")
    srv = api.Server(4 << 30, 4, m_cube, steps_per_tick=4)
    srv.set_network("cube", m_cube, rho_min=8.5)
    srv.set_network("cylinder", m_cyl)
    ta = srv.submit(A[0], [A[1]] * 3, "cube", api.RB_PATH_NN, "bf16", 9, skin=0.4)
    tb = srv.submit(B[0], [B[1]] * 3, "cylinder", api.RB_PATH_NN, "bf16", 9, skin=0.4)
    tc = srv.submit(C[0], [C[1]] * 3, "cylinder", api.RB_PATH_NN, "bf16", 9, skin=0.4)
    fins = {}
    for t, name in ((ta, "cube"), (tb, "cylinder"), (tc, "cylinder2")):
        r = srv.wait(t)
        assert r["status"] == 0 and r["steps_done"] == 9 and r["fell_back"] == 0, r
        fins[name] = srv.fetch_state(t)
    srv.close()
    keys = ("pos", "quat", "vel", "angmom")
    for (st, L, _), shape, m, name in ((A, "cube", m_cube, "cube"), (B, "cylinder", m_cyl, "cylinder"),
                                       (C, "cylinder", m_cyl, "cylinder2")):
        s = api.System(len(st["pos"]), [L] * 3, shape, skin=0.4)
        s.set_state(*(torch.from_numpy(np.ascontiguousarray(st[k])).cuda() for k in keys))
        if shape == "cube":
            s.set_nn_fallback(8.5)
        s.step(9, 0.002, path=api.RB_PATH_NN, mlp=m, precision="bf16")
        own = s.get_state(to_host=True)
        for k in keys:
            a, b = np.asarray(fins[name][k], np.float64), np.asarray(own[k], np.float64)
            d = float(np.max(np.abs(a - b)))
            assert d <= 1e-5 * float(np.max(np.abs(b))), (name, k, d)
        if shape == "cube":  # the fallback took pairs in this run
            assert s.nn_fallback_count() > 0
    # the cylinder really ran on its own network: the cube network gives another trajectory
    s = api.System(len(B[0]["pos"]), [B[1]] * 3, "cylinder", skin=0.4)
    s.set_state(*(torch.from_numpy(np.ascontiguousarray(B[0][k])).cuda() for k in keys))
    s.step(9, 0.002, path=api.RB_PATH_NN, mlp=m_cube, precision="bf16")
    other = s.get_state(to_host=True)
    assert not np.array_equal(np.asarray(other["vel"]), fins["cylinder"]["vel"])
    with pytest.raises(api.RBError):
        api.Server(1 << 30, 2, m_cube).set_network("custom", api.MLP(128, 3))
    with pytest.raises(api.RBError):
        api.Server(1 << 30, 2, m_cube).set_network("cube", m_cube, rho_min=-1.0)


def test_network_that_fails_mid_run_rolls_back_to_the_tick():
    """A network that is exactly zero while every pair is farther than
    rho_thr and overflows to infinity as soon as one comes closer: two cubes
    coasting towards each other cross rho_thr in the third tick of four steps.
    The replica is rolled back to that tick's start (with the next tick
    already queued, which is voided) and continues on the bead path; both
    force fields are exactly zero at these distances, so it ends bit for bit
    where the bead path alone ends."""
    import torch

    from paper_2402_12199_gb300 import api

    W, D, n_in = 128, 3, 10
    flat = np.zeros(2 * n_in + W * n_in + W + (D - 1) * (W * W + W) + W + 1 + 2, np.float32)
    flat[n_in:2 * n_in] = 1.0                      # inv_sd: raw features
    W1, b1 = 2 * n_in, 2 * n_in + W * n_in
    W2 = b1 + W
    W3 = W2 + W * W + W
    wo = W3 + W * W + W
    a, rho_thr = 1e25, 9.1
    flat[W1 + 7] = -a                              # unit 0 of layer 1 reads rho (feature 7)
    flat[b1] = a * rho_thr                         # z = a (rho_thr - rho)
    flat[W2] = 1e25                                # overflows once z > 0
    flat[W3] = 1.0
    flat[wo] = 1.0
    flat[-2] = 1.0                                 # e_scale
    m = api.MLP(W, D)
    m.set_params(flat)
    L = 40.0
    st = {"pos": np.array([[10.0, 20.0, 20.0, 0.0], [19.3, 20.0, 20.0, 0.0]], np.float32),
          "quat": np.array([[1.0, 0.0, 0.0, 0.0]] * 2, np.float32),
          "vel": np.array([[5.0, 0.0, 0.0, 0.0], [-5.0, 0.0, 0.0, 0.0]], np.float32),
          "angmom": np.zeros((2, 4), np.float32)}
    srv = api.Server(1 << 30, 2, m, steps_per_tick=4)
    t = srv.submit(st, [L] * 3, "cube", api.RB_PATH_NN, "bf16", 24)
    r = srv.wait(t)
    fin = srv.fetch_state(t)
    srv.close()
    assert r["status"] == 0 and r["steps_done"] == 24 and r["fell_back"] == 1, r
    keys = ("pos", "quat", "vel", "angmom")
    s = api.System(2, [L] * 3, "cube")
    s.set_state(*(torch.from_numpy(st[k]).cuda() for k in keys))
    s.step(24, 0.002, path=api.RB_PATH_BEADS)
    ref = s.get_state(to_host=True)
    for k in keys:
        assert np.array_equal(np.asarray(ref[k]), fin[k]), k
    # the separation did cross rho_thr (9.3 - 24 x 0.02 = 8.82)
    assert fin["pos"][1, 0] - fin["pos"][0, 0] < rho_thr
