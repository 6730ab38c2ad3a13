"""The cylinder workload at full size: 100k cylinders (8 stacked rings of 19
hexagonally packed beads), packing fraction 0.15, network width 256.

Covers, on the GPU against the FP64 oracle: the bead sum and both network
precisions on sampled bodies of the 100k-body system, the adjoint of the
width-256 network against central finite differences of the oracle's FP64
energy (h = 1e-4), and a 1M-pair on-device training set (contact bisection +
bead-sum labels) checked on a sample."""
import numpy as np
import pytest

from oracle import bodies, nn, sampler
from paper_2402_12199_gb300 import inputs
from tests.helpers import (TOL_BF16, TOL_F32, assert_parity, canonical_margin, gpu_system,
                           make_state, oracle_beads, oracle_nn, rel_err)

pytestmark = pytest.mark.gpu

N_CYL, PHI_CYL, SEED_CYL, WIDTH = 100_000, 0.15, 4, 256


@pytest.fixture(scope="module", autouse=True)
def _built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()


@pytest.fixture(scope="module")
def system100k():
    st, L, tmpl = make_state(N_CYL, PHI_CYL, SEED_CYL, "cylinder")
    rng = np.random.default_rng(11)
    idx = rng.choice(N_CYL, 32, replace=False)
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
    return st, L, tmpl, idx, pairs


def _net(seed):
    mu, isd = inputs.feature_normalisation(6.0, 11.44)
    return inputs.mlp_params(WIDTH, 3, seed, mu=mu, inv_sd=isd, e_scale=1.1, e_shift=-0.1)


def test_bead_forces_sampled_100k_cylinders(system100k):
    st, L, tmpl, idx, pairs = system100k
    s = gpu_system(st, L, "cylinder")
    res = s.forces_beads()
    n_pairs = s.build_pairs()
    s.sync()
    assert len(pairs) > 32
    F, T, _, _, _ = oracle_beads(st, L, tmpl, pairs)
    assert_parity(res["force"][:, :3].double().cpu().numpy()[idx], F[idx], TOL_F32)
    assert_parity(res["torque"][:, :3].double().cpu().numpy()[idx], T[idx], TOL_F32)
    # about 2.7 half pairs per body at this density
    assert 150_000 < n_pairs < 500_000


@pytest.mark.parametrize("precision,tol", [("fp32", TOL_F32), ("bf16", TOL_BF16)])
def test_nn_width256_sampled_100k_cylinders(system100k, precision, tol):
    from paper_2402_12199_gb300 import api

    st, L, tmpl, idx, pairs = system100k
    flat = _net(21)
    m = api.MLP(WIDTH, 3)
    m.set_params(flat)
    s = gpu_system(st, L, "cylinder")
    r = s.forces_nn(m, precision)
    s.sync()
    assert canonical_margin(st, pairs) > 1e-6
    F, T, _, _, _ = oracle_nn(st, L, tmpl, flat, WIDTH, pairs=pairs)
    assert_parity(r["force"][:, :3].double().cpu().numpy()[idx], F[idx], tol)
    assert_parity(r["torque"][:, :3].double().cpu().numpy()[idx], T[idx], tol)


def test_width256_adjoint_matches_central_differences():
    """F_j = -dE/dR, tau_j = -dE/dtheta_j, tau_i = -dE/dtheta_i: the GPU's FP32
    adjoint against central differences (h = 1e-4) of the oracle's FP64
    energy, body i at the origin with the identity orientation."""
    import torch

    from paper_2402_12199_gb300 import api

    flat = _net(22)
    p = nn.unpack(flat.astype(np.float64), WIDTH, 3)
    c7 = inputs.pair_configs(96, 23, 6.0, 11.4)
    c7 = c7[np.abs(c7[:, 3]) > 1e-2]  # away from the canonical-sign switch
    n = len(c7)
    cfg8 = np.zeros((n, 8), np.float32)
    cfg8[:, :3] = c7[:, :3]
    cfg8[:, 4:] = c7[:, 3:]
    m = api.MLP(WIDTH, 3)
    m.set_params(flat)
    out = m.pairs(torch.from_numpy(cfg8).cuda(), "fp32").double().cpu().numpy()
    # differences are taken at the FP32 configuration the GPU saw
    R = cfg8[:, :3].astype(np.float64)
    qj = cfg8[:, 4:].astype(np.float64)
    qi = np.zeros((n, 4))
    qi[:, 0] = 1.0

    def energy(R_, qi_, qj_):
        t = torch.as_tensor
        s = nn._to_body(t(qi_), t(R_))
        return nn.config_energy(p, s, nn._qmul(nn._qconj(t(qi_)), t(qj_))).detach().numpy()

    h = 1e-4
    Fj, ti, tj = np.zeros((n, 3)), np.zeros((n, 3)), np.zeros((n, 3))
    for k in range(3):
        e = np.eye(3)[k] * h
        rp = np.broadcast_to(bodies.qexp(e), (n, 4))
        rm = np.broadcast_to(bodies.qexp(-e), (n, 4))
        Fj[:, k] = -(energy(R + e, qi, qj) - energy(R - e, qi, qj)) / (2 * h)
        tj[:, k] = -(energy(R, qi, bodies.qmul(rp, qj)) - energy(R, qi, bodies.qmul(rm, qj))) / (2 * h)
        ti[:, k] = -(energy(R, bodies.qmul(rp, qi), qj) - energy(R, bodies.qmul(rm, qi), qj)) / (2 * h)
    assert_parity(out[:, 0:3], Fj, TOL_F32)
    assert_parity(out[:, 4:7], ti, TOL_F32)
    assert_parity(out[:, 8:11], tj, TOL_F32)


def test_sampler_one_million_cylinder_pairs():
    import torch

    from paper_2402_12199_gb300 import api

    tmpl = bodies.cylinder_template()
    Rc = bodies.pair_cutoff(tmpl)
    s = api.System(8, [60.0] * 3, "cylinder")
    n = 1_000_000
    u = inputs.sampler_uniforms(n, 41)
    cfg, lab, rc = api.sample_pairs(s, torch.from_numpy(u).cuda())
    torch.cuda.synchronize()
    assert bool(torch.isfinite(lab).all()) and bool(torch.isfinite(cfg).all())
    rho = torch.linalg.norm(cfg[:, :3], dim=1)
    assert bool((rho >= rc - 1e-4).all()) and bool((rho <= Rc + 1e-4).all())
    # contact distances lie between the inscribed and circumscribed bounds
    r_circ = float(np.sqrt((tmpl ** 2).sum(1).max()))
    assert float(rc.min()) > 1.0 - 1e-4 and float(rc.max()) < 2 * r_circ + 1.0 + 1e-4
    rng = np.random.default_rng(42)
    pick = np.sort(rng.choice(n, 64, replace=False))
    c = cfg[pick].double().cpu().numpy()
    got = lab[pick].double().cpu().numpy()
    ref = sampler.label_pairs(np.concatenate([c[:, :3], c[:, 4:8]], 1), tmpl)
    assert_parity(got[:, 0:3], ref[:, 1:4], TOL_F32)
    assert_parity(got[:, 4:7], ref[:, 4:7], TOL_F32)
    assert_parity(got[:, 8:11], ref[:, 7:10], TOL_F32)
    d, q = sampler.draws_to_config(u[pick].astype(np.float64))
    for b in range(0, 64, 8):
        assert float(rc[pick[b]]) == pytest.approx(sampler.contact_distance(d[b], q[b], tmpl, Rc),
                                                   abs=2e-5)
