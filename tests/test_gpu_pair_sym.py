"""Pair-symmetrised network evaluation (rb_mlp_set_pair_symmetrised: the
energy of every pair averaged over both choices of reference body) against
the FP64 oracle at each precision's tolerance, its invariance under
relabelling the bodies on the GPU, switching it off again, and an MD run."""
import numpy as np
import pytest

import oracle
from oracle import bodies, nn
from paper_2402_12199_gb300 import inputs
from tests.helpers import (TOL_BF16, TOL_F32, assert_parity, canonical_margin, gpu_system,
                           make_state, rel_err)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()


def params(seed, depth=3, width=128):
    mu, isd = inputs.feature_normalisation(5.0, 9.43)
    return inputs.mlp_params(width, depth, seed, mu=mu, inv_sd=isd, e_scale=1.5, e_shift=-0.2)


def oracle_sym(st, L, tmpl, flat, width=128, depth=3):
    pos = st["pos"][:, :3].astype(np.float64)
    quat = st["quat"].astype(np.float64)
    box = np.array([L] * 3)
    pairs = oracle.pairs_bruteforce(pos, box, bodies.pair_cutoff(tmpl))
    p = nn.unpack(np.asarray(flat, dtype=np.float64), width, depth)
    F, T, E, per = nn.forces_nn_symmetrised(p, pos, quat, box, pairs)
    return F, T, E, per, pairs


@pytest.mark.parametrize("precision,tol", [("fp32", TOL_F32), ("f16x3", TOL_F32), ("bf16", TOL_BF16)])
def test_pair_symmetrised_forces_parity(precision, tol):
    from paper_2402_12199_gb300 import api

    st, L, tmpl = make_state(1500, 0.20, 21)
    flat = params(22)
    m = api.MLP(128, 3)
    m.set_params(flat)
    m.set_pair_symmetrised(True)
    s = gpu_system(st, L)
    r = s.forces_nn(m, precision, energy=True)
    s.sync()
    F, T, E, per, pairs = oracle_sym(st, L, tmpl, flat)
    assert canonical_margin(st, pairs) > 1e-5
    assert_parity(r["force"][:, :3].double().cpu().numpy(), F, tol)
    assert_parity(r["torque"][:, :3].double().cpu().numpy(), T, tol)
    assert abs(r["energy"] - E) < tol * np.abs(per).sum()
    # switched off again: the plain evaluation (i < j, i the reference)
    m.set_pair_symmetrised(False)
    r0 = s.forces_nn(m, precision, energy=True)
    s.sync()
    F0, T0, E0, per0 = nn.forces_nn(nn.unpack(flat.astype(np.float64), 128, 3),
                                    st["pos"][:, :3].astype(np.float64), st["quat"].astype(np.float64),
                                    np.array([L] * 3), pairs)
    assert_parity(r0["force"][:, :3].double().cpu().numpy(), F0, tol)
    assert abs(r0["energy"] - E0) < tol * np.abs(per0).sum()


def test_pair_symmetrised_relabelling_invariance_on_gpu():
    import torch

    from paper_2402_12199_gb300 import api

    st, L, tmpl = make_state(1200, 0.20, 31)
    m = api.MLP(128, 3)
    m.set_params(params(32))
    perm = np.random.default_rng(33).permutation(len(st["pos"]))
    st2 = {k: np.ascontiguousarray(v[perm]) for k, v in st.items()}
    out = {}
    for sym in (True, False):
        m.set_pair_symmetrised(sym)
        a, b = gpu_system(st, L), gpu_system(st2, L)
        ra, rb_ = a.forces_nn(m, "fp32", energy=True), b.forces_nn(m, "fp32", energy=True)
        b.sync()
        Fa = ra["force"][:, :3].double().cpu().numpy()
        Fb = rb_["force"][:, :3].double().cpu().numpy()
        out[sym] = (abs(rb_["energy"] - ra["energy"]) / abs(ra["energy"]), rel_err(Fb, Fa[perm]))
    # symmetrised: the same up to FP32 rounding; plain: the labels matter
    assert out[True][0] < 1e-5 and out[True][1] < 1e-5, out
    assert out[False][0] > 10 * out[True][0] or out[False][1] > 10 * out[True][1], out


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_pair_symmetrised_md_conserves_momentum(precision):
    from paper_2402_12199_gb300 import api

    st, L, tmpl = make_state(800, 0.2, 41)
    m = api.MLP(128, 3)
    m.set_params(params(42))
    m.set_pair_symmetrised(True)
    s = gpu_system(st, L)
    s.set_skin(0.4)
    v0 = s.get_state(to_host=True)["vel"][:, :3].astype(np.float64).sum(0)
    s.forces_nn(m, precision)
    e0 = sum(s.energy())
    s.step(100, 0.002, path=api.RB_PATH_NN, mlp=m, precision=precision)
    e1 = sum(s.energy())
    cur = s.get_state(to_host=True)
    s.sync()
    assert np.all(np.isfinite(cur["pos"]))
    v1 = cur["vel"][:, :3].astype(np.float64).sum(0)
    scale = np.abs(cur["vel"][:, :3]).sum()
    assert np.abs(v1 - v0).max() < 1e-5 * scale
    assert abs(e1 - e0) < 1e-2 * len(st["pos"]), (e0, e1)
