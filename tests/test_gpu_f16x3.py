"""FP32-accurate tensor-core network path (RB_F16X3: operands split into two
power-of-two-scaled FP16 parts, three tcgen05 products accumulated in FP32)
against the FP64 oracle at the FP32 tolerance: pair outputs over several
tiles with ragged tails and every supported depth, weights and inputs far
from unit scale (the per-row and per-matrix scaling), whole-system forces,
torques and energy, an MD run, and the unsupported shapes."""
import numpy as np
import pytest

from oracle import nn
from paper_2402_12199_gb300 import inputs
from tests.helpers import (TOL_F32, assert_parity, canonical_margin, gpu_system, make_state,
                           oracle_nn, rel_err)

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


def cfg8(cfg7):
    c = np.zeros((len(cfg7), 8), np.float32)
    c[:, :3] = cfg7[:, :3]
    c[:, 4:] = cfg7[:, 3:]
    return c


def _check_pairs(flat, depth, n, seed, tol=TOL_F32):
    import torch

    from paper_2402_12199_gb300 import api

    m = api.MLP(128, depth)
    m.set_params(flat)
    cfg7 = inputs.pair_configs(n, seed, 5.0, 9.4)
    out = m.pairs(torch.from_numpy(cfg8(cfg7)).cuda(), "f16x3").double().cpu().numpy()
    p = nn.unpack(flat.astype(np.float64), 128, depth)
    c = torch.as_tensor(cfg7.astype(np.float64))
    E, Fj, ti, tj = nn.predict_labels(p, c[:, :3], c[:, 3:])
    assert_parity(out[:, 0:3], Fj.numpy(), tol)
    assert_parity(out[:, 4:7], ti.numpy(), tol)
    assert_parity(out[:, 8:11], tj.numpy(), tol)
    assert_parity(out[:, 3], E.detach().numpy(), tol)
    assert np.all(out[:, [7, 11]] == 0.0)


@pytest.mark.parametrize("n,depth", [(4096, 3), (1000, 3), (129, 3), (1, 3), (777, 2), (300, 1)])
def test_nn_pairs_f16x3_parity(n, depth):
    _check_pairs(params(17 + n, depth), depth, n, 41 + n)


@pytest.mark.parametrize("factors", [(1e-4, 1.0, 1.0), (1.0, 3e3, 1e-3), (50.0, 1e-2, 20.0)])
def test_nn_pairs_f16x3_far_from_unit_scale(factors):
    """Weight matrices scaled by powers far from 1 (the FP16 range alone would
    underflow or overflow the split parts); the per-matrix and per-row
    scales must keep FP32 accuracy."""
    depth, width = 3, 128
    flat = params(5, depth).astype(np.float64)
    o_W1 = 20  # flat layout: mu (10), 1/sd (10), W_1, b_1, then W_l, b_l per layer
    flat[o_W1:o_W1 + width * 10] *= factors[0]
    o = o_W1 + width * 10 + width
    for l in range(2, depth + 1):
        flat[o:o + width * width] *= factors[l - 1]
        o += width * width + width
    _check_pairs(flat.astype(np.float32), depth, 1500, 77)


def test_nn_pairs_f16x3_empty_and_unsupported_shapes():
    import torch

    from paper_2402_12199_gb300 import api

    m = api.MLP(128, 3)
    m.set_params(params(3))
    out = m.pairs(torch.zeros((0, 8), dtype=torch.float32, device="cuda"), "f16x3")
    assert out.shape[0] == 0
    for width, depth in ((64, 3), (256, 3), (128, 4)):
        w = api.MLP(width, depth)
        w.set_params(inputs.mlp_params(width, depth, 9))
        with pytest.raises(api.RBError):
            w.pairs(torch.zeros((4, 8), dtype=torch.float32, device="cuda"), "f16x3")


def test_nn_system_forces_f16x3_parity():
    from paper_2402_12199_gb300 import api

    st, L, tmpl = make_state(2000, 0.20, 12)
    flat = params(3)
    m = api.MLP(128, 3)
    m.set_params(flat)
    s = gpu_system(st, L)
    r = s.forces_nn(m, "f16x3", energy=True)
    s.sync()
    F, T, E, per, pairs = oracle_nn(st, L, tmpl, flat, 128)
    assert canonical_margin(st, pairs) > 1e-5
    assert_parity(r["force"][:, :3].double().cpu().numpy(), F, TOL_F32)
    assert_parity(r["torque"][:, :3].double().cpu().numpy(), T, TOL_F32)
    assert abs(r["energy"] - E) < TOL_F32 * np.abs(per).sum()


def test_nn_f16x3_matches_fp32_path_in_md():
    """50 NVE steps on the F16X3 path stay within FP32 rounding of the SIMT
    FP32 path (same network, same start) and conserve energy like it."""
    from paper_2402_12199_gb300 import api

    st, L, tmpl = make_state(512, 0.2, 6)
    m = api.MLP(128, 3)
    m.set_params(params(4))
    a = gpu_system(st, L)
    b = gpu_system(st, L)
    a.forces_nn(m, "fp32")
    b.forces_nn(m, "f16x3")
    e0 = sum(b.energy())
    a.step(50, 0.002, path=api.RB_PATH_NN, mlp=m, precision="fp32")
    b.step(50, 0.002, path=api.RB_PATH_NN, mlp=m, precision="f16x3")
    e1 = sum(b.energy())
    pa = a.get_state(to_host=True)["pos"][:, :3].astype(np.float64)
    pb = b.get_state(to_host=True)["pos"][:, :3].astype(np.float64)
    b.sync()
    assert abs(e1 - e0) < 1e-2 * 512, (e0, e1)
    d = pb - pa
    d -= L * np.round(d / L)
    assert np.abs(d).max() < 1e-3, np.abs(d).max()
