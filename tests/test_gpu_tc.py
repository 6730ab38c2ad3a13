"""Tensor-core (tcgen05, BF16 operands, FP32 accumulation) network path: a
single-tile GEMM check, then network forces/torques against the FP64 oracle
within the BF16 tolerance."""
import numpy as np
import pytest

from oracle import nn
from paper_2402_12199_gb300 import inputs
from tests.helpers import (TOL_BF16, assert_parity, canonical_margin, gpu_system, make_state,
                           oracle_nn, rel_err)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()


def bf16(t):
    return t.to(__import__("torch").bfloat16).double()


@pytest.mark.parametrize("N,K", [(128, 128), (128, 64), (16, 128), (64, 64)])
def test_tc_gemm_tile(N, K):
    import torch

    from paper_2402_12199_gb300 import api

    g = torch.Generator().manual_seed(N * 1000 + K)
    A = torch.randn(128, K, generator=g)
    B = torch.randn(N, K, generator=g)
    D = api.tc_gemm_check(A.cuda(), B.cuda()).double().cpu()
    ref = bf16(A) @ bf16(B).T  # exact products of the BF16-rounded operands
    assert torch.allclose(D, ref, rtol=1e-5, atol=1e-4), (D - ref).abs().max()


def params(seed, depth=3, width=128):
    mu, isd = inputs.feature_normalisation(5.0, 9.43)
    return inputs.mlp_params(width, depth, seed, mu=mu, inv_sd=isd, e_scale=1.5, e_shift=-0.2)


def cfg8(cfg7):
    c = np.zeros((len(cfg7), 8), np.float32)
    c[:, :3] = cfg7[:, :3]
    c[:, 4:] = cfg7[:, 3:]
    return c


@pytest.mark.parametrize("n,depth,width", [(4096, 3, 128), (1000, 3, 128), (1, 3, 128), (777, 2, 128),
                                           (300, 1, 128), (4096, 3, 256), (1000, 3, 256),
                                           (777, 2, 256), (300, 1, 256), (1, 3, 256)])
def test_nn_pairs_bf16_parity(n, depth, width):
    import torch

    from paper_2402_12199_gb300 import api

    flat = params(7 + n, depth, width)
    m = api.MLP(width, depth)
    m.set_params(flat)
    cfg7 = inputs.pair_configs(n, 31 + n, 5.0, 9.4)
    out = m.pairs(torch.from_numpy(cfg8(cfg7)).cuda(), "bf16").double().cpu().numpy()
    p = nn.unpack(flat.astype(np.float64), width, depth)
    c = torch.as_tensor(cfg7.astype(np.float64))
    E, Fj, ti, tj = nn.predict_labels(p, c[:, :3], c[:, 3:])
    assert_parity(out[:, 0:3], Fj.numpy(), TOL_BF16)
    assert_parity(out[:, 4:7], ti.numpy(), TOL_BF16)
    assert_parity(out[:, 8:11], tj.numpy(), TOL_BF16)
    assert_parity(out[:, 3], E.detach().numpy(), TOL_BF16)


@pytest.mark.parametrize("width", [128, 256])
def test_nn_system_forces_bf16_parity(width):
    from paper_2402_12199_gb300 import api

    st, L, tmpl = make_state(2000, 0.20, 12)
    flat = params(3, 3, width)
    m = api.MLP(width, 3)
    m.set_params(flat)
    s = gpu_system(st, L)
    r = s.forces_nn(m, "bf16", energy=True)
    s.sync()
    F, T, E, per, pairs = oracle_nn(st, L, tmpl, flat, width)
    assert canonical_margin(st, pairs) > 1e-5
    assert_parity(r["force"][:, :3].double().cpu().numpy(), F, TOL_BF16)
    assert_parity(r["torque"][:, :3].double().cpu().numpy(), T, TOL_BF16)
    assert abs(r["energy"] - E) < TOL_BF16 * np.abs(per).sum()


@pytest.mark.parametrize("width", [128, 256])
def test_nn_bf16_md_steps_run_and_conserve(width):
    from paper_2402_12199_gb300 import api

    st, L, tmpl = make_state(512, 0.2, 6)
    m = api.MLP(width, 3)
    m.set_params(params(4, 3, width))
    s = gpu_system(st, L)
    s.forces_nn(m, "bf16")
    e0 = sum(s.energy())
    s.step(50, 0.002, path=api.RB_PATH_NN, mlp=m, precision="bf16")
    e1 = sum(s.energy())
    s.sync()
    assert abs(e1 - e0) < 1e-2 * 512, (e0, e1)


def test_nn_skin_identical_forces_bf16():
    from paper_2402_12199_gb300 import api

    st, L, tmpl = make_state(3000, 0.2, 72)
    m = api.MLP(128, 3)
    m.set_params(params(11))
    a = gpu_system(st, L)
    b = gpu_system(st, L)
    b.set_skin(0.4)
    ra = a.forces_nn(m, "bf16")
    rb = b.forces_nn(m, "bf16")
    b.sync()
    assert bool((ra["force"] == rb["force"]).all()) and bool((ra["torque"] == rb["torque"]).all())
