"""The FP32-accurate tensor-core GEMM of the training pass (rb_gemm_f32:
split TF32 operands, three tcgen05 products, FP32 accumulation) against the
FP64 product of the same FP32 operands, on the training shapes (batch-long
forward and reverse products, the split-K weight gradients with a transposed
operand), ragged shapes over several tiles, a single row, K = 0, and alpha /
beta.  Operand rows span six decades.  The bounds are relative to
sum_k |a_mk b_kn|: at most 2e-5, with the median within the FP32 accumulation
error (1e-6 + 1e-7 sqrt(K)); an unsplit TF32 product (2^-11 per product, about
4e-5 of the scale at K = 128) or a dropped cross term fails them."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()


def _operand(rng, rows, cols):
    x = rng.standard_normal((rows, cols))
    x *= 10.0 ** rng.uniform(-3, 3, size=(rows, 1))
    return x.astype(np.float32)


def _check(M, N, K, a_t=False, b_t=False, alpha=1.0, beta=0.0, seed=0, split_k=True):
    import torch

    from paper_2402_12199_gb300 import api

    rng = np.random.default_rng(seed)
    A = _operand(rng, K, M).T if a_t else _operand(rng, M, K)  # a_t: unit stride along M
    B = _operand(rng, N, K).T if b_t else _operand(rng, K, N)
    C0 = rng.standard_normal((M, N)).astype(np.float32)
    At = torch.from_numpy(np.ascontiguousarray(A.T)).cuda().T if a_t else torch.from_numpy(A).cuda()
    Bt = torch.from_numpy(np.ascontiguousarray(B.T)).cuda().T if b_t else torch.from_numpy(B).cuda()
    assert (At.stride(0) == 1) == (a_t and M > 1) or K <= 1
    C = torch.from_numpy(C0.copy()).cuda()
    api.gemm_f32(At, Bt, C, alpha, beta, split_k)
    got = C.double().cpu().numpy()
    A64, B64 = A.astype(np.float64), B.astype(np.float64)
    ref = alpha * (A64 @ B64) + beta * C0.astype(np.float64)
    scale = np.abs(alpha) * (np.abs(A64) @ np.abs(B64)) + np.abs(beta * C0) + 1e-30
    err = np.abs(got - ref) / scale
    assert err.max() < 2e-5, (M, N, K, err.max())
    if K >= 8:  # FP32 accumulation: about 2^-24 sqrt(K) of sum |a b| for a long K
        assert np.median(err) < 1e-6 + 1e-7 * np.sqrt(K), (M, N, K, np.median(err))
    return err


@pytest.mark.parametrize("M,N,K", [(4096, 128, 128), (4096, 256, 256), (4096, 128, 16),
                                   (4096, 256, 16), (1000, 48, 100), (129, 17, 33), (1, 32, 700)])
def test_products(M, N, K):
    _check(M, N, K, seed=M + N + K)


@pytest.mark.parametrize("M,N,K", [(128, 128, 4096), (256, 256, 4096), (128, 16, 4096),
                                   (32, 4, 4096), (100, 40, 1500)])
@pytest.mark.parametrize("split_k", [True, False])
def test_weight_gradients_split_k(M, N, K, split_k):
    # gW[o][i] = sum_b G[b][o] H[b][i]: A = G^T with unit stride along M
    _check(M, N, K, a_t=True, split_k=split_k, seed=M * N + K)


def test_transposed_b_alpha_beta_and_empty_k():
    _check(300, 64, 96, b_t=True, alpha=-0.5, beta=0.75, seed=1)
    _check(300, 64, 1200, a_t=True, b_t=True, alpha=2.0, beta=1.0, seed=2)
    _check(77, 33, 0, alpha=1.0, beta=0.5, seed=3)


def test_split_k_is_deterministic():
    import torch

    from paper_2402_12199_gb300 import api

    rng = np.random.default_rng(7)
    A = torch.from_numpy(_operand(rng, 4096, 128)).cuda().T  # 128 x 4096, unit stride along M
    B = torch.from_numpy(_operand(rng, 4096, 128)).cuda()
    c1 = api.gemm_f32(A, B)
    c2 = api.gemm_f32(A, B)
    assert torch.equal(c1, c2)
