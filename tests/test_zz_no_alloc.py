"""rb_forces_beads_noalloc: the allocation-free bead-sum entry point for callers
that cannot call cudaMalloc.  Its results must match rb_forces_beads (the
entry point that owns its memory) on the same state, on two calls in a row
(the second reuses the shared fixed-size scratch left by the first)."""
import ctypes

import numpy as np
import pytest

from tests.helpers import TOL_F32, assert_parity, gpu_system, make_state, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    from paper_2402_12199_gb300 import _lib

    __graft_entry__.build()
    L = ctypes.CDLL(_lib.SO)
    f = L.rb_forces_beads_noalloc
    f.restype = ctypes.c_int32
    f.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.POINTER(ctypes.c_float), ctypes.c_float,
                  ctypes.c_float, ctypes.c_float, ctypes.c_void_p, ctypes.c_void_p,
                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    L.rb_last_error.restype = ctypes.c_char_p
    return L


def call_noalloc(lib, st, L, shape_id=0):
    import torch

    n = len(st["pos"])
    pos = torch.from_numpy(st["pos"]).cuda()
    quat = torch.from_numpy(st["quat"]).cuda()
    F = torch.full((n, 4), float("nan"), device="cuda")
    T = torch.full((n, 4), float("nan"), device="cuda")
    box = (ctypes.c_float * 3)(L, L, L)
    rc = lib.rb_forces_beads_noalloc(shape_id, n, box, 1.0, 1.0, 2.5, pos.data_ptr(),
                                     quat.data_ptr(), F.data_ptr(), T.data_ptr(),
                                     torch.cuda.current_stream().cuda_stream)
    return rc, F, T


@pytest.mark.parametrize("shape,shape_id,phi", [("cube", 0, (0.20, 0.12)), ("cylinder", 1, (0.15, 0.10))])
def test_noalloc_matches_allocating_entry_point_twice(lib, shape, shape_id, phi):
    """The cube (125 beads, five-bead columns) and the cylinder (152 beads,
    eight-bead columns, the kernel instance for templates above 128 beads)."""
    cases = [make_state(1500, phi[0], 21, shape), make_state(700, phi[1], 22, shape)]
    for st, L, _ in cases:
        rc, F, T = call_noalloc(lib, st, L, shape_id)
        assert rc == 0, lib.rb_last_error().decode()
        ref = gpu_system(st, L, shape).forces_beads()
        Fr = ref["force"].double().cpu().numpy()
        Tr = ref["torque"].double().cpu().numpy()
        assert np.isfinite(F.cpu().numpy()).all()
        assert_parity(F[:, :3].double().cpu().numpy(), Fr[:, :3], TOL_F32)
        assert_parity(T[:, :3].double().cpu().numpy(), Tr[:, :3], TOL_F32)
        assert np.abs(F[:, 3].double().cpu().numpy() - Fr[:, 3]).max() <= TOL_F32 * max(
            1.0, np.abs(Fr[:, 3]).max())


def test_noalloc_rejects_sizes_beyond_its_limit(lib):
    st, L, _ = make_state(2049, 0.20, 23)
    rc, F, T = call_noalloc(lib, st, L)
    assert rc == 1
    assert b"2048" in lib.rb_last_error()
