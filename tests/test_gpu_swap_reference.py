"""rb_pairs_swap_reference (the same sampled pairs described from the other
body, in place) against the FP64 oracle's swap of the same data, against the
oracle's bead sum evaluated afresh at the swapped configurations, and swapped
twice."""
import numpy as np
import pytest

from oracle import bodies, sampler
from paper_2402_12199_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()


def to7(cfg8, lab12):
    c = np.concatenate([cfg8[:, :3], cfg8[:, 4:8]], axis=1)
    l = np.concatenate([lab12[:, 3:4], lab12[:, 0:3], lab12[:, 4:7], lab12[:, 8:11]], axis=1)
    return c, l


@pytest.mark.parametrize("shape", ["cube", "cylinder"])
def test_swap_reference_matches_oracle_and_fresh_bead_labels(shape):
    import torch

    from paper_2402_12199_gb300 import api

    s = api.System(8, [70.0] * 3, shape)
    u = torch.from_numpy(inputs.sampler_uniforms(64, 61)).cuda()
    cfg, lab, _ = api.sample_pairs(s, u)
    c0, l0 = to7(cfg.double().cpu().numpy(), lab.double().cpu().numpy())
    api.pairs_swap_reference(cfg, lab)
    torch.cuda.synchronize()
    c1, l1 = to7(cfg.double().cpu().numpy(), lab.double().cpu().numpy())
    # the oracle's swap of the same (FP32) data
    rc, rl = sampler.swap_reference(c0, l0)
    assert np.abs(c1 - rc).max() < 1e-5 * max(1.0, np.abs(rc).max())
    scale = np.abs(rl).max()
    assert np.abs(l1 - rl).max() < 1e-5 * scale
    # exact physics: the bead sum of the swapped configurations
    tmpl = bodies.cube_template() if shape == "cube" else bodies.cylinder_template()
    fresh = sampler.label_pairs(c1[:16], tmpl)
    assert np.abs(l1[:16] - fresh).max() < 1e-4 * np.abs(fresh).max()
    # twice: back to the start (FP32 rounding)
    api.pairs_swap_reference(cfg, lab)
    torch.cuda.synchronize()
    c2, l2 = to7(cfg.double().cpu().numpy(), lab.double().cpu().numpy())
    assert np.abs(c2 - c0).max() < 1e-5 * max(1.0, np.abs(c0).max())
    assert np.abs(l2 - l0).max() < 1e-5 * np.abs(l0).max()


def test_swap_reference_configurations_only_and_empty():
    import torch

    from paper_2402_12199_gb300 import api

    s = api.System(8, [60.0] * 3, "cube")
    u = torch.from_numpy(inputs.sampler_uniforms(10, 62)).cuda()
    cfg, lab, _ = api.sample_pairs(s, u)
    c = cfg.clone()
    api.pairs_swap_reference(c)  # no labels
    api.pairs_swap_reference(cfg, lab)
    torch.cuda.synchronize()
    assert torch.equal(c, cfg)
    api.pairs_swap_reference(torch.zeros((0, 8), device="cuda"))
