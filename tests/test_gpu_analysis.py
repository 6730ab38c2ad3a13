"""GPU analyses against the oracle: g(r) bin counts against the oracle's FP64
counts from the plain definition before and after MD (exact, except that a
pair within FP32 rounding of a bin edge may land in the neighbouring bin),
g(r) normalisation,
MSD and MSR of free flight and free rotation against their closed forms, and
MSD / MSR of an interacting run against the oracle's FP64 evaluation of the
GPU's own state and image counters."""
import numpy as np
import pytest

from oracle import analysis, bodies
from tests.helpers import gpu_system, make_state

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()


def edge_tol(L, r_max):
    """Bound on the FP32 error of a minimum-image distance: each component of
    p_j - p_i is rounded once at the scale of the box (half an ulp of L),
    sqrt and the bin scale add ~1e-7 relative; 1e-5 r_max is several times
    that for the boxes here."""
    ulp = np.spacing(np.float32(L)).astype(np.float64)
    bound = np.sqrt(3.0) * 0.5 * ulp + 4e-7 * r_max
    tol = 1e-5 * r_max
    assert tol > 3 * bound
    return tol


def check_counts(got, ref, edges):
    """Integer counts from the GPU against the oracle's: a bin may differ only
    by pairs within FP32 rounding of one of its two edges, the total only by
    pairs at r_max, and the sum of the differences by at most two per such
    pair."""
    got = np.asarray(got, dtype=np.int64)
    d = np.abs(got - ref)
    assert np.all(d <= edges[:-1] + edges[1:]), np.nonzero(d > edges[:-1] + edges[1:])
    assert abs(got.sum() - ref.sum()) <= edges[-1]
    assert d.sum() <= 2 * edges.sum()
    return int(d.sum())


@pytest.mark.parametrize("r_max,n_bins", [(9.0, 180), (8.6, 7), (9.3, 4096)])
def test_gr_counts_match_definition(r_max, n_bins):
    st, L, tmpl = make_state(4096, 0.20, 41)
    s = gpu_system(st, L)
    s.set_skin(0.3)
    tol = edge_tol(L, r_max)
    c0 = s.gr_counts(r_max, n_bins).cpu().numpy()
    ref0 = analysis.gr_counts(st["pos"], [L] * 3, r_max, n_bins)
    check_counts(c0, ref0, analysis.gr_edge_counts(st["pos"], [L] * 3, r_max, n_bins, tol))
    s.step(60, 0.004)
    pos = s.get_state(to_host=True)["pos"]
    c1 = s.gr_counts(r_max, n_bins).cpu().numpy()
    ref1 = analysis.gr_counts(pos, [L] * 3, r_max, n_bins)
    check_counts(c1, ref1, analysis.gr_edge_counts(pos, [L] * 3, r_max, n_bins, tol))
    assert ref1.sum() > 0


def test_gr_accumulates_and_normalises():
    st, L, tmpl = make_state(2000, 0.15, 42)
    s = gpu_system(st, L)
    tol = edge_tol(L, 9.0)
    c = s.gr_counts(9.0, 90)
    ref = analysis.gr_counts(st["pos"], [L] * 3, 9.0, 90)
    edges = analysis.gr_edge_counts(st["pos"], [L] * 3, 9.0, 90, tol)
    s.step(20, 0.004)
    c = s.gr_counts(9.0, 90, c)
    pos = s.get_state(to_host=True)["pos"]
    ref = ref + analysis.gr_counts(pos, [L] * 3, 9.0, 90)
    edges = edges + analysis.gr_edge_counts(pos, [L] * 3, 9.0, 90, tol)
    counts = c.cpu().numpy().astype(np.int64)
    check_counts(counts, ref, edges)
    g = s.gr_normalise(counts, 9.0, 2)
    np.testing.assert_allclose(g, analysis.gr_normalise(counts, 9.0, 2, 2000, L ** 3), rtol=1e-12)


def test_msd_msr_of_free_bodies_match_closed_forms():
    """Dilute cubes all drifting with one velocity (so no two ever meet) across
    the periodic box, each a freely rotating spherical top: MSD = |v|^2 t^2
    and MSR = <sin^2(|L| t / (2 I))>."""
    st, L, tmpl = make_state(512, 0.001, 43)
    st = dict(st)
    st["vel"] = np.zeros_like(st["vel"])
    st["vel"][:, :3] = np.array([61.0, -47.5, 38.25], dtype=np.float32)
    st["angmom"] = st["angmom"] * 3.0
    s = gpu_system(st, L)
    assert s.build_pairs() == 0
    s.set_reference()
    dt, n = 0.01, 400
    s.step(n, dt)
    msd, msr = s.msd_msr()
    img = s.images()
    s.sync()
    assert np.abs(img[:, :3]).max() >= 1  # crossed the box
    t = dt * n
    v = st["vel"][:, :3].astype(np.float64)
    assert msd == pytest.approx(np.mean(np.sum(v * v, axis=1)) * t * t, rel=1e-5)
    w = np.linalg.norm(st["angmom"][:, :3].astype(np.float64), axis=1) / 500.0
    assert msr == pytest.approx(np.mean(np.sin(0.5 * w * t) ** 2), rel=1e-4)


def test_msd_msr_match_oracle_on_interacting_run():
    st, L, tmpl = make_state(1000, 0.20, 44)
    st = dict(st)
    st["vel"] = st["vel"] * 10.0
    # put the outermost lattice layer 0.1 sigma inside the x = L face, so
    # centres cross it within the run
    st["pos"] = st["pos"].copy()
    st["pos"][:, 0] = np.mod(st["pos"][:, 0] + (L - 0.1 - st["pos"][:, 0].max()), L)
    s = gpu_system(st, L)
    s.step(10, 0.002)
    ref = s.get_state(to_host=True)
    ref_img = s.images()
    s.set_reference()
    s.step(200, 0.002)
    cur = s.get_state(to_host=True)
    img = s.images()
    msd, msr = s.msd_msr()
    s.sync()
    assert np.abs(img - ref_img).max() >= 1
    box = np.array([L] * 3)
    assert msd == pytest.approx(analysis.msd(cur["pos"], img, ref["pos"], ref_img, box), rel=1e-12)
    assert msr == pytest.approx(analysis.msr(cur["quat"], ref["quat"]), rel=1e-12)


def test_images_reset_by_set_state_and_reference_required():
    import torch

    from paper_2402_12199_gb300 import api

    st, L, tmpl = make_state(200, 0.01, 45)
    st = dict(st)
    st["vel"] = st["vel"] * 2000.0
    s = gpu_system(st, L)
    with pytest.raises(api.RBError):
        s.msd_msr()
    s.step(100, 0.01)
    assert np.abs(s.images()).max() >= 1
    s.set_state(torch.from_numpy(st["pos"]).cuda())
    assert np.abs(s.images()).max() == 0
    with pytest.raises(api.RBError):
        s.gr_counts(bodies.pair_cutoff(tmpl) + 1.0, 10)
