"""The C ABI library builds, loads and exports every symbol declared in
include/*.h (no compute: runs without a GPU)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*[A-Za-z_][\w\s\*]*?\b(rb_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2402_12199_gb300 import _lib, build_lib

    build_lib.build()
    return ctypes.CDLL(_lib.SO)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["rb_create_system", "rb_forces_beads", "rb_forces_nn", "rb_step",
                     "rb_energy", "rb_nn_pairs", "rb_mlp_create"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_signatures_cover_exports(lib):
    from paper_2402_12199_gb300 import _lib

    for n in _lib.SIGNATURES:
        assert hasattr(lib, n), n


def test_library_reports_version_without_gpu(lib):
    lib.rb_abi_version.restype = ctypes.c_int32
    assert lib.rb_abi_version() >= 1
    lib.rb_mlp_n_params.restype = ctypes.c_int64
    lib.rb_mlp_n_params.argtypes = [ctypes.c_int32, ctypes.c_int32]
    assert lib.rb_mlp_n_params(128, 3) == 2 * 10 + 128 * 10 + 128 + 2 * (128 * 128 + 128) + 128 + 3
    assert lib.rb_mlp_n_params(0, 3) < 0


@pytest.mark.parametrize("shape", ["cube", "cylinder", "box", "cut cube"])
def test_template_symmetry_matches_the_oracle_without_gpu(lib, shape):
    """rb_template_symmetry (host code) finds the same point group, in the same
    order, as the oracle's independent search."""
    import numpy as np

    from oracle import bodies, symmetry
    from paper_2402_12199_gb300 import api

    tmpl = {"cube": bodies.cube_template(), "cylinder": bodies.cylinder_template(),
            "box": np.stack(np.meshgrid(np.arange(3) - 1.0, np.arange(4) - 1.5,
                                        np.arange(6) - 2.5, indexing="ij"), -1).reshape(-1, 3),
            "cut cube": bodies.cube_template()[:-1]}[shape]
    q, inv = api.template_symmetry(tmpl)
    qo, invo = symmetry.point_group(tmpl)
    assert inv == invo
    assert q.shape == qo.shape
    np.testing.assert_allclose(q, qo, atol=1e-7)


def test_fnet_parameter_count_matches_the_oracle_layout_without_gpu(lib):
    from oracle import fnet

    lib.rb_fnet_n_params.restype = ctypes.c_int64
    lib.rb_fnet_n_params.argtypes = [ctypes.c_int32, ctypes.c_int32]
    for w, d in ((16, 1), (32, 3), (64, 2)):
        assert lib.rb_fnet_n_params(w, d) == 5 * fnet.net_size(w, d)
    assert lib.rb_fnet_n_params(0, 3) == -1
    assert lib.rb_fnet_n_params(32, 0) == -1


def test_system_footprint_without_gpu(lib):
    from paper_2402_12199_gb300 import api

    lib.rb_system_footprint.restype = ctypes.c_int64
    lib.rb_system_footprint.argtypes = [ctypes.c_void_p]
    sizes = []
    for n in (1000, 2000, 4000):
        d = api._desc(n, [200.0] * 3, "cube")
        sizes.append(lib.rb_system_footprint(ctypes.byref(d)))
    assert all(b > 0 for b in sizes)
    # linear in the body count at a fixed box: equal increments
    assert sizes[2] - sizes[1] == 2 * (sizes[1] - sizes[0])
    bad = api._desc(1, [200.0] * 3, "cube")
    bad.n_bodies = 0
    assert lib.rb_system_footprint(ctypes.byref(bad)) == -1
    assert lib.rb_system_footprint(None) == -1
