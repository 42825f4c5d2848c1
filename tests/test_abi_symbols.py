"""CPU checks of the C-ABI library: it loads without a GPU and exports every
function that include/vne.h declares; the host-only colouring matches the
oracle's greedy colouring."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2212_09642_gb300 import _build, vne
    _build.build()
    return vne.load()


def _declared():
    hdr = open(os.path.join(ROOT, "include", "vne.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    return sorted(set(re.findall(r"\b(vne_[a-z0-9_]+)\s*\(", hdr)))


def test_header_declares_the_boundary():
    names = _declared()
    for required in ["vne_create_density_matrix", "vne_entropy_hutchinson", "vne_entropy_hutchpp",
                     "vne_entropy_probing", "vne_quadform_batch"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_declares_every_header_function(lib):
    from paper_2212_09642_gb300 import vne
    assert set(_declared()) <= set(vne.exported_symbols())


def test_version_and_options_without_gpu(lib):
    from paper_2212_09642_gb300 import vne
    assert "sm_103a" in vne.vne_version()
    o = vne.options()
    assert o.reorth == -1 and o.n_inf_poles == 2 and o.cg_tol == 1e-8


@pytest.mark.parametrize("d", [1, 2, 3])
def test_host_greedy_coloring_matches_oracle(lib, d):
    from oracle import coloring
    from paper_2212_09642_gb300 import graphs, vne
    for g in (graphs.barabasi_albert(400, 3, 5), graphs.random_geometric(500, 0.08, 2), graphs.grid2d(9, 11)):
        got, s = vne.vne_greedy_coloring(g.n, g.rowptr, g.col, d)
        want = coloring.greedy_distance_coloring(g, d)
        assert np.array_equal(got, want)
        assert s == want.max() + 1


def test_null_handles_are_rejected_without_a_gpu(lib):
    """Every entry point checks its handle before touching the device."""
    from paper_2212_09642_gb300 import vne
    k = __import__("ctypes").c_int32()
    assert lib.vne_matrix_coloring(None, 2, None, None, None) == vne.VNE_EINVAL
    assert lib.vne_entropy_probing_auto(None, 1e-3, 30, 8, vne._COLORING_FN(), None, None, None, None) == vne.VNE_EINVAL
    assert lib.vne_ctx_last_poly_dim(None, __import__("ctypes").byref(k)) == vne.VNE_EINVAL
    assert lib.vne_ctx_last_steps(None, __import__("ctypes").byref(k)) == vne.VNE_EINVAL
    assert lib.vne_entropy_probing(None, None, 2, 30, None, 0, None, None, None) == vne.VNE_EINVAL


def test_options_layout_matches_the_header(lib):
    """The binding's vne_options has the C struct's size (defaults written by
    the library land in the right fields)."""
    from paper_2212_09642_gb300 import vne
    o = vne.options()
    assert o.quad_tol == 0.0 and o.check_every == 0 and o.spectrum_min == 0.0 and o.probe_offset == 0
    assert vne.vne_probing_report.eps_abs.offset == 24 and __import__("ctypes").sizeof(vne.vne_probing_report) == 80
