"""The C-ABI library builds, loads and exports every entry point that
include/feast.h declares; host-only entry points agree with the oracle.
No compute call touches a GPU here."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
import paper_1605_08771_gb300 as fg

HEADER = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "feast.h")


@pytest.fixture(scope="module")
def L():
    fg.build_library()
    return fg.lib()


def declared():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"\b(feast_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared()
    for required in ["feast_init", "feast_interval_solve", "feast_filter_apply", "feast_finalize",
                     "feast_strerror", "feast_opts_default"]:
        assert required in names


def test_every_declared_symbol_is_exported(L):
    for name in declared():
        assert hasattr(L, name), name
    assert sorted(fg.EXPORTS) == declared()


def test_contour_nodes_match_oracle(L):
    for (a, b, nc, asp) in [(-1.0, 1.0, 8, 1.0), (0.5, 3.0, 3, 1.0), (-7.0, 2.0, 16, 0.3), (1.0, 2.0, 1, 1.0)]:
        z, w = fg.feast_contour_nodes(a, b, nc, asp)
        zo, wo = oracle.contour_nodes(a, b, nc, asp)
        np.testing.assert_allclose(z, zo, rtol=0, atol=1e-14 * max(1, abs(a), abs(b)))
        np.testing.assert_allclose(w, wo, rtol=0, atol=1e-14 * max(1, abs(a), abs(b)))


def test_opts_default(L):
    o = fg.feast_opts_default()
    assert (o.variant, o.s, o.prec, o.max_iter, o.refine_max) == (0, 3, 0, 100, 10)
    assert o.aspect == 1.0 and o.anorm == 0.0 and o.x0 is None


def test_argument_errors_without_device(L):
    evals = np.zeros(4)
    res = np.zeros(4)
    mf, it = ctypes.c_int(), ctypes.c_int()
    dp = ctypes.POINTER(ctypes.c_double)
    code = L.feast_interval_solve(None, None, 0, 10, 10, -1.0, 1.0, 4, 8, 1e-10, None,
                                  evals.ctypes.data_as(dp), None, res.ctypes.data_as(dp),
                                  ctypes.byref(mf), ctypes.byref(it), None)
    assert code == -1
    z = np.zeros(4)
    assert L.feast_contour_nodes(1.0, -1.0, 2, 1.0, z.ctypes.data_as(dp), z.ctypes.data_as(dp)) == -1
    assert L.feast_contour_nodes(-1.0, 1.0, 0, 1.0, z.ctypes.data_as(dp), z.ctypes.data_as(dp)) == -1
    assert fg.feast_strerror(-5).startswith("subspace size")
    assert fg.feast_strerror(0) == "success"


def test_offset_contour_nodes_match_oracle(L):
    # the moved-node interpolatory rule: library (host code) against the oracle
    for (a, b, nc) in [(-1.0, 1.0, 8), (0.5, 3.0, 3), (-7.0, 2.0, 16)]:
        d = 0.2 * np.sin(np.arange(nc) + 1.0)
        z, w = fg.feast_contour_nodes_offset(a, b, nc, d)
        zo, wo = oracle.quadrature.contour_nodes_offset(a, b, nc, d)
        np.testing.assert_allclose(z, zo, rtol=0, atol=1e-13 * max(1, abs(a), abs(b)))
        np.testing.assert_allclose(w, wo, rtol=0, atol=1e-13 * max(1, abs(a), abs(b)))
        z0, w0 = fg.feast_contour_nodes_offset(a, b, nc, np.zeros(nc))
        zg, wg = fg.feast_contour_nodes(a, b, nc, 1.0)
        np.testing.assert_allclose(z0, zg, atol=1e-14 * max(1, abs(a), abs(b)))
    with pytest.raises(fg.FeastError):
        fg.feast_contour_nodes_offset(-1.0, 1.0, 8, np.array([0, 0, 0, 3.0, -3.0, 0, 0, 0]))


def test_moments_count_matches_oracle(L):
    from oracle.density import count_estimate, exact_moments
    lam = np.concatenate([np.linspace(-9, -2, 70), np.linspace(-0.6, 0.6, 25), np.linspace(2, 9, 70)])
    mu = exact_moments(lam, 0.0, 10.0, 64)
    for (a, b) in [(-1.3, 1.3), (-10.0, 10.0), (0.1, 5.0)]:
        assert abs(fg.feast_moments_count(mu, 0.0, 10.0, a, b, lam.size)
                   - count_estimate(mu, 0.0, 10.0, a, b, lam.size)) < 1e-9
    assert fg.feast_mlp_param_count() == 64 * 256 + 256 + 2 * (256 * 256 + 256) + 256 * 9 + 9


def test_circle_nodes_match_oracle(L):
    # the whole-circle rule of general matrices: library (host code) against
    # the oracle
    for (c, r, nc) in [(0.0, 1.0, 8), (0.3 - 0.7j, 2.5, 5), (-4.0 + 1.0j, 0.01, 16), (1.0j, 3.0, 1)]:
        z, w = fg.feast_circle_nodes(c, r, nc)
        zo, wo = oracle.quadrature.circle_nodes(c, r, nc)
        scale = max(1.0, abs(c), r)
        np.testing.assert_allclose(z, zo, rtol=0, atol=1e-14 * scale)
        np.testing.assert_allclose(w, wo, rtol=0, atol=1e-14 * scale)
    dp = ctypes.POINTER(ctypes.c_double)
    z = np.zeros(8)
    assert L.feast_circle_nodes(0.0, 0.0, -1.0, 2, z.ctypes.data_as(dp), z.ctypes.data_as(dp)) == -1
    assert L.feast_circle_nodes(0.0, 0.0, 1.0, 0, z.ctypes.data_as(dp), z.ctypes.data_as(dp)) == -1
    assert L.feast_circle_nodes(float("nan"), 0.0, 1.0, 2, z.ctypes.data_as(dp), z.ctypes.data_as(dp)) == -1
