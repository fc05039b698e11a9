"""Host-side checks of the C ABI (no GPU needed): the library loads and
exports every entry point include/hps.h declares, argument checks fail with
the documented codes before any device work, and the node layout agrees
with the oracle's."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle as O
from paper_1812_07167_gb300 import build as B
from paper_1812_07167_gb300 import hps

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()


def _declared():
    src = open(os.path.join(ROOT, "include", "hps.h")).read()
    return sorted(set(re.findall(r"\b(hps_[a-zA-Z0-9_]+)\s*\(", src)))


def test_header_and_binding_agree():
    assert _declared() == sorted(hps.EXPORTS)


def test_library_exports_every_declared_symbol():
    L = ctypes.CDLL(hps.LIB_PATH)
    for name in _declared():
        assert hasattr(L, name), name


def test_strerror_codes():
    for code in range(8):
        assert hps.hps_strerror(code)
    assert hps.hps_strerror(99) == "unknown error"


@pytest.mark.parametrize("m,my,p", [(1, 1, 4), (2, 2, 8), (4, 4, 16), (8, 8, 6), (4, 2, 6), (1, 8, 6), (16, 2, 4)])
def test_nodes_match_oracle(m, my, p):
    pr = hps.Problem(m, p, 10.0, 10.0, -1.0, 2.0, 0.5, 1.0, my=my)
    lxy, bxy = hps.hps_nodes(pr)
    olxy, obxy = O.nodes(O.Problem(m, p, 10.0, 10.0, -1.0, 2.0, 0.5, 1.0, my=my))
    np.testing.assert_allclose(lxy, olxy, rtol=0, atol=1e-15)
    np.testing.assert_allclose(bxy, obxy, rtol=0, atol=1e-15)


def _desc(**kw):
    base = dict(x0=0.0, x1=1.0, y0=0.0, y1=1.0, mx=4, my=4, p=8, q=6, kappa=5.0, eta_re=5.0,
                eta_im=0.0, precision=0, fp64_levels=0, refine_steps=0)
    base.update(kw)
    return hps.hps_desc(**base)


@pytest.mark.parametrize("bad", [
    dict(mx=3, my=3), dict(mx=4, my=3), dict(mx=2048, my=2), dict(mx=0, my=0), dict(p=3), dict(p=33), dict(q=65), dict(q=-2),
    dict(kappa=0.0), dict(kappa=-1.0), dict(eta_re=0.0, eta_im=1.0), dict(x1=0.0),
    dict(y1=-1.0), dict(precision=7), dict(precision=-1), dict(kappa=float("nan")),
    dict(precision=1, fp64_levels=-2), dict(fp64_native=2), dict(fp64_native=-1), dict(leaf_form=2),
    dict(leaf_form=-1),
])
def test_invalid_descriptor_is_rejected_before_device_work(bad):
    d = _desc(**bad)
    c = np.ones(4 * 4 * 36)
    h = ctypes.c_void_p()
    assert hps.lib().hps_build(ctypes.byref(d), c.ctypes.data, None, ctypes.byref(h)) == hps.HPS_EINVAL
    assert hps.lib().hps_nodes(ctypes.byref(d), None, None) == hps.HPS_EINVAL
    assert h.value is None


def test_null_arguments():
    d = _desc()
    h = ctypes.c_void_p()
    assert hps.lib().hps_build(ctypes.byref(d), None, None, ctypes.byref(h)) == hps.HPS_EINVAL
    assert hps.lib().hps_build(None, None, None, ctypes.byref(h)) == hps.HPS_EINVAL
    assert hps.lib().hps_solve(None, None, None, None, 1, None) == hps.HPS_EINVAL
    assert hps.lib().hps_root_R(None, None, 0, None) == hps.HPS_EINVAL
    assert hps.lib().hps_leaf_ops(None, 0, None, None, None, None) == hps.HPS_EINVAL
    assert hps.lib().hps_status(None, None, None, None) == hps.HPS_EINVAL
    assert hps.lib().hps_info(None, None) == hps.HPS_EINVAL
    assert hps.lib().hps_free(None) == hps.HPS_OK


def test_memory_cap_refuses_before_allocating(monkeypatch):
    monkeypatch.setenv("HPS_MEM_CAP_BYTES", "1000")
    d = _desc()
    c = np.ones(16 * 36)
    h = ctypes.c_void_p()
    assert hps.lib().hps_build(ctypes.byref(d), c.ctypes.data, None, ctypes.byref(h)) == hps.HPS_ENOMEM


def test_q_zero_means_p_minus_2():
    d = _desc(q=0)
    lxy = np.zeros((16, 60, 2))
    assert hps.lib().hps_nodes(ctypes.byref(d), lxy.ctypes.data, None) == hps.HPS_OK


def test_plan_reports_sizes_without_device_work():
    d = _desc(mx=16, my=16, p=16, q=14, kappa=80.0, eta_re=80.0)
    info = hps.hps_info_t()
    assert hps.lib().hps_plan(ctypes.byref(d), ctypes.byref(info)) == hps.HPS_OK
    assert info.leaves == 256 and info.levels == 8 and info.dof == 256 * 252
    # Sec. 2.4 storage: X = [Psi | Y] and G X per leaf, 7 blocks per merge
    assert 0.39e9 < info.operator_bytes < 0.41e9
    assert info.build_scratch_bytes > 0 and info.solve_ws_bytes_per_rhs > 0
    dm = _desc(mx=16, my=16, p=16, q=14, kappa=80.0, eta_re=80.0, precision=1)
    im = hps.hps_info_t()
    assert hps.lib().hps_plan(ctypes.byref(dm), ctypes.byref(im)) == hps.HPS_OK
    assert im.operator_bytes < 0.6 * info.operator_bytes
    bad = _desc(mx=3, my=3)
    assert hps.lib().hps_plan(ctypes.byref(bad), ctypes.byref(info)) == hps.HPS_EINVAL


def test_zgemm_argument_checks_need_no_device():
    L = hps.lib()
    a = np.zeros(16, complex)
    assert L.hps_zgemm(0, 2, 2, 1, a.ctypes.data, a.ctypes.data, a.ctypes.data, 0, None) == hps.HPS_EINVAL
    assert L.hps_zgemm(2, 2, 2, 1, a.ctypes.data, a.ctypes.data, a.ctypes.data, 4, None) == hps.HPS_EINVAL
    # host arrays are refused (device memory only)
    assert L.hps_zgemm(2, 2, 2, 1, a.ctypes.data, a.ctypes.data, a.ctypes.data, 1, None) == hps.HPS_EINVAL


def test_zinv_and_wait_check_argument_checks_need_no_device():
    L = hps.lib()
    a = np.zeros(16, complex)
    bad = ctypes.c_int(7)
    # n < 2, batch < 1, mode not 0 / 1, host arrays: refused before any device work
    assert L.hps_zinv(1, 1, a.ctypes.data, a.ctypes.data, 0, ctypes.byref(bad), None) == hps.HPS_EINVAL
    assert bad.value == -1
    assert L.hps_zinv(2, 0, a.ctypes.data, a.ctypes.data, 0, None, None) == hps.HPS_EINVAL
    assert L.hps_zinv(2, 1, a.ctypes.data, a.ctypes.data, 2, None, None) == hps.HPS_EINVAL
    assert L.hps_zinv(2, 1, a.ctypes.data, a.ctypes.data, 0, None, None) == hps.HPS_EINVAL
    assert L.hps_check_wait(0, None) == hps.HPS_EINVAL
    assert L.hps_check_wait(2001, None) == hps.HPS_EINVAL


def test_plan_of_a_rectangular_grid():
    info = hps.hps_plan(hps.Problem(8, 16, 40.0, 40.0, my=2))
    assert info.leaves == 16 and info.levels == 4 and info.n_bdry == 2 * (8 + 2) * 14


@pytest.mark.parametrize("form", [hps.HPS_LEAF_LU, hps.HPS_LEAF_INVERSE])
def test_plan_limits_match_the_documented_sizes(form):
    """hps_plan's HPS_ENOTSUP boundary is the one include/hps.h states for
    hps_build: p <= 25, up to 512 leaves a side at p = 16, 256 at p = 24."""
    def code(m, p):
        try:
            hps.hps_plan(hps.Problem(m, p, 10.0, 10.0, leaf_form=form))
            return hps.HPS_OK
        except hps.HPSError as e:
            return e.code
    assert code(1, 25) == hps.HPS_OK
    assert code(1, 26) == hps.HPS_ENOTSUP
    assert code(512, 16) == hps.HPS_OK
    assert code(1024, 16) == hps.HPS_ENOTSUP
    assert code(256, 24) == hps.HPS_OK
    assert code(512, 24) == hps.HPS_ENOTSUP


def test_plan_counts_of_the_two_leaf_forms():
    """hps_plan's flop and byte counts follow the leaf form: the LU form's
    leaf work is n^3/3 + nb n^2 complex multiply-adds; the inverse form's is
    the complex64 inverse (n^3), G X (nb n p) and two refinement steps of two
    n^3 products each (the residual on the tensor cores, the correction), in
    1 + 1 + (4 + 1) + (2 + 1) + 1 launches for one chunk of leaves instead of
    1 (the second step reuses the first one's split of B);
    the LU form stores n row indices and n row scales a leaf beside the
    factors."""
    m, p = 8, 16
    lu = hps.hps_plan(hps.Problem(m, p, 10.0, 10.0, leaf_form=hps.HPS_LEAF_LU))
    inv = hps.hps_plan(hps.Problem(m, p, 10.0, 10.0, leaf_form=hps.HPS_LEAF_INVERSE))
    n, nb, leaves = p * p - 4, 4 * (p - 2), m * m
    assert inv.build_flops - lu.build_flops == leaves * 8 * (
        (n ** 3 + nb * n * p + 2 * 2 * n ** 3) - (n ** 3 // 3 + nb * n * n))
    assert lu.operator_bytes - inv.operator_bytes == leaves * n * (4 + 8)
    assert lu.solve_flops == inv.solve_flops
    assert inv.build_launches == lu.build_launches + 10 and lu.solve_launches == inv.solve_launches


@pytest.mark.parametrize("bad", [float("nan"), float("inf"), -float("inf")])
def test_non_finite_host_coefficients_are_rejected(bad):
    """A host c with a NaN or an infinity is HPS_EINVAL before any device work."""
    d = _desc()
    c = np.ones(4 * 4 * 36)
    c[77] = bad
    h = ctypes.c_void_p()
    assert hps.lib().hps_build(ctypes.byref(d), c.ctypes.data, None, ctypes.byref(h)) == hps.HPS_EINVAL
    assert h.value is None


def test_binding_fails_loudly_without_the_library(monkeypatch):
    """No CPU fallback: with the shared library absent, the first call raises
    instead of computing anything."""
    monkeypatch.setattr(hps, "_lib", None)
    monkeypatch.setattr(hps, "LIB_PATH", os.path.join(os.path.dirname(hps.LIB_PATH), "missing_libhps.so"))
    with pytest.raises(RuntimeError, match="not built"):
        hps.lib()
    with pytest.raises(RuntimeError, match="not built"):
        hps.hps_plan(hps.Problem(4, 8, 10.0, 10.0))


def test_gauss_interface_arguments():
    """q: 0 or p-2 (Chebyshev edge nodes) or 1..64 Gauss-Legendre nodes per
    leaf edge; the mixed path keeps the Chebyshev edges (its refinement
    residual is that system's); a batch shares one q.  Checked before any
    device work."""
    info = hps.hps_info_t()
    for q, code in ((0, hps.HPS_OK), (14, hps.HPS_OK), (1, hps.HPS_OK), (12, hps.HPS_OK), (64, hps.HPS_OK),
                    (65, hps.HPS_EINVAL), (-1, hps.HPS_EINVAL)):
        d = hps.Problem(4, 16, 10.0, 10.0).desc()
        d.q = q
        assert hps.lib().hps_plan(ctypes.byref(d), ctypes.byref(info)) == code, q
        if code == hps.HPS_OK:
            assert info.n_bdry == 2 * 8 * (q or 14)
    dm = hps.Problem(4, 16, 10.0, 10.0, precision=hps.HPS_MIXED, q=12).desc()
    assert hps.lib().hps_plan(ctypes.byref(dm), ctypes.byref(info)) == hps.HPS_ENOTSUP
    ds = (hps.hps_desc * 2)(hps.Problem(4, 8, 10.0, 10.0, q=4).desc(), hps.Problem(4, 8, 10.0, 10.0, q=5).desc())
    c = np.ones(16 * 36)
    cs = (ctypes.c_void_p * 2)(c.ctypes.data, c.ctypes.data)
    hs = (ctypes.c_void_p * 2)()
    assert hps.lib().hps_build_batch(2, ds, cs, None, hs) == hps.HPS_EINVAL
