"""Ragged batches of independent problems built together (hps_build_batch).

Every problem of a batch is compared with the same problem built alone
(solutions and root operators within 1e-12 relative for FP64: the batch runs
the same kernels, only their launch shapes differ), and samples of them with
the oracle at the parity bar (1e-10 FP64, 1e-8 mixed after refinement).
"""
import os

import numpy as np
import pytest

import oracle as O
from paper_1812_07167_gb300 import hps
from paper_1812_07167_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def device():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    hps.lib()
    yield


def _rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def _solve(h, s, t):
    pr = h.pr
    u = torch.empty((s.shape[0], pr.leaves, pr.n), dtype=torch.complex128, device="cuda")
    hps.hps_solve(h, torch.from_numpy(s).cuda(), torch.from_numpy(t).cuda(), u, s.shape[0],
                  torch.cuda.current_stream())
    torch.cuda.synchronize()
    return u.cpu().numpy()


def _root(h):
    R = np.zeros((h.pr.nbdry, h.pr.nbdry), complex)
    hps.hps_root_R(h, R, torch.cuda.current_stream())
    return R


def _problems(spec, p, precision=hps.HPS_FP64, leaf_form=hps.HPS_LEAF_LU):
    probs, cs = [], []
    for k, (m, kappa, eta, dom) in enumerate(spec):
        probs.append(hps.Problem(m, p, kappa, eta, *dom, precision=precision, leaf_form=leaf_form))
        c, _, _ = W.random_data(m, p, kappa, eta, seed=500 + k)
        cs.append(c)
    return probs, cs


def _check_against_alone(probs, cs, tol, nrhs=2, tol_R=None):
    st = torch.cuda.current_stream()
    hb = hps.hps_build_batch(probs, [torch.from_numpy(c).cuda() for c in cs], st)
    assert hps.hps_status(hb[0], st)[0] == hps.HPS_OK
    for k, (pr, c) in enumerate(zip(probs, cs)):
        ha = hps.hps_build(pr, torch.from_numpy(c).cuda(), st)
        _, s, t = W.random_data(pr.m, pr.p, pr.kappa, pr.eta, seed=900 + k, nrhs=nrhs, my=pr.ny)
        assert _rel(_solve(hb[k], s, t), _solve(ha, s, t)) < tol, (k, pr)
        # the root operator of a mixed build carries complex64 rounding from
        # the lower levels (no refinement acts on it)
        assert _rel(_root(hb[k]), _root(ha)) < (tol_R or tol), (k, pr)
        assert hb[k].info().operator_bytes == ha.info().operator_bytes
        ha.free()
    return hb


@pytest.mark.parametrize("form", [hps.HPS_LEAF_LU, hps.HPS_LEAF_INVERSE])
def test_ragged_fp64_batch_matches_separate_builds(form):
    spec = [(4, 20.0, 20.0, (0, 1, 0, 1)), (1, 7.0, 3.0 + 1.0j, (0, 1, 0, 0.5)),
            (8, 30.0, 30.0, (0, 1, 0, 1)), (2, 9.0, 9.0 - 2.0j, (-1, 1, 0, 1)),
            (4, 15.0, 6.0, (0, 2, 0, 1)), (8, 25.0, 25.0, (0, 1, 0, 1))]
    probs, cs = _problems(spec, 12, leaf_form=form)
    hb = _check_against_alone(probs, cs, 1e-12)
    for h in hb:
        h.free()


@pytest.mark.parametrize("k", [0, 3])
def test_batch_member_against_oracle(k):
    spec = [(8, 30.0, 30.0, (0, 1, 0, 1)), (4, 12.0, 5.0 + 1.0j, (0, 2, 0, 1)),
            (2, 9.0, 9.0, (0, 1, 0, 1)), (4, 20.0, 20.0, (0, 1, 0, 0.5))]
    probs, cs = _problems(spec, 10)
    st = torch.cuda.current_stream()
    hb = hps.hps_build_batch(probs, cs, st)  # host c
    pr = probs[k]
    _, s, t = W.random_data(pr.m, pr.p, pr.kappa, pr.eta, seed=77, nrhs=2)
    u = _solve(hb[k], s, t)
    opr = O.Problem(pr.m, pr.p, pr.kappa, pr.eta, pr.x0, pr.x1, pr.y0, pr.y1)
    nt = os.cpu_count() or 1
    with O.Tree(opr, cs[k], nthreads=nt) as T:
        uo = T.solve(s, t, nthreads=nt)
        Ro = T.root_R()
    assert _rel(u, uo) < 1e-10
    assert _rel(_root(hb[k]), Ro) < 1e-10
    for h in hb:
        h.free()


def test_config4_shape_fp64_and_mixed():
    """m in {8, 16, 32}, p = 16, kappa in [20, 200], random media: the ragged
    batching workload at reduced count."""
    rng = W.uniform(100, 12)
    spec = []
    for k in range(6):
        m = (8, 16, 32)[int(rng[2 * k] * 3)]
        kap = 20.0 + 180.0 * rng[2 * k + 1]
        spec.append((m, kap, kap, (0, 1, 0, 1)))
    probs, cs = _problems(spec, 16)
    hb = _check_against_alone(probs, cs, 1e-12, nrhs=1)
    for h in hb:
        h.free()
    pm, _ = _problems(spec, 16, hps.HPS_MIXED)
    hm = _check_against_alone(pm, cs, 1e-9, nrhs=1, tol_R=1e-4)
    # the mixed members reach the FP64 solution after refinement
    hf = hps.hps_build_batch(probs, cs, torch.cuda.current_stream())
    for k in range(len(spec)):
        _, s, t = W.random_data(spec[k][0], 16, spec[k][1], spec[k][2], seed=3, nrhs=1)
        assert _rel(_solve(hm[k], s, t), _solve(hf[k], s, t)) < 1e-8
    for h in hm + hf:
        h.free()


def test_handles_outlive_each_other():
    spec = [(4, 10.0, 10.0, (0, 1, 0, 1)), (2, 8.0, 8.0, (0, 1, 0, 1)), (4, 12.0, 12.0, (0, 1, 0, 1))]
    probs, cs = _problems(spec, 8)
    hb = hps.hps_build_batch(probs, cs, torch.cuda.current_stream())
    _, s, t = W.random_data(4, 8, 12.0, 12.0, seed=1)
    before = _solve(hb[2], s, t)
    hb[0].free()
    hb[1].free()
    assert np.array_equal(_solve(hb[2], s, t), before)
    hb[2].free()


def test_batch_argument_errors():
    L = hps.lib()
    assert L.hps_build_batch(0, None, None, None, None) == hps.HPS_OK
    assert L.hps_build_batch(-1, None, None, None, None) == hps.HPS_EINVAL
    probs = [hps.Problem(2, 8, 5.0, 5.0), hps.Problem(2, 10, 5.0, 5.0)]
    cs = [np.ones((4, 36)), np.ones((4, 64))]
    with pytest.raises(hps.HPSError) as e:
        hps.hps_build_batch(probs, cs)
    assert e.value.code == hps.HPS_EINVAL
    probs = [hps.Problem(2, 8, 5.0, 5.0), hps.Problem(2, 8, 5.0, 5.0, precision=hps.HPS_MIXED)]
    with pytest.raises(hps.HPSError) as e:
        hps.hps_build_batch(probs, [np.ones((4, 36))] * 2)
    assert e.value.code == hps.HPS_EINVAL
    probs = [hps.Problem(2, 8, 5.0, 5.0), hps.Problem(2, 8, 5.0, 5.0, leaf_form=hps.HPS_LEAF_INVERSE)]
    with pytest.raises(hps.HPSError) as e:
        hps.hps_build_batch(probs, [np.ones((4, 36))] * 2)
    assert e.value.code == hps.HPS_EINVAL


@pytest.mark.parametrize("m,precision,form", [(1, 0, 0), (4, 0, 0), (16, 0, 0), (64, 0, 0), (16, 1, 0), (64, 1, 0),
                                              (16, 0, 1), (64, 1, 1)])
def test_planned_launch_count_is_what_the_build_launches(m, precision, form):
    pr = hps.Problem(m, 16, 40.0, 40.0, precision=precision, leaf_form=form)
    c, _, _ = W.random_data(m, 16, 40.0, 40.0, seed=2)
    h = hps.hps_build(pr, torch.from_numpy(c).cuda(), torch.cuda.current_stream())
    assert h.info().build_launches == hps.hps_plan(pr).build_launches
    h.free()


def test_batch_with_rectangular_members():
    """Rectangular grids whose first merges have the square grids' shapes
    batch with them; a grid whose axes stop alternating earlier does not."""
    probs = [hps.Problem(4, 8, 10.0, 10.0), hps.Problem(4, 8, 12.0, 12.0, 0.0, 1.0, 0.0, 0.5, my=2),
             hps.Problem(2, 8, 9.0, 9.0)]
    cs = [W.random_data(pr.m, 8, pr.kappa, pr.kappa, seed=20 + k, my=pr.ny)[0] for k, pr in enumerate(probs)]
    for h in _check_against_alone(probs, cs, 1e-12):
        h.free()
    bad = [hps.Problem(4, 8, 10.0, 10.0), hps.Problem(2, 8, 10.0, 10.0, my=8)]
    cb = [W.random_data(pr.m, 8, 10.0, 10.0, seed=1, my=pr.ny)[0] for pr in bad]
    with pytest.raises(hps.HPSError) as e:
        hps.hps_build_batch(bad, cb)
    assert e.value.code == hps.HPS_EINVAL


@pytest.mark.parametrize("precision,form", [(hps.HPS_FP64, hps.HPS_LEAF_LU), (hps.HPS_MIXED, hps.HPS_LEAF_LU),
                                            (hps.HPS_FP64, hps.HPS_LEAF_INVERSE)])
def test_rebuild_replays_the_build_as_a_graph(precision, form):
    """hps_rebuild with new coefficients gives the operators of a fresh build
    with those coefficients (first call captures the graph, later ones
    replay it), for a single build and for a batch."""
    st = torch.cuda.current_stream()
    probs = [hps.Problem(4, 10, 14.0, 14.0, precision=precision, leaf_form=form),
             hps.Problem(8, 10, 20.0, 20.0, precision=precision, leaf_form=form),
             hps.Problem(2, 10, 9.0, 9.0, precision=precision, leaf_form=form)]
    c0 = [W.random_data(pr.m, 10, pr.kappa, pr.kappa, seed=60 + k)[0] for k, pr in enumerate(probs)]
    hb = hps.hps_build_batch(probs, c0, st)
    for rnd in range(3):
        cn = [W.random_data(pr.m, 10, pr.kappa, pr.kappa, seed=70 + 10 * rnd + k)[0] for k, pr in enumerate(probs)]
        # the handles in another order than they were built in
        perm = [2, 0, 1]
        hps.hps_rebuild([hb[i] for i in perm], [torch.from_numpy(cn[i]).cuda() for i in perm], st)
        assert hps.hps_status(hb[0], st)[0] == hps.HPS_OK
        for k, pr in enumerate(probs):
            ha = hps.hps_build(pr, cn[k], st)  # pr carries the same leaf form
            _, s, t = W.random_data(pr.m, 10, pr.kappa, pr.kappa, seed=5 + k, nrhs=2)
            tol = 1e-12 if precision == hps.HPS_FP64 else 1e-9
            assert _rel(_solve(hb[k], s, t), _solve(ha, s, t)) < tol, (rnd, k)
            ha.free()
    L = hps.lib()
    arr = (__import__("ctypes").c_void_p * 1)(hb[0].ptr)
    carr = (__import__("ctypes").c_void_p * 1)(torch.from_numpy(c0[0]).cuda().data_ptr())
    assert L.hps_rebuild(1, arr, carr, None) == hps.HPS_EINVAL  # not all handles of the batch
    hb[1].free()
    assert L.hps_rebuild(1, arr, carr, None) == hps.HPS_EINVAL
    for h in (hb[0], hb[2]):
        h.free()


def test_tuned_choices_keep_results_and_launch_counts():
    """hps_tune measures the kernel choices of a ragged batch; builds after it
    use them, with the same results (1e-12) and a planned launch count that
    still equals the launches made."""
    probs = [hps.Problem(16, 12, 30.0, 30.0), hps.Problem(8, 12, 20.0, 20.0), hps.Problem(4, 12, 9.0, 9.0)]
    cs = [W.random_data(pr.m, 12, pr.kappa, pr.kappa, seed=90 + k)[0] for k, pr in enumerate(probs)]
    st = torch.cuda.current_stream()
    before = []
    for pr, c in zip(probs, cs):
        h = hps.hps_build(pr, c, st)
        _, s, t = W.random_data(pr.m, 12, pr.kappa, pr.kappa, seed=3, nrhs=2)
        before.append(_solve(h, s, t))
        h.free()
    n = hps.hps_tune(probs, st)
    assert n > 0
    assert hps.hps_tune(probs, st) == 0  # measured shapes are kept
    for k, (pr, c) in enumerate(zip(probs, cs)):
        h = hps.hps_build(pr, c, st)
        _, s, t = W.random_data(pr.m, 12, pr.kappa, pr.kappa, seed=3, nrhs=2)
        assert _rel(_solve(h, s, t), before[k]) < 1e-12
        assert h.info().build_launches == hps.hps_plan(pr).build_launches
        h.free()
    hb = _check_against_alone(probs, cs, 1e-12)
    for h in hb:
        h.free()
