"""The one-launch solve (opt-in with HPS_SOLVE_ENGINE=1; one or two
right-hand sides: the whole of Algorithm 2 as one persistent cooperative
launch over a recorded program) against the same solve launched step by step
(the default) and against the oracle: both
leaf forms, complex128 and mixed precision (whose refinement records a second
program with the interface jumps), Gauss-Legendre interfaces, a rectangular
tree, host and device arrays, and new arrays in a later call (the program is
recorded relative to s, t, u and the workspace)."""
import numpy as np
import pytest

import oracle as O
from paper_1812_07167_gb300 import hps
from paper_1812_07167_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def _solve(h, pr, s, t, engine, monkeypatch):
    monkeypatch.setenv("HPS_SOLVE_ENGINE", "1" if engine else "0")  # (opt-in: "1")
    st = torch.cuda.current_stream()
    R = s.shape[0]
    u = torch.empty((R, pr.leaves, pr.n), dtype=torch.complex128, device="cuda")
    hps.hps_solve(h, torch.from_numpy(s).cuda(), torch.from_numpy(t).cuda(), u, R, st)
    torch.cuda.synchronize()
    assert hps.hps_status(h, st)[0] == hps.HPS_OK
    return u.cpu().numpy()


@pytest.mark.parametrize("m,my,p,form,prec,q,R", [
    (16, 16, 16, hps.HPS_LEAF_INVERSE, hps.HPS_FP64, 0, 1),
    (16, 16, 16, hps.HPS_LEAF_LU, hps.HPS_FP64, 0, 2),
    (8, 8, 12, hps.HPS_LEAF_INVERSE, hps.HPS_MIXED, 0, 1),
    (8, 8, 12, hps.HPS_LEAF_LU, hps.HPS_MIXED, 0, 2),
    (8, 4, 10, hps.HPS_LEAF_INVERSE, hps.HPS_FP64, 0, 2),
    (4, 4, 16, hps.HPS_LEAF_INVERSE, hps.HPS_FP64, 12, 1),
    (4, 4, 16, hps.HPS_LEAF_LU, hps.HPS_FP64, 16, 2),
    (1, 1, 8, hps.HPS_LEAF_INVERSE, hps.HPS_FP64, 0, 1),
])
def test_one_launch_solve_matches_step_by_step_and_oracle(m, my, p, form, prec, q, R, monkeypatch):
    kappa = 2.5 * p
    pr = hps.Problem(m, p, kappa, kappa, my=my, q=q, leaf_form=form, precision=prec)
    rng = np.random.default_rng(m * 7 + p + R)
    c = 0.5 + rng.random((pr.leaves, pr.ni))
    s = rng.standard_normal((R, pr.leaves, pr.ni)) + 1j * rng.standard_normal((R, pr.leaves, pr.ni))
    t = rng.standard_normal((R, pr.nbdry)) + 1j * rng.standard_normal((R, pr.nbdry))
    st = torch.cuda.current_stream()
    h = hps.hps_build(pr, torch.from_numpy(c).cuda(), st)
    ue = _solve(h, pr, s, t, True, monkeypatch)
    ul = _solve(h, pr, s, t, False, monkeypatch)
    # the same solve in another order of summation
    assert _rel(ue, ul) < (1e-12 if prec == hps.HPS_FP64 else 1e-9)
    # a second call with new arrays reuses the recorded program
    s2, t2 = 2.0 * s[::-1].copy(), -t[::-1].copy()
    ue2 = _solve(h, pr, s2, t2, True, monkeypatch)
    ul2 = _solve(h, pr, s2, t2, False, monkeypatch)
    assert _rel(ue2, ul2) < (1e-12 if prec == hps.HPS_FP64 else 1e-9)
    # host arrays (staged) take the same program
    monkeypatch.setenv("HPS_SOLVE_ENGINE", "1")
    uh = np.zeros((R, pr.leaves, pr.n), complex)
    hps.hps_solve(h, s, t, uh, R, st)
    assert _rel(uh, ue) < 1e-14
    h.free()
    opr = O.Problem(m, p, kappa, kappa, my=my, q=q)
    with O.Tree(opr, c, nthreads=O.max_threads()) as T:
        uo = T.solve(s, t, nthreads=O.max_threads())
    assert _rel(ue, uo) < (1e-10 if prec == hps.HPS_FP64 else 1e-8)


def test_one_launch_solve_timing(monkeypatch):
    """16 x 16 leaves, p = 16, 1 right-hand side: device time of the
    one-launch solve and of the step-by-step one (the default), printed."""
    wl = W.point_sources(m=16)
    pr = hps.Problem(wl.m, wl.p, wl.kappa, wl.eta, leaf_form=hps.HPS_LEAF_INVERSE)
    lxy, bxy = hps.hps_nodes(pr)
    c, s, t = wl.sample(lxy, bxy)
    st = torch.cuda.current_stream()
    h = hps.hps_build(pr, torch.from_numpy(c).cuda(), st)
    sd = torch.from_numpy(np.ascontiguousarray(s[None])).cuda()
    td = torch.from_numpy(np.ascontiguousarray(t[None])).cuda()
    u = torch.empty((1, pr.leaves, pr.n), dtype=torch.complex128, device="cuda")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ms, us = {}, {}
    for eng in ("1", "0"):
        monkeypatch.setenv("HPS_SOLVE_ENGINE", eng)
        for _ in range(3):
            hps.hps_solve(h, sd, td, u, 1, st)
        times = []
        for _ in range(20):
            e0.record(st)
            hps.hps_solve(h, sd, td, u, 1, st)
            e1.record(st)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        ms[eng] = float(np.median(times))
        us[eng] = u.cpu().numpy()
    print(f"1-RHS solve, device ms: one launch {ms['1']:.3f}, step by step {ms['0']:.3f}")
    h.free()
    assert _rel(us["1"], us["0"]) < 1e-12
