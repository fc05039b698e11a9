"""Continuous batching on the GPU: hps_solve_batch and the request loop.

Every result of a served mix (solves batched with whatever arrived beside
them, builds running concurrently on other streams) is compared with the
same request done alone: within 1e-12 relative for the FP64 path (the
batched kernels differ from the lone ones only in summation order) and 1e-8
for the mixed path after refinement.
"""
import numpy as np
import pytest

from paper_1812_07167_gb300 import hps, serve
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


def _build(pr, c):
    h = hps.hps_build(pr, torch.from_numpy(np.ascontiguousarray(c)).cuda(), torch.cuda.current_stream())
    assert hps.hps_status(h, torch.cuda.current_stream())[0] == hps.HPS_OK
    return h


def _alone(h, s, t):
    pr = h.pr
    u = torch.empty((s.shape[0], pr.leaves, pr.n), dtype=torch.complex128, device="cuda")
    hps.hps_solve(h, s, t, u, s.shape[0], torch.cuda.current_stream())
    torch.cuda.synchronize()
    return u.cpu().numpy()


def test_solve_batch_matches_separate_solves():
    m, p, kappa = 4, 16, 25.0
    pr = hps.Problem(m, p, kappa, kappa)
    c, _, _ = W.random_data(m, p, kappa, kappa, seed=3)
    h = _build(pr, c)
    _, s1, t1 = W.random_data(m, p, kappa, kappa, seed=41, nrhs=3)
    _, s2, t2 = W.random_data(m, p, kappa, kappa, seed=42, nrhs=2)
    _, s3, t3 = W.random_data(m, p, kappa, kappa, seed=43, nrhs=7)
    d1 = (torch.from_numpy(s1).cuda(), torch.from_numpy(t1).cuda())
    u1 = torch.empty((3, pr.leaves, pr.n), dtype=torch.complex128, device="cuda")
    u2 = np.zeros((2, pr.leaves, pr.n), complex)          # host request
    u3 = torch.empty((7, pr.leaves, pr.n), dtype=torch.complex128, device="cuda")
    hps.hps_solve_batch(h, [d1[0], None, s2, torch.from_numpy(s3).cuda()],
                        [d1[1], None, t2, torch.from_numpy(t3).cuda()],
                        [u1, None, u2, u3], [3, 0, 2, 7], torch.cuda.current_stream())
    torch.cuda.synchronize()
    assert _rel(u1.cpu().numpy(), _alone(h, *d1)) < 1e-12
    assert _rel(u2, _alone(h, torch.from_numpy(s2).cuda(), torch.from_numpy(t2).cuda())) < 1e-12
    assert _rel(u3.cpu().numpy(), _alone(h, torch.from_numpy(s3).cuda(), torch.from_numpy(t3).cuda())) < 1e-12
    L = hps.lib()
    arr = __import__("ctypes").c_void_p * 1
    nr = (__import__("ctypes").c_int * 1)(-1)
    assert L.hps_solve_batch(h.ptr, -1, None, None, None, None, None) == hps.HPS_EINVAL
    assert L.hps_solve_batch(h.ptr, 1, arr(None), arr(None), arr(None), nr, None) == hps.HPS_EINVAL
    nr[0] = 2
    assert L.hps_solve_batch(h.ptr, 1, arr(None), arr(None), arr(None), nr, None) == hps.HPS_EINVAL
    assert L.hps_solve_batch(h.ptr, 0, None, None, None, None, None) == hps.HPS_OK
    assert L.hps_reserve(h.ptr, -1) == hps.HPS_EINVAL
    h.free()


@pytest.mark.parametrize("precision,tol", [(hps.HPS_FP64, 1e-12), (hps.HPS_MIXED, 1e-8)])
def test_each_result_same_alone_and_in_the_mix(precision, tol):
    m, p, kappa = 8, 16, 40.0
    pr = hps.Problem(m, p, kappa, kappa, precision=precision)
    c, _, _ = W.random_data(m, p, kappa, kappa, seed=8)
    h = _build(pr, c)
    sched = W.request_stream(11, 48, 4000.0, nrhs_max=12, build_m=(2, 4))
    reqs = []
    for k, d in enumerate(sched):
        if d["kind"] == "solve":
            _, s, t = W.random_data(m, p, kappa, kappa, seed=d["seed"], nrhs=d["nrhs"])
            reqs.append(serve.Request(k, d["arrival"], "solve", key="main", nrhs=d["nrhs"],
                                      s=torch.from_numpy(s).cuda(), t=torch.from_numpy(t).cuda()))
        else:
            bp = hps.Problem(d["m"], p, d["kappa"], d["kappa"], precision=precision)
            bc, _, _ = W.random_data(d["m"], p, d["kappa"], d["kappa"], seed=d["seed"])
            reqs.append(serve.Request(k, d["arrival"], "build", problem=bp,
                                      c=torch.from_numpy(bc).cuda()))
    torch.cuda.synchronize()
    srv = serve.Server(max_batch_rhs=40, reserve_bytes=1 << 30)
    srv.add_solver("main", h)
    srv.run(reqs)
    torch.cuda.synchronize()
    st = serve.summarize(reqs)
    assert st["failed"] == 0
    assert st["builds"] >= 1
    assert st["batches"] < st["solves"], st  # requests were batched together
    for r in reqs:
        if r.kind == "solve":
            assert _rel(r.u.cpu().numpy(), _alone(h, r.s, r.t)) < tol, r.rid
        else:
            hb = _build(r.problem, r.c.cpu().numpy())
            _, s, t = W.random_data(r.problem.m, p, r.problem.kappa, r.problem.eta, seed=5, nrhs=2)
            sd, td = torch.from_numpy(s).cuda(), torch.from_numpy(t).cuda()
            assert _rel(_alone(r.handle, sd, td), _alone(hb, sd, td)) < tol, r.rid
            hb.free()
    srv.release_built()
    h.free()
