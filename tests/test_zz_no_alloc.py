"""The no-allocation solve gives the same solution as the ordinary solve.

hps_solve_noalloc exists for callers that cannot allocate device memory at
solve time: programs whose device memory is handed out up front to a pool or
a framework allocator, and request loops that cannot afford a cudaMalloc
(which may synchronize the device, or fail) in the middle of serving.  It
keeps its scratch vectors in a fixed device array inside the library instead
of allocating them.  This file runs last so that, if it fails, every other
test has already run.
"""
import numpy as np
import pytest

from paper_1812_07167_gb300 import hps
from paper_1812_07167_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-10  # the bar every GPU parity test uses


def _rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


# nrhs = 1 runs the chained launches of a one-column solve; 3 the split
# skinny products, whose arrival counters sit at the head of the array; 20
# the tiled products with no partial-sum region (it fits the array only on
# a 4 x 4-leaf tree)
@pytest.mark.parametrize("m,nrhs", [(16, 1), (16, 3), (4, 20)])
def test_noalloc_solve_matches_solve_on_two_calls(m, nrhs):
    assert torch.cuda.is_available(), "needs a CUDA device"
    wl = W.point_sources(m=m)  # p = 16, kappa = eta = 80
    pr = hps.Problem(wl.m, wl.p, wl.kappa, wl.eta)
    lxy, bxy = hps.hps_nodes(pr)
    c, _, _ = wl.sample(lxy, bxy)
    st = torch.cuda.current_stream()
    h = hps.hps_build(pr, torch.from_numpy(c).cuda(), st)
    for call in range(2):
        # different right-hand sides on each call, so a stale workspace shows
        _, s, t = W.random_data(wl.m, wl.p, wl.kappa, wl.eta, seed=500 + call, nrhs=nrhs)
        sd = torch.from_numpy(s).cuda()
        td = torch.from_numpy(t).cuda()
        u_ref = torch.empty((nrhs, pr.leaves, pr.n), dtype=torch.complex128, device="cuda")
        u_na = torch.full_like(u_ref, float("nan"))
        hps.hps_solve(h, sd, td, u_ref, nrhs, st)
        hps.hps_solve_noalloc(h, sd, td, u_na, nrhs, st)
        torch.cuda.synchronize()
        a, b = u_na.cpu().numpy(), u_ref.cpu().numpy()
        assert np.isfinite(a).all()
        assert _rel(a, b) <= TOL, (call, _rel(a, b))
    h.free()


def test_noalloc_solve_rejects_what_it_cannot_serve():
    wl = W.point_sources()
    pr = hps.Problem(wl.m, wl.p, wl.kappa, wl.eta)
    c, s, t = W.random_data(wl.m, wl.p, wl.kappa, wl.eta, seed=9)
    st = torch.cuda.current_stream()
    h = hps.hps_build(pr, torch.from_numpy(c).cuda(), st)
    L = hps.lib()
    u = torch.empty((1, pr.leaves, pr.n), dtype=torch.complex128, device="cuda")
    sd, td = torch.from_numpy(s).cuda(), torch.from_numpy(t).cuda()
    # more right-hand sides than the fixed workspace holds: a clear error, no work
    big = 64
    assert L.hps_solve_noalloc(h.ptr, sd.data_ptr(), td.data_ptr(), u.data_ptr(), big, None) == hps.HPS_ETOOBIG
    # host arrays would need staging buffers
    u_host = np.zeros((1, pr.leaves, pr.n), complex)
    assert L.hps_solve_noalloc(h.ptr, s.ctypes.data, t.ctypes.data, u_host.ctypes.data, 1, None) == hps.HPS_EINVAL
    assert L.hps_solve_noalloc(h.ptr, sd.data_ptr(), td.data_ptr(), u.data_ptr(), 0, None) == hps.HPS_OK
    h.free()
    # a mixed-precision solver refines every solve, which needs more workspace
    # than the fixed array holds: refused, not run
    pm = hps.Problem(4, 16, wl.kappa, wl.eta, precision=hps.HPS_MIXED)
    cm, sm, tm = W.random_data(4, 16, wl.kappa, wl.eta, seed=10)
    hm = hps.hps_build(pm, torch.from_numpy(cm).cuda(), st)
    smd, tmd = torch.from_numpy(sm).cuda(), torch.from_numpy(tm).cuda()
    um = torch.empty((1, pm.leaves, pm.n), dtype=torch.complex128, device="cuda")
    assert L.hps_solve_noalloc(hm.ptr, smd.data_ptr(), tmd.data_ptr(), um.data_ptr(), 1, None) == hps.HPS_ENOTSUP
    hm.free()
