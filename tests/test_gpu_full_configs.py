"""The largest workloads at their full sizes, against answers fixed from
outside the CUDA path.

* 64 x 64 leaves, p = 16, kappa = eta = 300, the seeded random medium with
  eight Gaussian sources: the complex128 path and the mixed path against the
  oracle's own full build and solve (Algorithm 1 and 2 on the host cores,
  about a minute and a half), u at every node and the root ItI operator.
* 128 x 128 leaves, p = 16, kappa = eta = 600, the seeded random medium of
  the serving workload, with a manufactured solution that is a polynomial of
  degree p - 1 in x and y: the discretisation reproduces it at every node to
  rounding (Sec. 2.1's collocation, impedance and interface rows hold exactly
  for it), so both paths are compared with the exact values.  This reaches
  the n3 = 1792 interface inverses of the root merge and the chunked leaf
  launch of 16,384 leaves.

Bars: 1e-10 relative for the complex128 path, 1e-8 for the mixed path after
refinement (max-abs over all nodes for u, Frobenius for R).
"""
import time

import numpy as np
import pytest

import oracle as O
from paper_1812_07167_gb300 import hps
from paper_1812_07167_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-10
TOL_MIXED = 1e-8


def _rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def _build(pr, c):
    st = torch.cuda.current_stream()
    h = hps.hps_build(pr, torch.from_numpy(np.ascontiguousarray(c)).cuda(), st)
    code, lev, box = hps.hps_status(h, st)
    assert code == hps.HPS_OK, (code, lev, box)
    return h


def _solve(h, s, t):
    pr = h.pr
    s = np.ascontiguousarray(s, dtype=np.complex128).reshape(-1, pr.leaves, pr.ni)
    nrhs = s.shape[0]
    t = np.ascontiguousarray(t, dtype=np.complex128).reshape(nrhs, pr.nbdry)
    ud = torch.empty((nrhs, pr.leaves, pr.n), dtype=torch.complex128, device="cuda")
    hps.hps_solve(h, torch.from_numpy(s).cuda(), torch.from_numpy(t).cuda(), ud, nrhs,
                  torch.cuda.current_stream())
    torch.cuda.synchronize()
    return ud.cpu().numpy()


def _root_R(h):
    R = np.zeros((h.pr.nbdry, h.pr.nbdry), complex)
    hps.hps_root_R(h, R)
    return R


def test_random_medium_64x64_kappa300_against_oracle():
    assert torch.cuda.is_available(), "needs a CUDA device"
    wl = W.random_medium_sources(64, 16, 300.0)  # random medium seed 2, sources seed 1002
    pf = hps.Problem(wl.m, wl.p, wl.kappa, wl.eta)
    pm = hps.Problem(wl.m, wl.p, wl.kappa, wl.eta, precision=hps.HPS_MIXED)
    lxy, bxy = hps.hps_nodes(pf)
    c, s, t = wl.sample(lxy, bxy)

    h64 = _build(pf, c)
    u64 = _solve(h64, s[None], t[None])[0]
    R64 = _root_R(h64)
    h64.free()
    hmx = _build(pm, c)  # library defaults: the top 4 merge levels in complex128, 2 refinement steps
    umx = _solve(hmx, s[None], t[None])[0]
    Rmx = _root_R(hmx)
    hmx.free()

    t0 = time.perf_counter()
    opr = O.Problem(wl.m, wl.p, wl.kappa, wl.eta)
    nth = O.max_threads()
    with O.Tree(opr, c, nthreads=nth) as T:
        assert T.status == 0
        uo = T.solve(s[None], t[None], nthreads=nth)[0]
        Ro = T.root_R()
    print(f"oracle 64 x 64 build + solve on {nth} threads: {time.perf_counter() - t0:.1f} s")

    e64, emx = _rel(u64, uo), _rel(umx, uo)
    r64 = float(np.linalg.norm(R64 - Ro) / np.linalg.norm(Ro))
    rmx = float(np.linalg.norm(Rmx - Ro) / np.linalg.norm(Ro))
    print(f"64 x 64, kappa 300 vs oracle: u complex128 {e64:.2e}, mixed {emx:.2e}; "
          f"root R complex128 {r64:.2e}, mixed (not refined) {rmx:.2e}")
    assert e64 <= TOL
    assert r64 <= TOL
    assert emx <= TOL_MIXED
    # the mixed root R carries the complex64 lower levels (it is not refined)
    assert rmx <= 1e-3


def test_polynomial_128x128_kappa600_every_node():
    assert torch.cuda.is_available(), "needs a CUDA device"
    m, p, kappa = 128, 16, 600.0
    wl = W.polynomial_solution(m, p, kappa, kappa, c=W.random_medium(3))
    pf = hps.Problem(m, p, kappa, kappa)
    pm = hps.Problem(m, p, kappa, kappa, precision=hps.HPS_MIXED)
    info = hps.hps_plan(pf)
    assert info.levels == 14
    lxy, bxy = hps.hps_nodes(pf)
    c, s, t = wl.sample(lxy, bxy)
    ue = wl.u_exact(lxy[..., 0], lxy[..., 1])
    for pr, tol in ((pf, TOL), (pm, TOL_MIXED)):
        h = _build(pr, c)
        u = _solve(h, s[None], t[None])[0]
        h.free()
        err = _rel(u, ue)
        print(f"128 x 128, kappa 600, polynomial solution, precision {pr.precision}: {err:.2e}")
        assert np.isfinite(u).all()
        assert err <= tol
        del u
