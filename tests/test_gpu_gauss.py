"""Boundary data on q Gauss-Legendre nodes per leaf edge (q != p - 2), through
the C ABI, against the oracle's build + solve of the same discretisation:
u at every node and the root ItI operator (on the Gauss nodes), both leaf
forms, square and rectangular trees, q below and above p - 2.  For q >= p - 2
the solution also equals the Chebyshev-edge solver's when the boundary data
agree.  Bar: 1e-10 relative (max-abs for u, Frobenius for R)."""
import numpy as np
import pytest

import oracle as O
from paper_1812_07167_gb300 import hps

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-10


def _rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def _data(pr, seed, nrhs=1):
    rng = np.random.default_rng(seed)
    c = 0.5 + rng.random((pr.leaves, pr.ni))
    s = rng.standard_normal((nrhs, pr.leaves, pr.ni)) + 1j * rng.standard_normal((nrhs, pr.leaves, pr.ni))
    t = rng.standard_normal((nrhs, pr.nbdry)) + 1j * rng.standard_normal((nrhs, pr.nbdry))
    return c, s, t


def _gpu(pr, c, s, t):
    st = torch.cuda.current_stream()
    h = hps.hps_build(pr, torch.from_numpy(c).cuda(), st)
    code, lev, box = hps.hps_status(h, st)
    assert code == hps.HPS_OK, (code, lev, box)
    nrhs = s.shape[0]
    u = torch.empty((nrhs, pr.leaves, pr.n), dtype=torch.complex128, device="cuda")
    hps.hps_solve(h, torch.from_numpy(s).cuda(), torch.from_numpy(t).cuda(), u, nrhs, st)
    R = np.zeros((pr.nbdry, pr.nbdry), complex)
    hps.hps_root_R(h, R, gauss_basis=True)
    torch.cuda.synchronize()
    return h, u.cpu().numpy(), R


@pytest.mark.parametrize("m,my,p,q,form,eta", [
    (1, 1, 8, 4, hps.HPS_LEAF_LU, 6.0),
    (2, 2, 8, 4, hps.HPS_LEAF_LU, 6.0),
    (2, 2, 8, 9, hps.HPS_LEAF_INVERSE, 6.0 - 2.0j),
    (4, 2, 10, 5, hps.HPS_LEAF_LU, 8.0),
    (4, 4, 16, 12, hps.HPS_LEAF_LU, 20.0),
    (4, 4, 16, 16, hps.HPS_LEAF_INVERSE, 20.0),
    (8, 8, 12, 6, hps.HPS_LEAF_LU, 15.0 + 5.0j),
    (16, 16, 16, 12, hps.HPS_LEAF_LU, 80.0),
    (16, 16, 16, 16, hps.HPS_LEAF_LU, 80.0),
])
def test_gauss_interfaces_match_oracle(m, my, p, q, form, eta):
    kappa = abs(eta)
    pr = hps.Problem(m, p, kappa, eta, my=my, q=q, leaf_form=form)
    opr = O.Problem(m, p, kappa, eta, my=my, q=q)
    assert pr.nbdry == opr.nbdry
    lxy, bxy = hps.hps_nodes(pr)
    olxy, obxy = O.nodes(opr)
    assert np.abs(bxy - obxy).max() < 1e-14 and np.abs(lxy - olxy).max() < 1e-14
    c, s, t = _data(pr, seed=m * 100 + q, nrhs=2)
    h, u, R = _gpu(pr, c, s, t)
    with O.Tree(opr, c, nthreads=O.max_threads()) as T:
        uo = T.solve(s, t, nthreads=O.max_threads())
        Ro = T.root_R()
    eu = _rel(u, uo)
    eR = float(np.linalg.norm(R - Ro) / np.linalg.norm(Ro))
    print(f"{m}x{my} p={p} q={q} form={form}: u {eu:.2e}, root R {eR:.2e}")
    assert eu <= TOL and eR <= TOL
    # only the Gauss basis exists for the root operator here
    Rc = np.zeros_like(R)
    assert hps.lib().hps_root_R(h.ptr, Rc.ctypes.data, 0, None) == hps.HPS_EINVAL
    h.free()


def test_gauss_q_at_least_p_minus_2_equals_chebyshev_solver():
    m, p, q = 8, 12, 14
    pg, pn = hps.Problem(m, p, 30.0, 30.0, q=q), hps.Problem(m, p, 30.0, 30.0)
    c, s, tn = _data(pn, seed=3)
    # the same boundary data: the Chebyshev-node interpolant at the Gauss nodes
    Pm, _ = O.edge_interp(p, q)
    tg = np.ascontiguousarray((Pm @ tn.reshape(-1, p - 2).T).T.reshape(1, -1))
    hg, ug, _ = _gpu(pg, c, s, tg)
    hn, un, _ = _gpu(pn, c, s, tn)
    hg.free()
    hn.free()
    assert _rel(ug, un) <= TOL


def test_gauss_solve_without_allocation_and_wide_solve():
    pr = hps.Problem(4, 16, 20.0, 20.0, q=10)
    c, s, t = _data(pr, seed=9, nrhs=40)
    st = torch.cuda.current_stream()
    h = hps.hps_build(pr, torch.from_numpy(c).cuda(), st)
    sd, td = torch.from_numpy(s).cuda(), torch.from_numpy(t).cuda()
    u40 = torch.empty((40, pr.leaves, pr.n), dtype=torch.complex128, device="cuda")
    hps.hps_solve(h, sd, td, u40, 40, st)  # 40 right-hand sides: the wide leaf step
    u1 = torch.empty((1, pr.leaves, pr.n), dtype=torch.complex128, device="cuda")
    hps.hps_solve_noalloc(h, sd[:1].contiguous(), td[:1].contiguous(), u1, 1, st)
    torch.cuda.synchronize()
    with O.Tree(O.Problem(4, 16, 20.0, 20.0, q=10), c) as T:
        uo = T.solve(s, t)
    assert _rel(u40.cpu().numpy(), uo) <= TOL
    assert _rel(u1.cpu().numpy()[0], uo[0]) <= TOL
    h.free()
