"""The complex128 product emulated on the bf16 tensor cores (Ozaki scheme)
against the FP64-pipe product and against numpy, on shapes that span tiles
with ragged edges, and on rows and columns of very different magnitudes (the
scheme scales each row of A and column of B separately); the 5-slice form
(complex64 accuracy) against its error bound."""
import numpy as np
import pytest

from paper_1812_07167_gb300 import hps

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _rand(shape, rng):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def _run(A, B, emulated):
    Ad = torch.from_numpy(np.ascontiguousarray(A)).cuda()
    Bd = torch.from_numpy(np.ascontiguousarray(B)).cuda()
    batch, K, M = A.shape
    N = B.shape[1]
    Cd = torch.empty((batch, N, M), dtype=torch.complex128, device="cuda")
    hps.hps_zgemm(Ad, Bd, Cd, emulated, torch.cuda.current_stream())
    torch.cuda.synchronize()
    return Cd.cpu().numpy()


# one 128 x 128 tile (its slice pairs split over 9 CTAs and summed by the
# reduce pass), 64-wide tiles (N <= 64), ragged edges in M, N and K, a
# batch, two K chunks of 896, and many tiles with one CTA each
@pytest.mark.parametrize("M,N,K,batch", [(128, 128, 64, 1), (64, 64, 64, 1), (100, 37, 83, 3),
                                         (224, 448, 224, 2), (33, 130, 300, 1), (896, 512, 600, 1),
                                         (300, 200, 1000, 1), (252, 48, 252, 7), (1100, 1300, 200, 1)])
def test_emulated_product_matches_fp64(M, N, K, batch):
    rng = np.random.default_rng(M * 7 + N)
    # stored transposed: A[b] is K x M row-major = M x K column-major
    A = _rand((batch, K, M), rng)
    B = _rand((batch, N, K), rng)
    Ce = _run(A, B, 1)
    Cf = _run(A, B, 0)
    ref = np.einsum("bki,bjk->bji", A, B)  # C[b][j][i] = sum_k A(i,k) B(k,j)
    scale = np.abs(A).max() * np.abs(B).max() * K
    assert np.abs(Ce - ref).max() / scale < 1e-15
    assert np.abs(Cf - ref).max() / scale < 1e-15
    assert np.abs(Ce - Cf).max() / np.abs(ref).max() < 1e-13


def test_rows_and_columns_of_wide_dynamic_range():
    rng = np.random.default_rng(5)
    M, N, K = 96, 80, 128
    A = _rand((1, K, M), rng) * (10.0 ** rng.integers(-12, 12, size=M))[None, None, :]
    B = _rand((1, N, K), rng) * (10.0 ** rng.integers(-12, 12, size=N))[None, :, None]
    Ce = _run(A, B, 1)
    ref = np.einsum("bki,bjk->bji", A, B)
    # error of each entry relative to its own row and column scale
    ra = np.abs(A[0]).max(axis=0)  # per row i of A
    cb = np.abs(B[0]).max(axis=1)  # per column j of B
    bound = K * np.outer(cb, ra)[None] * 2.0 ** -52
    assert np.all(np.abs(Ce - ref) <= bound)


# the 5-slice product (the build's complex64 products: the mixed path's lower
# levels): every entry within K 2^-26 max|A_i.| max|B_.j| of the exact
# product, the complex64 level, also for rows and columns of very different
# magnitudes; and truly a 5-slice product (far from the 9-slice accuracy)
@pytest.mark.parametrize("M,N,K,batch,wide", [(128, 128, 64, 1, False), (100, 37, 83, 3, False),
                                              (252, 252, 252, 4, False), (896, 512, 600, 1, False),
                                              (300, 200, 1000, 1, False), (96, 80, 128, 1, True)])
def test_five_slice_product_has_complex64_accuracy(M, N, K, batch, wide):
    rng = np.random.default_rng(M + 3 * K)
    A = _rand((batch, K, M), rng)
    B = _rand((batch, N, K), rng)
    if wide:
        A = A * (10.0 ** rng.integers(-12, 12, size=M))[None, None, :]
        B = B * (10.0 ** rng.integers(-12, 12, size=N))[None, :, None]
    C4 = _run(A, B, 2)
    ref = np.einsum("bki,bjk->bji", A, B)
    ra = np.abs(A).max(axis=1)  # [batch][M]: max over k of row i of A
    cb = np.abs(B).max(axis=2)  # [batch][N]: max over k of column j of B
    scale = cb[:, :, None] * ra[:, None, :]
    err = np.abs(C4 - ref) / scale
    assert err.max() <= K * 2.0 ** -26
    assert err.max() > 2.0 ** -45


def test_zero_operand_gives_zero():
    A = np.zeros((1, 70, 40), complex)
    B = _rand((1, 50, 70), np.random.default_rng(1))
    assert np.all(_run(A, B, 1) == 0)
    assert np.all(_run(A, B, 2) == 0)


@pytest.mark.parametrize("m,p,kappa", [(16, 16, 80.0), (32, 12, 60.0)])
def test_build_with_tensor_core_products_matches_fp64_pipes(m, p, kappa):
    from paper_1812_07167_gb300 import workloads as W

    c, s, t = W.random_data(m, p, kappa, kappa, seed=m + p, nrhs=2)
    st = torch.cuda.current_stream()
    out = []
    for native in (0, 1):
        pr = hps.Problem(m, p, kappa, kappa, fp64_native=native)
        h = hps.hps_build(pr, torch.from_numpy(c).cuda(), st)
        assert hps.hps_status(h, st)[0] == hps.HPS_OK
        u = torch.empty((2, pr.leaves, pr.n), dtype=torch.complex128, device="cuda")
        hps.hps_solve(h, torch.from_numpy(s).cuda(), torch.from_numpy(t).cuda(), u, 2, st)
        R = np.zeros((pr.nbdry, pr.nbdry), complex)
        hps.hps_root_R(h, R, st)
        out.append((u.cpu().numpy(), R, h.info().build_launches, hps.hps_plan(pr).build_launches))
        h.free()
    (ue, Re, le, pe), (uf, Rf, lf, pf) = out
    assert np.abs(ue - uf).max() / np.abs(uf).max() < 1e-12
    assert np.linalg.norm(Re - Rf) / np.linalg.norm(Rf) < 1e-12
    assert le == pe and lf == pf
    assert le > lf  # the emulated products are three launches each


def test_wide_rhs_solve_on_tensor_cores_matches_fp64_pipes_and_oracle():
    """64 right-hand sides at 16 x 16 leaves: the leaf products of the solve
    run on the tensor cores; u matches the all-FP64-pipe solve (1e-12) and
    the oracle (1e-10)."""
    import os
    import oracle as O
    from paper_1812_07167_gb300 import workloads as W

    m, p, kappa, R = 16, 16, 50.0, 64
    c, s, t = W.random_data(m, p, kappa, kappa, seed=12, nrhs=R)
    st = torch.cuda.current_stream()
    us = []
    for native in (0, 1):
        pr = hps.Problem(m, p, kappa, kappa, fp64_native=native)
        h = hps.hps_build(pr, torch.from_numpy(c).cuda(), st)
        u = torch.empty((R, pr.leaves, pr.n), dtype=torch.complex128, device="cuda")
        hps.hps_solve(h, torch.from_numpy(s).cuda(), torch.from_numpy(t).cuda(), u, R, st)
        torch.cuda.synchronize()
        us.append(u.cpu().numpy())
        h.free()
    assert np.abs(us[0] - us[1]).max() / np.abs(us[1]).max() < 1e-12
    opr = O.Problem(m, p, kappa, kappa)
    nt = os.cpu_count() or 1
    with O.Tree(opr, c, nthreads=nt) as T:
        uo = T.solve(s[:4], t[:4], nthreads=nt)
    assert np.abs(us[0][:4] - uo).max() / np.abs(uo).max() < 1e-10


# complex64 arithmetic on the FP32 pipes (the refinement corrections' and the
# mixed path's products): the 128 x 128-tile kernel where the shape allows
# (M, N >= 96), the index-mapped tile kernels otherwise; every entry within
# K 2^-21 (|A| |B|)(i, j) of the exact product (operands rounded to complex64
# and the sums in complex64)
@pytest.mark.parametrize("M,N,K,batch", [(252, 252, 252, 4), (128, 128, 16, 1), (250, 130, 77, 2),
                                         (1000, 300, 200, 1), (100, 37, 83, 3), (96, 96, 1, 5)])
def test_complex64_product_has_complex64_accuracy(M, N, K, batch):
    rng = np.random.default_rng(M + N + K)
    A = _rand((batch, K, M), rng)
    B = _rand((batch, N, K), rng)
    C = _run(A, B, 3)
    ref = np.einsum("bki,bjk->bji", A, B)
    bound = K * 2.0 ** -21 * np.einsum("bki,bjk->bji", np.abs(A), np.abs(B))
    assert np.all(np.abs(C - ref) <= bound)
    assert np.abs(C - ref).max() / np.abs(ref).max() > 1e-12  # (truly complex64)
