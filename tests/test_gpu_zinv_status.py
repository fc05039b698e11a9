"""The interface-inverse kernels on their own (hps_zinv: Sec. 2.2's W^-1 as
a batched inverse) against numpy, in every regime the build takes (one CTA
or cluster a matrix; one launch a panel for small batches; the refined
complex64 inverse), and the device-side failure reporting: a matrix with an
exactly zero pivot column comes back as HPS_ESINGULAR with its index while
the rest of the batch is inverted, and the products' bounded pipeline wait
gives up on a barrier nothing completes, records a timeout and leaves the
context usable (no fault, no hang: the failure is planted in the data or in
a barrier, never in the device)."""
import time

import numpy as np
import pytest

from paper_1812_07167_gb300 import hps

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _matrices(n, batch, seed):
    """Well-conditioned complex matrices (cond ~ 3): I + G / (2 sqrt n)."""
    rng = np.random.default_rng(seed)
    G = rng.standard_normal((batch, n, n)) + 1j * rng.standard_normal((batch, n, n))
    return np.eye(n)[None] + G / (2.0 * np.sqrt(2.0 * n))


def _zinv(A, mode):
    Ad = torch.from_numpy(np.ascontiguousarray(A)).cuda()
    Xd = torch.empty_like(Ad)
    code, bad = hps.hps_zinv(Ad, Xd, mode, torch.cuda.current_stream())
    return code, bad, Xd.cpu().numpy()


# (n, batch, mode): clusters over many matrices (n = 2 is the smallest
# interface, p = 4); the per-panel launches for small batches in complex128
# (mode 0) and the refined complex64 inverse (mode 1) with its residual on
# the FP64 pipes (n = 100) or the tensor cores (n >= 448), up to the root
# interface of a 128 x 128-leaf tree
@pytest.mark.parametrize("n,batch,mode", [(2, 3, 0), (14, 40, 0), (56, 300, 0), (100, 2, 0), (100, 2, 1),
                                          (224, 64, 1), (448, 1, 1), (896, 1, 0), (1792, 1, 1)])
def test_batched_inverse_matches_numpy(n, batch, mode):
    A = _matrices(n, batch, seed=n + batch)
    code, bad, X = _zinv(A, mode)
    assert code == hps.HPS_OK and bad == -1
    ref = np.linalg.inv(A)
    err = np.linalg.norm(X - ref, axis=(1, 2)) / np.linalg.norm(ref, axis=(1, 2))
    assert err.max() < 5e-12  # complex128 accuracy in both modes (complex64 alone: ~1e-7)
    I = np.eye(n)[None]
    assert np.abs(A @ X - I).max() < 1e-11


@pytest.mark.parametrize("n,batch,mode", [(56, 4, 0), (100, 3, 0), (100, 3, 1)])
def test_zero_pivot_column_is_reported_with_its_matrix(n, batch, mode):
    A = _matrices(n, batch, seed=7)
    # a zero row of the row-major array is a zero column of the column-major
    # matrix: its elimination step finds no nonzero pivot candidate
    A[batch - 2, 5, :] = 0.0
    code, bad, X = _zinv(A, mode)
    assert code == hps.HPS_ESINGULAR
    assert bad == batch - 2
    for b in range(batch):
        if b != batch - 2:
            ref = np.linalg.inv(A[b])
            assert np.linalg.norm(X[b] - ref) / np.linalg.norm(ref) < 5e-12


def test_bounded_wait_gives_up_and_the_context_stays_usable():
    st = torch.cuda.current_stream()
    t0 = time.perf_counter()
    code = hps.hps_check_wait(200, st)
    dt = time.perf_counter() - t0
    assert code == hps.HPS_ETIMEOUT
    assert 0.15 < dt < 10.0
    # the device still runs the library's kernels, the tensor-core product too
    rng = np.random.default_rng(3)
    A = rng.standard_normal((1, 300, 200)) + 1j * rng.standard_normal((1, 300, 200))
    B = rng.standard_normal((1, 150, 300)) + 1j * rng.standard_normal((1, 150, 300))
    Ad, Bd = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    Cd = torch.empty((1, 150, 200), dtype=torch.complex128, device="cuda")
    hps.hps_zgemm(Ad, Bd, Cd, 1, st)
    ref = np.einsum("bki,bjk->bji", A, B)
    assert np.abs(Cd.cpu().numpy() - ref).max() / np.abs(ref).max() < 1e-13
