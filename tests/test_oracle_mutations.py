"""The oracle's pins catch plausible mistakes.

Each case plants one mistake (a wrong sign, a dropped term, a transposed
operand, a wrong index) in a copy of the oracle's C source, compiles it on
the CPU, and checks that the polynomial-exactness pin, the dense
global-solve pin or the two-leaf interface-conditioning pin then fails.  The unmodified oracle passes both (see
test_oracle_pins.py)."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "hps_oracle.c")

MUTATIONS = {
    "F_eta_sign": ("F[(size_t)k * n + j] = v + I * eta * idn;", "F[(size_t)k * n + j] = v - I * eta * idn;"),
    "west_normal_sign": ("(side == 0 || side == 3) ? -1.0 : 1.0", "(side == 0) ? -1.0 : 1.0"),
    "dropped_kappa": ("v -= kappa * kappa * c[q];", "v -= kappa * c[q];"),
    "cheb_diag_sign": ("D[i * p + i] = -rowsum;", "D[i * p + i] = rowsum;"),
    "cheb_scale": ("double s = 2.0 / (b - a);", "double s = 1.0 / (b - a);"),
    "W_identity_sign": ("W[i * n3 + i] += 1.0;", "W[i * n3 + i] -= 1.0;"),
    "W_transposed": ("matmul(n3, n3, n3, R33b, R33a, W);", "matmul(n3, n3, n3, R33a, R33b, W);"),
    "Phib_term_sign": ("-R31a[i * n1 + j] - S2[i * n1 + j]", "-R31a[i * n1 + j] + S2[i * n1 + j]"),
    "R13a_index": ("R13a[i * n3 + j] = A->R[(size_t)I1[i] * na + I3a[j]];",
                   "R13a[i * n3 + j] = A->R[(size_t)I1[i] * na + I3b[j]];"),
    "htau_sign": ("hv[tau][i] = ha[b->I1[i]] + x1[i];", "hv[tau][i] = ha[b->I1[i]] - x1[i];"),
    "t3b_tilde_sign": ("-(h3a[i] + w1[i]) + w2[i]", "-(h3a[i] - w1[i]) + w2[i]"),
    "down_t3a_sign": ("tv[2 * tau][b->I3a[i]] = t3a[i] + tta[tau][i];",
                      "tv[2 * tau][b->I3a[i]] = t3a[i] - tta[tau][i];"),
    "Rtau_diag_block": ("((j >= n1) ? R22b[i * n2 + (j - n1)] : 0.0)", "0.0"),
    "norm1_row_sums": ("s += cabs(A[(size_t)i * n + j]);", "s += cabs(A[(size_t)j * n + i]);"),
    "condW_without_inverse": ("P->condW = norm1(n3, W) * norm1(n3, Winv);", "P->condW = norm1(n3, W);"),
}

CHECK = r"""
import sys, numpy as np
sys.path.insert(0, %(root)r)
import oracle as O
from paper_1812_07167_gb300 import workloads as W
worst = 0.0
wl = W.polynomial_solution(4, 8, 9.0, 4.0 - 1.0j, domain=(0.0, 2.0, 0.0, 1.0))
pr = O.Problem(4, 8, wl.kappa, wl.eta, 0.0, 2.0, 0.0, 1.0)
lxy, bxy = O.nodes(pr)
c, s, t = wl.sample(lxy, bxy)
with O.Tree(pr, c) as T:
    u = T.solve(s[None], t[None])[0]
ue = wl.u_exact(lxy[..., 0], lxy[..., 1])
poly = float(np.nan_to_num(np.abs(u - ue).max() / np.abs(ue).max(), nan=1e300))
pr2 = O.Problem(2, 8, 6.0, 2.0 + 1.0j)
c2, s2, t2 = W.random_data(2, 8, 6.0, 2.0 + 1.0j, seed=3)
try:
    ub = O.brute(pr2, c2, s2[0], t2[0])
    with O.Tree(pr2, c2) as T2:
        u2 = T2.solve(s2, t2)[0]
    brute = float(np.nan_to_num(np.abs(u2 - ub).max() / np.abs(ub).max(), nan=1e300))
except Exception:
    brute = 1e300
# cond_1(W) of the one merge of a 2 x 1 grid against W assembled from the
# leaves' ItI operators (west leaf's east edge, east leaf's west edge)
pr3 = O.Problem(2, 8, 12.0, 3.0 - 2.0j, my=1)
c3, _, _ = W.random_data(2, 8, 12.0, 3.0 - 2.0j, seed=5, my=1)
e = pr3.e
Ra, Rb = O.leaf(pr3, c3[0])[2], O.leaf(pr3, c3[1])[2]
Wm = np.eye(e) - Rb[3 * e:, 3 * e:] @ Ra[e:2 * e, e:2 * e]
with O.Tree(pr3, c3) as T3:
    cw = T3.cond_W()[0]
cond = abs(cw / np.linalg.cond(Wm, 1) - 1.0)
print(poly, brute, cond)
"""


def _run_variant(tmp_path, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, old
    mutated = tmp_path / "hps_oracle_mut.c"
    mutated.write_text(src.replace(old, new))
    lib = tmp_path / "liboracle_mut.so"
    subprocess.run(["gcc", "-O1", "-std=gnu11", "-fopenmp", "-fPIC", "-shared", "-o", str(lib),
                    str(mutated), "-lm"], check=True)
    env = dict(os.environ, HPS_ORACLE_LIB=str(lib), OMP_NUM_THREADS="1")
    out = subprocess.run([sys.executable, "-c", CHECK % {"root": ROOT}], env=env, check=True,
                         capture_output=True, text=True, timeout=300)
    return tuple(map(float, out.stdout.split()[-3:]))


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name, tmp_path):
    old, new = MUTATIONS[name]
    poly, brute, cond = _run_variant(tmp_path, old, new)
    assert poly > 1e-6 or brute > 1e-6 or cond > 1e-6, (name, poly, brute, cond)


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_unmutated_copy_passes(tmp_path):
    poly, brute, cond = _run_variant(tmp_path, "int ora_max_threads(void) {", "int ora_max_threads(void) {")
    assert poly < 1e-10 and brute < 1e-10 and cond < 1e-8
