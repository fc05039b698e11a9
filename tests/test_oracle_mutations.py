"""The oracle's pins catch plausible mistakes.

Each case plants one mistake (a wrong sign, a dropped term, a transposed
operand, a wrong index) in a copy of the oracle's C source, compiles it on
the CPU, and checks that the polynomial-exactness pin, the dense
global-solve pin, the two-leaf interface-conditioning pin or one of the
Gauss-Legendre interface pins then fails.  The unmodified oracle passes both (see
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
    # the Gauss-Legendre interface mode
    "legendre_recurrence": ("((2.0 * k - 1.0) * z * b - (k - 1.0) * a) / k", "((2.0 * k - 1.0) * z * b - k * a) / k"),
    "gauss_P_reversed": ("Ph[(size_t)(side * q + a) * nbc + side * e + j] = T->Pm[a * e + j];",
                         "Ph[(size_t)(side * q + a) * nbc + side * e + j] = T->Pm[a * e + (e - 1 - j)];"),
    "gauss_Q_reversed": ("Qh[(size_t)(side * e + j) * nb + side * q + a] = T->Qm[j * q + a];",
                         "Qh[(size_t)(side * e + j) * nb + side * q + a] = T->Qm[(e - 1 - j) * q + a];"),
    "gauss_lagrange_node": ("if (k != j) v *= (x - xs[k]) / (xs[j] - xs[k]);",
                            "if (k != j) v *= (x - xs[k]) / (xs[k] - xs[j]);"),
    "brute_gauss_coupling_sign": ("A[row * N + tbase + k] = 1.0;", "A[row * N + tbase + k] = -1.0;"),
    "brute_gauss_Q_sign": ("A[row * N + tbase + side * q + a] = -Qm[j * q + a];",
                           "A[row * N + tbase + side * q + a] = Qm[j * q + a];"),
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
# Gauss-Legendre interfaces: a degree q-1 polynomial is reproduced, and the
# hierarchical solve equals the dense global system of that discretisation
try:
    wg = W.polynomial_solution(2, 8, 9.0, 4.0 - 1.0j, deg=3)
    prg = O.Problem(2, 8, wg.kappa, wg.eta, q=4)
    lg, bg = O.nodes(prg)
    cg, sg, tg = wg.sample(lg, bg)
    with O.Tree(prg, cg) as Tg:
        ug = Tg.solve(sg[None], tg[None])[0]
    ueg = wg.u_exact(lg[..., 0], lg[..., 1])
    g1 = float(np.abs(ug - ueg).max() / np.abs(ueg).max())
    prb = O.Problem(2, 8, 6.0, 2.0 + 1.0j, q=5)
    rb = np.random.default_rng(1)
    cb = 0.5 + rb.random((4, 36))
    sb = rb.standard_normal((4, 36)) + 0j
    tb = rb.standard_normal(prb.nbdry) + 1j * rb.standard_normal(prb.nbdry)
    with O.Tree(prb, cb) as Tb:
        uh = Tb.solve(sb[None], tb[None])[0]
    ubb = O.brute(prb, cb, sb, tb)
    g2 = float(np.abs(uh - ubb).max() / np.abs(ubb).max())
    g3 = float(np.abs(O.gauss_nodes(7) - np.polynomial.legendre.leggauss(7)[0]).max())
    gauss = float(np.nan_to_num(max(g1, g2, g3), nan=1e300))
except Exception:
    gauss = 1e300
print(poly, brute, cond, gauss)
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
    out = subprocess.run([sys.executable, "-c", CHECK % {"root": ROOT}], env=env,
                         capture_output=True, text=True, timeout=300)
    if out.returncode != 0:
        # the planted mistake made the oracle abort (e.g. a boundary node of one
        # box that matches no node of its neighbour): caught, by every pin
        return (1e300,) * 4
    return tuple(map(float, out.stdout.split()[-4:]))


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name, tmp_path):
    old, new = MUTATIONS[name]
    poly, brute, cond, gauss = _run_variant(tmp_path, old, new)
    assert poly > 1e-6 or brute > 1e-6 or cond > 1e-6 or gauss > 1e-6, (name, poly, brute, cond, gauss)


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_unmutated_copy_passes(tmp_path):
    poly, brute, cond, gauss = _run_variant(tmp_path, "int ora_max_threads(void) {", "int ora_max_threads(void) {")
    assert poly < 1e-10 and brute < 1e-10 and cond < 1e-8 and gauss < 1e-10
