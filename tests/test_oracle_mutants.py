"""Mutation check of the oracle's pins.

Each case plants one plausible mistake in a copy of one oracle module (or of the shared
input generator): a dropped term, a wrong sign, a transposed operand, a wrong or shifted
index, an off-by-one in a comparison. A child process loads the mutated source in place of
the module and runs the CPU pin tests (``tests/test_oracle_*.py``) against it; every mutant
must make at least one pin fail. A control run with the source unchanged must pass, so a
failure is the mutant's doing and not the harness's.

The mistake is planted in the oracle, on the CPU; nothing here touches the CUDA library.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PIN_FILES = [
    "tests/test_oracle_tt_svd.py",
    "tests/test_oracle_householder.py",
    "tests/test_oracle_model_inputs.py",
    "tests/test_oracle_thick_bounds.py",
    "tests/test_oracle_two_sided.py",
]

# child: replace `old` by `new` (exactly one occurrence) in the module's source, register the
# result under the module's name before anything imports it, then run the pins
CHILD = r"""
import importlib, os, sys, types
root, modname, old, new = sys.argv[1:5]
sys.path.insert(0, root)
pkg, _, leaf = modname.rpartition(".")
parent = importlib.import_module(pkg)
path = os.path.join(root, *modname.split(".")) + ".py"
src = open(path).read()
if src.count(old) != 1:
    print("MUTATION SITE NOT UNIQUE:", src.count(old)); sys.exit(97)
mod = types.ModuleType(modname)
mod.__file__ = path
mod.__package__ = pkg
sys.modules[modname] = mod
exec(compile(src.replace(old, new), path, "exec"), mod.__dict__)
setattr(parent, leaf, mod)
import pytest
sys.exit(pytest.main(sys.argv[5:] + ["-x", "-q", "-p", "no:cacheprovider", "-m", "not gpu"]))
"""

# (module, source fragment, mutated fragment, what the mistake breaks)
MUTANTS = [
    # Alg. 1 and its helpers
    ("oracle.tt_svd_oracle", 'np.reshape(a, shape, order="F")', 'np.reshape(a, shape, order="C")',
     "Sec. 2.1: unfoldings are Fortran-order reshapes"),
    ("oracle.tt_svd_oracle", "tol / math.sqrt(d - 1) * frobenius_norm(X)", "tol / math.sqrt(d) * frobenius_norm(X)",
     "Alg. 1 line 1: the tolerance is split over d - 1 steps"),
    ("oracle.tt_svd_oracle", "math.sqrt(float(np.dot(x, x)))", "float(np.dot(x, x))",
     "Alg. 1 line 1: ||X||_F, not its square"),
    ("oracle.tt_svd_oracle", "if tail[j] <= d2)", "if tail[j] < d2)",
     "Alg. 1 line 8: '<=' in the tail test"),
    ("oracle.tt_svd_oracle", "        tail[j] = acc\n", "        tail[j + 1] = acc\n",
     "Alg. 1 line 8: the tail after sigma_j"),
    ("oracle.tt_svd_oracle", "    return max(r, 1)\n", "    return r\n",
     "r >= 1 (r_0 = r_d = 1, non-empty cores)"),
    ("oracle.tt_svd_oracle", "W = U[:, :rr] * S[:rr]", "W = U[:, :rr]",
     "Alg. 1 line 11: W = U_r diag(sigma_r)"),
    ("oracle.tt_svd_oracle", "freshape(Vt[:rr, :], (rr, ni, r[i]))", "freshape(Vt[:rr, :], (rr, r[i], ni))",
     "Alg. 1 line 9: core index order (r_{i-1}, n_i, r_i)"),
    ("oracle.tt_svd_oracle", "res.discarded2[i] = float(np.sum(S[rr:] ** 2))",
     "res.discarded2[i] = float(np.sum(S[rr + 1:] ** 2))", "discarded energy: all sigma after the kept r"),
    ("oracle.tt_svd_oracle", "        A = freshape(A, (N, rk1))\n", "        A = np.reshape(A, (N, rk1))\n",
     "Sec. 2.1.2: contraction of the train (Fortran order)"),
    ("oracle.tt_svd_oracle", "rows = int(np.prod(n[: i - 1]))\n        r[i - 1]",
     "rows = int(np.prod(n[: i]))\n        r[i - 1]", "rank caps: rows of the unfolding at step i"),
    ("oracle.tt_svd_oracle", "rows = int(np.prod(n[:k]))", "rows = int(np.prod(n[:k + 1]))",
     "brute-force unfolding (n_1..n_k) x (n_{k+1}..n_d)"),
    # Alg. 6 and the TSQR trees
    ("oracle.householder", "    if u[0] > 0:\n", "    if u[0] < 0:\n",
     "Alg. 6: alpha takes the sign opposite to the pivot"),
    ("oracle.householder", "    t = t - alpha * u[0]\n", "    t = t + alpha * u[0]\n",
     "Alg. 6: t <- t - alpha u_1"),
    ("oracle.householder", "    u[0] = u[0] - alpha\n", "    u[0] = u[0] + alpha\n",
     "Alg. 6: u_1 <- u_1 - alpha"),
    ("oracle.householder", "w = np.concatenate(([R[j, k]], M[:, k]))", "w = np.concatenate(([0.0], M[:, k]))",
     "Alg. 6: the reflector acts on row j of R"),
    ("oracle.householder", "            R[j, k] = w[0]\n", "            R[j, k] = R[j, k]\n",
     "Alg. 6: the updated row j of R is kept"),
    ("oracle.householder", "qless_householder_block(Rs[a], Rs[a + 1], eps)",
     "qless_householder_block(Rs[a], np.zeros_like(Rs[a + 1]), eps)", "Sec. 3.2: the tree merges both R's"),
    ("oracle.householder", "W[s:s + nb, :]", "W[s:s + nb - 1, :]",
     "Sec. 3.2: the flat tree covers every row"),
    # Alg. 2 (TSQR TT-SVD)
    ("oracle.tt_svd_tsqr", "Y = W @ Vt[:rr, :].T", "Y = W @ Vt[:, :rr]",
     "Alg. 2 line 11: W V_{:,1:r} (transposed operand)"),
    ("oracle.tt_svd_tsqr", "math.sqrt(float(np.sum(S ** 2)))", "float(np.sum(S ** 2))",
     "Alg. 2 line 7: delta from ||Sigma||_F"),
    ("oracle.tt_svd_tsqr", "W = freshape(Y, (nbar // (n[i - 2] * rr), n[i - 2] * rr))",
     "W = freshape(Y, (nbar // (n[i - 1] * rr), n[i - 1] * rr))", "Alg. 2 line 11: the next unfolding takes n_{i-1}"),
    # Sec. 4 model
    ("oracle.model", "return (n / nb) * 2.0 * m * (m + 1) * (nb + 1)", "return (n / nb) * 2.0 * m * m * (nb + 1)",
     "Sec. 4.1.1: m (m + 1) (n_b + 1) FMAs per block"),
    ("oracle.model", "return float(es) * n * (m + k)", "return float(es) * n * m",
     "Sec. 4.1.2: the TSMM writes Y"),
    ("oracle.model", "es * (2.0 * nbar / (1.0 - fbar) + fbar * nbar / (1.0 - fbar))",
     "es * (nbar / (1.0 - fbar) + fbar * nbar / (1.0 - fbar))", "Eq. TT-SVD_data_volume: two reads per step"),
    ("oracle.model", "2.0 * nbar * r_max * (1.0 / fbar + 2.0 / (1.0 - fbar))",
     "2.0 * nbar * r_max * (1.0 / fbar + 1.0 / (1.0 - fbar))", "Eq. TT-SVD_operations"),
    ("oracle.model", "if m >= max(m_min, r_est / f1_min):", "if m >= max(m_min, r_est * f1_min):",
     "Alg. 3 line 1 threshold"),
    # Alg. 3 and Alg. 4
    ("oracle.thick_bounds", "rec = tt_svd(freshape(Tbar, [r] + n[d - k:]), r_max)",
     "rec = tt_svd(freshape(Tbar, [r] + n[d - k:][::-1]), r_max)", "Alg. 3 line 4: dimension order of T_bar"),
    ("oracle.thick_bounds", "freshape(Tl, (a * b, r)) @ S0,", "freshape(Tl, (a * b, r)),",
     "Alg. 3: the recovered first factor is absorbed into the next core"),
    ("oracle.two_sided", "cores[a - 1] = freshape(U[:, :r], (rL, n[a - 1], r))",
     "cores[a - 1] = freshape(U[:, :r] * S[:r], (rL, n[a - 1], r))", "Alg. 4: left cores are orthonormal"),
    ("oracle.two_sided", "Z = freshape(S[:r, None] * Vt[:r, :], [r] + mid[1:] + [rR])",
     "Z = freshape(Vt[:r, :], [r] + mid[1:] + [rR])", "Alg. 4: Sigma V^T carries the remainder"),
    ("oracle.tt_svd_oracle", "    return float(np.max(np.abs(T @ T.T - np.eye(r0))))\n",
     "    return float(np.max(np.abs(T @ T.T)))\n", "orthonormality defect: T T^T - I"),
    ("oracle.tt_svd_oracle", "    for j in (r - 1, r):\n", "    for j in (r,):\n",
     "rank tie: the tail test at r - 1 and at r"),
    ("oracle.tt_svd_oracle", "        nbar = nbar * rr // cols  # line 10", "        nbar = nbar // cols  # line 10",
     "Alg. 1 line 10: n_bar <- n_bar r_{i-1} / (n_i r_i)"),
    ("oracle.householder", "    beta = 1.0 / math.sqrt(t)\n", "    beta = 1.0 / t\n",
     "Alg. 6: beta = 1 / sqrt(t), so ||v||^2 = 2"),
    # the shared counter-based generator (Philox4x32-10, Salmon et al. 2011) and input recipes
    ("paper_2102_00104_gb300.inputs", "for rnd in range(10):", "for rnd in range(9):",
     "Philox4x32-10: ten rounds"),
    ("paper_2102_00104_gb300.inputs", "b = (y >> np.uint32(6))", "b = (y >> np.uint32(7))",
     "53-bit fraction from two 32-bit words"),
    ("paper_2102_00104_gb300.inputs", "X += E * (noise_rel / np.sqrt(np.sum(E * E)))", "X += E * noise_rel",
     "planted tensor: noise relative to ||X||_F, not per entry"),
]


def run_child(modname, old, new):
    return subprocess.run([sys.executable, "-c", CHILD, ROOT, modname, old, new] + PIN_FILES,
                          cwd=ROOT, capture_output=True, text=True, timeout=300)


def test_harness_passes_unmutated():
    p = run_child("oracle.tt_svd_oracle", "def freshape(", "def freshape(")
    assert p.returncode == 0, p.stdout[-2000:] + p.stderr[-2000:]


@pytest.mark.parametrize("modname,old,new,why", MUTANTS, ids=[f"{m[0].split('.')[-1]}-{i}" for i, m in enumerate(MUTANTS)])
def test_mutant_is_caught(modname, old, new, why):
    p = run_child(modname, old, new)
    assert p.returncode != 97, f"mutation site not found exactly once: {old!r}"
    # exit code 1: at least one pin failed (2 or more would be a harness or collection error)
    assert p.returncode == 1, f"mutant survived ({why}): rc={p.returncode}\n" + p.stdout[-1500:] + p.stderr[-1500:]
