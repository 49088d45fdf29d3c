"""The native FP64 form's W V_r on the warp-specialised tcgen05 pipeline (TMA tile loads,
FP16 Ozaki digits, level sums in tensor memory, integer combination): each output within a
few units of 2^-53 of sum_k |W_ik| |V_kj| of the exact product (rational arithmetic on
sampled rows), on the shapes and value patterns its digit split has to get right: ragged
row tails, m not a multiple of 16, row maxima just below a power of two (where the scale
exponent is raised by one), zero rows, rows of subnormal numbers, non-finite entries, and
a W that cannot be mapped by TMA (the Ozaki mma.sync kernel runs instead)."""
from fractions import Fraction

import numpy as np
import pytest
import torch

from paper_2102_00104_gb300 import api, capi
from tests.gpu_common import colmajor, ensure_lib

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_lib()
    capi.tt_tune_set("tsmm.ws", 1)


def exact_rows(W, V, rows, k):
    out = np.empty((len(rows), k))
    for a, i in enumerate(rows):
        wi = [Fraction(float(x)) for x in W[i]]
        for j in range(k):
            out[a, j] = float(sum(x * Fraction(float(v)) for x, v in zip(wi, V[:, j])))
    return out


def product(W, V, k):
    return api.tsmm(colmajor(W), torch.from_numpy(V).cuda(), k, arith="f64").t().cpu().numpy()


def check(W, V, k, Y, sample, ulps=4, maxima=False):
    """|Y - WV| <= ulps 2^-53 sum_k |W_ik| |V_kj| on the sampled rows.  maxima: the bound of
    a fixed-point splitting, whose digits are exact relative to the largest entry of each row
    of W and column of V, is max(sum_k |W_ik| |V_kj|, max_k |W_ik| max_k |V_kj|); one unit of
    the subnormal range is allowed where the result itself is subnormal."""
    ref = exact_rows(W, V, sample, k)
    Ws, Vk = np.abs(W[sample]), np.abs(V[:, :k])
    bound = Ws @ Vk
    if maxima:
        bound = np.maximum(bound, np.max(Ws, axis=1)[:, None] * np.max(Vk, axis=0)[None, :])
    err = np.abs(Y[sample] - ref)
    ok = err <= ulps * 2.0 ** -53 * bound + 2.0 ** -1073
    assert ok.all(), (np.argwhere(~ok)[:4].tolist(), np.max(err / np.where(bound > 0, bound, 1)))


@pytest.mark.parametrize("rows,m,k", [(128, 16, 1), (129, 16, 16), (1000, 33, 7), (5000, 48, 16),
                                      (300001, 64, 10), (4097, 64, 16), (20000, 17, 3)])
def test_ws_product_is_fp64_accurate(rows, m, k):
    rng = np.random.default_rng(rows * 3 + m)
    W = rng.standard_normal((rows, m)) * np.exp2(rng.integers(-40, 40, size=(rows, 1)))
    V = np.linalg.qr(rng.standard_normal((m, m)))[0]
    Y = product(W, V, k)
    sample = sorted(set(rng.choice(rows, size=min(rows, 48), replace=False).tolist()) | {0, rows - 1})
    check(W, V, k, Y, sample)


def test_ws_edge_rows():
    # row maxima at and just below a power of two, of either sign; zero rows; rows of
    # subnormal numbers; a row whose maximum is the smallest normal number; huge rows
    rng = np.random.default_rng(7)
    rows, m, k = 1024, 64, 10
    W = rng.standard_normal((rows, m))
    W[1, 5] = np.nextafter(2.0, 0.0)
    W[2, 9] = -np.nextafter(2.0, 0.0)
    W[3, :] = 1.9961
    W[4, :] = -np.nextafter(4.0, 0.0)
    W[5, :] = 0.0
    W[6, :] = rng.standard_normal(m) * 2.0 ** -1060          # subnormal entries
    W[7, :] = rng.standard_normal(m) * 2.0 ** -1022
    W[8, :] = rng.standard_normal(m) * 2.0 ** 1000
    W[9, ::2] = 0.0
    W[10, 3] = 2.0 ** 1023 * np.nextafter(2.0, 0.0)          # the largest finite number
    W[10, 4:] = 0.0
    V = np.linalg.qr(rng.standard_normal((m, m)))[0]
    Y = product(W, V, k)
    assert np.all(Y[5] == 0.0)
    check(W, V, k, Y, list(range(12)) + [rows - 1], ulps=8, maxima=True)


def test_ws_column_scales_of_v():
    # columns of V of very different magnitudes, one of them zero
    rng = np.random.default_rng(11)
    rows, m, k = 5000, 32, 12
    W = rng.standard_normal((rows, m))
    V = rng.standard_normal((m, m)) * np.exp2(rng.integers(-300, 300, size=(1, m)))
    V[:, 2] = 0.0
    V[:, 5] = np.nextafter(2.0, 0.0)
    Y = product(W, V, k)
    assert np.all(Y[:, 2] == 0.0)
    check(W, V, k, Y, list(range(0, rows, 250)), ulps=8, maxima=True)


def test_ws_nonfinite_rows_stay_in_their_rows():
    rng = np.random.default_rng(5)
    rows, m, k = 2000, 64, 10
    W = rng.standard_normal((rows, m))
    W[17, 3] = np.nan
    W[400, 60] = np.inf
    V = np.linalg.qr(rng.standard_normal((m, m)))[0]
    Y = product(W, V, k)
    assert np.all(np.isnan(Y[17])) and np.all(np.isnan(Y[400]))
    good = [i for i in range(0, rows, 37) if i not in (17, 400)]
    assert np.all(np.isfinite(Y[good]))
    check(W, V, k, Y, good)


def test_ws_equals_ozaki_kernel_and_unaligned_fallback():
    # the pipeline against the mma.sync Ozaki kernel (tsmm.ws off): both FP64-accurate; and a
    # W starting 8 bytes off a 16-byte boundary (no tensor map: the Ozaki kernel runs)
    rng = np.random.default_rng(9)
    rows, m, k = 100000, 64, 10
    W = rng.standard_normal((rows, m))
    V = np.linalg.qr(rng.standard_normal((m, m)))[0]
    Yw = product(W, V, k)
    capi.tt_tune_set("tsmm.ws", 0)
    try:
        Yo = product(W, V, k)
    finally:
        capi.tt_tune_set("tsmm.ws", 1)
    bound = np.abs(W) @ np.abs(V[:, :k])
    assert np.max(np.abs(Yw - Yo) / bound) <= 8 * 2.0 ** -53
    buf = torch.empty(rows * m + 1, dtype=torch.float64, device="cuda")
    Wd = buf[1:].view(m, rows)
    Wd.copy_(torch.from_numpy(np.ascontiguousarray(W.T)))
    Yu = api.tsmm(Wd, torch.from_numpy(V).cuda(), k, arith="f64").t().cpu().numpy()
    assert np.max(np.abs(Yu - Yo) / bound) <= 8 * 2.0 ** -53


def _run_tt(X, r_max, arith):
    from tests.gpu_common import fortran_flat
    plan = api.TTSVDPlan(X.shape, r_max, 0.0, torch.float64, arith, want_sigma=True)
    plan.run(fortran_flat(X))
    return plan.result()


@pytest.mark.parametrize("arith", ["df", "f64"])
def test_ws_inside_tt_svd_matches_oracle_and_ozaki_kernel(arith):
    # the whole TT-SVD with the pipeline as its first products (float-float V and Y in the
    # float-float form, FP64 in the native form) against the Alg. 1 oracle, and against the
    # same plan with the mma.sync Ozaki kernel
    from oracle import tt_svd_oracle as O
    from paper_2102_00104_gb300.inputs import uniform_tensor
    X = uniform_tensor((8,) * 7, seed=21)
    res = _run_tt(X, 8, arith)
    capi.tt_tune_set("tsmm.ws", 0)
    try:
        res_oz = _run_tt(X, 8, arith)
    finally:
        capi.tt_tune_set("tsmm.ws", 1)
    ref = O.tt_svd(X, 8)
    assert res.ranks == ref.ranks == res_oz.ranks
    smax = max(s[0] for s in ref.sigmas.values())
    bar = 1e-10 if arith == "df" else 1e-12
    for i, s in ref.sigmas.items():
        g, go = res.sigma.get(i), res_oz.sigma.get(i)
        if g is None or torch.isnan(g).any():
            continue
        k = ref.ranks[i - 1]
        assert np.max(np.abs(g.cpu().numpy()[:k] - s[:k])) <= bar * smax
        assert np.max(np.abs(g.cpu().numpy()[:k] - go.cpu().numpy()[:k])) <= bar * smax
    nx = np.linalg.norm(X)
    err = np.linalg.norm(O.tt_full(res.core_arrays()) - X) / nx
    err_ref = np.linalg.norm(O.tt_full(ref.cores) - X) / nx
    assert abs(err - err_ref) <= bar
