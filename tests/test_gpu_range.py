"""FP64 inputs of any finite magnitude through the default (float-float) FP64 form.

Float-float has FP32's exponent range, so the engine reads X as X 2^-k with an exact
power of two k from X's largest magnitude (a strided sample, checked by the first TSQR
level, which runs again when it meets an entry far above the sample) and scales sigma,
the discarded energy and the last core back.  Every case meets the FP64 bar of the other
parity tests against the Alg. 1 oracle: ranks exact, kept sigma within 1e-10 sigma_max,
reconstruction error within 1e-10 of the oracle's, cores orthonormal.
"""
import numpy as np
import pytest
import torch

from oracle import tt_svd_oracle as O
from paper_2102_00104_gb300 import api
from paper_2102_00104_gb300.inputs import uniform_tensor
from tests.gpu_common import colmajor, ensure_lib, fortran_flat
from tests.test_gpu_tt_svd import compare, run_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_lib()


# (2^-400: the oracle's and the test's own FP64 norms of X still stay in range)
SCALES = [2.0 ** 100, 2.0 ** -100, 1e30, 1e-30, 2.0 ** 500, 2.0 ** -400]


@pytest.mark.parametrize("scale", SCALES)
@pytest.mark.parametrize("dims,r_max", [((4,) * 6, 5), ((8, 8, 8, 8, 8), 10), ((4,) * 9, 2)])
def test_scaled_tensor(scale, dims, r_max):
    X = uniform_tensor(dims, seed=31) * scale
    compare(X, run_gpu(X, r_max), O.tt_svd(X, r_max), 1e-10)


def test_subnormal_values_are_read_exactly():
    # every entry below DBL_MIN (its squares underflow even in FP64, so the comparison
    # scales back by the exact power of two: the oracle runs on Xs 2^p, which is exact,
    # and sigma and the norm-carrying first core of the GPU result are scaled by 2^p)
    dims, r_max, p = (4,) * 6, 4, 1030
    Xs = np.ldexp(uniform_tensor(dims, seed=32), -p)
    assert np.all(np.abs(Xs) < np.finfo(np.float64).tiny)
    res = run_gpu(Xs, r_max)
    up = lambda t: t * 2.0 ** (p // 2) * 2.0 ** (p - p // 2)  # exact: two powers of two
    res.cores[0] = up(res.cores[0])
    res.sigma = {i: up(s) for i, s in res.sigma.items()}
    X = np.ldexp(Xs, p)
    # err2 of Xs itself (~2^-2p) is below FP64's range: it is not compared
    compare(X, res, O.tt_svd(X, r_max), 1e-10, check_err2=False)


def test_deep_subnormal_values():
    # entries near 2^-1074 have few significant bits and so have the FP64 outputs: sigma
    # (itself subnormal) is checked to within a few units of 2^-1074, the ranks exactly
    dims, r_max, p = (4,) * 6, 4, 1060
    Xs = np.ldexp(uniform_tensor(dims, seed=32), -p)
    res = run_gpu(Xs, r_max)
    ref = O.tt_svd(np.ldexp(Xs, p), r_max)
    assert res.ranks == ref.ranks
    for i, s_ref in ref.sigmas.items():
        g = res.sigma.get(i)
        if g is None or torch.isnan(g).any():
            continue
        k = ref.ranks[i - 1]
        got = np.ldexp(g.cpu().numpy()[:k], p)
        tol = 1e-10 * ref.sigmas[6][0] + np.ldexp(4.0, p - 1074)
        assert np.max(np.abs(got - s_ref[:k])) <= tol, (i, got, s_ref[:k])


def column_span(dims, seed):
    """Slabs of the last index scaled from 1e-20 to 1e20: a 1e40 spread across the
    columns of the first unfolding."""
    X = uniform_tensor(dims, seed=seed)
    n = dims[-1]
    return X * (10.0 ** np.linspace(-20, 20, n))[None, ...].reshape((1,) * (len(dims) - 1) + (n,))


@pytest.mark.parametrize("dims,r_max", [((4, 4, 4, 4, 4, 5), 6), ((8, 8, 8, 8, 9), 10)])
def test_magnitudes_across_columns(dims, r_max):
    X = column_span(dims, 33)
    compare(X, run_gpu(X, r_max), O.tt_svd(X, r_max), 1e-10)


def test_outlier_outside_the_sample_reruns_the_first_level():
    # 4^9 entries: the strided sample takes every 4th one, so an entry at index 1 is not
    # in it; 1e25 against uniform[0,1) values is far above the sample's range
    dims = (4,) * 9
    X = uniform_tensor(dims, seed=34)
    flat = X.ravel(order="F")
    flat[1] = 1e25
    X = flat.reshape(dims, order="F")
    compare(X, run_gpu(X, 4), O.tt_svd(X, 4), 1e-10)


@pytest.mark.parametrize("scale", [1e30, 1e-30])
def test_scaled_from_host_and_variants(scale):
    dims, r_max = (8, 8, 8, 8, 8), 10
    X = uniform_tensor(dims, seed=35) * scale
    ref = O.tt_svd(X, r_max)
    # X in pinned host memory (host-side sample)
    plan = api.TTSVDPlan(dims, r_max, 0.0, torch.float64, "df", want_sigma=True)
    plan.run_host(fortran_flat(X).cpu().pin_memory(), chunks=4)
    compare(X, plan.result(), ref, 1e-10)
    # native FP64 arithmetic needs no shift; it must agree as well
    compare(X, run_gpu(X, r_max, arith="f64"), ref, 1e-10)
    # two-sided variant (Alg. 4) and thick-bounds variant (Alg. 3)
    from oracle.thick_bounds import tt_svd_thick
    from oracle.two_sided import tt_svd_two_sided
    nx = np.linalg.norm(X)
    for kw, oref in (({"two_sided": True}, tt_svd_two_sided(X, r_max)),
                     ({"thick": (16, 0.5)}, tt_svd_thick(X, r_max, 16, 0.5))):
        p = api.TTSVDPlan(dims, r_max, 0.0, torch.float64, "df", **kw)
        p.run(fortran_flat(X))
        res = p.result()
        assert res.ranks == oref.ranks
        err = np.linalg.norm(O.tt_full(res.core_arrays()) - X) / nx
        err_ref = np.linalg.norm(O.tt_full(oref.cores) - X) / nx
        assert abs(err - err_ref) <= 1e-10, (kw, err, err_ref)
        assert abs(res.err2 - oref.err2) <= 1e-10 * nx * nx


@pytest.mark.parametrize("scale", [1e-30, 1e30, 2.0 ** 600])
def test_tsqr_building_block_scaled(scale):
    rng = np.random.default_rng(36)
    W = rng.random((70000, 40)) * scale
    R = api.tsqr(colmajor(W)).cpu().numpy()
    sig = np.linalg.svd(R, compute_uv=False)
    ref = np.linalg.svd(W, compute_uv=False)
    assert np.max(np.abs(sig - ref)) <= 1e-12 * ref[0]


@pytest.mark.parametrize("scale", [2.0 ** 100, 2.0 ** -100, 2.0 ** -120])
def test_scaled_fp32_form(scale):
    # FP32 storage: squares of 2^-100 or 2^100 values leave FP32's range, so the FP32 form
    # reads its input shifted as well; the bar is the FP32 form's 1e-5
    dims, r_max = (8, 8, 8, 8, 8), 16
    X32 = (uniform_tensor(dims, seed=37) * scale).astype(np.float32).astype(np.float64)
    res = run_gpu(X32, r_max, dtype=torch.float32)
    compare(X32, res, O.tt_svd(X32, r_max), 1e-5)


def test_tsqr_building_block_fp32_tiny():
    rng = np.random.default_rng(38)
    W = (rng.random((70000, 40)) * 2.0 ** -110).astype(np.float32)
    R = api.tsqr(colmajor(W, torch.float32)).cpu().numpy()
    sig = np.linalg.svd(R, compute_uv=False)
    ref = np.linalg.svd(W.astype(np.float64), compute_uv=False)
    assert np.max(np.abs(sig - ref)) <= 2e-5 * ref[0]


@pytest.mark.parametrize("bad", [np.nan, np.inf, -np.inf])
@pytest.mark.parametrize("where", [0, 4000, 8 ** 5 - 1])
@pytest.mark.parametrize("dtype,arith", [(torch.float64, "df"), (torch.float64, "f64"), (torch.float32, "df")])
def test_non_finite_input_is_reported(bad, where, dtype, arith):
    # a NaN or an infinity anywhere in X must surface as TT_ENUMERIC (a non-finite singular
    # value), never as a finite result: the digit extraction of the tensor-core products
    # reads exponent fields and could otherwise turn such a value into finite garbage
    X = uniform_tensor((8,) * 5, seed=5)
    Xf = X.ravel(order="F").copy()
    Xf[where] = bad
    plan = api.TTSVDPlan((8,) * 5, 10, 0.0, dtype, arith, want_sigma=True)
    plan.run(torch.from_numpy(Xf).to("cuda", dtype))
    assert plan.device_status() == api.capi.TT_ENUMERIC
