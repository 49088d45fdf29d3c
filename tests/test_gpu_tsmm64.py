"""The native FP64 form's W V_r on the tensor cores (FP64-accurate Ozaki splitting): each
output is within a few units of 2^-53 of sum_k |W_ik| |V_kj| of the exact product, checked
entry by entry against rational arithmetic on sampled rows; the FP64 FMA form (m < 16)
and the float-float form are checked the same way at their own bounds."""
from fractions import Fraction

import numpy as np
import pytest
import torch

from paper_2102_00104_gb300 import api
from tests.gpu_common import colmajor, ensure_lib

pytestmark = pytest.mark.gpu


def exact_rows(W, V, rows, k):
    """Exact W[rows] V[:, :k] (rationals), rounded to FP64 at the end."""
    out = np.empty((len(rows), k))
    for a, i in enumerate(rows):
        wi = [Fraction(float(x)) for x in W[i]]
        for j in range(k):
            out[a, j] = float(sum(x * Fraction(float(v)) for x, v in zip(wi, V[:, j])))
    return out


@pytest.mark.parametrize("rows,m,k,scale", [(100000, 64, 10, 1.0), (70001, 80, 32, 1e-30),
                                            (5000, 96, 7, 3e20), (4096, 17, 1, 1.0), (3000, 12, 5, 1.0),
                                            (20000, 64, 10, 1e-280), (20000, 64, 10, 1e280),
                                            # r > 32: two launches of up to 32 columns
                                            (30000, 64, 50, 1.0), (4096, 96, 64, 1.0), (3000, 40, 33, 1.0)])
def test_native_fp64_product_is_fp64_accurate(rows, m, k, scale):
    ensure_lib()
    rng = np.random.default_rng(rows + m)
    W = (rng.standard_normal((rows, m)) * scale) * np.exp2(rng.integers(-20, 20, size=(rows, 1)))
    V = np.linalg.qr(rng.standard_normal((m, m)))[0]
    Y = api.tsmm(colmajor(W), torch.from_numpy(V).cuda(), k, arith="f64").t().cpu().numpy()
    sample = list(rng.choice(rows, size=40, replace=False)) + [0, rows - 1]
    ref = exact_rows(W, V, sample, k)
    bound = np.abs(W[sample]) @ np.abs(V[:, :k])  # sum_k |W_ik| |V_kj|
    err = np.abs(Y[sample] - ref) / bound
    assert np.max(err) <= 4 * 2.0 ** -53, np.max(err)
    # the float-float form's product is ~2^-46 normwise: the FP64 form is well below it.
    # The stand-alone float-float product computes in FP32's exponent range (row maxima
    # within [2^-100, 2^100]; tt_svd brings its input there first), so it is compared only
    # where the rows stay inside it
    rowmax = np.max(np.abs(W), axis=1)
    if m >= 16 and rowmax.min() >= 2.0 ** -100 and rowmax.max() <= 2.0 ** 100:
        Ydf = api.tsmm(colmajor(W), torch.from_numpy(V).cuda(), k).t().cpu().numpy()
        err_df = np.max(np.abs(Ydf[sample] - ref) / bound)
        assert err_df <= 2.0 ** -40
