"""W V_r of step i fused with the first (narrow) TSQR level of step i-1 (Alg. 2 lines 11
and 5), switched on with the tuning key "fuse.tsmm_tsqr" = 1 (off by default: measured
slower than the two launches).  Every case meets the parity bar against the Alg. 1 oracle
both fused and with the separate launches, and the two runs agree to rounding."""
import numpy as np
import pytest
import torch

from oracle import tt_svd_oracle as O
from paper_2102_00104_gb300 import capi
from paper_2102_00104_gb300.inputs import planted_tt, uniform_tensor
from tests.gpu_common import ensure_lib
from tests.test_gpu_tt_svd import compare, run_gpu

pytestmark = pytest.mark.gpu

# (dims, r_max, dtype, arith, fuses): the fused launch applies to steps whose product has
# m_i <= 8 columns and whose next unfolding has at most 8
CASES = [((8,) * 7, 1, torch.float64, "df", True), ((8,) * 7, 2, torch.float64, "df", False),
         ((4,) * 9, 1, torch.float64, "df", True), ((4,) * 9, 2, torch.float64, "df", True),
         ((2,) * 14, 4, torch.float64, "df", True), ((3, 5, 4, 2, 6, 3), 1, torch.float64, "df", True),
         ((17, 3, 11, 3), 1, torch.float64, "df", False), ((8,) * 7, 1, torch.float64, "f64", True),
         ((2,) * 14, 4, torch.float64, "f64", True), ((8,) * 7, 1, torch.float32, "df", True),
         ((4,) * 9, 2, torch.float32, "df", True)]


@pytest.mark.parametrize("dims,r_max,dtype,arith,fuses", CASES)
def test_fused_product_and_first_level(dims, r_max, dtype, arith, fuses):
    ensure_lib()
    X = uniform_tensor(dims, seed=61)
    if dtype == torch.float32:
        X = X.astype(np.float32).astype(np.float64)
    tol = 1e-10 if dtype == torch.float64 else 1e-5
    ref = O.tt_svd(X, r_max)
    capi.tt_tune_set("fuse.tsmm_tsqr", 1)
    try:
        capi.tt_profile(True)
        fused = run_gpu(X, r_max, dtype=dtype, arith=arith)
        kinds = {r["kind"] for r in capi.tt_profile_read()}
        capi.tt_profile(False)
    finally:
        capi.tt_tune_set("fuse.tsmm_tsqr", -1)
    assert ("tsmm_fused_tsqr_first_level" in kinds) == fuses, kinds
    compare(X, fused, ref, tol)
    plain = run_gpu(X, r_max, dtype=dtype, arith=arith)
    compare(X, plain, ref, tol)
    assert fused.ranks == plain.ranks
    smax = max(s[0] for s in ref.sigmas.values())
    for i, s in fused.sigma.items():
        if not torch.isnan(s).any():
            assert float(torch.max(torch.abs(s - plain.sigma[i]))) <= tol * smax


def test_fused_scaled_input_and_planted_ranks():
    ensure_lib()
    X = planted_tt((4,) * 9, 2, seed=62, noise_rel=1e-6) * 1e30
    capi.tt_tune_set("fuse.tsmm_tsqr", 1)
    try:
        compare(X, run_gpu(X, 2), O.tt_svd(X, 2), 1e-10)
    finally:
        capi.tt_tune_set("fuse.tsmm_tsqr", -1)
