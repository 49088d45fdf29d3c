"""GB300 (sm_103a) TT-SVD engine: the truncated tensor-train SVD of a dense tensor,
core by core (Alg. 2 of Roehrig-Zoellner, Thies, Basermann), as hand-written CUDA
behind the C ABI of include/tt_svd.h.

``capi``   ctypes binding with the C names (argument marshalling only)
``api``    PyTorch-facing helpers (device memory, streams): tt_svd, TTSVDPlan, ...
``inputs`` seeded synthetic inputs shared with the tests and the oracle
``build``  compiles libttsvd.so in-tree with nvcc for sm_103a
"""
from . import capi  # noqa: F401  (loads the library lazily, on first call)


def __getattr__(name):
    # the torch-facing helpers are imported on first use so that ``inputs`` and
    # ``capi`` stay importable without initialising PyTorch
    if name in ("tt_svd", "TTSVDPlan", "TTResult", "gen_uniform", "tsqr", "small_svd", "tsmm"):
        from . import api
        return getattr(api, name)
    raise AttributeError(name)
