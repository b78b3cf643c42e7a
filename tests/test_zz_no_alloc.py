"""The allocation-free overlap product against the regular one.

efe_apply_M_noalloc serves callers that cannot allocate device memory at call
time (latency-critical loops that cannot take cudaMalloc's synchronisation,
fixed memory budgets): its scratch is a static device array shared by all calls.  Two
consecutive calls through the C ABI must each reproduce efe_apply_M.  This file
is collected last so a failure here never hides another test's result.
"""
import numpy as np
import pytest

import workloads as W
from tests.gpu_util import cuda_available, gpu_system, rel_err, to_dev, torch

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not cuda_available(), reason="needs a CUDA GPU")]


def test_apply_M_noalloc_matches_apply_M_twice():
    s = W.tiny(seed=11, cells=(2, 2, 2), max_depth=3)
    G = gpu_system(s)
    for seed, N in [(41, 9), (42, 33)]:
        X = to_dev(W.random_block(s, N, seed=seed))
        ref = G.apply_M(X)
        Y = torch.full_like(X, float("nan"))
        G.apply_M_noalloc(X, Y)
        torch.cuda.synchronize()
        assert torch.isfinite(Y).all()
        assert rel_err(Y, ref.cpu().numpy()) < 1e-12
