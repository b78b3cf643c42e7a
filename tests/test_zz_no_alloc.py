"""The allocation-free overlap product against the regular one.

efe_apply_M_noalloc serves callers that cannot allocate device memory at call
time (latency-critical loops that cannot take cudaMalloc's synchronisation,
fixed memory budgets): its scratch is a static device array shared by all calls.  Two
consecutive calls through the C ABI must each reproduce efe_apply_M.  This file
is collected last so a failure here never hides another test's result.
"""
import ctypes as C

import pytest

import workloads as W
from tests.gpu_util import cuda_available, gpu_system, rel_err, to_dev, torch

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not cuda_available(), reason="needs a CUDA GPU")]

SCRATCH_DOUBLES = 1 << 21


def test_apply_M_noalloc_matches_apply_M_twice():
    s = W.tiny(seed=11, cells=(2, 2, 2), max_depth=3)
    G = gpu_system(s)
    # N = 3 takes the narrow segment kernel, 9 and 33 the column-parallel one
    for seed, N in [(41, 9), (42, 33), (43, 3)]:
        X = to_dev(W.random_block(s, N, seed=seed))
        ref = G.apply_M(X)
        Y = torch.full_like(X, float("nan"))
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        G.apply_M_noalloc(X, Y)
        G.apply_M_noalloc(X, Y)
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        assert free1 == free0, "the allocation-free product changed the device's free memory"
        assert torch.isfinite(Y).all()
        assert rel_err(Y, ref.cpu().numpy()) < 1e-12


def test_apply_M_noalloc_rejects_sizes_beyond_its_scratch():
    """A block needing more than 2^21 scratch doubles (n_segments x N) is refused
    before any device work and leaves Y untouched.  The blocks are real
    allocations of the claimed size, so nothing could be read or written out of
    bounds even if the check were missing."""
    from paper_1610_02121_gb300 import EfeError
    s = W.tiny(seed=11, cells=(2, 2, 2), max_depth=3)
    G = gpu_system(s)
    assert G.n_enrich > 0
    N = SCRATCH_DOUBLES // G.n_enrich + 1      # n_segments >= n_enrich rows
    X = torch.zeros((G.rows, N), dtype=torch.float64, device="cuda")
    Y = torch.full_like(X, 3.0)
    with pytest.raises(EfeError) as e:
        G.apply_M_noalloc(X, Y)
    assert e.value.code == 1
    torch.cuda.synchronize()
    assert bool((Y == 3.0).all())
    # X and Y must not overlap
    Xs = to_dev(W.random_block(s, 5, seed=3))
    keep = Xs.clone()
    rc = G.L.efe_apply_M_noalloc(G.h, C.c_void_p(Xs.data_ptr()), Xs.stride(0), 5, C.c_void_p(Xs.data_ptr()),
                                 Xs.stride(0), G._stream())
    assert rc == 1
    torch.cuda.synchronize()
    assert torch.equal(Xs, keep)
