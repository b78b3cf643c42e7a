"""Batched systems in one CUDA graph and the cell-kernel autotuner.

The graph replays exactly the kernel sequence of the per-system steps (the
same deterministic kernels in the same order per system), so its results must
equal the sequential path bit for bit; a second replay with new filter bounds
must equal a fresh sequential step with those bounds (the coefficients are
refreshed through the graph's copy nodes, not baked in)."""
import numpy as np
import pytest

import workloads as W
from tests.gpu_util import cuda_available, gpu_system, to_dev, torch

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not cuda_available(), reason="needs a CUDA GPU")]


@pytest.fixture(scope="module")
def systems():
    ss = [W.tiny(seed=11), W.tiny(seed=12, cells=(3, 2, 2)), W.hydrogen(cells=4, half=10.0, tau=1e-7, max_depth=6)]
    return ss, [gpu_system(s) for s in ss]


def _blocks(ss, Ns):
    return [to_dev(W.initial_block(s, N, seed=3 + i)) for i, (s, N) in enumerate(zip(ss, Ns))]


def _bounds(Gs, Xs):
    a, b, a0 = [], [], []
    for G, X in zip(Gs, Xs):
        e, _ = G.rayleigh_ritz(X)
        a.append(e.max())
        a0.append(e.min())
        b.append(G.upper_bound(X[:, -1].contiguous(), 10))
    return a, b, a0


@pytest.mark.parametrize("prec,tail", [("fp64", 0), ("tf32x3", 2)])
def test_batch_graph_equals_sequential(systems, prec, tail):
    from paper_1610_02121_gb300 import Batch
    ss, Gs = systems
    Ns = [12, 20, 8]
    X0 = _blocks(ss, Ns)
    a, b, a0 = _bounds(Gs, X0)
    B = Batch(Gs)
    try:
        Xg = [x.clone() for x in X0]
        Xs = [x.clone() for x in X0]
        B.chfsi_step(Xg, 9, a, b, a0, precision=prec, fp64_tail=tail, graph=True)
        B.chfsi_step(Xs, 9, a, b, a0, precision=prec, fp64_tail=tail, graph=False)
        for g, q in zip(Xg, Xs):
            assert torch.equal(g, q)
        nodes, kn = B.graph_nodes()
        assert kn > 0 and nodes >= kn
        # new bounds, same buffers: replay (no new recording) == sequential
        a2 = [x * 1.01 for x in a]
        Xg2 = Xg
        Xs2 = [x.clone() for x in Xg]
        B.chfsi_step(Xg2, 9, a2, b, a0, precision=prec, fp64_tail=tail, graph=True)
        assert B.graph_nodes() == (nodes, kn)
        B.chfsi_step(Xs2, 9, a2, b, a0, precision=prec, fp64_tail=tail, graph=False)
        for g, q in zip(Xg2, Xs2):
            assert torch.equal(g, q)
    finally:
        B.close()


def test_autotune_picks_a_tile_and_keeps_results(systems):
    ss, Gs = systems
    G = Gs[0]
    X = to_dev(W.initial_block(ss[0], 40, seed=5))
    a, b, a0 = _bounds([G], [X])
    ref = X.clone()
    G.chfsi_step(ref, 7, a[0], b[0], a0[0], precision="tf32x3", fp64_tail=1)
    tile, ms = G.autotune(40, "tf32x3")
    assert tile in (64, 96, 160) and np.all(ms > 0)
    got = X.clone()
    G.chfsi_step(got, 7, a[0], b[0], a0[0], precision="tf32x3", fp64_tail=1)
    # another column tile regroups the columns; each column's products and sums are unchanged
    assert (got - ref).abs().max().item() <= 1e-6 * ref.abs().max().item()


@pytest.mark.parametrize("prec,m,tol", [("fp64", 7, 1e-9), ("tf32x3", 7, 5e-5), ("bf16", 1, 5e-2)])
def test_batch_each_system_matches_oracle(systems, prec, m, tol):
    """Every system of a batched graph step (three meshes and block widths)
    against the oracle's scaled filter of that system: FP64 to rounding, the
    3-term TF32 split to FP32 grade, BF16 operands to BF16 grade (one degree)."""
    from oracle.chfsi import chebyshev_filter_scaled
    from oracle.operators import Discretisation
    from paper_1610_02121_gb300 import Batch
    from tests.gpu_util import rel_err
    ss, Gs = systems
    Ns = [12, 20, 8]
    X0 = _blocks(ss, Ns)
    a, b, a0 = _bounds(Gs, X0)
    B = Batch(Gs)
    try:
        Xg = [x.clone() for x in X0]
        B.chfsi_step(Xg, m, a, b, a0, precision=prec, fp64_tail=0, graph=True)
    finally:
        B.close()
    for s, x0, xg, ai, bi, a0i in zip(ss, X0, Xg, a, b, a0):
        d = Discretisation(s)
        ref = chebyshev_filter_scaled(d.apply_Htilde, x0.cpu().numpy(), m, ai, bi, a0i)
        assert rel_err(xg, ref) < tol, s["name"]
