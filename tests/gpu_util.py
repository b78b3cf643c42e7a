"""Helpers shared by the GPU parity tests (CUDA path through the C ABI vs the oracle)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def cuda_available():
    return torch.cuda.is_available()


def gpu_system(system):
    import __graft_entry__ as g
    g.build()
    from paper_1610_02121_gb300 import System
    S = System(system)
    S.set_potential_analytic()
    return S


def to_dev(X):
    return torch.from_numpy(np.ascontiguousarray(X)).to("cuda")


def rel_err(a, ref):
    a = a.detach().cpu().numpy() if hasattr(a, "detach") else np.asarray(a)
    ref = np.asarray(ref)
    return np.abs(a - ref).max() / max(np.abs(ref).max(), 1e-300)
