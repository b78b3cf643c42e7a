"""The C-ABI library builds, loads and exports every symbol include/efe.h declares (no GPU needed)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "efe.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(efe_[a-zA-Z0-9_]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol():
    import __graft_entry__ as g
    g.build()
    from paper_1610_02121_gb300 import LIB_PATH, SYMBOLS
    lib = ctypes.CDLL(LIB_PATH)
    names = _declared()
    assert len(names) >= 16
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(SYMBOLS) == names


def test_product_does_not_import_oracle():
    pkg = os.path.join(ROOT, "paper_1610_02121_gb300")
    for dp, _, fs in os.walk(pkg):
        for f in fs:
            if f.endswith((".py", ".cu", ".cpp", ".h")):
                src = open(os.path.join(dp, f)).read()
                assert "import oracle" not in src and "from oracle" not in src, f


def test_binding_rejects_bad_blocks_before_any_launch():
    """The binding validates every vector block on the host (no GPU involved):
    wrong dtype, row count, output shape or strides raise before a pointer is
    passed to the library."""
    import pytest
    torch = pytest.importorskip("torch")
    from paper_1610_02121_gb300._lib import check_block
    rows = 40
    good = torch.zeros((rows, 5), dtype=torch.float64)
    with pytest.raises(ValueError, match="float64"):
        check_block(torch.zeros((rows, 5), dtype=torch.float32), rows)
    with pytest.raises(ValueError, match="rows"):
        check_block(torch.zeros((rows - 1, 5), dtype=torch.float64), rows)
    with pytest.raises(ValueError, match="2-D"):
        check_block(torch.zeros(rows, dtype=torch.float64), rows)
    with pytest.raises(ValueError, match="differs"):
        check_block(torch.zeros((rows, 4), dtype=torch.float64), rows, like=good)
    with pytest.raises(ValueError, match="stride"):
        check_block(torch.zeros((5, rows), dtype=torch.float64).T, rows)
    with pytest.raises(TypeError):
        check_block(good.numpy(), rows)
    # a well-formed block that is not on a CUDA device is refused last
    with pytest.raises(ValueError, match="CUDA"):
        check_block(good, rows, like=good)
