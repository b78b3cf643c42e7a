"""GB300-native enriched finite-element ChFSI (Kanungo & Gavini, arXiv:1610.02121).

The compute path is the CUDA library ``libefe.so`` (C ABI: include/efe.h);
``System`` is its thin ctypes binding.  Build the library with
``paper_1610_02121_gb300.build.build()``.
"""
from ._lib import Batch, Mlp, System, EfeError, PREC, SYMBOLS, LIB_PATH, KB_HA_PER_K, fermi, load, launch_count  # noqa: F401
