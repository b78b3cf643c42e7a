"""Plain FP64 CPU oracle for the enriched finite-element ChFSI method.

TEST INFRASTRUCTURE ONLY.  Nothing in the product package imports, links or
executes this package; only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may use it.

Every function is a slow, direct restatement of the paper
(Kanungo & Gavini, "Large-scale all-electron density functional theory
calculations using an enriched finite element basis", arXiv:1610.02121),
each citing the section / equation it follows.  It shares no code, tables or
helpers with the CUDA path in ``paper_1610_02121_gb300``; the only common
module is ``workloads`` (seeded synthetic inputs, no method arithmetic).

Parity status per function is listed in each module header.  Functions whose
correctness has no independent pin say "parity unpinned".
"""
