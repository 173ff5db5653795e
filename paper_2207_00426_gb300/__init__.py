"""Parallel square-root smoothers (arXiv 2207.00426) on GB300.

The compute path lives in the CUDA library ``libsqsm.so`` (sources under
``csrc/``, C ABI in ``include/sqsm.h``).  ``binding`` marshals arguments to
it; nothing in this package computes the method on the CPU.  Submodules are
imported explicitly (``from paper_2207_00426_gb300 import binding``), so that
``workloads`` can be used on a machine without a GPU.
"""
