"""GB300-native Zippel reconstruction step (arXiv 2505.24256).

The compute path is the C-ABI library ``libzr.so`` built from ``csrc/`` (CUDA
for sm_103a); :mod:`paper_2505_24256_gb300.zr` is its thin ctypes binding.
:mod:`paper_2505_24256_gb300.workloads` generates seeded synthetic inputs.
"""

__all__ = ["zr", "workloads"]
