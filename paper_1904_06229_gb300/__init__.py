"""GB300-native matrix permanents: the Gray-code Glynn/Ryser sum of
Lundow & Markstrom (arXiv:1904.06229) as sm_103a CUDA kernels behind a C ABI.

Importing the package loads nothing; `paper_1904_06229_gb300.perm` loads the
CUDA library on first use and raises if it is missing.
"""
__all__ = ["perm", "workloads"]
