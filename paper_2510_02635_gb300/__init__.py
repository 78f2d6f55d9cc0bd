"""GB300-native localized stochastic FBSDE solver (arXiv 2510.02635), hot path in CUDA.

The compute path lives in the C-ABI shared library built from ``csrc/``;
``paper_2510_02635_gb300.fbsde`` is the thin Python binding over it.
"""
