"""GB300-native RIS field engine (arXiv 2402.13034): C-ABI CUDA library plus a thin binding.

The CUDA library is loaded lazily by :mod:`paper_2402_13034_gb300.risrt`; importing the package
itself loads nothing, so the seeded input generators in :mod:`.scenarios` work on machines
without a GPU.
"""
