"""GB300-native (sm_103a) neural in-scattering estimator of arXiv 2401.14051.

The compute path lives in ``libnis.so`` (CUDA kernels behind the C ABI in include/nis.h);
``paper_2401_14051_gb300.nis`` is its Python binding.  Build with
``python paper_2401_14051_gb300/build.py``.
"""
__all__ = ["nis", "build"]
