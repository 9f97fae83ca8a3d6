"""GB300-native staggered Dslash / even-odd CG library (paper arXiv 1311.2719's hot path).

Import ``paper_1311_2719_gb300.qcd`` for the binding of the CUDA library (libqcd.so); it is not
imported here so that the seeded input generators in ``inputs`` load without a built library.
"""
__all__ = ["inputs", "qcd"]
