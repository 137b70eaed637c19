"""SU(3) Landau / Coulomb gauge fixing by checkerboard overrelaxation on GB300.

The compute path is the CUDA library ``libgf.so`` (built from ``csrc/``) behind the
C ABI declared in ``include/gf.h``; ``gf`` is its thin Python binding and
``fields`` makes seeded synthetic input fields.  Importing the package does not load
the CUDA library; importing ``gf`` does, and fails loudly if it is missing.
"""
__all__ = ["fields", "gf"]
