"""GB300-native explicit RK3 time step of the 3D compressible Navier-Stokes
equations on a periodic grid (the Taylor-Green vortex solver of OpenSBLI,
arXiv:1609.01277), behind a C-ABI library ``libosb``.

Import ``paper_1609_01277_gb300.osb`` for the binding; this package
initialiser stays import-light so that ``inputs`` can be used without CUDA.
"""
__all__ = ["inputs", "osb"]
