"""GB300-native dual-primal IETI (FETI-DP) solver for 3D curl-curl magnetostatics
on multipatch spline discretisations (arXiv 2501.04340).

``workloads`` holds the seeded input generator; ``ieti`` the ctypes binding of
the CUDA library ``libieti.so`` (import it explicitly: it needs the built library).
"""
