"""GB300-native pseudo-spectral Navier-Stokes solver (Mortensen, EuroSciPy 2015).

The compute path is libdns.so (hand-written CUDA for sm_103a behind the C
ABI of include/dns.h); ``dns`` is its ctypes binding, ``inputs`` the seeded
synthetic fields, ``build`` the in-tree nvcc build."""
from . import inputs  # noqa: F401

__all__ = ["dns", "inputs", "build"]
