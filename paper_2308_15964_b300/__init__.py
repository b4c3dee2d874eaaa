"""B300-native device-scheduled STF tile-task DAG (tiled Cholesky and solve).

The C-ABI library ``libspx.so`` (built from ``csrc/``) holds the whole hot
path; ``spx`` is its thin ctypes binding.  Submodules are imported on demand
so that the seeded input generators can be used without the CUDA library.
"""
__all__ = ["spx", "inputs", "cholesky"]
