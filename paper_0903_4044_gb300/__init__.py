"""GB300 (sm_103a) BGK phase-space solver behind a C ABI (include/bgk.h).

Submodules:
  bgk        ctypes binding of libbgk.so, C names (argument marshalling only)
  solver     Solver object and builders for the shock and cavity problems
  workloads  seeded synthetic inputs and raw workload parameters
  build      in-tree nvcc build of libbgk.so

Imports are lazy so that ``workloads`` can be used without loading the
CUDA library.
"""

__all__ = ["bgk", "solver", "workloads", "build"]
