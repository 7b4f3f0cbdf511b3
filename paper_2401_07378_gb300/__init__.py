"""GB300 (sm_103a) implementation of the NNS-EMD hot path (arXiv 2401.07378).

* ``paper_2401_07378_gb300.nnsemd``     -- ctypes binding of include/nnsemd.h
  (loads the CUDA library; raises if it is not built).
* ``paper_2401_07378_gb300.build``      -- in-tree nvcc build of that library.
* ``paper_2401_07378_gb300.workloads``  -- seeded synthetic inputs.

Importing the package itself loads nothing, so the generators and the build
step work on machines without a GPU.
"""

__all__ = ["build", "nnsemd", "workloads"]
