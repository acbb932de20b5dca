"""B300 (sm_103a) library for Vectorial Ray Tracing in freeform gradient-index
media (Chavez-Islas et al.): batched rays, constant optical-path steps,
vectorial Snell refraction, TIR and boundary refraction, in CUDA kernels
behind the C ABI of include/grin.h.

Submodules: `tracer` (the binding: Context, Medium, RayBatch, trace,
trace_host), `workloads` (seeded synthetic media and ray bundles), `build`
(in-tree nvcc build of lib/libgrin_vrt.so).  Importing the package does not
load the CUDA library; the first Context does, and fails loudly if the
library is missing.
"""

__all__ = ["tracer", "workloads", "build"]
