// fwd_integ.cu -- single-grid plane-sweep forward fused with the step that
// integrates the source terms into the flow fields (base + dt * source
// term); the kernel templates are in fwd_sweep.cuh.
#include "fwd_sweep.cuh"

namespace advect {

cudaError_t launch_fwd_sweep_integ(int dtype, const FwdArgs& a, const SweepCfg& cfg, int* flag,
                                   cudaStream_t st) {
  if (a.i1 <= a.i0) return cudaSuccess;
  switch (dtype) {
    case kF64: return launch_t<double, true>(a, cfg, flag, st);
    case kF32: return launch_t<float, true>(a, cfg, flag, st);
    case kF16S: return launch_t<__half, true>(a, cfg, flag, st);
    case kF64FF: return launch_t<f64ff, true>(a, cfg, flag, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace advect
