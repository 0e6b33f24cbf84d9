// fwd_sweep.cu -- single-grid plane-sweep forward (the source terms); the
// kernel templates are in fwd_sweep.cuh.
#include "fwd_sweep.cuh"

namespace advect {

size_t sweep_smem_bytes(int nz, int elem, const SweepCfg& cfg) {
  // the F16S sweep keeps its coefficient table after the ring
  return sweep::ring_bytes(cfg.nb, (size_t)3 * (cfg.ty + 2) * nz * elem) +
         (elem == 2 ? sweep::h16::table_bytes(nz) : 0);
}

// levels per thread of the forward sweep: binary64 2, binary32 4, binary16 8
int sweep_vec(int elem) { return elem == 8 ? 2 : (elem == 4 ? 4 : 8); }

cudaError_t launch_fwd_sweep(int dtype, const FwdArgs& a, const SweepCfg& cfg, int* flag, cudaStream_t st) {
  if (a.i1 <= a.i0) return cudaSuccess;
  if (a.integ) return launch_fwd_sweep_integ(dtype, a, cfg, flag, st);
  switch (dtype) {
    case kF64: return launch_t<double, false>(a, cfg, flag, st);
    case kF32: return launch_t<float, false>(a, cfg, flag, st);
    case kF16S: return launch_t<__half, false>(a, cfg, flag, st);
    case kF64FF: return launch_t<f64ff, false>(a, cfg, flag, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace advect
