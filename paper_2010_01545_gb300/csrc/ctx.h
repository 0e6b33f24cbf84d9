// ctx.h -- the opaque advect_ctx behind the C ABI (internal).
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/advect.h"
#include "kernels.h"

namespace advect {

// One grid of a context (a single-grid context has exactly one).
struct Member {
  int nx = 0, ny = 0, nz = 0;
  double tcx = 0, tcy = 0;
  std::vector<double> h_tabs;   // masked tables, host copy (tzc1|tzc2|tzd1|tzd2)
  double* d_tabs = nullptr;     // device binary64 tables (one allocation with f_tabs)
  float* f_tabs = nullptr;      // device binary32 tables
};

// Device staging buffers and streams of the host-buffer pipeline.
struct HostPath {
  size_t bytes = 0;
  void* d_in[3] = {nullptr, nullptr, nullptr};
  void* d_out[3] = {nullptr, nullptr, nullptr};
  cudaStream_t s_in = nullptr, s_k = nullptr, s_out = nullptr;
  static constexpr int kMaxChunks = 64;
  int nchunk = 32;  // ADVECT_HOST_CHUNKS (1..64) at create time overrides
  cudaEvent_t ev_in[kMaxChunks] = {};
  cudaEvent_t ev_k[kMaxChunks] = {};
};

}  // namespace advect

struct advect_ctx {
  bool ensemble = false;
  advect_dtype dtype = ADVECT_F64;
  int device = 0;
  int sms = 152;  // multiprocessors of the device (read at create time)
  int f64_levels = 0;
  int* d_flag = nullptr;  // device error flag (non-zero: a bounded wait gave up)
  std::vector<advect::Member> members;
  std::string fwd_name, adj_name;
  int fwd_kind = 0, adj_kind = 0;  // kernel variant chosen at create time
  advect::SweepCfg sweep{};      // forward plane-sweep tile (ty == 0: not usable)
  advect::SweepCfg adj_sweep{};  // adjoint plane-sweep tile
  advect::HostPath hp;
  void* ens = nullptr;  // ensemble state (ens.cu)
  bool tune_fwd = false, tune_adj = false;  // tune on the next forward / adjoint call
  // Test-only fault injection for the bounded-wait path (ADVECT_TEST_SKIP_PLANE,
  // ADVECT_TEST_WAIT_CYCLES read at create time): the sweep kernels never issue
  // the copy of that plane index of each tile, so waits on it run out.
  int test_skip_plane = -1;
  long long wait_budget = 2LL * 1000 * 1000 * 1000;
  std::string cfg_text[2];                  // storage for advect_tuned_config

  // step != NULL: the integration epilogue (base fields step->b, NULL for
  // the winds, and step->dt); such calls never run the tuner, because an
  // in-place step must not be applied more than once.
  struct Step {
    const void* b[3];
    double dt;
  };
  advect_status launch_forward(const void* u, const void* v, const void* w, void* su, void* sv,
                               void* sw, const advect::Scales& sc, int i0, int i1, cudaStream_t st,
                               const Step* step = nullptr);
  advect_status ensure_host_path(size_t bytes);
  void release();
};

namespace advect {
// Kernel selection and launch (dispatch.cu).
void select_kernels(advect_ctx& ctx);
SweepCfg default_sweep(int nz, int elem);  // ty == 0: the shape cannot use the plane sweep
// The forward tile a new context of this element type (Dtype) starts from,
// before the tuning cache or an environment override.
SweepCfg default_fwd_sweep(int nz, int dtype);
cudaError_t tune_single(advect_ctx& ctx, int adj, const FwdArgs* fa, const AdjArgs* aa, cudaStream_t st);
cudaError_t launch_fwd(const advect_ctx& ctx, const FwdArgs& a, cudaStream_t st);
cudaError_t launch_adj(const advect_ctx& ctx, const AdjArgs& a, cudaStream_t st);
}  // namespace advect
