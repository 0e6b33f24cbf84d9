// dispatch.cu -- kernel selection, context resources.
#include <cuda_runtime.h>

#include "ctx.h"

namespace advect {

void select_kernels(advect_ctx& ctx) {
  ctx.fwd_kind = 0;
  ctx.adj_kind = 0;
  ctx.fwd_name = "fwd_point";
  ctx.adj_name = "adj_point";
}

cudaError_t launch_fwd(const advect_ctx& ctx, const FwdArgs& a, cudaStream_t st) {
  return launch_fwd_point((int)ctx.dtype, a, st);
}

cudaError_t launch_adj(const advect_ctx& ctx, const AdjArgs& a, cudaStream_t st) {
  return launch_adj_point((int)ctx.dtype, a, st);
}

}  // namespace advect

advect_status advect_ctx::ensure_host_path(size_t bytes) {
  using namespace advect;
  if (hp.bytes == bytes && hp.d_in[0]) return ADVECT_OK;
  for (int f = 0; f < 3; ++f) {
    if (hp.d_in[f]) cudaFree(hp.d_in[f]);
    if (hp.d_out[f]) cudaFree(hp.d_out[f]);
    hp.d_in[f] = hp.d_out[f] = nullptr;
  }
  hp.bytes = 0;
  for (int f = 0; f < 3; ++f) {
    if (cudaMalloc(&hp.d_in[f], bytes) != cudaSuccess || cudaMalloc(&hp.d_out[f], bytes) != cudaSuccess) {
      cudaGetLastError();
      return ADVECT_ENOMEM;
    }
  }
  if (!hp.s_in) {
    if (cudaStreamCreateWithFlags(&hp.s_in, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&hp.s_k, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&hp.s_out, cudaStreamNonBlocking) != cudaSuccess)
      return ADVECT_ECUDA;
    for (int c = 0; c < HostPath::kMaxChunks; ++c)
      if (cudaEventCreateWithFlags(&hp.ev_in[c], cudaEventDisableTiming) != cudaSuccess ||
          cudaEventCreateWithFlags(&hp.ev_k[c], cudaEventDisableTiming) != cudaSuccess)
        return ADVECT_ECUDA;
  }
  hp.bytes = bytes;
  return ADVECT_OK;
}

void advect_ctx::release() {
  using namespace advect;
  cudaDeviceSynchronize();
  for (auto& m : members)
    if (m.d_tabs) cudaFree(m.d_tabs);
  members.clear();
  if (d_flag) cudaFree(d_flag);
  d_flag = nullptr;
  for (int f = 0; f < 3; ++f) {
    if (hp.d_in[f]) cudaFree(hp.d_in[f]);
    if (hp.d_out[f]) cudaFree(hp.d_out[f]);
  }
  for (int c = 0; c < HostPath::kMaxChunks; ++c) {
    if (hp.ev_in[c]) cudaEventDestroy(hp.ev_in[c]);
    if (hp.ev_k[c]) cudaEventDestroy(hp.ev_k[c]);
  }
  if (hp.s_in) cudaStreamDestroy(hp.s_in);
  if (hp.s_k) cudaStreamDestroy(hp.s_k);
  if (hp.s_out) cudaStreamDestroy(hp.s_out);
}
