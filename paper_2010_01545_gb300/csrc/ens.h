// ens.h -- ensemble state and launch (internal; see ens.cu).
#pragma once

#include <cuda_runtime.h>

#include <string>

#include "../../include/advect.h"

struct advect_ctx;

namespace advect {

struct EnsCfg {
  int lx;   // x-planes per tile
  int nb;   // ring slots
  int occ;  // CTAs per SM the registers are capped for (2, 3 or 4)
};

struct EnsState;

EnsState* ens_new(advect_ctx& ctx);
void ens_free(EnsState* st);
advect_status ens_check_members(const advect_ctx& ctx, std::string& why);
EnsCfg& ens_cfg(EnsState& st, int adj);
size_t ens_smem_bytes(const EnsState& st, int adj, const EnsCfg& cfg);
bool ens_ptrs_changed(EnsState& st, int adj, const void* const* const* in, int n_in, void* const* const* out,
                      int n_members);
cudaError_t ens_run(advect_ctx& ctx, EnsState& st, int adj, const EnsCfg& cfg, const void* const* const* in,
                    void* const* const* out, bool ptrs_changed, cudaStream_t stream, bool use_graph);

}  // namespace advect
