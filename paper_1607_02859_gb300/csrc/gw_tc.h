// Tensor-core (tcgen05) split-precision contractions (internal).
#pragma once

#include "gw_kernels.h"

namespace gw {

// G_occ / G_unocc rows as 3 fp16 (or bf16) split products on tcgen05 with FP32
// accumulation in tensor memory.
gw_status tc_green_rows(gw_ctx* ctx, const GridInfo& g, int n_b, int n_occ, const void* psi,
                        const GreenScales& gs, int r0, int n_rows, gw_prec prec, void* g_occ, void* g_unocc,
                        cudaStream_t st);
// chi rows = -2 G_occ o conj(G_unocc) with both tiles accumulated in tensor memory.
gw_status tc_chi_rows(gw_ctx* ctx, const GridInfo& g, int n_b, int n_occ, const void* psi, const GreenScales& gs,
                      int r0, int n_rows, gw_prec prec, void* chi, cudaStream_t st);

}  // namespace gw
