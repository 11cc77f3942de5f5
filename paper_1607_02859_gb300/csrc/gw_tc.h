// Tensor-core (tcgen05) split-precision contractions (internal).
#pragma once

#include "gw_kernels.h"

namespace gw {

// Scratch the two calls below need for n_rows rows (with_tmp: room for an
// output the caller did not supply).
size_t tc_scratch_bytes(const GridInfo& g, int n_b, int n_occ, int n_rows, bool with_tmp);
// G_occ / G_unocc rows as 3 fp16 (or bf16) split products on tcgen05 with FP32
// accumulation in tensor memory.  Either output may be NULL.  prep_b = false
// reuses the psi-only operand an earlier call left in the same scratch.
gw_status tc_green_rows(gw_ctx* ctx, const GridInfo& g, int n_b, int n_occ, const void* psi,
                        const GreenScales& gs, int r0, int n_rows, gw_prec prec, void* g_occ, void* g_unocc,
                        void* scratch, bool prep_b, cudaStream_t st);
// chi rows = -2 G_occ o conj(G_unocc) with both tiles accumulated in tensor memory.
gw_status tc_chi_rows(gw_ctx* ctx, const GridInfo& g, int n_b, int n_occ, const void* psi, const GreenScales& gs,
                      int r0, int n_rows, gw_prec prec, void* chi, void* scratch, bool prep_b, cudaStream_t st);
// Synchronises and reports a time-out of the tensor-core pipeline waits
// (GW_ERR_TIMEOUT) recorded in `scratch` since its last prep_b call.
gw_status tc_check(gw_ctx* ctx, void* scratch, cudaStream_t st);

}  // namespace gw
