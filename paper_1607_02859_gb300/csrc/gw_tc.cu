// Tensor-core split-precision contractions.
#include "gw_tc.h"

namespace gw {

gw_status tc_green_rows(gw_ctx* ctx, const GridInfo&, int, int, const void*, const GreenScales&, int, int, gw_prec,
                        void*, void*, cudaStream_t) {
  return fail(ctx, GW_ERR_UNSUPPORTED, "tensor-core precisions are not built yet");
}
gw_status tc_chi_rows(gw_ctx* ctx, const GridInfo&, int, int, const void*, const GreenScales&, int, int, gw_prec,
                      void*, cudaStream_t) {
  return fail(ctx, GW_ERR_UNSUPPORTED, "tensor-core precisions are not built yet");
}

}  // namespace gw
