// Tensor-core (tcgen05) forms of the per-element networks: BF16 and FP8 with FP32 accumulation.
#include "fnn_internal.cuh"

namespace fnn {

fnn_status upload_tc_weights(fnn_ctx *ctx, const fnn_weights *hw) {
  (void)ctx;
  (void)hw;
  return FNN_OK;
}

void free_tc(fnn_ctx *ctx) { (void)ctx; }

fnn_status mlp_tc_forward_backward(fnn_ctx *ctx, const fnn_nlist *nl, fnn_precision prec, cudaStream_t s) {
  (void)nl;
  (void)prec;
  (void)s;
  ctx->last_error = "tensor-core precision forms are not built yet";
  return FNN_E_INVALID;
}

}  // namespace fnn
