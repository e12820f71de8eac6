// Tensor-core (tcgen05) split-precision Sigma path -- placeholder until the
// kernels land; reports GF2_ERR_UNSUPPORTED.
#include "gf2_internal.cuh"

gf2_status gf2_tc_prepare_integrals(gf2_ctx *ctx) { (void)ctx; return GF2_ERR_UNSUPPORTED; }

gf2_status gf2_sigma_tc(gf2_ctx *ctx, const double *, int, int, double *, int) {
  return gf2_fail(ctx, GF2_ERR_UNSUPPORTED, "tensor-core path not built");
}
