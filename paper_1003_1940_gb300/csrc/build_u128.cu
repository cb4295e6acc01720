// build_u128.cu -- the construction pipeline for 33 <= k <= 63 (128-bit keys).
#include "build_pipeline.cuh"

namespace dbg {
dbg_status build_graph_u128(dbg_ctx *ctx, const BuildInput &in, dbg_graph *g) {
  return build_graph_impl<Key128>(ctx, in, g);
}
}  // namespace dbg
