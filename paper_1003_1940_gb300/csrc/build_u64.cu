// build_u64.cu -- the construction pipeline for k <= 31 (64-bit keys).
#include "build_pipeline.cuh"

namespace dbg {
dbg_status build_graph_u64(dbg_ctx *ctx, const BuildInput &in, dbg_graph *g) {
  return build_graph_impl<uint64_t>(ctx, in, g);
}
}  // namespace dbg
