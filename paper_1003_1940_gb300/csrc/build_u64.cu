// build_u64.cu -- the construction pipeline for k <= 31 (64-bit keys).
#include "build_pipeline.cuh"

namespace dbg {
dbg_status build_graph_u64(dbg_ctx *ctx, const BuildInput &in, dbg_graph *g) {
  return build_graph_impl<uint64_t>(ctx, in, g);
}
}  // namespace dbg

namespace dbg {
dbg_status autotune_u64(dbg_ctx *ctx, uint64_t n, double *ms_keys, double *ms_pairs) {
  DBG_TRY((autotune_kind<uint64_t, false>(ctx, n, ms_keys)));
  return autotune_kind<uint64_t, true>(ctx, n, ms_pairs);
}
const char *sort_variant_name_u64(bool pairs, uint32_t v, uint32_t *count) {
  return pairs ? variant_name<uint64_t, true>(v, count) : variant_name<uint64_t, false>(v, count);
}
}  // namespace dbg

namespace dbg {
dbg_status build_bucketed_u64(dbg_ctx *ctx, const BucketInput &in, uint64_t budget, dbg_graph *g, uint32_t *eb,
                              uint32_t *nb) {
  return build_bucketed_impl<uint64_t>(ctx, in, budget, g, eb, nb);
}
}  // namespace dbg
