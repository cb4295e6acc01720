// build_u128.cu -- the construction pipeline for 33 <= k <= 63 (128-bit keys).
#include "build_pipeline.cuh"

namespace dbg {
dbg_status build_graph_u128(dbg_ctx *ctx, const BuildInput &in, dbg_graph *g) {
  return build_graph_impl<Key128>(ctx, in, g);
}
}  // namespace dbg

namespace dbg {
dbg_status autotune_u128(dbg_ctx *ctx, uint64_t n, double *ms_keys, double *ms_pairs) {
  DBG_TRY((autotune_kind<Key128, false>(ctx, n, ms_keys)));
  return autotune_kind<Key128, true>(ctx, n, ms_pairs);
}
const char *sort_variant_name_u128(bool pairs, uint32_t v, uint32_t *count) {
  return pairs ? variant_name<Key128, true>(v, count) : variant_name<Key128, false>(v, count);
}
}  // namespace dbg

namespace dbg {
dbg_status build_bucketed_u128(dbg_ctx *ctx, const BucketInput &in, uint64_t budget, dbg_graph *g, uint32_t *eb,
                               uint32_t *nb) {
  return build_bucketed_impl<Key128>(ctx, in, budget, g, eb, nb);
}
}  // namespace dbg
