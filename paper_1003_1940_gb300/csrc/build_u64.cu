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

namespace dbg {
// flag[v] = 1 when node v's k-mer lies in at least t distinct reads
static __global__ void k_roadmap_flags(const uint32_t *__restrict__ reads_per_node, uint64_t V, uint32_t t,
                                       uint32_t *__restrict__ flag) {
  for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < V; v += (uint64_t)gridDim.x * blockDim.x)
    flag[v] = reads_per_node[v] >= t ? 1u : 0u;
}

// the flagged node IDs, ascending, at their scanned positions
static __global__ void k_roadmap_write(const uint32_t *__restrict__ flag, const uint64_t *__restrict__ pos,
                                       uint64_t V, uint32_t *__restrict__ ids) {
  for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < V; v += (uint64_t)gridDim.x * blockDim.x)
    if (flag[v]) ids[pos[v]] = (uint32_t)v;
}

// The roadmap (Section 7: VELVET keeps the k-mers present in at least 2
// reads): the IDs of the nodes held by at least t distinct reads.
dbg_status roadmap_nodes(dbg_ctx *ctx, const dbg_graph *g, uint32_t t, uint32_t *d_ids, uint64_t *count) {
  cudaStream_t s = ctx->stream;
  const uint64_t V = g->num_nodes;
  *count = 0;
  if (V == 0) return DBG_OK;
  DevBuf flag, pos;
  DBG_TRY(alloc_buf(ctx, flag, V * 4));
  DBG_TRY(alloc_buf(ctx, pos, (V + 1) * 8));
  DBG_LAUNCH(ctx, ST_NODE_MULT, 8.0 * V,
             k_roadmap_flags<<<grid_for(V, 256 * 8), 256, 0, s>>>(g->node_reads.as<uint32_t>(), V, t,
                                                                  flag.as<uint32_t>()));
  uint32_t low = 0;
  DBG_TRY(scan_u32(ctx, flag.as<uint32_t>(), V, pos.as<uint64_t>(), &low, ST_NODE_MULT));
  DBG_TRY(read_small(ctx, pos.as<uint64_t>() + V, sizeof(uint64_t), count));
  if (d_ids && *count)
    DBG_LAUNCH(ctx, ST_NODE_MULT, 16.0 * V,
               k_roadmap_write<<<grid_for(V, 256 * 8), 256, 0, s>>>(flag.as<uint32_t>(), pos.as<uint64_t>(), V,
                                                                    d_ids));
  DBG_CUDA_TRY(cudaGetLastError());
  DBG_CUDA_TRY(cudaStreamSynchronize(s));
  return check_device_error(ctx);
}
}  // namespace dbg
