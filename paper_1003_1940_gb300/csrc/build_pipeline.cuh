// build_pipeline.cuh -- host side of dbg_build for one key width: plans the
// buffers, launches STEP-1..4 on the context's stream, and fills the graph.
#pragma once

#include <algorithm>
#include <cmath>
#include <cstring>
#include <type_traits>

#include "k_build.cuh"
#include "k_segsort.cuh"

namespace dbg {

inline int passes_for_bits(int bits) { return (bits + RADIX_BITS - 1) / RADIX_BITS; }

// items per thread of the build's run-length reduce and node-ID scans
constexpr int BUILD_SCAN_ITEMS = 8;
constexpr int BUILD_SCAN_TILE = SCAN_BLOCK * BUILD_SCAN_ITEMS;

// ---------------------------------------------------------------------------
// Radix sort variants.  Every compiled onesweep configuration of a key kind
// sorts identically; they differ in tile shape, load path and ranking
// method.  The context keeps one choice per kind (default, set by the
// caller, or picked by dbg_autotune).
// ---------------------------------------------------------------------------
using SortLaunchFn = void (*)(dbg_ctx *ctx, const void *kin, void *kout, const uint32_t *vin, uint32_t *vout,
                              uint64_t n, int shift, const uint64_t *digit_base, uint32_t epoch);

struct SortVariant {
  const char *name;
  int tile;
  SortLaunchFn launch;
};

template <class K, bool V, int BLOCK, int ITEMS, int RANK, bool TMA, int MINB, bool EARLY, bool DIRECT = false,
          int LB = 1>
void launch_onesweep(dbg_ctx *ctx, const void *kin, void *kout, const uint32_t *vin, uint32_t *vout, uint64_t n,
                     int shift, const uint64_t *digit_base, uint32_t epoch) {
  auto kern = k_onesweep<K, V, BLOCK, ITEMS, RANK, TMA, MINB, EARLY, DIRECT, LB>;
  constexpr size_t smem = sizeof(OnesweepSmem<K, V, BLOCK, ITEMS>);
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
  const uint64_t tiles = (n + BLOCK * ITEMS - 1) / (BLOCK * ITEMS);
  kern<<<(unsigned)tiles, BLOCK, smem, ctx->stream>>>(static_cast<const K *>(kin), static_cast<K *>(kout), vin,
                                                      vout, n, shift, digit_base, ctx->d_status, ctx->d_counters,
                                                      epoch, ctx->spin_limit, ctx->d_err);
}

template <class K, bool V, int BLOCK, int ITEMS, int RANK, int MINB, int LB, int HB = 4, bool BULK = false>
void launch_onesweep_p(dbg_ctx *ctx, const void *kin, void *kout, const uint32_t *vin, uint32_t *vout, uint64_t n,
                       int shift, const uint64_t *digit_base, uint32_t epoch) {
  auto kern = k_onesweep_p<K, V, BLOCK, ITEMS, RANK, MINB, LB, HB, BULK>;
  constexpr size_t smem = sizeof(OnesweepPSmem<K, V, BLOCK, ITEMS, RANK, HB, BULK>);
  static_assert(smem <= 227 * 1024, "onesweep variant exceeds the shared memory of a CTA");
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
  const uint64_t tiles = (n + BLOCK * ITEMS - 1) / (BLOCK * ITEMS);
  const unsigned grid = (unsigned)std::min<uint64_t>(tiles, (uint64_t)MINB * (uint64_t)ctx->num_sms);
  kern<<<grid, BLOCK, smem, ctx->stream>>>(static_cast<const K *>(kin), static_cast<K *>(kout), vin, vout, n, shift,
                                           digit_base, ctx->d_status, ctx->d_counters, epoch, ctx->spin_limit,
                                           ctx->d_err);
}

#define DBG_SVP(K, V, B, I, R, M, L, NAME) \
  SortVariant { NAME, (B) * (I), &launch_onesweep_p<K, V, B, I, R, M, L> }
#define DBG_SVH(K, V, B, I, R, M, L, NAME) \
  SortVariant { NAME, (B) * (I), &launch_onesweep_p<K, V, B, I, R, M, L, 2> }
#define DBG_SVB(K, V, B, I, R, M, L, NAME) \
  SortVariant { NAME, (B) * (I), &launch_onesweep_p<K, V, B, I, R, M, L, 2, true> }
#define DBG_SV(K, V, B, I, R, T, M, NAME) \
  SortVariant { NAME, (B) * (I), &launch_onesweep<K, V, B, I, R, T, M, false> }
#define DBG_SVE(K, V, B, I, R, T, M, NAME) \
  SortVariant { NAME, (B) * (I), &launch_onesweep<K, V, B, I, R, T, M, true> }
#define DBG_SVL(K, V, B, I, R, T, M, E, L, NAME) \
  SortVariant { NAME, (B) * (I), &launch_onesweep<K, V, B, I, R, T, M, E, false, L> }
#define DBG_SVD(K, V, B, I, R, T, M, E, NAME) \
  SortVariant { NAME, (B) * (I), &launch_onesweep<K, V, B, I, R, T, M, E, true> }

// kinds: 0 = 64-bit keys, 1 = 64-bit keys + payload, 2 = 128-bit keys,
// 3 = 128-bit keys + payload
template <class K, bool V> struct SortKind;
template <> struct SortKind<uint64_t, false> {
  static constexpr int kind = 0;
  static const SortVariant *table(int *count) {
    static const SortVariant t[] = {
        DBG_SV(uint64_t, false, 256, 16, RANK_BALLOT, false, 1, "256x16 ballot ldg"),
        DBG_SV(uint64_t, false, 256, 16, RANK_MATCH, false, 1, "256x16 match ldg"),
        DBG_SV(uint64_t, false, 256, 16, RANK_MATCH, true, 1, "256x16 match tma"),
        DBG_SV(uint64_t, false, 256, 12, RANK_MATCH, true, 3, "256x12 match tma occ3"),
        DBG_SV(uint64_t, false, 256, 12, RANK_ATOMIC, true, 3, "256x12 atomic tma occ3"),
        DBG_SV(uint64_t, false, 256, 8, RANK_MATCH, true, 4, "256x8 match tma occ4"),
        DBG_SV(uint64_t, false, 512, 8, RANK_MATCH, true, 2, "512x8 match tma occ2"),
        DBG_SVE(uint64_t, false, 256, 12, RANK_ATOMIC, true, 3, "256x12 atomic tma occ3 early"),
        DBG_SVE(uint64_t, false, 256, 12, RANK_MATCH, true, 3, "256x12 match tma occ3 early"),
        DBG_SVE(uint64_t, false, 256, 8, RANK_ATOMIC, true, 4, "256x8 atomic tma occ4 early"),
        DBG_SVE(uint64_t, false, 256, 16, RANK_ATOMIC, true, 2, "256x16 atomic tma occ2 early"),
        DBG_SV(uint64_t, false, 256, 8, RANK_ATOMIC, true, 4, "256x8 atomic tma occ4"),
        DBG_SV(uint64_t, false, 256, 10, RANK_ATOMIC, true, 3, "256x10 atomic tma occ3"),
        DBG_SV(uint64_t, false, 384, 8, RANK_ATOMIC, true, 2, "384x8 atomic tma occ2"),
        DBG_SV(uint64_t, false, 512, 6, RANK_ATOMIC, true, 2, "512x6 atomic tma occ2"),
        DBG_SVD(uint64_t, false, 256, 12, RANK_ATOMIC, true, 3, false, "256x12 atomic tma occ3 direct"),
        DBG_SVD(uint64_t, false, 256, 12, RANK_ATOMIC, false, 3, false, "256x12 atomic ldg occ3 direct"),
        DBG_SVD(uint64_t, false, 256, 16, RANK_ATOMIC, false, 2, false, "256x16 atomic ldg occ2 direct"),
        DBG_SVD(uint64_t, false, 256, 12, RANK_ATOMIC, true, 3, true, "256x12 atomic tma occ3 early direct"),
        DBG_SVL(uint64_t, false, 256, 12, RANK_ATOMIC, true, 3, false, 4, "256x12 atomic tma occ3 lb4"),
        DBG_SVL(uint64_t, false, 256, 12, RANK_ATOMIC, true, 3, true, 4, "256x12 atomic tma occ3 early lb4"),
        DBG_SVL(uint64_t, false, 256, 12, RANK_ATOMIC, true, 3, true, 8, "256x12 atomic tma occ3 early lb8"),
        DBG_SVL(uint64_t, false, 256, 16, RANK_ATOMIC, true, 2, true, 8, "256x16 atomic tma occ2 early lb8"),
        DBG_SVL(uint64_t, false, 256, 12, RANK_ATOMIC, true, 3, false, 8, "256x12 atomic tma occ3 lb8"),
        DBG_SVL(uint64_t, false, 256, 12, RANK_ATOMIC, true, 3, false, 16, "256x12 atomic tma occ3 lb16"),
        DBG_SVL(uint64_t, false, 256, 16, RANK_ATOMIC, true, 2, false, 4, "256x16 atomic tma occ2 lb4"),
        DBG_SVL(uint64_t, false, 256, 8, RANK_ATOMIC, true, 4, false, 4, "256x8 atomic tma occ4 lb4"),
        DBG_SVL(uint64_t, false, 256, 10, RANK_ATOMIC, true, 3, false, 8, "256x10 atomic tma occ3 lb8"),
        DBG_SVP(uint64_t, false, 256, 12, RANK_ATOMIC, 3, 4, "256x12 atomic persistent occ3 lb4"),
        DBG_SVP(uint64_t, false, 256, 12, RANK_ATOMIC, 3, 8, "256x12 atomic persistent occ3 lb8"),
        DBG_SVP(uint64_t, false, 256, 8, RANK_ATOMIC, 4, 4, "256x8 atomic persistent occ4 lb4"),
        DBG_SVP(uint64_t, false, 256, 12, RANK_MATCH, 3, 4, "256x12 match persistent occ3 lb4"),
        DBG_SVP(uint64_t, false, 256, 16, RANK_ATOMIC, 2, 4, "256x16 atomic persistent occ2 lb4"),
        DBG_SVP(uint64_t, false, 512, 8, RANK_ATOMIC, 2, 4, "512x8 atomic persistent occ2 lb4"),
        DBG_SVP(uint64_t, false, 1024, 8, RANK_ATOMIC, 1, 4, "1024x8 atomic persistent occ1 lb4"),
        DBG_SVP(uint64_t, false, 1024, 8, RANK_ATOMIC, 1, 8, "1024x8 atomic persistent occ1 lb8"),
        DBG_SVP(uint64_t, false, 768, 8, RANK_ATOMIC, 1, 4, "768x8 atomic persistent occ1 lb4"),
        DBG_SVP(uint64_t, false, 1024, 10, RANK_ATOMIC, 1, 8, "1024x10 atomic persistent occ1 lb8"),
        DBG_SVP(uint64_t, false, 1024, 9, RANK_ATOMIC, 1, 8, "1024x9 atomic persistent occ1 lb8"),
        DBG_SVH(uint64_t, false, 1024, 10, RANK_ATOMIC, 1, 8, "1024x10 atomic persistent occ1 lb8 h16"),
        DBG_SVH(uint64_t, false, 1024, 11, RANK_ATOMIC, 1, 8, "1024x11 atomic persistent occ1 lb8 h16"),
        DBG_SVH(uint64_t, false, 1024, 12, RANK_MATCH, 1, 8, "1024x12 match persistent occ1 lb8 h16"),
        DBG_SVB(uint64_t, false, 1024, 10, RANK_ATOMIC, 1, 8, "1024x10 atomic persistent occ1 lb8 h16 bulk"),
        DBG_SVB(uint64_t, false, 1024, 11, RANK_MATCH, 1, 8, "1024x11 match persistent occ1 lb8 h16 bulk"),
        DBG_SVB(uint64_t, false, 1024, 12, RANK_MATCH, 1, 8, "1024x12 match persistent occ1 lb8 h16 bulk"),
    };
    *count = sizeof(t) / sizeof(t[0]);
    return t;
  }
};
template <> struct SortKind<uint64_t, true> {
  static constexpr int kind = 1;
  static const SortVariant *table(int *count) {
    static const SortVariant t[] = {
        DBG_SV(uint64_t, true, 256, 12, RANK_BALLOT, false, 1, "256x12 ballot ldg"),
        DBG_SV(uint64_t, true, 256, 12, RANK_MATCH, true, 1, "256x12 match tma"),
        DBG_SV(uint64_t, true, 256, 8, RANK_MATCH, true, 3, "256x8 match tma occ3"),
        DBG_SV(uint64_t, true, 256, 8, RANK_ATOMIC, true, 3, "256x8 atomic tma occ3"),
        DBG_SVE(uint64_t, true, 256, 8, RANK_ATOMIC, true, 3, "256x8 atomic tma occ3 early"),
        DBG_SVE(uint64_t, true, 256, 12, RANK_ATOMIC, true, 2, "256x12 atomic tma occ2 early"),
        DBG_SV(uint64_t, true, 256, 10, RANK_ATOMIC, true, 3, "256x10 atomic tma occ3"),
        DBG_SV(uint64_t, true, 384, 8, RANK_ATOMIC, true, 2, "384x8 atomic tma occ2"),
        DBG_SVD(uint64_t, true, 256, 10, RANK_ATOMIC, true, 3, false, "256x10 atomic tma occ3 direct"),
        DBG_SVD(uint64_t, true, 256, 8, RANK_ATOMIC, false, 3, false, "256x8 atomic ldg occ3 direct"),
        DBG_SVL(uint64_t, true, 256, 10, RANK_ATOMIC, true, 3, true, 4, "256x10 atomic tma occ3 early lb4"),
        DBG_SVL(uint64_t, true, 256, 10, RANK_ATOMIC, true, 3, false, 4, "256x10 atomic tma occ3 lb4"),
        DBG_SVL(uint64_t, true, 256, 10, RANK_ATOMIC, true, 3, false, 8, "256x10 atomic tma occ3 lb8"),
        DBG_SVL(uint64_t, true, 256, 8, RANK_ATOMIC, true, 3, false, 8, "256x8 atomic tma occ3 lb8"),
        DBG_SVP(uint64_t, true, 256, 8, RANK_ATOMIC, 3, 4, "256x8 atomic persistent occ3 lb4"),
        DBG_SVP(uint64_t, true, 256, 10, RANK_ATOMIC, 2, 4, "256x10 atomic persistent occ2 lb4"),
        DBG_SVP(uint64_t, true, 256, 6, RANK_ATOMIC, 4, 4, "256x6 atomic persistent occ4 lb4"),
        DBG_SVP(uint64_t, true, 1024, 6, RANK_ATOMIC, 1, 4, "1024x6 atomic persistent occ1 lb4"),
        DBG_SVP(uint64_t, true, 1024, 6, RANK_ATOMIC, 1, 8, "1024x6 atomic persistent occ1 lb8"),
        DBG_SVH(uint64_t, true, 1024, 7, RANK_ATOMIC, 1, 8, "1024x7 atomic persistent occ1 lb8 h16"),
        DBG_SVB(uint64_t, true, 1024, 6, RANK_ATOMIC, 1, 8, "1024x6 atomic persistent occ1 lb8 h16 bulk"),
        DBG_SVB(uint64_t, true, 1024, 7, RANK_MATCH, 1, 8, "1024x7 match persistent occ1 lb8 h16 bulk"),
    };
    *count = sizeof(t) / sizeof(t[0]);
    return t;
  }
};
template <> struct SortKind<Key128, false> {
  static constexpr int kind = 2;
  static const SortVariant *table(int *count) {
    static const SortVariant t[] = {
        DBG_SV(Key128, false, 256, 8, RANK_BALLOT, false, 1, "256x8 ballot ldg"),
        DBG_SV(Key128, false, 256, 8, RANK_MATCH, true, 1, "256x8 match tma"),
        DBG_SV(Key128, false, 256, 6, RANK_MATCH, true, 3, "256x6 match tma occ3"),
        DBG_SVE(Key128, false, 256, 6, RANK_ATOMIC, true, 3, "256x6 atomic tma occ3 early"),
        DBG_SVE(Key128, false, 256, 8, RANK_ATOMIC, true, 2, "256x8 atomic tma occ2 early"),
        DBG_SVD(Key128, false, 256, 8, RANK_ATOMIC, true, 2, true, "256x8 atomic tma occ2 early direct"),
        DBG_SVL(Key128, false, 256, 8, RANK_ATOMIC, true, 2, true, 4, "256x8 atomic tma occ2 early lb4"),
        DBG_SVL(Key128, false, 256, 8, RANK_ATOMIC, true, 2, false, 8, "256x8 atomic tma occ2 lb8"),
        DBG_SVL(Key128, false, 256, 6, RANK_ATOMIC, true, 3, false, 8, "256x6 atomic tma occ3 lb8"),
        DBG_SVP(Key128, false, 256, 6, RANK_ATOMIC, 3, 4, "256x6 atomic persistent occ3 lb4"),
        DBG_SVP(Key128, false, 256, 8, RANK_ATOMIC, 2, 4, "256x8 atomic persistent occ2 lb4"),
        DBG_SVP(Key128, false, 1024, 4, RANK_ATOMIC, 1, 4, "1024x4 atomic persistent occ1 lb4"),
        DBG_SVP(Key128, false, 1024, 5, RANK_ATOMIC, 1, 8, "1024x5 atomic persistent occ1 lb8"),
        DBG_SVH(Key128, false, 1024, 6, RANK_MATCH, 1, 8, "1024x6 match persistent occ1 lb8 h16"),
        DBG_SVB(Key128, false, 1024, 5, RANK_ATOMIC, 1, 8, "1024x5 atomic persistent occ1 lb8 h16 bulk"),
    };
    *count = sizeof(t) / sizeof(t[0]);
    return t;
  }
};
template <> struct SortKind<Key128, true> {
  static constexpr int kind = 3;
  static const SortVariant *table(int *count) {
    static const SortVariant t[] = {
        DBG_SV(Key128, true, 256, 8, RANK_BALLOT, false, 1, "256x8 ballot ldg"),
        DBG_SV(Key128, true, 256, 8, RANK_MATCH, true, 1, "256x8 match tma"),
        DBG_SV(Key128, true, 256, 6, RANK_MATCH, true, 3, "256x6 match tma occ3"),
        DBG_SVE(Key128, true, 256, 6, RANK_ATOMIC, true, 3, "256x6 atomic tma occ3 early"),
        DBG_SVD(Key128, true, 256, 6, RANK_ATOMIC, true, 3, true, "256x6 atomic tma occ3 early direct"),
        DBG_SVL(Key128, true, 256, 6, RANK_ATOMIC, true, 3, true, 4, "256x6 atomic tma occ3 early lb4"),
        DBG_SVL(Key128, true, 256, 6, RANK_ATOMIC, true, 3, false, 8, "256x6 atomic tma occ3 lb8"),
        DBG_SVP(Key128, true, 256, 6, RANK_ATOMIC, 2, 4, "256x6 atomic persistent occ2 lb4"),
        DBG_SVP(Key128, true, 1024, 3, RANK_ATOMIC, 1, 4, "1024x3 atomic persistent occ1 lb4"),
        DBG_SVB(Key128, true, 1024, 3, RANK_ATOMIC, 1, 8, "1024x3 atomic persistent occ1 lb8 h16 bulk"),
    };
    *count = sizeof(t) / sizeof(t[0]);
    return t;
  }
};
#undef DBG_SV
#undef DBG_SVP
#undef DBG_SVH
#undef DBG_SVB
#undef DBG_SVE
#undef DBG_SVD
#undef DBG_SVL

template <class K, bool V>
const SortVariant &chosen_variant(dbg_ctx *ctx) {
  int count = 0;
  const SortVariant *t = SortKind<K, V>::table(&count);
  int v = ctx->sort_variant[SortKind<K, V>::kind];
  if (v < 0 || v >= count) v = 0;
  return t[v];
}

template <class F>
inline void set_smem_attrs(F kern, size_t smem) {
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
}

// Ascending LSD radix sort of n keys (with optional u32 payloads) whose
// significant bits are the low `bits`.  `hist` holds the per-pass digit
// histograms (passes x 256), already accumulated by the producer kernel.
// Passes below first_pass are skipped: the keys are then sorted by their
// bits from 8 * first_pass - adj up (stably; for keys without payload, with
// the partition-first switch on, keys equal in those bits end in no
// particular order).  Pass p takes the 8 bits from 8 p - adj up: adj > 0
// aligns the top pass with the top of a key of 8 P - adj bits, so that the
// passes from first_pass up resolve whole bytes of it.  On return the data is in *keys / *vals (the buffers may have
// been swapped with *alt_keys / *alt_vals).
template <class K, bool HAS_VAL>
dbg_status radix_sort(dbg_ctx *ctx, K **keys, K **alt_keys, uint32_t **vals, uint32_t **alt_vals, uint64_t n,
                      int bits, const unsigned long long *d_hist, uint64_t *d_digit_base, int first_pass = 0,
                      int adj = 0) {
  if (n <= 1) return DBG_OK;
  const SortVariant &sv = chosen_variant<K, HAS_VAL>(ctx);
  const int passes = passes_for_bits(bits);
  const uint64_t tiles = (n + sv.tile - 1) / sv.tile;
  if (tiles > 0x7fffffffull) return DBG_EOVERFLOW;
  DBG_TRY(ensure_status(ctx, (size_t)tiles * RADIX));
  cudaStream_t s = ctx->stream;
  DBG_LAUNCH(ctx, HAS_VAL ? ST_SORT_NODES : ST_SORT_EDGES, 0.0,
             k_digit_base<<<passes, RADIX, 0, s>>>(d_hist, d_digit_base));
  int p = first_pass;
  if (!HAS_VAL && ctx->partition_first && p < passes) {
    // the first pass of keys without payload as a partition (no look-back)
    constexpr int tile = PART_BLOCK * PartShape<K>::ITEMS;
    constexpr size_t smem = sizeof(PartSmem<K>);
    set_smem_attrs(k_partition<K>, smem);
    const uint64_t tiles = (n + tile - 1) / tile;
    const unsigned grid = (unsigned)std::min<uint64_t>(tiles, 3ull * (uint64_t)ctx->num_sms);
    DBG_LAUNCH(ctx, ST_PARTITION_EDGES, 2.0 * (double)n * (double)sizeof(K),
               k_partition<K><<<grid, PART_BLOCK, smem, s>>>(
                   *keys, *alt_keys, n, p * RADIX_BITS - adj,
                   reinterpret_cast<unsigned long long *>(d_digit_base + p * RADIX), ctx->spin_limit, ctx->d_err));
    std::swap(*keys, *alt_keys);
    p++;
  }
  for (; p < passes; p++) {
    uint32_t epoch;
    DBG_TRY(next_epoch(ctx, &epoch));
    DBG_CUDA_TRY(cudaMemsetAsync(ctx->d_counters, 0, sizeof(uint32_t), s));
    DBG_LAUNCH(ctx, HAS_VAL ? ST_SORT_NODES : ST_SORT_EDGES,
               2.0 * (double)n * (double)(sizeof(K) + (HAS_VAL ? sizeof(uint32_t) : 0)),
               sv.launch(ctx, *keys, *alt_keys, HAS_VAL ? *vals : nullptr, HAS_VAL ? *alt_vals : nullptr, n,
                         p * RADIX_BITS - adj, d_digit_base + p * RADIX, epoch));
    std::swap(*keys, *alt_keys);
    if (HAS_VAL) std::swap(*vals, *alt_vals);
  }
  DBG_CUDA_TRY(cudaGetLastError());
  return DBG_OK;
}

// ---------------------------------------------------------------------------
// Hybrid sort: global onesweep passes over the high digits, then one local
// pass (k_seg_sort) that finishes each group-aligned tile in shared memory.
// ---------------------------------------------------------------------------
template <class K> struct SegShape;
template <> struct SegShape<uint64_t> {
  static constexpr int ITEMS = 24, TILE = 4096;  // capacity 6144: groups of up to 2048 keys
  static constexpr double MAX_MEAN = 128.0;
};
template <> struct SegShape<Key128> {
  static constexpr int ITEMS = 12, TILE = 2048;  // capacity 3072: groups of up to 1024 keys
  static constexpr double MAX_MEAN = 64.0;
};

// The first global pass of the hybrid sort of n keys of `bits` bits: the
// largest p >= 2 for which keys sharing their bits from 8p up form groups of
// at most MAX_MEAN keys on average (for uniform keys); 0 = no hybrid.
template <class K>
int hybrid_first_pass(uint64_t n, int bits) {
  const int P = passes_for_bits(bits);
  for (int p = P; p >= 2; p--) {
    const int hi = bits - RADIX_BITS * p;
    if (hi <= 0) {
      if (n <= (uint64_t)SegShape<K>::TILE) return p;  // one tile holds every key
      continue;
    }
    if ((double)n <= SegShape<K>::MAX_MEAN * std::ldexp(1.0, hi)) return p;
  }
  return 0;
}

// ranking method of the local sort, by variant number (kinds 4 and 5)
inline int local_rank_method(dbg_ctx *ctx, bool wide) {
  static const int methods[] = {RANK_MATCH, RANK_ATOMIC, RANK_BALLOT};
  const int v = ctx->sort_variant[wide ? 5 : 4];
  return methods[(v >= 0 && v < 6) ? v % 3 : 0];
}

inline unsigned grid_for(uint64_t n, int per_block) {
  uint64_t g = (n + per_block - 1) / per_block;
  return (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(g, 0x7fffffffull));
}

// Exclusive scan of n u32 values into n + 1 u64 (the last is the total).
inline dbg_status scan_u32(dbg_ctx *ctx, const uint32_t *in, uint64_t n, uint64_t *out, uint32_t *total, int stage) {
  cudaStream_t s = ctx->stream;
  const uint64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
  DBG_TRY(ensure_status(ctx, tiles));
  uint32_t epoch;
  DBG_TRY(next_epoch(ctx, &epoch));
  DBG_CUDA_TRY(cudaMemsetAsync(ctx->d_counters, 0, 2 * sizeof(uint32_t), s));
  DBG_LAUNCH(ctx, stage, 12.0 * n,
             k_scan_excl<<<(unsigned)tiles, SCAN_BLOCK, 0, s>>>(in, n, out, ctx->d_status, ctx->d_counters, epoch,
                                                                ctx->spin_limit, ctx->d_err, ctx->d_counters + 1));
  DBG_CUDA_TRY(cudaGetLastError());
  return read_small(ctx, ctx->d_counters + 1, sizeof(uint32_t), total);
}

// K4 by reduce-then-scan: unique keys into `uniq`, run heads into headpos
// (E + 1 entries, the last = n); returns E.
template <class K>
dbg_status run_length_reduce(dbg_ctx *ctx, const K *sorted, uint64_t n, K *uniq, uint32_t *headpos, uint64_t *E) {
  cudaStream_t s = ctx->stream;
  const uint64_t tiles = (n + RS_TILE - 1) / RS_TILE;
  DevBuf counts, toff;
  DBG_TRY(alloc_buf(ctx, counts, tiles * 4));
  DBG_TRY(alloc_buf(ctx, toff, (tiles + 1) * 8));
  DBG_LAUNCH(ctx, ST_RLE, (double)n * sizeof(K),
             k_count_heads<K><<<(unsigned)tiles, SCAN_BLOCK, 0, s>>>(sorted, nullptr, n, counts.as<uint32_t>(),
                                                                   nullptr));
  uint32_t total = 0;
  DBG_TRY(scan_u32(ctx, counts.as<uint32_t>(), tiles, toff.as<uint64_t>(), &total, ST_RLE));
  DBG_LAUNCH(ctx, ST_RLE, (double)n * sizeof(K) + (double)total * (sizeof(K) + 4),
             k_write_heads<K><<<(unsigned)tiles, SCAN_BLOCK, 0, s>>>(sorted, n, toff.as<uint64_t>(), uniq, headpos));
  DBG_CUDA_TRY(cudaGetLastError());
  *E = total;
  return DBG_OK;
}

// Tile bounds of the local pass over n keys sorted by their bits from
// low_bits up, and the oversize tiles (longer than the shared-memory
// capacity) gathered into *gk / *gv and sorted over every digit.  Returns the
// number of gathered keys in *G (0: none).
template <class K, bool HAS_VAL>
dbg_status seg_prepare(dbg_ctx *ctx, const K *kin, const uint32_t *vin, uint64_t n, int low_bits, int key_bits,
                       DevBuf &bound, DevBuf &osize, DevBuf &ooff, DevBuf &gk, DevBuf &gv, uint32_t *G, int stage) {
  using Sh = SegShape<K>;
  cudaStream_t s = ctx->stream;
  const uint64_t tiles = (n + Sh::TILE - 1) / Sh::TILE;
  if (tiles > 0x7fffffffull) return DBG_EOVERFLOW;
  DBG_TRY(alloc_buf(ctx, bound, (tiles + 1) * 8));
  DBG_TRY(alloc_buf(ctx, osize, tiles * 4));
  DBG_TRY(alloc_buf(ctx, ooff, (tiles + 1) * 8));
  DBG_LAUNCH(ctx, stage, 0.0,
             k_seg_bounds<K><<<grid_for(tiles + 1, 256), 256, 0, s>>>(kin, n, low_bits, Sh::TILE, tiles,
                                                                     bound.as<uint64_t>()));
  DBG_LAUNCH(ctx, stage, 0.0,
             k_seg_oversize<<<grid_for(tiles, 256), 256, 0, s>>>(bound.as<uint64_t>(), tiles,
                                                                 (uint32_t)(SEG_BLOCK * Sh::ITEMS),
                                                                 osize.as<uint32_t>()));
  DBG_TRY(scan_u32(ctx, osize.as<uint32_t>(), tiles, ooff.as<uint64_t>(), G, stage));
  if (*G == 0) return DBG_OK;
  // the oversize tiles, gathered in order and sorted over every digit
  const uint64_t g = *G;
  DevBuf galt, gvalt, small;
  DBG_TRY(alloc_buf(ctx, gk, g * sizeof(K)));
  DBG_TRY(alloc_buf(ctx, galt, g * sizeof(K)));
  if (HAS_VAL) {
    DBG_TRY(alloc_buf(ctx, gv, g * 4));
    DBG_TRY(alloc_buf(ctx, gvalt, g * 4));
  }
  DBG_TRY(alloc_buf(ctx, small, MAX_PASSES * RADIX * 16));
  unsigned long long *hist = small.as<unsigned long long>();
  uint64_t *dbase = reinterpret_cast<uint64_t *>(hist + MAX_PASSES * RADIX);
  const int passes = passes_for_bits(key_bits);
  DBG_LAUNCH(ctx, stage, 2.0 * g * (sizeof(K) + (HAS_VAL ? 4 : 0)),
             k_seg_gather<K, HAS_VAL><<<(unsigned)std::min<uint64_t>(tiles, 152ull * 8), 256, 0, s>>>(
                 kin, vin, bound.as<uint64_t>(), osize.as<uint32_t>(), ooff.as<uint64_t>(), tiles, gk.as<K>(),
                 HAS_VAL ? gv.as<uint32_t>() : nullptr));
  DBG_CUDA_TRY(cudaMemsetAsync(hist, 0, MAX_PASSES * RADIX * 8, s));
  DBG_LAUNCH(ctx, stage, (double)g * sizeof(K),
             k_digit_hist<K><<<std::min(grid_for(g, 256 * 16), 152u * 8), 256, 0, s>>>(gk.as<K>(), g, 0, passes,
                                                                                       hist));
  K *kp = gk.as<K>(), *ka = galt.as<K>();
  uint32_t *vp = HAS_VAL ? gv.as<uint32_t>() : nullptr, *va = HAS_VAL ? gvalt.as<uint32_t>() : nullptr;
  DBG_TRY((radix_sort<K, HAS_VAL>(ctx, &kp, &ka, &vp, &va, g, key_bits, hist, dbase)));
  if (kp != gk.as<K>()) std::swap(gk, galt);
  if (HAS_VAL && vp != gv.as<uint32_t>()) std::swap(gv, gvalt);
  ctx->local_sort_fallbacks++;
  return DBG_OK;
}

// The local pass over node records sorted by their bits from low_bits up:
// k_seg_sort writes the fully sorted records to kout / vout.
template <class K>
dbg_status seg_sort_records(dbg_ctx *ctx, const K *kin, const uint32_t *vin, K *kout, uint32_t *vout, uint64_t n,
                            int low_bits, int key_bits) {
  using Sh = SegShape<K>;
  DevBuf bound, osize, ooff, gk, gv;
  uint32_t G = 0;
  DBG_TRY((seg_prepare<K, true>(ctx, kin, vin, n, low_bits, key_bits, bound, osize, ooff, gk, gv, &G,
                                ST_LOCAL_SORT_NODES)));
  const int rank = local_rank_method(ctx, sizeof(K) == 16);
  const uint64_t tiles = (n + Sh::TILE - 1) / Sh::TILE;
  {
    if (ctx->seg_rank && (sizeof(K) == 16 || low_bits + 13 <= 64)) {
      // ranking within groups; tiles with a long group are listed and
      // sorted by the digit passes
      static_assert(SegRankSmem<K>::CAP == SEG_BLOCK * Sh::ITEMS, "same tile capacity as the digit-pass kernel");
      set_smem_attrs(k_seg_rank<K>, sizeof(SegRankSmem<K>));
      DevBuf fb;
      DBG_TRY(alloc_buf(ctx, fb, (tiles + 1) * 4));
      uint32_t *fb_count = fb.as<uint32_t>(), *fb_list = fb_count + 1;
      DBG_CUDA_TRY(cudaMemsetAsync(fb_count, 0, 4, ctx->stream));
      DBG_LAUNCH(ctx, ST_LOCAL_SORT_NODES, 2.0 * (double)n * (sizeof(K) + 4),
                 k_seg_rank<K><<<(unsigned)tiles, RANK_BLOCK, sizeof(SegRankSmem<K>), ctx->stream>>>(
                     kin, vin, bound.as<uint64_t>(), osize.as<uint32_t>(), ooff.as<uint64_t>(), gk.as<K>(),
                     gv.as<uint32_t>(), kout, vout, low_bits, fb_list, fb_count));
      DBG_CUDA_TRY(cudaGetLastError());
      uint32_t nfb = 0;
      DBG_TRY(read_small(ctx, fb_count, sizeof(uint32_t), &nfb));
      ctx->rank_fallback_tiles += nfb;
      if (nfb == 0) return DBG_OK;
      auto kern = rank == RANK_MATCH    ? k_seg_sort<K, Sh::ITEMS, RANK_MATCH>
                  : rank == RANK_ATOMIC ? k_seg_sort<K, Sh::ITEMS, RANK_ATOMIC>
                                        : k_seg_sort<K, Sh::ITEMS, RANK_BALLOT>;
      constexpr size_t smem = sizeof(SegSortSmem<K, true, Sh::ITEMS>);
      set_smem_attrs(kern, smem);
      const unsigned grid = (unsigned)std::min<uint64_t>(nfb, 2ull * (uint64_t)std::max(1, ctx->num_sms));
      DBG_LAUNCH(ctx, ST_LOCAL_SORT_NODES, 0.0,
                 kern<<<grid, SEG_BLOCK, smem, ctx->stream>>>(
                     kin, vin, bound.as<uint64_t>(), osize.as<uint32_t>(), ooff.as<uint64_t>(), gk.as<K>(),
                     gv.as<uint32_t>(), kout, vout, low_bits, key_bits, fb_list, fb_count));
      DBG_CUDA_TRY(cudaGetLastError());
      return DBG_OK;
    }
  }
  const int v = ctx->sort_variant[sizeof(K) == 16 ? 5 : 4];
  if (v >= 3) {
    // the wide form: 384 threads x (2/3 of the items), the same capacity
    constexpr int WB = 384, WI = Sh::ITEMS * SEG_BLOCK / WB;
    static_assert(WB * WI == SEG_BLOCK * Sh::ITEMS, "same tile capacity");
    auto kern = rank == RANK_MATCH    ? k_seg_sort<K, WI, RANK_MATCH, WB>
                : rank == RANK_ATOMIC ? k_seg_sort<K, WI, RANK_ATOMIC, WB>
                                      : k_seg_sort<K, WI, RANK_BALLOT, WB>;
    constexpr size_t smem = sizeof(SegSortSmem<K, true, WI, WB>);
    set_smem_attrs(kern, smem);
    DBG_LAUNCH(ctx, ST_LOCAL_SORT_NODES, 2.0 * (double)n * (sizeof(K) + 4),
               kern<<<(unsigned)tiles, WB, smem, ctx->stream>>>(
                   kin, vin, bound.as<uint64_t>(), osize.as<uint32_t>(), ooff.as<uint64_t>(), gk.as<K>(),
                   gv.as<uint32_t>(), kout, vout, low_bits, key_bits, nullptr, nullptr));
    DBG_CUDA_TRY(cudaGetLastError());
    return DBG_OK;
  }
  auto kern = rank == RANK_MATCH    ? k_seg_sort<K, Sh::ITEMS, RANK_MATCH>
              : rank == RANK_ATOMIC ? k_seg_sort<K, Sh::ITEMS, RANK_ATOMIC>
                                    : k_seg_sort<K, Sh::ITEMS, RANK_BALLOT>;
  constexpr size_t smem = sizeof(SegSortSmem<K, true, Sh::ITEMS>);
  set_smem_attrs(kern, smem);
  DBG_LAUNCH(ctx, ST_LOCAL_SORT_NODES, 2.0 * (double)n * (sizeof(K) + 4),
             kern<<<(unsigned)tiles, SEG_BLOCK, smem, ctx->stream>>>(
                 kin, vin, bound.as<uint64_t>(), osize.as<uint32_t>(), ooff.as<uint64_t>(), gk.as<K>(),
                 gv.as<uint32_t>(), kout, vout, low_bits, key_bits, nullptr, nullptr));
  DBG_CUDA_TRY(cudaGetLastError());
  return DBG_OK;
}

// The local pass of STEP-2 over n edge keys sorted by their bits from
// low_bits up.  Leaves the E distinct keys in kin[0, E) and their
// multiplicities in mult_out (allocated here); kstage (n keys) is scratch.
template <class K>
dbg_status seg_rle(dbg_ctx *ctx, K *kin, K *kstage, uint64_t n, int low_bits, int key_bits, DevBuf &mult_out,
                   uint64_t *E) {
  using Sh = SegShape<K>;
  cudaStream_t s = ctx->stream;
  DevBuf bound, osize, ooff, gk, gv, gheads, guniq;
  uint32_t G = 0;
  DBG_TRY((seg_prepare<K, false>(ctx, kin, nullptr, n, low_bits, key_bits, bound, osize, ooff, gk, gv, &G,
                                 ST_LOCAL_SORT_EDGES)));
  uint64_t H = 0;
  if (G > 0) {
    DBG_TRY(alloc_buf(ctx, guniq, (uint64_t)G * sizeof(K)));
    DBG_TRY(alloc_buf(ctx, gheads, ((uint64_t)G + 1) * 4));
    DBG_TRY(run_length_reduce<K>(ctx, gk.as<K>(), G, guniq.as<K>(), gheads.as<uint32_t>(), &H));
  }
  const uint64_t tiles = (n + Sh::TILE - 1) / Sh::TILE;
  DevBuf mstage, tcount, toff;
  DBG_TRY(alloc_buf(ctx, mstage, n * 4));
  DBG_TRY(alloc_buf(ctx, tcount, tiles * 4));
  DBG_TRY(alloc_buf(ctx, toff, (tiles + 1) * 8));
  const int rank = local_rank_method(ctx, sizeof(K) == 16);
  auto radix = rank == RANK_MATCH    ? k_seg_rle<K, Sh::ITEMS, RANK_MATCH>
               : rank == RANK_ATOMIC ? k_seg_rle<K, Sh::ITEMS, RANK_ATOMIC>
                                     : k_seg_rle<K, Sh::ITEMS, RANK_BALLOT>;
  constexpr size_t rsmem = sizeof(SegSortSmem<K, false, Sh::ITEMS>);
  set_smem_attrs(radix, rsmem);
  bool counted = false;
  {
    if (ctx->count_first) {
      // count-first; the tiles that overflow their table are listed (after
      // a counter word) and sorted copy by copy
      auto count = rank == RANK_MATCH    ? k_seg_count<K, RANK_MATCH>
                   : rank == RANK_ATOMIC ? k_seg_count<K, RANK_ATOMIC>
                                         : k_seg_count<K, RANK_BALLOT>;
      const size_t csmem = rank == RANK_MATCH    ? sizeof(SegCountSmem<K, RANK_MATCH>)
                           : rank == RANK_ATOMIC ? sizeof(SegCountSmem<K, RANK_ATOMIC>)
                                                 : sizeof(SegCountSmem<K, RANK_BALLOT>);
      set_smem_attrs(count, csmem);
      DevBuf over;
      DBG_TRY(alloc_buf(ctx, over, (tiles + 2) * 4));
      uint32_t *over_count = over.as<uint32_t>(), *rank_fb = over_count + 1, *over_list = over_count + 2;
      DBG_CUDA_TRY(cudaMemsetAsync(over_count, 0, 8, s));
      DBG_LAUNCH(ctx, ST_LOCAL_SORT_EDGES, (double)n * sizeof(K),
                 count<<<(unsigned)tiles, SEG_BLOCK, csmem, s>>>(
                     kin, bound.as<uint64_t>(), osize.as<uint32_t>(), ooff.as<uint64_t>(), guniq.as<K>(),
                     gheads.as<uint32_t>(), (uint32_t)H, kstage, mstage.as<uint32_t>(), tcount.as<uint32_t>(),
                     over_list, over_count, low_bits, key_bits, ctx->seg_rank, rank_fb));
      DBG_CUDA_TRY(cudaGetLastError());
      uint32_t nover_fb[2] = {0, 0};
      DBG_TRY(read_small(ctx, over_count, 2 * sizeof(uint32_t), nover_fb));
      const uint32_t nover = nover_fb[0];
      ctx->count_overflow_tiles += nover;
      ctx->rank_fallback_tiles += nover_fb[1];
      if (nover > 0)
        DBG_LAUNCH(ctx, ST_LOCAL_SORT_EDGES, 0.0,
                   radix<<<nover, SEG_BLOCK, rsmem, s>>>(
                       kin, bound.as<uint64_t>(), osize.as<uint32_t>(), ooff.as<uint64_t>(), guniq.as<K>(),
                       gheads.as<uint32_t>(), (uint32_t)H, kstage, mstage.as<uint32_t>(), tcount.as<uint32_t>(),
                       low_bits, key_bits, over_list));
      counted = true;
    }
  }
  if (!counted)
    DBG_LAUNCH(ctx, ST_LOCAL_SORT_EDGES, (double)n * sizeof(K),
               radix<<<(unsigned)tiles, SEG_BLOCK, rsmem, s>>>(
                   kin, bound.as<uint64_t>(), osize.as<uint32_t>(), ooff.as<uint64_t>(), guniq.as<K>(),
                   gheads.as<uint32_t>(), (uint32_t)H, kstage, mstage.as<uint32_t>(), tcount.as<uint32_t>(),
                   low_bits, key_bits, nullptr));
  DBG_CUDA_TRY(cudaGetLastError());
  uint32_t total = 0;
  DBG_TRY(scan_u32(ctx, tcount.as<uint32_t>(), tiles, toff.as<uint64_t>(), &total, ST_LOCAL_SORT_EDGES));
  *E = total;
  DBG_TRY(alloc_buf(ctx, mult_out, std::max<uint64_t>(1, total) * 4));
  DBG_LAUNCH(ctx, ST_LOCAL_SORT_EDGES, 2.0 * total * (sizeof(K) + 4),
             k_seg_compact<K><<<(unsigned)std::min<uint64_t>(tiles, 152ull * 16), 256, 0, s>>>(
                 bound.as<uint64_t>(), tcount.as<uint32_t>(), toff.as<uint64_t>(), tiles, kstage,
                 mstage.as<uint32_t>(), kin, mult_out.as<uint32_t>()));
  DBG_CUDA_TRY(cudaGetLastError());
  return DBG_OK;
}

// STEP-3's stable sort of R node records: hybrid (global passes from q0
// up, then the local pass) when q0 > 0, else every digit globally.  The
// producers accumulated the histograms of passes q0 and up only (with the
// digit alignment adj, which needs q0 > 0).
template <class K>
dbg_status sort_records(dbg_ctx *ctx, K **rk, K **rk_alt, uint32_t **rv, uint32_t **rv_alt, uint64_t R, int nbits,
                        int q0, unsigned long long *d_hist, uint64_t *d_digit_base, int adj = 0) {
  if (q0 > 0 && R > 1) {
    DBG_TRY((radix_sort<K, true>(ctx, rk, rk_alt, rv, rv_alt, R, nbits, d_hist, d_digit_base, q0, adj)));
    DBG_TRY(seg_sort_records<K>(ctx, *rk, *rv, *rk_alt, *rv_alt, R, RADIX_BITS * q0 - adj, nbits));
    std::swap(*rk, *rk_alt);
    std::swap(*rv, *rv_alt);
    return DBG_OK;
  }
  return radix_sort<K, true>(ctx, rk, rk_alt, rv, rv_alt, R, nbits, d_hist, d_digit_base);
}

// K6 by reduce-then-scan over R sorted node records; returns the node count
// and the number of edge ends.  E_all > 0: the records hold both ends of
// all E_all edges, and src / dst are written through the partition of the
// edge ends by edge range (k_scatter_ends) instead of at random.  adj_side
// (E_all > 0 only): the payloads carry the side bits, stored per slot.
template <class K>
dbg_status assign_node_ids(dbg_ctx *ctx, const K *rk, const uint32_t *rv, uint64_t R, K *node_keys,
                           uint64_t *row_ptr, dbg_graph *g, uint32_t base_v, uint64_t base_slot, uint64_t *V,
                           uint64_t *ends, uint64_t E_all = 0, uint8_t *adj_side = nullptr) {
  cudaStream_t s = ctx->stream;
  const uint64_t tiles = (R + RS_TILE - 1) / RS_TILE;
  DevBuf hc, ec, ho, eo;
  DBG_TRY(alloc_buf(ctx, hc, tiles * 4));
  DBG_TRY(alloc_buf(ctx, ec, tiles * 4));
  DBG_TRY(alloc_buf(ctx, ho, (tiles + 1) * 8));
  DBG_TRY(alloc_buf(ctx, eo, (tiles + 1) * 8));
  DBG_LAUNCH(ctx, ST_NODE_IDS, (double)R * (sizeof(K) + 4),
             k_count_heads<K><<<(unsigned)tiles, SCAN_BLOCK, 0, s>>>(rk, rv, R, hc.as<uint32_t>(), ec.as<uint32_t>()));
  uint32_t nv = 0, ne = 0;
  DBG_TRY(scan_u32(ctx, hc.as<uint32_t>(), tiles, ho.as<uint64_t>(), &nv, ST_NODE_IDS));
  DBG_TRY(scan_u32(ctx, ec.as<uint32_t>(), tiles, eo.as<uint64_t>(), &ne, ST_NODE_IDS));
  if (E_all > 0) {
    int bshift = 10;
    while ((E_all + (1ull << bshift) - 1) >> bshift > 256) bshift++;
    DevBuf part, fill;
    DBG_TRY(alloc_buf(ctx, part, 2 * E_all * 8));
    DBG_TRY(alloc_buf(ctx, fill, 256 * 4));
    DBG_CUDA_TRY(cudaMemsetAsync(fill.p, 0, 256 * 4, s));
    const double wbytes = (double)R * (sizeof(K) + 4) + (double)nv * (sizeof(K) + 8) + (double)ne * (adj_side ? 14 : 13);
    if constexpr (sizeof(K) == 8) {
      // persistent CTAs, two per SM, with the next tile's records in flight
      constexpr size_t smem = sizeof(WriteNodesSmem<K>);
      set_smem_attrs(k_write_nodes_p<K, true>, smem);
      const unsigned grid = (unsigned)std::min<uint64_t>(tiles, 2ull * (uint64_t)ctx->num_sms);
      DBG_LAUNCH(ctx, ST_NODE_IDS, wbytes,
                 k_write_nodes_p<K, true><<<grid, SCAN_BLOCK, smem, s>>>(
                     rk, rv, R, ho.as<uint64_t>(), eo.as<uint64_t>(), node_keys, row_ptr, g->src.as<uint32_t>(),
                     g->dst.as<uint32_t>(), g->adj_edge.as<uint32_t>(), g->adj_role.as<uint8_t>(), base_v,
                     base_slot, part.as<uint64_t>(), fill.as<uint32_t>(), bshift, ctx->spin_limit, ctx->d_err,
                     adj_side));
    } else {
      DBG_LAUNCH(ctx, ST_NODE_IDS, wbytes,
                 k_write_nodes<K, true><<<(unsigned)tiles, SCAN_BLOCK, 0, s>>>(
                     rk, rv, R, ho.as<uint64_t>(), eo.as<uint64_t>(), node_keys, row_ptr, g->src.as<uint32_t>(),
                     g->dst.as<uint32_t>(), g->adj_edge.as<uint32_t>(), g->adj_role.as<uint8_t>(), base_v,
                     base_slot, part.as<uint64_t>(), fill.as<uint32_t>(), bshift, adj_side));
    }
    DBG_LAUNCH(ctx, ST_NODE_IDS, 2.0 * E_all * (8 + 4),
               k_scatter_ends<<<grid_for(2 * E_all, 256 * 16), 256, 0, s>>>(part.as<uint64_t>(), 2 * E_all,
                                                                          g->src.as<uint32_t>(),
                                                                          g->dst.as<uint32_t>()));
  } else {
    DBG_LAUNCH(ctx, ST_NODE_IDS, (double)R * (sizeof(K) + 4) + (double)nv * (sizeof(K) + 8) + (double)ne * 9,
               k_write_nodes<K, false><<<(unsigned)tiles, SCAN_BLOCK, 0, s>>>(
                   rk, rv, R, ho.as<uint64_t>(), eo.as<uint64_t>(), node_keys, row_ptr, g->src.as<uint32_t>(),
                   g->dst.as<uint32_t>(), g->adj_edge.as<uint32_t>(), g->adj_role.as<uint8_t>(), base_v, base_slot,
                   nullptr, nullptr, 0));
  }
  DBG_CUDA_TRY(cudaGetLastError());
  *V = nv;
  *ends = ne;
  return DBG_OK;
}

// Node multiplicities: the k-mers of the reads (each read of length L >= k
// holds L - k + 1), emitted, sorted and counted like STEP-2's edge keys.  The
// distinct canonical k-mers of the reads of length >= k are exactly the
// nodes, in the same ascending order, so counts[i] belongs to node i; *Vk =
// their number, which the caller checks against |V|.
template <class K>
dbg_status count_node_kmers(dbg_ctx *ctx, const DevBuf &packed, const DevBuf &base_off, const uint32_t *d_lengths,
                            uint64_t n, uint64_t N, uint32_t k, unsigned long long *d_hist,
                            uint64_t *d_digit_base, DevBuf &counts, uint64_t *Vk) {
  cudaStream_t s = ctx->stream;
  *Vk = 0;
  if (n == 0) return DBG_OK;
  // the k-mers number at most N + n (N edge instances, one more k-mer per
  // read); the offsets' scan keeps 32-bit totals
  if (N + n > 0xffffffffull) {
    set_error("%llu edge instances and %llu reads: too many k-mers to count in one build",
              (unsigned long long)N, (unsigned long long)n);
    return DBG_EOVERFLOW;
  }
  DevBuf per, koff;
  DBG_TRY(alloc_buf(ctx, per, n * sizeof(uint32_t)));
  DBG_TRY(alloc_buf(ctx, koff, (n + 1) * sizeof(uint64_t)));
  DBG_LAUNCH(ctx, ST_NODE_MULT, 8.0 * n,
             k_kmer_counts<<<grid_for(n, 256), 256, 0, s>>>(d_lengths, n, k, per.as<uint32_t>()));
  uint32_t low32 = 0;
  DBG_TRY(scan_u32(ctx, per.as<uint32_t>(), n, koff.as<uint64_t>(), &low32, ST_NODE_MULT));
  uint64_t M = 0;
  DBG_TRY(read_small(ctx, koff.as<uint64_t>() + n, sizeof(uint64_t), &M));
  if (M == 0) return DBG_OK;
  const int kbits = 2 * (int)k;
  const int passes = passes_for_bits(kbits);
  const int p0 = ctx->hybrid_sort ? hybrid_first_pass<K>(M, kbits) : 0;
  DevBuf ka, kb, headpos;
  DBG_TRY(alloc_buf(ctx, ka, M * sizeof(K)));
  DBG_TRY(alloc_buf(ctx, kb, M * sizeof(K)));
  DBG_CUDA_TRY(cudaMemsetAsync(d_hist, 0, MAX_PASSES * RADIX * sizeof(unsigned long long), s));
  // emitting with k - 1 gives windows of k bases at the k-mer offsets
  DBG_LAUNCH(ctx, ST_NODE_MULT, 8.0 * n + (double)M * sizeof(K),
             k_emit<K><<<(unsigned)std::min<uint64_t>(grid_for(n, EMIT_BLOCK / 32), 152ull * 64), EMIT_BLOCK, 0, s>>>(
                 packed.as<uint64_t>(), base_off.as<uint64_t>(), koff.as<uint64_t>(), n, k - 1, ka.as<K>(), p0,
                 passes, d_hist, nullptr));
  DBG_CUDA_TRY(cudaGetLastError());
  K *kp = ka.as<K>(), *alt = kb.as<K>();
  uint32_t *vn = nullptr, *van = nullptr;
  uint64_t D = 0;
  if (p0 > 0) {
    DBG_TRY((radix_sort<K, false>(ctx, &kp, &alt, &vn, &van, M, kbits, d_hist, d_digit_base, p0)));
    DBG_TRY(seg_rle<K>(ctx, kp, alt, M, RADIX_BITS * p0, kbits, counts, &D));
  } else {
    DBG_TRY(alloc_buf(ctx, headpos, (M + 1) * sizeof(uint32_t)));
    DBG_TRY((radix_sort<K, false>(ctx, &kp, &alt, &vn, &van, M, kbits, d_hist, d_digit_base)));
    DBG_TRY(run_length_reduce<K>(ctx, kp, M, alt, headpos.as<uint32_t>(), &D));
    DBG_TRY(alloc_buf(ctx, counts, std::max<uint64_t>(1, D) * sizeof(uint32_t)));
    DBG_LAUNCH(ctx, ST_NODE_MULT, 8.0 * D,
               k_counts_from_heads<<<grid_for(D, 256), 256, 0, s>>>(headpos.as<uint32_t>(), D,
                                                                   counts.as<uint32_t>()));
  }
  DBG_CUDA_TRY(cudaGetLastError());
  DBG_TRY(check_device_error(ctx));
  *Vk = D;
  return DBG_OK;
}

// Distinct reads per node (the roadmap counts): every k-mer of the reads
// with its read index, stably sorted by key (the records of one key keep
// their read order, which is ascending), then per key the number of records
// that start its run or follow a record of another read.  As for the
// multiplicities, the distinct keys are exactly the nodes, in node order.
template <class K>
dbg_status count_node_reads(dbg_ctx *ctx, const DevBuf &packed, const DevBuf &base_off, const uint32_t *d_lengths,
                            uint64_t n, uint64_t N, uint32_t k, unsigned long long *d_hist,
                            uint64_t *d_digit_base, DevBuf &counts, uint64_t *Vk) {
  cudaStream_t s = ctx->stream;
  *Vk = 0;
  if (n == 0) return DBG_OK;
  if (N + n > 0xffffffffull) {
    set_error("%llu edge instances and %llu reads: too many k-mers to count in one build",
              (unsigned long long)N, (unsigned long long)n);
    return DBG_EOVERFLOW;
  }
  DevBuf per, koff;
  DBG_TRY(alloc_buf(ctx, per, n * sizeof(uint32_t)));
  DBG_TRY(alloc_buf(ctx, koff, (n + 1) * sizeof(uint64_t)));
  DBG_LAUNCH(ctx, ST_NODE_MULT, 8.0 * n,
             k_kmer_counts<<<grid_for(n, 256), 256, 0, s>>>(d_lengths, n, k, per.as<uint32_t>()));
  uint32_t low32 = 0;
  DBG_TRY(scan_u32(ctx, per.as<uint32_t>(), n, koff.as<uint64_t>(), &low32, ST_NODE_MULT));
  uint64_t M = 0;
  DBG_TRY(read_small(ctx, koff.as<uint64_t>() + n, sizeof(uint64_t), &M));
  if (M == 0) return DBG_OK;
  per.release();
  const int kbits = 2 * (int)k;
  const int q0 = ctx->hybrid_sort ? hybrid_first_pass<K>(M, kbits) : 0;
  DevBuf ka, kb, va, vb;
  DBG_TRY(alloc_buf(ctx, ka, M * sizeof(K)));
  DBG_TRY(alloc_buf(ctx, kb, M * sizeof(K)));
  DBG_TRY(alloc_buf(ctx, va, M * sizeof(uint32_t)));
  DBG_TRY(alloc_buf(ctx, vb, M * sizeof(uint32_t)));
  DBG_CUDA_TRY(cudaMemsetAsync(d_hist, 0, MAX_PASSES * RADIX * sizeof(unsigned long long), s));
  // windows of k bases at the k-mer offsets, each with its read index
  DBG_LAUNCH(ctx, ST_NODE_MULT, 8.0 * n + (double)M * (sizeof(K) + 4),
             k_emit<K><<<(unsigned)std::min<uint64_t>(grid_for(n, EMIT_BLOCK / 32), 152ull * 64), EMIT_BLOCK, 0, s>>>(
                 packed.as<uint64_t>(), base_off.as<uint64_t>(), koff.as<uint64_t>(), n, k - 1, ka.as<K>(), q0,
                 passes_for_bits(kbits), d_hist, nullptr, va.as<uint32_t>()));
  DBG_CUDA_TRY(cudaGetLastError());
  koff.release();
  K *kp = ka.as<K>(), *kalt = kb.as<K>();
  uint32_t *vp = va.as<uint32_t>(), *valt = vb.as<uint32_t>();
  DBG_TRY((sort_records<K>(ctx, &kp, &kalt, &vp, &valt, M, kbits, q0, d_hist, d_digit_base)));
  // flags into the free payload buffer, their scan, the key runs
  DBG_LAUNCH(ctx, ST_NODE_MULT, (double)M * (2 * sizeof(K) + 12),
             k_read_change_flags<K><<<grid_for(M, 256 * 8), 256, 0, s>>>(kp, vp, M, valt));
  DevBuf F, headpos;
  DBG_TRY(alloc_buf(ctx, F, (M + 1) * sizeof(uint64_t)));
  uint32_t low = 0;
  DBG_TRY(scan_u32(ctx, valt, M, F.as<uint64_t>(), &low, ST_NODE_MULT));
  DBG_TRY(alloc_buf(ctx, headpos, (M + 1) * sizeof(uint32_t)));
  uint64_t D = 0;
  DBG_TRY(run_length_reduce<K>(ctx, kp, M, kalt, headpos.as<uint32_t>(), &D));
  DBG_TRY(alloc_buf(ctx, counts, std::max<uint64_t>(1, D) * sizeof(uint32_t)));
  DBG_LAUNCH(ctx, ST_NODE_MULT, 12.0 * D,
             k_counts_between<<<grid_for(D, 256), 256, 0, s>>>(headpos.as<uint32_t>(), F.as<uint64_t>(), D,
                                                               counts.as<uint32_t>()));
  DBG_CUDA_TRY(cudaGetLastError());
  DBG_TRY(check_device_error(ctx));
  *Vk = D;
  return DBG_OK;
}

template <class K>
dbg_status build_graph_impl(dbg_ctx *ctx, const BuildInput &in, dbg_graph *g) {
  cudaStream_t s = ctx->stream;
  const uint32_t k = in.k;
  const uint64_t n = in.n;
  g->k = k;
  g->key_words = sizeof(K) / 8;

  // ---- per-read offsets (exclusive scans of L and max(0, L - k)) ----
  DevBuf base_off, edge_off, tile_sums, small;
  const uint64_t off_tiles = (n + OFF_TILE - 1) / OFF_TILE;
  DBG_TRY(alloc_buf(ctx, base_off, (n + 1) * sizeof(uint64_t)));
  DBG_TRY(alloc_buf(ctx, edge_off, (n + 1) * sizeof(uint64_t)));
  DBG_TRY(alloc_buf(ctx, tile_sums, std::max<uint64_t>(1, off_tiles) * sizeof(Sum3)));
  DBG_TRY(alloc_buf(ctx, small, 64 * sizeof(uint64_t) + (MAX_PASSES * RADIX) * 16));
  uint64_t *d_totals = small.as<uint64_t>();
  unsigned long long *d_hist = reinterpret_cast<unsigned long long *>(d_totals + 64);
  uint64_t *d_digit_base = reinterpret_cast<uint64_t *>(d_hist + MAX_PASSES * RADIX);
  if (n > 0) {
    DBG_LAUNCH(ctx, ST_OFFSETS, 4.0 * n,
               k_read_tile_sums<<<(unsigned)off_tiles, OFF_BLOCK, 0, s>>>(in.d_lengths, n, k, tile_sums.as<Sum3>()));
  }
  {
    DBG_LAUNCH(ctx, ST_OFFSETS, 0.0,
               k_scan_tile_sums<<<1, 1024, 0, s>>>(tile_sums.as<Sum3>(), (uint32_t)off_tiles, d_totals,
                                      base_off.as<uint64_t>(), edge_off.as<uint64_t>(), n));
  }
  if (n > 0) {
    DBG_LAUNCH(ctx, ST_OFFSETS, 20.0 * n,
               k_read_offsets<<<(unsigned)off_tiles, OFF_BLOCK, 0, s>>>(in.d_lengths, n, k, tile_sums.as<Sum3>(),
                                                             base_off.as<uint64_t>(), edge_off.as<uint64_t>()));
  }
  DBG_CUDA_TRY(cudaGetLastError());
  uint64_t totals[3];
  DBG_TRY(read_small(ctx, d_totals, sizeof(totals), totals));
  const uint64_t total_bases = totals[0], N = totals[1], I = totals[2];
  tile_sums.release();
  g->num_instances = N;
  if (N > 0xffffffffull) {
    set_error("%llu edge instances exceed one in-memory build (2^32 - 1)", (unsigned long long)N);
    return DBG_EOVERFLOW;
  }

  // ---- K2 set-up: key buffers and histograms come first, so that host
  // reads can be emitted chunk by chunk as they are packed ----
  const int kbits = 2 * ((int)k + 1);
  const int kpasses = passes_for_bits(kbits);
  DevBuf keys_a, keys_b, headpos, mult_tmp, uniq;
  uint64_t E = 0;
  K *sorted = nullptr;
  // the hybrid sort needs the histograms of its global passes only
  const int p0 = ctx->hybrid_sort ? hybrid_first_pass<K>(N, kbits) : 0;
  if (N > 0) {
    DBG_TRY(alloc_buf(ctx, keys_a, N * sizeof(K)));
    DBG_TRY(alloc_buf(ctx, keys_b, N * sizeof(K)));
    DBG_CUDA_TRY(cudaMemsetAsync(d_hist, 0, MAX_PASSES * RADIX * sizeof(unsigned long long), s));
  }
  DevBuf packed;
  const uint64_t nwords = (total_bases + 31) / 32;
  // K2 emit over the keys [krange[0], krange[1]) (all of them: nullptr)
  auto emit = [&](const uint64_t *krange, double bytes) -> dbg_status {
    DBG_LAUNCH(ctx, ST_EMIT, bytes,
               k_emit<K><<<(unsigned)std::min<uint64_t>(grid_for(n, EMIT_BLOCK / 32), 152ull * 64), EMIT_BLOCK, 0,
                           s>>>(packed.as<uint64_t>(), base_off.as<uint64_t>(), edge_off.as<uint64_t>(), n, k,
                                keys_a.as<K>(), p0, kpasses, d_hist, krange));
    DBG_CUDA_TRY(cudaGetLastError());
    return DBG_OK;
  };

  // ---- K1 pack (+ K2 emit) ----
  DBG_TRY(alloc_buf(ctx, packed, (nwords + 3) * sizeof(uint64_t)));
  DBG_CUDA_TRY(cudaMemsetAsync(packed.as<uint64_t>() + nwords, 0, 3 * sizeof(uint64_t), s));
  bool emitted = false;
  if (nwords > 0 && !in.h_reads) {
    DBG_LAUNCH(ctx, ST_PACK, (double)total_bases + 8.0 * nwords,
               k_pack<<<grid_for(nwords, 256), 256, 0, s>>>(in.reads, total_bases, packed.as<uint64_t>(), nwords,
                                                 ctx->d_err));
  } else if (nwords > 0) {
    // host reads: chunks are copied on a stream of their own into two
    // staging buffers in turn while the build's stream packs the previous
    // chunk and emits the reads that end in the chunks packed so far
    const uint64_t chunk = 256ull << 20;  // bases per copy (a multiple of 32)
    const uint32_t chunks = (uint32_t)((total_bases + chunk - 1) / chunk);
    DBG_TRY(ensure_copy_stream(ctx));
    cudaStream_t cs = ctx->copy_stream;
    DevBuf stage[2], kbound;
    const uint64_t slen = std::min(chunk, total_bases);
    DBG_TRY(alloc_buf(ctx, stage[0], slen));
    if (chunks > 1) DBG_TRY(alloc_buf(ctx, stage[1], slen));
    DBG_TRY(alloc_buf(ctx, kbound, (chunks + 1) * sizeof(uint64_t)));
    if (N > 0)
      DBG_LAUNCH(ctx, ST_EMIT, 0.0,
                 k_chunk_key_bounds<<<grid_for(chunks + 1, 64), 64, 0, s>>>(
                     base_off.as<uint64_t>(), edge_off.as<uint64_t>(), n, chunk, chunks, kbound.as<uint64_t>()));
    EventSet ev;
    DBG_TRY(ev.create(2 * chunks + 1));
    cudaEvent_t ready = ev.e[2 * chunks];  // the stage buffers exist on the build's stream
    DBG_CUDA_TRY(cudaEventRecord(ready, s));
    DBG_CUDA_TRY(cudaStreamWaitEvent(cs, ready, 0));
    for (uint32_t c = 0; c < chunks; c++) {
      const uint64_t off = (uint64_t)c * chunk, len = std::min(chunk, total_bases - off);
      DevBuf &st = stage[c & 1];
      if (c >= 2) DBG_CUDA_TRY(cudaStreamWaitEvent(cs, ev.e[2 * (c - 2) + 1], 0));  // packed c - 2
      DBG_CUDA_TRY(cudaMemcpyAsync(st.p, in.reads + off, len, cudaMemcpyHostToDevice, cs));
      DBG_CUDA_TRY(cudaEventRecord(ev.e[2 * c], cs));
      DBG_CUDA_TRY(cudaStreamWaitEvent(s, ev.e[2 * c], 0));
      DBG_LAUNCH(ctx, ST_PACK, (double)len * 1.25,
                 k_pack_at<<<grid_for((len + 31) / 32, 256), 256, 0, s>>>(st.as<uint8_t>(), len,
                                                                        packed.as<uint64_t>(), off / 32, ctx->d_err));
      DBG_CUDA_TRY(cudaEventRecord(ev.e[2 * c + 1], s));
      if (N > 0) DBG_TRY(emit(kbound.as<uint64_t>() + c, (double)len / 4.0 + (double)N * sizeof(K) / chunks));
    }
    emitted = true;
  }

  // ---- K2 emit + digit histograms, K3 sort, K4 run-length reduce ----
  if (N > 0) {
    if (!emitted) DBG_TRY(emit(nullptr, 8.0 * nwords + 16.0 * n + (double)N * sizeof(K)));
    DBG_CUDA_TRY(cudaGetLastError());
    K *kp = keys_a.as<K>(), *alt = keys_b.as<K>();
    uint32_t *vn = nullptr, *van = nullptr;
    if (p0 > 0) {
      // high digits globally, then the local sort with the run-length
      // reduce: distinct keys into alt, multiplicities into mult_tmp
      DBG_TRY((radix_sort<K, false>(ctx, &kp, &alt, &vn, &van, N, kbits, d_hist, d_digit_base, p0)));
      DBG_TRY(seg_rle<K>(ctx, kp, alt, N, RADIX_BITS * p0, kbits, mult_tmp, &E));
      std::swap(kp, alt);  // the distinct keys are in the sort's buffer
    } else {
      // every digit globally, then the run-length reduce
      DBG_TRY(alloc_buf(ctx, headpos, (N + 1) * sizeof(uint32_t)));
      DBG_TRY((radix_sort<K, false>(ctx, &kp, &alt, &vn, &van, N, kbits, d_hist, d_digit_base)));
      DBG_TRY(run_length_reduce<K>(ctx, kp, N, alt, headpos.as<uint32_t>(), &E));
    }
    DBG_TRY(check_device_error(ctx));
    // keep the buffer holding the unique keys (alt); the sorted keys are done
    if (alt == keys_b.as<K>()) { uniq = std::move(keys_b); keys_a.release(); }
    else { uniq = std::move(keys_a); keys_b.release(); }
  }
  if (E >= 0x80000000ull) {
    set_error("%llu unique edges exceed one in-memory build (2^31 - 1)", (unsigned long long)E);
    return DBG_EOVERFLOW;
  }
  g->num_edges = E;

  // ---- node multiplicities (optional), while the packed reads are here ----
  DevBuf node_counts, read_counts;
  uint64_t Vk = 0, Vr = 0;
  if (ctx->node_mult)
    DBG_TRY(count_node_kmers<K>(ctx, packed, base_off, in.d_lengths, n, N, k, d_hist, d_digit_base, node_counts,
                                &Vk));
  if (ctx->node_reads)
    DBG_TRY(count_node_reads<K>(ctx, packed, base_off, in.d_lengths, n, N, k, d_hist, d_digit_base, read_counts,
                                &Vr));

  // ---- K5 edge ends + records of reads of length k ----
  const uint64_t R = 2 * E + I;
  const int nbits = 2 * (int)k;
  const int npasses = passes_for_bits(nbits);
  DBG_TRY(alloc_buf(ctx, g->edge_keys, std::max<uint64_t>(1, E) * sizeof(K)));
  DBG_TRY(alloc_buf(ctx, g->mult, std::max<uint64_t>(1, E) * sizeof(uint32_t)));
  DBG_TRY(alloc_buf(ctx, g->orient, std::max<uint64_t>(1, E)));
  DevBuf rk_a, rk_b, rv_a, rv_b;
  DBG_TRY(alloc_buf(ctx, rk_a, std::max<uint64_t>(1, R) * sizeof(K)));
  DBG_TRY(alloc_buf(ctx, rk_b, std::max<uint64_t>(1, R) * sizeof(K)));
  DBG_TRY(alloc_buf(ctx, rv_a, std::max<uint64_t>(1, R) * sizeof(uint32_t)));
  DBG_TRY(alloc_buf(ctx, rv_b, std::max<uint64_t>(1, R) * sizeof(uint32_t)));
  DBG_CUDA_TRY(cudaMemsetAsync(d_hist, 0, MAX_PASSES * RADIX * sizeof(unsigned long long), s));
  // records ranked within groups: align the digits with the top of the
  // 2k-bit key, so that the global passes resolve 8 bits each of it and
  // leave short groups
  int adj = ctx->seg_rank ? (8 - nbits % 8) % 8 : 0;
  int q0 = ctx->hybrid_sort ? hybrid_first_pass<K>(R, nbits + adj) : 0;
  if (q0 == 0) {
    adj = 0;
    q0 = ctx->hybrid_sort ? hybrid_first_pass<K>(R, nbits) : 0;
  }
  // below 2^29 edges the payloads carry both sides of each edge end, and
  // the node IDs pass stores them per adjacency slot (for the compaction)
  const bool sides = E > 0 && E < (1ull << 29);
  if (E > 0) {
    DBG_LAUNCH(ctx, ST_ENDPOINTS, (double)E * (3 * sizeof(K) + 4 + 4 + 1 + 8),
               k_endpoints<K><<<grid_for(E, EMIT_TILE), EMIT_BLOCK, 0, s>>>(
        uniq.as<K>(), headpos.p ? headpos.as<uint32_t>() : nullptr, mult_tmp.as<uint32_t>(), E, k,
        g->edge_keys.as<K>(), g->mult.as<uint32_t>(),
        g->orient.as<uint8_t>(), rk_a.as<K>(), rv_a.as<uint32_t>(), q0, npasses, d_hist, adj, sides));
  }
  if (I > 0) {
    DBG_CUDA_TRY(cudaMemsetAsync(ctx->d_counters + 2, 0, sizeof(uint32_t), s));
    DBG_LAUNCH(ctx, ST_ENDPOINTS, (double)n * 4 + (double)I * (sizeof(K) + 4),
               k_isolated<K><<<grid_for(n, 256), 256, 0, s>>>(packed.as<uint64_t>(), base_off.as<uint64_t>(),
                                                   in.d_lengths, n, k, rk_a.as<K>() + 2 * E,
                                                   rv_a.as<uint32_t>() + 2 * E, ctx->d_counters + 2, q0, npasses,
                                                   d_hist, adj));
  }
  DBG_CUDA_TRY(cudaGetLastError());
  uniq.release();
  headpos.release();
  mult_tmp.release();
  packed.release();
  base_off.release();
  edge_off.release();

  // ---- STEP-3 sort of the node records (stable: payload order kept) ----
  K *rk = rk_a.as<K>(), *rk_alt = rk_b.as<K>();
  uint32_t *rv = rv_a.as<uint32_t>(), *rv_alt = rv_b.as<uint32_t>();
  DBG_TRY((sort_records<K>(ctx, &rk, &rk_alt, &rv, &rv_alt, R, nbits, q0, d_hist, d_digit_base, adj)));

  // ---- K6 node IDs + adjacency rows, K7 neighbours ----
  DevBuf row_tmp;
  DBG_TRY(alloc_buf(ctx, row_tmp, (R + 1) * sizeof(uint64_t)));
  DBG_TRY(alloc_buf(ctx, g->src, std::max<uint64_t>(1, E) * sizeof(uint32_t)));
  DBG_TRY(alloc_buf(ctx, g->dst, std::max<uint64_t>(1, E) * sizeof(uint32_t)));
  DBG_TRY(alloc_buf(ctx, g->adj_edge, std::max<uint64_t>(1, 2 * E) * sizeof(uint32_t)));
  DBG_TRY(alloc_buf(ctx, g->adj_role, std::max<uint64_t>(1, 2 * E)));
  DBG_TRY(alloc_buf(ctx, g->adj_nbr, std::max<uint64_t>(1, 2 * E) * sizeof(uint32_t)));
  if (sides) DBG_TRY(alloc_buf(ctx, g->adj_side, 2 * E));
  uint64_t V = 0;
  if (R > 0) {
    // node keys go to the free record buffer first (|V| is known only after)
    uint64_t ends = 0;
    DBG_TRY(assign_node_ids<K>(ctx, rk, rv, R, rk_alt, row_tmp.as<uint64_t>(), g, 0u, 0ull, &V, &ends, E,
                               sides ? g->adj_side.as<uint8_t>() : nullptr));
    DBG_TRY(check_device_error(ctx));
    if (ends != 2 * E) {
      set_error("adjacency holds %llu edge ends, expected %llu", (unsigned long long)ends,
                (unsigned long long)(2 * E));
      return DBG_EINTERNAL;
    }
  }
  g->num_nodes = V;
  if (ctx->node_mult) {
    if (Vk != V) {
      set_error("node multiplicities: %llu distinct k-mers for %llu nodes", (unsigned long long)Vk,
                (unsigned long long)V);
      return DBG_EINTERNAL;
    }
    if (V == 0) DBG_TRY(alloc_buf(ctx, node_counts, sizeof(uint32_t)));
    g->node_mult = std::move(node_counts);
  }
  if (ctx->node_reads) {
    if (Vr != V) {
      set_error("node read counts: %llu distinct k-mers for %llu nodes", (unsigned long long)Vr,
                (unsigned long long)V);
      return DBG_EINTERNAL;
    }
    if (V == 0) DBG_TRY(alloc_buf(ctx, read_counts, sizeof(uint32_t)));
    g->node_reads = std::move(read_counts);
  }
  DBG_TRY(alloc_buf(ctx, g->node_keys, std::max<uint64_t>(1, V) * sizeof(K)));
  DBG_TRY(alloc_buf(ctx, g->row_ptr, (V + 1) * sizeof(uint64_t)));
  if (V > 0) {
    Span sp(ctx, ST_COPIES, 2.0 * V * (sizeof(K) + 8), 0);
    DBG_CUDA_TRY(cudaMemcpyAsync(g->node_keys.p, rk_alt, V * sizeof(K), cudaMemcpyDeviceToDevice, s));
    DBG_CUDA_TRY(cudaMemcpyAsync(g->row_ptr.p, row_tmp.p, (V + 1) * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
  } else {
    DBG_CUDA_TRY(cudaMemsetAsync(g->row_ptr.p, 0, sizeof(uint64_t), s));
  }
  if (E > 0) {
    DBG_LAUNCH(ctx, ST_ADJACENCY, 2.0 * E * (4 + 1 + 4 + 4),
               k_adj_nbr<<<grid_for(2 * E, 256 * 8), 256, 0, s>>>(g->adj_edge.as<uint32_t>(), g->adj_role.as<uint8_t>(),
                                                     g->src.as<uint32_t>(), g->dst.as<uint32_t>(), 2 * E,
                                                     g->adj_nbr.as<uint32_t>()));
    DBG_CUDA_TRY(cudaGetLastError());
  }
  DBG_CUDA_TRY(cudaStreamSynchronize(s));
  return check_device_error(ctx);
}

}  // namespace dbg

namespace dbg {

// ---------------------------------------------------------------------------
// Autotuner: times one digit pass of every variant of a key kind on n
// synthetic keys (a counter-based hash of the index, so all digits vary) and
// keeps the fastest.  ms_out[v] receives each variant's pass time.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t tune_hash(uint64_t x) {
  x += 0x9e3779b97f4a7c15ull;
  x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ull;
  x = (x ^ (x >> 27)) * 0x94d049bb133111ebull;
  return x ^ (x >> 31);
}

template <class K>
__global__ void k_tune_fill(K *keys, uint32_t *vals, uint64_t n) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    K k;
    if constexpr (sizeof(K) == 8) {
      k = tune_hash(i);
    } else {
      k = Key128{tune_hash(2 * i), tune_hash(2 * i + 1)};
    }
    keys[i] = k;
    if (vals) vals[i] = (uint32_t)i;
  }
}

// digit histogram of one 8-bit digit position of arbitrary keys
template <class K>
__global__ void k_tune_hist(const K *keys, uint64_t n, int shift, unsigned long long *hist) {
  __shared__ uint32_t h[RADIX];
  for (int i = threadIdx.x; i < RADIX; i += blockDim.x) h[i] = 0;
  __syncthreads();
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
    atomicAdd(&h[KeyOps<K>::digit(keys[i], shift, RADIX_BITS)], 1u);
  __syncthreads();
  for (int i = threadIdx.x; i < RADIX; i += blockDim.x)
    if (h[i]) atomicAdd(hist + i, (unsigned long long)h[i]);
}

template <class K, bool V>
dbg_status autotune_kind(dbg_ctx *ctx, uint64_t n, double *ms_out) {
  cudaStream_t s = ctx->stream;
  int count = 0;
  const SortVariant *t = SortKind<K, V>::table(&count);
  DevBuf ka, kb, va, vb, small;
  DBG_TRY(alloc_buf(ctx, ka, n * sizeof(K)));
  DBG_TRY(alloc_buf(ctx, kb, n * sizeof(K)));
  if (V) {
    DBG_TRY(alloc_buf(ctx, va, n * 4));
    DBG_TRY(alloc_buf(ctx, vb, n * 4));
  }
  DBG_TRY(alloc_buf(ctx, small, RADIX * 16));
  unsigned long long *hist = small.as<unsigned long long>();
  uint64_t *dbase = reinterpret_cast<uint64_t *>(hist + RADIX);
  k_tune_fill<K><<<1024, 256, 0, s>>>(ka.as<K>(), V ? va.as<uint32_t>() : nullptr, n);
  DBG_CUDA_TRY(cudaMemsetAsync(hist, 0, RADIX * 8, s));
  k_tune_hist<K><<<1024, 256, 0, s>>>(ka.as<K>(), n, 8, hist);
  k_digit_base<<<1, RADIX, 0, s>>>(hist, dbase);
  int min_tile = t[0].tile;
  for (int v = 0; v < count; v++) min_tile = std::min(min_tile, t[v].tile);
  DBG_TRY(ensure_status(ctx, ((n + min_tile - 1) / min_tile) * RADIX));
  cudaEvent_t e0, e1;
  DBG_CUDA_TRY(cudaEventCreate(&e0));
  DBG_CUDA_TRY(cudaEventCreate(&e1));
  int best = 0;
  double best_ms = 1e30;
  for (int v = 0; v < count; v++) {
    float total = 0.f;
    for (int rep = 0; rep < 4; rep++) {
      uint32_t epoch;
      DBG_TRY(next_epoch(ctx, &epoch));
      DBG_CUDA_TRY(cudaMemsetAsync(ctx->d_counters, 0, sizeof(uint32_t), s));
      cudaEventRecord(e0, s);
      t[v].launch(ctx, ka.p, kb.p, V ? va.as<uint32_t>() : nullptr, V ? vb.as<uint32_t>() : nullptr, n, 8, dbase,
                  epoch);
      cudaEventRecord(e1, s);
      DBG_CUDA_TRY(cudaEventSynchronize(e1));
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep > 0) total += ms;  // the first launch is a warm-up
    }
    const double ms = total / 3.0;
    if (ms_out) ms_out[v] = ms;
    if (ms < best_ms) {
      best_ms = ms;
      best = v;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  DBG_CUDA_TRY(cudaGetLastError());
  DBG_TRY(check_device_error(ctx));
  ctx->sort_variant[SortKind<K, V>::kind] = best;
  return DBG_OK;
}

template <class K, bool V>
const char *variant_name(uint32_t v, uint32_t *count) {
  int c = 0;
  const SortVariant *t = SortKind<K, V>::table(&c);
  *count = (uint32_t)c;
  return v < (uint32_t)c ? t[v].name : nullptr;
}

}  // namespace dbg

namespace dbg {

// ---------------------------------------------------------------------------
// The bucket path (dbg_build_bucketed): Section 5's out-of-core
// construction with key-range partitioning in place of the external merge.
// ---------------------------------------------------------------------------
// Cuts the prefix bins into consecutive ranges of at most `cap` items (a
// single bin above cap gets a range of its own).
inline std::vector<std::pair<uint32_t, uint32_t>> plan_ranges(const uint64_t *hist, uint64_t cap,
                                                              std::vector<uint64_t> *sizes) {
  std::vector<std::pair<uint32_t, uint32_t>> out;
  uint32_t lo = 0;
  uint64_t acc = 0;
  for (uint32_t b = 0; b < (uint32_t)PREFIX_BINS; b++) {
    if (acc > 0 && acc + hist[b] > cap) {
      out.emplace_back(lo, b);
      sizes->push_back(acc);
      lo = b;
      acc = 0;
    }
    acc += hist[b];
  }
  out.emplace_back(lo, (uint32_t)PREFIX_BINS);
  sizes->push_back(acc);
  return out;
}

static dbg_status scan_flags(dbg_ctx *ctx, const uint32_t *in, uint64_t n, uint64_t *out, uint32_t *total) {
  cudaStream_t s = ctx->stream;
  const uint64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
  DBG_TRY(ensure_status(ctx, tiles));
  uint32_t epoch;
  DBG_TRY(next_epoch(ctx, &epoch));
  DBG_CUDA_TRY(cudaMemsetAsync(ctx->d_counters, 0, 2 * sizeof(uint32_t), s));
  DBG_LAUNCH(ctx, ST_NODE_IDS, 12.0 * n,
             k_scan_excl<<<(unsigned)tiles, SCAN_BLOCK, 0, s>>>(in, n, out, ctx->d_status, ctx->d_counters, epoch,
                                                                ctx->spin_limit, ctx->d_err, ctx->d_counters + 1));
  DBG_CUDA_TRY(cudaGetLastError());
  return read_small(ctx, ctx->d_counters + 1, sizeof(uint32_t), total);
}

template <class K>
dbg_status concat_chunks(dbg_ctx *ctx, std::vector<DevBuf> &chunks, const std::vector<uint64_t> &counts,
                         size_t elem, void *dst) {
  uint64_t at = 0;
  for (size_t i = 0; i < chunks.size(); i++) {
    if (counts[i])
      DBG_CUDA_TRY(cudaMemcpyAsync(static_cast<char *>(dst) + at * elem, chunks[i].p, counts[i] * elem,
                                   cudaMemcpyDeviceToDevice, ctx->stream));
    at += counts[i];
    chunks[i].release();
  }
  return DBG_OK;
}

template <class K>
dbg_status build_bucketed_impl(dbg_ctx *ctx, const BucketInput &in, uint64_t budget, dbg_graph *g,
                               uint32_t *n_edge_buckets, uint32_t *n_node_buckets) {
  cudaStream_t s = ctx->stream;
  const uint32_t k = in.k;
  const uint64_t n = in.n;
  const int m = (int)k + 1;
  const uint64_t w = sizeof(K);
  g->k = k;
  g->key_words = sizeof(K) / 8;
  DBG_CUDA_TRY(cudaStreamSynchronize(s));  // the pinned mirror is free

  // ---- per-read offsets ----
  DevBuf base_off, edge_off, tile_sums, small;
  const uint64_t off_tiles = (n + OFF_TILE - 1) / OFF_TILE;
  DBG_TRY(alloc_buf(ctx, base_off, (n + 1) * 8));
  DBG_TRY(alloc_buf(ctx, edge_off, (n + 1) * 8));
  DBG_TRY(alloc_buf(ctx, tile_sums, std::max<uint64_t>(1, off_tiles) * sizeof(Sum3)));
  DBG_TRY(alloc_buf(ctx, small, 64 * 8 + MAX_PASSES * RADIX * 16 + PREFIX_BINS * 8));
  uint64_t *d_totals = small.as<uint64_t>();
  unsigned long long *d_hist = reinterpret_cast<unsigned long long *>(d_totals + 64);
  uint64_t *d_digit_base = reinterpret_cast<uint64_t *>(d_hist + MAX_PASSES * RADIX);
  unsigned long long *d_phist = reinterpret_cast<unsigned long long *>(d_digit_base + MAX_PASSES * RADIX);
  if (n > 0)
    DBG_LAUNCH(ctx, ST_OFFSETS, 4.0 * n,
               k_read_tile_sums<<<(unsigned)off_tiles, OFF_BLOCK, 0, s>>>(in.d_lengths, n, k, tile_sums.as<Sum3>()));
  DBG_LAUNCH(ctx, ST_OFFSETS, 0.0,
             k_scan_tile_sums<<<1, 1024, 0, s>>>(tile_sums.as<Sum3>(), (uint32_t)off_tiles, d_totals,
                                                 base_off.as<uint64_t>(), edge_off.as<uint64_t>(), n));
  if (n > 0)
    DBG_LAUNCH(ctx, ST_OFFSETS, 20.0 * n,
               k_read_offsets<<<(unsigned)off_tiles, OFF_BLOCK, 0, s>>>(in.d_lengths, n, k, tile_sums.as<Sum3>(),
                                                                        base_off.as<uint64_t>(),
                                                                        edge_off.as<uint64_t>()));
  DBG_CUDA_TRY(cudaGetLastError());
  uint64_t totals[3];
  DBG_TRY(read_small(ctx, d_totals, sizeof(totals), totals));
  const uint64_t total_bases = totals[0], N = totals[1], I = totals[2];
  tile_sums.release();
  g->num_instances = N;

  // ---- pack the reads once; host reads stream through a staging buffer ----
  DevBuf packed;
  const uint64_t nwords = (total_bases + 31) / 32;
  DBG_TRY(alloc_buf(ctx, packed, (nwords + 3) * 8));
  DBG_CUDA_TRY(cudaMemsetAsync(packed.as<uint64_t>() + nwords, 0, 3 * 8, s));
  if (nwords > 0) {
    if (in.reads_on_device) {
      DBG_LAUNCH(ctx, ST_PACK, (double)total_bases * 1.25,
                 k_pack<<<grid_for(nwords, 256), 256, 0, s>>>(reinterpret_cast<const uint8_t *>(in.reads),
                                                              total_bases, packed.as<uint64_t>(), nwords, ctx->d_err));
    } else {
      const uint64_t chunk = 256ull << 20;  // bases per staged copy (a multiple of 32)
      DevBuf stage;
      DBG_TRY(alloc_buf(ctx, stage, std::min(chunk, total_bases)));
      for (uint64_t off = 0; off < total_bases; off += chunk) {
        const uint64_t len = std::min(chunk, total_bases - off);
        DBG_CUDA_TRY(cudaMemcpyAsync(stage.p, in.reads + off, len, cudaMemcpyHostToDevice, s));
        DBG_LAUNCH(ctx, ST_PACK, (double)len * 1.25,
                   k_pack_at<<<grid_for((len + 31) / 32, 256), 256, 0, s>>>(stage.as<uint8_t>(), len,
                                                                          packed.as<uint64_t>(), off / 32,
                                                                          ctx->d_err));
      }
      DBG_CUDA_TRY(cudaStreamSynchronize(s));  // the staging buffer is released next
    }
  }
  DBG_CUDA_TRY(cudaGetLastError());
  DBG_TRY(check_device_error(ctx));

  // ---- edge-key ranges ----
  const unsigned emit_grid = (unsigned)std::min<uint64_t>(grid_for(n, EMIT_BLOCK / 32), 152ull * 64);
  std::vector<uint64_t> hist(PREFIX_BINS, 0);
  if (N > 0) {
    DBG_CUDA_TRY(cudaMemsetAsync(d_phist, 0, PREFIX_BINS * 8, s));
    DBG_LAUNCH(ctx, ST_EMIT, 8.0 * nwords + 16.0 * n,
               k_emit_prefix_hist<K><<<emit_grid, EMIT_BLOCK, 0, s>>>(packed.as<uint64_t>(), base_off.as<uint64_t>(),
                                                                      edge_off.as<uint64_t>(), n, k, d_phist));
    DBG_CUDA_TRY(cudaMemcpyAsync(hist.data(), d_phist, PREFIX_BINS * 8, cudaMemcpyDeviceToHost, s));
    DBG_CUDA_TRY(cudaStreamSynchronize(s));
  }
  const uint64_t persistent = (nwords + 3) * 8 + (n + 1) * 16;
  const uint64_t room = budget > persistent ? budget - persistent : 0;
  const uint64_t key_cap = std::max<uint64_t>(1ull << 16, room / (2 * w + 4 + 4));
  std::vector<uint64_t> sizes;
  auto ranges = plan_ranges(hist.data(), key_cap, &sizes);
  *n_edge_buckets = (uint32_t)ranges.size();

  const int kbits = 2 * m;
  const int kpasses = passes_for_bits(kbits);
  std::vector<DevBuf> ck, cm, co;
  std::vector<uint64_t> ce;
  uint64_t E = 0;
  for (size_t b = 0; b < ranges.size(); b++) {
    const uint64_t cnt = sizes[b];
    if (cnt == 0) continue;
    DevBuf ka, kb, headpos;
    DBG_TRY(alloc_buf(ctx, ka, cnt * w));
    DBG_TRY(alloc_buf(ctx, kb, cnt * w));
    DBG_TRY(alloc_buf(ctx, headpos, (cnt + 1) * 4));
    DBG_CUDA_TRY(cudaMemsetAsync(d_hist, 0, MAX_PASSES * RADIX * 8, s));
    DBG_CUDA_TRY(cudaMemsetAsync(ctx->d_counters + 8, 0, 4, s));
    DBG_LAUNCH(ctx, ST_EMIT, 8.0 * nwords + 16.0 * n + (double)cnt * w,
               k_emit_range<K><<<emit_grid, EMIT_BLOCK, 0, s>>>(packed.as<uint64_t>(), base_off.as<uint64_t>(),
                                                                edge_off.as<uint64_t>(), n, k, ranges[b].first,
                                                                ranges[b].second, ka.as<K>(), ctx->d_counters + 8,
                                                                kpasses, d_hist));
    DBG_CUDA_TRY(cudaGetLastError());
    K *kp = ka.as<K>(), *alt = kb.as<K>();
    uint32_t *vn = nullptr, *van = nullptr;
    uint64_t eb64 = 0;
    const int p0 = ctx->hybrid_sort ? hybrid_first_pass<K>(cnt, kbits) : 0;
    if (p0 > 0) {
      // multiplicities go where the run heads would (headpos is cnt + 1 long)
      DBG_TRY((radix_sort<K, false>(ctx, &kp, &alt, &vn, &van, cnt, kbits, d_hist, d_digit_base, p0)));
      DevBuf mdense;
      DBG_TRY(seg_rle<K>(ctx, kp, alt, cnt, RADIX_BITS * p0, kbits, mdense, &eb64));
      if (eb64) DBG_CUDA_TRY(cudaMemcpyAsync(headpos.p, mdense.p, eb64 * 4, cudaMemcpyDeviceToDevice, s));
      std::swap(kp, alt);  // the distinct keys are in the sort's buffer
    } else {
      DBG_TRY((radix_sort<K, false>(ctx, &kp, &alt, &vn, &van, cnt, kbits, d_hist, d_digit_base)));
      DBG_TRY(run_length_reduce<K>(ctx, kp, cnt, alt, headpos.as<uint32_t>(), &eb64));
    }
    DBG_TRY(check_device_error(ctx));
    const uint32_t eb = (uint32_t)eb64;
    DevBuf k1, m1, o1;
    DBG_TRY(alloc_buf(ctx, k1, std::max<uint64_t>(1, eb) * w));
    DBG_TRY(alloc_buf(ctx, m1, std::max<uint64_t>(1, eb) * 4));
    DBG_TRY(alloc_buf(ctx, o1, std::max<uint64_t>(1, eb)));
    if (eb)
      DBG_LAUNCH(ctx, ST_ENDPOINTS, (double)eb * (2 * w + 9),
                 k_edge_finish<K><<<grid_for(eb, 256), 256, 0, s>>>(alt, p0 > 0 ? nullptr : headpos.as<uint32_t>(),
                                                                   headpos.as<uint32_t>(), eb, k, k1.as<K>(),
                                                                   m1.as<uint32_t>(), o1.as<uint8_t>()));
    ck.push_back(std::move(k1));
    cm.push_back(std::move(m1));
    co.push_back(std::move(o1));
    ce.push_back(eb);
    E += eb;
  }
  if (E >= 0x80000000ull) {
    set_error("%llu unique edges exceed one build (2^31 - 1)", (unsigned long long)E);
    return DBG_EOVERFLOW;
  }
  g->num_edges = E;
  const uint64_t E1 = std::max<uint64_t>(1, E);
  DBG_TRY(alloc_buf(ctx, g->edge_keys, E1 * w));
  DBG_TRY(alloc_buf(ctx, g->mult, E1 * 4));
  DBG_TRY(alloc_buf(ctx, g->orient, E1));
  DBG_TRY(concat_chunks<K>(ctx, ck, ce, w, g->edge_keys.p));
  DBG_TRY(concat_chunks<K>(ctx, cm, ce, 4, g->mult.p));
  DBG_TRY(concat_chunks<K>(ctx, co, ce, 1, g->orient.p));

  // ---- node-key ranges ----
  DBG_TRY(alloc_buf(ctx, g->src, E1 * 4));
  DBG_TRY(alloc_buf(ctx, g->dst, E1 * 4));
  DBG_TRY(alloc_buf(ctx, g->adj_edge, 2 * E1 * 4));
  DBG_TRY(alloc_buf(ctx, g->adj_role, 2 * E1));
  DBG_TRY(alloc_buf(ctx, g->adj_nbr, 2 * E1 * 4));
  std::fill(hist.begin(), hist.end(), 0);
  if (E > 0) {
    DBG_CUDA_TRY(cudaMemsetAsync(d_phist, 0, PREFIX_BINS * 8, s));
    DBG_LAUNCH(ctx, ST_ENDPOINTS, (double)E * w,
               k_node_prefix_hist<K><<<grid_for(E, 256 * 8), 256, 0, s>>>(g->edge_keys.as<K>(), E, k, d_phist));
    DBG_CUDA_TRY(cudaMemcpyAsync(hist.data(), d_phist, PREFIX_BINS * 8, cudaMemcpyDeviceToHost, s));
    DBG_CUDA_TRY(cudaStreamSynchronize(s));
  }
  const uint64_t held = persistent + E1 * (w + 4 + 1 + 4 + 4 + 2 * 9);
  const uint64_t room2 = budget > held ? budget - held : 0;
  const uint64_t rec_cap = std::max<uint64_t>(1ull << 16, room2 / (2 * (w + 4) + 16));
  sizes.clear();
  auto nranges = plan_ranges(hist.data(), rec_cap, &sizes);
  *n_node_buckets = (uint32_t)nranges.size();
  DevBuf flags, pos;
  if (E > 0) {
    DBG_TRY(alloc_buf(ctx, flags, 2 * E * 4));
    DBG_TRY(alloc_buf(ctx, pos, (2 * E + 1) * 8));
  }
  const int nbits = 2 * (int)k;
  const int npasses = passes_for_bits(nbits);
  std::vector<DevBuf> cnk, crp;
  std::vector<uint64_t> cv;
  uint64_t base_v = 0, base_slot = 0;
  for (size_t c = 0; c < nranges.size(); c++) {
    const uint32_t lo = nranges[c].first, hi = nranges[c].second;
    uint32_t Rc = 0;
    if (E > 0) {
      DBG_LAUNCH(ctx, ST_ENDPOINTS, (double)E * w + 8.0 * E,
                 k_flag_ends<K><<<grid_for(E, 256 * 8), 256, 0, s>>>(g->edge_keys.as<K>(), E, k, lo, hi,
                                                                    flags.as<uint32_t>()));
      DBG_TRY(scan_flags(ctx, flags.as<uint32_t>(), 2 * E, pos.as<uint64_t>(), &Rc));
    }
    const uint64_t cap = (uint64_t)Rc + I;
    if (cap == 0) continue;
    DevBuf ra, rb, va, vb, row_tmp;
    DBG_TRY(alloc_buf(ctx, ra, cap * w));
    DBG_TRY(alloc_buf(ctx, rb, cap * w));
    DBG_TRY(alloc_buf(ctx, va, cap * 4));
    DBG_TRY(alloc_buf(ctx, vb, cap * 4));
    DBG_CUDA_TRY(cudaMemsetAsync(d_hist, 0, MAX_PASSES * RADIX * 8, s));
    if (Rc > 0)
      DBG_LAUNCH(ctx, ST_ENDPOINTS, (double)E * (w + 8) + (double)Rc * (w + 4),
                 k_gather_ends<K><<<grid_for(E, 256 * 8), 256, 0, s>>>(g->edge_keys.as<K>(), E, k,
                                                                      flags.as<uint32_t>(), pos.as<uint64_t>(),
                                                                      ra.as<K>(), va.as<uint32_t>(), npasses,
                                                                      d_hist));
    uint64_t R = Rc;
    if (I > 0) {
      DBG_CUDA_TRY(cudaMemsetAsync(ctx->d_counters + 9, 0, 4, s));
      DBG_LAUNCH(ctx, ST_ENDPOINTS, (double)n * 4,
                 k_isolated_range<K><<<grid_for(n, 256), 256, 0, s>>>(packed.as<uint64_t>(), base_off.as<uint64_t>(),
                                                                     in.d_lengths, n, k, lo, hi, ra.as<K>() + Rc,
                                                                     va.as<uint32_t>() + Rc, ctx->d_counters + 9,
                                                                     npasses, d_hist));
      uint32_t iso = 0;
      DBG_TRY(read_small(ctx, ctx->d_counters + 9, 4, &iso));
      R += iso;
    }
    if (R == 0) continue;
    K *rk = ra.as<K>(), *rk_alt = rb.as<K>();
    uint32_t *rv = va.as<uint32_t>(), *rv_alt = vb.as<uint32_t>();
    const int q0 = ctx->hybrid_sort ? hybrid_first_pass<K>(R, nbits) : 0;
    DBG_TRY((sort_records<K>(ctx, &rk, &rk_alt, &rv, &rv_alt, R, nbits, q0, d_hist, d_digit_base)));
    DBG_TRY(alloc_buf(ctx, row_tmp, (R + 1) * 8));
    uint64_t tot[2] = {0, 0};
    DBG_TRY(assign_node_ids<K>(ctx, rk, rv, R, rk_alt, row_tmp.as<uint64_t>(), g, (uint32_t)base_v, base_slot,
                               &tot[0], &tot[1]));
    DBG_TRY(check_device_error(ctx));
    const uint64_t Vc = tot[0];
    DevBuf nk, rp;
    DBG_TRY(alloc_buf(ctx, nk, std::max<uint64_t>(1, Vc) * w));
    DBG_TRY(alloc_buf(ctx, rp, std::max<uint64_t>(1, Vc) * 8));
    if (Vc) {
      DBG_CUDA_TRY(cudaMemcpyAsync(nk.p, rk_alt, Vc * w, cudaMemcpyDeviceToDevice, s));
      DBG_CUDA_TRY(cudaMemcpyAsync(rp.p, row_tmp.p, Vc * 8, cudaMemcpyDeviceToDevice, s));
    }
    cnk.push_back(std::move(nk));
    crp.push_back(std::move(rp));
    cv.push_back(Vc);
    base_v += Vc;
    base_slot += tot[1];
  }
  if (base_slot != 2 * E) {
    set_error("adjacency holds %llu edge ends, expected %llu", (unsigned long long)base_slot,
              (unsigned long long)(2 * E));
    return DBG_EINTERNAL;
  }
  const uint64_t V = base_v;
  g->num_nodes = V;
  DBG_TRY(alloc_buf(ctx, g->node_keys, std::max<uint64_t>(1, V) * w));
  DBG_TRY(alloc_buf(ctx, g->row_ptr, (V + 1) * 8));
  DBG_TRY(concat_chunks<K>(ctx, cnk, cv, w, g->node_keys.p));
  DBG_TRY(concat_chunks<K>(ctx, crp, cv, 8, g->row_ptr.p));
  uint64_t *last = reinterpret_cast<uint64_t *>(ctx->h_pinned + 64);  // pinned: safe for an async copy
  *last = 2 * E;
  DBG_CUDA_TRY(cudaMemcpyAsync(g->row_ptr.as<uint64_t>() + V, last, 8, cudaMemcpyHostToDevice, s));
  if (E > 0)
    DBG_LAUNCH(ctx, ST_ADJACENCY, 2.0 * E * 13,
               k_adj_nbr<<<grid_for(2 * E, 256 * 8), 256, 0, s>>>(g->adj_edge.as<uint32_t>(), g->adj_role.as<uint8_t>(),
                                                                 g->src.as<uint32_t>(), g->dst.as<uint32_t>(), 2 * E,
                                                                 g->adj_nbr.as<uint32_t>()));
  DBG_CUDA_TRY(cudaGetLastError());
  DBG_CUDA_TRY(cudaStreamSynchronize(s));
  return check_device_error(ctx);
}

}  // namespace dbg
