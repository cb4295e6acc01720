// k_segsort.cuh -- the local half of the hybrid radix sort (K3 / STEP-2 and
// STEP-3).  The global onesweep passes sort the keys by their high bits only
// (the digits at and above bit `low_bits`), which leaves every group of keys
// with equal high bits contiguous.  One CTA then finishes a run of whole
// groups in shared memory: tile t covers [bound[t], bound[t+1]), where
// bound[t] is the start of the group holding position t * TILE_T (found by
// binary search, the high bits being sorted), so no group is split between
// CTAs, and the keys are sorted by their remaining bits with an in-shared-
// memory LSD radix sort.  Because the global passes are stable and the local
// passes are stable, the result equals a full stable LSD sort.
//
// A tile longer than the shared-memory capacity (it holds a group of more
// keys than that, e.g. a tandem repeat's (k+1)-mer) is "oversize": the host
// gathers all oversize tiles into one buffer, sorts it with the global
// passes over every digit, and the local kernels copy those results into
// place instead of sorting.
//
// k_seg_sort sorts (key, payload) records (STEP-3's node records), with 256
// threads of 24 items (126 registers, 2 CTAs per SM) or, in its wide form,
// 384 threads of 16 items: the same capacity with half again the warps.
// k_seg_rle finishes STEP-2 on the edge keys: it sorts them and writes each
// distinct key once with the length of its run (its multiplicity) into the
// tile's own range; k_seg_compact then packs the tiles' outputs.  Equal keys share their high bits, so no run of
// equal keys crosses a tile boundary.  k_seg_count does the same work by
// counting each tile's copies in a hash table first and sorting only the
// distinct keys.
#pragma once

#include "k_build.cuh"

namespace dbg {

constexpr int SEG_BLOCK = 256;

template <class K, bool HAS_VAL, int ITEMS, int BLOCK = SEG_BLOCK>
struct SegSortSmem {
  static constexpr int WARPS = BLOCK / 32;
  static constexpr int CAP = BLOCK * ITEMS;
  K keys[CAP];
  uint32_t vals[HAS_VAL ? CAP : 1];
  uint32_t whist[WARPS][RADIX];
  uint32_t match[WARPS][RADIX + 1];
  uint32_t cnt[ITEMS * WARPS + 1];
  uint32_t hpos[HAS_VAL ? 1 : CAP + 1];  // run heads' positions by rank (run-length reduce)
  uint32_t tmp[8];
  uint64_t bound[2];
  K base;
  uint32_t tile, passes, excl, total, spread_bits;
};

// bound[t] for t in [0, tiles]: the first index of the group holding
// position t * tile_keys (n for positions past the end).  The high bits are
// sorted, so a binary search finds it; it starts in the last 8192 keys
// before the position unless the group is longer.
template <class K>
__global__ void k_seg_bounds(const K *__restrict__ keys, uint64_t n, int low_bits, uint64_t tile_keys,
                             uint64_t tiles, uint64_t *__restrict__ bound) {
  for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t <= tiles; t += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t pos = t * tile_keys;
    uint64_t b;
    if (t == tiles || pos >= n) {
      b = n;
    } else if (pos == 0) {
      b = 0;
    } else {
      const K target = KeyOps<K>::shr(keys[pos], low_bits);
      uint64_t lo = pos > 8192 ? pos - 8192 : 0, hi = pos;
      if (lo > 0 && !KeyOps<K>::less(KeyOps<K>::shr(keys[lo], low_bits), target)) lo = 0;
      while (lo < hi) {  // first index whose high bits are not below target
        const uint64_t mid = lo + (hi - lo) / 2;
        if (KeyOps<K>::less(KeyOps<K>::shr(keys[mid], low_bits), target)) lo = mid + 1;
        else hi = mid;
      }
      b = lo;
    }
    bound[t] = b;
  }
}

// osize[t] = the tile's length if it exceeds cap (an oversize tile), else 0.
static __global__ void k_seg_oversize(const uint64_t *__restrict__ bound, uint64_t tiles, uint32_t cap,
                                      uint32_t *__restrict__ osize) {
  for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < tiles; t += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t sz = bound[t + 1] - bound[t];
    osize[t] = sz > cap ? (uint32_t)sz : 0u;
  }
}

// Copies every oversize tile to gk[ooff[t] ...] (and its payloads), in tile
// order, so that one sort of the gathered keys sorts each of them.
template <class K, bool HAS_VAL>
__global__ void k_seg_gather(const K *__restrict__ kin, const uint32_t *__restrict__ vin,
                             const uint64_t *__restrict__ bound, const uint32_t *__restrict__ osize,
                             const uint64_t *__restrict__ ooff, uint64_t tiles, K *__restrict__ gk,
                             uint32_t *__restrict__ gv) {
  for (uint64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
    const uint32_t sz = osize[t];
    if (sz == 0) continue;
    const uint64_t s = bound[t], o = ooff[t];
    for (uint32_t j = threadIdx.x; j < sz; j += blockDim.x) {
      gk[o + j] = kin[s + j];
      if (HAS_VAL) gv[o + j] = vin[s + j];
    }
  }
}

// The tile's range, its base (the first key with the low bits cleared) and
// the number of local passes, into shared memory.  The caller checks that
// the tile is not oversize.
template <class K, class S>
__device__ __forceinline__ void seg_setup(S &sm, const K *__restrict__ kin, const uint64_t *__restrict__ bound,
                                          uint32_t tile, int low_bits, int key_bits) {
  if (threadIdx.x == 0) {
    const uint64_t s = bound[tile], e = bound[tile + 1];
    sm.bound[0] = s;
    sm.bound[1] = e;
    if (e > s) {
      const K first = kin[s], last = kin[e - 1];
      sm.base = KeyOps<K>::sub(first, KeyOps<K>::mask_low(first, low_bits));
      const int spread_bits =
          KeyOps<K>::bitlen(KeyOps<K>::sub(KeyOps<K>::shr(last, low_bits), KeyOps<K>::shr(first, low_bits)));
      sm.passes = (uint32_t)((min(low_bits + spread_bits, key_bits) + RADIX_BITS - 1) / RADIX_BITS);
      sm.spread_bits = (uint32_t)spread_bits;
    }
  }
  __syncthreads();
}

// first index in sorted a[0, m) whose value is >= x
__device__ __forceinline__ uint32_t lower_bound_u32(const uint32_t *__restrict__ a, uint32_t m, uint64_t x) {
  uint32_t lo = 0, hi = m;
  while (lo < hi) {
    const uint32_t mid = lo + (hi - lo) / 2;
    if ((uint64_t)a[mid] < x) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// One stable ranking step: item i of this warp gets its rank among the
// warp's equal digits so far, packed as (rank << 9) | digit, with digit
// RADIX for invalid items.  Order: item, then lane.  An item is valid if its
// index wofs + 32 i + lane is below lim.
template <class K, int ITEMS, int RANK, class S>
__device__ __forceinline__ void rank_items(S &sm, const K (&key)[ITEMS], uint32_t (&rank)[ITEMS], int nitems,
                                           uint32_t wofs, uint32_t lim, int shift) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned lt_mask = (1u << lane) - 1u;
#pragma unroll
  for (int i = 0; i < ITEMS; i++) {
    if (i >= nitems) break;  // warp-uniform
    const bool valid = wofs + i * 32 + lane < lim;
    const uint32_t d = valid ? KeyOps<K>::digit(key[i], shift, RADIX_BITS) : (uint32_t)RADIX;
    unsigned peers;
    if (RANK == RANK_MATCH) {
      peers = __match_any_sync(0xffffffffu, d);
    } else if (RANK == RANK_ATOMIC) {
      atomicOr(&sm.match[warp][d], 1u << lane);
      __syncwarp();
      peers = sm.match[warp][d];
      __syncwarp();
      if (lane == __ffs(peers) - 1) sm.match[warp][d] = 0;
    } else {
      peers = 0xffffffffu;
#pragma unroll
      for (int bt = 0; bt <= RADIX_BITS; bt++) {
        const bool bit = (d >> bt) & 1u;
        const unsigned bal = __ballot_sync(0xffffffffu, bit);
        peers &= bit ? bal : ~bal;
      }
    }
    const int leader = __ffs(peers) - 1;
    uint32_t before = 0;
    if (lane == leader && valid) {
      before = sm.whist[warp][d];
      sm.whist[warp][d] = before + __popc(peers);
    }
    before = __shfl_sync(0xffffffffu, before, leader);
    rank[i] = ((before + __popc(peers & lt_mask)) << 9) | d;
    __syncwarp();
  }
}

// Turns the per-warp digit counts into each warp's first position per digit
// (digit-major, then warp); returns the number of ranked keys to all threads.
template <class S>
__device__ __forceinline__ uint32_t digit_positions(S &sm) {
  const int tid = threadIdx.x;
  __syncthreads();
  uint32_t c = 0;
  if (tid < RADIX)
#pragma unroll
    for (int w = 0; w < S::WARPS; w++) c += sm.whist[w][tid];
  const uint32_t start = block_excl_scan_256(c, sm.tmp);
  if (tid < RADIX) {
    uint32_t run = start;
#pragma unroll
    for (int w = 0; w < S::WARPS; w++) {
      const uint32_t x = sm.whist[w][tid];
      sm.whist[w][tid] = run;
      run += x;
    }
    if (tid == RADIX - 1) sm.total = run;
  }
  __syncthreads();
  return sm.total;
}

template <class K, bool HAS_VAL, int ITEMS, class S>
__device__ __forceinline__ void scatter_items(S &sm, const K (&key)[ITEMS], const uint32_t (&val)[ITEMS],
                                              const uint32_t (&rank)[ITEMS], int nitems) {
  const int warp = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < ITEMS; i++) {
    if (i >= nitems) break;
    const uint32_t d = rank[i] & 0x1ffu;
    if (d < RADIX) {
      const uint32_t q = sm.whist[warp][d] + (rank[i] >> 9);
      sm.keys[q] = key[i];
      if (HAS_VAL) sm.vals[q] = val[i];
    }
  }
}

// Loads the consecutive keys [wofs, wofs + 32 * nitems) of the staging area
// (item-major; valid below lim) and zeroes the warp counters for the next
// pass.  The caller synchronises before ranking.
template <class K, bool HAS_VAL, int ITEMS, class S>
__device__ __forceinline__ void reload_items(S &sm, K (&key)[ITEMS], uint32_t (&val)[ITEMS], int nitems,
                                             uint32_t wofs, uint32_t lim) {
  const int lane = threadIdx.x & 31;
  __syncthreads();
#pragma unroll
  for (int i = 0; i < ITEMS; i++) {
    if (i >= nitems) break;
    const uint32_t j = wofs + i * 32 + lane;
    if (j < lim) {
      key[i] = sm.keys[j];
      if (HAS_VAL) val[i] = sm.vals[j];
    }
  }
  for (int i = threadIdx.x; i < S::WARPS * RADIX; i += S::WARPS * 32) (&sm.whist[0][0])[i] = 0;
}

// Records: tile t sorted in shared memory into kout / vout at its own range;
// an oversize tile copies its slice of the gathered, globally sorted records
// (gk / gv at ooff[t]).
template <class K, int ITEMS, int RANK, int BLOCK>
__device__ __forceinline__ void seg_sort_tile(
    SegSortSmem<K, true, ITEMS, BLOCK> &sm, uint32_t tile, const K *__restrict__ kin, const uint32_t *__restrict__ vin,
    const uint64_t *__restrict__ bound, const uint32_t *__restrict__ osize, const uint64_t *__restrict__ ooff,
    const K *__restrict__ gk, const uint32_t *__restrict__ gv, K *__restrict__ kout, uint32_t *__restrict__ vout,
    int low_bits, int key_bits) {
  using S = SegSortSmem<K, true, ITEMS, BLOCK>;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (osize[tile]) {
    const uint64_t s = bound[tile], o = ooff[tile];
    for (uint32_t j = tid; j < osize[tile]; j += BLOCK) {
      kout[s + j] = gk[o + j];
      vout[s + j] = gv[o + j];
    }
    return;
  }
  for (int i = tid; i < S::WARPS * RADIX; i += BLOCK) (&sm.whist[0][0])[i] = 0;
  for (int i = tid; i < S::WARPS * (RADIX + 1); i += BLOCK) (&sm.match[0][0])[i] = 0;
  seg_setup<K>(sm, kin, bound, tile, low_bits, key_bits);
  const uint64_t s = sm.bound[0];
  const uint32_t cnt = (uint32_t)(sm.bound[1] - s);
  if (cnt == 0) return;
  const K base = sm.base;
  const int passes = (int)sm.passes;
  // the keys spread evenly over the warps: warp w holds the consecutive
  // keys [w * 32 * ipw, (w + 1) * 32 * ipw), item-major
  const int ipw = (int)((cnt + BLOCK - 1) / BLOCK);
  const uint32_t wofs = (uint32_t)warp * 32u * ipw;
  K key[ITEMS];
  uint32_t val[ITEMS];
  uint32_t rank[ITEMS];
#pragma unroll
  for (int i = 0; i < ITEMS; i++) {
    const uint32_t j = wofs + i * 32 + lane;
    const bool in = i < ipw && j < cnt;
    key[i] = in ? KeyOps<K>::sub(kin[s + j], base) : KeyOps<K>::zero();
    val[i] = in ? vin[s + j] : 0u;
  }
  for (int p = 0; p < passes; p++) {
    if (p > 0) {
      reload_items<K, true, ITEMS>(sm, key, val, ipw, wofs, cnt);
      __syncthreads();
    }
    rank_items<K, ITEMS, RANK>(sm, key, rank, ipw, wofs, cnt, p * RADIX_BITS);
    digit_positions(sm);
    scatter_items<K, true, ITEMS>(sm, key, val, rank, ipw);
  }
  __syncthreads();
  for (uint32_t j = tid; j < cnt; j += BLOCK) {
    kout[s + j] = KeyOps<K>::add(sm.keys[j], base);
    vout[s + j] = sm.vals[j];
  }
}

// One CTA per tile; or, with a tile list, a grid of CTAs that take the
// *list_count listed tiles in turn.
template <class K, int ITEMS, int RANK, int BLOCK = SEG_BLOCK>
__global__ __launch_bounds__(BLOCK, 2) void k_seg_sort(
    const K *__restrict__ kin, const uint32_t *__restrict__ vin, const uint64_t *__restrict__ bound,
    const uint32_t *__restrict__ osize, const uint64_t *__restrict__ ooff, const K *__restrict__ gk,
    const uint32_t *__restrict__ gv, K *__restrict__ kout, uint32_t *__restrict__ vout, int low_bits, int key_bits,
    const uint32_t *__restrict__ tile_list = nullptr, const uint32_t *__restrict__ list_count = nullptr) {
  using S = SegSortSmem<K, true, ITEMS, BLOCK>;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  S &sm = *reinterpret_cast<S *>(smem_raw);
  if (!tile_list) {
    seg_sort_tile<K, ITEMS, RANK, BLOCK>(sm, blockIdx.x, kin, vin, bound, osize, ooff, gk, gv, kout, vout, low_bits,
                                         key_bits);
    return;
  }
  const uint32_t n = *list_count;
  for (uint32_t q = blockIdx.x; q < n; q += gridDim.x) {
    seg_sort_tile<K, ITEMS, RANK, BLOCK>(sm, tile_list[q], kin, vin, bound, osize, ooff, gk, gv, kout, vout,
                                         low_bits, key_bits);
    __syncthreads();
  }
}

// Records by ranking within groups.  The tile's keys are already ordered
// by their high bits (from low_bits up), so a record's place in the sorted
// tile is its group's start plus the number of records of its group that
// precede it: those with a smaller key, or an equal key and an earlier
// position (which keeps the sort stable).  A 64-bit record is staged in
// shared memory as one word, (low bits << 13) | position, and ranked by
// comparing that word with the group's others; a 128-bit record as its key,
// compared whole with the position as tie-break.  No digit pass and no
// block barrier is needed past the staging.  The work is the sum of the
// squared group lengths, small when the global passes leave groups of a
// few dozen records.  A tile with a group longer than RANK_GROUP_MAX is
// listed in fb_list for the digit-pass kernel instead.
constexpr int RANK_BLOCK = 512;
constexpr uint32_t RANK_GROUP_MAX = 512;

template <class K>
struct SegRankSmem {
  static constexpr int CAP = SEG_BLOCK * (sizeof(K) == 8 ? 24 : 12);  // the digit-pass kernel's capacity
  static constexpr int ITEMS = CAP / RANK_BLOCK;
  static_assert(CAP <= 8192, "positions fit 13 bits");
  using W = std::conditional_t<sizeof(K) == 8, uint64_t, K>;
  W pk[CAP];  // 64-bit: (low bits << 13) | position; 128-bit: the key
  uint32_t val[CAP];
  uint16_t ord[CAP];           // group of each record
  uint16_t gstart[CAP + 1];    // first position of each group, then cnt
  uint32_t cnt[ITEMS * (RANK_BLOCK / 32) + 1];
  uint32_t maxg;
};

template <class K>
__global__ __launch_bounds__(RANK_BLOCK, 2) void k_seg_rank(
    const K *__restrict__ kin, const uint32_t *__restrict__ vin, const uint64_t *__restrict__ bound,
    const uint32_t *__restrict__ osize, const uint64_t *__restrict__ ooff, const K *__restrict__ gk,
    const uint32_t *__restrict__ gv, K *__restrict__ kout, uint32_t *__restrict__ vout, int low_bits,
    uint32_t *__restrict__ fb_list, uint32_t *__restrict__ fb_count) {
  using S = SegRankSmem<K>;
  constexpr int ITEMS = S::ITEMS;
  constexpr bool WIDE = sizeof(K) == 16;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  S &sm = *reinterpret_cast<S *>(smem_raw);
  const int tid = threadIdx.x;
  const uint32_t tile = blockIdx.x;
  const uint64_t s = bound[tile];
  if (osize[tile]) {
    const uint64_t o = ooff[tile];
    for (uint32_t j = tid; j < osize[tile]; j += RANK_BLOCK) {
      kout[s + j] = gk[o + j];
      vout[s + j] = gv[o + j];
    }
    return;
  }
  const uint32_t cnt = (uint32_t)(bound[tile + 1] - s);
  if (cnt == 0) return;
  if (tid == 0) sm.maxg = 0;
  // stage the records; a group starts where the high bits change
  bool head[ITEMS];
  uint32_t rk[ITEMS];
#pragma unroll
  for (int i = 0; i < ITEMS; i++) {
    const uint32_t j = (uint32_t)i * RANK_BLOCK + tid;
    head[i] = false;
    if (j < cnt) {
      const K x = kin[s + j];
      head[i] = j == 0 || !KeyOps<K>::eq(KeyOps<K>::shr(x, low_bits), KeyOps<K>::shr(kin[s + j - 1], low_bits));
      if constexpr (WIDE) {
        sm.pk[j] = x;
      } else {
        sm.pk[j] = ((x & ((1ull << low_bits) - 1ull)) << 13) | j;
      }
      sm.val[j] = vin[s + j];
    }
  }
  const uint32_t G = tile_flag_ranks<RANK_BLOCK, ITEMS>(head, rk, sm.cnt);
#pragma unroll
  for (int i = 0; i < ITEMS; i++) {
    const uint32_t j = (uint32_t)i * RANK_BLOCK + tid;
    if (j < cnt) {
      const uint32_t o = rk[i] + (head[i] ? 1u : 0u) - 1u;
      sm.ord[j] = (uint16_t)o;
      if (head[i]) sm.gstart[o] = (uint16_t)j;
    }
  }
  if (tid == 0) sm.gstart[G] = (uint16_t)cnt;
  __syncthreads();
  uint32_t mg = 0;
  for (uint32_t o = tid; o < G; o += RANK_BLOCK) mg = max(mg, (uint32_t)sm.gstart[o + 1] - sm.gstart[o]);
  mg = __reduce_max_sync(0xffffffffu, mg);
  if ((tid & 31) == 0 && mg) atomicMax(&sm.maxg, mg);
  __syncthreads();
  if (sm.maxg > RANK_GROUP_MAX) {
    if (tid == 0) fb_list[atomicAdd(fb_count, 1u)] = tile;
    return;
  }
  for (uint32_t i = tid; i < cnt; i += RANK_BLOCK) {
    const uint32_t o = sm.ord[i], a = sm.gstart[o], b = sm.gstart[o + 1];
    uint32_t r = 0;
    if constexpr (WIDE) {
      const K x = sm.pk[i];
      for (uint32_t t = a; t < b; t++) {
        const K y = sm.pk[t];
        r += (KeyOps<K>::less(y, x) || (t < i && KeyOps<K>::eq(y, x))) ? 1u : 0u;
      }
      kout[s + a + r] = x;
    } else {
      const uint64_t p = sm.pk[i];
#pragma unroll 4
      for (uint32_t t = a; t < b; t++) r += sm.pk[t] < p ? 1u : 0u;
      kout[s + a + r] = kin[s + i];
    }
    vout[s + a + r] = sm.val[i];
  }
}

// Edge keys (STEP-2's local pass).  Tile t writes its distinct keys and
// their multiplicities at the start of its own range, ustage / mstage[bound[t]
// ...], and their number to tcount[t]; a scan of tcount and k_seg_compact
// then make the dense edge list.  No tile waits for another.

// The distinct keys of an oversize tile, from the gathered, globally sorted
// and reduced keys (guniq, run heads gheads at the positions of the gathered
// buffer, H runs in all, gheads[H] = its length).
template <class K>
__device__ __forceinline__ void seg_rle_gathered(uint32_t tile, const uint64_t *__restrict__ bound,
                                                 const uint32_t *__restrict__ osize, const uint64_t *__restrict__ ooff,
                                                 const K *__restrict__ guniq, const uint32_t *__restrict__ gheads,
                                                 uint32_t H, K *__restrict__ ustage, uint32_t *__restrict__ mstage,
                                                 uint32_t *__restrict__ tcount) {
  const uint64_t o = ooff[tile], s = bound[tile];
  const uint32_t h0 = lower_bound_u32(gheads, H, o), h1 = lower_bound_u32(gheads, H, o + osize[tile]);
  for (uint32_t r = threadIdx.x; r < h1 - h0; r += blockDim.x) {
    ustage[s + r] = guniq[h0 + r];
    mstage[s + r] = gheads[h0 + r + 1] - gheads[h0 + r];
  }
  if (threadIdx.x == 0) tcount[tile] = h1 - h0;
}

// Block radix local sort + RLE, one CTA per tile (every tile, or the tiles
// of tile_list when it is not null).
template <class K, int ITEMS, int RANK>
__global__ __launch_bounds__(SEG_BLOCK, 2) void k_seg_rle(
    const K *__restrict__ kin, const uint64_t *__restrict__ bound, const uint32_t *__restrict__ osize,
    const uint64_t *__restrict__ ooff, const K *__restrict__ guniq, const uint32_t *__restrict__ gheads, uint32_t H,
    K *__restrict__ ustage, uint32_t *__restrict__ mstage, uint32_t *__restrict__ tcount, int low_bits,
    int key_bits, const uint32_t *__restrict__ tile_list) {
  using S = SegSortSmem<K, false, ITEMS>;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  S &sm = *reinterpret_cast<S *>(smem_raw);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t tile = tile_list ? tile_list[blockIdx.x] : blockIdx.x;
  {
    if (osize[tile]) {
      seg_rle_gathered<K>(tile, bound, osize, ooff, guniq, gheads, H, ustage, mstage, tcount);
      return;
    }
    for (int i = tid; i < S::WARPS * RADIX; i += SEG_BLOCK) (&sm.whist[0][0])[i] = 0;
    for (int i = tid; i < S::WARPS * (RADIX + 1); i += SEG_BLOCK) (&sm.match[0][0])[i] = 0;
    seg_setup<K>(sm, kin, bound, tile, low_bits, key_bits);
    const uint64_t s = sm.bound[0];
    const uint32_t cnt = (uint32_t)(sm.bound[1] - s);
    const K base = sm.base;
    uint32_t rank[ITEMS];
    if (cnt > 0) {
      const int passes = (int)sm.passes;
      const int ipw = (int)((cnt + SEG_BLOCK - 1) / SEG_BLOCK);
      const uint32_t wofs = (uint32_t)warp * 32u * ipw;
      K key[ITEMS];
      uint32_t none[ITEMS];
#pragma unroll
      for (int i = 0; i < ITEMS; i++) {
        const uint32_t j = wofs + i * 32 + lane;
        key[i] = (i < ipw && j < cnt) ? KeyOps<K>::sub(kin[s + j], base) : KeyOps<K>::zero();
      }
      for (int p = 0; p < passes; p++) {
        if (p > 0) {
          reload_items<K, false, ITEMS>(sm, key, none, ipw, wofs, cnt);
          __syncthreads();
        }
        rank_items<K, ITEMS, RANK>(sm, key, rank, ipw, wofs, cnt, p * RADIX_BITS);
        digit_positions(sm);
        scatter_items<K, false, ITEMS>(sm, key, none, rank, ipw);
      }
    }
    __syncthreads();
    // distinct keys: the first key of each run; a run's length is the
    // distance to the next run's first key
    bool head[ITEMS];
#pragma unroll
    for (int i = 0; i < ITEMS; i++) {
      const uint32_t j = (uint32_t)i * SEG_BLOCK + tid;
      head[i] = j < cnt && (j == 0 || !KeyOps<K>::eq(sm.keys[j], sm.keys[j - 1]));
    }
    const uint32_t count = tile_flag_ranks<SEG_BLOCK, ITEMS>(head, rank, sm.cnt);
#pragma unroll
    for (int i = 0; i < ITEMS; i++)
      if (head[i]) sm.hpos[rank[i]] = (uint32_t)i * SEG_BLOCK + tid;
    if (tid == 0) sm.hpos[count] = cnt;
    __syncthreads();
#pragma unroll
    for (int i = 0; i < ITEMS; i++) {
      if (head[i]) {
        const uint32_t j = (uint32_t)i * SEG_BLOCK + tid;
        ustage[s + rank[i]] = KeyOps<K>::add(sm.keys[j], base);
        mstage[s + rank[i]] = sm.hpos[rank[i] + 1] - j;
      }
    }
    if (tid == 0) tcount[tile] = count;
  }
}

// Edge keys, counted before they are sorted.  A tile of the local pass
// holds every copy of each of its keys, and at read coverage c a tile of n
// keys holds about n / c distinct ones, so k_seg_count counts the copies
// first, in a shared-memory hash table of TBL slots (linear probing; a slot
// is claimed by compare-and-swap and counted by atomic add), packs the
// occupied slots to the front of the table in slot order, and then orders
// only the distinct keys.  The output is that of k_seg_rle: each distinct
// key once, in order, with its multiplicity (STEP-2), staged in the tile's
// own range.  The table is small so that several CTAs share an SM; a tile
// whose keys do not fit (a probe longer than PROBES slots) is listed in
// over_list and sorted by k_seg_rle instead.
//
// Ordering the distinct keys.  With rank_groups set, the distinct keys are
// bucketed by their high bits (from low_bits up) -- the tile's groups, in
// order; where those bits span more than TBL values, by their top bits, so
// that a bucket holds 2, 4, ... adjacent groups -- and each key goes to its
// bucket's start plus the number of the bucket's keys below it; a tile
// with a bucket of more than COUNT_GROUP_MAX distinct keys is radix-sorted
// by the 8-bit passes instead (and counted in rank_fb).  (Packing a 64-bit
// key's offset and its count into one slot word, counted by 64-bit shared
// atomic adds, measured 1.9x slower: the hot slots of a 30x-covered key
// serialise.)
constexpr uint32_t COUNT_GROUP_MAX = 256;

// Hash-table slots of the counting pass.  The empty mark is the all-ones
// key, which no key offset reaches: an offset is key - base <= key, and the
// all-ones key (T repeated) is never canonical, its reverse complement (A
// repeated) being smaller.
template <class K>
struct SlotOps;

// claim(p, d) returns the slot's key, having stored d there if it was empty
// (then it returns empty): the caller has found d's slot when it gets empty
// or d, and probes on otherwise.
template <>
struct SlotOps<uint64_t> {
  __device__ static uint64_t empty() { return ~0ull; }
  // Fibonacci hashing: the high 32 bits of d times 2^64 / golden ratio
  __device__ static uint32_t hash(uint64_t d) { return (uint32_t)((d * 0x9e3779b97f4a7c15ull) >> 32); }
  __device__ static uint64_t claim(uint64_t *p, uint64_t d) {
    // a 64-bit load is single-copy atomic, so it settles most probes
    // without an atomic operation
    const uint64_t cur = *reinterpret_cast<const volatile uint64_t *>(p);
    if (cur != ~0ull) return cur;
    return atomicCAS(reinterpret_cast<unsigned long long *>(p), ~0ull, d);
  }
};

template <>
struct SlotOps<Key128> {
  __device__ static Key128 empty() { return Key128{~0ull, ~0ull}; }
  __device__ static uint32_t hash(Key128 d) {
    return (uint32_t)(((d.lo ^ (d.hi * 0x9e3779b97f4a7c15ull)) * 0xc2b2ae3d27d4eb4full) >> 32);
  }
  // every probe is a 128-bit compare-and-swap, which also reads the slot
  // whole (two 64-bit loads could see a slot half written)
  __device__ static Key128 claim(Key128 *p, Key128 d) {
    Key128 old;
    asm volatile(
        "{\n .reg .b128 c, n, o;\n mov.b128 c, {%2, %3};\n mov.b128 n, {%4, %5};\n"
        " atom.shared.cas.b128 o, [%6], c, n;\n mov.b128 {%0, %1}, o;\n}"
        : "=l"(old.hi), "=l"(old.lo)
        : "l"(~0ull), "l"(~0ull), "l"(d.hi), "l"(d.lo), "r"(smem_u32(p))
        : "memory");
    return old;
  }
};

template <class K, int RANK>
struct SegCountSmem {
  static constexpr int WARPS = SEG_BLOCK / 32;
  static constexpr int TBL = 2048;                // hash slots
  static constexpr int TBITS = 11;                // log2(TBL)
  static constexpr int ITEMS = TBL / SEG_BLOCK;   // distinct keys per thread in the sort
  static constexpr int LOAD = 8;                  // keys per thread per load batch
  static constexpr uint32_t PROBES = 64;          // longest probe before the tile overflows
  static_assert((1 << TBITS) == TBL, "table size");
  K keys[TBL];         // hash slots; then the distinct keys, packed and sorted
  uint32_t vals[TBL];  // copies per slot; then per distinct key
  uint16_t perm[TBL];  // distinct keys bucketed by group
  uint32_t gst[TBL];   // distinct keys per group, then where each group ends
  uint32_t whist[WARPS][RADIX];
  uint32_t match[RANK == RANK_ATOMIC ? WARPS : 1][RADIX + 1];
  uint32_t cnt[ITEMS * WARPS + 1];
  uint32_t tmp[8];
  uint64_t bound[2];
  K base;
  uint32_t tile, passes, excl, total, spread_bits, overflow, maxg;
};

// high bits of a key offset, as a group index within the tile
template <class K>
__device__ __forceinline__ uint32_t group_of(K d, int low_bits) {
  return (uint32_t)KeyOps<K>::words_lo(KeyOps<K>::shr(d, low_bits));
}

template <class K, int RANK>
__global__ __launch_bounds__(SEG_BLOCK, 4) void k_seg_count(
    const K *__restrict__ kin, const uint64_t *__restrict__ bound, const uint32_t *__restrict__ osize,
    const uint64_t *__restrict__ ooff, const K *__restrict__ guniq, const uint32_t *__restrict__ gheads, uint32_t H,
    K *__restrict__ ustage, uint32_t *__restrict__ mstage, uint32_t *__restrict__ tcount,
    uint32_t *__restrict__ over_list, uint32_t *__restrict__ over_count, int low_bits, int key_bits,
    int rank_groups, uint32_t *__restrict__ rank_fb) {
  using S = SegCountSmem<K, RANK>;
  using O = SlotOps<K>;
  constexpr int ITEMS = S::ITEMS;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  S &sm = *reinterpret_cast<S *>(smem_raw);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t tile = blockIdx.x;
  if (osize[tile]) {
    seg_rle_gathered<K>(tile, bound, osize, ooff, guniq, gheads, H, ustage, mstage, tcount);
    return;
  }
  for (int i = tid; i < S::WARPS * RADIX; i += SEG_BLOCK) (&sm.whist[0][0])[i] = 0;
  if (RANK == RANK_ATOMIC)
    for (int i = tid; i < S::WARPS * (RADIX + 1); i += SEG_BLOCK) (&sm.match[0][0])[i] = 0;
  for (int j = tid; j < S::TBL; j += SEG_BLOCK) {
    sm.keys[j] = O::empty();
    sm.vals[j] = 0;
  }
  if (tid == 0) sm.overflow = 0;
  seg_setup<K>(sm, kin, bound, tile, low_bits, key_bits);  // synchronises
  const uint64_t s = sm.bound[0];
  const uint32_t cnt = (uint32_t)(sm.bound[1] - s);
  const K base = sm.base;
  // the tile's path (uniform): ranked by buckets of groups
  const bool by_groups = rank_groups && cnt > 0;
  const int bshift = (int)sm.spread_bits > S::TBITS ? (int)sm.spread_bits - S::TBITS : 0;
  // count: each key into its slot, LOAD keys per thread at a time
  for (uint32_t j0 = 0; j0 < cnt; j0 += S::LOAD * SEG_BLOCK) {
    K d[S::LOAD];
#pragma unroll
    for (int i = 0; i < S::LOAD; i++) {
      const uint32_t j = j0 + (uint32_t)i * SEG_BLOCK + tid;
      d[i] = j < cnt ? KeyOps<K>::sub(kin[s + j], base) : O::empty();
    }
    if (*reinterpret_cast<volatile uint32_t *>(&sm.overflow)) break;
#pragma unroll
    for (int i = 0; i < S::LOAD; i++) {
      if (KeyOps<K>::eq(d[i], O::empty())) continue;
      uint32_t h = O::hash(d[i]) >> (32 - S::TBITS);
      bool done = false;
      for (uint32_t probe = 0; probe < S::PROBES; probe++) {
        const K cur = O::claim(&sm.keys[h], d[i]);
        if (KeyOps<K>::eq(cur, O::empty()) || KeyOps<K>::eq(cur, d[i])) {
          atomicAdd(&sm.vals[h], 1u);
          done = true;
          break;
        }
        h = (h + 1) & (S::TBL - 1);
      }
      if (!done) sm.overflow = 1;
    }
  }
  __syncthreads();
  if (sm.overflow) {
    if (tid == 0) over_list[atomicAdd(over_count, 1u)] = tile;
    return;
  }
  // pack the occupied slots to the front in slot order: a slot moves to its
  // rank among the occupied slots (at most its own index) once every slot
  // has been read
  uint32_t D;
  {
    K pk[ITEMS];
    uint32_t pc[ITEMS], pr[ITEMS];
    bool occ[ITEMS];
#pragma unroll
    for (int i = 0; i < ITEMS; i++) {
      const uint32_t j = (uint32_t)i * SEG_BLOCK + tid;
      pk[i] = sm.keys[j];
      pc[i] = sm.vals[j];
      occ[i] = !KeyOps<K>::eq(pk[i], O::empty());
    }
    D = tile_flag_ranks<SEG_BLOCK, ITEMS>(occ, pr, sm.cnt);
#pragma unroll
    for (int i = 0; i < ITEMS; i++) {
      if (occ[i]) {
        sm.keys[pr[i]] = pk[i];
        sm.vals[pr[i]] = pc[i];
      }
    }
  }
  __syncthreads();
  const int gshift = low_bits + bshift;  // a key offset's bucket bits
  bool ranked = false;
  if (by_groups && D > 0) {
    // bucket the distinct keys: counts, exclusive scan (ITEMS consecutive
    // buckets per thread), then placement
    const uint32_t G = 1u << ((int)sm.spread_bits - bshift);
    for (uint32_t o = tid; o < G; o += SEG_BLOCK) sm.gst[o] = 0;
    if (tid == 0) sm.maxg = 0;
    __syncthreads();
    for (uint32_t r = tid; r < D; r += SEG_BLOCK) atomicAdd(&sm.gst[group_of<K>(sm.keys[r], gshift)], 1u);
    __syncthreads();
    uint32_t gc[ITEMS], sum = 0, mx = 0;
#pragma unroll
    for (int i = 0; i < ITEMS; i++) {
      const uint32_t o = (uint32_t)tid * ITEMS + i;
      gc[i] = o < G ? sm.gst[o] : 0u;
      sum += gc[i];
      mx = max(mx, gc[i]);
    }
    uint32_t run = block_excl_scan_256(sum, sm.tmp);
#pragma unroll
    for (int i = 0; i < ITEMS; i++) {
      const uint32_t o = (uint32_t)tid * ITEMS + i;
      if (o < G) sm.gst[o] = run;
      run += gc[i];
    }
    mx = __reduce_max_sync(0xffffffffu, mx);
    if (lane == 0 && mx) atomicMax(&sm.maxg, mx);
    __syncthreads();
    if (sm.maxg <= COUNT_GROUP_MAX) {
      for (uint32_t r = tid; r < D; r += SEG_BLOCK)
        sm.perm[atomicAdd(&sm.gst[group_of<K>(sm.keys[r], gshift)], 1u)] = (uint16_t)r;
      __syncthreads();
      // bucket o now spans [gst[o - 1], gst[o]) (from 0 for o = 0)
      for (uint32_t q = tid; q < D; q += SEG_BLOCK) {
        const uint32_t r = sm.perm[q], o = group_of<K>(sm.keys[r], gshift);
        const uint32_t a = o ? sm.gst[o - 1] : 0u, b = sm.gst[o];
        const K x = sm.keys[r];
        uint32_t below = 0;
        for (uint32_t t = a; t < b; t++) below += KeyOps<K>::less(sm.keys[sm.perm[t]], x) ? 1u : 0u;
        ustage[s + a + below] = KeyOps<K>::add(x, base);
        mstage[s + a + below] = sm.vals[r];
      }
      ranked = true;
    }
  }
  if (!ranked && D > 0) {
    if (rank_groups && tid == 0) atomicAdd(rank_fb, 1u);
    // sort the D distinct keys (with their counts) by their offset bits
    const int passes = (int)sm.passes;
    const int ipw = (int)((D + SEG_BLOCK - 1) / SEG_BLOCK);
    const uint32_t wofs = (uint32_t)warp * 32u * ipw;
    K key[ITEMS];
    uint32_t val[ITEMS], rank[ITEMS];
#pragma unroll
    for (int i = 0; i < ITEMS; i++) {
      const uint32_t j = wofs + i * 32 + lane;
      const bool in = i < ipw && j < D;
      key[i] = in ? sm.keys[j] : KeyOps<K>::zero();
      val[i] = in ? sm.vals[j] : 0u;
    }
    for (int p = 0; p < passes; p++) {
      if (p > 0) {
        reload_items<K, true, ITEMS>(sm, key, val, ipw, wofs, D);
        __syncthreads();
      }
      rank_items<K, ITEMS, RANK>(sm, key, rank, ipw, wofs, D, p * RADIX_BITS);
      digit_positions(sm);
      scatter_items<K, true, ITEMS>(sm, key, val, rank, ipw);
    }
    __syncthreads();
    for (uint32_t r = tid; r < D; r += SEG_BLOCK) {
      ustage[s + r] = KeyOps<K>::add(sm.keys[r], base);
      mstage[s + r] = sm.vals[r];
    }
  }
  if (tid == 0) tcount[tile] = D;
}

// Moves every tile's distinct keys from its staging range to the dense
// edge list (toff = exclusive scan of tcount).
template <class K>
__global__ void k_seg_compact(const uint64_t *__restrict__ bound, const uint32_t *__restrict__ tcount,
                              const uint64_t *__restrict__ toff, uint64_t tiles, const K *__restrict__ ustage,
                              const uint32_t *__restrict__ mstage, K *__restrict__ uniq, uint32_t *__restrict__ mult) {
  for (uint64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
    const uint64_t s = bound[t], o = toff[t];
    const uint32_t c = tcount[t];
    for (uint32_t r = threadIdx.x; r < c; r += blockDim.x) {
      uniq[o + r] = ustage[s + r];
      mult[o + r] = mstage[s + r];
    }
  }
}

}  // namespace dbg
