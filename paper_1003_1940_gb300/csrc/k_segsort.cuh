// k_segsort.cuh -- the local half of the hybrid radix sort (K3 / STEP-2 and
// STEP-3).  The global onesweep passes sort the keys by their high bits only
// (the digits at and above bit `low_bits`), which leaves every group of keys
// with equal high bits contiguous.  One CTA then finishes a run of whole
// groups in shared memory: the tile of nominal size TILE_T is stretched to
// start and end on group boundaries, so no group is split between CTAs, and
// the keys are sorted by their remaining bits with an in-shared-memory LSD
// radix sort.  Because the global passes are stable and the local passes are
// stable, the result equals a full stable LSD sort.
//
// k_seg_sort sorts (key, payload) records (STEP-3's node records).
// k_seg_rle finishes STEP-2 on the edge keys: it sorts them and writes each
// distinct key once with the length of its run (its multiplicity), at an
// offset found by decoupled look-back over the tiles' distinct-key counts.
// Equal keys share their high bits, so no run of equal keys crosses a tile
// boundary.
//
// A group longer than the window TILE_CAP - TILE_T cannot be aligned; the
// tiles around it set *oversize and do nothing, and the host then finishes
// with the remaining global passes instead.
#pragma once

#include "k_build.cuh"

namespace dbg {

constexpr int SEG_BLOCK = 256;

template <class K, bool HAS_VAL, int ITEMS>
struct SegSortSmem {
  static constexpr int WARPS = SEG_BLOCK / 32;
  static constexpr int CAP = SEG_BLOCK * ITEMS;
  K keys[CAP];
  uint32_t vals[HAS_VAL ? CAP : 1];
  uint32_t whist[WARPS][RADIX];
  uint32_t match[WARPS][RADIX + 1];
  uint32_t cnt[ITEMS * WARPS + 1];
  uint32_t hpos[HAS_VAL ? 1 : CAP + 1];  // run heads' positions by rank (run-length reduce)
  uint32_t tmp[8];
  uint64_t bound[2];
  K base;
  uint32_t tile, passes, fail, excl, total;
};

// First index q in [pos, pos + window) that starts a group (q >= n counts as
// a start); false if there is none.  Called by one whole warp; pos >= 1.
template <class K>
__device__ __forceinline__ bool find_group_start(const K *__restrict__ keys, uint64_t n, uint64_t pos,
                                                 uint64_t window, int low_bits, uint64_t *out) {
  const int lane = threadIdx.x & 31;
  for (uint64_t q0 = pos; q0 < pos + window; q0 += 32) {
    const uint64_t q = q0 + lane;
    bool start = false;
    if (q < pos + window) {
      if (q >= n)
        start = true;
      else
        start = !KeyOps<K>::eq(KeyOps<K>::shr(keys[q], low_bits), KeyOps<K>::shr(keys[q - 1], low_bits));
    }
    const unsigned m = __ballot_sync(0xffffffffu, start);
    if (m) {
      *out = q0 + (uint64_t)(__ffs(m) - 1);
      return true;
    }
  }
  return false;
}

// The tile's group-aligned range [s, e) into sm.bound, its base (the first
// key with the low bits cleared) and the number of local passes.  Returns
// false (after flagging *oversize) if the range could not be aligned.
template <class K, int TILE_T, class S>
__device__ __forceinline__ bool seg_setup(S &sm, const K *__restrict__ kin, uint64_t n, int low_bits, int key_bits,
                                          uint32_t tile, uint32_t *oversize) {
  constexpr uint64_t WINDOW = S::CAP - TILE_T;
  static_assert(TILE_T < S::CAP && WINDOW <= TILE_T, "tile shape");
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp < 2) {
    const uint64_t pos = (uint64_t)(tile + warp) * TILE_T;
    uint64_t b = 0;
    bool ok = true;
    if (pos == 0) b = 0;
    else if (pos >= n) b = n;
    else ok = find_group_start(kin, n, pos, WINDOW, low_bits, &b);
    if (lane == 0) {
      sm.bound[warp] = b;
      if (!ok) atomicOr(&sm.fail, 1u);
    }
  }
  __syncthreads();
  const uint64_t s = sm.bound[0], e = sm.bound[1];
  if (sm.fail || e < s || e - s > (uint64_t)S::CAP) {
    if (threadIdx.x == 0) atomicOr(oversize, 1u);
    return false;
  }
  if (threadIdx.x == 0 && e > s) {
    const K first = kin[s], last = kin[e - 1];
    sm.base = KeyOps<K>::sub(first, KeyOps<K>::mask_low(first, low_bits));
    const int spread_bits =
        KeyOps<K>::bitlen(KeyOps<K>::sub(KeyOps<K>::shr(last, low_bits), KeyOps<K>::shr(first, low_bits)));
    sm.passes = (uint32_t)((min(low_bits + spread_bits, key_bits) + RADIX_BITS - 1) / RADIX_BITS);
  }
  __syncthreads();
  return true;
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
  for (int i = threadIdx.x; i < S::WARPS * RADIX; i += SEG_BLOCK) (&sm.whist[0][0])[i] = 0;
}

template <class K, bool HAS_VAL, int ITEMS, int TILE_T, int RANK>
__global__ __launch_bounds__(SEG_BLOCK, 2) void k_seg_sort(
    const K *__restrict__ kin, const uint32_t *__restrict__ vin, K *__restrict__ kout, uint32_t *__restrict__ vout,
    uint64_t n, int low_bits, int key_bits, uint32_t *oversize) {
  using S = SegSortSmem<K, HAS_VAL, ITEMS>;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  S &sm = *reinterpret_cast<S *>(smem_raw);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int i = tid; i < S::WARPS * RADIX; i += SEG_BLOCK) (&sm.whist[0][0])[i] = 0;
  for (int i = tid; i < S::WARPS * (RADIX + 1); i += SEG_BLOCK) (&sm.match[0][0])[i] = 0;
  if (tid == 0) sm.fail = 0;
  __syncthreads();
  if (!seg_setup<K, TILE_T>(sm, kin, n, low_bits, key_bits, blockIdx.x, oversize)) return;
  const uint64_t s = sm.bound[0];
  const uint32_t cnt = (uint32_t)(sm.bound[1] - s);
  if (cnt == 0) return;
  const K base = sm.base;
  const int passes = (int)sm.passes;
  // the keys spread evenly over the warps: warp w holds the consecutive
  // keys [w * 32 * ipw, (w + 1) * 32 * ipw), item-major
  const int ipw = (int)((cnt + SEG_BLOCK - 1) / SEG_BLOCK);
  const uint32_t wofs = (uint32_t)warp * 32u * ipw;
  K key[ITEMS];
  uint32_t val[ITEMS];
  uint32_t rank[ITEMS];
#pragma unroll
  for (int i = 0; i < ITEMS; i++) {
    const uint32_t j = wofs + i * 32 + lane;
    const bool in = i < ipw && j < cnt;
    key[i] = in ? KeyOps<K>::sub(kin[s + j], base) : KeyOps<K>::zero();
    val[i] = (HAS_VAL && in) ? vin[s + j] : 0u;
  }
  for (int p = 0; p < passes; p++) {
    if (p > 0) {
      reload_items<K, HAS_VAL, ITEMS>(sm, key, val, ipw, wofs, cnt);
      __syncthreads();
    }
    rank_items<K, ITEMS, RANK>(sm, key, rank, ipw, wofs, cnt, p * RADIX_BITS);
    digit_positions(sm);
    scatter_items<K, HAS_VAL, ITEMS>(sm, key, val, rank, ipw);
  }
  __syncthreads();
  for (uint32_t j = tid; j < cnt; j += SEG_BLOCK) {
    kout[s + j] = KeyOps<K>::add(sm.keys[j], base);
    if (HAS_VAL) vout[s + j] = sm.vals[j];
  }
}

template <class K, int ITEMS, int TILE_T, int RANK>
__global__ __launch_bounds__(SEG_BLOCK, 2) void k_seg_rle(
    const K *__restrict__ kin, K *__restrict__ uniq, uint32_t *__restrict__ mult, uint64_t n, int low_bits,
    int key_bits, uint64_t *status, uint32_t *ticket, uint32_t epoch, uint32_t spin_limit, uint32_t *err,
    uint32_t *oversize, uint32_t *total) {
  using S = SegSortSmem<K, false, ITEMS>;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  S &sm = *reinterpret_cast<S *>(smem_raw);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int i = tid; i < S::WARPS * RADIX; i += SEG_BLOCK) (&sm.whist[0][0])[i] = 0;
  for (int i = tid; i < S::WARPS * (RADIX + 1); i += SEG_BLOCK) (&sm.match[0][0])[i] = 0;
  if (tid == 0) {
    sm.tile = atomicAdd(ticket, 1u);
    sm.fail = 0;
  }
  __syncthreads();
  const uint32_t tile = sm.tile;
  const uint64_t num_tiles = (n + TILE_T - 1) / TILE_T;
  if (!seg_setup<K, TILE_T>(sm, kin, n, low_bits, key_bits, tile, oversize)) {
    // successors must still find this tile's word in their look-back
    if (tid == 0) st_relaxed(status + tile, lb_word(epoch, tile == 0 ? LB_INCLUSIVE : LB_AGGREGATE, 0));
    return;
  }
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
  const uint32_t excl = tile_prefix(status, tile, count, epoch, spin_limit, err, &sm.excl);
#pragma unroll
  for (int i = 0; i < ITEMS; i++) {
    if (head[i]) {
      const uint32_t j = (uint32_t)i * SEG_BLOCK + tid;
      uniq[excl + rank[i]] = KeyOps<K>::add(sm.keys[j], base);
      mult[excl + rank[i]] = sm.hpos[rank[i] + 1] - j;
    }
  }
  if (tile + 1 == num_tiles && tid == 0) *total = excl + count;
}

}  // namespace dbg
