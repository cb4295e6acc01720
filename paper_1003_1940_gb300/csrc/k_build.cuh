// k_build.cuh -- kernels of the sort-based construction (Section 3,
// BiConstruct STEP-1..4) and the pipeline that runs them, templated on the
// key width: uint64_t for k <= 31 ((k+1)-mers of <= 64 bits), Key128 above.
//
// Data layout in HBM for one build (N edge instances, E unique edges):
//   reads    ASCII, back to back                          total_bases bytes
//   packed   2-bit codes, base i at bits 63-2(i%32) of word i/32 (MSB first)
//   base_off / edge_off  per-read exclusive prefix of L and max(0, L-k)
//   keys     N canonical (k+1)-mer keys, double-buffered for the radix sort
//   uniq, headpos        E unique keys and the index of each run's head
//   records  2E (+ reads of length k) node keys + u32 payload (e<<1|role),
//            double-buffered for the radix sort
// and the graph's own arrays (node keys, edge keys, src, dst, orient, mult,
// row_ptr, adjacency).
#pragma once

#include <algorithm>
#include <cstdint>
#include <type_traits>

#include "dbg_device.cuh"
#include "dbg_internal.h"

namespace dbg {

constexpr int RADIX_BITS = 8;
constexpr int RADIX = 1 << RADIX_BITS;
constexpr int MAX_PASSES = 16;             // 128-bit keys / 8-bit digits
constexpr uint32_t REC_NONE = 0xffffffffu;  // payload of a node record that is not an edge end

// ---------------------------------------------------------------------------
// small block-wide helpers
// ---------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ T warp_incl_scan(T v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T u = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += u;
  }
  return v;
}

// Exclusive scan of one value per thread over the first 256 threads of the
// block (all threads must call it).  `tmp` holds 8 entries.
__device__ __forceinline__ uint32_t block_excl_scan_256(uint32_t v, uint32_t *tmp) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  uint32_t incl = warp_incl_scan(v);
  if (tid < 256 && lane == 31) tmp[warp] = incl;
  __syncthreads();
  uint32_t add = 0;
  if (tid < 256)
    for (int w = 0; w < warp; w++) add += tmp[w];
  __syncthreads();
  return add + incl - v;
}

// ---------------------------------------------------------------------------
// read offsets: base_off[r] = sum of L before r, edge_off[r] = sum of
// max(0, L - k) before r, plus the number of reads of length exactly k.
// Three phases: per-tile sums, one-block scan of the tile sums, per-tile
// exclusive scan.  All values are 64-bit.
// ---------------------------------------------------------------------------
constexpr int OFF_BLOCK = 256, OFF_ITEMS = 16, OFF_TILE = OFF_BLOCK * OFF_ITEMS;

struct Sum3 {
  uint64_t bases, edges, iso;
};

__device__ __forceinline__ Sum3 warp_reduce3(Sum3 s) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s.bases += __shfl_xor_sync(0xffffffffu, s.bases, o);
    s.edges += __shfl_xor_sync(0xffffffffu, s.edges, o);
    s.iso += __shfl_xor_sync(0xffffffffu, s.iso, o);
  }
  return s;
}

static __global__ void k_read_tile_sums(const uint32_t *__restrict__ len, uint64_t n, uint32_t k,
                                 Sum3 *__restrict__ tile_sums) {
  __shared__ Sum3 part[OFF_BLOCK / 32];
  const uint64_t base = (uint64_t)blockIdx.x * OFF_TILE;
  Sum3 s{0, 0, 0};
  for (int i = 0; i < OFF_ITEMS; i++) {
    uint64_t r = base + (uint64_t)i * OFF_BLOCK + threadIdx.x;
    if (r < n) {
      uint32_t L = len[r];
      s.bases += L;
      s.edges += L > k ? L - k : 0;
      s.iso += L == k;
    }
  }
  s = warp_reduce3(s);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    Sum3 t{0, 0, 0};
    for (int w = 0; w < OFF_BLOCK / 32; w++) {
      t.bases += part[w].bases; t.edges += part[w].edges; t.iso += part[w].iso;
    }
    tile_sums[blockIdx.x] = t;
  }
}

__device__ __forceinline__ Sum3 add3(Sum3 a, Sum3 b) { return Sum3{a.bases + b.bases, a.edges + b.edges, a.iso + b.iso}; }

__device__ __forceinline__ Sum3 warp_incl_scan3(Sum3 v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const Sum3 t{__shfl_up_sync(0xffffffffu, v.bases, o), __shfl_up_sync(0xffffffffu, v.edges, o),
                 __shfl_up_sync(0xffffffffu, v.iso, o)};
    if (lane >= o) v = add3(v, t);
  }
  return v;
}

// one block: exclusive scan of the tile sums in place, blockDim.x at a time
// (warp scans, then a scan of the warp totals); totals -> totals[0..2]
static __global__ void k_scan_tile_sums(Sum3 *tile_sums, uint32_t num_tiles, uint64_t *totals,
                                 uint64_t *base_off, uint64_t *edge_off, uint64_t n) {
  __shared__ Sum3 wsum[32];
  __shared__ Sum3 carry;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  if (threadIdx.x == 0) carry = Sum3{0, 0, 0};
  __syncthreads();
  for (uint32_t start = 0; start < num_tiles; start += blockDim.x) {
    const uint32_t i = start + threadIdx.x;
    const Sum3 v = i < num_tiles ? tile_sums[i] : Sum3{0, 0, 0};
    const Sum3 inc = warp_incl_scan3(v);
    if (lane == 31) wsum[warp] = inc;
    __syncthreads();
    if (warp == 0) {
      const Sum3 t = lane < nwarps ? wsum[lane] : Sum3{0, 0, 0};
      const Sum3 ti = warp_incl_scan3(t);
      if (lane < nwarps) wsum[lane] = Sum3{ti.bases - t.bases, ti.edges - t.edges, ti.iso - t.iso};
    }
    __syncthreads();
    const Sum3 before = add3(carry, wsum[warp]);
    const Sum3 excl = Sum3{before.bases + inc.bases - v.bases, before.edges + inc.edges - v.edges,
                           before.iso + inc.iso - v.iso};
    if (i < num_tiles) tile_sums[i] = excl;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry = add3(excl, v);
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    totals[0] = carry.bases;
    totals[1] = carry.edges;
    totals[2] = carry.iso;
    base_off[n] = carry.bases;
    edge_off[n] = carry.edges;
  }
}

static __global__ void k_read_offsets(const uint32_t *__restrict__ len, uint64_t n, uint32_t k,
                               const Sum3 *__restrict__ tile_sums, uint64_t *__restrict__ base_off,
                               uint64_t *__restrict__ edge_off) {
  // blocked: thread t owns reads [base + t*ITEMS, base + (t+1)*ITEMS)
  const uint64_t base = (uint64_t)blockIdx.x * OFF_TILE + (uint64_t)threadIdx.x * OFF_ITEMS;
  uint32_t L[OFF_ITEMS];
  uint64_t sb = 0, se = 0;
  for (int i = 0; i < OFF_ITEMS; i++) {
    uint64_t r = base + i;
    L[i] = r < n ? len[r] : 0;
    sb += L[i];
    se += L[i] > k ? L[i] - k : 0;
  }
  // block exclusive scans of the per-thread sums, in 64 bits
  __shared__ uint64_t wsum_b[OFF_BLOCK / 32], wsum_e[OFF_BLOCK / 32];
  uint64_t ib = warp_incl_scan(sb), ie = warp_incl_scan(se);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 31) { wsum_b[warp] = ib; wsum_e[warp] = ie; }
  __syncthreads();
  uint64_t ab = 0, ae = 0;
  for (int w = 0; w < warp; w++) { ab += wsum_b[w]; ae += wsum_e[w]; }
  uint64_t ob = tile_sums[blockIdx.x].bases + ab + ib - sb;
  uint64_t oe = tile_sums[blockIdx.x].edges + ae + ie - se;
  for (int i = 0; i < OFF_ITEMS; i++) {
    uint64_t r = base + i;
    if (r < n) {
      base_off[r] = ob;
      edge_off[r] = oe;
    }
    ob += L[i];
    oe += L[i] > k ? L[i] - k : 0;
  }
}

// ---------------------------------------------------------------------------
// K1 pack: ASCII -> 2-bit codes, 32 bases per 64-bit word.  code(c) =
// ((c >> 1) ^ (c >> 2)) & 3 maps 'A','C','G','T' (0x41,0x43,0x47,0x54) to
// 0,1,2,3; any other byte sets ERR_BAD_BASE.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t pack4(uint32_t x, bool &ok) {
  uint32_t okm = __vcmpeq4(x, 0x41414141u) | __vcmpeq4(x, 0x43434343u) |
                 __vcmpeq4(x, 0x47474747u) | __vcmpeq4(x, 0x54545454u);
  ok = ok && (okm == 0xffffffffu);
  uint32_t c = ((x >> 1) ^ (x >> 2)) & 0x03030303u;
  // byte 0 holds the first base; it goes to the most significant position
  return ((c & 3u) << 6) | (((c >> 8) & 3u) << 4) | (((c >> 16) & 3u) << 2) | ((c >> 24) & 3u);
}

static __global__ void k_pack(const uint8_t *__restrict__ ascii, uint64_t total, uint64_t *__restrict__ packed,
                       uint64_t nwords, uint32_t *err) {
  const bool aligned = (reinterpret_cast<uintptr_t>(ascii) & 15u) == 0;
  for (uint64_t w = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; w < nwords;
       w += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t b0 = w * 32;
    uint64_t word = 0;
    bool ok = true;
    if (aligned && b0 + 32 <= total) {
      const uint4 *p = reinterpret_cast<const uint4 *>(ascii + b0);
      uint4 a = __ldg(p), b = __ldg(p + 1);
      uint32_t v[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
#pragma unroll
      for (int i = 0; i < 8; i++) word = (word << 8) | pack4(v[i], ok);
    } else {
      for (int i = 0; i < 32; i++) {
        uint64_t b = b0 + i;
        uint32_t code = 0;
        if (b < total) {
          uint8_t c = ascii[b];
          bool good = c == 'A' || c == 'C' || c == 'G' || c == 'T';
          ok = ok && good;
          code = ((c >> 1) ^ (c >> 2)) & 3u;
        }
        word = (word << 2) | code;
      }
    }
    packed[w] = word;
    if (!ok) atomicOr(err, ERR_BAD_BASE);
  }
}

// The m bases starting at base position p, in the low 2m bits.
template <class K> __device__ __forceinline__ K load_window(const uint64_t *packed, uint64_t p, int m);

template <>
__device__ __forceinline__ uint64_t load_window<uint64_t>(const uint64_t *packed, uint64_t p, int m) {
  const uint64_t w = p >> 5;
  const int o = (int)(p & 31) * 2;
  uint64_t a = __ldg(packed + w), b = __ldg(packed + w + 1);
  uint64_t v = o ? (a << o) | (b >> (64 - o)) : a;
  return v >> (64 - 2 * m);
}

template <>
__device__ __forceinline__ Key128 load_window<Key128>(const uint64_t *packed, uint64_t p, int m) {
  const uint64_t w = p >> 5;
  const int o = (int)(p & 31) * 2;
  uint64_t a = __ldg(packed + w), b = __ldg(packed + w + 1), c = __ldg(packed + w + 2);
  uint64_t hi = o ? (a << o) | (b >> (64 - o)) : a;
  uint64_t lo = o ? (b << o) | (c >> (64 - o)) : b;
  return KeyOps<Key128>::shr(Key128{hi, lo}, 128 - 2 * m);
}

// ---------------------------------------------------------------------------
// K2 emit (STEP-1): key edge_off[r] + j of read r is the canonical (k+1)-mer
// min(z, revcomp z) of z = r[j .. j+k].  The block also accumulates the
// digit histograms of the sort's global radix passes (one upfront histogram
// for all of them, as in onesweep).
// ---------------------------------------------------------------------------
constexpr int EMIT_BLOCK = 256, EMIT_ITEMS = 8, EMIT_TILE = EMIT_BLOCK * EMIT_ITEMS;

__device__ __forceinline__ uint64_t last_le(const uint64_t *__restrict__ a, uint64_t lo, uint64_t hi,
                                            uint64_t x) {
  // largest i in [lo, hi) with a[i] <= x (a nondecreasing, a[lo] <= x)
  while (hi - lo > 1) {
    uint64_t mid = lo + (hi - lo) / 2;
    if (__ldg(a + mid) <= x) lo = mid; else hi = mid;
  }
  return lo;
}

template <class K>
__global__ __launch_bounds__(EMIT_BLOCK) void k_emit(const uint64_t *__restrict__ packed,
                                                     const uint64_t *__restrict__ base_off,
                                                     const uint64_t *__restrict__ edge_off, uint64_t n_reads,
                                                     uint32_t k, K *__restrict__ keys, int first, int passes,
                                                     unsigned long long *__restrict__ hist,
                                                     const uint64_t *__restrict__ krange,
                                                     uint32_t *__restrict__ read_of = nullptr) {
  // Every warp takes a contiguous, 32-aligned range of the keys to emit
  // (all of the N edge instances, or [krange[0], krange[1]) of them when
  // krange is given), so lanes stay busy across read ends and every
  // warp-wide store writes 32 consecutive keys.  A lane follows the
  // read that holds its key: one binary search per warp, then a step to the
  // next read when the key passes the current one's end.  The digit
  // histograms of passes [first, passes) are accumulated on the way.
  __shared__ uint32_t s_hist[MAX_PASSES * RADIX];
  for (int i = threadIdx.x; i < passes * RADIX; i += EMIT_BLOCK) s_hist[i] = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const uint64_t warps = (uint64_t)gridDim.x * (EMIT_BLOCK / 32);
  const uint64_t wid = (uint64_t)blockIdx.x * (EMIT_BLOCK / 32) + (threadIdx.x >> 5);
  const int m = (int)k + 1;
  const int G = passes - first;  // histogrammed passes
  uint32_t *hbase = s_hist + first * RADIX;
  const uint64_t lo = krange ? krange[0] : 0, hi = krange ? krange[1] : __ldg(edge_off + n_reads);
  const uint64_t per = ((hi - lo + warps - 1) / warps + 31) & ~31ull;
  const uint64_t a = lo + wid * per, b = min(a + per, hi);
  if (a < b) {
    // the read holding key a + lane: the last read starting at or before a,
    // then forward (reads without keys are stepped over)
    uint64_t r = last_le(edge_off, 0, n_reads, a);
    uint64_t e_hi = __ldg(edge_off + r + 1), pos = __ldg(base_off + r) - __ldg(edge_off + r);
    for (uint64_t i = a + lane; i < b; i += 32) {
      while (i >= e_hi) {
        r++;
        const uint64_t e_lo = e_hi;
        e_hi = __ldg(edge_off + r + 1);
        pos = __ldg(base_off + r) - e_lo;
      }
      const K z = load_window<K>(packed, pos + i, m);
      const K key = kmin(z, revcomp(z, m));
      keys[i] = key;
      if (read_of) read_of[i] = (uint32_t)r;
      if (G <= 4) {
        // the histogrammed digits are the low bytes of one shifted word
        const uint32_t w = (uint32_t)KeyOps<K>::words_lo(KeyOps<K>::shr(key, first * RADIX_BITS));
#pragma unroll
        for (int g = 0; g < 4; g++)
          if (g < G) atomicAdd(hbase + g * RADIX + ((w >> (8 * g)) & 0xffu), 1u);
      } else {
        for (int ps = first; ps < passes; ps++)
          atomicAdd(&s_hist[ps * RADIX + KeyOps<K>::digit(key, ps * RADIX_BITS, RADIX_BITS)], 1u);
      }
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < passes * RADIX; i += EMIT_BLOCK)
    if (s_hist[i]) atomicAdd(hist + i, (unsigned long long)s_hist[i]);
}

// Node multiplicities: the k-mers of read r (L >= k of them: L - k + 1) and,
// after their sort and run-length reduce, each distinct k-mer's count from
// the run heads (headpos[E] = the number of k-mers).
static __global__ void k_kmer_counts(const uint32_t *__restrict__ len, uint64_t n, uint32_t k,
                                     uint32_t *__restrict__ out) {
  for (uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (uint64_t)gridDim.x * blockDim.x)
    out[r] = len[r] >= k ? len[r] - k + 1 : 0u;
}

static __global__ void k_counts_from_heads(const uint32_t *__restrict__ headpos, uint64_t E,
                                           uint32_t *__restrict__ counts) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < E; i += (uint64_t)gridDim.x * blockDim.x)
    counts[i] = headpos[i + 1] - headpos[i];
}

// Distinct reads per node: over (k-mer key, read) records sorted by key with
// the reads of one key in ascending order, flag[i] = 1 where record i starts
// a key's run or holds another read than record i - 1.
template <class K>
__global__ void k_read_change_flags(const K *__restrict__ keys, const uint32_t *__restrict__ read_of, uint64_t M,
                                    uint32_t *__restrict__ flag) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += (uint64_t)gridDim.x * blockDim.x)
    flag[i] = (i == 0 || !KeyOps<K>::eq(keys[i], keys[i - 1]) || read_of[i] != read_of[i - 1]) ? 1u : 0u;
}

// counts[j] = flags in key run j = F[headpos[j + 1]] - F[headpos[j]] (F the
// exclusive scan of the flags, headpos the runs' first records, then M)
static __global__ void k_counts_between(const uint32_t *__restrict__ headpos, const uint64_t *__restrict__ F,
                                        uint64_t D, uint32_t *__restrict__ counts) {
  for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < D; j += (uint64_t)gridDim.x * blockDim.x)
    counts[j] = (uint32_t)(F[headpos[j + 1]] - F[headpos[j]]);
}

// Host reads arrive in chunks of `chunk` bases; once chunks 0..c are packed,
// the reads that end in them can be emitted.  bound[c + 1] = the first key
// of the first read that does not (edge_off of the number of reads whose
// bases all lie below (c + 1) * chunk), bound[0] = 0.
static __global__ void k_chunk_key_bounds(const uint64_t *__restrict__ base_off,
                                          const uint64_t *__restrict__ edge_off, uint64_t n, uint64_t chunk,
                                          uint32_t chunks, uint64_t *__restrict__ bound) {
  for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c <= chunks; c += gridDim.x * blockDim.x) {
    if (c == 0) {
      bound[0] = 0;
      continue;
    }
    const uint64_t end = (uint64_t)c * chunk;
    uint64_t lo = 0, hi = n;  // largest r in [0, n] with base_off[r] <= end
    while (lo < hi) {
      const uint64_t mid = hi - (hi - lo) / 2;
      if (base_off[mid] <= end) lo = mid;
      else hi = mid - 1;
    }
    bound[c] = edge_off[lo];
  }
}

// Digit histograms of passes [first, last) of n keys (any order): what the
// producer kernels skipped when only the high digits were to be sorted
// globally.
template <class K>
__global__ void k_digit_hist(const K *__restrict__ keys, uint64_t n, int first, int last,
                             unsigned long long *__restrict__ hist) {
  __shared__ uint32_t h[MAX_PASSES * RADIX];
  for (int i = threadIdx.x; i < MAX_PASSES * RADIX; i += blockDim.x) h[i] = 0;
  __syncthreads();
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    const K key = keys[i];
    for (int ps = first; ps < last; ps++) atomicAdd(&h[ps * RADIX + KeyOps<K>::digit(key, ps * RADIX_BITS, RADIX_BITS)], 1u);
  }
  __syncthreads();
  for (int i = first * RADIX + threadIdx.x; i < last * RADIX; i += blockDim.x)
    if (h[i]) atomicAdd(hist + i, (unsigned long long)h[i]);
}

// digit_base[p][d] = number of keys whose digit p is below d
static __global__ void k_digit_base(const unsigned long long *__restrict__ hist, uint64_t *__restrict__ digit_base) {
  __shared__ uint64_t s[RADIX];
  const int p = blockIdx.x, d = threadIdx.x;
  s[d] = hist[p * RADIX + d];
  __syncthreads();
  if (d == 0) {
    uint64_t run = 0;
    for (int i = 0; i < RADIX; i++) {
      uint64_t c = s[i];
      s[i] = run;
      run += c;
    }
  }
  __syncthreads();
  digit_base[p * RADIX + d] = s[d];
}

// ---------------------------------------------------------------------------
// TMA bulk copies and mbarriers (inline PTX)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// generic-proxy writes to shared memory before an async-proxy (TMA) write
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// one bulk copy global -> shared, completing `bytes` on the mbarrier
__device__ __forceinline__ void tma_load_bulk(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
// one bulk copy shared -> global in this thread's bulk async-group (both
// addresses 16-byte aligned, bytes a multiple of 16)
__device__ __forceinline__ void tma_store_bulk(void *dst, const void *src, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_u32(src)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// this thread's bulk stores have read their shared-memory source
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// this thread's bulk stores are complete
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
// bounded wait on an mbarrier phase; false when the limit was reached
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, uint32_t spin_limit) {
  for (uint32_t i = 0; i <= spin_limit; i++) {
    if (mbar_try_wait(bar, parity)) return true;
    if (i > 64) __nanosleep(64);
  }
  return false;
}

// ---------------------------------------------------------------------------
// First radix pass of keys without payload, as a partition: an LSD sort's
// first pass need not keep the input order of equal digits (any input order
// is as good as another), so each key takes its rank among the tile's keys
// of its digit from a shared-memory atomic add, the tile reserves its part of
// every digit's bucket with one global atomic add per digit (cursor[d]
// starts at the bucket's first index), and the keys are staged in shared
// memory by digit so that each run is written contiguously.  No tile waits
// for another.  The order within a bucket varies from run to run; the later
// passes are stable, so the sorted result does not.
//
// Persistent CTAs (a few per SM) take tiles t, t + grid, ...; while one
// tile is ranked and written, the next one arrives in the other buffer by
// one bulk copy (full tiles from a 16-byte aligned source; the last, partial
// tile by plain loads).  A tile is staged in its own buffer: its keys are in
// registers by then.
// ---------------------------------------------------------------------------
constexpr int PART_BLOCK = 256;
template <class K> struct PartShape { static constexpr int ITEMS = 32768 / (PART_BLOCK * (int)sizeof(K)); };

template <class K>
struct PartSmem {
  static constexpr int ITEMS = PartShape<K>::ITEMS, TILE = PART_BLOCK * ITEMS;
  K buf[2][TILE];
  unsigned long long gbase[RADIX];
  uint64_t bar[2];
  uint32_t cnt[RADIX], off[RADIX], tmp[8];
};

template <class K>
__global__ __launch_bounds__(PART_BLOCK, 3) void k_partition(const K *__restrict__ in, K *__restrict__ out,
                                                             uint64_t n, int shift,
                                                             unsigned long long *__restrict__ cursor,
                                                             uint32_t spin_limit, uint32_t *__restrict__ err) {
  using S = PartSmem<K>;
  constexpr int ITEMS = S::ITEMS, TILE = S::TILE;
  constexpr uint32_t BYTES = TILE * sizeof(K);
  extern __shared__ __align__(128) unsigned char smem_raw[];
  S &sm = *reinterpret_cast<S *>(smem_raw);
  const int tid = threadIdx.x;
  const uint64_t tiles = (n + TILE - 1) / TILE;
  const bool aligned = (reinterpret_cast<uintptr_t>(in) & 15) == 0;
  auto bulk_ok = [&](uint64_t t) { return aligned && (t + 1) * (uint64_t)TILE <= n; };
  if (tid == 0) {
    mbar_init(&sm.bar[0], 1);
    mbar_init(&sm.bar[1], 1);
    mbar_init_fence();
  }
  __syncthreads();
  uint64_t t = blockIdx.x;
  if (tid == 0 && t < tiles && bulk_ok(t)) {
    mbar_expect_tx(&sm.bar[0], BYTES);
    tma_load_bulk(sm.buf[0], in + t * TILE, BYTES, &sm.bar[0]);
  }
  uint32_t phase = 0;  // bit b: parity of buffer b's next completion
  for (int it = 0; t < tiles; t += gridDim.x, it++) {
    const int b = it & 1;
    const uint64_t tn = t + gridDim.x;
    const bool next_bulk = tn < tiles && bulk_ok(tn);
    if (tid == 0 && next_bulk) {
      mbar_expect_tx(&sm.bar[b ^ 1], BYTES);
      tma_load_bulk(sm.buf[b ^ 1], in + tn * TILE, BYTES, &sm.bar[b ^ 1]);
    }
    sm.cnt[tid] = 0;  // PART_BLOCK == RADIX
    const uint64_t base = t * TILE;
    const uint32_t tcount = n - base < (uint64_t)TILE ? (uint32_t)(n - base) : (uint32_t)TILE;
    const bool bulk = bulk_ok(t);
    if (bulk) {
      const bool ok = __syncthreads_and(mbar_wait(&sm.bar[b], (phase >> b) & 1u, spin_limit));
      phase ^= 1u << b;
      if (!ok) {
        // give up on this launch; first let the copies in flight land
        if (tid == 0) atomicOr(err, ERR_TIMEOUT);
        mbar_wait(&sm.bar[b], (phase >> b) & 1u ^ 1u, spin_limit);
        if (next_bulk) mbar_wait(&sm.bar[b ^ 1], (phase >> (b ^ 1)) & 1u, spin_limit);
        return;
      }
    } else {
      __syncthreads();
    }
    K key[ITEMS];
    uint32_t rd[ITEMS];  // rank << 8 | digit
#pragma unroll
    for (int i = 0; i < ITEMS; i++) {
      const uint32_t j = (uint32_t)i * PART_BLOCK + tid;
      if (j < tcount) {
        key[i] = bulk ? sm.buf[b][j] : in[base + j];
        const uint32_t d = KeyOps<K>::digit(key[i], shift, RADIX_BITS);
        rd[i] = (atomicAdd(&sm.cnt[d], 1u) << 8) | d;
      }
    }
    __syncthreads();
    const uint32_t c = sm.cnt[tid];
    sm.off[tid] = block_excl_scan_256(c, sm.tmp);
    const unsigned long long g = c ? atomicAdd(cursor + tid, (unsigned long long)c) : 0ull;
    __syncthreads();
#pragma unroll
    for (int i = 0; i < ITEMS; i++) {
      const uint32_t j = (uint32_t)i * PART_BLOCK + tid;
      if (j < tcount) sm.buf[b][sm.off[rd[i] & 0xffu] + (rd[i] >> 8)] = key[i];
    }
    sm.gbase[tid] = g;
    __syncthreads();
    for (uint32_t q = tid; q < tcount; q += PART_BLOCK) {
      const K k = sm.buf[b][q];
      const uint32_t d = KeyOps<K>::digit(k, shift, RADIX_BITS);
      const uint64_t dst = sm.gbase[d] + (q - sm.off[d]);
      if (dst >= n) {  // only reachable if the digit counts were inconsistent
        atomicOr(err, ERR_INTERNAL);
        continue;
      }
      out[dst] = k;
    }
    // this buffer's next use is a bulk copy (async proxy) after these
    // generic-proxy accesses
    fence_proxy_async_smem();
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// K3 onesweep radix pass (Adinets & Merrill): one launch per 8-bit digit,
// one CTA per tile.  Tiles are taken in launch order from an atomic ticket,
// so every tile a tile waits for belongs to a CTA that is already running.
// Per tile:
//   1. load the keys (and payloads) -- LOAD_TMA: one TMA bulk copy into
//      shared memory completing on an mbarrier; else warp-striped coalesced
//      loads -- and rank each key among the equal digits of its warp, stably
//      (item order, then lane order), with warp-private digit counters.  The
//      peer lanes holding the same digit come from RANK_BALLOT (one ballot
//      per digit bit), RANK_ATOMIC (shared-memory atomicOr of lane bits) or
//      RANK_MATCH (the hardware match.any instruction);
//   2. publish the tile's per-digit counts, look back over predecessor tiles
//      for each digit's exclusive prefix, publish the inclusive prefix;
//   3. stage the keys in shared memory in digit order and write each digit's
//      run to digit_base[d] + prefix (contiguous, coalesced).
// ---------------------------------------------------------------------------
enum : int { RANK_BALLOT = 0, RANK_ATOMIC = 1, RANK_MATCH = 2 };

template <class K, bool HAS_VAL, int BLOCK, int ITEMS>
struct OnesweepSmem {
  static constexpr int WARPS = BLOCK / 32;
  static constexpr int TILE = BLOCK * ITEMS;
  K keys[TILE];
  uint32_t vals[HAS_VAL ? TILE : 1];
  uint32_t whist[WARPS][RADIX];
  uint32_t match[WARPS][RADIX + 1];
  uint32_t tile_start[RADIX];
  uint32_t early[RADIX];
  uint64_t gbase[RADIX];
  uint64_t bar;
  uint32_t tmp[8];
  uint32_t tile;
};

template <class K, bool HAS_VAL, int BLOCK, int ITEMS, int RANK, bool LOAD_TMA, int MIN_BLOCKS, bool EARLY,
          bool DIRECT = false, int LB = 1>
__global__ __launch_bounds__(BLOCK, MIN_BLOCKS) void k_onesweep(
    const K *__restrict__ kin, K *__restrict__ kout, const uint32_t *__restrict__ vin, uint32_t *__restrict__ vout,
    uint64_t n, int shift, const uint64_t *__restrict__ digit_base, uint64_t *__restrict__ status,
    uint32_t *ticket, uint32_t epoch, uint32_t spin_limit, uint32_t *err) {
  using S = OnesweepSmem<K, HAS_VAL, BLOCK, ITEMS>;
  constexpr int WARPS = S::WARPS;
  constexpr int TILE = S::TILE;
  static_assert(BLOCK >= RADIX, "one thread per digit");
  extern __shared__ __align__(128) unsigned char smem_raw[];
  S &sm = *reinterpret_cast<S *>(smem_raw);

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int i = tid; i < WARPS * RADIX; i += BLOCK) (&sm.whist[0][0])[i] = 0;
  if (RANK == RANK_ATOMIC)
    for (int i = tid; i < WARPS * (RADIX + 1); i += BLOCK) (&sm.match[0][0])[i] = 0;
  if (EARLY && tid < RADIX) sm.early[tid] = 0;
  if (tid == 0) {
    sm.tile = atomicAdd(ticket, 1u);
    if (LOAD_TMA) {
      mbar_init(&sm.bar, 1);
      mbar_init_fence();
    }
  }
  __syncthreads();
  const uint32_t tile = sm.tile;
  const uint64_t base = (uint64_t)tile * TILE;
  const uint32_t tile_n = (uint32_t)min((uint64_t)TILE, n - base);
  // a full tile of 16-byte aligned data arrives by one bulk copy
  const bool bulk = LOAD_TMA && tile_n == TILE &&
                    ((reinterpret_cast<uintptr_t>(kin) | (HAS_VAL ? reinterpret_cast<uintptr_t>(vin) : 0)) & 15) == 0;
  if (bulk) {
    if (tid == 0) {
      const uint32_t kb = TILE * sizeof(K), vb = HAS_VAL ? TILE * sizeof(uint32_t) : 0;
      mbar_expect_tx(&sm.bar, kb + vb);
      tma_load_bulk(sm.keys, kin + base, kb, &sm.bar);
      if (HAS_VAL) tma_load_bulk(sm.vals, vin + base, vb, &sm.bar);
    }
    if (!__syncthreads_and(mbar_wait(&sm.bar, 0, spin_limit))) {
      // give up on this launch; first let the copy in flight land (a CTA
      // must not retire with a bulk copy into its shared memory pending)
      if (tid == 0) atomicOr(err, ERR_TIMEOUT);
      mbar_wait(&sm.bar, 0, spin_limit);
      return;
    }
  }

  const int wofs = warp * 32 * ITEMS;
  K key[ITEMS];
  uint32_t val[ITEMS];
  uint32_t rank[ITEMS];
#pragma unroll
  for (int i = 0; i < ITEMS; i++) {
    const uint32_t li = wofs + i * 32 + lane;
    if (bulk) {
      key[i] = sm.keys[li];
      if (HAS_VAL) val[i] = sm.vals[li];
    } else if (li < tile_n) {
      key[i] = kin[base + li];
      if (HAS_VAL) val[i] = vin[base + li];
    } else {
      key[i] = KeyOps<K>::zero();
      val[i] = 0;
    }
  }
  // EARLY: count the tile's digits, publish, look back and publish the
  // inclusive prefix before ranking, so that successors never wait for
  // this tile's ranking
  uint32_t excl_early = 0;
  if (EARLY) {
#pragma unroll
    for (int i = 0; i < ITEMS; i++)
      if ((uint32_t)(wofs + i * 32 + lane) < tile_n)
        atomicAdd(&sm.early[KeyOps<K>::digit(key[i], shift, RADIX_BITS)], 1u);
    __syncthreads();
    if (tid < RADIX) {
      const uint32_t c = sm.early[tid];
      uint64_t *st = status + (size_t)tile * RADIX + tid;
      if (tile == 0) {
        st_relaxed(st, lb_word(epoch, LB_INCLUSIVE, c));
      } else {
        st_relaxed(st, lb_word(epoch, LB_AGGREGATE, c));
        excl_early = LB > 1 ? lookback_exclusive_batched<LB>(status + tid, RADIX, tile, epoch, spin_limit, err)
                            : lookback_exclusive(status + tid, RADIX, tile, epoch, spin_limit, err);
        st_relaxed(st, lb_word(epoch, LB_INCLUSIVE, excl_early + c));
      }
    }
  }
  const unsigned lt_mask = (1u << lane) - 1u;
#pragma unroll
  for (int i = 0; i < ITEMS; i++) {
    const bool valid = (uint32_t)(wofs + i * 32 + lane) < tile_n;
    // digit, or RADIX for slots past the end of the input
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
    // rank within the tile's digit run so far, with the digit in the low 9 bits
    rank[i] = ((before + __popc(peers & lt_mask)) << 9) | d;
    __syncwarp();
  }
  __syncthreads();

  uint32_t cnt = 0;
  if (tid < RADIX) {
#pragma unroll
    for (int w = 0; w < WARPS; w++) cnt += sm.whist[w][tid];
    if (!EARLY)
      st_relaxed(status + (size_t)tile * RADIX + tid, lb_word(epoch, tile == 0 ? LB_INCLUSIVE : LB_AGGREGATE, cnt));
  }
  const uint32_t tstart = block_excl_scan_256(cnt, sm.tmp);
  if (tid < RADIX) {
    // each warp's first slot for this digit in the tile's digit-ordered staging
    uint32_t run = tstart;
#pragma unroll
    for (int w = 0; w < WARPS; w++) {
      const uint32_t c = sm.whist[w][tid];
      sm.whist[w][tid] = run;
      run += c;
    }
    uint32_t excl = excl_early;
    if (!EARLY && tile > 0) {
      excl = LB > 1 ? lookback_exclusive_batched<LB>(status + tid, RADIX, tile, epoch, spin_limit, err)
                    : lookback_exclusive(status + tid, RADIX, tile, epoch, spin_limit, err);
      st_relaxed(status + (size_t)tile * RADIX + tid, lb_word(epoch, LB_INCLUSIVE, excl + cnt));
    }
    sm.gbase[tid] = digit_base[tid] + excl - tstart;
  }
  __syncthreads();

  if (DIRECT) {
    // each key straight from its register to its final position; the L2
    // merges the partial sectors of neighbouring keys before DRAM sees them
#pragma unroll
    for (int i = 0; i < ITEMS; i++) {
      const uint32_t d = rank[i] & 0x1ffu;
      if (d < RADIX) {
        const uint64_t dst = sm.gbase[d] + sm.whist[warp][d] + (rank[i] >> 9);
        if (dst >= n) {  // only reachable if the digit counts were inconsistent
          atomicOr(err, ERR_INTERNAL);
          continue;
        }
        kout[dst] = key[i];
        if (HAS_VAL) vout[dst] = val[i];
      }
    }
    return;
  }
  // stage in digit order (the tile's keys are all in registers now)
#pragma unroll
  for (int i = 0; i < ITEMS; i++) {
    const uint32_t d = rank[i] & 0x1ffu;
    if (d < RADIX) {
      const uint32_t p = sm.whist[warp][d] + (rank[i] >> 9);
      sm.keys[p] = key[i];
      if (HAS_VAL) sm.vals[p] = val[i];
    }
  }
  __syncthreads();
  for (uint32_t j = tid; j < tile_n; j += BLOCK) {
    const K kk = sm.keys[j];
    const uint32_t d = KeyOps<K>::digit(kk, shift, RADIX_BITS);
    const uint64_t dst = sm.gbase[d] + j;
    if (dst >= n) {  // only reachable if the digit counts were inconsistent
      atomicOr(err, ERR_INTERNAL);
      continue;
    }
    kout[dst] = kk;
    if (HAS_VAL) vout[dst] = sm.vals[j];
  }
}

// ---------------------------------------------------------------------------
// K3 onesweep pass, persistent form: MIN_BLOCKS CTAs per SM each loop over
// tiles taken from the atomic ticket.  Once a tile's inclusive prefix is
// published, the CTA takes its next ticket and starts that tile's bulk copy
// into its other buffer, so the copy lands while the current tile is staged
// (in its own buffer: its keys are in registers by then) and written.  A
// ticket is taken only by a CTA that holds no unpublished tile, so every
// look-back ends.  Ranking and look-back are those of k_onesweep.
// ---------------------------------------------------------------------------
// HB: bytes of a per-warp digit counter (2 halves the counters' shared
// memory; a tile holds fewer than 2^16 keys); the lane-mask rows exist for
// shared-memory atomicOr ranking only.
// BULK: each digit's run is written out by bulk copies (cp.async.bulk),
// which proceed while the CTA ranks its next tile.  A bulk copy moves whole
// 16-byte units between 16-byte aligned addresses, so the run of digit d is
// staged from slot place_d congruent to its first output index modulo ALIGN
// (the elements in 16 bytes of keys and of payloads): place_d lies in
// [start_d + (ALIGN-1) d, start_d + (ALIGN-1)(d+1)), start_d the run's
// unpadded start, so runs never overlap and the tile needs (ALIGN-1) * 256
// extra slots.
template <class K, bool HAS_VAL, int BLOCK, int ITEMS, int RANK = RANK_ATOMIC, int HB = 4, bool BULK = false>
struct OnesweepPSmem {
  static constexpr int WARPS = BLOCK / 32;
  static constexpr int TILE = BLOCK * ITEMS;
  static constexpr int ALIGN = !BULK ? 1 : HAS_VAL ? 4 : (sizeof(K) >= 16 ? 1 : 16 / (int)sizeof(K));
  static constexpr int SLOTS = TILE + (ALIGN - 1) * RADIX;
  static_assert(HB == 4 || (HB == 2 && SLOTS < 65536), "digit counters must hold a tile's keys");
  using Hist = std::conditional_t<HB == 2, uint16_t, uint32_t>;
  K keys[2][SLOTS];
  uint32_t vals[2][HAS_VAL ? SLOTS : 1];
  Hist whist[WARPS][RADIX];
  uint32_t match[RANK == RANK_ATOMIC ? WARPS : 1][RADIX + 1];
  uint64_t gbase[RADIX];
  uint64_t bar[2];
  uint32_t tmp[8];
  uint32_t tnext;
};

template <class K, bool HAS_VAL, int BLOCK, int ITEMS, int RANK, int MIN_BLOCKS, int LB, int HB = 4,
          bool BULK = false>
__global__ __launch_bounds__(BLOCK, MIN_BLOCKS) void k_onesweep_p(
    const K *__restrict__ kin, K *__restrict__ kout, const uint32_t *__restrict__ vin, uint32_t *__restrict__ vout,
    uint64_t n, int shift, const uint64_t *__restrict__ digit_base, uint64_t *__restrict__ status,
    uint32_t *ticket, uint32_t epoch, uint32_t spin_limit, uint32_t *err) {
  using S = OnesweepPSmem<K, HAS_VAL, BLOCK, ITEMS, RANK, HB, BULK>;
  using Hist = typename S::Hist;
  constexpr int WARPS = S::WARPS;
  constexpr int TILE = S::TILE;
  constexpr uint32_t KB = TILE * sizeof(K), VB = HAS_VAL ? TILE * sizeof(uint32_t) : 0;
  static_assert(BLOCK >= RADIX, "one thread per digit");
  extern __shared__ __align__(128) unsigned char smem_raw[];
  S &sm = *reinterpret_cast<S *>(smem_raw);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint64_t tiles = (n + TILE - 1) / TILE;
  const bool aligned =
      ((reinterpret_cast<uintptr_t>(kin) | (HAS_VAL ? reinterpret_cast<uintptr_t>(vin) : 0)) & 15) == 0;
  auto bulk_ok = [&](uint64_t t) { return aligned && (t + 1) * (uint64_t)TILE <= n; };
  auto issue = [&](uint64_t t, int b) {
    mbar_expect_tx(&sm.bar[b], KB + VB);
    tma_load_bulk(sm.keys[b], kin + t * TILE, KB, &sm.bar[b]);
    if (HAS_VAL) tma_load_bulk(sm.vals[b], vin + t * TILE, VB, &sm.bar[b]);
  };
  // bulk write-out needs 16-byte aligned outputs; else the runs are staged
  // unpadded and written by plain stores
  const bool bulk_out =
      BULK && ((reinterpret_cast<uintptr_t>(kout) | (HAS_VAL ? reinterpret_cast<uintptr_t>(vout) : 0)) & 15) == 0;
  constexpr uint32_t AL = (uint32_t)S::ALIGN;
  if (RANK == RANK_ATOMIC)
    for (int i = tid; i < WARPS * (RADIX + 1); i += BLOCK) (&sm.match[0][0])[i] = 0;
  if (tid == 0) {
    mbar_init(&sm.bar[0], 1);
    mbar_init(&sm.bar[1], 1);
    mbar_init_fence();
    const uint32_t t0 = atomicAdd(ticket, 1u);
    sm.tnext = t0;
    if (t0 < tiles && bulk_ok(t0)) issue(t0, 0);
  }
  __syncthreads();
  uint32_t tile = sm.tnext;
  uint32_t phase = 0;  // bit b: parity of buffer b's next completion
  for (int it = 0; tile < tiles; it++) {
    const int b = it & 1;
    for (int i = tid; i < WARPS * RADIX; i += BLOCK) (&sm.whist[0][0])[i] = 0;
    const uint64_t base = (uint64_t)tile * TILE;
    const uint32_t tile_n = n - base < (uint64_t)TILE ? (uint32_t)(n - base) : (uint32_t)TILE;
    const bool bulk = bulk_ok(tile);
    if (bulk) {
      const bool ok = __syncthreads_and(mbar_wait(&sm.bar[b], (phase >> b) & 1u, spin_limit));
      phase ^= 1u << b;
      if (!ok) {
        // give up on this launch; first let the copies in flight land
        if (tid == 0) atomicOr(err, ERR_TIMEOUT);
        mbar_wait(&sm.bar[b], ((phase >> b) & 1u) ^ 1u, spin_limit);
        if (BULK && tid < RADIX) bulk_wait_all();
        return;
      }
    } else {
      __syncthreads();
    }
    const int wofs = warp * 32 * ITEMS;
    K key[ITEMS];
    uint32_t val[ITEMS];
    uint32_t rank[ITEMS];
#pragma unroll
    for (int i = 0; i < ITEMS; i++) {
      const uint32_t li = wofs + i * 32 + lane;
      if (bulk) {
        key[i] = sm.keys[b][li];
        if (HAS_VAL) val[i] = sm.vals[b][li];
      } else if (li < tile_n) {
        key[i] = kin[base + li];
        if (HAS_VAL) val[i] = vin[base + li];
      } else {
        key[i] = KeyOps<K>::zero();
        val[i] = 0;
      }
    }
    const unsigned lt_mask = (1u << lane) - 1u;
#pragma unroll
    for (int i = 0; i < ITEMS; i++) {
      const bool valid = (uint32_t)(wofs + i * 32 + lane) < tile_n;
      const uint32_t d = valid ? KeyOps<K>::digit(key[i], shift, RADIX_BITS) : (uint32_t)RADIX;
      unsigned peers;
      if (RANK == RANK_MATCH) {
        peers = __match_any_sync(0xffffffffu, d);
      } else {
        atomicOr(&sm.match[warp][d], 1u << lane);
        __syncwarp();
        peers = sm.match[warp][d];
        __syncwarp();
        if (lane == __ffs(peers) - 1) sm.match[warp][d] = 0;
      }
      const int leader = __ffs(peers) - 1;
      uint32_t before = 0;
      if (lane == leader && valid) {
        before = sm.whist[warp][d];
        sm.whist[warp][d] = (Hist)(before + __popc(peers));
      }
      before = __shfl_sync(0xffffffffu, before, leader);
      rank[i] = ((before + __popc(peers & lt_mask)) << 9) | d;
      __syncwarp();
    }
    __syncthreads();
    uint32_t cnt = 0;
    if (tid < RADIX) {
#pragma unroll
      for (int w = 0; w < WARPS; w++) cnt += sm.whist[w][tid];
      st_relaxed(status + (size_t)tile * RADIX + tid, lb_word(epoch, tile == 0 ? LB_INCLUSIVE : LB_AGGREGATE, cnt));
    }
    const uint32_t tstart = block_excl_scan_256(cnt, sm.tmp);
    uint64_t gstart = 0;  // (thread d < 256) digit d's first output index in this tile
    uint32_t place = 0;   // and the slot its run is staged from
    if (tid < RADIX) {
      uint32_t excl = 0;
      if (tile > 0) {
        excl = LB > 1 ? lookback_exclusive_batched<LB>(status + tid, RADIX, tile, epoch, spin_limit, err)
                      : lookback_exclusive(status + tid, RADIX, tile, epoch, spin_limit, err);
        st_relaxed(status + (size_t)tile * RADIX + tid, lb_word(epoch, LB_INCLUSIVE, excl + cnt));
      }
      gstart = digit_base[tid] + excl;
      place = tstart;
      if (BULK && bulk_out)
        place = tstart + (AL - 1) * tid + (uint32_t)((gstart - tstart - (AL - 1) * tid) & (AL - 1));
      uint32_t run = place;
#pragma unroll
      for (int w = 0; w < WARPS; w++) {
        const uint32_t c = sm.whist[w][tid];
        sm.whist[w][tid] = (Hist)run;
        run += c;
      }
      sm.gbase[tid] = gstart - place;
      // the other buffer's bulk stores (the previous tile) have read it
      if (BULK) bulk_wait_read();
    }
    __syncthreads();
    // this tile's prefix is published: take the next ticket and start its
    // copy, which lands while this tile is staged and written
    if (tid == 0) {
      const uint32_t tn = atomicAdd(ticket, 1u);
      sm.tnext = tn;
      if (tn < tiles && bulk_ok(tn)) issue(tn, b ^ 1);
    }
#pragma unroll
    for (int i = 0; i < ITEMS; i++) {
      const uint32_t d = rank[i] & 0x1ffu;
      if (d < RADIX) {
        const uint32_t q = sm.whist[warp][d] + (rank[i] >> 9);
        sm.keys[b][q] = key[i];
        if (HAS_VAL) sm.vals[b][q] = val[i];
      }
    }
    if (BULK && bulk_out) {
      // the staged runs are read by the async proxy: thread d writes digit
      // d's run, its unaligned ends by plain stores and the rest by bulk
      // copies that complete while the next tile is ranked
      fence_proxy_async_smem();
      __syncthreads();
      if (tid < RADIX && cnt > 0) {
        if (gstart + cnt > n) {  // only reachable if the digit counts were inconsistent
          atomicOr(err, ERR_INTERNAL);
        } else {
          const uint32_t head = min(cnt, (uint32_t)((AL - (uint32_t)(gstart & (AL - 1))) & (AL - 1)));
          const uint32_t mid = (cnt - head) & ~(AL - 1);
          for (uint32_t j = 0; j < cnt; j++) {
            if (j == head && mid > 0) {
              tma_store_bulk(kout + gstart + head, &sm.keys[b][place + head], mid * (uint32_t)sizeof(K));
              if (HAS_VAL) tma_store_bulk(vout + gstart + head, &sm.vals[b][place + head], mid * 4u);
              j += mid - 1;
              continue;
            }
            kout[gstart + j] = sm.keys[b][place + j];
            if (HAS_VAL) vout[gstart + j] = sm.vals[b][place + j];
          }
          bulk_commit();
        }
      }
    } else {
      __syncthreads();
      for (uint32_t j = tid; j < tile_n; j += BLOCK) {
        const K kk = sm.keys[b][j];
        const uint32_t d = KeyOps<K>::digit(kk, shift, RADIX_BITS);
        const uint64_t dst = sm.gbase[d] + j;
        if (dst >= n) {  // only reachable if the digit counts were inconsistent
          atomicOr(err, ERR_INTERNAL);
          continue;
        }
        kout[dst] = kk;
        if (HAS_VAL) vout[dst] = sm.vals[b][j];
      }
    }
    // this buffer's next use is a bulk copy (async proxy) after these
    // generic-proxy accesses
    fence_proxy_async_smem();
    __syncthreads();
    tile = sm.tnext;
  }
  if (BULK && tid < RADIX) bulk_wait_all();
}

// ---------------------------------------------------------------------------
// K4 run-length reduce (STEP-2): unique keys of the sorted array and the
// index of the first element of each run, by a single pass with look-back.
// The last tile writes headpos[E] = n and E itself to *total.
// ---------------------------------------------------------------------------
constexpr int SCAN_BLOCK = 256, SCAN_ITEMS = 16, SCAN_TILE = SCAN_BLOCK * SCAN_ITEMS;

// Block-wide ranks of per-item flags in index order for the strided layout
// (item i of thread t at i*BLOCK + t).  Returns the tile's flag count;
// rank_out[i] = flags before item i of this thread within the tile.
template <int BLOCK, int ITEMS>
__device__ __forceinline__ uint32_t tile_flag_ranks(const bool (&flag)[ITEMS], uint32_t (&rank_out)[ITEMS],
                                                    uint32_t *s_cnt /* ITEMS*WARPS */) {
  constexpr int WARPS = BLOCK / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
#pragma unroll
  for (int i = 0; i < ITEMS; i++) {
    const unsigned b = __ballot_sync(0xffffffffu, flag[i]);
    rank_out[i] = __popc(b & lt);
    if (lane == 0) s_cnt[i * WARPS + warp] = __popc(b);
  }
  __syncthreads();
  if (warp == 0) {
    constexpr int PER = (ITEMS * WARPS + 31) / 32;
    uint32_t v[PER];
    uint32_t s = 0;
#pragma unroll
    for (int j = 0; j < PER; j++) {
      const int idx = lane * PER + j;
      v[j] = idx < ITEMS * WARPS ? s_cnt[idx] : 0;
      s += v[j];
    }
    const uint32_t incl = warp_incl_scan(s);
    uint32_t run = incl - s;
#pragma unroll
    for (int j = 0; j < PER; j++) {
      const int idx = lane * PER + j;
      if (idx < ITEMS * WARPS) s_cnt[idx] = run;
      run += v[j];
    }
    if (lane == 31) s_cnt[ITEMS * WARPS] = incl;
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < ITEMS; i++) rank_out[i] += s_cnt[i * WARPS + warp];
  return s_cnt[ITEMS * WARPS];
}

// warp 0 publishes the tile's count and looks back; returns the exclusive
// prefix to every thread through shared memory
__device__ __forceinline__ uint32_t tile_prefix(uint64_t *status, uint32_t tile, uint32_t count, uint32_t epoch,
                                                uint32_t spin_limit, uint32_t *err, uint32_t *s_slot) {
  if (threadIdx.x < 32) {
    uint32_t excl = 0;
    if (tile == 0) {
      if (threadIdx.x == 0) st_relaxed(status, lb_word(epoch, LB_INCLUSIVE, count));
    } else {
      if (threadIdx.x == 0) st_relaxed(status + tile, lb_word(epoch, LB_AGGREGATE, count));
      excl = lookback_exclusive_warp(status, tile, epoch, spin_limit, err);
      if (threadIdx.x == 0) st_relaxed(status + tile, lb_word(epoch, LB_INCLUSIVE, excl + count));
    }
    if (threadIdx.x == 0) *s_slot = excl;
  }
  __syncthreads();
  return *s_slot;
}

template <class K, int ITEMS = SCAN_ITEMS>
__global__ __launch_bounds__(SCAN_BLOCK) void k_rle(const K *__restrict__ keys, uint64_t n, K *__restrict__ uniq,
                                                    uint32_t *__restrict__ headpos, uint64_t *status,
                                                    uint32_t *ticket, uint32_t epoch, uint32_t spin_limit,
                                                    uint32_t *err, uint32_t *total) {
  constexpr int WARPS = SCAN_BLOCK / 32;
  constexpr int TILE = SCAN_BLOCK * ITEMS;
  __shared__ uint32_t s_cnt[ITEMS * WARPS + 1];
  __shared__ uint32_t s_tile, s_excl;
  if (threadIdx.x == 0) s_tile = atomicAdd(ticket, 1u);
  __syncthreads();
  const uint32_t tile = s_tile;
  const uint64_t base = (uint64_t)tile * TILE;
  K key[ITEMS];
  bool head[ITEMS];
  uint32_t rank[ITEMS];
#pragma unroll
  for (int i = 0; i < ITEMS; i++) {
    const uint64_t idx = base + (uint64_t)i * SCAN_BLOCK + threadIdx.x;
    head[i] = false;
    if (idx < n) {
      key[i] = keys[idx];
      head[i] = idx == 0 || !KeyOps<K>::eq(key[i], keys[idx - 1]);
    }
  }
  const uint32_t count = tile_flag_ranks<SCAN_BLOCK, ITEMS>(head, rank, s_cnt);
  const uint32_t excl = tile_prefix(status, tile, count, epoch, spin_limit, err, &s_excl);
#pragma unroll
  for (int i = 0; i < ITEMS; i++) {
    if (head[i]) {
      const uint64_t idx = base + (uint64_t)i * SCAN_BLOCK + threadIdx.x;
      const uint32_t pos = excl + rank[i];
      uniq[pos] = key[i];
      headpos[pos] = (uint32_t)idx;
    }
  }
  if (base + TILE >= n && threadIdx.x == 0) {
    headpos[excl + count] = (uint32_t)n;
    *total = excl + count;
  }
}

// Exclusive scan of u32 values with decoupled look-back; out is 64-bit.
// The last tile writes out[n] = total and *total.
static __global__ __launch_bounds__(SCAN_BLOCK) void k_scan_excl(const uint32_t *__restrict__ in, uint64_t n,
                                                          uint64_t *__restrict__ out, uint64_t *status,
                                                          uint32_t *ticket, uint32_t epoch, uint32_t spin_limit,
                                                          uint32_t *err, uint32_t *total) {
  constexpr int WARPS = SCAN_BLOCK / 32;
  __shared__ uint32_t s_w[WARPS * SCAN_ITEMS + 1];
  __shared__ uint32_t s_tile, s_excl;
  if (threadIdx.x == 0) s_tile = atomicAdd(ticket, 1u);
  __syncthreads();
  const uint32_t tile = s_tile;
  // blocked per thread: thread t owns [base + t*ITEMS, +ITEMS)
  const uint64_t base = (uint64_t)tile * SCAN_TILE + (uint64_t)threadIdx.x * SCAN_ITEMS;
  uint32_t v[SCAN_ITEMS];
  uint32_t sum = 0;
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; i++) {
    v[i] = base + i < n ? in[base + i] : 0u;
    sum += v[i];
  }
  const uint32_t incl = warp_incl_scan(sum);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 31) s_w[warp] = incl;
  __syncthreads();
  uint32_t wadd = 0, tile_total = 0;
  for (int w = 0; w < WARPS; w++) {
    if (w < warp) wadd += s_w[w];
    tile_total += s_w[w];
  }
  const uint32_t excl_tile = tile_prefix(status, tile, tile_total, epoch, spin_limit, err, &s_excl);
  uint64_t run = (uint64_t)excl_tile + wadd + incl - sum;
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; i++) {
    if (base + i < n) out[base + i] = run;
    run += v[i];
  }
  if ((uint64_t)(tile + 1) * SCAN_TILE >= n && threadIdx.x == 0) {
    out[n] = (uint64_t)excl_tile + tile_total;
    *total = excl_tile + tile_total;
  }
}

// ---------------------------------------------------------------------------
// K5 edge ends (STEP-1 decoding + STEP-3 collection).  The unique key z is
// the canonical (k+1)-mer; x = its first k bases, y = its last k bases.
// With x^, y^ their canonical forms and o = 1 where the k-mer is the
// negative strand, STEP-1's table gives (x^, y^, o1, o2) if x^ <= y^ and
// (y^, x^, not o2, not o1) otherwise.  Writes orient, mult, a copy of the
// key into the graph, and two node records per edge (payload e<<1 | role),
// and accumulates the digit histograms of the node sort (pass ps takes the
// 8 bits from 8 ps - adj up).  The multiplicity comes from the run heads
// (headpos) or directly from mult_in.  With `sides` (E < 2^29), each payload
// also carries the side of its own end (bit 30) and of the edge's other end
// (bit 31), for k_write_nodes to store per adjacency slot.
// ---------------------------------------------------------------------------

// Side of an edge end (0 = left, 1 = right): the src end (role 0) of
// (u, v, o1, o2) sits on u's right side if o1 = 0, else its left; the dst
// end (role 1) on v's left side if o2 = 0, else its right.
__device__ __forceinline__ uint32_t end_side(uint8_t orient, uint32_t role) {
  const uint32_t o1 = orient >> 1, o2 = orient & 1u;
  return role == 0 ? (o1 ? 0u : 1u) : (o2 ? 1u : 0u);
}

template <class K>
__global__ __launch_bounds__(EMIT_BLOCK) void k_endpoints(const K *__restrict__ uniq,
                                                          const uint32_t *__restrict__ headpos,
                                                          const uint32_t *__restrict__ mult_in, uint64_t E,
                                                          uint32_t k, K *__restrict__ edge_keys,
                                                          uint32_t *__restrict__ mult,
                                                          uint8_t *__restrict__ orient, K *__restrict__ rkeys,
                                                          uint32_t *__restrict__ rvals, int first, int passes,
                                                          unsigned long long *__restrict__ hist, int adj = 0,
                                                          bool sides = false) {
  __shared__ uint32_t s_hist[MAX_PASSES * RADIX];
  for (int i = threadIdx.x; i < passes * RADIX; i += EMIT_BLOCK) s_hist[i] = 0;
  __syncthreads();
  const int kk = (int)k;
  for (uint64_t e = (uint64_t)blockIdx.x * EMIT_TILE + threadIdx.x; e < min(E, (uint64_t)(blockIdx.x + 1) * EMIT_TILE);
       e += EMIT_BLOCK) {
    const K z = uniq[e];
    const K x = KeyOps<K>::shr(z, 2);
    const K y = KeyOps<K>::mask_low(z, 2 * kk);
    const K xh = kmin(x, revcomp(x, kk));
    const K yh = kmin(y, revcomp(y, kk));
    const uint32_t o1 = !KeyOps<K>::eq(x, xh), o2 = !KeyOps<K>::eq(y, yh);
    K s, d;
    uint32_t a, b;
    if (!KeyOps<K>::less(yh, xh)) { s = xh; d = yh; a = o1; b = o2; }
    else { s = yh; d = xh; a = !o2; b = !o1; }
    edge_keys[e] = z;
    const uint8_t o = (uint8_t)((a << 1) | b);
    orient[e] = o;
    mult[e] = headpos ? headpos[e + 1] - headpos[e] : mult_in[e];
    const uint32_t s0 = sides ? end_side(o, 0) : 0u, s1 = sides ? end_side(o, 1) : 0u;
    rkeys[2 * e] = s;
    rvals[2 * e] = (uint32_t)(e << 1) | s0 << 30 | s1 << 31;
    rkeys[2 * e + 1] = d;
    rvals[2 * e + 1] = (uint32_t)(e << 1) | 1u | s1 << 30 | s0 << 31;
    for (int ps = first; ps < passes; ps++) {
      atomicAdd(&s_hist[ps * RADIX + KeyOps<K>::digit(s, ps * RADIX_BITS - adj, RADIX_BITS)], 1u);
      atomicAdd(&s_hist[ps * RADIX + KeyOps<K>::digit(d, ps * RADIX_BITS - adj, RADIX_BITS)], 1u);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < passes * RADIX; i += EMIT_BLOCK)
    if (s_hist[i]) atomicAdd(hist + i, (unsigned long long)s_hist[i]);
}

// Reads of length exactly k: their k-mer is a node with no edge (Section 2
// takes every k-mer of the reads).  One record each, payload REC_NONE,
// appended after the edge ends.
template <class K>
__global__ void k_isolated(const uint64_t *__restrict__ packed, const uint64_t *__restrict__ base_off,
                           const uint32_t *__restrict__ len, uint64_t n, uint32_t k, K *__restrict__ rkeys,
                           uint32_t *__restrict__ rvals, uint32_t *slot, int first, int passes,
                           unsigned long long *__restrict__ hist, int adj = 0) {
  for (uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (uint64_t)gridDim.x * blockDim.x) {
    if (len[r] != k) continue;
    const K x = load_window<K>(packed, base_off[r], (int)k);
    const K xh = kmin(x, revcomp(x, (int)k));
    const uint32_t i = atomicAdd(slot, 1u);
    rkeys[i] = xh;
    rvals[i] = REC_NONE;
    for (int ps = first; ps < passes; ps++)
      atomicAdd(hist + ps * RADIX + KeyOps<K>::digit(xh, ps * RADIX_BITS - adj, RADIX_BITS), 1ull);
  }
}


// K7 neighbour of every adjacency slot: the edge's other end.
// (Eight slots per thread at a time: their edge words, then their
// gathers, then their stores.)
static __global__ void k_adj_nbr(const uint32_t *__restrict__ adj_edge, const uint8_t *__restrict__ adj_role,
                          const uint32_t *__restrict__ src, const uint32_t *__restrict__ dst, uint64_t n,
                          uint32_t *__restrict__ nbr) {
  constexpr int U = 8;
  const uint64_t step = (uint64_t)blockDim.x * U;
  for (uint64_t p0 = (uint64_t)blockIdx.x * step + threadIdx.x; p0 < n; p0 += (uint64_t)gridDim.x * step) {
    uint32_t e[U], v[U];
    uint8_t r[U];
#pragma unroll
    for (int u = 0; u < U; u++) {
      const uint64_t p = p0 + (uint64_t)u * blockDim.x;
      e[u] = p < n ? adj_edge[p] : 0u;
      r[u] = p < n ? adj_role[p] : 0;
    }
#pragma unroll
    for (int u = 0; u < U; u++)
      v[u] = p0 + (uint64_t)u * blockDim.x < n ? (r[u] ? __ldg(src + e[u]) : __ldg(dst + e[u])) : 0u;
#pragma unroll
    for (int u = 0; u < U; u++) {
      const uint64_t p = p0 + (uint64_t)u * blockDim.x;
      if (p < n) nbr[p] = v[u];
    }
  }
}

// node keys as 1 or 2 words; row_ptr shrink copies are plain memcpy

}  // namespace dbg

namespace dbg {

// ---------------------------------------------------------------------------
// Key-range buckets (the bucket path of dbg_build_bucketed).  A key's prefix
// is its top PREFIX_BITS bits (all its bits when it is shorter).
// ---------------------------------------------------------------------------
constexpr int PREFIX_BITS = 12;
constexpr int PREFIX_BINS = 1 << PREFIX_BITS;

template <class K>
__device__ __forceinline__ uint32_t key_prefix(const K &key, int key_bits) {
  const int pb = key_bits < PREFIX_BITS ? key_bits : PREFIX_BITS;
  return KeyOps<K>::digit(key, key_bits - pb, pb);
}

// Histogram of the prefixes of the canonical (k+1)-mer keys (one warp per read).
template <class K>
__global__ __launch_bounds__(EMIT_BLOCK) void k_emit_prefix_hist(const uint64_t *__restrict__ packed,
                                                                 const uint64_t *__restrict__ base_off,
                                                                 const uint64_t *__restrict__ edge_off,
                                                                 uint64_t n_reads, uint32_t k,
                                                                 unsigned long long *__restrict__ hist) {
  __shared__ uint32_t s_hist[PREFIX_BINS];
  for (int i = threadIdx.x; i < PREFIX_BINS; i += EMIT_BLOCK) s_hist[i] = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, m = (int)k + 1;
  const uint64_t warps = (uint64_t)gridDim.x * (EMIT_BLOCK / 32);
  for (uint64_t r = (uint64_t)blockIdx.x * (EMIT_BLOCK / 32) + (threadIdx.x >> 5); r < n_reads; r += warps) {
    const uint64_t e0 = __ldg(edge_off + r), cnt = __ldg(edge_off + r + 1) - e0, p0 = __ldg(base_off + r);
    for (uint64_t j = lane; j < cnt; j += 32) {
      const K z = load_window<K>(packed, p0 + j, m);
      atomicAdd(&s_hist[key_prefix(kmin(z, revcomp(z, m)), 2 * m)], 1u);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < PREFIX_BINS; i += EMIT_BLOCK)
    if (s_hist[i]) atomicAdd(hist + i, (unsigned long long)s_hist[i]);
}

// STEP-1 restricted to keys whose prefix lies in [lo, hi): the keys of one
// bucket, appended in any order (the sort that follows orders them), with
// the digit histograms of its radix passes.
template <class K>
__global__ __launch_bounds__(EMIT_BLOCK) void k_emit_range(const uint64_t *__restrict__ packed,
                                                           const uint64_t *__restrict__ base_off,
                                                           const uint64_t *__restrict__ edge_off, uint64_t n_reads,
                                                           uint32_t k, uint32_t lo, uint32_t hi,
                                                           K *__restrict__ keys, uint32_t *count, int passes,
                                                           unsigned long long *__restrict__ hist) {
  __shared__ uint32_t s_hist[MAX_PASSES * RADIX];
  for (int i = threadIdx.x; i < passes * RADIX; i += EMIT_BLOCK) s_hist[i] = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, m = (int)k + 1;
  const uint64_t warps = (uint64_t)gridDim.x * (EMIT_BLOCK / 32);
  for (uint64_t r = (uint64_t)blockIdx.x * (EMIT_BLOCK / 32) + (threadIdx.x >> 5); r < n_reads; r += warps) {
    const uint64_t e0 = __ldg(edge_off + r), cnt = __ldg(edge_off + r + 1) - e0, p0 = __ldg(base_off + r);
    for (uint64_t j0 = 0; j0 < cnt; j0 += 32) {
      const uint64_t j = j0 + lane;
      K key = KeyOps<K>::zero();
      bool in = false;
      if (j < cnt) {
        const K z = load_window<K>(packed, p0 + j, m);
        key = kmin(z, revcomp(z, m));
        const uint32_t pf = key_prefix(key, 2 * m);
        in = pf >= lo && pf < hi;
      }
      const unsigned b = __ballot_sync(0xffffffffu, in);
      if (!b) continue;
      uint32_t base = 0;
      if (lane == 0) base = atomicAdd(count, (uint32_t)__popc(b));
      base = __shfl_sync(0xffffffffu, base, 0);
      if (in) {
        keys[base + __popc(b & ((1u << lane) - 1u))] = key;
        for (int ps = 0; ps < passes; ps++)
          atomicAdd(&s_hist[ps * RADIX + KeyOps<K>::digit(key, ps * RADIX_BITS, RADIX_BITS)], 1u);
      }
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < passes * RADIX; i += EMIT_BLOCK)
    if (s_hist[i]) atomicAdd(hist + i, (unsigned long long)s_hist[i]);
}

// The two node keys (x^, y^) of an edge key, by STEP-1's table; orient.
template <class K>
__device__ __forceinline__ void edge_ends(const K &z, int k, K &s, K &d, uint32_t &orient) {
  const K x = KeyOps<K>::shr(z, 2);
  const K y = KeyOps<K>::mask_low(z, 2 * k);
  const K xh = kmin(x, revcomp(x, k));
  const K yh = kmin(y, revcomp(y, k));
  const uint32_t o1 = !KeyOps<K>::eq(x, xh), o2 = !KeyOps<K>::eq(y, yh);
  if (!KeyOps<K>::less(yh, xh)) {
    s = xh; d = yh; orient = (o1 << 1) | o2;
  } else {
    s = yh; d = xh; orient = ((!o2) << 1) | (!o1);
  }
}

// Edges of one bucket: key, multiplicity (from the run heads, or directly
// from mult_in) and orientation.
template <class K>
__global__ void k_edge_finish(const K *__restrict__ uniq, const uint32_t *__restrict__ headpos,
                              const uint32_t *__restrict__ mult_in, uint64_t E, uint32_t k,
                              K *__restrict__ edge_keys, uint32_t *__restrict__ mult, uint8_t *__restrict__ orient) {
  for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < E; e += (uint64_t)gridDim.x * blockDim.x) {
    const K z = uniq[e];
    K s, d;
    uint32_t o;
    edge_ends(z, (int)k, s, d, o);
    edge_keys[e] = z;
    orient[e] = (uint8_t)o;
    mult[e] = headpos ? headpos[e + 1] - headpos[e] : mult_in[e];
  }
}

// Histogram of the prefixes of both node keys of every edge, and of the
// k-mers of reads of length exactly k.
template <class K>
__global__ void k_node_prefix_hist(const K *__restrict__ edge_keys, uint64_t E, uint32_t k,
                                   unsigned long long *__restrict__ hist) {
  __shared__ uint32_t s_hist[PREFIX_BINS];
  for (int i = threadIdx.x; i < PREFIX_BINS; i += blockDim.x) s_hist[i] = 0;
  __syncthreads();
  for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < E; e += (uint64_t)gridDim.x * blockDim.x) {
    K s, d;
    uint32_t o;
    edge_ends(edge_keys[e], (int)k, s, d, o);
    atomicAdd(&s_hist[key_prefix(s, 2 * (int)k)], 1u);
    atomicAdd(&s_hist[key_prefix(d, 2 * (int)k)], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < PREFIX_BINS; i += blockDim.x)
    if (s_hist[i]) atomicAdd(hist + i, (unsigned long long)s_hist[i]);
}

// 1 for every edge end (slot 2e + role) whose node key prefix is in [lo, hi).
template <class K>
__global__ void k_flag_ends(const K *__restrict__ edge_keys, uint64_t E, uint32_t k, uint32_t lo, uint32_t hi,
                            uint32_t *__restrict__ flags) {
  for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < E; e += (uint64_t)gridDim.x * blockDim.x) {
    K s, d;
    uint32_t o;
    edge_ends(edge_keys[e], (int)k, s, d, o);
    const uint32_t ps = key_prefix(s, 2 * (int)k), pd = key_prefix(d, 2 * (int)k);
    flags[2 * e] = ps >= lo && ps < hi;
    flags[2 * e + 1] = pd >= lo && pd < hi;
  }
}

// The flagged edge ends as node records, in (e, role) order (positions from
// an exclusive scan of the flags), with the node-sort digit histograms.
template <class K>
__global__ void k_gather_ends(const K *__restrict__ edge_keys, uint64_t E, uint32_t k,
                              const uint32_t *__restrict__ flags, const uint64_t *__restrict__ pos,
                              K *__restrict__ rkeys, uint32_t *__restrict__ rvals, int passes,
                              unsigned long long *__restrict__ hist) {
  __shared__ uint32_t s_hist[MAX_PASSES * RADIX];
  for (int i = threadIdx.x; i < passes * RADIX; i += blockDim.x) s_hist[i] = 0;
  __syncthreads();
  for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < E; e += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t f0 = flags[2 * e], f1 = flags[2 * e + 1];
    if (!f0 && !f1) continue;
    K s, d;
    uint32_t o;
    edge_ends(edge_keys[e], (int)k, s, d, o);
    for (int role = 0; role < 2; role++) {
      if (!(role ? f1 : f0)) continue;
      const K nk = role ? d : s;
      const uint64_t p = pos[2 * e + role];
      rkeys[p] = nk;
      rvals[p] = (uint32_t)(e << 1) | (uint32_t)role;
      for (int ps = 0; ps < passes; ps++)
        atomicAdd(&s_hist[ps * RADIX + KeyOps<K>::digit(nk, ps * RADIX_BITS, RADIX_BITS)], 1u);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < passes * RADIX; i += blockDim.x)
    if (s_hist[i]) atomicAdd(hist + i, (unsigned long long)s_hist[i]);
}

// Reads of length exactly k whose k-mer prefix is in [lo, hi): one record
// each (payload REC_NONE), appended at rkeys + *slot.
template <class K>
__global__ void k_isolated_range(const uint64_t *__restrict__ packed, const uint64_t *__restrict__ base_off,
                                 const uint32_t *__restrict__ len, uint64_t n, uint32_t k, uint32_t lo, uint32_t hi,
                                 K *__restrict__ rkeys, uint32_t *__restrict__ rvals, uint32_t *slot, int passes,
                                 unsigned long long *__restrict__ hist) {
  for (uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (uint64_t)gridDim.x * blockDim.x) {
    if (len[r] != k) continue;
    const K x = load_window<K>(packed, base_off[r], (int)k);
    const K xh = kmin(x, revcomp(x, (int)k));
    const uint32_t pf = key_prefix(xh, 2 * (int)k);
    if (pf < lo || pf >= hi) continue;
    const uint32_t i = atomicAdd(slot, 1u);
    rkeys[i] = xh;
    rvals[i] = REC_NONE;
    for (int ps = 0; ps < passes; ps++)
      atomicAdd(hist + ps * RADIX + KeyOps<K>::digit(xh, ps * RADIX_BITS, RADIX_BITS), 1ull);
  }
}

// Copies a chunk of ASCII reads and packs it into the packed array at base
// position `at` (a multiple of 32).
static __global__ void k_pack_at(const uint8_t *__restrict__ ascii, uint64_t total, uint64_t *__restrict__ packed,
                          uint64_t word0, uint32_t *err) {
  const uint64_t nwords = (total + 31) / 32;
  for (uint64_t w = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; w < nwords; w += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t word = 0;
    bool ok = true;
    for (int i = 0; i < 32; i++) {
      const uint64_t b = w * 32 + i;
      uint32_t code = 0;
      if (b < total) {
        const uint8_t c = ascii[b];
        ok = ok && (c == 'A' || c == 'C' || c == 'G' || c == 'T');
        code = ((c >> 1) ^ (c >> 2)) & 3u;
      }
      word = (word << 2) | code;
    }
    packed[word0 + w] = word;
    if (!ok) atomicOr(err, ERR_BAD_BASE);
  }
}

}  // namespace dbg

namespace dbg {

// ---------------------------------------------------------------------------
// Reduce-then-scan forms of K4 and K6 (no look-back): a counting pass per
// tile, an exclusive scan of the tile counts, and a writing pass that
// recomputes the flags.  Layout of a tile: item i of thread t at
// i * SCAN_BLOCK + t.
// ---------------------------------------------------------------------------
constexpr int RS_ITEMS = 16, RS_TILE = SCAN_BLOCK * RS_ITEMS;

// previous element of item (i, t) in the strided layout: (i, t - 1), from
// the neighbouring lane or, for lane 0, from memory
template <class K>
__device__ __forceinline__ K prev_key(const K *keys, uint64_t idx, uint64_t n, const K &mine) {
  const int lane = threadIdx.x & 31;
  K p;
  if constexpr (sizeof(K) == 8) {
    p = __shfl_up_sync(0xffffffffu, mine, 1);
  } else {
    p.hi = __shfl_up_sync(0xffffffffu, mine.hi, 1);
    p.lo = __shfl_up_sync(0xffffffffu, mine.lo, 1);
  }
  if (lane == 0 && idx > 0 && idx <= n) p = keys[idx - 1];
  return p;
}

// heads per tile: counts[t] (and, when `vals` is given, edge-end records
// per tile in counts2[t])
template <class K>
__global__ __launch_bounds__(SCAN_BLOCK) void k_count_heads(const K *__restrict__ keys, const uint32_t *__restrict__ vals,
                                                            uint64_t n, uint32_t *__restrict__ counts,
                                                            uint32_t *__restrict__ counts2) {
  __shared__ uint32_t s_red[2][SCAN_BLOCK / 32];
  const uint64_t base = (uint64_t)blockIdx.x * RS_TILE;
  uint32_t c = 0, c2 = 0;
#pragma unroll 4
  for (int i = 0; i < RS_ITEMS; i++) {
    const uint64_t idx = base + (uint64_t)i * SCAN_BLOCK + threadIdx.x;
    const bool in = idx < n;
    const K k = in ? keys[idx] : KeyOps<K>::zero();
    const K p = prev_key(keys, idx, n, k);
    if (in && (idx == 0 || !KeyOps<K>::eq(k, p))) c++;
    if (vals && in && vals[idx] != REC_NONE) c2++;
  }
  c = __reduce_add_sync(0xffffffffu, c);
  c2 = __reduce_add_sync(0xffffffffu, c2);
  if ((threadIdx.x & 31) == 0) {
    s_red[0][threadIdx.x >> 5] = c;
    s_red[1][threadIdx.x >> 5] = c2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t a = 0, b = 0;
    for (int w = 0; w < SCAN_BLOCK / 32; w++) {
      a += s_red[0][w];
      b += s_red[1][w];
    }
    counts[blockIdx.x] = a;
    if (counts2) counts2[blockIdx.x] = b;
  }
}

// K4 writing pass: unique keys and run heads at the scanned tile offsets;
// the last tile writes headpos[E] = n.
template <class K>
__global__ __launch_bounds__(SCAN_BLOCK) void k_write_heads(const K *__restrict__ keys, uint64_t n,
                                                            const uint64_t *__restrict__ tile_off,
                                                            K *__restrict__ uniq, uint32_t *__restrict__ headpos) {
  constexpr int WARPS = SCAN_BLOCK / 32;
  __shared__ uint32_t s_cnt[RS_ITEMS * WARPS + 1];
  const uint64_t base = (uint64_t)blockIdx.x * RS_TILE;
  K key[RS_ITEMS];
  bool head[RS_ITEMS];
  uint32_t rank[RS_ITEMS];
#pragma unroll
  for (int i = 0; i < RS_ITEMS; i++) {
    const uint64_t idx = base + (uint64_t)i * SCAN_BLOCK + threadIdx.x;
    const bool in = idx < n;
    key[i] = in ? keys[idx] : KeyOps<K>::zero();
    const K p = prev_key(keys, idx, n, key[i]);
    head[i] = in && (idx == 0 || !KeyOps<K>::eq(key[i], p));
  }
  const uint32_t count = tile_flag_ranks<SCAN_BLOCK, RS_ITEMS>(head, rank, s_cnt);
  const uint64_t off = tile_off[blockIdx.x];
#pragma unroll
  for (int i = 0; i < RS_ITEMS; i++) {
    if (head[i]) {
      uniq[off + rank[i]] = key[i];
      headpos[off + rank[i]] = (uint32_t)(base + (uint64_t)i * SCAN_BLOCK + threadIdx.x);
    }
  }
  if (base + RS_TILE >= n && threadIdx.x == 0) headpos[off + count] = (uint32_t)n;
}

// K6 node IDs (STEP-3) + adjacency rows (STEP-4), the writing pass.  Over
// the node records sorted by key (stable, so edge ends precede isolated
// records within a node and are in (e, role) order): node ID = number of run
// heads up to the record minus one; adjacency slot = number of edge-end
// records before it -- from the scanned per-tile counts of run heads (hoff)
// and edge ends (eoff).  (base_v, base_slot) are added to the IDs and slots,
// for a node-key range built after others.  The last tile writes row_ptr[V].
//
// PART = true: instead of writing src[e] / dst[e] at random, the edge ends
// (e << 1 | role, node ID) are partitioned by e >> bshift into ends[] (bucket
// b at b << (bshift + 1): every edge has exactly two ends, so the buckets
// are full and dense), for k_scatter_ends to write with each bucket's part
// of src / dst resident in L2.
template <class K, bool PART>
__global__ __launch_bounds__(SCAN_BLOCK, 2) void k_write_nodes(
    const K *__restrict__ rkeys, const uint32_t *__restrict__ rvals, uint64_t R, const uint64_t *__restrict__ hoff,
    const uint64_t *__restrict__ eoff, K *__restrict__ node_keys, uint64_t *__restrict__ row_ptr,
    uint32_t *__restrict__ src, uint32_t *__restrict__ dst, uint32_t *__restrict__ adj_edge,
    uint8_t *__restrict__ adj_role, uint32_t base_v, uint64_t base_slot, uint64_t *__restrict__ ends,
    uint32_t *__restrict__ bucket_fill, int bshift, uint8_t *__restrict__ adj_side = nullptr) {
  constexpr int WARPS = SCAN_BLOCK / 32;
  __shared__ uint32_t s_cnt_h[RS_ITEMS * WARPS + 1], s_cnt_e[RS_ITEMS * WARPS + 1];
  __shared__ uint32_t s_bcnt[PART ? 256 : 1], s_bbase[PART ? 256 : 1];
  if (PART) s_bcnt[threadIdx.x] = 0;  // SCAN_BLOCK == 256 buckets at most
  const uint64_t base = (uint64_t)blockIdx.x * RS_TILE;
  K key[RS_ITEMS];
  uint32_t val[RS_ITEMS];
  bool head[RS_ITEMS], end[RS_ITEMS];
  uint32_t rh[RS_ITEMS], re[RS_ITEMS];
#pragma unroll
  for (int i = 0; i < RS_ITEMS; i++) {
    const uint64_t idx = base + (uint64_t)i * SCAN_BLOCK + threadIdx.x;
    const bool in = idx < R;
    key[i] = in ? rkeys[idx] : KeyOps<K>::zero();
    val[i] = in ? rvals[idx] : REC_NONE;
    const K p = prev_key(rkeys, idx, R, key[i]);
    head[i] = in && (idx == 0 || !KeyOps<K>::eq(key[i], p));
    end[i] = val[i] != REC_NONE;
  }
  tile_flag_ranks<SCAN_BLOCK, RS_ITEMS>(head, rh, s_cnt_h);
  tile_flag_ranks<SCAN_BLOCK, RS_ITEMS>(end, re, s_cnt_e);
  const uint64_t xh = hoff[blockIdx.x], xe = eoff[blockIdx.x];
#pragma unroll
  for (int i = 0; i < RS_ITEMS; i++) {
    const uint64_t idx = base + (uint64_t)i * SCAN_BLOCK + threadIdx.x;
    if (idx >= R) continue;
    const uint64_t id = xh + rh[i] + (head[i] ? 1u : 0u) - 1u;
    const uint64_t slot = xe + re[i];
    if (head[i]) {
      node_keys[id] = key[i];
      row_ptr[id] = base_slot + slot;
    }
    if (end[i]) {
      if (adj_side) {  // the two side bits on top of the payload
        adj_side[base_slot + slot] = (uint8_t)(val[i] >> 30);
        val[i] &= 0x3fffffffu;
      }
      const uint32_t e = val[i] >> 1, role = val[i] & 1u;
      adj_edge[base_slot + slot] = e;
      adj_role[base_slot + slot] = (uint8_t)role;
      if (PART) {
        rh[i] = (uint32_t)id;                           // keep the node ID
        re[i] = atomicAdd(&s_bcnt[e >> bshift], 1u);  // rank within the block's part of the bucket
      } else {
        (role ? dst : src)[e] = base_v + (uint32_t)id;
      }
    }
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) row_ptr[hoff[gridDim.x]] = base_slot + eoff[gridDim.x];
  if (PART) {
    __syncthreads();
    if (s_bcnt[threadIdx.x]) s_bbase[threadIdx.x] = atomicAdd(bucket_fill + threadIdx.x, s_bcnt[threadIdx.x]);
    __syncthreads();
#pragma unroll
    for (int i = 0; i < RS_ITEMS; i++) {
      const uint64_t idx = base + (uint64_t)i * SCAN_BLOCK + threadIdx.x;
      if (idx >= R || !end[i]) continue;
      const uint32_t b = (val[i] >> 1) >> bshift;
      ends[((uint64_t)b << (bshift + 1)) + s_bbase[b] + re[i]] = ((uint64_t)val[i] << 32) | (base_v + rh[i]);
    }
  }
}

// The same writing pass with persistent CTAs (two per SM) over the tiles t,
// t + grid, ...: while one tile is flagged, ranked and written, the next
// tile's records arrive by bulk copy in the other buffer (full tiles of
// 16-byte aligned arrays; the last tile by plain loads into the buffer).
template <class K>
struct WriteNodesSmem {
  static constexpr int WARPS = SCAN_BLOCK / 32;
  K keys[2][RS_TILE];
  uint32_t vals[2][RS_TILE];
  uint32_t cnt_h[RS_ITEMS * WARPS + 1], cnt_e[RS_ITEMS * WARPS + 1];
  uint32_t bcnt[256], bbase[256];
  uint64_t bar[2];
};

template <class K, bool PART>
__global__ __launch_bounds__(SCAN_BLOCK, 2) void k_write_nodes_p(
    const K *__restrict__ rkeys, const uint32_t *__restrict__ rvals, uint64_t R, const uint64_t *__restrict__ hoff,
    const uint64_t *__restrict__ eoff, K *__restrict__ node_keys, uint64_t *__restrict__ row_ptr,
    uint32_t *__restrict__ src, uint32_t *__restrict__ dst, uint32_t *__restrict__ adj_edge,
    uint8_t *__restrict__ adj_role, uint32_t base_v, uint64_t base_slot, uint64_t *__restrict__ ends,
    uint32_t *__restrict__ bucket_fill, int bshift, uint32_t spin_limit, uint32_t *__restrict__ err,
    uint8_t *__restrict__ adj_side = nullptr) {
  using S = WriteNodesSmem<K>;
  constexpr uint32_t KB = RS_TILE * sizeof(K), VB = RS_TILE * sizeof(uint32_t);
  extern __shared__ __align__(128) unsigned char smem_raw[];
  S &sm = *reinterpret_cast<S *>(smem_raw);
  const int tid = threadIdx.x;
  const uint64_t tiles = (R + RS_TILE - 1) / RS_TILE;
  const bool aligned = ((reinterpret_cast<uintptr_t>(rkeys) | reinterpret_cast<uintptr_t>(rvals)) & 15) == 0;
  auto bulk_ok = [&](uint64_t t) { return aligned && (t + 1) * (uint64_t)RS_TILE <= R; };
  auto issue = [&](uint64_t t, int b) {
    mbar_expect_tx(&sm.bar[b], KB + VB);
    tma_load_bulk(sm.keys[b], rkeys + t * RS_TILE, KB, &sm.bar[b]);
    tma_load_bulk(sm.vals[b], rvals + t * RS_TILE, VB, &sm.bar[b]);
  };
  if (tid == 0) {
    mbar_init(&sm.bar[0], 1);
    mbar_init(&sm.bar[1], 1);
    mbar_init_fence();
  }
  __syncthreads();
  uint64_t t = blockIdx.x;
  if (tid == 0 && t < tiles && bulk_ok(t)) issue(t, 0);
  uint32_t phase = 0;  // bit b: parity of buffer b's next completion
  for (int it = 0; t < tiles; t += gridDim.x, it++) {
    const int b = it & 1;
    const uint64_t tn = t + gridDim.x;
    const bool next_bulk = tn < tiles && bulk_ok(tn);
    if (tid == 0 && next_bulk) issue(tn, b ^ 1);
    if (PART) sm.bcnt[tid] = 0;  // SCAN_BLOCK == 256 buckets at most
    const uint64_t base = t * RS_TILE;
    const uint32_t tcount = R - base < (uint64_t)RS_TILE ? (uint32_t)(R - base) : (uint32_t)RS_TILE;
    if (bulk_ok(t)) {
      const bool ok = __syncthreads_and(mbar_wait(&sm.bar[b], (phase >> b) & 1u, spin_limit));
      phase ^= 1u << b;
      if (!ok) {
        // give up on this launch; first let the copies in flight land
        if (tid == 0) atomicOr(err, ERR_TIMEOUT);
        mbar_wait(&sm.bar[b], ((phase >> b) & 1u) ^ 1u, spin_limit);
        if (next_bulk) mbar_wait(&sm.bar[b ^ 1], (phase >> (b ^ 1)) & 1u, spin_limit);
        return;
      }
    } else {
      for (uint32_t j = tid; j < tcount; j += SCAN_BLOCK) {
        sm.keys[b][j] = rkeys[base + j];
        sm.vals[b][j] = rvals[base + j];
      }
      __syncthreads();
    }
    uint32_t val[RS_ITEMS];
    bool head[RS_ITEMS], end[RS_ITEMS];
    uint32_t rh[RS_ITEMS], re[RS_ITEMS];
#pragma unroll
    for (int i = 0; i < RS_ITEMS; i++) {
      const uint32_t j = (uint32_t)i * SCAN_BLOCK + tid;
      const bool in = j < tcount;
      val[i] = in ? sm.vals[b][j] : REC_NONE;
      bool h = false;
      if (in) {
        const K k = sm.keys[b][j];
        if (j > 0) h = !KeyOps<K>::eq(k, sm.keys[b][j - 1]);
        else h = base == 0 || !KeyOps<K>::eq(k, rkeys[base - 1]);
      }
      head[i] = h;
      end[i] = val[i] != REC_NONE;
    }
    tile_flag_ranks<SCAN_BLOCK, RS_ITEMS>(head, rh, sm.cnt_h);
    tile_flag_ranks<SCAN_BLOCK, RS_ITEMS>(end, re, sm.cnt_e);
    const uint64_t xh = hoff[t], xe = eoff[t];
#pragma unroll
    for (int i = 0; i < RS_ITEMS; i++) {
      const uint32_t j = (uint32_t)i * SCAN_BLOCK + tid;
      if (j >= tcount) continue;
      const uint64_t id = xh + rh[i] + (head[i] ? 1u : 0u) - 1u;
      const uint64_t slot = xe + re[i];
      if (head[i]) {
        node_keys[id] = sm.keys[b][j];
        row_ptr[id] = base_slot + slot;
      }
      if (end[i]) {
        if (adj_side) {  // the two side bits on top of the payload
          adj_side[base_slot + slot] = (uint8_t)(val[i] >> 30);
          val[i] &= 0x3fffffffu;
        }
        const uint32_t e = val[i] >> 1, role = val[i] & 1u;
        adj_edge[base_slot + slot] = e;
        adj_role[base_slot + slot] = (uint8_t)role;
        if (PART) {
          rh[i] = (uint32_t)id;                             // keep the node ID
          re[i] = atomicAdd(&sm.bcnt[e >> bshift], 1u);  // rank within the tile's part of the bucket
        } else {
          (role ? dst : src)[e] = base_v + (uint32_t)id;
        }
      }
    }
    if (t == tiles - 1 && tid == 0) row_ptr[hoff[tiles]] = base_slot + eoff[tiles];
    if (PART) {
      __syncthreads();
      if (sm.bcnt[tid]) sm.bbase[tid] = atomicAdd(bucket_fill + tid, sm.bcnt[tid]);
      __syncthreads();
#pragma unroll
      for (int i = 0; i < RS_ITEMS; i++) {
        const uint32_t j = (uint32_t)i * SCAN_BLOCK + tid;
        if (j >= tcount || !end[i]) continue;
        const uint32_t bk = (val[i] >> 1) >> bshift;
        ends[((uint64_t)bk << (bshift + 1)) + sm.bbase[bk] + re[i]] = ((uint64_t)val[i] << 32) | (base_v + rh[i]);
      }
    }
    // this buffer's next use is a bulk copy (async proxy) after these
    // generic-proxy accesses
    fence_proxy_async_smem();
    __syncthreads();
  }
}

// src[e] / dst[e] from the partitioned edge ends, swept in order so that the
// part of src / dst being written stays in L2.
// Each thread loads STREAM_U entries before it stores any, so that many
// loads are in flight.
constexpr int STREAM_U = 8;

static __global__ void k_scatter_ends(const uint64_t *__restrict__ ends, uint64_t n, uint32_t *__restrict__ src,
                                      uint32_t *__restrict__ dst) {
  const uint64_t step = (uint64_t)blockDim.x * STREAM_U;
  for (uint64_t i0 = (uint64_t)blockIdx.x * step + threadIdx.x; i0 < n; i0 += (uint64_t)gridDim.x * step) {
    uint64_t w[STREAM_U];
#pragma unroll
    for (int u = 0; u < STREAM_U; u++) {
      const uint64_t i = i0 + (uint64_t)u * blockDim.x;
      w[u] = i < n ? ends[i] : 0;
    }
#pragma unroll
    for (int u = 0; u < STREAM_U; u++) {
      if (i0 + (uint64_t)u * blockDim.x >= n) break;
      const uint32_t v = (uint32_t)(w[u] >> 32);
      ((v & 1u) ? dst : src)[v >> 1] = (uint32_t)w[u];
    }
  }
}

}  // namespace dbg
