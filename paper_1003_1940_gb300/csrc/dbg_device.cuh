// dbg_device.cuh -- device-side building blocks shared by the kernels:
// 2-bit k-mer keys of one or two 64-bit words, reverse complement, digit
// extraction, and the decoupled look-back used by the single-pass scans.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace dbg {

// ---------------------------------------------------------------------------
// device error word bits (OR-ed into ctx->d_err, read once per call)
// ---------------------------------------------------------------------------
enum : uint32_t {
  ERR_BAD_BASE = 1u,    // a byte outside {A,C,G,T}
  ERR_TIMEOUT = 2u,     // a look-back spin reached its iteration limit
  ERR_OVERFLOW = 4u,    // a count exceeded its 32-bit field
  ERR_INTERNAL = 8u,    // an internal consistency check failed
};

// ---------------------------------------------------------------------------
// keys
// ---------------------------------------------------------------------------
// A 128-bit key: high word first in memory, matching the C ABI's layout.
struct __align__(16) Key128 {
  uint64_t hi, lo;
};

template <class K> struct KeyOps;

template <> struct KeyOps<uint64_t> {
  static constexpr int kBits = 64;
  __host__ __device__ static uint64_t zero() { return 0; }
  __device__ static bool less(uint64_t a, uint64_t b) { return a < b; }
  __device__ static bool eq(uint64_t a, uint64_t b) { return a == b; }
  // digit of `bits` bits starting at bit `shift` (bits <= 16)
  __device__ static uint32_t digit(uint64_t a, int shift, int bits) {
    return (uint32_t)(a >> shift) & ((1u << bits) - 1u);
  }
  __device__ static uint64_t shr(uint64_t a, int s) { return s >= 64 ? 0 : a >> s; }
  __device__ static uint64_t mask_low(uint64_t a, int nbits) {
    return nbits >= 64 ? a : (a & ((1ull << nbits) - 1ull));
  }
  __device__ static uint64_t low2(uint64_t a) { return a & 3ull; }
  __device__ static uint64_t words_hi(uint64_t) { return 0; }
  __device__ static uint64_t words_lo(uint64_t a) { return a; }
  __device__ static uint64_t sub(uint64_t a, uint64_t b) { return a - b; }
  __device__ static uint64_t add(uint64_t a, uint64_t b) { return a + b; }
  // number of significant bits (0 for 0)
  __device__ static int bitlen(uint64_t a) { return a ? 64 - __clzll((long long)a) : 0; }
};

template <> struct KeyOps<Key128> {
  static constexpr int kBits = 128;
  __host__ __device__ static Key128 zero() { return Key128{0, 0}; }
  __device__ static bool less(Key128 a, Key128 b) {
    return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo);
  }
  __device__ static bool eq(Key128 a, Key128 b) { return a.hi == b.hi && a.lo == b.lo; }
  __device__ static uint32_t digit(Key128 a, int shift, int bits) {
    uint64_t w;
    if (shift >= 64) w = a.hi >> (shift - 64);
    else if (shift == 0) w = a.lo;
    else w = (a.lo >> shift) | (a.hi << (64 - shift));
    return (uint32_t)w & ((1u << bits) - 1u);
  }
  __device__ static Key128 shr(Key128 a, int s) {
    if (s == 0) return a;
    if (s >= 128) return Key128{0, 0};
    if (s >= 64) return Key128{0, a.hi >> (s - 64)};
    return Key128{a.hi >> s, (a.lo >> s) | (a.hi << (64 - s))};
  }
  __device__ static Key128 mask_low(Key128 a, int nbits) {
    if (nbits >= 128) return a;
    if (nbits >= 64) return Key128{nbits == 64 ? 0 : (a.hi & ((1ull << (nbits - 64)) - 1ull)), a.lo};
    return Key128{0, a.lo & ((1ull << nbits) - 1ull)};
  }
  __device__ static uint64_t low2(Key128 a) { return a.lo & 3ull; }
  __device__ static uint64_t words_hi(Key128 a) { return a.hi; }
  __device__ static uint64_t words_lo(Key128 a) { return a.lo; }
  __device__ static Key128 sub(Key128 a, Key128 b) {
    return Key128{a.hi - b.hi - (a.lo < b.lo ? 1ull : 0ull), a.lo - b.lo};
  }
  __device__ static Key128 add(Key128 a, Key128 b) {
    const uint64_t lo = a.lo + b.lo;
    return Key128{a.hi + b.hi + (lo < a.lo ? 1ull : 0ull), lo};
  }
  __device__ static int bitlen(Key128 a) {
    return a.hi ? 128 - __clzll((long long)a.hi) : (a.lo ? 64 - __clzll((long long)a.lo) : 0);
  }
};

// Swap the two bits of every 2-bit group.
__device__ __forceinline__ uint64_t swap_bit_pairs(uint64_t x) {
  return ((x >> 1) & 0x5555555555555555ull) | ((x & 0x5555555555555555ull) << 1);
}

// Reverse complement of an m-mer (m <= 32) held in the low 2m bits: the
// complement of code c is 3 - c = c ^ 3, so complementing is a bitwise NOT;
// bit reversal reverses the base order but also swaps the two bits inside
// every base, which swap_bit_pairs undoes.
__device__ __forceinline__ uint64_t revcomp(uint64_t x, int m) {
  return swap_bit_pairs(__brevll(~x)) >> (64 - 2 * m);
}

__device__ __forceinline__ Key128 revcomp(Key128 x, int m) {
  // reverse the full 128 bits, then move the m bases down to the low end
  uint64_t hi = swap_bit_pairs(__brevll(~x.lo));
  uint64_t lo = swap_bit_pairs(__brevll(~x.hi));
  int s = 128 - 2 * m;
  if (s == 0) return Key128{hi, lo};
  if (s >= 64) return Key128{0, hi >> (s - 64)};
  return Key128{hi >> s, (lo >> s) | (hi << (64 - s))};
}

template <class K>
__device__ __forceinline__ K kmin(K a, K b) {
  return KeyOps<K>::less(b, a) ? b : a;
}

// ---------------------------------------------------------------------------
// relaxed global loads/stores for the look-back status words
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t ld_relaxed(const uint64_t *p) {
  uint64_t v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_relaxed(uint64_t *p, uint64_t v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// A look-back status word: [epoch:30 | flag:2 | count:32].  The epoch is
// the number of the scan (or sort pass) that wrote it, so a status array
// never needs clearing between scans: words of older scans read as "not
// ready".  flag 1 = tile aggregate, 2 = inclusive prefix.
enum : uint32_t { LB_AGGREGATE = 1u, LB_INCLUSIVE = 2u };

__device__ __forceinline__ uint64_t lb_word(uint32_t epoch, uint32_t flag, uint32_t count) {
  return ((uint64_t)(epoch & 0x3fffffffu) << 34) | ((uint64_t)flag << 32) | count;
}
__device__ __forceinline__ uint32_t lb_epoch(uint64_t w) { return (uint32_t)(w >> 34); }
__device__ __forceinline__ uint32_t lb_flag(uint64_t w) { return (uint32_t)(w >> 32) & 3u; }
__device__ __forceinline__ uint32_t lb_count(uint64_t w) { return (uint32_t)w; }

// Exclusive prefix of one counter over all tiles before `tile`, by
// decoupled look-back (Merrill & Garland).  Called by one thread per
// counter; status[t * stride] is tile t's word.  Spins at most spin_limit
// times per predecessor; on timeout it sets ERR_TIMEOUT and returns the
// partial sum (the caller's output is then discarded by the host).
__device__ __forceinline__ uint32_t lookback_exclusive(uint64_t *status, size_t stride,
                                                       uint32_t tile, uint32_t epoch,
                                                       uint32_t spin_limit, uint32_t *err) {
  uint32_t sum = 0;
  int64_t t = (int64_t)tile - 1;
  const uint32_t ep = epoch & 0x3fffffffu;
  while (t >= 0) {
    uint64_t w;
    uint32_t spins = 0;
    for (;;) {
      w = ld_relaxed(status + (size_t)t * stride);
      if (lb_epoch(w) == ep && lb_flag(w) != 0) break;
      if (++spins > spin_limit) {
        atomicOr(err, ERR_TIMEOUT);
        return sum;
      }
      __nanosleep(32);
    }
    sum += lb_count(w);
    if (lb_flag(w) == LB_INCLUSIVE) break;
    --t;
  }
  return sum;
}

// As lookback_exclusive, but loads BATCH predecessors' words at once, so a
// run of tiles that have published only their aggregates costs one memory
// round trip per BATCH tiles instead of one per tile.
template <int BATCH>
__device__ __forceinline__ uint32_t lookback_exclusive_batched(uint64_t *status, size_t stride, uint32_t tile,
                                                               uint32_t epoch, uint32_t spin_limit, uint32_t *err) {
  uint32_t sum = 0;
  int64_t t = (int64_t)tile - 1;
  const uint32_t ep = epoch & 0x3fffffffu;
  while (t >= 0) {
    uint64_t w[BATCH];
#pragma unroll
    for (int j = 0; j < BATCH; j++) w[j] = t - j >= 0 ? ld_relaxed(status + (size_t)(t - j) * stride) : 0;
#pragma unroll
    for (int j = 0; j < BATCH; j++) {
      if (t - j < 0) return sum;
      uint32_t spins = 0;
      while (!(lb_epoch(w[j]) == ep && lb_flag(w[j]) != 0)) {
        if (++spins > spin_limit) {
          atomicOr(err, ERR_TIMEOUT);
          return sum;
        }
        __nanosleep(32);
        w[j] = ld_relaxed(status + (size_t)(t - j) * stride);
      }
      sum += lb_count(w[j]);
      if (lb_flag(w[j]) == LB_INCLUSIVE) return sum;
    }
    t -= BATCH;
  }
  return sum;
}

// Warp-wide exclusive prefix of one counter: all 32 lanes look back over 32
// predecessors at a time.  Returns the same value in every lane.
__device__ __forceinline__ uint32_t lookback_exclusive_warp(uint64_t *status, uint32_t tile,
                                                            uint32_t epoch, uint32_t spin_limit,
                                                            uint32_t *err) {
  const unsigned lane = threadIdx.x & 31u;
  const uint32_t ep = epoch & 0x3fffffffu;
  uint32_t sum = 0;
  int64_t window_end = (int64_t)tile - 1;  // highest predecessor not yet summed
  while (window_end >= 0) {
    int64_t t = window_end - (int64_t)lane;
    uint64_t w = 0;
    bool ready = true;
    if (t >= 0) {
      uint32_t spins = 0;
      for (;;) {
        w = ld_relaxed(status + t);
        if (lb_epoch(w) == ep && lb_flag(w) != 0) break;
        if (++spins > spin_limit) { ready = false; break; }
        __nanosleep(32);
      }
    }
    if (!__all_sync(0xffffffffu, ready)) {
      if (lane == 0) atomicOr(err, ERR_TIMEOUT);
      return sum;
    }
    // lanes 0.. hold predecessors window_end, window_end-1, ...; stop at the
    // first inclusive prefix (lowest lane that has one)
    unsigned incl = __ballot_sync(0xffffffffu, t >= 0 && lb_flag(w) == LB_INCLUSIVE);
    unsigned take = incl ? ((incl & (0u - incl)) << 1) - 1u : 0xffffffffu;  // lanes <= first incl
    uint32_t c = ((take >> lane) & 1u) && t >= 0 ? lb_count(w) : 0u;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    sum += c;
    if (incl) break;
    window_end -= 32;
  }
  return sum;
}

}  // namespace dbg
