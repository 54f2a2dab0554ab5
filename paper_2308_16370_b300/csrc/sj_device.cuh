// Device helpers shared by the sieved-join kernels (sm_103a).
//
//  * fmix64 and the Bloom filter bit positions (Sec. 2.1 steps 1 and 3; the
//    paper leaves the hash family open, see sievejoin.h for the reading used)
//  * the status word bits that bounded device waits set instead of hanging
//  * a block-wide exclusive scan and a decoupled look-back over tiles
//    (single-pass, order-preserving prefix sums for stream compaction)
#pragma once

#include <stdint.h>

namespace sj {

constexpr uint32_t kErrTimeout = 1u;
constexpr uint32_t kErrTableFull = 2u;
constexpr uint32_t kErrOverflow = 4u;

// Spin bound for look-back / pending-slot waits: ~2^22 polls with a growing
// nanosleep backoff (capped at 256 ns), i.e. about a second at most.
constexpr uint32_t kSpinLimit = 1u << 22;

constexpr int kBlock = 256;  // threads per CTA of every streaming kernel

__device__ __forceinline__ uint64_t fmix64(uint64_t x) {
  x ^= x >> 33;
  x *= 0xff51afd7ed558ccdull;
  x ^= x >> 33;
  x *= 0xc4ceb9fe1a85ec53ull;
  x ^= x >> 33;
  return x;
}

__device__ __forceinline__ uint64_t key_hash(int32_t key, uint64_t seed) {
  return fmix64((uint64_t)(uint32_t)key ^ seed);
}

// Filter view passed by value to kernels.  nblocks is read from device memory
// because a filter built from a compacted relation is sized on the device.
struct FilterView {
  const uint32_t* words;
  const uint64_t* hdr;  // hdr[0] = nblocks, hdr[1] = rows inserted
  uint32_t k;
  uint32_t layout;      // 0 = blocked 256-bit, 1 = classic
  uint64_t seed;
};

__device__ __forceinline__ bool bit_of4(uint64_t q0, uint64_t q1, uint64_t q2, uint64_t q3,
                                        uint32_t bit) {
  const uint32_t i = bit >> 6;
  const uint64_t lo = (i & 1) ? q1 : q0;
  const uint64_t hi = (i & 1) ? q3 : q2;
  const uint64_t q = (i & 2) ? hi : lo;
  return (q >> (bit & 63)) & 1ull;
}

// Membership test.  Blocked layout: one 32-byte sector (two 16-byte loads
// through the read-only path), then k bit tests in registers.
__device__ __forceinline__ bool filter_contains(const FilterView& f, uint64_t nblocks,
                                                int32_t key) {
  const uint64_t h = key_hash(key, f.seed);
  if (f.layout == 0) {
    const uint64_t blk = ((h >> 32) * nblocks) >> 32;
    const ulonglong2* p = reinterpret_cast<const ulonglong2*>(f.words + blk * 8);
    const ulonglong2 a = __ldg(p);
    const ulonglong2 b = __ldg(p + 1);
    bool ok = true;
    for (uint32_t i = 0; i < f.k; ++i) {
      const uint32_t bit = (uint32_t)(h >> (8 * i)) & 255u;
      ok &= bit_of4(a.x, a.y, b.x, b.y, bit);
    }
    return ok;
  }
  const uint64_t m = nblocks * 256ull;
  const uint64_t h1 = h & 0xffffffffull;
  const uint64_t h2 = (h >> 32) | 1ull;
  for (uint32_t i = 0; i < f.k; ++i) {
    const uint64_t g = (h1 + (uint64_t)i * h2) % m;
    if (!((__ldg(f.words + (g >> 5)) >> (g & 31)) & 1u)) return false;
  }
  return true;
}

__device__ __forceinline__ uint64_t ld_volatile_u64(const uint64_t* p) {
  return *reinterpret_cast<const volatile uint64_t*>(p);
}
__device__ __forceinline__ uint32_t ld_volatile_u32(const uint32_t* p) {
  return *reinterpret_cast<const volatile uint32_t*>(p);
}
__device__ __forceinline__ void st_volatile_u64(uint64_t* p, uint64_t v) {
  *reinterpret_cast<volatile uint64_t*>(p) = v;
}
__device__ __forceinline__ void st_volatile_u32(uint32_t* p, uint32_t v) {
  *reinterpret_cast<volatile uint32_t*>(p) = v;
}

// ------------------------------------------------------------------ block scan
// Exclusive scan of one uint64 per thread over a 256-thread block; returns the
// thread's exclusive prefix and writes the block total to *total (all threads).
template <int NCH>
struct Vec {
  uint64_t v[NCH];
};

template <int NCH>
__device__ __forceinline__ Vec<NCH> block_exclusive_scan(Vec<NCH> x, Vec<NCH>* total,
                                                         Vec<NCH>* s_warp /* [8] */) {
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  Vec<NCH> inc = x;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
#pragma unroll
    for (int c = 0; c < NCH; ++c) {
      const uint64_t y = __shfl_up_sync(0xffffffffu, inc.v[c], d);
      if (lane >= d) inc.v[c] += y;
    }
  }
  if (lane == 31) s_warp[warp] = inc;
  __syncthreads();
  Vec<NCH> wpre;
  Vec<NCH> tot;
#pragma unroll
  for (int c = 0; c < NCH; ++c) { wpre.v[c] = 0; tot.v[c] = 0; }
#pragma unroll
  for (int w = 0; w < kBlock / 32; ++w) {
#pragma unroll
    for (int c = 0; c < NCH; ++c) {
      if (w < warp) wpre.v[c] += s_warp[w].v[c];
      tot.v[c] += s_warp[w].v[c];
    }
  }
  __syncthreads();  // s_warp may be reused by the caller
  Vec<NCH> ex;
#pragma unroll
  for (int c = 0; c < NCH; ++c) ex.v[c] = wpre.v[c] + inc.v[c] - x.v[c];
  *total = tot;
  return ex;
}

// ------------------------------------------------------------------ look-back
// Tile states for a decoupled look-back scan (Merrill and Garland, 2016):
// flag 0 = not ready, 1 = aggregate published, 2 = inclusive prefix published.
// Values are written before their flag, with a fence in between.
template <int NCH>
struct LookBack {
  uint32_t* flags;  // [ntiles], zeroed before the launch
  uint64_t* agg;    // [ntiles * NCH]
  uint64_t* inc;    // [ntiles * NCH]
  uint32_t* status;
};

template <int NCH>
__device__ __forceinline__ void lb_publish(const LookBack<NCH>& lb, uint32_t tile, uint32_t flag,
                                           const Vec<NCH>& v) {
  uint64_t* dst = (flag == 2 ? lb.inc : lb.agg) + (uint64_t)tile * NCH;
#pragma unroll
  for (int c = 0; c < NCH; ++c) st_volatile_u64(dst + c, v.v[c]);
  __threadfence();
  st_volatile_u32(lb.flags + tile, flag);
}

// Called by warp 0 of a tile > 0.  Returns the exclusive prefix of `tile`
// (all lanes).  Waits on predecessors are bounded: on timeout the status word
// gets kErrTimeout and the missing predecessor counts as an inclusive 0, so the
// kernel always finishes (its output is then reported as invalid by the host).
template <int NCH>
__device__ __forceinline__ Vec<NCH> lb_exclusive(const LookBack<NCH>& lb, uint32_t tile) {
  const int lane = threadIdx.x & 31;
  Vec<NCH> excl;
#pragma unroll
  for (int c = 0; c < NCH; ++c) excl.v[c] = 0;
  int64_t j = (int64_t)tile - 1;
  while (true) {
    const int64_t idx = j - lane;
    uint32_t f = 2;
    Vec<NCH> v;
#pragma unroll
    for (int c = 0; c < NCH; ++c) v.v[c] = 0;
    if (idx >= 0) {
      f = ld_volatile_u32(lb.flags + idx);
      uint32_t spins = 0, ns = 8;
      while (f == 0) {
        if (++spins > kSpinLimit) break;
        __nanosleep(ns);
        if (ns < 256) ns <<= 1;
        f = ld_volatile_u32(lb.flags + idx);
      }
      if (f == 0) {
        atomicOr(lb.status, kErrTimeout);
        f = 2;
      } else {
        __threadfence();
        const uint64_t* src = (f == 2 ? lb.inc : lb.agg) + (uint64_t)idx * NCH;
#pragma unroll
        for (int c = 0; c < NCH; ++c) v.v[c] = ld_volatile_u64(src + c);
      }
    }
    const uint32_t pmask = __ballot_sync(0xffffffffu, f == 2);
    const int stop = pmask ? (__ffs(pmask) - 1) : 31;
#pragma unroll
    for (int c = 0; c < NCH; ++c) {
      uint64_t x = (lane <= stop) ? v.v[c] : 0ull;
#pragma unroll
      for (int d = 16; d > 0; d >>= 1) x += __shfl_xor_sync(0xffffffffu, x, d);
      excl.v[c] += x;
    }
    if (pmask) break;
    j -= 32;
  }
  return excl;
}

}  // namespace sj
