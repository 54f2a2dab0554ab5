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
constexpr uint32_t kErrCapacity = 8u;  // a device-sized output outgrew its buffer

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

// fmix64 of (uint64(uint32 key) xor seed) in 32-bit operations, for the hot
// probe loops.  With x = seed_hi : (key xor seed_lo), the first xor-shift
// only folds seed_hi >> 1 into the low word and the first multiply's
// seed_hi * C1 term is a constant, so both are computed once per launch
// (Key32Hash) and a key costs one xor, five multiplies and two xor-shifts.
// The result equals fmix64 bit for bit.
struct Key32Hash {
  uint32_t a;  // seed_lo ^ (seed_hi >> 1)
  uint32_t b;  // low 32 bits of seed_hi * C1_lo
  uint64_t seed64;
};
__device__ __forceinline__ Key32Hash key32_hash_fold(uint64_t seed) {
  const uint32_t slo = (uint32_t)seed, shi = (uint32_t)(seed >> 32);
  Key32Hash f;
  f.a = slo ^ (shi >> 1);
  f.b = shi * 0xed558ccdu;
  f.seed64 = seed;
  return f;
}
__device__ __forceinline__ void key32_hash(const Key32Hash& f, uint32_t key, uint32_t& hi,
                                           uint32_t& lo) {
  const uint32_t l = key ^ f.a;
  // (seed_hi : l) * 0xff51afd7ed558ccd mod 2^64
  const uint64_t p = (uint64_t)l * 0xed558ccdu + ((uint64_t)f.b << 32);
  const uint32_t xh = (uint32_t)(p >> 32) + l * 0xff51afd7u;
  const uint32_t xl = (uint32_t)p ^ (xh >> 1);
  // (xh : xl) * 0xc4ceb9fe1a85ec53 mod 2^64
  const uint64_t q = (uint64_t)xl * 0x1a85ec53u;
  hi = (uint32_t)(q >> 32) + xl * 0xc4ceb9feu + xh * 0x1a85ec53u;
  lo = (uint32_t)q ^ (hi >> 1);
}

// 1 << (s mod 32) in one funnel shift.
__device__ __forceinline__ uint32_t bit_of(uint32_t s) { return __funnelshift_l(0u, 1u, s); }

// Register-blocked mask of k = K bits from the low word of the hash.
template <int K>
__device__ __forceinline__ uint32_t reg32_mask_fs(uint32_t lo) {
  uint32_t m = bit_of(lo);
#pragma unroll
  for (int i = 1; i < K; ++i) m |= bit_of(lo >> (5 * i));
  return m;
}

// L2 policy that keeps a filter resident while key columns stream past it.
__device__ __forceinline__ uint64_t l2_evict_last_policy() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
// Read-only filter word load (L1-cacheable) with an L2 eviction hint.
__device__ __forceinline__ uint32_t ld_filter_word(const uint32_t* p, uint64_t pol) {
  uint32_t v;
  asm("ld.global.nc.L2::cache_hint.b32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
  return v;
}

// Filter view passed by value to kernels.  nblocks is read from device memory
// because a filter built from a compacted relation is sized on the device.
struct FilterView {
  const uint32_t* words;
  const uint64_t* hdr;  // hdr[0] = nblocks, hdr[1] = rows inserted
  uint32_t k;
  uint32_t layout;      // 0 = register-blocked 32-bit word, 1 = blocked 256-bit, 2 = classic
  uint64_t seed;
};

// Register-blocked layout: the word holding all k bits of a key and the mask
// of those bits (bit i = (h >> 5i) & 31).  nwords = 8 * nblocks < 2^35; the
// multiply-shift range reduction takes the high half of h.
__device__ __forceinline__ uint64_t reg32_word(uint64_t h, uint64_t nwords) {
  return ((h >> 32) * nwords) >> 32;
}
__device__ __forceinline__ uint32_t reg32_mask(uint32_t hlo, uint32_t k) {
  uint32_t m = 0;
#pragma unroll
  for (uint32_t i = 0; i < 6; ++i)
    if (i < k) m |= 1u << ((hlo >> (5 * i)) & 31u);
  return m;
}

// Compile-time-k variants (the hot loops dispatch on k once per tile).
template <int K>
__device__ __forceinline__ uint32_t reg32_mask_k(uint32_t hlo) {
  uint32_t m = 0;
#pragma unroll
  for (int i = 0; i < K; ++i) m |= 1u << ((hlo >> (5 * i)) & 31u);
  return m;
}

// Word index when the filter has fewer than 2^32 words: one high multiply.
__device__ __forceinline__ uint32_t reg32_word32(uint64_t h, uint32_t nwords) {
  return __umulhi((uint32_t)(h >> 32), nwords);
}

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
    const uint32_t m = reg32_mask((uint32_t)h, f.k);
    return (__ldg(f.words + reg32_word(h, nblocks * 8)) & m) == m;
  }
  if (f.layout == 1) {
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

template <int NCH, int NT = kBlock>
__device__ __forceinline__ Vec<NCH> block_exclusive_scan(Vec<NCH> x, Vec<NCH>* total,
                                                         Vec<NCH>* s_warp /* [NT / 32] */) {
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
  for (int w = 0; w < NT / 32; ++w) {
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
// Tile states for a decoupled look-back scan (Merrill and Garland, 2016).  Each
// channel of a tile is ONE 64-bit word: epoch (16 bits) | state (2 bits) |
// value (46 bits), state 0 = not ready, 1 = tile aggregate, 2 = inclusive
// prefix.  Flag and value travel in one single-copy-atomic store, so neither
// side needs a fence.  A word whose epoch differs from this launch's reads as
// "not ready": the states need no clearing between launches as long as every
// launch on the same scratch uses a new epoch (or the words are zeroed and
// epoch 0 is used).  With two channels a reader retries until both words show
// the same state.
constexpr int kValueBits = 46;
constexpr uint64_t kValueMask = (1ull << kValueBits) - 1;

template <int NCH>
struct LookBack {
  uint64_t* st;      // [ntiles * NCH]
  uint32_t* status;
  uint32_t epoch;    // < 2^16
};

template <int NCH>
__device__ __forceinline__ void lb_publish(const LookBack<NCH>& lb, uint32_t tile, uint32_t state,
                                           const Vec<NCH>& v) {
  const uint64_t tag = ((uint64_t)lb.epoch << 48) | ((uint64_t)state << kValueBits);
#pragma unroll
  for (int c = 0; c < NCH; ++c)
    st_volatile_u64(lb.st + (uint64_t)tile * NCH + c, tag | (v.v[c] & kValueMask));
}

// State of a packed word under this launch's epoch.
template <int NCH>
__device__ __forceinline__ uint32_t lb_state(const LookBack<NCH>& lb, uint64_t w) {
  return (uint32_t)(w >> 48) == lb.epoch ? (uint32_t)(w >> kValueBits) & 3u : 0u;
}

// Read the NCH words of one tile; returns their common state (0 if not ready
// or inconsistent) and the values.
template <int NCH>
__device__ __forceinline__ uint32_t lb_read(const LookBack<NCH>& lb, int64_t idx, Vec<NCH>* v) {
  uint32_t s0 = 0;
#pragma unroll
  for (int c = 0; c < NCH; ++c) {
    const uint64_t w = ld_volatile_u64(lb.st + (uint64_t)idx * NCH + c);
    const uint32_t s = lb_state(lb, w);
    if (c == 0) s0 = s;
    else if (s != s0) s0 = 0;
    v->v[c] = w & kValueMask;
  }
  return s0;
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
      f = lb_read(lb, idx, &v);
      uint32_t spins = 0, ns = 8;
      while (f == 0) {
        if (++spins > kSpinLimit) break;
        __nanosleep(ns);
        if (ns < 256) ns <<= 1;
        f = lb_read(lb, idx, &v);
      }
      if (f == 0) {
        atomicOr(lb.status, kErrTimeout);
        f = 2;
#pragma unroll
        for (int c = 0; c < NCH; ++c) v.v[c] = 0;
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

// 4-byte asynchronous global -> shared copy (cached in L1).  Landing probe
// words in shared memory instead of registers lets one thread keep dozens of
// filter reads in flight.
__device__ __forceinline__ void cp_async4(uint32_t* smem_dst, const uint32_t* gsrc) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;" ::: "memory");
}

// One 32-byte filter block in a single request (256-bit vector load).  The
// read-only variant is for filters no kernel writes while it runs; the
// L1-cacheable variant is for the build, where a stale copy only costs a
// redundant atomicOr.
__device__ __forceinline__ void ld_block32_nc(const uint32_t* p, uint64_t& q0, uint64_t& q1,
                                              uint64_t& q2, uint64_t& q3) {
  asm("ld.global.nc.v4.u64 {%0, %1, %2, %3}, [%4];"
      : "=l"(q0), "=l"(q1), "=l"(q2), "=l"(q3)
      : "l"(p));
}
__device__ __forceinline__ void ld_block32_ca(const uint32_t* p, uint64_t& q0, uint64_t& q1,
                                              uint64_t& q2, uint64_t& q3) {
  asm volatile("ld.global.ca.v4.u64 {%0, %1, %2, %3}, [%4];"
               : "=l"(q0), "=l"(q1), "=l"(q2), "=l"(q3)
               : "l"(p));
}

// Draw this CTA's tile ticket.  The CTA that draws the last ticket of the grid
// resets the counter, so the next launch on the same scratch starts at 0
// without a memset (every ticket of this launch has been drawn by then).
__device__ __forceinline__ uint32_t draw_ticket(uint32_t* counter) {
  const uint32_t t = atomicAdd(counter, 1u);
  if (t == gridDim.x - 1) atomicExch(counter, 0u);
  return t;
}

// Ticket for a grid whose CTAs loop over `ntiles` tiles: every CTA draws
// until it gets a ticket >= ntiles, so the launch draws ntiles + gridDim.x
// tickets in all, and the CTA that draws the last one resets the counter.
__device__ __forceinline__ uint32_t draw_ticket_loop(uint32_t* counter, uint64_t ntiles) {
  const uint32_t t = atomicAdd(counter, 1u);
  if ((uint64_t)t == ntiles + gridDim.x - 1) atomicExch(counter, 0u);
  return t;
}

}  // namespace sj
