// sm_103a kernels of the sieved multi-way join.
//
//   k_bloom_build    -- Bloom filter build (Sec. 2.1 step 1): atomicOr into an
//                       L2-resident filter, repeated (word, mask) pairs skipped
//   k_bloom_probe    -- membership test (Sec. 2.1 step 3)
//   k_sieve_chunk    -- one pruning step (Sec. 2.2): key loads, filter probes,
//                       survivor bits by warp ballots, order-preserving
//                       compaction with chunk offsets from per-32-chunk
//                       group sums (or a CTA-wide decoupled look-back)
//   k_sieve_batch, k_bloom_build_batch -- the sieve steps / filter builds of
//                       many queries' pruning phases in one launch each
//   k_insert_*       -- insert maintenance of a built filter (Sec. 2.4)
//   k_group_offsets  -- row-group offsets of a multimap (one atomic per tile)
//   k_mm_*           -- multimap hash join level (Sec. 2.2 enumeration phase)
//   k_agg_*          -- last join level folded into COUNT(*) / SUM
//   k_pair_*, k_gather_i32, k_triangles -- the cyclic query with its closing
//                       filter (Sec. 2.3)
//
// Nothing here is a dense contraction, so there are no tensor-core paths: all
// kernels are bound by HBM bandwidth or by L2 latency of random accesses.
#include "sj_kernels.cuh"

namespace sj {

namespace {

constexpr uint64_t kTableSeed = 0x9e3779b97f4a7c15ull;
// fmix64(uint32(key) xor kTableSeed) with the seed's terms folded at compile time
constexpr uint32_t kTableHashA = (uint32_t)kTableSeed ^ ((uint32_t)(kTableSeed >> 32) >> 1);
constexpr uint32_t kTableHashB = (uint32_t)(kTableSeed >> 32) * 0xed558ccdu;

// Home bucket of a key: the low word of fmix64(uint32(key) xor kTableSeed).
__device__ __forceinline__ uint32_t table_bucket(int32_t key, uint32_t mask) {
  const Key32Hash h = {kTableHashA, kTableHashB, kTableSeed};
  uint32_t hi, lo;
  key32_hash(h, (uint32_t)key, hi, lo);
  return lo & mask;
}

// A table whose mask was written on the device (k_table_init) reads it once.
__device__ __forceinline__ Table resolve(Table t) {
  if (t.mask_dev) t.bucket_mask = __ldg(t.mask_dev);
  return t;
}

__device__ __forceinline__ int64_t dev_n(const uint64_t* n_dev, int64_t n_host) {
  return n_dev ? (int64_t)__ldg(n_dev) : n_host;
}

// Sum of the SUM terms of one row, int64 arithmetic mod 2^64.  The loop has a
// constant trip count so the kernel-parameter arrays are indexed statically.
__device__ __forceinline__ uint64_t term_sum(const Terms& t, int64_t row) {
  uint64_t v = 0;
#pragma unroll
  for (int i = 0; i < kMaxTerms; ++i) {
    if (i < t.n) {
      if (t.col_hi[i]) {
        const uint64_t lo = (uint32_t)__ldg(t.col[i] + row);
        const uint64_t hi = (uint32_t)__ldg(t.col_hi[i] + row);
        v += lo | (hi << 32);
      } else {
        v += (uint64_t)(int64_t)__ldg(t.col[i] + row);
      }
    }
  }
  return v;
}

// ---------------------------------------------------------------- Bloom build
__device__ __forceinline__ void or_bits(uint32_t* p, uint32_t mask) {
  // Read first: under skew most repeated keys find their bits already set and
  // skip the atomic entirely (L2-coherent load, bypassing L1).
  if ((__ldcg(p) & mask) != mask) atomicOr(p, mask);
}

// Per-CTA cache of key hashes this CTA has already inserted, so a key repeated
// many times (Zipf-hot keys) issues about one atomicOr per CTA instead of one
// per occurrence: a stale L1 copy of a hot word would otherwise keep every
// occurrence on the slow same-address atomic path.  A slot holds a whole
// 64-bit hash written in one store; a hash equal to 0 is never skipped, since
// 0 also marks an empty slot.
constexpr int kSeenSlots = 2048;

__device__ __forceinline__ bool seen_before(unsigned long long* seen, uint64_t h) {
  const uint32_t slot = (uint32_t)(h ^ (h >> 29)) & (kSeenSlots - 1);
  if (h != 0 && seen[slot] == h) return true;
  seen[slot] = h;
  return false;
}

__device__ __forceinline__ void bloom_insert_classic(const BloomBuildArgs& a, uint64_t nb,
                                                     int32_t key) {
  const uint64_t h = key_hash(key, a.seed);
  const uint64_t m = nb * 256ull;
  const uint64_t h1 = h & 0xffffffffull;
  const uint64_t h2 = (h >> 32) | 1ull;
  for (uint32_t i = 0; i < a.k; ++i) {
    const uint64_t g = (h1 + (uint64_t)i * h2) % m;
    or_bits(a.words + (g >> 5), 1u << (g & 31));
  }
}

// Blocked layout, four keys at a time: the four 32-byte blocks are loaded
// first (L1-cacheable, so repeated hot keys hit L1 instead of one L2 slice),
// then an atomicOr is issued only for bits that are still clear.  A stale L1
// copy can only cause a redundant OR, never a lost bit.
__device__ __forceinline__ void bloom_insert_blocked4(const BloomBuildArgs& a, uint64_t nb,
                                                      const int32_t (&key)[4], uint32_t live,
                                                      unsigned long long* seen) {
  uint64_t h[4];
  uint32_t* base[4];
  uint64_t q[4][4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    h[j] = key_hash(key[j], a.seed);
    base[j] = a.words + (((h[j] >> 32) * nb) >> 32) * 8;
    ld_block32_ca(base[j], q[j][0], q[j][1], q[j][2], q[j][3]);
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    if (!((live >> j) & 1u)) continue;
    bool all = true;
#pragma unroll
    for (uint32_t i = 0; i < 4; ++i)
      if (i < a.k) all &= bit_of4(q[j][0], q[j][1], q[j][2], q[j][3], (uint32_t)(h[j] >> (8 * i)) & 255u);
    if (all || seen_before(seen, h[j])) continue;
#pragma unroll
    for (uint32_t i = 0; i < 4; ++i) {
      if (i < a.k) {
        const uint32_t bit = (uint32_t)(h[j] >> (8 * i)) & 255u;
        if (!bit_of4(q[j][0], q[j][1], q[j][2], q[j][3], bit))
          atomicOr(base[j] + (bit >> 5), 1u << (bit & 31));
      }
    }
  }
}

// Register-blocked layout, four keys at a time: load the four words first
// (L1-cacheable), then one atomicOr per key whose bits are not all set yet.
__device__ __forceinline__ void bloom_insert_reg4(const BloomBuildArgs& a, uint64_t nb,
                                                  const int32_t (&key)[4], uint32_t live,
                                                  unsigned long long* seen) {
  uint32_t* p[4];
  uint32_t m[4], cur[4];
  uint64_t h[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    h[j] = key_hash(key[j], a.seed);
    p[j] = a.words + reg32_word(h[j], nb * 8);
    m[j] = reg32_mask((uint32_t)h[j], a.k);
    cur[j] = __ldca(p[j]);
  }
#pragma unroll
  for (int j = 0; j < 4; ++j)
    if (((live >> j) & 1u) && (cur[j] & m[j]) != m[j] && !seen_before(seen, h[j]))
      atomicOr(p[j], m[j]);
}

// Register-blocked layout, kBuildKeys keys per thread per round: the key
// vectors, then all the filter words are loaded before any atomic, so a thread
// has kBuildKeys independent L2 reads in flight instead of a serial chain.
constexpr int kBuildVecs = 2;
constexpr int kBuildKeys = 4 * kBuildVecs;

template <int K>
__device__ __forceinline__ void bloom_insert_regN(const BloomBuildArgs& a, uint32_t nwords,
                                                  const int32_t (&key)[kBuildKeys], uint32_t live,
                                                  unsigned long long* seen) {
  uint32_t w[kBuildKeys], cur[kBuildKeys], m[kBuildKeys];
#pragma unroll
  for (int j = 0; j < kBuildKeys; ++j) {
    const uint64_t h = key_hash(key[j], a.seed);
    w[j] = reg32_word32(h, nwords);
    m[j] = K > 0 ? reg32_mask_k<(K > 0 ? K : 1)>((uint32_t)h) : reg32_mask((uint32_t)h, a.k);
  }
#pragma unroll
  for (int j = 0; j < kBuildKeys; ++j) cur[j] = __ldca(a.words + w[j]);
  // the CTA cache is keyed by (word, mask): two keys with the same pair set
  // the same bits, so skipping the second one's OR loses nothing, and the keys
  // need not stay in registers
#pragma unroll
  for (int j = 0; j < kBuildKeys; ++j)
    if (((live >> j) & 1u) && (cur[j] & m[j]) != m[j] &&
        !seen_before(seen, ((uint64_t)w[j] << 32) | m[j]))
      atomicOr(a.words + w[j], m[j]);
}

__global__ void __launch_bounds__(kBlock, 4) k_bloom_build(BloomBuildArgs a) {
  __shared__ unsigned long long s_seen[kSeenSlots];
  for (int i = threadIdx.x; i < kSeenSlots; i += blockDim.x) s_seen[i] = 0ull;
  __syncthreads();
  const int64_t n = a.n_dev ? (int64_t)(*a.n_dev) : a.n_host;
  uint64_t nb = ((uint64_t)a.bits_per_key * (uint64_t)n + 255ull) / 256ull;
  if (nb < 1) nb = 1;
  if (nb > a.nblocks_cap) nb = a.nblocks_cap;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    a.hdr[0] = nb;
    a.hdr[1] = (uint64_t)n;
  }
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int4* kv = reinterpret_cast<const int4*>(a.keys);
  if (a.layout == 0 && nb * 8 < (1ull << 32)) {
    const uint32_t nwords = (uint32_t)(nb * 8);
    // rounds of kBuildKeys keys per thread: vector v of a round is key vector
    // base + v * stride, so every warp load is one contiguous 512 B
    const int64_t nvec = (n + 3) >> 2;
    const int64_t nfull = n >> 2;  // vectors of 4 valid keys
    // the next round's key vectors are loaded before this round's inserts, so
    // a round waits on the filter words only
    int4 xv[kBuildVecs];
#pragma unroll
    for (int v = 0; v < kBuildVecs; ++v) {
      const int64_t i = gid + v * stride;
      xv[v] = i < nfull ? __ldcs(kv + i) : make_int4(0, 0, 0, 0);
    }
    for (int64_t base = gid; base < nvec; base += kBuildVecs * stride) {
      int32_t k16[kBuildKeys];
      uint32_t live = 0;
#pragma unroll
      for (int v = 0; v < kBuildVecs; ++v) {
        const int64_t i = base + v * stride;
        if (i < nfull) {
          const int4 x = xv[v];
          k16[4 * v] = x.x;
          k16[4 * v + 1] = x.y;
          k16[4 * v + 2] = x.z;
          k16[4 * v + 3] = x.w;
          live |= 0xfu << (4 * v);
        } else {
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            k16[4 * v + e] = 0;
            if (i < nvec && (i << 2) + e < n) {
              k16[4 * v + e] = __ldcs(a.keys + (i << 2) + e);
              live |= 1u << (4 * v + e);
            }
          }
        }
      }
#pragma unroll
      for (int v = 0; v < kBuildVecs; ++v) {
        const int64_t i = base + kBuildVecs * stride + v * stride;
        xv[v] = i < nfull ? __ldcs(kv + i) : make_int4(0, 0, 0, 0);
      }
      switch (a.k) {
        case 3: bloom_insert_regN<3>(a, nwords, k16, live, s_seen); break;
        case 4: bloom_insert_regN<4>(a, nwords, k16, live, s_seen); break;
        default: bloom_insert_regN<0>(a, nwords, k16, live, s_seen); break;
      }
    }
    return;
  }
  const int64_t nvec = (n + 3) >> 2;
  for (int64_t i = gid; i < nvec; i += stride) {
    int32_t k4[4];
    uint32_t live = 0xfu;
    if ((i << 2) + 4 <= n) {
      const int4 v = __ldcs(kv + i);
      k4[0] = v.x;
      k4[1] = v.y;
      k4[2] = v.z;
      k4[3] = v.w;
    } else {
      live = 0;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        k4[e] = 0;
        if ((i << 2) + e < n) {
          k4[e] = __ldcs(a.keys + (i << 2) + e);
          live |= 1u << e;
        }
      }
    }
    if (a.layout == 0) {
      bloom_insert_reg4(a, nb, k4, live, s_seen);
    } else if (a.layout == 1) {
      bloom_insert_blocked4(a, nb, k4, live, s_seen);
    } else {
#pragma unroll
      for (int e = 0; e < 4; ++e)
        if ((live >> e) & 1u) bloom_insert_classic(a, nb, k4[e]);
    }
  }
}

__global__ void __launch_bounds__(kBlock) k_bloom_probe(BloomProbeArgs a) {
  const uint64_t nb = __ldg(a.f.hdr);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride)
    a.out[i] = filter_contains(a.f, nb, __ldg(a.keys + i)) ? 1 : 0;
}

// ---------------------------------------------------------------- sieve
// Test NK keys against one filter or predicate; returns the passing subset
// of `live`.  For the blocked layout all loads are issued before any bit is
// tested, so one thread keeps up to 4 * NK filter-word loads in flight.
// Tests of NK keys against one predicate or filter; each returns the passing
// subset of `live`.  All filter loads of the NK keys are issued before any bit
// is tested so they are in flight together; dead keys read word 0 (an L1 hit)
// instead of branching.  One function per layout keeps register use per call
// site to what that layout needs.
template <int NK>
__device__ __forceinline__ uint32_t test_pred(const SieveTest& t, const int32_t* key, uint32_t live) {
  uint32_t pass = 0;
#pragma unroll
  for (int j = 0; j < NK; ++j) pass |= (key[j] >= t.lo && key[j] < t.hi) ? (1u << j) : 0u;
  return pass & live;
}

template <int NK>
__device__ __forceinline__ uint32_t test_reg32(const SieveTest& t, uint64_t nb, const int32_t* key,
                                               uint32_t live) {
  uint32_t hlo[NK], w[NK];
#pragma unroll
  for (int j = 0; j < NK; ++j) {
    const uint64_t h = key_hash(key[j], t.f.seed);
    hlo[j] = (uint32_t)h;
    w[j] = __ldg(t.f.words + (((live >> j) & 1u) ? reg32_word(h, nb * 8) : 0));
  }
  uint32_t pass = 0;
#pragma unroll
  for (int j = 0; j < NK; ++j) {
    const uint32_t m = reg32_mask(hlo[j], t.f.k);
    pass |= ((w[j] & m) == m) ? (1u << j) : 0u;
  }
  return pass & live;
}

// Register-blocked probe with k and a 32-bit word count fixed at compile
// time: the word index is one high multiply and the mask k shift-ors.
template <int NK, int K>
__device__ __forceinline__ uint32_t test_reg32_k(const SieveTest& t, uint32_t nwords,
                                                 const int32_t* key, uint32_t live) {
  uint32_t hlo[NK], w[NK];
#pragma unroll
  for (int j = 0; j < NK; ++j) {
    const uint64_t h = key_hash(key[j], t.f.seed);
    hlo[j] = (uint32_t)h;
    w[j] = __ldg(t.f.words + (((live >> j) & 1u) ? reg32_word32(h, nwords) : 0u));
  }
  uint32_t pass = 0;
#pragma unroll
  for (int j = 0; j < NK; ++j) {
    const uint32_t m = reg32_mask_k<K>(hlo[j]);
    pass |= ((w[j] & m) == m) ? (1u << j) : 0u;
  }
  return pass & live;
}

template <int NK>
__device__ __forceinline__ uint32_t test_blocked(const SieveTest& t, uint64_t nb, const int32_t* key,
                                                 uint32_t live) {
  uint64_t h[NK];
  uint64_t q[NK][4];
#pragma unroll
  for (int j = 0; j < NK; ++j) {
    h[j] = key_hash(key[j], t.f.seed);
    const uint32_t* base =
        ((live >> j) & 1u) ? t.f.words + (((h[j] >> 32) * nb) >> 32) * 8 : t.f.words;
    ld_block32_nc(base, q[j][0], q[j][1], q[j][2], q[j][3]);
  }
  uint32_t pass = 0;
#pragma unroll
  for (int j = 0; j < NK; ++j) {
    bool ok = true;
#pragma unroll
    for (uint32_t i = 0; i < 4; ++i)
      if (i < t.f.k)
        ok &= bit_of4(q[j][0], q[j][1], q[j][2], q[j][3], (uint32_t)(h[j] >> (8 * i)) & 255u);
    pass |= ok ? (1u << j) : 0u;
  }
  return pass & live;
}

// All 8 keys of a lane against one test.
template <int K>
__device__ __forceinline__ uint32_t test8(const SieveTest& t, const int32_t* key, uint32_t live) {
  if (K > 0) {
    const uint32_t nw = (uint32_t)(__ldg(t.f.hdr) * 8);
    return test_reg32_k<8, K>(t, nw, key, live);
  }
  if (t.is_pred) return test_pred<8>(t, key, live);
  const uint64_t nb = __ldg(t.f.hdr);
  if (t.f.layout == 0) {
    if (nb * 8 < (1ull << 32)) {
      const uint32_t nw = (uint32_t)(nb * 8);
      switch (t.f.k) {
        case 1: return test_reg32_k<8, 1>(t, nw, key, live);
        case 2: return test_reg32_k<8, 2>(t, nw, key, live);
        case 3: return test_reg32_k<8, 3>(t, nw, key, live);
        case 4: return test_reg32_k<8, 4>(t, nw, key, live);
        default: break;
      }
    }
    return test_reg32<8>(t, nb, key, live);
  }
  if (t.f.layout == 1) {
    uint32_t pass = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q)
      pass |= test_blocked<2>(t, nb, key + 2 * q, (live >> (2 * q)) & 0x3u) << (2 * q);
    return pass;
  }
  uint32_t pass = 0;
#pragma unroll
  for (int j = 0; j < 8; ++j)
    if ((live >> j) & 1u) pass |= filter_contains(t.f, nb, key[j]) ? (1u << j) : 0u;
  return pass;
}

// ---------------------------------------------------------------- chunked sieve
// One launch per sieve step (Sec. 2.2 pruning phase).  A CTA draws a ticket t
// and owns rows [t C, t C + C), C = a.chunk_rows (a multiple of 2048, at most
// kCkMaxRows):
//  1. probe: each warp takes 256-row tiles of the chunk; lane l loads rows
//     32 j + l (j < 8: coalesced 128-byte loads, the next tile's keys loading
//     while this one is tested) and one ballot per j gives the survivor bits
//     of rows 32 j .. 32 j + 31 in row order; lane 0 stores the tile's eight
//     words in shared memory;
//  2. count: a block scan of the tiles' popcounts gives each tile's offset in
//     the chunk and the chunk total, which is published in the chunk's state
//     word and added to its group's word (groups of 32 chunks);
//  3. list: every survivor's row offset (16 bits) goes to its rank in a
//     shared-memory list;
//  4. offset: the sum of the earlier groups (each once all 32 of its chunks
//     have arrived) plus the states of the earlier chunks of the chunk's own
//     group (bounded waits); without group words, a look-back in which the
//     whole CTA reads the states of the 1024 chunks before it at once and
//     sums back to the nearest inclusive prefix;
//  5. write: thread i moves survivors i, i + 256, ... of every column, so a
//     chunk's gathers are in flight together and its output stores contiguous;
//  6. filters that the following builds write (a.zero_*) are cleared here,
//     sized by the step's own output: the chunk with output rows [p, p + c)
//     clears words [W(p), W(p + c)) with W(x) = 8 ceil(bpk x / 256), so the
//     launch clears exactly the words of a filter over its total rows; chunk 0
//     also clears the first block (the filter of an empty relation).
// Survivors are written in input order, as by the other sieve kernels.

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Keys of one warp tile: row base + 32 j + lane; rows at or beyond n read 0.
__device__ __forceinline__ void ck_load8(const int32_t* col, int64_t base, int64_t n, int lane,
                                         int32_t (&k)[8]) {
  const int32_t* p = col + base + lane;
  if (base + kCkTileRows <= n) {
#pragma unroll
    for (int j = 0; j < 8; ++j) k[j] = __ldcs(p + 32 * j);
  } else {
#pragma unroll
    for (int j = 0; j < 8; ++j) k[j] = (base + 32 * j + lane < n) ? __ldcs(p + 32 * j) : 0;
  }
}

// Hot path: one register-blocked filter with k = K and fewer than 2^32 words.
template <int K>
__device__ __forceinline__ void ck_test_reg32(const uint32_t* words, uint32_t nwords,
                                              const Key32Hash& hf, uint64_t pol,
                                              const int32_t (&key)[8], int64_t base, int64_t n,
                                              int lane, uint32_t (&b)[8]) {
  uint32_t w[8], m[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    uint32_t hi, lo;
    key32_hash(hf, (uint32_t)key[j], hi, lo);
    m[j] = reg32_mask_fs<K>(lo);
    w[j] = ld_filter_word(words + __umulhi(hi, nwords), pol);
  }
  if (base + kCkTileRows <= n) {
#pragma unroll
    for (int j = 0; j < 8; ++j) b[j] = __ballot_sync(0xffffffffu, (~w[j] & m[j]) == 0u);
  } else {
#pragma unroll
    for (int j = 0; j < 8; ++j)
      b[j] = __ballot_sync(0xffffffffu, (~w[j] & m[j]) == 0u && base + 32 * j + lane < n);
  }
}

// One row against one test (any layout, or a range predicate).
__device__ __forceinline__ bool test_one(const SieveTest& t, int32_t key) {
  if (t.is_pred) return key >= t.lo && key < t.hi;
  return filter_contains(t.f, __ldg(t.f.hdr), key);
}

// Any tests: predicates and filters of every layout.  The first test runs on
// the tile's 8 keys per lane; the rows it keeps are listed in the warp's
// shared-memory list (`wlist`, 256 entries) and each lane then takes one of
// them, loading its keys for all remaining tests at once and testing them
// together (one dependent round instead of one per test); survivors set
// their bit in the warp's 8 words `wbits` (row order).
__device__ __forceinline__ void ck_test_generic(const SieveArgs& a, int32_t (&key)[8], int64_t base,
                                                int64_t n, int lane, uint32_t (&b)[8], uint16_t* wlist,
                                                uint32_t* wbits) {
  uint32_t alive = 0;
#pragma unroll
  for (int j = 0; j < 8; ++j) alive |= (base + 32 * j + lane < n) ? (1u << j) : 0u;
  if (a.ntest > 0) alive = test8<0>(a.test[0], key, alive);
  if (a.ntest > 1) {
    const uint32_t c = __popc(alive);
    uint32_t inc = c;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, inc, d);
      if (lane >= d) inc += y;
    }
    const uint32_t total = __shfl_sync(0xffffffffu, inc, 31);
    uint32_t pos = inc - c;
#pragma unroll
    for (int j = 0; j < 8; ++j)
      if ((alive >> j) & 1u) wlist[pos++] = (uint16_t)(32 * j + lane);
    if (lane < 8) wbits[lane] = 0u;
    __syncwarp();
    for (uint32_t r = lane; r < total; r += 32) {
      const uint32_t row = wlist[r];
      int32_t k[kMaxTests];
#pragma unroll
      for (int t = 1; t < kMaxTests; ++t)
        k[t] = t < a.ntest ? __ldcs(a.test[t].col + base + row) : 0;
      bool ok = true;
#pragma unroll
      for (int t = 1; t < kMaxTests; ++t)
        if (t < a.ntest) ok &= test_one(a.test[t], k[t]);
      if (ok) atomicOr(wbits + (row >> 5), 1u << (row & 31));
    }
    __syncwarp();
#pragma unroll
    for (int j = 0; j < 8; ++j) b[j] = wbits[j];
    __syncwarp();  // wlist and wbits serve the warp's next tile
    return;
  }
#pragma unroll
  for (int j = 0; j < 8; ++j) b[j] = __ballot_sync(0xffffffffu, (alive >> j) & 1u);
}

// Exclusive prefix of chunk t > 0 (all threads get it).  The CTA reads the
// states of chunks t - 1 .. t - 1024 at once, four per thread, waits (bounded)
// until each holds at least its aggregate, and sums back to the nearest chunk
// holding an inclusive prefix; a window without one is added whole and the
// next window read.  A wait that gives up records kErrTimeout and counts the
// chunk as an inclusive 0, so the kernel always finishes.
__device__ uint64_t ck_lookback(const LookBack<1>& lb, uint32_t t, int* s_stop, uint64_t* s_red) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int R = kCkWindow / kCkThreads;
  uint64_t excl = 0;
  int64_t hi = (int64_t)t - 1;
  for (;;) {
    uint64_t w[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int64_t idx = hi - (tid + kCkThreads * r);
      w[r] = idx >= 0 ? ld_volatile_u64(lb.st + idx) : 0ull;
    }
    int best = 0x7fffffff;
    uint64_t v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int d = tid + kCkThreads * r;
      const int64_t idx = hi - d;
      uint32_t s = 2;
      v[r] = 0;
      if (idx >= 0) {
        s = lb_state<1>(lb, w[r]);
        uint32_t spins = 0, ns = 8;
        while (s == 0) {
          if (++spins > kSpinLimit) break;
          __nanosleep(ns);
          if (ns < 256) ns <<= 1;
          w[r] = ld_volatile_u64(lb.st + idx);
          s = lb_state<1>(lb, w[r]);
        }
        if (s == 0) {
          atomicOr(lb.status, kErrTimeout);
          s = 2;
        } else {
          v[r] = w[r] & kValueMask;
        }
      }
      if (s == 2 && d < best) best = d;
    }
    if (tid == 0) *s_stop = 0x7fffffff;
    __syncthreads();
    if (best != 0x7fffffff) atomicMin(s_stop, best);
    __syncthreads();
    const int stop = *s_stop;
    uint64_t part = 0;
#pragma unroll
    for (int r = 0; r < R; ++r)
      if (tid + kCkThreads * r <= stop) part += v[r];
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) part += __shfl_xor_sync(0xffffffffu, part, d);
    if (lane == 0) s_red[warp] = part;
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kCkThreads / 32; ++i) excl += s_red[i];
    __syncthreads();  // s_stop and s_red are reused
    if (stop != 0x7fffffff) return excl;
    hi -= kCkWindow;
  }
}

// Exclusive prefix of chunk t from the group words (all threads get it).
// Chunk t's kept-row count is in its state word and in grp[t / 32]
// (arrivals << 32 | sum of counts).  Warp 0 adds the earlier groups, each once
// it shows all 32 arrivals (their chunks hold earlier tickets, so they are
// running or done); warp 1 adds the state words of the earlier chunks of t's
// own group.  A chunk reads at most t / 32 + 31 words, where the look-back
// reads all t states of the chunks before it.  A wait that gives up records
// kErrTimeout and counts as 0, so the kernel always finishes.
__device__ uint64_t ck_group_prefix(const LookBack<1>& lb, const uint64_t* grp, uint32_t t,
                                    uint64_t* s_red) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t g = t >> 5;
  uint64_t part = 0;
  if (warp == 0) {
    for (uint32_t g0 = 0; g0 < g; g0 += 32) {
      const uint32_t gi = g0 + lane;
      if (gi >= g) continue;
      uint64_t w = ld_volatile_u64(grp + gi);
      uint32_t spins = 0, ns = 8;
      while ((w >> 32) != 32u) {
        if (++spins > kSpinLimit) break;
        __nanosleep(ns);
        if (ns < 256) ns <<= 1;
        w = ld_volatile_u64(grp + gi);
      }
      if ((w >> 32) == 32u) part += w & 0xffffffffull;
      else atomicOr(lb.status, kErrTimeout);
    }
  } else if (warp == 1) {
    const uint32_t ti = (g << 5) + (uint32_t)lane;
    if (ti < t) {
      uint64_t w = ld_volatile_u64(lb.st + ti);
      uint32_t spins = 0, ns = 8;
      while (lb_state<1>(lb, w) == 0) {
        if (++spins > kSpinLimit) break;
        __nanosleep(ns);
        if (ns < 256) ns <<= 1;
        w = ld_volatile_u64(lb.st + ti);
      }
      if (lb_state<1>(lb, w) != 0) part = w & kValueMask;
      else atomicOr(lb.status, kErrTimeout);
    }
  }
  if (warp < 2) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) part += __shfl_xor_sync(0xffffffffu, part, d);
    if (lane == 0) s_red[warp] = part;
  }
  __syncthreads();
  const uint64_t p = s_red[0] + s_red[1];
  __syncthreads();  // s_red is reused
  return p;
}

// Every CTA of a group-prefix launch calls this after its last read of the
// group words; the last one to arrive clears the `ngroups` group words and the
// finish counter, so the next launch on the same scratch starts from zeros.
__device__ __forceinline__ void ck_group_finish(uint64_t* grp, uint32_t* fin, uint32_t ngroups) {
  __shared__ uint32_t s_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();  // this CTA's group atomic is performed before it counts as finished
    s_last = atomicAdd(fin, 1u) == gridDim.x - 1 ? 1u : 0u;
    if (s_last) __threadfence();
  }
  __syncthreads();
  if (s_last) {
    for (uint32_t i = threadIdx.x; i < ngroups; i += blockDim.x) grp[i] = 0ull;
    if (threadIdx.x == 0) *fin = 0u;
  }
}

// Step 5: survivors i = tid, tid + 256, ... of NC columns, U per thread in flight.
template <int NC, int U>
__device__ __forceinline__ void ck_write(const SieveArgs& a, int64_t cbase, uint64_t prefix,
                                         uint32_t total, const uint16_t* s_list) {
  for (uint32_t i0 = threadIdx.x; i0 < total; i0 += U * kCkThreads) {
    int32_t v[NC][U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const uint32_t i = i0 + u * kCkThreads;
      const int64_t row = cbase + (i < total ? s_list[i] : 0);
#pragma unroll
      for (int c = 0; c < NC; ++c)
        if (c < a.nout && i < total) v[c][u] = __ldcs(a.in[c] + row);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const uint32_t i = i0 + u * kCkThreads;
#pragma unroll
      for (int c = 0; c < NC; ++c)
        if (c < a.nout && i < total) a.out[c][prefix + i] = v[c][u];
    }
  }
}

// Step 6: clear words [W(p0), W(p1)) of every filter the next builds write.
__device__ __forceinline__ void ck_zero(const SieveArgs& a, uint64_t p0, uint64_t p1, bool first) {
  for (int z = 0; z < a.nzero; ++z) {
    const uint64_t bpk = a.zero_bpk[z];
    uint64_t lo = 8 * ((bpk * p0 + 255) / 256);
    uint64_t hi = 8 * ((bpk * p1 + 255) / 256);
    if (first) {
      lo = 0;
      if (hi < 8) hi = 8;
    }
    if (hi > a.zero_cap_words[z]) hi = a.zero_cap_words[z];
    uint4* q = reinterpret_cast<uint4*>(a.zero_words[z]);
    for (uint64_t i = lo / 4 + threadIdx.x; i < hi / 4; i += kCkThreads) q[i] = make_uint4(0, 0, 0, 0);
  }
}

// Steps 3 and 5 of a chunk whose survivor bits (s_bits) and tile offsets
// (s_toff, ntile + 1 entries) are known: survivors are listed kCkList ranks
// per round in shared memory (row offsets in the chunk) and written, round by
// round.  `resolve` runs once, between the first round's listing and its
// writes (all threads call it), and returns the chunk's output offset.
template <class Resolve>
__device__ __forceinline__ uint64_t ck_list_and_write(const SieveArgs& a, int64_t cbase, int ntile,
                                                      uint32_t total, const uint32_t* s_bits,
                                                      const uint32_t* s_toff, uint16_t* s_list,
                                                      Resolve resolve) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint64_t prefix = 0;
  for (uint32_t r0 = 0; r0 == 0 || r0 < total; r0 += kCkList) {
    const uint32_t r1 = r0 + kCkList;
    if (r0 > 0) __syncthreads();  // the previous round's list is consumed
    for (int T = warp; T < ntile; T += kCkThreads / 32) {
      const uint32_t tb = s_toff[T];
      if (tb >= r1 || s_toff[T + 1] <= r0) continue;  // no rank of this round (warp-uniform)
      const uint32_t wj = lane < 8 ? s_bits[T * 8 + lane] : 0u;
      const uint32_t cj = __popc(wj);
      uint32_t inc = cj;
#pragma unroll
      for (int d = 1; d < 8; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, d);
        if (lane >= d) inc += y;
      }
      const uint32_t exj = inc - cj;
      uint32_t nz = __ballot_sync(0xffffffffu, wj != 0u);
      while (nz) {
        const int j = __ffs(nz) - 1;
        nz &= nz - 1;
        const uint32_t bj = __shfl_sync(0xffffffffu, wj, j);
        const uint32_t ej = __shfl_sync(0xffffffffu, exj, j);
        const uint32_t rank = tb + ej + __popc(bj & lanemask_lt());
        if (((bj >> lane) & 1u) && rank >= r0 && rank < r1)
          s_list[rank - r0] = (uint16_t)(T * kCkTileRows + 32 * j + lane);
      }
    }
    if (r0 == 0) prefix = resolve();
    __syncthreads();  // this round's list is complete
    const uint32_t m = total - r0 < (uint32_t)kCkList ? total - r0 : (uint32_t)kCkList;
    if (a.nout <= 2) ck_write<2, 4>(a, cbase, prefix + r0, m, s_list);
    else if (a.nout <= 4) ck_write<4, 2>(a, cbase, prefix + r0, m, s_list);
    else ck_write<kMaxCols, 1>(a, cbase, prefix + r0, m, s_list);
  }
  return prefix;
}

// Shared memory of one chunk of the chunked sieve.
struct CkSmem {
  static constexpr int kMaxTiles = kCkMaxRows / kCkTileRows;
  __align__(16) uint32_t bits[kMaxTiles * 8];
  uint32_t toff[kMaxTiles + 1];
  uint16_t list[kCkList];               // phase 1: each warp's 256-entry row list (generic tests)
  uint32_t wbits[kCkThreads / 32][8];   // phase 1: each warp's survivor words (generic tests)
  Vec<1> warp[kCkThreads / 32];
  uint64_t red[kCkThreads / 32];
  int stop;
};
static_assert(kCkList >= (kCkThreads / 32) * kCkTileRows, "a warp's row list needs 256 entries");

// Chunk t of the sieve step `a` (steps 1-6 of k_sieve_chunk); every thread of
// the CTA calls it.
template <int K>
__device__ __forceinline__ void ck_run_chunk(const SieveArgs& a, uint32_t t, CkSmem& sm) {
  uint32_t* s_bits = sm.bits;
  uint32_t* s_toff = sm.toff;
  uint16_t* s_list = sm.list;
  Vec<1>* s_warp = sm.warp;
  uint64_t* s_red = sm.red;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t n = a.n_dev ? (int64_t)(*a.n_dev) : a.n_host;
  const int64_t C = a.chunk_rows;
  const int64_t nchunks = (n + C - 1) / C;
  if ((int64_t)t >= nchunks) {
    if (t == 0) {  // empty input
      if (tid == 0) {
        *a.out_n = 0;
        if (a.out_n2) *a.out_n2 = 0;
      }
      ck_zero(a, 0, 0, true);
    }
    return;
  }
  const int64_t cbase = (int64_t)t * C;
  const int64_t crows = n - cbase < C ? n - cbase : C;
  const int ntile = (int)((crows + kCkTileRows - 1) / kCkTileRows);

  // 1. probe
  {
    const int32_t* col0 = a.ntest > 0 ? a.test[0].col : nullptr;
    uint32_t nwords = 0;
    Key32Hash hf = {0, 0, 0};
    uint64_t pol = 0;
    if (K > 0) {
      nwords = (uint32_t)(__ldg(a.test[0].f.hdr) * 8);
      hf = key32_hash_fold(a.test[0].f.seed);
      pol = l2_evict_last_policy();
    }
    int32_t cur[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) cur[j] = 0;
    if (warp < ntile && col0) ck_load8(col0, cbase + (int64_t)warp * kCkTileRows, n, lane, cur);
    for (int T = warp; T < ntile; T += kCkThreads / 32) {
      const int64_t base = cbase + (int64_t)T * kCkTileRows;
      // the warp's next tile loads while this one is tested
      int32_t nxt[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) nxt[j] = 0;
      const int Tn = T + kCkThreads / 32;
      if (Tn < ntile && col0) ck_load8(col0, cbase + (int64_t)Tn * kCkTileRows, n, lane, nxt);
      uint32_t b[8];
      if (K > 0) ck_test_reg32<(K > 0 ? K : 1)>(a.test[0].f.words, nwords, hf, pol, cur, base, n, lane, b);
      else ck_test_generic(a, cur, base, n, lane, b, s_list + warp * kCkTileRows, sm.wbits[warp]);
      if (lane == 0) {
        uint4* d = reinterpret_cast<uint4*>(s_bits + T * 8);
        d[0] = make_uint4(b[0], b[1], b[2], b[3]);
        d[1] = make_uint4(b[4], b[5], b[6], b[7]);
      }

#pragma unroll
      for (int j = 0; j < 8; ++j) cur[j] = nxt[j];
    }
  }
  __syncthreads();

  // 2. count: tile offsets and the chunk total
  uint32_t total;
  {
    uint32_t c = 0;
    if (tid < ntile) {
      const uint4 x = reinterpret_cast<const uint4*>(s_bits)[2 * tid];
      const uint4 y = reinterpret_cast<const uint4*>(s_bits)[2 * tid + 1];
      c = __popc(x.x) + __popc(x.y) + __popc(x.z) + __popc(x.w) + __popc(y.x) + __popc(y.y) +
          __popc(y.z) + __popc(y.w);
    }
    Vec<1> cv, tot;
    cv.v[0] = c;
    const Vec<1> ex = block_exclusive_scan<1, kCkThreads>(cv, &tot, s_warp);
    if (tid < ntile) s_toff[tid] = (uint32_t)ex.v[0];
    total = (uint32_t)tot.v[0];
    if (tid == 0) s_toff[ntile] = total;
  }
  if (tid == 0) {
    Vec<1> agg;
    agg.v[0] = total;
    lb_publish<1>(a.lb, t, (t == 0 && !a.grp) ? 2u : 1u, agg);
    if (a.grp) atomicAdd(reinterpret_cast<unsigned long long*>(a.grp + (t >> 5)), (1ull << 32) | total);
  }
  __syncthreads();

  // 3.-5. survivors listed, offset (group prefix or look-back), writes
  const uint64_t prefix = ck_list_and_write(a, cbase, ntile, total, s_bits, s_toff, s_list, [&]() {
    uint64_t p = 0;
    if (a.grp) {
      p = ck_group_prefix(a.lb, a.grp, t, s_red);
    } else if (t > 0) {
      p = ck_lookback(a.lb, t, &sm.stop, s_red);
      if (tid == 0) {
        Vec<1> inc;
        inc.v[0] = p + total;
        lb_publish<1>(a.lb, t, 2u, inc);
      }
    }
    if ((int64_t)t == nchunks - 1 && tid == 0) {
      *a.out_n = p + total;
      if (a.out_n2) *a.out_n2 = p + total;
    }
    return p;
  });

  // 6. clear the next filters' words
  ck_zero(a, prefix, prefix + total, t == 0);
}

template <int K>
__global__ void __launch_bounds__(kCkThreads, K > 0 ? kCkMinBlocks : 4) k_sieve_chunk(SieveArgs a) {
  __shared__ CkSmem sm;
  __shared__ uint32_t s_ticket;
  if (threadIdx.x == 0) s_ticket = draw_ticket(a.tile_counter);
  __syncthreads();
  ck_run_chunk<K>(a, s_ticket, sm);
  if (a.grp) {
    const int64_t n = a.n_dev ? (int64_t)(*a.n_dev) : a.n_host;
    const int64_t nchunks = (n + a.chunk_rows - 1) / a.chunk_rows;
    ck_group_finish(a.grp, a.fin, (uint32_t)((nchunks + 31) / 32));
  }
}

// Many sieve steps in one launch (the serving runtime's batches): task i's
// chunks are the global tickets [chunk0[i], chunk0[i + 1]), numbered from the
// tasks' row bounds; a CTA draws a global ticket, finds its task by binary
// search, copies the task's arguments to shared memory and runs that chunk
// of that task.  A chunk waits (look-back) only on earlier chunks of its own
// task, which hold earlier tickets, so the tasks run as one stream of work.
template <int K>
__global__ void __launch_bounds__(kCkThreads, 4) k_sieve_batch(SieveBatchArgs b) {
  __shared__ CkSmem sm;
  __shared__ SieveArgs s_args;
  __shared__ uint32_t s_ticket;
  __shared__ int s_task;
  if (threadIdx.x == 0) {
    const uint32_t g = draw_ticket(b.ticket);
    int lo = 0, hi = b.ntask - 1;  // last task whose first chunk is <= g
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if ((uint64_t)__ldg(b.chunk0 + mid) <= g) lo = mid;
      else hi = mid - 1;
    }
    s_task = lo;
    s_ticket = g - (uint32_t)__ldg(b.chunk0 + lo);
  }
  __syncthreads();
  const uint32_t* src = reinterpret_cast<const uint32_t*>(b.tasks + s_task);
  uint32_t* dst = reinterpret_cast<uint32_t*>(&s_args);
  for (int i = threadIdx.x; i < (int)(sizeof(SieveArgs) / 4); i += kCkThreads) dst[i] = __ldg(src + i);
  __syncthreads();
  ck_run_chunk<K>(s_args, s_ticket, sm);
}

// ---------------------------------------------------------------- insert maintenance
__global__ void __launch_bounds__(kBlock) k_insert_check(InsertArgs a) {
  __shared__ unsigned long long s_c[3];
  if (threadIdx.x < 3) s_c[threadIdx.x] = 0ull;
  __syncthreads();
  const uint64_t nb = __ldg(a.f.hdr);
  unsigned long long c[3] = {0ull, 0ull, 0ull};
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride) {
    bool pass = true;
    for (int g = 0; g < a.ngate && pass; ++g)
      pass = filter_contains(a.gate[g].f, __ldg(a.gate[g].f.hdr), __ldg(a.gate[g].col + i));
    uint8_t st = 0;
    if (pass) st = filter_contains(a.f, nb, __ldg(a.keys + i)) ? 1 : 2;
    a.status[i] = st;
    c[st] += 1;
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    unsigned long long v = c[k];
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(&s_c[k], v);
  }
  __syncthreads();
  if (threadIdx.x < 3 && s_c[threadIdx.x]) atomicAdd(a.counts + threadIdx.x, s_c[threadIdx.x]);
}

// Set the k bits of `key` in a filter of nb blocks (any layout).
__device__ __forceinline__ void filter_or_key(uint32_t* words, uint64_t nb, uint32_t k, uint32_t layout,
                                              uint64_t seed, int32_t key) {
  const uint64_t h = key_hash(key, seed);
  if (layout == 0) {
    atomicOr(words + reg32_word(h, nb * 8), reg32_mask((uint32_t)h, k));
  } else if (layout == 1) {
    const uint64_t blk = ((h >> 32) * nb) >> 32;
    for (uint32_t i = 0; i < k; ++i) {
      const uint32_t bit = (uint32_t)(h >> (8 * i)) & 255u;
      atomicOr(words + blk * 8 + (bit >> 5), 1u << (bit & 31));
    }
  } else {
    const uint64_t m = nb * 256ull;
    const uint64_t h1 = h & 0xffffffffull;
    const uint64_t h2 = (h >> 32) | 1ull;
    for (uint32_t i = 0; i < k; ++i) {
      const uint64_t g = (h1 + (uint64_t)i * h2) % m;
      atomicOr(words + (g >> 5), 1u << (g & 31));
    }
  }
}

__global__ void __launch_bounds__(kBlock) k_insert_or(InsertArgs a) {
  const uint64_t nb = __ldg(a.f.hdr);
  if (blockIdx.x == 0 && threadIdx.x == 0) a.hdr[1] += a.counts[2];
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride)
    if (a.status[i] == 2) filter_or_key(a.words, nb, a.f.k, a.f.layout, a.f.seed, __ldg(a.keys + i));
}

// ---------------------------------------------------------------- batched Bloom build
// Many filter builds in one launch: task i's rows are the global rows
// [row0[i], row0[i + 1]) (from the tasks' row bounds); each thread takes rows
// by grid stride, finds the task by binary search and ORs the key's bits in
// (any layout).  The row with local index 0 writes the task's header.
__global__ void __launch_bounds__(kBlock) k_bloom_build_batch(BuildBatchArgs b) {
  const int64_t total = __ldg(b.row0 + b.ntask);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int task = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) {
    if (__ldg(b.row0 + task + 1) <= i || __ldg(b.row0 + task) > i) {
      int lo = 0, hi = b.ntask - 1;  // last task starting at or before i
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(b.row0 + mid) <= i) lo = mid;
        else hi = mid - 1;
      }
      task = lo;
    }
    const BloomBuildArgs& t = b.tasks[task];
    const int64_t r = i - __ldg(b.row0 + task);
    const int64_t n = t.n_dev ? (int64_t)__ldg(t.n_dev) : t.n_host;
    uint64_t nb = ((uint64_t)t.bits_per_key * (uint64_t)n + 255ull) / 256ull;
    if (nb < 1) nb = 1;
    if (nb > t.nblocks_cap) nb = t.nblocks_cap;
    if (r == 0) {
      t.hdr[0] = nb;
      t.hdr[1] = (uint64_t)n;
    }
    if (r < n) filter_or_key(t.words, nb, t.k, t.layout, t.seed, __ldg(t.keys + r));
  }
}

// ---------------------------------------------------------------- group offsets
__global__ void __launch_bounds__(kBlock) k_group_offsets(GroupOffArgs a) {
  __shared__ Vec<2> s_warp[kBlock / 32];
  __shared__ unsigned long long s_base;
  const int tid = threadIdx.x;
  const int64_t n = a.n_dev ? (int64_t)__ldg(a.n_dev) : a.n_host;
  const int64_t ntiles = (n + kGroupTile - 1) / kGroupTile;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t base = tile * kGroupTile;
    uint32_t x[8];
#pragma unroll
    for (int v = 0; v < 2; ++v) {
      const int64_t r0 = base + (int64_t)(v * kBlock + tid) * 4;
      if (r0 + 4 <= n) {
        const uint4 q = __ldg(reinterpret_cast<const uint4*>(a.cnt + r0));
        x[4 * v] = q.x;
        x[4 * v + 1] = q.y;
        x[4 * v + 2] = q.z;
        x[4 * v + 3] = q.w;
      } else {
#pragma unroll
        for (int e = 0; e < 4; ++e) x[4 * v + e] = (r0 + e < n) ? __ldg(a.cnt + r0 + e) : 0u;
      }
    }
    Vec<2> sv, tot;
    sv.v[0] = (uint64_t)x[0] + x[1] + x[2] + x[3];
    sv.v[1] = (uint64_t)x[4] + x[5] + x[6] + x[7];
    const Vec<2> ex = block_exclusive_scan<2>(sv, &tot, s_warp);
    if (tid == 0) s_base = atomicAdd(a.cursor, (unsigned long long)(tot.v[0] + tot.v[1]));
    __syncthreads();
    const uint64_t gb = s_base;
#pragma unroll
    for (int v = 0; v < 2; ++v) {
      uint64_t run = gb + (v ? tot.v[0] : 0) + ex.v[v];
      const int64_t r0 = base + (int64_t)(v * kBlock + tid) * 4;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        if (r0 + e < n) a.off[r0 + e] = run;
        run += x[4 * v + e];
      }
    }
    __syncthreads();  // s_base is rewritten by the next tile
  }
}

// ---------------------------------------------------------------- hash tables
// Slot holding `key` (the key in the low word, 1 in the high word so that key
// 0 differs from an empty slot); inserted if absent.  Returns -1 with
// kErrTableFull when the probe sequence is exhausted.  A multimap groups its
// rows by this slot index, so no dense key ids (and no shared id counter) are
// needed.
__device__ __forceinline__ int64_t table_find_or_insert(const Table& t, int32_t key,
                                                      uint32_t* status) {
  uint32_t b = table_bucket(key, t.bucket_mask);
  const unsigned long long want = (1ull << 32) | (uint32_t)key;
  for (uint32_t step = 0; step <= t.bucket_mask; ++step) {
    unsigned long long* bk = t.slots + (uint64_t)b * 4;
#pragma unroll 1
    for (int s = 0; s < 4; ++s) {
      unsigned long long v = ld_volatile_u64(reinterpret_cast<const uint64_t*>(bk + s));
      if (v == 0) {
        v = atomicCAS(bk + s, 0ull, want);
        if (v == 0) return (int64_t)b * 4 + s;
      }
      if (v == want) return (int64_t)b * 4 + s;
    }
    b = (b + 1) & t.bucket_mask;
  }
  atomicOr(status, kErrTableFull);
  return -1;
}

// Read-only lookup after the build finished, starting at bucket b: slot index
// of `key`, or -1.
__device__ __forceinline__ int64_t table_find_at(const Table& t, int32_t key, uint32_t b) {
  const uint64_t lo = (uint32_t)key;
  for (uint32_t step = 0; step <= t.bucket_mask; ++step) {
    const ulonglong2* p = reinterpret_cast<const ulonglong2*>(t.slots + (uint64_t)b * 4);
    const ulonglong2 q0 = __ldg(p);
    const ulonglong2 q1 = __ldg(p + 1);
    const uint64_t sl[4] = {q0.x, q0.y, q1.x, q1.y};
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      if (sl[s] == 0) return -1;
      if ((sl[s] & 0xffffffffull) == lo) return (int64_t)b * 4 + s;
    }
    b = (b + 1) & t.bucket_mask;
  }
  return -1;
}
__device__ __forceinline__ int64_t table_find(const Table& t, int32_t key) {
  return table_find_at(t, key, table_bucket(key, t.bucket_mask));
}

// Slot of `key` when it sits in one of the first two slots of its home
// bucket (the common case at load <= 1/2), -1 when that half-bucket shows it
// absent, else the full probe.
__device__ __forceinline__ int64_t table_find_first(const Table& t, int32_t key, uint32_t b,
                                                    ulonglong2 q) {
  const uint64_t lo = (uint32_t)key;
  if (q.x == 0) return -1;
  if ((q.x & 0xffffffffull) == lo) return (int64_t)b * 4;
  if (q.y == 0) return -1;
  if ((q.y & 0xffffffffull) == lo) return (int64_t)b * 4 + 1;
  return table_find_at(t, key, b);
}

// Per-CTA aggregation of skewed keys: a CTA takes kAggRows rows per round and
// combines the rows of each key in a shared-memory table before touching the
// global table, so a key repeated r times in a round costs one global insert
// and one global atomic instead of r: the thread that entered the key in the
// shared table (its leader) does both for the whole round.  Without it, the
// first rows of a Zipf-hot key would all race on the same global slot with
// compare-and-swaps that serialise.
constexpr int kAggPerThread = 2;
constexpr int kAggRows = kBlock * kAggPerThread;
constexpr int kAggSlotsLog2 = 10;
constexpr int kAggSlots = 1 << kAggSlotsLog2;  // 2x the rows of a round: never full
static_assert(kAggSlots >= 2 * kAggRows, "per-CTA table must hold every key of a round");

// Shared-memory entry of `key` (entries hold (1 << 32) | key, 0 = empty),
// inserted if absent; *lead is set for the one caller that inserted it.
// Returns -1 if the table is full.
__device__ __forceinline__ int smem_key_slot(unsigned long long* s_key, int32_t key, bool* lead) {
  const unsigned long long want = (1ull << 32) | (uint32_t)key;
  uint32_t h = ((uint32_t)key * 2654435761u) >> (32 - kAggSlotsLog2);
  *lead = false;
  for (int p = 0; p < kAggSlots; ++p) {
    const unsigned long long cur = s_key[h];
    if (cur == want) return (int)h;
    if (cur == 0ull) {
      const unsigned long long old = atomicCAS(s_key + h, 0ull, want);
      if (old == 0ull) {
        *lead = true;
        return (int)h;
      }
      if (old == want) return (int)h;
    }
    h = (h + 1) & (kAggSlots - 1);
  }
  return -1;
}

__global__ void __launch_bounds__(kBlock) k_mm_insert(MMInsertArgs a) {
  __shared__ unsigned long long s_key[kAggSlots];  // tagged key, 0 = empty
  __shared__ uint32_t s_cnt[kAggSlots];            // rows of the round, then their global base
  __shared__ uint32_t s_slot[kAggSlots];           // the key's table slot, 0xffffffff = none
  a.t = resolve(a.t);
  a.n = dev_n(a.n_dev, a.n);
  const int tid = threadIdx.x;
  for (int64_t r0 = (int64_t)blockIdx.x * kAggRows; r0 < a.n; r0 += (int64_t)gridDim.x * kAggRows) {
    for (int i = tid; i < kAggSlots; i += kBlock) {
      s_key[i] = 0ull;
      s_cnt[i] = 0;
    }
    __syncthreads();
    int32_t key[kAggPerThread];
    int j[kAggPerThread];
    bool lead[kAggPerThread];
    uint32_t lr[kAggPerThread];
    int64_t sl[kAggPerThread];  // rows of a full shared table go straight to the global one
#pragma unroll
    for (int e = 0; e < kAggPerThread; ++e) {
      const int64_t row = r0 + e * kBlock + tid;
      j[e] = -1;
      lead[e] = false;
      lr[e] = 0;
      sl[e] = -1;
      if (row < a.n) {
        key[e] = __ldcs(a.keys + row);
        j[e] = smem_key_slot(s_key, key[e], &lead[e]);
        if (j[e] >= 0) {
          lr[e] = atomicAdd(s_cnt + j[e], 1u);
        } else {
          sl[e] = table_find_or_insert(a.t, key[e], a.status);
          if (sl[e] >= 0) lr[e] = atomicAdd(a.cnt + sl[e], 1u);
        }
      }
    }
    __syncthreads();
#pragma unroll
    for (int e = 0; e < kAggPerThread; ++e) {
      if (!lead[e]) continue;
      const int64_t g = table_find_or_insert(a.t, key[e], a.status);
      s_slot[j[e]] = g >= 0 ? (uint32_t)g : 0xffffffffu;
      if (g >= 0) s_cnt[j[e]] = atomicAdd(a.cnt + g, s_cnt[j[e]]);
    }
    __syncthreads();
#pragma unroll
    for (int e = 0; e < kAggPerThread; ++e) {
      const int64_t row = r0 + e * kBlock + tid;
      if (j[e] >= 0) {
        const uint32_t g = s_slot[j[e]];
        if (g != 0xffffffffu) {
          a.rid[row] = g;
          a.rank[row] = s_cnt[j[e]] + lr[e];
        }
      } else if (sl[e] >= 0) {
        a.rid[row] = (uint32_t)sl[e];
        a.rank[row] = lr[e];
      }
    }
    __syncthreads();  // the table is cleared by the next round
  }
}

__global__ void __launch_bounds__(kBlock) k_mm_scatter(MMScatterArgs a) {
  a.n = dev_n(a.n_dev, a.n);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride)
    a.rows[__ldg(a.off + __ldg(a.rid + i)) + __ldg(a.rank + i)] = (int32_t)i;
}

__global__ void __launch_bounds__(kBlock) k_mm_probe(MMProbeArgs a) {
  __shared__ uint32_t s_tile;
  __shared__ Vec<3> s_warp[kBlock / 32];
  __shared__ uint64_t s_prefix[2];
  const int tid = threadIdx.x;
  a.t = resolve(a.t);
  const int64_t n = dev_n(a.n_dev, a.n);
  const int64_t ntiles = (n + kProbeTile - 1) / kProbeTile;
  for (;;) {
  if (tid == 0) s_tile = draw_ticket_loop(a.tile_counter, (uint64_t)ntiles);
  __syncthreads();
  const uint32_t tile = s_tile;
  if ((int64_t)tile >= ntiles) {
    if (tile == 0 && tid == 0) {
      a.totals[0] = 0;
      a.totals[1] = 0;
    }
    break;
  }
  const int64_t base = (int64_t)tile * kProbeTile;
  // the 8 keys of a thread, then their 8 home half-buckets read together,
  // then the row counts of the hits together: three round trips per tile
  int32_t kk[8];
  uint32_t okm = 0;
#pragma unroll
  for (int v = 0; v < 2; ++v) {
    const int64_t r0 = base + (int64_t)(v * kBlock + tid) * 4;
    if (r0 + 4 <= n) {
      const int4 x = __ldcs(reinterpret_cast<const int4*>(a.keys + r0));
      kk[4 * v] = x.x; kk[4 * v + 1] = x.y; kk[4 * v + 2] = x.z; kk[4 * v + 3] = x.w;
      okm |= 0xfu << (4 * v);
    } else {
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        kk[4 * v + e] = 0;
        if (r0 + e < n) {
          kk[4 * v + e] = __ldcs(a.keys + r0 + e);
          okm |= 1u << (4 * v + e);
        }
      }
    }
  }
  uint32_t bk[8];
  ulonglong2 q[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    bk[j] = table_bucket(kk[j], a.t.bucket_mask);
    q[j] = ((okm >> j) & 1u) ? __ldg(reinterpret_cast<const ulonglong2*>(a.t.slots + (uint64_t)bk[j] * 4))
                             : make_ulonglong2(0ull, 0ull);
  }
  int32_t id[8];
  uint32_t m[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int64_t s = ((okm >> j) & 1u) ? table_find_first(a.t, kk[j], bk[j], q[j]) : -1;
    id[j] = (int32_t)s;
  }
#pragma unroll
  for (int j = 0; j < 8; ++j) m[j] = id[j] >= 0 ? __ldg(a.cnt + id[j]) : 0u;
  // scan channels: [0] hit counts of chunks 0 and 1 packed (32 bits each),
  // [1] output tuples of chunk 0, [2] output tuples of chunk 1
  Vec<3> c;
  uint32_t hits[2] = {0, 0};
  uint64_t msum[2] = {0, 0};
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    hits[i >> 2] += m[i] ? 1u : 0u;
    msum[i >> 2] += m[i];
  }
  c.v[0] = (uint64_t)hits[0] | ((uint64_t)hits[1] << 32);
  c.v[1] = msum[0];
  c.v[2] = msum[1];
  Vec<3> tot;
  const Vec<3> ex = block_exclusive_scan<3>(c, &tot, s_warp);
  const uint64_t hits0 = tot.v[0] & 0xffffffffull, hits1 = tot.v[0] >> 32;
  const uint64_t tile_hits = hits0 + hits1;
  const uint64_t tile_tuples = tot.v[1] + tot.v[2];
  if (tid < 32) {
    Vec<2> aggv;
    aggv.v[0] = tile_hits;
    aggv.v[1] = tile_tuples;
    if (tile == 0) {
      if (tid == 0) {
        lb_publish<2>(a.lb, 0, 2, aggv);
        s_prefix[0] = 0;
        s_prefix[1] = 0;
      }
    } else {
      if (tid == 0) lb_publish<2>(a.lb, tile, 1, aggv);
      const Vec<2> e = lb_exclusive<2>(a.lb, tile);
      if (tid == 0) {
        Vec<2> incv;
        incv.v[0] = e.v[0] + tile_hits;
        incv.v[1] = e.v[1] + tile_tuples;
        lb_publish<2>(a.lb, tile, 2, incv);
        s_prefix[0] = e.v[0];
        s_prefix[1] = e.v[1];
      }
    }
  }
  __syncthreads();
  const uint64_t p_hits = s_prefix[0], p_tuples = s_prefix[1];
  if ((int64_t)tile == ntiles - 1 && tid == 0) {
    a.totals[0] = p_hits + tile_hits;
    a.totals[1] = p_tuples + tile_tuples;
  }
#pragma unroll
  for (int v = 0; v < 2; ++v) {
    uint64_t q = p_hits + (v ? hits0 : 0) + ((ex.v[0] >> (32 * v)) & 0xffffffffull);
    uint64_t o = p_tuples + (v ? tot.v[1] : 0) + ex.v[1 + v];
    const int64_t r0 = base + (int64_t)(v * kBlock + tid) * 4;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      if (m[4 * v + e]) {
        a.prow[q] = (int32_t)(r0 + e);
        a.pid[q] = id[4 * v + e];
        a.o[q] = o;
        ++q;
        o += m[4 * v + e];
      }
    }
  }
  }  // tile loop (the scan's barriers order s_tile / s_prefix reuse)
}

// Largest q in [lo, hi] with o[q] <= j (o strictly increasing, o[lo] <= j),
// by a whole warp: each round the 32 lanes test 32 evenly spaced entries and
// keep the interval after the last one that is <= j, so a search over Q
// entries takes about log32(Q) dependent loads instead of the log2(Q) of a
// per-thread binary search.  All lanes return the answer.
__device__ __forceinline__ uint64_t warp_upper_q(const uint64_t* o, uint64_t lo, uint64_t hi,
                                                 uint64_t j) {
  const int lane = threadIdx.x & 31;
  for (;;) {
    const uint64_t n = hi - lo + 1;
    const uint64_t step = n <= 32 ? 1 : (n + 31) / 32;  // 32 steps cover [lo, hi]
    const uint64_t pos = lo + (uint64_t)lane * step;
    const bool le = pos <= hi && __ldg(o + pos) <= j;
    const uint32_t m = __ballot_sync(0xffffffffu, le);  // lane 0 always: o[lo] <= j
    const int k = 31 - __clz(m);
    if (step == 1) return lo + (uint64_t)k;
    const uint64_t nlo = lo + (uint64_t)k * step;
    const uint64_t nhi = nlo + step - 1;
    lo = nlo;
    if (nhi < hi) hi = nhi;
  }
}

// Expansion: one thread per output tuple j; its hit is the largest q with
// o[q] <= j and its build row the (j - o[q])-th row of that key's group, so a
// hot key's fan-out is spread over as many threads as it has outputs.  A CTA
// takes kExpRange consecutive outputs [J0, J1): warps 0 and 1 find the hits
// holding J0 and J1 - 1 (warp_upper_q), the offsets of the hits in between
// (at most kExpRange, as every hit has at least one output) go to shared
// memory, and each thread finds its output's hit there, so an output waits on
// a few global round trips instead of a binary search through global memory.
constexpr int kExpRange = kBlock;
__device__ __forceinline__ void expand_ranges(const MMExpandArgs& a, uint64_t Q, uint64_t lim) {
  __shared__ uint64_t s_o[kExpRange];
  __shared__ uint64_t s_q[2];
  const int tid = threadIdx.x, warp = tid >> 5;
  for (uint64_t J0 = (uint64_t)blockIdx.x * kExpRange; J0 < lim; J0 += (uint64_t)gridDim.x * kExpRange) {
    const uint64_t J1 = J0 + kExpRange < lim ? J0 + kExpRange : lim;
    if (warp < 2) {
      const uint64_t q = warp_upper_q(a.o, 0, Q - 1, warp == 0 ? J0 : J1 - 1);
      if ((tid & 31) == 0) s_q[warp] = q;
    }
    __syncthreads();
    const uint64_t q0 = s_q[0];
    const uint32_t nq = (uint32_t)(s_q[1] - q0 + 1);
    if ((uint32_t)tid < nq) s_o[tid] = __ldg(a.o + q0 + tid);
    __syncthreads();
    const uint64_t j = J0 + (uint64_t)tid;
    if (j < J1) {
      uint32_t lo = 0, hi = nq - 1;  // largest i with s_o[i] <= j; s_o[0] <= J0 <= j
      while (lo < hi) {
        const uint32_t mid = (lo + hi + 1) >> 1;
        if (s_o[mid] <= j) lo = mid;
        else hi = mid - 1;
      }
      const uint64_t q = q0 + lo;
      const uint64_t t = j - s_o[lo];
      const int32_t prow = __ldg(a.prow + q);
      const int32_t brow = __ldg(a.rows + __ldg(a.off + __ldg(a.pid + q)) + t);
#pragma unroll
      for (int c = 0; c < kMaxCols; ++c)
        if (c < a.nout) a.out[c][j] = __ldg(a.src[c] + (a.src_build[c] ? brow : prow));
      if (a.psum_out) {
        const uint64_t ps = a.psum_in ? __ldg(a.psum_in + prow) : term_sum(a.probe_terms, prow);
        a.psum_out[j] = ps + term_sum(a.build_terms, brow);
      }
    }
    __syncthreads();  // s_o and s_q are rewritten for the next range
  }
}

// Host-sized expand: T and Q known on the host.
__global__ void __launch_bounds__(kBlock) k_mm_expand(MMExpandArgs a) {
  if (a.T > 0) expand_ranges(a, a.Q, a.T);
}

// Device-sized expand: T and Q come from the probe's totals on the device;
// outputs beyond `cap` are not written and the overflow is reported, so the
// host can rerun the level with an exact buffer.
__global__ void __launch_bounds__(kBlock) k_mm_expand_dev(MMExpandArgs a) {
  const uint64_t Q = __ldg(a.totals_dev);
  const uint64_t T = __ldg(a.totals_dev + 1);
  const uint64_t lim = T < a.cap ? T : a.cap;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *a.n_out = lim;
    if (T > a.cap) atomicOr(a.status, kErrCapacity);
  }
  expand_ranges(a, Q, lim);
}

__global__ void __launch_bounds__(kBlock) k_table_init(TableInitArgs a) {
  const int64_t n = dev_n(a.n_dev, a.n_host);
  uint64_t nslots = 64;
  while (nslots < 2 * (uint64_t)n) nslots <<= 1;
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  if (gid == 0) {
    *a.mask_out = (uint32_t)(nslots / 4 - 1);
    if (a.nslots_out) *a.nslots_out = (uint32_t)nslots;
    if (a.zero64) *a.zero64 = 0ull;
  }
  for (int64_t i = gid; i < (int64_t)nslots; i += stride) {
    a.slots[i] = 0ull;
    if (a.pairs) a.pairs[i] = make_ulonglong2(0ull, 0ull);
  }
  if (a.cnt)
    for (int64_t i = gid; i < (int64_t)nslots; i += stride) a.cnt[i] = 0u;
}

// ---------------------------------------------------------------- aggregate level

__global__ void __launch_bounds__(kBlock, 4) k_agg_insert(AggInsertArgs a) {
  __shared__ unsigned long long s_key[kAggSlots];  // tagged key, 0 = empty
  __shared__ uint32_t s_cnt[kAggSlots];
  __shared__ unsigned long long s_sum[kAggSlots];
  a.t = resolve(a.t);
  a.n = dev_n(a.n_dev, a.n);
  const bool with_sum = a.terms.n || a.vals;
  const int tid = threadIdx.x;
  for (int64_t r0 = (int64_t)blockIdx.x * kAggRows; r0 < a.n; r0 += (int64_t)gridDim.x * kAggRows) {
    for (int i = tid; i < kAggSlots; i += kBlock) {
      s_key[i] = 0ull;
      s_cnt[i] = 0;
      s_sum[i] = 0ull;
    }
    __syncthreads();
    int32_t key[kAggPerThread];
    int j[kAggPerThread];
    bool lead[kAggPerThread];
#pragma unroll
    for (int e = 0; e < kAggPerThread; ++e) {
      const int64_t row = r0 + e * kBlock + tid;
      j[e] = -1;
      lead[e] = false;
      if (row < a.n) {
        key[e] = __ldcs(a.keys + row);
        const uint64_t val = with_sum ? (a.vals ? __ldg(a.vals + row) : term_sum(a.terms, row)) : 0ull;
        j[e] = smem_key_slot(s_key, key[e], &lead[e]);
        if (j[e] >= 0) {
          atomicAdd(s_cnt + j[e], 1u);
          if (with_sum) atomicAdd(s_sum + j[e], (unsigned long long)val);
        } else {  // full shared table: straight to the global one
          const int64_t sl = table_find_or_insert(a.t, key[e], a.status);
          if (sl >= 0) {
            atomicAdd(&a.cs[sl].x, 1ull);
            if (with_sum) atomicAdd(&a.cs[sl].y, (unsigned long long)val);
          }
        }
      }
    }
    __syncthreads();
#pragma unroll
    for (int e = 0; e < kAggPerThread; ++e) {
      if (!lead[e]) continue;
      const int64_t sl = table_find_or_insert(a.t, key[e], a.status);
      if (sl >= 0) {
        atomicAdd(&a.cs[sl].x, (unsigned long long)s_cnt[j[e]]);
        if (with_sum) atomicAdd(&a.cs[sl].y, s_sum[j[e]]);
      }
    }
    __syncthreads();  // the table is cleared by the next round
  }
}

struct U128 {
  uint64_t lo, hi;
};
__device__ __forceinline__ void add128(U128& x, uint64_t lo, uint64_t hi) {
  const uint64_t nl = x.lo + lo;
  x.hi += hi + (nl < x.lo ? 1ull : 0ull);
  x.lo = nl;
}

// One probe row per thread and iteration: the table is small and cache
// resident here, so occupancy (32 registers, 8 CTAs per SM) hides latency
// better than batching rows per thread.

// Probe of the final level's (count, sum) table.  The common shape -- a long
// probe relation whose SUM term is at most one int32 column -- takes 4 rows per
// thread with the next 4 keys already in flight, so each iteration waits on two
// table round trips only; a row's term is read only if its key matches.
__global__ void __launch_bounds__(kBlock, 4) k_agg_probe(AggProbeArgs a) {
  __shared__ uint64_t s_red[3][kBlock / 32];
  a.t = resolve(a.t);
  a.n = dev_n(a.n_dev, a.n);
  U128 cnt = {0, 0};
  uint64_t sum = 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int32_t* tcol = a.probe_terms.n == 1 ? a.probe_terms.col[0] : nullptr;
  const bool fast = ((reinterpret_cast<uintptr_t>(a.keys) & 15u) == 0) && !a.psum_in &&
                    a.probe_terms.n <= 1 &&
                    (!tcol || (!a.probe_terms.col_hi[0] && (reinterpret_cast<uintptr_t>(tcol) & 15u) == 0));
  int64_t tail = 0;
  if (fast) {
    const int64_t n4 = a.n / 4;
    tail = n4 * 4;
    const int4* k4 = reinterpret_cast<const int4*>(a.keys);
    int4 k = make_int4(0, 0, 0, 0);
    if (tid < n4) k = __ldcs(k4 + tid);
    for (int64_t g = tid; g < n4; g += stride) {
      int4 kn = make_int4(0, 0, 0, 0);
      if (g + stride < n4) kn = __ldcs(k4 + g + stride);
      const int32_t kk[4] = {k.x, k.y, k.z, k.w};
      int32_t vv[4];
      uint32_t b[4];
      ulonglong2 q[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        b[e] = table_bucket(kk[e], a.t.bucket_mask);
        q[e] = __ldg(reinterpret_cast<const ulonglong2*>(a.t.slots + (uint64_t)b[e] * 4));
      }
      int64_t sl[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) sl[e] = table_find_first(a.t, kk[e], b[e], q[e]);
      // the SUM term of a row is read only when its key matches, so rows
      // without a match cost no term read (a term column in host memory is
      // read only where a row matches)
      ulonglong2 cs[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        cs[e] = sl[e] >= 0 ? __ldg(a.cs + sl[e]) : make_ulonglong2(0ull, 0ull);
        vv[e] = (sl[e] >= 0 && tcol) ? __ldcs(tcol + 4 * g + e) : 0;
      }
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        add128(cnt, cs[e].x, 0);
        sum += (uint64_t)(int64_t)vv[e] * cs[e].x + cs[e].y;
      }
      k = kn;
    }
  }
  for (int64_t i = tail + tid; i < a.n; i += stride) {
    const int64_t s = table_find(a.t, __ldcs(a.keys + i));
    if (s < 0) continue;
    const ulonglong2 cs = __ldg(a.cs + s);  // count and sum share a sector
    const uint64_t ps = a.psum_in ? __ldg(a.psum_in + i) : term_sum(a.probe_terms, i);
    add128(cnt, cs.x, 0);
    sum += ps * cs.x + cs.y;
  }
  // block reduction of (count lo, count hi, sum)
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) {
    const uint64_t lo = __shfl_xor_sync(0xffffffffu, cnt.lo, d);
    const uint64_t hi = __shfl_xor_sync(0xffffffffu, cnt.hi, d);
    add128(cnt, lo, hi);
    sum += __shfl_xor_sync(0xffffffffu, sum, d);
  }
  if (lane == 0) {
    s_red[0][warp] = cnt.lo;
    s_red[1][warp] = cnt.hi;
    s_red[2][warp] = sum;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    U128 c = {0, 0};
    uint64_t sm = 0;
    for (int w = 0; w < kBlock / 32; ++w) {
      add128(c, s_red[0][w], s_red[1][w]);
      sm += s_red[2][w];
    }
    const unsigned long long old = atomicAdd(a.result + 0, (unsigned long long)c.lo);
    const uint64_t carry = (old + c.lo < old) ? 1ull : 0ull;
    if (c.hi + carry) atomicAdd(a.result + 1, (unsigned long long)(c.hi + carry));
    atomicAdd(a.result + 2, (unsigned long long)sm);
  }
}

__global__ void __launch_bounds__(kBlock) k_sum_terms(SumTermsArgs a) {
  __shared__ uint64_t s_red[kBlock / 32];
  uint64_t sum = 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride)
    sum += term_sum(a.terms, i);
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, d);
  if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = sum;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint64_t sm = 0;
    for (int w = 0; w < kBlock / 32; ++w) sm += s_red[w];
    atomicAdd(a.result + 2, (unsigned long long)sm);
  }
}


// ---------------------------------------------------------------- cyclic query
// Sec. 2.3: for a cyclic join the filter of the closing condition is rebuilt
// on the fly.  For E(a,b) |x| E(b,c) |x| E(c,a) the closing relation is E
// itself on the pair (c, a): a Bloom filter over packed edge pairs screens
// every wedge before the exact pair-set lookup.
__device__ __forceinline__ uint64_t pack_pair(int32_t s, int32_t d) {
  return ((uint64_t)(uint32_t)s << 32) | (uint32_t)d;
}

__global__ void __launch_bounds__(kBlock) k_pair_filter_build(PairFilterBuildArgs a) {
  __shared__ unsigned long long s_seen[kSeenSlots];
  for (int i = threadIdx.x; i < kSeenSlots; i += blockDim.x) s_seen[i] = 0ull;
  __syncthreads();
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    a.hdr[0] = a.nblocks;
    a.hdr[1] = (uint64_t)a.n;
  }
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride) {
    const uint64_t h = fmix64(pack_pair(__ldcs(a.src + i), __ldcs(a.dst + i)) ^ a.seed);
    uint32_t* p = a.words + reg32_word(h, a.nblocks * 8);
    const uint32_t m = reg32_mask((uint32_t)h, a.k);
    if ((__ldca(p) & m) != m && !seen_before(s_seen, h)) atomicOr(p, m);
  }
}

__device__ __forceinline__ uint32_t pair_bucket(uint64_t v, uint32_t mask) {
  return (uint32_t)fmix64(v ^ kTableSeed) & mask;
}

__global__ void __launch_bounds__(kBlock) k_pairset_insert(PairSetArgs a) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride) {
    const int32_t s = __ldcs(a.src + i), d = __ldcs(a.dst + i);
    if (s == d) continue;  // not an edge of the query (no self-loops); (-1, -1) would be the empty code
    const unsigned long long v = pack_pair(s, d) + 1ull;
    uint32_t b = pair_bucket(v, a.t.bucket_mask);
    bool done = false;
    for (uint32_t step = 0; step <= a.t.bucket_mask && !done; ++step) {
      unsigned long long* bk = a.t.slots + (uint64_t)b * 4;
#pragma unroll 1
      for (int s = 0; s < 4 && !done; ++s) {
        unsigned long long cur = ld_volatile_u64(reinterpret_cast<const uint64_t*>(bk + s));
        if (cur == 0) cur = atomicCAS(bk + s, 0ull, v);
        done = (cur == 0 || cur == v);
      }
      b = (b + 1) & a.t.bucket_mask;
    }
    if (!done) atomicOr(a.status, kErrTableFull);
  }
}

// Slots hold pair + 1 and 0 marks an empty slot; the one pair whose code is 0,
// (-1, -1), is a self-loop, which the set never holds, so self-loop pairs are
// answered without a lookup.
__device__ __forceinline__ bool pairset_contains(const Table& t, uint64_t pair) {
  if ((uint32_t)(pair >> 32) == (uint32_t)pair) return false;
  const unsigned long long v = pair + 1ull;
  uint32_t b = pair_bucket(v, t.bucket_mask);
  for (uint32_t step = 0; step <= t.bucket_mask; ++step) {
    const ulonglong2* p = reinterpret_cast<const ulonglong2*>(t.slots + (uint64_t)b * 4);
    const ulonglong2 q0 = __ldg(p);
    const ulonglong2 q1 = __ldg(p + 1);
    if (q0.x == v || q0.y == v || q1.x == v || q1.y == v) return true;
    if (q0.x == 0 || q0.y == 0 || q1.x == 0 || q1.y == 0) return false;
    b = (b + 1) & t.bucket_mask;
  }
  return false;
}

// Adjacency list (offset, length) of vertex v, or length 0.
__device__ __forceinline__ void adj_of(const Adjacency& g, int32_t v, uint64_t* off, uint32_t* len) {
  const int64_t s = table_find(g.t, v);
  if (s < 0) {
    *off = 0;
    *len = 0;
    return;
  }
  *off = __ldg(g.off + s);
  *len = __ldg(g.cnt + s);
}

// Persistent warps take 32 edges (a, b) at a time.  For each edge the warp
// walks the shorter of out(b) and in(a); a candidate c closes a triangle when
// the pair (c, a) [walking out(b)] or (b, c) [walking in(a)] is an edge: the
// pair filter screens it, the pair set confirms it.  Counts go to the
// subquery whose vertex range holds a.
// Each directed 3-cycle x -> y -> z -> x (distinct vertices: the edges are
// distinct and hold no self-loops) is the three ordered answers (x, y, z),
// (y, z, x) and (z, x, y).  It is enumerated once, from its smallest vertex:
// an edge (a, b) with a < b, and a third vertex c > a from the shorter of
// out(b) and in(a), checked against the closing pair (c, a) or (b, c); the
// three answers are then added to the subqueries of a, b and c.
__device__ __forceinline__ int sub_of(const int32_t* s_cuts, int nsub, int32_t v) {
  int lo = 0, hi = nsub;  // largest i with cuts[i] <= v
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (s_cuts[mid] <= v) lo = mid;
    else hi = mid - 1;
  }
  return lo < nsub ? lo : nsub - 1;
}

__global__ void __launch_bounds__(kBlock) k_triangles(TriangleArgs a) {
  __shared__ int32_t s_cuts[257];
  __shared__ unsigned long long s_cnt[256];
  for (int i = threadIdx.x; i <= a.nsub; i += blockDim.x) s_cuts[i] = a.cuts[i];
  for (int i = threadIdx.x; i < a.nsub; i += blockDim.x) s_cnt[i] = 0ull;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const uint64_t pnb = __ldg(a.pf.hdr);
  unsigned long long checked = 0, passed = 0;
  while (true) {
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(a.work, 32ull);
    base = __shfl_sync(0xffffffffu, base, 0);
    if (base >= (unsigned long long)a.ne) break;
    const int64_t e = (int64_t)base + lane;
    int32_t va = 0, vb = 0;
    uint64_t off = 0;
    uint32_t len = 0, side = 0;
    if (e < a.ne) {
      va = __ldg(a.src + e);
      vb = __ldg(a.dst + e);
      if (va < vb) {  // a is the cycle's smallest vertex only if a < b
        uint64_t o1, o2;
        uint32_t l1, l2;
        adj_of(a.out, vb, &o1, &l1);
        adj_of(a.in, va, &o2, &l2);
        side = l1 <= l2 ? 0u : 1u;
        off = side ? o2 : o1;
        len = side ? l2 : l1;
      }
    }
    for (int j = 0; j < 32; ++j) {
      const uint32_t L = __shfl_sync(0xffffffffu, len, j);
      if (L == 0) continue;
      const uint64_t O = __shfl_sync(0xffffffffu, off, j);
      const uint32_t S = __shfl_sync(0xffffffffu, side, j);
      const int32_t A = __shfl_sync(0xffffffffu, va, j);
      const int32_t B = __shfl_sync(0xffffffffu, vb, j);
      // the far endpoints, read contiguously from the neighbour arrays
      const int32_t* nbr = S ? a.in_nbr : a.out_nbr;
      unsigned long long found = 0;
      for (uint32_t t = lane; t < L; t += 32) {
        const int32_t v = __ldg(nbr + O + t);
        if (v <= A || v == B) continue;  // c must be above a (and differ from b)
        const uint64_t pair = S ? pack_pair(B, v) : pack_pair(v, A);
        ++checked;
        const uint64_t h = fmix64(pair ^ a.pf.seed);
        const uint32_t m = reg32_mask((uint32_t)h, a.pf.k);
        if ((__ldg(a.pf.words + reg32_word(h, pnb * 8)) & m) == m) {
          ++passed;
          if (pairset_contains(a.pairs, pair)) {
            ++found;
            atomicAdd(s_cnt + sub_of(s_cuts, a.nsub, v), 1ull);
          }
        }
      }
#pragma unroll
      for (int d = 16; d > 0; d >>= 1) found += __shfl_xor_sync(0xffffffffu, found, d);
      if (lane == 0 && found) {
        atomicAdd(s_cnt + sub_of(s_cuts, a.nsub, A), found);
        atomicAdd(s_cnt + sub_of(s_cuts, a.nsub, B), found);
      }
    }
  }
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) {
    checked += __shfl_xor_sync(0xffffffffu, checked, d);
    passed += __shfl_xor_sync(0xffffffffu, passed, d);
  }
  if (lane == 0) {
    atomicAdd(a.stats + 0, checked);
    atomicAdd(a.stats + 1, passed);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < a.nsub; i += blockDim.x)
    if (s_cnt[i]) atomicAdd(a.counts + i, s_cnt[i]);
}

__global__ void __launch_bounds__(kBlock) k_gather_i32(const int32_t* col, const int32_t* idx, int64_t n,
                                                      int32_t* out) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    out[i] = __ldg(col + __ldg(idx + i));
}

// Self-test of the bounded waits: one warp polls `flag` (which nothing sets)
// with the same bound and backoff as the look-back, then records a timeout.
__global__ void k_wait_flag(const uint32_t* flag, uint32_t* status) {
  uint32_t spins = 0, ns = 8;
  uint32_t f = ld_volatile_u32(flag);
  while (f == 0) {
    if (++spins > kSpinLimit) break;
    __nanosleep(ns);
    if (ns < 256) ns <<= 1;
    f = ld_volatile_u32(flag);
  }
  if (f == 0 && threadIdx.x == 0) atomicOr(status, kErrTimeout);
}

int host_grid(int64_t work, int per_block, int cap) {
  int64_t g = (work + per_block - 1) / per_block;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (int)g;
}

// Launch at the device's highest stream priority (cudaLaunchAttributePriority;
// inside a stream capture it becomes the kernel node's priority).  The
// pruning phase's kernels use it so that the CTA scheduler gives them SMs
// ahead of table builds running on another stream.
int critical_priority() {
  static int prio = [] {
    int least = 0, greatest = 0;
    if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    return greatest;
  }();
  return prio;
}

template <typename... KArgs, typename... Args>
void launch_hi(void (*kernel)(KArgs...), unsigned grid, unsigned block, cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributePriority;
  attr[0].val.priority = critical_priority();
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kernel, args...);
}

}  // namespace

// ---------------------------------------------------------------- launchers
void launch_bloom_build(const BloomBuildArgs& a, int64_t n_upper, int num_sms, cudaStream_t s) {
  launch_hi(k_bloom_build, (unsigned)host_grid(n_upper, kBlock * kBuildKeys, num_sms * 3), kBlock, s, a);
}

void launch_bloom_probe(const BloomProbeArgs& a, int num_sms, cudaStream_t s) {
  k_bloom_probe<<<host_grid(a.n, kBlock * 4, num_sms * 8), kBlock, 0, s>>>(a);
}

int sieve_chunk_rows(int64_t n_upper, int num_sms) {
  // one chunk per CTA slot of the GPU (kCkWaveBlocks per SM), so that one
  // wave splits the rows evenly; whole warp tiles, at least one tile per warp
  const int64_t slots = (int64_t)(num_sms > 0 ? num_sms : 1) * kCkWaveBlocks;
  int64_t c = (n_upper + slots - 1) / slots;
  c = (c + kCkTileRows - 1) / kCkTileRows * kCkTileRows;
  if (c < kCkChunkQuantum) c = kCkChunkQuantum;
  if (c > kCkMaxRows) c = kCkMaxRows;
  return (int)c;
}

void launch_sieve_chunk(const SieveArgs& a, int64_t n_upper, int num_sms, cudaStream_t s) {
  (void)num_sms;
  int64_t g = (n_upper + a.chunk_rows - 1) / a.chunk_rows;
  if (g < 1) g = 1;
  const bool fast = a.ntest == 1 && !a.test[0].is_pred && a.test[0].f.layout == 0 &&
                    a.test[0].f.k >= 1 && a.test[0].f.k <= 4 && a.fast_words_ok;
  if (!fast) {
    launch_hi(k_sieve_chunk<0>, (unsigned)g, kCkThreads, s, a);
    return;
  }
  switch (a.test[0].f.k) {
    case 1: launch_hi(k_sieve_chunk<1>, (unsigned)g, kCkThreads, s, a); break;
    case 2: launch_hi(k_sieve_chunk<2>, (unsigned)g, kCkThreads, s, a); break;
    case 3: launch_hi(k_sieve_chunk<3>, (unsigned)g, kCkThreads, s, a); break;
    default: launch_hi(k_sieve_chunk<4>, (unsigned)g, kCkThreads, s, a); break;
  }
}

void launch_filter_insert(const InsertArgs& a, int num_sms, cudaStream_t s) {
  const int g = host_grid(a.n, kBlock * 4, num_sms * 8);
  k_insert_check<<<g, kBlock, 0, s>>>(a);
  k_insert_or<<<g, kBlock, 0, s>>>(a);
}

void launch_bloom_build_batch(const BuildBatchArgs& b, int64_t total_rows, int num_sms, cudaStream_t s) {
  launch_hi(k_bloom_build_batch, (unsigned)host_grid(total_rows, kBlock * 4, num_sms * 8), kBlock, s, b);
}

void launch_sieve_batch(const SieveBatchArgs& b, int64_t total_chunks, int k_all, cudaStream_t s) {
  const unsigned g = (unsigned)(total_chunks > 0 ? total_chunks : 1);
  switch (k_all) {
    case 1: launch_hi(k_sieve_batch<1>, g, kCkThreads, s, b); break;
    case 2: launch_hi(k_sieve_batch<2>, g, kCkThreads, s, b); break;
    case 3: launch_hi(k_sieve_batch<3>, g, kCkThreads, s, b); break;
    case 4: launch_hi(k_sieve_batch<4>, g, kCkThreads, s, b); break;
    default: launch_hi(k_sieve_batch<0>, g, kCkThreads, s, b); break;
  }
}

void launch_group_offsets(const GroupOffArgs& a, int64_t n_upper, int num_sms, cudaStream_t s) {
  k_group_offsets<<<host_grid(n_upper, kGroupTile, 4 * num_sms), kBlock, 0, s>>>(a);
}

void launch_mm_insert(const MMInsertArgs& a, int num_sms, cudaStream_t s) {
  k_mm_insert<<<host_grid(a.n, kAggRows, num_sms * 4), kBlock, 0, s>>>(a);
}

void launch_mm_scatter(const MMScatterArgs& a, int num_sms, cudaStream_t s) {
  k_mm_scatter<<<host_grid(a.n, kBlock, num_sms * 8), kBlock, 0, s>>>(a);
}

void launch_mm_probe(const MMProbeArgs& a, int num_sms, cudaStream_t s) {
  k_mm_probe<<<host_grid(a.n, kProbeTile, 4 * num_sms), kBlock, 0, s>>>(a);
}

void launch_mm_expand(const MMExpandArgs& a, cudaStream_t s) {
  k_mm_expand<<<host_grid((int64_t)a.T, kBlock, 1 << 30), kBlock, 0, s>>>(a);
}

void launch_mm_expand_dev(const MMExpandArgs& a, int num_sms, cudaStream_t s) {
  k_mm_expand_dev<<<num_sms * 8, kBlock, 0, s>>>(a);
}

void launch_table_init(const TableInitArgs& a, int64_t cap_slots, int num_sms, cudaStream_t s) {
  k_table_init<<<host_grid(cap_slots, kBlock * 8, num_sms * 8), kBlock, 0, s>>>(a);
}

void launch_agg_insert(const AggInsertArgs& a, int num_sms, cudaStream_t s) {
  k_agg_insert<<<host_grid(a.n, kAggRows, num_sms * 4), kBlock, 0, s>>>(a);
}

void launch_agg_probe(const AggProbeArgs& a, int num_sms, cudaStream_t s) {
  k_agg_probe<<<host_grid(a.n, kBlock, num_sms * 8), kBlock, 0, s>>>(a);
}

void launch_pair_filter_build(const PairFilterBuildArgs& a, int num_sms, cudaStream_t s) {
  k_pair_filter_build<<<host_grid(a.n, kBlock * 4, num_sms * 4), kBlock, 0, s>>>(a);
}

void launch_pairset_insert(const PairSetArgs& a, int num_sms, cudaStream_t s) {
  k_pairset_insert<<<host_grid(a.n, kBlock, num_sms * 8), kBlock, 0, s>>>(a);
}

void launch_gather_i32(const int32_t* col, const int32_t* idx, int64_t n, int32_t* out, int num_sms,
                       cudaStream_t s) {
  k_gather_i32<<<host_grid(n, kBlock * 4, num_sms * 8), kBlock, 0, s>>>(col, idx, n, out);
}

void launch_triangles(const TriangleArgs& a, int num_sms, cudaStream_t s) {
  k_triangles<<<num_sms * 8, kBlock, 0, s>>>(a);
}

void launch_wait_flag(const uint32_t* flag, uint32_t* status, cudaStream_t s) {
  k_wait_flag<<<1, 32, 0, s>>>(flag, status);
}

void launch_sum_terms(const SumTermsArgs& a, int num_sms, cudaStream_t s) {
  k_sum_terms<<<host_grid(a.n, kBlock, num_sms * 8), kBlock, 0, s>>>(a);
}

}  // namespace sj
