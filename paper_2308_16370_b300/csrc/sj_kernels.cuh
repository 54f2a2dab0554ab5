// Kernel argument blocks and host-side launchers of the sieved-join kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "sj_device.cuh"

namespace sj {

constexpr int kMaxCols = 8;
constexpr int kMaxTests = 5;   // one range predicate + up to four filters
constexpr int kMaxTerms = 8;

// ------------------------------------------------------------------ Bloom build
struct BloomBuildArgs {
  const int32_t* keys;
  int64_t n_host;          // used when n_dev is null
  const uint64_t* n_dev;   // device row count of a compacted relation, or null
  uint64_t* hdr;           // hdr[0] = nblocks, hdr[1] = rows inserted (written)
  uint32_t* words;         // zeroed, nblocks_cap * 8 words
  uint64_t nblocks_cap;
  uint32_t bits_per_key, k, layout;
  uint64_t seed;
};
void launch_bloom_build(const BloomBuildArgs& a, int64_t n_upper, int num_sms, cudaStream_t s);

struct BloomProbeArgs {
  FilterView f;
  const int32_t* keys;
  int64_t n;
  uint8_t* out;
};
void launch_bloom_probe(const BloomProbeArgs& a, int num_sms, cudaStream_t s);

// ------------------------------------------------------------------ sieve
constexpr int kMaxZero = 4;    // filters one chunked sieve step zeroes for the builds after it

// One test of a sieve step: a range predicate (lo <= v < hi) or a filter probe.
struct SieveTest {
  const int32_t* col;
  int32_t is_pred;
  int32_t lo, hi;
  FilterView f;
};

struct SieveArgs {
  const int32_t* in[kMaxCols];
  int32_t* out[kMaxCols];
  int32_t out_is_vec[kMaxCols];  // out column j is the first test's column
  int nout;
  int ntest;
  SieveTest test[kMaxTests];
  int64_t n_host;
  const uint64_t* n_dev;
  uint64_t* out_n;        // kept rows (written by the last chunk)
  uint64_t* out_n2;       // optional second copy (per-step statistics), or null
  uint32_t* tile_counter; // chunk ticket: 0 at launch (reset by the kernel for the next one)
  LookBack<1> lb;         // one state word per chunk
  int32_t fast_words_ok;  // filter word count of test 0 is below 2^32
  // chunked sieve (k_sieve_chunk)
  int32_t chunk_rows;     // rows per chunk, a multiple of kCkTileRows, at most kCkMaxRows
  int32_t nzero;          // filters the following builds write: zeroed here, see k_sieve_chunk
  uint32_t* zero_words[kMaxZero];
  uint32_t zero_bpk[kMaxZero];
  uint64_t zero_cap_words[kMaxZero];
  // group prefix (k_sieve_chunk): one word per 32 chunks, arrivals << 32 |
  // kept rows, and a counter of finished CTAs; both zero at launch and
  // cleared again by the launch's last CTA.  Null: the chunk offsets come
  // from the look-back over the chunk states instead.
  uint64_t* grp;
  uint32_t* fin;
};

// Chunked single-launch sieve (k_sieve_chunk).  A CTA takes one chunk of
// chunk_rows rows by ticket: it probes the chunk (survivor bits per row in
// shared memory), lists its survivors in shared memory, gets its output offset
// from the counts of the chunks before it and writes its survivors.  The
// offset is the sum of the earlier groups of 32 chunks (a.grp) plus the
// states of the earlier chunks of its own group, or, without a.grp, a
// decoupled look-back over the chunk states (read 1024 at a time by the whole
// CTA).  Scratch: one ticket counter and one state word per chunk
// (a.tile_counter, a.lb), plus the group words and finish counter.  One wave of CTAs
// covers the input (chunks of up to kCkMaxRows rows; larger inputs take
// several waves), so a launch runs fastest when it has the GPU to itself.
constexpr int kCkThreads = 256;
constexpr int kCkTileRows = 256;                 // warp tile: 8 rows per lane, row = 32 j + lane
constexpr int kCkChunkQuantum = kCkTileRows * (kCkThreads / 32);
constexpr int kCkMaxRows = 16384;                // rows per chunk (row offsets fit 16 bits)
constexpr int kCkMinBlocks = 5;                  // resident CTAs per SM (48 registers, no spills)
constexpr int kCkWaveBlocks = kCkMinBlocks;      // CTAs per SM one launch's chunks are sized for
constexpr int kCkList = 2048;                    // survivors listed per round (2 bytes each)
constexpr int kCkWindow = 4 * kCkThreads;        // chunk states read per look-back round
// Rows per chunk for a launch over at most n_upper rows.
int sieve_chunk_rows(int64_t n_upper, int num_sms);
void launch_sieve_chunk(const SieveArgs& a, int64_t n_upper, int num_sms, cudaStream_t s);



// Many sieve steps in one launch (k_sieve_batch): tasks[i] is a full sieve
// step (chunk_rows, lb.st pointing at its own chunk states; tile_counter is
// not used), chunk0[i] the global ticket of its first chunk (chunk0[ntask] =
// the total), both in device memory; `ticket` is 0 at launch and reset by the
// kernel.  k_all: the k of every task when all are single register-blocked
// filter tests with k <= 4 and fewer than 2^32 words, else 0.
struct SieveBatchArgs {
  const SieveArgs* tasks;
  const int64_t* chunk0;
  int ntask;
  uint32_t* ticket;
};
void launch_sieve_batch(const SieveBatchArgs& b, int64_t total_chunks, int k_all, cudaStream_t s);

// Many filter builds in one launch (k_bloom_build_batch): tasks[i] and
// row0[i] (the global index of its first row; row0[ntask] = the total of the
// tasks' row bounds) in device memory.  Words must be cleared beforehand.
struct BuildBatchArgs {
  const BloomBuildArgs* tasks;
  const int64_t* row0;
  int ntask;
};
void launch_bloom_build_batch(const BuildBatchArgs& b, int64_t total_rows, int num_sms, cudaStream_t s);

// ------------------------------------------------------------------ insert maintenance
// Sec. 2.4: new tuples of a relation whose filter exists.  k_insert_check
// classifies every row against the filter as it was before the call (gated by
// a neighbour's filter / key already contained / new); k_insert_or then sets
// the bits of the new rows' keys and adds their number to the filter header.
struct InsertArgs {
  FilterView f;               // the filter being maintained
  uint32_t* words;            // its words (written by k_insert_or)
  uint64_t* hdr;              // its header: hdr[1] += rows inserted
  const int32_t* keys;
  int64_t n;
  int ngate;
  SieveTest gate[kMaxTests];  // filter tests of the neighbours' filters (col = gate column)
  uint8_t* status;            // per row: 0 gated, 1 contained, 2 new
  unsigned long long* counts; // [3], zeroed before k_insert_check
};
void launch_filter_insert(const InsertArgs& a, int num_sms, cudaStream_t s);

// ------------------------------------------------------------------ group offsets
// Start of every table slot's row group in a multimap (CSR by slot).  Groups
// only need disjoint ranges, not slot order, so each tile of slots takes its
// range from one atomicAdd on a cursor (zeroed before the launch) and scans
// its own counts: one pass, no tile waits for another.
struct GroupOffArgs {
  const uint32_t* cnt;    // rows per slot
  uint64_t* off;          // group start per slot (written)
  int64_t n_host;         // slots, when n_dev is null
  const uint32_t* n_dev;  // device slot count, or null
  unsigned long long* cursor;
};
constexpr int kGroupTile = kBlock * 8;
void launch_group_offsets(const GroupOffArgs& a, int64_t n_upper, int num_sms, cudaStream_t s);

// ------------------------------------------------------------------ hash tables
// Open addressing, linear probing over buckets of four 8-byte slots (one
// 32-byte sector).  A slot is 0 when empty, else (tag << 32) | uint32(key).
struct Table {
  unsigned long long* slots;
  uint32_t bucket_mask;                // nbuckets - 1, nbuckets a power of two
  const uint32_t* mask_dev = nullptr;  // if set: the mask, written on the device by k_table_init
};

// Device-side sizing of a table (k_table_init): nslots = power of two >= max(64, 2n)
// for the n read from n_dev, mask written to *mask_out, slots (and the
// optional per-slot arrays) zeroed up to nslots, *zero64 = 0.
struct TableInitArgs {
  unsigned long long* slots;
  uint32_t* mask_out;
  const uint64_t* n_dev;
  int64_t n_host;
  ulonglong2* pairs;              // optional, nslots entries
  uint32_t* cnt;                  // optional, nslots entries to clear
  uint32_t* nslots_out;           // optional: receives nslots
  unsigned long long* zero64 = nullptr;  // optional word cleared (a group-offset cursor)
};
void launch_table_init(const TableInitArgs& a, int64_t cap_slots, int num_sms, cudaStream_t s);

struct MMInsertArgs {       // multimap build, pass 1: key slots and per-row rank
  const int32_t* keys;
  int64_t n;
  Table t;
  uint32_t* cnt;            // [nslots] zeroed: rows per key slot
  uint32_t* rid;            // [n] row -> key slot
  uint32_t* rank;           // [n] row -> rank among rows of its key
  uint32_t* status;
  const uint64_t* n_dev = nullptr;  // device row count (overrides n)
};
void launch_mm_insert(const MMInsertArgs& a, int num_sms, cudaStream_t s);

struct MMScatterArgs {      // multimap build, pass 2: rows grouped by key id
  const uint32_t* rid;
  const uint32_t* rank;
  const uint64_t* off;
  int64_t n;
  int32_t* rows;
  const uint64_t* n_dev = nullptr;
};
void launch_mm_scatter(const MMScatterArgs& a, int num_sms, cudaStream_t s);

struct MMProbeArgs {        // probe + compaction of matching probe rows
  const int32_t* keys;
  int64_t n;
  Table t;
  const uint32_t* cnt;
  int32_t* prow;            // matching probe row
  int32_t* pid;             // its key id
  uint64_t* o;              // exclusive prefix of match counts
  uint64_t* totals;         // [0] = matching rows, [1] = output tuples
  uint32_t* tile_counter;
  LookBack<2> lb;
  const uint64_t* n_dev = nullptr;
};
constexpr int kProbeTile = kBlock * 8;
void launch_mm_probe(const MMProbeArgs& a, int num_sms, cudaStream_t s);

struct Terms {              // SUM terms read from one side's columns
  const int32_t* col[kMaxTerms];     // int32 term, or low word of an int64 term
  const int32_t* col_hi[kMaxTerms];  // high word of an int64 term, else null
  int n;
};

struct MMExpandArgs {       // one output tuple per (matching probe row, build row)
  uint64_t T;
  uint64_t Q;
  const uint64_t* o;
  const int32_t* prow;
  const int32_t* pid;
  const uint64_t* off;
  const int32_t* rows;
  const int32_t* src[kMaxCols];  // source column of each output column
  int32_t src_build[kMaxCols];   // 1 = indexed by build row, 0 = by probe row
  int32_t* out[kMaxCols];
  int nout;
  const uint64_t* psum_in;       // null: use probe_terms
  Terms probe_terms;
  Terms build_terms;
  uint64_t* psum_out;            // null: no SUM carried
  // device-sized mode: Q and T from totals_dev, at most `cap` outputs written,
  // min(T, cap) stored to *n_out, kErrCapacity recorded if T > cap
  const uint64_t* totals_dev = nullptr;
  uint64_t cap = 0;
  uint64_t* n_out = nullptr;
  uint32_t* status = nullptr;
};
void launch_mm_expand(const MMExpandArgs& a, cudaStream_t s);
// Device-sized expand: grid-stride over T read on the device.
void launch_mm_expand_dev(const MMExpandArgs& a, int num_sms, cudaStream_t s);

struct AggInsertArgs {
  const int32_t* keys;
  int64_t n;
  Table t;
  Terms terms;
  const uint64_t* vals;     // per-row value instead of terms, or null
  ulonglong2* cs;           // [nslots] (count, sum) per slot, zeroed
  uint32_t* status;
  const uint64_t* n_dev = nullptr;
};
void launch_agg_insert(const AggInsertArgs& a, int num_sms, cudaStream_t s);

struct AggProbeArgs {
  const int32_t* keys;
  int64_t n;
  Table t;
  const ulonglong2* cs;     // [nslots] (count, sum) per slot
  const uint64_t* psum_in;
  Terms probe_terms;
  unsigned long long* result;  // [0] count lo, [1] count hi, [2] sum; zeroed
  uint32_t* status;
  const uint64_t* n_dev = nullptr;
};
void launch_agg_probe(const AggProbeArgs& a, int num_sms, cudaStream_t s);

struct SumTermsArgs {
  int64_t n;
  Terms terms;
  unsigned long long* result;  // [2] += sum
};
void launch_sum_terms(const SumTermsArgs& a, int num_sms, cudaStream_t s);
void launch_wait_flag(const uint32_t* flag, uint32_t* status, cudaStream_t s);

// ------------------------------------------------------------------ cyclic query
// Edge pairs are packed (src << 32) | dst.  The pair filter uses the
// register-blocked layout over h = fmix64(pair ^ seed); the pair set is an
// open-addressing table whose slots hold pair + 1 (0 = empty).
struct PairFilterBuildArgs {
  const int32_t* src;
  const int32_t* dst;
  int64_t n;
  uint64_t* hdr;
  uint32_t* words;   // zeroed, nblocks * 8 words
  uint64_t nblocks;
  uint32_t k;
  uint64_t seed;
};
void launch_pair_filter_build(const PairFilterBuildArgs& a, int num_sms, cudaStream_t s);

struct PairSetArgs {
  const int32_t* src;
  const int32_t* dst;
  int64_t n;
  Table t;
  uint32_t* status;
};
void launch_pairset_insert(const PairSetArgs& a, int num_sms, cudaStream_t s);

struct Adjacency {          // multimap of edge ids keyed by one endpoint
  Table t;
  const uint32_t* cnt;
  const uint64_t* off;
  const int32_t* rows;
};

struct TriangleArgs {
  const int32_t* src;
  const int32_t* dst;
  int64_t ne;
  Adjacency out;            // keyed by src
  Adjacency in;             // keyed by dst
  const int32_t* out_nbr;   // dst of out.rows[t], in the same order (read contiguously)
  const int32_t* in_nbr;    // src of in.rows[t], in the same order
  FilterView pf;            // pair filter (register-blocked)
  Table pairs;              // exact pair set
  const int32_t* cuts;      // nsub + 1, increasing
  int nsub;                 // <= 256
  unsigned long long* counts;   // [nsub], zeroed
  unsigned long long* stats;    // [0] candidates checked, [1] passed the pair filter; zeroed
  unsigned long long* work;     // edge cursor, zeroed
};
void launch_triangles(const TriangleArgs& a, int num_sms, cudaStream_t s);
// out[i] = col[idx[i]] for i < n.
void launch_gather_i32(const int32_t* col, const int32_t* idx, int64_t n, int32_t* out, int num_sms,
                       cudaStream_t s);

}  // namespace sj
