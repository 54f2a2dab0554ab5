// Host side of the C ABI declared in include/sievejoin.h: contexts, relation
// and filter handles, the pruning-phase driver (Sec. 2.2, sj_sieve_path) and
// the left-deep hash-join driver (Sec. 2.2 enumeration phase, sj_join).
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <functional>
#include <map>
#include <memory>
#include <string>
#include <utility>
#include <vector>

#include "sievejoin.h"
#include "sj_kernels.cuh"

using namespace sj;

namespace {

constexpr size_t kAlign = 256;
inline size_t round_up(size_t x, size_t a = kAlign) { return (x + a - 1) / a * a; }

// d_misc layout (uint64 words)
constexpr int kMiscStatus = 0;   // uint32 status bits in the low half
constexpr int kMiscResult = 1;   // [1..3] count lo, count hi, sum
constexpr int kMiscTotals = 4;   // [4..5] matching probe rows, output tuples
constexpr int kMiscSteps = 8;    // [8 .. 8 + kMaxSlots) per-step row counts
constexpr int kMaxSlots = 120;
constexpr int kMiscWords = kMiscSteps + kMaxSlots;
// internal status: a device-sized join outgrew a buffer and must be rerun
constexpr sj_status kRetry = 100;
// d_misc words of the device-sized join: per-level totals and output counts
constexpr int kMiscLevelTotals = kMiscSteps + 96;  // 2 words per level, 8 levels
constexpr int kMiscLevelCount = kMiscSteps + 112;  // 1 word per level
// the same words as statistics slots (profiling resolves bytes from them)
constexpr int kSlotLevelTotals = kMiscLevelTotals - kMiscSteps;
constexpr int kSlotLevelCount = kMiscLevelCount - kMiscSteps;

struct ProfRec {
  int kind;
  cudaEvent_t e0, e1;
  double bytes;       // fixed part
  int slot_a, slot_b; // deferred parts: per_a * count[slot_a] + per_b * count[slot_b]
  double per_a, per_b;
};

}  // namespace

struct sj_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  sj_alloc_fn alloc = nullptr;
  sj_free_fn free_ = nullptr;
  void* user = nullptr;
  int num_sms = 148;
  std::string err;
  uint64_t* d_misc = nullptr;
  uint64_t* h_misc = nullptr;  // pinned
  uint8_t* scratch = nullptr;
  size_t scratch_bytes = 0;
  uint32_t epoch = 0;  // state-word epoch of the last scan launch
  cudaEvent_t ev_wait = nullptr;  // host waits on one point of the stream
  // second stream: the device-sized join builds its multimaps there while the
  // main stream probes; it has its own scan scratch
  cudaStream_t side = nullptr;
  uint8_t* scratch2 = nullptr;
  size_t scratch2_bytes = 0;
  uint32_t epoch2 = 0;
  cudaEvent_t ev_ready = nullptr;
  cudaEvent_t ev_built[SJ_MAX_REL] = {};
  // CUDA graphs of the device-sized sieved join, per query shape: a repeated
  // query replays one graph instead of enqueueing ~40 operations.  A graph
  // bakes in arena addresses (valid while arena_gen is unchanged) and the
  // intermediate buffer sizes it was captured with.
  struct GraphEntry {
    cudaGraphExec_t exec = nullptr;
    std::vector<uint64_t> caps;
    uint64_t gen = 0;
    int64_t nkernels = 0;
    int64_t h2d_bytes = 0;      // host-to-device copies inside the graph (staged columns)
    bool failed = false;        // capture not possible for this shape
    std::vector<ProfRec> prof;  // launch events inside the graph (profiled capture); owned
  };
  std::map<uint64_t, GraphEntry> graphs;  // key: query signature, profiling flag
  int64_t graph_replays = 0, graph_captures = 0, graph_failures = 0;
  std::string graph_why;
  bool capturing = false;  // no allocator calls while a graph is captured
  bool graphs_on = true;   // capture repeated query shapes (sj_graphs_enable)
  cudaStream_t cap_stream = nullptr;  // captures run here (the user's stream may be the legacy one)
  uint64_t arena_gen = 0;
  // per query shape: output tuples of each join level in the last exact run,
  // used to size the buffers of the device-sized (host-sync-free) join
  std::map<uint64_t, std::vector<uint64_t>> plan_caps;
  std::map<uint64_t, int> plan_runs;  // device-sized runs per query shape (graph capture from the 2nd)
  // per-call arena (sj_sieve_join): temporaries are bump-allocated from one
  // device block and released together, instead of one allocator call each
  struct {
    bool on = false;
    uint8_t* base = nullptr;
    size_t size = 0, off = 0, peak = 0, spilled = 0;
    std::vector<std::pair<void*, size_t>> overflow;
  } arena;
  int64_t launches = 0;
  int64_t h2d_bytes = 0;
  int64_t d2h_bytes = 0;
  bool prof_on = false;
  uint32_t prof_mask = 0xffffffffu;  // kernel classes profiled while prof_on
  std::vector<ProfRec> prof;
  std::vector<cudaEvent_t> ev_pool;
  // copy stream of host-mapped relations' staged columns, in plan order
  cudaStream_t copy = nullptr;
  cudaEvent_t ev_copy_fork = nullptr;
  cudaEvent_t ev_copied[SJ_MAX_REL] = {};
  // pinned staging of sj_sieve_path_batch (launch arguments, counts read back)
  uint8_t* h_batch = nullptr;
  size_t h_batch_bytes = 0;
  bool batch_pending = false;  // a copy from h_batch may still be in flight
  size_t ev_used = 0;
  double prof_ms[SJ_K_COUNT] = {};
  double prof_gap_ms[SJ_K_COUNT] = {};  // device idle after a launch of each class
  double prof_bytes[SJ_K_COUNT] = {};
  int64_t prof_n[SJ_K_COUNT] = {};
};

struct sj_rel_s {
  int ncols = 0;
  int64_t nrows = 0;   // host row count (-1 while only the device knows it)
  int64_t cap = 0;     // allocated rows
  int32_t* cols[SJ_MAX_COLS] = {};
  uint64_t* d_n = nullptr;  // device row count (compacted relations), else null
  void* mem = nullptr;
  size_t mem_bytes = 0;
  bool host_mapped = false;  // columns are page-locked host memory (SJ_HOST_MAPPED)
};

struct sj_filter_s {
  sj_filter_params p{};
  uint64_t* hdr = nullptr;   // device: nblocks, rows inserted
  uint32_t* words = nullptr;
  uint64_t nblocks_cap = 0;
  void* mem = nullptr;
  size_t mem_bytes = 0;
};

namespace {

sj_status fail(sj_ctx* c, sj_status s, const std::string& msg) {
  if (c) c->err = msg;
  return s;
}

#define SJ_CUDA(c, call)                                                              \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess)                                                            \
      return fail((c), SJ_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

#define SJ_TRY(expr)              \
  do {                            \
    sj_status s_ = (expr);        \
    if (s_ != SJ_OK) return s_;   \
  } while (0)

void* raw_alloc(sj_ctx* c, size_t bytes) {
  void* p = nullptr;
  if (c->capturing) return nullptr;  // the capture is abandoned instead
  if (c->alloc) {
    p = c->alloc(bytes, c->user);
  } else if (cudaMallocAsync(&p, bytes, c->stream) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  return p;
}

void raw_free(sj_ctx* c, void* p, size_t bytes) {
  if (!p) return;
  if (c->free_) c->free_(p, bytes, c->user);
  else cudaFreeAsync(p, c->stream);
}

bool in_arena(const sj_ctx* c, const void* p) {
  const uint8_t* q = static_cast<const uint8_t*>(p);
  return c->arena.base && q >= c->arena.base && q < c->arena.base + c->arena.size;
}

// Device memory for temporaries.  Inside an arena scope it is bump-allocated
// (or, when the arena is full, allocated and released with the scope).
// `persistent` allocations (results handed to the caller, context state)
// always bypass the arena.
void* dalloc(sj_ctx* c, size_t bytes, bool persistent = false) {
  bytes = round_up(bytes ? bytes : 1);
  if (c->arena.on && !persistent) {
    auto& A = c->arena;
    if (A.off + bytes <= A.size) {
      void* p = A.base + A.off;
      A.off += bytes;
      A.peak = std::max(A.peak, A.off + A.spilled);
      return p;
    }
    // counted in full, so that the arena grows to hold every block of the scope
    A.spilled += bytes;
    A.peak = std::max(A.peak, A.off + A.spilled);
    void* p = raw_alloc(c, bytes);
    if (p) A.overflow.emplace_back(p, bytes);
    return p;
  }
  return raw_alloc(c, bytes);
}

void dfree(sj_ctx* c, void* p, size_t bytes) {
  if (!p) return;
  bytes = round_up(bytes ? bytes : 1);
  if (c->arena.on) {
    if (in_arena(c, p)) return;
    for (auto& o : c->arena.overflow)
      if (o.first == p) return;  // released when the arena scope ends
  }
  raw_free(c, p, bytes);
}

void arena_begin(sj_ctx* c) {
  c->arena.on = true;
  c->arena.off = 0;
  c->arena.peak = 0;
  c->arena.spilled = 0;
}

// End the scope: release overflow blocks and grow the arena to the peak seen,
// so the next call of the same size needs no allocator call at all.  All
// releases are stream-ordered after the work that used the memory.
void arena_end(sj_ctx* c) {
  auto& A = c->arena;
  A.on = false;
  for (auto& o : A.overflow) raw_free(c, o.first, o.second);
  A.overflow.clear();
  if (A.peak > A.size) {
    raw_free(c, A.base, A.size);
    const size_t nb = round_up(A.peak + A.peak / 4, 1 << 20);
    A.base = static_cast<uint8_t*>(raw_alloc(c, nb));
    A.size = A.base ? nb : 0;
    c->arena_gen++;  // graphs holding the old addresses are stale
  }
  A.off = 0;
}

// Temporaries of one call, released (stream-ordered) when the call returns.
struct Temps {
  sj_ctx* c;
  std::vector<std::pair<void*, size_t>> v;
  explicit Temps(sj_ctx* cc) : c(cc) {}
  ~Temps() {
    for (auto& x : v) dfree(c, x.first, x.second);
  }
  template <class T>
  T* get(size_t n_elems, sj_status* st) {
    const size_t bytes = n_elems * sizeof(T);
    void* p = dalloc(c, bytes);
    if (!p) {
      *st = SJ_ENOMEM;
      return nullptr;
    }
    v.emplace_back(p, bytes);
    return static_cast<T*>(p);
  }
};

// Reasons of failed captures, each kept once.
void note_graph_failure(sj_ctx* c, const std::string& why) {
  if (c->graph_why.find(why) != std::string::npos || c->graph_why.size() > 400) return;
  if (!c->graph_why.empty()) c->graph_why += "; ";
  c->graph_why += why;
}

void drop_graph(sj_ctx::GraphEntry& G) {
  if (G.exec) cudaGraphExecDestroy(G.exec);
  for (auto& r : G.prof) {
    cudaEventDestroy(r.e0);
    cudaEventDestroy(r.e1);
  }
  G = sj_ctx::GraphEntry{};
}

// Profiling of one replay: the graph's own launch events, resolved with the
// per-step counts the replay copied back.
void prof_replay(sj_ctx* c, const sj_ctx::GraphEntry& G) {
  for (size_t i = 0; i < G.prof.size(); ++i) {
    const ProfRec& r = G.prof[i];
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.e0, r.e1) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    double bytes = r.bytes;
    if (r.slot_a >= 0) bytes += r.per_a * (double)c->h_misc[kMiscSteps + r.slot_a];
    if (r.slot_b >= 0) bytes += r.per_b * (double)c->h_misc[kMiscSteps + r.slot_b];
    c->prof_ms[r.kind] += ms;
    c->prof_bytes[r.kind] += bytes;
    c->prof_n[r.kind] += 1;
    float gap = 0.f;
    if (i + 1 < G.prof.size() && cudaEventElapsedTime(&gap, r.e1, G.prof[i + 1].e0) == cudaSuccess &&
        gap > 0.f)
      c->prof_gap_ms[r.kind] += gap;
    cudaGetLastError();
  }
}

cudaEvent_t take_event(sj_ctx* c) {
  if (c->ev_used == c->ev_pool.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    c->ev_pool.push_back(e);
  }
  return c->ev_pool[c->ev_used++];
}

// Bracket a kernel launch with profiling events when enabled.
struct Launch {
  sj_ctx* c;
  ProfRec rec{};
  bool on;
  Launch(sj_ctx* cc, int kind, double bytes, int slot_a = -1, double per_a = 0, int slot_b = -1,
         double per_b = 0)
      : c(cc), on(cc->prof_on && ((cc->prof_mask >> kind) & 1u)) {
    c->launches++;
    if (!on) return;
    rec.kind = kind;
    rec.bytes = bytes;
    rec.slot_a = slot_a;
    rec.per_a = per_a;
    rec.slot_b = slot_b;
    rec.per_b = per_b;
    rec.e0 = take_event(c);
    rec.e1 = take_event(c);
    if (rec.e0) record(rec.e0);
  }
  ~Launch() {
    if (!on || !rec.e0 || !rec.e1) return;
    record(rec.e1);
    c->prof.push_back(rec);
  }
  // inside a graph capture the record must become a node of its own, so that
  // every replay records the event
  void record(cudaEvent_t e) {
    if (c->capturing) cudaEventRecordWithFlags(e, c->stream, cudaEventRecordExternal);
    else cudaEventRecord(e, c->stream);
  }
};

// A launch whose algorithmic bytes are `per` bytes per row, the rows being the
// device count in statistics slot `slot` (resolved once it is read back), or
// the host-known n when slot < 0.
inline Launch rows_launch(sj_ctx* c, int kind, double per, int slot, int64_t n_host) {
  return slot >= 0 ? Launch(c, kind, 0.0, slot, per) : Launch(c, kind, per * (double)std::max<int64_t>(n_host, 0));
}

sj_status check_launch(sj_ctx* c, const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(c, SJ_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
  return SJ_OK;
}

// Synchronise, read the misc block back and turn device status bits into errors.
// Status bits of h_misc (already copied back and synchronised).
sj_status read_status(sj_ctx* c) {
  const uint32_t st = (uint32_t)(c->h_misc[kMiscStatus] & 0xffffffffu);
  if (st) {
    SJ_CUDA(c, cudaMemsetAsync(c->d_misc + kMiscStatus, 0, sizeof(uint64_t), c->stream));
    if (st & kErrTimeout) return fail(c, SJ_ETIMEOUT, "a bounded device wait timed out");
    if (st & kErrTableFull) return fail(c, SJ_ETABLEFULL, "hash table probe chain exhausted");
    if (st == kErrCapacity) return kRetry;  // a device-sized buffer was too small
    return fail(c, SJ_ECUDA, "device status word set");
  }
  return SJ_OK;
}

sj_status enqueue_readback(sj_ctx* c) {
  SJ_CUDA(c, cudaMemcpyAsync(c->h_misc, c->d_misc, kMiscWords * sizeof(uint64_t),
                             cudaMemcpyDeviceToHost, c->stream));
  c->d2h_bytes += kMiscWords * sizeof(uint64_t);
  return SJ_OK;
}

sj_status sync_read(sj_ctx* c) {
  SJ_TRY(enqueue_readback(c));
  SJ_CUDA(c, cudaStreamSynchronize(c->stream));
  return read_status(c);
}

uint32_t* status_ptr(sj_ctx* c) { return reinterpret_cast<uint32_t*>(c->d_misc + kMiscStatus); }

// Scratch for one compaction scan: a kAlign-byte header with the tile ticket
// counter (byte 0) and the finish counter of a group-prefix sieve (byte 4),
// then the group words (one for every 33 words of the area, so at least one
// per 32 state words; their place depends only on the area's size), then NCH
// packed state words per tile.  States carry a per-launch epoch, and the
// kernels reset the ticket counter, the group words and the finish counter,
// so the area is zeroed only when (re)allocated or when the 16-bit epoch
// wraps.
template <int NCH>
sj_status scratch_for(sj_ctx* c, int64_t ntiles, uint32_t** counter, LookBack<NCH>* lb,
                      uint64_t** grp = nullptr, uint32_t** fin = nullptr) {
  if (ntiles < 1) ntiles = 1;
  const size_t need = kAlign + 33 * 8 * (((size_t)ntiles * NCH + 31) / 32 + 1);
  if (need > c->scratch_bytes) {
    // the old scratch may still be used by enqueued work: stream-ordered free
    raw_free(c, c->scratch, c->scratch_bytes);
    const size_t nb = round_up(std::max(need, c->scratch_bytes * 2));
    c->scratch = static_cast<uint8_t*>(dalloc(c, nb, true));
    c->scratch_bytes = c->scratch ? nb : 0;
    c->arena_gen++;  // graphs holding the old scratch are stale
    if (!c->scratch) return fail(c, SJ_ENOMEM, "scratch allocation failed");
    SJ_CUDA(c, cudaMemsetAsync(c->scratch, 0, nb, c->stream));
    c->epoch = 0;
  }
  if (++c->epoch >= (1u << 16)) {
    SJ_CUDA(c, cudaMemsetAsync(c->scratch, 0, c->scratch_bytes, c->stream));
    c->epoch = 1;
  }
  const size_t ngrp = (c->scratch_bytes - kAlign) / 8 / 33;
  *counter = reinterpret_cast<uint32_t*>(c->scratch);
  if (grp) *grp = reinterpret_cast<uint64_t*>(c->scratch + kAlign);
  if (fin) *fin = reinterpret_cast<uint32_t*>(c->scratch + 4);
  lb->st = reinterpret_cast<uint64_t*>(c->scratch + kAlign) + ngrp;
  lb->status = status_ptr(c);
  lb->epoch = c->epoch;
  return SJ_OK;
}

// --------------------------------------------------------------- relations
sj_rel new_rel(sj_ctx* c, int ncols, int64_t cap, bool persistent = false) {
  sj_rel r = new sj_rel_s();
  const size_t colb = round_up((size_t)std::max<int64_t>(cap, 1) * 4);
  r->mem_bytes = kAlign + colb * (size_t)ncols;
  r->mem = dalloc(c, r->mem_bytes, persistent);
  if (!r->mem) {
    delete r;
    return nullptr;
  }
  r->ncols = ncols;
  r->cap = cap;
  r->nrows = -1;
  r->d_n = static_cast<uint64_t*>(r->mem);
  uint8_t* p = static_cast<uint8_t*>(r->mem) + kAlign;
  for (int j = 0; j < ncols; ++j) r->cols[j] = reinterpret_cast<int32_t*>(p + colb * j);
  return r;
}

void free_rel(sj_ctx* c, sj_rel r) {
  if (!r) return;
  dfree(c, r->mem, r->mem_bytes);
  delete r;
}

sj_rel view_of(const sj_rel_s* src) {
  sj_rel r = new sj_rel_s(*src);
  r->mem = nullptr;
  r->mem_bytes = 0;
  return r;
}

int64_t rel_cap(const sj_rel_s* r) { return r->d_n ? r->cap : r->nrows; }

struct TestSpec {
  int col;
  bool is_pred;
  int32_t lo, hi;
  sj_filter f;
};

FilterView view(const sj_filter_s* f) {
  FilterView v;
  v.words = f->words;
  v.hdr = f->hdr;
  v.k = f->p.k;
  v.layout = f->p.layout;
  v.seed = f->p.seed;
  return v;
}

// One sieve step without synchronising: kept rows of `in` into a new relation.
// `slot` >= 0 also stores the kept-row count in the per-step statistics;
// `slot_in` is the statistics slot of `in`'s own count (deferred profiling bytes).
// `zero` lists filters (allocated, words not cleared) that the builds following
// this step write from its output: the step clears exactly the words they use.
sj_status sieve_step_timed(sj_ctx* c, const sj_rel_s* in, const std::vector<TestSpec>& tests,
                           int slot, int slot_in, sj_rel* out,
                           const std::vector<sj_filter>* zero = nullptr) {
  const int64_t cap = rel_cap(in);
  sj_rel r = new_rel(c, in->ncols, cap);
  if (!r) return fail(c, SJ_ENOMEM, "sieve output allocation failed");
  SieveArgs a;
  memset(&a, 0, sizeof(a));
  a.ntest = (int)tests.size();
  for (size_t t = 0; t < tests.size(); ++t) {
    a.test[t].col = in->cols[tests[t].col];
    a.test[t].is_pred = tests[t].is_pred ? 1 : 0;
    a.test[t].lo = tests[t].lo;
    a.test[t].hi = tests[t].hi;
    if (!tests[t].is_pred) a.test[t].f = view(tests[t].f);
  }
  a.nout = in->ncols;
  for (int j = 0; j < in->ncols; ++j) {
    a.in[j] = in->cols[j];
    a.out[j] = r->cols[j];
    a.out_is_vec[j] = (!tests.empty() && tests[0].col == j) ? 1 : 0;
  }
  a.n_host = in->d_n ? 0 : in->nrows;
  a.n_dev = in->d_n;
  a.out_n = r->d_n;
  a.out_n2 = slot >= 0 ? c->d_misc + kMiscSteps + slot : nullptr;
  a.fast_words_ok = 1;
  if (!tests.empty() && !tests[0].is_pred && tests[0].f->nblocks_cap * 8 >= (1ull << 32)) a.fast_words_ok = 0;
  if (zero) {
    for (sj_filter f : *zero) {
      if (a.nzero == kMaxZero) break;
      a.zero_words[a.nzero] = f->words;
      a.zero_bpk[a.nzero] = f->p.bits_per_key;
      a.zero_cap_words[a.nzero] = f->nblocks_cap * 8;
      a.nzero++;
    }
  }
  a.chunk_rows = sieve_chunk_rows(cap, c->num_sms);
  sj_status st = scratch_for<1>(c, (cap + a.chunk_rows - 1) / a.chunk_rows, &a.tile_counter, &a.lb,
                                &a.grp, &a.fin);
  if (st != SJ_OK) {
    free_rel(c, r);
    return st;
  }
  // algorithmic bytes: the first tested column of every input row; each kept
  // row's other columns read and all of its columns written
  const int nvec = tests.empty() ? 0 : 1;
  const double per_in = 4.0 * nvec;
  const double per_out = 4.0 * (in->ncols - nvec) + 4.0 * in->ncols;
  {
    Launch L = in->d_n ? Launch(c, SJ_K_SIEVE, 0, slot_in, per_in, slot, per_out)
                       : Launch(c, SJ_K_SIEVE, per_in * (double)in->nrows, slot, per_out);
    launch_sieve_chunk(a, cap, c->num_sms, c->stream);
  }
  st = check_launch(c, "k_sieve_chunk");
  if (st != SJ_OK) {
    free_rel(c, r);
    return st;
  }
  *out = r;
  return SJ_OK;
}

sj_filter_params norm_params(const sj_filter_params* p) {
  sj_filter_params q{};
  if (p) q = *p;
  if (q.bits_per_key == 0) q.bits_per_key = 8;
  if (q.k == 0) q.k = 3;
  return q;
}

sj_status check_params(sj_ctx* c, const sj_filter_params& p) {
  if (p.layout > SJ_CLASSIC) return fail(c, SJ_EINVAL, "unknown filter layout");
  if (p.layout == SJ_REGBLOCKED32 && p.k > 6)
    return fail(c, SJ_EINVAL, "register-blocked filter needs k <= 6");
  if (p.layout == SJ_BLOCKED256 && p.k > 4) return fail(c, SJ_EINVAL, "blocked filter needs k <= 4");
  if (p.layout == SJ_CLASSIC && p.k > 8) return fail(c, SJ_EINVAL, "classic filter needs k <= 8");
  if (p.bits_per_key > 1024) return fail(c, SJ_EINVAL, "bits_per_key must be <= 1024");
  return SJ_OK;
}

// Allocate a filter for a build over `rel` (capacity from its row bound); its
// words are not cleared.
sj_status alloc_filter(sj_ctx* c, const sj_rel_s* rel, const sj_filter_params& p, sj_filter* out) {
  const int64_t cap = rel_cap(rel);
  sj_filter f = new sj_filter_s();
  f->p = p;
  uint64_t nbc = ((uint64_t)p.bits_per_key * (uint64_t)cap + 255) / 256;
  if (nbc < 1) nbc = 1;
  f->nblocks_cap = nbc;
  f->mem_bytes = kAlign + nbc * 32;
  f->mem = dalloc(c, f->mem_bytes);
  if (!f->mem) {
    delete f;
    return fail(c, SJ_ENOMEM, "filter allocation failed");
  }
  f->hdr = static_cast<uint64_t*>(f->mem);
  f->words = reinterpret_cast<uint32_t*>(static_cast<uint8_t*>(f->mem) + kAlign);
  *out = f;
  return SJ_OK;
}

// Build filter `f` over column `col` of `rel` without synchronising.  Unless
// `cleared` (the sieve step that produced `rel` cleared the words), the words
// the filter can use are cleared first.
sj_status launch_build(sj_ctx* c, sj_filter f, const sj_rel_s* rel, int col, int slot_in,
                       bool cleared) {
  const sj_filter_params& p = f->p;
  if (!cleared) {
    cudaError_t e = cudaMemsetAsync(f->words, 0, f->nblocks_cap * 32, c->stream);
    if (e != cudaSuccess) return fail(c, SJ_ECUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
  }
  BloomBuildArgs a;
  a.keys = rel->cols[col];
  a.n_host = rel->d_n ? 0 : rel->nrows;
  a.n_dev = rel->d_n;
  a.hdr = f->hdr;
  a.words = f->words;
  a.nblocks_cap = f->nblocks_cap;
  a.bits_per_key = p.bits_per_key;
  a.k = p.k;
  a.layout = p.layout;
  a.seed = p.seed;
  // algorithmic bytes: 4 per key read plus the filter's bits written once
  const double per_key = 4.0 + p.bits_per_key / 8.0;
  {
    Launch L = rel->d_n ? Launch(c, SJ_K_BLOOM_BUILD, 0, slot_in, per_key)
                        : Launch(c, SJ_K_BLOOM_BUILD, per_key * (double)rel->nrows);
    launch_bloom_build(a, rel_cap(rel), c->num_sms, c->stream);
  }
  return check_launch(c, "k_bloom_build");
}

// Build a filter over column `col` of `rel` without synchronising.
sj_status build_filter_nosync(sj_ctx* c, const sj_rel_s* rel, int col, const sj_filter_params& p,
                              int slot_in, sj_filter* out) {
  sj_filter f = nullptr;
  SJ_TRY(alloc_filter(c, rel, p, &f));
  const sj_status st = launch_build(c, f, rel, col, slot_in, false);
  if (st != SJ_OK) {
    dfree(c, f->mem, f->mem_bytes);
    delete f;
    return st;
  }
  *out = f;
  return SJ_OK;
}

void free_filter(sj_ctx* c, sj_filter f) {
  if (!f) return;
  dfree(c, f->mem, f->mem_bytes);
  delete f;
}

// Resolve deferred algorithmic bytes of profiled launches from step counts.
void prof_resolve(sj_ctx* c, size_t from) {
  for (size_t i = from; i < c->prof.size(); ++i) {
    ProfRec& r = c->prof[i];
    if (r.slot_a >= 0) {
      r.bytes += r.per_a * (double)c->h_misc[kMiscSteps + r.slot_a];
      r.slot_a = -1;
    }
    if (r.slot_b >= 0) {
      r.bytes += r.per_b * (double)c->h_misc[kMiscSteps + r.slot_b];
      r.slot_b = -1;
    }
  }
}

// --------------------------------------------------------------- join tree
struct Tree {
  std::vector<int> parent, pedge, post, pre;
  std::vector<std::vector<int>> children;
};

int edge_col(const sj_edge& e, int rel) { return e.rel_a == rel ? e.col_a : e.col_b; }

sj_status validate_path(sj_ctx* c, const sj_path* p, const sj_rel* rels, Tree* tr) {
  if (!p || p->nrel < 1 || p->nrel > SJ_MAX_REL) return fail(c, SJ_EINVAL, "nrel out of range");
  const int n = p->nrel;
  if (!rels) return fail(c, SJ_EINVAL, "null relations");
  for (int i = 0; i < n; ++i)
    if (!rels[i]) return fail(c, SJ_EINVAL, "null relation handle");
  if (n > 1 && !p->edges) return fail(c, SJ_EINVAL, "null edges");
  std::vector<std::vector<std::pair<int, int>>> adj(n);
  for (int e = 0; e < n - 1; ++e) {
    const sj_edge& E = p->edges[e];
    if (E.rel_a < 0 || E.rel_a >= n || E.rel_b < 0 || E.rel_b >= n || E.rel_a == E.rel_b)
      return fail(c, SJ_EINVAL, "edge relation out of range");
    if (E.col_a < 0 || E.col_a >= rels[E.rel_a]->ncols || E.col_b < 0 ||
        E.col_b >= rels[E.rel_b]->ncols)
      return fail(c, SJ_EINVAL, "edge column out of range");
    adj[E.rel_a].push_back({E.rel_b, e});
    adj[E.rel_b].push_back({E.rel_a, e});
  }
  if (p->preds)
    for (int i = 0; i < n; ++i)
      if (p->preds[i].col >= rels[i]->ncols) return fail(c, SJ_EINVAL, "predicate column out of range");
  const int root = p->root < 0 ? n - 1 : p->root;
  if (root >= n) return fail(c, SJ_EINVAL, "root out of range");
  tr->parent.assign(n, -1);
  tr->pedge.assign(n, -1);
  tr->children.assign(n, {});
  std::vector<int> seen(n, 0), bfs{root};
  seen[root] = 1;
  for (size_t q = 0; q < bfs.size(); ++q) {
    const int v = bfs[q];
    for (auto& ue : adj[v]) {
      if (seen[ue.first]) continue;
      seen[ue.first] = 1;
      tr->parent[ue.first] = v;
      tr->pedge[ue.first] = ue.second;
      tr->children[v].push_back(ue.first);
      bfs.push_back(ue.first);
    }
  }
  if ((int)bfs.size() != n) return fail(c, SJ_EINVAL, "join graph is not a connected tree");
  // depth-first orders
  std::vector<std::pair<int, size_t>> st{{root, 0}};
  tr->pre.push_back(root);
  while (!st.empty()) {
    auto& top = st.back();
    if (top.second < tr->children[top.first].size()) {
      const int ch = tr->children[top.first][top.second++];
      tr->pre.push_back(ch);
      st.push_back({ch, 0});
    } else {
      tr->post.push_back(top.first);
      st.pop_back();
    }
  }
  return SJ_OK;
}

bool has_pred(const sj_path* p, int i) { return p->preds && p->preds[i].col >= 0; }

}  // namespace

// ======================================================================== C ABI
extern "C" {

const char* sj_version(void) { return "0.1.0"; }

const char* sj_status_str(sj_status s) {
  switch (s) {
    case SJ_OK: return "ok";
    case SJ_EINVAL: return "invalid argument";
    case SJ_ENOMEM: return "out of device memory";
    case SJ_ETABLEFULL: return "hash table full";
    case SJ_ETIMEOUT: return "device wait timed out";
    case SJ_EOVERFLOW: return "COUNT overflow";
    case SJ_ECUDA: return "CUDA error";
  }
  return "unknown status";
}

const char* sj_last_error(const sj_ctx* c) { return c ? c->err.c_str() : "null context"; }

sj_status sj_create(sj_ctx** out, int device, void* stream, sj_alloc_fn alloc, sj_free_fn free_,
                    void* user) {
  if (!out) return SJ_EINVAL;
  if ((alloc == nullptr) != (free_ == nullptr)) return SJ_EINVAL;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return SJ_ECUDA;
  }
  if (cudaSetDevice(device) != cudaSuccess) return SJ_ECUDA;
  sj_ctx* c = new sj_ctx();
  c->device = device;
  c->stream = static_cast<cudaStream_t>(stream);
  c->alloc = alloc;
  c->free_ = free_;
  c->user = user;
  cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
  if (!alloc) {
    // keep freed blocks in the device pool instead of returning them to the OS
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
      uint64_t thr = UINT64_MAX;
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
  }
  c->d_misc = static_cast<uint64_t*>(dalloc(c, kMiscWords * sizeof(uint64_t)));
  if (!c->d_misc || cudaMallocHost(&c->h_misc, kMiscWords * sizeof(uint64_t)) != cudaSuccess ||
      cudaMemsetAsync(c->d_misc, 0, kMiscWords * sizeof(uint64_t), c->stream) != cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess) {
    cudaGetLastError();
    if (c->d_misc) dfree(c, c->d_misc, kMiscWords * sizeof(uint64_t));
    if (c->h_misc) cudaFreeHost(c->h_misc);
    delete c;
    return SJ_ENOMEM;
  }
  *out = c;
  return SJ_OK;
}

sj_status sj_destroy(sj_ctx* c) {
  if (!c) return SJ_EINVAL;
  cudaStreamSynchronize(c->stream);
  if (c->side) {
    cudaStreamSynchronize(c->side);
    if (c->scratch2) {
      std::swap(c->stream, c->side);
      raw_free(c, c->scratch2, c->scratch2_bytes);
      std::swap(c->stream, c->side);
      cudaStreamSynchronize(c->side);
    }
    cudaStreamDestroy(c->side);
  }
  for (auto& kv : c->graphs) drop_graph(kv.second);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  if (c->copy) {
    cudaStreamSynchronize(c->copy);
    cudaStreamDestroy(c->copy);
  }
  if (c->ev_copy_fork) cudaEventDestroy(c->ev_copy_fork);
  for (auto e : c->ev_copied)
    if (e) cudaEventDestroy(e);
  if (c->ev_ready) cudaEventDestroy(c->ev_ready);
  for (auto e : c->ev_built)
    if (e) cudaEventDestroy(e);
  raw_free(c, c->scratch, c->scratch_bytes);
  raw_free(c, c->arena.base, c->arena.size);
  raw_free(c, c->d_misc, kMiscWords * sizeof(uint64_t));
  cudaStreamSynchronize(c->stream);
  cudaFreeHost(c->h_misc);
  if (c->h_batch) cudaFreeHost(c->h_batch);
  for (auto e : c->ev_pool) cudaEventDestroy(e);
  if (c->ev_wait) cudaEventDestroy(c->ev_wait);
  delete c;
  return SJ_OK;
}

sj_status sj_sync(sj_ctx* c) {
  if (!c) return SJ_EINVAL;
  return sync_read(c);
}

sj_status sj_load_relation(sj_ctx* c, int ncols, const int32_t* const* cols, int64_t nrows,
                           int where, sj_rel* out) {
  if (!c || !out || !cols) return fail(c, SJ_EINVAL, "null argument");
  if (ncols < 1 || ncols > SJ_MAX_COLS) return fail(c, SJ_EINVAL, "ncols out of range");
  if (nrows < 0 || nrows >= (int64_t(1) << 31)) return fail(c, SJ_EINVAL, "nrows out of range");
  if (where < SJ_DEVICE_BORROW || where > SJ_HOST_MAPPED) return fail(c, SJ_EINVAL, "bad 'where'");
  for (int j = 0; j < ncols; ++j) {
    if (!cols[j] && nrows > 0) return fail(c, SJ_EINVAL, "null column pointer");
    if (where != SJ_HOST_COPY && (reinterpret_cast<uintptr_t>(cols[j]) & 15))
      return fail(c, SJ_EINVAL, "columns must be 16-byte aligned");
  }
  if (where == SJ_DEVICE_BORROW || where == SJ_HOST_MAPPED) {
    int32_t* dcols[SJ_MAX_COLS] = {};
    for (int j = 0; j < ncols; ++j) {
      dcols[j] = const_cast<int32_t*>(cols[j]);
      if (where == SJ_HOST_MAPPED && cols[j]) {
        // the device address of a page-locked host buffer (equal to the host
        // address under unified addressing)
        void* d = nullptr;
        if (cudaHostGetDevicePointer(&d, const_cast<int32_t*>(cols[j]), 0) != cudaSuccess || !d) {
          cudaGetLastError();
          return fail(c, SJ_EINVAL, "SJ_HOST_MAPPED column is not page-locked host memory the device can address");
        }
        if (reinterpret_cast<uintptr_t>(d) & 15) return fail(c, SJ_EINVAL, "columns must be 16-byte aligned");
        dcols[j] = static_cast<int32_t*>(d);
      }
    }
    sj_rel r = new sj_rel_s();
    r->ncols = ncols;
    r->nrows = nrows;
    r->cap = nrows;
    r->host_mapped = where == SJ_HOST_MAPPED;
    for (int j = 0; j < ncols; ++j) r->cols[j] = dcols[j];
    *out = r;
    return SJ_OK;
  }
  sj_rel r = new_rel(c, ncols, nrows);
  if (!r) return fail(c, SJ_ENOMEM, "relation allocation failed");
  r->d_n = nullptr;  // host-known count
  r->nrows = nrows;
  const cudaMemcpyKind kind = where == SJ_HOST_COPY ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  for (int j = 0; j < ncols; ++j) {
    if (nrows == 0) break;
    cudaError_t e = cudaMemcpyAsync(r->cols[j], cols[j], (size_t)nrows * 4, kind, c->stream);
    if (e != cudaSuccess) {
      free_rel(c, r);
      return fail(c, SJ_ECUDA, std::string("cudaMemcpyAsync: ") + cudaGetErrorString(e));
    }
    if (kind == cudaMemcpyHostToDevice) c->h2d_bytes += nrows * 4;
  }
  *out = r;
  return SJ_OK;
}

sj_status sj_rel_info(sj_rel r, int64_t* nrows, int* ncols, const int32_t** cols) {
  if (!r) return SJ_EINVAL;
  if (nrows) *nrows = r->nrows;
  if (ncols) *ncols = r->ncols;
  if (cols)
    for (int j = 0; j < SJ_MAX_COLS; ++j) cols[j] = j < r->ncols ? r->cols[j] : nullptr;
  return SJ_OK;
}

sj_status sj_free_rel(sj_ctx* c, sj_rel r) {
  if (!c || !r) return SJ_EINVAL;
  free_rel(c, r);
  return SJ_OK;
}

sj_status sj_build_filter(sj_ctx* c, sj_rel rel, int key_col, const sj_pred* pred,
                          const sj_filter_params* params, sj_filter* out) {
  if (!c || !rel || !out) return fail(c, SJ_EINVAL, "null argument");
  if (rel->nrows < 0) return fail(c, SJ_EINVAL, "relation row count unknown");
  if (key_col < 0 || key_col >= rel->ncols) return fail(c, SJ_EINVAL, "key column out of range");
  const sj_filter_params p = norm_params(params);
  SJ_TRY(check_params(c, p));
  if (pred && pred->col >= 0) {
    if (pred->col >= rel->ncols) return fail(c, SJ_EINVAL, "predicate column out of range");
    // select the rows passing the predicate, then size the filter by them
    std::vector<TestSpec> t{{pred->col, true, pred->lo, pred->hi, nullptr}};
    sj_rel sel = nullptr;
    SJ_TRY(sieve_step_timed(c, rel, t, 0, -1, &sel));
    sj_status st = sync_read(c);
    if (st == SJ_OK) {
      sel->nrows = (int64_t)c->h_misc[kMiscSteps + 0];
      sel->d_n = nullptr;
      prof_resolve(c, 0);
      st = build_filter_nosync(c, sel, key_col, p, -1, out);
    }
    free_rel(c, sel);
    return st;
  }
  return build_filter_nosync(c, rel, key_col, p, -1, out);
}

sj_status sj_filter_info(sj_ctx* c, sj_filter f, uint64_t* nblocks, uint64_t* n_inserted,
                         const uint32_t** words) {
  if (!c || !f) return fail(c, SJ_EINVAL, "null argument");
  uint64_t h[2];
  SJ_CUDA(c, cudaMemcpyAsync(h, f->hdr, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
  c->d2h_bytes += sizeof(h);
  SJ_TRY(sync_read(c));
  if (nblocks) *nblocks = h[0];
  if (n_inserted) *n_inserted = h[1];
  if (words) *words = f->words;
  return SJ_OK;
}

sj_status sj_filter_probe(sj_ctx* c, sj_filter f, const int32_t* keys, int64_t n, uint8_t* out) {
  if (!c || !f || (n > 0 && (!keys || !out)) || n < 0) return fail(c, SJ_EINVAL, "bad argument");
  if (n == 0) return SJ_OK;
  BloomProbeArgs a;
  a.f = view(f);
  a.keys = keys;
  a.n = n;
  a.out = out;
  {
    Launch L(c, SJ_K_OTHER, 5.0 * (double)n);
    launch_bloom_probe(a, c->num_sms, c->stream);
  }
  return check_launch(c, "k_bloom_probe");
}

sj_status sj_filter_insert(sj_ctx* c, sj_filter f, sj_rel rel, int key_col, int ngate,
                           const int* gate_cols, const sj_filter* gates, uint8_t* status_out,
                           int64_t* counts) {
  if (!c || !f || !rel) return fail(c, SJ_EINVAL, "null argument");
  if (key_col < 0 || key_col >= rel->ncols) return fail(c, SJ_EINVAL, "key column out of range");
  if (ngate < 0 || ngate > SJ_MAX_PROBES || (ngate > 0 && (!gate_cols || !gates)))
    return fail(c, SJ_EINVAL, "bad gates");
  for (int g = 0; g < ngate; ++g) {
    if (!gates[g]) return fail(c, SJ_EINVAL, "null gate filter");
    if (gate_cols[g] < 0 || gate_cols[g] >= rel->ncols) return fail(c, SJ_EINVAL, "gate column out of range");
  }
  if (rel->nrows < 0) return fail(c, SJ_EINVAL, "relation row count unknown");
  const int64_t n = rel->nrows;
  sj_status st = SJ_OK;
  Temps tmp(c);
  uint8_t* status = status_out ? status_out : tmp.get<uint8_t>((size_t)std::max<int64_t>(n, 1), &st);
  unsigned long long* cnt = tmp.get<unsigned long long>(3, &st);
  if (st != SJ_OK) return fail(c, st, "insert scratch allocation failed");
  SJ_CUDA(c, cudaMemsetAsync(cnt, 0, 3 * sizeof(unsigned long long), c->stream));
  InsertArgs a;
  memset(&a, 0, sizeof(a));
  a.f = view(f);
  a.words = f->words;
  a.hdr = f->hdr;
  a.keys = rel->cols[key_col];
  a.n = n;
  a.ngate = ngate;
  for (int g = 0; g < ngate; ++g) {
    a.gate[g].col = rel->cols[gate_cols[g]];
    a.gate[g].f = view(gates[g]);
  }
  a.status = status;
  a.counts = cnt;
  {
    Launch L(c, SJ_K_BLOOM_BUILD, (4.0 + 4.0 * ngate + 1.0) * (double)n);
    c->launches++;  // two kernels
    launch_filter_insert(a, c->num_sms, c->stream);
  }
  SJ_TRY(check_launch(c, "k_insert_check + k_insert_or"));
  if (counts) {
    unsigned long long h[3];
    SJ_CUDA(c, cudaMemcpyAsync(h, cnt, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
    c->d2h_bytes += sizeof(h);
    SJ_CUDA(c, cudaStreamSynchronize(c->stream));
    for (int k = 0; k < 3; ++k) counts[k] = (int64_t)h[k];
  }
  return SJ_OK;
}

sj_status sj_free_filter(sj_ctx* c, sj_filter f) {
  if (!c || !f) return SJ_EINVAL;
  free_filter(c, f);
  return SJ_OK;
}

sj_status sj_sieve(sj_ctx* c, sj_rel rel, int nprobe, const int* key_cols, const sj_filter* filters,
                   const sj_pred* pred, sj_rel* out, int64_t* nrows_out) {
  if (!c || !rel || !out) return fail(c, SJ_EINVAL, "null argument");
  if (rel->nrows < 0) return fail(c, SJ_EINVAL, "relation row count unknown");
  if (nprobe < 0 || nprobe > SJ_MAX_PROBES || (nprobe > 0 && (!key_cols || !filters)))
    return fail(c, SJ_EINVAL, "bad probe list");
  std::vector<TestSpec> t;
  if (pred && pred->col >= 0) {
    if (pred->col >= rel->ncols) return fail(c, SJ_EINVAL, "predicate column out of range");
    t.push_back({pred->col, true, pred->lo, pred->hi, nullptr});
  }
  for (int j = 0; j < nprobe; ++j) {
    if (key_cols[j] < 0 || key_cols[j] >= rel->ncols || !filters[j])
      return fail(c, SJ_EINVAL, "bad probe column or filter");
    t.push_back({key_cols[j], false, 0, 0, filters[j]});
  }
  sj_rel r = nullptr;
  const size_t p0 = c->prof.size();
  SJ_TRY(sieve_step_timed(c, rel, t, 0, -1, &r));
  sj_status st = sync_read(c);
  if (st != SJ_OK) {
    free_rel(c, r);
    return st;
  }
  prof_resolve(c, p0);
  r->nrows = (int64_t)c->h_misc[kMiscSteps + 0];
  if (nrows_out) *nrows_out = r->nrows;
  *out = r;
  return SJ_OK;
}

}  // extern "C"

namespace {
// Called once per relation as soon as its last sieve step is enqueued.
// `slot` is the statistics slot of its device row count (-1: not sieved, the
// host knows the count).
// The pruning schedule of one query (Sec. 2.2): predicate selections first;
// with SJ_FWD_BWD pass 1 in post-order (a relation is sieved by its
// children's filters, then builds the filter it sends to its parent) and
// pass 2 in pre-order (a relation is sieved by its parent's filter, then
// builds one filter per child).  A leaf's pass-1 filter may be handed in
// (Sec. 2.3).  kOpFinal marks the point after which a relation is not
// sieved again.  Filter ids index `given` (a handed-in filter, else null).
enum { kOpStep, kOpBuild, kOpFinal };
struct PruneOp {
  int type, rel, kind;                      // kind: step kind for statistics
  std::vector<std::pair<int, int>> probes;  // (column, filter id)
  bool pred;
  int col, fid;                             // build: column and filter id
};
struct PrunePlan {
  std::vector<PruneOp> ops;
  std::vector<sj_filter> given;
};

sj_status plan_pruning(sj_ctx* c, const sj_path* path, const Tree& tr, const sj_sieve_opts& o,
                       PrunePlan* out) {
  const int n = path->nrel;
  std::vector<PruneOp>& ops = out->ops;
  std::vector<sj_filter>& fl = out->given;
  ops.clear();
  fl.clear();
  auto new_fid = [&]() { fl.push_back(nullptr); return (int)fl.size() - 1; };
  for (int i = 0; i < n; ++i)
    if (has_pred(path, i)) ops.push_back({kOpStep, i, 0, {}, true, -1, -1});
  if (o.passes == SJ_NO_SIEVE || n == 1)
    for (int i = 0; i < n; ++i) ops.push_back({kOpFinal, i, 0, {}, false, -1, -1});
  if (o.passes == SJ_NO_SIEVE || n == 1) return SJ_OK;
  std::vector<int> up(n, -1), down(n, -1);
  if (o.passes == SJ_FWD_BWD) {
    for (int v : tr.post) {
      if (!tr.children[v].empty()) {
        if ((int)tr.children[v].size() > SJ_MAX_PROBES)
          return fail(c, SJ_EINVAL, "a relation has more than 4 children");
        PruneOp op{kOpStep, v, 1, {}, false, -1, -1};
        for (int ch : tr.children[v]) op.probes.push_back({edge_col(path->edges[tr.pedge[ch]], v), up[ch]});
        ops.push_back(op);
      }
      if (tr.parent[v] >= 0) {
        up[v] = new_fid();
        if (tr.children[v].empty() && o.leaf_filters && o.leaf_filters[v])
          fl[up[v]] = o.leaf_filters[v];  // reused (Sec. 2.3); owned by the caller
        else
          ops.push_back({kOpBuild, v, 0, {}, false, edge_col(path->edges[tr.pedge[v]], v), up[v]});
      }
    }
  }
  for (int v : tr.pre) {
    if (tr.parent[v] >= 0)
      ops.push_back({kOpStep, v, 2, {{edge_col(path->edges[tr.pedge[v]], v), down[v]}}, false, -1, -1});
    ops.push_back({kOpFinal, v, 0, {}, false, -1, -1});  // v is not sieved again
    for (int ch : tr.children[v]) {
      down[ch] = new_fid();
      ops.push_back({kOpBuild, v, 0, {}, false, edge_col(path->edges[tr.pedge[ch]], v), down[ch]});
    }
  }
  return SJ_OK;
}

// Columns of host-mapped relations that the query reads in full -- the
// column a filter is built from before the relation's first sieve step, the
// first tested column of that step, the join columns of a relation the
// pruning never sieves -- are copied to the device on the context's copy
// stream, relation by relation in the order the schedule first touches them,
// each relation's copies followed by an event that the pruning waits on
// before its first operation on that relation; so later copies overlap the
// earlier relations' work, and each such column crosses the host link once
// as one bulk copy.  Every other read of a mapped column (the surviving rows
// a sieve step gathers, the terms of matching rows) stays on the host.
// `staged` receives the path with those relations replaced by views over the
// copies, and the events.
struct StagedPath {
  sj_path path{};
  sj_rel rels[SJ_MAX_REL] = {};
  cudaEvent_t ready[SJ_MAX_REL] = {};
  std::vector<std::unique_ptr<sj_rel_s>> views;
};

sj_status ensure_copy_stream(sj_ctx* c) {
  if (!c->copy && cudaStreamCreateWithFlags(&c->copy, cudaStreamNonBlocking) != cudaSuccess)
    return fail(c, SJ_ECUDA, "copy stream creation failed");
  if (!c->ev_copy_fork && cudaEventCreateWithFlags(&c->ev_copy_fork, cudaEventDisableTiming) != cudaSuccess)
    return fail(c, SJ_ECUDA, "event creation failed");
  for (auto& e : c->ev_copied)
    if (!e && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess)
      return fail(c, SJ_ECUDA, "event creation failed");
  return SJ_OK;
}

sj_status stage_mapped(sj_ctx* c, const sj_path* path, const sj_sieve_opts* opts, Temps& tmp,
                       StagedPath* staged) {
  staged->path = *path;
  bool any = false;
  for (int i = 0; i < path->nrel; ++i) {
    staged->rels[i] = path->rels[i];
    any = any || (path->rels[i] && path->rels[i]->host_mapped && path->rels[i]->nrows > 0);
  }
  staged->path.rels = staged->rels;
  if (!any) return SJ_OK;
  Tree tr;
  SJ_TRY(validate_path(c, path, path->rels, &tr));
  sj_sieve_opts o{};
  if (opts) o = *opts;
  PrunePlan pl;
  SJ_TRY(plan_pruning(c, path, tr, o, &pl));
  // full reads per column, and the order in which relations are first used
  std::vector<std::vector<int>> reads(path->nrel, std::vector<int>(SJ_MAX_COLS, 0));
  std::vector<char> stepped(path->nrel, 0), seen(path->nrel, 0);
  std::vector<int> order;
  for (const PruneOp& op : pl.ops) {
    const int i = op.rel;
    if (!seen[i]) {
      seen[i] = 1;
      order.push_back(i);
    }
    if (stepped[i]) continue;
    if (op.type == kOpBuild) reads[i][op.col]++;
    if (op.type == kOpStep) {
      reads[i][op.pred ? path->preds[i].col : op.probes[0].first]++;
      stepped[i] = 1;
    }
  }
  for (int i = 0; i < path->nrel; ++i)
    if (!stepped[i])
      for (int e = 0; e + 1 < path->nrel; ++e) {
        const sj_edge& E = path->edges[e];
        if (E.rel_a == i) reads[i][E.col_a]++;
        if (E.rel_b == i) reads[i][E.col_b]++;
      }
  SJ_TRY(ensure_copy_stream(c));
  bool forked = false;
  for (int i : order) {
    const sj_rel_s* r = path->rels[i];
    if (!r->host_mapped || r->nrows == 0) continue;
    std::unique_ptr<sj_rel_s> v;
    for (int j = 0; j < r->ncols; ++j) {
      if (reads[i][j] < 1) continue;
      if (!forked) {
        // the copy stream starts after everything already on the context stream
        SJ_CUDA(c, cudaEventRecord(c->ev_copy_fork, c->stream));
        SJ_CUDA(c, cudaStreamWaitEvent(c->copy, c->ev_copy_fork, 0));
        forked = true;
      }
      if (!v) v.reset(view_of(r));
      sj_status st = SJ_OK;
      int32_t* d = tmp.get<int32_t>((size_t)r->nrows, &st);
      if (st != SJ_OK) return fail(c, st, "staging allocation failed");
      SJ_CUDA(c, cudaMemcpyAsync(d, r->cols[j], (size_t)r->nrows * 4, cudaMemcpyHostToDevice, c->copy));
      c->h2d_bytes += r->nrows * 4;
      v->cols[j] = d;
    }
    if (v) {
      SJ_CUDA(c, cudaEventRecord(c->ev_copied[i], c->copy));
      staged->ready[i] = c->ev_copied[i];
      staged->rels[i] = v.get();
      staged->views.push_back(std::move(v));
    }
  }
  return SJ_OK;
}

using FinalHook = std::function<sj_status(int rel, const sj_rel_s* r, int slot)>;
sj_status sieve_path_impl(sj_ctx* c, const sj_path* path, const sj_sieve_opts* opts, sj_rel* out_sieved,
                          sj_sieve_stats* stats, bool sync_end, const FinalHook* on_final = nullptr,
                          const cudaEvent_t* ready = nullptr);
}

extern "C" sj_status sj_sieve_path(sj_ctx* c, const sj_path* path, const sj_sieve_opts* opts,
                                   sj_rel* out_sieved, sj_sieve_stats* stats) {
  return sieve_path_impl(c, path, opts, out_sieved, stats, true);
}

namespace {
sj_status sieve_path_batch_impl(sj_ctx* c, int nq, const sj_path* paths, const sj_sieve_opts* opts,
                                sj_rel* out_sieved, sj_sieve_stats* stats);
}

extern "C" sj_status sj_sieve_path_batch(sj_ctx* c, int nq, const sj_path* paths,
                                         const sj_sieve_opts* opts, sj_rel* out_sieved,
                                         sj_sieve_stats* stats) {
  if (!c) return SJ_EINVAL;
  // temporaries from the context's arena (the handed-out relations are not)
  arena_begin(c);
  const sj_status st = sieve_path_batch_impl(c, nq, paths, opts, out_sieved, stats);
  arena_end(c);
  return st;
}

namespace {
// The pruning phase.  With sync_end the call ends with one synchronisation and
// every output handle knows its row count; without it the outputs keep their
// counts on the device only (nrows = -1) for a device-sized join to read.
// `ready` (optional, one per relation): an event the context stream waits on
// before the first operation on that relation (its columns are being staged).
sj_status sieve_path_impl(sj_ctx* c, const sj_path* path, const sj_sieve_opts* opts, sj_rel* out_sieved,
                          sj_sieve_stats* stats, bool sync_end, const FinalHook* on_final,
                          const cudaEvent_t* ready) {
  if (!c || !path || !out_sieved) return fail(c, SJ_EINVAL, "null argument");
  Tree tr;
  SJ_TRY(validate_path(c, path, path->rels, &tr));
  const int n = path->nrel;
  for (int i = 0; i < n; ++i)
    if (path->rels[i]->nrows < 0) return fail(c, SJ_EINVAL, "relation row count unknown");
  sj_sieve_opts o{};
  if (opts) o = *opts;
  const sj_filter_params fp = norm_params(&o.filter);
  SJ_TRY(check_params(c, fp));
  if (o.passes < SJ_FWD_BWD || o.passes > SJ_NO_SIEVE) return fail(c, SJ_EINVAL, "bad passes");

  const size_t p0 = c->prof.size();
  std::vector<sj_rel> cur(n, nullptr);   // owned temporaries (null = the input itself)
  std::vector<int> last_slot(n, -1);     // step slot holding the relation's current count
  std::vector<sj_filter> filters;        // filters this call built (freed at the end)
  struct StepRec { int kind, rel, slot_in, slot_out; int64_t rows_in_host; };
  std::vector<StepRec> steps;
  int slot = 0;
  uint64_t filter_bytes = 0;

  // The schedule is planned first, then run: a sieve step knows which filters
  // are built from its output next (before that relation is sieved again) and
  // clears their words itself.  Filter ids index `fl`.
  PrunePlan plan;
  SJ_TRY(plan_pruning(c, path, tr, o, &plan));
  const std::vector<PruneOp>& ops = plan.ops;
  std::vector<sj_filter> fl = plan.given;

  auto cleanup = [&]() {
    for (auto f : filters) free_filter(c, f);
    filters.clear();
    for (int i = 0; i < n; ++i) {
      free_rel(c, cur[i]);
      cur[i] = nullptr;
    }
  };
  auto rel_of = [&](int i) -> const sj_rel_s* { return cur[i] ? cur[i] : path->rels[i]; };
  std::vector<char> cleared(fl.size(), 0);
  std::vector<char> waited(n, 0);
  sj_status st = SJ_OK;
  for (size_t q = 0; q < ops.size() && st == SJ_OK; ++q) {
    const PruneOp& op = ops[q];
    const int i = op.rel;
    if (ready && ready[i] && !waited[i]) {
      waited[i] = 1;
      if (cudaStreamWaitEvent(c->stream, ready[i], 0) != cudaSuccess) {
        st = fail(c, SJ_ECUDA, "cudaStreamWaitEvent failed");
        break;
      }
    }
    if (op.type == kOpFinal) {
      if (on_final) st = (*on_final)(i, rel_of(i), last_slot[i]);
    } else if (op.type == kOpBuild) {
      sj_filter f = fl[op.fid];
      if (!f) {
        st = alloc_filter(c, rel_of(i), fp, &f);
        if (st != SJ_OK) break;
        fl[op.fid] = f;
        filters.push_back(f);
        filter_bytes += f->nblocks_cap * 32;
      }
      st = launch_build(c, f, rel_of(i), op.col, last_slot[i], cleared[op.fid] != 0);
    } else {
      if (slot >= kMaxSlots || (int)steps.size() >= SJ_MAX_STEPS) {
        st = fail(c, SJ_EINVAL, "too many sieve steps");
        break;
      }
      std::vector<TestSpec> t;
      if (op.pred) t.push_back({path->preds[i].col, true, path->preds[i].lo, path->preds[i].hi, nullptr});
      for (auto& pr : op.probes) t.push_back({pr.first, false, 0, 0, fl[pr.second]});
      // the filters built from this step's output before relation i is sieved again
      std::vector<sj_filter> zero;
      for (size_t u = q + 1; u < ops.size() && st == SJ_OK; ++u) {
        if (ops[u].rel != i) continue;
        if (ops[u].type == kOpStep) break;
        if (ops[u].type != kOpBuild || (int)zero.size() == kMaxZero) continue;
        sj_filter f = nullptr;
        st = alloc_filter(c, cur[i] ? cur[i] : path->rels[i], fp, &f);
        if (st != SJ_OK) break;
        fl[ops[u].fid] = f;
        cleared[ops[u].fid] = 1;
        filters.push_back(f);
        filter_bytes += f->nblocks_cap * 32;
        zero.push_back(f);
      }
      if (st != SJ_OK) break;
      sj_rel r = nullptr;
      const sj_rel_s* in = rel_of(i);
      st = sieve_step_timed(c, in, t, slot, last_slot[i], &r, &zero);
      if (st != SJ_OK) break;
      steps.push_back({op.kind, i, last_slot[i], slot, in->d_n ? -1 : in->nrows});
      free_rel(c, cur[i]);
      cur[i] = r;
      last_slot[i] = slot++;
    }
  }
  if (st == SJ_OK && sync_end) st = sync_read(c);
  if (st != SJ_OK) {
    cleanup();
    return st;
  }
  if (sync_end) prof_resolve(c, p0);
  for (auto f : filters) free_filter(c, f);
  filters.clear();
  for (int i = 0; i < n; ++i) {
    if (cur[i]) {
      cur[i]->nrows = sync_end ? (int64_t)c->h_misc[kMiscSteps + last_slot[i]] : -1;
      out_sieved[i] = cur[i];
    } else {
      out_sieved[i] = view_of(path->rels[i]);
    }
  }
  if (!sync_end) return SJ_OK;
  if (stats) {
    memset(stats, 0, sizeof(*stats));
    stats->nsteps = (int)steps.size();
    for (size_t s = 0; s < steps.size(); ++s) {
      stats->step[s].kind = steps[s].kind;
      stats->step[s].rel = steps[s].rel;
      stats->step[s].rows_in = steps[s].slot_in >= 0
                                   ? (int64_t)c->h_misc[kMiscSteps + steps[s].slot_in]
                                   : steps[s].rows_in_host;
      stats->step[s].rows_out = (int64_t)c->h_misc[kMiscSteps + steps[s].slot_out];
    }
    for (int i = 0; i < n; ++i) stats->rows_final[i] = out_sieved[i]->nrows;
    stats->filter_bytes = filter_bytes;
  }
  return SJ_OK;
}

// ------------------------------------------------------------ batched pruning
// The pruning phases of many queries in lock step (the serving runtime's
// batches).  Every sieve step and filter build of every query gets a level,
// one more than the levels of what it reads: the step that produced its input
// relation and the builds of the filters it probes.  The steps of one level,
// over all queries, run as one k_sieve_batch launch and the builds of one
// level as one k_bloom_build_batch launch, so a batch takes as many launches
// as its longest schedule has levels instead of the sum over its queries.
// Each query gets exactly the filters and sieved relations its own
// sj_sieve_path computes: same schedule, same filter sizes, same order of
// surviving rows.  All relation versions stay allocated until the call ends.
struct BVer {
  const sj_rel_s* in = nullptr;  // version 0: the caller's relation
  sj_rel r = nullptr;            // later versions: a step's output
  int step = -1;                 // producing step
  int level = 0;
  int64_t cap = 0;
};
struct BFilter {
  sj_filter f = nullptr;
  int q = -1, ver = -1, col = 0, level = 0;
  bool given = false, cleared = false;
};
struct BStep {
  int q, rel, kind, level, ver_in, ver_out;
  bool pred;
  int32_t lo, hi;
  int pred_col;
  std::vector<std::pair<int, int>> probes;  // (column, batch filter id)
  std::vector<int> zero;                    // batch filter ids cleared by this step
  int chunk_rows = 0;
  int64_t nchunks = 0, chunk_g = 0;         // chunk_g: first chunk state of the call
};

sj_status sieve_path_batch_impl(sj_ctx* c, int nq, const sj_path* paths, const sj_sieve_opts* opts,
                                sj_rel* out_sieved, sj_sieve_stats* stats) {
  if (!c || nq < 0 || (nq > 0 && (!paths || !out_sieved))) return fail(c, SJ_EINVAL, "null argument");
  if (nq == 0) return SJ_OK;
  std::vector<BVer> vers;
  std::vector<BFilter> bf;
  std::vector<BStep> steps;
  std::vector<std::vector<int>> final_ver(nq);
  std::vector<sj_filter_params> qp(nq);
  int maxL = 0;

  // plan every query and give each operation its level
  for (int q = 0; q < nq; ++q) {
    const sj_path* path = &paths[q];
    Tree tr;
    SJ_TRY(validate_path(c, path, path->rels, &tr));
    const int n = path->nrel;
    for (int i = 0; i < n; ++i)
      if (path->rels[i]->nrows < 0) return fail(c, SJ_EINVAL, "relation row count unknown");
    sj_sieve_opts o{};
    if (opts) o = opts[q];
    qp[q] = norm_params(&o.filter);
    SJ_TRY(check_params(c, qp[q]));
    if (o.passes < SJ_FWD_BWD || o.passes > SJ_NO_SIEVE) return fail(c, SJ_EINVAL, "bad passes");
    PrunePlan pl;
    SJ_TRY(plan_pruning(c, path, tr, o, &pl));
    std::vector<int> fid(pl.given.size(), -1), cur(n);
    for (size_t k = 0; k < pl.given.size(); ++k) {
      if (!pl.given[k]) continue;
      BFilter b;
      b.f = pl.given[k];
      b.q = q;
      b.given = true;
      fid[k] = (int)bf.size();
      bf.push_back(b);
    }
    for (int i = 0; i < n; ++i) {
      BVer v;
      v.in = path->rels[i];
      v.cap = rel_cap(path->rels[i]);
      cur[i] = (int)vers.size();
      vers.push_back(v);
    }
    int nsteps_q = 0;
    for (size_t u = 0; u < pl.ops.size(); ++u) {
      const PruneOp& op = pl.ops[u];
      const int i = op.rel;
      if (op.type == kOpFinal) continue;
      if (op.type == kOpBuild) {
        if (fid[op.fid] < 0) {
          fid[op.fid] = (int)bf.size();
          bf.push_back(BFilter());
        }
        BFilter& b = bf[fid[op.fid]];
        b.q = q;
        b.ver = cur[i];
        b.col = op.col;
        b.level = vers[cur[i]].level + 1;
        maxL = std::max(maxL, b.level);
        continue;
      }
      if (++nsteps_q > SJ_MAX_STEPS) return fail(c, SJ_EINVAL, "too many sieve steps");
      BStep st{};
      st.q = q;
      st.rel = i;
      st.kind = op.kind;
      st.ver_in = cur[i];
      st.pred = op.pred;
      st.pred_col = op.pred ? path->preds[i].col : -1;
      st.lo = op.pred ? path->preds[i].lo : 0;
      st.hi = op.pred ? path->preds[i].hi : 0;
      st.level = vers[cur[i]].level + 1;
      for (auto& pr : op.probes) {
        st.probes.push_back({pr.first, fid[pr.second]});
        st.level = std::max(st.level, bf[fid[pr.second]].level + 1);
      }
      // the filters built from this step's output before relation i is sieved again
      for (size_t w = u + 1; w < pl.ops.size(); ++w) {
        const PruneOp& nx = pl.ops[w];
        if (nx.rel != i) continue;
        if (nx.type == kOpStep) break;
        if (nx.type != kOpBuild || (int)st.zero.size() == kMaxZero || fid[nx.fid] >= 0) continue;
        fid[nx.fid] = (int)bf.size();
        BFilter b;
        b.cleared = true;
        bf.push_back(b);
        st.zero.push_back(fid[nx.fid]);
      }
      maxL = std::max(maxL, st.level);
      BVer v;
      v.step = (int)steps.size();
      v.level = st.level;
      v.cap = vers[cur[i]].cap;
      st.ver_out = (int)vers.size();
      vers.push_back(v);
      cur[i] = st.ver_out;
      steps.push_back(st);
    }
    final_ver[q] = cur;
  }

  // allocations: step outputs, one block for all built filters (the ones no
  // step clears first, then the cleared ones), one block for the launch
  // arguments and the per-step counts
  void* fblock = nullptr;
  size_t fblock_bytes = 0, fclear_bytes = 0;
  void* ablock = nullptr;
  size_t ablock_bytes = 0;
  auto cleanup = [&]() {
    for (auto& v : vers) free_rel(c, v.r);
    for (auto& b : bf)
      if (!b.given) delete b.f;
    dfree(c, fblock, fblock_bytes);
    dfree(c, ablock, ablock_bytes);
  };
  std::vector<char> is_final(vers.size(), 0);
  for (int q = 0; q < nq; ++q)
    for (int i = 0; i < paths[q].nrel; ++i) is_final[final_ver[q][i]] = 1;
  for (auto& st : steps) {
    const BVer& vin = vers[st.ver_in];
    const sj_rel_s* in = vin.r ? vin.r : vin.in;
    vers[st.ver_out].r = new_rel(c, in->ncols, vin.cap, is_final[st.ver_out] != 0);
    if (!vers[st.ver_out].r) {
      cleanup();
      return fail(c, SJ_ENOMEM, "sieve output allocation failed");
    }
  }
  std::vector<uint64_t> qfilter_bytes(nq, 0);
  for (int pass = 0; pass < 2; ++pass) {
    for (auto& b : bf) {
      if (b.given || b.cleared != (pass == 1)) continue;
      const sj_filter_params& p = qp[b.q];
      uint64_t nbc = ((uint64_t)p.bits_per_key * (uint64_t)vers[b.ver].cap + 255) / 256;
      if (nbc < 1) nbc = 1;
      b.f = new sj_filter_s();
      b.f->p = p;
      b.f->nblocks_cap = nbc;
      b.f->mem_bytes = fblock_bytes;  // offset until the block exists
      fblock_bytes += kAlign + round_up(nbc * 32);
      qfilter_bytes[b.q] += nbc * 32;
    }
    if (pass == 0) fclear_bytes = fblock_bytes;
  }
  if (fblock_bytes) {
    fblock = dalloc(c, fblock_bytes);
    if (!fblock) {
      cleanup();
      return fail(c, SJ_ENOMEM, "filter allocation failed");
    }
    for (auto& b : bf) {
      if (b.given) continue;
      uint8_t* base = static_cast<uint8_t*>(fblock) + b.f->mem_bytes;
      b.f->mem = nullptr;  // part of the block
      b.f->mem_bytes = 0;
      b.f->hdr = reinterpret_cast<uint64_t*>(base);
      b.f->words = reinterpret_cast<uint32_t*>(base + kAlign);
    }
  }

  // per level: the steps and builds, their argument arrays and prefixes
  std::vector<std::vector<int>> lsteps(maxL + 1), lbuilds(maxL + 1);
  for (size_t s = 0; s < steps.size(); ++s) lsteps[steps[s].level].push_back((int)s);
  for (size_t k = 0; k < bf.size(); ++k)
    if (!bf[k].given) lbuilds[bf[k].level].push_back((int)k);
  int64_t total_chunks = 0;
  for (auto& st : steps) {
    st.chunk_rows = sieve_chunk_rows(vers[st.ver_in].cap, c->num_sms);
    st.nchunks = std::max<int64_t>(1, (vers[st.ver_in].cap + st.chunk_rows - 1) / st.chunk_rows);
    st.chunk_g = total_chunks;
    total_chunks += st.nchunks;
  }
  struct LevelOff { size_t sargs, schunk0, bargs, brow0; int64_t nchunks, nrows; int k_all; };
  std::vector<LevelOff> lo(maxL + 1);
  size_t off = 0;
  auto take = [&](size_t bytes) { const size_t o = off; off = round_up(off + bytes, 16); return o; };
  for (int L = 1; L <= maxL; ++L) {
    lo[L].sargs = take(sizeof(SieveArgs) * lsteps[L].size());
    lo[L].schunk0 = take(sizeof(int64_t) * (lsteps[L].size() + 1));
    lo[L].bargs = take(sizeof(BloomBuildArgs) * lbuilds[L].size());
    lo[L].brow0 = take(sizeof(int64_t) * (lbuilds[L].size() + 1));
  }
  const size_t args_bytes = off;
  const size_t counts_off = take(sizeof(uint64_t) * std::max<size_t>(steps.size(), 1));
  ablock_bytes = off;
  ablock = dalloc(c, ablock_bytes);
  if (!ablock) {
    cleanup();
    return fail(c, SJ_ENOMEM, "batch argument allocation failed");
  }
  uint8_t* dA = static_cast<uint8_t*>(ablock);
  uint64_t* d_counts = reinterpret_cast<uint64_t*>(dA + counts_off);
  // pinned staging: the arguments, then the counts read back
  if (c->batch_pending) {
    cudaStreamSynchronize(c->stream);
    c->batch_pending = false;
  }
  if (c->h_batch_bytes < ablock_bytes) {
    if (c->h_batch) cudaFreeHost(c->h_batch);
    c->h_batch = nullptr;
    c->h_batch_bytes = 0;
    void* h = nullptr;
    if (cudaHostAlloc(&h, round_up(ablock_bytes * 2), cudaHostAllocDefault) != cudaSuccess) {
      cudaGetLastError();
      cleanup();
      return fail(c, SJ_ENOMEM, "pinned staging allocation failed");
    }
    c->h_batch = static_cast<uint8_t*>(h);
    c->h_batch_bytes = round_up(ablock_bytes * 2);
  }
  uint8_t* hA = c->h_batch;
  uint32_t* ticket = nullptr;
  LookBack<1> lb;
  sj_status st = scratch_for<1>(c, total_chunks, &ticket, &lb);
  if (st != SJ_OK) {
    cleanup();
    return st;
  }
  auto rel_of_ver = [&](int v) -> const sj_rel_s* { return vers[v].r ? vers[v].r : vers[v].in; };
  for (int L = 1; L <= maxL; ++L) {
    SieveArgs* sa = reinterpret_cast<SieveArgs*>(hA + lo[L].sargs);
    int64_t* c0 = reinterpret_cast<int64_t*>(hA + lo[L].schunk0);
    int64_t acc = 0;
    int k_all = -1;
    for (size_t t = 0; t < lsteps[L].size(); ++t) {
      const BStep& S = steps[lsteps[L][t]];
      const sj_rel_s* in = rel_of_ver(S.ver_in);
      const sj_rel_s* r = vers[S.ver_out].r;
      SieveArgs& a = sa[t];
      memset(&a, 0, sizeof(a));
      if (S.pred) {
        a.test[a.ntest].col = in->cols[S.pred_col];
        a.test[a.ntest].is_pred = 1;
        a.test[a.ntest].lo = S.lo;
        a.test[a.ntest].hi = S.hi;
        a.ntest++;
      }
      for (auto& pr : S.probes) {
        a.test[a.ntest].col = in->cols[pr.first];
        a.test[a.ntest].f = view(bf[pr.second].f);
        a.ntest++;
      }
      const int vec_col = S.pred ? S.pred_col : (S.probes.empty() ? -1 : S.probes[0].first);
      a.nout = in->ncols;
      for (int j = 0; j < in->ncols; ++j) {
        a.in[j] = in->cols[j];
        a.out[j] = r->cols[j];
        a.out_is_vec[j] = j == vec_col ? 1 : 0;
      }
      a.n_host = in->d_n ? 0 : in->nrows;
      a.n_dev = in->d_n;
      a.out_n = r->d_n;
      a.out_n2 = d_counts + lsteps[L][t];
      a.tile_counter = ticket;
      a.lb = lb;
      a.lb.st = lb.st + S.chunk_g;
      a.fast_words_ok = 1;
      if (!S.pred && !S.probes.empty() && bf[S.probes[0].second].f->nblocks_cap * 8 >= (1ull << 32))
        a.fast_words_ok = 0;
      for (int z : S.zero) {
        a.zero_words[a.nzero] = bf[z].f->words;
        a.zero_bpk[a.nzero] = bf[z].f->p.bits_per_key;
        a.zero_cap_words[a.nzero] = bf[z].f->nblocks_cap * 8;
        a.nzero++;
      }
      a.chunk_rows = S.chunk_rows;
      c0[t] = acc;
      acc += S.nchunks;
      const bool fast = a.ntest == 1 && !a.test[0].is_pred && a.test[0].f.layout == 0 &&
                        a.test[0].f.k >= 1 && a.test[0].f.k <= 4 && a.fast_words_ok;
      const int kk = fast ? (int)a.test[0].f.k : 0;
      k_all = (k_all < 0 || k_all == kk) ? kk : 0;
    }
    c0[lsteps[L].size()] = acc;
    lo[L].nchunks = acc;
    lo[L].k_all = k_all < 0 ? 0 : k_all;
    BloomBuildArgs* ba = reinterpret_cast<BloomBuildArgs*>(hA + lo[L].bargs);
    int64_t* r0 = reinterpret_cast<int64_t*>(hA + lo[L].brow0);
    int64_t racc = 0;
    for (size_t t = 0; t < lbuilds[L].size(); ++t) {
      const BFilter& b = bf[lbuilds[L][t]];
      const sj_rel_s* rel = rel_of_ver(b.ver);
      BloomBuildArgs& a = ba[t];
      memset(&a, 0, sizeof(a));
      a.keys = rel->cols[b.col];
      a.n_host = rel->d_n ? 0 : rel->nrows;
      a.n_dev = rel->d_n;
      a.hdr = b.f->hdr;
      a.words = b.f->words;
      a.nblocks_cap = b.f->nblocks_cap;
      a.bits_per_key = b.f->p.bits_per_key;
      a.k = b.f->p.k;
      a.layout = b.f->p.layout;
      a.seed = b.f->p.seed;
      r0[t] = racc;
      racc += std::max<int64_t>(1, vers[b.ver].cap);
    }
    r0[lbuilds[L].size()] = racc;
    lo[L].nrows = racc;
  }

  // enqueue: clear the filters no step clears, copy the arguments, then two
  // launches per level; one synchronisation at the end
  const size_t p0 = c->prof.size();
  struct LRec { int L; bool build; size_t idx; };
  std::vector<LRec> recs;
  if (fclear_bytes) {
    cudaError_t e = cudaMemsetAsync(fblock, 0, fclear_bytes, c->stream);
    if (e != cudaSuccess) {
      cleanup();
      return fail(c, SJ_ECUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
    }
  }
  cudaError_t e = cudaMemcpyAsync(dA, hA, args_bytes, cudaMemcpyHostToDevice, c->stream);
  if (e != cudaSuccess) {
    cleanup();
    return fail(c, SJ_ECUDA, std::string("cudaMemcpyAsync: ") + cudaGetErrorString(e));
  }
  c->h2d_bytes += (int64_t)args_bytes;
  c->batch_pending = true;
  for (int L = 1; L <= maxL && st == SJ_OK; ++L) {
    if (!lbuilds[L].empty()) {
      BuildBatchArgs b;
      b.tasks = reinterpret_cast<const BloomBuildArgs*>(dA + lo[L].bargs);
      b.row0 = reinterpret_cast<const int64_t*>(dA + lo[L].brow0);
      b.ntask = (int)lbuilds[L].size();
      const size_t before = c->prof.size();
      {
        Launch rec(c, SJ_K_BLOOM_BUILD, 0.0);
        launch_bloom_build_batch(b, lo[L].nrows, c->num_sms, c->stream);
      }
      if (c->prof.size() > before) recs.push_back({L, true, before});
      st = check_launch(c, "k_bloom_build_batch");
    }
    if (st == SJ_OK && !lsteps[L].empty()) {
      SieveBatchArgs b;
      b.tasks = reinterpret_cast<const SieveArgs*>(dA + lo[L].sargs);
      b.chunk0 = reinterpret_cast<const int64_t*>(dA + lo[L].schunk0);
      b.ntask = (int)lsteps[L].size();
      b.ticket = ticket;
      const size_t before = c->prof.size();
      {
        Launch rec(c, SJ_K_SIEVE, 0.0);
        launch_sieve_batch(b, lo[L].nchunks, lo[L].k_all, c->stream);
      }
      if (c->prof.size() > before) recs.push_back({L, false, before});
      st = check_launch(c, "k_sieve_batch");
    }
  }
  uint64_t* h_counts = reinterpret_cast<uint64_t*>(hA + counts_off);
  if (st == SJ_OK && !steps.empty()) {
    e = cudaMemcpyAsync(h_counts, d_counts, sizeof(uint64_t) * steps.size(), cudaMemcpyDeviceToHost,
                        c->stream);
    if (e != cudaSuccess) st = fail(c, SJ_ECUDA, std::string("cudaMemcpyAsync: ") + cudaGetErrorString(e));
    c->d2h_bytes += (int64_t)(sizeof(uint64_t) * steps.size());
  }
  if (st == SJ_OK) st = sync_read(c);
  if (st != SJ_OK) {
    cudaStreamSynchronize(c->stream);
    c->batch_pending = false;
    cleanup();
    return st;
  }
  c->batch_pending = false;
  auto rows_of_ver = [&](int v) -> int64_t {
    return vers[v].step >= 0 ? (int64_t)h_counts[vers[v].step] : vers[v].in->nrows;
  };
  // algorithmic bytes of the profiled launches, as for the one-query launches
  for (auto& R : recs) {
    double bytes = 0;
    if (R.build) {
      for (int k : lbuilds[R.L])
        bytes += (4.0 + bf[k].f->p.bits_per_key / 8.0) * (double)rows_of_ver(bf[k].ver);
    } else {
      for (int s : lsteps[R.L]) {
        const BStep& S = steps[s];
        const int ncols = rel_of_ver(S.ver_in)->ncols;
        bytes += 4.0 * (double)rows_of_ver(S.ver_in) +
                 (4.0 * (ncols - 1) + 4.0 * ncols) * (double)h_counts[s];
      }
    }
    c->prof[R.idx].bytes = bytes;
  }
  prof_resolve(c, p0);
  // hand out the final versions; free the rest
  for (size_t v = 0; v < vers.size(); ++v) {
    if (!vers[v].r) continue;
    vers[v].r->nrows = rows_of_ver((int)v);
    // the count is known now: later calls size their work by it, not by the
    // input's row bound
    vers[v].r->cap = vers[v].r->nrows;
    if (!is_final[v]) free_rel(c, vers[v].r);
    vers[v].r = is_final[v] ? vers[v].r : nullptr;
  }
  for (int q = 0; q < nq; ++q) {
    for (int i = 0; i < paths[q].nrel; ++i) {
      const int v = final_ver[q][i];
      out_sieved[(size_t)q * SJ_MAX_REL + i] = vers[v].r ? vers[v].r : view_of(vers[v].in);
    }
    if (stats) {
      sj_sieve_stats& S = stats[q];
      memset(&S, 0, sizeof(S));
      for (const BStep& b : steps) {
        if (b.q != q) continue;
        auto& x = S.step[S.nsteps++];
        x.kind = b.kind;
        x.rel = b.rel;
        x.rows_in = rows_of_ver(b.ver_in);
        x.rows_out = rows_of_ver(b.ver_out);
      }
      for (int i = 0; i < paths[q].nrel; ++i) S.rows_final[i] = rows_of_ver(final_ver[q][i]);
      S.filter_bytes = qfilter_bytes[q];
    }
  }
  for (auto& b : bf)
    if (!b.given) delete b.f;
  dfree(c, fblock, fblock_bytes);
  dfree(c, ablock, ablock_bytes);
  return SJ_OK;
}

}  // namespace

// ======================================================================== join
namespace {

struct LevelPlan {
  int rel, rel_col;       // relation added at this level and its key column
  int probe_rel, probe_col;  // already-joined column it is equal to
};

// Left-deep order: start at relation 0, then repeatedly the lowest-index
// relation adjacent to the joined set.
std::vector<LevelPlan> join_order(const sj_path* p) {
  std::vector<LevelPlan> plan;
  std::vector<int> in(p->nrel, 0);
  in[0] = 1;
  for (int added = 1; added < p->nrel; ++added) {
    LevelPlan best{-1, 0, 0, 0};
    for (int e = 0; e < p->nrel - 1; ++e) {
      const sj_edge& E = p->edges[e];
      for (int side = 0; side < 2; ++side) {
        const int x = side ? E.rel_b : E.rel_a, cx = side ? E.col_b : E.col_a;
        const int y = side ? E.rel_a : E.rel_b, cy = side ? E.col_a : E.col_b;
        if (in[x] && !in[y] && (best.rel < 0 || y < best.rel)) best = {y, cy, x, cx};
      }
    }
    in[best.rel] = 1;
    plan.push_back(best);
  }
  return plan;
}

Terms terms_of(const sj_rel_s* r, int rel, int nrefs, const sj_colref* refs) {
  Terms t;
  memset(&t, 0, sizeof(t));
  for (int k = 0; k < nrefs; ++k) {
    if (refs[k].rel != rel) continue;
    t.col[t.n] = r->cols[refs[k].col];
    t.col_hi[t.n] = refs[k].wide ? r->cols[refs[k].col + 1] : nullptr;
    t.n++;
  }
  return t;
}

uint64_t pow2_at_least(uint64_t x) {
  uint64_t p = 1;
  while (p < x) p <<= 1;
  return p;
}

using ColKey = std::pair<int, int>;

struct Inter {
  std::map<ColKey, const int32_t*> cols;
  int64_t n = 0;
  uint64_t* psum = nullptr;
  bool base = true;  // still relation 0 itself
  std::vector<std::pair<void*, size_t>> mem;
};

void free_inter(sj_ctx* c, Inter& in) {
  for (auto& m : in.mem) dfree(c, m.first, m.second);
  in.mem.clear();
}

struct Table2 {
  Table t;
  uint64_t nslots;
};

// Largest hash-table build side: slot counts (up to 2^31 here) and row ids
// are held in 32 bits on the device.
constexpr int64_t kMaxTableRows = int64_t(1) << 30;

sj_status make_table(sj_ctx* c, Temps& tmp, int64_t nrows, Table2* out) {
  if (nrows > kMaxTableRows) return fail(c, SJ_EINVAL, "hash-table build side above 2^30 rows");
  sj_status st = SJ_OK;
  const uint64_t nslots = pow2_at_least(std::max<uint64_t>(64, 2 * (uint64_t)nrows));
  unsigned long long* slots = tmp.get<unsigned long long>(nslots, &st);
  if (!slots) return fail(c, st, "hash table allocation failed");
  SJ_CUDA(c, cudaMemsetAsync(slots, 0, nslots * 8, c->stream));
  out->t.slots = slots;
  out->t.bucket_mask = (uint32_t)(nslots / 4 - 1);
  out->nslots = nslots;
  return SJ_OK;
}

// Multimap of row ids keyed by `keys` (the same build as a join level): rows
// are grouped by the table slot of their key.
sj_status build_adjacency(sj_ctx* c, Temps& tmp, const int32_t* keys, int64_t n, Adjacency* g) {
  sj_status st = SJ_OK;
  Table2 tb;
  SJ_TRY(make_table(c, tmp, n, &tb));
  const int64_t ns = (int64_t)tb.nslots;
  uint32_t* cnt = tmp.get<uint32_t>(ns, &st);
  uint32_t* rid = tmp.get<uint32_t>(n, &st);
  uint32_t* rank = tmp.get<uint32_t>(n, &st);
  uint64_t* off = tmp.get<uint64_t>(ns, &st);
  int32_t* rows = tmp.get<int32_t>(n, &st);
  if (st != SJ_OK) return fail(c, st, "adjacency allocation failed");
  SJ_CUDA(c, cudaMemsetAsync(cnt, 0, (size_t)ns * 4, c->stream));
  MMInsertArgs mi{keys, n, tb.t, cnt, rid, rank, status_ptr(c)};
  {
    Launch L(c, SJ_K_HT_BUILD, 12.0 * (double)n);
    launch_mm_insert(mi, c->num_sms, c->stream);
  }
  SJ_TRY(check_launch(c, "k_mm_insert"));
  unsigned long long* cursor = tmp.get<unsigned long long>(1, &st);
  if (st != SJ_OK) return fail(c, st, "adjacency allocation failed");
  SJ_CUDA(c, cudaMemsetAsync(cursor, 0, sizeof(unsigned long long), c->stream));
  GroupOffArgs ga{cnt, off, ns, nullptr, cursor};
  {
    Launch L(c, SJ_K_HT_BUILD, 12.0 * (double)ns);
    launch_group_offsets(ga, ns, c->num_sms, c->stream);
  }
  SJ_TRY(check_launch(c, "k_group_offsets"));
  MMScatterArgs ms{rid, rank, off, n, rows};
  {
    Launch L(c, SJ_K_HT_BUILD, 20.0 * (double)n);
    launch_mm_scatter(ms, c->num_sms, c->stream);
  }
  SJ_TRY(check_launch(c, "k_mm_scatter"));
  g->t = tb.t;
  g->cnt = cnt;
  g->off = off;
  g->rows = rows;
  return SJ_OK;
}

}  // namespace

sj_status join_impl(sj_ctx* c, const sj_path* path, const sj_rel* inputs, int mode, int nrefs,
                    const sj_colref* refs, sj_result* result, std::vector<uint64_t>* levelT);

extern "C" sj_status sj_join(sj_ctx* c, const sj_path* path, const sj_rel* inputs, int mode,
                             int nrefs, const sj_colref* refs, sj_result* result) {
  if (!c) return SJ_EINVAL;
  // temporaries from the context's arena (results are allocated outside it)
  arena_begin(c);
  const sj_status st = join_impl(c, path, inputs, mode, nrefs, refs, result, nullptr);
  arena_end(c);
  return st;
}

// The enumeration phase with host-known sizes (one synchronisation per level);
// `levelT` (optional) receives the output tuples of every multimap level.
sj_status join_impl(sj_ctx* c, const sj_path* path, const sj_rel* inputs, int mode, int nrefs,
                    const sj_colref* refs, sj_result* result, std::vector<uint64_t>* levelT) {
  if (!c || !path || !result) return fail(c, SJ_EINVAL, "null argument");
  Tree tr;
  SJ_TRY(validate_path(c, path, path->rels, &tr));
  const int n = path->nrel;
  if (mode != SJ_COUNT_SUM && mode != SJ_MATERIALIZE) return fail(c, SJ_EINVAL, "bad mode");
  if (nrefs < 0 || nrefs > SJ_MAX_TERMS || (nrefs > 0 && !refs))
    return fail(c, SJ_EINVAL, "bad column references");
  if (mode == SJ_MATERIALIZE && nrefs < 1) return fail(c, SJ_EINVAL, "MATERIALIZE needs refs");
  std::vector<const sj_rel_s*> rels(n);
  for (int i = 0; i < n; ++i) {
    rels[i] = inputs ? inputs[i] : path->rels[i];
    if (!rels[i]) return fail(c, SJ_EINVAL, "null input relation");
    if (rels[i]->ncols != path->rels[i]->ncols) return fail(c, SJ_EINVAL, "input column count differs");
    if (rels[i]->nrows < 0) return fail(c, SJ_EINVAL, "relation row count unknown");
  }
  for (int k = 0; k < nrefs; ++k) {
    const sj_colref& r = refs[k];
    if (r.rel < 0 || r.rel >= n || r.col < 0 || r.col + (r.wide ? 1 : 0) >= rels[r.rel]->ncols)
      return fail(c, SJ_EINVAL, "column reference out of range");
    if (mode == SJ_MATERIALIZE && r.wide) return fail(c, SJ_EINVAL, "MATERIALIZE takes int32 refs");
  }

  // predicates of raw inputs
  std::vector<sj_rel> sel(n, nullptr);
  struct SelGuard {
    sj_ctx* c;
    std::vector<sj_rel>* v;
    ~SelGuard() {
      for (auto r : *v) free_rel(c, r);
    }
  } sel_guard{c, &sel};
  if (!inputs && path->preds) {
    bool any = false;
    const size_t p0 = c->prof.size();
    for (int i = 0; i < n; ++i) {
      if (!has_pred(path, i)) continue;
      std::vector<TestSpec> t{{path->preds[i].col, true, path->preds[i].lo, path->preds[i].hi, nullptr}};
      SJ_TRY(sieve_step_timed(c, rels[i], t, i, -1, &sel[i]));
      any = true;
    }
    if (any) {
      SJ_TRY(sync_read(c));
      prof_resolve(c, p0);
      for (int i = 0; i < n; ++i)
        if (sel[i]) {
          sel[i]->nrows = (int64_t)c->h_misc[kMiscSteps + i];
          rels[i] = sel[i];
        }
    }
  }

  memset(result, 0, sizeof(*result));
  const bool want_sum = mode == SJ_COUNT_SUM && nrefs > 0;
  const int nsm = c->num_sms;

  if (n == 1) {
    const sj_rel_s* r0 = rels[0];
    if (mode == SJ_COUNT_SUM) {
      result->count = (uint64_t)r0->nrows;
      if (want_sum && r0->nrows > 0) {
        SJ_CUDA(c, cudaMemsetAsync(c->d_misc + kMiscResult, 0, 3 * 8, c->stream));
        SumTermsArgs a;
        a.n = r0->nrows;
        a.terms = terms_of(r0, 0, nrefs, refs);
        a.result = reinterpret_cast<unsigned long long*>(c->d_misc + kMiscResult);
        {
          Launch L(c, SJ_K_AGG, 4.0 * a.terms.n * (double)a.n);
          launch_sum_terms(a, nsm, c->stream);
        }
        SJ_TRY(check_launch(c, "k_sum_terms"));
        SJ_TRY(sync_read(c));
        result->sum = c->h_misc[kMiscResult + 2];
      }
      return SJ_OK;
    }
    sj_rel out = new_rel(c, nrefs, r0->nrows, true);
    if (!out) return fail(c, SJ_ENOMEM, "result allocation failed");
    out->d_n = nullptr;
    out->nrows = r0->nrows;
    for (int k = 0; k < nrefs && r0->nrows > 0; ++k) {
      cudaError_t e = cudaMemcpyAsync(out->cols[k], r0->cols[refs[k].col], (size_t)r0->nrows * 4,
                                      cudaMemcpyDeviceToDevice, c->stream);
      if (e != cudaSuccess) {
        free_rel(c, out);
        return fail(c, SJ_ECUDA, std::string("cudaMemcpyAsync: ") + cudaGetErrorString(e));
      }
    }
    sj_status st = sync_read(c);
    if (st != SJ_OK) {
      free_rel(c, out);
      return st;
    }
    result->count = (uint64_t)out->nrows;
    result->rows = out;
    return SJ_OK;
  }

  const std::vector<LevelPlan> plan = join_order(path);
  Inter in;
  in.n = rels[0]->nrows;
  for (int col = 0; col < rels[0]->ncols; ++col) in.cols[{0, col}] = rels[0]->cols[col];
  std::vector<int> joined(n, 0);
  joined[0] = 1;
  uint64_t intermediate = 0;
  sj_rel out_rel = nullptr;
  sj_status st = SJ_OK;
  if (!c->ev_wait && cudaEventCreateWithFlags(&c->ev_wait, cudaEventDisableTiming) != cudaSuccess)
    return fail(c, SJ_ECUDA, "event creation failed");

  // Multimap tables of the non-final levels depend only on their relation, so
  // each is enqueued ahead of the wait for the previous level's totals.
  Temps keep(c);
  std::vector<Adjacency> tables(plan.size());
  std::vector<char> built(plan.size(), 0);
  auto is_mm = [&](size_t L) { return !(L + 1 == plan.size() && mode == SJ_COUNT_SUM); };
  auto enqueue_build = [&](size_t L) -> sj_status {
    const sj_rel_s* Bl = rels[plan[L].rel];
    built[L] = 1;
    tables[L] = Adjacency{};
    if (Bl->nrows == 0) return SJ_OK;
    return build_adjacency(c, keep, Bl->cols[plan[L].rel_col], Bl->nrows, &tables[L]);
  };

  for (size_t L = 0; L < plan.size() && st == SJ_OK; ++L) {
    const LevelPlan& lp = plan[L];
    const sj_rel_s* B = rels[lp.rel];
    const int64_t nb = B->nrows;
    const int64_t np = in.n;
    const bool last = L + 1 == plan.size();
    joined[lp.rel] = 1;
    const int32_t* pk = in.cols.at({lp.probe_rel, lp.probe_col});
    Temps tmp(c);

    if (last && mode == SJ_COUNT_SUM) {
      if (np == 0 || nb == 0) break;  // empty join
      // Per-key (count, sum) table on the smaller side, probed by the other:
      // COUNT += cnt and SUM += value(probe row) * cnt + sum for every hit.
      const bool swap = np < nb;  // build on the intermediate, probe with the relation
      const int64_t n_build = swap ? np : nb;
      Table2 tb;
      if ((st = make_table(c, tmp, n_build, &tb)) != SJ_OK) break;
      ulonglong2* cs = tmp.get<ulonglong2>(tb.nslots, &st);
      if (st != SJ_OK) {
        fail(c, st, "aggregate table allocation failed");
        break;
      }
      cudaMemsetAsync(cs, 0, tb.nslots * 16, c->stream);
      cudaMemsetAsync(c->d_misc + kMiscResult, 0, 3 * 8, c->stream);
      Terms none;
      memset(&none, 0, sizeof(none));
      const Terms rel_terms = want_sum ? terms_of(B, lp.rel, nrefs, refs) : none;
      const Terms base_terms = (want_sum && in.base) ? terms_of(rels[0], 0, nrefs, refs) : none;
      const uint64_t* inter_vals = (want_sum && !in.base) ? in.psum : nullptr;
      AggInsertArgs ai;
      ai.keys = swap ? pk : B->cols[lp.rel_col];
      ai.n = n_build;
      ai.t = tb.t;
      ai.terms = swap ? base_terms : rel_terms;
      ai.vals = swap ? inter_vals : nullptr;
      ai.cs = cs;
      ai.status = status_ptr(c);
      {
        Launch Lk(c, SJ_K_AGG, (4.0 + 4.0 * ai.terms.n + (ai.vals ? 8.0 : 0.0)) * (double)n_build);
        launch_agg_insert(ai, nsm, c->stream);
      }
      if ((st = check_launch(c, "k_agg_insert")) != SJ_OK) break;
      AggProbeArgs ap;
      ap.keys = swap ? B->cols[lp.rel_col] : pk;
      ap.n = swap ? nb : np;
      ap.t = tb.t;
      ap.cs = cs;
      ap.probe_terms = swap ? rel_terms : base_terms;
      ap.psum_in = swap ? nullptr : inter_vals;
      ap.result = reinterpret_cast<unsigned long long*>(c->d_misc + kMiscResult);
      ap.status = status_ptr(c);
      {
        // the key of every probe row; a matching row's terms are not counted
        // (their count is known only on the device)
        Launch Lk(c, SJ_K_AGG, 4.0 * (double)ap.n);
        launch_agg_probe(ap, nsm, c->stream);
      }
      if ((st = check_launch(c, "k_agg_probe")) != SJ_OK) break;
      if ((st = sync_read(c)) != SJ_OK) break;
      const uint64_t lo = c->h_misc[kMiscResult], hi = c->h_misc[kMiscResult + 1];
      if (hi != 0 || lo >= (1ull << 63)) {
        st = fail(c, SJ_EOVERFLOW, "COUNT(*) reached 2^63");
        break;
      }
      result->count = lo;
      result->sum = c->h_misc[kMiscResult + 2];
      break;
    }

    // ---- multimap level: build on B, probe with the intermediate, expand
    // columns that must survive this level
    std::vector<ColKey> carried;
    if (last) {
      for (int k = 0; k < nrefs; ++k) carried.push_back({refs[k].rel, refs[k].col});
    } else {
      std::map<ColKey, int> need;
      for (size_t L2 = L + 1; L2 < plan.size(); ++L2)
        if (joined[plan[L2].probe_rel]) need[{plan[L2].probe_rel, plan[L2].probe_col}] = 1;
      if (mode == SJ_MATERIALIZE)
        for (int k = 0; k < nrefs; ++k)
          if (joined[refs[k].rel]) need[{refs[k].rel, refs[k].col}] = 1;
      for (auto& kv : need) carried.push_back(kv.first);
    }
    const bool carry_sum = want_sum && !last;

    uint64_t Q = 0, T = 0;
    int32_t *prow = nullptr, *pid = nullptr;
    uint64_t* o = nullptr;
    if (!built[L] && (st = enqueue_build(L)) != SJ_OK) break;
    const Adjacency& G = tables[L];
    if (np > 0 && nb > 0) {
      prow = tmp.get<int32_t>(np, &st);
      pid = tmp.get<int32_t>(np, &st);
      o = tmp.get<uint64_t>(np, &st);
      if (st != SJ_OK) {
        fail(c, st, "join level allocation failed");
        break;
      }
      MMProbeArgs mp;
      mp.keys = pk;
      mp.n = np;
      mp.t = G.t;
      mp.cnt = G.cnt;
      mp.prow = prow;
      mp.pid = pid;
      mp.o = o;
      mp.totals = c->d_misc + kMiscTotals;
      if ((st = scratch_for<2>(c, (np + kProbeTile - 1) / kProbeTile, &mp.tile_counter, &mp.lb)) !=
          SJ_OK)
        break;
      {
        Launch Lk(c, SJ_K_HT_PROBE, 4.0 * (double)np);
        launch_mm_probe(mp, c->num_sms, c->stream);
      }
      if ((st = check_launch(c, "k_mm_probe")) != SJ_OK) break;
      // read the level's totals at an event, and let the next level's table
      // build run on the device meanwhile
      if (cudaMemcpyAsync(c->h_misc + kMiscTotals, c->d_misc + kMiscTotals, 16,
                          cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
          cudaEventRecord(c->ev_wait, c->stream) != cudaSuccess) {
        st = fail(c, SJ_ECUDA, "level totals readback failed");
        break;
      }
      c->d2h_bytes += 16;
      if (L + 1 < plan.size() && is_mm(L + 1) && !built[L + 1] && (st = enqueue_build(L + 1)) != SJ_OK)
        break;
      if (cudaEventSynchronize(c->ev_wait) != cudaSuccess) {
        st = fail(c, SJ_ECUDA, "level totals wait failed");
        break;
      }
      Q = c->h_misc[kMiscTotals];
      T = c->h_misc[kMiscTotals + 1];
      if (c->prof_on && !c->prof.empty()) {
        for (size_t r = c->prof.size(); r-- > 0;)
          if (c->prof[r].kind == SJ_K_HT_PROBE) {
            c->prof[r].bytes += 16.0 * (double)Q;
            break;
          }
      }
    }
    if (levelT) levelT->push_back(T);
    const int32_t* rows = G.rows;
    const uint64_t* off = G.off;
    if (!last) intermediate += T;
    if (T >= (uint64_t(1) << 31) * 16) {
      st = fail(c, SJ_ENOMEM, "intermediate result too large");
      break;
    }

    // outputs of this level
    Inter nx;
    nx.n = (int64_t)T;
    nx.base = false;
    std::vector<int32_t*> outs;
    if (last) {
      out_rel = new_rel(c, nrefs, (int64_t)T, true);
      if (!out_rel) {
        st = fail(c, SJ_ENOMEM, "result allocation failed");
        break;
      }
      out_rel->d_n = nullptr;
      out_rel->nrows = (int64_t)T;
      for (int k = 0; k < nrefs; ++k) outs.push_back(out_rel->cols[k]);
    } else {
      for (auto& ck : carried) {
        void* p = dalloc(c, std::max<uint64_t>(T, 1) * 4);
        if (!p) {
          st = SJ_ENOMEM;
          break;
        }
        nx.mem.push_back({p, std::max<uint64_t>(T, 1) * 4});
        nx.cols[ck] = static_cast<int32_t*>(p);
        outs.push_back(static_cast<int32_t*>(p));
      }
      if (st == SJ_OK && carry_sum) {
        void* p = dalloc(c, std::max<uint64_t>(T, 1) * 8);
        if (!p) st = SJ_ENOMEM;
        else {
          nx.mem.push_back({p, std::max<uint64_t>(T, 1) * 8});
          nx.psum = static_cast<uint64_t*>(p);
        }
      }
      if (st != SJ_OK) {
        free_inter(c, nx);
        fail(c, st, "intermediate allocation failed");
        break;
      }
    }
    if (T > 0) {
      // one expand launch per group of at most kMaxCols output columns
      const size_t ncar = carried.size();
      for (size_t c0 = 0; c0 < std::max<size_t>(ncar, 1) && st == SJ_OK; c0 += kMaxCols) {
        MMExpandArgs ex;
        memset(&ex, 0, sizeof(ex));
        ex.T = T;
        ex.Q = Q;
        ex.o = o;
        ex.prow = prow;
        ex.pid = pid;
        ex.off = off;
        ex.rows = rows;
        const size_t c1 = std::min(ncar, c0 + kMaxCols);
        for (size_t k = c0; k < c1; ++k) {
          const ColKey ck = carried[k];
          const int slot = (int)(k - c0);
          ex.src_build[slot] = ck.first == lp.rel ? 1 : 0;
          ex.src[slot] = ck.first == lp.rel ? B->cols[ck.second] : in.cols.at(ck);
          ex.out[slot] = outs[k];
        }
        ex.nout = (int)(c1 - c0);
        if (c0 == 0 && carry_sum) {
          ex.psum_out = nx.psum;
          if (in.base) ex.probe_terms = terms_of(rels[0], 0, nrefs, refs);
          else ex.psum_in = in.psum;
          ex.build_terms = terms_of(B, lp.rel, nrefs, refs);
        }
        {
          const double per = 8.0 * ex.nout + (ex.psum_out ? 16.0 : 0.0) + 12.0;
          Launch Lk(c, SJ_K_HT_EXPAND, per * (double)T);
          launch_mm_expand(ex, c->stream);
        }
        st = check_launch(c, "k_mm_expand");
      }
    }
    if (st != SJ_OK) {
      free_inter(c, nx);
      break;
    }
    free_inter(c, in);
    in = std::move(nx);
    if (last) {
      result->count = T;
      st = sync_read(c);
    }
  }
  free_inter(c, in);
  if (st != SJ_OK) {
    free_rel(c, out_rel);
    return st;
  }
  if (mode == SJ_MATERIALIZE) {
    if (!out_rel) {  // an empty level before the last
      out_rel = new_rel(c, nrefs, 0, true);
      if (!out_rel) return fail(c, SJ_ENOMEM, "result allocation failed");
      out_rel->d_n = nullptr;
      out_rel->nrows = 0;
    }
    result->rows = out_rel;
    result->count = (uint64_t)out_rel->nrows;
  }
  result->intermediate = intermediate;
  return SJ_OK;
}

// ======================================================================== device-sized join
namespace {

struct AsyncInter {
  std::map<ColKey, const int32_t*> cols;
  const uint64_t* n_dev = nullptr;  // null: n_host is the row count
  int slot = -1;                    // statistics slot of *n_dev (profiling), -1 if unknown
  int64_t n_host = 0;
  int64_t cap = 0;                  // rows allocated
  const uint64_t* psum = nullptr;
  bool base = true;
};

// Multimap build whose row count may be known on the device only: the table
// is allocated for `cap` rows and sized and cleared by k_table_init.
// n_slot: statistics slot of the device row count (-1: n_host is exact).
// Algorithmic bytes per row: at least 2 table slots of 8 + 4 bytes cleared
// and, for the offsets, read and written (12 bytes each); 12 (key read, slot
// and rank written); 20 (slot, rank, offset read, row written).
sj_status build_adjacency_dev(sj_ctx* c, Temps& tmp, const int32_t* keys, const uint64_t* n_dev,
                              int64_t n_host, int64_t cap, uint32_t* mask, uint32_t* nslots_dev,
                              Adjacency* g, int n_slot) {
  if (cap > kMaxTableRows) return fail(c, SJ_EINVAL, "hash-table build side above 2^30 rows");
  sj_status st = SJ_OK;
  const int sms = c->num_sms;
  const int64_t capn = std::max<int64_t>(cap, 1);
  const uint64_t cap_slots = pow2_at_least(std::max<uint64_t>(64, 2 * (uint64_t)capn));
  unsigned long long* slots = tmp.get<unsigned long long>(cap_slots, &st);
  uint32_t* cnt = tmp.get<uint32_t>(cap_slots, &st);
  uint32_t* rid = tmp.get<uint32_t>(capn, &st);
  uint32_t* rank = tmp.get<uint32_t>(capn, &st);
  uint64_t* off = tmp.get<uint64_t>(cap_slots, &st);
  int32_t* rows = tmp.get<int32_t>(capn, &st);
  unsigned long long* cursor = tmp.get<unsigned long long>(1, &st);
  if (st != SJ_OK) return fail(c, st, "adjacency allocation failed");
  TableInitArgs ti{slots, mask, n_dev, n_host, nullptr, cnt, nslots_dev, cursor};
  {
    Launch L = rows_launch(c, SJ_K_HT_BUILD, 24.0, n_slot, n_host);
    launch_table_init(ti, (int64_t)cap_slots, sms, c->stream);
  }
  SJ_TRY(check_launch(c, "k_table_init"));
  Table t;
  t.slots = slots;
  t.bucket_mask = 0;
  t.mask_dev = mask;
  MMInsertArgs mi{keys, cap, t, cnt, rid, rank, status_ptr(c)};
  mi.n_dev = n_dev;
  if (!n_dev) mi.n = n_host;
  {
    Launch L = rows_launch(c, SJ_K_HT_BUILD, 12.0, n_slot, n_host);
    launch_mm_insert(mi, sms, c->stream);
  }
  SJ_TRY(check_launch(c, "k_mm_insert"));
  GroupOffArgs ga{cnt, off, 0, nslots_dev, cursor};
  {
    Launch L = rows_launch(c, SJ_K_HT_BUILD, 24.0, n_slot, n_host);
    launch_group_offsets(ga, (int64_t)cap_slots, sms, c->stream);
  }
  SJ_TRY(check_launch(c, "k_group_offsets"));
  MMScatterArgs ms{rid, rank, off, n_dev ? cap : n_host, rows};
  ms.n_dev = n_dev;
  {
    Launch L = rows_launch(c, SJ_K_HT_BUILD, 20.0, n_slot, n_host);
    launch_mm_scatter(ms, sms, c->stream);
  }
  SJ_TRY(check_launch(c, "k_mm_scatter"));
  g->t = t;
  g->cnt = cnt;
  g->off = off;
  g->rows = rows;
  return SJ_OK;
}

// Enqueue on the side stream (with its own scratch) while in scope.
struct OnSide {
  sj_ctx* c;
  explicit OnSide(sj_ctx* cc) : c(cc) { flip(); }
  ~OnSide() { flip(); }
  void flip() {
    std::swap(c->stream, c->side);
    std::swap(c->scratch, c->scratch2);
    std::swap(c->scratch_bytes, c->scratch2_bytes);
    std::swap(c->epoch, c->epoch2);
  }
};

// Waits for the side stream when a call leaves early (on success the main
// stream has already waited for all of its work).
struct SideDrain {
  sj_ctx* c;
  ~SideDrain() {
    if (c->side && !c->capturing) cudaStreamSynchronize(c->side);
  }
};

sj_status ensure_side(sj_ctx* c, int nlev) {
  int prio_least = 0, prio_greatest = 0;
  if (cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest) != cudaSuccess) {
    cudaGetLastError();
    prio_least = 0;
  }
  if (!c->side && cudaStreamCreateWithPriority(&c->side, cudaStreamNonBlocking, prio_least) != cudaSuccess)
    return fail(c, SJ_ECUDA, "side stream creation failed");
  if (!c->ev_ready && cudaEventCreateWithFlags(&c->ev_ready, cudaEventDisableTiming) != cudaSuccess)
    return fail(c, SJ_ECUDA, "event creation failed");
  for (int L = 0; L < nlev; ++L)
    if (!c->ev_built[L] && cudaEventCreateWithFlags(&c->ev_built[L], cudaEventDisableTiming) != cudaSuccess)
      return fail(c, SJ_ECUDA, "event creation failed");
  return SJ_OK;
}

sj_status device_sized_result(sj_ctx* c, int nlev, sj_result* result, std::vector<uint64_t>* levelT);

// COUNT/SUM join with every size kept on the device: no host round trip
// until the one synchronisation at the end.  caps[L] bounds the output of
// multimap level L; a level that outgrows it records kErrCapacity and the call
// returns kRetry (the caller reruns the exact, synchronising join).
sj_status join_async(sj_ctx* c, const sj_path* path, const sj_rel* in_rels, int nrefs,
                     const sj_colref* refs, const std::vector<uint64_t>& caps, sj_result* result,
                     std::vector<uint64_t>* levelT, const std::vector<Adjacency>* prebuilt,
                     bool finish = true, const std::vector<int>* rel_slot = nullptr) {
  const int n = path->nrel;
  std::vector<const sj_rel_s*> rels(in_rels, in_rels + n);
  const std::vector<LevelPlan> plan = join_order(path);
  if (plan.size() != caps.size() + 1) return kRetry;
  const bool want_sum = nrefs > 0;
  Temps keep(c);
  sj_status st = SJ_OK;
  uint32_t* small = keep.get<uint32_t>(64, &st);
  if (st != SJ_OK) return fail(c, st, "allocation failed");
  SJ_CUDA(c, cudaMemsetAsync(c->d_misc + kMiscResult, 0, 3 * 8, c->stream));
  AsyncInter in;
  for (int col = 0; col < rels[0]->ncols; ++col) in.cols[{0, col}] = rels[0]->cols[col];
  in.n_dev = rels[0]->d_n;
  in.n_host = rels[0]->nrows;
  in.cap = rel_cap(rels[0]);
  auto slot_of = [&](int i) { return (rel_slot && rels[i]->d_n) ? (*rel_slot)[i] : -1; };
  in.slot = slot_of(0);
  std::vector<int> joined(n, 0);
  joined[0] = 1;
  Terms none;
  memset(&none, 0, sizeof(none));
  // the multimap of every non-final level depends only on its relation:
  // all of them are built on the side stream while the main stream probes
  const int nlev = (int)plan.size() - 1;
  std::vector<Adjacency> built(std::max(nlev, 0));
  SideDrain drain{c};
  if (prebuilt) {
    if ((int)prebuilt->size() != nlev) return kRetry;
    built = *prebuilt;  // enqueued on the side stream during the pruning phase
  } else if (nlev > 0) {
    SJ_TRY(ensure_side(c, nlev));
    SJ_CUDA(c, cudaEventRecord(c->ev_ready, c->stream));
    OnSide side(c);
    SJ_CUDA(c, cudaStreamWaitEvent(c->stream, c->ev_ready, 0));
    for (int L = 0; L < nlev; ++L) {
      const sj_rel_s* B = rels[plan[L].rel];
      SJ_TRY(build_adjacency_dev(c, keep, B->cols[plan[L].rel_col], B->d_n, B->nrows, rel_cap(B),
                                 small + 2 * L, small + 2 * L + 1, &built[L], slot_of(plan[L].rel)));
      SJ_CUDA(c, cudaEventRecord(c->ev_built[L], c->stream));
    }
  }
  for (size_t L = 0; L < plan.size(); ++L) {
    const LevelPlan& lp = plan[L];
    const sj_rel_s* B = rels[lp.rel];
    joined[lp.rel] = 1;
    const int32_t* pk = in.cols.at({lp.probe_rel, lp.probe_col});
    const int64_t capB = rel_cap(B);
    if (L + 1 == plan.size()) {
      // final level: per-key (count, sum) table on the side with the smaller capacity
      const bool swap = in.cap < capB;
      const Terms rel_terms = want_sum ? terms_of(B, lp.rel, nrefs, refs) : none;
      const Terms base_terms = (want_sum && in.base) ? terms_of(rels[0], 0, nrefs, refs) : none;
      const uint64_t* inter_vals = (want_sum && !in.base) ? in.psum : nullptr;
      const int64_t cap_build = swap ? in.cap : capB;
      const uint64_t cap_slots = pow2_at_least(std::max<uint64_t>(64, 2 * (uint64_t)std::max<int64_t>(cap_build, 1)));
      unsigned long long* slots = keep.get<unsigned long long>(cap_slots, &st);
      ulonglong2* cs = keep.get<ulonglong2>(cap_slots, &st);
      if (st != SJ_OK) return fail(c, st, "aggregate table allocation failed");
      TableInitArgs ti{slots, small + 2 * L, swap ? in.n_dev : B->d_n, swap ? in.n_host : B->nrows,
                       cs, nullptr, nullptr};
      const int bslot = swap ? in.slot : slot_of(lp.rel);
      const int64_t bhost = swap ? in.n_host : B->nrows;
      const int pslot = swap ? slot_of(lp.rel) : in.slot;
      const int64_t phost = swap ? B->nrows : in.n_host;
      {
        // at least 2 slots of 8 + 16 bytes cleared per build row
        Launch Lk = rows_launch(c, SJ_K_AGG, 48.0, bslot, bhost);
        launch_table_init(ti, (int64_t)cap_slots, c->num_sms, c->stream);
      }
      SJ_TRY(check_launch(c, "k_table_init"));
      Table t;
      t.slots = slots;
      t.bucket_mask = 0;
      t.mask_dev = small + 2 * L;
      AggInsertArgs ai;
      ai.keys = swap ? pk : B->cols[lp.rel_col];
      ai.n = swap ? (in.n_dev ? in.cap : in.n_host) : (B->d_n ? capB : B->nrows);
      ai.n_dev = swap ? in.n_dev : B->d_n;
      ai.t = t;
      ai.terms = swap ? base_terms : rel_terms;
      ai.vals = swap ? inter_vals : nullptr;
      ai.cs = cs;
      ai.status = status_ptr(c);
      {
        // key and SUM terms (or the intermediate's partial sum) per build row
        Launch Lk = rows_launch(c, SJ_K_AGG, 4.0 + 4.0 * ai.terms.n + (ai.vals ? 8.0 : 0.0), bslot, bhost);
        launch_agg_insert(ai, c->num_sms, c->stream);
      }
      SJ_TRY(check_launch(c, "k_agg_insert"));
      AggProbeArgs ap;
      ap.keys = swap ? B->cols[lp.rel_col] : pk;
      ap.n = swap ? (B->d_n ? capB : B->nrows) : (in.n_dev ? in.cap : in.n_host);
      ap.n_dev = swap ? B->d_n : in.n_dev;
      ap.t = t;
      ap.cs = cs;
      ap.probe_terms = swap ? rel_terms : base_terms;
      ap.psum_in = swap ? nullptr : inter_vals;
      ap.result = reinterpret_cast<unsigned long long*>(c->d_misc + kMiscResult);
      ap.status = status_ptr(c);
      {
        // the key of every probe row (a matching row's SUM terms or partial
        // sum are read too but not counted: their count is known only on the
        // device)
        Launch Lk = rows_launch(c, SJ_K_AGG, 4.0, pslot, phost);
        launch_agg_probe(ap, c->num_sms, c->stream);
      }
      SJ_TRY(check_launch(c, "k_agg_probe"));
      break;
    }
    // ---- multimap level
    const Adjacency G = built[L];
    SJ_CUDA(c, cudaStreamWaitEvent(c->stream, c->ev_built[L], 0));
    const int64_t capP = std::max<int64_t>(in.cap, 1);
    int32_t* prow = keep.get<int32_t>(capP, &st);
    int32_t* pid = keep.get<int32_t>(capP, &st);
    uint64_t* o = keep.get<uint64_t>(capP, &st);
    if (st != SJ_OK) return fail(c, st, "join level allocation failed");
    uint64_t* totals = c->d_misc + kMiscLevelTotals + 2 * L;
    MMProbeArgs mp;
    mp.keys = pk;
    mp.n = in.n_dev ? in.cap : in.n_host;
    mp.n_dev = in.n_dev;
    mp.t = G.t;
    mp.cnt = G.cnt;
    mp.prow = prow;
    mp.pid = pid;
    mp.o = o;
    mp.totals = totals;
    SJ_TRY(scratch_for<2>(c, (capP + kProbeTile - 1) / kProbeTile, &mp.tile_counter, &mp.lb));
    {
      // 4 bytes per probe row (key), 16 per matching row (row, id and offset written)
      Launch Lk = in.slot >= 0 ? Launch(c, SJ_K_HT_PROBE, 0.0, in.slot, 4.0, kSlotLevelTotals + 2 * (int)L, 16.0)
                               : Launch(c, SJ_K_HT_PROBE, 4.0 * (double)std::max<int64_t>(in.n_host, 0),
                                        kSlotLevelTotals + 2 * (int)L, 16.0);
      launch_mm_probe(mp, c->num_sms, c->stream);
    }
    SJ_TRY(check_launch(c, "k_mm_probe"));
    std::map<ColKey, int> need;
    for (size_t L2 = L + 1; L2 < plan.size(); ++L2)
      if (joined[plan[L2].probe_rel]) need[{plan[L2].probe_rel, plan[L2].probe_col}] = 1;
    std::vector<ColKey> carried;
    for (auto& kv : need) carried.push_back(kv.first);
    const uint64_t C = std::max<uint64_t>(caps[L], 1);
    AsyncInter nx;
    nx.base = false;
    nx.cap = (int64_t)C;
    nx.n_dev = c->d_misc + kMiscLevelCount + L;
    nx.slot = kSlotLevelCount + (int)L;
    for (auto& ck : carried) nx.cols[ck] = keep.get<int32_t>(C, &st);
    uint64_t* psum_out = want_sum ? keep.get<uint64_t>(C, &st) : nullptr;
    if (st != SJ_OK) return fail(c, st, "intermediate allocation failed");
    nx.psum = psum_out;
    const size_t ncar = carried.size();
    for (size_t c0 = 0; c0 < std::max<size_t>(ncar, 1); c0 += kMaxCols) {
      MMExpandArgs ex;
      memset(&ex, 0, sizeof(ex));
      ex.o = o;
      ex.prow = prow;
      ex.pid = pid;
      ex.off = G.off;
      ex.rows = G.rows;
      const size_t c1 = std::min(ncar, c0 + kMaxCols);
      for (size_t k = c0; k < c1; ++k) {
        const ColKey ck = carried[k];
        const int slot = (int)(k - c0);
        ex.src_build[slot] = ck.first == lp.rel ? 1 : 0;
        ex.src[slot] = ck.first == lp.rel ? B->cols[ck.second] : in.cols.at(ck);
        ex.out[slot] = const_cast<int32_t*>(nx.cols[ck]);
      }
      ex.nout = (int)(c1 - c0);
      if (c0 == 0 && want_sum) {
        ex.psum_out = psum_out;
        if (in.base) ex.probe_terms = terms_of(rels[0], 0, nrefs, refs);
        else ex.psum_in = in.psum;
        ex.build_terms = terms_of(B, lp.rel, nrefs, refs);
      }
      ex.totals_dev = totals;
      ex.cap = C;
      ex.n_out = c->d_misc + kMiscLevelCount + L;
      ex.status = status_ptr(c);
      {
        // per output tuple: each carried column read and written, the partial
        // sum read and written, and the tuple's probe row, key id and offset
        const double per = 8.0 * ex.nout + (ex.psum_out ? 16.0 : 0.0) + 12.0;
        Launch Lk(c, SJ_K_HT_EXPAND, 0.0, kSlotLevelCount + (int)L, per);
        launch_mm_expand_dev(ex, c->num_sms, c->stream);
      }
      SJ_TRY(check_launch(c, "k_mm_expand_dev"));
    }
    in = std::move(nx);
  }
  if (!finish) return enqueue_readback(c);  // graph capture: results read at replay
  SJ_TRY(sync_read(c));
  prof_resolve(c, 0);
  return device_sized_result(c, (int)plan.size() - 1, result, levelT);
}

// COUNT, SUM and per-level sizes of a finished device-sized join, from h_misc.
sj_status device_sized_result(sj_ctx* c, int nlev, sj_result* result, std::vector<uint64_t>* levelT) {
  const uint64_t lo = c->h_misc[kMiscResult], hi = c->h_misc[kMiscResult + 1];
  if (hi != 0 || lo >= (1ull << 63)) return fail(c, SJ_EOVERFLOW, "COUNT(*) reached 2^63");
  memset(result, 0, sizeof(*result));
  result->count = lo;
  result->sum = c->h_misc[kMiscResult + 2];
  for (int L = 0; L < nlev; ++L) {
    const uint64_t T = c->h_misc[kMiscLevelTotals + 2 * L + 1];
    result->intermediate += T;
    if (levelT) levelT->push_back(T);
  }
  return SJ_OK;
}

uint64_t mix_in(uint64_t h, uint64_t v) {
  h ^= v + 0x9e3779b97f4a7c15ull + (h << 6) + (h >> 2);
  return h;
}

// Signature of a query shape for the capacity cache.
uint64_t path_signature(const sj_path* p, const sj_sieve_opts* o, int mode, int nrefs,
                        const sj_colref* refs) {
  uint64_t h = 0x51e7e70117ull;
  h = mix_in(h, (uint64_t)p->nrel);
  h = mix_in(h, (uint64_t)(int64_t)p->root);
  for (int i = 0; i < p->nrel; ++i) {
    // the device addresses, not the handle: a graph of this shape reads the
    // columns directly, so a new handle over the same buffers (a relation
    // reloaded each request) replays it; changed contents are caught by the
    // buffer-overflow check of the device-sized run
    const sj_rel_s* r = p->rels[i];
    h = mix_in(h, (uint64_t)r->nrows);
    h = mix_in(h, (uint64_t)reinterpret_cast<uintptr_t>(r->d_n));
    for (int j = 0; j < r->ncols; ++j) h = mix_in(h, (uint64_t)reinterpret_cast<uintptr_t>(r->cols[j]));
    if (p->preds)
      h = mix_in(h, ((uint64_t)(uint32_t)p->preds[i].col << 40) ^ ((uint64_t)(uint32_t)p->preds[i].lo << 20) ^
                        (uint64_t)(uint32_t)p->preds[i].hi);
  }
  for (int e = 0; e + 1 < p->nrel; ++e)
    h = mix_in(h, ((uint64_t)p->edges[e].rel_a << 48) ^ ((uint64_t)p->edges[e].col_a << 32) ^
                      ((uint64_t)p->edges[e].rel_b << 16) ^ (uint64_t)p->edges[e].col_b);
  if (o) {
    h = mix_in(h, (uint64_t)o->passes);
    h = mix_in(h, ((uint64_t)o->filter.bits_per_key << 32) ^ ((uint64_t)o->filter.k << 8) ^ o->filter.layout);
    h = mix_in(h, o->filter.seed);
    if (o->leaf_filters)
      for (int i = 0; i < p->nrel; ++i) {
        const sj_filter_s* f = o->leaf_filters[i];
        h = mix_in(h, (uint64_t)reinterpret_cast<uintptr_t>(f));
        if (f) {
          h = mix_in(h, (uint64_t)reinterpret_cast<uintptr_t>(f->words));
          h = mix_in(h, (uint64_t)reinterpret_cast<uintptr_t>(f->hdr));
        }
      }
  }
  h = mix_in(h, (uint64_t)mode);
  for (int k = 0; k < nrefs; ++k)
    h = mix_in(h, ((uint64_t)refs[k].rel << 32) ^ ((uint64_t)refs[k].col << 8) ^ (uint64_t)refs[k].wide);
  return h;
}

}  // namespace

// ======================================================================== profiling
extern "C" {

sj_status sj_prof_enable(sj_ctx* c, int on) {
  if (!c) return SJ_EINVAL;
  c->prof_on = on != 0;
  return SJ_OK;
}

sj_status sj_prof_kinds(sj_ctx* c, uint32_t mask) {
  if (!c) return SJ_EINVAL;
  c->prof_mask = mask;
  return SJ_OK;
}

static sj_status prof_collect(sj_ctx* c) {
  SJ_CUDA(c, cudaStreamSynchronize(c->stream));
  for (size_t i = 0; i < c->prof.size(); ++i) {
    const ProfRec& r = c->prof[i];
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.e0, r.e1) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    c->prof_ms[r.kind] += ms;
    c->prof_bytes[r.kind] += r.bytes;
    c->prof_n[r.kind] += 1;
    float gap = 0.f;
    if (i + 1 < c->prof.size() &&
        cudaEventElapsedTime(&gap, r.e1, c->prof[i + 1].e0) == cudaSuccess && gap > 0.f)
      c->prof_gap_ms[r.kind] += gap;
    cudaGetLastError();
  }
  c->prof.clear();
  c->ev_used = 0;
  return SJ_OK;
}

sj_status sj_prof_reset(sj_ctx* c) {
  if (!c) return SJ_EINVAL;
  SJ_CUDA(c, cudaStreamSynchronize(c->stream));
  c->prof.clear();
  c->ev_used = 0;
  for (int k = 0; k < SJ_K_COUNT; ++k) {
    c->prof_ms[k] = 0;
    c->prof_gap_ms[k] = 0;
    c->prof_bytes[k] = 0;
    c->prof_n[k] = 0;
  }
  c->launches = 0;
  c->h2d_bytes = 0;
  c->d2h_bytes = 0;
  return SJ_OK;
}

sj_status sj_prof_read(sj_ctx* c, int kind, int64_t* launches, double* ms, double* bytes) {
  if (!c || kind < 0 || kind >= SJ_K_COUNT) return fail(c, SJ_EINVAL, "bad profiling kind");
  SJ_TRY(prof_collect(c));
  if (launches) *launches = c->prof_n[kind];
  if (ms) *ms = c->prof_ms[kind];
  if (bytes) *bytes = c->prof_bytes[kind];
  return SJ_OK;
}

sj_status sj_prof_gaps(sj_ctx* c, double* gap_ms) {
  if (!c || !gap_ms) return SJ_EINVAL;
  SJ_TRY(prof_collect(c));
  for (int k = 0; k < SJ_K_COUNT; ++k) gap_ms[k] = c->prof_gap_ms[k];
  return SJ_OK;
}

sj_status sj_graphs_enable(sj_ctx* c, int on) {
  if (!c) return SJ_EINVAL;
  c->graphs_on = on != 0;
  if (!c->graphs_on) {
    cudaStreamSynchronize(c->stream);
    for (auto& kv : c->graphs) drop_graph(kv.second);
    c->graphs.clear();
  }
  return SJ_OK;
}

sj_status sj_graph_stats(sj_ctx* c, int64_t* replays, int64_t* captures, int64_t* failures, char* why,
                         int len) {
  if (!c) return SJ_EINVAL;
  if (replays) *replays = c->graph_replays;
  if (captures) *captures = c->graph_captures;
  if (failures) *failures = c->graph_failures;
  if (why && len > 0) {
    strncpy(why, c->graph_why.c_str(), (size_t)len - 1);
    why[len - 1] = 0;
  }
  return SJ_OK;
}

sj_status sj_counters(sj_ctx* c, int64_t* launches, int64_t* h2d_bytes, int64_t* d2h_bytes) {
  if (!c) return SJ_EINVAL;
  if (launches) *launches = c->launches;
  if (h2d_bytes) *h2d_bytes = c->h2d_bytes;
  if (d2h_bytes) *d2h_bytes = c->d2h_bytes;
  return SJ_OK;
}

}  // extern "C"

// ======================================================================== cyclic query
namespace {

}  // namespace

extern "C" sj_status sj_triangles(sj_ctx* c, sj_rel edges, int nsub, const int32_t* cuts,
                                  int sieve_rounds, const sj_filter_params* params,
                                  uint64_t* counts, sj_tri_stats* stats) {
  if (!c || !edges || !cuts || !counts) return fail(c, SJ_EINVAL, "null argument");
  if (edges->ncols < 2 || edges->nrows < 0) return fail(c, SJ_EINVAL, "edges need 2 columns");
  if (nsub < 1 || nsub > 256) return fail(c, SJ_EINVAL, "nsub must be in 1..256");
  for (int i = 0; i < nsub; ++i)
    if (cuts[i + 1] <= cuts[i]) return fail(c, SJ_EINVAL, "cuts must increase");
  sj_filter_params fp = norm_params(params);
  fp.layout = SJ_REGBLOCKED32;
  SJ_TRY(check_params(c, fp));
  if (sieve_rounds < 0) sieve_rounds = 2;
  if (sieve_rounds > 8) return fail(c, SJ_EINVAL, "sieve_rounds must be <= 8");

  // ---- pruning: keep (a, b) with b among the sources and a among the targets
  const size_t p0 = c->prof.size();
  sj_rel cur = nullptr;
  const sj_rel_s* E = edges;
  int slot_in = -1;
  for (int r = 0; r < sieve_rounds; ++r) {
    sj_filter fs = nullptr, fd = nullptr;
    sj_status st = build_filter_nosync(c, E, 0, fp, slot_in, &fs);
    if (st == SJ_OK) st = build_filter_nosync(c, E, 1, fp, slot_in, &fd);
    sj_rel nx = nullptr;
    if (st == SJ_OK) {
      std::vector<TestSpec> t{{1, false, 0, 0, fs}, {0, false, 0, 0, fd}};
      st = sieve_step_timed(c, E, t, r, slot_in, &nx);
    }
    free_filter(c, fs);
    free_filter(c, fd);
    if (st != SJ_OK) {
      free_rel(c, cur);
      return st;
    }
    free_rel(c, cur);
    cur = nx;
    E = cur;
    slot_in = r;
  }
  sj_status st = sync_read(c);
  if (st != SJ_OK) {
    free_rel(c, cur);
    return st;
  }
  prof_resolve(c, p0);
  const int64_t ne = slot_in >= 0 ? (int64_t)c->h_misc[kMiscSteps + slot_in] : edges->nrows;
  if (cur) cur->nrows = ne;
  struct RelGuard {
    sj_ctx* c;
    sj_rel r;
    ~RelGuard() { free_rel(c, r); }
  } guard{c, cur};
  for (int i = 0; i < nsub; ++i) counts[i] = 0;
  if (stats) {
    memset(stats, 0, sizeof(*stats));
    stats->edges_in = edges->nrows;
    stats->edges_sieved = ne;
  }
  if (ne == 0) return SJ_OK;

  Temps tmp(c);
  Adjacency out{}, in{};
  SJ_TRY(build_adjacency(c, tmp, E->cols[0], ne, &out));
  SJ_TRY(build_adjacency(c, tmp, E->cols[1], ne, &in));
  // each adjacency's far endpoints in its own row order, so the enumeration
  // reads them contiguously instead of one random edge lookup per candidate
  int32_t* out_nbr = tmp.get<int32_t>((size_t)ne, &st);
  int32_t* in_nbr = tmp.get<int32_t>((size_t)ne, &st);
  if (st != SJ_OK) return fail(c, st, "neighbour array allocation failed");
  {
    Launch L(c, SJ_K_HT_BUILD, 24.0 * (double)ne);
    launch_gather_i32(E->cols[1], out.rows, ne, out_nbr, c->num_sms, c->stream);
    launch_gather_i32(E->cols[0], in.rows, ne, in_nbr, c->num_sms, c->stream);
  }
  SJ_TRY(check_launch(c, "k_gather_i32"));

  // closing-pair filter, rebuilt from the pruned edges (Sec. 2.3)
  uint64_t nb = ((uint64_t)fp.bits_per_key * (uint64_t)ne + 255) / 256;
  if (nb < 1) nb = 1;
  uint8_t* fmem = tmp.get<uint8_t>(kAlign + nb * 32, &st);
  if (!fmem) return fail(c, st, "pair filter allocation failed");
  SJ_CUDA(c, cudaMemsetAsync(fmem, 0, kAlign + nb * 32, c->stream));
  PairFilterBuildArgs pf{E->cols[0], E->cols[1], ne, reinterpret_cast<uint64_t*>(fmem),
                         reinterpret_cast<uint32_t*>(fmem + kAlign), nb, fp.k, fp.seed};
  {
    Launch L(c, SJ_K_BLOOM_BUILD, (8.0 + fp.bits_per_key / 8.0) * (double)ne);
    launch_pair_filter_build(pf, c->num_sms, c->stream);
  }
  SJ_TRY(check_launch(c, "k_pair_filter_build"));

  // exact pair set
  Table2 ps;
  SJ_TRY(make_table(c, tmp, ne, &ps));
  PairSetArgs pa{E->cols[0], E->cols[1], ne, ps.t, status_ptr(c)};
  {
    Launch L(c, SJ_K_HT_BUILD, 16.0 * (double)ne);
    launch_pairset_insert(pa, c->num_sms, c->stream);
  }
  SJ_TRY(check_launch(c, "k_pairset_insert"));

  int32_t* dcuts = tmp.get<int32_t>((size_t)nsub + 1, &st);
  unsigned long long* dcnt = tmp.get<unsigned long long>((size_t)nsub + 3, &st);
  if (st != SJ_OK) return fail(c, st, "allocation failed");
  SJ_CUDA(c, cudaMemcpyAsync(dcuts, cuts, ((size_t)nsub + 1) * 4, cudaMemcpyHostToDevice, c->stream));
  c->h2d_bytes += ((int64_t)nsub + 1) * 4;
  SJ_CUDA(c, cudaMemsetAsync(dcnt, 0, ((size_t)nsub + 3) * 8, c->stream));
  TriangleArgs ta;
  ta.src = E->cols[0];
  ta.dst = E->cols[1];
  ta.ne = ne;
  ta.out = out;
  ta.in = in;
  ta.out_nbr = out_nbr;
  ta.in_nbr = in_nbr;
  ta.pf.words = pf.words;
  ta.pf.hdr = pf.hdr;
  ta.pf.k = fp.k;
  ta.pf.layout = SJ_REGBLOCKED32;
  ta.pf.seed = fp.seed;
  ta.pairs = ps.t;
  ta.cuts = dcuts;
  ta.nsub = nsub;
  ta.counts = dcnt;
  ta.stats = dcnt + nsub;
  ta.work = dcnt + nsub + 2;
  {
    Launch L(c, SJ_K_OTHER, 8.0 * (double)ne);
    launch_triangles(ta, c->num_sms, c->stream);
  }
  SJ_TRY(check_launch(c, "k_triangles"));
  std::vector<unsigned long long> h((size_t)nsub + 2);
  SJ_CUDA(c, cudaMemcpyAsync(h.data(), dcnt, ((size_t)nsub + 2) * 8, cudaMemcpyDeviceToHost, c->stream));
  c->d2h_bytes += ((int64_t)nsub + 2) * 8;
  SJ_TRY(sync_read(c));
  uint64_t tot = 0;
  for (int i = 0; i < nsub; ++i) {
    counts[i] = h[i];
    tot += h[i];
  }
  if (stats) {
    stats->candidates = h[nsub];
    stats->filter_passed = h[nsub + 1];
    stats->triangles = tot;
  }
  return SJ_OK;
}

namespace {

// Pruning phase and device-sized join enqueued back to back.  Each multimap
// level's relation is final as soon as its last sieve step is enqueued: its
// build starts then, on the side stream, overlapping the remaining sieve
// steps.  With finish = false nothing waits (graph capture).
sj_status run_device_sized(sj_ctx* c, const sj_path* path, const sj_sieve_opts* opts, int nrefs,
                           const sj_colref* refs, const std::vector<uint64_t>& caps, sj_rel* sieved,
                           sj_result* result, std::vector<uint64_t>* T, bool finish) {
  const std::vector<LevelPlan> plan = join_order(path);
  const int nlev = (int)plan.size() - 1;
  std::vector<Adjacency> built(std::max(nlev, 0));
  Temps bt(c);  // arena memory: lives until the arena scope ends
  sj_status st = SJ_OK;
  uint32_t* smallb = bt.get<uint32_t>(2 * SJ_MAX_REL, &st);
  if (st != SJ_OK) return fail(c, st, "allocation failed");
  StagedPath sp;
  SJ_TRY(stage_mapped(c, path, opts, bt, &sp));
  path = &sp.path;
  std::vector<int> level_of(path->nrel, -1);
  for (int L = 0; L < nlev; ++L) level_of[plan[L].rel] = L;
  SJ_TRY(ensure_side(c, nlev));
  // each level's multimap is built on the side stream as soon as the pruning
  // phase is done with its relation, overlapping the remaining sieve steps
  // (those launch at a higher priority, see launch_sieve_chunk)
  std::vector<int> rel_slot(path->nrel, -1);
  const FinalHook hook = [&](int i, const sj_rel_s* r, int slot) -> sj_status {
    rel_slot[i] = slot;
    const int L = level_of[i];
    if (L < 0) return SJ_OK;
    SJ_CUDA(c, cudaEventRecord(c->ev_ready, c->stream));
    OnSide side(c);
    SJ_CUDA(c, cudaStreamWaitEvent(c->stream, c->ev_ready, 0));
    SJ_TRY(build_adjacency_dev(c, bt, r->cols[plan[L].rel_col], r->d_n, r->nrows, rel_cap(r),
                               smallb + 2 * L, smallb + 2 * L + 1, &built[L], r->d_n ? slot : -1));
    SJ_CUDA(c, cudaEventRecord(c->ev_built[L], c->stream));
    return SJ_OK;
  };
  st = sieve_path_impl(c, path, opts, sieved, nullptr, false, &hook, sp.ready);
  if (st == SJ_OK) st = join_async(c, path, sieved, nrefs, refs, caps, result, T, &built, finish, &rel_slot);
  if (c->side && !c->capturing) cudaStreamSynchronize(c->side);  // before the arena is released
  if (c->copy && !c->capturing) cudaStreamSynchronize(c->copy);  // idem (a call that failed midway)
  return st;
}

// Capture the device-sized query as a CUDA graph for later calls of the same
// shape.  Runs in its own arena scope, after a plain run sized the arena.
void capture_graph(sj_ctx* c, uint64_t key, const sj_path* path, const sj_sieve_opts* opts, int nrefs,
                   const sj_colref* refs, const std::vector<uint64_t>& caps) {
  auto& G = c->graphs[key];
  drop_graph(G);
  G.failed = true;
  const int64_t launches0 = c->launches, d2h0 = c->d2h_bytes, h2d0 = c->h2d_bytes;
  const size_t prof0 = c->prof.size(), ev0 = c->ev_used;
  arena_begin(c);
  const uint64_t gen = c->arena_gen;
  sj_rel sieved[SJ_MAX_REL] = {};
  cudaGraph_t graph = nullptr;
  // the capture stream has the device's highest priority and the side stream
  // its lowest, and the graph keeps those per node: the critical path's
  // kernels (pruning, probes) get SMs before the side stream's table builds
  int prio_least = 0, prio_greatest = 0;
  if (cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest) != cudaSuccess) {
    cudaGetLastError();
    prio_least = prio_greatest = 0;
  }
  if (!c->cap_stream &&
      cudaStreamCreateWithPriority(&c->cap_stream, cudaStreamNonBlocking, prio_greatest) != cudaSuccess) {
    cudaGetLastError();
    c->cap_stream = nullptr;
  }
  // the user's stream (possibly the legacy default stream, which cannot be
  // captured) is set aside while the capture runs on the private stream
  const bool swapped = c->cap_stream != nullptr;
  if (swapped) std::swap(c->stream, c->cap_stream);
  if (swapped && cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
    c->capturing = true;
    // state words, group words and tickets start from zero in every replay
    sj_status st = SJ_OK;
    if (c->scratch && cudaMemsetAsync(c->scratch, 0, c->scratch_bytes, c->stream) != cudaSuccess)
      st = SJ_ECUDA;
    if (st == SJ_OK && c->scratch2 &&
        cudaMemsetAsync(c->scratch2, 0, c->scratch2_bytes, c->stream) != cudaSuccess)
      st = SJ_ECUDA;
    sj_result dummy;
    if (st == SJ_OK) st = run_device_sized(c, path, opts, nrefs, refs, caps, sieved, &dummy, nullptr, false);
    c->capturing = false;
    if (st != SJ_OK) note_graph_failure(c, "enqueue: " + c->err);
    const cudaError_t e = cudaStreamEndCapture(c->stream, &graph);
    if (e != cudaSuccess) note_graph_failure(c, std::string("end capture: ") + cudaGetErrorString(e));
    cudaError_t ei = cudaSuccess;
    if (st == SJ_OK && e == cudaSuccess && graph &&
        (ei = cudaGraphInstantiate(&G.exec, graph, cudaGraphInstantiateFlagUseNodePriority)) == cudaSuccess) {
      G.failed = false;
      G.caps = caps;
      G.nkernels = c->launches - launches0;
      G.h2d_bytes = c->h2d_bytes - h2d0;
    } else {
      if (ei != cudaSuccess) note_graph_failure(c, std::string("instantiate: ") + cudaGetErrorString(ei));
      G.exec = nullptr;
    }
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
  } else {
    note_graph_failure(c, "begin capture failed");
    cudaGetLastError();
  }
  // the launch events recorded inside the graph now belong to it
  G.prof.assign(c->prof.begin() + prof0, c->prof.end());
  c->prof.resize(prof0);
  c->ev_pool.erase(c->ev_pool.begin() + ev0, c->ev_pool.begin() + c->ev_used);
  c->ev_used = ev0;
  if (swapped) std::swap(c->stream, c->cap_stream);
  for (int i = 0; i < path->nrel; ++i) free_rel(c, sieved[i]);
  arena_end(c);
  if (c->arena_gen != gen && G.exec) {  // the capture outgrew the arena
    drop_graph(G);
    G.failed = true;
    note_graph_failure(c, "arena grew during capture");
  }
  // a capture that failed because the arena was too small is retried by the
  // next call (the arena has grown since); other failures are final
  G.gen = (G.failed && c->arena_gen != gen) ? gen : c->arena_gen;
  if (G.failed) c->graph_failures++;
  else c->graph_captures++;
  c->launches = launches0;
  c->d2h_bytes = d2h0;
  c->h2d_bytes = h2d0;
}

}  // namespace

extern "C" sj_status sj_sieve_join(sj_ctx* c, const sj_path* path, const sj_sieve_opts* opts,
                                   int mode, int nrefs, const sj_colref* refs, sj_result* result,
                                   sj_sieve_stats* stats) {
  if (!c || !path || !result) return fail(c, SJ_EINVAL, "null argument");
  if (path->nrel < 1 || path->nrel > SJ_MAX_REL || !path->rels) return fail(c, SJ_EINVAL, "bad path");
  for (int i = 0; i < path->nrel; ++i)
    if (!path->rels[i] || path->rels[i]->nrows < 0) return fail(c, SJ_EINVAL, "bad relation handle");
  sj_rel sieved[SJ_MAX_REL] = {};
  const uint64_t sig = path_signature(path, opts, mode, nrefs, refs);
  auto it = c->plan_caps.find(sig);
  const bool device_sized = mode == SJ_COUNT_SUM && path->nrel >= 2 && !stats && it != c->plan_caps.end();
  std::vector<uint64_t> T;
  sj_status st = SJ_OK;
  bool exact = !device_sized;
  if (device_sized) {
    // sizes stay on the device: one synchronisation for the whole query
    std::vector<uint64_t> caps;
    for (uint64_t t : it->second) caps.push_back(2 * t + 4096);
    const uint64_t gkey = mix_in(sig, c->prof_on ? (uint64_t)c->prof_mask : 0ull);
    auto g = c->graphs.find(gkey);
    const bool replay = g != c->graphs.end() && g->second.exec && g->second.caps == caps &&
                        g->second.gen == c->arena_gen;
    if (replay) {
      // the whole query is one graph launch and one synchronisation
      if (cudaGraphLaunch(g->second.exec, c->stream) != cudaSuccess ||
          cudaStreamSynchronize(c->stream) != cudaSuccess) {
        cudaGetLastError();
        return fail(c, SJ_ECUDA, "graph replay failed");
      }
      c->launches += g->second.nkernels;
      c->d2h_bytes += kMiscWords * sizeof(uint64_t);
      c->h2d_bytes += g->second.h2d_bytes;
      c->graph_replays++;
      if (c->prof_on) prof_replay(c, g->second);
      st = read_status(c);
      if (st == SJ_OK) st = device_sized_result(c, (int)caps.size(), result, &T);
      if (st == kRetry) {
        T.clear();
        exact = true;  // an intermediate outgrew its buffer: exact rerun
      } else if (st != SJ_OK) {
        return st;
      }
    } else {
      arena_begin(c);
      const size_t p0 = c->prof.size();
      st = run_device_sized(c, path, opts, nrefs, refs, caps, sieved, result, &T, true);
      if (st == SJ_OK) prof_resolve(c, p0);
      if (st == kRetry) {
        // an intermediate outgrew its buffer: take the sizes to the host and
        // rerun the enumeration exactly
        T.clear();
        st = SJ_OK;
        prof_resolve(c, p0);
        for (int i = 0; i < path->nrel && st == SJ_OK; ++i) {
          if (sieved[i] && sieved[i]->d_n && sieved[i]->nrows < 0) {
            uint64_t v = 0;
            if (cudaMemcpyAsync(&v, sieved[i]->d_n, 8, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
                cudaStreamSynchronize(c->stream) != cudaSuccess)
              st = fail(c, SJ_ECUDA, "row count readback failed");
            sieved[i]->nrows = (int64_t)v;
          }
        }
        if (st == SJ_OK) st = join_impl(c, path, sieved, mode, nrefs, refs, result, &T);
      }
      for (int i = 0; i < path->nrel; ++i) {
        free_rel(c, sieved[i]);
        sieved[i] = nullptr;
      }
      arena_end(c);
      // a shape is captured once it has run device-sized before: one-off
      // shapes (common in serving) do not pay for a capture
      const int runs = ++c->plan_runs[sig];
      const bool capture = st == SJ_OK && runs >= 2 && c->graphs_on &&
                           (g == c->graphs.end() || !g->second.failed || g->second.gen != c->arena_gen);
      if (st == SJ_OK) {
        if (c->plan_caps.size() > 4096) {
          c->plan_caps.clear();
          c->plan_runs.clear();
        }
        c->plan_caps[sig] = T;
      }
      if (capture) {
        std::vector<uint64_t> next;
        for (uint64_t t : T) next.push_back(2 * t + 4096);
        if (c->graphs.size() >= 64) {
          for (auto& kv : c->graphs) drop_graph(kv.second);
          c->graphs.clear();
        }
        capture_graph(c, gkey, path, opts, nrefs, refs, next);
      }
      return st;
    }
  }
  if (exact) {
    arena_begin(c);
    {
      Temps stage_mem(c);
      StagedPath sp;
      st = stage_mapped(c, path, opts, stage_mem, &sp);
      if (st == SJ_OK) st = sieve_path_impl(c, &sp.path, opts, sieved, stats, true, nullptr, sp.ready);
      if (st == SJ_OK) st = join_impl(c, &sp.path, sieved, mode, nrefs, refs, result, &T);
      for (int i = 0; i < path->nrel; ++i) free_rel(c, sieved[i]);
      if (c->copy) cudaStreamSynchronize(c->copy);  // before the arena is released
    }
    arena_end(c);
  }
  if (st == SJ_OK && mode == SJ_COUNT_SUM && path->nrel >= 2) {
    if (c->plan_caps.size() > 4096) {
      c->plan_caps.clear();
      c->plan_runs.clear();
    }
    c->plan_caps[sig] = T;
  }
  return st;
}

extern "C" sj_status sj_selftest_wait_timeout(sj_ctx* c) {
  if (!c) return SJ_EINVAL;
  Temps tmp(c);
  sj_status st = SJ_OK;
  uint32_t* flag = tmp.get<uint32_t>(1, &st);
  if (st != SJ_OK) return fail(c, st, "self-test allocation failed");
  SJ_CUDA(c, cudaMemsetAsync(flag, 0, 4, c->stream));
  {
    Launch L(c, SJ_K_OTHER, 0.0);
    launch_wait_flag(flag, status_ptr(c), c->stream);
  }
  SJ_TRY(check_launch(c, "k_wait_flag"));
  return sync_read(c);
}
