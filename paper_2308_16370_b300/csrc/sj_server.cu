// Query server: continuous batching of sieved joins over resident relations,
// with a device-side cache of the reusable leaf filters (Sec. 2.3).
//
// Host-only runtime built on the public C ABI.  Each of the `nslots` worker
// threads owns one context and one CUDA stream; a FIFO queue feeds them, and
// a query is admitted when a worker is free and its memory estimate fits in
// the budget next to the queries already running (a query larger than the
// whole budget runs alone).  Cached filters are built once, on the stream of
// the worker that first needs them; other workers order their use after the
// build with an event, so no worker waits on the host for another's GPU work.
// In batch mode a free worker takes up to `batch` queued queries that fit the
// budget together and prunes them with one sj_sieve_path_batch call (two
// launches per schedule level for the whole group), then runs each query's
// join over its pruned relations (sj_join with them as inputs).  A query over
// more than batch_max_rows rows runs alone: a batch moves in lock step, so
// one large query would hold back every small one in it.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <tuple>
#include <vector>

#include "sievejoin.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Pending {
  sj_query q;
  uint64_t ticket;
  uint64_t est_bytes;
  uint64_t rows;  // rows of its relations in all
  double submit_ms;
};

using CacheKey = std::tuple<int32_t, int32_t, int32_t, int32_t, int32_t>;  // rel, col, pcol, lo, hi

struct CacheEntry {
  sj_filter f = nullptr;
  cudaEvent_t ready = nullptr;
  int builder = -1;     // worker whose context owns the filter
  bool building = true;
  bool failed = false;
};

}  // namespace

struct sj_server {
  sj_server_opts opts{};
  Clock::time_point t0;
  std::vector<sj_rel> rels;
  std::vector<uint64_t> rel_bytes;
  std::vector<int64_t> rel_rows;
  std::vector<int> rel_ncols;
  std::vector<sj_ctx*> ctxs;
  std::vector<cudaStream_t> streams;
  std::vector<std::thread> threads;

  std::mutex mu;
  std::condition_variable cv_work, cv_done, cv_cache;
  std::deque<Pending> queue;
  std::vector<sj_completion> done;
  uint64_t next_ticket = 1;
  uint64_t inflight_bytes = 0;
  int running = 0;
  bool stopping = false;
  sj_server_stats st{};
  std::map<CacheKey, CacheEntry> cache;

  double now_ms() const {
    return std::chrono::duration<double, std::milli>(Clock::now() - t0).count();
  }
};

namespace {

// Leaves of the join tree rooted at `root`: degree-1 positions other than the root.
std::vector<int> leaves_of(const sj_query& q, int root) {
  std::vector<int> deg(q.nrel, 0);
  for (int e = 0; e < q.nrel - 1; ++e) {
    deg[q.edges[e].rel_a]++;
    deg[q.edges[e].rel_b]++;
  }
  std::vector<int> out;
  if (q.nrel < 2) return out;
  for (int v = 0; v < q.nrel; ++v)
    if (deg[v] == 1 && v != root) out.push_back(v);
  return out;
}

// Column of position v on its only edge.
int leaf_col(const sj_query& q, int v) {
  for (int e = 0; e < q.nrel - 1; ++e) {
    if (q.edges[e].rel_a == v) return q.edges[e].col_a;
    if (q.edges[e].rel_b == v) return q.edges[e].col_b;
  }
  return 0;
}

// The cached leaf filter for (relation, column, predicate), built on this
// worker's stream if absent.  Returns null on failure.
sj_filter cached_filter(sj_server* s, int w, int rel_id, int col, const sj_pred& pred, bool* hit) {
  const CacheKey key{rel_id, col, pred.col, pred.col >= 0 ? pred.lo : 0, pred.col >= 0 ? pred.hi : 0};
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->cache.find(key);
  if (it != s->cache.end()) {
    // another worker may still be enqueueing the build: wait (bounded) for the event
    for (int i = 0; i < 60000 && it->second.building; ++i)
      s->cv_cache.wait_for(lk, std::chrono::milliseconds(1));
    if (it->second.building || it->second.failed) return nullptr;
    *hit = true;
    s->st.cache_hits++;
    cudaEvent_t ev = it->second.ready;
    sj_filter f = it->second.f;
    lk.unlock();
    cudaStreamWaitEvent(s->streams[w], ev, 0);
    return f;
  }
  CacheEntry& ent = s->cache[key];
  s->st.cache_misses++;
  lk.unlock();
  sj_filter f = nullptr;
  const sj_pred* pp = pred.col >= 0 ? &pred : nullptr;
  cudaEvent_t ev = nullptr;
  bool ok = sj_build_filter(s->ctxs[w], s->rels[rel_id], col, pp, &s->opts.filter, &f) == SJ_OK &&
            cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess &&
            cudaEventRecord(ev, s->streams[w]) == cudaSuccess;
  lk.lock();
  ent.f = f;
  ent.ready = ev;
  ent.builder = w;
  ent.building = false;
  ent.failed = !ok;
  s->st.cached_filters += ok ? 1 : 0;
  s->cv_cache.notify_all();
  *hit = false;
  return ok ? f : nullptr;
}

void run_query(sj_server* s, int w, const Pending& p, sj_completion* c) {
  const sj_query& q = p.q;
  sj_ctx* ctx = s->ctxs[w];
  sj_rel rels[SJ_MAX_REL];
  for (int i = 0; i < q.nrel; ++i) rels[i] = s->rels[q.rel[i]];
  sj_path path;
  path.nrel = q.nrel;
  path.root = q.root;
  path.rels = rels;
  path.edges = q.edges;
  path.preds = q.preds;
  const int root = q.root < 0 ? q.nrel - 1 : q.root;

  sj_filter leaf[SJ_MAX_REL] = {};
  c->cache_hits = 0;
  if (s->opts.cache_filters) {
    for (int v : leaves_of(q, root)) {
      bool hit = false;
      leaf[v] = cached_filter(s, w, q.rel[v], leaf_col(q, v), q.preds[v], &hit);
      c->cache_hits += hit ? 1 : 0;
    }
  }
  sj_sieve_opts o{};
  o.passes = s->opts.passes;
  o.filter = s->opts.filter;
  o.leaf_filters = s->opts.cache_filters ? leaf : nullptr;
  sj_result res{};
  const sj_status st = sj_sieve_join(ctx, &path, &o, SJ_COUNT_SUM, q.nterms, q.terms, &res, nullptr);
  c->status = st;
  c->count = res.count;
  c->sum = res.sum;
}

// Hand a finished query to the pollers.
void deliver(sj_server* s, sj_completion c) {
  c.done_ms = s->now_ms();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->done.push_back(c);
    s->st.completed++;
    if (c.status != SJ_OK) s->st.failed++;
  }
  s->cv_done.notify_all();
}

// Batch mode: prune the group in one call, then join each query over its
// pruned relations.  If the batched call fails (out of memory, say), every
// query of the group runs alone instead.  Each query is delivered as soon as
// its join is done.
void run_group(sj_server* s, int w, const std::vector<Pending>& ps, std::vector<sj_completion>* cs) {
  const int nq = (int)ps.size();
  sj_ctx* ctx = s->ctxs[w];
  std::vector<sj_rel> rels((size_t)nq * SJ_MAX_REL, nullptr);
  std::vector<sj_filter> leaf((size_t)nq * SJ_MAX_REL, nullptr);
  std::vector<sj_path> paths(nq);
  std::vector<sj_sieve_opts> opts(nq);
  for (int k = 0; k < nq; ++k) {
    const sj_query& q = ps[k].q;
    sj_rel* r = &rels[(size_t)k * SJ_MAX_REL];
    for (int i = 0; i < q.nrel; ++i) r[i] = s->rels[q.rel[i]];
    paths[k].nrel = q.nrel;
    paths[k].root = q.root;
    paths[k].rels = r;
    paths[k].edges = q.edges;
    paths[k].preds = q.preds;
    (*cs)[k].cache_hits = 0;
    sj_filter* lf = &leaf[(size_t)k * SJ_MAX_REL];
    if (s->opts.cache_filters) {
      const int root = q.root < 0 ? q.nrel - 1 : q.root;
      for (int v : leaves_of(q, root)) {
        bool hit = false;
        lf[v] = cached_filter(s, w, q.rel[v], leaf_col(q, v), q.preds[v], &hit);
        (*cs)[k].cache_hits += hit ? 1 : 0;
      }
    }
    opts[k] = sj_sieve_opts{};
    opts[k].passes = s->opts.passes;
    opts[k].filter = s->opts.filter;
    opts[k].leaf_filters = s->opts.cache_filters ? lf : nullptr;
  }
  std::vector<sj_rel> sieved((size_t)nq * SJ_MAX_REL, nullptr);
  if (sj_sieve_path_batch(ctx, nq, paths.data(), opts.data(), sieved.data(), nullptr) != SJ_OK) {
    for (int k = 0; k < nq; ++k) {
      run_query(s, w, ps[k], &(*cs)[k]);
      deliver(s, (*cs)[k]);
    }
    return;
  }
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->st.batches++;
    if (nq > s->st.peak_batch) s->st.peak_batch = nq;
  }
  for (int k = 0; k < nq; ++k) {
    const sj_query& q = ps[k].q;
    sj_rel* in = &sieved[(size_t)k * SJ_MAX_REL];
    sj_result res{};
    const sj_status st = sj_join(ctx, &paths[k], in, SJ_COUNT_SUM, q.nterms, q.terms, &res);
    (*cs)[k].status = st;
    (*cs)[k].count = res.count;
    (*cs)[k].sum = res.sum;
    for (int i = 0; i < q.nrel; ++i) sj_free_rel(ctx, in[i]);
    deliver(s, (*cs)[k]);
  }
}

void worker(sj_server* s, int w) {
  cudaSetDevice(s->opts.device);
  const int batch = s->opts.batch > 1 ? s->opts.batch : 1;
  while (true) {
    std::vector<Pending> ps;
    uint64_t bytes = 0;
    bool grouped = false;  // pruned by one batched call (possibly a group of one)
    {
      std::unique_lock<std::mutex> lk(s->mu);
      while (true) {
        if (!s->queue.empty()) {
          const uint64_t need = s->queue.front().est_bytes;
          if (s->running == 0 || s->inflight_bytes + need <= s->opts.hbm_budget) break;
        } else if (s->stopping) {
          return;
        }
        s->cv_work.wait_for(lk, std::chrono::milliseconds(50));
      }
      // the head of the queue; in batch mode, unless it is a large query,
      // then the small queries behind it (within a window of the queue, in
      // arrival order) that fit the budget next to it
      auto small = [&](const Pending& x) {
        return s->opts.batch_max_rows == 0 || x.rows <= s->opts.batch_max_rows;
      };
      ps.push_back(s->queue.front());
      s->queue.pop_front();
      bytes += ps[0].est_bytes;
      grouped = batch > 1 && small(ps[0]);
      if (grouped) {
        const size_t window = 4 * (size_t)batch;
        for (size_t i = 0; i < s->queue.size() && i < window && (int)ps.size() < batch;) {
          const Pending& x = s->queue[i];
          if (!small(x)) {
            ++i;
            continue;
          }
          if (s->inflight_bytes + bytes + x.est_bytes > s->opts.hbm_budget) break;
          bytes += x.est_bytes;
          ps.push_back(x);
          s->queue.erase(s->queue.begin() + (long)i);
        }
      }
      s->inflight_bytes += bytes;
      s->running += (int)ps.size();
      if (s->inflight_bytes > s->st.peak_inflight_bytes) s->st.peak_inflight_bytes = s->inflight_bytes;
      if (s->running > s->st.peak_concurrency) s->st.peak_concurrency = s->running;
    }
    std::vector<sj_completion> cs(ps.size());
    const double start = s->now_ms();
    for (size_t k = 0; k < ps.size(); ++k) {
      cs[k] = sj_completion{};
      cs[k].ticket = ps[k].ticket;
      cs[k].submit_ms = ps[k].submit_ms;
      cs[k].start_ms = start;
    }
    if (grouped) {
      run_group(s, w, ps, &cs);
    } else {
      run_query(s, w, ps[0], &cs[0]);
      deliver(s, cs[0]);
    }
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->inflight_bytes -= bytes;
      s->running -= (int)ps.size();
    }
    s->cv_work.notify_all();
  }
}

}  // namespace

extern "C" {

sj_status sj_server_create(sj_server** out, const sj_server_opts* opts) {
  if (!out || !opts) return SJ_EINVAL;
  sj_server* s = new sj_server();
  s->opts = *opts;
  if (s->opts.nslots <= 0) s->opts.nslots = 4;
  if (s->opts.nslots > 64) s->opts.nslots = 64;
  if (s->opts.batch > 1024) s->opts.batch = 1024;
  s->t0 = Clock::now();
  if (cudaSetDevice(s->opts.device) != cudaSuccess) {
    delete s;
    return SJ_ECUDA;
  }
  if (s->opts.hbm_budget == 0) {
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    s->opts.hbm_budget = fr / 2;
  }
  for (int w = 0; w < s->opts.nslots; ++w) {
    cudaStream_t st;
    sj_ctx* c = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
        sj_create(&c, s->opts.device, st, nullptr, nullptr, nullptr) != SJ_OK) {
      for (size_t i = 0; i < s->ctxs.size(); ++i) {
        sj_destroy(s->ctxs[i]);
        cudaStreamDestroy(s->streams[i]);
      }
      delete s;
      return SJ_ECUDA;
    }
    // a serving stream is mostly distinct query shapes: a graph capture would
    // add a query's worth of host time to one request and rarely be replayed
    sj_graphs_enable(c, 0);
    s->streams.push_back(st);
    s->ctxs.push_back(c);
  }
  for (int w = 0; w < s->opts.nslots; ++w) s->threads.emplace_back(worker, s, w);
  *out = s;
  return SJ_OK;
}

sj_status sj_server_add_relation(sj_server* s, int ncols, const int32_t* const* dev_cols,
                                 int64_t nrows, int32_t* rel_id) {
  if (!s || !rel_id) return SJ_EINVAL;
  sj_rel r = nullptr;
  const sj_status st = sj_load_relation(s->ctxs[0], ncols, dev_cols, nrows, SJ_DEVICE_BORROW, &r);
  if (st != SJ_OK) return st;
  std::lock_guard<std::mutex> lk(s->mu);
  *rel_id = (int32_t)s->rels.size();
  s->rels.push_back(r);
  s->rel_bytes.push_back((uint64_t)nrows * 4 * (uint64_t)ncols);
  s->rel_rows.push_back(nrows);
  s->rel_ncols.push_back(ncols);
  return SJ_OK;
}

sj_status sj_server_submit(sj_server* s, const sj_query* q, uint64_t* ticket) {
  if (!s || !q || q->nrel < 1 || q->nrel > SJ_MAX_REL || q->nterms < 0 || q->nterms > SJ_MAX_TERMS)
    return SJ_EINVAL;
  Pending p;
  p.q = *q;
  p.rows = 0;
  uint64_t bytes = 64ull << 20;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    for (int i = 0; i < q->nrel; ++i) {
      if (q->rel[i] < 0 || q->rel[i] >= (int32_t)s->rels.size()) return SJ_EINVAL;
      bytes += 3 * s->rel_bytes[q->rel[i]];  // sieved copies, filters and tables
      p.rows += (uint64_t)s->rel_rows[q->rel[i]];
    }
    for (int e = 0; e < q->nrel - 1; ++e) {
      const sj_edge& E = q->edges[e];
      if (E.rel_a < 0 || E.rel_a >= q->nrel || E.rel_b < 0 || E.rel_b >= q->nrel ||
          E.col_a < 0 || E.col_a >= s->rel_ncols[q->rel[E.rel_a]] || E.col_b < 0 ||
          E.col_b >= s->rel_ncols[q->rel[E.rel_b]])
        return SJ_EINVAL;
    }
    p.est_bytes = bytes;
    p.ticket = s->next_ticket++;
    p.submit_ms = s->now_ms();
    s->queue.push_back(p);
    s->st.submitted++;
    if (ticket) *ticket = p.ticket;
  }
  s->cv_work.notify_one();
  return SJ_OK;
}

sj_status sj_server_poll(sj_server* s, sj_completion* out, int max, int* n, int wait_ms) {
  if (!s || !n || (max > 0 && !out)) return SJ_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  if (s->done.empty() && wait_ms > 0)
    s->cv_done.wait_for(lk, std::chrono::milliseconds(wait_ms), [&] { return !s->done.empty(); });
  const int k = std::min<int>(max, (int)s->done.size());
  for (int i = 0; i < k; ++i) out[i] = s->done[i];
  s->done.erase(s->done.begin(), s->done.begin() + k);
  *n = k;
  return SJ_OK;
}

sj_status sj_server_stats_get(sj_server* s, sj_server_stats* stats) {
  if (!s || !stats) return SJ_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  *stats = s->st;
  return SJ_OK;
}

sj_status sj_server_destroy(sj_server* s) {
  if (!s) return SJ_EINVAL;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stopping = true;
  }
  s->cv_work.notify_all();
  for (auto& t : s->threads) t.join();
  for (auto st : s->streams) cudaStreamSynchronize(st);
  for (auto& kv : s->cache) {
    if (kv.second.f) sj_free_filter(s->ctxs[kv.second.builder], kv.second.f);
    if (kv.second.ready) cudaEventDestroy(kv.second.ready);
  }
  for (sj_rel r : s->rels) sj_free_rel(s->ctxs[0], r);
  for (size_t i = 0; i < s->ctxs.size(); ++i) {
    sj_destroy(s->ctxs[i]);
    cudaStreamDestroy(s->streams[i]);
  }
  delete s;
  return SJ_OK;
}

}  // extern "C"
