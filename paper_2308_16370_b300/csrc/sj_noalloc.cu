// Allocation-free variant of one sieve step.
//
// Some callers cannot call cudaMalloc (or any allocating routine) at the point
// where they want to sieve: code running inside a custom allocator or memory
// manager, or a runtime that hands out only pre-reserved buffers and forbids
// allocations on its hot path.  sj_sieve_noalloc serves them: the caller
// passes inputs and outputs, and the only scratch the step needs (the chunk
// ticket, the look-back chunk states and a filter header) lives in the
// fixed-size file-scope device array below, which every GPU that loads this
// library holds until the process exits.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "sievejoin.h"
#include "sj_kernels.cuh"

namespace {

// Largest relation one call accepts, and the scratch it implies: the chunked
// sieve takes at most kCkMaxRows rows per chunk, or one chunk per CTA slot of
// the GPU when that is more rows (at most 8192 chunks up to 2^27 rows on any
// GPU with fewer than 1638 SMs; checked per call).
constexpr int64_t kMaxRows = SJ_NOALLOC_MAX_ROWS;
constexpr int64_t kMaxChunks = (kMaxRows + sj::kCkMaxRows - 1) / sj::kCkMaxRows;
constexpr int64_t kMaxGroups = (kMaxChunks + 31) / 32;
constexpr size_t kOffCounter = 0;    // uint32 chunk ticket
constexpr size_t kOffStatus = 64;    // uint32 status word (when the caller passes none)
constexpr size_t kOffHdr = 128;      // uint64 nblocks, uint64 rows inserted
constexpr size_t kOffFin = 192;      // uint32 finished-CTA counter of the group prefix
constexpr size_t kOffGroups = 256;   // one word per 32 chunks (arrivals, kept rows)
constexpr size_t kOffStates = kOffGroups + 8 * kMaxGroups;  // one packed state word per chunk
constexpr size_t kScratchBytes = kOffStates + 8 * kMaxChunks;  // 66 KiB + 256 B

static __device__ __align__(256) unsigned char g_sieve_scratch[kScratchBytes];

// Device-side set-up of one call: clear what must start at zero and write the
// filter header the sieve kernel reads.  Device code names the array directly.
__global__ void k_noalloc_prepare(uint64_t nblocks, uint32_t nchunks, int clear_status) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) {
    *reinterpret_cast<uint32_t*>(g_sieve_scratch + kOffCounter) = 0u;
    *reinterpret_cast<uint32_t*>(g_sieve_scratch + kOffFin) = 0u;
    if (clear_status) *reinterpret_cast<uint32_t*>(g_sieve_scratch + kOffStatus) = 0u;
    uint64_t* hdr = reinterpret_cast<uint64_t*>(g_sieve_scratch + kOffHdr);
    hdr[0] = nblocks;
    hdr[1] = 0;
  }
  uint64_t* states = reinterpret_cast<uint64_t*>(g_sieve_scratch + kOffStates);
  for (uint32_t t = i; t < nchunks; t += gridDim.x * blockDim.x) states[t] = 0ull;
  uint64_t* groups = reinterpret_cast<uint64_t*>(g_sieve_scratch + kOffGroups);
  for (uint32_t t = i; t < (nchunks + 31) / 32; t += gridDim.x * blockDim.x) groups[t] = 0ull;
}

// Host code must not use g_sieve_scratch as an address: in host code the name
// is a host-side stand-in.  The device address is looked up once per device.
constexpr int kMaxDevices = 64;
unsigned char* g_dev_addr[kMaxDevices] = {};
int g_dev_sms[kMaxDevices] = {};
std::mutex g_mu;

sj_status scratch_address(int device, unsigned char** out, int* num_sms, const char** err) {
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_dev_addr[device]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_sieve_scratch);
    if (e != cudaSuccess || !p) {
      if (err) *err = "cudaGetSymbolAddress of the sieve scratch array failed";
      return SJ_ECUDA;
    }
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || sms < 1) {
      cudaGetLastError();
      if (err) *err = "cudaDeviceGetAttribute(multiprocessor count) failed";
      return SJ_ECUDA;
    }
    g_dev_addr[device] = static_cast<unsigned char*>(p);
    g_dev_sms[device] = sms;
  }
  *out = g_dev_addr[device];
  *num_sms = g_dev_sms[device];
  return SJ_OK;
}

}  // namespace

extern "C" sj_status sj_sieve_noalloc(void* cuda_stream, int ncols, const int32_t* const* in_cols,
                                      int64_t nrows, int key_col, const uint32_t* filter_words,
                                      uint64_t nblocks, const sj_filter_params* params,
                                      int32_t* const* out_cols, uint64_t* out_count,
                                      uint32_t* status, const char** err) {
  auto bad = [&](const char* m) {
    if (err) *err = m;
    return SJ_EINVAL;
  };
  if (ncols < 1 || ncols > SJ_MAX_COLS) return bad("ncols must be in 1..SJ_MAX_COLS");
  if (nrows < 0) return bad("nrows must be >= 0");
  if (nrows > kMaxRows) return bad("nrows exceeds SJ_NOALLOC_MAX_ROWS (the fixed scratch size)");
  if (key_col < 0 || key_col >= ncols) return bad("key_col out of range");
  if (!in_cols || !out_cols || !out_count || !filter_words || !params)
    return bad("null argument");
  if (nblocks < 1 || nblocks >= (uint64_t(1) << 32)) return bad("nblocks must be in 1..2^32-1");
  if (params->layout > SJ_CLASSIC) return bad("unknown filter layout");
  if ((params->layout == SJ_REGBLOCKED32 && (params->k < 1 || params->k > 6)) ||
      (params->layout == SJ_BLOCKED256 && (params->k < 1 || params->k > 4)) ||
      (params->layout == SJ_CLASSIC && (params->k < 1 || params->k > 8)))
    return bad("k out of range for the layout");
  if (reinterpret_cast<uintptr_t>(filter_words) & 15) return bad("filter words must be 16-byte aligned");
  for (int j = 0; j < ncols; ++j) {
    if (!in_cols[j] || !out_cols[j]) return bad("null column pointer");
    if ((reinterpret_cast<uintptr_t>(in_cols[j]) | reinterpret_cast<uintptr_t>(out_cols[j])) & 15)
      return bad("columns must be 16-byte aligned");
  }
  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess || device < 0 || device >= kMaxDevices) {
    cudaGetLastError();
    if (err) *err = "no usable current CUDA device";
    return SJ_ECUDA;
  }
  unsigned char* base = nullptr;
  int num_sms = 0;
  sj_status st = scratch_address(device, &base, &num_sms, err);
  if (st != SJ_OK) return st;

  cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
  const int chunk_rows = sj::sieve_chunk_rows(nrows, num_sms);
  const int64_t nchunks = (nrows + chunk_rows - 1) / chunk_rows;
  if (nchunks > kMaxChunks) {
    if (err) *err = "too many chunks for the fixed scratch on this GPU";
    return SJ_EINVAL;
  }
  const uint32_t prep_grid = (uint32_t)((nchunks + 255) / 256 > 0 ? (nchunks + 255) / 256 : 1);
  k_noalloc_prepare<<<prep_grid, 256, 0, stream>>>(nblocks, (uint32_t)nchunks, status ? 0 : 1);

  sj::SieveArgs a = {};
  a.ntest = 1;
  a.test[0].col = in_cols[key_col];
  a.test[0].is_pred = 0;
  a.test[0].f.words = filter_words;
  a.test[0].f.hdr = reinterpret_cast<const uint64_t*>(base + kOffHdr);
  a.test[0].f.k = params->k;
  a.test[0].f.layout = params->layout;
  a.test[0].f.seed = params->seed;
  a.nout = ncols;
  for (int j = 0; j < ncols; ++j) {
    a.in[j] = in_cols[j];
    a.out[j] = out_cols[j];
    a.out_is_vec[j] = j == key_col ? 1 : 0;
  }
  a.n_host = nrows;
  a.n_dev = nullptr;
  a.out_n = out_count;
  a.out_n2 = nullptr;
  a.tile_counter = reinterpret_cast<uint32_t*>(base + kOffCounter);
  a.lb.st = reinterpret_cast<uint64_t*>(base + kOffStates);
  a.lb.status = status ? status : reinterpret_cast<uint32_t*>(base + kOffStatus);
  a.lb.epoch = 0;  // the states are zeroed by k_noalloc_prepare
  a.grp = reinterpret_cast<uint64_t*>(base + kOffGroups);  // zeroed there too
  a.fin = reinterpret_cast<uint32_t*>(base + kOffFin);
  a.chunk_rows = chunk_rows;
  a.fast_words_ok = 1;  // nblocks < 2^32 is checked above, but the word count must be too
  if (nblocks * 8 >= (uint64_t(1) << 32)) a.fast_words_ok = 0;
  sj::launch_sieve_chunk(a, nrows, num_sms, stream);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    if (err) *err = cudaGetErrorString(e);
    return SJ_ECUDA;
  }
  return SJ_OK;
}
