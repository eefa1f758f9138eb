// sw_search_noalloc: a single-query search that allocates no memory.
//
// Some callers cannot allocate device memory while they search: a service
// that pins its whole memory budget at start-up and must not grow it, a
// real-time loop in which a cudaMalloc may synchronise the device and stall
// every stream, or a host that runs this library inside a fixed arena it does
// not control.  For them this entry point keeps every scratch buffer the
// inter-task kernel needs (the query profile, the task list, the counters)
// in one file-scope __device__ array of
// kNoAllocScratchBytes.  Every GPU that loads the library holds that array
// until the process exits; the caller passes the prepared database, the query
// and the output buffer, and nothing is allocated per call.
#include <cstdio>
#include <mutex>

#include "internal.h"
#include "../../include/swgb.h"

namespace swgb {
namespace {

constexpr size_t kNoAllocScratchBytes = 16u << 20;  // 16 MiB per device
constexpr int kNoAllocMaxQuery = 768;               // one chunk: 32 lanes x 24 rows
// the task list takes 16 bytes per 8 sequences at most (chains of more than
// 16 lanes: one chain per warp, 8 warps per CTA)
constexpr int64_t kNoAllocMaxSeqs = 8000000;
constexpr int kNoAllocThreads = 256;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) uint8_t g_noalloc_scratch[kNoAllocScratchBytes];

// Scratch layout (byte offsets).
constexpr size_t kOffWords = 0;      // int32 [0] task counter, [1] task count, [2] status
constexpr size_t kOffQDesc = 256;    // one QDesc
constexpr size_t kOffSubmat = 512;   // 400 bytes
constexpr size_t kOffQuery = 1024;   // up to kNoAllocMaxQuery residues
constexpr size_t kOffProf = 2048;    // one profile chunk: 21 x round_up(L*R, 128) bytes
constexpr size_t kProfMax = 21 * 768;
constexpr size_t kOffTasks = kOffProf + kProfMax;  // the task list
static_assert(kOffTasks % 16 == 0, "tasks are 16-byte records");

struct DeviceSetup {
  uint8_t *scratch = nullptr;  // device address of g_noalloc_scratch on this device
  int occ16 = 0, occ24 = 0;    // resident CTAs per SM of the two kernel instances used
};
DeviceSetup g_setup[kMaxDevices];
std::mutex g_setup_mutex;

// Tiles of `chains` consecutive units (one database sequence per unit: the
// int32 form, unit u = sorted position u); the database is sorted longest
// first, so the tiles are too.
__global__ void noalloc_plan_kernel(Task *tasks, int32_t n, int32_t chains, int32_t *n_tasks) {
  const int32_t nt = (n + chains - 1) / chains;
  const int32_t stride = gridDim.x * blockDim.x;
  for (int32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < nt; t += stride) {
    Task tk;
    tk.q = 0;
    tk.unit_begin = t * chains;
    tk.unit_count = min(chains, n - t * chains);
    tk.pad_ = 0;
    tasks[t] = tk;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *n_tasks = nt;
}

inline size_t round_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

int fail_msg(int code, const char *fmt, long long a = 0, long long b = 0) {
  char buf[256];
  snprintf(buf, sizeof buf, fmt, a, b);
  return set_last_error(code, buf);
}

int cuda_err(cudaError_t e, const char *what) {
  char buf[256];
  snprintf(buf, sizeof buf, "sw_search_noalloc: %s: %s", what, cudaGetErrorString(e));
  return set_last_error(e == cudaErrorMemoryAllocation ? SW_ENOMEM : SW_ECUDA, buf);
}

}  // namespace
}  // namespace swgb

using namespace swgb;

extern "C" int sw_search_noalloc(const sw_db *db, const uint8_t *query, int64_t m, const int8_t *submat,
                                 int32_t gap_open, int32_t gap_extend, int32_t *scores_dev, void *stream) {
  clear_last_error();
  if (!db) return fail_msg(SW_EINVAL, "sw_search_noalloc: null database");
  if (m < 0 || m > kNoAllocMaxQuery)
    return fail_msg(SW_EINVAL, "sw_search_noalloc: query length %lld outside 0..%lld", (long long)m,
                    (long long)kNoAllocMaxQuery);
  if (m > 0 && !query) return fail_msg(SW_EINVAL, "sw_search_noalloc: null query");
  for (int64_t i = 0; i < m; ++i)
    if (query[i] >= kAlphabet) return fail_msg(SW_EINVAL, "sw_search_noalloc: residue code %lld >= 20", query[i]);
  if (!submat) return fail_msg(SW_EINVAL, "sw_search_noalloc: null submat");
  int smin = 127, smax = -128;
  for (int i = 0; i < kAlphabet * kAlphabet; ++i) {
    smin = submat[i] < smin ? submat[i] : smin;
    smax = submat[i] > smax ? submat[i] : smax;
  }
  if (smin < -64 || smax > 63) return fail_msg(SW_EINVAL, "sw_search_noalloc: submat entries must lie in [-64, 63]");
  if (gap_open < 0 || gap_extend < 0 || (int64_t)gap_open + 2 * (int64_t)gap_extend > 1024)
    return fail_msg(SW_EINVAL, "sw_search_noalloc: gap penalties out of range (%lld, %lld)", gap_open, gap_extend);
  const DbView &v = db_view(db);
  const int64_t n = v.n;
  if (n > kNoAllocMaxSeqs)
    return fail_msg(SW_EINVAL, "sw_search_noalloc: database of %lld sequences exceeds the maximum %lld", (long long)n,
                    (long long)kNoAllocMaxSeqs);
  if (n == 0) return SW_OK;
  if (!scores_dev) return fail_msg(SW_EINVAL, "sw_search_noalloc: null scores");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_err(e, "cudaGetDevice");
  if (dev != db_device(db))
    return fail_msg(SW_EINVAL, "sw_search_noalloc: the current device %lld is not the database's device %lld", dev,
                    db_device(db));
  if (dev >= kMaxDevices)
    return fail_msg(SW_EINVAL, "sw_search_noalloc: device index %lld is beyond the %lld devices this entry point "
                    "supports", dev, kMaxDevices);
  cudaPointerAttributes pa;
  if (cudaPointerGetAttributes(&pa, scores_dev) != cudaSuccess || pa.type != cudaMemoryTypeDevice) {
    cudaGetLastError();
    return fail_msg(SW_EINVAL, "sw_search_noalloc: scores must be device memory");
  }

  // One-time set-up per device (the current one): the device address of the
  // scratch array and the kernel's shared-memory limit.
  DeviceSetup setup;
  {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    DeviceSetup &st = g_setup[dev];
    if (!st.scratch) {
      void *p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess) return cuda_err(e, "cudaGetSymbolAddress");
      const size_t smem = inter_smem_bytes((int)round_up(kProfMax, 128), 2, kNoAllocThreads);
      st.occ16 = inter_max_ctas_per_sm(16, kFormInt32, kNoAllocThreads, smem);
      st.occ24 = inter_max_ctas_per_sm(24, kFormInt32, kNoAllocThreads, smem);
      if (st.occ16 <= 0 || st.occ24 <= 0) return fail_msg(SW_ECUDA, "sw_search_noalloc: kernel configuration failed");
      st.scratch = static_cast<uint8_t *>(p);
    }
    setup = st;
  }

  // Plan: a single chunk of L lanes x R rows covers the query.
  const int R = m > 32 * 16 ? 24 : 16;
  int L = (int)((m + R - 1) / R);
  L = L < 4 ? 4 : (L > 32 ? 32 : L);
  QDesc d{};
  d.m = (int32_t)m;
  d.L = L;
  d.R = R;
  d.nchunks = 1;
  d.chunk_stride = (int32_t)round_up((size_t)profile_slots(L) * R, 128);
  d.chunk_bytes = kProfRows * d.chunk_stride;
  d.prof_off = 0;
  d.qoff = 0;
  const int warps = kNoAllocThreads / 32;
  const int chains = warps * (32 / L);
  const int64_t n_tasks = (n + chains - 1) / chains;
  if (kOffTasks + sizeof(Task) * (size_t)n_tasks > kNoAllocScratchBytes)
    return fail_msg(SW_EINVAL, "sw_search_noalloc: database of %lld sequences does not fit the scratch", (long long)n);

  uint8_t *scr = setup.scratch;
  int32_t *words = reinterpret_cast<int32_t *>(scr + kOffWords);
  Task *tasks = reinterpret_cast<Task *>(scr + kOffTasks);
  cudaStream_t s = (cudaStream_t)stream;

  // The scratch keeps the previous call's contents: counters start at zero.
  if ((e = cudaMemsetAsync(words, 0, 16, s)) != cudaSuccess) return cuda_err(e, "memset");
  if ((e = cudaMemcpyAsync(scr + kOffQDesc, &d, sizeof d, cudaMemcpyHostToDevice, s)) != cudaSuccess)
    return cuda_err(e, "upload");
  if ((e = cudaMemcpyAsync(scr + kOffSubmat, submat, 400, cudaMemcpyHostToDevice, s)) != cudaSuccess)
    return cuda_err(e, "upload");
  if (m > 0 && (e = cudaMemcpyAsync(scr + kOffQuery, query, (size_t)m, cudaMemcpyHostToDevice, s)) != cudaSuccess)
    return cuda_err(e, "upload");
  const int64_t pblocks = (n_tasks + kNoAllocThreads - 1) / kNoAllocThreads;
  const int pgrid = (int)(pblocks > 1024 ? 1024 : pblocks);
  noalloc_plan_kernel<<<pgrid, kNoAllocThreads, 0, s>>>(tasks, (int32_t)n, chains, words + 1);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_err(e, "plan kernel");
  Scoring sc{};
  sc.go = gap_open + gap_extend;
  sc.ge = gap_extend;
  sc.pad = smin < 0 ? smin : 0;
  sc.maxp = smax > 0 ? smax : 0;
  sc.thresh = 32767 - sc.maxp;
  if ((e = launch_build_profiles(scr + kOffQuery, reinterpret_cast<const QDesc *>(scr + kOffQDesc), 1,
                                 reinterpret_cast<const int8_t *>(scr + kOffSubmat), sc.pad, scr + kOffProf, s)) !=
      cudaSuccess)
    return cuda_err(e, "profile kernel");

  InterArgs a{};
  a.db = v;
  a.unit_pos = db_ident(db);  // the database's own [0, 1, ..., n - 1]: unit u is sorted position u
  a.n_unit_pos = n + 1;
  a.prof_bytes = (int64_t)kProfMax;
  a.out_size = n;
  a.qd = reinterpret_cast<const QDesc *>(scr + kOffQDesc);
  a.tasks = tasks;
  a.n_tasks = words + 1;
  a.task_counter = words + 0;
  a.prof = scr + kOffProf;
  a.pbuf_bytes = (int32_t)round_up((size_t)d.chunk_bytes, 128);
  a.gbuf = reinterpret_cast<uint2 *>(scr);  // a single chunk never touches the boundary strip
  a.gbuf_stride = 0;
  a.out = scores_dev;
  a.out_stride = n;
  a.sc = sc;
  a.status = words + 2;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int occ = R == 24 ? setup.occ24 : setup.occ16;
  const int64_t gmax = (int64_t)(sms > 0 ? sms : 1) * occ;
  const int grid = (int)(n_tasks < gmax ? n_tasks : gmax);
  a.pbuf_count = 2;
  const size_t smem = inter_smem_bytes(a.pbuf_bytes, a.pbuf_count, kNoAllocThreads);
  if ((e = launch_inter(a, R, kFormInt32, grid, kNoAllocThreads, smem, s)) != cudaSuccess) return cuda_err(e, "DP kernel");

  int32_t status = 0;
  if ((e = cudaMemcpyAsync(&status, words + 2, 4, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
    return cuda_err(e, "status read");
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_err(e, "synchronise");
  if (status == SW_ETIMEOUT) return fail_msg(SW_ETIMEOUT, "sw_search_noalloc: a bounded device wait expired");
  if (status == kStatusBounds) return fail_msg(SW_ECUDA, "sw_search_noalloc: an index check failed (checked build)");
  return SW_OK;
}
