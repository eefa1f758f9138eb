// C-ABI entry points (include/swgb.h): database packing, query planning and the
// search pipeline (profile -> DP kernels -> overflow rescue), all on one GPU.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "../../include/swgb.h"
#include "internal.h"

using namespace swgb;

namespace {

thread_local std::string g_err;

int fail(int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

int cuda_fail(cudaError_t e, const char *what) {
  if (e == cudaErrorMemoryAllocation) return fail(SW_ENOMEM, "%s: %s", what, cudaGetErrorString(e));
  return fail(SW_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define SW_CUDA(call, what)                   \
  do {                                        \
    cudaError_t e_ = (call);                  \
    if (e_ != cudaSuccess) return cuda_fail(e_, what); \
  } while (0)

inline int64_t round_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

int sm_count(int dev) {
  int n = 0;
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n > 0 ? n : 1;
}

int check_seqs(const uint8_t *res, const int64_t *off, int64_t n, const char *what) {
  if (n < 0) return fail(SW_EINVAL, "%s: negative sequence count", what);
  if (!off) return fail(SW_EINVAL, "%s: null offsets", what);
  if (off[0] != 0) return fail(SW_EINVAL, "%s: offsets[0] must be 0", what);
  for (int64_t i = 0; i < n; ++i)
    if (off[i + 1] < off[i]) return fail(SW_EINVAL, "%s: offsets decrease at %lld", what, (long long)i);
  const int64_t total = off[n];
  if (total > 0 && !res) return fail(SW_EINVAL, "%s: null residues", what);
  for (int64_t i = 0; i < total; ++i)
    if (res[i] >= kAlphabet) return fail(SW_EINVAL, "%s: residue code %d >= 20 at %lld", what, (int)res[i], (long long)i);
  return SW_OK;
}

bool is_device_ptr(const void *p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

struct sw_db {
  int device = 0;
  int64_t n = 0, total = 0;
  DbView view{};
  void *block = nullptr;
  size_t bytes = 0;
  int32_t max_npad = 0;
  double mean_npad = 0;
};

struct sw_queries {
  const sw_db *db = nullptr;
  int64_t nq = 0;
  int mode = SW_MODE_PACKED;
  int R = 16;
  Scoring sc{};
  std::vector<QDesc> qd;
  int64_t n_units = 0;
  int64_t n_tasks = 0, n_rtask_cap = 0;
  int grid = 1, rgrid = 1;
  int pbuf_bytes = 0;
  size_t smem = 0;
  int32_t gbuf_stride = 0;
  // device memory (one stream-ordered allocation)
  void *block = nullptr;
  size_t bytes = 0;
  cudaStream_t alloc_stream = nullptr;
  uint8_t *d_qres = nullptr;
  int8_t *d_submat = nullptr;
  QDesc *d_qd = nullptr;
  Task *d_tasks = nullptr, *d_rtasks = nullptr;
  int32_t *d_units = nullptr;
  uint8_t *d_prof = nullptr;
  int64_t prof_bytes = 0;
  uint2 *d_gbuf = nullptr;
  int32_t *d_words = nullptr;  // [0] task counter, [1] rescue counter, [2] status, [3] rescue n_tasks, [4.. 4+nq) flag counts
  int32_t *d_ntasks = nullptr; // constant: main n_tasks
  int32_t *d_flag_pos = nullptr;
  int64_t h2d_bytes = 0;
  bool timing = false, timed = false;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
};

namespace {

// Lanes per chain for one query at R rows per lane: minimise padded rows x
// pipeline fill x idle lanes, with a small charge per chunk for the
// boundary strip and the CTA barrier.
int choose_lanes(int m, int R, double mean_n) {
  int bestL = 8;
  double best = 1e300;
  for (int L = 4; L <= 32; ++L) {
    const int LR = L * R;
    const int C = std::max(1, (m + LR - 1) / LR);
    const double rows = (double)C * LR;
    const int G = 32 / L;
    const double lane_eff = (double)(G * L) / 32.0;
    const double fill = (mean_n + L - 1 + 8) / std::max(1.0, mean_n);
    const double cost = rows * fill / lane_eff * (1.0 + 0.01 * C);
    if (cost < best - 1e-9) {
      best = cost;
      bestL = L;
    }
  }
  return bestL;
}

int env_int(const char *name, int dflt) {
  const char *v = getenv(name);
  return v && *v ? atoi(v) : dflt;
}

}  // namespace

extern "C" {

const char *sw_last_error(void) { return g_err.c_str(); }

int sw_db_prepare(const uint8_t *residues, const int64_t *offsets, int64_t n_seqs, void *stream, sw_db **out) {
  g_err.clear();
  if (!out) return fail(SW_EINVAL, "sw_db_prepare: null output handle");
  *out = nullptr;
  if (int rc = check_seqs(residues, offsets, n_seqs, "sw_db_prepare")) return rc;
  if (n_seqs >= (int64_t)1 << 30) return fail(SW_EINVAL, "sw_db_prepare: too many sequences");
  cudaStream_t s = (cudaStream_t)stream;
  sw_db *db = new sw_db();
  SW_CUDA(cudaGetDevice(&db->device), "cudaGetDevice");
  db->n = n_seqs;
  db->total = n_seqs ? offsets[n_seqs] : 0;

  std::vector<int32_t> order(n_seqs), len(n_seqs), npad(n_seqs);
  std::vector<int64_t> off(n_seqs);
  for (int64_t i = 0; i < n_seqs; ++i) {
    const int64_t L = offsets[i + 1] - offsets[i];
    if (L > (int64_t)1 << 28) {
      delete db;
      return fail(SW_EINVAL, "sw_db_prepare: sequence %lld too long", (long long)i);
    }
    len[i] = (int32_t)L;
  }
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return len[a] > len[b]; });
  int64_t padded = 0;
  std::vector<int32_t> slen(n_seqs);
  for (int64_t k = 0; k < n_seqs; ++k) {
    slen[k] = len[order[k]];
    npad[k] = (int32_t)std::max<int64_t>(kColBlock, round_up(slen[k], kColBlock));
    off[k] = padded;
    padded += npad[k];
    db->max_npad = std::max(db->max_npad, npad[k]);
  }
  db->mean_npad = n_seqs ? (double)padded / n_seqs : 0;
  std::vector<uint8_t> packed((size_t)std::max<int64_t>(padded, 16), (uint8_t)kPadCode);
  for (int64_t k = 0; k < n_seqs; ++k)
    if (slen[k]) memcpy(&packed[off[k]], residues + offsets[order[k]], (size_t)slen[k]);

  const size_t b_res = round_up((int64_t)packed.size(), 256);
  const size_t b_off = round_up(8 * std::max<int64_t>(n_seqs, 1), 256);
  const size_t b_i32 = round_up(4 * std::max<int64_t>(n_seqs, 1), 256);
  db->bytes = b_res + b_off + 3 * b_i32;
  cudaError_t e = cudaMalloc(&db->block, db->bytes);
  if (e != cudaSuccess) {
    delete db;
    return cuda_fail(e, "sw_db_prepare: device allocation");
  }
  uint8_t *p = (uint8_t *)db->block;
  db->view.res = p;
  db->view.off = (const int64_t *)(p + b_res);
  db->view.npad = (const int32_t *)(p + b_res + b_off);
  db->view.len = (const int32_t *)(p + b_res + b_off + b_i32);
  db->view.perm = (const int32_t *)(p + b_res + b_off + 2 * b_i32);
  db->view.n = n_seqs;
  e = cudaMemcpyAsync((void *)db->view.res, packed.data(), packed.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && n_seqs) {
    e = cudaMemcpyAsync((void *)db->view.off, off.data(), 8 * n_seqs, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync((void *)db->view.npad, npad.data(), 4 * n_seqs, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync((void *)db->view.len, slen.data(), 4 * n_seqs, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync((void *)db->view.perm, order.data(), 4 * n_seqs, cudaMemcpyHostToDevice, s);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    cudaFree(db->block);
    delete db;
    return cuda_fail(e, "sw_db_prepare: upload");
  }
  *out = db;
  return SW_OK;
}

int sw_db_free(sw_db *db) {
  g_err.clear();
  if (!db) return SW_OK;
  if (db->block) cudaFree(db->block);
  delete db;
  return SW_OK;
}

int sw_db_stats(const sw_db *db, int64_t *n_seqs, int64_t *residues, int64_t *device_bytes) {
  g_err.clear();
  if (!db) return fail(SW_EINVAL, "sw_db_stats: null handle");
  if (n_seqs) *n_seqs = db->n;
  if (residues) *residues = db->total;
  if (device_bytes) *device_bytes = (int64_t)db->bytes;
  return SW_OK;
}

int sw_queries_prepare(const sw_db *db, const uint8_t *queries, const int64_t *q_offsets, int64_t n_queries,
                       const int8_t *submat, int32_t gap_open, int32_t gap_extend, int32_t mode, int32_t cutover,
                       void *stream, sw_queries **out) {
  g_err.clear();
  (void)cutover;
  if (!out) return fail(SW_EINVAL, "sw_queries_prepare: null output handle");
  *out = nullptr;
  if (!db) return fail(SW_EINVAL, "sw_queries_prepare: null database");
  if (!submat) return fail(SW_EINVAL, "sw_queries_prepare: null submat");
  if (mode != SW_MODE_INT32 && mode != SW_MODE_PACKED) return fail(SW_EINVAL, "sw_queries_prepare: bad mode %d", mode);
  if (gap_open < 0 || gap_extend < 0 || (int64_t)gap_open + 2 * (int64_t)gap_extend > 1024)
    return fail(SW_EINVAL, "sw_queries_prepare: gap penalties out of range (%d, %d)", gap_open, gap_extend);
  if (int rc = check_seqs(queries, q_offsets, n_queries, "sw_queries_prepare")) return rc;
  int smin = 127, smax = -128;
  for (int i = 0; i < kAlphabet * kAlphabet; ++i) {
    smin = std::min<int>(smin, submat[i]);
    smax = std::max<int>(smax, submat[i]);
  }
  if (smin < -64 || smax > 63) return fail(SW_EINVAL, "sw_queries_prepare: submat entries must lie in [-64, 63]");
  if (n_queries * std::max<int64_t>(db->n, 1) >= ((int64_t)1 << 31))
    return fail(SW_EINVAL, "sw_queries_prepare: n_queries * n_db must be < 2^31");
  for (int64_t i = 0; i < n_queries; ++i)
    if (q_offsets[i + 1] - q_offsets[i] > (1 << 24)) return fail(SW_EINVAL, "sw_queries_prepare: query too long");

  cudaStream_t s = (cudaStream_t)stream;
  sw_queries *Q = new sw_queries();
  Q->db = db;
  Q->nq = n_queries;
  Q->mode = mode;
  Q->alloc_stream = s;
  const bool packed = mode == SW_MODE_PACKED;
  Scoring &sc = Q->sc;
  sc.go = gap_open + gap_extend;
  sc.ge = gap_extend;
  sc.kbias = std::max(0, -smin);
  sc.maxp = std::max(0, smax);
  sc.bias = sc.go + sc.ge + sc.kbias;
  sc.thresh = 32767 - sc.maxp;

  int R = env_int("SWGB_R", 16);
  if (!inter_supported_R(R)) R = 16;
  Q->R = R;
  const int threads = inter_threads();
  const int warps = threads / 32;
  const double mean_n = std::max(16.0, db->mean_npad);
  const int forceL = env_int("SWGB_L", 0);

  // --- per-query plan
  Q->qd.resize(n_queries);
  int64_t prof = 0;
  int maxc = 16;
  bool chunked = false;
  for (int64_t q = 0; q < n_queries; ++q) {
    QDesc &d = Q->qd[q];
    d.m = (int32_t)(q_offsets[q + 1] - q_offsets[q]);
    d.R = R;
    d.L = (forceL >= 4 && forceL <= 32) ? forceL : choose_lanes(std::max(1, d.m), R, mean_n);
    const int LR = d.L * R;
    d.nchunks = std::max(1, (d.m + LR - 1) / LR);
    d.chunk_stride = (int32_t)round_up(LR, 128);
    d.chunk_bytes = kProfRows * d.chunk_stride;
    d.prof_off = prof;
    d.qoff = q_offsets[q];
    prof += (int64_t)d.nchunks * d.chunk_bytes;
    maxc = std::max(maxc, d.chunk_bytes);
    chunked |= d.nchunks > 1;
  }
  Q->prof_bytes = std::max<int64_t>(prof, 16);
  Q->pbuf_bytes = (int)round_up(maxc, 128);

  // --- units (sorted positions) and tasks, longest first
  const int64_t n = db->n;
  Q->n_units = packed ? (n + 1) / 2 : n;
  std::vector<int32_t> units(std::max<int64_t>(1, packed ? 2 * Q->n_units : n));
  if (packed) {
    for (int64_t u = 0; u < Q->n_units; ++u) {
      units[2 * u] = (int32_t)(2 * u);
      units[2 * u + 1] = (int32_t)std::min<int64_t>(2 * u + 1, n - 1);
    }
  } else {
    for (int64_t u = 0; u < n; ++u) units[u] = (int32_t)u;
  }
  struct TW {
    Task t;
    double w;
  };
  std::vector<TW> tw;
  std::vector<int32_t> h_npad;
  if (n) {
    h_npad.resize(n);
    SW_CUDA(cudaMemcpy(h_npad.data(), db->view.npad, 4 * n, cudaMemcpyDeviceToHost), "sw_queries_prepare: read db");
  }
  int64_t rcap = 0;
  for (int64_t q = 0; q < n_queries && Q->n_units > 0; ++q) {
    const QDesc &d = Q->qd[q];
    const int chains = warps * (32 / d.L);
    for (int64_t u0 = 0; u0 < Q->n_units; u0 += chains) {
      Task t;
      t.q = (int32_t)q;
      t.unit_begin = (int32_t)u0;
      t.unit_count = (int32_t)std::min<int64_t>(chains, Q->n_units - u0);
      t.pad_ = 0;
      const int32_t first = units[packed ? 2 * u0 : u0];
      tw.push_back({t, (double)d.nchunks * d.L * d.R * (h_npad[first] + d.L + 8)});
    }
    rcap += (n + chains - 1) / chains;
  }
  std::stable_sort(tw.begin(), tw.end(), [](const TW &a, const TW &b) { return a.w > b.w; });
  Q->n_tasks = (int64_t)tw.size();
  Q->n_rtask_cap = packed ? rcap : 0;

  // --- launch geometry
  const int sms = sm_count(db->device);
  Q->smem = inter_smem_bytes(Q->pbuf_bytes, threads);
  if (Q->smem > 200 * 1024) {
    delete Q;
    return fail(SW_EINVAL, "sw_queries_prepare: profile chunk too large");
  }
  const int occ = inter_max_ctas_per_sm(R, packed, threads, Q->smem);
  const int occ32 = inter_max_ctas_per_sm(R, false, threads, Q->smem);
  Q->grid = (int)std::max<int64_t>(1, std::min<int64_t>(Q->n_tasks, (int64_t)sms * occ));
  Q->rgrid = std::max(1, sms * occ32);
  const int gslots = std::max(Q->grid, Q->rgrid);
  Q->gbuf_stride = chunked ? (int32_t)round_up(std::max(16, db->max_npad), 16) : 2;

  // --- device allocation (stream ordered)
  const int64_t nqm = std::max<int64_t>(n_queries, 1);
  const size_t b_qres = round_up(std::max<int64_t>(q_offsets[n_queries], 16), 256);
  const size_t b_sub = 512;
  const size_t b_qd = round_up(sizeof(QDesc) * nqm, 256);
  const size_t b_tasks = round_up(sizeof(Task) * std::max<int64_t>(Q->n_tasks, 1), 256);
  const size_t b_rtasks = round_up(sizeof(Task) * std::max<int64_t>(Q->n_rtask_cap, 1), 256);
  const size_t b_units = round_up(4 * (int64_t)units.size(), 256);
  const size_t b_prof = round_up(Q->prof_bytes, 256);
  const size_t b_gbuf = round_up((int64_t)gslots * warps * 8 * (int64_t)Q->gbuf_stride * 8, 256);
  const size_t b_words = round_up(4 * (8 + nqm), 256);
  const size_t b_flag = packed ? round_up(4 * nqm * std::max<int64_t>(n, 1), 256) : 0;
  Q->bytes = b_qres + b_sub + b_qd + b_tasks + b_rtasks + b_units + b_prof + b_gbuf + b_words + b_flag;
  cudaError_t e = cudaMallocAsync(&Q->block, Q->bytes, s);
  if (e != cudaSuccess) {
    delete Q;
    return cuda_fail(e, "sw_queries_prepare: device allocation");
  }
  uint8_t *p = (uint8_t *)Q->block;
  auto take = [&](size_t b) {
    uint8_t *r = p;
    p += b;
    return r;
  };
  Q->d_qres = take(b_qres);
  Q->d_submat = (int8_t *)take(b_sub);
  Q->d_qd = (QDesc *)take(b_qd);
  Q->d_tasks = (Task *)take(b_tasks);
  Q->d_rtasks = (Task *)take(b_rtasks);
  Q->d_units = (int32_t *)take(b_units);
  Q->d_prof = take(b_prof);
  Q->d_gbuf = (uint2 *)take(b_gbuf);
  Q->d_words = (int32_t *)take(b_words);
  Q->d_flag_pos = packed ? (int32_t *)take(b_flag) : nullptr;
  Q->d_ntasks = Q->d_words + 4 + nqm + 1;  // past the zeroed region

  Q->h2d_bytes = q_offsets[n_queries] + 400 + (int64_t)sizeof(QDesc) * n_queries + (int64_t)sizeof(Task) * Q->n_tasks +
                 4 * (int64_t)units.size() + 4;
  std::vector<Task> tasks(Q->n_tasks);
  for (int64_t i = 0; i < Q->n_tasks; ++i) tasks[i] = tw[i].t;
  int32_t nt32 = (int32_t)Q->n_tasks;
  e = cudaSuccess;
  if (q_offsets[n_queries] > 0)
    e = cudaMemcpyAsync(Q->d_qres, queries, q_offsets[n_queries], cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(Q->d_submat, submat, 400, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && n_queries)
    e = cudaMemcpyAsync(Q->d_qd, Q->qd.data(), sizeof(QDesc) * n_queries, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && Q->n_tasks)
    e = cudaMemcpyAsync(Q->d_tasks, tasks.data(), sizeof(Task) * Q->n_tasks, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(Q->d_units, units.data(), 4 * units.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(Q->d_words, 0, b_words, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(Q->d_ntasks, &nt32, 4, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    cudaFreeAsync(Q->block, s);
    delete Q;
    return cuda_fail(e, "sw_queries_prepare: upload");
  }
  *out = Q;
  return SW_OK;
}

int sw_queries_free(sw_queries *q) {
  g_err.clear();
  if (!q) return SW_OK;
  if (q->block) {
    cudaFreeAsync(q->block, q->alloc_stream);
    cudaStreamSynchronize(q->alloc_stream);
  }
  if (q->ev0) cudaEventDestroy(q->ev0);
  if (q->ev1) cudaEventDestroy(q->ev1);
  delete q;
  return SW_OK;
}

int sw_search_prepared(const sw_db *db, const sw_queries *Q, int32_t *scores_dev, void *stream) {
  g_err.clear();
  if (!db || !Q) return fail(SW_EINVAL, "sw_search_prepared: null handle");
  if (Q->db != db) return fail(SW_EINVAL, "sw_search_prepared: query batch prepared for another database");
  if (Q->nq == 0 || db->n == 0) return SW_OK;
  if (!scores_dev) return fail(SW_EINVAL, "sw_search_prepared: null scores");
  cudaStream_t s = (cudaStream_t)stream;
  const bool packed = Q->mode == SW_MODE_PACKED;
  const int threads = inter_threads();

  SW_CUDA(cudaMemsetAsync(Q->d_words, 0, 4 * (4 + Q->nq), s), "memset");
  SW_CUDA(launch_build_profiles(Q->d_qres, Q->d_qd, (int32_t)Q->nq, Q->d_submat, Q->sc.kbias, Q->d_prof, s),
          "profile kernel");

  InterArgs a{};
  a.db = db->view;
  a.unit_pos = Q->d_units;
  a.qd = Q->d_qd;
  a.tasks = Q->d_tasks;
  a.n_tasks = Q->d_ntasks;
  a.task_counter = Q->d_words + 0;
  a.prof = Q->d_prof;
  a.pbuf_bytes = Q->pbuf_bytes;
  a.gbuf = Q->d_gbuf;
  a.gbuf_stride = Q->gbuf_stride;
  a.out = scores_dev;
  a.out_stride = db->n;
  a.flag_count = Q->d_words + 4;
  a.flag_pos = Q->d_flag_pos;
  a.sc = Q->sc;
  a.status = Q->d_words + 2;
  if (Q->timing) SW_CUDA(cudaEventRecord(Q->ev0, s), "event");
  SW_CUDA(launch_inter(a, Q->R, packed, Q->grid, threads, Q->smem, s), "DP kernel");
  if (Q->timing) {
    SW_CUDA(cudaEventRecord(Q->ev1, s), "event");
    const_cast<sw_queries *>(Q)->timed = true;
  }

  if (packed) {
    SW_CUDA(launch_rescue_tasks(Q->d_words + 4, Q->d_qd, (int32_t)Q->nq, db->n, threads / 32, Q->d_rtasks,
                                Q->d_words + 3, Q->d_words + 1, s),
            "rescue task kernel");
    InterArgs r = a;
    r.unit_pos = Q->d_flag_pos;
    r.tasks = Q->d_rtasks;
    r.n_tasks = Q->d_words + 3;
    r.task_counter = Q->d_words + 1;
    r.flag_count = nullptr;
    r.flag_pos = nullptr;
    SW_CUDA(launch_inter(r, Q->R, false, Q->rgrid, threads, Q->smem, s), "rescue kernel");
  }
  return SW_OK;
}

int sw_queries_status(const sw_queries *Q, void *stream, int64_t *rescued) {
  g_err.clear();
  if (!Q) return fail(SW_EINVAL, "sw_queries_status: null handle");
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<int32_t> w(4 + Q->nq);
  SW_CUDA(cudaMemcpyAsync(w.data(), Q->d_words, 4 * w.size(), cudaMemcpyDeviceToHost, s), "status read");
  SW_CUDA(cudaStreamSynchronize(s), "status sync");
  if (rescued) {
    int64_t t = 0;
    if (Q->mode == SW_MODE_PACKED)
      for (int64_t q = 0; q < Q->nq; ++q) t += w[4 + q];
    *rescued = t;
  }
  if (w[2] == SW_ETIMEOUT) return fail(SW_ETIMEOUT, "a bounded device wait expired");
  return SW_OK;
}

int sw_queries_set_timing(sw_queries *q, int32_t enable) {
  g_err.clear();
  if (!q) return fail(SW_EINVAL, "sw_queries_set_timing: null handle");
  if (enable && !q->ev0) {
    SW_CUDA(cudaEventCreate(&q->ev0), "cudaEventCreate");
    SW_CUDA(cudaEventCreate(&q->ev1), "cudaEventCreate");
  }
  q->timing = enable != 0;
  q->timed = false;
  return SW_OK;
}

int sw_queries_kernel_ms(const sw_queries *q, void *stream, float *ms) {
  g_err.clear();
  if (!q || !ms) return fail(SW_EINVAL, "sw_queries_kernel_ms: null argument");
  if (!q->timing || !q->timed) return fail(SW_EINVAL, "sw_queries_kernel_ms: no timed search");
  SW_CUDA(cudaStreamSynchronize((cudaStream_t)stream), "sync");
  SW_CUDA(cudaEventElapsedTime(ms, q->ev0, q->ev1), "cudaEventElapsedTime");
  return SW_OK;
}

int sw_queries_info(const sw_queries *q, int64_t *h2d_bytes, int64_t *device_bytes, int64_t *n_tasks) {
  g_err.clear();
  if (!q) return fail(SW_EINVAL, "sw_queries_info: null handle");
  if (h2d_bytes) *h2d_bytes = q->h2d_bytes;
  if (device_bytes) *device_bytes = (int64_t)q->bytes;
  if (n_tasks) *n_tasks = q->n_tasks;
  return SW_OK;
}

int sw_search(const sw_db *db, const uint8_t *queries, const int64_t *q_offsets, int64_t n_queries,
              const int8_t *submat, int32_t gap_open, int32_t gap_extend, int32_t mode, int32_t *scores_out,
              void *stream) {
  g_err.clear();
  if (!db) return fail(SW_EINVAL, "sw_search: null database");
  if (n_queries > 0 && db->n > 0 && !scores_out) return fail(SW_EINVAL, "sw_search: null scores");
  sw_queries *Q = nullptr;
  int rc = sw_queries_prepare(db, queries, q_offsets, n_queries, submat, gap_open, gap_extend, mode, 0, stream, &Q);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t count = n_queries * db->n;
  int32_t *dst = scores_out;
  void *tmp = nullptr;
  const bool dev = count > 0 && is_device_ptr(scores_out);
  if (count > 0 && !dev) {
    cudaError_t e = cudaMallocAsync(&tmp, 4 * count, s);
    if (e != cudaSuccess) {
      sw_queries_free(Q);
      return cuda_fail(e, "sw_search: score buffer");
    }
    dst = (int32_t *)tmp;
  }
  rc = count > 0 ? sw_search_prepared(db, Q, dst, stream) : SW_OK;
  if (rc == SW_OK && count > 0 && !dev) {
    cudaError_t e = cudaMemcpyAsync(scores_out, dst, 4 * count, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) rc = cuda_fail(e, "sw_search: score copy");
  }
  if (rc == SW_OK) rc = sw_queries_status(Q, stream, nullptr);
  if (tmp) cudaFreeAsync(tmp, s);
  std::string keep = g_err;
  sw_queries_free(Q);
  g_err = keep;
  return rc;
}

}  // extern "C"
