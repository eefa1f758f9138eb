// sw_traceback: one optimal local alignment per hit, on the traceback kernels
// (k_trace.cu).
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <vector>

#include "host_pool.h"
#include "internal.h"
#include "../../include/swgb.h"

namespace swgb {
namespace {

inline int64_t tr_round_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

int tr_fail(int code, const char *fmt, long long a = 0, long long b = 0) {
  char buf[256];
  snprintf(buf, sizeof buf, fmt, a, b);
  return set_last_error(code, buf);
}

int tr_cuda(cudaError_t e, const char *what) {
  char buf[256];
  snprintf(buf, sizeof buf, "sw_traceback: %s: %s", what, cudaGetErrorString(e));
  return set_last_error(e == cudaErrorMemoryAllocation ? SW_ENOMEM : SW_ECUDA, buf);
}

struct TraceScratch {
  void *block = nullptr;
  cudaStream_t s = nullptr;
  ~TraceScratch() {
    if (block) {
      cudaFreeAsync(block, s);
      cudaStreamSynchronize(s);
    }
  }
};

}  // namespace
}  // namespace swgb

using namespace swgb;

extern "C" int sw_traceback(const sw_db *db, const uint8_t *queries, const int64_t *q_offsets, int64_t n_queries,
                            const sw_hit *hits, int64_t n_hits, const int8_t *submat, int32_t gap_open,
                            int32_t gap_extend, sw_alignment *out, uint8_t *ops, int64_t ops_capacity,
                            void *stream) {
  clear_last_error();
  if (!db) return tr_fail(SW_EINVAL, "sw_traceback: null database");
  if (n_hits < 0 || n_queries < 0) return tr_fail(SW_EINVAL, "sw_traceback: negative count");
  if (n_hits == 0) return SW_OK;
  if (!hits || !out || !q_offsets || !submat) return tr_fail(SW_EINVAL, "sw_traceback: null argument");
  if (q_offsets[0] != 0) return tr_fail(SW_EINVAL, "sw_traceback: q_offsets[0] must be 0");
  for (int64_t i = 0; i < n_queries; ++i)
    if (q_offsets[i + 1] < q_offsets[i]) return tr_fail(SW_EINVAL, "sw_traceback: offsets decrease at %lld", i);
  if (q_offsets[n_queries] > 0 && !queries) return tr_fail(SW_EINVAL, "sw_traceback: null queries");
  for (int64_t i = 0; i < q_offsets[n_queries]; ++i)
    if (queries[i] >= kAlphabet) return tr_fail(SW_EINVAL, "sw_traceback: residue code %lld >= 20", queries[i]);
  int smin = 127, smax = -128;
  for (int i = 0; i < kAlphabet * kAlphabet; ++i) {
    smin = std::min<int>(smin, submat[i]);
    smax = std::max<int>(smax, submat[i]);
  }
  if (smin < -64 || smax > 63) return tr_fail(SW_EINVAL, "sw_traceback: submat entries must lie in [-64, 63]");
  if (gap_open < 0 || gap_extend < 0 || (int64_t)gap_open + 2 * (int64_t)gap_extend > 1024)
    return tr_fail(SW_EINVAL, "sw_traceback: gap penalties out of range (%lld, %lld)", gap_open, gap_extend);
  const int64_t ndb = db_view(db).n;

  // per-hit layout: direction nibbles, operations
  const int chunk = trace_rows_per_chunk();
  std::vector<TraceHit> th((size_t)n_hits);
  int64_t dir_bytes = 0, strip_entries = 0, ops_bytes = 0;
  int max_chunks = 1;
  for (int64_t h = 0; h < n_hits; ++h) {
    const int32_t qi = hits[h].query, ti = hits[h].target;
    if (qi < 0 || qi >= n_queries) return tr_fail(SW_EINVAL, "sw_traceback: hit %lld: query index %lld out of range", h, qi);
    if (ti < 0 || ti >= ndb) return tr_fail(SW_EINVAL, "sw_traceback: hit %lld: target index %lld out of range", h, ti);
    const int64_t pos = db_sorted_pos(db, ti);
    TraceHit &x = th[h];
    x.qoff = q_offsets[qi];
    x.m = (int32_t)(q_offsets[qi + 1] - q_offsets[qi]);
    x.toff = db_sorted_off(db, pos);
    x.n = db_sorted_len(db, pos);
    x.npad = db_sorted_npad(db, pos);
    x.mrow = (int32_t)std::max<int64_t>(chunk, tr_round_up(x.m, chunk));
    x.dir_off = dir_bytes;
    x.strip_off = strip_entries;
    x.ops_off = ops_bytes;
    strip_entries += tr_round_up(x.npad, 32);
    dir_bytes += tr_round_up((int64_t)x.mrow * x.npad / 2, 256);
    ops_bytes += (int64_t)x.m + x.n;
    max_chunks = std::max(max_chunks, x.mrow / chunk);
  }
  if (ops_bytes > ops_capacity)
    return tr_fail(SW_EINVAL, "sw_traceback: ops buffer holds %lld bytes, the hits need %lld", ops_capacity,
                   ops_bytes);
  if (ops_bytes > 0 && !ops) return tr_fail(SW_EINVAL, "sw_traceback: null ops");

  const int64_t b_q = tr_round_up(std::max<int64_t>(q_offsets[n_queries], 1), 256);
  const int64_t b_sub = 512, b_hits = tr_round_up((int64_t)sizeof(TraceHit) * n_hits, 256);
  const int64_t b_res = tr_round_up((int64_t)sizeof(TraceResult) * n_hits, 256);
  const int64_t b_ops = tr_round_up(std::max<int64_t>(ops_bytes, 1), 256);
  const int64_t b_strip = tr_round_up(strip_entries * (int64_t)sizeof(uint2), 256);
  const int64_t bytes = b_q + b_sub + b_hits + b_res + b_strip + b_ops + dir_bytes;
  cudaStream_t s = (cudaStream_t)stream;
  TraceScratch sc;
  sc.s = s;
  cudaError_t e = pool_alloc(&sc.block, (size_t)bytes, s);
  if (e != cudaSuccess) {
    sc.block = nullptr;
    return tr_cuda(e, "device allocation");
  }
  uint8_t *p = (uint8_t *)sc.block;
  TraceArgs a{};
  uint8_t *d_q = p;
  int8_t *d_sub = (int8_t *)(d_q + b_q);
  TraceHit *d_hits = (TraceHit *)((uint8_t *)d_sub + b_sub);
  TraceResult *d_res = (TraceResult *)((uint8_t *)d_hits + b_hits);
  uint2 *d_strip = (uint2 *)((uint8_t *)d_res + b_res);
  uint8_t *d_ops = (uint8_t *)d_strip + b_strip;
  uint8_t *d_dirs = d_ops + b_ops;
  a.qres = d_q;
  a.tres = db_view(db).res;
  a.submat = d_sub;
  a.hits = d_hits;
  a.nhits = (int32_t)n_hits;
  a.dirs = d_dirs;
  a.ops = d_ops;
  a.results = d_res;
  a.strips = d_strip;
  a.sc.go = gap_open + gap_extend;
  a.sc.ge = gap_extend;
  a.sc.pad = std::min(0, smin);
  a.sc.maxp = std::max(0, smax);
  a.sc.thresh = 32767 - a.sc.maxp;

  if (q_offsets[n_queries] > 0) e = cudaMemcpyAsync(d_q, queries, q_offsets[n_queries], cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_sub, submat, 400, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_hits, th.data(), sizeof(TraceHit) * n_hits, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return tr_cuda(e, "upload");
  if ((e = launch_trace(a, trace_warps(max_chunks), s)) != cudaSuccess) return tr_cuda(e, "traceback kernels");
  std::vector<TraceResult> res((size_t)n_hits);
  e = cudaMemcpyAsync(res.data(), d_res, sizeof(TraceResult) * n_hits, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && ops_bytes > 0) e = cudaMemcpyAsync(ops, d_ops, ops_bytes, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return tr_cuda(e, "results");
  for (int64_t h = 0; h < n_hits; ++h)
    if (res[h].n_ops < 0) return tr_fail(SW_ETIMEOUT, "sw_traceback: hit %lld: a bounded device wait expired", h);
  for (int64_t h = 0; h < n_hits; ++h) {
    sw_alignment &o = out[h];
    o.score = res[h].score;
    o.q_begin = res[h].begin_i;
    o.q_end = res[h].end_i;
    o.t_begin = res[h].begin_j;
    o.t_end = res[h].end_j;
    o.n_ops = res[h].n_ops;
    o.ops_offset = th[h].ops_off;
  }
  return SW_OK;
}
