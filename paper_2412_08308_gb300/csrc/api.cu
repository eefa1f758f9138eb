// C-ABI entry points (include/swgb.h): database packing, query planning and the
// search pipeline (profile -> DP kernels -> overflow rescue), all on one GPU.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <limits>
#include <memory>
#include <mutex>
#include <tuple>
#include <numeric>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/swgb.h"
#include "host_pool.h"
#include "internal.h"

using namespace swgb;

namespace {

// NVTX range around the host-side enqueue of one stage of a search (profile,
// DP kernels, rescue), for timeline tools; free when no tool is attached.
struct StageRange {
  explicit StageRange(const char *name) { nvtxRangePushA(name); }
  ~StageRange() { nvtxRangePop(); }
};

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

// transposed jobs: rows per lane, and each lane's rows as two half-chains a
// column apart or not
constexpr int kTrackRows = 16;
constexpr bool kTrackSplit = false;
// packed mode: the solo queries' profiles hold 32-bit entries, so that the
// two-sequence form pairs them by a multiply-add on the FMA pipe instead of
// a byte shuffle on the ALU pipe (the int32 rescue reads the same entries)
constexpr bool kWideSolo = true;


int sm_count(int dev) {
  int n = 0;
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n > 0 ? n : 1;
}

// Launch occupancies depend only on the device, the kernel and its launch
// shape, so each is asked of the runtime once per process (the query, and the
// shared-memory attribute it sets, cost tens of microseconds per plan).
// kind: 0 inter-task (a = R, b = form), 1 band-stream (a = R), 2 transposed
// (a = R, b = split).  Failures (0) are not kept.
int cached_occupancy(int kind, int a, int b, int threads, size_t smem) {
  static std::mutex mu;
  static std::map<std::tuple<int, int, int, int, int, size_t>, int> memo;
  int dev = 0;
  cudaGetDevice(&dev);
  const auto key = std::make_tuple(dev, kind, a, b, threads, smem);
  {
    std::lock_guard<std::mutex> lock(mu);
    auto it = memo.find(key);
    if (it != memo.end()) return it->second;
  }
  const int n = kind == 0 ? inter_max_ctas_per_sm(a, b, threads, smem)
                : kind == 1 ? band_max_ctas_per_sm(a)
                            : track_max_ctas_per_sm(a, b != 0);
  if (n > 0) {
    std::lock_guard<std::mutex> lock(mu);
    memo[key] = n;
  }
  return n;
}

// The stream-ordered pool that every query batch's device block comes from,
// one per device, created on first use: freed blocks stay reserved up to
// 1 GiB, so that planning a batch after another does not map fresh memory
// (the default pool returns it at every synchronisation: ~0.1-0.2 ms per
// plan).  Its own pool, so that the process's default pool keeps its settings.
cudaError_t batch_pool(cudaMemPool_t *pool) {
  static std::mutex mu;
  static std::map<int, cudaMemPool_t> pools;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  auto it = pools.find(dev);
  if (it != pools.end()) {
    *pool = it->second;
    return cudaSuccess;
  }
  cudaMemPoolProps props{};
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = dev;
  cudaMemPool_t p = nullptr;
  e = cudaMemPoolCreate(&p, &props);
  if (e != cudaSuccess) return e;
  uint64_t keep = (uint64_t)1 << 30;
  e = cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
  if (e != cudaSuccess) {
    cudaMemPoolDestroy(p);
    return e;
  }
  pools[dev] = p;
  *pool = p;
  return cudaSuccess;
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

// --- the database in row tracks (transposed jobs, k_band.cu) ----------------
// Sequences (sorted order, longest first), padded to whole lanes of tR rows,
// go to the 16-bit tracks (f = 0; two tracks share each word) when their
// length is at most `cut`, else to int32 tracks (f = 1).  A sequence longer
// than a band (32 tR rows) gets a track of its own, whose bands run as a
// pipeline; the others are packed into one-band tracks without crossing a
// band boundary (each into the first of the last 64 open tracks with room),
// so those bands depend on no other band.  Empty sequences score 0 without a
// lane.
struct TrackSeg {
  int32_t pos, row0, rows, bin;  // sequence, first row in its track, rows (whole lanes), track
};
struct TrackBins {
  std::vector<TrackSeg> seg[2];
  std::vector<int32_t> used[2];  // rows of each track
};
// a pipeline of bands: one int32 track, or two 16-bit tracks sharing words
struct TrackPipe {
  int32_t packed, nb, lane0;
};

void bin_tracks(const std::vector<int32_t> &len, int tR, int32_t cut, TrackBins &b) {
  const int32_t kRows = 32 * tR;  // rows per band
  for (int f = 0; f < 2; ++f) {
    b.seg[f].clear();
    b.used[f].clear();
  }
  for (size_t k = 0; k < len.size(); ++k) {
    if (len[k] == 0) continue;
    const int f = len[k] <= cut ? 0 : 1;
    const int32_t rows = (int32_t)round_up(len[k], tR);
    std::vector<int32_t> &U = b.used[f];
    if (rows > kRows) {
      b.seg[f].push_back({(int32_t)k, 0, rows, (int32_t)U.size()});
      U.push_back(rows);
      continue;
    }
    size_t i = U.size();
    for (size_t j = U.size() > 64 ? U.size() - 64 : 0; j < U.size(); ++j)
      if (U[j] <= kRows - rows) {
        i = j;
        break;
      }
    if (i == U.size()) U.push_back(0);
    b.seg[f].push_back({(int32_t)k, U[i], rows, (int32_t)i});
    U[i] += rows;
  }
}

// Bands of one query over all pipelines: the tracks ordered by band count
// (longest first), 16-bit ones paired.
int64_t track_bands(const TrackBins &b, int tR) {
  const int32_t kRows = 32 * tR;
  int64_t total = 0;
  for (int f = 0; f < 2; ++f) {
    std::vector<int32_t> nb(b.used[f].size());
    for (size_t t = 0; t < nb.size(); ++t) nb[t] = (b.used[f][t] + kRows - 1) / kRows;
    std::sort(nb.begin(), nb.end(), std::greater<int32_t>());
    for (size_t i = 0; i < nb.size(); i += (f == 0 ? 2 : 1)) total += nb[i];
  }
  return total;
}

// The pipelines (deeper first; 16-bit ones pair consecutive tracks in that
// order) and their lane table: band b, lane l of a pipeline covers rows
// (32 b + l) tR .. + tR - 1 of its track(s); each segment writes its own
// lanes (whole lanes from a lane boundary), the others stay idle.
void lay_tracks(const TrackBins &b, int tR, std::vector<TrackPipe> &pipes, std::vector<TrackLane> &lanes) {
  const int32_t kRows = 32 * tR;
  pipes.clear();
  lanes.clear();
  for (int f = 0; f < 2; ++f) {
    const std::vector<int32_t> &U = b.used[f];
    const int32_t B = (int32_t)U.size();
    auto bands = [&](int32_t t) { return (int32_t)((U[t] + kRows - 1) / kRows); };
    std::vector<int32_t> order(B), base(B), high(B);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int32_t x, int32_t y) { return bands(x) > bands(y); });
    const int32_t step = f == 0 ? 2 : 1;
    for (int32_t i = 0; i < B; i += step) {
      const int32_t ta = order[i], tb = (f == 0 && i + 1 < B) ? order[i + 1] : -1;
      const int32_t nb = std::max(bands(ta), tb >= 0 ? bands(tb) : 1);
      TrackPipe pp{f == 0 ? 1 : 0, nb, (int32_t)lanes.size()};
      base[ta] = pp.lane0;
      high[ta] = 0;
      if (tb >= 0) {
        base[tb] = pp.lane0;
        high[tb] = 1;
      }
      lanes.resize(lanes.size() + 32 * (size_t)nb, TrackLane{-1, 0, -1, 0});
      pipes.push_back(pp);
    }
    for (const TrackSeg &g : b.seg[f]) {
      TrackLane *L = lanes.data() + base[g.bin] + g.row0 / tR;
      for (int32_t k = 0; k < g.rows / tR; ++k) {
        if (high[g.bin]) {
          L[k].pb = g.pos;
          L[k].rb = k * tR;
        } else {
          L[k].pa = g.pos;
          L[k].ra = k * tR;
        }
      }
    }
  }
  std::stable_sort(pipes.begin(), pipes.end(), [](const TrackPipe &x, const TrackPipe &y) { return x.nb > y.nb; });
}

// Row-track layouts a database keeps (built on first use, its lane table on
// the device): at most this many, each with at most this many bytes of lanes;
// other layouts are built for every plan.
constexpr size_t kTrackLayouts = 8;
constexpr int64_t kTrackLayoutBytes = (int64_t)64 << 20;

}  // namespace

struct sw_db {
  int device = 0;
  int64_t n = 0, total = 0;
  DbView view{};
  void *block = nullptr;
  size_t bytes = 0;
  int32_t max_npad = 0;
  double mean_npad = 0;
  std::vector<int32_t> h_npad;  // padded lengths in sorted order
  std::vector<int32_t> h_len;   // true lengths in sorted order
  std::vector<int32_t> h_pos;   // sorted position of each sequence, caller order
  std::vector<int64_t> h_off;   // residue offsets in sorted order
  // device [0, 1, ..., n - 1, n - 1]: the sorted positions of the database
  // units (one sequence, or two consecutive ones in packed mode, the last
  // repeated when n is odd), shared by every query batch
  const int32_t *d_ident = nullptr;
  // per mode (0 int32: one sequence per unit; 1 packed: two), built on first
  // use: the count of units of each padded length / 16 and the prefix sums
  // of the units' lengths, so that planning a batch does not walk every unit
  struct UnitStats {
    std::vector<int64_t> hist, prefix;
  };
  mutable std::mutex stats_mu;
  mutable std::unique_ptr<UnitStats> unit_stats[2];
  const UnitStats &units(bool packed) const {
    std::lock_guard<std::mutex> lock(stats_mu);
    std::unique_ptr<UnitStats> &u = unit_stats[packed ? 1 : 0];
    if (!u) {
      u.reset(new UnitStats());
      const int64_t nu = packed ? (n + 1) / 2 : n;
      u->hist.assign((size_t)max_npad / 16 + 1, 0);
      u->prefix.assign((size_t)nu + 1, 0);
      for (int64_t k = 0; k < nu; ++k) {
        const int32_t len = h_npad[(size_t)std::min<int64_t>(packed ? 2 * k : k, n - 1)];
        ++u->hist[(size_t)len / 16];
        u->prefix[(size_t)k + 1] = u->prefix[(size_t)k] + len;
      }
    }
    return *u;
  }
  // transposed jobs: the database's row tracks for one lane height and one
  // 16-bit / int32 routing (cut), with the lane table on the device, shared
  // by every query batch that plans them
  struct TrackLayout {
    int32_t tR = 0, cut = 0;
    int64_t bands = 0;    // bands of one query over all pipelines
    int64_t n_lanes = 0;
    std::vector<TrackPipe> pipes;
    TrackLane *d_lanes = nullptr;
  };
  mutable std::mutex track_mu;
  mutable std::vector<std::unique_ptr<TrackLayout>> track_layouts;
  // the layout for (tR, cut), built and uploaded on stream s on first use
  // (synchronising s), or nullptr: not kept (too large, too many, called on
  // another device, or a CUDA error) -- the caller then builds it itself
  const TrackLayout *track_layout(int tR, int32_t cut, cudaStream_t s) const {
    std::lock_guard<std::mutex> lock(track_mu);
    for (const std::unique_ptr<TrackLayout> &t : track_layouts)
      if (t->tR == tR && t->cut == cut) return t.get();
    int dev = -1;
    if (track_layouts.size() >= kTrackLayouts || cudaGetDevice(&dev) != cudaSuccess || dev != device) {
      cudaGetLastError();
      return nullptr;
    }
    // at most one lane per tR residues and one more per sequence
    if ((total / tR + n) * (int64_t)sizeof(TrackLane) > kTrackLayoutBytes) return nullptr;
    TrackBins b;
    bin_tracks(h_len, tR, cut, b);
    std::unique_ptr<TrackLayout> t(new TrackLayout());
    t->tR = tR;
    t->cut = cut;
    std::vector<TrackLane> lanes;
    lay_tracks(b, tR, t->pipes, lanes);
    for (const TrackPipe &p : t->pipes) t->bands += p.nb;
    t->n_lanes = (int64_t)lanes.size();
    if (!lanes.empty()) {
      void *d = nullptr;
      cudaError_t e = cudaMalloc(&d, sizeof(TrackLane) * lanes.size());
      if (e == cudaSuccess) e = cudaMemcpyAsync(d, lanes.data(), sizeof(TrackLane) * lanes.size(), cudaMemcpyHostToDevice, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) {
        if (d) cudaFree(d);
        cudaGetLastError();
        return nullptr;
      }
      t->d_lanes = (TrackLane *)d;
    }
    track_layouts.push_back(std::move(t));
    return track_layouts.back().get();
  }
};

struct sw_queries {
  const sw_db *db = nullptr;
  int64_t nq = 0;
  int mode = SW_MODE_PACKED;
  int R = 16, Ri = 16;
  Scoring sc{};
  std::vector<QDesc> qd, qdi;  // inter-task and intra-task plans per query
  std::vector<QDesc> qdp;      // query-track plans (packed mode, inter-task kernel)
  std::vector<TrackChunk> track;  // their chunk descriptors
  int64_t n_units = 0, n_long = 0, n_upos = 0, n_ipos32 = 0;
  int64_t n_tasks = 0, n_itasks = 0, n_itasks32 = 0, n_rtask_cap = 0;
  int64_t npairs = 0, n_ptasks = 0, n_solo = 0, n_single = 0;
  bool inter_may_flag = false;  // some packed inter-task pair can exceed the 16-bit threshold
  int grid = 1, rgrid = 1, igrid = 1, pgrid = 1, threads = 256;
  int solo_form = kFormPacked, rescue_form = kFormInt32;  // forms (with kFormWide) of the solo and rescue launches
  int pbuf_bytes = 0, ipbuf_bytes = 0, ppbuf_bytes = 0;
  int pbuf_count = 2, ppbuf_count = 2;  // profile buffers of the two inter-task launches
  size_t smem = 0, ismem = 0, psmem = 0;
  int32_t gbuf_stride = 0, igbuf_stride = 0;
  int64_t long_stride = 1;
  // device memory (one stream-ordered allocation)
  void *block = nullptr;
  size_t bytes = 0;
  cudaStream_t alloc_stream = nullptr;
  cudaStream_t side = nullptr;  // second stream for the intra-task kernel
  cudaEvent_t fork = nullptr, join = nullptr;
  // third stream: the int32 intra-task launch beside the packed one
  cudaStream_t side2 = nullptr;
  cudaEvent_t join2 = nullptr;
  uint8_t *d_qres = nullptr;
  int8_t *d_submat = nullptr;
  QDesc *d_qd = nullptr, *d_qdi = nullptr, *d_qdp = nullptr;
  TrackChunk *d_track = nullptr;
  Task *d_tasks = nullptr, *d_itasks = nullptr, *d_itasks32 = nullptr, *d_rtasks = nullptr, *d_ptasks = nullptr;
  int32_t *d_ipos32 = nullptr, *d_upos = nullptr;
  uint8_t *d_prof = nullptr;
  int64_t prof_bytes = 0;
  uint2 *d_gbuf = nullptr, *d_igbuf = nullptr;
  int32_t *d_words = nullptr;
  int32_t *d_flag_pos = nullptr, *d_iflag_pos = nullptr;
  // band-stream jobs (small batches): long queries against every unit, the
  // other queries against the long units
  int64_t n_bjobs = 0, n_bands = 0, n_btargets = 0, band_ring_bytes = 0;
  int bgrid = 1, bR = 8;
  bool bone = false;  // band-stream launch limited to one CTA per SM
  // transposed jobs (small batches): database row tracks against each short query
  int64_t n_tjobs = 0, n_tbands = 0, n_tlanes = 0, track_ring_bytes = 0, qt_bytes = 16;
  int tgrid = 1, tR = 16;
  TrackJob *d_tjobs = nullptr;
  int32_t *d_tjob_of = nullptr;
  TrackLane *d_tlanes = nullptr;
  bool tlanes_shared = false;  // d_tlanes is the database's kept lane table, not in the block
  uint8_t *d_qt = nullptr;
  int64_t *d_qt_off = nullptr;
  int32_t *d_qt_npad = nullptr;
  unsigned long long *d_trings = nullptr;
  BandJob *d_bjobs = nullptr;
  int32_t *d_bjob_of = nullptr;
  int2 *d_btpos = nullptr;
  unsigned long long *d_brings = nullptr;
  int64_t h2d_bytes = 0;
  bool timing = false, timed = false;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  cudaGraphExec_t gexec = nullptr;  // captured search (sw_search_graph)
  const sw_db *gdb = nullptr;
  int32_t *gscores = nullptr;
  // word layout: [0] inter counter, [1] inter rescue counter, [2] status, [3] inter rescue tasks,
  // [4] intra (packed) counter, [5] intra (int32) counter, [6] query-pair counter, [7] band counter,
  // (the transposed jobs' counter is word [1], the inter rescue counter, unused in small batches)
  // [8, 8+nq) inter flag counts, [8+nq, 8+2nq) intra flag counts   -- zeroed every search
  // [8+2nq] inter tasks, [9+2nq] intra packed tasks, [10+2nq] intra int32 tasks,
  // [11+2nq] query-pair tasks -- constants
  int64_t zero_words() const { return 8 + 2 * nq; }
};

namespace {

// Lanes per chain for one query at R rows per lane: minimise padded rows x
// steps per column (fill[L], below) x idle lanes, with a small charge per
// chunk for the boundary strip and the CTA barrier.  (Against the measured
// time of the 20-query benchmark with L forced to 4..32, this model is
// proportional to within 1.5 %.)
int choose_lanes(int m, int R, const double *fill, int Lmax = 32) {
  int bestL = 4;
  double best = 1e300;
  for (int L = 4; L <= Lmax; ++L) {
    const int LR = L * R;
    const int C = std::max(1, (m + LR - 1) / LR);
    const double rows = (double)C * LR;
    const int G = 32 / L;
    const double lane_eff = (double)(G * L) / 32.0;
    const double cost = rows * fill[L] / lane_eff * (1.0 + 0.001 * C);
    if (cost < best - 1e-9) {
      best = cost;
      bestL = L;
    }
  }
  return bestL;
}

void free_queries(sw_queries *q) {
  if (!q) return;
  if (q->block) {
    cudaFreeAsync(q->block, q->alloc_stream);
    cudaStreamSynchronize(q->alloc_stream);
  }
  if (q->ev0) cudaEventDestroy(q->ev0);
  if (q->ev1) cudaEventDestroy(q->ev1);
  if (q->gexec) cudaGraphExecDestroy(q->gexec);
  if (q->fork) cudaEventDestroy(q->fork);
  if (q->join) cudaEventDestroy(q->join);
  if (q->side) cudaStreamDestroy(q->side);
  if (q->join2) cudaEventDestroy(q->join2);
  if (q->side2) cudaStreamDestroy(q->side2);
  delete q;
}

}  // namespace

namespace swgb {
const DbView &db_view(const sw_db *db) { return db->view; }
int db_device(const sw_db *db) { return db->device; }
const int32_t *db_ident(const sw_db *db) { return db->d_ident; }
int64_t db_sorted_pos(const sw_db *db, int64_t caller_index) { return db->h_pos[caller_index]; }
int32_t db_sorted_len(const sw_db *db, int64_t pos) { return db->h_len[pos]; }
int32_t db_sorted_npad(const sw_db *db, int64_t pos) { return db->h_npad[pos]; }
int64_t db_sorted_off(const sw_db *db, int64_t pos) { return db->h_off[pos]; }
cudaError_t pool_alloc(void **ptr, size_t bytes, cudaStream_t s) {
  cudaMemPool_t pool = nullptr;
  cudaError_t e = batch_pool(&pool);
  return e == cudaSuccess ? cudaMallocFromPoolAsync(ptr, bytes, pool, s) : e;
}
int set_last_error(int code, const char *msg) { return fail(code, "%s", msg); }
void clear_last_error() { g_err.clear(); }
}  // namespace swgb

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
  db->h_npad = npad;
  db->h_len = slen;
  db->h_off = off;
  db->h_pos.assign(n_seqs, 0);
  for (int64_t k = 0; k < n_seqs; ++k) db->h_pos[order[k]] = (int32_t)k;
  std::vector<uint8_t> packed((size_t)std::max<int64_t>(padded, 16), (uint8_t)kPadCode);
  for (int64_t k = 0; k < n_seqs; ++k)
    if (slen[k]) memcpy(&packed[off[k]], residues + offsets[order[k]], (size_t)slen[k]);

  const size_t b_res = round_up((int64_t)packed.size(), 256);
  const size_t b_off = round_up(8 * std::max<int64_t>(n_seqs, 1), 256);
  const size_t b_i32 = round_up(4 * std::max<int64_t>(n_seqs, 1), 256);
  const size_t b_ident = round_up(4 * (n_seqs + 1), 256);
  db->bytes = b_res + b_off + 3 * b_i32 + b_ident;
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
  db->view.res_bytes = (int64_t)packed.size();
  db->d_ident = (const int32_t *)(p + b_res + b_off + 3 * b_i32);
  std::vector<int32_t> ident((size_t)n_seqs + 1);
  for (int64_t k = 0; k <= n_seqs; ++k) ident[k] = (int32_t)std::max<int64_t>(0, std::min<int64_t>(k, n_seqs - 1));
  e = cudaMemcpyAsync((void *)db->view.res, packed.data(), packed.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && n_seqs) {
    e = cudaMemcpyAsync((void *)db->view.off, off.data(), 8 * n_seqs, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync((void *)db->view.npad, npad.data(), 4 * n_seqs, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync((void *)db->view.len, slen.data(), 4 * n_seqs, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync((void *)db->view.perm, order.data(), 4 * n_seqs, cudaMemcpyHostToDevice, s);
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync((void *)db->d_ident, ident.data(), 4 * ident.size(), cudaMemcpyHostToDevice, s);
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
  for (const std::unique_ptr<sw_db::TrackLayout> &t : db->track_layouts)
    if (t->d_lanes) cudaFree(t->d_lanes);
  delete db;
  return SW_OK;
}

int sw_db_stats(const sw_db *db, int64_t *n_seqs, int64_t *residues, int64_t *device_bytes) {
  g_err.clear();
  if (!db) return fail(SW_EINVAL, "sw_db_stats: null handle");
  if (n_seqs) *n_seqs = db->n;
  if (residues) *residues = db->total;
  if (device_bytes) {
    int64_t b = (int64_t)db->bytes;
    std::lock_guard<std::mutex> lock(db->track_mu);
    for (const std::unique_ptr<sw_db::TrackLayout> &t : db->track_layouts)
      b += t->n_lanes * (int64_t)sizeof(TrackLane);
    *device_bytes = b;
  }
  return SW_OK;
}

namespace {

// a DP task and its modelled cost (tasks are sorted longest first)
struct TW {
  Task t;
  double w;
};

// The planner's large host tables, one set per thread, emptied at the start
// of each plan but keeping their memory.
struct PlanScratch {
  std::vector<BandJob> bjobs;
  std::vector<int32_t> bjob_of;
  std::vector<int2> btpos;
  std::vector<TrackJob> tjobs;
  std::vector<int32_t> tjob_of;
  std::vector<TrackLane> tlanes;
  std::vector<TrackPipe> tpipes;
  TrackBins bins;
  std::vector<uint8_t> stage;  // the plan's upload, laid out like its device block
  std::vector<TW> tw;
  std::vector<Task> tasks;
};

PlanScratch &plan_scratch() {
  static thread_local PlanScratch ps;
  ps.bjobs.clear();
  ps.bjob_of.clear();
  ps.btpos.clear();
  ps.tjobs.clear();
  ps.tjob_of.clear();
  ps.tlanes.clear();
  ps.tpipes.clear();
  ps.tw.clear();
  ps.tasks.clear();
  return ps;
}

}  // namespace

int sw_queries_prepare(const sw_db *db, const uint8_t *queries, const int64_t *q_offsets, int64_t n_queries,
                       const int8_t *submat, int32_t gap_open, int32_t gap_extend, int32_t mode,
                       const sw_options *opts, void *stream, sw_queries **out) {
  g_err.clear();
  if (!out) return fail(SW_EINVAL, "sw_queries_prepare: null output handle");
  *out = nullptr;
  if (!db) return fail(SW_EINVAL, "sw_queries_prepare: null database");
  if (!submat) return fail(SW_EINVAL, "sw_queries_prepare: null submat");
  if (mode != SW_MODE_INT32 && mode != SW_MODE_PACKED) return fail(SW_EINVAL, "sw_queries_prepare: bad mode %d", mode);
  if (gap_open < 0 || gap_extend < 0 || (int64_t)gap_open + 2 * (int64_t)gap_extend > 1024)
    return fail(SW_EINVAL, "sw_queries_prepare: gap penalties out of range (%d, %d)", gap_open, gap_extend);
  sw_options o{};
  if (opts) o = *opts;
  if (o.reserved[0]) return fail(SW_EINVAL, "sw_queries_prepare: reserved option fields must be 0");
  const int bR = o.band_rows ? o.band_rows : 16;
  if (!band_supported_R(bR)) return fail(SW_EINVAL, "sw_queries_prepare: band_rows must be 8 or 16");
  if (o.band_stream < 0 || o.band_stream > 2) return fail(SW_EINVAL, "sw_queries_prepare: band_stream must be 0, 1 or 2");
  if (o.query_pairs != 0 && o.query_pairs != 1) return fail(SW_EINVAL, "sw_queries_prepare: query_pairs must be 0 or 1");
  int R = o.rows_per_lane ? o.rows_per_lane : 24;
  const int Ri = o.intra_rows ? o.intra_rows : 16;
  const int forceL = o.lanes_per_chain;
  const int cutover = o.cutover > 0 ? o.cutover : 2048;
  if (!inter_supported_R(R)) return fail(SW_EINVAL, "sw_queries_prepare: rows_per_lane must be 4, 8, 12, 16 or 24");
  if (Ri != 8 && Ri != 16) return fail(SW_EINVAL, "sw_queries_prepare: intra_rows must be 8 or 16");
  if (forceL && (forceL < 4 || forceL > 32)) return fail(SW_EINVAL, "sw_queries_prepare: lanes_per_chain must be 4..32");
  if (o.cutover < 0) return fail(SW_EINVAL, "sw_queries_prepare: negative cutover");
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
  Q->Ri = Ri;
  const bool packed = mode == SW_MODE_PACKED;
  Scoring &sc = Q->sc;
  sc.go = gap_open + gap_extend;
  sc.ge = gap_extend;
  sc.pad = std::min(0, smin);
  sc.maxp = std::max(0, smax);
  sc.thresh = 32767 - sc.maxp;

  const int sms = sm_count(db->device);
  const int64_t n = db->n;
  const std::vector<int32_t> &npad = db->h_npad;

  // --- units (sorted positions); a unit is long when its first (longest) sequence reaches the cutover
  // (unit u: sorted positions 2u and min(2u + 1, n - 1) in packed mode, u in
  // int32 mode; the database's identity array holds them on the device)
  Q->n_units = packed ? (n + 1) / 2 : n;
  auto unit_seq = [&](int64_t i) { return (int32_t)std::min<int64_t>(i, n - 1); };
  auto unit_len = [&](int64_t u) { return npad[unit_seq(packed ? 2 * u : u)]; };
  // (units are sorted by length, longest first: the long ones are a prefix)
  int64_t n_long = 0, hi = Q->n_units;
  while (n_long < hi) {
    const int64_t mid = (n_long + hi) / 2;
    if (unit_len(mid) >= cutover) n_long = mid + 1;
    else hi = mid;
  }
  Q->n_long = n_long;
  static const sw_db::UnitStats kNoUnits{{0}, {0}};
  const sw_db::UnitStats &ust = n > 0 ? db->units(packed) : kNoUnits;
  int32_t max_short = 16, max_long = 16;
  const double sum_short = n > 0 ? (double)(ust.prefix[(size_t)Q->n_units] - ust.prefix[(size_t)n_long]) : 0.0;
  if (n_long < Q->n_units) max_short = unit_len(n_long);
  if (n_long) max_long = unit_len(0);
  // fill[L]: steps a chain of L lanes spends per real column of a short unit.
  // A pass over a unit of n padded columns takes n + lag steps (lag = L - 1,
  // or 2 L - 1 for the split lanes of the 16-bit forms) rounded up to whole
  // 16-column blocks.  fill for the solo plans of this mode; fillq (below)
  // for the query-pair plans.
  // (padded lengths are multiples of 16 and every long unit is longer than
  // every short one, so the short units' counts are the first bins)
  std::vector<int64_t> len_hist(max_short / kColBlock + 1, 0);
  if (n_long < Q->n_units)
    std::copy(ust.hist.begin(), ust.hist.begin() + std::min(len_hist.size(), ust.hist.size()), len_hist.begin());
  auto make_fill = [&](int form, double *out) {
    for (int L = 0; L <= 32; ++L) {
      const int lag = L > 0 ? inter_chain_lag(R, form, L) : 0;
      double steps = 0;
      for (size_t b = 1; b < len_hist.size(); ++b)
        steps += (double)len_hist[b] * (double)((b * kColBlock + lag + kColBlock - 1) / kColBlock * kColBlock);
      out[L] = sum_short > 0 ? steps / sum_short : 1.0;
    }
  };
  double fill[33];
  make_fill(packed ? kFormPacked : kFormInt32, fill);

  // --- rows per lane and CTA size of the inter-task kernel.  A small batch
  // (few units x queries) cannot fill the GPU with 16-row lanes: halve the
  // rows per lane (twice the lanes, half the per-step dependency chain), and
  // shrink CTAs until the tasks cover every SM twice.
  const int64_t n_short = Q->n_units - n_long;
  auto lanes_needed = [&](int rr) {
    double lanes = 0;
    for (int64_t q = 0; q < n_queries; ++q) {
      const int m = std::max<int>(1, (int)(q_offsets[q + 1] - q_offsets[q]));
      lanes += (double)n_short * (forceL ? forceL : choose_lanes(m, rr, fill));
    }
    return lanes;
  };
  // A small batch is latency-bound: each chain's sweep over its longest
  // sequence is the critical path, multiplied by the number of chunks.  Use
  // the fewest chunks the lanes allow (one chunk of up to 32 lanes) rather
  // than the fewest idle lanes.
  const bool latency_bound = lanes_needed(16) < (double)sms * 2048;
  if (!o.rows_per_lane && latency_bound) R = 8;
  Q->R = R;
  auto pick_lanes = [&](int m, int Lmax) {
    if (forceL) return std::min(forceL, Lmax);
    if (latency_bound) return std::min(Lmax, std::max(4, (m + R - 1) / R));
    return choose_lanes(m, R, fill, Lmax);
  };
  int warps = inter_threads() / 32;
  for (; warps > 2; warps /= 2) {
    int64_t tasks = 0;
    for (int64_t q = 0; q < n_queries; ++q) {
      const int m = std::max<int>(1, (int)(q_offsets[q + 1] - q_offsets[q]));
      const int chains = warps * (32 / pick_lanes(m, 32));
      tasks += (n_short + chains - 1) / chains;
    }
    if (tasks >= 2 * sms) break;
  }
  const int threads = warps * 32;
  Q->threads = threads;
  auto qlen = [&](int64_t q) { return (int32_t)(q_offsets[q + 1] - q_offsets[q]); };
  auto may_flag = [&](int64_t q, int32_t n_upper) {
    return packed && (int64_t)sc.maxp * std::min<int64_t>(qlen(q), n_upper) > sc.thresh;
  };

  // --- small batches: band-stream jobs and transposed jobs (k_band.cu).  In
  // a batch too small to fill the GPU, the longest chains of the inter-task
  // kernel set the time while most SMs idle, so:
  //  - a query of at least two bands (2 x 32 x band_rows rows; 1,024 with the
  //    default 16 rows per lane) runs against every database unit as
  //    pipelines of bands, one warp each: a job is one query and a stream of
  //    units, all its bands sweeping the stream together.  A unit whose pair
  //    with the query could pass the 16-bit range is split into its
  //    sequences in int32; the others keep two sequences per word.  Streams
  //    are cut so that every warp of one launch gets about two jobs' worth
  //    of columns (one unit at least);
  //  - every shorter query runs transposed: the database sequences are the
  //    rows, stacked in row tracks of whole lanes (16 rows; 8 beside
  //    band-stream jobs; 24 when that gives one band per SM sub-partition),
  //    and the query the columns; each band of a track is one warp, several
  //    short sequences share a band, and the bands of a longer one run as a
  //    pipeline.  In packed mode two tracks share each word (their
  //    substitution bytes paired per row), except sequences whose pair with
  //    the longest of these queries could pass the 16-bit range (int32
  //    tracks).
  // The inter- and intra-task kernels are then not used.  If the rings (one
  // entry per column between consecutive bands) do not fit a memory budget,
  // the batch takes the regular plan.
  std::vector<char> band_q(n_queries, 0), track_q(n_queries, 0), small_q(n_queries, 0);
  // (the planner's large tables live in per-thread buffers that keep their
  // memory from one plan to the next: fresh allocations of a few hundred KB
  // each cost their page faults again, ~0.2-0.8 ms per plan)
  PlanScratch &scratch = plan_scratch();
  std::vector<BandJob> &bjobs = scratch.bjobs;
  std::vector<int32_t> &bjob_of = scratch.bjob_of;
  std::vector<int2> &btpos = scratch.btpos;
  std::vector<TrackJob> &tjobs = scratch.tjobs;
  std::vector<int32_t> &tjob_of = scratch.tjob_of;
  std::vector<TrackLane> &tlanes = scratch.tlanes;
  std::vector<int64_t> qt_off(std::max<int64_t>(n_queries, 1), 0);
  std::vector<int32_t> qt_npad(std::max<int64_t>(n_queries, 1), 16);
  bool band_mode = false;
  if (o.band_stream != 1 && (o.band_stream == 2 || latency_bound) && n > 0 && n_queries > 0) {
    const int brows = 32 * bR;
    bool any_band = false, any_track = false;
    for (int64_t q = 0; q < n_queries; ++q) {
      band_q[q] = qlen(q) >= 2 * brows;
      track_q[q] = !band_q[q];
      any_band |= band_q[q] != 0;
      any_track |= track_q[q] != 0;
    }
    const int bmax = any_band ? cached_occupancy(1, bR, 0, 0, 0) : 1;
    int bocc = bmax;
    // transposed jobs beside band-stream jobs take 8-row lanes: twice the
    // bands, each half the work per step, which fill in around the
    // band-stream pipelines (homolog workload 2.29 -> 2.14 ms, A/B medians);
    // alone (one short query) 16-row lanes are faster (0.081 against 0.084 ms)
    const int tRows = any_band ? 8 : kTrackRows;
    int tocc = any_track ? cached_occupancy(2, tRows, kTrackSplit ? 1 : 0, 0, 0) : 1;
    int64_t ring = 0, band = 0, tring = 0, tband = 0, n_tlanes = 0;
    if (bocc > 0 && tocc > 0) {
      // band jobs: each band query against every unit
      struct BList {
        int32_t q, packed, nb;
        std::vector<int2> t;
        std::vector<int32_t> w;  // columns of each unit
        int64_t cols = 0, widest = 0;
      };
      std::vector<BList> lists;
      double total = 0;
      for (int64_t q = 0; q < n_queries; ++q) {
        if (!band_q[q]) continue;
        const int32_t nb = std::max(1, (qlen(q) + brows - 1) / brows);
        BList lp{(int32_t)q, 1, nb, {}, {}, 0}, li{(int32_t)q, 0, nb, {}, {}, 0};
        for (int64_t u = 0; u < Q->n_units; ++u) {
          const int32_t a = unit_seq(packed ? 2 * u : u), b = packed ? unit_seq(2 * u + 1) : a;
          if (packed && !may_flag(q, unit_len(u))) {
            lp.t.push_back(make_int2(a, b));
            lp.w.push_back(std::max(npad[a], npad[b]));
            lp.cols += lp.w.back();
          } else {
            li.t.push_back(make_int2(a, a));
            li.w.push_back(npad[a]);
            li.cols += npad[a];
            if (b != a) {
              li.t.push_back(make_int2(b, b));
              li.w.push_back(npad[b]);
              li.cols += npad[b];
            }
          }
        }
        for (BList *L : {&lp, &li})
          if (!L->t.empty()) {
            total += (double)L->nb * (double)L->cols;
            for (int32_t x : L->w) L->widest = std::max<int64_t>(L->widest, x);
            lists.push_back(std::move(*L));
          }
      }
      // Streams are cut into jobs of about per_warp columns, two jobs per warp
      // of the launch (a warp that finishes early takes a band of the second
      // wave, whose pipeline fill overlaps the first wave's drain).  Units
      // are not cut, so an int32 unit wider than per_warp makes a job that
      // sets the pace of the launch: it runs in bands of half the height
      // (half the work per step; its steps run one after the other), and if
      // its steps, slowed by the other warps that share its SM sub-partition
      // (those of every CTA on the SM, all computing), would outlast the
      // launch's average load, the launch keeps one CTA per SM (a choice
      // only for band heights whose CTAs fit twice on an SM).
      constexpr double kWaves = 2.0;
      const int wpc = band_threads() / 32;  // warps per CTA
      auto per_warp_at = [&](int occ) {
        return std::max<int64_t>(1, (int64_t)std::ceil(total / ((double)sms * occ * wpc * kWaves)));
      };
      if (bocc > 1) {
        const int64_t pw = per_warp_at(bocc);
        double crit = 0;  // steps of the widest oversized int32 unit, in full-height band steps
        for (const BList &L : lists)
          if (!L.packed && L.widest > pw) crit = std::max(crit, 0.5 * (double)L.widest);
        const double warps_per_smsp = (double)bocc * wpc / 4.0;
        const double load = total / ((double)sms * 4.0);  // full-height band steps per SM sub-partition
        if (crit * warps_per_smsp > 1.3 * load) bocc = 1;
      }
      const int64_t per_warp = per_warp_at(bocc);
      for (const BList &L : lists) {
        size_t i = 0;
        while (i < L.t.size()) {
          BandJob j{};
          j.q = L.q;
          j.form = L.packed ? kBandPacked : kBandInt32;
          j.nb = L.nb;
          j.t_begin = (int32_t)btpos.size();
          int64_t cols = 0;
          while (i < L.t.size() && (cols == 0 || cols + L.w[i] <= per_warp)) {
            btpos.push_back(L.t[i]);
            cols += L.w[i];
            ++i;
          }
          j.t_count = (int32_t)(btpos.size() - j.t_begin);
          j.cols = cols;
          // an int32 unit wider than the budget (a long query against a long
          // sequence whose pair could pass the 16-bit range) makes the job
          // that sets the pace of the launch: bands of half the height halve
          // the work of each of its steps, which run one after the other
          if (!L.packed && cols > per_warp) {
            j.form = kBandInt32Half;
            j.nb = std::max(1, (qlen(L.q) + brows / 2 - 1) / (brows / 2));
          }
          bjobs.push_back(j);
        }
      }
      // longest streams first: their bands are handed out first
      std::stable_sort(bjobs.begin(), bjobs.end(), [](const BandJob &x, const BandJob &y) {
        return (int64_t)x.nb * x.cols > (int64_t)y.nb * y.cols;
      });
      for (size_t k = 0; k < bjobs.size(); ++k) {
        bjobs[k].band0 = (int32_t)band;
        bjobs[k].ring0 = ring;
        ring += (int64_t)(bjobs[k].nb - 1) * bjobs[k].cols;
        for (int b = 0; b < bjobs[k].nb; ++b) bjob_of.push_back((int32_t)k);
        band += bjobs[k].nb;
      }

      // transposed jobs: the database in row tracks, each short query as columns
      int32_t mtq = 0;
      int64_t qt = 0;
      int64_t n_track_q = 0;
      for (int64_t q = 0; q < n_queries; ++q) {
        if (!track_q[q]) continue;
        ++n_track_q;
        mtq = std::max(mtq, qlen(q));
        qt_npad[q] = (int32_t)std::max<int64_t>(kColBlock, round_up(qlen(q), kColBlock));
        qt_off[q] = qt;
        qt += qt_npad[q];
      }
      Q->qt_bytes = std::max<int64_t>(qt, 16);
      // a sequence takes the 16-bit tracks (packed mode) unless its pair with
      // the longest of these queries could pass the 16-bit range: a length
      // cut that depends on the queries only through that longest one
      const int32_t cut = !packed ? -1
                          : (int64_t)sc.maxp * mtq <= sc.thresh ? std::numeric_limits<int32_t>::max()
                                                                : sc.thresh / sc.maxp;
      // the jobs: each pipeline once per query (deeper pipelines first)
      auto make_jobs = [&](const std::vector<TrackPipe> &pipes) {
        tjobs.clear();
        tjob_of.clear();
        tring = 0;
        tband = 0;
        for (const TrackPipe &pp : pipes)
          for (int64_t q = 0; q < n_queries; ++q) {
            if (!track_q[q]) continue;
            TrackJob j{};
            j.q = (int32_t)q;
            j.packed = pp.packed;
            j.nb = pp.nb;
            j.band0 = (int32_t)tband;
            j.lane0 = pp.lane0;
            j.ring0 = tring;
            tring += (int64_t)(pp.nb - 1) * qt_npad[q];
            for (int32_t b = 0; b < pp.nb; ++b) tjob_of.push_back((int32_t)tjobs.size());
            tband += pp.nb;
            tjobs.push_back(j);
          }
      };
      if (any_track) {
        // one wave of 16-row bands that leaves some SM sub-partitions two
        // bands: 24-row lanes (768-row bands, one CTA of 4 warps per SM) when
        // their bands then fit one per sub-partition -- each band's steps no
        // longer share the issue slots.  One 144-residue query x 2,000
        // proteins, packed: 0.081-0.085 -> 0.066 ms (32-row lanes the same);
        // int32 (twice the bands) and larger databases stay at 16 rows
        // (8,000 proteins: 0.189 ms at 16 rows, 0.228 at 24).  The layouts
        // come from the database's kept ones where it keeps them, so that
        // repeated searches skip the binning and the lane upload.
        TrackBins &bins = scratch.bins;
        TrackBins bins24;
        int tR = tRows;
        const sw_db::TrackLayout *lay = db->track_layout(tR, cut, s);
        if (!lay) bin_tracks(db->h_len, tR, cut, bins);
        const int64_t subparts = 4 * (int64_t)sms;
        const int64_t bands16 =
            (!any_band && tRows == 16) ? (lay ? lay->bands : track_bands(bins, 16)) * n_track_q : 0;
        if (bands16 > subparts && bands16 <= subparts * tocc) {
          const int occ24 = cached_occupancy(2, 24, 0, 0, 0);
          const sw_db::TrackLayout *lay24 = nullptr;
          int64_t bands24 = 0;
          if (occ24 > 0) {
            lay24 = db->track_layout(24, cut, s);
            if (!lay24) bin_tracks(db->h_len, 24, cut, bins24);
            bands24 = (lay24 ? lay24->bands : track_bands(bins24, 24)) * n_track_q;
          }
          if (occ24 > 0 && bands24 <= subparts && bands24 <= (int64_t)sms * occ24 * (track_threads() / 32)) {
            tR = 24;
            tocc = occ24;
            lay = lay24;
            if (!lay) std::swap(bins, bins24);
          }
        }
        if (lay) {
          make_jobs(lay->pipes);
          Q->d_tlanes = lay->d_lanes;  // the database's (not the batch's block)
          n_tlanes = lay->n_lanes;
        } else {
          lay_tracks(bins, tR, scratch.tpipes, tlanes);
          make_jobs(scratch.tpipes);
          n_tlanes = (int64_t)tlanes.size();
        }
        Q->tR = tR;
      }
      const int64_t kBandRingBudget = (int64_t)4 << 30;
      band_mode = 8 * (ring + tring) <= kBandRingBudget && band + tband < ((int64_t)1 << 30) &&
                  n_tlanes < ((int64_t)1 << 31);
      if (band_mode) {
        Q->n_bjobs = (int64_t)bjobs.size();
        Q->n_bands = band;
        Q->n_btargets = (int64_t)btpos.size();
        Q->band_ring_bytes = 8 * ring;
        Q->bR = bR;
        Q->bgrid = (int)std::max<int64_t>(1, std::min<int64_t>((band + band_threads() / 32 - 1) / (band_threads() / 32),
                                                               (int64_t)sms * bocc));
        Q->bone = bocc == 1 && bmax > 1;
        Q->n_tjobs = (int64_t)tjobs.size();
        Q->n_tbands = tband;
        Q->n_tlanes = n_tlanes;
        Q->tlanes_shared = Q->d_tlanes != nullptr;
        Q->track_ring_bytes = 8 * tring;
        Q->tgrid = (int)std::max<int64_t>(1, std::min<int64_t>((tband + track_threads() / 32 - 1) / (track_threads() / 32),
                                                               (int64_t)sms * tocc));
        for (int64_t q = 0; q < n_queries; ++q) small_q[q] = band_q[q] || track_q[q];
      }
    }
    if (!band_mode) {
      std::fill(band_q.begin(), band_q.end(), 0);
      std::fill(track_q.begin(), track_q.end(), 0);
      bjobs.clear();
      bjob_of.clear();
      btpos.clear();
      tjobs.clear();
      tjob_of.clear();
      tlanes.clear();
      Q->d_tlanes = nullptr;
    }
  }

  // --- query tracks (packed mode).  Two queries share one chain, one per
  // 16-bit half: the database residue of a column is common to both, so one
  // 32-bit profile word per row feeds both halves and the residue-pair byte
  // shuffle of the two-sequence form disappears.  Each half runs a track of
  // queries laid end to end chunk by chunk, so queries of different lengths
  // share chains without idle rows (greedy longest-first packing into
  // balanced tracks).  Only queries that cannot pass the 16-bit threshold
  // against the short database units join tracks (the form has no rescue
  // pass); the others keep the two-sequence form.
  const int64_t s0 = packed ? std::min<int64_t>(n, 2 * n_long) : n_long;  // first short sequence
  Q->n_single = n - s0;
  std::vector<int32_t> in_track(n_queries, 0), elig;
  if (packed && o.query_pairs == 0 && n_queries >= 2 && Q->n_single > 0) {
    for (int64_t q = 0; q < n_queries; ++q)
      if (!may_flag(q, max_short) && !small_q[q]) elig.push_back((int32_t)q);
    if (elig.size() < 2) elig.clear();
  }
  for (int32_t q : elig) in_track[q] = 1;
  // Two ways to lay the eligible queries out, priced with the same model as
  // choose_lanes (padded rows x steps per column / lane use, the two halves of
  // a plan running max(track) chunks), the cheaper one kept:
  //  - grouped tracks: the queries sorted by length and cut into K consecutive
  //    groups, each packed longest first into two balanced tracks.  K grows
  //    with the query count (at least 8 queries per plan keep the tracks
  //    balanced) and so that every resident CTA sees several tiles;
  //  - pairs: neighbours in length order whose shorter one has at least 3/4
  //    of the longer one's rows share a plan (one query per track); the
  //    others keep the two-sequence form (two database sequences per chain;
  //    pairing their scores costs a seventh instruction per word, priced as
  //    7/6 of the query-pair form's time per cell).
  // Each plan has its own lanes per chain.  (Many queries of similar length
  // favour pairs: each pair's L fits its length; few queries of spread-out
  // lengths favour tracks: no idle half.)
  auto chunks_of = [&](int32_t q, int L) { return std::max(1, (qlen(q) + L * R - 1) / (L * R)); };
  double fillq[33];
  make_fill(kFormQPair, fillq);
  // best L for a group packed into two tracks, and its modelled cost
  auto plan_group = [&](const std::vector<int32_t> &grp, std::vector<int32_t> *tr, int *Lout) {
    auto pack = [&](int L, std::vector<int32_t> *out) {
      int64_t load[2] = {0, 0};
      for (int32_t q : grp) {
        const int t = load[1] < load[0] ? 1 : 0;
        if (out) out[t].push_back(q);
        load[t] += chunks_of(q, L);
      }
      return std::max(load[0], load[1]);
    };
    auto cost_of = [&](int L) {
      const double eff = (double)((32 / L) * L) / 32.0;
      return (double)pack(L, nullptr) * L * R * fillq[L] / eff * (1.0 + 0.001 * (double)pack(L, nullptr) /
                                                                          std::max<size_t>(1, grp.size()) * 2);
    };
    int Lp = 4;
    if (forceL) {
      Lp = forceL;
    } else if (latency_bound) {
      int mmax = 1;
      for (int32_t q : grp) mmax = std::max(mmax, qlen(q));
      Lp = std::min(32, std::max(4, (mmax + R - 1) / R));
    } else {
      double best = 1e300;
      for (int L = 4; L <= 32; ++L) {
        const double c = cost_of(L);
        if (c < best - 1e-9) {
          best = c;
          Lp = L;
        }
      }
    }
    if (tr) pack(Lp, tr);
    if (Lout) *Lout = Lp;
    return cost_of(Lp);
  };
  auto solo_cost = [&](int32_t q) {  // two-sequence form: half the columns, 7/6 the instructions per word
    double best = 1e300;
    for (int L = 4; L <= 32; ++L) {
      const int C = chunks_of(q, L);
      const double eff = (double)((32 / L) * L) / 32.0;
      best = std::min(best, (double)C * L * R * fill[L] / eff * (1.0 + 0.001 * C));
    }
    return best * 7.0 / 12.0;
  };
  std::vector<std::vector<int32_t>> tracks;  // 2 per plan
  std::vector<int> plan_L;
  if (!elig.empty()) {
    std::vector<int32_t> ord = elig;
    std::stable_sort(ord.begin(), ord.end(), [&](int32_t x, int32_t y) { return qlen(x) > qlen(y); });
    const int64_t ne = (int64_t)ord.size();
    // grouped tracks
    std::vector<std::vector<int32_t>> tA;
    std::vector<int> LA;
    double costA = 0;
    {
      const int64_t tiles8 = std::max<int64_t>(1, (Q->n_single + warps * 4 - 1) / (warps * 4));
      int64_t K = std::max<int64_t>((8 * 2 * (int64_t)sms + tiles8 - 1) / tiles8, std::min<int64_t>(8, ne / 8));
      K = std::max<int64_t>(1, std::min<int64_t>(K, ne / 2));
      for (int64_t p = 0; p < K; ++p) {
        std::vector<int32_t> grp(ord.begin() + ne * p / K, ord.begin() + ne * (p + 1) / K);
        std::vector<int32_t> tr[2];
        int Lp = 4;
        costA += plan_group(grp, tr, &Lp);
        tA.push_back(tr[0]);
        tA.push_back(tr[1]);
        LA.push_back(Lp);
      }
    }
    // pairs
    std::vector<std::vector<int32_t>> tB;
    std::vector<int> LB;
    std::vector<int32_t> soloB;
    double costB = 0;
    for (int64_t i = 0; i < ne; ++i) {
      const int32_t x = ord[i];
      if (i + 1 < ne && 4 * (int64_t)qlen(ord[i + 1]) >= 3 * (int64_t)qlen(x)) {
        std::vector<int32_t> grp{x, ord[i + 1]}, tr[2];
        int Lp = 4;
        costB += plan_group(grp, tr, &Lp);
        tB.push_back(tr[0]);
        tB.push_back(tr[1]);
        LB.push_back(Lp);
        ++i;
      } else {
        soloB.push_back(x);
        costB += solo_cost(x);
      }
    }
    if (costB < costA) {
      tracks = tB;
      plan_L = LB;
      for (int32_t q : soloB) in_track[q] = 0;
    } else {
      tracks = tA;
      plan_L = LA;
    }
  }
  Q->n_solo = 0;  // queries with a profile of their own (not in query-pair tracks, not band-stream jobs)
  for (int64_t q = 0; q < n_queries; ++q) Q->n_solo += (in_track[q] || small_q[q]) ? 0 : 1;
  Q->npairs = (int64_t)plan_L.size();  // track plans

  // --- per-query plans and profile layout (queries in a pair get no solo profile)
  Q->qd.resize(n_queries);
  Q->qdi.resize(n_queries);
  int64_t prof = 0;
  int maxc = 16, maxci = 16, maxcp = 16;
  bool chunked = false, ichunked = false;
  for (int64_t q = 0; q < n_queries; ++q) {
    QDesc &d = Q->qd[q];
    d.m = qlen(q);
    d.R = R;
    d.L = pick_lanes(std::max(1, d.m), 32);
    const int LR = d.L * R;
    d.nchunks = std::max(1, (d.m + LR - 1) / LR);
    d.wide = packed && kWideSolo ? 1 : 0;
    d.chunk_stride = (int32_t)round_up((int64_t)profile_slots(d.L) * R * (d.wide ? 4 : 1), 128);
    d.chunk_bytes = (in_track[q] || small_q[q]) ? 0 : kProfRows * d.chunk_stride;
    d.prof_off = prof;
    d.qoff = q_offsets[q];
    prof += (int64_t)d.nchunks * d.chunk_bytes;
    maxc = std::max(maxc, d.chunk_bytes);
    chunked |= d.chunk_bytes > 0 && d.nchunks > 1;
  }
  // track plans: 4-byte entries; every plan uses the chunk layout of 32 lane
  // slots of R words (the most any L needs), so one kernel builds all of
  // them; chunks of all plans in table order, plan p's from track_off
  Q->qdp.resize(Q->npairs);
  Q->track.clear();
  {
    const int32_t stride = (int32_t)round_up(4 * (int64_t)32 * R, 128);
    for (int64_t p = 0; p < Q->npairs; ++p) {
      QDesc &d = Q->qdp[p];
      const int LR = plan_L[p] * R;
      std::vector<TrackChunk> half[2];
      for (int h = 0; h < 2; ++h)
        for (int32_t q : tracks[2 * p + h]) {
          const int C = std::max(1, (qlen(q) + LR - 1) / LR);
          for (int k = 0; k < C; ++k) {
            TrackChunk t{};
            t.qa = q;
            t.ka = k;
            t.flags = (k == 0 ? kStartA : 0) | (k == C - 1 ? kEndA : 0);
            half[h].push_back(t);
          }
        }
      const size_t nc = std::max(half[0].size(), half[1].size());
      d.track_off = (int32_t)Q->track.size();
      for (size_t c = 0; c < nc; ++c) {
        TrackChunk t{};
        t.qa = c < half[0].size() ? half[0][c].qa : -1;
        t.ka = c < half[0].size() ? half[0][c].ka : 0;
        t.qb = c < half[1].size() ? half[1][c].qa : -1;
        t.kb = c < half[1].size() ? half[1][c].ka : 0;
        t.flags = (c < half[0].size() ? half[0][c].flags : 0) | (c < half[1].size() ? half[1][c].flags * 2 : 0);
        t.L = plan_L[p];
        Q->track.push_back(t);
      }
      d.m = (int32_t)nc * LR;
      d.L = plan_L[p];
      d.R = R;
      d.nchunks = (int32_t)nc;
      d.chunk_stride = stride;
      d.chunk_bytes = kProfRows * stride;
      d.prof_off = prof;
      d.qoff = 0;
      prof += (int64_t)nc * d.chunk_bytes;
      maxcp = std::max(maxcp, d.chunk_bytes);
      chunked |= nc > 1;
    }
  }
  if (n_long && !band_mode) {
    const int wmax = intra_threads() / 32;
    for (int64_t q = 0; q < n_queries; ++q) {
      QDesc &d = Q->qdi[q];
      d.m = Q->qd[q].m;
      d.R = Ri;
      const int w = (int)std::min<int64_t>(wmax, std::max<int64_t>(1, (d.m + 32 * Ri - 1) / (32 * Ri)));
      d.L = 32 * w;
      const int LR = d.L * Ri;
      d.nchunks = std::max(1, (d.m + LR - 1) / LR);
      d.chunk_stride = (int32_t)round_up((int64_t)profile_slots(d.L) * Ri, 128);
      d.chunk_bytes = kProfRows * d.chunk_stride;
      d.prof_off = prof;
      d.qoff = q_offsets[q];
      prof += (int64_t)d.nchunks * d.chunk_bytes;
      maxci = std::max(maxci, d.chunk_bytes);
      ichunked |= d.nchunks > 1;
    }
  }
  Q->prof_bytes = std::max<int64_t>(prof, 16);
  Q->pbuf_bytes = (int)round_up(maxc, 128);
  Q->ipbuf_bytes = (int)round_up(maxci, 128);
  Q->ppbuf_bytes = (int)round_up(maxcp, 128);

  // --- tasks, longest first
  std::vector<TW> twi, twi32, twp;
  std::vector<TW> &tw = scratch.tw;
  std::vector<int32_t> ipos32;  // database positions of the int32 intra-task units
  int64_t rcap = 0;
  // (a pair of sequences scores at most max(SM) * min(m, n): a packed lane
  // that cannot pass the threshold needs no rescue pass)
  for (int64_t p = 0; p < Q->npairs; ++p) {  // query pairs x single short sequences
    const QDesc &d = Q->qdp[p];
    const int chains = warps * (32 / d.L);
    for (int64_t i0 = 0; i0 < Q->n_single; i0 += chains) {
      Task t{(int32_t)p, (int32_t)i0, (int32_t)std::min<int64_t>(chains, Q->n_single - i0), 0};
      twp.push_back({t, (double)d.nchunks * d.L * d.R * (npad[s0 + i0] + d.L + 8)});
    }
  }
  std::vector<size_t> tw_runs;  // start of each query's tiles in tw (each run is longest first already)
  for (int64_t q = 0; q < n_queries && Q->n_units > n_long; ++q) {
    if (in_track[q] || small_q[q]) continue;
    const QDesc &d = Q->qd[q];
    const int chains = warps * (32 / d.L);
    tw_runs.push_back(tw.size());
    tw.reserve(tw.size() + (size_t)((Q->n_units - n_long + chains - 1) / chains));
    for (int64_t u0 = n_long; u0 < Q->n_units; u0 += chains) {
      Task t{(int32_t)q, (int32_t)u0, (int32_t)std::min<int64_t>(chains, Q->n_units - u0), 0};
      tw.push_back({t, (double)d.nchunks * d.L * d.R * (unit_len(u0) + d.L + 8)});
    }
    rcap += (n + chains - 1) / chains;
    Q->inter_may_flag |= may_flag(q, max_short);
  }
  // long units: packed intra-task kernel where no lane can saturate, int32
  // otherwise (recomputing a saturated long matrix would cost more than
  // computing it once in int32)
  for (int64_t q = 0; q < n_queries && n_long && !band_mode; ++q) {
    const QDesc &d = Q->qdi[q];
    for (int64_t u = 0; u < n_long; ++u) {
      const double w = (double)d.nchunks * d.L * d.R * (unit_len(u) + d.L);
      if (packed && !may_flag(q, unit_len(u))) {
        twi.push_back({Task{(int32_t)q, (int32_t)u, 1, 0}, w});
        continue;
      }
      const int32_t a = unit_seq(packed ? 2 * u : u);
      const int32_t b = packed ? unit_seq(2 * u + 1) : a;
      twi32.push_back({Task{(int32_t)q, (int32_t)ipos32.size(), 1, 0}, 2 * w});
      ipos32.push_back(a);
      if (b != a) {
        twi32.push_back({Task{(int32_t)q, (int32_t)ipos32.size(), 1, 0}, 2 * w});
        ipos32.push_back(b);
      }
    }
  }
  // all tiles longest first (ties in query order): the stable merge of the
  // queries' runs, each already longest first (units are sorted), in place
  // of a full sort of up to a few hundred thousand tiles
  {
    auto longer = [](const TW &a, const TW &b) { return a.w > b.w; };
    tw_runs.push_back(tw.size());
    while (tw_runs.size() > 2) {
      std::vector<size_t> next;
      for (size_t i = 0; i + 2 < tw_runs.size(); i += 2) {
        std::inplace_merge(tw.begin() + tw_runs[i], tw.begin() + tw_runs[i + 1], tw.begin() + tw_runs[i + 2], longer);
        next.push_back(tw_runs[i]);
      }
      if (tw_runs.size() % 2 == 0) next.push_back(tw_runs[tw_runs.size() - 2]);
      next.push_back(tw_runs.back());
      tw_runs.swap(next);
    }
  }
  std::stable_sort(twi.begin(), twi.end(), [](const TW &a, const TW &b) { return a.w > b.w; });
  std::stable_sort(twi32.begin(), twi32.end(), [](const TW &a, const TW &b) { return a.w > b.w; });
  // track tiles plan by plan (each plan's profile stays hot in L2 while the
  // CTAs stream it), longest tiles first within a plan
  std::stable_sort(twp.begin(), twp.end(),
                   [](const TW &a, const TW &b) { return a.t.q != b.t.q ? a.t.q < b.t.q : a.w > b.w; });
  Q->n_ptasks = (int64_t)twp.size();
  Q->n_tasks = (int64_t)tw.size();
  Q->n_itasks = (int64_t)twi.size();
  Q->n_itasks32 = (int64_t)twi32.size();
  Q->n_ipos32 = (int64_t)ipos32.size();
  Q->long_stride = std::max<int64_t>(1, packed ? 2 * n_long : n_long);
  Q->n_rtask_cap = Q->inter_may_flag ? rcap : 0;

  // --- launch geometry
  // two CTAs per SM need at most (228 KB - 2 x 1 KB reserved) / 2 of shared
  // memory each: drop to one profile buffer where two would not fit
  const size_t kTwoCtaSmem = 113 * 1024;
  Q->pbuf_count = inter_smem_bytes(Q->pbuf_bytes, 2, threads) <= kTwoCtaSmem ? 2 : 1;
  Q->ppbuf_count = inter_smem_bytes(Q->ppbuf_bytes, 2, threads) <= kTwoCtaSmem ? 2 : 1;
  Q->smem = inter_smem_bytes(Q->pbuf_bytes, Q->pbuf_count, threads);
  Q->psmem = inter_smem_bytes(Q->ppbuf_bytes, Q->ppbuf_count, threads);
  Q->ismem = intra_smem_bytes(Q->ipbuf_bytes);
  if (Q->smem > 200 * 1024 || Q->psmem > 200 * 1024 || (n_long && Q->ismem > 220 * 1024)) {
    delete Q;
    return fail(SW_EINVAL, "sw_queries_prepare: profile chunk too large for shared memory");
  }
  Q->solo_form = packed ? (kFormPacked | (kWideSolo ? kFormWide : 0)) : kFormInt32;
  Q->rescue_form = packed && kWideSolo ? (kFormInt32 | kFormWide) : kFormInt32;
  const int occ = cached_occupancy(0, R, Q->solo_form, threads, Q->smem);
  const int occ32 = cached_occupancy(0, R, Q->rescue_form, threads, Q->smem);
  const int occp = Q->n_ptasks ? cached_occupancy(0, R, kFormQPair, threads, Q->psmem) : 1;
  if (occ <= 0 || occ32 <= 0 || occp <= 0) {
    delete Q;
    return fail(SW_ECUDA, "sw_queries_prepare: cannot configure the inter-task kernel");
  }
  if (n_long) {
    cudaError_t ce = configure_intra(Ri, packed);
    if (ce == cudaSuccess && packed) ce = configure_intra(Ri, false);
    if (ce != cudaSuccess) {
      delete Q;
      return cuda_fail(ce, "sw_queries_prepare: cannot configure the intra-task kernel");
    }
  }
  Q->grid = (int)std::max<int64_t>(1, std::min<int64_t>(Q->n_tasks, (int64_t)sms * occ));
  Q->rgrid = std::max(1, sms * occ32);
  Q->pgrid = (int)std::max<int64_t>(1, std::min<int64_t>(Q->n_ptasks, (int64_t)sms * occp));
  Q->igrid = (int)std::max<int64_t>(1, std::min<int64_t>(std::max(Q->n_itasks, Q->n_itasks32), sms));
  const int gslots = std::max(std::max(Q->grid, Q->rgrid), Q->pgrid);
  Q->gbuf_stride = chunked ? (int32_t)round_up(std::max<int32_t>(16, max_short), 16) : 2;
  Q->igbuf_stride = ichunked ? (int32_t)round_up(std::max<int32_t>(16, max_long), 16) : 2;

  // --- device allocation (stream ordered)
  const int64_t nqm = std::max<int64_t>(n_queries, 1);
  const size_t b_qres = round_up(std::max<int64_t>(q_offsets[n_queries], 16), 256);
  const size_t b_sub = 512;
  const size_t b_qd = round_up(sizeof(QDesc) * nqm, 256);
  const size_t b_tasks = round_up(sizeof(Task) * std::max<int64_t>(Q->n_tasks, 1), 256);
  const size_t b_itasks = round_up(sizeof(Task) * std::max<int64_t>(Q->n_itasks, 1), 256);
  const size_t b_itasks32 = round_up(sizeof(Task) * std::max<int64_t>(Q->n_itasks32, 1), 256);
  const size_t b_ipos32 = round_up(4 * std::max<int64_t>((int64_t)ipos32.size(), 1), 256);
  const size_t b_rtasks = round_up(sizeof(Task) * std::max<int64_t>(Q->n_rtask_cap, 1), 256);
  const size_t b_qdp = round_up(sizeof(QDesc) * std::max<int64_t>(Q->npairs, 1), 256);
  const size_t b_track = round_up(sizeof(TrackChunk) * std::max<int64_t>((int64_t)Q->track.size(), 1), 256);
  const size_t b_ptasks = round_up(sizeof(Task) * std::max<int64_t>(Q->n_ptasks, 1), 256);
  const size_t b_prof = round_up(Q->prof_bytes, 256);
  const size_t b_gbuf = round_up((int64_t)gslots * warps * 8 * (int64_t)Q->gbuf_stride * 8, 256);
  // (two intra-task launches at once, packed and int32, each with its strips)
  const int ilaunches = Q->n_itasks && Q->n_itasks32 ? 2 : 1;
  const size_t b_igbuf = round_up((int64_t)ilaunches * Q->igrid * (int64_t)Q->igbuf_stride * 8, 256);
  const size_t b_words = round_up(4 * (12 + 2 * nqm), 256);  // zeroed words + 3 constants
  const size_t b_flag = Q->inter_may_flag ? round_up(4 * nqm * std::max<int64_t>(n, 1), 256) : 0;
  const size_t b_iflag = packed ? round_up(4 * nqm * Q->long_stride, 256) : 0;
  const size_t b_bjobs = round_up((int64_t)sizeof(BandJob) * std::max<int64_t>(Q->n_bjobs, 1), 256);
  const size_t b_bjobof = round_up(4 * std::max<int64_t>(Q->n_bands, 1), 256);
  const size_t b_btpos = round_up((int64_t)sizeof(int2) * std::max<int64_t>(Q->n_btargets, 1), 256);
  const size_t b_brings = Q->n_bjobs ? round_up(std::max<int64_t>(Q->band_ring_bytes, 8), 256) : 0;
  const bool tmode = Q->n_tjobs > 0;
  const size_t b_tjobs = tmode ? round_up((int64_t)sizeof(TrackJob) * Q->n_tjobs, 256) : 0;
  const size_t b_tjobof = tmode ? round_up(4 * Q->n_tbands, 256) : 0;
  const size_t b_tlanes = tmode && !Q->tlanes_shared ? round_up((int64_t)sizeof(TrackLane) * Q->n_tlanes, 256) : 0;
  const size_t b_qt = tmode ? round_up(Q->qt_bytes, 256) : 0;
  const size_t b_qtoff = tmode ? round_up(8 * nqm, 256) : 0;
  const size_t b_qtnpad = tmode ? round_up(4 * nqm, 256) : 0;
  const size_t b_trings = tmode ? round_up(std::max<int64_t>(Q->track_ring_bytes, 8), 256) : 0;
  Q->bytes = b_tjobs + b_tjobof + b_tlanes + b_qt + b_qtoff + b_qtnpad + b_trings + b_qres + b_sub + 2 * b_qd + b_tasks + b_itasks + b_itasks32 + b_ipos32 + b_rtasks + b_prof +
             b_gbuf + b_igbuf + b_words + b_flag + b_iflag + b_qdp + b_ptasks + b_track + b_bjobs + b_bjobof +
             b_btpos + b_brings;
  cudaMemPool_t pool = nullptr;
  cudaError_t e = batch_pool(&pool);
  if (e == cudaSuccess) e = cudaMallocFromPoolAsync(&Q->block, Q->bytes, pool, s);
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
  // the regions the host fills come first, back to back, so that one copy
  // uploads them (with the zeroed status words and their constants)
  Q->d_qres = take(b_qres);
  Q->d_submat = (int8_t *)take(b_sub);
  Q->d_qd = (QDesc *)take(b_qd);
  Q->d_qdi = (QDesc *)take(b_qd);
  Q->d_tasks = (Task *)take(b_tasks);
  Q->d_itasks = (Task *)take(b_itasks);
  Q->d_itasks32 = (Task *)take(b_itasks32);
  Q->d_ipos32 = (int32_t *)take(b_ipos32);
  Q->d_words = (int32_t *)take(b_words);
  Q->d_qdp = (QDesc *)take(b_qdp);
  Q->d_track = (TrackChunk *)take(b_track);
  Q->d_ptasks = (Task *)take(b_ptasks);
  Q->d_bjobs = (BandJob *)take(b_bjobs);
  Q->d_bjob_of = (int32_t *)take(b_bjobof);
  Q->d_btpos = (int2 *)take(b_btpos);
  if (tmode) {
    Q->d_tjobs = (TrackJob *)take(b_tjobs);
    Q->d_tjob_of = (int32_t *)take(b_tjobof);
    if (!Q->tlanes_shared) Q->d_tlanes = (TrackLane *)take(b_tlanes);
    Q->d_qt = take(b_qt);
    Q->d_qt_off = (int64_t *)take(b_qtoff);
    Q->d_qt_npad = (int32_t *)take(b_qtnpad);
  }
  const size_t up_bytes = (size_t)(p - (uint8_t *)Q->block);
  // device-only regions
  Q->d_rtasks = (Task *)take(b_rtasks);
  Q->d_prof = take(b_prof);
  Q->d_gbuf = (uint2 *)take(b_gbuf);
  Q->d_igbuf = (uint2 *)take(b_igbuf);
  Q->d_flag_pos = Q->inter_may_flag ? (int32_t *)take(b_flag) : nullptr;
  Q->d_iflag_pos = packed ? (int32_t *)take(b_iflag) : nullptr;
  Q->d_brings = Q->n_bjobs ? (unsigned long long *)take(b_brings) : nullptr;
  if (tmode) Q->d_trings = (unsigned long long *)take(b_trings);
  Q->d_upos = const_cast<int32_t *>(db->d_ident) + s0;  // the short sequences, in sorted order
  Q->n_upos = n + 1 - s0;

  std::vector<Task> &tasks = scratch.tasks;
  tasks.resize((size_t)Q->n_tasks);
  std::vector<Task> itasks(Q->n_itasks), itasks32(Q->n_itasks32), ptasks(Q->n_ptasks);
  for (int64_t i = 0; i < Q->n_ptasks; ++i) ptasks[i] = twp[i].t;
  for (int64_t i = 0; i < Q->n_tasks; ++i) tasks[i] = tw[i].t;
  for (int64_t i = 0; i < Q->n_itasks; ++i) itasks[i] = twi[i].t;
  for (int64_t i = 0; i < Q->n_itasks32; ++i) itasks32[i] = twi32[i].t;
  const int32_t consts[4] = {(int32_t)Q->n_tasks, (int32_t)Q->n_itasks, (int32_t)Q->n_itasks32,
                             (int32_t)Q->n_ptasks};
  Q->h2d_bytes = q_offsets[n_queries] + 400 + 2 * (int64_t)sizeof(QDesc) * n_queries +
                 (int64_t)sizeof(QDesc) * Q->npairs + (int64_t)sizeof(TrackChunk) * (int64_t)Q->track.size() +
                 (int64_t)sizeof(Task) * (Q->n_tasks + Q->n_itasks + Q->n_itasks32 + Q->n_ptasks) +
                 4 * (int64_t)ipos32.size() + 16 + (int64_t)sizeof(BandJob) * Q->n_bjobs + 4 * Q->n_bands +
                 (int64_t)sizeof(int2) * Q->n_btargets + (int64_t)sizeof(TrackJob) * Q->n_tjobs + 4 * Q->n_tbands +
                 (Q->tlanes_shared ? 0 : (int64_t)sizeof(TrackLane) * Q->n_tlanes) +
                 (tmode ? Q->qt_bytes + 12 * n_queries : 0);
  // stage the host tables at their offsets in the block (the rest zero:
  // padding and the status words) and upload them with one copy
  std::vector<uint8_t> &stage = scratch.stage;
  stage.assign(up_bytes, 0);
  auto put = [&](const void *dst, const void *src, size_t bytes) {
    if (bytes) memcpy(stage.data() + ((const uint8_t *)dst - (const uint8_t *)Q->block), src, bytes);
  };
  put(Q->d_qres, queries, (size_t)q_offsets[n_queries]);
  put(Q->d_submat, submat, 400);
  if (n_queries) put(Q->d_qd, Q->qd.data(), sizeof(QDesc) * n_queries);
  if (n_queries && n_long) put(Q->d_qdi, Q->qdi.data(), sizeof(QDesc) * n_queries);
  put(Q->d_tasks, tasks.data(), sizeof(Task) * Q->n_tasks);
  put(Q->d_itasks, itasks.data(), sizeof(Task) * Q->n_itasks);
  if (Q->n_itasks32) {
    put(Q->d_itasks32, itasks32.data(), sizeof(Task) * Q->n_itasks32);
    put(Q->d_ipos32, ipos32.data(), 4 * ipos32.size());
  }
  if (Q->npairs) {
    put(Q->d_qdp, Q->qdp.data(), sizeof(QDesc) * Q->npairs);
    put(Q->d_track, Q->track.data(), sizeof(TrackChunk) * Q->track.size());
    put(Q->d_ptasks, ptasks.data(), sizeof(Task) * Q->n_ptasks);
  }
  if (Q->n_bjobs) {
    put(Q->d_bjobs, bjobs.data(), sizeof(BandJob) * Q->n_bjobs);
    put(Q->d_bjob_of, bjob_of.data(), 4 * Q->n_bands);
    put(Q->d_btpos, btpos.data(), sizeof(int2) * Q->n_btargets);
  }
  if (tmode) {
    put(Q->d_tjobs, tjobs.data(), sizeof(TrackJob) * Q->n_tjobs);
    put(Q->d_tjob_of, tjob_of.data(), 4 * Q->n_tbands);
    if (!Q->tlanes_shared) put(Q->d_tlanes, tlanes.data(), sizeof(TrackLane) * Q->n_tlanes);
    uint8_t *qtp = stage.data() + (Q->d_qt - (uint8_t *)Q->block);
    memset(qtp, kPadCode, (size_t)Q->qt_bytes);
    for (int64_t q = 0; q < n_queries; ++q)
      if (track_q[q] && qlen(q) > 0) memcpy(qtp + qt_off[q], queries + q_offsets[q], (size_t)qlen(q));
    put(Q->d_qt_off, qt_off.data(), 8 * n_queries);
    put(Q->d_qt_npad, qt_npad.data(), 4 * n_queries);
  }
  put(Q->d_words + Q->zero_words(), consts, sizeof consts);
  e = cudaMemcpyAsync(Q->block, stage.data(), up_bytes, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && ((n_long && !band_mode) || Q->n_bjobs)) {
    e = cudaStreamCreateWithFlags(&Q->side, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&Q->fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&Q->join, cudaEventDisableTiming);
    if (e == cudaSuccess && Q->n_itasks && Q->n_itasks32) {
      e = cudaStreamCreateWithFlags(&Q->side2, cudaStreamNonBlocking);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&Q->join2, cudaEventDisableTiming);
    }
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    free_queries(Q);
    return cuda_fail(e, "sw_queries_prepare: upload");
  }
  *out = Q;
  return SW_OK;
}

int sw_queries_free(sw_queries *q) {
  g_err.clear();
  free_queries(q);
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
  const int threads = Q->threads;
  const int nq = (int)Q->nq;
  int32_t *w = Q->d_words;

  SW_CUDA(cudaMemsetAsync(w, 0, 4 * Q->zero_words(), s), "memset");
  std::unique_ptr<StageRange> stage(new StageRange("swgb: query profiles"));
  if (Q->n_solo)
    SW_CUDA(launch_build_profiles(Q->d_qres, Q->d_qd, nq, Q->d_submat, Q->sc.pad, Q->d_prof, s), "profile kernel");
  if (Q->npairs)
    SW_CUDA(launch_build_track_profiles(Q->d_qres, Q->d_qd, Q->d_qdp, Q->d_track, (int32_t)Q->track.size(),
                                        Q->d_submat, Q->sc.pad, Q->d_prof, s),
            "track profile kernel");
  if (Q->n_itasks || Q->n_itasks32)
    SW_CUDA(launch_build_profiles(Q->d_qres, Q->d_qdi, nq, Q->d_submat, Q->sc.pad, Q->d_prof, s),
            "profile kernel");

  stage.reset(new StageRange("swgb: dynamic programming"));
  // band-stream and transposed jobs add their scores with atomicMax: every score starts at 0
  const bool small = Q->n_bjobs || Q->n_tjobs;
  if (small) SW_CUDA(cudaMemsetAsync(scores_dev, 0, 4 * (size_t)Q->nq * (size_t)db->n, s), "memset");
  const bool band_timing = Q->timing && small;
  if (band_timing) SW_CUDA(cudaEventRecord(Q->ev0, s), "event");

  InterArgs a{};
  a.db = db->view;
  a.unit_pos = db->d_ident;
  a.n_unit_pos = db->n + 1;
  a.prof = Q->d_prof;
  a.prof_bytes = Q->prof_bytes;
  a.out = scores_dev;
  a.out_stride = db->n;
  a.out_size = Q->nq * db->n;
  a.sc = Q->sc;
  a.status = w + 2;

  // long database units: intra-task kernel on the side stream, concurrently;
  // int32 matrices (those that could saturate 16 bits) on a third stream
  // when packed ones exist too, so that neither waits for the other.  In
  // small batches the band-stream jobs take the side stream instead.
  if (Q->side) {
    SW_CUDA(cudaEventRecord(Q->fork, s), "event");
    SW_CUDA(cudaStreamWaitEvent(Q->side, Q->fork, 0), "event");
    if (Q->side2) SW_CUDA(cudaStreamWaitEvent(Q->side2, Q->fork, 0), "event");
    if (Q->n_bjobs) {
      SW_CUDA(cudaMemsetAsync(Q->d_brings, 0, (size_t)Q->band_ring_bytes, Q->side), "memset");
      BandArgs ba{};
      ba.db = db->view;
      ba.tpos = Q->d_btpos;
      ba.jobs = Q->d_bjobs;
      ba.band_job = Q->d_bjob_of;
      ba.nbands = (int32_t)Q->n_bands;
      ba.band_counter = w + 7;
      ba.qres = Q->d_qres;
      ba.qd = Q->d_qd;
      ba.submat = Q->d_submat;
      ba.rings = Q->d_brings;
      ba.out = scores_dev;
      ba.out_stride = db->n;
      ba.out_size = Q->nq * db->n;
      ba.ring_entries = Q->band_ring_bytes / 8;
      ba.n_tpos = Q->n_btargets;
      ba.sc = Q->sc;
      ba.status = w + 2;
      ba.short_int = packed ? 1 : 0;
      SW_CUDA(launch_band(ba, Q->bR, Q->bgrid, Q->bone, Q->side), "band-stream kernel");
    }
    InterArgs b = a;
    b.qd = Q->d_qdi;
    b.pbuf_bytes = Q->ipbuf_bytes;
    b.gbuf = Q->d_igbuf;
    b.gbuf_stride = Q->igbuf_stride;
    b.flag_count = w + 8 + nq;
    b.flag_pos = Q->d_iflag_pos;
    b.flag_stride = Q->long_stride;
    b.flag_size = Q->nq * Q->long_stride;
    if (Q->n_itasks) {  // packed units that cannot saturate
      b.tasks = Q->d_itasks;
      b.n_tasks = w + Q->zero_words() + 1;
      b.task_counter = w + 4;
      SW_CUDA(launch_intra(b, Q->Ri, true, Q->igrid, Q->ismem, Q->side), "intra-task kernel");
    }
    if (Q->n_itasks32) {  // single sequences in int32
      b.unit_pos = Q->d_ipos32;
      b.n_unit_pos = Q->n_ipos32;
      b.tasks = Q->d_itasks32;
      b.n_tasks = w + Q->zero_words() + 2;
      b.task_counter = w + 5;
      cudaStream_t st = Q->side;
      if (Q->side2) {
        st = Q->side2;
        b.gbuf = Q->d_igbuf + (size_t)Q->igrid * Q->igbuf_stride;
      }
      SW_CUDA(launch_intra(b, Q->Ri, false, Q->igrid, Q->ismem, st), "intra-task kernel (int32)");
      if (Q->side2) SW_CUDA(cudaEventRecord(Q->join2, Q->side2), "event");
    }
    SW_CUDA(cudaEventRecord(Q->join, Q->side), "event");
  }

  if (Q->n_tjobs) {  // transposed jobs, on the caller's stream beside the band-stream ones
    SW_CUDA(cudaMemsetAsync(Q->d_trings, 0, (size_t)Q->track_ring_bytes, s), "memset");
    TrackArgs ta{};
    ta.db = db->view;
    ta.lanes = Q->d_tlanes;
    ta.jobs = Q->d_tjobs;
    ta.band_job = Q->d_tjob_of;
    ta.nbands = (int32_t)Q->n_tbands;
    ta.band_counter = w + 1;
    ta.qt = Q->d_qt;
    ta.qt_off = Q->d_qt_off;
    ta.qt_npad = Q->d_qt_npad;
    ta.submat = Q->d_submat;
    ta.rings = Q->d_trings;
    ta.out = scores_dev;
    ta.out_stride = db->n;
    ta.sc = Q->sc;
    ta.status = w + 2;
    ta.n_lanes = Q->n_tlanes;
    ta.ring_entries = Q->track_ring_bytes / 8;
    ta.out_size = Q->nq * db->n;
    ta.qt_bytes = Q->qt_bytes;
    SW_CUDA(launch_track(ta, Q->tR, kTrackSplit, Q->tgrid, s), "band-stream kernel (transposed jobs)");
  }
  if (Q->timing && !band_timing && (Q->n_tasks || Q->n_ptasks)) SW_CUDA(cudaEventRecord(Q->ev0, s), "event");
  if (Q->n_ptasks) {  // query pairs, one short database sequence per chain
    InterArgs p = a;
    p.qd = Q->d_qdp;
    p.track = Q->d_track;
    p.unit_pos = Q->d_upos;
    p.n_unit_pos = Q->n_upos;
    p.tasks = Q->d_ptasks;
    p.n_tasks = w + Q->zero_words() + 3;
    p.task_counter = w + 6;
    p.pbuf_bytes = Q->ppbuf_bytes;
    p.pbuf_count = Q->ppbuf_count;
    p.gbuf = Q->d_gbuf;
    p.gbuf_stride = Q->gbuf_stride;
    p.flag_count = nullptr;
    p.flag_pos = nullptr;
    p.flag_stride = 0;
    SW_CUDA(launch_inter(p, Q->R, kFormQPair, Q->pgrid, threads, Q->psmem, s), "inter-task kernel (query pairs)");
  }
  if (Q->n_tasks) {
    a.qd = Q->d_qd;
    a.tasks = Q->d_tasks;
    a.n_tasks = w + Q->zero_words();
    a.task_counter = w + 0;
    a.pbuf_bytes = Q->pbuf_bytes;
    a.pbuf_count = Q->pbuf_count;
    a.gbuf = Q->d_gbuf;
    a.gbuf_stride = Q->gbuf_stride;
    a.flag_count = w + 8;
    a.flag_pos = Q->d_flag_pos;
    a.flag_stride = db->n;
    a.flag_size = Q->inter_may_flag ? Q->nq * db->n : 0;
    SW_CUDA(launch_inter(a, Q->R, Q->solo_form, Q->grid, threads, Q->smem, s), "inter-task kernel");
  }
  if (Q->timing && !band_timing && (Q->n_tasks || Q->n_ptasks)) {
    SW_CUDA(cudaEventRecord(Q->ev1, s), "event");
    const_cast<sw_queries *>(Q)->timed = true;
  }
  if (Q->n_tasks) {
    if (Q->inter_may_flag) {
      stage.reset(new StageRange("swgb: int32 rescue"));
      SW_CUDA(launch_rescue_tasks(w + 8, Q->d_qd, nq, db->n, threads / 32, 0, Q->d_rtasks, w + 3, w + 1, s),
              "rescue task kernel");
      InterArgs r = a;
      r.unit_pos = Q->d_flag_pos;
      r.n_unit_pos = Q->nq * db->n;
      r.tasks = Q->d_rtasks;
      r.n_tasks = w + 3;
      r.task_counter = w + 1;
      r.flag_count = nullptr;
      r.flag_pos = nullptr;
      SW_CUDA(launch_inter(r, Q->R, Q->rescue_form, Q->rgrid, threads, Q->smem, s), "inter-task rescue kernel");
    }
  }
  if (Q->side) SW_CUDA(cudaStreamWaitEvent(s, Q->join, 0), "event");
  if (Q->side2) SW_CUDA(cudaStreamWaitEvent(s, Q->join2, 0), "event");
  if (band_timing) {
    SW_CUDA(cudaEventRecord(Q->ev1, s), "event");
    const_cast<sw_queries *>(Q)->timed = true;
  }
  return SW_OK;
}

int sw_search_graph(const sw_db *db, sw_queries *Q, int32_t *scores_dev, void *stream) {
  g_err.clear();
  if (!db || !Q) return fail(SW_EINVAL, "sw_search_graph: null handle");
  if (!stream) return fail(SW_EINVAL, "sw_search_graph: stream capture needs a non-default stream");
  if (Q->nq == 0 || db->n == 0) return SW_OK;
  cudaStream_t s = (cudaStream_t)stream;
  if (!Q->gexec || Q->gdb != db || Q->gscores != scores_dev) {
    if (Q->gexec) {
      cudaGraphExecDestroy(Q->gexec);
      Q->gexec = nullptr;
    }
    SW_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture");
    const bool timing = Q->timing;
    Q->timing = false;
    int rc = sw_search_prepared(db, Q, scores_dev, stream);
    Q->timing = timing;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(s, &graph);
    if (rc != SW_OK) {
      if (graph) cudaGraphDestroy(graph);
      return rc;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&Q->gexec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      Q->gexec = nullptr;
      return cuda_fail(e, "cudaGraphInstantiate");
    }
    Q->gdb = db;
    Q->gscores = scores_dev;
  }
  SW_CUDA(cudaGraphLaunch(Q->gexec, s), "cudaGraphLaunch");
  return SW_OK;
}

int sw_queries_status(const sw_queries *Q, void *stream, int64_t *rescued) {
  g_err.clear();
  if (!Q) return fail(SW_EINVAL, "sw_queries_status: null handle");
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<int32_t> w(Q->zero_words());
  SW_CUDA(cudaMemcpyAsync(w.data(), Q->d_words, 4 * w.size(), cudaMemcpyDeviceToHost, s), "status read");
  SW_CUDA(cudaStreamSynchronize(s), "status sync");
  int64_t inter_flags = 0, intra_flags = 0;
  for (int64_t q = 0; q < Q->nq; ++q) {
    inter_flags += w[8 + q];
    intra_flags += w[8 + Q->nq + q];
  }
  if (rescued) *rescued = inter_flags;
  if (w[2] == SW_ETIMEOUT) return fail(SW_ETIMEOUT, "a bounded device wait expired");
  if (w[2] == kStatusSaturated) return fail(SW_ECUDA, "internal error: a query-pair lane passed its bound");
  if (w[2] == kStatusBounds) return fail(SW_ECUDA, "internal error: an index left its buffer (checked build)");
  if (intra_flags) return fail(SW_ECUDA, "internal error: a packed intra-task lane passed its bound");
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

int sw_queries_info(const sw_queries *q, int64_t *h2d_bytes, int64_t *device_bytes, int64_t *n_tasks,
                    int64_t *launches) {
  g_err.clear();
  if (!q) return fail(SW_EINVAL, "sw_queries_info: null handle");
  if (launches) {
    int64_t k = 0;
    if (q->nq > 0 && q->db->n > 0) {
      k = (q->n_solo ? 1 : 0) + (q->npairs ? 1 : 0) + ((q->n_itasks || q->n_itasks32) ? 1 : 0);  // profile builds
      k += (q->n_tasks ? 1 : 0) + (q->n_ptasks ? 1 : 0);  // inter-task kernels
      k += (q->n_tasks && q->inter_may_flag) ? 2 : 0;     // rescue tasks + int32 rescue
      k += (q->n_itasks ? 1 : 0) + (q->n_itasks32 ? 1 : 0);
      k += q->n_bjobs ? 1 : 0;  // band-stream kernel
      k += q->n_tjobs ? 1 : 0;  // transposed jobs
    }
    *launches = k;
  }
  if (h2d_bytes) *h2d_bytes = q->h2d_bytes;
  if (device_bytes) *device_bytes = (int64_t)q->bytes;
  if (n_tasks) *n_tasks = q->n_tasks + q->n_itasks + q->n_itasks32 + q->n_ptasks;
  return SW_OK;
}

int sw_search(const sw_db *db, const uint8_t *queries, const int64_t *q_offsets, int64_t n_queries,
              const int8_t *submat, int32_t gap_open, int32_t gap_extend, int32_t mode, int32_t *scores_out,
              void *stream) {
  g_err.clear();
  if (!db) return fail(SW_EINVAL, "sw_search: null database");
  if (n_queries > 0 && db->n > 0 && !scores_out) return fail(SW_EINVAL, "sw_search: null scores");
  sw_queries *Q = nullptr;
  int rc = sw_queries_prepare(db, queries, q_offsets, n_queries, submat, gap_open, gap_extend, mode, nullptr, stream,
                              &Q);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t count = n_queries * db->n;
  int32_t *dst = scores_out;
  void *tmp = nullptr;
  const bool dev = count > 0 && is_device_ptr(scores_out);
  if (count > 0 && !dev) {
    cudaError_t e = swgb::pool_alloc(&tmp, 4 * count, s);
    if (e != cudaSuccess) {
      free_queries(Q);
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
  free_queries(Q);
  g_err = keep;
  return rc;
}

}  // extern "C"
