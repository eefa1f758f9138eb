// sw_align_pair: the score of one long (query, target) pair, computed by the
// pair-band kernel (k_pair.cu) as a pipeline of query-row bands, one per
// warp, across every warp of every SM.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <vector>

#include "host_pool.h"
#include "internal.h"
#include "../../include/swgb.h"

namespace swgb {
namespace {

inline int64_t round_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

int pair_fail(int code, const char *fmt, long long a = 0, long long b = 0) {
  char buf[256];
  snprintf(buf, sizeof buf, fmt, a, b);
  return set_last_error(code, buf);
}

int pair_cuda(cudaError_t e, const char *what) {
  char buf[256];
  snprintf(buf, sizeof buf, "sw_align_pair: %s: %s", what, cudaGetErrorString(e));
  return set_last_error(e == cudaErrorMemoryAllocation ? SW_ENOMEM : SW_ECUDA, buf);
}

int check_codes(const uint8_t *p, int64_t len, const char *what) {
  char buf[128];
  if (len > 0 && !p) {
    snprintf(buf, sizeof buf, "sw_align_pair: null %s", what);
    return set_last_error(SW_EINVAL, buf);
  }
  for (int64_t i = 0; i < len; ++i)
    if (p[i] >= kAlphabet) {
      snprintf(buf, sizeof buf, "sw_align_pair: %s residue code %d >= 20 at %lld", what, (int)p[i], (long long)i);
      return set_last_error(SW_EINVAL, buf);
    }
  return SW_OK;
}

// Device scratch of one call, released on every exit path.
struct PairScratch {
  void *block = nullptr;
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  ~PairScratch() {
    if (block) {
      cudaFreeAsync(block, s);
      cudaStreamSynchronize(s);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  }
};

}  // namespace
}  // namespace swgb

using namespace swgb;

extern "C" int sw_align_pair(const uint8_t *query, int64_t m, const uint8_t *target, int64_t n,
                             const int8_t *submat, int32_t gap_open, int32_t gap_extend,
                             const sw_pair_options *opts, int32_t *score, float *kernel_ms, void *stream) {
  clear_last_error();
  if (!score) return pair_fail(SW_EINVAL, "sw_align_pair: null score");
  *score = 0;
  if (kernel_ms) *kernel_ms = 0.f;
  if (m < 0 || n < 0) return pair_fail(SW_EINVAL, "sw_align_pair: negative length (%lld, %lld)", m, n);
  if (m >= ((int64_t)1 << 31) || n >= ((int64_t)1 << 31) - 32)
    return pair_fail(SW_EINVAL, "sw_align_pair: sequence too long (%lld, %lld)", m, n);
  if (int rc = check_codes(query, m, "query")) return rc;
  if (int rc = check_codes(target, n, "target")) return rc;
  if (!submat) return pair_fail(SW_EINVAL, "sw_align_pair: null submat");
  int smin = 127, smax = -128;
  for (int i = 0; i < kAlphabet * kAlphabet; ++i) {
    smin = std::min<int>(smin, submat[i]);
    smax = std::max<int>(smax, submat[i]);
  }
  if (smin < -64 || smax > 63) return pair_fail(SW_EINVAL, "sw_align_pair: submat entries must lie in [-64, 63]");
  if (gap_open < 0 || gap_extend < 0 || (int64_t)gap_open + 2 * (int64_t)gap_extend > 1024)
    return pair_fail(SW_EINVAL, "sw_align_pair: gap penalties out of range (%lld, %lld)", gap_open, gap_extend);
  sw_pair_options o{};
  if (opts) o = *opts;
  for (int i = 0; i < 4; ++i)
    if (o.reserved[i]) return pair_fail(SW_EINVAL, "sw_align_pair: reserved option fields must be 0");
  if (o.ring_columns != 0 && (o.ring_columns < 256 || o.ring_columns % kColBlock))
    return pair_fail(SW_EINVAL, "sw_align_pair: ring_columns must be 0 or a multiple of 16 >= 256 (got %lld)",
                     o.ring_columns);
  if (o.band_warps < 0 || o.band_warps > 16)
    return pair_fail(SW_EINVAL, "sw_align_pair: band_warps must be 0..16 (got %lld)", o.band_warps);
  if (o.rows_per_lane != 0 && o.rows_per_lane != 4 && o.rows_per_lane != 8 && o.rows_per_lane != 16 &&
      o.rows_per_lane != 24)
    return pair_fail(SW_EINVAL, "sw_align_pair: rows_per_lane must be 0, 4, 8, 16 or 24 (got %lld)",
                     o.rows_per_lane);
  if (o.max_ctas < 0) return pair_fail(SW_EINVAL, "sw_align_pair: negative max_ctas");
  if (m == 0 || n == 0) return SW_OK;
  // H <= max(SM) * min(m, n); the boundary entries between bands keep H and
  // F + Go in 31 bits each
  if ((int64_t)std::max(0, smax) * std::min(m, n) + (int64_t)gap_open + gap_extend >= ((int64_t)1 << 31))
    return pair_fail(SW_EINVAL, "sw_align_pair: scores could pass 2^31 - 1 - Go (max(SM) %lld x %lld residues)",
                     smax, std::min(m, n));

  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, sms = 1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return pair_cuda(e, "cudaGetDevice");
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);

  // geometry: bands of 32 * R query rows, one warp each; each warp stages its
  // band's profile (21 residue rows) in shared memory
  // Bands in flight are the parallelism, one warp each; the warps of a CTA are
  // the bands per SM, so that every SM gets bands.  Rows per lane 16, or 8
  // when that leaves fewer than 3 bands per SM (more, shorter bands fill the
  // SMs better there, while elsewhere the longer ramp of the band pipeline
  // and the per-column overhead of shorter bands cost more; 4 and 24 rows
  // measured slower on every pair).
  const int R = o.rows_per_lane ? o.rows_per_lane : ((m + 511) / 512 < 3 * (int64_t)sms ? 8 : 16);
  const int64_t B = 32 * (int64_t)R;
  const int64_t nbands64 = (m + B - 1) / B;
  if (nbands64 >= ((int64_t)1 << 31)) return pair_fail(SW_EINVAL, "sw_align_pair: too many bands");
  const int64_t npad = std::max<int64_t>(kColBlock, round_up(n, kColBlock));
  QDesc qd{};
  qd.m = (int32_t)m;
  qd.L = 32;
  qd.R = R;
  qd.nchunks = (int32_t)nbands64;
  qd.chunk_stride = (int32_t)round_up((int64_t)profile_slots(32) * R, 128);
  qd.chunk_bytes = kProfRows * qd.chunk_stride;
  const int pbuf_bytes = (int)round_up(qd.chunk_bytes, 128);
  int warps = (int)std::min<int64_t>(16, std::max<int64_t>(1, (nbands64 + sms - 1) / sms));
  while (warps > 1 && pair_smem_bytes(pbuf_bytes, warps) > 200 * 1024) --warps;
  if (o.band_warps) warps = std::min(warps, o.band_warps);
  const int threads = 32 * warps;
  const size_t smem = pair_smem_bytes(pbuf_bytes, warps);
  if (smem > 200 * 1024) return pair_fail(SW_EINVAL, "sw_align_pair: band profile too large for shared memory");
  const int occ = pair_max_ctas_per_sm(R, threads, smem);
  if (occ <= 0) return pair_fail(SW_ECUDA, "sw_align_pair: cannot configure the pair kernel");
  // every SM gets a CTA (the kernel deals bands to the SMs in turn)
  int64_t grid = std::min<int64_t>(std::max<int64_t>((nbands64 + warps - 1) / warps, std::min<int64_t>(sms, nbands64)),
                                   (int64_t)sms * occ);
  if (o.max_ctas) grid = std::min<int64_t>(grid, o.max_ctas);
  const int64_t gw = grid * warps;
  const int64_t nslots = std::min<int64_t>(nbands64, gw + 1);

  // boundary rings: a band runs at most `window` columns ahead of the band
  // below it, which hands consumed columns back every cons_every blocks (at
  // most an eighth of the ring).  The band below may still be queued behind a
  // band of the same round on its warp, so the first band of a round must be
  // able to finish while each band of the round holds a full ring: rings of
  // at least npad / (warps of the grid) columns, plus the hand-back interval
  // and the lead of a band over the one below.  32,768 columns by default:
  // shorter rings stall the last bands of a round while the band below waits
  // for its warp (7M x 5M: 2,447 GCUPS at 8,192, 2,485 from 16,384 up; 3M x
  // 3M: 2,281 and 2,325 from 32,768 up).
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) free_b = (size_t)1 << 30;
  int64_t window = o.ring_columns ? o.ring_columns : 32768;
  window = std::max<int64_t>(window, round_up(((npad + gw - 1) / gw + 64) * 8 / 7 + 1, kColBlock));
  window = std::min<int64_t>(window, npad);
  const int cons_every = (int)std::max<int64_t>(1, std::min<int64_t>(16, window / kColBlock / 8));

  // device scratch: query, target, matrix, plan, profile, strips, progress, result words
  const size_t b_q = round_up(m, 256), b_t = round_up(npad, 256), b_sub = 512, b_qd = 256;
  const size_t b_prof = round_up(nbands64 * (int64_t)qd.chunk_bytes, 256);
  const size_t b_strip = round_up(nslots * window * (int64_t)sizeof(unsigned long long), 256);
  const size_t b_prog = round_up(4 * nbands64, 256), b_words = 256;
  const size_t bytes = b_q + b_t + b_sub + b_qd + b_prof + b_strip + b_prog + b_words;
  if (bytes > free_b)
    return pair_fail(SW_ENOMEM, "sw_align_pair: needs %lld bytes of device memory, %lld free", (long long)bytes,
                     (long long)free_b);
  PairScratch sc;
  sc.s = s;
  e = pool_alloc(&sc.block, bytes, s);
  if (e != cudaSuccess) {
    sc.block = nullptr;
    return pair_cuda(e, "device allocation");
  }
  uint8_t *p = (uint8_t *)sc.block;
  uint8_t *d_q = p;
  uint8_t *d_t = d_q + b_q;
  int8_t *d_sub = (int8_t *)(d_t + b_t);
  QDesc *d_qd = (QDesc *)((uint8_t *)d_sub + b_sub);
  uint8_t *d_prof = (uint8_t *)d_qd + b_qd;
  unsigned long long *d_strip = (unsigned long long *)(d_prof + b_prof);
  int32_t *d_prog = (int32_t *)((uint8_t *)d_strip + b_strip);  // [nbands] columns consumed
  int32_t *d_words = (int32_t *)((uint8_t *)d_prog + b_prog);  // [0] best, [1] status

  std::vector<uint8_t> tpad((size_t)npad, (uint8_t)kPadCode);
  memcpy(tpad.data(), target, (size_t)n);
  e = cudaMemcpyAsync(d_q, query, (size_t)m, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_t, tpad.data(), (size_t)npad, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_sub, submat, 400, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_qd, &qd, sizeof qd, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_strip, 0, b_strip + b_prog + b_words, s);
  if (e != cudaSuccess) return pair_cuda(e, "upload");

  Scoring scr{};
  scr.go = gap_open + gap_extend;
  scr.ge = gap_extend;
  scr.pad = std::min(0, smin);
  scr.maxp = std::max(0, smax);
  scr.thresh = 32767 - scr.maxp;
  e = launch_build_profiles(d_q, d_qd, 1, d_sub, scr.pad, d_prof, s);
  if (e != cudaSuccess) return pair_cuda(e, "profile kernel");

  PairBandArgs a{};
  a.target = d_t;
  a.npad = (int32_t)npad;
  a.nbands = (int32_t)nbands64;
  a.prof = d_prof;
  a.band_bytes = qd.chunk_bytes;
  a.stride = qd.chunk_stride;
  a.pbuf_bytes = pbuf_bytes;
  a.strips = d_strip;
  a.nslots = (int32_t)nslots;
  a.window = (int32_t)window;
  a.cons_every = cons_every;
  a.cons = d_prog;
  a.best = d_words;
  a.status = d_words + 1;
  a.sc = scr;
  if (kernel_ms) {
    if ((e = cudaEventCreate(&sc.e0)) != cudaSuccess || (e = cudaEventCreate(&sc.e1)) != cudaSuccess)
      return pair_cuda(e, "cudaEventCreate");
    if ((e = cudaEventRecord(sc.e0, s)) != cudaSuccess) return pair_cuda(e, "event");
  }
  e = launch_pair(a, R, (int)grid, threads, smem, s);
  if (e != cudaSuccess) return pair_cuda(e, "pair kernel");
  if (kernel_ms && (e = cudaEventRecord(sc.e1, s)) != cudaSuccess) return pair_cuda(e, "event");
  int32_t words[2] = {0, 0};
  e = cudaMemcpyAsync(words, d_words, sizeof words, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return pair_cuda(e, "result");
  if (words[1] == SW_ETIMEOUT) return pair_fail(SW_ETIMEOUT, "sw_align_pair: a bounded device wait expired");
  if (kernel_ms) cudaEventElapsedTime(kernel_ms, sc.e0, sc.e1);
  *score = words[0];
  return SW_OK;
}
