// Band-stream kernel: long queries, and long database sequences, of small
// batches (Sec. 2.2 Eqs. 1-3; Sec. 3.1 "long kernel"; Fig. 1 intra-sequence
// parallelism), for sm_103a.
//
// In a small batch a long query (thousands of rows) against a few thousand
// database sequences leaves the inter-task kernel one chain per database
// unit, each chain sweeping its unit once per chunk of query rows, chunk
// after chunk: the longest chains set the time while most SMs idle.  Here the
// query's rows are cut into bands of 32 lanes x R rows, one warp each, and
// all bands of a *job* -- a query and a stream of database units -- run as a
// pipeline: the warp of band b sweeps the units of the stream one after the
// other, and reads the bottom row of band b - 1 for each column from a ring
// in global memory as soon as band b - 1 has written it.  A job's stream is
// short enough (a few thousand columns) that many jobs run at once, and every
// unit's cells are spread over all the job's warps instead of one.
//
// Forms: int32 cells, one database sequence per unit (Algorithm 1's
// statements in int32 batches; in 16-bit batches, for the pairs that could
// pass the 16-bit range, the one-operation F chain), or two sequences per
// unit in the 16-bit halves of a word (only for pairs that cannot pass the
// 16-bit range, so no rescue is needed).  A
// lane's R rows form one chain down the column (no split lanes: the pipeline
// lag between consecutive bands is then 31 columns instead of 63, which
// measured faster here, where several bands share each SM sub-partition).
//
// Rings and progress.  Each ring holds one 64-bit entry per column of the
// job's whole stream, zeroed before the launch, and is written once: the
// writer (band b's last lane) stores (H | 1 << 31, F) with one relaxed 64-bit
// store, and the reader (band b + 1, lanes 0..15, a block of 16 columns ahead)
// reloads until bit 31 is set.  H is below 2^31 (int32: bounded by the host;
// 16-bit halves: both halves non-negative, so bit 31 is the high half's sign
// bit, 0).  No band ever waits for a band below it (the rings never wrap), and
// warps take their bands from an atomic counter in order, so every band a
// warp waits on was taken earlier by a warp that is running: the pipeline
// cannot deadlock whatever the launch's residency.  Every wait is bounded.
//
// Scores: each band keeps its running best per unit and adds it to the
// caller-order output with atomicMax (the host zeroes the jobs' output rows
// first); the maximum over the bands is the unit's score.
#include <algorithm>
#include "devutil.cuh"
#include "dp_common.cuh"
#include "internal.h"
#include "../../include/swgb.h"

namespace swgb {
namespace {

// 12 warps, one band at a time each, one CTA per SM with up to 168
// registers a thread (the 512-row bands' profiles take 134 KB of shared
// memory).  Homolog workload, ms per search (packed / int32): 8 warps at 128
// registers (one or two CTAs per SM) 2.14 / 3.43; 10 warps 2.15 / 3.71; 12
// warps 1.95 / 3.31 (2.10 / 3.28 capped at 128 registers); 14 warps 2.33 /
// 3.50; 16 warps 2.37 / 3.25.
constexpr int kBandStreamThreads = 384;
constexpr int kLag = 32 - 1;  // a band's last lane trails its first by 31 columns
constexpr int kSubmatBytes = 512;
// R rows per lane: bands of 32 R query rows; a band's profile is [21][32 lanes
// x R] bytes, followed by its residue slots (2 x 32 B) and boundary slots (2 x
// 16 x 8 B)
template <int R>
constexpr int kProfBytes = kProfRows * 32 * R;
template <int R>
constexpr int kWarpBytes = ((kProfBytes<R> + 320) + 127) / 128 * 128;

// A band's profile in the warp's shared-memory block: byte [c][lane * R + r]
// = SM(Q[row], c) for row = band * 32 R + lane * R + r, the pad value for the
// pad residue (c = 20) and rows past the query's end.
template <int R>
__device__ __forceinline__ void build_band_profile(uint8_t *prof, const int8_t *sm, const uint8_t *q, int m,
                                                   int row0, int lane, int32_t pad) {
  uint8_t codes[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int row = row0 + lane * R + r;
    codes[r] = row < m ? q[row] : (uint8_t)kPadCode;
  }
  for (int c = 0; c < kProfRows; ++c) {
#pragma unroll
    for (int w = 0; w < R / 4; ++w) {
      uint32_t v = 0;
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int code = codes[4 * w + b];
        const int32_t s = (c < kAlphabet && code < kAlphabet) ? (int32_t)sm[code * kAlphabet + c] : pad;
        v |= ((uint32_t)s & 0xffu) << (8 * b);
      }
      *reinterpret_cast<uint32_t *>(prof + c * 32 * R + lane * R + 4 * w) = v;
    }
  }
}

// One band over one database unit (columns sbase .. sbase + npad - 1 of the
// job's stream).  Returns false when a wait expired.
template <int R, int FORM, bool SHORTF>
__device__ __forceinline__ bool band_unit(const BandArgs &a, const uint8_t *__restrict__ prof, uint8_t *ring,
                                          const int lane, const int posA, const int posB, const int64_t sbase,
                                          const unsigned long long *ring_in, unsigned long long *ring_out,
                                          const Consts &cs, Word<FORM> &Sout) {
  using W = Word<FORM>;
  constexpr bool PACKED = FORM == kFormPacked;
  const W H0 = (W)0;
  const W F0 = PACKED ? (W)cs.F0W : (W)0;
  const int npa = a.db.npad[posA];
  const int npb = PACKED ? a.db.npad[posB] : 0;
  const int npad = max(npa, npb);
  const uint8_t *resA = a.db.res + a.db.off[posA];
  const uint8_t *resB = a.db.res + a.db.off[posB];
  constexpr int LAG = kLag;
  const int nblk = (npad + LAG + kColBlock - 1) / kColBlock;
  const int nreal = npad / kColBlock;
  const bool prev = ring_in != nullptr, next = ring_out != nullptr;
  const bool lead = lane == 0;
  const bool tail = lane == 31 && next;
  const int src = lane > 0 ? lane - 1 : lane;

  LaneState<R, FORM> st;
  lane_reset(st, cs);
  W outH = H0, outF = F0, S = (W)0;
  uint32_t outRes = kPadPair;
  uint8_t *rres = ring;                              // [slot][2 seqs][16 B] residue codes
  uint2 *rgb = reinterpret_cast<uint2 *>(ring + 64);  // [slot][16] (H, F) of the band above
  const uint8_t *prow = prof + lane * R;
  bool failed = false;

  auto prefetch = [&](int blk) {
    uint8_t *d = rres + (blk & 1) * 32;
    const int col = blk * kColBlock;
    if (col < npa && in_range(resA + col + 15 - a.db.res, a.db.res_bytes, a.status)) cp_async16(d, resA + col);
    else *reinterpret_cast<uint4 *>(d) = make_uint4(0x14141414u, 0x14141414u, 0x14141414u, 0x14141414u);
    if (PACKED) {
      if (col < npb && in_range(resB + col + 15 - a.db.res, a.db.res_bytes, a.status)) cp_async16(d + 16, resB + col);
      else *reinterpret_cast<uint4 *>(d + 16) = make_uint4(0x14141414u, 0x14141414u, 0x14141414u, 0x14141414u);
    }
    cp_async_commit();
  };
  if (lead) {
    prefetch(0);
    prefetch(1);
  }

  // reading side: the next block to load (lanes 0..15 hold one entry each)
  int64_t rpos = sbase;
  unsigned long long pend = 0ull;
  auto load = [&]() {
    if (lane < kColBlock && in_range(ring_in - a.rings + rpos + lane, a.ring_entries, a.status))
      pend = ld_relaxed_u64(ring_in + rpos + lane);
  };
  // wait until the loaded entries are written, unpack them into `slot`, advance
  auto land = [&](int slot) {
    bool ok = lane >= kColBlock || (pend >> 31 & 1ull);
    long long t0 = 0;
    bool waited = false;
    while (!__all_sync(0xffffffffu, ok)) {
      if (!waited) {
        t0 = clock64();
        waited = true;
      }
      if (__any_sync(0xffffffffu, clock64() - t0 > kWaitBudgetCycles)) {
        failed = true;
        if (lead) atomicExch(a.status, SW_ETIMEOUT);
        return;
      }
      if (!ok) {
        __nanosleep(32);  // (a waiting band leaves the issue slots to the bands that compute)
        if (in_range(ring_in - a.rings + rpos + lane, a.ring_entries, a.status))
          pend = ld_relaxed_u64(ring_in + rpos + lane);
        ok = (pend >> 31 & 1ull) != 0ull;
      }
    }
    if (lane < kColBlock)
      rgb[slot * kColBlock + lane] = make_uint2((uint32_t)pend & 0x7fffffffu, (uint32_t)(pend >> 32));
    rpos += kColBlock;
    __syncwarp();
  };
  // both boundary slots start as the matrix top boundary (a band without a
  // band above keeps it; the others overwrite them block by block)
  if (lane < kColBlock) {
    rgb[lane] = make_uint2((uint32_t)H0, (uint32_t)F0);
    rgb[kColBlock + lane] = make_uint2((uint32_t)H0, (uint32_t)F0);
  }
  __syncwarp();
  if (prev && nreal > 0) {
    load();
    land(0);
    if (!failed && nreal > 1) load();
  }

  int64_t wpos = sbase;
  for (int blk = 0; blk < nblk && !failed; ++blk) {
    const uint2 *gslot = rgb + (blk & 1) * kColBlock;
    const uint32_t *rw = reinterpret_cast<const uint32_t *>(rres + (blk & 1) * 32);
    if (lead) cp_async_wait<1>();
#pragma unroll 1
    for (int g4 = 0; g4 < kColBlock / 4; ++g4) {
      const uint32_t wa = rw[g4], wb = PACKED ? rw[4 + g4] : 0u;  // (used by lane 0 only)
#pragma unroll
      for (int s4 = 0; s4 < 4; ++s4) {
        const int s = g4 * 4 + s4;
        const int t = blk * kColBlock + s;
        W inH = (W)__shfl_sync(0xffffffffu, outH, src);
        W inF = (W)__shfl_sync(0xffffffffu, outF, src);
        uint32_t inRes = __shfl_sync(0xffffffffu, outRes, src);
        if (lead) {
          // (the residue ring holds the pad code past the unit's end, the
          // boundary slot the top boundary where no band lies above)
          inRes = PACKED ? prmt(wa, wb, sel_pair(s4)) : prmt(wa, 0u, sel_one(s4));
          const uint2 v = gslot[s];
          inH = (W)v.x;
          inF = (W)v.y;
        }
        if constexpr (kChecked) inRes = checked_codes<FORM>(inRes, a.status);
        column_step<R, FORM, SHORTF>(st, prow, 32 * R, inRes, inH, inF, cs, S, outH, outF, 0);
        outRes = inRes;
        if (tail) {
          const int j = t - LAG;
          if (j >= 0 && j < npad && in_range(ring_out - a.rings + wpos, a.ring_entries, a.status)) {
            const uint32_t lo = (uint32_t)outH | 0x80000000u;
            st_relaxed_u64(ring_out + wpos, ((unsigned long long)(uint32_t)outF << 32) | lo);
            ++wpos;
          }
        }
      }
    }
    if (lead) {
      if (blk + 2 < nblk) prefetch(blk + 2);
      else cp_async_commit();
    }
    if (prev && blk + 1 < nreal) {
      land((blk + 1) & 1);
      if (!failed && blk + 2 < nreal) load();
    } else if (prev && blk + 1 < nblk) {
      // the padding blocks after the last real one: top boundary again
      if (lane < kColBlock) rgb[((blk + 1) & 1) * kColBlock + lane] = make_uint2((uint32_t)H0, (uint32_t)F0);
      __syncwarp();
    }
  }
  if (lead) cp_async_wait<0>();
  Sout = S;
  return !failed;
}

template <int R>
__global__ void __launch_bounds__(kBandStreamThreads, 1) band_stream_kernel(const BandArgs a) {
  constexpr int RH = R / 2;  // rows per lane of kBandInt32Half jobs
  extern __shared__ __align__(128) uint8_t smem[];
  int8_t *sm = reinterpret_cast<int8_t *>(smem);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint8_t *prof = smem + kSubmatBytes + (size_t)warp * kWarpBytes<R>;
  uint8_t *ring = prof + kProfBytes<R>;
  for (int i = threadIdx.x; i < kAlphabet * kAlphabet; i += blockDim.x) sm[i] = a.submat[i];
  __syncthreads();
  const Consts cs = make_consts(a.sc);

  for (;;) {
    int g = 0;
    if (lane == 0) g = atomicAdd(a.band_counter, 1);
    g = __shfl_sync(0xffffffffu, g, 0);
    if (g >= a.nbands) break;
    const BandJob job = a.jobs[a.band_job[g]];
    const int b = g - job.band0;
    const QDesc qd = a.qd[job.q];
    const bool half = job.form == kBandInt32Half;
    __syncwarp();
    if (half) build_band_profile<RH>(prof, sm, a.qres + qd.qoff, qd.m, b * 32 * RH, lane, a.sc.pad);
    else build_band_profile<R>(prof, sm, a.qres + qd.qoff, qd.m, b * 32 * R, lane, a.sc.pad);
    __syncwarp();
    const unsigned long long *ring_in = b > 0 ? a.rings + job.ring0 + (int64_t)(b - 1) * job.cols : nullptr;
    unsigned long long *ring_out = b + 1 < job.nb ? a.rings + job.ring0 + (int64_t)b * job.cols : nullptr;
    int32_t *orow = a.out + (int64_t)job.q * a.out_stride;
    int64_t sbase = 0;
    bool ok = true;
    for (int t = 0; t < job.t_count && ok; ++t) {
      int2 p = make_int2(0, 0);
      if (in_range(job.t_begin + t, a.n_tpos, a.status)) p = a.tpos[job.t_begin + t];
      if (!in_range(p.x, a.db.n, a.status) || !in_range(p.y, a.db.n, a.status)) p = make_int2(0, 0);
      if (job.form == kBandPacked) {
        uint32_t S = 0u;
        // the one-operation F chain in 16-row lanes (3 % faster on the homolog
        // workload; with 8 rows 2 % slower)
        ok = band_unit<R, kFormPacked, (R >= 16)>(a, prof, ring, lane, p.x, p.y, sbase, ring_in, ring_out, cs, S);
        for (int d = 16; d > 0; d >>= 1) S = __vmaxs2(S, __shfl_xor_sync(0xffffffffu, S, d));
        if (ok && lane == 0) {
          if (in_range(job.q * a.out_stride + a.db.perm[p.x], a.out_size, a.status))
            atomicMax(&orow[a.db.perm[p.x]], (int32_t)(S & 0xffffu));
          if (p.y != p.x && in_range(job.q * a.out_stride + a.db.perm[p.y], a.out_size, a.status))
            atomicMax(&orow[a.db.perm[p.y]], (int32_t)(S >> 16));
        }
        sbase += max(a.db.npad[p.x], a.db.npad[p.y]);
      } else {
        int32_t S = 0;
        // (the int32 units of a 16-bit batch: the one-operation F chain too)
        if (half && a.short_int)
          ok = band_unit<RH, kFormInt32, true>(a, prof, ring, lane, p.x, p.x, sbase, ring_in, ring_out, cs, S);
        else if (half) ok = band_unit<RH, kFormInt32, false>(a, prof, ring, lane, p.x, p.x, sbase, ring_in, ring_out, cs, S);
        else if (a.short_int)
          ok = band_unit<R, kFormInt32, true>(a, prof, ring, lane, p.x, p.x, sbase, ring_in, ring_out, cs, S);
        else ok = band_unit<R, kFormInt32, false>(a, prof, ring, lane, p.x, p.x, sbase, ring_in, ring_out, cs, S);
        for (int d = 16; d > 0; d >>= 1) S = max(S, __shfl_xor_sync(0xffffffffu, S, d));
        if (ok && lane == 0 && in_range(job.q * a.out_stride + a.db.perm[p.x], a.out_size, a.status))
          atomicMax(&orow[a.db.perm[p.x]], S);
        sbase += a.db.npad[p.x];
      }
    }
    __syncwarp();
    if (!ok) break;
  }
}

// ---------------------------------------------------------------------------
// Transposed jobs: database row tracks against one query (see TrackArgs in
// internal.h).  The query residues are the columns; the bands' rows are
// database sequences stacked in row tracks.
//
// Two row tracks share a word in the 16-bit forms; their substitution scores
// come from two byte tables, one per track (rows [0, 21) and [21, 42) of the
// band's profile), paired into the two halves by a byte shuffle: the column's
// residue code c is passed as the pair (c, c + 21) to the two-sequence cell
// form.  (One table of query-pair words would save the shuffle but take
// twice the shared memory, and so half the resident warps.)
// ---------------------------------------------------------------------------

// 4 warps, one per SM sub-partition: a small batch has few bands, and CTAs
// of 8 warps put two on each sub-partition of half the SMs while the others
// idle
constexpr int kTrackThreads = 128;
template <int R>
constexpr int kTrackStride = 32 * R;                                // bytes per residue row of one table
template <int R>
constexpr int kTrackProfBytes = 2 * kProfRows * kTrackStride<R>;    // two tables of [21][32 lanes x R] bytes
template <int R>
constexpr int kTrackWarpBytes = ((kTrackProfBytes<R> + 320) + 127) / 128 * 128;

// Profile of a band's rows: the substitution score of query residue c
// (column) against each database row, SM(c, D[row]) (the query residue is
// the matrix's row index): table t, byte (c, lane, r) at (21 t + c) * stride
// + lane * R + r, for the low (t = 0) and high (t = 1) track.  Rows past a
// sequence's end, idle lanes and the pad residue (c = 20) hold the pad value.
template <int R, bool TWO>
__device__ __forceinline__ void build_track_profile(uint8_t *prof, const int8_t *sm, const DbView &db,
                                                    const TrackLane &L, int lane, int32_t pad, int32_t *status) {
#pragma unroll
  for (int t = 0; t < (TWO ? 2 : 1); ++t) {
    const int32_t pos = t ? L.pb : L.pa, r0 = t ? L.rb : L.ra;
    const bool ok = pos >= 0 && in_range(pos, db.n, status);
    const int32_t len = ok ? db.len[pos] : 0;
    const uint8_t *res = db.res + (ok ? db.off[pos] : 0);
    uint8_t code[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int32_t row = r0 + r;
      code[r] = (ok && row < len && in_range(res + row - db.res, db.res_bytes, status)) ? res[row] : (uint8_t)kPadCode;
    }
    for (int c = 0; c < kProfRows; ++c) {
#pragma unroll
      for (int i = 0; i < R / 4; ++i) {
        uint32_t v = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int r = 4 * i + j;
          const int32_t x = (c < kAlphabet && code[r] < kAlphabet) ? (int32_t)sm[c * kAlphabet + code[r]] : pad;
          v |= ((uint32_t)x & 0xffu) << (8 * j);
        }
        *reinterpret_cast<uint32_t *>(prof + (t * kProfRows + c) * kTrackStride<R> + lane * R + 4 * i) = v;
      }
    }
  }
}

// One band of a row track over all columns of its query.  keepH / addF: the
// lane's restart masks (a half whose rows start a sequence takes the matrix
// top boundary (0, F0) instead of the row above).  SPLIT: the lane's rows as
// two half-chains a column apart (column_step_split).  Returns false when a
// wait expired.
template <int R, int FORM, bool SPLIT>
__device__ __forceinline__ bool track_pass(const TrackArgs &a, const uint8_t *__restrict__ prof, uint8_t *ring,
                                           const int lane, const uint8_t *resQ, const int npad,
                                           const unsigned long long *ring_in, unsigned long long *ring_out,
                                           const Word<FORM> keepH, const Word<FORM> addF, const Consts &cs,
                                           Word<FORM> &Sout) {
  using W = Word<FORM>;
  constexpr bool PACKED = FORM != kFormInt32;
  constexpr int LAG = SPLIT ? 2 * 32 - 1 : 32 - 1;
  const W H0 = (W)0;
  const W F0 = PACKED ? (W)cs.F0W : (W)0;
  const int nblk = (npad + LAG + kColBlock - 1) / kColBlock;
  const int nreal = npad / kColBlock;
  const bool prev = ring_in != nullptr, next = ring_out != nullptr;
  const bool lead = lane == 0;
  const bool tail = lane == 31 && next;
  const int src = lane > 0 ? lane - 1 : lane;
  const uint8_t *prow = prof + lane * R;
  // the column's residue code(s): one table, or the pair (c, c + 21) of the two tables
  constexpr uint32_t kPadRes = PACKED ? (kPadCode | ((kPadCode + kProfRows) << 16)) : kPadCode;

  LaneState<R, FORM> st;
  lane_reset(st, cs);
  W outH = H0, outF = F0, S = (W)0;
  uint32_t outRes = kPadRes;
  // split lanes: the lower half's residue, diagonal H, incoming H (int32) and F, best
  uint32_t prevRes = kPadRes;
  W hdiagB = H0, midH = H0, midF = F0, S2 = (W)0;
  uint8_t *rres = ring;                              // [slot][16 B] query residue codes
  uint2 *rgb = reinterpret_cast<uint2 *>(ring + 64);  // [slot][16] (H, F) of the band above
  bool failed = false;

  auto prefetch = [&](int blk) {
    uint8_t *d = rres + (blk & 1) * 32;
    const int col = blk * kColBlock;
    if (col < npad && in_range(resQ + col + 15 - a.qt, a.qt_bytes, a.status)) cp_async16(d, resQ + col);
    else *reinterpret_cast<uint4 *>(d) = make_uint4(0x14141414u, 0x14141414u, 0x14141414u, 0x14141414u);
    cp_async_commit();
  };
  if (lead) {
    prefetch(0);
    prefetch(1);
  }

  int64_t rpos = 0;
  unsigned long long pend = 0ull;
  auto load = [&]() {
    if (lane < kColBlock && in_range(ring_in - a.rings + rpos + lane, a.ring_entries, a.status))
      pend = ld_relaxed_u64(ring_in + rpos + lane);
  };
  auto land = [&](int slot) {
    bool ok = lane >= kColBlock || (pend >> 31 & 1ull);
    long long t0 = 0;
    bool waited = false;
    while (!__all_sync(0xffffffffu, ok)) {
      if (!waited) {
        t0 = clock64();
        waited = true;
      }
      if (__any_sync(0xffffffffu, clock64() - t0 > kWaitBudgetCycles)) {
        failed = true;
        if (lead) atomicExch(a.status, SW_ETIMEOUT);
        return;
      }
      if (!ok) {
        __nanosleep(32);
        if (in_range(ring_in - a.rings + rpos + lane, a.ring_entries, a.status))
          pend = ld_relaxed_u64(ring_in + rpos + lane);
        ok = (pend >> 31 & 1ull) != 0ull;
      }
    }
    if (lane < kColBlock)
      rgb[slot * kColBlock + lane] = make_uint2((uint32_t)pend & 0x7fffffffu, (uint32_t)(pend >> 32));
    rpos += kColBlock;
    __syncwarp();
  };
  if (lane < kColBlock) {
    rgb[lane] = make_uint2((uint32_t)H0, (uint32_t)F0);
    rgb[kColBlock + lane] = make_uint2((uint32_t)H0, (uint32_t)F0);
  }
  __syncwarp();
  if (prev && nreal > 0) {
    load();
    land(0);
    if (!failed && nreal > 1) load();
  }

  for (int blk = 0; blk < nblk && !failed; ++blk) {
    const uint2 *gslot = rgb + (blk & 1) * kColBlock;
    const uint32_t *rw = reinterpret_cast<const uint32_t *>(rres + (blk & 1) * 32);
    if (lead) cp_async_wait<1>();
#pragma unroll 1
    for (int g4 = 0; g4 < kColBlock / 4; ++g4) {
      const uint32_t wa = rw[g4];  // (used by lane 0 only)
#pragma unroll
      for (int s4 = 0; s4 < 4; ++s4) {
        const int s = g4 * 4 + s4;
        const int t = blk * kColBlock + s;
        W inH = (W)__shfl_sync(0xffffffffu, outH, src);
        W inF = (W)__shfl_sync(0xffffffffu, outF, src);
        uint32_t inRes = __shfl_sync(0xffffffffu, outRes, src);
        if (lead) {
          const uint32_t c = prmt(wa, 0u, sel_one(s4));
          inRes = PACKED ? (c | ((c + kProfRows) << 16)) : c;
          const uint2 v = gslot[s];
          inH = (W)v.x;
          inF = (W)v.y;
        }
        // a half whose rows start a sequence: the top boundary
        inH = (W)((uint32_t)inH & (uint32_t)keepH);
        inF = (W)(((uint32_t)inF & (uint32_t)keepH) | (uint32_t)addF);
        if constexpr (kChecked) {
          if ((inRes & 0xffffu) > (uint32_t)kPadCode ||
              (PACKED && (inRes >> 16) - (uint32_t)kProfRows > (uint32_t)kPadCode) || (!PACKED && (inRes >> 16))) {
            atomicExch(a.status, kStatusBounds);
            inRes = kPadRes;
          }
        }
        if constexpr (SPLIT && PACKED) {
          uint32_t s1 = (uint32_t)S, s2 = (uint32_t)S2, hb = (uint32_t)hdiagB, mf = (uint32_t)midF, oh, of;
          column_step_split<R, FORM>(st, hb, mf, prow, kTrackStride<R>, inRes, prevRes, (uint32_t)inH, (uint32_t)inF,
                                     cs, s1, s2, oh, of, 0);
          S = (W)s1;
          S2 = (W)s2;
          hdiagB = (W)hb;
          midF = (W)mf;
          outH = (W)oh;
          outF = (W)of;
        } else if constexpr (SPLIT) {
          int32_t s1 = (int32_t)S, s2 = (int32_t)S2, hb = (int32_t)hdiagB, mh = (int32_t)midH, mf = (int32_t)midF;
          int32_t oh, of;
          column_step_split_int<R>(st, hb, mh, mf, prow, kTrackStride<R>, inRes, prevRes, (int32_t)inH, (int32_t)inF,
                                   cs, s1, s2, oh, of);
          S = (W)s1;
          S2 = (W)s2;
          hdiagB = (W)hb;
          midH = (W)mh;
          midF = (W)mf;
          outH = (W)oh;
          outF = (W)of;
        } else {
          column_step<R, FORM, PACKED>(st, prow, kTrackStride<R>, inRes, inH, inF, cs, S, outH, outF, 0);
        }
        if constexpr (SPLIT) {
          outRes = prevRes;
          prevRes = inRes;
        } else {
          outRes = inRes;
        }
        if (tail) {
          const int j = t - LAG;
          if (j >= 0 && j < npad && in_range(ring_out - a.rings + j, a.ring_entries, a.status)) {
            const uint32_t lo = (uint32_t)outH | 0x80000000u;
            st_relaxed_u64(ring_out + j, ((unsigned long long)(uint32_t)outF << 32) | lo);
          }
        }
      }
    }
    if (lead) {
      if (blk + 2 < nblk) prefetch(blk + 2);
      else cp_async_commit();
    }
    if (prev && blk + 1 < nreal) {
      land((blk + 1) & 1);
      if (!failed && blk + 2 < nreal) load();
    } else if (prev && blk + 1 < nblk) {
      if (lane < kColBlock) rgb[((blk + 1) & 1) * kColBlock + lane] = make_uint2((uint32_t)H0, (uint32_t)F0);
      __syncwarp();
    }
  }
  if (lead) cp_async_wait<0>();
  Sout = SPLIT ? score_max<FORM>(S, S2) : S;
  return !failed;
}

// The best score of each sequence among a band's lanes (its rows are
// contiguous lanes): a segmented maximum down the lanes, keyed by the
// sequence; the last lane of each segment adds it to the caller-order score
// with atomicMax (a sequence spanning several bands gets one per band).
__device__ __forceinline__ void track_scores(const TrackArgs &a, int32_t q, int32_t key, int32_t v, int lane) {
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int32_t ov = __shfl_up_sync(0xffffffffu, v, d);
    const int32_t ok = __shfl_up_sync(0xffffffffu, key, d);
    if (lane >= d && ok == key) v = max(v, ov);
  }
  const int32_t nk = __shfl_down_sync(0xffffffffu, key, 1);
  if ((lane == 31 || nk != key) && key >= 0 && in_range(key, a.db.n, a.status)) {
    const int64_t i = (int64_t)q * a.out_stride + a.db.perm[key];
    if (in_range(i, a.out_size, a.status)) atomicMax(&a.out[i], v);
  }
}

template <int R, bool SPLIT>
__global__ void __launch_bounds__(kTrackThreads, R == 8 ? 4 : R == 16 ? 2 : 1) band_track_kernel(const TrackArgs a) {
  extern __shared__ __align__(128) uint8_t smem[];
  int8_t *sm = reinterpret_cast<int8_t *>(smem);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint8_t *prof = smem + kSubmatBytes + (size_t)warp * kTrackWarpBytes<R>;
  uint8_t *ring = prof + kTrackProfBytes<R>;
  for (int i = threadIdx.x; i < kAlphabet * kAlphabet; i += blockDim.x) sm[i] = a.submat[i];
  __syncthreads();
  const Consts cs = make_consts(a.sc);
  const TrackLane idle{-1, 0, -1, 0};
  // a lane continues the sequence of the row above (in at least one used half)
  auto continues = [](const TrackLane &L, bool packed) {
    return (L.pa >= 0 && L.ra > 0) || (packed && L.pb >= 0 && L.rb > 0);
  };

  for (;;) {
    int g = 0;
    if (lane == 0) g = atomicAdd(a.band_counter, 1);
    g = __shfl_sync(0xffffffffu, g, 0);
    if (g >= a.nbands) break;
    const TrackJob job = a.jobs[a.band_job[g]];
    const int b = g - job.band0;
    const bool packed = job.packed != 0;
    const int64_t li = (int64_t)job.lane0 + 32 * (int64_t)b + lane;
    const TrackLane L = in_range(li, a.n_lanes, a.status) ? a.lanes[li] : idle;
    // the band reads the band above when its first lane continues a sequence;
    // it writes for the band below when that one's first lane does
    const bool prev = b > 0 && __shfl_sync(0xffffffffu, (int)continues(L, packed), 0) != 0;
    int nxt = 0;
    if (lane == 0 && b + 1 < job.nb) {
      const int64_t ln = (int64_t)job.lane0 + 32 * (int64_t)(b + 1);
      nxt = in_range(ln, a.n_lanes, a.status) && continues(a.lanes[ln], packed) ? 1 : 0;
    }
    const bool next = __shfl_sync(0xffffffffu, nxt, 0) != 0;
    const int32_t npad = a.qt_npad[job.q];
    const uint8_t *resQ = a.qt + a.qt_off[job.q];
    const unsigned long long *ring_in = prev ? a.rings + job.ring0 + (int64_t)(b - 1) * npad : nullptr;
    unsigned long long *ring_out = next ? a.rings + job.ring0 + (int64_t)b * npad : nullptr;
    const bool ra0 = L.pa < 0 || L.ra == 0, rb0 = L.pb < 0 || L.rb == 0;  // halves that restart
    __syncwarp();
    bool ok;
    if (packed) {
      build_track_profile<R, true>(prof, sm, a.db, L, lane, a.sc.pad, a.status);
      __syncwarp();
      const uint32_t mask = (ra0 ? 0x0000ffffu : 0u) | (rb0 ? 0xffff0000u : 0u);
      uint32_t S = 0u;
      ok = track_pass<R, kFormPacked, SPLIT>(a, prof, ring, lane, resQ, npad, ring_in, ring_out, ~mask, cs.F0W & mask,
                                          cs, S);
      track_scores(a, job.q, L.pa, (int32_t)(S & 0xffffu), lane);
      track_scores(a, job.q, L.pb, (int32_t)(S >> 16), lane);
    } else {
      build_track_profile<R, false>(prof, sm, a.db, L, lane, a.sc.pad, a.status);
      __syncwarp();
      int32_t S = 0;
      ok = track_pass<R, kFormInt32, SPLIT>(a, prof, ring, lane, resQ, npad, ring_in, ring_out, ra0 ? 0 : -1, 0, cs, S);
      track_scores(a, job.q, L.pa, S, lane);
    }
    __syncwarp();
    if (!ok) break;
  }
}

template <int R>
size_t smem_of() {
  return kSubmatBytes + (size_t)(kBandStreamThreads / 32) * kWarpBytes<R>;
}

// Dynamic shared memory that leaves room for only one band-stream CTA per SM
// (more than half of an SM's shared memory), or 0 if a block may not take it.
size_t one_cta_smem() {
  int dev = 0, per_sm = 0, per_block = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&per_block, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  const size_t want = ((size_t)per_sm / 2 + 1024 + 127) / 128 * 128;
  return want <= (size_t)per_block ? want : 0;
}

template <int R>
int occupancy_of() {
  // the limit admits the one-CTA-per-SM reservation as well
  const size_t limit = std::max(smem_of<R>(), one_cta_smem());
  if (cudaFuncSetAttribute(band_stream_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)limit) !=
      cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, band_stream_kernel<R>, kBandStreamThreads,
                                                    smem_of<R>()) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

template <int R>
size_t track_smem() { return kSubmatBytes + (size_t)(kTrackThreads / 32) * kTrackWarpBytes<R>; }

template <int R, bool SPLIT>
int track_occupancy() {
  if (cudaFuncSetAttribute(band_track_kernel<R, SPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)track_smem<R>()) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, band_track_kernel<R, SPLIT>, kTrackThreads,
                                                    track_smem<R>()) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

}  // namespace

int track_threads() { return kTrackThreads; }

bool track_supported_R(int R) { return R == 8 || R == 16 || R == 24; }

int track_max_ctas_per_sm(int R, bool split) {
  if (R == 8) return split ? track_occupancy<8, true>() : track_occupancy<8, false>();
  if (R == 16) return split ? track_occupancy<16, true>() : track_occupancy<16, false>();
  if (R == 24 && !split) return track_occupancy<24, false>();
  return 0;
}

cudaError_t launch_track(const TrackArgs &a, int R, bool split, int grid, cudaStream_t s) {
  const int T = kTrackThreads;
  if (R == 8 && split) band_track_kernel<8, true><<<grid, T, track_smem<8>(), s>>>(a);
  else if (R == 8) band_track_kernel<8, false><<<grid, T, track_smem<8>(), s>>>(a);
  else if (R == 16 && split) band_track_kernel<16, true><<<grid, T, track_smem<16>(), s>>>(a);
  else if (R == 16) band_track_kernel<16, false><<<grid, T, track_smem<16>(), s>>>(a);
  else if (R == 24 && !split) band_track_kernel<24, false><<<grid, T, track_smem<24>(), s>>>(a);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

int band_threads() { return kBandStreamThreads; }
bool band_supported_R(int R) { return R == 8 || R == 16; }
size_t band_smem_bytes(int R) { return R == 16 ? smem_of<16>() : smem_of<8>(); }
int band_max_ctas_per_sm(int R) { return R == 8 ? occupancy_of<8>() : R == 16 ? occupancy_of<16>() : 0; }

cudaError_t launch_band(const BandArgs &a, int R, int grid, bool one_per_sm, cudaStream_t s) {
  // one CTA per SM: the launch takes more than half of an SM's shared memory,
  // so that the hardware never places two on an SM, whatever else (the
  // transposed jobs beside it, a kernel finishing before it) holds the SMs
  // when its CTAs are placed
  const size_t extra = one_per_sm ? one_cta_smem() : 0;
  if (R == 8) band_stream_kernel<8><<<grid, kBandStreamThreads, std::max(extra, smem_of<8>()), s>>>(a);
  else if (R == 16) band_stream_kernel<16><<<grid, kBandStreamThreads, std::max(extra, smem_of<16>()), s>>>(a);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

}  // namespace swgb
