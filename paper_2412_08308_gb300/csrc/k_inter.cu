// Inter-task Smith-Waterman/Gotoh kernels (Sec. 2.2 Eqs. 1-3; Sec. 3.1 "short
// kernel"; Fig. 1 inter-sequence parallelism), re-designed for sm_103a.
//
// Work decomposition
// ------------------
// A *chain* of L lanes (4 <= L <= 32, several chains per warp) computes the
// alignment matrix of one query against one database sequence (int32 form),
// against two sequences at once (packed form: two 16-bit cells per 32-bit
// register), or of two queries against one sequence (query-pair form).  Lane
// k of a chain owns R consecutive query rows of the current *chunk* of L*R
// rows and sweeps the database columns; lane k works on column t-k at step t,
// receiving the bottom row (H, F) of lane k-1 and the residue code(s) through
// warp shuffles.  This is an anti-diagonal wavefront inside a warp: cells on
// one anti-diagonal of lanes run in the same step.  In the 16-bit forms a
// lane's rows are two half-chains a column apart (column_step_split), so lane
// k works on column t-2k and its two halves' dependency chains interleave.
//
// The query is processed chunk by chunk.  All chains of a CTA work on the same
// query and move from chunk to chunk together: the profile slice of the next
// chunk is staged into shared memory by a 1-D bulk TMA copy while the current
// one is used, and the bottom boundary row of a chunk goes through a global
// scratch strip to lane 0 of the same chain in the next chunk (prefetched with
// cp.async into a small per-chain shared-memory ring).
//
// Persistent CTAs pull (query, tile of database units) tasks from an atomic
// counter; tasks are ordered longest first.
//
// Cell arithmetic
// ---------------
// int32 form: the twelve-instruction body of Algorithm 1, one cell per lane op.
// packed forms: two cells per 32-bit word, each 16-bit half a signed cell
// value (two database sequences, or two queries against one sequence);
// additions are per-half (__vadd2 / __vsub2, no carry crosses the halves) and
// maxima are per-half VIMNMX (__vmaxs2, __vimax_s16x2_relu for the zero floor).
// E and F never fall below -Go, so no half wraps downward; a half whose final
// score exceeds 32767 - max(SM) may have wrapped upward and is flagged and
// recomputed exactly in int32 (rescue pass; query pairs are planned only where
// no half can pass that bound, and a half that does sets an error status).
#include "devutil.cuh"
#include "dp_common.cuh"
#include "internal.h"
#include "../../include/swgb.h"

namespace swgb {
namespace {

constexpr int kThreads = 256;
constexpr int kChainsPerWarpMax = 8;  // lanes per chain >= 4
constexpr int kRingBytes = 320;       // residues: 2 slots x 2 seqs x 16 B; boundary: 2 slots x 16 x 8 B

// 16-bit forms with split lanes (column_step_split): two half-chains per
// lane, lanes two columns apart.
template <int R, int FORM>
constexpr bool kSplit = FORM != kFormInt32 && R % 8 == 0;
// steps from a chain's first lane reaching a column to its last lane leaving it
template <int R, int FORM>
__host__ __device__ constexpr int chain_lag(int L) { return kSplit<R, FORM> ? 2 * L - 1 : L - 1; }

// One pass of a chain over all columns of its unit for the rows of one chunk.
// restart (16-bit forms): halves whose rows start a new query in this chunk;
// they take the matrix top boundary instead of the strip of the chunk above.
template <int R, int FORM, bool WIDE>
__device__ __forceinline__ void chain_pass(const uint8_t *__restrict__ pch, const int stride, const int L,
                                           const int k, const int lane, const int slot, const int gstride,
                                           const bool live, const int nblk,
                                           const int npad, const int npa, const int npb,
                                           const uint8_t *__restrict__ resA, const uint8_t *__restrict__ resB,
                                           uint8_t *ring, uint2 *gb, const bool prev, const bool next,
                                           const uint32_t restart, const Consts &cs, Word<FORM> &S,
                                           const uint8_t *res0, const int64_t res_bytes, const int gb_len,
                                           int32_t *status) {
  using W = Word<FORM>;
  constexpr bool PACKED = FORM != kFormInt32;      // 16-bit halves
  constexpr bool PAIRS = FORM == kFormPacked;      // two database sequences per unit
  constexpr bool SPLIT = kSplit<R, FORM>;
  const W H0 = (W)0;
  const W F0 = PACKED ? (W)cs.F0W : (W)0;
  LaneState<R, FORM> st;
  lane_reset(st, cs);
  W outH = H0, outF = F0;
  // residue code(s) of the column; one database sequence: the bare code
  constexpr uint32_t kPadRes = PAIRS ? kPadPair : (uint32_t)kPadCode;
  uint32_t outRes = kPadRes;
  // split lanes: the lower half's residue, diagonal H and incoming F, best
  uint32_t prevRes = kPadRes, hdiagB = 0u, midF = (uint32_t)F0, S2 = 0u;
  const int src = (k > 0) ? lane - 1 : lane;
  const bool lead = live && k == 0;
  const bool tail = live && (k == L - 1) && next;
  uint8_t *rres = ring;                                  // [slot][seq][16 B]
  uint2 *rgb = reinterpret_cast<uint2 *>(ring + 64);     // [slot][16]
  // this lane's profile slot: R bytes, or (query pairs, wide entries) R/4
  // 16-byte groups gstride apart
  const uint8_t *prow = (FORM == kFormQPair || WIDE) ? pch + slot * 16 : pch + slot * R;

  auto prefetch = [&](int blk) {
    const int slot = blk & 1;
    const int col = blk * kColBlock;
    uint8_t *d = rres + slot * 32;
    if (col < npa && in_range(resA + col + 15 - res0, res_bytes, status)) cp_async16(d, resA + col);
    else *reinterpret_cast<uint4 *>(d) = make_uint4(0x14141414u, 0x14141414u, 0x14141414u, 0x14141414u);
    if (PAIRS) {
      if (col < npb && in_range(resB + col + 15 - res0, res_bytes, status)) cp_async16(d + 16, resB + col);
      else *reinterpret_cast<uint4 *>(d + 16) = make_uint4(0x14141414u, 0x14141414u, 0x14141414u, 0x14141414u);
    }
    if (prev && col < npad && in_range(col + 15, gb_len, status)) {
#pragma unroll
      for (int i = 0; i < 8; ++i) cp_async16(rgb + slot * 16 + 2 * i, gb + col + 2 * i);
    } else {
      // the matrix top boundary (first chunk, or padding columns)
#pragma unroll
      for (int i = 0; i < 8; ++i)
        reinterpret_cast<uint4 *>(rgb + slot * 16)[i] = make_uint4((uint32_t)H0, (uint32_t)F0, (uint32_t)H0, (uint32_t)F0);
    }
    cp_async_commit();
  };
  if (lead) {
    prefetch(0);
    prefetch(1);
  }

  for (int blk = 0; blk < nblk; ++blk) {
    const uint32_t *rw = reinterpret_cast<const uint32_t *>(rres + (blk & 1) * 32);  // this block's residue words
    uint2 *gslot = rgb + (blk & 1) * 16;
    // lane 0's columns of this block are all real or all padding (npad is a
    // multiple of 16); real ones of a later chunk come from the strip
    const bool from_strip = prev && blk * kColBlock < npad;
    if (lead) {
      cp_async_wait<1>();
      if (PACKED && restart && from_strip) {  // (this thread's own cp.async data, already landed)
#pragma unroll
        for (int i = 0; i < kColBlock; ++i) {
          const uint2 v = gslot[i];
          gslot[i] = make_uint2(v.x & ~restart, (v.y & ~restart) | ((uint32_t)F0 & restart));
        }
      }
    }
    // 4 groups of 4 steps; only the 4 steps are unrolled, which keeps the loop
    // body small enough for the instruction cache
#pragma unroll 1
    for (int g4 = 0; g4 < kColBlock / 4; ++g4) {
      // four residues of each sequence (used by the lead lane only)
      const uint32_t wa = rw[g4], wb = PAIRS ? rw[4 + g4] : 0u;
#pragma unroll
      for (int s4 = 0; s4 < 4; ++s4) {
        const int s = g4 * 4 + s4;
        const int t = blk * kColBlock + s;
        W inH = (W)__shfl_sync(0xffffffffu, outH, src);
        W inF = (W)__shfl_sync(0xffffffffu, outF, src);
        uint32_t inRes = __shfl_sync(0xffffffffu, outRes, src);
        if (lead) {
          // (the residue ring holds the pad code past the end of a sequence,
          // the boundary slot the top boundary where there is no chunk above;
          // the first lane of a chain without a unit keeps its own pad values,
          // its ring is never filled)
          inRes = PAIRS ? prmt(wa, wb, sel_pair(s4)) : prmt(wa, 0u, sel_one(s4));
          const uint2 v = gslot[s];
          inH = (W)v.x;
          inF = (W)v.y;
        }
        if constexpr (kChecked) inRes = checked_codes<FORM>(inRes, status);
        if constexpr (SPLIT) {
          uint32_t s = (uint32_t)S, oh, of;
          column_step_split<R, FORM, WIDE>(st, hdiagB, midF, prow, stride, inRes, prevRes, (uint32_t)inH, (uint32_t)inF,
                                     cs, s, S2, oh, of, gstride);
          S = (W)s;
          outH = (W)oh;
          outF = (W)of;
          outRes = prevRes;
          prevRes = inRes;
        } else {
          column_step<R, FORM, false, WIDE>(st, prow, stride, inRes, inH, inF, cs, S, outH, outF, gstride);
          outRes = inRes;
        }
        if (tail) {
          const int j = t - chain_lag<R, FORM>(L);
          if ((unsigned)j < (unsigned)npad && in_range(j, gb_len, status))
            gb[j] = make_uint2((uint32_t)outH, (uint32_t)outF);
        }
      }
    }
    if (lead) {
      if (blk + 2 < nblk) prefetch(blk + 2);
      else cp_async_commit();
    }
  }
  if (lead) cp_async_wait<0>();
  if constexpr (SPLIT) S = score_max<FORM>(S, (W)S2);
}

template <int R, int FORM, bool WIDE>
__global__ void __launch_bounds__(kThreads, 2) inter_kernel(const InterArgs a) {
  using W = Word<FORM>;
  constexpr bool PAIRS = FORM == kFormPacked;
  extern __shared__ __align__(128) uint8_t smem[];
  uint64_t *mbar = reinterpret_cast<uint64_t *>(smem);
  volatile int *s_task = reinterpret_cast<volatile int *>(smem + 16);
  uint8_t *pbuf = smem + 128;
  uint8_t *rings = pbuf + a.pbuf_count * a.pbuf_bytes;
  const bool dbl = a.pbuf_count == 2;

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
  const Consts cs = make_consts(a.sc);

  if (threadIdx.x == 0) {
    mbar_init(&mbar[0], 1);
    mbar_init(&mbar[1], 1);
    fence_mbar_init();
  }
  __syncthreads();
  uint32_t par0 = 0u, par1 = 0u;
  const int n_tasks = *a.n_tasks;

  for (;;) {
    if (threadIdx.x == 0) *s_task = atomicAdd(a.task_counter, 1);
    __syncthreads();
    const int t = *s_task;
    if (t >= n_tasks) break;

    const Task tk = a.tasks[t];
    const QDesc qd = a.qd[tk.q];
    const int L = qd.L;
    const int G = 32 / L;
    const int cw = lane / L;
    const int k = lane - cw * L;
    const int ci = warp * G + cw;
    const bool live = (cw < G) && (ci < tk.unit_count);
    // profile slot (lanes of chains past the last one reuse an in-range slot)
    const int slot = cw < G ? lane : k;
    const int gstride = profile_slots(L) * 16;
    int posA = 0, posB = 0, npa = 0, npb = 0;
    if (live) {
      const int u = tk.unit_begin + ci;
      const int iB = PAIRS ? 2 * u + 1 : u;
      if (in_range(iB, a.n_unit_pos, a.status)) {
        posA = a.unit_pos[PAIRS ? 2 * u : u];
        posB = PAIRS ? a.unit_pos[iB] : posA;
      }
      if (!in_range(posA, a.db.n, a.status) || !in_range(posB, a.db.n, a.status)) posA = posB = 0;
      npa = a.db.npad[posA];
      npb = PAIRS ? a.db.npad[posB] : 0;
    }
    const int npad = max(npa, npb);
    const int nblk =
        __reduce_max_sync(0xffffffffu, live ? (npad + chain_lag<R, FORM>(L) + kColBlock - 1) / kColBlock : 0);
    const uint8_t *resA = a.db.res + (live ? a.db.off[posA] : 0);
    const uint8_t *resB = a.db.res + (live ? a.db.off[posB] : 0);
    const int cslot = warp * kChainsPerWarpMax + min(cw, kChainsPerWarpMax - 1);
    uint8_t *ring = rings + cslot * kRingBytes;
    uint2 *gb = a.gbuf + ((size_t)blockIdx.x * nwarps * kChainsPerWarpMax + cslot) * (size_t)a.gbuf_stride;

    auto issue = [&](int c) {
      const int b = dbl ? (c & 1) : 0;
      const int64_t end = qd.prof_off + (int64_t)(c + 1) * qd.chunk_bytes;
      if (!in_range(end - 1, a.prof_bytes, a.status) || (kChecked && qd.chunk_bytes > a.pbuf_bytes)) {
        mbar_arrive_expect_tx(&mbar[b], 0u);  // (checked build: the copy is skipped, the phase completes)
        return;
      }
      mbar_arrive_expect_tx(&mbar[b], (uint32_t)qd.chunk_bytes);
      bulk_g2s(pbuf + b * a.pbuf_bytes, a.prof + qd.prof_off + (int64_t)c * qd.chunk_bytes,
               (uint32_t)qd.chunk_bytes, &mbar[b]);
    };
    if (threadIdx.x == 0) {
      issue(0);
      if (dbl && qd.nchunks > 1) issue(1);
    }

    W S = (W)0;
    for (int c = 0; c < qd.nchunks; ++c) {
      const int b = dbl ? (c & 1) : 0;
      TrackChunk tc{};
      uint32_t restart = 0u;
      if constexpr (FORM == kFormQPair) {
        tc = a.track[qd.track_off + c];
        restart = ((tc.flags & kStartA) ? 0x0000ffffu : 0u) | ((tc.flags & kStartB) ? 0xffff0000u : 0u);
      }
      const bool ok = mbar_wait_bounded(&mbar[b], b ? par1 : par0);
      if (b) par1 ^= 1u;
      else par0 ^= 1u;
      if (!__syncthreads_and(ok)) {
        if (threadIdx.x == 0) atomicExch(a.status, SW_ETIMEOUT);
        return;
      }
      chain_pass<R, FORM, WIDE>(pbuf + b * a.pbuf_bytes, qd.chunk_stride, L, k, lane, slot, gstride, live, nblk, npad,
                          npa, npb, resA, resB, ring, gb, c > 0, c + 1 < qd.nchunks, restart, cs, S,
                          a.db.res, a.db.res_bytes, a.gbuf_stride, a.status);
      __syncthreads();
      // the buffer just used is free: load the chunk after the one in flight
      // (one buffer: the next chunk, while the other CTA on this SM computes)
      if (threadIdx.x == 0 && c + (dbl ? 2 : 1) < qd.nchunks) issue(c + (dbl ? 2 : 1));
      if constexpr (FORM == kFormQPair) {
        // a half whose query ends in this chunk: its best over the chain's
        // lanes is the score; the half then starts from zero
        if (tc.flags & (kEndA | kEndB)) {
          W m = S;
          for (int d = 1; d < L; d <<= 1)
            m = score_max<FORM>(m, (W)__shfl_sync(0xffffffffu, m, (k + d < L) ? lane + d : lane));
          const bool endA = (tc.flags & kEndA) && tc.qa >= 0, endB = (tc.flags & kEndB) && tc.qb >= 0;
          if (live && k == 0) {
            const int32_t sa = (int32_t)((uint32_t)m & 0xffffu), sb = (int32_t)((uint32_t)m >> 16);
            const int32_t p = a.db.perm[posA];
            const int64_t ia = (int64_t)tc.qa * a.out_stride + p, ib = (int64_t)tc.qb * a.out_stride + p;
            if (endA && in_range(ia, a.out_size, a.status)) a.out[ia] = sa;
            if (endB && in_range(ib, a.out_size, a.status)) a.out[ib] = sb;
            if ((endA && sa > a.sc.thresh) || (endB && sb > a.sc.thresh)) atomicExch(a.status, kStatusSaturated);
          }
          S = (W)((uint32_t)S & ~(((tc.flags & kEndA) ? 0x0000ffffu : 0u) | ((tc.flags & kEndB) ? 0xffff0000u : 0u)));
        }
      }
    }

    if constexpr (FORM != kFormQPair) {
      // max over the chain's lanes
      for (int d = 1; d < L; d <<= 1)
        S = score_max<FORM>(S, (W)__shfl_sync(0xffffffffu, S, (k + d < L) ? lane + d : lane));
      if (live && k == 0) write_scores<FORM>(S, posA, posB, tk.q, qd, a);
    }
  }
}

template <int R, int FORM, bool WIDE>
cudaError_t launch_one(const InterArgs &a, int grid, int threads, size_t smem, cudaStream_t s) {
  inter_kernel<R, FORM, WIDE><<<grid, threads, smem, s>>>(a);
  return cudaGetLastError();
}

// Raise the dynamic shared-memory limit of an instantiation (done at plan time,
// never inside a launch sequence that may be captured into a graph) and return
// its resident CTAs per SM for the given block size and shared memory.
template <int R, int FORM, bool WIDE>
int configure_one(int threads, size_t smem) {
  auto kern = inter_kernel<R, FORM, WIDE>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, threads, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

}  // namespace

int inter_threads() { return kThreads; }

size_t inter_smem_bytes(int pbuf_bytes, int pbuf_count, int threads) {
  return 128 + (size_t)pbuf_count * pbuf_bytes + (size_t)(threads / 32) * kChainsPerWarpMax * kRingBytes;
}

#define SWGB_INTER_R_LIST(X) X(4) X(8) X(12) X(16) X(24)

bool inter_supported_R(int R) {
#define SWGB_CASE(RR) if (R == RR) return true;
  SWGB_INTER_R_LIST(SWGB_CASE)
#undef SWGB_CASE
  return false;
}

int inter_chain_lag(int R, int form, int L) {
  form &= ~kFormWide;  // (the lag does not depend on the profile's entry width)
#define SWGB_CASE(RR)                                                    \
  if (R == RR) {                                                         \
    if (form == kFormInt32) return chain_lag<RR, kFormInt32>(L);        \
    if (form == kFormPacked) return chain_lag<RR, kFormPacked>(L);      \
    if (form == kFormQPair) return chain_lag<RR, kFormQPair>(L);        \
  }
  SWGB_INTER_R_LIST(SWGB_CASE)
#undef SWGB_CASE
  return L - 1;
}

cudaError_t launch_inter(const InterArgs &a, int R, int form, int grid, int threads, size_t smem,
                         cudaStream_t s) {
#define SWGB_CASE(RR)                                                                                 \
  if (R == RR) {                                                                                      \
    if (form == kFormInt32) return launch_one<RR, kFormInt32, false>(a, grid, threads, smem, s);      \
    if (form == kFormPacked) return launch_one<RR, kFormPacked, false>(a, grid, threads, smem, s);    \
    if (form == kFormQPair) return launch_one<RR, kFormQPair, false>(a, grid, threads, smem, s);      \
    if (form == (kFormInt32 | kFormWide)) return launch_one<RR, kFormInt32, true>(a, grid, threads, smem, s);   \
    if (form == (kFormPacked | kFormWide)) return launch_one<RR, kFormPacked, true>(a, grid, threads, smem, s); \
  }
  SWGB_INTER_R_LIST(SWGB_CASE)
#undef SWGB_CASE
  return cudaErrorInvalidValue;
}

int inter_max_ctas_per_sm(int R, int form, int threads, size_t smem) {
#define SWGB_CASE(RR)                                                                              \
  if (R == RR) {                                                                                   \
    if (form == kFormInt32) return configure_one<RR, kFormInt32, false>(threads, smem);            \
    if (form == kFormPacked) return configure_one<RR, kFormPacked, false>(threads, smem);          \
    if (form == kFormQPair) return configure_one<RR, kFormQPair, false>(threads, smem);            \
    if (form == (kFormInt32 | kFormWide)) return configure_one<RR, kFormInt32, true>(threads, smem);   \
    if (form == (kFormPacked | kFormWide)) return configure_one<RR, kFormPacked, true>(threads, smem); \
  }
  SWGB_INTER_R_LIST(SWGB_CASE)
#undef SWGB_CASE
  return 0;
}

}  // namespace swgb
