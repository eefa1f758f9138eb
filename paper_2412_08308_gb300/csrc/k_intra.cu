// Intra-task Smith-Waterman/Gotoh kernel for long database sequences (Sec. 2.2
// Eqs. 1-3; Sec. 3.1 "long kernel"; Fig. 1 intra-sequence parallelism),
// re-designed for sm_103a.
//
// One CTA computes one (query, database unit) matrix with a single chain of
// 32*W lanes spanning its W warps: lane g owns R consecutive rows of the
// current chunk of 32*W*R query rows and works on column t - g at global step
// t.  Inside a warp the bottom (H, F) of a lane and the residue codes move to
// the next lane by shuffle, as in the inter-task kernel; between warps they
// go through a ring in shared memory.  Each warp publishes how many columns
// it has written to its ring (producer) and read from the ring of the warp
// before it (consumer) once per block of 16 steps; the waits are bounded (a
// wait that exceeds the clock budget sets SW_ETIMEOUT and the CTA stops at the
// next barrier).  The profile chunk is staged once per chunk by a bulk TMA
// copy; the last warp's bottom row goes to a global strip that warp 0 reads
// back in the next chunk.
#include "devutil.cuh"
#include "dp_common.cuh"
#include "internal.h"
#include "../../include/swgb.h"

namespace swgb {
namespace {

constexpr int kIntraThreads = 512;  // 16 warps
constexpr int kWarpsMax = kIntraThreads / 32;
constexpr int kRing = 64;           // ring entries (columns) between consecutive warps

struct IntraShared {
  uint64_t mbar;
  int32_t task;
  int32_t abort;
  int32_t prod[kWarpsMax];  // columns written by warp w into its ring
  int32_t cons[kWarpsMax];  // columns read by warp w from the ring of warp w-1
  uint32_t smax[kWarpsMax];
};

__device__ __forceinline__ bool wait_at_least(volatile int32_t *p, int32_t v, volatile int32_t *abort) {
  if (*p >= v) return true;
  const long long t0 = clock64();
  while (*p < v) {
    if (*abort) return false;
    if (clock64() - t0 > kWaitBudgetCycles) return false;
    __nanosleep(32);
  }
  return true;
}

// One chunk of 32*Wq*R query rows against one database unit: the chain of
// Wq warps sweeps all columns; warp w > 0 reads the bottom row of warp w-1
// from the shared-memory ring, warp 0 reads the CTA's strip (prev) or the
// matrix top boundary, and the last warp writes the strip for the next chunk
// (next); the CTA barrier between chunks separates the two.
template <int R, int FORM>
__device__ __forceinline__ void sweep_chunk(IntraShared *sh, const uint8_t *pbuf, const int chunk_stride,
                                            uint4 *rings, const int Wq, const int warp, const int lane,
                                            const uint8_t *resA, const uint8_t *resB, const int npa, const int npb,
                                            const int npad, const bool prev, const bool next, uint2 *gb,
                                            int32_t *status, const Consts &cs, Word<FORM> &S,
                                            const uint8_t *res0, const int64_t res_bytes, const int gb_len) {
  using W = Word<FORM>;
  constexpr bool PACKED = FORM != kFormInt32;
  // split lanes (two half-chains a column apart): a warp's last lane trails
  // its first by 63 columns instead of 31
  constexpr int LAG = 2 * 32 - 1;
  const W H0 = (W)0;
  const W F0 = PACKED ? (W)cs.F0W : (W)0;
  volatile int32_t *vabort = &sh->abort;
  const int nblk = (npad + LAG + kColBlock - 1) / kColBlock;
  uint4 *ring_in = rings + (warp > 0 ? warp - 1 : 0) * kRing;
  uint4 *ring_out = rings + warp * kRing;
  const int g = warp * 32 + lane;
  const int src = lane > 0 ? lane - 1 : lane;

  LaneState<R, FORM> st;
  lane_reset(st, cs);
  W outH = H0, outF = F0;
  uint32_t outRes = kPadPair;
  // split lanes: the lower half's residue, diagonal H, incoming H and F, best
  uint32_t prevRes = kPadPair;
  W hdiagB = H0, midH = H0, midF = F0, S2 = (W)0;
  const uint8_t *prow = pbuf + g * R;
  const bool first = warp == 0, last = warp == Wq - 1;
  // warp 0 reads residues and (after the first chunk) the boundary strip one
  // block ahead: lane 0 holds the residue vectors, lanes 0..15 one strip entry each
  const uint4 padv = make_uint4(0x14141414u, 0x14141414u, 0x14141414u, 0x14141414u);
  uint4 ra4n = padv, rb4n = padv;
  uint2 gvn = make_uint2(0u, 0u);
  auto fetch = [&](int col) {
    if (lane == 0 && col < npad) {
      ra4n = col < npa && in_range(resA + col + 15 - res0, res_bytes, status)
                 ? *reinterpret_cast<const uint4 *>(resA + col) : padv;
      if (PACKED)
        rb4n = col < npb && in_range(resB + col + 15 - res0, res_bytes, status)
                   ? *reinterpret_cast<const uint4 *>(resB + col) : padv;
    }
    if (prev && lane < kColBlock && col + lane < npad && in_range(col + lane, gb_len, status))
      gvn = __ldcg(gb + col + lane);
  };
  if (first) fetch(0);
  for (int blk = 0; blk < nblk; ++blk) {
    const int col0 = blk * kColBlock;
    // producer: room in the ring for the columns this block writes
    // consumer: the previous warp has written the columns this block reads
    if (lane == 0) {
      bool okw = true;
      if (!last) okw &= wait_at_least(&sh->cons[warp + 1], col0 + kColBlock - LAG - kRing, vabort);
      if (!first) okw &= wait_at_least(&sh->prod[warp - 1], min(col0 + kColBlock, npad), vabort);
      if (!okw && !*vabort) {
        *vabort = 1;
        atomicExch(status, SW_ETIMEOUT);
      }
      __threadfence_block();
    }
    __syncwarp();
    if (*vabort) return;
    const uint4 ra4 = ra4n, rb4 = rb4n;
    const uint2 gv = gvn;
    if (first) fetch(col0 + kColBlock);
    const bool real = col0 < npad;  // block-uniform: npad is a multiple of 16
#pragma unroll 1
    for (int g4 = 0; g4 < kColBlock / 4; ++g4) {
      const uint32_t wa = word_of(ra4, g4), wb = word_of(rb4, g4);
#pragma unroll
      for (int s4 = 0; s4 < 4; ++s4) {
        const int s = g4 * 4 + s4;
        const int tau = col0 + s;  // this warp's local step: lane 0 is at column tau
        W inH = (W)__shfl_sync(0xffffffffu, outH, src);
        W inF = (W)__shfl_sync(0xffffffffu, outF, src);
        uint32_t inRes = __shfl_sync(0xffffffffu, outRes, src);
        uint32_t gx = 0u, gy = 0u;
        if (first && prev) {  // warp-uniform
          gx = __shfl_sync(0xffffffffu, gv.x, s);
          gy = __shfl_sync(0xffffffffu, gv.y, s);
        }
        if (lane == 0) {
          if (!real) {
            inH = H0;
            inF = F0;
            inRes = kPadPair;
          } else if (first) {
            inRes = PACKED ? prmt(wa, wb, sel_pair(s4)) : prmt(wa, 0u, sel_one(s4));
            if (prev) {
              inH = (W)gx;
              inF = (W)gy;
            } else {
              inH = H0;
              inF = F0;
            }
          } else {
            const uint4 v = ring_in[tau % kRing];
            inH = (W)v.x;
            inF = (W)v.y;
            inRes = v.z;
          }
        }
        if constexpr (kChecked) inRes = checked_codes<FORM>(inRes, status);
        if constexpr (PACKED) {
          uint32_t s = (uint32_t)S, s2 = (uint32_t)S2, hb = (uint32_t)hdiagB, mf = (uint32_t)midF, oh, of;
          column_step_split<R, FORM>(st, hb, mf, prow, chunk_stride, inRes, prevRes, (uint32_t)inH, (uint32_t)inF,
                                     cs, s, s2, oh, of, 0);
          S = (W)s;
          S2 = (W)s2;
          hdiagB = (W)hb;
          midF = (W)mf;
          outH = (W)oh;
          outF = (W)of;
        } else {
          int32_t s = (int32_t)S, s2 = (int32_t)S2, hb = (int32_t)hdiagB, mh = (int32_t)midH, mf = (int32_t)midF;
          int32_t oh, of;
          column_step_split_int<R>(st, hb, mh, mf, prow, chunk_stride, inRes, prevRes, (int32_t)inH, (int32_t)inF,
                                   cs, s, s2, oh, of);
          S = (W)s;
          S2 = (W)s2;
          hdiagB = (W)hb;
          midH = (W)mh;
          midF = (W)mf;
          outH = (W)oh;
          outF = (W)of;
        }
        outRes = prevRes;
        prevRes = inRes;
        if (lane == 31) {
          const int col = tau - LAG;
          if (col >= 0 && col < npad) {
            if (!last) ring_out[col % kRing] = make_uint4((uint32_t)outH, (uint32_t)outF, outRes, 0u);
            else if (next && in_range(col, gb_len, status)) gb[col] = make_uint2((uint32_t)outH, (uint32_t)outF);
          }
        }
      }
    }
    __syncwarp();
    if (lane == 31 && !last) {
      __threadfence_block();
      const int written = min(max(0, col0 + kColBlock - LAG), npad);
      *(volatile int32_t *)&sh->prod[warp] = written;
    }
    if (lane == 0 && !first) *(volatile int32_t *)&sh->cons[warp] = min(col0 + kColBlock, npad);
  }
  S = score_max<FORM>(S, S2);
}

template <int R, bool PACKED>
__global__ void __launch_bounds__(kIntraThreads, 1) intra_kernel(const InterArgs a) {
  constexpr int FORM = PACKED ? kFormPacked : kFormInt32;
  using W = Word<FORM>;
  extern __shared__ __align__(128) uint8_t smem[];
  IntraShared *sh = reinterpret_cast<IntraShared *>(smem);
  uint8_t *pbuf = smem + 256;
  uint4 *rings = reinterpret_cast<uint4 *>(pbuf + a.pbuf_bytes);  // [warp][kRing]

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const Consts cs = make_consts(a.sc);
  volatile int32_t *vabort = &sh->abort;

  if (threadIdx.x == 0) {
    mbar_init(&sh->mbar, 1);
    sh->abort = 0;
    fence_mbar_init();
  }
  __syncthreads();
  uint32_t parity = 0;
  const int n_tasks = *a.n_tasks;

  for (;;) {
    if (threadIdx.x == 0) sh->task = atomicAdd(a.task_counter, 1);
    __syncthreads();
    const int t = sh->task;
    if (t >= n_tasks || sh->abort) break;

    const Task tk = a.tasks[t];
    const QDesc qd = a.qd[tk.q];
    const int Wq = qd.L / 32;  // warps of the chain for this query
    const int u = tk.unit_begin;
    int posA = 0, posB = 0;
    if (in_range(PACKED ? 2 * u + 1 : u, a.n_unit_pos, a.status)) {
      posA = a.unit_pos[PACKED ? 2 * u : u];
      posB = PACKED ? a.unit_pos[2 * u + 1] : posA;
    }
    if (!in_range(posA, a.db.n, a.status) || !in_range(posB, a.db.n, a.status)) posA = posB = 0;
    const int npa = a.db.npad[posA];
    const int npb = PACKED ? a.db.npad[posB] : 0;
    const int npad = max(npa, npb);
    const uint8_t *resA = a.db.res + a.db.off[posA];
    const uint8_t *resB = a.db.res + a.db.off[posB];
    uint2 *gb = a.gbuf + (size_t)blockIdx.x * a.gbuf_stride;

    W S = (W)0;
    for (int c = 0; c < qd.nchunks; ++c) {
      if (threadIdx.x < kWarpsMax) {
        sh->prod[threadIdx.x] = 0;
        sh->cons[threadIdx.x] = 0;
      }
      if (threadIdx.x == 0) {
        if (in_range(qd.prof_off + (int64_t)(c + 1) * qd.chunk_bytes - 1, a.prof_bytes, a.status) &&
            (!kChecked || qd.chunk_bytes <= a.pbuf_bytes)) {
          mbar_arrive_expect_tx(&sh->mbar, (uint32_t)qd.chunk_bytes);
          bulk_g2s(pbuf, a.prof + qd.prof_off + (int64_t)c * qd.chunk_bytes, (uint32_t)qd.chunk_bytes, &sh->mbar);
        } else {
          mbar_arrive_expect_tx(&sh->mbar, 0u);  // (checked build: the copy is skipped, the phase completes)
        }
      }
      __syncthreads();
      const bool ok = mbar_wait_bounded(&sh->mbar, parity);
      parity ^= 1u;
      if (!__syncthreads_and(ok)) {
        if (threadIdx.x == 0) atomicExch(a.status, SW_ETIMEOUT);
        return;
      }
      if (warp < Wq)
        sweep_chunk<R, FORM>(sh, pbuf, qd.chunk_stride, rings, Wq, warp, lane, resA, resB, npa, npb, npad, c > 0,
                             c + 1 < qd.nchunks, gb, a.status, cs, S, a.db.res, a.db.res_bytes, a.gbuf_stride);
      __syncthreads();  // chunk done: ring counters, strip and profile buffer are free
      if (*vabort) return;
    }

    // max over the whole chain
    for (int d = 16; d > 0; d >>= 1) S = score_max<FORM>(S, (W)__shfl_xor_sync(0xffffffffu, S, d));
    if (lane == 0) sh->smax[warp] = (uint32_t)S;
    __syncthreads();
    if (threadIdx.x == 0) {
      W m = (W)sh->smax[0];
      for (int w = 1; w < Wq; ++w) m = score_max<FORM>(m, (W)sh->smax[w]);
      write_scores<FORM>(m, posA, posB, tk.q, qd, a);
    }
    __syncthreads();
  }
}

template <int R, bool PACKED>
cudaError_t launch_intra_one(const InterArgs &a, int grid, size_t smem, cudaStream_t s) {
  intra_kernel<R, PACKED><<<grid, kIntraThreads, smem, s>>>(a);
  return cudaGetLastError();
}

constexpr int kIntraSmemMax = 220 * 1024;

template <int R, bool PACKED>
cudaError_t configure_intra_one() {
  return cudaFuncSetAttribute(intra_kernel<R, PACKED>, cudaFuncAttributeMaxDynamicSharedMemorySize, kIntraSmemMax);
}

}  // namespace

int intra_threads() { return kIntraThreads; }

size_t intra_smem_bytes(int pbuf_bytes) {
  return 256 + (size_t)pbuf_bytes + (size_t)kWarpsMax * kRing * sizeof(uint4);
}

cudaError_t configure_intra(int R, bool packed) {
  if (R == 8) return packed ? configure_intra_one<8, true>() : configure_intra_one<8, false>();
  if (R == 16) return packed ? configure_intra_one<16, true>() : configure_intra_one<16, false>();
  return cudaErrorInvalidValue;
}

cudaError_t launch_intra(const InterArgs &a, int R, bool packed, int grid, size_t smem, cudaStream_t s) {
  if (R == 8) return packed ? launch_intra_one<8, true>(a, grid, smem, s) : launch_intra_one<8, false>(a, grid, smem, s);
  if (R == 16)
    return packed ? launch_intra_one<16, true>(a, grid, smem, s) : launch_intra_one<16, false>(a, grid, smem, s);
  return cudaErrorInvalidValue;
}

}  // namespace swgb
