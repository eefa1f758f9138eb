// Traceback of selected hits: one optimal local alignment per (query,
// database sequence) pair, the alignment output the paper's score-only search
// leaves out (Sec. 2.2: H records the best score of an alignment ending at
// each cell; the alignment itself is the path that produced it).
//
// Fill: one CTA per hit.  Its warps take the hit's chunks of 512 query rows
// in turn (warp w: chunks w, w + W, ...), each warp the int32 chain of the
// inter-task kernel (32 lanes of 16 rows) over every target column, and the
// bottom row of a chunk goes to the warp of the next chunk through a ring in
// shared memory, so the chunks run as a pipeline instead of one after the
// other.  The last warp's bottom row goes to a global strip of the whole row
// instead (the first warp reads it in its next round): a ring there could
// fill while the first warp is still busy with its current chunk, and the
// pipeline would wait on itself.  Per cell the fill records 4 bits of provenance: where H came from (0
// = the zero floor, 1 = the diagonal, 2 = E, 3 = F; ties in that order) and
// whether E and F extend a gap (else they open one).  It also keeps the first
// cell (row-major) holding the best score.  Walk: one thread per hit follows
// the bits back from that cell to a cell whose H came from the floor.
#include <algorithm>

#include "devutil.cuh"
#include "dp_common.cuh"
#include "internal.h"
#include "../../include/swgb.h"

namespace swgb {
namespace {

constexpr int kTraceR = 16;         // rows per lane
constexpr int kTraceChunk = 32 * kTraceR;
constexpr int kTraceWarpsMax = 8;   // chunks of one hit in flight
constexpr int kTraceRing = 128;     // columns per ring between consecutive warps

struct TraceShared {
  int32_t prod[kTraceWarpsMax];  // columns written to warp w's ring, all rounds together
  int32_t cons[kTraceWarpsMax];  // columns of warp w's ring read by the next warp, likewise
  int32_t abort;
  int32_t bs[kTraceWarpsMax], bi[kTraceWarpsMax], bj[kTraceWarpsMax];
};

// shared memory: the counters above, then per warp a profile and a ring
constexpr size_t kTraceHead = (sizeof(TraceShared) + 127) / 128 * 128;

__device__ __forceinline__ bool earlier(int32_t s, int32_t i, int32_t j, int32_t bs, int32_t bi, int32_t bj) {
  // better score, or the same score at a cell earlier in row-major order
  return s > bs || (s == bs && (i < bi || (i == bi && j < bj)));
}

__device__ __forceinline__ bool trace_wait(volatile int32_t *p, int32_t v, volatile int32_t *abort) {
  if (*p >= v) return true;
  const long long t0 = clock64();
  while (*p < v) {
    if (*abort) return false;
    if (clock64() - t0 > kLongWaitBudgetCycles) return false;
    __nanosleep(32);
  }
  return true;
}

__host__ __device__ constexpr size_t trace_prof_bytes() { return (size_t)kProfRows * 32 * sizeof(uint4); }  // per warp
__host__ __device__ constexpr size_t trace_ring_bytes() { return (size_t)kTraceRing * sizeof(uint2); }      // per warp

__global__ void __launch_bounds__(32 * kTraceWarpsMax) trace_fill_kernel(const TraceArgs a) {
  constexpr int R = kTraceR;
  extern __shared__ __align__(16) uint8_t smem[];
  TraceShared *sh = reinterpret_cast<TraceShared *>(smem);
  const int W = blockDim.x >> 5;
  uint4 *prof_all = reinterpret_cast<uint4 *>(smem + kTraceHead);                      // [warp][21][32]
  uint2 *rings = reinterpret_cast<uint2 *>(smem + kTraceHead + W * trace_prof_bytes());  // [warp][ring]
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const TraceHit hit = a.hits[blockIdx.x];
  if (threadIdx.x < kTraceWarpsMax) {
    sh->prod[threadIdx.x] = 0;
    sh->cons[threadIdx.x] = 0;
  }
  if (threadIdx.x == 0) sh->abort = 0;
  __syncthreads();
  volatile int32_t *vabort = &sh->abort;
  const uint8_t *q = a.qres + hit.qoff;
  const uint8_t *t = a.tres + hit.toff;
  uint8_t *dirs = a.dirs + hit.dir_off;
  const int go = a.sc.go, ge = a.sc.ge;
  const int src = lane > 0 ? lane - 1 : 0;
  const int nchunks = hit.mrow / kTraceChunk;
  const int npad = hit.npad;
  const int nsteps = (npad + 31 + kColBlock - 1) / kColBlock * kColBlock;
  uint4 *prof = prof_all + warp * kProfRows * 32;
  const int wprev = (warp + W - 1) % W;
  uint2 *ring_in = rings + wprev * kTraceRing;
  uint2 *ring_out = rings + warp * kTraceRing;
  uint2 *strip = a.strips + hit.strip_off;  // the last warp's bottom rows, for the first warp's next round
  const bool strip_in = warp == 0, strip_out = warp == W - 1;
  int32_t bs = 0, bi = 0, bj = 0;  // best score and its cell (1-based), this lane

  for (int c = warp; c < nchunks; c += W) {
    const int row0 = c * kTraceChunk + lane * R;  // 0-based first row of this lane
    // this lane's profile: 16 rows' scores per residue code (pad code 20: the pad score)
    for (int res = 0; res < kProfRows; ++res) {
      uint32_t w4[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        uint32_t word = 0u;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int row = row0 + 4 * k + i;
          const int qc = row < hit.m ? q[row] : 0;
          const int v = res < kAlphabet ? a.submat[qc * kAlphabet + res] : a.sc.pad;
          word |= ((uint32_t)v & 0xffu) << (8 * i);
        }
        w4[k] = word;
      }
      prof[res * 32 + lane] = make_uint4(w4[0], w4[1], w4[2], w4[3]);
    }
    __syncwarp();
    const bool prev = c > 0, next = c + 1 < nchunks;
    // ring counters run over all rounds: chunk c's columns start at (c / W) * npad
    const int32_t base_out = (c / W) * npad;
    const int32_t base_in = prev ? ((c - 1) / W) * npad : 0;
    int32_t Hl[R], El[R];
#pragma unroll
    for (int r = 0; r < R; ++r) Hl[r] = El[r] = 0;
    int32_t hdiag = 0, outH = 0, outF = 0;
    uint32_t outRes = kPadCode;
    for (int blk = 0; blk < nsteps / kColBlock; ++blk) {
      const int col0 = blk * kColBlock;
      // the chunk above has written this block's columns; room in this warp's ring
      bool ok = true;
      if (lane == 0 && prev) ok &= trace_wait(&sh->prod[wprev], base_in + min(col0 + kColBlock, npad), vabort);
      if (lane == 31 && next && !strip_out) {
        const int jmax = min(col0 + kColBlock - 1 - 31, npad - 1);
        if (jmax >= 0) ok &= trace_wait(&sh->cons[warp], base_out + jmax + 1 - kTraceRing, vabort);
      }
      if (!ok) *vabort = 1;
      __syncwarp();
      if (*vabort) break;
      __threadfence_block();
#pragma unroll 4
      for (int s = 0; s < kColBlock; ++s) {
        int32_t inH = __shfl_sync(0xffffffffu, outH, src);
        int32_t inF = __shfl_sync(0xffffffffu, outF, src);
        uint32_t res = __shfl_sync(0xffffffffu, outRes, src);
        const int col = col0 + s - lane;  // 0-based column of this lane
        if (lane == 0) {
          res = col < npad ? t[col] : kPadCode;
          if (prev && col < npad) {
            const uint2 v = strip_in ? __ldcg(strip + col) : ring_in[col % kTraceRing];
            inH = (int32_t)v.x;
            inF = (int32_t)v.y;
          } else {
            inH = inF = 0;
          }
        }
        const uint4 pv = prof[res * 32 + lane];
        const uint32_t pw[4] = {pv.x, pv.y, pv.z, pv.w};
        int32_t hu = inH, fu = inF, hul = hdiag, mstep = 0;
        uint32_t nib[2] = {0u, 0u};
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const int32_t e_ext = El[r] - ge, e_open = Hl[r] - go;
          const int32_t f_ext = fu - ge, f_open = hu - go;
          const int32_t e = max(e_ext, e_open), f = max(f_ext, f_open);
          const int32_t dg = hul + (int32_t)prmt(pw[r >> 2], 0u, sel_sext(r & 3));
          const int32_t hh = max(max(dg, e), max(f, 0));
          const uint32_t hsrc = hh == 0 ? 0u : hh == dg ? 1u : hh == e ? 2u : 3u;
          const uint32_t bits = hsrc | ((e_ext > e_open) ? 4u : 0u) | ((f_ext > f_open) ? 8u : 0u);
          nib[r >> 3] |= bits << (4 * (r & 7));
          mstep = max(mstep, hh);
          hul = Hl[r];
          Hl[r] = hh;
          El[r] = e;
          hu = hh;
          fu = f;
        }
        // the best cell: only a step whose maximum reaches the best so far
        // needs the row-by-row test (cells past the query or the target excluded)
        if (mstep >= bs && col >= 0 && col < hit.n) {
#pragma unroll
          for (int r = 0; r < R; ++r) {
            const int row = row0 + r;
            if (row < hit.m && earlier(Hl[r], row + 1, col + 1, bs, bi, bj)) {
              bs = Hl[r];
              bi = row + 1;
              bj = col + 1;
            }
          }
        }
        hdiag = inH;
        outH = hu;
        outF = fu;
        outRes = res;
        if (col >= 0 && col < npad) {
          // rows row0 .. row0+15 of column col: 8 bytes (column-major, mrow rows)
          *reinterpret_cast<uint2 *>(dirs + ((int64_t)col * hit.mrow + row0) / 2) = make_uint2(nib[0], nib[1]);
          if (lane == 31 && next) {
            const uint2 v = make_uint2((uint32_t)outH, (uint32_t)outF);
            if (strip_out) __stcg(strip + col, v);
            else ring_out[col % kTraceRing] = v;
          }
        }
      }
      // publish: columns written to this warp's ring, columns read from the one before
      __syncwarp();
      if (lane == 31 && next) {
        __threadfence_block();
        *(volatile int32_t *)&sh->prod[warp] = base_out + min(max(0, col0 + kColBlock - 31), npad);
      }
      if (lane == 0 && prev) *(volatile int32_t *)&sh->cons[wprev] = base_in + min(col0 + kColBlock, npad);
    }
    __syncwarp();
    if (*vabort) break;
  }
  // best over the warp, then over the warps; first in row-major order among equal scores
  for (int d = 16; d > 0; d >>= 1) {
    const int32_t os = __shfl_xor_sync(0xffffffffu, bs, d);
    const int32_t oi = __shfl_xor_sync(0xffffffffu, bi, d);
    const int32_t oj = __shfl_xor_sync(0xffffffffu, bj, d);
    if (earlier(os, oi, oj, bs, bi, bj)) {
      bs = os;
      bi = oi;
      bj = oj;
    }
  }
  if (lane == 0) {
    sh->bs[warp] = bs;
    sh->bi[warp] = bi;
    sh->bj[warp] = bj;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < W; ++w)
      if (earlier(sh->bs[w], sh->bi[w], sh->bj[w], bs, bi, bj)) {
        bs = sh->bs[w];
        bi = sh->bi[w];
        bj = sh->bj[w];
      }
    TraceResult res{};
    res.score = bs;
    res.end_i = bi;
    res.end_j = bj;
    res.n_ops = *vabort ? -1 : 0;
    a.results[blockIdx.x] = res;
  }
}

// Walk back from the best cell: in H, the floor ends the alignment, the
// diagonal aligns Q[i] with D[j] ('M'), E and F switch state; in E a target
// residue faces a gap ('D'), in F a query residue ('I'); the extension bit
// keeps the state, else the walk returns to H.  Operations are written from
// the last to the first, then reversed.
__global__ void trace_walk_kernel(const TraceArgs a) {
  const int h = blockIdx.x * blockDim.x + threadIdx.x;
  if (h >= a.nhits) return;
  const TraceHit hit = a.hits[h];
  TraceResult res = a.results[h];
  if (res.n_ops < 0) return;  // the fill gave up on a wait
  const uint8_t *dirs = a.dirs + hit.dir_off;
  uint8_t *ops = a.ops + hit.ops_off;
  int i = res.end_i, j = res.end_j, state = 0;
  int64_t k = 0;
  const int64_t cap = (int64_t)hit.m + hit.n;
  if (res.score > 0) {
    while (i > 0 && j > 0 && k < cap) {
      const int64_t cell = (int64_t)(j - 1) * hit.mrow + (i - 1);
      const uint32_t bits = (dirs[cell >> 1] >> (4 * (cell & 1))) & 0xfu;
      if (state == 0) {
        const uint32_t hsrc = bits & 3u;
        if (hsrc == 0u) break;
        if (hsrc == 1u) {
          ops[k++] = 'M';
          --i;
          --j;
        } else {
          state = hsrc == 2u ? 1 : 2;
        }
      } else if (state == 1) {
        ops[k++] = 'D';
        state = (bits & 4u) ? 1 : 0;
        --j;
      } else {
        ops[k++] = 'I';
        state = (bits & 8u) ? 2 : 0;
        --i;
      }
    }
  }
  for (int64_t x = 0, y = k - 1; x < y; ++x, --y) {
    const uint8_t tmp = ops[x];
    ops[x] = ops[y];
    ops[y] = tmp;
  }
  res.begin_i = res.score > 0 ? i : 0;
  res.begin_j = res.score > 0 ? j : 0;
  res.n_ops = (int32_t)k;
  if (res.score == 0) res.end_i = res.end_j = 0;
  a.results[h] = res;
}

}  // namespace

int trace_rows_per_chunk() { return kTraceChunk; }

int trace_warps(int max_chunks) { return std::max(1, std::min(kTraceWarpsMax, max_chunks)); }

size_t trace_smem_bytes(int warps) { return kTraceHead + (size_t)warps * (trace_prof_bytes() + trace_ring_bytes()); }

cudaError_t launch_trace(const TraceArgs &a, int warps, cudaStream_t s) {
  if (a.nhits <= 0) return cudaSuccess;
  const size_t smem = trace_smem_bytes(warps);
  cudaError_t e = cudaFuncSetAttribute(trace_fill_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  trace_fill_kernel<<<a.nhits, 32 * warps, smem, s>>>(a);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  trace_walk_kernel<<<(a.nhits + 127) / 128, 128, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace swgb
