// Traceback of selected hits: one optimal local alignment per (query,
// database sequence) pair, the alignment output the paper's score-only search
// leaves out (Sec. 2.2: H records the best score of an alignment ending at
// each cell; the alignment itself is the path that produced it).
//
// Fill: one warp per hit runs the int32 chain of the inter-task kernel (32
// lanes of R rows, chunk by chunk through a global strip) and records, per
// cell, 4 bits of provenance: where H came from (0 = the zero floor, 1 = the
// diagonal, 2 = E, 3 = F; ties in that order) and whether E and F extend a gap
// (else they open one).  It also keeps the first cell (row-major) holding the
// best score.  Walk: one thread per hit follows the bits back from that cell
// to a cell whose H came from the floor.
#include "devutil.cuh"
#include "internal.h"
#include "../../include/swgb.h"

namespace swgb {
namespace {

constexpr int kTraceR = 16;     // rows per lane
constexpr int kTraceWarps = 4;  // hits per CTA

__device__ __forceinline__ bool earlier(int32_t s, int32_t i, int32_t j, int32_t bs, int32_t bi, int32_t bj) {
  // better score, or the same score at a cell earlier in row-major order
  return s > bs || (s == bs && (i < bi || (i == bi && j < bj)));
}

__global__ void __launch_bounds__(32 * kTraceWarps) trace_fill_kernel(const TraceArgs a) {
  constexpr int R = kTraceR;
  __shared__ int8_t sm[kAlphabet * kProfRows];  // SM(query code, target code), pad column 20
  for (int i = threadIdx.x; i < kAlphabet * kProfRows; i += blockDim.x) {
    const int qc = i / kProfRows, tc = i % kProfRows;
    sm[i] = tc < kAlphabet ? a.submat[qc * kAlphabet + tc] : (int8_t)a.sc.pad;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int h = blockIdx.x * kTraceWarps + (threadIdx.x >> 5);
  if (h >= a.nhits) return;
  const TraceHit hit = a.hits[h];
  const uint8_t *q = a.qres + hit.qoff;
  const uint8_t *t = a.tres + hit.toff;
  uint8_t *dirs = a.dirs + hit.dir_off;
  uint2 *strip = a.strips + hit.strip_off;
  const int go = a.sc.go, ge = a.sc.ge;
  const int src = lane > 0 ? lane - 1 : 0;
  const int nchunks = hit.mrow / (32 * R);
  int32_t bs = 0, bi = 0, bj = 0;  // best score and its cell (1-based), this lane

  for (int c = 0; c < nchunks; ++c) {
    const int row0 = c * 32 * R + lane * R;  // 0-based first row of this lane
    int qc[R];
#pragma unroll
    for (int r = 0; r < R; ++r) qc[r] = row0 + r < hit.m ? q[row0 + r] : 0;
    int32_t Hl[R], El[R];
#pragma unroll
    for (int r = 0; r < R; ++r) Hl[r] = El[r] = 0;
    int32_t hdiag = 0, outH = 0, outF = 0;
    uint32_t outRes = kPadCode;
    for (int step = 0; step < hit.npad + 31; ++step) {
      int32_t inH = __shfl_sync(0xffffffffu, outH, src);
      int32_t inF = __shfl_sync(0xffffffffu, outF, src);
      uint32_t res = __shfl_sync(0xffffffffu, outRes, src);
      const int col = step - lane;  // 0-based column of this lane
      if (lane == 0) {
        res = col < hit.npad ? t[col] : kPadCode;
        inH = c > 0 && col < hit.npad ? (int32_t)strip[col].x : 0;
        inF = c > 0 && col < hit.npad ? (int32_t)strip[col].y : 0;
      }
      const int8_t *srow = sm + res;  // sm[qc * 21 + res]
      int32_t hu = inH, fu = inF, hul = hdiag;
      uint32_t nib[R / 8];
#pragma unroll
      for (int w = 0; w < R / 8; ++w) nib[w] = 0u;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int32_t e_ext = El[r] - ge, e_open = Hl[r] - go;
        const int32_t f_ext = fu - ge, f_open = hu - go;
        const int32_t e = max(e_ext, e_open), f = max(f_ext, f_open);
        const int32_t dg = hul + srow[qc[r] * kProfRows];
        const int32_t hh = max(max(dg, e), max(f, 0));
        const uint32_t hsrc = hh == 0 ? 0u : hh == dg ? 1u : hh == e ? 2u : 3u;
        const uint32_t bits = hsrc | ((e_ext > e_open) ? 4u : 0u) | ((f_ext > f_open) ? 8u : 0u);
        nib[r / 8] |= bits << (4 * (r % 8));
        const int row = row0 + r;
        if (col >= 0 && col < hit.n && row < hit.m && earlier(hh, row + 1, col + 1, bs, bi, bj)) {
          bs = hh;
          bi = row + 1;
          bj = col + 1;
        }
        hul = Hl[r];
        Hl[r] = hh;
        El[r] = e;
        hu = hh;
        fu = f;
      }
      hdiag = inH;
      outH = hu;
      outF = fu;
      outRes = res;
      if (col >= 0 && col < hit.npad) {
        // rows row0 .. row0+R-1 of column col: R nibbles, R/2 bytes (column-major, mrow rows)
        uint2 *dst = reinterpret_cast<uint2 *>(dirs + ((int64_t)col * hit.mrow + row0) / 2);
#pragma unroll
        for (int w = 0; w < R / 8; w += 2) dst[w / 2] = make_uint2(nib[w], nib[w + 1]);
        if (lane == 31 && c + 1 < nchunks) strip[col] = make_uint2((uint32_t)outH, (uint32_t)outF);
      }
    }
    __syncwarp();
    __threadfence_block();  // the strip written by lane 31 is read by lane 0 in the next chunk
  }
  // best over the warp, first in row-major order among equal scores
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
    TraceResult res{};
    res.score = bs;
    res.end_i = bi;
    res.end_j = bj;
    a.results[h] = res;
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

int trace_rows_per_chunk() { return 32 * kTraceR; }

cudaError_t launch_trace(const TraceArgs &a, cudaStream_t s) {
  if (a.nhits <= 0) return cudaSuccess;
  trace_fill_kernel<<<(a.nhits + kTraceWarps - 1) / kTraceWarps, 32 * kTraceWarps, 0, s>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  trace_walk_kernel<<<(a.nhits + 127) / 128, 128, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace swgb
