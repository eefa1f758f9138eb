// Pair-band kernel: one long (query, target) pair, int32 cells (the pairwise
// alignment of two long sequences, Sec. 2.2 case (a); Fig. 1 intra-sequence
// parallelism).  Band b is query rows [32 R b, 32 R (b+1)): one warp is a
// chain of 32 lanes of R rows (the inter-task chain of k_inter.cu) that sweeps
// every target column.  Warp w of the grid takes bands w, w + warps, ... in
// order (warps numbered across the SMs first, so that even a few bands per SM
// land on every SM); a band's top boundary is the bottom row of the band
// above, read from that band's ring as soon as the entries are there, so the
// bands run as a pipeline over every warp of every SM.  All warps are resident (cooperative
// launch), a band waits only on the band above (data) and on the band below
// (room in its ring), and every wait is bounded.
//
// Boundary rings
// --------------
// Band b writes its bottom row to ring b mod nslots, `window` columns long
// (column j at j mod window).  An entry is one 64-bit word written by one
// relaxed store, so the band below can tell a fresh entry from the one it
// replaces by two tag bits, with no flag and no fence on the producer's side:
//   low word  = H | (lap parity << 31)            lap = j / window
//   high word = (F + Go) | (generation bit << 31)  generation = b / nslots,
//                                                  bit = its parity inverted
// A location holds either the entry the reader waits for or the one written
// before it there: the previous lap of the same band (other lap parity) or the
// last lap of the band that used the ring before (other generation parity), or
// zeros (generation bit 0, which no band of generation 0 writes).  The reader
// hands consumed columns back through a counter (release/acquire), so a band
// never overwrites an entry that the band below has not read.  H lies in
// [0, 2^31 - Go) (the host bounds the scores) and F in [-Go, H] (H takes the
// maximum with F; H >= 0 bounds F below by -Go), so both fields fit 31 bits.
#include "devutil.cuh"
#include "dp_common.cuh"
#include "internal.h"
#include "../../include/swgb.h"

namespace swgb {
namespace {

constexpr int kPairThreads = 512;  // at most 16 warps per CTA, one band each
// Split lanes (column_step_split_int): two half-chains per lane, lanes two
// columns apart, so a band's last lane trails its first by 63 columns.
template <int R>
constexpr bool kBandSplit = R % 8 == 0;
template <int R>
constexpr int kBandLag = kBandSplit<R> ? 2 * 32 - 1 : 32 - 1;
constexpr int kBandRingBytes = 320;  // residues: 2 slots x 32 B; boundary: 2 slots x 16 x 8 B

struct BandIO {
  const unsigned long long *in;  // ring of the band above
  unsigned long long *out;       // this band's ring
  int32_t *cons_in;              // columns of `in` consumed, published for the band above
  const int32_t *cons_out;       // columns of `out` consumed by the band below
  int32_t window;
  uint32_t gen_in, gen_out;      // generation tag bits of the two rings (0 or 1)
  int32_t cons_every;            // blocks between publications of cons_in
  int32_t *status;
};

__device__ __forceinline__ uint32_t band_gen(int b, int nslots) { return ((uint32_t)(b / nslots) & 1u) ^ 1u; }

// One band over all target columns.  Lane 0 takes the residues (cp.async ring,
// two blocks ahead) and the band above's entries; lanes 0..15 load the entries
// of block blk + 2 at the end of block blk and check their tags at the end of
// block blk + 1 (loading again until they are fresh), then unpack them into
// the shared-memory slot lane 0 reads.  Lane 31 stores one entry per column.
// With split lanes each lane runs two half-chains a column apart (see
// column_step_split_int).
// Returns false when a wait expired.
template <int R>
__device__ __forceinline__ bool band_pass(const uint8_t *__restrict__ pch, const int stride, const int lane,
                                          const int nblk, const int npad, const uint8_t *__restrict__ target,
                                          uint8_t *ring, const bool prev, const bool next, const Consts &cs,
                                          int32_t &S, const BandIO &x) {
  using W = int32_t;
  LaneState<R, kFormInt32> st;
  lane_reset(st, cs);
  W outH = 0, outF = 0;
  uint32_t outRes = kPadPair;
  // split lanes: the lower half's residue, diagonal H, incoming H and F, best
  uint32_t prevRes = kPadPair;
  int32_t hdiagB = 0, midH = 0, midF = 0, S2 = 0;
  const int src = lane > 0 ? lane - 1 : lane;
  const bool lead = lane == 0;
  const bool tail = lane == 31 && next;
  const int nreal = npad / kColBlock;                // blocks of real columns
  uint8_t *rres = ring;                              // [slot][16 B] residue codes
  uint2 *rgb = reinterpret_cast<uint2 *>(ring + 64);  // [slot][16] (H, F) of the band above
  const uint8_t *prow = pch + lane * R;
  bool failed = false;

  auto prefetch = [&](int blk) {
    uint8_t *d = rres + (blk & 1) * 32;
    const int col = blk * kColBlock;
    if (col < npad) cp_async16(d, target + col);
    else *reinterpret_cast<uint4 *>(d) = make_uint4(0x14141414u, 0x14141414u, 0x14141414u, 0x14141414u);
    cp_async_commit();
  };
  if (lead) {
    prefetch(0);
    prefetch(1);
  }

  // reading side: ring position and lap parity of the next block to load
  int rpos = 0, consumed = 0, since = 0;
  uint32_t rlap = 0u;
  unsigned long long pend = 0ull;
  auto load = [&]() {
    if (lane < kColBlock) pend = ld_relaxed_u64(x.in + rpos + lane);
  };
  auto fresh = [&](unsigned long long v) {
    return ((uint32_t)v >> 31) == rlap && (uint32_t)(v >> 63) == x.gen_in;
  };
  // wait until the loaded entries are fresh, unpack them into `slot`, advance
  auto land = [&](int slot) {
    bool ok = lane >= kColBlock || fresh(pend);
    long long t0 = 0;
    bool waited = false;
    while (!__all_sync(0xffffffffu, ok)) {
      if (!waited) {
        t0 = clock64();
        waited = true;
      }
      if (__any_sync(0xffffffffu, clock64() - t0 > kLongWaitBudgetCycles)) {
        failed = true;
        if (lead) atomicExch(x.status, SW_ETIMEOUT);
        return;
      }
      if (!ok) {
        pend = ld_relaxed_u64(x.in + rpos + lane);
        ok = fresh(pend);
      }
    }
    if (lane < kColBlock) {
      const int32_t h = (int32_t)((uint32_t)pend & 0x7fffffffu);
      const int32_t f = (int32_t)((uint32_t)(pend >> 32) & 0x7fffffffu) - cs.go;
      rgb[slot * kColBlock + lane] = make_uint2((uint32_t)h, (uint32_t)f);
    }
    consumed += kColBlock;
    rpos += kColBlock;
    if (rpos == x.window) {
      rpos = 0;
      rlap ^= 1u;
    }
    __syncwarp();
    // hand the columns back every few blocks and at the end (the release orders
    // the loads of lanes 0..15, which the warp barrier above ordered first)
    if (++since == x.cons_every || consumed == npad) {
      since = 0;
      if (lead) st_release(x.cons_in, consumed);
    }
  };
  // both boundary slots start as the matrix top boundary (the band without
  // a band above keeps it; the others overwrite block by block, and the two
  // padding blocks at the end get it back below)
  if (lane < kColBlock) {
    rgb[lane] = make_uint2(0u, 0u);
    rgb[kColBlock + lane] = make_uint2(0u, 0u);
  }
  __syncwarp();
  if (prev) {
    load();
    land(0);
    if (!failed && nreal > 1) load();
  }

  // writing side: ring position, lap parity, room as last read
  int wpos = 0, seen_cons = 0;
  uint32_t wlap = 0u;
  const uint32_t gen_bit = x.gen_out << 31;

  for (int blk = 0; blk < nblk && !failed; ++blk) {
    if (tail) {
      // room in this band's ring for the columns this block writes
      const int jmax = min(blk * kColBlock + kColBlock - 1 - kBandLag<R>, npad - 1);
      const int need = jmax + 1 - x.window;
      if (jmax >= 0 && seen_cons < need) {
        seen_cons = wait_flag_value(x.cons_out, need, kLongWaitBudgetCycles);
        if (seen_cons < need) {
          failed = true;
          atomicExch(x.status, SW_ETIMEOUT);
        }
      }
    }
    if (__any_sync(0xffffffffu, failed)) {
      failed = true;
      break;
    }
    const uint2 *gslot = rgb + (blk & 1) * kColBlock;
    const uint32_t *rw = reinterpret_cast<const uint32_t *>(rres + (blk & 1) * 32);  // this block's residues
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
          // (the ring holds the pad code past the target's end, the slot the
          // top boundary where no band lies above)
          inRes = prmt(wa, 0u, sel_one(s4));
          const uint2 v = gslot[s];
          inH = (W)v.x;
          inF = (W)v.y;
        }
        if constexpr (kBandSplit<R>) {
          column_step_split_int<R>(st, hdiagB, midH, midF, prow, stride, inRes, prevRes, inH, inF, cs, S, S2, outH,
                                   outF);
          outRes = prevRes;
          prevRes = inRes;
        } else {
          column_step<R, kFormInt32>(st, prow, stride, inRes, inH, inF, cs, S, outH, outF);
          outRes = inRes;
        }
        if (tail) {
          const int j = t - kBandLag<R>;
          if (j >= 0 && j < npad) {
            const uint32_t lo = (uint32_t)outH | (wlap << 31);
            const uint32_t hi = (uint32_t)(outF + cs.go) | gen_bit;
            st_relaxed_u64(x.out + wpos, ((unsigned long long)hi << 32) | lo);
            if (++wpos == x.window) {
              wpos = 0;
              wlap ^= 1u;
            }
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
      if (lane < kColBlock) rgb[((blk + 1) & 1) * kColBlock + lane] = make_uint2(0u, 0u);
      __syncwarp();
    }
  }
  if (lead) cp_async_wait<0>();
  S = max(S, S2);
  return !failed;
}

template <int R>
__global__ void __launch_bounds__(kPairThreads, 1) pair_band_kernel(const PairBandArgs a) {
  extern __shared__ __align__(128) uint8_t smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
  uint8_t *pbuf = smem + (size_t)warp * (a.pbuf_bytes + kBandRingBytes);
  uint8_t *ring = pbuf + a.pbuf_bytes;
  const Consts cs = make_consts(a.sc);
  const int nblk = (a.npad + kBandLag<R> + kColBlock - 1) / kColBlock;
  int32_t S = 0;
  // global warp g = warp * grid + CTA: bands spread over the SMs first
  for (int b = warp * gridDim.x + blockIdx.x; b < a.nbands; b += gridDim.x * nw) {
    const uint4 *src = reinterpret_cast<const uint4 *>(a.prof + (int64_t)b * a.band_bytes);
    for (int i = lane; i < a.band_bytes / 16; i += 32) reinterpret_cast<uint4 *>(pbuf)[i] = __ldg(src + i);
    __syncwarp();
    BandIO x;
    x.in = a.strips + (size_t)((b + a.nslots - 1) % a.nslots) * a.window;
    x.out = a.strips + (size_t)(b % a.nslots) * a.window;
    x.cons_in = a.cons + (b > 0 ? b - 1 : 0);
    x.cons_out = a.cons + b;
    x.window = a.window;
    x.gen_in = band_gen(b > 0 ? b - 1 : 0, a.nslots);
    x.gen_out = band_gen(b, a.nslots);
    x.cons_every = a.cons_every;
    x.status = a.status;
    const bool ok = band_pass<R>(pbuf, a.stride, lane, nblk, a.npad, a.target, ring, b > 0, b + 1 < a.nbands,
                                 cs, S, x);
    __syncwarp();
    if (!ok) break;
  }
  for (int d = 16; d > 0; d >>= 1) S = max(S, __shfl_xor_sync(0xffffffffu, S, d));
  if (lane == 0) atomicMax(a.best, S);
}

template <int R>
int configure_pair_one(int threads, size_t smem) {
  auto kern = pair_band_kernel<R>;
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

template <int R>
cudaError_t launch_pair_one(const PairBandArgs &a, int grid, int threads, size_t smem, cudaStream_t s) {
  void *args[] = {(void *)&a};
  return cudaLaunchCooperativeKernel((const void *)pair_band_kernel<R>, dim3(grid), dim3(threads), args, smem, s);
}

}  // namespace

size_t pair_smem_bytes(int pbuf_bytes, int warps) { return (size_t)warps * (pbuf_bytes + kBandRingBytes); }

int pair_max_ctas_per_sm(int R, int threads, size_t smem) {
  if (R == 4) return configure_pair_one<4>(threads, smem);
  if (R == 8) return configure_pair_one<8>(threads, smem);
  if (R == 16) return configure_pair_one<16>(threads, smem);
  if (R == 24) return configure_pair_one<24>(threads, smem);
  return 0;
}

cudaError_t launch_pair(const PairBandArgs &a, int R, int grid, int threads, size_t smem, cudaStream_t s) {
  if (R == 4) return launch_pair_one<4>(a, grid, threads, smem, s);
  if (R == 8) return launch_pair_one<8>(a, grid, threads, smem, s);
  if (R == 16) return launch_pair_one<16>(a, grid, threads, smem, s);
  if (R == 24) return launch_pair_one<24>(a, grid, threads, smem, s);
  return cudaErrorInvalidValue;
}

}  // namespace swgb
