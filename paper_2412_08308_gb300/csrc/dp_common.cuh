// Cell arithmetic shared by the inter-task, intra-task and pair-band kernels:
// one column step of R query rows owned by one lane (Sec. 2.2 Eqs. 1-3), or,
// with split lanes, the lane's two halves of R/2 rows a column apart.
//
// int32 form: Algorithm 1's statements, one cell per lane op.
// packed form: two cells per 32-bit word, each 16-bit half a signed cell value.
// On sm_103 the integer ALU pipe (which executes every max, PRMT and IADD)
// issues a warp instruction every second cycle, and the FMA pipe is a second
// pipe of the same width that executes the per-half 16x2 adds (__vadd2 /
// __vsub2).  So a word update spends its 5 maxima on the ALU pipe (the zero
// floor of Eq. 1 is free in __vimax_s16x2_relu) and its 4 additions on the FMA
// pipe.  Per-half adds never carry into the other half; a half whose running
// score exceeds 32767 - max(SM) may have wrapped and is recomputed in int32.
#pragma once

#include <cstdint>
#include <type_traits>

#include "internal.h"

namespace swgb {

constexpr uint32_t kPadPair = 20u | (20u << 16);

// Checked build (-DSW_CHECK): every index into a packed residue buffer, a
// profile, a boundary strip or ring, or an output is tested before the
// access; an index outside its buffer records kStatusBounds in the status
// word and the access is skipped (no trap, no assert).  The regular build
// compiles the tests away.
#ifdef SW_CHECK
constexpr bool kChecked = true;
#else
constexpr bool kChecked = false;
#endif

__device__ __forceinline__ bool in_range(int64_t i, int64_t n, int32_t *status) {
  if constexpr (kChecked) {
    if (i < 0 || i >= n) {
      atomicExch(status, kStatusBounds);
      return false;
    }
  }
  return true;
}

// Profile row codes of a column (0..20, 20 = pad), as the form reads them:
// the low byte (int32 forms), the two 16-bit halves (two sequences per word)
// or the whole word (query pairs, one bare code).  A code past the pad row is
// reported and replaced by the pad code.
template <int FORM>
__device__ __forceinline__ uint32_t checked_codes(uint32_t res, int32_t *status) {
  if constexpr (kChecked) {
    bool bad;
    if constexpr (FORM == kFormPacked) bad = (res & 0xffffu) > (uint32_t)kPadCode || (res >> 16) > (uint32_t)kPadCode;
    else if constexpr (FORM == kFormQPair) bad = res > (uint32_t)kPadCode;
    else bad = (res & 0xffu) > (uint32_t)kPadCode;
    if (bad) {
      atomicExch(status, kStatusBounds);
      return FORM == kFormPacked ? kPadPair : (uint32_t)kPadCode;
    }
  }
  return res;
}

struct Consts {
  // packed: (x, x) in both 16-bit halves
  uint32_t goW, geW, F0W, E0W;
  // int32
  int32_t go, ge;
};

__device__ __forceinline__ Consts make_consts(const Scoring &sc) {
  Consts c;
  c.goW = (uint32_t)sc.go * 0x10001u;
  c.geW = (uint32_t)sc.ge * 0x10001u;
  const uint32_t ngo = (uint32_t)(-sc.go) & 0xffffu;  // E, F start at -Go (any value <= 0 works)
  c.F0W = ngo | (ngo << 16);
  c.E0W = c.F0W;
  c.go = sc.go;
  c.ge = sc.ge;
  return c;
}

// PTX prmt.b32 (default mode): each selector nibble picks one of the 8 bytes
// {b, a}; a set nibble msb replicates the sign of the picked byte instead.
// (CUDA's __byte_perm masks the nibbles to 3 bits, so it cannot express the
// sign-replicate form used here.)
__device__ __forceinline__ uint32_t prmt(uint32_t a, uint32_t b, uint32_t sel) {
  uint32_t d;
  asm("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(sel));
  return d;
}

// Selectors.  pair(i) -> (byte i of a, its sign, byte i of b, its sign): the two
// bytes sign-extended into the 16-bit halves (residue codes < 128 come out
// zero-extended).  sext(i) -> byte i of a sign-extended to 32 bits.
// one(i) -> byte i of a, zero-extended from b = 0.
__host__ __device__ constexpr uint32_t sel_pair(int i) {
  return (uint32_t)i | ((uint32_t)(i | 8) << 4) | ((uint32_t)(4 + i) << 8) | ((uint32_t)((4 + i) | 8) << 12);
}
__host__ __device__ constexpr uint32_t sel_sext(int i) {
  return (uint32_t)i | ((uint32_t)(i | 8) << 4) | ((uint32_t)(i | 8) << 8) | ((uint32_t)(i | 8) << 12);
}
__host__ __device__ constexpr uint32_t sel_one(int i) { return 0x4440u | (uint32_t)i; }
// the low 16-bit half of a, sign-extended to 32 bits
__host__ __device__ constexpr uint32_t sel_sext16() { return 0x9910u; }

// R 32-bit profile entries of one residue in the wide layout (R/4 16-byte
// groups, `gstride` bytes apart: the lanes' groups interleaved)
template <int N>
__device__ __forceinline__ void load_groups(const uint8_t *p, int gstride, uint32_t (&w)[N]) {
  static_assert(N % 4 == 0, "whole groups");
#pragma unroll
  for (int i = 0; i < N / 4; ++i) {
    const uint4 v = *reinterpret_cast<const uint4 *>(p + i * gstride);
    w[4 * i + 0] = v.x; w[4 * i + 1] = v.y; w[4 * i + 2] = v.z; w[4 * i + 3] = v.w;
  }
}

template <int R>
__device__ __forceinline__ void load_prof(const uint8_t *p, uint32_t (&w)[R / 4]) {
  static_assert(R % 4 == 0, "rows per lane must be a multiple of 4");
  if constexpr (R % 16 == 0) {
#pragma unroll
    for (int i = 0; i < R / 16; ++i) {
      const uint4 v = reinterpret_cast<const uint4 *>(p)[i];
      w[4 * i + 0] = v.x; w[4 * i + 1] = v.y; w[4 * i + 2] = v.z; w[4 * i + 3] = v.w;
    }
  } else if constexpr (R % 8 == 0) {
#pragma unroll
    for (int i = 0; i < R / 8; ++i) {
      const uint2 v = reinterpret_cast<const uint2 *>(p)[i];
      w[2 * i + 0] = v.x; w[2 * i + 1] = v.y;
    }
  } else {
#pragma unroll
    for (int i = 0; i < R / 4; ++i) w[i] = reinterpret_cast<const uint32_t *>(p)[i];
  }
}

// N profile bytes at byte OFF of an 8-byte-aligned slot, as N/4 words, by the
// widest aligned loads (the halves of a 24-byte slot start at 0 and 12).
template <int N, int OFF, int W = 0>
__device__ __forceinline__ void load_prof_at(const uint8_t *p, uint32_t (&w)[N / 4]) {
  static_assert(N % 4 == 0 && OFF % 4 == 0, "whole words");
  constexpr int b = 4 * W;
  if constexpr (b < N) {
    if constexpr ((OFF + b) % 8 == 0 && b + 8 <= N) {
      const uint2 v = *reinterpret_cast<const uint2 *>(p + OFF + b);
      w[W] = v.x;
      w[W + 1] = v.y;
      load_prof_at<N, OFF, W + 2>(p, w);
    } else {
      w[W] = *reinterpret_cast<const uint32_t *>(p + OFF + b);
      load_prof_at<N, OFF, W + 1>(p, w);
    }
  }
}

__device__ __forceinline__ uint32_t word_of(const uint4 &v, int i) {
  return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w;
}

// N rows [R0, R0 + N) of one column, 32-bit words of two 16-bit cells
// (Eqs. 1-3 per half).  hd0 is H of the row above R0 at the previous column,
// p the rows' substitution words; E (per row, this column) and f (passed down
// the column) are updated in place, S keeps the running best.  Per word five
// maxima, the zero floor riding on the one with F, and four per-half
// additions, H - Go shared by the E and F updates.  The terms that do not
// depend on the row above, max(H_diag + SM, E), are formed for all N rows
// first: the previous column's H is then dead before any row is rewritten
// (no register copies), and only max(., F), the subtraction and the F update
// remain on the chain down the rows.  (Computing the next F from
// max(hd + p, E, 0) - Go instead of H - Go, which is equal because Ge <= Go,
// shortens that chain further but costs a fifth addition and measured
// slower.)
template <int R0, int N, int R>
__device__ __forceinline__ void word_rows(uint32_t hd0, const uint32_t (&p)[N], uint32_t (&E)[R],
                                          uint32_t (&Hl)[R], uint32_t &f, uint32_t &S, const Consts &cs) {
  static_assert(R0 + N <= R, "rows in range");
  uint32_t tt[N];
  tt[0] = __vmaxs2(__vadd2(hd0, p[0]), E[R0]);
#pragma unroll
  for (int r = 1; r < N; ++r) tt[r] = __vmaxs2(__vadd2(Hl[R0 + r - 1], p[r]), E[R0 + r]);
#pragma unroll
  for (int r = 0; r < N; ++r) {
    const uint32_t h = __vimax_s16x2_relu(tt[r], f);  // max(H_diag + SM, E, F, 0)
    S = __vmaxs2(S, h);
    const uint32_t hgo = __vsub2(h, cs.goW);
    E[R0 + r] = __vmaxs2(__vsub2(E[R0 + r], cs.geW), hgo);
    f = __vmaxs2(__vsub2(f, cs.geW), hgo);
    Hl[R0 + r] = h;
  }
}

// word_rows with a one-operation chain down the rows, for kernels bound by
// one chain's latency rather than by throughput (the band-stream and
// transposed jobs of small batches).  U = max(H_diag + SM, E, 0) does not
// depend on the row above; since Ge <= Go, the F passed down is
// max(F - Ge, H - Go) = max(F - Ge, U - Go, F - Go) = max(F - Ge, U - Go), so
// the only operation on the chain is that max-add, and H = max(U, F), the
// running best and E' = max(E - Ge, H - Go) hang off it.  Same five maxima
// per word as word_rows, one more addition (U - Go beside H - Go).
template <int R0, int N, int R>
__device__ __forceinline__ void word_rows_short(uint32_t hd0, const uint32_t (&p)[N], uint32_t (&E)[R],
                                                uint32_t (&Hl)[R], uint32_t &f, uint32_t &S, const Consts &cs) {
  static_assert(R0 + N <= R, "rows in range");
  uint32_t u[N];
  u[0] = __vimax_s16x2_relu(__vadd2(hd0, p[0]), E[R0]);  // max(H_diag + SM, E, 0)
#pragma unroll
  for (int r = 1; r < N; ++r) u[r] = __vimax_s16x2_relu(__vadd2(Hl[R0 + r - 1], p[r]), E[R0 + r]);
#pragma unroll
  for (int r = 0; r < N; ++r) {
    const uint32_t h = __vmaxs2(u[r], f);  // H = max(U, F)
    f = __vmaxs2(__vsub2(f, cs.geW), __vsub2(u[r], cs.goW));
    S = __vmaxs2(S, h);
    E[R0 + r] = __vmaxs2(__vsub2(E[R0 + r], cs.geW), __vsub2(h, cs.goW));
    Hl[R0 + r] = h;
  }
}

template <int FORM>
using Word = typename std::conditional<FORM != kFormInt32, uint32_t, int32_t>::type;

// N rows [R0, R0 + N) of one column in int32, Algorithm 1 statement by
// statement.  hul is H of the row above R0 at the previous column, (hu, fu) H
// and F of that row at this column (replaced by those of row R0 + N - 1); pb
// the rows' profile bytes, four per word; E and Hl hold the previous column's
// E and H per row and are updated in place; S keeps the running best.
// sm_of(r): the substitution score of row R0 + r (one sign extension on the
// ALU pipe from a profile byte, or from the low half of a 32-bit entry).
template <int R0, int N, int R, class SmOf>
__device__ __forceinline__ void int_rows_of(int32_t hul, SmOf sm_of, int32_t (&E)[R], int32_t (&Hl)[R], int32_t &hu,
                                            int32_t &fu, int32_t &S, const Consts &cs) {
  static_assert(R0 + N <= R, "rows in range");
#pragma unroll
  for (int r = 0; r < N; ++r) {
    const int32_t sm = sm_of(r);
    const int32_t e1 = E[R0 + r] - cs.ge;
    const int32_t e2 = Hl[R0 + r] - cs.go;
    const int32_t e = max(e1, e2);
    const int32_t f1 = fu - cs.ge;
    const int32_t f2 = hu - cs.go;
    const int32_t f = max(f1, f2);
    int32_t h = hul + sm;
    h = max(h, e);
    h = max(h, f);
    h = max(h, 0);
    S = max(S, h);
    hul = Hl[R0 + r];
    Hl[R0 + r] = h;
    E[R0 + r] = e;
    hu = h;
    fu = f;
  }
}

template <int R0, int N, int R>
__device__ __forceinline__ void int_rows(int32_t hul, const uint32_t (&pb)[N / 4], int32_t (&E)[R], int32_t (&Hl)[R],
                                         int32_t &hu, int32_t &fu, int32_t &S, const Consts &cs) {
  static_assert(N % 4 == 0, "whole profile words");
  int_rows_of<R0, N, R>(hul, [&](int r) { return (int32_t)prmt(pb[r >> 2], 0u, sel_sext(r & 3)); }, E, Hl, hu, fu, S,
                        cs);
}

// int_rows with the one-operation F chain of word_rows_short, for the int32
// units of the 16-bit path's small-batch jobs (pairs that could pass the
// 16-bit range): the F of the row below is max(F - Ge, U - Go) with
// U = max(H_diag + SM, E, 0), equal to Eq. 3's max(F - Ge, H - Go) because
// H = max(U, F) and Ge <= Go; U does not depend on the row above, so the
// chain down the rows is one subtraction and one maximum per row.  Same
// interface and operation count as int_rows (the plain int32 form keeps
// Algorithm 1's statement order).
template <int R0, int N, int R>
__device__ __forceinline__ void int_rows_short(int32_t hul, const uint32_t (&pb)[N / 4], int32_t (&E)[R],
                                               int32_t (&Hl)[R], int32_t &hu, int32_t &fu, int32_t &S,
                                               const Consts &cs) {
  static_assert(R0 + N <= R && N % 4 == 0, "rows in range, whole profile words");
  int32_t f = max(fu - cs.ge, hu - cs.go);  // the first row's F from the (H, F) above (Eq. 3)
#pragma unroll
  for (int r = 0; r < N; ++r) {
    const int32_t sm = (int32_t)prmt(pb[r >> 2], 0u, sel_sext(r & 3));
    const int32_t e = max(E[R0 + r] - cs.ge, Hl[R0 + r] - cs.go);
    const int32_t u = max(max(hul + sm, e), 0);
    const int32_t h = max(u, f);
    S = max(S, h);
    hul = Hl[R0 + r];
    Hl[R0 + r] = h;
    E[R0 + r] = e;
    if (r + 1 < N) {
      f = max(f - cs.ge, u - cs.go);
    } else {
      hu = h;
      fu = f;
    }
  }
}

// Per-lane DP state of R rows.
template <int R, int FORM>
struct LaneState {
  Word<FORM> Hl[R];  // H of each row at the previous column
  Word<FORM> E[R];   // packed: E of each row at the current column; int32: E at the previous column
  Word<FORM> hdiag;  // H of the row above this lane's first row, previous column
};

template <int R, int FORM>
__device__ __forceinline__ void lane_reset(LaneState<R, FORM> &st, const Consts &cs) {
  using W = Word<FORM>;
  constexpr bool PACKED = FORM != kFormInt32;
  const W E0 = PACKED ? (W)cs.E0W : (W)0;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    st.Hl[r] = (W)0;
    st.E[r] = E0;
  }
  st.hdiag = (W)0;
}

// One column: inputs are the (H, F) pair passed down from the row above this
// lane's rows and the residue code(s) of the column; prow points at this
// lane's R profile entries of residue row 0 (rows are `stride` bytes apart).
// Query-pair form: res is the bare residue code (no second code in the high
// half); prow points at this lane's first 16-byte group of four words; its
// R/4 groups are `gstride` bytes apart (lanes interleaved, so the
// 32 lanes of a warp read 32 consecutive 16-byte groups: no bank conflict).
// Outputs the (H, F) pair for the row below: int32 passes (H, F) of the last
// row; packed passes (H of the last row, F of the row below it).
// SHORTF: rows by word_rows_short / int_rows_short, the one-operation chain.
// WIDE (two-sequence and int32 forms): the profile holds 32-bit entries, the
// score in the low 16-bit half (zero-extended), in the query-pair form's
// group layout; the two sequences' entries are paired by one multiply-add
// (FMA pipe) instead of a byte shuffle (ALU pipe).
template <int R, int FORM, bool SHORTF = false, bool WIDE = false>
__device__ __forceinline__ void column_step(LaneState<R, FORM> &st, const uint8_t *prow, int stride,
                                            uint32_t res, Word<FORM> inH, Word<FORM> inF, const Consts &cs,
                                            Word<FORM> &S, Word<FORM> &outH, Word<FORM> &outF, int gstride = 0) {
  using W = Word<FORM>;
  if constexpr (FORM == kFormQPair) {
    // the two queries' scores for this column's residue, one word per row
    uint32_t pw[R];
#pragma unroll
    for (int i = 0; i < R / 4; ++i) {
      const uint4 v = *reinterpret_cast<const uint4 *>(prow + res * stride + i * gstride);
      pw[4 * i + 0] = v.x; pw[4 * i + 1] = v.y; pw[4 * i + 2] = v.z; pw[4 * i + 3] = v.w;
    }
    uint32_t f = (uint32_t)inF, s = (uint32_t)S;
    if constexpr (SHORTF) word_rows_short<0, R>((uint32_t)st.hdiag, pw, st.E, st.Hl, f, s, cs);
    else word_rows<0, R>((uint32_t)st.hdiag, pw, st.E, st.Hl, f, s, cs);
    S = (W)s;
    outH = st.Hl[R - 1];
    outF = (W)f;
  } else if constexpr (FORM == kFormPacked) {
    uint32_t pw[R];
    if constexpr (WIDE) {
      uint32_t pa[R], pb[R];
      load_groups<R>(prow + (res & 0xffu) * stride, gstride, pa);
      load_groups<R>(prow + (res >> 16) * stride, gstride, pb);
#pragma unroll
      for (int r = 0; r < R; ++r) pw[r] = pb[r] * 0x10000u + pa[r];  // (SM_a, SM_b)
    } else {
      uint32_t pa[R / 4], pb[R / 4];
      load_prof<R>(prow + (res & 0xffu) * stride, pa);
      load_prof<R>(prow + (res >> 16) * stride, pb);
#pragma unroll
      for (int r = 0; r < R; ++r) pw[r] = prmt(pa[r >> 2], pb[r >> 2], sel_pair(r & 3));  // (SM_a, SM_b), signed halves
    }
    uint32_t f = (uint32_t)inF, s = (uint32_t)S;
    if constexpr (SHORTF) word_rows_short<0, R>((uint32_t)st.hdiag, pw, st.E, st.Hl, f, s, cs);
    else word_rows<0, R>((uint32_t)st.hdiag, pw, st.E, st.Hl, f, s, cs);
    S = (W)s;
    outH = st.Hl[R - 1];
    outF = (W)f;
  } else if constexpr (WIDE) {
    static_assert(!SHORTF, "the wide int32 rows follow Algorithm 1");
    uint32_t pw[R];
    load_groups<R>(prow + (res & 0xffu) * stride, gstride, pw);
    int32_t hu = inH, fu = inF, s = S;
    int_rows_of<0, R, R>(st.hdiag, [&](int r) { return (int32_t)prmt(pw[r], 0u, sel_sext16()); }, st.E, st.Hl, hu,
                         fu, s, cs);
    S = (W)s;
    outH = (W)hu;
    outF = (W)fu;
  } else {
    uint32_t pa[R / 4];
    load_prof<R>(prow + (res & 0xffu) * stride, pa);
    int32_t hu = inH, fu = inF, s = S;
    if constexpr (SHORTF) int_rows_short<0, R>(st.hdiag, pa, st.E, st.Hl, hu, fu, s, cs);
    else int_rows<0, R>(st.hdiag, pa, st.E, st.Hl, hu, fu, s, cs);
    S = (W)s;
    outH = (W)hu;
    outF = (W)fu;
  }
  st.hdiag = inH;
}

// 16-bit forms with two independent half-chains per lane: rows [0, R/2) at
// column c and rows [R/2, R) at column c - 1, one step behind, so that the
// two F/H dependency chains down the rows interleave.  The upper half's F
// output and its bottom H feed the lower half one step later (midF, hdiagB);
// the lane passes on the lower half's bottom row, of column c - 1, so lane
// k + 1 works two columns behind lane k.  resA / resB: the residue code(s) of
// column c / c - 1.  S and S2 keep the halves' running best.
template <int R, int FORM, bool WIDE = false>
__device__ __forceinline__ void column_step_split(LaneState<R, FORM> &st, uint32_t &hdiagB, uint32_t &midF,
                                                  const uint8_t *prow, int stride, uint32_t resA, uint32_t resB,
                                                  uint32_t inH, uint32_t inF, const Consts &cs, uint32_t &S,
                                                  uint32_t &S2, uint32_t &outH, uint32_t &outF, int gstride) {
  static_assert(FORM != kFormInt32 && R % 8 == 0, "16-bit forms, halves of whole 4-row groups");
  constexpr int H2 = R / 2;
  // substitution words of the upper half (column c) and the lower half (column c - 1)
  uint32_t pa[H2], pb[H2];
  if constexpr (FORM == kFormQPair) {
#pragma unroll
    for (int i = 0; i < H2 / 4; ++i) {
      const uint4 v = *reinterpret_cast<const uint4 *>(prow + resA * stride + i * gstride);
      pa[4 * i + 0] = v.x; pa[4 * i + 1] = v.y; pa[4 * i + 2] = v.z; pa[4 * i + 3] = v.w;
      const uint4 w = *reinterpret_cast<const uint4 *>(prow + resB * stride + (H2 / 4 + i) * gstride);
      pb[4 * i + 0] = w.x; pb[4 * i + 1] = w.y; pb[4 * i + 2] = w.z; pb[4 * i + 3] = w.w;
    }
  } else if constexpr (WIDE) {
    // two database sequences, 32-bit entries: each word pairs them by one multiply-add
    uint32_t a0[H2], a1[H2], b0[H2], b1[H2];
    load_groups<H2>(prow + (resA & 0xffu) * stride, gstride, a0);
    load_groups<H2>(prow + (resA >> 16) * stride, gstride, a1);
    load_groups<H2>(prow + (resB & 0xffu) * stride + (H2 / 4) * gstride, gstride, b0);
    load_groups<H2>(prow + (resB >> 16) * stride + (H2 / 4) * gstride, gstride, b1);
#pragma unroll
    for (int r = 0; r < H2; ++r) {
      pa[r] = a1[r] * 0x10000u + a0[r];
      pb[r] = b1[r] * 0x10000u + b0[r];
    }
  } else {
    // two database sequences: each word pairs their profile bytes (PRMT)
    uint32_t a0[H2 / 4], a1[H2 / 4], b0[H2 / 4], b1[H2 / 4];
    load_prof_at<H2, 0>(prow + (resA & 0xffu) * stride, a0);
    load_prof_at<H2, 0>(prow + (resA >> 16) * stride, a1);
    load_prof_at<H2, H2>(prow + (resB & 0xffu) * stride, b0);
    load_prof_at<H2, H2>(prow + (resB >> 16) * stride, b1);
#pragma unroll
    for (int r = 0; r < H2; ++r) {
      pa[r] = prmt(a0[r >> 2], a1[r >> 2], sel_pair(r & 3));
      pb[r] = prmt(b0[r >> 2], b1[r >> 2], sel_pair(r & 3));
    }
  }
  const uint32_t diagB_next = st.Hl[H2 - 1];  // H of the upper half's last row at column c - 1
  // lower half first in program order (its inputs are ready), then the upper
  uint32_t f = midF, s2 = S2;
  word_rows<H2, H2>(hdiagB, pb, st.E, st.Hl, f, s2, cs);
  outH = st.Hl[R - 1];
  outF = f;
  S2 = s2;
  f = inF;
  uint32_t s = S;
  word_rows<0, H2>(st.hdiag, pa, st.E, st.Hl, f, s, cs);
  S = s;
  midF = f;
  hdiagB = diagB_next;
  st.hdiag = inH;
}

// int32 form with split lanes (the pair-band kernel): rows [0, R/2) at column
// c, rows [R/2, R) at column c - 1.  The upper half's last row (H, F) of the
// step before (midH, midF) and its H of the step before that (hdiagB) feed
// the lower half; the lane passes on the lower half's last row, of column
// c - 1.  resA / resB: the residue code of column c / c - 1.
template <int R>
__device__ __forceinline__ void column_step_split_int(LaneState<R, kFormInt32> &st, int32_t &hdiagB, int32_t &midH,
                                                      int32_t &midF, const uint8_t *prow, int stride, uint32_t resA,
                                                      uint32_t resB, int32_t inH, int32_t inF, const Consts &cs,
                                                      int32_t &S, int32_t &S2, int32_t &outH, int32_t &outF) {
  static_assert(R % 8 == 0, "halves of whole profile words");
  constexpr int H2 = R / 2;
  uint32_t pa[H2 / 4], pb[H2 / 4];
  load_prof_at<H2, 0>(prow + (resA & 0xffu) * stride, pa);
  load_prof_at<H2, H2>(prow + (resB & 0xffu) * stride, pb);
  // lower half first in program order (its inputs are ready), then the upper
  int32_t hu = midH, fu = midF, s2 = S2;
  int_rows<H2, H2>(hdiagB, pb, st.E, st.Hl, hu, fu, s2, cs);
  outH = hu;
  outF = fu;
  S2 = s2;
  hdiagB = midH;
  hu = inH;
  fu = inF;
  int32_t s = S;
  int_rows<0, H2>(st.hdiag, pa, st.E, st.Hl, hu, fu, s, cs);
  S = s;
  midH = hu;
  midF = fu;
  st.hdiag = inH;
}

template <int FORM>
__device__ __forceinline__ Word<FORM> score_max(Word<FORM> a, Word<FORM> b) {
  if constexpr (FORM != kFormInt32) return (Word<FORM>)__vmaxs2((uint32_t)a, (uint32_t)b);
  else return max(a, b);
}

// Epilogue for one database unit: flag possible overflows (packed) and scatter
// to caller order.  (The query-pair form writes its scores per query-track
// chunk, in the inter-task kernel.)
template <int FORM>
__device__ __forceinline__ void write_scores(Word<FORM> S, int posA, int posB, int q, const QDesc &qd,
                                             const InterArgs &a) {
  static_assert(FORM != kFormQPair, "query-pair scores are written per track chunk");
  constexpr bool PACKED = FORM == kFormPacked;
  const DbView &db = a.db;
  const Scoring &sc = a.sc;
  int32_t *out = a.out;
  int32_t *flag_count = a.flag_count;
  int32_t *flag_pos = a.flag_pos;
  const int64_t row = (int64_t)q * a.out_stride;
  const int64_t frow = (int64_t)q * a.flag_stride;
  if (!in_range(posA, db.n, a.status) || !in_range(posB, db.n, a.status)) return;
  if constexpr (PACKED) {
    const int32_t sa = (int32_t)((uint32_t)S & 0xffffu), sb = (int32_t)((uint32_t)S >> 16);
    if (sa > sc.thresh) {
      const int i = atomicAdd(&flag_count[q], 1);
      if (in_range(frow + i, a.flag_size, a.status)) flag_pos[frow + i] = posA;
    }
    if (in_range(row + db.perm[posA], a.out_size, a.status)) out[row + db.perm[posA]] = sa;
    if (posB != posA) {
      if (sb > sc.thresh) {
        const int i = atomicAdd(&flag_count[q], 1);
        if (in_range(frow + i, a.flag_size, a.status)) flag_pos[frow + i] = posB;
      }
      if (in_range(row + db.perm[posB], a.out_size, a.status)) out[row + db.perm[posB]] = sb;
    }
  } else {
    if (in_range(row + db.perm[posA], a.out_size, a.status)) out[row + db.perm[posA]] = (int32_t)S;
  }
}

}  // namespace swgb
