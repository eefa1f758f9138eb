// Support kernels: query-profile construction and rescue-task construction.
#include "internal.h"

namespace swgb {
namespace {

// Query profile (Sec. 2.2: the SM(Q[i], D[j]) term of Eq. 1, tabulated per
// database residue): signed byte P[c][i] = SM(Q[i], c) for residue c = 0..19
// and query row i; the pad residue (c = 20) and rows past the query end hold
// `pad` = min(0, min SM).  Layout per query: nchunks chunks, each
// [21][chunk_stride] bytes, chunk c covering rows c*L*R .. c*L*R + L*R - 1.
// A residue row holds profile_slots(L) slots of R bytes; slot s serves lane
// k = s mod L, i.e. rows k*R .. k*R + R - 1 of the chunk.  Bytes past the
// last slot hold `pad` too.
__global__ void build_profiles_kernel(const uint8_t *__restrict__ qres, const QDesc *__restrict__ qd,
                                      const int8_t *__restrict__ submat, int32_t pad,
                                      uint8_t *__restrict__ prof) {
  __shared__ int8_t sm[kAlphabet * kAlphabet];
  for (int i = threadIdx.x; i < kAlphabet * kAlphabet; i += blockDim.x) sm[i] = submat[i];
  __syncthreads();
  const QDesc d = qd[blockIdx.y];
  const uint8_t *q = qres + d.qoff;
  const int LR = d.L * d.R;
  const int slots = profile_slots(d.L);
  const int64_t words = (int64_t)d.nchunks * d.chunk_bytes / 4;
  uint32_t *out = reinterpret_cast<uint32_t *>(prof + d.prof_off);
  if (d.wide) {
    // 32-bit entries, the score zero-extended in the low half, in the group
    // layout of the query-track profile below (word j of group i of slot s at
    // word (i * slots + s) * 4 + j of the residue row: row (s mod L) * R +
    // 4 i + j of the chunk)
    const int cw = d.chunk_bytes / 4, rw = d.chunk_stride / 4;
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < words; w += (int64_t)gridDim.x * blockDim.x) {
      const int c = (int)(w / cw);
      const int rem = (int)(w - (int64_t)c * cw);
      const int rho = rem / rw;
      const int wi = rem - rho * rw;
      const int gi = wi / (4 * slots), slot = (wi >> 2) - gi * slots;
      const int x = (slot % d.L) * d.R + 4 * gi + (wi & 3);  // row within the chunk
      int32_t val = pad;
      if (wi < slots * d.R && rho < kAlphabet && c * LR + x < d.m) val = sm[q[c * LR + x] * kAlphabet + rho];
      out[w] = (uint32_t)val & 0xffffu;
    }
    return;
  }
  for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < words; w += (int64_t)gridDim.x * blockDim.x) {
    const int64_t x0 = 4 * w;
    const int c = (int)(x0 / d.chunk_bytes);
    const int rem = (int)(x0 - (int64_t)c * d.chunk_bytes);
    const int rho = rem / d.chunk_stride;
    const int xb = rem - rho * d.chunk_stride;
    uint32_t v = 0;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int slot = (xb + b) / d.R;
      const int row = c * LR + (slot % d.L) * d.R + (xb + b - slot * d.R);
      int32_t val = pad;
      if (slot < slots && row < d.m && rho < kAlphabet) val = sm[q[row] * kAlphabet + rho];
      v |= ((uint32_t)val & 0xffu) << (8 * b);
    }
    out[w] = v;
  }
}

// Query-track profile (query-pair form): for chunk c of a track plan, one
// 32-bit entry per (residue, row) holding SM(Qa[i], c) in the low and SM(Qb[i], c)
// in the high 16-bit half (both sign-extended), where Qa, Qb are the queries the
// two halves run in this chunk and i the row within that query's own chunk.
// Rows past a query's end, idle halves, the pad residue and unused entries hold
// `pad`.  Layout per chunk: [21][chunk_stride] bytes; within a residue row the
// lane slots' four-word groups are interleaved: with S = profile_slots(L)
// slots, word j of group i of slot s sits at word (i*S + s)*4 + j and holds row
// (s mod L)*R + 4*i + j of the chunk, so the lanes of a warp read 32
// consecutive 16-byte groups.  All plans share R and the chunk size and their
// chunks are stored in table order, so chunk c of the table (a block row,
// blockIdx.y, strided) sits at plan->prof_off + c * chunk_bytes; L comes with
// each chunk.
__global__ void build_track_profiles_kernel(const uint8_t *__restrict__ qres, const QDesc *__restrict__ qdq,
                                            const QDesc *__restrict__ plan, const TrackChunk *__restrict__ track,
                                            int32_t nchunks, const int8_t *__restrict__ submat, int32_t pad,
                                            uint8_t *__restrict__ prof) {
  __shared__ int8_t sm[kAlphabet * kAlphabet];
  for (int i = threadIdx.x; i < kAlphabet * kAlphabet; i += blockDim.x) sm[i] = submat[i];
  __syncthreads();
  const QDesc d = *plan;
  const int words = d.chunk_bytes / 4;
  for (int c = blockIdx.y; c < nchunks; c += gridDim.y) {
    const TrackChunk tc = track[c];
    const int LR = tc.L * d.R;
    const int slots = profile_slots(tc.L);
    const uint8_t *qa = tc.qa >= 0 ? qres + qdq[tc.qa].qoff : qres;
    const uint8_t *qb = tc.qb >= 0 ? qres + qdq[tc.qb].qoff : qres;
    const int ma = tc.qa >= 0 ? qdq[tc.qa].m : 0, mb = tc.qb >= 0 ? qdq[tc.qb].m : 0;
    const int ra = tc.ka * LR, rb = tc.kb * LR;  // first row of this chunk in each query
    uint32_t *out = reinterpret_cast<uint32_t *>(prof + d.prof_off + (int64_t)c * d.chunk_bytes);
    for (int w = blockIdx.x * blockDim.x + threadIdx.x; w < words; w += gridDim.x * blockDim.x) {
      const int rho = (4 * w) / d.chunk_stride;
      const int wi = (4 * w - rho * d.chunk_stride) / 4;
      const int gi = wi / (4 * slots), slot = (wi >> 2) - gi * slots;
      const int x = (slot % tc.L) * d.R + 4 * gi + (wi & 3);  // row within the chunk
      int32_t va = pad, vb = pad;
      if (wi < slots * d.R && rho < kAlphabet) {
        if (ra + x < ma) va = sm[qa[ra + x] * kAlphabet + rho];
        if (rb + x < mb) vb = sm[qb[rb + x] * kAlphabet + rho];
      }
      out[w] = ((uint32_t)va & 0xffffu) | ((uint32_t)vb << 16);
    }
  }
}

// One task per tile of up to chains-per-CTA flagged sequences of one query.
__global__ void rescue_tasks_kernel(const int32_t *__restrict__ flag_count, const QDesc *__restrict__ qd,
                                    int32_t nq, int64_t stride, int32_t warps_per_cta, int32_t units_per_task,
                                    Task *__restrict__ tasks,
                                    int32_t *__restrict__ n_tasks, int32_t *__restrict__ counter) {
  __shared__ int32_t part[1024];
  const int tid = threadIdx.x, nt = blockDim.x;
  const int per = (nq + nt - 1) / nt;
  const int q0 = min(nq, tid * per), q1 = min(nq, q0 + per);
  int32_t mine = 0;
  for (int q = q0; q < q1; ++q) {
    const int chains = units_per_task > 0 ? units_per_task : warps_per_cta * (32 / qd[q].L);
    mine += (flag_count[q] + chains - 1) / chains;
  }
  part[tid] = mine;
  __syncthreads();
  for (int off = 1; off < nt; off <<= 1) {  // inclusive scan
    const int32_t v = tid >= off ? part[tid - off] : 0;
    __syncthreads();
    part[tid] += v;
    __syncthreads();
  }
  int32_t base = part[tid] - mine;
  for (int q = q0; q < q1; ++q) {
    const int chains = units_per_task > 0 ? units_per_task : warps_per_cta * (32 / qd[q].L);
    const int cnt = flag_count[q];
    for (int t0 = 0; t0 < cnt; t0 += chains) {
      Task tk;
      tk.q = q;
      tk.unit_begin = (int32_t)(q * stride + t0);
      tk.unit_count = min(chains, cnt - t0);
      tk.pad_ = 0;
      tasks[base++] = tk;
    }
  }
  if (tid == nt - 1) {
    *n_tasks = part[tid];
    *counter = 0;
  }
}

}  // namespace

cudaError_t launch_build_profiles(const uint8_t *qres, const QDesc *qd, int32_t nq, const int8_t *submat,
                                  int32_t pad, uint8_t *prof, cudaStream_t s) {
  if (nq <= 0) return cudaSuccess;
  const int gx = (int)std::max<int64_t>(8, std::min<int64_t>(1024, 1024 / nq));  // few queries: more blocks each
  int64_t done = 0;
  while (done < nq) {  // grid.y is limited to 65535
    const int chunk = (int)std::min<int64_t>(65535, nq - done);
    dim3 grid(gx, chunk);
    build_profiles_kernel<<<grid, 256, 0, s>>>(qres, qd + done, submat, pad, prof);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    done += chunk;
  }
  return cudaSuccess;
}

cudaError_t launch_build_track_profiles(const uint8_t *qres, const QDesc *qdq, const QDesc *plan,
                                        const TrackChunk *track, int32_t nchunks, const int8_t *submat, int32_t pad,
                                        uint8_t *prof, cudaStream_t s) {
  if (nchunks <= 0) return cudaSuccess;
  dim3 grid(4, std::min(nchunks, 65535));
  build_track_profiles_kernel<<<grid, 256, 0, s>>>(qres, qdq, plan, track, nchunks, submat, pad, prof);
  return cudaGetLastError();
}

cudaError_t launch_rescue_tasks(const int32_t *flag_count, const QDesc *qd, int32_t nq, int64_t stride,
                                int32_t warps_per_cta, int32_t units_per_task, Task *tasks, int32_t *n_tasks,
                                int32_t *counter, cudaStream_t s) {
  rescue_tasks_kernel<<<1, 1024, 0, s>>>(flag_count, qd, nq, stride, warps_per_cta, units_per_task, tasks, n_tasks,
                                         counter);
  return cudaGetLastError();
}

}  // namespace swgb
