// Internal declarations shared by the host API (api.cu) and the kernel
// translation units.  Not part of the public interface.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

struct sw_db;

namespace swgb {

constexpr int kAlphabet = 20;      // residue codes 0..19
constexpr int kPadCode = 20;       // pad residue: profile row of the most negative score
constexpr int kProfRows = 21;      // profile rows: 20 residues + pad
constexpr int kColBlock = 16;      // columns per unrolled block / residue vector
constexpr int kMinPad = 48;        // minimum padded database length (>= max lanes per chain + 16)
constexpr int kMaxLanesPerChain = 32;

// Scoring constants, derived once per query batch on the host.
struct Scoring {
  int32_t go;      // Go of Eqs. 2-3 = gap_open + gap_extend
  int32_t ge;      // Ge of Eqs. 2-3 = gap_extend
  int32_t pad;     // profile value of pad rows and the pad residue: min(0, min SM)
  int32_t maxp;    // max(0, max SM)
  int32_t thresh;  // a packed 16-bit lane may have wrapped only if its score S > thresh
};

// Per-query descriptor for the dynamic-programming kernels, or (query-track
// plans of the query-pair form) per plan.
struct QDesc {
  int32_t m;         // query length (track plans: nchunks * L * R)
  int32_t L;         // lanes per chain (1..32)
  int32_t R;         // rows per lane
  int32_t nchunks;   // ceil(m / (L*R)) (>= 1); track plans: chunks of the longer track
  int32_t chunk_bytes;  // bytes of one profile chunk = 21 * chunk_stride
  int32_t chunk_stride; // bytes per profile row within a chunk (>= L*R entries, multiple of 128)
  int64_t prof_off;  // byte offset of chunk 0 in the profile buffer
  int64_t qoff;      // offset of the query residues in the query residue buffer
  int32_t track_off; // track plans: index of the plan's first TrackChunk
  int32_t wide;      // solo plans: 1 = 32-bit entries (the score zero-extended in the low
                     // half) in the query-pair group layout; 0 = bytes
};

// Query tracks (query-pair form).  The two 16-bit halves of a chain each run
// a track: queries laid end to end, chunk by chunk (every query padded to
// whole chunks).  Chunk c of a plan computes chunk ka of query qa in the low
// half and chunk kb of query qb in the high half; a half whose query starts
// in the chunk takes the matrix top boundary instead of the boundary strip,
// and a half whose query ends in it has its scores written after it.
struct TrackChunk {
  int32_t qa, qb;  // query per half, -1 = idle
  int32_t ka, kb;  // chunk index within that query
  int32_t flags;   // kStartA | kStartB | kEndA | kEndB
  int32_t L;       // lanes per chain of the chunk's plan
  int32_t pad_[2];
};
constexpr int32_t kStartA = 1, kStartB = 2, kEndA = 4, kEndB = 8;

// Lane slots per profile row.  A chain of L <= 32 lanes shares its warp with
// 32/L - 1 other chains of the same query; the profile row holds one copy of
// the L lanes' entries per chain, so lane l of the warp reads slot l and the
// 32 lanes touch 32 distinct slots (no shared-memory bank conflict).  Chains
// of more than 32 lanes (the intra-task kernel) use one slot per lane.
__host__ __device__ inline int profile_slots(int L) { return L >= 32 ? L : (32 / L) * L; }

// Forms of the dynamic-programming kernels.
constexpr int kFormInt32 = 0;   // one database sequence per chain, 32-bit cells
constexpr int kFormPacked = 1;  // two database sequences per chain, 16-bit halves
constexpr int kFormQPair = 2;   // two queries per chain (one sequence), 16-bit halves
// host flag on kFormInt32 / kFormPacked for launch_inter and
// inter_max_ctas_per_sm: the queries' profiles hold 32-bit entries (the score
// zero-extended in the low half) in the query-pair form's group layout
constexpr int kFormWide = 16;
constexpr int32_t kStatusSaturated = 100;  // device status: a lane that could not saturate did
constexpr int32_t kStatusBounds = 101;     // device status (checked build): an index left its buffer

// A unit of DP work for one chain: one database sequence (int32 form) or
// two (packed form), given as positions in the length-sorted database.
struct Task {
  int32_t q;           // query index
  int32_t unit_begin;  // first unit of the tile
  int32_t unit_count;  // units in the tile (<= chains per CTA)
  int32_t pad_;
};

struct DbView {
  const uint8_t *res;   // packed residues, sorted order
  int64_t res_bytes;    // bytes of the packed residue buffer
  const int64_t *off;   // [n] byte offset of sorted sequence k (16-byte aligned)
  const int32_t *npad;  // [n] padded length (multiple of 16, >= kMinPad)
  const int32_t *len;   // [n] true length
  const int32_t *perm;  // [n] sorted position -> caller index
  int64_t n;
};

struct InterArgs {
  DbView db;
  const int32_t *unit_pos;  // packed: 2 sorted positions per unit; int32: 1 per unit
  const QDesc *qd;
  const TrackChunk *track;  // query-pair form: chunk descriptors of the track plans
  const Task *tasks;
  const int32_t *n_tasks;   // device word: number of tasks
  int32_t *task_counter;    // device word, zeroed before launch
  const uint8_t *prof;      // profile chunks (see QDesc)
  int32_t pbuf_bytes;       // shared-memory bytes per profile buffer (>= every chunk_bytes)
  int32_t pbuf_count;       // inter-task kernel: 2 = next chunk loads while the current one is in use, 1 = in turn
  uint2 *gbuf;              // chunk boundary scratch, per (CTA, chain slot): gbuf_stride entries
  int32_t gbuf_stride;
  int32_t *out;             // [nq][out_stride] scores in caller order
  int64_t out_stride;
  int32_t *flag_count;      // packed: [nq] number of flagged sequences per query
  int32_t *flag_pos;        // packed: [nq][flag_stride] flagged sorted positions
  int64_t flag_stride;
  Scoring sc;
  int32_t *status;          // device status word (SW_ETIMEOUT on an expired wait)
  // buffer sizes, tested by the checked build (-DSW_CHECK) before every access
  int64_t prof_bytes;       // bytes of `prof`
  int64_t out_size;         // entries of `out`
  int64_t n_unit_pos;       // entries of `unit_pos`
  int64_t flag_size;        // entries of `flag_pos`
};

// Arguments of the pair-band kernel (k_pair.cu): one long pair, int32 cells,
// one band of 32 * R query rows per warp.
struct PairBandArgs {
  const uint8_t *target;   // target codes padded with the pad code to npad (a multiple of 16)
  int32_t npad;
  int32_t nbands;
  const uint8_t *prof;     // nbands profile chunks of band_bytes = rows * stride (L = 32)
  int32_t band_bytes, stride, pbuf_bytes;
  unsigned long long *strips;  // [nslots][window] rings of tagged bottom-row entries, zeroed before launch
  int32_t nslots;          // >= (warps of the grid) + 1, or nbands
  int32_t window;          // columns per ring (a multiple of 16, >= 256)
  int32_t cons_every;      // blocks of 16 columns between hand-backs of consumed columns
  int32_t *cons;           // [nbands] columns consumed by the band below, zeroed before launch
  int32_t *best;           // max over all cells (atomicMax), zeroed before launch
  int32_t *status;         // SW_ETIMEOUT on an expired wait
  Scoring sc;
};
size_t pair_smem_bytes(int pbuf_bytes, int warps);
int pair_max_ctas_per_sm(int R, int threads, size_t smem);
cudaError_t launch_pair(const PairBandArgs &a, int R, int grid, int threads, size_t smem, cudaStream_t s);

// Band-stream kernel (k_band.cu): in small batches, a long query's rows (or a
// short query's against long database units) cut into bands of 32 lanes x R
// rows, one warp each, all bands of a job running as a pipeline over the
// job's stream of database units.
// BandJob::form
constexpr int32_t kBandInt32 = 0;      // one sequence per unit, int32 cells, bands of 32 R rows
constexpr int32_t kBandPacked = 1;     // two sequences per unit in the 16-bit halves (pairs that
                                       // cannot pass the 16-bit range), bands of 32 R rows
constexpr int32_t kBandInt32Half = 2;  // int32 as kBandInt32, bands of 32 R / 2 rows
struct BandJob {
  int32_t q;        // query: its rows are cut into the bands; its row of scores is written
  int32_t form;     // kBandInt32, kBandPacked or kBandInt32Half
  int32_t nb;       // bands (32 R or 32 R / 2 query rows each)
  int32_t t_begin;  // first unit in BandArgs::tpos
  int32_t t_count;  // units of the stream, in order
  int32_t band0;    // global index of the job's band 0
  int64_t ring0;    // entry offset of the job's ring 0 (between bands 0 and 1) in BandArgs::rings
  int64_t cols;     // columns of the stream (sum of the units' padded lengths): the length of each ring
};
struct BandArgs {
  DbView db;
  const int2 *tpos;           // units: sorted positions (A, B); B = A for one sequence
  const BandJob *jobs;
  const int32_t *band_job;    // [nbands] job of each global band (jobs' bands consecutive, in band order)
  int32_t nbands;
  int32_t *band_counter;      // device word, zeroed before the launch: hands out bands in index order
  const uint8_t *qres;        // query residues
  const QDesc *qd;            // m and qoff of every query
  const int8_t *submat;       // 20x20
  unsigned long long *rings;  // (nb - 1) rings of `cols` entries per job, zeroed before the launch
  int32_t *out;               // [nq][out_stride] scores in caller order; the jobs' rows zeroed before
  int64_t out_stride;
  Scoring sc;
  int32_t *status;            // SW_ETIMEOUT on an expired wait
  int32_t short_int;          // 1 (16-bit batches): int32 units with the one-operation F chain;
                              // 0 (int32 batches): Algorithm 1's statement order
  // buffer sizes, tested by the checked build (-DSW_CHECK) before every access
  int64_t ring_entries;       // entries of `rings`
  int64_t out_size;           // entries of `out`
  int64_t n_tpos;             // entries of `tpos`
};
// Transposed jobs of the band-stream kernel (k_band.cu): for the short queries
// of a small batch the database sequences are the rows -- stacked end to end
// in row tracks, each padded to whole lanes of R rows -- and the query is the
// columns.  A track is cut into bands of 32 lanes x R rows, one warp each; a
// lane whose first row starts a sequence takes the matrix top boundary instead
// of the row above, so one band holds several short sequences, and the bands
// of a sequence that spans several run as a pipeline, as above.
struct TrackLane {
  int32_t pa, ra;  // rows of the low half (int32: the only track): sorted position, first row (-1: idle lane)
  int32_t pb, rb;  // rows of the high half (16-bit halves only)
};
struct TrackJob {
  int32_t q;       // the query: the columns, and the row of scores written
  int32_t packed;  // 1: two row tracks in the 16-bit halves; 0: one track, int32 cells
  int32_t nb;      // bands
  int32_t band0;   // global index of the job's band 0
  int32_t lane0;   // band b's lanes at TrackArgs::lanes[lane0 + 32 b ...]
  int32_t pad_;
  int64_t ring0;   // entry offset of ring 0 (between bands 0 and 1); rings are qt_npad[q] long
};
struct TrackArgs {
  DbView db;                  // the rows' sequences
  const TrackLane *lanes;
  const TrackJob *jobs;
  const int32_t *band_job;    // [nbands] job of each global band
  int32_t nbands;
  int32_t *band_counter;      // zeroed before the launch
  const uint8_t *qt;          // queries padded to multiples of 16 with the pad code
  const int64_t *qt_off;      // [nq] offset of each padded query in qt
  const int32_t *qt_npad;     // [nq] padded length
  const int8_t *submat;       // 20x20 (row = query residue)
  unsigned long long *rings;  // zeroed before the launch
  int32_t *out;               // [nq][out_stride] caller order, the jobs' rows zeroed before (atomicMax)
  int64_t out_stride;
  Scoring sc;
  int32_t *status;
  // buffer sizes, tested by the checked build (-DSW_CHECK) before every access
  int64_t n_lanes, ring_entries, out_size, qt_bytes;
};
// R: rows per lane of the transposed jobs (8 or 16: bands of 256 or 512 database rows);
// split: each lane's rows as two half-chains a column apart (see column_step_split)
bool track_supported_R(int R);
int track_max_ctas_per_sm(int R, bool split);  // plan time: raises the shared-memory limit; 0 on failure
int track_threads();
cudaError_t launch_track(const TrackArgs &a, int R, bool split, int grid, cudaStream_t s);

int band_threads();
bool band_supported_R(int R);  // rows per lane: 8 or 16 (bands of 256 or 512 query rows)
size_t band_smem_bytes(int R);
int band_max_ctas_per_sm(int R);  // plan time: raises the shared-memory limit; 0 on failure
// one_per_sm: reserve shared memory so that the launch places at most one CTA per SM
cudaError_t launch_band(const BandArgs &a, int R, int grid, bool one_per_sm, cudaStream_t s);

// Traceback of selected hits (k_trace.cu): one warp per hit fills 4-bit
// provenance codes per cell, one thread per hit walks them back.
struct TraceHit {
  int64_t qoff;       // query residues in qres
  int64_t toff;       // target residues in tres (the database's sorted, padded residues)
  int64_t dir_off;    // bytes into dirs: mrow * npad / 2, column-major nibbles (row i of column j at j * mrow + i)
  int64_t strip_off;  // uint2 entries into strips: npad (bottom rows passed from the last warp to the first)
  int64_t ops_off;    // bytes into ops: m + n
  int32_t m, n, npad, mrow;  // query and target lengths, padded target length, rows padded to whole chunks
};
struct TraceResult {
  int32_t score, end_i, end_j;  // best score and its cell (1-based row, column; first in row-major order)
  int32_t begin_i, begin_j;     // the alignment covers rows begin_i+1 .. end_i, columns begin_j+1 .. end_j
  int32_t n_ops;                // -1: the fill gave up on a bounded wait
};
struct TraceArgs {
  const uint8_t *qres, *tres;
  const int8_t *submat;  // 20x20
  const TraceHit *hits;
  int32_t nhits;
  uint8_t *dirs;
  uint2 *strips;
  uint8_t *ops;
  TraceResult *results;
  Scoring sc;
};
int trace_rows_per_chunk();
int trace_warps(int max_chunks);  // warps per CTA of the fill: chunks of one hit in flight
size_t trace_smem_bytes(int warps);
cudaError_t launch_trace(const TraceArgs &a, int warps, cudaStream_t s);

// launchers (k_inter.cu)
int inter_threads();
bool inter_supported_R(int R);
// Steps between a chain's first lane reaching a column and its last lane
// leaving it (L - 1; 2 L - 1 for the split query-pair lanes).
int inter_chain_lag(int R, int form, int L);
size_t inter_smem_bytes(int pbuf_bytes, int pbuf_count, int threads);
cudaError_t launch_inter(const InterArgs &a, int R, int form, int grid, int threads, size_t smem,
                         cudaStream_t s);
// Raises the instantiation's shared-memory limit (plan time only) and returns resident CTAs per SM
// (0 on failure).
int inter_max_ctas_per_sm(int R, int form, int threads, size_t smem);

// intra-task kernel (k_intra.cu): one CTA of intra_threads() per (query, unit) task;
// QDesc::L = 32 * warps of the chain.
int intra_threads();
size_t intra_smem_bytes(int pbuf_bytes);
cudaError_t configure_intra(int R, bool packed);  // plan time: raise the shared-memory limit
cudaError_t launch_intra(const InterArgs &a, int R, bool packed, int grid, size_t smem, cudaStream_t s);

// support kernels (k_support.cu)
cudaError_t launch_build_profiles(const uint8_t *qres, const QDesc *qd, int32_t nq, const int8_t *submat,
                                  int32_t pad, uint8_t *prof, cudaStream_t s);
// Query-pair tables: per chunk [21][chunk_stride] bytes of 32-bit words
// (SM(Qa[i], c) & 0xffff) | (SM(Qb[i], c) << 16).
cudaError_t launch_build_track_profiles(const uint8_t *qres, const QDesc *qdq, const QDesc *plan,
                                        const TrackChunk *track, int32_t nchunks, const int8_t *submat, int32_t pad,
                                        uint8_t *prof, cudaStream_t s);
// Build rescue tasks from the per-query flag counts: tiles of warps_per_cta * (32 / L) flagged
// positions (units_per_task == 0) or of units_per_task positions; flagged positions of query q
// start at q * stride.  Writes the task count to *n_tasks and zeroes *counter.
cudaError_t launch_rescue_tasks(const int32_t *flag_count, const QDesc *qd, int32_t nq, int64_t stride,
                                int32_t warps_per_cta, int32_t units_per_task, Task *tasks, int32_t *n_tasks,
                                int32_t *counter, cudaStream_t s);

// Accessors for translation units other than api.cu (the sw_db layout is private to it).
const DbView &db_view(const struct ::sw_db *db);
int db_device(const struct ::sw_db *db);
// device [0, 1, ..., n - 1, n - 1]: sorted positions, usable as one-sequence units
const int32_t *db_ident(const struct ::sw_db *db);
int64_t db_sorted_pos(const struct ::sw_db *db, int64_t caller_index);  // caller order -> sorted position
int32_t db_sorted_len(const struct ::sw_db *db, int64_t pos);           // true length at a sorted position
int32_t db_sorted_npad(const struct ::sw_db *db, int64_t pos);          // padded length at a sorted position
int64_t db_sorted_off(const struct ::sw_db *db, int64_t pos);           // residue offset at a sorted position
// Record the thread's last error message (see sw_last_error) and return `code`.
int set_last_error(int code, const char *msg);
void clear_last_error();

}  // namespace swgb
