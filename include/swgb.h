/*
 * swgb -- score-only Smith-Waterman protein database search on one GB300.
 *
 * The operation (Sec. 2.2, Eqs. 1-3 of "SYCL vs CUDA performance portability
 * with SW#", arXiv 2412.08308): for every query Q (length m) and every
 * database sequence D (length n) compute the local alignment score
 *
 *   S(Q, D) = max over i, j of H[i][j], with
 *   H[i][j] = max(0, H[i-1][j-1] + SM(Q[i], D[j]), E[i][j], F[i][j])   (Eq. 1)
 *   E[i][j] = max(H[i][j-1] - Go, E[i][j-1] - Ge)                      (Eq. 2)
 *   F[i][j] = max(H[i-1][j] - Go, F[i-1][j] - Ge)                      (Eq. 3)
 *
 * with H, E, F = 0 on row 0 and column 0.  The paper's database search scores
 * proteins with BLOSUM62 and gap penalties 10/2 (Sec. 4.1).
 *
 * Conventions of this interface
 * -----------------------------
 *  - Residues are uint8 codes 0..19 (the caller's alphabet order).  Any other
 *    code is rejected with SW_EINVAL.  Zero-length sequences are legal and
 *    score 0.
 *  - submat is a row-major 20x20 int8 table: row = query residue, column =
 *    database residue.  Entries must lie in [-64, 63].
 *  - Gaps: a run of k gap positions costs gap_open + k * gap_extend.  In Eqs.
 *    2-3 that is Go = gap_open + gap_extend, Ge = gap_extend; "10/2" gives
 *    10 + 2k.  Both penalties must be >= 0 and gap_open + 2*gap_extend <= 1024.
 *  - Sequence sets are passed as one concatenated residue array plus an int64
 *    offset array with n+1 entries (offsets[0] = 0, non-decreasing,
 *    offsets[n] = total residues).
 *  - Scores are int32, laid out [n_queries][n_db] in the caller's order.
 *  - Every entry point returns an SW_* status; on failure sw_last_error()
 *    gives a message (thread-local, valid until the next call on the thread).
 *    Nothing is thrown across this interface.
 *  - One CUDA device: the current device of the calling thread when the
 *    database is prepared.  All work is ordered on the caller's stream
 *    (a cudaStream_t passed as void*; NULL = legacy default stream).
 *
 * Ownership: the caller owns every buffer it passes.  sw_db and sw_queries
 * own the device memory they allocate and release it in their *_free call.
 * Handles are not thread-safe: use one handle per thread or serialise.
 */
#ifndef SWGB_H
#define SWGB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define SW_OK 0
#define SW_EINVAL 1   /* invalid argument: bad code, offsets, penalties, sizes, pointers */
#define SW_ENOMEM 2   /* device or host allocation failed */
#define SW_ECUDA 3    /* a CUDA runtime call failed */
#define SW_ETIMEOUT 4 /* a bounded device-side wait expired; results are invalid */

/* arithmetic forms of the dynamic-programming kernels */
#define SW_MODE_INT32 0  /* plain 32-bit cells: the paper's Algorithm 1 body, one cell per lane op */
#define SW_MODE_PACKED 1 /* two 16-bit cells per 32-bit word, saturation flags, exact int32 rescue */

typedef struct sw_db sw_db;
typedef struct sw_queries sw_queries;

/*
 * sw_db_prepare -- pack a protein database into device memory (one-time).
 *
 * Sorts the sequences by length, pads each to a multiple of 16 residues with
 * a neutral pad code, and uploads the packed residues, the permutation back
 * to caller order and per-sequence metadata to the current device.  The
 * packed database stays resident until sw_db_free.  (Sec. 3.1: SW# assigns
 * database sequences to its kernels by length.)
 *
 *   residues  host pointer, offsets[n_seqs] bytes of codes 0..19
 *   offsets   host pointer, n_seqs + 1 int64 entries
 *   n_seqs    >= 0 (an empty database is legal)
 *   stream    cudaStream_t for the upload; the call returns after it completes
 *   out       receives the new handle
 *
 * Errors: SW_EINVAL (null pointers, bad offsets or codes), SW_ENOMEM, SW_ECUDA.
 */
int sw_db_prepare(const uint8_t *residues, const int64_t *offsets, int64_t n_seqs,
                  void *stream, sw_db **out);

/*
 * sw_db_free -- release a database made by sw_db_prepare and its device
 * memory (the protein database of the paper's search, Sec. 4.1, which stays
 * resident between searches here).  NULL is accepted.  The caller must not free a database while a search that uses it
 * may still run on a stream, nor while a prepared query batch planned against
 * it is still in use.  Errors: none (always SW_OK).
 */
int sw_db_free(sw_db *db);

/*
 * Sizes of a prepared database: sequence count, residue count, device bytes.
 * The device bytes include the row-track lane tables the database keeps for
 * the transposed jobs of small batches (sw_search): each is built on the
 * first search that plans it (one per lane height and 16-bit / int32
 * routing of the sequences, at most 8, each at most 64 MiB; others are built
 * for every search) and freed by sw_db_free.
 */
int sw_db_stats(const sw_db *db, int64_t *n_seqs, int64_t *residues, int64_t *device_bytes);

/* Tuning knobs of a query batch; zero-initialise and set what you need.  Every
 * field left at 0 takes its default.  (The paper's SW# splits database
 * sequences between a short and a long kernel by length, Sec. 3.1.) */
typedef struct sw_options {
  int32_t cutover;         /* database units whose longer sequence has at least this many
                              residues use the intra-task (multi-warp) kernel; 0 = 2048;
                              a value above every length sends everything inter-task */
  int32_t rows_per_lane;   /* query rows per lane of the inter-task kernel: 4, 8, 12, 16 or 24;
                              0 = 24, or 8 for batches too small to fill the GPU */
  int32_t lanes_per_chain; /* lanes per chain of the inter-task kernel, 4..32; 0 = chosen per query */
  int32_t intra_rows;      /* query rows per lane of the intra-task kernel: 8 or 16; 0 = 16 */
  int32_t query_pairs;     /* packed mode, inter-task kernel: 0 = pair queries of similar length
                              into the two 16-bit halves where no lane can overflow (one
                              database sequence per chain), 1 = never pair (two database
                              sequences per chain for every query) */
  int32_t band_stream;     /* batches too small to fill the GPU (0 = auto) run in the band-stream
                              kernel instead of the inter- and intra-task kernels: a query of at
                              least two bands (see band_rows) against every database unit, its
                              rows cut into bands, one warp each, the bands of a query running
                              as a pipeline over a stream of units; every shorter query
                              transposed, the database sequences stacked as rows in bands of
                              256 to 768 rows and the query's residues as the columns; 1 = never;
                              2 = for every batch, however large */
  int32_t band_rows;       /* query rows per lane of the band-stream kernel: 8 or 16 (bands of
                              256 or 512 rows); 0 = 16 */
  int32_t reserved[1];     /* must be 0 */
} sw_options;

/*
 * sw_queries_prepare -- upload a batch of queries and plan the search.
 *
 * Copies the queries and the scoring parameters to the device, chooses the
 * kernel tiling for each query, and allocates all device scratch the search
 * needs, so that sw_search_prepared allocates nothing and can be captured in
 * a CUDA graph.  The query profile (P[c][i] = SM(Q[i], c), the substitution
 * term of Eq. 1 tabulated per residue) is built on the device in every search.
 *
 *   queries, q_offsets, n_queries   host pointers, same layout as the database
 *   submat                          host pointer, 20x20 int8 (see above)
 *   gap_open, gap_extend            see the gap convention above
 *   mode                            SW_MODE_INT32 or SW_MODE_PACKED
 *   opts                            host pointer to tuning knobs, or NULL for defaults
 *   stream                          upload stream; the call returns after it completes
 *   out                             receives the new handle
 *
 * Memory: the batch's device scratch is one block from a stream-ordered
 * memory pool that the library creates for each device on first use (not
 * the device's default pool); blocks freed by sw_queries_free stay reserved
 * in that pool, up to 1 GiB, for later batches.  A batch too small to fill
 * the GPU may also make the database build one of the row-track lane tables
 * it keeps (see sw_db_stats; a cudaMalloc and a synchronisation of `stream`,
 * once per table), so do not prepare batches on a device while another
 * thread captures a CUDA graph in global mode.  The planner keeps its host
 * tables in per-thread buffers between calls.  Calls from several threads
 * are safe.
 *
 * Errors: SW_EINVAL (bad arguments or knobs), SW_ENOMEM, SW_ECUDA.
 */
int sw_queries_prepare(const sw_db *db, const uint8_t *queries, const int64_t *q_offsets,
                       int64_t n_queries, const int8_t *submat, int32_t gap_open,
                       int32_t gap_extend, int32_t mode, const sw_options *opts, void *stream,
                       sw_queries **out);

/* Release a prepared query batch.  NULL is accepted. */
int sw_queries_free(sw_queries *q);

/*
 * sw_search_prepared -- score every prepared query against the database:
 * S(Q, D) = max over all cells of H of Eqs. 1-3 (Sec. 2.2) for every pair,
 * with the batch's scoring (BLOSUM62 and gaps 10/2 in the paper's protein
 * search, Sec. 4.1).  The int32 form runs the cell body of Algorithm 1; the
 * packed form runs the same recurrences in 16-bit halves and recomputes in
 * int32 every pair whose score could have left the 16-bit range (the paper's
 * future work on lower-precision integers, Sec. 6), so both give the exact
 * int32 score.
 *
 * Device-only and asynchronous: enqueues profile construction, the
 * dynamic-programming kernels, (packed mode) overflow detection and the exact
 * int32 rescue, and the scatter to caller order on `stream`, then returns.
 * No allocation and no host synchronisation happen inside.
 *
 *   scores_dev  DEVICE pointer, n_queries * n_db int32, written in caller order
 *
 * Errors: SW_EINVAL (null / mismatched handles, host pointer), SW_ECUDA.
 * A bounded device wait that expires is reported by the next
 * sw_queries_status call as SW_ETIMEOUT.
 */
int sw_search_prepared(const sw_db *db, const sw_queries *q, int32_t *scores_dev, void *stream);

/*
 * sw_search_graph -- the same search as sw_search_prepared, captured once into
 * a CUDA graph and replayed.  The first call on q (and any later call with a
 * different database or scores_dev) captures the whole enqueue sequence of
 * sw_search_prepared on `stream` and instantiates it; every call then launches
 * the graph on `stream`.  `stream` must not be the legacy default stream
 * (NULL): stream capture needs a created stream.  Timing events
 * (sw_queries_set_timing) are not recorded inside the graph.  The graph is
 * released by sw_queries_free.  Errors: as sw_search_prepared, plus SW_EINVAL
 * for a NULL stream.
 */
int sw_search_graph(const sw_db *db, sw_queries *q, int32_t *scores_dev, void *stream);

/*
 * sw_queries_status -- read back the device status of the last search on q.
 * Synchronises `stream`.  *rescued receives the number of (query, sequence)
 * pairs whose packed score saturated and was recomputed in int32 (0 in int32
 * mode).  Returns SW_ETIMEOUT if a bounded device wait expired.
 */
int sw_queries_status(const sw_queries *q, void *stream, int64_t *rescued);

/*
 * sw_queries_set_timing -- when enable != 0, every later sw_search_prepared on
 * q records CUDA events around its main dynamic-programming kernel (off by
 * default, so that a search can be captured in a CUDA graph).
 * sw_queries_kernel_ms -- synchronise `stream` and return in *ms the duration
 * of that kernel in the last timed search.  Errors: SW_EINVAL if timing is off
 * or no timed search ran, SW_ECUDA.
 */
int sw_queries_set_timing(sw_queries *q, int32_t enable);
int sw_queries_kernel_ms(const sw_queries *q, void *stream, float *ms);

/*
 * sw_queries_info -- sizes of a prepared batch: bytes copied host->device by
 * sw_queries_prepare (*h2d_bytes), device bytes it holds (*device_bytes), the
 * number of DP tasks (*n_tasks) and the number of kernels one search launches
 * (*launches).  Any output may be NULL.
 */
int sw_queries_info(const sw_queries *q, int64_t *h2d_bytes, int64_t *device_bytes, int64_t *n_tasks,
                    int64_t *launches);

/*
 * sw_search -- one-call database search: the local alignment score of Eqs.
 * 1-3 (Sec. 2.2) for every (query, database sequence) pair, as the paper's
 * protein database search computes it (Sec. 4.1: BLOSUM62, gaps 10/2, queries
 * against a database of proteins).  Prepares the queries, searches, copies
 * the scores out and releases the batch.
 *
 *   db                              a prepared database
 *   queries, q_offsets, n_queries   host pointers, same layout as the database
 *   submat, gap_open, gap_extend    see the conventions above
 *   mode                            SW_MODE_INT32 or SW_MODE_PACKED (same scores)
 *   scores_out  host or device pointer, n_queries * n_db int32, caller order;
 *               owned by the caller
 *   stream      stream for the work
 *
 * The call allocates and frees its own scratch (the batch's block and, for
 * host scores, a device score buffer, both from the library's stream-ordered
 * memory pool of the current device, which keeps up to 1 GiB of freed blocks
 * for the next call) and returns when the scores are in place.  Errors: as
 * sw_queries_prepare / sw_search_prepared, plus SW_ETIMEOUT.
 */
int sw_search(const sw_db *db, const uint8_t *queries, const int64_t *q_offsets, int64_t n_queries,
              const int8_t *submat, int32_t gap_open, int32_t gap_extend, int32_t mode,
              int32_t *scores_out, void *stream);

/*
 * sw_search_noalloc -- score one query against a prepared database without
 * allocating any memory.  (The paper has no counterpart: this serves callers
 * that cannot allocate device memory while they search -- a service that fixes
 * its memory budget at start-up, a real-time loop in which a cudaMalloc could
 * synchronise the device and stall every stream, a host that runs the library
 * inside an arena it does not control.)
 *
 * Every scratch buffer the search needs (the query profile, the task list,
 * three counters) lives in one 16 MiB static device array that each GPU
 * loading this library holds until the process exits; the call makes no
 * cudaMalloc or cudaFree and calls no allocating library routine.  It
 * computes exact int32 scores with the inter-task kernel, the whole query in
 * one chunk of up to 32 lanes (16 rows per lane for queries of up to 512
 * residues, 24 above), database sequences of every length included, and
 * returns after the scores are in place (it synchronises `stream`).
 *
 *   db          a prepared database on the calling thread's current device
 *   query, m    host pointer to m residue codes 0..19, 0 <= m <= 768
 *   submat      host pointer, 20x20 int8; gap_open, gap_extend as sw_search
 *   scores_dev  DEVICE pointer to n_db int32, written in the caller's order
 *   stream      stream for the work (NULL = legacy default stream)
 *
 * Limits: queries of at most 768 residues, databases of at most 8,000,000
 * sequences, current devices 0..63; anything beyond is rejected with
 * SW_EINVAL and a message.
 * The first call on a device looks up the device address of the scratch
 * array and configures the kernel; make that first call before any CUDA
 * stream capture on that device.  All calls on a device share the array and
 * it keeps the previous call's contents: calls whose GPU work could overlap
 * (from several host threads, or on several streams) race and must be
 * serialised by the caller.
 * Errors: SW_EINVAL, SW_ECUDA, SW_ETIMEOUT.
 */
int sw_search_noalloc(const sw_db *db, const uint8_t *query, int64_t m, const int8_t *submat,
                      int32_t gap_open, int32_t gap_extend, int32_t *scores_dev, void *stream);

/*
 * sw_align_pair -- score-only local alignment of two long sequences (the
 * pairwise alignment of two long DNA sequences, Sec. 2.2 case (a) and Sec. 4.1;
 * Eqs. 1-3 with the gap convention above), on one GPU.
 *
 * The query rows are cut into bands of 32 * rows_per_lane rows, one per warp:
 * a warp is a chain of 32 lanes that sweeps the band across the whole target,
 * and band b starts on a column as soon as band b-1 has finished it, so the
 * bands run as a pipeline over every warp of every SM (a cooperative launch;
 * every wait between warps is bounded).  Cells are int32 (a million-residue
 * identity scores 10^6 with +1 matches); the bottom rows passed between bands
 * keep H and F + Go in 31 bits, so the call requires
 * max(SM) * min(m, n) + gap_open + gap_extend < 2^31.
 *
 *   query, m     host pointer to m residue codes 0..19 (DNA: any 4 or 5 of
 *                them, e.g. A C G T N = 0 1 2 3 4), m < 2^31
 *   target, n    host pointer to n codes, n < 2^31 - 32
 *   submat       host pointer, 20x20 int8 (row = query code, column = target
 *                code), entries in [-64, 63]; DNA +1/-3: +1 on the diagonal of
 *                the codes used, -3 elsewhere
 *   gap_open, gap_extend   a gap of length k costs gap_open + k * gap_extend
 *   opts         host pointer or NULL (defaults)
 *   score        host pointer, receives S = max(0, max H)
 *   kernel_ms    host pointer or NULL: duration of the band kernel
 *   stream       stream for the work (NULL = legacy default); the call
 *                allocates its device scratch (a ring of boundary rows per
 *                band in flight, 8 bytes per column, 32,768 columns by
 *                default; the query profile; the target), returns when the
 *                score is in *score and frees the scratch
 *
 * Errors: SW_EINVAL, SW_ENOMEM, SW_ECUDA, SW_ETIMEOUT.
 */
typedef struct sw_pair_options {
  int32_t band_warps;     /* at most this many warps (bands in flight) per CTA, 1..16; 0 = enough
                             to give every SM bands, at most 16 */
  int32_t rows_per_lane;  /* 4, 8, 16 or 24 (a band is 32 x rows_per_lane query rows); 0 = 16, or 8
                             when 512-row bands would give fewer than 3 per SM */
  int32_t max_ctas;       /* at most this many CTAs; 0 = all that fit */
  int32_t ring_columns;   /* columns each band's boundary ring holds, a multiple of 16 >= 256 (a band
                             runs at most that far ahead of the band below); 0 = automatic */
  int32_t reserved[4];    /* must be 0 */
} sw_pair_options;

int sw_align_pair(const uint8_t *query, int64_t m, const uint8_t *target, int64_t n, const int8_t *submat,
                  int32_t gap_open, int32_t gap_extend, const sw_pair_options *opts, int32_t *score,
                  float *kernel_ms, void *stream);

/*
 * sw_traceback -- one optimal local alignment for each of a list of hits
 * (query, database sequence) of a search, the alignment behind a score
 * (Sec. 2.2: H[i][j] is the best score of an alignment ending at cell (i, j);
 * the path that produced it is the alignment).  The paper's search reports
 * scores only; this recovers the alignments of the hits a caller keeps.
 *
 * One CTA per hit recomputes the pair's matrix in int32, its warps taking
 * the query's 512-row chunks as a pipeline, and records 4 bits per cell (where
 * H came from; whether E and F extend a gap); one thread per hit walks them
 * back from the first cell, in row-major order, that holds the score.  Device
 * memory: about m * n / 2 bytes per hit (held during the call).
 *
 *   db                    a prepared database
 *   queries, q_offsets, n_queries   host pointers, as sw_queries_prepare
 *   hits, n_hits          host array of (query index, database sequence index
 *                         in the caller's order)
 *   submat, gap_open, gap_extend    as sw_search
 *   out                   host array of n_hits sw_alignment
 *   ops, ops_capacity     host buffer for the operations of all hits: hit h
 *                         gets m + n bytes at out[h].ops_offset (m, n its
 *                         lengths); ops_capacity must be at least their sum
 *   stream                stream for the work; the call returns when done
 *
 * Operations, first to last: 'M' aligns query[i] with target[j], 'I' a query
 * residue with a gap, 'D' a target residue with a gap.  An alignment scores
 * the substitution scores of its 'M' pairs minus gap_open + k * gap_extend per
 * maximal run of k 'I' or k 'D'; that is out[h].score.  A score of 0 gives an
 * empty alignment.
 * Errors: SW_EINVAL (bad indices, small ops buffer), SW_ENOMEM, SW_ECUDA,
 * SW_ETIMEOUT (a bounded wait between the warps of a hit expired).
 */
typedef struct sw_hit {
  int32_t query;   /* index into the query batch */
  int32_t target;  /* database sequence, caller order */
} sw_hit;

typedef struct sw_alignment {
  int32_t score;
  int32_t q_begin, q_end;  /* the alignment covers query[q_begin, q_end) (0-based) */
  int32_t t_begin, t_end;  /* and target[t_begin, t_end) */
  int32_t n_ops;           /* operations at ops[ops_offset, ops_offset + n_ops) */
  int64_t ops_offset;
} sw_alignment;

int sw_traceback(const sw_db *db, const uint8_t *queries, const int64_t *q_offsets, int64_t n_queries,
                 const sw_hit *hits, int64_t n_hits, const int8_t *submat, int32_t gap_open, int32_t gap_extend,
                 sw_alignment *out, uint8_t *ops, int64_t ops_capacity, void *stream);

/*
 * sw_selftest_wait -- check that the library's bounded device waits give up.
 * Every wait between warps or CTAs in the kernels (for a counter another warp
 * raises, or an mbarrier phase a bulk copy completes) stops after a clock
 * budget and reports SW_ETIMEOUT instead of hanging.  This runs one such wait
 * against a condition nothing fulfils, on one GPU thread:
 *
 *   which          0: a progress counter that stays 0 (the pair-band
 *                  kernel's waits for room), given budget_cycles cycles;
 *                  1: an mbarrier phase that never completes (the profile
 *                  waits), with the kernels' own budget of about one second
 *   budget_cycles  clock cycles for which == 0, in (0, 2^32]; ignored for 1
 *   status_out     host pointer: SW_ETIMEOUT when the wait gave up (the
 *                  expected outcome), SW_OK if it was fulfilled
 *   stream         stream for the work; the call returns when done
 *
 * No fault and no hang: the kernel returns after the budget and the context
 * stays usable.  Errors: SW_EINVAL, SW_ENOMEM, SW_ECUDA.
 */
int sw_selftest_wait(int32_t which, int64_t budget_cycles, int32_t *status_out, void *stream);

/*
 * sw_last_error -- the message of the last failed call on this thread, or ""
 * if it succeeded.  The paper has no error interface; the message names the
 * argument or CUDA call that failed (the status code of every entry point
 * carries the class: SW_EINVAL, SW_ENOMEM, SW_ECUDA, SW_ETIMEOUT).  The
 * string is owned by the library and stays valid until the next call of
 * this library on the same thread.
 */
const char *sw_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SWGB_H */
