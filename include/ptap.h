/*
 * ptap.h -- C ABI of the GB300 all-at-once sparse triple product C = P^T A P.
 *
 * The operation (Kong, "Parallel memory-efficient all-at-once algorithms for
 * the sparse matrix triple products in multigrid methods"):
 *
 *   A is n x n, P is n x m (Section 2), C = P^T A P is m x m (Section 3,
 *   Eq. 4).  C is formed all at once as a sum of outer products of the rows of
 *   P and the rows of A P (Eq. 9), so neither A P nor P^T is ever stored.  The
 *   work splits into a symbolic phase that preallocates C without any
 *   floating point (Section 2, Alg. 1-2; Section 3, Alg. 7) and a numeric
 *   phase that fills the preallocated values (Alg. 8) and may be repeated
 *   whenever the values of A or P change (Section 4.1: one symbolic and
 *   eleven numeric products; Section 4.2, Table 8: caching symbolic data).
 *
 * Conventions for every entry point:
 *  - Matrices are CSR with int32 row pointers and column indices.  Columns
 *    must be sorted ascending and unique within each row; duplicates are
 *    rejected, not summed.  Explicitly stored zeros are structural entries.
 *  - Values are float64 (PTAP_F64) or float32 (PTAP_F32); A, P and C of one
 *    plan share one dtype.  float32 plans accumulate in float32.
 *  - Every pointer in a ptap_csr and every value buffer is a DEVICE pointer
 *    owned by the caller, unless stated otherwise.  The library never frees
 *    caller memory.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Calls are asynchronous on it, except where a call says it
 *    synchronises.
 *  - Every call returns PTAP_OK (0) or one of the PTAP_ERR_* codes below; no
 *    C++ exception crosses this boundary.  A failed call leaves its outputs
 *    unspecified and allocates nothing that outlives it.
 *  - C's pattern is structural: an entry reached through the patterns of P,
 *    A and P is kept even where its value cancels to zero.  Column indices of
 *    C are sorted ascending per row; rows may be empty.
 */
#ifndef PTAP_H
#define PTAP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes ------------------------------------------------------ */
#define PTAP_OK 0
#define PTAP_ERR_INVALID 1     /* null pointer, shape or dtype mismatch, bad CSR */
#define PTAP_ERR_PATTERN 2     /* inputs do not match the pattern the plan was built for */
#define PTAP_ERR_OVERFLOW 3    /* nnz(C) or an intermediate count >= 2^31 */
#define PTAP_ERR_OOM 4         /* an allocation failed */
#define PTAP_ERR_SPILL 5       /* a device hash table ran out of space (status word) */
#define PTAP_ERR_TIMEOUT 6     /* a bounded device wait gave up */
#define PTAP_ERR_CUDA 7        /* any other CUDA failure */
#define PTAP_ERR_UNSUPPORTED 8 /* a valid request this build does not implement */

/* ---- types ------------------------------------------------------------ */
typedef enum { PTAP_F64 = 0, PTAP_F32 = 1 } ptap_dtype;

/* A CSR matrix on the device.  row_ptr has nrows+1 entries, col_idx and val
 * nnz entries; nnz must equal row_ptr[nrows].  val may be NULL for calls that
 * only need the pattern.  All pointers are caller-owned device memory. */
typedef struct {
  int32_t nrows;
  int32_t ncols;
  int64_t nnz;
  const int32_t* row_ptr;
  const int32_t* col_idx;
  const void* val;
  int32_t dtype; /* ptap_dtype */
} ptap_csr;

/* Optional device allocator.  alloc returns device memory of `bytes` bytes
 * usable on `stream` (NULL on failure); free releases it.  When a NULL
 * allocator is passed the library uses cudaMallocAsync/cudaFreeAsync on the
 * call's stream. */
typedef struct {
  void* (*alloc)(size_t bytes, void* stream, void* ctx);
  void (*free)(void* ptr, size_t bytes, void* stream, void* ctx);
  void* ctx;
} ptap_allocator;

/* Numeric scheme. */
#define PTAP_MODE_AUTO 0
#define PTAP_MODE_OWNER 1  /* coarse-row chunks accumulated on chip, written once */
#define PTAP_MODE_ATOMIC 2 /* Alg. 8 literally: per fine row, atomic scatter into C */

/* Tuning knobs; zero selects the built-in default for a field. */
typedef struct {
  int32_t mode;           /* PTAP_MODE_* */
  int32_t chunk_entries;  /* C entries accumulated per CTA in owner mode: 64..65536 (class-program
                             kernels; clamped so the accumulator fits shared memory: 49152 for
                             FP32 and 24576 for FP64 with 227 KB per CTA) or 64..16384
                             (general kernels); 0 = default */
  int32_t block_threads;  /* threads per CTA of the numeric kernels: 64, 128, 256, or 512/1024
                             for the class-program kernels (the general and batch kernels use
                             at most 256); 0 = default 256 */
  int32_t group_lanes;    /* lanes that cooperate on one fine row: 4, 8, 16 or 32 */
  int32_t ap_slots;       /* hash slots per group for one row of A P */
  int32_t debug_checks;   /* nonzero: validate CSR inputs on the device */
  int32_t force_spill;    /* nonzero: shrink on-chip tables to exercise spill paths */
  int32_t class_programs; /* 0: run fine rows of one structure class in lockstep from a
                             per-class program where the patterns allow (owner mode);
                             -1: always use the general kernel */
  int32_t visit_block_log2; /* class-program visit order: runs of one class inside blocks
                               of 2^b consecutive fine rows (0: one block per chunk) */
  int32_t specialize;     /* k > 0: compile straight-line code (NVRTC, at symbolic time) for
                             at most k classes covering most fine rows; 0 or -1: class
                             programs are interpreted */
  int32_t cache_indices;  /* cached intermediates of the class-program kernels in the sense
                             of Section 4.2 (memory traded for time):
                             1: the plan stores, for every entry of A, the first position of
                             P's row for its column (nnz(A) int32), so the kernels skip one
                             dependent lookup per entry;
                             2: the plan stores per visit of a fine row to a chunk, in
                             warp-sized lane-major records, those positions for the row's
                             entries of A and the accumulator offsets of its P(I,:) rows
                             (int32 and uint16 per lane), so the kernels read them with
                             coalesced loads and skip P(I,:)'s column lookups; plans with
                             compact chunks, or records past 32 GB, fall back to 1;
                             0: off */
  int32_t general_kernel; /* general owner-mode kernel (rows outside the class programs):
                             0 = sort-based, one warp per fine row (default);
                             1 = hash tables per group of group_lanes lanes */
  int32_t compact_chunks; /* L > 0: owner-mode chunks are grown breadth-first over the graph
                             of C's pattern, by runs of L consecutive coarse rows (L <= 4096),
                             into compact regions instead of being cut as ranges of
                             consecutive rows, so fewer fine rows reach two chunks.  Used by
                             the class-program kernels only: a plan that ends on the general
                             kernel, has a run of rows longer than a chunk or more chunks
                             than the packed row locations can name keeps ranges
                             (ptap_stats.compact_chunks says which).  Plans with
                             compact chunks are refused (PTAP_ERR_UNSUPPORTED) by
                             ptap_batch_numeric_noalloc; 0: ranges */
  int32_t specialize_scope; /* with specialize = k > 0: 0 = the plan compiles its own kernel
                               at symbolic time (default); 1 = the plan compiles nothing, and a
                               batch that includes it (ptap_batch_create) compiles one kernel for
                               the most visited classes over all its plans */
  int32_t specialize_async; /* with specialize = k > 0 and scope 0: nonzero compiles the plan's
                               code in a background thread, so ptap_symbolic returns without
                               waiting for NVRTC; numeric calls run the interpreter until the
                               compiled kernel is loaded, then switch to it (ptap_stats'
                               n_specialized stays 0 until then).  0: compile at symbolic time */
  int32_t reserved[1];
} ptap_config;

/* Statistics of a plan (host struct filled by ptap_plan_stats).  The byte
 * counts are the quantity the paper compares between algorithms: memory that
 * includes the storage of C (Section 4.1, the "Mem" columns of Tables 1, 3
 * and 7). */
typedef struct {
  int32_t n, m;
  int64_t nnz_a, nnz_p, nnz_c;
  int64_t plan_bytes;        /* device bytes the plan holds between calls */
  int64_t peak_bytes;        /* high-water mark of library-held device bytes */
  int64_t symbolic_peak_bytes;
  int32_t n_chunks;          /* owner-mode chunks */
  int32_t n_heavy_chunks;    /* chunks whose C rows exceed on-chip capacity */
  int64_t chunk_fine_rows;   /* sum over chunks of the fine rows each visits */
  int32_t n_spill_rows_symbolic; /* coarse rows whose pattern needed the global table */
  int32_t mode;              /* numeric scheme the plan uses */
  int32_t chunk_entries, block_threads, group_lanes, ap_slots;
  int32_t kind;              /* 0 all-at-once plan, 1 two-step plan */
  int32_t fast_path;         /* 1 if the numeric phase runs per-class programs */
  int32_t n_classes;         /* distinct fine-row structure classes */
  int32_t n_segments;        /* same-class runs over all chunks */
  int32_t n_pieces;          /* warp-sized pieces of those runs */
  int32_t n_specialized;     /* classes running as compiled straight-line code */
  int32_t specialized_permille; /* share of fine-row visits they cover, in 1/1000 */
  int32_t specialize_us;     /* time spent generating and compiling that code */
  int32_t compact_chunks;    /* 1 if the chunks are grown regions of C's graph */
  int32_t cache_indices;     /* cached indices the plan holds: 0 none, 1 per entry of A,
                                2 per visit (piece records) */
  int64_t cached_index_bytes; /* device bytes of those cached indices (in plan_bytes) */
} ptap_stats;

typedef struct ptap_plan ptap_plan;
typedef struct ptap_batch ptap_batch;

/* ---- entry points ----------------------------------------------------- */

/* Symbolic all-at-once product (Section 3, Alg. 7; Alg. 1 for one row of
 * A P).  Validates A (n x n) and P (n x m), computes the structural pattern
 * of C = P^T A P and the numeric schedule, and returns a library-owned plan
 * in *out.  Values of A and P are not read.  `cfg` and `alloc` may be NULL.
 * Synchronises `stream` (once, to size C).  Errors: PTAP_ERR_INVALID,
 * PTAP_ERR_OVERFLOW (nnz(C) >= 2^31), PTAP_ERR_OOM, PTAP_ERR_SPILL,
 * PTAP_ERR_CUDA. */
int ptap_symbolic(const ptap_csr* A, const ptap_csr* P, const ptap_config* cfg,
                  const ptap_allocator* alloc, void* stream, ptap_plan** out);

/* Pattern of C held by the plan: the preallocated structure of C that the
 * symbolic phase determines without floating point (Section 2, after Alg. 2;
 * Section 3, Alg. 7, where the counts preallocate C).  *m rows, *nnz entries,
 * device pointers to row_ptr (m+1) and col_idx (nnz, ascending per row),
 * owned by the plan and valid until ptap_plan_destroy.  Any output pointer
 * may be NULL.  Errors: PTAP_ERR_INVALID for a NULL plan. */
int ptap_plan_pattern(const ptap_plan* plan, int32_t* m, int64_t* nnz,
                      const int32_t** row_ptr, const int32_t** col_idx);

/* Numeric all-at-once product (Section 3, Eq. 9, Alg. 8): writes the nnz(C)
 * values of C = P^T A P into C_val (caller-owned device buffer, dtype of the
 * plan), in the order of the plan's pattern.  A and P must have the patterns
 * the plan was built from (checked by shape and nnz: PTAP_ERR_PATTERN).  No
 * auxiliary A P or P^T is formed.  Asynchronous; allocates nothing. */
int ptap_numeric(ptap_plan* plan, const ptap_csr* A, const ptap_csr* P, void* C_val,
                 void* stream);

/* Numeric product from host-resident values (the paper's numeric phase,
 * Section 3, Eq. 9, repeated as values change, Section 4.1).  A and P give the
 * device patterns exactly as for ptap_numeric (their `val` fields are
 * ignored); A_val_host (nnz(A) values), P_val_host (nnz(P) values) and
 * C_val_host (nnz(C) values, written) are host arrays of the plan's dtype.
 * The values are staged through two plan-owned sets of device buffers
 * (allocated on the first call with the plan's allocator; 2 * (nnz(A) +
 * nnz(P) + nnz(C)) values) on two internal streams: the next call's upload
 * overlaps this call's product and download.  When `stream` has completed,
 * C_val_host holds the result.  Page-locked host arrays give asynchronous
 * copies; pageable ones still work, with copies that block the host.  Calls
 * on one plan must come from one host thread; the host arrays of a call must
 * stay valid (inputs unmodified) until `stream` has completed that call.
 * Errors as ptap_numeric, plus PTAP_ERR_OOM for the staging buffers. */
int ptap_numeric_host(ptap_plan* plan, const ptap_csr* A, const ptap_csr* P, const void* A_val_host,
                      const void* P_val_host, void* C_val_host, void* stream);

/* Backward of C = P^T A P (not in the paper).  Given G = dL/dC as nnz(C)
 * values on the plan's pattern, writes dL/dA = (P G P^T) restricted to the
 * pattern of A into dA (nnz(A) values) and dL/dP = (A P G^T + A^T P G)
 * restricted to the pattern of P into dP (nnz(P) values).  Either output may
 * be NULL to skip it.  Row by row, all at once: no product matrix is stored.
 * Asynchronous; allocates nothing. */
int ptap_backward(ptap_plan* plan, const ptap_csr* A, const ptap_csr* P, const void* G,
                  void* dA, void* dP, void* stream);

/* Two-step comparator (Section 3, Eq. 6, Alg. 5-6): builds C~ = A P and P^T
 * explicitly, then C = P^T C~.  The symbolic call returns a plan of kind 1
 * that holds those auxiliary matrices; ptap_numeric on that plan runs the
 * two-step numeric phase.  Same conventions as ptap_symbolic. */
int ptap_two_step_symbolic(const ptap_csr* A, const ptap_csr* P, const ptap_config* cfg,
                           const ptap_allocator* alloc, void* stream, ptap_plan** out);

/* Batched numeric products of uneven sizes: the repeated numeric phase
 * (Section 4.1, one symbolic and many numeric products) of many plans at
 * once, each plan holding its cached symbolic data (Section 4.2).  `plans`,
 * `A` and `P` (host arrays of `count` elements) and `C_vals` (host array of
 * device pointers) fix the problems once; the batch copies their descriptors
 * and a queue of their chunks, longest first, to the device.  All plans must
 * be all-at-once plans of one dtype.  Plans that run class programs share one
 * persistent launch; when any of them was built with specialize = k > 0 the
 * batch compiles (NVRTC, at creation) one kernel for the k most visited
 * class programs over all of them, pooled by their bytes.  The other plans
 * share a second launch of the general kernel; they must agree on
 * group_lanes, ap_slots and force_spill (PTAP_ERR_INVALID otherwise) and
 * must not use compact chunks (PTAP_ERR_UNSUPPORTED).  Synchronises `stream`.
 * Errors: as ptap_numeric for each problem, PTAP_ERR_OOM. */
int ptap_batch_create(ptap_plan* const* plans, const ptap_csr* A, const ptap_csr* P,
                      void* const* C_vals, int32_t count, const ptap_allocator* alloc,
                      void* stream, ptap_batch** out);

/* Runs every product of the batch: a counter reset and at most two
 * persistent launches (class-program problems, general problems) over the
 * work queues.  Reads the current values behind the pointers given at
 * creation, so it can be captured once in a CUDA graph and replayed after the
 * values change (Section 4.1's repeated numeric products).  Asynchronous;
 * allocates nothing. */
int ptap_batch_numeric(ptap_batch* batch, void* stream);

/* Frees the batch's descriptors and queues (not the plans, which the caller
 * still owns and must outlive the batch).  NULL is a no-op. */
void ptap_batch_destroy(ptap_batch* batch);

/* Statistics of a plan (Section 4.1, "Mem"; see ptap_stats), written into
 * the caller's host struct.  Errors: PTAP_ERR_INVALID for NULL arguments. */
int ptap_plan_stats(const ptap_plan* plan, ptap_stats* out);

/* Reads and clears the plan's device status word (synchronises `stream`):
 * PTAP_OK, or the PTAP_ERR_* code a kernel of this plan recorded (a device
 * table that ran out of space, an input that did not match the pattern).
 * The paper has no counterpart: its hash tables grow on the host. */
int ptap_plan_check(ptap_plan* plan, void* stream);

/* Frees everything the plan holds: C's pattern, the schedule and the cached
 * symbolic data of Section 4.2 (stream-ordered on the plan's stream).  NULL is
 * a no-op. */
void ptap_plan_destroy(ptap_plan* plan);

/* Static description of an error code. */
const char* ptap_error_string(int code);

/* Version of this library as major*10000 + minor*100 + patch. */
int ptap_version(void);

/* ---- value movement of the row-partitioned product ----------------------
 * With A's and P's fine rows split into blocks over processes (Section 2,
 * Eq. 1-3), a process gathers the rows of P that its block of A references
 * but others own (P~_r, one sparse exchange per phase, Section 2, Alg. 2 and
 * 4) and sends the outer-product contributions it made to coarse rows that
 * others own (C_s, Section 3, Alg. 7-8) to their owners, who add them.  The
 * index lists are fixed by the symbolic phase; these calls move the values
 * of each numeric phase.  All pointers are device pointers; values have the
 * given dtype.  Asynchronous on `stream`; allocate nothing.
 *
 * ptap_gather: out[e] = src[src_idx[e]] for e < n (packing a send buffer).
 * ptap_scatter_add: dst[dst_idx[e]] += src[src_idx[e]] (src_idx NULL: src[e])
 * for e < n; the positions dst_idx[0..n) must be distinct within one call
 * (the entries are added without atomics).
 * Errors: PTAP_ERR_INVALID for a negative n, a bad dtype or a NULL pointer
 * with n > 0; PTAP_ERR_CUDA for a launch failure. */
int ptap_gather(const void* src, const int32_t* src_idx, int64_t n, int32_t dtype, void* out,
                void* stream);
int ptap_scatter_add(const void* src, const int32_t* src_idx, const int32_t* dst_idx, int64_t n,
                     int32_t dtype, void* dst, void* stream);

/* ---- levels of an algebraic multigrid hierarchy ---------------------------
 * The paper's application forms a twelve-level hierarchy with eleven triple
 * products (Section 4.2.2, Tables 5-6), taking its coarsening from a cited
 * work.  These calls build one reading of it on the device -- smoothed
 * aggregation -- so that C = P^T A P of every level runs through this
 * library: aggregate the fine rows, form P = (I - omega D^-1 A) T from the
 * tentative prolongator T(i, agg(i)) = 1, then ptap_symbolic / ptap_numeric.
 * A must be square, hold its diagonal and be symmetric in magnitude (the
 * strength of an edge is |A(i,j)| read from row i).
 *
 * ptap_aggregate: repeated pairwise matching.  A round: every unmatched node
 * picks the unmatched neighbour node with the largest key (strength, hash of
 * the node pair), where the strength between two nodes is the largest
 * |A(i,j)| over their members; mutual picks are matched.  Rounds repeat until
 * none matches or `rounds` is reached; then up to `rounds` more rounds key
 * the edges by the hash alone (random priorities, which converge fast where
 * long chains of decreasing strength slow the first phase).  A node still
 * unmatched joins the pair with which it has the strongest edge, and stays
 * alone only without a paired neighbour.  Each of `passes` (0..8) passes
 * matches the previous pass's nodes.  Writes agg[i] (device, A.nrows
 * entries, caller-owned) in 0..*n_agg-1 and *n_agg (host).  Deterministic.
 * Synchronises `stream`; scratch comes from `alloc` (NULL: cudaMallocAsync)
 * and is freed before return.  Errors: PTAP_ERR_INVALID, PTAP_ERR_OOM,
 * PTAP_ERR_CUDA. */
int ptap_aggregate(const ptap_csr* A, int32_t passes, int32_t rounds, int32_t* agg, int32_t* n_agg,
                   const ptap_allocator* alloc, void* stream);

/* The smoothed prolongator of an aggregation: an opaque, library-owned
 * object holding the pattern of P = (I - omega D^-1 A_F) T, n x n_agg, with
 * sorted columns.  A_F is A filtered by strength: it keeps the diagonal and
 * the off-diagonal entries with |A(i,j)| >= theta * max_{k != i} |A(i,k)|
 * (0 <= theta <= 1; theta = 0 keeps every entry); D = diag(A).
 * ptap_prolongator_symbolic reads A (values too: the strong entries are
 * settled here and kept, so the pattern does not move with later values)
 * and agg (copied); synchronises `stream`.  ptap_prolongator_pattern returns
 * its sizes and device pointers (valid until destroy).
 * ptap_prolongator_numeric writes the nnz(P) values P(i,a) = [agg(i) = a] -
 * omega / A(i,i) * sum_{j in A_F(i,:), agg(j) = a} A(i,j) into P_val
 * (caller-owned device buffer of A's dtype); A must have the pattern given
 * at symbolic time (PTAP_ERR_PATTERN); asynchronous, allocates nothing, and
 * may be repeated whenever A's values change.
 * ptap_prolongator_check reads and clears its device status word
 * (PTAP_ERR_INVALID for a row without a diagonal entry).  Destroy frees it
 * (NULL is a no-op). */
typedef struct ptap_prolongator ptap_prolongator;
int ptap_prolongator_symbolic(const ptap_csr* A, const int32_t* agg, int32_t n_agg, double theta,
                              const ptap_allocator* alloc, void* stream, ptap_prolongator** out);
int ptap_prolongator_pattern(const ptap_prolongator* P, int32_t* nrows, int32_t* ncols, int64_t* nnz,
                             const int32_t** row_ptr, const int32_t** col_idx);
int ptap_prolongator_numeric(ptap_prolongator* P, const ptap_csr* A, double omega, void* P_val,
                             void* stream);
int ptap_prolongator_check(ptap_prolongator* P, void* stream);
void ptap_prolongator_destroy(ptap_prolongator* P);

/* ---- batched numeric products that allocate nothing ---------------------
 * The paper has no counterpart to this entry point.  It serves callers that
 * cannot allocate device memory when the products run: solvers that reserve
 * their whole device footprint in their own pool up front and forbid any
 * later cudaMalloc, and latency-critical code that cannot afford the implicit
 * device synchronisation of a cudaMalloc/cudaFree.  Their plans are built
 * beforehand (ptap_symbolic, which does allocate); this call then runs the
 * numeric products of `count` plans in one persistent launch, like
 * ptap_batch_numeric, without creating a batch object.
 *
 * Arguments are as for ptap_batch_create: host arrays of `count` plans
 * (all-at-once plans of one dtype and one configuration), of A and P
 * descriptors matching each plan, and of caller-owned device buffers for the
 * values of each C.  The work counter, the problem descriptors and the work
 * queue live in one file-scope device array of PTAP_NOALLOC_SCRATCH_BYTES
 * (8 MiB) that every GPU that loads this library holds until the process
 * exits; the call calls no cudaMalloc, cudaFree or other allocating routine.
 * The first call on a device looks up that array's device address (once per
 * device, with the device current); make that first call before any stream
 * capture.  Every call shares the array and it keeps the last call's
 * contents: each call clears the work counter itself, and calls whose work
 * overlaps on the GPU race on the array, so callers must serialise them.
 * The products run on the general owner-mode kernel.  Its on-chip
 * accumulator also holds column indices, so for plans built with large
 * chunks (the class-program kernels take up to 49152 entries) it is lowered
 * to what a CTA's shared memory holds; chunks above that accumulate in C
 * with atomics instead (same result, slower).
 * The descriptors and the queue are staged from a process-wide host buffer
 * that the next call reuses, so while `stream` is capturing the call
 * launches nothing and returns PTAP_ERR_UNSUPPORTED.
 * Errors: PTAP_ERR_OVERFLOW when count > PTAP_NOALLOC_MAX_PROBLEMS or the
 * plans hold more than PTAP_NOALLOC_MAX_ITEMS owner-mode chunks in total;
 * PTAP_ERR_INVALID when the plans differ in dtype or configuration;
 * PTAP_ERR_UNSUPPORTED for plans with compact chunks, during stream capture,
 * or when even a 64-entry accumulator does not fit shared memory; otherwise
 * as ptap_batch_create.  Asynchronous on `stream`. */
#define PTAP_NOALLOC_SCRATCH_BYTES (8u << 20)
#define PTAP_NOALLOC_MAX_PROBLEMS 1024
#define PTAP_NOALLOC_MAX_ITEMS 1000000
int ptap_batch_numeric_noalloc(ptap_plan* const* plans, const ptap_csr* A, const ptap_csr* P,
                               void* const* C_vals, int32_t count, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* PTAP_H */
