/*
 * hss.h -- C ABI of the GB300 randomized HSS compression library.
 *
 * The method is randomized Hierarchically Semi-Separable (HSS) compression of
 * a dense n x n matrix (Rouet, Li, Ghysels, Napov, arXiv:1503.05464):
 *   - HSS representation and cluster tree ............ Section 2.1, Fig. 1
 *   - randomized compression ......................... Section 2.2, Algorithm 1
 *   - interpolative decomposition (truncated CPQR) ... Section 2.2, Section 3.1
 *   - adaptive sampling (late notification) .......... Section 3.2, Algorithm 5
 *   - HSS matrix-vector product ...................... Section 2.3, Algorithm 2
 *   - ULV-like factorization ......................... Section 2.4, Algorithm 3
 *   - solution with the ULV factors .................. Section 2.5, Algorithm 4
 *
 * Conventions for every entry point:
 *   - Matrix and vector pointers are DEVICE pointers owned by the caller,
 *     unless a parameter says "host".  Dense matrices are row-major with a
 *     leading dimension (elements between consecutive rows) >= the row length.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Work is stream-ordered; entry points that must read results
 *     back (hss_compress reads ranks to size its storage) synchronize `stream`.
 *   - Errors are returned as hss_status codes; no exception or abort crosses
 *     the ABI.  A handle keeps a message for its last error
 *     (hss_last_error); calls without a handle keep a thread-local message
 *     readable with hss_last_error(NULL).
 *   - Device memory that a handle needs is allocated by the library with
 *     stream-ordered cudaMallocAsync and released by hss_destroy.
 */
#ifndef HSS_H
#define HSS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hss_s* hss_t;

typedef enum {
  HSS_OK = 0,
  HSS_ERR_INVALID = 1,   /* bad argument (size, pointer, leading dimension, option) */
  HSS_ERR_OOM = 2,       /* device allocation failed */
  HSS_ERR_CUDA = 3,      /* a CUDA call or kernel launch failed */
  HSS_ERR_RANK_CAP = 4,  /* adaptive sampling reached d_max before every node compressed */
  HSS_ERR_SINGULAR = 5,  /* zero pivot in the root LU of the ULV factorization */
  HSS_ERR_TIMEOUT = 6,   /* a device-side wait gave up after its iteration limit */
  HSS_ERR_STATE = 7      /* call out of order (e.g. hss_solve before hss_factor) */
} hss_status;

typedef enum { HSS_F32 = 0, HSS_F64 = 1 } hss_dtype;

/* Arithmetic of the sampling products S^r = A R and S^c = A^T R (step 2 of
 * the compression algorithm, Section 2.2).  R is bfloat16-exact, so the
 * split modes only split A.  For HSS_F64 inputs only NATIVE is accepted. */
typedef enum {
  HSS_SAMPLE_NATIVE = 0, /* FP32 (or FP64) fused multiply-add, no tensor cores  */
  HSS_SAMPLE_TF32 = 1,   /* A rounded to TF32 (nearest), tensor cores, FP32 acc. */
  HSS_SAMPLE_BF16X2 = 2, /* A = hi + lo (two bfloat16 terms), FP32 accumulation */
  HSS_SAMPLE_BF16X3 = 3  /* A = hi + mid + lo (three bfloat16 terms)            */
} hss_sample_mode;

/* Compression options (Section 2.2, Section 3.2). */
typedef struct {
  int32_t leaf_size;     /* cluster tree: bisect [lo,hi) while hi-lo > leaf_size  */
  double rtol;           /* ID stops at the first |R_ii| <= max(rtol |R_11|, atol) */
  double atol;           /* absolute floor of that test (0 = relative only)      */
  int32_t d0;            /* initial number of random sample columns              */
  int32_t d_step;        /* columns added when a node's rank is too large         */
  int32_t d_max;         /* cap on the sample count (0 = n)                      */
  int32_t oversample_p;  /* a node fails iff d < m and rank > d - oversample_p    */
  int32_t sample_mode;   /* hss_sample_mode                                      */
  uint64_t seed;         /* seed of the counter-based Gaussian generator of R    */
  /* Cluster tree (Section 2.1; Section 4 compares balanced binary trees with
   * unbalanced "comb" trees).  NULL = bisection by leaf_size.  Otherwise a
   * host array of tree_nodes split points, one per node in breadth-first
   * order (root first; the two children of a node are consecutive, left
   * first, and come after every node of the parent's depth that precedes
   * it): tree[q] = -1 makes node q a leaf, any lo < tree[q] < hi splits
   * node q = [lo, hi) into [lo, tree[q]) and [tree[q], hi).  The root is
   * [0, n).  Read during hss_compress / hss_batch_submit only (copied).
   * INVALID if a split is out of range or the count does not match. */
  const int64_t* tree;
  int32_t tree_nodes;
  /* 1: the caller guarantees A = A^T (not checked).  One R serves both
   * samples (Section 2.2), so S^c = A^T R = S^r: the column side of every
   * node repeats its row side -- one ID per node instead of two, V = U,
   * I^c = I^r; B12 and B21 are still read from A.  0: general A. */
  int32_t symmetric;
} hss_opts;

/* Statistics of a handle (Table 3's columns: max rank, factor sizes, time). */
typedef struct {
  int64_t n;
  int32_t nodes, leaves, levels;
  int32_t max_rank_r, max_rank_c;   /* largest U / V generator rank            */
  int32_t d_final;                  /* sample count at the end of compression  */
  int32_t passes;                   /* adaptive passes (1 = no restart)        */
  int64_t bytes_hss;                /* device bytes of D, B, E, permutations   */
  int64_t bytes_ulv;                /* device bytes of the ULV factors         */
  double ms_compress;               /* wall time of hss_compress              */
  double ms_sample;                 /* device time in the fused sampling kernel */
  double ms_id;                     /* device time in the batched ID kernel    */
  double ms_levels;                 /* host wall time of the level loop        */
  double flops_sample;              /* 4 n^2 d summed over passes              */
  double flops_id;                  /* FP64 flops of the IDs: sum over node sides
                                       of sum_{i<k} 4 (d - i)(m - i) (the CPQR),
                                       plus (m - k) k^2 (T = R1^{-1} R2) where
                                       the side passes the adaptive test      */
  int32_t factored;                 /* 1 after hss_factor                      */
  int64_t launches;                 /* kernels launched by hss_compress        */
  int64_t bytes_d2h;                /* bytes read back to the host (ranks)     */
  double ms_host_id_launch;         /* host time preparing and launching IDs   */
  double ms_host_wait;              /* host time blocked on the rank readback  */
  double ms_host_sample;            /* host wall time of the sampling passes   */
  int64_t id_launches;              /* ID kernel launches of hss_compress      */
  double flops_id_solve;            /* the T = R1^{-1} R2 part of flops_id     */
} hss_info_t;

/* Fills *opts with defaults: leaf_size 128, rtol 1e-6, atol 0, d0 64,
 * d_step 32, d_max 0 (= n), oversample_p 10, NATIVE sampling, seed 0,
 * tree NULL (bisection), symmetric 0. */
hss_status hss_default_opts(hss_opts* opts);

/*
 * hss_compress -- randomized HSS compression (Algorithm 1 with Algorithm 5's
 * late-notification adaptive sampling, processed level by level).
 *   A      device, n x n row-major, leading dimension lda >= n, dtype
 *          HSS_F32 or HSS_F64.  Borrowed for the call only: D and B blocks
 *          are copied out, the caller may free A afterwards.
 *   opts   host; NULL = hss_default_opts.
 *   out    host; receives a new handle (NULL on error).
 * Errors: INVALID (n < 1, lda < n, bad options), OOM, CUDA, TIMEOUT (a
 * bounded device-side wait of the sampling or ID kernels gave up; no handle),
 * RANK_CAP (the handle is still returned in *out with the nodes that did
 * compress, and must be destroyed).  Synchronizes `stream`.
 */
hss_status hss_compress(const void* A, int64_t n, int64_t lda, hss_dtype dtype,
                        const hss_opts* opts, void* stream, hss_t* out);

/*
 * Matrix-free access to A: the randomized compression needs only products
 * of A and A^T with random blocks and selected entries of A (Section 2.2;
 * A "does not need to be explicitly formed").  Both callbacks run on the
 * thread that called hss_compress_matfree, queue their device work on
 * `stream` (the compression's stream) and return 0 on success.  Every
 * buffer they receive is device memory of the library, valid until the work
 * they queue has completed; elements have the handle's dtype.
 */
typedef struct {
  /* Sr[:, 0:c] = A R and, when Sc is not NULL, Sc[:, 0:c] = A^T R for the
   * n x c block R (all rows; no leaf masking).  R, Sr, Sc row-major with
   * leading dimensions ldr, lds. */
  int (*sample)(void* ctx, int64_t c, const void* R, int64_t ldr, void* Sr, void* Sc,
                int64_t lds, void* stream);
  /* out[i * ldo + j] = A(rows[i], cols[j]) for i < nr, j < nc (rows, cols:
   * int32 indices in [0, n)). */
  int (*extract)(void* ctx, const int32_t* rows, int64_t nr, const int32_t* cols, int64_t nc,
                 void* out, int64_t ldo, void* stream);
  void* ctx;
} hss_matfree;

/*
 * hss_compress_matfree -- hss_compress for a matrix given only through
 * `ops` (host struct, read during the call).  The leaf blocks D and the
 * generators B are extracted; the leaf samples are formed after the
 * products as S(I_t,:) - D_t R(I_t,:) (Algorithm 1 as printed), and
 * hss_opts.sample_mode is not used (the callback's arithmetic is).
 * Errors: as hss_compress, plus INVALID when a callback returns non-zero
 * (no handle).  Synchronizes `stream`.
 */
hss_status hss_compress_matfree(int64_t n, hss_dtype dtype, const hss_matfree* ops,
                                const hss_opts* opts, void* stream, hss_t* out);

/*
 * hss_matvec -- B = H X with the compressed form (Algorithm 2).
 *   X  device, n x nrhs row-major, ldx >= nrhs, the handle's dtype.
 *   B  device, n x nrhs row-major, ldb >= nrhs; must not overlap X.
 * Errors: INVALID, OOM, CUDA.  Stream-ordered: the call returns without
 * waiting for the device (its small tables go up through pinned blocks of
 * the calling thread, eight of which may be in flight).
 */
hss_status hss_matvec(hss_t h, const void* X, int64_t ldx, int64_t nrhs,
                      void* B, int64_t ldb, void* stream);

/*
 * hss_factor -- ULV-like factorization of the compressed form (Algorithm 3),
 * in FP64 whatever the handle's dtype.  Errors: SINGULAR (zero pivot in the
 * root LU), OOM, CUDA.  Synchronizes `stream`.
 */
hss_status hss_factor(hss_t h, void* stream);

/*
 * hss_solve -- X = H^{-1} B with the ULV factors (Algorithm 4).
 *   B  device, n x nrhs row-major, ldb >= nrhs, the handle's dtype.
 *   X  device, n x nrhs row-major, ldx >= nrhs (may equal B when ldx == ldb).
 * Errors: STATE (no hss_factor yet), INVALID, OOM, CUDA.  Stream-ordered,
 * returning without waiting for the device, as hss_matvec.
 */
hss_status hss_solve(hss_t h, const void* B, int64_t ldb, int64_t nrhs,
                     void* X, int64_t ldx, void* stream);

/* hss_info -- statistics of the handle into *info (host). */
hss_status hss_info(hss_t h, hss_info_t* info);

/*
 * hss_node_ranks -- per-node ranks, nodes numbered breadth-first (root 0,
 * children of a node are consecutive).  lo, hi, kr, kc are host arrays of
 * `cap` entries (any may be NULL); entry i gets node i's interval [lo, hi)
 * and its row / column rank (-1 for the root).  Returns the node count in
 * *count.  Errors: INVALID (cap smaller than the node count).
 */
hss_status hss_node_ranks(hss_t h, int32_t* lo, int32_t* hi, int32_t* kr,
                          int32_t* kc, int32_t cap, int32_t* count);

/* hss_kernel_launches -- number of CUDA kernels this library has launched in
 * the calling process so far (all threads, all handles). */
int64_t hss_kernel_launches(void);

/* hss_destroy -- frees every device buffer of the handle (NULL is a no-op). */
void hss_destroy(hss_t h);

/* hss_last_error -- message of the last failed call on h (NULL: the calling
 * thread's last failed call that had no handle).  Never NULL. */
const char* hss_last_error(hss_t h);

/* ---------------------------------------------------------------------------
 * Batched compression (many matrices in lockstep) and its incremental form.
 *
 * A batch holds jobs of one dtype on one stream.  Each hss_batch_step runs
 * one round: new jobs build their tree and draw their first samples; every
 * other job processes one tree level (Algorithm 1, Algorithm 5 per node),
 * and the level work of all jobs goes into shared launches (one ID launch for
 * every node side of every job, one rank read-back per round).  Jobs may be
 * submitted between steps (continuous batching).
 * ------------------------------------------------------------------------- */
typedef struct hss_batch_s* hss_batch_t;

/* Creates an empty batch.  Errors: INVALID. */
hss_status hss_batch_create(hss_dtype dtype, void* stream, hss_batch_t* out);

/* Queues the compression of A (device, n x n row-major, lda; the batch's
 * dtype).  A must stay valid until the job finishes (hss_batch_take
 * succeeds).  *ticket identifies the job.  Errors: INVALID (bad A, n, lda,
 * options; message in hss_batch_last_error). */
hss_status hss_batch_submit(hss_batch_t b, const void* A, int64_t n, int64_t lda,
                            const hss_opts* opts, int64_t* ticket);

/* Runs one round; *active receives the number of jobs still running.
 * Synchronizes the stream once per round (rank read-back).  Errors: CUDA,
 * OOM (batch-wide failures); a job's own failure is reported by take. */
hss_status hss_batch_step(hss_batch_t b, int32_t* active);

/* Hands over the handle of a finished job (the batch forgets the ticket).
 * Returns the job's status: OK, RANK_CAP (handle still returned), or its
 * error (no handle); STATE if the job is still running; INVALID for an
 * unknown ticket. */
hss_status hss_batch_take(hss_batch_t b, int64_t ticket, hss_t* out);

/* Message of the batch's last failed call (never NULL). */
const char* hss_batch_last_error(hss_batch_t b);

/* Destroys the batch and every job not taken. */
void hss_batch_destroy(hss_batch_t b);

/* Compresses `count` matrices together (one batch run to completion).
 *   A, n, lda: host arrays of count entries (A[i] device pointers).
 *   opts: NULL (defaults), one hss_opts (opts_stride = 0) or count of them
 *   (opts_stride = 1).  out: host array of count handles; status: optional
 *   host array of count per-matrix statuses.  Returns the first non-OK
 *   status.  Synchronizes the stream. */
hss_status hss_compress_batched(int32_t count, const void* const* A, const int64_t* n,
                                const int64_t* lda, hss_dtype dtype, const hss_opts* opts,
                                int32_t opts_stride, void* stream, hss_t* out,
                                hss_status* status);

/*
 * hss_factor_batched -- hss_factor (Algorithm 3) of `count` handles of one
 * dtype together: level by level from each tree's deepest level, the nodes
 * of all handles at that round share one launch.  Each node's arithmetic is
 * that of hss_factor, so the factors are bitwise the same.
 *   hs: host array of count handles; status: optional host array of count
 *   per-handle statuses (each handle keeps its own message).
 * Returns the first non-OK status (INVALID for mixed dtypes).  Synchronizes
 * the stream.
 */
hss_status hss_factor_batched(int32_t count, hss_t* hs, void* stream, hss_status* status);

/*
 * hss_solve_batched -- hss_solve (Algorithm 4) of `count` systems on handles
 * of one dtype: X[q] = H_q^{-1} B[q], with B[q], X[q] device n_q x nrhs[q]
 * row-major (ldb[q], ldx[q]); all host arrays of count entries.  The upward
 * and downward sweeps of all systems share one launch per round; the
 * results are bitwise those of one hss_solve per system.  A handle may
 * appear more than once.  Returns the first non-OK status; status: optional
 * per-system statuses.  Stream-ordered.
 */
hss_status hss_solve_batched(int32_t count, hss_t* hs, const void* const* B, const int64_t* ldb,
                             const int64_t* nrhs, void* const* X, const int64_t* ldx,
                             void* stream, hss_status* status);

/* ---------------------------------------------------------------------------
 * Step-level entry points.  They run single steps of the compression on
 * caller buffers; hss_compress runs the same kernels.
 * ------------------------------------------------------------------------- */

/*
 * hss_random_gaussian -- columns [c0, c1) of the n x d random matrix R of
 * Section 2.2.  R[i, j] is a standard Gaussian from the splitmix64 sequence
 * (outputs 2q+1 and 2q+2 for q = i*2^32 + j, Box-Muller in FP64) rounded to
 * the nearest bfloat16, stored as dtype.
 *   R  device, row-major, ldr >= c1; row i, column j at R[i*ldr + j].
 * Errors: INVALID, CUDA.  Stream-ordered.
 */
hss_status hss_random_gaussian(uint64_t seed, int64_t n, int64_t c0, int64_t c1,
                               void* R, int64_t ldr, hss_dtype dtype, void* stream);

/*
 * hss_sample -- fused sampling (Section 2.2, step 2): for columns [c0, c1)
 *   Sr[:, c] = (A - D) R[:, c],   Sc[:, c] = (A - D)^T R[:, c],
 * reading every tile of A from device memory once for both products.  D is
 * the block diagonal of the leaf blocks A(I_t, I_t) of the cluster tree given
 * by `leaf_starts` (host, nleaf+1 increasing offsets, leaf_starts[0] = 0,
 * leaf_starts[nleaf] = n); nleaf = 0 means no masking (D = 0).  With the
 * mask, Sr(I_t, :) is Algorithm 1's S^r_loc = S^r(I_t,:) - D_t R(I_t,:).
 *   A  device n x n row-major (lda);  R, Sr, Sc device n x ld row-major with
 *   ldr / lds >= c1.  mode: hss_sample_mode (NATIVE only for HSS_F64).
 *   Sc may be NULL: only Sr is formed (a symmetric A, whose S^c is S^r; the
 *   tensor-core kernel then skips the column product), with the same bits
 *   in Sr as when Sc is given.
 * The split-BF16 modes on the tensor cores accumulate in FP32 over at most
 * 24 MMAs at a time and sum those partial results in FP32 on the CUDA cores.
 * Errors: INVALID, OOM (scratch for the partial sums), CUDA, TIMEOUT (a
 * bounded pipeline wait of the tensor-core kernel gave up).  The tensor-core
 * path synchronizes the stream to read its error flag; the others are
 * stream-ordered.
 */
hss_status hss_sample(const void* A, int64_t n, int64_t lda, hss_dtype dtype,
                      const void* R, int64_t ldr, int64_t c0, int64_t c1,
                      void* Sr, void* Sc, int64_t lds,
                      const int64_t* leaf_starts, int32_t nleaf, int32_t mode,
                      void* stream);

/*
 * hss_id_batched -- interpolative decompositions [X, J] = ID(Y_b, eps) of a
 * batch of matrices by truncated column-pivoted QR in FP64 (Section 2.2,
 * Section 3.1): the factorization of Y_b (d_b x m_b) stops at the first i
 * with |R_ii| <= max(rtol |R_11|, atol), k_b = i (min(d_b, m_b) if none).
 *   Yt     device array (count entries) of device pointers; Y_b is stored
 *          TRANSPOSED, as m_b rows of d_b values: column j of Y_b is the
 *          contiguous row Yt[b] + j*ldy[b].  dtype of the values: dtype.
 *   m, d, ldy   device int32 arrays (count entries).
 *   perm   device array of device int32 pointers, m_b entries each: on return
 *          perm[b][0..k) = J (pivot order), perm[b][k..m) = the other
 *          columns in increasing order.
 *   E      device array of device double pointers; E_b is written as a dense
 *          (m_b - k_b) x k_b row-major matrix (ld = k_b), so each buffer
 *          needs m_b * min(d_b, m_b) doubles at most.  E = (R1^{-1} R2)^T,
 *          so that X^T = Pi [I; E] with Pi the permutation `perm`.
 *   k      device int32 array (count): the ranks.
 * A few large items are spread over all SMs (a cooperative launch whose CTAs
 * meet at a bounded barrier in global memory); the results are bitwise the
 * same either way.
 * Errors: INVALID, OOM, CUDA, TIMEOUT (a barrier wait of that mode gave up;
 * the outputs are then undefined).  Stream-ordered, except that the
 * spread-out mode synchronizes the stream to read its error flag.
 */
hss_status hss_id_batched(int32_t count, const void* const* Yt, const int32_t* m,
                          const int32_t* d, const int32_t* ldy, hss_dtype dtype,
                          double rtol, double atol, int32_t* const* perm,
                          double* const* E, int32_t* k, void* stream);

/*
 * hss_sample_noalloc -- hss_sample for callers that cannot allocate device
 * memory.  The paper has no counterpart: this is a deployment variant.  Two
 * kinds of caller need it: a host application whose own memory manager owns
 * the whole GPU (memory taken behind its back breaks its budget), and a
 * serving loop that allows no allocator call once it runs, because cudaMalloc
 * and cudaFree can block or synchronize the device and stall other work.
 *   Same arguments, layouts and results as hss_sample; the caller still
 *   provides A, R, Sr and Sc.  The scratch (partial sums of both products,
 *   the leaf mask) lives in fixed file-scope device arrays of the library,
 *   about 36 MiB on every GPU that loads it, held until the process exits.
 *   Limits: n <= 2048, c1 - c0 <= 64, nleaf <= 2048; larger problems, and any
 *   call whose scratch need exceeds the fixed arrays, return HSS_ERR_INVALID
 *   before any work is queued (use hss_sample).  It calls no cudaMalloc,
 *   cudaFree or other allocating routine.
 *   The first call on a device looks up the arrays' device addresses with
 *   cudaGetSymbolAddress (with that device current); make that first call
 *   before any stream capture.  leaf_starts is copied to the device with
 *   cudaMemcpyAsync from the caller's host memory: from pageable memory that
 *   copy returns only once the bytes are staged, pinned memory keeps it
 *   asynchronous.  The split-BF16 modes on the tensor cores synchronize the
 *   stream to read their error flag, as in hss_sample.
 *   Every call shares the same arrays, which keep the last call's contents
 *   (nothing in them needs to start at zero: a call writes every entry it
 *   reads); calls whose GPU work overlaps -- two streams, two threads --
 *   race on them, so serialize them.
 * Errors: INVALID, CUDA, TIMEOUT (message in hss_last_error(NULL)).
 */
hss_status hss_sample_noalloc(const void* A, int64_t n, int64_t lda, hss_dtype dtype,
                              const void* R, int64_t ldr, int64_t c0, int64_t c1,
                              void* Sr, void* Sc, int64_t lds,
                              const int64_t* leaf_starts, int32_t nleaf, int32_t mode,
                              void* stream);

/*
 * hss_pool_bytes -- device memory of the library's private stream-ordered
 * pool on the current device: *used = bytes currently handed out (handles,
 * temporaries of calls in flight), *reserved = bytes the pool holds from the
 * device (freed memory is kept for reuse).  Either pointer may be NULL.  The
 * fixed arrays of hss_sample_noalloc are not part of the pool.
 * Errors: CUDA.
 */
hss_status hss_pool_bytes(int64_t* used, int64_t* reserved);

/*
 * hss_tuner_stats -- state of the library's measuring tuner of the ID launch
 * shape (threads per column).  Launches are grouped into shape classes; the
 * first launches of a class time the instruction-count model's choice and
 * its neighbours with CUDA events (the results do not depend on the choice),
 * later ones use the fastest.  Outputs (any may be NULL): classes seen,
 * classes settled, timed trial launches.  HSS_AUTOTUNE=0 in the environment
 * switches the tuner off (the model's choice everywhere).  Never fails.
 */
hss_status hss_tuner_stats(int32_t* classes, int32_t* settled, int32_t* trials);

/* ---------------------------------------------------------------------------
 * Fault injection, for testing how a caller handles failures (the paper has
 * no counterpart).  Nothing here faults the GPU: an allocation failure is
 * simulated on the host, and a device-side wait is only made to give up
 * early, after which the kernel returns its error status normally.
 * ------------------------------------------------------------------------- */
typedef enum {
  HSS_FAULT_NONE = 0,        /* clear every injected fault                          */
  HSS_FAULT_OOM = 1,         /* the value-th device allocation from now (1 = the
                                next) fails with HSS_ERR_OOM, once                  */
  HSS_FAULT_WAIT_LIMIT = 2   /* the bounded barrier wait of the ID's spread-out
                                (group) mode gives up after `value` clock cycles
                                instead of about 2^33; 0 restores the default       */
} hss_fault;

/*
 * hss_set_fault -- arms (or, with HSS_FAULT_NONE, clears) one injected fault
 * for the whole process.  The environment variable HSS_FAULT, read when the
 * library loads, arms the same faults without a call: "oom:N" or
 * "wait:CYCLES".  Errors: INVALID (unknown kind, negative value).
 */
hss_status hss_set_fault(int32_t kind, int64_t value);

#ifdef __cplusplus
}
#endif

#endif /* HSS_H */
