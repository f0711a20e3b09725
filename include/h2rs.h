/*
 * h2rs — strong recursive skeletonisation (RS-S) factorisation and solve of a
 * symmetric H^2 matrix on one NVIDIA B300 (sm_103a).
 *
 * The method is that of "Linear Complexity H^2 Direct Solver for Fine-Grained
 * Parallel Architectures" (Boukaram, Keyes, Li, Liu, Turkiyyah): the factorisation
 * of Alg. 1 / Alg. 2 (Sec. 2.1-2.2, Eq. 2.1) and the solve of Alg. 3 (Sec. 2.3).
 * Iterative refinement with a float64 H^2 residual is added on top of the paper's
 * solve so that a reduced-precision factor can reach a float64 backward error.
 *
 * Conventions
 *  - All functions return 0 (H2_OK) on success and a negative H2_ERR_* code on
 *    failure; h2_last_error() returns a thread-local message for the last failure.
 *    No C++ exception crosses this interface and no kernel traps.
 *  - Vectors are in cluster-tree order (the order of h2_matrix_desc.node_start);
 *    multiple right-hand sides are column-major with a leading dimension.
 *  - Dense blocks are column-major float64.
 *  - Nodes of the complete binary cluster tree use heap numbering: level l holds
 *    the ids 2^l-1 .. 2^(l+1)-2, node g has children 2g+1 and 2g+2.
 *  - A batch of independent matrices (h2_matrix_create_batch) is one h2_matrix whose
 *    vectors are the systems' vectors stacked in the caller's order.
 *  - "device" pointers are CUDA device pointers of the current device; the
 *    library runs every kernel on the stream given in the options / descriptor
 *    (NULL = the legacy default stream).
 */
#ifndef H2RS_H
#define H2RS_H

#include <stdint.h>

#if defined(__GNUC__)
#define H2_API __attribute__((visibility("default")))
#else
#define H2_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status codes */
enum {
    H2_OK = 0,
    H2_ERR_ARG = -1,            /* invalid argument or inconsistent descriptor       */
    H2_ERR_OOM = -2,            /* device or host allocation failed                   */
    H2_ERR_SINGULAR = -3,       /* zero or non-finite pivot in a redundant/top block  */
    H2_ERR_RANK_CAP = -4,       /* augmented rank above h2_factor_opts.k_cap          */
    H2_ERR_NONFINITE = -5,      /* non-finite value in an input or a result          */
    H2_ERR_NO_CONVERGENCE = -6, /* refinement did not reach the tolerance in maxit   */
    H2_ERR_TIMEOUT = -7,        /* a bounded device wait gave up                      */
    H2_ERR_CUDA = -8,           /* a CUDA runtime call failed                         */
    H2_ERR_STATE = -9           /* object used in a wrong state                       */
};

/* working precision of the factorisation and of the solve that applies it */
enum {
    H2_PREC_FP64 = 0,           /* float64 everywhere                                 */
    H2_PREC_FP32 = 1,           /* float32 factor and solve; the top-level dense LU
                                   and the refinement residual stay float64           */
    H2_PREC_TF32X3 = 2          /* as H2_PREC_FP32, with the Schur update on the tensor
                                   cores: float32 operands split into two TF32 parts
                                   (hi*hi + hi*lo + lo*hi, float32 accumulation; about
                                   7e-7 relative error per product sum against 1e-7
                                   for float32 FMA)                                  */
};

/* ------------------------------------------------------------------ H^2 matrix */
/*
 * Descriptor of a symmetric H^2 matrix A = H + D (Sec. 1.1, Fig. 1-3):
 *   admissible blocks  A_st = U_s S_st U_t^T  with nested orthonormal bases
 *   U_p = diag(U_c1, U_c2) [E_c1; E_c2], and dense near-field blocks on the
 *   inadmissible leaf pairs.  All index arrays are HOST arrays; the four value
 *   arrays U, E, S, D are host or device arrays (values_on_device).
 *
 *   n               matrix size
 *   depth           d: leaves at level d, root at level 0 (nnodes = 2^(d+1)-1)
 *   node_start[g]   first tree-order index of node g         (nnodes)
 *   node_size[g]    number of indices of node g              (nnodes)
 *   rank[g]         basis rank k_g of node g                 (nnodes)
 *   U_off[i]        leaf i (node 2^d-1+i): U_i = U[U_off[i] ..], node_size x rank
 *                   (2^d + 1 entries, last = total)
 *   E_off[g]        transfer E_g (rank_g x rank_parent), g >= 1; E_off[0] = 0
 *                   (nnodes + 1 entries)
 *   adm_ptr[g]      CSR over all nodes of the admissible pairs (s = g, t) of the
 *   adm_col[e]      same level (nnodes + 1 / nadm entries), symmetric pattern,
 *                   columns sorted, no pair also inadmissible (all checked)
 *   S_off[e]        coupling S_st (rank_s x rank_t) of entry e (nadm + 1 entries)
 *   inad_ptr[g]     CSR over all nodes of the inadmissible pairs of the same
 *   inad_col[e]     level, including (g, g), symmetric pattern (checked),
 *                   columns sorted (checked)
 *   D_off[j]        dense block (size_s x size_t) of the j-th inadmissible entry of
 *                   a LEAF row, in CSR order (nnear + 1 entries)
 * The library copies everything it needs; the caller keeps ownership of its
 * arrays, which may be freed after h2_matrix_create returns.
 */
typedef struct {
    int64_t n;
    int32_t depth;
    int32_t values_on_device;
    const int64_t* node_start;
    const int64_t* node_size;
    const int64_t* rank;
    const int64_t* U_off;
    const double* U;
    const int64_t* E_off;
    const double* E;
    const int64_t* adm_ptr;
    const int64_t* adm_col;
    const int64_t* S_off;
    const double* S;
    const int64_t* inad_ptr;
    const int64_t* inad_col;
    const int64_t* D_off;
    const double* D;
    void* stream;               /* cudaStream_t used for the copies */
} h2_matrix_desc;

typedef struct h2_matrix h2_matrix;   /* opaque: device copy of A + its level plans */
typedef struct h2_factor h2_factor;   /* opaque: owns all device memory of Z         */

/* Copy A to the device and plan its level structure (near-field graph, greedy
 * colouring, fill pattern, Schur target lists; Sec. 2.2).  *out is set on success.
 * Errors: H2_ERR_ARG (inconsistent descriptor), H2_ERR_OOM, H2_ERR_CUDA. */
H2_API int h2_matrix_create(const h2_matrix_desc* desc, h2_matrix** out);
H2_API void h2_matrix_destroy(h2_matrix* A);

/* A batch of nsys independent symmetric H^2 matrices (descs[0..nsys-1], each as for
 * h2_matrix_create, of any sizes and depths) as one block-diagonal h2_matrix.  The
 * trees are aligned by height above the leaves, so every level of the factorisation
 * and of the solve treats the boxes of all systems in the same kernel launches
 * (Sec. 2.2 applied to a forest; the paper treats one matrix).  Vectors are the
 * systems' tree-order vectors stacked in the order of descs (system s starts at row
 * sum_{q<s} descs[q].n).  The values are copied with descs[s].values_on_device; every
 * copy runs on descs[0].stream.  Errors as h2_matrix_create. */
H2_API int h2_matrix_create_batch(int32_t nsys, const h2_matrix_desc* descs, h2_matrix** out);

/* Number of systems of A and their row offsets (sys_offset: nsys+1 entries, last = n);
 * either output may be NULL.  Errors: H2_ERR_ARG. */
H2_API int h2_matrix_batch_info(const h2_matrix* A, int32_t* nsys, int64_t* sys_offset);

/* y = A x in float64: the H^2 matrix-vector product of the format of Sec. 1.1
 * (Fig. 1-3): upsweep through the nested bases, couplings S_st, downsweep, dense
 * near field.  x: n x nrhs (ldx >= n), y: n x nrhs (ldy >= n); both device pointers
 * when on_device != 0, else host pointers (copied in and out).  Errors: H2_ERR_ARG,
 * H2_ERR_CUDA. */
H2_API int h2_matvec(const h2_matrix* A, int32_t nrhs, const double* x, int64_t ldx,
              double* y, int64_t ldy, int32_t on_device);

/* The same product with no device allocation.  The paper has no counterpart: it is
 * for callers that may not allocate device memory while it runs, such as an
 * application that reserves all of the GPU's memory for itself up front and forbids
 * any further cudaMalloc/cudaFree (or stream-ordered allocation) by the libraries it
 * calls.  The coefficient vectors live in one static device array of
 * H2_MATVEC_STATIC_WORDS doubles (32 MiB) that every GPU loading the library keeps
 * until the process exits.  x and y (n x nrhs, ldx/ldy >= n) must be device (or
 * managed) memory of the matrix's device, and that device must be current; host or
 * other-device pointers are rejected with H2_ERR_ARG.  Calls needing more than the
 * array (2 * sum(rank) * nrhs doubles) return H2_ERR_ARG with a message.  The first
 * call on a device looks up the array's device address, so make that first call
 * before any stream capture.  The call waits for the matrix's stream to finish
 * before it returns.  All calls share the array and it keeps the last call's contents
 * (every value read is written first within a call); calls that overlap on the GPU
 * race, so serialise them.  Errors: H2_ERR_ARG, H2_ERR_CUDA. */
#define H2_MATVEC_STATIC_WORDS (1 << 22)
H2_API int h2_matvec_static(const h2_matrix* A, int32_t nrhs, const double* x, int64_t ldx,
                            double* y, int64_t ldy);

/* ------------------------------------------------------------- factorisation */
typedef struct {
    double eps_lu;              /* truncation threshold of the fill (Alg. 1)           */
    double norm_a;              /* ||A||_2 supplied by the caller: eps_fill = eps_lu*norm_a */
    int32_t precision;          /* H2_PREC_*                                           */
    int32_t flags;              /* H2_FLAG_* bits, 0 by default                        */
    void* stream;               /* cudaStream_t for every kernel of this factor        */
    const double* sys_norm_a;   /* batch: ||A_s||_2 of every system (host, nsys values,
                                   copied); NULL = norm_a for all.  Each system's
                                   eps_fill and backward error use its own norm       */
    const int32_t* force_ranks; /* debug (host, copied; NULL = off): the augmented rank
                                   k~_i of every box of every skeletonised level, levels
                                   0 (leaves) .. nlevels-1 concatenated in the box order
                                   of h2_layout_get / h2_plan_query (the box counts of
                                   those levels, summed).  The factorisation then keeps
                                   k~_i - k_i fill vectors (the largest singular values,
                                   clamped to what the box can hold) instead of
                                   truncating at eps_fill, so that its layouts can be
                                   compared entry by entry with another factorisation
                                   of the same matrix (e.g. float32 against float64).  */
    int32_t k_cap;              /* cap on every augmented rank k~_i (0 = none): the
                                   ranks are checked on the host when they are read
                                   back after each level, and a level with a rank above
                                   the cap fails with H2_ERR_RANK_CAP (h2_last_error
                                   names the first such box and level; retry with a
                                   larger cap).  Negative: H2_ERR_ARG.                   */
} h2_factor_opts;

/* h2_factor_opts.flags: time every factorisation kernel launch with CUDA events
 * (h2_factor_stats.kernel_ms / kernel_launches); adds about a microsecond per launch */
#define H2_FLAG_TIME_KERNELS 1
/* h2_factor_opts.flags, for testing the failure path only: every wait of the
 * tensor-core Schur pipeline (H2_PREC_TF32X3) gives up after one SM cycle instead of
 * about two seconds, so the factorisation fails with H2_ERR_TIMEOUT (the kernel still
 * waits, with the full budget, for the MMAs it issued before freeing tensor memory);
 * the library stays usable afterwards */
#define H2_FLAG_DEBUG_SHORT_WAIT 2
/* h2_factor_opts.flags: how D_RR^-1 (Sec. 2.1, Eq. 2.1) is applied in W_U, W_L and the
 * diagonal solve step.  By default H2_PREC_FP32 / H2_PREC_FP64 use triangular solves
 * with the LU factors and H2_PREC_TF32X3 forms D_RR^-1 explicitly and applies it as
 * GEMMs; these flags override the default (setting both is H2_ERR_ARG).  Triangular
 * solves are the more accurate on ill-conditioned problems. */
#define H2_FLAG_W_TRIANGULAR 4
#define H2_FLAG_W_INVERSE 8

/* kernel ids of h2_factor_stats.kernel_* */
enum {
    H2_K_GATHER = 0,            /* fill-row gather Y = (I - V V^T) F                   */
    H2_K_BASIS = 1,             /* R-factor of Y^T + Jacobi SVD + completion          */
    H2_K_PROJ = 2,              /* Q~^T B and B Q~ projections                         */
    H2_K_ZERO = 3,              /* truncation / eliminated rows and columns           */
    H2_K_LU = 4,                /* LU of the redundant blocks                          */
    H2_K_TRSM = 5,              /* W_U and W_L triangular solves                       */
    H2_K_SCHUR = 6,             /* target-owned Schur update                           */
    H2_K_CLOSE = 7,             /* level close (blocks and bases)                      */
    H2_K_TOP = 8,               /* top-level assembly and float64 LU                   */
    H2_K_LOAD = 9,              /* leaf near-field and basis load                      */
    H2_K_PACK = 10,             /* TF32 hi / lo packing of the tensor-core Schur operands */
    H2_K_COUNT = 11
};

/* Factorise A (Alg. 1): levels d..t, greedy colours in order, per colour the
 * batched basis augmentation (QR of the fill row + one-sided Jacobi SVD), orthogonal
 * completion, projection, partial LU and target-owned Schur update; level close;
 * float64 dense LU of the top level.  The factor keeps a pointer to A's plans, so A
 * must outlive it.  Errors: H2_ERR_ARG, H2_ERR_OOM, H2_ERR_SINGULAR (see
 * h2_factor_stats: error_level / error_box), H2_ERR_NONFINITE, H2_ERR_CUDA. */
H2_API int h2_factor_create(const h2_matrix* A, const h2_factor_opts* opts, h2_factor** out);
H2_API void h2_factor_destroy(h2_factor* Z);

/* Solve A x = b with the factor (Alg. 3), in place: b (n x nrhs, ldb >= n) is
 * overwritten with x.  Device pointer when on_device != 0, else host (copied).
 * The solve runs in the factor's precision.  Errors: H2_ERR_ARG, H2_ERR_CUDA. */
H2_API int h2_solve(const h2_factor* Z, int32_t nrhs, double* b, int64_t ldb, int32_t on_device);

/* Iterative refinement in float64: x0 = solve(b), then corrections
 * x_{k+1} = x_k + solve(b - A x_k); once a correction fails to halve the backward
 * error (eps_lu * cond(A) near 1) the remaining corrections are restarted flexible
 * GMRES(30) cycles on A d = b - A x_k right-preconditioned by the factor (the
 * preconditioned basis is kept, so a reduced-precision solve need not be linear).  Stops when the max over columns (and, for a batch, over systems s) of
 * ||b_s - A_s x_s|| / (||A_s|| ||x_s||) <= tol or after maxit corrections (plain steps
 * plus GMRES iterations).  b, x: n x nrhs (device
 * when on_device != 0).  *iters receives the number of corrections, *berr the final
 * backward error.  Returns H2_ERR_NO_CONVERGENCE (x still written) if tol was not
 * reached. */
H2_API int h2_refine_solve(const h2_factor* Z, const h2_matrix* A, int32_t nrhs,
                    const double* b, int64_t ldb, double* x, int64_t ldx,
                    double tol, int32_t maxit, int32_t on_device,
                    int32_t* iters, double* berr);

/* ------------------------------------------------------------------ inspection */
typedef struct {
    int32_t nlevels;            /* skeletonised levels (d .. t); for a batch, forest
                                   levels holding at least one skeletonised box       */
    int32_t top_level;          /* t, or -1 when no block is admissible; for a batch,
                                   the smallest t over the systems (forest levels)    */
    int64_t top_size;           /* order of the dense top-level matrix; for a batch,
                                   the sum of the systems' top orders                 */
    int64_t factor_bytes;       /* device bytes held by the factor                     */
    int64_t peak_bytes;         /* peak device bytes during the factorisation          */
    int32_t error_level;        /* level / local box of the last singular pivot, or -1 */
    int32_t error_box;
    double factor_ms;           /* device time of the last factorisation               */
    double phase_ms[8];         /* augment, complete+project, lu+trsm, schur, close,
                                   top, leaf load, other                              */
    double phase_flops[8];      /* algorithmic flops of the same phases                */
    double phase_bytes[8];      /* algorithmic bytes of the same phases                */
    double kernel_ms[16];       /* H2_FLAG_TIME_KERNELS: summed launch times per H2_K_* */
    int64_t kernel_launches[16];
    double host_ms[4];          /* host time of the factorisation: per-level work lists,
                                   their uploads, level setup + close bookkeeping, and
                                   waits for the per-level rank read-back            */
    double schur_reread_bytes;  /* Schur operand bytes counted once per target a
                                   contributor feeds (the kernel's L2 re-reads); the
                                   Schur entry of phase_bytes counts every operand once
                                   per colour and every target once (read + write)    */
} h2_factor_stats;

H2_API int h2_factor_stats_get(const h2_factor* Z, h2_factor_stats* out);

/* Per-level layout of the factorisation, levels numbered 0 = leaves (depth d) up to
 * nlevels-1 (level t); for a batch, forest levels (every system's boxes at that height,
 * see h2_plan_query_batch for each box's system and state).  h2_layout_counts gives the number of boxes and blocks;
 * h2_layout_get fills caller arrays (any may be NULL):
 *   sizes[nbox]   n_i at that level       ranks[nbox]  augmented rank k~_i
 *   colour[nbox]  greedy colour            row_ptr[nbox+1], col[nblk], kind[nblk]
 *   offset[nblk+1] prefix sums of n_j*n_k over the merged (near + fill) block list
 *   kind: 0 near-field block, 1 fill-in block. */
H2_API int h2_layout_counts(const h2_factor* Z, int32_t level, int64_t* nbox, int64_t* nblk);
H2_API int h2_layout_get(const h2_factor* Z, int32_t level, int64_t* sizes, int64_t* ranks,
                  int32_t* colour, int64_t* row_ptr, int64_t* col, int32_t* kind,
                  int64_t* offset);

/* Host-only query of the level plan (no GPU needed): for the skeletonised level
 * `level` (0 = leaves), the number of boxes and of merged blocks, the greedy colour
 * of every box and the merged block CSR with kinds, exactly as h2_factor_create
 * will use them.  Only the index arrays of the descriptor are read.  Arrays may be
 * NULL (counts only).  Errors: H2_ERR_ARG (also for a level that is not skeletonised). */
H2_API int h2_plan_query(const h2_matrix_desc* desc, int32_t level, int64_t* nbox, int64_t* nblk,
                  int32_t* colour, int64_t* row_ptr, int64_t* col, int32_t* kind);

/* The same for a batch (as h2_matrix_create_batch): forest level `level` counted from
 * the leaves, up to and including the last level, which holds dense top matrices only.
 * Per box additionally: state (0 above its system's top, 1 skeletonised at this level,
 * 2 part of its system's dense top matrix; colour is -1 unless 1) and system (index
 * into descs).  Boxes of one system are contiguous and in their tree's order. */
H2_API int h2_plan_query_batch(int32_t nsys, const h2_matrix_desc* descs, int32_t level, int64_t* nbox,
                               int64_t* nblk, int32_t* colour, int64_t* row_ptr, int64_t* col,
                               int32_t* kind, int32_t* state, int32_t* system);

/* Number of CUDA kernels this library has launched in the process so far (all
 * entry points; for counting launches inside a timed region). */
H2_API int64_t h2_kernel_launch_count(void);

H2_API const char* h2_last_error(void);
H2_API const char* h2_version(void);

#ifdef __cplusplus
}
#endif
#endif /* H2RS_H */
