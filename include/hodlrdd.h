/*
 * hodlrdd.h -- C ABI of the GB300 HODLRdD library (libhodlrdd.so).
 *
 * HODLRdD (Khan, Kandappan, Ambikasaran) represents a kernel matrix
 * K(i,j) = F(x_i, x_j) on N points in d dimensions (Section "Preliminaries",
 * kernel matrix) hierarchically: a balanced 2^d tree (Section "Construction of
 * the tree"), interaction lists under the HODLRdD weak admissibility condition
 * (far-field and vertex-sharing clusters are admissible; Table "Notations" and
 * the admissibility definition), every admissible block compressed by ACA
 * (Eq. keq1 / keq2, Algorithm 1), and an almost-linear matrix-vector product
 * (Algorithm 2). This library builds that representation on one GPU and applies
 * it with hand-written CUDA kernels.
 *
 * Conventions for every call:
 *  - Every function returns an int status (enum hodlrdd_status); nothing aborts.
 *    hodlrdd_last_error() gives a human-readable detail for the calling thread.
 *  - Pointer arguments marked "host or device" may point to host memory (pageable
 *    or pinned) or to device memory of the current device; the library finds out
 *    which with cudaPointerGetAttributes.
 *  - Invalid arguments are rejected on the host before any GPU work.
 *  - No type from CUDA or PyTorch appears here: a stream is passed as void*
 *    (a cudaStream_t; NULL is the legacy default stream).
 */
#ifndef HODLRDD_H
#define HODLRDD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hodlrdd_s* hodlrdd_handle;

enum hodlrdd_status {
  HODLRDD_OK = 0,
  HODLRDD_ERR_INVALID = 1,     /* bad argument (checked on the host) */
  HODLRDD_ERR_OOM = 2,         /* a device or host allocation failed; nothing leaks */
  HODLRDD_ERR_CUDA = 3,        /* a CUDA call failed; see hodlrdd_last_error() */
  HODLRDD_ERR_UNSUPPORTED = 4, /* valid but not supported (e.g. precision/nrhs combination) */
  HODLRDD_ERR_TIMEOUT = 5,     /* a bounded device-side wait gave up */
  HODLRDD_ERR_NUMERIC = 6      /* non-finite values met during the build */
};

/* Kernel functions F(x, y) of r = |x - y|_2. The paper's list F1..F8 (Section
 * "Preliminaries") plus the kernels of its experiments. Singular kernels
 * (LOG, INV_R, INV_R2_4D) evaluate to 0 at r = 0 (the matvec experiment sets
 * K(i,i) = 0). */
enum hodlrdd_kernel {
  HODLRDD_K_LOG = 0,        /* log r                                   (F2) */
  HODLRDD_K_INV_R = 1,      /* 1 / r                                   (F1) */
  HODLRDD_K_MATERN32 = 2,   /* (1 + sqrt(3) r / l) exp(-sqrt(3) r / l), l = p0 */
  HODLRDD_K_GAUSS = 3,      /* exp(-r^2 / (2 h^2)), h = p0 */
  HODLRDD_K_EXP = 4,        /* exp(-r / l), l = p0                     (F8) */
  HODLRDD_K_INV_R2_4D = 5,  /* -1 / (4 pi^2 r^2): 4D Laplace Green's function */
  HODLRDD_K_R = 6,          /* r                                       (F5) */
  HODLRDD_K_SIN = 7,        /* sin r                                   (F6) */
  HODLRDD_K_INV_SQRT1P = 8  /* 1 / sqrt(1 + r)                         (F7) */
};

/* Storage precision of the low-rank factors and arithmetic of the matvec.
 *  FP64: factors FP64, all arithmetic FP64; x and y are double.
 *  FP32: factors FP32, arithmetic FP32; x and y are float.
 *  FP16 / BF16: factors 16-bit with one FP32 scale per factor column, kernel
 *  evaluation and accumulation FP32; x and y are float.
 *  FP32_FP16: arithmetic FP32; each block's leading ACA terms stored in FP32 and
 *  its trailing terms, those after the last term with ||u_k|| ||v_k|| above
 *  2^-13 of the block's Frobenius norm (estimated from the terms), in FP16 with
 *  one FP32 power-of-two scale per column, so that their rounding stays below
 *  the FP32 rounding of the block; x and y are float. Right-hand sides are
 *  applied in chunks of at most 8.
 *  FP16X2: the low-rank applies run on the tensor cores (FP16 operands, FP32
 *  accumulation in tensor memory). Each factor entry is stored as two FP16
 *  numbers, hi = fp16(v / s) and lo = fp16((v / s - hi) 2^11), s a power of two
 *  per column, so that hi + 2^-11 lo keeps about 22 significant bits over the
 *  whole FP32 range; the vector operands are split the same way and the three
 *  products hi.hi, hi.lo, lo.hi are accumulated (the error stays at FP32 size).
 *  A block's trailing terms (as in FP32_FP16) keep the high part only.
 *  Right-hand sides go in chunks of 64 (fewer are padded); x and y are float;
 *  d <= 4 and lowrank_form 0. The near field is evaluated in FP32.
 * The compression itself (ACA) always runs in FP64. */
enum hodlrdd_precision {
  HODLRDD_PREC_FP64 = 0,
  HODLRDD_PREC_FP32 = 1,
  HODLRDD_PREC_FP16 = 2,
  HODLRDD_PREC_BF16 = 3,
  HODLRDD_PREC_FP32_FP16 = 4,
  HODLRDD_PREC_FP16X2 = 5
};

typedef struct hodlrdd_options {
  int precision;        /* enum hodlrdd_precision; default FP64 */
  int dense_if_cheaper; /* 1 (default): an IL block whose factors would hold at least
                           as many numbers as the block, p (m + n) >= m n, is applied
                           exactly by evaluating the kernel on the fly (no storage).
                           0: every IL block is applied through its ACA factors, as
                           in Algorithm 2.
                           2: the rule holds at the leaf level only; coarser IL
                           blocks keep their ACA factors whatever their rank (for the
                           tensor-core form, which streams a factor entry in less time
                           than it evaluates a kernel entry on the fly). */
  int max_nrhs;         /* >= 1 (default 8). Right-hand sides are processed in chunks
                           through a workspace sized at build: chunks of up to 16 for
                           FP32 handles with d <= 4 when max_nrhs >= 16, else up to 8;
                           any nrhs is accepted */
  int aca_max_rank;     /* cap on the ACA rank of blocks larger than 2048 rows or
                           columns (default 1024); a block that does not converge
                           within its cap is applied exactly instead */
  int near_mode;        /* leaf-level dense work of the packed path (FP32/FP16/BF16,
                           d <= 3, one right-hand side): 0 (default) chooses by work,
                           1 = one tile per parent box over the children of the
                           parent and of its neighbours sharing a d' >= 1 face (low-rank
                           leaf IL blocks inside the tile are subtracted), 2 = one task
                           per leaf box over its near and dense IL lists */
  int admissible_face_dim; /* admissibility of touching boxes: the largest
                           dimension of a shared face for which an IL block is still
                           compressed. 0 (default): HODLRdD (far-field and
                           vertex-sharing); -1: strong, far-field only (H-matrix);
                           d - 1: weak, every sibling (HODLR). Valid: -1 .. d - 1 */
  int lowrank_form;     /* what a low-rank block keeps after the build (Eq. keq2).
                           0 (default): the factors U_b (|I| x p) and V_b (|J| x p),
                           streamed from HBM by every product.
                           1: the memory-efficient skeleton form: the ACA pivot rows
                           sigma and columns tau and the LU factors of K(sigma, tau)
                           (p x p, FP64); each product evaluates K(sigma, J) and
                           K(I, tau) on the fly and solves with L and U. The FP32
                           form keeps the leading terms an FP32 evaluation resolves
                           (see skeleton_terms) and stores W = U^-1 L^-1 instead. Needs
                           precision FP64 or FP32, d <= 4 and ranks <= 1024; right-hand
                           sides are applied one at a time. The build still holds the
                           FP64 factors of every block while it runs. */
  int near_coords;      /* coordinates of the single-right-hand-side FP32 near-field
                           tiles (FP32/FP16/BF16 forms, d <= 3). 0 (default): each
                           box-relative coordinate as an FP32 pair hi + lo, so that a
                           distance keeps FP32 relative accuracy however close the two
                           points are. 1: hi only, about 40% fewer operations per pair;
                           a distance r then carries an absolute error of about
                           2^-24 h (h the leaf box size), a relative error 2^-24 h / r */
  int fp64_near;        /* near field of FP64 handles for one right-hand side at a
                           time, d <= 4. 0 (default): FP64 arithmetic. 1: float-float
                           arithmetic on the FP32 pipes (an unevaluated sum of two
                           FP32 numbers, about 48 significant bits; coordinates in
                           box units on a 2^-21 grid plus an FP32 remainder), about
                           10x the FP64 rate on a GPU whose FP64 rate is 1/64 of its
                           FP32 rate; kernel values carry a relative error of about
                           2^-44 (1e-13) instead of 2^-52. Not available for sin r
                           (HODLRDD_ERR_UNSUPPORTED). Ignored by other precisions. */
  int near_sms;         /* streaming multiprocessors given to the near field of the
                           single-right-hand-side FP32 tiles (FP32/FP16/BF16/FP32_FP16
                           forms, d <= 3), -1 or 0 .. SMs - 1. 0 (default): the near field
                           runs beside the low-rank applies on every SM. R > 0: the
                           persistent apply kernels run on SMs - R CTAs that reserve a
                           whole SM's shared memory each, and the near field runs as R
                           persistent CTAs of the same size (all its passes in one
                           launch, tasks taken from a counter), so that neither shares
                           an SM with the other. Products are the same in both
                           settings (each pass sums into a buffer of its own; the
                           buffers are added in pass order, the order in which the
                           shared setting accumulates them). -1: the build times
                           products with 0 and with R from about SMs / 8 to 9 SMs / 32
                           and keeps the fastest (hodlrdd_stats.near_sms). */
  int reserved[2];      /* set to 0 */
} hodlrdd_options;

#define HODLRDD_MAX_LEVELS 64

typedef struct hodlrdd_stats {
  int d;
  int kappa;                 /* number of tree levels below the root (leaf level) */
  int precision;
  int max_rank;              /* largest ACA rank over all low-rank blocks */
  int64_t N;
  int64_t n_blocks;          /* IL blocks over all levels */
  int64_t n_lowrank;         /* of which applied through factors */
  int64_t n_dense;           /* of which applied exactly */
  int64_t n_rank_capped;     /* of which hit aca_max_rank (applied exactly) */
  int64_t n_near;            /* leaf near-field blocks (self + d' >= 1 neighbours) */
  int64_t factor_elems;      /* sum over low-rank blocks of p (m + n) */
  int64_t factor_bytes;      /* bytes of packed factors (incl. padding and scales) */
  int64_t dense_pairs;       /* kernel evaluations per matvec and right-hand side */
  int64_t boxes_per_level[HODLRDD_MAX_LEVELS];
  int64_t blocks_per_level[HODLRDD_MAX_LEVELS];
  int max_rank_per_level[HODLRDD_MAX_LEVELS];
  double mean_rank_per_level[HODLRDD_MAX_LEVELS];
  double t_tree_ms;          /* bounding cube, Morton keys, sort, level tables */
  double t_classify_ms;      /* interaction and near lists */
  double t_aca_ms;           /* both ACA passes */
  double t_pack_ms;          /* factor packing / precision conversion, task lists */
  double t_build_ms;         /* whole build, wall clock */
  int64_t device_bytes;      /* device memory held by the handle */
  int64_t factor_bytes_u;    /* bytes of the U panels (per level and target box; FP32_FP16:
                                both element types) */
  int64_t factor_bytes_v;    /* bytes of the V panels (per level and source box) */
  int64_t total_rank;        /* sum of ranks: length of the t vector of the V-apply */
  int lowrank_form;          /* the build option (0 factors, 1 skeleton) */
  int64_t skeleton_bytes;    /* skeleton form: bytes of the LU factors, pivot lists and task
                                lists (factor_bytes then counts the LU factors and pivots) */
  int64_t skeleton_pairs;    /* skeleton form: kernel evaluations of its low-rank blocks per
                                product and right-hand side, sum of p' (|I| + |J|) */
  int64_t tail_cols;         /* FP32_FP16: factor columns stored in FP16 (of total_rank) */
  int64_t skeleton_terms;    /* skeleton form: sum of the kept ranks p'. FP64 keeps every ACA
                                term (p' = p); FP32 keeps the leading terms whose pivot is at
                                least 2^-23 of the largest pivot before it */
  int near_sms;              /* the option near_sms in use (-1 resolved by the build) */
} hodlrdd_stats;

/* Fills *opt with the defaults described above. */
int hodlrdd_options_default(hodlrdd_options* opt);

/*
 * Builds the HODLRdD representation of K on the current CUDA device
 * (Algorithm 1: form the 2^d tree, then compress every IL block with ACA).
 *
 *  points         host or device, N x d FP64, row-major (point i at points[i*d]),
 *                 original order; finite values only (else HODLRDD_ERR_INVALID).
 *  d              1..8.      N  >= 1, < 2^31.
 *  kernel_id      enum hodlrdd_kernel.
 *  kernel_params  host array of 4 doubles {scale, diag, p0, p1} or NULL for
 *                 {1, 0, 0, 0}: K(i,j) = scale * F(x_i, x_j; p0, p1) + diag * [i == j].
 *                 MATERN32, GAUSS, EXP need p0 > 0.
 *  leaf_size      N_max of the paper: the tree is refined until every leaf holds at
 *                 most leaf_size points (Algorithm 1's level rule); >= 1.
 *  tol            ACA tolerance (relative, Frobenius estimate), > 0.
 *  opt            NULL for defaults.
 *  out            receives the handle.
 *
 * The points are copied into library-owned memory: the caller may free them on
 * return. The call is synchronous (returns after all device work completes) and
 * thread-safe for distinct handles. The handle owns all its device memory until
 * hodlrdd_destroy.
 */
int hodlrdd_build(const double* points, int d, int64_t N, int kernel_id, const double* kernel_params,
                  int leaf_size, double tol, hodlrdd_handle* out);
int hodlrdd_build_ex(const double* points, int d, int64_t N, int kernel_id, const double* kernel_params,
                     int leaf_size, double tol, const hodlrdd_options* opt, hodlrdd_handle* out);

/*
 * y = K x (Algorithm 2): per-level low-rank applies, leaf near field evaluated on
 * the fly, all in the handle's precision.
 *
 *  x, y    host or device, N x nrhs row-major (column c of point i at [i*nrhs + c]),
 *          ORIGINAL point order; double for FP64 handles, float otherwise. y is
 *          overwritten, never accumulated. x and y must not overlap.
 *  nrhs    >= 1.
 *  stream  cudaStream_t (as void*); NULL = legacy default stream.
 *
 * With device x and y the call is asynchronous on `stream`: it only enqueues
 * kernels and allocates nothing. With host x or y it stages through buffers the
 * handle owns and returns after y is written (synchronous), also when it fails.
 * A handle's workspace is shared: concurrent matvecs on one handle from
 * different streams must be serialised by the caller. The device current when
 * the call is made must be the one the handle was built on (else
 * HODLRDD_ERR_INVALID).
 */
int hodlrdd_matvec(hodlrdd_handle h, const void* x, void* y, int nrhs, void* stream);

/*
 * y = K x exactly as hodlrdd_matvec computes it (same kernels, same result), for
 * callers that must not allocate device memory: a serving loop whose device
 * memory another allocator reserved up front, or a loop that cannot take the
 * synchronisation a cudaMalloc/cudaFree may bring. The paper has no counterpart;
 * it is a library addition.
 *
 * Host x or y pass through one fixed scratch array in the library's static device
 * memory (16 MiB per device) instead of buffers the handle grows: this call runs
 * no cudaMalloc, cudaFree or allocating library. The staged bytes,
 * round_up(N*nrhs*esize, 256) for a host x plus N*nrhs*esize for a host y (esize
 * 8 for FP64 handles, else 4), must be <= 16 MiB, else HODLRDD_ERR_INVALID with
 * the sizes in hodlrdd_last_error() and nothing enqueued. Nothing in the scratch
 * has to start at zero. Device x and y need no scratch.
 *
 * The first call on a device does set-up (it looks up the scratch's device
 * address, which also loads this part of the library's device code): make it
 * before any stream capture. Profiling must be off (HODLRDD_ERR_INVALID
 * otherwise). Arguments, layout and synchronisation as hodlrdd_matvec. All calls
 * on one device share the one scratch: two calls in flight at the same time on
 * the same device (from several threads, or one thread's asynchronous work on
 * other streams) race on it and must be serialised by the caller. As for
 * hodlrdd_matvec, the current device must be the handle's, and a call with a
 * host buffer returns only after its copies have finished, also when it fails.
 */
int hodlrdd_matvec_noalloc(hodlrdd_handle h, const void* x, void* y, int nrhs, void* stream);

/*
 * y = K x by direct summation over all N^2 pairs, K(i,j) = scale * F(x_i, x_j) +
 * diag * [i == j] (the kernel matrix of Section "Preliminaries"; the product
 * HODLRdD approximates), evaluated on the fly in FP32: a comparator for the
 * hierarchical product, not part of Algorithm 2.
 *
 *  x, y    device, N floats each, ORIGINAL point order; y is overwritten. They
 *          must not overlap. One right-hand side.
 *  h       a handle of precision FP32, FP16 or BF16 with d <= 3, else
 *          HODLRDD_ERR_UNSUPPORTED; host pointers give HODLRDD_ERR_INVALID.
 *
 * Asynchronous on `stream`; uses the handle's matvec workspace (serialise with
 * matvecs on other streams). The first call allocates 32 N bytes of
 * cube-relative coordinates, kept until hodlrdd_destroy.
 */
int hodlrdd_direct(hodlrdd_handle h, const void* x, void* y, void* stream);

/*
 * Solves K x = b, K the handles' kernel matrix, by restarted GMRES on a fast
 * operator inside iterative refinement with the FP64 operator: the use of the
 * hierarchical product for the second-kind integral equation (I + K/N) u = b
 * (diag = 1, scale = 1/N) of the paper's numerical experiments. Each
 * refinement step solves A d = r with GMRES(restart) on `inner` (classical
 * Gram-Schmidt applied twice, FP64 dot products) to a relative reduction of
 * inner_tol, then x += d and r = b - K x with the FP64 matvec of `outer`. x0 = 0;
 * stops when ||b - K x||_2 <= tol ||b||_2 for the FP64 operator.
 *
 *  inner   any-precision handle (FP32 / FP16 / BF16 for speed, FP64 works).
 *  outer   FP64 handle of the same points and kernel (may be `inner` itself).
 *  b, x    device, N doubles each, ORIGINAL point order; x is overwritten;
 *          they must not overlap.
 *  opt     NULL for the defaults (hodlrdd_solve_options_default).
 *  stats   optional.
 *
 * Synchronous. The Krylov basis (N x (restart + 1) values) and the other
 * scratch are allocated on the first solve with `inner` (or when a later solve
 * needs more) and kept in that handle until it is destroyed, so repeated solves
 * allocate nothing; one solve at a time per inner handle.
 * HODLRDD_ERR_NUMERIC when tol is not reached within max_refine steps (x holds
 * the last iterate). HODLRDD_ERR_TIMEOUT when a bounded device-side wait of a
 * product on either handle expired since that handle's error word was last
 * read (x is then invalid); the solve reads and clears both words.
 */
typedef struct hodlrdd_solve_options {
  double tol;           /* relative residual of the FP64 operator (default 1e-10) */
  double inner_tol;     /* residual reduction per inner GMRES solve (default 1e-5) */
  int restart;          /* GMRES restart length (default 50) */
  int max_inner_iters;  /* fast matvecs per refinement step (default 500) */
  int max_refine;       /* refinement steps (default 20) */
  int reserved[5];      /* set to 0 */
} hodlrdd_solve_options;

typedef struct hodlrdd_solve_stats {
  int refinements;       /* FP64 residual evaluations after an inner solve */
  int inner_iterations;  /* fast-operator matvecs in GMRES */
  double residual;       /* final ||b - K x|| / ||b|| with the FP64 operator */
} hodlrdd_solve_stats;

int hodlrdd_solve_options_default(hodlrdd_solve_options* opt);
int hodlrdd_solve(hodlrdd_handle inner, hodlrdd_handle outer, const double* b, double* x,
                  const hodlrdd_solve_options* opt, hodlrdd_solve_stats* stats, void* stream);

/*
 * Batched products over many resident handles (uneven trees, one request per
 * handle): the library's addition for serving many instances at once. The
 * requests are captured once into a CUDA graph, spread over up to 8 streams
 * inside it so small trees run side by side, and every hodlrdd_batch_run replays
 * it with one graph launch.
 *
 * hodlrdd_batch_create
 *  handles  count distinct handles (a handle may appear once); none profiling.
 *  nrhs     right-hand sides of each request (>= 1).
 *  Applies every request once (set-up), then captures; allocates the batch's
 *  own input and output buffers (N_i x nrhs_i each). The handles must outlive
 *  the batch and must not run other work while a batch run is in flight.
 * hodlrdd_batch_run
 *  x[i], y[i]  host or device, N_i x nrhs_i row-major, ORIGINAL point order, in
 *              the element type of handle i. Copies in, one graph launch,
 *              copies out, all on `stream`; synchronous when any pointer is on
 *              the host. Results equal those of hodlrdd_matvec on each handle
 *              (bitwise).
 */
typedef struct hodlrdd_batch_s* hodlrdd_batch;
int hodlrdd_batch_create(const hodlrdd_handle* handles, const int* nrhs, int count, hodlrdd_batch* out);
int hodlrdd_batch_run(hodlrdd_batch b, const void* const* x, void* const* y, void* stream);
int hodlrdd_batch_destroy(hodlrdd_batch b);

/*
 * A forest: products over many trees of the tensor-core form (FP16X2) merged
 * into one launch per stage. The paper's kernel-SVM experiment (numerical
 * experiments, "HODLRdD accelerated classical kernel SVM") trains on several
 * data sets of uneven size, each iteration one product K v per kernel matrix;
 * a forest serves such a set of independent products with the launches of one
 * tree: one gather, one V-apply and one U-apply over the
 * panels of all trees (the persistent CTAs balanced over the whole forest),
 * one near-field launch per pass (pass k holds the k-th near-field range of
 * every tree) and one final sum.
 *
 * hodlrdd_forest_create
 *  handles  count distinct handles, all of precision HODLRDD_PREC_FP16X2 with a
 *           bounded kernel (not 1/r or 1/r^2), the same d (<= 4), kernel and
 *           shape parameters (scale and diagonal may differ), on the current
 *           device, none profiling. They must outlive the forest; the forest
 *           copies their factor planes, panels and near-field tables, so a
 *           later hodlrdd_import_factors on a handle does not reach it.
 *  nrhs     right-hand sides of each tree's request, 1..64.
 *  Errors: HODLRDD_ERR_INVALID (NULL, count < 1, a repeated handle, nrhs out of
 *  range, profiling on), HODLRDD_ERR_UNSUPPORTED (another precision or kernel,
 *  trees that differ in d or kernel, sizes beyond 32-bit panel indices),
 *  HODLRDD_ERR_OOM, HODLRDD_ERR_CUDA.
 * hodlrdd_forest_run
 *  x[i], y[i]  host or device FP32, N_i x nrhs_i row-major, ORIGINAL point
 *              order. Runs on the forest's own streams after the work already
 *              queued on `stream`, and returns when y is written (synchronous).
 *              Each y[i] equals hodlrdd_matvec on handle i up to the order of
 *              FP32 additions (the same arithmetic on the same data).
 *  HODLRDD_ERR_TIMEOUT when a bounded device-side wait expired (y invalid).
 * hodlrdd_forest_stats
 *  out[7] = total points, bytes of the factor planes (both stages), apply
 *  panels, near-field passes, kernel launches per run (one CUDA graph launch
 *  replays them), and the fixed cost per panel (bytes' worth) that the
 *  autotuner picked for the V-apply's and the U-apply's panel schedule.
 * Creation also tunes: each apply stage's persistent-CTA panel ranges are
 *  rebuilt for a few fixed costs per panel, timed, and the fastest kept; then
 *  one run's launches are captured into a CUDA graph that every run replays.
 */
typedef struct hodlrdd_forest_s* hodlrdd_forest;
int hodlrdd_forest_create(const hodlrdd_handle* handles, const int* nrhs, int count, hodlrdd_forest* out);
int hodlrdd_forest_run(hodlrdd_forest f, const void* const* x, void* const* y, void* stream);
int hodlrdd_forest_stats(hodlrdd_forest f, int64_t* out);
/* Stage times of one extra run of the forest on the inputs of its last run
 * (CUDA events; synchronous): ms[5] = gather, V-apply, U-apply with the sums of
 * cut panels, near field (second stream), whole run. */
int hodlrdd_forest_profile(hodlrdd_forest f, double* ms);
int hodlrdd_forest_destroy(hodlrdd_forest f);

/*
 * Waits for all device work (cudaDeviceSynchronize) and reports failures the
 * handle's matvec kernels recorded on the device: HODLRDD_ERR_TIMEOUT when one of
 * their bounded waits expired (the y of that matvec is then invalid). Clears the
 * recorded failure. Failure detection for callers that keep matvecs asynchronous.
 */
int hodlrdd_sync(hodlrdd_handle h);

/* Frees the handle and all device memory it holds. NULL is accepted. */
int hodlrdd_destroy(hodlrdd_handle h);

/* Sizes, ranks and phase timings of the build (the paper reports maximum rank,
 * memory of the representation and initialisation time). */
int hodlrdd_get_stats(hodlrdd_handle h, hodlrdd_stats* s);

/* Static description of a status code. */
const char* hodlrdd_error_string(int status);
/* Detail of the last failure on the calling thread (never NULL). */
const char* hodlrdd_last_error(void);

/*
 * Stage timing of subsequent matvecs (tracing). With on = 1 every matvec records
 * CUDA events on its own stream between its stages; on = 0 stops recording.
 * Enabling resets the accumulated values.
 */
int hodlrdd_set_profiling(hodlrdd_handle h, int on);

/*
 * Accumulated stage times since profiling was enabled (synchronises with the
 * recorded events): ms[4] = gather, V-apply, U-apply, near field + combine;
 * *chunks = number of right-hand-side chunks timed; *launches = kernels the
 * handle's matvecs have launched since the build (counted whether or not
 * profiling is on). Any pointer may be NULL.
 */
int hodlrdd_get_profile(hodlrdd_handle h, double* ms, int64_t* chunks, int64_t* launches);

/* ---------------------------------------------------------------------------
 * Introspection: copies of the integer structure, for bit-exact checks.
 * All output arrays are host memory sized by the caller from hodlrdd_get_stats
 * and hodlrdd_get_level.
 * ------------------------------------------------------------------------- */

/* perm[i] = original index of the point at tree position i; keys[i] = its Morton
 * key (B = min(32, floor(63/d)) bits per dimension, dimension k at bit k of each
 * d-bit level digit, coarse level first). Either pointer may be NULL. */
int hodlrdd_get_tree(hodlrdd_handle h, int64_t* perm, uint64_t* keys);

/* Bounding cube: lo[d], side_inv[0] = side, side_inv[1] = 2^B / side. */
int hodlrdd_get_cube(hodlrdd_handle h, double* lo, double* side_inv);

/* Level l (0..kappa): *nboxes non-empty boxes; bstart[nboxes+1] tree-order point
 * offsets; bkey[nboxes] box keys (the top l digits of the Morton key). Either
 * array may be NULL (query *nboxes first). */
int hodlrdd_get_level(hodlrdd_handle h, int l, int64_t* nboxes, int64_t* bstart, uint64_t* bkey);

/* Interaction lists of level l (1..kappa): CSR off[nboxes+1], idx[off[nboxes]]
 * (source box indices, ascending per target box). *nnz receives off[nboxes];
 * off / idx may be NULL. */
int hodlrdd_get_il(hodlrdd_handle h, int l, int64_t* nnz, int64_t* off, int64_t* idx);

/* Leaf near lists (self and boxes sharing a d' >= 1 hyper-surface), same CSR form. */
int hodlrdd_get_near(hodlrdd_handle h, int64_t* nnz, int64_t* off, int64_t* idx);

/* Per IL block, in CSR order (levels ascending, then target, then source), 9
 * int64: level, target box, source box, I0, m, J0, n, rank, dense. */
int hodlrdd_get_blocks(hodlrdd_handle h, int64_t* rec);

/* ACA pivots (block-local row / column indices, in pivot order) of block b;
 * arrays of length >= rank. */
int hodlrdd_get_pivots(hodlrdd_handle h, int64_t b, int64_t* sigma, int64_t* tau);

/* FP64 copy of block b's factors as applied (after the precision conversion and
 * scales): U m x rank, V n x rank, column-major. HODLRDD_ERR_UNSUPPORTED for a
 * handle in the skeleton form (it keeps no factors). */
int hodlrdd_get_factors(hodlrdd_handle h, int64_t b, double* U, double* V);

/*
 * Replaces every IL block's factors with caller-supplied ones (host arrays, FP64):
 * rank[b] and dense[b] per block in CSR order; U_all / V_all hold, block after
 * block, U_b (m x rank, column-major) and V_b (n x rank). The factors are then
 * packed in the handle's precision exactly as after hodlrdd_build. Used to check
 * the matvec against a reference representation independently of the ACA.
 * HODLRDD_ERR_UNSUPPORTED for a handle in the skeleton form (imported factors
 * carry no pivots).
 */
int hodlrdd_import_factors(hodlrdd_handle h, const int32_t* rank, const int32_t* dense, const double* U_all,
                           const double* V_all);

/*
 * Test entry for the bounded device-side waits: runs, on the handle's stream,
 * one wait on an mbarrier phase that nothing completes, bounded by `cycles`
 * SM clock cycles (at most 8e9, about 4 s); it then records an error code in the
 * handle's error word exactly as an expired wait in a matvec kernel does, and
 * returns. The next hodlrdd_sync reports HODLRDD_ERR_TIMEOUT and clears the
 * word; the handle stays usable. Synchronous.
 */
int hodlrdd_debug_expire_wait(hodlrdd_handle h, long long cycles);

/*
 * Test entry for the failure paths of device allocations: the k-th following
 * device allocation of the library (k >= 0, counted process-wide) fails as if
 * the device were out of memory, once; k < 0 turns the injection off.
 * Optional scratch (the ACA's one-pass pool) is not counted. Always HODLRDD_OK.
 */
int hodlrdd_debug_fail_alloc_after(int64_t k);

/*
 * Test entry: caps the device pool in which the ACA keeps each block's factors
 * during its one pass (bytes; -1 restores the default, half of the free device
 * memory beyond 2 GB, at most 128 GB; 0 disables it). Blocks that do not fit are
 * recomputed by a second pass with the same arithmetic, so the factors do not
 * depend on the cap. Process-wide; always HODLRDD_OK.
 */
int hodlrdd_debug_aca_pool_bytes(int64_t bytes);

/*
 * Measurement aid (the paper has no counterpart): throughput of the arithmetic
 * pipes the on-the-fly kernel evaluation and the FP64 form are bound by, on the
 * current device, each timed with CUDA events on `stream` (best of three
 * launches that fill every SM with independent dependency chains). Changes no
 * device setting: the numbers are those of the clocks the GPU runs at.
 *
 *  out[0]  FP32 FMA throughput, TFLOP/s (2 flops per FMA)
 *  out[1]  FP64 FMA throughput, TFLOP/s
 *  out[2]  MUFU rsqrt.approx.f32, G operations/s
 *  out[3]  MUFU ex2.approx.f32, G operations/s
 *  n       entries of out to fill (<= 4 used). Synchronous; allocates 16 bytes.
 */
int hodlrdd_probe_peaks(double* out, int n, void* stream);

/*
 * Test entry of the float-float kernel evaluation that the FP64 near field uses
 * with fp64_near = 1: out[i] = F(s[i]) for the kernel (kernel_id, params as in
 * hodlrdd_build) and squared distances s[i] >= 0, evaluated as the near field
 * does at box size h (s / h^2 in box units, the box size folded into the
 * per-level constants). Host arrays of n values; synchronous. Errors:
 * HODLRDD_ERR_INVALID (NULL, n < 0, h <= 0), HODLRDD_ERR_UNSUPPORTED (sin r or
 * an unknown kernel).
 */
int hodlrdd_debug_ff_eval(int kernel_id, const double* params, double h, const double* s, double* out, int64_t n);

/*
 * Serving: a request loop over models kept resident under a device-memory
 * budget (the library's addition for many instances of uneven size arriving
 * over time, such as the paper's batched uses).
 *
 * hodlrdd_server_create
 *  budget_bytes  device bytes the resident handles may hold (hodlrdd_stats
 *                device_bytes, summed); during a build the new handle may
 *                briefly exceed it.
 *  workers       host threads (1..64) on the current device, each with a
 *                high-priority CUDA stream for products and a low-priority one
 *                for solves. Queued products start before queued solves (they are
 *                short), and at most workers - 1 solves run at once (with more
 *                than one worker) so that one worker stays free for products;
 *                each kind starts in arrival order. Products of different models
 *                run side by side; requests for one model run one at a time,
 *                except that products of one model queued while another of its
 *                products waits are batched: a worker that starts a product takes
 *                the model's other queued products along (up to 64 columns, see
 *                hodlrdd_server_set_batching) and runs them as one product over
 *                their columns side by side (FP32-I/O precisions with stored
 *                factors; FP64 models and the skeleton form run products alone).
 * hodlrdd_server_add
 *  Registers a model (host copy of the points; same arguments as
 *  hodlrdd_build_ex, opt may be NULL). It is built on its first request and
 *  stays resident until the budget needs its memory: then the least recently
 *  used idle models are destroyed, and rebuilt when asked for again.
 *  *model_id receives 0, 1, 2, ... in registration order.
 * hodlrdd_server_submit
 *  kind = HODLRDD_REQ_MATVEC: y = K x, x and y as for hodlrdd_matvec (host or
 *  device, element type of the model's precision).
 *  kind = HODLRDD_REQ_SOLVE: K u = b column by column through hodlrdd_solve
 *  with the model as the fast operator and an FP64 twin of it (built on the
 *  first solve, counted in the budget) as the refinement operator; x = b and
 *  y = u are HOST arrays of N x nrhs doubles, original point order. The twin
 *  evaluates its near field in float-float (fp64_near = 1) where that exists
 *  (d <= 4, every kernel but sin r): about 1e-13 per kernel value, far below the
 *  refinement's tolerance, at about 10x the FP64 rate.
 *  Buffers must stay valid until the request is waited for. Asynchronous;
 *  *request_id identifies the request.
 * hodlrdd_server_wait
 *  Blocks until the request has finished and returns its status (the worker's
 *  error detail is copied to the calling thread's hodlrdd_last_error); a request
 *  is waited for once. latency_ms (optional, two doubles) receives the
 *  submit-to-done and the start-to-done (service) times in milliseconds.
 * hodlrdd_server_stats
 *  out[0] resident device bytes, out[1] resident models, out[2] builds so far,
 *  out[3] evictions so far, out[4] queued requests not yet started.
 * hodlrdd_server_destroy
 *  Finishes queued requests, stops the workers, destroys every handle.
 * hodlrdd_server_set_batching
 *  max_cols >= 0: columns of one batched product (default 64); 0 or 1 turns
 *  batching off.
 * hodlrdd_server_batch_stats
 *  out[0] batched products run so far (batches of two or more requests),
 *  out[1] requests served by them.
 * Results equal those of hodlrdd_matvec / hodlrdd_solve on the model's handle
 * alone: bitwise for a product that runs alone; a batched product's columns go
 * through the handle's chunks of several right-hand sides (uncompensated FP32
 * accumulation, tensor-core chunks for FP16X2), which stay within those forms'
 * stated bounds of the single-column product.
 */
enum { HODLRDD_REQ_MATVEC = 0, HODLRDD_REQ_SOLVE = 1 };
typedef struct hodlrdd_server_s* hodlrdd_server;
int hodlrdd_server_create(int64_t budget_bytes, int workers, hodlrdd_server* out);
int hodlrdd_server_add(hodlrdd_server s, const double* points, int d, int64_t N, int kernel_id,
                       const double* kernel_params, int leaf_size, double tol, const hodlrdd_options* opt,
                       int64_t* model_id);
int hodlrdd_server_submit(hodlrdd_server s, int64_t model_id, int kind, const void* x, void* y, int nrhs,
                          int64_t* request_id);
int hodlrdd_server_wait(hodlrdd_server s, int64_t request_id, double* latency_ms);
int hodlrdd_server_stats(hodlrdd_server s, int64_t* out);
int hodlrdd_server_set_batching(hodlrdd_server s, int max_cols);
int hodlrdd_server_batch_stats(hodlrdd_server s, int64_t* out);
int hodlrdd_server_destroy(hodlrdd_server s);

#ifdef __cplusplus
}
#endif

#endif /* HODLRDD_H */
