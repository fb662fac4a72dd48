/*
 * mht.h -- C ABI of the butterfly-accelerated manifold harmonic transform (BF-MHT).
 *
 * The transform (Sec. 1, Eq. MHT-sum): given n points x_j on a manifold and the first m
 * Laplace-Beltrami eigenfunctions phi_k, Phi is the n x m matrix Phi_jk = phi_k(x_j), and
 *     synthesis   f = Phi c                    (mht_synthesize)
 *     analysis    c = Phi^H diag(w) f          (mht_analyze; the fast adjoint of Sec. 1,
 *                                               Phi^H the conjugate transpose, w >= 0)
 * are applied through a row-wise butterfly factorization of Phi (Sec. 2, Algorithm 1;
 * streaming post-order build of Sec. 4, Algorithm 3) with a Fiedler space tree (Sec. 3,
 * Algorithm 2) and an eigenvalue-ordered frequency tree.  The factorization is built in
 * FP64 on the host; the apply runs as CUDA kernels on the caller's stream.
 *
 * Conventions for every entry point:
 *  - Return value: MHT_OK or an error code; on error mht_last_error() returns a message
 *    (thread-local, valid until the next call on the same thread).  No exception crosses
 *    the ABI.  A failed apply leaves its outputs unspecified.
 *  - Element types.  A plan has a field (real/complex) and an apply mode:
 *      MHT_APPLY_FP64  -> vectors are double (real) or interleaved (re, im) double pairs;
 *      MHT_APPLY_FP32 / MHT_APPLY_3XTF32 / MHT_APPLY_6XBF16 -> float or interleaved float pairs.
 *  - Vector layout: column-major.  c is m x nrhs with leading dimension ldc >= m (counted
 *    in elements, one complex value = one element); f is n x nrhs with ldf >= n.  Rows are
 *    in the caller's ORIGINAL point / mode order (the order the problem was given in).
 *  - Device memory is owned by the caller.  The library never allocates device memory:
 *    the caller queries sizes (mht_plan_device_bytes), allocates, and binds the buffers
 *    (mht_plan_bind_device).  Host memory of a plan is owned by the plan.
 *  - Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Device applies are asynchronous; input and output buffers must not alias and must stay
 *    valid until the stream reaches the end of the call.  Two applies on one plan must not
 *    run concurrently (they share the plan's bound workspace).
 */
#ifndef MHT_H
#define MHT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mht_plan mht_plan;
typedef struct mht_batch mht_batch;

typedef enum {
  MHT_OK = 0,
  MHT_ERR_INVALID_ARG = 1, /* a NULL, size, stride or enum argument is out of range   */
  MHT_ERR_OOM = 2,         /* host allocation failed, or a caller buffer is too small */
  MHT_ERR_CALLBACK = 3,    /* the user's Phi evaluator returned non-zero              */
  MHT_ERR_NUMERIC = 4,     /* NaN/Inf met while building the factorization            */
  MHT_ERR_CUDA = 5,        /* a CUDA runtime call failed (message has the CUDA error) */
  MHT_ERR_FORMAT = 6,      /* plan file or imported factors are malformed             */
  MHT_ERR_TIMEOUT = 7,     /* a bounded device wait ran out (persistent batched apply)*/
  MHT_ERR_UNSUPPORTED = 8, /* valid request this build does not implement             */
  MHT_ERR_NOT_BOUND = 9    /* apply called before mht_plan_bind_device                */
} mht_status;

typedef enum { MHT_REAL = 0, MHT_COMPLEX = 1 } mht_field;

typedef enum {
  MHT_APPLY_FP64 = 0,  /* factors and vectors in double, FP64 arithmetic                */
  MHT_APPLY_FP32 = 1,  /* factors and vectors in float, FP32 SIMT arithmetic            */
  MHT_APPLY_3XTF32 = 2, /* float data; multi-RHS block products on the tensor cores with
                           each operand split into two TF32 parts (22 of FP32's 24 bits) and
                           three products (hi*hi + hi*lo + lo*hi), FP32 accumulation;
                           single-RHS applies use the FP32 kernels                     */
  MHT_APPLY_6XBF16 = 3  /* float data; multi-RHS block products on the tensor cores with
                           each operand split exactly into three BF16 parts and the six
                           products down to order 2^-16 (x0y0 + x0y1 + x1y0 + x0y2 + x1y1 +
                           x2y0), FP32 accumulation: FP32 accuracy; single-RHS applies use
                           the FP32 kernels                                             */
} mht_apply_mode;

typedef enum {
  MHT_TREE_AUTO = 0,        /* RECT for MHT_EVAL_TORUS, FIEDLER_MESH when problem->tris
                               is given, FIEDLER otherwise                            */
  MHT_TREE_FIEDLER = 1,     /* Algorithm 2, mesh-free rule: sign of phi_2 of a kNN
                               heat-kernel graph Laplacian on each node's points      */
  MHT_TREE_RECT = 2,        /* flat periodic square: exact Neumann Fiedler function of
                               each node's rectangle (midpoint cut of the longer side;
                               sin(x1) at the periodic root)                          */
  MHT_TREE_PCA_MEDIAN = 3,  /* median split along the principal axis (equal sizes)     */
  MHT_TREE_GIVEN = 4,       /* problem->space_perm / space_offsets are used as is      */
  MHT_TREE_FIEDLER_MESH = 5 /* Algorithm 2, patch rule (Sec. 3, Eq. neumann-eigenproblem):
                               the points are the vertices of the triangle mesh
                               problem->tris; each node holds a set of triangles (the
                               patches P) and of points; phi_2 = second eigenfunction of
                               K phi = lambda M phi on the node's sub-mesh (P1 cotangent
                               stiffness K, lumped mass M: the homogeneous Neumann
                               condition is the natural one); M_1 = {P : integral of
                               phi_2 over P <= 0} (exact for P1: area / 3 x the sum of
                               the vertex values); a point goes to M_1's side when it is
                               a vertex of a triangle of M_1 (the closed patch set),
                               else to M_2's                                           */
} mht_tree_kind;

typedef enum {
  MHT_ID_AUTO = 0,      /* BLOCKED for large problems (n m >= 2^28), else CLASSICAL          */
  MHT_ID_CLASSICAL = 1, /* Householder QR with column pivoting, one column at a time        */
  MHT_ID_BLOCKED = 2    /* QR with randomized block pivoting (Gaussian sketch of b + 8 rows
                           picks 64 pivots at a time; compact-WY panel updates) for blocks with
                           min(M, K) >= 128, and a Gram-matrix pivoted-Cholesky certificate
                           that skips the QR of very tall full-rank blocks (M >= 16 K);
                           real and complex Phi                                              */
} mht_id_method;

typedef enum {
  MHT_EVAL_CALLBACK = 0, /* problem->eval(ctx, rows, nrows, cols, ncols, out)           */
  MHT_EVAL_TORUS = 1,    /* Phi_jk = exp(i k_k . x_j), Eq. 2D-DFT; points (n x 2),
                            problem->torus_modes (m x 2 int64); field must be COMPLEX   */
  MHT_EVAL_SPHERE = 2,   /* orthonormal real spherical harmonics, column k = l^2+l+mm,
                            cos(mm lon) for mm > 0, sin(|mm| lon) for mm < 0, no
                            Condon-Shortley phase; points (n x 3); field must be REAL    */
  MHT_EVAL_DENSE = 3     /* problem->dense: column-major n x m FP64 (interleaved pairs if
                            complex) with leading dimension ld_dense >= n               */
} mht_eval_kind;

/* Entries of Phi in FP64 for original indices rows[0..nrows) x cols[0..ncols), written
 * column-major to out[nrows * ncols] (interleaved (re, im) pairs if complex).  Called
 * concurrently from several host threads.  Return 0 on success, non-zero to abort the
 * build with MHT_ERR_CALLBACK. */
typedef int (*mht_eval_fn)(void* ctx, const int64_t* rows, int64_t nrows,
                           const int64_t* cols, int64_t ncols, double* out);

typedef struct {
  int64_t n, m;                 /* points (rows of Phi) and modes (columns)            */
  mht_field field;
  const double* eigenvalues;    /* [m] defines the frequency order (stable sort)       */
  mht_eval_kind eval_kind;
  mht_eval_fn eval;             /* MHT_EVAL_CALLBACK                                   */
  void* eval_ctx;
  const double* points;         /* [n * dim] row-major; trees and built-in evaluators  */
  int32_t dim;
  const int64_t* torus_modes;   /* [m * 2] for MHT_EVAL_TORUS                          */
  const double* dense;          /* MHT_EVAL_DENSE                                      */
  int64_t ld_dense;
  const int64_t* space_perm;    /* MHT_TREE_GIVEN: [n] tree order -> original point    */
  const int64_t* space_offsets; /* MHT_TREE_GIVEN: [2^L + 1] leaf ranges, depth L      */
  const double* weights;        /* [n] quadrature / mass weights w for analysis; NULL = 1 */
  const int64_t* tris;          /* [ntris * 3] vertex indices (into points, dim 3) of a
                                   triangle mesh for MHT_TREE_FIEDLER_MESH; or NULL      */
  int64_t ntris;
} mht_problem;

typedef struct {
  double eps;          /* ID tolerance: rank = #{k : |R_kk| > eps |R_11|}              */
  int64_t leaf_size;   /* L = max(0, ceil(log2(n / leaf_size))) unless levels >= 0      */
  int32_t levels;      /* < 0: derive L from leaf_size                                */
  mht_apply_mode mode;
  mht_tree_kind tree;
  uint64_t seed;       /* row sampling and Lanczos start vectors                       */
  int32_t num_threads; /* host threads for the build; 0 = OpenMP default               */
  double oversample;   /* row-sampled IDs use min(|tau|, ceil(oversample * K) + 16) rows, a
                          heuristic that costs accuracy at tight eps; <= 0 disables
                          sampling (exact IDs on all rows, the recommended setting)     */
  mht_id_method id_method; /* pivoting strategy of the IDs                                */
} mht_options;

/* Factors as plain arrays: the content of a factorization, in the notation of Sec. 2.
 * Blocks at level l (0..L) are numbered b = tau * 2^(L-l) + nu (tau at depth l of the
 * space tree, nu at height l of the frequency tree).  Block b has rank r = ranks[l*2^L+b]
 * and input size K (level 0: |nu|; level l >= 1: ranks of blocks (p, 2nu) and (p, 2nu+1)
 * at level l-1 added, p = tau / 2).  local_perm lists K local input indices with the r
 * skeleton indices first; transfer holds T~ (r x (K-r), row-major), so that the block's
 * interpolation matrix is [I | T~] P^T.  column_bases holds U_tau = Phi(tau, J_tau) for each
 * space leaf tau (|tau| x r_L row-major, rows in tree order).  All arrays are concatenated
 * level by level, block by block.  Complex values are interleaved (re, im) pairs. */
typedef struct {
  int64_t n, m;
  int32_t levels;
  mht_field field;
  int64_t* space_perm;     /* [n] tree-order position -> original point index          */
  int64_t* space_offsets;  /* [2^L + 1]                                                */
  int64_t* mode_perm;      /* [m] frequency-order position -> original mode index      */
  int64_t* mode_offsets;   /* [2^L + 1]                                                */
  int32_t* ranks;          /* [(L + 1) * 2^L]                                          */
  int32_t* local_perm;     /* [sum of K over all blocks]                               */
  double* transfer;        /* [sum of r (K - r)] (x2 if complex)                       */
  double* column_bases;    /* [sum of |tau| r_L] (x2 if complex)                       */
  double* weights;         /* [n] or NULL: read by import; written by export when the
                              plan has analysis weights (left as is otherwise)        */
} mht_factors;

typedef struct {
  int64_t n, m;
  int32_t levels;
  mht_field field;
  mht_apply_mode mode;
  double eps;
  int64_t blocks_per_level;     /* 2^L                                                  */
  int64_t local_perm_entries;   /* sizes of the mht_factors arrays                      */
  int64_t transfer_entries;     /* complex entries count once                           */
  int64_t column_basis_entries;
  int64_t stored_entries;       /* transfer + column-basis entries (the applied data)   */
  int64_t max_rank;
  int64_t workspace_entries_per_rhs;
  size_t factor_bytes;          /* device bytes of the packed factors                   */
  size_t algorithmic_bytes;     /* bytes one single-RHS apply must move: stored entries,
                                   index lists, descriptors, c and f (see the design notes) */
  double build_seconds;
} mht_plan_info_t;

typedef struct {
  int64_t rank_min, rank_median, rank_max, rank_sum;
  int64_t transfer_entries;     /* T~ entries at this level (level L+1: column bases)   */
  size_t bytes;                 /* packed device bytes of this stage's factors          */
  size_t algorithmic_bytes;     /* bytes one single-RHS launch of this stage must move:
                                   stored matrix entries, index lists, descriptors, the
                                   input entries it gathers and the outputs it writes   */
} mht_level_info_t;

/* ---- build, import, export -------------------------------------------------------- */

/* Builds the butterfly factorization of Phi (Algorithms 1-3) in FP64 on the host and packs
 * it for the device.  *out receives a new plan owned by the caller (free with
 * mht_destroy).  Errors: INVALID_ARG (sizes, enums, missing evaluator data), CALLBACK,
 * NUMERIC, OOM. */
mht_status mht_build_plan(const mht_problem* problem, const mht_options* options,
                          mht_plan** out);

/* Entries Phi(rows, cols) of the problem's evaluator -- the values mht_build_plan factors
 * (Sec. 1, Eq. MHT-sum: Phi_jk = phi_k(x_j)) -- in FP64, column-major out[nrows * ncols],
 * interleaved (re, im) when problem->field is MHT_COMPLEX.  rows are original point indices
 * in [0, n), cols original mode indices in [0, m); out is caller-owned host memory.  Only the
 * evaluator fields of the problem are read (eigenvalues and weights are not needed).
 * Errors: INVALID_ARG (NULL pointers, negative counts, indices out of range, missing
 * evaluator data), CALLBACK. */
mht_status mht_problem_eval(const mht_problem* problem, const int64_t* rows, int64_t nrows,
                            const int64_t* cols, int64_t ncols, double* out);

/* Creates a plan from explicit factors (layout above); the arrays are copied and may be
 * freed after the call.  options->mode selects the apply precision; other option fields
 * are ignored.  Errors: INVALID_ARG, FORMAT (inconsistent ranks, permutations, offsets). */
mht_status mht_plan_import(const mht_factors* factors, const mht_options* options,
                           mht_plan** out);

/* Creates an independent plan with the same factors as `src`, packed for options->mode (for
 * example an FP64 plan beside an FP32 one, to measure the FP32 rounding error of an apply).
 * The copy is unbound.  Errors: INVALID_ARG. */
mht_status mht_plan_clone(const mht_plan* src, const mht_options* options, mht_plan** out);

/* Copies the plan's FP64 factors into caller arrays sized from mht_plan_info (scalar
 * fields of *factors are filled in; array pointers may be NULL to skip an array). */
mht_status mht_plan_export(const mht_plan* plan, mht_factors* factors);

mht_status mht_plan_info(const mht_plan* plan, mht_plan_info_t* info);

/* level in 0..L for transfer levels, L+1 for the column bases U. */
mht_status mht_plan_level_info(const mht_plan* plan, int32_t level, mht_level_info_t* info);

/* ---- device binding ------------------------------------------------------------------ */

/* Device bytes the caller must provide: the packed factors (fixed) and a workspace that
 * serves applies with up to max_nrhs right-hand sides (intermediate butterfly vectors and
 * host-transfer staging).  Both buffers need 256-byte alignment. */
mht_status mht_plan_device_bytes(const mht_plan* plan, int64_t max_nrhs,
                                 size_t* factor_bytes, size_t* workspace_bytes);

/* Uploads the packed factors into factor_dev (cudaMemcpyAsync on `stream`, complete when
 * the call returns) and records both buffers in the plan.  The buffers stay owned by the
 * caller and must outlive the plan's use.  Re-binding replaces the previous binding.
 * Errors: INVALID_ARG (NULL, misaligned, too small), CUDA. */
mht_status mht_plan_bind_device(mht_plan* plan, void* factor_dev, size_t factor_bytes,
                                void* workspace_dev, size_t workspace_bytes,
                                int64_t max_nrhs, void* stream);

/* ---- applies ------------------------------------------------------------------------- */

/* f = Phi c (synthesis, Eq. MHT-sum): leaf stage V, transfer levels l = 1..L, column
 * bases U, each a CUDA kernel launch on `stream`.  c_dev: m x nrhs, f_dev: n x nrhs device
 * arrays in the plan's element type.  1 <= nrhs <= the bound max_nrhs. */
mht_status mht_synthesize(mht_plan* plan, const void* c_dev, int64_t ldc, void* f_dev,
                          int64_t ldf, int64_t nrhs, void* stream);

/* f = Phi diag(s) c: synthesis of diagonally scaled coefficients, the scale s (device, m real
 * entries in the plan's precision, caller's mode order) applied inside the leaf stage's gather
 * (no extra pass).  With s = sqrt(S(lambda_k)) and c = white noise this samples a Gaussian
 * random field of spectral density S (Sec. 7.2); with s = F(lambda_k) it applies a spectral
 * filter to given coefficients.  Same layout rules as mht_synthesize. */
mht_status mht_synthesize_scaled(mht_plan* plan, const void* c_dev, int64_t ldc, const void* scale_dev,
                                 void* f_dev, int64_t ldf, int64_t nrhs, void* stream);

/* f_out = Phi diag(F) Phi^H W f_in (weighted != 0; Phi^H f_in otherwise): spectral filtering of
 * point values (Sec. 7.1), or the covariance product Phi S Phi^H of Sec. 7.2.  Analysis, the diagonal
 * (fused into synthesis' leaf stage) and synthesis run as one CUDA graph, captured on the first
 * call with these arguments and replayed by later calls with the same ones (pointers, leading
 * dimensions, RHS count, weighting, apply mode and autotuning state).  F: device, m real entries
 * in the plan's precision, caller's mode order.  The coefficients pass through the workspace's
 * host-staging area, so a filter call must not overlap a host-buffer transform on the plan.
 * f_in and f_out: n x nrhs, must not alias.  Errors as mht_synthesize. */
mht_status mht_filter(mht_plan* plan, const void* f_in_dev, int64_t ldi, void* f_out_dev, int64_t ldo,
                      int64_t nrhs, const void* filter_dev, int32_t weighted, void* stream);

/* Inverse transform (Sec. 7.1, Eq. inverse-MHT): c = argmin_c ||Phi c - f||_2 for each of the
 * nrhs columns, by LSQR (Paige & Saunders 1982) on the butterfly apply: one synthesis and one
 * analysis per iteration, FP64 scalar recurrences on the host.  A column stops when its
 * residual estimate falls below tol * ||f|| or its normal-equation residual estimate
 * ||Phi^H r|| below tol * ||Phi|| ||r||, or after max_iter iterations.  scratch_dev: caller
 * device memory of mht_lsqr_scratch_bytes, 256-byte aligned.  Synchronizes `stream` every
 * iteration.  *iters (optional): iterations run; *relres (optional): the largest final
 * ||r|| / ||f|| estimate over the columns.  Layout and errors as mht_analyze. */
mht_status mht_lsqr_scratch_bytes(const mht_plan* plan, int64_t nrhs, size_t* bytes);
mht_status mht_inverse_lsqr(mht_plan* plan, const void* f_dev, int64_t ldf, void* c_dev, int64_t ldc,
                            int64_t nrhs, void* scratch_dev, size_t scratch_bytes, int32_t max_iter,
                            double tol, void* stream, int32_t* iters, double* relres);

/* f = diag(w) Phi c: synthesis followed by the analysis weights (the adjoint of weighted
 * analysis, used for its gradient).  Same layout rules as mht_synthesize. */
mht_status mht_synthesize_weighted(mht_plan* plan, const void* c_dev, int64_t ldc, void* f_dev,
                                   int64_t ldf, int64_t nrhs, void* stream);

/* c = Phi^H diag(w) f if weighted (w from the problem or factors; all ones if none was
 * given), else c = Phi^H f: the transposed sweep U^H, R^H for l = L..1, V^H (leaves last),
 * gather form without atomics.  Same layout rules as mht_synthesize. */
mht_status mht_analyze(mht_plan* plan, const void* f_dev, int64_t ldf, void* c_dev,
                       int64_t ldc, int64_t nrhs, int32_t weighted, void* stream);

/* The same transforms on HOST arrays: the input is copied to device staging inside the
 * bound workspace, the transform runs, and the result is copied back; the call returns
 * after the stream has finished.  Host arrays should be pinned for full copy speed. */
mht_status mht_synthesize_host(mht_plan* plan, const void* c_host, int64_t ldc, void* f_host,
                               int64_t ldf, int64_t nrhs, void* stream);
mht_status mht_analyze_host(mht_plan* plan, const void* f_host, int64_t ldf, void* c_host,
                            int64_t ldc, int64_t nrhs, int32_t weighted, void* stream);

/* Number of kernel launches one mht_synthesize / mht_analyze call makes for nrhs. */
mht_status mht_apply_launch_count(const mht_plan* plan, int64_t nrhs, int64_t* launches);

/* Synthesis f = Phi c of one vector for callers that cannot allocate device memory: code
 * that runs where cudaMalloc is not allowed (for instance inside a framework that owns the
 * device memory, or a region that must not allocate).  The paper has no counterpart; this
 * is a deployment variant of the persistent synthesis for real FP32 plans.  Its scratch
 * (a status word, the per-level butterfly vectors, per-block completion counters and the
 * work-queue head) lives in a fixed array of MHT_NOALLOC_SCRATCH_BYTES inside this library,
 * which every GPU that loads the library reserves until the process exits; a plan that needs
 * more is rejected with MHT_ERR_UNSUPPORTED and a message that gives both sizes, and FP64 or
 * complex plans with MHT_ERR_UNSUPPORTED.  Nothing is allocated: the caller passes factor_dev
 * (the plan's packed factors on the device, 256-byte aligned -- for instance the buffer given
 * to mht_plan_bind_device), c_dev (m floats) and f_dev (n floats).  The first call on a device
 * looks up the array's address on that device; make that call before any stream capture.  All
 * calls share the one array, which keeps the previous call's contents (the call clears the
 * counters and the queue head, which must start at zero): calls that overlap on the GPU -- on
 * different streams or from different threads -- race and give wrong results, so serialize
 * them.  The kernel's waits are bounded (2 s); a wait that gives up sets a bit of the array's
 * status word (the bits of mht_plan_check), stops the launch and leaves f unspecified.  The
 * word is sticky -- later calls abort at once while it is set -- until mht_noalloc_check
 * reads and clears it.  Asynchronous on `stream`. */
#define MHT_NOALLOC_SCRATCH_BYTES (16u << 20)
mht_status mht_synthesize_noalloc(const mht_plan* plan, const void* factor_dev, const void* c_dev,
                                  void* f_dev, void* stream);

/* Reads and clears the status word of mht_synthesize_noalloc's scratch array on the current
 * device (synchronizes `stream`; allocates nothing).  Returns MHT_OK with *flags = 0 when every
 * bounded wait of the no-alloc calls since the last check completed, else MHT_ERR_TIMEOUT with
 * the bits (those of mht_plan_check) in *flags. */
mht_status mht_noalloc_check(void* stream, int32_t* flags);

/* Testing aid for the failure path of mht_synthesize_noalloc: hold != 0 raises the completion
 * target of one leaf-stage block in the caller's factor image factor_dev to a count that is
 * never reached, so that the next no-alloc call gives up its bounded dependency wait (2 s),
 * stops every CTA and reports bit 8 through mht_noalloc_check, leaving the context usable;
 * hold == 0 restores the value from the plan.  Synchronous on `stream`. */
mht_status mht_noalloc_debug_hold(const mht_plan* plan, void* factor_dev, int32_t hold, void* stream);

/* Testing aid for the out-of-memory path: while `bytes` is non-zero, packing a plan image larger
 * than `bytes` (build, import, load, clone) fails as a host allocation failure does, with
 * MHT_ERR_OOM and no plan created.  0 removes the limit.  Process-wide. */
mht_status mht_debug_host_alloc_limit(size_t bytes);

/* Reads and clears the device status word of the bound workspace (synchronizes `stream`).
 * Every device wait of the apply kernels is bounded (2 s); one that gives up sets a bit and
 * the outputs of that apply are unspecified.  ANY nonzero value means that; the bits say
 * which wait gave up:
 *   1  per-stage kernel: a bulk copy of factor rows did not arrive;
 *   2  persistent all-stage kernel: a free copy slot or item-queue slot did not come;
 *   4  persistent all-stage kernel: a chunk of factor rows or the staged input did not arrive;
 *   8  persistent all-stage kernel: a dependency (completion counter of the previous stage);
 *   16 persistent all-stage kernel: the next work item or a free input buffer did not come;
 *   32 tensor-core kernel: completion of the block products (tensor-core MMAs).
 * While the word is nonzero, the persistent kernels abort at once.  Returns MHT_OK with
 * *flags = 0 when every wait since the last check completed, MHT_ERR_TIMEOUT (and the flags)
 * otherwise. */
mht_status mht_plan_check(mht_plan* plan, void* stream, int32_t* flags);

/* Apply path: 0 = automatic (currently one launch per stage, the faster path on the
 * measured workloads), 1 = one launch per stage, 2 = one persistent launch per direction that
 * runs every stage (up to 8 RHS; MHT_ERR_UNSUPPORTED if it does not fit).  Both paths compute
 * the same result. */
mht_status mht_plan_set_path(mht_plan* plan, int32_t path);

/* Switches the arithmetic of later applies between MHT_APPLY_FP32, MHT_APPLY_3XTF32 and
 * MHT_APPLY_6XBF16 on a plan whose factors are stored in float (all read the same packed image,
 * so no rebinding is needed).  MHT_ERR_INVALID_ARG for an FP64 plan or for MHT_APPLY_FP64, whose
 * storage precision differs.  The block products of the apply (Sec. 2) with a block of
 * vectors take the tensor-core path only in the two split modes and from 16 real (8 complex)
 * RHS on: one persistent launch per stage, tiles of 128 rows x up to 64 accumulator columns
 * fed by 2-D TMA tensor maps; complex products run as real products of twice the width. */
mht_status mht_plan_set_mode(mht_plan* plan, mht_apply_mode mode);

/* Autotuner: times the candidate launch configurations of every stage of both directions
 * for `nrhs` right-hand sides (SIMT RHS tile 1/2/4/8, bulk-copy ring of 1-8 slots of 16/32/64
 * KB, resident CTAs per SM, and in the split tensor-core modes the tensor-core kernel) on the
 * bound workspace, keeps the fastest per stage, and then (up to 8 RHS, automatic path) times
 * groupings of the small stages at both ends of each direction into one persistent launch; later applies with exactly `nrhs` RHS use them (others use the
 * defaults).  Runs the stages on zeroed workspace buffers only (the caller's vectors are not
 * touched) and synchronizes `stream`; takes about a second on a 15 GB plan.  Results equal
 * the untuned apply's within rounding (RHS tile and kernel change the summation order).
 * Errors: INVALID_ARG (nrhs < 1 or > the bound max_nrhs), NOT_BOUND, CUDA. */
mht_status mht_plan_autotune(mht_plan* plan, int64_t nrhs, void* stream);
/* The tuned configuration of one stage (direction 0 synthesis / 1 analysis; stage 0..L+1):
 * cfg[5] = {tensor cores (0/1), RHS tile, ring slots, CTAs per SM, slot KB} (0 = the default)
 * and its measured milliseconds.  stage = -1: the direction's stage grouping, cfg[1] = how many
 * stages at its start and cfg[2] = how many at its end run as one persistent launch each (with
 * per-block dependency counters; 0 = none), and the direction's measured milliseconds.  The
 * autotuner keeps a grouping only when it is at least 2% faster than one launch per stage.
 * INVALID_ARG if the plan has not been tuned. */
mht_status mht_plan_tune_info(const mht_plan* plan, int32_t direction, int32_t stage, int32_t* cfg, double* ms);

/* Stage timing for benchmarks.  While enabled, every apply on the plan records a CUDA
 * event before and after each kernel launch (on the apply's stream).
 * mht_plan_stage_times waits for the recorded events, returns the summed milliseconds and
 * launch counts (arrays of L+3 entries: ID levels 0..L and the column bases for per-stage
 * launches, then entry L+2 for persistent launches that run all stages) for direction 0
 * (synthesis) or 1 (analysis), and clears the record.  Enabling costs one event record per
 * launch; disabled (the default) it costs nothing. */
mht_status mht_plan_profile(mht_plan* plan, int32_t enable);
mht_status mht_plan_stage_times(mht_plan* plan, int32_t direction, double* ms, int64_t* launches);

/* ---- batched ragged apply ---------------------------------------------------------------
 * Many FP32 plans (instances of different n, m, depth L, real or complex) and their RHS
 * counts applied together: every stage of every instance runs in ONE persistent kernel
 * launch per direction, replayed from a CUDA graph (a counter reset and the kernel).  Work
 * items of all instances share one queue in dependency order (the phases of Sec. 2's apply:
 * V, then R for l = 1..L, then U, per instance; the adjoint in reverse), so small instances
 * and the tails of large stages overlap instead of each paying a launch and a drain.
 * Results equal the per-plan mht_synthesize / mht_analyze (same kernels' arithmetic).
 *
 * Lifecycle: mht_batch_create (host only; the plans must stay alive until
 * mht_batch_bind_device returns) -> mht_batch_device_bytes -> mht_batch_bind_device
 * (uploads the packed factors into caller memory, synchronous) -> mht_batch_set_io (fixes
 * the caller's device vectors: c_i column-major m_i x nrhs_i with leading dimension ldc[i],
 * f_i n_i x nrhs_i with ldf[i]; complex instances use interleaved float pairs) ->
 * mht_batch_synthesize / mht_batch_analyze (asynchronous on `stream`) -> mht_batch_destroy.
 * Calls on one batch must not overlap on the GPU (they share the workspace).
 * Errors: INVALID_ARG (NULL, count <= 0, FP64 plan, bad RHS count or leading dimension),
 * NOT_BOUND, UNSUPPORTED (a block too wide for shared memory), CUDA. */
mht_status mht_batch_create(mht_plan* const* plans, int32_t count, const int64_t* nrhs, mht_batch** out);
mht_status mht_batch_device_bytes(const mht_batch* batch, size_t* image_bytes, size_t* workspace_bytes);
mht_status mht_batch_bind_device(mht_batch* batch, void* image_dev, size_t image_bytes, void* workspace_dev,
                                 size_t workspace_bytes, void* stream);
mht_status mht_batch_set_io(mht_batch* batch, void* const* c_dev, const int64_t* ldc, void* const* f_dev,
                            const int64_t* ldf, void* stream);
/* f_i = Phi_i c_i for every instance. */
mht_status mht_batch_synthesize(mht_batch* batch, void* stream);
/* c_i = Phi_i^H W_i f_i (weighted != 0) or Phi_i^H f_i for every instance. */
mht_status mht_batch_analyze(mht_batch* batch, int32_t weighted, void* stream);
/* MHT_APPLY_FP32 (default): the persistent FP32 kernel above.  MHT_APPLY_3XTF32 or
 * MHT_APPLY_6XBF16: every instance runs its own per-stage apply (tcgen05 split block products
 * from 16 real / 8 complex RHS on, FP32 kernels below that) on eight forked streams, all
 * captured once into one CUDA graph and replayed; results equal mht_synthesize / mht_analyze of
 * each plan in that mode. */
mht_status mht_batch_set_mode(mht_batch* batch, mht_apply_mode mode);
/* 1 (default): launches replay CUDA graphs; 0: plain stream launches (same work). */
mht_status mht_batch_set_graph(mht_batch* batch, int32_t use_graph);
/* Work items per direction and CTAs of one persistent launch (needs a current device). */
mht_status mht_batch_info(const mht_batch* batch, int64_t* items_synthesis, int64_t* items_analysis,
                          int32_t* grid);
/* Reads and clears the batch's device status word (synchronizes `stream`); TIMEOUT if a
 * bounded wait gave up (bit 0: a bulk copy, bit 1: a dependency). */
mht_status mht_batch_check(mht_batch* batch, void* stream, int32_t* flags);
/* Autotuner of the batched launch: times one synthesis + analysis for every (ring slots,
 * resident CTAs per SM) pair that fits and keeps the fastest for later launches (the CUDA
 * graphs are rebuilt).  Overwrites the batch's f and c vectors; synchronizes `stream`;
 * *best_ms (optional) receives the time of the chosen pair for both directions. */
mht_status mht_batch_autotune(mht_batch* batch, void* stream, double* best_ms);
/* Testing aid for the failure path of the batched FP32 kernel: makes the dependency of one
 * phase (1..L+1) of one instance impossible to satisfy on the device, so that the next launch
 * of that direction gives up its bounded wait (2 s), stops every CTA through the abort word and
 * reports MHT_ERR_TIMEOUT (flag 2) through mht_batch_check, leaving the context usable.
 * mht_batch_set_io restores the records.  Synchronous on `stream`. */
mht_status mht_batch_debug_hold(mht_batch* batch, int32_t direction, int32_t instance, int32_t phase,
                                void* stream);
mht_status mht_batch_destroy(mht_batch* batch);

/* ---- persistence and lifetime -------------------------------------------------------- */

/* Versioned binary plan file with an FNV-1a 64-bit checksum over the payload; the plan
 * file is the checkpoint of an expensive build.  Load errors: FORMAT, OOM, INVALID_ARG. */
mht_status mht_plan_save(const mht_plan* plan, const char* path);
mht_status mht_plan_load(const char* path, const mht_options* options, mht_plan** out);

/* Frees the plan's host memory (device buffers stay with the caller).  NULL is a no-op. */
mht_status mht_destroy(mht_plan* plan);

const char* mht_last_error(void);
const char* mht_version(void);

#ifdef __cplusplus
}
#endif
#endif /* MHT_H */
