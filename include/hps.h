/*
 * hps.h -- C ABI of the GB300 (sm_103a) library for the batched leaf-box
 * reduction of the two-level HPS solver (Kump, Yesypenko, Martinsson,
 * "A Two-Level Direct Solver for the Hierarchical Poincare-Steklov Method",
 * arXiv:2503.04033).
 *
 * The PDE (Eq. 1, Eq. 2):  -Lap u - kappa^2 b(x) u = f in the box, u = g on
 * its boundary.  Each leaf box carries a p x p x p tensor grid of
 * Chebyshev-Lobatto nodes (Sec. 2.1).  Edge and corner nodes are dropped
 * (Remark 1), which leaves
 *     n = (p-2)^3 interior nodes and m = 6 (p-2)^2 face nodes per box.
 * The library computes, for every box in a batch, the blocks of the paper's
 * static condensation (Sec. 2.2, Eq. 5 to Eq. 8):
 *     S = -A_ii^{-1} A_ib        solution operator   (n x m)
 *     T = A_bb + A_bi S          DtN map             (m x m)
 *     v = A_ii^{-1} f_i,  h = A_bi v                 particular solution, flux
 *     u_i = v + S u_b                                interior reconstruction
 *
 * Layouts (all row-major, boxes outermost, double precision, device memory
 * unless stated):
 *   grid node (i,j,k), 0 <= i,j,k < p            index i + p j + p^2 k
 *   interior node (i,j,k), 1 <= i,j,k <= p-2      index (i-1) + q (j-1) + q^2 (k-1), q = p-2
 *   face f in the order x-, x+, y-, y+, z-, z+   face node (a,b) (a the lower free axis,
 *                                                 1 <= a,b <= q) has index f q^2 + (a-1) + q (b-1)
 *   b  [nbox][p^3]    f  [nbox][nrhs][p^3]    S  [nbox][n][m]    T  [nbox][m][m]
 *   v  [nbox][nrhs][n]   h  [nbox][nrhs][m]   u_b [nbox][nrhs][m]   u_i [nbox][nrhs][n]
 * Face rows of T and h take the OUTWARD normal derivative of each box (the
 * flux-continuity rows of Eq. 4 sum the two boxes' outward derivatives).
 *
 * "Device memory" means any address the GPU can dereference: an output such
 * as T may also be pinned (page-locked, mapped) host memory, which the
 * kernels then write across the host link (T is written once, by the D_n
 * products at the end of the call), so no separate download is needed.
 * Inputs are read several times and belong in device memory proper.
 *
 * Ownership: the caller owns every input and output buffer.  The context owns
 * its workspace (device memory it allocates on first use, up to the limit given
 * to hps_create) and small per-(p, h) operator tables.
 *
 * Asynchrony: the leaf calls enqueue work on `stream` (a cudaStream_t passed as
 * void*, NULL = legacy default stream) and return once it is enqueued.  The
 * return value covers argument, allocation and launch errors.  Per-box numerical
 * outcome is written to box_status[nbox] (device int array, may be NULL) and is
 * valid after the stream has been synchronised:
 *   0              the box succeeded
 *   HPS_ESINGULAR  an exactly zero pivot appeared in the LU of A_ii
 *   HPS_ENOCONV    mixed precision: the FP64 refinement did not reach its tolerance
 *   HPS_EINVAL     a non-finite value of b (or f, u_b) was seen in the box
 * No C++ exception crosses this interface.  A context may be used by one host
 * thread at a time; calls on the same context serialise on its workspace.
 */
#ifndef HPS_H
#define HPS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hps_ctx hps_ctx;

typedef enum {
    HPS_OK = 0,
    HPS_EINVAL = 1,      /* bad argument (size, pointer, non-finite parameter) */
    HPS_ENOMEM = 2,      /* workspace limit too small for one box, or allocation failed */
    HPS_ESINGULAR = 3,   /* per box: zero pivot in the LU of A_ii */
    HPS_ENOCONV = 4,     /* per box: FP64 refinement did not converge */
    HPS_ECUDA = 5,       /* a CUDA runtime call failed */
    HPS_ETIMEOUT = 6     /* reserved: a bounded device wait gave up */
} hps_status;

/* Arithmetic of the LU and the triangular solves.  HPS_FP64 runs everything
 * in FP64 (the plain path).  HPS_FP32_IR factors A_ii in FP32 on the tensor
 * cores (3-term TF32 split products with FP32 accumulation) and recovers FP64
 * accuracy by iterative refinement: residuals R = -A_ib - A_ii X computed
 * matrix-free in FP64, corrections solved with the FP32 factors, X updated in
 * FP64; the D_n product forming T is FP64.  HPS_BF16_IR is the same
 * refinement with the tensor-core products taken in BF16 with FP32
 * accumulation: each operand is split into three BF16 pieces (successive
 * roundings of the remainder) and six kind::f16 products per K step keep every
 * term above FP32 rounding, so the factors are as accurate as FP32's.  Without
 * tensor cores (HPS_OPT_TENSOR_CORES = 0) it runs as HPS_FP32_IR. */
typedef enum { HPS_FP64 = 0, HPS_FP32_IR = 1, HPS_BF16_IR = 2 } hps_precision;

/* One class of boxes: polynomial order p (3 <= p <= 24), box side lengths
 * h[0..2] (> 0), wavenumber kappa (finite).  All boxes of a call share it.
 * beta: NULL for the operator of Eq. 2, -Lap u - kappa^2 b u; or device
 * [nbox][3][p^3] (per box, like b: the x, y and z components at every node)
 * for -Lap u + div(beta u) - kappa^2 b u, the first-order term of the
 * convection-diffusion example of Sec. 4.4 (collocated by the product rule
 * along each grid line).  Read by the leaf calls, hps_leaf_factor (which
 * keeps a copy) and hps_leaf_apply; hps_dtn_gate and the no-allocation entry
 * point take NULL only.  With beta the first refinement residual is FP64
 * too. */
typedef struct {
    int p;
    double h[3];
    double kappa;
    const double* beta;
} hps_leaf_kind;

/* Tunables for hps_set_option (value is a double). */
typedef enum {
    HPS_OPT_IR_MAX_ITERS = 1,   /* corrections in FP32_IR mode, default 8, range 0..20 */
    HPS_OPT_IR_TOL = 2,         /* a box stops refining when its predicted remaining error is below tol
                                   relative to ||X||_F (default 1e-11, a decade below the 1e-10 relative
                                   accuracy the FP32_IR path is meant to deliver on T and u, so that an
                                   interface solve built on the leaf maps keeps its own accuracy):
                                   ||dX_k|| min(1, 10 ||dX_k||/||dX_k-1||) from the second
                                   correction on (the first ends the refinement only when it is itself
                                   below tol), or when ||dX|| is below 1e-11 ||X|| and shrank by less
                                   than half (the residual's noise floor); converged boxes skip later
                                   steps */
    HPS_OPT_BLOCK = 3,          /* LU block size NB: 0 = automatic, else 32, 64 or 128 */
    HPS_OPT_TENSOR_CORES = 4,   /* FP32 products on tcgen05 (1, default) or CUDA cores (0) */
    HPS_OPT_SYNC = 5,           /* 1: synchronise the stream and return the first box failure */
    HPS_OPT_AUTOTUNE = 6,       /* 1: time the LU block candidates on each new (p, precision, tensor-core)
                                   combination (on up to 8 of the call's boxes, synchronising the stream) and
                                   keep the fastest; the choices persist in the file named by the
                                   environment variable HPS_TUNE_CACHE, when set */
    HPS_OPT_GRAPHS = 7,         /* 1: capture each distinct leaf call (same sizes, buffers and options) into a
                                   CUDA graph on first use and replay the graph afterwards */
    HPS_OPT_TC_EPILOGUE = 8,    /* tcgen05 update epilogue: 0 (default) moves source and result tiles by TMA
                                   wherever the output is 16-byte aligned, 1 always uses the cp.async form */
    /* option 9 is not used */
    HPS_OPT_LU_UNIT = 10,       /* 4 (default), 8, 2 or 1: on the tensor-core path, up to this many consecutive
                                   LU steps are joined into one unit (look-ahead on the later panels of the
                                   unit, one update of unit-width K over every later column and one product
                                   per unit in the solves); 1: one step at a time.  Results agree to
                                   rounding */
    HPS_OPT_TC_FUSE = 11,       /* gathers of the backward solves written by the previous product's TMA
                                   epilogue: -1 (default) where that measured faster (3 x TF32 operands),
                                   0 never, 1 always; results are bit-identical either way */
    HPS_OPT_RESIDUAL_DF = 12,   /* precision of the refinement residuals B - A_ii X in FP32_IR and BF16_IR
                                   mode.  3 (default): the first residual, of the low-precision solution
                                   X0 itself (exact in FP32), in double-float arithmetic on the FP32 pipes
                                   (about 2^-46 relative to the sum of the terms' magnitudes); the later
                                   ones in double-float as well (each FP64 entry of X split into two
                                   floats) for boxes whose first correction was at most 3e-4 of X, whose
                                   A_ii then amplifies residual errors little enough for that floor to
                                   stay a factor 5 under 1e-10, and in FP64 for every other box.
                                   2: double-float first residual, every later one in FP64.
                                   1: double-float first residual whose correction never ends the
                                   refinement, later ones in FP64.  0: every residual in FP64 */
    HPS_OPT_FP16_OPERANDS = 13, /* 1 (default): FP32_IR tensor-core products split each operand into two FP16
                                   values (hi + lo, 22 bits as with 3 x TF32) under exact power-of-two scales
                                   of the left operand's K columns and the right operand's columns, which
                                   halves the operand bytes and doubles the MMA rate; 0: 3 x TF32 */
    HPS_OPT_GROUPS_CONCURRENT = 14, /* 1 (default): the groups of one hps_leaf_groups call run concurrently, each
                                   on its own stream and workspace slice, when the whole batch's workspace
                                   fits at once (else one after another, chunked); 0: one after another */
    HPS_OPT_TEST_SINGULAR_BOX = 100, /* test hook: zero row 0 of A_ii of this box index (-1 = off),
                                        which makes that box exactly singular (host-side fault injection) */
    HPS_OPT_TEST_TC_TIMEOUT = 101    /* test hook: 1 arms it once.  In the next FP32_IR / BF16_IR call on the
                                        tensor cores, one update product issues no operand loads, so its first
                                        bounded mbarrier wait runs out (after 2 ms instead of 2 s); the
                                        launch drains what it has in flight, frees its tensor memory and
                                        returns, and every box of the call reports HPS_ETIMEOUT.  No GPU
                                        fault is involved and the context stays usable.  Calls with the hook
                                        armed bypass the CUDA-graph cache */
} hps_option;

/* Creates a context on CUDA device `device`.  workspace_bytes_max bounds the
 * device workspace the context may allocate (0 = 85% of the memory free at
 * the first leaf call).  Batches larger than the workspace holds are processed
 * in chunks.  *ctx is NULL on failure. */
hps_status hps_create(hps_ctx** ctx, int device, size_t workspace_bytes_max);

/* Frees the context and its device memory.  Synchronises the device first. */
void hps_destroy(hps_ctx* ctx);

hps_status hps_set_option(hps_ctx* ctx, int option, double value);

/* n = (p-2)^3 and m = 6 (p-2)^2 (Remark 1); HPS_EINVAL unless 3 <= p <= 24. */
hps_status hps_leaf_sizes(int p, int* n, int* m);

/* Host helper: coordinates of the p^3 Chebyshev-Lobatto nodes of the box
 * [lo, lo + h] (Sec. 2.1), written to host array xyz[p^3][3] in grid order. */
hps_status hps_leaf_nodes(int p, const double lo[3], const double h[3], double* xyz);

/* Device workspace bytes one box needs for a DtN build at order p. */
size_t hps_workspace_per_box(int p, hps_precision prec);

/* Build stage, per box (Algorithm 1, the loop over boxes; Eq. 8):
 * forms A^tau from b, factors A_ii with partial pivoting, and writes
 *   T[nbox][m][m] = A_bb + A_bi S            (required)
 *   S[nbox][n][m] = -A_ii^{-1} A_ib          (optional: NULL = do not store S)
 * b[nbox][p^3] holds b at every grid node; only interior values enter.
 * nbox = 0 is a no-op.  HPS_EINVAL for nbox < 0, T == NULL with nbox > 0,
 * a bad kind or precision. */
hps_status hps_leaf_build_dtn(hps_ctx* ctx, const hps_leaf_kind* kind, int nbox,
                              const double* b, double* T, double* S,
                              hps_precision prec, int* box_status, void* stream);

/* Solve stage, first loop (Sec. 2.2 steps 1-2; Algorithm 2): re-forms and
 * re-factors A_ii (the paper recomputes rather than stores it) and writes
 *   v[nbox][nrhs][n] = A_ii^{-1} f_i,   h[nbox][nrhs][m] = A_bi v.
 * The caller's equivalent load on the faces is g_b = f_b - h (f_b = 0 on
 * interfaces).  1 <= nrhs <= 256. */
hps_status hps_leaf_particular(hps_ctx* ctx, const hps_leaf_kind* kind, int nbox, int nrhs,
                               const double* b, const double* f, double* v, double* h,
                               hps_precision prec, int* box_status, void* stream);

/* Solve stage, last loop (Sec. 2.2 step 4; Algorithm 2): u_i = v + S u_b.
 * If S is non-NULL ([nbox][n][m], e.g. from hps_leaf_build_dtn) it is applied
 * directly; if NULL, S u_b is recomputed as -A_ii^{-1} (A_ib u_b) from b
 * (the paper's recompute mode).  v may be NULL (treated as zero). */
hps_status hps_leaf_reconstruct(hps_ctx* ctx, const hps_leaf_kind* kind, int nbox, int nrhs,
                                const double* b, const double* S, const double* v,
                                const double* ub, double* ui,
                                hps_precision prec, int* box_status, void* stream);

/* One group of a mixed batch (Sec. 3.2: separate stacked arrays for each
 * order p when p varies from box to box): boxes of one order p and side h,
 * each with its own wavenumber.  T (and optionally S) request the DtN build;
 * nrhs > 0 requests particular solutions for nrhs body loads per box.  Both
 * come from ONE factorisation of each A_ii, whose right-hand side is
 * [-A_ib | f_i].  Layouts as for the single-kind calls. */
typedef struct {
    int p;
    double h[3];
    int nbox;
    const double* kappa;   /* host [nbox]: wavenumber of each box (finite) */
    const double* b;       /* device [nbox][p^3] */
    double* T;             /* device [nbox][m][m] or NULL (no DtN build) */
    double* S;             /* device [nbox][n][m] or NULL */
    int nrhs;              /* 0..256 loads per box */
    const double* f;       /* device [nbox][nrhs][p^3] */
    double* v;             /* device [nbox][nrhs][n] = A_ii^{-1} f_i */
    double* hflux;         /* device [nbox][nrhs][m] = A_bi v */
    int* box_status;       /* device [nbox] or NULL */
} hps_leaf_group;

/* Runs every group of a mixed batch on `stream` (groups in order, each in
 * chunks of its workspace), with CUDA-graph replay and block autotuning when
 * those options are on.  HPS_EINVAL for a bad group (order, sizes, pointers,
 * non-finite kappa) or a group with neither T nor loads. */
hps_status hps_leaf_groups(hps_ctx* ctx, int ngroups, const hps_leaf_group* groups, hps_precision prec,
                           void* stream);

/* ---- Learned low-rank DtN correction (beyond the paper, which always
 * computes T exactly).  A three-layer MLP maps the p^3 samples of b of a box
 * (input x = 2 (b - 1)) to factors U, V (m x rank); the predicted map is
 * T_hat = T0 + s U V^T with T0 the DtN map of the same box for b = 1.
 * Weights live in FP32 (master, Adam moments); every product runs on the
 * tensor cores (tcgen05) with BF16 operands -- weights, activations, deltas
 * and the scaled loss residual rounded to BF16 where they are made -- and
 * FP32 accumulation; all kernels are this library's own. */
typedef struct hps_mlp hps_mlp;

/* n_in -> n_h1 -> n_h2 -> 2 m rank, ReLU hidden layers, He-uniform weights
 * from a splitmix64 stream seeded by `seed`. */
hps_status hps_mlp_create(int device, int n_in, int n_h1, int n_h2, int m, int rank, unsigned long long seed,
                          hps_mlp** out);
void hps_mlp_destroy(hps_mlp* net);
size_t hps_mlp_num_params(const hps_mlp* net);

/* Copies all parameters (which = 0) or the last gradients (which = 1) as one
 * FP32 host array W0, c0, W1, c1, W2, c2 (W_l row-major [in][out]); to_device
 * = 1 loads parameters from the host instead (not allowed for gradients). */
hps_status hps_mlp_copy_params(hps_mlp* net, int which, float* host, int to_device);

/* U, V [B][m][rank] (device, FP64) from b_in [B][n_in] (device). */
hps_status hps_mlp_forward(hps_mlp* net, int B, const double* b_in, double* U, double* V, void* stream);

/* Gradients of L = mean over boxes and entries of (U V^T - (T - T0) / scale)^2
 * for a batch b_in [B][n_in], exact maps T [B][m][m] and the b = 1 map
 * T0 [m][m] (device); the loss is returned on the host when loss_out is
 * non-NULL (this synchronises).  Equivalent to hps_mlp_target into a buffer
 * the network owns, then hps_mlp_grad_target. */
hps_status hps_mlp_grad(hps_mlp* net, int B, const double* b_in, const double* T, const double* T0, double scale,
                        double* loss_out, void* stream);

/* Training targets D[b] = float((T[b] - T0) / scale) (device; T [nbox][m][m],
 * T0 [m][m] shared, D [nbox][m][m] FP32), formed once per training set so
 * that each step reads 4 bytes per entry instead of two FP64 maps. */
hps_status hps_mlp_target(int nbox, int m, const double* T, const double* T0, double scale, float* D, void* stream);

/* Gradients of L = mean over boxes and entries of (U V^T - D)^2 for a batch
 * b_in [B][n_in] and FP32 targets D [B][m][m] (device); loss as in
 * hps_mlp_grad. */
hps_status hps_mlp_grad_target(hps_mlp* net, int B, const double* b_in, const float* D, double* loss_out,
                               void* stream);

/* One Adam update with the last gradients. */
hps_status hps_mlp_adam_step(hps_mlp* net, float lr, float beta1, float beta2, float eps, void* stream);

/* T[b] = T0 + scale U[b] V[b]^T (device, FP64; T0 [m][m] shared). */
hps_status hps_lowrank_dtn(int nbox, int m, int rank, const double* T0, double scale, const double* U,
                           const double* V, double* T, void* stream);

/* Residual gate of predicted maps T_hat [nbox][m][m] (device) for boxes with
 * coefficients b [nbox][p^3]: for nprobe seeded Gaussian traces phi per box
 * (splitmix64 of seed and the element index, Box-Muller), T phi is computed as
 * A_bb phi + A_bi w with A_ii w = -A_ib phi solved by `iters` Richardson steps
 * preconditioned with the b = 1 block's inverse (FP64 LU, cached per
 * (p, h, kappa)); err[box] = ||T_hat phi - T phi|| / ||T phi|| and accept[box]
 * = 1 when err <= tol and the last Richardson step was below 1e-8 relative
 * (device arrays).  Boxes that fail go to the exact path. */
hps_status hps_dtn_gate(hps_ctx* ctx, const hps_leaf_kind* kind, int nbox, const double* b, const double* T_hat,
                        int nprobe, unsigned long long seed, int iters, double tol, int* accept, double* err,
                        void* stream);

/* Host helper for the interface system (Sec. 3.1: row and column index
 * arrays that align each T^tau with the global interface unknowns; Fig. 5).
 * Boxes form an nb[0] x nb[1] x nb[2] grid, box index bx + nx (by + ny bz).
 * Interface faces are numbered x-normal first ((ix-1) + (nx-1)(by + ny bz)),
 * then y-normal (Fx + bx + nx((iy-1) + (ny-1) bz)), then z-normal
 * (Fx + Fy + bx + nx(by + ny (iz-1))); boundary (Dirichlet) faces x-normal
 * (s + 2(by + ny bz)), then y (Dx + s + 2(bx + nx bz)), then z
 * (Dx + Dy + s + 2(bx + nx by)), s = 0 low side, 1 high side.  A face's q^2
 * nodes keep the box-local face order, so global id = face id * q^2 + local.
 * Outputs (host arrays, unsummed COO triplets in box order, row-major within a
 * box block): interface x interface entries of every T^tau in
 * rows/cols/vals, interface x Dirichlet entries in rows_d/cols_d/vals_d.
 * Duplicate (row, col) pairs are to be summed (two boxes share each face).
 * Call with NULL arrays to query nnz, nnz_d, n_iface and n_dir.
 * T_host is [nbox][m][m] on the host. */
hps_status hps_assemble_interface_blocks(int p, const int nb[3], const double* T_host,
                                         int64_t* nnz, int64_t* rows, int64_t* cols, double* vals,
                                         int64_t* nnz_d, int64_t* rows_d, int64_t* cols_d, double* vals_d,
                                         int64_t* n_iface, int64_t* n_dir);

/* Diagnostics of the last leaf call on this context: per box, the number of
 * refinement corrections applied and the final relative correction
 * ||dX||_F/||X||_F (0 for FP64).  Host arrays of length nbox (either may be
 * NULL); synchronises the context's last stream. */
hps_status hps_last_refinement(hps_ctx* ctx, int nbox, int* iters, double* rel_correction);

/* FP64 DtN build (the same result as hps_leaf_build_dtn with HPS_FP64 and
 * S = NULL) for callers that cannot allocate device memory: a host program
 * whose GPU memory is owned by another allocator (for example a framework's
 * caching allocator that has reserved the device), or a latency-critical loop
 * where cudaMalloc/cudaFree would stall on an implicit device synchronisation.
 * The paper has no counterpart; this is a deployment variant.
 * It allocates nothing.  All scratch (operator tables, status words, the LU
 * workspace) lives in one file-scope device array of 64 MiB that every GPU
 * loading this library holds until the process exits.  The caller passes
 * b[nbox][p^3], T[nbox][m][m] and optionally box_status[nbox] (device);
 * batches larger than the scratch holds run in chunks on `stream`.
 * Returns HPS_ENOMEM (nothing enqueued) when one box's workspace exceeds the
 * scratch: p <= 14 fits (p = 12 needs ~22 MiB per box, p = 13 ~37 MiB and
 * p = 14 ~60 MiB, one box per chunk), p >= 15 returns HPS_ENOMEM; with
 * box_status NULL the status words also come from the scratch (4 bytes/box).
 * The operator tables are built on the device by a small kernel (no host
 * copy); every call enqueues only kernels and memsets on `stream`.
 * The first call on a device looks up the array's device address (once per
 * device, with that device current); make that first call before any stream
 * capture.  Every call shares the one array and leaves its contents behind
 * (the call clears the status words it uses): calls that overlap on the GPU
 * (concurrent streams, several host threads) race on it and must be
 * serialised by the caller. */
hps_status hps_leaf_build_dtn_noalloc(const hps_leaf_kind* kind, int nbox, const double* b, double* T,
                                      int* box_status, void* stream);

/* ---- Stored factorisations (factor once, solve many) ----------------------
 *
 * The interior blocks of a batch of boxes factored once and kept on the
 * device, so that later loads reuse them: the build stage applied once and
 * every time step (or load batch) only solves, as the paper does for its
 * Crank-Nicolson time stepping, where the same operator serves every step
 * (Sec. 4.4).  hps_leaf_factor builds and factors A_ii of nbox boxes of one
 * kind (b as in hps_leaf_build_dtn; it is not read after the call returns,
 * kappa^2 b being kept) in the given precision, allocating device memory for
 * the factors and for solves of up to nrhs_max (1..256) right-hand sides, and
 * returns the handle in *out.  box_status (device [nbox], or NULL) receives
 * each box's factorisation status (HPS_ESINGULAR for a singular A_ii).
 * Returns HPS_ENOMEM when the factors do not fit.  The handle belongs to ctx
 * (destroy it before the context) and its calls are serialised with ctx's.
 *
 * hps_leaf_solve_factored: v = A_ii^{-1} f_i and h = A_bi v for nrhs <=
 * nrhs_max loads, layouts as in hps_leaf_particular (Sec. 2.2 steps 1-2,
 * Algorithm 2).  hps_leaf_reconstruct_factored: u_i = v + S u_b with S
 * applied by solves, layouts as in hps_leaf_reconstruct (Sec. 2.2 step 4).
 * Both refine to FP64 accuracy on the mixed paths as the one-shot calls do,
 * write each box's status to box_status (device [nbox], or NULL; a box whose
 * factorisation failed keeps that status) and return HPS_EINVAL for nrhs out
 * of range or NULL arrays.  Several solves may follow one factorisation; they
 * share the handle's workspace, so solves on different streams must be
 * ordered by the caller.  With HPS_OPT_GRAPHS each distinct solve (same
 * arrays, nrhs and refinement options) is captured into a CUDA graph once
 * and replayed afterwards, as the time steps of a loop are. */
typedef struct hps_leaf_factors hps_leaf_factors;
hps_status hps_leaf_factor(hps_ctx* ctx, const hps_leaf_kind* kind, int nbox, const double* b, int nrhs_max,
                           hps_precision precision, int* box_status, void* stream, hps_leaf_factors** out);
hps_status hps_leaf_solve_factored(hps_leaf_factors* factors, int nrhs, const double* f, double* v, double* h,
                                   int* box_status, void* stream);
hps_status hps_leaf_reconstruct_factored(hps_leaf_factors* factors, int nrhs, const double* v, const double* ub,
                                         double* ui, int* box_status, void* stream);
void hps_leaf_factors_destroy(hps_leaf_factors* factors);

/* ---- Interface solve on the GPU (nested dissection over the box grid) -----
 *
 * The interface system of Sec. 3.1 for an nb[0] x nb[1] x nb[2] grid of leaf
 * boxes of order p: at every face node shared by two boxes the outward fluxes
 * T^tau u_b^tau + h^tau of both add up to zero (Eq. 4 with f_b = 0), and u = g
 * is known on the faces of the outer boundary (moved to the right-hand side).
 * The paper factors it on the host with MUMPS (Sec. 3.2).  Here it is
 * factored on the device by the hierarchical merge that Sec. 3 recalls from
 * the original HPS method: the box range is halved along its longest axis
 * (in boxes, ties to the lower axis) recursively; each merge of halves a, b
 * eliminates the nodes of the face between them (3) against the halves'
 * other boundary nodes (1, 2):
 *     W = T^a_33 + T^b_33,  S = -W^{-1} [T^a_31  T^b_32],
 *     merged map  diag(T^a_11, T^b_22) + [T^a_13; T^b_23] S,
 * with an FP64 LU with partial pivoting of W per merge, all merges of a level
 * in one batch.  Pivoting is local to each W (MUMPS may pivot more widely).
 *
 * hps_interface_factor: T device [nbox][m][m], the leaf DtN maps (boxes x
 * fastest, then y, then z), read during the call only (their columns on the
 * outer faces are copied for the Dirichlet term).  nrhs_max (1..256): the
 * largest nrhs of later solves.  precision: HPS_FP64 factors and stores every
 * W^{-1}, S and merged-map block in FP64; HPS_FP32_IR does so in FP32 (the
 * tensor-core LU with 3 x BF16 operands and FP32 accumulation for separators
 * of 256 and more unknowns, the CUDA-core FP32 LU below) and keeps a copy of
 * T in FP64, from which each
 * solve refines its answer: with u the current face values, every box's flux
 * T^tau u^tau + h^tau sums, over the boxes sharing a node, to the residual of
 * the interface equations, and solving the system with those fluxes as loads
 * gives the correction; corrections stop on the device when one is below
 * 1e-14 of ||u|| or shrank by less than half, after at most 10.  Other
 * precisions: HPS_EINVAL.  Synchronous: it returns once the factorisation has
 * finished on `stream`.  Returns HPS_EINVAL for bad arguments, HPS_ENOMEM
 * when device memory runs out or a separator exceeds 14,000 nodes (an
 * 8 x 8 x 8 grid at p = 16 has 12,544 at the top), HPS_ESINGULAR when some
 * W had an exactly zero pivot (no handle is made).
 *
 * hps_interface_solve: h device [nbox][nrhs][m], the leaf fluxes (the h of
 * hps_leaf_particular / hps_leaf_solve_factored); g device [nbox][nrhs][m] or
 * NULL, the Dirichlet values, read only on each box's faces that lie on the
 * outer boundary (NULL: g = 0).  Writes u_b device [nbox][nrhs][m], the face
 * values of every box (the interface solution on shared faces, g on outer
 * ones) in the layout hps_leaf_reconstruct reads (Sec. 2.2 step 3,
 * Algorithm 2).  Enqueued on `stream`, allocates nothing; solves on one
 * handle share its buffers and must not overlap.  HPS_EINVAL for nrhs out
 * of range or NULL arrays.
 *
 * hps_interface_info: merges, levels, largest separator (nodes) and the
 * device bytes the handle holds.  hps_interface_last_refinement
 * (synchronises the device): the corrections the last HPS_FP32_IR solve took
 * and its last relative correction ||du|| / ||u|| (0 and 0 for HPS_FP64).
 *
 * hps_interface_plan (host only, no GPU): the merge tree.  *n_merge = nbox - 1
 * merges, numbered nbox .. 2 nbox - 2 in order of height (root last); leaves
 * are the boxes 0 .. nbox-1.  nodes [n_merge][8]: child a, child b, height,
 * axis, na1, nsep, nb2, offset into lists; lists holds a1 (na1), a3 (nsep),
 * b2 (nb2), b3 (nsep): face slots of the children (a leaf's slot is its local
 * face 0..5; a merge's slot i is the i-th face of its boundary, which lists
 * a's faces at a1 and then b's at b2).  a1/b2: faces off the separator,
 * a3/b3: separator faces, both in the same order.  Call with NULL arrays to
 * get the sizes. */
typedef struct hps_interface hps_interface;
hps_status hps_interface_factor(hps_ctx* ctx, int p, const int nb[3], const double* T, int nrhs_max,
                                hps_precision precision, void* stream, hps_interface** out);
hps_status hps_interface_solve(hps_interface* iface, int nrhs, const double* h, const double* g, double* ub,
                               void* stream);
hps_status hps_interface_info(const hps_interface* iface, int* n_merge, int* n_levels, int* max_separator,
                              size_t* bytes);
hps_status hps_interface_last_refinement(hps_interface* iface, int* corrections, double* rel_correction);
void hps_interface_destroy(hps_interface* iface);
hps_status hps_interface_plan(int p, const int nb[3], int* n_merge, int* n_list, int* nodes, int* lists);

/* The same for an nb[0] x nb[1] grid of 2-D boxes (hps_leaf2d_solve's maps
 * T [nbox][m][m], m = 4 (p-2); h, g, u_b [nbox][nrhs][m]): the grid is split
 * the same way, a "face" being an edge of p - 2 nodes (slots 0..3 of a leaf:
 * x-, x+, y-, y+).  Solve, info, refinement report and destroy are the
 * calls above. */
hps_status hps_interface2d_factor(hps_ctx* ctx, int p, const int nb[2], const double* T, int nrhs_max,
                                  hps_precision precision, void* stream, hps_interface** out);
hps_status hps_interface2d_plan(int p, const int nb[2], int* n_merge, int* n_list, int* nodes, int* lists);

/* ---- The 2-D leaf reduction (FP64) ----------------------------------------
 *
 * The method in two dimensions (Sec. 1; Sec. 3.2 sizes the 2-D DtN maps at
 * about 4p x 4p): per box a p x p Chebyshev-Lobatto grid on [lo, lo + h],
 * corners dropped (Remark 1), n = (p-2)^2 interior and m = 4 (p-2) edge nodes,
 * the operator -Lap u - kappa^2 b u with edge rows the outward normal
 * derivative.  Layouts (row-major, boxes outermost, device memory):
 *   grid node (i,j), 0 <= i,j < p                 index i + p j
 *   interior node (i,j), 1 <= i,j <= p-2           index (i-1) + q (j-1)
 *   edge f in the order x-, x+, y-, y+; edge node with free index a (1..q)
 *                                                 index f q + (a-1)
 *   b [nbox][p^2]   f [nbox][nrhs][p^2]   T [nbox][m][m]   S [nbox][n][m]
 *   v [nbox][nrhs][n]   h [nbox][nrhs][m]   u_b [nbox][nrhs][m]   u_i [nbox][nrhs][n]
 *
 * hps_leaf2d_solve: one FP64 LU with partial pivoting of A_ii per box
 * carrying [-A_ib | f_i] gives S = -A_ii^{-1} A_ib, T = A_bb + A_bi S
 * (Sec. 2.2, Eq. 8) and, for nrhs (0..256) loads, v = A_ii^{-1} f_i and
 * h = A_bi v (Algorithm 2).  T, S: either may be NULL (not both when
 * nrhs = 0); f, v, h are required when nrhs > 0.  h[2] > 0 are the box
 * sides, p in 3..24.  box_status (device [nbox] or NULL) as for the 3-D
 * calls.  Workspace comes from the stream-ordered allocator
 * (cudaMallocAsync) and is released on the stream; the differentiation
 * tables travel as kernel parameters, so the call makes no host copy.  HPS_EINVAL for bad
 * arguments, HPS_ENOMEM when the workspace cannot be allocated.
 *
 * hps_leaf2d_reconstruct: u_i = v + S u_b (Sec. 2.2 step 4) with S from
 * hps_leaf2d_solve; v may be NULL (then u_i = S u_b). */
hps_status hps_leaf2d_solve(int p, const double h[2], double kappa, int nbox, const double* b, int nrhs,
                            const double* f, double* T, double* S, double* v, double* hflux, int* box_status,
                            void* stream);
hps_status hps_leaf2d_reconstruct(int p, int nbox, int nrhs, const double* S, const double* v, const double* ub,
                                  double* ui, void* stream);

/* Operators with cross terms on Legendre face grids (Remark 1 of Sec. 2.1;
 * Sec. 4.3's curved domains need them).  The operator is
 *   A u = -sum_{a,b} C_ab(x) d_a d_b u + sum_a d_a(x) d_a u - kappa^2 b(x) u
 * with a symmetric coefficient tensor C.  Cross terms couple interior nodes
 * to edge and corner nodes, so the face data lives on a (p-1) x (p-1) tensor
 * grid of Gauss-Legendre nodes per face instead of the (p-2) x (p-2)
 * Chebyshev face nodes: m = 6 (p-1)^2 Legendre face nodes, n = (p-2)^3
 * interior nodes, p in 4..16.  Boundary Chebyshev nodes take their values
 * from the faces' Legendre data by polynomial interpolation (degree p-2 per
 * face coordinate); a node on several faces (edges, corners) takes the
 * average over them.  Neumann data are the outward normal derivatives at
 * each face's p x p Chebyshev nodes interpolated (degree p-1) to its Legendre
 * nodes.  Layouts (row-major, boxes outermost, device memory):
 *   grid node (i,j,k)                              index i + p j + p^2 k
 *   interior node (i,j,k), 1 <= i,j,k <= p-2       index (i-1) + q (j-1) + q^2 (k-1)
 *   Legendre node (s,t) of face f (x-, x+, y-, y+, z-, z+; s along the
 *   face's lower free axis)                        index f (p-1)^2 + s + (p-1) t
 *   C [nbox][6][p^3] (C11, C22, C33, C12, C13, C23 at every grid node)
 *   d [nbox][3][p^3] or NULL   b [nbox][p^3]   f [nbox][nrhs][p^3]
 *   T [nbox][m][m]   S [nbox][n][m]   v [nbox][nrhs][n]   h [nbox][nrhs][m]
 *
 * hps_leaf_cross_sizes: n and m of order p.
 * hps_leaf_cross_nodes: coordinates xyz [m][3] (host) of the Legendre face
 * nodes of the box [lo, lo + h].
 * hps_leaf_cross_solve (FP64): one LU with partial pivoting of A_II per box
 * carrying [-A_IE P | f_I] gives S = -A_II^{-1} A_IE P (P: Legendre data to
 * boundary Chebyshev values), T = Q N [S; P] (the DtN map on the Legendre
 * grids) and, for nrhs (0..256) loads, v = A_II^{-1} f_I and h = Q N [v; 0]
 * (Sec. 2.2 and Algorithms 1 and 2 with these index sets).  T, S: either may
 * be NULL (not both when nrhs = 0).  box_status as for the other leaf calls.
 * Workspace from the stream-ordered allocator, released on the stream;
 * HPS_EINVAL for bad arguments, HPS_ENOMEM when it cannot be allocated.
 * The interpolation tables (T_E alone is m x m doubles) are built on the
 * host and copied from pageable memory: the copy is staged before the call
 * returns, and the call cannot be captured into a CUDA graph.
 * hps_leaf_cross_reconstruct: u_i = v + S u_b with S from hps_leaf_cross_solve
 * (v may be NULL), u_b [nbox][nrhs][m] on the Legendre grids. */
hps_status hps_leaf_cross_sizes(int p, int* n, int* m);
hps_status hps_leaf_cross_nodes(int p, const double lo[3], const double h[3], double* xyz);
hps_status hps_leaf_cross_solve(int p, const double h[3], double kappa, int nbox, const double* C, const double* d,
                                const double* b, int nrhs, const double* f, double* T, double* S, double* v,
                                double* hflux, int* box_status, void* stream);
hps_status hps_leaf_cross_reconstruct(int p, int nbox, int nrhs, const double* S, const double* v, const double* ub,
                                      double* ui, void* stream);

/* ---- Mixed orders (adaptive p; Sec. 6 names adaptivity in the local order
 * as a setting the two-level scheme can serve).  Box tau of the grid
 * nb[0] x nb[1] x nb[2] (index bx + nx (by + ny bz), as for
 * hps_assemble_interface_blocks) has order p_box[tau] (3..24) and its own DtN
 * map T_tau [m_tau][m_tau] and flux h_tau [m_tau] from hps_leaf_groups.  A
 * face shared by boxes of different orders carries its unknowns on the face
 * grid of the higher order (its interior Chebyshev-Lobatto points in each
 * free direction); the other box sees them through polynomial interpolation
 * P to its own face nodes and returns its fluxes through the interpolation
 * Q the other way.  Interface system: sum_tau Q_tau T_tau P_tau u = -sum_tau
 * Q_tau h_tau on the interface unknowns, the Dirichlet unknowns carrying g.
 * Numbering: faces as for hps_assemble_interface_blocks (interface faces,
 * then Dirichlet faces), each face's unknowns contiguous in face-local order
 * (lower free axis fastest); Dirichlet unknowns after the interface ones.
 * Host routines, O(q^6) per box for the assembly; HPS_EINVAL for bad sizes,
 * orders or NULL arrays.
 * hps_mixed_layout: the counts, face orders face_p [n_faces] and the first
 * unknown of each face face_off [n_faces + 1] (either may be NULL).
 * hps_mixed_face_coords: coordinates [n_iface + n_dir][3] of every unknown
 * for the domain [lo, lo + L].
 * hps_mixed_assemble: unsummed COO triplets of the interface x interface
 * (rows, cols, vals) and interface x Dirichlet (rows_d, cols_d: Dirichlet
 * index, vals_d) blocks from the host maps T[tau]; NULL arrays query nnz and
 * nnz_d.
 * hps_mixed_reduce: r [n_iface + n_dir] = sum_tau Q_tau h_tau from host
 * fluxes hflux[tau] [m_tau].
 * hps_mixed_traces: ub[tau] [m_tau] = P_tau u for the host vector u
 * [n_iface + n_dir] (interface solution, then Dirichlet values). */
hps_status hps_mixed_layout(const int nb[3], const int* p_box, int64_t* n_iface, int64_t* n_dir, int* face_p,
                            int64_t* face_off);
hps_status hps_mixed_face_coords(const int nb[3], const int* p_box, const double lo[3], const double L[3],
                                 double* xyz);
hps_status hps_mixed_assemble(const int nb[3], const int* p_box, const double* const* T, int64_t* nnz, int64_t* rows,
                              int64_t* cols, double* vals, int64_t* nnz_d, int64_t* rows_d, int64_t* cols_d,
                              double* vals_d);
hps_status hps_mixed_reduce(const int nb[3], const int* p_box, const double* const* hflux, double* r);
hps_status hps_mixed_traces(const int nb[3], const int* p_box, const double* u, double* const* ub);

/* ---- Leaf impedance-to-impedance maps (the ItI variant of HPS that the
 * two-level scheme adapts to, Sec. 6).  For each box, R [m][m] (complex)
 * takes impedance data f = du/dn + i eta u on the face nodes to
 * g = du/dn - i eta u for the solution of the homogeneous equation, from the
 * kept-node collocation system of Sec. 2.1 / Eq. 2 with i eta added on the
 * face rows' own unknowns:
 *     [A_ii, A_ib; A_bi, A_bb + i eta I] [u_i; u_b] = [0; f],  R f = f - 2 i eta u_b.
 * A_ii is never inverted on its own, so R exists where kappa^2 is a
 * Dirichlet eigenvalue of the box; elsewhere R = (T - i eta I)(T + i eta I)^{-1}.
 * FP64: each box's system, in real form (size 2 (n + m), m right-hand
 * sides), is factored by the batched LU with partial pivoting.
 * kind: p in 4..16, h, kappa as for hps_leaf_build_dtn, beta NULL (no
 * first-order term); eta finite, nonzero;
 * b: device [nbox][p^3]; R: device [nbox][m][m] complex, interleaved (real,
 * imaginary) FP64 pairs, row r = output face node, column c = input face
 * node, face order as for T.  box_status: device [nbox] or NULL, as for the
 * other leaf calls.  Workspace from the stream-ordered allocator
 * (2 (n + m) x (2 (n + m) + m) doubles per box), released on the stream;
 * the differentiation tables are formed on the device, so the call makes no
 * host copy.  HPS_EINVAL for bad arguments, HPS_ENOMEM when it cannot be
 * allocated. */
hps_status hps_leaf_iti(const hps_leaf_kind* kind, double eta, int nbox, const double* b, double* R, int* box_status,
                        void* stream);

/* The same system with more outputs (all complex, interleaved, device;
 * NULL where not wanted): R as above; S [nbox][n][m], the interior solution
 * for unit incoming impedance data; for nrhs (0..256) loads f [nbox][nrhs][p^3]
 * (real, interior values read) solved with zero incoming impedance data, the
 * interior solution v [nbox][nrhs][n] and its outgoing impedance data
 * hout [nbox][nrhs][m] = -2 i eta u_b.  HPS_EINVAL as for hps_leaf_iti, or
 * when nothing is requested. */
hps_status hps_leaf_iti_solve(const hps_leaf_kind* kind, double eta, int nbox, const double* b, int nrhs,
                              const double* f, double* R, double* S, double* v, double* hout, int* box_status,
                              void* stream);

/* Box solutions from incoming impedance data fin [nbox][nrhs][m] (device,
 * complex): u_i = S fin + v into ui [nbox][nrhs][n] (needs S; v may be
 * NULL) and the face values u_b = (fin - (R fin + hout)) / (2 i eta) into
 * ub [nbox][nrhs][m] (needs R; hout may be NULL); either output may be
 * NULL, not both. */
hps_status hps_leaf_iti_reconstruct(int p, double eta, int nbox, int nrhs, const double* R, const double* S,
                                    const double* v, const double* hout, const double* fin, double* ui, double* ub,
                                    void* stream);

/* Host assembly of the two-level system on ItI maps for an nb[0] x nb[1] x
 * nb[2] grid of order-p boxes (4..16; box index bx + nx (by + ny bz)).
 * Unknowns: each box's incoming impedance data on its m face nodes, index
 * box m + r.  A face shared by boxes tau and sigma: the incoming data of one
 * side is minus the outgoing data of the other, f_tau + R_sigma f_sigma =
 * -hout_sigma at the matching node (same within-face index on the opposite
 * local face); a Dirichlet face (u = g): (R_tau - I) f_tau = -hout_tau -
 * 2 i eta g.  hps_iti_assemble: unsummed COO triplets (complex vals,
 * interleaved) from the host maps R [nbox][m][m]; NULL arrays query nnz.
 * hps_iti_rhs: rhs [nbox m] (complex) from host hout [nbox][m] (one load,
 * or NULL) and the real Dirichlet values g_face [nbox][m] at each box's face
 * nodes (read on boundary faces only; NULL for g = 0). */
hps_status hps_iti_assemble(int p, const int nb[3], const double* R, int64_t* nnz, int64_t* rows, int64_t* cols,
                            double* vals);
hps_status hps_iti_rhs(int p, const int nb[3], double eta, const double* hout, const double* g_face, double* rhs);

/* The collocation operator applied to full nodal fields: out = A u at every
 * interior node of each box, the interior rows of Eq. 2 (-Laplacian by the
 * three grid lines through the node, minus kappa^2 b u), and 0 at the face,
 * edge and corner nodes.  u and out: device [nbox][nfield][p^3] in node order
 * (edge and corner values of u are not read), b as in hps_leaf_build_dtn.
 * Time stepping uses it for the right-hand side (I + dt/2 A) u^n of a
 * Crank-Nicolson step (Sec. 4.4).  HPS_EINVAL for bad sizes or NULL arrays. */
hps_status hps_leaf_apply(hps_ctx* ctx, const hps_leaf_kind* kind, int nbox, int nfield, const double* b,
                          const double* u, double* out, void* stream);

/* Optional per-kernel timing.  hps_profile_enable(ctx, 1) makes the leaf calls
 * bracket every kernel launch with CUDA events on the caller's stream and
 * record each launch's algorithmic flops (2 M N K for an update product, the
 * dense method's count) and bytes.  hps_profile_get synchronises and returns,
 * for kernel class cls (0 operator build, 1 panel factorisation, 2 CUDA-core
 * update product, 3 tensor-core update product, 4 row gather of the products,
 * 5 FP64 refinement residual, 6 refinement update, 7 D_n product,
 * 8 tensor-core update product of the refinement solves, 9 split copies of
 * the LU operators, 10 double-float first residual, 11 bookkeeping:
 * permutation composition and inversion, refinement checks, kappa^2 b,
 * output transposes and stored-S reconstruction), the accumulated launches,
 * milliseconds, flops and bytes since the last reset.  Refinement launches
 * skip boxes that have converged, so classes 5, 6 and 8 count the work of
 * every box and overstate flops and bytes.  Returns HPS_EINVAL for cls
 * outside 0..11. */
hps_status hps_profile_enable(hps_ctx* ctx, int on);
hps_status hps_profile_reset(hps_ctx* ctx);
hps_status hps_profile_get(hps_ctx* ctx, int cls, long long* launches, double* ms, double* flops, double* bytes);

const char* hps_status_string(hps_status s);

/* Self-test of the FP64 <-> FP32 conversions that the refinement kernels run
 * on the integer pipe (IEEE-754 round to nearest even, hardware conversion for
 * values outside the normal range): n values on device `device` (random bit
 * patterns over all exponents, values at the float range limits, exact
 * rounding ties) are converted both ways and compared bit for bit with the
 * hardware conversions.  mismatches[0] receives the double -> float
 * mismatches, mismatches[1] the float -> double ones (host array of 2).
 * Allocates 16 bytes of device memory for the call; synchronises. */
hps_status hps_selftest_conversions(int device, long long n, unsigned long long seed, long long* mismatches);

#ifdef __cplusplus
}
#endif

#endif /* HPS_H */
