/*
 * parament.h -- C ABI of the GB300 parallel-in-time propagator.
 *
 * Method (Herb & Welter, "Parallel time integration using Batched BLAS
 * routines", arXiv 2108.07126): for H(t) = H0 + sum_k c_k(t) H_k (Sec. 2,
 * Eq. format_control) the library forms, for every slice j of duration dt,
 * the Hermitian exponent G_j (midpoint rule, Sec. 3.2; fourth-order Magnus
 * exponent, Sec. 4), the slice propagator U_j = exp(-i G_j) (Sec. 2.1), and
 * the ordered product U(T) = U_N ... U_1 (Sec. 2, Eq. slices) by a pairwise
 * product tree (Sec. 2.2).  Usage follows the paper's state machine (Sec. 6,
 * Fig. 5): create -> set_hamiltonians -> set_controls -> propagate (repeat)
 * -> destroy.
 *
 * Conventions shared by every entry point:
 *   - Every function returns a parament_status; nothing throws across the ABI.
 *   - Complex matrices are dense, row-major, interleaved (re, im): the layout
 *     of numpy/torch complex64 / complex128 arrays.
 *   - A pointer argument may be host or device memory; the library asks the
 *     CUDA runtime which one it is.  Device pointers are used in place, host
 *     data is staged through buffers owned by the context.
 *   - Work is enqueued on the context's stream.  A call that writes to host
 *     memory waits for its own result; otherwise calls return without waiting.
 *   - A context is neither thread-safe nor reentrant (Sec. 6): concurrent calls
 *     on one context, or overlapping propagations of one context on several
 *     streams, race on its workspace.  Distinct contexts are independent.
 *   - Calling out of order returns PARAMENT_ERR_STATE and changes nothing.
 */
#ifndef PARAMENT_H
#define PARAMENT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PARAMENT_VERSION_MAJOR 0
#define PARAMENT_VERSION_MINOR 1

typedef struct parament_ctx parament_ctx;

typedef enum {
    PARAMENT_OK = 0,
    PARAMENT_ERR_INVALID_VALUE = 1, /* bad argument: null pointer, size out of range */
    PARAMENT_ERR_STATE = 2,         /* call out of the create/set/propagate order */
    PARAMENT_ERR_ALLOC = 3,         /* device or host allocation failed */
    PARAMENT_ERR_CUDA = 4,          /* a CUDA runtime call failed (text in parament_last_error) */
    PARAMENT_ERR_NONFINITE = 5,     /* NaN/Inf in Hamiltonians or controls */
    PARAMENT_ERR_NOT_HERMITIAN = 6, /* H0 or some H_k is not Hermitian (tolerance: option) */
    PARAMENT_ERR_TIMEOUT = 7,       /* a bounded device-side wait expired */
    PARAMENT_ERR_UNSUPPORTED = 8    /* valid request this build does not implement */
} parament_status;

/* storage type of Hamiltonians and of the propagator U */
typedef enum { PARAMENT_C64 = 0, PARAMENT_C128 = 1 } parament_dtype;
/* storage type of the real control samples */
typedef enum { PARAMENT_F32 = 0, PARAMENT_F64 = 1 } parament_real_dtype;

/*
 * Exponent of one slice t_j = j dt .. t_j + dt; S = number of samples per control.
 *  MIDPOINT:          G_j = dt H(t_j + dt/2), one sample per slice, S = N
 *                     (Sec. 3.2: G = H dt; Sec. 4: Omega_1 by the mid-point rule).
 *  MAGNUS4_GL2:       G_j = dt/2 (H1 + H2) + i sqrt(3) dt^2 / 12 [H1, H2], H1, H2 sampled at
 *                     t_j + dt (1/2 -+ sqrt(3)/6), S = 2N, samples interleaved per slice
 *                     (Sec. 4, Eq. magnus: Omega_1 + Omega_2 on two Gauss-Legendre nodes).
 *  MAGNUS4_SIMPSON:   G_j = dt/6 (H1 + 4 H2 + H3) + i dt^2 / 12 [H1, H3], samples at
 *                     t_j, t_j + dt/2, t_j + dt shared between neighbours, S = 2N + 1
 *                     (Sec. 4 and Eq. magnus_coeffs, commutator sign taken from Omega_2).
 * The Magnus exponents are expanded into effective controls: the basis
 * {H0, H_k, i[H0, H_k], i[H_k, H_k'] (k < k')}, 1 + K(K+3)/2 Hermitian matrices
 * (Sec. 4, Eq. magnus_coeffs), built once by set_hamiltonians.
 */
typedef enum {
    PARAMENT_MIDPOINT = 0,
    PARAMENT_MAGNUS4_GL2 = 1,
    PARAMENT_MAGNUS4_SIMPSON = 2
} parament_integrator;

/*
 * Arithmetic of the exponential and of the product tree.
 *  FP64: everything in double.
 *  FP32: exponent assembly, exponential and the in-block tree in float; the
 *        norm bound that picks the Taylor degree and the number of squarings,
 *        and the product tree above the thread-block level, in double.
 *  FP32_TC_TF32X3: FP32 with the complex products of large d on the tensor
 *        cores: every FP32 operand split into two round-to-nearest TF32 terms,
 *        three MMAs per real product (hi*hi + hi*lo + lo*hi), FP32 accumulation
 *        with a fresh accumulator per k-chunk; FP64 norm bound and FP64 top
 *        tree as in FP32.  d in 17..256: tcgen05 with tensor-memory
 *        accumulators (d <= 64: working matrices in shared memory, the four real
 *        products of a complex product in one M = 128 MMA chain; d = 129..256:
 *        four 128 x 128 output blocks per product).  d <= 16:
 *        PARAMENT_ERR_UNSUPPORTED.  parament_stats.product_backends names the
 *        code that ran.
 *  FP32_TC_BF16X3: FP32 with every operand split into three round-to-nearest
 *        BF16 terms (x = b0 + b1 + b2, 24 significant bits) and the six products
 *        b0 b0 + b0 b1 + b1 b0 + b0 b2 + b1 b1 + b2 b0 per real product on the
 *        tensor cores (tcgen05 kind::f16), FP32 accumulation with a fresh
 *        accumulator per k-chunk.  d in 17..256: tcgen05; d <= 16:
 *        PARAMENT_ERR_UNSUPPORTED.
 */
typedef enum {
    PARAMENT_PREC_FP64 = 0,
    PARAMENT_PREC_FP32 = 1,
    PARAMENT_PREC_FP32_TC_BF16X3 = 2,
    PARAMENT_PREC_FP32_TC_TF32X3 = 3
} parament_precision;

/* keys of parament_set_option / parament_get_option */
typedef enum {
    /* 0 (default) = choose the Taylor degree per slice from the norm bound;
       m > 0 = force degree m (one of 1, 2, 4, 6, 9, 12), squarings still from the bound */
    PARAMENT_OPT_TAYLOR_DEGREE = 1,
    /* thread blocks of the fused kernel; 0 (default) = fill every SM */
    PARAMENT_OPT_GRID_BLOCKS = 2,
    /* warps per thread block; 0 (default) = largest that fits shared memory (at most 16 for FP32
       d in 9..16, 8 otherwise) */
    PARAMENT_OPT_BLOCK_WARPS = 3,
    /* 1 (default) = reject non-Hermitian H in set_hamiltonians; 0 = skip the check */
    PARAMENT_OPT_CHECK_HERMITIAN = 4,
    /* extra squarings added to every slice (default 0; accuracy experiments) */
    PARAMENT_OPT_EXTRA_SQUARINGS = 5,
    /* Hermiticity tolerance in units of 1e-12 relative to max |H_ab| (default 1000, i.e. 1e-9) */
    PARAMENT_OPT_HERMITIAN_TOL_E12 = 7,
    /* gradient: slices per sub-chunk of the adjoint sweep (0 = auto: a whole leaf when it fits the
       workspace cap); leaves longer than a sub-chunk are re-computed from checkpoints */
    PARAMENT_OPT_GRAD_SUBCHUNK = 8,
    /* gradient: cap in MiB on the per-slice prefix buffer of the adjoint sweep (default 4096) */
    PARAMENT_OPT_WORKSPACE_MB = 9,
    /* batched: target slices per leaf (0 = default 64) */
    PARAMENT_OPT_BATCH_LEAF_STEPS = 10,
    /* batched: work items per SM (0 = default 32) */
    PARAMENT_OPT_BATCH_ITEMS_PER_SM = 11,
    /* batched: 1 (default) = capture set-up and launch in a CUDA graph and replay it; 0 = launch directly */
    PARAMENT_OPT_BATCH_GRAPH = 12,
    /* exponential of parament_propagate: 0 (default) = Taylor with scaling and squaring, degree per
       slice; 1 = the paper's Chebyshev series (Sec. 2.1, Algorithm 1) with one spectral interval
       [-beta, beta] for all slices (beta = largest per-slice norm bound, found on the device) and the
       degree of Eq. error_chebychev; every d and precision.  Trajectories reject it
       (PARAMENT_ERR_UNSUPPORTED); the gradient always uses the Taylor exponential */
    PARAMENT_OPT_EXP_METHOD = 13,
    /* FP32 and tensor-core precisions: 1 (default) = one Newton-Schulz step R <- R (3 I - R^dagger R) / 2
       on every leaf product (the exact product is unitary; FP32 rounding that repeats from slice to
       slice, and the truncating tensor-core accumulation, otherwise drift R off the unitary group
       linearly in the leaf length); 0 = plain products */
    PARAMENT_OPT_UNITARY_STEP = 14,
    /* batched, tensor-core precisions: bit mask of the dimension classes whose products run on the
       CUDA cores instead of tcgen05 (bit 0: d 17..32, bit 1: d 33..64, bit 2: d 65..128); default 0.
       parament_batch_autotune sets it. */
    PARAMENT_OPT_BATCH_CUDA_CORE_CLASSES = 15
} parament_option;

/* per-call diagnostics of the most recent propagate (see parament_get_stats) */
typedef struct {
    int64_t n_steps;          /* slices propagated */
    int32_t dim;              /* d */
    int32_t n_basis;          /* 1 + number of (effective) controls */
    int32_t grid_blocks;      /* thread blocks launched */
    int32_t block_threads;    /* threads per block */
    int32_t leaves;           /* sequential leaf products below the pairwise tree */
    int32_t max_degree;       /* largest Taylor degree used */
    int32_t max_squarings;    /* largest number of squarings used */
    int32_t grad_subchunk;    /* slices per sub-chunk of the latest gradient (0 if none) */
    int64_t exp_products;     /* complex d x d products in exponentials and squarings */
    int64_t tree_products;    /* complex d x d products in the product tree */
    uint32_t device_status;   /* PARAMENT_DEV_* bits raised by the kernels */
    uint32_t product_backends; /* PARAMENT_BACKEND_* bits: the code that ran the complex products */
    double kernel_ms;         /* device time of the propagation kernels (events) */
} parament_stats;

/* product back-ends reported in parament_stats.product_backends (a batched call ORs the
   back-ends of its dimension classes) */
#define PARAMENT_BACKEND_CUDA_CORES 0x1u /* FP32 / FP64 fused multiply-adds */
#define PARAMENT_BACKEND_MMA_SYNC 0x2u   /* warp-level mma.sync instructions (no path of this build uses them) */
#define PARAMENT_BACKEND_TCGEN05 0x4u    /* tcgen05.mma with tensor-memory accumulators */

#define PARAMENT_DEV_NONFINITE_NORM 0x1u /* a slice's norm bound was NaN/Inf */
#define PARAMENT_DEV_NORM_CAPPED 0x2u    /* a norm exceeded the largest scaling in the table */
#define PARAMENT_DEV_TENSOR_TIMEOUT 0x4u /* a bounded tensor-core wait gave up; the result is invalid */

/* Library version as major * 1000 + minor. */
int parament_version(void);

/*
 * Create a context on CUDA device `device`, enqueuing on `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).  *out receives the
 * handle, owned by the caller, released by parament_destroy.  Sec. 6: the
 * context stores the integrator state.
 */
int parament_create(parament_ctx **out, int device, void *cuda_stream);

/* Release a context and every device buffer it owns; NULL is a no-op.
   Waits for the context's stream.  Sec. 6 (Parament_free). */
int parament_destroy(parament_ctx *ctx);

/* Switch the stream later calls enqueue on (NULL = legacy default stream). */
int parament_set_stream(parament_ctx *ctx, void *cuda_stream);

/*
 * Upload H0 (d x d) and the K control Hamiltonians Hk (K x d x d, contiguous)
 * and choose the integrator (Sec. 6, Parament_setHamiltonian; the Magnus
 * choice makes the library form the commutator basis here, Sec. 4).
 * `dtype` is the storage type of H0/Hk and of every later U_out.  The data are
 * copied; the caller keeps ownership.  1 <= d <= 256 (PARAMENT_ERR_UNSUPPORTED
 * above; d is padded with zeros to the next power of two, which is exact),
 * 0 <= K <= 16.  Hk may be NULL when K = 0.
 * Resets any controls set before.  Errors: INVALID_VALUE, NONFINITE,
 * NOT_HERMITIAN (checked on the device; the call waits for the check).
 */
int parament_set_hamiltonians(parament_ctx *ctx, int dim, int n_ctrl, const void *H0, const void *Hk,
                              parament_dtype dtype, parament_integrator integrator);

/*
 * Set the control samples c (K x S, row-major, c[k * S + s]) for n_steps
 * slices of duration dt (Sec. 3.2: amplitudes sampled at equidistant times;
 * S per integrator as documented above).  A device pointer is borrowed, not
 * copied: it must stay valid and unchanged until the propagations that use
 * it have run on the stream.  Page-locked (pinned) host memory is borrowed the
 * same way: the kernels read it in place over the host link, so the transfer
 * overlaps the computation.  Other host data is copied into a context buffer
 * (asynchronously on the context's stream).
 * 0 <= n_steps < 2^31 (0 gives U = I), dt finite.  Requires set_hamiltonians.
 */
int parament_set_controls(parament_ctx *ctx, const void *c, parament_real_dtype cdtype, int64_t n_steps,
                          double dt);

/*
 * Compute U(T) = U_N ... U_1 into U_out (d x d, the dtype of
 * set_hamiltonians) with arithmetic `prec` (Sec. 2, Eq. slices; Sec. 2.2).
 * One kernel launch (d <= 16: groups of lanes of one warp per slice, matrices
 * in shared memory; d > 16: one thread block per leaf, matrices in an
 * L2-resident scratch region, products as block-wide tiled GEMMs).  Per
 * slice it forms G_j from the control samples, bounds
 * ||G_j||_1 in FP64 from the coefficients (Sec. 3.2's triangle-inequality
 * bound, per slice), evaluates a Taylor polynomial of exp(-i G_j / 2^s)
 * (Paterson-Stockmeyer) and squares s times, multiplies consecutive slices in
 * sequential leaves, then combines the leaves pairwise in shared memory and
 * the blocks' partial products pairwise through global memory.
 * Requires set_hamiltonians and set_controls.
 */
int parament_propagate(parament_ctx *ctx, void *U_out, parament_precision prec);

/*
 * Gate-fidelity loss and its gradient with respect to every control sample
 * (Sec. 7 names GRAPE-type optimal control as the application; the paper gives
 * no gradient formula).  With z = Tr(V^dagger U(T)):
 *   *loss_out = 1 - |z|^2 / d^2                         (host double; NULL = skip, no wait)
 *   grad_out[k * S + s] = dL / dc_k(sample s)           (K x S; double for FP64, float for FP32;
 *                                                        S = N midpoint, 2N GL4, 2N + 1 Simpson)
 * U = S_j U_j P_{j-1}; dz/dc = Tr(L_{X_j}(P_{j-1} V^dagger S_j) dX_j/dc) with X_j = -i G_j,
 * dX_j/dc = -i sum_e (d gamma_e / dc) B_e over the effective-control basis (Sec. 4, Eq.
 * magnus_coeffs: H0, H_k, i[H0, H_k], i[H_k, H_l]), and L_X the Frechet derivative of exp, taken
 * as the upper-right block of exp([[X, Lambda], [0, X]]).  The prefixes P and suffixes S come from
 * the forward tree: leaf and block products of the forward kernel, exclusive scans over them, then
 * per leaf a forward sweep (prefixes, re-computed from checkpoints for long leaves) and a backward
 * sweep.  A Simpson end sample belongs to two slices and receives both contributions.  d <= 16:
 * groups of lanes of one warp per leaf; d = 17..256: one thread block per leaf (FP64 Hillis-Steele
 * scans of the leaf products for the prefixes, the suffixes, U(T) and z; block-wide products).
 * V: d x d in the dtype of set_hamiltonians; U_out: optional U(T).  Pointers host or device.
 * Errors: UNSUPPORTED for the tensor-core precisions; STATE before set_controls.
 */
int parament_propagate_grad(parament_ctx *ctx, const void *V, double *loss_out, void *grad_out, void *U_out,
                            parament_precision prec);

/*
 * Trajectory: the propagator (or a state) at intermediate times (Sec. 2: Eq. slices read at
 * t_n = n dt instead of T; the states psi(t) = U(t) psi_0 of the Schroedinger equation).
 * Outputs after slices n = every, 2 every, ..., and after the last slice N when N is not a
 * multiple of `every`: n_out = ceil(N / every) entries, output o after min((o + 1) every, N) slices.
 *   psi0 == NULL: out = U(t_n), [n_out][d][d] complex (the dtype of set_hamiltonians)
 *   psi0 != NULL: out = U(t_n) psi0, [n_out][d] complex; psi0 is [d] in the same dtype
 * Pointers host or device (a host `out` is filled before the call returns).  The library writes
 * out and keeps no reference to it or to psi0 after the call.  Method: one forward pass that keeps
 * every leaf and block product, exclusive FP64 prefix scans over them (as for the gradient), then a
 * second pass in which every leaf starts from its prefix and writes its running product at the
 * output slices.  Taylor exponential, FP64 or FP32, every d and integrator (d > 16: one leaf
 * per thread block, FP64 prefixes by a Hillis-Steele scan over the leaf products).  N = 0 writes
 * nothing (out may then be NULL).  Errors: INVALID_VALUE for a null out or every < 1; UNSUPPORTED for
 * tensor-core precisions or the Chebyshev option; STATE before set_controls.
 */
int parament_propagate_trajectory(parament_ctx *ctx, const void *psi0, void *out, int64_t every,
                                  parament_precision prec);

/* One problem of a batched call; all pointers are device memory owned by the caller. */
typedef struct {
    int dim;            /* d, 1..128 */
    int n_ctrl;         /* K, 0..16 */
    const void *H0;     /* d x d, dtype of the call */
    const void *Hk;     /* K x d x d (may be NULL when K = 0) */
    const void *c;      /* K x S real samples, cdtype of the call, S as for set_controls */
    int64_t n_steps;    /* N >= 0 */
    double dt;          /* slice duration */
    void *U_out;        /* d x d result, dtype of the call */
} parament_instance;

/*
 * Propagate many independent problems of uneven dimension and step count in
 * one persistent kernel launch (the paper propagates one problem per call;
 * batching many is an extension).  Every instance is cut into work items by
 * its cost (d^3 N); one block per SM takes items from an atomic queue,
 * largest first, and runs the body that fits the instance's dimension;
 * instances combine their pieces through their own pairwise arrival trees.
 * The set-up (all bases) and the launch are captured in a CUDA graph that is
 * replayed while the instance shapes stay the same (option
 * PARAMENT_OPT_BATCH_GRAPH; the context must have a non-default stream).
 * cdtype must match prec (F64 with FP64, F32 with FP32 and the tensor-core
 * precisions).  With FP32_TC_TF32X3 / FP32_TC_BF16X3 the instances of d >= 17
 * run their products on tcgen05, except the dimension classes listed in
 * PARAMENT_OPT_BATCH_CUDA_CORE_CLASSES; d <= 16 always runs on the CUDA cores.
 * Basis matrices are not pruned and Hermiticity is not checked.  Returns
 * without waiting.  Contexts keep the batch plan, so the same context must not
 * run two batches concurrently.
 */
int parament_propagate_batched(parament_ctx *ctx, const parament_instance *inst, int n_inst, parament_dtype dtype,
                               parament_real_dtype cdtype, parament_integrator integrator, parament_precision prec);

/*
 * Autotuner of the batched launch.  (1) Times the batch for every pair of
 * (target slices per leaf in {32, 128}) x (work items per SM in
 * {8, 16, 32, 64}).  (2) For the tensor-core precisions, then times every
 * choice of product back-end (tcgen05 or CUDA cores) for each dimension class
 * present (d 17..32, 33..64, 65..128) with the best split, and (3) if a class
 * moved to the CUDA cores, the split again.  Keeps the fastest in the context
 * options PARAMENT_OPT_BATCH_LEAF_STEPS, PARAMENT_OPT_BATCH_ITEMS_PER_SM and
 * PARAMENT_OPT_BATCH_CUDA_CORE_CLASSES and reports them (and the time in ms)
 * through the optional outputs.  Waits for the GPU.
 */
int parament_batch_autotune(parament_ctx *ctx, const parament_instance *inst, int n_inst, parament_dtype dtype,
                            parament_real_dtype cdtype, parament_integrator integrator, parament_precision prec,
                            int *best_leaf_steps, int *best_items_per_sm, double *best_ms,
                            unsigned *cuda_core_classes);

/* Diagnostics of the latest propagate; waits for the stream. */
int parament_get_stats(parament_ctx *ctx, parament_stats *out);

/* Set / read a numerics or launch option (parament_option).  Sec. 6 mentions
   helper functions that tweak the numerics, e.g. the series degree. */
int parament_set_option(parament_ctx *ctx, int key, int64_t value);
int parament_get_option(const parament_ctx *ctx, int key, int64_t *value);

/*
 * Taylor threshold theta_m for unit roundoff `u`: the largest x with
 * x^(m+1)/(m+1)! * e^x <= u, the truncation bound of the degree-m Taylor
 * polynomial of exp(A) for ||A|| <= x.  Host-only helper (no GPU needed);
 * returns a negative value for m < 1.
 */
double parament_taylor_theta(int m, double u);

/*
 * Degree m and squarings s the kernels use for a slice whose norm bound is
 * `norm_bound` (>= ||G||_1), at unit roundoff u (2^-53 for FP64, 2^-24 for
 * FP32): among m in {1, 2, 4, 6, 9, 12} (Paterson-Stockmeyer products
 * 0, 1, 2, 3, 4, 5) and s >= 0 with norm_bound / 2^s <= theta_m(u / 2^s), the
 * pair with the fewest complex products (PS products + s).  force_m = 0 lets
 * m vary, otherwise m = force_m.  Host-only helper (no GPU needed).
 * Errors: INVALID_VALUE for bad arguments, UNSUPPORTED if no s <= 62 suffices.
 */
int parament_taylor_choice(double norm_bound, double u, int force_m, int *m_out, int *s_out);

/*
 * --- Propagation without allocation -----------------------------------------
 * The paper has no counterpart to this entry point.  It serves callers that
 * cannot allocate device memory: an application or framework that owns all
 * device memory through its own allocator, or a latency-critical loop that
 * cannot afford the device-wide synchronisation of cudaMalloc / cudaFree.
 *
 * One call does what set_hamiltonians + set_controls + propagate do, without a
 * context and without allocating anything (no cudaMalloc, cudaFree or
 * allocating library routine).  Its intermediates live in one static device
 * array of PARAMENT_NOALLOC_SCRATCH_BYTES bytes (about 1.6 MiB) that every GPU
 * which loads the library holds until the process exits.
 *   - H0 (d x d), Hk (K x d x d), c (K x S), U_out (d x d): device pointers,
 *     layouts and S as for the context API; `dtype` for H and U, `cdtype` must
 *     match `prec` (F64 with FP64, F32 with FP32).  U_out must be aligned to
 *     its element (8 bytes for C64, 16 for C128) and c to its real type.  The
 *     caller owns them all.
 *   - device_status: NULL = return without waiting.  Otherwise the call waits
 *     for its work on the stream and stores there the PARAMENT_DEV_* bits the
 *     kernel raised (PARAMENT_DEV_NONFINITE_NORM: NaN or Inf reached a norm
 *     bound, i.e. in H0, Hk or c, and U is not valid; PARAMENT_DEV_NORM_CAPPED:
 *     a slice needed more squarings than the table holds).  This path does not
 *     check H or c for NaN / Inf before the launch, so that word is its only
 *     report of non-finite input.
 *   - Limits: d <= PARAMENT_NOALLOC_MAX_DIM, 1 + K (midpoint) or
 *     1 + K (K + 3) / 2 (Magnus) <= PARAMENT_NOALLOC_MAX_BASIS, at most
 *     PARAMENT_NOALLOC_MAX_BLOCKS thread blocks (more slices run in longer
 *     leaves).  Beyond a limit, or a precision other than FP64 / FP32:
 *     UNSUPPORTED.  Host pointers, misaligned pointers, mismatched or unknown
 *     dtypes, d < 1, bad sizes: INVALID_VALUE.  Non-finite dt: NONFINITE.
 *   - The first call on a device, with that device current, looks up the
 *     array's device address (cudaGetSymbolAddress); make that first call
 *     before any stream capture.
 *   - Every call shares the array, which keeps the latest call's contents
 *     (the arrival counters are cleared by each call).  Calls whose work
 *     overlaps on the GPU -- on two streams, or from two host threads -- race
 *     on it and corrupt each other's results: keep them on one stream.
 *   - Unlike set_hamiltonians it neither checks Hermiticity nor drops
 *     identically zero basis matrices; U equals parament_propagate's up to
 *     rounding.  Work is enqueued on cuda_stream (NULL = legacy default
 *     stream); the call returns without waiting.
 */
#define PARAMENT_NOALLOC_MAX_DIM 16
#define PARAMENT_NOALLOC_MAX_BASIS 45
#define PARAMENT_NOALLOC_MAX_BLOCKS 304
#define PARAMENT_NOALLOC_SCRATCH_BYTES 1641472
int parament_propagate_noalloc(int dim, int n_ctrl, const void *H0, const void *Hk, parament_dtype dtype,
                               parament_integrator integrator, const void *c, parament_real_dtype cdtype,
                               int64_t n_steps, double dt, void *U_out, parament_precision prec, void *cuda_stream,
                               uint32_t *device_status);

/*
 * Chebyshev exponential (Sec. 2.1): the largest half-width beta of the spectral
 * interval [-beta, beta] for which the truncation bound of Eq. error_chebychev,
 * eps = 4 (exp(1 - y^2) y)^(m+1), y = 2 beta / (4m + 4), stays below u (with
 * u = 2^-24 / 2^-53 this is Table 1).  Host-only; -1 for m outside [1, 48].
 */
double parament_chebyshev_theta(int m, double u);

/* Smallest degree m <= 48 whose Chebyshev bound covers half-width beta at u; -1 if none. */
int parament_chebyshev_degree(double half_width, double u);

/* Bessel functions J_0(x) .. J_n(x), x >= 0, n <= 48 (Miller's backward recurrence), the
   Chebyshev coefficients a_k = (-i)^k J_k(beta) of Sec. 2.1; host-only, the kernels use the same code. */
int parament_bessel_j(int n, double x, double *out);

/*
 * --- Measured peaks ----------------------------------------------------------
 * Not part of the paper's method: a measurement helper for reporting rooflines.
 * Times, on device `device` and stream `cuda_stream` (NULL = legacy default),
 * the rates the propagator's kernels are bound by, in TFLOP/s (2 flops per
 * multiply-add):
 *   fp32_tflops / fp64_tflops: independent fused multiply-add chains on the CUDA
 *     cores over a grid that fills every SM (the best of a few chain counts and
 *     occupancies); the *_max_clock figures count flops per SM clock cycle
 *     (clock64) instead of per second and scale them to the maximum SM clock, so
 *     they do not depend on the clock the GPU ran during the measurement;
 *   tf32_tflops / bf16_tflops: a stream of dense tcgen05 MMAs (M = 128, N = 256,
 *     K = 8 TF32 or 16 BF16, FP32 accumulation in tensor memory) issued by one
 *     thread per SM on operands in shared memory.
 * Each figure is the median of three timed launches (CUDA events) after a
 * warm-up launch, about 2 s in all; the call waits for the stream.  Allocates
 * two small device buffers (released before it returns).  Errors: CUDA,
 * TIMEOUT (a bounded wait on the tensor cores gave up; the figures are invalid).
 */
typedef struct {
    double fp32_tflops;
    double fp64_tflops;
    double tf32_tflops;
    double bf16_tflops;
    int32_t sm_count;
    int32_t reserved;
    double max_sm_clock_mhz;      /* the device's reported maximum SM clock */
    double fp32_tflops_max_clock; /* flops per SM clock cycle (clock64) x the maximum SM clock */
    double fp64_tflops_max_clock;
} parament_peaks;
int parament_measure_peaks(int device, void *cuda_stream, parament_peaks *out);

/* Static text for a status code. */
const char *parament_status_string(int status);

/* Text of the last error on this context (empty if none); valid until the next call. */
const char *parament_last_error(const parament_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* PARAMENT_H */
