/*
 * sfmm.h -- C ABI of the GB300 solid-harmonic translation library.
 *
 * Batched M2M, M2L and L2L translations of solid-harmonic expansions for the
 * Laplace kernel 1/|x-y| (Kirchhart, "solidfmm: A highly optimised library of
 * operations on the solid harmonics for use in fast multipole methods",
 * arXiv 2202.02847).  Every translation is computed by the rotation-based
 * factorisation of Sec. 2.4 / Sec. 3.4: scale the shift to unit length
 * (eq. scaling), rotate about z, swap x and z (Dehnen's matrices, eq.
 * swaptransform, in the reduced real form of eq. FGmappings), rotate about z,
 * swap again, translate along the z axis in O(P^3) (eq. zm2lkernels for M2L),
 * and undo the change of coordinates.  Kernels are hand-written CUDA for
 * sm_103a (GB300) and run asynchronously on the caller's stream.
 *
 * ------------------------------------------------------------------ data
 * Solid (Sec. 2.1, Fig. 1).  An expansion of order P has coefficients
 * C_n^m, 0 <= n < P, |m| <= n, with C_n^{-m} = (-1)^m conj(C_n^m); only m >= 0
 * is stored, Im C_n^0 is stored as 0.  A solid is P(P+1) contiguous reals
 * (double for SFMM_F64 handles, float for SFMM_F32): row n occupies reals
 * [n(n+1), (n+1)(n+2)) as  Re C_n^0 .. Re C_n^n, Im C_n^0 .. Im C_n^n.
 * (The paper's Fig. 1 gives the positions in a figure that is not available;
 * this row-wise Re/Im split is the layout its swap buffers use, Sec. 3.3.)
 *
 * Expansions (Sec. 2.1, eq. MLexpansions):
 *   multipole about x_A:  phi(x) = sum_{n,m} M_n^m conj(S_n^m(x - x_A))
 *   local about x_B:      phi(x) = sum_{n,m} L_n^m conj(R_n^m(x - x_B))
 * with R, S the regular and singular harmonics of the Appendix (no
 * Condon-Shortley phase; R_n^m = r^n P_n^m(cos t) e^{im p}/(n+m)!,
 * S_n^m = (n-m)! P_n^m(cos t) e^{im p}/r^{n+1}).
 *
 * Shift vectors are 3 reals (x, y, z) of the handle's dtype:
 *   r = (centre of the output expansion) - (centre of the input expansion),
 * i.e. r = x_B - x_A for M2L (Sec. 2.1, r_AB).  M2L needs r != 0 and the
 * expansions well separated; M2M and L2L with r = 0 copy the input.
 *
 * Orders (Sec. 1.1, mixed-order translations): the input has order p_in and
 * the output order p_out, 1 <= p_in, p_out <= P_max of the handle.  M2L is the
 * double-height kernel (Sec. 2.1, eq. m2lkernels, right): every output
 * coefficient depends on every input coefficient.
 *
 * -------------------------------------------------------------- semantics
 * All pointers passed to the *_batch / *_lists calls are DEVICE pointers; the
 * caller owns every array and keeps it alive until the stream reaches the
 * work.  Calls enqueue work on `stream` and return without synchronising.
 * Host-detectable errors are returned synchronously and enqueue nothing;
 * errors found by a kernel are recorded in the handle's device status word,
 * read (and cleared) by sfmm_sync_status().  No C++ exception crosses this
 * interface.  A handle is immutable after sfmm_create and may be used from
 * several host threads and streams at once (Sec. 1.1, thread safe).
 * count = 0 is a no-op returning SFMM_OK.
 */
#ifndef SFMM_H
#define SFMM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *sfmm_stream; /* = cudaStream_t; NULL = legacy default stream */

typedef struct sfmm_ctx *sfmm_handle;

typedef enum { SFMM_F32 = 0, SFMM_F64 = 1 } sfmm_dtype;

typedef enum {
    SFMM_OK = 0,
    SFMM_ERR_ARG = 1,          /* null pointer, negative count, bad enum       */
    SFMM_ERR_ORDER = 2,        /* p_in / p_out outside [1, P_max]              */
    SFMM_ERR_NOMEM = 3,        /* device or host allocation failed             */
    SFMM_ERR_CUDA = 4,         /* a CUDA runtime call failed                   */
    SFMM_ERR_TIMEOUT = 5,      /* a bounded device wait gave up                */
    SFMM_ERR_UNSUPPORTED = 6,  /* valid request this build cannot serve        */
    SFMM_ERR_DEVICE = 7        /* a kernel rejected its input (status word)    */
} sfmm_status;

typedef enum { SFMM_M2M = 0, SFMM_M2L = 1, SFMM_L2L = 2 } sfmm_op;

/* Human-readable name of a status code (static storage, never NULL). */
const char *sfmm_status_string(sfmm_status s);

/*
 * Precomputation (Sec. 3.1): build the tables for orders up to P_max on the
 * current CUDA device and return a handle owning them.
 *   - Dehnen's swap matrices B_n (Appendix recurrence, computed exactly: every
 *     entry is an integer over 2^n), brought to the orthonormal basis
 *     Rhat = R sqrt((n-m)!(n+m)!), Shat = S / sqrt((n-m)!(n+m)!), where one
 *     symmetric orthogonal matrix serves both the M and the L side, then
 *     reduced to the real chequerboard matrices F_n, G_n (eq. FGmappings,
 *     Fig. 2) and packed without their structural zeros;
 *   - the z-axis translation matrices of M2L (eq. zm2l-matrix, factorials),
 *     M2M and L2L in the same basis.
 * 1 <= P_max <= 64 for SFMM_F64; 1 <= P_max <= 30 for SFMM_F32 (the orders
 * of the paper's workloads; FP32 coefficients of unit-sized boxes stay in
 * range there, whereas coefficients of boxes much smaller or larger than the
 * shift unit leave the FP32 range at high order whatever the algorithm, since
 * R_n^m ~ r^n / (n+m)! and S_n^m ~ (n-m)!/r^(n+1)).  Also allocates the
 * handle's global scratch (see sfmm_reserve_scratch): 2 P_max (P_max + 1)
 * reals per lane for 8 warps per SM, e.g. 29 MB at P_max = 10 and 1.3 GB at
 * P_max = 64 in FP64 on 152 SMs.  Synchronous.
 * Errors: SFMM_ERR_ARG (out == NULL, bad dtype), SFMM_ERR_ORDER (P_max),
 * SFMM_ERR_NOMEM, SFMM_ERR_CUDA.  On error *out is set to NULL.
 */
sfmm_status sfmm_create(int P_max, sfmm_dtype dtype, sfmm_handle *out);

/* Release a handle (synchronises the device first).  NULL is accepted. */
sfmm_status sfmm_destroy(sfmm_handle h);

/* P_max and dtype of a handle (either output pointer may be NULL). */
sfmm_status sfmm_get_info(sfmm_handle h, int *P_max, sfmm_dtype *dtype);

/*
 * Batched translations (Sec. 3.4 for M2L; M2M and L2L are the variants the
 * paper implements but does not print, Sec. 1.2).  For i < count:
 *   out[i]  = T(in[i], shift[3i..3i+2])          (accumulate == 0)
 *   out[i] += T(in[i], shift[3i..3i+2])          (accumulate != 0)
 * with T = M2M, M2L or L2L from order p_in to order p_out:
 *   M2M: M'_n^m = sum_{k<=n} sum_l M_k^l R_{n-k}^{m-l}(-r)
 *   M2L: L_n^m  = (-1)^n sum_{k<p_in} sum_l conj(M_k^l) S_{n+k}^{m+l}(r)
 *   L2L: L'_n^m = sum_{k>=n} sum_l L_k^l conj(R_{k-n}^{l-m}(r))
 * in  : device array of `count` device pointers, each to a solid of order p_in
 * out : device array of `count` device pointers, each to a solid of order p_out;
 *       within one call the out[i] must not overlap each other or any in[j]
 *       (each output receives exactly one result per call).
 * shift: device array of 3*count reals (handle dtype), r = new - old centre.
 * Solids must be aligned to the element size.  One GPU thread computes one
 * translation; results do not depend on the batch they are computed in.
 * Errors: SFMM_ERR_ARG, SFMM_ERR_ORDER, SFMM_ERR_UNSUPPORTED, SFMM_ERR_CUDA.
 */
sfmm_status sfmm_m2m_batch(sfmm_handle h, const void *const *in, void *const *out,
                           const void *shift, int p_in, int p_out, long long count,
                           int accumulate, sfmm_stream stream);
sfmm_status sfmm_m2l_batch(sfmm_handle h, const void *const *in, void *const *out,
                           const void *shift, int p_in, int p_out, long long count,
                           int accumulate, sfmm_stream stream);
sfmm_status sfmm_l2l_batch(sfmm_handle h, const void *const *in, void *const *out,
                           const void *shift, int p_in, int p_out, long long count,
                           int accumulate, sfmm_stream stream);

/*
 * Interaction lists (target-major CSR), the form an FMM pass uses: for every
 * target t < n_targets,
 *   out[t] (+)= sum_{j = offsets[t]}^{offsets[t+1]-1} T(src[j], shift[3j..3j+2])
 * summed in a fixed order that depends only on the lists and the handle's
 * policy (deterministic: the same lists give bitwise the same result on every
 * run).  With accumulate == 0 out[t] is overwritten (a target with an empty
 * list receives zeros).
 * src    : device array of nnz = offsets[n_targets] device pointers (order p_in)
 * shift  : device array of 3*nnz reals, r = target centre - source centre
 * offsets: device array of n_targets+1 non-decreasing long long, offsets[0] = 0
 * out    : device array of n_targets distinct device pointers (order p_out),
 *          not overlapping any source
 * Work split: G lanes share a target (G = 32 for M2L, 8 for M2M and L2L), so
 * a list of length L costs ceil(L / G) translations on the critical path.
 * Lane i of a group sums the sources j = offsets[t] + i, + i + G, ... in
 * order, and the G partial sums are added in lane order (the unrolled
 * kernels add the G lanes' results round by round instead).  The generic
 * kernels keep a lane's partial sum in the handle's global scratch; under
 * SFMM_POLICY_SHARED, or when the scratch has no room for the orders, one
 * thread walks each whole list in order.  Targets whose lists have similar
 * lengths should be adjacent (the FMM planner sorts them by length).
 * Errors: as for the batch calls.
 */
sfmm_status sfmm_translate_lists(sfmm_handle h, sfmm_op op, const void *const *src,
                                 const void *shift, const long long *offsets,
                                 void *const *out, int p_in, int p_out,
                                 long long n_targets, int accumulate, sfmm_stream stream);

/*
 * Mixed-order lists in one launch (Sec. 1.1, mixed-order translations, as
 * used by adaptive variable-order FMMs).  One persistent launch serves several
 * classes of target-major lists that share one CSR (src, shift, offsets, out
 * as in sfmm_translate_lists): class k applies op_k from order p_in_k to
 * p_out_k to the targets [target_begin_k, target_end_k).  Classes may come in
 * any order and must not overlap.  Class k spreads each list over
 * lanes_per_target_k lanes and sums in the fixed order that
 * sfmm_translate_lists uses for that many lanes (1: one thread walks the list
 * in order).  Work is dealt to warps in chunks of 32 / lanes_per_target
 * targets of one class.  The rotated solids (and the lanes' partial sums)
 * live in the handle's global scratch, which must hold one slot for the
 * largest orders of the call (sfmm_reserve_scratch).  classes is a HOST
 * array (copied into the launch); 1 <= n_classes <= SFMM_MAX_CLASSES.
 * Errors: SFMM_ERR_ARG, SFMM_ERR_ORDER, SFMM_ERR_UNSUPPORTED (no scratch),
 * SFMM_ERR_CUDA.
 */
#define SFMM_MAX_CLASSES 256
typedef struct {
    int op;                   /* sfmm_op */
    int p_in, p_out;
    int lanes_per_target;     /* 0 (32 for M2L, 8 for M2M, L2L), 1, 2, 4, 8, 16 or 32 */
    long long target_begin;   /* first target of the class */
    long long target_end;     /* one past the last */
} sfmm_list_class;

sfmm_status sfmm_translate_lists_multi(sfmm_handle h, const sfmm_list_class *classes,
                                       int n_classes, const void *const *src,
                                       const void *shift, const long long *offsets,
                                       void *const *out, int accumulate, sfmm_stream stream);

/*
 * A whole translation pass in one persistent launch (Sec. 1.1: M2M, M2L and
 * L2L of mixed orders are the operations of an FMM pass; an adaptive pass is
 * M2M level by level, the M2L lists, L2L level by level).  Each class is one
 * (op, p_in, p_out) applied to its own target-major lists, with the semantics
 * of sfmm_translate_lists for those arrays (src: nnz device pointers to solids
 * of order p_in; shift: 3 nnz reals, r = target centre - source centre;
 * offsets: n_targets + 1 non-decreasing long long; out: n_targets distinct
 * device pointers to solids of order p_out; accumulate as there;
 * lanes_per_target as in sfmm_list_class).  Classes carry a phase number and
 * come in non-decreasing phase order: every class of phase k starts only after
 * every class of the phases before it has finished (so a phase may read what
 * earlier phases wrote), while the classes of one phase run concurrently and
 * must not write the same target.  The launch is cooperative: all its CTAs
 * are resident, and they meet at a grid barrier between phases; a barrier
 * that is not reached within 2 s sets bit 32 of the status word
 * (sfmm_sync_status) and the launch ends.  Rotated solids and partial sums
 * live in the handle's global scratch, which must hold one slot for the
 * largest orders (sfmm_reserve_scratch).  classes is a HOST array (copied into
 * the launch).  1 <= n_classes <= SFMM_MAX_PASS_CLASSES, at most
 * SFMM_MAX_PASS_PHASES distinct phases.
 * Errors: SFMM_ERR_ARG, SFMM_ERR_ORDER, SFMM_ERR_UNSUPPORTED (no scratch, too
 * many phases), SFMM_ERR_CUDA (including a device that cannot run the
 * cooperative launch).
 */
#define SFMM_MAX_PASS_CLASSES 320
#define SFMM_MAX_PASS_PHASES 64
typedef struct {
    int op;                   /* sfmm_op */
    int p_in, p_out;
    int lanes_per_target;     /* 0 (32 for M2L, 8 for M2M, L2L), 1, 2, 4, 8, 16 or 32 */
    int phase;                /* non-decreasing over the classes of a call */
    int accumulate;
    long long n_targets;
    const void *const *src;
    const void *shift;
    const long long *offsets;
    void *const *out;
} sfmm_pass_class;

sfmm_status sfmm_translate_pass(sfmm_handle h, const sfmm_pass_class *classes, int n_classes,
                                sfmm_stream stream);

/*
 * Launch policies (the tile-size choice of Sec. 3.2, made per order on the
 * GPU): which kernel variant serves (op, p_in, p_out) on this handle and how
 * many warps a block has (0 = automatic).
 *   SFMM_POLICY_AUTO     - built-in choice: unrolled if compiled (not for
 *                          FP64 batch calls of order 12, where the generic
 *                          kernel below is faster); batch calls
 *                          the warp-cooperative kernel for FP32 M2L of orders
 *                          16..31, FP32 M2M / L2L of orders 22..31 and FP64
 *                          M2L of orders 30..31; else shared
 *                          memory while enough warps fit per SM (FP64: two
 *                          blocks of two or more warps; FP32: eight warps);
 *                          else the global scratch (launches that use
 *                          the scratch of one handle run one after another,
 *                          whatever their streams, through an event of the
 *                          handle; launches captured into a CUDA graph skip
 *                          that event, so a captured graph is not ordered
 *                          against other work on the same handle: give each
 *                          graph a handle of its own)
 *   SFMM_POLICY_UNROLLED - fixed-order kernel; only p_in = p_out <= 12
 *   SFMM_POLICY_SHARED   - generic kernel, working set in shared memory
 *   SFMM_POLICY_GLOBAL   - generic kernel, rotated solid in the global scratch
 *   SFMM_POLICY_WIDE     - warp-cooperative kernel (a warp translates 4 FP32 or
 *                          2 FP64 solids together, its lanes splitting every
 *                          row and column of Sec. 3.4 by coefficient index);
 *                          batch calls with max(p_in, p_out) <= 31 only (lists
 *                          calls take the AUTO choice)
 * Set policies before launching work with the handle (the table is not
 * synchronised against concurrent launches).  Errors: SFMM_ERR_ARG,
 * SFMM_ERR_ORDER, SFMM_ERR_UNSUPPORTED (variant cannot serve these orders).
 */
typedef enum {
    SFMM_POLICY_AUTO = 0,
    SFMM_POLICY_UNROLLED = 1,
    SFMM_POLICY_SHARED = 2,
    SFMM_POLICY_GLOBAL = 3,
    SFMM_POLICY_WIDE = 4
} sfmm_policy;

sfmm_status sfmm_set_policy(sfmm_handle h, sfmm_op op, int p_in, int p_out,
                            sfmm_policy policy, int warps_per_block);

/*
 * Allocate (or grow) the handle's global scratch so that the global-scratch
 * variants can serve orders up to p_in_max with eight resident warps per SM:
 * 2 p_in_max (p_in_max + 1) reals per lane, a rotated solid and a partial
 * output sum (sfmm_create reserves it for P_max).  Synchronous; not to be
 * called while work using the handle is in flight.  Errors: SFMM_ERR_ARG,
 * SFMM_ERR_ORDER, SFMM_ERR_NOMEM.
 */
sfmm_status sfmm_reserve_scratch(sfmm_handle h, int p_in_max);

/*
 * Shift-grouped M2L on one level of a uniform octree, on the tensor cores.
 * The paper notes that with a finite set of shift vectors the translation
 * matrices can be stored and applied to many solids at once as BLAS
 * matrix-matrix products (Sec. 2.2).  On a uniform level the M2L shifts of the
 * standard interaction list are the 316 integer offsets u (box units,
 * max|u_i| in {2,3}); for P = 16 each has one real 256x256 matrix in the
 * box-scaled orthonormal basis, built once (in FP64, with this library's
 * rotation-based M2L applied to the basis vectors) by sfmm_grid_create, which
 * also allocates the workspaces (synchronous).
 * sfmm_grid_m2l: L (+)= M2L of every box's interaction list on an nside^3 grid
 * (nside a multiple of 8, box i at (ix*nside + iy)*nside + iz, solids of order
 * 16 stored contiguously, FP64 device arrays M and L).  Operands are split
 * into two FP16 parts (hi + lo, 22 significant bits; operator rows and the
 * call's sources each scaled by a power of two into the FP16 range, undone
 * exactly on output) and multiplied as three products with FP32 accumulation
 * over 2 offsets, then added into float-float sums per target (about 48
 * bits) and written once in FP64: every target within 1e-5 (weighted
 * coefficient error) of the FP64 rotation path, and the same result on every
 * run.  Asynchronous on `stream`; one call at a time per grid object.  A
 * device-side wait that gives up sets bit 4 of the handle's status word
 * (sfmm_sync_status); bit 8 means that, after such a time-out, copies or MMAs
 * already issued did not finish within 2 s either (the kernel then keeps its
 * tensor memory allocated); bit 16 means the kernel found its shared memory
 * misaligned for its 128-byte swizzled tiles and did nothing.
 * Errors: SFMM_ERR_ARG, SFMM_ERR_ORDER (handle not FP64 or P_max < 16),
 * SFMM_ERR_UNSUPPORTED (P != 16), SFMM_ERR_NOMEM, SFMM_ERR_CUDA.
 * sfmm_grid_inject_timeout: fault injection for tests of the time-out path.
 * With after_chunks > 0, the copy thread of every CTA of the following calls
 * acts as if its wait for a free pipeline stage had timed out once it has
 * issued that many operand chunks: the kernel then takes its time-out path
 * (status bit 4, the MMA and epilogue roles give up, bounded drain of the
 * copies and MMAs in flight, tensor memory freed) and the call's result is
 * undefined.  after_chunks = 0 turns the injection off.  No GPU fault is
 * involved: the injected time-out is the host's request.  Errors: SFMM_ERR_ARG.
 */
typedef struct sfmm_grid_ctx *sfmm_grid;
sfmm_status sfmm_grid_create(sfmm_handle h, int P, int nside, sfmm_grid *out);
sfmm_status sfmm_grid_m2l(sfmm_grid g, double box_size, const void *M, void *L, int accumulate,
                          sfmm_stream stream);
sfmm_status sfmm_grid_destroy(sfmm_grid g);
sfmm_status sfmm_grid_inject_timeout(sfmm_grid g, long long after_chunks);

/*
 * Particle-to-expansion helpers (not part of the paper's translation library;
 * they build inputs on the device).  Points are sorted by box: box b owns
 * points [offsets[b], offsets[b+1]).  For every box b < n_boxes:
 *   P2M: out_b = sum_j q_j R_n^m(y_j - centre_b)   (multipole, order P)
 *   P2L: out_b = sum_j q_j S_n^m(y_j - centre_b)   (local, order P)
 * (eq. MLexpansions with the addition theorem 1/|x-y| = sum R(y) conj(S(x))).
 * points: device, 3*N reals; q: device, N reals; offsets: device, n_boxes+1;
 * centres: device, 3*n_boxes reals; out: device, n_boxes solids of order P
 * stored contiguously with stride P(P+1) reals (overwritten).
 */
sfmm_status sfmm_p2m_boxes(sfmm_handle h, int P, const void *points, const void *q,
                           const long long *offsets, const void *centres, void *out,
                           long long n_boxes, sfmm_stream stream);
sfmm_status sfmm_p2l_boxes(sfmm_handle h, int P, const void *points, const void *q,
                           const long long *offsets, const void *centres, void *out,
                           long long n_boxes, sfmm_stream stream);

/*
 * Read and clear the handle's device status word after `stream` has drained
 * (synchronises the stream).  *device_status receives the raw word (0 = no
 * kernel reported an error); returns SFMM_ERR_DEVICE if it was non-zero.
 */
sfmm_status sfmm_sync_status(sfmm_handle h, sfmm_stream stream, int *device_status);

/*
 * Batched translations that allocate nothing (the paper has no counterpart;
 * this is an interface for callers that cannot allocate device memory where
 * they translate: a plug-in inside a host framework that hands out a fixed
 * device-memory budget and owns every allocation, or a real-time loop where
 * cudaMalloc/cudaFree and the device synchronisation they imply are not
 * allowed).  Same arguments and results as sfmm_m2m/m2l/l2l_batch with the
 * op selected by `op`, computed by the global-scratch variant of the batch
 * kernel whose scratch is a fixed 16 MiB device array inside the library
 * (held by every GPU that loads the library until the process exits) instead
 * of memory owned by the handle.  It calls no cudaMalloc, cudaFree or other
 * allocating routine.
 * Limits: p_in, p_out in [1, P_max] (else SFMM_ERR_ORDER); one warp's slot of
 * 32 p_in (p_in+1) reals must fit in the 16 MiB array, which holds for every
 * order a handle accepts (else SFMM_ERR_UNSUPPORTED); fewer warps run at once
 * when p_in is large, any count is served.
 * Set-up: the first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current and caches it; make that
 * first call before any stream capture.  The current device must be the
 * handle's device (else SFMM_ERR_ARG).
 * Sharing: every call on a device uses the same array, which keeps the last
 * call's contents (each thread overwrites its whole slot before reading it, so
 * nothing needs clearing).  Calls whose kernels overlap on the GPU (different
 * streams, any handle) race on the array: order them on one stream or with
 * events.
 */
sfmm_status sfmm_translate_batch_noalloc(sfmm_handle h, sfmm_op op, const void *const *in,
                                         void *const *out, const void *shift, int p_in,
                                         int p_out, long long count, int accumulate,
                                         sfmm_stream stream);

/*
 * Host-side introspection of the precomputed tables (no GPU, no handle).
 * sfmm_host_swap_matrices: the dense reduced swap matrices F_n and G_n of
 * eq. FGmappings in the orthonormal basis (row m, column l, (n+1)^2 doubles
 * each; the chequerboard zeros of Fig. 2 are stored as exact zeros), the
 * matrices every swap step of every translation applies.  0 <= n <= 63.
 * sfmm_host_ztranslate: the dense z-axis translation block of column m for op
 * at order P ((P-m)^2 doubles, row n-m, column k-m, orthonormal basis; for M2L
 * eq. zm2lkernels (double height) with factorials (n+k)!, eq. zm2l-matrix).
 * Errors: SFMM_ERR_ARG (null output, bad op), SFMM_ERR_ORDER (n, P, m range).
 */
sfmm_status sfmm_host_swap_matrices(int n, double *F, double *G);
sfmm_status sfmm_host_ztranslate(sfmm_op op, int P, int m, double *T);

#ifdef __cplusplus
}
#endif

#endif /* SFMM_H */
