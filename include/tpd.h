/*
 * tpd.h -- C ABI of libtpd.so: the tensorized Pauli decomposition
 * (Hantzko, Binkowski, Gupta, arXiv:2310.13421) on one GB300 GPU.
 *
 * What is computed.  For A in Mat(2^n), the Pauli weights (Sec. II.A, Eq. 2)
 *
 *     w_t = 2^-n tr(sigma^t A),     t in {0,1,2,3}^n = {I,X,Y,Z}^n,
 *
 * by the paper's cumulative matrix weights (Eq. 4): for every qubit the four
 * blocks A11, A12, A21, A22 of a 2x2 block partition become
 *     I: (A11 + A22)/2,  X: (A12 + A21)/2,  Y: i (A12 - A21)/2,  Z: (A11 - A22)/2,
 * and by Eq. 5 applying this to all qubits yields the scalars w_t (Sec. III).
 *
 * Conventions used by every entry point.
 *  - Matrices are dense, row-major, N x N with N = 2^n, complex interleaved
 *    (re, im): complex128 = two doubles, complex64 = two floats.
 *  - Qubit j = 1..n (tensor factor j of Eq. 1) is row/column index bit n-j:
 *    the first factor picks the quadrant of Eq. 3.
 *  - Results are written IN PLACE in "RC layout": the weight of string t sits
 *    at the flat position r*N + c whose row bit r_{n-j} and column bit c_{n-j}
 *    satisfy t_j = 2 r_{n-j} + c_{n-j}  (I at (0,0), X at (0,1), Y at (1,0),
 *    Z at (1,1) of each qubit's 2x2 block, exactly where Eq. 4 puts them).
 *  - All pointers passed as "device" must be device memory of the current
 *    CUDA device, owned by the caller; the library never allocates, frees or
 *    retains them.  All work is enqueued asynchronously on `stream`
 *    (a cudaStream_t, NULL = legacy default stream).
 *  - Every argument is checked before anything is enqueued; on error nothing
 *    is launched and the buffer is untouched.  No entry point traps, asserts
 *    on the device or waits without a bound.
 *  - Status codes are returned; tpd_status_string() names them.
 */
#ifndef TPD_H_
#define TPD_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  TPD_OK = 0,
  TPD_ERR_INVALID_ARG = 1,  /* bad n, dtype, precision, count, null pointer */
  TPD_ERR_UNSUPPORTED = 2,  /* combination not implemented (COMPENSATED with C128, zero
                               skipping in batched or partial calls) */
  TPD_ERR_MISALIGNED = 3,   /* pointer not aligned to the element size */
  TPD_ERR_WORKSPACE = 4,    /* workspace missing or smaller than *_workspace_size() */
  TPD_ERR_CUDA = 5,         /* a CUDA call failed (launch error, no device, ...) */
  TPD_ERR_TIMEOUT = 6       /* a bounded device-side wait gave up (batched path) */
} tpd_status;

typedef enum {
  TPD_C128 = 0,             /* complex128 storage (16 bytes per element) */
  TPD_C64 = 1               /* complex64 storage (8 bytes per element) */
} tpd_dtype;

/* Arithmetic of the butterfly.  Every mode applies Eq. 4 level by level; they
 * differ only in how the sums are rounded. */
typedef enum {
  TPD_PREC_DEFAULT = 0,      /* C128 -> TPD_PREC_FIXED, C64 -> TPD_PREC_PLAIN */
  TPD_PREC_PLAIN = 1,        /* IEEE adds in the storage precision (fp64 / fp32),
                                rounded after every level as in the paper */
  TPD_PREC_COMPENSATED = 2,  /* C64 only: fp32 sums carried with TwoSum error terms
                                (Ogita-Rump-Oishi cascaded summation) across the
                                levels of a pass, one rounding per pass */
  TPD_PREC_FIXED = 3         /* block fixed point: a pass of K levels only adds
                                elements of one "class" (the same X-mask on its
                                levels, Eq. 4, and the same other column bits);
                                each class is put on its own binary point, its
                                2^K-term sums are exact in 64-bit integers, and
                                every output is rounded to the storage type once
                                per pass (round to nearest even).  A component
                                is truncated (toward zero) only where it lies far
                                below its class's largest: the error stays below
                                2^(K-61) of that largest.  So a weight's error is
                                set by its own X-mask's entries, as in IEEE
                                arithmetic, never by larger entries elsewhere in
                                the matrix, and Hermitian inputs give exactly real
                                weights.  Whole complex64 matrices of n <= 4 run
                                the compensated kernel */
} tpd_precision;

typedef struct {
  int precision;    /* tpd_precision */
  int skip_zero;    /* 1: skip all-zero tiles exactly (the zero-CMW pruning of
                       Alg. 1/2: Omega = 0 implies all its weights are 0).
                       Needs a workspace of tpd_workspace_size() bytes. */
  int tile_bits;    /* 0 = planner default; otherwise log2 of the elements in a
                       tile (9..13), for tuning */
  int max_levels;   /* 0 = planner default; otherwise the most qubit levels fused
                       into one pass (1..6), for tuning */
  int variant;      /* kernel form, for tuning: 0 = default (a single complex128
                       matrix without zero skipping or partial masks runs the
                       block fixed point's first pass, and the 2^11-element
                       last pass of n = 15, as persistent CTAs, two per SM,
                       each copying its next tile into shared memory while it
                       finishes the current one), 1 = one CTA per tile
                       (complex128 tiles of 2^13 elements otherwise run as a
                       cluster of two 256-thread CTAs sharing the tile through
                       distributed shared memory),
                       2 = persistent CTAs that prefetch the next tile (complex128
                       block fixed point, single matrix, no zero skipping),
                       3 / 4 = one CTA per tile compiled for 2 / 3 CTAs per SM
                       (tiles of up to 2^12 elements),
                       5 = one CTA per tile with every pass's tile layout read
                       from its run-time descriptor (by default, passes whose
                       layout is one of the library's compiled shapes run a
                       kernel with that layout built in; all forms give
                       identical results).
                       Batched calls: 0, 1, 3, 4 = one launch per (qubit count,
                       pass) over all matrices of that qubit count (the fastest
                       form measured on GB300); 2 = the whole batch in ONE
                       persistent kernel launch when every matrix has n <= 6 or
                       a plan of 2^12-element tiles (else as 0) */
  void** pass_events; /* profiling, may be NULL: num_events cudaEvent_t handles
                       (created by the caller); tpd_decompose / tpd_compose
                       record event 0 before the first pass and event p+1 after
                       pass p, on `stream`, for p < num_events - 1 (passes run
                       in L2 chunks record their events together after the last
                       of them) */
  int num_events;
  int l2_chunk_mb;  /* single matrices: 0 = off (default), > 0 = chunk size in MB.
                       The first passes whose tiles together leave global bits
                       free run chunk by chunk (the elements agreeing on those
                       bits), so a chunk stays in the GPU's L2 from one pass to
                       the next and HBM sees one read and one write for all of
                       them.  On GB300 the many smaller launches cost more than
                       the traffic saves (n = 14: 6.2 ms with 64 MB chunks
                       against 5.2 ms), hence off by default.  Not with
                       skip_zero, partial masks or variant 2. */
} tpd_options;

/* Zero-initialised defaults (precision DEFAULT, no skip, planner tiles). */
void tpd_options_init(tpd_options* opt);

/* Bytes of device workspace tpd_decompose / tpd_compose need for (n, dtype,
 * opt): what one pass hands to the next besides the matrix itself -- with
 * opt->skip_zero, one nonzero flag byte per tile of every pass after the
 * first.  0 without skip_zero and for one-pass plans.  Returns 0 for invalid
 * arguments. */
size_t tpd_workspace_size(int n, int dtype, const tpd_options* opt);

/* Pauli decomposition in place (Eq. 2 via Eqs. 3-5).
 *   A          device, N*N complex of `dtype`, 16-byte (C128) or 8-byte (C64)
 *              aligned; on return holds 2^-n tr(sigma^t A) in RC layout.
 *   n          qubits, 1 <= n <= 16 (n = 16 C128 is 64 GiB).
 *   opt        may be NULL (defaults).
 *   workspace  device, tpd_workspace_size() bytes, may be NULL when that is 0.
 *   stream     cudaStream_t.
 * Errors: INVALID_ARG, UNSUPPORTED, MISALIGNED, WORKSPACE, CUDA. */
tpd_status tpd_decompose(void* A, int n, int dtype, const tpd_options* opt,
                         void* workspace, size_t workspace_bytes, void* stream);

/* Pauli composition in place: C holds weights w_t in RC layout, on return it
 * holds  scale * sum_t w_t sigma^t  (Eq. 2, left side).  With scale = 2^-n
 * this is the adjoint of tpd_decompose (the Pauli strings are Hermitian, so
 * the decomposition's adjoint is 2^-n times composition).  Per qubit:
 * a00 = I + Z, a01 = X - iY, a10 = X + iY, a11 = I - Z.
 * Arguments as tpd_decompose; scale must be finite and nonzero.  A scale that
 * is a power of two is applied exactly. */
tpd_status tpd_compose(void* C, int n, int dtype, double scale, const tpd_options* opt,
                       void* workspace, size_t workspace_bytes, void* stream);

/* End to end from host memory: copy A_host (N*N complex of `dtype`, host,
 * ideally pinned) into the caller's device buffer dev_A (device, N*N elements,
 * aligned as for tpd_decompose), decompose it in place, and copy the weights
 * (RC layout) back into W_host (host; may equal A_host).  All three steps are
 * enqueued on `stream` and the call returns without waiting; the host buffers
 * must stay valid until the stream reaches this point.
 * Errors as tpd_decompose; host pointers must be non-NULL. */
tpd_status tpd_decompose_host(const void* A_host, void* W_host, void* dev_A, int n, int dtype,
                              const tpd_options* opt, void* workspace, size_t workspace_bytes,
                              void* stream);

/* Decomposition for callers that cannot allocate device memory.
 *
 * The paper has no counterpart: this entry point exists for callers that may
 * not call cudaMalloc or an allocating library -- for instance code running
 * where a custom allocator owns all device memory, or a real-time path that
 * must not allocate or synchronise.  It behaves like tpd_decompose, but its
 * workspace (the per-class binary points of the complex128 block fixed point
 * and the zero-skip flags that passes hand to one another) is a fixed array
 * of TPD_NOALLOC_SCRATCH_BYTES in the library's own device memory, present on
 * every GPU that loads the library until the process exits; the default
 * complex128 plans fit up to n = 14 (40 MiB at n = 14).  The caller still
 * passes the matrix A (device, in place).
 *   - Plans whose workspace (tpd_workspace_size) exceeds the array are
 *     rejected with TPD_ERR_WORKSPACE before anything is enqueued; use
 *     tpd_decompose with a caller buffer for those.
 *   - The first call on a device looks up the array's device address with
 *     that device current.  That look-up loads the library's device code for
 *     this entry point, and with CUDA's lazy module loading (the default) the
 *     array is allocated by the CUDA runtime at that moment: make one call on
 *     each device (any n, e.g. n = 1) before any stream capture and before the
 *     point from which nothing may be allocated.  Later calls allocate nothing.
 *   - All calls on a device share the one array, and a call leaves its
 *     contents behind (each call clears what it needs cleared).  Calls whose
 *     work overlaps on the GPU (different streams, no ordering) race on it.
 *   - Nothing is allocated or freed after that first call, by the library or
 *     by a library it calls.
 * Arguments and other errors as tpd_decompose. */
#define TPD_NOALLOC_SCRATCH_BYTES ((size_t)64 << 20)
tpd_status tpd_decompose_noalloc(void* A, int n, int dtype, const tpd_options* opt, void* stream);

/* Device workspace for the batched calls over `count` matrices with qubit
 * counts ns[0..count) (host array). Returns 0 for invalid arguments. */
size_t tpd_batched_workspace_size(const int* ns, int count, int dtype, const tpd_options* opt);

/* Batched decomposition in place of `count` independent matrices.
 *   ptrs_dev   device array of `count` device pointers (matrix i at ptrs_dev[i]).
 *   ns_dev     device array of `count` ints, ns_dev[i] = n_i (same values as ns).
 *   ns         host array of the same n_i, 1 <= n_i <= 12, used for planning.
 *   workspace  device, tpd_batched_workspace_size() bytes (required).  Its
 *              first bytes hold the status word read by tpd_batch_status.
 * The matrices must not overlap.  The enqueued work (a memset of the control
 * words and the kernel launches) depends only on the arguments (no host
 * synchronisation), so it can be captured in a CUDA graph.  By default one
 * kernel launch per (qubit count, pass) covers all matrices of that qubit
 * count; with tpd_options.variant = 2 the whole batch runs in ONE persistent
 * kernel launch: CTAs claim tiles in order, and a tile of a later pass waits,
 * with a bound, for the tiles of its own matrix's previous pass.  A wait that
 * gives up, or ns_dev disagreeing with ns, is reported by tpd_batch_status
 * (the results are then invalid; with ns_dev inconsistent nothing is
 * touched).  No device-side wait is unbounded. */
tpd_status tpd_decompose_batched(void* const* ptrs_dev, const int* ns_dev, const int* ns,
                                 int count, int dtype, const tpd_options* opt,
                                 void* workspace, size_t workspace_bytes, void* stream);

/* Batched composition, scale_mode 0: scale 1, scale_mode 1: scale 2^-n_i
 * (the adjoint of tpd_decompose_batched).  Arguments as above. */
tpd_status tpd_compose_batched(void* const* ptrs_dev, const int* ns_dev, const int* ns,
                               int count, int dtype, int scale_mode, const tpd_options* opt,
                               void* workspace, size_t workspace_bytes, void* stream);

/* Partial decomposition (Alg. 3, Sec. III): only the weights of a given list
 * of strings -- the paper's quaternary subtree T of the strings of interest.
 * Two steps, because the first is host work:
 *
 * tpd_partial_prepare  computes, on the host, which tiles of which pass the
 *   requested weights depend on and uploads that, with the strings' RC
 *   positions, into `workspace` (device, tpd_partial_workspace_size() bytes).
 *   strings: host array of `count` base-4 string indices
 *   s = sum_j t_j 4^(n-j) (t_1 most significant, I=0 X=1 Y=2 Z=3), each
 *   < 4^n; duplicates allowed.  Synchronises `stream` (the host arrays are
 *   temporary), so call it outside stream capture.
 * tpd_decompose_partial  runs the passes on A in place, each skipping the
 *   tiles no requested weight depends on, and gathers the requested weights,
 *   in request order, into `weights` (device, count elements of `dtype`).
 *   Afterwards A holds the requested weights at their RC positions; its other
 *   elements are unspecified.  The same (n, dtype, opt, count) as the prepare
 *   call, and the workspace it filled; the call enqueues only, so it can be
 *   captured in a CUDA graph and repeated.
 * A weight depends on the positions whose already-applied levels hold its
 * symbols and whose later levels lie on its quads' diagonal (I, Z) or
 * anti-diagonal (X, Y) (Eq. 4); every pass skips the tiles holding none of
 * them (2^(levels after the pass) tile ids per string at most).  The
 * requested weights equal those of tpd_decompose with the same options bit
 * for bit, for finite inputs, in every precision (in the block fixed point
 * the elements a requested weight's class sums lie in its dependency cone, so
 * skipped tiles never enter its binary point).
 * opt->skip_zero is not supported (TPD_ERR_UNSUPPORTED).
 * Errors: as tpd_decompose; INVALID_ARG also for a string index >= 4^n. */
size_t tpd_partial_workspace_size(int n, int dtype, const tpd_options* opt, size_t count);
tpd_status tpd_partial_prepare(int n, int dtype, const tpd_options* opt, const unsigned long long* strings,
                               size_t count, void* workspace, size_t workspace_bytes, void* stream);
tpd_status tpd_decompose_partial(void* A, int n, int dtype, const tpd_options* opt, size_t count, void* workspace,
                                 size_t workspace_bytes, void* weights, void* stream);

/* The paper's output form (Alg. 1 and 2 return the list L of strings with a
 * nonzero weight): from weights W in RC layout (device, N*N of `dtype`, as a
 * decomposition leaves them), the entries with |Re w| > tol or |Im w| > tol
 * (tol = 0: the exact "nonzero" of the paper; NaN is kept), in increasing
 * base-4 string index s = sum_j t_j 4^(n-j) (t_1 most significant).
 *   strings   device, capacity uint64: the string indices.
 *   weights   device, capacity elements of `dtype`: their weights.
 *   count     device, one uint64: the number of entries (all of them; only
 *             the first `capacity` are written).
 *   workspace device, tpd_nonzero_workspace_size(n) bytes, 256-byte aligned.
 * The order does not depend on scheduling.  Asynchronous on `stream`.
 * Errors: INVALID_ARG, MISALIGNED, WORKSPACE, CUDA. */
size_t tpd_nonzero_workspace_size(int n);
tpd_status tpd_nonzero_list(const void* W, int n, int dtype, double tol, unsigned long long* strings,
                            void* weights, size_t capacity, unsigned long long* count, void* workspace,
                            size_t workspace_bytes, void* stream);

/* Sparse input (the cost model of Sec. IV: m nonzero entries, p contributing
 * strings): the decomposition of a complex128 matrix given by its nonzero
 * entries, computed level by level as in Alg. 2 -- each entry of a CMW feeds
 * two entries of the next level's CMWs (Eq. 4), equal positions are summed,
 * zero sums are dropped (the zero-CMW pruning) -- and returned as the paper's
 * list L sorted by string index, in the form of tpd_nonzero_list.
 *   rows, cols  device, nnz ints each: 0 <= r, c < 2^n (duplicates are added).
 *   values      device, nnz complex128.
 *   n           1..15.
 *   max_entries the most entries any level may hold (device memory grows with
 *               it: about 52 bytes per entry); more sets *status to
 *               TPD_ERR_WORKSPACE and the list is incomplete.  A level holds
 *               at most 2x the entries of the one before.
 *   strings, weights, capacity, count   as tpd_nonzero_list.
 *   status      device, one unsigned (may be NULL): TPD_OK or TPD_ERR_WORKSPACE.
 *   workspace   device, tpd_sparse_workspace_size(max_entries) bytes, 256-byte aligned.
 * Sums are exact (int64 on one binary point per X-mask r xor c, which no
 * level changes), each weight is rounded once; the result does not depend on
 * scheduling.  Enqueued on
 * `stream` only (no host synchronisation).  C128 only (UNSUPPORTED otherwise).
 * Errors: INVALID_ARG, UNSUPPORTED, MISALIGNED, WORKSPACE, CUDA. */
size_t tpd_sparse_workspace_size(size_t max_entries);
tpd_status tpd_decompose_coo(const int* rows, const int* cols, const void* values, size_t nnz, int n, int dtype,
                             size_t max_entries, unsigned long long* strings, void* weights, size_t capacity,
                             unsigned long long* count, unsigned* status, void* workspace, size_t workspace_bytes,
                             void* stream);

/* Decomposition in the Weyl (clock-and-shift) basis of n qudits of dimension
 * d -- the tensorized basis Sec. V (Conclusion and Outlook) names as the
 * natural next candidate for the method.  With omega = exp(2 pi i / d),
 * X|j> = |j+1 mod d>, Z|j> = omega^j |j> and W_{a,b} = X^a Z^b (a tensor
 * product over the qudits, qudit 1 the most significant base-d digit of the
 * row and column index), it computes in place
 *
 *     c_{a,b} = d^-n tr(W_{a,b}^* A),          A = sum_{a,b} c_{a,b} W_{a,b},
 *
 * by the recursion of Eqs. 3-5 with d x d blocks: each qudit level turns
 * every d x d block into the d^2 cumulative weights
 * Omega_{a,b} = d^-1 sum_c omega^(-b c) A_{c+a, c}.
 *   A       device, d^n x d^n complex of `dtype` (row-major, 16- / 8-byte
 *           aligned); on return the weight c_{a,b} sits at the position whose
 *           row digit of each qudit is b_j and column digit (a_j + b_j) mod d
 *           (for d = 2 the Pauli RC layout, with c_{1,1} = i w_Y since
 *           XZ = -iY).
 *   n, d    1 <= n, 2 <= d <= 5, d^n <= 65536.
 *   dtype   TPD_C128 or TPD_C64.
 *   opt     may be NULL (defaults); only opt->precision is read:
 *           DEFAULT / FIXED: complex128 with d <= 4 in a block fixed point --
 *             the d elements each DFT combines (one cyclic diagonal of a
 *             block) on their own binary point in int64, the DFT exact for
 *             d = 2, 4 and with sqrt(3) rounded once on that grid for d = 3,
 *             one rounding to double per output and level (d = 2, 4 integer
 *             inputs: exact); classes meeting Inf/NaN in IEEE fp64;
 *           PLAIN (and DEFAULT for d = 5): IEEE fp64, rounded every level;
 *           complex64: fp32, rounded every level (FIXED and COMPENSATED are
 *           INVALID_ARG for complex64, FIXED for d = 5).
 * One kernel launch per qudit; no workspace; asynchronous on `stream`.
 * Errors: INVALID_ARG, MISALIGNED, CUDA. */
tpd_status tpd_weyl_decompose(void* A, int n, int d, int dtype, const tpd_options* opt, void* stream);

/* Weyl-basis composition in place: C holds the weights c_{a,b} in the layout
 * tpd_weyl_decompose leaves; on return it holds scale * sum c_{a,b} W_{a,b}
 * (scale = d^-n: the adjoint of tpd_weyl_decompose, W_{a,b} being unitary;
 * applied on the last level, exactly where it is a power of two).  scale
 * finite and nonzero.  Arguments, arithmetic and errors as
 * tpd_weyl_decompose. */
tpd_status tpd_weyl_compose(void* C, int n, int d, int dtype, double scale, const tpd_options* opt,
                            void* stream);

/* Decomposition in the generalized Gell-Mann basis of n qudits of dimension
 * d -- the other tensorized basis Sec. V (Conclusion and Outlook) names as a
 * natural candidate for the method.  One qudit's d^2 Hermitian elements are
 * labelled by a position (r, c) of the d x d grid (E_jk the matrix unit):
 *     (0, 0)           the identity                                   tr(G^2) = d
 *     (l, l), l >= 1   D_l = sqrt(2 / (l (l+1))) (sum_{m<l} E_mm - l E_ll)     2
 *     (j, k), j < k    S_jk = E_jk + E_kj                                       2
 *     (k, j), j < k    A_jk = -i E_jk + i E_kj                                  2
 * (d = 2: I, X, Y, Z at the positions Eq. 4 gives their weights; d = 3:
 * Gell-Mann's lambda_1..lambda_8).  An n-qudit element is the tensor product
 * over the digit pairs of its label (qudit 1 the most significant base-d
 * digit of row and column), N_(r,c) the product of the traces, and in place
 *
 *     g_(r,c) = tr(G_(r,c) A) / N_(r,c),       A = sum_(r,c) g_(r,c) G_(r,c),
 *
 * by the recursion of Eqs. 3-5 with d x d blocks: each qudit level maps every
 * block x to (x_jk + x_kj)/2 at (j, k), i (x_jk - x_kj)/2 at (k, j),
 * c_l/2 (sum_{m<l} x_mm - l x_ll) at (l, l) and (1/d) sum_m x_mm at (0, 0)
 * (c_l = sqrt(2 / (l (l+1)))); for d = 2 this is Eq. 4.
 *   A       device, d^n x d^n complex of `dtype` (row-major, 16- / 8-byte
 *           aligned); on return g_(r,c) sits at row r, column c.
 *   n, d    1 <= n, 2 <= d <= 5, d^n <= 65536.
 *   dtype   TPD_C128 (IEEE fp64) or TPD_C64 (fp32), rounded every level,
 *           no fused multiply-adds: a Hermitian input gives exactly real
 *           coefficients.
 *   opt     may be NULL; opt->precision DEFAULT or PLAIN (the same
 *           arithmetic); FIXED and COMPENSATED are INVALID_ARG.
 * One kernel launch per qudit; no workspace; asynchronous on `stream`.
 * Errors: INVALID_ARG, MISALIGNED, CUDA. */
tpd_status tpd_gellmann_decompose(void* A, int n, int d, int dtype, const tpd_options* opt, void* stream);

/* Generalized Gell-Mann composition in place: C holds g_(r,c) at row r,
 * column c; on return it holds scale * sum g_(r,c) G_(r,c) (scale applied on
 * the last level; scale = 1 inverts tpd_gellmann_decompose).  The adjoint of
 * the decomposition is this composition applied to g_(r,c) / N_(r,c).  scale
 * finite and nonzero.  Arguments, arithmetic and errors as
 * tpd_gellmann_decompose. */
tpd_status tpd_gellmann_compose(void* C, int n, int d, int dtype, double scale, const tpd_options* opt,
                                void* stream);

/* Layout conversion, out of place.  RC is the layout every decomposition
 * leaves (see the conventions above); STRING puts the weight of
 * t = (t_1, ..., t_n) at the base-4 index s = sum_j t_j 4^(n-j) (t_1 most
 * significant; the labelling of Sec. II, Eq. 2), so bit 2b+1 of s is row bit
 * r_b and bit 2b is column bit c_b.
 *   src, dst   device, N*N elements of `dtype` each, aligned as for
 *              tpd_decompose; they must not overlap.
 *   to_string  1: RC -> STRING, 0: STRING -> RC.
 * Errors: INVALID_ARG (n outside 1..16, null, overlap), MISALIGNED, CUDA. */
tpd_status tpd_convert_layout(const void* src, void* dst, int n, int dtype, int to_string, void* stream);

/* Sum of squared magnitudes: *result = sum_i |x_i|^2 over `count` complex
 * elements of `dtype`, accumulated in fp64 in a fixed order (the same bits on
 * every call).  With w the weights of A, Parseval's identity for the
 * orthogonal Pauli basis (tr(sigma^s sigma^t) = 2^n delta_st, Sec. II) gives
 * ||A||_F^2 = 2^n sum_t |w_t|^2: the pair of sums checks a decomposition.
 *   x          device, count elements.  count >= 0 (0 gives 0).
 *   result     device, one double.
 *   workspace  device, TPD_SUMSQ_WORKSPACE_BYTES bytes.
 * Errors: INVALID_ARG, MISALIGNED, WORKSPACE, CUDA. */
#define TPD_SUMSQ_WORKSPACE_BYTES ((size_t)8192)
tpd_status tpd_sum_squares(const void* x, size_t count, int dtype, double* result, void* workspace,
                           size_t workspace_bytes, void* stream);

/* Status of the last batched call that used `workspace` (device): TPD_OK,
 * TPD_ERR_TIMEOUT (a bounded device-side wait gave up), TPD_ERR_INVALID_ARG
 * (ns_dev disagreed with ns), or TPD_ERR_CUDA if the status cannot be read.
 * Waits for `stream` to reach this point (host synchronisation: call it
 * outside stream capture). */
tpd_status tpd_batch_status(const void* workspace, void* stream);

/* Test hook, host only: while `on` is nonzero, batched calls that take the
 * persistent form (variant 2) make every tile of a pass after the first wait for one more
 * completed tile of the previous pass than there are, so each such wait runs
 * into its bound and tpd_batch_status reports TPD_ERR_TIMEOUT.  It exercises
 * the timeout path without any fault; the results of such calls are invalid. */
void tpd_test_hold_batch_waits(int on);

/* Tuned defaults.  Registers tile_bits, max_levels and variant of `tuned`
 * for (n, dtype, precision); every later call for that key whose options
 * leave all three at 0 (or pass opt == NULL) uses them instead of the
 * planner's defaults -- the batched calls per qubit count.  The project's
 * autotuner (paper_2310_13421_gb300/autotune.py) times candidates and sets
 * them.  tuned == NULL removes the entry.  Host only, thread-safe.
 * Errors: INVALID_ARG (bad key or values). */
tpd_status tpd_tune_set(int n, int dtype, int precision, const tpd_options* tuned);

/* Forget every tuned default. */
void tpd_tune_clear(void);

/* Describe the pass plan the library uses for (n, dtype, opt) as a
 * NUL-terminated text (one line per pass: levels, tile bits, tile count, the
 * CTAs per SM its kernel is compiled for, stages) written to buf (at most len
 * bytes).  Host only, no device call.  Returns the number
 * of passes, or -1 on invalid arguments. */
int tpd_plan_describe(int n, int dtype, const tpd_options* opt, char* buf, size_t len);

/* Name of a status code (static string). */
const char* tpd_status_string(int status);

/* Library version: major*10000 + minor*100 + patch. */
int tpd_version(void);

#ifdef __cplusplus
}
#endif

#endif /* TPD_H_ */
