/*
 * rqrcp.h -- C ABI of librqrcp, a GB300 (sm_103a) implementation of randomized QR with
 * column pivoting (RQRCP) from Xiao, Gu, Langou, "Fast parallel randomized QR with column
 * pivoting algorithms for reliable low-rank matrix approximations" (HiPC 2017).
 *
 * Conventions shared by every entry point
 *  - Matrices are column-major: element (i,j) of X with leading dimension ldx is X[j*ldx+i].
 *    Indices are 0-based (the paper is 1-based).
 *  - A sketching matrix Omega is row-major l x m: element (r,q) is Omega[r*ldo+q], ldo >= m.
 *  - Every pointer named A, B, Omega, jpvt, tau, L, Q1, work is a DEVICE pointer on the
 *    current CUDA device, owned by the caller; the library allocates no device memory.
 *    Scratch space comes from `work` (size from rqrcp_workspace_size, 256-byte aligned).
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls only enqueue work;
 *    they return before it runs.  rqrcp_read_status synchronises the stream and reports
 *    device-side failures of the last call that used `work`.
 *  - Return value: 0 on success; -i when the i-th argument (1-based) is invalid, as in
 *    LAPACK's info; a positive RQRCP_ERR_* code otherwise.  Invalid arguments are
 *    rejected before anything is enqueued.
 *  - Calls that share `work` must not overlap on the GPU; distinct work buffers may run
 *    concurrently on distinct streams.
 */
#ifndef RQRCP_H
#define RQRCP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RQRCP_OK 0
#define RQRCP_ERR_CUDA 1        /* a CUDA runtime call failed (launch, memset, sync) */
#define RQRCP_ERR_NONFINITE 2   /* the sketch of A holds NaN or Inf: A is not finite */
#define RQRCP_ERR_TIMEOUT 3     /* a grid-wide barrier inside a kernel gave up waiting */
#define RQRCP_ERR_WORKSPACE 4   /* work is NULL, misaligned or smaller than required */
#define RQRCP_ERR_UNSUPPORTED 5 /* the shape exceeds what the library keeps on chip */

#define RQRCP_PREC_FP64 0  /* plain form: every step in IEEE double */
#define RQRCP_PREC_MIXED 1 /* mixed form: FP32 storage, FP64 reflector generation */

/* Human-readable text for a return code (static string, never NULL). */
const char* rqrcp_error_string(int code);

/*
 * Bytes of scratch that rqrcp_factor / rqrcp_factor_with_omega (precision FP64) or
 * rqrcp_factor_mixed (precision MIXED) need for an m x n problem with target rank k,
 * block size b and oversampling p.  Returns 0 if the arguments are invalid.
 */
size_t rqrcp_workspace_size(int64_t m, int64_t n, int64_t k, int64_t b, int64_t p, int precision);

/*
 * Gaussian sketching matrix of Alg. 2 ("Generate i.i.d Gaussian matrix Omega in
 * N(0,1)^{(b+p) x m}"), drawn on the HOST: rqrcp_generate_omega_host writes Omega (l x m,
 * row-major, ldo >= m) into host memory.  Element with flat index q = r*m + c is lane q%4 of
 * Philox4x64-10 (Salmon et al., SC'11) evaluated at counter (q/4,0,0,0) with key (seed,0);
 * lanes (0,1) and (2,3) are Box-Muller pairs: u1 = ((w0>>11)+1)*2^-53, u2 = (w1>>11)*2^-53,
 * z_even = sqrt(-2 ln u1) cos(2 pi u2), z_odd = sqrt(-2 ln u1) sin(2 pi u2), evaluated in IEEE
 * double with the C library's log, sqrt, cos and sin and no fused multiply-add.  The draw runs
 * on host threads (the bits do not depend on their number).  Every seeded entry point of this
 * library uses exactly this draw (its FP32 form rounds it to float), so a caller holding the
 * same C library reproduces the sketch bit for bit.  Errors: -1 l < 1, -2 m < 1, -4 Omega NULL,
 * -5 ldo < m.
 *
 * rqrcp_generate_omega / rqrcp_generate_omega_f32 write the same draw (FP64, or rounded to FP32)
 * into DEVICE memory on `stream`: one copy from pageable host memory (the last (seed, l, m) draw
 * is kept on the host for reuse).  Such a copy may synchronise the host with the stream and cannot
 * be captured in a CUDA graph; the seeded factorizations below use the same path.
 */
int rqrcp_generate_omega_host(int64_t l, int64_t m, uint64_t seed, double* Omega, int64_t ldo);
int rqrcp_generate_omega(int64_t l, int64_t m, uint64_t seed, double* Omega, int64_t ldo, void* stream);
int rqrcp_generate_omega_f32(int64_t l, int64_t m, uint64_t seed, float* Omega, int64_t ldo, void* stream);

/*
 * Sketch B = Omega A (Alg. 2, "Compute B = Omega A").  A is m x n (lda >= m), Omega is
 * l x m row-major (ldo >= m), B is l x n (ldb >= l).  FP64 throughout.  `work` needs
 * rqrcp_workspace_size(m, n, 1, l, 0, RQRCP_PREC_FP64) bytes.
 */
int rqrcp_sketch(int64_t m, int64_t n, const double* A, int64_t lda, const double* Omega, int64_t l,
                 int64_t ldo, double* B, int64_t ldb, void* work, size_t work_bytes, void* stream);

/*
 * Randomized QRCP, Alg. 2, plain FP64 form, with the sketch drawn from `seed` as in
 * rqrcp_generate_omega.  Requires 1 <= k <= min(m,n), b >= 1, p >= 0, lda >= m.
 * Block by block (block size bb = min(b, k-i)): partial QRCP on the sketch B picks bb
 * pivots, the columns of A are swapped, the panel A(i:m, i:i+bb) gets an unpivoted
 * Householder QR, the trailing columns get the compact-WY update Q^T, and B is updated
 * by Eq. (4) (B(0:bb,trail) <- R_hat12 - R_hat11 R11^{-1} R12) without re-sketching.
 * Output mirrors LAPACK xGEQP3: A holds R in its upper trapezoid (rows 0..k-1) and the
 * updated trailing block R22 = A(k:m, k:n); the reflector tails sit below the diagonal of
 * columns 0..k-1 (xLARFG convention, v(0) = 1 implied); tau[0..k) their scalars;
 * jpvt[0..n) the permutation, 0-based: column c of A*Pi is column jpvt[c] of the input.
 * Argmax ties go to the smallest current column position.  Rank guard: if the largest
 * remaining sketch norm^2 falls to (10*max(m,n)*2^-53)^2 times the largest initial one,
 * pivoting stops for good (the remaining columns keep their order, B is no longer
 * updated); the number of pivots taken before that is the rank.  rank_out (DEVICE pointer to
 * one int64, may be NULL) receives the rank in stream order, when the factorization has run;
 * rqrcp_read_status reports it too.  The seeded sketch is rqrcp_generate_omega's draw, copied
 * from pageable host memory at the start of the call (not capturable in a CUDA graph; use
 * rqrcp_factor_with_omega there).
 * Limits of the library: l = b+p <= 1024 and the sketch and panel must fit in shared
 * memory across the GPU (checked; RQRCP_ERR_UNSUPPORTED otherwise).
 */
int rqrcp_factor(int64_t m, int64_t n, double* A, int64_t lda, int64_t k, int64_t b, int64_t p,
                 uint64_t seed, int32_t* jpvt, double* tau, int64_t* rank_out, void* work, size_t work_bytes,
                 void* stream);

/* As rqrcp_factor, with the l x m sketching matrix Omega (l = b+p, row-major, ldo >= m, device
 * memory) supplied by the caller instead of drawn from a seed.  Nothing is copied from the host. */
int rqrcp_factor_with_omega(int64_t m, int64_t n, double* A, int64_t lda, int64_t k, int64_t b,
                            int64_t p, const double* Omega, int64_t ldo, int32_t* jpvt, double* tau,
                            int64_t* rank_out, void* work, size_t work_bytes, void* stream);

#define RQRCP_UPDATE_EQ4 4 /* sketch update of Eq. (4) (Duersch-Gu): the default */
#define RQRCP_UPDATE_EQ5 5 /* sketch update of Eq. (5) (Martinsson et al.) */

/*
 * Plain FP64 form of Alg. 2 with the choice of the sketch update between pivot blocks.
 * Omega: the l x m sketching matrix (row-major, ldo >= m) or NULL to draw it from `seed` as in
 * rqrcp_generate_omega (ldo is then ignored).  formula:
 *   RQRCP_UPDATE_EQ4  Eq. (4): the QRCP of each block runs on B in place and the top bb rows of
 *                     the trailing sketch become R_hat12 - R_hat11 R11^{-1} R12 (rqrcp_factor);
 *   RQRCP_UPDATE_EQ5  Eq. (5): the QRCP runs on a copy of B; B is only permuted, Omega_bar =
 *                     Omega Q is kept up to date (the block's reflectors applied from the right,
 *                     as a compact-WY update of the m x l matrix Omega_bar^T) and the trailing
 *                     sketch becomes B2 - Omega_bar_1 R12 (all l rows).  The caller's Omega is
 *                     copied into the workspace, never written.
 * Both give the same pivots in exact arithmetic (Sec. 3.2 and 3.3.1); Eq. (5) reads and writes the m x l
 * Omega_bar once more per block.  Errors as in rqrcp_factor, with argument numbers in this list:
 * -10 ldo < m with Omega given, -11 formula not one of RQRCP_UPDATE_*, -12 jpvt NULL, -13 tau
 * NULL.  Workspace: rqrcp_workspace_size(..., RQRCP_PREC_FP64).
 */
int rqrcp_factor_ex(int64_t m, int64_t n, double* A, int64_t lda, int64_t k, int64_t b, int64_t p,
                    uint64_t seed, const double* Omega, int64_t ldo, int formula, int32_t* jpvt, double* tau,
                    int64_t* rank_out, void* work, size_t work_bytes, void* stream);

/*
 * Spectrum-revealing QR, Alg. 3 (Sec. IV-E), plain FP64.  Steps:
 *   1. RQRCP to rank l (Alg. 2 with Eq. (4), block size b, oversampling p, sketch from `seed` or
 *      the caller's Omega as in rqrcp_factor_ex; the sketch is updated after the last block too).
 *   2. The extra pivot: the trailing column with the largest r_i = ||B(:, i)||^2 / (b+p) moves to
 *      position l, one Householder step reduces A(l:m, l), and r_i -= R(l, i)^2.
 *   3. g_2 ~ |alpha|/sqrt(d) ||Omega_g R_hat^{-T}||_{1,2}, with R_hat the leading (l+1) x (l+1)
 *      block of R and alpha = R(l, l).  Omega_g is a fresh d x (l+1) Gaussian per estimate:
 *      estimate t uses rqrcp_generate_omega(d, l+1, seed_g + t).
 *   4. While g_2 > g, fewer than max_swaps swaps so far, and the RQRCP stage's rank guard did
 *      not fire before l pivots (R_hat would be singular to working precision): the worst
 *      column of R_hat (the largest column of Omega_g R_hat^{-T}) moves to position l by a
 *      round-robin rotation.  Givens rotations restore the upper-trapezoidal form,
 *      r_l = R(l,l)^2, r_i += R(l,i)^2, then steps 2 and 3 again.
 * Output: A is overwritten with the explicit R of A(:, jpvt) = Q R.  R(0:l+1, :) is upper
 * trapezoidal, the trailing block R22 = A(l+1:m, l+1:n), and every entry below the diagonal of
 * columns 0..l is zero.  Q is not formed.  jpvt (n, device) is 0-based.  info (host, 4
 * doubles, may be NULL) receives the swap count, the last g_2 estimate, |alpha| and the RQRCP
 * stage's rank (pivots before its guard fired; l if it never did).  The call
 * synchronises `stream` once per g_2 estimate.  Requires 1 <= l < min(m, n), g > 1, 1 <= d <=
 * 65535, (l+1)*8 bytes of shared memory per block.  Errors: -1 m, -2 n, -3 A, -4 lda, -5 l, -6 b,
 * -7 p, -10 ldo < m with Omega given, -11 g, -12 d, -14 max_swaps, -15 jpvt; RQRCP_ERR_*
 * otherwise.  Workspace: rqrcp_srqr_workspace_size(m, n, l, b, p, d) bytes (0 if invalid).
 */
size_t rqrcp_srqr_workspace_size(int64_t m, int64_t n, int64_t l, int64_t b, int64_t p, int64_t d);
int rqrcp_srqr(int64_t m, int64_t n, double* A, int64_t lda, int64_t l, int64_t b, int64_t p, uint64_t seed,
               const double* Omega, int64_t ldo, double g, int64_t d, uint64_t seed_g, int64_t max_swaps,
               int32_t* jpvt, double* info, void* work, size_t work_bytes, void* stream);

/*
 * Mixed form of Alg. 2: A is FP32 (lda >= m).  The sketch B = Omega A (Alg. 2, the sketch
 * step) is formed from Omega and A rounded to BF16 (round to nearest even) with FP32
 * accumulation; the pivot search, the compact-WY trailing updates (TF32 hi/lo parts on the
 * tensor cores, FP32-level accuracy) and Eq. (4) run in FP32 arithmetic; every Householder
 * reflector (column norm, beta, tau) of the panel is generated in FP64 and tau is returned in
 * FP64.  Arguments and output layout as in rqrcp_factor; the rank guard uses 2^-6 in place of
 * 10*max(m,n)*2^-53 (about five times the relative noise BF16 rounding leaves in a sketch column:
 * rank below that level is not resolved by this sketch).  RQRCP_TENSOR_CORES=0 in the environment
 * (read once per process) runs the FP32 form's contractions, and the batched kernel's sketch and
 * trailing update, as FP32 SIMT code instead of on the tensor cores, for A/B timing; the
 * accuracy class is the same.  Where the trailing matrix is larger than about 128 MiB, two
 * consecutive blocks share one pass of the trailing update (the second block's Gram is taken
 * before the first block's update and corrected); RQRCP_PAIRED=0 turns that off, =1 uses it at
 * every size (read once per process).  Its backward error stays in the same class (5.9e-7 against
 * 3.9e-7 per block on the 32768 x 16384, k = 512 workload).
 */
int rqrcp_factor_mixed(int64_t m, int64_t n, float* A, int64_t lda, int64_t k, int64_t b, int64_t p,
                       uint64_t seed, int32_t* jpvt, double* tau, int64_t* rank_out, void* work,
                       size_t work_bytes, void* stream);

#define RQRCP_SKETCH_BF16 0 /* sketch operands rounded to BF16, FP32 accumulation */
#define RQRCP_SKETCH_FP32 1 /* sketch with FP32-level accuracy (TF32 hi/lo parts, or FP32 FMA) */

/* rqrcp_factor_mixed with the sketching matrix and the sketch precision chosen by the caller.
 * Omega: the l x m FP32 sketching matrix (device, row-major, ldo >= m), or NULL to draw it from
 * `seed` as rqrcp_generate_omega_f32 does (ldo is then ignored; with Omega given nothing is copied
 * from the host).  sketch: RQRCP_SKETCH_BF16 (as
 * rqrcp_factor_mixed) or RQRCP_SKETCH_FP32, which uses the rank guard 10*sqrt(max(m,n))*2^-24
 * (about ten times the rounding noise of an FP32 sketch column).  Errors as rqrcp_factor_mixed,
 * with -10 ldo < m with Omega given, -11 sketch invalid, -12 jpvt NULL, -13 tau NULL. */
int rqrcp_factor_mixed_ex(int64_t m, int64_t n, float* A, int64_t lda, int64_t k, int64_t b, int64_t p,
                          uint64_t seed, const float* Omega, int64_t ldo, int sketch, int32_t* jpvt, double* tau,
                          int64_t* rank_out, void* work, size_t work_bytes, void* stream);

/*
 * QR with tournament pivoting on the sketch in place of Alg. 2's partial QRCP on B (the paper's
 * future work, Sec. VI: "QR with tournament pivoting in place of partial QRCP"; Demmel, Grigori,
 * Gu and Xiang, SIAM J. Matrix Anal. Appl. 36 (2015)).  For each block of bb = min(b, k - i)
 * pivots the n - i trailing sketch columns are split into leaf groups of G consecutive columns;
 * each leaf chooses min(bb, its size) columns by bb greedy steps of Alg. 1 (squared norms of the
 * trailing rows recomputed at every step, the largest first, ties to the smallest position); each
 * node of a tree with fan-in F chooses min(bb, candidates) of its children's choices the same way,
 * reading the children's columns as they were at the start of the block, concatenated in child
 * order; the root's choices, in their order, are the block's pivots.  The rank guard tests each
 * chosen column's trailing squared norm at its step against the bound of the corresponding
 * greedy entry point.  Everything else (panel, compact-WY update, Eq. (4)) is as in rqrcp_factor
 * (FP64) or rqrcp_factor_mixed_ex (FP32); the workspace is the same.  group_cols: 0 for
 * G = max(2b, ceil((n - i) / SMs)), lowered to the largest group one SM holds; > 0 for G =
 * group_cols (at least b).  F = 4, or 2 when four blocks of candidates do not fit one SM.
 * Errors: as rqrcp_factor_ex with -11 group_cols < 0 (FP64 form); as rqrcp_factor_mixed_ex with
 * -12 group_cols < 0 and -13 jpvt, -14 tau (FP32 form); RQRCP_ERR_UNSUPPORTED when b + p > 256
 * or a group does not fit one SM's shared memory.
 */
int rqrcp_factor_tournament(int64_t m, int64_t n, double* A, int64_t lda, int64_t k, int64_t b, int64_t p,
                            uint64_t seed, const double* Omega, int64_t ldo, int64_t group_cols, int32_t* jpvt,
                            double* tau, int64_t* rank_out, void* work, size_t work_bytes, void* stream);
int rqrcp_factor_mixed_tournament(int64_t m, int64_t n, float* A, int64_t lda, int64_t k, int64_t b, int64_t p,
                                  uint64_t seed, const float* Omega, int64_t ldo, int sketch, int64_t group_cols,
                                  int32_t* jpvt, double* tau, int64_t* rank_out, void* work, size_t work_bytes,
                                  void* stream);

/* The leaf group size G and the fan-in F that the tournament entry points use for a block of bb
 * pivots (block size b, oversampling p) over ncols trailing columns of elem_bytes-byte elements
 * (8: FP64 form, 4: FP32 form), with the caller's group_cols (0: automatic).  Host only; reads the
 * current device's SM count and shared-memory size.  Errors: -1 ncols < 1, -2 bb not in
 * [1, ncols], -3 b not in [bb, 128], -4 p < 0, -5 elem_bytes, -6 group_cols < 0, -7/-8 NULL
 * outputs; RQRCP_ERR_UNSUPPORTED as above. */
int rqrcp_tournament_config(int64_t ncols, int64_t bb, int64_t b, int64_t p, int elem_bytes, int64_t group_cols,
                            int64_t* group_out, int64_t* fanin_out);

/*
 * Synchronises `stream`, then reads the device-side status left in `work` by the last
 * factorization: returns RQRCP_OK, RQRCP_ERR_NONFINITE or RQRCP_ERR_TIMEOUT (or
 * RQRCP_ERR_CUDA if the synchronisation itself fails) and stores the rank (number of
 * pivots chosen before the rank guard fired, k if it never fired) in *rank if non-NULL.
 */
int rqrcp_read_status(const void* work, int64_t* rank, void* stream);

/*
 * Low-rank approximation L = Q1 [R11 R12] Pi^T (Sec. I-A) from the output of
 * rqrcp_factor: Afact (m x n, ldaf), tau (k), jpvt (n).  Q1 (required, ldq >= m) receives
 * the m x k matrix Q1 = H_0 ... H_{k-1} I(:,0:k); L (m x n, ldl >= m) receives the product,
 * or is skipped when L is NULL.  `work` needs rqrcp_lowrank_workspace_size(m, n, k) bytes.
 * The _f32 twin takes the FP32 output of rqrcp_factor_mixed (tau stays FP64).
 */
size_t rqrcp_lowrank_workspace_size(int64_t m, int64_t n, int64_t k);
int rqrcp_lowrank(int64_t m, int64_t n, int64_t k, const double* Afact, int64_t ldaf, const double* tau,
                  const int32_t* jpvt, double* L, int64_t ldl, double* Q1, int64_t ldq, void* work,
                  size_t work_bytes, void* stream);
int rqrcp_lowrank_f32(int64_t m, int64_t n, int64_t k, const float* Afact, int64_t ldaf, const double* tau,
                      const int32_t* jpvt, float* L, int64_t ldl, float* Q1, int64_t ldq, void* work,
                      size_t work_bytes, void* stream);

/*
 * FP64 outputs of the mixed form with one FP64 reorthogonalisation pass (the paper's low-rank
 * factors Q1 and [R11 R12], Sec. I-A; the pass itself is not in the paper).  From the output of
 * rqrcp_factor_mixed (Afact FP32, tau FP64) forms Q1 (m x k, FP64, ldq >= m) and
 * R = [R11 R12] (k x n, FP64, ldr >= k, zero below the diagonal), measures
 * e = ||Q1^T Q1 - I||_F and, when e > tol, applies one CholQR pass on the device:
 * G = Q1^T Q1 = S^T S (S upper), Q1 <- Q1 S^{-1}, R <- S R, which keeps Q1 R unchanged.  The
 * decision is taken on the device (no host synchronisation); *orth (device, may be NULL)
 * receives e.  `work` needs rqrcp_reorth_workspace_size(m, n, k) bytes.  A Gram matrix that
 * is not positive definite is reported as RQRCP_ERR_NONFINITE by rqrcp_read_status(work).
 */
size_t rqrcp_reorth_workspace_size(int64_t m, int64_t n, int64_t k);
int rqrcp_lowrank_reorth(int64_t m, int64_t n, int64_t k, const float* Afact, int64_t ldaf, const double* tau,
                         double* Q1, int64_t ldq, double* R, int64_t ldr, double tol, double* orth, void* work,
                         size_t work_bytes, void* stream);

/*
 * Gradient of the truncated factorization with the permutation held fixed (the paper has
 * the forward only; this is the adjoint of what Alg. 2 computes for the first k columns).
 * With X = A Pi = [X1 X2], X1 = Q1 R11 and R12 = Q1^T X2, given upstream gradients dQ1
 * (m x k, lddq) and dR = [dR11 dR12] (k x n, lddr; only the upper triangle of dR11 is read),
 * writes dA (m x n, ldda):  dX2 = Q1 dR12;  dQ' = dQ1 + X2 dR12^T;
 * M = R11 dR11^T - dQ'^T Q1;  dX1 = (dQ' + Q1 copyltu(M)) R11^{-T}, copyltu(M) =
 * tril(M) + tril(M,-1)^T;  dA(:, jpvt[c]) = dX(:, c).  Inputs: the original A (lda), jpvt
 * (n, from the forward), Q1 (ldq) and R = [R11 R12] (k x n, ldr, R11 read as upper
 * triangular), all device memory.  A zero diagonal entry of R11 gives a zero gradient
 * column.  `work` needs rqrcp_backward_workspace_size(m, n, k, precision) bytes.
 */
size_t rqrcp_backward_workspace_size(int64_t m, int64_t n, int64_t k, int precision);
int rqrcp_backward(int64_t m, int64_t n, int64_t k, const double* A, int64_t lda, const int32_t* jpvt,
                   const double* Q1, int64_t ldq, const double* R, int64_t ldr, const double* dQ1,
                   int64_t lddq, const double* dR, int64_t lddr, double* dA, int64_t ldda, void* work,
                   size_t work_bytes, void* stream);
int rqrcp_backward_f32(int64_t m, int64_t n, int64_t k, const float* A, int64_t lda, const int32_t* jpvt,
                       const float* Q1, int64_t ldq, const float* R, int64_t ldr, const float* dQ1,
                       int64_t lddq, const float* dR, int64_t lddr, float* dA, int64_t ldda, void* work,
                       size_t work_bytes, void* stream);

/*
 * Sketch B = Omega A for callers that cannot allocate device memory.  The paper has no
 * counterpart: this is a deployment convenience around the same sketch as rqrcp_sketch.
 * Who needs it: code that is handed only the input and output pointers (a plugin or
 * callback behind a narrow C interface with no allocator and no workspace to pass), and
 * code that must not call cudaMalloc/cudaFree because of the device-wide synchronisation
 * those calls imply.  Arguments and layouts are those of rqrcp_sketch, minus the workspace.
 * Scratch: a fixed array of 8 MiB of device memory that every GPU which loads the library
 * holds until the process exits; a problem needs n * l * 8 bytes of it for one split
 * (n * l <= 1,048,544), larger ones are rejected with RQRCP_ERR_UNSUPPORTED before anything
 * is enqueued.  The first call on each device looks the array's address up (with that
 * device current); make that first call before any stream capture.  No cudaMalloc,
 * cudaFree or allocating library routine is called.  Every call on a device shares that
 * device's one array, which keeps the last call's contents; the status block is cleared at
 * the start of each call.  Calls on the same device that overlap on the GPU (different
 * streams or different host threads) race on the array, so serialise them.  Device-side
 * status (non-finite sketch) is not reported: every column of B is written, and a column of A
 * holding NaN or Inf gives a non-finite column of B.
 */
int rqrcp_sketch_noalloc(int64_t m, int64_t n, const double* A, int64_t lda, const double* Omega, int64_t l,
                         int64_t ldo, double* B, int64_t ldb, void* stream);

/*
 * Batched randomized QRCP of many independent FP32 matrices of uneven shapes in ONE persistent
 * launch (the paper factors one matrix at a time; batching is the GPU form of running Alg. 2 on
 * many small problems).  `descs` is a device array of `count` descriptors, 72 bytes each, with
 * this layout (8-byte aligned, in order): float* A, int32_t* jpvt (n), double* tau (k),
 * int64_t* rank (1), int64_t m, int64_t n, int64_t k, int64_t lda, int32_t b, int32_t tiles.
 * `tiles` picks the tile shapes of the matrix's contractions (0: the library's default rules; an OR
 * of RQRCP_TILES_*, e.g. from the autotuner): the trailing update C -= V Y on 64 x 128 FP32 SIMT
 * tiles (UPDATE_SIMT) or 128 x 64 tcgen05 tiles (UPDATE_TC; default: tcgen05 for b > 16), the
 * sketch on SIMT tiles instead of tcgen05 (SKETCH_SIMT), the Gram V^T [V C] on 64 x 128 tiles
 * instead of the smallest of 16 x 512 / 32 x 256 / 64 x 128 that holds b rows (GRAM_RT64).
 * Every matrix needs 1 <= k <= min(m,n) <= max(m_max, n_max), m <= m_max, n <= n_max,
 * 1 <= b <= b_max <= 64 (b is per matrix, e.g. from the autotuner).  `order` (device, count
 * ints) is the processing order (largest first balances best); one block per SM takes the next
 * matrix from an atomic counter and factors it alone.  All matrices share one FP32 sketching
 * matrix Omega (device, l_max x m_max row-major with ldo >= m_max, l_max = b_max + p; e.g.
 * rqrcp_generate_omega_f32's draw, made once before the batched calls); matrix i uses its leading
 * (b_i + p) x m_i block.  Per-matrix results as rqrcp_factor_mixed;
 * rank is -1 when the sketch of that matrix is not finite, and -2 when a tensor-core wait of
 * the block factoring it gave up after 2 s (that block then stops taking matrices; the others
 * finish the batch; matrices never taken keep rank 0).  The call is one kernel and a memset on
 * `stream`, copies nothing from the host and allocates nothing (graph-capturable).  Errors: -1
 * count < 0, -2 descs NULL, -3 order NULL, -4 m_max, -5 n_max, -6 b_max, -7 p, -8 Omega NULL,
 * -9 ldo < m_max.  Each block holds all of its SM's tensor
 * memory for the launch.  `work` needs rqrcp_batched_workspace_size(m_max, n_max, b_max, p)
 * bytes.  Limits: the block's shared memory (max(8 m_max floats, 168 KB) + n_max doubles +
 * b_max^2 doubles + ~3 KB) must fit, else RQRCP_ERR_UNSUPPORTED (m_max <= ~5600 with
 * n_max = 2048, b_max = 64).
 */
#define RQRCP_TILES_UPDATE_SIMT 1
#define RQRCP_TILES_UPDATE_TC 2
#define RQRCP_TILES_SKETCH_SIMT 4
#define RQRCP_TILES_GRAM_RT64 8
size_t rqrcp_batched_workspace_size(int64_t m_max, int64_t n_max, int64_t b_max, int64_t p);
int rqrcp_factor_batched(int64_t count, const void* descs, const int* order, int64_t m_max, int64_t n_max,
                         int64_t b_max, int64_t p, const float* Omega, int64_t ldo, void* work, size_t work_bytes,
                         void* stream);

/*
 * Kernel-level timing for measurement (not part of the method).  Between
 * rqrcp_profile_begin and rqrcp_profile_end, every kernel the library enqueues is
 * bracketed by a pair of CUDA events on its stream, and the algorithmic work of the
 * launch (flops and bytes that the step must do, not what the kernel happens to move)
 * is accumulated per kernel class.  rqrcp_profile_end synchronises the device, turns
 * the recording off and, for each class c < min(nmax, RQRCP_PROFILE_CLASSES), writes
 * launches[c], the summed event time ms[c], flops[c] and bytes[c] (any pointer may be
 * NULL).  Host-side state is global to the process; not thread-safe.
 */
#define RQRCP_PROFILE_CLASSES 14
int rqrcp_profile_begin(void);
int rqrcp_profile_end(int nmax, int64_t* launches, double* ms, double* flops, double* bytes);
const char* rqrcp_profile_class_name(int cls);

/*
 * Throughput probes for the roofline denominators (measurement, not part of the method).  kind:
 *   RQRCP_PROBE_DFMA     register-resident FP64 FMA chains (8 per thread, 64 warps per SM)
 *   RQRCP_PROBE_FFMA     the same in FP32
 *   RQRCP_PROBE_TC_TF32  back-to-back tcgen05.mma kind::tf32, M = 128, N = 256, K = 8, one
 *                        CTA per SM, operands in shared memory, accumulator in tensor memory
 *   RQRCP_PROBE_TC_BF16  the same with kind::f16 on BF16 operands (K = 16)
 * One untimed launch, then one launch timed with CUDA events on `stream`; the call synchronises
 * the stream.  *tflops receives the dense rate (2 flops per multiply-add) and *ms (may be NULL)
 * the timed launch's duration.  Errors: -1 kind, -2 tflops NULL; RQRCP_ERR_TIMEOUT if a
 * tensor-core wait gave up (2 s), RQRCP_ERR_CUDA otherwise.
 */
#define RQRCP_PROBE_DFMA 0
#define RQRCP_PROBE_FFMA 1
#define RQRCP_PROBE_TC_TF32 2
#define RQRCP_PROBE_TC_BF16 3
int rqrcp_peak_probe(int kind, double* tflops, double* ms, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* RQRCP_H */
