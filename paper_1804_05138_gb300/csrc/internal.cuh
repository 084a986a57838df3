// internal.cuh -- shared device helpers and kernel launchers of librqrcp (not part of the ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "../../include/rqrcp.h"

namespace rq {

// Device-side status block at the head of every workspace (zeroed by the host before a call).
struct Status {
    int error;                     // RQRCP_OK or an RQRCP_ERR_* code set by a kernel
    int guard;                     // 1 once the rank guard fired
    long long rank;                // pivots chosen before the guard fired
    unsigned long long bar;        // grid barrier: arrivals (low 32 bits), generation (high 32 bits)
    unsigned long long nu0bits;    // bits of the largest initial sketch column norm^2 (>= 0)
    long long pad[12];
};
static_assert(sizeof(Status) <= 256, "status block must fit in 256 bytes");

constexpr unsigned long long kWaitLimitNs = 2000000000ull;  // 2 s per barrier wait

__device__ __forceinline__ unsigned long long globaltimer_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ int status_error(const Status* st)
{
    return *(volatile const int*)&st->error;
}

__device__ __forceinline__ void set_error(Status* st, int code)
{
    atomicCAS(&st->error, 0, code);
}

__device__ __forceinline__ unsigned long long ld_acquire_gpu(const unsigned long long* p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// Waits longer than this also watch the status word (a block that met an error has left).
constexpr unsigned long long kErrorWatchNs = 20000;

// Grid-wide barrier for cooperatively launched kernels.  One 64-bit word holds the arrivals of
// the current barrier (low half) and its generation (high half).  A block arrives with one
// acquire-release add, which also tells it the generation; the last arrival resets the count
// and opens the next generation with a single release add of 2^32 - G; the others poll the word
// with acquire loads.  The count is back at 0 after every barrier, so launches of any grid size
// can share the word.  Every wait is bounded: a wait longer than kErrorWatchNs returns false as
// soon as any block has recorded an error, and after kWaitLimitNs the block records
// RQRCP_ERR_TIMEOUT and returns false; callers then leave the kernel.
__device__ __forceinline__ bool grid_barrier(Status* st)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned long long G = gridDim.x;
        unsigned long long old;
        asm volatile("atom.add.acq_rel.gpu.global.u64 %0, [%1], %2;" : "=l"(old) : "l"(&st->bar), "l"(1ull) : "memory");
        const unsigned int gen = (unsigned int)(old >> 32);
        int ok = 1;
        if ((old & 0xffffffffull) == G - 1) {
            asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(&st->bar), "l"((1ull << 32) - G) : "memory");
        } else {
            const unsigned long long t0 = globaltimer_ns();
            while ((unsigned int)(ld_acquire_gpu(&st->bar) >> 32) == gen) {
                const unsigned long long dt = globaltimer_ns() - t0;
                if (dt > kErrorWatchNs && status_error(st)) {
                    ok = 0;
                    break;
                }
                if (dt > kWaitLimitNs) {
                    set_error(st, RQRCP_ERR_TIMEOUT);
                    ok = 0;
                    break;
                }
            }
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Householder scalars (xLARFG convention) from alpha = x(1) and ss = ||x(2:)||^2, in FP64,
// computed by a whole warp: beta = -sign(alpha) sqrt(alpha^2 + ss), and the two divisions
// tau = (beta - alpha) / beta and scal = 1 / (alpha - beta) run on lanes 0 and 1 at once (FP64
// division and square root are long dependent chains on this part).  ss = 0 gives tau = scal = 0
// and beta = alpha.  All 32 lanes must call it with the same alpha and ss; every lane gets the
// results.
__device__ __forceinline__ void warp_larfg(double alpha, double ss, double& tau, double& beta, double& scal)
{
    beta = alpha;
    tau = 0.0;
    scal = 0.0;
    if (ss != 0.0) {
        const int lane = threadIdx.x & 31;
        const double nrm = sqrt(alpha * alpha + ss);
        beta = (alpha >= 0.0) ? -nrm : nrm;
        const double num = lane == 0 ? beta - alpha : 1.0;
        const double den = lane == 0 ? beta : alpha - beta;
        const double q = num / den;
        tau = __shfl_sync(0xffffffffu, q, 0);
        scal = __shfl_sync(0xffffffffu, q, 1);
    }
}

template <typename T>
__device__ __forceinline__ T ld_cg(const T* p) { return __ldcg(p); }

// ---------------------------------------------------------------------------------------
// Launchers (each returns cudaSuccess or the launch error).
// ---------------------------------------------------------------------------------------
struct DevInfo {
    int sms;
    int max_smem_optin;
};
const DevInfo& dev_info();

// Kernel attributes such as the dynamic shared-memory limit are set per device: the flags that
// record "already set" are kept per device, indexed by the calling thread's current device.
constexpr int kMaxDevices = 64;
// The calling thread's current device, or -1 if it cannot be read or has no slot (>= kMaxDevices).
inline int current_device()
{
    int d = 0;
    if (cudaGetDevice(&d) != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    return (d < 0 || d >= kMaxDevices) ? -1 : d;
}

// "Done once on this device" flag, safe when several host threads call the library.  A device
// without a slot (current_device() < 0) gets no flag: the guarded work is redone on every call
// there instead of borrowing another device's flag.
struct DevFlag {
    std::atomic<bool> f[kMaxDevices];
    bool done() const
    {
        const int d = current_device();
        return d >= 0 && f[d].load(std::memory_order_acquire);
    }
    void set()
    {
        const int d = current_device();
        if (d >= 0) f[d].store(true, std::memory_order_release);
    }
};

// Allow a kernel the largest dynamic shared memory the device grants next to the kernel's
// own static shared memory.  Returns the runtime error, if any.
template <typename K>
cudaError_t allow_max_dynamic_smem(K kernel)
{
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, (const void*)kernel);
    if (e != cudaSuccess) return e;
    const int maxdyn = dev_info().max_smem_optin - (int)fa.sharedSizeBytes;
    return cudaFuncSetAttribute((const void*)kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, maxdyn);
}

// Omega (l x m row-major, ldo >= m) from Philox4x64-10 + Box-Muller, drawn on the host (threads
// over Philox blocks; the bits do not depend on the thread count).
void host_omega(int64_t l, int64_t m, uint64_t seed, double* out, int64_t ldo);
// The same draw copied into device memory Om (row-major, ldo) on stream s, FP64 or rounded to FP32.
// The copy is from pageable host memory: it cannot be captured in a CUDA graph.
template <typename T>
cudaError_t launch_omega(int64_t l, int64_t m, uint64_t seed, T* Om, int64_t ldo, cudaStream_t s);

// Split-K partial products P[sp][c][r] = sum_{q in chunk sp} X(q, r) * C(q, c), r < M, c < N.
// X is K x M column-major (ldx), C is K x N column-major (ldc).  maskX: X has the unit-lower
// reflector structure (X(q,r) = 0 for q < r, 1 for q == r).  maskC: the first maskC columns
// of C have the same structure.  kchunk must be a multiple of 16.  bf16 (FP32 only): both operands
// are rounded to BF16 (round to nearest even) as they are read (the BF16 sketch).
template <typename T>
cudaError_t launch_gemm_tn(const T* X, int64_t ldx, const T* C, int64_t ldc, int64_t M, int64_t N,
                           int64_t K, int64_t kchunk, double* P, int maskX, int64_t maskC,
                           const Status* st, cudaStream_t s, int bf16 = 0);

// Blocks of the SIMT split-K contraction (launch_gemm_tn) resident per SM for FP64 (8) or FP32 (4)
// elements and an M-row result, and the rows of one of its tiles (48, 64, 80 or 96: a result of up
// to 96 rows is one tile, larger ones are 64-row tiles).
int gemm_tn_blocks_per_sm(int elem_bytes, int64_t M);
int gemm_tn_tile_rows(int64_t M);

// Tensor-core (tcgen05 kind::tf32, 3xTF32) split-K contraction with the output of
// launch_gemm_tn<float>: X(q, r) = X[r * ldx + q] (q < K, r < M; unit-lower reflector structure
// for r < maskX), C(q, c) = C[c * ldc + q] (c < N; the structure for c < maskC).  C must be
// 16-byte aligned with ldc % 4 == 0 (tc_gemm_supported); xs (16-byte aligned,
// tc_xsplit_bytes(M, K)) receives the TF32 parts of X.  kchunk must come from tc_kchunk with
// the same bf16 flag and M.  bf16: both operands rounded to BF16 (round to nearest even), products on
// the kind::f16 tensor path with FP32 accumulation (the BF16 sketch; no reflector masks).  maskC0
// moves C's masked columns to maskC0 .. maskC0 + maskC - 1 (the structure relative to maskC0).
bool tc_gemm_supported(long long M, long long ldc, const void* C, int bf16 = 0);
size_t tc_xsplit_bytes(long long M, long long K);
long long tc_kchunk(long long N, long long K, int& nsplit, int bf16 = 0, long long M = 96);
cudaError_t launch_gemm_tn_tc(const float* X, long long ldx, const float* C, long long ldc, long long M, long long N,
                              long long K, long long kchunk, double* P, long long maskX, long long maskC, float* xs,
                              const Status* st, cudaStream_t s, int bf16 = 0, long long maskC0 = 0);
// Tensor-core (tcgen05 kind::tf32, 3xTF32) form of launch_gemm_update<float> without colmap:
// C(mr x nt) -= V(mr x kb) Y(kb x nt), kb <= 64, V unit-lower for rows r < maskV.  C must be
// 16-byte aligned with ldc % 4 == 0 (tc_update_supported); ys (16-byte aligned,
// tc_update_ws_bytes(nt)) receives the TF32 parts of Y.
bool tc_update_supported(long long kb, long long ldc, const void* C);
size_t tc_update_ws_bytes(long long nt, int kp = 64);
cudaError_t launch_gemm_update_tc(float* C, long long ldc, const float* V, long long ldv, const double* Y, long long ldy,
                                  long long mr, long long nt, int kb, long long maskV, float* ys, const Status* st,
                                  cudaStream_t s);
// Two blocks in one pass: C(mr x nt) -= V(mr x kb) [Y; Y2], kb <= 128, rows 0..kb1-1 of the
// contraction from Y (ldy) and kb1..kb-1 from Y2 (ldy2); V's columns j >= maskC0 carry the unit-lower
// structure relative to column maskC0 in rows r < maskV.  ys needs tc_update_ws_bytes(nt, 128).
bool tc_update2_supported(long long ldc, const void* C);
cudaError_t launch_gemm_update_tc2(float* C, long long ldc, const float* V, long long ldv, const double* Y,
                                   long long ldy, const double* Y2, long long ldy2, int kb1, long long mr, long long nt,
                                   int kb, long long maskV, int maskC0, float* ys, const Status* st, cudaStream_t s);
bool tensor_cores_enabled();

// General 3xTF32 tensor-core contraction (mm_tc.cu):
//   D(r, dcol(c)) = alpha sum_q A(r, q) B(q, c) + beta D0(r, dcol(c)),  r < M, c < N, q < K,
// dcol(c) = dmap ? dmap[c] : c.  A(r, q) = A[q lda + r] or, kmajor, A[r lda + q]; A must be
// 16-byte aligned with lda % 4 == 0 (mm_tc_supported).  B is given as TF32 planes written by
// launch_mm_planes (mm_planes_bytes(K, N), 16-byte aligned): B(q, c) = src[kq ldk + c ldn] with
// kq = kmap ? kmap[q] : q, zero where kmap[q] < kmin.  nsplit > 1 splits K: split z writes its
// partial product to D + z dz (beta must be 0); launch_mm_sum adds the splits.  Masks for reflector
// blocks V stored in place (unit lower, other data above the diagonal): amask 1 makes A = V or,
// kmajor, A = V^T; planes mask 1 makes B unit lower, mask 2 upper (B(q, c) = 0 for q > c).
bool mm_tc_supported(const void* A, long long lda);
size_t mm_planes_bytes(long long K, long long N);
int mm_max_split();
int mm_choose_split(long long M, long long N, long long K, int min_chunks);
cudaError_t launch_mm_planes(const float* src, long long ldk, long long ldn, const int32_t* kmap, long long kmin,
                             long long K, long long N, float* planes, const Status* st, cudaStream_t s,
                             int mask = 0);
cudaError_t launch_mm_tc(bool kmajor, const float* A, long long lda, const float* planes, long long M, long long N,
                         long long K, int nsplit, float alpha, float beta, const float* D0, long long ldd0, float* D,
                         long long ldd, long long dz, const int32_t* dmap, Status* st, cudaStream_t s,
                         int amask = 0);
// FP32 low-rank outputs on the tensor cores (lowrank.cu): Q1 = I(:, 0:k) - V T V1^T with all k
// reflectors in one compact WY form (T^{-1} = diag(1 / tau) + striu(V^T V)), and, if L is not null,
// L(:, jpvt[c]) = Q1 [R11 R12](:, c).  Usable when lowrank_f32_tc_ok (k <= 256, aligned operands);
// work (256-byte aligned) needs lowrank_f32_tc_bytes(m, n, k) and gets its status block at the head.
template <typename T>
cudaError_t launch_eye(T* Q, int64_t ldq, int64_t m, int64_t k, cudaStream_t s);
bool lowrank_f32_tc_ok(int64_t k, const float* Afact, int64_t ldaf, const float* Q1, int64_t ldq);
size_t lowrank_f32_tc_bytes(int64_t m, int64_t n, int64_t k);
int lowrank_f32_tc(int64_t m, int64_t n, int64_t k, const float* Afact, int64_t ldaf, const double* tau,
                   const int32_t* jpvt, float* L, int64_t ldl, float* Q1, int64_t ldq, void* work, cudaStream_t s);

// D(r, c) = D0(r, c) (if D0) + sum_{z < nz} P[z dz + c ldp + r], r < M, c < N (compensated sum).
cudaError_t launch_mm_sum(const float* P, long long ldp, long long dz, int nz, long long M, long long N, const float* D0,
                          long long ldd0, float* D, long long ldd, const Status* st, cudaStream_t s);

// C(mr x nc) -= V(mr x kb) * Y(kb x nc).  maskV: V has the unit-lower reflector structure.
// colmap (optional): column c of the product goes to column colmap[c] of C.
template <typename T>
cudaError_t launch_gemm_update(T* C, int64_t ldc, const T* V, int64_t ldv, const double* Y, int64_t ldy,
                               int64_t mr, int64_t nc, int64_t kb, int maskV, const int32_t* colmap,
                               const Status* st, cudaStream_t s);

// B(0:l, j) = sum_sp P[sp][j][0:l]; records max column norm^2 and non-finite entries.
template <typename T>
cudaError_t launch_sketch_reduce(const double* P, int nsplit, int64_t l, int64_t n, T* B, int64_t ldb,
                                 Status* st, cudaStream_t s);

// Gram = sum_sp P[sp][0:bb][0:bb]; T (bb x bb, forward columnwise compact WY) from Gram and tau.
cudaError_t launch_tform(const double* P, int nsplit, int64_t ncols, int bb, const double* tau,
                         double* Tm, const Status* st, cudaStream_t s);

// Y(:, c) = op(T) * sum_sp P[sp][c0 + c][0:bb], c < nc, op(T) = T^T if transT else T.  fp32c:
// FP32 arithmetic with FP64-class accuracy (two-float operands, compensated sums) for the FP32
// form; otherwise IEEE double.
cudaError_t launch_reduce_y(const double* P, int nsplit, int64_t ncols, int64_t c0, int bb, const double* Tm,
                            int transT, double* Y, int64_t nc, const Status* st, cudaStream_t s, int fp32c = 0);

// Cooperative pivot search on B(:, i:n) (bb steps of QRCP on the sketch).  `cand` is
// pivot_cand_bytes(l) of candidate buffers followed by the swap map (1 + 4*bb int64).
// launch_index: the pivot search's position among the call's pivot searches (0, 1, 2, ...):
// consecutive searches use the two arrival counters at the head of `cand` in turn.
template <typename T>
cudaError_t launch_pivot(T* B, int64_t ldb, int l, int64_t n, int64_t i, int bb, int32_t* jpvt,
                         int32_t* piv, void* cand, double guard_rel2, Status* st, cudaStream_t s,
                         int launch_index);
size_t pivot_cand_bytes(int l);
// The head of `cand`: the pivot searches' arrival counters, which must be zero before a
// factorization's first pivot search.
size_t pivot_slot_bytes();

// QR with tournament pivoting on B(:, i:n) in place of the partial QRCP (the same outputs as
// launch_pivot: B transformed and permuted, jpvt, piv, the swap map).  tournament_config gives the
// leaf group size and the fan-in for a block with ncols trailing columns (group_cols 0: automatic;
// > 0: that size, at least b), or false when the block does not fit one SM.  ws: tournament_ws_bytes.
bool tournament_config(int64_t ncols, int bb, int64_t b, int l, int elem_bytes, int64_t group_cols, int64_t* gs_out,
                       int* fanin_out);
size_t tournament_ws_bytes(int64_t n, int l, int64_t b, int elem_bytes);
template <typename T>
cudaError_t launch_tournament(T* B, int64_t ldb, int l, int64_t n, int64_t i, int bb, int64_t b, int64_t gs,
                              int fanin, int32_t* jpvt, int32_t* piv, void* ws, long long* swapmap, T* tmp,
                              double guard_rel2, Status* st, cudaStream_t s);

// Column swaps of A following the net column map written by the pivot kernel
// (swapmap[0] = count, then (destination, source) position pairs); tmp holds 2*bb columns.
template <typename T>
cudaError_t launch_swaps(T* A, int64_t lda, int64_t m, int bb, const long long* swapmap, T* tmp,
                         const Status* st, cudaStream_t s);

// Correction split of a paired block step (update.cu): Pc[(c0 + c) bb + r] = -(Gx Y0(:, cy0 + c))(r)
// for c < nt, r < bb <= 64, Gx(r, q) = P2[q bb + r], Y0 column-major (ldy).  launch_split_sum first
// sums ns2 splits of length len, stride apart, into the first, in place.
cudaError_t launch_split_sum(double* P2, int ns2, int64_t len, int64_t stride, const Status* st, cudaStream_t s);
cudaError_t launch_wy_corr(const double* P2, int bb, const double* Y0, int64_t ldy, int64_t cy0, int64_t nt, int64_t c0,
                           double* Pc, const Status* st, cudaStream_t s);

// Status block reset (rank = k) and jpvt = 0..n-1.
cudaError_t launch_init(Status* st, int64_t k, int32_t* jpvt, int64_t n, cudaStream_t s);

// Cooperative Householder panel QR of A(i:m, i:i+bb) (FP64 reflector generation).  skip (FP32 form
// only, device int, may be null): the kernel returns at once when *skip == 0 (the CholeskyQR2 panel
// factored the panel).
template <typename T>
cudaError_t launch_panel(T* A, int64_t lda, int64_t m1, int bb, double* tau, double* part, Status* st,
                         cudaStream_t s, const int* skip = nullptr);

// CholeskyQR2 panel with Householder reconstruction for the FP32 form (cholqr.cu): writes the panel's
// R, reflector tails and tau in the layout of launch_panel<float>, or leaves the panel untouched and
// sets *flag_out = 1 when the panel is too ill-conditioned (launch_panel with skip = that flag then
// factors it).  ws: cholqr_ws_bytes(m1) bytes, 256-byte aligned.
bool cholqr_supported(int bb);
bool cholqr_enabled();
size_t cholqr_ws_bytes(int64_t m_max);
cudaError_t launch_cholqr_panel(float* A, int64_t lda, int64_t m1, int bb, double* tau, void* ws, int** flag_out,
                                const Status* st, cudaStream_t s);
size_t panel_part_bytes(int bb);
bool panel_fits(int64_t m1, int bb, int elem_bytes);
bool pivot_fits(int64_t ncols, int l, int elem_bytes);

// Eq. (4): Omega_hat_11 = R_hat11 R11^{-1}, then B(0:bb, i+bb:n) -= Omega_hat_11 R12.
template <typename T>
cudaError_t launch_bupdate(T* B, int64_t ldb, const T* A, int64_t lda, int64_t i, int bb, int64_t n,
                           double* What, const Status* st, cudaStream_t s);

// Eq. (5), last step: B(:, c0:c0+nt) = Bc(:, c0:c0+nt) - sum_sp P[sp][c][0:l] (ld l for B and
// Bc), written to both B and Bc.  Skipped once the rank guard has fired.
template <typename T>
cudaError_t launch_bfinish(T* B, T* Bc, int l, int64_t c0, int64_t nt, const double* P, int nsplit,
                           const Status* st, cudaStream_t s);

// Alg. 3 (SRQR) on the explicit R in A (srqr.cu).  info (device, 4 doubles): g_2 estimate,
// its worst column, |alpha|, and the tau of the latest one-step reflector.
// prepare: zero the reflector tails of columns 0..l-1; r_i = ||B(:, i)||^2 / ls for i >= l.
cudaError_t launch_srqr_prepare(double* A, int64_t lda, int64_t m, int64_t l, int64_t n, const double* B, int ls,
                                double* r, const Status* st, cudaStream_t s);
// extra pivot: argmax r -> column l, one Householder step on A(l:m, l:n), r_i -= A(l,i)^2.
cudaError_t launch_srqr_extra_pivot(double* A, int64_t lda, int64_t m, int64_t l, int64_t n, double* r,
                                    int32_t* jpvt, double* info, const Status* st, cudaStream_t s);
// g_2 estimate with the d x (l+1) Gaussian drawn from `seed` (Og, X: d*(l+1) doubles each).
cudaError_t launch_srqr_g2(const double* A, int64_t lda, int64_t l, int64_t d, uint64_t seed, double* Og, double* X,
                           double* info, const Status* st, cudaStream_t s);
size_t srqr_solve_smem(int64_t l);
// one swap: round robin of columns imax..l, Givens re-triangularisation (cs: 2*(l+1) doubles),
// r_l = R(l,l)^2 and r_i += R(l,i)^2.
cudaError_t launch_srqr_swap(double* A, int64_t lda, int64_t l, int64_t n, int64_t imax, int32_t* jpvt, double* cs,
                             double* r, const Status* st, cudaStream_t s);

// Opt-in kernel timing (prof.cu): classes in the order of rqrcp_profile_class_name.
enum ProfClass {
    K_OMEGA = 0, K_SKETCH_GEMM, K_SKETCH_REDUCE, K_PIVOT, K_SWAP, K_PANEL,
    K_WY_GEMM, K_TFORM, K_REDUCE_Y, K_WY_UPDATE, K_BUPDATE, K_LOWRANK_MISC, K_BACKWARD, K_BATCHED
};
bool prof_on();
void prof_begin(int cls, cudaStream_t s);
void prof_end(int cls, double flops, double bytes, cudaStream_t s);

}  // namespace rq
