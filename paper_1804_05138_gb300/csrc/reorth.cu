// reorth.cu -- FP64 Q1 and R from the mixed (FP32) factorization, with one CholQR
// reorthogonalisation pass applied when ||Q1^T Q1 - I||_F exceeds a tolerance:
//   G = Q1^T Q1,  G = S^T S (Cholesky, S upper),  Q1 <- Q1 S^{-1},  [R11 R12] <- S [R11 R12],
// which leaves Q1 [R11 R12] unchanged in exact arithmetic.  The decision is taken on the device
// (a flag in the workspace) so the whole sequence runs without a host synchronisation.
// Not in the paper: it restores FP64 orthogonality to the Q1 of the FP32 form.
#include <cmath>

#include "internal.cuh"

namespace rq {

template <typename T>
int lowrank_q1_only(int64_t m, int64_t k, const T* Afact, int64_t ldaf, const double* tau, T* Q1, int64_t ldq,
                    void* work, size_t work_bytes, cudaStream_t s);

namespace {

constexpr int kBlk = 64;
constexpr size_t kAl = 256;
size_t alr(size_t x) { return (x + kAl - 1) & ~(kAl - 1); }

// V64(r, c) = Afact(r, c) widened to FP64 (the reflector columns 0..k-1).
__global__ void widen_kernel(const float* __restrict__ A, int64_t lda, int64_t m, int64_t k, double* __restrict__ V)
{
    for (int64_t c = blockIdx.y; c < k; c += gridDim.y)
        for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < m; r += (int64_t)gridDim.x * blockDim.x)
            V[c * m + r] = (double)A[c * lda + r];
}

// R(q, c) = Afact(q, c) for q <= c, 0 below (k x n), FP64.
__global__ void rfp64_kernel(const float* __restrict__ A, int64_t lda, int64_t k, int64_t n, double* __restrict__ R,
                             int64_t ldr)
{
    for (int64_t c = blockIdx.x; c < n; c += gridDim.x)
        for (int64_t q = threadIdx.x; q < k; q += blockDim.x) R[c * ldr + q] = (q <= c) ? (double)A[c * lda + q] : 0.0;
}

// G = sum of the split-K partials (k x k); per-block partial sums of ||G - I||_F^2.
__global__ void gram_kernel(const double* __restrict__ P, int nsplit, int64_t k, double* __restrict__ G,
                            double* __restrict__ blocksum)
{
    __shared__ double red[256];
    double acc = 0.0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < k * k; e += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int sp = 0; sp < nsplit; ++sp) s += P[(int64_t)sp * k * k + e];
        G[e] = s;
        const int64_t a = e % k, b = e / k;
        const double d = s - (a == b ? 1.0 : 0.0);
        acc += d * d;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) blocksum[blockIdx.x] = red[0];
}

// orth = sqrt(sum of block sums) (fixed order); flag = orth > tol.
__global__ void orth_kernel(const double* __restrict__ blocksum, int nblocks, double tol, double* __restrict__ orth,
                            int* __restrict__ flag)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < nblocks; ++i) s += blocksum[i];
        const double o = sqrt(s);
        *orth = o;
        *flag = (o > tol) ? 1 : 0;
    }
}

// Cholesky G = L L^T (lower triangle of G as the working copy), one cooperative kernel: at step
// j every block reads column j (finished by its owner at step j-1), forms d = sqrt(G(j,j)) and
// l = G(j:k, j)/d, and updates the columns c > j it owns (c = g mod nblocks): G(c:k, c) -= l_c l(c:k).
// The owner of column j writes S(j, j:k) = l^T into Su (the upper factor S = L^T), a separate
// buffer, so no block reads a column while it is rewritten.  A non-positive pivot records
// RQRCP_ERR_NONFINITE.
__global__ void chol_kernel(double* __restrict__ G, int64_t k, double* __restrict__ Su, const int* __restrict__ flag,
                            Status* st)
{
    if (*flag == 0 || status_error(st)) return;
    extern __shared__ double col[];  // l(j:k)
    const int nb = gridDim.x, g = blockIdx.x;
    for (int64_t j = 0; j < k; ++j) {
        for (int64_t r = j + threadIdx.x; r < k; r += blockDim.x) col[r - j] = ld_cg(&G[j * k + r]);
        __syncthreads();
        const double gjj = col[0];
        if (!(gjj > 0.0)) {
            if (threadIdx.x == 0 && g == 0) set_error(st, RQRCP_ERR_NONFINITE);
            return;
        }
        const double d = sqrt(gjj);
        for (int64_t r = threadIdx.x; r < k - j; r += blockDim.x) col[r] = (r == 0) ? d : col[r] / d;
        __syncthreads();
        if ((j % nb) == g)
            for (int64_t r = j + threadIdx.x; r < k; r += blockDim.x) Su[r * k + j] = col[r - j];
        for (int64_t c = j + 1 + ((g - (j + 1) % nb) + nb) % nb; c < k; c += nb) {
            const double lc = col[c - j];
            for (int64_t r = c + threadIdx.x; r < k; r += blockDim.x) G[c * k + r] -= lc * col[r - j];
        }
        if (!grid_barrier(st)) return;
    }
}

// Off-diagonal block for the solve: Sb[c * jb + q] = S(j0 + q, j1 + c), c < k - j1.
__global__ void s_block_kernel(const double* __restrict__ Su, int64_t k, int64_t j0, int jb, int64_t j1,
                               double* __restrict__ Sb, const int* __restrict__ flag)
{
    if (*flag == 0) return;
    for (int64_t c = blockIdx.x; c < k - j1; c += gridDim.x)
        for (int q = threadIdx.x; q < jb; q += blockDim.x) Sb[c * jb + q] = Su[(j1 + c) * k + j0 + q];
}

// Forward substitution on rows of X, in place, for the diagonal block J = [j0, j0+jb) of X S = Q:
// x_j = (q_j - sum_{i<j in J} S(i, j) x_i) / S(j, j).
__global__ void trsm_fwd_kernel(double* __restrict__ X, int64_t ldx, int64_t m, const double* __restrict__ Su, int64_t k,
                                int64_t j0, int jb, const int* __restrict__ flag)
{
    if (*flag == 0) return;
    __shared__ double Ls[kBlk * kBlk];  // Ls[i * jb + j] = S(j0 + i, j0 + j), j >= i
    for (int e = threadIdx.x; e < jb * jb; e += blockDim.x) {
        const int j = e % jb, i = e / jb;
        Ls[e] = (j >= i) ? Su[(j0 + j) * k + j0 + i] : 0.0;
    }
    __syncthreads();
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < m; r += (int64_t)gridDim.x * blockDim.x) {
        for (int j = 0; j < jb; ++j) {
            double s = X[(j0 + j) * ldx + r];
            for (int i = 0; i < j; ++i) s -= Ls[i * jb + j] * X[(j0 + i) * ldx + r];
            X[(j0 + j) * ldx + r] = s / Ls[j * jb + j];
        }
    }
}

// Y = -R (k x n, ld k) in FP64 for the update GEMM; R <- Rnew afterwards.
__global__ void neg_copy_kernel(const double* __restrict__ R, int64_t ldr, int64_t k, int64_t n, double* __restrict__ Y,
                                const int* __restrict__ flag)
{
    if (*flag == 0) return;
    for (int64_t c = blockIdx.x; c < n; c += gridDim.x)
        for (int64_t q = threadIdx.x; q < k; q += blockDim.x) Y[c * k + q] = -R[c * ldr + q];
}

__global__ void zero_or_keep_kernel(double* __restrict__ C, int64_t ldc, int64_t k, int64_t n, const int* __restrict__ flag)
{
    if (*flag == 0) return;
    for (int64_t c = blockIdx.x; c < n; c += gridDim.x)
        for (int64_t q = threadIdx.x; q < k; q += blockDim.x) C[c * ldc + q] = 0.0;
}

__global__ void copy_back_kernel(const double* __restrict__ C, int64_t k, int64_t n, double* __restrict__ R, int64_t ldr,
                                 const int* __restrict__ flag)
{
    if (*flag == 0) return;
    for (int64_t c = blockIdx.x; c < n; c += gridDim.x)
        for (int64_t q = threadIdx.x; q < k; q += blockDim.x) R[c * ldr + q] = C[c * k + q];
}

// Flag-gated wrapper so the update GEMM is skipped when no reorthogonalisation is needed:
// the status block's error field is reused as the gate (set to a private code when not needed).
__global__ void gate_kernel(Status* st, const int* __restrict__ flag)
{
    if (threadIdx.x == 0 && blockIdx.x == 0 && *flag == 0) atomicCAS(&st->error, 0, -1);
}

__global__ void ungate_kernel(Status* st)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) atomicCAS(&st->error, -1, 0);
}

unsigned gcap(int64_t want)
{
    if (want < 1) return 1;
    const int64_t cap = (int64_t)dev_info().sms * 8;
    return (unsigned)(want > cap ? cap : want);
}

struct ReLayout {
    size_t status, flag, orth, blocksum, P, G, Su, Sb, V64, Y, Rn, lowrank, total;
};

ReLayout re_layout(int64_t m, int64_t n, int64_t k, size_t lowrank_bytes)
{
    ReLayout L{};
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = alr(off + bytes);
        return o;
    };
    L.status = take(sizeof(Status));
    L.flag = take(sizeof(int));
    L.orth = take(sizeof(double));
    L.blocksum = take(1024 * sizeof(double));
    L.P = take((size_t)16 * k * k * sizeof(double));
    L.G = take((size_t)k * k * sizeof(double));
    L.Su = take((size_t)k * k * sizeof(double));
    L.Sb = take((size_t)kBlk * k * sizeof(double));
    L.V64 = take((size_t)m * k * sizeof(double));
    L.Y = take((size_t)k * n * sizeof(double));
    L.Rn = take((size_t)k * n * sizeof(double));
    L.lowrank = take(lowrank_bytes);
    L.total = off;
    return L;
}

#define RQR_CHECK(expr)                 \
    do {                                \
        if ((expr) != cudaSuccess) {    \
            cudaGetLastError();         \
            return RQRCP_ERR_CUDA;      \
        }                               \
    } while (0)

}  // namespace
}  // namespace rq

using namespace rq;

extern "C" size_t rqrcp_lowrank_workspace_size(int64_t m, int64_t n, int64_t k);

extern "C" {

__attribute__((visibility("default"))) size_t rqrcp_reorth_workspace_size(int64_t m, int64_t n, int64_t k)
{
    if (m < 1 || n < 1 || k < 1 || k > (m < n ? m : n)) return 0;
    return re_layout(m, n, k, rqrcp_lowrank_workspace_size(m, k, k)).total;
}

__attribute__((visibility("default"))) int rqrcp_lowrank_reorth(int64_t m, int64_t n, int64_t k, const float* Afact,
                                                                int64_t ldaf, const double* tau, double* Q1,
                                                                int64_t ldq, double* R, int64_t ldr, double tol,
                                                                double* orth, void* work, size_t work_bytes,
                                                                void* stream)
{
    if (m < 1) return -1;
    if (n < 1) return -2;
    if (k < 1 || k > (m < n ? m : n)) return -3;
    if (Afact == nullptr) return -4;
    if (ldaf < m) return -5;
    if (tau == nullptr) return -6;
    if (Q1 == nullptr) return -7;
    if (ldq < m) return -8;
    if (R == nullptr) return -9;
    if (ldr < k) return -10;
    if (!(tol >= 0.0)) return -11;
    const size_t lr_bytes = rqrcp_lowrank_workspace_size(m, k, k);
    const ReLayout L = re_layout(m, n, k, lr_bytes);
    if (work == nullptr || (reinterpret_cast<uintptr_t>(work) & (kAl - 1)) != 0 || work_bytes < L.total)
        return RQRCP_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    char* w = static_cast<char*>(work);
    Status* st = reinterpret_cast<Status*>(w + L.status);
    int* flag = reinterpret_cast<int*>(w + L.flag);
    double* orth_dev = reinterpret_cast<double*>(w + L.orth);
    double* blocksum = reinterpret_cast<double*>(w + L.blocksum);
    double* P = reinterpret_cast<double*>(w + L.P);
    double* G = reinterpret_cast<double*>(w + L.G);
    double* Su = reinterpret_cast<double*>(w + L.Su);
    double* Sb = reinterpret_cast<double*>(w + L.Sb);
    double* V64 = reinterpret_cast<double*>(w + L.V64);
    double* Y = reinterpret_cast<double*>(w + L.Y);
    double* Rn = reinterpret_cast<double*>(w + L.Rn);
    void* lr_work = w + L.lowrank;
    const bool prof = prof_on();
    if (prof) prof_begin(K_LOWRANK_MISC, s);

    // FP64 Q1 from the FP32 reflectors, FP64 R = triu(Afact(0:k, :))
    const int64_t gx = (m + 255) / 256 > 16 ? 16 : (m + 255) / 256;
    widen_kernel<<<dim3((unsigned)gx, gcap(k)), 256, 0, s>>>(Afact, ldaf, m, k, V64);
    RQR_CHECK(cudaGetLastError());
    if (int e = lowrank_q1_only<double>(m, k, V64, m, tau, Q1, ldq, lr_work, lr_bytes, s)) return e;
    rfp64_kernel<<<gcap(n), 256, 0, s>>>(Afact, ldaf, k, n, R, ldr);
    RQR_CHECK(cudaGetLastError());
    RQR_CHECK(launch_init(st, k, nullptr, 0, s));
    // G = Q1^T Q1 and ||G - I||_F
    {
        const int64_t tiles = ((k + 63) / 64) * ((k + 63) / 64);
        int64_t S = (4 * (int64_t)dev_info().sms + tiles - 1) / tiles;
        if (S > 16) S = 16;
        if (S > (m + 63) / 64) S = (m + 63) / 64;
        if (S < 1) S = 1;
        int64_t kc = (m + S - 1) / S;
        kc = ((kc + 15) / 16) * 16;
        const int ns = (int)((m + kc - 1) / kc);
        RQR_CHECK(launch_gemm_tn<double>(Q1, ldq, Q1, ldq, k, k, m, kc, P, 0, 0, st, s));
        const unsigned nbs = gcap((k * k + 255) / 256) > 1024 ? 1024 : gcap((k * k + 255) / 256);
        gram_kernel<<<nbs, 256, 0, s>>>(P, ns, k, G, blocksum);
        RQR_CHECK(cudaGetLastError());
        orth_kernel<<<1, 32, 0, s>>>(blocksum, (int)nbs, tol, orth_dev, flag);
        RQR_CHECK(cudaGetLastError());
    }
    // Cholesky (cooperative), gated by the flag
    {
        static DevFlag attr_set;
        if (!attr_set.done()) {
            if (allow_max_dynamic_smem(chol_kernel) != cudaSuccess) {
                cudaGetLastError();
                return RQRCP_ERR_CUDA;
            }
            attr_set.set();
        }
        const size_t smem = sizeof(double) * (size_t)k;
        int per_sm = 0;
        RQR_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, chol_kernel, 256, smem));
        int64_t nb = k < dev_info().sms ? k : dev_info().sms;
        if (nb > (int64_t)per_sm * dev_info().sms) nb = (int64_t)per_sm * dev_info().sms;
        RQR_CHECK(cudaMemsetAsync(Su, 0, sizeof(double) * (size_t)k * k, s));
        int64_t kv = k;
        void* args[] = {&G, &kv, &Su, &flag, &st};
        RQR_CHECK(cudaLaunchCooperativeKernel((const void*)chol_kernel, dim3((unsigned)nb), dim3(256), args, smem, s));
    }
    gate_kernel<<<1, 32, 0, s>>>(st, flag);
    RQR_CHECK(cudaGetLastError());
    // Q1 <- Q1 S^{-1}: diagonal blocks forward, later columns updated with the update GEMM
    for (int64_t j0 = 0; j0 < k; j0 += kBlk) {
        const int jb = (int)(kBlk < k - j0 ? kBlk : k - j0);
        trsm_fwd_kernel<<<gcap((m + 127) / 128), 128, 0, s>>>(Q1, ldq, m, Su, k, j0, jb, flag);
        RQR_CHECK(cudaGetLastError());
        const int64_t j1 = j0 + jb;
        if (j1 < k) {
            s_block_kernel<<<gcap(k - j1), 64, 0, s>>>(Su, k, j0, jb, j1, Sb, flag);
            RQR_CHECK(cudaGetLastError());
            RQR_CHECK(launch_gemm_update<double>(Q1 + j1 * ldq, ldq, Q1 + j0 * ldq, ldq, Sb, jb, m, k - j1, jb, 0,
                                                 nullptr, st, s));
        }
    }
    // [R11 R12] <- S [R11 R12]:  Rn = 0;  Rn -= S (-R);  R = Rn
    neg_copy_kernel<<<gcap(n), 256, 0, s>>>(R, ldr, k, n, Y, flag);
    zero_or_keep_kernel<<<gcap(n), 256, 0, s>>>(Rn, k, k, n, flag);
    RQR_CHECK(cudaGetLastError());
    RQR_CHECK(launch_gemm_update<double>(Rn, k, Su, k, Y, k, k, n, k, 0, nullptr, st, s));
    copy_back_kernel<<<gcap(n), 256, 0, s>>>(Rn, k, n, R, ldr, flag);
    RQR_CHECK(cudaGetLastError());
    ungate_kernel<<<1, 32, 0, s>>>(st);
    RQR_CHECK(cudaGetLastError());
    if (orth) RQR_CHECK(cudaMemcpyAsync(orth, orth_dev, sizeof(double), cudaMemcpyDeviceToDevice, s));
    if (prof) prof_end(K_LOWRANK_MISC, 2.0 * m * (double)k * k + (double)m * k * k + 2.0 * (double)k * k * n,
                       8.0 * (3.0 * m * k + 2.0 * (double)k * n), s);
    return RQRCP_OK;
}

}  // extern "C"
