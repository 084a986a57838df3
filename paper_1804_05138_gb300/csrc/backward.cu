// backward.cu -- adjoint of the truncated factorization with the permutation held fixed.
//
// Forward (what RQRCP computes for the first k columns): X = A Pi = [X1 X2], X1 = Q1 R11
// (Householder QR), R12 = Q1^T X2.  Given upstream gradients dQ1 (m x k) and dR = [dR11 dR12]
// (k x n, only the upper triangle of dR11 counts), the gradient with respect to A is
//   dX2 = Q1 dR12
//   dQ' = dQ1 + X2 dR12^T
//   M   = R11 dR11^T - dQ'^T Q1,   C = copyltu(M) = tril(M) + tril(M,-1)^T
//   dX1 = (dQ' + Q1 C) R11^{-T}
//   dA(:, jpvt[c]) = dX(:, c).
// This is the thin-QR adjoint (X1 = Q1 R11) plus the wide block R12 = Q1^T X2; the paper has no
// backward, it is the differentiable form built on its factorization.  Contractions reuse the
// split-K and update GEMM kernels; R11^{-T} is a blocked back substitution (64-column diagonal
// blocks solved row-parallel, off-diagonal blocks applied with the update GEMM).
#include "internal.cuh"

namespace rq {
namespace {

constexpr int kTrsmBlock = 64;

// Y1[c * k + q] = -dR(q, k + c): the k x (n-k) block -dR12 in FP64.
template <typename T>
__global__ void neg_dr12_kernel(const T* __restrict__ dR, int64_t lddr, int64_t k, int64_t nt, double* __restrict__ Y1)
{
    for (int64_t c = blockIdx.x; c < nt; c += gridDim.x)
        for (int64_t q = threadIdx.x; q < k; q += blockDim.x) Y1[c * k + q] = -(double)dR[(k + c) * lddr + q];
}

// Y2[q * nt + c] = -dR(q, k + c): the (n-k) x k block -dR12^T in FP64.
template <typename T>
__global__ void neg_dr12t_kernel(const T* __restrict__ dR, int64_t lddr, int64_t k, int64_t nt, double* __restrict__ Y2)
{
    for (int64_t q = blockIdx.x; q < k; q += gridDim.x)
        for (int64_t c = threadIdx.x; c < nt; c += blockDim.x) Y2[q * nt + c] = -(double)dR[(k + c) * lddr + q];
}

// dst(:, dstmap ? dstmap[c] : c) = src(:, srcmap ? srcmap[c] : c), m rows, nc columns.
template <typename T>
__global__ void copy_cols_kernel(const T* __restrict__ src, int64_t lds, const int32_t* __restrict__ srcmap,
                                 T* __restrict__ dst, int64_t ldd, const int32_t* __restrict__ dstmap, int64_t m,
                                 int64_t nc)
{
    for (int64_t c = blockIdx.y; c < nc; c += gridDim.y) {
        const int64_t cs = srcmap ? (int64_t)srcmap[c] : c;
        const int64_t cd = dstmap ? (int64_t)dstmap[c] : c;
        for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < m; r += (int64_t)gridDim.x * blockDim.x)
            dst[cd * ldd + r] = src[cs * lds + r];
    }
}

// Cneg(a,b) = Cneg(b,a) = -M(a,b) for a >= b, with M = R11 dR11^T - W and W(a,b) the split-K
// sum of dQ'^T Q1 (P[sp][b][a]).  R11 and dR11 are read as upper triangular.
template <typename T>
__global__ void mfuse_kernel(const T* __restrict__ R, int64_t ldr, const T* __restrict__ dR, int64_t lddr,
                             const double* __restrict__ P, int nsplit, int64_t k, double* __restrict__ Cneg)
{
    const int64_t total = k * k;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t a = e % k, b = e / k;
        if (a < b) continue;
        double s = 0.0;
        for (int64_t q = a; q < k; ++q) s += (double)R[q * ldr + a] * (double)dR[q * lddr + b];
        double w = 0.0;
        for (int sp = 0; sp < nsplit; ++sp) w += P[((int64_t)sp * k + b) * k + a];
        const double mab = s - w;
        Cneg[b * k + a] = -mab;
        Cneg[a * k + b] = -mab;
    }
}

// In place on rows of Z: solve X(:, J) R11(J, J)^T = Z(:, J), J = [j0, j0 + jb), by back
// substitution x_j = (z_j - sum_{q > j} R11(j, q) x_q) / R11(j, j); one thread per row.
template <typename T>
__global__ void trsm_diag_kernel(T* __restrict__ Z, int64_t ldz, int64_t m, const T* __restrict__ R, int64_t ldr,
                                 int64_t j0, int jb)
{
    __shared__ double Rs[kTrsmBlock * kTrsmBlock];  // Rs[q * jb + j] = R11(j0 + j, j0 + q)
    for (int e = threadIdx.x; e < jb * jb; e += blockDim.x) {
        const int j = e % jb, q = e / jb;
        Rs[e] = (q >= j) ? (double)R[(j0 + q) * ldr + j0 + j] : 0.0;
    }
    __syncthreads();
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < m; r += (int64_t)gridDim.x * blockDim.x) {
        for (int j = jb - 1; j >= 0; --j) {
            double s = (double)Z[(j0 + j) * ldz + r];
            for (int q = j + 1; q < jb; ++q) s -= Rs[q * jb + j] * (double)Z[(j0 + q) * ldz + r];
            const double d = Rs[j * jb + j];
            Z[(j0 + j) * ldz + r] = (T)((d == 0.0) ? 0.0 : s / d);
        }
    }
}

// Y3[c * jb + q] = R11(c, j0 + q) for c < j0: the block R11(0:j0, J)^T in FP64.
template <typename T>
__global__ void r11t_block_kernel(const T* __restrict__ R, int64_t ldr, int64_t j0, int jb, double* __restrict__ Y3)
{
    for (int64_t c = blockIdx.x; c < j0; c += gridDim.x)
        for (int q = threadIdx.x; q < jb; q += blockDim.x) Y3[c * jb + q] = (double)R[(j0 + q) * ldr + c];
}

unsigned grid_cap(int64_t want)
{
    if (want < 1) return 1;
    const int64_t cap = (int64_t)dev_info().sms * 16;
    return (unsigned)(want > cap ? cap : want);
}

constexpr size_t kAlignB = 256;
size_t al(size_t x) { return (x + kAlignB - 1) & ~(kAlignB - 1); }
constexpr int kMaxSplitB = 16;

struct BwdLayout {
    size_t status, P, Y1, Y2, Cneg, Y3, X2, Qp, total;
};

BwdLayout bwd_layout(int64_t m, int64_t n, int64_t k, size_t esz)
{
    BwdLayout L{};
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = al(off + bytes);
        return o;
    };
    const int64_t nt = n - k;
    L.status = take(sizeof(Status));
    L.P = take((size_t)kMaxSplitB * k * k * sizeof(double));
    L.Y1 = take((size_t)k * (nt > 0 ? nt : 1) * sizeof(double));
    L.Y2 = take((size_t)k * (nt > 0 ? nt : 1) * sizeof(double));
    L.Cneg = take((size_t)k * k * sizeof(double));
    L.Y3 = take((size_t)kTrsmBlock * k * sizeof(double));
    L.X2 = take((size_t)m * (nt > 0 ? nt : 1) * esz);
    L.Qp = take((size_t)m * k * esz);
    L.total = off;
    return L;
}

#define RQB_CHECK(expr)                 \
    do {                                \
        if ((expr) != cudaSuccess) {    \
            cudaGetLastError();         \
            return RQRCP_ERR_CUDA;      \
        }                               \
    } while (0)

template <typename T>
int backward_impl(int64_t m, int64_t n, int64_t k, const T* A, int64_t lda, const int32_t* jpvt, const T* Q1,
                  int64_t ldq, const T* R, int64_t ldr, const T* dQ1, int64_t lddq, const T* dR, int64_t lddr, T* dA,
                  int64_t ldda, void* work, size_t work_bytes, cudaStream_t s)
{
    if (m < 1) return -1;
    if (n < 1) return -2;
    if (k < 1 || k > (m < n ? m : n)) return -3;
    if (A == nullptr) return -4;
    if (lda < m) return -5;
    if (jpvt == nullptr) return -6;
    if (Q1 == nullptr) return -7;
    if (ldq < m) return -8;
    if (R == nullptr) return -9;
    if (ldr < k) return -10;
    if (dQ1 == nullptr) return -11;
    if (lddq < m) return -12;
    if (dR == nullptr) return -13;
    if (lddr < k) return -14;
    if (dA == nullptr) return -15;
    if (ldda < m) return -16;
    const BwdLayout L = bwd_layout(m, n, k, sizeof(T));
    if (work == nullptr || (reinterpret_cast<uintptr_t>(work) & (kAlignB - 1)) != 0 || work_bytes < L.total)
        return RQRCP_ERR_WORKSPACE;
    char* w = static_cast<char*>(work);
    Status* st = reinterpret_cast<Status*>(w + L.status);
    double* P = reinterpret_cast<double*>(w + L.P);
    double* Y1 = reinterpret_cast<double*>(w + L.Y1);
    double* Y2 = reinterpret_cast<double*>(w + L.Y2);
    double* Cneg = reinterpret_cast<double*>(w + L.Cneg);
    double* Y3 = reinterpret_cast<double*>(w + L.Y3);
    T* X2 = reinterpret_cast<T*>(w + L.X2);
    T* Qp = reinterpret_cast<T*>(w + L.Qp);
    const int64_t nt = n - k;
    const bool prof = prof_on();
    if (prof) prof_begin(K_BACKWARD, s);

    RQB_CHECK(launch_init(st, k, nullptr, 0, s));
    RQB_CHECK(cudaMemset2DAsync(dA, ldda * sizeof(T), 0, m * sizeof(T), n, s));
    if (nt > 0) {
        // dX2 = Q1 dR12, scattered to columns jpvt[k..n)
        neg_dr12_kernel<T><<<grid_cap(nt), 128, 0, s>>>(dR, lddr, k, nt, Y1);
        RQB_CHECK(cudaGetLastError());
        RQB_CHECK(launch_gemm_update<T>(dA, ldda, Q1, ldq, Y1, k, m, nt, k, 0, jpvt + k, st, s));
    }
    // dQ' = dQ1 + X2 dR12^T
    copy_cols_kernel<T><<<dim3(grid_cap((m + 255) / 256 > 16 ? 16 : (m + 255) / 256), grid_cap(k)), 256, 0, s>>>(
        dQ1, lddq, nullptr, Qp, m, nullptr, m, k);
    RQB_CHECK(cudaGetLastError());
    if (nt > 0) {
        copy_cols_kernel<T><<<dim3(grid_cap((m + 255) / 256 > 16 ? 16 : (m + 255) / 256), grid_cap(nt)), 256, 0, s>>>(
            A, lda, jpvt + k, X2, m, nullptr, m, nt);
        RQB_CHECK(cudaGetLastError());
        neg_dr12t_kernel<T><<<grid_cap(k), 256, 0, s>>>(dR, lddr, k, nt, Y2);
        RQB_CHECK(cudaGetLastError());
        RQB_CHECK(launch_gemm_update<T>(Qp, m, X2, m, Y2, nt, m, k, nt, 0, nullptr, st, s));
    }
    // W = dQ'^T Q1 (split-K), M = R11 dR11^T - W, Cneg = -copyltu(M)
    {
        const int64_t tiles = ((k + 63) / 64) * ((k + 63) / 64);
        int64_t S = (4 * (int64_t)dev_info().sms + tiles - 1) / tiles;
        if (S > kMaxSplitB) S = kMaxSplitB;
        if (S > (m + 63) / 64) S = (m + 63) / 64;
        if (S < 1) S = 1;
        int64_t kc = (m + S - 1) / S;
        kc = ((kc + 15) / 16) * 16;
        const int ns = (int)((m + kc - 1) / kc);
        RQB_CHECK(launch_gemm_tn<T>(Qp, m, Q1, ldq, k, k, m, kc, P, 0, 0, st, s));
        mfuse_kernel<T><<<grid_cap((k * k + 255) / 256), 256, 0, s>>>(R, ldr, dR, lddr, P, ns, k, Cneg);
        RQB_CHECK(cudaGetLastError());
    }
    // Z = dQ' + Q1 copyltu(M)
    RQB_CHECK(launch_gemm_update<T>(Qp, m, Q1, ldq, Cneg, k, m, k, k, 0, nullptr, st, s));
    // dX1 = Z R11^{-T}: diagonal blocks from the last one backwards
    for (int64_t j1 = k; j1 > 0;) {
        const int64_t j0 = j1 > kTrsmBlock ? j1 - kTrsmBlock : 0;
        const int jb = (int)(j1 - j0);
        trsm_diag_kernel<T><<<grid_cap((m + 127) / 128), 128, 0, s>>>(Qp, m, m, R, ldr, j0, jb);
        RQB_CHECK(cudaGetLastError());
        if (j0 > 0) {
            r11t_block_kernel<T><<<grid_cap(j0), 64, 0, s>>>(R, ldr, j0, jb, Y3);
            RQB_CHECK(cudaGetLastError());
            RQB_CHECK(launch_gemm_update<T>(Qp, m, Qp + j0 * m, m, Y3, jb, m, j0, jb, 0, nullptr, st, s));
        }
        j1 = j0;
    }
    // dA(:, jpvt[c]) = dX1(:, c), c < k
    copy_cols_kernel<T><<<dim3(grid_cap((m + 255) / 256 > 16 ? 16 : (m + 255) / 256), grid_cap(k)), 256, 0, s>>>(
        Qp, m, nullptr, dA, ldda, jpvt, m, k);
    RQB_CHECK(cudaGetLastError());
    if (prof) {
        const double fl = 4.0 * m * (double)nt * k + 4.0 * m * (double)k * k + (double)m * k * k;
        prof_end(K_BACKWARD, fl, (double)sizeof(T) * (2.0 * m * n + 3.0 * m * k), s);
    }
    return RQRCP_OK;
}

}  // namespace
}  // namespace rq

using namespace rq;

extern "C" {

__attribute__((visibility("default"))) size_t rqrcp_backward_workspace_size(int64_t m, int64_t n, int64_t k,
                                                                            int precision)
{
    if (m < 1 || n < 1 || k < 1 || k > (m < n ? m : n)) return 0;
    if (precision != RQRCP_PREC_FP64 && precision != RQRCP_PREC_MIXED) return 0;
    return bwd_layout(m, n, k, precision == RQRCP_PREC_FP64 ? sizeof(double) : sizeof(float)).total;
}

__attribute__((visibility("default"))) int rqrcp_backward(int64_t m, int64_t n, int64_t k, const double* A, int64_t lda,
                                                          const int32_t* jpvt, const double* Q1, int64_t ldq,
                                                          const double* R, int64_t ldr, const double* dQ1,
                                                          int64_t lddq, const double* dR, int64_t lddr, double* dA,
                                                          int64_t ldda, void* work, size_t work_bytes, void* stream)
{
    return backward_impl<double>(m, n, k, A, lda, jpvt, Q1, ldq, R, ldr, dQ1, lddq, dR, lddr, dA, ldda, work,
                                 work_bytes, (cudaStream_t)stream);
}

__attribute__((visibility("default"))) int rqrcp_backward_f32(int64_t m, int64_t n, int64_t k, const float* A,
                                                              int64_t lda, const int32_t* jpvt, const float* Q1,
                                                              int64_t ldq, const float* R, int64_t ldr,
                                                              const float* dQ1, int64_t lddq, const float* dR,
                                                              int64_t lddr, float* dA, int64_t ldda, void* work,
                                                              size_t work_bytes, void* stream)
{
    return backward_impl<float>(m, n, k, A, lda, jpvt, Q1, ldq, R, ldr, dQ1, lddq, dR, lddr, dA, ldda, work,
                                work_bytes, (cudaStream_t)stream);
}

}  // extern "C"
