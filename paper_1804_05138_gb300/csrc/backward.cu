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

// ipiv[jpvt[c]] = c: the inverse permutation.
__global__ void ipiv_kernel(const int32_t* __restrict__ jpvt, int64_t n, int32_t* __restrict__ ipiv)
{
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x)
        ipiv[jpvt[c]] = (int32_t)c;
}

// FP32: C(a, b) = C(b, a) = M(a, b) for a >= b, M = R11 dR11^T - W with W(a, b) the sum (in FP64) of
// the split partials P[(z k + b) k + a] of dQ'^T Q1.  A block of 32 x 8 threads covers the 32 x 32
// tile of rows a and columns b; R11(a, q) and dR11(b, q) for 32 values of q at a time are staged in
// shared memory, and each thread sums its four columns b over q >= a (R11 and dR11 read as upper
// triangular).
__global__ void mfuse_f32_kernel(const float* __restrict__ R, int64_t ldr, const float* __restrict__ dR, int64_t lddr,
                                 const float* __restrict__ P, int nz, int64_t k, float* __restrict__ C)
{
    if (blockIdx.x < blockIdx.y) return;  // the tile lies above the diagonal
    __shared__ float Ra[32][33], Db[32][33];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int64_t a0 = (int64_t)blockIdx.x * 32, b0 = (int64_t)blockIdx.y * 32;
    const int64_t a = a0 + tx;
    float s[4] = {0.f, 0.f, 0.f, 0.f};
    for (int64_t q0 = a0; q0 < k; q0 += 32) {
        for (int qq = ty; qq < 32; qq += 8) {
            const int64_t q = q0 + qq;
            Ra[qq][tx] = (q < k && a < k) ? R[q * ldr + a] : 0.f;
            Db[qq][tx] = (q < k && b0 + tx < k) ? dR[q * lddr + b0 + tx] : 0.f;
        }
        __syncthreads();
#pragma unroll 8
        for (int qq = 0; qq < 32; ++qq) {
            const float ra = (q0 + qq >= a) ? Ra[qq][tx] : 0.f;
#pragma unroll
            for (int i = 0; i < 4; ++i) s[i] = fmaf(ra, Db[qq][ty + 8 * i], s[i]);
        }
        __syncthreads();
    }
    if (a >= k) return;
    double w[4] = {0.0, 0.0, 0.0, 0.0};
    for (int z0 = 0; z0 < nz; z0 += 4) {  // 16 loads in flight per step
        float pv[4][4];
#pragma unroll
        for (int zz = 0; zz < 4; ++zz)
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int64_t b = b0 + ty + 8 * i;
                pv[zz][i] = (z0 + zz < nz && b < k) ? P[((int64_t)(z0 + zz) * k + b) * k + a] : 0.f;
            }
#pragma unroll
        for (int zz = 0; zz < 4; ++zz)
#pragma unroll
            for (int i = 0; i < 4; ++i) w[i] += (double)pv[zz][i];
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int64_t b = b0 + ty + 8 * i;
        if (b >= k || a < b) continue;
        const float mab = (float)((double)s[i] - w[i]);
        C[b * k + a] = mab;
        C[a * k + b] = mab;
    }
}

// Back substitution on 32 unknowns held in registers against the upper triangle of Rs (leading
// dimension 32): x_j <- x_j rinv[j], then x_i -= Rs[j 32 + i] x_j for i < j.
__device__ __forceinline__ void solve32(float (&x)[32], const float* Rs, const float* rinv)
{
#pragma unroll
    for (int j = 31; j >= 0; --j) {
        x[j] *= rinv[j];
        const float xj = x[j];
#pragma unroll
        for (int i4 = 0; 4 * i4 < j; ++i4) {
            const float4 rr = *reinterpret_cast<const float4*>(Rs + j * 32 + 4 * i4);
            x[4 * i4] = fmaf(-rr.x, xj, x[4 * i4]);
            x[4 * i4 + 1] = fmaf(-rr.y, xj, x[4 * i4 + 1]);
            x[4 * i4 + 2] = fmaf(-rr.z, xj, x[4 * i4 + 2]);
            x[4 * i4 + 3] = fmaf(-rr.w, xj, x[4 * i4 + 3]);
        }
    }
}

// FP32, in place on rows of Z: solve X(:, J) R11(J, J)^T = Z(:, J) - X(:, C) R11(J, C)^T for
// J = [j0, j0 + jb), jb <= 32, with the already solved columns C = [j0 + 32, j0 + 32 + nc) read back
// from Z (nc <= 32).  One thread per row, the 32 unknowns in registers, column-oriented back
// substitution (x_j <- x_j / R11(j, j), then x_i -= R11(i, j) x_j for i < j).  The solved block
// goes back to Z (later blocks' updates read it) and to dA(:, jpvt[j0 + j]).
__global__ void __launch_bounds__(64) trsm_rows_f32_kernel(float* __restrict__ Z, int64_t ldz, int64_t m,
                                                           const float* __restrict__ R, int64_t ldr, int64_t j0, int jb,
                                                           int nc, const int32_t* __restrict__ jpvt,
                                                           float* __restrict__ dA, int64_t ldda)
{
    __shared__ __align__(16) float Rs[64 * 32];  // Rs[j * 32 + i] = R11(j0 + i, j0 + j), i < 32, j < 64
    __shared__ float rinv[32];
    __shared__ int64_t dcol[32];
    // staging: all 32 loads of a thread issued together (64 threads, blockDim must be 64)
    float rv[32];
#pragma unroll
    for (int u = 0; u < 32; ++u) {
        const int e = threadIdx.x + 64 * u;
        const int i = e % 32, j = e / 32;
        const bool use = i < jb && ((j < jb && i < j) || (j >= 32 && j < 32 + nc));
        rv[u] = use ? R[(j0 + j) * ldr + j0 + i] : 0.f;
    }
#pragma unroll
    for (int u = 0; u < 32; ++u) Rs[threadIdx.x + 64 * u] = rv[u];
    for (int j = threadIdx.x; j < 32; j += blockDim.x) {
        const float d = j < jb ? R[(j0 + j) * ldr + j0 + j] : 0.f;
        rinv[j] = d != 0.f ? 1.f / d : 0.f;
        dcol[j] = j < jb ? (int64_t)jpvt[j0 + j] : 0;
    }
    __syncthreads();
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < m; r += (int64_t)gridDim.x * blockDim.x) {
        float* zr = Z + j0 * ldz + r;
        float x[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) x[j] = j < jb ? zr[j * ldz] : 0.f;
        if (nc > 0) {
            float xc[32];  // the solved columns, loaded together
#pragma unroll
            for (int j = 0; j < 32; ++j) xc[j] = j < nc ? zr[(32 + j) * ldz] : 0.f;
#pragma unroll
            for (int j = 0; j < 32; ++j) {
#pragma unroll
                for (int i4 = 0; i4 < 8; ++i4) {
                    const float4 rr = *reinterpret_cast<const float4*>(Rs + (32 + j) * 32 + 4 * i4);
                    x[4 * i4] = fmaf(-rr.x, xc[j], x[4 * i4]);
                    x[4 * i4 + 1] = fmaf(-rr.y, xc[j], x[4 * i4 + 1]);
                    x[4 * i4 + 2] = fmaf(-rr.z, xc[j], x[4 * i4 + 2]);
                    x[4 * i4 + 3] = fmaf(-rr.w, xc[j], x[4 * i4 + 3]);
                }
            }
        }
        solve32(x, Rs, rinv);
#pragma unroll
        for (int j = 0; j < 32; ++j)
            if (j < jb) {
                zr[j * ldz] = x[j];
                dA[dcol[j] * ldda + r] = x[j];
            }
    }
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

// FP32 workspace of the tensor-core path: inverse permutation, B planes (one buffer reused by every
// contraction), split partials, C = copyltu(M), and dQ' / Z with a 16-byte-multiple leading dimension.
constexpr int kMaxSplitP2 = 8;

struct BwdTcLayout {
    size_t status, ipiv, planes, part, C, Qp, total;
    int64_t ldqp;
};

BwdTcLayout bwd_tc_layout(int64_t m, int64_t n, int64_t k)
{
    BwdTcLayout L{};
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = al(off + bytes);
        return o;
    };
    const int64_t nt = n - k;
    L.ldqp = (m + 3) / 4 * 4;
    size_t pl = mm_planes_bytes(k, nt > 0 ? nt : 1);
    for (size_t x : {mm_planes_bytes(n, k), mm_planes_bytes(m, k), mm_planes_bytes(k, k),
                     mm_planes_bytes(kTrsmBlock, k)})
        if (x > pl) pl = x;
    size_t part = (size_t)kMaxSplitP2 * L.ldqp * k;
    if ((size_t)mm_max_split() * k * k > part) part = (size_t)mm_max_split() * k * k;
    L.status = take(sizeof(Status));
    L.ipiv = take((size_t)n * sizeof(int32_t));
    L.planes = take(pl);
    L.part = take(part * sizeof(float));
    L.C = take((size_t)k * k * sizeof(float));
    L.Qp = take((size_t)L.ldqp * k * sizeof(float));
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

// FP32 backward with every contraction on the tensor cores (launch_mm_tc).  The column gather of X2
// is folded into the contraction dQ' = dQ1 + A B' (B'(j, q) = dR(q, ipiv[j]) for non-leading j,
// zero for the k leading columns), and every product that ends in dA writes its columns through
// jpvt, so dA needs no clearing and no final scatter.
int backward_f32_tc(int64_t m, int64_t n, int64_t k, const float* A, int64_t lda, const int32_t* jpvt,
                    const float* Q1, int64_t ldq, const float* R, int64_t ldr, const float* dQ1, int64_t lddq,
                    const float* dR, int64_t lddr, float* dA, int64_t ldda, char* w, cudaStream_t s)
{
    const BwdTcLayout L = bwd_tc_layout(m, n, k);
    Status* st = reinterpret_cast<Status*>(w + L.status);
    int32_t* ipiv = reinterpret_cast<int32_t*>(w + L.ipiv);
    float* PL = reinterpret_cast<float*>(w + L.planes);
    float* Part = reinterpret_cast<float*>(w + L.part);
    float* Cm = reinterpret_cast<float*>(w + L.C);
    float* Qp = reinterpret_cast<float*>(w + L.Qp);
    const int64_t ldqp = L.ldqp;
    const int64_t nt = n - k;
    RQB_CHECK(launch_init(st, k, nullptr, 0, s));
    ipiv_kernel<<<grid_cap((n + 255) / 256), 256, 0, s>>>(jpvt, n, ipiv);
    RQB_CHECK(cudaGetLastError());
    if (nt > 0) {
        // dA(:, jpvt[k + c]) = Q1 dR12
        RQB_CHECK(launch_mm_planes(dR + k * lddr, 1, lddr, nullptr, 0, k, nt, PL, st, s));
        RQB_CHECK(launch_mm_tc(false, Q1, ldq, PL, m, nt, k, 1, 1.f, 0.f, nullptr, 0, dA, ldda, 0, jpvt + k, st, s));
        // dQ' = dQ1 + X2 dR12^T = dQ1 + A B'
        RQB_CHECK(launch_mm_planes(dR, lddr, 1, ipiv, k, n, k, PL, st, s));
        int S2 = mm_choose_split(m, k, n, 8);
        if (S2 > kMaxSplitP2) S2 = kMaxSplitP2;
        if (S2 <= 1) {
            RQB_CHECK(launch_mm_tc(false, A, lda, PL, m, k, n, 1, 1.f, 1.f, dQ1, lddq, Qp, ldqp, 0, nullptr, st, s));
        } else {
            RQB_CHECK(launch_mm_tc(false, A, lda, PL, m, k, n, S2, 1.f, 0.f, nullptr, 0, Part, ldqp, ldqp * k, nullptr,
                                   st, s));
            RQB_CHECK(launch_mm_sum(Part, ldqp, ldqp * k, S2, m, k, dQ1, lddq, Qp, ldqp, st, s));
        }
    } else {
        RQB_CHECK(launch_mm_sum(nullptr, 0, 0, 0, m, k, dQ1, lddq, Qp, ldqp, st, s));
    }
    // W = dQ'^T Q1 (split partials), C = copyltu(R11 dR11^T - W)
    {
        RQB_CHECK(launch_mm_planes(Q1, 1, ldq, nullptr, 0, m, k, PL, st, s));
        const int S3 = mm_choose_split(k, k, m, 8);
        RQB_CHECK(launch_mm_tc(true, Qp, ldqp, PL, k, k, m, S3, 1.f, 0.f, nullptr, 0, Part, k, k * k, nullptr, st, s));
        const unsigned gt = (unsigned)((k + 31) / 32);
        mfuse_f32_kernel<<<dim3(gt, gt), dim3(32, 8), 0, s>>>(R, ldr, dR, lddr, Part, S3, k, Cm);
        RQB_CHECK(cudaGetLastError());
    }
    // Z = dQ' + Q1 C
    RQB_CHECK(launch_mm_planes(Cm, 1, k, nullptr, 0, k, k, PL, st, s));
    RQB_CHECK(launch_mm_tc(false, Q1, ldq, PL, m, k, k, 1, 1.f, 1.f, Qp, ldqp, Qp, ldqp, 0, nullptr, st, s));
    // dX1 = Z R11^{-T}, diagonal blocks from the last one backwards, written to dA(:, jpvt[0:k])
    for (int64_t j1 = k; j1 > 0;) {
        const int64_t j0 = j1 > kTrsmBlock ? j1 - kTrsmBlock : 0;
        const int jb = (int)(j1 - j0);
        if (jb > 32) {  // the upper half first, then the lower half coupled to it
            trsm_rows_f32_kernel<<<grid_cap((m + 63) / 64), 64, 0, s>>>(Qp, ldqp, m, R, ldr, j0 + 32, jb - 32, 0,
                                                                        jpvt, dA, ldda);
            RQB_CHECK(cudaGetLastError());
        }
        trsm_rows_f32_kernel<<<grid_cap((m + 63) / 64), 64, 0, s>>>(Qp, ldqp, m, R, ldr, j0, jb < 32 ? jb : 32,
                                                                    jb > 32 ? jb - 32 : 0, jpvt, dA, ldda);
        RQB_CHECK(cudaGetLastError());
        if (j0 > 0) {
            // Z(:, 0:j0) -= X(:, J) R11(0:j0, J)^T
            RQB_CHECK(launch_mm_planes(R + j0 * ldr, ldr, 1, nullptr, 0, jb, j0, PL, st, s));
            RQB_CHECK(launch_mm_tc(false, Qp + j0 * ldqp, ldqp, PL, m, j0, jb, 1, -1.f, 1.f, Qp, ldqp, Qp, ldqp, 0,
                                   nullptr, st, s));
        }
        j1 = j0;
    }
    return RQRCP_OK;
}

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
    if (sizeof(T) == 4 && tensor_cores_enabled() && mm_tc_supported(A, lda) && mm_tc_supported(Q1, ldq)) {
        if (work_bytes < bwd_tc_layout(m, n, k).total) return RQRCP_ERR_WORKSPACE;
        const bool prof = prof_on();
        if (prof) prof_begin(K_BACKWARD, s);
        const int rc = backward_f32_tc(m, n, k, reinterpret_cast<const float*>(A), lda, jpvt,
                                       reinterpret_cast<const float*>(Q1), ldq, reinterpret_cast<const float*>(R), ldr,
                                       reinterpret_cast<const float*>(dQ1), lddq, reinterpret_cast<const float*>(dR),
                                       lddr, reinterpret_cast<float*>(dA), ldda, w, s);
        if (rc != RQRCP_OK) return rc;
        if (prof) {
            const int64_t nt = n - k;
            const double fl = 4.0 * m * (double)nt * k + 4.0 * m * (double)k * k + (double)m * k * k;
            prof_end(K_BACKWARD, fl, 4.0 * (2.0 * m * n + 3.0 * m * k), s);
        }
        return RQRCP_OK;
    }
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
    if (precision == RQRCP_PREC_FP64) return bwd_layout(m, n, k, sizeof(double)).total;
    const size_t simt = bwd_layout(m, n, k, sizeof(float)).total, tc = bwd_tc_layout(m, n, k).total;
    return simt > tc ? simt : tc;
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
