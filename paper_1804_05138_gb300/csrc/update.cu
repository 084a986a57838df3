// update.cu -- small kernels around the hot loop of Alg. 2:
//  * status / jpvt initialisation;
//  * "Swap (j_1..j_b) and (i:i+b-1) columns in A": gather the moved columns into scratch,
//    then scatter them to their new positions (whole columns, all m rows, coalesced);
//  * Eq. (4): B(0:bb, i+bb:n) <- R_hat12 - Omega_hat_11 R12 with Omega_hat_11 = R_hat11 R11^{-1}
//    from the forward substitution Omega_hat_11 R11 = R_hat11 (both upper triangular);
//  * the last step of Eq. (5): B(:, i+bb:n) <- B2 - Omega_bar_1 R12 from the split-K partials of
//    Omega_bar_1 R12.
#include "internal.cuh"

namespace rq {
namespace {

__global__ void init_kernel(Status* st, int64_t k, int32_t* jpvt, int64_t n)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t == 0) {
        st->error = 0;
        st->guard = 0;
        st->rank = k;
        st->bar = 0;
        st->nu0bits = 0;
    }
    for (int64_t j = t; j < n; j += (int64_t)gridDim.x * blockDim.x) jpvt[j] = (int32_t)j;
}

template <typename T>
__global__ void swap_gather_kernel(const T* __restrict__ A, int64_t lda, int64_t m,
                                   const long long* __restrict__ swapmap, T* __restrict__ tmp, const Status* st)
{
    if (status_error(st)) return;
    const long long cnt = swapmap[0];
    const long long e = blockIdx.y;
    if (e >= cnt) return;
    const long long src = swapmap[1 + 2 * e + 1];
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < m; r += (int64_t)gridDim.x * blockDim.x)
        tmp[e * m + r] = A[src * lda + r];
}

template <typename T>
__global__ void swap_scatter_kernel(T* __restrict__ A, int64_t lda, int64_t m,
                                    const long long* __restrict__ swapmap, const T* __restrict__ tmp,
                                    const Status* st)
{
    if (status_error(st)) return;
    const long long cnt = swapmap[0];
    const long long e = blockIdx.y;
    if (e >= cnt) return;
    const long long dst = swapmap[1 + 2 * e];
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < m; r += (int64_t)gridDim.x * blockDim.x)
        A[dst * lda + r] = tmp[e * m + r];
}

// One block per row r of Omega_hat_11 = R_hat11 R11^{-1}: the rows of the forward substitution
// Omega_hat_11(r,j) = (R_hat11(r,j) - sum_{q=r}^{j-1} Omega_hat_11(r,q) R11(q,j)) / R11(j,j)
// are independent.  R11(r:bb, r:bb) goes to shared memory; warp 0 runs the substitution column by
// column: lane j mod 32 owns column j, finishes Omega_hat_11(r,q) at step q (a multiplication by the
// reciprocal of R11(q,q), computed up front) and broadcasts it, and every lane subtracts its terms
// from the columns it owns.  One product, one shuffle and one FMA per step: no reduction tree and no
// division on the chain.
template <typename T>
__global__ void bsolve_kernel(const T* __restrict__ B, int64_t ldb, const T* __restrict__ A, int64_t lda,
                              int64_t i, int bb, double* __restrict__ What, const Status* st)
{
    if (status_error(st) || *(volatile const int*)&st->guard) return;
    extern __shared__ double sm[];
    const int r = blockIdx.x;
    const int w = bb - r;
    double* Rs = sm;          // Rs[jj * w + qq] = R11(r + qq, r + jj), qq <= jj
    double* Wr = sm + w * w;  // Omega_hat_11(r, r..bb-1)
    for (int e = threadIdx.x; e < w * w; e += blockDim.x) {
        const int qq = e % w, jj = e / w;
        Rs[e] = (qq <= jj) ? (double)A[(i + r + jj) * lda + i + r + qq] : 0.0;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        constexpr int NJ = 4;  // columns per lane (bb <= 128)
        const int lane = threadIdx.x;
        double acc[NJ], rinv[NJ];
#pragma unroll
        for (int u = 0; u < NJ; ++u) {
            const int jj = lane + 32 * u;
            const double rjj = jj < w ? Rs[jj * w + jj] : 1.0;
            acc[u] = jj < w ? (double)B[(i + r + jj) * ldb + r] : 0.0;
            rinv[u] = rjj == 0.0 ? 0.0 : 1.0 / rjj;  // a zero diagonal gives a zero column
        }
        for (int qq = 0; qq < w; ++qq) {
            const int u0 = qq >> 5;
            double x = 0.0;
#pragma unroll
            for (int u = 0; u < NJ; ++u)
                if (u == u0) x = acc[u] * rinv[u];
            x = __shfl_sync(0xffffffffu, x, qq & 31);
            if (lane == (qq & 31)) Wr[qq] = x;
#pragma unroll
            for (int u = 0; u < NJ; ++u) {
                const int jj = lane + 32 * u;
                if (jj > qq && jj < w) acc[u] = fma(-x, Rs[jj * w + qq], acc[u]);
            }
        }
    }
    __syncthreads();
    for (int j = threadIdx.x; j < bb; j += blockDim.x) What[(int64_t)j * bb + r] = (j < r) ? 0.0 : Wr[j - r];
}

// B(r, c) -= sum_{q >= r} What(r, q) * A(i+q, c) for the trailing columns c (the top bb rows of
// Eq. (4)), in T arithmetic.  One block per 64 trailing columns: the R12 tile A(i:i+bb, c0:c0+64)
// and B's top rows land in shared memory with coalesced column reads; Omega_hat_11 (zero below
// its diagonal) is staged as T, 64 of its rows at a time; every thread owns a 4 x 4 register
// tile (rows tm + 16 a, columns tn + 16 b) and runs the contraction over q >= the chunk's first
// row, the zeros taking the rest of the triangle.
template <typename T>
__global__ void __launch_bounds__(256) bapply_kernel(T* __restrict__ B, int64_t ldb, const T* __restrict__ A,
                                                     int64_t lda, int64_t i, int bb, int64_t n,
                                                     const double* __restrict__ What, const Status* st)
{
    if (status_error(st) || *(volatile const int*)&st->guard) return;
    constexpr int TC = 64;                        // columns per block, and rows per What chunk
    constexpr int LD = TC + 1;                    // padded row stride of the A and B tiles
    extern __shared__ __align__(16) unsigned char smb[];
    T* As = reinterpret_cast<T*>(smb);            // [q][c]: A(i+q, c0+c), bb x LD
    T* Bs = As + (size_t)bb * LD;                 // [r][c]: B(r, c0+c),   bb x LD
    T* Ws = Bs + (size_t)bb * LD;                 // [q][r - r0]: What(r, q), bb x TC
    const int tid = threadIdx.x;
    const int64_t c0 = i + bb + (int64_t)blockIdx.x * TC;
    const int nc = (int)min((int64_t)TC, n - c0);
    for (int e = tid; e < bb * TC; e += blockDim.x) {
        const int q = e % bb, c = e / bb;         // consecutive threads read one column: coalesced
        const bool in = c < nc;
        As[(size_t)q * LD + c] = in ? A[(c0 + c) * lda + i + q] : T(0);
        Bs[(size_t)q * LD + c] = in ? B[(c0 + c) * ldb + q] : T(0);
    }
    const int tm = tid & 15, tn = tid >> 4;
    for (int r0 = 0; r0 < bb; r0 += TC) {
        __syncthreads();
        for (int e = tid; e < bb * TC; e += blockDim.x) {
            const int rr = e % TC, q = e / TC;    // What is column-major: What[q * bb + r]
            Ws[e] = r0 + rr < bb ? (T)What[(size_t)q * bb + r0 + rr] : T(0);
        }
        __syncthreads();
        T acc[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
        for (int q = r0; q < bb; ++q) {           // What(r, q) = 0 for q < r
            T w[4], x[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) w[a] = Ws[(size_t)q * TC + tm + 16 * a];
#pragma unroll
            for (int b = 0; b < 4; ++b) x[b] = As[(size_t)q * LD + tn + 16 * b];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] = fma(w[a], x[b], acc[a][b]);
        }
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            const int r = r0 + tm + 16 * a;
            if (r < bb)
#pragma unroll
                for (int b = 0; b < 4; ++b) Bs[(size_t)r * LD + tn + 16 * b] -= acc[a][b];
        }
    }
    __syncthreads();
    for (int e = tid; e < bb * TC; e += blockDim.x) {
        const int q = e % bb, c = e / bb;
        if (c < nc) B[(c0 + c) * ldb + q] = Bs[(size_t)q * LD + c];
    }
}

// Eq. (5), last step: B(:, c0+c) = Bc(:, c0+c) - sum_sp P[sp][c][0:l] for c < nt, the partials
// holding Omega_bar_1 R12 with Omega_bar_1 the columns i:i+bb of Omega Q_tilde.  Bc is the sketch
// as permuted by this block's pivots but not transformed by its QRCP; both buffers take the
// result: B for the next pivot search (which transforms it in place), Bc as its untouched copy.
template <typename T>
__global__ void bfinish_kernel(T* __restrict__ B, T* __restrict__ Bc, int l, int64_t c0, int64_t nt,
                               const double* __restrict__ P, int nsplit, const Status* st)
{
    if (status_error(st) || *(volatile const int*)&st->guard) return;
    const int64_t total = (int64_t)l * nt;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = e / l;
        const int r = (int)(e - c * l);
        double s = 0.0;
        for (int sp = 0; sp < nsplit; ++sp) s += P[((int64_t)sp * nt + c) * l + r];
        const int64_t at = (c0 + c) * l + r;
        const T v = (T)((double)Bc[at] - s);
        B[at] = v;
        Bc[at] = v;
    }
}

// Two blocks in one trailing update: block i+1's Gram is taken from the trailing matrix before block
// i's update, V1^T C, and corrected by V1^T (V0 Y0) = Gx Y0.  This writes the correction as one more
// split of the partial buffer: Pc[(c0 + c) * bb + r] = -sum_q Gx(r, q) Y0(q, cy0 + c) for c < nt,
// r < bb, with Gx(r, q) = P2[q * bb + r] (V1^T V0 over the rows of V0 below its triangle, its splits
// already summed).  FP32 products and sums (the Gram itself is FP32-accurate; float-pair sums here
// measured no better); kCorrCols columns per block, sixteen per thread advanced together.
constexpr int kCorrCols = 64;

__global__ void __launch_bounds__(256) wy_corr_kernel(const double* __restrict__ P2, int bb,
                                                      const double* __restrict__ Y0, int64_t ldy, int64_t cy0,
                                                      int64_t nt, int64_t c0, double* __restrict__ Pc,
                                                      const Status* st)
{
    if (status_error(st)) return;
    __shared__ float Gs[64][65], Ys[kCorrCols][65];
    const int tid = threadIdx.x;
    const int64_t cb = (int64_t)blockIdx.x * kCorrCols;
    for (int e = tid; e < 64 * 64; e += blockDim.x) {
        const int r = e % 64, q = e / 64;
        Gs[r][q] = (r < bb && q < bb) ? (float)P2[(int64_t)q * bb + r] : 0.f;
    }
    for (int e = tid; e < 64 * kCorrCols; e += blockDim.x) {
        const int r = e % 64, cc = e / 64;
        const int64_t c = cb + cc;
        Ys[cc][r] = (r < bb && c < nt) ? (float)Y0[(cy0 + c) * ldy + r] : 0.f;
    }
    __syncthreads();
    const int r = tid & 63, cg = tid >> 6;
    if (r >= bb) return;
    constexpr int NU = kCorrCols / 4;
    float acc[NU];
#pragma unroll
    for (int u = 0; u < NU; ++u) acc[u] = 0.f;
#pragma unroll 4
    for (int q = 0; q < 64; ++q) {
        const float g = Gs[r][q];
#pragma unroll
        for (int u = 0; u < NU; ++u) acc[u] = fmaf(g, Ys[cg + 4 * u][q], acc[u]);
    }
#pragma unroll
    for (int u = 0; u < NU; ++u) {
        const int64_t c = cb + cg + 4 * u;
        if (c < nt) Pc[(c0 + c) * bb + r] = -(double)acc[u];
    }
}

// P2[e] = sum_sp P2[sp * stride + e] for e < len: the splits summed into the first (each entry read
// before it is written, by the same thread).
__global__ void split_sum_kernel(double* __restrict__ P2, int ns, int64_t len, int64_t stride, const Status* st)
{
    if (status_error(st)) return;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < len; e += (int64_t)gridDim.x * blockDim.x) {
        double g = 0.0;
        for (int sp = 0; sp < ns; ++sp) g += P2[sp * stride + e];
        P2[e] = g;
    }
}

}  // namespace

cudaError_t launch_split_sum(double* P2, int ns2, int64_t len, int64_t stride, const Status* st, cudaStream_t s)
{
    split_sum_kernel<<<16, 256, 0, s>>>(P2, ns2, len, stride, st);
    return cudaGetLastError();
}

cudaError_t launch_wy_corr(const double* P2, int bb, const double* Y0, int64_t ldy, int64_t cy0, int64_t nt, int64_t c0,
                           double* Pc, const Status* st, cudaStream_t s)
{
    if (nt <= 0) return cudaSuccess;
    if (bb < 1 || bb > 64) return cudaErrorInvalidValue;
    wy_corr_kernel<<<(unsigned)((nt + kCorrCols - 1) / kCorrCols), 256, 0, s>>>(P2, bb, Y0, ldy, cy0, nt, c0, Pc, st);
    return cudaGetLastError();
}

cudaError_t launch_init(Status* st, int64_t k, int32_t* jpvt, int64_t n, cudaStream_t s)
{
    int64_t grid = (n + 255) / 256;
    if (grid < 1) grid = 1;
    if (grid > 1024) grid = 1024;
    init_kernel<<<(unsigned)grid, 256, 0, s>>>(st, k, jpvt, n);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_swaps(T* A, int64_t lda, int64_t m, int bb, const long long* swapmap, T* tmp,
                         const Status* st, cudaStream_t s)
{
    int64_t gx = (m + 255) / 256;
    if (gx > 16) gx = 16;
    dim3 grid((unsigned)gx, (unsigned)(2 * bb));
    swap_gather_kernel<T><<<grid, 256, 0, s>>>(A, lda, m, swapmap, tmp, st);
    swap_scatter_kernel<T><<<grid, 256, 0, s>>>(A, lda, m, swapmap, tmp, st);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_bupdate(T* B, int64_t ldb, const T* A, int64_t lda, int64_t i, int bb, int64_t n,
                           double* What, const Status* st, cudaStream_t s)
{
    static DevFlag attr_set;
    if (!attr_set.done()) {
        if (cudaError_t e = allow_max_dynamic_smem(bsolve_kernel<T>)) return e;
        if (cudaError_t e = allow_max_dynamic_smem(bapply_kernel<T>)) return e;
        attr_set.set();
    }
    const size_t smem = sizeof(double) * ((size_t)bb * bb + (size_t)bb);
    bsolve_kernel<T><<<bb, 128, smem, s>>>(B, ldb, A, lda, i, bb, What, st);
    const int64_t nt = n - i - bb;
    const size_t smem_apply = sizeof(T) * (size_t)bb * (2 * 65 + 64);
    if (nt > 0)
        bapply_kernel<T><<<(unsigned)((nt + 63) / 64), 256, smem_apply, s>>>(B, ldb, A, lda, i, bb, n, What, st);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_bfinish(T* B, T* Bc, int l, int64_t c0, int64_t nt, const double* P, int nsplit,
                           const Status* st, cudaStream_t s)
{
    const int64_t total = (int64_t)l * nt;
    if (total <= 0) return cudaSuccess;
    int64_t grid = (total + 255) / 256;
    const int64_t cap = 8 * (int64_t)dev_info().sms;
    if (grid > cap) grid = cap;
    bfinish_kernel<T><<<(unsigned)grid, 256, 0, s>>>(B, Bc, l, c0, nt, P, nsplit, st);
    return cudaGetLastError();
}

#define RQ_INST(T)                                                                                    \
    template cudaError_t launch_bfinish<T>(T*, T*, int, int64_t, int64_t, const double*, int, const Status*, \
                                           cudaStream_t);                                             \
    template cudaError_t launch_swaps<T>(T*, int64_t, int64_t, int, const long long*, T*, const Status*, \
                                         cudaStream_t);                                               \
    template cudaError_t launch_bupdate<T>(T*, int64_t, const T*, int64_t, int64_t, int, int64_t,     \
                                           double*, const Status*, cudaStream_t);
RQ_INST(double)
RQ_INST(float)
#undef RQ_INST

}  // namespace rq
