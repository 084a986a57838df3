// srqr.cu -- Alg. 3 (SRQR, Sec. IV-E) after its RQRCP stage, on the explicit R held in A:
//  * the extra pivot: the trailing column with the largest estimate r_i (sketch column norm^2
//    / (b+p), downdated row by row) moves to position l, one Householder step reduces
//    A(l:m, l), and the estimates lose the new row l;
//  * the randomized estimate g_2 ~ |alpha|/sqrt(d) ||Omega R_hat^{-T}||_{1,2} with a d x (l+1)
//    Gaussian Omega (one back substitution per row of Omega, in shared memory);
//  * one swap of the loop: round-robin rotation of columns imax..l, Givens rotations on rows
//    (j, j+1) restoring the upper-trapezoidal form (the rotations are found in one block on
//    the Hessenberg part, then applied to the columns l..n-1 one thread per column), and the
//    estimates regain row l.
// Swaps are rare (the paper finds none on real data), so these kernels favour simplicity:
// single-block steps where the algorithm is sequential, grid-stride loops elsewhere.
#include "internal.cuh"

namespace rq {
namespace {

constexpr int kT = 1024;

__device__ __forceinline__ double& at(double* A, int64_t lda, int64_t i, int64_t j) { return A[j * lda + i]; }

// Block-wide (value, index) maximum, larger value first, then smaller index.
__device__ void block_argmax(double& v, int64_t& idx, double* sv, int64_t* si)
{
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffffu, v, o);
        const int64_t oi = __shfl_xor_sync(0xffffffffu, idx, o);
        if (ov > v || (ov == v && oi < idx)) { v = ov; idx = oi; }
    }
    if (lane == 0) { sv[wid] = v; si[wid] = idx; }
    __syncthreads();
    if (wid == 0) {
        const int nw = blockDim.x >> 5;
        v = lane < nw ? sv[lane] : -INFINITY;
        idx = lane < nw ? si[lane] : INT64_MAX;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double ov = __shfl_xor_sync(0xffffffffu, v, o);
            const int64_t oi = __shfl_xor_sync(0xffffffffu, idx, o);
            if (ov > v || (ov == v && oi < idx)) { v = ov; idx = oi; }
        }
        if (lane == 0) { sv[0] = v; si[0] = idx; }
    }
    __syncthreads();
    v = sv[0];
    idx = si[0];
    __syncthreads();
}

__device__ double block_sum(double v, double* sv)
{
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) sv[wid] = v;
    __syncthreads();
    if (wid == 0) {
        v = lane < (int)(blockDim.x >> 5) ? sv[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) sv[0] = v;
    }
    __syncthreads();
    v = sv[0];
    __syncthreads();
    return v;
}

// A becomes the explicit R: the reflector tails below the diagonal of columns 0..l-1 are zeroed.
__global__ void srqr_zero_tails_kernel(double* A, int64_t lda, int64_t m, int64_t l, const Status* st)
{
    if (status_error(st)) return;
    const int64_t total = m * l;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = e / m, i = e - j * m;
        if (i > j) at(A, lda, i, j) = 0.0;
    }
}

// Alg. 3 "r_i = r_hat_i / (b+p)": one warp per trailing column of the final sketch B (ld ls).
__global__ void srqr_rinit_kernel(const double* B, int ls, int64_t l, int64_t n, double* r, const Status* st)
{
    if (status_error(st)) return;
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = l + warp; i < n; i += nwarps) {
        double ss = 0.0;
        for (int q = lane; q < ls; q += 32) ss = fma(B[i * ls + q], B[i * ls + q], ss);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
        if (lane == 0) r[i] = ss / (double)ls;
    }
}

// Extra pivot, part 1 (one block): argmax of r over l..n-1 (ties to the smallest position), then
// the swap of that column with column l in A (all m rows), jpvt and r.
__global__ void __launch_bounds__(kT) srqr_pivot_kernel(double* A, int64_t lda, int64_t m, int64_t l, int64_t n,
                                                        double* r, int32_t* jpvt, const Status* st)
{
    if (status_error(st)) return;
    __shared__ double sv[32];
    __shared__ int64_t si[32];
    double v = -INFINITY;
    int64_t idx = INT64_MAX;
    for (int64_t i = l + threadIdx.x; i < n; i += blockDim.x)
        if (r[i] > v) { v = r[i]; idx = i; }
    block_argmax(v, idx, sv, si);
    const int64_t sel = (idx == INT64_MAX) ? l : idx;
    if (sel == l) return;
    for (int64_t i = threadIdx.x; i < m; i += blockDim.x) {
        const double t = at(A, lda, i, l);
        at(A, lda, i, l) = at(A, lda, i, sel);
        at(A, lda, i, sel) = t;
    }
    if (threadIdx.x == 0) {
        const int32_t tj = jpvt[l]; jpvt[l] = jpvt[sel]; jpvt[sel] = tj;
        const double tr = r[l]; r[l] = r[sel]; r[sel] = tr;
    }
}

// Extra pivot, part 2 (one block): the reflector of A(l:m, l) in the xLARFG convention
// (beta = -sign(alpha) ||x||, tau = (beta - alpha)/beta, tail scaled by 1/(alpha - beta);
// tau = 0 when the tail is zero).  tau goes to info[3].
__global__ void __launch_bounds__(kT) srqr_house_kernel(double* A, int64_t lda, int64_t m, int64_t l, double* info,
                                                        const Status* st)
{
    if (status_error(st)) return;
    __shared__ double sv[32];
    double* x = &at(A, lda, l, l);
    const int64_t len = m - l;
    // read before the block sum: its barriers order every thread's read before thread 0
    // overwrites x[0] with beta
    const double alpha = x[0];
    double ss = 0.0;
    for (int64_t i = 1 + threadIdx.x; i < len; i += blockDim.x) ss = fma(x[i], x[i], ss);
    ss = block_sum(ss, sv);
    if (len <= 1 || ss == 0.0) {
        if (threadIdx.x == 0) info[3] = 0.0;
        return;
    }
    const double nrm = sqrt(alpha * alpha + ss);
    const double beta = (alpha >= 0.0) ? -nrm : nrm;
    const double scal = 1.0 / (alpha - beta);
    for (int64_t i = 1 + threadIdx.x; i < len; i += blockDim.x) x[i] *= scal;
    if (threadIdx.x == 0) {
        info[3] = (beta - alpha) / beta;
        x[0] = beta;
    }
}

// Extra pivot, part 3: y <- (I - tau v v^T) y for every trailing column y = A(l:m, s), s > l,
// v = [1; A(l+1:m, l)]; one warp per column.
__global__ void srqr_house_apply_kernel(double* A, int64_t lda, int64_t m, int64_t l, int64_t n, const double* info,
                                        const Status* st)
{
    if (status_error(st)) return;
    const double tau = info[3];
    if (tau == 0.0) return;
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const double* v = &at(A, lda, l, l);
    const int64_t len = m - l;
    for (int64_t s = l + 1 + warp; s < n; s += nwarps) {
        double* y = &at(A, lda, l, s);
        double w = 0.0;
        for (int64_t i = 1 + lane; i < len; i += 32) w = fma(v[i], y[i], w);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
        w = (w + y[0]) * tau;
        for (int64_t i = 1 + lane; i < len; i += 32) y[i] = fma(-w, v[i], y[i]);
        if (lane == 0) y[0] -= w;
    }
}

// Extra pivot, part 4: zero the reflector tail A(l+1:m, l) (R is explicit), |alpha| = |A(l,l)|
// to info[2], and r_i -= A(l, i)^2 for i > l.
__global__ void srqr_downdate_kernel(double* A, int64_t lda, int64_t m, int64_t l, int64_t n, double* r, double* info,
                                     const Status* st)
{
    if (status_error(st)) return;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    if (t == 0) info[2] = fabs(at(A, lda, l, l));
    for (int64_t i = l + 1 + t; i < m; i += stride) at(A, lda, i, l) = 0.0;
    for (int64_t i = l + 1 + t; i < n; i += stride) {
        const double a = at(A, lda, l, i);
        r[i] -= a * a;
    }
}

// g_2 estimate, part 1: row q of X = Omega R_hat^{-T} solves R_hat x = Omega(q, :)^T, R_hat the
// leading (l+1) x (l+1) block of R; column-oriented back substitution in shared memory, one
// block per row of Omega.
__global__ void __launch_bounds__(kT) srqr_solve_kernel(const double* A, int64_t lda, int64_t l, const double* Og,
                                                        double* X, const Status* st)
{
    if (status_error(st)) return;
    extern __shared__ double xs[];
    const int64_t w = l + 1;
    const int64_t q = blockIdx.x;
    for (int64_t j = threadIdx.x; j < w; j += blockDim.x) xs[j] = Og[q * w + j];
    __syncthreads();
    for (int64_t j = w - 1; j >= 0; --j) {
        if (threadIdx.x == 0) xs[j] = xs[j] / A[j * lda + j];
        __syncthreads();
        const double y = xs[j];
        const double* col = A + j * lda;
        for (int64_t i = threadIdx.x; i < j; i += blockDim.x) xs[i] = fma(-col[i], y, xs[i]);
        __syncthreads();
    }
    for (int64_t j = threadIdx.x; j < w; j += blockDim.x) X[q * w + j] = xs[j];
}

// g_2 estimate, part 2 (one block): column norms of X (d x (l+1), row-major), their maximum
// and its column (ties to the smallest), g_2 = |alpha|/sqrt(d) max -> info[0], the column ->
// info[1].  A zero diagonal entry of R_hat gives g_2 = +inf at the first such column.
__global__ void __launch_bounds__(kT) srqr_g2_kernel(const double* A, int64_t lda, int64_t l, int64_t d,
                                                     const double* X, double* info, const Status* st)
{
    if (status_error(st)) return;
    __shared__ double sv[32];
    __shared__ int64_t si[32];
    const int64_t w = l + 1;
    double zv = -INFINITY;
    int64_t zi = INT64_MAX;
    for (int64_t j = threadIdx.x; j < w; j += blockDim.x)
        if (A[j * lda + j] == 0.0 && zi == INT64_MAX) { zv = 0.0; zi = j; }
    block_argmax(zv, zi, sv, si);
    double v = -INFINITY;
    int64_t idx = INT64_MAX;
    for (int64_t j = threadIdx.x; j < w; j += blockDim.x) {
        double ss = 0.0;
        for (int64_t q = 0; q < d; ++q) ss = fma(X[q * w + j], X[q * w + j], ss);
        const double c = sqrt(ss);
        if (c > v) { v = c; idx = j; }
    }
    block_argmax(v, idx, sv, si);
    if (threadIdx.x == 0) {
        if (zi != INT64_MAX) {
            info[0] = INFINITY;
            info[1] = (double)zi;
        } else {
            info[0] = info[2] / sqrt((double)d) * v;
            info[1] = (double)idx;
        }
    }
}

// Swap, part 1: round robin -- column imax moves to position l and the columns imax+1..l move
// left by one, in rows 0..l (rows below l are zero in these columns) and in jpvt.
__global__ void srqr_rotate_kernel(double* A, int64_t lda, int64_t l, int64_t imax, int32_t* jpvt, const Status* st)
{
    if (status_error(st)) return;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = t; i <= l; i += stride) {
        const double first = at(A, lda, i, imax);
        for (int64_t j = imax; j < l; ++j) at(A, lda, i, j) = at(A, lda, i, j + 1);
        at(A, lda, i, l) = first;
    }
    if (t == 0) {
        const int32_t first = jpvt[imax];
        for (int64_t j = imax; j < l; ++j) jpvt[j] = jpvt[j + 1];
        jpvt[l] = first;
    }
}

// Swap, part 2 (one block): Givens rotations j = imax..l-1 on rows (j, j+1), each found from
// (R(j,j), R(j+1,j)) after the rotations before it and applied to the columns j..l-1 of the
// Hessenberg part; (c, s) go to cs[2j], cs[2j+1] (c = 1, s = 0 where R(j+1,j) is already zero).
__global__ void __launch_bounds__(kT) srqr_givens_kernel(double* A, int64_t lda, int64_t l, int64_t imax, double* cs,
                                                         const Status* st)
{
    if (status_error(st)) return;
    __shared__ double sc, ss;
    __shared__ int rot;
    for (int64_t j = imax; j < l; ++j) {
        if (threadIdx.x == 0) {
            const double a = at(A, lda, j, j), b = at(A, lda, j + 1, j);
            if (b != 0.0) {
                const double h = hypot(a, b);
                sc = a / h;
                ss = b / h;
                rot = 1;
            } else {
                sc = 1.0;
                ss = 0.0;
                rot = 0;
            }
            cs[2 * j] = sc;
            cs[2 * j + 1] = ss;
        }
        __syncthreads();
        if (rot) {
            const double c = sc, s = ss;
            for (int64_t col = j + threadIdx.x; col < l; col += blockDim.x) {
                const double x = at(A, lda, j, col), y = at(A, lda, j + 1, col);
                at(A, lda, j, col) = c * x + s * y;
                at(A, lda, j + 1, col) = -s * x + c * y;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) at(A, lda, j + 1, j) = 0.0;
        __syncthreads();
    }
}

// Swap, part 3: the same rotations, in order, on the columns l..n-1, one thread per column
// (a two-row carry down rows imax..l); then the estimates regain row l:
// r_l = R(l,l)^2 and r_i += R(l,i)^2 for i > l.
__global__ void srqr_givens_rest_kernel(double* A, int64_t lda, int64_t l, int64_t n, int64_t imax, const double* cs,
                                        double* r, const Status* st)
{
    if (status_error(st)) return;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t col = l + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; col < n; col += stride) {
        double x = at(A, lda, imax, col);
        for (int64_t j = imax; j < l; ++j) {
            const double c = cs[2 * j], s = cs[2 * j + 1];
            const double y = at(A, lda, j + 1, col);
            at(A, lda, j, col) = c * x + s * y;
            x = -s * x + c * y;
        }
        at(A, lda, l, col) = x;
        if (col == l) r[l] = x * x;
        else r[col] += x * x;
    }
}

int grid_for(int64_t work, int threads)
{
    int64_t g = (work + threads - 1) / threads;
    const int64_t cap = 8 * (int64_t)dev_info().sms;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (int)g;
}

}  // namespace

cudaError_t launch_srqr_prepare(double* A, int64_t lda, int64_t m, int64_t l, int64_t n, const double* B, int ls,
                                double* r, const Status* st, cudaStream_t s)
{
    srqr_zero_tails_kernel<<<grid_for(m * l, 256), 256, 0, s>>>(A, lda, m, l, st);
    srqr_rinit_kernel<<<grid_for(32 * (n - l), 256), 256, 0, s>>>(B, ls, l, n, r, st);
    return cudaGetLastError();
}

cudaError_t launch_srqr_extra_pivot(double* A, int64_t lda, int64_t m, int64_t l, int64_t n, double* r,
                                    int32_t* jpvt, double* info, const Status* st, cudaStream_t s)
{
    srqr_pivot_kernel<<<1, kT, 0, s>>>(A, lda, m, l, n, r, jpvt, st);
    srqr_house_kernel<<<1, kT, 0, s>>>(A, lda, m, l, info, st);
    srqr_house_apply_kernel<<<grid_for(32 * (n - l), 256), 256, 0, s>>>(A, lda, m, l, n, info, st);
    srqr_downdate_kernel<<<grid_for(m > n ? m - l : n - l, 256), 256, 0, s>>>(A, lda, m, l, n, r, info, st);
    return cudaGetLastError();
}

size_t srqr_solve_smem(int64_t l) { return sizeof(double) * (size_t)(l + 1); }

cudaError_t launch_srqr_g2(const double* A, int64_t lda, int64_t l, int64_t d, uint64_t seed, double* Og, double* X,
                           double* info, const Status* st, cudaStream_t s)
{
    static DevFlag attr_set;
    if (!attr_set.done()) {
        if (cudaError_t e = allow_max_dynamic_smem(srqr_solve_kernel)) return e;
        attr_set.set();
    }
    if (cudaError_t e = launch_omega<double>(d, l + 1, seed, Og, l + 1, s)) return e;
    srqr_solve_kernel<<<(unsigned)d, kT, srqr_solve_smem(l), s>>>(A, lda, l, Og, X, st);
    srqr_g2_kernel<<<1, kT, 0, s>>>(A, lda, l, d, X, info, st);
    return cudaGetLastError();
}

cudaError_t launch_srqr_swap(double* A, int64_t lda, int64_t l, int64_t n, int64_t imax, int32_t* jpvt, double* cs,
                             double* r, const Status* st, cudaStream_t s)
{
    srqr_rotate_kernel<<<grid_for(l + 1, 256), 256, 0, s>>>(A, lda, l, imax, jpvt, st);
    srqr_givens_kernel<<<1, kT, 0, s>>>(A, lda, l, imax, cs, st);
    srqr_givens_rest_kernel<<<grid_for(n - l, 128), 128, 0, s>>>(A, lda, l, n, imax, cs, r, st);
    return cudaGetLastError();
}

}  // namespace rq
