// cholqr.cu -- the unpivoted panel QR of Alg. 2 ("Do unpivoted QR on A(i:m, i:i+b-1)") for the FP32
// form by CholeskyQR2 with Householder reconstruction, instead of one grid-wide step per column.
//
// For the (m1 x bb) FP32 panel P (bb <= 64):
//   pass 1  G1 = P^T P (Dot2 sums of exact FP32 products per block, FP64 across blocks in a fixed
//           order), G1 = R1^T R1 (FP64 Cholesky);
//   pass 2  Q1 = P R1^{-1} row by row (forward substitution with R1 as float pairs and Dot2 sums,
//           rounded to FP32), G2 = Q1^T Q1, G2 = R2^T R2; R = R2 R1 and P = (Q1 R2^{-1}) R;
//   rebuild with Q2 = Q1 R2^{-1} (orthonormal to FP32 level), the LU factorization without pivoting
//           Q2 - S = [L1; L2] U, S = diag(s_j) with s_j = -sign of the j-th pivot, gives the
//           Householder vectors V = [L1; L2] (unit lower), tau_j = -s_j U(j,j) and R_house = S R:
//           the representation xGEQRF computes (xLARFG sign convention), up to rounding (Ballard
//           et al., "Reconstructing Householder vectors from tall-skinny QR", 2014).  The top bb rows
//           of Q2 are formed and factored in FP64 in one block; the rows below are V2 = Q1 (U R2)^{-1},
//           again row by row with float-pair coefficients.
// CholeskyQR2 needs kappa(P) well below u^{-1/2} of the Gram's arithmetic; a pivot of G1 below
// 2^-36 of its diagonal entry (kappa(P) beyond about 2.6e5), or a pivot of G2 below 1/2, sets a
// flag on the device: the panel is then left untouched and the cooperative Householder panel
// kernel launched after this one factors it instead (it reads the flag and returns at once when
// the CholeskyQR2 result was written).  No host synchronisation.
#include "internal.cuh"

namespace rq {
namespace {

constexpr int kCqrMaxB = 64;
constexpr int kCqrNE = kCqrMaxB * (kCqrMaxB + 1) / 2;  // packed upper-triangle entries
constexpr int kCqrRows = 256;                          // panel rows per block of the row passes
constexpr int kCqrThreads = 256;
constexpr int kCqrSmallThreads = 512;

// entry e of the packed upper triangle (row-major): (i, j), i <= j
__device__ __forceinline__ void tri_ij(int e, int bb, int& i, int& j)
{
    int r = 0, start = 0;
    while (start + (bb - r) <= e) {
        start += bb - r;
        ++r;
    }
    i = r;
    j = r + (e - start);
}

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e)
{
    s = a + b;
    const float z = s - a;
    e = (a - (s - z)) + (b - z);
}

// (sh, sl) += x * y with the product's rounding error (FMA) and the sum's (TwoSum) carried in sl.
__device__ __forceinline__ void dot2_add(float& sh, float& sl, float x, float y)
{
    const float p = x * y;
    const float pe = fmaf(x, y, -p);
    float t, e;
    two_sum(sh, p, t, e);
    sh = t;
    sl += e + pe;
}

// Row solve q R = p for one row (R upper bb x bb as float pairs Rh/Rl, row-major [q * ld + c]) with
// Dot2 sums; rinv[c] = 1 / R(c, c) in FP32.  q may alias p.
__device__ __forceinline__ void row_solve(float* q, const float* p, int bb, const float* Rh, const float* Rl, int ld,
                                          const float* rinv)
{
    for (int c = 0; c < bb; ++c) {
        float sh = p[c], sl = 0.f;
        for (int k = 0; k < c; ++k) {
            const float qk = q[k];
            dot2_add(sh, sl, -qk, Rh[k * ld + c]);
            sl = fmaf(-qk, Rl[k * ld + c], sl);
        }
        q[c] = (sh + sl) * rinv[c];
    }
}

// Pass 1 (Rh == nullptr): Gram partials of the panel rows of this block.  Pass 2: first Q1 = P R1^{-1}
// for the block's rows (stored to Q1, ld m1), then the Gram partials of Q1.  part[g * NE + e] (FP64).
__global__ void __launch_bounds__(kCqrThreads) cqr_gram_kernel(const float* __restrict__ P, int64_t ldp, int64_t m1,
                                                               int bb, const float* __restrict__ R1h,
                                                               const float* __restrict__ R1l,
                                                               const float* __restrict__ r1inv, float* __restrict__ Q1,
                                                               double* __restrict__ part, const int* flag,
                                                               const Status* st)
{
    if (status_error(st)) return;
    if (R1h != nullptr && *(volatile const int*)flag) return;  // pass 1 already chose the fallback
    extern __shared__ float cqr_sm[];
    float(*X)[kCqrMaxB + 1] = reinterpret_cast<float(*)[kCqrMaxB + 1]>(cqr_sm);  // kCqrRows rows
    float* sRh = cqr_sm + kCqrRows * (kCqrMaxB + 1);
    float* sRl = sRh + kCqrMaxB * kCqrMaxB;
    float* sri = sRl + kCqrMaxB * kCqrMaxB;
    const int tid = threadIdx.x;
    const int64_t r0 = (int64_t)blockIdx.x * kCqrRows;
    const int nr = (int)min((int64_t)kCqrRows, m1 - r0);
    for (int e = tid; e < nr * bb; e += kCqrThreads) {
        const int r = e % nr, c = e / nr;
        X[r][c] = P[(int64_t)c * ldp + r0 + r];
    }
    if (R1h != nullptr) {
        for (int e = tid; e < bb * bb; e += kCqrThreads) {
            const int o = (e / bb) * kCqrMaxB + e % bb;
            sRh[o] = R1h[o];
            sRl[o] = R1l[o];
        }
        for (int e = tid; e < bb; e += kCqrThreads) sri[e] = r1inv[e];
    }
    __syncthreads();
    if (R1h != nullptr) {
        // this thread's row, solved in place in the shared tile (stride kCqrMaxB + 1: no bank conflicts)
        if (tid < nr) row_solve(X[tid], X[tid], bb, sRh, sRl, kCqrMaxB, sri);
        __syncthreads();
        for (int e = tid; e < nr * bb; e += kCqrThreads) {
            const int r = e % nr, c = e / nr;
            Q1[(int64_t)c * m1 + r0 + r] = X[r][c];
        }
    }
    const int ne = bb * (bb + 1) / 2;
    for (int e = tid; e < ne; e += kCqrThreads) {
        int i, j;
        tri_ij(e, bb, i, j);
        float sh = 0.f, sl = 0.f;
        for (int r = 0; r < nr; ++r) dot2_add(sh, sl, X[r][i], X[r][j]);
        part[(size_t)blockIdx.x * kCqrNE + e] = (double)sh + (double)sl;
    }
}

// G[e] = sum over blocks g (in order) of part[g * NE + e].
__global__ void cqr_reduce_kernel(const double* __restrict__ part, int nblk, int ne, double* __restrict__ G,
                                  const int* flag, int pass, const Status* st)
{
    if (status_error(st)) return;
    if (pass == 2 && *(volatile const int*)flag) return;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ne) return;
    double s0 = 0.0, s1 = 0.0;
    int g = 0;
    for (; g + 1 < nblk; g += 2) {
        s0 += part[(size_t)g * kCqrNE + e];
        s1 += part[(size_t)(g + 1) * kCqrNE + e];
    }
    if (g < nblk) s0 += part[(size_t)g * kCqrNE + e];
    G[e] = s0 + s1;
}

// One block: Cholesky G = R^T R in FP64 (right-looking, reciprocal square roots), the fallback test,
// R as float pairs (row-major, ld kCqrMaxB) with FP32 reciprocals of its diagonal, and for pass 2 the
// product R = R2 R1 (FP64) into Rprod.
__global__ void __launch_bounds__(kCqrSmallThreads) cqr_chol_kernel(const double* __restrict__ Gpk, int bb, int pass,
                                                                    double* __restrict__ R, float* __restrict__ Rh,
                                                                    float* __restrict__ Rl, float* __restrict__ rinv,
                                                                    const double* __restrict__ R1,
                                                                    double* __restrict__ Rprod, int* flag,
                                                                    const Status* st)
{
    if (status_error(st)) return;
    if (pass == 2 && *(volatile const int*)flag) return;
    __shared__ double S[kCqrMaxB][kCqrMaxB + 1];
    __shared__ double d0[kCqrMaxB];
    __shared__ int s_fail;
    const int tid = threadIdx.x;
    for (int e = tid; e < bb * bb; e += kCqrSmallThreads) S[e / bb][e % bb] = 0.0;
    if (tid == 0) s_fail = 0;
    __syncthreads();
    const int ne = bb * (bb + 1) / 2;
    for (int e = tid; e < ne; e += kCqrSmallThreads) {
        int i, j;
        tri_ij(e, bb, i, j);
        S[i][j] = Gpk[e];
    }
    __syncthreads();
    for (int j = tid; j < bb; j += kCqrSmallThreads) d0[j] = S[j][j];
    __syncthreads();
    const double thr = pass == 1 ? 1.4551915228366852e-11 /* 2^-36 */ : 0.5;
    for (int j = 0; j < bb; ++j) {
        const double djj = S[j][j];
        const bool ok = djj > thr * d0[j] && djj > 0.0;
        const double rs = ok ? rsqrt(djj) : 0.0;
        __syncthreads();
        if (!ok) {
            if (tid == 0) s_fail = 1;
            break;
        }
        // row j of R: S(j, j:) * rs; trailing update S(r, c) -= R(j, r) R(j, c), j < r <= c
        for (int c = j + tid; c < bb; c += kCqrSmallThreads) S[j][c] = c == j ? djj * rs : S[j][c] * rs;
        __syncthreads();
        const int w = bb - j - 1;
        for (int e = tid; e < w * w; e += kCqrSmallThreads) {
            const int r = j + 1 + e / w, c = j + 1 + e % w;
            if (r <= c) S[r][c] -= S[j][r] * S[j][c];
        }
        __syncthreads();
    }
    __syncthreads();
    if (s_fail) {
        if (tid == 0) *flag = 1;
        return;
    }
    for (int e = tid; e < bb * bb; e += kCqrSmallThreads) {
        const int i = e / bb, j = e % bb;
        const double v = i <= j ? S[i][j] : 0.0;
        R[i * kCqrMaxB + j] = v;
        const float h = (float)v;
        Rh[i * kCqrMaxB + j] = h;
        Rl[i * kCqrMaxB + j] = (float)(v - (double)h);
    }
    for (int j = tid; j < bb; j += kCqrSmallThreads) rinv[j] = (float)(1.0 / S[j][j]);
    if (pass == 1 && tid == 0) *flag = 0;
    if (pass == 2) {
        // Rprod = R2 R1 (both upper): (i, j) = sum_{i <= q <= j} R2(i, q) R1(q, j)
        __syncthreads();
        for (int e = tid; e < bb * bb; e += kCqrSmallThreads) {
            const int i = e / bb, j = e % bb;
            double s = 0.0;
            for (int q = i; q <= j; ++q) s += S[i][q] * R1[q * kCqrMaxB + j];
            Rprod[i * kCqrMaxB + j] = i <= j ? s : 0.0;
        }
    }
}

// One block: Q2top = Q1(0:bb, :) R2^{-1} (row solves), its LU without pivoting with the signs
// s_j = -sign(pivot), tau_j = -s_j U(j, j), W = U R2 as float pairs for the rows below, and the
// panel's top bb rows: R_house = S (R2 R1) on and above the diagonal, L1 below it.
__global__ void __launch_bounds__(kCqrSmallThreads) cqr_lu_kernel(
    const float* __restrict__ Q1, int64_t m1, int bb, const float* __restrict__ R2h, const float* __restrict__ R2l,
    const float* __restrict__ r2inv, const double* __restrict__ R2, const double* __restrict__ Rprod,
    float* __restrict__ A, int64_t lda, double* __restrict__ tau, float* __restrict__ Wh, float* __restrict__ Wl,
    float* __restrict__ winv, const int* flag, const Status* st)
{
    if (status_error(st)) return;
    if (*(volatile const int*)flag) return;
    extern __shared__ double cqr_lu_sm[];
    double(*U)[kCqrMaxB + 1] = reinterpret_cast<double(*)[kCqrMaxB + 1]>(cqr_lu_sm);
    double* sgn = cqr_lu_sm + kCqrMaxB * (kCqrMaxB + 1);
    float* sRh = reinterpret_cast<float*>(sgn + kCqrMaxB);
    float* sRl = sRh + kCqrMaxB * kCqrMaxB;
    float* sri = sRl + kCqrMaxB * kCqrMaxB;
    float(*Xq)[kCqrMaxB + 1] = reinterpret_cast<float(*)[kCqrMaxB + 1]>(sri + kCqrMaxB);
    const int tid = threadIdx.x;
    for (int e = tid; e < bb * bb; e += kCqrSmallThreads) {
        sRh[(e / bb) * kCqrMaxB + e % bb] = R2h[(e / bb) * kCqrMaxB + e % bb];
        sRl[(e / bb) * kCqrMaxB + e % bb] = R2l[(e / bb) * kCqrMaxB + e % bb];
        Xq[e % bb][e / bb] = Q1[(int64_t)(e / bb) * m1 + e % bb];
    }
    for (int e = tid; e < bb; e += kCqrSmallThreads) sri[e] = r2inv[e];
    __syncthreads();
    // Q2 rows = Q1 rows R2^{-1} (row solves; the FP32 result is what the rows below see too)
    if (tid < bb) row_solve(Xq[tid], Xq[tid], bb, sRh, sRl, kCqrMaxB, sri);
    __syncthreads();
    for (int e = tid; e < bb * bb; e += kCqrSmallThreads) U[e / bb][e % bb] = (double)Xq[e / bb][e % bb];
    __syncthreads();
    // LU of Q2top - S, right-looking, FP64; the sign is chosen at each pivot
    for (int j = 0; j < bb; ++j) {
        if (tid == 0) {
            const double s = U[j][j] >= 0.0 ? -1.0 : 1.0;
            sgn[j] = s;
            U[j][j] -= s;
        }
        __syncthreads();
        const double piv = U[j][j];
        const double rp = 1.0 / piv;
        for (int r = j + 1 + tid; r < bb; r += kCqrSmallThreads) U[r][j] *= rp;
        __syncthreads();
        const int w = bb - j - 1;
        for (int e = tid; e < w * w; e += kCqrSmallThreads) {
            const int r = j + 1 + e / w, c = j + 1 + e % w;
            U[r][c] -= U[r][j] * U[j][c];
        }
        __syncthreads();
    }
    // tau, the panel's top rows, and W = U R2 (upper x upper) as float pairs
    for (int j = tid; j < bb; j += kCqrSmallThreads) tau[j] = -sgn[j] * U[j][j];
    for (int e = tid; e < bb * bb; e += kCqrSmallThreads) {
        const int i = e / bb, j = e % bb;
        const float v = i <= j ? (float)(sgn[i] * Rprod[i * kCqrMaxB + j]) : (float)U[i][j];
        A[(int64_t)j * lda + i] = v;
        double w = 0.0;
        for (int q = i; q <= j; ++q) w += U[i][q] * R2[q * kCqrMaxB + j];
        w = i <= j ? w : 0.0;
        const float h = (float)w;
        Wh[i * kCqrMaxB + j] = h;
        Wl[i * kCqrMaxB + j] = (float)(w - (double)h);
        if (i == j) winv[i] = (float)(1.0 / w);
    }
}

// Rows r >= bb of the panel: V(r, :) = Q1(r, :) (U R2)^{-1}, one row per thread.
__global__ void __launch_bounds__(kCqrThreads) cqr_vform_kernel(const float* __restrict__ Q1, int64_t m1, int bb,
                                                                const float* __restrict__ Wh,
                                                                const float* __restrict__ Wl,
                                                                const float* __restrict__ winv, float* __restrict__ A,
                                                                int64_t lda, const int* flag, const Status* st)
{
    if (status_error(st)) return;
    if (*(volatile const int*)flag) return;
    extern __shared__ float cqr_v_sm[];
    float(*X)[kCqrMaxB + 1] = reinterpret_cast<float(*)[kCqrMaxB + 1]>(cqr_v_sm);  // kCqrThreads rows
    float* sWh = cqr_v_sm + kCqrThreads * (kCqrMaxB + 1);
    float* sWl = sWh + kCqrMaxB * kCqrMaxB;
    float* swi = sWl + kCqrMaxB * kCqrMaxB;
    const int tid = threadIdx.x;
    for (int e = tid; e < bb * bb; e += kCqrThreads) {
        sWh[(e / bb) * kCqrMaxB + e % bb] = Wh[(e / bb) * kCqrMaxB + e % bb];
        sWl[(e / bb) * kCqrMaxB + e % bb] = Wl[(e / bb) * kCqrMaxB + e % bb];
    }
    for (int e = tid; e < bb; e += kCqrThreads) swi[e] = winv[e];
    const int64_t rb0 = bb + (int64_t)blockIdx.x * kCqrThreads;
    const int nr = (int)min((int64_t)kCqrThreads, m1 - rb0);
    for (int e = tid; e < nr * bb; e += kCqrThreads) {
        const int r = e % nr, c = e / nr;
        X[r][c] = Q1[(int64_t)c * m1 + rb0 + r];
    }
    __syncthreads();
    if (tid < nr) row_solve(X[tid], X[tid], bb, sWh, sWl, kCqrMaxB, swi);
    __syncthreads();
    for (int e = tid; e < nr * bb; e += kCqrThreads) {
        const int r = e % nr, c = e / nr;
        A[(int64_t)c * lda + rb0 + r] = X[r][c];
    }
}

constexpr size_t kGramSmem = sizeof(float) * ((size_t)kCqrRows * (kCqrMaxB + 1) + 2 * kCqrMaxB * kCqrMaxB + kCqrMaxB);
constexpr size_t kVformSmem = sizeof(float) * ((size_t)kCqrThreads * (kCqrMaxB + 1) + 2 * kCqrMaxB * kCqrMaxB + kCqrMaxB);
constexpr size_t kLuSmem = sizeof(double) * ((size_t)kCqrMaxB * (kCqrMaxB + 1) + kCqrMaxB) +
                           sizeof(float) * (2 * kCqrMaxB * kCqrMaxB + kCqrMaxB + (size_t)kCqrMaxB * (kCqrMaxB + 1));

}  // namespace

// Regions of the CholeskyQR2 workspace for an m1-row panel, each 256-byte aligned, in this order:
// partial Grams, reduced Gram, R1, R2, R2 R1 (FP64), R1, R2, U R2 as float pairs, three reciprocal
// vectors, Q1 (m1 x 64 FP32), the fallback flag.
size_t cholqr_region_bytes(int i, int64_t m1)
{
    const int64_t nblk = (m1 + kCqrRows - 1) / kCqrRows;
    switch (i) {
    case 0: return sizeof(double) * (size_t)nblk * kCqrNE;
    case 1: return sizeof(double) * kCqrNE;
    case 2: case 3: case 4: return sizeof(double) * kCqrMaxB * kCqrMaxB;
    case 5: case 6: case 7: case 8: case 9: case 10: return sizeof(float) * kCqrMaxB * kCqrMaxB;
    case 11: case 12: case 13: return sizeof(float) * kCqrMaxB;
    case 14: return sizeof(float) * (size_t)m1 * kCqrMaxB;
    default: return 256;
    }
}
constexpr int kCqrRegions = 16;

size_t cholqr_ws_bytes(int64_t m_max)
{
    size_t b = 0;
    for (int i = 0; i < kCqrRegions; ++i) b += (cholqr_region_bytes(i, m_max) + 255) & ~(size_t)255;
    return b;
}

bool cholqr_supported(int bb) { return bb >= 1 && bb <= kCqrMaxB; }

cudaError_t launch_cholqr_panel(float* A, int64_t lda, int64_t m1, int bb, double* tau, void* ws, int** flag_out,
                                const Status* st, cudaStream_t s)
{
    char* w = static_cast<char*>(ws);
    const int nblk = (int)((m1 + kCqrRows - 1) / kCqrRows);
    char* reg[kCqrRegions];
    for (int i = 0; i < kCqrRegions; ++i) {
        reg[i] = w;
        w += (cholqr_region_bytes(i, m1) + 255) & ~(size_t)255;
    }
    double* part = reinterpret_cast<double*>(reg[0]);
    double* G = reinterpret_cast<double*>(reg[1]);
    double* R1 = reinterpret_cast<double*>(reg[2]);
    double* R2 = reinterpret_cast<double*>(reg[3]);
    double* Rp = reinterpret_cast<double*>(reg[4]);
    float* R1h = reinterpret_cast<float*>(reg[5]);
    float* R1l = reinterpret_cast<float*>(reg[6]);
    float* R2h = reinterpret_cast<float*>(reg[7]);
    float* R2l = reinterpret_cast<float*>(reg[8]);
    float* Wh = reinterpret_cast<float*>(reg[9]);
    float* Wl = reinterpret_cast<float*>(reg[10]);
    float* r1i = reinterpret_cast<float*>(reg[11]);
    float* r2i = reinterpret_cast<float*>(reg[12]);
    float* wi = reinterpret_cast<float*>(reg[13]);
    float* Q1 = reinterpret_cast<float*>(reg[14]);
    int* flag = reinterpret_cast<int*>(reg[15]);
    *flag_out = flag;
    const int ne = bb * (bb + 1) / 2;
    const unsigned rb = (unsigned)((ne + 127) / 128);
    static DevFlag attr_set;
    if (!attr_set.done()) {
        cudaError_t e = cudaFuncSetAttribute((const void*)cqr_gram_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)kGramSmem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute((const void*)cqr_vform_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)kVformSmem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute((const void*)cqr_lu_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)kLuSmem);
        if (e != cudaSuccess) return e;
        attr_set.set();
    }
    // pass 1
    cqr_gram_kernel<<<nblk, kCqrThreads, kGramSmem, s>>>(A, lda, m1, bb, nullptr, nullptr, nullptr, nullptr, part, flag,
                                                        st);
    cqr_reduce_kernel<<<rb, 128, 0, s>>>(part, nblk, ne, G, flag, 1, st);
    cqr_chol_kernel<<<1, kCqrSmallThreads, 0, s>>>(G, bb, 1, R1, R1h, R1l, r1i, nullptr, nullptr, flag, st);
    // pass 2 (Q1 = P R1^{-1} fused with its Gram)
    cqr_gram_kernel<<<nblk, kCqrThreads, kGramSmem, s>>>(A, lda, m1, bb, R1h, R1l, r1i, Q1, part, flag, st);
    cqr_reduce_kernel<<<rb, 128, 0, s>>>(part, nblk, ne, G, flag, 2, st);
    cqr_chol_kernel<<<1, kCqrSmallThreads, 0, s>>>(G, bb, 2, R2, R2h, R2l, r2i, R1, Rp, flag, st);
    // Householder reconstruction
    cqr_lu_kernel<<<1, kCqrSmallThreads, kLuSmem, s>>>(Q1, m1, bb, R2h, R2l, r2i, R2, Rp, A, lda, tau, Wh, Wl, wi,
                                                        flag, st);
    if (m1 > bb)
        cqr_vform_kernel<<<(unsigned)((m1 - bb + kCqrThreads - 1) / kCqrThreads), kCqrThreads, kVformSmem, s>>>(
            Q1, m1, bb, Wh, Wl, wi, A, lda, flag, st);
    return cudaGetLastError();
}

}  // namespace rq
