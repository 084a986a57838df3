// gemm.cu -- SIMT contractions of the RQRCP hot loop (FP64 and FP32 storage).
//
//  gemm_tn   : split-K partials of X^T C for a short-and-wide result (M <= ~128 rows):
//              the sketch B = Omega A (X = Omega^T) and W = V^T [V C] of the compact-WY
//              update (X = V, first bb columns of C are V itself, giving the Gram V^T V).
//  gemm_update: C -= V Y, the rank-bb trailing update of Alg. 2 ("A(i:m,i+b:n) <- Q^T A").
//  sketch_reduce / tform / reduce_y: fixed-order reductions of the split-K partials, the
//              initial sketch norms, and the compact-WY factor T (LAPACK xLARFT, forward,
//              columnwise: T(j,j) = tau_j, T(0:j,j) = -tau_j T(0:j,0:j) V(:,0:j)^T v_j).
//
// Both contractions are K-major reads of column-major operands staged through shared
// memory in 16-deep slices; each thread owns a 4x4 register tile strided by 16 so that
// shared-memory reads are conflict-free and global reads are 128-byte coalesced.
#include <cuda_bf16.h>

#include "internal.cuh"

namespace rq {
namespace {

constexpr int TM = 64, TN = 64, TK = 16, NT = 256;

// Round to BF16 (round to nearest even) and back: the operand rounding of the BF16 sketch.
__device__ __forceinline__ float round_bf16(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }
__device__ __forceinline__ double round_bf16(double v) { return v; }

// Value of the reflector matrix V at (row q, column r) given the stored entry.
template <typename T>
__device__ __forceinline__ T vmask(T stored, int64_t q, int64_t r)
{
    return q > r ? stored : (q == r ? T(1) : T(0));
}

// RA register rows per thread: the block's tile is TMX = 16 RA rows of the result by TN columns
// (RA = 4 for the compact-WY Gram with bb <= 64; 3, 5 or 6 so that a sketch of l = b + p rows fits
// one tile without computing rows beyond l).
template <typename T, int RA>
__global__ void __launch_bounds__(NT) gemm_tn_kernel(const T* __restrict__ X, int64_t ldx,
                                                     const T* __restrict__ C, int64_t ldc, int64_t M,
                                                     int64_t N, int64_t K, int64_t kchunk,
                                                     double* __restrict__ P, int maskX, int64_t maskC,
                                                     int bf16, const Status* st)
{
    constexpr int TMX = 16 * RA;
    static_assert((TK * TMX) % NT == 0, "the X slice must split evenly over the block");
    if (status_error(st)) return;
    __shared__ T Xs[TK][TMX + 1];
    __shared__ T Cs[TK][TN + 1];
    const int tid = threadIdx.x;
    const int tm = tid & 15, tn = tid >> 4;
    const int64_t m0 = (int64_t)blockIdx.x * TMX;
    const int64_t n0 = (int64_t)blockIdx.y * TN;
    const int64_t kbeg = (int64_t)blockIdx.z * kchunk;
    const int64_t kend = min(K, kbeg + kchunk);

    // Two-level accumulation: a 64-deep inner sum in T, folded into an outer T sum.
    T acc[RA][4], outer[RA][4];
#pragma unroll
    for (int a = 0; a < RA; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = outer[a][b] = T(0);

    int inner = 0;
    for (int64_t k0 = kbeg; k0 < kend; k0 += TK) {
#pragma unroll
        for (int it = 0; it < (TK * TMX) / NT; ++it) {
            const int e = tid + it * NT;
            const int kk = e & (TK - 1);
            const int mm = e / TK;
            const int64_t q = k0 + kk;
            const int64_t r = m0 + mm;
            T v = T(0);
            if (q < kend && r < M) {
                v = X[r * ldx + q];
                if (maskX) v = vmask(v, q, r);
                if (bf16) v = round_bf16(v);
            }
            Xs[kk][mm] = v;
        }
#pragma unroll
        for (int it = 0; it < (TK * TN) / NT; ++it) {
            const int e = tid + it * NT;
            const int kk = e & (TK - 1);
            const int nn = e / TK;
            const int64_t q = k0 + kk;
            const int64_t c = n0 + nn;
            T v = T(0);
            if (q < kend && c < N) {
                v = C[c * ldc + q];
                if (c < maskC) v = vmask(v, q, c);
                if (bf16) v = round_bf16(v);
            }
            Cs[kk][nn] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < TK; ++kk) {
            T xa[RA], cb[4];
#pragma unroll
            for (int a = 0; a < RA; ++a) xa[a] = Xs[kk][tm + 16 * a];
#pragma unroll
            for (int b = 0; b < 4; ++b) cb[b] = Cs[kk][tn + 16 * b];
#pragma unroll
            for (int a = 0; a < RA; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] = fma(xa[a], cb[b], acc[a][b]);
        }
        __syncthreads();
        if (++inner == 4) {
            inner = 0;
#pragma unroll
            for (int a = 0; a < RA; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    outer[a][b] += acc[a][b];
                    acc[a][b] = T(0);
                }
        }
    }
    double* Pz = P + (int64_t)blockIdx.z * N * M;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        const int64_t c = n0 + tn + 16 * b;
        if (c >= N) continue;
#pragma unroll
        for (int a = 0; a < RA; ++a) {
            const int64_t r = m0 + tm + 16 * a;
            if (r < M) Pz[c * M + r] = (double)outer[a][b] + (double)acc[a][b];
        }
    }
}

// Register rows per thread of the SIMT contraction for an M-row result: one tile of 48, 64, 80 or
// 96 rows when M fits, else 64-row tiles.
inline int gemm_tn_ra(int64_t M) { return M <= 48 ? 3 : M <= 64 ? 4 : M <= 80 ? 5 : M <= 96 ? 6 : 4; }

template <typename T>
__global__ void __launch_bounds__(NT) gemm_update_kernel(T* __restrict__ C, int64_t ldc,
                                                         const T* __restrict__ V, int64_t ldv,
                                                         const double* __restrict__ Y, int64_t ldy,
                                                         int64_t mr, int64_t nc, int64_t kb, int maskV,
                                                         const int32_t* __restrict__ colmap,
                                                         const Status* st)
{
    if (status_error(st)) return;
    __shared__ T Vs[TK][TM + 1];
    __shared__ T Ys[TK][TN + 1];
    const int tid = threadIdx.x;
    const int tm = tid & 15, tn = tid >> 4;
    const int64_t r0 = (int64_t)blockIdx.x * TM;
    const int64_t c0 = (int64_t)blockIdx.y * TN;
    T acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = T(0);

    for (int64_t q0 = 0; q0 < kb; q0 += TK) {
#pragma unroll
        for (int it = 0; it < (TK * TM) / NT; ++it) {
            const int e = tid + it * NT;
            const int rr = e & (TM - 1);
            const int kk = e / TM;
            const int64_t r = r0 + rr, q = q0 + kk;
            T v = T(0);
            if (r < mr && q < kb) {
                v = V[q * ldv + r];
                if (maskV) v = vmask(v, r, q);
            }
            Vs[kk][rr] = v;
        }
#pragma unroll
        for (int it = 0; it < (TK * TN) / NT; ++it) {
            const int e = tid + it * NT;
            const int kk = e & (TK - 1);
            const int cc = e / TK;
            const int64_t q = q0 + kk, c = c0 + cc;
            Ys[kk][cc] = (q < kb && c < nc) ? (T)Y[c * ldy + q] : T(0);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < TK; ++kk) {
            T va[4], yb[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) va[a] = Vs[kk][tm + 16 * a];
#pragma unroll
            for (int b = 0; b < 4; ++b) yb[b] = Ys[kk][tn + 16 * b];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] = fma(va[a], yb[b], acc[a][b]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        const int64_t c = c0 + tn + 16 * b;
        if (c >= nc) continue;
        const int64_t cd = colmap ? (int64_t)colmap[c] : c;
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            const int64_t r = r0 + tm + 16 * a;
            if (r < mr) C[cd * ldc + r] -= acc[a][b];
        }
    }
}

// One warp per column of B: sum the split-K partials in split order, store, and fold the
// column norm^2 into the running maximum (non-negative doubles order like their bits).
template <typename T>
__global__ void sketch_reduce_kernel(const double* __restrict__ P, int nsplit, int64_t l, int64_t n,
                                     T* __restrict__ B, int64_t ldb, Status* st)
{
    // a non-finite sketch column flagged by another block of this launch does not stop the others:
    // every column of B is written (NaN/Inf where the input is not finite)
    const int e0 = status_error(st);
    if (e0 != 0 && e0 != RQRCP_ERR_NONFINITE) return;
    const int lane = threadIdx.x & 31;
    const int64_t j = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    if (j >= n) return;
    double nu = 0.0;
    bool finite = true;
    for (int64_t r = lane; r < l; r += 32) {
        double s = 0.0;
        for (int sp = 0; sp < nsplit; ++sp) s += P[((int64_t)sp * n + j) * l + r];
        const T v = (T)s;
        B[j * ldb + r] = v;
        finite = finite && isfinite((double)v);
        nu += (double)v * (double)v;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nu += __shfl_xor_sync(0xffffffffu, nu, o);
    finite = __all_sync(0xffffffffu, finite);
    if (lane == 0) {
        if (!finite || !isfinite(nu)) set_error(st, RQRCP_ERR_NONFINITE);
        else atomicMax(&st->nu0bits, (unsigned long long)__double_as_longlong(nu));
    }
}

// One block per row r of T.  The rows of the forward columnwise recurrence are independent:
// T(r,r) = tau_r and T(r,j) = -tau_j sum_{q=r}^{j-1} T(r,q) G(q,j), G = V^T V.  The block sums
// G(r:bb, r:bb) from the split-K partials into shared memory (each thread keeps kTfEnt entries in
// flight, the splits outermost, so a pass costs one memory round trip per split); warp 0 runs the
// recurrence column by column: lane j mod 32 owns column j, finishes T(r,q)
// at step q and broadcasts it, and every lane adds its terms to the columns it owns (one product,
// one shuffle and one FMA per step).
constexpr int kTfEnt = 16;      // G entries per thread in flight
constexpr int kTfThreads = 256;
__global__ void __launch_bounds__(kTfThreads) tform_kernel(const double* __restrict__ P, int nsplit, int64_t ncols, int bb,
                             const double* __restrict__ tau, double* __restrict__ Tm, const Status* st)
{
    if (status_error(st)) return;
    extern __shared__ double sm[];
    const int r = blockIdx.x;
    const int w = bb - r;
    double* Gs = sm;          // Gs[jj * w + qq] = G(r + qq, r + jj), qq < jj
    double* Tr = sm + w * w;  // T(r, r..bb-1)
    const int64_t stride = ncols * bb;
    for (int e0 = 0; e0 < w * w; e0 += kTfEnt * (int)blockDim.x) {
        double acc[kTfEnt];
        int64_t off[kTfEnt];
#pragma unroll
        for (int u = 0; u < kTfEnt; ++u) {
            const int e = e0 + u * (int)blockDim.x + (int)threadIdx.x;
            const int qq = e % w, jj = e / w;
            acc[u] = 0.0;
            off[u] = (e < w * w && qq < jj) ? (int64_t)(r + jj) * bb + r + qq : -1;
        }
        for (int sp = 0; sp < nsplit; ++sp)
#pragma unroll
            for (int u = 0; u < kTfEnt; ++u)
                if (off[u] >= 0) acc[u] += P[sp * stride + off[u]];
#pragma unroll
        for (int u = 0; u < kTfEnt; ++u) {
            const int e = e0 + u * (int)blockDim.x + (int)threadIdx.x;
            if (e < w * w) Gs[e] = acc[u];
        }
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        constexpr int NJ = 4;  // columns per lane (bb <= 128)
        const int lane = threadIdx.x;
        double acc[NJ], tj[NJ];
#pragma unroll
        for (int u = 0; u < NJ; ++u) {
            const int jj = lane + 32 * u;
            acc[u] = 0.0;
            tj[u] = jj < w ? tau[r + jj] : 0.0;
        }
        for (int qq = 0; qq < w; ++qq) {
            const int u0 = qq >> 5;
            double x = 0.0;
#pragma unroll
            for (int u = 0; u < NJ; ++u)
                if (u == u0) x = qq == 0 ? tj[u] : -tj[u] * acc[u];
            x = __shfl_sync(0xffffffffu, x, qq & 31);
            if (lane == (qq & 31)) Tr[qq] = x;
#pragma unroll
            for (int u = 0; u < NJ; ++u) {
                const int jj = lane + 32 * u;
                if (jj > qq && jj < w) acc[u] = fma(x, Gs[jj * w + qq], acc[u]);
            }
        }
    }
    __syncthreads();
    for (int j = threadIdx.x; j < bb; j += blockDim.x) Tm[(int64_t)j * bb + r] = (j < r) ? 0.0 : Tr[j - r];
}

// One warp per column c: W = sum of partials (column c0 + c), Y(:,c) = T^T W (transT) or T W.
__global__ void reduce_y_kernel(const double* __restrict__ P, int nsplit, int64_t ncols, int64_t c0, int bb,
                                const double* __restrict__ Tm, int transT, double* __restrict__ Y, int64_t nc,
                                const Status* st)
{
    if (status_error(st)) return;
    extern __shared__ double sm[];
    // Ts[q * ldT + r] = op(T)(r, q): lanes (r) read consecutive words
    const int ldT = bb | 1;
    double* Ts = sm;                      // bb x ldT
    const int nw = blockDim.x / 32;
    double* Wsh = sm + (size_t)bb * ldT;  // nw x bb
    for (int e = threadIdx.x; e < bb * bb; e += blockDim.x) {
        const int r = e % bb, q = e / bb;  // T column-major: T(a, b) = Tm[b * bb + a]
        Ts[q * ldT + r] = transT ? Tm[r * bb + q] : Tm[q * bb + r];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    double* Wc = Wsh + w * bb;
    for (int64_t c = (int64_t)blockIdx.x * nw + w; c < nc; c += (int64_t)gridDim.x * nw) {
        const int64_t col = c0 + c;
        for (int q = lane; q < bb; q += 32) {  // four partial sums in flight
            const double* pe = P + col * bb + q;
            const int64_t stride = ncols * bb;
            double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
            int sp = 0;
            for (; sp + 4 <= nsplit; sp += 4) {
                s0 += pe[(sp + 0) * stride];
                s1 += pe[(sp + 1) * stride];
                s2 += pe[(sp + 2) * stride];
                s3 += pe[(sp + 3) * stride];
            }
            for (; sp < nsplit; ++sp) s0 += pe[sp * stride];
            Wc[q] = (s0 + s1) + (s2 + s3);
        }
        __syncwarp();
        for (int r = lane; r < bb; r += 32) {
            double s = 0.0;
            if (transT)
                for (int q = 0; q <= r; ++q) s += Ts[q * ldT + r] * Wc[q];
            else
                for (int q = r; q < bb; ++q) s += Ts[q * ldT + r] * Wc[q];
            Y[c * bb + r] = s;
        }
        __syncwarp();
    }
}

// reduce_y for the FP32 form: the same Y = op(T) W, W = sum_sp P[sp], with FP32 arithmetic of
// FP64-class accuracy.  T and the FP64 sums W are split into two floats each (x = hi + lo); every
// term op(T)(r,q) W(q,c) enters as an error-free product hi*hi' (FMA residual) plus the cross
// terms, summed with TwoSum and a carried compensation (Ogita, Rump, Oishi, Dot2).  One block per
// 64 columns; every thread owns a 4 x 4 register tile (rows tm + 16 a, columns tn + 16 b) and runs
// the full contraction over q, the zeros of the triangle taking the rest.
__global__ void __launch_bounds__(256) reduce_y_f32c_kernel(const double* __restrict__ P, int nsplit, int64_t ncols,
                                                            int64_t c0, int bb, const double* __restrict__ Tm,
                                                            int transT, double* __restrict__ Y, int64_t nc,
                                                            const Status* st)
{
    if (status_error(st)) return;
    extern __shared__ __align__(16) float smf[];
    const int ld = 65;
    float* Th = smf;               // [q][r] = op(T)(r, q), bb x ld
    float* Tl = Th + 64 * ld;
    float* Wh = Tl + 64 * ld;      // [q][c] = W(q, c), bb x ld
    float* Wl = Wh + 64 * ld;
    const int tid = threadIdx.x, tm = tid & 15, tn = tid >> 4;
    const int64_t cb = (int64_t)blockIdx.x * 64;
#pragma unroll
    for (int u = 0; u < 16; ++u) {  // 16 entries per thread, all loads in flight
        const int e = tid + 256 * u;
        const int r = e & 63, q = e >> 6;  // T column-major: T(a, b) = Tm[b * bb + a]
        double tv = 0.0;
        if (r < bb && q < bb) tv = transT ? Tm[r * bb + q] : Tm[q * bb + r];
        const float h = (float)tv;
        Th[q * ld + r] = h;
        Tl[q * ld + r] = (float)(tv - (double)h);
    }
    {  // W = sum of the split partials: 16 entries per thread, the splits outermost
        double acc[16];
        int64_t off[16];
        const int64_t stride = ncols * bb;
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            const int e = tid + 256 * u;
            const int q = e & 63, c = e >> 6;  // P[sp][col][q]: q fastest, coalesced
            acc[u] = 0.0;
            off[u] = (q < bb && cb + c < nc) ? (c0 + cb + c) * bb + q : -1;
        }
        for (int sp = 0; sp < nsplit; ++sp)
#pragma unroll
            for (int u = 0; u < 16; ++u)
                if (off[u] >= 0) acc[u] += P[sp * stride + off[u]];
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            const int e = tid + 256 * u;
            const int q = e & 63, c = e >> 6;
            const float h = (float)acc[u];
            Wh[q * ld + c] = h;
            Wl[q * ld + c] = (float)(acc[u] - (double)h);
        }
    }
    __syncthreads();
    float sh[4][4], cp[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) sh[a][b] = cp[a][b] = 0.f;
    for (int q = 0; q < bb; ++q) {
        float th[4], tl[4], wh[4], wl[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            th[a] = Th[q * ld + tm + 16 * a];
            tl[a] = Tl[q * ld + tm + 16 * a];
        }
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            wh[b] = Wh[q * ld + tn + 16 * b];
            wl[b] = Wl[q * ld + tn + 16 * b];
        }
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const float pr = th[a] * wh[b];
                const float pe = fmaf(th[a], wh[b], -pr);
                const float t = sh[a][b] + pr;
                const float z = t - sh[a][b];
                const float er = (sh[a][b] - (t - z)) + (pr - z);
                sh[a][b] = t;
                cp[a][b] += er + pe + fmaf(th[a], wl[b], tl[a] * wh[b]);
            }
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int r = tm + 16 * a;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int64_t c = cb + tn + 16 * b;
            if (r < bb && c < nc) Y[c * bb + r] = (double)sh[a][b] + (double)cp[a][b];
        }
    }
}

}  // namespace

template <typename T, int RA>
int occupancy_of_gemm_tn()
{
    static std::atomic<int> occ{0};
    int v = occ.load(std::memory_order_relaxed);
    if (v == 0) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, gemm_tn_kernel<T, RA>, NT, 0) != cudaSuccess || v < 1) {
            cudaGetLastError();
            v = 1;
        }
        occ.store(v, std::memory_order_relaxed);
    }
    return v;
}

int gemm_tn_blocks_per_sm(int elem_bytes, int64_t M)
{
    const int ra = gemm_tn_ra(M);
    if (elem_bytes == 8) {
        switch (ra) {
        case 3: return occupancy_of_gemm_tn<double, 3>();
        case 5: return occupancy_of_gemm_tn<double, 5>();
        case 6: return occupancy_of_gemm_tn<double, 6>();
        default: return occupancy_of_gemm_tn<double, 4>();
        }
    }
    switch (ra) {
    case 3: return occupancy_of_gemm_tn<float, 3>();
    case 5: return occupancy_of_gemm_tn<float, 5>();
    case 6: return occupancy_of_gemm_tn<float, 6>();
    default: return occupancy_of_gemm_tn<float, 4>();
    }
}

int gemm_tn_tile_rows(int64_t M) { return 16 * gemm_tn_ra(M); }

template <typename T>
cudaError_t launch_gemm_tn(const T* X, int64_t ldx, const T* C, int64_t ldc, int64_t M, int64_t N,
                           int64_t K, int64_t kchunk, double* P, int maskX, int64_t maskC,
                           const Status* st, cudaStream_t s, int bf16)
{
    if (M <= 0 || N <= 0 || K <= 0) return cudaSuccess;
    const int ra = gemm_tn_ra(M);
    const int64_t tmx = 16 * ra;
    dim3 grid((unsigned)((M + tmx - 1) / tmx), (unsigned)((N + TN - 1) / TN), (unsigned)((K + kchunk - 1) / kchunk));
    switch (ra) {
    case 3: gemm_tn_kernel<T, 3><<<grid, NT, 0, s>>>(X, ldx, C, ldc, M, N, K, kchunk, P, maskX, maskC, bf16, st); break;
    case 5: gemm_tn_kernel<T, 5><<<grid, NT, 0, s>>>(X, ldx, C, ldc, M, N, K, kchunk, P, maskX, maskC, bf16, st); break;
    case 6: gemm_tn_kernel<T, 6><<<grid, NT, 0, s>>>(X, ldx, C, ldc, M, N, K, kchunk, P, maskX, maskC, bf16, st); break;
    default: gemm_tn_kernel<T, 4><<<grid, NT, 0, s>>>(X, ldx, C, ldc, M, N, K, kchunk, P, maskX, maskC, bf16, st);
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_gemm_update(T* C, int64_t ldc, const T* V, int64_t ldv, const double* Y, int64_t ldy,
                               int64_t mr, int64_t nc, int64_t kb, int maskV, const int32_t* colmap,
                               const Status* st, cudaStream_t s)
{
    if (mr <= 0 || nc <= 0 || kb <= 0) return cudaSuccess;
    dim3 grid((unsigned)((mr + TM - 1) / TM), (unsigned)((nc + TN - 1) / TN));
    gemm_update_kernel<T><<<grid, NT, 0, s>>>(C, ldc, V, ldv, Y, ldy, mr, nc, kb, maskV, colmap, st);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_sketch_reduce(const double* P, int nsplit, int64_t l, int64_t n, T* B, int64_t ldb,
                                 Status* st, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    const int threads = 256, cols_per_block = threads / 32;
    sketch_reduce_kernel<T><<<(unsigned)((n + cols_per_block - 1) / cols_per_block), threads, 0, s>>>(
        P, nsplit, l, n, B, ldb, st);
    return cudaGetLastError();
}

cudaError_t launch_tform(const double* P, int nsplit, int64_t ncols, int bb, const double* tau,
                         double* Tm, const Status* st, cudaStream_t s)
{
    const size_t smem = sizeof(double) * ((size_t)bb * bb + (size_t)bb);
    static DevFlag attr_set;
    if (!attr_set.done()) {
        if (cudaError_t e = allow_max_dynamic_smem(tform_kernel)) return e;
        attr_set.set();
    }
    tform_kernel<<<bb, kTfThreads, smem, s>>>(P, nsplit, ncols, bb, tau, Tm, st);
    return cudaGetLastError();
}

cudaError_t launch_reduce_y(const double* P, int nsplit, int64_t ncols, int64_t c0, int bb, const double* Tm,
                            int transT, double* Y, int64_t nc, const Status* st, cudaStream_t s, int fp32c)
{
    if (nc <= 0) return cudaSuccess;
    const int threads = 256, nw = threads / 32;
    const size_t smem = sizeof(double) * ((size_t)bb * (bb | 1) + (size_t)nw * bb);
    static DevFlag attr_set;
    if (!attr_set.done()) {
        if (cudaError_t e = allow_max_dynamic_smem(reduce_y_kernel)) return e;
        attr_set.set();
    }
    if (fp32c && bb <= 64) {
        static DevFlag set_c;
        if (!set_c.done()) {
            if (cudaError_t e = allow_max_dynamic_smem(reduce_y_f32c_kernel)) return e;
            set_c.set();
        }
        const size_t smem_c = sizeof(float) * 4 * 64 * 65;
        reduce_y_f32c_kernel<<<(unsigned)((nc + 63) / 64), 256, smem_c, s>>>(P, nsplit, ncols, c0, bb, Tm, transT, Y,
                                                                            nc, st);
        return cudaGetLastError();
    }
    int64_t grid = (nc + nw - 1) / nw;
    const int64_t cap = (int64_t)dev_info().sms * 4;
    if (grid > cap) grid = cap;
    reduce_y_kernel<<<(unsigned)grid, threads, smem, s>>>(P, nsplit, ncols, c0, bb, Tm, transT, Y, nc, st);
    return cudaGetLastError();
}

#define RQ_INST(T)                                                                                   \
    template cudaError_t launch_gemm_tn<T>(const T*, int64_t, const T*, int64_t, int64_t, int64_t,  \
                                           int64_t, int64_t, double*, int, int64_t, const Status*,  \
                                           cudaStream_t, int);                                      \
    template cudaError_t launch_gemm_update<T>(T*, int64_t, const T*, int64_t, const double*,       \
                                               int64_t, int64_t, int64_t, int64_t, int,             \
                                               const int32_t*, const Status*, cudaStream_t);        \
    template cudaError_t launch_sketch_reduce<T>(const double*, int, int64_t, int64_t, T*, int64_t, \
                                                 Status*, cudaStream_t);
RQ_INST(double)
RQ_INST(float)
#undef RQ_INST

}  // namespace rq
