// panel.cu -- "Do unpivoted QR on A(i:m, i:i+b-1)" (Alg. 2) as one cooperative kernel.
//
// The (m-i) x bb panel is split into contiguous row ranges, one per block, held in shared
// memory in FP64 for the whole factorization (FP32 panels are widened on load).  For each
// column j (reflector H_j, xLARFG convention):
//   A. every block forms partial dot products of column j with columns j..bb-1 over its rows
//      below the diagonal; the block owning row j also publishes that row;
//   B. one bounded grid barrier;
//   C. every block sums the partials in block order (identical in every block), forms
//      alpha, ||x||, beta, tau and scal = 1/(alpha - beta) in FP64, turns its part of column j
//      into the reflector tail v = scal * x and updates columns k > j by
//      a_k -= (tau * v^T a_k) v, with v^T a_k = a_k(j) + scal * (x^T a_k) from the partials.
// Partials and the diagonal row are double-buffered by the parity of j, so one barrier per
// column suffices.
#include <cstdlib>

#include "internal.cuh"

namespace rq {
namespace {

__host__ __device__ inline int pow2_at_least(int x)
{
    int p = 32;
    while (p < x) p <<= 1;
    return p;
}

// Sum of p[h * stride] for h = start, start + step, ... < G, in a fixed order, so the same value
// in every block.  Few terms (n <= 16, e.g. up to 64 blocks): batches of 8 loads at clamped (always
// valid) addresses, summed in two chains with the out-of-range slots as exact zeros; the step is
// then one or two L2 round trips.  More terms: up to 40 loads in flight, one chain (with 100+
// blocks the all-to-all read of the partials is bound by L2 bandwidth, and this form measured
// faster there).
__device__ __forceinline__ double sum_partials(const double* p, int G, int start, int step, size_t stride)
{
    const int n = start < G ? (G - 1 - start) / step + 1 : 0;
    if (n <= 16) {
        double s0 = 0.0, s1 = 0.0;
        for (int u = 0; u < n; u += 8) {
            double v[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int uu = u + q < n ? u + q : n - 1;
                v[q] = ld_cg(p + (size_t)(start + uu * step) * stride);
            }
#pragma unroll
            for (int q = 0; q < 8; q += 2) {
                s0 += u + q < n ? v[q] : 0.0;
                s1 += u + q + 1 < n ? v[q + 1] : 0.0;
            }
        }
        return s0 + s1;
    }
    constexpr int U = 40;
    double s = 0.0;
    for (int h0 = start; h0 < G; h0 += U * step) {
        double v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int h = h0 + u * step;
            v[u] = h < G ? ld_cg(p + (size_t)h * stride) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (h0 + u * step < G) s += v[u];
    }
    return s;
}

// Sum of red[c * bbp + k] over c < nchunk, even and odd c in two chains, fixed order.
__device__ __forceinline__ double sum_chunks(const double* red, int nchunk, int bbp, int k)
{
    double a = 0.0, b = 0.0;
    for (int c = 0; c + 1 < nchunk; c += 2) {
        a += red[c * bbp + k];
        b += red[(c + 1) * bbp + k];
    }
    if (nchunk & 1) a += red[(nchunk - 1) * bbp + k];
    return a + b;
}

// 256 threads: measured faster per column than 512 (the cross-block sums dominate, not the
// per-row work).
constexpr int kPanelThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kPanelThreads) panel_kernel(T* __restrict__ A, int64_t lda, int64_t m1, int bb,
                                                    int64_t rpb, double* __restrict__ tau,
                                                    double* __restrict__ part, Status* st)
{
    if (status_error(st)) return;
    const int G = gridDim.x, g = blockIdx.x, tid = threadIdx.x, NTH = blockDim.x;
    extern __shared__ __align__(16) double S[];
    const int ldS = (int)(rpb | 1);
    const int bbp = pow2_at_least(bb);   // threads per row-chunk group
    const int nchunk = NTH / bbp;        // >= 1 because bb <= 256 < NTH
    double* red = S + (size_t)ldS * bb;  // nchunk x bbp
    double* wk = red + (size_t)nchunk * bbp;
    double* sums = wk + bbp;
    double* dg = sums + bbp;  // the published diagonal row
    double* diag = part + 2 * (size_t)G * bb;  // 2 x bb, after the partials
    __shared__ double sh_tau, sh_beta, sh_scal;

    const int64_t r0 = (int64_t)g * rpb;
    const int nrow = (int)max((int64_t)0, min(rpb, m1 - r0));
    for (int k = 0; k < bb; ++k)
        for (int r = tid; r < nrow; r += NTH) S[(size_t)k * ldS + r] = (double)A[(int64_t)k * lda + r0 + r];
    __syncthreads();
    const int kidx = tid % bbp, chunk = tid / bbp;

    for (int j = 0; j < bb; ++j) {
        const int buf = j & 1;
        const int nk = bb - j;  // columns j..bb-1
        // A. partial dots over local rows strictly below row j
        const int rstart = (int)max((int64_t)0, (int64_t)j + 1 - r0);
        if (kidx < nk) {
            const double* xj = S + (size_t)j * ldS;
            const double* xk = S + (size_t)(j + kidx) * ldS;
            double s = 0.0;
            for (int r = rstart + chunk; r < nrow; r += nchunk) s += xj[r] * xk[r];
            red[chunk * bbp + kidx] = s;
        }
        __syncthreads();
        if (tid < nk) part[((size_t)buf * G + g) * bb + tid] = sum_chunks(red, nchunk, bbp, tid);
        if (r0 <= j && j < r0 + nrow) {
            const int rj = (int)(j - r0);
            for (int kk = tid; kk < nk; kk += NTH) diag[(size_t)buf * bb + kk] = S[(size_t)(j + kk) * ldS + rj];
        }
        // B. barrier
        if (!grid_barrier(st)) return;
        // C. reduce the blocks' partials (every thread takes blocks h = chunk (mod nchunk) of one
        //    column, then the nchunk group sums are added in group order: identical in every block)
        {
            double s = 0.0;
            if (kidx < nk) s = sum_partials(part + (size_t)buf * G * bb + kidx, G, chunk, nchunk, (size_t)bb);
            red[chunk * bbp + kidx] = s;
            if (tid < nk) dg[tid] = ld_cg(&diag[(size_t)buf * bb + tid]);
        }
        __syncthreads();
        if (tid < nk) sums[tid] = sum_chunks(red, nchunk, bbp, tid);
        __syncthreads();
        if (tid < 32) {
            double tj, beta, scal;
            warp_larfg(dg[0], sums[0], tj, beta, scal);
            if (tid == 0) {
                sh_tau = tj;
                sh_beta = beta;
                sh_scal = scal;
                if (g == 0) tau[j] = tj;
            }
        }
        __syncthreads();
        if (tid > 0 && tid < nk) wk[tid] = sh_tau * (dg[tid] + sh_scal * sums[tid]);
        double* xj = S + (size_t)j * ldS;
        if (sh_tau != 0.0)
            for (int r = rstart + tid; r < nrow; r += NTH) xj[r] *= sh_scal;
        __syncthreads();
        if (sh_tau != 0.0) {
            for (int r = rstart + tid; r < nrow; r += NTH) {
                const double v = xj[r];
                for (int kk = 1; kk < nk; ++kk) S[(size_t)(j + kk) * ldS + r] -= wk[kk] * v;
            }
            if (r0 <= j && j < r0 + nrow) {
                const int rj = (int)(j - r0);
                for (int kk = 1 + tid; kk < nk; kk += NTH) S[(size_t)(j + kk) * ldS + rj] -= wk[kk];
            }
        }
        if (r0 <= j && j < r0 + nrow && tid == 0) S[(size_t)j * ldS + (j - r0)] = sh_beta;
        __syncthreads();
    }
    for (int k = 0; k < bb; ++k)
        for (int r = tid; r < nrow; r += NTH) A[(int64_t)k * lda + r0 + r] = (T)S[(size_t)k * ldS + r];
}

// FP32 panel of the mixed form.  Storage and the reflector application stay in FP32; the
// dot products use the compensated Dot2 scheme (Ogita, Rump, Oishi, "Accurate sum and dot
// product", SIAM J. Sci. Comput. 2005: TwoProduct by FMA, TwoSum, compensation carried
// separately), each thread's (sum, compensation) pair is widened to FP64 for the cross-thread
// and cross-block sums, and every reflector (norm, beta, tau, 1/(alpha-beta)) is formed in
// FP64.  Same block layout and barrier pattern as the FP64 panel.
__device__ __forceinline__ void dot2_acc(float x, float y, float& s, float& c)
{
    const float p = x * y;
    const float e = fmaf(x, y, -p);      // exact product error
    const float t = s + p;
    const float z = t - s;
    const float q = (s - (t - z)) + (p - z);  // exact sum error
    s = t;
    c += q + e;
}

__global__ void __launch_bounds__(kPanelThreads) panel_f32_kernel(float* __restrict__ A, int64_t lda, int64_t m1, int bb,
                                                        int64_t rpb, double* __restrict__ tau,
                                                        double* __restrict__ part, Status* st,
                                                        const int* __restrict__ skip)
{
    if (status_error(st)) return;
    // the CholeskyQR2 panel (cholqr.cu) already factored this panel unless it set its fallback flag
    if (skip != nullptr && *(volatile const int*)skip == 0) return;
    const int G = gridDim.x, g = blockIdx.x, tid = threadIdx.x, NTH = blockDim.x;
    extern __shared__ __align__(16) double smd[];
    const int bbp = pow2_at_least(bb);
    const int nchunk = NTH / bbp;
    double* red = smd;                    // nchunk x bbp
    double* sums = red + (size_t)nchunk * bbp;
    double* dg = sums + bbp;  // the published diagonal row
    float* wk = reinterpret_cast<float*>(dg + bbp);  // bbp floats
    float* S = wk + bbp;                  // ldS x bb
    const int ldS = (int)(rpb | 1);
    double* diag = part + 2 * (size_t)G * bb;
    __shared__ double sh_tau, sh_beta, sh_scal;

    const int64_t r0 = (int64_t)g * rpb;
    const int nrow = (int)max((int64_t)0, min(rpb, m1 - r0));
    for (int k = 0; k < bb; ++k)
        for (int r = tid; r < nrow; r += NTH) S[(size_t)k * ldS + r] = A[(int64_t)k * lda + r0 + r];
    __syncthreads();
    const int kidx = tid % bbp, chunk = tid / bbp;

    for (int j = 0; j < bb; ++j) {
        const int buf = j & 1;
        const int nk = bb - j;
        const int rstart = (int)max((int64_t)0, (int64_t)j + 1 - r0);
        if (kidx < nk) {
            const float* xj = S + (size_t)j * ldS;
            const float* xk = S + (size_t)(j + kidx) * ldS;
            float sacc = 0.f, cacc = 0.f;
            for (int r = rstart + chunk; r < nrow; r += nchunk) dot2_acc(xj[r], xk[r], sacc, cacc);
            red[chunk * bbp + kidx] = (double)sacc + (double)cacc;
        }
        __syncthreads();
        if (tid < nk) part[((size_t)buf * G + g) * bb + tid] = sum_chunks(red, nchunk, bbp, tid);
        if (r0 <= j && j < r0 + nrow) {
            const int rj = (int)(j - r0);
            for (int kk = tid; kk < nk; kk += NTH) diag[(size_t)buf * bb + kk] = (double)S[(size_t)(j + kk) * ldS + rj];
        }
        if (!grid_barrier(st)) return;
        {
            double sv = 0.0;
            if (kidx < nk) sv = sum_partials(part + (size_t)buf * G * bb + kidx, G, chunk, nchunk, (size_t)bb);
            red[chunk * bbp + kidx] = sv;
            if (tid < nk) dg[tid] = ld_cg(&diag[(size_t)buf * bb + tid]);
        }
        __syncthreads();
        if (tid < nk) sums[tid] = sum_chunks(red, nchunk, bbp, tid);
        __syncthreads();
        if (tid < 32) {
            double tj, beta, scal;
            warp_larfg(dg[0], sums[0], tj, beta, scal);
            if (tid == 0) {
                sh_tau = tj;
                sh_beta = beta;
                sh_scal = scal;
                if (g == 0) tau[j] = tj;
            }
        }
        __syncthreads();
        if (tid > 0 && tid < nk)
            wk[tid] = (float)(sh_tau * (dg[tid] + sh_scal * sums[tid]));
        float* xj = S + (size_t)j * ldS;
        if (sh_tau != 0.0)
            for (int r = rstart + tid; r < nrow; r += NTH) xj[r] = (float)((double)xj[r] * sh_scal);
        __syncthreads();
        if (sh_tau != 0.0) {
            for (int r = rstart + tid; r < nrow; r += NTH) {
                const float v = xj[r];
                for (int kk = 1; kk < nk; ++kk) S[(size_t)(j + kk) * ldS + r] = fmaf(-wk[kk], v, S[(size_t)(j + kk) * ldS + r]);
            }
            if (r0 <= j && j < r0 + nrow) {
                const int rj = (int)(j - r0);
                for (int kk = 1 + tid; kk < nk; kk += NTH) S[(size_t)(j + kk) * ldS + rj] -= wk[kk];
            }
        }
        if (r0 <= j && j < r0 + nrow && tid == 0) S[(size_t)j * ldS + (j - r0)] = (float)sh_beta;
        __syncthreads();
    }
    for (int k = 0; k < bb; ++k)
        for (int r = tid; r < nrow; r += NTH) A[(int64_t)k * lda + r0 + r] = S[(size_t)k * ldS + r];
}

size_t panel_f32_smem(int64_t rpb, int bb)
{
    const int bbp = pow2_at_least(bb);
    const int nchunk = kPanelThreads / bbp;
    return sizeof(double) * ((size_t)nchunk * bbp + 2 * (size_t)bbp) + sizeof(float) * ((size_t)bbp + (size_t)(rpb | 1) * bb);
}

size_t panel_smem(int64_t rpb, int bb)
{
    const int bbp = pow2_at_least(bb);
    const int nchunk = kPanelThreads / bbp;
    return sizeof(double) * ((size_t)(rpb | 1) * bb + (size_t)nchunk * bbp + 3 * (size_t)bbp);
}

// Rows per block at least RQRCP_PANEL_MIN_ROWS (default 64), at most one block per SM.
int64_t panel_min_rows()
{
    static int64_t v = -1;
    if (v < 0) {
        const char* e = getenv("RQRCP_PANEL_MIN_ROWS");
        v = (e != nullptr && atoll(e) > 0) ? atoll(e) : 64;
    }
    return v;
}

// Blocks of the panel kernel: rows per block at least RQRCP_PANEL_MIN_ROWS, at most one block
// per SM, and enough blocks for each block's rows to fit in shared memory.
int64_t panel_blocks(int64_t m1, int bb, int elem_bytes)
{
    const int64_t rows = panel_min_rows();
    int64_t G = (m1 + rows - 1) / rows;
    const int64_t sms = dev_info().sms;
    if (G > sms) G = sms;
    if (G < 1) G = 1;
    const size_t lim = (size_t)dev_info().max_smem_optin - 1024;
    auto fits = [&](int64_t g) {
        const int64_t rpb = (m1 + g - 1) / g;
        return (elem_bytes == 4 ? panel_f32_smem(rpb, bb) : panel_smem(rpb, bb)) <= lim;
    };
    while (G < sms && !fits(G)) ++G;
    return G;
}

}  // namespace

size_t panel_part_bytes(int bb)
{
    // 2 x (max blocks) x bb partials + 2 x bb diagonal row
    return sizeof(double) * (2 * (size_t)1024 * bb + 2 * (size_t)bb);
}

bool panel_fits(int64_t m1, int bb, int elem_bytes)
{
    if (bb > 256) return false;
    const int64_t G = panel_blocks(m1, bb, elem_bytes);
    const int64_t rpb = (m1 + G - 1) / G;
    const size_t smem = elem_bytes == 4 ? panel_f32_smem(rpb, bb) : panel_smem(rpb, bb);
    return smem <= (size_t)dev_info().max_smem_optin - 1024;
}

template <typename T>
cudaError_t launch_panel(T* A, int64_t lda, int64_t m1, int bb, double* tau, double* part, Status* st,
                         cudaStream_t s, const int* skip)
{
    constexpr bool f32 = sizeof(T) == 4;
    const void* kern = f32 ? (const void*)panel_f32_kernel : (const void*)panel_kernel<double>;
    static DevFlag attr_set;
    if (!attr_set.done()) {
        if (cudaError_t e = f32 ? allow_max_dynamic_smem(panel_f32_kernel) : allow_max_dynamic_smem(panel_kernel<double>))
            return e;
        attr_set.set();
    }
    const int64_t G = panel_blocks(m1, bb, (int)sizeof(T));
    const int64_t rpb = (m1 + G - 1) / G;
    const size_t smem = f32 ? panel_f32_smem(rpb, bb) : panel_smem(rpb, bb);
    const int threads = kPanelThreads;
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
    if (e != cudaSuccess) return e;
    if ((int64_t)per_sm * dev_info().sms < G) return cudaErrorCooperativeLaunchTooLarge;
    int64_t ldav = lda, m1v = m1, rpbv = rpb;
    int bbv = bb;
    const int* skipv = skip;
    void* args_f64[] = {&A, &ldav, &m1v, &bbv, &rpbv, &tau, &part, &st};
    void* args_f32[] = {&A, &ldav, &m1v, &bbv, &rpbv, &tau, &part, &st, &skipv};
    return cudaLaunchCooperativeKernel(kern, dim3((unsigned)G), dim3(threads), f32 ? args_f32 : args_f64, smem, s);
}

template cudaError_t launch_panel<double>(double*, int64_t, int64_t, int, double*, double*, Status*, cudaStream_t,
                                          const int*);
template cudaError_t launch_panel<float>(float*, int64_t, int64_t, int, double*, double*, Status*, cudaStream_t,
                                         const int*);

}  // namespace rq
