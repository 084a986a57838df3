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
#include "internal.cuh"

namespace rq {
namespace {

__host__ __device__ inline int pow2_at_least(int x)
{
    int p = 32;
    while (p < x) p <<= 1;
    return p;
}

template <typename T>
__global__ void __launch_bounds__(256) panel_kernel(T* __restrict__ A, int64_t lda, int64_t m1, int bb,
                                                    int64_t rpb, double* __restrict__ tau,
                                                    double* __restrict__ part, Status* st)
{
    if (status_error(st)) return;
    const int G = gridDim.x, g = blockIdx.x, tid = threadIdx.x, NTH = blockDim.x;
    extern __shared__ __align__(16) double S[];
    const int ldS = (int)(rpb | 1);
    const int bbp = pow2_at_least(bb);   // threads per row-chunk group
    const int nchunk = NTH / bbp;        // >= 1 because bb <= 256 and NTH == 256
    double* red = S + (size_t)ldS * bb;  // nchunk x bbp
    double* wk = red + (size_t)nchunk * bbp;
    double* diag = part + 2 * (size_t)G * bb;  // 2 x bb, after the partials
    __shared__ double sh_tau, sh_beta, sh_scal;

    const int64_t r0 = (int64_t)g * rpb;
    const int nrow = (int)max((int64_t)0, min(rpb, m1 - r0));
    for (int64_t e = tid; e < (int64_t)nrow * bb; e += NTH) {
        const int r = (int)(e % nrow), k = (int)(e / nrow);
        S[(size_t)k * ldS + r] = (double)A[(int64_t)k * lda + r0 + r];
    }
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
        if (tid < nk) {
            double s = 0.0;
            for (int c = 0; c < nchunk; ++c) s += red[c * bbp + tid];
            part[((size_t)buf * G + g) * bb + tid] = s;
        }
        if (r0 <= j && j < r0 + nrow) {
            const int rj = (int)(j - r0);
            for (int kk = tid; kk < nk; kk += NTH) diag[(size_t)buf * bb + kk] = S[(size_t)(j + kk) * ldS + rj];
        }
        // B. barrier
        if (!grid_barrier(st)) return;
        // C. reduce in block order, reflector, update
        if (tid < nk) {
            double s = 0.0;
            for (int h = 0; h < G; ++h) s += ld_cg(&part[((size_t)buf * G + h) * bb + tid]);
            red[tid] = s;
        }
        __syncthreads();
        if (tid == 0) {
            const double alpha = ld_cg(&diag[(size_t)buf * bb]);
            const double ss = red[0];
            double tj = 0.0, beta = alpha, scal = 0.0;
            if (ss != 0.0) {
                const double nrm = sqrt(alpha * alpha + ss);
                beta = (alpha >= 0.0) ? -nrm : nrm;
                tj = (beta - alpha) / beta;
                scal = 1.0 / (alpha - beta);
            }
            sh_tau = tj;
            sh_beta = beta;
            sh_scal = scal;
            if (g == 0) tau[j] = tj;
        }
        __syncthreads();
        if (tid > 0 && tid < nk) wk[tid] = sh_tau * (ld_cg(&diag[(size_t)buf * bb + tid]) + sh_scal * red[tid]);
        double* xj = S + (size_t)j * ldS;
        if (sh_tau != 0.0)
            for (int r = rstart + tid; r < nrow; r += NTH) xj[r] *= sh_scal;
        __syncthreads();
        if (sh_tau != 0.0) {
            const int ncol = nk - 1;
            const int rows = nrow - rstart;
            for (int64_t e = tid; e < (int64_t)rows * ncol; e += NTH) {
                const int r = rstart + (int)(e % rows), kk = 1 + (int)(e / rows);
                S[(size_t)(j + kk) * ldS + r] -= wk[kk] * xj[r];
            }
            if (r0 <= j && j < r0 + nrow) {
                const int rj = (int)(j - r0);
                for (int kk = 1 + tid; kk < nk; kk += NTH) S[(size_t)(j + kk) * ldS + rj] -= wk[kk];
            }
        }
        if (r0 <= j && j < r0 + nrow && tid == 0) S[(size_t)j * ldS + (j - r0)] = sh_beta;
        __syncthreads();
    }
    for (int64_t e = tid; e < (int64_t)nrow * bb; e += NTH) {
        const int r = (int)(e % nrow), k = (int)(e / nrow);
        A[(int64_t)k * lda + r0 + r] = (T)S[(size_t)k * ldS + r];
    }
}

size_t panel_smem(int64_t rpb, int bb)
{
    const int bbp = pow2_at_least(bb);
    const int nchunk = 256 / bbp;
    return sizeof(double) * ((size_t)(rpb | 1) * bb + (size_t)nchunk * bbp + (size_t)bbp);
}

int64_t panel_blocks(int64_t m1)
{
    int64_t G = (m1 + 63) / 64;
    if (G > dev_info().sms) G = dev_info().sms;
    return G < 1 ? 1 : G;
}

}  // namespace

size_t panel_part_bytes(int bb)
{
    // 2 x (max blocks) x bb partials + 2 x bb diagonal row
    return sizeof(double) * (2 * (size_t)1024 * bb + 2 * (size_t)bb);
}

bool panel_fits(int64_t m1, int bb, int /*elem_bytes*/)
{
    if (bb > 256) return false;
    const int64_t G = panel_blocks(m1);
    const int64_t rpb = (m1 + G - 1) / G;
    return panel_smem(rpb, bb) <= (size_t)dev_info().max_smem_optin - 1024;
}

template <typename T>
cudaError_t launch_panel(T* A, int64_t lda, int64_t m1, int bb, double* tau, double* part, Status* st,
                         cudaStream_t s)
{
    static bool attr_set = false;
    if (!attr_set) {
        if (cudaError_t e = allow_max_dynamic_smem(panel_kernel<T>)) return e;
        attr_set = true;
    }
    const int64_t G = panel_blocks(m1);
    const int64_t rpb = (m1 + G - 1) / G;
    const size_t smem = panel_smem(rpb, bb);
    const int threads = 256;
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, panel_kernel<T>, threads, smem);
    if (e != cudaSuccess) return e;
    if ((int64_t)per_sm * dev_info().sms < G) return cudaErrorCooperativeLaunchTooLarge;
    int64_t ldav = lda, m1v = m1, rpbv = rpb;
    int bbv = bb;
    void* args[] = {&A, &ldav, &m1v, &bbv, &rpbv, &tau, &part, &st};
    return cudaLaunchCooperativeKernel((const void*)panel_kernel<T>, dim3((unsigned)G), dim3(threads), args, smem, s);
}

template cudaError_t launch_panel<double>(double*, int64_t, int64_t, int, double*, double*, Status*, cudaStream_t);
template cudaError_t launch_panel<float>(float*, int64_t, int64_t, int, double*, double*, Status*, cudaStream_t);

}  // namespace rq
