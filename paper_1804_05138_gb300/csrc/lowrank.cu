// lowrank.cu -- helpers of the low-rank product L = Q1 [R11 R12] Pi^T (Sec. I-A).
#include "internal.cuh"

namespace rq {
namespace {

// Rk(q, c) = -R(q, c) for q <= c (upper trapezoid of the first k rows), 0 below; ld = k.
template <typename T>
__global__ void rk_kernel(const T* __restrict__ Af, int64_t ldaf, int64_t k, int64_t n, double* __restrict__ Rk)
{
    for (int64_t c = blockIdx.x; c < n; c += gridDim.x)
        for (int64_t q = threadIdx.x; q < k; q += blockDim.x) Rk[c * k + q] = (q <= c) ? -(double)Af[c * ldaf + q] : 0.0;
}

// Q(:, 0:k) = I(:, 0:k).
template <typename T>
__global__ void eye_kernel(T* __restrict__ Q, int64_t ldq, int64_t m, int64_t k)
{
    for (int64_t c = blockIdx.x; c < k; c += gridDim.x)
        for (int64_t r = threadIdx.x; r < m; r += blockDim.x) Q[c * ldq + r] = (r == c) ? T(1) : T(0);
}

unsigned grid_for(int64_t total)
{
    int64_t g = (total + 255) / 256;
    if (g > 65535) g = 65535;
    const int64_t cap = (int64_t)dev_info().sms * 16;
    if (g > cap) g = cap;
    return (unsigned)(g < 1 ? 1 : g);
}

}  // namespace

template <typename T>
cudaError_t launch_lowrank_rk(const T* Af, int64_t ldaf, int64_t k, int64_t n, double* Rk, cudaStream_t s)
{
    rk_kernel<T><<<grid_for(n * 256), 256, 0, s>>>(Af, ldaf, k, n, Rk);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_eye(T* Q, int64_t ldq, int64_t m, int64_t k, cudaStream_t s)
{
    eye_kernel<T><<<grid_for(k * 256), 256, 0, s>>>(Q, ldq, m, k);
    return cudaGetLastError();
}

template cudaError_t launch_lowrank_rk<double>(const double*, int64_t, int64_t, int64_t, double*, cudaStream_t);
template cudaError_t launch_lowrank_rk<float>(const float*, int64_t, int64_t, int64_t, double*, cudaStream_t);
template cudaError_t launch_eye<double>(double*, int64_t, int64_t, int64_t, cudaStream_t);
template cudaError_t launch_eye<float>(float*, int64_t, int64_t, int64_t, cudaStream_t);

}  // namespace rq
