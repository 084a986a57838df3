// lowrank.cu -- helpers of the low-rank product L = Q1 [R11 R12] Pi^T (Sec. I-A).
#include "internal.cuh"

namespace rq {
namespace {

// Rk(q, c) = -R(q, c) for q <= c (upper trapezoid of the first k rows), 0 below; ld = k.
__global__ void rk_kernel(const double* __restrict__ Af, int64_t ldaf, int64_t k, int64_t n, double* __restrict__ Rk)
{
    const int64_t total = k * n;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t q = e % k, c = e / k;
        Rk[e] = (q <= c) ? -Af[c * ldaf + q] : 0.0;
    }
}

// Q(:, 0:k) = I(:, 0:k).
__global__ void eye_kernel(double* __restrict__ Q, int64_t ldq, int64_t m, int64_t k)
{
    const int64_t total = m * k;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e % m, c = e / m;
        Q[c * ldq + r] = (r == c) ? 1.0 : 0.0;
    }
}

unsigned grid_for(int64_t total)
{
    int64_t g = (total + 255) / 256;
    const int64_t cap = (int64_t)dev_info().sms * 16;
    if (g > cap) g = cap;
    return (unsigned)(g < 1 ? 1 : g);
}

}  // namespace

cudaError_t launch_lowrank_rk(const double* Af, int64_t ldaf, int64_t k, int64_t n, double* Rk, cudaStream_t s)
{
    rk_kernel<<<grid_for(k * n), 256, 0, s>>>(Af, ldaf, k, n, Rk);
    return cudaGetLastError();
}

cudaError_t launch_eye(double* Q, int64_t ldq, int64_t m, int64_t k, cudaStream_t s)
{
    eye_kernel<<<grid_for(m * k), 256, 0, s>>>(Q, ldq, m, k);
    return cudaGetLastError();
}

}  // namespace rq
