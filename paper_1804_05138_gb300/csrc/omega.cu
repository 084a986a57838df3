// omega.cu -- Gaussian sketching matrix of Alg. 2 on the device.
//
// Philox4x64-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3",
// SC'11): ten rounds of two 64x64->128-bit multiplies with the Weyl-sequence key schedule.
// Each thread produces one 4-word block = two Box-Muller pairs = four N(0,1) entries.
#include "internal.cuh"

namespace rq {
namespace {

struct Philox4x64 {
    static constexpr unsigned long long kMul0 = 0xD2E7470EE14C6C93ull;
    static constexpr unsigned long long kMul1 = 0xCA5A826395121157ull;
    static constexpr unsigned long long kWeyl0 = 0x9E3779B97F4A7C15ull;  // golden ratio
    static constexpr unsigned long long kWeyl1 = 0xBB67AE8584CAA73Bull;  // sqrt(3) - 1

    __device__ static void block(unsigned long long c0, unsigned long long c1, unsigned long long c2,
                                 unsigned long long c3, unsigned long long k0, unsigned long long k1,
                                 unsigned long long out[4])
    {
#pragma unroll
        for (int round = 0; round < 10; ++round) {
            const unsigned long long hi0 = __umul64hi(kMul0, c0), lo0 = kMul0 * c0;
            const unsigned long long hi1 = __umul64hi(kMul1, c2), lo1 = kMul1 * c2;
            const unsigned long long n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
            c0 = n0;
            c1 = lo1;
            c2 = n2;
            c3 = lo0;
            k0 += kWeyl0;
            k1 += kWeyl1;
        }
        out[0] = c0;
        out[1] = c1;
        out[2] = c2;
        out[3] = c3;
    }
};

template <typename T>
__global__ void omega_kernel(int64_t l, int64_t m, uint64_t seed, T* __restrict__ Om, int64_t ldo)
{
    const int64_t total = l * m;
    const int64_t nblk = (total + 3) / 4;
    const double two53 = 1.0 / 9007199254740992.0;
    for (int64_t blk = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; blk < nblk;
         blk += (int64_t)gridDim.x * blockDim.x) {
        unsigned long long w[4];
        Philox4x64::block((unsigned long long)blk, 0, 0, 0, seed, 0, w);
#pragma unroll
        for (int pair = 0; pair < 2; ++pair) {
            const double u1 = ((double)(w[2 * pair] >> 11) + 1.0) * two53;  // (0, 1]
            const double u2 = (double)(w[2 * pair + 1] >> 11) * two53;      // [0, 1)
            const double rho = sqrt(-2.0 * log(u1));
            double sn, cs;
            sincospi(2.0 * u2, &sn, &cs);
            const int64_t q0 = blk * 4 + 2 * pair;
            if (q0 < total) Om[(q0 / m) * ldo + (q0 % m)] = (T)(rho * cs);
            if (q0 + 1 < total) Om[((q0 + 1) / m) * ldo + ((q0 + 1) % m)] = (T)(rho * sn);
        }
    }
}

}  // namespace

template <typename T>
cudaError_t launch_omega(int64_t l, int64_t m, uint64_t seed, T* Om, int64_t ldo, cudaStream_t s)
{
    const int64_t nblk = (l * m + 3) / 4;
    if (nblk == 0) return cudaSuccess;
    const int threads = 256;
    int64_t grid = (nblk + threads - 1) / threads;
    const int64_t cap = (int64_t)dev_info().sms * 8;
    if (grid > cap) grid = cap;
    omega_kernel<T><<<(unsigned)grid, threads, 0, s>>>(l, m, seed, Om, ldo);
    return cudaGetLastError();
}

template cudaError_t launch_omega<double>(int64_t, int64_t, uint64_t, double*, int64_t, cudaStream_t);
template cudaError_t launch_omega<float>(int64_t, int64_t, uint64_t, float*, int64_t, cudaStream_t);

}  // namespace rq
