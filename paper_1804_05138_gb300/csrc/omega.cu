// omega.cu -- the Gaussian sketching matrix of Alg. 2 ("Generate i.i.d. Gaussian matrix Omega"),
// drawn on the host and copied to the device.
//
// Philox4x64-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3",
// SC'11): ten rounds of two 64x64 -> 128-bit multiplies with the Weyl-sequence key schedule.  One
// 4-word block gives two Box-Muller pairs (Box & Muller 1958), i.e. four N(0,1) entries.  The host
// draw uses the C library's log, sqrt, cos and sin in IEEE double with no contraction of
// multiplies and adds (the library is built with -ffp-contract=off), so the same seed gives the
// same bits wherever this host code runs against the same C library.  The FP32 form's Omega is
// that FP64 draw rounded to float.
//
// Device copies go through launch_omega: the host draw of the last (seed, l, m) is cached per
// element type, copied with one cudaMemcpy2DAsync from pageable memory, and kept alive until the
// copy has completed on the stream (a host callback releases it).
#include <cmath>
#include <cstring>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "internal.cuh"

namespace rq {
namespace {

struct PhiloxHost {
    static constexpr uint64_t kMul0 = 0xD2E7470EE14C6C93ull;
    static constexpr uint64_t kMul1 = 0xCA5A826395121157ull;
    static constexpr uint64_t kWeyl0 = 0x9E3779B97F4A7C15ull;  // golden ratio
    static constexpr uint64_t kWeyl1 = 0xBB67AE8584CAA73Bull;  // sqrt(3) - 1

    // counter (c0, 0, 0, 0), key (k0, 0)
    static void block(uint64_t c0, uint64_t k0, uint64_t w[4])
    {
        uint64_t x0 = c0, x1 = 0, x2 = 0, x3 = 0, k1 = 0;
        for (int round = 0; round < 10; ++round) {
            const unsigned __int128 a = (unsigned __int128)kMul0 * x0;
            const unsigned __int128 b = (unsigned __int128)kMul1 * x2;
            const uint64_t a_hi = (uint64_t)(a >> 64), a_lo = (uint64_t)a;
            const uint64_t b_hi = (uint64_t)(b >> 64), b_lo = (uint64_t)b;
            x0 = b_hi ^ x1 ^ k0;
            x1 = b_lo;
            x2 = a_hi ^ x3 ^ k1;
            x3 = a_lo;
            k0 += kWeyl0;
            k1 += kWeyl1;
        }
        w[0] = x0;
        w[1] = x1;
        w[2] = x2;
        w[3] = x3;
    }
};

// Philox blocks [blk0, blk1) of the draw: flat element q = r*m + c goes to out[r*ldo + c].
void draw_range(int64_t blk0, int64_t blk1, int64_t l, int64_t m, uint64_t seed, double* out, int64_t ldo)
{
    const double inv2p53 = 1.0 / 9007199254740992.0;  // 2^-53
    const double two_pi = 6.283185307179586476925286766559;
    const int64_t total = l * m;
    for (int64_t blk = blk0; blk < blk1; ++blk) {
        uint64_t w[4];
        PhiloxHost::block((uint64_t)blk, seed, w);
        for (int pair = 0; pair < 2; ++pair) {
            const double u1 = ((double)(w[2 * pair] >> 11) + 1.0) * inv2p53;  // (0, 1]
            const double u2 = (double)(w[2 * pair + 1] >> 11) * inv2p53;      // [0, 1)
            const double rho = std::sqrt(-2.0 * std::log(u1));
            const double theta = two_pi * u2;
            const int64_t q = blk * 4 + 2 * pair;
            if (q < total) out[(q / m) * ldo + q % m] = rho * std::cos(theta);
            if (q + 1 < total) out[((q + 1) / m) * ldo + (q + 1) % m] = rho * std::sin(theta);
        }
    }
}

template <typename T>
struct OmegaCache {
    std::mutex mu;
    uint64_t seed = 0;
    int64_t l = 0, m = 0;
    std::shared_ptr<std::vector<T>> data;
};

template <typename T>
OmegaCache<T>& omega_cache()
{
    static OmegaCache<T> c;
    return c;
}

// The host draw of (seed, l, m) as a dense row-major l x m array of T, from the cache.
template <typename T>
std::shared_ptr<std::vector<T>> cached_draw(int64_t l, int64_t m, uint64_t seed)
{
    OmegaCache<T>& c = omega_cache<T>();
    std::lock_guard<std::mutex> lock(c.mu);
    if (c.data && c.seed == seed && c.l == l && c.m == m) return c.data;
    auto v = std::make_shared<std::vector<T>>((size_t)(l * m));
    if constexpr (sizeof(T) == sizeof(double)) {
        host_omega(l, m, seed, v->data(), m);
    } else {
        std::vector<double> d((size_t)(l * m));
        host_omega(l, m, seed, d.data(), m);
        for (size_t i = 0; i < d.size(); ++i) (*v)[i] = (T)d[i];
    }
    c.seed = seed;
    c.l = l;
    c.m = m;
    c.data = v;
    return v;
}

template <typename T>
void CUDART_CB release_draw(void* p)
{
    delete static_cast<std::shared_ptr<std::vector<T>>*>(p);
}

}  // namespace

void host_omega(int64_t l, int64_t m, uint64_t seed, double* out, int64_t ldo)
{
    const int64_t nblk = (l * m + 3) / 4;
    unsigned nth = std::thread::hardware_concurrency();
    if (nth < 1) nth = 1;
    if (nth > 64) nth = 64;
    if (nblk < 8192) nth = 1;
    if (nth == 1) {
        draw_range(0, nblk, l, m, seed, out, ldo);
        return;
    }
    std::vector<std::thread> pool;
    const int64_t per = (nblk + nth - 1) / nth;
    for (unsigned t = 0; t < nth; ++t) {
        const int64_t b0 = (int64_t)t * per, b1 = b0 + per < nblk ? b0 + per : nblk;
        if (b0 >= b1) break;
        pool.emplace_back(draw_range, b0, b1, l, m, seed, out, ldo);
    }
    for (auto& th : pool) th.join();
}

template <typename T>
cudaError_t launch_omega(int64_t l, int64_t m, uint64_t seed, T* Om, int64_t ldo, cudaStream_t s)
{
    if (l * m == 0) return cudaSuccess;
    std::shared_ptr<std::vector<T>> v;
    try {
        v = cached_draw<T>(l, m, seed);
    } catch (...) {
        return cudaErrorMemoryAllocation;  // host memory for the draw
    }
    cudaError_t e = cudaMemcpy2DAsync(Om, (size_t)ldo * sizeof(T), v->data(), (size_t)m * sizeof(T),
                                      (size_t)m * sizeof(T), (size_t)l, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    // keep the host array alive until the copy has run
    auto* hold = new std::shared_ptr<std::vector<T>>(std::move(v));
    e = cudaLaunchHostFunc(s, release_draw<T>, hold);
    if (e != cudaSuccess) {
        // the callback was not enqueued: wait for the copy, then release the array here
        cudaGetLastError();
        e = cudaStreamSynchronize(s);
        delete hold;
    }
    return e;
}

template cudaError_t launch_omega<double>(int64_t, int64_t, uint64_t, double*, int64_t, cudaStream_t);
template cudaError_t launch_omega<float>(int64_t, int64_t, uint64_t, float*, int64_t, cudaStream_t);

}  // namespace rq

using namespace rq;

extern "C" __attribute__((visibility("default"))) int rqrcp_generate_omega_host(int64_t l, int64_t m, uint64_t seed,
                                                                                double* Omega, int64_t ldo)
{
    if (l < 1) return -1;
    if (m < 1) return -2;
    if (Omega == nullptr) return -4;
    if (ldo < m) return -5;
    try {
        host_omega(l, m, seed, Omega, ldo);
    } catch (...) {
        return RQRCP_ERR_CUDA;  // no host thread could be started
    }
    return RQRCP_OK;
}
