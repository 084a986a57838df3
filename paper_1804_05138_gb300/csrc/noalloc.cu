// noalloc.cu -- rqrcp_sketch_noalloc: the sketch B = Omega A without any allocation by the
// caller or by the library.
//
// Its scratch (a status block and the split-K partial sums) lives in one file-scope device
// array of fixed size, created when the library is loaded onto a device and kept until the
// process exits.  Host code cannot use the array's name as a device address, so the first
// call on each device looks the address up with cudaGetSymbolAddress (with that device
// current) and caches it.
#include <mutex>

#include "internal.cuh"

namespace rq {
namespace {

constexpr size_t kNoAllocScratchBytes = size_t(8) << 20;  // 8 MiB per device
constexpr size_t kStatusBytes = 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_noalloc_mu;
void* g_noalloc_addr[64] = {};

// Device address of g_noalloc_scratch on the current device (looked up once per device).
int noalloc_scratch(void** out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return RQRCP_ERR_CUDA;
    }
    if (dev < 0 || dev >= 64) return RQRCP_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (g_noalloc_addr[dev] == nullptr) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) {
            cudaGetLastError();
            return RQRCP_ERR_CUDA;
        }
        g_noalloc_addr[dev] = p;
    }
    *out = g_noalloc_addr[dev];
    return RQRCP_OK;
}

}  // namespace
}  // namespace rq

using namespace rq;

extern "C" __attribute__((visibility("default"))) int rqrcp_sketch_noalloc(int64_t m, int64_t n, const double* A,
                                                                           int64_t lda, const double* Omega,
                                                                           int64_t l, int64_t ldo, double* B,
                                                                           int64_t ldb, void* stream)
{
    if (m < 1) return -1;
    if (n < 1) return -2;
    if (A == nullptr) return -3;
    if (lda < m) return -4;
    if (Omega == nullptr) return -5;
    if (l < 1) return -6;
    if (ldo < m) return -7;
    if (B == nullptr) return -8;
    if (ldb < l) return -9;
    // one split's partial sums must fit next to the status block
    const size_t per_split = (size_t)n * (size_t)l * sizeof(double);
    if (per_split > kNoAllocScratchBytes - kStatusBytes) return RQRCP_ERR_UNSUPPORTED;
    void* base = nullptr;
    if (int e = noalloc_scratch(&base)) return e;
    Status* st = static_cast<Status*>(base);
    double* P = reinterpret_cast<double*>(static_cast<char*>(base) + kStatusBytes);
    cudaStream_t s = (cudaStream_t)stream;

    // split K = m into at most 16 chunks, limited by what fits in the scratch
    int64_t max_split = (int64_t)((kNoAllocScratchBytes - kStatusBytes) / per_split);
    if (max_split > 16) max_split = 16;
    const int64_t tiles = ((l + 63) / 64) * ((n + 63) / 64);
    int64_t S = (4 * (int64_t)dev_info().sms + tiles - 1) / tiles;
    if (S > max_split) S = max_split;
    if (S > (m + 63) / 64) S = (m + 63) / 64;
    if (S < 1) S = 1;
    int64_t kchunk = (m + S - 1) / S;
    kchunk = ((kchunk + 15) / 16) * 16;
    const int nsplit = (int)((m + kchunk - 1) / kchunk);

    // the status block must start at zero on every call (the array keeps the last call's data)
    if (launch_init(st, 0, nullptr, 0, s) != cudaSuccess) return RQRCP_ERR_CUDA;
    if (launch_gemm_tn<double>(Omega, ldo, A, lda, l, n, m, kchunk, P, 0, 0, st, s) != cudaSuccess)
        return RQRCP_ERR_CUDA;
    if (launch_sketch_reduce<double>(P, nsplit, l, n, B, ldb, st, s) != cudaSuccess) return RQRCP_ERR_CUDA;
    return RQRCP_OK;
}
