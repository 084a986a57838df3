// peaks.cu -- compute-throughput probes that give the roofline denominators this library reports
// against (measurement code, not part of the method): register-resident FP64 and FP32 FMA chains
// on every SM, and back-to-back tcgen05.mma (kind::tf32 and kind::f16 with BF16 operands) from
// shared memory into tensor memory on every SM.  Each probe is timed with CUDA events on the
// caller's stream and synchronises it.
#include "tc_common.cuh"

namespace rq {
namespace {

constexpr int kChains = 8;  // independent FMA chains per thread

__device__ int g_probe_sink;    // written only if a chain ends on an impossible value
__device__ int g_probe_error;   // a tensor-core probe block whose wait timed out

template <typename T>
__global__ void __launch_bounds__(256) fma_probe_kernel(T b, T c, int iters)
{
    T a[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) a[j] = (T)(threadIdx.x + j);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int j = 0; j < kChains; ++j) a[j] = fma(a[j], b, c);
    }
    T s = 0;
#pragma unroll
    for (int j = 0; j < kChains; ++j) s += a[j];
    if (s == (T)-1.2345e-7) g_probe_sink = 1;
}

// One block per SM: thread 0 issues `iters` MMAs of M = 128, N = 256 from zeroed shared-memory
// operands (K-major, 128-byte swizzle) into one tensor-memory accumulator, then waits (bounded) for
// their completion before the tensor memory is freed.
template <bool BF>
__global__ void __launch_bounds__(128, 1) tc_probe_kernel(int iters)
{
    extern __shared__ unsigned char smraw[];
    unsigned char* base = reinterpret_cast<unsigned char*>(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
    unsigned char* sa = base;                 // 128 rows x 128 bytes
    unsigned char* sb = base + 128 * 128;     // 256 rows x 128 bytes
    __shared__ __align__(8) uint64_t done;
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x;
    for (int i = tid; i < (128 + 256) * 128 / 16; i += blockDim.x)
        reinterpret_cast<int4*>(base)[i] = make_int4(0, 0, 0, 0);
    // the zeroed operands are read by the tensor core through the async proxy
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (tid < 32) tc::tmem_alloc(&tmem_base, 256);
    if (tid == 0) {
        tc::mbar_init(&done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = tmem_base;
    if (tid == 0) {
        const uint64_t da = tc::umma_desc(sa), db = tc::umma_desc(sb);
        const uint32_t idesc = BF ? tc::idesc_bf16(128, 256) : tc::idesc_tf32(128, 256);
        for (int it = 0; it < iters; ++it) {
            const int k = it & 3;  // the four 32-byte K steps of the 128-byte rows
            if (BF)
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
                    "l"(da + 2 * k), "l"(db + 2 * k), "r"(idesc), "r"(it > 0 ? 1 : 0)
                    : "memory");
            else
                tc::mma_tf32_ss(tmem, da + 2 * k, db + 2 * k, idesc, it > 0 ? 1 : 0);
        }
        tc::mma_commit(&done);
        if (!tc::mbar_wait(&done, 0, nullptr)) {
            atomicExch(&g_probe_error, 1);
            tc::mbar_wait(&done, 0, nullptr);  // one more bounded wait before freeing tensor memory
        }
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (tid < 32) tc::tmem_dealloc(tmem, 256);
}

struct Timer {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    Timer()
    {
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
    }
    ~Timer()
    {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
    }
};

}  // namespace
}  // namespace rq

using namespace rq;

extern "C" __attribute__((visibility("default"))) int rqrcp_peak_probe(int kind, double* tflops, double* ms,
                                                                       void* stream)
{
    if (kind < RQRCP_PROBE_DFMA || kind > RQRCP_PROBE_TC_BF16) return -1;
    if (tflops == nullptr) return -2;
    cudaStream_t s = (cudaStream_t)stream;
    const int sms = dev_info().sms;
    Timer t;
    double flops = 0.0;
    auto launch = [&](bool timed) -> cudaError_t {
        if (timed) cudaEventRecord(t.e0, s);
        if (kind == RQRCP_PROBE_DFMA || kind == RQRCP_PROBE_FFMA) {
            const int threads = 256, blocks = sms * 8, iters = kind == RQRCP_PROBE_DFMA ? 4096 : 65536;
            if (kind == RQRCP_PROBE_DFMA)
                fma_probe_kernel<double><<<blocks, threads, 0, s>>>(0.999999, 1e-9, iters);
            else
                fma_probe_kernel<float><<<blocks, threads, 0, s>>>(0.999999f, 1e-9f, iters);
            flops = 2.0 * kChains * (double)iters * threads * blocks;
        } else {
            const bool bf = kind == RQRCP_PROBE_TC_BF16;
            const int iters = 16384;
            // operands need 1 KB + 48 KB; ask for more than half of the SM's shared memory so that one
            // block runs per SM and each holds its SM's tensor pipe alone
            const size_t smem = 120 * 1024;
            if (bf) {
                cudaFuncSetAttribute((const void*)tc_probe_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem);
                tc_probe_kernel<true><<<sms, 128, smem, s>>>(iters);
            } else {
                cudaFuncSetAttribute((const void*)tc_probe_kernel<false>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                tc_probe_kernel<false><<<sms, 128, smem, s>>>(iters);
            }
            flops = 2.0 * 128 * 256 * (bf ? 16 : 8) * (double)iters * sms;
        }
        if (timed) cudaEventRecord(t.e1, s);
        return cudaGetLastError();
    };
    int zero = 0;
    if (cudaMemcpyToSymbolAsync(g_probe_error, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        launch(false) != cudaSuccess || launch(true) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return RQRCP_ERR_CUDA;
    }
    int err = 0;
    float el = 0.f;
    if (cudaMemcpyFromSymbol(&err, g_probe_error, sizeof(int)) != cudaSuccess ||
        cudaEventElapsedTime(&el, t.e0, t.e1) != cudaSuccess) {
        cudaGetLastError();
        return RQRCP_ERR_CUDA;
    }
    if (err) return RQRCP_ERR_TIMEOUT;
    *tflops = el > 0.f ? flops / ((double)el * 1e-3) / 1e12 : 0.0;
    if (ms) *ms = el;
    return RQRCP_OK;
}
