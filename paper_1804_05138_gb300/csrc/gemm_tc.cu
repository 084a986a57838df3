// gemm_tc.cu -- tensor-core (tcgen05, kind::tf32) form of the split-K contraction
//   P[sp][c][r] = sum_{q in split sp} X(q, r) C(q, c),  r < M <= 128, c < N,
// for the FP32 form: the sketch B = Omega A (X = Omega^T) and W = V^T [V C] of the compact-WY
// update (X = V).  Both use 3xTF32: each operand x = hi + lo with hi = tf32(x), lo = tf32(x - hi),
// and x y ~ hi hi' + hi lo' + lo hi' (the lo lo' term, below 2^-22 |x y|, dropped).
//
// One block of 128 threads computes 128 columns of C against all M rows of X over one K split.
// Tiles are K-major (32 FP32 = one 128-byte swizzle row per column), brought in by TMA
// (cp.async.bulk.tensor, 128-byte swizzle) into a ring of stages with mbarrier completion.  All
// threads round each tile to TF32 hi parts in place, write the lo parts to a twin buffer and
// apply the unit-lower reflector mask where the tile covers the diagonal; one thread issues the
// chunk's tcgen05.mma chain into tensor memory and commits it to the stage's "empty" barrier.
// The accumulation over K happens outside the tensor core: each 32-row chunk's product is read
// back (tcgen05.ld) and summed in FP32 registers with round-to-nearest, folded into a
// compensated sum every TC_FOLD chunks, so the tensor core's own accumulator only ever adds the
// twelve products of one chunk.  The epilogue writes the FP64 partials.  Every wait is bounded;
// on timeout the block records RQRCP_ERR_TIMEOUT, waits (bounded) for its copies and MMA chains
// in flight and frees its tensor memory.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "internal.cuh"

namespace rq {
namespace {

constexpr int TC_THREADS = 128;
constexpr int TC_KC = 32;       // K per stage: one 128-byte swizzle row of FP32
constexpr int TC_NA = 128;      // columns of C per block (MMA M)
constexpr int TC_STAGES = 3;
constexpr unsigned long long kTcWaitNs = 2000000000ull;

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* b, unsigned cnt)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(cnt) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_wait(uint64_t* b, unsigned parity)
{
    const unsigned long long t0 = globaltimer_ns();
    for (;;) {
        unsigned ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(ok)
            : "r"(su32(b)), "r"(parity)
            : "memory");
        if (ok) return true;
        if (globaltimer_ns() - t0 > kTcWaitNs) return false;
    }
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            su32(dst)),
        "l"(map), "r"(x), "r"(y), "r"(su32(bar))
        : "memory");
}
// UMMA shared-memory descriptor: K-major, 128-byte swizzle, 8-row atoms 1024 bytes apart.
__device__ __forceinline__ uint64_t umma_desc(const void* base)
{
    const uint64_t addr = su32(base);
    return ((addr >> 4) & 0x3FFFull) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) | ((uint64_t)1 << 46) |
           ((uint64_t)2 << 61);
}
// Instruction descriptor: D FP32, A and B TF32, both K-major, N >> 3, M >> 4.
__device__ __forceinline__ uint32_t idesc_tf32(int m, int n)
{
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}
__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc, int acc)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(
            tmem_d),
        "l"(da), "l"(db), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar))
                 : "memory");
}
__device__ __forceinline__ float tf32_rn(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Apply the unit-lower reflector mask and (split3) the TF32 hi/lo split to one tile of `rows`
// 128-byte rows (row j holds K elements k0..k0+31 of column col0 + j, 16-byte chunks swizzled by
// j mod 8).  Columns c = col0 + j < mask_lim carry the reflector structure: element (q, c) with
// q = k0 + kk becomes 0 above the diagonal (q < c) and 1 on it.  hi = tf32(x), lo = tf32(x - hi).
__device__ __forceinline__ void prep_tile(float* hi, float* lo, int rows, int k0, long long col0, long long mask_lim,
                                          int split3)
{
    for (int e4 = threadIdx.x; e4 < rows * 8; e4 += TC_THREADS) {
        const int j = e4 >> 3, cp = e4 & 7;
        float4 v = reinterpret_cast<float4*>(hi)[e4];
        const long long c = col0 + j;
        if (c < mask_lim) {
            const int kk0 = ((cp ^ (j & 7)) << 2);
            float* vv = reinterpret_cast<float*>(&v);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const long long q = (long long)k0 + kk0 + u;
                if (q < c) vv[u] = 0.f;
                else if (q == c) vv[u] = 1.f;
            }
        }
        if (split3) {
            float4 h, l;
            h.x = tf32_rn(v.x); l.x = tf32_rn(v.x - h.x);
            h.y = tf32_rn(v.y); l.y = tf32_rn(v.y - h.y);
            h.z = tf32_rn(v.z); l.z = tf32_rn(v.z - h.z);
            h.w = tf32_rn(v.w); l.w = tf32_rn(v.w - h.w);
            reinterpret_cast<float4*>(hi)[e4] = h;
            reinterpret_cast<float4*>(lo)[e4] = l;
        } else if (c < mask_lim) {
            reinterpret_cast<float4*>(hi)[e4] = v;
        }
    }
}

struct TcArgs {
    int M, Nb;               // rows of X used (<= Nb), MMA N (multiple of 16)
    long long N, K;          // columns of C, contraction length
    long long kchunk;        // K per split (multiple of TC_KC)
    int xx0, xy0, cx0, cy0;  // tensor-map coordinates of X(0,0) and C(0,0)
    long long maskX, maskC;  // X columns r < maskX / C columns c < maskC carry the reflector mask
    int split3;
    int nst;                 // pipeline stages
    unsigned tmem_cols;
};

constexpr int TC_FOLD = 16;  // chunks summed in FP32 registers between compensated folds

// Per block: 128 columns of C x all Nb rows of X over one K split.  Chunk kc's products go to
// TMEM buffer kc % 2 (Nb columns each), started fresh (the hi*lo and lo*hi MMAs first, then hi*hi,
// so that the accumulator's roundings on the large terms are only the four hi*hi steps).  While
// chunk kc runs on the tensor pipe, every thread adds its row of chunk kc-1's buffer into FP32
// registers (acc); every TC_FOLD chunks acc is folded into an FP32 shared-memory sum S with the
// error-free TwoSum transformation, the rounding error carried back into acc (compensated sum).
template <int NBMAX>
__global__ void __launch_bounds__(TC_THREADS, 1)
    gemm_tn_tc_kernel(const __grid_constant__ CUtensorMap mapC, const __grid_constant__ CUtensorMap mapX, TcArgs a,
                      double* __restrict__ P, Status* st)
{
    __shared__ int s_skip;
    if (threadIdx.x == 0) s_skip = status_error(st);
    __syncthreads();
    if (s_skip) return;  // block-uniform: warp 0's tensor-memory allocation is warp-collective
    extern __shared__ unsigned char smraw[];
    unsigned char* base = reinterpret_cast<unsigned char*>(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
    const int tileC = TC_NA * TC_KC * 4;     // 16 KB
    const int tileX = a.Nb * TC_KC * 4;      // Nb * 128 bytes
    const int stage_bytes = 2 * tileC + 2 * tileX;
    const int nst = a.nst;
    float* Ssum = reinterpret_cast<float*>(base + (size_t)nst * stage_bytes);  // [c][row], Nb x 128
    __shared__ __align__(8) uint64_t full[4], empty[4];
    __shared__ uint32_t tmem_base;
    __shared__ int s_fail;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_base)),
                     "r"(a.tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int s = 0; s < nst; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        s_fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int e = tid; e < TC_NA * a.Nb; e += TC_THREADS) Ssum[e] = 0.f;
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = tmem_base;
    const long long n0 = (long long)blockIdx.x * TC_NA;
    const long long kbeg = (long long)blockIdx.y * a.kchunk;
    const long long kend = min(a.K, kbeg + a.kchunk);
    const int nchunks = (int)((kend - kbeg + TC_KC - 1) / TC_KC);
    const uint32_t idesc = idesc_tf32(TC_NA, a.Nb);
    auto stage_ptr = [&](int s) { return base + (size_t)s * stage_bytes; };
    int issued = 0;   // chunks whose TMA thread 0 has issued
    int landed = 0;   // chunks whose TMA thread 0 has seen complete
    int mma_done = 0; // chunks whose MMA chain this thread has seen complete
    auto issue = [&](int kc) {
        const int s = kc % nst;
        unsigned char* sp = stage_ptr(s);
        const int k0 = (int)(kbeg + (long long)kc * TC_KC);
        mbar_expect_tx(&full[s], tileC + tileX);
        tma_load_2d(sp, &mapC, a.cx0 + k0, a.cy0 + (int)n0, &full[s]);
        tma_load_2d(sp + 2 * tileC, &mapX, a.xx0 + k0, a.xy0, &full[s]);
    };
    if (tid == 0)
        for (; issued < nst && issued < nchunks; ++issued) issue(issued);

    float acc[NBMAX];
#pragma unroll
    for (int j = 0; j < NBMAX; ++j) acc[j] = 0.f;
    const int row = 32 * warp + lane;  // row of D = column n0 + row of C
    // add chunk kc's TMEM buffer (after its MMA chain completed) into acc
    auto drain = [&](int kc) -> bool {
        bool ok = mbar_wait(&empty[kc % nst], (unsigned)(kc / nst) & 1u);
        ok = __all_sync(0xffffffffu, ok);
        if (!ok) return false;
        mma_done = kc + 1;
        fence_after();
        const uint32_t tb = tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)((kc & 1) * a.Nb);
#pragma unroll
        for (int c0 = 0; c0 < NBMAX; c0 += 16) {
            if (c0 < a.Nb) {
                uint32_t r[16];
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                    "[%16];"
                    : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                      "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                      "=r"(r[15])
                    : "r"(tb + (uint32_t)c0));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int j = 0; j < 16; ++j) acc[c0 + j] += __uint_as_float(r[j]);
            }
        }
        return true;
    };
    // compensated fold: (S, e) = TwoSum(S, acc), acc = e
    auto fold = [&]() {
#pragma unroll
        for (int j = 0; j < NBMAX; ++j) {
            if (j < a.Nb) {
                const float sv = Ssum[j * TC_NA + row];
                const float t = sv + acc[j];
                const float bp = t - sv;
                const float e = (sv - (t - bp)) + (acc[j] - bp);
                Ssum[j * TC_NA + row] = t;
                acc[j] = e;
            }
        }
    };

    bool ok = true;      // false once this thread's warp saw a wait run out
    int mma_issued = 0;  // chunks whose MMA chain thread 0 has issued
    for (int kc = 0; kc < nchunks; ++kc) {
        const int s = kc % nst;
        unsigned char* sp = stage_ptr(s);
        float* cHi = reinterpret_cast<float*>(sp);
        float* cLo = reinterpret_cast<float*>(sp + tileC);
        float* xHi = reinterpret_cast<float*>(sp + 2 * tileC);
        float* xLo = reinterpret_cast<float*>(sp + 2 * tileC + tileX);
        const int k0 = (int)(kbeg + (long long)kc * TC_KC);
        if (ok && !mbar_wait(&full[s], (unsigned)(kc / nst) & 1u)) ok = false;
        if (!ok) s_fail = 1;
        else if (tid == 0) landed = kc + 1;
        const long long mc = (a.maskC > n0 && k0 < a.maskC) ? a.maskC : 0;
        const long long mx = (k0 < a.maskX) ? a.maskX : 0;
        if (ok) {
            if (a.split3 || mc) prep_tile(cHi, cLo, TC_NA, k0, n0, mc, a.split3);
            if (a.split3 || mx) prep_tile(xHi, xLo, a.Nb, k0, 0, mx, a.split3);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        fence_before();
        __syncthreads();
        fence_after();
        if (s_fail) break;  // block-uniform: read after the barrier, written only before it
        if (tid == 0) {
            const uint32_t td = tmem + (uint32_t)((kc & 1) * a.Nb);
            int acc_on = 0;
            if (a.split3) {
#pragma unroll
                for (int k = 0; k < TC_KC / 8; ++k) {
                    mma_tf32(td, umma_desc(reinterpret_cast<unsigned char*>(cHi) + k * 32),
                             umma_desc(reinterpret_cast<unsigned char*>(xLo) + k * 32), idesc, acc_on);
                    acc_on = 1;
                    mma_tf32(td, umma_desc(reinterpret_cast<unsigned char*>(cLo) + k * 32),
                             umma_desc(reinterpret_cast<unsigned char*>(xHi) + k * 32), idesc, 1);
                }
            }
#pragma unroll
            for (int k = 0; k < TC_KC / 8; ++k) {
                mma_tf32(td, umma_desc(reinterpret_cast<unsigned char*>(cHi) + k * 32),
                         umma_desc(reinterpret_cast<unsigned char*>(xHi) + k * 32), idesc, acc_on);
                acc_on = 1;
            }
            mma_commit(&empty[s]);
            mma_issued = kc + 1;
        }
        if (kc >= 1) {
            if (!drain(kc - 1)) {
                ok = false;
                s_fail = 1;  // seen by every thread at the next iteration's barrier
            } else {
                if (kc % TC_FOLD == 0) fold();
                // stage (kc - 1) % nst is free again: bring in chunk kc - 1 + nst
                if (tid == 0 && issued < nchunks) issue(issued++);
            }
        }
    }
    if (ok && !s_fail && nchunks > 0 && !drain(nchunks - 1)) ok = false;
    if (!ok) s_fail = 1;
    __syncthreads();
    if (!s_fail && nchunks > 0) {
        fold();
        const long long c = n0 + row;
        double* Pz = P + (long long)blockIdx.y * a.N * a.M;
#pragma unroll
        for (int j = 0; j < NBMAX; ++j)
            if (j < a.M && c < a.N) Pz[c * a.M + j] = (double)Ssum[j * TC_NA + row] + (double)acc[j];
    } else if (s_fail && tid == 0) {
        set_error(st, RQRCP_ERR_TIMEOUT);
        // bounded waits for the copies and MMA chains still in flight
        for (int kc = landed; kc < issued; ++kc) mbar_wait(&full[kc % nst], (unsigned)(kc / nst) & 1u);
        for (int kc = mma_done; kc < mma_issued; ++kc) mbar_wait(&empty[kc % nst], (unsigned)(kc / nst) & 1u);
    }
    fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(a.tmem_cols) : "memory");
}

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (fn == nullptr) {
        cudaDriverEntryPointQueryResult q;
        void* p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            cudaGetLastError();
    }
    return fn;
}

// 2-D FP32 tensor map over a column-major (or row-major, by swapping roles) array with `inner`
// contiguous elements per line, `outer` lines `ld` elements apart; box = 32 x box_outer, 128B swizzle.
bool encode_map(CUtensorMap* map, const float* base, long long inner, long long outer, long long ld, int box_outer)
{
    auto enc = tensor_map_encoder();
    if (enc == nullptr) return false;
    cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)outer};
    cuuint64_t strides[1] = {(cuuint64_t)ld * 4};
    cuuint32_t box[2] = {(cuuint32_t)TC_KC, (cuuint32_t)box_outer};
    cuuint32_t es[2] = {1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

namespace {

size_t tc_smem_bytes(int Nb, int nst)
{
    return 1024 + (size_t)nst * (2 * (size_t)TC_NA * TC_KC * 4 + 2 * (size_t)Nb * TC_KC * 4) +
           (size_t)TC_NA * Nb * sizeof(float);
}

// Dynamic shared memory a kernel may use next to its static shared memory.
template <int NBMAX>
size_t tc_dyn_limit()
{
    static size_t lim = 0;
    if (lim == 0) {
        cudaFuncAttributes fa;
        if (cudaFuncGetAttributes(&fa, (const void*)gemm_tn_tc_kernel<NBMAX>) != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        lim = (size_t)dev_info().max_smem_optin - fa.sharedSizeBytes;
    }
    return lim;
}

size_t tc_dyn_limit_for(int Nb)
{
    return Nb <= 32 ? tc_dyn_limit<32>() : Nb <= 64 ? tc_dyn_limit<64>() : tc_dyn_limit<128>();
}

// Pipeline depth: 4 stages where they fit, else 3 or 2 (0: not even 2 fit).
int tc_stages(int Nb)
{
    const size_t lim = tc_dyn_limit_for(Nb);
    for (int nst = 4; nst >= 2; --nst)
        if (tc_smem_bytes(Nb, nst) <= lim) return nst;
    return 0;
}

}  // namespace

bool tc_gemm_supported(long long M, long long ldx, long long ldc, const void* X, const void* C)
{
    if (!(M >= 1 && M <= 128 && (ldx % 4) == 0 && (ldc % 4) == 0 && ((uintptr_t)X % 16) == 0 &&
          ((uintptr_t)C % 16) == 0 && tensor_map_encoder() != nullptr))
        return false;
    return tc_stages((int)(((M + 15) / 16) * 16)) >= 2;
}

// Split-K chunk for the tensor-core kernel (one resident block per SM): the split count S <= 16
// minimising waves x (rows per split + a pipeline fill of about three chunks), splits of at
// least 256 rows; a multiple of 32.
long long tc_kchunk(long long N, long long K, int& nsplit)
{
    const long long ntiles = (N + TC_NA - 1) / TC_NA;
    const long long sms = dev_info().sms;
    long long smax = (K + 255) / 256;
    if (smax > 16) smax = 16;
    if (smax < 1) smax = 1;
    long long best = 1, best_cost = -1;
    for (long long S = 1; S <= smax; ++S) {
        const long long rows = ((K + S - 1) / S + TC_KC - 1) / TC_KC * TC_KC;
        const long long waves = (ntiles * S + sms - 1) / sms;
        const long long cost = waves * (rows + 3 * TC_KC);
        if (best_cost < 0 || cost < best_cost) {
            best_cost = cost;
            best = S;
        }
    }
    long long kc = (K + best - 1) / best;
    kc = ((kc + TC_KC - 1) / TC_KC) * TC_KC;
    nsplit = (int)((K + kc - 1) / kc);
    return kc;
}

// X given as (matrix base, ld, coordinates of X(0,0)): X(q, r) lives at
// base[(xy0 + r) * ldx + xx0 + q] (each of the M lines holds K contiguous elements), the same
// for C(q, c) at cbase[(cy0 + c) * ldc + cx0 + q].  Extents: X lines xlines, C lines clines,
// inner lengths xinner / cinner (TMA fills zeros beyond the matrices).
cudaError_t launch_gemm_tn_tc(const float* xbase, long long ldx, long long xinner, long long xlines, int xx0, int xy0,
                              const float* cbase, long long ldc, long long cinner, long long clines, int cx0, int cy0,
                              long long M, long long N, long long K, long long kchunk, double* P, long long maskX,
                              long long maskC, int split3, const Status* st, cudaStream_t s)
{
    CUtensorMap mapC, mapX;
    const int Nb = (int)(((M + 15) / 16) * 16);
    const int nst = tc_stages(Nb);
    if (nst < 2) return cudaErrorInvalidValue;
    if (!encode_map(&mapC, cbase, cinner, clines, ldc, TC_NA)) return cudaErrorInvalidValue;
    if (!encode_map(&mapX, xbase, xinner, xlines, ldx, Nb)) return cudaErrorInvalidValue;
    TcArgs a;
    a.M = (int)M;
    a.Nb = Nb;
    a.N = N;
    a.K = K;
    a.kchunk = kchunk;
    a.xx0 = xx0;
    a.xy0 = xy0;
    a.cx0 = cx0;
    a.cy0 = cy0;
    a.maskX = maskX;
    a.maskC = maskC;
    a.split3 = split3;
    a.nst = nst;
    unsigned cols = 32;
    while ((int)cols < 2 * Nb) cols <<= 1;
    a.tmem_cols = cols;
    const size_t smem = tc_smem_bytes(Nb, nst);
    dim3 grid((unsigned)((N + TC_NA - 1) / TC_NA), (unsigned)((K + kchunk - 1) / kchunk));
    auto run = [&](auto kern, bool& attr_set) -> cudaError_t {
        if (!attr_set) {
            if (cudaError_t e = allow_max_dynamic_smem(kern)) return e;
            attr_set = true;
        }
        kern<<<grid, TC_THREADS, smem, s>>>(mapC, mapX, a, P, const_cast<Status*>(st));
        return cudaGetLastError();
    };
    static bool set32 = false, set64 = false, set128 = false;
    if (Nb <= 32) return run(gemm_tn_tc_kernel<32>, set32);
    if (Nb <= 64) return run(gemm_tn_tc_kernel<64>, set64);
    return run(gemm_tn_tc_kernel<128>, set128);
}

}  // namespace rq
