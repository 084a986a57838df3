// update_tc.cu -- tensor-core (tcgen05, kind::tf32) form of the compact-WY trailing update of the
// FP32 form (Alg. 2's block step, the Householder block applied as I - V T V^T):
//   C(mr x nt) -= V(mr x kb) Y(kb x nt),  kb <= KP (64, or 128 for two blocks applied in one pass),
// with Y = T^T W coming from the FP64 reduction.  Both operands are split into TF32 parts
// (x = hi + lo, hi = tf32(x), lo = tf32(x - hi)) and V Y = V_hi [Y_hi Y_lo] + V_lo [Y_hi Y_lo].
//
// A persistent kernel: block b of G owns the contiguous run [b T / G, (b+1) T / G) of the T tiles
// (128 rows x 64 columns of C) in band-major order.  Per 128-row band the workers load V's band,
// split it and store it to tensor memory as the MMA's A operand (hi parts in KP columns, lo parts
// in KP more).  Per tile, a TMA producer warp loads the pre-split Y tile ([Y_hi; Y_lo] as a
// 128-row K-major B operand, 128-byte swizzle) into the Y ring and the C tile (128 rows x 64
// columns, column-major) into the C ring; one thread issues 2 ceil(kb / 8) MMAs (the A_lo products
// first; at KP = 128 the later K first) into one of two accumulators (128 x 128: the Y_hi half,
// then the Y_lo half), which frees the Y stage when they complete; sixteen worker warps read the
// accumulator (tcgen05.ld), subtract it from the C tile in shared memory and hand the tile back
// to the producer, which writes it with a TMA store before reusing the C stage.  Every wait is
// bounded; on timeout the block records RQRCP_ERR_TIMEOUT, lets its copies land and frees its
// tensor memory.
#include "tc_common.cuh"

namespace rq {
namespace {
using namespace tc;

constexpr int UT_WARPS_W = 16;               // worker warps (four per tensor-memory lane quarter)
constexpr int UT_WORKERS = 32 * UT_WARPS_W;
constexpr int UT_THREADS = 64 + UT_WORKERS;  // + TMA producer warp + MMA warp
constexpr int UT_BM = 128;                   // rows of C per band (MMA M)
constexpr int UT_BN = 64;                    // columns of C per tile (MMA N = 2 UT_BN)
constexpr int UT_KSUB = 2 * UT_BN * 128;     // bytes of one 32-long K slice of the Y tile (128 lines)
constexpr int UT_TILE_C = UT_BM * UT_BN * 4;      // 32 KB: [column][row]
constexpr unsigned UT_TMEM_COLS = 512;  // D0 (0..127), D1 (128..255), A hi (256..256+KP-1), A lo (256+KP..)

// KP: contraction length padded (kb <= KP); Y tile (KP / 32 slices of 128 lines x 128 bytes); the
// Y tiles and the C tiles go through rings of their own (a Y stage is free once the tile's MMAs
// complete, a C stage only after the drain and the store): NY Y stages, NC C stages.  At KP = 128
// two 64 KB Y stages and three C stages fit where three whole stages would not.
template <int KP> struct UtCfg {
    static constexpr int NY = KP == 64 ? 3 : 2;
    static constexpr int NC = 3;
    static constexpr int TILE_Y = 2 * UT_BN * KP * 4;
    static constexpr int SMEM = NY * TILE_Y + NC * UT_TILE_C;
};

// Y (kb x nt FP64: row k < kb1 of column c at Y[c * ldy + k], row k >= kb1 at Y2[c * ldy2 + k - kb1])
// -> ys: for tile t = c / 64, j = c % 64, line t * 128 + j holds tf32(y(:, c)) and line
// t * 128 + 64 + j holds tf32(y - tf32(y)), KP values per line (zero for k >= kb and for c >= nt).
template <int KP>
__global__ void ysplit_kernel(const double* __restrict__ Y, long long ldy, const double* __restrict__ Y2,
                              long long ldy2, int kb1, int kb, long long nt, long long ntiles, float* __restrict__ ys,
                              const Status* st)
{
    if (status_error(st)) return;
    const long long total = ntiles * UT_BN * KP;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(e % KP);
        const long long c = e / KP;
        const long long t = c / UT_BN;
        const int j = (int)(c % UT_BN);
        float h = 0.f, l = 0.f;
        if (c < nt && k < kb) {
            const double y = k < kb1 ? Y[c * ldy + k] : Y2[c * ldy2 + (k - kb1)];
            h = tf32_rn((float)y);
            l = tf32_rn((float)(y - (double)h));
        }
        ys[(t * 2 * UT_BN + j) * KP + k] = h;
        ys[(t * 2 * UT_BN + UT_BN + j) * KP + k] = l;
    }
}

struct UtArgs {
    long long mr, nt;      // rows and columns of C
    int kb, ksteps;        // contraction length (<= KP), MMA k-steps ceil(kb / 8)
    long long maskV;       // rows r < maskV of V's columns j >= maskC0 carry the unit-lower structure
    int maskC0;            // (relative to column maskC0: V(r, j) = 0 for r < j - maskC0, 1 for r == j - maskC0)
    long long ntiles;      // 64-column tiles per band
    long long total;       // bands * ntiles
};

template <int KP>
__global__ void __launch_bounds__(UT_THREADS, 1)
    update_tc_kernel(const __grid_constant__ CUtensorMap mapC, const __grid_constant__ CUtensorMap mapY,
                     const float* __restrict__ V, long long ldv, UtArgs a, Status* st)
{
    constexpr int NY = UtCfg<KP>::NY, NC = UtCfg<KP>::NC;
    constexpr int UT_TILE_Y = UtCfg<KP>::TILE_Y;
    __shared__ int s_skip;
    if (threadIdx.x == 0) s_skip = status_error(st);
    __syncthreads();
    if (s_skip) return;  // block-uniform: warp 1's tensor-memory allocation is warp-collective
    extern __shared__ unsigned char smraw[];
    unsigned char* base = reinterpret_cast<unsigned char*>(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t fullY[NY], freeY[NY], fullC[NC], cdone[NC], aready, accfull[2], accempty[2];
    __shared__ uint32_t tmem_base;
    __shared__ volatile int s_fail;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp == 1) tmem_alloc(&tmem_base, UT_TMEM_COLS);
    if (tid == 0) {
        for (int s = 0; s < NY; ++s) {
            mbar_init(&fullY[s], 1);
            mbar_init(&freeY[s], 1);
        }
        for (int s = 0; s < NC; ++s) {
            mbar_init(&fullC[s], 1);
            mbar_init(&cdone[s], UT_WARPS_W);
        }
        mbar_init(&aready, UT_WARPS_W);
        for (int b = 0; b < 2; ++b) {
            mbar_init(&accfull[b], 1);
            mbar_init(&accempty[b], UT_WARPS_W);
        }
        s_fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = tmem_base;
    const uint32_t tA = tmem + 256;
    const long long g0 = a.total * blockIdx.x / gridDim.x;
    const long long g1 = a.total * (blockIdx.x + 1) / gridDim.x;
    auto ystage = [&](int s) { return base + (size_t)s * UT_TILE_Y; };
    auto cstage = [&](int s) { return base + (size_t)NY * UT_TILE_Y + (size_t)s * UT_TILE_C; };
    auto fail = [&]() {
        s_fail = 1;
        set_error(st, RQRCP_ERR_TIMEOUT);
    };

    if (warp == 0) {
        if (lane == 0) {
            int px[NC], py[NC];  // C coordinates of the tile held by each C stage
            long long t = 0;
            bool ok = true;
            for (long long g = g0; g < g1; ++g, ++t) {
                const int sy = (int)(t % NY), sc = (int)(t % NC);
                if (t >= NC) {
                    // the C stage's previous tile is finished: store it, and reuse the stage once the
                    // store has read it
                    if (!mbar_wait(&cdone[sc], (unsigned)((t - NC) / NC) & 1u, &s_fail)) {
                        fail();
                        ok = false;
                        break;
                    }
                    tma_store_2d(&mapC, px[sc], py[sc], cstage(sc));
                    bulk_commit();
                    bulk_wait_read();
                }
                // the Y stage is free once the MMAs of its previous tile have completed
                if (t >= NY && !mbar_wait(&freeY[sy], (unsigned)((t - NY) / NY) & 1u, &s_fail)) {
                    fail();
                    ok = false;
                    break;
                }
                const long long band = g / a.ntiles, ct = g % a.ntiles;
                px[sc] = (int)(band * UT_BM);
                py[sc] = (int)(ct * UT_BN);
                mbar_expect_tx(&fullY[sy], UT_TILE_Y);
#pragma unroll
                for (int u = 0; u < KP / 32; ++u)
                    tma_load_2d(ystage(sy) + u * UT_KSUB, &mapY, 32 * u, (int)(ct * 2 * UT_BN), &fullY[sy]);
                mbar_expect_tx(&fullC[sc], UT_TILE_C);
                tma_load_2d(cstage(sc), &mapC, px[sc], py[sc], &fullC[sc]);
            }
            if (ok) {
                for (long long u = (t > NC ? t - NC : 0); u < t; ++u) {
                    const int sc = (int)(u % NC);
                    if (!mbar_wait(&cdone[sc], (unsigned)(u / NC) & 1u, &s_fail)) {
                        fail();
                        ok = false;
                        break;
                    }
                    tma_store_2d(&mapC, px[sc], py[sc], cstage(sc));
                    bulk_commit();
                }
            }
            bulk_wait_all();
            if (!ok) {  // loads still in flight land before the block leaves (bounded)
                for (long long u = (t > NY ? t - NY : 0); u < t; ++u)
                    mbar_wait(&fullY[u % NY], (unsigned)(u / NY) & 1u, nullptr);
                for (long long u = (t > NC ? t - NC : 0); u < t; ++u)
                    mbar_wait(&fullC[u % NC], (unsigned)(u / NC) & 1u, nullptr);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = idesc_tf32(UT_BM, 2 * UT_BN);
            long long t = 0, run = 0, prev_band = -1, issued = 0;
            for (long long g = g0; g < g1; ++g, ++t) {
                const long long band = g / a.ntiles;
                if (band != prev_band) {
                    if (!mbar_wait(&aready, (unsigned)(run & 1), &s_fail)) {
                        fail();
                        break;
                    }
                    ++run;
                    prev_band = band;
                }
                const int sy = (int)(t % NY), b = (int)(t & 1);
                if (!mbar_wait(&fullY[sy], (unsigned)(t / NY) & 1u, &s_fail) ||
                    (t >= 2 && !mbar_wait(&accempty[b], (unsigned)((t - 2) >> 1) & 1u, &s_fail))) {
                    fail();
                    break;
                }
                fence_after();
                const unsigned char* yt = ystage(sy);
                const uint32_t td = tmem + (uint32_t)(b * 2 * UT_BN);
                // K = 128 (two blocks): the second block's k-steps first.  Its products are of the size
                // of the trailing matrix after the first block's update, which can be far smaller than
                // the first block's; accumulated first, they are not rounded against the large sum.
                for (int kx = 0; kx < a.ksteps; ++kx) {
                    const int kk = KP == 128 ? a.ksteps - 1 - kx : kx;
                    mma_tf32_ts(td, tA + KP + 8 * kk, umma_desc(yt + (kk >> 2) * UT_KSUB + (kk & 3) * 32), idesc,
                                kx > 0 ? 1 : 0);
                }
                for (int kx = 0; kx < a.ksteps; ++kx) {
                    const int kk = KP == 128 ? a.ksteps - 1 - kx : kx;
                    mma_tf32_ts(td, tA + 8 * kk, umma_desc(yt + (kk >> 2) * UT_KSUB + (kk & 3) * 32), idesc, 1);
                }
                mma_commit(&freeY[sy]);
                mma_commit(&accfull[b]);
                issued = t + 1;
            }
            // every MMA chain completes before tensor memory is freed (bounded)
            if (issued > 0)
                mbar_wait(&accfull[(issued - 1) & 1], (unsigned)(((issued - 1) >> 1) & 1), nullptr);
        }
    } else {
        const int q = warp & 3;         // tensor-memory lane quarter
        const int h = (warp - 2) >> 2;  // 16-column quarter of the tile (and of V's 64 columns)
        const int row = 32 * q + lane;  // row within the band
        const uint32_t lane_base = (uint32_t)(32 * q) << 16;
        long long t = 0, prev_band = -1;
        bool ok = true;
        for (long long g = g0; g < g1; ++g, ++t) {
            const long long band = g / a.ntiles;
            if (band != prev_band) {
                // A <- V's band: row band * 128 + row, columns 16h + 64p .. 16h + 64p + 15 (every MMA
                // of the previous band has completed: this thread drained its last accumulator)
                const long long r = band * UT_BM + row;
#pragma unroll
                for (int part = 0; part < KP / 64; ++part) {
                    uint32_t hi[16], lo[16];
#pragma unroll
                    for (int u = 0; u < 16; ++u) {
                        const int j = 16 * h + 64 * part + u;
                        float v = 0.f;
                        if (r < a.mr && j < a.kb) {
                            v = V[(long long)j * ldv + r];
                            const int jm = j - a.maskC0;
                            if (r < a.maskV && jm >= 0) {
                                if (r < jm) v = 0.f;
                                else if (r == jm) v = 1.f;
                            }
                        }
                        const float hv = tf32_rn(v);
                        hi[u] = __float_as_uint(hv);
                        lo[u] = __float_as_uint(tf32_rn(v - hv));
                    }
                    const uint32_t ta = tA + lane_base + (uint32_t)(16 * h + 64 * part);
                    asm volatile(
                        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(
                            ta),
                        "r"(hi[0]), "r"(hi[1]), "r"(hi[2]), "r"(hi[3]), "r"(hi[4]), "r"(hi[5]), "r"(hi[6]), "r"(hi[7]),
                        "r"(hi[8]), "r"(hi[9]), "r"(hi[10]), "r"(hi[11]), "r"(hi[12]), "r"(hi[13]), "r"(hi[14]),
                        "r"(hi[15])
                        : "memory");
                    asm volatile(
                        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(
                            ta + KP),
                        "r"(lo[0]), "r"(lo[1]), "r"(lo[2]), "r"(lo[3]), "r"(lo[4]), "r"(lo[5]), "r"(lo[6]), "r"(lo[7]),
                        "r"(lo[8]), "r"(lo[9]), "r"(lo[10]), "r"(lo[11]), "r"(lo[12]), "r"(lo[13]), "r"(lo[14]),
                        "r"(lo[15])
                        : "memory");
                }
                asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
                fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&aready);
                prev_band = band;
            }
            const int sc = (int)(t % NC), b = (int)(t & 1);
            bool okw = mbar_wait(&accfull[b], (unsigned)(t >> 1) & 1u, &s_fail);
            okw = okw && mbar_wait(&fullC[sc], (unsigned)(t / NC) & 1u, &s_fail);  // C tile visible here
            if (!__all_sync(0xffffffffu, okw)) {
                ok = false;
                break;
            }
            fence_after();
            uint32_t rh[16], rl[16];
            const uint32_t td = tmem + lane_base + (uint32_t)(b * 2 * UT_BN + 16 * h);
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                : "=r"(rh[0]), "=r"(rh[1]), "=r"(rh[2]), "=r"(rh[3]), "=r"(rh[4]), "=r"(rh[5]), "=r"(rh[6]), "=r"(rh[7]),
                  "=r"(rh[8]), "=r"(rh[9]), "=r"(rh[10]), "=r"(rh[11]), "=r"(rh[12]), "=r"(rh[13]), "=r"(rh[14]),
                  "=r"(rh[15])
                : "r"(td));
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                : "=r"(rl[0]), "=r"(rl[1]), "=r"(rl[2]), "=r"(rl[3]), "=r"(rl[4]), "=r"(rl[5]), "=r"(rl[6]), "=r"(rl[7]),
                  "=r"(rl[8]), "=r"(rl[9]), "=r"(rl[10]), "=r"(rl[11]), "=r"(rl[12]), "=r"(rl[13]), "=r"(rl[14]),
                  "=r"(rl[15])
                : "r"(td + UT_BN));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&accempty[b]);
            float* ctile = reinterpret_cast<float*>(cstage(sc));
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                float* x = ctile + (16 * h + u) * UT_BM + row;
                *x = *x - (__uint_as_float(rl[u]) + __uint_as_float(rh[u]));
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(&cdone[sc]);
        }
        if (!ok) fail();
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 1) tmem_dealloc(tmem, UT_TMEM_COLS);
}

template <int KP>
size_t ut_smem_bytes()
{
    return 1024 + (size_t)UtCfg<KP>::SMEM;
}

template <int KP>
bool ut_fits()
{
    static int fits = -1;
    if (fits < 0) {
        cudaFuncAttributes fa;
        if (cudaFuncGetAttributes(&fa, (const void*)update_tc_kernel<KP>) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        fits = ut_smem_bytes<KP>() + fa.sharedSizeBytes <= (size_t)dev_info().max_smem_optin ? 1 : 0;
    }
    return fits == 1;
}

// C -= V [Y; Y2] with rows 0..kb1-1 of the contraction from Y and kb1..kb-1 from Y2 (Y2 may be null
// when kb1 == kb).
template <int KP>
cudaError_t launch_update_tc_impl(float* C, long long ldc, const float* V, long long ldv, const double* Y,
                                  long long ldy, const double* Y2, long long ldy2, int kb1, long long mr, long long nt,
                                  int kb, long long maskV, int maskC0, float* ys, const Status* st, cudaStream_t s)
{
    if (mr <= 0 || nt <= 0) return cudaSuccess;
    if (((uintptr_t)ys % 16) != 0 || kb < 1 || kb > KP || kb1 < 0 || kb1 > kb || (kb1 < kb && Y2 == nullptr))
        return cudaErrorInvalidValue;
    const long long ntiles = (nt + UT_BN - 1) / UT_BN;
    {
        const long long total = ntiles * UT_BN * KP;
        long long blocks = (total + 255) / 256;
        if (blocks > 4L * dev_info().sms) blocks = 4L * dev_info().sms;
        ysplit_kernel<KP><<<(unsigned)blocks, 256, 0, s>>>(Y, ldy, Y2, ldy2, kb1, kb, nt, ntiles, ys, st);
        if (cudaError_t e = cudaGetLastError()) return e;
    }
    CUtensorMap mapC, mapY;
    if (!tc_encode_2d(&mapC, C, mr, nt, ldc, UT_BM, UT_BN, false)) return cudaErrorInvalidValue;
    if (!tc_encode_2d(&mapY, ys, KP, ntiles * 2 * UT_BN, KP, 32, 2 * UT_BN, true)) return cudaErrorInvalidValue;
    UtArgs a;
    a.mr = mr;
    a.nt = nt;
    a.kb = kb;
    a.ksteps = (kb + 7) / 8;
    a.maskV = maskV;
    a.maskC0 = maskC0;
    a.ntiles = ntiles;
    a.total = ((mr + UT_BM - 1) / UT_BM) * ntiles;
    static DevFlag attr_set;
    if (!attr_set.done()) {
        if (cudaError_t e = allow_max_dynamic_smem(update_tc_kernel<KP>)) return e;
        attr_set.set();
    }
    long long grid = dev_info().sms;
    if (grid > a.total) grid = a.total;
    update_tc_kernel<KP><<<(unsigned)grid, UT_THREADS, ut_smem_bytes<KP>(), s>>>(mapC, mapY, V, ldv, a,
                                                                               const_cast<Status*>(st));
    return cudaGetLastError();
}

}  // namespace

bool tc_update_supported(long long kb, long long ldc, const void* C)
{
    if (!(kb >= 1 && kb <= 64 && (ldc % 4) == 0 && ((uintptr_t)C % 16) == 0 && tc_encoder_available())) return false;
    return ut_fits<64>();
}

bool tc_update2_supported(long long ldc, const void* C)
{
    if (!((ldc % 4) == 0 && ((uintptr_t)C % 16) == 0 && tc_encoder_available())) return false;
    return ut_fits<128>();
}

size_t tc_update_ws_bytes(long long nt, int kp)
{
    return (size_t)((nt + UT_BN - 1) / UT_BN) * 2 * UT_BN * (size_t)kp * sizeof(float);
}

cudaError_t launch_gemm_update_tc(float* C, long long ldc, const float* V, long long ldv, const double* Y, long long ldy,
                                  long long mr, long long nt, int kb, long long maskV, float* ys, const Status* st,
                                  cudaStream_t s)
{
    return launch_update_tc_impl<64>(C, ldc, V, ldv, Y, ldy, nullptr, 0, kb, mr, nt, kb, maskV, 0, ys, st, s);
}

cudaError_t launch_gemm_update_tc2(float* C, long long ldc, const float* V, long long ldv, const double* Y,
                                   long long ldy, const double* Y2, long long ldy2, int kb1, long long mr, long long nt,
                                   int kb, long long maskV, int maskC0, float* ys, const Status* st, cudaStream_t s)
{
    return launch_update_tc_impl<128>(C, ldc, V, ldv, Y, ldy, Y2, ldy2, kb1, mr, nt, kb, maskV, maskC0, ys, st, s);
}

}  // namespace rq
