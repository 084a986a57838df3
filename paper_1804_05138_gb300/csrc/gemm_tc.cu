// gemm_tc.cu -- tensor-core (tcgen05, kind::tf32) form of the split-K contraction
//   P[sp][c][r] = sum_{q in split sp} X(q, r) C(q, c),  r < M <= 96, c < N,
// for the FP32 form: the sketch B = Omega A (X = Omega^T) and W = V^T [V C] of the compact-WY
// update (X = V).  Each operand is split x = hi + lo with hi = tf32(x), lo = tf32(x - hi) (exact to
// about 2^-23 |x|), and x y = hi hi' + hi lo' + lo hi' + lo lo' on the TF32 tensor cores.
//
// One block (a TMA producer warp, an MMA warp and sixteen worker warps) computes 128 columns of C
// against all M rows of X over one K split.  X is split into TF32 hi/lo parts once per launch
// (xsplit_kernel) and used as one B operand of N = 2 Nb rows, [X_hi; X_lo]; C chunks of 32 rows
// arrive raw by TMA (cp.async.bulk.tensor, 128-byte swizzle) into a ring of stages.  The workers
// split each C chunk into TF32 hi/lo parts and store them as the MMA's A operand in tensor memory
// (tcgen05.st), so the tensor core reads only X from shared memory; one thread issues the chunk's
// eight tcgen05.mma (A_lo and A_hi against [X_hi; X_lo], the four products hi hi', hi lo', lo hi',
// lo lo' in two accumulator halves).  The accumulation over K happens outside the tensor core:
// each chunk's product is read back (tcgen05.ld) and summed in FP32 registers with
// round-to-nearest, folded into a compensated sum every TC_FOLD chunks, so the tensor core's own
// accumulator only ever adds the eight products of one chunk.  The epilogue
// writes the FP64 partials.  Every wait is bounded; on timeout the block records
// RQRCP_ERR_TIMEOUT, waits (bounded) for its copies and MMA chains in flight and frees its
// tensor memory.
#include "tc_common.cuh"

namespace rq {
namespace {

constexpr int TC_WARPS_W = 16;                // worker warps (four per tensor-memory lane quarter)
constexpr int TC_WORKERS = 32 * TC_WARPS_W;
constexpr int TC_THREADS = 64 + TC_WORKERS;   // + TMA producer warp + MMA warp
constexpr int TC_KC = 32;       // K per stage: one 128-byte swizzle row of FP32
constexpr int TC_NA = 128;      // columns of C per block (MMA M)
constexpr int TC_MAXST = 8;
constexpr int TC_FOLD = 16;     // chunks summed in FP32 registers between compensated folds
using namespace tc;

// X(q, r) (q < K, r < M, line r at X + r * ldx; unit-lower reflector structure for r < maskX) ->
// TF32 parts xh[r * ldk + q] = tf32(x), xl[r * ldk + q] = tf32(x - tf32(x)); lines M <= r < gridDim.y
// are zero.  One grid row per line r.
__global__ void xsplit_kernel(const float* __restrict__ X, long long ldx, long long K, int M, long long maskX,
                              long long ldk, float* __restrict__ xh, float* __restrict__ xl, const Status* st)
{
    if (status_error(st)) return;
    const long long r = blockIdx.y;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < K; q += (long long)gridDim.x * blockDim.x) {
        float v = r < M ? X[r * ldx + q] : 0.f;
        if (r < maskX) {
            if (q < r) v = 0.f;
            else if (q == r) v = 1.f;
        }
        const float h = tf32_rn(v);
        xh[r * ldk + q] = h;
        xl[r * ldk + q] = tf32_rn(v - h);
    }
}

// BF16 form of xsplit_kernel: xb[r * ldk + q] = bf16(x) (round to nearest even); lines M <= r <
// gridDim.y are zero.
__global__ void xsplit_bf16_kernel(const float* __restrict__ X, long long ldx, long long K, int M, long long ldk,
                                   __nv_bfloat16* __restrict__ xb, const Status* st)
{
    if (status_error(st)) return;
    const long long r = blockIdx.y;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < K; q += (long long)gridDim.x * blockDim.x)
        xb[r * ldk + q] = __float2bfloat16_rn(r < M ? X[r * ldx + q] : 0.f);
}

struct TcArgs {
    int M, Nb;               // rows of X used (<= Nb), MMA N (multiple of 16)
    long long N, K;          // columns of C, contraction length
    long long kchunk;        // K per split (multiple of TC_KC)
    long long maskC;         // C columns maskC0 <= c < maskC0 + maskC carry the reflector mask
    long long maskC0;        // (relative to column maskC0)
    int nst;                 // pipeline stages (2..TC_MAXST)
    unsigned tmem_cols;
};

// Per block: 128 columns of C x all Nb rows of X over one K split, by three warp roles that hand
// work to each other through mbarriers (no block-wide barrier inside the K loop).  Tensor memory
// holds two accumulator buffers D0, D1 (2 Nb columns each: products with X_hi, then with X_lo)
// and two operand buffers A0, A1 (64 columns: the TF32 hi parts of a 32-row chunk of C^T, then
// its lo parts).
//   warp 0 (one lane)  TMA producer: raw C chunk + the pre-split [X_hi; X_lo] chunk -> stage
//                      kc % nst once the stage's previous MMA chain has completed (empty[s]).
//   warps 2..17        workers (four per tensor-memory lane quarter, each on 8 of the chunk's 32
//                      rows): read their C column's 8 values from the landed stage, apply the
//                      reflector mask, split into TF32 hi/lo and store them to A[kc % 2] with
//                      tcgen05.st (aready); then drain chunk kc-1's accumulator: tcgen05.ld of
//                      their row and column quarter in both halves, FP32 round-to-nearest add
//                      into registers (accempty).  Every TC_FOLD chunks a compensated fold (TwoSum, error carried
//                      back) into a second register set.  A[kc % 2] is free again once chunk kc-2's
//                      accumulator has been drained, which the worker itself waited for.
//   warp 1 (one lane)  MMA issuer: D[kc % 2] = A_lo [X_hi; X_lo] + A_hi [X_hi; X_lo] over the
//                      chunk (the small A_lo products first, so the accumulator of the large terms
//                      rounds only the four hi*hi steps) once aready and accempty allow; commits to
//                      empty[s] and accfull[kc % 2].
//
// BF16 form (the sketch): 64-row chunks (two 32-row C boxes), A = the chunk rounded to BF16 (pairs
// of rows packed per 32-bit tensor-memory column, 32 columns per buffer), X pre-rounded to BF16
// (one Nb-row operand, 64 K per 128-byte row), four kind::f16 MMAs per chunk into an Nb-column
// accumulator; no reflector mask.
template <int NBMAX, bool BF>
__global__ void __launch_bounds__(TC_THREADS, 1)
    gemm_tn_tc_kernel(const __grid_constant__ CUtensorMap mapC, const __grid_constant__ CUtensorMap mapX, TcArgs a,
                      double* __restrict__ P, Status* st)
{
    constexpr int CQ = NBMAX / 4;          // register columns per worker (a quarter of the MMA N)
    constexpr int KC = BF ? 64 : TC_KC;    // rows of C per chunk
    constexpr int ACOLS = BF ? 32 : 64;    // tensor-memory columns of one A buffer
    __shared__ int s_skip;
    if (threadIdx.x == 0) s_skip = status_error(st);
    __syncthreads();
    if (s_skip) return;  // block-uniform: warp 1's tensor-memory allocation is warp-collective
    extern __shared__ unsigned char smraw[];
    unsigned char* base = reinterpret_cast<unsigned char*>(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
    const int tileC = TC_NA * KC * 4;                      // raw FP32 C chunk (16 or 32 KB)
    const int tileX = (BF ? a.Nb : 2 * a.Nb) * 128;        // BF16 X, or [X_hi; X_lo]: rows of 128 bytes
    const int dcols = BF ? a.Nb : 2 * a.Nb;                // MMA N = accumulator columns
    const int stage_bytes = tileC + tileX;
    const int nst = a.nst;
    __shared__ __align__(8) uint64_t full[TC_MAXST], empty[TC_MAXST], aready[2], accfull[2], accempty[2];
    __shared__ uint32_t tmem_base;
    __shared__ volatile int s_fail;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp == 1) {
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
        for (int b = 0; b < 2; ++b) {
            mbar_init(&aready[b], TC_WARPS_W);
            mbar_init(&accfull[b], 1);
            mbar_init(&accempty[b], TC_WARPS_W);
        }
        s_fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = tmem_base;
    const uint32_t tA = tmem + (uint32_t)(2 * dcols);  // D0, D1 (dcols each), then A0, A1 (ACOLS each)
    const long long n0 = (long long)blockIdx.x * TC_NA;
    const long long kbeg = (long long)blockIdx.y * a.kchunk;
    const long long kend = min(a.K, kbeg + a.kchunk);
    const int nchunks = (int)((kend - kbeg + KC - 1) / KC);
    auto stage_ptr = [&](int s) { return base + (size_t)s * stage_bytes; };
    auto fail = [&]() {
        s_fail = 1;
        set_error(st, RQRCP_ERR_TIMEOUT);
    };

    if (warp == 0) {
        if (lane == 0) {
            int issued = 0;
            for (int kc = 0; kc < nchunks; ++kc) {
                const int s = kc % nst;
                if (kc >= nst && !mbar_wait(&empty[s], (unsigned)((kc - nst) / nst) & 1u, &s_fail)) {
                    fail();
                    break;
                }
                unsigned char* sp = stage_ptr(s);
                const int k0 = (int)(kbeg + (long long)kc * KC);
                mbar_expect_tx(&full[s], tileC + tileX);
                tma_load_2d(sp, &mapC, k0, (int)n0, &full[s]);
                if (BF) tma_load_2d(sp + tileC / 2, &mapC, k0 + 32, (int)n0, &full[s]);
                tma_load_2d(sp + tileC, &mapX, k0, 0, &full[s]);
                issued = kc + 1;
            }
            // the copies still in flight land before the block leaves (bounded)
            for (int kc = (issued > nst ? issued - nst : 0); kc < issued; ++kc)
                mbar_wait(&full[kc % nst], (unsigned)(kc / nst) & 1u, nullptr);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = BF ? idesc_bf16(TC_NA, a.Nb) : idesc_tf32(TC_NA, 2 * a.Nb);
            int issued = 0;
            for (int kc = 0; kc < nchunks; ++kc) {
                const int s = kc % nst, b = kc & 1;
                if (!mbar_wait(&aready[b], (unsigned)(kc >> 1) & 1u, &s_fail) ||
                    (kc >= 2 && !mbar_wait(&accempty[b], (unsigned)((kc - 2) >> 1) & 1u, &s_fail))) {
                    fail();
                    break;
                }
                fence_after();
                const unsigned char* xt = stage_ptr(s) + tileC;
                const uint32_t td = tmem + (uint32_t)(b * dcols);
                const uint32_t ta = tA + (uint32_t)(b * ACOLS);
                // k-step k starts 32 bytes further into the 128-byte swizzle rows: the descriptor's
                // address field (bytes >> 4, 14 bits, tile below 256 KB) advances by 2 without carry
                const uint64_t dx = umma_desc(xt);
                if (BF) {
#pragma unroll
                    for (int k = 0; k < 4; ++k) mma_bf16_ts(td, ta + 8 * k, dx + 2 * k, idesc, k > 0 ? 1 : 0);
                } else {
#pragma unroll
                    for (int k = 0; k < TC_KC / 8; ++k) mma_tf32_ts(td, ta + 32 + 8 * k, dx + 2 * k, idesc, k > 0 ? 1 : 0);
#pragma unroll
                    for (int k = 0; k < TC_KC / 8; ++k) mma_tf32_ts(td, ta + 8 * k, dx + 2 * k, idesc, 1);
                }
                mma_commit(&empty[s]);
                mma_commit(&accfull[b]);
                issued = kc + 1;
            }
            // every MMA chain completes before tensor memory is freed (bounded)
            if (issued > 0) mbar_wait(&empty[(issued - 1) % nst], (unsigned)((issued - 1) / nst) & 1u, nullptr);
        }
    } else {
        const int q = warp & 3;             // tensor-memory lane quarter this warp may access
        const int h = (warp - 2) >> 2;      // column quarter (drain) and 8-row slice (operand store)
        const int qc = a.Nb >> 2;           // accumulator columns per worker warp (multiple of 4)
        const int cb = h * qc;
        const int row = 32 * q + lane;      // row of D / A = column n0 + row of C
        const uint32_t lane_base = (uint32_t)(32 * q) << 16;
        const long long c = n0 + row;
        float acc[CQ], sum[CQ];
#pragma unroll
        for (int j = 0; j < CQ; ++j) acc[j] = sum[j] = 0.f;
        auto drain = [&](int kc) -> bool {
            const bool ok = mbar_wait(&accfull[kc & 1], (unsigned)(kc >> 1) & 1u, &s_fail);
            if (!__all_sync(0xffffffffu, ok)) return false;
            fence_after();
            // column j of this quarter: X_hi product at tb + j, X_lo product at tb + Nb + j (BF16:
            // the one product at tb + j); groups of up to 8 columns: all loads in flight, one wait
            const uint32_t tb = tmem + lane_base + (uint32_t)((kc & 1) * dcols + cb);
#pragma unroll
            for (int g0 = 0; g0 < CQ; g0 += 8) {
                if (g0 < qc) {
                    uint32_t rh[8], rl[8];
#pragma unroll
                    for (int c0 = 0; c0 < 8 && g0 + c0 < CQ; c0 += 4) {
                        if (g0 + c0 < qc) {
                            asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                                         : "=r"(rh[c0]), "=r"(rh[c0 + 1]), "=r"(rh[c0 + 2]), "=r"(rh[c0 + 3])
                                         : "r"(tb + (uint32_t)(g0 + c0)));
                            if (!BF)
                                asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                                             : "=r"(rl[c0]), "=r"(rl[c0 + 1]), "=r"(rl[c0 + 2]), "=r"(rl[c0 + 3])
                                             : "r"(tb + (uint32_t)(a.Nb + g0 + c0)));
                        }
                    }
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                    for (int c0 = 0; c0 < 8 && g0 + c0 < CQ; c0 += 4) {
                        if (g0 + c0 < qc) {
#pragma unroll
                            for (int u = 0; u < 4; ++u)
                                acc[g0 + c0 + u] += BF ? __uint_as_float(rh[c0 + u])
                                                       : __uint_as_float(rl[c0 + u]) + __uint_as_float(rh[c0 + u]);
                        }
                    }
                }
            }
            fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&accempty[kc & 1]);
            return true;
        };
        // compensated fold: (sum, e) = TwoSum(sum, acc), acc = e
        auto fold = [&]() {
#pragma unroll
            for (int j = 0; j < CQ; ++j) {
                const float t = sum[j] + acc[j];
                const float bp = t - sum[j];
                const float e = (sum[j] - (t - bp)) + (acc[j] - bp);
                sum[j] = t;
                acc[j] = e;
            }
        };
        bool ok = true;
        for (int kc = 0; kc < nchunks; ++kc) {
            const int s = kc % nst;
            if (!__all_sync(0xffffffffu, mbar_wait(&full[s], (unsigned)(kc / nst) & 1u, &s_fail))) {
                ok = false;
                break;
            }
            const unsigned char* tile = stage_ptr(s);
            const int k0 = (int)(kbeg + (long long)kc * KC);
            if (BF) {
                // rows 16h .. 16h + 15 of the chunk for column c: box h / 2, four swizzled 16-byte
                // pieces of its row `row`; packed as BF16 pairs (even row in the low half)
                const unsigned char* box = tile + (h >> 1) * (tileC / 2) + row * 128;
                uint32_t pk[8];
#pragma unroll
                for (int pc = 0; pc < 4; ++pc) {
                    const int piece = (4 * (h & 1) + pc) ^ (row & 7);
                    const float4 f = *reinterpret_cast<const float4*>(box + piece * 16);
                    const __nv_bfloat162 p0 = __floats2bfloat162_rn(f.x, f.y);
                    const __nv_bfloat162 p1 = __floats2bfloat162_rn(f.z, f.w);
                    pk[2 * pc] = *reinterpret_cast<const uint32_t*>(&p0);
                    pk[2 * pc + 1] = *reinterpret_cast<const uint32_t*>(&p1);
                }
                const uint32_t ta = tA + lane_base + (uint32_t)((kc & 1) * ACOLS + 8 * h);
                asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(ta),
                             "r"(pk[0]), "r"(pk[1]), "r"(pk[2]), "r"(pk[3]), "r"(pk[4]), "r"(pk[5]), "r"(pk[6]),
                             "r"(pk[7])
                             : "memory");
            } else {
                // this thread's 8 values: rows k0 + 8h .. k0 + 8h + 7 of column c, two swizzled
                // 16-byte pieces of the tile's row `row`
                float v[8];
#pragma unroll
                for (int pc = 0; pc < 2; ++pc) {
                    const int piece = (2 * h + pc) ^ (row & 7);
                    const float4 f = *reinterpret_cast<const float4*>(tile + row * 128 + piece * 16);
                    v[4 * pc] = f.x;
                    v[4 * pc + 1] = f.y;
                    v[4 * pc + 2] = f.z;
                    v[4 * pc + 3] = f.w;
                }
                if (c - a.maskC0 >= 0 && c - a.maskC0 < a.maskC && k0 < a.maskC) {
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const long long qq = (long long)k0 + 8 * h + u;
                        if (qq < c - a.maskC0) v[u] = 0.f;
                        else if (qq == c - a.maskC0) v[u] = 1.f;
                    }
                }
                uint32_t hi[8], lo[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const float hv = tf32_rn(v[u]);
                    hi[u] = __float_as_uint(hv);
                    lo[u] = __float_as_uint(tf32_rn(v[u] - hv));
                }
                const uint32_t ta = tA + lane_base + (uint32_t)((kc & 1) * ACOLS + 8 * h);
                asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(ta),
                             "r"(hi[0]), "r"(hi[1]), "r"(hi[2]), "r"(hi[3]), "r"(hi[4]), "r"(hi[5]), "r"(hi[6]),
                             "r"(hi[7])
                             : "memory");
                asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(ta + 32),
                             "r"(lo[0]), "r"(lo[1]), "r"(lo[2]), "r"(lo[3]), "r"(lo[4]), "r"(lo[5]), "r"(lo[6]),
                             "r"(lo[7])
                             : "memory");
            }
            asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
            fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&aready[kc & 1]);
            if (kc >= 1) {
                if (!drain(kc - 1)) {
                    ok = false;
                    break;
                }
                if (kc % TC_FOLD == 0) fold();
            }
        }
        if (ok && nchunks > 0 && !drain(nchunks - 1)) ok = false;
        if (!ok) {
            fail();
        } else if (nchunks > 0) {
            fold();
            double* Pz = P + (long long)blockIdx.y * a.N * a.M;
            if (c < a.N) {
#pragma unroll
                for (int j = 0; j < CQ; ++j)
                    if (j < qc && cb + j < a.M) Pz[c * a.M + cb + j] = (double)sum[j] + (double)acc[j];
            }
        }
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(a.tmem_cols) : "memory");
}

// 3xTF32 contraction for M <= 64 (the Gram [V^T V | V^T C] of the compact-WY update), with
// 64-row chunks, three products and separate split and drain warps:
//   * a chunk is two 32-row boxes of C (128 columns) and two 32-row boxes of [X_hi; X_lo];
//   * per chunk the MMA warp issues eight A_hi x [X_hi; X_lo] MMAs (N = 2 Nb) and then eight
//     A_lo x X_hi MMAs (N = Nb) into the chunk's accumulator: hi hi' lands alone in columns
//     0..Nb-1 (eight accumulation steps per chunk), hi lo' + lo hi' in Nb..2Nb-1 (the lo lo'
//     product, below 2^-22 of the product, is dropped);
//   * warps 2..9 (two per tensor-memory lane quarter, 32 rows of the chunk each) split the landed
//     C tile into TF32 hi/lo parts and store them to the chunk's A buffer in tensor memory;
//   * warps 10..17 (two per lane quarter, Nb/2 output columns each) drain the accumulator of the
//     previous chunk into FP32 registers while the next chunk is split and multiplied; every
//     TC_FOLD3 chunks a compensated fold (TwoSum) into a second register set.
// Tensor memory: D0, D1 (2 Nb columns each), then A0, A1 (128 columns each: 64 hi, 64 lo).
constexpr int TC3_KC = 64;
constexpr int TC3_MAXST = 6;
constexpr int TC3_FOLD = 8;  // 64-row chunks summed in FP32 registers between compensated folds

template <int NBMAX>
__global__ void __launch_bounds__(TC_THREADS, 1)
    gemm_tn_tc3_kernel(const __grid_constant__ CUtensorMap mapC, const __grid_constant__ CUtensorMap mapX, TcArgs a,
                       double* __restrict__ P, Status* st)
{
    constexpr int KC = TC3_KC;
    constexpr int CQ = NBMAX / 2;  // output columns per drain thread (upper bound)
    __shared__ int s_skip;
    if (threadIdx.x == 0) s_skip = status_error(st);
    __syncthreads();
    if (s_skip) return;  // block-uniform: warp 1's tensor-memory allocation is warp-collective
    extern __shared__ unsigned char smraw[];
    unsigned char* base = reinterpret_cast<unsigned char*>(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
    const int Nb = a.Nb;
    const int boxC = TC_NA * 32 * 4;           // one 32-row box of C: 16 KB
    const int boxX = 2 * Nb * 128;             // one 32-row box of [X_hi; X_lo]
    const int tileC = 2 * boxC, tileX = 2 * boxX;
    const int dcols = 2 * Nb;
    const int stage_bytes = tileC + tileX;
    const int nst = a.nst;
    __shared__ __align__(8) uint64_t full[TC3_MAXST], empty[TC3_MAXST], aready[2], accfull[2], accempty[2];
    __shared__ uint32_t tmem_base;
    __shared__ volatile int s_fail;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp == 1) {
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
        for (int b = 0; b < 2; ++b) {
            mbar_init(&aready[b], 8);
            mbar_init(&accfull[b], 1);
            mbar_init(&accempty[b], 8);
        }
        s_fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = tmem_base;
    const uint32_t tA = tmem + (uint32_t)(2 * dcols);
    const long long n0 = (long long)blockIdx.x * TC_NA;
    const long long kbeg = (long long)blockIdx.y * a.kchunk;
    const long long kend = min(a.K, kbeg + a.kchunk);
    const int nchunks = (int)((kend - kbeg + KC - 1) / KC);
    auto stage_ptr = [&](int s) { return base + (size_t)s * stage_bytes; };
    auto fail = [&]() {
        s_fail = 1;
        set_error(st, RQRCP_ERR_TIMEOUT);
    };

    if (warp == 0) {
        if (lane == 0) {
            int issued = 0;
            for (int kc = 0; kc < nchunks; ++kc) {
                const int s = kc % nst;
                if (kc >= nst && !mbar_wait(&empty[s], (unsigned)((kc - nst) / nst) & 1u, &s_fail)) {
                    fail();
                    break;
                }
                unsigned char* sp = stage_ptr(s);
                const int k0 = (int)(kbeg + (long long)kc * KC);
                mbar_expect_tx(&full[s], tileC + tileX);
                tma_load_2d(sp, &mapC, k0, (int)n0, &full[s]);
                tma_load_2d(sp + boxC, &mapC, k0 + 32, (int)n0, &full[s]);
                tma_load_2d(sp + tileC, &mapX, k0, 0, &full[s]);
                tma_load_2d(sp + tileC + boxX, &mapX, k0 + 32, 0, &full[s]);
                issued = kc + 1;
            }
            // the copies still in flight land before the block leaves (bounded)
            for (int kc = (issued > nst ? issued - nst : 0); kc < issued; ++kc)
                mbar_wait(&full[kc % nst], (unsigned)(kc / nst) & 1u, nullptr);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t id_full = idesc_tf32(TC_NA, 2 * Nb), id_half = idesc_tf32(TC_NA, Nb);
            int issued = 0;
            for (int kc = 0; kc < nchunks; ++kc) {
                const int s = kc % nst, b = kc & 1;
                if (!mbar_wait(&aready[b], (unsigned)(kc >> 1) & 1u, &s_fail) ||
                    (kc >= 2 && !mbar_wait(&accempty[b], (unsigned)((kc - 2) >> 1) & 1u, &s_fail))) {
                    fail();
                    break;
                }
                fence_after();
                const unsigned char* xt = stage_ptr(s) + tileC;
                const uint32_t td = tmem + (uint32_t)(b * dcols);
                const uint32_t ta = tA + (uint32_t)(b * 2 * KC);
                const uint64_t dx0 = umma_desc(xt), dx1 = umma_desc(xt + boxX);
                // k-step j starts 32 bytes further into the 128-byte swizzle rows of its box: the
                // descriptor's address field (bytes >> 4) advances by 2 without carry
#pragma unroll
                for (int j = 0; j < KC / 8; ++j)
                    mma_tf32_ts(td, ta + 8 * j, (j < 4 ? dx0 : dx1) + 2 * (j & 3), id_full, j > 0 ? 1 : 0);
                // the small lo hi' products join hi lo' in columns Nb..2Nb-1, so that the accumulator
                // of the large hi hi' terms takes only the chunk's eight steps
#pragma unroll
                for (int j = 0; j < KC / 8; ++j)
                    mma_tf32_ts(td + (uint32_t)Nb, ta + KC + 8 * j, (j < 4 ? dx0 : dx1) + 2 * (j & 3), id_half, 1);
                mma_commit(&empty[s]);
                mma_commit(&accfull[b]);
                issued = kc + 1;
            }
            // every MMA chain completes before tensor memory is freed (bounded)
            if (issued > 0) mbar_wait(&empty[(issued - 1) % nst], (unsigned)((issued - 1) / nst) & 1u, nullptr);
        }
    } else if (warp < 10) {
        // split warps: lane quarter q, rows 32 h2 .. 32 h2 + 31 of each chunk (box h2)
        const int q = warp & 3, h2 = (warp - 2) >> 2;
        const int row = 32 * q + lane;
        const uint32_t lane_base = (uint32_t)(32 * q) << 16;
        const long long c = n0 + row;
        for (int kc = 0; kc < nchunks; ++kc) {
            const int s = kc % nst, b = kc & 1;
            // the landed stage, and A[b] free again: the MMAs of chunk kc - 2 have completed
            bool ok = mbar_wait(&full[s], (unsigned)(kc / nst) & 1u, &s_fail);
            if (ok && kc >= 2) ok = mbar_wait(&accfull[b], (unsigned)((kc - 2) >> 1) & 1u, &s_fail);
            if (!__all_sync(0xffffffffu, ok)) {
                fail();
                break;
            }
            fence_after();
            const unsigned char* box = stage_ptr(s) + h2 * boxC + row * 128;
            const int k0 = (int)(kbeg + (long long)kc * KC) + 32 * h2;
            const uint32_t ta = tA + lane_base + (uint32_t)(b * 2 * KC + 32 * h2);
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                float v[16];
#pragma unroll
                for (int pc = 0; pc < 4; ++pc) {
                    const int piece = (4 * half + pc) ^ (row & 7);
                    const float4 f = *reinterpret_cast<const float4*>(box + piece * 16);
                    v[4 * pc] = f.x;
                    v[4 * pc + 1] = f.y;
                    v[4 * pc + 2] = f.z;
                    v[4 * pc + 3] = f.w;
                }
                if (c - a.maskC0 >= 0 && c - a.maskC0 < a.maskC && k0 < a.maskC) {
#pragma unroll
                    for (int u = 0; u < 16; ++u) {
                        const long long qq = (long long)k0 + 16 * half + u;
                        if (qq < c - a.maskC0) v[u] = 0.f;
                        else if (qq == c - a.maskC0) v[u] = 1.f;
                    }
                }
                uint32_t hi[16], lo[16];
#pragma unroll
                for (int u = 0; u < 16; ++u) {
                    const float hv = tf32_rn(v[u]);
                    hi[u] = __float_as_uint(hv);
                    lo[u] = __float_as_uint(tf32_rn(v[u] - hv));
                }
                const uint32_t th = ta + (uint32_t)(16 * half), tl = th + (uint32_t)KC;
                asm volatile(
                    "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                    "%16};" ::"r"(th),
                    "r"(hi[0]), "r"(hi[1]), "r"(hi[2]), "r"(hi[3]), "r"(hi[4]), "r"(hi[5]), "r"(hi[6]), "r"(hi[7]),
                    "r"(hi[8]), "r"(hi[9]), "r"(hi[10]), "r"(hi[11]), "r"(hi[12]), "r"(hi[13]), "r"(hi[14]),
                    "r"(hi[15])
                    : "memory");
                asm volatile(
                    "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                    "%16};" ::"r"(tl),
                    "r"(lo[0]), "r"(lo[1]), "r"(lo[2]), "r"(lo[3]), "r"(lo[4]), "r"(lo[5]), "r"(lo[6]), "r"(lo[7]),
                    "r"(lo[8]), "r"(lo[9]), "r"(lo[10]), "r"(lo[11]), "r"(lo[12]), "r"(lo[13]), "r"(lo[14]),
                    "r"(lo[15])
                    : "memory");
            }
            asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
            fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&aready[b]);
        }
    } else {
        // drain warps: lane quarter q, output columns cb .. cb + qc - 1
        const int q = warp & 3, hd = (warp - 10) >> 2;
        const int qc = Nb >> 1;
        const int cb = hd * qc;
        const int row = 32 * q + lane;
        const uint32_t lane_base = (uint32_t)(32 * q) << 16;
        const long long c = n0 + row;
        float acc[CQ], sum[CQ];
#pragma unroll
        for (int j = 0; j < CQ; ++j) acc[j] = sum[j] = 0.f;
        auto fold = [&]() {
#pragma unroll
            for (int j = 0; j < CQ; ++j) {
                const float t = sum[j] + acc[j];
                const float bp = t - sum[j];
                const float e = (sum[j] - (t - bp)) + (acc[j] - bp);
                sum[j] = t;
                acc[j] = e;
            }
        };
        bool ok = true;
        for (int kc = 0; kc < nchunks; ++kc) {
            const int b = kc & 1;
            if (!__all_sync(0xffffffffu, mbar_wait(&accfull[b], (unsigned)(kc >> 1) & 1u, &s_fail))) {
                ok = false;
                break;
            }
            fence_after();
            const uint32_t tb = tmem + lane_base + (uint32_t)(b * dcols + cb);
            // groups of 8 columns: the X_hi product at tb + j, the X_lo product at tb + Nb + j
#pragma unroll
            for (int g0 = 0; g0 < CQ; g0 += 8) {
                if (g0 < qc) {
                    uint32_t rh[8], rl[8];
                    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                                 : "=r"(rh[0]), "=r"(rh[1]), "=r"(rh[2]), "=r"(rh[3]), "=r"(rh[4]), "=r"(rh[5]),
                                   "=r"(rh[6]), "=r"(rh[7])
                                 : "r"(tb + (uint32_t)g0));
                    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                                 : "=r"(rl[0]), "=r"(rl[1]), "=r"(rl[2]), "=r"(rl[3]), "=r"(rl[4]), "=r"(rl[5]),
                                   "=r"(rl[6]), "=r"(rl[7])
                                 : "r"(tb + (uint32_t)(Nb + g0)));
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                    for (int u = 0; u < 8; ++u) acc[g0 + u] += __uint_as_float(rl[u]) + __uint_as_float(rh[u]);
                }
            }
            fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&accempty[b]);
            if ((kc + 1) % TC3_FOLD == 0) fold();
        }
        if (!ok) {
            fail();
        } else if (nchunks > 0) {
            fold();
            double* Pz = P + (long long)blockIdx.y * a.N * a.M;
            if (c < a.N) {
#pragma unroll
                for (int j = 0; j < CQ; ++j)
                    if (j < qc && cb + j < a.M) Pz[c * a.M + cb + j] = (double)sum[j] + (double)acc[j];
            }
        }
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(a.tmem_cols) : "memory");
}

}  // namespace

namespace {

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

// TC_KC x box_outer box with 128-byte swizzle over K-major FP32 lines.
bool encode_map(CUtensorMap* map, const float* base, long long inner, long long outer, long long ld, int box_outer)
{
    return tc_encode_2d(map, base, inner, outer, ld, TC_KC, box_outer, true);
}

size_t tc_smem_bytes(int Nb, int nst, bool bf)
{
    const size_t stage = bf ? (size_t)TC_NA * 64 * 4 + (size_t)Nb * 128 : (size_t)TC_NA * TC_KC * 4 + 2 * (size_t)Nb * 128;
    return 1024 + (size_t)nst * stage;
}

// Dynamic shared memory a kernel may use next to its static shared memory.
template <int NBMAX, bool BF>
size_t tc_dyn_limit()
{
    static std::atomic<size_t> lim{0};
    size_t v = lim.load(std::memory_order_relaxed);
    if (v == 0) {
        cudaFuncAttributes fa;
        if (cudaFuncGetAttributes(&fa, (const void*)gemm_tn_tc_kernel<NBMAX, BF>) != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        v = (size_t)dev_info().max_smem_optin - fa.sharedSizeBytes;
        lim.store(v, std::memory_order_relaxed);
    }
    return v;
}

size_t tc_dyn_limit_for(int Nb, bool bf)
{
    if (bf) return Nb <= 32 ? tc_dyn_limit<32, true>() : Nb <= 64 ? tc_dyn_limit<64, true>() : tc_dyn_limit<96, true>();
    return Nb <= 32 ? tc_dyn_limit<32, false>() : Nb <= 64 ? tc_dyn_limit<64, false>() : tc_dyn_limit<96, false>();
}

// The 3xTF32 contraction for M <= 64 (gemm_tn_tc3_kernel): stage = two C boxes + two X boxes.
size_t tc3_smem_bytes(int Nb, int nst) { return 1024 + (size_t)nst * ((size_t)TC_NA * TC3_KC * 4 + 4 * (size_t)Nb * 128); }

template <int NBMAX>
size_t tc3_dyn_limit()
{
    static std::atomic<size_t> lim{0};
    size_t v = lim.load(std::memory_order_relaxed);
    if (v == 0) {
        cudaFuncAttributes fa;
        if (cudaFuncGetAttributes(&fa, (const void*)gemm_tn_tc3_kernel<NBMAX>) != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        v = (size_t)dev_info().max_smem_optin - fa.sharedSizeBytes;
        lim.store(v, std::memory_order_relaxed);
    }
    return v;
}

int tc3_stages(int Nb)
{
    const size_t lim = Nb <= 16 ? tc3_dyn_limit<16>() : Nb <= 32 ? tc3_dyn_limit<32>() : tc3_dyn_limit<64>();
    for (int nst = TC3_MAXST; nst >= 2; --nst)
        if (tc3_smem_bytes(Nb, nst) <= lim) return nst;
    return 0;
}

// Pipeline depth: TC_MAXST stages where they fit, else fewer (0: not even 2 fit).
int tc_stages(int Nb, bool bf)
{
    const size_t lim = tc_dyn_limit_for(Nb, bf);
    for (int nst = TC_MAXST; nst >= 2; --nst)
        if (tc_smem_bytes(Nb, nst, bf) <= lim) return nst;
    return 0;
}

}  // namespace

bool tc_encoder_available() { return tensor_map_encoder() != nullptr; }

bool tc_encode_2d(CUtensorMap* map, const float* base, long long inner, long long outer, long long ld, int box_inner,
                  int box_outer, bool swizzle128)
{
    return tc_encode_2d_typed(map, base, 4, inner, outer, ld, box_inner, box_outer, swizzle128);
}

bool tc_encode_2d_typed(CUtensorMap* map, const void* base, int elem_bytes, long long inner, long long outer,
                        long long ld, int box_inner, int box_outer, bool swizzle128)
{
    auto enc = tensor_map_encoder();
    if (enc == nullptr || (elem_bytes != 4 && elem_bytes != 2)) return false;
    cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)outer};
    cuuint64_t strides[1] = {(cuuint64_t)ld * elem_bytes};
    cuuint32_t box[2] = {(cuuint32_t)box_inner, (cuuint32_t)box_outer};
    cuuint32_t es[2] = {1, 1};
    return enc(map, elem_bytes == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
               const_cast<void*>(base), dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
               swizzle128 ? CU_TENSOR_MAP_L2_PROMOTION_L2_256B : CU_TENSOR_MAP_L2_PROMOTION_NONE,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool tc_gemm_supported(long long M, long long ldc, const void* C, int bf16)
{
    if (!(M >= 1 && M <= 96 && (ldc % 4) == 0 && ((uintptr_t)C % 16) == 0 && tensor_map_encoder() != nullptr))
        return false;
    const int Nb = (int)(((M + 15) / 16) * 16);
    if (!bf16 && Nb <= 64) return tc3_stages(Nb) >= 2;
    return tc_stages(Nb, bf16 != 0) >= 2;
}

size_t tc_xsplit_bytes(long long M, long long K)
{
    return 2 * (size_t)((M + 15) / 16 * 16) * (size_t)((K + 3) / 4 * 4) * sizeof(float);
}

// Split-K chunk for the tensor-core kernel (one resident block per SM): the split count S <= 16
// minimising waves x (rows per split + a pipeline fill of about three chunks), splits of at
// least 256 rows; a multiple of the chunk height (64 for the BF16 form and for M <= 64, else 32).
long long tc_kchunk(long long N, long long K, int& nsplit, int bf16, long long M)
{
    const long long KC = (bf16 || M <= 64) ? 64 : TC_KC;
    const long long ntiles = (N + TC_NA - 1) / TC_NA;
    const long long sms = dev_info().sms;
    long long smax = (K + 255) / 256;
    if (smax > 16) smax = 16;
    if (smax < 1) smax = 1;
    long long best = 1, best_cost = -1;
    for (long long S = 1; S <= smax; ++S) {
        const long long rows = ((K + S - 1) / S + KC - 1) / KC * KC;
        const long long waves = (ntiles * S + sms - 1) / sms;
        const long long cost = waves * (rows + 3 * KC);
        if (best_cost < 0 || cost < best_cost) {
            best_cost = cost;
            best = S;
        }
    }
    long long kc = (K + best - 1) / best;
    kc = ((kc + KC - 1) / KC) * KC;
    nsplit = (int)((K + kc - 1) / kc);
    return kc;
}

cudaError_t launch_gemm_tn_tc(const float* X, long long ldx, const float* C, long long ldc, long long M, long long N,
                              long long K, long long kchunk, double* P, long long maskX, long long maskC, float* xs,
                              const Status* st, cudaStream_t s, int bf16, long long maskC0)
{
    const bool bf = bf16 != 0;
    const int Nb = (int)(((M + 15) / 16) * 16);
    const int nst = tc_stages(Nb, bf);
    if (nst < 2 || ((uintptr_t)xs % 16) != 0 || (bf && (maskX != 0 || maskC != 0)) || maskC0 < 0)
        return cudaErrorInvalidValue;
    CUtensorMap mapC, mapX;
    {
        long long gx = (K + 255) / 256;
        if (gx > 64) gx = 64;
        if (bf) {
            // Nb lines of ldk BF16 values (lines M.. zero)
            const long long ldk = (K + 7) / 8 * 8;
            __nv_bfloat16* xb = reinterpret_cast<__nv_bfloat16*>(xs);
            xsplit_bf16_kernel<<<dim3((unsigned)gx, (unsigned)Nb), 256, 0, s>>>(X, ldx, K, (int)M, ldk, xb, st);
            if (cudaError_t e = cudaGetLastError()) return e;
            if (!tc_encode_2d_typed(&mapX, xb, 2, K, Nb, ldk, 64, Nb, true)) return cudaErrorInvalidValue;
        } else {
            // Nb lines of ldk FP32 hi parts (lines M.. zero), then the lo parts: [X_hi; X_lo]
            const long long ldk = (K + 3) / 4 * 4;
            float* xh = xs;
            float* xl = xs + (size_t)Nb * ldk;
            xsplit_kernel<<<dim3((unsigned)gx, (unsigned)Nb), 256, 0, s>>>(X, ldx, K, (int)M, maskX, ldk, xh, xl, st);
            if (cudaError_t e = cudaGetLastError()) return e;
            if (!encode_map(&mapX, xh, K, 2 * Nb, ldk, 2 * Nb)) return cudaErrorInvalidValue;
        }
    }
    if (!encode_map(&mapC, C, K, N, ldc, TC_NA)) return cudaErrorInvalidValue;
    if (!bf && Nb <= 64) {
        // 3xTF32, 64-row chunks, three products (gemm_tn_tc3_kernel)
        const int nst3 = tc3_stages(Nb);
        if (nst3 < 2 || kchunk % TC3_KC != 0) return cudaErrorInvalidValue;
        TcArgs a3;
        a3.M = (int)M;
        a3.Nb = Nb;
        a3.N = N;
        a3.K = K;
        a3.kchunk = kchunk;
        a3.maskC = maskC;
        a3.maskC0 = maskC0;
        a3.nst = nst3;
        a3.tmem_cols = 512;  // D0, D1 (2 Nb each), A0, A1 (128 each)
        const size_t smem3 = tc3_smem_bytes(Nb, nst3);
        dim3 grid3((unsigned)((N + TC_NA - 1) / TC_NA), (unsigned)((K + kchunk - 1) / kchunk));
        auto run3 = [&](auto kern, DevFlag& attr_set) -> cudaError_t {
            if (!attr_set.done()) {
                if (cudaError_t e = allow_max_dynamic_smem(kern)) return e;
                attr_set.set();
            }
            kern<<<grid3, TC_THREADS, smem3, s>>>(mapC, mapX, a3, P, const_cast<Status*>(st));
            return cudaGetLastError();
        };
        static DevFlag set3[3];
        if (Nb <= 16) return run3(gemm_tn_tc3_kernel<16>, set3[0]);
        if (Nb <= 32) return run3(gemm_tn_tc3_kernel<32>, set3[1]);
        return run3(gemm_tn_tc3_kernel<64>, set3[2]);
    }
    TcArgs a;
    a.M = (int)M;
    a.Nb = Nb;
    a.N = N;
    a.K = K;
    a.kchunk = kchunk;
    a.maskC = maskC;
    a.maskC0 = maskC0;
    a.nst = nst;
    unsigned cols = 32;
    const int need = bf ? 2 * Nb + 64 : 4 * Nb + 128;  // D0, D1, A0, A1
    while ((int)cols < need) cols <<= 1;
    a.tmem_cols = cols;
    const size_t smem = tc_smem_bytes(Nb, nst, bf);
    dim3 grid((unsigned)((N + TC_NA - 1) / TC_NA), (unsigned)((K + kchunk - 1) / kchunk));
    auto run = [&](auto kern, DevFlag& attr_set) -> cudaError_t {
        if (!attr_set.done()) {
            if (cudaError_t e = allow_max_dynamic_smem(kern)) return e;
            attr_set.set();
        }
        kern<<<grid, TC_THREADS, smem, s>>>(mapC, mapX, a, P, const_cast<Status*>(st));
        return cudaGetLastError();
    };
    static DevFlag set[6];
    if (bf) {
        if (Nb <= 32) return run(gemm_tn_tc_kernel<32, true>, set[3]);
        if (Nb <= 64) return run(gemm_tn_tc_kernel<64, true>, set[4]);
        return run(gemm_tn_tc_kernel<96, true>, set[5]);
    }
    if (Nb <= 32) return run(gemm_tn_tc_kernel<32, false>, set[0]);
    if (Nb <= 64) return run(gemm_tn_tc_kernel<64, false>, set[1]);
    return run(gemm_tn_tc_kernel<96, false>, set[2]);
}

}  // namespace rq
