// mm_tc.cu -- general FP32 contraction on the tensor cores (tcgen05 kind::tf32, 3xTF32), used by
// the FP32 backward of the truncated factorization:
//   D(r, dcol(c)) = alpha sum_q A(r, q) B(q, c) + beta D0(r, dcol(c)),  r < M, c < N, q < K,
// dcol(c) = dmap[c] (a column scatter) or c.  A is M x K column-major (A(r, q) = A[q lda + r]) or,
// K-major, A(r, q) = A[r lda + q] (the transpose of a column-major K x M matrix).  B comes as TF32
// planes (launch_mm_planes): for each 128-column tile of B, 128 lines of tf32(B(:, c)) followed by
// 128 lines of tf32(B - tf32(B)), each line the K values of one column, zero-padded to a multiple
// of 32.  The product is A_hi B_hi + A_hi B_lo + A_lo B_hi (x = hi + lo, hi = tf32(x),
// lo = tf32(x - hi)), accumulated in FP32 in tensor memory.
//
// One block per 128 x 128 tile of D and contraction range (blockIdx.z splits K; split z writes
// D + z dz, the caller sums the splits).  Roles: a TMA producer warp loads per 32-long chunk of K
// the B planes' tile (128-byte swizzle, K-major: the MMA's B operand) and A's 128 x 32 tile into a
// stage; eight worker warps split A's tile into TF32 parts and store them to tensor memory (the
// MMA's A operand, hi parts in 32 columns and lo parts in 32 more); one thread issues the twelve
// MMAs of the chunk (four K-steps of 8, three products each) and commits them to the stage's
// "free" barrier; after the last chunk the workers read the 128 x 128 accumulator (tcgen05.ld)
// and write D with plain coalesced stores (one column of 32 rows per warp store), applying
// alpha, beta and the column map.  Two stages and 256 tensor-memory columns per block let two
// blocks share an SM, so one block's epilogue overlaps the other's MMAs.  Every wait is
// bounded; on timeout the block records RQRCP_ERR_TIMEOUT, lets its copies land and frees its
// tensor memory.
#include "df.cuh"
#include "tc_common.cuh"

namespace rq {
namespace {
using namespace tc;

constexpr int MM_BM = 128;                        // rows of D per tile (MMA M)
constexpr int MM_BN = 128;                        // columns of D per tile (MMA N)
constexpr int MM_KC = 32;                         // contraction chunk: one 128-byte span of TF32
constexpr int MM_NST = 2;                         // pipeline stages
constexpr int MM_WW = 8;                          // worker warps (two per tensor-memory lane quarter)
constexpr int MM_THREADS = 64 + 32 * MM_WW;       // + TMA producer warp + MMA warp
constexpr int MM_TILE_B = 2 * MM_BN * MM_KC * 4;  // 32 KB: 128 hi lines, then 128 lo lines
constexpr int MM_TILE_A = MM_BM * MM_KC * 4;      // 16 KB
constexpr int MM_STAGE = MM_TILE_B + MM_TILE_A;
constexpr unsigned MM_TMEM_COLS = 256;            // accumulator 0..127; A stage s at 128 + 64 s
constexpr int MM_MAX_SPLIT = 64;

long long mm_kp(long long K) { return (K + MM_KC - 1) / MM_KC * MM_KC; }
long long mm_ntiles(long long N) { return (N + MM_BN - 1) / MM_BN; }

// planes (see the file comment) of B(q, c) = src[kq * ldk + c * ldn], kq = kmap ? kmap[q] : q;
// zero where q >= K, c >= N or kmap[q] < kmin.  mask 1: B is unit lower (B(q, c) = 0 for q < c,
// 1 for q == c, as the reflector block V); mask 2: B is upper (B(q, c) = 0 for q > c).
__global__ void mm_planes_kernel(const float* __restrict__ src, long long ldk, long long ldn,
                                 const int32_t* __restrict__ kmap, long long kmin, long long K, long long N,
                                 int mask, long long kp, long long ntiles, float* __restrict__ planes,
                                 const Status* st)
{
    if (status_error(st)) return;
    const long long total = ntiles * MM_BN * kp;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const long long q = e % kp, c = e / kp;
        const long long t = c / MM_BN;
        const long long j = c % MM_BN;
        float h = 0.f, l = 0.f;
        if (q < K && c < N) {
            long long kq = q;
            bool keep = true;
            if (kmap != nullptr) {
                kq = kmap[q];
                keep = kq >= kmin;
            }
            if (mask == 1 && q <= c) {
                keep = false;
                if (q == c) h = 1.f;
            }
            if (mask == 2 && q > c) keep = false;
            if (keep) {
                const float v = src[kq * ldk + c * ldn];
                h = tf32_rn(v);
                l = tf32_rn(v - h);
            }
        }
        planes[(t * 2 * MM_BN + j) * kp + q] = h;
        planes[(t * 2 * MM_BN + MM_BN + j) * kp + q] = l;
    }
}

struct MmArgs {
    long long M, N;        // D is M x N
    long long nchunks;     // ceil(K / 32)
    long long cps;         // chunks per split
    float alpha, beta;
    const float* D0;
    long long ldd0;
    float* D;
    long long ldd, dz;     // split z writes D + z * dz
    const int32_t* dmap;   // column map of D and D0 (null: identity)
    int amask;             // 1: A is a unit-lower reflector block (see mm_tc_kernel)
};

__device__ __forceinline__ void tmem_st16(uint32_t addr, const uint32_t (&v)[16])
{
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(
            addr),
        "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]),
        "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15])
        : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t addr, uint32_t (&v)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
          "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(addr));
}

// KMAJ: A(r, q) = A[r lda + q] (tile loaded as 128 lines of 32 values, 128-byte swizzle);
// otherwise A(r, q) = A[q lda + r] (tile loaded as 32 columns of 128 rows).  amask: the stored
// matrix is a unit-lower reflector block V (V(i, j) = 0 for i < j, 1 for i == j; the strict upper
// part holds other data): A = V (A(r, q) = V(r, q)) or, KMAJ, A = V^T (A(r, q) = V(q, r)).
template <bool KMAJ>
__global__ void __launch_bounds__(MM_THREADS, 2)
    mm_tc_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, MmArgs a,
                 Status* st)
{
    __shared__ int s_skip;
    if (threadIdx.x == 0) s_skip = status_error(st);
    __syncthreads();
    if (s_skip) return;  // block-uniform: warp 1's tensor-memory allocation is warp-collective
    extern __shared__ unsigned char smraw[];
    unsigned char* base = reinterpret_cast<unsigned char*>(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t full[MM_NST], freed[MM_NST], aready[MM_NST], accfull;
    __shared__ uint32_t tmem_base;
    __shared__ volatile int s_fail;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp == 1) tmem_alloc(&tmem_base, MM_TMEM_COLS);
    if (tid == 0) {
        for (int s = 0; s < MM_NST; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&freed[s], 1);
            mbar_init(&aready[s], MM_WW);
        }
        mbar_init(&accfull, 1);
        s_fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = tmem_base;
    const long long c0 = (long long)blockIdx.x * MM_BN, r0 = (long long)blockIdx.y * MM_BM;
    const long long jbeg = (long long)blockIdx.z * a.cps;
    const long long jend = (jbeg + a.cps < a.nchunks) ? jbeg + a.cps : a.nchunks;
    const int nch = (int)(jend - jbeg);  // >= 1: the launcher leaves no split empty
    auto fail = [&]() {
        s_fail = 1;
        set_error(st, RQRCP_ERR_TIMEOUT);
    };

    if (warp == 0) {
        if (lane == 0) {
            int t = 0;
            bool ok = true;
            for (; t < nch; ++t) {
                const int s = t % MM_NST;
                if (t >= MM_NST && !mbar_wait(&freed[s], (unsigned)(t / MM_NST - 1) & 1u, &s_fail)) {
                    fail();
                    ok = false;
                    break;
                }
                unsigned char* sp = base + (size_t)s * MM_STAGE;
                const int q0 = (int)((jbeg + t) * MM_KC);
                mbar_expect_tx(&full[s], MM_STAGE);
                tma_load_2d(sp, &mapB, q0, (int)(blockIdx.x * 2 * MM_BN), &full[s]);
                if (KMAJ)
                    tma_load_2d(sp + MM_TILE_B, &mapA, q0, (int)r0, &full[s]);
                else
                    tma_load_2d(sp + MM_TILE_B, &mapA, (int)r0, q0, &full[s]);
            }
            if (!ok)  // loads still in flight (chunks t - MM_NST .. t - 1) land before the block leaves
                for (int u = (t > MM_NST ? t - MM_NST : 0); u < t; ++u)
                    mbar_wait(&full[u % MM_NST], (unsigned)(u / MM_NST) & 1u, nullptr);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = idesc_tf32(MM_BM, MM_BN);
            int issued = 0;
            for (int t = 0; t < nch; ++t) {
                const int s = t % MM_NST;
                const unsigned ph = (unsigned)(t / MM_NST) & 1u;
                if (!mbar_wait(&full[s], ph, &s_fail) || !mbar_wait(&aready[s], ph, &s_fail)) {
                    fail();
                    break;
                }
                fence_after();
                const unsigned char* bt = base + (size_t)s * MM_STAGE;
                const uint32_t ta = tmem + 128 + 64 * s;
#pragma unroll
                for (int kk = 0; kk < MM_KC / 8; ++kk) {
                    const uint64_t bh = umma_desc(bt + 32 * kk);
                    const uint64_t bl = umma_desc(bt + MM_TILE_B / 2 + 32 * kk);
                    mma_tf32_ts(tmem, ta + 32 + 8 * kk, bh, idesc, (t > 0 || kk > 0) ? 1 : 0);  // A_lo B_hi
                    mma_tf32_ts(tmem, ta + 8 * kk, bl, idesc, 1);                               // A_hi B_lo
                    mma_tf32_ts(tmem, ta + 8 * kk, bh, idesc, 1);                               // A_hi B_hi
                }
                mma_commit(&freed[s]);
                issued = t + 1;
            }
            if (issued == nch) mma_commit(&accfull);
            // every MMA completes before tensor memory is freed (bounded)
            if (issued > 0)
                mbar_wait(&freed[(issued - 1) % MM_NST], (unsigned)((issued - 1) / MM_NST) & 1u, nullptr);
        }
    } else {
        const int q = warp & 3;         // tensor-memory lane quarter
        const int g = (warp - 2) >> 2;  // half: A columns 16 g .. 16 g + 15 of a chunk, D columns 64 g ..
        const int row = 32 * q + lane;  // row within the tile
        const uint32_t lane_base = (uint32_t)(32 * q) << 16;
        bool ok = true;
        for (int t = 0; t < nch; ++t) {
            const int s = t % MM_NST;
            bool okw = true;
            if (t >= MM_NST) okw = mbar_wait(&freed[s], (unsigned)(t / MM_NST - 1) & 1u, &s_fail);
            okw = okw && mbar_wait(&full[s], (unsigned)(t / MM_NST) & 1u, &s_fail);
            if (!__all_sync(0xffffffffu, okw)) {
                ok = false;
                break;
            }
            fence_after();
            const float* at = reinterpret_cast<const float*>(base + (size_t)s * MM_STAGE + MM_TILE_B);
            float v[16];
            if (KMAJ) {
                // line `row` holds A(r0 + row, q0 .. q0 + 31); 16-byte chunk c sits at c ^ (row & 7)
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int ch = (4 * g + u) ^ (row & 7);
                    const float4 x = *reinterpret_cast<const float4*>(at + row * MM_KC + 4 * ch);
                    v[4 * u] = x.x;
                    v[4 * u + 1] = x.y;
                    v[4 * u + 2] = x.z;
                    v[4 * u + 3] = x.w;
                }
            } else {
#pragma unroll
                for (int u = 0; u < 16; ++u) v[u] = at[(16 * g + u) * MM_BM + row];
            }
            if (a.amask) {
                const long long rr = r0 + row, q0 = (jbeg + t) * MM_KC + 16 * g;
#pragma unroll
                for (int u = 0; u < 16; ++u) {
                    const long long i = KMAJ ? q0 + u : rr, j = KMAJ ? rr : q0 + u;  // V(i, j)
                    if (i <= j) v[u] = (i == j) ? 1.f : 0.f;
                }
            }
            uint32_t hi[16], lo[16];
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                const float h = tf32_rn(v[u]);
                hi[u] = __float_as_uint(h);
                lo[u] = __float_as_uint(tf32_rn(v[u] - h));
            }
            const uint32_t ta = tmem + 128 + 64 * s + lane_base + (uint32_t)(16 * g);
            tmem_st16(ta, hi);
            tmem_st16(ta + 32, lo);
            asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
            fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&aready[s]);
        }
        if (ok && !__all_sync(0xffffffffu, mbar_wait(&accfull, 0u, &s_fail))) ok = false;
        if (ok) {
            fence_after();
            const long long r = r0 + row;
            float* Dz = a.D + (long long)blockIdx.z * a.dz;
#pragma unroll 1
            for (int u = 0; u < 4; ++u) {
                uint32_t acc[16];
                tmem_ld16(tmem + lane_base + (uint32_t)(64 * g + 16 * u), acc);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                // the column map and D0 values of these 16 columns are loaded before any store (D0 may
                // be D itself), so each group of 16 costs one memory round trip, not sixteen
                const long long cb = c0 + 64 * g + 16 * u;
                int cd[16];
#pragma unroll
                for (int w = 0; w < 16; ++w)
                    cd[w] = (a.dmap != nullptr && cb + w < a.N) ? a.dmap[cb + w] : (int)(cb + w);
                float d0[16];
#pragma unroll
                for (int w = 0; w < 16; ++w)
                    d0[w] = (a.beta != 0.f && r < a.M && cb + w < a.N) ? a.D0[(long long)cd[w] * a.ldd0 + r] : 0.f;
                if (r < a.M) {
#pragma unroll
                    for (int w = 0; w < 16; ++w)
                        if (cb + w < a.N)
                            Dz[(long long)cd[w] * a.ldd + r] = fmaf(a.beta, d0[w], a.alpha * __uint_as_float(acc[w]));
                }
            }
        }
        if (!ok) fail();
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 1) tmem_dealloc(tmem, MM_TMEM_COLS);
}

size_t mm_smem_bytes() { return 1024 + (size_t)MM_NST * MM_STAGE; }

// Sum of split partials: D(r, c) = D0(r, c) + sum_z P[z dz + c ldp + r] (r < M, c < N), a compensated sum.
__global__ void mm_sum_kernel(const float* __restrict__ P, long long ldp, long long dz, int nz, long long M, long long N,
                              const float* __restrict__ D0, long long ldd0, float* __restrict__ D, long long ldd,
                              const Status* st)
{
    if (status_error(st)) return;
    const long long total = M * N;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const long long r = e % M, c = e / M;
        float sh = D0 != nullptr ? D0[c * ldd0 + r] : 0.f, sl = 0.f;
        for (int z0 = 0; z0 < nz; z0 += 4) {  // four loads in flight per step, compensated sum in order
            float pv[4];
#pragma unroll
            for (int zz = 0; zz < 4; ++zz) pv[zz] = z0 + zz < nz ? P[(z0 + zz) * dz + c * ldp + r] : 0.f;
#pragma unroll
            for (int zz = 0; zz < 4; ++zz) {
                const df t = df_two_sum(sh, pv[zz]);
                sh = t.h;
                sl += t.l;
            }
        }
        D[c * ldd + r] = sh + sl;
    }
}

}  // namespace

bool mm_tc_supported(const void* A, long long lda)
{
    if (A == nullptr || ((uintptr_t)A % 16) != 0 || (lda % 4) != 0 || !tc_encoder_available()) return false;
    static int fits = -1;
    if (fits < 0) {
        cudaFuncAttributes f0, f1;
        if (cudaFuncGetAttributes(&f0, (const void*)mm_tc_kernel<false>) != cudaSuccess ||
            cudaFuncGetAttributes(&f1, (const void*)mm_tc_kernel<true>) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        const size_t st = f0.sharedSizeBytes > f1.sharedSizeBytes ? f0.sharedSizeBytes : f1.sharedSizeBytes;
        fits = mm_smem_bytes() + st <= (size_t)dev_info().max_smem_optin ? 1 : 0;
    }
    return fits == 1;
}

size_t mm_planes_bytes(long long K, long long N)
{
    if (K < 1 || N < 1) return 0;
    return (size_t)mm_ntiles(N) * 2 * MM_BN * (size_t)mm_kp(K) * sizeof(float);
}

int mm_max_split() { return MM_MAX_SPLIT; }

// Splits of the contraction for an M x N result: enough blocks for two per SM, each split at
// least min_chunks chunks of 32, at most MM_MAX_SPLIT.
int mm_choose_split(long long M, long long N, long long K, int min_chunks)
{
    const long long tiles = mm_ntiles(N) * ((M + MM_BM - 1) / MM_BM);
    const long long nch = mm_kp(K) / MM_KC;
    long long S = (2LL * dev_info().sms) / (tiles > 0 ? tiles : 1);
    const long long smax = nch / (min_chunks > 0 ? min_chunks : 1);
    if (S > smax) S = smax;
    if (S > MM_MAX_SPLIT) S = MM_MAX_SPLIT;
    if (S < 1) S = 1;
    const long long cps = (nch + S - 1) / S;
    return (int)((nch + cps - 1) / cps);
}

cudaError_t launch_mm_planes(const float* src, long long ldk, long long ldn, const int32_t* kmap, long long kmin,
                             long long K, long long N, float* planes, const Status* st, cudaStream_t s, int mask)
{
    if (K < 1 || N < 1) return cudaSuccess;
    if (((uintptr_t)planes % 16) != 0) return cudaErrorInvalidValue;
    const long long kp = mm_kp(K), ntiles = mm_ntiles(N);
    const long long total = ntiles * MM_BN * kp;
    long long blocks = (total + 255) / 256;
    if (blocks > 8L * dev_info().sms) blocks = 8L * dev_info().sms;
    mm_planes_kernel<<<(unsigned)blocks, 256, 0, s>>>(src, ldk, ldn, kmap, kmin, K, N, mask, kp, ntiles, planes, st);
    return cudaGetLastError();
}

cudaError_t launch_mm_tc(bool kmajor, const float* A, long long lda, const float* planes, long long M, long long N,
                         long long K, int nsplit, float alpha, float beta, const float* D0, long long ldd0, float* D,
                         long long ldd, long long dz, const int32_t* dmap, Status* st, cudaStream_t s, int amask)
{
    if (M <= 0 || N <= 0) return cudaSuccess;
    if (K < 1 || (nsplit > 1 && beta != 0.f) || (beta != 0.f && D0 == nullptr)) return cudaErrorInvalidValue;
    if (((uintptr_t)planes % 16) != 0 || !mm_tc_supported(A, lda)) return cudaErrorInvalidValue;
    const long long kp = mm_kp(K), ntiles = mm_ntiles(N), bands = (M + MM_BM - 1) / MM_BM;
    if (bands > 65535 || nsplit > 65535) return cudaErrorInvalidValue;
    MmArgs a;
    a.M = M;
    a.N = N;
    a.nchunks = kp / MM_KC;
    long long S = nsplit < 1 ? 1 : nsplit;
    if (S > a.nchunks) S = a.nchunks;
    a.cps = (a.nchunks + S - 1) / S;
    S = (a.nchunks + a.cps - 1) / a.cps;  // no empty split
    a.alpha = alpha;
    a.beta = beta;
    a.D0 = D0;
    a.ldd0 = ldd0;
    a.D = D;
    a.ldd = ldd;
    a.dz = S > 1 ? dz : 0;
    a.dmap = dmap;
    a.amask = amask;
    CUtensorMap mapA, mapB;
    const bool okA = kmajor ? tc_encode_2d(&mapA, A, K, M, lda, MM_KC, MM_BM, true)
                            : tc_encode_2d(&mapA, A, M, K, lda, MM_BM, MM_KC, false);
    if (!okA) return cudaErrorInvalidValue;
    if (!tc_encode_2d(&mapB, planes, kp, ntiles * 2 * MM_BN, kp, MM_KC, 2 * MM_BN, true)) return cudaErrorInvalidValue;
    static DevFlag attr_set;
    if (!attr_set.done()) {
        for (auto kern : {mm_tc_kernel<false>, mm_tc_kernel<true>}) {
            if (cudaError_t e = allow_max_dynamic_smem(kern)) return e;
            if (cudaError_t e = cudaFuncSetAttribute((const void*)kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                                     100))
                return e;
        }
        attr_set.set();
    }
    const dim3 grid((unsigned)ntiles, (unsigned)bands, (unsigned)S);
    if (kmajor)
        mm_tc_kernel<true><<<grid, MM_THREADS, mm_smem_bytes(), s>>>(mapA, mapB, a, st);
    else
        mm_tc_kernel<false><<<grid, MM_THREADS, mm_smem_bytes(), s>>>(mapA, mapB, a, st);
    return cudaGetLastError();
}

cudaError_t launch_mm_sum(const float* P, long long ldp, long long dz, int nz, long long M, long long N, const float* D0,
                          long long ldd0, float* D, long long ldd, const Status* st, cudaStream_t s)
{
    if (M <= 0 || N <= 0) return cudaSuccess;
    long long blocks = (M * N + 255) / 256;
    if (blocks > 8L * dev_info().sms) blocks = 8L * dev_info().sms;
    mm_sum_kernel<<<(unsigned)blocks, 256, 0, s>>>(P, ldp, dz, nz, M, N, D0, ldd0, D, ldd, st);
    return cudaGetLastError();
}

}  // namespace rq
