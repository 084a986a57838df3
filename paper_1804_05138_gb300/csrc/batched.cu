// batched.cu -- many independent randomized QRCPs (Alg. 2) of uneven shapes in one persistent
// launch.  Every block (one per SM) repeatedly takes the next matrix from a work queue (an
// atomic counter over a caller-given order, largest first) and factors that matrix alone,
// with block-level synchronisation only:
//   sketch      B = Omega(0:l, 0:m) A on the tensor cores (tcgen05, 3xTF32, accumulator in
//               tensor memory, per-chunk read-back with compensated sums), B row-major (ld = n);
//   pivots      Alg. 1 on B with physical column swaps (ties to the smallest position), norms
//               of rows t..l-1 recomputed while the reflector is applied, FP64 reflector;
//   panel       left-looking in sub-panels of 8 columns held in shared memory, every
//               reflector (norm, beta, tau) formed in FP64;
//   sums        the per-term sums feeding norms and reflectors (column norms of B, the panel's
//               dot products) are Dot2 sums of exact FP32 products carried as float pairs, then
//               combined across the block in FP64: FP64-class results without a per-term FP64
//               operation, which runs at a small fraction of the FP32 rate on this part;
//   update      W = V^T [V C] (Gram and V^T C in one pass, tiled FP32 SIMT with compensated
//               accumulation), T (xLARFT order, FP64), Y = T^T W, C -= V Y (3xTF32 on the tensor
//               cores for b > 16, else FP32 SIMT);
//   Eq. (4)     Omega_hat_11 = R_hat11 R11^{-1} row by row, B(0:bb, trail) -= Omega_hat_11 R12.
// FP32 storage (the mixed form); the rank guard of the single-matrix path applies per matrix.
#include "tc_common.cuh"

namespace rq {

struct BatchDesc {
    float* A;
    int32_t* jpvt;
    double* tau;
    long long* rank;  // pivots before the rank guard fired; -1 when the sketch is not finite
    long long m, n, k, lda;
    int b, tiles;  // tiles: RQRCP_TILES_* choices of the contractions' tile shapes (0 = default rules)
};

namespace {

constexpr int BT = 512;          // threads per block
constexpr int NW = BT / 32;      // warps
constexpr int SW = 8;            // sub-panel width of the panel factorization
constexpr int kTile = 64;        // GEMM tile edge
constexpr int kKu = 64;          // largest K of the update contraction (b <= 64)
constexpr int kLdT = kTile + 1;  // padded shared-memory tile stride

struct Smem {
    float* G;       // union: the panel's sub-panel S, or the contractions' ring / tiles
    uint64_t* mbar; // two mbarriers: tensor-core MMA completion per accumulator buffer
    int* mph;       // completed phases of the two mbarriers
    uint32_t tmem;  // tensor memory of the block (kTmemCols columns)
    int tc;         // 1: the sketch and the trailing update on the tensor cores
    float* S;       // SW x m_max sub-panel
    double* nu;     // n_max sketch norms
    double* Tm;     // b_max x b_max: T, then Omega_hat_11
    float* Xs;      // kKu x kLdT GEMM tile (inside G)
    float* Cs;      // kKu x kLdT GEMM tile (inside G)
    float* vs;      // l_max reflector of the pivot search
    double* red;    // NW x SW block-reduction scratch
    double* sc;     // scalars: tau, beta, scal, guard, ...
    float* scf;     // FP32 coefficients of the panel's rank-1 steps
    int* piv;       // b_max pivot targets
    long long* lpos;
};

__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float x)
{
    const float t = hi + x;
    const float z = t - hi;
    lo += (hi - (t - z)) + (x - z);
    hi = t;
}

// Dot2 step (Ogita, Rump and Oishi, "Accurate sum and dot product", 2005): the product's
// rounding error (by FMA) and the sum's (TwoSum) go into lo, so hi + lo carries a sum of exact
// FP32 products to about twice FP32 precision, with no FP64 arithmetic per term.
__device__ __forceinline__ void dot2_acc(float& hi, float& lo, float x, float y)
{
    const float p = x * y;
    const float pe = fmaf(x, y, -p);
    const float t = hi + p;
    const float z = t - hi;
    lo += ((hi - (t - z)) + (p - z)) + pe;
    hi = t;
}

// Sum of NV float-pair (hi + lo) values over the block, in fixed order: pairs are combined
// across each warp with TwoSum (no FP64 instruction on 32 lanes), the NV warp totals by NV
// threads in FP64.  out[i] (FP64) and, scaled by scale[i] when scale is given, outf[i] = (float)
// (scale_i * out[i]) are visible to every thread on return.
template <int NV>
__device__ void block_sum2(float (&h)[NV], float (&l)[NV], double* red, double* out, const double* scale = nullptr,
                           float* outf = nullptr)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < NV; ++i) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float oh = __shfl_xor_sync(0xffffffffu, h[i], o);
            const float ol = __shfl_xor_sync(0xffffffffu, l[i], o);
            const float t = h[i] + oh;
            const float z = t - h[i];
            l[i] += ol + ((h[i] - (t - z)) + (oh - z));
            h[i] = t;
        }
    }
    if (lane == 0)
#pragma unroll
        for (int i = 0; i < NV; ++i) red[w * NV + i] = (double)h[i] + (double)l[i];
    __syncthreads();
    if (threadIdx.x < NV) {
        double s = 0.0;
        for (int ww = 0; ww < NW; ++ww) s += red[ww * NV + threadIdx.x];
        out[threadIdx.x] = s;
        if (outf) outf[threadIdx.x] = (float)(scale[threadIdx.x] * s);
    }
    __syncthreads();
}

// Asynchronous 4-byte global -> shared copies (cp.async), grouped per K-slice.
__device__ __forceinline__ void cp_async4(float* dst, const float* src)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Ring of K-slices for the contractions: kRing stages, the largest being the 32 x 32 X slice
// plus the 32 x 256 C slice.
constexpr int kRing = 4;
constexpr int kStageFloats = 32 * (32 + 256);
constexpr int kGemmFloats = kRing * kStageFloats;

// Out(M x N) = X^T C; X is K x M (ldx), C is K x N (ldc), column-major.  maskX / maskC: unit-
// lower reflector structure of X / of the first maskC columns of C.  out_rowmajor stores
// Out(r, c) at r*ldo + c, else at c*ldo + r.  Output tiles are RT x CT (RT * CT = 8192: 16 x 512,
// 32 x 256 or 64 x 128, the smallest RT >= M when M <= 32, so a short X wastes no rows); every
// thread owns a 4 x 4 block of them.  K is consumed in KS-deep slices that stream through a ring
// of kRing shared-memory stages by cp.async, kRing - 1 slices in flight while one is multiplied
// (a single block per SM has to keep that many bytes moving on its own).  A slice is stored
// k-major with the element (k, j) of row k at j ^ k: the copies (lanes along k) then hit distinct
// banks, and a thread reads its 4 rows and its 4 columns as two 16-byte words whose lanes are
// permuted by the low bits of k.  Interior slices copy from per-thread base pointers; slices that
// touch an edge or the unit-lower structure take the checked path, which stores the entries that
// structure fixes (0 or 1) directly.  Up to 64 terms are summed in FP32 and folded into a
// compensated (TwoSum) total.
template <int RT>
__device__ void blk_gemm_tn_rt(const float* X, long long ldx, int maskX, const float* C, long long ldc, long long maskC,
                               long long M, long long N, long long K, float* Out, long long ldo, int out_rowmajor,
                               const Smem& sm)
{
    constexpr int CT = 8192 / RT;
    constexpr int KS = RT == 16 ? 16 : 32;
    constexpr int SX = KS * RT, STG = KS * (RT + CT);
    constexpr int PX = (KS * RT + BT - 1) / BT, PC = (KS * CT) / BT;
    constexpr int CPI = BT / KS;  // rows / columns one pass of the block copies
    constexpr int FOLD = 64 / KS;  // slices per FP32 partial sum
    static_assert(STG <= kStageFloats, "stage exceeds the ring's stage size");
    static_assert(KS <= RT && KS <= CT, "the k-swizzle must stay inside a row");
    float* ring = sm.G;
    const int tid = threadIdx.x, tm = tid % (RT / 4), tn = tid / (RT / 4);
    const int ck = tid % KS, cm = tid / KS;  // this thread's copy coordinates in a slice
    const long long nsl = (K + KS - 1) / KS;
    const long long xstep = (long long)CPI * ldx, cstep = (long long)CPI * ldc;
    for (long long m0 = 0; m0 < M; m0 += RT)
        for (long long n0 = 0; n0 < N; n0 += CT) {
            const float* xsrc = X + (m0 + cm) * ldx + ck;
            const float* csrc = C + (n0 + cm) * ldc + ck;
            const bool inner = m0 + RT <= M && n0 + CT <= N;
            // copy slice j into stage j % kRing (one commit group per slice, possibly empty)
            auto issue = [&](long long j) {
                if (j < nsl) {
                    float* Xs = ring + (j % kRing) * STG;
                    float* Cs = Xs + SX;
                    const long long k0 = j * KS;
                    if (inner && k0 + KS <= K && (!maskX || k0 >= m0 + RT) && (n0 >= maskC || k0 >= maskC)) {
#pragma unroll
                        for (int it = 0; it < PX; ++it) {
                            const int mm = cm + it * CPI;
                            if (PX * BT == KS * RT || mm < RT) cp_async4(Xs + ck * RT + (mm ^ ck), xsrc + it * xstep + k0);
                        }
#pragma unroll
                        for (int it = 0; it < PC; ++it) {
                            const int mm = cm + it * CPI;
                            cp_async4(Cs + ck * CT + (mm ^ ck), csrc + it * cstep + k0);
                        }
                    } else {
#pragma unroll
                        for (int it = 0; it < PX; ++it) {
                            const int mm = cm + it * CPI;
                            if (mm < RT) {
                                const long long q = k0 + ck, r = m0 + mm;
                                float* dst = Xs + ck * RT + (mm ^ ck);
                                if (q >= K || r >= M) *dst = 0.f;
                                else if (maskX && q <= r) *dst = q == r ? 1.f : 0.f;
                                else cp_async4(dst, X + r * ldx + q);
                            }
                        }
#pragma unroll
                        for (int it = 0; it < PC; ++it) {
                            const int mm = cm + it * CPI;
                            const long long q = k0 + ck, c = n0 + mm;
                            float* dst = Cs + ck * CT + (mm ^ ck);
                            if (q >= K || c >= N) *dst = 0.f;
                            else if (c < maskC && q <= c) *dst = q == c ? 1.f : 0.f;
                            else cp_async4(dst, C + c * ldc + q);
                        }
                    }
                }
                cp_async_commit();
            };
            float acc[4][4], hi[4][4], lo[4][4];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] = hi[a][b] = lo[a][b] = 0.f;
#pragma unroll
            for (int j = 0; j < kRing - 1; ++j) issue(j);
            int slice = 0;
            for (long long j = 0; j < nsl; ++j) {
                cp_async_wait<kRing - 2>();  // this thread's copies of slice j have landed
                __syncthreads();             // everyone's have; stage (j - 1) % kRing is free
                issue(j + kRing - 1);
                const float* Xs = ring + (j % kRing) * STG;
                const float* Cs = Xs + SX;
#pragma unroll
                for (int kk = 0; kk < KS; ++kk) {
                    const float4 xv = *reinterpret_cast<const float4*>(Xs + kk * RT + ((4 * tm) ^ (kk & ~3)));
                    const float4 cv = *reinterpret_cast<const float4*>(Cs + kk * CT + ((4 * tn) ^ (kk & ~3)));
                    const float xr[4] = {xv.x, xv.y, xv.z, xv.w}, cr[4] = {cv.x, cv.y, cv.z, cv.w};
#pragma unroll
                    for (int a = 0; a < 4; ++a)
#pragma unroll
                        for (int b = 0; b < 4; ++b)
                            acc[a][b] = fmaf(xr[a ^ (kk & 3)], cr[b ^ (kk & 3)], acc[a][b]);
                }
                if (++slice == FOLD) {
                    slice = 0;
#pragma unroll
                    for (int a = 0; a < 4; ++a)
#pragma unroll
                        for (int b = 0; b < 4; ++b) {
                            two_sum_acc(hi[a][b], lo[a][b], acc[a][b]);
                            acc[a][b] = 0.f;
                        }
                }
            }
            cp_async_wait<0>();
            __syncthreads();  // the ring is reused by the next tile
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    two_sum_acc(hi[a][b], lo[a][b], acc[a][b]);
                    const long long r = m0 + 4 * tm + a, c = n0 + 4 * tn + b;
                    if (r < M && c < N) {
                        const float v = hi[a][b] + lo[a][b];
                        if (out_rowmajor) Out[r * ldo + c] = v;
                        else Out[c * ldo + r] = v;
                    }
                }
        }
}

// ---- tensor-core form of the contraction (tcgen05, 3xTF32) ----
// Out(M x N) = X^T C as D = C^T X on the tensor cores, one 128-column tile of C at a time: the
// MMA's A operand is a 128 x 32 chunk of C (lane = column c, K = 32 rows), its B operand the
// NB x 32 chunk of X (NB = M rounded up to 16), both K-major with the 128-byte swizzle in shared
// memory.  cp.async writes each chunk's raw FP32 values straight into their swizzled places (the
// unit-lower structure and the edges by direct stores); a pass over the stage then splits every
// value in place into x_hi = tf32(x) and, next to it, x_lo = tf32(x - x_hi).  B is [X_hi; X_lo]
// (2 NB lines), so a chunk is eight MMAs of N = 2 NB: A_lo first, then A_hi, against both halves
// (all four products; lo lo is below the others' rounding).  The accumulator (double-buffered in
// tensor memory) only ever holds one chunk's products; each is read back by all 16 warps (warp w:
// lane quarter w % 4, column quarter w / 4) and summed in FP32 registers, with a compensated fold
// every 16 chunks, as in the single-matrix 3xTF32 contraction.  Every wait is bounded.
constexpr int kTmemCols = 512;
constexpr int kTcA = 128 * 32 * 4;  // one 128-line x 32-element TF32 tile (16 KB)
constexpr int kTcNbMax = 96;
constexpr int kTcRing = 3;
__host__ __device__ constexpr int tc_stage_bytes(int nb) { return 2 * kTcA + 2 * nb * 128; }

// Byte offset of element (line, k) of a K-major tile of 32-element (128-byte) lines with the
// 128-byte swizzle: 16-byte piece k / 4 of line `line` sits at piece (k / 4) ^ (line % 8).
__device__ __forceinline__ int sw128(int line, int k)
{
    return line * 128 + ((((k >> 2) ^ line) & 7) << 4) + ((k & 3) << 2);
}

template <int CQ>
__device__ bool blk_gemm_tn_tc(const float* X, long long ldx, int maskX, const float* C, long long ldc, long long maskC,
                               long long M, long long N, long long K, float* Out, long long ldo, int out_rowmajor,
                               const Smem& sm)
{
    using namespace tc;
    constexpr int NB = 4 * CQ;
    constexpr int SB = tc_stage_bytes(NB);
    constexpr int XO = 2 * kTcA;  // offset of [X_hi; X_lo] in a stage
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // the ring starts at the first 1024-byte boundary of the region (the swizzle atoms)
    unsigned char* ring = reinterpret_cast<unsigned char*>(sm.G) + ((1024u - (su32(sm.G) & 1023u)) & 1023u);
    const long long nsl = (K + 31) / 32;
    uint32_t ph[2] = {(uint32_t)sm.mph[0], (uint32_t)sm.mph[1]};
    const uint32_t idesc = idesc_tf32(128, 2 * NB);
    const int qd = warp & 3, hd = warp >> 2;  // drain: lane quarter, column quarter
    const int kk = tid & 31, l0 = tid >> 5;   // copies: k of the chunk, first line
    bool ok = true;
    uint32_t g = 0;  // chunks issued in this call: accumulator buffer g & 1
    for (long long n0 = 0; n0 < N && ok; n0 += 128) {
        auto issue = [&](long long j) {
            if (j < nsl) {
                unsigned char* st = ring + (j % kTcRing) * SB;
                const long long q = j * 32 + kk;
#pragma unroll
                for (int it = 0; it < 8; ++it) {
                    const int cl = l0 + 16 * it;
                    const long long c = n0 + cl;
                    float* dst = reinterpret_cast<float*>(st + sw128(cl, kk));
                    if (q >= K || c >= N) *dst = 0.f;
                    else if (c < maskC && q <= c) *dst = q == c ? 1.f : 0.f;
                    else cp_async4(dst, C + c * ldc + q);
                }
#pragma unroll
                for (int it = 0; it < NB / 16; ++it) {
                    const int r = l0 + 16 * it;
                    float* dst = reinterpret_cast<float*>(st + XO + sw128(r, kk));
                    if (q >= K || r >= M) *dst = 0.f;
                    else if (maskX && q <= r) *dst = q == r ? 1.f : 0.f;
                    else cp_async4(dst, X + (long long)r * ldx + q);
                }
            }
            cp_async_commit();
        };
        float acc[CQ], sum[CQ];
#pragma unroll
        for (int j = 0; j < CQ; ++j) acc[j] = sum[j] = 0.f;
        // read back chunk gg's products (both halves) and add them to acc
        auto drain = [&](uint32_t gg) -> bool {
            const int b = (int)(gg & 1u);
            const bool w_ok = mbar_wait(&sm.mbar[b], ph[b] & 1u, nullptr);
            ++ph[b];
            if (__syncthreads_or(w_ok ? 0 : 1)) return false;
            fence_after();
            const uint32_t tb = sm.tmem + ((uint32_t)(32 * qd) << 16) + (uint32_t)(b * 2 * NB + hd * CQ);
            // groups of up to 8 columns: both halves' loads in flight, one wait per group
#pragma unroll
            for (int g0 = 0; g0 < CQ; g0 += 8) {
                uint32_t rh[8], rl[8];
#pragma unroll
                for (int c0 = 0; c0 < 8; c0 += 4) {
                    if (g0 + c0 < CQ) {
                        asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                                     : "=r"(rh[c0]), "=r"(rh[c0 + 1]), "=r"(rh[c0 + 2]), "=r"(rh[c0 + 3])
                                     : "r"(tb + (uint32_t)(g0 + c0)));
                        asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                                     : "=r"(rl[c0]), "=r"(rl[c0 + 1]), "=r"(rl[c0 + 2]), "=r"(rl[c0 + 3])
                                     : "r"(tb + (uint32_t)(NB + g0 + c0)));
                    }
                }
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    if (g0 + u < CQ) acc[g0 + u] += __uint_as_float(rl[u]) + __uint_as_float(rh[u]);
            }
            fence_before();
            return true;
        };
        auto fold = [&]() {  // (sum, acc) = TwoSum(sum, acc)
#pragma unroll
            for (int j = 0; j < CQ; ++j) {
                const float t = sum[j] + acc[j];
                const float z = t - sum[j];
                acc[j] = (sum[j] - (t - z)) + (acc[j] - z);
                sum[j] = t;
            }
        };
        issue(0);
        issue(1);
        long long j = 0;
        for (; j < nsl; ++j) {
            cp_async_wait<1>();  // this thread's copies of chunk j have landed
            __syncthreads();
            unsigned char* st = ring + (j % kTcRing) * SB;
            for (int e = tid; e < 1024 + NB * 8; e += BT) {
                float4* p = e < 1024 ? reinterpret_cast<float4*>(st) + e : reinterpret_cast<float4*>(st + XO) + (e - 1024);
                float4* pl = e < 1024 ? p + 1024 : p + NB * 8;
                const float4 v = *p;
                float4 hv, lv;
                hv.x = tf32_rn(v.x);
                hv.y = tf32_rn(v.y);
                hv.z = tf32_rn(v.z);
                hv.w = tf32_rn(v.w);
                lv.x = tf32_rn(v.x - hv.x);
                lv.y = tf32_rn(v.y - hv.y);
                lv.z = tf32_rn(v.z - hv.z);
                lv.w = tf32_rn(v.w - hv.w);
                *p = hv;
                *pl = lv;
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncthreads();
            if (tid == 0) {
                fence_after();
                const int b = (int)(g & 1u);
                const uint64_t da = umma_desc(st), dal = umma_desc(st + kTcA), dx = umma_desc(st + XO);
                const uint32_t td = sm.tmem + (uint32_t)(b * 2 * NB);
#pragma unroll
                for (int k = 0; k < 4; ++k) mma_tf32_ss(td, dal + 2 * k, dx + 2 * k, idesc, k > 0 ? 1 : 0);
#pragma unroll
                for (int k = 0; k < 4; ++k) mma_tf32_ss(td, da + 2 * k, dx + 2 * k, idesc, 1);
                mma_commit(&sm.mbar[b]);
            }
            ++g;
            if (j > 0) {
                if (!drain(g - 2)) {
                    ok = false;
                    break;
                }
                if (j % 16 == 0) fold();
            }
            issue(j + 2);  // into the stage chunk j - 1 used; its MMAs have completed
        }
        if (ok && nsl > 0 && !drain(g - 1)) ok = false;
        cp_async_wait<0>();
        __syncthreads();
        if (!ok) break;
        fold();
        const long long c = n0 + 32 * qd + lane;
#pragma unroll
        for (int jj = 0; jj < CQ; ++jj) {
            const long long r = hd * CQ + jj;
            if (r < M && c < N) {
                const float v = sum[jj] + acc[jj];
                if (out_rowmajor) Out[r * ldo + c] = v;
                else Out[c * ldo + r] = v;
            }
        }
    }
    __syncthreads();
    if (tid == 0) {
        sm.mph[0] = (int)ph[0];
        sm.mph[1] = (int)ph[1];
    }
    __syncthreads();
    return ok;
}

// tensor == 1 and M <= kTcNbMax: the tensor-core form; false only if a tensor-core wait timed
// out.  The sketch (Omega shared by all blocks, resident in L2; M = b + p rows would waste up to
// half of a SIMT tile) runs on the tensor cores; the Gram V^T [V C] stays on the SIMT form, which
// keeps more bytes in flight per block than the tensor-core stages (raw, hi and lo parts) allow.
__device__ bool blk_gemm_tn(const float* X, long long ldx, int maskX, const float* C, long long ldc, long long maskC,
                            long long M, long long N, long long K, float* Out, long long ldo, int out_rowmajor,
                            const Smem& sm, int tensor, int rt_min = 0)
{
    if (M <= 0 || N <= 0) return true;
    if (tensor && M <= kTcNbMax) {
        switch ((int)((M + 15) / 16)) {
        case 1: return blk_gemm_tn_tc<4>(X, ldx, maskX, C, ldc, maskC, M, N, K, Out, ldo, out_rowmajor, sm);
        case 2: return blk_gemm_tn_tc<8>(X, ldx, maskX, C, ldc, maskC, M, N, K, Out, ldo, out_rowmajor, sm);
        case 3: return blk_gemm_tn_tc<12>(X, ldx, maskX, C, ldc, maskC, M, N, K, Out, ldo, out_rowmajor, sm);
        case 4: return blk_gemm_tn_tc<16>(X, ldx, maskX, C, ldc, maskC, M, N, K, Out, ldo, out_rowmajor, sm);
        case 5: return blk_gemm_tn_tc<20>(X, ldx, maskX, C, ldc, maskC, M, N, K, Out, ldo, out_rowmajor, sm);
        default: return blk_gemm_tn_tc<24>(X, ldx, maskX, C, ldc, maskC, M, N, K, Out, ldo, out_rowmajor, sm);
        }
    }
    // the smallest RT >= M (and >= rt_min): RT x (8192 / RT) output tiles
    const long long Mr = M > rt_min ? M : rt_min;
    if (Mr <= 16) blk_gemm_tn_rt<16>(X, ldx, maskX, C, ldc, maskC, M, N, K, Out, ldo, out_rowmajor, sm);
    else if (Mr <= 32) blk_gemm_tn_rt<32>(X, ldx, maskX, C, ldc, maskC, M, N, K, Out, ldo, out_rowmajor, sm);
    else blk_gemm_tn_rt<64>(X, ldx, maskX, C, ldc, maskC, M, N, K, Out, ldo, out_rowmajor, sm);
    return true;
}

// C(M x N) -= V(M x K) Y(K x N), column-major, K <= 64; V with the optional unit-lower
// structure.  64 x 128 tiles, rows of tiles outermost; each tile's C block, Y block and V band
// stream through a ring of NST shared-memory stages by cp.async (V and Y come from L2), so
// NST - 1 tiles are in flight while one is multiplied.  Lane l of warp w owns rows l, l + 32 and
// columns 8w..8w+7 of the tile, so its C entries are written back 128 bytes per warp store.
// C is kept [col][row], V [k][row], Y [k][col] with the element (k, c) at c ^ k, which spreads
// the copies (lanes along k) over the banks and lets a warp read its eight columns as two
// 16-byte words, permuted by the low bits of k.  K is zero-padded to K4, a multiple of 4; a stage
// holds 8192 + 192 K4 floats, three of them when they fit in kURingFloats, else two.
constexpr int kUR = 64, kUC = 128;
constexpr int kURingFloats = 3 * (kUR * kUC + 32 * (kUR + kUC));
static_assert(kTcRing * tc_stage_bytes(kTcNbMax) <= kURingFloats * 4, "tensor-core ring exceeds the shared region");

template <int NST>
__device__ void blk_gemm_update_n(float* C, long long ldc, const float* V, long long ldv, int maskV, const float* Y,
                                  long long ldy, long long M, long long N, long long K, int K4, const Smem& sm)
{
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const long long nrt = (M + kUR - 1) / kUR, nct = (N + kUC - 1) / kUC;
    const long long ntile = nrt * nct;
    const int SF = kUR * kUC + K4 * (kUR + kUC);
    int klog = 2;
    while ((1 << klog) < K4) ++klog;
    const int kmask = (1 << klog) - 1;  // K slots of the Y copy (a power of two >= K4)
    float* ring = sm.G;
    const int rr = tid & (kUR - 1), cc0 = tid / kUR;
    auto issue = [&](long long t) {
        if (t < ntile) {
            float* Cs = ring + (t % NST) * SF;
            float* Ys = Cs + kUR * kUC;
            float* Vs = Ys + K4 * kUC;
            const long long r0 = (t / nct) * kUR, c0 = (t % nct) * kUC;
            // C block, rows fastest
            if (r0 + kUR <= M && c0 + kUC <= N) {
                const float* src = C + (c0 + cc0) * ldc + r0 + rr;
                const long long step = (long long)(BT / kUR) * ldc;
#pragma unroll
                for (int it = 0; it < kUR * kUC / BT; ++it)
                    cp_async4(Cs + (cc0 + it * (BT / kUR)) * kUR + rr, src + it * step);
            } else {
#pragma unroll
                for (int it = 0; it < kUR * kUC / BT; ++it) {
                    const int cc = cc0 + it * (BT / kUR);
                    const long long r = r0 + rr, c = c0 + cc;
                    float* dst = Cs + cc * kUR + rr;
                    if (r < M && c < N) cp_async4(dst, C + c * ldc + r);
                    else *dst = 0.f;
                }
            }
            // V band, rows fastest
            for (int kk = cc0; kk < K4; kk += BT / kUR) {
                const long long r = r0 + rr;
                float* dst = Vs + kk * kUR + rr;
                if (kk >= K || r >= M) *dst = 0.f;
                else if (maskV && r <= kk) *dst = r == kk ? 1.f : 0.f;
                else cp_async4(dst, V + (long long)kk * ldv + r);
            }
            // Y block, K fastest
            {
                const int kk = tid & kmask;
                if (kk < K4)
                    for (int cc = tid >> klog; cc < kUC; cc += BT >> klog) {
                        const long long c = c0 + cc;
                        float* dst = Ys + kk * kUC + (cc ^ kk);
                        if (kk < K && c < N) cp_async4(dst, Y + c * ldy + kk);
                        else *dst = 0.f;
                    }
            }
        }
        cp_async_commit();
    };
#pragma unroll
    for (int j = 0; j < NST - 1; ++j) issue(j);
    for (long long t = 0; t < ntile; ++t) {
        cp_async_wait<NST - 2>();
        __syncthreads();
        issue(t + NST - 1);
        const float* Cs = ring + (t % NST) * SF;
        const float* Ys = Cs + kUR * kUC;
        const float* Vs = Ys + K4 * kUC;
        const long long r0 = (t / nct) * kUR, c0 = (t % nct) * kUC;
        float acc[2][8];
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int b = 0; b < 8; ++b) acc[a][b] = 0.f;
        for (int k0 = 0; k0 < K4; k0 += 4) {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int kk = k0 + u;
                const float va[2] = {Vs[kk * kUR + lane], Vs[kk * kUR + lane + 32]};
                const float4 y0 = *reinterpret_cast<const float4*>(Ys + kk * kUC + ((8 * w) ^ k0));
                const float4 y1 = *reinterpret_cast<const float4*>(Ys + kk * kUC + ((8 * w + 4) ^ k0));
                const float yr[8] = {y0.x, y0.y, y0.z, y0.w, y1.x, y1.y, y1.z, y1.w};
#pragma unroll
                for (int a = 0; a < 2; ++a)
#pragma unroll
                    for (int b = 0; b < 4; ++b) {
                        acc[a][b] = fmaf(va[a], yr[b ^ u], acc[a][b]);
                        acc[a][4 + b] = fmaf(va[a], yr[4 + (b ^ u)], acc[a][4 + b]);
                    }
            }
        }
#pragma unroll
        for (int b = 0; b < 8; ++b)
#pragma unroll
            for (int a = 0; a < 2; ++a) {
                const int r_ = lane + 32 * a, cc = 8 * w + b;
                const long long r = r0 + r_, c = c0 + cc;
                if (r < M && c < N) C[c * ldc + r] = Cs[cc * kUR + r_] - acc[a][b];
            }
    }
    cp_async_wait<0>();
    __syncthreads();  // the ring is reused by whatever follows
}

__device__ void blk_gemm_update(float* C, long long ldc, const float* V, long long ldv, int maskV, const float* Y,
                                long long ldy, long long M, long long N, long long K, const Smem& sm)
{
    if (M <= 0 || N <= 0) return;
    const int K4 = (int)((K + 3) & ~3LL);
    const int SF = kUR * kUC + K4 * (kUR + kUC);
    if (3 * SF <= kURingFloats) blk_gemm_update_n<3>(C, ldc, V, ldv, maskV, Y, ldy, M, N, K, K4, sm);
    else blk_gemm_update_n<2>(C, ldc, V, ldv, maskV, Y, ldy, M, N, K, K4, sm);
}

// Tensor-core form of C(M x N) -= V(M x K) Y(K x N) (K <= 64, V with the optional unit-lower
// structure), 3xTF32 with all four products: 128 x 64 tiles of C, rows of tiles outermost.  The
// MMA's A operand is the 128-row band of V (K-major, 128-byte swizzle, KB = ceil(K / 32) blocks of
// 32 K), copied once per band and split in place into V_hi with V_lo next to it; B is the tile's
// [Y_hi; Y_lo] (128 lines: 64 columns of hi parts, then 64 of lo parts), double-buffered, so the
// copy of the next tile's Y overlaps this tile.  Per tile one thread issues 8 KB MMAs (A_lo, then
// A_hi, against [Y_hi; Y_lo], N = 128) into one of two accumulator buffers in tensor memory.  C
// never passes through shared memory: each thread loads its 16 entries of the next tile into
// registers while the current tile is multiplied (a second tile ahead measured slower), and the
// epilogue (warp w: lane quarter w % 4,
// columns 16 (w / 4) .. + 15) writes C - (D_hi + D_lo) back with 128-byte warp stores.
template <int KB>
__device__ bool blk_gemm_update_tc(float* C, long long ldc, const float* V, long long ldv, int maskV, const float* Y,
                                   long long ldy, long long M, long long N, long long K, const Smem& sm)
{
    using namespace tc;
    constexpr int kTR = 128, kTC = 64;
    constexpr int A_BYTES = 2 * kTcA;                 // hi + lo of one 32-K block of the V band
    constexpr int B_BYTES = kTC * 2 * 128;            // [Y_hi; Y_lo] of one 32-K block (16 KB)
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    unsigned char* base = reinterpret_cast<unsigned char*>(sm.G) + ((1024u - (su32(sm.G) & 1023u)) & 1023u);
    unsigned char* Ab = base;                          // KB blocks of A_BYTES
    unsigned char* Bb = base + KB * A_BYTES;           // 2 buffers x KB blocks of B_BYTES
    auto bblk = [&](int buf, int kb) { return Bb + (buf * KB + kb) * B_BYTES; };
    const int ksteps = (int)((K + 7) / 8);
    const uint32_t idesc = idesc_tf32(128, 2 * kTC);
    uint32_t ph[2] = {(uint32_t)sm.mph[0], (uint32_t)sm.mph[1]};
    const int qd = warp & 3, hd = warp >> 2;
    const int er = 32 * qd + lane;                     // epilogue row of the tile
    bool ok = true;
    uint32_t g = 0;                                    // tiles issued: accumulator buffer g & 1
    const long long nct = (N + kTC - 1) / kTC;
    for (long long r0 = 0; r0 < M && ok; r0 += kTR) {
        // ---- V band: copy (lanes along rows), then split in place
        for (int e = tid; e < kTR * 32 * KB; e += BT) {
            const int r = e & (kTR - 1), k = e >> 7;
            const long long row = r0 + r;
            float* dst = reinterpret_cast<float*>(Ab + (k >> 5) * A_BYTES + sw128(r, k & 31));
            if (k >= K || row >= M) *dst = 0.f;
            else if (maskV && row <= k) *dst = row == k ? 1.f : 0.f;
            else cp_async4(dst, V + (long long)k * ldv + row);
        }
        cp_async_commit();
        auto issue_y = [&](long long t, int buf) {
            if (t < nct) {
                const long long c0 = t * kTC;
                for (int e = tid; e < kTC * 32 * KB; e += BT) {
                    const int k = e & 31, c = (e >> 5) & (kTC - 1), kb = e >> 11;
                    const long long kk = kb * 32 + k, col = c0 + c;
                    float* dst = reinterpret_cast<float*>(bblk(buf, kb) + sw128(c, k));
                    if (kk < K && col < N) cp_async4(dst, Y + col * ldy + kk);
                    else *dst = 0.f;
                }
            }
            cp_async_commit();
        };
        auto load_c = [&](long long t, float (&cv)[16]) {
            const long long row = r0 + er, c0 = t * kTC + 16 * hd;
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const long long col = c0 + j;
                cv[j] = (t < nct && row < M && col < N) ? C[col * ldc + row] : 0.f;
            }
        };
        auto split = [&](unsigned char* blk, int nf4, int lo_off) {  // nf4 float4 of hi, lo at + lo_off bytes
            for (int e = tid; e < nf4; e += BT) {
                float4* p = reinterpret_cast<float4*>(blk) + e;
                float4* pl = reinterpret_cast<float4*>(blk + lo_off) + e;
                const float4 v = *p;
                float4 hv, lv;
                hv.x = tf32_rn(v.x); hv.y = tf32_rn(v.y); hv.z = tf32_rn(v.z); hv.w = tf32_rn(v.w);
                lv.x = tf32_rn(v.x - hv.x); lv.y = tf32_rn(v.y - hv.y);
                lv.z = tf32_rn(v.z - hv.z); lv.w = tf32_rn(v.w - hv.w);
                *p = hv;
                *pl = lv;
            }
        };
        issue_y(0, 0);
        float cp_[16], cn[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) cp_[j] = 0.f;
        load_c(0, cn);
        cp_async_wait<1>();  // the V band has landed
        __syncthreads();
#pragma unroll
        for (int kb = 0; kb < KB; ++kb) split(Ab + kb * A_BYTES, kTcA / 16, kTcA);
        // epilogue of tile tt (accumulator buffer gg & 1) with C values cv
        auto epilogue = [&](long long tt, uint32_t gg, const float (&cv)[16]) -> bool {
            const int b = (int)(gg & 1u);
            const bool w_ok = mbar_wait(&sm.mbar[b], ph[b] & 1u, nullptr);
            ++ph[b];
            if (__syncthreads_or(w_ok ? 0 : 1)) return false;
            fence_after();
            const uint32_t tb = sm.tmem + ((uint32_t)(32 * qd) << 16) + (uint32_t)(b * 2 * kTC + 16 * hd);
            uint32_t dh[16], dl[16];
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                : "=r"(dh[0]), "=r"(dh[1]), "=r"(dh[2]), "=r"(dh[3]), "=r"(dh[4]), "=r"(dh[5]), "=r"(dh[6]),
                  "=r"(dh[7]), "=r"(dh[8]), "=r"(dh[9]), "=r"(dh[10]), "=r"(dh[11]), "=r"(dh[12]), "=r"(dh[13]),
                  "=r"(dh[14]), "=r"(dh[15])
                : "r"(tb));
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                : "=r"(dl[0]), "=r"(dl[1]), "=r"(dl[2]), "=r"(dl[3]), "=r"(dl[4]), "=r"(dl[5]), "=r"(dl[6]),
                  "=r"(dl[7]), "=r"(dl[8]), "=r"(dl[9]), "=r"(dl[10]), "=r"(dl[11]), "=r"(dl[12]), "=r"(dl[13]),
                  "=r"(dl[14]), "=r"(dl[15])
                : "r"(tb + (uint32_t)kTC));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            fence_before();
            const long long row = r0 + er, c0 = tt * kTC + 16 * hd;
            if (row < M)
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const long long col = c0 + j;
                    if (col < N) C[col * ldc + row] = cv[j] - (__uint_as_float(dl[j]) + __uint_as_float(dh[j]));
                }
            return true;
        };
        for (long long t = 0; t < nct; ++t) {
            const int buf = (int)(t & 1);
            cp_async_wait<0>();  // this thread's copies of Y(t) (and of the band) have landed
            __syncthreads();
#pragma unroll
            for (int kb = 0; kb < KB; ++kb) split(bblk(buf, kb), kTC * 8, kTC * 128);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncthreads();
            if (tid == 0) {
                fence_after();
                const uint32_t td = sm.tmem + (uint32_t)((g & 1u) * 2 * kTC);
                int first = 1;
                for (int half = 0; half < 2; ++half)  // A_lo, then A_hi
#pragma unroll
                    for (int kb = 0; kb < KB; ++kb) {
                        const uint64_t da = umma_desc(Ab + kb * A_BYTES + (half == 0 ? kTcA : 0));
                        const uint64_t db = umma_desc(bblk(buf, kb));
#pragma unroll
                        for (int s4 = 0; s4 < 4; ++s4)
                            if (kb * 4 + s4 < ksteps) {
                                mma_tf32_ss(td, da + 2 * s4, db + 2 * s4, idesc, first ? 0 : 1);
                                first = 0;
                            }
                    }
                mma_commit(&sm.mbar[g & 1u]);
            }
            ++g;
            // the previous tile: its product (which also frees Y buffer buf ^ 1), then C - D
            if (t > 0 && !epilogue(t - 1, g - 2, cp_)) {
                ok = false;
                break;
            }
            issue_y(t + 1, buf ^ 1);
#pragma unroll
            for (int j = 0; j < 16; ++j) cp_[j] = cn[j];  // C of tile t for its epilogue
            load_c(t + 1, cn);                             // next tile's C, in flight meanwhile
        }
        if (ok && !epilogue(nct - 1, g - 1, cp_)) ok = false;
        cp_async_wait<0>();
        __syncthreads();
    }
    __syncthreads();
    if (tid == 0) {
        sm.mph[0] = (int)ph[0];
        sm.mph[1] = (int)ph[1];
    }
    __syncthreads();
    return ok;
}

// Order key of a squared norm: non-negative doubles order as their bit patterns read as signed
// 64-bit integers and negative values map below them, so the compares stay off the FP64 pipe.
__device__ __forceinline__ long long nkey(double v)
{
    const long long b = __double_as_longlong(v);
    return b < 0 ? -1LL : b;
}
__device__ __forceinline__ bool beats(double v1, long long p1, double v2, long long p2)
{
    const long long k1 = nkey(v1), k2 = nkey(v2);
    return k1 > k2 || (k1 == k2 && p1 < p2);
}

// argmax over (value, position), ties to the smaller position; result broadcast via sm.sc/lpos.
__device__ void blk_argmax(double v, long long p, const Smem& sm, double& bv, long long& bp)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffffu, v, o);
        const long long op = __shfl_xor_sync(0xffffffffu, p, o);
        if (beats(ov, op, v, p)) { v = ov; p = op; }
    }
    if (lane == 0) { sm.red[w] = v; sm.lpos[w] = p; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double vb = sm.red[0];
        long long pb = sm.lpos[0];
        for (int ww = 1; ww < NW; ++ww)
            if (beats(sm.red[ww], sm.lpos[ww], vb, pb)) { vb = sm.red[ww]; pb = sm.lpos[ww]; }
        sm.sc[8] = vb;
        sm.lpos[NW] = pb;
    }
    __syncthreads();
    bv = sm.sc[8];
    bp = sm.lpos[NW];
    __syncthreads();
}

// Partial QRCP (Alg. 1) on the row-major sketch B (l x n, ld n), trailing columns i..n-1, bb
// steps.  Returns the number of pivots taken (< bb when the rank guard fires).
__device__ int blk_pivot(float* B, long long n, int l, long long i, int bb, int32_t* jpvt, double guard,
                         const Smem& sm)
{
    const int tid = threadIdx.x;
    for (long long c = i + tid; c < n; c += BT) {
        float h = 0.f, lo = 0.f;
        for (int r = 0; r < l; ++r) {
            const float x = B[(long long)r * n + c];
            dot2_acc(h, lo, x, x);
        }
        sm.nu[c] = (double)h + (double)lo;
    }
    __syncthreads();
    for (int t = 0; t < bb; ++t) {
        const long long c0 = i + t;
        double mv = -1.0;
        long long mp = 0x7fffffffffffffffLL;
        for (long long c = c0 + tid; c < n; c += BT)
            if (beats(sm.nu[c], c, mv, mp)) { mv = sm.nu[c]; mp = c; }
        double bv;
        long long j;
        blk_argmax(mv, mp, sm, bv, j);
        if (!(bv > guard)) return t;
        if (tid == 0) sm.piv[t] = (int)j;
        if (j != c0) {
            for (int r = tid; r < l; r += BT) {
                const float a = B[(long long)r * n + c0];
                B[(long long)r * n + c0] = B[(long long)r * n + j];
                B[(long long)r * n + j] = a;
            }
            if (tid == 0) {
                const double tn = sm.nu[c0];
                sm.nu[c0] = sm.nu[j];
                sm.nu[j] = tn;
                const int32_t tj = jpvt[c0];
                jpvt[c0] = jpvt[j];
                jpvt[j] = tj;
            }
        }
        __syncthreads();
        // reflector of B(t:l, c0), FP64, xLARFG convention
        if (tid < 32) {
            double ss = 0.0;
            for (int r = t + 1 + tid; r < l; r += 32) {
                const double x = B[(long long)r * n + c0];
                ss += x * x;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
            double tau, beta, scal;
            warp_larfg((double)B[(long long)t * n + c0], ss, tau, beta, scal);
            if (tid == 0) {
                sm.sc[0] = tau;
                sm.sc[1] = beta;
                sm.sc[2] = scal;
            }
        }
        __syncthreads();
        const double tau = sm.sc[0];
        for (int r = t + 1 + tid; r < l; r += BT) sm.vs[r] = (float)((double)B[(long long)r * n + c0] * sm.sc[2]);
        if (tid == 0) sm.vs[t] = 1.f;
        __syncthreads();
        for (int r = t + tid; r < l; r += BT) B[(long long)r * n + c0] = (r == t) ? (float)sm.sc[1] : 0.f;
        const float tauf = (float)tau;
        const bool refl = tau != 0.0;
        for (long long c = c0 + 1 + tid; c < n; c += BT) {
            float w = 0.f;
            if (refl)
                for (int r = t; r < l; ++r) w = fmaf(sm.vs[r], B[(long long)r * n + c], w);
            const float wt = w * tauf;
            float h = 0.f, lo = 0.f;
            for (int r = t; r < l; ++r) {
                float x = B[(long long)r * n + c];
                if (refl) {
                    x = fmaf(-wt, sm.vs[r], x);
                    B[(long long)r * n + c] = x;
                }
                if (r > t) dot2_acc(h, lo, x, x);
            }
            sm.nu[c] = (double)h + (double)lo;
        }
        __syncthreads();
    }
    return bb;
}

// Householder QR of the panel P (m1 x bb, ldp) in place: left-looking over sub-panels of SW
// columns held in shared memory; tau (FP64) out.
__device__ void blk_panel(float* P, long long ldp, long long m1, int bb, double* tau, const Smem& sm)
{
    const int tid = threadIdx.x;
    for (int s0 = 0; s0 < bb; s0 += SW) {
        const int sw = (bb - s0) < SW ? (bb - s0) : SW;
        for (int cc = 0; cc < sw; ++cc)
            for (long long r = tid; r < m1; r += BT) sm.S[cc * m1 + r] = P[(s0 + cc) * ldp + r];
        __syncthreads();
        // earlier reflectors of this panel, in order
        for (int h = 0; h < s0; ++h) {
            float sh[SW], sl[SW];
#pragma unroll
            for (int cc = 0; cc < SW; ++cc) sh[cc] = sl[cc] = 0.f;
            const float* vh = P + (long long)h * ldp;
            for (long long r = h + tid; r < m1; r += BT) {
                const float x = (r == h) ? 1.f : vh[r];
#pragma unroll
                for (int cc = 0; cc < SW; ++cc)
                    if (cc < sw) dot2_acc(sh[cc], sl[cc], x, sm.S[cc * m1 + r]);
            }
            // coefficients tau_h * (v_h^T S(:, cc)), rounded to FP32 once
            if (tid < SW) sm.sc[32 + tid] = tau[h];
            block_sum2<SW>(sh, sl, sm.red, sm.sc + 16, sm.sc + 32, sm.scf);
            float cf[SW];
#pragma unroll
            for (int cc = 0; cc < SW; ++cc) cf[cc] = sm.scf[cc];
            for (long long r = h + tid; r < m1; r += BT) {
                const float x = (r == h) ? 1.f : vh[r];
#pragma unroll
                for (int cc = 0; cc < SW; ++cc)
                    if (cc < sw) sm.S[cc * m1 + r] -= cf[cc] * x;
            }
            __syncthreads();
        }
        // factor the sub-panel columns
        for (int jj = 0; jj < sw; ++jj) {
            const long long j = s0 + jj;  // panel row/column index of the diagonal
            float sh[SW], sl[SW];
#pragma unroll
            for (int cc = 0; cc < SW; ++cc) sh[cc] = sl[cc] = 0.f;
            for (long long r = j + 1 + tid; r < m1; r += BT) {
                const float x = sm.S[jj * m1 + r];
#pragma unroll
                for (int cc = 0; cc < SW; ++cc)
                    if (cc >= jj && cc < sw) dot2_acc(sh[cc], sl[cc], x, sm.S[cc * m1 + r]);
            }
            block_sum2<SW>(sh, sl, sm.red, sm.sc + 16);
            if (tid < 32) {
                double tj, beta, scal;
                warp_larfg((double)sm.S[jj * m1 + j], sm.sc[16 + jj], tj, beta, scal);
                // lane cc: the FP32 coefficient tau * v^T a_cc of the update of column cc
                if (tid < SW)
                    sm.scf[tid] = (tid > jj && tid < sw)
                                      ? (float)(tj * ((double)sm.S[tid * m1 + j] + scal * sm.sc[16 + tid])) : 0.f;
                if (tid == 0) {
                    sm.sc[0] = tj;
                    sm.sc[1] = beta;
                    sm.sc[2] = scal;
                    tau[j] = tj;
                    sm.scf[SW] = (float)scal;
                }
            }
            __syncthreads();
            if (sm.sc[0] != 0.0) {
                const float scalf = sm.scf[SW];
                float cf[SW];
#pragma unroll
                for (int cc = 0; cc < SW; ++cc) cf[cc] = sm.scf[cc];
                for (long long r = j + 1 + tid; r < m1; r += BT) {
                    const float vr = sm.S[jj * m1 + r] * scalf;
                    sm.S[jj * m1 + r] = vr;
#pragma unroll
                    for (int cc = 0; cc < SW; ++cc)
                        if (cc > jj && cc < sw) sm.S[cc * m1 + r] -= cf[cc] * vr;
                }
                if (tid == 0)
                    for (int cc = jj + 1; cc < sw; ++cc) sm.S[cc * m1 + j] -= cf[cc];
            }
            __syncthreads();
            if (tid == 0) sm.S[jj * m1 + j] = (float)sm.sc[1];
            __syncthreads();
        }
        for (int cc = 0; cc < sw; ++cc)
            for (long long r = tid; r < m1; r += BT) P[(s0 + cc) * ldp + r] = sm.S[cc * m1 + r];
        __syncthreads();
    }
}

// T (bb x bb, FP64, column-major in sm.Tm) from the Gram G(q, j) = W[j*bb + q] and tau.
__device__ void blk_tform(const float* W, int bb, const double* tau, const Smem& sm)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int e = threadIdx.x; e < bb * bb; e += BT) sm.Tm[e] = 0.0;
    __syncthreads();
    for (int r = w; r < bb; r += NW) {
        if (lane == 0) sm.Tm[r * bb + r] = tau[r];
        __syncwarp();
        for (int j = r + 1; j < bb; ++j) {
            double s = 0.0;
            for (int q = r + lane; q < j; q += 32) s += sm.Tm[q * bb + r] * (double)W[(long long)j * bb + q];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) sm.Tm[j * bb + r] = -tau[j] * s;
            __syncwarp();
        }
    }
    __syncthreads();
}

// Omega_hat_11 (bb x bb, FP64, in sm.Tm) from R_hat11 = B(0:bb, i:i+bb) (row-major, ld n) and
// R11 = A(i:i+bb, i:i+bb): row recurrences, one warp per row.
__device__ void blk_bsolve(const float* B, long long n, const float* A, long long lda, long long i, int bb, const Smem& sm)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int e = threadIdx.x; e < bb * bb; e += BT) sm.Tm[e] = 0.0;
    __syncthreads();
    for (int r = w; r < bb; r += NW) {
        for (int j = r; j < bb; ++j) {
            double s = 0.0;
            for (int q = r + lane; q < j; q += 32) s += sm.Tm[q * bb + r] * (double)A[(i + j) * lda + i + q];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) {
                const double rjj = (double)A[(i + j) * lda + i + j];
                sm.Tm[j * bb + r] = (rjj == 0.0) ? 0.0 : ((double)B[(long long)r * n + i + j] - s) / rjj;
            }
            __syncwarp();
        }
    }
    __syncthreads();
}

// Factors one matrix; false if a tensor-core wait timed out (the matrix's rank is then -2).
__device__ bool factor_one(const BatchDesc& d, const float* Om, long long ldo, int p, float* Bw, float* Ww, float* Yw,
                           const Smem& sm)
{
    const int tid = threadIdx.x;
    const long long m = d.m, n = d.n, k = d.k, lda = d.lda;
    const int b = d.b;
    const int l = b + p;
    float* A = d.A;
    for (long long c = tid; c < n; c += BT) d.jpvt[c] = (int32_t)c;
    // sketch B = Omega(0:l, 0:m) A, row-major l x n
    const int tiles = d.tiles;
    if (!blk_gemm_tn(Om, ldo, 0, A, lda, 0, l, n, m, Bw, n, 1, sm, (tiles & RQRCP_TILES_SKETCH_SIMT) ? 0 : sm.tc)) {
        if (tid == 0) *d.rank = -2;
        __syncthreads();
        return false;
    }
    __syncthreads();
    // largest initial sketch column norm^2 and finiteness
    double mx = 0.0;
    bool finite = true;
    for (long long c = tid; c < n; c += BT) {
        float h = 0.f, lo = 0.f;
        for (int r = 0; r < l; ++r) {
            const float x = Bw[(long long)r * n + c];
            dot2_acc(h, lo, x, x);
        }
        const double s = (double)h + (double)lo;
        finite = finite && isfinite(s);
        mx = fmax(mx, s);
    }
    const int all_finite = __syncthreads_and(finite ? 1 : 0);
    double bv;
    long long bp;
    blk_argmax(mx, 0, sm, bv, bp);
    if (!all_finite) {
        if (tid == 0) *d.rank = -1;
        __syncthreads();
        return true;
    }
    const double gtol = 10.0 * sqrt((double)(m > n ? m : n)) * 5.9604644775390625e-08;
    const double guard = gtol * gtol * bv;
    bool pivoting = true;
    long long rank = k;
    for (long long i = 0; i < k; i += b) {
        const int bb = (int)(b < k - i ? b : k - i);
        int steps = 0;
        if (pivoting) {
            steps = blk_pivot(Bw, n, l, i, bb, d.jpvt, guard, sm);
            if (steps < bb) {
                pivoting = false;
                rank = i + steps;
            }
        }
        // swap the chosen columns of A into place, in pivot order
        for (int t = 0; t < steps; ++t) {
            const long long a = i + t, j = sm.piv[t];
            if (j != a)
                for (long long r = tid; r < m; r += BT) {
                    const float x = A[a * lda + r];
                    A[a * lda + r] = A[j * lda + r];
                    A[j * lda + r] = x;
                }
            __syncthreads();
        }
        float* Vp = A + i * lda + i;
        const long long m1 = m - i;
        blk_panel(Vp, lda, m1, bb, d.tau + i, sm);
        const long long nt = n - i - bb;
        if (nt <= 0) continue;
        // W = V^T [V C] (bb x (n-i), column-major ld bb), T, Y = T^T W(:, bb:), C -= V Y
        if (!blk_gemm_tn(Vp, lda, 1, Vp, lda, bb, bb, n - i, m1, Ww, bb, 0, sm, 0,
                         (tiles & RQRCP_TILES_GRAM_RT64) ? 64 : 0)) {
            if (tid == 0) *d.rank = -2;
            __syncthreads();
            return false;
        }
        __syncthreads();
        blk_tform(Ww, bb, d.tau + i, sm);
        {
            // Y = T^T W(:, bb:) in FP32 with FP64-class accuracy: T = Th + Tl (two floats), the
            // products and their sum compensated (Dot2: error-free product by FMA, TwoSum)
            const int ldt = bb + 1;
            float* Th = sm.Xs;                  // [q][r], ldt-padded: lanes (r) read consecutive words
            float* Tl = sm.Xs + kKu * kLdT;     // the Cs half of the GEMM region
            for (int e = tid; e < bb * bb; e += BT) {
                const int q = e % bb, r = e / bb;
                const double tv = q <= r ? sm.Tm[r * bb + q] : 0.0;
                const float h = (float)tv;
                Th[q * ldt + r] = h;
                Tl[q * ldt + r] = (float)(tv - (double)h);
            }
            __syncthreads();
            for (long long e = tid; e < (long long)bb * nt; e += BT) {
                const int r = (int)(e % bb);
                const long long c = e / bb;
                const float* w = Ww + (bb + c) * bb;
                float sacc = 0.f, cmp = 0.f;
                for (int q = 0; q <= r; ++q) {
                    const float wq = w[q], th = Th[q * ldt + r];
                    const float pr = th * wq;
                    const float pe = fmaf(th, wq, -pr);
                    const float t2 = sacc + pr;
                    const float z = t2 - sacc;
                    cmp += ((sacc - (t2 - z)) + (pr - z)) + pe + Tl[q * ldt + r] * wq;
                    sacc = t2;
                }
                Yw[c * bb + r] = sacc + cmp;
            }
            __syncthreads();
        }
        // default: tensor cores for bb > 16 (measured 9 % faster at bb = 32); at bb = 16 the SIMT
        // form, whose shared-memory ring keeps more of C in flight, measured 13 % faster; the
        // descriptor's tile choice overrides the rule either way
        const bool update_tc = sm.tc && ((tiles & RQRCP_TILES_UPDATE_TC) ? true
                                         : (tiles & RQRCP_TILES_UPDATE_SIMT) ? false : bb > 16);
        if (update_tc) {
            const bool u_ok = bb <= 32 ? blk_gemm_update_tc<1>(Vp + (long long)bb * lda, lda, Vp, lda, 1, Yw, bb, m1, nt, bb, sm)
                                       : blk_gemm_update_tc<2>(Vp + (long long)bb * lda, lda, Vp, lda, 1, Yw, bb, m1, nt, bb, sm);
            if (!u_ok) {
                if (tid == 0) *d.rank = -2;
                __syncthreads();
                return false;
            }
        } else {
            blk_gemm_update(Vp + (long long)bb * lda, lda, Vp, lda, 1, Yw, bb, m1, nt, bb, sm);
        }
        __syncthreads();
        if (pivoting && i + bb < k) {
            blk_bsolve(Bw, n, A, lda, i, bb, sm);
            // Eq. (4): B(0:bb, c) -= Omega_hat_11 R12(:, c) in FP32 (Omega_hat_11 upper, from FP64):
            // every thread owns columns c, register accumulators for the bb rows, R12 read once
            float* Wf = sm.Xs;  // [q][r] = Omega_hat_11(r, q), row q contiguous
            for (int e = tid; e < bb * bb; e += BT) Wf[e] = (float)sm.Tm[e];  // Tm[q * bb + r]
            __syncthreads();
            for (long long c = i + bb + tid; c < n; c += BT) {
                float acc[kKu];
#pragma unroll
                for (int r = 0; r < kKu; ++r) acc[r] = 0.f;
                const float* a = A + c * lda + i;
#pragma unroll
                for (int q = 0; q < kKu; ++q) {
                    if (q < bb) {
                        const float aq = a[q];
                        const float* wq = Wf + q * bb;
#pragma unroll
                        for (int r = 0; r <= q; ++r) acc[r] = fmaf(wq[r], aq, acc[r]);  // Omega_hat_11(r, q), r <= q
                    }
                }
#pragma unroll
                for (int r = 0; r < kKu; ++r)
                    if (r < bb) Bw[(long long)r * n + c] -= acc[r];
            }
            __syncthreads();
        }
    }
    if (tid == 0) *d.rank = rank;
    __syncthreads();
    return true;
}

// The panel's sub-panel and the contractions' shared-memory buffers are never live at the
// same time, so they share one region.
__host__ __device__ inline size_t union_floats(long long m_max)
{
    size_t f = (size_t)SW * (size_t)m_max;
    if (f < (size_t)kGemmFloats) f = kGemmFloats;
    if (f < (size_t)kURingFloats) f = (size_t)kURingFloats;
    return f;
}

__global__ void __launch_bounds__(BT, 1) batched_kernel(const BatchDesc* __restrict__ descs, const int* __restrict__ order,
                                                        int count, const float* __restrict__ Om, long long ldo, int p,
                                                        long long m_max, long long n_max, int b_max, char* ws,
                                                        size_t ws_per_block, int* counter, int tc)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    Smem sm;
    size_t off = 0;
    auto carve = [&](size_t bytes) {
        unsigned char* ptr = smraw + off;
        off = (off + bytes + 15) & ~(size_t)15;
        return ptr;
    };
    const int l_max = b_max + p;
    sm.G = reinterpret_cast<float*>(carve(sizeof(float) * union_floats(m_max) + 1024));  // + room to align the tensor-core ring
    sm.S = sm.G;
    sm.Xs = sm.G;
    sm.Cs = sm.G + kKu * kLdT;
    sm.nu = reinterpret_cast<double*>(carve(sizeof(double) * (size_t)n_max));
    sm.Tm = reinterpret_cast<double*>(carve(sizeof(double) * (size_t)b_max * b_max));
    sm.vs = reinterpret_cast<float*>(carve(sizeof(float) * (size_t)l_max));
    sm.red = reinterpret_cast<double*>(carve(sizeof(double) * NW * SW));
    sm.sc = reinterpret_cast<double*>(carve(sizeof(double) * 40));
    sm.scf = reinterpret_cast<float*>(carve(sizeof(float) * (SW + 1)));
    sm.piv = reinterpret_cast<int*>(carve(sizeof(int) * (size_t)b_max));
    sm.lpos = reinterpret_cast<long long*>(carve(sizeof(long long) * (NW + 1)));

    char* mine = ws + (size_t)blockIdx.x * ws_per_block;
    float* Bw = reinterpret_cast<float*>(mine);
    float* Ww = Bw + (size_t)l_max * n_max;
    float* Yw = Ww + (size_t)b_max * (n_max + b_max);
    // tensor memory (the whole of it: one block per SM) and the two MMA-completion barriers
    __shared__ __align__(8) uint64_t s_mbar[2];
    __shared__ int s_mph[2];
    __shared__ uint32_t s_tmem;
    if (tc && (threadIdx.x >> 5) == 0) tc::tmem_alloc(&s_tmem, kTmemCols);
    if (threadIdx.x == 0) {
        tc::mbar_init(&s_mbar[0], 1);
        tc::mbar_init(&s_mbar[1], 1);
        s_mph[0] = s_mph[1] = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    sm.mbar = s_mbar;
    sm.mph = s_mph;
    sm.tmem = tc ? s_tmem : 0u;
    sm.tc = tc;

    __shared__ int s_next;
    for (;;) {
        if (threadIdx.x == 0) s_next = atomicAdd(counter, 1);
        __syncthreads();
        const int idx = s_next;
        __syncthreads();
        if (idx >= count) break;
        const BatchDesc d = descs[order[idx]];
        if (!factor_one(d, Om, ldo, p, Bw, Ww, Yw, sm)) break;  // a tensor-core wait timed out
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (tc && (threadIdx.x >> 5) == 0) tc::tmem_dealloc(sm.tmem, kTmemCols);
}

size_t batched_smem_bytes(long long m_max, long long n_max, int b_max, int p)
{
    size_t off = 0;
    auto take = [&](size_t bytes) { off = (off + bytes + 15) & ~(size_t)15; };
    take(sizeof(float) * union_floats(m_max) + 1024);
    take(sizeof(double) * (size_t)n_max);
    take(sizeof(double) * (size_t)b_max * b_max);
    take(sizeof(float) * (size_t)(b_max + p));
    take(sizeof(double) * NW * SW);
    take(sizeof(double) * 40);
    take(sizeof(float) * (SW + 1));
    take(sizeof(int) * (size_t)b_max);
    take(sizeof(long long) * (NW + 1));
    return off;
}

size_t batched_ws_per_block(long long n_max, int b_max, int p)
{
    const size_t floats = (size_t)(b_max + p) * n_max + (size_t)b_max * (n_max + b_max) + (size_t)b_max * n_max;
    return ((floats * sizeof(float)) + 255) & ~(size_t)255;
}

}  // namespace
}  // namespace rq

using namespace rq;

extern "C" {

__attribute__((visibility("default"))) size_t rqrcp_batched_workspace_size(int64_t m_max, int64_t n_max, int64_t b_max,
                                                                           int64_t p)
{
    if (m_max < 1 || n_max < 1 || b_max < 1 || b_max > 64 || p < 0 || b_max + p > 1024) return 0;
    const int blocks = dev_info().sms;
    // counter + per-block scratch
    size_t off = 256;
    off += (size_t)blocks * batched_ws_per_block(n_max, (int)b_max, (int)p);
    return off;
}

__attribute__((visibility("default"))) int rqrcp_factor_batched(int64_t count, const void* descs, const int* order,
                                                                int64_t m_max, int64_t n_max, int64_t b_max,
                                                                int64_t p, const float* Omega, int64_t ldo,
                                                                void* work, size_t work_bytes, void* stream)
{
    if (count < 0) return -1;
    if (count > 0 && descs == nullptr) return -2;
    if (count > 0 && order == nullptr) return -3;
    if (m_max < 1) return -4;
    if (n_max < 1) return -5;
    if (b_max < 1 || b_max > 64) return -6;
    if (p < 0 || b_max + p > 1024) return -7;
    if (Omega == nullptr) return -8;
    if (ldo < m_max) return -9;
    const size_t need = rqrcp_batched_workspace_size(m_max, n_max, b_max, p);
    if (work == nullptr || (reinterpret_cast<uintptr_t>(work) & 255) != 0 || work_bytes < need)
        return RQRCP_ERR_WORKSPACE;
    const size_t smem = batched_smem_bytes(m_max, n_max, (int)b_max, (int)p);
    if (smem > (size_t)dev_info().max_smem_optin - 1024) return RQRCP_ERR_UNSUPPORTED;
    if (count == 0) return RQRCP_OK;
    cudaStream_t s = (cudaStream_t)stream;
    char* w = static_cast<char*>(work);
    int* counter = reinterpret_cast<int*>(w);
    char* scratch = w + 256;
    static DevFlag attr_set;
    if (!attr_set.done()) {
        if (allow_max_dynamic_smem(batched_kernel) != cudaSuccess) {
            cudaGetLastError();
            return RQRCP_ERR_CUDA;
        }
        attr_set.set();
    }
    const bool prof = prof_on();
    if (prof) prof_begin(K_BATCHED, s);
    if (cudaMemsetAsync(counter, 0, sizeof(int), s) != cudaSuccess) {
        cudaGetLastError();
        return RQRCP_ERR_CUDA;
    }
    batched_kernel<<<dev_info().sms, BT, smem, s>>>(static_cast<const BatchDesc*>(descs), order, (int)count, Omega,
                                                     (long long)ldo, (int)p, (long long)m_max, (long long)n_max,
                                                     (int)b_max, scratch, batched_ws_per_block(n_max, (int)b_max, (int)p),
                                                     counter, tensor_cores_enabled() ? 1 : 0);
    if (cudaGetLastError() != cudaSuccess) return RQRCP_ERR_CUDA;
    if (prof) prof_end(K_BATCHED, 0.0, 0.0, s);
    return RQRCP_OK;
}

}  // extern "C"
