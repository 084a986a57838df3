// lowrank.cu -- helpers of the low-rank product L = Q1 [R11 R12] Pi^T (Sec. I-A).
#include "df.cuh"
#include "internal.cuh"

namespace rq {
namespace {

// Rk(q, c) = -R(q, c) for q <= c (upper trapezoid of the first k rows), 0 below; ld = k.
template <typename T>
__global__ void rk_kernel(const T* __restrict__ Af, int64_t ldaf, int64_t k, int64_t n, double* __restrict__ Rk)
{
    for (int64_t c = blockIdx.x; c < n; c += gridDim.x)
        for (int64_t q = threadIdx.x; q < k; q += blockDim.x) Rk[c * k + q] = (q <= c) ? -(double)Af[c * ldaf + q] : 0.0;
}

// Q(:, 0:k) = I(:, 0:k).
template <typename T>
__global__ void eye_kernel(T* __restrict__ Q, int64_t ldq, int64_t m, int64_t k)
{
    for (int64_t c = blockIdx.x; c < k; c += gridDim.x)
        for (int64_t r = threadIdx.x; r < m; r += blockDim.x) Q[c * ldq + r] = (r == c) ? T(1) : T(0);
}

// Packed strict upper triangle of G = V^T V from the split partials P[(z k + d) k + c] (c < d):
// Gp[d (d - 1) / 2 + c] = sum_z P (compensated sum, rounded once).  Block d, threads over c.
__global__ void gpack_kernel(const float* __restrict__ P, int nz, int64_t k, float* __restrict__ Gp)
{
    for (int64_t d = blockIdx.x; d < k; d += gridDim.x)
        for (int64_t c = threadIdx.x; c < d; c += blockDim.x) {
            float gh = 0.f, gl = 0.f;  // compensated sum (TwoSum): FP64 issues slowly on this part
            for (int z0 = 0; z0 < nz; z0 += 8) {
                float pv[8];
#pragma unroll
                for (int zz = 0; zz < 8; ++zz) pv[zz] = z0 + zz < nz ? P[((int64_t)(z0 + zz) * k + d) * k + c] : 0.f;
#pragma unroll
                for (int zz = 0; zz < 8; ++zz) {
                    const df t = df_two_sum(gh, pv[zz]);
                    gh = t.h;
                    gl += t.l;
                }
            }
            Gp[d * (d - 1) / 2 + c] = gh + gl;
        }
}

constexpr int kZWarps = 8;
constexpr int kZMaxK = 256;  // unknowns per warp: eight per lane in registers

// Back-substitution steps d = min(j, 32 T + 31) down to 32 T: z_d = tau_d b_d (b_d broadcast from
// register T of lane d % 32), then b_c -= G(c, d) z_d for c < d (registers t <= T) and b_d <- z_d.
template <int T>
__device__ __forceinline__ void wy_z_steps(float (&b)[8], int j, const float* taus, const float* Gs, int lane)
{
    const int dhi = j < 32 * T + 31 ? j : 32 * T + 31;
    for (int d = dhi; d >= 32 * T; --d) {
        const float* gcol = Gs + d * (d - 1) / 2;
        float g[T + 1];
#pragma unroll
        for (int t = 0; t <= T; ++t) {
            const int c = lane + 32 * t;
            g[t] = c < d ? gcol[c] : 0.f;
        }
        const float zd = taus[d] * __shfl_sync(0xffffffffu, b[T], d & 31);
#pragma unroll
        for (int t = 0; t < T; ++t) b[t] = fmaf(-g[t], zd, b[t]);
        const int c = lane + 32 * T;
        b[T] = c < d ? fmaf(-g[T], zd, b[T]) : (c == d ? zd : b[T]);
    }
}

// Z = T V1^T (k x k, column-major) for the compact WY form Q = I - V T V^T of H_0 ... H_{k-1}: T is
// upper triangular with T^{-1} = diag(1 / tau) + striu(V^T V), so column j of Z solves
// T^{-1} z = V(j, 0:k)^T by back substitution, z_d = tau_d (b_d - sum_{c > d} G(d, c) z_c) in the
// column-oriented order.  V(j, c) is 0 for c > j, so z_c = 0 there.  A reflector with tau = 0
// (H = I) gets z = 0 and adds nothing.  One warp per column j, the right-hand side in registers
// (c = lane + 32 t); the packed G of the columns the block needs is staged in shared memory.
__global__ void __launch_bounds__(32 * kZWarps) wy_z_kernel(const float* __restrict__ Af, int64_t ldaf,
                                                            const double* __restrict__ tau, const float* __restrict__ Gp,
                                                            int64_t k, float* __restrict__ Z)
{
    extern __shared__ float zsm[];
    float* taus = zsm;         // k
    float* Gs = zsm + kZMaxK;  // packed G, columns d <= jmax
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t j0 = (int64_t)blockIdx.x * kZWarps;
    const int64_t jmax = (j0 + kZWarps - 1 < k - 1) ? j0 + kZWarps - 1 : k - 1;
    for (int64_t c = threadIdx.x; c <= jmax; c += blockDim.x) taus[c] = (float)tau[c];
    const int64_t ng4 = (jmax * (jmax + 1) / 2 + 3) / 4;  // staged as float4, eight loads in flight
    const float4* G4 = reinterpret_cast<const float4*>(Gp);
    float4* Gs4 = reinterpret_cast<float4*>(Gs);
    for (int64_t e0 = threadIdx.x; e0 < ng4; e0 += 8 * (int64_t)blockDim.x) {
        float4 v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int64_t e = e0 + (int64_t)u * blockDim.x;
            if (e < ng4) v[u] = G4[e];
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int64_t e = e0 + (int64_t)u * blockDim.x;
            if (e < ng4) Gs4[e] = v[u];
        }
    }
    __syncthreads();
    const int64_t j = j0 + warp;
    if (j >= k) return;
    float b[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) {
        const int64_t c = lane + 32 * t;
        b[t] = c < j ? Af[c * ldaf + j] : (c == j ? 1.f : 0.f);
    }
    // steps d = j .. 0 in groups of 32 sharing the register t = d / 32 that holds b_d
    switch ((int)(j >> 5)) {
    case 7: wy_z_steps<7>(b, (int)j, taus, Gs, lane); [[fallthrough]];
    case 6: wy_z_steps<6>(b, (int)j, taus, Gs, lane); [[fallthrough]];
    case 5: wy_z_steps<5>(b, (int)j, taus, Gs, lane); [[fallthrough]];
    case 4: wy_z_steps<4>(b, (int)j, taus, Gs, lane); [[fallthrough]];
    case 3: wy_z_steps<3>(b, (int)j, taus, Gs, lane); [[fallthrough]];
    case 2: wy_z_steps<2>(b, (int)j, taus, Gs, lane); [[fallthrough]];
    case 1: wy_z_steps<1>(b, (int)j, taus, Gs, lane); [[fallthrough]];
    default: wy_z_steps<0>(b, (int)j, taus, Gs, lane);
    }
#pragma unroll
    for (int t = 0; t < 8; ++t) {
        const int64_t c = lane + 32 * t;
        if (c < k) Z[j * k + c] = c <= j ? b[t] : 0.f;
    }
}

size_t wy_z_smem(int64_t k) { return (size_t)(kZMaxK + k * (k - 1) / 2 + 4) * sizeof(float); }

unsigned grid_for(int64_t total)
{
    int64_t g = (total + 255) / 256;
    if (g > 65535) g = 65535;
    const int64_t cap = (int64_t)dev_info().sms * 16;
    if (g > cap) g = cap;
    return (unsigned)(g < 1 ? 1 : g);
}

}  // namespace

template <typename T>
cudaError_t launch_lowrank_rk(const T* Af, int64_t ldaf, int64_t k, int64_t n, double* Rk, cudaStream_t s)
{
    rk_kernel<T><<<grid_for(n * 256), 256, 0, s>>>(Af, ldaf, k, n, Rk);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_eye(T* Q, int64_t ldq, int64_t m, int64_t k, cudaStream_t s)
{
    eye_kernel<T><<<grid_for(k * 256), 256, 0, s>>>(Q, ldq, m, k);
    return cudaGetLastError();
}

// FP32 tensor-core form of the low-rank outputs (see internal.cuh): all k reflectors at once.
namespace {
constexpr size_t kLrAlign = 256;
size_t lr_al(size_t x) { return (x + kLrAlign - 1) & ~(kLrAlign - 1); }
// The tensor core accumulates in FP32: the contractions run as splits of at most two 32-row chunks
// (64 terms, as the factorization's Gram folds its accumulator), the splits summed with compensation.
constexpr int kLrMaxSplit = 64;
constexpr int kLrChunks = 2;

struct LrTcLayout {
    size_t status, planes, part, gp, z, total;
};

LrTcLayout lr_tc_layout(int64_t m, int64_t n, int64_t k)
{
    LrTcLayout L{};
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = lr_al(off + bytes);
        return o;
    };
    size_t pl = mm_planes_bytes(m, k);
    for (size_t x : {mm_planes_bytes(k, k), mm_planes_bytes(k, n)})
        if (x > pl) pl = x;
    L.status = take(sizeof(Status));
    L.planes = take(pl);
    const int64_t sq = (k + 32 * kLrChunks - 1) / (32 * kLrChunks);  // splits of V Z (K = k)
    size_t part = (size_t)kLrMaxSplit * k * k;
    if ((size_t)sq * m * k > part) part = (size_t)sq * m * k;
    L.part = take(part * sizeof(float));
    L.gp = take((size_t)(k * (k - 1) / 2 + 4) * sizeof(float));  // read as float4
    L.z = take((size_t)k * k * sizeof(float));
    L.total = off;
    return L;
}
}  // namespace

size_t lowrank_f32_tc_bytes(int64_t m, int64_t n, int64_t k) { return lr_tc_layout(m, n, k).total; }

bool lowrank_f32_tc_ok(int64_t k, const float* Afact, int64_t ldaf, const float* Q1, int64_t ldq)
{
    return k >= 1 && k <= kZMaxK && tensor_cores_enabled() && mm_tc_supported(Afact, ldaf) &&
           mm_tc_supported(Q1, ldq) && wy_z_smem(k) <= (size_t)dev_info().max_smem_optin;
}

#define LR_CHECK(expr)                  \
    do {                                \
        if ((expr) != cudaSuccess) {    \
            cudaGetLastError();         \
            return RQRCP_ERR_CUDA;      \
        }                               \
    } while (0)

int lowrank_f32_tc(int64_t m, int64_t n, int64_t k, const float* Afact, int64_t ldaf, const double* tau,
                   const int32_t* jpvt, float* L, int64_t ldl, float* Q1, int64_t ldq, void* work, cudaStream_t s)
{
    const LrTcLayout Lw = lr_tc_layout(m, n, k);
    char* w = static_cast<char*>(work);
    Status* st = reinterpret_cast<Status*>(w + Lw.status);
    float* PL = reinterpret_cast<float*>(w + Lw.planes);
    float* Part = reinterpret_cast<float*>(w + Lw.part);
    float* Gp = reinterpret_cast<float*>(w + Lw.gp);
    float* Z = reinterpret_cast<float*>(w + Lw.z);
    LR_CHECK(launch_init(st, k, nullptr, 0, s));
    // G = V^T V (strict upper part used), split over the m rows
    LR_CHECK(launch_mm_planes(Afact, 1, ldaf, nullptr, 0, m, k, PL, st, s, 1));
    int S = mm_choose_split(k, k, m, kLrChunks);
    if (S > kLrMaxSplit) S = kLrMaxSplit;
    LR_CHECK(launch_mm_tc(true, Afact, ldaf, PL, k, k, m, S, 1.f, 0.f, nullptr, 0, Part, k, k * k, nullptr, st, s, 1));
    gpack_kernel<<<(unsigned)(k < 1024 ? k : 1024), 256, 0, s>>>(Part, S, k, Gp);
    LR_CHECK(cudaGetLastError());
    // Z = T V1^T, then Q1 = I(:, 0:k) - V Z
    static DevFlag attr_set;
    if (!attr_set.done()) {
        LR_CHECK(allow_max_dynamic_smem(wy_z_kernel));
        attr_set.set();
    }
    wy_z_kernel<<<(unsigned)((k + kZWarps - 1) / kZWarps), 32 * kZWarps, wy_z_smem(k), s>>>(Afact, ldaf, tau, Gp, k, Z);
    LR_CHECK(cudaGetLastError());
    LR_CHECK(launch_mm_planes(Z, 1, k, nullptr, 0, k, k, PL, st, s, 0));
    LR_CHECK(launch_eye<float>(Q1, ldq, m, k, s));
    const int sq = (int)((k + 32 * kLrChunks - 1) / (32 * kLrChunks));
    if (sq <= 1) {
        LR_CHECK(launch_mm_tc(false, Afact, ldaf, PL, m, k, k, 1, -1.f, 1.f, Q1, ldq, Q1, ldq, 0, nullptr, st, s, 1));
    } else {
        LR_CHECK(launch_mm_tc(false, Afact, ldaf, PL, m, k, k, sq, -1.f, 0.f, nullptr, 0, Part, m, m * k, nullptr, st, s,
                              1));
        LR_CHECK(launch_mm_sum(Part, m, m * k, sq, m, k, Q1, ldq, Q1, ldq, st, s));
    }
    if (L == nullptr) return RQRCP_OK;
    // L(:, jpvt[c]) = Q1 [R11 R12](:, c)
    LR_CHECK(launch_mm_planes(Afact, 1, ldaf, nullptr, 0, k, n, PL, st, s, 2));
    LR_CHECK(launch_mm_tc(false, Q1, ldq, PL, m, n, k, 1, 1.f, 0.f, nullptr, 0, L, ldl, 0, jpvt, st, s, 0));
    return RQRCP_OK;
}

template cudaError_t launch_lowrank_rk<double>(const double*, int64_t, int64_t, int64_t, double*, cudaStream_t);
template cudaError_t launch_lowrank_rk<float>(const float*, int64_t, int64_t, int64_t, double*, cudaStream_t);
template cudaError_t launch_eye<double>(double*, int64_t, int64_t, int64_t, cudaStream_t);
template cudaError_t launch_eye<float>(float*, int64_t, int64_t, int64_t, cudaStream_t);

}  // namespace rq
