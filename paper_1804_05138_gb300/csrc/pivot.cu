// pivot.cu -- "Partial QRCP on B(:,i:n) to get b pivots" (Alg. 2), i.e. Alg. 1 run on the
// l x (n-i) sketch for bb steps, as one cooperative kernel.
//
// Each block keeps a contiguous slice of B's trailing columns in shared memory for the whole
// block of pivot steps.  Per step t (pivot position c = i + t):
//   1. every block finds its best column by squared norm of rows t..l-1 (recomputed, Alg. 1
//      "Update r_s"), ties to the smallest current position, and publishes the value, the
//      position and the whole column into a double-buffered candidate slot;
//   2. each block then adds one to this launch's arrival counter (a release add) and waits,
//      bounded, until the counter shows all G blocks of this step (no separate barrier word, no
//      generation flip: one round trip less than a grid barrier);
//   3. every block reads all candidates, picks the same winner, regenerates the same
//      Householder reflector (xLARFG convention, FP64) from the winner's column and applies
//      it to its own columns.  The swap "c <-> winner" is pure bookkeeping: the slot that
//      held position c takes the winner's old position.
// After the last step the slices are written back to B in the new column order, block 0
// applies the transpositions to jpvt and records the net column map used to swap A.
// Rank guard: if the best remaining norm^2 is not above guard_rel2 * (largest initial
// sketch norm^2), pivoting stops for good at this step.
#include "df.cuh"
#include "pivot_common.cuh"

namespace rq {
namespace {

constexpr int kMaxCand = 1024;  // maximum blocks of the cooperative launch
constexpr int kCounterBytes = 256;  // two arrival counters (launches alternate), zeroed per call
constexpr int kMaxBB = 128;     // largest block size b the factorizations accept

// Block-wide argmax: warp shuffles, then warp 0 reduces the warps' winners (slots 0..31 of the
// shared arrays); the result goes through slot 32, which the next call writes only after its
// first barrier, so every thread has read it by then.
__device__ void block_argmax(double& v, long long& p, int& idx, double* sv, long long* sp, int* si)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    warp_argmax(v, p, idx);
    if (lane == 0) { sv[w] = v; sp[w] = p; si[w] = idx; }
    __syncthreads();
    if (w == 0) {
        double vv = lane < nw ? sv[lane] : -1.0;
        long long pp = lane < nw ? sp[lane] : LLONG_MAX;
        int ii = lane < nw ? si[lane] : -1;
        warp_argmax(vv, pp, ii);
        if (lane == 0) { sv[32] = vv; sp[32] = pp; si[32] = ii; }
    }
    __syncthreads();
    v = sv[32]; p = sp[32]; idx = si[32];
}

// FP32 form: one 64-bit key per candidate that orders as (norm, -position): the norm's bits
// (non-negative floats order as their bit patterns, a NaN above every number), then kRelMax minus
// the position relative to i, then a 10-bit index (the slot within the block, or the block within
// the grid).  0 is "no candidate".  One 64-bit max per shuffle level replaces the three-part compare.
constexpr unsigned long long kRelMax = 0x3FFFFFull;  // positions relative to i below 2^22
__device__ __forceinline__ unsigned long long fkey(float v, long long relpos, int idx)
{
    if (v < 0.f) return 0ull;
    return ((unsigned long long)(__float_as_uint(v) & 0x7FFFFFFFu) << 32) |
           ((kRelMax - (unsigned long long)relpos) << 10) | (unsigned long long)idx;
}
__device__ __forceinline__ unsigned long long warp_max_key(unsigned long long k)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long x = __shfl_xor_sync(0xffffffffu, k, o);
        k = x > k ? x : k;
    }
    return k;
}
// Block-wide maximum of the threads' keys (slot 32 of sk broadcasts it, written only after the
// next call's first barrier).
__device__ unsigned long long block_max_key(unsigned long long k, unsigned long long* sk)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    k = warp_max_key(k);
    if (lane == 0) sk[w] = k;
    __syncthreads();
    if (w == 0) {
        unsigned long long kk = lane < nw ? sk[lane] : 0ull;
        kk = warp_max_key(kk);
        if (lane == 0) sk[32] = kk;
    }
    __syncthreads();
    return sk[32];
}

template <typename T>
__global__ void __launch_bounds__(1024) pivot_kernel(T* __restrict__ B, int64_t ldb, int l, int64_t n,
                                                     int64_t i, int bb, int64_t cpb, int tpc,
                                                     int32_t* __restrict__ jpvt, int32_t* __restrict__ piv,
                                                     long long* __restrict__ swapmap,
                                                     double* __restrict__ cval, long long* __restrict__ cpos,
                                                     T* __restrict__ ccol, unsigned long long* __restrict__ ctrs,
                                                     int parity, double guard_rel2, Status* st)
{
    if (status_error(st)) return;
    const int G = gridDim.x, g = blockIdx.x, tid = threadIdx.x, NTH = blockDim.x;
    if (*(volatile int*)&st->guard) {  // pivoting switched off by an earlier block
        if (g == 0) {
            for (int t = tid; t < bb; t += NTH) piv[t] = (int32_t)(i + t);
            if (tid == 0) swapmap[0] = 0;
        }
        return;
    }
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int ldS = l | 1;  // odd stride: conflict-free column-per-thread access
    T* cols = reinterpret_cast<T*>(smem_raw);
    size_t off = ((size_t)cpb * ldS * sizeof(T) + 15) & ~(size_t)15;
    long long* pos = reinterpret_cast<long long*>(smem_raw + off);
    off += (size_t)cpb * sizeof(long long);
    double* xs = reinterpret_cast<double*>(smem_raw + off);
    off += (size_t)l * sizeof(double);
    T* vT = reinterpret_cast<T*>(smem_raw + off);
    off += ((size_t)l * sizeof(T) + 15) & ~(size_t)15;
    long long* pivs = reinterpret_cast<long long*>(smem_raw + off);
    off += (size_t)bb * sizeof(long long);
    int* active = reinterpret_cast<int*>(smem_raw + off);
    off += (size_t)cpb * sizeof(int);
    off = (off + 7) & ~(size_t)7;
    void* fin_scr = smem_raw + off;  // finish_pivots scratch (block 0)

    __shared__ double red_v[33];
    __shared__ long long red_p[33];
    __shared__ int red_i[33];
    __shared__ unsigned long long red_k[33];
    __shared__ double sh_tau, sh_beta, sh_scal;
    __shared__ float sh_scl;  // FP32 form: the low half of the float pair 1 / (alpha - beta)
    constexpr bool F = sizeof(T) == 4;  // FP32 form: packed keys, float-pair reflector scalars

    const int64_t nprime = n - i;
    const int64_t s0 = (int64_t)g * cpb;
    const int nloc = (int)max((int64_t)0, min(cpb, nprime - s0));
    for (int64_t e = tid; e < (int64_t)nloc * l; e += NTH) {
        const int s = (int)(e / l), r = (int)(e % l);
        cols[(size_t)s * ldS + r] = B[(i + s0 + s) * ldb + r];
    }
    for (int s = tid; s < nloc; s += NTH) {
        pos[s] = i + s0 + s;
        active[s] = 1;
    }
    __syncthreads();
    // Thread layout: tpc adjacent threads share column slot `sl`, thread `sub` takes rows
    // r = sub, sub + tpc, ...  Column sums combine the tpc partials by shuffles.
    const int sub = tid % tpc;
    const int slots_per_pass = NTH / tpc;
    const int my_slot0 = tid / tpc;
    // initial squared norms of rows 0..l-1 (recomputed from the rows, Alg. 1 "Update r_s"); each
    // column's first thread keeps the best of its columns for step 0
    double lbv = -1.0;
    long long lbp = LLONG_MAX;
    int lbs = -1;
    unsigned long long lk = 0ull;
    for (int sl = my_slot0; sl - my_slot0 < ((nloc + slots_per_pass - 1) / slots_per_pass) * slots_per_pass;
         sl += slots_per_pass) {
        T part = T(0);
        if (sl < nloc) {
            const T* col = cols + (size_t)sl * ldS;
            for (int r = sub; r < l; r += tpc) part = fma(col[r], col[r], part);
        }
        part = column_sum(part, tpc);
        if (sl < nloc && sub == 0) {
            if constexpr (F) {
                const unsigned long long k = fkey((float)part, pos[sl] - i, sl);
                lk = k > lk ? k : lk;
            } else if (better((double)part, pos[sl], lbv, lbp)) {
                lbv = (double)part;
                lbp = pos[sl];
                lbs = sl;
            }
        }
    }
    unsigned long long* ctr = ctrs + parity;
    if (g == 0 && tid == 0) ctrs[parity ^ 1] = 0;  // the next launch's counter (this call's launches alternate)
    __shared__ int s_ok;
    const double guard = guard_rel2 * __longlong_as_double((long long)st->nu0bits);

    int steps = bb;
    for (int t = 0; t < bb; ++t) {
        const long long c = i + t;
        const int buf = t & 1;
        // 1. the block's candidate from its threads' bests (norms of rows t..l-1)
        double myv = lbv;
        long long myp = lbp;
        int mys = lbs;
        if constexpr (F) {  // one key: the slot in its low bits, replaced by the block index
            const unsigned long long mk = block_max_key(lk, red_k);
            mys = mk ? (int)(mk & 0x3FFull) : -1;
            if (tid == 0)
                reinterpret_cast<unsigned long long*>(cval)[buf * kMaxCand + g] =
                    mk ? ((mk & ~0x3FFull) | (unsigned long long)g) : 0ull;
        } else {
            block_argmax(myv, myp, mys, red_v, red_p, red_i);
            if (tid == 0) {
                cval[buf * kMaxCand + g] = myv;
                cpos[buf * kMaxCand + g] = myp;
            }
        }
        if (mys >= 0)
            for (int r = tid; r < l; r += NTH)
                ccol[((size_t)buf * kMaxCand + g) * l + r] = cols[(size_t)mys * ldS + r];
        // 2. arrive, then wait until all G blocks of this step have arrived
        __syncthreads();
        if (tid == 0) {
            asm volatile("red.release.gpu.global.add.u64 [%0], 1;" ::"l"(ctr) : "memory");
            const unsigned long long want = (unsigned long long)G * (unsigned long long)(t + 1);
            const unsigned long long t0 = globaltimer_ns();
            int ok = 1;
            while (ld_acquire_gpu(ctr) < want) {
                const unsigned long long dt = globaltimer_ns() - t0;
                if (dt > kErrorWatchNs && status_error(st)) {
                    ok = 0;
                    break;
                }
                if (dt > kWaitLimitNs) {
                    set_error(st, RQRCP_ERR_TIMEOUT);
                    ok = 0;
                    break;
                }
            }
            s_ok = ok;
        }
        __syncthreads();
        if (!s_ok) return;
        // 3. global winner (identical in every block): warp 0 reads the G candidates, eight
        //    per lane in flight at a time, and reduces them; slot 32 broadcasts the result
        if (F && tid < 32) {
            const unsigned long long* ck = reinterpret_cast<const unsigned long long*>(cval) + buf * kMaxCand;
            unsigned long long wk = 0ull;
            for (int h0 = tid; h0 < G; h0 += 8 * 32) {
                unsigned long long kk[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) kk[u] = h0 + 32 * u < G ? ld_cg(&ck[h0 + 32 * u]) : 0ull;
#pragma unroll
                for (int u = 0; u < 8; ++u) wk = kk[u] > wk ? kk[u] : wk;
            }
            wk = warp_max_key(wk);
            if (tid == 0) {
                red_v[32] = wk ? (double)__uint_as_float((unsigned)(wk >> 32)) : -1.0;
                red_p[32] = wk ? i + (long long)(kRelMax - ((wk >> 10) & kRelMax)) : LLONG_MAX;
                red_i[32] = wk ? (int)(wk & 0x3FFull) : -1;
            }
        } else if (!F && tid < 32) {
            double wv = -1.0;
            long long wp = LLONG_MAX;
            int wg = -1;
            for (int h0 = tid; h0 < G; h0 += 8 * 32) {
                double vv[8];
                long long pp[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int h = h0 + 32 * u;
                    vv[u] = h < G ? ld_cg(&cval[buf * kMaxCand + h]) : -1.0;
                    pp[u] = h < G ? ld_cg(&cpos[buf * kMaxCand + h]) : LLONG_MAX;
                }
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    if (better(vv[u], pp[u], wv, wp)) { wv = vv[u]; wp = pp[u]; wg = h0 + 32 * u; }
            }
            warp_argmax(wv, wp, wg);
            if (tid == 0) { red_v[32] = wv; red_p[32] = wp; red_i[32] = wg; }
        }
        __syncthreads();
        const double wv = red_v[32];
        const long long wp = red_p[32];
        const int wg = red_i[32];
        if (!(wv > guard)) {  // also catches "no candidate" (-1) and NaN
            if (g == 0 && tid == 0) {
                st->guard = 1;
                st->rank = c;
            }
            steps = t;
            break;
        }
        if constexpr (F) {
            float* xf = reinterpret_cast<float*>(xs);
            for (int r = tid; r < l; r += NTH) xf[r] = ld_cg(&ccol[((size_t)buf * kMaxCand + wg) * l + r]);
        } else {
            for (int r = tid; r < l; r += NTH) xs[r] = (double)ld_cg(&ccol[((size_t)buf * kMaxCand + wg) * l + r]);
        }
        __syncthreads();
        // Householder reflector from rows t..l-1 of the winner (xLARFG), warp 0, fixed order.  FP32
        // form: Dot2 sum of squares and float-pair square root and divisions (about 44 bits, no FP64
        // instruction on the chain)
        if (F && tid < 32) {
            const float* xf = reinterpret_cast<const float*>(xs);
            float qh = 0.f, ql = 0.f;
            for (int r = t + 1 + tid; r < l; r += 32) dot2_add(qh, ql, xf[r], xf[r]);
            df ssd = df_quick(qh, ql);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1)
                ssd = df_add(ssd, {__shfl_xor_sync(0xffffffffu, ssd.h, o), __shfl_xor_sync(0xffffffffu, ssd.l, o)});
            const float alpha = xf[t];
            float tauf = 0.f, betaf = alpha;
            df scal = {0.f, 0.f};
            if (ssd.h != 0.f) {
                const df nrm = df_sqrt(df_add(df_mul({alpha, 0.f}, {alpha, 0.f}), ssd));
                const df beta = alpha >= 0.f ? df_neg(nrm) : nrm;
                const df tau = df_mul(df_add(beta, {-alpha, 0.f}), df_rcp(beta));
                scal = df_rcp(df_add({alpha, 0.f}, df_neg(beta)));
                tauf = tau.h + tau.l;
                betaf = beta.h + beta.l;
            }
            if (tid == 0) {
                sh_tau = tauf;
                sh_beta = betaf;
                sh_scal = scal.h;
                sh_scl = scal.l;
                if (g == 0) pivs[t] = wp;
            }
        } else if (!F && tid < 32) {
            double ss = 0.0;
            for (int r = t + 1 + tid; r < l; r += 32) ss += xs[r] * xs[r];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
            double tau, beta, scal;
            warp_larfg(xs[t], ss, tau, beta, scal);
            if (tid == 0) {
                sh_tau = tau;
                sh_beta = beta;
                sh_scal = scal;
                if (g == 0) pivs[t] = wp;
            }
        }
        __syncthreads();
        if constexpr (F) {
            const float* xf = reinterpret_cast<const float*>(xs);
            const df sc = {(float)sh_scal, sh_scl};
            for (int r = t + 1 + tid; r < l; r += NTH) {
                const df v = df_mul({xf[r], 0.f}, sc);
                vT[r] = v.h + v.l;
            }
        } else {
            for (int r = t + 1 + tid; r < l; r += NTH) vT[r] = (T)(xs[r] * sh_scal);
        }
        if (tid == 0) vT[t] = T(1);
        __syncthreads();
        // 4. apply H to every remaining column, then the norms of rows t+1..l-1 for step t+1
        const T tauT = (T)sh_tau;
        const bool apply = sh_tau != 0.0;
        lbv = -1.0;
        lbp = LLONG_MAX;
        lbs = -1;
        lk = 0ull;
        for (int sl = my_slot0; sl - my_slot0 < ((nloc + slots_per_pass - 1) / slots_per_pass) * slots_per_pass;
             sl += slots_per_pass) {
            const bool mine = sl < nloc;
            T* col = cols + (size_t)(mine ? sl : 0) * ldS;
            const bool winner = mine && pos[sl] == wp;
            const bool live = mine && active[sl] && !winner;
            // rows owned by this thread at and below t: r = t + ((sub - t) mod tpc) + j*tpc
            const int r0 = t + ((sub - (t % tpc)) + tpc) % tpc;
            T w = T(0);
            if (live && apply)
                for (int r = r0; r < l; r += tpc) w = fma(vT[r], col[r], w);
            w = column_sum(w, tpc);
            T nu = T(0);
            if (live) {
                const T wt = w * tauT;
                for (int r = r0; r < l; r += tpc) {
                    T x = col[r];
                    if (apply) x = fma(-wt, vT[r], x);
                    col[r] = x;
                    if (r > t) nu = fma(x, x, nu);
                }
            }
            nu = column_sum(nu, tpc);
            if (mine && sub == 0) {
                if (winner) {
                    active[sl] = 0;
                    pos[sl] = c;
                } else {
                    if (pos[sl] == c) pos[sl] = wp;  // the column displaced by the swap
                    if constexpr (F) {
                        if (active[sl]) {
                            const unsigned long long k = fkey((float)nu, pos[sl] - i, sl);
                            lk = k > lk ? k : lk;
                        }
                    } else if (active[sl] && better((double)nu, pos[sl], lbv, lbp)) {
                        lbv = (double)nu;
                        lbp = pos[sl];
                        lbs = sl;
                    }
                }
            }
            if (winner)  // becomes column c of R_hat
                for (int r = r0; r < l; r += tpc) col[r] = (r == t) ? (T)sh_beta : T(0);
        }
        __syncthreads();
    }
    // write the slices back in the new column order
    for (int64_t e = tid; e < (int64_t)nloc * l; e += NTH) {
        const int s = (int)(e / l), r = (int)(e % l);
        B[pos[s] * ldb + r] = cols[(size_t)s * ldS + r];
    }
    if (g == 0) {
        for (int t = steps + tid; t < bb; t += NTH) pivs[t] = i + t;
        __syncthreads();
        // jpvt, piv and the net column map (count, then (destination, source) pairs)
        finish_pivots(i, bb, pivs, jpvt, piv, swapmap, fin_scr);
    }
}

struct PivotCfg {
    int grid, threads;
    int64_t cpb;
    size_t smem;
};

template <typename T>
size_t pivot_smem(int64_t cpb, int l, int bb)
{
    const int ldS = l | 1;
    size_t off = ((size_t)cpb * ldS * sizeof(T) + 15) & ~(size_t)15;
    off += (size_t)cpb * sizeof(long long) + (size_t)l * sizeof(double);
    off += ((size_t)l * sizeof(T) + 15) & ~(size_t)15;
    off += (size_t)bb * sizeof(long long) + (size_t)cpb * sizeof(int);
    off = (off + 7) & ~(size_t)7;
    off += finish_scratch_bytes(bb);
    return off;
}

}  // namespace

size_t pivot_slot_bytes() { return kCounterBytes; }

size_t pivot_cand_bytes(int l)
{
    return kCounterBytes + 2 * (size_t)kMaxCand * (sizeof(double) + sizeof(long long)) +
           2 * (size_t)kMaxCand * l * sizeof(double);
}

bool pivot_fits(int64_t ncols, int l, int elem_bytes)
{
    if (l > 1024) return false;
    if (ncols >= (int64_t)kRelMax) return false;  // the FP32 form's keys hold positions in 22 bits
    const int64_t G = dev_info().sms;
    const int64_t cpb = (ncols + G - 1) / G;
    if (cpb > 1024) return false;
    const size_t need = elem_bytes == 8 ? pivot_smem<double>(cpb, l, kMaxBB) : pivot_smem<float>(cpb, l, kMaxBB);
    return need <= (size_t)dev_info().max_smem_optin - 2048;
}

template <typename T>
cudaError_t launch_pivot(T* B, int64_t ldb, int l, int64_t n, int64_t i, int bb, int32_t* jpvt,
                         int32_t* piv, void* cand, double guard_rel2, Status* st, cudaStream_t s,
                         int launch_index)
{
    static DevFlag attr_set;
    if (!attr_set.done()) {
        if (cudaError_t e = allow_max_dynamic_smem(pivot_kernel<T>)) return e;
        attr_set.set();
    }
    const int64_t nprime = n - i;
    // every SM takes a slice of at least 8 columns; tpc threads share a column
    int64_t G = (nprime + 7) / 8;
    if (G > dev_info().sms) G = dev_info().sms;
    if (G < 1) G = 1;
    const int64_t cpb = (nprime + G - 1) / G;
    int tpc = 4;
    while (tpc > 1 && cpb * tpc > 1024) tpc >>= 1;
    int threads = (int)(((cpb * tpc + 31) / 32) * 32);
    if (threads < 64) threads = 64;
    if (threads > 1024) threads = 1024;
    const size_t smem = pivot_smem<T>(cpb, l, bb);
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pivot_kernel<T>, threads, smem);
    if (e != cudaSuccess) return e;
    if ((int64_t)per_sm * dev_info().sms < G) return cudaErrorCooperativeLaunchTooLarge;

    char* cb = static_cast<char*>(cand);
    unsigned long long* ctrs = reinterpret_cast<unsigned long long*>(cb);
    cb += kCounterBytes;
    double* cval = reinterpret_cast<double*>(cb);
    long long* cpos = reinterpret_cast<long long*>(cb + 2 * (size_t)kMaxCand * sizeof(double));
    T* ccol = reinterpret_cast<T*>(cb + 2 * (size_t)kMaxCand * (sizeof(double) + sizeof(long long)));
    // the swap map lives right after the candidate columns
    long long* swapmap = reinterpret_cast<long long*>(static_cast<char*>(cand) + pivot_cand_bytes(l));
    int bbv = bb;
    int lv = l;
    int64_t ldbv = ldb, nv = n, iv = i, cpbv = cpb;
    int tpcv = tpc;
    double gr = guard_rel2;
    // launches of one call alternate between the two counters (the call zeroes both first)
    int parity = launch_index & 1;
    void* args[] = {&B,    &ldbv, &lv,  &nv,   &iv,     &bbv, &cpbv, &tpcv, &jpvt,
                    &piv,  &swapmap, &cval, &cpos, &ccol, &ctrs, &parity, &gr, &st};
    return cudaLaunchCooperativeKernel((const void*)pivot_kernel<T>, dim3((unsigned)G), dim3(threads), args, smem, s);
}

template cudaError_t launch_pivot<double>(double*, int64_t, int, int64_t, int64_t, int, int32_t*, int32_t*,
                                          void*, double, Status*, cudaStream_t, int);
template cudaError_t launch_pivot<float>(float*, int64_t, int, int64_t, int64_t, int, int32_t*, int32_t*,
                                         void*, double, Status*, cudaStream_t, int);

}  // namespace rq
