// tournament.cu -- "Partial QRCP on B(:,i:n) to get b pivots" (Alg. 2) by QR with tournament
// pivoting, the replacement for the partial QRCP on B that the paper names as future work (Sec. VI;
// Demmel, Grigori, Gu and Xiang, "Communication avoiding rank revealing QR factorization with column
// pivoting", SIAM J. Matrix Anal. Appl. 36, 2015).
//
// For the block at column i with bb pivots over the n' = n - i trailing sketch columns (l rows):
//   leaves  P = ceil(n' / gs) groups of gs consecutive columns, one thread block each: the group's
//           columns go to shared memory and bb greedy steps of Alg. 1 (squared norms of the trailing
//           rows recomputed at every step, the largest first, ties to the smallest position) choose
//           min(bb, group size) of them;
//   levels  each node (one thread block) gathers the columns that its `fanin` children chose, as they
//           were in B, concatenated in child order, and chooses min(bb, candidates) of them the same
//           way; one launch per level until one node is left;
//   final   one block factors the root's columns in the order chosen by Householder QR with FP64
//           reflector scalars (the rank guard tests each chosen column's trailing squared norm at its
//           step), and turns the choices into the block's transpositions, jpvt, piv and the net
//           column map;
//   apply   every other trailing column of B gets the reflectors, each chosen one its column of
//           R_hat, in place; the swap kernels then move the columns as the transpositions say.
// The selection steps compute their reflectors in the sketch's precision T: only their choices are
// kept.  No host synchronisation; every wait is a barrier inside one block.
#include "pivot_common.cuh"

namespace rq {
namespace {

constexpr int kFanin = 4;
constexpr int kSelMaxCols = 1024;  // candidates of one selection block (tpc >= 1 thread per column)
constexpr int kFinalThreads = 256;
constexpr int kApplyThreads = 256;
constexpr int kApplyTpc = 8;       // threads per column in the apply kernel
constexpr int kApplyCols = kApplyThreads / kApplyTpc;
constexpr int kMaxL = 256;

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

// Shared memory of one selection block with room for nc candidate columns.
template <typename T>
__host__ __device__ inline size_t select_smem(int nc, int l, int bb)
{
    const int ldS = l | 1;
    return align16((size_t)nc * ldS * sizeof(T)) + align16((size_t)nc * sizeof(long long)) +
           align16((size_t)nc * sizeof(int)) + align16((size_t)l * sizeof(T)) + (size_t)bb * sizeof(long long);
}

inline int select_tpc(int nc) { return nc <= 256 ? 4 : (nc <= 512 ? 2 : 1); }
inline int select_threads(int nc)
{
    int t = ((nc * select_tpc(nc) + 31) / 32) * 32;
    return t < 64 ? 64 : t;
}

// Greedy choice of `steps` of the nc columns cols(:, s) (shared memory, stride ldS, l rows), whose
// positions are cpos[s]: Alg. 1 with the squared norms of rows t..l-1 recomputed at every step,
// the largest first, ties to the smallest position; each step's reflector (xLARFG convention, in T)
// is applied to the columns still in the running.  out[t] = the position chosen at step t.  tpc
// adjacent threads share a column; every thread of the block calls this.
template <typename T>
__device__ void select_columns(T* cols, int ldS, const long long* cpos, int nc, int l, int steps, int tpc,
                               int* active, T* vT, long long* out, double* sv, long long* sp, int* si, T* stau)
{
    const int tid = threadIdx.x, nth = blockDim.x, lane = tid & 31, w = tid >> 5, nw = nth >> 5;
    const int sub = tid % tpc, spp = nth / tpc, slot0 = tid / tpc;
    const int passes = (nc + spp - 1) / spp;
    for (int s = tid; s < nc; s += nth) active[s] = 1;
    __syncthreads();
    for (int t = 0; t < steps; ++t) {
        double bv = -1.0;
        long long bp = LLONG_MAX;
        int bs = -1;
        const T tauT = t > 0 ? *stau : T(0);
        for (int k = 0; k < passes; ++k) {
            const int s = slot0 + k * spp;
            const bool live = s < nc && active[s];
            T* col = cols + (size_t)(s < nc ? s : 0) * ldS;
            if (t > 0 && tauT != T(0)) {  // the previous step's reflector on rows t-1 .. l-1
                const int u = t - 1;
                const int r0 = u + ((sub - (u % tpc)) + tpc) % tpc;
                T d = T(0);
                if (live)
                    for (int r = r0; r < l; r += tpc) d = fma(vT[r], col[r], d);
                d = column_sum(d, tpc);
                if (live) {
                    const T dt = d * tauT;
                    for (int r = r0; r < l; r += tpc) col[r] = fma(-dt, vT[r], col[r]);
                }
            }
            const int r1 = t + ((sub - (t % tpc)) + tpc) % tpc;
            T nu = T(0);
            if (live)
                for (int r = r1; r < l; r += tpc) nu = fma(col[r], col[r], nu);
            nu = column_sum(nu, tpc);
            if (live && better((double)nu, cpos[s], bv, bp)) {
                bv = (double)nu;
                bp = cpos[s];
                bs = s;
            }
        }
        warp_argmax(bv, bp, bs);
        if (lane == 0) {
            sv[w] = bv;
            sp[w] = bp;
            si[w] = bs;
        }
        __syncthreads();
        if (w == 0) {  // the block's winner and its reflector
            double vv = lane < nw ? sv[lane] : -1.0;
            long long pp = lane < nw ? sp[lane] : LLONG_MAX;
            int ii = lane < nw ? si[lane] : -1;
            warp_argmax(vv, pp, ii);
            const T* x = cols + (size_t)(ii >= 0 ? ii : 0) * ldS;
            T ss = T(0);
            for (int r = t + 1 + lane; r < l; r += 32) ss = fma(x[r], x[r], ss);
            ss = column_sum(ss, 32);
            const T alpha = x[t];
            T tau = T(0), scal = T(0);
            if (ss != T(0)) {
                const T nrm = sqrt(alpha * alpha + ss);
                const T beta = alpha >= T(0) ? -nrm : nrm;
                tau = (beta - alpha) / beta;
                scal = T(1) / (alpha - beta);
            }
            for (int r = t + 1 + lane; r < l; r += 32) vT[r] = x[r] * scal;
            if (lane == 0) {
                vT[t] = T(1);
                *stau = tau;
                out[t] = pp;
                if (ii >= 0) active[ii] = 0;
            }
        }
        __syncthreads();
    }
}

// One selection node.  Level 0: node g takes the columns i + g gs .. min(i + (g+1) gs, n) - 1.
// Level > 0: node g takes the choices of nodes g fanin .. (g+1) fanin - 1 of the previous level
// (cand_in, cnt_in; `nprev` nodes there).  Writes its choices to cand_out[g bb ..] and their count.
template <typename T>
__global__ void __launch_bounds__(1024) tp_select_kernel(const T* __restrict__ B, int64_t ldb, int l, int64_t i,
                                                         int64_t n, int bb, int64_t gs, int level,
                                                         const long long* __restrict__ cand_in,
                                                         const int* __restrict__ cnt_in, int nprev, int fanin,
                                                         long long* __restrict__ cand_out, int* __restrict__ cnt_out,
                                                         int tpc, const Status* st)
{
    if (status_error(st)) return;
    if (*(volatile const int*)&st->guard) return;  // pivoting switched off by an earlier block
    extern __shared__ __align__(16) unsigned char tp_sm[];
    const int ldS = l | 1;
    const int g = blockIdx.x, tid = threadIdx.x, nth = blockDim.x;
    // candidate count and positions
    int nc;
    int64_t c0 = 0;
    if (level == 0) {
        c0 = i + (int64_t)g * gs;
        const int64_t c1 = c0 + gs < n ? c0 + gs : n;
        nc = (int)(c1 - c0);
    } else {
        nc = 0;
        for (int c = g * fanin; c < (g + 1) * fanin && c < nprev; ++c) nc += cnt_in[c];
    }
    T* cols = reinterpret_cast<T*>(tp_sm);
    size_t off = align16((size_t)nc * ldS * sizeof(T));
    long long* cpos = reinterpret_cast<long long*>(tp_sm + off);
    off += align16((size_t)nc * sizeof(long long));
    int* active = reinterpret_cast<int*>(tp_sm + off);
    off += align16((size_t)nc * sizeof(int));
    T* vT = reinterpret_cast<T*>(tp_sm + off);
    off += align16((size_t)l * sizeof(T));
    long long* out = reinterpret_cast<long long*>(tp_sm + off);
    __shared__ double sv[32];
    __shared__ long long sp[32];
    __shared__ int si[32];
    __shared__ T stau;
    if (level == 0) {
        for (int s = tid; s < nc; s += nth) cpos[s] = c0 + s;
    } else {
        for (int e = tid; e < nc; e += nth) {  // candidate e: child c, its choice e - (earlier counts)
            int c = g * fanin, rem = e;
            while (rem >= cnt_in[c]) {
                rem -= cnt_in[c];
                ++c;
            }
            cpos[e] = cand_in[(size_t)c * bb + rem];
        }
    }
    __syncthreads();
    for (int e = tid; e < nc * l; e += nth) {
        const int s = e / l, r = e - s * l;
        cols[(size_t)s * ldS + r] = B[cpos[s] * ldb + r];
    }
    const int steps = bb < nc ? bb : nc;
    select_columns<T>(cols, ldS, cpos, nc, l, steps, tpc, active, vT, out, sv, sp, si, &stau);
    for (int t = tid; t < steps; t += nth) cand_out[(size_t)g * bb + t] = out[t];
    if (tid == 0) cnt_out[g] = steps;
}

// The root's bb columns (positions sel[0..bb), taken from B as it is) factored in that order by
// Householder QR, FP64 reflector scalars (xLARFG), the application in T: V(:, t) (rows t..l-1, 1 at
// t, zero above) and tau_t of every step taken, and the chosen column's R_hat column (rows 0..t-1
// as transformed, beta at t, zero below).  The rank guard stops at the first step whose chosen
// column has a trailing squared norm not above the guard.  Then the transpositions i + t <-> the
// chosen column's position at step t, jpvt, piv and the net column map; *steps_out = the steps
// taken.  One block.
template <typename T>
__global__ void __launch_bounds__(kFinalThreads) tp_final_kernel(const T* __restrict__ B, int64_t ldb, int l,
                                                                 int64_t i, int bb, const long long* __restrict__ sel,
                                                                 int32_t* __restrict__ jpvt, int32_t* __restrict__ piv,
                                                                 long long* __restrict__ swapmap, T* __restrict__ Vg,
                                                                 double* __restrict__ taug, T* __restrict__ Rg,
                                                                 int* __restrict__ steps_out, double guard_rel2,
                                                                 Status* st)
{
    if (status_error(st)) return;
    extern __shared__ __align__(16) unsigned char tp_sm[];
    const int ldS = l | 1;
    T* cols = reinterpret_cast<T*>(tp_sm);
    size_t off = align16((size_t)bb * ldS * sizeof(T));
    T* vT = reinterpret_cast<T*>(tp_sm + off);
    off += align16((size_t)l * sizeof(T));
    long long* pivs = reinterpret_cast<long long*>(tp_sm + off);
    off += (size_t)bb * sizeof(long long);
    long long* ssel = reinterpret_cast<long long*>(tp_sm + off);
    off += (size_t)bb * sizeof(long long);
    int* cur = reinterpret_cast<int*>(tp_sm + off);
    off += (size_t)2 * bb * sizeof(int);
    int* who = reinterpret_cast<int*>(tp_sm + off);
    off += (size_t)2 * bb * sizeof(int);
    void* fin = tp_sm + ((off + 7) & ~(size_t)7);
    __shared__ double s_tau;
    __shared__ int s_stop;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5, nw = kFinalThreads / 32;
    const bool pivot_off = *(volatile int*)&st->guard != 0;
    int steps = 0;
    if (!pivot_off) {
        for (int t = tid; t < bb; t += kFinalThreads) ssel[t] = sel[t];
        __syncthreads();
        for (int e = tid; e < bb * l; e += kFinalThreads) {
            const int s = e / l, r = e - s * l;
            cols[(size_t)s * ldS + r] = B[ssel[s] * ldb + r];
        }
        __syncthreads();
        const double guard = guard_rel2 * __longlong_as_double((long long)st->nu0bits);
        steps = bb;
        for (int t = 0; t < bb; ++t) {
            const T* x = cols + (size_t)t * ldS;
            if (w == 0) {
                double ss = 0.0;
                for (int r = t + 1 + lane; r < l; r += 32) {
                    const double v = (double)x[r];
                    ss += v * v;
                }
                ss = column_sum(ss, 32);
                const double alpha = (double)x[t];
                const bool stop = !(alpha * alpha + ss > guard);  // also catches NaN
                double tau, beta, scal;
                warp_larfg(alpha, ss, tau, beta, scal);
                if (!stop) {
                    for (int r = t + 1 + lane; r < l; r += 32) vT[r] = (T)((double)x[r] * scal);
                    for (int r = lane; r < l; r += 32) {
                        Rg[(size_t)t * l + r] = r < t ? x[r] : (r == t ? (T)beta : T(0));
                        Vg[(size_t)t * l + r] = r < t ? T(0) : (r == t ? T(1) : (T)((double)x[r] * scal));
                    }
                }
                if (lane == 0) {
                    s_stop = stop ? 1 : 0;
                    s_tau = tau;
                    if (!stop) {
                        vT[t] = T(1);
                        taug[t] = tau;
                    }
                }
            }
            __syncthreads();
            if (s_stop) {
                steps = t;
                break;
            }
            const T tauT = (T)s_tau;
            if (tauT != T(0))
                for (int c = t + 1 + w; c < bb; c += nw) {
                    T* y = cols + (size_t)c * ldS;
                    T d = T(0);
                    for (int r = t + lane; r < l; r += 32) d = fma(vT[r], y[r], d);
                    d = column_sum(d, 32);
                    const T dt = d * tauT;
                    for (int r = t + lane; r < l; r += 32) y[r] = fma(-dt, vT[r], y[r]);
                }
            __syncthreads();
        }
        if (steps < bb && tid == 0) {
            st->guard = 1;
            st->rank = i + steps;
        }
    }
    if (tid == 0) {
        // Positions that can move: slot s < bb is position i + s, slot bb + t is position sel[t]
        // (used when sel[t] >= i + bb).  cur[s]: the slot where the column that started at slot s
        // now is; who[s]: the starting slot of the column now at slot s.
        for (int q = 0; q < 2 * bb; ++q) cur[q] = who[q] = q;
        for (int t = 0; t < steps; ++t) {
            const int ss = ssel[t] < i + bb ? (int)(ssel[t] - i) : bb + t;
            const int sp = cur[ss];
            pivs[t] = sp < bb ? i + sp : ssel[sp - bb];
            if (sp != t) {
                const int o = who[t];
                who[t] = ss;
                who[sp] = o;
                cur[ss] = t;
                cur[o] = sp;
            }
        }
        for (int t = steps; t < bb; ++t) pivs[t] = i + t;
        *steps_out = steps;
    }
    __syncthreads();
    finish_pivots(i, bb, pivs, jpvt, piv, swapmap, fin);
}

// Every trailing column j of B: the chosen ones (sel[t], t < steps) get their R_hat column, the
// others the reflectors V(:, 0..steps-1) in order (rows t..l-1 for reflector t), in place.
// kApplyTpc threads per column, each owning the rows r = sub (mod kApplyTpc).
template <typename T>
__global__ void __launch_bounds__(kApplyThreads) tp_apply_kernel(T* __restrict__ B, int64_t ldb, int l, int64_t i,
                                                                 int64_t n, int bb, const long long* __restrict__ sel,
                                                                 const T* __restrict__ Vg,
                                                                 const double* __restrict__ taug,
                                                                 const T* __restrict__ Rg,
                                                                 const int* __restrict__ steps_in, const Status* st)
{
    if (status_error(st)) return;
    const int steps = *steps_in;
    if (steps == 0) return;
    extern __shared__ __align__(16) unsigned char tp_sm[];
    T* Vs = reinterpret_cast<T*>(tp_sm);
    size_t off = align16((size_t)steps * l * sizeof(T));
    T* taus = reinterpret_cast<T*>(tp_sm + off);
    off += align16((size_t)steps * sizeof(T));
    long long* ssel = reinterpret_cast<long long*>(tp_sm + off);
    off += align16((size_t)steps * sizeof(long long));
    T* xs = reinterpret_cast<T*>(tp_sm + off);
    const int tid = threadIdx.x;
    for (int e = tid; e < steps * l; e += kApplyThreads) Vs[e] = Vg[e];
    for (int t = tid; t < steps; t += kApplyThreads) {
        taus[t] = (T)taug[t];
        ssel[t] = sel[t];
    }
    __syncthreads();
    const int cl = tid / kApplyTpc, sub = tid % kApplyTpc;
    const int64_t j = i + (int64_t)blockIdx.x * kApplyCols + cl;
    const bool valid = j < n;
    int ts = -1;
    if (valid)
        for (int t = 0; t < steps; ++t)
            if (ssel[t] == j) ts = t;
    T* x = xs + (size_t)cl * l;
    T* bj = B + (valid ? j : i) * ldb;
    const bool doit = valid && ts < 0;
    if (valid && ts >= 0)
        for (int r = sub; r < l; r += kApplyTpc) bj[r] = Rg[(size_t)ts * l + r];
    if (doit)
        for (int r = sub; r < l; r += kApplyTpc) x[r] = bj[r];
    for (int t = 0; t < steps; ++t) {  // uniform trip count: every lane reaches the shuffles
        const T* v = Vs + (size_t)t * l;
        const int r0 = t + ((sub - (t % kApplyTpc)) + kApplyTpc) % kApplyTpc;
        T d = T(0);
        if (doit)
            for (int r = r0; r < l; r += kApplyTpc) d = fma(v[r], x[r], d);
        d = column_sum(d, kApplyTpc);
        if (doit) {
            const T dt = d * taus[t];
            for (int r = r0; r < l; r += kApplyTpc) x[r] = fma(-dt, v[r], x[r]);
        }
    }
    if (doit)
        for (int r = sub; r < l; r += kApplyTpc) bj[r] = x[r];
}

size_t final_smem(int bb, int l, int es)
{
    const int ldS = l | 1;
    size_t off = align16((size_t)bb * ldS * es) + align16((size_t)l * es) + (size_t)2 * bb * sizeof(long long) +
                 (size_t)4 * bb * sizeof(int);
    return ((off + 7) & ~(size_t)7) + finish_scratch_bytes(bb);
}

size_t apply_smem(int bb, int l, int es)
{
    return align16((size_t)bb * l * es) + align16((size_t)bb * es) + align16((size_t)bb * sizeof(long long)) +
           (size_t)kApplyCols * l * es;
}

size_t sel_smem_bytes(int nc, int l, int bb, int es)
{
    return es == 8 ? select_smem<double>(nc, l, bb) : select_smem<float>(nc, l, bb);
}

// Regions of the tournament workspace: two levels of choices (positions and counts), V, R_hat,
// tau, the step count.
struct TpRegions {
    size_t cand[2], cnt[2], V, R, tau, steps, total;
};
TpRegions tp_regions(int64_t n, int l, int64_t b, int es)
{
    const int64_t p0 = (n + b - 1) / b;  // leaf groups hold at least b columns
    TpRegions R{};
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = (off + bytes + 255) & ~(size_t)255;
        return o;
    };
    for (int q = 0; q < 2; ++q) {
        R.cand[q] = take((size_t)p0 * b * sizeof(long long));
        R.cnt[q] = take((size_t)p0 * sizeof(int));
    }
    R.V = take((size_t)l * b * es);
    R.R = take((size_t)l * b * es);
    R.tau = take((size_t)b * sizeof(double));
    R.steps = take(sizeof(int));
    R.total = off;
    return R;
}

}  // namespace

size_t tournament_ws_bytes(int64_t n, int l, int64_t b, int elem_bytes) { return tp_regions(n, l, b, elem_bytes).total; }

bool tournament_config(int64_t ncols, int bb, int64_t b, int l, int elem_bytes, int64_t group_cols, int64_t* gs_out,
                       int* fanin_out)
{
    if (l > kMaxL || bb < 1 || b < bb || ncols < bb) return false;
    if (dev_info().sms < 1 || dev_info().max_smem_optin < 4096) return false;  // no usable device
    const size_t cap = (size_t)dev_info().max_smem_optin - 1024;
    if (final_smem(bb, l, elem_bytes) > cap || apply_smem(bb, l, elem_bytes) > cap) return false;
    int fanin = kFanin;
    while (fanin > 2 && (fanin * bb > kSelMaxCols || sel_smem_bytes(fanin * bb, l, bb, elem_bytes) > cap)) --fanin;
    if (fanin * bb > kSelMaxCols || sel_smem_bytes(fanin * bb, l, bb, elem_bytes) > cap) return false;
    // the largest leaf group that one block holds
    int64_t gmax = kSelMaxCols;
    while (gmax > b && sel_smem_bytes((int)gmax, l, bb, elem_bytes) > cap) gmax -= 8;
    if (gmax < b || sel_smem_bytes((int)gmax, l, bb, elem_bytes) > cap) return false;
    int64_t gs;
    if (group_cols > 0) {
        if (group_cols < b || group_cols > gmax) return false;
        gs = group_cols;
    } else {
        const int64_t sms = dev_info().sms;
        gs = (ncols + sms - 1) / sms;
        if (gs < 2 * b) gs = 2 * b;
        if (gs > gmax) gs = gmax;
    }
    *gs_out = gs;
    *fanin_out = fanin;
    return true;
}

template <typename T>
cudaError_t launch_tournament(T* B, int64_t ldb, int l, int64_t n, int64_t i, int bb, int64_t b, int64_t gs,
                              int fanin, int32_t* jpvt, int32_t* piv, void* ws, long long* swapmap, T* tmp,
                              double guard_rel2, Status* st, cudaStream_t s)
{
    static DevFlag attr_set;
    if (!attr_set.done()) {
        if (cudaError_t e = allow_max_dynamic_smem(tp_select_kernel<T>)) return e;
        if (cudaError_t e = allow_max_dynamic_smem(tp_final_kernel<T>)) return e;
        if (cudaError_t e = allow_max_dynamic_smem(tp_apply_kernel<T>)) return e;
        attr_set.set();
    }
    const int es = (int)sizeof(T);
    const TpRegions R = tp_regions(n, l, b, es);
    char* w = static_cast<char*>(ws);
    long long* cand[2] = {reinterpret_cast<long long*>(w + R.cand[0]), reinterpret_cast<long long*>(w + R.cand[1])};
    int* cnt[2] = {reinterpret_cast<int*>(w + R.cnt[0]), reinterpret_cast<int*>(w + R.cnt[1])};
    T* V = reinterpret_cast<T*>(w + R.V);
    T* Rh = reinterpret_cast<T*>(w + R.R);
    double* tau = reinterpret_cast<double*>(w + R.tau);
    int* steps = reinterpret_cast<int*>(w + R.steps);
    const int64_t np = n - i;
    int nodes = (int)((np + gs - 1) / gs);
    // leaves
    {
        const int nc = (int)(gs < np ? gs : np);
        tp_select_kernel<T><<<nodes, select_threads(nc), select_smem<T>(nc, l, bb), s>>>(
            B, ldb, l, i, n, bb, gs, 0, nullptr, nullptr, 0, fanin, cand[0], cnt[0], select_tpc(nc), st);
    }
    int q = 0;
    while (nodes > 1) {  // one launch per level of the tree
        const int next = (nodes + fanin - 1) / fanin;
        const int nc = fanin * bb;
        tp_select_kernel<T><<<next, select_threads(nc), select_smem<T>(nc, l, bb), s>>>(
            B, ldb, l, i, n, bb, gs, 1, cand[q], cnt[q], nodes, fanin, cand[q ^ 1], cnt[q ^ 1], select_tpc(nc), st);
        q ^= 1;
        nodes = next;
    }
    tp_final_kernel<T><<<1, kFinalThreads, final_smem(bb, l, es), s>>>(B, ldb, l, i, bb, cand[q], jpvt, piv, swapmap, V,
                                                                      tau, Rh, steps, guard_rel2, st);
    tp_apply_kernel<T><<<(unsigned)((np + kApplyCols - 1) / kApplyCols), kApplyThreads, apply_smem(bb, l, es), s>>>(
        B, ldb, l, i, n, bb, cand[q], V, tau, Rh, steps, st);
    if (cudaError_t e = cudaGetLastError()) return e;
    // the chosen columns to i .. i+bb-1, the displaced ones to the chosen columns' old places
    return launch_swaps<T>(B, ldb, l, bb, swapmap, tmp, st, s);
}

template cudaError_t launch_tournament<double>(double*, int64_t, int, int64_t, int64_t, int, int64_t, int64_t, int,
                                               int32_t*, int32_t*, void*, long long*, double*, double, Status*,
                                               cudaStream_t);
template cudaError_t launch_tournament<float>(float*, int64_t, int, int64_t, int64_t, int, int64_t, int64_t, int,
                                              int32_t*, int32_t*, void*, long long*, float*, double, Status*,
                                              cudaStream_t);

}  // namespace rq
