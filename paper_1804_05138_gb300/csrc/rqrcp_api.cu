// rqrcp_api.cu -- C ABI of librqrcp: argument checks, workspace carving and the block loop of
// Alg. 2 (randomized QRCP) enqueued on the caller's stream.
//
// Per block i (bb = min(b, k-i)), all on one stream with no host synchronisation:
//   pivot   : partial QRCP on B(:, i:n)                     (cooperative kernel)
//   swaps   : move the chosen columns of A into place       (gather + scatter)
//   panel   : Householder QR of A(i:m, i:i+bb), FP64 reflector generation (cooperative kernel)
//   gemm_tn : [V^T V | V^T A(i:m, i+bb:n)] as split-K partials
//   tform   : T of the compact WY form I - V T V^T
//   reduce_y: Y = T^T V^T A(i:m, i+bb:n)
//   update  : A(i:m, i+bb:n) -= V Y                         (rows i..i+bb-1 become R12)
//   bupdate : Eq. (4) on the top bb rows of the trailing sketch
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>

#include "internal.cuh"

namespace rq {

namespace {
void query_dev_info(int d, DevInfo& out)
{
    out.sms = 0;
    out.max_smem_optin = 0;
    cudaDeviceGetAttribute(&out.sms, cudaDevAttrMultiProcessorCount, d);
    cudaDeviceGetAttribute(&out.max_smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, d);
    cudaGetLastError();
}
}  // namespace

// Attributes of the calling thread's current device, queried once per device (under a lock, so
// that concurrent first calls are safe); a device without a slot is queried on every call.
const DevInfo& dev_info()
{
    static DevInfo cache[kMaxDevices];
    static std::atomic<bool> have[kMaxDevices];
    static std::mutex mu;
    const int d = current_device();
    if (d < 0) {
        thread_local DevInfo uncached;
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess) cudaGetLastError();
        query_dev_info(dev, uncached);
        return uncached;
    }
    if (!have[d].load(std::memory_order_acquire)) {
        std::lock_guard<std::mutex> lock(mu);
        if (!have[d].load(std::memory_order_relaxed)) {
            query_dev_info(d, cache[d]);
            have[d].store(true, std::memory_order_release);
        }
    }
    return cache[d];
}

template <typename T>
cudaError_t launch_lowrank_rk(const T* Af, int64_t ldaf, int64_t k, int64_t n, double* Rk, cudaStream_t s);

// RQRCP_TENSOR_CORES=0 in the environment selects the SIMT contractions for the FP32 form.
bool tensor_cores_enabled()
{
    static int v = -1;
    if (v < 0) {
        const char* e = getenv("RQRCP_TENSOR_CORES");
        v = (e != nullptr && e[0] == '0') ? 0 : 1;
    }
    return v == 1;
}
// Paired block steps of the FP32 form (two blocks, one update pass) run where the trailing matrix is
// larger than about this part's L2 (129 MB): below that the pass they save is served from L2 and
// their extra launches cost more.  RQRCP_PAIRED=0 in the environment turns them off, =1 uses them at
// every size (for A/B timing and tests).
constexpr double kPairMinBytes = 128.0 * 1024 * 1024;
int paired_mode()  // 0 off, 1 always, 2 by size
{
    static int v = -1;
    if (v < 0) {
        const char* e = getenv("RQRCP_PAIRED");
        v = (e != nullptr && e[0] == '0') ? 0 : (e != nullptr && e[0] == '1') ? 1 : 2;
    }
    return v;
}
// RQRCP_PANEL=householder in the environment keeps the FP32 form on the cooperative Householder
// panel (one grid-wide step per column) instead of the CholeskyQR2 panel, for A/B timing.
bool cholqr_enabled()
{
    static int v = -1;
    if (v < 0) {
        const char* e = getenv("RQRCP_PANEL");
        v = (e != nullptr && (e[0] == 'h' || e[0] == 'H')) ? 0 : 1;
    }
    return v == 1;
}
template <typename T>
cudaError_t launch_eye(T* Q, int64_t ldq, int64_t m, int64_t k, cudaStream_t s);

namespace {

constexpr int kMaxSplit = 16;
constexpr size_t kAlign = 256;

size_t align_up(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }

struct Layout {
    size_t status, omega, B, Bc, P, Y, Tm, What, piv, cand, part, tmp, xs, cqr, tp, Y2, total;
};

Layout make_layout(int64_t m, int64_t n, int64_t b, int64_t p, size_t esz)
{
    const int64_t l = b + p;
    Layout L{};
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = align_up(off + bytes);
        return o;
    };
    L.status = take(sizeof(Status));
    L.omega = take((size_t)l * m * esz);
    L.B = take((size_t)l * n * esz);
    // FP64 form: the untransformed copy of the sketch that Eq. (5) updates
    L.Bc = take(esz == sizeof(double) ? (size_t)l * n * esz : 0);
    // one split more than the contractions use: a paired block step's correction (FP32 form)
    L.P = take((size_t)(kMaxSplit + 1) * n * (size_t)(l > b ? l : b) * sizeof(double));
    // Y holds T^T W for the trailing columns, and for the l columns of Omega_bar^T under Eq. (5)
    L.Y = take((size_t)b * (size_t)(n > l ? n : l) * sizeof(double));
    L.Tm = take((size_t)b * b * sizeof(double));
    L.What = take((size_t)b * b * sizeof(double));
    L.piv = take((size_t)b * sizeof(int32_t));
    L.cand = take(pivot_cand_bytes((int)l) + sizeof(long long) * (1 + 4 * (size_t)b));
    L.part = take(panel_part_bytes((int)b));
    L.tmp = take((size_t)2 * b * (size_t)(m > l ? m : l) * esz);  // 2b columns of A, or of the sketch
    {
        // TF32 parts of Omega / V (contraction) and of Y (update); used one after the other
        const size_t xs = tc_xsplit_bytes(l > b ? l : b, m), ys = tc_update_ws_bytes(n, 128);
        L.xs = take(esz == sizeof(float) ? (xs > ys ? xs : ys) : 0);
    }
    // FP32 form: the CholeskyQR2 panel's partial Grams, factors and Q1 (m x 64)
    L.cqr = take(esz == sizeof(float) ? cholqr_ws_bytes(m) : 0);
    // QR with tournament pivoting: the tree's choices, the root's reflectors and R_hat columns
    L.tp = take(tournament_ws_bytes(n, (int)l, b, (int)esz));
    // FP32 form, paired block steps: block i+1's Y
    L.Y2 = take(esz == sizeof(float) ? (size_t)b * n * sizeof(double) : 0);
    L.total = off;
    return L;
}

// Split-K factor for an M x N result contracted over K on the SIMT contraction (tiles of
// gemm_tn_tile_rows(M) x 64): the split count S <= max_split minimising waves x (rows per split + a
// fixed cost of 64 rows), a wave being the blocks resident on the whole GPU at once; splits of at
// least 64 rows.
void choose_split(int64_t M, int64_t N, int64_t K, int& nsplit, int64_t& kchunk, int elem_bytes = 8,
                  int64_t max_split = kMaxSplit)
{
    const int64_t tr = gemm_tn_tile_rows(M);
    const int64_t tiles = ((M + tr - 1) / tr) * ((N + 63) / 64);
    const int64_t wave = (int64_t)gemm_tn_blocks_per_sm(elem_bytes, M) * dev_info().sms;
    int64_t smax = (K + 63) / 64;
    if (smax > max_split) smax = max_split;
    if (smax < 1) smax = 1;
    int64_t best = 1, best_cost = -1;
    for (int64_t S = 1; S <= smax; ++S) {
        const int64_t rows = ((K + S - 1) / S + 15) / 16 * 16;
        const int64_t waves = (tiles * S + wave - 1) / wave;
        const int64_t cost = waves * (rows + 64);
        if (best_cost < 0 || cost < best_cost) {
            best_cost = cost;
            best = S;
        }
    }
    kchunk = (K + best - 1) / best;
    kchunk = ((kchunk + 15) / 16) * 16;
    nsplit = (int)((K + kchunk - 1) / kchunk);
}

template <typename T>
struct Prec;
template <>
struct Prec<double> {
    static constexpr double unit_roundoff = 1.1102230246251565e-16;  // 2^-53
};
template <>
struct Prec<float> {
    static constexpr double unit_roundoff = 5.9604644775390625e-08;  // 2^-24
};

#define RQ_CHECK(expr)                          \
    do {                                        \
        if ((expr) != cudaSuccess) {            \
            cudaGetLastError();                 \
            return RQRCP_ERR_CUDA;              \
        }                                       \
    } while (0)

// Launch with optional event bracketing and the algorithmic work of the launch.
#define RQ_LAUNCH(cls, flops, bytes, expr)                      \
    do {                                                        \
        const bool prof_ = prof_on();                           \
        if (prof_) prof_begin((cls), s);                        \
        RQ_CHECK(expr);                                         \
        if (prof_) prof_end((cls), (double)(flops), (double)(bytes), s); \
    } while (0)

int check_work(void* work, size_t work_bytes, size_t need)
{
    if (work == nullptr || (reinterpret_cast<uintptr_t>(work) & (kAlign - 1)) != 0 || work_bytes < need)
        return RQRCP_ERR_WORKSPACE;
    return RQRCP_OK;
}

template <typename T>
int factor_impl(int64_t m, int64_t n, T* A, int64_t lda, int64_t k, int64_t b, int64_t p, uint64_t seed,
                const T* Omega_user, int64_t ldo, int32_t* jpvt, double* tau, int64_t* rank_out, void* work,
                size_t work_bytes, cudaStream_t s, int sketch_bf16 = 0, int formula = RQRCP_UPDATE_EQ4,
                bool final_b = false, int64_t tp_group = -1)
{
    const int64_t l = b + p;
    const Layout L = make_layout(m, n, b, p, sizeof(T));
    if (int e = check_work(work, work_bytes, L.total)) return e;
    if (l > 1024 || b > 128 || !pivot_fits(n, (int)l, (int)sizeof(T)) || !panel_fits(m, (int)b, (int)sizeof(T)))
        return RQRCP_ERR_UNSUPPORTED;
    char* w = static_cast<char*>(work);
    Status* st = reinterpret_cast<Status*>(w + L.status);
    T* Om = reinterpret_cast<T*>(w + L.omega);
    T* B = reinterpret_cast<T*>(w + L.B);
    double* P = reinterpret_cast<double*>(w + L.P);
    double* Y = reinterpret_cast<double*>(w + L.Y);
    double* Tm = reinterpret_cast<double*>(w + L.Tm);
    double* What = reinterpret_cast<double*>(w + L.What);
    int32_t* piv = reinterpret_cast<int32_t*>(w + L.piv);
    void* cand = w + L.cand;
    const long long* swapmap = reinterpret_cast<const long long*>(w + L.cand + pivot_cand_bytes((int)l));
    double* part = reinterpret_cast<double*>(w + L.part);
    T* tmp = reinterpret_cast<T*>(w + L.tmp);
    T* Bc = reinterpret_cast<T*>(w + L.Bc);
    const bool eq5 = formula == RQRCP_UPDATE_EQ5;
    if (eq5 && sizeof(T) != sizeof(double)) return RQRCP_ERR_UNSUPPORTED;
    // tp_group >= 0: QR with tournament pivoting on B (Eq. (4) only); every block must fit one SM
    const bool tourn = tp_group >= 0;
    if (tourn) {
        if (eq5) return RQRCP_ERR_UNSUPPORTED;
        for (int64_t i = 0; i < k; i += b) {
            int64_t gs;
            int fan;
            if (!tournament_config(n - i, (int)(b < k - i ? b : k - i), b, (int)l, (int)sizeof(T), tp_group, &gs, &fan))
                return RQRCP_ERR_UNSUPPORTED;
        }
    }

    RQ_CHECK(launch_init(st, k, jpvt, n, s));
    RQ_CHECK(cudaMemsetAsync(cand, 0, pivot_slot_bytes(), s));
    const double es = (double)sizeof(T);
    const T* Omega = Omega_user;
    if (Omega == nullptr) {
        RQ_LAUNCH(K_OMEGA, 0, l * m * es, launch_omega<T>(l, m, seed, Om, m, s));
        Omega = Om;
        ldo = m;
    } else if (eq5) {  // Eq. (5) updates Omega_bar = Omega Q in place: work on a copy
        RQ_CHECK(cudaMemcpy2DAsync(Om, (size_t)m * sizeof(T), Omega_user, (size_t)ldo * sizeof(T),
                                   (size_t)m * sizeof(T), (size_t)l, cudaMemcpyDeviceToDevice, s));
        Omega = Om;
        ldo = m;
    }
    // Alg. 2: B = Omega A
    {
        int ns;
        int64_t kc;
        // FP32 form: the BF16 sketch (operands rounded to BF16, FP32 accumulation) or the
        // FP32-accurate one; both on the tensor cores when the layout allows
        const int bf = sizeof(T) == 4 && sketch_bf16 ? 1 : 0;
        const bool tc = sizeof(T) == 4 && tensor_cores_enabled() && tc_gemm_supported(l, lda, (const void*)A, bf);
        if (tc) {
            kc = tc_kchunk(n, m, ns, bf, l);
            RQ_LAUNCH(K_SKETCH_GEMM, 2.0 * l * m * n, (double)m * n * es + (double)l * m * es,
                      launch_gemm_tn_tc((const float*)Omega, ldo, (const float*)A, lda, l, n, m, kc, P, 0, 0,
                                        reinterpret_cast<float*>(w + L.xs), st, s, bf));
        } else {
            choose_split(l, n, m, ns, kc, (int)sizeof(T));
            RQ_LAUNCH(K_SKETCH_GEMM, 2.0 * l * m * n, (double)m * n * es + (double)l * m * es,
                      launch_gemm_tn<T>(Omega, ldo, A, lda, l, n, m, kc, P, 0, 0, st, s, bf));
        }
        RQ_LAUNCH(K_SKETCH_REDUCE, 0, (double)ns * l * n * 8 + (double)l * n * es,
                  launch_sketch_reduce<T>(P, ns, l, n, B, l, st, s));
        if (eq5) RQ_CHECK(cudaMemcpyAsync(Bc, B, (size_t)l * n * sizeof(T), cudaMemcpyDeviceToDevice, s));
    }
    // guard tolerance: 10 max(m,n) u for FP64 (the oracle's reading); FP32 storage uses
    // 10 sqrt(max(m,n)) u, about ten times the rounding noise of an FP32 sketch column; the BF16
    // sketch 2^-6, about five times the 2^-8.5 relative noise its operand rounding leaves in a
    // sketch column
    const double mn = (double)(m > n ? m : n);
    const double gtol = (sizeof(T) == 4 && sketch_bf16) ? ldexp(1.0, -6)
                                                        : 10.0 * (sizeof(T) == 8 ? mn : sqrt(mn)) * Prec<T>::unit_roundoff;
    const double guard_rel2 = gtol * gtol;
    // pivots on the sketch (Alg. 2: partial QRCP on B(:, i:n)) and the column swaps of A
    auto pivot_swap = [&](int64_t i, int bb) -> int {
        const double np = (double)(n - i);
        if (tourn) {
            int64_t gs;
            int fan;
            tournament_config(n - i, bb, b, (int)l, (int)sizeof(T), tp_group, &gs, &fan);
            RQ_LAUNCH(K_PIVOT, 4.0 * l * np * bb, 2.0 * l * np * es,
                      launch_tournament<T>(B, l, (int)l, n, i, bb, b, gs, fan, jpvt, piv, w + L.tp,
                                           const_cast<long long*>(swapmap), tmp, guard_rel2, st, s));
        } else {
            RQ_LAUNCH(K_PIVOT, 4.0 * l * np * bb, 2.0 * l * np * es,
                      launch_pivot<T>(B, l, (int)l, n, i, bb, jpvt, piv, cand, guard_rel2, st, s, (int)(i / b)));
        }
        RQ_LAUNCH(K_SWAP, 0, 4.0 * bb * m * es, launch_swaps<T>(A, lda, m, bb, swapmap, tmp, st, s));
        if (eq5 && i + bb < k)  // the same column moves on the untransformed sketch
            RQ_LAUNCH(K_SWAP, 0, 4.0 * bb * l * es, launch_swaps<T>(Bc, l, l, bb, swapmap, tmp, st, s));
        return RQRCP_OK;
    };
    // unpivoted QR of the panel A(i:m, i:i+bb)
    auto panel = [&](int64_t i, int bb) -> int {
        T* Vp = A + i * lda + i;
        const int64_t mr = m - i;
        if (sizeof(T) == 4 && cholqr_enabled() && cholqr_supported(bb)) {
            // CholeskyQR2 + Householder reconstruction; the cooperative Householder panel after it
            // returns at once unless the panel was too ill-conditioned for CholeskyQR2
            int* cqr_flag = nullptr;
            const bool prof_ = prof_on();
            if (prof_) prof_begin(K_PANEL, s);
            RQ_CHECK(launch_cholqr_panel(reinterpret_cast<float*>(Vp), lda, mr, bb, tau + i, w + L.cqr, &cqr_flag, st,
                                         s));
            RQ_CHECK(launch_panel<T>(Vp, lda, mr, bb, tau + i, part, st, s, cqr_flag));
            if (prof_) prof_end(K_PANEL, 2.0 * mr * bb * bb - 2.0 * bb * bb * bb / 3.0, 2.0 * mr * bb * es, s);
        } else {
            RQ_LAUNCH(K_PANEL, 2.0 * mr * bb * bb - 2.0 * bb * bb * bb / 3.0, 2.0 * mr * bb * es,
                      launch_panel<T>(Vp, lda, mr, bb, tau + i, part, st, s));
        }
        return RQRCP_OK;
    };
    // [V^T V | V^T C] over rows i..m-1 and columns i..n-1 into the split partials P (ns splits)
    auto gram = [&](int64_t i, int bb, bool tc, int& ns) -> int {
        T* Vp = A + i * lda + i;
        const int64_t mr = m - i;
        const double np = (double)(n - i);
        int64_t kc;
        if (tc) {
            kc = tc_kchunk(n - i, mr, ns, 0, bb);
            RQ_LAUNCH(K_WY_GEMM, 2.0 * bb * mr * np, (double)mr * np * es,
                      launch_gemm_tn_tc((const float*)Vp, lda, (const float*)Vp, lda, bb, n - i, mr, kc, P, bb, bb,
                                        reinterpret_cast<float*>(w + L.xs), st, s));
        } else {
            choose_split(bb, n - i, mr, ns, kc, (int)sizeof(T));
            RQ_LAUNCH(K_WY_GEMM, 2.0 * bb * mr * np, (double)mr * np * es,
                      launch_gemm_tn<T>(Vp, lda, Vp, lda, bb, n - i, mr, kc, P, 1, bb, st, s));
        }
        return RQRCP_OK;
    };
    for (int64_t i = 0; i < k; i += b) {
        const int bb = (int)(b < k - i ? b : k - i);
        if (int e = pivot_swap(i, bb)) return e;
        if (int e = panel(i, bb)) return e;
        T* Vp = A + i * lda + i;
        const int64_t mr = m - i;
        const int64_t nt = n - i - bb;
        if (nt <= 0) continue;
        const bool tc = sizeof(T) == 4 && tensor_cores_enabled() && tc_gemm_supported(bb, lda, (const void*)Vp);
        int ns;
        if (int e = gram(i, bb, tc, ns)) return e;
        RQ_LAUNCH(K_TFORM, (double)bb * bb * bb / 3.0, (double)ns * bb * bb * 8,
                  launch_tform(P, ns, n - i, bb, tau + i, Tm, st, s));
        RQ_LAUNCH(K_REDUCE_Y, (double)bb * bb * nt, ((double)ns + 1.0) * bb * nt * 8,
                  launch_reduce_y(P, ns, n - i, bb, bb, Tm, 1, Y, nt, st, s, sizeof(T) == 4 ? 1 : 0));
        // FP32 form: blocks i and i + 1 share one pass of the trailing update.  Block i updates now
        // only what block i + 1 needs (its R12 rows for Eq. (4), then, after block i + 1's pivots,
        // the panel's columns); block i + 1's Gram is taken from the trailing matrix before block i's
        // update and corrected by (V1^T V0) Y0; then C -= [V0 V1] [Y0; Y1] in one pass (K = 2b).
        const int64_t j = i + bb;
        const int pmode = paired_mode();
        const bool big = (double)(m - j) * (double)(n - j - b) * sizeof(float) >= kPairMinBytes;
        const bool pair = sizeof(T) == 4 && tc && !eq5 && (pmode == 1 || (pmode == 2 && big)) && bb == b && b <= 64 &&
                          j + b <= k &&
                          n - j - b > 0 && tc_update_supported(bb, lda, (const void*)(Vp + (int64_t)bb * lda)) &&
                          tc_update_supported(bb, lda, (const void*)(A + j * lda + j)) &&
                          tc_update2_supported(lda, (const void*)(A + (j + b) * lda + j)) &&
                          tc_gemm_supported(b, lda, (const void*)(A + j * lda + j));
        if (!pair) {
            if (sizeof(T) == 4 && tensor_cores_enabled() && tc_update_supported(bb, lda, Vp + (int64_t)bb * lda))
                RQ_LAUNCH(K_WY_UPDATE, 2.0 * bb * mr * nt, 2.0 * mr * nt * es + (double)mr * bb * es,
                          launch_gemm_update_tc((float*)(Vp + (int64_t)bb * lda), lda, (const float*)Vp, lda, Y, bb, mr,
                                                nt, bb, bb, reinterpret_cast<float*>(w + L.xs), st, s));
            else
                RQ_LAUNCH(K_WY_UPDATE, 2.0 * bb * mr * nt, 2.0 * mr * nt * es + (double)mr * bb * es,
                          launch_gemm_update<T>(Vp + (int64_t)bb * lda, lda, Vp, lda, Y, bb, mr, nt, bb, 1, nullptr, st,
                                                s));
            // final_b: also after the last block, so that B sketches R22 (Alg. 3 reads its norms)
            if ((i + bb < k || final_b) && !eq5)
                RQ_LAUNCH(K_BUPDATE, (double)bb * bb * bb / 3.0 + (double)bb * bb * nt, 2.0 * bb * nt * es,
                          launch_bupdate<T>(B, l, A, lda, i, bb, n, What, st, s));
            if (i + bb < k && eq5) {
                // Eq. (5): Omega_bar <- Omega_bar Q_tilde, i.e. Omega_bar^T(i:m, :) <- Q_tilde^T
                // Omega_bar^T(i:m, :), the compact-WY update of the trailing matrix with C the m x l
                // column-major view of the row-major Omega_bar; then B2 <- B2 - Omega_bar_1 R12.
                T* OmT = Om + i;
                int ns2;
                int64_t kc2;
                // only bb x l outputs (two 64-wide tiles): more K splits than kMaxSplit, as many as
                // the partial buffer (kMaxSplit * n * max(l, b) doubles) holds, keep the GPU busy
                const int64_t pcap = (int64_t)kMaxSplit * n * (l > b ? l : b);
                choose_split(bb, l, mr, ns2, kc2, (int)sizeof(T), pcap / ((int64_t)bb * l));
                RQ_LAUNCH(K_BUPDATE, 2.0 * bb * mr * l, (double)mr * l * es,
                          launch_gemm_tn<T>(Vp, lda, OmT, m, bb, l, mr, kc2, P, 1, 0, st, s));
                RQ_LAUNCH(K_BUPDATE, (double)bb * bb * l, ((double)ns2 + 1.0) * bb * l * 8,
                          launch_reduce_y(P, ns2, l, 0, bb, Tm, 1, Y, l, st, s));
                RQ_LAUNCH(K_BUPDATE, 2.0 * bb * mr * l, 2.0 * mr * l * es,
                          launch_gemm_update<T>(OmT, m, Vp, lda, Y, bb, mr, l, bb, 1, nullptr, st, s));
                choose_split(l, nt, bb, ns2, kc2, (int)sizeof(T));
                RQ_LAUNCH(K_BUPDATE, 2.0 * l * bb * nt, (double)bb * nt * es + (double)l * bb * es,
                          launch_gemm_tn<T>(OmT, m, Vp + (int64_t)bb * lda, lda, l, nt, bb, kc2, P, 0, 0, st, s));
                RQ_LAUNCH(K_BUPDATE, 0, (double)ns2 * l * nt * 8 + 3.0 * l * nt * es,
                          launch_bfinish<T>(B, Bc, (int)l, i + bb, nt, P, ns2, st, s));
            }
            continue;
        }
        float* xs = reinterpret_cast<float*>(w + L.xs);
        double* Y1 = reinterpret_cast<double*>(w + L.Y2);
        // block i: its R12 rows (rows i..j-1 of the trailing columns), then Eq. (4)
        RQ_LAUNCH(K_WY_UPDATE, 2.0 * bb * bb * nt, 2.0 * bb * nt * es,
                  launch_gemm_update_tc((float*)(Vp + (int64_t)bb * lda), lda, (const float*)Vp, lda, Y, bb, bb, nt, bb,
                                        bb, xs, st, s));
        RQ_LAUNCH(K_BUPDATE, (double)bb * bb * bb / 3.0 + (double)bb * bb * nt, 2.0 * bb * nt * es,
                  launch_bupdate<T>(B, l, A, lda, i, bb, n, What, st, s));
        // block i + 1: pivots and swaps (Y0's columns follow A's), then its panel's columns take block
        // i's update (rows j..m-1) before the panel is factored
        if (int e = pivot_swap(j, b)) return e;
        RQ_LAUNCH(K_SWAP, 0, 4.0 * b * bb * 8,
                  launch_swaps<double>(Y - j * bb, bb, bb, b, swapmap, reinterpret_cast<double*>(tmp), st, s));
        const int64_t mr1 = m - j, nt1 = n - j - b;
        float* const A0low = (float*)(A + i * lda + j);  // V0's rows j..m-1 (below its triangle)
        RQ_LAUNCH(K_WY_UPDATE, 2.0 * bb * mr1 * b, 2.0 * mr1 * b * es + (double)mr1 * bb * es,
                  launch_gemm_update_tc((float*)(A + j * lda + j), lda, A0low, lda, Y, bb, mr1, b, bb, 0, xs, st, s));
        if (int e = panel(j, b)) return e;
        // block i + 1's Gram over rows j..m-1 of columns i..n-1 before block i's update, in one pass:
        // V1^T [V0low V1 C] (V1's reflector mask on the second 64 columns); partial column c holds
        // V1^T V0low for c < bb, V1^T V1 for bb <= c < bb + b, and V1^T C beyond
        {
            int ns1;
            const int64_t nc1 = n - i;
            const int64_t kc1 = tc_kchunk(nc1, mr1, ns1, 0, b);
            RQ_LAUNCH(K_WY_GEMM, 2.0 * b * mr1 * (double)nc1, (double)mr1 * nc1 * es,
                      launch_gemm_tn_tc((const float*)(A + j * lda + j), lda, A0low, lda, b, nc1, mr1, kc1, P, b, b, xs,
                                        st, s, 0, bb));
            RQ_LAUNCH(K_TFORM, (double)b * b * b / 3.0, (double)ns1 * b * b * 8,
                      launch_tform(P + (size_t)bb * b, ns1, nc1, b, tau + j, Tm, st, s));
            // V1^T V0low summed into split 0, then the correction -(V1^T V0low) Y0 as split ns1, then
            // Y1 = T1^T (W1 + correction)
            if (ns1 > 1)
                RQ_LAUNCH(K_REDUCE_Y, (double)ns1 * b * bb, (double)(ns1 + 1) * b * bb * 8,
                          launch_split_sum(P, ns1, (int64_t)b * bb, nc1 * b, st, s));
            RQ_LAUNCH(K_REDUCE_Y, 2.0 * b * bb * nt1, (double)bb * nt1 * 8 * 2,
                      launch_wy_corr(P, b, Y, bb, b, nt1, bb + b, P + (size_t)ns1 * nc1 * b, st, s));
            RQ_LAUNCH(K_REDUCE_Y, (double)b * b * nt1, ((double)ns1 + 2.0) * b * nt1 * 8,
                      launch_reduce_y(P, ns1 + 1, nc1, bb + b, b, Tm, 1, Y1, nt1, st, s, 1));
        }
        // the trailing matrix of block i + 1, rows j..m-1: C -= [V0low V1] [Y0(:, b:); Y1]
        RQ_LAUNCH(K_WY_UPDATE, 2.0 * (bb + b) * mr1 * nt1, 2.0 * mr1 * nt1 * es + (double)mr1 * (bb + b) * es,
                  launch_gemm_update_tc2((float*)(A + (j + b) * lda + j), lda, A0low, lda, Y + (int64_t)b * bb, bb, Y1,
                                         b, bb, mr1, nt1, bb + b, b, bb, xs, st, s));
        if (j + b < k || final_b)
            RQ_LAUNCH(K_BUPDATE, (double)b * b * b / 3.0 + (double)b * b * nt1, 2.0 * b * nt1 * es,
                      launch_bupdate<T>(B, l, A, lda, j, b, n, What, st, s));
        i += b;  // block i + 1 is done
    }
    if (rank_out != nullptr)
        RQ_CHECK(cudaMemcpyAsync(rank_out, &st->rank, sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
    return RQRCP_OK;
}

// Alg. 3 workspace: the RQRCP layout, then r (n), the Gaussian and X of the g_2 estimate
// (d*(l+1) each), the Givens pairs (2*(l+1)), info (4) and the RQRCP stage's tau (l).
struct SrqrLayout {
    Layout f;
    size_t r, Og, X, cs, info, tau, total;
};

SrqrLayout make_srqr_layout(int64_t m, int64_t n, int64_t l, int64_t b, int64_t p, int64_t d)
{
    SrqrLayout S{};
    S.f = make_layout(m, n, b, p, sizeof(double));
    size_t off = S.f.total;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = align_up(off + bytes);
        return o;
    };
    S.r = take(sizeof(double) * (size_t)n);
    S.Og = take(sizeof(double) * (size_t)d * (size_t)(l + 1));
    S.X = take(sizeof(double) * (size_t)d * (size_t)(l + 1));
    S.cs = take(sizeof(double) * 2 * (size_t)(l + 1));
    S.info = take(sizeof(double) * 4);
    S.tau = take(sizeof(double) * (size_t)l);
    S.total = off;
    return S;
}

int validate_factor(int64_t m, int64_t n, const void* A, int64_t lda, int64_t k, int64_t b, int64_t p,
                    const void* jpvt, const void* tau)
{
    if (m < 1) return -1;
    if (n < 1) return -2;
    if (A == nullptr) return -3;
    if (lda < m) return -4;
    if (k < 1 || k > (m < n ? m : n)) return -5;
    if (b < 1) return -6;
    if (p < 0) return -7;
    if (jpvt == nullptr) return -9;
    if (tau == nullptr) return -10;
    return 0;
}

}  // namespace
}  // namespace rq

using namespace rq;

extern "C" size_t rqrcp_lowrank_workspace_size(int64_t m, int64_t n, int64_t k);

namespace rq {
namespace {
template <typename T>
int lowrank_impl(int64_t m, int64_t n, int64_t k, const T* Afact, int64_t ldaf, const double* tau,
                 const int32_t* jpvt, T* L, int64_t ldl, T* Q1, int64_t ldq, void* work, size_t work_bytes,
                 void* stream)
{
    if (m < 1) return -1;
    if (n < 1) return -2;
    if (k < 1 || k > (m < n ? m : n)) return -3;
    if (Afact == nullptr) return -4;
    if (ldaf < m) return -5;
    if (tau == nullptr) return -6;
    if (L != nullptr && jpvt == nullptr) return -7;
    if (L != nullptr && ldl < m) return -9;
    if (Q1 == nullptr) return -10;
    if (ldq < m) return -11;
    const size_t need = rqrcp_lowrank_workspace_size(m, n, k);
    if (int e = check_work(work, work_bytes, need)) return e;
    cudaStream_t s = (cudaStream_t)stream;
    if (sizeof(T) == 4 && lowrank_f32_tc_ok(k, reinterpret_cast<const float*>(Afact), ldaf,
                                            reinterpret_cast<const float*>(Q1), ldq))
        return lowrank_f32_tc(m, n, k, reinterpret_cast<const float*>(Afact), ldaf, tau, jpvt,
                              reinterpret_cast<float*>(L), ldl, reinterpret_cast<float*>(Q1), ldq, work, s);
    const int64_t bb = 64;
    char* w = static_cast<char*>(work);
    size_t off = 0;
    Status* st = reinterpret_cast<Status*>(w);
    off = align_up(off + sizeof(Status));
    double* P = reinterpret_cast<double*>(w + off);
    off = align_up(off + (size_t)kMaxSplit * (size_t)(k > bb ? k : bb) * bb * sizeof(double));
    double* Tm = reinterpret_cast<double*>(w + off);
    off = align_up(off + (size_t)bb * bb * sizeof(double));
    double* Y = reinterpret_cast<double*>(w + off);
    RQ_CHECK(launch_init(st, k, nullptr, 0, s));
    // Q1 = H_0 ... H_{k-1} I(:, 0:k), accumulated backwards block by block:
    // Q1(i:m, :) <- (I - V T V^T) Q1(i:m, :).
    RQ_CHECK(launch_eye<T>(Q1, ldq, m, k, s));
    const int64_t last = ((k - 1) / bb) * bb;
    for (int64_t i = last; i >= 0; i -= bb) {
        const int kb = (int)(bb < k - i ? bb : k - i);
        const T* Vp = Afact + i * ldaf + i;
        const int64_t mr = m - i;
        int ns;
        int64_t kc;
        choose_split(kb, kb, mr, ns, kc, (int)sizeof(T));
        RQ_CHECK(launch_gemm_tn<T>(Vp, ldaf, Vp, ldaf, kb, kb, mr, kc, P, 1, kb, st, s));
        RQ_CHECK(launch_tform(P, ns, kb, kb, tau + i, Tm, st, s));
        const int64_t nq = k - i;  // columns of Q1 touched by this block: i..k-1
        choose_split(kb, nq, mr, ns, kc, (int)sizeof(T));
        RQ_CHECK(launch_gemm_tn<T>(Vp, ldaf, Q1 + i * ldq + i, ldq, kb, nq, mr, kc, P, 1, 0, st, s));
        RQ_CHECK(launch_reduce_y(P, ns, nq, 0, kb, Tm, 0, Y, nq, st, s));
        RQ_CHECK(launch_gemm_update<T>(Q1 + i * ldq + i, ldq, Vp, ldaf, Y, kb, mr, nq, kb, 1, nullptr, st, s));
    }
    // L(:, jpvt[c]) = Q1 [R11 R12](:, c)  as  L -= Q1 (-Rk) with a column scatter.
    if (L == nullptr) return RQRCP_OK;
    RQ_CHECK(launch_lowrank_rk<T>(Afact, ldaf, k, n, Y, s));
    RQ_CHECK(cudaMemset2DAsync(L, ldl * sizeof(T), 0, m * sizeof(T), n, s));
    RQ_CHECK(launch_gemm_update<T>(L, ldl, Q1, ldq, Y, k, m, n, k, 0, jpvt, st, s));
    return RQRCP_OK;
}

}  // namespace

// Q1 only (no low-rank product, no permutation), for the FP64 reorthogonalisation path.
template <typename T>
int lowrank_q1_only(int64_t m, int64_t k, const T* Afact, int64_t ldaf, const double* tau, T* Q1, int64_t ldq,
                    void* work, size_t work_bytes, cudaStream_t s)
{
    return lowrank_impl<T>(m, k, k, Afact, ldaf, tau, nullptr, nullptr, m, Q1, ldq, work, work_bytes, s);
}
template int lowrank_q1_only<double>(int64_t, int64_t, const double*, int64_t, const double*, double*, int64_t,
                                     void*, size_t, cudaStream_t);

}  // namespace rq

extern "C" {

__attribute__((visibility("default"))) const char* rqrcp_error_string(int code)
{
    if (code < 0) return "invalid argument (the negated return value is its 1-based position)";
    switch (code) {
    case RQRCP_OK: return "success";
    case RQRCP_ERR_CUDA: return "a CUDA runtime call failed";
    case RQRCP_ERR_NONFINITE: return "the sketch of A is not finite (A holds NaN or Inf)";
    case RQRCP_ERR_TIMEOUT: return "a grid-wide barrier timed out inside a kernel";
    case RQRCP_ERR_WORKSPACE: return "workspace missing, misaligned (256 B) or too small";
    case RQRCP_ERR_UNSUPPORTED: return "shape beyond what the library keeps in shared memory";
    default: return "unknown error code";
    }
}

__attribute__((visibility("default"))) size_t rqrcp_workspace_size(int64_t m, int64_t n, int64_t k, int64_t b,
                                                                   int64_t p, int precision)
{
    if (m < 1 || n < 1 || k < 1 || b < 1 || p < 0) return 0;
    if (precision != RQRCP_PREC_FP64 && precision != RQRCP_PREC_MIXED) return 0;
    return make_layout(m, n, b, p, precision == RQRCP_PREC_FP64 ? sizeof(double) : sizeof(float)).total;
}

__attribute__((visibility("default"))) int rqrcp_generate_omega(int64_t l, int64_t m, uint64_t seed, double* Omega,
                                                                int64_t ldo, void* stream)
{
    if (l < 1) return -1;
    if (m < 1) return -2;
    if (Omega == nullptr) return -4;
    if (ldo < m) return -5;
    return launch_omega<double>(l, m, seed, Omega, ldo, (cudaStream_t)stream) == cudaSuccess ? RQRCP_OK
                                                                                             : RQRCP_ERR_CUDA;
}

__attribute__((visibility("default"))) int rqrcp_generate_omega_f32(int64_t l, int64_t m, uint64_t seed, float* Omega,
                                                                    int64_t ldo, void* stream)
{
    if (l < 1) return -1;
    if (m < 1) return -2;
    if (Omega == nullptr) return -4;
    if (ldo < m) return -5;
    return launch_omega<float>(l, m, seed, Omega, ldo, (cudaStream_t)stream) == cudaSuccess ? RQRCP_OK
                                                                                            : RQRCP_ERR_CUDA;
}

__attribute__((visibility("default"))) int rqrcp_sketch(int64_t m, int64_t n, const double* A, int64_t lda,
                                                        const double* Omega, int64_t l, int64_t ldo, double* B,
                                                        int64_t ldb, void* work, size_t work_bytes, void* stream)
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
    const Layout L = make_layout(m, n, l, 0, sizeof(double));
    if (int e = check_work(work, work_bytes, L.total)) return e;
    cudaStream_t s = (cudaStream_t)stream;
    char* w = static_cast<char*>(work);
    Status* st = reinterpret_cast<Status*>(w + L.status);
    double* P = reinterpret_cast<double*>(w + L.P);
    RQ_CHECK(launch_init(st, 0, nullptr, 0, s));
    int ns;
    int64_t kc;
    choose_split(l, n, m, ns, kc);
    RQ_CHECK(launch_gemm_tn<double>(Omega, ldo, A, lda, l, n, m, kc, P, 0, 0, st, s));
    RQ_CHECK(launch_sketch_reduce<double>(P, ns, l, n, B, ldb, st, s));
    return RQRCP_OK;
}

__attribute__((visibility("default"))) int rqrcp_factor(int64_t m, int64_t n, double* A, int64_t lda, int64_t k,
                                                        int64_t b, int64_t p, uint64_t seed, int32_t* jpvt,
                                                        double* tau, int64_t* rank_out, void* work,
                                                        size_t work_bytes, void* stream)
{
    if (int e = validate_factor(m, n, A, lda, k, b, p, jpvt, tau)) return e;
    return factor_impl<double>(m, n, A, lda, k, b, p, seed, nullptr, 0, jpvt, tau, rank_out, work, work_bytes,
                               (cudaStream_t)stream);
}

__attribute__((visibility("default"))) int rqrcp_factor_with_omega(int64_t m, int64_t n, double* A, int64_t lda,
                                                                   int64_t k, int64_t b, int64_t p,
                                                                   const double* Omega, int64_t ldo, int32_t* jpvt,
                                                                   double* tau, int64_t* rank_out, void* work,
                                                                   size_t work_bytes, void* stream)
{
    if (int e = validate_factor(m, n, A, lda, k, b, p, jpvt, tau)) return e <= -9 ? e - 1 : e;
    if (Omega == nullptr) return -8;
    if (ldo < m) return -9;
    return factor_impl<double>(m, n, A, lda, k, b, p, 0, Omega, ldo, jpvt, tau, rank_out, work, work_bytes,
                               (cudaStream_t)stream);
}

__attribute__((visibility("default"))) int rqrcp_factor_ex(int64_t m, int64_t n, double* A, int64_t lda, int64_t k,
                                                           int64_t b, int64_t p, uint64_t seed, const double* Omega,
                                                           int64_t ldo, int formula, int32_t* jpvt, double* tau,
                                                           int64_t* rank_out, void* work, size_t work_bytes,
                                                           void* stream)
{
    if (int e = validate_factor(m, n, A, lda, k, b, p, jpvt, tau)) return e <= -9 ? e - 3 : e;
    if (Omega != nullptr && ldo < m) return -10;
    if (formula != RQRCP_UPDATE_EQ4 && formula != RQRCP_UPDATE_EQ5) return -11;
    return factor_impl<double>(m, n, A, lda, k, b, p, seed, Omega, Omega != nullptr ? ldo : 0, jpvt, tau, rank_out,
                               work, work_bytes, (cudaStream_t)stream, 0, formula);
}

__attribute__((visibility("default"))) size_t rqrcp_srqr_workspace_size(int64_t m, int64_t n, int64_t l, int64_t b,
                                                                        int64_t p, int64_t d)
{
    if (m < 2 || n < 2 || l < 1 || l >= (m < n ? m : n) || b < 1 || p < 0 || d < 1) return 0;
    return make_srqr_layout(m, n, l, b, p, d).total;
}

__attribute__((visibility("default"))) int rqrcp_srqr(int64_t m, int64_t n, double* A, int64_t lda, int64_t l,
                                                      int64_t b, int64_t p, uint64_t seed, const double* Omega,
                                                      int64_t ldo, double g, int64_t d, uint64_t seed_g,
                                                      int64_t max_swaps, int32_t* jpvt, double* info_out, void* work,
                                                      size_t work_bytes, void* stream)
{
    if (m < 2) return -1;
    if (n < 2) return -2;
    if (A == nullptr) return -3;
    if (lda < m) return -4;
    if (l < 1 || l >= (m < n ? m : n)) return -5;
    if (b < 1) return -6;
    if (p < 0) return -7;
    if (Omega != nullptr && ldo < m) return -10;
    if (!(g > 1.0)) return -11;
    if (d < 1 || d > 65535) return -12;
    if (max_swaps < 0) return -14;
    if (jpvt == nullptr) return -15;
    const SrqrLayout S = make_srqr_layout(m, n, l, b, p, d);
    if (int e = check_work(work, work_bytes, S.total)) return e;
    if (srqr_solve_smem(l) > (size_t)dev_info().max_smem_optin) return RQRCP_ERR_UNSUPPORTED;
    cudaStream_t s = (cudaStream_t)stream;
    char* w = static_cast<char*>(work);
    double* tau = reinterpret_cast<double*>(w + S.tau);
    // Alg. 3 "Compute Q, R, Pi with Algorithm 2" (to rank l; B updated after the last block too)
    if (int e = factor_impl<double>(m, n, A, lda, l, b, p, seed, Omega, Omega != nullptr ? ldo : 0, jpvt, tau,
                                    nullptr, w, S.f.total, s, 0, RQRCP_UPDATE_EQ4, true))
        return e;
    Status* st = reinterpret_cast<Status*>(w + S.f.status);
    const double* B = reinterpret_cast<const double*>(w + S.f.B);
    double* r = reinterpret_cast<double*>(w + S.r);
    double* Og = reinterpret_cast<double*>(w + S.Og);
    double* X = reinterpret_cast<double*>(w + S.X);
    double* cs = reinterpret_cast<double*>(w + S.cs);
    double* info = reinterpret_cast<double*>(w + S.info);
    const int ls = (int)(b + p);
    RQ_CHECK(launch_srqr_prepare(A, lda, m, l, n, B, ls, r, st, s));
    RQ_CHECK(launch_srqr_extra_pivot(A, lda, m, l, n, r, jpvt, info, st, s));
    RQ_CHECK(launch_srqr_g2(A, lda, l, d, seed_g, Og, X, info, st, s));
    int64_t swaps = 0;
    double h[4];
    Status hs{};
    for (;;) {
        // the loop test needs g_2 on the host: one synchronisation per estimate (swaps are rare)
        RQ_CHECK(cudaMemcpyAsync(h, info, sizeof(h), cudaMemcpyDeviceToHost, s));
        RQ_CHECK(cudaMemcpyAsync(&hs, st, sizeof(Status), cudaMemcpyDeviceToHost, s));
        RQ_CHECK(cudaStreamSynchronize(s));
        if (hs.error != 0) return hs.error;
        // a rank guard that fired before l pivots leaves R_hat singular to working precision
        if (!(h[0] > g) || swaps >= max_swaps || hs.rank < l) break;
        const int64_t imax = (int64_t)h[1];
        if (imax < 0 || imax > l) return RQRCP_ERR_CUDA;
        RQ_CHECK(launch_srqr_swap(A, lda, l, n, imax, jpvt, cs, r, st, s));
        RQ_CHECK(launch_srqr_extra_pivot(A, lda, m, l, n, r, jpvt, info, st, s));
        ++swaps;
        RQ_CHECK(launch_srqr_g2(A, lda, l, d, seed_g + (uint64_t)swaps, Og, X, info, st, s));
    }
    if (info_out != nullptr) {
        info_out[0] = (double)swaps;
        info_out[1] = h[0];
        info_out[2] = h[2];
        info_out[3] = (double)hs.rank;
    }
    return RQRCP_OK;
}

__attribute__((visibility("default"))) int rqrcp_factor_mixed(int64_t m, int64_t n, float* A, int64_t lda, int64_t k,
                                                              int64_t b, int64_t p, uint64_t seed, int32_t* jpvt,
                                                              double* tau, int64_t* rank_out, void* work,
                                                              size_t work_bytes, void* stream)
{
    if (int e = validate_factor(m, n, A, lda, k, b, p, jpvt, tau)) return e;
    return factor_impl<float>(m, n, A, lda, k, b, p, seed, nullptr, 0, jpvt, tau, rank_out, work, work_bytes,
                              (cudaStream_t)stream, 1);
}

__attribute__((visibility("default"))) int rqrcp_factor_mixed_ex(int64_t m, int64_t n, float* A, int64_t lda,
                                                                 int64_t k, int64_t b, int64_t p, uint64_t seed,
                                                                 const float* Omega, int64_t ldo, int sketch,
                                                                 int32_t* jpvt, double* tau, int64_t* rank_out,
                                                                 void* work, size_t work_bytes, void* stream)
{
    if (int e = validate_factor(m, n, A, lda, k, b, p, jpvt, tau)) return e <= -9 ? e - 3 : e;
    if (Omega != nullptr && ldo < m) return -10;
    if (sketch != RQRCP_SKETCH_BF16 && sketch != RQRCP_SKETCH_FP32) return -11;
    return factor_impl<float>(m, n, A, lda, k, b, p, seed, Omega, Omega != nullptr ? ldo : 0, jpvt, tau, rank_out,
                              work, work_bytes, (cudaStream_t)stream, sketch == RQRCP_SKETCH_BF16 ? 1 : 0);
}

__attribute__((visibility("default"))) int rqrcp_tournament_config(int64_t ncols, int64_t bb, int64_t b, int64_t p,
                                                                   int elem_bytes, int64_t group_cols,
                                                                   int64_t* group_out, int64_t* fanin_out)
{
    if (ncols < 1) return -1;
    if (bb < 1 || bb > ncols) return -2;
    if (b < bb || b > 128) return -3;
    if (p < 0) return -4;
    if (elem_bytes != 4 && elem_bytes != 8) return -5;
    if (group_cols < 0) return -6;
    if (group_out == nullptr) return -7;
    if (fanin_out == nullptr) return -8;
    int64_t gs;
    int fan;
    if (!tournament_config(ncols, (int)bb, b, (int)(b + p), elem_bytes, group_cols, &gs, &fan))
        return RQRCP_ERR_UNSUPPORTED;
    *group_out = gs;
    *fanin_out = fan;
    return RQRCP_OK;
}

__attribute__((visibility("default"))) int rqrcp_factor_tournament(int64_t m, int64_t n, double* A, int64_t lda,
                                                                   int64_t k, int64_t b, int64_t p, uint64_t seed,
                                                                   const double* Omega, int64_t ldo,
                                                                   int64_t group_cols, int32_t* jpvt, double* tau,
                                                                   int64_t* rank_out, void* work, size_t work_bytes,
                                                                   void* stream)
{
    if (int e = validate_factor(m, n, A, lda, k, b, p, jpvt, tau)) return e <= -9 ? e - 3 : e;
    if (Omega != nullptr && ldo < m) return -10;
    if (group_cols < 0) return -11;
    return factor_impl<double>(m, n, A, lda, k, b, p, seed, Omega, Omega != nullptr ? ldo : 0, jpvt, tau, rank_out,
                               work, work_bytes, (cudaStream_t)stream, 0, RQRCP_UPDATE_EQ4, false, group_cols);
}

__attribute__((visibility("default"))) int rqrcp_factor_mixed_tournament(int64_t m, int64_t n, float* A, int64_t lda,
                                                                         int64_t k, int64_t b, int64_t p,
                                                                         uint64_t seed, const float* Omega,
                                                                         int64_t ldo, int sketch, int64_t group_cols,
                                                                         int32_t* jpvt, double* tau,
                                                                         int64_t* rank_out, void* work,
                                                                         size_t work_bytes, void* stream)
{
    if (int e = validate_factor(m, n, A, lda, k, b, p, jpvt, tau)) return e <= -9 ? e - 4 : e;
    if (Omega != nullptr && ldo < m) return -10;
    if (sketch != RQRCP_SKETCH_BF16 && sketch != RQRCP_SKETCH_FP32) return -11;
    if (group_cols < 0) return -12;
    return factor_impl<float>(m, n, A, lda, k, b, p, seed, Omega, Omega != nullptr ? ldo : 0, jpvt, tau, rank_out,
                              work, work_bytes, (cudaStream_t)stream, sketch == RQRCP_SKETCH_BF16 ? 1 : 0,
                              RQRCP_UPDATE_EQ4, false, group_cols);
}

__attribute__((visibility("default"))) int rqrcp_read_status(const void* work, int64_t* rank, void* stream)
{
    if (work == nullptr) return -1;
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) {
        cudaGetLastError();
        return RQRCP_ERR_CUDA;
    }
    Status h;
    if (cudaMemcpy(&h, work, sizeof(Status), cudaMemcpyDeviceToHost) != cudaSuccess) {
        cudaGetLastError();
        return RQRCP_ERR_CUDA;
    }
    if (rank) *rank = h.rank;
    return h.error;
}

__attribute__((visibility("default"))) size_t rqrcp_lowrank_workspace_size(int64_t m, int64_t n, int64_t k)
{
    if (m < 1 || n < 1 || k < 1) return 0;
    const int64_t bb = 64;
    size_t off = 0;
    off = align_up(off + sizeof(Status));
    off = align_up(off + (size_t)kMaxSplit * (size_t)(k > bb ? k : bb) * bb * sizeof(double));  // P
    off = align_up(off + (size_t)bb * bb * sizeof(double));                                        // Tm
    off = align_up(off + (size_t)k * (size_t)(n > bb ? n : bb) * sizeof(double));                 // Y / Rk
    const size_t tc = lowrank_f32_tc_bytes(m, n, k);  // the FP32 tensor-core form
    return off > tc ? off : tc;
}

__attribute__((visibility("default"))) int rqrcp_lowrank(int64_t m, int64_t n, int64_t k, const double* Afact,
                                                         int64_t ldaf, const double* tau, const int32_t* jpvt,
                                                         double* L, int64_t ldl, double* Q1, int64_t ldq,
                                                         void* work, size_t work_bytes, void* stream)
{
    return lowrank_impl<double>(m, n, k, Afact, ldaf, tau, jpvt, L, ldl, Q1, ldq, work, work_bytes, stream);
}

__attribute__((visibility("default"))) int rqrcp_lowrank_f32(int64_t m, int64_t n, int64_t k, const float* Afact,
                                                             int64_t ldaf, const double* tau, const int32_t* jpvt,
                                                             float* L, int64_t ldl, float* Q1, int64_t ldq,
                                                             void* work, size_t work_bytes, void* stream)
{
    return lowrank_impl<float>(m, n, k, Afact, ldaf, tau, jpvt, L, ldl, Q1, ldq, work, work_bytes, stream);
}

}  // extern "C"
