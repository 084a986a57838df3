// cholqr.cu -- the unpivoted panel QR of Alg. 2 ("Do unpivoted QR on A(i:m, i:i+b-1)") for the FP32
// form by CholeskyQR2 with Householder reconstruction, instead of one grid-wide step per column.
//
// For the (m1 x bb) FP32 panel P (bb <= 64):
//   pass 1  G1 = P^T P (FP32 sums folded into float pairs every 32 rows, FP64 across blocks in a
//           fixed order), G1 = R1^T R1 (Cholesky in float-pair arithmetic, about 44 significant bits,
//           on G1 scaled by a power of two);
//   pass 2  Q1 = P R1^{-1} row by row (forward substitution in FP32 with R1 rounded to FP32: the
//           substitution is backward stable), G2 = Q1^T Q1, G2 = R2^T R2; R = R2 R1 and
//           P = (Q1 R2^{-1}) R;
//   rebuild with Q2 = Q1 R2^{-1} (orthonormal to FP32 level), the LU factorization without pivoting
//           Q2 - S = [L1; L2] U, S = diag(s_j) with s_j = -sign of the j-th pivot, gives the
//           Householder vectors V = [L1; L2] (unit lower), tau_j = -s_j U(j,j) and R_house = S R:
//           the representation xGEQRF computes (xLARFG sign convention), up to rounding (Ballard
//           et al., "Reconstructing Householder vectors from tall-skinny QR", 2014).  The top bb rows
//           of Q2 are formed and factored in one block; the rows below are V2 = Q1 (U R2)^{-1}, one
//           row per thread.
// The two Cholesky factorizations run in float pairs (Dekker products by FMA, Knuth sums) because
// one SM issues FP64 at a small fraction of its FP32 rate, the LU in FP32 (its factors become the
// FP32 reflectors); their steps deal the trailing entries out evenly over the block's threads from
// a table and take one barrier each.  CholeskyQR2 needs kappa(P) well
// below the inverse square root of the Gram's precision: a pivot of G1 below 2^-20 of its diagonal
// entry (kappa(P) beyond about 1e3; G1 is summed in FP32), or a pivot of G2 below 1/2, sets a flag;
// the panel is then left untouched and the cooperative Householder panel kernel launched after this
// one factors it instead (it reads the flag and returns at once when the CholeskyQR2 result was
// written).  No host synchronisation.
#include "df.cuh"
#include "internal.cuh"

namespace rq {
namespace {

constexpr int kCqrMaxB = 64;
constexpr int kLd = kCqrMaxB + 1;                      // odd stride: a column of a row-major tile hits distinct banks
constexpr int kLx = kCqrMaxB + 4;                      // Gram tiles: 16-byte aligned rows for 128-bit loads
constexpr int kCqrNE = kCqrMaxB * (kCqrMaxB + 1) / 2;  // packed upper-triangle entries
constexpr int kCqrRows = 128;                          // panel rows per Gram block
constexpr int kGramTiles = 16 * 17 / 2;                // 4 x 4 micro-tiles on and above the diagonal
constexpr int kGramThreads = 160;
constexpr int kSolveThreads = 128;                     // one panel row per thread
constexpr int kSmallThreads = 512;
constexpr int kRedWarps = 8;
// pass-1 pivot test: the Gram G1 is summed in FP32 (folded into pairs), so CholeskyQR2 is kept only
// while kappa(P) stays below about 2^10
constexpr float kCqrPass1Thr = 9.5367431640625e-07f;  // 2^-20

// --------------------------------------------------------------------------- index tables
// packed upper-triangle index of (i, j), i <= j, row-major
__device__ __forceinline__ int tri_index(int i, int j, int bb) { return i * bb - i * (i - 1) / 2 + (j - i); }
// first entry of shell m = min(r, c) when a bb x bb square is listed shell by shell
__device__ __forceinline__ int sq_start(int m, int bb) { return 2 * bb * m - m * m; }
__device__ __forceinline__ int tab_r(uint16_t t) { return t & 0xff; }
__device__ __forceinline__ int tab_c(uint16_t t) { return t >> 8; }

// tab[tri_index(i, j, bb)] = (i, j): the entries of rows > j form the suffix from tri_index(j+1, j+1).
__device__ void build_tri_table(uint16_t* tab, int bb)
{
    const int i = threadIdx.x;
    if (i < bb) {
        const int base = tri_index(i, i, bb);
        for (int j = i; j < bb; ++j) tab[base + j - i] = (uint16_t)(i | (j << 8));
    }
}
// The bb x bb square shell by shell: shell m lists (m, m), (m, m+1 .. bb-1), (m+1 .. bb-1, m); the
// entries with min(r, c) > j form the suffix from sq_start(j + 1).
__device__ void build_sq_table(uint16_t* tab, int bb)
{
    const int m = threadIdx.x;
    if (m < bb) {
        int e = sq_start(m, bb);
        tab[e++] = (uint16_t)(m | (m << 8));
        for (int c = m + 1; c < bb; ++c) tab[e++] = (uint16_t)(m | (c << 8));
        for (int r = m + 1; r < bb; ++r) tab[e++] = (uint16_t)(r | (m << 8));
    }
}

// ------------------------------------------------------------------------------- row solves
// x := x R^{-1} for one row held in registers (x(c) = 0 for c >= bb): R upper triangular in FP32,
// row-major with ld kCqrMaxB, 16-byte aligned, zero outside its bb x bb upper triangle; (rh, rl) the
// float pairs of 1 / R(c, c), (1, 0) for c >= bb.  Column-oriented substitution: q(c) = x(c) / R(c, c),
// then x(j) -= q(c) R(c, j) for j > c, in FP32 with FMA.  Every thread of a warp reads the same R
// entries (broadcast loads).
__device__ __forceinline__ void row_solve_regs(float (&x)[kCqrMaxB], const float* __restrict__ R, const float* rh,
                                               const float* rl)
{
#pragma unroll
    for (int c = 0; c < kCqrMaxB; ++c) {
        const float q = fmaf(x[c], rl[c], x[c] * rh[c]);
        x[c] = q;
        const float4* Rc = reinterpret_cast<const float4*>(R + c * kCqrMaxB);
#pragma unroll
        for (int t = (c + 1) >> 2; t < kCqrMaxB / 4; ++t) {
            const float4 v = Rc[t];
            if (4 * t + 0 > c) x[4 * t + 0] = fmaf(-q, v.x, x[4 * t + 0]);
            if (4 * t + 1 > c) x[4 * t + 1] = fmaf(-q, v.y, x[4 * t + 1]);
            if (4 * t + 2 > c) x[4 * t + 2] = fmaf(-q, v.z, x[4 * t + 2]);
            if (4 * t + 3 > c) x[4 * t + 3] = fmaf(-q, v.w, x[4 * t + 3]);
        }
    }
}

// Y(r, 0:bb) = X(r, 0:bb) R^{-1} for the rows r = row0 .. row0 + nrows - 1 of the column-major X (ld ldx)
// and Y (ld ldy), one row per thread (coalesced column loads and stores): R is the bb x bb upper
// triangle of Rg (FP32, row-major, ld kCqrMaxB) and (rhg, rlg) the pairs of its diagonal's
// reciprocals.  Returns at once when the flag is set.
__global__ void __launch_bounds__(kSolveThreads) cqr_solve_kernel(const float* __restrict__ X, int64_t ldx,
                                                                  float* __restrict__ Y, int64_t ldy, int64_t row0,
                                                                  int64_t nrows, int bb, const float* __restrict__ Rg,
                                                                  const float* __restrict__ rhg,
                                                                  const float* __restrict__ rlg, const int* flag,
                                                                  const Status* st)
{
    if (status_error(st)) return;
    if (*(volatile const int*)flag) return;
    __shared__ __align__(16) float sR[kCqrMaxB * kCqrMaxB];
    __shared__ float srh[kCqrMaxB], srl[kCqrMaxB];
    const int tid = threadIdx.x;
    for (int e = tid; e < kCqrMaxB * kCqrMaxB; e += kSolveThreads) {
        const int i = e >> 6, j = e & (kCqrMaxB - 1);
        sR[e] = (i <= j && j < bb) ? Rg[e] : 0.f;
    }
    if (tid < kCqrMaxB) {
        srh[tid] = tid < bb ? rhg[tid] : 1.f;
        srl[tid] = tid < bb ? rlg[tid] : 0.f;
    }
    __syncthreads();
    const int64_t r = (int64_t)blockIdx.x * kSolveThreads + tid;
    if (r >= nrows) return;
    const float* xr = X + row0 + r;
    float x[kCqrMaxB];
#pragma unroll
    for (int c = 0; c < kCqrMaxB; ++c) x[c] = c < bb ? xr[(int64_t)c * ldx] : 0.f;
    row_solve_regs(x, sR, srh, srl);
    float* yr = Y + row0 + r;
#pragma unroll
    for (int c = 0; c < kCqrMaxB; ++c)
        if (c < bb) yr[(int64_t)c * ldy] = x[c];
}

// ------------------------------------------------------------------------------------ Gram
// Gram partials of the kCqrRows-row block g of X (m1 x bb, column-major, ld ldx): part[g * NE + e]
// (FP64) for the packed upper triangle.  Thread t < 136 owns the 4 x 4 micro-tile (I, J), I <= J, of
// the 64 x 64 Gram (two 128-bit shared loads and 16 FMA per row), FP32 sums folded into float pairs
// every 32 rows.  In pass 2 the kernel returns at once when the flag is set.
__global__ void __launch_bounds__(kGramThreads) cqr_gram_kernel(const float* __restrict__ X, int64_t ldx, int64_t m1,
                                                                int bb, double* __restrict__ part, const int* flag,
                                                                int pass, const Status* st)
{
    if (status_error(st)) return;
    if (pass == 2 && *(volatile const int*)flag) return;
    __shared__ __align__(16) float T[kCqrRows][kLx];
    const int tid = threadIdx.x;
    const int64_t r0 = (int64_t)blockIdx.x * kCqrRows;
    const int nr = (int)min((int64_t)kCqrRows, m1 - r0);
    for (int e = tid; e < kCqrRows * kCqrMaxB; e += kGramThreads) {
        const int r = e & (kCqrRows - 1), c = e >> 7;
        T[r][c] = (r < nr && c < bb) ? X[(int64_t)c * ldx + r0 + r] : 0.f;
    }
    __syncthreads();
    if (tid >= kGramTiles) return;
    int I = 0, rem = tid;
    while (rem >= 16 - I) {
        rem -= 16 - I;
        ++I;
    }
    const int J = I + rem;
    if (4 * J >= bb) return;  // the tile holds no entry (i, j), i <= j < bb
    float a[16], sh[16], sl[16];
#pragma unroll
    for (int t = 0; t < 16; ++t) a[t] = sh[t] = sl[t] = 0.f;
    for (int rb = 0; rb < nr; rb += 32) {
        const int re = min(nr, rb + 32);
#pragma unroll 4
        for (int r = rb; r < re; ++r) {
            const float4 x = *reinterpret_cast<const float4*>(&T[r][4 * I]);
            const float4 y = *reinterpret_cast<const float4*>(&T[r][4 * J]);
            const float xv[4] = {x.x, x.y, x.z, x.w}, yv[4] = {y.x, y.y, y.z, y.w};
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) a[4 * u + v] = fmaf(xv[u], yv[v], a[4 * u + v]);
        }
#pragma unroll
        for (int t = 0; t < 16; ++t) {
            const df s = df_two_sum(sh[t], a[t]);
            sh[t] = s.h;
            sl[t] += s.l;
            a[t] = 0.f;
        }
    }
    double* out = part + (size_t)blockIdx.x * kCqrNE;
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int i = 4 * I + u, j = 4 * J + v;
            if (i <= j && j < bb) out[tri_index(i, j, bb)] = (double)sh[4 * u + v] + (double)sl[4 * u + v];
        }
}

// G[e] = sum over blocks g of part[g * NE + e]: 32 entries per block (coalesced rows of part), warp w
// sums the blocks g = w (mod 8) in order, then the eight sums are added in warp order.
__global__ void __launch_bounds__(32 * kRedWarps) cqr_reduce_kernel(const double* __restrict__ part, int nblk,
                                                                    int ne, double* __restrict__ G, const int* flag,
                                                                    int pass, const Status* st)
{
    if (status_error(st)) return;
    if (pass == 2 && *(volatile const int*)flag) return;
    __shared__ double red[kRedWarps][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int e = blockIdx.x * 32 + lane;
    double s = 0.0;
    if (e < ne)
        for (int g = w; g < nblk; g += kRedWarps) s += part[(size_t)g * kCqrNE + e];
    red[w][lane] = s;
    __syncthreads();
    if (w == 0 && e < ne) {
        double t = red[0][lane];
        for (int k = 1; k < kRedWarps; ++k) t += red[k][lane];
        G[e] = t;
    }
}

// ------------------------------------------------------------------------- small factorizations
// Right-looking Cholesky G = R^T R of the bb x bb float-pair matrix (H, L) (upper triangle, stride
// kLd), in place, by all the block's threads.  Step j subtracts A(j, r) A(j, c) / A(j, j) from every
// (r, c) with j < r <= c, the entries dealt out evenly over the threads through the table tab
// (build_tri_table), and ends with one barrier; row j stays unscaled until the end, when
// R(j, c) = A(j, c) / sqrt(A(j, j)).  Returns false (uniformly in the block) if a pivot is not above
// thr times its original diagonal entry d0.  The caller has synchronised the block after filling
// (H, L), tab and d0; rs: 2 kCqrMaxB floats of scratch.
__device__ bool df_cholesky(float (*H)[kLd], float (*L)[kLd], int bb, const uint16_t* tab, const float* d0, float thr,
                            float* rs)
{
    const int tid = threadIdx.x, nt = blockDim.x;
    const int ne = bb * (bb + 1) / 2;
    for (int j = 0; j < bb; ++j) {
        const df d = {H[j][j], L[j][j]};
        // the pivot test in FP32 (every thread reads the same values: uniform)
        if (!(d.h > thr * d0[j])) return false;
        const df rd = df_rcp(d);
        for (int e = tri_index(j + 1, j + 1, bb) + tid; e < ne; e += nt) {
            const uint16_t t = tab[e];
            const int r = tab_r(t), c = tab_c(t);
            const df a = df_mul({H[j][r], L[j][r]}, rd);
            const df v = df_fms({H[r][c], L[r][c]}, a, {H[j][c], L[j][c]});
            H[r][c] = v.h;
            L[r][c] = v.l;
        }
        __syncthreads();
    }
    if (tid < bb) {
        const df y = df_rsqrt({H[tid][tid], L[tid][tid]});
        rs[tid] = y.h;
        rs[kCqrMaxB + tid] = y.l;
    }
    __syncthreads();
    for (int e = tid; e < ne; e += nt) {
        const uint16_t t = tab[e];
        const int i = tab_r(t), c = tab_c(t);
        const df v = df_mul({H[i][c], L[i][c]}, {rs[i], rs[kCqrMaxB + i]});
        H[i][c] = v.h;
        L[i][c] = v.l;
    }
    __syncthreads();
    return true;
}

// Pass-1 factor: the Cholesky factor R1 of G1 (scaled by a power of two for the pair arithmetic and
// scaled back), as float pairs Rh/Rl (row-major, ld kCqrMaxB, the bb x bb upper triangle) with the
// pairs of 1 / R1(j, j).  flag = 0 on success, 1 when the panel goes to the Householder fallback.
__global__ void __launch_bounds__(kSmallThreads) cqr_small1_kernel(const double* __restrict__ Gpk, int bb,
                                                                   float* __restrict__ Rh, float* __restrict__ Rl,
                                                                   float* __restrict__ rh, float* __restrict__ rl,
                                                                   int* flag, const Status* st)
{
    if (status_error(st)) return;
    __shared__ float H[kCqrMaxB][kLd], L[kCqrMaxB][kLd];
    __shared__ float d0[kCqrMaxB], rs[2 * kCqrMaxB];
    __shared__ uint16_t tab[kCqrNE];
    __shared__ double wmax[2];
    const int tid = threadIdx.x, ne = bb * (bb + 1) / 2;
    build_tri_table(tab, bb);
    if (tid < 64) {
        double m = tid < bb ? Gpk[tri_index(tid, tid, bb)] : 0.0;
        if (!(m <= 1.7976931348623157e308)) m = 0.0;  // a non-finite Gram: its pivots fail below
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
        if ((tid & 31) == 0) wmax[tid >> 5] = m;
    }
    __syncthreads();
    const double mx = fmax(wmax[0], wmax[1]);
    // 2^-2e with 2^e near sqrt(mx): the scaled diagonal is within [1/4, 4]
    const int ex = mx > 0.0 ? ilogb(mx) / 2 : 0;
    const double sc = ldexp(1.0, -2 * ex);
    for (int e = tid; e < ne; e += kSmallThreads) {
        const uint16_t t = tab[e];
        const int i = tab_r(t), c = tab_c(t);
        const df v = df_of(Gpk[e] * sc);
        H[i][c] = v.h;
        L[i][c] = v.l;
        if (i == c) d0[i] = v.h;
    }
    __syncthreads();
    if (!df_cholesky(H, L, bb, tab, d0, kCqrPass1Thr, rs)) {
        if (tid == 0) *flag = 1;
        return;
    }
    // R1 = R1_scaled 2^ex
    const float un = ldexpf(1.0f, ex);
    for (int e = tid; e < ne; e += kSmallThreads) {
        const uint16_t t = tab[e];
        const int i = tab_r(t), c = tab_c(t);
        Rh[i * kCqrMaxB + c] = H[i][c] * un;
        Rl[i * kCqrMaxB + c] = L[i][c] * un;
    }
    if (tid < bb) {
        const df r = df_rcp({H[tid][tid] * un, L[tid][tid] * un});
        rh[tid] = r.h;
        rl[tid] = r.l;
    }
    if (tid == 0) *flag = 0;
}

// Pass-2 factor and the reconstruction, in one block: R2 from G2 (fallback if a pivot is below 1/2),
// R = R2 R1, Q2top = Q1(0:bb, :) R2^{-1}, its LU without pivoting with s_j = -sign(pivot),
// tau_j = -s_j U(j, j), W = U R2 in FP32 (with the pairs of 1 / W(j, j)) for the rows below, and the
// panel's top bb rows: R_house = S R on and above the diagonal, L1 below it.
struct Small2Smem {
    float H[kCqrMaxB][kLd], L[kCqrMaxB][kLd];    // G2, then R2 (upper triangle)
    float UH[kCqrMaxB][kLd], UL[kCqrMaxB][kLd];  // Q2top, then its LU
    float E[kCqrMaxB][kLd];                      // R2 - I in FP32
    float R1[kCqrMaxB][kLd];                     // R1 in FP32
    __align__(16) float R2f[kCqrMaxB * kCqrMaxB];  // R2 in FP32 for the row solve (ld kCqrMaxB)
    float r2h[kCqrMaxB], r2l[kCqrMaxB];
    float pvh[kCqrMaxB], pvl[kCqrMaxB], rph[kCqrMaxB], rpl[kCqrMaxB], sgn[kCqrMaxB];
    float d0[kCqrMaxB], rs[2 * kCqrMaxB];
    uint16_t tri[kCqrNE];
    uint16_t sq[kCqrMaxB * kCqrMaxB];
};

__global__ void __launch_bounds__(kSmallThreads) cqr_small2_kernel(
    const double* __restrict__ Gpk, int bb, const float* __restrict__ R1h, const float* __restrict__ R1l,
    const float* __restrict__ Q1, int64_t m1, float* __restrict__ A, int64_t lda, double* __restrict__ tau,
    float* __restrict__ Wg, float* __restrict__ wh, float* __restrict__ wl, int* flag, const Status* st)
{
    if (status_error(st)) return;
    if (*(volatile const int*)flag) return;
    extern __shared__ __align__(16) unsigned char cqr_s2_raw[];
    Small2Smem& S = *reinterpret_cast<Small2Smem*>(cqr_s2_raw);
    const int tid = threadIdx.x, tx = tid & 63, ty = tid >> 6;
    const int ne = bb * (bb + 1) / 2, nsq = bb * bb;
    build_tri_table(S.tri, bb);
    build_sq_table(S.sq, bb);
    __syncthreads();
    for (int e = tid; e < ne; e += kSmallThreads) {
        const uint16_t t = S.tri[e];
        const int i = tab_r(t), c = tab_c(t);
        const df v = df_of(Gpk[e]);
        S.H[i][c] = v.h;
        S.L[i][c] = v.l;
        if (i == c) S.d0[i] = v.h;
    }
    __syncthreads();
    if (!df_cholesky(S.H, S.L, bb, S.tri, S.d0, 0.5f, S.rs)) {
        if (tid == 0) *flag = 1;
        return;
    }
    // R2 in FP32 (padded) for the row solve, E = R2 - I, R1 in FP32; the reciprocal pairs of R2's diagonal
    for (int e = tid; e < kCqrMaxB * kCqrMaxB; e += kSmallThreads) {
        const int i = e >> 6, j = e & (kCqrMaxB - 1);
        const bool in = i <= j && j < bb;
        S.R2f[e] = in ? S.H[i][j] : 0.f;
        S.E[i][j] = in ? (S.H[i][j] - (i == j ? 1.f : 0.f)) + S.L[i][j] : 0.f;
        S.R1[i][j] = in ? R1h[i * kCqrMaxB + j] : 0.f;
    }
    if (tid < kCqrMaxB) {
        const df r = tid < bb ? df_rcp({S.H[tid][tid], S.L[tid][tid]}) : df{1.f, 0.f};
        S.r2h[tid] = r.h;
        S.r2l[tid] = r.l;
    }
    __syncthreads();
    // Q2top rows = Q1top rows R2^{-1}, one row per thread
    if (tid < bb) {
        float x[kCqrMaxB];
#pragma unroll
        for (int c = 0; c < kCqrMaxB; ++c) x[c] = c < bb ? Q1[(int64_t)c * m1 + tid] : 0.f;
        row_solve_regs(x, S.R2f, S.r2h, S.r2l);
#pragma unroll
        for (int c = 0; c < kCqrMaxB; ++c) {
            S.UH[tid][c] = x[c];
            S.UL[tid][c] = 0.f;
        }
    }
    __syncthreads();
    // LU of Q2top - S in FP32, right-looking: step j subtracts U(r, j) U(j, c) / piv_j from every
    // (r, c) with r, c > j (dealt out evenly through the shell table), one barrier per step; the
    // pivots and the scaling of column j into L(:, j) are applied after the last step.  Working
    // precision suffices here (the reconstruction is stable with the LU in working precision,
    // Ballard et al. 2014): L and U become the FP32 reflectors, tau and W, and R does not depend on
    // them.  Every pivot has |piv| = |a| + 1 >= 1 (s_j = -sign(a)), so the LU needs no pivoting.
    for (int j = 0; j < bb; ++j) {
        const float a = S.UH[j][j];
        const float s = a >= 0.f ? -1.f : 1.f;
        const float piv = a - s;
        const float rp = 1.f / piv;
        if (tid == 0) {
            S.pvh[j] = piv;
            S.pvl[j] = 0.f;
            S.rph[j] = rp;
            S.rpl[j] = 0.f;
            S.sgn[j] = s;
        }
        for (int e = sq_start(j + 1, bb) + tid; e < nsq; e += kSmallThreads) {
            const uint16_t t = S.sq[e];
            const int r = tab_r(t), c = tab_c(t);
            S.UH[r][c] = fmaf(-(S.UH[r][j] * rp), S.UH[j][c], S.UH[r][c]);
        }
        __syncthreads();
    }
    if (tx < bb)
        for (int r = ty; r < bb; r += kSmallThreads / 64) {
            if (r == tx)
                S.UH[r][tx] = S.pvh[tx];
            else if (r > tx)
                S.UH[r][tx] *= S.rph[tx];
        }
    __syncthreads();
    // tau, the panel's top rows (R_house = S R2 R1 above, L1 below the diagonal) and W = U R2.
    // R2 = I + E with E at the level of Q1's departure from orthogonality (FP32 rounding), so
    // R2 R1 = R1 + E R1 and U R2 = U + U E: the leading terms stay float pairs and the small
    // corrections are plain FP32 sums.
    if (tid < bb) tau[tid] = -(double)S.sgn[tid] * df_dbl({S.pvh[tid], S.pvl[tid]});
    if (tx < bb)
        for (int i = ty; i < bb; i += kSmallThreads / 64) {
            const int j = tx;
            float out;
            if (i <= j) {
                float cr = 0.f, cw = 0.f;
                for (int q = i; q <= j; ++q) {
                    cr = fmaf(S.E[i][q], S.R1[q][j], cr);
                    cw = fmaf(S.UH[i][q], S.E[q][j], cw);
                }
                const df r = df_add({R1h[i * kCqrMaxB + j], R1l[i * kCqrMaxB + j]}, {cr, 0.f});
                const df w = df_add({S.UH[i][j], S.UL[i][j]}, {cw, 0.f});
                out = S.sgn[i] * (r.h + r.l);
                Wg[i * kCqrMaxB + j] = w.h + w.l;
                if (i == j) {
                    const df wr = df_rcp(w);
                    wh[i] = wr.h;
                    wl[i] = wr.l;
                }
            } else {
                out = S.UH[i][j] + S.UL[i][j];
            }
            A[(int64_t)j * lda + i] = out;
        }
}

constexpr size_t kSmall2Smem = sizeof(Small2Smem);

// Regions of the CholeskyQR2 workspace for an m1-row panel, each 256-byte aligned, in this order:
// partial Grams, reduced Gram, R1 as float pairs, W = U R2 in FP32, the reciprocal pairs of their
// diagonals, Q1 (m1 x 64 FP32), the fallback flag.
constexpr int kCqrRegions = 9;
size_t cholqr_region_bytes(int i, int64_t m1)
{
    const int64_t nblk = (m1 + kCqrRows - 1) / kCqrRows;
    switch (i) {
    case 0: return sizeof(double) * (size_t)nblk * kCqrNE;
    case 1: return sizeof(double) * kCqrNE;
    case 2: case 3: case 4: return sizeof(float) * kCqrMaxB * kCqrMaxB;
    case 5: case 6: return 2 * sizeof(float) * kCqrMaxB;
    case 7: return sizeof(float) * (size_t)m1 * kCqrMaxB;
    default: return 256;
    }
}

}  // namespace

size_t cholqr_ws_bytes(int64_t m_max)
{
    size_t b = 0;
    for (int i = 0; i < kCqrRegions; ++i) b += (cholqr_region_bytes(i, m_max) + 255) & ~(size_t)255;
    return b;
}

bool cholqr_supported(int bb) { return bb >= 1 && bb <= kCqrMaxB; }

cudaError_t launch_cholqr_panel(float* A, int64_t lda, int64_t m1, int bb, double* tau, void* ws, int** flag_out,
                                const Status* st, cudaStream_t s)
{
    char* w = static_cast<char*>(ws);
    const int nblk = (int)((m1 + kCqrRows - 1) / kCqrRows);
    char* reg[kCqrRegions];
    for (int i = 0; i < kCqrRegions; ++i) {
        reg[i] = w;
        w += (cholqr_region_bytes(i, m1) + 255) & ~(size_t)255;
    }
    double* part = reinterpret_cast<double*>(reg[0]);
    double* G = reinterpret_cast<double*>(reg[1]);
    float* R1h = reinterpret_cast<float*>(reg[2]);
    float* R1l = reinterpret_cast<float*>(reg[3]);
    float* W = reinterpret_cast<float*>(reg[4]);
    float* r1h = reinterpret_cast<float*>(reg[5]);
    float* r1l = r1h + kCqrMaxB;
    float* wrh = reinterpret_cast<float*>(reg[6]);
    float* wrl = wrh + kCqrMaxB;
    float* Q1 = reinterpret_cast<float*>(reg[7]);
    int* flag = reinterpret_cast<int*>(reg[8]);
    *flag_out = flag;
    const int ne = bb * (bb + 1) / 2;
    const unsigned rb = (unsigned)((ne + 31) / 32);
    const unsigned sb = (unsigned)((m1 + kSolveThreads - 1) / kSolveThreads);
    static DevFlag attr_set;
    if (!attr_set.done()) {
        const cudaError_t e = cudaFuncSetAttribute((const void*)cqr_small2_kernel,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmall2Smem);
        if (e != cudaSuccess) return e;
        attr_set.set();
    }
    // pass 1
    cqr_gram_kernel<<<nblk, kGramThreads, 0, s>>>(A, lda, m1, bb, part, flag, 1, st);
    cqr_reduce_kernel<<<rb, 32 * kRedWarps, 0, s>>>(part, nblk, ne, G, flag, 1, st);
    cqr_small1_kernel<<<1, kSmallThreads, 0, s>>>(G, bb, R1h, R1l, r1h, r1l, flag, st);
    // pass 2: Q1 = P R1^{-1}, its Gram
    cqr_solve_kernel<<<sb, kSolveThreads, 0, s>>>(A, lda, Q1, m1, 0, m1, bb, R1h, r1h, r1l, flag, st);
    cqr_gram_kernel<<<nblk, kGramThreads, 0, s>>>(Q1, m1, m1, bb, part, flag, 2, st);
    cqr_reduce_kernel<<<rb, 32 * kRedWarps, 0, s>>>(part, nblk, ne, G, flag, 2, st);
    // R2, R = R2 R1, the reconstruction and the panel's top rows
    cqr_small2_kernel<<<1, kSmallThreads, kSmall2Smem, s>>>(G, bb, R1h, R1l, Q1, m1, A, lda, tau, W, wrh, wrl, flag,
                                                           st);
    // the rows below: V2 = Q1 W^{-1}
    if (m1 > bb)
        cqr_solve_kernel<<<(unsigned)((m1 - bb + kSolveThreads - 1) / kSolveThreads), kSolveThreads, 0, s>>>(
            Q1, m1, A, lda, bb, m1 - bb, bb, W, wrh, wrl, flag, st);
    return cudaGetLastError();
}

}  // namespace rq
