/*
 * rqrcp_oracle.c -- plain, slow, obviously-correct FP64 CPU oracle for randomized
 * QR with column pivoting (Xiao, Gu, Langou, "Fast parallel randomized QR with
 * column pivoting algorithms for reliable low-rank matrix approximations", HiPC 2017).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code, header
 * or constant table with the CUDA path of the package; it implements every step
 * again from the paper.
 *
 * Conventions: all matrices are column-major, element (i,j) of X with leading
 * dimension ldx lives at X[j*ldx + i].  Indices are 0-based; the paper is 1-based.
 * Omega is row-major l x m (element (r,q) at Omega[r*m + q]).
 * Arithmetic is IEEE double throughout; loops run in the order the paper states.
 * OpenMP (when compiled with -fopenmp) only splits independent columns between
 * threads; the arithmetic of each column is the same sequential loop either way.
 *
 * Readings where the paper is silent (each also listed in the design notes):
 *  - Householder reflectors follow the LAPACK xLARFG convention:
 *    beta = -sign(alpha)*||x||, tau = (beta-alpha)/beta, v = x(2:)/(alpha-beta), v(1)=1,
 *    tau = 0 when x(2:) = 0.  sign(alpha) is + for alpha >= 0 (also for -0.0).
 *    The norm is sqrt(alpha^2 + sum x(2:)^2) without scaling: entries must stay
 *    below ~1e150 in magnitude.
 *  - argmax ties go to the smallest current column position.
 *  - column norms on B are recomputed at every pivot step (Alg. 1 "Update r_s").
 *  - rank guard: a pivot step whose largest remaining sketch norm^2 is at most
 *    (10*max(m,n)*2^-53)^2 times the largest initial sketch column norm^2 stops
 *    pivoting for good; the remaining columns keep their order, blocks keep their
 *    static boundaries and B is no longer updated.
 *  - if a diagonal entry of R11 is exactly zero the matching column of
 *    Omega_hat_11 is set to zero instead of dividing.
 *  - BF16 sketch (the mixed form's sketch step, orc_rqrcp2 with sketch_bf16 = 1): every
 *    element of Omega and of A is first rounded to FP32, then to BF16 (8 significant bits,
 *    round to nearest, ties to even); the products and their sums are then formed exactly
 *    as in the FP64 sketch.  Only the initial sketch sees the rounding.
 *  - SRQR (Alg. 3, orc_srqr) works on an explicit R.  Its RQRCP stage is Alg. 2 with Eq. (4)
 *    to rank l; the sketch after the last block's update is the sketch of R22 whose column
 *    norms / (b+p) start the estimates r_i (Eq. (4) and Eq. (5) give the same norms).  The
 *    downdated estimates are used as they are, negative or not (only their argmax matters).
 *    Estimate t of g_2 draws a fresh d x (l+1) Gaussian from orc_omega(d, l+1, seed_g + t).
 *    A zero diagonal entry of R_hat gives g_2 = +inf with that column as the worst one.  The
 *    round-robin swap moves the worst column to position l and shifts the columns after it
 *    left by one; Givens rotations on rows (j, j+1), j = worst..l-1, across all n columns
 *    restore the upper-trapezoidal form.  "r_{l+1} = R_{l+1,l+1}^2" is the squared norm of
 *    the column now at position l, whose entries below row l are zero.  The swap loop is
 *    capped at max_swaps (the paper only states that it ends), and skipped when the RQRCP
 *    stage's rank guard fired before l pivots (R_hat is then singular to working precision).
 *  - QR with tournament pivoting on B (the paper's future work, Sec. VI; orc_tournament and
 *    orc_rqrcp3 with group sizes): the leaves are consecutive groups of gs columns of B(:, i:n)
 *    in their positions at the start of the block; a node concatenates the choices of fanin
 *    consecutive groups in group order, each group's choices in the order they were taken, and
 *    reads them from B as it was at the start of the block; every choice is Alg. 1 on rows
 *    0..l-1 of its candidates with ties to the smallest position.  The block's pivots are the
 *    root's choices in their order; the rank guard tests the norm^2 of the chosen column's
 *    trailing rows at its step (against the same bound as the greedy search).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_EXPORT __attribute__((visibility("default")))

#define AT(X, ld, i, j) (X)[(size_t)(j) * (size_t)(ld) + (size_t)(i)]

/* ------------------------------------------------------------------------- */
/* BF16 rounding from the format's definition: BF16 keeps the sign, the 8-bit  */
/* exponent and the top 7 fraction bits of an IEEE single.  x is rounded to     */
/* single first; the 16 dropped bits are rounded to nearest, ties to the even   */
/* kept pattern.  Finite inputs below the BF16 overflow threshold only.         */
/* ------------------------------------------------------------------------- */
static double round_bf16(double x)
{
    float f = (float)x;
    uint32_t u;
    memcpy(&u, &f, sizeof u);
    const uint32_t dropped = u & 0xFFFFu;
    uint32_t kept = u & 0xFFFF0000u;
    if (dropped > 0x8000u || (dropped == 0x8000u && (kept & 0x10000u))) kept += 0x10000u;
    memcpy(&f, &kept, sizeof f);
    return (double)f;
}

ORC_EXPORT void orc_round_bf16(int64_t n, const double* x, double* y)
{
    for (int64_t i = 0; i < n; ++i) y[i] = round_bf16(x[i]);
}

/* ------------------------------------------------------------------------- */
/* Philox4x64-10 counter-based generator, from its published definition:      */
/* Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3",  */
/* SC'11.  Round: (x0,x1,x2,x3) -> (hi(M1*x2)^x1^k0, lo(M1*x2),                */
/*                                  hi(M0*x0)^x3^k1, lo(M0*x0)); key += Weyl.  */
/* ------------------------------------------------------------------------- */
ORC_EXPORT void orc_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4])
{
    const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
    uint64_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint64_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        unsigned __int128 p0 = (unsigned __int128)M0 * x0;
        unsigned __int128 p1 = (unsigned __int128)M1 * x2;
        uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
        uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
        uint64_t y0 = hi1 ^ x1 ^ k0, y1 = lo1, y2 = hi0 ^ x3 ^ k1, y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
        k0 += W0; k1 += W1;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/*
 * Omega in N(0,1)^{l x m} (Alg. 2, "Generate i.i.d Gaussian matrix").  Element with
 * row-major flat index q = r*m + c takes lane q%4 of the Philox block with counter
 * (q/4, 0, 0, 0) and key (seed, 0).  Lanes (0,1) and (2,3) form Box-Muller pairs
 * (Box & Muller 1958): u1 = (w0>>11 + 1)*2^-53 in (0,1], u2 = (w1>>11)*2^-53 in [0,1),
 * rho = sqrt(-2 ln u1), z_even = rho cos(2 pi u2), z_odd = rho sin(2 pi u2).
 */
ORC_EXPORT void orc_omega(int64_t l, int64_t m, uint64_t seed, double* Omega)
{
    const double two53 = 1.0 / 9007199254740992.0;
    int64_t total = l * m;
#pragma omp parallel for schedule(static)
    for (int64_t blk = 0; blk < (total + 3) / 4; ++blk) {
        uint64_t ctr[4] = {(uint64_t)blk, 0, 0, 0}, key[2] = {seed, 0}, w[4];
        orc_philox4x64_10(ctr, key, w);
        for (int pair = 0; pair < 2; ++pair) {
            double u1 = ((double)(w[2 * pair] >> 11) + 1.0) * two53;
            double u2 = (double)(w[2 * pair + 1] >> 11) * two53;
            double rho = sqrt(-2.0 * log(u1));
            double theta = 2.0 * M_PI * u2;
            int64_t q0 = blk * 4 + 2 * pair;
            if (q0 < total) Omega[q0] = rho * cos(theta);
            if (q0 + 1 < total) Omega[q0 + 1] = rho * sin(theta);
        }
    }
}

/* ------------------------------------------------------------------------- */
/* Householder reflector (Alg. 1, "Form Householder reflection H_i"), xLARFG    */
/* convention.  On entry x[0..len) is the column; on exit x[0] = beta and      */
/* x[1..len) holds the tail of v (v[0] = 1 implicit).  Returns tau.            */
/* ------------------------------------------------------------------------- */
static double house_gen(int64_t len, double* x)
{
    if (len <= 1) return 0.0;
    double ss = 0.0;
    for (int64_t r = 1; r < len; ++r) ss += x[r] * x[r];
    if (ss == 0.0) return 0.0;
    double alpha = x[0];
    double nrm = sqrt(alpha * alpha + ss);
    double beta = (alpha >= 0.0) ? -nrm : nrm;
    double tau = (beta - alpha) / beta;
    double scal = 1.0 / (alpha - beta);
    for (int64_t r = 1; r < len; ++r) x[r] *= scal;
    x[0] = beta;
    return tau;
}

/* y <- (I - tau v v^T) y for a column y of length len; v = [1; vt[1..len)]. */
static void house_apply(int64_t len, const double* v, double tau, double* y)
{
    if (tau == 0.0) return;
    double w = y[0];
    for (int64_t r = 1; r < len; ++r) w += v[r] * y[r];
    w *= tau;
    y[0] -= w;
    for (int64_t r = 1; r < len; ++r) y[r] -= w * v[r];
}

static void swap_cols(double* X, int64_t ldx, int64_t rows, int64_t a, int64_t b)
{
    if (a == b) return;
    for (int64_t r = 0; r < rows; ++r) {
        double t = AT(X, ldx, r, a);
        AT(X, ldx, r, a) = AT(X, ldx, r, b);
        AT(X, ldx, r, b) = t;
    }
}

/* ------------------------------------------------------------------------- */
/* Alg. 1: QR with column pivoting, k steps, column norms recomputed from the  */
/* trailing rows at every step (Alg. 1 "Update r_s = ||A(i+1:m,s)||").         */
/* ------------------------------------------------------------------------- */
ORC_EXPORT int orc_qrcp(int64_t m, int64_t n, double* A, int64_t lda, int64_t k,
                        int32_t* jpvt, double* tau)
{
    if (m < 0 || n < 0 || k < 1 || k > (m < n ? m : n) || lda < (m > 1 ? m : 1)) return -1;
    for (int64_t j = 0; j < n; ++j) jpvt[j] = (int32_t)j;
    for (int64_t i = 0; i < k; ++i) {
        int64_t best = i;
        double bestv = -1.0;
        for (int64_t s = i; s < n; ++s) {
            double nu = 0.0;
            for (int64_t r = i; r < m; ++r) nu += AT(A, lda, r, s) * AT(A, lda, r, s);
            if (nu > bestv) { bestv = nu; best = s; }
        }
        swap_cols(A, lda, m, i, best);
        int32_t tp = jpvt[i]; jpvt[i] = jpvt[best]; jpvt[best] = tp;
        double* x = &AT(A, lda, i, i);
        tau[i] = house_gen(m - i, x);
#pragma omp parallel for schedule(static)
        for (int64_t s = i + 1; s < n; ++s) house_apply(m - i, x, tau[i], &AT(A, lda, i, s));
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* One selection of QR with tournament pivoting (Demmel, Grigori, Gu, Xiang,    */
/* "Communication avoiding rank revealing QR factorization with column          */
/* pivoting", SIAM J. Matrix Anal. Appl. 36 (2015)): Alg. 1 for `steps` steps   */
/* on the nc candidate columns X(:, cand[s] - pos0) (l rows, ld l), copied to   */
/* W first; the squared norms of rows t..l-1 are recomputed at every step and   */
/* the largest wins, ties to the smallest position cand[s].  out[t] = the       */
/* position chosen at step t; *mingap is lowered to (nu_max - nu_second) /      */
/* nu_max of every step (1.0 with a single candidate, 0.0 if nu_max is 0).      */
/* ------------------------------------------------------------------------- */
static void tour_select(const double* X, int64_t l, int64_t pos0, const int64_t* cand, int64_t nc,
                        int64_t steps, int64_t* out, double* mingap, double* W, char* act)
{
    for (int64_t s = 0; s < nc; ++s) {
        memcpy(&AT(W, l, 0, s), &AT(X, l, 0, cand[s] - pos0), sizeof(double) * (size_t)l);
        act[s] = 1;
    }
    for (int64_t t = 0; t < steps; ++t) {
        int64_t best = -1;
        double v1 = -1.0, v2 = -1.0;
        for (int64_t s = 0; s < nc; ++s) {
            if (!act[s]) continue;
            double nu = 0.0;
            for (int64_t r = t; r < l; ++r) nu += AT(W, l, r, s) * AT(W, l, r, s);
            if (best < 0 || nu > v1 || (nu == v1 && cand[s] < cand[best])) {
                if (best >= 0) v2 = v1;
                v1 = nu;
                best = s;
            } else if (nu > v2) {
                v2 = nu;
            }
        }
        const double gap = v2 < 0.0 ? 1.0 : (v1 > 0.0 ? (v1 - v2) / v1 : 0.0);
        if (gap < *mingap) *mingap = gap;
        out[t] = cand[best];
        act[best] = 0;
        double* x = &AT(W, l, t, best);
        const double tb = house_gen(l - t, x);
        for (int64_t s = 0; s < nc; ++s)
            if (act[s]) house_apply(l - t, x, tb, &AT(W, l, t, s));
    }
}

/* ------------------------------------------------------------------------- */
/* QR with tournament pivoting, the choice of bb of the nc columns of X (l x nc, */
/* ld l; column s has position pos0 + s): leaves are the consecutive groups of   */
/* gs columns, each choosing min(bb, its size) columns by tour_select; while     */
/* more than one group is left, each run of fanin consecutive groups becomes one */
/* group that chooses min(bb, candidates) of its children's choices              */
/* (concatenated in child order), read from X.  sel[0..min(bb, nc)) receives     */
/* the last group's choices in their order; returns that count, or -1.          */
/* ------------------------------------------------------------------------- */
ORC_EXPORT int64_t orc_tournament(const double* X, int64_t l, int64_t nc, int64_t pos0, int64_t bb, int64_t gs,
                                  int64_t fanin, int64_t* sel, double* mingap)
{
    if (l < 1 || nc < 1 || bb < 1 || gs < 1 || fanin < 2) return -1;
    int64_t P = (nc + gs - 1) / gs;
    int64_t* ch = (int64_t*)malloc(sizeof(int64_t) * (size_t)(P * bb));   /* choices per group */
    int64_t* cnt = (int64_t*)malloc(sizeof(int64_t) * (size_t)P);
    int64_t* nch = (int64_t*)malloc(sizeof(int64_t) * (size_t)(P * bb));
    int64_t* ncnt = (int64_t*)malloc(sizeof(int64_t) * (size_t)P);
    int64_t* cand = (int64_t*)malloc(sizeof(int64_t) * (size_t)(fanin * bb > gs ? fanin * bb : gs));
    const int64_t wcols = fanin * bb > gs ? fanin * bb : gs;
    double* W = (double*)malloc(sizeof(double) * (size_t)(l * wcols));
    char* act = (char*)malloc((size_t)wcols);
    if (!ch || !cnt || !nch || !ncnt || !cand || !W || !act) {
        free(ch); free(cnt); free(nch); free(ncnt); free(cand); free(W); free(act);
        return -1;
    }
    double gap = 1.0;
    for (int64_t g = 0; g < P; ++g) {   /* leaves */
        const int64_t c0 = g * gs, c1 = (g + 1) * gs < nc ? (g + 1) * gs : nc;
        for (int64_t s = c0; s < c1; ++s) cand[s - c0] = pos0 + s;
        cnt[g] = bb < c1 - c0 ? bb : c1 - c0;
        tour_select(X, l, pos0, cand, c1 - c0, cnt[g], &ch[g * bb], &gap, W, act);
    }
    while (P > 1) {                     /* one level of the reduction tree */
        const int64_t P2 = (P + fanin - 1) / fanin;
        for (int64_t q = 0; q < P2; ++q) {
            int64_t nc2 = 0;
            for (int64_t g = q * fanin; g < (q + 1) * fanin && g < P; ++g)
                for (int64_t t = 0; t < cnt[g]; ++t) cand[nc2++] = ch[g * bb + t];
            ncnt[q] = bb < nc2 ? bb : nc2;
            tour_select(X, l, pos0, cand, nc2, ncnt[q], &nch[q * bb], &gap, W, act);
        }
        memcpy(ch, nch, sizeof(int64_t) * (size_t)(P2 * bb));
        memcpy(cnt, ncnt, sizeof(int64_t) * (size_t)P2);
        P = P2;
    }
    const int64_t ns = cnt[0];
    memcpy(sel, ch, sizeof(int64_t) * (size_t)ns);
    if (mingap) *mingap = gap;
    free(ch); free(cnt); free(nch); free(ncnt); free(cand); free(W); free(act);
    return ns;
}

/* ------------------------------------------------------------------------- */
/* Alg. 2: randomized QRCP.                                                    */
/*   formula == 4 : B updated by Eq. (4) (Duersch-Gu), in place, after the      */
/*                  partial QRCP on B has transformed it.                       */
/*   formula == 5 : B updated by Eq. (5) (Martinsson et al.): the partial QRCP  */
/*                  runs on a copy; B itself is only permuted, and               */
/*                  B_trail <- B2 - Omega_bar_1 R12 with Omega_bar = Omega Q.    */
/* Outputs: A overwritten with R (upper trapezoid, R22 = A(k:m,k:n)) and the    */
/* reflector tails below the diagonal of columns 0..k-1; tau[0..k); jpvt (0-    */
/* based, A_in(:,jpvt[c]) is column c of A*Pi); *rank_out = pivots taken before */
/* the rank guard fired (k if never).  gaps (k entries, optional) receives for  */
/* every pivot step (nu_max - nu_second)/nu_max over the candidate sketch norms */
/* (1.0 with a single candidate, -1.0 where no pivot was chosen).  Bout (l x n,  */
/* optional) receives B after the last block (formula 4: the transformed and    */
/* updated sketch; formula 5: the permuted sketch Omega_bar_2 R22).             */
/* ------------------------------------------------------------------------- */
ORC_EXPORT int orc_rqrcp2(int64_t m, int64_t n, double* A, int64_t lda, int64_t k, int64_t b,
                          int64_t p, const double* Omega, int formula, int sketch_bf16, int32_t* jpvt,
                          double* tau, int64_t* rank_out, double* gaps, double* Bout);
ORC_EXPORT int orc_rqrcp3(int64_t m, int64_t n, double* A, int64_t lda, int64_t k, int64_t b,
                          int64_t p, const double* Omega, int formula, int sketch_bf16, const int64_t* tgs,
                          int64_t fanin, int32_t* jpvt, double* tau, int64_t* rank_out, double* gaps,
                          double* Bout);

ORC_EXPORT int orc_rqrcp(int64_t m, int64_t n, double* A, int64_t lda, int64_t k, int64_t b,
                         int64_t p, const double* Omega, int formula, int32_t* jpvt, double* tau,
                         int64_t* rank_out, double* gaps, double* Bout)
{
    return orc_rqrcp2(m, n, A, lda, k, b, p, Omega, formula, 0, jpvt, tau, rank_out, gaps, Bout);
}

/* orc_rqrcp with the choice of sketch: sketch_bf16 = 0 the FP64 sketch, 1 the BF16 sketch.    */
ORC_EXPORT int orc_rqrcp2(int64_t m, int64_t n, double* A, int64_t lda, int64_t k, int64_t b,
                          int64_t p, const double* Omega, int formula, int sketch_bf16, int32_t* jpvt,
                          double* tau, int64_t* rank_out, double* gaps, double* Bout)
{
    return orc_rqrcp3(m, n, A, lda, k, b, p, Omega, formula, sketch_bf16, NULL, 0, jpvt, tau, rank_out, gaps,
                      Bout);
}

/* orc_rqrcp2 with the pivot rule: tgs == NULL the partial QRCP of Alg. 2 (Alg. 1 on B); else QR  */
/* with tournament pivoting on B (formula 4 only), tgs[q] the leaf group size of block q (the     */
/* block starting at column q*b) and fanin the tree's fan-in.  gaps[c] of a tournament block is   */
/* the smallest gap of all the choices the block's tournament made.                               */
ORC_EXPORT int orc_rqrcp3(int64_t m, int64_t n, double* A, int64_t lda, int64_t k, int64_t b,
                          int64_t p, const double* Omega, int formula, int sketch_bf16, const int64_t* tgs,
                          int64_t fanin, int32_t* jpvt, double* tau, int64_t* rank_out, double* gaps,
                          double* Bout)
{
    if (m < 1 || n < 1) return -1;
    if (lda < m) return -4;
    if (k < 1 || k > (m < n ? m : n)) return -5;
    if (b < 1) return -6;
    if (p < 0) return -7;
    if (formula != 4 && formula != 5) return -9;
    if (tgs && (formula != 4 || fanin < 2)) return -11;
    const int64_t l = b + p;
    double* B = (double*)malloc(sizeof(double) * (size_t)(l * n));
    double* Bq = (double*)malloc(sizeof(double) * (size_t)(l * n));   /* QRCP copy (formula 5) */
    double* Wh = (double*)malloc(sizeof(double) * (size_t)(b * b));   /* Omega_hat_11 */
    double* Ob = NULL;                                                /* Omega_bar, row-major l x m */
    if (!B || !Bq || !Wh) { free(B); free(Bq); free(Wh); return 1; }
    if (formula == 5) {
        Ob = (double*)malloc(sizeof(double) * (size_t)(l * m));
        if (!Ob) { free(B); free(Bq); free(Wh); return 1; }
        memcpy(Ob, Omega, sizeof(double) * (size_t)(l * m));
    }

    /* Alg. 2: B = Omega A, summed over q in increasing order (BF16 sketch: on the rounded
       operands). */
    if (sketch_bf16) {
        double* Or = (double*)malloc(sizeof(double) * (size_t)(l * m));
        if (!Or) { free(B); free(Bq); free(Wh); free(Ob); return 1; }
        for (int64_t e = 0; e < l * m; ++e) Or[e] = round_bf16(Omega[e]);
#pragma omp parallel for schedule(static)
        for (int64_t j = 0; j < n; ++j)
            for (int64_t r = 0; r < l; ++r) {
                double s = 0.0;
                for (int64_t q = 0; q < m; ++q) s += Or[r * m + q] * round_bf16(AT(A, lda, q, j));
                AT(B, l, r, j) = s;
            }
        free(Or);
    } else {
#pragma omp parallel for schedule(static)
        for (int64_t j = 0; j < n; ++j)
            for (int64_t r = 0; r < l; ++r) {
                double s = 0.0;
                for (int64_t q = 0; q < m; ++q) s += Omega[r * m + q] * AT(A, lda, q, j);
                AT(B, l, r, j) = s;
            }
    }
    for (int64_t j = 0; j < n; ++j) jpvt[j] = (int32_t)j;
    if (gaps) for (int64_t c = 0; c < k; ++c) gaps[c] = -1.0;

    double nu0max = 0.0;
    for (int64_t j = 0; j < n; ++j) {
        double nu = 0.0;
        for (int64_t r = 0; r < l; ++r) nu += AT(B, l, r, j) * AT(B, l, r, j);
        if (nu > nu0max) nu0max = nu;
    }
    const double gtol = 10.0 * (double)(m > n ? m : n) * ldexp(1.0, -53);
    const double guard = gtol * gtol * nu0max;
    int pivoting = 1;
    int64_t rank = k;

    for (int64_t i = 0; i < k; i += b) {
        const int64_t bb = (b < k - i) ? b : (k - i);
        int pivoted_block = pivoting;

        /* --- Alg. 2 "Partial QRCP on B(:,i:n) to get b pivots" (Alg. 1 on B) --- */
        if (pivoting) {
            double* Q = B;
            if (formula == 5) { memcpy(Bq, B, sizeof(double) * (size_t)(l * n)); Q = Bq; }
            /* tournament: the block's pivots chosen up front from B(:, i:n) as it is now; who[]
               and where[] follow the transpositions (position -> original position and back) */
            int64_t* tsel = NULL;
            int64_t* who = NULL;
            int64_t* where = NULL;
            double tgap = 1.0;
            if (tgs) {
                tsel = (int64_t*)malloc(sizeof(int64_t) * (size_t)bb);
                who = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
                where = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
                if (!tsel || !who || !where ||
                    orc_tournament(&AT(Q, l, 0, i), l, n - i, i, bb, tgs[i / b], fanin, tsel, &tgap) != bb) {
                    free(tsel); free(who); free(where); free(B); free(Bq); free(Wh); free(Ob);
                    return 1;
                }
                for (int64_t j = 0; j < n; ++j) who[j] = where[j] = j;
            }
            for (int64_t t = 0; t < bb; ++t) {
                const int64_t c = i + t;
                int64_t best = c;
                double v1 = -1.0, v2 = -1.0;
                if (tgs) {
                    best = where[tsel[t]];
                    v1 = 0.0;
                    for (int64_t r = t; r < l; ++r) v1 += AT(Q, l, r, best) * AT(Q, l, r, best);
                } else {
                    for (int64_t s = c; s < n; ++s) {
                        double nu = 0.0;
                        for (int64_t r = t; r < l; ++r) nu += AT(Q, l, r, s) * AT(Q, l, r, s);
                        if (nu > v1) { v2 = v1; v1 = nu; best = s; }
                        else if (nu > v2) v2 = nu;
                    }
                }
                if (v1 <= guard) { pivoting = 0; rank = c; break; }
                if (gaps) gaps[c] = tgs ? tgap : ((v2 < 0.0) ? 1.0 : (v1 - v2) / v1);
                if (tgs) {   /* the transposition c <-> best in the position maps */
                    const int64_t oc = who[c], ob = who[best];
                    who[c] = ob; who[best] = oc;
                    where[ob] = c; where[oc] = best;
                }
                /* Alg. 2 "Swap ... columns in A, Pi" (and in B). */
                swap_cols(A, lda, m, c, best);
                swap_cols(B, l, l, c, best);
                if (formula == 5) swap_cols(Bq, l, l, c, best);
                int32_t tp = jpvt[c]; jpvt[c] = jpvt[best]; jpvt[best] = tp;
                /* Householder on Q(t:l, c), applied to Q(t:l, c+1:n). */
                double* x = &AT(Q, l, t, c);
                double tb = house_gen(l - t, x);
#pragma omp parallel for schedule(static)
                for (int64_t s = c + 1; s < n; ++s) house_apply(l - t, x, tb, &AT(Q, l, t, s));
                for (int64_t r = t + 1; r < l; ++r) x[r - t] = 0.0; /* R_hat is upper */
            }
            free(tsel); free(who); free(where);
        }

        /* --- Alg. 2 "unpivoted QR on A(i:m, i:i+b-1)" --- */
        for (int64_t j = 0; j < bb; ++j) {
            const int64_t col = i + j;
            double* x = &AT(A, lda, col, col);
            tau[col] = house_gen(m - col, x);
            for (int64_t s = col + 1; s < i + bb; ++s) house_apply(m - col, x, tau[col], &AT(A, lda, col, s));
        }

        /* --- Alg. 2 "A(i:m,i+b:n) <- Q_tilde^T A(i:m,i+b:n)": reflectors one at a time --- */
#pragma omp parallel for schedule(static)
        for (int64_t s = i + bb; s < n; ++s)
            for (int64_t j = 0; j < bb; ++j) {
                const int64_t col = i + j;
                house_apply(m - col, &AT(A, lda, col, col), tau[col], &AT(A, lda, col, s));
            }

        /* --- B update, only while pivoting is still on after this block --- */
        if (!(pivoted_block && pivoting) || i + bb >= n) continue;
        if (formula == 4) {
            /* Eq. (4): B(0:bb, trail) <- R_hat12 - Omega_hat_11 R12, with
               Omega_hat_11 = R_hat11 R11^{-1} from Omega_hat_11 R11 = R_hat11
               (forward substitution over columns; both factors upper triangular). */
            for (int64_t j = 0; j < bb; ++j) {
                const double rjj = AT(A, lda, i + j, i + j);
                for (int64_t r = 0; r < bb; ++r) {
                    double s = AT(B, l, r, i + j);
                    for (int64_t q = 0; q < j; ++q) s -= Wh[q * b + r] * AT(A, lda, i + q, i + j);
                    Wh[j * b + r] = (rjj == 0.0) ? 0.0 : s / rjj;
                }
            }
#pragma omp parallel for schedule(static)
            for (int64_t s = i + bb; s < n; ++s)
                for (int64_t r = 0; r < bb; ++r) {
                    double acc = AT(B, l, r, s);
                    for (int64_t q = 0; q < bb; ++q) acc -= Wh[q * b + r] * AT(A, lda, i + q, s);
                    AT(B, l, r, s) = acc;
                }
        } else {
            /* Eq. (5): Omega_bar <- Omega_bar Q_tilde (reflectors applied from the right
               to the columns i..m-1 of Omega_bar, in order i, i+1, ...), then
               B(:, trail) <- B(:, trail) - Omega_bar(:, i:i+bb) R12. */
#pragma omp parallel for schedule(static)
            for (int64_t r = 0; r < l; ++r) {
                double* orow = &Ob[r * m];
                for (int64_t j = 0; j < bb; ++j) {
                    const int64_t col = i + j;
                    const double* v = &AT(A, lda, col, col);
                    if (tau[col] == 0.0) continue;
                    double w = orow[col];
                    for (int64_t q = col + 1; q < m; ++q) w += orow[q] * v[q - col];
                    w *= tau[col];
                    orow[col] -= w;
                    for (int64_t q = col + 1; q < m; ++q) orow[q] -= w * v[q - col];
                }
            }
#pragma omp parallel for schedule(static)
            for (int64_t s = i + bb; s < n; ++s)
                for (int64_t r = 0; r < l; ++r) {
                    double acc = AT(B, l, r, s);
                    for (int64_t q = 0; q < bb; ++q) acc -= Ob[r * m + i + q] * AT(A, lda, i + q, s);
                    AT(B, l, r, s) = acc;
                }
        }
    }
    if (rank_out) *rank_out = rank;
    if (Bout) memcpy(Bout, B, sizeof(double) * (size_t)(l * n));
    free(B); free(Bq); free(Wh); free(Ob);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Alg. 3 (SRQR, Sec. IV-E) on an explicit R.                                  */
/* ------------------------------------------------------------------------- */

/* Alg. 3 "Swap ... One-step QR factorization of A(l+1:m,l+1:n) ... |alpha| = R_{l+1,l+1}  */
/* ... r_i = r_i - A(l+1,i)^2": move the trailing column with the largest estimate r_i to  */
/* position l, reduce R(l:m, l) to its first entry with one reflector applied to the       */
/* trailing columns, and downdate the estimates by the new row l.  Returns |alpha|.         */
static double srqr_extra_pivot(int64_t m, int64_t n, int64_t l, double* R, int32_t* jpvt, double* r)
{
    int64_t best = l;
    for (int64_t i = l + 1; i < n; ++i)
        if (r[i] > r[best]) best = i;
    swap_cols(R, m, m, l, best);
    int32_t tp = jpvt[l]; jpvt[l] = jpvt[best]; jpvt[best] = tp;
    double tr = r[l]; r[l] = r[best]; r[best] = tr;
    double* x = &AT(R, m, l, l);
    const double t = house_gen(m - l, x);
    for (int64_t s = l + 1; s < n; ++s) house_apply(m - l, x, t, &AT(R, m, l, s));
    for (int64_t i = l + 1; i < m; ++i) AT(R, m, i, l) = 0.0;
    for (int64_t i = l + 1; i < n; ++i) r[i] -= AT(R, m, l, i) * AT(R, m, l, i);
    return fabs(AT(R, m, l, l));
}

/* Alg. 3 "g_2 ~ |alpha|/sqrt(d) ||Omega R_hat^{-T}||_{1,2}": X = Omega R_hat^{-T} row by row  */
/* (row q of X is R_hat^{-1} times row q of Omega, by back substitution on the leading     */
/* (l+1) x (l+1) block of R); ||X||_{1,2} is its largest column norm.  *imax receives that   */
/* column.  A zero diagonal entry of R_hat gives g_2 = +inf with *imax at that column.       */
static double srqr_g2(int64_t m, int64_t l, const double* R, double alpha, int64_t d, const double* Og,
                      double* X, double* cn, int64_t* imax)
{
    const int64_t w = l + 1;
    for (int64_t j = 0; j < w; ++j)
        if (AT(R, m, j, j) == 0.0) { *imax = j; return INFINITY; }
    for (int64_t q = 0; q < d; ++q)
        for (int64_t j = w - 1; j >= 0; --j) {
            double acc = Og[q * w + j];
            for (int64_t c = j + 1; c < w; ++c) acc -= AT(R, m, j, c) * X[q * w + c];
            X[q * w + j] = acc / AT(R, m, j, j);
        }
    int64_t best = 0;
    for (int64_t j = 0; j < w; ++j) {
        double ss = 0.0;
        for (int64_t q = 0; q < d; ++q) ss += X[q * w + j] * X[q * w + j];
        cn[j] = sqrt(ss);
        if (cn[j] > cn[best]) best = j;
    }
    *imax = best;
    return alpha / sqrt((double)d) * cn[best];
}

/*
 * SRQR: RQRCP to rank l (Alg. 2, Eq. (4), sketch Omega of b+p rows), then the extra pivot
 * chosen from the final sketch's column norms / (b+p), the randomized estimate of g_2 with a
 * fresh d x (l+1) Gaussian matrix per estimate (estimate t draws orc_omega(d, l+1, seed_g+t)),
 * and while g_2 > g: the worst column of R_hat (largest column of Omega R_hat^{-T}) rotated to
 * position l (round robin: the columns after it move left by one), Givens rotations on rows
 * (j, j+1) restoring the upper-trapezoidal form, the estimates r updated by row l, and a new
 * extra pivot.  At most max_swaps swaps.
 * R (m x n, ld m) receives the explicit factor: R(0:l+1, :) upper trapezoidal and the
 * trailing block R(l+1:m, l+1:n); A(:, jpvt) = Q R for an orthogonal Q (not formed).
 * Requires 1 <= l < min(m, n), g > 1, d >= 1.  Outputs: *swaps_out, the last *g2_out,
 * *alpha_out = |R(l, l)| and *rank_out, the pivots of the RQRCP stage before its rank guard
 * fired (l if it never did).  With rank < l, R_hat is singular to working precision and the
 * swap loop is skipped (g_2 is still estimated once).  Returns 0, a negative argument
 * position, or 1 on allocation failure.
 */
ORC_EXPORT int orc_srqr(int64_t m, int64_t n, const double* A, int64_t lda, int64_t l, int64_t b, int64_t p,
                        const double* Omega, double g, int64_t d, uint64_t seed_g, int64_t max_swaps,
                        double* R, int32_t* jpvt, int64_t* swaps_out, double* g2_out, double* alpha_out,
                        int64_t* rank_out)
{
    if (m < 2) return -1;
    if (n < 2) return -2;
    if (lda < m) return -4;
    if (l < 1 || l >= (m < n ? m : n)) return -5;
    if (b < 1) return -6;
    if (p < 0) return -7;
    if (!(g > 1.0)) return -9;
    if (d < 1) return -10;
    if (max_swaps < 0) return -12;
    const int64_t ls = b + p, w = l + 1;
    double* W = (double*)malloc(sizeof(double) * (size_t)(m * n));
    double* tau = (double*)malloc(sizeof(double) * (size_t)l);
    double* Bs = (double*)malloc(sizeof(double) * (size_t)(ls * n));
    double* r = (double*)malloc(sizeof(double) * (size_t)n);
    double* Og = (double*)malloc(sizeof(double) * (size_t)(d * w));
    double* X = (double*)malloc(sizeof(double) * (size_t)(d * w));
    double* cn = (double*)malloc(sizeof(double) * (size_t)w);
    int rc = 1;
    if (!W || !tau || !Bs || !r || !Og || !X || !cn) goto done;
    for (int64_t j = 0; j < n; ++j)
        for (int64_t i = 0; i < m; ++i) AT(W, m, i, j) = AT(A, lda, i, j);
    int64_t rank;
    rc = orc_rqrcp2(m, n, W, m, l, b, p, Omega, 4, 0, jpvt, tau, &rank, NULL, Bs);
    if (rc != 0) goto done;
    /* explicit R: upper trapezoid of the first l rows, and the trailing block W(l:m, l:n) */
    for (int64_t j = 0; j < n; ++j)
        for (int64_t i = 0; i < m; ++i)
            AT(R, m, i, j) = (i < l) ? (i <= j ? AT(W, m, i, j) : 0.0) : (j >= l ? AT(W, m, i, j) : 0.0);
    /* Alg. 3 "r_i = r_hat_i / (b+p)": squared column norms of the final sketch of R22 */
    for (int64_t i = l; i < n; ++i) {
        double ss = 0.0;
        for (int64_t q = 0; q < ls; ++q) ss += AT(Bs, ls, q, i) * AT(Bs, ls, q, i);
        r[i] = ss / (double)ls;
    }
    double alpha = srqr_extra_pivot(m, n, l, R, jpvt, r);
    int64_t imax, swaps = 0;
    orc_omega(d, w, seed_g, Og);
    double g2 = srqr_g2(m, l, R, alpha, d, Og, X, cn, &imax);
    while (g2 > g && swaps < max_swaps && rank >= l) {
        /* round robin: column imax goes to position l, columns imax+1..l move left by one */
        for (int64_t j = imax; j < l; ++j) {
            swap_cols(R, m, m, j, j + 1);
            int32_t tp = jpvt[j]; jpvt[j] = jpvt[j + 1]; jpvt[j + 1] = tp;
        }
        /* Givens rotations on rows (j, j+1) zero the subdiagonal of R(0:l+1, imax:l) */
        for (int64_t j = imax; j < l; ++j) {
            const double a = AT(R, m, j, j), bsub = AT(R, m, j + 1, j);
            if (bsub != 0.0) {
                const double h = hypot(a, bsub), c = a / h, sn = bsub / h;
                for (int64_t col = j; col < n; ++col) {
                    const double x = AT(R, m, j, col), y = AT(R, m, j + 1, col);
                    AT(R, m, j, col) = c * x + sn * y;
                    AT(R, m, j + 1, col) = -sn * x + c * y;
                }
            }
            AT(R, m, j + 1, j) = 0.0;
        }
        /* Alg. 3 "r_{l+1} = R_{l+1,l+1}^2; r_i = r_i + A(l+1,i)^2": row l rejoins the trailing rows */
        r[l] = AT(R, m, l, l) * AT(R, m, l, l);
        for (int64_t i = l + 1; i < n; ++i) r[i] += AT(R, m, l, i) * AT(R, m, l, i);
        alpha = srqr_extra_pivot(m, n, l, R, jpvt, r);
        ++swaps;
        orc_omega(d, w, seed_g + (uint64_t)swaps, Og);
        g2 = srqr_g2(m, l, R, alpha, d, Og, X, cn, &imax);
    }
    if (swaps_out) *swaps_out = swaps;
    if (g2_out) *g2_out = g2;
    if (alpha_out) *alpha_out = alpha;
    if (rank_out) *rank_out = rank;
    rc = 0;
done:
    free(W); free(tau); free(Bs); free(r); free(Og); free(X); free(cn);
    return rc;
}

/* ------------------------------------------------------------------------- */
/* Q = H_0 H_1 ... H_{k-1} restricted to its first ncols columns (Alg. 2,      */
/* "Q is the product of Q_tilde").  Backward accumulation on the identity.     */
/* ------------------------------------------------------------------------- */
ORC_EXPORT void orc_form_q(int64_t m, int64_t k, const double* A, int64_t lda, const double* tau,
                           int64_t ncols, double* Q, int64_t ldq)
{
    for (int64_t j = 0; j < ncols; ++j)
        for (int64_t r = 0; r < m; ++r) AT(Q, ldq, r, j) = (r == j) ? 1.0 : 0.0;
    for (int64_t h = k - 1; h >= 0; --h) {
#pragma omp parallel for schedule(static)
        for (int64_t j = 0; j < ncols; ++j) house_apply(m - h, &AT(A, lda, h, h), tau[h], &AT(Q, ldq, h, j));
    }
}

/* x <- H_0 H_1 ... H_{k-1} x for one vector x of length m (Q times x, Alg. 2 output). */
ORC_EXPORT void orc_apply_q(int64_t m, int64_t k, const double* A, int64_t lda, const double* tau, double* x)
{
    for (int64_t h = k - 1; h >= 0; --h) house_apply(m - h, &AT(A, lda, h, h), tau[h], x + h);
}

/* ------------------------------------------------------------------------- */
/* Low-rank product L = Q1 [R11 R12] Pi^T (Sec. I-A): column jpvt[c] of L is   */
/* Q1 times column c of the k x n upper trapezoid of the factored A.  Q1       */
/* (m x k, optional) receives the first k columns of Q.                        */
/* ------------------------------------------------------------------------- */
ORC_EXPORT int orc_lowrank(int64_t m, int64_t n, int64_t k, const double* A, int64_t lda,
                           const double* tau, const int32_t* jpvt, double* L, int64_t ldl, double* Q1)
{
    double* Q = (double*)malloc(sizeof(double) * (size_t)(m * k));
    if (!Q) return 1;
    orc_form_q(m, k, A, lda, tau, k, Q, m);
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < n; ++c) {
        int64_t top = (c + 1 < k) ? c + 1 : k;
        double* out = &AT(L, ldl, 0, jpvt[c]);
        for (int64_t r = 0; r < m; ++r) out[r] = 0.0;
        for (int64_t q = 0; q < top; ++q) {
            double rq = AT(A, lda, q, c);
            for (int64_t r = 0; r < m; ++r) out[r] += AT(Q, m, r, q) * rq;
        }
    }
    if (Q1) memcpy(Q1, Q, sizeof(double) * (size_t)(m * k));
    free(Q);
    return 0;
}
