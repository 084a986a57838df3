// pivot_common.cuh -- pieces shared by the two pivot searches on the sketch B (pivot.cu: the
// partial QRCP of Alg. 2; tournament.cu: QR with tournament pivoting): the argmax order on squared
// norms, warp and column reductions, and the bookkeeping that turns a block's transpositions into
// jpvt, the pivot list and the net column map of the swap kernels.
#pragma once

#include <climits>

#include "internal.cuh"

namespace rq {

// Order key of a squared norm: non-negative doubles order as their bit patterns read as signed
// 64-bit integers, and every negative value (the "no candidate" -1.0) maps below them.  Integer
// compares keep the argmax off the FP64 pipe; the order is that of the values.
__device__ __forceinline__ long long norm_key(double v)
{
    const long long b = __double_as_longlong(v);
    return b < 0 ? -1LL : b;
}

// (v1, p1) before (v2, p2): the larger norm, ties to the smaller position.
__device__ __forceinline__ bool better(double v1, long long p1, double v2, long long p2)
{
    const long long k1 = norm_key(v1), k2 = norm_key(v2);
    return k1 > k2 || (k1 == k2 && p1 < p2);
}

// Warp-wide argmax over (value, position, index) triples by shuffles; every lane ends with the
// warp's winner.
__device__ __forceinline__ void warp_argmax(double& v, long long& p, int& idx)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffffu, v, o);
        const long long op = __shfl_xor_sync(0xffffffffu, p, o);
        const int oi = __shfl_xor_sync(0xffffffffu, idx, o);
        if (better(ov, op, v, p)) {
            v = ov;
            p = op;
            idx = oi;
        }
    }
}

// Per-column reduction over the tpc threads that share a column (adjacent lanes).
template <typename T>
__device__ __forceinline__ T column_sum(T v, int tpc)
{
    for (int o = 1; o < tpc; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Shared-memory scratch of finish_pivots for a block of bb pivots.
__host__ __device__ constexpr size_t finish_scratch_bytes(int bb)
{
    return (size_t)2 * bb * (2 * sizeof(long long) + sizeof(int32_t));
}

// The block's transpositions (i + t <-> pivs[t]), t = 0 .. bb-1, applied in order to the column
// positions: piv[t] = pivs[t]; jpvt permuted the same way; swapmap = the count, then (destination,
// source) pairs of every position whose column moved (the net map the swap kernels apply).  Only
// the positions i .. i+bb-1 and the pivs[t] can move; one thread per such position follows it
// through the bb transpositions, so no thread walks a list.  Every thread of the block calls this
// (it synchronises the block); pivs is shared memory, scr holds finish_scratch_bytes(bb) bytes of
// shared memory aligned to 8 bytes.
__device__ inline void finish_pivots(long long i, int bb, const long long* pivs, int32_t* jpvt, int32_t* piv,
                                     long long* swapmap, void* scr)
{
    long long* sdst = static_cast<long long*>(scr);
    long long* ssrc = sdst + 2 * bb;
    int32_t* sjv = reinterpret_cast<int32_t*>(ssrc + 2 * bb);
    const int tid = threadIdx.x, nth = blockDim.x;
    for (int t = tid; t < bb; t += nth) piv[t] = (int32_t)pivs[t];
    for (int q = tid; q < 2 * bb; q += nth) {
        long long x;
        bool valid = true;
        if (q < bb) {
            x = i + q;
        } else {
            const int t = q - bb;
            x = pivs[t];
            if (x < i + bb) valid = false;  // listed among i .. i+bb-1 already
            for (int u = 0; u < t && valid; ++u)
                if (pivs[u] == x) valid = false;  // listed by an earlier step
        }
        long long y = x;
        if (valid)
            for (int t = 0; t < bb; ++t) {
                const long long c = i + t, p = pivs[t];
                if (y == c)
                    y = p;
                else if (y == p)
                    y = c;
            }
        sdst[q] = valid ? y : -1;
        ssrc[q] = x;
        sjv[q] = (valid && y != x) ? jpvt[x] : 0;
    }
    __syncthreads();
    for (int q = tid; q < 2 * bb; q += nth)
        if (sdst[q] >= 0 && sdst[q] != ssrc[q]) jpvt[sdst[q]] = sjv[q];
    if (tid < 32) {
        long long cnt = 0;
        for (int q0 = 0; q0 < 2 * bb; q0 += 32) {
            const int q = q0 + tid;
            const bool mv = q < 2 * bb && sdst[q] >= 0 && sdst[q] != ssrc[q];
            const unsigned m = __ballot_sync(0xffffffffu, mv);
            if (mv) {
                const long long e = cnt + __popc(m & ((1u << tid) - 1u));
                swapmap[1 + 2 * e] = sdst[q];
                swapmap[2 + 2 * e] = ssrc[q];
            }
            cnt += __popc(m);
        }
        if (tid == 0) swapmap[0] = cnt;
    }
}

}  // namespace rq
