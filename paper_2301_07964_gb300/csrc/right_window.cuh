// Delayed right updates of one tile of rows by the group's reflectors, with a sliding window
// (Alg. 4, first loop), in native FP64.  Shared by the FP64 apply kernel (stage2.cu) and the
// emulated ones (emu.cu, emu_tc.cu), which run the staircase blocks of their tiles through it.
//
// Rows x0 .. x0+NR-1 (NR = NT/4, four lanes per row: lane l of a row owns entries l, l+4, ...
// of each reflector) receive the reflectors of blocks kstart down to kstop, each block's in
// sweep order, through a window of w = r + qg - 1 columns in shared memory (sm: w*(NR+1) +
// qg*r + qg doubles).  kind 0, 1 (A, B): reflector Z^_k^j applies to row x only while
// x < i4(k, j), the rows the generate phase did not update; kind 2, 3 (Z, Q): all rows.  A
// warp none of whose rows takes a reflector skips it (an FP64 instruction costs the same
// whether one lane or all are active, and in the staircase blocks about half of the pairs of
// 8-row band and reflector are idle).
// The next window's new columns are loaded into registers while the current window is updated.
// tid is the thread's index in its group of NT threads and bar the id of that group's barrier
// (0 for a whole block).
#pragma once

#include "hts_internal.cuh"

namespace hts {

constexpr int kRightLanes = 4;

template <int NT>
__device__ __forceinline__ void right_window_rows(double *X, int ld, int kind, const double *Vs, const double *Ts,
                                                  int kdim, int n, int r, int j1, int qg, int x0, int kstart,
                                                  int kstop, double *sm, int tid, int bar)
{
    constexpr int NR = NT / kRightLanes;                    // rows per thread block
    constexpr int kPrefetch = kMaxR * NR / NT;              // new elements per thread
    const int LDS = NR + 1;
    const int w = r + qg - 1;
    double *buf = sm;                       // [w][LDS]: row rr of the tile, window column p
    double *vr = buf + (size_t)w * LDS;     // [qg][r]
    double *tr = vr + (size_t)qg * r;       // [qg]
    const int rr = tid / kRightLanes, sub = tid % kRightLanes;
    const int x = x0 + rr;

    // window kstart: all w columns
    {
        const int c0 = j1 + kstart * r + 1;
        for (int e = tid; e < w * NR; e += NT) {
            const int p = e / NR, re = e % NR;
            const int c = c0 + p, xr = x0 + re;
            if (c <= n && xr <= n) buf[p * LDS + re] = X[AT(ld, xr, c)];
        }
    }
    double pre[kPrefetch];
    for (int k = kstart; k >= kstop; --k) {
        const int c0 = j1 + k * r + 1;
        for (int e = tid; e < qg * r; e += NT) {
            const int sidx = e / r, i = e % r;
            vr[e] = Vs[((size_t)sidx * kdim + k) * r + i];
        }
        for (int e = tid; e < qg; e += NT) tr[e] = Ts[(size_t)e * kdim + k];
        // prefetch the r new columns of window k-1 (columns c0-r .. c0-1)
        if (k > kstop) {
#pragma unroll
            for (int t = 0; t < kPrefetch; ++t) {
                const int e = tid + t * NT;
                const int p = e / NR, re = e % NR;
                const int c = c0 - r + p, xr = x0 + re;
                pre[t] = (p < r && xr <= n) ? X[AT(ld, xr, c)] : 0.0;
            }
        }
        group_sync(bar, NT);
        for (int sidx = 0; sidx < qg; ++sidx) {
            const double tau = tr[sidx];
            if (tau == 0.0) continue;
            const int jj = j1 + sidx;
            const bool active = x <= n && (kind > 1 || x < j1 + 1 + imax(0, (k + jj - j1 - qg) * r));
            if (!__any_sync(0xffffffffu, active)) continue;   // the loop is warp-uniform up to here
            const int mlen = imin(r, n - (jj + k * r));
            const double *v = vr + sidx * r;
            double *b = buf + sidx * LDS + rr;
            double d = 0.0;
            if (active)
                for (int i = sub; i < mlen; i += kRightLanes) d += b[i * LDS] * v[i];
            d += __shfl_xor_sync(0xffffffffu, d, 1);
            d += __shfl_xor_sync(0xffffffffu, d, 2);
            d *= tau;
            if (active)
                for (int i = sub; i < mlen; i += kRightLanes) b[i * LDS] -= d * v[i];
        }
        group_sync(bar, NT);
        // store the columns that leave the window, keep the overlap, insert the prefetch
        const int plo = (k > kstop) ? qg - 1 : 0;
        const int np = w - plo;
        for (int e = tid; e < np * NR; e += NT) {
            const int p = plo + e / NR, re = e % NR;
            const int c = c0 + p, xr = x0 + re;
            if (c <= n && xr <= n) X[AT(ld, xr, c)] = buf[p * LDS + re];
        }
        if (k > kstop) {
            group_sync(bar, NT);
            for (int e = tid; e < (qg - 1) * NR; e += NT) {
                const int p = e / NR, re = e % NR;
                buf[(p + r) * LDS + re] = buf[p * LDS + re];
            }
            group_sync(bar, NT);
#pragma unroll
            for (int t = 0; t < kPrefetch; ++t) {
                const int e = tid + t * NT;
                const int p = e / NR, re = e % NR;
                if (p < r) buf[p * LDS + re] = pre[t];
            }
            group_sync(bar, NT);
        }
    }
}

}  // namespace hts
