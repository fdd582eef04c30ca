// Generate phase of stage 2 (Alg. 3 of Steel & Vandebril): the near-diagonal bulge chase of
// one group of qg sweeps j1 .. j1+qg-1.
//
// Thread block s owns sweep j = j1 + s and walks its blocks k = 0, 1, ...  Step (k, j) may
// start once sweep j-1 has finished block k+2: (k, j) reads the column that (k+1, j-1)
// mixed, and its band update writes the pivot row of (k+2, j-1).  Sweeps therefore advance as
// a wavefront three blocks apart, synchronised through one progress word per sweep (release /
// acquire at GPU scope, waits bounded in time).
//
// Each sweep also has a helper block.  A step's band update covers rows i4 .. i3; only the
// rows from cr = j1 + k r + 1 down are ever read by a later step of the group (pivot columns,
// B blocks); the rows above exist to keep the group's reflectors in order for the delayed
// updates.  The main block updates rows >= cr and publishes; the helper block then updates
// rows i4 .. cr-1 and publishes its own progress, on which the next sweep waits (block k+1 of
// the helper before step k).
//
// One step, in native FP64:
//   1. prefetch: pivot column segment A(rlo:rhi, jb), the block's newest B column, the earlier
//      sweeps' left reflectors of block k and the rest of the B block (one memory round trip);
//   2. lazy left updates of the two segments by those reflectors (warp 0: A, warp 1: B);
//   3. left reflector Q^_k^j reducing A(i1:i2, jb);
//   4. B block := Q^ B block;
//   5. RQ of the B block, last row first, accumulating the right factor G (W G = R~);
//   6. opposite reflector Z^_k^j mapping the first row of Q~ = G(:, 1)^T to beta e_1;
//   7. band update A(cr:i3, i1:i2) Z^, B(cr:i2, i1:i2) Z^, with B(i1+1:i2, i1) = 0 exactly
//      (rows i4 .. cr-1 by the helper block);
//   8. publish block k of sweep j.
// Block-level updates use groups of 8 lanes per row or column (3-level reductions), so one
// round covers up to 32 rows.
#include "schedule.cuh"

namespace hts {

namespace {

constexpr int kLds = kMaxR + 1;              // leading dimension of the shared r x r tiles
constexpr int kGrp = 8;                      // lanes per row / column group
constexpr int kNGrp = kGenThreads / kGrp;    // groups per thread block
constexpr int kSlots = kMaxR / kGrp;         // elements per lane of a row of length <= kMaxR

__device__ __forceinline__ double grp_sum(double v)
{
    v += __shfl_xor_sync(0xffffffffu, v, 4);
    v += __shfl_xor_sync(0xffffffffu, v, 2);
    v += __shfl_xor_sync(0xffffffffu, v, 1);
    return v;
}

}  // namespace

__global__ void __launch_bounds__(kGenThreads) k_s2_generate(GenArgs a)
{
    __shared__ double col[2 * kMaxR];       // pivot column segment
    __shared__ double bcol[2 * kMaxR];      // newest B column segment
    __shared__ double W[kMaxR * kLds];      // B block (row-major), then the RQ work array
    __shared__ double G[kMaxR * kLds];      // accumulated right factor of the RQ (row-major)
    __shared__ double lv[kMaxR * kMaxR];    // earlier sweeps' left reflectors of block k
    __shared__ double lt[kMaxR];            // and their taus
    __shared__ double vv[kMaxR];            // current reflector
    __shared__ double s_tau;
    __shared__ int s_abort;

    const bool helper = (int)blockIdx.x >= a.qg;
    const int s = helper ? (int)blockIdx.x - a.qg : (int)blockIdx.x;
    const int j = a.j1 + s;
    const int n = a.n, r = a.r, j1 = a.j1, qg = a.qg;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int gl = lane & (kGrp - 1);
    const int kdim = a.R.kdim;
    const int kl = nblocks_lazy(n, r, j);
    const int kg = nblocks_gen(n, r, j);
    const int kl_prev = s > 0 ? nblocks_lazy(n, r, j - 1) : 0;
    double *VQs = a.R.VQ + (size_t)s * kdim * r;
    double *VZs = a.R.VZ + (size_t)s * kdim * r;
    double *TQs = a.R.TQ + (size_t)s * kdim;
    double *TZs = a.R.TZ + (size_t)s * kdim;
    double *A = a.A, *B = a.B;
    const int lda = a.lda, ldb = a.ldb;
    const int nlazy = j - j1;

    for (int k = kg + tid; !helper && k < kdim; k += kGenThreads) {   // blocks this sweep does not reach
        TQs[k] = 0.0;
        TZs[k] = 0.0;
    }
    if (tid == 0) s_abort = __ldcg(a.status) != 0;   // an earlier kernel of this call failed
    __syncthreads();
    if (s_abort) return;
    unsigned long long *hflags = a.flags + a.qmax;       // progress of the helper blocks

    if (helper) {
        // Band rows above the critical rows of each step: rows i4 .. cr-1, where cr = j1+kr+1
        // is the first row of block k that any step reads.  They only carry the ordering of
        // the group's reflectors, so they are updated here, behind the main block.
        for (int k = 0; k < kg; ++k) {
            if (tid == 0) {
                const bool ok = wait_at_least(a.flags + s, a.epoch | (unsigned long long)(k + 1), a.status, a.group, k, j) &&
                                (s == 0 || wait_at_least(hflags + s - 1, a.epoch | (unsigned long long)(k + 2), a.status,
                                                         a.group, k, j));
                s_abort = !ok;
            }
            __syncthreads();
            if (s_abort) return;
            const StepGeom g = step_geom(n, r, j1, qg, k, j);
            const int m = g.i2 - g.i1 + 1;
            const int cr = j1 + k * r + 1;
            const double tz = __ldcg(TZs + k);
            if (tid < kMaxR) vv[tid] = tid < m ? __ldcg(VZs + (size_t)k * r + tid) : 0.0;
            __syncthreads();
            const int na = imax(0, imin(cr - 1, g.i3) - g.i4 + 1), nbr = imax(0, imin(cr - 1, g.i2) - g.i4 + 1);
            if (tz != 0.0) band_rows(A, lda, B, ldb, g.i4, na, nbr, g.i1, m, tz, vv, false);
            __threadfence();
            __syncthreads();
            if (tid == 0) st_release_u64(hflags + s, a.epoch | (unsigned long long)(k + 1));
        }
        if (tid == 0) st_release_u64(hflags + s, a.epoch | 0xffffffffULL);
        return;
    }

    __shared__ UpdWait uw;   // the previous group's update tiles (look-ahead), checked by thread 0
    if (tid == 0) uw.init(a.uflags, a.uplan, a.uepoch, n);
    for (int k = 0; k < kl; ++k) {
        // ---- wait until sweep j-1 has finished block k+2 (or all of its blocks), and its helper
        //      block k+1: the helper's rows of block k+1 include the upper rows of this step's
        //      newest B column (read by the prefetch) and share column i2 with this step's band;
        //      and until the previous group's update has finished the tiles this step touches
        if (tid == 0) {
            const StepGeom gk = step_geom(n, r, j1, qg, k, j);
            s_abort = !uw.wait_for(gk.i2, gk.i3, a.status, a.group, k, j);
        }
        if (tid == 0 && s > 0 && !s_abort)
            s_abort = !(wait_at_least(a.flags + s - 1, a.epoch | (unsigned long long)imin(k + 3, kl_prev), a.status,
                                      a.group, k, j) &&
                        wait_at_least(hflags + s - 1, a.epoch | (unsigned long long)(k + 2), a.status, a.group, k, j));
        __syncthreads();
        if (s_abort) return;

        const StepGeom g = step_geom(n, r, j1, qg, k, j);
        const bool gen = k < kg;
        const int rlo = j1 + k * r + 1;
        const int rhi = imin(j + (k + 1) * r, n);
        const int L = rhi - rlo + 1;
        const int cb = g.i1 + r - 1;
        const bool hasb = cb <= n;
        const int m = g.i2 - g.i1 + 1;
        const int off = j - j1;

        // ---- 1. prefetch
        for (int i = tid; i < L; i += kGenThreads) {
            col[i] = __ldcg(A + AT(lda, rlo + i, g.jb));
            if (hasb) bcol[i] = __ldcg(B + AT(ldb, rlo + i, cb));
        }
        for (int e = tid; e < nlazy * r; e += kGenThreads) {
            const int sh = e / r, i = e % r;
            lv[e] = (k < nblocks_gen(n, r, j1 + sh)) ? __ldcg(a.R.VQ + ((size_t)sh * kdim + k) * r + i) : 0.0;
        }
        for (int e = tid; e < nlazy; e += kGenThreads)
            lt[e] = (k < nblocks_gen(n, r, j1 + e)) ? __ldcg(a.R.TQ + (size_t)e * kdim + k) : 0.0;
        if (gen) {
            for (int e = tid; e < m * m; e += kGenThreads) {
                const int i = e % m, c = e / m;
                if (!(hasb && c == m - 1)) W[i * kLds + c] = __ldcg(B + AT(ldb, g.i1 + i, g.i1 + c));
            }
        }
        __syncthreads();

        // ---- 2. lazy left updates (warp 0: A segment, warp 1: B segment)
        if (L > 0 && (warp == 0 || (warp == 1 && hasb))) {
            double *seg = (warp == 0) ? col : bcol;
            for (int sh = 0; sh < nlazy; ++sh) {
                const double tau = lt[sh];
                if (tau == 0.0) continue;
                const int jh = j1 + sh;
                const int mh = imin(jh + (k + 1) * r, n) - (jh + k * r + 1) + 1;
                const double v = lane < mh ? lv[sh * r + lane] : 0.0;
                const double x = lane < mh ? seg[sh + lane] : 0.0;
                const double d = warp_sum(v * x) * tau;
                if (lane < mh) seg[sh + lane] = x - d * v;
                __syncwarp();
            }
        }
        __syncthreads();

        // ---- 3. left reflector Q^_k^j
        if (gen && warp == 0) {
            const double x = lane < m ? col[off + lane] : 0.0;
            double beta, vi;
            const double tau = warp_larfg_fast(x, m, lane, &beta, &vi);
            if (lane < r) VQs[(size_t)k * r + lane] = lane < m ? vi : 0.0;
            vv[lane] = lane < m ? vi : 0.0;
            if (lane < m) col[off + lane] = (lane == 0) ? beta : 0.0;
            if (lane == 0) {
                TQs[k] = tau;
                s_tau = tau;
            }
        }
        if (gen && hasb)
            for (int i = tid; i < m; i += kGenThreads) W[i * kLds + m - 1] = bcol[off + i];
        __syncthreads();
        for (int i = tid; i < L; i += kGenThreads) {
            A[AT(lda, rlo + i, g.jb)] = col[i];
            if (hasb) B[AT(ldb, rlo + i, cb)] = bcol[i];
        }

        if (gen) {
            // ---- 4. B block := Q^ B block (one 8-lane group per column)
            const double tq = s_tau;
            if (tq != 0.0) {
                for (int cbase = warp * 4; cbase < m; cbase += kNGrp) {
                    const int c = cbase + (lane >> 3);
                    double d = 0.0;
#pragma unroll
                    for (int sl = 0; sl < kSlots; ++sl) {
                        const int i = gl + kGrp * sl;
                        if (c < m && i < m) d += W[i * kLds + c] * vv[i];
                    }
                    d = grp_sum(d) * tq;
#pragma unroll
                    for (int sl = 0; sl < kSlots; ++sl) {
                        const int i = gl + kGrp * sl;
                        if (c < m && i < m) W[i * kLds + c] -= d * vv[i];
                    }
                }
            }
            __syncthreads();
            for (int e = tid; e < m * m; e += kGenThreads) {
                const int i = e % m, c = e / m;
                B[AT(ldb, g.i1 + i, g.i1 + c)] = W[i * kLds + c];
                G[i * kLds + c] = (i == c) ? 1.0 : 0.0;
            }
            __syncthreads();

            // ---- 5. RQ of the block, last row first
            for (int sr = m; sr >= 2; --sr) {
                if (warp == 0) {
                    // pivot W(sr, sr) on lane 0, then W(sr, sr-1), ..., W(sr, 1)
                    const double x = lane < sr ? W[(sr - 1) * kLds + (sr - 1 - lane)] : 0.0;
                    double beta, vi;
                    const double tau = warp_larfg_fast(x, sr, lane, &beta, &vi);
                    if (lane < sr) vv[sr - 1 - lane] = vi;
                    if (lane == 0) s_tau = tau;
                }
                __syncthreads();
                const double tr = s_tau;
                if (tr != 0.0) {
                    const int nrows = (sr - 1) + m;   // W rows 1..sr-1 and all rows of G
                    for (int rb = warp * 4; rb < nrows; rb += kNGrp) {
                        const int row = rb + (lane >> 3);
                        const bool live = row < nrows;
                        double *Mrow = live ? (row < sr - 1 ? &W[row * kLds] : &G[(row - (sr - 1)) * kLds]) : W;
                        double d = 0.0;
#pragma unroll
                        for (int sl = 0; sl < kSlots; ++sl) {
                            const int c = gl + kGrp * sl;
                            if (live && c < sr) d += Mrow[c] * vv[c];
                        }
                        d = grp_sum(d) * tr;
#pragma unroll
                        for (int sl = 0; sl < kSlots; ++sl) {
                            const int c = gl + kGrp * sl;
                            if (live && c < sr) Mrow[c] -= d * vv[c];
                        }
                    }
                }
                __syncthreads();
            }

            // ---- 6. opposite reflector Z^_k^j reducing the first row of Q~
            if (warp == 0) {
                const double x = lane < m ? G[lane * kLds] : 0.0;
                double beta, vi;
                const double tz = warp_larfg_fast(x, m, lane, &beta, &vi);
                if (lane < r) VZs[(size_t)k * r + lane] = lane < m ? vi : 0.0;
                vv[lane] = lane < m ? vi : 0.0;
                if (lane == 0) {
                    TZs[k] = tz;
                    s_tau = tz;
                }
            }
            __syncthreads();

            // ---- 7. band updates of the critical rows (rows >= cr = j1+kr+1; the rows above
            //      go to the helper block)
            const double tz = s_tau;
            const int x0 = imax(g.i4, j1 + k * r + 1);
            const int na = imax(0, g.i3 - x0 + 1), nbr = imax(0, g.i2 - x0 + 1);
            band_rows(A, lda, B, ldb, x0, na, nbr, g.i1, m, tz, vv, true);
        }

        // ---- 8. publish block k of this sweep
        __threadfence();
        __syncthreads();
        if (tid == 0 && !(a.stall && s == 0))
            st_release_u64(a.flags + s, a.epoch | (unsigned long long)(k + 1));
    }
}

cudaError_t launch_s2_generate(const GenArgs &a, cudaStream_t st)
{
    void *args[] = {(void *)&a};
    // qg main blocks (one per sweep) and qg helper blocks
    return cudaLaunchCooperativeKernel((const void *)k_s2_generate, dim3(2 * a.qg), dim3(kGenThreads), args, 0, st);
}

}  // namespace hts
