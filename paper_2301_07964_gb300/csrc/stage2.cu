// Stage 2 of the two-stage HT reduction: r-HT pencil -> HT pencil by bulge chasing
// (Steel & Vandebril, Section "Reduction to Hessenberg-triangular form").
//
// One group of qg consecutive sweeps j1 .. j1+qg-1 is processed by three launches:
//   k_s2_generate     Alg. 3 (generate phase): the near-diagonal chase.  One thread block
//                     per sweep; block s runs sweep j1+s over its blocks k and waits (bounded)
//                     on block s-1, so the sweeps advance as a wavefront three blocks apart.
//   k_s2_apply_right  Alg. 4, right-hand part: the delayed Z^ reflectors on the rows of A
//                     and B above the generate band, and on all rows of Z; the Q^ reflectors
//                     on all rows of Q.
//   k_s2_apply_left   Alg. 4, left-hand part: the delayed Q^ reflectors on the columns of A
//                     and B right of the columns the generate phase already updated.
// The delayed updates walk the blocks k from the last to the first with a sliding window of
// r + qg - 1 columns (rows), so every element is read and written once per group; inside
// the window the group's reflectors are applied one at a time in FP64.
#include "hts_internal.cuh"

namespace hts {

__device__ __forceinline__ unsigned long long globaltimer_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

constexpr int kLds = kMaxR + 1;   // leading dimension of the shared r x r tiles

// ---------------------------------------------------------------------------------------
// Generate phase (Alg. 3).  Thread block s owns sweep j = j1 + s.
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kGenThreads) k_s2_generate(GenArgs a)
{
    __shared__ double col[2 * kMaxR];   // pivot column segment A(rlo:rhi, jb)
    __shared__ double bcol[2 * kMaxR];  // B(rlo:rhi, i1+r-1), the block's newest column
    __shared__ double W[kMaxR * kLds];  // B block, then its RQ work array
    __shared__ double G[kMaxR * kLds];  // accumulated right factor of the RQ
    __shared__ double vv[kMaxR];        // current reflector vector
    __shared__ double s_tau;
    __shared__ int s_abort;

    const int s = blockIdx.x;
    const int j = a.j1 + s;
    const int n = a.n, r = a.r, j1 = a.j1, qg = a.qg;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nwarps = kGenThreads / 32;
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

    // blocks this sweep does not reach carry no reflector
    for (int k = kg + tid; k < kdim; k += kGenThreads) {
        TQs[k] = 0.0;
        TZs[k] = 0.0;
    }
    if (tid == 0) s_abort = __ldcg(a.status) != 0;   // an earlier kernel of this call failed
    __syncthreads();
    if (s_abort) return;

    for (int k = 0; k < kl; ++k) {
        // ---- wait until sweep j-1 has finished block k+2 (or all of its blocks)
        if (tid == 0 && s > 0) {
            const unsigned long long need = a.epoch | (unsigned long long)imin(k + 3, kl_prev);
            const unsigned long long t0 = globaltimer_ns();
            long long polls = 0;
            while (ld_acquire_u64(a.flags + s - 1) < need) {
                if (++polls > kSpinLimit || globaltimer_ns() - t0 > kWaitLimitNs) {
                    record_error(a.status, HTS_ERR_TIMEOUT, 0, a.group, k, j);
                    s_abort = 1;
                    break;
                }
            }
        }
        __syncthreads();
        if (s_abort) return;

        const StepGeom g = step_geom(n, r, j1, qg, k, j);
        const bool gen = k < kg;
        const int rlo = j1 + k * r + 1;
        const int rhi = imin(j + (k + 1) * r, n);
        const int L = rhi - rlo + 1;
        const int cb = g.i1 + r - 1;
        const bool hasb = cb <= n;

        // ---- load the pivot column segment and the block's newest B column
        for (int i = tid; i < L; i += kGenThreads) {
            col[i] = __ldcg(A + AT(lda, rlo + i, g.jb));
            if (hasb) bcol[i] = __ldcg(B + AT(ldb, rlo + i, cb));
        }
        __syncthreads();

        // ---- lazy left updates: the earlier sweeps' reflectors of block k (warp 0: A,
        //      warp 1: B)
        if (L > 0 && (warp == 0 || (warp == 1 && hasb))) {
            double *seg = (warp == 0) ? col : bcol;
            for (int jh = j1; jh < j; ++jh) {
                if (k >= nblocks_gen(n, r, jh)) continue;
                const int sh = jh - j1;
                const double tau = __ldcg(a.R.TQ + (size_t)sh * kdim + k);
                if (tau == 0.0) continue;
                const int mh = imin(jh + (k + 1) * r, n) - (jh + k * r + 1) + 1;
                const double v = lane < mh ? __ldcg(a.R.VQ + ((size_t)sh * kdim + k) * r + lane) : 0.0;
                const double x = lane < mh ? seg[sh + lane] : 0.0;
                const double d = warp_sum(v * x) * tau;
                if (lane < mh) seg[sh + lane] = x - d * v;
                __syncwarp();
            }
        }
        __syncthreads();

        // ---- left reflector Q^_k^j reducing A(i1:i2, jb)
        const int m = g.i2 - g.i1 + 1;
        const int off = j - j1;            // offset of row i1 in the segment
        if (gen && warp == 0) {
            const double x = lane < m ? col[off + lane] : 0.0;
            double beta, vi;
            const double tau = warp_larfg(x, m, lane, &beta, &vi);
            if (lane < r) VQs[(size_t)k * r + lane] = lane < m ? vi : 0.0;
            vv[lane] = lane < m ? vi : 0.0;
            if (lane < m) col[off + lane] = (lane == 0) ? beta : 0.0;
            if (lane == 0) {
                TQs[k] = tau;
                s_tau = tau;
            }
        }
        __syncthreads();
        for (int i = tid; i < L; i += kGenThreads) {
            A[AT(lda, rlo + i, g.jb)] = col[i];
            if (hasb) B[AT(ldb, rlo + i, cb)] = bcol[i];
        }

        if (gen) {
            // ---- B block B(i1:i2, i1:i2) := Q^ B(i1:i2, i1:i2)
            for (int e = tid; e < m * m; e += kGenThreads) {
                const int i = e % m, c = e / m;
                double v;
                if (hasb && c == m - 1) v = bcol[off + i];   // column i1+r-1 = i2
                else v = __ldcg(B + AT(ldb, g.i1 + i, g.i1 + c));
                W[i * kLds + c] = v;
            }
            __syncthreads();
            const double tq = s_tau;
            if (tq != 0.0) {
                for (int c = warp; c < m; c += nwarps) {
                    const double w = lane < m ? W[lane * kLds + c] : 0.0;
                    const double d = warp_sum(w * vv[lane]) * tq;
                    if (lane < m) W[lane * kLds + c] = w - d * vv[lane];
                }
            }
            __syncthreads();
            for (int e = tid; e < m * m; e += kGenThreads) {
                const int i = e % m, c = e / m;
                B[AT(ldb, g.i1 + i, g.i1 + c)] = W[i * kLds + c];
                G[i * kLds + c] = (i == c) ? 1.0 : 0.0;
            }
            __syncthreads();

            // ---- RQ of the block, last row first: W G = R~, so the first row of Q~ is
            //      G(:, 1)^T
            for (int sr = m; sr >= 2; --sr) {
                if (warp == 0) {
                    // pivot W(sr, sr) goes to lane 0, W(sr, sr-1), ..., W(sr, 1) follow
                    const double x = lane < sr ? W[(sr - 1) * kLds + (sr - 1 - lane)] : 0.0;
                    double beta, vi;
                    const double tau = warp_larfg(x, sr, lane, &beta, &vi);
                    if (lane < sr) vv[sr - 1 - lane] = vi;
                    if (lane == 0) s_tau = tau;
                }
                __syncthreads();
                const double tr = s_tau;
                if (tr != 0.0) {
                    const int nrows = (sr - 1) + m;
                    const double vl = lane < sr ? vv[lane] : 0.0;
                    for (int row = warp; row < nrows; row += nwarps) {
                        double *Mrow = row < sr - 1 ? &W[row * kLds] : &G[(row - (sr - 1)) * kLds];
                        const double w = lane < sr ? Mrow[lane] : 0.0;
                        const double d = warp_sum(w * vl) * tr;
                        if (lane < sr) Mrow[lane] = w - d * vl;
                    }
                }
                __syncthreads();
            }

            // ---- opposite reflector Z^_k^j reducing the first row of Q~
            if (warp == 0) {
                const double x = lane < m ? G[lane * kLds] : 0.0;
                double beta, vi;
                const double tz = warp_larfg(x, m, lane, &beta, &vi);
                if (lane < r) VZs[(size_t)k * r + lane] = lane < m ? vi : 0.0;
                vv[lane] = lane < m ? vi : 0.0;
                if (lane == 0) {
                    TZs[k] = tz;
                    s_tau = tz;
                }
            }
            __syncthreads();

            // ---- band updates A(i4:i3, i1:i2) Z^ and B(i4:i2, i1:i2) Z^; the first column
            //      of the B block is reduced exactly
            const double tz = s_tau;
            const int na = imax(0, g.i3 - g.i4 + 1), nbr = imax(0, g.i2 - g.i4 + 1);
            for (int t = tid; t < na + nbr; t += kGenThreads) {
                const bool isA = t < na;
                const int x = g.i4 + (isA ? t : t - na);
                double *base = isA ? A : B;
                const int ld = isA ? lda : ldb;
                double rowv[kMaxR];
                double d = 0.0;
#pragma unroll
                for (int c = 0; c < kMaxR; ++c) {
                    if (c < m) {
                        rowv[c] = __ldcg(base + AT(ld, x, g.i1 + c));
                        d += rowv[c] * vv[c];
                    }
                }
                d *= tz;
#pragma unroll
                for (int c = 0; c < kMaxR; ++c) {
                    if (c < m) {
                        double val = rowv[c] - d * vv[c];
                        if (!isA && c == 0 && x > g.i1) val = 0.0;
                        base[AT(ld, x, g.i1 + c)] = val;
                    }
                }
            }
        }

        // ---- publish block k of this sweep
        __threadfence();
        __syncthreads();
        if (tid == 0 && !(a.stall && s == 0))
            st_release_u64(a.flags + s, a.epoch | (unsigned long long)(k + 1));
    }
}

// ---------------------------------------------------------------------------------------
// Delayed right updates (Alg. 4, first loop).  One thread per row; blockIdx.y selects the
// matrix.  kind 0 = A, 1 = B (Z^ reflectors, rows x < i4(k, j) only: the generate phase
// updated the rest), 2 = Z (Z^ reflectors, all rows), 3 = Q (Q^ reflectors, all rows).
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kApplyThreads) k_s2_apply_right(ApplyArgs a)
{
    extern __shared__ double sm[];
    const int NT = kApplyThreads;
    const int n = a.n, r = a.r, j1 = a.j1, qg = a.qg;
    const int w = r + qg - 1;
    double *buf = sm;                       // [w][NT]
    double *vr = buf + (size_t)w * NT;      // [qg][r]
    double *tr = vr + (size_t)qg * r;       // [qg]
    const int mi = blockIdx.y;
    const int kind = a.kind[mi];
    double *X = a.M[mi];
    const int ld = a.ld[mi];
    const int tid = threadIdx.x;
    const int x0 = blockIdx.x * NT + 1;
    const int x = x0 + tid;
    const bool rowok = x <= n;
    const int kmax = nblocks_gen(n, r, j1) - 1;
    const int kdim = a.R.kdim;
    const double *Vs = (kind == 3) ? a.R.VQ : a.R.VZ;
    const double *Ts = (kind == 3) ? a.R.TQ : a.R.TZ;

    if (__ldcg(a.status) != 0) return;
    int kstop = 0;
    if (kind <= 1) {
        // rows x0.. need block k only while x0 < i4(k, j1+qg-1) = j1 + 1 + max(0, (k-1) r)
        kstop = (x0 <= j1) ? 0 : (x0 - j1 - 1) / r + 2;
        if (kstop > kmax) return;
    }

    for (int k = kmax; k >= kstop; --k) {
        const int c0 = j1 + k * r + 1;
        __syncthreads();
        for (int e = tid; e < qg * r; e += NT) {
            const int sidx = e / r, i = e % r;
            vr[e] = Vs[((size_t)sidx * kdim + k) * r + i];
        }
        for (int e = tid; e < qg; e += NT) tr[e] = Ts[(size_t)e * kdim + k];
        __syncthreads();
        if (!rowok) continue;
        const int pnew = (k == kmax) ? w : r;
        for (int p = 0; p < pnew; ++p) {
            const int c = c0 + p;
            if (c <= n) buf[p * NT + tid] = X[AT(ld, x, c)];
        }
        for (int sidx = 0; sidx < qg; ++sidx) {
            const double tau = tr[sidx];
            if (tau == 0.0) continue;
            const int jj = j1 + sidx;
            if (kind <= 1 && !(x < j1 + 1 + imax(0, (k + jj - j1 - qg) * r))) continue;
            const int mlen = imin(r, n - (jj + k * r));
            const double *v = vr + sidx * r;
            double *b = buf + sidx * NT + tid;
            double d = 0.0;
            for (int i = 0; i < mlen; ++i) d += b[i * NT] * v[i];
            d *= tau;
            for (int i = 0; i < mlen; ++i) b[i * NT] -= d * v[i];
        }
        if (k > kstop) {
            for (int p = qg - 1; p < w; ++p) {
                const int c = c0 + p;
                if (c <= n) X[AT(ld, x, c)] = buf[p * NT + tid];
            }
            for (int p = 0; p <= qg - 2; ++p) buf[(p + r) * NT + tid] = buf[p * NT + tid];
        } else {
            for (int p = 0; p < w; ++p) {
                const int c = c0 + p;
                if (c <= n) X[AT(ld, x, c)] = buf[p * NT + tid];
            }
        }
    }
}

// ---------------------------------------------------------------------------------------
// Delayed left updates (Alg. 4, second loop).  One thread per column; blockIdx.y = 0 for A
// (columns c > jb(k, j1+qg-1)), 1 for B (columns c > i2(k, j1+qg-1)).  The columns up to
// those limits received the group's left reflectors during the generate phase.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ int left_cut(int isB, int n, int r, int jl, int k)
{
    return isB ? imin(jl + (k + 1) * r, n) : jl + imax(0, (k - 1) * r + 1);
}

__global__ void __launch_bounds__(kApplyThreads) k_s2_apply_left(LeftArgs a)
{
    extern __shared__ double sm[];
    const int NT = kApplyThreads;
    const int LDS = NT + 1;
    const int n = a.n, r = a.r, j1 = a.j1, qg = a.qg;
    const int w = r + qg - 1;
    const int jl = j1 + qg - 1;
    double *buf = sm;                       // [w][LDS], column cc of the tile at buf[p*LDS+cc]
    double *vr = buf + (size_t)w * LDS;     // [qg][r]
    double *tr = vr + (size_t)qg * r;       // [qg]
    const int isB = blockIdx.y;
    double *X = isB ? a.B : a.A;
    const int ld = isB ? a.ldb : a.lda;
    const int tid = threadIdx.x;
    const int cbase = blockIdx.x * NT + 1;
    const int c = cbase + tid;
    const int clast = imin(cbase + NT - 1, n);
    const int kdim = a.R.kdim;
    const int kmax = nblocks_gen(n, r, j1) - 1;

    if (__ldcg(a.status) != 0) return;
    int ktop = -1;
    for (int k = kmax; k >= 0; --k)
        if (left_cut(isB, n, r, jl, k) < clast) { ktop = k; break; }
    if (ktop < 0) return;

    for (int k = ktop; k >= 0; --k) {
        const int R0 = j1 + k * r + 1;
        __syncthreads();
        for (int e = tid; e < qg * r; e += NT) {
            const int sidx = e / r, i = e % r;
            vr[e] = a.R.VQ[((size_t)sidx * kdim + k) * r + i];
        }
        for (int e = tid; e < qg; e += NT) tr[e] = a.R.TQ[(size_t)e * kdim + k];
        const int pnew = (k == ktop) ? w : r;
        for (int e = tid; e < pnew * NT; e += NT) {
            const int p = e % pnew, cc = e / pnew;
            const int row = R0 + p, colx = cbase + cc;
            if (row <= n && colx <= n) buf[p * LDS + cc] = X[AT(ld, row, colx)];
        }
        __syncthreads();
        if (c <= n && c > left_cut(isB, n, r, jl, k)) {
            for (int sidx = 0; sidx < qg; ++sidx) {
                const double tau = tr[sidx];
                if (tau == 0.0) continue;
                const int mlen = imin(r, n - (j1 + sidx + k * r));
                const double *v = vr + sidx * r;
                double *b = buf + sidx * LDS + tid;
                double d = 0.0;
                for (int i = 0; i < mlen; ++i) d += b[i * LDS] * v[i];
                d *= tau;
                for (int i = 0; i < mlen; ++i) b[i * LDS] -= d * v[i];
            }
        }
        __syncthreads();
        const int plo = (k > 0) ? qg - 1 : 0;
        const int np = w - plo;
        for (int e = tid; e < np * NT; e += NT) {
            const int p = plo + e % np, cc = e / np;
            const int row = R0 + p, colx = cbase + cc;
            if (row <= n && colx <= n) X[AT(ld, row, colx)] = buf[p * LDS + cc];
        }
        __syncthreads();
        if (k > 0)
            for (int p = 0; p <= qg - 2; ++p) buf[(p + r) * LDS + tid] = buf[p * LDS + tid];
    }
}

// ---------------------------------------------------------------------------------------
// Utilities
// ---------------------------------------------------------------------------------------
__global__ void k_set_identity(double *M, int ld, int n)
{
    const int c = blockIdx.y + 1;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x + 1; i <= n; i += gridDim.x * blockDim.x)
        M[AT(ld, i, c)] = (i == c) ? 1.0 : 0.0;
}

// Zero A below its first subdiagonal (band = 1) or B below its diagonal (band = 0).
__global__ void k_zero_below(double *M, int ld, int n, int band)
{
    const int c = blockIdx.y + 1;
    for (int i = c + band + 1 + blockIdx.x * blockDim.x + threadIdx.x; i <= n; i += gridDim.x * blockDim.x)
        M[AT(ld, i, c)] = 0.0;
}

// ---------------------------------------------------------------------------------------
// Host-side launchers
// ---------------------------------------------------------------------------------------
cudaError_t launch_s2_generate(const GenArgs &a, cudaStream_t st)
{
    void *args[] = {(void *)&a};
    return cudaLaunchCooperativeKernel((const void *)k_s2_generate, dim3(a.qg), dim3(kGenThreads), args, 0, st);
}

size_t apply_right_smem(int r, int qg) { return sizeof(double) * ((size_t)(r + qg - 1) * kApplyThreads + (size_t)qg * r + qg); }
size_t apply_left_smem(int r, int qg) { return sizeof(double) * ((size_t)(r + qg - 1) * (kApplyThreads + 1) + (size_t)qg * r + qg); }

cudaError_t launch_s2_apply_right(const ApplyArgs &a, int nmat, cudaStream_t st)
{
    const size_t sm = apply_right_smem(a.r, a.qg);
    cudaError_t e = cudaFuncSetAttribute(k_s2_apply_right, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    dim3 grid((a.n + kApplyThreads - 1) / kApplyThreads, nmat);
    k_s2_apply_right<<<grid, kApplyThreads, sm, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_s2_apply_left(const LeftArgs &a, cudaStream_t st)
{
    const size_t sm = apply_left_smem(a.r, a.qg);
    cudaError_t e = cudaFuncSetAttribute(k_s2_apply_left, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    dim3 grid((a.n + kApplyThreads - 1) / kApplyThreads, 2);
    k_s2_apply_left<<<grid, kApplyThreads, sm, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_set_identity(double *M, int ld, int n, cudaStream_t st)
{
    dim3 grid((n + 255) / 256, n);
    k_set_identity<<<grid, 256, 0, st>>>(M, ld, n);
    return cudaGetLastError();
}

cudaError_t launch_zero_below(double *M, int ld, int n, int band, cudaStream_t st)
{
    if (n <= band + 1) return cudaSuccess;
    dim3 grid((n + 255) / 256, n);
    k_zero_below<<<grid, 256, 0, st>>>(M, ld, n, band);
    return cudaGetLastError();
}

}  // namespace hts
