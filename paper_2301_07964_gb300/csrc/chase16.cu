// Generate phase of stage 2 (Alg. 3) for r <= 16: the near-diagonal bulge chase of one group
// of qg sweeps, organised around the cost of FP64 on this GPU.
//
// An FP64 instruction occupies the FP64 unit of its SM sub-partition for about 64 cycles
// whether 1 or 32 lanes are active, and the four sub-partitions of an SM share little else.
// The chase is a chain of dependent steps, so its length is set by the FP64 instructions and
// warp collectives on that chain.  The block therefore splits roles by sub-partition (warp w
// runs on sub-partition w mod 4):
//   warp 0        the panel: every step of the sequential chain (reflector generation, the
//                 elimination's pivot steps with the update of the next row), lanes as columns;
//   warps 1 .. 3  bulk updates of the current reflector or elimination step;
//   warp 4        progress waits; while the elimination runs, the stores of the finished column
//                 segments and the loads of the next block's lazy data;
//   warps 5 .. 7  the band rows of A and B, held in registers (one thread per row), and three
//                 more bulk warps of the elimination.
//
// One step (k, j), sweep j waiting as in the general kernel (chase.cu) for block k+2 of sweep
// j-1 and block k+1 of its helper:
//   1. prefetch the pivot column segment, the block's newest B column, the earlier sweeps'
//      left reflectors of block k with their Gram entries, the B block and the band rows;
//   2. lazy left updates, aggregated: with w_b = tau_b u_b.x and g_ab = tau_b u_a.u_b (a < b,
//      the Gram entries, formed by the helper blocks as each reflector appears) the
//      coefficients of the sequential application are d_b = w_b - sum_{a<b} d_a g_ab, and
//      x -= sum_b d_b u_b (warp 1: pivot column, warp 2: B column);
//   3. left reflector Q^_k^j from the pivot column (panel) while the bulk warps form the
//      B block's column dots with it; then the block update;
//   4. the direction z of the opposite reflector: W z parallel to e_1 for the B block W, by
//      column elimination with partial pivoting, last row first, with look-ahead (the panel
//      takes step t to the next row and chooses step t+1 there while the bulk warps apply
//      step t to the other rows of W and to the accumulated column operations G).  Should the
//      residual check of step 5 fail, the step is repeated with the RQ of W, whose reflectors
//      are scaled, c (|u|^2 I - 2 u u^T) with c a power of two (a square root but no
//      division; the scaling leaves the direction of G's first column, the RQ's z, unchanged);
//   5. opposite reflector Z^_k^j from z (panel) while the band threads form their dots with z
//      (for the block rows below the first these are the entries Z^ zeroes, checked against
//      2^-44 max|W| max|z|); then the band update, with B(i1+1:i2, i1) = 0 exactly;
//   6. publish block k of sweep j.
// Reflectors are stored as (u, tau) with H = I - tau u u^T, u = x - beta e_1, tau = 2/|u|^2 and
// beta = -sign(x_1) |x| (the sign of LAPACK's dlarfg); tau = 0 is the identity.
#include "schedule.cuh"

namespace hts {

namespace {

constexpr int kM = 16;          // largest block
constexpr int kLD = kM + 1;     // leading dimension of the shared tiles
constexpr unsigned kFull = 0xffffffffu;

// Sum over the 16 lanes of each half-warp; every lane receives its half's sum.
__device__ __forceinline__ double sum16(double v)
{
    v += __shfl_xor_sync(kFull, v, 8);
    v += __shfl_xor_sync(kFull, v, 4);
    v += __shfl_xor_sync(kFull, v, 2);
    v += __shfl_xor_sync(kFull, v, 1);
    return v;
}

__device__ __forceinline__ bool is_zero(double v) { return (__double_as_longlong(v) << 1) == 0; }

// A sum of squares nxo and the pivot alpha far from over- and underflow; tested on the exponent
// bits.
__device__ __forceinline__ bool safe_sums(double nxo, double alpha)
{
    const int en = (__double2hiint(nxo) >> 20) & 0x7ff;
    const int ea = (__double2hiint(alpha) >> 20) & 0x7ff;
    return en > 60 && en < 1986 && ea < 1500;
}

// -sign(alpha) nrm, sign(0) = +1 (sign bit arithmetic).
__device__ __forceinline__ double neg_sign_of(double alpha, double nrm)
{
    const int sa = __double2hiint(alpha) & 0x80000000;
    return __hiloint2double(__double2hiint(nrm) ^ sa ^ 0x80000000, __double2loint(nrm));
}

// Householder vector of the panel lanes' x (lane c holds x_c, pivot at lane piv, entries
// beyond len zero).  Returns u_c in the calling lane, and beta, |u|^2; `esc` receives the
// power of two the vector was scaled by (x_used = x 2^-esc, 0 unless the sums were unsafe).
// ident: x has no entries below the pivot (the reflector is the identity).
__device__ __forceinline__ double panel_house(double x, int c, int piv, int len, double *beta, double *un2, int *esc,
                                              bool *ident)
{
    double sq = (c < len && c != piv) ? x : 0.0;
    double nxo = sum16(sq * sq);
    double alpha = __shfl_sync(kFull, x, piv);
    *esc = 0;
    if (is_zero(nxo)) {
        *ident = true;
        *beta = alpha;
        *un2 = 0.0;
        return 0.0;
    }
    *ident = false;
    if (!safe_sums(nxo, alpha)) {
        // rare: rescale by a power of two so that the largest entry is in [1, 2)
        double mx = (c < len) ? fabs(x) : 0.0;
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(kFull, mx, o));
        const int e = ilogb(mx);
        x = scalbn(x, -e);
        *esc = e;
        sq = (c < len && c != piv) ? x : 0.0;
        nxo = sum16(sq * sq);
        alpha = __shfl_sync(kFull, x, piv);
    }
    const double nx = fma(alpha, alpha, nxo);
    const double nrm = nx * rsqrt(nx);
    const double b = neg_sign_of(alpha, nrm);
    const double up = alpha - b;
    *beta = b;
    *un2 = fma(up, up, nxo);
    return (c == piv) ? up : ((c < len) ? x : 0.0);
}

// For a positive normal d = f 2^e with f in [1, 2): *s1 = f (d's significand, by bit
// arithmetic rather than a multiplication on the FP64 unit) and *s2 = 2^(1-e).
__device__ __forceinline__ void pow2_scale(double d, double *s1, double *s2)
{
    const int hi = __double2hiint(d), eb = (hi >> 20) & 0x7ff;
    *s1 = __hiloint2double((hi & 0x000fffff) | 0x3ff00000, __double2loint(d));
    *s2 = __hiloint2double((2047 - eb) << 20, 0);
}

__device__ __forceinline__ void named_barrier(int id, int nthreads)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// The left reflectors of block kk of sweeps j1 .. j1+ns-1, their taus and Gram entries into
// shared memory (threads t0, t0 + nt, ...).  Reflectors that do not exist read as zero.
__device__ __forceinline__ void load_lazy(const GenArgs &a, int kk, int ns, double *lv, double *lt, double *gr, int t0,
                                          int nt)
{
    const int n = a.n, r = a.r, j1 = a.j1, kdim = a.R.kdim, qm = a.qmax;
    for (int e = t0; e < ns * r; e += nt) {
        const int sh = e / r, i = e % r;
        lv[sh * kLD + i] = (kk < nblocks_gen(n, r, j1 + sh)) ? __ldcg(a.R.VQ + ((size_t)sh * kdim + kk) * r + i) : 0.0;
    }
    for (int e = t0; e < ns; e += nt)
        lt[e] = (kk < nblocks_gen(n, r, j1 + e)) ? __ldcg(a.R.TQ + (size_t)e * kdim + kk) : 0.0;
    for (int e = t0; e < ns * ns; e += nt) {
        const int ra = e / ns, rb = e % ns;
        gr[ra * kM + rb] = (ra < rb && kk < nblocks_gen(n, r, j1 + rb))
                               ? __ldcg(a.gram + ((size_t)kk * qm + ra) * qm + rb) : 0.0;
    }
}

// Index ranges of step (k, j) of the main block (see step_geom): pivot column segment
// rows rlo .. rhi (L of them), newest B column cb, block size m, and the band rows the main
// block updates: A rows x0 .. i3 (na), B rows x0 .. i1-1 above the block (nbt), then the
// block rows (nband in all; rows i4 .. cr-1 belong to the helper block).
struct StepInfo {
    StepGeom g;
    bool gen, hasb;
    int rlo, L, cb, m, x0, na, nbt, nband;
};

__device__ __forceinline__ StepInfo step_info(int n, int r, int j1, int qg, int kg, int k, int j)
{
    StepInfo I;
    I.g = step_geom(n, r, j1, qg, k, j);
    I.gen = k < kg;
    I.rlo = j1 + k * r + 1;
    I.L = imin(j + (k + 1) * r, n) - I.rlo + 1;
    I.cb = I.g.i1 + r - 1;
    I.hasb = I.cb <= n;
    I.m = I.g.i2 - I.g.i1 + 1;
    I.x0 = imax(I.g.i4, I.rlo);
    I.na = I.gen ? imax(0, I.g.i3 - I.x0 + 1) : 0;
    I.nbt = I.gen ? I.g.i1 - I.x0 : 0;
    I.nband = I.gen ? I.na + I.nbt + I.m : 0;
    return I;
}

// Bulk part of one RQ step: the rows of W above the next pivot row and all rows of G, three
// lanes per row, E elements per lane (E = ceil((piv + 1) / 3) covers the live columns).
template <int E>
__device__ __forceinline__ void rq_bulk(double *W, double *G, const double *hu, double s1, double sc2, int piv, int m,
                                        int bw, int lane)
{
    const int nrows = (piv - 1) + m;
    const int rho = bw * 10 + lane / 3, sub = lane % 3;
    const bool own = lane < 30 && rho < nrows;
    double *rowp = (rho < piv - 1) ? &W[rho * kLD] : &G[(rho - (piv - 1)) * kLD];
    double yv[E], uv[E];
    double p = 0.0;
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int cc = sub + 3 * e;
        const bool in = own && cc <= piv;
        yv[e] = in ? rowp[cc] : 0.0;
        uv[e] = in ? hu[cc] : 0.0;
        p = fma(yv[e], uv[e], p);
    }
    const int base = lane - sub;
    const double p1 = __shfl_sync(kFull, p, (base + 1) & 31);
    const double p2 = __shfl_sync(kFull, p, (base + 2) & 31);
    const double p0 = __shfl_sync(kFull, p, base & 31);
    const double cf = (p0 + p1 + p2) * sc2;
    if (own) {
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int cc = sub + 3 * e;
            if (cc <= piv) rowp[cc] = fma(-cf, uv[e], s1 * yv[e]);
        }
    }
}

// One step of the column elimination on the panel row x (lane c holds x_c, both half-warps
// the same).  Returns the pivot p, the active column of largest |x_c| (compared on the high
// word of the encoding, so within a factor 1 + 2^-20 of the largest), or -1 when the row
// vanishes on the active columns; sets a = x_p 2^-e (x_p's sign, |a| in [1, 2)) and
// b_c = x_c 2^-e, with 2^e the power of two of x_p (b_c = 0 for c = p, inactive columns and
// entries below 2^(e-1022), whose share is far below rounding).  Column c then becomes
// a col_c - b_c col_p, which clears x_c up to rounding with multipliers |b_c / a| <= 1 + 2^-19.
// No FP64 instruction: integer maximum, ballot and bit arithmetic.  *bad: x_p outside
// [2^-959, 2^960], where the growth of at most 4 per step could leave the exponent range.
__device__ __forceinline__ int elim_step(double x, unsigned act, int c, double *a, double *b, bool *bad)
{
    const bool on = (act >> c) & 1u;
    const int hx = __double2hiint(x);
    const unsigned key = on ? (unsigned)(hx & 0x7fffffff) : 0u;
    const unsigned kmax = __reduce_max_sync(kFull, key);
    *a = 1.0;
    *b = 0.0;
    *bad = false;
    if (kmax == 0u) return -1;
    const int p = __ffs(__ballot_sync(kFull, key == kmax) & 0xffffu) - 1;
    const int hp = __shfl_sync(kFull, hx, p), lp = __shfl_sync(kFull, __double2loint(x), p);
    const int ebp = (hp >> 20) & 0x7ff;
    *bad = ebp < 64 || ebp > 1983;
    *a = __hiloint2double((hp & 0x800fffff) | 0x3ff00000, lp);
    const int ebx = (hx >> 20) & 0x7ff, ebn = ebx - ebp + 1023;
    if (on && c != p && ebx != 0 && ebn >= 1)
        *b = __hiloint2double((hx & 0x800fffff) | (ebn << 20), __double2loint(x));
    return p;
}

// Bulk of one elimination step: column c of W rows 0 .. rho-2 and of the accumulated column
// operations G becomes a col_c - b_c col_p, for the active columns c != p (the set bits of cols).
// G's column c is zero outside the rows of the retired pivots and its diagonal, and every
// active column's diagonal is the same product D of the earlier steps' a, so only the G rows
// ret[0 .. ng-1] take part: the retired pivots in order, then p itself, whose diagonal D stands
// in for G(p, p).  W rows and G rows are at most m - 1 <= 15: lane i of each half-warp takes
// row i, the two half-warps the two columns of a pair, warp bw of the six bulk warps every
// sixth pair.
__device__ __forceinline__ void elim_bulk(double *W, double *G, const double *b, double a, double D, int p,
                                          unsigned cols, const int *ret, int ng, int rho, int bw, int lane)
{
    const int i = lane & 15, h = lane >> 4, nw = rho - 1;
    const bool own = i < nw + ng;
    double *rowp = (i < nw) ? &W[i * kLD] : &G[(own ? ret[i - nw] : 0) * kLD];
    const double vp = own ? ((i == nw + ng - 1) ? D : rowp[p]) : 0.0;
    const int nc = __popc(cols);
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const int k = 2 * (bw + 6 * e) + h;
        if (own && k < nc) {
            const int cc = (int)__fns(cols, 0u, k + 1);   // the k-th active column (0-based k)
            rowp[cc] = fma(-b[cc], vp, a * rowp[cc]);
        }
    }
}

}  // namespace

__global__ void __launch_bounds__(kGenThreads, 1) k_s2_chase16(GenArgs a)
{
    __shared__ double col[2 * kMaxR];      // pivot column segment
    __shared__ double bcol[2 * kMaxR];     // newest B column segment
    __shared__ double W[kM * kLD];         // B block (row-major), then the elimination's (or RQ's) work array
    __shared__ double Wq[kM * kLD];        // B block after Q^ (band rows i1 .. i2 of B)
    __shared__ double G[kM * kLD];         // accumulated column operations (or the RQ's right factor)
    __shared__ double lvb[2][kM * kLD];    // earlier sweeps' left reflectors of block k (buffer k & 1)
    __shared__ double ltb[2][kM];
    __shared__ double grb[2][kM * kM];     // their Gram entries tau_b u_a.u_b, a < b
    __shared__ double hu[2][kM];           // RQ reflector vectors (double buffered)
    __shared__ double hs[2][2];            // RQ scale factors {s1, sc2}; s1 = 0: identity
    __shared__ double pu[kM];              // current Q^ / Z^ vector
    __shared__ double ps[2];               // {tau applied to the unscaled data, beta}
    __shared__ double vv[kM];              // helper block: current reflector
    __shared__ double eb[2][kM];           // elimination steps: multipliers b (double buffered)
    __shared__ double2 eaD[2];             // ... {a, the product D of the earlier steps' a}
    __shared__ int4 epc[2];                // ... {pivot column (-1: the row vanished), the other
                                           //     active columns as a bit mask, G rows taking part}
    __shared__ int eret[kM];               // pivots in the order they were chosen
    __shared__ double zv[kM];              // z, the direction of the opposite reflector
    __shared__ int s_ew[2];                // biased exponent of max |W| (the B block after Q^)
    __shared__ int s_ez;                   // biased exponent of max |z|
    __shared__ int s_redo;                 // the elimination failed its checks: use the RQ
    __shared__ int s_abort;

    const bool helper = (int)blockIdx.x >= a.qg;
    const int s = helper ? (int)blockIdx.x - a.qg : (int)blockIdx.x;
    const int j = a.j1 + s;
    const int n = a.n, r = a.r, j1 = a.j1, qg = a.qg;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
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
    const int qm = a.qmax;

    for (int k = kg + tid; !helper && k < kdim; k += kGenThreads) {   // blocks this sweep does not reach
        TQs[k] = 0.0;
        TZs[k] = 0.0;
    }
    if (tid == 0) {
        s_abort = __ldcg(a.status) != 0;   // an earlier kernel of this call failed
        s_redo = 0;
    }
    __syncthreads();
    if (s_abort) return;
    unsigned long long *hflags = a.flags + a.qmax;       // progress of the helper blocks

    if (helper) {
        // Rows i4 .. cr-1 of each step's band (cr = j1+kr+1, the first row any later step of
        // the group reads), and the Gram entries of this sweep's left reflector of block k
        // with the earlier sweeps' ones, which the later sweeps' lazy updates use.
        for (int k = 0; k < kg; ++k) {
            if (tid == 0) {
                const bool ok =
                    wait_at_least(a.flags + s, a.epoch | (unsigned long long)(k + 1), a.status, a.group, k, j) &&
                    (s == 0 ||
                     wait_at_least(hflags + s - 1, a.epoch | (unsigned long long)(k + 2), a.status, a.group, k, j));
                s_abort = !ok;
            }
            __syncthreads();
            if (s_abort) return;
            const StepGeom g = step_geom(n, r, j1, qg, k, j);
            const int m = g.i2 - g.i1 + 1;
            const int cr = j1 + k * r + 1;
            const double tz = __ldcg(TZs + k);
            if (tid < kM) vv[tid] = tid < m ? __ldcg(VZs + (size_t)k * r + tid) : 0.0;
            // Gram column s of block k: tau_s u_a . u_s for the earlier sweeps a < s
            if (warp == 7 && lane < s) {
                const double tq = __ldcg(TQs + k);
                const int ra = lane;
                const int ma = imin(r, n - (j1 + ra + k * r)), ms = imin(r, n - (j + k * r));
                const double *ua = a.R.VQ + ((size_t)ra * kdim + k) * r;   // rows ra .. of the segment
                const double *us = VQs + (size_t)k * r;                      // rows s ..
                double d0 = 0.0, d1 = 0.0;
                const int hi = imin(ra + ma, s + ms);
                for (int i = s; i < hi; i += 2) {
                    d0 = fma(__ldcg(ua + i - ra), __ldcg(us + i - s), d0);
                    if (i + 1 < hi) d1 = fma(__ldcg(ua + i + 1 - ra), __ldcg(us + i + 1 - s), d1);
                }
                a.gram[((size_t)k * qm + ra) * qm + s] = tq * (d0 + d1);
            }
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

    const int c = lane & 15;   // panel lanes: column index (both half-warps hold the same data)
    double brow[kM];           // band threads: their row

    const int bt = tid - 160;   // band thread index (warps 5 .. 7)
    // Global loads of a step's pivot column segment, B column, B block and band rows, into
    // registers (the band rows straight into brow); committed to shared memory later.
    double pc = 0.0, pb = 0.0, pw = 0.0;
    auto issue_loads = [&](const StepInfo &I) {
        if (tid < I.L) {
            pc = __ldcg(A + AT(lda, I.rlo + tid, I.g.jb));
            if (I.hasb) pb = __ldcg(B + AT(ldb, I.rlo + tid, I.cb));
        }
        if (I.gen && tid < I.m * I.m) {
            const int i = tid % I.m, cc = tid / I.m;
            if (!(I.hasb && cc == I.m - 1)) pw = __ldcg(B + AT(ldb, I.g.i1 + i, I.g.i1 + cc));
        }
        if (bt >= 0 && bt < I.na + I.nbt) {
            const bool isA = bt < I.na;
            const int x = I.x0 + (isA ? bt : bt - I.na);
            const double *src = isA ? A + AT(lda, x, I.g.i1) : B + AT(ldb, x, I.g.i1);
            const size_t ld = isA ? (size_t)lda : (size_t)ldb;
#pragma unroll
            for (int cc = 0; cc < kM; ++cc) brow[cc] = (cc < I.m) ? __ldcg(src + cc * ld) : 0.0;
        }
    };
    auto commit_loads = [&](const StepInfo &I) {
        if (tid < I.L) {
            col[tid] = pc;
            if (I.hasb) bcol[tid] = pb;
        }
        if (I.gen && tid < I.m * I.m) {
            const int i = tid % I.m, cc = tid / I.m;
            if (!(I.hasb && cc == I.m - 1)) W[i * kLD + cc] = pw;
            G[i * kLD + cc] = (i == cc) ? 1.0 : 0.0;
        }
    };
    // step k waits until sweep j-1 has finished block k+2 (or all of its blocks) and its helper
    // block k+1 (whose rows of block k+1 hold the upper rows of step k's B column)
    auto wait_deps = [&](int k) -> bool {
        return wait_at_least(a.flags + s - 1, a.epoch | (unsigned long long)imin(k + 3, kl_prev), a.status, a.group,
                             k, j) &&
               wait_at_least(hflags + s - 1, a.epoch | (unsigned long long)(k + 2), a.status, a.group, k, j);
    };

    // the previous group's update tiles this sweep's steps touch (look-ahead): thread 128
    // checks them step by step before the step's loads
    __shared__ UpdWait uw;   // thread 128's progress through those tiles
    if (tid == 128) uw.init(a.uflags, a.uplan, a.uepoch, n);
    auto wait_upd = [&](int k) -> bool {
        const StepGeom gk = step_geom(n, r, j1, qg, k, j);
        return uw.wait_for(gk.i2, gk.i3, a.status, a.group, k, j);
    };

    // step 0's dependencies and data
    if (tid == 128) s_abort = !(wait_upd(0) && (s == 0 || wait_deps(0)));
    __syncthreads();
    if (s_abort) return;
    StepInfo I = step_info(n, r, j1, qg, kg, 0, j);
    issue_loads(I);
    commit_loads(I);
    load_lazy(a, 0, nlazy, lvb[0], ltb[0], grb[0], tid, kGenThreads);
    __syncthreads();

    for (int k = 0; k < kl; ++k) {
        const StepGeom g = I.g;
        const bool gen = I.gen;
        const int rlo = I.rlo;
        const int L = I.L;
        const int cb = I.cb;
        const bool hasb = I.hasb;
        const int m = I.m;
        const int off = j - j1;
        const int x0 = I.x0, na = I.na, nbt = I.nbt, nband = I.nband;
        double *lv = lvb[k & 1], *lt = ltb[k & 1], *gr = grb[k & 1];

        // ---- 2. lazy left updates (warp 1: pivot column, warp 2: B column)
        if (nlazy > 0 && L > 0 && (warp == 1 || (warp == 2 && hasb))) {
            double *seg = (warp == 1) ? col : bcol;
            const int ns = nlazy;
            // lanes 2b and 2b+1 form w_b, each over every other entry of reflector b
            const int lb = lane >> 1, part = lane & 1;
            double wv = 0.0;
            if (lb < ns) {
                const int mb = imin(r, n - (j1 + lb + k * r));
                const double *ub = lv + lb * kLD;
                const double *xs = seg + lb;
                double d0 = 0.0, d1 = 0.0;
                for (int i = part; i < mb; i += 4) {
                    d0 = fma(ub[i], xs[i], d0);
                    if (i + 2 < mb) d1 = fma(ub[i + 2], xs[i + 2], d1);
                }
                wv = d0 + d1;
            }
            wv += __shfl_xor_sync(kFull, wv, 1);
            if (lb < ns) wv *= lt[lb];
            for (int ra = 0; ra + 1 < ns; ++ra) {
                const double da = __shfl_sync(kFull, wv, 2 * ra);
                if (lb > ra && lb < ns) wv = fma(-da, gr[ra * kM + lb], wv);
            }
            // lanes 2b, 2b+1 hold d_b; lane i: x_i -= sum_b d_b u_b(i - b)  (L <= 31)
            double e0 = 0.0, e1 = 0.0;
            for (int rb = 0; rb < ns; ++rb) {
                const double db = __shfl_sync(kFull, wv, 2 * rb);
                const int mb = imin(r, n - (j1 + rb + k * r));
                const int i0 = lane - rb;
                const double u = (i0 >= 0 && i0 < mb) ? lv[rb * kLD + i0] : 0.0;
                if (rb & 1) e1 = fma(db, u, e1);
                else e0 = fma(db, u, e0);
            }
            if (lane < L) seg[lane] -= e0 + e1;
        }
        __syncthreads();

        if (gen) {
            // ---- 3. left reflector Q^ from col[off .. off+m-1] (panel); column dots (warps 1, 2)
            double pdot = 0.0, y[4], y0 = 0.0;
            const int qcol = (warp - 1) * 8 + (lane >> 2), qsub = lane & 3;   // warps 1, 2: column, row set
            const bool qown = (warp == 1 || warp == 2) && qcol < m;
            const bool qfromb = hasb && qcol == m - 1;
            if (warp == 0) {
                const double x = (c < m) ? col[off + c] : 0.0;
                double beta, un2;
                int esc;
                bool ident;
                const double u = panel_house(x, c, 0, m, &beta, &un2, &esc, &ident);
                const double tau = ident ? 0.0 : 2.0 * __drcp_rn(un2);
                if (lane < kM) pu[lane] = u;
                if (lane == 0) {
                    ps[0] = ident ? 0.0 : (esc ? scalbn(tau, -esc) : tau);
                    ps[1] = ident ? beta : (esc ? scalbn(beta, esc) : beta);
                    TQs[k] = tau;
                }
                if (lane < r) VQs[(size_t)k * r + lane] = (!ident && lane < m) ? u : 0.0;
            } else if (warp == 1 || warp == 2) {
                // every lane of both warps takes part in the shuffles; lanes without a column
                // contribute zeros
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int i = qsub + 4 * e;
                    y[e] = (qown && i < m) ? (qfromb ? bcol[off + i] : W[i * kLD + qcol]) : 0.0;
                    if (qown && i < m) pdot = fma(y[e], col[off + i], pdot);
                }
                pdot += __shfl_xor_sync(kFull, pdot, 1);
                pdot += __shfl_xor_sync(kFull, pdot, 2);
                if (qown) y0 = qfromb ? bcol[off] : W[qcol];   // read before any lane rewrites row 0
            }
            __syncthreads();
            unsigned wkey = 0u;
            if (qown) {
                const double tau = ps[0], beta = ps[1];
                const double cf = tau != 0.0 ? fma(-beta, y0, pdot) * tau : 0.0;
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int i = qsub + 4 * e;
                    if (i < m) {
                        const double v = fma(-cf, pu[i], y[e]);
                        W[i * kLD + qcol] = v;
                        Wq[i * kLD + qcol] = v;
                        const unsigned vk = (unsigned)(__double2hiint(v) & 0x7fffffff);
                        wkey = vk > wkey ? vk : wkey;
                    }
                }
            }
            if (warp == 1 || warp == 2) {
                wkey = __reduce_max_sync(kFull, wkey);
                if (lane == 0) s_ew[warp - 1] = (int)(wkey >> 20);
            }
            if (warp == 0 && ps[0] != 0.0 && lane < m) col[off + lane] = (lane == 0) ? ps[1] : 0.0;
            __syncthreads();
        }

        // pivot and B column segments are final (the B column's block rows are rewritten with
        // the band); warp 4 stores them while the elimination runs
        if (warp == 4) {
            for (int i = lane; i < L; i += 32) {
                A[AT(lda, rlo + i, g.jb)] = col[i];
                if (hasb) B[AT(ldb, rlo + i, cb)] = bcol[i];
            }
            // the earlier sweeps' data of block k+1 is final: sweep j-1 has finished block k+2
            // and its helper block k+1 (the waits of this step)
            if (k + 1 < kl) load_lazy(a, k + 1, nlazy, lvb[(k + 1) & 1], ltb[(k + 1) & 1], grb[(k + 1) & 1], lane, 32);
        }

        // ---- 4. the direction z of the opposite reflector, W z = lambda e_1 (warps 0 .. 3, 5 .. 7), and
        // ---- 5. Z^ from z with the band update.  Attempt 0 finds z by column elimination with
        //      partial pivoting (W M upper triangular up to a column order; z is the column of M
        //      that no step retired): its chain per row is an integer pivot search and one
        //      multiply-add, where each RQ reflector needs a reduction and a square root.  The
        //      band dots of the block rows below the first are the entries Z^ zeroes, (W z)_i;
        //      if one exceeds 2^-44 max|W| max|z|, or a pivot leaves the safe exponent range,
        //      nothing is written and attempt 1 takes z from the RQ of W (Alg. 3's opposite
        //      reflector: the first column of the RQ's accumulated right factor).
        for (int attempt = 0; attempt < 2; ++attempt) {
            if (attempt == 1) {
                for (int e = tid; e < m * m; e += kGenThreads) {
                    const int i = e / m, cc = e % m;
                    W[i * kLD + cc] = Wq[i * kLD + cc];
                    G[i * kLD + cc] = (i == cc) ? 1.0 : 0.0;
                }
                __syncthreads();
                if (tid == 0) s_redo = 0;
            }
            if (tid == 0 && m < 2) zv[0] = 1.0;   // a 1 x 1 block: z = e_1
            const bool elim = !a.direct_rq;
            if (attempt == 0 && !elim && gen && m >= 2 && tid == 0) s_redo = 1;   // tests: RQ only
            if (gen && m >= 2 && (attempt == 0 ? (elim && warp != 4) : warp < 4)) {
                if (attempt == 0) {
                    unsigned act = (1u << m) - 1u;   // panel: active columns, current step
                    int p = -1, nret = 0;
                    double a = 1.0, b = 0.0, D = 1.0;
                    bool bad = false;
                    // publish step (p, a, b) into slot sl: multipliers, the product D of the
                    // earlier steps' a, the list of the other active columns, the pivot order
                    auto publish = [&](int sl) {
                        if (lane < kM) eb[sl][lane] = b;
                        if (lane == 0) {
                            // two 16-byte stores carry the step; the bulk finds its columns in the mask
                            eaD[sl] = make_double2(a, D);
                            epc[sl] = make_int4(p, p >= 0 ? (int)(act & ~(1u << p)) : 0, nret + 1, 0);
                            if (p >= 0) eret[nret] = p;
                            if (bad) s_redo = 1;
                        }
                        if (p >= 0) {
                            ++nret;
                            D *= a;
                        }
                    };
                    if (warp == 0) {
                        const double x = (c < m) ? W[(m - 1) * kLD + c] : 0.0;
                        p = elim_step(x, act, c, &a, &b, &bad);
                        publish(0);
                    }
                    named_barrier(4, 224);
                    for (int t = 0; t + 1 < m; ++t) {
                        const int rho = m - 1 - t, cur = t & 1;
                        if (warp == 0) {
                            if (rho >= 2) {
                                // row rho-1 under step t (look-ahead), then step t+1 on it
                                double y = (c < m) ? W[(rho - 1) * kLD + c] : 0.0;
                                if (p >= 0) {
                                    const double yn = fma(-b, __shfl_sync(kFull, y, p), a * y);
                                    if (((act >> c) & 1u) && c != p) y = yn;
                                    act &= ~(1u << p);
                                }
                                p = elim_step(y, act, c, &a, &b, &bad);
                                publish(cur ^ 1);
                            }
                        } else {
                            // bulk (warps 1 .. 3, 5 .. 7): step t on W rows 0 .. rho-2 and on G
                            const int4 st = epc[cur];
                            if (st.x >= 0) {
                                const double2 ad = eaD[cur];
                                elim_bulk(W, G, eb[cur], ad.x, ad.y, st.x, (unsigned)st.y, eret, st.z, rho,
                                          warp < 4 ? warp - 1 : warp - 2, lane);
                            }
                        }
                        named_barrier(4, 224);
                    }
                    if (warp == 0) {
                        // z is the one column no step retired (the lowest, if rows vanished); its
                        // diagonal is the product of all steps' a
                        const unsigned fin = (p >= 0 && m >= 2) ? act & ~(1u << p) : act;
                        const int cs = __ffs(fin) - 1;
                        if (lane < kM) zv[lane] = (lane < m) ? ((lane == cs) ? D : G[lane * kLD + cs]) : 0.0;
                    }
                } else {
                    // RQ of the B block with look-ahead
                    double u = 0.0, s1 = 0.0, sc2 = 0.0;   // panel: current reflector
                    if (warp == 0) {
                        const int piv = m - 1;
                        const double x = (c <= piv) ? W[piv * kLD + c] : 0.0;
                        double beta, un2;
                        int esc;
                        bool ident;
                        u = panel_house(x, c, piv, piv + 1, &beta, &un2, &esc, &ident);
                        if (!ident) pow2_scale(un2, &s1, &sc2);
                        if (lane < kM) hu[0][lane] = u;
                        if (lane == 0) {
                            hs[0][0] = s1;
                            hs[0][1] = sc2;
                        }
                    }
                    named_barrier(1, 128);
                    for (int t = 0; t + 1 < m; ++t) {
                        const int piv = m - 1 - t, cur = t & 1;
                        if (warp == 0) {
                            if (piv >= 2) {
                                // next pivot row y (columns 0 .. piv): apply reflector t, then form
                                // reflector t+1 from y'(0 .. piv-1).  The scaled reflector multiplies
                                // norms by s1 and leaves y'_piv final, so |y'(0 .. piv-1)|^2 =
                                // s1^2 |y|^2 - y'_piv^2: the upper half-warp sums |y|^2 in the same
                                // instructions that sum u.y in the lower half, which takes the second
                                // reduction off the chain.  Where that difference loses more than two bits
                                // to cancellation, or the sums approach over- or underflow, the reflector
                                // is formed from y' directly.  The part below the pivot, nx - alpha^2,
                                // only enters |u|^2 >= nx, so its absolute error (a few ulps of nx)
                                // perturbs the reflector by a few ulps relative to the entries it
                                // annihilates.  When those entries are zero the reflector changes the sign
                                // of the pivot coordinate only; G's zeros stay exact and the direction of
                                // G(:, 1), all that the RQ is used for, keeps its value up to sign.
                                const bool hi = lane >= 16;
                                const double a1 = (s1 != 0.0) ? s1 : 1.0, a2 = (s1 != 0.0) ? sc2 : 0.0;
                                double y = (c <= piv) ? W[(piv - 1) * kLD + c] : 0.0;
                                const double h = sum16(y * (hi ? y : u)) * (hi ? a1 * a1 : a2);
                                const double hx = __shfl_xor_sync(kFull, h, 16);
                                y = fma(-(hi ? hx : h), u, a1 * y);
                                const double S = hi ? h : hx;
                                const double ypiv = __shfl_sync(kFull, y, piv);
                                const double alpha = __shfl_sync(kFull, y, piv - 1);
                                const double nx = fma(-ypiv, ypiv, S), nxo = fma(-alpha, alpha, nx);
                                double beta, un2;
                                int esc;
                                bool ident;
                                if (safe_sums(nx, alpha) &&
                                    __double_as_longlong(nx) >= __double_as_longlong(S) - (2ll << 52)) {
                                    const double nrm = nx * rsqrt(nx);
                                    const double up = alpha - neg_sign_of(alpha, nrm);
                                    un2 = fma(up, up, nxo);
                                    u = (c == piv - 1) ? up : ((c < piv) ? y : 0.0);
                                    ident = false;
                                } else {
                                    u = panel_house(y, c, piv - 1, piv, &beta, &un2, &esc, &ident);
                                }
                                s1 = 0.0;
                                if (!ident) pow2_scale(un2, &s1, &sc2);
                                if (lane < kM) hu[cur ^ 1][lane] = u;
                                if (lane == 0) {
                                    hs[cur ^ 1][0] = s1;
                                    hs[cur ^ 1][1] = sc2;
                                }
                            }
                        } else {
                            // bulk: W rows 0 .. piv-2 and G rows 0 .. m-1, three lanes per row, only the
                            // live columns 0 .. piv; a warp without rows skips the step
                            const double bs1 = hs[cur][0];
                            const int bw = warp - 1;
                            if (bs1 != 0.0 && bw * 10 < (piv - 1) + m) {
                                const double bsc2 = hs[cur][1];
                                switch ((piv + 3) / 3) {
                                case 6: rq_bulk<6>(W, G, hu[cur], bs1, bsc2, piv, m, bw, lane); break;
                                case 5: rq_bulk<5>(W, G, hu[cur], bs1, bsc2, piv, m, bw, lane); break;
                                case 4: rq_bulk<4>(W, G, hu[cur], bs1, bsc2, piv, m, bw, lane); break;
                                case 3: rq_bulk<3>(W, G, hu[cur], bs1, bsc2, piv, m, bw, lane); break;
                                case 2: rq_bulk<2>(W, G, hu[cur], bs1, bsc2, piv, m, bw, lane); break;
                                default: rq_bulk<1>(W, G, hu[cur], bs1, bsc2, piv, m, bw, lane); break;
                                }
                            }
                        }
                        named_barrier(1, 128);
                    }
                    if (warp == 0 && lane < kM) zv[lane] = (lane < m) ? G[lane * kLD] : 0.0;
                }
            }
            __syncthreads();

            // warp 4 takes the next step's dependencies while Z^ and the band update run
            if (attempt == 0 && tid == 128 && k + 1 < kl) s_abort = !(wait_upd(k + 1) && (s == 0 || wait_deps(k + 1)));

            if (gen) {
                // ---- 5. opposite reflector Z^ from z (panel); band dots (warps 5 .. 7)
                double p = 0.0;
                const bool band = bt >= 0 && bt < nband;
                const bool isA = bt < na;
                const int xrow = isA ? x0 + bt : x0 + (bt - na);
                if (warp == 0) {
                    const double x = (c < m) ? zv[c] : 0.0;
                    double beta, un2;
                    int esc;
                    bool ident;
                    const double u = panel_house(x, c, 0, m, &beta, &un2, &esc, &ident);
                    const double tau = ident ? 0.0 : 2.0 * __drcp_rn(un2);
                    if (lane < kM) pu[lane] = u;
                    if (lane == 0) {
                        ps[0] = ident ? 0.0 : (esc ? scalbn(tau, -esc) : tau);
                        ps[1] = ident ? beta : (esc ? scalbn(beta, esc) : beta);
                        TZs[k] = tau;
                    }
                    if (lane < r) VZs[(size_t)k * r + lane] = (!ident && lane < m) ? u : 0.0;
                    if (attempt == 0) {
                        const unsigned zk = __reduce_max_sync(kFull, (unsigned)(__double2hiint(x) & 0x7fffffff));
                        if (lane == 0) s_ez = (int)(zk >> 20);
                    }
                } else if (band) {
                    if (bt >= na + nbt) {
                        const int bi = bt - na - nbt;
#pragma unroll
                        for (int cc = 0; cc < kM; ++cc) brow[cc] = (cc < m) ? Wq[bi * kLD + cc] : 0.0;
                    } else if (!isA && hasb) {
                        // the B column cb above the block carries the lazy updates of step 2
                        const double v = bcol[xrow - rlo];
#pragma unroll
                        for (int cc = 0; cc < kM; ++cc)
                            if (cc == m - 1) brow[cc] = v;
                    }
                    double p0 = 0.0, p1 = 0.0;
#pragma unroll
                    for (int cc = 0; cc < kM; cc += 2) {
                        if (cc < m) p0 = fma(brow[cc], zv[cc], p0);
                        if (cc + 1 < m) p1 = fma(brow[cc + 1], zv[cc + 1], p1);
                    }
                    p = p0 + p1;
                }
                if (warp == 0 || warp >= 5) named_barrier(2, 128);
                if (attempt == 0 && warp >= 5) {
                    // the entries the reflector zeroes, (W z)_i / |z|, for the block rows below the first
                    if (band && !isA && xrow > g.i1 && !is_zero(p)) {
                        const int epx = (__double2hiint(p) >> 20) & 0x7ff;
                        if (epx > imax(s_ew[0], s_ew[1]) + s_ez - 1068) s_redo = 1;
                    }
                    named_barrier(3, 96);
                }
                if (band && (attempt == 1 || !s_redo)) {
                    const double tau = ps[0], beta = ps[1];
                    if (tau != 0.0) {
                        const double cf = fma(-beta, brow[0], p) * tau;
#pragma unroll
                        for (int cc = 0; cc < kM; ++cc) brow[cc] = fma(-cf, pu[cc], brow[cc]);
                    }
                    if (!isA && xrow > g.i1) brow[0] = 0.0;   // the reduced column of the B block
                    double *dst = isA ? A + AT(lda, xrow, g.i1) : B + AT(ldb, xrow, g.i1);
                    const size_t ld = isA ? (size_t)lda : (size_t)ldb;
#pragma unroll
                    for (int cc = 0; cc < kM; ++cc)
                        if (cc < m) dst[cc * ld] = brow[cc];
                }
            }
            __syncthreads();
            // count the steps whose elimination failed its checks (status word slot 5)
            if (attempt == 0 && s_redo && !a.direct_rq && tid == 0) atomicAdd(a.status + kStatusFallbacks, 1);
            if (!s_redo) break;
        }

        // ---- 6. publish block k of this sweep; the next step's global loads (its dependencies
        //      were acquired by warp 4 above, and this step's band stores are ordered before
        //      them by the barrier above) are in flight while the stores of this step are fenced
        const bool more = k + 1 < kl && !s_abort;
        StepInfo In = I;
        if (more) {
            In = step_info(n, r, j1, qg, kg, k + 1, j);
            issue_loads(In);
        }
        __threadfence();
        __syncthreads();
        if (tid == 0 && !(a.stall && s == 0))
            st_release_u64(a.flags + s, a.epoch | (unsigned long long)(k + 1));
        if (s_abort) return;
        if (more) {
            commit_loads(In);
            I = In;
            __syncthreads();
        }
    }
}

cudaError_t launch_s2_chase16(const GenArgs &a, cudaStream_t st)
{
    void *args[] = {(void *)&a};
    return cudaLaunchCooperativeKernel((const void *)k_s2_chase16, dim3(2 * a.qg), dim3(kGenThreads), args, 0, st);
}

}  // namespace hts
