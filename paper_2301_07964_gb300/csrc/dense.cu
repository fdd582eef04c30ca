// Dense FP64 building blocks of stages 0 and 1 (QR of B, Alg. 1): Householder QR of a panel,
// the triangular factor of a block reflector (forward, columnwise), and the RQ + LQ
// factorisation of one B block that yields the opposite reflectors of Alg. 1.  The block
// reflectors' products with the matrices are plain GEMMs, done by cuBLAS (stage01.cu).
//
// Block reflectors are used in compact WY form: H_1 H_2 ... H_b = I - V T V^T with V unit
// lower trapezoidal (explicit ones and zeros) and T upper triangular (both dense buffers).
#include "hts_internal.cuh"

namespace hts {

// ---------------------------------------------------------------------------------------
// Householder QR of the m x b panel P (column-major, ld) in one thread block (dlarfg
// convention).  On exit the upper triangle of P holds R; V (m x b, ldv) receives the unit
// lower trapezoidal reflector vectors and tau[0..b) the factors; the entries of P below the
// diagonal are set to zero.
// ---------------------------------------------------------------------------------------
constexpr int kPanelThreads = 256;

__device__ double block_sum(double v, double *red)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    return s;
}

__global__ void __launch_bounds__(kPanelThreads) k_panel_qr(int m, int b, double *P, int ld, double *V, int ldv,
                                                             double *tau)
{
    __shared__ double red[32];
    __shared__ double s_beta, s_tau, s_scale;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nw = kPanelThreads / 32;
    for (int c = 0; c < b && c < m; ++c) {
        // reflector from P(c:m, c)
        double part = 0.0;
        for (int i = c + 1 + tid; i < m; i += kPanelThreads) {
            const double x = P[(size_t)i + (size_t)c * ld];
            part += x * x;
        }
        const double ssq = block_sum(part, red);
        if (tid == 0) {
            const double alpha = P[(size_t)c + (size_t)c * ld];
            if (ssq == 0.0) {
                s_tau = 0.0;
                s_beta = alpha;
                s_scale = 0.0;
            } else {
                const double nrm = sqrt(alpha * alpha + ssq);
                const double beta = (alpha >= 0.0) ? -nrm : nrm;
                s_tau = (beta - alpha) / beta;
                s_scale = 1.0 / (alpha - beta);
                s_beta = beta;
            }
            tau[c] = s_tau;
        }
        __syncthreads();
        const double tc = s_tau, sc = s_scale;
        for (int i = tid; i < m; i += kPanelThreads) {
            double vi;
            if (i < c) vi = 0.0;
            else if (i == c) vi = 1.0;
            else vi = P[(size_t)i + (size_t)c * ld] * sc;
            if (tc == 0.0 && i > c) vi = 0.0;
            V[(size_t)i + (size_t)c * ldv] = vi;
        }
        __syncthreads();
        if (tid == 0) P[(size_t)c + (size_t)c * ld] = s_beta;
        for (int i = c + 1 + tid; i < m; i += kPanelThreads) P[(size_t)i + (size_t)c * ld] = 0.0;
        // apply to the remaining panel columns (one warp per column)
        if (tc != 0.0) {
            for (int cc = c + 1 + warp; cc < b; cc += nw) {
                double d = 0.0;
                for (int i = c + lane; i < m; i += 32) d += V[(size_t)i + (size_t)c * ldv] * P[(size_t)i + (size_t)cc * ld];
                d = warp_sum(d) * tc;
                for (int i = c + lane; i < m; i += 32) P[(size_t)i + (size_t)cc * ld] -= d * V[(size_t)i + (size_t)c * ldv];
            }
        }
        __syncthreads();
    }
    for (int c = m; c < b; ++c) {   // more columns than rows: nothing left to reduce
        if (tid == 0) tau[c] = 0.0;
        for (int i = tid; i < m; i += kPanelThreads) V[(size_t)i + (size_t)c * ldv] = 0.0;
    }
}

// ---------------------------------------------------------------------------------------
// T (b x b, ldt) of H_1 ... H_b = I - V T V^T from S = V^T V (b x b) and tau: forward,
// columnwise: T(i, i) = tau_i, T(0:i, i) = -tau_i T(0:i, 0:i) S(0:i, i).  One thread block.
// ---------------------------------------------------------------------------------------
__global__ void k_larft(int b, const double *S, int lds, const double *tau, double *T, int ldt)
{
    __shared__ double tmp[256];
    const int tid = threadIdx.x;
    for (int e = tid; e < b * b; e += blockDim.x) T[(e % b) + (size_t)(e / b) * ldt] = 0.0;
    __syncthreads();
    for (int i = 0; i < b; ++i) {
        const double ti = tau[i];
        // w = S(0:i, i) -> tmp; T(0:i, i) = -ti T(0:i, 0:i) w
        for (int e = tid; e < i; e += blockDim.x) tmp[e] = S[e + (size_t)i * lds];
        __syncthreads();
        for (int row = tid; row < i; row += blockDim.x) {
            double acc = 0.0;
            for (int l = row; l < i; ++l) acc += T[row + (size_t)l * ldt] * tmp[l];
            T[row + (size_t)i * ldt] = -ti * acc;
        }
        if (tid == 0) T[i + (size_t)i * ldt] = ti;
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------------------
// Opposite reflectors of one filled B block (Alg. 1, right-hand part): RQ of the m x m block
// W = R~ Q~ (Householder, last row first), then the LQ factorisation of the first l rows of Q~;
// the LQ reflectors (stored as columns of V, m x l, unit lower trapezoidal in the block's column
// index) and tau_lq are returned.  Applying H_1 ... H_l from the right reduces the first l
// columns of the block.  One thread block; W and the l x m matrix M = Q~(0:l, :) live in
// shared memory.
//
// The RQ is bound by the SM's FP64 throughput (2 FMA per clock), so its reflectors are kept
// as u = x - beta e_s with tau = 1 / (beta (beta - alpha)) (no rescaling pass, one
// reciprocal), the scalars of a step are formed by warp 0 alone, and the rows are updated four
// lanes to a row, all rows in one pass: the dot products then need two shuffle-adds per eight
// rows instead of a five-level warp reduction per row.  The row stride m + 4 keeps the four
// lanes of the eight rows of a warp on distinct banks.
// ---------------------------------------------------------------------------------------
constexpr int kRQThreads = 512;
constexpr int kRQPad = 4;

__global__ void __launch_bounds__(kRQThreads) k_block_rq_lq(int m, int l, const double *Bblk, int ldb,
                                                             double *V, int ldv, double *tau_lq)
{
    extern __shared__ double sh[];
    const int ldw = m + kRQPad;
    double *W = sh;                          // m x m, row-major: W[i * ldw + c]
    double *Ms = W + (size_t)m * ldw;        // l x m, row-major
    double *rqt = Ms + (size_t)l * ldw;      // m taus of the RQ reflectors
    double *vec = rqt + m;                   // m
    __shared__ double red[32];
    __shared__ double s_tau, s_beta, s_scale;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nw = kRQThreads / 32;

    for (int e = tid; e < m * m; e += kRQThreads) {
        const int i = e % m, c = e / m;
        W[i * ldw + c] = Bblk[(size_t)i + (size_t)c * ldb];
    }
    __syncthreads();
    // RQ: for s = m-1 .. 1 (0-based pivot row s, pivot column s); reflector u_s in row s of W
    // (u_s(s) = alpha - beta), tau in rqt[s] (0: the identity)
    const int row = tid >> 2, sub = tid & 3;   // m <= 128 = kRQThreads / 4 rows: one pass
    for (int s = m - 1; s >= 1; --s) {
        if (warp == 0) {
            double p0 = 0.0, p1 = 0.0;
            for (int c = lane; c < s; c += 64) {
                p0 = fma(W[s * ldw + c], W[s * ldw + c], p0);
                if (c + 32 < s) p1 = fma(W[s * ldw + c + 32], W[s * ldw + c + 32], p1);
            }
            const double ssq = warp_sum(p0 + p1);
            if (lane == 0) {
                const double alpha = W[s * ldw + s];
                double tau = 0.0;
                if (ssq != 0.0) {
                    const double nrm = sqrt(fma(alpha, alpha, ssq));
                    const double beta = (alpha >= 0.0) ? -nrm : nrm;
                    tau = 1.0 / (beta * (beta - alpha));
                    W[s * ldw + s] = alpha - beta;
                }
                rqt[s] = tau;
            }
        }
        __syncthreads();
        const double ts = rqt[s];
        // rows 0 .. s-1 := row - tau (row . u) u^T; a warp whose rows are all >= s skips
        if (ts != 0.0 && (warp << 3) < s) {
            const bool act = row < s;
            const double *u = W + (size_t)s * ldw;
            double *w = W + (size_t)row * ldw;
            double d0 = 0.0, d1 = 0.0;
            if (act)
                for (int c = sub; c <= s; c += 8) {
                    d0 = fma(w[c], u[c], d0);
                    if (c + 4 <= s) d1 = fma(w[c + 4], u[c + 4], d1);
                }
            double d = d0 + d1;
            d += __shfl_xor_sync(0xffffffffu, d, 1);
            d += __shfl_xor_sync(0xffffffffu, d, 2);
            d *= ts;
            if (act)
                for (int c = sub; c <= s; c += 4) w[c] = fma(-d, u[c], w[c]);
        }
        __syncthreads();
    }
    // M = E_l^T Q~ with Q~ = H_(1) H_(2) ... H_(m-1), where H_(s) = I - tau_s u_s u_s^T acts on
    // columns 0..s: the reflectors applied to the l rows of M in that order, a warp per row
    for (int e = tid; e < l * m; e += kRQThreads) {
        const int t = e / m, c = e % m;
        Ms[t * ldw + c] = (t == c) ? 1.0 : 0.0;
    }
    __syncthreads();
    for (int s = 1; s <= m - 1; ++s) {
        const double ts = rqt[s];
        if (ts != 0.0) {
            const double *u = W + (size_t)s * ldw;
            for (int t = warp; t < l; t += nw) {
                double d = 0.0;
                for (int c = lane; c <= s; c += 32) d = fma(Ms[t * ldw + c], u[c], d);
                d = warp_sum(d) * ts;
                for (int c = lane; c <= s; c += 32) Ms[t * ldw + c] = fma(-d, u[c], Ms[t * ldw + c]);
            }
        }
        __syncthreads();
    }
    // LQ of M (l x m): reflector t reduces M(t, t:m) to beta e_1, applied to rows t+1..l-1
    for (int t = 0; t < l; ++t) {
        double part = 0.0;
        for (int c = t + 1 + tid; c < m; c += kRQThreads) part += Ms[t * ldw + c] * Ms[t * ldw + c];
        const double ssq = block_sum(part, red);
        if (tid == 0) {
            const double alpha = Ms[t * ldw + t];
            if (ssq == 0.0) {
                s_tau = 0.0; s_beta = alpha; s_scale = 0.0;
            } else {
                const double nrm = sqrt(alpha * alpha + ssq);
                const double beta = (alpha >= 0.0) ? -nrm : nrm;
                s_tau = (beta - alpha) / beta;
                s_scale = 1.0 / (alpha - beta);
                s_beta = beta;
            }
            tau_lq[t] = s_tau;
        }
        __syncthreads();
        const double tt = s_tau, sc = s_scale;
        for (int c = tid; c < m; c += kRQThreads) {
            double vc;
            if (c < t) vc = 0.0;
            else if (c == t) vc = 1.0;
            else vc = (tt == 0.0) ? 0.0 : Ms[t * ldw + c] * sc;
            vec[c] = vc;
            V[(size_t)c + (size_t)t * ldv] = vc;
        }
        __syncthreads();
        if (tt != 0.0) {
            for (int row = t + 1 + warp; row < l; row += nw) {
                double d = 0.0;
                for (int c = t + lane; c < m; c += 32) d += Ms[row * ldw + c] * vec[c];
                d = warp_sum(d) * tt;
                for (int c = t + lane; c < m; c += 32) Ms[row * ldw + c] -= d * vec[c];
            }
        }
        __syncthreads();
    }
}

size_t block_rq_lq_smem(int m, int l) { return sizeof(double) * ((size_t)(m + l) * (m + kRQPad) + 2 * (size_t)m); }

cudaError_t launch_panel_qr(int m, int b, double *P, int ld, double *V, int ldv, double *tau, cudaStream_t st)
{
    k_panel_qr<<<1, kPanelThreads, 0, st>>>(m, b, P, ld, V, ldv, tau);
    return cudaGetLastError();
}

cudaError_t launch_larft(int b, const double *S, int lds, const double *tau, double *T, int ldt, cudaStream_t st)
{
    k_larft<<<1, 256, 0, st>>>(b, S, lds, tau, T, ldt);
    return cudaGetLastError();
}

cudaError_t launch_block_rq_lq(int m, int l, const double *Bblk, int ldb, double *V, int ldv, double *tau_lq,
                               cudaStream_t st)
{
    const size_t sm = block_rq_lq_smem(m, l);
    cudaError_t e = cudaFuncSetAttribute(k_block_rq_lq, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_block_rq_lq<<<1, kRQThreads, sm, st>>>(m, l, Bblk, ldb, V, ldv, tau_lq);
    return cudaGetLastError();
}

}  // namespace hts
