// Batched reduction of many small pencils in one launch (hts_reduce_batched).
//
// One thread block reduces one whole pencil: QR of B (stage 0), Alg. 1 with n_b = r (stage
// 1) and Alg. 2 (stage 2).  Every reflector is applied on its own, in the order the
// algorithms state, with the work of each application spread over the block (one warp per
// column for left applications, one thread per row for right applications).  Blocks are
// launched largest pencil first, so the hardware's in-order block dispatch gives a
// longest-processing-time schedule; many small pencils keep every SM busy.
#include <algorithm>

#include "hts_internal.cuh"

namespace hts {

namespace {

constexpr int kBT = 256;            // threads per pencil
constexpr int kBW = kBT / 32;
constexpr int kBatchMaxN = 512;     // reflector buffer length (largest pencil)
constexpr int kBatchMaxBlk = 64;    // largest B block (p * r) of stage 1 kept in shared memory

struct BatchShared {
    double v[kBatchMaxN];                        // current reflector (explicit v_0 = 1)
    double W[kBatchMaxBlk * (kBatchMaxBlk + 1)];  // B block for the RQ (row-major)
    double Mq[16 * (kBatchMaxBlk + 1)];          // first rows of the RQ's orthogonal factor
    double rqt[kBatchMaxBlk];
    double red[kBW];
    double tau, beta, scale;
};

__device__ __forceinline__ double bsum(double x, BatchShared &S)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    x = warp_sum(x);
    __syncthreads();
    if (lane == 0) S.red[warp] = x;
    __syncthreads();
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < kBW; ++w) s += S.red[w];
    return s;
}

__device__ __forceinline__ double bmax(double x, BatchShared &S)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    x = warp_max(x);
    __syncthreads();
    if (lane == 0) S.red[warp] = x;
    __syncthreads();
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < kBW; ++w) s = fmax(s, S.red[w]);
    return s;
}

// Householder data (dlarfg convention) of the vector with pivot alpha and other entries
// get(0 .. cnt-1): S.tau, S.beta, and S.scale, the factor that turns an entry into its
// component of v (v_pivot = 1).  The sum of squares is formed directly and, when it leaves
// [1e-290, 1e290] or alpha exceeds 1e145, again with every entry divided by the largest
// magnitude, so that no intermediate over- or underflows.  tau = 0 (the identity) only when
// every other entry is exactly zero.  Called by the whole block.
template <class Get>
__device__ void blk_house(double alpha, int cnt, Get get, BatchShared &S)
{
    double part = 0.0;
    for (int i = threadIdx.x; i < cnt; i += kBT) part = fma(get(i), get(i), part);
    double ssq = bsum(part, S);
    double scale = 1.0;
    if (!(ssq >= 1e-290 && ssq <= 1e290) || fabs(alpha) > 1e145) {   // uniform over the block
        double mp = 0.0;
        for (int i = threadIdx.x; i < cnt; i += kBT) mp = fmax(mp, fabs(get(i)));
        const double mx = bmax(mp, S);
        if (mx == 0.0) {
            ssq = 0.0;
        } else {
            scale = fmax(mx, fabs(alpha));
            const double rs = 1.0 / scale;
            part = 0.0;
            for (int i = threadIdx.x; i < cnt; i += kBT) {
                const double t = get(i) * rs;
                part = fma(t, t, part);
            }
            ssq = bsum(part, S);
        }
    }
    if (threadIdx.x == 0) {
        if (cnt <= 0 || ssq == 0.0) {
            S.tau = 0.0; S.beta = alpha; S.scale = 0.0;
        } else {
            const double as = alpha / scale;
            const double nrm = scale * sqrt(fma(as, as, ssq));
            const double b = alpha >= 0.0 ? -nrm : nrm;
            S.tau = (b - alpha) / b;
            S.scale = 1.0 / (alpha - b);
            S.beta = b;
        }
    }
    __syncthreads();
}

// Reflector (dlarfg convention) from m entries x[0], x[inc], ...; v goes to S.v (v_0 = 1),
// tau / beta to S.tau / S.beta; x is overwritten by (beta, 0, ..., 0).
__device__ void blk_larfg(double *x, long inc, int m, BatchShared &S)
{
    blk_house(x[0], m - 1, [&](int i) { return x[(i + 1) * inc]; }, S);
    for (int i = threadIdx.x; i < m; i += kBT) {
        S.v[i] = (i == 0) ? 1.0 : x[i * inc] * S.scale;
        x[i * inc] = (i == 0) ? S.beta : 0.0;
    }
    __syncthreads();
}

// M(r0:r0+m-1, c0:c1) := H M(...), one warp per column
__device__ void blk_left(double *M, int ld, int r0, int m, int c0, int c1, const BatchShared &S)
{
    const double tau = S.tau;
    if (tau == 0.0 || c1 < c0) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (m <= 16) {
        // short reflectors (stage 2's r <= 16, the ends of stages 0 and 1): g lanes per column,
        // 32/g columns per warp, so that a column's dot product takes log2(g) shuffle-adds
        // instead of five (FP64 instructions are the cost on this GPU, whatever their lanes)
        const int g = m <= 4 ? 4 : (m <= 8 ? 8 : 16);
        const int per = 32 / g, sub = lane & (g - 1), slot = lane / g;
        const double v = sub < m ? S.v[sub] : 0.0;
        for (int cb = c0 + warp * per; cb <= c1; cb += kBW * per) {   // uniform per warp
            const int c = cb + slot;
            const bool own = c <= c1 && sub < m;
            double *col = own ? M + AT(ld, r0, c) : nullptr;
            const double x = own ? col[sub] : 0.0;
            double d = x * v;
            for (int o = 1; o < g; o <<= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
            d *= tau;
            if (own) col[sub] = x - d * v;
        }
        return;
    }
    for (int c = c0 + warp; c <= c1; c += kBW) {
        double *col = M + AT(ld, r0, c);
        double d = 0.0;
        for (int i = lane; i < m; i += 32) d += S.v[i] * col[i];
        d = warp_sum(d) * tau;
        for (int i = lane; i < m; i += 32) col[i] -= d * S.v[i];
    }
}

// M(x0:x1, c0:c0+m-1) := M(...) H, one thread per row
__device__ void blk_right(double *M, int ld, int x0, int x1, int c0, int m, const BatchShared &S)
{
    const double tau = S.tau;
    if (tau == 0.0) return;
    for (int x = x0 + threadIdx.x; x <= x1; x += kBT) {
        double *row = M + AT(ld, x, c0);
        double d0 = 0.0, d1 = 0.0;
        int i = 0;
        for (; i + 1 < m; i += 2) {
            d0 += row[(size_t)i * ld] * S.v[i];
            d1 += row[(size_t)(i + 1) * ld] * S.v[i + 1];
        }
        if (i < m) d0 += row[(size_t)i * ld] * S.v[i];
        const double d = (d0 + d1) * tau;
        for (int c = 0; c < m; ++c) row[(size_t)c * ld] -= d * S.v[c];
    }
}

// RQ of the m x m block already in S.W (row-major, ld m+1), last row first; reflectors kept in
// the zeroed part of S.W, taus in S.rqt.  Then S.Mq (l x m) = first l rows of Q~.
__device__ void blk_rq_first_rows(int m, int l, BatchShared &S)
{
    const int ldw = m + 1;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int s = m - 1; s >= 1; --s) {
        const double *wrow = &S.W[s * ldw];
        blk_house(wrow[s], s, [&](int c) { return wrow[c]; }, S);
        if (threadIdx.x == 0) S.rqt[s] = S.tau;
        __syncthreads();
        for (int c = threadIdx.x; c < s; c += kBT) S.W[s * ldw + c] *= S.scale;
        __syncthreads();
        const double ts = S.rqt[s];
        if (ts != 0.0) {
            for (int row = warp; row < s; row += kBW) {
                double d = 0.0;
                for (int c = lane; c <= s; c += 32) d += S.W[row * ldw + c] * (c == s ? 1.0 : S.W[s * ldw + c]);
                d = warp_sum(d) * ts;
                for (int c = lane; c <= s; c += 32) S.W[row * ldw + c] -= d * (c == s ? 1.0 : S.W[s * ldw + c]);
            }
        }
        __syncthreads();
    }
    for (int e = threadIdx.x; e < l * m; e += kBT) S.Mq[(e / m) * ldw + e % m] = (e / m == e % m) ? 1.0 : 0.0;
    __syncthreads();
    for (int s = 1; s <= m - 1; ++s) {
        const double ts = S.rqt[s];
        if (ts != 0.0) {
            for (int t = warp; t < l; t += kBW) {
                double d = 0.0;
                for (int c = lane; c <= s; c += 32) d += S.Mq[t * ldw + c] * (c == s ? 1.0 : S.W[s * ldw + c]);
                d = warp_sum(d) * ts;
                for (int c = lane; c <= s; c += 32) S.Mq[t * ldw + c] -= d * (c == s ? 1.0 : S.W[s * ldw + c]);
            }
        }
        __syncthreads();
    }
}

__device__ void load_block(const double *B, int ldb, int i1, int m, BatchShared &S)
{
    for (int e = threadIdx.x; e < m * m; e += kBT) {
        const int i = e % m, c = e / m;
        S.W[i * (m + 1) + c] = B[AT(ldb, i1 + i, i1 + c)];
    }
    __syncthreads();
}

}  // namespace

struct BatchDesc {
    double *A, *B, *Q, *Z;
    int n, r, lda, ldb, ldq, ldz;
};

__host__ __device__ __forceinline__ size_t round256(size_t x) { return (x + 255) / 256 * 256; }

// What a launch reads besides the descriptors: written once by the plan, then fixed.
struct BatchHead {
    int count, compq, compz, p;
};

// Reduction of pencil pid (its descriptor d) by the whole block.
__device__ void reduce_pencil(const BatchDesc &d, int pid, int p_param, int compq, int compz, int *status,
                              BatchShared &S)
{
    const int n = d.n, r = d.r;
    double *A = d.A, *B = d.B;
    double *Q = compq ? d.Q : nullptr, *Z = compz ? d.Z : nullptr;
    // NaN / Inf among the pencil's inputs: record it (the first one of the batch is reported)
    // and leave this pencil alone; the other pencils are reduced
    {
        int bad = 0;
        for (int e = threadIdx.x; e < n * n && !bad; e += kBT) {
            const int i = e % n + 1, c = e / n + 1;
            const int which = (((__double_as_longlong(A[AT(d.lda, i, c)]) >> 52) & 0x7ff) == 0x7ff) ? 1
                              : (((__double_as_longlong(B[AT(d.ldb, i, c)]) >> 52) & 0x7ff) == 0x7ff) ? 2
                              : (compq == HTS_COMP_UPDATE &&
                                 ((__double_as_longlong(Q[AT(d.ldq, i, c)]) >> 52) & 0x7ff) == 0x7ff) ? 3
                              : (compz == HTS_COMP_UPDATE &&
                                 ((__double_as_longlong(Z[AT(d.ldz, i, c)]) >> 52) & 0x7ff) == 0x7ff) ? 4
                                                                                                  : 0;
            if (which) {
                record_error(status, HTS_ERR_NONFINITE, pid, which - 1, i, c);
                bad = 1;
            }
        }
        if (__syncthreads_or(bad)) return;
    }
    // identity initialisation
    for (int e = threadIdx.x; e < n * n; e += kBT) {
        const int i = e % n + 1, c = e / n + 1;
        if (compq == HTS_COMP_INIT) Q[AT(d.ldq, i, c)] = (i == c) ? 1.0 : 0.0;
        if (compz == HTS_COMP_INIT) Z[AT(d.ldz, i, c)] = (i == c) ? 1.0 : 0.0;
    }
    __syncthreads();

    // ---- stage 0: QR of B
    for (int j = 1; j <= n - 1; ++j) {
        const int m = n - j + 1;
        blk_larfg(B + AT(d.ldb, j, j), 1, m, S);
        blk_left(B, d.ldb, j, m, j + 1, n, S);
        blk_left(A, d.lda, j, m, 1, n, S);
        if (Q) blk_right(Q, d.ldq, 1, n, j, m, S);
        __syncthreads();
    }
    if (n <= 2) return;

    // ---- stage 1: Alg. 1 with n_b = r
    const int nb = r;
    const int p = (p_param > 0) ? p_param : imin(8, imax(2, kBatchMaxBlk / nb));
    for (int j = 1; j <= n - 2; j += nb) {
        const int j1 = j, j2 = imin(n, j + nb - 1);
        const int num = n - nb - j + 1, den = (p - 1) * nb;
        const int nblocks = num > 0 ? (num + den - 1) / den : 0;
        for (int k = nblocks - 1; k >= 0; --k) {
            const int i1 = j + nb + k * (p - 1) * nb;
            const int i2 = imin(n, i1 + p * nb - 1);
            for (int c = j1; c <= j2; ++c) {
                const int rs = i1 + (c - j1);
                if (rs > i2) break;
                const int m = i2 - rs + 1;
                blk_larfg(A + AT(d.lda, rs, c), 1, m, S);
                blk_left(A, d.lda, rs, m, c + 1, n, S);
                blk_left(B, d.ldb, rs, m, i1, n, S);
                if (Q) blk_right(Q, d.ldq, 1, n, rs, m, S);
                __syncthreads();
            }
        }
        for (int k = nblocks - 1; k >= 0; --k) {
            const int i1 = j + nb + k * (p - 1) * nb;
            const int i2 = imin(n, i1 + p * nb - 1);
            const int m = i2 - i1 + 1, l = imin(nb, m);
            load_block(B, d.ldb, i1, m, S);
            blk_rq_first_rows(m, l, S);
            for (int t = 0; t < l; ++t) {
                const int len = m - t;
                blk_larfg(&S.Mq[t * (m + 1) + t], 1, len, S);
                // the remaining rows of Mq
                if (S.tau != 0.0) {
                    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
                    for (int row = t + 1 + warp; row < l; row += kBW) {
                        double dd = 0.0;
                        for (int c = lane; c < len; c += 32) dd += S.Mq[row * (m + 1) + t + c] * S.v[c];
                        dd = warp_sum(dd) * S.tau;
                        for (int c = lane; c < len; c += 32) S.Mq[row * (m + 1) + t + c] -= dd * S.v[c];
                    }
                }
                blk_right(A, d.lda, 1, n, i1 + t, len, S);
                blk_right(B, d.ldb, 1, i2, i1 + t, len, S);
                if (Z) blk_right(Z, d.ldz, 1, n, i1 + t, len, S);
                __syncthreads();
                for (int x = i1 + t + 1 + threadIdx.x; x <= i2; x += kBT) B[AT(d.ldb, x, i1 + t)] = 0.0;
                __syncthreads();
            }
        }
    }

    // ---- stage 2: Alg. 2
    for (int j = 1; j <= n - 2 && r > 1; ++j) {
        const int nblocks = 1 + (n - j - 2) / r;
        for (int k = 0; k < nblocks; ++k) {
            const int jb = j + imax(0, (k - 1) * r + 1);
            const int i1 = j + k * r + 1;
            const int i2 = imin(j + (k + 1) * r, n);
            const int i3 = imin(j + (k + 2) * r, n);
            const int m = i2 - i1 + 1;
            blk_larfg(A + AT(d.lda, i1, jb), 1, m, S);
            blk_left(A, d.lda, i1, m, jb + 1, n, S);
            blk_left(B, d.ldb, i1, m, i1, n, S);
            if (Q) blk_right(Q, d.ldq, 1, n, i1, m, S);
            __syncthreads();
            load_block(B, d.ldb, i1, m, S);
            blk_rq_first_rows(m, 1, S);
            blk_larfg(&S.Mq[0], 1, m, S);
            blk_right(A, d.lda, 1, i3, i1, m, S);
            blk_right(B, d.ldb, 1, i2, i1, m, S);
            if (Z) blk_right(Z, d.ldz, 1, n, i1, m, S);
            __syncthreads();
            for (int x = i1 + 1 + threadIdx.x; x <= i2; x += kBT) B[AT(d.ldb, x, i1)] = 0.0;
            __syncthreads();
        }
    }
}

// Persistent launch: each block takes the next pencil of the largest-first order from a device
// queue (one atomic counter, zeroed before the launch) until the batch is used up.  The queue
// keeps the longest-processing-time order of a one-block-per-pencil launch while the grid stays
// at what the SMs hold at once.
__global__ void __launch_bounds__(kBT) k_reduce_batched(const BatchHead *head, unsigned *next, const BatchDesc *desc,
                                                         const int *order, int *status)
{
    __shared__ BatchShared S;
    __shared__ int s_idx;
    const BatchHead h = *head;
    for (;;) {
        if (threadIdx.x == 0) s_idx = (int)atomicAdd(next, 1u);
        __syncthreads();
        const int idx = s_idx;
        __syncthreads();   // s_idx is taken again by the next round
        if (idx >= h.count) return;
        const int pid = order[idx];
        reduce_pencil(desc[pid], pid, h.p, h.compq, h.compz, status, S);
        __syncthreads();
    }
}

// Workspace of a batch: [head | queue counter at byte 128] [descriptors] [order], each part
// 256-byte aligned.
size_t batch_work_bytes(int count)
{
    return 256 + round256((size_t)count * sizeof(BatchDesc)) + round256((size_t)count * sizeof(int));
}

void batch_stage(void *host, int count, const int *n, const int *r, double *const *A, const int *lda,
                 double *const *B, const int *ldb, double *const *Q, const int *ldq, double *const *Z, const int *ldz,
                 int compq, int compz, int p)
{
    unsigned char *w = static_cast<unsigned char *>(host);
    BatchHead *h = reinterpret_cast<BatchHead *>(w);
    h->count = count; h->compq = compq; h->compz = compz; h->p = p;
    *reinterpret_cast<unsigned *>(w + 128) = 0u;
    BatchDesc *d = reinterpret_cast<BatchDesc *>(w + 256);
    int *order = reinterpret_cast<int *>(w + 256 + round256((size_t)count * sizeof(BatchDesc)));
    for (int i = 0; i < count; ++i) {
        d[i].A = A[i]; d[i].B = B[i];
        d[i].Q = compq ? Q[i] : nullptr; d[i].Z = compz ? Z[i] : nullptr;
        d[i].n = n[i]; d[i].r = r[i]; d[i].lda = lda[i]; d[i].ldb = ldb[i];
        d[i].ldq = compq ? ldq[i] : 1; d[i].ldz = compz ? ldz[i] : 1;
        order[i] = i;
    }
    std::stable_sort(order, order + count, [&](int a, int b2) { return n[a] > n[b2]; });
}

// per_sm: persistent blocks per SM (0 or more than fit: as many as fit).
cudaError_t launch_reduce_batched(void *work, int count, int num_sms, int per_sm_req, int *status, cudaStream_t st)
{
    static int fit = 0;
    if (fit == 0) {
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_reduce_batched, kBT, 0) != cudaSuccess || b < 1) b = 1;
        fit = b;
    }
    const int per_sm = (per_sm_req > 0 && per_sm_req < fit) ? per_sm_req : fit;
    unsigned char *w = static_cast<unsigned char *>(work);
    cudaError_t e = cudaMemsetAsync(w + 128, 0, sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
    const int grid = imax(1, imin(count, per_sm * num_sms));
    const size_t off_order = 256 + round256((size_t)count * sizeof(BatchDesc));
    k_reduce_batched<<<grid, kBT, 0, st>>>(reinterpret_cast<const BatchHead *>(w), reinterpret_cast<unsigned *>(w + 128),
                                           reinterpret_cast<const BatchDesc *>(w + 256),
                                           reinterpret_cast<const int *>(w + off_order), status);
    return cudaGetLastError();
}

int batch_max_n() { return kBatchMaxN; }
int batch_max_block() { return kBatchMaxBlk; }

}  // namespace hts
