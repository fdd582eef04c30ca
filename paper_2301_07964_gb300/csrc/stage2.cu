// Stage 2 of the two-stage HT reduction: r-HT pencil -> HT pencil by bulge chasing
// (Steel & Vandebril, Section "Reduction to Hessenberg-triangular form").
//
// One group of qg consecutive sweeps j1 .. j1+qg-1 is processed by three launches:
//   k_s2_generate     Alg. 3 (generate phase): the near-diagonal chase (chase.cu).
//   k_s2_apply_right  Alg. 4, right-hand part: the delayed Z^ reflectors on the rows of A
//                     and B above the generate band, and on all rows of Z; the Q^ reflectors
//                     on all rows of Q.
//   k_s2_apply_left   Alg. 4, left-hand part: the delayed Q^ reflectors on the columns of A
//                     and B right of the columns the generate phase already updated.
// The delayed updates walk the blocks k from the last to the first with a sliding window of
// r + qg - 1 columns (rows), so every element is read and written once per group; inside
// the window the group's reflectors are applied one at a time in FP64.
#include "right_window.cuh"
#include "schedule.cuh"

namespace hts {

// ---------------------------------------------------------------------------------------
// Delayed right updates (Alg. 4, first loop).  One thread per row; blockIdx.y selects the
// matrix.  kind 0 = A, 1 = B (Z^ reflectors, rows x < i4(k, j) only: the generate phase
// updated the rest), 2 = Z (Z^ reflectors, all rows), 3 = Q (Q^ reflectors, all rows).
// ---------------------------------------------------------------------------------------

// One tile of rows (tile*NR+1 .., NR = NT/4) of matrix a.M[mi], by NT threads of a group with
// barrier id bar.
template <int NT>
__device__ __forceinline__ void right_tile_fp64(const ApplyArgs &a, int mi, int tile, double *sm, int tid, int bar)
{
    constexpr int NR = NT / kRightLanes;                    // rows per tile
    const int n = a.n, r = a.r, j1 = a.j1, qg = a.qg;
    const int kind = a.kind[mi];
    const int x0 = tile * NR + 1;
    const int kmax = nblocks_gen(n, r, j1) - 1;
    if (x0 > n) return;
    int kstop = 0;
    if (kind <= 1) {
        // rows x0.. need block k only while x0 < i4(k, j1+qg-1) = j1 + 1 + max(0, (k-1) r)
        kstop = (x0 <= j1) ? 0 : (x0 - j1 - 1) / r + 2;
        if (kstop > kmax) return;
    }
    right_window_rows<NT>(a.M[mi], a.ld[mi], kind, (kind == 3) ? a.R.VQ : a.R.VZ, (kind == 3) ? a.R.TQ : a.R.TZ,
                          a.R.kdim, n, r, j1, qg, x0, kmax, kstop, sm, tid, bar);
}

template <int NT>
__global__ void __launch_bounds__(NT) k_s2_apply_right(ApplyArgs a)
{
    extern __shared__ double sm[];
    if (__ldcg(a.status) != 0) return;
    right_tile_fp64<NT>(a, blockIdx.y, blockIdx.x, sm, threadIdx.x, 0);
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

// Four lanes share a column: lane l of the group owns rows l, l+4, ... of each reflector, so a
// column's chain of dependent operations is a quarter as long as with one thread per column.
constexpr int kLeftThreads = 128;
constexpr int kLeftLanes = 4;
constexpr int kLeftCols = kLeftThreads / kLeftLanes;   // columns per thread block

// One column tile (columns ctile*kLeftCols+1 ..) of the left update of A (isB = 0) or B, by
// the kLeftThreads threads tid of a group whose barrier is bar (0: a whole block).
__device__ __forceinline__ void left_tile(const LeftArgs &a, int isB, int ctile, double *sm, int tid, int bar)
{
    const int NT = kLeftThreads;
    const int NC = kLeftCols;
    const int LDS = NC + 1;
    const int n = a.n, r = a.r, j1 = a.j1, qg = a.qg;
    const int w = r + qg - 1;
    const int jl = j1 + qg - 1;
    double *buf = sm;                       // [w][LDS]: column cc of the tile at buf[p*LDS+cc]
    double *vr = buf + (size_t)w * LDS;     // [qg][r]
    double *tr = vr + (size_t)qg * r;       // [qg]
    double *X = isB ? a.B : a.A;
    const int ld = isB ? a.ldb : a.lda;
    const int cc = tid / kLeftLanes, sub = tid % kLeftLanes;
    const int cbase = ctile * NC + 1;
    const int c = cbase + cc;
    const int clast = imin(cbase + NC - 1, n);
    const int kdim = a.R.kdim;
    const int kmax = nblocks_gen(n, r, j1) - 1;

    int ktop = -1;
    for (int k = kmax; k >= 0; --k)
        if (left_cut(isB, n, r, jl, k) < clast) { ktop = k; break; }
    if (ktop < 0 || cbase > n) return;

    for (int k = ktop; k >= 0; --k) {
        const int R0 = j1 + k * r + 1;
        group_sync(bar, NT);
        for (int e = tid; e < qg * r; e += NT) {
            const int sidx = e / r, i = e % r;
            vr[e] = a.R.VQ[((size_t)sidx * kdim + k) * r + i];
        }
        for (int e = tid; e < qg; e += NT) tr[e] = a.R.TQ[(size_t)e * kdim + k];
        const int pnew = (k == ktop) ? w : r;
        for (int e = tid; e < pnew * NC; e += NT) {
            const int p = e % pnew, ce = e / pnew;
            const int row = R0 + p, colx = cbase + ce;
            if (row <= n && colx <= n) buf[p * LDS + ce] = X[AT(ld, row, colx)];
        }
        group_sync(bar, NT);
        const bool active = c <= n && c > left_cut(isB, n, r, jl, k);
        for (int sidx = 0; sidx < qg; ++sidx) {
            const double tau = tr[sidx];
            if (tau == 0.0) continue;
            const int mlen = imin(r, n - (j1 + sidx + k * r));
            const double *v = vr + sidx * r;
            double *b = buf + sidx * LDS + cc;
            double d = 0.0;
            if (active)
                for (int i = sub; i < mlen; i += kLeftLanes) d += b[i * LDS] * v[i];
            d += __shfl_xor_sync(0xffffffffu, d, 1);
            d += __shfl_xor_sync(0xffffffffu, d, 2);
            d *= tau;
            if (active)
                for (int i = sub; i < mlen; i += kLeftLanes) b[i * LDS] -= d * v[i];
        }
        group_sync(bar, NT);
        const int plo = (k > 0) ? qg - 1 : 0;
        const int np = w - plo;
        for (int e = tid; e < np * NC; e += NT) {
            const int p = plo + e % np, ce = e / np;
            const int row = R0 + p, colx = cbase + ce;
            if (row <= n && colx <= n) X[AT(ld, row, colx)] = buf[p * LDS + ce];
        }
        group_sync(bar, NT);
        if (k > 0)
            for (int e = tid; e < (qg - 1) * NC; e += NT) {
                const int p = e / NC, ce = e % NC;
                buf[(p + r) * LDS + ce] = buf[p * LDS + ce];
            }
    }
}

__global__ void __launch_bounds__(kLeftThreads) k_s2_apply_left(LeftArgs a)
{
    extern __shared__ double sm[];
    if (__ldcg(a.status) != 0) return;
    // the rightmost tiles carry the most work: they start first
    left_tile(a, blockIdx.y, gridDim.x - 1 - blockIdx.x, sm, threadIdx.x, 0);
}

// ---------------------------------------------------------------------------------------
// Look-ahead update launch in native FP64 (schedule.cuh): one block per SM with kUpdFp64Workers
// workers of 128 threads (barrier id w+1), each with its own slice of shared memory.
// ---------------------------------------------------------------------------------------
constexpr int kUpdFp64Workers = 4;
constexpr int kUpdThreads = 128;

__global__ void __launch_bounds__(kUpdThreads * kUpdFp64Workers, 1) k_s2_update_fp64(UpdFp64Args a)
{
    extern __shared__ double upd_sm[];
    __shared__ int slot[kUpdFp64Workers];
    const int worker = threadIdx.x / kUpdThreads, tid = threadIdx.x % kUpdThreads;
    double *sm = upd_sm + (size_t)worker * a.smem_doubles;
    const int wb = 1 + worker;
    update_worker<kUpdThreads>(a.s, tid, wb, &slot[worker], [&](const Task &T) {
        if (T.kind == kTaskRight) right_tile_fp64<kUpdThreads>(a.right, T.mat, T.tile, sm, tid, wb);
        else if (T.kind == kTaskLeft) left_tile(a.left, T.mat, T.tile, sm, tid, wb);
        else if (T.kind == kTaskQZ) right_tile_fp64<kUpdThreads>(a.qz, T.mat, T.tile, sm, tid, wb);
    });
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

// Zero A below its first subdiagonal (band = 1) or B below its diagonal (band = 0); skipped
// once an earlier kernel of the call has recorded an error.
__global__ void k_zero_below(double *M, int ld, int n, int band, const int *status)
{
    if (__ldcg(status) != 0) return;
    const int c = blockIdx.y + 1;
    for (int i = c + band + 1 + blockIdx.x * blockDim.x + threadIdx.x; i <= n; i += gridDim.x * blockDim.x)
        M[AT(ld, i, c)] = 0.0;
}

// Entries a call reads that are NaN or infinite (exponent field all ones): column c, rows 1 ..
// min(n, c + lower).  The first one found is recorded as HTS_ERR_NONFINITE with {0, which, row,
// column}; every kernel of the reduction that checks the status word then does nothing.
__global__ void k_scan_nonfinite(const double *M, int ld, int n, int lower, int which, int *status)
{
    const int c = blockIdx.y + 1;
    const int last = imin(n, c + lower);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x + 1; i <= last; i += gridDim.x * blockDim.x) {
        const long long bits = __double_as_longlong(__ldg(M + AT(ld, i, c)));
        if (((bits >> 52) & 0x7ff) == 0x7ff) record_error(status, HTS_ERR_NONFINITE, 0, which, i, c);
    }
}

// ---------------------------------------------------------------------------------------
// Host-side launchers
// ---------------------------------------------------------------------------------------
size_t apply_right_smem(int r, int qg, int rows) { return sizeof(double) * ((size_t)(r + qg - 1) * (rows + 1) + (size_t)qg * r + qg); }
size_t apply_left_smem(int r, int qg) { return sizeof(double) * ((size_t)(r + qg - 1) * (kLeftCols + 1) + (size_t)qg * r + qg); }

// The A / B launch uses small blocks.  The Q / Z launch (side stream, overlapping the next
// group's chase) uses 512-thread blocks that reserve more shared memory than an SM hosting a
// chase block has left, so it never shares an SM, and its FP64 pipes, with the chase.
constexpr int kRightThreadsAB = 128;
constexpr int kRightThreadsQZ = 512;
constexpr size_t kQZSmemReserve = 201 * 1024;

cudaError_t launch_s2_apply_right(const ApplyArgs &a, int nmat, cudaStream_t st)
{
    const bool qz = a.kind[0] >= 2;
    cudaError_t e;
    if (!qz) {
        const int rows = kRightThreadsAB / kRightLanes;
        const size_t sm = apply_right_smem(a.r, a.qg, rows);
        e = cudaFuncSetAttribute(k_s2_apply_right<kRightThreadsAB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        dim3 grid((a.n + rows - 1) / rows, nmat);
        k_s2_apply_right<kRightThreadsAB><<<grid, kRightThreadsAB, sm, st>>>(a);
    } else {
        const int rows = kRightThreadsQZ / kRightLanes;
        size_t sm = apply_right_smem(a.r, a.qg, rows);
        if (sm < kQZSmemReserve) sm = kQZSmemReserve;
        e = cudaFuncSetAttribute(k_s2_apply_right<kRightThreadsQZ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        dim3 grid((a.n + rows - 1) / rows, nmat);
        k_s2_apply_right<kRightThreadsQZ><<<grid, kRightThreadsQZ, sm, st>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t launch_s2_apply_left(const LeftArgs &a, cudaStream_t st)
{
    const size_t sm = apply_left_smem(a.r, a.qg);
    cudaError_t e = cudaFuncSetAttribute(k_s2_apply_left, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    dim3 grid((a.n + kLeftCols - 1) / kLeftCols, 2);
    k_s2_apply_left<<<grid, kLeftThreads, sm, st>>>(a);
    return cudaGetLastError();
}

int update_fp64_workers() { return kUpdFp64Workers; }

// Shared memory of one native update worker, in doubles (a multiple of 2, so that every
// worker's slice stays 16-byte aligned).
int update_fp64_smem_doubles(int r, int qg)
{
    const size_t b = apply_right_smem(r, qg, kUpdThreads / kRightLanes);
    const size_t l = apply_left_smem(r, qg);
    const size_t d = (b > l ? b : l) / sizeof(double);
    return (int)((d + 1) & ~(size_t)1);
}

cudaError_t launch_s2_update_fp64(const UpdFp64Args &a, int ctas, cudaStream_t st)
{
    // at least 116 KiB, so that two blocks never share an SM and the free SMs stay whole
    size_t sm = (size_t)kUpdFp64Workers * a.smem_doubles * sizeof(double);
    if (sm < 116 * 1024) sm = 116 * 1024;
    cudaError_t e = cudaFuncSetAttribute(k_s2_update_fp64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_s2_update_fp64<<<ctas, kUpdThreads * kUpdFp64Workers, sm, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_set_identity(double *M, int ld, int n, cudaStream_t st)
{
    dim3 grid((n + 255) / 256, n);
    k_set_identity<<<grid, 256, 0, st>>>(M, ld, n);
    return cudaGetLastError();
}

cudaError_t launch_zero_below(double *M, int ld, int n, int band, const int *status, cudaStream_t st)
{
    if (n <= band + 1) return cudaSuccess;
    dim3 grid((n + 255) / 256, n);
    k_zero_below<<<grid, 256, 0, st>>>(M, ld, n, band, status);
    return cudaGetLastError();
}

cudaError_t launch_scan_nonfinite(const double *M, int ld, int n, int lower, int which, int *status, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    dim3 grid((n + 255) / 256, n);
    k_scan_nonfinite<<<grid, 256, 0, st>>>(M, ld, n, lower, which, status);
    return cudaGetLastError();
}

}  // namespace hts
