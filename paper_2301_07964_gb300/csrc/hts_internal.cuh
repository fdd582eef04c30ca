// Internal definitions shared by the stage-2 kernels and the C-ABI layer.
//
// Index convention: the paper's 1-based (row, column) indices are used throughout the
// scheduling code; AT() converts to a column-major offset.
#pragma once

#include <cublas_v2.h>
#include <cuda.h>   // CUtensorMap (the encoder is resolved at run time; no link to the driver library)
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/hts.h"
#include "../../include/hts_profile.h"

// Per-launch CUDA-event records of the optional profiler (include/hts_profile.h).
struct hts_prof_state {
    int enabled;
    int cap, used, dropped;
    cudaEvent_t *ev;     // 2 * cap events: start, end of launch i
    int *kind;
    double *flops, *bytes, *mma;
};

struct hts_ctx {
    int device;
    int *d_status;   // device status word: [0] code, [1..4] {pencil, group, k, j}
    int *h_status;   // pinned host mirror used by hts_sync_status
    hts_prof_state prof;
    // Streams beside the caller's (created once by hts_create): `upd` carries the look-ahead
    // update launches, `side` the Q / Z updates of the serial schedule; events order them
    // against the caller's stream, one per reflector set.
    cudaStream_t side, upd;
    cudaEvent_t ev_gen[3];   // reflector set s written (generate and block formation done)
    cudaEvent_t ev_qz[3];    // serial schedule: set s no longer read by its Q / Z update
    cudaEvent_t ev_upd[3];   // look-ahead: update launch u (u mod 3) finished
    int num_sms;
    int batch_per_sm;        // blocks per SM of the planned batched launches (0: as many as fit)
    cublasHandle_t blas;     // the WY products of stages 0 and 1 (plain DGEMMs)
};

namespace hts {

constexpr int kStatusWords = 8;
constexpr int kStatusFallbacks = 5;  // status word slot: opposite-reflector steps redone with the RQ
constexpr int kMaxR = 32;            // reflector length limit of the warp-level chase
constexpr int kGenThreads = 256;     // threads of one generate (chase) block
constexpr int kApplyThreads = 64;    // threads (rows or columns) of one apply block
constexpr long long kSpinLimit = 1LL << 24;   // bounded waits: polls before giving up
constexpr unsigned long long kWaitLimitNs = 2000000000ULL;   // ... or 2 s of wall clock

__host__ __device__ __forceinline__ int imin(int a, int b) { return a < b ? a : b; }
__host__ __device__ __forceinline__ int imax(int a, int b) { return a > b ? a : b; }

__host__ __device__ __forceinline__ size_t AT(int ld, int i, int j)
{
    return (size_t)(i - 1) + (size_t)(j - 1) * (size_t)ld;
}

// Number of blocks of sweep j that carry reflectors (Alg. 2: 1 + floor((n-j-2)/r)).
__host__ __device__ __forceinline__ int nblocks_gen(int n, int r, int j)
{
    return (n - j - 2 >= 0) ? 1 + (n - j - 2) / r : 0;
}

// Number of blocks of sweep j visited by the generate phase (Alg. 3: 2 + floor((n-j-1)/r)).
// The blocks beyond nblocks_gen only receive the lazy left updates of their pivot column.
__host__ __device__ __forceinline__ int nblocks_lazy(int n, int r, int j)
{
    return 2 + (n - j - 1) / r;
}

// Index ranges of step (k, j) inside the group that starts at sweep j1 and has qg sweeps.
//  jb: pivot column; i1..i2: rows of the left reflector and columns of the right one;
//  i3: last row of A the right reflector touches (Alg. 2); i4: first row of the band that
//  the generate phase updates.  i4 follows the row-range derivation of the text
//  (j1 + 1 + max(0, (k + j - j1 - q) r)); Alg. 3 prints a value 2r larger, which leaves
//  rows of the B block without the preceding right reflector when its opposite reflector is formed.
struct StepGeom {
    int jb, i1, i2, i3, i4;
};

__host__ __device__ __forceinline__ StepGeom step_geom(int n, int r, int j1, int qg, int k, int j)
{
    StepGeom g;
    g.jb = j + imax(0, (k - 1) * r + 1);
    g.i1 = j + k * r + 1;
    g.i2 = imin(j + (k + 1) * r, n);
    g.i3 = imin(j + (k + 2) * r, n);
    g.i4 = j1 + 1 + imax(0, (k + j - j1 - qg) * r);
    return g;
}

// Reflector storage for one group: slot s = j - j1, block k.
//   V[(s * kdim + k) * r + i], i < r (v[0] = 1 stored explicitly, zero padded)
//   T[s * kdim + k]            (tau = 0: no reflector / identity)
struct ReflectorSet {
    double *VQ, *TQ, *VZ, *TZ;
    int kdim;
};

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_u64(unsigned long long *p, unsigned long long v)
{
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Record the first device-side error; later errors are dropped.
__device__ __forceinline__ void record_error(int *status, int code, int a, int b, int c, int d)
{
    if (atomicCAS(status, 0, code) == 0) {
        status[1] = a;
        status[2] = b;
        status[3] = c;
        status[4] = d;
        __threadfence();
    }
}

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double warp_max(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Householder reflector in the LAPACK dlarfg convention, computed by one full warp.
// Lane i holds x_i for i < m (x_0 = alpha), garbage-free zero elsewhere.  Returns tau and
// sets *beta and v_i (v_0 = 1) in the calling lane's register.  tau = 0 when x_2..x_m = 0.
// The sum of squares is formed directly and recomputed with scaling only when it
// over- or underflows.
__device__ __forceinline__ double warp_larfg(double xi, int m, int lane, double *beta, double *vi)
{
    double alpha = __shfl_sync(0xffffffffu, xi, 0);
    double t = (lane >= 1 && lane < m) ? xi : 0.0;
    double ssq = warp_sum(t * t);
    double xnorm2 = ssq;
    double scale = 1.0;
    if (!(ssq >= 1e-290 && ssq <= 1e290) || fabs(alpha) > 1e145) {
        double mx = warp_max(fabs(t));
        mx = fmax(mx, fabs(alpha));
        if (mx == 0.0) {
            *beta = alpha;
            *vi = (lane == 0) ? 1.0 : 0.0;
            return 0.0;
        }
        scale = mx;
        double ts = t / mx;
        xnorm2 = warp_sum(ts * ts);
    }
    if (xnorm2 == 0.0) {
        *beta = alpha;
        *vi = (lane == 0) ? 1.0 : 0.0;
        return 0.0;
    }
    double as = alpha / scale;
    double nrm = scale * sqrt(as * as + xnorm2);
    double b = (alpha >= 0.0) ? -nrm : nrm;
    double tau = (b - alpha) / b;
    double sc = 1.0 / (alpha - b);
    *beta = b;
    *vi = (lane == 0) ? 1.0 : ((lane < m) ? xi * sc : 0.0);
    return tau;
}

// Barrier of a group of nthreads threads: a whole block with id 0 (nthreads = its size), or
// one worker of a persistent block with its own id.
__device__ __forceinline__ void group_sync(int id, int nthreads)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// The same barrier, returning whether any thread of the group passed v = true: a decision
// (stop, skip) that every thread of the group takes alike.
__device__ __forceinline__ bool group_sync_or(int id, int nthreads, bool v)
{
    int any;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.b32 p, %1, 0;\n\tbar.red.or.pred q, %2, %3, p;\n\tselp.s32 %0, 1, 0, q;\n\t}"
        : "=r"(any)
        : "r"(v ? 1 : 0), "r"(id), "r"(nthreads)
        : "memory");
    return any != 0;
}

// Brackets one kernel launch with profiler events when profiling is on (profile.cu).
struct ProfScope {
    hts_ctx *ctx;
    cudaStream_t st;
    int idx;
    ProfScope(hts_ctx *c, cudaStream_t s);
    void done(int kind, double flops, double bytes, double mma_flops = 0.0);
};


// Task layout of one update launch: the A / B updates of a group (if ab) and the Q / Z update of
// the group before it (nqz matrices).  Tickets 0 .. 4U-1 form U slots {right A, right B, left A,
// left B}: slot u holds right tile T0+u and left tiles Cs[m]+u-D[m], so that a left tile comes
// after the right tiles it waits for.  Then the right tiles 0 .. T0-1 of A and B, then the Q / Z
// tiles.
struct TaskPlan {
    int TL;         // lines per tile (rows of a right tile, columns of a left one)
    int ntiles;     // tiles of TL lines covering n
    int ab;         // the launch carries a group's A / B updates
    int T0, Tend;   // right tiles T0 .. Tend: rows below j1 that still need blocks of the group
    int Cs[2], Ce;  // left tiles Cs[m] .. Ce of A (m = 0) and B (m = 1) with work
    int D[2];       // slot lag of the left tiles
    int U;          // slots
    int nrect;      // right tiles above the group (A and B)
    int nqz;        // matrices of the Q / Z update (0, 1 or 2)
    int total;      // tasks
};

// Arguments of the stage-2 launches (kernels in stage2.cu).
struct GenArgs {
    double *A;
    double *B;
    int lda, ldb;
    int n, r, j1, qg, group;
    ReflectorSet R;
    unsigned long long *flags;   // progress words: [0, qmax) main blocks, [qmax, 2 qmax) helpers
    int qmax;
    double *gram;                // tau_b u_a.u_b of the group's left reflectors per block:
                                 // gram[(k * qmax + a) * qmax + b], a < b (written by helpers)
    unsigned long long epoch;    // (group + 1) << 32
    int *status;
    int stall;                   // fault injection: slot 0 never publishes (tests only)
    int direct_rq;               // tests: the r <= 16 chase takes every direction from the RQ
    // look-ahead: the previous group's update launch runs beside this chase; each step waits
    // for the tiles of A and B it touches (uflags null: nothing to wait for)
    const unsigned long long *uflags;
    TaskPlan uplan;
    unsigned long long uepoch;
};

// kind 0 = A, 1 = B (Z^ reflectors on rows x < i4(k, j)), 2 = Z (Z^, all rows),
// 3 = Q (Q^, all rows)
struct ApplyArgs {
    double *M[4];
    int ld[4];
    int kind[4];
    int n, r, j1, qg;
    ReflectorSet R;
    const int *status;
};

// Block formation (emu.cu): the products U^Q_k, U^Z_k of a group's reflectors per block k,
// stored as BF16 digit planes.
struct FormUArgs {
    int n, r, j1, qg;
    ReflectorSet R;
    uint2 *planesQ, *planesZ;
    const int *status;
    int umma;   // plane layout: 0 = mma.sync B fragments (emu.cu), 1 = tcgen05 operand (emu_tc.cu)
};

// Emulated delayed updates (emu.cu).  kind 0 = A rows, 1 = B rows (the staircase blocks of
// each tile in native FP64 from the reflectors in R), 2 = Z rows, 3 = Q rows, 4 = A columns,
// 5 = B columns (left updates).
struct EmuArgs {
    double *M[4];
    int ld[4];
    int kind[4];
    int n, r, j1, qg;
    const uint2 *planesQ, *planesZ;
    ReflectorSet R;
    const int *status;
};

// Look-ahead update launch (schedule.cuh): the tasks of one group's A / B updates and of the
// previous group's Q / Z update, the tile flags they publish and the launch's ticket counter.
struct UpdSched {
    TaskPlan P;
    unsigned long long *tflags;   // 4 * P.ntiles words (see tile_flag)
    unsigned long long epoch;     // published value: this group's index + 1
    unsigned *ticket;
    int *status;
    int group, n, r;
};

struct LeftArgs {
    double *A;
    double *B;
    int lda, ldb;
    int n, r, j1, qg;
    ReflectorSet R;
    const int *status;
};

cudaError_t launch_s2_generate(const GenArgs &a, cudaStream_t st);
cudaError_t launch_s2_chase16(const GenArgs &a, cudaStream_t st);
cudaError_t launch_s2_form_u(const FormUArgs &a, cudaStream_t st);
cudaError_t launch_s2_emu_apply(const EmuArgs &a, int nmat, cudaStream_t st);
size_t emu_plane_bytes(int kdim);
bool emu_supported(int r, int qg);
cudaError_t launch_s2_apply_right(const ApplyArgs &a, int nmat, cudaStream_t st);
// Look-ahead update launches: `ab` carries A (M[0], kind 0 / 4) and B (M[1], kind 1 / 5) of the
// group, `qz` the previous group's Q / Z; `ctas` persistent blocks.
struct UpdEmuArgs {
    EmuArgs right, left, qz;
    UpdSched s;
};
cudaError_t launch_s2_update_emu(const UpdEmuArgs &a, int ctas, cudaStream_t st);
struct UpdFp64Args {
    ApplyArgs right, qz;
    LeftArgs left;
    UpdSched s;
    int smem_doubles;   // shared memory of one worker
};
int update_fp64_smem_doubles(int r, int qg);
// tcgen05 update launch (emu_tc.cu): A / B of the group with the tensor maps of its U planes,
// Q / Z of the previous group with its own.
struct UpdTcArgs {
    CUtensorMap map_z, map_q, map_qz_z, map_qz_q;
    EmuArgs right, left, qz;
    UpdSched s;
};
cudaError_t launch_s2_update_tc(const UpdTcArgs &a, int ctas, cudaStream_t st);
cudaError_t encode_plane_map(CUtensorMap *map, const void *planes, int kdim);
int update_tc_workers();
int update_tc_lines();
bool update_tc_supported(int r, int qg);
int update_fp64_workers();
int update_emu_workers();
cudaError_t launch_s2_update_fp64(const UpdFp64Args &a, int ctas, cudaStream_t st);
cudaError_t launch_s2_apply_left(const LeftArgs &a, cudaStream_t st);
cudaError_t launch_set_identity(double *M, int ld, int n, cudaStream_t st);
cudaError_t launch_zero_below(double *M, int ld, int n, int band, const int *status, cudaStream_t st);
cudaError_t launch_scan_nonfinite(const double *M, int ld, int n, int lower, int which, int *status, cudaStream_t st);

// Batched reduction (batch.cu): the workspace holds a head, the queue counter, the
// descriptors and the largest-first order; batch_stage writes that image in host memory.
size_t batch_work_bytes(int count);
void batch_stage(void *host, int count, const int *n, const int *r, double *const *A, const int *lda,
                 double *const *B, const int *ldb, double *const *Q, const int *ldq, double *const *Z, const int *ldz,
                 int compq, int compz, int p);
cudaError_t launch_reduce_batched(void *work, int count, int num_sms, int per_sm, int *status, cudaStream_t st);
int batch_max_n();
int batch_max_block();

// Stages 0 and 1 (stage01.cu) and workspace sizes.
size_t stage01_workspace_bytes(int n, int r, int p);
size_t stage2_workspace_bytes(int n, int r);
size_t stage2_workspace_bytes_mode(int n, int r, hts_gemm_mode mode);
cudaError_t run_stage0(cublasHandle_t blas, int n, double *A, int lda, double *B, int ldb, double *Q, int ldq, void *work, int r, int p,
                       cudaStream_t st);
cudaError_t run_stage1(cublasHandle_t blas, int n, int nb, int p, double *A, int lda, double *B, int ldb, double *Q, int ldq,
                       double *Z, int ldz, void *work, cudaStream_t st);

// Same reflector as warp_larfg with one reciprocal square root and one reciprocal on the
// dependent path: with rs = 1/||x||, beta = -sign(alpha) ||x||, tau = 1 + |alpha| rs and
// v_i = x_i sign(alpha) rs / tau.  Falls back to the scaled form when the sum of squares
// leaves the safe range.
__device__ __forceinline__ double warp_larfg_fast(double xi, int m, int lane, double *beta, double *vi)
{
    const double alpha = __shfl_sync(0xffffffffu, xi, 0);
    const double t = (lane >= 1 && lane < m) ? xi : 0.0;
    const double ssq = warp_sum(t * t);
    if (ssq == 0.0) {
        *beta = alpha;
        *vi = (lane == 0) ? 1.0 : 0.0;
        return 0.0;
    }
    if (!(ssq >= 1e-290 && ssq <= 1e290) || fabs(alpha) > 1e145) return warp_larfg(xi, m, lane, beta, vi);
    const double nrm2 = fma(alpha, alpha, ssq);
    const double rs = rsqrt(nrm2);
    const double sa = alpha >= 0.0 ? 1.0 : -1.0;
    const double tau = fma(fabs(alpha), rs, 1.0);
    *beta = -sa * (nrm2 * rs);
    const double sc = sa * rs * __drcp_rn(tau);
    *vi = (lane == 0) ? 1.0 : ((lane < m) ? xi * sc : 0.0);
    return tau;
}

__device__ __forceinline__ unsigned long long globaltimer_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait (one thread) until *flag >= need; on expiry records HTS_ERR_TIMEOUT.  Gives up
// at once (without recording) when another block has recorded an error, since the flag may
// then never be set.
__device__ __forceinline__ bool wait_at_least(const unsigned long long *flag, unsigned long long need, int *status, int group, int k,
                              int j)
{
    const unsigned long long t0 = globaltimer_ns();
    long long polls = 0;
    while (ld_acquire_u64(flag) < need) {
        ++polls;
        if ((polls & 255) == 0 && *(volatile int *)status != 0) return false;
        if (polls > kSpinLimit || globaltimer_ns() - t0 > kWaitLimitNs) {
            record_error(status, HTS_ERR_TIMEOUT, 0, group, k, j);
            return false;
        }
    }
    return true;
}

// Rows x0 .. x0+na-1 of A and x0 .. x0+nbr-1 of B, columns i1 .. i1+m-1, times Z^ = I - tz v v^T
// (one thread per row).  zero_first: B(x, i1) := 0 exactly for x > i1 (the reduced column).
__device__ __forceinline__ void band_rows(double *A, int lda, double *B, int ldb, int x0, int na, int nbr, int i1, int m, double tz,
                          const double *vv, bool zero_first)
{
    for (int t = threadIdx.x; t < na + nbr; t += kGenThreads) {
        const bool isA = t < na;
        const int x = x0 + (isA ? t : t - na);
        double *base = isA ? A : B;
        const int ld = isA ? lda : ldb;
        double rowv[kMaxR];
        double d0 = 0.0, d1 = 0.0;
#pragma unroll
        for (int c = 0; c < kMaxR; ++c) {
            if (c < m) {
                rowv[c] = __ldcg(base + AT(ld, x, i1 + c));
                if (c & 1) d1 += rowv[c] * vv[c];
                else d0 += rowv[c] * vv[c];
            }
        }
        const double d = (d0 + d1) * tz;
#pragma unroll
        for (int c = 0; c < kMaxR; ++c) {
            if (c < m) {
                double val = rowv[c] - d * vv[c];
                if (zero_first && !isA && c == 0 && x > i1) val = 0.0;
                base[AT(ld, x, i1 + c)] = val;
            }
        }
    }
}


}  // namespace hts
