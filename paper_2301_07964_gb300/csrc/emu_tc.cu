// Emulated-FP64 delayed updates of stage 2 (Alg. 4, the "update" tasks) on the fifth-generation
// tensor cores: tcgen05.mma with the accumulators in tensor memory (TMEM), the reflector
// products U_k brought into shared memory by the tensor memory accelerator (TMA).
//
// A tile is 128 lines (rows of X for the right updates and for Q / Z, columns of X for the left
// updates), one per TMEM lane and one per thread of a 128-thread worker.  Per block k, from the
// last to the first, the lines' window of w = r + qg - 1 <= 32 positions (r = 16) is multiplied
// by U_k (w x w, zero padded to 32 x 32) in emulated FP64 (emu_arith.cuh): every line is a
// fixed-point integer with its own power-of-two unit, split into 8 base-256 digits, and the
// 36 digit pairs (i, t) with i + t <= 7 are accumulated per level L = i + t in FP32 (exact:
// every partial sum is an integer below 2^22).  With the 8 digit planes of the lines
// (A_i, 128 x 32 BF16) and U's 8 transposed digit planes stacked along N (B, 32 x 256 BF16),
// one MMA per digit i covers all its levels at once:
//     D[:, 32 i .. 255] += A_i B[:, 0 .. 255 - 32 i]      (M = 128, N = 32 (8 - i), K = 32),
// so a window is 16 tcgen05.mma (two K = 16 steps per digit) into 256 TMEM columns, level L
// at columns 32 L .. 32 L + 31.  The epilogue reads the levels back with tcgen05.ld, combines
// them in 64-bit integer arithmetic, stores the positions that leave the window and keeps the
// w - r overlap positions for the next block; the next window's r new positions are loaded
// while the MMAs run.
//
// Line activity.  Right updates of A and B: a 32-row subtile s takes blocks kmax .. kT_s + 1
// here (every reflector of those blocks is still pending for all its rows) and the staircase
// blocks kT_s .. kstop_s afterwards, reflector by reflector in native FP64 (right_window.cuh),
// as the 32-row tiles of the mma.sync kernel do.  Left updates: column c takes blocks from the
// last one whose cut lies left of c down to 0.  A line loads its whole window when it becomes
// active and stores its whole window after its last block; inactive lines contribute no loads
// and no stores (their rows of A_i are left as they are and their results are discarded).
//
// Block structure: one block per SM (192 KiB of shared memory), two workers of 128 threads with
// their own TMEM columns (2 x 256 of the SM's 512), operand buffers and mbarriers; thread 0 of a
// worker issues its MMAs and TMA copies.  While one worker's MMAs run, the other's epilogue
// does; the workers take tiles from the look-ahead schedule (schedule.cuh).
#include <cuda.h>

#include "emu_arith.cuh"
#include "right_window.cuh"
#include "schedule.cuh"

namespace hts {

using namespace emu;

namespace {

constexpr int kTcLines = 128;                       // lines per tile (MMA M, TMEM lanes)
constexpr int kTcWorkers = 2;                       // tiles in flight per block
constexpr int kTcThreads = 128;                     // threads per worker, one per line
constexpr int kWin = 32;                            // window positions (MMA K)
constexpr int kSlide = 16;                          // r: the window slides by r positions per block
constexpr int kTmemCols = kDigits * kWin;           // 8 levels x 32 positions per tile
constexpr int kDigitPlane = kTcLines * kWin * 2;    // one digit plane of the lines: 8 KiB
constexpr int kUBytes = kDigits * kWin * kWin * 2;  // U's 8 digit planes: 16 KiB
constexpr unsigned kLBO = 128;                      // K-adjacent core matrices
constexpr unsigned kSBO = 512;                      // row-group-adjacent core matrices
// instruction descriptor of kind::f16: D FP32 (bit 4), A and B BF16 (bits 7, 10), both
// K-major, M / 16 at bit 24; N / 8 goes to bit 17
constexpr unsigned kIdescBase = (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(kTcLines >> 4) << 24);

struct TcWorker {
    unsigned char A[kDigits * kDigitPlane];   // digit planes of the lines (64 KiB)
    unsigned char U[2][kUBytes];              // U_k and U_{k-1} (2 x 16 KiB)
};

struct TcShared {
    TcWorker w[kTcWorkers];
    unsigned long long bar_u[kTcWorkers][2];   // TMA of U into buffer b
    unsigned long long bar_d[kTcWorkers];      // the window's MMAs are done
    unsigned tmem_base;
    int slot[kTcWorkers];
    int abort[kTcWorkers];
};

// ---- PTX wrappers -------------------------------------------------------------------------

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// Wait until the phase with parity `parity` of the barrier has completed; false after the
// library's wait limit (2 s or 2^24 polls).
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned parity)
{
    const unsigned a = smem_u32(bar);
    const unsigned long long t0 = globaltimer_ns();
    for (long long it = 0;; ++it) {
        unsigned ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(a), "r"(parity)
            : "memory");
        if (ok) return true;
        if (it > kSpinLimit || globaltimer_ns() - t0 > kWaitLimitNs) return false;
    }
}

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int c0, int c1, int c2,
                                            unsigned long long *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(smem_u32(dst)), "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Shared memory descriptor of a K-major operand without swizzle (start address, LBO, SBO in
// units of 16 bytes; bit 46 is the descriptor version of this architecture).
__device__ __forceinline__ unsigned long long smem_desc(unsigned addr)
{
    return (unsigned long long)((addr & 0x3FFFFu) >> 4) | ((unsigned long long)(kLBO >> 4) << 16) |
           ((unsigned long long)(kSBO >> 4) << 32) | (1ull << 46);
}

__device__ __forceinline__ void tc_mma(unsigned dtmem, unsigned long long adesc, unsigned long long bdesc,
                                       unsigned idesc, int accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\ttcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(dtmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void tc_commit(unsigned long long *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// The 8 levels of 8 consecutive positions (TMEM columns 32 L + c0 .. 32 L + c0 + 7 of the
// warp's 32 lanes) in one statement together with the wait for them: tcgen05.ld writes its
// registers asynchronously, so nothing may read (or move) them before tcgen05.wait::ld, and
// keeping both in one asm statement leaves the compiler no room to do so.  The memory clobber
// keeps the statement after the MMA-completion wait and the thread-sync fence before it.
__device__ __forceinline__ void tc_ld_levels(unsigned taddr, unsigned (&v)[kDigits][8])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%64];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%8, %9, %10, %11, %12, %13, %14, %15}, [%65];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%16, %17, %18, %19, %20, %21, %22, %23}, [%66];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%24, %25, %26, %27, %28, %29, %30, %31}, [%67];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%32, %33, %34, %35, %36, %37, %38, %39}, [%68];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%40, %41, %42, %43, %44, %45, %46, %47}, [%69];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%48, %49, %50, %51, %52, %53, %54, %55}, [%70];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%56, %57, %58, %59, %60, %61, %62, %63}, [%71];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(v[0][0]), "=r"(v[0][1]), "=r"(v[0][2]), "=r"(v[0][3]), "=r"(v[0][4]), "=r"(v[0][5]), "=r"(v[0][6]),
          "=r"(v[0][7]), "=r"(v[1][0]), "=r"(v[1][1]), "=r"(v[1][2]), "=r"(v[1][3]), "=r"(v[1][4]), "=r"(v[1][5]),
          "=r"(v[1][6]), "=r"(v[1][7]), "=r"(v[2][0]), "=r"(v[2][1]), "=r"(v[2][2]), "=r"(v[2][3]), "=r"(v[2][4]),
          "=r"(v[2][5]), "=r"(v[2][6]), "=r"(v[2][7]), "=r"(v[3][0]), "=r"(v[3][1]), "=r"(v[3][2]), "=r"(v[3][3]),
          "=r"(v[3][4]), "=r"(v[3][5]), "=r"(v[3][6]), "=r"(v[3][7]), "=r"(v[4][0]), "=r"(v[4][1]), "=r"(v[4][2]),
          "=r"(v[4][3]), "=r"(v[4][4]), "=r"(v[4][5]), "=r"(v[4][6]), "=r"(v[4][7]), "=r"(v[5][0]), "=r"(v[5][1]),
          "=r"(v[5][2]), "=r"(v[5][3]), "=r"(v[5][4]), "=r"(v[5][5]), "=r"(v[5][6]), "=r"(v[5][7]), "=r"(v[6][0]),
          "=r"(v[6][1]), "=r"(v[6][2]), "=r"(v[6][3]), "=r"(v[6][4]), "=r"(v[6][5]), "=r"(v[6][6]), "=r"(v[6][7]),
          "=r"(v[7][0]), "=r"(v[7][1]), "=r"(v[7][2]), "=r"(v[7][3]), "=r"(v[7][4]), "=r"(v[7][5]), "=r"(v[7][6]),
          "=r"(v[7][7])
        : "r"(taddr), "r"(taddr + kWin), "r"(taddr + 2 * kWin), "r"(taddr + 3 * kWin), "r"(taddr + 4 * kWin),
          "r"(taddr + 5 * kWin), "r"(taddr + 6 * kWin), "r"(taddr + 7 * kWin)
        : "memory");
}

// Byte offset of (row m, k) in a K-major core-matrix layout with K = 32.
__device__ __forceinline__ unsigned kmaj_off(int m, int k)
{
    return (unsigned)((m >> 3) * kSBO + (k >> 3) * kLBO + (m & 7) * 16 + (k & 7) * 2);
}

// Per-worker pipeline state (the same in every thread of the worker).
struct TcPhase {
    unsigned u[2];   // parity of the next phase of bar_u[b]
    unsigned d;      // parity of the next phase of bar_d
};

// Arguments of one tile: the matrix, its kind (0, 1 right A / B; 2, 3 Z / Q; 4, 5 left A / B),
// the group and the tensor map of its U planes.
struct TcTile {
    double *X;
    size_t ld;
    int kind, n, r, j1, qg;
    const CUtensorMap *map;
    ReflectorSet R;
};

// Window position p of line `line` at block k: its matrix element.
__device__ __forceinline__ double *elem(const TcTile &t, int line, int pos)
{
    return (t.kind >= 4) ? t.X + (size_t)(pos - 1) + (size_t)(line - 1) * t.ld
                         : t.X + (size_t)(line - 1) + (size_t)(pos - 1) * t.ld;
}

// One tile of 128 lines by one worker (tid = 0 .. 127, barrier wb).
__device__ void tc_tile(const TcTile &t, int tile, TcWorker &W, unsigned long long *bar_u, unsigned long long *bar_d,
                        unsigned tmem, int *abort, TcPhase &ph, int tid, int wb, int *status)
{
    constexpr int r = kSlide;   // the launcher admits r = 16 only
    const int n = t.n, j1 = t.j1, qg = t.qg;
    const int w = r + qg - 1;
    const int jl = j1 + qg - 1;
    const int kmax = nblocks_gen(n, r, j1) - 1;
    const int l0 = tile * kTcLines + 1;
    if (l0 > n || kmax < 0) return;
    const int lastline = imin(l0 + kTcLines - 1, n);
    const int line = l0 + tid;
    const bool lvalid = line <= n;
    const bool left = t.kind >= 4;
    const bool ab_right = t.kind <= 1;

    // blocks this line takes here: khi .. klo (khi < klo: none)
    int khi = kmax, klo = 0;
    int K_hi = kmax, K_lo = 0;   // the tile's range (uniform)
    if (ab_right) {
        auto kT_of = [&](int s) {
            const int llast = imin(l0 + 32 * s + 31, n);
            return (llast <= j1) ? -1 : qg + (llast - j1 - 1) / r;
        };
        klo = kT_of(tid >> 5) + 1;
        K_lo = kT_of(0) + 1;
    } else if (left) {
        // column c takes the blocks whose cut lies left of it: k <= khi(c), the cut rising with k
        const int isB = t.kind == 5;
        auto khi_of = [&](int c) {
            int kk = kmax;
            while (kk >= 0 && left_cut_of(isB, n, r, jl, kk) >= c) --kk;
            return kk;
        };
        khi = khi_of(line);
        K_hi = khi_of(lastline);
    }
    if (!lvalid) { khi = -1; klo = 0; }

    if (K_hi >= K_lo && K_hi >= 0) {
        const int wq = (tid >> 5);   // warp of the worker = TMEM lane quarter
        const unsigned tl = tmem + ((unsigned)(32 * wq) << 16);
        int buf = 0;
        // U of the first block
        if (tid == 0) {
            mbar_expect_tx(&bar_u[buf], kUBytes);
            tma_load_3d(W.U[buf], t.map, 0, 0, K_hi, &bar_u[buf]);
        }
        double fresh[kWin];
        long long carry[16];
        int cu = 0;
        bool bad = false;                 // this thread met a wait that ran out
        int u_pend = buf;                 // buffer with a TMA copy in flight (thread 0), or -1
        unsigned u_par = ph.u[buf];       // the phase that copy completes
#pragma unroll
        for (int p = 0; p < kWin; ++p) fresh[p] = 0.0;
#pragma unroll
        for (int p = 0; p < 16; ++p) carry[p] = 0;
        // first window's data of the lines active at K_hi
        if (K_hi <= khi && K_hi >= klo) {
            const int c0 = j1 + K_hi * r + 1;
#pragma unroll
            for (int p = 0; p < kWin; ++p)
                if (p < (K_hi == khi ? w : r) && c0 + p <= n) fresh[p] = *elem(t, line, c0 + p);
        }

        for (int k = K_hi; k >= K_lo; --k) {
            const bool act = k <= khi && k >= klo;
            const bool first = k == khi;
            const bool last = k == klo;
            const int c0 = j1 + k * r + 1;
            int ua = 0;
            if (act) {
                // the window's unit: 2^(ua + 62) above its largest entry
                int em = kZeroExp;
#pragma unroll
                for (int p = 0; p < kWin; ++p) {
                    if (p < w) {
                        if (first || p < r) em = imax(em, exp_of_f64(fresh[p]));
                        else em = imax(em, exp_of_fixed(carry[(p - r) & 15], cu));
                    }
                }
                ua = (em == kZeroExp ? 0 : em + 2) - 64;
                // digit planes of this line (row tid of A_i)
#pragma unroll
                for (int c = 0; c < kWin / 8; ++c) {
                    unsigned dg[8][kDigits];
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const int p = 8 * c + j;
                        long long x = 0;
                        if (p < w) x = (first || p < r) ? f64_to_fixed(fresh[p], ua) : refix(carry[(p - r) & 15], cu, ua);
                        digits_bf16(x, dg[j]);
                    }
#pragma unroll
                    for (int i = 0; i < kDigits; ++i) {
                        const uint4 v = make_uint4(pack_bf16(dg[0][i], dg[1][i]), pack_bf16(dg[2][i], dg[3][i]),
                                                   pack_bf16(dg[4][i], dg[5][i]), pack_bf16(dg[6][i], dg[7][i]));
                        *reinterpret_cast<uint4 *>(W.A + i * kDigitPlane + kmaj_off(tid, 8 * c)) = v;
                    }
                }
            }
            fence_async_smem();
            tc_fence_before();
            if (group_sync_or(wb, kTcThreads, bad)) {
                bad = true;
                break;
            }
            if (tid == 0) {
                tc_fence_after();
                if (!mbar_wait(&bar_u[buf], ph.u[buf])) {
                    record_error(status, HTS_ERR_TIMEOUT, 0, -2, k, tile);
                    bad = true;
                    tc_commit(bar_d);   // no MMAs: the others' wait ends, the tile stops next
                } else {
                    u_pend = -1;
                    const unsigned a0 = smem_u32(W.A), b0 = smem_u32(W.U[buf]);
#pragma unroll
                    for (int i = 0; i < kDigits; ++i) {
                        const unsigned idesc = kIdescBase | ((unsigned)((kWin * (kDigits - i)) >> 3) << 17);
#pragma unroll
                        for (int kk = 0; kk < 2; ++kk)
                            tc_mma(tmem + kWin * i, smem_desc(a0 + i * kDigitPlane + kk * 2 * kLBO),
                                   smem_desc(b0 + kk * 2 * kLBO), idesc, (i > 0 || kk > 0) ? 1 : 0);
                    }
                    tc_commit(bar_d);
                    // U of the next block into the other buffer (its last reader, the previous
                    // window's MMAs, has completed)
                    if (k - 1 >= K_lo) {
                        mbar_expect_tx(&bar_u[buf ^ 1], kUBytes);
                        tma_load_3d(W.U[buf ^ 1], t.map, 0, 0, k - 1, &bar_u[buf ^ 1]);
                        u_pend = buf ^ 1;
                        u_par = ph.u[buf ^ 1];
                    }
                }
            }
            ph.u[buf] ^= 1u;
            buf ^= 1;
            // the next window's new positions, while the MMAs run (this window's are consumed)
            const int kn = k - 1;
#pragma unroll
            for (int p = 0; p < kWin; ++p) fresh[p] = 0.0;
            if (kn >= K_lo && kn <= khi && kn >= klo) {
                const int cn = j1 + kn * r + 1;
                const int cnt = (kn == khi) ? w : r;
#pragma unroll
                for (int p = 0; p < kWin; ++p)
                    if (p < cnt && cn + p <= n) fresh[p] = *elem(t, line, cn + p);
            }
            if (!mbar_wait(bar_d, ph.d)) {
                record_error(status, HTS_ERR_TIMEOUT, 0, -3, k, tile);
                bad = true;
            }
            ph.d ^= 1u;
            tc_fence_after();
            // levels -> results, 8 positions at a time; positions that leave the window are
            // stored, the overlap is kept
            const int cu_new = ua + 3;
#pragma unroll
            for (int c = 0; c < kWin / 8; ++c) {
                unsigned lv[kDigits][8];
                tc_ld_levels(tl + 8 * c, lv);
                if (act) {
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const int p = 8 * c + j;
                        if (p < w) {
                            const long long v = combine_levels(
                                __uint_as_float(lv[0][j]), __uint_as_float(lv[1][j]), __uint_as_float(lv[2][j]),
                                __uint_as_float(lv[3][j]), __uint_as_float(lv[4][j]), __uint_as_float(lv[5][j]),
                                __uint_as_float(lv[6][j]), __uint_as_float(lv[7][j]));
                            if (last || p >= w - r) {
                                if (c0 + p <= n) *elem(t, line, c0 + p) = fixed_to_f64(v, cu_new);
                            }
                            if (p < w - r) carry[p & 15] = v;
                        }
                    }
                }
            }
            if (act) cu = cu_new;
            tc_fence_before();
        }
        if (group_sync_or(wb, kTcThreads, bad)) {
            // stop the tile: let a copy into U that is still in flight land (bounded) before
            // the buffer is reused or the block exits, and the other tiles of this worker end
            if (tid == 0) {
                if (u_pend >= 0 && !mbar_wait(&bar_u[u_pend], u_par)) record_error(status, HTS_ERR_TIMEOUT, 0, -4, 0, tile);
                *(volatile int *)abort = 1;
            }
            group_sync(wb, kTcThreads);
            return;
        }
    }

    // staircase blocks of the right updates of A and B, per 32-row subtile, in native FP64
    if (ab_right && !*(volatile int *)abort) {
        for (int s = 0; s < kTcLines / 32; ++s) {
            const int x0 = l0 + 32 * s;
            if (x0 > n) break;
            const int llast = imin(x0 + 31, n);
            const int kT = (llast <= j1) ? -1 : qg + (llast - j1 - 1) / r;
            const int skstart = imin(kT, kmax);
            const int skstop = (x0 <= j1) ? 0 : (x0 - j1 - 1) / r + 2;
            if (skstop <= skstart)
                right_window_rows<kTcThreads>(t.X, (int)t.ld, t.kind, t.R.VZ, t.R.TZ, t.R.kdim, n, r, j1, qg, x0,
                                              skstart, skstop, reinterpret_cast<double *>(W.A), tid, wb);
            group_sync(wb, kTcThreads);
        }
    }
}

}  // namespace

// ---------------------------------------------------------------------------------------
// Persistent look-ahead update launch on the tensor cores (schedule.cuh): one block per SM,
// two workers taking 128-line tiles in ticket order.
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kTcThreads * kTcWorkers, 1) k_s2_update_tc(const __grid_constant__ UpdTcArgs a)
{
    extern __shared__ __align__(1024) unsigned char tc_smem_raw[];
    // operand buffers on a 1 KiB boundary (TMA destinations need 128 bytes)
    TcShared &S = *reinterpret_cast<TcShared *>(tc_smem_raw + ((1024u - (smem_u32(tc_smem_raw) & 1023u)) & 1023u));
    const int worker = threadIdx.x / kTcThreads, tid = threadIdx.x % kTcThreads;
    if (threadIdx.x < 32) {
        // all 512 TMEM columns: one block per SM (its shared memory excludes a second)
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&S.tmem_base)),
                     "r"(kTmemCols * kTcWorkers)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 0) {
        for (int wk = 0; wk < kTcWorkers; ++wk) {
            mbar_init(&S.bar_u[wk][0], 1);
            mbar_init(&S.bar_u[wk][1], 1);
            mbar_init(&S.bar_d[wk], 1);
            S.abort[wk] = 0;
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tmem = S.tmem_base + (unsigned)(worker * kTmemCols);
    TcWorker &W = S.w[worker];
    TcPhase ph;
    ph.u[0] = ph.u[1] = 0;
    ph.d = 0;
    const int wb = 1 + worker;
    update_worker<kTcThreads>(a.s, tid, wb, &S.slot[worker], [&](const Task &T) {
        // an empty slot of the ticket layout (a row of the plan without this kind of tile)
        if (S.abort[worker] || T.kind == kTaskNone) return;
        TcTile tt;
        if (T.kind == kTaskQZ) {
            tt.X = a.qz.M[T.mat]; tt.ld = (size_t)a.qz.ld[T.mat]; tt.kind = a.qz.kind[T.mat];
            tt.n = a.qz.n; tt.r = a.qz.r; tt.j1 = a.qz.j1; tt.qg = a.qz.qg; tt.R = a.qz.R;
            tt.map = tt.kind == 3 ? &a.map_qz_q : &a.map_qz_z;
        } else {
            const EmuArgs &e = (T.kind == kTaskRight) ? a.right : a.left;
            tt.X = e.M[T.mat]; tt.ld = (size_t)e.ld[T.mat]; tt.kind = e.kind[T.mat];
            tt.n = e.n; tt.r = e.r; tt.j1 = e.j1; tt.qg = e.qg; tt.R = e.R;
            tt.map = (T.kind == kTaskRight) ? &a.map_z : &a.map_q;
        }
        tc_tile(tt, T.tile, W, S.bar_u[worker], &S.bar_d[worker], tmem, &S.abort[worker], ph, tid, wb, a.s.status);
    });
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (threadIdx.x < 32)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(S.tmem_base), "r"(kTmemCols * kTcWorkers)
                     : "memory");
}

// ---------------------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------------------
namespace {

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

}  // namespace

int update_tc_workers() { return kTcWorkers; }
int update_tc_lines() { return kTcLines; }
bool update_tc_supported(int r, int qg) { return r == kSlide && qg >= 1 && r + qg - 1 <= kWin; }

// Tensor map of one plane set: kdim blocks of U_k, each 32 rows of 256 BF16 (16 KiB).
cudaError_t encode_plane_map(CUtensorMap *map, const void *planes, int kdim)
{
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return cudaErrorNotSupported;
    const cuuint64_t dims[3] = {256, 32, (cuuint64_t)kdim};
    const cuuint64_t strides[2] = {512, (cuuint64_t)kUBytes};
    const cuuint32_t box[3] = {256, 32, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void *>(planes), dims, strides, box,
                           estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t launch_s2_update_tc(const UpdTcArgs &a, int ctas, cudaStream_t st)
{
    const int sm = (int)sizeof(TcShared) + 1024;   // room to align the base to 1 KiB
    cudaError_t e = cudaFuncSetAttribute(k_s2_update_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    if (e != cudaSuccess) return e;
    k_s2_update_tc<<<ctas, kTcThreads * kTcWorkers, sm, st>>>(a);
    return cudaGetLastError();
}

}  // namespace hts
