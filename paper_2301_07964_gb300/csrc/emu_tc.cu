// Emulated-FP64 delayed updates of stage 2 (Alg. 4, the "update" tasks) on the fifth-generation
// tensor cores: tcgen05.mma with the accumulators in tensor memory (TMEM), the reflector
// products U_k brought into shared memory by the tensor memory accelerator (TMA).
//
// A tile is 64 lines (rows of X for the right updates and for Q / Z, columns of X for the left
// updates), each in two MMA rows (TMEM lanes l and l + 64).  Per block k, from the last to
// the first, the lines' window of
// w = r + qg - 1 <= 32 positions (r = 16) is multiplied by U_k (w x w, zero padded to 32 x 32)
// in emulated FP64 (emu_arith.cuh): every line is a fixed-point integer with its own
// power-of-two unit, split into 8 base-256 digits, and the 36 digit pairs (i, t) with
// i + t <= 7 are accumulated per level L = i + t in FP32 (exact: every partial sum is an
// integer below 2^22).  With the 8 digit planes of the rows (A_i, 128 x 32 FP16) and U's 8
// transposed digit planes stacked along N (B, 32 x 256 FP16; a digit in [-128, 127] is exact in
// FP16, and two of them come out of one byte permute and one packed subtraction), one MMA per
// digit i covers all its levels at once:
//     D[:, 32 i .. 255] += A_i B[:, 0 .. 255 - 32 i]      (M = 128, N = 32 (8 - i), K = 32),
// so a window is 16 tcgen05.mma (two K = 16 steps per digit) into 256 TMEM columns, level L
// at columns 32 L .. 32 L + 31.  The epilogue reads the levels back with tcgen05.ld, combines
// them in 64-bit integer arithmetic, stores the positions that leave the window and keeps the
// w - r overlap positions for the next block.
//
// The windows of a tile form a chain (consecutive windows overlap), and the chain of the tile
// on the diagonal is what the next group's chase waits for, so a window's latency is what
// counts.  A tile is therefore worked by a whole block: 512 threads, eight per line, and one
// more warp whose first thread issues the TMA copies and the MMAs (an MMA issue holds its
// thread for about as long as the tensor core runs, which would otherwise delay that warp's
// share of the epilogue).  Each line occupies two MMA rows, so that the threads reading its
// results from TMEM sit on all four lane quarters (all four SM sub-partitions), and the thread
// with part j = 0..7 holds positions 2j, 2j+1 and 16+2j, 17+2j, at K = 4j .. 4j+3 of the
// operands (tc_kidx: one 8-byte store per digit plane and row).  The slide by r = 16 positions
// maps position p of window k to position p + 16 of window k-1, so the overlap stays in the
// thread that computed it; the eight threads of a line exchange only the exponent of the
// window's largest entry, through shared memory.  The MMA computes both rows of a line (the
// same products).
//
// Line activity.  Right updates of A and B: a 32-row subtile s takes blocks kmax .. kT_s + 1
// here (every reflector of those blocks is still pending for all its rows) and the staircase
// blocks kT_s .. kstop_s afterwards, reflector by reflector in native FP64 (right_window.cuh),
// the two subtiles side by side.  Left updates: column c takes blocks from the last one whose
// cut lies left of c down to 0.  A line loads its whole window when it becomes active and
// stores its whole window after its last block; inactive lines contribute no loads and no
// stores (their rows of A_i are left as they are and their results are discarded).
//
// One block per SM (544 threads at up to 120 registers), all 512 TMEM columns as two
// accumulators of 256, so that the MMAs of window k run while the half of window k+1 that
// leaves the window is combined and stored; the issuing thread copies the next window's U_k
// while the current one is used.
// The blocks take tiles from the look-ahead schedule (schedule.cuh).
#include <cuda.h>

#include "emu_arith.cuh"
#include "right_window.cuh"
#include "schedule.cuh"

namespace hts {

using namespace emu;

namespace {

constexpr int kTcRows = 128;                        // MMA M, TMEM lanes
constexpr int kTcLines = 64;                        // lines per tile, each in rows l and l + 64
constexpr int kTcSplit = 8;                         // threads per line
constexpr int kLineThreads = kTcLines * kTcSplit;   // the lines' threads (4 per TMEM lane)
constexpr int kIssuer = kLineThreads;               // thread of the extra warp that issues TMA and MMA
constexpr int kTcThreads = kLineThreads + 32;       // one tile per block
constexpr int kTcPos = 4;                           // window positions per thread
constexpr int kWin = 32;                            // window positions (MMA K)
constexpr int kSlide = 16;                          // r: the window slides by r positions per block
constexpr int kTmemCols = kDigits * kWin;           // 8 levels x 32 positions
constexpr int kDigitPlane = kTcRows * kWin * 2;     // one digit plane of the rows: 8 KiB
constexpr int kUBytes = kDigits * kWin * kWin * 2;  // U's 8 digit planes: 16 KiB
constexpr int kStairGroup = 128;                    // threads per 32-row subtile in the staircase
constexpr int kStairDoubles = 2048;                 // shared scratch per subtile (16 KiB)
constexpr unsigned kLBO = 128;                      // K-adjacent core matrices
constexpr unsigned kSBO = 512;                      // row-group-adjacent core matrices
// instruction descriptor of kind::f16: D FP32 (bit 4), A and B FP16 (type 0 at bits 7 and 10),
// both K-major, M / 16 at bit 24; N / 8 goes to bit 17
constexpr unsigned kIdescBase = (1u << 4) | ((unsigned)(kTcRows >> 4) << 24);
constexpr int kWorkerBar = 5;                       // the tile's barrier (1..4: staircase subtiles)

static_assert(kTcSplit * kTcPos == kWin, "a line's positions are split over its threads");
static_assert(2 * kTcLines == kTcRows && kLineThreads == 4 * kTcRows, "two rows per line, four threads per row");
static_assert(4 * kStairDoubles * 8 <= kDigits * kDigitPlane, "staircase scratch fits the digit planes");

struct TcShared {
    unsigned char A[kDigits * kDigitPlane];   // digit planes of the lines (64 KiB)
    unsigned char U[2][kUBytes];              // U_k and U_{k-1} (2 x 16 KiB)
    int em[kTcSplit][kTcLines];               // exponents of the threads' parts of the window
    unsigned long long bar_u[2];              // TMA of U into buffer b
    unsigned long long bar_d[2];              // the MMAs into accumulator b are done
    unsigned tmem_base;
    int slot;
    int abort;
};

// Window position of the k-th entry of the thread with part j (j = 0..7): 2j, 2j+1 in the
// first half, 16+2j, 17+2j in the second, so that the slide by 16 keeps the overlap in-thread.
__device__ __forceinline__ int pos_of(int j, int k) { return (k < 2) ? 2 * j + k : kSlide + 2 * j + (k - 2); }

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

// The 8 levels of 2 consecutive positions (TMEM columns 32 L + c0, 32 L + c0 + 1 of the
// warp's 32 lanes) in one statement together with the wait for them: tcgen05.ld writes its
// registers asynchronously, so nothing may read (or move) them before tcgen05.wait::ld, and
// keeping both in one asm statement leaves the compiler no room to do so.
__device__ __forceinline__ void tc_ld_levels2(unsigned taddr, unsigned (&v)[kDigits][2])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0, %1}, [%16];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x2.b32 {%2, %3}, [%17];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x2.b32 {%4, %5}, [%18];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x2.b32 {%6, %7}, [%19];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x2.b32 {%8, %9}, [%20];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x2.b32 {%10, %11}, [%21];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x2.b32 {%12, %13}, [%22];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x2.b32 {%14, %15}, [%23];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(v[0][0]), "=r"(v[0][1]), "=r"(v[1][0]), "=r"(v[1][1]), "=r"(v[2][0]), "=r"(v[2][1]), "=r"(v[3][0]),
          "=r"(v[3][1]), "=r"(v[4][0]), "=r"(v[4][1]), "=r"(v[5][0]), "=r"(v[5][1]), "=r"(v[6][0]), "=r"(v[6][1]),
          "=r"(v[7][0]), "=r"(v[7][1])
        : "r"(taddr), "r"(taddr + kWin), "r"(taddr + 2 * kWin), "r"(taddr + 3 * kWin), "r"(taddr + 4 * kWin),
          "r"(taddr + 5 * kWin), "r"(taddr + 6 * kWin), "r"(taddr + 7 * kWin)
        : "memory");
}

// Byte offset of (row m, k) in a K-major core-matrix layout with K = 32.
__device__ __forceinline__ unsigned kmaj_off(int m, int k)
{
    return (unsigned)((m >> 3) * kSBO + (k >> 3) * kLBO + (m & 7) * 16 + (k & 7) * 2);
}

// Pipeline state of the block (the same in every thread).
struct TcPhase {
    unsigned u[2];   // parity of the next phase of bar_u[b]
    unsigned d[2];   // parity of the next phase of bar_d[b]
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

// Window position p of line `line`: its matrix element (pos = the matrix column for rows,
// the matrix row for columns).
__device__ __forceinline__ double *elem(const TcTile &t, int line, int pos)
{
    return (t.kind >= 4) ? t.X + (size_t)(pos - 1) + (size_t)(line - 1) * t.ld
                         : t.X + (size_t)(line - 1) + (size_t)(pos - 1) * t.ld;
}

// Loads of a line's window entries: positions pos_of(j, k) < cnt of the window at column (or
// row) c0, for k = 0 .. kn-1 (the others read as zero).
__device__ __forceinline__ void load_part(const TcTile &t, int line, int j, int c0, int cnt, int kn,
                                          double (&v)[kTcPos])
{
#pragma unroll
    for (int k = 0; k < kTcPos; ++k) {
        const int p = pos_of(j, k);
        v[k] = (k < kn && p < cnt && c0 + p <= t.n) ? *elem(t, line, c0 + p) : 0.0;
    }
}

// One half of a window's results (half 0: positions 2j, 2j+1, half 1: 16+2j, 17+2j): the 8
// levels read from the accumulator at taddr (the thread's lane quarter, column 0 of the
// accumulator), combined into integers in units 2^cu_new.  Positions that leave the window
// (p >= w - r, or every position in the line's last window) are stored; half 0 keeps the
// overlap (p < w - r) in carry.  The TMEM read is warp-wide, so every thread takes part.
__device__ __forceinline__ void epilogue_half(const TcTile &t, int line, int j, unsigned taddr, int half, bool act,
                                              bool last, int c0, int cu_new, int w, int r, long long (&carry)[2])
{
    unsigned lv[kDigits][2];
    tc_ld_levels2(taddr + (unsigned)pos_of(j, 2 * half), lv);
    if (!act) return;
#pragma unroll
    for (int kk = 0; kk < 2; ++kk) {
        const int p = pos_of(j, 2 * half + kk);
        if (p < w) {
            const long long v = combine_levels_folded(__uint_as_float(lv[0][kk]), __uint_as_float(lv[1][kk]),
                                                      __uint_as_float(lv[2][kk]), __uint_as_float(lv[3][kk]),
                                                      __uint_as_float(lv[4][kk]), __uint_as_float(lv[5][kk]),
                                                      __uint_as_float(lv[6][kk]), __uint_as_float(lv[7][kk]));
            if ((last || p >= w - r) && c0 + p <= t.n) *elem(t, line, c0 + p) = fixed_to_f64(v, cu_new);
            if (half == 0) carry[kk] = (p < w - r) ? v : 0;
        }
    }
}

// One tile of 64 lines by the block's 512 line threads; the issuing warp (tid >= 512) takes no
// line.  Line thread tid (warp w, lane) reads TMEM lane L = 32 (w mod 4) + lane, the MMA row of
// line l = L mod 64 (rows l and l + 64 both hold that line), and works the positions
// pos_of(j, *) of the line with j = 2 (w / 4) + L / 64.
__device__ void tc_tile(const TcTile &t, int tile, TcShared &S, unsigned tmem, TcPhase &ph, int tid, int *status)
{
    constexpr int r = kSlide;   // the launcher admits r = 16 only
    const int n = t.n, j1 = t.j1, qg = t.qg;
    const int w = r + qg - 1;
    const int jl = j1 + qg - 1;
    const int kmax = nblocks_gen(n, r, j1) - 1;
    const int l0 = tile * kTcLines + 1;
    if (l0 > n || kmax < 0) return;
    const bool liner = tid < kLineThreads;   // false: the issuing warp
    const int qd = (tid >> 5) & 3, L = 32 * qd + (tid & 31);   // lane quarter, TMEM lane
    const int m = L & (kTcLines - 1), j = liner ? 2 * (tid >> 7) + (L >> 6) : 0;   // line of the tile, part
    const int lastline = imin(l0 + kTcLines - 1, n);
    const int line = l0 + m;
    const bool lvalid = liner && line <= n;
    const bool left = t.kind >= 4;
    const bool ab_right = t.kind <= 1;

    // blocks this line takes here: khi .. klo (khi < klo: none); the tile's range K_hi .. K_lo
    int khi = kmax, klo = 0;
    int K_hi = kmax, K_lo = 0;
    if (ab_right) {
        auto kT_of = [&](int s) {
            const int llast = imin(l0 + 32 * s + 31, n);
            return (llast <= j1) ? -1 : qg + (llast - j1 - 1) / r;
        };
        klo = kT_of(m >> 5) + 1;   // the line's 32-row subtile
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
        // Software pipeline over the windows, two TMEM accumulators (columns 0 and 256):
        //   window k:   exponent, digits and MMAs (they need the overlap of window k+1),
        //   meanwhile   the positions of window k+1 that leave it (second half) are combined and stored,
        //   then        window k's first half (the overlap of window k-1) is combined.
        // The chain from one window to the next is thus first half, exponent, digits, MMA.
        const unsigned tl = tmem + ((unsigned)(32 * qd) << 16);
        int ubuf = 0, dbuf = 0;
        int u_pend = 0;               // issuer: buffer with a TMA copy in flight, or -1
        unsigned u_par = ph.u[0];     // the phase that copy completes
        bool bad = false;             // this thread met a wait that ran out
        if (tid == kIssuer) {
            mbar_expect_tx(&S.bar_u[0], kUBytes);
            tma_load_3d(S.U[0], t.map, 0, 0, K_hi, &S.bar_u[0]);
        }
        double fresh[kTcPos];
        long long carry[2] = {0, 0};
        int cu = 0;
        if (K_hi <= khi && K_hi >= klo)
            load_part(t, line, j, j1 + K_hi * r + 1, K_hi == khi ? w : r, K_hi == khi ? kTcPos : 2, fresh);
        else
            load_part(t, line, j, 0, 0, 0, fresh);
        // the window whose second half is still in TMEM
        bool p_act = false;
        int p_c0 = 0, p_cu = 0;

        int k = K_hi;
        for (;; --k) {
            const bool act = k <= khi && k >= klo;
            const bool first = k == khi;
            const bool last = k == klo;
            const int c0 = j1 + k * r + 1;
            // ---- window k: the unit 2^(ua + 62) above its largest entry, over the line's 8 threads
            int e = kZeroExp;
            if (act) {
#pragma unroll
                for (int h = 0; h < kTcPos; ++h) {
                    if (pos_of(j, h) < w) {
                        if (first || h < 2) e = imax(e, exp_of_f64(fresh[h]));
                        else e = imax(e, exp_of_fixed(carry[h - 2], cu));
                    }
                }
            }
            if (liner) S.em[j][m] = e;
            group_sync(kWorkerBar, kTcThreads);
            int em = S.em[0][m];
#pragma unroll
            for (int q = 1; q < kTcSplit; ++q) em = imax(em, S.em[q][m]);
            const int ua = (em == kZeroExp ? 0 : em + 2) - 64;
            if (act) {
                // this thread's digits: its four positions sit at K = 4j .. 4j+3 (tc_kidx), one
                // 8-byte store per plane into each of the line's two rows
                long long x[kTcPos];
#pragma unroll
                for (int h = 0; h < kTcPos; ++h) {
                    x[h] = 0;
                    if (pos_of(j, h) < w) x[h] = (first || h < 2) ? f64_to_fixed(fresh[h], ua) : refix(carry[h - 2], cu, ua);
                }
                unsigned d01[kDigits], d23[kDigits];
                digit_pairs_f16(x[0], x[1], d01);
                digit_pairs_f16(x[2], x[3], d23);
                const unsigned o0 = kmaj_off(m, tc_kidx(pos_of(j, 0)));
                const unsigned o1 = kmaj_off(m + kTcLines, tc_kidx(pos_of(j, 0)));
#pragma unroll
                for (int i = 0; i < kDigits; ++i) {
                    unsigned char *pl = S.A + i * kDigitPlane;
                    *reinterpret_cast<uint2 *>(pl + o0) = make_uint2(d01[i], d23[i]);
                    *reinterpret_cast<uint2 *>(pl + o1) = make_uint2(d01[i], d23[i]);
                }
            }
            fence_async_smem();
            tc_fence_before();
            if (group_sync_or(kWorkerBar, kTcThreads, bad)) {
                bad = true;
                break;
            }
            if (tid == kIssuer) {
                tc_fence_after();
                if (!mbar_wait(&S.bar_u[ubuf], ph.u[ubuf])) {
                    record_error(status, HTS_ERR_TIMEOUT, 0, -2, k, tile);
                    bad = true;
                    tc_commit(&S.bar_d[dbuf]);   // no MMAs: the others' wait ends, the tile stops next
                } else {
                    u_pend = -1;
                    const unsigned a0 = smem_u32(S.A), b0 = smem_u32(S.U[ubuf]);
                    const unsigned dcol = tmem + (unsigned)(dbuf * kTmemCols);
#pragma unroll
                    for (int i = 0; i < kDigits; ++i) {
                        const unsigned idesc = kIdescBase | ((unsigned)((kWin * (kDigits - i)) >> 3) << 17);
#pragma unroll
                        for (int kk = 0; kk < 2; ++kk)
                            tc_mma(dcol + kWin * i, smem_desc(a0 + i * kDigitPlane + kk * 2 * kLBO),
                                   smem_desc(b0 + kk * 2 * kLBO), idesc, (i > 0 || kk > 0) ? 1 : 0);
                    }
                    tc_commit(&S.bar_d[dbuf]);
                    // U of the next block into the other buffer (its last reader, the previous
                    // window's MMAs, has completed)
                    if (k - 1 >= K_lo) {
                        mbar_expect_tx(&S.bar_u[ubuf ^ 1], kUBytes);
                        tma_load_3d(S.U[ubuf ^ 1], t.map, 0, 0, k - 1, &S.bar_u[ubuf ^ 1]);
                        u_pend = ubuf ^ 1;
                        u_par = ph.u[ubuf ^ 1];
                    }
                }
            }
            ph.u[ubuf] ^= 1u;
            ubuf ^= 1;
            if (liner) {
                // the next window's new positions, while the MMAs run (this window's are consumed)
                {
                    const int kn = k - 1;
                    if (kn >= K_lo && kn <= khi && kn >= klo)
                        load_part(t, line, j, j1 + kn * r + 1, kn == khi ? w : r, kn == khi ? kTcPos : 2, fresh);
                }
                // ---- the second half of window k+1 (positions 16 .. w-1 leave it), while the MMAs run
                if (k < K_hi)
                    epilogue_half(t, line, j, tl + (unsigned)((dbuf ^ 1) * kTmemCols), 1, p_act, true, p_c0, p_cu, w, r,
                                  carry);
                // ---- the first half of window k: the overlap of window k-1 (and position 15)
                if (!mbar_wait(&S.bar_d[dbuf], ph.d[dbuf])) {
                    record_error(status, HTS_ERR_TIMEOUT, 0, -3, k, tile);
                    bad = true;
                }
                tc_fence_after();
                epilogue_half(t, line, j, tl + (unsigned)(dbuf * kTmemCols), 0, act, last, c0, ua + 3, w, r, carry);
            }
            ph.d[dbuf] ^= 1u;
            p_act = act;
            p_c0 = c0;
            p_cu = ua + 3;
            if (act) cu = ua + 3;
            dbuf ^= 1;
            tc_fence_before();
            if (k == K_lo) break;
        }
        // the second half of the last window
        if (liner && !bad) {
            tc_fence_after();
            epilogue_half(t, line, j, tl + (unsigned)((dbuf ^ 1) * kTmemCols), 1, p_act, true, p_c0, p_cu, w, r, carry);
            tc_fence_before();
        }
        if (group_sync_or(kWorkerBar, kTcThreads, bad)) {
            // stop the tile: let a copy into U that is still in flight land (bounded) before
            // the buffer is reused or the block exits, and the other tiles of the block end
            if (tid == kIssuer) {
                if (u_pend >= 0 && !mbar_wait(&S.bar_u[u_pend], u_par)) record_error(status, HTS_ERR_TIMEOUT, 0, -4, 0, tile);
                *(volatile int *)&S.abort = 1;
            }
            group_sync(kWorkerBar, kTcThreads);
            return;
        }
    }

    // staircase blocks of the right updates of A and B in native FP64, the two 32-row subtiles
    // side by side (128 threads each, the others idle; their rows were stored above)
    if (ab_right) {
        const int s = tid / kStairGroup;
        const int x0 = l0 + 32 * s;
        if (s < kTcLines / 32 && x0 <= n) {
            const int llast = imin(x0 + 31, n);
            const int kT = (llast <= j1) ? -1 : qg + (llast - j1 - 1) / r;
            const int skstart = imin(kT, kmax);
            const int skstop = (x0 <= j1) ? 0 : (x0 - j1 - 1) / r + 2;
            if (skstop <= skstart)
                right_window_rows<kStairGroup>(t.X, (int)t.ld, t.kind, t.R.VZ, t.R.TZ, t.R.kdim, n, r, j1, qg, x0,
                                               skstart, skstop,
                                               reinterpret_cast<double *>(S.A) + (size_t)s * kStairDoubles,
                                               tid % kStairGroup, 1 + s);
        }
        group_sync(kWorkerBar, kTcThreads);
    }
}

}  // namespace

// ---------------------------------------------------------------------------------------
// Persistent look-ahead update launch on the tensor cores (schedule.cuh): one block per SM,
// taking 64-line tiles in ticket order.
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kTcThreads, 1) k_s2_update_tc(const __grid_constant__ UpdTcArgs a)
{
    extern __shared__ __align__(1024) unsigned char tc_smem_raw[];
    // operand buffers on a 1 KiB boundary (TMA destinations need 128 bytes)
    TcShared &S = *reinterpret_cast<TcShared *>(tc_smem_raw + ((1024u - (smem_u32(tc_smem_raw) & 1023u)) & 1023u));
    const int tid = threadIdx.x;
    if (tid < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&S.tmem_base)),
                     "r"(2 * kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        mbar_init(&S.bar_u[0], 1);
        mbar_init(&S.bar_u[1], 1);
        mbar_init(&S.bar_d[0], 1);
        mbar_init(&S.bar_d[1], 1);
        S.abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tmem = S.tmem_base;
    TcPhase ph;
    ph.u[0] = ph.u[1] = 0;
    ph.d[0] = ph.d[1] = 0;
    update_worker<kTcThreads>(a.s, tid, kWorkerBar, &S.slot, [&](const Task &T) {
        // an empty slot of the ticket layout (a row of the plan without this kind of tile)
        if (*(volatile int *)&S.abort || T.kind == kTaskNone) return;
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
        tc_tile(tt, T.tile, S, tmem, ph, tid, a.s.status);
    });
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid < 32)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(S.tmem_base), "r"(2 * kTmemCols)
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

int update_tc_workers() { return 1; }
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
    k_s2_update_tc<<<ctas, kTcThreads, sm, st>>>(a);
    return cudaGetLastError();
}

}  // namespace hts
