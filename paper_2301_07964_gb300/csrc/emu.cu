// Delayed updates of stage 2 as small dense products, in emulated FP64 on the BF16 tensor
// cores (HTS_GEMM_EMU_BF16).
//
// Block formation (Alg. 4, "form compact WY" / the accumulated reflector blocks): for each
// block k of a group, the group's qg reflectors of that block act on one window of
// w = r + qg - 1 consecutive indices.  Their product in sweep order
//     U^Z_k = Z^_k^{j1} Z^_k^{j1+1} ... Z^_k^{j1+qg-1},  U^Q_k = Q^_k^{j1} ... Q^_k^{j1+qg-1}
// is formed explicitly as a w x w matrix (k_s2_form_u).  The delayed updates then become
//     X(rows, window k) := X(rows, window k) U_k           (A, B rows above the band; Z; Q)
//     X(window k, cols)^T := X(window k, cols)^T U^Q_k     (the left updates of A and B)
// for k from the last block to the first; consecutive windows overlap in qg - 1 indices, so
// a tile of rows keeps the overlap in registers and streams r new columns per block.
//
// Emulation.  Every operand is written as a fixed-point integer with a shared scale, x =
// round(v 2^-unit), split into 8 balanced base-256 digits d_1..d_8 in [-128, 127]
// (x = sum d_i 256^(8-i)); each digit is exact in BF16.  A product of a row window with U_k
// is the sum over digit pairs (i, t) of (digits_i of the rows) (digits_t of U_k), weighted by
// 256^-(i+t); pairs with the same level i + t share an FP32 accumulator, in which every partial
// sum is an integer below 2^22 and hence exact.  Levels 2..9 are formed (36 products, each a
// 16 x 8 x 16 BF16 mma.sync) and summed in 64-bit integer arithmetic.  Row scales are powers of
// two taken from the largest entry of each row window (2^e > max |a|, a = x 2^(e-62)); U_k
// (orthogonal, entries in [-1, 1]) uses the fixed scale 2^-61.  The error of a product is
// below 2^(e-55): U's rounding contributes at most 2^-62 sum |a_k|, the dropped levels about
// 2^(e-58) for typical digits (2^(e-53) for adversarial ones), far below one FP64 rounding unit
// of the window's largest entry.  No FP64 instruction runs in the update loop: FP64 values enter and leave
// through integer bit manipulation of their IEEE-754 encoding.
#include "emu_arith.cuh"
#include "right_window.cuh"
#include "schedule.cuh"

namespace hts {

using namespace emu;

namespace {

constexpr int kEmuWarps = 2;               // 16-line slabs per apply block
constexpr int kEmuRows = 16 * kEmuWarps;   // rows (or columns) per apply block

__device__ __forceinline__ void mma_bf16(float (&d)[4], const unsigned (&a)[4], unsigned b0, unsigned b1)
{
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                 "{%0,%1,%2,%3};"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }


}  // namespace

// ---------------------------------------------------------------------------------------
// Block formation: one warp per (block k, reflector family).  U (w x w, zero padded to
// 32 x 32) starts as the identity and is multiplied from the right by the group's reflectors
// of block k in sweep order (lane = row of U).  The result is stored as digit planes laid
// out as the B operand of mma.m16n8k16: word ((t * 2 + kt) * 4 + nt) * 32 + lane holds, for
// lane = 4 g + c, the digit t of U(16 kt + 2c + {0, 1}, 8 nt + g) and of
// U(16 kt + 2c + {8, 9}, 8 nt + g).
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(128) k_s2_form_u(FormUArgs a)
{
    __shared__ double Us[4][32 * 33];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int k = blockIdx.x * 4 + warp;
    const int fam = blockIdx.y;   // 0: Q^ reflectors, 1: Z^ reflectors
    const int kmax = nblocks_gen(a.n, a.r, a.j1) - 1;
    if (k > kmax || __ldcg(a.status) != 0) return;   // no block-wide barrier follows
    const int w = a.r + a.qg - 1;
    const int kdim = a.R.kdim;
    double *U = Us[warp];
    for (int c = 0; c < 32; ++c) U[lane * 33 + c] = (lane == c && lane < w) ? 1.0 : 0.0;
    const double *V = fam ? a.R.VZ : a.R.VQ;
    const double *T = fam ? a.R.TZ : a.R.TQ;
    for (int s = 0; s < a.qg; ++s) {
        const double tau = __ldcg(T + (size_t)s * kdim + k);
        if (tau == 0.0) continue;
        const int mlen = imin(a.r, a.n - (a.j1 + s + k * a.r));
        const double *v = V + ((size_t)s * kdim + k) * a.r;
        double *row = U + lane * 33 + s;
        double d0 = 0.0, d1 = 0.0;
        for (int i = 0; i < mlen; i += 2) {
            d0 = fma(row[i], __ldcg(v + i), d0);
            if (i + 1 < mlen) d1 = fma(row[i + 1], __ldcg(v + i + 1), d1);
        }
        const double d = (d0 + d1) * tau;
        for (int i = 0; i < mlen; ++i) row[i] = fma(-d, __ldcg(v + i), row[i]);
    }
    __syncwarp();
    if (a.umma) {
        // tcgen05 B operand of block k: the transposed FP16 digit planes U_t^T stacked along N
        // (N = 32 t + output position, K = tc_kidx(input position)), K-major core matrices of
        // 8 x 16 bytes, LBO 128 B, SBO 512 B.  Lane = input position; lanes 2i, 2i+1 share a word
        // (tc_kidx keeps them adjacent).
        unsigned char *blk = reinterpret_cast<unsigned char *>((fam ? a.planesZ : a.planesQ) + (size_t)k * kPlaneWords);
        const int kx = tc_kidx(lane);
        for (int col = 0; col < 32; ++col) {
            unsigned d[kDigits];
            digit_pairs_f16(f64_to_fixed(U[lane * 33 + col], kUnitU), 0, d);   // low halves
#pragma unroll
            for (int t = 0; t < kDigits; ++t) {
                const unsigned nb = __shfl_down_sync(0xffffffffu, d[t], 1);
                if ((lane & 1) == 0) {
                    const int nn = 32 * t + col;
                    const size_t off = (size_t)(nn >> 3) * 512 + (kx >> 3) * 128 + (nn & 7) * 16 + (kx & 7) * 2;
                    *reinterpret_cast<unsigned *>(blk + off) = pack_f16(d[t], nb);
                }
            }
        }
        return;
    }
    const int g = lane >> 2, c = lane & 3;
    uint2 *out = (fam ? a.planesZ : a.planesQ) + (size_t)k * kPlaneWords;
#pragma unroll
    for (int kt = 0; kt < 2; ++kt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
            const int col = 8 * nt + g, r0 = 16 * kt + 2 * c;
            unsigned e0[kDigits], e1[kDigits], e8[kDigits], e9[kDigits];
            digits_bf16(f64_to_fixed(U[r0 * 33 + col], kUnitU), e0);
            digits_bf16(f64_to_fixed(U[(r0 + 1) * 33 + col], kUnitU), e1);
            digits_bf16(f64_to_fixed(U[(r0 + 8) * 33 + col], kUnitU), e8);
            digits_bf16(f64_to_fixed(U[(r0 + 9) * 33 + col], kUnitU), e9);
#pragma unroll
            for (int t = 0; t < kDigits; ++t)
                out[((t * 2 + kt) * 4 + nt) * 32 + lane] = make_uint2(pack_bf16(e0[t], e1[t]), pack_bf16(e8[t], e9[t]));
        }
}

// ---------------------------------------------------------------------------------------
// Emulated delayed update.  A block owns 32 lines (rows of X for the right updates, columns
// of X for the left updates) in two slabs of 16 (small blocks, so that several run on one SM
// out of phase with each other), and each slab's window of 32 positions
// (window index p = column c0 + p, or row R0 + p, with c0 = R0 = j1 + k r + 1).  Two warps
// share a slab: half 0 holds positions 0..15 (operand k-tile 0), half 1 positions 16..31.
// Lane 4 g + c holds lines g and g + 8 at positions 16 kt + 8 h + 2 c + {0, 1}: exactly the
// A-operand positions of mma.m16n8k16 and the result positions of its accumulator.  Per
// block k of the group:
//   half 0: the scale of each line (its largest entry over the new columns and the carried
//           positions), hands the carry (last window's positions 0 .. w-r-1, which become
//           16 .. 16+w-r-1) and the scales to half 1, and loads the next window's new columns;
//   both:   digits of their own k-tile, exchanged through shared memory; products for their
//           own two n-tiles (half 0: output positions 0..15, half 1: 16..31); results;
//   half 1: stores its positions (they leave the window); half 0 keeps its positions as the
//           next carry (all positions are stored after the last block).
// The slide by r = 16 positions is one k-tile, which is why this kernel needs r = 16.
// ---------------------------------------------------------------------------------------
constexpr int kEmuThreads = 64 * kEmuWarps;   // two warps per 16-line slab

struct EmuSmem {
    uint2 planes[2][kPlaneWords];           // U digit planes of blocks k and k-1
    uint4 dig[kEmuWarps][2][kDigits][32];   // A-operand digits of each half, [slab][half][t][lane]
    long long carry[kEmuWarps][8][32];      // carried window positions, [slab][slot][lane]
    int unit[kEmuWarps][2][32];             // scales of the two lines of each lane
};

template <int HALF>
__device__ __forceinline__ void emu_worker(const EmuArgs &a, EmuSmem &S, int kind, double *X, size_t ld,
                                           const uint2 *P, int l0, int kbeg, int kend, int tid, int wb)
{
    const int lane = tid & 31, slab = (tid >> 5) >> 1;
    const int g = lane >> 2, c = lane & 3;
    const int n = a.n, r = a.r, j1 = a.j1, qg = a.qg;
    const int w = r + qg - 1;
    const int jl = j1 + qg - 1;
    const bool left = kind >= 4;
    const int bar = wb + 1 + slab;
    const int lineA = l0 + slab * 16 + g, lineB = lineA + 8;   // lines of rr = 0, 1
    auto addr = [=](int ln, int p, int k) -> double * {
        const int pos = j1 + k * r + 1 + p;   // matrix column (right) or row (left)
        return left ? X + (size_t)(pos - 1) + (size_t)(ln - 1) * ld : X + (size_t)(ln - 1) + (size_t)(pos - 1) * ld;
    };
    auto valid = [=](int ln, int p, int k) -> bool { return ln <= n && p < w && j1 + k * r + 1 + p <= n; };

    double dv[2][2][2];        // half 0: FP64 values entering at positions 8 h + 2 c + pair
    long long xc[2][2][2];     // half 0: carried positions (the next window's k-tile 1)
    int uc[2] = {0, 0};        // their scales
    if (HALF == 0) {
        // first window: positions of k-tile 1 become the carry at their own scale
        int em[2] = {kZeroExp, kZeroExp};
        double v1[2][2][2];
#pragma unroll
        for (int rr = 0; rr < 2; ++rr)
#pragma unroll
            for (int h = 0; h < 2; ++h)
#pragma unroll
                for (int pr = 0; pr < 2; ++pr) {
                    const int ln = rr ? lineB : lineA;
                    const int p = 8 * h + 2 * c + pr;
                    dv[rr][h][pr] = valid(ln, p, kbeg) ? *addr(ln, p, kbeg) : 0.0;
                    v1[rr][h][pr] = valid(ln, p + 16, kbeg) ? *addr(ln, p + 16, kbeg) : 0.0;
                    em[rr] = imax(em[rr], exp_of_f64(v1[rr][h][pr]));
                }
#pragma unroll
        for (int rr = 0; rr < 2; ++rr) {
            em[rr] = imax(em[rr], __shfl_xor_sync(0xffffffffu, em[rr], 1));
            em[rr] = imax(em[rr], __shfl_xor_sync(0xffffffffu, em[rr], 2));
            uc[rr] = (em[rr] == kZeroExp ? 0 : em[rr] + 2) - 64;
#pragma unroll
            for (int h = 0; h < 2; ++h)
#pragma unroll
                for (int pr = 0; pr < 2; ++pr) xc[rr][h][pr] = f64_to_fixed(v1[rr][h][pr], uc[rr]);
        }
    }

    for (int k = kbeg; k >= kend; --k) {
        const bool last = (k == kend);
        const int buf = (kbeg - k) & 1;
        // next block's planes (all threads)
        if (!last) {
            const uint4 *src = reinterpret_cast<const uint4 *>(P + (size_t)(k - 1) * kPlaneWords);
            uint4 *dst = reinterpret_cast<uint4 *>(S.planes[buf ^ 1]);
            for (int e = tid; e < kPlaneWords / 2; e += kEmuThreads) cp_async16(dst + e, src + e);
        }
        cp_async_commit();

        // ---- scales and carry (half 0 -> half 1)
        long long xv[2][2][2];   // this half's window positions in units 2^ua
        int ua[2];
        if (HALF == 0) {
#pragma unroll
            for (int rr = 0; rr < 2; ++rr) {
                int em = kZeroExp;
#pragma unroll
                for (int h = 0; h < 2; ++h)
#pragma unroll
                    for (int pr = 0; pr < 2; ++pr) {
                        em = imax(em, exp_of_f64(dv[rr][h][pr]));
                        em = imax(em, exp_of_fixed(xc[rr][h][pr], uc[rr]));
                    }
                em = imax(em, __shfl_xor_sync(0xffffffffu, em, 1));
                em = imax(em, __shfl_xor_sync(0xffffffffu, em, 2));
                ua[rr] = (em == kZeroExp ? 0 : em + 2) - 64;   // |x| < 2^62
                S.unit[slab][rr][lane] = ua[rr];
#pragma unroll
                for (int h = 0; h < 2; ++h)
#pragma unroll
                    for (int pr = 0; pr < 2; ++pr)
                        S.carry[slab][(rr * 2 + h) * 2 + pr][lane] = refix(xc[rr][h][pr], uc[rr], ua[rr]);
            }
        }
        group_sync(bar, 64);
        if (HALF == 1) {
#pragma unroll
            for (int rr = 0; rr < 2; ++rr) {
                ua[rr] = S.unit[slab][rr][lane];
#pragma unroll
                for (int h = 0; h < 2; ++h)
#pragma unroll
                    for (int pr = 0; pr < 2; ++pr) xv[rr][h][pr] = S.carry[slab][(rr * 2 + h) * 2 + pr][lane];
            }
        } else {
            // this window's new columns in fixed point (after the hand-off, so that half 1 is
            // not kept waiting), then the next window's new columns (positions 0 .. r-1)
#pragma unroll
            for (int rr = 0; rr < 2; ++rr)
#pragma unroll
                for (int h = 0; h < 2; ++h)
#pragma unroll
                    for (int pr = 0; pr < 2; ++pr) xv[rr][h][pr] = f64_to_fixed(dv[rr][h][pr], ua[rr]);
#pragma unroll
            for (int rr = 0; rr < 2; ++rr)
#pragma unroll
                for (int h = 0; h < 2; ++h)
#pragma unroll
                    for (int pr = 0; pr < 2; ++pr) {
                        const int ln = rr ? lineB : lineA;
                        const int p = 8 * h + 2 * c + pr;
                        dv[rr][h][pr] = (!last && valid(ln, p, k - 1)) ? *addr(ln, p, k - 1) : 0.0;
                    }
        }

        // ---- digits of this half's k-tile, exchanged with the other half
        unsigned af[kDigits][2][4];
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int rr = 0; rr < 2; ++rr) {
                unsigned d0[kDigits], d1[kDigits];
                digits_bf16(xv[rr][h][0], d0);
                digits_bf16(xv[rr][h][1], d1);
#pragma unroll
                for (int t = 0; t < kDigits; ++t) af[t][HALF][2 * h + rr] = pack_bf16(d0[t], d1[t]);
            }
#pragma unroll
        for (int t = 0; t < kDigits; ++t)
            S.dig[slab][HALF][t][lane] = make_uint4(af[t][HALF][0], af[t][HALF][1], af[t][HALF][2], af[t][HALF][3]);
        group_sync(bar, 64);
#pragma unroll
        for (int t = 0; t < kDigits; ++t) {
            const uint4 o = S.dig[slab][HALF ^ 1][t][lane];
            af[t][HALF ^ 1][0] = o.x;
            af[t][HALF ^ 1][1] = o.y;
            af[t][HALF ^ 1][2] = o.z;
            af[t][HALF ^ 1][3] = o.w;
        }

        // ---- line activity (left updates: columns right of the cut of block k)
        bool act0 = true, act1 = true;
        if (left) {
            const int cut = (kind == 5) ? imin(jl + (k + 1) * r, n) : jl + imax(0, (k - 1) * r + 1);
            act0 = lineA > cut;
            act1 = lineB > cut;
        }

        cp_async_wait<1>();
        group_sync(wb, kEmuThreads);
        const uint2 *pl = S.planes[buf];

        // ---- products for this half's two n-tiles; results replace xv
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int nt = 2 * HALF + h;
            float acc[kTopLevel - 1][4];
#pragma unroll
            for (int d = 0; d < kTopLevel - 1; ++d)
#pragma unroll
                for (int e = 0; e < 4; ++e) acc[d][e] = 0.0f;
#pragma unroll
            for (int t = 0; t < kDigits; ++t) {
                const uint2 b0 = pl[((t * 2 + 0) * 4 + nt) * 32 + lane];
                const uint2 b1 = pl[((t * 2 + 1) * 4 + nt) * 32 + lane];
#pragma unroll
                for (int i = 0; i < kDigits; ++i) {
                    if (i + t + 2 <= kTopLevel) {   // level (i+1) + (t+1)
                        mma_bf16(acc[i + t], af[i][0], b0.x, b0.y);
                        mma_bf16(acc[i + t], af[i][1], b1.x, b1.y);
                    }
                }
            }
            // levels 2..9 -> one integer in units 2^(ua + 3): level L weighs 2^(8 (8 - L))
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int c2 = f32_exact_int(acc[0][e]), c3 = f32_exact_int(acc[1][e]);
                const int c4 = f32_exact_int(acc[2][e]), c5 = f32_exact_int(acc[3][e]);
                const int c6 = f32_exact_int(acc[4][e]), c7 = f32_exact_int(acc[5][e]);
                const int c8 = f32_exact_int(acc[6][e]), c9 = f32_exact_int(acc[7][e]);
                const int lo = (c7 << 8) + c8 + ((c9 + 128) >> 8);
                const int mid = (c5 << 8) + c6;
                const long long hi = ((long long)c2 << 16) + (long long)((c3 << 8) + c4);
                const long long val = (hi << 32) + ((long long)mid << 16) + (long long)lo;
                const int rr = e >> 1, pr = e & 1;
                const bool act = rr ? act1 : act0;
                xv[rr][h][pr] = act ? val : refix(xv[rr][h][pr], ua[rr], ua[rr] + 3);
            }
        }
        group_sync(wb, kEmuThreads);   // planes[buf] is refilled by the next iteration's copy

        // ---- positions leaving the window; half 0 keeps the carry
#pragma unroll
        for (int rr = 0; rr < 2; ++rr) {
            const int ln = rr ? lineB : lineA;
#pragma unroll
            for (int h = 0; h < 2; ++h)
#pragma unroll
                for (int pr = 0; pr < 2; ++pr) {
                    const int p = 16 * HALF + 8 * h + 2 * c + pr;
                    if ((last || p >= w - r) && valid(ln, p, k))
                        *addr(ln, p, k) = fixed_to_f64(xv[rr][h][pr], ua[rr] + 3);
                    if (HALF == 0) xc[rr][h][pr] = (p < w - r) ? xv[rr][h][pr] : 0;
                }
            uc[rr] = ua[rr] + 3;
        }
    }
}

// One tile of an emulated delayed update: lines tile*32+1 .. of matrix a.M[mi], by the 128
// threads tid = 0..127 of a group whose barrier is wb (slab barriers wb+1, wb+2).  Right
// updates of A and B also run the tile's staircase blocks in native FP64.
__device__ __forceinline__ void emu_tile(const EmuArgs &a, EmuSmem &S, int mi, int tile, int tid, int wb)
{
    const int warp = tid >> 5;
    const int n = a.n, r = a.r, j1 = a.j1, qg = a.qg;
    const int kind = a.kind[mi];
    const bool left = kind >= 4;
    double *X = a.M[mi];
    const size_t ld = (size_t)a.ld[mi];
    const uint2 *P = (kind == 3 || left) ? a.planesQ : a.planesZ;
    const int kmax = nblocks_gen(n, r, j1) - 1;
    const int jl = j1 + qg - 1;

    const int l0 = tile * kEmuRows + 1;
    const int llast = imin(l0 + kEmuRows - 1, n);
    int kbeg = kmax, kend = 0;
    int skstart = -1, skstop = 0;   // staircase blocks (rows of A and B)
    if (kind <= 1) {
        // rows of A and B: blocks whose whole reflector set is still pending for every row
        // of the tile are emulated; the blocks below them down to the last one any row of the
        // tile needs (x < i4(k, j1+qg-1) = j1 + 1 + max(0, (k-1) r)) form the staircase,
        // applied reflector by reflector in native FP64 afterwards
        const int kT = (llast <= j1) ? -1 : qg + (llast - j1 - 1) / r;
        kend = kT + 1;
        skstart = imin(kT, kmax);
        skstop = (l0 <= j1) ? 0 : (l0 - j1 - 1) / r + 2;
    } else if (left) {
        const int isB = kind == 5;
        kbeg = -1;
        for (int k = kmax; k >= 0; --k) {
            const int cut = isB ? imin(jl + (k + 1) * r, n) : jl + imax(0, (k - 1) * r + 1);
            if (cut < llast) { kbeg = k; break; }
        }
    }
    if (l0 > n) return;

    if (kbeg >= kend) {
        // U planes of block kbeg
        {
            const uint4 *src = reinterpret_cast<const uint4 *>(P + (size_t)kbeg * kPlaneWords);
            uint4 *dst = reinterpret_cast<uint4 *>(S.planes[0]);
            for (int e = tid; e < kPlaneWords / 2; e += kEmuThreads) cp_async16(dst + e, src + e);
            cp_async_commit();
        }
        if (warp & 1) emu_worker<1>(a, S, kind, X, ld, P, l0, kbeg, kend, tid, wb);
        else emu_worker<0>(a, S, kind, X, ld, P, l0, kbeg, kend, tid, wb);
        cp_async_wait<0>();
    }
    if (kind <= 1 && skstop <= skstart) {
        group_sync(wb, kEmuThreads);   // the tile's emulated results are stored; shared memory is reused
        right_window_rows<kEmuThreads>(X, (int)ld, kind, a.R.VZ, a.R.TZ, a.R.kdim, n, r, j1, qg, l0, skstart,
                                       skstop, reinterpret_cast<double *>(&S), tid, wb);
    }
}

__global__ void __launch_bounds__(kEmuThreads) k_s2_emu_apply(EmuArgs a)
{
    extern __shared__ __align__(16) unsigned char emu_smem[];
    EmuSmem &S = *reinterpret_cast<EmuSmem *>(emu_smem);
    if (__ldcg(a.status) != 0) return;
    const int kind = a.kind[blockIdx.y];
    // left updates walk the column tiles from the right
    const int tile = kind >= 4 ? (int)(gridDim.x - 1 - blockIdx.x) : (int)blockIdx.x;
    emu_tile(a, S, blockIdx.y, tile, threadIdx.x, 0);
}

// ---------------------------------------------------------------------------------------
// Look-ahead update launch (schedule.cuh): one block per SM with kUpdEmuWorkers independent
// workers of 128 threads, each with its own shared memory and barriers (ids 3w+1 .. 3w+3), taking
// the tiles of the group's A / B updates and of the previous group's Q / Z update in ticket order.
// The blocks leave the remaining SMs to the chase of the next group, which runs beside them.
// ---------------------------------------------------------------------------------------
constexpr int kUpdEmuWorkers = 3;

__global__ void __launch_bounds__(kEmuThreads * kUpdEmuWorkers, 1) k_s2_update_emu(UpdEmuArgs a)
{
    extern __shared__ __align__(16) unsigned char upd_smem[];
    __shared__ int slot[kUpdEmuWorkers];
    const int worker = threadIdx.x / kEmuThreads, tid = threadIdx.x % kEmuThreads;
    EmuSmem &S = reinterpret_cast<EmuSmem *>(upd_smem)[worker];
    const int wb = 1 + 3 * worker;
    update_worker<kEmuThreads>(a.s, tid, wb, &slot[worker], [&](const Task &T) {
        if (T.kind == kTaskRight) emu_tile(a.right, S, T.mat, T.tile, tid, wb);
        else if (T.kind == kTaskLeft) emu_tile(a.left, S, T.mat, T.tile, tid, wb);
        else if (T.kind == kTaskQZ) emu_tile(a.qz, S, T.mat, T.tile, tid, wb);
    });
}

// ---------------------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------------------
size_t emu_plane_bytes(int kdim) { return (size_t)kdim * kPlaneWords * sizeof(uint2); }

bool emu_supported(int r, int qg) { return r == 16 && qg >= 1 && r + qg - 1 <= 32; }

cudaError_t launch_s2_form_u(const FormUArgs &a, cudaStream_t st)
{
    const int kmax = nblocks_gen(a.n, a.r, a.j1) - 1;
    if (kmax < 0) return cudaSuccess;
    dim3 grid((kmax + 1 + 3) / 4, 2);
    k_s2_form_u<<<grid, 128, 0, st>>>(a);
    return cudaGetLastError();
}

int update_emu_workers() { return kUpdEmuWorkers; }

cudaError_t launch_s2_update_emu(const UpdEmuArgs &a, int ctas, cudaStream_t st)
{
    const int sm = (int)(kUpdEmuWorkers * sizeof(EmuSmem));
    cudaError_t e = cudaFuncSetAttribute(k_s2_update_emu, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    if (e != cudaSuccess) return e;
    k_s2_update_emu<<<ctas, kEmuThreads * kUpdEmuWorkers, sm, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_s2_emu_apply(const EmuArgs &a, int nmat, cudaStream_t st)
{
    if (nmat <= 0) return cudaSuccess;
    const int sm = (int)sizeof(EmuSmem);
    cudaError_t e = cudaFuncSetAttribute(k_s2_emu_apply, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    if (e != cudaSuccess) return e;
    dim3 grid((a.n + kEmuRows - 1) / kEmuRows, nmat);
    k_s2_emu_apply<<<grid, kEmuThreads, sm, st>>>(a);
    return cudaGetLastError();
}

}  // namespace hts
