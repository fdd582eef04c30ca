// C-ABI entry points of the HT-reduction library (declared in include/hts.h).
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "schedule.cuh"

namespace hts {

namespace {

struct DeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) return;
        ok = (prev == dev) || (cudaSetDevice(dev) == cudaSuccess);
    }
    ~DeviceGuard()
    {
        if (ok && prev >= 0) cudaSetDevice(prev);
    }
};

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Workspace layout of stage 2: three reflector sets (group g uses set g mod 3; the look-ahead
// update of group g+1 still reads set g for its Q / Z part while group g+2 generates into the
// next one), one progress word per sweep slot and helper, the tile flags and ticket counters of
// the look-ahead updates and, for the emulated updates, the digit planes of the blocks'
// reflector products (one plane set per reflector set).  The words from off_flags up to
// total_fp64 are cleared at the start of every call.
constexpr int kSets = 3;

struct S2Layout {
    int kdim, qmax, ntiles, nticket;
    size_t off_vq[kSets], off_tq[kSets], off_vz[kSets], off_tz[kSets], off_gram[kSets];
    size_t off_flags, off_tflags, off_tick, total_fp64;
    size_t off_pq[kSets], off_pz[kSets], total;
};

S2Layout s2_layout(int n, int r)
{
    S2Layout L;
    L.kdim = 2 + n / (r > 0 ? r : 1);
    L.qmax = r;
    const size_t nv = (size_t)L.qmax * L.kdim * r * sizeof(double);
    const size_t nt = (size_t)L.qmax * L.kdim * sizeof(double);
    size_t o = 0;
    for (int b = 0; b < kSets; ++b) {
        L.off_vq[b] = o; o = align_up(o + nv, 256);
        L.off_tq[b] = o; o = align_up(o + nt, 256);
        L.off_vz[b] = o; o = align_up(o + nv, 256);
        L.off_tz[b] = o; o = align_up(o + nt, 256);
        L.off_gram[b] = o;   // the Gram entries are used by the r <= 16 chase only
        if (r <= 16) o = align_up(o + (size_t)L.kdim * L.qmax * L.qmax * sizeof(double), 256);
    }
    L.off_flags = o; o = align_up(o + 2 * (size_t)L.qmax * sizeof(unsigned long long), 256);
    L.ntiles = (n + 31) / 32;   // tiles of the smallest tile height (32 lines)
    L.off_tflags = o; o = align_up(o + 4 * (size_t)L.ntiles * sizeof(unsigned long long), 256);
    L.nticket = n + 2;   // one per update launch: at most n - 2 groups plus the closing Q / Z launch
    L.off_tick = o; o = align_up(o + (size_t)L.nticket * sizeof(unsigned), 256);
    L.total_fp64 = o;
    const size_t np = emu_plane_bytes(L.kdim);
    for (int b = 0; b < kSets; ++b) {
        L.off_pq[b] = o; o = align_up(o + np, 256);
        L.off_pz[b] = o; o = align_up(o + np, 256);
    }
    L.total = o;
    return L;
}

size_t s2_bytes(int n, int r, hts_gemm_mode mode)
{
    const S2Layout L = s2_layout(n, r);
    return mode == HTS_GEMM_EMU_BF16 ? L.total : L.total_fp64;
}

bool bad_matrix(const double *M, int ld, int n) { return M == nullptr || ld < (n > 1 ? n : 1); }

hts_status check_common(hts_ctx *ctx, int n, int r, const double *A, int lda, const double *B, int ldb,
                        hts_comp compq, const double *Q, int ldq, hts_comp compz, const double *Z, int ldz,
                        hts_gemm_mode mode)
{
    if (!ctx || n < 0 || r < 1) return HTS_ERR_ARG;
    if (n == 0) return HTS_OK;
    if (bad_matrix(A, lda, n) || bad_matrix(B, ldb, n)) return HTS_ERR_ARG;
    if (compq < HTS_COMP_NONE || compq > HTS_COMP_UPDATE) return HTS_ERR_ARG;
    if (compz < HTS_COMP_NONE || compz > HTS_COMP_UPDATE) return HTS_ERR_ARG;
    if (compq != HTS_COMP_NONE && bad_matrix(Q, ldq, n)) return HTS_ERR_ARG;
    if (compz != HTS_COMP_NONE && bad_matrix(Z, ldz, n)) return HTS_ERR_ARG;
    if (mode != HTS_GEMM_FP64 && mode != HTS_GEMM_EMU_BF16) return HTS_ERR_ARG;
    return HTS_OK;
}

hts_status cuda_status(cudaError_t e) { return e == cudaSuccess ? HTS_OK : HTS_ERR_CUDA; }

// Scan of the entries a call reads for NaN / Inf (reported as HTS_ERR_NONFINITE by
// hts_sync_status): A on and above its lowA-th subdiagonal, B on and above its lowB-th, and Q,
// Z where the call multiplies into them (HTS_COMP_UPDATE).
hts_status scan_inputs(hts_ctx *ctx, int n, const double *A, int lda, int lowA, const double *B, int ldb, int lowB,
                       hts_comp compq, const double *Q, int ldq, hts_comp compz, const double *Z, int ldz,
                       cudaStream_t st)
{
    int *s = ctx->d_status;
    if (launch_scan_nonfinite(A, lda, n, lowA, 0, s, st) != cudaSuccess) return HTS_ERR_CUDA;
    if (launch_scan_nonfinite(B, ldb, n, lowB, 1, s, st) != cudaSuccess) return HTS_ERR_CUDA;
    if (compq == HTS_COMP_UPDATE && launch_scan_nonfinite(Q, ldq, n, n, 2, s, st) != cudaSuccess) return HTS_ERR_CUDA;
    if (compz == HTS_COMP_UPDATE && launch_scan_nonfinite(Z, ldz, n, n, 3, s, st) != cudaSuccess) return HTS_ERR_CUDA;
    return HTS_OK;
}

// The emulated updates keep one window of r + q - 1 <= 32 indices in the registers of a warp
// and slide it by one 16-wide operand tile per block: r = 16 only, with 8 digits per operand.
hts_status check_emu(hts_gemm_mode mode, int r, int q, const hts_params *p)
{
    if (mode != HTS_GEMM_EMU_BF16) return HTS_OK;
    if (p && p->emu_slices != 0 && p->emu_slices != 8) return HTS_ERR_UNSUPPORTED;
    if (p && p->tile_m != 0 && p->tile_m != 32 && p->tile_m != 64) return HTS_ERR_UNSUPPORTED;
    return emu_supported(r, q) ? HTS_OK : HTS_ERR_UNSUPPORTED;
}

// Block height (in units of r) of stage 1: the paper's p = 8 by default, limited so that one
// p*r x p*r B block fits in shared memory for its RQ (p*r <= 128).
int stage1_p(const hts_params *prm, int r)
{
    const int cap = imax(2, 128 / imax(r, 1));
    if (prm && prm->p > 0) return prm->p;
    return imin(8, cap);
}

// Algorithmic cost of one group's three launches, for the profiler.  Flops: 4 per element
// and reflector (dot product + update).  Bytes: every element a launch must change is read
// and written once (16 bytes).
struct GroupCost {
    double f_gen, b_gen, f_right, b_right, f_qz, b_qz, f_left, b_left;
    double f_stair, b_stair, m_right, m_qz, m_left, f_form;   // emulated mode
};

// First block of row tile T (of `rows` rows) that the emulated right update of A and B does
// not take: blocks k > kT(T) have their whole reflector set pending for every row of T.
int emu_tile_kT(int n, int r, int j1, int qg, int rows, int x)
{
    const int xt = imin(((x - 1) / rows + 1) * rows, n);
    return (xt <= j1) ? -1 : qg + (xt - j1 - 1) / r;
}

GroupCost s2_group_cost(int n, int r, int j1, int qg, bool hasQ, bool hasZ, bool emu)
{
    GroupCost c{};
    const int jl = j1 + qg - 1;
    const int kmax = nblocks_gen(n, r, j1) - 1;
    const int er = 32;   // rows per tile of the emulated right update
    for (int j = j1; j <= jl; ++j) {
        const int kg = nblocks_gen(n, r, j);
        for (int k = 0; k < kg; ++k) {
            const StepGeom g = step_geom(n, r, j1, qg, k, j);
            const double m = g.i2 - g.i1 + 1;
            const double rowsA = imax(0, g.i3 - g.i4 + 1), rowsB = imax(0, g.i2 - g.i4 + 1);
            double rq = 0.0;
            for (int sr = 2; sr <= (int)m; ++sr) rq += 4.0 * sr * (sr - 1 + m);
            c.f_gen += 8.0 * m * (j - j1) + 4.0 * m * m + rq + 4.0 * m * (rowsA + rowsB);
            c.b_gen += 16.0 * (m * (rowsA + rowsB) + m * m + 2.0 * (m + j - j1));
            const double above = g.i4 - 1;   // rows of A and B the apply phase updates
            double stair = 0.0;
            if (emu) {
                // rows x < i4 of tiles with kT >= k stay with the FP64 staircase kernel
                for (int x = 1; x <= (int)above; x += er)
                    if (emu_tile_kT(n, r, j1, qg, er, x) >= k) stair += imin(er, (int)above - x + 1);
            }
            c.f_right += 4.0 * m * 2.0 * (above - stair);
            c.f_stair += 4.0 * m * 2.0 * stair;
            c.f_qz += 4.0 * m * ((hasZ ? n : 0) + (hasQ ? n : 0));
            const int cutA = jl + imax(0, (k - 1) * r + 1);
            const int cutB = imin(jl + (k + 1) * r, n);
            c.f_left += 4.0 * m * ((double)imax(0, n - cutA) + imax(0, n - cutB));
            c.f_form += 2.0 * 4.0 * m * (r + qg - 1);
        }
    }
    // right: rows x of A and B from the first block they need to column n; Z, Q all of it
    double elems = 0.0, stair_elems = 0.0;
    for (int x = 1; x <= n; ++x) {
        const int kf = (x <= j1) ? 0 : (x - j1 - 1) / r + 2;
        if (kf <= kmax) {
            elems += n - (j1 + kf * r);
            if (emu) {
                const int kT = imin(kmax, emu_tile_kT(n, r, j1, qg, er, x));
                if (kT >= kf) stair_elems += imin(n, j1 + kT * r + r + qg - 1) - (j1 + kf * r);
            }
        }
    }
    c.b_right = 16.0 * 2.0 * (elems - stair_elems);
    c.b_stair = 16.0 * 2.0 * stair_elems;
    c.b_qz = 16.0 * ((hasZ ? 1 : 0) + (hasQ ? 1 : 0)) * (double)n * (n - j1);
    // left: column c of A / B from row j1+1 down to the bottom of the lowest block it needs
    double le = 0.0;
    for (int isB = 0; isB < 2; ++isB)
        for (int k = kmax; k >= 0; --k) {
            const int cut = isB ? imin(jl + (k + 1) * r, n) : jl + imax(0, (k - 1) * r + 1);
            const int cutn = (k < kmax) ? (isB ? imin(jl + (k + 2) * r, n) : jl + imax(0, k * r + 1)) : n;
            // columns in (cut, cutn] have block k as their lowest block
            const int ncol = imax(0, imin(cutn, n) - cut);
            const int rows = imin(n, j1 + qg - 1 + (k + 1) * r) - j1;
            le += (double)ncol * rows;
        }
    c.b_left = 16.0 * le;
    if (emu) {
        // tensor-core work: 288 mma.m16n8k16 (4096 flops each) per 16-line slab and window step
        const double step = (er / 16) * 288.0 * 4096.0;   // one tile: 288 mma per 16-line slab
        const int ntile = (n + er - 1) / er;
        for (int t = 0; t < ntile; ++t) {
            const int l0 = t * er + 1, llast = imin(l0 + er - 1, n);
            const int kT = (llast <= j1) ? -1 : qg + (llast - j1 - 1) / r;
            if (kmax > kT) c.m_right += 2.0 * step * (kmax - kT);
            c.m_qz += step * (kmax + 1) * ((hasZ ? 1 : 0) + (hasQ ? 1 : 0));
            for (int isB = 0; isB < 2; ++isB)
                for (int k = kmax; k >= 0; --k) {
                    const int cut = isB ? imin(jl + (k + 1) * r, n) : jl + imax(0, (k - 1) * r + 1);
                    if (cut < llast) { c.m_left += step * (k + 1); break; }
                }
        }
    }
    return c;
}

}  // namespace

// Bytes of caller scratch stage 2 alone needs in native FP64 mode (two reflector sets and
// the progress words).
size_t stage2_workspace_bytes(int n, int r) { return s2_layout(n, r).total_fp64; }

// ... and in the given update mode (the emulated mode adds the digit planes).
size_t stage2_workspace_bytes_mode(int n, int r, hts_gemm_mode mode) { return s2_bytes(n, r, mode); }

namespace {

struct S2Ptrs {
    ReflectorSet R[kSets];
    uint2 *PQ[kSets], *PZ[kSets];
    double *gram[kSets];
    unsigned long long *fl, *tfl;
    unsigned *tick;
};

S2Ptrs s2_ptrs(const S2Layout &L, void *work)
{
    S2Ptrs P;
    char *w = static_cast<char *>(work);
    for (int b = 0; b < kSets; ++b) {
        P.PQ[b] = reinterpret_cast<uint2 *>(w + L.off_pq[b]);
        P.PZ[b] = reinterpret_cast<uint2 *>(w + L.off_pz[b]);
        P.R[b].VQ = reinterpret_cast<double *>(w + L.off_vq[b]);
        P.R[b].TQ = reinterpret_cast<double *>(w + L.off_tq[b]);
        P.R[b].VZ = reinterpret_cast<double *>(w + L.off_vz[b]);
        P.R[b].TZ = reinterpret_cast<double *>(w + L.off_tz[b]);
        P.R[b].kdim = L.kdim;
        P.gram[b] = reinterpret_cast<double *>(w + L.off_gram[b]);
    }
    P.fl = reinterpret_cast<unsigned long long *>(w + L.off_flags);
    P.tfl = reinterpret_cast<unsigned long long *>(w + L.off_tflags);
    P.tick = reinterpret_cast<unsigned *>(w + L.off_tick);
    return P;
}

EmuArgs emu_args(double *M0, int ld0, int kind0, double *M1, int ld1, int kind1, int n, int r, int j1, int qg,
                 const S2Ptrs &P, int set, const int *status)
{
    EmuArgs e;
    e.M[0] = M0; e.ld[0] = ld0; e.kind[0] = kind0;
    e.M[1] = M1; e.ld[1] = ld1; e.kind[1] = kind1;
    for (int i = 2; i < 4; ++i) { e.M[i] = nullptr; e.ld[i] = 1; e.kind[i] = 0; }
    e.n = n; e.r = r; e.j1 = j1; e.qg = qg;
    e.planesQ = P.PQ[set]; e.planesZ = P.PZ[set]; e.R = P.R[set]; e.status = status;
    return e;
}

ApplyArgs apply_args(double *M0, int ld0, int kind0, double *M1, int ld1, int kind1, int n, int r, int j1, int qg,
                     const S2Ptrs &P, int set, const int *status)
{
    ApplyArgs a;
    a.M[0] = M0; a.ld[0] = ld0; a.kind[0] = kind0;
    a.M[1] = M1; a.ld[1] = ld1; a.kind[1] = kind1;
    for (int i = 2; i < 4; ++i) { a.M[i] = nullptr; a.ld[i] = 1; a.kind[i] = 0; }
    a.n = n; a.r = r; a.j1 = j1; a.qg = qg; a.R = P.R[set]; a.status = status;
    return a;
}

// One look-ahead update launch (schedule.cuh): A / B updates of the group (j1, qg, set), Q / Z
// update of the group (pj1, pqg, pset), persistent blocks on the SMs the next chase leaves free.
cudaError_t launch_update(hts_ctx *ctx, bool emu, const UpdSched &us, double *A, int lda, double *B, int ldb,
                          double *const *qzM, const int *qzld, const int *qzkind, int n, int r, int j1, int qg,
                          int set, int pj1, int pqg, int pset, int q, const S2Ptrs &P, const CUtensorMap *maps,
                          cudaStream_t st)
{
    if (us.P.total <= 0) return cudaSuccess;
    const int workers = maps ? update_tc_workers() : emu ? update_emu_workers() : update_fp64_workers();
    int ctas = imax(1, ctx->num_sms - 2 * q);
    ctas = imin(ctas, (us.P.total + workers - 1) / workers);
    int *status = ctx->d_status;
    if (maps) {
        // tensor-core kernel: maps[2 s] / maps[2 s + 1] are the Z / Q planes of set s
        UpdTcArgs ua;
        ua.map_z = maps[2 * set];
        ua.map_q = maps[2 * set + 1];
        ua.map_qz_z = maps[2 * pset];
        ua.map_qz_q = maps[2 * pset + 1];
        ua.right = emu_args(A, lda, 0, B, ldb, 1, n, r, j1, qg, P, set, status);
        ua.left = emu_args(A, lda, 4, B, ldb, 5, n, r, j1, qg, P, set, status);
        ua.qz = emu_args(qzM[0], qzld[0], qzkind[0], qzM[1], qzld[1], qzkind[1], n, r, pj1, pqg, P, pset, status);
        ua.s = us;
        return launch_s2_update_tc(ua, ctas, st);
    }
    if (emu) {
        UpdEmuArgs ua;
        ua.right = emu_args(A, lda, 0, B, ldb, 1, n, r, j1, qg, P, set, status);
        ua.left = emu_args(A, lda, 4, B, ldb, 5, n, r, j1, qg, P, set, status);
        ua.qz = emu_args(qzM[0], qzld[0], qzkind[0], qzM[1], qzld[1], qzkind[1], n, r, pj1, pqg, P, pset, status);
        ua.s = us;
        return launch_s2_update_emu(ua, ctas, st);
    }
    UpdFp64Args uf;
    uf.right = apply_args(A, lda, 0, B, ldb, 1, n, r, j1, qg, P, set, status);
    uf.qz = apply_args(qzM[0], qzld[0], qzkind[0], qzM[1], qzld[1], qzkind[1], n, r, pj1, pqg, P, pset, status);
    uf.left.A = A; uf.left.B = B; uf.left.lda = lda; uf.left.ldb = ldb;
    uf.left.n = n; uf.left.r = r; uf.left.j1 = j1; uf.left.qg = qg; uf.left.R = P.R[set]; uf.left.status = status;
    uf.s = us;
    uf.smem_doubles = update_fp64_smem_doubles(r, q);
    return launch_s2_update_fp64(uf, ctas, st);
}

}  // namespace

// Stage 2 driver: the group loop of generate / apply launches.  Default (look-ahead, Section
// "Parallel stage two"): per group g on the caller's stream the chase (Alg. 3) and, in emulated
// mode, the block formation; then on the update stream one persistent launch with g's A / B
// updates and g-1's Q / Z update (Alg. 4), beside the chase of group g+1, which waits tile by
// tile for the A / B elements it touches (schedule.cuh).  With HTS_FLAG_SERIAL_UPDATES each
// group's A / B updates follow its chase on the caller's stream and only the Q / Z update
// overlaps the next chase (side stream).
hts_status run_stage2(hts_ctx *ctx, int n, int r, double *A, int lda, double *B, int ldb,
                      double *Q, int ldq, double *Z, int ldz, int q, int flags, int tile_m, hts_gemm_mode mode,
                      void *work, cudaStream_t st)
{
    if (n <= 2 || r <= 1) return HTS_OK;
    const S2Layout L = s2_layout(n, r);
    const S2Ptrs P = s2_ptrs(L, work);
    const bool emu = mode == HTS_GEMM_EMU_BF16;
    const bool lookahead = !(flags & HTS_FLAG_SERIAL_UPDATES);
    int *status = ctx->d_status;
    cudaError_t e = cudaMemsetAsync(static_cast<char *>(work) + L.off_flags, 0, L.total_fp64 - L.off_flags, st);
    if (e != cudaSuccess) return HTS_ERR_CUDA;
    const bool qz = (Q != nullptr) || (Z != nullptr);
    const int nqz = (Z ? 1 : 0) + (Q ? 1 : 0);
    double *qzM[2] = {Z ? Z : Q, Z ? Q : nullptr};
    const int qzld[2] = {Z ? ldz : ldq, ldq};
    const int qzkind[2] = {Z ? 2 : 3, 3};
    cudaStream_t side = lookahead ? ctx->upd : ctx->side;
    // the emulated look-ahead updates run on the tcgen05 kernel (64-line tiles) unless the
    // mma.sync kernel (32-line tiles) is asked for or the tensor maps cannot be made
    CUtensorMap maps[2 * kSets];
    bool tc = emu && lookahead && tile_m != 32 && update_tc_supported(r, q);
    for (int b = 0; tc && b < kSets; ++b)
        tc = encode_plane_map(&maps[2 * b], P.PZ[b], L.kdim) == cudaSuccess &&
             encode_plane_map(&maps[2 * b + 1], P.PQ[b], L.kdim) == cudaSuccess;
    const int TL = tc ? update_tc_lines() : 32;

    int group = 0, prev_set = 0, prev_j1 = 0, prev_qg = 0;
    TaskPlan prev_plan = task_plan(n, r, 1, 1, false, 0, TL);
    GroupCost prev_gc{};
    for (int j1 = 1; j1 <= n - 2; j1 += q, ++group) {
        const int qg = imin(q, n - 2 - j1 + 1);
        const int set = group % kSets;
        const GroupCost gc = ctx->prof.enabled ? s2_group_cost(n, r, j1, qg, Q != nullptr, Z != nullptr, emu)
                                               : GroupCost{};
        // set g mod 3 was last read by the update launch of group g-2 (Q / Z of group g-3)
        if (lookahead && group >= 2 && cudaStreamWaitEvent(st, ctx->ev_upd[(group - 2) % kSets], 0) != cudaSuccess)
            return HTS_ERR_CUDA;
        if (!lookahead && qz && group >= 3 && cudaStreamWaitEvent(st, ctx->ev_qz[set], 0) != cudaSuccess)
            return HTS_ERR_CUDA;

        GenArgs ga;
        ga.A = A; ga.B = B; ga.lda = lda; ga.ldb = ldb;
        ga.n = n; ga.r = r; ga.j1 = j1; ga.qg = qg; ga.group = group;
        ga.R = P.R[set]; ga.flags = P.fl; ga.qmax = L.qmax;
        ga.gram = P.gram[set];
        ga.epoch = (unsigned long long)(group + 1) << 32;
        ga.status = status;
        ga.stall = (flags & HTS_FLAG_TEST_STALL) ? 1 : 0;
        ga.direct_rq = (flags & HTS_FLAG_TEST_DIRECT_RQ) ? 1 : 0;
        ga.uflags = (lookahead && group >= 1) ? P.tfl : nullptr;
        ga.uplan = prev_plan;
        ga.uepoch = (unsigned long long)group;   // the previous group's update publishes group
        {
            ProfScope ps(ctx, st);
            e = (r <= 16) ? launch_s2_chase16(ga, st) : launch_s2_generate(ga, st);
            if (e != cudaSuccess) return HTS_ERR_CUDA;
            ps.done(HTS_K_GENERATE, gc.f_gen, gc.b_gen);
        }
        if (emu) {
            FormUArgs fa;
            fa.n = n; fa.r = r; fa.j1 = j1; fa.qg = qg; fa.R = P.R[set];
            fa.planesQ = P.PQ[set]; fa.planesZ = P.PZ[set]; fa.status = status; fa.umma = tc ? 1 : 0;
            ProfScope ps(ctx, st);
            if ((e = launch_s2_form_u(fa, st)) != cudaSuccess) return HTS_ERR_CUDA;
            ps.done(HTS_K_FORM_U, gc.f_form, 0.0);
        }

        if (lookahead) {
            if (cudaEventRecord(ctx->ev_gen[set], st) != cudaSuccess) return HTS_ERR_CUDA;
            if (cudaStreamWaitEvent(side, ctx->ev_gen[set], 0) != cudaSuccess) return HTS_ERR_CUDA;
            const int nq = group >= 1 ? nqz : 0;
            UpdSched us;
            us.P = task_plan(n, r, j1, qg, true, nq, TL);
            us.tflags = P.tfl; us.epoch = (unsigned long long)(group + 1); us.ticket = P.tick + group;
            us.status = status; us.group = group; us.n = n; us.r = r;
            ProfScope ps(ctx, side);
            if ((e = launch_update(ctx, emu, us, A, lda, B, ldb, qzM, qzld, qzkind, n, r, j1, qg, set, prev_j1, prev_qg,
                                   prev_set, q, P, tc ? maps : nullptr, side)) != cudaSuccess)
                return HTS_ERR_CUDA;
            ps.done(HTS_K_UPDATE, gc.f_right + gc.f_stair + gc.f_left + (nq ? prev_gc.f_qz : 0.0),
                    gc.b_right + gc.b_stair + gc.b_left + (nq ? prev_gc.b_qz : 0.0),
                    emu ? gc.m_right + gc.m_left + (nq ? prev_gc.m_qz : 0.0) : 0.0);
            if (cudaEventRecord(ctx->ev_upd[group % kSets], side) != cudaSuccess) return HTS_ERR_CUDA;
            prev_plan = us.P;
        } else {
            if (emu) {
                const EmuArgs ea = emu_args(A, lda, 0, B, ldb, 1, n, r, j1, qg, P, set, status);
                ProfScope ps(ctx, st);
                if ((e = launch_s2_emu_apply(ea, 2, st)) != cudaSuccess) return HTS_ERR_CUDA;
                ps.done(HTS_K_EMU_RIGHT, gc.f_right + gc.f_stair, gc.b_right + gc.b_stair, gc.m_right);
                const EmuArgs el = emu_args(A, lda, 4, B, ldb, 5, n, r, j1, qg, P, set, status);
                ProfScope pl(ctx, st);
                if ((e = launch_s2_emu_apply(el, 2, st)) != cudaSuccess) return HTS_ERR_CUDA;
                pl.done(HTS_K_EMU_LEFT, gc.f_left, gc.b_left, gc.m_left);
            } else {
                const ApplyArgs aa = apply_args(A, lda, 0, B, ldb, 1, n, r, j1, qg, P, set, status);
                ProfScope ps(ctx, st);
                if ((e = launch_s2_apply_right(aa, 2, st)) != cudaSuccess) return HTS_ERR_CUDA;
                ps.done(HTS_K_APPLY_RIGHT, gc.f_right, gc.b_right);
                LeftArgs la;
                la.A = A; la.B = B; la.lda = lda; la.ldb = ldb;
                la.n = n; la.r = r; la.j1 = j1; la.qg = qg; la.R = P.R[set]; la.status = status;
                ProfScope pl(ctx, st);
                if ((e = launch_s2_apply_left(la, st)) != cudaSuccess) return HTS_ERR_CUDA;
                pl.done(HTS_K_APPLY_LEFT, gc.f_left, gc.b_left);
            }
            // Q and Z on the side stream after this group's A / B updates, beside the next chase
            if (qz) {
                if (cudaEventRecord(ctx->ev_gen[set], st) != cudaSuccess) return HTS_ERR_CUDA;
                if (cudaStreamWaitEvent(side, ctx->ev_gen[set], 0) != cudaSuccess) return HTS_ERR_CUDA;
                ProfScope ps(ctx, side);
                if (emu) {
                    const EmuArgs eq = emu_args(qzM[0], qzld[0], qzkind[0], qzM[1], qzld[1], qzkind[1], n, r, j1, qg, P,
                                                set, status);
                    if ((e = launch_s2_emu_apply(eq, nqz, side)) != cudaSuccess) return HTS_ERR_CUDA;
                    ps.done(HTS_K_EMU_QZ, gc.f_qz, gc.b_qz, gc.m_qz);
                } else {
                    const ApplyArgs aq = apply_args(qzM[0], qzld[0], qzkind[0], qzM[1], qzld[1], qzkind[1], n, r, j1,
                                                    qg, P, set, status);
                    if ((e = launch_s2_apply_right(aq, nqz, side)) != cudaSuccess) return HTS_ERR_CUDA;
                    ps.done(HTS_K_APPLY_QZ, gc.f_qz, gc.b_qz);
                }
                if (cudaEventRecord(ctx->ev_qz[set], side) != cudaSuccess) return HTS_ERR_CUDA;
            }
        }
        prev_gc = gc;
        prev_set = set;
        prev_j1 = j1;
        prev_qg = qg;
    }
    if (lookahead) {
        int last = group - 1;   // index of the last update launch
        if (qz) {
            // the closing launch: the last group's Q / Z update
            UpdSched us;
            us.P = task_plan(n, r, 1, 1, false, nqz, TL);
            us.tflags = P.tfl; us.epoch = (unsigned long long)(group + 1); us.ticket = P.tick + group;
            us.status = status; us.group = group; us.n = n; us.r = r;
            ProfScope ps(ctx, side);
            if ((e = launch_update(ctx, emu, us, A, lda, B, ldb, qzM, qzld, qzkind, n, r, prev_j1, prev_qg, prev_set,
                                   prev_j1, prev_qg, prev_set, q, P, tc ? maps : nullptr, side)) != cudaSuccess)
                return HTS_ERR_CUDA;
            ps.done(HTS_K_UPDATE, prev_gc.f_qz, prev_gc.b_qz, emu ? prev_gc.m_qz : 0.0);
            if (cudaEventRecord(ctx->ev_upd[group % kSets], side) != cudaSuccess) return HTS_ERR_CUDA;
            last = group;
        }
        if (last >= 0 && cudaStreamWaitEvent(st, ctx->ev_upd[last % kSets], 0) != cudaSuccess) return HTS_ERR_CUDA;
    } else if (qz && group >= 1 && cudaStreamWaitEvent(st, ctx->ev_qz[(group - 1) % kSets], 0) != cudaSuccess) {
        return HTS_ERR_CUDA;
    }
    if (!(flags & HTS_FLAG_NO_CLEAN)) {
        ProfScope ps(ctx, st);
        if ((e = launch_zero_below(A, lda, n, 1, status, st)) != cudaSuccess) return HTS_ERR_CUDA;
        if ((e = launch_zero_below(B, ldb, n, 0, status, st)) != cudaSuccess) return HTS_ERR_CUDA;
        ps.done(HTS_K_UTIL, 0.0, 0.0);
    }
    return HTS_OK;
}

}  // namespace hts

using namespace hts;

extern "C" {

const char *hts_status_string(hts_status s)
{
    switch (s) {
    case HTS_OK: return "HTS_OK";
    case HTS_ERR_ARG: return "HTS_ERR_ARG";
    case HTS_ERR_CUDA: return "HTS_ERR_CUDA";
    case HTS_ERR_WORKSPACE: return "HTS_ERR_WORKSPACE";
    case HTS_ERR_TIMEOUT: return "HTS_ERR_TIMEOUT";
    case HTS_ERR_NONFINITE: return "HTS_ERR_NONFINITE";
    case HTS_ERR_UNSUPPORTED: return "HTS_ERR_UNSUPPORTED";
    }
    return "unknown hts_status";
}

hts_status hts_create(hts_ctx **ctx, int device)
{
    if (!ctx) return HTS_ERR_ARG;
    *ctx = nullptr;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) return HTS_ERR_CUDA;
    DeviceGuard g(device);
    if (!g.ok) return HTS_ERR_CUDA;
    hts_ctx *c = static_cast<hts_ctx *>(std::calloc(1, sizeof(hts_ctx)));
    if (!c) return HTS_ERR_CUDA;
    c->device = device;
    int lo_prio = 0, hi_prio = 0;
    bool ok = cudaMalloc(&c->d_status, kStatusWords * sizeof(int)) == cudaSuccess &&
              cudaMemset(c->d_status, 0, kStatusWords * sizeof(int)) == cudaSuccess &&
              cudaMallocHost(&c->h_status, kStatusWords * sizeof(int)) == cudaSuccess &&
              cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device) == cudaSuccess &&
              cudaDeviceGetStreamPriorityRange(&lo_prio, &hi_prio) == cudaSuccess &&
              cudaStreamCreateWithPriority(&c->side, cudaStreamNonBlocking, lo_prio) == cudaSuccess &&
              cudaStreamCreateWithPriority(&c->upd, cudaStreamNonBlocking, lo_prio) == cudaSuccess &&
              cublasCreate(&c->blas) == CUBLAS_STATUS_SUCCESS;
    for (int b = 0; ok && b < 3; ++b)
        ok = cudaEventCreateWithFlags(&c->ev_gen[b], cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&c->ev_qz[b], cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&c->ev_upd[b], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        hts_destroy(c);
        return HTS_ERR_CUDA;
    }
    *ctx = c;
    return HTS_OK;
}

void hts_destroy(hts_ctx *ctx)
{
    if (!ctx) return;
    DeviceGuard g(ctx->device);
    if (ctx->prof.cap > 0) {
        hts_kernel_profile tmp[HTS_K_NKINDS];
        hts_profile_end(ctx, tmp, nullptr);
    }
    if (ctx->side) cudaStreamSynchronize(ctx->side);
    if (ctx->upd) cudaStreamSynchronize(ctx->upd);
    for (int b = 0; b < 3; ++b) {
        if (ctx->ev_gen[b]) cudaEventDestroy(ctx->ev_gen[b]);
        if (ctx->ev_qz[b]) cudaEventDestroy(ctx->ev_qz[b]);
        if (ctx->ev_upd[b]) cudaEventDestroy(ctx->ev_upd[b]);
    }
    if (ctx->blas) cublasDestroy(ctx->blas);
    if (ctx->side) cudaStreamDestroy(ctx->side);
    if (ctx->upd) cudaStreamDestroy(ctx->upd);
    if (ctx->d_status) cudaFree(ctx->d_status);
    if (ctx->h_status) cudaFreeHost(ctx->h_status);
    std::free(ctx);
}

hts_status hts_workspace_size(int n, int r, const hts_params *p, size_t *bytes)
{
    if (!bytes || n < 0 || r < 1) return HTS_ERR_ARG;
    const size_t s2 = s2_layout(n, r).total;   // covers both update modes
    const size_t s01 = stage01_workspace_bytes(n, r, stage1_p(p, r));
    *bytes = s2 > s01 ? s2 : s01;
    return HTS_OK;
}

hts_status hts_reduce_stage2(hts_ctx *ctx, int n, int r, double *A, int lda, double *B, int ldb,
                             hts_comp compq, double *Q, int ldq, hts_comp compz, double *Z, int ldz,
                             hts_gemm_mode mode, const hts_params *p, void *work, size_t work_bytes,
                             void *stream)
{
    hts_status s = check_common(ctx, n, r, A, lda, B, ldb, compq, Q, ldq, compz, Z, ldz, mode);
    if (s != HTS_OK || n == 0) return s;
    if (r > kMaxR) return HTS_ERR_UNSUPPORTED;
    int q = (p && p->q > 0) ? p->q : r;
    if (q > r) return HTS_ERR_ARG;
    if ((s = check_emu(mode, r, q, p)) != HTS_OK) return s;
    const int flags = p ? p->flags : 0;
    const bool needs_work = n > 2 && r > 1;
    if (needs_work) {
        if (!work || (reinterpret_cast<uintptr_t>(work) & 255u)) return HTS_ERR_WORKSPACE;
        if (work_bytes < s2_bytes(n, r, mode)) return HTS_ERR_WORKSPACE;
    }
    DeviceGuard g(ctx->device);
    if (!g.ok) return HTS_ERR_CUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    double *Qp = compq == HTS_COMP_NONE ? nullptr : Q;
    double *Zp = compz == HTS_COMP_NONE ? nullptr : Z;
    {
        ProfScope ps(ctx, st);
        if ((s = scan_inputs(ctx, n, A, lda, r, B, ldb, 0, compq, Q, ldq, compz, Z, ldz, st)) != HTS_OK) return s;
        ps.done(HTS_K_UTIL, 0.0, 0.0);
    }
    if (compq == HTS_COMP_INIT || compz == HTS_COMP_INIT) {
        ProfScope ps(ctx, st);
        if (compq == HTS_COMP_INIT && (s = cuda_status(launch_set_identity(Q, ldq, n, st))) != HTS_OK) return s;
        if (compz == HTS_COMP_INIT && (s = cuda_status(launch_set_identity(Z, ldz, n, st))) != HTS_OK) return s;
        ps.done(HTS_K_UTIL, 0.0, 0.0);
    }
    return run_stage2(ctx, n, r, A, lda, B, ldb, Qp, ldq, Zp, ldz, q, flags, p ? p->tile_m : 0, mode, work, st);
}

static hts_status check_stage1_args(hts_ctx *ctx, int n, int r, const hts_params *p, void *work, size_t work_bytes)
{
    if (r >= n) return HTS_ERR_ARG;
    if (r > 64) return HTS_ERR_UNSUPPORTED;
    const int pp = stage1_p(p, r);
    if (pp < 2) return HTS_ERR_ARG;
    if (pp * r > 128) return HTS_ERR_UNSUPPORTED;
    size_t need = 0;
    hts_workspace_size(n, r, p, &need);
    if (!work || (reinterpret_cast<uintptr_t>(work) & 255u) || work_bytes < need) return HTS_ERR_WORKSPACE;
    (void)ctx;
    return HTS_OK;
}

hts_status hts_reduce_stage1(hts_ctx *ctx, int n, int r, double *A, int lda, double *B, int ldb,
                             hts_comp compq, double *Q, int ldq, hts_comp compz, double *Z, int ldz,
                             hts_gemm_mode mode, const hts_params *p, void *work, size_t work_bytes,
                             void *stream)
{
    hts_status s = check_common(ctx, n, r, A, lda, B, ldb, compq, Q, ldq, compz, Z, ldz, mode);
    if (s != HTS_OK || n == 0) return s;
    if (mode != HTS_GEMM_FP64) return HTS_ERR_UNSUPPORTED;
    if ((s = check_stage1_args(ctx, n, r, p, work, work_bytes)) != HTS_OK) return s;
    DeviceGuard g(ctx->device);
    if (!g.ok) return HTS_ERR_CUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    double *Qp = compq == HTS_COMP_NONE ? nullptr : Q;
    double *Zp = compz == HTS_COMP_NONE ? nullptr : Z;
    ProfScope ps(ctx, st);
    if ((s = scan_inputs(ctx, n, A, lda, n, B, ldb, 0, compq, Q, ldq, compz, Z, ldz, st)) != HTS_OK) return s;
    if (compq == HTS_COMP_INIT && launch_set_identity(Q, ldq, n, st) != cudaSuccess) return HTS_ERR_CUDA;
    if (compz == HTS_COMP_INIT && launch_set_identity(Z, ldz, n, st) != cudaSuccess) return HTS_ERR_CUDA;
    if (launch_zero_below(B, ldb, n, 0, ctx->d_status, st) != cudaSuccess) return HTS_ERR_CUDA;
    if (run_stage1(ctx->blas, n, r, stage1_p(p, r), A, lda, B, ldb, Qp, ldq, Zp, ldz, work, st) != cudaSuccess)
        return HTS_ERR_CUDA;
    ps.done(HTS_K_STAGE1, 0.0, 0.0);
    return HTS_OK;
}

hts_status hts_reduce(hts_ctx *ctx, int n, int r, double *A, int lda, double *B, int ldb,
                      hts_comp compq, double *Q, int ldq, hts_comp compz, double *Z, int ldz,
                      hts_gemm_mode mode, const hts_params *p, void *work, size_t work_bytes, void *stream)
{
    hts_status s = check_common(ctx, n, r, A, lda, B, ldb, compq, Q, ldq, compz, Z, ldz, mode);
    if (s != HTS_OK || n == 0) return s;
    if (n <= 2) {
        // a 1 x 1 or 2 x 2 pencil is in HT form once B is triangular: stage 0 alone
        size_t need = 0;
        hts_workspace_size(n, r, p, &need);
        if (!work || (reinterpret_cast<uintptr_t>(work) & 255u) || work_bytes < need) return HTS_ERR_WORKSPACE;
        DeviceGuard g(ctx->device);
        if (!g.ok) return HTS_ERR_CUDA;
        cudaStream_t st = static_cast<cudaStream_t>(stream);
        if ((s = scan_inputs(ctx, n, A, lda, n, B, ldb, n, compq, Q, ldq, compz, Z, ldz, st)) != HTS_OK) return s;
        if (compq == HTS_COMP_INIT && launch_set_identity(Q, ldq, n, st) != cudaSuccess) return HTS_ERR_CUDA;
        if (compz == HTS_COMP_INIT && launch_set_identity(Z, ldz, n, st) != cudaSuccess) return HTS_ERR_CUDA;
        if (run_stage0(ctx->blas, n, A, lda, B, ldb, compq == HTS_COMP_NONE ? nullptr : Q, ldq, work, r, stage1_p(p, r),
                       st) != cudaSuccess)
            return HTS_ERR_CUDA;
        return HTS_OK;
    }
    if ((s = check_stage1_args(ctx, n, r, p, work, work_bytes)) != HTS_OK) return s;
    if (r > kMaxR) return HTS_ERR_UNSUPPORTED;
    int q = (p && p->q > 0) ? p->q : r;
    if (q > r) return HTS_ERR_ARG;
    if ((s = check_emu(mode, r, q, p)) != HTS_OK) return s;
    DeviceGuard g(ctx->device);
    if (!g.ok) return HTS_ERR_CUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    double *Qp = compq == HTS_COMP_NONE ? nullptr : Q;
    double *Zp = compz == HTS_COMP_NONE ? nullptr : Z;
    {
        ProfScope ps(ctx, st);
        if ((s = scan_inputs(ctx, n, A, lda, n, B, ldb, n, compq, Q, ldq, compz, Z, ldz, st)) != HTS_OK) return s;
        if (compq == HTS_COMP_INIT && launch_set_identity(Q, ldq, n, st) != cudaSuccess) return HTS_ERR_CUDA;
        if (compz == HTS_COMP_INIT && launch_set_identity(Z, ldz, n, st) != cudaSuccess) return HTS_ERR_CUDA;
        if (run_stage0(ctx->blas, n, A, lda, B, ldb, Qp, ldq, work, r, stage1_p(p, r), st) != cudaSuccess) return HTS_ERR_CUDA;
        if (run_stage1(ctx->blas, n, r, stage1_p(p, r), A, lda, B, ldb, Qp, ldq, Zp, ldz, work, st) != cudaSuccess)
            return HTS_ERR_CUDA;
        ps.done(HTS_K_STAGE1, 0.0, 0.0);
    }
    return run_stage2(ctx, n, r, A, lda, B, ldb, Qp, ldq, Zp, ldz, q, p ? p->flags : 0, p ? p->tile_m : 0, mode, work,
                      st);
}

hts_status hts_workspace_size_batched(int count, const int *n, const int *r, const hts_params *p, size_t *bytes)
{
    (void)p;
    if (!bytes || count < 0 || (count > 0 && (!n || !r))) return HTS_ERR_ARG;
    for (int i = 0; i < count; ++i)
        if (n[i] < 0 || r[i] < 1) return HTS_ERR_ARG;
    *bytes = batch_work_bytes(count) + 256;
    return HTS_OK;
}

namespace {

// Argument checks shared by the batched calls; *pp receives stage 1's p (0: the default).
hts_status check_batched(int count, const int *n, const int *r, double *const *A, const int *lda, double *const *B,
                         const int *ldb, hts_comp compq, double *const *Q, const int *ldq, hts_comp compz,
                         double *const *Z, const int *ldz, hts_gemm_mode mode, const hts_params *p, int *pp)
{
    if (!n || !r || !A || !lda || !B || !ldb) return HTS_ERR_ARG;
    if (compq < HTS_COMP_NONE || compq > HTS_COMP_UPDATE || compz < HTS_COMP_NONE || compz > HTS_COMP_UPDATE)
        return HTS_ERR_ARG;
    if ((compq != HTS_COMP_NONE && (!Q || !ldq)) || (compz != HTS_COMP_NONE && (!Z || !ldz))) return HTS_ERR_ARG;
    if (mode != HTS_GEMM_FP64 && mode != HTS_GEMM_EMU_BF16) return HTS_ERR_ARG;
    if (mode != HTS_GEMM_FP64) return HTS_ERR_UNSUPPORTED;
    *pp = (p && p->p > 0) ? p->p : 0;
    if (p && p->tile_n < 0) return HTS_ERR_ARG;
    for (int i = 0; i < count; ++i) {
        if (n[i] < 1 || r[i] < 1 || (n[i] > 2 && r[i] >= n[i])) return HTS_ERR_ARG;
        if (bad_matrix(A[i], lda[i], n[i]) || bad_matrix(B[i], ldb[i], n[i])) return HTS_ERR_ARG;
        if (compq != HTS_COMP_NONE && bad_matrix(Q[i], ldq[i], n[i])) return HTS_ERR_ARG;
        if (compz != HTS_COMP_NONE && bad_matrix(Z[i], ldz[i], n[i])) return HTS_ERR_ARG;
        if (n[i] > batch_max_n() || r[i] > 16) return HTS_ERR_UNSUPPORTED;
        const int pe = *pp > 0 ? *pp : imin(8, imax(2, batch_max_block() / r[i]));
        if (pe < 2 || pe * r[i] > batch_max_block()) return HTS_ERR_UNSUPPORTED;
    }
    return HTS_OK;
}

bool batch_work_ok(const void *work, size_t work_bytes, int count)
{
    return work && !(reinterpret_cast<uintptr_t>(work) & 255u) && work_bytes >= batch_work_bytes(count);
}

}  // namespace

hts_status hts_plan_batched(hts_ctx *ctx, int count, const int *n, const int *r, double *const *A, const int *lda,
                            double *const *B, const int *ldb, hts_comp compq, double *const *Q, const int *ldq,
                            hts_comp compz, double *const *Z, const int *ldz, hts_gemm_mode mode,
                            const hts_params *p, void *work, size_t work_bytes, void *stream)
{
    if (!ctx || count < 1) return HTS_ERR_ARG;
    int pp = 0;
    const hts_status cs = check_batched(count, n, r, A, lda, B, ldb, compq, Q, ldq, compz, Z, ldz, mode, p, &pp);
    if (cs != HTS_OK) return cs;
    if (!batch_work_ok(work, work_bytes, count)) return HTS_ERR_WORKSPACE;
    DeviceGuard g(ctx->device);
    if (!g.ok) return HTS_ERR_CUDA;
    // the workspace image (descriptors and the largest-first order) staged on the host; a copy
    // from pageable memory is staged by the runtime before cudaMemcpyAsync returns
    std::vector<unsigned char> img(batch_work_bytes(count));
    batch_stage(img.data(), count, n, r, A, lda, B, ldb, Q, ldq, Z, ldz, (int)compq, (int)compz, pp);
    if (cudaMemcpyAsync(work, img.data(), img.size(), cudaMemcpyHostToDevice, static_cast<cudaStream_t>(stream)) !=
        cudaSuccess)
        return HTS_ERR_CUDA;
    ctx->batch_per_sm = p ? p->tile_n : 0;
    return HTS_OK;
}

hts_status hts_reduce_batched_planned(hts_ctx *ctx, int count, void *work, size_t work_bytes, void *stream)
{
    if (!ctx || count < 1) return HTS_ERR_ARG;
    if (!batch_work_ok(work, work_bytes, count)) return HTS_ERR_WORKSPACE;
    DeviceGuard g(ctx->device);
    if (!g.ok) return HTS_ERR_CUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    ProfScope ps(ctx, st);
    if (launch_reduce_batched(work, count, ctx->num_sms, ctx->batch_per_sm, ctx->d_status, st) != cudaSuccess)
        return HTS_ERR_CUDA;
    ps.done(HTS_K_BATCH, 0.0, 0.0);
    return HTS_OK;
}

hts_status hts_reduce_batched(hts_ctx *ctx, int count, const int *n, const int *r,
                              double *const *A, const int *lda, double *const *B, const int *ldb,
                              hts_comp compq, double *const *Q, const int *ldq,
                              hts_comp compz, double *const *Z, const int *ldz,
                              hts_gemm_mode mode, const hts_params *p, void *work, size_t work_bytes,
                              void *stream)
{
    if (!ctx || count < 0) return HTS_ERR_ARG;
    if (count == 0) return HTS_OK;
    const hts_status s = hts_plan_batched(ctx, count, n, r, A, lda, B, ldb, compq, Q, ldq, compz, Z, ldz, mode, p,
                                          work, work_bytes, stream);
    if (s != HTS_OK) return s;
    return hts_reduce_batched_planned(ctx, count, work, work_bytes, stream);
}

hts_status hts_fallback_count(hts_ctx *ctx, void *stream, long long *count)
{
    if (!ctx || !count) return HTS_ERR_ARG;
    DeviceGuard g(ctx->device);
    if (!g.ok) return HTS_ERR_CUDA;
    if (cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess) return HTS_ERR_CUDA;
    int v = 0;
    if (cudaMemcpy(&v, ctx->d_status + kStatusFallbacks, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemset(ctx->d_status + kStatusFallbacks, 0, sizeof(int)) != cudaSuccess)
        return HTS_ERR_CUDA;
    *count = v;
    return HTS_OK;
}

hts_status hts_sync_status(hts_ctx *ctx, void *stream, int info[4])
{
    if (!ctx) return HTS_ERR_ARG;
    DeviceGuard g(ctx->device);
    if (!g.ok) return HTS_ERR_CUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (cudaStreamSynchronize(st) != cudaSuccess) return HTS_ERR_CUDA;
    if (cudaMemcpy(ctx->h_status, ctx->d_status, kStatusWords * sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        return HTS_ERR_CUDA;
    if (cudaMemset(ctx->d_status, 0, kStatusFallbacks * sizeof(int)) != cudaSuccess) return HTS_ERR_CUDA;
    if (info)
        for (int i = 0; i < 4; ++i) info[i] = ctx->h_status[1 + i];
    return static_cast<hts_status>(ctx->h_status[0]);
}

}  // extern "C"
