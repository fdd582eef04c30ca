// Look-ahead schedule of stage 2 (Section "Parallel stage two": the generation of group g+1's
// reflectors overlaps the application of group g's).
//
// The delayed updates of group g (Alg. 4) run as one persistent launch whose workers take
// tasks in ticket order, while the chase of group g+1 (Alg. 3) runs beside it.  A task is one
// tile of TL lines (32 for the mma.sync kernel, 64 for the tcgen05 kernel):
//   right tile T of A or B   rows TL T+1 .. TL T+TL, every block k the rows still need (the
//                            windows from the last block to the first, then the staircase);
//   left tile C of A or B    columns TL C+1 .. TL C+TL, blocks from the lowest one whose cut lies
//                            left of the tile up to block 0;
//   Q / Z tile of the previous group (g-1), all blocks.
// A right tile and a left tile of the same matrix share elements, and the right update of each
// row is a chain over its blocks from the last to the first (consecutive windows overlap), as is
// the left update of each column.  The two directions commute, so the rule is only that they
// do not run on the same element at once: a left tile waits until every right tile of its
// matrix whose rows it reaches is done.  Rows 1 .. j1 (the right tiles above the group) meet
// no left tile and no later chase step; they run after the others.
//
// Each finished tile of A or B publishes epoch g+1 in its flag.  Step (k, j) of group g+1 reads
// and writes A and B only in rows <= i3(k, j) and columns <= i2(k, j); it waits for the right
// tiles of those rows and the left tiles of those columns.  Dependencies always point to lower
// tickets, which workers that are running already hold, so every wait ends.
#pragma once

#include "hts_internal.cuh"

namespace hts {

enum { kTaskNone = 0, kTaskRight = 1, kTaskLeft = 2, kTaskQZ = 3 };

struct Task {
    int kind, mat, tile;
};

// Left cut of block k (Alg. 4 with the reading of its start columns): the left update of
// block k covers the columns right of it.
__host__ __device__ __forceinline__ int left_cut_of(int isB, int n, int r, int jl, int k)
{
    return isB ? imin(jl + (k + 1) * r, n) : jl + imax(0, (k - 1) * r + 1);
}

__host__ __device__ inline TaskPlan task_plan(int n, int r, int j1, int qg, bool ab, int nqz, int TL)
{
    TaskPlan P;
    P.TL = TL;
    P.ntiles = (n + TL - 1) / TL;
    P.ab = ab ? 1 : 0;
    P.T0 = 0; P.Tend = -1; P.Cs[0] = P.Cs[1] = 0; P.Ce = -1; P.D[0] = P.D[1] = 0;
    P.U = 0; P.nrect = 0; P.nqz = nqz;
    if (ab) {
        const int kmax = nblocks_gen(n, r, j1) - 1;
        const int jl = j1 + qg - 1;
        P.T0 = j1 / TL;
        // a right tile needs blocks while its first row l0 <= j1 + max(0, kmax-1) r
        const int lmax = j1 + imax(0, kmax - 1) * r;
        P.Tend = imin(P.ntiles - 1, (lmax - 1) / TL);
        P.Ce = P.ntiles - 1;
        int U = P.Tend - P.T0 + 1;
        for (int m = 0; m < 2; ++m) {
            const int cut0 = left_cut_of(m, n, r, jl, 0);
            P.Cs[m] = cut0 >= n ? P.ntiles : cut0 / TL;
            // a left tile C reaches rows <= TL(C+1) + 2r - 1 (A) or <= TL(C+1) (B)
            P.D[m] = P.Cs[m] - P.T0 + (m == 0 ? 1 + (2 * r - 1) / TL : 0);
            if (P.Cs[m] <= P.Ce) U = imax(U, P.Ce - P.Cs[m] + P.D[m] + 1);
        }
        P.U = imax(U, 0);
        P.nrect = 2 * P.T0;
    }
    P.total = 4 * P.U + P.nrect + nqz * P.ntiles;
    return P;
}

__host__ __device__ __forceinline__ Task task_of(const TaskPlan &P, int t)
{
    Task T{kTaskNone, 0, 0};
    if (t < 4 * P.U) {
        const int u = t >> 2, slot = t & 3;
        if (slot < 2) {
            if (P.T0 + u <= P.Tend) T = Task{kTaskRight, slot, P.T0 + u};
        } else {
            const int m = slot - 2, C = P.Cs[m] + u - P.D[m];
            if (C >= P.Cs[m] && C <= P.Ce) T = Task{kTaskLeft, m, C};
        }
        return T;
    }
    t -= 4 * P.U;
    if (t < P.nrect) return Task{kTaskRight, t & 1, t >> 1};
    t -= P.nrect;
    if (P.nqz > 0) return Task{kTaskQZ, t % P.nqz, t / P.nqz};
    return T;
}

// Flag words of the A / B tiles: [(kind * 2 + mat) * ntiles + tile], kind 0 right, 1 left.
__host__ __device__ __forceinline__ size_t tile_flag(int ntiles, int kind, int mat, int tile)
{
    return (size_t)(kind * 2 + mat) * ntiles + tile;
}

// Last right tile of matrix `mat` a left tile C waits for.
__host__ __device__ __forceinline__ int left_dep_tile(const TaskPlan &P, int n, int r, int mat, int C)
{
    const int clast = imin((C + 1) * P.TL, n);
    const int rmax = imin(n, clast + (mat == 0 ? 2 * r - 1 : 0));
    return imin(P.Tend, (rmax - 1) / P.TL);
}

// Last tiles a chase step that touches rows <= i3 and columns <= i2 waits for: right tiles
// T0 .. *nr and left tiles Cs[m] .. *nl.
__host__ __device__ __forceinline__ void upd_wait_range(const TaskPlan &P, int n, int i2, int i3, int *nr, int *nl)
{
    *nr = imin(P.Tend, (imin(i3, n) - 1) / P.TL);
    *nl = imin(P.Ce, (imin(i2, n) - 1) / P.TL);
}

// Progress of one chase block through the previous group's update tiles (used by one thread).
struct UpdWait {
    const unsigned long long *flags;   // null: nothing to wait for (first group)
    TaskPlan P;
    unsigned long long epoch;          // the previous group's epoch (its index + 1)
    int n;
    int next[4];                       // next tile to check: right A, right B, left A, left B

    __device__ __forceinline__ void init(const unsigned long long *f, const TaskPlan &plan, unsigned long long ep, int nn)
    {
        flags = f;
        P = plan;
        epoch = ep;
        n = nn;
        next[0] = next[1] = P.T0;
        next[2] = P.Cs[0];
        next[3] = P.Cs[1];
    }

    // Wait until every tile that rows <= i3 and columns <= i2 lie in is done.
    __device__ __forceinline__ bool wait_for(int i2, int i3, int *status, int group, int k, int j)
    {
        if (!flags) return true;
        int nr, nl;
        upd_wait_range(P, n, i2, i3, &nr, &nl);
        for (int q = 0; q < 4; ++q) {
            const int last = q < 2 ? nr : nl;
            const int kind = q < 2 ? 0 : 1, mat = q & 1;
            for (; next[q] <= last; ++next[q])
                if (!wait_at_least(flags + tile_flag(P.ntiles, kind, mat, next[q]), epoch, status, group, k, j))
                    return false;
        }
        return true;
    }
};

// Worker loop of a persistent update launch: NT threads (tid 0 .. NT-1, barrier wb) take tasks
// in ticket order and run them with run(task).  A left tile first waits for the right tiles of
// its matrix that it overlaps; every finished tile of A or B publishes the launch's epoch.
// The loop ends when the tickets are used up, or when an error has been recorded (then the
// chase's bounded waits on the unpublished tiles give up as well).
template <int NT, class Run>
__device__ __forceinline__ void update_worker(const UpdSched &s, int tid, int wb, volatile int *slot, Run run)
{
    for (;;) {
        if (tid == 0) {
            int t = (int)atomicAdd(s.ticket, 1u);
            if (*(volatile int *)s.status != 0) {
                t = s.P.total;
            } else if (t < s.P.total) {
                const Task T = task_of(s.P, t);
                if (T.kind == kTaskLeft) {
                    const int last = left_dep_tile(s.P, s.n, s.r, T.mat, T.tile);
                    for (int q = s.P.T0; q <= last; ++q)
                        if (!wait_at_least(s.tflags + tile_flag(s.P.ntiles, 0, T.mat, q), s.epoch, s.status, s.group,
                                           -1, T.tile)) {
                            t = s.P.total;
                            break;
                        }
                }
            }
            *slot = t;
        }
        group_sync(wb, NT);
        const int t = *slot;
        if (t >= s.P.total) return;
        const Task T = task_of(s.P, t);
        run(T);
        __threadfence();
        group_sync(wb, NT);
        if (tid == 0 && (T.kind == kTaskRight || T.kind == kTaskLeft))
            st_release_u64(s.tflags + tile_flag(s.P.ntiles, T.kind == kTaskLeft ? 1 : 0, T.mat, T.tile), s.epoch);
    }
}

}  // namespace hts
