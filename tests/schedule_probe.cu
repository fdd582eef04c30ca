// Host-side probe of the look-ahead task schedule (paper_2301_07964_gb300/csrc/schedule.cuh),
// built and run by tests/test_schedule_host.py: prints the plan of one update launch, its tasks
// in ticket order with the last right tile each left task waits for, and the wait range of
// every chase step of the next group.  No GPU is needed.
#include <cstdio>
#include <cstdlib>

#include "../paper_2301_07964_gb300/csrc/schedule.cuh"

using namespace hts;

int main(int argc, char **argv)
{
    if (argc < 8) return 2;
    const int n = atoi(argv[1]), r = atoi(argv[2]), j1 = atoi(argv[3]), qg = atoi(argv[4]);
    const int ab = atoi(argv[5]), nqz = atoi(argv[6]), TL = atoi(argv[7]);
    const TaskPlan P = task_plan(n, r, j1, qg, ab != 0, nqz, TL);
    printf("plan %d %d %d %d %d %d %d %d %d %d %d %d\n", P.ntiles, P.ab, P.T0, P.Tend, P.Cs[0], P.Cs[1], P.Ce,
           P.D[0], P.D[1], P.U, P.nrect, P.total);
    for (int t = 0; t < P.total; ++t) {
        const Task T = task_of(P, t);
        const int dep = T.kind == kTaskLeft ? left_dep_tile(P, n, r, T.mat, T.tile) : -1;
        printf("task %d %d %d %d %d\n", t, T.kind, T.mat, T.tile, dep);
    }
    // the next group's chase steps (k, j): rows <= i3, columns <= i2
    const int j1n = j1 + qg;
    for (int j = j1n; j <= j1n + qg - 1 && j <= n - 2; ++j)
        for (int k = 0; k < nblocks_lazy(n, r, j); ++k) {
            const StepGeom g = step_geom(n, r, j1n, qg, k, j);
            int nr, nl;
            upd_wait_range(P, n, g.i2, g.i3, &nr, &nl);
            printf("wait %d %d %d %d\n", j, k, nr, nl);
        }
    return 0;
}
