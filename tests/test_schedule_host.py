"""Host-side checks of the look-ahead schedule of stage 2 (csrc/schedule.cuh).

The update launch of group g runs beside the chase of group g+1, so three properties carry the
correctness of the overlap; they are checked here, without a GPU, on the task list the library's
own code produces (tests/schedule_probe.cu, compiled with nvcc for the host):

1. every tile with work appears exactly once (right tiles of A and B, left tiles of A and B,
   the rows above the group, the Q / Z tiles);
2. a left tile and a right tile of the same matrix that share an element are ordered: the left
   tile waits for the right one, which holds a lower ticket (so every wait ends);
3. every element of A and B that a step (k, j) of group g+1 touches, and that an update tile of
   group g writes, lies in a tile the step waits for.

The element sets are restated here from the method's index formulas (Alg. 3 / Alg. 4 with the
readings the library follows): the step's band rows i4 .. i3 and columns i1 .. i2, its pivot
column and B block; a right tile writes its own rows from the first column of its first block;
a left tile writes its own columns from row j1 + 1 to the last row of its lowest block.
"""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


@pytest.fixture(scope="module")
def probe(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path_factory.mktemp("probe") / "schedule_probe")
    subprocess.run([nvcc, "-std=c++17", "-O1", "-I", os.path.join(ROOT, "include"), "-o", exe,
                    os.path.join(HERE, "schedule_probe.cu")], check=True, capture_output=True)
    return exe


def run_probe(exe, n, r, j1, qg, TL, ab=1, nqz=2):
    out = subprocess.run([exe, str(n), str(r), str(j1), str(qg), str(ab), str(nqz), str(TL)], check=True,
                         capture_output=True, text=True).stdout.split("\n")
    plan, tasks, waits = None, [], {}
    for line in out:
        f = line.split()
        if not f:
            continue
        if f[0] == "plan":
            keys = ("ntiles", "ab", "T0", "Tend", "Cs0", "Cs1", "Ce", "D0", "D1", "U", "nrect", "total")
            plan = dict(zip(keys, map(int, f[1:])))
        elif f[0] == "task":
            tasks.append(tuple(map(int, f[1:])))
        elif f[0] == "wait":
            j, k, nr, nl = map(int, f[1:])
            waits[(j, k)] = (nr, nl)
    return plan, tasks, waits


def nblocks_gen(n, r, j):
    return 1 + (n - j - 2) // r if n - j - 2 >= 0 else 0


def step_geom(n, r, j1, qg, k, j):
    jb = j + max(0, (k - 1) * r + 1)
    i1 = j + k * r + 1
    i2 = min(j + (k + 1) * r, n)
    i3 = min(j + (k + 2) * r, n)
    i4 = j1 + 1 + max(0, (k + j - j1 - qg) * r)
    return jb, i1, i2, i3, i4


def left_cut(isB, n, r, jl, k):
    return min(jl + (k + 1) * r, n) if isB else jl + max(0, (k - 1) * r + 1)


def right_tile_cols(n, r, j1, T, TL):
    """First column a right tile of group j1 writes (None: the tile has no work)."""
    kmax = nblocks_gen(n, r, j1) - 1
    l0 = T * TL + 1
    if l0 > n:
        return None
    kstop = 0 if l0 <= j1 else (l0 - j1 - 1) // r + 2
    if kstop > kmax:
        return None
    return j1 + kstop * r + 1


def left_tile_rows(n, r, j1, qg, m, C, TL):
    """Last row a left tile of group j1 writes (None: no work); rows start at j1 + 1."""
    kmax = nblocks_gen(n, r, j1) - 1
    jl = j1 + qg - 1
    clast = min((C + 1) * TL, n)
    if C * TL + 1 > n:
        return None
    for k in range(kmax, -1, -1):
        if left_cut(m, n, r, jl, k) < clast:
            return min(n, j1 + k * r + r + qg - 1)
    return None


def step_elements(n, r, j1, qg, k, j):
    """(row, column) ranges of A and B a chase step of the group (j1, qg) reads or writes:
    list of (mat, r0, r1, c0, c1)."""
    jb, i1, i2, i3, i4 = step_geom(n, r, j1, qg, k, j)
    rlo = j1 + k * r + 1
    rhi = min(j + (k + 1) * r, n)
    els = []
    if rlo <= rhi:
        els.append((0, rlo, rhi, jb, jb))                  # pivot column segment (lazy updates)
        cb = i1 + r - 1
        if cb <= n:
            els.append((1, rlo, rhi, cb, cb))              # newest B column
    if k < nblocks_gen(n, r, j) and i1 <= i2:
        els.append((0, i4, i3, i1, i2))                    # band of A
        els.append((1, i4, i2, i1, i2))                    # band and block of B
    return els


CASES = [(200, 16, 16), (300, 16, 7), (257, 8, 8), (129, 4, 3), (400, 32, 32), (333, 32, 13), (96, 8, 1),
         (64, 3, 2), (1000, 16, 16)]


@pytest.mark.parametrize("TL", [32, 64, 128])
@pytest.mark.parametrize("n,r,q", CASES)
def test_schedule_covers_and_orders(probe, n, r, q, TL):
    groups = list(range(1, n - 1, q))
    for gi, j1 in enumerate(groups[:-1]):
        qg = min(q, n - 2 - j1 + 1)
        P, tasks, waits = run_probe(probe, n, r, j1, qg, TL)
        ticket = {}
        for t, kind, mat, tile, dep in tasks:
            if kind == 0:
                continue
            key = (kind, mat, tile)
            assert key not in ticket, ("task twice", key)
            ticket[key] = (t, dep)
        # 1. coverage
        nt = P["ntiles"]
        for m in (0, 1):
            for T in range(nt):
                has = right_tile_cols(n, r, j1, T, TL) is not None
                assert ((1, m, T) in ticket) == has, ("right tile", m, T, has)
                if has and T < P["T0"]:
                    assert (T + 1) * TL <= j1    # the rows above the group
            for C in range(nt):
                has = left_tile_rows(n, r, j1, qg, m, C, TL) is not None
                assert ((2, m, C) in ticket) == has, ("left tile", m, C, has)
        for m in (0, 1):
            for T in range(nt):
                assert (3, m, T) in ticket
        # 2. left / right conflicts are ordered and the left tile waits for the right one
        for (kind, m, C), (t, dep) in ticket.items():
            if kind != 2:
                continue
            rmax = left_tile_rows(n, r, j1, qg, m, C, TL)
            for T in range(nt):
                c0 = right_tile_cols(n, r, j1, T, TL)
                if c0 is None:
                    continue
                rows = (T * TL + 1, min((T + 1) * TL, n))
                cols = (C * TL + 1, min((C + 1) * TL, n))
                share = rows[0] <= rmax and rows[1] >= j1 + 1 and cols[1] >= c0
                if share:
                    assert P["T0"] <= T <= dep, ("left tile does not wait", m, C, T, dep)
                    assert ticket[(1, m, T)][0] < t, ("right tile after left tile", m, C, T)
        # 3. the next group's steps wait for every tile they share an element with
        j1n = j1 + qg
        qn = min(q, n - 2 - j1n + 1)
        for (j, k), (nr, nl) in waits.items():
            for (m, r0, r1, c0, c1) in step_elements(n, r, j1n, qn, k, j):
                if r0 > r1 or c0 > c1:
                    continue
                for T in range(nt):
                    cf = right_tile_cols(n, r, j1, T, TL)
                    if cf is None:
                        continue
                    if T * TL + 1 <= r1 and min((T + 1) * TL, n) >= r0 and c1 >= cf:
                        assert P["T0"] <= T <= nr, ("step does not wait for right tile", j, k, m, T, nr)
                for C in range(nt):
                    rmax = left_tile_rows(n, r, j1, qg, m, C, TL)
                    if rmax is None:
                        continue
                    if C * TL + 1 <= c1 and min((C + 1) * TL, n) >= c0 and r0 <= rmax and r1 >= j1 + 1:
                        assert P["Cs%d" % m] <= C <= nl, ("step does not wait for left tile", j, k, m, C, nl)


def test_closing_launch_has_only_qz_tiles(probe):
    P, tasks, _ = run_probe(probe, 300, 16, 1, 16, 32, ab=0, nqz=1)
    assert P["total"] == P["ntiles"] and all(k == 3 for _, k, _, _, _ in tasks)
