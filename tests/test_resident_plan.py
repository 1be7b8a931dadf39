"""Host-side check of the on-chip batched kernel's work partition and
shared-memory indices (csrc/bte_resident.cu), restated here in Python: for
every rank of a cluster and every thread of a 512-thread CTA, the interior
row chains, the boundary-row units and the edge rows they push into the
neighbours' halo rows, the row-0/1 sums and the initial load.

Checked for each shape: every shared-memory access lies inside its array
(rows 0 .. rows_per+1, columns 0 .. P-1), reads and writes alike, including
the clamped iterations that store nothing; every row of the CTA is written
exactly once per half-step (interior chains plus boundary units); rows
outside 0..N are only ever read from the zero halo rows that nothing
writes; a row pushed into a neighbour's halo row (distributed shared
memory) is the row that halo row stands for.  No GPU is needed: the kernel's index
arithmetic is evaluated for all threads on the CPU."""
import itertools

import pytest

NTHR = 512


def _cdiv(a, b):
    return -(-a // b)


def _check_shape(N1, M1, C, V):
    rows_per = _cdiv(N1, C)
    ncg = _cdiv(M1, V)
    LG = V
    P = LG + ncg * V + V
    N = N1 - 1

    def rank_rows(rank):
        r0 = min(N1, rank * rows_per)
        r1 = min(N1, r0 + rows_per)
        return r0, r1, r1 - r0

    for rank in range(C):
        r0, r1, R = rank_rows(rank)
        have_up = r0 >= 1 and R > 0
        have_dn = r1 <= N and R > 0
        # shared row s of this CTA holds global row r0 - 1 + s after the load
        loaded = {s for s in range(R + 2) if 0 <= r0 - 1 + s <= N}
        written = {}

        def read(s, lo_col, hi_col, own=True, nb=None):
            assert 0 <= s <= rows_per + 1, (N1, M1, C, rank, s)
            assert 0 <= lo_col and hi_col < P, (N1, M1, C, rank, lo_col, hi_col, P)
            if own:
                n = r0 - 1 + s
                if not 0 <= n <= N:
                    # outside the grid: must be a zero halo row nothing writes
                    assert s in (0, R + 1) and s not in loaded, (N1, C, rank, s)

        def write(s, g):
            assert 1 <= s <= R, (N1, M1, C, rank, s, R)
            written[(s, g)] = written.get((s, g), 0) + 1

        # interior rows 1..R-2: chains of stride 2 over each thread's row block
        cpp = min(ncg, NTHR)
        rsplit = NTHR // cpp
        npass = _cdiv(ncg, cpp)
        nint = R - 2 if R > 2 else 0
        nrow = _cdiv(nint, rsplit)
        for tid in range(NTHR):
            gl, rp = tid % cpp, tid // cpp
            t_on = rp < rsplit
            lo = 1 + rp * nrow
            for pss in range(npass):
                g = pss * cpp + gl
                g_on = t_on and g < ncg
                m0 = (g if g_on else 0) * V
                for ch in (0, 1):
                    ln = (nrow + 1 - ch) // 2
                    if ln == 0:
                        continue
                    i0 = lo + ch
                    il = min(i0, R - 2)
                    read(il, LG + m0 - 1, LG + m0 + V)           # other grid, row il-1
                    for ii in range(ln):
                        i = i0 + 2 * ii
                        on = g_on and i < R - 1
                        il = min(i, R - 2)
                        assert il >= 1
                        read(il + 2, LG + m0 - 1, LG + m0 + V)   # other grid, row il+1
                        read(il + 1, LG + m0, LG + m0 + V - 1)   # own cells (loaded first)
                        assert 0 <= il + 1 <= rows_per + 1       # sR[il + 1]
                        if on:
                            write(il + 1, g)
        # boundary rows 0 and R-1: every read in this CTA's shared memory
        # (the halo rows hold the neighbours' edge rows, pushed to them)
        nbnd = 2 if R >= 2 else R
        for tid in range(NTHR):
            for u in range(tid, nbnd * ncg, NTHR):
                b, g = divmod(u, ncg)
                il = 0 if b == 0 else R - 1
                m0 = g * V
                read(il, LG + m0 - 1, LG + m0 + V)
                read(il + 2, LG + m0 - 1, LG + m0 + V)
                read(il + 1, LG + m0, LG + m0 + V - 1)
                write(il + 1, g)
                if il == 0 and have_up:
                    # pushed into rank-1's halo row below its last own row
                    _, r1n, Rn = rank_rows(rank - 1)
                    assert Rn == rows_per and r1n == r0
                    assert rows_per + 1 > Rn                    # a halo row, not one of its own rows
                if il == R - 1 and have_dn:
                    # pushed into rank+1's halo row 0, which stands for row r1 - 1
                    r0n, _, Rn = rank_rows(rank + 1)
                    assert Rn >= 1 and r0n - 1 == r0 + R - 1      # shared row 0 is not one of its own rows
        # every own row written exactly once per half-step
        assert set(written) == {(s, g) for s in range(1, R + 1) for g in range(ncg)}, (N1, M1, C, rank)
        assert all(c == 1 for c in written.values()), (N1, M1, C, rank)
        # rank 0 adds rows 0 (a) and 1 (b): shared rows 1 and 2
        if rank == 0:
            for g in range(ncg):
                read(1, LG + g * V, LG + g * V + V - 1)
                if R >= 2:
                    read(2, LG + g * V, LG + g * V + V - 1)
                else:
                    assert 2 == R + 1                           # zero halo when there is no row 1


SHAPES = list(itertools.product([1, 2, 3, 4, 5, 7, 21, 64, 101, 201],
                                [3, 5, 33, 201, 1021, 2001, 2500],
                                [1, 2, 4, 8, 16]))


@pytest.mark.parametrize("V", [4, 2])
def test_partition_and_indices(V):
    n = 0
    for N1, M1, C in SHAPES:
        # the tier rule gives each CTA of a cluster of C > 1 at least two rows
        if C > 1 and _cdiv(N1, C) < 2:
            continue
        _check_shape(N1, M1, C, V)
        n += 1
    assert n > 200
