"""Host-side check of the on-chip mode over several clusters
(csrc/bte_wide.cu, bte_tuning.resident = 3), no GPU needed.

The kernel's partition and data movement are mirrored in Python for every
CTA of several launch shapes: which rows and columns a CTA owns, which
values of the other grid a half-step reads (rows n-1 and n+1 at columns
m-1 and m+1), and where each of them comes from -- the CTA's own cells,
the halo rows that the CTAs above and below push (their first or last own
row), or the halo columns filled from the exchange area that CTAs of the
neighbouring clusters write (their first or last own column) as tagged
exchange words.  The checks: every cell is owned exactly once; every value
read comes from the CTA that makes it, through a word that writer fills and
this reader polls (the lane mapping of the kernel's warp 0 covers each word
read); every reader of a CTA's words is a CTA whose words it polls (so a
word is not rewritten before it is read); and every shared-memory and
exchange index is in bounds.  The host's automatic choice of the launch
shape is mirrored too and pinned through the workspace size the library
reports.
"""
import pytest

from paper_1401_6047_gb300 import bte
from paper_1401_6047_gb300 import workloads as W

SMEM_MAX = 232448


def cdiv(a, b):
    return -(-a // b)


def wide_smem(rp, wc, elem):
    wp = wc + 2
    arr = (rp + 2) * wp
    b = (4 * arr + 2 * wp + rp + 2) * elem
    return (b + 15) // 16 * 16


def plan(n1, m1, elem, cols=0):
    """(C, G, Wc, rows_per) as the host picks them."""
    for c in (16, 8, 4, 2, 1):
        if c > 1 and cdiv(n1, c) < 2:
            continue
        rp = cdiv(n1, c)
        wc = cols
        if not wc:
            auto = 32 if elem == 8 else 128
            g = max(min(cdiv(m1, auto), max(1, 128 // c)), 1)
            wc = cdiv(m1, g)
            while (wide_smem(rp, wc, elem) > SMEM_MAX or rp * wc > 480) and cdiv(m1, wc) < 32:
                g0 = cdiv(m1, wc)
                wc = (m1 + g0) // (g0 + 1)
        g = cdiv(m1, wc)
        if g > 32 or wide_smem(rp, wc, elem) > SMEM_MAX or rp * wc > 480:
            continue
        return c, g, wc, rp
    return None


class Cta:
    def __init__(self, g, rank, N, M, C, G, wc, rp):
        n1 = N + 1
        self.g, self.rank = g, rank
        self.r0 = min(n1, rank * rp)
        self.r1 = min(n1, self.r0 + rp)
        self.R = self.r1 - self.r0
        self.c0 = g * wc
        self.have_up = self.R > 0 and self.r0 >= 1
        self.have_dn = self.R > 0 and self.r1 <= N


def xword(buf, grid, side, ab, part, g, n, G, n1, W):
    return ((((((buf * 2 + grid) * 2 + side) * 2 + ab) * W + part) * G + g) * n1 + n)


SHAPES = [
    # (N, M, wide_cols): the grid is (N + 1) x (M + 1); 0 = automatic
    (30, 200, 0),
    (30, 200, 29),
    (9, 36, 8),
    (40, 300, 64),
    (1, 12, 3),
    (4, 20, 1),
    (64, 699, 90),
    (100, 999, 0),
    (64, 699, 0),
]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("W", [1, 2])  # 32-bit parts per value: FP32, FP64
@pytest.mark.parametrize("hs", [0, 1, 2, 3])  # the half-step that writes
def test_partition_exchange_and_waits(shape, W, hs):
    N, M, cols = shape
    n1, m1 = N + 1, M + 1
    C, G, wc, rp = plan(n1, m1, 4, cols)
    assert (G - 1) * wc <= M < G * wc, "every block holds a real column"
    ctas = {(g, r): Cta(g, r, N, M, C, G, wc, rp) for g in range(G) for r in range(C)}
    owner = {}
    for (g, r), t in ctas.items():
        for il in range(t.R):
            for j in range(wc):
                m = t.c0 + j
                if m <= M:
                    assert (t.r0 + il, m) not in owner
                    owner[(t.r0 + il, m)] = (g, r)
    assert len(owner) == n1 * m1

    wp = wc + 2
    arr = (rp + 2) * wp
    nslots = 16 * W * G * n1
    buf = (hs >> 1) & 1  # the writer's buffer, the one its readers poll at hs + 1
    # writes of one half-step: DSMEM pushes (target CTA, shared index) and
    # exchange slots, by the cell rule of the kernel
    pushes, slots = {}, {}
    for (g, r), t in ctas.items():
        for il in range(t.R):
            for j in range(wc):
                n, lc = t.r0 + il, j + 1
                for o in (0, 2):
                    for ab in (0, 1):
                        own = (o + ab) * arr + (il + 1) * wp + lc
                        assert 0 <= own < 4 * arr
                        if il == 0 and t.have_up:
                            idx = (rp + 1) * wp + (o + ab) * arr + lc
                            assert 0 <= idx < 4 * arr
                            pushes[((g, r - 1), idx)] = (n, t.c0 + j)
                        if il == t.R - 1 and t.have_dn:
                            idx = (o + ab) * arr + lc
                            assert 0 <= idx < 4 * arr
                            pushes[((g, r + 1), idx)] = (n, t.c0 + j)
                        for part in range(W):
                            if j == 0 and g > 0:
                                k = xword(buf, o >> 1, 0, ab, part, g, n, G, n1, W)
                                assert 0 <= k < nslots and (k not in slots or slots[k][0] == (g, r))
                                slots[k] = ((g, r), (n, t.c0))
                            if j == wc - 1 and g + 1 < G:
                                k = xword(buf, o >> 1, 1, ab, part, g, n, G, n1, W)
                                assert 0 <= k < nslots and (k not in slots or slots[k][0] == (g, r))
                                slots[k] = ((g, r), (n, t.c0 + j))
    readers, polls = {}, {}
    for (g, r), t in ctas.items():
        if t.R == 0:
            continue
        # every value of the other grid a half-step reads
        for il in range(t.R):
            for j in range(wc):
                for dn_ in (-1, 1):
                    for dm in (-1, 1):
                        n, m = t.r0 + il + dn_, t.c0 + j + dm
                        li, lc = il + 1 + dn_, j + 1 + dm
                        assert 0 <= li <= t.R + 1 and 0 <= lc <= wc + 1
                        if n < 0 or n > N or m < 0 or m > M:
                            continue  # zero: a halo cell nothing writes
                        src = owner[(n, m)]
                        if 1 <= li <= t.R and 1 <= lc <= wc:
                            assert src == (g, r)
                        elif 1 <= lc <= wc:
                            # halo row, pushed by the CTA above / below
                            for o in (0, 2):
                                assert pushes[((g, r), o * arr + li * wp + lc)] == (n, m)
                            assert src == (g, r - 1 if li == 0 else r + 1)
                        else:
                            # halo column from the exchange words, polled by
                            # the kernel's lane mapping of warp 0
                            side = 0 if lc == wc + 1 else 1
                            gg = g + 1 if lc == wc + 1 else g - 1
                            polled = set()
                            for q in range(4 * W * (t.R + 2)):
                                qs, qab, qpart, qli = q & 1, (q >> 1) & 1, (q >> 2) % W, q // (4 * W)
                                qn, qg = t.r0 - 1 + qli, (g + 1 if qs else g - 1)
                                if 0 <= qn <= N and 0 <= qg < G:
                                    polled.add((qs ^ 1, qab, qpart, qg, qn, qli, (wc + 1) if qs else 0))
                            for grid in (0, 1):
                                for ab in (0, 1):
                                    for part in range(W):
                                        assert (side, ab, part, gg, n, li, lc) in polled
                                        k = xword(buf, grid, side, ab, part, gg, n, G, n1, W)
                                        assert slots[k] == (src, (n, m))
                            readers.setdefault(src, set()).add((g, r))
                            polls.setdefault((g, r), set()).add(src)
    for w, rs in readers.items():
        for rd in rs:
            assert rd in polls.get(w, set()), "a writer polls the words of each reader of its words"


@pytest.mark.parametrize("p,prec", [
    (W.c1_fp64(), W.FP64), (W.c1_fp64(), W.FP32_MIXED), (W.c2(W.FP32_MIXED), W.FP32_MIXED),
    (W.paper_table1(W.FP32_MIXED), W.FP32_MIXED)])
def test_host_plan_through_workspace_size(p, prec):
    """The workspace of mode 3 is that of mode 0 plus the tagged edge-column
    words (two buffers) and the per-cluster sums of 8192 steps, for
    the (C, G) the mirrored plan picks; grids that need more than 480 cells
    per CTA in 32 clusters (401 x 4001, 120 x 4000) are refused."""
    p = p.replace(precision=prec)
    elem = 8 if prec == W.FP64 else 4
    pl = plan(p.n_max + 1, p.m_points, elem)
    if pl is None:
        with pytest.raises(bte.BteError) as e:
            bte.workspace_size(p, resident=3)
        assert e.value.code == bte.EINVAL
        assert p.cells > 32 * 16 * 480
        return
    C, G, wc, rp = pl
    al = lambda x: cdiv(x, 256) * 256
    extra = al(16 * (elem // 4) * G * (p.n_max + 1) * 8) + al(8192 * G * 16)
    assert bte.workspace_size(p, resident=3) == bte.workspace_size(p) + extra
    if p.n_max == 30 and p.m_points == 201:
        assert (C, G, wc) == ((16, 7, 29) if elem == 8 else (16, 2, 101))


def test_rejects_bad_wide_options():
    p = W.c1_fp64()
    for kw in (dict(resident=4), dict(resident=3, wide_cols=-1), dict(resident=3, wide_cols=4097),
               dict(resident=3, wide_cols=6),     # 6 columns: 34 clusters, above 32
               dict(resident=3, wide_cols=300)):  # 2 x 300 cells or more per CTA: above 480
        with pytest.raises(bte.BteError) as e:
            bte.workspace_size(p, **kw)
        assert e.value.code == bte.EINVAL
