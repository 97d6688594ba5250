"""Host logic of the persistent segment launch (no GPU): the wait lists.

Between two sweeps a block must wait for every block that writes a row one of
its items reads (its input for the next sweep) and for every block that reads a
row it writes (their reads must end before it overwrites them).  An item of
rows [y0, y1) reads rows y0 - 2 .. y1 + 1 of every x segment (wrapped where y is
periodic), so both relations are "some item of one block reads a row that an
item of the other writes".  The library's lists are checked against that
relation computed by brute force over all pairs of items.
"""
import numpy as np
import pytest

from paper_1901_02716_gb300 import _build
from paper_1901_02716_gb300 import maclab as M


@pytest.fixture(scope="module", autouse=True)
def _built():
    _build.build()


def brute_force(items, ny, py, blocks):
    nw = 4 * blocks
    owner = [(i % nw) // 4 for i in range(len(items))]

    def reads(i):
        y0, y1 = items[i][2], items[i][3]
        out = set()
        for y in range(y0 - 2, y1 + 2):
            if 0 <= y < ny:
                out.add(y)
            elif py:
                out.add(y % ny)
        return out

    writes = [set(range(it[2], it[3])) for it in items]
    want = [set() for _ in range(blocks)]
    for i in range(len(items)):
        r = reads(i)
        for j in range(len(items)):
            if owner[i] != owner[j] and r & writes[j]:
                want[owner[i]].add(owner[j])
                want[owner[j]].add(owner[i])
    return want


@pytest.mark.parametrize("nx,ny,py,rows,blocks", [
    (8, 12, 1, 4, 2), (64, 64, 1, 8, 1), (136, 45, 0, 2, 7), (256, 256, 0, 2, 96),
    (256, 40, 1, 3, 5), (512, 17, 1, 2, 456), (1024, 64, 0, 4, 50), (32, 3, 1, 2, 3)])
def test_wait_lists_match_brute_force(nx, ny, py, rows, blocks):
    items, waits = M.maclab_debug_segment_waits(nx, ny, py, rows, blocks)
    assert len(items) > 0
    # the items tile the rows: every row once per x segment
    nseg = int(items[:, 1].max()) + 1
    cover = np.zeros((nseg, ny), dtype=int)
    for it in items:
        assert it[0] == 0 and 0 <= it[2] < it[3] <= ny and it[3] - it[2] <= rows
        cover[it[1], it[2]:it[3]] += 1
    assert (cover == 1).all()
    # offsets, then the lists: no self, no repeats, in range
    assert len(waits) >= blocks + 1 and waits[blocks] == len(waits)
    got = []
    for b in range(blocks):
        lst = list(waits[waits[b]:waits[b + 1]])
        assert len(lst) == len(set(lst)) and b not in lst
        assert all(0 <= c < blocks for c in lst)
        got.append(set(lst))
    assert got == brute_force(items.tolist(), ny, py, blocks)


def test_wait_lists_reject_bad_shapes():
    for args in ((6, 8, 0, 2, 1), (8, 0, 0, 2, 1), (8, 8, 0, 0, 1), (8, 8, 0, 2, 0)):
        with pytest.raises(M.MacLABError):
            M.maclab_debug_segment_waits(*args)


def brute_force_batch(items, ny, py, blocks):
    """The same relation over several domains: rows of different domains
    never meet."""
    nw = 4 * blocks
    owner = [(i % nw) // 4 for i in range(len(items))]

    def reads(i):
        d, y0, y1 = items[i][0], items[i][2], items[i][3]
        out = set()
        for y in range(y0 - 2, y1 + 2):
            if 0 <= y < ny[d]:
                out.add((d, y))
            elif py[d]:
                out.add((d, y % ny[d]))
        return out

    writes = [{(it[0], y) for y in range(it[2], it[3])} for it in items]
    want = [set() for _ in range(blocks)]
    for i in range(len(items)):
        r = reads(i)
        for j in range(len(items)):
            if owner[i] != owner[j] and r & writes[j]:
                want[owner[i]].add(owner[j])
                want[owner[j]].add(owner[i])
    return want


@pytest.mark.parametrize("seed,count,rows,blocks", [(1, 3, 2, 4), (2, 5, 4, 9), (3, 8, 3, 17), (4, 2, 16, 1),
                                                    (5, 6, 2, 40)])
def test_batch_wait_lists_match_brute_force(seed, count, rows, blocks):
    rng = np.random.default_rng(seed)
    nx = 4 * rng.integers(2, 40, size=count)
    ny = rng.integers(1, 30, size=count)
    py = rng.integers(0, 2, size=count)
    items, waits = M.maclab_debug_batch_waits(nx, ny, py, rows, blocks)
    # the domains' items tile each domain's rows once per x segment, in domain order
    assert (np.diff(items[:, 0]) >= 0).all()
    for d in range(count):
        it = items[items[:, 0] == d]
        nseg = int(it[:, 1].max()) + 1
        cover = np.zeros((nseg, ny[d]), dtype=int)
        for row in it:
            assert 0 <= row[2] < row[3] <= ny[d] and row[3] - row[2] <= rows
            cover[row[1], row[2]:row[3]] += 1
        assert (cover == 1).all()
    assert len(waits) >= blocks + 1 and waits[blocks] == len(waits)
    got = []
    for b in range(blocks):
        lst = list(waits[waits[b]:waits[b + 1]])
        assert len(lst) == len(set(lst)) and b not in lst
        assert all(0 <= c < blocks for c in lst)
        got.append(set(lst))
    assert got == brute_force_batch(items.tolist(), ny.tolist(), py.tolist(), blocks)


def test_batch_wait_lists_of_one_domain_equal_the_segment_lists():
    for nx, ny, py, rows, blocks in ((64, 64, 1, 8, 3), (136, 45, 0, 2, 7)):
        a = M.maclab_debug_segment_waits(nx, ny, py, rows, blocks)
        b = M.maclab_debug_batch_waits([nx], [ny], [py], rows, blocks)
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_batch_wait_lists_reject_bad_shapes():
    for args in (([6], [8], [0], 2, 1), ([8], [0], [0], 2, 1), ([8], [8], [0], 0, 1), ([8], [8], [0], 2, 0),
                 ([8, 10], [8, 8], [0, 1], 2, 1)):
        with pytest.raises(M.MacLABError):
            M.maclab_debug_batch_waits(*args)
