"""Host logic of the naive split form's pair-GEMM schedules, read from the library itself
(nspt_debug_pair_schedule, no GPU needed) and checked exhaustively for T = 0..90 and 255:

* the product (Eq. 5): every pair (l, j) with l + j <= T is computed exactly once, into
  output order k = l + j;
* the backward: every pair (k, m) with m <= k <= T exactly once, into output order j = k - m,
  for gA (left operand gC_k at slot k, right operand B_m at slot T - m) and gB (left A_m at
  slot T - m, right gC_k at slot k);
* no launch writes one (accumulator, order) twice (its GEMMs run concurrently);
* a plain write is the first write of its (accumulator, order), an accumulating write
  follows a write or lands on an accumulator zeroed beforehand (the product's second one,
  both of the backward's), and the product's first accumulator ends up written at every
  order;
* launches are balanced (at most 1.15 times the mean number of pair products for T >= 8).
"""
import ctypes

import pytest

T_VALUES = list(range(0, 91)) + [255]


@pytest.fixture(scope="module")
def L():
    import paper_2001_02835_b300 as n
    return n.lib()


def schedule(L, T, kind):
    n = L.nspt_debug_pair_schedule(T, kind, None, 0)
    assert n > 0
    buf = (ctypes.c_int * (7 * n))()
    assert L.nspt_debug_pair_schedule(T, kind, buf, 7 * n) == n
    return [tuple(buf[7 * i:7 * i + 7]) for i in range(n)]


def pairs_of(group, T, kind):
    """(first index, second index, output order) of each pair product of a batched GEMM."""
    launch, acc, l0, r0, o0, cnt, plain = group
    out = []
    for t in range(cnt):
        ls, rs, o = l0 + t, r0 + t, o0 + 2 * t
        assert 0 <= ls <= T and 0 <= rs <= T and 0 <= o <= T
        if kind == 0:
            out.append((ls, rs, o))                 # (l, j), k = l + j
        elif kind == 1:
            out.append((ls, T - rs, o))             # (k, m): gC_k at slot k, B_m at slot T - m
        else:
            out.append((rs, T - ls, o))             # (k, m): A_m at slot T - m, gC_k at slot k
    return out


@pytest.mark.parametrize("kind", [0, 1, 2])
def test_pair_schedules_cover_every_pair_once_without_conflicts(L, kind):
    for T in T_VALUES:
        sched = schedule(L, T, kind)
        launches = sorted({g[0] for g in sched})
        assert launches == list(range(len(launches))), (T, kind)
        seen = set()
        written = [set(), set(range(T + 1))]       # the product's second accumulator is zeroed
        if kind != 0:
            written = [set(range(T + 1)), set(range(T + 1))]   # the backward zeroes both
        sizes = []
        for lc in launches:
            keys, size = set(), 0
            for g in (g for g in sched if g[0] == lc):
                acc, plain = g[1], g[6]
                assert acc in (0, 1)
                for a, b, o in pairs_of(g, T, kind):
                    if kind == 0:
                        assert o == a + b and a + b <= T, (T, g)
                    else:
                        assert o == a - b and 0 <= b <= a <= T, (T, kind, g)
                    assert (a, b) not in seen, (T, kind, a, b)
                    seen.add((a, b))
                    assert (acc, o) not in keys, (T, kind, lc, acc, o)
                    keys.add((acc, o))
                    if plain:
                        assert o not in written[acc], (T, kind, g)
                    else:
                        assert o in written[acc], (T, kind, g)
                size += g[5]
            for acc, o in keys:
                written[acc].add(o)
            sizes.append(size)
        assert len(seen) == (T + 1) * (T + 2) // 2, (T, kind)
        assert written[0] == set(range(T + 1))
        if T >= 8:
            assert max(sizes) <= 1.15 * sum(sizes) / len(sizes), (T, kind, sizes)


def test_pair_schedule_arguments(L):
    assert L.nspt_debug_pair_schedule(-1, 0, None, 0) == -1
    assert L.nspt_debug_pair_schedule(256, 0, None, 0) == -1
    assert L.nspt_debug_pair_schedule(3, 3, None, 0) == -1
    # a buffer too short for every GEMM: as many as fit are written, the count is returned
    buf = (ctypes.c_int * 7)(*([99] * 7))
    n = L.nspt_debug_pair_schedule(7, 0, buf, 7)
    assert n > 1 and list(buf) != [99] * 7
