"""The schedule of the fused FP64 factor step (one cooperative launch per block
step, no grid barriers), replayed on the CPU.

The kernel gives tile (r, c) of the extended lower triangle to CTA u(r, c) mod G
(u = column-major index), and each CTA walks phases 1(k) (update column k+1 at
step k, then finalize it), 2(k) (update column k+2) and 3(k) (update columns
>= k+3) in the order 1(k), 2(k), 1(k+1), 3(k), ... Its only waits are on
finalized tiles: tile (r, c) is final once the row counter pdone[r] > c (the
bulk phase 3(k) instead waits once for the whole of column k). This
replay checks, for block counts, arrowheads, the last block, Schur updates on
or off and grid sizes from 2 to 608 (2 to 4 CTAs per SM on 152 SMs), that (1) the operations are exactly the tile
Cholesky's (every update U(r, c, k), k < c, once; every finalization once),
(2) each tile sees its updates in k order and is finalized after all of them,
and (3) the CTAs, each in its own order, always complete: flags only grow, so
completing under one interleaving means no interleaving can deadlock.
"""
import itertools

import pytest


def _schedule(nt, na, nxt, schur, G):
    E = nt * (1 + nxt) + na
    Ecol = E if schur else nt

    def off(c):
        return c * E - c * (c - 1) // 2

    items = [[] for _ in range(G)]

    def column(c, k, fin):
        for r in range(c, E):
            cta = (off(c) + r - c) % G
            if k >= 0:
                items[cta].append(("U", r, c, k))
            if fin:
                items[cta].append(("F", r, c))

    for ph in range(-3, 3 * (nt - 1) + 5):
        if ph % 3 == 0:
            k = ph // 3
            if k < nt and k + 1 < Ecol:
                column(k + 1, k, k + 1 < nt)
        elif ph % 3 == 2:
            k = (ph - 2) // 3
            if ph >= 2 and k < nt and k + 2 < Ecol:
                column(k + 2, k, False)
        else:
            k = (ph - 4) // 3
            if ph >= 4 and k < nt and k + 3 < Ecol:
                for c in range(k + 3, Ecol):
                    for r in range(c, E):
                        items[(off(c) + r - c) % G].append(("B", r, c, k))
    return E, Ecol, items


def _replay(E, items):
    pdone = [0] * E
    colcnt = [0] * E
    last = {}
    ptr = [0] * len(items)
    moved = True
    while moved:
        moved = False
        for g, lst in enumerate(items):
            while ptr[g] < len(lst):
                it = lst[ptr[g]]
                if it[0] in ("U", "B"):
                    _, r, c, k = it
                    if it[0] == "U" and not (pdone[r] > k and pdone[c] > k):
                        break
                    if it[0] == "B" and colcnt[k] < E - k:  # the whole of column k is final
                        break
                    assert last.get((r, c), -1) == k - 1
                    last[(r, c)] = k
                else:
                    _, r, c = it
                    assert last.get((r, c), -1) == c - 1
                    if r != c and not pdone[c] > c:
                        break
                    assert pdone[r] == c
                    pdone[r] = c + 1
                    colcnt[c] += 1
                ptr[g] += 1
                moved = True
    return all(ptr[g] == len(lst) for g, lst in enumerate(items))


@pytest.mark.parametrize("nt,na,nxt,schur", list(itertools.product([1, 2, 3, 5, 8, 33, 64], [0, 1, 2],
                                                                    [0, 1], [0, 1])))
def test_factor_step_schedule_is_complete_and_deadlock_free(nt, na, nxt, schur):
    for G in (2, 3, 7, 304, 456, 608):
        E, Ecol, items = _schedule(nt, na, nxt, schur, G)
        ops = [("U",) + it[1:] if it[0] == "B" else it for lst in items for it in lst]
        want = {("U", r, c, k) for c in range(Ecol) for r in range(c, E) for k in range(min(c, nt))}
        want |= {("F", r, c) for c in range(nt) for r in range(c, E)}
        assert len(ops) == len(set(ops)) and set(ops) == want
        assert _replay(E, items)


def test_bulk_phase_splits_evenly():
    # phase 3(k) is one contiguous range of column-major indices: every CTA gets
    # floor or ceil of its share
    nt, na, nxt, G = 64, 1, 1, 304
    E, Ecol, items = _schedule(nt, na, nxt, 1, G)
    for k in (0, 20, 50):
        per = [sum(1 for it in lst if it[0] == "B" and it[3] == k) for lst in items]
        assert max(per) - min(per) <= 1
