"""Size bound and coverage of the substitution copy schedule (host logic, no GPU).

The library builds, once per simulation, the per-warp list of chunks that the
pipelined substitutions copy (forward, then backward). Per block row k the
leader takes the coupling block to the previous (forward) or next (backward)
row and the diagonal inverse (forward: in one copy with the block when both
fit half a FIFO, the inverse then read from the panel's diagonal slot); the
other warps split the columns of panel k+1
before its block k into three contiguous shares, each copied in pieces of at
most pc columns, pc = max(1, (FIFO / 2 - 4) // n2) with the per-warp FIFO
((panel_words rounded up to 4 + 4 * 1032) // 4 rounded down to 4, minus 64
partial-sum elements). The buffer holding the lists is sized by a closed-form
bound: kSolveWarps + 1 list starts plus n_sub (4 Sx + 16) descriptors. This
test enumerates the lists that way for many layouts and basis sizes (panel
words taken at their smallest, which gives the most pieces), checks the
bound, that every piece fits half a FIFO, and that every block of the
envelope is copied exactly once per direction."""
import numpy as np
import pytest

NW = 4       # warps per CTA of the reduced solve
RING = 4     # slots of the factorisation ring
SLOT = 32 * 32 + 8
PART = 64    # partial-sum elements at the start of each warp's region


def jlo(k, Sx):
    return max(0, k - Sx)


def fifo_cap(panel_words):
    area = ((panel_words + 3) & ~3) + RING * SLOT
    return ((area // NW) & ~3) - PART


def piece_cols(panel_words, n2):
    return max(1, (fifo_cap(panel_words) // 2 - 4) // n2)


def fwd_pair(panel_words, nprev, nk):
    """The leader's forward coupling block and the panel's diagonal slot
    (holding the inverse) travel in one copy when they fit half a FIFO."""
    return (nprev + nk) * nk + 3 <= fifo_cap(panel_words) // 2


def warp_lists(NE, Sx):
    nsub = len(NE)
    xoff = np.concatenate([[0], np.cumsum(NE)])
    pw = max(int(NE[k]) * int(xoff[k + 1] - xoff[jlo(k, Sx)]) for k in range(nsub))
    lists = [[] for _ in range(NW)]
    for direction in (1, -1):
        rows = range(nsub) if direction > 0 else range(nsub - 1, -1, -1)
        for k in rows:
            npv = int(NE[k - 1]) if k >= 1 else 0
            if direction > 0 and fwd_pair(pw, npv, int(NE[k])):
                lists[0].append(("pair", direction, k, [k - 1] if k >= 1 else [], (npv + NE[k]) * NE[k]))
                lists[0].append(("inverse-in-slot", direction, k, None, 0))
            else:
                if direction > 0 and k >= 1:
                    lists[0].append(("panel", direction, k, [k - 1], NE[k - 1] * NE[k]))
                if direction < 0 and k <= nsub - 2:
                    lists[0].append(("panel", direction, k + 1, [k], NE[k] * NE[k + 1]))
                lists[0].append(("inverse", direction, k, None, NE[k] ** 2))
            if k + 1 >= nsub:
                continue
            base = xoff[jlo(k + 1, Sx)]
            C = int(xoff[k] - base)
            n2 = int(NE[k + 1])
            pc = piece_cols(pw, n2)
            for w in range(1, NW):
                c0, c1 = C * (w - 1) // (NW - 1), C * w // (NW - 1)
                for c in range(c0, c1, pc):
                    ce = min(c + pc, c1)
                    cols = (base + c, base + ce)  # global columns covered
                    lists[w].append(("piece", direction, k + 1, cols, (ce - c) * n2))
    return lists, xoff, pw


def sched_words(n_sub, Sx):
    return NW + 1 + n_sub * (4 * Sx + 16)


LAYOUTS = [(1, 1), (1, 7), (2, 1), (2, 2), (3, 5), (4, 4), (8, 8), (16, 16), (32, 2), (5, 40), (64, 3), (6, 22),
           (32, 32)]


@pytest.mark.parametrize("Sx,Sy", LAYOUTS)
@pytest.mark.parametrize("sizes", ["small", "uniform", "large"])
def test_schedule_fits_its_bound_and_covers_the_envelope(Sx, Sy, sizes):
    nsub = Sx * Sy
    rng = np.random.default_rng(Sx * 1000 + Sy)
    NE = {"small": np.full(nsub, 5), "uniform": rng.integers(5, 31, nsub), "large": np.full(nsub, 32)}[sizes]
    lists, xoff, pw = warp_lists(NE, Sx)
    total = sum(1 for l in lists for c in l if c[0] != "inverse-in-slot")
    assert NW + 1 + total <= sched_words(nsub, Sx)
    half = fifo_cap(pw) // 2
    assert all(c[4] + 3 <= half for l in lists for c in l if c[0] in ("piece", "pair"))  # two in flight
    assert all(c[4] + 3 <= fifo_cap(pw) for l in lists for c in l)
    for direction in (1, -1):
        # columns of each panel row r covered: leader blocks and the other warps' pieces
        cover = {r: np.zeros(int(xoff[r] - xoff[jlo(r, Sx)]), dtype=int) for r in range(nsub)}
        for l in lists:
            for c in l:
                if c[1] != direction or c[0] in ("inverse", "inverse-in-slot"):
                    continue
                r = c[2]
                b = xoff[jlo(r, Sx)]
                if c[0] in ("panel", "pair"):
                    for j in c[3]:
                        cover[r][xoff[j] - b: xoff[j + 1] - b] += 1
                else:
                    cover[r][c[3][0] - b: c[3][1] - b] += 1
        for r in range(nsub):
            assert np.all(cover[r] == 1), (direction, r)
        inv = sorted(c[2] for c in lists[0] if c[0] in ("inverse", "inverse-in-slot") and c[1] == direction)
        assert inv == list(range(nsub))
