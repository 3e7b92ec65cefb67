"""Size bound of the substitution copy schedule (host logic, no GPU).

The library builds, once per simulation, the per-warp list of chunks that the
pipelined substitutions copy (forward, then backward). The buffer holding it
is sized by a closed-form bound: kSolveWarps + 1 list starts plus n_sub (2 Sx
+ 3) descriptors. This test enumerates the chunk lists the same way (block
rows in order; the leader takes the coupling block to the previous/next row
and the diagonal inverse, the other warps take the coupling blocks of the
rows within the envelope, dealt in turn) for many subdomain layouts and
checks the bound, and that every chunk of the envelope is copied exactly once
per direction."""
import pytest

NW = 4  # warps per CTA of the reduced solve


def jlo(k, Sx):
    return max(0, k - Sx)


def n_citems(nsub, Sx, direction, k):
    if direction > 0:
        return max(0, min(k - 1 + Sx, nsub - 1) - k) if k >= 1 else 0
    return k - jlo(k + 1, Sx) if k <= nsub - 2 else 0


def warp_lists(nsub, Sx):
    lists = [[] for _ in range(NW)]
    for direction in (1, -1):
        rows = range(nsub) if direction > 0 else range(nsub - 1, -1, -1)
        for k in rows:
            # leader: coupling block to the previous (forward) / next (backward) row, then L_kk^-1
            if direction > 0 and k >= 1:  # row k at block k-1
                lists[0].append(("panel", direction, k, k - 1))
            if direction < 0 and k <= nsub - 2:  # row k+1 at block k
                lists[0].append(("panel", direction, k + 1, k))
            lists[0].append(("inverse", direction, k))
            for i in range(n_citems(nsub, Sx, direction, k)):
                w = 1 + i % (NW - 1)
                if direction > 0:  # row k+1+i at block k-1
                    lists[w].append(("panel", direction, k + 1 + i, k - 1))
                else:  # row k+1 at block jlo(k+1)+i
                    lists[w].append(("panel", direction, k + 1, jlo(k + 1, Sx) + i))
    return lists


def sched_words(n_sub, Sx):
    return NW + 1 + n_sub * (2 * Sx + 3)


@pytest.mark.parametrize("Sx,Sy", [(1, 1), (1, 7), (2, 1), (2, 2), (3, 5), (4, 4), (8, 8), (16, 16),
                                   (32, 2), (5, 40), (64, 3), (6, 22)])
def test_schedule_fits_its_bound_and_covers_the_envelope(Sx, Sy):
    nsub = Sx * Sy
    lists = warp_lists(nsub, Sx)
    total = sum(len(l) for l in lists)
    assert NW + 1 + total <= sched_words(nsub, Sx)
    # every off-diagonal block (r, j) of the envelope, jlo(r) <= j < r, is copied once per
    # direction: forward as (row r at block j), backward as (row r at block j) too
    for direction in (1, -1):
        got = sorted((c[2], c[3]) for l in lists for c in l if c[0] == "panel" and c[1] == direction)
        want = sorted((r, j) for r in range(nsub) for j in range(jlo(r, Sx), r))
        assert got == want
        inv = sorted(c[2] for c in lists[0] if c[0] == "inverse" and c[1] == direction)
        assert inv == list(range(nsub))
