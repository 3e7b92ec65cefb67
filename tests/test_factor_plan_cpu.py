"""The mixed solver's refactorisation schedule, whole and staged (host only).

The plan of each step comes from the library itself (lrbms_test_factor_plan
calls the same function the factor kernel runs); the state updates between
steps are the kernels' bookkeeping on success: a whole factorisation sets
the factor age to 1, the last stage of a staged build switches to the built
buffer and sets age 1, and every solve adds 1 to the age."""
import numpy as np
import pytest

AGE, REFACTOR, BUF, STAGED = 6, 7, 8, 9


@pytest.fixture(scope="module")
def L():
    from paper_1405_2810_gb300 import build, lrbms
    build.build()
    return lrbms


def run(L, n_sub, P, R, n_steps, force_at=()):
    """Per step: (plan, buffer the solve uses, step at which each row of
    that factor was computed)."""
    info = np.zeros(12, dtype=np.int32)
    made = {0: np.full(n_sub, -1), 1: np.full(n_sub, -1)}  # step each row of each buffer was computed
    out = []
    for t in range(n_steps):
        if t in force_at:
            info[REFACTOR] = 1
        k0, k1, buf, whole, last = L.lrbms_test_factor_plan(n_sub, P, R, info)
        made[buf][k0:k1] = t
        if whole:
            info[AGE], info[REFACTOR], info[STAGED] = 1, 0, 0
        elif last:
            info[BUF], info[AGE], info[STAGED] = buf, 1, 1
        used = int(info[BUF])
        out.append(((k0, k1, buf, whole, last), used, made[used].copy()))
        info[AGE] += 1  # the solve
    return out


@pytest.mark.parametrize("n_sub", [1, 2, 5, 16, 64, 256])
@pytest.mark.parametrize("P", [1, 2, 3, 4, 8, 12])
def test_whole_refactorisation_every_period(L, n_sub, P):
    steps = run(L, n_sub, P, 1, 6 * P + 3)
    whole_at = [t for t, (p, _, _) in enumerate(steps) if p[3]]
    assert whole_at == list(range(0, 6 * P + 3, P))
    for t, (p, used, rows) in enumerate(steps):
        assert p[3] or p[1] <= p[0]  # only whole factorisations
        assert used == 0 and np.all(rows == t - t % P)  # the factor of the period's first step


@pytest.mark.parametrize("n_sub", [1, 2, 5, 16, 64, 256])
@pytest.mark.parametrize("P,R", [(2, 2), (3, 2), (4, 4), (8, 2), (8, 4), (8, 8), (12, 5)])
def test_staged_builds(L, n_sub, P, R):
    n = 8 * P + 1
    steps = run(L, n_sub, P, R, n)
    assert [t for t, (p, _, _) in enumerate(steps) if p[3]] == [0]  # one whole factorisation, the first
    assert [t for t, (p, _, _) in enumerate(steps) if p[4]] == list(range(P, n, P))  # a new factor every P steps
    cap = -(-n_sub // R)
    for t, (p, used, rows) in enumerate(steps):
        k0, k1, buf, whole, last = p
        if not whole:
            assert k1 - k0 <= cap
            if k1 > k0:
                assert buf != (used if not last else 1 - used)  # builds go to the idle buffer
        assert np.all(rows >= 0)  # the factor in use is complete
        if t >= P:
            # rows of the factor in use: from the R steps of its build, the oldest at most P + R - 1 back
            assert rows.max() - rows.min() <= R - 1 and t - rows.min() <= P + R - 1
            assert np.all(np.diff(rows) >= 0)  # built in row order
    # each build computes every row exactly once, in order, in consecutive stages
    for b in range(1, n // P):
        stage_steps = range(b * P - R + 1, b * P + 1)
        ranges = [steps[t][0][:2] for t in stage_steps]
        assert ranges[0][0] == 0 and ranges[-1][1] == n_sub
        assert all(ranges[i][1] == ranges[i + 1][0] for i in range(R - 1))


def test_forced_refactorisation_restarts_the_build(L):
    """A solve that needed too many passes (or a stage with a non-positive
    pivot) forces a whole factorisation at the next step; staging resumes
    from the first stage afterwards."""
    P, R, n_sub = 8, 4, 64
    steps = run(L, n_sub, P, R, 40, force_at={6})
    whole_at = [t for t, (p, _, _) in enumerate(steps) if p[3]]
    assert whole_at == [0, 6]
    assert [t for t, (p, _, _) in enumerate(steps) if p[4]] == [14, 22, 30, 38]
    assert steps[11][0][:2] == (0, 16)  # first stage of the build after the forced factorisation


def test_plan_rejects_bad_sizes(L):
    info = np.zeros(12, dtype=np.int32)
    for args in ((0, 8, 1), (4, 0, 1), (4, 8, 0), (4, 4, 5)):
        with pytest.raises(L.LrbmsError):
            L.lrbms_test_factor_plan(*args, info)
