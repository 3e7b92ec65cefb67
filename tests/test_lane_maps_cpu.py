"""Index logic of two solve routines, emulated lane by lane on the CPU (host
logic, no GPU):

- the FP64 residual's row sharing: p = floor(32 / N_E) lanes per row, lane
  q N_E + i summing the columns c = q (mod p) of row i, the partials met by
  shuffles from lanes i + u N_E;
- the single-warp diagonal block: right-looking Cholesky with lane = row
  (the update also runs over entries above the diagonal, which are never
  read) and the inverse row by row with lane = column over a zero-filled Y,
  on a work area whose unused entries hold NaN.
"""
import numpy as np
import pytest

rng = np.random.default_rng(20)


def _strided(a, ia, sa, x, ix, sx, n):
    return sum(a[ia + c * sa] * x[ix + c * sx] for c in range(n))


@pytest.mark.parametrize("NE", list(range(1, 33)))
def test_residual_row_sharing(NE):
    for Nl, Nr in ((1, 32), (7, 13), (32, 1)):
        Dg = rng.standard_normal((NE, NE)); Dg = Dg + Dg.T
        Bl = rng.standard_normal((Nl, NE))  # left neighbour block [N_{E-1}][N_E]
        Br = rng.standard_normal((NE, Nr))  # right neighbour block [N_E][N_{E+1}]
        xE, xl, xr = rng.standard_normal(NE), rng.standard_normal(Nl), rng.standard_normal(Nr)
        a = np.concatenate([Dg.reshape(-1), Bl.reshape(-1), Br.reshape(-1)])
        oL, oR = NE * NE, NE * NE + Nl * NE
        x = np.concatenate([xE, xl, xr])
        p = 32 // NE
        part = np.zeros(32)
        for lane in range(32):
            q, i = divmod(lane, NE)
            if q < p:
                part[lane] = (_strided(a, i + q * NE, p * NE, x, q, p, (NE - q + p - 1) // p)
                              + _strided(a, oL + i + q * NE, p * NE, x, NE + q, p, (Nl - q + p - 1) // p)
                              + _strided(a, oR + i * Nr + q, p, x, NE + Nl + q, p, (Nr - q + p - 1) // p))
        got = [part[i] + sum(part[(i + u * NE) & 31] for u in range(1, p)) for i in range(NE)]
        np.testing.assert_allclose(got, Dg @ xE + Bl.T @ xl + Br @ xr, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("N", [1, 2, 3, 5, 17, 31, 32])
def test_single_warp_diagonal_block(N):
    M = rng.standard_normal((N, N))
    A = M @ M.T + N * np.eye(N)
    ldd = N | 1
    W = np.full(4128, np.nan)  # the work area (the factor ring), unused entries NaN
    Y0 = (N * ldd + 3) & ~3
    dinv0 = Y0 + ((N * N + 3) & ~3)
    assert dinv0 + 32 <= W.size
    for i in range(N):
        W[i * ldd: i * ldd + i + 1] = A[i, : i + 1]  # lower triangle, lanes <= i
    for c in range(N):
        piv = W[c * ldd + c]
        d = np.sqrt(piv)
        li = np.zeros(32)
        for lane in range(c + 1, N):
            li[lane] = W[lane * ldd + c] / d
            W[lane * ldd + c] = li[lane]
        W[c * ldd + c] = d
        W[dinv0 + c] = 1.0 / d
        col = np.array([W[t * ldd + c] for t in range(N)])
        for lane in range(N):  # every t > c, also above the diagonal
            for t in range(c + 1, N):
                W[lane * ldd + t] -= li[lane] * col[t]
    L = np.array([[W[i * ldd + t] if t <= i else 0.0 for t in range(N)] for i in range(N)])
    np.testing.assert_allclose(L @ L.T, A, rtol=1e-12, atol=1e-11 * N)
    W[Y0:Y0 + N * N] = 0.0
    for i in range(N):
        s = np.array([(1.0 if lane == i else 0.0) - sum(W[i * ldd + t] * W[Y0 + t * N + lane] for t in range(i))
                      for lane in range(32)])
        for lane in range(min(i + 1, N)):
            W[Y0 + i * N + lane] = s[lane] * W[dinv0 + i]
    Y = W[Y0:Y0 + N * N].reshape(N, N)
    np.testing.assert_allclose(Y @ L, np.eye(N), atol=1e-10)
    assert not np.any(np.triu(Y, 1))
