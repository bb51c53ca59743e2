"""The block-Jacobi preconditioner's 6x6 inverse (Sec. 7) as the PCG forms
it on the device -- from the block's lower triangle, with Newton-refined
pivot reciprocals: Gauss-Jordan sweeps in double-float pairs on eight lanes
per block (mode 0, the default precision), LDLᵀ in FP64 (mode 1, the FP64
variant) or LDLᵀ in FP64 on FP32 blocks (mode 2) -- against the FP64
inverse from LAPACK,
over conditioning from 1 to 1e6, magnitudes from 1e-33 to 1e6 (the smallest
below the range where the reciprocal's FP32 seed is used), an upper triangle
that differs from the lower one, and blocks that are not positive
definite."""
import numpy as np
import pytest

import paper_1904_13073_gb300 as sw

from gpu_helpers import ensure_built

pytestmark = pytest.mark.gpu

TRI = [(r, c) for r in range(6) for c in range(r + 1)]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_built()


def _spd(rng, cond, scale):
    q, _ = np.linalg.qr(rng.standard_normal((6, 6)))
    ev = np.geomspace(1.0, cond, 6)
    rng.shuffle(ev)
    return scale * (q * ev) @ q.T


def _blocks(rng):
    out, conds = [], []
    for cond in (1.0, 10.0, 1e3, 1e6):
        for scale in (1e-33, 1e-6, 1.0, 1e6):
            for _ in range(4):
                out.append(_spd(rng, cond, scale))
                conds.append(cond)
    return np.array(out), np.array(conds)


def _packed(m):
    return np.array([m[r, c] for r, c in TRI])


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_block_inverse_matches_lapack(mode):
    fp64 = mode == 1
    rng = np.random.default_rng(5)
    B, conds = _blocks(rng)
    dt = np.float64 if fp64 else np.float32
    Bd = B.astype(dt)
    # the upper triangle off by a few ulps: the device reads the lower one
    Bd[::3, 1, 4] = np.nextafter(np.nextafter(Bd[::3, 1, 4], np.inf), np.inf)
    inv, ok = sw.sw_debug_block_inverse(Bd, mode=mode)
    assert ok.all()
    for k in range(len(Bd)):
        S = np.tril(Bd[k].astype(np.float64))
        S = S + np.tril(S, -1).T
        want = _packed(np.linalg.inv(S))
        got = inv[k].astype(np.float64)
        big = np.abs(want).max()
        if fp64:
            tol = 1e-13 * conds[k] * big
        else:   # the FP32 result: one rounding, plus an error far below it (46-48-bit arithmetic)
            tol = np.spacing(np.abs(want).astype(np.float32)).astype(np.float64) + 1e-12 * conds[k] * big
        assert np.all(np.abs(got - want) <= tol), (k, conds[k], np.abs(got - want).max(), big)


def test_block_inverse_flags_blocks_that_are_not_positive_definite():
    rng = np.random.default_rng(6)
    good = _spd(rng, 10.0, 1.0)
    neg = good.copy()
    neg[5, 5] = -1.0                       # last pivot negative
    q, _ = np.linalg.qr(rng.standard_normal((6, 6)))
    indef = (q * np.array([3.0, 2.0, 1.0, -0.5, 1.0, 2.0])) @ q.T
    zero = np.zeros((6, 6))
    semi = np.diag([1.0, 1.0, 1.0, 1.0, 1.0, 0.0])   # singular: a zero pivot
    B = np.array([good, neg, indef, zero, semi])
    for mode in (0, 1, 2):
        _, ok = sw.sw_debug_block_inverse(B, mode=mode)
        assert ok.tolist() == [True, False, False, False, False]


def test_block_inverse_of_a_diagonal_block_is_exact_reciprocals():
    """Diagonal input: M⁻¹ is the reciprocals of the diagonal, correctly
    rounded to FP32 (FP32 mode) and within an ulp of the FP64 quotient."""
    d = np.array([1.0, 3.0, 7.0, 1e-5, 12345.678, 0.1])
    inv, ok = sw.sw_debug_block_inverse(np.diag(d)[None], fp64=True)
    assert ok[0]
    diag = inv[0][[0, 2, 5, 9, 14, 20]]
    assert np.all(np.abs(diag - 1.0 / d) <= np.spacing(1.0 / d))
    assert np.all(inv[0][[1, 3, 4, 6, 7, 8]] == 0.0)
    want = (1.0 / d.astype(np.float32).astype(np.float64)).astype(np.float32)
    for mode in (0, 2):
        inv32, ok = sw.sw_debug_block_inverse(np.diag(d).astype(np.float32)[None], mode=mode)
        assert ok[0]
        np.testing.assert_array_equal(inv32[0][[0, 2, 5, 9, 14, 20]], want)
