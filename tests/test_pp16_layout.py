"""Layout algebra of the FP32 d = 16 packed-FMA product (csrc/pm_pp16.cuh), restated in numpy.

The kernel keeps 16 x 16 complex matrices as 16-byte chunks that pair two consecutive k of a
row (row layout, left operand) or of a column (column layout, right operand), multiplies the
k-pairs with two-wide FMAs and adds the even-k and odd-k halves at the end; an anti-Hermitian
right operand is read from its row layout with the real parts negated.  These tests check that
algebra, the lane tiling (every output owned once) and the shared-memory bank claims of its
comments, on the CPU.  The GPU parity tests check the kernel itself against the oracle.
"""

import numpy as np

RS = 9  # chunks (16 bytes) per physical row


def prow(i):
    return (i >> 1) + 8 * (i & 1)


def orow(a, r):
    return 2 * a + (r & 1) + 8 * (r >> 1)


def row_layout(M):
    """chunk (i, p) = (Re M[i,2p], Re M[i,2p+1], Im M[i,2p], Im M[i,2p+1]) at physical row prow(i)."""
    out = np.zeros((16, RS, 4))
    for i in range(16):
        for p in range(8):
            out[prow(i), p] = [M[i, 2 * p].real, M[i, 2 * p + 1].real, M[i, 2 * p].imag, M[i, 2 * p + 1].imag]
    return out


def col_layout(M):
    return row_layout(M.T)


def packed_product(Al, Bl, anti_hermitian_b=False):
    """C = A B from R(A) and C(B) (or R(B) of an anti-Hermitian B) by two-wide k-pair sums."""
    C = np.zeros((16, 16), np.complex128)
    for i in range(16):
        for j in range(16):
            sr = np.zeros(2)
            si = np.zeros(2)
            for p in range(8):
                ar, ai = Al[prow(i), p, 0:2], Al[prow(i), p, 2:4]
                x, y = Bl[prow(j), p, 0:2], Bl[prow(j), p, 2:4]
                if anti_hermitian_b:
                    n = -x
                    sr += ar * x + ai * y  # -(Re C)
                    si += ar * y + ai * n
                else:
                    n = -y
                    sr += ar * x + ai * n
                    si += ar * y + ai * x
            re = sr[0] + sr[1]
            C[i, j] = (-re if anti_hermitian_b else re) + 1j * (si[0] + si[1])
    return C


def rand_c(rng, shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def test_general_product():
    rng = np.random.default_rng(1)
    A, B = rand_c(rng, (16, 16)), rand_c(rng, (16, 16))
    C = packed_product(row_layout(A), col_layout(B))
    assert np.max(np.abs(C - A @ B)) < 1e-12


def test_anti_hermitian_operand_from_row_layout():
    rng = np.random.default_rng(2)
    G = rand_c(rng, (16, 16))
    G = (G + G.conj().T) / 2
    X = -1j * G  # the scaled exponent: anti-Hermitian
    X2 = packed_product(row_layout(X), row_layout(X), anti_hermitian_b=True)
    assert np.max(np.abs(X2 - X @ X)) < 1e-12
    Y = rand_c(rng, (16, 16))
    assert np.max(np.abs(packed_product(row_layout(Y), row_layout(X), True) - Y @ X)) < 1e-12


def test_lane_tiles_cover_the_output_once():
    owned = np.zeros((16, 16), int)
    for lane in range(32):
        a, b = lane >> 3, lane & 7
        for r in range(4):
            for c in range(2):
                owned[orow(a, r), 2 * b + c] += 1
    assert np.all(owned == 1)
    assert sorted(prow(i) for i in range(16)) == list(range(16))


def banks_of_16b(offsets):
    """4-byte banks touched by 16-byte accesses at the given byte offsets."""
    return [((o // 4) + k) % 32 for o in offsets for k in range(4)]


def test_quarter_warp_accesses_are_conflict_free():
    """Per quarter warp (8 lanes): the left-operand loads read one 16-byte word; the right-operand
    loads and both stores touch eight distinct words in 32 distinct banks."""
    for q in range(4):
        lanes = range(8 * q, 8 * q + 8)
        for p in range(8):
            for r in range(4):
                words = {(prow(orow(l >> 3, r)) * RS + p) * 16 for l in lanes}
                assert len(words) == 1
            for c in range(2):
                offs = [(prow(2 * (l & 7) + c) * RS + p) * 16 for l in lanes]
                assert len(set(offs)) == 8 and len(set(banks_of_16b(offs))) == 32
        for r in range(4):  # row-layout store
            offs = [(prow(orow(l >> 3, r)) * RS + (l & 7)) * 16 for l in lanes]
            assert len(set(banks_of_16b(offs))) == 32
        for c in range(2):  # column-layout store, both row pairs
            for h in range(2):
                offs = [(prow(2 * (l & 7) + c) * RS + (l >> 3) + 4 * h) * 16 for l in lanes]
                assert len(set(banks_of_16b(offs))) == 32
