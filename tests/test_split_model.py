"""A model, in numpy, of the arithmetic of the split product (balanced base-256
digits, one integer sum per level m = s + t, the epilogue's 64-bit / FP32
combination, optionally drained every C terms), checked against facts fixed
outside it: exact reconstruction of the digits, the FP64 product to the
digits' rounding level, and the size of the level sums that the FP32
accumulators must hold exactly (below 2^24).

The smooth case is a rank-one problem with evenly spaced poles and a smooth
positive z, and the row multiplied is the one parallel to z: the rows next to a
merge's split behave like it on matrices with smooth eigenvectors.  Over the
whole reduction its level-3 sums exceed 2^24 at K = 16384, which is the
exactness defect of the product path's default schedule; drained every 256
terms they stay below 2^23.  Verification only; the product path is CUDA."""
import numpy as np
import pytest

S = 7


def digits(x):
    """Balanced base-256 digits of round(x 2^56): d_0 carries the rest, d_1..d_6 in [-128, 127]."""
    F = np.rint(np.ldexp(np.asarray(x, dtype=np.float64), 56)).astype(np.int64)
    G = F + np.int64(sum(128 << (8 * i) for i in range(6)))
    out = [G >> 48]
    for sh in range(40, -1, -8):
        out.append(((G >> sh) & 255) - 128)
    return out


def level_sums(Ad, Ud, sl):
    """Exact integer level sums P_m over the terms in slice sl (float64 holds them exactly)."""
    return [sum(Ad[a][..., sl].astype(np.float64) @ Ud[m - a][sl].astype(np.float64) for a in range(m + 1))
            for m in range(S)]


def combine(A, U, chunk):
    """The epilogue: hi = sum_m<5 P_m 2^(8(4-m)) in 64-bit integers (exact) and
    lo = sum of 2^-8 P_6 + P_5 in FP32, both accumulated over chunks of `chunk`
    terms; C = (2^10 hi + round(4 lo)) 2^-58 (one conversion to double).  Also the
    largest |P_m| of any chunk."""
    Ad, Ud = digits(A), digits(U)
    K = A.shape[-1]
    hi = 0
    lo = np.float32(0.0)
    big = np.zeros(S)
    for c0 in range(0, K, chunk):
        P = level_sums(Ad, Ud, slice(c0, c0 + chunk))
        big = np.maximum(big, [np.abs(p).max() for p in P])
        hi = hi + sum(P[m].astype(np.int64) * (1 << (8 * (4 - m))) for m in range(5))
        lo = (lo + (P[6] * (1.0 / 256.0)).astype(np.float32)).astype(np.float32)
        lo = (lo + P[5].astype(np.float32)).astype(np.float32)
    I = hi * 1024 + np.rint(np.float32(4.0) * lo).astype(np.int64)
    return np.ldexp(I.astype(np.float64), -58), big


def test_digits_reconstruct_exactly():
    g = np.random.default_rng(1)
    x = np.concatenate([g.uniform(-1, 1, 4000), [1.0, -1.0, 0.0, 2.0 ** -57, -(2.0 ** -30), 1 - 2.0 ** -53]])
    d = digits(x)
    F = np.rint(np.ldexp(x, 56)).astype(np.int64)
    rebuilt = sum(d[s].astype(np.int64) << (8 * (6 - s)) for s in range(S))
    assert np.array_equal(rebuilt, F)
    assert np.all(np.abs(d[0]) <= 256)
    for s in range(1, S):
        assert d[s].min() >= -128 and d[s].max() <= 127
    # every digit is an integer that BF16 holds exactly (at most 8 significant bits)
    for s in range(S):
        v = np.abs(d[s])
        v = v[v > 0]
        assert np.all((v >> np.maximum(np.floor(np.log2(v)).astype(np.int64) - 7, 0)) << np.maximum(
            np.floor(np.log2(v)).astype(np.int64) - 7, 0) == v)


@pytest.mark.parametrize("chunk", [4096, 256])
def test_combination_matches_fp64_product(chunk):
    g = np.random.default_rng(2)
    K = 4096
    A = g.standard_normal((8, K))
    A /= np.linalg.norm(A, axis=1, keepdims=True)
    U = g.standard_normal((K, 16))
    U /= np.linalg.norm(U, axis=0, keepdims=True)
    C, big = combine(A, U, chunk)
    # dropped levels s + t >= 7 and the digit rounding: about 2^-56 per term pair
    assert np.abs(C - A @ U).max() <= 2.0 ** -50
    assert big.max() < 2.0 ** 24


def smooth_rank_one(orc, K):
    k = np.arange(K)
    D = np.linspace(-1.0, 1.0, K)
    z = np.sin(np.pi * (k + 1) / (K + 1)) + 0.1
    z /= np.linalg.norm(z)
    org, tau, _, _ = orc.secular(D, z, 1.0, max_iter=2000)
    zh = orc.lowner(D, z, 1.0, org, tau)
    s = orc.colnorm(D, org, tau, zh)
    cols = np.arange(0, K, 32)
    U = zh[:, None] * s[None, cols] / ((D[:, None] - D[org[cols]][None, :]) - tau[None, cols])
    return zh[None, :], U


def test_smooth_row_level_sums_need_chunked_drains(orc):
    A, U = smooth_rank_one(orc, 16384)
    C_whole, big_whole = combine(A, U, 16384)
    C_256, big_256 = combine(A, U, 256)
    # the model's combination is exact either way (integer sums)
    assert np.abs(C_whole - C_256).max() <= 2.0 ** -52
    assert np.abs(C_256 - A @ U).max() <= 2.0 ** -48
    # over the whole reduction the level-3 sums leave FP32's exact-integer range ...
    assert big_whole[3] > 2.0 ** 24
    # ... drained every 256 terms every level stays below 2^23
    assert big_256.max() < 2.0 ** 23


def test_hermite_8192_top_merge_rows_next_to_the_split(orc):
    """The same on a real merge: the top merge of the Hermite matrix (Example 2 family)
    of order 8192, children solved exactly, its top part's last eight rows (the rows
    next to the split) against every column of Qhat."""
    sla = pytest.importorskip("scipy.linalg")
    from paper_2008_01990_gb300 import inputs
    n = 8192
    d, e = inputs.hermite_tridiag(n)
    k = n // 2
    b = e[k - 1]
    d1 = d[:k].copy()
    d1[-1] -= abs(b)
    d2 = d[k:].copy()
    d2[0] -= abs(b)
    l1, Q1 = sla.eigh_tridiagonal(d1, e[:k - 1])
    l2, Q2 = sla.eigh_tridiagonal(d2, e[k:])
    z = np.concatenate([Q1[-1], np.sign(b) * Q2[0]]) / np.sqrt(2.0)
    K, kept, defl, D2, z2, Qr, t1, t2 = orc.deflate(np.concatenate([l1, l2]), z, 2.0 * abs(b))
    assert t2 == 0  # no rotations: the top part's columns are Q1's kept columns
    Dk, zk = D2[kept], z2[kept]
    rho = 2.0 * abs(b)
    org, tau, _, _ = orc.secular(Dk, zk, rho, max_iter=2000)
    zh = orc.lowner(Dk, zk, rho, org, tau)
    s = orc.colnorm(Dk, org, tau, zh)
    top = kept < k
    A = Q1[-8:, kept[top]]
    U = zh[top][:, None] * s[None, :] / ((Dk[top][:, None] - Dk[org][None, :]) - tau[None, :])
    kk = A.shape[1]
    C_whole, big_whole = combine(A, U, kk)
    C_256, big_256 = combine(A, U, 256)
    assert np.abs(C_256 - A @ U).max() <= 2.0 ** -48
    assert big_whole[3] > 2.0 ** 24
    assert big_256.max() < 2.0 ** 23


def magic_bits(v):
    """The epilogue's conversion of an exact FP32 integer |v| < 2^22: the bit pattern of
    v + 1.5 2^23 (computed in FP32), read as an unsigned integer."""
    return (np.asarray(v, dtype=np.float32) + np.float32(12582912.0)).view(np.uint32).astype(np.uint64)


def test_fp32_integer_conversion_by_offset():
    # every representable integer |v| < 2^22 maps to 0x4B400000 + v (no rounding in [2^23, 2^24))
    v = np.arange(-(1 << 22) + 1, 1 << 22, dtype=np.int64)
    b = magic_bits(v.astype(np.float32)).astype(np.int64)
    assert np.array_equal(b - 0x4B400000, v)
    # negative zero behaves like zero
    assert int(magic_bits(np.float32(-0.0))) == 0x4B400000


def test_offset_sums_modulo_2_64_recover_the_level_combination():
    """hi = sum over hand-offs and levels of bits(P_m) 2^(8(4-m)) kept modulo 2^64, minus the
    summed offsets, equals sum P_m 2^(8(4-m)) in exact integers (Python ints)."""
    g = np.random.default_rng(5)
    for trial in range(50):
        chunks = int(g.integers(1, 40))
        P = g.integers(-(1 << 22) + 1, 1 << 22, size=(chunks, 5))
        hu, bias, exact = 0, 0, 0
        for c in range(chunks):
            for m in range(5):
                sh = 8 * (4 - m)
                hu = (hu + (int(magic_bits(np.float32(P[c, m]))) << sh)) % (1 << 64)
                bias = (bias + (0x4B400000 << sh)) % (1 << 64)
                exact += int(P[c, m]) << sh
        got = (hu - bias) % (1 << 64)
        if got >= 1 << 63:
            got -= 1 << 64
        assert got == exact
