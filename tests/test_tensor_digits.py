"""Host-side pins of the arithmetic the tensor layout relies on (the signed-digit
form of the limb decomposition of Sec. 4.1, run on bf16 tensor cores with f32
accumulation), restated here in numpy from the mathematics, independent of the
CUDA sources:

- a residue x < 2^30 has signed base-256 digits d_0..d_2 in [-128, 127] and d_3 in
  [0, 64] with x = sum 256^l d_l;
- every such digit is exact in bf16;
- f32 sums of up to 1024 digit products (each at most 2^14 in magnitude) are exact
  integers whatever the summation order, including the extreme 2^24;
- recombining the 16 digit-product sums with weights 2^(8(a+b)) mod q gives the
  modular product sum, and the int64 intermediate stays below 2^58;
- adding a digit to the bit pattern of 1.5 * 2^23 and subtracting 1.5 * 2^23 gives
  the digit as f32, whose top 16 bits are its bf16 encoding."""
import numpy as np
import pytest

Q = (1073479681, 1072496641)  # the two primes of the 1 GiB configuration (n = 4096, p = 2^16)


def signed_digits(x):
    """x: uint array < 2^30 -> int64 array [..., 4] of signed base-256 digits."""
    v = x.astype(np.int64)
    out = []
    for _ in range(3):
        low = v & 0xFF
        d = np.where(low >= 128, low - 256, low)
        out.append(d)
        v = (v - d) >> 8
    out.append(v)
    return np.stack(out, axis=-1)


def to_bf16_and_back(f32):
    """Round-to-nearest-even f32 -> bf16 -> f32."""
    bits = f32.astype(np.float32).view(np.uint32).astype(np.uint64)
    rounded = (bits + 0x7FFF + ((bits >> 16) & 1)) >> 16
    return (rounded << 16).astype(np.uint32).view(np.float32)


def edge_residues():
    vals = [0, 1, 127, 128, 129, 255, 256, 257, 32767, 32768, 65535, 65536, (1 << 24) - 1, 1 << 24,
            (1 << 30) - 1, 0x00808080, 0x00FF7F80, 0x3F807F80]
    vals += [q - 1 for q in Q] + [q // 2 for q in Q]
    return np.array(vals, dtype=np.uint64)


def test_signed_digits_recombine_and_stay_in_range():
    rng = np.random.default_rng(1)
    x = np.concatenate([edge_residues(), rng.integers(0, 1 << 30, size=200000, dtype=np.uint64)])
    d = signed_digits(x)
    w = np.array([1, 256, 65536, 1 << 24], dtype=np.int64)
    assert np.array_equal((d * w).sum(axis=-1), x.astype(np.int64))
    assert d[..., :3].min() >= -128 and d[..., :3].max() <= 127
    assert d[..., 3].min() >= 0 and d[..., 3].max() <= 64


def test_every_digit_is_exact_in_bf16():
    d = np.arange(-128, 129, dtype=np.int64).astype(np.float32)
    assert np.array_equal(to_bf16_and_back(d), d)
    # and a 9-bit odd integer is not: the range above is the whole exact range needed
    assert to_bf16_and_back(np.array([257.0], dtype=np.float32))[0] != 257.0


@pytest.mark.parametrize("kind", ["random", "all_min", "alternating"])
def test_f32_sums_of_1024_digit_products_are_exact(kind):
    rng = np.random.default_rng(2)
    K = 1024
    if kind == "random":
        a = rng.integers(-128, 128, size=(64, K))
        b = rng.integers(-128, 128, size=(64, K))
    elif kind == "all_min":  # every product (-128)(-128) = 2^14: the sum is exactly 2^24
        a = np.full((4, K), -128)
        b = np.full((4, K), -128)
    else:
        a = np.tile(np.array([-128, 127]), (8, K // 2))
        b = np.tile(np.array([127, -128]), (8, K // 2))
    prods = (a * b).astype(np.int64)
    exact = prods.sum(axis=1)
    assert np.abs(exact).max() <= 1 << 24
    pf = prods.astype(np.float32)
    # sequential left-to-right, pairwise (numpy's reduction), and shuffled orders
    seq = np.cumsum(pf, axis=1, dtype=np.float32)[:, -1]
    pair = np.add.reduce(pf, axis=1, dtype=np.float32)
    perm = rng.permutation(K)
    shuf = np.cumsum(pf[:, perm], axis=1, dtype=np.float32)[:, -1]
    for s in (seq, pair, shuf):
        assert np.array_equal(s.astype(np.int64), exact)
    if kind == "all_min":
        assert exact[0] == 1 << 24


def test_weighted_recombination_is_the_modular_product():
    rng = np.random.default_rng(3)
    for q in Q:
        M, K, N = 6, 1024, 5
        A = rng.integers(0, q, size=(M, K), dtype=np.uint64)
        B = rng.integers(0, q, size=(K, N), dtype=np.uint64)
        A[0] = q - 1  # the largest residues
        B[:, 0] = q - 1
        dA, dB = signed_digits(A), signed_digits(B)  # [M, K, 4], [K, N, 4]
        # P[a][b] = sum_k dA[., k, a] * dB[k, ., b]: 16 exact digit-product sums
        P = np.einsum("mka,knb->mnab", dA, dB)
        assert np.abs(P).max() <= K * (1 << 14)
        wt = np.array([[pow(2, 8 * (a + b), q) for b in range(4)] for a in range(4)], dtype=np.int64)
        # int64 sum as the epilogue forms it: |sum| < 16 * 2^24 * 2^30 = 2^58
        T = (P.astype(object) * wt.astype(object)).sum(axis=(2, 3))
        assert max(abs(int(t)) for t in T.ravel()) < 1 << 58
        got = np.array([[int(t) % q for t in row] for row in T], dtype=object)
        want = np.array([[sum(int(A[m, k]) * int(B[k, n]) for k in range(K)) % q for n in range(N)]
                         for m in range(M)], dtype=object)
        assert (got == want).all()


def test_bit_pattern_conversion_gives_the_bf16_digit():
    d = np.arange(-128, 128, dtype=np.int64)
    f = (np.int64(0x4B400000) + d).astype(np.uint32).view(np.float32) - np.float32(12582912.0)
    assert np.array_equal(f, d.astype(np.float32))
    top = (f.view(np.uint32) >> 16).astype(np.uint16)
    ref = (to_bf16_and_back(d.astype(np.float32)).view(np.uint32) >> 16).astype(np.uint16)
    assert np.array_equal(top, ref)
    assert np.all((f.view(np.uint32) & 0xFFFF) == 0)  # nothing below the bf16 bits
