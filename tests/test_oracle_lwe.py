"""Pins for the oracle's scalar-HE (LWE) DB GEMM (Sec. 2.5, Sec. 4.1, App. A.1):
pure-Python brute force on tiny shapes, including the extremes of signed INT8 and of
Z_{2^32}; the byte-plane identity of Sec. 4.1 (A Q = sum_k 2^(8k) A Q_k mod 2^32
with Q_k the k-th bytes of Q); and a toy SimplePIR round trip: the client's query
q = A_lwe s + e + Delta u_i*, the server's answer DB q and hint DB A_lwe, and the
client's decryption returns column i* of the DB."""
import numpy as np
import pytest

import synth

MOD = 1 << 32


def brute(A, Q):
    D1, D0 = A.shape
    return [[sum(int(A[i, j]) * int(Q[b, j]) for j in range(D0)) % MOD for i in range(D1)] for b in range(Q.shape[0])]


@pytest.mark.parametrize("D1,D0,B", [(1, 1, 1), (3, 7, 2), (5, 64, 3), (9, 33, 4)])
def test_brute_force(orc, D1, D0, B):
    rng = np.random.default_rng(D1 * 100 + D0)
    A = rng.integers(-128, 128, size=(D1, D0)).astype(np.int8)
    Q = rng.integers(0, MOD, size=(B, D0), dtype=np.uint64).astype(np.uint32)
    assert orc.lwe_gemm(A, Q).tolist() == brute(A, Q)


def test_extremes_wrap_around(orc):
    D0 = 40
    A = np.array([[-128] * D0, [127] * D0, [-1, 1] * (D0 // 2)], dtype=np.int8)
    Q = np.array([[MOD - 1] * D0, [1 << 31] * D0, list(range(D0))], dtype=np.uint32)
    got = orc.lwe_gemm(A, Q).tolist()
    assert got == brute(A, Q)
    assert got[0][0] == (-128 * (MOD - 1) * D0) % MOD


def test_byte_plane_identity(orc):
    rng = np.random.default_rng(4)
    A = rng.integers(-128, 128, size=(6, 96)).astype(np.int8)
    Q = rng.integers(0, MOD, size=(3, 96), dtype=np.uint64).astype(np.uint32)
    total = np.zeros((3, 6), dtype=np.uint64)
    for k in range(4):
        Qk = ((Q >> (8 * k)) & 0xFF).astype(np.uint32)
        total = (total + (orc.lwe_gemm(A, Qk).astype(np.uint64) << (8 * k))) % MOD
    assert np.array_equal(total.astype(np.uint32), orc.lwe_gemm(A, Q))


def test_simplepir_round_trip(orc):
    """App. A.1 LWE with p = 2^8, q = 2^32, Delta = 2^24 (toy dimension n = 64)."""
    D1, D0, n, B = 24, 256, 64, 3
    delta = 1 << 24
    rng = np.random.default_rng(7)
    db = rng.integers(-128, 128, size=(D1, D0)).astype(np.int8)
    A_lwe = synth.u64(5, synth.STREAM_A, 0, D0 * n).reshape(D0, n).astype(np.uint64) & 0xFFFFFFFF
    s = synth.ternary_secret(5, n).astype(np.int64)
    # hint = DB A_lwe (offline): columns of A_lwe act as n query vectors
    hint = orc.lwe_gemm(db, A_lwe.T.astype(np.uint32)).T.astype(np.int64)  # [D1][n]
    idx = synth.query_indices(5, B, 1, D0)
    Q = np.empty((B, D0), dtype=np.uint32)
    for b in range(B):
        e = synth.gaussian_error(5, D0, start=b * D0).astype(np.int64)
        As = (A_lwe.astype(object).dot(s.astype(object)))
        q = [(int(As[j]) + int(e[j]) + (delta if j == int(idx[b]) else 0)) % MOD for j in range(D0)]
        Q[b] = np.array(q, dtype=np.uint64).astype(np.uint32)
    ans = orc.lwe_gemm(db, Q)  # [B][D1]
    for b in range(B):
        for i in range(D1):
            phase = (int(ans[b, i]) - sum(int(hint[i, t]) * int(s[t]) for t in range(n))) % MOD
            phase = phase - MOD if phase >= MOD // 2 else phase
            m = round(phase / delta) % 256
            assert m == int(db[i, int(idx[b])]) % 256, (b, i)
