"""Pins for the oracle's NTT: evaluation at the roots of X^n + 1 computed in pure
Python, the convolution theorem against a pure-Python schoolbook negacyclic
product, round trips and linearity."""
import numpy as np
import pytest


def brv(x, bits):
    return int(format(x, "0%db" % bits)[::-1], 2) if bits else 0


def py_negacyclic(a, b, q):
    n = len(a)
    out = [0] * n
    for s in range(n):
        for t in range(n):
            k = s + t
            if k < n:
                out[k] = (out[k] + a[s] * b[t]) % q
            else:
                out[k - n] = (out[k - n] - a[s] * b[t]) % q
    return out


def params_for(orc, n):
    log2p = max(1, (2 * n).bit_length() - 1)  # p = 2n keeps M = 2n
    q = orc.select_primes(n, log2p, 1)[0]
    return q, orc.find_psi(q, n)


@pytest.mark.parametrize("n", [2, 4, 8, 16, 32])
def test_definition_is_evaluation_at_odd_root_powers(orc, n):
    q, psi = params_for(orc, n)
    rng = np.random.default_rng(n)
    a = rng.integers(0, q, size=n, dtype=np.uint64).astype(np.uint32)
    A = orc.ntt_definition(a, q, psi)
    bits = n.bit_length() - 1
    for k in range(n):
        x = pow(psi, 2 * brv(k, bits) + 1, q)
        assert pow(x, n, q) == q - 1  # a root of X^n + 1
        val = 0
        for coef in reversed([int(v) for v in a]):  # Horner
            val = (val * x + coef) % q
        assert int(A[k]) == val


@pytest.mark.parametrize("n", [2, 8, 64, 256, 1024, 2048])
def test_fast_matches_definition(orc, n):
    q, psi = params_for(orc, n)
    rng = np.random.default_rng(100 + n)
    a = rng.integers(0, q, size=n, dtype=np.uint64).astype(np.uint32)
    assert np.array_equal(orc.ntt_fwd(a, q, psi), orc.ntt_definition(a, q, psi))
    A = orc.ntt_definition(a, q, psi)
    assert np.array_equal(orc.ntt_inv(A, q, psi), a)
    if n <= 256:
        assert np.array_equal(orc.intt_definition(A, q, psi), a)


@pytest.mark.parametrize("n", [4, 16, 32])
def test_c_schoolbook_matches_python(orc, n):
    q, _ = params_for(orc, n)
    rng = np.random.default_rng(7 * n)
    a = rng.integers(0, q, size=n, dtype=np.uint64).astype(np.uint32)
    b = rng.integers(0, q, size=n, dtype=np.uint64).astype(np.uint32)
    ref = py_negacyclic([int(v) for v in a], [int(v) for v in b], q)
    assert [int(v) for v in orc.negacyclic_schoolbook(a, b, q)] == ref


@pytest.mark.parametrize("n", [4, 16, 64, 512, 2048])
def test_convolution_theorem(orc, n):
    """INTT(NTT(a) * NTT(b)) is the product in Z_q[X]/(X^n + 1)."""
    q, psi = params_for(orc, n)
    rng = np.random.default_rng(11 * n)
    a = rng.integers(0, q, size=n, dtype=np.uint64).astype(np.uint32)
    b = rng.integers(0, q, size=n, dtype=np.uint64).astype(np.uint32)
    A, Bh = orc.ntt_fwd(a, q, psi), orc.ntt_fwd(b, q, psi)
    prod = ((A.astype(np.uint64) * Bh.astype(np.uint64)) % np.uint64(q)).astype(np.uint32)
    got = orc.ntt_inv(prod, q, psi)
    if n <= 64:
        ref = np.array(py_negacyclic([int(v) for v in a], [int(v) for v in b], q), dtype=np.uint32)
    else:
        ref = orc.negacyclic_schoolbook(a, b, q)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("n,log2p", [(2048, 12), (4096, 16), (8192, 16)])
def test_config_rings_roundtrip_and_linearity(orc, n, log2p):
    P = orc.make_params(n, log2p, 2, 2, 2)
    rng = np.random.default_rng(n)
    for q, psi in zip(P.qs, P.psis):
        a = rng.integers(0, q, size=n, dtype=np.uint64).astype(np.uint32)
        b = rng.integers(0, q, size=n, dtype=np.uint64).astype(np.uint32)
        A, Bh = orc.ntt_fwd(a, q, psi), orc.ntt_fwd(b, q, psi)
        assert np.array_equal(orc.ntt_inv(A, q, psi), a)
        s = ((a.astype(np.uint64) + b.astype(np.uint64)) % np.uint64(q)).astype(np.uint32)
        S = ((A.astype(np.uint64) + Bh.astype(np.uint64)) % np.uint64(q)).astype(np.uint32)
        assert np.array_equal(orc.ntt_fwd(s, q, psi), S)
        # X * a(X) is a negacyclic shift: coefficient n-1 wraps to 0 with a minus sign
        x = np.zeros(n, dtype=np.uint32)
        x[1] = 1
        X = orc.ntt_fwd(x, q, psi)
        XA = ((X.astype(np.uint64) * A.astype(np.uint64)) % np.uint64(q)).astype(np.uint32)
        shifted = np.roll(a, 1)
        shifted[0] = (q - int(a[-1])) % q
        assert np.array_equal(orc.ntt_inv(XA, q, psi), shifted)


def test_rns_batch_matches_single(orc):
    P = orc.make_params(2048, 12, 2, 2, 2)
    rng = np.random.default_rng(3)
    polys = np.stack([rng.integers(0, q, size=(5, 2048), dtype=np.uint64).astype(np.uint32) for q in P.qs], axis=1)
    out = orc.ntt_fwd_rns(P, polys, nthreads=3)
    for c in range(5):
        for j, (q, psi) in enumerate(zip(P.qs, P.psis)):
            assert np.array_equal(out[c, j], orc.ntt_fwd(polys[c, j], q, psi))
    assert np.array_equal(orc.ntt_inv_rns(P, out), polys)
