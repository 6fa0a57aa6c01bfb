"""Pins for the oracle's RGSW-RLWE external product and the folding of the remaining
dimensions (Sec. 3.2, Sec. 3.6; gadget of App. D.3):

- RGSW(1) (x) Enc(m) decrypts to m, RGSW(0) (x) Enc(m) to 0, and RGSW(X^k) (x) Enc(m) to
  the negacyclic product X^k m (pure-Python shift).  The added noise stays inside the
  worst-case bound sum over 2 ell digits of n (t - 1) 19.
- Folding 2^levels ciphertexts of distinct messages with RGSW encryptions of the bits
  of c* decrypts to message c*, for every c*.
- End to end on the tiny configuration: the first-dimension answer of a one-hot query,
  folded with the bits of c*, decrypts to the single record DB[i*][c*].
"""
import numpy as np
import pytest

import synth

ERR_BOUND = 19


def client(P, seed, count):
    s = synth.ternary_secret(seed, P.n)
    a = synth.uniform_residues(seed, synth.STREAM_A, count, P.n, P.qs)
    e = synth.gaussian_error(seed, count * P.n).reshape(count, P.n)
    return s, a, e


def ext_noise_bound(P, ell, w):
    return 2 * ell * P.n * ((1 << w) - 1) * ERR_BOUND


def rgsw_of(orc, P, s, mu, ell, seed):
    a = synth.uniform_residues(seed, synth.STREAM_KEY_A, 2 * ell, P.n, P.qs)
    e = synth.gaussian_error(seed, 2 * ell * P.n, stream=synth.STREAM_KEY_ERROR).reshape(2 * ell, P.n)
    return orc.rgsw_encrypt(P, s, mu, ell, a, e)


def negacyclic_shift(m, k, p):
    n = len(m)
    out = [0] * n
    for t in range(n):
        e = t + k
        if e < n:
            out[e] = int(m[t]) % p
        else:
            out[e - n] = (-int(m[t])) % p
    return out


@pytest.mark.parametrize("L,ell", [(2, 4), (2, 6), (3, 4)])
def test_external_product(orc, L, ell):
    P = orc.make_params(512, 10, 1, 1, L)
    n, p = P.n, 1 << P.log2p
    w = orc.gadget_bits(P, ell)
    s, a, e = client(P, 60 + L, 1)
    m = np.random.default_rng(ell).integers(0, p, size=n).astype(np.uint32)
    ct = orc.bfv_encrypt(P, s, a[0], e[0], m)
    for mu_k, want in ((None, np.zeros(n, dtype=np.uint32)), (0, m),
                       (5, np.array(negacyclic_shift(m, 5, p), dtype=np.uint32))):
        mu = np.zeros(n, dtype=np.uint32)
        if mu_k is not None:
            mu[mu_k] = 1
        out = orc.external_product(P, rgsw_of(orc, P, s, mu, ell, seed=70 + (mu_k or 0)), ell, ct)
        assert np.array_equal(orc.bfv_decrypt(P, s, out), want), mu_k
        # the input noise is moved by mu (zero, itself, or shifted), plus the digits' errors
        assert np.abs(orc.bfv_noise(P, s, out, want)).max() <= ERR_BOUND + ext_noise_bound(P, ell, w)


@pytest.mark.parametrize("levels", [1, 3])
def test_fold_selects_every_index(orc, levels):
    P = orc.make_params(256, 10, 1, 1, 2)
    n, p, ell = P.n, 1 << P.log2p, 4
    count = 1 << levels
    s, a, e = client(P, 80 + levels, count)
    msgs = np.random.default_rng(levels).integers(0, p, size=(count, n)).astype(np.uint32)
    cts = np.stack([orc.bfv_encrypt(P, s, a[j], e[j], msgs[j]) for j in range(count)])
    for c_star in range(count):
        bits = [(c_star >> l) & 1 for l in range(levels)]
        out = orc.fold(P, cts, levels, orc.rgsw_bits(P, s, bits, ell, seed=c_star), ell)
        assert np.array_equal(orc.bfv_decrypt(P, s, out), msgs[c_star]), c_star


def test_first_dimension_then_fold_decrypts_one_record(orc):
    n, log2p, D1, D2, ell = 2048, 12, 16, 16, 6
    P = orc.make_params(n, log2p, D1, D2, 2)
    raw = synth.raw_db(0, synth.raw_db_bytes(n, log2p, D1, D2))
    for seed in (1, 2):
        idx = int(synth.query_indices(seed, 1, D1, D2)[0])
        i_star, c_star = divmod(idx, D2)
        s, a, e = client(P, seed, D1)
        Q = orc.encrypt_query(P, s, a, e, i_star)[None]
        R = orc.answer(P, raw, Q)[0]  # [D2][2][L][n]
        levels = (D2 - 1).bit_length()
        bits = [(c_star >> l) & 1 for l in range(levels)]
        out = orc.fold(P, R, levels, orc.rgsw_bits(P, s, bits, ell, seed=seed), ell)
        assert np.array_equal(orc.bfv_decrypt(P, s, out), orc.unpack_poly(raw, log2p, n, i_star * D2 + c_star))


def schoolbook_negacyclic(a, b, q):
    """(a * b) mod (X^n + 1, q), plain double loop over Python integers."""
    n = len(a)
    out = [0] * n
    for i in range(n):
        ai = int(a[i])
        if ai == 0:
            continue
        for j in range(n):
            k = i + j
            if k < n:
                out[k] += ai * int(b[j])
            else:
                out[k - n] -= ai * int(b[j])
    return [v % q for v in out]


@pytest.mark.parametrize("L,ell", [(1, 3), (2, 4), (3, 5)])
def test_noiseless_external_product_is_the_ring_product(orc, L, ell):
    """With zero masks and zero errors, RGSW(mu) is the bare gadget (mu t^k in the
    a-part of row k, in the b-part of row ell + k).  The external product must then
    give exactly (mu * c_a, mu * c_b) in R_q, since the digits recombine to the lift
    of each coefficient: an exact identity that a mis-paired row or digit, a wrong
    base or a dropped negacyclic sign breaks."""
    P = orc.make_params(64, 10, 1, 1, L)
    n = P.n
    rng = np.random.default_rng(L * 10 + ell)
    mu = np.zeros(n, dtype=np.uint32)
    mu[[0, 3, n - 1]] = [1, 2, 1]  # a small polynomial touching the wrap-around
    zero_a = np.zeros((2 * ell, L, n), dtype=np.uint32)
    zero_e = np.zeros((2 * ell, n), dtype=np.int8)
    s = synth.ternary_secret(5, n)
    G = orc.rgsw_encrypt(P, s, mu, ell, zero_a, zero_e)
    ct = np.stack([np.stack([rng.integers(0, q, size=n, dtype=np.uint64).astype(np.uint32) for q in P.qs])
                   for _ in range(2)])
    out = orc.external_product(P, G, ell, ct)
    for comp in range(2):
        for j, q in enumerate(P.qs):
            assert out[comp, j].tolist() == schoolbook_negacyclic(mu, ct[comp, j], q), (comp, j)
