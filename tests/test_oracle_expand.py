"""Pins for the oracle's query expansion (Sec. 3.5; App. C.2, SealPIR's recursion
with the 2^-levels pre-scaling; gadget of App. D.3).

- Substitution tau_g against polynomial evaluation: (tau_g a)(w) = a(w^g) at every
  primitive 2n-th root w, by Horner in pure Python.
- tau_g is a ring automorphism, tau_g tau_h = tau_{gh mod 2n}, with the schoolbook
  negacyclic product.
- The gadget base is t = 2^ceil(log2 q / ell) from the bit length of q.
- Subs(Enc(m), g) decrypts to tau_g(m), with its noise inside the worst-case bound
  of one key switch.
- Expansion recovers every coefficient, including the exact aliasing of
  coefficients at and above 2^levels.  Its noise stays inside the bound derived from
  the recursion.
- A packed one-hot query, expanded and answered, decrypts to the requested DB row
  on the tiny configuration at L = 2 and on a 3-prime configuration.
"""
import numpy as np
import pytest

import synth

ERR_BOUND = 19  # |e| <= 19 for the clipped Gaussian (App. A.1)


def horner(coeffs, x, q):
    acc = 0
    for c in reversed(coeffs):
        acc = (acc * x + int(c)) % q
    return acc


@pytest.mark.parametrize("g", [3, 5, 17, 31, 33])
def test_automorphism_is_evaluation_at_powers(orc, g):
    P = orc.make_params(16, 4, 1, 1, 1)
    q, psi, n = P.qs[0], P.psis[0], P.n
    a = synth.uniform_residues(g, synth.STREAM_UNIFORM, 1, n, P.qs).reshape(n)
    ta = orc.automorphism(a, q, g)
    for k in range(n):
        w = pow(psi, 2 * k + 1, q)
        assert horner(ta, w, q) == horner(a, pow(w, g, q), q)


def test_automorphism_is_a_ring_automorphism(orc):
    P = orc.make_params(32, 4, 1, 1, 1)
    q, n = P.qs[0], P.n
    a, b = synth.uniform_residues(3, synth.STREAM_UNIFORM, 2, n, P.qs).reshape(2, n)
    for g in (3, 7, n + 1, 2 * n - 1):
        lhs = orc.automorphism(orc.negacyclic_schoolbook(a, b, q), q, g)
        rhs = orc.negacyclic_schoolbook(orc.automorphism(a, q, g), orc.automorphism(b, q, g), q)
        assert np.array_equal(lhs, rhs), g
    for g, h in ((3, 5), (n + 1, 7), (2 * n - 1, 2 * n - 1)):
        assert np.array_equal(orc.automorphism(orc.automorphism(a, q, h), q, g),
                              orc.automorphism(a, q, g * h % (2 * n))), (g, h)


@pytest.mark.parametrize("L,ell", [(1, 2), (2, 4), (2, 6), (3, 4), (4, 5)])
def test_gadget_base(orc, L, ell):
    P = orc.make_params(64, 8, 1, 1, L)
    q, _ = orc.modulus_info(P)
    w = orc.gadget_bits(P, ell)
    assert w == -(-(q - 1).bit_length() // ell)  # ceil(ceil(log2 q) / ell); q is odd
    assert (1 << (w * ell)) >= q > (1 << (w * (ell - 1)))


def client(P, seed, count):
    s = synth.ternary_secret(seed, P.n)
    a = synth.uniform_residues(seed, synth.STREAM_A, count, P.n, P.qs)
    e = synth.gaussian_error(seed, count * P.n).reshape(count, P.n)
    return s, a, e


def tau_plain(m, p, g):
    """tau_g on a plaintext polynomial over Z_p, in pure Python."""
    n = len(m)
    out = [0] * n
    for t in range(n):
        e = t * g % (2 * n)
        if e < n:
            out[e] = int(m[t]) % p
        else:
            out[e - n] = (-int(m[t])) % p
    return out


def ks_noise_bound(P, ell, w):
    """Worst case of one key switch: sum_k d_k e_k with digits < 2^w, |e_k| <= 19."""
    return ell * P.n * ((1 << w) - 1) * ERR_BOUND


@pytest.mark.parametrize("L,ell", [(2, 4), (2, 6), (3, 5)])
def test_subs_decrypts_to_substituted_message(orc, L, ell):
    P = orc.make_params(512, 10, 1, 1, L)
    n, p = P.n, 1 << P.log2p
    s, a, e = client(P, 11 + L, 1)
    m = np.random.default_rng(ell).integers(0, p, size=n).astype(np.uint32)
    ct = orc.bfv_encrypt(P, s, a[0], e[0], m)
    w = orc.gadget_bits(P, ell)
    for g in (n + 1, n // 2 + 1, 2 * n - 1):
        ka = synth.uniform_residues(g, synth.STREAM_KEY_A, ell, n, P.qs)
        ke = synth.gaussian_error(g, ell * n, stream=synth.STREAM_KEY_ERROR).reshape(ell, n)
        ksk = orc.ksk_gen(P, s, g, ell, ka, ke)
        out = orc.subs(P, ct, g, ksk, ell)
        want = np.array(tau_plain(m, p, g), dtype=np.uint32)
        assert np.array_equal(orc.bfv_decrypt(P, s, out), want), g
        noise = np.abs(orc.bfv_noise(P, s, out, want)).max()
        assert noise <= ERR_BOUND + ks_noise_bound(P, ell, w)


def expansion_noise_bound(P, levels, ell, w):
    """Fresh error plus level j's key-switch noise doubled by each later level."""
    return ERR_BOUND + ((1 << levels) - 1) * ks_noise_bound(P, ell, w)


@pytest.mark.parametrize("L,levels,ell", [(2, 3, 4), (2, 4, 6), (3, 4, 4)])
def test_expansion_recovers_every_coefficient(orc, L, levels, ell):
    P = orc.make_params(256, 10, 1, 1, L)
    n, p, C = P.n, 1 << P.log2p, 1 << levels
    s, a, e = client(P, 20 + levels, 1)
    keys = orc.expansion_keys(P, s, levels, ell, seed=30 + L)
    w = orc.gadget_bits(P, ell)
    m = np.random.default_rng(levels).integers(0, p, size=n).astype(np.uint32)
    ct = orc.bfv_encrypt(P, s, a[0], e[0], m)
    out = orc.expand(P, ct, levels, ell, keys, C)
    worst = 0
    for k in range(C):
        # ciphertext k holds the coefficients of m at k + 2^levels u, moved to 2^levels u
        want = np.zeros(n, dtype=np.uint32)
        want[0::C] = m[k::C]
        assert np.array_equal(orc.bfv_decrypt(P, s, out[k]), want), k
        worst = max(worst, int(np.abs(orc.bfv_noise(P, s, out[k], want)).max()))
    assert worst <= expansion_noise_bound(P, levels, ell, w)
    # fewer outputs are a prefix of the full expansion
    assert np.array_equal(orc.expand(P, ct, levels, ell, keys, C - 3), out[:C - 3])


def decrypt_expanded_answer(orc, n, log2p, D1, D2, L, ell, seed):
    P = orc.make_params(n, log2p, D1, D2, L)
    levels = (D1 - 1).bit_length()
    raw = synth.raw_db(seed, synth.raw_db_bytes(n, log2p, D1, D2))
    idx = int(synth.query_indices(seed, 1, D1, D2)[0])
    i_star = idx // D2
    s, a, e = client(P, seed, 1)
    keys = orc.expansion_keys(P, s, levels, ell, seed=seed)
    packed = orc.encrypt_packed_query(P, s, a[0], e[0], i_star)
    Q = orc.expand(P, packed, levels, ell, keys, D1)[None]  # [1][D1][2][L][n]
    for i in range(D1):  # each expanded ciphertext encrypts [i == i*]
        want = np.zeros(n, dtype=np.uint32)
        want[0] = 1 if i == i_star else 0
        assert np.array_equal(orc.bfv_decrypt(P, s, Q[0, i]), want), i
    R = orc.answer(P, raw, Q)
    for c in range(D2):
        want = orc.unpack_poly(raw, log2p, n, i_star * D2 + c)
        assert np.array_equal(orc.bfv_decrypt(P, s, R[0, c]), want), c


def test_expanded_query_answers_tiny_config(orc):
    decrypt_expanded_answer(orc, 2048, 12, 16, 16, L=2, ell=6, seed=1)


def test_expanded_query_answers_three_primes(orc):
    decrypt_expanded_answer(orc, 2048, 16, 32, 4, L=3, ell=4, seed=2)


def tau(a, g, q):
    """a(X) -> a(X^g) in Z_q[X]/(X^n + 1): coefficient t moves to t*g mod 2n, negated
    past n (restated here in pure Python)."""
    n = len(a)
    out = [0] * n
    for t in range(n):
        e = (t * g) % (2 * n)
        if e < n:
            out[e] = (out[e] + int(a[t])) % q
        else:
            out[e - n] = (out[e - n] - int(a[t])) % q
    return out


def negacyclic(a, b, q):
    n = len(a)
    out = [0] * n
    for i in range(n):
        ai = int(a[i])
        if ai:
            for j in range(n):
                k = i + j
                if k < n:
                    out[k] += ai * int(b[j])
                else:
                    out[k - n] -= ai * int(b[j])
    return [v % q for v in out]


@pytest.mark.parametrize("L,ell,g", [(1, 3, 65), (2, 4, 33), (3, 5, 17)])
def test_noiseless_subs_has_the_substituted_phase(orc, L, ell, g):
    """With zero masks and zero errors the key-switching key adds no noise, so
    Subs(ct, g) must have exactly the phase tau_g(c_a * s + c_b): tau_g is a ring
    homomorphism.  An exact identity, whatever the key's sign convention."""
    P = orc.make_params(64, 10, 1, 1, L)
    n = P.n
    rng = np.random.default_rng(L * 100 + g)
    s = synth.ternary_secret(7 + L, n)
    ksk = orc.ksk_gen(P, s, g, ell, np.zeros((ell, L, n), dtype=np.uint32), np.zeros((ell, n), dtype=np.int8))
    ct = np.stack([np.stack([rng.integers(0, q, size=n, dtype=np.uint64).astype(np.uint32) for q in P.qs])
                   for _ in range(2)])
    out = orc.subs(P, ct, g, ksk, ell)
    for j, q in enumerate(P.qs):
        s_q = [int(v) % q for v in s]
        phase_in = [(x + y) % q for x, y in zip(negacyclic(ct[0, j], s_q, q), ct[1, j])]
        phase_out = [(x + y) % q for x, y in zip(negacyclic(out[0, j], s_q, q), out[1, j])]
        assert phase_out == tau(phase_in, g, q), j


# --- the two digit orders of the key switch (App. D.3) ----------------------
#
# The oracle's expansion takes the gadget digits of the level input's a-part and
# moves them with the ciphertext (the digits lie in (-t, t)); the textbook key switch
# decomposes the substituted a-part tau_g(a X^-C) instead (digits in [0, t)).  The
# output ciphertexts differ, but both digit sets recombine to tau_g(a X^-C), so with
# error-free keys both have exactly the phase tau_g((a s + b) X^-C).

def crt_lift(residues, qs):
    """x in [0, prod q) with x = r_j mod q_j, in pure Python."""
    Q = 1
    for q in qs:
        Q *= q
    x = 0
    for r, q in zip(residues, qs):
        Qj = Q // q
        x += int(r) * Qj * pow(Qj, -1, q)
    return x % Q


def shift_div(a, C, q):
    """a X^-C in Z_q[X]/(X^n + 1), pure Python."""
    n = len(a)
    out = [0] * n
    for t in range(n):
        if t >= C:
            out[t - C] = int(a[t]) % q
        else:
            out[t + n - C] = (-int(a[t])) % q
    return out


def all_galois(n):
    return [n // (1 << j) + 1 for j in range(n.bit_length() - 1)]


@pytest.mark.parametrize("L,ell", [(1, 3), (2, 4), (3, 5)])
def test_moved_digits_recombine_to_the_substituted_a_part(orc, L, ell):
    """sum_k t^k tau_g(d_k X^-C) = tau_g(a X^-C) mod every q_j, for the digits d_k of
    a's CRT lift, every expansion Galois element g and both shifts of its level;
    the moved digits lie in (-t, t).  Pure Python over the integers."""
    P = orc.make_params(32, 6, 1, 1, L)
    n, qs = P.n, P.qs
    w = orc.gadget_bits(P, ell)
    a = synth.uniform_residues(40 + L, synth.STREAM_UNIFORM, 1, n, qs).reshape(L, n)
    x = [crt_lift([a[j][t] for j in range(L)], qs) for t in range(n)]
    digits = [[(xt >> (w * k)) & ((1 << w) - 1) for xt in x] for k in range(ell)]
    for lev, g in enumerate(all_galois(n)):
        for C in (0, 1 << lev):
            for j, q in enumerate(qs):
                want = tau([int(v) for v in a[j]], g, q) if C == 0 else tau(shift_div(a[j], C, q), g, q)
                acc = [0] * n
                for k in range(ell):
                    # move the integer digit with its sign: X^-C then tau_g, kept signed
                    moved = [0] * n
                    for t in range(n):
                        v, e0 = digits[k][t], t - C
                        if e0 < 0:
                            v, e0 = -v, e0 + n
                        e1 = e0 * g % (2 * n)
                        if e1 >= n:
                            v, e1 = -v, e1 - n
                        moved[e1] = v
                    assert all(-(1 << w) < v < (1 << w) for v in moved)
                    acc = [u + (v << (w * k)) for u, v in zip(acc, moved)]
                assert [u % q for u in acc] == want, (g, C, j)


def phase(orc_, ct, s, q, j):
    s_q = [int(v) % q for v in s]
    return [(x + y) % q for x, y in zip(negacyclic(ct[0, j], s_q, q), ct[1, j])]


@pytest.mark.parametrize("L,ell", [(1, 3), (2, 4), (3, 5)])
def test_both_digit_orders_have_the_substituted_phase(orc, L, ell):
    """With error-free keys (uniform masks, zero errors) the key switch adds no noise:
    Subs(ct X^-C, g) in either digit order has exactly the phase tau_g(phi X^-C),
    phi = c_a s + c_b, for every expansion Galois element and both shifts of its
    level.  The two ciphertexts themselves differ (their a-parts are different key
    combinations), so the choice of order fixes the output bits."""
    P = orc.make_params(32, 6, 1, 1, L)
    n = P.n
    s = synth.ternary_secret(50 + L, n)
    rng = np.random.default_rng(60 + L)
    ct = np.stack([np.stack([rng.integers(0, q, size=n, dtype=np.uint64).astype(np.uint32) for q in P.qs])
                   for _ in range(2)])
    differ = 0
    for lev, g in enumerate(all_galois(n)):
        ka = synth.uniform_residues(g, synth.STREAM_KEY_A, ell, n, P.qs)
        ksk = orc.ksk_gen(P, s, g, ell, ka, np.zeros((ell, n), dtype=np.int8))
        for C in (0, 1 << lev):
            moved = orc.subs_shift(P, ct, C, g, ksk, ell, textbook=False)
            text = orc.subs_shift(P, ct, C, g, ksk, ell, textbook=True)
            differ += int(not np.array_equal(moved, text))
            for j, q in enumerate(P.qs):
                want = tau(shift_div(phase(orc, ct, s, q, j), C, q), g, q)
                assert phase(orc, moved, s, q, j) == want, (g, C, j)
                assert phase(orc, text, s, q, j) == want, (g, C, j)
    assert differ > 0


@pytest.mark.parametrize("L,levels,ell", [(1, 3, 3), (2, 4, 4), (3, 3, 5)])
def test_expansion_digit_orders_agree_on_every_phase(orc, L, levels, ell):
    """Whole expansions in both orders with error-free keys: every output has the same
    phase; with noisy keys both decrypt to the same coefficients within the bound."""
    P = orc.make_params(64, 8, 1, 1, L)
    n, p, C = P.n, 1 << P.log2p, 1 << levels
    s, a, e = client(P, 70 + L, 1)
    m = np.random.default_rng(L).integers(0, p, size=n).astype(np.uint32)
    ct = orc.bfv_encrypt(P, s, a[0], e[0], m)
    ka = np.stack([synth.uniform_residues(80 + lev, synth.STREAM_KEY_A, ell, n, P.qs) for lev in range(levels)])
    clean = np.stack([orc.ksk_gen(P, s, g, ell, ka[lev], np.zeros((ell, n), dtype=np.int8))
                      for lev, g in enumerate(orc.expansion_galois(n, levels))])
    out_m = orc.expand(P, ct, levels, ell, clean, C)
    out_t = orc.expand_textbook(P, ct, levels, ell, clean, C)
    for k in range(C):
        for j, q in enumerate(P.qs):
            assert phase(orc, out_m[k], s, q, j) == phase(orc, out_t[k], s, q, j), (k, j)
    keys = orc.expansion_keys(P, s, levels, ell, seed=90 + L)
    w = orc.gadget_bits(P, ell)
    out_t = orc.expand_textbook(P, ct, levels, ell, keys, C)
    for k in range(C):
        want = np.zeros(n, dtype=np.uint32)
        want[0::C] = m[k::C]
        assert np.array_equal(orc.bfv_decrypt(P, s, out_t[k]), want), k
        assert np.abs(orc.bfv_noise(P, s, out_t[k], want)).max() <= expansion_noise_bound(P, levels, ell, w)
