"""Pins for the oracle's modulus switching to q_0 (App. D.5, error analysis of RLWE
modulus switching): coefficients built as x = t Q' + r, whose rounded quotient is
t or t + 1 by construction; the identity when nothing is dropped; the rounding
error of a switched ciphertext against the bound of App. D.5 (each coefficient
rounded to within 1/2, so |E| <= (1 + ||s||_1) / 2 in the new units); and
decryption after switching, for fresh encryptions and for a whole PIR answer."""
import numpy as np
import pytest

import synth


def residues(P, xs):
    """[len(xs)] Python ints in [0, q) -> residues [L][len(xs)]."""
    return np.array([[x % q for x in xs] for q in P.qs], dtype=np.uint32)


@pytest.mark.parametrize("L", [2, 3, 4])
def test_switch_of_constructed_values(orc, L):
    n = 16
    P = orc.make_params(n, 8, 1, 1, L)
    q0 = P.qs[0]
    Qd = 1
    for qj in P.qs[1:]:
        Qd *= qj
    rng = np.random.default_rng(L)
    half = (Qd - 1) // 2
    cases = []  # (t, r, expected)
    for t in [0, 1, q0 - 1, int(rng.integers(0, q0))]:
        for r in [0, 1, half, half + 1, Qd - 1, int(rng.integers(0, 1 << 62)) % Qd]:
            cases.append((t, r, (t + (1 if r > half else 0)) % q0))
    while len(cases) % n:
        cases.append((0, 0, 0))
    xs = [t * Qd + r for t, r, _ in cases]
    assert max(xs) < q0 * Qd
    res = residues(P, xs)  # [L][count*n] -> polys [count][L][n]
    polys = res.reshape(L, -1, n).transpose(1, 0, 2).copy()
    got = orc.modswitch(P, polys).reshape(-1)
    assert [int(v) for v in got] == [e for _, _, e in cases]


def test_single_prime_is_identity(orc):
    P = orc.make_params(32, 8, 1, 1, 1)
    a = synth.uniform_residues(5, synth.STREAM_UNIFORM, 3, 32, P.qs).reshape(3, 1, 32)
    assert np.array_equal(orc.modswitch(P, a), a[:, 0])


def client(P, seed, count):
    s = synth.ternary_secret(seed, P.n)
    a = synth.uniform_residues(seed, synth.STREAM_A, count, P.n, P.qs)
    e = synth.gaussian_error(seed, count * P.n).reshape(count, P.n)
    return s, a, e


@pytest.mark.parametrize("n,log2p", [(2048, 12), (4096, 16)])
def test_rounding_error_bound_and_decryption(orc, n, log2p):
    P = orc.make_params(n, log2p, 1, 1, 2)
    q0 = P.qs[0]
    q, _ = orc.modulus_info(P)
    s, a, e = client(P, 40 + log2p, 2)
    s1 = int(np.abs(s.astype(np.int64)).sum())
    rng = np.random.default_rng(n)
    for k in range(2):
        m = rng.integers(0, 1 << log2p, size=n).astype(np.uint32)
        ct = orc.bfv_encrypt(P, s, a[k], e[k], m)
        sw = orc.modswitch(P, ct)  # [2][n] over q_0
        assert sw.shape == (2, n) and int(sw.max()) < q0
        assert np.array_equal(orc.bfv_decrypt_q0(P, s, sw), m)
        phi = orc.bfv_phase(P, s, ct)  # over q
        phi0 = orc.bfv_phase_q0(P, s, sw)  # over q_0
        worst = 0
        for t in range(n):
            # phi0 = (q_0 / q) phi + E  (mod q_0), so q phi0 - q_0 phi = q E (mod q q_0)
            d = (int(phi0[t]) * q - q0 * phi[t]) % (q * q0)
            d = d - q * q0 if d > (q * q0) // 2 else d
            worst = max(worst, abs(d))
        assert 2 * worst <= q * (1 + s1)
        # and far inside it, as the App. D.5 tail bound predicts for i.i.d. roundings
        assert worst < q * 8 * np.sqrt(n + 1)


def test_decryption_after_switching_the_answer(orc):
    """The tiny configuration: the switched answer still decrypts, column by column,
    to the DB row the query selects."""
    n, log2p, D1, D2 = 2048, 12, 16, 16
    P = orc.make_params(n, log2p, D1, D2, 2)
    raw = synth.raw_db(0, synth.raw_db_bytes(n, log2p, D1, D2))
    idx = int(synth.query_indices(1, 1, D1, D2)[0])
    i_star = idx // D2
    s, a, e = client(P, 1, D1)
    Q = orc.encrypt_query(P, s, a, e, i_star)[None]
    R = orc.answer(P, raw, Q)  # [1][D2][2][L][n]
    S = orc.modswitch(P, R)  # [1][D2][2][n]
    assert S.shape == (1, D2, 2, n)
    for c in range(D2):
        want = orc.unpack_poly(raw, log2p, n, i_star * D2 + c)
        assert np.array_equal(orc.bfv_decrypt_q0(P, s, S[0, c]), want), c


def test_planted_rounding_mistake_is_caught(orc):
    """A switch that truncates instead of rounding disagrees with the oracle on the
    constructed values above half way."""
    P = orc.make_params(16, 8, 1, 1, 2)
    q0, q1 = P.qs
    xs = [t * q1 + r for t in (5, 77) for r in ((q1 + 1) // 2, q1 - 1)] * 4
    polys = residues(P, xs).reshape(2, -1, 16).transpose(1, 0, 2).copy()
    got = [int(v) for v in orc.modswitch(P, polys).reshape(-1)]
    truncated = [(x // q1) % q0 for x in xs]
    assert all(g == t + 1 for g, t in zip(got, truncated))
