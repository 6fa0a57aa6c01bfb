"""Pins for the oracle's parameter generation (App. A.4, App. A.2) against an
independent primality library, the defining congruences and the paper's printed
identities."""
import numpy as np
import pytest

from golden.read import paper_values

CONFIG_RINGS = [(2048, 12), (4096, 16), (8192, 16)]


def test_is_prime_against_sympy(orc):
    sympy = pytest.importorskip("sympy")
    rng = np.random.default_rng(5)
    xs = list(range(0, 2000)) + [int(v) for v in rng.integers(2 ** 29, 2 ** 30, size=3000)]
    # strong pseudoprimes / Carmichael numbers that fool weaker tests
    xs += [561, 1105, 1729, 2047, 3215031751, 2152302898747, 3474749660383, 341550071728321,
           3825123056546413051, (1 << 61) - 1, (1 << 62) - 57, 18446744073709551557]
    for x in xs:
        assert orc.is_prime(x) == sympy.isprime(x), x


@pytest.mark.parametrize("n,log2p", CONFIG_RINGS + [(16, 4), (1024, 11)])
def test_primes_congruences_and_maximality(orc, n, log2p):
    sympy = pytest.importorskip("sympy")
    qs = orc.select_primes(n, log2p, 2)
    M = max(2 * n, 1 << log2p)
    assert qs[0] > qs[1]
    for q in qs:
        assert 2 ** 29 < q < 2 ** 30          # 30-bit primes
        assert sympy.isprime(q)
        assert q % (2 * n) == 1               # NTT-friendly (App. A.4)
        assert q % (1 << log2p) == 1          # q = 1 mod p (App. A.4)
    # the two largest such primes: nothing prime = 1 mod M above q1 except q0
    c = ((2 ** 30 - 2) // M) * M + 1
    while c > qs[1]:
        if c != qs[0]:
            assert not sympy.isprime(c), c
        c -= M


def test_config1_primes_are_1_mod_4096(orc):
    # the tiny configuration asks for two 30-bit primes = 1 mod 4096 (n = 2048, p = 2^12)
    for q in orc.select_primes(2048, 12, 2):
        assert q % 4096 == 1


@pytest.mark.parametrize("n,log2p", CONFIG_RINGS + [(8, 4), (64, 7)])
def test_psi_primitive_and_minimal(orc, n, log2p):
    for q in orc.select_primes(n, log2p, 2):
        psi = orc.find_psi(q, n)
        assert pow(psi, n, q) == q - 1        # psi^n = -1: a root of X^n + 1
        assert pow(psi, 2 * n, q) == 1        # hence order exactly 2n
        e = (q - 1) // (2 * n)
        for h in range(2, 200):
            cand = pow(h, e, q)
            if pow(cand, n, q) == q - 1:
                assert cand == psi            # the smallest such generator h
                break


@pytest.mark.parametrize("n,log2p", CONFIG_RINGS)
def test_delta_identity(orc, n, log2p):
    """App. A.4: Delta * p + 1 = q with Delta = floor(q/p)."""
    assert paper_values()["delta_identity"] == "Delta*p+1==q"
    P = orc.make_params(n, log2p, 4, 4, 2)
    q, delta = orc.modulus_info(P)
    assert q == P.qs[0] * P.qs[1]
    assert delta == q // (1 << log2p)
    assert delta * (1 << log2p) + 1 == q


def test_lazy_reduction_headroom():
    """Sec. 4.2: primes < 2^29 let a u64 accumulator take 32 products; the same bound
    for our 30-bit primes is 16 products."""
    pv = paper_values()
    k29 = (2 ** 64 - 1) // (2 ** 29 - 1) ** 2
    assert k29 >= pv["lazy_macs_prime_bits29"]
    k30 = (2 ** 64 - 1) // (2 ** 30 - 1) ** 2
    assert k30 == 16
