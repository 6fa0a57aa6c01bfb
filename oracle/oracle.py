"""ctypes binding of the C oracle (``pir_oracle.c``) plus numpy conveniences.

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the
CPU-baseline leg of the benchmark, never by the product path.

Parity: pinned (see ``pir_oracle.c`` header); every function here is a thin
marshalling wrapper, the arithmetic is in C.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

ORC_MAX_L = 4


class OrcParams(C.Structure):
    _fields_ = [
        ("n", C.c_uint32),
        ("L", C.c_uint32),
        ("log2p", C.c_uint32),
        ("D1", C.c_uint32),
        ("D2", C.c_uint32),
        ("q", C.c_uint64 * ORC_MAX_L),
        ("psi", C.c_uint64 * ORC_MAX_L),
    ]

    @property
    def qs(self):
        return [int(self.q[j]) for j in range(self.L)]

    @property
    def psis(self):
        return [int(self.psi[j]) for j in range(self.L)]


_lib = None
U32P = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")
U64P = np.ctypeslib.ndpointer(dtype=np.uint64, flags="C_CONTIGUOUS")
I64P = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
I8P = np.ctypeslib.ndpointer(dtype=np.int8, flags="C_CONTIGUOUS")
U8P = np.ctypeslib.ndpointer(dtype=np.uint8, flags="C_CONTIGUOUS")
PP = C.POINTER(OrcParams)


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        sig = {
            "orc_is_prime": (C.c_int, [C.c_uint64]),
            "orc_powmod": (C.c_uint64, [C.c_uint64, C.c_uint64, C.c_uint64]),
            "orc_select_primes": (C.c_int, [C.c_uint32, C.c_uint32, C.c_uint32, U64P]),
            "orc_find_psi": (C.c_uint64, [C.c_uint64, C.c_uint32]),
            "orc_make_params": (C.c_int, [C.c_uint32] * 5 + [PP]),
            "orc_ntt_definition": (None, [U32P, U32P, C.c_uint32, C.c_uint64, C.c_uint64]),
            "orc_intt_definition": (None, [U32P, U32P, C.c_uint32, C.c_uint64, C.c_uint64]),
            "orc_ntt_fwd": (None, [U32P, C.c_uint32, C.c_uint64, C.c_uint64]),
            "orc_ntt_inv": (None, [U32P, C.c_uint32, C.c_uint64, C.c_uint64]),
            "orc_ntt_fwd_rns_mt": (None, [PP, U32P, C.c_uint64, C.c_int]),
            "orc_ntt_inv_rns_mt": (None, [PP, U32P, C.c_uint64, C.c_int]),
            "orc_negacyclic_schoolbook": (None, [U32P, U32P, U32P, C.c_uint32, C.c_uint64]),
            "orc_unpack_poly": (None, [U8P, C.c_uint32, C.c_uint32, C.c_uint64, U32P]),
            "orc_encode_polys": (None, [PP, U8P, U64P, C.c_uint64, U32P, C.c_int]),
            "orc_answer_encoded": (None, [PP, U32P, C.c_uint32, U32P, C.c_uint32, U32P, C.c_int]),
            "orc_answer": (C.c_int, [PP, U8P, U32P, C.c_uint32, U32P, C.c_uint32, U32P, C.c_int]),
            "orc_answer_schoolbook": (None, [PP, U8P, U32P, C.c_uint32, U32P]),
            "orc_modulus_info": (None, [PP, U64P, U64P]),
            "orc_bfv_encrypt": (None, [PP, I8P, U32P, I8P, U32P, U32P]),
            "orc_bfv_decrypt": (None, [PP, I8P, U32P, U32P]),
            "orc_bfv_noise": (None, [PP, I8P, U32P, U32P, I64P]),
            "orc_bfv_phase": (None, [PP, I8P, U32P, U64P]),
            "orc_freivalds": (C.c_longlong, [PP, U8P, U32P, C.c_uint32, U32P, U32P, C.c_int]),
            "orc_modswitch": (None, [PP, U32P, C.c_uint64, U32P]),
            "orc_bfv_phase_q0": (None, [PP, I8P, U32P, U64P]),
            "orc_bfv_decrypt_q0": (None, [PP, I8P, U32P, U32P]),
            "orc_lwe_gemm": (None, [I8P, C.c_uint32, C.c_uint32, U32P, C.c_uint32, U32P]),
            "orc_rgsw_encrypt": (None, [PP, I8P, U32P, C.c_uint32, U32P, I8P, U32P]),
            "orc_external_product": (None, [PP, U32P, C.c_uint32, U32P, U32P]),
            "orc_fold": (None, [PP, U32P, C.c_uint32, U32P, C.c_uint32, U32P]),
            "orc_automorphism": (None, [U32P, U32P, C.c_uint32, C.c_uint64, C.c_uint32]),
            "orc_gadget_bits": (C.c_uint32, [PP, C.c_uint32]),
            "orc_ksk_gen": (None, [PP, I8P, C.c_uint32, C.c_uint32, U32P, I8P, U32P]),
            "orc_subs": (None, [PP, U32P, C.c_uint32, U32P, C.c_uint32, U32P]),
            "orc_expand": (None, [PP, U32P, C.c_uint32, C.c_uint32, U32P, C.c_uint32, U32P]),
            "orc_subs_textbook": (None, [PP, U32P, C.c_uint32, C.c_uint32, U32P, C.c_uint32, U32P]),
            "orc_subs_moved": (None, [PP, U32P, C.c_uint32, C.c_uint32, U32P, C.c_uint32, U32P]),
            "orc_expand_textbook": (None, [PP, U32P, C.c_uint32, C.c_uint32, U32P, C.c_uint32, U32P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def default_threads() -> int:
    return max(1, len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count() or 1)


def _u32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.uint32)


# --- parameters ------------------------------------------------------------

def is_prime(x: int) -> bool:
    return bool(lib().orc_is_prime(x))


def select_primes(n: int, log2p: int, L: int = 2):
    out = np.zeros(ORC_MAX_L, dtype=np.uint64)
    if lib().orc_select_primes(n, log2p, L, out) != 0:
        raise ValueError("no primes")
    return [int(v) for v in out[:L]]


def find_psi(q: int, n: int) -> int:
    return int(lib().orc_find_psi(q, n))


def make_params(n: int, log2p: int, D1: int, D2: int, L: int = 2) -> OrcParams:
    P = OrcParams()
    if lib().orc_make_params(n, log2p, D1, D2, L, C.byref(P)) != 0:
        raise ValueError("bad parameters")
    return P


def modulus_info(P: OrcParams):
    qv = np.zeros(2, dtype=np.uint64)
    dv = np.zeros(2, dtype=np.uint64)
    lib().orc_modulus_info(C.byref(P), qv, dv)
    return int(qv[0]) | (int(qv[1]) << 64), int(dv[0]) | (int(dv[1]) << 64)


# --- NTT -------------------------------------------------------------------

def ntt_definition(a, q: int, psi: int) -> np.ndarray:
    a = _u32(a)
    out = np.empty_like(a)
    lib().orc_ntt_definition(a, out, a.size, q, psi)
    return out


def intt_definition(a, q: int, psi: int) -> np.ndarray:
    a = _u32(a)
    out = np.empty_like(a)
    lib().orc_intt_definition(a, out, a.size, q, psi)
    return out


def ntt_fwd(a, q: int, psi: int) -> np.ndarray:
    a = _u32(a).copy()
    lib().orc_ntt_fwd(a, a.size, q, psi)
    return a


def ntt_inv(a, q: int, psi: int) -> np.ndarray:
    a = _u32(a).copy()
    lib().orc_ntt_inv(a, a.size, q, psi)
    return a


def ntt_fwd_rns(P: OrcParams, polys, nthreads: int | None = None) -> np.ndarray:
    """polys [..., L, n] -> forward NTT of every row (row j under q_j)."""
    a = _u32(polys).copy()
    count = a.size // (P.L * P.n)
    lib().orc_ntt_fwd_rns_mt(C.byref(P), a.reshape(-1), count, nthreads or default_threads())
    return a


def ntt_inv_rns(P: OrcParams, polys, nthreads: int | None = None) -> np.ndarray:
    a = _u32(polys).copy()
    count = a.size // (P.L * P.n)
    lib().orc_ntt_inv_rns_mt(C.byref(P), a.reshape(-1), count, nthreads or default_threads())
    return a


def negacyclic_schoolbook(a, b, q: int) -> np.ndarray:
    a = _u32(a)
    b = _u32(b)
    out = np.empty_like(a)
    lib().orc_negacyclic_schoolbook(a, b, out, a.size, q)
    return out


# --- DB --------------------------------------------------------------------

def unpack_poly(raw, log2p: int, n: int, poly: int) -> np.ndarray:
    out = np.empty(n, dtype=np.uint32)
    lib().orc_unpack_poly(np.ascontiguousarray(raw, dtype=np.uint8), log2p, n, poly, out)
    return out


def encode_polys(P: OrcParams, raw, poly_ids, nthreads: int | None = None) -> np.ndarray:
    """NTT form of DB polys ``poly_ids`` (= i*D2 + c): [count][L][n]."""
    ids = np.ascontiguousarray(poly_ids, dtype=np.uint64)
    out = np.empty((ids.size, P.L, P.n), dtype=np.uint32)
    lib().orc_encode_polys(C.byref(P), np.ascontiguousarray(raw, dtype=np.uint8), ids, ids.size,
                           out.reshape(-1), nthreads or default_threads())
    return out


# --- answer ----------------------------------------------------------------

def answer(P: OrcParams, raw, queries, cols=None, nthreads: int | None = None) -> np.ndarray:
    """Responses [B][ncols][2][L][n] for queries [B][D1][2][L][n] (coefficient form)."""
    q = _u32(queries)
    B = q.size // (P.D1 * 2 * P.L * P.n)
    cols = np.arange(P.D2, dtype=np.uint32) if cols is None else _u32(cols)
    out = np.empty((B, cols.size, 2, P.L, P.n), dtype=np.uint32)
    rc = lib().orc_answer(C.byref(P), np.ascontiguousarray(raw, dtype=np.uint8), q.reshape(-1), B, cols, cols.size,
                          out.reshape(-1), nthreads or default_threads())
    if rc != 0:
        raise MemoryError("oracle answer: out of memory")
    return out


def answer_encoded(P: OrcParams, dbhat_cols, qhat, nthreads: int | None = None) -> np.ndarray:
    """dbhat_cols [ncols][D1][L][n], qhat [B][D1][2][L][n] (NTT form) -> responses
    [B][ncols][2][L][n] (coefficient form)."""
    d = _u32(dbhat_cols)
    qh = _u32(qhat)
    ncols = d.size // (P.D1 * P.L * P.n)
    B = qh.size // (P.D1 * 2 * P.L * P.n)
    out = np.empty((B, ncols, 2, P.L, P.n), dtype=np.uint32)
    lib().orc_answer_encoded(C.byref(P), d.reshape(-1), ncols, qh.reshape(-1), B, out.reshape(-1),
                             nthreads or default_threads())
    return out


def answer_schoolbook(P: OrcParams, raw, queries) -> np.ndarray:
    q = _u32(queries)
    B = q.size // (P.D1 * 2 * P.L * P.n)
    out = np.empty((B, P.D2, 2, P.L, P.n), dtype=np.uint32)
    lib().orc_answer_schoolbook(C.byref(P), np.ascontiguousarray(raw, dtype=np.uint8), q.reshape(-1), B,
                                out.reshape(-1))
    return out


def freivalds(P: OrcParams, raw, queries, responses, r, nthreads: int | None = None) -> int:
    q = _u32(queries)
    B = q.size // (P.D1 * 2 * P.L * P.n)
    bad = lib().orc_freivalds(C.byref(P), np.ascontiguousarray(raw, dtype=np.uint8), q.reshape(-1), B,
                              _u32(responses).reshape(-1), _u32(r).reshape(-1), nthreads or default_threads())
    if bad < 0:
        raise MemoryError("oracle freivalds: out of memory")
    return int(bad)


# --- toy BFV client --------------------------------------------------------

def bfv_encrypt(P: OrcParams, s, a, e, m) -> np.ndarray:
    ct = np.empty((2, P.L, P.n), dtype=np.uint32)
    lib().orc_bfv_encrypt(C.byref(P), np.ascontiguousarray(s, dtype=np.int8), _u32(a).reshape(-1),
                          np.ascontiguousarray(e, dtype=np.int8), _u32(m), ct.reshape(-1))
    return ct


def bfv_decrypt(P: OrcParams, s, ct) -> np.ndarray:
    m = np.empty(P.n, dtype=np.uint32)
    lib().orc_bfv_decrypt(C.byref(P), np.ascontiguousarray(s, dtype=np.int8), _u32(ct).reshape(-1), m)
    return m


def bfv_noise(P: OrcParams, s, ct, m) -> np.ndarray:
    out = np.empty(P.n, dtype=np.int64)
    lib().orc_bfv_noise(C.byref(P), np.ascontiguousarray(s, dtype=np.int8), _u32(ct).reshape(-1), _u32(m), out)
    return out


def bfv_phase(P: OrcParams, s, ct) -> list:
    """Phase a*s + b mod q per coefficient, as Python ints in [0, q)."""
    out = np.empty(2 * P.n, dtype=np.uint64)
    lib().orc_bfv_phase(C.byref(P), np.ascontiguousarray(s, dtype=np.int8), _u32(ct).reshape(-1), out)
    return [int(out[2 * t]) | (int(out[2 * t + 1]) << 64) for t in range(P.n)]


def modswitch(P: OrcParams, polys) -> np.ndarray:
    """Modulus switching to q_0: polys [..., L, n] coefficient form -> [..., n],
    each coefficient round(x q_0 / q) mod q_0."""
    a = _u32(polys)
    lead = a.shape[:-2]
    assert a.shape[-2:] == (P.L, P.n)
    count = int(np.prod(lead)) if lead else 1
    out = np.empty(lead + (P.n,), dtype=np.uint32)
    lib().orc_modswitch(C.byref(P), a.reshape(-1), count, out.reshape(-1))
    return out


def bfv_phase_q0(P: OrcParams, s, ct) -> np.ndarray:
    """Phase a*s + b mod q_0 of a switched ciphertext [2][n]."""
    out = np.empty(P.n, dtype=np.uint64)
    lib().orc_bfv_phase_q0(C.byref(P), np.ascontiguousarray(s, dtype=np.int8), _u32(ct).reshape(-1), out)
    return out


def bfv_decrypt_q0(P: OrcParams, s, ct) -> np.ndarray:
    """Decryption of a switched ciphertext [2][n] over q_0."""
    m = np.empty(P.n, dtype=np.uint32)
    lib().orc_bfv_decrypt_q0(C.byref(P), np.ascontiguousarray(s, dtype=np.int8), _u32(ct).reshape(-1), m)
    return m


# --- RGSW external products (remaining dimensions) --------------------------

def rgsw_encrypt(P: OrcParams, s, mu, ell: int, a, e) -> np.ndarray:
    """RGSW(mu): [2 ell][2][L][n]; mu [n] small non-negative, a [2 ell][L][n], e [2 ell][n]."""
    out = np.empty((2 * ell, 2, P.L, P.n), dtype=np.uint32)
    lib().orc_rgsw_encrypt(C.byref(P), np.ascontiguousarray(s, dtype=np.int8), _u32(mu), ell, _u32(a).reshape(-1),
                           np.ascontiguousarray(e, dtype=np.int8).reshape(-1), out.reshape(-1))
    return out


def rgsw_bits(P: OrcParams, s, bits, ell: int, seed: int) -> np.ndarray:
    """RGSW encryptions of the constant polynomials bits[l] (one per folding level),
    [levels][2 ell][2][L][n], from seeded draws (masks STREAM_KEY_A, errors STREAM_KEY_ERROR)."""
    import synth
    out = np.empty((len(bits), 2 * ell, 2, P.L, P.n), dtype=np.uint32)
    for l, bit in enumerate(bits):
        mu = np.zeros(P.n, dtype=np.uint32)
        mu[0] = int(bit)
        a = synth.uniform_residues(seed, synth.STREAM_KEY_A, 2 * ell, P.n, P.qs, start=(1000 + l) * 2 * ell)
        e = synth.gaussian_error(seed, 2 * ell * P.n, start=(1000 + l) * 2 * ell * P.n,
                                 stream=synth.STREAM_KEY_ERROR).reshape(2 * ell, P.n)
        out[l] = rgsw_encrypt(P, s, mu, ell, a, e)
    return out


def external_product(P: OrcParams, rgsw, ell: int, ct) -> np.ndarray:
    out = np.empty((2, P.L, P.n), dtype=np.uint32)
    lib().orc_external_product(C.byref(P), _u32(rgsw).reshape(-1), ell, _u32(ct).reshape(-1), out.reshape(-1))
    return out


def fold(P: OrcParams, cts, levels: int, rgsw, ell: int) -> np.ndarray:
    """Fold 2^levels ciphertexts [2^levels][2][L][n] into one with RGSW selection bits."""
    out = np.empty((2, P.L, P.n), dtype=np.uint32)
    lib().orc_fold(C.byref(P), _u32(cts).reshape(-1), levels, _u32(rgsw).reshape(-1), ell, out.reshape(-1))
    return out


# --- scalar-HE (LWE) DB GEMM ------------------------------------------------

def lwe_gemm(A, Q) -> np.ndarray:
    """out[b][i] = sum_j A[i][j] Q[b][j] mod 2^32; A [D1][D0] int8, Q [B][D0] uint32."""
    A = np.ascontiguousarray(A, dtype=np.int8)
    Q = _u32(Q)
    D1, D0 = A.shape
    B = Q.shape[0]
    assert Q.shape == (B, D0)
    out = np.empty((B, D1), dtype=np.uint32)
    lib().orc_lwe_gemm(A.reshape(-1), D1, D0, Q.reshape(-1), B, out.reshape(-1))
    return out


# --- query expansion -------------------------------------------------------

def automorphism(a, q: int, g: int) -> np.ndarray:
    """a(X) -> a(X^g) mod (X^n + 1, q), g odd."""
    a = _u32(a)
    out = np.empty_like(a)
    lib().orc_automorphism(a, out, a.size, q, g)
    return out


def gadget_bits(P: OrcParams, ell: int) -> int:
    """w with gadget base t = 2^w = 2^ceil(log2 q / ell)."""
    return int(lib().orc_gadget_bits(C.byref(P), ell))


def expansion_galois(n: int, levels: int):
    """The substitution exponents g_j = n / 2^j + 1 of the expansion levels."""
    return [n // (1 << j) + 1 for j in range(levels)]


def ksk_gen(P: OrcParams, s, g: int, ell: int, a, e) -> np.ndarray:
    """Key-switching key tau_g(s) -> s: [ell][2][L][n].  a [ell][L][n], e [ell][n]."""
    out = np.empty((ell, 2, P.L, P.n), dtype=np.uint32)
    lib().orc_ksk_gen(C.byref(P), np.ascontiguousarray(s, dtype=np.int8), g, ell, _u32(a).reshape(-1),
                      np.ascontiguousarray(e, dtype=np.int8).reshape(-1), out.reshape(-1))
    return out


def expansion_keys(P: OrcParams, s, levels: int, ell: int, seed: int) -> np.ndarray:
    """All expansion keys [levels][ell][2][L][n] from seeded client draws (masks from
    STREAM_KEY_A, errors from STREAM_KEY_ERROR)."""
    import synth
    keys = np.empty((levels, ell, 2, P.L, P.n), dtype=np.uint32)
    for j, g in enumerate(expansion_galois(P.n, levels)):
        a = synth.uniform_residues(seed, synth.STREAM_KEY_A, ell, P.n, P.qs, start=j * ell)
        e = synth.gaussian_error(seed, ell * P.n, start=j * ell * P.n, stream=synth.STREAM_KEY_ERROR).reshape(ell, P.n)
        keys[j] = ksk_gen(P, s, g, ell, a, e)
    return keys


def subs(P: OrcParams, ct, g: int, ksk, ell: int) -> np.ndarray:
    out = np.empty((2, P.L, P.n), dtype=np.uint32)
    lib().orc_subs(C.byref(P), _u32(ct).reshape(-1), g, _u32(ksk).reshape(-1), ell, out.reshape(-1))
    return out


def subs_shift(P: OrcParams, ct, shift: int, g: int, ksk, ell: int, textbook: bool) -> np.ndarray:
    """Subs(ct X^-shift, g).  textbook: gadget digits of the substituted a-part;
    otherwise the digits of ct's a-part moved along (the order expand uses)."""
    out = np.empty((2, P.L, P.n), dtype=np.uint32)
    f = lib().orc_subs_textbook if textbook else lib().orc_subs_moved
    f(C.byref(P), _u32(ct).reshape(-1), shift, g, _u32(ksk).reshape(-1), ell, out.reshape(-1))
    return out


def expand_textbook(P: OrcParams, ct, levels: int, ell: int, keys, count: int) -> np.ndarray:
    """expand() with every key switch in the textbook digit order."""
    out = np.empty((count, 2, P.L, P.n), dtype=np.uint32)
    lib().orc_expand_textbook(C.byref(P), _u32(ct).reshape(-1), levels, ell, _u32(keys).reshape(-1), count,
                              out.reshape(-1))
    return out


def expand(P: OrcParams, ct, levels: int, ell: int, keys, count: int) -> np.ndarray:
    """Expansion of one packed ciphertext [2][L][n] into count ciphertexts [count][2][L][n]."""
    out = np.empty((count, 2, P.L, P.n), dtype=np.uint32)
    lib().orc_expand(C.byref(P), _u32(ct).reshape(-1), levels, ell, _u32(keys).reshape(-1), count, out.reshape(-1))
    return out


def encrypt_packed_query(P: OrcParams, s, a, e, i_star: int) -> np.ndarray:
    """The packed first-dimension query: one ciphertext of m = X^i* (App. C.2),
    which expands to the D1 ciphertexts Enc([i == i*]).  a [L][n], e [n]."""
    m = np.zeros(P.n, dtype=np.uint32)
    m[i_star] = 1
    return bfv_encrypt(P, s, a, e, m)


def encrypt_query(P: OrcParams, s, a, e, i_star: int) -> np.ndarray:
    """One-hot first-dimension query: D1 ciphertexts, ct_i = Enc(m = [i == i*]) as a
    constant polynomial.  a [D1][L][n], e [D1][n] are the client's draws.
    Returns [D1][2][L][n]."""
    out = np.empty((P.D1, 2, P.L, P.n), dtype=np.uint32)
    m = np.zeros(P.n, dtype=np.uint32)
    for i in range(P.D1):
        m[0] = 1 if i == i_star else 0
        out[i] = bfv_encrypt(P, s, a[i], e[i], m)
    return out
