"""Seeded synthetic inputs for the PIR scan: database bytes, query indices and the
client's random draws (secret, uniform ``a``, Gaussian error).

This module holds none of the method's arithmetic.  It only draws numbers; the
oracle and the CUDA library both take what it returns as inputs.  It sits outside
both (a top-level module of its own): the oracle, the tests and the benchmark
import it, and it imports neither the oracle nor the library package.

Generator: SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014), used counter-style.  Value ``idx`` of stream
``stream`` under ``seed`` is ``mix(key(seed, stream) + (idx + 1) * GAMMA)``, so any
element can be regenerated on its own and a stream can be produced in chunks.

Workload shape (the paper's DBs are synthetic, 1-byte records, Sec. 6.1): the
raw DB is uniform random bytes; read as a little-endian stream of log2(p)-bit
coefficients this gives uniform plaintext coefficients in [0, p).
"""
from __future__ import annotations

import math

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_STREAM_MUL = 0xD1B54A32D192ED03

# stream identifiers
STREAM_DB = 1
STREAM_INDEX = 2
STREAM_SECRET = 3
STREAM_A = 4
STREAM_ERROR = 5
STREAM_FREIVALDS = 6
STREAM_UNIFORM = 7
STREAM_KEY_A = 8      # expansion-key masks
STREAM_KEY_ERROR = 9  # expansion-key errors

_MASK64 = (1 << 64) - 1


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def _mix_int(z: int) -> int:
    z &= _MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
    return z ^ (z >> 31)


def stream_key(seed: int, stream: int) -> int:
    return _mix_int(_mix_int(seed) ^ ((stream * _STREAM_MUL) & _MASK64))


def u64(seed: int, stream: int, start: int, count: int) -> np.ndarray:
    """Values ``start .. start+count-1`` of one counter-based stream (uint64)."""
    key = np.uint64(stream_key(seed, stream))
    with np.errstate(over="ignore"):
        idx = np.arange(start + 1, start + count + 1, dtype=np.uint64)
        return _mix(key + idx * GAMMA)


def raw_db(seed: int, nbytes: int, chunk_words: int = 1 << 24) -> np.ndarray:
    """Uniform random DB bytes (the raw, unencoded database)."""
    nwords = (nbytes + 7) // 8
    out = np.empty(nwords * 8, dtype=np.uint8)
    words = out.view(np.uint64)
    for s in range(0, nwords, chunk_words):
        c = min(chunk_words, nwords - s)
        words[s:s + c] = u64(seed, STREAM_DB, s, c)
    return out[:nbytes]


def query_indices(seed: int, B: int, D1: int, D2: int) -> np.ndarray:
    """B record indices uniform in [0, D1*D2); index -> (i*, c*) = divmod(idx, D2)."""
    v = u64(seed, STREAM_INDEX, 0, B)
    return (v % np.uint64(D1 * D2)).astype(np.int64)


def ternary_secret(seed: int, n: int, which: int = 0) -> np.ndarray:
    """Uniform ternary secret in {-1, 0, 1}^n (App. A.2), as int8."""
    v = u64(seed, STREAM_SECRET, which * n, n)
    return ((v % np.uint64(3)).astype(np.int16) - 1).astype(np.int8)


def uniform_residues(seed: int, stream: int, count: int, n: int, qs, start: int = 0) -> np.ndarray:
    """``count`` RNS polynomials [count][L][n] with residue j uniform mod qs[j]
    (uniform mod q_j per row is uniform mod q by CRT)."""
    L = len(qs)
    v = u64(seed, stream, start * L * n, count * L * n).reshape(count, L, n)
    out = np.empty((count, L, n), dtype=np.uint32)
    for j, q in enumerate(qs):
        out[:, j, :] = (v[:, j, :] % np.uint64(q)).astype(np.uint32)
    return out


def _gaussian_thresholds(sigma: float, bound: int) -> np.ndarray:
    xs = np.arange(-bound, bound + 1, dtype=np.float64)
    w = np.exp(-(xs ** 2) / (2.0 * sigma * sigma))
    cdf = np.cumsum(w) / w.sum()
    th = [min(int(c * 2.0 ** 64), _MASK64) for c in cdf]
    th[-1] = _MASK64
    return np.array(th, dtype=np.uint64)


def gaussian_error(seed: int, count: int, start: int = 0, sigma: float = 3.2, bound: int = 19,
                   stream: int = STREAM_ERROR) -> np.ndarray:
    """Discrete Gaussian draws with standard deviation sigma, clipped to |e| <= bound
    (App. A.1: sigma = 3.2, |e| < 6 sigma), by inversion of the cumulative table."""
    th = _gaussian_thresholds(sigma, bound)
    u = u64(seed, stream, start, count)
    k = np.searchsorted(th, u, side="right")
    k = np.minimum(k, 2 * bound)
    return (k.astype(np.int16) - bound).astype(np.int8)


def freivalds_vector(seed: int, qs, D2: int) -> np.ndarray:
    """Random r[j][c] in [0, q_j) for the Freivalds check."""
    L = len(qs)
    v = u64(seed, STREAM_FREIVALDS, 0, L * D2).reshape(L, D2)
    out = np.empty((L, D2), dtype=np.uint32)
    for j, q in enumerate(qs):
        out[j] = (v[j] % np.uint64(q)).astype(np.uint32)
    return out


def raw_db_bytes(n: int, log2p: int, D1: int, D2: int) -> int:
    bits = n * log2p * D1 * D2
    return bits // 8


def noise_sigma_estimate(n: int, log2p: int, D1: int, sigma: float = 3.2) -> float:
    """Standard deviation of one response coefficient's noise, sum over D1*n terms
    DB * e with DB uniform in [0, p) and e of std sigma (App. D style estimate)."""
    p = 2.0 ** log2p
    return math.sqrt(D1 * n) * math.sqrt((p - 1) * (2 * p - 1) / 6.0) * sigma


# --- the same streams generated by torch (device-side, for inputs too large for host) ---

def _i64(v: int) -> int:
    """The two's-complement int64 with the bits of the u64 value v."""
    v &= _MASK64
    return v - (1 << 64) if v >= (1 << 63) else v


def _srl(x, k: int):
    """Logical right shift of int64 tensors holding u64 bits."""
    return (x >> k) & ((1 << (64 - k)) - 1)


def _mix_torch(z):
    z = (z ^ _srl(z, 30)) * _i64(0xBF58476D1CE4E5B9)
    z = (z ^ _srl(z, 27)) * _i64(0x94D049BB133111EB)
    return z ^ _srl(z, 31)


def u64_torch(seed: int, stream: int, start: int, count: int, device=None):
    """u64(seed, stream, start, count) as an int64 tensor with the same bits."""
    import torch
    idx = torch.arange(start + 1, start + count + 1, dtype=torch.int64, device=device)
    z = _i64(stream_key(seed, stream)) + idx * _i64(int(GAMMA))
    return _mix_torch(z)


def uniform_residues_torch(seed: int, stream: int, count: int, n: int, qs, device=None, start: int = 0,
                           chunk: int = 1 << 24):
    """uniform_residues(...) generated on `device`: int32 tensor [count][L][n] holding
    the u32 residues (the same values as the numpy version)."""
    import torch
    L = len(qs)
    total = count * L * n
    out = torch.empty(total, dtype=torch.int32, device=device)
    j_of = None
    for s0 in range(0, total, chunk):
        c = min(chunk, total - s0)
        x = u64_torch(seed, stream, start * L * n + s0, c, device)
        pos = torch.arange(s0, s0 + c, dtype=torch.int64, device=device)
        j_of = (pos // n) % L
        hi, lo = _srl(x, 32), x & 0xFFFFFFFF
        res = torch.empty_like(x)
        for j, q in enumerate(qs):
            sel = j_of == j
            r = ((hi[sel] % q) * ((1 << 32) % q) + lo[sel]) % q
            res[sel] = r
        out[s0:s0 + c] = res.to(torch.int32)
    return out.view(count, L, n)


def raw_db_torch(seed: int, nbytes: int, device=None, chunk_words: int = 1 << 27):
    """raw_db(seed, nbytes) generated on `device` (uint8 tensor, the same bytes)."""
    import torch
    nwords = (nbytes + 7) // 8
    out = torch.empty(nwords * 8, dtype=torch.uint8, device=device)
    words = out.view(torch.int64)
    for s0 in range(0, nwords, chunk_words):
        c = min(chunk_words, nwords - s0)
        words[s0:s0 + c] = u64_torch(seed, STREAM_DB, s0, c, device)
    return out[:nbytes]


def raw_db_slab(seed: int, start: int, nbytes: int) -> np.ndarray:
    """Bytes [start, start + nbytes) of raw_db(seed, ...), regenerated on their own
    (the stream is counter based); start must be a multiple of 8."""
    assert start % 8 == 0
    w0 = start // 8
    nw = (nbytes + 7) // 8
    return u64(seed, STREAM_DB, w0, nw).view(np.uint8)[:nbytes]
