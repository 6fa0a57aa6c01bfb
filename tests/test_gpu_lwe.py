"""GPU parity of the scalar-HE (LWE) DB GEMM (Sec. 2.5, Sec. 4.1) through the C ABI:
pir_lwe_answer on the tensor path (mma.sync s8 x u8 on byte planes) and the CUDA-core
dp4a path against the oracle, bit for bit, on ragged shapes (rows, K tails, query
counts around the 8- and 16-query tiles), INT8 and Z_2^32 extremes, a large case on
sampled rows, a toy SimplePIR round trip that decrypts, and the argument checks."""
import numpy as np
import pytest

import paper_2606_11536_gb300 as g
from gpu_util import empty_u32, from_dev, to_dev
import synth

pytestmark = pytest.mark.gpu
MOD = 1 << 32


def dev_i8(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.int8).reshape(-1)).cuda()


def run(A, Q, path):
    D1, D0 = A.shape
    B = Q.shape[0]
    out = empty_u32(B * D1)
    g.pir_lwe_answer(dev_i8(A), D1, D0, to_dev(Q), B, out, path=path)
    return from_dev(out, (B, D1))


def rand(D1, D0, B, seed):
    rng = np.random.default_rng(seed)
    A = rng.integers(-128, 128, size=(D1, D0)).astype(np.int8)
    Q = rng.integers(0, MOD, size=(B, D0), dtype=np.uint64).astype(np.uint32)
    return A, Q


@pytest.mark.parametrize("path", [g.PIR_LWE_TENSOR, g.PIR_LWE_SIMT, g.PIR_LWE_AUTO])
@pytest.mark.parametrize("D1,D0,B", [
    (1, 16, 1), (100, 128, 2), (257, 144, 3), (1000, 1024, 5), (300, 272, 8), (513, 640, 9), (64, 256, 16),
    (777, 384, 17), (256, 1152, 33),
])
def test_matches_oracle(orc, path, D1, D0, B):
    A, Q = rand(D1, D0, B, D1 + D0 + B)
    assert np.array_equal(run(A, Q, path), orc.lwe_gemm(A, Q))


@pytest.mark.parametrize("path", [g.PIR_LWE_TENSOR, g.PIR_LWE_SIMT])
def test_extremes(orc, path):
    D1, D0, B = 40, 4096, 9
    A = np.full((D1, D0), -128, dtype=np.int8)
    A[1::2] = 127
    Q = np.full((B, D0), MOD - 1, dtype=np.uint32)
    Q[1::3] = 1 << 31
    Q[2::3, ::2] = 0
    assert np.array_equal(run(A, Q, path), orc.lwe_gemm(A, Q))


@pytest.mark.parametrize("path", [g.PIR_LWE_TENSOR, g.PIR_LWE_SIMT])
def test_large_sampled_rows(orc, path):
    D1, D0, B = 16384, 8192, 32
    A, Q = rand(D1, D0, B, 11)
    got = run(A, Q, path)
    rows = np.array([0, 1, 63, 64, 255, 4097, 9999, D1 - 1])
    assert np.array_equal(got[:, rows], orc.lwe_gemm(A[rows], Q))


def test_simplepir_round_trip(orc):
    D1, D0, n, B = 200, 1024, 64, 12
    delta = 1 << 24
    rng = np.random.default_rng(3)
    db = rng.integers(-128, 128, size=(D1, D0)).astype(np.int8)
    A_lwe = (synth.u64(6, synth.STREAM_A, 0, D0 * n).reshape(D0, n) & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    s = synth.ternary_secret(6, n).astype(np.int64)
    hint = orc.lwe_gemm(db, A_lwe.T.copy()).T.astype(np.int64)  # [D1][n], offline
    As = (A_lwe.astype(np.int64) @ s) % MOD
    idx = synth.query_indices(6, B, 1, D0)
    Q = np.empty((B, D0), dtype=np.uint32)
    for b in range(B):
        e = synth.gaussian_error(6, D0, start=b * D0).astype(np.int64)
        q = (As + e) % MOD
        q[int(idx[b])] = (q[int(idx[b])] + delta) % MOD
        Q[b] = q.astype(np.uint32)
    ans = run(db, Q, g.PIR_LWE_AUTO).astype(np.int64)
    phase = (ans - (hint @ s)[None, :] % MOD) % MOD
    phase = np.where(phase >= MOD // 2, phase - MOD, phase)
    m = np.round(phase / delta).astype(np.int64) % 256
    for b in range(B):
        assert np.array_equal(m[b], db[:, int(idx[b])].astype(np.int64) % 256), b


def test_arguments():
    A = dev_i8(np.zeros(64 * 40, dtype=np.int8))
    Q = to_dev(np.zeros(40 * 2, dtype=np.uint32))
    out = empty_u32(2 * 64)
    for bad in ((A, 64, 40, Q, 2, out, 1),      # D0 not a multiple of 16
                (A, 64, 32, Q, 0, out, 1),      # no queries
                (A, 64, 32, Q, 2, out, 7)):     # unknown path
        with pytest.raises(g.PirError) as ei:
            g.pir_lwe_answer(*bad[:6], path=bad[6])
        assert ei.value.status == 1
