"""GPU NTT parity: ntt_fwd / ntt_inv through the C ABI, bit-exact against the
oracle's NTT (itself pinned to the definition and schoolbook products)."""
import numpy as np
import pytest

import paper_2606_11536_gb300 as g
from gpu_util import empty_u32, from_dev, to_dev
import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,log2p,L,count", [(2048, 12, 2, 7), (4096, 16, 2, 33), (8192, 16, 2, 5),
                                              (4096, 16, 1, 3), (2048, 16, 3, 4), (8192, 16, 4, 2)])
def test_ntt_fwd_inv_match_oracle(orc, n, log2p, L, count):
    p = g.pir_make_params(n, log2p, 1, 1, L)
    P = orc.make_params(n, log2p, 1, 1, L)
    a = synth.uniform_residues(n + count, synth.STREAM_UNIFORM, count, n, P.qs)
    # include the extreme residues 0 and q-1
    a[0, :, :4] = 0
    for j, q in enumerate(P.qs):
        a[0, j, 4:8] = q - 1
    d = to_dev(a)
    g.ntt_fwd(p, d)
    A = from_dev(d, a.shape)
    assert np.array_equal(A, orc.ntt_fwd_rns(P, a))
    g.ntt_inv(p, d)
    assert np.array_equal(from_dev(d, a.shape), a)
    # inverse of arbitrary NTT-domain data against the oracle's inverse
    d2 = to_dev(a)
    g.ntt_inv(p, d2)
    assert np.array_equal(from_dev(d2, a.shape), orc.ntt_inv_rns(P, a))


def test_ntt_sweep_many_polys(orc):
    """A larger batch (grid of thousands of CTAs), checked on sampled rows."""
    n, count = 4096, 4096
    p = g.pir_make_params(n, 16, 1, 1, 2)
    P = orc.make_params(n, 16, 1, 1, 2)
    a = synth.uniform_residues(77, synth.STREAM_UNIFORM, count, n, P.qs)
    d = to_dev(a)
    g.ntt_fwd(p, d)
    A = from_dev(d, a.shape)
    rows = np.random.default_rng(0).choice(count, size=24, replace=False)
    assert np.array_equal(A[rows], orc.ntt_fwd_rns(P, a[rows]))
    g.ntt_inv(p, d)
    assert np.array_equal(from_dev(d, a.shape), a)


def test_ntt_zero_count_is_ok():
    p = g.pir_make_params(4096, 16, 1, 1, 2)
    d = empty_u32(4)
    g.ntt_fwd(p, d, count=0)
