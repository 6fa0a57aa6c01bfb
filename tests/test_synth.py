"""The seeded generators: the torch (device-side) SplitMix64 streams reproduce the
numpy ones bit for bit, and the draws have the stated distributions."""
import numpy as np
import pytest

import synth


def test_splitmix64_reference_values():
    # SplitMix64 with state 0: the first outputs of the published generator
    # (Steele, Lea & Flood 2014; the same constants as Java's SplittableRandom)
    st = 0
    outs = []
    for _ in range(3):
        st = (st + 0x9E3779B97F4A7C15) & (2 ** 64 - 1)
        outs.append(synth._mix_int(st))
    assert outs[0] == 0xE220A8397B1DCDAF
    assert outs[1] == 0x6E789E6AA1B965F4
    assert outs[2] == 0x06C45D188009454F


def test_numpy_stream_matches_python_ints():
    key = synth.stream_key(7, 3)
    v = synth.u64(7, 3, 10, 5)
    for t in range(5):
        want = synth._mix_int(key + (10 + t + 1) * 0x9E3779B97F4A7C15)
        assert int(v[t]) == want


def test_torch_stream_matches_numpy():
    torch = pytest.importorskip("torch")
    a = synth.u64(11, 4, 123, 1000)
    b = synth.u64_torch(11, 4, 123, 1000).numpy().view(np.uint64)
    assert np.array_equal(a, b)
    qs = [1073479681, 1072496641]
    r1 = synth.uniform_residues(5, synth.STREAM_UNIFORM, 7, 64, qs, start=3)
    r2 = synth.uniform_residues_torch(5, synth.STREAM_UNIFORM, 7, 64, qs, start=3, chunk=100).numpy().view(np.uint32)
    assert np.array_equal(r1, r2)


def test_distributions():
    s = synth.ternary_secret(3, 30000)
    assert set(np.unique(s)) == {-1, 0, 1}
    assert abs(s.mean()) < 0.03
    e = synth.gaussian_error(3, 200000)
    assert abs(e.std() - 3.2) < 0.05 and np.abs(e).max() <= 19
    raw = synth.raw_db(0, 1 << 20)
    counts = np.bincount(raw, minlength=256)
    assert counts.min() > 3500 and counts.max() < 4700
    idx = synth.query_indices(1, 1000, 512, 256)
    assert idx.min() >= 0 and idx.max() < 512 * 256


def test_raw_db_on_device_and_slabs_match_host():
    torch = pytest.importorskip("torch")
    full = synth.raw_db(4, 5000)
    assert np.array_equal(synth.raw_db_torch(4, 5000, chunk_words=100).numpy(), full)
    assert np.array_equal(synth.raw_db_slab(4, 1024, 777), full[1024:1024 + 777])
