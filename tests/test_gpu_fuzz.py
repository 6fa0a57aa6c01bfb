"""Seeded random answers through the C ABI against the oracle, bit for bit: ring size,
prime count, plaintext width, DB shape, layout, batch, GEMM tile, K-chunk and
modulus switching drawn at random (within the documented shape rules), so that
combinations no hand-written case names are covered too."""
import numpy as np
import pytest

import paper_2606_11536_gb300 as g
from gpu_util import empty_u32, from_dev, random_queries, to_dev
import synth

pytestmark = pytest.mark.gpu


def draw(seed):
    rng = np.random.default_rng(1000 + seed)
    n = int(rng.choice([2048, 4096, 8192]))
    L = int(rng.choice([1, 2, 2, 3]))
    log2p = int(rng.choice([8, 12, 16]))
    layout = int(rng.random() < 0.25)
    D1 = 32 * int(rng.integers(1, 4)) if layout else int(rng.integers(1, 97))
    D2 = 4 * int(rng.integers(1, 11))
    B = int(rng.choice([1, 1, 2, 3, 4, 5, 9, 17]))
    while B * D1 * D2 * n > 6e7:  # keep the oracle fast
        B = max(1, B // 2)
        D1 = D1 if layout else max(1, D1 // 2)
    M = 2 * B
    if layout:
        Mp = (M + 15) // 16 * 16
        tile = int(rng.choice([t for t, ok in ((0, True), (1, True), (2, Mp % 32 == 0), (3, Mp % 64 == 0)) if ok]))
    else:
        tiles = [0] + [t for t, ok in ((1, M <= 2), (2, M <= 4), (3, M <= 8), (4, True), (5, True), (6, True),
                                       (7, M <= 8 and D2 <= 512), (8, True)) if ok]
        tile = int(rng.choice(tiles))
    k_chunk = 0 if rng.random() < 0.5 else int(rng.integers(1, D1 + 1))
    if layout and k_chunk:
        k_chunk = 32 * max(1, k_chunk // 32)
    flags = g.PIR_ANSWER_MODSWITCH if rng.random() < 0.3 else 0
    return n, L, log2p, layout, D1, D2, B, tile, k_chunk, flags


@pytest.mark.parametrize("seed", range(16))
def test_random_answer(orc, seed):
    n, L, log2p, layout, D1, D2, B, tile, k_chunk, flags = draw(seed)
    p = g.pir_make_params(n, log2p, D1, D2, L)
    P = orc.make_params(n, log2p, D1, D2, L)
    raw = synth.raw_db(seed, synth.raw_db_bytes(n, log2p, D1, D2))
    db = g.pir_setup_db(p, raw, layout=layout)
    try:
        Q = random_queries(P, B, 2000 + seed)
        want = orc.answer(P, raw, Q)
        if flags:
            want = orc.modswitch(P, want)
        rd = empty_u32(want.size)
        g.pir_answer_ex(db, to_dev(Q), B, rd, k_chunk=k_chunk, tile=tile, flags=flags)
        assert np.array_equal(from_dev(rd, want.shape), want), (n, L, log2p, layout, D1, D2, B, tile, k_chunk, flags)
        g.pir_check_device()
    finally:
        g.pir_free_db(db)


def test_tiles_that_do_not_hold_the_batch_are_refused(orc):
    p = g.pir_make_params(2048, 16, 32, 8, 2)
    P = orc.make_params(2048, 16, 32, 8, 2)
    raw = synth.raw_db(1, synth.raw_db_bytes(2048, 16, 32, 8))
    for layout, B, tile in ((0, 3, 1), (0, 3, 2), (0, 5, 3), (0, 5, 7), (1, 2, 2), (1, 2, 3), (0, 1, 9)):
        db = g.pir_setup_db(p, raw, layout=layout)
        try:
            Q = to_dev(random_queries(P, B, 3))
            with pytest.raises(g.PirError) as ei:
                g.pir_answer_ex(db, Q, B, empty_u32(B * 8 * 2 * 2 * 2048), tile=tile)
            assert ei.value.status == 1, (layout, B, tile)
        finally:
            g.pir_free_db(db)
