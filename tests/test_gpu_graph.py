"""Graph-captured answers and the autotuner, through the C ABI: a captured answer
replays bit-exact against the oracle on new query contents, and the tuned options
answer exactly too."""
import time

import numpy as np
import pytest

import paper_2606_11536_gb300 as g
from gpu_util import empty_u32, from_dev, random_queries, to_dev
import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("layout,B", [(0, 1), (0, 8), (1, 8)])
def test_graph_replays_match_oracle(orc, layout, B):
    n, log2p, D1, D2 = 2048, 16, 64, 24
    p = g.pir_make_params(n, log2p, D1, D2, 2)
    P = orc.make_params(n, log2p, D1, D2, 2)
    raw = synth.raw_db(70 + B, synth.raw_db_bytes(n, log2p, D1, D2))
    db = g.pir_setup_db(p, raw, layout=layout)
    try:
        qd = empty_u32(B * D1 * 2 * 2 * n)
        rd = empty_u32(B * D2 * 2 * 2 * n)
        graph = g.pir_graph_create(db, qd, B, rd)
        try:
            for seed in (1, 2):
                Q = random_queries(P, B, 300 + seed)
                qd.copy_(to_dev(Q))
                k0 = g.pir_kernel_launches()
                g.pir_graph_launch(graph)
                R = from_dev(rd, (B, D2, 2, 2, n))
                # NTT, transpose, GEMM, transpose, INTT; batch 1 on the plain layout fuses both
                # transposes away (NTT straight to the slot layout, scan straight to responses)
                assert g.pir_kernel_launches() - k0 == (3 if (layout == 0 and B == 1) else 5)
                assert np.array_equal(R, orc.answer(P, raw, Q)), seed
            g.pir_check_device()
        finally:
            g.pir_graph_destroy(graph)
    finally:
        g.pir_free_db(db)


def test_graph_refuses_flags_and_freed_handles(orc):
    p = g.pir_make_params(2048, 16, 32, 8, 2)
    db = g.pir_setup_db(p, synth.raw_db(5, synth.raw_db_bytes(2048, 16, 32, 8)))
    qd = empty_u32(32 * 2 * 2 * 2048)
    rd = empty_u32(8 * 2 * 2 * 2048)
    graph = g.pir_graph_create(db, qd, 1, rd)
    g.pir_graph_destroy(graph)
    with pytest.raises(g.PirError) as ei:
        g.pir_graph_launch(graph)
    assert ei.value.status == 6
    g.pir_free_db(db)


@pytest.mark.parametrize("layout,B", [(0, 1), (0, 4), (0, 16), (1, 16)])
def test_autotune_picks_an_exact_configuration(orc, layout, B):
    n, log2p, D1, D2 = 2048, 16, 128, 64
    p = g.pir_make_params(n, log2p, D1, D2, 2)
    P = orc.make_params(n, log2p, D1, D2, 2)
    raw = synth.raw_db(80 + B, synth.raw_db_bytes(n, log2p, D1, D2))
    db = g.pir_setup_db(p, raw, layout=layout)
    try:
        best = g.pir_autotune(db, B, reps=2)
        assert 1 <= best["tile"] <= g.pir_gemm_tiles(layout)
        t0 = time.perf_counter()
        assert g.pir_autotune(db, B) == best  # cached
        assert time.perf_counter() - t0 < 0.05
        Q = random_queries(P, B, 90 + B)
        qd, rd = to_dev(Q), empty_u32(B * D2 * 2 * 2 * n)
        g.pir_answer_ex(db, qd, B, rd, **best)
        assert np.array_equal(from_dev(rd, (B, D2, 2, 2, n)), orc.answer(P, raw, Q))
        g.pir_check_device()
    finally:
        g.pir_free_db(db)


def test_release_memory_gives_cached_scratch_back(orc):
    """An answer's scratch stays cached in the library's stream-ordered pool (the
    device's free memory stays lower after it); pir_release_memory gives it back,
    and answers still run and match the oracle afterwards."""
    import torch
    n, log2p, D1, D2, B = 4096, 16, 256, 8, 32
    p = g.pir_make_params(n, log2p, D1, D2, 2)
    P = orc.make_params(n, log2p, D1, D2, 2)
    raw = synth.raw_db(77, synth.raw_db_bytes(n, log2p, D1, D2))
    db = g.pir_setup_db(p, raw, layout=0)
    try:
        Q = random_queries(P, B, 78)
        qd, rd = to_dev(Q), empty_u32(B * D2 * 2 * 2 * n)
        torch.cuda.synchronize()
        g.pir_answer(db, qd, B, rd)  # about 1 GiB of scratch: the NTT-form copy and its slot layout
        torch.cuda.synchronize()
        free_cached = torch.cuda.mem_get_info()[0]
        g.pir_release_memory()
        torch.cuda.synchronize()
        free_released = torch.cuda.mem_get_info()[0]
        assert free_released - free_cached >= (512 << 20), (free_cached, free_released)
        cols = np.array([0, 7], dtype=np.uint32)
        rd2 = empty_u32(B * D2 * 2 * 2 * n)
        g.pir_answer(db, qd, B, rd2)
        R = from_dev(rd2, (B, D2, 2, 2, n))
        assert np.array_equal(R, from_dev(rd, R.shape))
        assert np.array_equal(R[:2][:, cols], orc.answer(P, raw, Q[:2], cols=cols))
        g.pir_check_device()
    finally:
        g.pir_free_db(db)
