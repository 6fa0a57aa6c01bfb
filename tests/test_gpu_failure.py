"""Failure detection without a GPU fault: the TMA-staged scan bounds every
barrier wait.  A test hook makes its consumers wait on a barrier nothing arrives
on; the wait runs out after about a second, the kernel sets the device error word
and returns, the host reads PIR_ERR_TIMEOUT, and the context stays usable."""
import numpy as np
import pytest

import paper_2606_11536_gb300 as g
from gpu_util import empty_u32, from_dev, random_queries, to_dev
import synth

pytestmark = pytest.mark.gpu


def test_bounded_wait_reports_timeout_and_context_survives(orc):
    n, log2p, D1, D2 = 2048, 16, 32, 16
    p = g.pir_make_params(n, log2p, D1, D2, 2)
    P = orc.make_params(n, log2p, D1, D2, 2)
    raw = synth.raw_db(12, synth.raw_db_bytes(n, log2p, D1, D2))
    db = g.pir_setup_db(p, raw)
    try:
        B = 1
        Q = random_queries(P, B, 3)
        qd = to_dev(Q)
        rd = empty_u32(B * D2 * 2 * 2 * n)
        g.pir_check_device()  # clean before
        g.pir_answer_ex(db, qd, B, rd, flags=g.PIR_ANSWER_TEST_STALL)
        with pytest.raises(g.PirError) as ei:
            g.pir_check_device()
        assert ei.value.status == 5  # PIR_ERR_TIMEOUT
        g.pir_check_device()  # the word was cleared
        # the non-blocking read sees the same word: set by a second stalled scan,
        # then cleared by the read
        g.pir_answer_ex(db, qd, B, rd, flags=g.PIR_ANSWER_TEST_STALL)
        import torch
        torch.cuda.synchronize()
        with pytest.raises(g.PirError) as ei:
            g.pir_device_status()
        assert ei.value.status == 5
        g.pir_device_status()
        g.pir_check_device()
        # the context still works and answers stay exact
        g.pir_answer(db, qd, B, rd)
        R = from_dev(rd, (B, D2, 2, 2, n))
        assert np.array_equal(R, orc.answer(P, raw, Q))
        g.pir_check_device()
    finally:
        g.pir_free_db(db)


def test_stall_hook_rejected_where_the_scan_does_not_run(orc):
    p = g.pir_make_params(2048, 16, 32, 16, 2)
    raw = synth.raw_db(1, synth.raw_db_bytes(2048, 16, 32, 16))
    db = g.pir_setup_db(p, raw)
    try:
        B = 8  # 16 rows: the tiled GEMM, not the TMA scan
        qd = empty_u32(B * 32 * 2 * 2 * 2048)
        rd = empty_u32(B * 16 * 2 * 2 * 2048)
        with pytest.raises(g.PirError) as ei:
            g.pir_answer_ex(db, qd, B, rd, flags=g.PIR_ANSWER_TEST_STALL)
        assert ei.value.status == 1
    finally:
        g.pir_free_db(db)
