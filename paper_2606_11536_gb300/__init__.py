"""GB300 (sm_103a) RLWE-PIR first-dimension scan.

The CUDA library is loaded on first use (``binding.lib()``); the package imports
without a GPU so that host logic and the seeded input generator work anywhere.
"""
from .binding import (  # noqa: F401
    PIR_LAYOUT_LIMB, PIR_LAYOUT_PLAIN, PIR_LAYOUT_TENSOR, Db, PirError, ntt_fwd, ntt_inv, pir_answer, pir_answer_ex, pir_db_bytes,
    pir_db_info, pir_db_read_poly, pir_free_db, pir_gemm_tiles, pir_make_params, pir_params_t, pir_setup_db,
    pir_status_str, pir_stage_times, pir_kernel_launches, PIR_ANSWER_STAGE_TIMES,
    PIR_ANSWER_TEST_STALL, pir_check_device, Graph, pir_graph_create, pir_graph_create_packed, pir_graph_launch, pir_graph_destroy,
    pir_autotune, pir_answer_noalloc, ntt_inv_modswitch, PIR_ANSWER_MODSWITCH, PIR_ANSWER_CHECK_INPUTS, Expander, pir_expander_create,
    pir_expander_free, pir_expand, pir_answer_packed, pir_lwe_answer, PIR_LWE_AUTO, PIR_LWE_TENSOR, PIR_LWE_SIMT,
    pir_probe_int8_mma, pir_fold, pir_answer_folded, Session, pir_answer_begin, pir_answer_chunk, pir_answer_end,
    pir_answer_abort, pir_release_memory, pir_device_status,
)
