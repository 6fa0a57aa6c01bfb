"""CPU-side checks of the C ABI library: it loads without a GPU, exports every
function include/gbpir.h declares, computes the same ring parameters as the
oracle, and rejects bad arguments with status codes (no GPU call is made)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import paper_2606_11536_gb300 as g
from golden.read import paper_values
from paper_2606_11536_gb300 import binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2606_11536_gb300 import build
    build.build()
    return binding.lib()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "gbpir.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z_0-9]*\s*\**\s*([A-Za-z_][A-Za-z_0-9]*)\s*\(", text, re.M)
    return sorted(set(n for n in names if n not in ("if", "while", "for")))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert {"pir_setup_db", "pir_answer", "ntt_fwd", "ntt_inv"} <= set(names)
    for name in names:
        assert hasattr(lib, name), name


def test_only_the_abi_is_exported(lib):
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", binding.LIB_PATH], capture_output=True, text=True).stdout
    syms = {line.split()[-1] for line in out.splitlines() if line.strip()}
    assert syms == set(declared_functions()), syms ^ set(declared_functions())


@pytest.mark.parametrize("n,log2p", [(2048, 12), (4096, 16), (8192, 16)])
def test_params_match_oracle(lib, orc, n, log2p):
    p = g.pir_make_params(n, log2p, 8, 8, 2)
    P = orc.make_params(n, log2p, 8, 8, 2)
    assert p.qs == P.qs and p.psis == P.psis


def test_param_errors(lib):
    for args in [(1024, 12, 4, 4, 2), (4096, 16, 0, 4, 2), (4096, 16, 4, 4, 0), (4096, 16, 4, 4, 5),
                 (4096, 0, 4, 4, 2), (4096, 29, 4, 4, 2), (3000, 16, 4, 4, 2)]:
        with pytest.raises(g.PirError) as ei:
            g.pir_make_params(*args)
        assert ei.value.status == 1


def test_status_strings(lib):
    for st in range(8):
        assert g.pir_status_str(st)
    assert g.pir_status_str(99) == "unknown status"


def test_bad_handle_and_arguments_without_gpu(lib):
    fake = g.Db(0xDEAD0, g.pir_make_params(2048, 12, 4, 4, 2), 0)
    with pytest.raises(g.PirError) as ei:
        g.pir_db_bytes(fake)
    assert ei.value.status == 6
    q = np.zeros(16, dtype=np.uint32)
    st = lib.pir_answer(C.c_void_p(0xDEAD0), C.c_void_p(q.ctypes.data), 1, C.c_void_p(q.ctypes.data), 0, None)
    assert st == 6
    assert lib.pir_free_db(C.c_void_p(0xDEAD0)) == 6
    # setup with a wrong raw size is refused before any device work
    p = g.pir_make_params(2048, 12, 4, 4, 2)
    raw = np.zeros(10, dtype=np.uint8)
    h = C.c_void_p()
    assert lib.pir_setup_db(C.byref(p), C.c_void_p(raw.ctypes.data), raw.nbytes, 0, 0, None, C.byref(h)) == 1
    # a tampered prime is refused
    bad = g.pir_make_params(2048, 12, 4, 4, 2)
    bad.q[0] += 2
    assert lib.ntt_fwd(C.byref(bad), None, 0, None) == 1
    # unknown layout
    assert lib.pir_setup_db(C.byref(p), C.c_void_p(raw.ctypes.data), raw.nbytes, 0, 7, None, C.byref(h)) == 1


def test_size_formulas_against_paper():
    """Sec. 1 / Sec. 3.6 print these sizes for N = 2^12 with 32-bit residues."""
    pv = paper_values()
    assert binding.poly_bytes(4096, 3) == pv["poly_bytes_n4096_L3"]
    assert binding.ct_bytes(4096, 3) == pv["ct_bytes_n4096_L3"]
    assert 256 * binding.poly_bytes(4096, 3) == pv["G_bytes_Dr256_n4096_L3"]
    assert 256 * binding.ct_bytes(4096, 3) == pv["out_cts_bytes_Dr256_n4096_L3"]
    assert binding.ct_bytes(4096, 1) == pv["response_bytes_n4096_L1"]


def test_config_sizes():
    """The configurations' raw / resident sizes: 768 KiB tiny DB; 1 GiB raw -> 4 GiB resident."""
    p = g.pir_make_params(2048, 12, 16, 16, 2)
    assert binding.raw_db_bytes(p) == 768 * 1024
    p = g.pir_make_params(4096, 16, 512, 256, 2)
    assert binding.raw_db_bytes(p) == 1 << 30 and binding.resident_db_bytes(p) == 4 << 30
    assert binding.query_bytes(p, 1) == 32 << 20 and binding.response_bytes(p, 1) == 16 << 20
    p = g.pir_make_params(4096, 16, 4096, 512, 2)
    assert binding.raw_db_bytes(p) == 16 << 30 and binding.resident_db_bytes(p) == 64 << 30


def test_bench_and_serving_use_exported_names():
    """Every `g.<name>` the benchmark and the serving layer call exists in the package
    (they run only on a GPU machine, so a missing export would surface only there)."""
    import re

    import paper_2606_11536_gb300 as g
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    for rel in ("bench.py", os.path.join("paper_2606_11536_gb300", "serving.py"), "__graft_entry__.py"):
        src = open(os.path.join(root, rel)).read()
        names = set(re.findall(r"\bg\.([A-Za-z_][A-Za-z0-9_]*)", src))
        missing = sorted(n for n in names if not hasattr(g, n))
        assert not missing, (rel, missing)


def test_session_and_tensor_layout_errors_without_gpu(lib):
    """The streamed-answer calls refuse unknown handles, and the tensor layout's shape
    rules are checked, before any device work."""
    q = np.zeros(16, dtype=np.uint32)
    o = binding.pir_answer_opts_t()
    h = C.c_void_p()
    assert lib.pir_answer_begin(C.c_void_p(0xDEAD0), 1, 64, None, C.byref(o), C.byref(h)) == 6
    assert lib.pir_answer_chunk(C.c_void_p(0xBEEF0), C.c_void_p(q.ctypes.data), 0, 1, 0) == 6
    assert lib.pir_answer_chunk(None, C.c_void_p(q.ctypes.data), 0, 1, 0) == 6
    assert lib.pir_answer_end(C.c_void_p(0xBEEF0), C.c_void_p(q.ctypes.data), 0) == 6
    assert lib.pir_answer_abort(C.c_void_p(0xBEEF0)) == 6
    assert lib.pir_answer_abort(None) == 6
    assert g.pir_gemm_tiles(g.PIR_LAYOUT_TENSOR) == 5
    # tensor layout: D1 a multiple of 64 and D2 of 32, refused as unsupported otherwise
    for D1, D2 in ((96, 32), (64, 36)):
        p = g.pir_make_params(2048, 12, D1, D2, 2)
        raw = np.zeros(binding.raw_db_bytes(p), dtype=np.uint8)
        st = lib.pir_setup_db(C.byref(p), C.c_void_p(raw.ctypes.data), raw.nbytes, 0, g.PIR_LAYOUT_TENSOR, None,
                              C.byref(h))
        assert st == 7, (D1, D2, st)


def test_answer_buffers_too_small_are_refused_before_the_library(lib):
    """The binding refuses query and response buffers smaller than the call reads
    or writes, before the library sees them; right-sized buffers reach the library
    (which then refuses the fake handle)."""
    p = g.pir_make_params(2048, 12, 4, 4, 2)
    fake = g.Db(0xDEAD0, p, 0)
    words = 4 * 2 * 2 * 2048  # one query [D1][2][L][n], one response [D2][2][L][n] (D1 = D2 = 4)
    q, r = np.zeros(words, np.uint32), np.zeros(words, np.uint32)
    for args in ((q[:-1], 1, r), (q, 1, r[:-1]), (q, 2, r)):
        with pytest.raises(ValueError):
            g.pir_answer(fake, *args)
    with pytest.raises(g.PirError) as ei:  # an explicit null stream: no CUDA needed here
        g.pir_answer(fake, q, 1, r, stream=0)
    assert ei.value.status == 6
    # modulus switching halves the response at L = 2
    with pytest.raises(g.PirError) as ei:
        g.pir_answer_ex(fake, q, 1, r[:words // 2], stream=0, flags=g.PIR_ANSWER_MODSWITCH)
    assert ei.value.status == 6
    with pytest.raises(ValueError):
        g.pir_answer_ex(fake, q, 1, r[:words // 2])
    # streamed pieces: 2 queries x 3 ciphertexts need more than q holds; the end call
    ses = g.Session(0xBEEF0, fake, 2, 4)
    with pytest.raises(ValueError):
        g.pir_answer_chunk(ses, q, 0, 3)
    with pytest.raises(ValueError):
        g.pir_answer_end(ses, r)
    assert ses.handle == 0xBEEF0  # a refused end leaves the session to the caller


def test_every_buffer_taking_call_refuses_short_buffers(lib):
    """Each call that takes caller buffers checks their sizes against the shapes it
    documents before the library sees them (a short device buffer would be written
    past its end, and a captured graph would keep doing so on every launch)."""
    n, L, D1, D2, B = 2048, 2, 4, 4, 2
    p = g.pir_make_params(n, 12, D1, D2, L)
    fake = g.Db(0xDEAD0, p, 0)
    ct = 2 * L * n  # words of one ciphertext
    ok_q, ok_r = np.zeros(B * D1 * ct, np.uint32), np.zeros(B * D2 * ct, np.uint32)

    def short(call, *args, **kw):
        with pytest.raises(ValueError, match="holds"):
            call(*args, **kw)

    short(g.pir_answer_noalloc, fake, ok_q[:-1], B, ok_r)
    short(g.pir_answer_noalloc, fake, ok_q, B, ok_r[:-1])
    short(g.pir_graph_create, fake, ok_q[:-1], B, ok_r)
    short(g.pir_graph_create, fake, ok_q, B, ok_r[:-1])
    short(g.pir_graph_create, fake, ok_q, B + 1, ok_r)
    # packed queries: one ciphertext per query
    ex = g.Expander(0xBEEF0, p, 2, 4)
    short(g.pir_answer_packed, fake, ex, np.zeros(B * ct - 1, np.uint32), B, ok_r)
    short(g.pir_answer_packed, fake, ex, np.zeros(B * ct, np.uint32), B, ok_r[:-1])
    short(g.pir_expand, ex, np.zeros(B * ct - 1, np.uint32), B, 4, np.zeros(B * 4 * ct, np.uint32))
    short(g.pir_expand, ex, np.zeros(B * ct, np.uint32), B, 4, np.zeros(B * 4 * ct - 1, np.uint32))
    short(g.pir_expander_create, p, 2, 4, np.zeros(2 * 4 * ct - 1, np.uint32))
    # folding: levels = log2 D2 = 2, 2 ell RGSW rows per level
    ell, lv = 3, 2
    rg = np.zeros(B * lv * 2 * ell * ct, np.uint32)
    short(g.pir_answer_folded, fake, ok_q, B, ell, rg[:-1], np.zeros(B * ct, np.uint32))
    short(g.pir_answer_folded, fake, ok_q, B, ell, rg, np.zeros(B * ct - 1, np.uint32))
    short(g.pir_answer_folded, fake, ok_q[:-1], B, ell, rg, np.zeros(B * ct, np.uint32))
    short(g.pir_fold, p, np.zeros(B * 4 * ct - 1, np.uint32), B, lv, ell, rg, np.zeros(B * ct, np.uint32))
    short(g.pir_fold, p, np.zeros(B * 4 * ct, np.uint32), B, lv, ell, rg[:-1], np.zeros(B * ct, np.uint32))
    short(g.pir_fold, p, np.zeros(B * 4 * ct, np.uint32), B, lv, ell, rg, np.zeros(B * ct - 1, np.uint32))
    # scalar-HE GEMM: db [D1][D0] int8, queries [B][D0], out [B][D1]
    short(g.pir_lwe_answer, np.zeros(64 * 32 - 1, np.int8), 64, 32, np.zeros(B * 32, np.uint32), B,
          np.zeros(B * 64, np.uint32))
    short(g.pir_lwe_answer, np.zeros(64 * 32, np.int8), 64, 32, np.zeros(B * 32 - 1, np.uint32), B,
          np.zeros(B * 64, np.uint32))
    short(g.pir_lwe_answer, np.zeros(64 * 32, np.int8), 64, 32, np.zeros(B * 32, np.uint32), B,
          np.zeros(B * 64 - 1, np.uint32))
    # NTTs with an explicit count larger than the buffer, and a short switched output
    short(g.ntt_fwd, p, np.zeros(3 * L * n, np.uint32), 4)
    short(g.ntt_inv, p, np.zeros(3 * L * n, np.uint32), 4)
    short(g.ntt_inv_modswitch, p, np.zeros(3 * L * n, np.uint32), np.zeros(3 * n - 1, np.uint32))
    # right-sized buffers pass the size checks and meet the device check instead
    with pytest.raises(ValueError, match="device"):
        g.pir_answer_noalloc(fake, ok_q, B, ok_r)
    with pytest.raises(ValueError, match="device"):
        g.pir_fold(p, np.zeros(B * 4 * ct, np.uint32), B, lv, ell, rg, np.zeros(B * ct, np.uint32))


def test_resident_bytes_follow_the_layout():
    p = g.pir_make_params(4096, 16, 512, 256, 2)
    assert binding.resident_db_bytes(p) == 4 << 30
    assert binding.resident_db_bytes(p, g.PIR_LAYOUT_LIMB) == 4 << 30
    assert binding.resident_db_bytes(p, g.PIR_LAYOUT_TENSOR) == 8 << 30
