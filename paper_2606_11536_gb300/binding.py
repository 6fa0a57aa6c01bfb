"""ctypes binding of ``libgbpir.so`` (C ABI in ``include/gbpir.h``).

Argument marshalling only: every step of the scan runs in the CUDA library.
Device buffers are torch CUDA tensors (uint32 / uint8, contiguous); host
buffers are numpy arrays or CPU tensors.  There is no CPU fallback: if the
library is missing the first call raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

PIR_MAX_L = 4
PIR_LAYOUT_PLAIN = 0
PIR_LAYOUT_LIMB = 1
PIR_LAYOUT_TENSOR = 2

STATUS = {
    0: "PIR_OK", 1: "PIR_ERR_ARG", 2: "PIR_ERR_OOM", 3: "PIR_ERR_ADMISSION", 4: "PIR_ERR_CUDA",
    5: "PIR_ERR_TIMEOUT", 6: "PIR_ERR_HANDLE", 7: "PIR_ERR_UNSUPPORTED",
}

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgbpir.so")


class PirError(RuntimeError):
    def __init__(self, status: int, what: str, detail: str = ""):
        self.status = status
        msg = "%s failed: %s" % (what, STATUS.get(status, str(status)))
        if detail:
            msg += " (%s)" % detail
        super().__init__(msg)


class pir_params_t(C.Structure):
    _fields_ = [
        ("n", C.c_uint32), ("L", C.c_uint32), ("log2p", C.c_uint32), ("D1", C.c_uint32), ("D2", C.c_uint32),
        ("q", C.c_uint32 * PIR_MAX_L), ("psi", C.c_uint32 * PIR_MAX_L),
    ]

    @property
    def qs(self):
        return [int(self.q[j]) for j in range(self.L)]

    @property
    def psis(self):
        return [int(self.psi[j]) for j in range(self.L)]

    def __repr__(self):
        return "pir_params_t(n=%d, L=%d, log2p=%d, D1=%d, D2=%d, q=%s, psi=%s)" % (
            self.n, self.L, self.log2p, self.D1, self.D2, self.qs, self.psis)


class pir_answer_opts_t(C.Structure):
    _fields_ = [("k_chunk", C.c_uint32), ("tile", C.c_uint32), ("flags", C.c_uint32)]


_lib = None


def lib():
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("CUDA library %s is missing: build it first (__graft_entry__.build())" % LIB_PATH)
        L = C.CDLL(LIB_PATH)
        P = C.POINTER(pir_params_t)
        vp, sz, u32, u64, i32 = C.c_void_p, C.c_size_t, C.c_uint32, C.c_uint64, C.c_int
        sigs = {
            "pir_make_params": (i32, [u32, u32, u32, u32, u32, P]),
            "pir_setup_db": (i32, [P, vp, sz, i32, i32, vp, C.POINTER(vp)]),
            "pir_answer": (i32, [vp, vp, u32, vp, i32, vp]),
            "pir_answer_ex": (i32, [vp, vp, u32, vp, i32, vp, C.POINTER(pir_answer_opts_t)]),
            "ntt_fwd": (i32, [P, vp, sz, vp]),
            "ntt_inv": (i32, [P, vp, sz, vp]),
            "ntt_inv_modswitch": (i32, [P, vp, sz, vp, vp]),
            "pir_free_db": (i32, [vp]),
            "pir_db_bytes": (i32, [vp, C.POINTER(sz)]),
            "pir_db_info": (i32, [vp, P, C.POINTER(i32)]),
            "pir_db_read_poly": (i32, [vp, u64, vp]),
            "pir_status_str": (C.c_char_p, [i32]),
            "pir_last_cuda_error": (C.c_char_p, []),
            "pir_gemm_tiles": (u32, [i32]),
            "pir_stage_times": (i32, [C.POINTER(C.c_double), C.POINTER(C.c_uint64)]),
            "pir_kernel_launches": (C.c_uint64, []),
            "pir_check_device": (i32, [vp]),
            "pir_release_memory": (i32, []),
            "pir_device_status": (i32, []),
            "pir_graph_create": (i32, [vp, vp, u32, vp, C.POINTER(pir_answer_opts_t), C.POINTER(vp)]),
            "pir_graph_create_packed": (i32, [vp, vp, vp, u32, vp, C.POINTER(pir_answer_opts_t), C.POINTER(vp)]),
            "pir_graph_launch": (i32, [vp, vp]),
            "pir_graph_destroy": (i32, [vp]),
            "pir_autotune": (i32, [vp, u32, vp, u32, C.POINTER(pir_answer_opts_t)]),
            "pir_answer_noalloc": (i32, [vp, vp, u32, vp, vp]),
            "pir_lwe_answer": (i32, [vp, u32, u32, vp, u32, vp, u32, vp]),
            "pir_fold": (i32, [P, vp, u32, u32, u32, vp, vp, vp]),
            "pir_answer_folded": (i32, [vp, vp, u32, u32, vp, vp, i32, vp, C.POINTER(pir_answer_opts_t)]),
            "pir_probe_int8_mma": (i32, [vp, C.POINTER(C.c_double)]),
            "pir_expander_create": (i32, [P, u32, u32, vp, i32, vp, C.POINTER(vp)]),
            "pir_expander_free": (i32, [vp]),
            "pir_expand": (i32, [vp, vp, u32, u32, vp, vp]),
            "pir_answer_packed": (i32, [vp, vp, vp, u32, vp, i32, vp, C.POINTER(pir_answer_opts_t)]),
            "pir_answer_begin": (i32, [vp, u32, u32, vp, C.POINTER(pir_answer_opts_t), C.POINTER(vp)]),
            "pir_answer_chunk": (i32, [vp, vp, u32, u32, i32]),
            "pir_answer_end": (i32, [vp, vp, i32]),
            "pir_answer_abort": (i32, [vp]),
        }
        for name, (res, args) in sigs.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(st: int, what: str):
    if st != 0:
        detail = ""
        if st == 4:
            detail = lib().pir_last_cuda_error().decode()
        raise PirError(st, what, detail)


def _stream_ptr(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def _ptr(buf):
    """(pointer, on_device, nbytes) of a torch tensor or numpy array."""
    if isinstance(buf, np.ndarray):
        if not buf.flags["C_CONTIGUOUS"]:
            raise ValueError("host buffer must be C-contiguous")
        return C.c_void_p(buf.ctypes.data), False, buf.nbytes
    import torch
    if isinstance(buf, torch.Tensor):
        if not buf.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return C.c_void_p(buf.data_ptr()), buf.is_cuda, buf.numel() * buf.element_size()
    raise TypeError("expected a numpy array or torch tensor, got %r" % type(buf))


# --- the ABI, one function per entry point ---------------------------------

def pir_make_params(n: int, log2p: int, D1: int, D2: int, L: int = 2) -> pir_params_t:
    p = pir_params_t()
    _check(lib().pir_make_params(n, log2p, D1, D2, L, C.byref(p)), "pir_make_params")
    return p


class Db:
    """A resident database handle (owns the device memory until freed)."""

    def __init__(self, handle: int, params: pir_params_t, layout: int):
        self.handle = handle
        self.params = params
        self.layout = layout

    def __repr__(self):
        return "Db(%r, layout=%d)" % (self.params, self.layout)


def pir_setup_db(params: pir_params_t, raw_db, layout: int = PIR_LAYOUT_PLAIN, stream=None) -> Db:
    ptr, on_dev, nbytes = _ptr(raw_db)
    h = C.c_void_p()
    _check(lib().pir_setup_db(C.byref(params), ptr, nbytes, int(on_dev), layout, _stream_ptr(stream), C.byref(h)),
           "pir_setup_db")
    return Db(h.value, params, layout)


def _answer_sizes(db: Db, B: int, flags: int = 0):
    """Bytes of B queries [B][D1][2][L][n] and of their responses [B][D2][2][L][n]
    ([B][D2][2][n] with PIR_ANSWER_MODSWITCH)."""
    p = db.params
    resp_l = 1 if flags & PIR_ANSWER_MODSWITCH else p.L
    return B * p.D1 * 2 * p.L * p.n * 4, B * p.D2 * 2 * resp_l * p.n * 4


def _require(what: str, have: int, need: int):
    """Refuse a buffer smaller than the call reads or writes, before the library
    touches it (on the device that would be an out-of-bounds access)."""
    if have < need:
        raise ValueError("%s buffer holds %d bytes, the call needs %d" % (what, have, need))


def pir_answer(db: Db, queries, B: int, responses, stream=None):
    qp, qdev, qn = _ptr(queries)
    rp, rdev, rn = _ptr(responses)
    if qdev != rdev:
        raise ValueError("queries and responses must both be host or both be device buffers")
    need_q, need_r = _answer_sizes(db, B)
    _require("query", qn, need_q)
    _require("response", rn, need_r)
    _check(lib().pir_answer(C.c_void_p(db.handle), qp, B, rp, int(qdev), _stream_ptr(stream)), "pir_answer")
    return responses


def pir_answer_ex(db: Db, queries, B: int, responses, stream=None, k_chunk: int = 0, tile: int = 0, flags: int = 0):
    qp, qdev, qn = _ptr(queries)
    rp, rdev, rn = _ptr(responses)
    if qdev != rdev:
        raise ValueError("queries and responses must both be host or both be device buffers")
    need_q, need_r = _answer_sizes(db, B, flags)
    _require("query", qn, need_q)
    _require("response", rn, need_r)
    o = pir_answer_opts_t(k_chunk, tile, flags)
    _check(lib().pir_answer_ex(C.c_void_p(db.handle), qp, B, rp, int(qdev), _stream_ptr(stream), C.byref(o)),
           "pir_answer_ex")
    return responses


PIR_NOALLOC_SCRATCH_BYTES = 64 << 20


def pir_answer_noalloc(db: Db, queries, B: int, responses, stream=None):
    """pir_answer on device buffers without any device allocation (scratch comes
    from the library's fixed per-GPU array); for callers that cannot allocate."""
    qp, qdev, qn = _ptr(queries)
    rp, rdev, rn = _ptr(responses)
    need_q, need_r = _answer_sizes(db, B)
    _require("query", qn, need_q)
    _require("response", rn, need_r)
    if not (qdev and rdev):
        raise ValueError("pir_answer_noalloc works on device buffers")
    _check(lib().pir_answer_noalloc(C.c_void_p(db.handle), qp, B, rp, _stream_ptr(stream)), "pir_answer_noalloc")
    return responses


def ntt_fwd(params: pir_params_t, polys, count: int | None = None, stream=None):
    ptr, dev, nbytes = _ptr(polys)
    cnt = nbytes // (4 * params.L * params.n) if count is None else count
    _require("polynomial", nbytes, cnt * 4 * params.L * params.n)
    if not dev:
        raise ValueError("ntt_fwd works on device memory")
    _check(lib().ntt_fwd(C.byref(params), ptr, cnt, _stream_ptr(stream)), "ntt_fwd")
    return polys


def ntt_inv(params: pir_params_t, polys, count: int | None = None, stream=None):
    ptr, dev, nbytes = _ptr(polys)
    cnt = nbytes // (4 * params.L * params.n) if count is None else count
    _require("polynomial", nbytes, cnt * 4 * params.L * params.n)
    if not dev:
        raise ValueError("ntt_inv works on device memory")
    _check(lib().ntt_inv(C.byref(params), ptr, cnt, _stream_ptr(stream)), "ntt_inv")
    return polys


def ntt_inv_modswitch(params: pir_params_t, polys, out, count: int | None = None, stream=None):
    """Inverse NTT of polys [count][L][n] (NTT form) with modulus switching to q_0
    fused in; writes out [count][n] over q_0."""
    ip, idev, nbytes = _ptr(polys)
    op, odev, on = _ptr(out)
    cnt = nbytes // (4 * params.L * params.n) if count is None else count
    _require("polynomial", nbytes, cnt * 4 * params.L * params.n)
    _require("output", on, cnt * 4 * params.n)
    if not (idev and odev):
        raise ValueError("ntt_inv_modswitch works on device memory")
    _check(lib().ntt_inv_modswitch(C.byref(params), ip, cnt, op, _stream_ptr(stream)), "ntt_inv_modswitch")
    return out


def pir_fold(params: pir_params_t, cts, B: int, levels: int, ell: int, rgsw, out, stream=None):
    """Fold cts [B][2^levels][2][L][n] with rgsw [B][levels][2 ell][2][L][n] into out [B][2][L][n]."""
    cp, cdev, cn = _ptr(cts)
    gp, gdev, gn = _ptr(rgsw)
    op, odev, on = _ptr(out)
    ct = ct_bytes(params.n, params.L)
    _require("ciphertext", cn, B * (1 << levels) * ct)
    _require("RGSW", gn, B * levels * 2 * ell * ct)
    _require("output", on, B * ct)
    if not (cdev and gdev and odev):
        raise ValueError("pir_fold works on device buffers")
    _check(lib().pir_fold(C.byref(params), cp, B, levels, ell, gp, op, _stream_ptr(stream)), "pir_fold")
    return out


def pir_answer_folded(db: Db, queries, B: int, ell: int, rgsw, responses, stream=None, tile: int = 0, flags: int = 0):
    """First-dimension answer folded over the remaining log2(D2) levels: responses [B][2][L][n]."""
    qp, qdev, qn = _ptr(queries)
    gp, gdev, gn = _ptr(rgsw)
    rp, rdev, rn = _ptr(responses)
    p = db.params
    levels = max(0, (p.D2 - 1).bit_length())
    _require("query", qn, _answer_sizes(db, B)[0])
    _require("RGSW", gn, B * levels * 2 * ell * ct_bytes(p.n, p.L))
    _require("response", rn, B * ct_bytes(p.n, 1 if flags & PIR_ANSWER_MODSWITCH else p.L))
    if not (qdev == gdev == rdev):
        raise ValueError("queries, rgsw and responses must all be host or all be device buffers")
    o = pir_answer_opts_t(0, tile, flags)
    _check(lib().pir_answer_folded(C.c_void_p(db.handle), qp, B, ell, gp, rp, int(qdev), _stream_ptr(stream),
                                   C.byref(o)), "pir_answer_folded")
    return responses


PIR_LWE_AUTO, PIR_LWE_TENSOR, PIR_LWE_SIMT = 0, 1, 2


def pir_lwe_answer(db, D1: int, D0: int, queries, B: int, out, path: int = PIR_LWE_AUTO, stream=None):
    """Scalar-HE DB GEMM out[b][i] = sum_j db[i][j] queries[b][j] mod 2^32 (device buffers:
    db [D1][D0] int8, queries [B][D0] uint32, out [B][D1] uint32)."""
    dp, ddev, dn = _ptr(db)
    qp, qdev, qn = _ptr(queries)
    op, odev, on = _ptr(out)
    _require("DB", dn, D1 * D0)
    _require("query", qn, B * D0 * 4)
    _require("output", on, B * D1 * 4)
    if not (ddev and qdev and odev):
        raise ValueError("pir_lwe_answer works on device buffers")
    _check(lib().pir_lwe_answer(dp, D1, D0, qp, B, op, path, _stream_ptr(stream)), "pir_lwe_answer")
    return out


def pir_probe_int8_mma(stream=None) -> float:
    """Measured INT8 mma.sync peak of this GPU in TOPS."""
    v = C.c_double()
    _check(lib().pir_probe_int8_mma(_stream_ptr(stream), C.byref(v)), "pir_probe_int8_mma")
    return v.value


class Expander:
    """A client's expansion keys loaded on the device (pir_expander_t)."""

    def __init__(self, handle: int, params: pir_params_t, levels: int, ell: int):
        self.handle, self.params, self.levels, self.ell = handle, params, levels, ell


def pir_expander_create(params: pir_params_t, levels: int, ell: int, keys, stream=None) -> Expander:
    """keys [levels][ell][2][L][n] (coefficient form), host array or device tensor."""
    kp, kdev, kn = _ptr(keys)
    _require("key", kn, levels * ell * ct_bytes(params.n, params.L))
    h = C.c_void_p()
    _check(lib().pir_expander_create(C.byref(params), levels, ell, kp, int(kdev), _stream_ptr(stream), C.byref(h)),
           "pir_expander_create")
    return Expander(h.value, params, levels, ell)


def pir_expander_free(ex: Expander):
    _check(lib().pir_expander_free(C.c_void_p(ex.handle)), "pir_expander_free")
    ex.handle = None


def pir_expand(ex: Expander, packed, B: int, count: int, out, stream=None):
    """Expand packed [B][2][L][n] into out [B][count][2][L][n] (device buffers)."""
    pp, pdev, pn = _ptr(packed)
    op, odev, on = _ptr(out)
    ct = ct_bytes(ex.params.n, ex.params.L)
    _require("packed query", pn, B * ct)
    _require("output", on, B * count * ct)
    if not (pdev and odev):
        raise ValueError("pir_expand works on device buffers")
    _check(lib().pir_expand(C.c_void_p(ex.handle), pp, B, count, op, _stream_ptr(stream)), "pir_expand")
    return out


def pir_answer_packed(db: Db, ex: Expander, packed, B: int, responses, stream=None, k_chunk: int = 0, tile: int = 0,
                      flags: int = 0):
    """pir_answer for packed queries [B][2][L][n]: expansion, then the scan."""
    pp, pdev, pn = _ptr(packed)
    rp, rdev, rn = _ptr(responses)
    if pdev != rdev:
        raise ValueError("packed queries and responses must both be host or both be device buffers")
    _require("packed query", pn, B * ct_bytes(db.params.n, db.params.L))
    _require("response", rn, _answer_sizes(db, B, flags)[1])
    o = pir_answer_opts_t(k_chunk, tile, flags)
    _check(lib().pir_answer_packed(C.c_void_p(db.handle), C.c_void_p(ex.handle), pp, B, rp, int(pdev),
                                   _stream_ptr(stream), C.byref(o)), "pir_answer_packed")
    return responses


def pir_free_db(db: Db):
    _check(lib().pir_free_db(C.c_void_p(db.handle)), "pir_free_db")
    db.handle = None


def pir_db_bytes(db: Db) -> int:
    v = C.c_size_t()
    _check(lib().pir_db_bytes(C.c_void_p(db.handle), C.byref(v)), "pir_db_bytes")
    return v.value


def pir_db_info(db: Db):
    p = pir_params_t()
    lay = C.c_int()
    _check(lib().pir_db_info(C.c_void_p(db.handle), C.byref(p), C.byref(lay)), "pir_db_info")
    return p, lay.value


def pir_db_read_poly(db: Db, poly_index: int) -> np.ndarray:
    out = np.empty((db.params.L, db.params.n), dtype=np.uint32)
    _check(lib().pir_db_read_poly(C.c_void_p(db.handle), poly_index, C.c_void_p(out.ctypes.data)),
           "pir_db_read_poly")
    return out


def pir_status_str(status: int) -> str:
    return lib().pir_status_str(status).decode()


def pir_gemm_tiles(layout: int) -> int:
    return int(lib().pir_gemm_tiles(layout))


PIR_ANSWER_STAGE_TIMES = 1
PIR_ANSWER_TEST_STALL = 2
PIR_ANSWER_MODSWITCH = 4
PIR_ANSWER_CHECK_INPUTS = 8
PIR_STAGES = 5
STAGE_NAMES = ("query_ntt", "query_transpose", "gemm", "result_transpose", "intt")


def pir_stage_times():
    """(ms per stage, launches per stage) of the timed answers since the last call."""
    ms = (C.c_double * PIR_STAGES)()
    ln = (C.c_uint64 * PIR_STAGES)()
    _check(lib().pir_stage_times(ms, ln), "pir_stage_times")
    return list(ms), list(ln)


class Graph:
    """A captured answer bound to fixed device buffers (pir_graph_t)."""

    def __init__(self, handle, db, queries, responses):
        self.handle = handle
        self.db = db
        self._keep = (queries, responses)  # the graph reads / writes these buffers


def pir_graph_create(db: Db, queries, B: int, responses, k_chunk: int = 0, tile: int = 0, flags: int = 0) -> Graph:
    qp, qdev, qn = _ptr(queries)
    rp, rdev, rn = _ptr(responses)
    need_q, need_r = _answer_sizes(db, B, flags)
    _require("query", qn, need_q)
    _require("response", rn, need_r)
    if not (qdev and rdev):
        raise ValueError("a graph binds device buffers")
    o = pir_answer_opts_t(k_chunk, tile, flags)
    h = C.c_void_p()
    _check(lib().pir_graph_create(C.c_void_p(db.handle), qp, B, rp, C.byref(o), C.byref(h)), "pir_graph_create")
    return Graph(h.value, db, queries, responses)


def pir_graph_create_packed(db: Db, ex: "Expander", packed, B: int, responses, tile: int = 0,
                            flags: int = 0) -> Graph:
    """A captured packed-query answer (expansion + answer) bound to fixed device buffers."""
    pp, pdev, pn = _ptr(packed)
    rp, rdev, rn = _ptr(responses)
    _require("packed query", pn, B * ct_bytes(db.params.n, db.params.L))
    _require("response", rn, _answer_sizes(db, B, flags)[1])
    if not (pdev and rdev):
        raise ValueError("a graph binds device buffers")
    o = pir_answer_opts_t(0, tile, flags)
    h = C.c_void_p()
    _check(lib().pir_graph_create_packed(C.c_void_p(db.handle), C.c_void_p(ex.handle), pp, B, rp, C.byref(o),
                                         C.byref(h)), "pir_graph_create_packed")
    g = Graph(h.value, db, packed, responses)
    g.expander = ex
    return g


class Session:
    """A streamed answer (pir_session_t): pieces of the queries along D1."""

    def __init__(self, handle, db, B, kc_max, flags=0):
        self.handle = handle
        self.db = db
        self.B = B
        self.kc_max = kc_max
        self.flags = flags
        self._keep = []  # device pieces are read in stream order: keep them alive


def pir_answer_begin(db: Db, B: int, kc_max: int, stream=None, tile: int = 0, flags: int = 0) -> Session:
    o = pir_answer_opts_t(0, tile, flags)
    h = C.c_void_p()
    _check(lib().pir_answer_begin(C.c_void_p(db.handle), B, kc_max, _stream_ptr(stream), C.byref(o), C.byref(h)),
           "pir_answer_begin")
    return Session(h.value, db, B, kc_max, flags)


def pir_answer_chunk(session: Session, queries, i0: int, kc: int):
    """Ciphertexts i0 .. i0+kc-1 of every query, [B][kc][2][L][n] (host or device)."""
    qp, qdev, qn = _ptr(queries)
    p = session.db.params
    _require("query", qn, session.B * kc * 2 * p.L * p.n * 4)
    _check(lib().pir_answer_chunk(C.c_void_p(session.handle), qp, i0, kc, int(qdev)), "pir_answer_chunk")
    if qdev:
        session._keep.append(queries)


def pir_answer_end(session: Session, responses):
    rp, rdev, rn = _ptr(responses)
    _require("response", rn, _answer_sizes(session.db, session.B, session.flags)[1])
    h, session.handle = session.handle, None
    try:
        _check(lib().pir_answer_end(C.c_void_p(h), rp, int(rdev)), "pir_answer_end")
    finally:
        session._keep = []
    return responses


def pir_answer_abort(session: Session):
    h, session.handle = session.handle, None
    session._keep = []
    _check(lib().pir_answer_abort(C.c_void_p(h)), "pir_answer_abort")


def pir_graph_launch(graph: Graph, stream=None):
    _check(lib().pir_graph_launch(C.c_void_p(graph.handle), _stream_ptr(stream)), "pir_graph_launch")


def pir_graph_destroy(graph: Graph):
    _check(lib().pir_graph_destroy(C.c_void_p(graph.handle)), "pir_graph_destroy")
    graph.handle = None


def pir_autotune(db: Db, B: int, stream=None, reps: int = 3):
    """Fastest (tile, k_chunk) for this DB and batch size, as a dict."""
    o = pir_answer_opts_t()
    _check(lib().pir_autotune(C.c_void_p(db.handle), B, _stream_ptr(stream), reps, C.byref(o)), "pir_autotune")
    return {"tile": int(o.tile), "k_chunk": int(o.k_chunk)}


def pir_check_device(stream=None):
    """Raises PirError(PIR_ERR_TIMEOUT) if a bounded kernel wait ran out since the last check."""
    _check(lib().pir_check_device(_stream_ptr(stream)), "pir_check_device")


def pir_kernel_launches() -> int:
    return int(lib().pir_kernel_launches())


def pir_device_status():
    """Raises PirError(PIR_ERR_TIMEOUT) if a bounded kernel wait ran out since the last
    read; waits for no device work (pir_check_device synchronizes first)."""
    _check(lib().pir_device_status(), "pir_device_status")


def pir_release_memory():
    """Gives the device memory the library keeps cached (answer and graph scratch)
    back, for allocations made outside the library (torch's)."""
    _check(lib().pir_release_memory(), "pir_release_memory")


# --- sizes (host logic) ----------------------------------------------------

def poly_bytes(n: int, L: int) -> int:
    """One RNS polynomial: L rows of n 32-bit residues."""
    return 4 * L * n


def ct_bytes(n: int, L: int) -> int:
    """One RLWE ciphertext: two RNS polynomials."""
    return 2 * poly_bytes(n, L)


def raw_db_bytes(p) -> int:
    return p.D1 * p.D2 * p.n * p.log2p // 8


def answer_scratch_bytes(p, layout: int, B: int) -> int:
    """Device scratch one answer of B queries takes inside the library with the whole
    of D1 at once: the NTT-form query copy (4 bytes per residue), the queries in the
    GEMM's layout (4 bytes per residue; 8 for the tensor layout's bf16 digits) and
    the slot-major result (4 bytes per residue of the 2B x D2 result polynomials)."""
    per_q = 2 * p.L * p.n * 4  # one ciphertext
    layout_q = 2 if layout == PIR_LAYOUT_TENSOR else 1
    return B * (p.D1 * per_q * (1 + layout_q) + p.D2 * per_q)


def resident_db_bytes(p, layout: int = PIR_LAYOUT_PLAIN) -> int:
    """Device bytes of the NTT-form DB: one u32 word (plain) or four u8 limbs (limb)
    per residue, four bf16 digits (tensor) per residue."""
    return (8 if layout == PIR_LAYOUT_TENSOR else 4) * p.L * p.n * p.D1 * p.D2


def query_bytes(p, B: int) -> int:
    return B * p.D1 * ct_bytes(p.n, p.L)


def response_bytes(p, B: int, modswitch: bool = False) -> int:
    """Response buffer bytes; with modulus switching the responses keep one prime."""
    return B * p.D2 * ct_bytes(p.n, 1 if modswitch else p.L)
