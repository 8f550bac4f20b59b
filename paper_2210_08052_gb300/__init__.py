"""Python binding of the GB300 spliced protein-to-genome DP library.

A thin ctypes layer over ``libmpdp.so`` (``include/mp_dp.h``): every call
marshals arguments and forwards to the C ABI of the same name.  All of the
alignment work runs in the library's CUDA kernels; there is no CPU path, and
importing a function fails loudly when the library has not been built.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

SO_PATH = _build.SO

MP_OK, MP_EINVAL, MP_ENOMEM, MP_EBUDGET, MP_ETIMEOUT = 0, -1, -2, -3, -4
MP_ECUDA, MP_EPENDING, MP_EAGAIN, MP_ETICKET, MP_ESTATE, MP_ETOOLARGE = -5, -6, -7, -8, -9, -10
MP_ST_RERUN, MP_ST_BADSEQ, MP_ST_BUDGET, MP_ST_TRACE, MP_ST_TIMEOUT, MP_ST_ERRMASK = 0x1, 0x10, 0x20, 0x40, 0x80, 0xF0
MP_PAIR_SCORE_ONLY = 0x1
MP_SPLICE_FINAL, MP_SPLICE_SIMPLE = 0, 1
MP_MODE_LOCAL, MP_MODE_GLOBAL, MP_MODE_EXTEND = 0, 1, 2
MP_DEBUG_NO_PUBLISH = 0x1
OP_NAMES = "MIDFGNUV"

EXPORTED = ["mp_dp_default_params", "mp_dp_init", "mp_dp_align_batch", "mp_dp_batch_upload",
            "mp_dp_batch_run", "mp_dp_batch_sync", "mp_dp_batch_download", "mp_dp_batch_free",
            "mp_dp_submit", "mp_dp_poll", "mp_dp_wait_any", "mp_dp_destroy", "mp_dp_strerror",
            "mp_dp_set_timing", "mp_dp_get_stats", "mp_dp_num_sms", "mp_dp_get_serve_stats",
            "mp_dp_score_pair_noalloc", "mp_dp_autotune", "mp_dp_set_tuning", "mp_dp_get_tuning",
            "mp_dp_tuning_save", "mp_dp_tuning_load", "mp_dp_exon_rescore", "mp_dp_debug_h",
            "mp_index_build", "mp_index_chain", "mp_index_download", "mp_index_free", "mp_dp_op_rates",
            "mp_chain_refine"]


class mp_dp_params(ctypes.Structure):
    _fields_ = [("q", ctypes.c_int32), ("e", ctypes.c_int32), ("f", ctypes.c_int32),
                ("r", ctypes.c_int32), ("stop", ctypes.c_int32),
                ("mat", (ctypes.c_int8 * 22) * 22),
                ("splice_model", ctypes.c_int32), ("mode", ctypes.c_int32),
                ("tb_budget_bytes", ctypes.c_uint64), ("force_int32", ctypes.c_int32),
                ("max_pairs_per_launch", ctypes.c_int32), ("wait_limit", ctypes.c_int32),
                ("debug_flags", ctypes.c_int32), ("autotune", ctypes.c_int32),
                ("splice_p", ctypes.c_int32), ("exon_rescore", ctypes.c_int32), ("reserved", ctypes.c_int32 * 1)]


class mp_op_rates(ctypes.Structure):
    _fields_ = [("max_u16x2", ctypes.c_double), ("viaddmax_u16x2", ctypes.c_double),
                ("vimax3_u16x2", ctypes.c_double), ("prmt", ctypes.c_double), ("lop3", ctypes.c_double),
                ("imad", ctypes.c_double), ("step_cells_per_clk_sm", ctypes.c_double),
                ("warps_per_sm_step", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class mp_profile_pos(ctypes.Structure):
    _fields_ = [("subst", ctypes.c_int16 * 21), ("gap_open", ctypes.c_int16), ("gap_ext", ctypes.c_int16),
                ("reserved", ctypes.c_int16)]


class mp_pair(ctypes.Structure):
    _fields_ = [("prot", ctypes.c_char_p), ("prot_len", ctypes.c_uint32),
                ("nt", ctypes.c_char_p), ("nt_len", ctypes.c_uint32),
                ("strand", ctypes.c_int8), ("flags", ctypes.c_uint32),
                ("profile", ctypes.POINTER(mp_profile_pos))]


def profile_array(prof) -> np.ndarray:
    """A profile query's positions as the C ABI takes them (mp_profile_pos
    records): prof is an int array of shape (|P| + 1, 23), row j holding
    the 21 substitution scores of position j (ARNDCQEGHILKMFPSTWYV, then
    the stop codon), its gap open and its gap extension cost."""
    prof = np.asarray(prof)
    if prof.ndim != 2 or prof.shape[1] != 23:
        raise ValueError("a profile is an array of shape (|P| + 1, 23)")
    out = np.zeros((prof.shape[0], 24), dtype=np.int16)
    out[:, :23] = prof
    return out


class mp_result(ctypes.Structure):
    _fields_ = [("score", ctypes.c_int32), ("status", ctypes.c_int32),
                ("prot_st", ctypes.c_int32), ("prot_en", ctypes.c_int32),
                ("nt_st", ctypes.c_int32), ("nt_en", ctypes.c_int32),
                ("n_cigar", ctypes.c_uint32), ("exon_score", ctypes.c_int32),
                ("cigar", ctypes.POINTER(ctypes.c_uint32))]


class mp_dp_stats(ctypes.Structure):
    _fields_ = [("cells", ctypes.c_double), ("dp_ms", ctypes.c_double), ("rerun_ms", ctypes.c_double),
                ("tb_ms", ctypes.c_double), ("pack_ms", ctypes.c_double), ("total_ms", ctypes.c_double),
                ("n_waves", ctypes.c_int32), ("n_rerun", ctypes.c_int32), ("n_launches", ctypes.c_int32),
                ("n_dp_launches", ctypes.c_int32), ("code_bytes", ctypes.c_uint64),
                ("record_bytes", ctypes.c_uint64), ("record_read_bytes", ctypes.c_uint64),
                ("boundary_bytes", ctypes.c_uint64)]


class mp_dp_tuning(ctypes.Structure):
    _fields_ = [("dp16_variant", ctypes.c_int32), ("dp16_ctas_per_sm", ctypes.c_int32),
                ("dp32_ctas_per_sm", ctypes.c_int32), ("wide_direct", ctypes.c_int32),
                ("overlap_waves", ctypes.c_int32), ("item_order", ctypes.c_int32), ("ms", ctypes.c_float),
                ("strip_width", ctypes.c_int32)]


TUNING_KEYS = ("dp16_variant", "dp16_ctas_per_sm", "dp32_ctas_per_sm", "wide_direct", "overlap_waves", "item_order",
               "strip_width", "ms")


class mp_dp_serve_stats(ctypes.Structure):
    _fields_ = [("completed", ctypes.c_uint64), ("batches", ctypes.c_uint64),
                ("mean_batch_pairs", ctypes.c_double), ("p50_ms", ctypes.c_double),
                ("p99_ms", ctypes.c_double), ("max_ms", ctypes.c_double)]


_lib = None


def lib():
    """Load libmpdp.so.  Raises if it has not been built: there is no fallback."""
    global _lib
    if _lib is None:
        if not os.path.exists(SO_PATH):
            raise RuntimeError(f"CUDA library not built ({SO_PATH}); run __graft_entry__.build()")
        L = ctypes.CDLL(SO_PATH)
        P = ctypes.POINTER
        vp = ctypes.c_void_p
        sig = {
            "mp_dp_default_params": (None, [P(mp_dp_params)]),
            "mp_dp_init": (ctypes.c_int, [P(vp), P(mp_dp_params), ctypes.c_int]),
            "mp_dp_align_batch": (ctypes.c_int, [vp, P(mp_pair), ctypes.c_size_t, P(mp_result)]),
            "mp_dp_batch_upload": (ctypes.c_int, [vp, P(mp_pair), ctypes.c_size_t, P(vp)]),
            "mp_dp_batch_run": (ctypes.c_int, [vp, vp]),
            "mp_dp_batch_sync": (ctypes.c_int, [vp]),
            "mp_dp_batch_download": (ctypes.c_int, [vp, vp, P(mp_result)]),
            "mp_dp_batch_free": (None, [vp, vp]),
            "mp_dp_submit": (ctypes.c_int, [vp, P(mp_pair), P(ctypes.c_uint64)]),
            "mp_dp_poll": (ctypes.c_int, [vp, ctypes.c_uint64, P(mp_result), ctypes.c_int64]),
            "mp_dp_wait_any": (ctypes.c_int, [vp, P(ctypes.c_uint64), P(mp_result), ctypes.c_int64]),
            "mp_dp_destroy": (None, [vp]),
            "mp_dp_strerror": (ctypes.c_char_p, [ctypes.c_int]),
            "mp_dp_set_timing": (ctypes.c_int, [vp, ctypes.c_int]),
            "mp_dp_get_stats": (ctypes.c_int, [vp, P(mp_dp_stats)]),
            "mp_dp_num_sms": (ctypes.c_int, [vp]),
            "mp_dp_op_rates": (ctypes.c_int, [ctypes.c_int, P(mp_op_rates)]),
            "mp_dp_get_serve_stats": (ctypes.c_int, [vp, P(mp_dp_serve_stats), ctypes.c_int]),
            "mp_dp_score_pair_noalloc": (ctypes.c_int, [P(mp_dp_params), vp, ctypes.c_uint32, vp, ctypes.c_uint32,
                                                        ctypes.c_int8, vp, vp]),
            "mp_dp_autotune": (ctypes.c_int, [vp, vp, P(mp_dp_tuning), P(mp_dp_tuning), ctypes.c_int,
                                              P(ctypes.c_int)]),
            "mp_dp_set_tuning": (ctypes.c_int, [vp, P(mp_dp_tuning)]),
            "mp_dp_get_tuning": (ctypes.c_int, [vp, vp, P(mp_dp_tuning)]),
            "mp_dp_tuning_save": (ctypes.c_int, [vp, ctypes.c_char_p]),
            "mp_dp_exon_rescore": (ctypes.c_int, [vp, P(mp_pair), ctypes.c_size_t, P(mp_result)]),
            "mp_dp_tuning_load": (ctypes.c_int, [vp, ctypes.c_char_p]),
            "mp_dp_debug_h": (ctypes.c_int, [vp, vp, ctypes.c_size_t, vp]),
            "mp_index_build": (ctypes.c_int, [vp, ctypes.c_char_p, ctypes.c_uint64, P(vp)]),
            "mp_index_chain": (ctypes.c_int, [vp, vp, vp, vp, vp, ctypes.c_uint32, ctypes.c_int32, vp, vp]),
            "mp_chain_refine": (ctypes.c_int, [vp, vp, ctypes.c_size_t, vp]),
            "mp_index_download": (ctypes.c_int, [vp, vp, vp, vp, P(ctypes.c_uint64)]),
            "mp_index_free": (None, [vp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class MPError(RuntimeError):
    def __init__(self, code, where=""):
        self.code = code
        msg = lib().mp_dp_strerror(code).decode()
        super().__init__(f"{where}: {msg} ({code})" if where else f"{msg} ({code})")


def _check(rc, where):
    if rc != MP_OK:
        raise MPError(rc, where)


# ------------------------------------------------------------------ params
def mp_dp_default_params(**overrides) -> mp_dp_params:
    p = mp_dp_params()
    lib().mp_dp_default_params(ctypes.byref(p))
    for k, v in overrides.items():
        if k == "mat":
            m = np.asarray(v, dtype=np.int64)
            for a in range(22):
                for b in range(22):
                    p.mat[a][b] = int(m[a, b])
        else:
            setattr(p, k, v)
    return p


def params_matrix(p: mp_dp_params) -> np.ndarray:
    return np.array([[p.mat[a][b] for b in range(22)] for a in range(22)], dtype=np.int32)


# ------------------------------------------------------------------- pairs
class _PairArray:
    """ctypes array of mp_pair; keeps the encoded sequences alive."""

    def __init__(self, pairs):
        self.keep = []
        n = len(pairs)
        self.arr = (mp_pair * max(n, 1))()
        for k, p in enumerate(pairs):
            prot, nt, strand, flags = _unpack_pair(p)
            self.keep.append(prot)
            self.keep.append(nt)
            self.arr[k].prot = prot
            self.arr[k].prot_len = len(prot)
            self.arr[k].nt = nt
            self.arr[k].nt_len = len(nt)
            self.arr[k].strand = strand
            self.arr[k].flags = flags
            prof = getattr(p, "profile", None)
            if prof is not None:
                pa = profile_array(prof)
                if pa.shape[0] != len(prot) + 1:
                    raise ValueError("a profile has |P| + 1 positions")
                self.keep.append(pa)
                self.arr[k].profile = pa.ctypes.data_as(ctypes.POINTER(mp_profile_pos))
        self.n = n


def _unpack_pair(p):
    if isinstance(p, (tuple, list)):
        prot, nt = p[0], p[1]
        strand = p[2] if len(p) > 2 else 1
        flags = p[3] if len(p) > 3 else 0
    else:
        prot, nt, strand = p.prot, p.nt, getattr(p, "strand", 1)
        flags = MP_PAIR_SCORE_ONLY if getattr(p, "score_only", False) else 0
    prot = prot.encode() if isinstance(prot, str) else bytes(prot)
    nt = nt.encode() if isinstance(nt, str) else bytes(nt)
    return prot, nt, int(strand), int(flags)


def result_dict(r: mp_result) -> dict:
    cig = [(OP_NAMES[r.cigar[k] & 0xF], r.cigar[k] >> 4) for k in range(r.n_cigar)] if r.n_cigar else []
    raw = [r.cigar[k] for k in range(r.n_cigar)] if r.n_cigar else []
    return dict(score=r.score, status=r.status, prot_st=r.prot_st, prot_en=r.prot_en,
                nt_st=r.nt_st, nt_en=r.nt_en, cigar=cig, cigar_raw=raw, exon_score=r.exon_score)


# ------------------------------------------------------------- C-ABI mirror
def mp_dp_init(params: mp_dp_params | None = None, device: int = 0) -> ctypes.c_void_p:
    ctx = ctypes.c_void_p()
    _check(lib().mp_dp_init(ctypes.byref(ctx), ctypes.byref(params) if params is not None else None, device),
           "mp_dp_init")
    return ctx


def mp_dp_destroy(ctx) -> None:
    lib().mp_dp_destroy(ctx)


class PairBatch(_PairArray):
    """A C-ABI array of mp_pair built once from host sequences (what a C
    caller passes to mp_dp_align_batch); reusable across calls."""


class RegionBatch(_PairArray):
    """mp_pair records pointing into two host buffers without copying: the
    proteins (ASCII, concatenated) and a genome (ASCII), with one record per
    (protein, genome interval, strand).  The buffers must stay alive and
    unchanged while the batch is in use (the object keeps references)."""

    def __init__(self, prot_buf, prot_off, prot_len, nt_buf, nt_off, nt_len, strand, flags=None):
        prot_buf = np.ascontiguousarray(prot_buf, dtype=np.uint8)
        nt_buf = np.ascontiguousarray(nt_buf, dtype=np.uint8)
        n = len(prot_off)
        prot_off, prot_len = np.asarray(prot_off, np.int64), np.asarray(prot_len, np.int64)
        nt_off, nt_len = np.asarray(nt_off, np.int64), np.asarray(nt_len, np.int64)
        if n and (prot_off.min() < 0 or (prot_off + prot_len).max() > len(prot_buf) or nt_off.min() < 0 or
                  (nt_off + nt_len).max() > len(nt_buf) or prot_len.max() >= 1 << 32 or nt_len.max() >= 1 << 32):
            raise ValueError("a record lies outside its buffer")
        dt = np.dtype({"names": ["prot", "prot_len", "nt", "nt_len", "strand", "flags", "profile"],
                       "formats": [np.uint64, np.uint32, np.uint64, np.uint32, np.int8, np.uint32, np.uint64],
                       "offsets": [mp_pair.prot.offset, mp_pair.prot_len.offset, mp_pair.nt.offset,
                                   mp_pair.nt_len.offset, mp_pair.strand.offset, mp_pair.flags.offset,
                                   mp_pair.profile.offset],
                       "itemsize": ctypes.sizeof(mp_pair)})
        rec = np.zeros(max(n, 1), dtype=dt)
        rec["prot"][:n] = prot_buf.ctypes.data + prot_off
        rec["prot_len"][:n] = prot_len
        rec["nt"][:n] = nt_buf.ctypes.data + nt_off
        rec["nt_len"][:n] = nt_len
        rec["strand"][:n] = np.asarray(strand, np.int8)
        rec["flags"][:n] = 0 if flags is None else np.asarray(flags, np.uint32)
        self.keep = [prot_buf, nt_buf, rec]
        self.arr = ctypes.cast(rec.ctypes.data, ctypes.POINTER(mp_pair))
        self.n = n


def mp_dp_align_batch(ctx, pairs, raw: bool = False):
    """Align pairs end to end (a list of pairs, or a PairBatch).  Returns a
    list of result dicts, or with raw=True a structured numpy array of the
    mp_result records."""
    pa = pairs if isinstance(pairs, _PairArray) else _PairArray(pairs)
    res = (mp_result * max(pa.n, 1))()
    _check(lib().mp_dp_align_batch(ctx, pa.arr, pa.n, res), "mp_dp_align_batch")
    return _results(res, pa.n, raw)


def _results(res, n, raw):
    if not raw:
        return [result_dict(res[k]) for k in range(n)]
    buf = np.frombuffer(res, dtype=np.dtype([("score", "<i4"), ("status", "<i4"), ("prot_st", "<i4"),
                                             ("prot_en", "<i4"), ("nt_st", "<i4"), ("nt_en", "<i4"),
                                             ("n_cigar", "<u4"), ("exon_score", "<i4"), ("cigar", "<u8")]),
                        count=n)
    return buf.copy()


def mp_dp_batch_upload(ctx, pairs):
    pa = pairs if isinstance(pairs, _PairArray) else _PairArray(pairs)
    b = ctypes.c_void_p()
    _check(lib().mp_dp_batch_upload(ctx, pa.arr, pa.n, ctypes.byref(b)), "mp_dp_batch_upload")
    return b, pa.n


def mp_dp_batch_run(ctx, batch) -> None:
    _check(lib().mp_dp_batch_run(ctx, batch[0]), "mp_dp_batch_run")


def mp_dp_batch_sync(ctx) -> None:
    _check(lib().mp_dp_batch_sync(ctx), "mp_dp_batch_sync")


def mp_dp_batch_download(ctx, batch, raw: bool = False):
    n = batch[1]
    res = (mp_result * max(n, 1))()
    _check(lib().mp_dp_batch_download(ctx, batch[0], res), "mp_dp_batch_download")
    return _results(res, n, raw)


def mp_dp_batch_free(ctx, batch) -> None:
    lib().mp_dp_batch_free(ctx, batch[0])


def mp_dp_submit(ctx, pair) -> int:
    pa = _PairArray([pair])
    t = ctypes.c_uint64()
    rc = lib().mp_dp_submit(ctx, pa.arr, ctypes.byref(t))
    if rc == MP_EAGAIN:
        return -1
    _check(rc, "mp_dp_submit")
    return t.value


def mp_dp_poll(ctx, ticket: int, timeout_us: int = -1):
    """Result dict, or None while pending (MP_EPENDING / MP_ETIMEOUT)."""
    r = mp_result()
    rc = lib().mp_dp_poll(ctx, ticket, ctypes.byref(r), timeout_us)
    if rc in (MP_EPENDING, MP_ETIMEOUT):
        return None
    _check(rc, "mp_dp_poll")
    return result_dict(r)


def mp_dp_wait_any(ctx, timeout_us: int = -1):
    """(ticket, result dict) of the next finished request, or None."""
    r = mp_result()
    t = ctypes.c_uint64()
    rc = lib().mp_dp_wait_any(ctx, ctypes.byref(t), ctypes.byref(r), timeout_us)
    if rc in (MP_EPENDING, MP_ETIMEOUT):
        return None
    _check(rc, "mp_dp_wait_any")
    return t.value, result_dict(r)


def mp_dp_set_timing(ctx, enable: bool = True) -> None:
    _check(lib().mp_dp_set_timing(ctx, 1 if enable else 0), "mp_dp_set_timing")


def mp_dp_get_stats(ctx) -> dict:
    s = mp_dp_stats()
    _check(lib().mp_dp_get_stats(ctx, ctypes.byref(s)), "mp_dp_get_stats")
    return {k: getattr(s, k) for k, _ in mp_dp_stats._fields_}


def mp_dp_get_serve_stats(ctx, reset: bool = False) -> dict:
    s = mp_dp_serve_stats()
    _check(lib().mp_dp_get_serve_stats(ctx, ctypes.byref(s), 1 if reset else 0), "mp_dp_get_serve_stats")
    return {k: getattr(s, k) for k, _ in mp_dp_serve_stats._fields_}


def _tuning_dict(t) -> dict:
    return {k: getattr(t, k) for k in TUNING_KEYS}


def mp_dp_autotune(ctx, batch) -> tuple[dict, list[dict]]:
    """Time the candidate launch configurations on an uploaded batch; the
    fastest becomes the context's choice for the batch's shape class.
    Returns (best, every candidate with its time)."""
    best = mp_dp_tuning()
    tried = (mp_dp_tuning * 32)()
    n = ctypes.c_int(0)
    _check(lib().mp_dp_autotune(ctx, batch[0], ctypes.byref(best), tried, 32, ctypes.byref(n)), "mp_dp_autotune")
    return _tuning_dict(best), [_tuning_dict(tried[k]) for k in range(min(n.value, 32))]


def mp_dp_set_tuning(ctx, tuning: dict | None = None) -> None:
    """Fix the launch configuration (dict with TUNING_KEYS, missing keys 0);
    None returns to the tuned table and the defaults."""
    if tuning is None:
        _check(lib().mp_dp_set_tuning(ctx, None), "mp_dp_set_tuning")
        return
    t = mp_dp_tuning()
    for k, v in tuning.items():
        setattr(t, k, v)
    _check(lib().mp_dp_set_tuning(ctx, ctypes.byref(t)), "mp_dp_set_tuning")


def mp_dp_get_tuning(ctx, batch) -> dict:
    t = mp_dp_tuning()
    _check(lib().mp_dp_get_tuning(ctx, batch[0], ctypes.byref(t)), "mp_dp_get_tuning")
    return _tuning_dict(t)


def mp_dp_tuning_save(ctx, path: str) -> None:
    _check(lib().mp_dp_tuning_save(ctx, os.fsencode(path)), "mp_dp_tuning_save")


def mp_dp_tuning_load(ctx, path: str) -> None:
    _check(lib().mp_dp_tuning_load(ctx, os.fsencode(path)), "mp_dp_tuning_load")


def mp_dp_exon_rescore(ctx, pairs, results) -> list:
    """Pseudogene-aware scores of alignments (result dicts from aligning the
    same pairs with this context).  Returns the exon_score of each pair."""
    pa = pairs if isinstance(pairs, _PairArray) else _PairArray(pairs)
    res = (mp_result * max(pa.n, 1))()
    keep = []
    for k, r in enumerate(results):
        for key in ("score", "status", "prot_st", "prot_en", "nt_st", "nt_en"):
            setattr(res[k], key, int(r[key]))
        raw = (ctypes.c_uint32 * max(1, len(r["cigar_raw"])))(*r["cigar_raw"])
        keep.append(raw)
        res[k].n_cigar = len(r["cigar_raw"])
        res[k].cigar = ctypes.cast(raw, ctypes.POINTER(ctypes.c_uint32))
        res[k].exon_score = int(r["score"])
    _check(lib().mp_dp_exon_rescore(ctx, pa.arr, pa.n, res), "mp_dp_exon_rescore")
    return [res[k].exon_score for k in range(pa.n)]


def mp_dp_num_sms(ctx) -> int:
    return lib().mp_dp_num_sms(ctx)


def mp_dp_op_rates(device: int = 0) -> dict:
    """Measured integer ceilings of the device (see mp_dp_op_rates in mp_dp.h)."""
    r = mp_op_rates()
    _check(lib().mp_dp_op_rates(device, ctypes.byref(r)), "mp_dp_op_rates")
    return {name: getattr(r, name) for name, _ in mp_op_rates._fields_ if name != "reserved"}


def mp_dp_debug_h(ctx, batch, k: int, nt_len: int, prot_len: int) -> np.ndarray:
    """Test hook: the stored H matrix of pair k ((nt_len+1) x (prot_len+1),
    aligned orientation) after mp_dp_batch_run + mp_dp_batch_sync."""
    h = np.empty((nt_len + 1) * (prot_len + 1), dtype=np.int32)
    _check(lib().mp_dp_debug_h(ctx, batch[0], k, h.ctypes.data), "mp_dp_debug_h")
    return h.reshape(nt_len + 1, prot_len + 1)


def mp_dp_score_pair_noalloc(params, d_prot: int, prot_len: int, d_nt: int, nt_len: int, strand: int,
                             d_out: int, stream: int = 0) -> int:
    """Allocation-free scoring of one pair from device pointers (see the C
    header).  Returns the C return code; d_out receives 4 int32."""
    return lib().mp_dp_score_pair_noalloc(ctypes.byref(params) if params is not None else None,
                                          ctypes.c_void_p(d_prot), prot_len, ctypes.c_void_p(d_nt), nt_len,
                                          strand, ctypes.c_void_p(d_out), ctypes.c_void_p(stream))


def mp_dp_strerror(code: int) -> str:
    return lib().mp_dp_strerror(code).decode()


class Context:
    """Owning wrapper: ``with Context() as ctx: ctx.align(pairs)``."""

    def __init__(self, params: mp_dp_params | None = None, device: int = 0, **overrides):
        if params is None and overrides:
            params = mp_dp_default_params(**overrides)
        self.params = params
        self.ctx = mp_dp_init(params, device)

    def align(self, pairs, raw=False):
        return mp_dp_align_batch(self.ctx, pairs, raw)

    def close(self):
        if self.ctx:
            mp_dp_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------- seeding and chaining
class mp_chain(ctypes.Structure):
    _fields_ = [("strand", ctypes.c_int32), ("n_anchors", ctypes.c_int32), ("score", ctypes.c_int64),
                ("x_first", ctypes.c_int64), ("x_last", ctypes.c_int64),
                ("y_first", ctypes.c_int64), ("y_last", ctypes.c_int64)]


CHAIN_DTYPE = np.dtype([("strand", "<i4"), ("n_anchors", "<i4"), ("score", "<i8"), ("x_first", "<i8"),
                        ("x_last", "<i8"), ("y_first", "<i8"), ("y_last", "<i8")])
CHAIN2_DTYPE = np.dtype([("n_anchors", "<i4"), ("reserved", "<i4"), ("score", "<i8"), ("x_first", "<i8"),
                         ("x_last", "<i8"), ("y_first", "<i8"), ("y_last", "<i8")])


def mp_chain_refine(ctx, pairs):
    """Second chaining round of each (protein, region, strand) pair (a list
    of pairs, or a PairBatch): structured array of mp_chain2 records."""
    pa = pairs if isinstance(pairs, _PairArray) else _PairArray(pairs)
    out = np.zeros(max(pa.n, 1), dtype=CHAIN2_DTYPE)
    _check(lib().mp_chain_refine(ctx, ctypes.cast(pa.arr, ctypes.c_void_p), pa.n, out.ctypes.data),
           "mp_chain_refine")
    return out[:pa.n]


def mp_index_build(ctx, genome):
    """Index a genome (ASCII bytes, str or uint8 array) on the context's
    device; returns the index handle."""
    g = np.ascontiguousarray(np.frombuffer(genome.encode() if isinstance(genome, str) else genome, dtype=np.uint8))
    idx = ctypes.c_void_p()
    _check(lib().mp_index_build(ctx, g.ctypes.data_as(ctypes.c_char_p), len(g), ctypes.byref(idx)),
           "mp_index_build")
    return idx


def mp_index_download(ctx, idx):
    """(offsets uint64[2^24 + 1], entries uint32[]) of an index (test hook)."""
    n = ctypes.c_uint64()
    _check(lib().mp_index_download(ctx, idx, None, None, ctypes.byref(n)), "mp_index_download")
    off = np.zeros((1 << 24) + 1, dtype=np.uint64)
    ent = np.zeros(max(1, n.value), dtype=np.uint32)
    _check(lib().mp_index_download(ctx, idx, off.ctypes.data, ent.ctypes.data, ctypes.byref(n)), "mp_index_download")
    return off, ent[:n.value]


def mp_index_chain(ctx, idx, prot_buf, prot_off, prot_len, top: int):
    """Chains of every protein (proteins in one ASCII buffer at prot_off,
    prot_len): (chains structured array [n_prot, top], n_chains uint32[n_prot])."""
    pb = np.ascontiguousarray(np.frombuffer(prot_buf.encode() if isinstance(prot_buf, str) else prot_buf,
                                            dtype=np.uint8))
    po = np.ascontiguousarray(prot_off, dtype=np.uint64)
    pl = np.ascontiguousarray(prot_len, dtype=np.uint32)
    n = len(po)
    ch = np.zeros((max(n, 1), top), dtype=CHAIN_DTYPE)
    nch = np.zeros(max(n, 1), dtype=np.uint32)
    _check(lib().mp_index_chain(ctx, idx, pb.ctypes.data, po.ctypes.data, pl.ctypes.data, n, top, ch.ctypes.data,
                                nch.ctypes.data), "mp_index_chain")
    return ch[:n], nch[:n]


def mp_index_free(idx) -> None:
    lib().mp_index_free(idx)
