"""CPU oracle for the spliced protein-to-genome DP (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its Python binding) never touches it.

The arithmetic lives in ``oracle.c`` (plain C, int32, full matrices): Eq. 7 of
Li 2022 ("DP for protein-to-genome alignment") in local mode with the final
splice model of the "Splice models" section.  This module only marshals
arguments through ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_SRC = os.path.join(_HERE, "oracle.c")
_SRCS = [_SRC, os.path.join(_HERE, "chain.c")]

AA = "ARNDCQEGHILKMFPSTWYV*X"
OP_NAMES = "MIDFGNUV"

# BLOSUM62 (Henikoff & Henikoff 1992), rows/cols in the order of AA[:20].
_BLOSUM62_ROWS = """
 4 -1 -2 -2  0 -1 -1  0 -2 -1 -1 -1 -1 -2 -1  1  0 -3 -2  0
-1  5  0 -2 -3  1  0 -2  0 -3 -2  2 -1 -3 -2 -1 -1 -3 -2 -3
-2  0  6  1 -3  0  0  0  1 -3 -3  0 -2 -3 -2  1  0 -4 -2 -3
-2 -2  1  6 -3  0  2 -1 -1 -3 -4 -1 -3 -3 -1  0 -1 -4 -3 -3
 0 -3 -3 -3  9 -3 -4 -3 -3 -1 -1 -3 -1 -2 -3 -1 -1 -2 -2 -1
-1  1  0  0 -3  5  2 -2  0 -3 -2  1  0 -3 -1  0 -1 -2 -1 -2
-1  0  0  2 -4  2  5 -2  0 -3 -3  1 -2 -3 -1  0 -1 -3 -2 -2
 0 -2  0 -1 -3 -2 -2  6 -2 -4 -4 -2 -3 -3 -2  0 -2 -2 -3 -3
-2  0  1 -1 -3  0  0 -2  8 -3 -3 -1 -2 -1 -2 -1 -2 -2  2 -3
-1 -3 -3 -3 -1 -3 -3 -4 -3  4  2 -3  1  0 -3 -2 -1 -3 -1  3
-1 -2 -3 -4 -1 -2 -3 -4 -3  2  4 -2  2  0 -3 -2 -1 -2 -1  1
-1  2  0 -1 -3  1  1 -2 -1 -3 -2  5 -1 -3 -1  0 -1 -3 -2 -2
-1 -1 -2 -3 -1  0 -2 -3 -2  1  2 -1  5  0 -2 -1 -1 -1 -1  1
-2 -3 -3 -3 -2 -3 -3 -3 -1  0  0 -3  0  6 -4 -2 -2  1  3 -1
-1 -2 -2 -1 -3 -1 -1 -2 -2 -3 -3 -1 -2 -4  7 -1 -1 -4 -3 -2
 1 -1  1  0 -1  0  0  0 -1 -2 -2  0 -1 -2 -1  4  1 -3 -2 -2
 0 -1  0 -1 -1 -1 -1 -2 -2 -1 -1 -1 -1 -2 -1  1  5 -2 -2  0
-3 -3 -4 -4 -2 -2 -3 -2 -2 -3 -2 -3 -1  1 -4 -3 -2 11  2 -3
-2 -2 -2 -3 -2 -1 -2 -3  2 -1 -1 -2 -1  3 -3 -2 -2  2  7 -1
 0 -3 -3 -3 -1 -2 -2 -3 -3  3  1 -2  1 -1 -2 -2  0 -3 -1  4
"""


def blosum62_22() -> np.ndarray:
    """22x22 int matrix in AA order: BLOSUM62 for the 20 amino acids,
    -4 against a protein '*' (BLOSUM62's stop column), -1 against X."""
    m = np.full((22, 22), -1, dtype=np.int32)
    rows = [list(map(int, r.split())) for r in _BLOSUM62_ROWS.strip().splitlines()]
    m[:20, :20] = np.array(rows, dtype=np.int32)
    m[:20, 20] = -4
    m[20, :20] = -4
    m[20, 20] = 1
    return m


class Params(ctypes.Structure):
    _fields_ = [("q", ctypes.c_int32), ("e", ctypes.c_int32), ("f", ctypes.c_int32),
                ("r", ctypes.c_int32), ("stop", ctypes.c_int32),
                ("mat", (ctypes.c_int32 * 22) * 22),
                ("splice_model", ctypes.c_int32), ("splice_p", ctypes.c_int32), ("mode", ctypes.c_int32),
                ("prof", ctypes.POINTER(ctypes.c_int32))]


class Result(ctypes.Structure):
    _fields_ = [("score", ctypes.c_int32), ("status", ctypes.c_int32),
                ("prot_st", ctypes.c_int32), ("prot_en", ctypes.c_int32),
                ("nt_st", ctypes.c_int32), ("nt_en", ctypes.c_int32),
                ("n_cigar", ctypes.c_int32)]


# Default penalties (the paper prints none; see the design notes).
DEFAULTS = dict(q=11, e=1, f=23, r=29, stop=23)


PROF_W = 23     # ints per position of a profile: 21 substitution scores, gap open, gap extension


def make_params(q=None, e=None, f=None, r=None, stop=None, mat=None, splice_model=0, splice_p=30,
                mode=0, prof=None) -> Params:
    """Scoring parameters; splice_model 0 is the final model, 1 the simple
    GT-AG model with cost splice_p; mode 0 local, 1 global (cell (0, 0) to
    (|T|, |P|)), 2 extension (from (0, 0), ending anywhere).  prof: None, or
    the position-specific costs of a profile query, an int array of shape
    (|P| + 1, 23): row j (j >= 1) holds the score of each translated code
    (ORC_AA order, 20 = stop codon) against residue position j, then the gap
    open and extension costs of column j (row 0: codons before the first
    residue)."""
    p = Params()
    if prof is not None:
        arr = np.ascontiguousarray(prof, dtype=np.int32)
        assert arr.ndim == 2 and arr.shape[1] == PROF_W
        p._prof_keep = arr                      # keeps the buffer alive with the struct
        p.prof = arr.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    p.splice_model, p.splice_p, p.mode = splice_model, splice_p, mode
    d = dict(DEFAULTS)
    for k, v in (("q", q), ("e", e), ("f", f), ("r", r), ("stop", stop)):
        if v is not None:
            d[k] = v
    p.q, p.e, p.f, p.r, p.stop = d["q"], d["e"], d["f"], d["r"], d["stop"]
    m = blosum62_22() if mat is None else np.asarray(mat, dtype=np.int32)
    for a in range(22):
        for b in range(22):
            p.mat[a][b] = int(m[a, b])
    return p


_lock = threading.Lock()
_lib = None


def build_oracle(force: bool = False) -> str:
    """Compile oracle.c into a shared library (plain gcc, -O2)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < max(os.path.getmtime(f) for f in _SRCS):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-shared", "-fPIC", "-o", tmp] + _SRCS + ["-lm"])
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build_oracle()
            L = ctypes.CDLL(_SO)
            L.orc_align.argtypes = [ctypes.POINTER(Params), ctypes.c_char_p, ctypes.c_int32,
                                    ctypes.c_char_p, ctypes.c_int32, ctypes.c_int32,
                                    ctypes.POINTER(Result), ctypes.POINTER(ctypes.c_uint32),
                                    ctypes.c_int32]
            L.orc_align.restype = ctypes.c_int
            L.orc_rescore.argtypes = [ctypes.POINTER(Params), ctypes.c_char_p, ctypes.c_int32,
                                      ctypes.c_char_p, ctypes.c_int32, ctypes.c_int32,
                                      ctypes.c_int32, ctypes.c_int32,
                                      ctypes.POINTER(ctypes.c_uint32), ctypes.c_int32,
                                      ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]
            L.orc_rescore.restype = ctypes.c_int32
            L.orc_translate.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int]
            L.orc_translate.restype = ctypes.c_int
            L.orc_donor.argtypes = [ctypes.POINTER(ctypes.c_int8), ctypes.c_int, ctypes.c_int]
            L.orc_donor_simple.argtypes = [ctypes.POINTER(ctypes.c_int8), ctypes.c_int, ctypes.c_int, ctypes.c_int]
            L.orc_acceptor_simple.argtypes = [ctypes.POINTER(ctypes.c_int8), ctypes.c_int, ctypes.c_int,
                                              ctypes.c_int]
            L.orc_donor.restype = ctypes.c_int
            L.orc_acceptor.argtypes = [ctypes.POINTER(ctypes.c_int8), ctypes.c_int, ctypes.c_int]
            L.orc_acceptor.restype = ctypes.c_int
            L.orc_aa_code.argtypes = [ctypes.c_int]
            L.orc_aa_code.restype = ctypes.c_int
            L.orc_nt_code.argtypes = [ctypes.c_int]
            L.orc_nt_code.restype = ctypes.c_int
            L.orc_score_end.argtypes = [ctypes.POINTER(Params), ctypes.c_char_p, ctypes.c_int32,
                                        ctypes.c_char_p, ctypes.c_int32, ctypes.c_int32,
                                        ctypes.POINTER(Result)]
            L.orc_score_end.restype = ctypes.c_int
            _lib = L
    return _lib


NEG_INF = -(2 ** 31) // 4


def align(prot: str, nt: str, strand: int = 1, params: Params | None = None):
    """Run the oracle on one pair.  Returns a dict with score, status,
    coordinates (0-based half-open; nt on the input's forward strand) and the
    CIGAR as a list of (op letter, length)."""
    L = lib()
    p = params if params is not None else make_params()
    pb = prot.encode() if isinstance(prot, str) else bytes(prot)
    tb = nt.encode() if isinstance(nt, str) else bytes(nt)
    cap = len(pb) + len(tb) + 2
    cig = (ctypes.c_uint32 * cap)()
    res = Result()
    rc = L.orc_align(ctypes.byref(p), pb, len(pb), tb, len(tb), int(strand), ctypes.byref(res), cig, cap)
    if rc != 0:
        raise ValueError("oracle rejected the input")
    ops = [(OP_NAMES[cig[k] & 0xF], cig[k] >> 4) for k in range(res.n_cigar)]
    raw = [cig[k] for k in range(res.n_cigar)]
    return dict(score=res.score, status=res.status, prot_st=res.prot_st, prot_en=res.prot_en,
                nt_st=res.nt_st, nt_en=res.nt_en, cigar=ops, cigar_raw=raw)


def score_end(prot: str, nt: str, strand: int = 1, params: Params | None = None):
    """Score and end cell of the best alignment with four rows of memory per
    state (for pairs too large for the full matrices of ``align``).  Returns
    a dict with score, prot_en and the genome end of the best cell: nt_en on
    strand +1, nt_st on strand -1 (the other genome coordinate is None)."""
    L = lib()
    p = params if params is not None else make_params()
    pb = prot.encode() if isinstance(prot, str) else bytes(prot)
    tb = nt.encode() if isinstance(nt, str) else bytes(nt)
    res = Result()
    if L.orc_score_end(ctypes.byref(p), pb, len(pb), tb, len(tb), int(strand), ctypes.byref(res)) != 0:
        raise ValueError("oracle rejected the input")
    return dict(score=res.score, prot_en=res.prot_en,
                nt_en=res.nt_en if strand > 0 else None, nt_st=res.nt_st if strand < 0 else None)


def rescore(prot: str, nt: str, strand: int, prot_st: int, nt_st_aligned: int, cigar_raw,
            params: Params | None = None):
    """Op-sum score of a CIGAR from a start cell (aligned orientation).
    Returns (score, prot_en, nt_en_aligned); score is NEG_INF if invalid."""
    L = lib()
    p = params if params is not None else make_params()
    pb = prot.encode() if isinstance(prot, str) else bytes(prot)
    tb = nt.encode() if isinstance(nt, str) else bytes(nt)
    arr = (ctypes.c_uint32 * max(1, len(cigar_raw)))(*cigar_raw)
    pe = ctypes.c_int32()
    te = ctypes.c_int32()
    s = L.orc_rescore(ctypes.byref(p), pb, len(pb), tb, len(tb), int(strand), int(prot_st),
                      int(nt_st_aligned), arr, len(cigar_raw), ctypes.byref(pe), ctypes.byref(te))
    return s, pe.value, te.value


def exon_sequence(nt: str, strand: int, res: dict) -> str:
    """The genome an alignment covers with its introns cut out, in the
    aligned orientation (Methods, "Avoiding pseudogenes": the translated
    coding region without introns).  Codons (M, D) and frameshift bases
    (F, G) are kept; an N intron is dropped; a U or V intron is dropped but
    the split codon's 3 bases around it are kept."""
    t = nt.upper() if strand > 0 else revcomp(nt)
    i = res["nt_st"] if strand > 0 else len(nt) - res["nt_en"]
    out = []
    for op, n in res["cigar"]:
        if op in "MD":
            out.append(t[i:i + 3 * n]); i += 3 * n
        elif op in "FG":
            out.append(t[i:i + n]); i += n
        elif op == "N":
            i += n
        elif op == "U":
            out.append(t[i:i + 1]); out.append(t[i + 1 + n:i + 3 + n]); i += n + 3
        elif op == "V":
            out.append(t[i:i + 2]); out.append(t[i + 2 + n:i + 3 + n]); i += n + 3
    return "".join(out)


def exon_score(prot: str, nt: str, strand: int = 1, params: Params | None = None, res: dict | None = None) -> int:
    """Pseudogene-aware score (Methods, "Avoiding pseudogenes"): the local DP
    score of the protein against the alignment's coding region without
    introns, less the intron cost r when the alignment has no intron.  An
    alignment of score 0 (none) keeps 0."""
    p = params if params is not None else make_params()
    r = res if res is not None else align(prot, nt, strand, p)
    if r["score"] <= 0 or not r["cigar"]:
        return r["score"]
    s2 = align(prot, exon_sequence(nt, strand, r), 1, p)["score"]
    single = not any(op in "NUV" for op, _ in r["cigar"])
    return s2 - (p.r if single else 0)


def profile_of(prot: str, params: Params | None = None) -> np.ndarray:
    """The profile that reproduces the position-independent scoring of
    `params` for protein `prot`: row j holds mat[c][P[j]] (and -stop for the
    stop codon) and the global q and e."""
    p = params if params is not None else make_params()
    m = len(prot)
    out = np.zeros((m + 1, PROF_W), dtype=np.int32)
    for j in range(1, m + 1):
        pc = lib().orc_aa_code(ord(prot[j - 1]))
        for c in range(20):
            out[j, c] = p.mat[c][pc]
        out[j, 20] = -p.stop
    out[:, 21] = p.q
    out[:, 22] = p.e
    return out


def encode_cigar(ops) -> list:
    """[(letter, len), ...] -> packed op words (len << 4 | code)."""
    return [(int(n) << 4) | OP_NAMES.index(c) for c, n in ops]


def cigar_str(ops) -> str:
    return "".join(f"{n}{c}" for c, n in ops)


def translate_codon(b1: int, b2: int, b3: int) -> str:
    return AA[lib().orc_translate(b1, b2, b3)]


def donor(nt: str, x: int) -> int:
    """d(x) of the final splice model; x is 1-based as in the paper."""
    codes = [0] + ["ACGT".index(c) for c in nt.upper()]
    arr = (ctypes.c_int8 * len(codes))(*codes)
    return lib().orc_donor(arr, len(nt), x)


def acceptor(nt: str, x: int) -> int:
    codes = [0] + ["ACGT".index(c) for c in nt.upper()]
    arr = (ctypes.c_int8 * len(codes))(*codes)
    return lib().orc_acceptor(arr, len(nt), x)


def fill_h(prot: str, nt: str, strand: int = 1, params: Params | None = None) -> np.ndarray:
    """The oracle's H matrix, (|T|+1) x (|P|+1), aligned orientation."""
    L = lib()
    p = params if params is not None else make_params()
    pb = prot.encode()
    tb = nt.encode()
    out = np.zeros((len(tb) + 1) * (len(pb) + 1), dtype=np.int32)
    L.orc_fill_h.argtypes = [ctypes.POINTER(Params), ctypes.c_char_p, ctypes.c_int32, ctypes.c_char_p,
                             ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p]
    if L.orc_fill_h(ctypes.byref(p), pb, len(pb), tb, len(tb), int(strand), out.ctypes.data) != 0:
        raise ValueError("oracle rejected the input")
    return out.reshape(len(tb) + 1, len(pb) + 1)


def donor_simple(nt: str, x: int, p: int) -> int:
    """d(x) of the simple GT-AG model with cost p; x is 1-based."""
    codes = [0] + ["ACGT".index(c) for c in nt.upper()]
    arr = (ctypes.c_int8 * len(codes))(*codes)
    return lib().orc_donor_simple(arr, len(nt), x, p)


def acceptor_simple(nt: str, x: int, p: int) -> int:
    codes = [0] + ["ACGT".index(c) for c in nt.upper()]
    arr = (ctypes.c_int8 * len(codes))(*codes)
    return lib().orc_acceptor_simple(arr, len(nt), x, p)


def revcomp(s: str) -> str:
    return s.upper().translate(str.maketrans("ACGT", "TGCA"))[::-1]


# ---------------------------------------------------------- seeding and chaining
class Chain(ctypes.Structure):
    _fields_ = [("strand", ctypes.c_int32), ("n_anchors", ctypes.c_int32), ("score", ctypes.c_int64),
                ("x_first", ctypes.c_int64), ("x_last", ctypes.c_int64),
                ("y_first", ctypes.c_int64), ("y_last", ctypes.c_int64)]


class Chain2(ctypes.Structure):
    _fields_ = [("n_anchors", ctypes.c_int32), ("reserved", ctypes.c_int32), ("score", ctypes.c_int64),
                ("x_first", ctypes.c_int64), ("x_last", ctypes.c_int64),
                ("y_first", ctypes.c_int64), ("y_last", ctypes.c_int64)]


CHAIN_K = 6
REFINE_K = 5                   # k-mer length of the second chaining round
CHAIN_SCALE = 65536


def _chain_lib():
    L = lib()
    if not hasattr(L, "_chain_ready"):
        L.orc_phi.argtypes = [ctypes.c_int]
        L.orc_phi.restype = ctypes.c_int
        L.orc_psi.argtypes = [ctypes.c_uint64, ctypes.c_int]
        L.orc_psi.restype = ctypes.c_uint64
        L.orc_index.argtypes = [ctypes.c_char_p, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
        L.orc_index.restype = ctypes.c_int64
        L.orc_gap.argtypes = [ctypes.c_int64, ctypes.c_int64]
        L.orc_gap.restype = ctypes.c_int64
        L.orc_gap_penalty.argtypes = [ctypes.c_int64]
        L.orc_gap_penalty.restype = ctypes.c_int64
        L.orc_anchors.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_char_p, ctypes.c_int64,
                                  ctypes.c_void_p, ctypes.c_int64]
        L.orc_anchors.restype = ctypes.c_int64
        L.orc_chain_anchors.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                        ctypes.POINTER(Chain), ctypes.c_void_p]
        L.orc_chain_anchors.restype = ctypes.c_int
        L.orc_refine_anchors.argtypes = [ctypes.c_char_p, ctypes.c_int64, ctypes.c_char_p, ctypes.c_int64,
                                         ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_int64]
        L.orc_refine_anchors.restype = ctypes.c_int64
        L.orc_refine_chain.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.POINTER(Chain2),
                                       ctypes.c_void_p]
        L.orc_refine_chain.restype = ctypes.c_int
        L._chain_ready = True
    return L


def phi(ch: str) -> int:
    """Reduced-alphabet code of an amino-acid letter (Methods, "Reduced alphabet")."""
    return _chain_lib().orc_phi(ord(ch))


def psi(key: int, bits: int) -> int:
    """The invertible k-mer hash over [0, 2^bits)."""
    return _chain_lib().orc_psi(key, bits)


def build_index(genome, k: int = CHAIN_K):
    """The k-mer index of a genome (ASCII str or bytes): (offsets, positions)
    as a CSR table over all 2^(4k) hash values; each position is
    strand << 31 | bin (bin = floor(x / 256), x on the strand's own
    coordinates)."""
    L = _chain_lib()
    g = genome.encode() if isinstance(genome, str) else bytes(genome)
    n = L.orc_index(g, len(g), k, None, None)
    if n < 0:
        raise MemoryError("oracle index")
    offsets = np.zeros((1 << (4 * k)) + 1, dtype=np.uint64)
    positions = np.zeros(max(n, 1), dtype=np.uint32)
    L.orc_index(g, len(g), k, offsets.ctypes.data, positions.ctypes.data)
    return offsets, positions[:n]


def anchors(offsets, positions, prot: str, k: int = CHAIN_K) -> np.ndarray:
    """The anchors (strand, x bin, y residue) of a protein against an index."""
    L = _chain_lib()
    pb = prot.encode() if isinstance(prot, str) else bytes(prot)
    n = L.orc_anchors(offsets.ctypes.data, positions.ctypes.data, k, pb, len(pb), None, 0)
    out = np.zeros((max(n, 1), 3), dtype=np.int64)
    L.orc_anchors(offsets.ctypes.data, positions.ctypes.data, k, pb, len(pb), out.ctypes.data, n)
    return out[:n]


def chain(anc, top: int, k: int = CHAIN_K):
    """Chain a protein's anchors (Eqs. 1-3 of "Chaining"): (chains, f) with
    the first `top` chains of at least two anchors as dicts (scores in
    units of 2^-16) and every anchor's chaining score in sorted order."""
    L = _chain_lib()
    anc = np.ascontiguousarray(anc, dtype=np.int64).reshape(-1, 3)
    n = len(anc)
    f = np.zeros(max(n, 1), dtype=np.int64)
    buf = (Chain * max(top, 1))()
    nc = L.orc_chain_anchors(anc.ctypes.data, n, k, top, buf, f.ctypes.data)
    if nc < 0:
        raise MemoryError("oracle chaining")
    keys = ("strand", "n_anchors", "score", "x_first", "x_last", "y_first", "y_last")
    return [{x: getattr(buf[t], x) for x in keys} for t in range(nc)], f[:n]


def gap(dx: int, dy: int) -> int:
    return _chain_lib().orc_gap(dx, dy)


def gap_penalty(g: int) -> int:
    """Eq. 3 in units of 2^-16, -1 for an infinite penalty."""
    return _chain_lib().orc_gap_penalty(g)


def refine_anchors(prot: str, nt: str, strand: int, k: int = REFINE_K) -> np.ndarray:
    """Second chaining round ("Chaining", last paragraph): every k-mer of the
    protein against every k-mer of the region's three frames on its aligned
    strand, as sorted (x, y) rows (x: base of the first codon, y: residue)."""
    L = _chain_lib()
    pb = prot.encode() if isinstance(prot, str) else bytes(prot)
    nb = nt.encode() if isinstance(nt, str) else bytes(nt)
    n = L.orc_refine_anchors(pb, len(pb), nb, len(nb), strand, k, None, 0)
    if n < 0:
        raise MemoryError("oracle anchors")
    out = np.zeros((max(n, 1), 2), dtype=np.int64)
    L.orc_refine_anchors(pb, len(pb), nb, len(nb), strand, k, out.ctypes.data, n)
    return out[:n]


def refine_chain(anc, k: int = REFINE_K):
    """The best chain of sorted (x, y) anchors with g' = 3 dy - dx and Eq. 3:
    (chain dict with n_anchors 0 if none, f of every anchor)."""
    L = _chain_lib()
    anc = np.ascontiguousarray(anc, dtype=np.int64).reshape(-1, 2)
    n = len(anc)
    f = np.zeros(max(n, 1), dtype=np.int64)
    c = Chain2()
    if L.orc_refine_chain(anc.ctypes.data, n, k, ctypes.byref(c), f.ctypes.data) < 0:
        raise MemoryError("oracle chaining")
    keys = ("n_anchors", "score", "x_first", "x_last", "y_first", "y_last")
    return {x: getattr(c, x) for x in keys}, f[:n]


def refine(prot: str, nt: str, strand: int, k: int = REFINE_K):
    """The pair's best second-round chain."""
    return refine_chain(refine_anchors(prot, nt, strand, k), k)[0]
