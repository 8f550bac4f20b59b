"""Helpers of the full-size parity tests: run the oracle over every pair of
a workload on all host cores (threads: the oracle's C calls release the
interpreter lock) and compare with the GPU results.

The full-matrix oracle (``oracle.align``) holds six int32 matrices per pair
(24 bytes per cell), so the pairs in flight are bounded by a byte budget;
the four-row fill (``oracle.score_end``) needs no such bound.
"""
from __future__ import annotations

import os
import threading
from concurrent.futures import ThreadPoolExecutor

KEYS = ("score", "prot_st", "prot_en", "nt_st", "nt_en", "cigar")


class _Budget:
    def __init__(self, cap: int):
        self.cap, self.used = cap, 0
        self.cv = threading.Condition()

    def take(self, n: int) -> int:
        n = min(n, self.cap)
        with self.cv:
            while self.used + n > self.cap:
                self.cv.wait()
            self.used += n
        return n

    def give(self, n: int) -> None:
        with self.cv:
            self.used -= n
            self.cv.notify_all()


def oracle_map(fn, pairs, idx, full: bool, mem_cap: int = 12 << 30):
    """fn(pair) for pairs[k], k in idx, on every host core, largest first;
    returns {k: result}.  full: fn holds the full matrices (bounded by
    mem_cap bytes in flight)."""
    idx = sorted(idx, key=lambda k: -pairs[k].cells)
    budget = _Budget(mem_cap)
    out = {}

    def one(k):
        p = pairs[k]
        need = budget.take(24 * (len(p.prot) + 1) * (len(p.nt) + 1)) if full else 0
        try:
            return k, fn(p)
        finally:
            if full:
                budget.give(need)

    with ThreadPoolExecutor(max_workers=os.cpu_count() or 1) as ex:
        for k, r in ex.map(one, idx):
            out[k] = r
    return out


def genome_end(res: dict, strand: int, n: int) -> int:
    """Row of the best cell in the aligned orientation from a result whose
    genome coordinates are on the forward strand."""
    return res["nt_en"] if strand > 0 else n - res["nt_st"]


def rescore_all(orc, pairs, got, skip=lambda p: False):
    """Every returned CIGAR rescored by the oracle's op-sum from its start:
    (k, rescored, reported) for each one that does not reproduce the score,
    protein end and genome end."""
    bad = []
    for k, (p, g) in enumerate(zip(pairs, got)):
        if skip(p) or g["score"] == 0:
            continue
        n = len(p.nt)
        st = g["nt_st"] if p.strand > 0 else n - g["nt_en"]
        sc, pe, te = orc.rescore(p.prot, p.nt, p.strand, g["prot_st"], st, g["cigar_raw"])
        if (sc, pe, te) != (g["score"], g["prot_en"], genome_end(g, p.strand, n)):
            bad.append((k, (sc, pe, te), (g["score"], g["prot_en"], genome_end(g, p.strand, n))))
    return bad
