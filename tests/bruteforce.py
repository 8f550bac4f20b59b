"""Path-enumeration statements of the spliced alignment score, used to pin
the oracle.

An alignment path is a start cell plus a sequence of operations, each with
an additive cost read off the transitions of Eq. 7 (Li 2022, "DP for
protein-to-genome alignment"):

  M      codon T[i+1..i+3] vs residue P[j+1]       (3, 1)  +s
  I k    k residues against no genome              (0, k)  -(q + e k)
  D k    k codons against no residue               (3k, 0) -(q + e k)
  F1/F2  1 or 2 nt for one residue ('$')           (1|2, 1) -f
  G1/G2  1 or 2 nt inserted ('+')                  (1|2, 0) -f
  N L    phase-0 intron T[i+1..i+L]                (L, 0)  -(r + d(i) + a(i+L))
  U L    phase-1: 1 nt, intron, 2 nt; one residue  (L+3, 1) -(r + d(i+1) + a(i+L+1))
  V L    phase-2: 2 nt, intron, 1 nt; one residue  (L+3, 1) -(r + d(i+2) + a(i+L+2))

U and V take every L >= -2: the literal recurrence lets the B and C states
close right after opening, and the enumeration mirrors that.  The split
codon of U and V is not scored (Methods, after Eq. 7).

Two enumerations are given: `all_paths` walks every operation sequence from
every start (exponential; tiny inputs only) and `segment_best` takes the
best score over operation sequences with a Bellman recursion over whole
operations (no I/D/A/B/C states).  Neither shares code with the oracle's DP.
"""
from __future__ import annotations

from functools import lru_cache

import oracle

NEG = float("-inf")
ORDER = {"M": 0, "I": 1, "D": 2, "F1": 3, "F2": 4, "G1": 5, "G2": 6, "N": 7, "U": 8, "V": 9}


def _simple_d(nt: str, x: int, p: int) -> int:
    """Simple GT-AG model: d(x) = 0 when the two bases after x (1-based
    x+1, x+2; 0-based x, x+1) spell GT, else p."""
    return 0 if 0 <= x and x + 2 <= len(nt) and nt[x:x + 2] == "GT" else p


def _simple_a(nt: str, x: int, p: int) -> int:
    """a(x) = 0 when the bases at 1-based x-1, x (0-based x-2, x-1) spell AG."""
    return 0 if 2 <= x <= len(nt) and nt[x - 2:x] == "AG" else p


class Problem:
    def __init__(self, prot: str, nt: str, q=11, e=1, f=23, r=29, stop=23, mat=None, splice_p=None, prof=None):
        """splice_p None: the final splice model (the oracle's tables, pinned
        on their own); an integer: the simple GT-AG model with that cost,
        written out here from its definition.  prof: position-specific costs
        of a profile query, rows j = 0..|P| of [21 substitution scores (the
        translated code's index, 20 = stop), gap open, gap extension]: a
        codon against position j scores prof[j][code]; an I run over
        residues j+1..j+k costs the open of j+1 and the extension of each;
        a D run of k codons after residue j costs the open and k extensions
        of position j."""
        self.prof = prof
        self.P = [oracle.AA.index(c) if c in oracle.AA else 21 for c in prot]
        self.T = ["ACGT".index(c) for c in nt]
        self.nt = nt
        self.n, self.m = len(nt), len(prot)
        self.q, self.e, self.f, self.r, self.stop = q, e, f, r, stop
        self.mat = oracle.blosum62_22() if mat is None else mat
        xs = range(-3, self.n + 4)
        if splice_p is None:
            self._d = [oracle.donor(nt, x) if nt else 30 for x in xs]
            self._a = [oracle.acceptor(nt, x) if nt else 30 for x in xs]
        else:
            self._d = [_simple_d(nt, x, splice_p) for x in xs]
            self._a = [_simple_a(nt, x, splice_p) for x in xs]

    def d(self, x):
        return self._d[x + 3]

    def a(self, x):
        return self._a[x + 3]

    def s(self, i, j):
        """Codon T[i+1..i+3] against residue P[j+1] (0-based T, P lists)."""
        aa = oracle.AA.index(oracle.translate_codon(self.T[i], self.T[i + 1], self.T[i + 2]))
        if self.prof is not None:
            return int(self.prof[j + 1][aa])
        if aa == 20:
            return -self.stop
        return int(self.mat[aa][self.P[j]])

    def gap_i(self, j, k):
        """Cost of an I run over residues j+1 .. j+k."""
        if self.prof is None:
            return self.q + self.e * k
        return int(self.prof[j + 1][21]) + sum(int(self.prof[t][22]) for t in range(j + 1, j + k + 1))

    def gap_d(self, j, k):
        """Cost of a D run of k codons after residue j."""
        if self.prof is None:
            return self.q + self.e * k
        return int(self.prof[j][21]) + int(self.prof[j][22]) * k

    def ops_from(self, i, j):
        """Every operation that can follow cell (i, j): (name, len, di, dj, cost)."""
        n, m = self.n, self.m
        q, e, f, r = self.q, self.e, self.f, self.r
        if i + 3 <= n and j + 1 <= m:
            yield ("M", 1, 3, 1, self.s(i, j))
        for k in range(1, m - j + 1):
            yield ("I", k, 0, k, -self.gap_i(j, k))
        for k in range(1, (n - i) // 3 + 1):
            yield ("D", k, 3 * k, 0, -self.gap_d(j, k))
        for L in (1, 2):
            if i + L <= n and j + 1 <= m:
                yield ("F%d" % L, L, L, 1, -f)
            if i + L <= n:
                yield ("G%d" % L, L, L, 0, -f)
        for L in range(1, n - i + 1):
            yield ("N", L, L, 0, -(r + self.d(i) + self.a(i + L)))
        if j + 1 <= m:
            for L in range(-2, n - i - 2):
                yield ("U", L, L + 3, 1, -(r + self.d(i + 1) + self.a(i + L + 1)))
                yield ("V", L, L + 3, 1, -(r + self.d(i + 2) + self.a(i + L + 2)))


def best_table(pb: Problem, mode: str = "local"):
    """best[i][j]: the best score of a path ending at cell (i, j), by a
    Bellman recursion over whole operations.  "local": paths start at any
    cell (the empty path scores 0, so no entry is below 0); "global" and
    "extend": paths start at (0, 0), unreachable cells stay at -inf."""
    n, m = pb.n, pb.m
    if mode == "local":
        best = [[0] * (m + 1) for _ in range(n + 1)]
    else:
        best = [[NEG] * (m + 1) for _ in range(n + 1)]
        best[0][0] = 0
    # process cells in order of i, then j (every op advances i or j)
    for i in range(n + 1):
        for j in range(m + 1):
            b = best[i][j]
            if b == NEG:
                continue
            for _, _, di, dj, c in pb.ops_from(i, j):
                if b + c > best[i + di][j + dj]:
                    best[i + di][j + dj] = b + c
    return best


def segment_best(pb: Problem) -> int:
    """Best local score: max over start cells and operation sequences."""
    return max(max(row) for row in best_table(pb, "local"))


def anchored_best(pb: Problem, mode: str) -> int:
    """Best score of a path from cell (0, 0): ending at (n, m) ("global") or
    anywhere, the empty path included ("extend")."""
    best = best_table(pb, mode)
    if mode == "global":
        return best[pb.n][pb.m]
    return max(max(row) for row in best)


def all_paths(pb: Problem, limit: int = 2_000_000):
    """Every (start, ops, end, score) path, by exhaustive depth-first walk."""
    out = []

    def walk(si, sj, i, j, ops, sc):
        out.append((si, sj, tuple(ops), i, j, sc))
        if len(out) > limit:
            raise RuntimeError("too many paths")
        for name, L, di, dj, c in pb.ops_from(i, j):
            ops.append((name, L))
            walk(si, sj, i + di, j + dj, ops, sc + c)
            ops.pop()

    for si in range(pb.n + 1):
        for sj in range(pb.m + 1):
            walk(si, sj, si, sj, [], 0)
    return out


def anchored_paths(pb: Problem, limit: int = 5_000_000):
    """Every path from cell (0, 0), by exhaustive depth-first walk:
    (ops, end i, end j, score)."""
    out = []

    def walk(i, j, ops, sc):
        out.append((tuple(ops), i, j, sc))
        if len(out) > limit:
            raise RuntimeError("too many paths")
        for name, L, di, dj, c in pb.ops_from(i, j):
            ops.append((name, L))
            walk(i + di, j + dj, ops, sc + c)
            ops.pop()

    walk(0, 0, [], 0)
    return out


def best_by_enumeration(paths) -> int:
    return max(max(p[5] for p in paths), 0)


def tie_rule_choice(paths):
    """Among optimal paths, pick the one the stated tie rules select:
    the end cell with the smallest i then j; then, reading the operations
    backwards from the end, stopping (restart) before any operation, and
    otherwise the earliest term of Eq. 7's printed order, with the shorter
    run first inside I, D and intron runs (open wins over extend)."""
    best = best_by_enumeration(paths)
    if best <= 0:
        return None
    opt = [p for p in paths if p[5] == best]
    ei, ej = min((p[3], p[4]) for p in opt)
    opt = [p for p in opt if (p[3], p[4]) == (ei, ej)]

    def key(p):
        return tuple((ORDER[name], L) for name, L in reversed(p[2]))

    return min(opt, key=key)


def to_cigar(ops):
    """Operation tuple -> oracle CIGAR [(letter, len)] with merged M runs."""
    out = []
    for name, L in ops:
        letter = name[0]
        if letter == "M" and out and out[-1][0] == "M":
            out[-1] = ("M", out[-1][1] + 1)
        else:
            out.append((letter, L))
    return out
