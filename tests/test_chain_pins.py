"""Pins for the seeding and chaining oracle (Li 2022, Methods: "Reduced
alphabet", "Indexing the genome", "Chaining", Eqs. 1-3).

The reduced alphabet is checked against the paper's table (a golden
fixture), the hash for invertibility, the index against a brute-force
enumeration written from the paper's description (string translation,
stop-free runs, k-mers), Eq. 1 and Eq. 3 against hand values and a
high-precision evaluation, and the chaining recurrence against the best
score over every chain enumerated one by one.
"""
import itertools
import math
import os
import random

import numpy as np
import pytest

import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
CODE_ACGT = "KNKNTTTTRSRSIIMIQHQHPPPPRRRRLLLLEDEDAAAAGGGGVVVV*Y*YSSSS*CWCLFLF"


def _groups():
    out = {}
    for line in open(os.path.join(GOLDEN, "reduced_alphabet.txt")):
        if line.startswith("#") or not line.strip():
            continue
        letters, v = line.split()
        for c in letters:
            out[c] = int(v)
    return out


def test_reduced_alphabet_matches_paper(orc):
    g = _groups()
    for c, v in g.items():
        assert orc.phi(c) == v, c
    for c in "BZUJO":                     # outside the 20 amino acids: X
        assert orc.phi(c) == g["X"]
    assert orc.phi("a") == g["A"]


@pytest.mark.parametrize("bits", [12, 16, 20])
def test_hash_is_invertible(orc, bits):
    vals = {orc.psi(x, bits) for x in range(1 << bits)}
    assert len(vals) == 1 << bits and max(vals) < 1 << bits


def test_hash_samples_about_half(orc):
    rng = random.Random(5)
    even = sum(1 for _ in range(20000) if orc.psi(rng.randrange(1 << 24), 24) % 2 == 0)
    assert 9500 < even < 10500


def _translate(s):
    return "".join(CODE_ACGT["ACGT".index(s[t]) * 16 + "ACGT".index(s[t + 1]) * 4 + "ACGT".index(s[t + 2])]
                   for t in range(0, len(s) - 2, 3))


def _brute_index(orc, genome, k=6):
    """(hash, strand << 31 | bin) of every sampled k-mer inside a stop-free
    run of at least 30 codons, in every frame of both strands."""
    g = _groups()
    comp = {"A": "T", "C": "G", "G": "C", "T": "A"}
    out = []
    for strand, seq in ((0, genome), (1, "".join(comp[c] for c in reversed(genome)))):
        for frame in range(3):
            aa = _translate(seq[frame:frame + 3 * ((len(seq) - frame) // 3)])
            for run in __import__("re").finditer(r"[^*]+", aa):
                a, b = run.start(), run.end()
                if b - a < 30:
                    continue
                for t in range(a, b - k + 1):
                    key = 0
                    for c in aa[t:t + k]:
                        key = key * 16 + g.get(c, g["X"])
                    h = orc.psi(key, 4 * k)
                    if h % 2 == 0:
                        out.append((h, (strand << 31) | ((frame + 3 * t) // 256)))
    return sorted(out)


def test_index_against_brute_force(orc):
    rng = np.random.default_rng(7)
    parts = [synth.random_dna(rng, 3000, 0.4)]
    for _ in range(4):                       # planted coding sequences: long open reading frames
        prot = synth.random_protein(rng, int(rng.integers(40, 120)))
        parts.append(synth.reverse_translate(rng, prot))
        parts.append(synth.random_dna(rng, int(rng.integers(100, 800)), 0.4))
    parts.append(synth.revcomp(synth.reverse_translate(rng, synth.random_protein(rng, 90))))
    genome = "".join(parts)
    off, pos = orc.build_index(genome)
    got = sorted((h, int(p)) for h in np.flatnonzero(np.diff(off)) for p in pos[off[h]:off[h + 1]])
    assert got == _brute_index(orc, genome)
    # positions within each hash value are ascending
    for h in np.flatnonzero(np.diff(off)):
        seg = pos[off[h]:off[h + 1]]
        assert (np.diff(seg.astype(np.int64)) >= 0).all()
    assert any(p >> 31 for _, p in got) and any(not p >> 31 for _, p in got)


def test_open_reading_frame_threshold(orc):
    """A stop-free run of 29 codons yields no entry; one of 30 yields every
    sampled k-mer of it (25 starts), at the bin of each k-mer's first base."""
    rng = np.random.default_rng(8)
    stops = "TAA"
    for L, want_any in ((29, False), (30, True)):
        prot = "".join(rng.choice(list("ACDEFGHIKLMNPQRSTVWY"), size=L))
        orf = synth.reverse_translate(rng, prot)
        # stops on every frame of both strands around it: TAA TAA TAA and TTA (revcomp of TAA)
        g = "TAATAATTA" + stops + orf + "TAATTATTA" + "TTATTATTA"
        off, pos = orc.build_index(g)
        entries = [(h, int(p)) for h in np.flatnonzero(np.diff(off)) for p in pos[off[h]:off[h + 1]]]
        fwd = [e for e in entries if not e[1] >> 31]
        assert bool(fwd) == want_any, (L, len(fwd))
        assert len(fwd) <= 25


def test_gap_eq1_hand_values(orc):
    # 3 dy within 256 (dx - 1) .. 256 (dx + 1): no certain gap
    assert orc.gap(1, 0) == 0 and orc.gap(1, 170) == 0 and orc.gap(2, 86) == 0 and orc.gap(2, 256) == 0
    assert orc.gap(2, 85) == 255 - 256 and orc.gap(2, 257) == 771 - 768
    assert orc.gap(0, 85) == 0 and orc.gap(0, 86) == 258 - 256
    # genome gap larger than the protein's: negative (an intron, say)
    assert orc.gap(10, 10) == 30 - 256 * 9
    # protein gap larger than the genome's: positive
    assert orc.gap(1, 200) == 600 - 512


def test_gap_penalty_eq3(orc):
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    S = 65536
    assert orc.gap_penalty(0) == 0
    assert orc.gap_penalty(200000) == -1 and orc.gap_penalty(-200000) == -1
    for g in (1, 2, 3, 7, 15, 100, 1023, 1024, 4097, 65535, 131071, 199999):
        lin = (g * S) // 3
        lg = int(mpmath.floor(mpmath.mpf(S) * mpmath.mpf("0.75") * mpmath.log(g + 1, 2)))
        assert orc.gap_penalty(g) == lin + lg, g
        assert orc.gap_penalty(-g) == min(lin, lg), g


def test_log_term_is_robust_to_rounding(orc):
    """floor(2^16 * 0.75 * log2(v)) for every v up to G: the value in
    double precision is exact for powers of two and at least 1e-6 from an
    integer otherwise, so any log2 within an ulp (host or device) gives the
    same integer."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 30
    for v in list(range(2, 5000)) + list(range(5000, 200001, 97)) + [151189]:
        t = mpmath.mpf(49152) * mpmath.log(v, 2)
        fr = float(t - mpmath.floor(t))
        if v & (v - 1):
            assert min(fr, 1 - fr) > 1e-6, v
        assert math.floor(49152.0 * math.log2(v)) == int(mpmath.floor(t)), v


def _pen(orc, a, b):
    p = orc.gap_penalty(orc.gap(b[1] - a[1], b[2] - a[2]))
    return None if p < 0 else p


def test_chaining_against_enumeration(orc):
    """f of every anchor equals the best k + sum(alpha - gamma) over every
    chain (x non-decreasing, y increasing, finite gamma) ending there,
    enumerated one by one; anchors on two strands never chain."""
    rng = random.Random(9)
    S, k = orc.CHAIN_SCALE, orc.CHAIN_K
    for _ in range(60):
        n = rng.randint(1, 8)
        anc = [(rng.randint(0, 1), rng.randint(0, 40), rng.randint(0, 60)) for _ in range(n)]
        chains, f = orc.chain(anc, 10)
        srt = sorted(anc)
        best = []
        for j, b in enumerate(srt):
            v = k * S
            for r in range(1, j + 1):
                for sub in itertools.combinations(range(j), r):
                    seq = [srt[t] for t in sub] + [b]
                    tot, ok = k * S, True
                    for a1, a2 in zip(seq, seq[1:]):
                        if a1[0] != a2[0] or a1[1] > a2[1] or a1[2] >= a2[2]:
                            ok = False
                            break
                        p = _pen(orc, a1, a2)
                        if p is None:
                            ok = False
                            break
                        tot += min(a2[2] - a1[2], k) * S - p
                    if ok:
                        v = max(v, tot)
            best.append(v)
        assert list(f) == best, (anc, list(f), best)
        for c in chains:
            assert c["n_anchors"] >= 2 and c["score"] > 0


def test_chain_across_an_intron_and_not_beyond_G(orc):
    """Anchors of two exons on one diagonal each, 2 kb apart: one chain of
    all of them (the log term makes the intron cheap); 300 kb apart: two."""
    for gap_bp, n_chains in ((2000, 1), (300000, 2)):
        anc = []
        for t in range(12):               # exon 1: residues 0..66, genome 0..200
            anc.append((0, (3 * 6 * t) // 256, 6 * t))
        x0 = (3 * 72 + gap_bp) // 256
        for t in range(12):               # exon 2 after the intron
            anc.append((0, x0 + (3 * 6 * t) // 256, 72 + 6 * t))
        chains, _ = orc.chain(anc, 5)
        assert len(chains) == n_chains, (gap_bp, chains)
        if n_chains == 1:
            assert chains[0]["n_anchors"] == 24


def test_protein_anchors_and_chains_find_a_planted_gene(orc):
    """A protein planted with two introns in a random genome: its best chain
    is on the planted strand and spans the planted gene's bins."""
    rng = np.random.default_rng(11)
    prot = synth.random_protein(rng, 300)
    gene, _ = synth.gen.plant_gene(rng, prot, 0.1, 0, [900, 1500], 0, 0, 0.4)
    left = synth.random_dna(rng, 200_000, 0.4)
    genome = left + gene + synth.random_dna(rng, 100_000, 0.4)
    off, pos = orc.build_index(genome)
    anc = orc.anchors(off, pos, prot)
    chains, _ = orc.chain(anc, 3)
    c = chains[0]
    assert c["strand"] == 0
    assert len(left) // 256 - 1 <= c["x_first"] <= c["x_last"] <= (len(left) + len(gene)) // 256 + 1
    assert c["n_anchors"] >= 20


# ------------------------------------------------------- second chaining round

def _brute_refine_anchors(prot, nt, strand, k=5):
    """Every (x, y) whose k codons on the aligned strand translate to a
    k-mer with the protein's reduced-alphabet codes at y..y+k-1."""
    g = _groups()
    comp = {"A": "T", "C": "G", "G": "C", "T": "A"}
    seq = nt if strand > 0 else "".join(comp[c] for c in reversed(nt))
    code = lambda c: g.get(c, g["X"])
    pk = [tuple(code(c) for c in prot[y:y + k]) for y in range(len(prot) - k + 1)]
    out = []
    for x in range(len(seq) - 3 * k + 1):
        gk = tuple(code(c) for c in _translate(seq[x:x + 3 * k]))
        out += [(x, y) for y in range(len(pk)) if pk[y] == gk]
    return sorted(out)


def test_refine_anchors_against_brute_force(orc):
    """All 5-mers of both sequences, no sampling or binning, all three frames
    of the aligned strand (stop codons included), both strands."""
    rng = np.random.default_rng(21)
    for trial in range(6):
        prot = synth.random_protein(rng, int(rng.integers(12, 60)))
        cds = synth.reverse_translate(rng, prot)
        region = synth.random_dna(rng, int(rng.integers(0, 90)), 0.4) + cds + synth.random_dna(rng, 40, 0.4)
        strand = 1 if trial % 2 == 0 else -1
        if strand < 0:
            region = synth.revcomp(region)
        got = [tuple(r) for r in orc.refine_anchors(prot, region, strand)]
        assert got == _brute_refine_anchors(prot, region, strand)
        assert len(got) >= len(prot) - 4          # the planted diagonal is there


def test_refine_gap_hand_values(orc):
    """g' = 3 dy - dx with Eq. 3: on the diagonal (dx = 3 dy) no penalty; one
    base more (dx = 3 dy + 1, g' = -1) costs min(1/3, 0.75 log2 2) = 1/3;
    one base less (g' = +1) costs 1/3 + 0.75."""
    S = orc.CHAIN_SCALE
    c, f = orc.refine_chain([(0, 0), (3, 1)])
    assert list(f) == [5 * S, 6 * S] and c["n_anchors"] == 2 and c["score"] == 6 * S
    _, f = orc.refine_chain([(0, 0), (4, 1)])
    assert f[1] == 6 * S - S // 3
    _, f = orc.refine_chain([(0, 0), (2, 1)])      # 6 - 1/3 - 0.75 < k: a new chain
    assert f[1] == 5 * S
    _, f = orc.refine_chain([(0, 0), (14, 5)])
    assert f[1] == 10 * S - (S // 3 + 3 * S // 4)
    # a gap of 60 bases inserted in the genome (dx = 3 dy + 60): min(20, 0.75 log2 61)
    _, f = orc.refine_chain([(0, 0), (75, 5)])
    assert f[1] == 10 * S - math.floor(0.75 * S * math.log2(61))
    # y must increase, x may repeat: (0, 5) after (0, 3) has g' = 6 (2 + 0.75
    # log2 7 > 2: a new chain); (9, 5) follows (0, 3) with g' = -3 (cost 1)
    _, f = orc.refine_chain([(0, 3), (0, 5), (9, 5)])
    assert list(f) == [5 * S, 5 * S, 6 * S]
    c, _ = orc.refine_chain([(7, 2)])
    assert c["n_anchors"] == 0 and c["score"] == 0


def test_refine_chain_against_enumeration(orc):
    """f of every anchor is the best k + sum(alpha - gamma(g')) over every
    chain ending there (x non-decreasing, y increasing), enumerated."""
    rng = random.Random(13)
    S, k = orc.CHAIN_SCALE, orc.REFINE_K
    for _ in range(60):
        n = rng.randint(1, 8)
        anc = sorted((rng.randint(0, 60), rng.randint(0, 25)) for _ in range(n))
        c, f = orc.refine_chain(anc)
        best = []
        for j, b in enumerate(anc):
            v = k * S
            for r in range(1, j + 1):
                for sub in itertools.combinations(range(j), r):
                    seq = [anc[t] for t in sub] + [b]
                    tot, ok = k * S, True
                    for a1, a2 in zip(seq, seq[1:]):
                        dx, dy = a2[0] - a1[0], a2[1] - a1[1]
                        if dx < 0 or dy <= 0:
                            ok = False
                            break
                        p = orc.gap_penalty(3 * dy - dx)
                        if p < 0:
                            ok = False
                            break
                        tot += min(dy, k) * S - p
                    if ok:
                        v = max(v, tot)
            best.append(v)
        assert list(f) == best, (anc, list(f), best)
        top = max(best) if best else None
        if c["n_anchors"]:
            assert c["score"] == top and c["n_anchors"] >= 2
        else:
            assert top is None or top == k * S


def test_refine_finds_the_planted_gene_at_base_resolution(orc):
    """A protein and its coding sequence (inside flanks, either strand): the
    best chain scores the protein's length (k for the first 5-mer, one per
    further residue on the diagonal) and spans it; with a 1-nt insertion in
    the middle the chain crosses the frameshift at the cost of Eq. 3."""
    rng = np.random.default_rng(5)
    S = orc.CHAIN_SCALE
    for strand in (1, -1):
        prot = synth.random_protein(rng, 150)
        cds = synth.reverse_translate(rng, prot)
        flank = synth.random_dna(rng, 300, 0.4)
        region = flank + cds + synth.random_dna(rng, 300, 0.4)
        if strand < 0:
            region = synth.revcomp(region)
        c = orc.refine(prot, region, strand)
        assert c["score"] == len(prot) * S
        assert c["y_first"] == 0 and c["y_last"] == len(prot) - 5
        assert c["x_last"] - c["x_first"] == 3 * (c["y_last"] - c["y_first"])
        assert c["x_first"] == 300
    prot = synth.random_protein(rng, 120)
    cds = synth.reverse_translate(rng, prot)
    shifted = cds[:180] + "A" + cds[180:]             # one extra base after residue 60
    c = orc.refine(prot, synth.random_dna(rng, 200, 0.4) + shifted + synth.random_dna(rng, 200, 0.4), 1)
    # the best chain crosses the shift: one link with dx = 3 dy + 1 (g' = -1,
    # penalty 1/3), every other link on a diagonal; residues 56..60 are lost
    # to the 5-mers that straddle the extra base at most
    assert c["y_first"] == 0 and c["y_last"] == len(prot) - 5
    assert c["x_last"] - c["x_first"] == 3 * (c["y_last"] - c["y_first"]) + 1
    assert len(prot) * S - 5 * S - S // 3 <= c["score"] <= len(prot) * S - S // 3
