"""Pins for the CPU oracle against what the paper and the mathematics fix.

Li 2022 (miniprot), Methods: Eq. 5 (AE86 affine gaps), Eq. 6 (frameshifts),
Eq. 7 (protein-to-genome DP), the final splice model ("Splice models") and
the worked alignment example ("Residue alignment with dynamic programming").
"""
import itertools
import os
import random

import numpy as np
import pytest

import bruteforce as bf
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _diag_sum(orc, prot):
    B = orc.blosum62_22()
    return int(sum(B[orc.AA.index(a), orc.AA.index(a)] for a in prot))


def _rand_prot(rng, n):
    return "".join(rng.choice("ARNDCQEGHILKMFPSTWYV") for _ in range(n))


# Genetic code (NCBI table 1) typed independently by the generator.
_CODE_ACGT = "KNKNTTTTRSRSIIMIQHQHPPPPRRRRLLLLEDEDAAAAGGGGVVVV*Y*YSSSS*CWCLFLF"


def _cds(rng, prot):
    syn = {}
    for k, aa in enumerate(_CODE_ACGT):
        syn.setdefault(aa, []).append("ACGT"[k // 16] + "ACGT"[(k // 4) % 4] + "ACGT"[k % 4])
    return "".join(rng.choice(syn[a]) for a in prot)


# ------------------------------------------------------------------ tables

def test_genetic_code_matches_independent_table(orc):
    for b1, b2, b3 in itertools.product(range(4), repeat=3):
        assert orc.translate_codon(b1, b2, b3) == _CODE_ACGT[16 * b1 + 4 * b2 + b3]
    # textbook spot checks
    assert orc.translate_codon(0, 3, 2) == "M"                     # ATG
    for s in ("TAA", "TAG", "TGA"):
        assert orc.translate_codon(*("ACGT".index(c) for c in s)) == "*"
    assert orc.translate_codon(3, 2, 2) == "W"                     # TGG


def test_blosum62_properties(orc):
    B = orc.blosum62_22()[:20, :20]
    assert (B == B.T).all()
    for k in range(20):
        assert B[k, k] == B[k].max() and (B[k] < B[k, k]).sum() == 19
    assert B.min() == -4 and B.max() == 11
    assert int(np.trace(B)) == 4 + 5 + 6 + 6 + 9 + 5 + 5 + 6 + 8 + 4 + 4 + 5 + 5 + 6 + 7 + 4 + 5 + 11 + 7 + 4


@pytest.mark.parametrize("motif,val", [("GTA", 0), ("GTG", 0), ("GTC", 8), ("GTT", 8),
                                       ("GCA", 15), ("GCT", 15), ("ATA", 21), ("ATG", 21),
                                       ("AGT", 30), ("CTA", 30), ("TTT", 30), ("GAA", 30)])
def test_donor_rows(orc, motif, val):
    # d(x) looks at T[x+1..x+3] (final model, "Splice models")
    nt = "CC" + motif + "CC"
    assert orc.donor(nt, 2) == val


@pytest.mark.parametrize("motif,val", [("CAG", 0), ("TAG", 0), ("AAG", 8), ("GAG", 8),
                                       ("CAC", 21), ("GAC", 21), ("TTG", 30), ("CAA", 30), ("AGG", 30)])
def test_acceptor_rows(orc, motif, val):
    # a(x) looks at T[x-2..x]
    nt = "TT" + motif + "TT"
    assert orc.acceptor(nt, 5) == val


def test_splice_out_of_range(orc):
    # bases outside T match nothing
    assert orc.donor("AAGT", 2) == 30          # GT at the end: third base missing -> not GT[ACGT]
    assert orc.donor("AAGC", 2) == 15          # two-base rows need only two bases
    assert orc.donor("AAG", 2) == 30
    assert orc.acceptor("AGTT", 2) == 30       # AG at the start: x-2 is outside T
    assert orc.acceptor("ACTT", 2) == 21
    assert orc.donor("GTA", 0) == 0 and orc.donor("GTA", -1) == 30
    assert orc.acceptor("CAG", 3) == 0 and orc.acceptor("CAG", 4) == 30


@pytest.mark.parametrize("p", [0, 7, 30])
def test_simple_model_rows(orc, p):
    """Simple GT-AG model (the definitions right after Eq. 7): every
    dinucleotide after a donor position or ending at an acceptor position;
    only GT and AG cost nothing."""
    for b1 in "ACGT":
        for b2 in "ACGT":
            dn = b1 + b2
            assert orc.donor_simple("A" + dn + "A", 1, p) == (0 if dn == "GT" else p), dn
            assert orc.acceptor_simple("A" + dn + "A", 3, p) == (0 if dn == "AG" else p), dn
    # bases outside T match nothing
    assert orc.donor_simple("AAG", 2, p) == p and orc.donor_simple("GT", 0, p) == 0
    assert orc.donor_simple("GT", -1, p) == p and orc.acceptor_simple("AG", 2, p) == 0
    assert orc.acceptor_simple("AG", 1, p) == p and orc.acceptor_simple("AG", 3, p) == p


# ----------------------------------------------------------- brute force

def _random_case(rng, n, m, valid=True):
    prot = _rand_prot(rng, m)
    if rng.random() < 0.5:
        # plant a codon-level copy so that positive paths exist
        nt = _cds(rng, prot)
        extra = "".join(rng.choice("ACGT") for _ in range(max(0, n - len(nt))))
        k = rng.randint(0, len(extra))
        nt = (extra[:k] + nt + extra[k:])[:n]
    else:
        nt = "".join(rng.choice("ACGT") for _ in range(n))
    if valid:
        f = rng.randint(1, 6)
        params = dict(q=rng.randint(0, 4), e=rng.randint(1, 3), f=f,
                      stop=rng.randint(1, 6))
        params["r"] = max(f, params["stop"], 4) + rng.randint(1, 4)
    else:
        params = dict(q=rng.randint(0, 5), e=rng.randint(0, 3), f=rng.randint(0, 12),
                      r=rng.randint(0, 12), stop=rng.randint(0, 10))
    return prot, nt, params


def test_exhaustive_enumeration_equals_oracle(orc):
    rng = random.Random(11)
    for k in range(50):
        n, m = (rng.randint(0, 6), rng.randint(0, 2)) if k < 40 else (rng.randint(4, 6), 3)
        prot, nt, params = _random_case(rng, n, m, valid=rng.random() < 0.5)
        paths = bf.all_paths(bf.Problem(prot, nt, **params))
        want = bf.best_by_enumeration(paths)
        got = orc.align(prot, nt, 1, orc.make_params(**params))["score"]
        assert got == want, (prot, nt, params)


def test_exhaustive_enumeration_larger_cases(orc):
    """Every path enumerated one by one at the largest sizes the CPU suite
    affords (7 nt x 3 aa: 1.9 M paths; 9 nt x 2 aa: 4.5 M paths), with a
    planted coding copy so that multi-op positive paths exist: the oracle's
    score is the best enumerated op-sum."""
    rng = random.Random(17)
    for n, m in ((7, 3), (9, 2)):
        prot = _rand_prot(rng, m)
        nt = (_cds(rng, prot) + "".join(rng.choice("ACGT") for _ in range(n)))[:n]
        params = dict(q=2, e=1, f=3, stop=4, r=7)
        paths = bf.all_paths(bf.Problem(prot, nt, **params), limit=6_000_000)
        want = bf.best_by_enumeration(paths)
        got = orc.align(prot, nt, 1, orc.make_params(**params))["score"]
        assert got == want, (prot, nt, len(paths))


def test_segment_recursion_equals_oracle(orc):
    rng = random.Random(12)
    for _ in range(150):
        n, m = rng.randint(0, 20), rng.randint(0, 5)
        prot, nt, params = _random_case(rng, n, m, valid=rng.random() < 0.5)
        want = bf.segment_best(bf.Problem(prot, nt, **params))
        got = orc.align(prot, nt, 1, orc.make_params(**params))["score"]
        assert got == want, (prot, nt, params)


def test_simple_model_against_enumeration(orc):
    """With the simple GT-AG model the oracle's score is the best path score
    of the enumerations (all three intron phases, with GT/AG and other
    splice sites), for several costs p."""
    rng = random.Random(17)
    for k in range(120):
        n, m = rng.randint(0, 20), rng.randint(0, 5)
        prot, nt, params = _random_case(rng, n, m, valid=True)
        if nt and rng.random() < 0.6:
            # plant splice signals so that cheap introns exist
            i = rng.randint(0, len(nt))
            nt = (nt[:i] + "GT" + "".join(rng.choice("ACGT") for _ in range(rng.randint(0, 4))) + "AG" + nt[i:])[:22]
        p = rng.choice([0, 3, 9, 30])
        want = bf.segment_best(bf.Problem(prot, nt, splice_p=p, **params))
        got = orc.align(prot, nt, 1, orc.make_params(splice_model=1, splice_p=p, **params))["score"]
        assert got == want, (prot, nt, params, p)
        if len(nt) <= 6 and m <= 2:
            assert got == bf.best_by_enumeration(bf.all_paths(bf.Problem(prot, nt, splice_p=p, **params)))


def test_simple_model_intron_costs(orc):
    """A GT...AG intron costs r under the simple model and r + 2p when the
    same intron has neither signal."""
    rng = random.Random(44)
    prot, nt, intron = _intron_case(rng, 0)
    for p in (0, 5, 30):
        r = orc.align(prot, nt, 1, orc.make_params(splice_model=1, splice_p=p))
        assert r["score"] == _diag_sum(orc, prot) - 29 and r["cigar"][1] == ("N", len(intron))
    # CA...TC instead of GT...AG: the intron pays r + 2p while that stays cheaper than the alternatives
    bad = nt.replace(intron, "CA" + intron[2:-2] + "TC")
    r = orc.align(prot, bad, 1, orc.make_params(splice_model=1, splice_p=3))
    assert r["score"] == _diag_sum(orc, prot) - 29 - 6 and r["cigar"][1] == ("N", len(intron))


def test_simple_model_rescoring(orc):
    """Op-sum rescoring under the simple model reproduces the DP score."""
    rng = random.Random(45)
    for _ in range(30):
        prot, nt, intron = _intron_case(rng, rng.randint(0, 2))
        p = rng.choice([0, 4, 30])
        params = orc.make_params(splice_model=1, splice_p=p)
        r = orc.align(prot, nt, 1, params)
        sc, pe, te = orc.rescore(prot, nt, 1, r["prot_st"], r["nt_st"], r["cigar_raw"], params)
        assert (sc, pe, te) == (r["score"], r["prot_en"], r["nt_en"])


def test_segment_recursion_default_params(orc):
    rng = random.Random(13)
    for _ in range(40):
        m = rng.randint(1, 5)
        prot = _rand_prot(rng, m)
        cds = _cds(rng, prot)
        nt = "".join(rng.choice("ACGT") for _ in range(rng.randint(0, 6))) + cds + \
             "".join(rng.choice("ACGT") for _ in range(rng.randint(0, 6)))
        assert orc.align(prot, nt)["score"] == bf.segment_best(bf.Problem(prot, nt))


def test_tie_rule_against_path_order(orc):
    """The oracle's path is the optimum the stated tie rules select among all
    enumerated optimal paths.  Small integer penalties make ties common."""
    rng = random.Random(14)
    mat = np.zeros((22, 22), dtype=np.int32)
    B = orc.blosum62_22()
    mat[:] = np.sign(B)           # values in {-1, 0, 1}: many equal-scoring paths
    mat[np.arange(20), np.arange(20)] = 2
    checked = 0
    for _ in range(80):
        n, m = rng.randint(3, 7), rng.randint(1, 2)
        prot = _rand_prot(rng, m)
        nt = "".join(rng.choice("ACGT") for _ in range(n))
        if rng.random() < 0.6:
            k = rng.randint(0, n - 3)
            nt = (nt[:k] + _cds(rng, prot) + nt[k:])[:n]
        params = dict(q=rng.randint(0, 2), e=1, f=rng.randint(1, 2), stop=1, r=3)
        pb = bf.Problem(prot, nt, mat=mat, **params)
        paths = bf.all_paths(pb)
        choice = bf.tie_rule_choice(paths)
        res = orc.align(prot, nt, 1, orc.make_params(mat=mat, **params))
        if choice is None:
            assert res["score"] == 0 and res["cigar"] == []
            continue
        si, sj, ops, ei, ej, sc = choice
        assert res["score"] == sc
        assert (res["prot_st"], res["prot_en"], res["nt_st"], res["nt_en"]) == (sj, ej, si, ei), (prot, nt, params)
        assert res["cigar"] == bf.to_cigar(ops), (prot, nt, params, ops)
        checked += 1
    assert checked > 40


# --------------------------------------------------- textbook special case

def _gotoh_local(a, b, S, q, e):
    """Textbook local alignment with affine gaps (Gotoh 1982; Eq. 5 form)."""
    NEG = -10 ** 9
    n, m = len(a), len(b)
    H = [[0] * (m + 1) for _ in range(n + 1)]
    E = [[NEG] * (m + 1) for _ in range(n + 1)]
    F = [[NEG] * (m + 1) for _ in range(n + 1)]
    best = 0
    for i in range(1, n + 1):
        for j in range(1, m + 1):
            E[i][j] = max(H[i][j - 1] - q, E[i][j - 1]) - e
            F[i][j] = max(H[i - 1][j] - q, F[i - 1][j]) - e
            H[i][j] = max(0, H[i - 1][j - 1] + S(a[i - 1], b[j - 1]), E[i][j], F[i][j])
            best = max(best, H[i][j])
    return best


def test_reduces_to_three_frame_gotoh(orc):
    """With f = r = 10^6 no frameshift or intron can win; the DP is then the
    AE86 local alignment (Eq. 5) of each translated frame against P."""
    rng = random.Random(21)
    B = orc.blosum62_22()
    for _ in range(40):
        m = rng.randint(1, 25)
        prot = _rand_prot(rng, m)
        nt = _cds(rng, _rand_prot(rng, rng.randint(0, 4))) + _cds(rng, prot)
        nt = list(nt)
        for _ in range(rng.randint(0, 6)):                     # point mutations
            nt[rng.randrange(len(nt))] = rng.choice("ACGT")
        for _ in range(rng.randint(0, 2)):                     # indels of 1 nt
            k = rng.randrange(len(nt))
            if rng.random() < 0.5:
                nt.insert(k, rng.choice("ACGT"))
            else:
                del nt[k]
        nt = "".join(nt)
        q, e, stop = rng.randint(1, 12), rng.randint(1, 3), rng.randint(1, 30)

        def S(x, y):
            return -stop if x == "*" else int(B[orc.AA.index(x), orc.AA.index(y)])

        want = 0
        for o in range(3):
            frame = [_CODE_ACGT[16 * "ACGT".index(nt[k]) + 4 * "ACGT".index(nt[k + 1]) + "ACGT".index(nt[k + 2])]
                     for k in range(o, len(nt) - 2, 3)]
            want = max(want, _gotoh_local(frame, prot, S, q, e))
        got = orc.align(prot, nt, 1, orc.make_params(q=q, e=e, f=10 ** 6, r=10 ** 6, stop=stop))["score"]
        assert got == want


# ----------------------------------------------------------- invariants

def test_exact_cds_scores_diagonal_sum(orc):
    rng = random.Random(31)
    for _ in range(30):
        prot = _rand_prot(rng, rng.randint(1, 200))
        r = orc.align(prot, _cds(rng, prot))
        assert r["score"] == _diag_sum(orc, prot)
        assert r["cigar"] == [("M", len(prot))]
        assert (r["prot_st"], r["prot_en"], r["nt_st"], r["nt_en"]) == (0, len(prot), 0, 3 * len(prot))


def test_minus_strand_matches_plus(orc):
    for k, p in enumerate(synth.config2(seed=100 + 0, n=6)):
        if len(p.prot) * len(p.nt) > 3_000_000:
            continue
        a = orc.align(p.prot, p.nt, p.strand)
        b = orc.align(p.prot, orc.revcomp(p.nt), -p.strand)
        assert a["score"] == b["score"]
        assert (a["prot_st"], a["prot_en"]) == (b["prot_st"], b["prot_en"])
        assert (a["nt_st"], a["nt_en"]) == (len(p.nt) - b["nt_en"], len(p.nt) - b["nt_st"])
        assert a["cigar"] == b["cigar"]


def test_cigar_rescoring_equals_score(orc):
    pairs = [synth.config1()] + [p for p in synth.config2(seed=101, n=12) if p.cells < 2_500_000]
    for p in pairs:
        r = orc.align(p.prot, p.nt, p.strand)
        n = len(p.nt)
        st_aligned = r["nt_st"] if p.strand > 0 else n - r["nt_en"]
        en_aligned = r["nt_en"] if p.strand > 0 else n - r["nt_st"]
        sc, pe, te = orc.rescore(p.prot, p.nt, p.strand, r["prot_st"], st_aligned, r["cigar_raw"])
        assert (sc, pe, te) == (r["score"], r["prot_en"], en_aligned)
        assert r["status"] == 0


# ------------------------------------------------------------ hand cases

def test_hand_ungapped_with_flanks(orc):
    rng = random.Random(41)
    prot = _rand_prot(rng, 40)
    nt = "TTTTTTTTTT" + _cds(rng, prot) + "TTTTTTTTTT"   # TTT codons are F, poly-T flanks
    r = orc.align(prot, nt)
    assert r["score"] >= _diag_sum(orc, prot)


def test_hand_frameshift_insertion_and_deletion(orc):
    """Eq. 6: one inserted base ('+', G1) costs f; a codon missing one base
    ('$', F2) costs f and leaves its residue unscored."""
    rng = random.Random(42)
    p1, p2 = _rand_prot(rng, 30), _rand_prot(rng, 30)
    c1, c2 = _cds(rng, p1), _cds(rng, p2)
    big = dict(r=10 ** 6)
    r = orc.align(p1 + p2, c1 + "A" + c2, 1, orc.make_params(**big))
    assert r["score"] == _diag_sum(orc, p1 + p2) - 23
    assert r["cigar"] == [("M", 30), ("G", 1), ("M", 30)]
    # a Met codon (ATG) that lost its last base, between two Trp (TGG): the
    # frame shifts back only through the '$' operation
    q1, q2 = p1[:-1] + "W", "W" + p2[1:]
    c1, c2 = _cds(rng, q1), _cds(rng, q2)
    r = orc.align(q1 + "M" + q2, c1 + "AT" + c2, 1, orc.make_params(**big))
    assert r["score"] == _diag_sum(orc, q1 + q2) - 23
    assert r["cigar"] == [("M", 30), ("F", 2), ("M", 30)]


def _intron_case(rng, phase, L=90):
    prot = _rand_prot(rng, 40)
    cds = _cds(rng, prot)
    cut = 3 * 20 + phase
    body = "".join(rng.choice("CT") for _ in range(L - 6))      # pyrimidine filler: no stop-free codon runs of note
    intron = "GTA" + body + "CAG"                               # d = 0, a = 0
    return prot, cds[:cut] + intron + cds[cut:], intron


@pytest.mark.parametrize("phase,op", [(0, "N"), (1, "U"), (2, "V")])
def test_hand_single_intron(orc, phase, op):
    """One GTA...CAG intron (d = a = 0) costs r; a split codon (phase 1/2)
    leaves its residue unscored (Methods, after Eq. 7)."""
    rng = random.Random(43 + phase)
    prot, nt, intron = _intron_case(rng, phase)
    r = orc.align(prot, nt)
    want = _diag_sum(orc, prot) - 29
    if phase:
        want -= _diag_sum(orc, prot[20])
    assert r["score"] == want
    if phase == 0:
        assert r["cigar"] == [("M", 20), ("N", len(intron)), ("M", 20)]
    else:
        assert r["cigar"] == [("M", 20), (op, len(intron)), ("M", 19)]


# ------------------------------------------- global and extension modes

def test_anchored_modes_against_segment_recursion(orc):
    """Global mode (path from cell (0, 0) to (|T|, |P|)) and extension mode
    (from (0, 0), ending anywhere): the oracle's score is the best op-sum over
    paths from (0, 0), with random penalties and both splice models."""
    rng = random.Random(71)
    for k in range(150):
        n, m = rng.randint(0, 14), rng.randint(0, 4)
        prot, nt, params = _random_case(rng, n, m, valid=True)
        simple = rng.random() < 0.3
        sp = dict(splice_p=rng.choice([0, 5, 30])) if simple else {}
        for mode, name in ((1, "global"), (2, "extend")):
            want = bf.anchored_best(bf.Problem(prot, nt, **params, **sp), name)
            got = orc.align(prot, nt, 1, orc.make_params(mode=mode, splice_model=1 if simple else 0, **params, **sp))
            assert got["score"] == want, (mode, prot, nt, params, sp)


def test_every_h_cell_against_segment_tables(orc):
    """Every cell of the oracle's H matrix is the best score of a path ending
    there (H is the maximum of Eq. 7's states, and each state the best over
    its paths): local mode against paths from any cell with the empty path at
    0, the anchored modes against paths from (0, 0).  A wrong boundary value
    (row 0, column 0) or a dropped term shows up in the cell it reaches."""
    rng = random.Random(73)
    for k in range(90):
        n, m = rng.randint(0, 16), rng.randint(0, 5)
        prot, nt, params = _random_case(rng, n, m, valid=rng.random() < 0.7)
        simple = rng.random() < 0.3
        sp = dict(splice_p=rng.choice([0, 5, 30])) if simple else {}
        pb = bf.Problem(prot, nt, **params, **sp)
        for mode, name in ((0, "local"), (1, "global"), (2, "extend")):
            want = np.array(bf.best_table(pb, name), dtype=np.float64)
            op = orc.make_params(mode=mode, splice_model=1 if simple else 0, **params, **sp)
            got = orc.fill_h(prot, nt, 1, op)
            assert got.shape == (n + 1, m + 1)
            assert np.array_equal(got.astype(np.float64), want), (mode, prot, nt, params, sp)


def test_anchored_modes_against_enumeration(orc):
    """The same against every enumerated path from (0, 0) on tiny inputs."""
    rng = random.Random(72)
    for _ in range(60):
        prot, nt, params = _random_case(rng, rng.randint(0, 6), rng.randint(0, 2), valid=True)
        paths = [p for p in bf.all_paths(bf.Problem(prot, nt, **params)) if p[0] == 0 and p[1] == 0]
        g = max(p[5] for p in paths if (p[3], p[4]) == (len(nt), len(prot)))
        x = max(p[5] for p in paths)
        assert orc.align(prot, nt, 1, orc.make_params(mode=1, **params))["score"] == g
        assert orc.align(prot, nt, 1, orc.make_params(mode=2, **params))["score"] == x


def test_anchored_modes_against_larger_enumeration(orc):
    """Every path from cell (0, 0) enumerated one by one at 7 nt x 3 aa
    (1.2 M paths) and 8 nt x 2 aa (0.8 M), with a planted coding copy: the
    global score is the best path ending at (|T|, |P|), the extension score
    the best path anywhere (the empty one included)."""
    rng = random.Random(73)
    for n, m in ((7, 3), (8, 2)):
        prot = _rand_prot(rng, m)
        nt = (_cds(rng, prot) + "".join(rng.choice("ACGT") for _ in range(n)))[:n]
        params = dict(q=2, e=1, f=3, stop=4, r=7)
        paths = bf.anchored_paths(bf.Problem(prot, nt, **params), limit=3_000_000)
        g = max(p[3] for p in paths if (p[1], p[2]) == (n, m))
        x = max(p[3] for p in paths)
        assert orc.align(prot, nt, 1, orc.make_params(mode=1, **params))["score"] == g, (prot, nt)
        assert orc.align(prot, nt, 1, orc.make_params(mode=2, **params))["score"] == x, (prot, nt)


def test_anchored_paths_rescore_and_span(orc):
    """Anchored alignments start at (0, 0); global ones end at (|T|, |P|);
    their CIGARs rescore to the score (negative scores included), on both
    strands."""
    rng = random.Random(73)
    for _ in range(40):
        prot, nt, params = _random_case(rng, rng.randint(3, 40), rng.randint(1, 8), valid=True)
        for mode in (1, 2):
            pp = orc.make_params(mode=mode, **params)
            for strand, t in ((1, nt), (-1, orc.revcomp(nt))):
                r = orc.align(prot, t, strand, pp)
                if mode == 2 and r["score"] == 0 and not r["cigar"]:
                    continue                                  # the empty extension
                st = 0 if strand > 0 else len(t) - r["nt_en"]
                assert r["prot_st"] == 0 and (r["nt_st"] == 0 if strand > 0 else r["nt_en"] == len(t))
                if mode == 1:
                    assert r["prot_en"] == len(prot) and (r["nt_en"] if strand > 0 else len(t) - r["nt_st"]) == len(t)
                if r["cigar"]:
                    sc, pe, te = orc.rescore(prot, t, strand, r["prot_st"], st, r["cigar_raw"], pp)
                    assert (sc, pe) == (r["score"], r["prot_en"])


def test_anchored_exact_cds(orc):
    """An exact coding sequence: global and extension scores equal the local
    one (Σ diag); with one extra codon before it, global pays one deletion
    q + e and extension too (the path must start at the genome's start)."""
    rng = random.Random(74)
    prot = _rand_prot(rng, 30)
    cds = _cds(rng, prot)
    diag = _diag_sum(orc, prot)
    for mode in (1, 2):
        assert orc.align(prot, cds, 1, orc.make_params(mode=mode))["score"] == diag
        r = orc.align(prot, "CCC" + cds, 1, orc.make_params(mode=mode))
        assert r["score"] == diag - 12 and r["cigar"] == [("D", 1), ("M", 30)]


# ------------------------------------------------------- pseudogenes

@pytest.mark.parametrize("phase", [0, 1, 2])
def test_exon_sequence_rebuilds_the_cds(orc, phase):
    """For an exact spliced copy the alignment's coding region without
    introns is the coding sequence itself (split codon kept for phases 1, 2),
    on either strand."""
    rng = random.Random(60 + phase)
    prot, nt, intron = _intron_case(rng, phase)
    cds = nt.replace(intron, "")
    for strand, t in ((1, nt), (-1, orc.revcomp(nt))):
        r = orc.align(prot, t, strand)
        assert orc.exon_sequence(t, strand, r) == cds


def test_exon_score_prefers_the_spliced_gene(orc):
    """Avoiding pseudogenes: against its spliced gene a protein pays the
    intron in the DP score but not in the exon score; against an unspliced
    copy (a processed pseudogene) the exon score pays r once more."""
    rng = random.Random(64)
    prot, gene, intron = _intron_case(rng, 0)
    pseudo = gene.replace(intron, "")
    diag = _diag_sum(orc, prot)
    rg, rp = orc.align(prot, gene), orc.align(prot, pseudo)
    assert rg["score"] == diag - 29 and rp["score"] == diag            # the DP favours the pseudogene
    assert orc.exon_score(prot, gene) == diag                             # intron-free region: Σ diag
    assert orc.exon_score(prot, pseudo) == diag - 29                      # single exon pays r
    assert orc.exon_score(prot, gene) > orc.exon_score(prot, pseudo)
    assert orc.exon_score("WWWW", "AAAAAAAAAAAA") == 0                    # no alignment


# ---------------------------------------------------------------- ties

def test_best_cell_tie_smallest_i(orc):
    r = orc.align("W", "TGGCCCTGG")
    assert (r["score"], r["nt_st"], r["nt_en"]) == (11, 0, 3)


def test_best_cell_tie_smallest_j(orc):
    r = orc.align("WW", "TGG")
    assert (r["score"], r["prot_st"], r["prot_en"]) == (11, 0, 1)


def test_restart_wins_tie_at_zero(orc):
    # ACT (Thr) vs A scores 0: the path restarts after it.
    r = orc.align("AW", "ACTTGG")
    assert r["score"] == 11
    assert (r["prot_st"], r["nt_st"], r["cigar"]) == (1, 3, [("M", 1)])


def test_empty_and_degenerate_inputs(orc):
    assert orc.align("", "ACGT")["score"] == 0
    assert orc.align("MW", "")["score"] == 0
    assert orc.align("W", "TG")["score"] == 0          # no full codon
    r = orc.align("P", "AAAAAA")                       # only negative cells
    assert r["score"] == 0 and r["cigar"] == [] and r["prot_en"] == 0


# ------------------------------------------------------ paper's example

def _read_golden(name):
    d = {}
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, v = line.split("=", 1)
            d[k.strip()] = v.strip()
    return d


def test_paper_worked_example(orc):
    """The worked alignment of the Methods section decodes to a valid path
    whose op-sum equals the hand total; the DP's optimum is at least that
    (it is not optimal: AAG/E scores +1 where the example uses '$$')."""
    g = _read_golden("paper_example.txt")
    prot, nt = g["prot"], g["genome"]
    ops = [(t[-1], int(t[:-1])) for t in g["cigar"].split()]
    cheap = {k: int(v) for k, v in (kv.split("=") for kv in g["cheap"].split())}
    for params, want in ((orc.make_params(**cheap), int(g["cheap_score"])),
                         (orc.make_params(), int(g["default_score"]))):
        sc, pe, te = orc.rescore(prot, nt, 1, 0, 0, orc.encode_cigar(ops), params)
        assert (sc, pe, te) == (want, len(prot), len(nt))
        r = orc.align(prot, nt, 1, params)
        assert r["score"] >= max(want, 0)
        sc2, pe2, te2 = orc.rescore(prot, nt, 1, r["prot_st"], r["nt_st"], r["cigar_raw"], params)
        assert (sc2, pe2, te2) == (r["score"], r["prot_en"], r["nt_en"])


# ------------------------------------------- score and end cell in four rows
def _best_cell(table, mode, n, m):
    """(score, i, j) of the best cell of a table of per-cell best path
    scores: the largest score, then the smallest i, then the smallest j
    (local: cells after a residue and a base, score 0 at (0, 0) when none is
    positive; extension: every cell; global: the cell (n, m))."""
    if mode == "global":
        return table[n][m], n, m
    best, bi, bj = 0, 0, 0
    for i in range(n + 1):
        for j in range(m + 1):
            if mode == "local" and (i == 0 or j == 0):
                continue
            if table[i][j] > best:
                best, bi, bj = table[i][j], i, j
    return best, bi, bj


def _end_of(res, strand, n):
    """The best cell's genome row in the aligned orientation."""
    return res["nt_en"] if strand > 0 else n - res["nt_st"]


def test_score_end_against_segment_recursion(orc):
    """The four-row fill's score and end cell equal the best cell of the
    Bellman recursion over whole operations (no DP states), in all three
    modes, both splice models, valid and invalid penalty sets."""
    rng = random.Random(91)
    modes = {0: "local", 1: "global", 2: "extend"}
    for k in range(60):
        prot, nt, params = _random_case(rng, rng.randint(0, 20), rng.randint(0, 5), valid=rng.random() < 0.6)
        sp = rng.randint(0, 9) if k % 3 == 0 else None
        pb = bf.Problem(prot, nt, splice_p=sp, **params)
        for mode in (0, 1, 2):
            want = _best_cell(bf.best_table(pb, modes[mode]), modes[mode], len(nt), len(prot))
            pp = orc.make_params(mode=mode, splice_model=0 if sp is None else 1,
                                 splice_p=30 if sp is None else sp, **params)
            got = orc.score_end(prot, nt, 1, pp)
            assert (got["score"], _end_of(got, 1, len(nt)), got["prot_en"]) == want, (prot, nt, params, mode)


def test_score_end_against_enumeration(orc):
    """Score and end cell against every enumerated path on tiny inputs: the
    best op-sum, ending at the smallest (i, j) among optimal paths."""
    rng = random.Random(92)
    for _ in range(40):
        prot, nt, params = _random_case(rng, rng.randint(1, 6), rng.randint(1, 2), valid=True)
        paths = bf.all_paths(bf.Problem(prot, nt, **params))
        best = bf.best_by_enumeration(paths)
        got = orc.score_end(prot, nt, 1, orc.make_params(**params))
        assert got["score"] == best
        if best > 0:
            assert (_end_of(got, 1, len(nt)), got["prot_en"]) == min((p[3], p[4]) for p in paths if p[5] == best)


def test_score_end_equals_full_oracle(orc):
    """On larger pairs (planted spliced genes with flanks, random regions,
    both strands) the four-row fill gives the full-matrix oracle's score and
    end cell in every mode, with default, random and tie-rich penalties."""
    rng = np.random.default_rng(93)
    r2 = random.Random(93)
    tie = np.sign(orc.blosum62_22()).astype(np.int32)
    tie[np.arange(20), np.arange(20)] = 2
    cases = []
    for k in range(24):
        m = int(rng.integers(5, 90))
        prot = synth.random_protein(rng, m)
        if k % 4 == 3:
            nt = synth.random_dna(rng, int(rng.integers(10, 900)))
        else:
            introns = [int(x) for x in rng.integers(40, 300, size=int(rng.integers(0, 3)))]
            nt, _ = synth.gen.plant_gene(rng, prot, 0.25, int(rng.integers(0, 3)), introns,
                                         int(rng.integers(0, 80)), int(rng.integers(0, 80)), 0.4)
        cases.append((prot, nt))
    psets = [dict(), dict(q=3, e=2, f=5, r=9, stop=4), dict(q=1, e=1, f=2, r=4, stop=1, mat=tie)]
    for k, (prot, nt) in enumerate(cases):
        for mode in (0, 1, 2):
            ps = psets[(k + mode) % 3]
            pp = orc.make_params(mode=mode, splice_model=k % 2, splice_p=r2.randint(0, 20), **ps)
            for strand, t in ((1, nt), (-1, orc.revcomp(nt))):
                full = orc.align(prot, t, strand, pp)
                got = orc.score_end(prot, t, strand, pp)
                assert got["score"] == full["score"], (k, mode, strand)
                if full["score"] > 0 or mode == 1:
                    assert got["prot_en"] == full["prot_en"], (k, mode, strand)
                    if strand > 0:
                        assert got["nt_en"] == full["nt_en"], (k, mode, strand)
                    else:
                        assert got["nt_st"] == full["nt_st"], (k, mode, strand)


# ------------------------------------- tie rule of the anchored tracebacks
def test_anchored_tie_rule_against_path_order(orc):
    """Global and extension modes: the oracle's path is the optimum the
    stated tie rules select among every enumerated path from cell (0, 0):
    the end cell (global: (|T|, |P|); extension: the smallest i, then j,
    among optimal ends, the empty path at (0, 0) included), then, reading
    the operations backwards, the earliest term of Eq. 7's printed order,
    the shorter run first inside I, D and intron runs.  Small integer
    penalties and a {-1, 0, 1, 2} matrix make ties common."""
    rng = random.Random(94)
    mat = np.sign(orc.blosum62_22()).astype(np.int32)
    mat[np.arange(20), np.arange(20)] = 2

    def key(p):
        return tuple((bf.ORDER[name], L) for name, L in reversed(p[0]))

    checked = {1: 0, 2: 0}
    for _ in range(90):
        n, m = rng.randint(2, 7), rng.randint(1, 2)
        prot = _rand_prot(rng, m)
        nt = "".join(rng.choice("ACGT") for _ in range(n))
        if rng.random() < 0.6:
            k = rng.randint(0, max(0, n - 3))
            nt = (nt[:k] + _cds(rng, prot) + nt[k:])[:n]
        params = dict(q=rng.randint(0, 2), e=1, f=rng.randint(1, 2), stop=1, r=3)
        paths = bf.anchored_paths(bf.Problem(prot, nt, mat=mat, **params))
        for mode in (1, 2):
            res = orc.align(prot, nt, 1, orc.make_params(mat=mat, mode=mode, **params))
            if mode == 1:
                ends = [p for p in paths if (p[1], p[2]) == (n, m)]
                best = max(p[3] for p in ends)
                opt = [p for p in ends if p[3] == best]
            else:
                best = max(p[3] for p in paths)            # the empty path scores 0
                if best == 0:
                    assert res["score"] == 0 and res["cigar"] == [], (prot, nt, params)
                    continue
                opt = [p for p in paths if p[3] == best]
                ei, ej = min((p[1], p[2]) for p in opt)
                opt = [p for p in opt if (p[1], p[2]) == (ei, ej)]
            choice = min(opt, key=key)
            ops, ei, ej, sc = choice
            assert res["score"] == sc, (prot, nt, params, mode)
            assert (res["prot_st"], res["prot_en"], res["nt_st"], res["nt_en"]) == (0, ej, 0, ei), \
                (prot, nt, params, mode)
            assert res["cigar"] == bf.to_cigar(ops), (prot, nt, params, mode, ops)
            checked[mode] += 1
    assert checked[1] > 40 and checked[2] > 30, checked


# ------------------------------------------ profile queries (Discussion)
def _random_profile(rng, m, lo=-6, hi=6, qmax=4, emax=3):
    """Position-specific costs: random scores per position and translated
    code (stop included), random gap open and extension per column."""
    prof = np.zeros((m + 1, 23), dtype=np.int32)
    for j in range(m + 1):
        prof[j, :21] = [rng.randint(lo, hi) for _ in range(21)]
        prof[j, 21] = rng.randint(0, qmax)
        prof[j, 22] = rng.randint(1, emax)
    prof[0, :21] = 0
    return prof


def test_profile_reduces_to_the_position_independent_model(orc):
    """A profile holding mat[c][P[j]], -stop and the global q, e at every
    position gives exactly the results of the position-independent scoring,
    in every mode and on both strands (the profile path's plumbing)."""
    rng = np.random.default_rng(95)
    for k in range(16):
        m = int(rng.integers(1, 60))
        prot = synth.random_protein(rng, m)
        introns = [int(x) for x in rng.integers(40, 200, size=int(rng.integers(0, 3)))]
        nt, _ = synth.gen.plant_gene(rng, prot, 0.25, int(rng.integers(0, 2)), introns,
                                     int(rng.integers(0, 60)), int(rng.integers(0, 60)), 0.4)
        for mode in (0, 1, 2):
            ps = dict(q=int(rng.integers(0, 12)), e=int(rng.integers(1, 4)), f=17, r=29, stop=11)
            base = orc.make_params(mode=mode, **ps)
            prof = orc.profile_of(prot, base)
            pp = orc.make_params(mode=mode, prof=prof, **ps)
            for strand, t in ((1, nt), (-1, orc.revcomp(nt))):
                a = orc.align(prot, t, strand, base)
                b = orc.align(prot, t, strand, pp)
                assert {x: a[x] for x in ("score", "prot_st", "prot_en", "nt_st", "nt_en", "cigar")} == \
                       {x: b[x] for x in ("score", "prot_st", "prot_en", "nt_st", "nt_en", "cigar")}, (k, mode)
                se = orc.score_end(prot, t, strand, pp)
                assert (se["score"], se["prot_en"]) == (a["score"], a["prot_en"])


def test_profile_against_segment_recursion(orc):
    """With arbitrary position-specific scores and gap costs the oracle's
    score, in every mode, and the four-row fill's end cell equal the best
    path of the operation-level recursion that charges each operation the
    profile's costs."""
    rng = random.Random(96)
    modes = {0: "local", 1: "global", 2: "extend"}
    for k in range(50):
        n, m = rng.randint(0, 18), rng.randint(0, 5)
        prot = _rand_prot(rng, m)
        nt = "".join(rng.choice("ACGT") for _ in range(n))
        if rng.random() < 0.5 and m:
            nt = (_cds(rng, prot) + nt)[:max(n, 3 * m)]
        prof = _random_profile(rng, m)
        ps = dict(q=3, e=1, f=rng.randint(2, 6), stop=3, r=rng.randint(7, 12))
        pb = bf.Problem(prot, nt, prof=prof, **ps)
        for mode in (0, 1, 2):
            pp = orc.make_params(mode=mode, prof=prof, **ps)
            want = _best_cell(bf.best_table(pb, modes[mode]), modes[mode], len(nt), len(prot))
            got = orc.align(prot, nt, 1, pp)
            assert got["score"] == want[0], (k, mode, prot, nt)
            se = orc.score_end(prot, nt, 1, pp)
            assert (se["score"], _end_of(se, 1, len(nt)), se["prot_en"]) == want, (k, mode)
            if got["cigar"]:
                st = got["nt_st"]
                sc, pe, te = orc.rescore(prot, nt, 1, got["prot_st"], st, got["cigar_raw"], pp)
                assert (sc, pe, te) == (got["score"], got["prot_en"], got["nt_en"]), (k, mode)


def test_profile_tie_rule_against_path_order(orc):
    """Local mode with a profile: the oracle's path is the optimum the
    stated tie rules select among all enumerated paths (tie-rich scores in
    {-1, 0, 1, 2})."""
    rng = random.Random(97)
    checked = 0
    for _ in range(70):
        n, m = rng.randint(3, 7), rng.randint(1, 2)
        prot = _rand_prot(rng, m)
        nt = "".join(rng.choice("ACGT") for _ in range(n))
        if rng.random() < 0.6:
            kk = rng.randint(0, n - 3)
            nt = (nt[:kk] + _cds(rng, prot) + nt[kk:])[:n]
        prof = _random_profile(rng, m, lo=-1, hi=2, qmax=2, emax=1)
        ps = dict(q=1, e=1, f=rng.randint(1, 2), stop=1, r=3)
        paths = bf.all_paths(bf.Problem(prot, nt, prof=prof, **ps))
        choice = bf.tie_rule_choice(paths)
        res = orc.align(prot, nt, 1, orc.make_params(prof=prof, **ps))
        if choice is None:
            assert res["score"] == 0 and res["cigar"] == []
            continue
        si, sj, ops, ei, ej, sc = choice
        assert res["score"] == sc
        assert (res["prot_st"], res["prot_en"], res["nt_st"], res["nt_en"]) == (sj, ej, si, ei)
        assert res["cigar"] == bf.to_cigar(ops), (prot, nt, ops)
        checked += 1
    assert checked > 30
