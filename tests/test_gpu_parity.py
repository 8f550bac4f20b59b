"""GPU vs oracle parity through the C ABI.

The bar is bit-exact equality of score, coordinates (0-based half-open) and
CIGAR with the oracle (plain C, int32, full matrices) on seeded inputs: tiny
exhaustive-size pairs, sizes spanning several 64-residue strips and 96-step
chunks with ragged tails, the 1,111-nt single pair, both strands, int16 saturation with the int32 re-run, and edge cases.
"""
import ctypes
import random

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

KEYS = ("score", "prot_st", "prot_en", "nt_st", "nt_en", "cigar")


@pytest.fixture(scope="module")
def mp():
    from paper_2210_08052_gb300 import build
    build.build()
    import paper_2210_08052_gb300 as m
    m.lib()
    return m


@pytest.fixture(scope="module")
def ctx(mp):
    c = mp.mp_dp_init(None, 0)
    yield c
    mp.mp_dp_destroy(c)


@pytest.fixture(scope="module")
def ctx32(mp):
    c = mp.mp_dp_init(mp.mp_dp_default_params(force_int32=1), 0)
    yield c
    mp.mp_dp_destroy(c)


def _orc_params(orc, p):
    return orc.make_params(q=p.q, e=p.e, f=p.f, r=p.r, stop=p.stop,
                           mat=np.array([[p.mat[a][b] for b in range(22)] for a in range(22)]),
                           splice_model=p.splice_model, splice_p=p.splice_p)


def _compare(orc, pairs, got, params=None, limit=5):
    bad = []
    for k, (p, g) in enumerate(zip(pairs, got)):
        w = orc.align(p.prot, p.nt, p.strand, params)
        diff = [key for key in KEYS if g[key] != w[key]]
        if diff or g["status"] & 0xF0:
            bad.append((k, diff, {key: g[key] for key in diff}, {key: w[key] for key in diff},
                        g["status"], len(p.prot), len(p.nt)))
            if len(bad) >= limit:
                break
    assert not bad, bad


def _rand_prot(rng, n):
    return "".join(rng.choice("ARNDCQEGHILKMFPSTWYV") for _ in range(n))


def test_config1_parity(mp, ctx, ctx32, orc):
    p = synth.config1()
    for c in (ctx, ctx32):
        got = mp.mp_dp_align_batch(c, [p])
        _compare(orc, [p], got)


def test_tiny_pairs(mp, ctx, orc):
    rng = random.Random(5)
    srng = np.random.default_rng(5)
    pairs = []
    for _ in range(1000):
        m, n = rng.randint(1, 8), rng.randint(1, 40)
        prot = _rand_prot(rng, m)
        if rng.random() < 0.6:
            nt = synth.reverse_translate(srng, prot)
            pad = synth.random_dna(srng, max(0, n - len(nt)))
            k = rng.randint(0, len(pad))
            nt = pad[:k] + nt + pad[k:]
        else:
            nt = synth.random_dna(srng, n)
        pairs.append(synth.Pair(prot, nt, rng.choice((1, -1))))
    got = mp.mp_dp_align_batch(ctx, pairs)
    _compare(orc, pairs, got)


@pytest.mark.parametrize("pset", [dict(q=2, e=1, f=3, r=6, stop=2), dict(q=0, e=1, f=1, r=5, stop=4),
                                  dict(q=5, e=2, f=9, r=12, stop=11)])
def test_tiny_pairs_other_params(mp, orc, pset):
    """Cheap penalties make frameshifts, introns and ties frequent."""
    params = mp.mp_dp_default_params(**pset)
    c = mp.mp_dp_init(params, 0)
    try:
        rng = random.Random(hash(tuple(pset.values())) & 0xffff)
        srng = np.random.default_rng(rng.randint(0, 1 << 30))
        pairs = []
        for _ in range(400):
            prot = _rand_prot(rng, rng.randint(1, 12))
            nt = synth.random_dna(srng, rng.randint(1, 60))
            if rng.random() < 0.5:
                region, _ = synth.gen.plant_gene(srng, prot, 0.2, rng.randint(0, 2),
                                                 [rng.randint(8, 30)] if rng.random() < 0.6 else [], 5, 5)
                nt = region
            pairs.append(synth.Pair(prot, nt, 1))
        got = mp.mp_dp_align_batch(c, pairs)
        _compare(orc, pairs, got, _orc_params(orc, params))
    finally:
        mp.mp_dp_destroy(c)


def _gene_pairs(seed, count, mmax, intron_max):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        m = int(rng.integers(1, mmax + 1))
        prot = synth.random_protein(rng, m)
        k = int(rng.integers(0, 4))
        lens = [int(rng.integers(30, intron_max)) for _ in range(k)]
        region, _ = synth.gen.plant_gene(rng, prot, float(rng.uniform(0.05, 0.4)), int(rng.integers(0, 3)),
                                         lens, int(rng.integers(0, 300)), int(rng.integers(0, 300)), 0.45)
        strand = 1
        if rng.random() < 0.5:
            region = synth.revcomp(region)
            strand = -1
        out.append(synth.Pair(prot, region, strand))
    return out


def test_sizes_across_strips_and_chunks(mp, ctx, ctx32, orc):
    """1..300 residues (up to 5 strips, ragged last strip) against regions of
    up to a few kb (many 96-step chunks, ragged last chunk)."""
    pairs = _gene_pairs(11, 160, 300, 900)
    got = mp.mp_dp_align_batch(ctx, pairs)
    _compare(orc, pairs, got)
    got32 = mp.mp_dp_align_batch(ctx32, pairs)
    assert [{k: g[k] for k in KEYS} for g in got32] == [{k: g[k] for k in KEYS} for g in got]


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_wide_strips_match_oracle(mp, orc, mode):
    """Pairs run in 128-residue strips (four residues per lane) give the
    oracle's score, coordinates and CIGAR in every mode: proteins of 1 to
    1,200 residues (one to ten 128-residue strips, ragged last strips, and
    the lengths that stay in 64-residue strips), regions spanning many
    chunks, both strands, score-only pairs among them."""
    rng = np.random.default_rng(160 + mode)
    pairs = []
    for m in list(rng.integers(1, 1200, size=40)) + [64, 65, 128, 129, 256, 257, 1152]:
        prot = synth.random_protein(rng, int(m))
        lens = [int(rng.integers(40, 700)) for _ in range(int(rng.integers(0, 3)))]
        flank = 30 if mode else 400
        region, _ = synth.gen.plant_gene(rng, prot, float(rng.uniform(0.05, 0.35)), int(rng.integers(0, 3)), lens,
                                         int(rng.integers(0, flank)), int(rng.integers(0, flank)), 0.45)
        strand = 1
        if rng.random() < 0.5:
            region, strand = synth.revcomp(region), -1
        pairs.append(synth.Pair(prot, region, strand, score_only=bool(rng.random() < 0.1)))
    params = mp.mp_dp_default_params(mode=mode)
    op = _orc_params(orc, params)
    op.mode = mode
    c = mp.mp_dp_init(params, 0)
    try:
        mp.mp_dp_set_tuning(c, dict(dp16_variant=1, overlap_waves=1, item_order=1, strip_width=2))
        for _ in range(2):                                # direct, then graph replay
            got = mp.mp_dp_align_batch(c, pairs)
            bad = []
            for k, (p, g) in enumerate(zip(pairs, got)):
                w = orc.align(p.prot, p.nt, p.strand, op)
                keys = ("score", "prot_en") if p.score_only and mode != 1 else KEYS
                if any(g[x] != w[x] for x in keys) or g["status"] & 0xF0:
                    bad.append((k, len(p.prot), len(p.nt), [x for x in keys if g[x] != w[x]], g["status"]))
            assert not bad, bad[:5]
    finally:
        mp.mp_dp_destroy(c)


def test_boundary_lengths(mp, ctx, orc):
    """Protein lengths at strip edges and regions at chunk edges."""
    rng = np.random.default_rng(3)
    pairs = []
    for m in (1, 2, 31, 32, 33, 63, 64, 65, 127, 128, 129):
        for n in (1, 2, 3, 4, 33, 63, 64, 65, 95, 96, 97, 159, 160, 161, 191, 192, 193, 300):
            prot = synth.random_protein(rng, m)
            cds = synth.reverse_translate(rng, prot)
            nt = (cds + synth.random_dna(rng, n))[:n] if rng.random() < 0.5 else synth.random_dna(rng, n)
            pairs.append(synth.Pair(prot, nt, 1 if rng.random() < 0.5 else -1))
    got = mp.mp_dp_align_batch(ctx, pairs)
    _compare(orc, pairs, got)


def test_strands_agree(mp, ctx):
    pairs = _gene_pairs(21, 60, 200, 600)
    flipped = [synth.Pair(p.prot, synth.revcomp(p.nt), -p.strand) for p in pairs]
    a = mp.mp_dp_align_batch(ctx, pairs)
    b = mp.mp_dp_align_batch(ctx, flipped)
    for p, x, y in zip(pairs, a, b):
        n = len(p.nt)
        assert x["score"] == y["score"] and x["cigar"] == y["cigar"]
        assert (x["prot_st"], x["prot_en"]) == (y["prot_st"], y["prot_en"])
        assert (x["nt_st"], x["nt_en"]) == (n - y["nt_en"], n - y["nt_st"])


def test_int16_saturation_reruns_exactly(mp, ctx, orc):
    """Scores past the int16 range (W-rich proteins, W:W = 11) are re-run in
    int32 on the GPU and still match the oracle exactly."""
    rng = np.random.default_rng(9)
    pairs = []
    for m in (3200, 3400):
        prot = "".join("W" if rng.random() < 0.9 else "C" for _ in range(m))
        cds = synth.reverse_translate(rng, prot)
        nt = synth.random_dna(rng, 100) + cds[: 3 * 1400] + "GTAAGT" + synth.random_dna(rng, 200) + "CAG" + \
            cds[3 * 1400:] + synth.random_dna(rng, 80)
        pairs.append(synth.Pair(prot, nt, 1))
    pairs.append(_gene_pairs(5, 1, 100, 200)[0])
    got = mp.mp_dp_align_batch(ctx, pairs)
    assert got[0]["status"] & 1 and got[1]["status"] & 1 and not got[2]["status"] & 1
    assert got[0]["score"] > 32767
    _compare(orc, pairs, got)


def test_edge_cases(mp, ctx, orc):
    pairs = [synth.Pair("", "ACGTACGT", 1), synth.Pair("MW", "", 1), synth.Pair("W", "TG", 1),
             synth.Pair("W", "TGG", 1), synth.Pair("W", "tgg", -1), synth.Pair("WW", "TGG", 1),
             synth.Pair("mkvw", "atgaaagtttgg", 1), synth.Pair("M*XBZUW", "ATGTAAGGGGGGGGGGTGG", 1),
             synth.Pair("P", "AAAAAA", 1)]
    got = mp.mp_dp_align_batch(ctx, pairs)
    _compare(orc, pairs, got)
    bad = mp.mp_dp_align_batch(ctx, [synth.Pair("MW", "ATGNTGG", 1), synth.Pair("W", "TGG", 1)])
    assert bad[0]["status"] & mp.MP_ST_BADSEQ and bad[0]["score"] == 0
    assert bad[1]["status"] == 0 and bad[1]["score"] == 11


def test_maximum_sizes(mp, ctx, orc):
    """A region of the largest accepted length (1,047,551 nt) around a
    planted gene, and a protein of the largest accepted length (1,048,575
    residues) against a region carrying a slice of it on the minus strand:
    each aligns as the oracle aligns a window holding the planted copy
    (score, CIGAR, coordinates shifted back), and each CIGAR rescores by
    op-sum to the score.  One past either limit is rejected."""
    rng = np.random.default_rng(170)
    nmax, pmax = (1 << 20) - 1025, (1 << 20) - 1
    prot = synth.random_protein(rng, 220)
    gene, _ = synth.gen.plant_gene(rng, prot, 0.2, 1, [400, 900], 600, 600, 0.45)
    left = 400_000
    region = synth.random_dna(rng, left) + gene + synth.random_dna(rng, nmax - left - len(gene))
    big = synth.random_protein(rng, pmax)
    k0 = 700_000
    gene2, _ = synth.gen.plant_gene(rng, big[k0:k0 + 150], 0.15, 0, [300], 200, 200, 0.45)
    pairs = [synth.Pair(prot, region, 1), synth.Pair(big, synth.revcomp(gene2), -1)]
    assert len(region) == nmax and len(big) == pmax
    got = mp.mp_dp_align_batch(ctx, pairs)
    w0 = orc.align(prot, gene, 1)
    p0 = k0 - 300
    w1 = orc.align(big[p0:k0 + 450], synth.revcomp(gene2), -1)
    want = [dict(w0, nt_st=w0["nt_st"] + left, nt_en=w0["nt_en"] + left),
            dict(w1, prot_st=w1["prot_st"] + p0, prot_en=w1["prot_en"] + p0)]
    for p, g, w in zip(pairs, got, want):
        assert g["status"] & 0xF0 == 0
        assert w["score"] > 300
        assert {k: g[k] for k in KEYS} == {k: w[k] for k in KEYS}
        n = len(p.nt)
        st = g["nt_st"] if p.strand > 0 else n - g["nt_en"]
        en = g["nt_en"] if p.strand > 0 else n - g["nt_st"]
        assert orc.rescore(p.prot, p.nt, p.strand, g["prot_st"], st, g["cigar_raw"]) == \
            (g["score"], g["prot_en"], en)
    for bad in (synth.Pair(prot, region + "A", 1), synth.Pair(big + "W", gene2, 1)):
        with pytest.raises(mp.MPError):
            mp.mp_dp_align_batch(ctx, [bad])


def test_score_only_pairs(mp, ctx, orc):
    pairs = _gene_pairs(31, 30, 150, 400)
    so = [synth.Pair(p.prot, p.nt, p.strand, True) for p in pairs]
    full = mp.mp_dp_align_batch(ctx, pairs)
    got = mp.mp_dp_align_batch(ctx, so)
    for p, g, f in zip(pairs, got, full):
        assert g["score"] == f["score"] and g["cigar"] == [] and g["prot_en"] == f["prot_en"]
        if f["score"] > 0:
            assert (g["nt_en"] if p.strand > 0 else g["nt_st"]) == (f["nt_en"] if p.strand > 0 else f["nt_st"])


def test_plain_per_pair_launches(mp, orc):
    pairs = _gene_pairs(41, 12, 200, 500)
    c = mp.mp_dp_init(mp.mp_dp_default_params(max_pairs_per_launch=1), 0)
    try:
        got = mp.mp_dp_align_batch(c, pairs)
        _compare(orc, pairs, got)
    finally:
        mp.mp_dp_destroy(c)


def test_repeated_runs_and_graph_replay(mp, ctx):
    pairs = _gene_pairs(51, 50, 250, 700)
    b = mp.mp_dp_batch_upload(ctx, pairs)
    try:
        outs = []
        for _ in range(4):               # run 1 direct, runs 2+ replay the captured graph
            mp.mp_dp_batch_run(ctx, b)
            mp.mp_dp_batch_sync(ctx)
            outs.append([{k: g[k] for k in KEYS} for g in mp.mp_dp_batch_download(ctx, b)])
        assert all(o == outs[0] for o in outs)
        assert outs[0] == [{k: g[k] for k in KEYS} for g in mp.mp_dp_align_batch(ctx, pairs)]
    finally:
        mp.mp_dp_batch_free(ctx, b)


def _code_bytes(m, n):
    """Traceback bytes of one pair: per 64-residue strip and 96-step chunk,
    128 B per step of H values plus 128 B of column maxima."""
    return -(-m // 64) * -(-(n + 63) // 96) * (96 * 128 + 128)


def test_small_budget_waves(mp, ctx, orc):
    """A budget smaller than the batch splits it into waves; a pair larger
    than the whole budget is scored without traceback (MP_ST_BUDGET)."""
    pairs = _gene_pairs(61, 40, 300, 800)
    need = sorted(_code_bytes(len(p.prot), len(p.nt)) for p in pairs)
    budget = need[-3] + 4096                      # the two largest pairs do not fit
    c = mp.mp_dp_init(mp.mp_dp_default_params(tb_budget_bytes=budget), 0)
    try:
        got = mp.mp_dp_align_batch(c, pairs)
        ref = mp.mp_dp_align_batch(ctx, pairs)
        for g, r, p in zip(got, ref, pairs):
            if _code_bytes(len(p.prot), len(p.nt)) > budget:
                assert g["status"] & mp.MP_ST_BUDGET
                assert g["score"] == r["score"] and g["prot_en"] == r["prot_en"]
            else:
                assert not g["status"] & mp.MP_ST_BUDGET
                assert {k: g[k] for k in KEYS} == {k: r[k] for k in KEYS}
        assert sum(1 for g in got if g["status"] & mp.MP_ST_BUDGET) == 2
        assert mp.mp_dp_get_stats(c)["n_waves"] > 1
        _compare(orc, pairs[:8], ref[:8])
    finally:
        mp.mp_dp_destroy(c)


def test_overlapped_waves(mp, ctx):
    """A batch needing several waves, with every pair under half the budget:
    with overlapped waves (the default) they alternate between two streams
    over two arena halves; without, they run one after the other at the
    whole budget.  Either way, with either item order, and switching between
    them on one batch (which re-plans it), the results equal the one-wave
    run, direct and replayed as a graph, with timing on."""
    pairs = _gene_pairs(63, 60, 300, 900)
    need = [_code_bytes(len(p.prot), len(p.nt)) for p in pairs]
    budget = max(3 * max(need), sum(need) // 3)
    ref = mp.mp_dp_align_batch(ctx, pairs)
    want = [{k: r[k] for k in KEYS} for r in ref]
    c = mp.mp_dp_init(mp.mp_dp_default_params(tb_budget_bytes=budget), 0)
    try:
        mp.mp_dp_set_timing(c, True)
        b = mp.mp_dp_batch_upload(c, pairs)
        waves = {}
        for ov, io in ((1, 1), (0, 1), (1, 0), (0, 0), (1, 1)):
            mp.mp_dp_set_tuning(c, dict(overlap_waves=ov, item_order=io))
            for _ in range(3):
                mp.mp_dp_batch_run(c, b)
                mp.mp_dp_batch_sync(c)
                got = mp.mp_dp_batch_download(c, b)
                assert [{k: g[k] for k in KEYS} for g in got] == want
                st = mp.mp_dp_get_stats(c)
                assert st["total_ms"] > 0 and st["dp_ms"] > 0
                waves[ov] = st["n_waves"]
        assert waves[1] >= 4 and 2 <= waves[0] < waves[1]
        mp.mp_dp_batch_free(c, b)
    finally:
        mp.mp_dp_destroy(c)


@pytest.mark.parametrize("splice_p", [0, 12, 30])
def test_simple_splice_model(mp, orc, splice_p):
    """The simple GT-AG splice model (cost p for a donor without GT or an
    acceptor without AG): gene pairs whose introns keep GT...AG or have their
    signals replaced, both strands, plus an int16-saturating pair (int32
    re-run), against the oracle under the same model."""
    rng = np.random.default_rng(80 + splice_p)
    pairs = []
    for k in range(40):
        m = int(rng.integers(20, 260))
        prot = synth.random_protein(rng, m)
        lens = [int(rng.integers(40, 700)) for _ in range(int(rng.integers(1, 4)))]
        if k % 2 == 0:
            region, _ = synth.gen.plant_gene(rng, prot, float(rng.uniform(0.05, 0.3)), int(rng.integers(0, 2)),
                                             lens, int(rng.integers(0, 200)), int(rng.integers(0, 200)), 0.45)
        else:
            # introns whose ends are neither GT nor AG
            cds = synth.reverse_translate(rng, prot)
            cuts = sorted(int(x) for x in rng.choice(np.arange(1, len(cds)), size=len(lens), replace=False))
            pieces, prev = [synth.random_dna(rng, int(rng.integers(0, 200)))], 0
            for cut, L in zip(cuts, lens):
                ends = [str(x) for x in rng.choice(["CA", "TC", "AA", "CC", "TT"], size=2)]
                pieces += [cds[prev:cut], ends[0] + synth.random_dna(rng, L - 4) + ends[1]]
                prev = cut
            pieces += [cds[prev:], synth.random_dna(rng, int(rng.integers(0, 200)))]
            region = "".join(pieces)
        strand = 1
        if rng.random() < 0.5:
            region, strand = synth.revcomp(region), -1
        pairs.append(synth.Pair(prot, region, strand))
    prot = "".join("W" if rng.random() < 0.9 else "C" for _ in range(3200))
    cds = synth.reverse_translate(rng, prot)
    pairs.append(synth.Pair(prot, synth.random_dna(rng, 60) + cds[:4800] + "GTAAGT" + synth.random_dna(rng, 120) +
                            "TAG" + cds[4800:] + synth.random_dna(rng, 40), 1))
    params = mp.mp_dp_default_params(splice_model=mp.MP_SPLICE_SIMPLE, splice_p=splice_p)
    c = mp.mp_dp_init(params, 0)
    try:
        got = mp.mp_dp_align_batch(c, pairs)
        got2 = mp.mp_dp_align_batch(c, pairs)             # graph replay
    finally:
        mp.mp_dp_destroy(c)
    assert got[-1]["status"] & 1                          # re-run in int32
    _compare(orc, pairs, got, _orc_params(orc, params))
    assert [{k: g[k] for k in KEYS} for g in got2] == [{k: g[k] for k in KEYS} for g in got]


def test_exon_rescore(mp, ctx, orc):
    """Pseudogene-aware scores: spliced genes, their processed (intron-free)
    copies, both strands, and pairs without an alignment; the library's
    exon_score equals the oracle's, from mp_dp_align_batch with
    params.exon_rescore and from mp_dp_exon_rescore on earlier results."""
    rng = np.random.default_rng(90)
    pairs = _gene_pairs(91, 24, 300, 900)
    for k in range(8):
        prot = synth.random_protein(rng, int(rng.integers(40, 300)))
        cds_only, _ = synth.gen.plant_gene(rng, prot, float(rng.uniform(0.05, 0.3)), 0, [],
                                           int(rng.integers(0, 200)), int(rng.integers(0, 200)), 0.45)
        strand = 1 if k % 2 == 0 else -1
        pairs.append(synth.Pair(prot, cds_only if strand > 0 else synth.revcomp(cds_only), strand))
    pairs.append(synth.Pair("WWWWWW", "A" * 60, 1))
    want = [orc.exon_score(p.prot, p.nt, p.strand) for p in pairs]
    c = mp.mp_dp_init(mp.mp_dp_default_params(exon_rescore=1), 0)
    try:
        got = mp.mp_dp_align_batch(c, pairs)
        got2 = mp.mp_dp_align_batch(c, pairs)
    finally:
        mp.mp_dp_destroy(c)
    assert [g["exon_score"] for g in got] == want
    assert [g["exon_score"] for g in got2] == want
    _compare(orc, pairs[:6], got[:6])                     # the alignments themselves are untouched
    plain = mp.mp_dp_align_batch(ctx, pairs)
    assert [g["exon_score"] for g in plain] == [g["score"] for g in plain]
    assert mp.mp_dp_exon_rescore(ctx, pairs, plain) == want
    # a single-exon alignment is also the best one inside its own region: its
    # exon score is its score less r
    for k in range(24, 32):
        assert got[k]["score"] == 0 or (not any(op in "NUV" for op, _ in got[k]["cigar"]) and
                                        want[k] == got[k]["score"] - 29)


def _anchored_pairs(seed, count, mmax):
    """Gene pairs with short flanks (the gap-closing and extension regions
    between anchors are short), several strips and chunks, both strands."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        m = int(rng.integers(1, mmax + 1))
        prot = synth.random_protein(rng, m)
        lens = [int(rng.integers(40, 600)) for _ in range(int(rng.integers(0, 3)))]
        region, _ = synth.gen.plant_gene(rng, prot, float(rng.uniform(0.0, 0.35)), int(rng.integers(0, 3)), lens,
                                         int(rng.integers(0, 40)), int(rng.integers(0, 40)), 0.45)
        strand = 1
        if rng.random() < 0.5:
            region, strand = synth.revcomp(region), -1
        out.append(synth.Pair(prot, region, strand))
    # unrelated protein and region: negative global scores
    for _ in range(3):
        m = int(rng.integers(20, 150))
        out.append(synth.Pair(synth.random_protein(rng, m), synth.random_dna(rng, int(rng.integers(50, 900))), 1))
    return out


@pytest.mark.parametrize("mode", [0, 1, 2])
@pytest.mark.parametrize("kernel", ["int16", "int16-w128", "int32"])
def test_stored_h_matches_oracle(mp, orc, mode, kernel):
    """Every stored H value of Eq. 7 (read back from the traceback stream,
    with the mode's row 0 and column 0) equals the oracle's H matrix, cell
    by cell, for pairs spanning several strips and chunks, both strands,
    in the int16 kernel (64- and 128-residue strips) and the int32 kernel."""
    pairs = _anchored_pairs(140 + mode, 6, 300 if kernel == "int16-w128" else 150)
    params = mp.mp_dp_default_params(mode=mode, force_int32=1 if kernel == "int32" else 0)
    op = _orc_params(orc, params)
    op.mode = mode
    c = mp.mp_dp_init(params, 0)
    try:
        if kernel == "int16-w128":
            mp.mp_dp_set_tuning(c, dict(dp16_variant=1, overlap_waves=1, item_order=1, strip_width=2))
        b = mp.mp_dp_batch_upload(c, pairs)
        mp.mp_dp_batch_run(c, b)
        mp.mp_dp_batch_sync(c)
        report = []
        for k, p in enumerate(pairs):
            got = mp.mp_dp_debug_h(c, b, k, len(p.nt), len(p.prot))
            want = orc.fill_h(p.prot, p.nt, p.strand, op)
            bad = np.argwhere(got != want)
            if bad.size:
                report.append(f"pair {k} |T|={len(p.nt)} |P|={len(p.prot)} strand={p.strand} bad={len(bad)} "
                              f"col0 {got[:10, 0].tolist()} want {want[:10, 0].tolist()} "
                              f"row1 {got[1, :6].tolist()} want {want[1, :6].tolist()} "
                              f"first {[(int(i), int(j), int(got[i, j]), int(want[i, j])) for i, j in bad[:4]]}")
        mp.mp_dp_batch_free(c, b)
        assert not report, "\n".join(report)
    finally:
        mp.mp_dp_destroy(c)


@pytest.mark.parametrize("pset", [dict(), dict(q=3, e=2, f=5, r=9, stop=4, splice_model=1, splice_p=7),
                                  dict(q=0, e=1, f=9, r=12, stop=4), dict(q=11, e=3, f=17, r=40, splice_model=1)])
def test_column0_against_oracle(mp, orc, pset):
    """Column 0 of the anchored modes (Eq. 7 with no residue consumed: D
    runs, G1, G2 and introns from row 0) against the oracle's, for regions of
    1 to 9,000 nt dense in GT and AG (so that the intron terms compete), with
    several penalty sets and both splice models; column 0 is the kernel that
    splits its rows into 32 segments and chains them."""
    rng = np.random.default_rng(171)
    pairs = []
    for n in (1, 2, 3, 5, 31, 32, 33, 95, 96, 97, 200, 511, 700, 1500, 4000, 9000):
        t = list(synth.random_dna(rng, n))
        i = 0
        while i + 1 < n:
            t[i:i + 2] = "AG" if rng.random() < 0.5 else "GT"
            i += int(rng.integers(7, 18))
        pairs.append(synth.Pair("M", "".join(t), 1))
    params = mp.mp_dp_default_params(mode=1, **pset)
    op = _orc_params(orc, params)
    op.mode = 1
    c = mp.mp_dp_init(params, 0)
    try:
        b = mp.mp_dp_batch_upload(c, pairs)
        mp.mp_dp_batch_run(c, b)
        mp.mp_dp_batch_sync(c)
        bad = []
        for k, p in enumerate(pairs):
            got = mp.mp_dp_debug_h(c, b, k, len(p.nt), 1)[:, 0]
            want = orc.fill_h(p.prot, p.nt, 1, op)[:, 0]
            rows = np.nonzero(got != want)[0]
            if rows.size:
                bad.append((len(p.nt), int(rows[0]), int(got[rows[0]]), int(want[rows[0]]), int(rows.size)))
        mp.mp_dp_batch_free(c, b)
    finally:
        mp.mp_dp_destroy(c)
    assert not bad, bad


@pytest.mark.parametrize("mode", [1, 2])
@pytest.mark.parametrize("splice_model", [0, 1])
def test_anchored_modes(mp, orc, mode, splice_model):
    """Global (gap closing: from the start of protein and region to both
    ends) and extension (from the start, ending anywhere) against the oracle:
    score, coordinates and CIGAR, with both splice models, the graph replay
    and score-only requests (which global mode still traces)."""
    pairs = _anchored_pairs(100 + mode + 10 * splice_model, 30, 300)
    params = mp.mp_dp_default_params(mode=mode, splice_model=splice_model, splice_p=15)
    c = mp.mp_dp_init(params, 0)
    try:
        got = mp.mp_dp_align_batch(c, pairs)
        got2 = mp.mp_dp_align_batch(c, pairs)
        so = mp.mp_dp_align_batch(c, [synth.Pair(p.prot, p.nt, p.strand, True) for p in pairs[:6]])
    finally:
        mp.mp_dp_destroy(c)
    op = _orc_params(orc, params)
    op.mode = mode
    _compare(orc, pairs, got, op)
    assert [{k: g[k] for k in KEYS} for g in got2] == [{k: g[k] for k in KEYS} for g in got]
    if mode == 1:
        assert min(g["score"] for g in got) < 0
        assert [g["score"] for g in so] == [g["score"] for g in got[:6]]
    else:
        assert [g["score"] for g in so] == [g["score"] for g in got[:6]]


@pytest.mark.parametrize("mode", [1, 2])
def test_anchored_modes_across_configurations(mp, orc, mode):
    """The global and extension modes under both int16 builds, both item
    orders and both wave policies, in a budget that needs several waves:
    results equal the oracle's, direct and replayed as a graph."""
    pairs = _anchored_pairs(130 + mode, 36, 260)
    need = [_code_bytes(len(p.prot), len(p.nt)) for p in pairs]
    budget = max(3 * max(need), sum(need) // 3)
    params = mp.mp_dp_default_params(mode=mode, tb_budget_bytes=budget)
    op = _orc_params(orc, params)
    op.mode = mode
    want = [orc.align(p.prot, p.nt, p.strand, op) for p in pairs]
    c = mp.mp_dp_init(params, 0)
    try:
        for v, ov, io in ((0, 1, 1), (1, 1, 0), (0, 0, 1), (1, 0, 0)):
            mp.mp_dp_set_tuning(c, dict(dp16_variant=v, overlap_waves=ov, item_order=io))
            for _ in range(2):
                got = mp.mp_dp_align_batch(c, pairs)
                bad = [k for k, (g, w) in enumerate(zip(got, want))
                       if any(g[key] != w[key] for key in KEYS) or g["status"] & 0xF0]
                assert not bad, (v, ov, io, bad[:5])
            assert mp.mp_dp_get_stats(c)["n_waves"] >= 2
    finally:
        mp.mp_dp_destroy(c)


def test_anchored_serving(mp, orc):
    """Requests served in global mode give the batch call's results."""
    pairs = _anchored_pairs(150, 24, 200)
    params = mp.mp_dp_default_params(mode=1)
    c = mp.mp_dp_init(params, 0)
    try:
        ref = mp.mp_dp_align_batch(c, pairs)
        tickets = [mp.mp_dp_submit(c, p) for p in pairs]
        got = {}
        while len(got) < len(tickets):
            r = mp.mp_dp_wait_any(c, 5_000_000)
            assert r is not None
            got[r[0]] = r[1]
        for t, r in zip(tickets, ref):
            assert {x: got[t][x] for x in KEYS} == {x: r[x] for x in KEYS}
    finally:
        mp.mp_dp_destroy(c)
    op = _orc_params(orc, params)
    op.mode = 1
    _compare(orc, pairs[:8], ref[:8], op)


def test_anchored_lower_bound_refused(mp):
    """An anchored pair whose H could fall below -2^27 (large gap extension
    and a long protein) is refused as a whole batch; the same pair in local
    mode (H never below 0) is accepted and scored."""
    rng = np.random.default_rng(172)
    prot = synth.random_protein(rng, 140_000)
    pair = synth.Pair(prot, "ATGGCCAAGTGG", 1)
    for mode in (1, 2):
        c = mp.mp_dp_init(mp.mp_dp_default_params(mode=mode, q=0, e=1000, f=5, r=10, stop=5), 0)
        try:
            with pytest.raises(mp.MPError):
                mp.mp_dp_align_batch(c, [pair])
        finally:
            mp.mp_dp_destroy(c)
    c = mp.mp_dp_init(mp.mp_dp_default_params(q=0, e=1000, f=5, r=10, stop=5), 0)
    try:
        got = mp.mp_dp_align_batch(c, [pair])
        assert got[0]["status"] & 0xF0 == 0
    finally:
        mp.mp_dp_destroy(c)


def test_anchored_int32_pairs(mp, orc):
    """Anchored pairs whose lower bound leaves the int16 range run in int32
    at once (here by a large gap extension e), against the oracle."""
    rng = np.random.default_rng(120)
    pairs = []
    for k in range(4):
        m = int(rng.integers(900, 1100))
        prot = synth.random_protein(rng, m)
        region, _ = synth.gen.plant_gene(rng, prot, 0.2, 1, [300], 500, 500, 0.45)
        pairs.append(synth.Pair(prot, region, 1 if k % 2 == 0 else -1))
    for mode in (1, 2):
        params = mp.mp_dp_default_params(mode=mode, e=6, q=9)
        c = mp.mp_dp_init(params, 0)
        try:
            got = mp.mp_dp_align_batch(c, pairs)
        finally:
            mp.mp_dp_destroy(c)
        op = _orc_params(orc, params)
        op.mode = mode
        _compare(orc, pairs, got, op)


def test_serving_alone_and_in_mix(mp, ctx):
    """Each request's result is the same served alone, in a burst with
    others in flight, and from the batch call."""
    pairs = _gene_pairs(71, 80, 250, 700)
    ref = mp.mp_dp_align_batch(ctx, pairs)
    c = mp.mp_dp_init(None, 0)
    try:
        alone = []
        for p in pairs[:10]:
            t = mp.mp_dp_submit(c, p)
            r = mp.mp_dp_poll(c, t, 30_000_000)
            assert r is not None
            alone.append(r)
        tickets = [mp.mp_dp_submit(c, p) for p in pairs]
        mix = {}
        while len(mix) < len(tickets):
            r = mp.mp_dp_wait_any(c, 5_000_000)
            assert r is not None
            mix[r[0]] = r[1]
        for k in range(10):
            assert {x: alone[k][x] for x in KEYS} == {x: ref[k][x] for x in KEYS}
        for t, r in zip(tickets, ref):
            assert {x: mix[t][x] for x in KEYS} == {x: r[x] for x in KEYS}
        assert mp.lib().mp_dp_poll(c, tickets[0], ctypes.byref(mp.mp_result()), 0) == mp.MP_ETICKET
    finally:
        mp.mp_dp_destroy(c)


def test_serving_admits_requests_up_to_the_whole_budget(mp, orc):
    """A request whose traceback exceeds a third of the budget (a slot's
    share) but fits the whole budget is served, alone and among small
    requests, with the batch call's result; one beyond the budget is
    refused with MP_EBUDGET."""
    rng = np.random.default_rng(77)
    prot = synth.random_protein(rng, 900)
    big, _ = synth.gen.plant_gene(rng, prot, 0.2, 1, [700, 2500], 3000, 3000, 0.4)
    big_pair = synth.Pair(prot, big, 1)
    # traceback bytes of the big pair: about 2 bytes per cell (here ~ 28 MB)
    budget = int(2.6 * big_pair.cells) + (4 << 20)
    assert 2 * big_pair.cells > budget / 3
    small = _gene_pairs(91, 30, 120, 300)
    params = mp.mp_dp_default_params(tb_budget_bytes=budget)
    c = mp.mp_dp_init(params, 0)
    try:
        want = mp.mp_dp_align_batch(c, [big_pair] + small)
        t = mp.mp_dp_submit(c, big_pair)
        r = mp.mp_dp_poll(c, t, 60_000_000)
        assert r is not None and {x: r[x] for x in KEYS} == {x: want[0][x] for x in KEYS}
        assert r["status"] & 0xF0 == 0
        tickets = [mp.mp_dp_submit(c, p) for p in small[:10]] + [mp.mp_dp_submit(c, big_pair)] + \
                  [mp.mp_dp_submit(c, p) for p in small[10:]]
        got = {}
        while len(got) < len(tickets):
            x = mp.mp_dp_wait_any(c, 30_000_000)
            assert x is not None
            got[x[0]] = x[1]
        order = small[:10] + [big_pair] + small[10:]
        refs = want[1:11] + [want[0]] + want[11:]
        for tk, r in zip(tickets, refs):
            assert {x: got[tk][x] for x in KEYS} == {x: r[x] for x in KEYS}
        w = orc.align(big_pair.prot, big_pair.nt, 1)
        assert {x: want[0][x] for x in KEYS} == {x: w[x] for x in KEYS}
        huge = synth.Pair(prot + prot, big + big, 1)
        with pytest.raises(mp.MPError):
            mp.mp_dp_submit(c, huge)
        assert len(order) == len(tickets)
    finally:
        mp.mp_dp_destroy(c)


def test_cooperating_wait_runs_out_without_fault(mp, ctx, orc):
    """Failure detection without a GPU fault: with every boundary row
    withheld, each warp waiting on the previous strip of its pair gives up
    after a short poll limit; the kernel completes, multi-strip pairs are
    reported MP_ST_TIMEOUT, single-strip pairs are unaffected, and the
    context and device stay usable."""
    pairs = _gene_pairs(81, 24, 300, 500)
    c = mp.mp_dp_init(mp.mp_dp_default_params(wait_limit=2000, debug_flags=mp.MP_DEBUG_NO_PUBLISH), 0)
    try:
        got = mp.mp_dp_align_batch(c, pairs)
        for p, g in zip(pairs, got):
            if len(p.prot) > 64:
                assert g["status"] & mp.MP_ST_TIMEOUT
            else:
                assert not g["status"] & 0xF0
        again = mp.mp_dp_align_batch(ctx, pairs)
        _compare(orc, pairs[:6], again[:6])
        assert any(len(p.prot) > 64 for p in pairs) and any(len(p.prot) <= 64 for p in pairs)
    finally:
        mp.mp_dp_destroy(c)


def _profile_for(orc, rng, prot, diag=None, jitter=2):
    """A profile query for `prot`: BLOSUM62's row of each residue perturbed
    per position (diag: the residue's own score replaced by that value), a
    stop-codon score, and random gap costs per column."""
    B = orc.blosum62_22()
    m = len(prot)
    prof = np.zeros((m + 1, 23), dtype=np.int32)
    for j in range(1, m + 1):
        pc = orc.AA.index(prot[j - 1]) if prot[j - 1] in orc.AA else 21
        prof[j, :20] = B[:20, pc] + rng.integers(-jitter, jitter + 1, size=20)
        if diag is not None and pc < 20:
            prof[j, pc] = diag
        prof[j, 20] = -int(rng.integers(10, 25))
    prof[:, 21] = rng.integers(4, 16, size=m + 1)
    prof[:, 22] = rng.integers(1, 4, size=m + 1)
    return prof


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_profile_queries_match_oracle(mp, orc, mode):
    """Profile queries (position-specific substitution scores and gap costs)
    give the oracle's score, coordinates and CIGAR in every mode, in the
    int16 kernel and the int32 kernel, with pseudogene-aware rescoring in
    local mode; a profile holding the default scoring reproduces the
    unprofiled results; a pair whose profile can pass the int16 range is
    re-run exactly; a profile whose scores break the intron rule is
    refused."""
    rng = np.random.default_rng(180 + mode)
    pairs = []
    for k in range(36):
        m = int(rng.integers(1, 320))
        prot = synth.random_protein(rng, m)
        lens = [int(rng.integers(40, 600)) for _ in range(int(rng.integers(0, 3)))]
        flank = 30 if mode else 300
        region, _ = synth.gen.plant_gene(rng, prot, float(rng.uniform(0.05, 0.35)), int(rng.integers(0, 3)), lens,
                                         int(rng.integers(0, flank)), int(rng.integers(0, flank)), 0.45)
        strand = 1
        if rng.random() < 0.5:
            region, strand = synth.revcomp(region), -1
        pairs.append(synth.Pair(prot, region, strand, profile=_profile_for(orc, rng, prot)))
    # a profile whose scores can pass the int16 range (re-run in int32)
    prot = synth.random_protein(rng, 420)
    region, _ = synth.gen.plant_gene(rng, prot, 0.0, 0, [300], 50, 50, 0.45)
    pairs.append(synth.Pair(prot, region, 1, profile=_profile_for(orc, rng, prot, diag=80)))
    # the default scoring as a profile
    plain = _gene_pairs(181, 8, 200, 500)
    base = mp.mp_dp_default_params(mode=mode)
    op = _orc_params(orc, base)
    op.mode = mode
    for p in plain:
        pairs.append(synth.Pair(p.prot, p.nt, p.strand, profile=orc.profile_of(p.prot, op)))
    for force in (0, 1):
        params = mp.mp_dp_default_params(mode=mode, force_int32=force, exon_rescore=1 if mode == 0 else 0)
        c = mp.mp_dp_init(params, 0)
        try:
            got = mp.mp_dp_align_batch(c, pairs)
            ref_plain = mp.mp_dp_align_batch(c, plain)
        finally:
            mp.mp_dp_destroy(c)
        bad = []
        for k, (p, g) in enumerate(zip(pairs, got)):
            pp = orc.make_params(mode=mode, prof=p.profile)
            w = orc.align(p.prot, p.nt, p.strand, pp)
            if any(g[x] != w[x] for x in KEYS) or g["status"] & 0xF0:
                bad.append((k, len(p.prot), [x for x in KEYS if g[x] != w[x]], g["status"]))
            elif mode == 0 and g["exon_score"] != orc.exon_score(p.prot, p.nt, p.strand, pp, w):
                bad.append((k, "exon_score", g["exon_score"]))
        assert not bad, (force, bad[:5])
        for g, r in zip(got[-len(plain):], ref_plain):
            assert {x: g[x] for x in KEYS} == {x: r[x] for x in KEYS}
        if not force and mode == 0:
            # local mode runs it in int16 first (the anchored modes send it to int32 at once)
            assert got[-len(plain) - 1]["status"] & mp.MP_ST_RERUN
    # serving takes the profile with the request
    c = mp.mp_dp_init(mp.mp_dp_default_params(mode=mode), 0)
    try:
        for p in pairs[:3]:
            t = mp.mp_dp_submit(c, p)
            r = mp.mp_dp_poll(c, t, 30_000_000)
            w = orc.align(p.prot, p.nt, p.strand, orc.make_params(mode=mode, prof=p.profile))
            assert {x: r[x] for x in KEYS} == {x: w[x] for x in KEYS}
        bad_prof = pairs[0].profile.copy()
        bad_prof[1, 3] = -40                       # r = 29 must exceed every negated score
        with pytest.raises(mp.MPError):
            mp.mp_dp_align_batch(c, [synth.Pair(pairs[0].prot, pairs[0].nt, pairs[0].strand, profile=bad_prof)])
    finally:
        mp.mp_dp_destroy(c)
