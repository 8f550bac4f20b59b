"""Seeding and chaining on the GPU against the oracle (Li 2022, Methods:
"Reduced alphabet", "Indexing the genome", "Chaining").

* The index of a genome with planted coding sequences on both strands and a
  stretch of non-ACGT letters equals the oracle's CSR table entry for entry.
* Every protein of the genome-scale workload shrunk 50 times (10 Mb genome,
  4,000 proteins) gets the oracle's chains, field by field, and the same
  number of chains (the first 3 and the first 30 of each).
* The candidate regions of those chains, aligned by the batch DP, match the
  oracle (the DP parity of the genome-scale workload is covered in
  test_gpu_genome).
* The second chaining round ("Chaining", last paragraph) gives every pair
  the oracle's best chain: synthetic pairs (planted genes with introns and
  frameshifts on either strand, unrelated regions, non-ACGT letters, pairs
  shorter than a 5-mer) and every candidate region of the shrunk workload.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

FIELDS = ("strand", "n_anchors", "score", "x_first", "x_last", "y_first", "y_last")


@pytest.fixture(scope="module")
def mp():
    from paper_2210_08052_gb300 import build
    build.build()
    import paper_2210_08052_gb300 as m
    m.lib()
    return m


def test_index_matches_oracle(mp, orc):
    rng = np.random.default_rng(21)
    parts = []
    for _ in range(30):
        parts.append(synth.random_dna(rng, int(rng.integers(20_000, 120_000)), 0.4))
        prot = synth.random_protein(rng, int(rng.integers(60, 600)))
        gene, _ = synth.gen.plant_gene(rng, prot, 0.1, 0, [int(rng.integers(80, 2000))], 0, 0, 0.4)
        parts.append(gene if rng.random() < 0.5 else synth.revcomp(gene))
    parts.append("ACGTNNNNNNACGTRYACGT" * 50)
    genome = "".join(parts)
    ctx = mp.mp_dp_init(None, 0)
    try:
        idx = mp.mp_index_build(ctx, genome)
        try:
            off, ent = mp.mp_index_download(ctx, idx)
        finally:
            mp.mp_index_free(idx)
        empty = mp.mp_index_build(ctx, "")
        eo, ee = mp.mp_index_download(ctx, empty)
        mp.mp_index_free(empty)
    finally:
        mp.mp_dp_destroy(ctx)
    woff, went = orc.build_index(genome)
    assert len(ent) == len(went) > 100_000
    assert (off == woff).all()
    assert (ent == went).all()
    assert not eo.any() and len(ee) == 0


@pytest.fixture(scope="module")
def genome_workload():
    return synth.config5(scale=0.02, host_seeding=False)


@pytest.mark.parametrize("top", [3, 30])
def test_chains_match_oracle(mp, orc, genome_workload, top):
    w = genome_workload
    ctx = mp.mp_dp_init(None, 0)
    try:
        idx = mp.mp_index_build(ctx, w.genome)
        try:
            chains, nch = mp.mp_index_chain(ctx, idx, w.prot_buf, w.prot_off, w.prot_len, top)
        finally:
            mp.mp_index_free(idx)
    finally:
        mp.mp_dp_destroy(ctx)
    off, pos = orc.build_index(w.genome.tobytes())
    bad = []
    total = 0
    for k in range(len(w.prot_len)):
        want, _ = orc.chain(orc.anchors(off, pos, w.protein(k)), top)
        total += len(want)
        if int(nch[k]) != len(want):
            bad.append((k, int(nch[k]), len(want)))
            continue
        for t, c in enumerate(want):
            got = {f: int(chains[k, t][f]) for f in FIELDS}
            if got != c:
                bad.append((k, t, got, c))
                break
    assert not bad, (len(bad), bad[:3])
    assert total > len(w.prot_len)
    # the planted genes' sources find their genes: the best chain of most
    # sources lies on the gene's strand and inside its bins
    src = np.flatnonzero(w.kind == 0)
    hit = 0
    for k in src:
        if nch[k] == 0:
            continue
        c = chains[k, 0]
        g = int(w.gene_of[k])
        G = len(w.genome)
        lo, hi = int(w.gene_start[g]), int(w.gene_end[g])
        if w.gene_strand[g] < 0:
            lo, hi = G - hi, G - lo
        hit += int(c["strand"] == (0 if w.gene_strand[g] > 0 else 1) and lo // 256 - 1 <= c["x_first"] and
                   c["x_last"] <= hi // 256 + 1)
    assert hit > 0.9 * len(src), (hit, len(src))


REFINE_FIELDS = ("n_anchors", "score", "x_first", "x_last", "y_first", "y_last")


def _refine_compare(mp, orc, pairs):
    import os
    from concurrent.futures import ThreadPoolExecutor

    ctx = mp.mp_dp_init(None, 0)
    try:
        got = mp.mp_chain_refine(ctx, pairs)
    finally:
        mp.mp_dp_destroy(ctx)
    # the oracle on every host core (its C calls release the interpreter lock)
    with ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        want = list(ex.map(lambda p: orc.refine(p.prot, p.nt, p.strand), pairs))
    bad = []
    for k, w in enumerate(want):
        g = {f: int(got[k][f]) for f in REFINE_FIELDS}
        if g != w:
            bad.append((k, g, w))
    assert not bad, (len(bad), bad[:3])
    return got


def test_refine_matches_oracle(mp, orc):
    """Second chaining round: every pair's best chain equals the oracle's,
    field by field — planted genes on both strands with introns and
    frameshifts, unrelated regions, pairs too short for a 5-mer, regions
    with letters outside ACGT."""
    rng = np.random.default_rng(33)
    pairs = []
    for t in range(120):
        prot = synth.random_protein(rng, int(rng.integers(6, 700)))
        kind = t % 4
        if kind == 3:
            nt = synth.random_dna(rng, int(rng.integers(15, 4000)), 0.4)
        else:
            introns = [int(rng.integers(80, 900)) for _ in range(int(rng.integers(0, 3)))]
            nt, _ = synth.gen.plant_gene(rng, prot, float(rng.uniform(0.0, 0.4)), int(rng.integers(0, 3)),
                                         introns, int(rng.integers(0, 800)), int(rng.integers(0, 800)), 0.4)
        if kind == 2 and len(nt) > 40:
            cut = int(rng.integers(10, len(nt) - 20))
            nt = nt[:cut] + "NNRY" + nt[cut:]
        strand = 1 if rng.random() < 0.5 else -1
        if strand < 0:
            nt = synth.revcomp(nt)
        pairs.append(synth.Pair(prot, nt, strand))
    pairs.append(synth.Pair("MKV", "ATGAAAGTT", 1))              # shorter than one 5-mer
    pairs.append(synth.Pair("MKVLA", "ATGAAAGTTCT", -1))
    got = _refine_compare(mp, orc, pairs)
    assert (got["n_anchors"] > 0).sum() > 80


def test_refine_genome_regions_match_oracle(mp, orc, genome_workload):
    """The candidate regions of the first round's chains (the genome-scale
    workload shrunk 50 times: about 12,000 regions), refined: every region
    equals the oracle."""
    w = genome_workload
    ctx = mp.mp_dp_init(None, 0)
    try:
        idx = mp.mp_index_build(ctx, w.genome)
        try:
            chains, nch = mp.mp_index_chain(ctx, idx, w.prot_buf, w.prot_off, w.prot_len, 3)
        finally:
            mp.mp_index_free(idx)
    finally:
        mp.mp_dp_destroy(ctx)
    wr = synth.regions_from_chains(w, chains, nch)
    pairs = [wr.pair(r) for r in range(wr.n_regions)]
    got = _refine_compare(mp, orc, pairs)
    assert len(pairs) > 10_000
    assert (got["n_anchors"] >= 2).mean() > 0.5
