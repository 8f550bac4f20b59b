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
