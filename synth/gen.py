"""Seeded generators for the benchmark and test workloads.

Each generator plants a protein's coding sequence, with substitutions,
frameshift indels and GT...AG introns, into random flanking sequence, the
way the paper's evaluation aligns proteomes of related species to a genome
(Results, "Evaluation datasets"; Table 1).  The real proteomes and genomes
are not available here; these shapes stand in for them.

Workloads (sizes as named by the benchmark configurations):
  config1  one pair: 120 aa; CDS 360 nt; 15% substitutions; one 1-nt
           insertion; introns of 150 and 400 nt; 100 nt flanks (1,111 nt).
  config2  4,096 pairs: protein log-normal (median 350, sigma 0.75,
           50..2,000 aa); Poisson(3) introns capped at 8, log-normal lengths
           (median 800, sigma 1.0, 60..20,000 nt); 10-40% substitutions;
           0-3 frameshift indels; 1 kb flanks at 40% GC; half reverse strand.
  config3  20,000 pairs: protein log-uniform 20..5,000 aa; introns as
           config2 with a 2% tail of 20-100 kb introns; region <= 200 kb;
           5% decoys (unrelated 40% GC region, score only).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

AA20 = "ARNDCQEGHILKMFPSTWYV"
# Background amino-acid frequencies (Robinson & Robinson 1991), AA20 order.
_FREQ = np.array([0.07805, 0.05129, 0.04487, 0.05364, 0.01925, 0.04264, 0.06295, 0.07377,
                  0.02199, 0.05142, 0.09019, 0.05744, 0.02243, 0.03856, 0.05203, 0.07120,
                  0.05841, 0.01330, 0.03216, 0.06441])
_FREQ = _FREQ / _FREQ.sum()

# Standard genetic code, codons enumerated with bases in A, C, G, T order.
_CODE_ACGT = "KNKNTTTTRSRSIIMIQHQHPPPPRRRRLLLLEDEDAAAAGGGGVVVV*Y*YSSSS*CWCLFLF"
_BASES = "ACGT"
_CODONS = [a + b + c for a in _BASES for b in _BASES for c in _BASES]
_SYN = {aa: [c for c, x in zip(_CODONS, _CODE_ACGT) if x == aa] for aa in AA20}

_COMP = str.maketrans("ACGTacgt", "TGCAtgca")


def revcomp(s: str) -> str:
    return s.translate(_COMP)[::-1]


@dataclass
class Pair:
    prot: str
    nt: str                 # as handed to the aligner (forward strand of the input)
    strand: int = 1         # +1, or -1: the gene lies on the reverse complement of nt
    score_only: bool = False
    truth: dict = field(default_factory=dict)
    profile: object = None  # optional position-specific costs of a profile query: (|P| + 1) x 23 ints

    @property
    def cells(self) -> int:
        return len(self.prot) * len(self.nt)


def pairs_cells(pairs) -> int:
    return int(sum(len(p.prot) * len(p.nt) for p in pairs))


_AA20_BYTES = np.frombuffer(AA20.encode(), dtype=np.uint8)
_BASE_BYTES = np.frombuffer(b"ACGT", dtype=np.uint8)


def random_protein(rng: np.random.Generator, n: int) -> str:
    idx = rng.choice(20, size=n, p=_FREQ)
    return _AA20_BYTES[idx].tobytes().decode()


def random_dna(rng: np.random.Generator, n: int, gc: float = 0.5) -> str:
    if n <= 0:
        return ""
    p = np.array([(1 - gc) / 2, gc / 2, gc / 2, (1 - gc) / 2])
    idx = rng.choice(4, size=n, p=p)
    return _BASE_BYTES[idx].tobytes().decode()


def reverse_translate(rng: np.random.Generator, prot: str) -> str:
    """Uniformly random synonymous codon per residue (no stop codons)."""
    u = rng.random(len(prot))
    return "".join(_SYN[a][int(x * len(_SYN[a]))] for a, x in zip(prot, u))


def _substitute(rng, cds: list, prot: str, rate: float) -> int:
    """Replace round(rate*len) codons by a codon of a different amino acid."""
    n = len(prot)
    k = int(round(rate * n))
    if k == 0:
        return 0
    pos = rng.choice(n, size=k, replace=False)
    for p in pos:
        old = prot[p]
        choices = [a for a in AA20 if a != old]
        new = choices[int(rng.integers(len(choices)))]
        syn = _SYN[new]
        cds[p] = syn[int(rng.integers(len(syn)))]
    return k


def _intron(rng, length: int, gc: float | None = None) -> str:
    body = random_dna(rng, length - 4, 0.5 if gc is None else gc)
    return "GT" + body + "AG"


def plant_gene(rng, prot: str, subst_rate: float, n_fs: int, intron_lens, flank5: int, flank3: int,
               flank_gc: float = 0.5, fs_insert_only: bool = False, fs_len=None):
    """Build a genomic region carrying a mutated, frameshifted, spliced copy
    of `prot`'s coding sequence.  Returns (region, truth)."""
    rt = reverse_translate(rng, prot)
    codons = [rt[k:k + 3] for k in range(0, len(rt), 3)]
    n_sub = _substitute(rng, codons, prot, subst_rate)
    cds = list("".join(codons))
    fs = []
    for _ in range(n_fs):
        if len(cds) < 4:
            break
        L = int(fs_len) if fs_len is not None else int(rng.integers(1, 3))
        pos = int(rng.integers(1, len(cds)))
        if fs_insert_only or rng.random() < 0.5:
            ins = random_dna(rng, L)
            cds[pos:pos] = list(ins)
            fs.append(("ins", pos, L))
        else:
            del cds[pos:pos + L]
            fs.append(("del", pos, L))
    cds = "".join(cds)
    # intron positions uniform over the CDS (so phases 0, 1 and 2 all occur)
    k = min(len(intron_lens), max(0, len(cds) - 1))
    intron_lens = list(intron_lens)[:k]
    cuts = sorted(rng.choice(np.arange(1, len(cds)), size=k, replace=False).tolist()) if k else []
    pieces, prev = [], 0
    for c, L in zip(cuts, intron_lens):
        pieces.append(cds[prev:c])
        pieces.append(_intron(rng, int(L)))
        prev = c
    pieces.append(cds[prev:])
    gene = "".join(pieces)
    region = random_dna(rng, flank5, flank_gc) + gene + random_dna(rng, flank3, flank_gc)
    truth = dict(n_sub=n_sub, frameshifts=fs, intron_cuts=cuts, intron_lens=list(map(int, intron_lens)),
                 gene_start=flank5, gene_end=flank5 + len(gene))
    return region, truth


def config1(seed: int = 0) -> Pair:
    """One pair: 120 aa, 15% substitutions, one 1-nt insertion, introns of
    150 and 400 nt, 100 nt flanks: 1,111 nt in total, forward strand."""
    rng = np.random.default_rng(seed)
    prot = random_protein(rng, 120)
    region, truth = plant_gene(rng, prot, 0.15, 1, [150, 400], 100, 100, fs_insert_only=True, fs_len=1)
    return Pair(prot, region, 1, False, truth)


def _lognormal_int(rng, median, sigma, lo, hi, size=None):
    x = np.exp(np.log(median) + sigma * rng.standard_normal(size))
    return np.clip(np.round(x), lo, hi).astype(np.int64)


def _gene_pair(rng, plen: int, intron_lens, flank: int = 1000, flank_gc: float = 0.4) -> Pair:
    prot = random_protein(rng, int(plen))
    rate = float(rng.uniform(0.10, 0.40))
    n_fs = int(rng.integers(0, 4))
    region, truth = plant_gene(rng, prot, rate, n_fs, intron_lens, flank, flank, flank_gc)
    strand = 1
    if rng.random() < 0.5:
        region = revcomp(region)
        strand = -1
    truth["subst_rate"] = rate
    return Pair(prot, region, strand, False, truth)


def config2(seed: int = 2, n: int = 4096) -> list:
    """Batched workload: `n` pairs (4,096 by default)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        plen = int(_lognormal_int(rng, 350, 0.75, 50, 2000))
        k = min(int(rng.poisson(3)), 8)
        lens = _lognormal_int(rng, 800, 1.0, 60, 20000, size=k).tolist() if k else []
        out.append(_gene_pair(rng, plen, lens))
    return out


def config3(seed: int = 3, n: int = 20000, max_region: int = 200_000) -> list:
    """Uneven-size stress workload: `n` pairs (20,000 by default)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        plen = int(np.round(np.exp(rng.uniform(np.log(20), np.log(5000)))))
        if rng.random() < 0.05:
            prot = random_protein(rng, plen)
            nt = random_dna(rng, int(np.clip(3 * plen + 2000 + rng.integers(0, 8000), 100, max_region)), 0.4)
            out.append(Pair(prot, nt, 1, True, dict(decoy=True)))
            continue
        k = min(int(rng.poisson(3)), 8)
        lens = []
        for _ in range(k):
            if rng.random() < 0.02:
                lens.append(int(np.round(np.exp(rng.uniform(np.log(20_000), np.log(100_000))))))
            else:
                lens.append(int(_lognormal_int(rng, 800, 1.0, 60, 20000)))
        budget = max_region - 2000 - 3 * plen - 8
        while lens and sum(lens) > budget:
            lens.pop(int(np.argmax(lens)))
        out.append(_gene_pair(rng, plen, lens))
    return out


def serving_pairs(seed: int = 4, n: int = 4096) -> list:
    """Requests for the serving loop, drawn from config2's distribution."""
    return config2(seed=seed, n=n)
