"""Genome-scale workload: a synthetic genome with planted genes, a protein
set aligned against it, and a simple host-side k-mer seed + chain step that
turns the protein set into candidate (protein, genome interval, strand)
pairs for the spliced DP.

Shapes (the genome-scale configuration): a 500 Mb genome of i.i.d.
nucleotides at 40% GC carrying 20,000 planted genes generated like the
4,096-pair workload; 200,000 proteins with that workload's length
distribution, of which 10% are the planted genes' source proteins and the
rest, in equal parts, paralog variants of a source at 50-70% identity and
unrelated random proteins.

The seed + chain step is a candidate generator, not the paper's chaining:
it follows the shape of the paper's index (Methods, "Indexing the genome":
k-mers of translated open reading frames of at least 30 amino acids on both
strands, half of them kept by a hash bit, positions binned by 256 bp) with
7-mers over the 20-letter alphabet, looks up the protein's k-mers kept by
the same rule, and chains each protein's anchors on one strand in two
levels: anchors on one diagonal (genome position minus 3 nt per residue,
within two bins) form an exon cluster; consecutive clusters of at least two
anchors each are linked when the protein advances and the genome gap left
after the residues between them is under 200 kb (an intron).  The 3 chains
with the most anchors are kept.  A chain's region spans its anchors,
extended by the unaligned protein length (3 nt per residue) and 1 kb on
each side, clipped to the genome.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .gen import (_CODE_ACGT, AA20, Pair, _lognormal_int, plant_gene, random_protein, revcomp, _FREQ,
                  _AA20_BYTES)

K = 7                    # k-mer length (amino acids)
BIN = 256                # genome position bin (bp)
MIN_ORF = 30             # shortest indexed open reading frame (amino acids)
MAX_GAP = 200_000        # largest genome distance between chained anchors (bp)
FLANK = 1000             # region padding beyond the chain's extrapolated ends (bp)
TOP = 3                  # chains kept per protein
MAX_OCC = 64             # k-mers occurring more often in the index are skipped

_NT_LUT = np.full(256, 255, dtype=np.uint8)
for _k, _c in enumerate(b"ACGT"):
    _NT_LUT[_c] = _k
    _NT_LUT[_c | 0x20] = _k
# codon index (16 b1 + 4 b2 + b3, A C G T) -> amino-acid index in AA20 order, 20 = stop
_AA_OF_CODON = np.array([20 if a == "*" else AA20.index(a) for a in _CODE_ACGT], dtype=np.uint8)
_AA_LUT = np.full(256, 20, dtype=np.uint8)
for _k, _c in enumerate(AA20.encode()):
    _AA_LUT[_c] = _k
_COMP_LUT = np.arange(256, dtype=np.uint8)
for _a, _b in zip(b"ACGTacgt", b"TGCAtgca"):
    _COMP_LUT[_a] = _b
_GOLD = np.uint64(0x9E3779B97F4A7C15)


@dataclass
class GenomeWorkload:
    genome: np.ndarray          # uint8 ASCII, forward strand
    prot_buf: np.ndarray        # uint8 ASCII, proteins concatenated
    prot_off: np.ndarray        # int64 per protein
    prot_len: np.ndarray        # int64 per protein
    kind: np.ndarray            # 0 source of a planted gene, 1 paralog variant, 2 unrelated
    gene_of: np.ndarray         # planted gene a source or paralog descends from; -1 for unrelated
    gene_start: np.ndarray      # planted gene body on the forward strand: [start, end)
    gene_end: np.ndarray
    gene_strand: np.ndarray
    reg_prot: np.ndarray        # candidate regions: protein index,
    reg_start: np.ndarray       # forward-strand interval [start, end),
    reg_end: np.ndarray
    reg_strand: np.ndarray      # +1 / -1 (align to the reverse complement),
    reg_anchors: np.ndarray     # and the chain's anchor count

    @property
    def n_regions(self) -> int:
        return len(self.reg_prot)

    def cells(self) -> float:
        return float(np.sum(self.prot_len[self.reg_prot] * (self.reg_end - self.reg_start)))

    def protein(self, k: int) -> str:
        o = int(self.prot_off[k])
        return self.prot_buf[o:o + int(self.prot_len[k])].tobytes().decode()

    def pair(self, r: int) -> Pair:
        """Candidate region r as a Pair (copies the sequences)."""
        nt = self.genome[int(self.reg_start[r]):int(self.reg_end[r])].tobytes().decode()
        return Pair(self.protein(int(self.reg_prot[r])), nt, int(self.reg_strand[r]))

    def region_arrays(self, idx=None):
        """(prot_off, prot_len, nt_off, nt_len, strand) of the regions, for a
        zero-copy pair array over prot_buf and genome."""
        idx = np.arange(self.n_regions) if idx is None else np.asarray(idx)
        p = self.reg_prot[idx]
        return (self.prot_off[p], self.prot_len[p], self.reg_start[idx], self.reg_end[idx] - self.reg_start[idx],
                self.reg_strand[idx])


# ------------------------------------------------------------- generation
def _random_genome(rng, n: int, gc: float) -> np.ndarray:
    """i.i.d. bases at the given GC fraction (in steps of 1/1000)."""
    g = int(round(gc * 500))
    lut = np.frombuffer(b"A" * (500 - g) + b"C" * g + b"G" * g + b"T" * (500 - g), dtype=np.uint8)
    out = np.empty(n, dtype=np.uint8)
    step = 1 << 26
    for s in range(0, n, step):
        e = min(n, s + step)
        out[s:e] = lut[rng.integers(0, 1000, size=e - s, dtype=np.int16)]
    return out


def _paralog(rng, src: np.ndarray, identity: float) -> np.ndarray:
    """Replace each residue (ASCII) with probability 1 - identity by a
    different residue drawn from the background frequencies."""
    out = _AA_LUT[src]
    hit = np.nonzero(rng.random(len(src)) >= identity)[0]
    if len(hit):
        new = rng.choice(20, size=len(hit), p=_FREQ).astype(np.uint8)
        same = new == out[hit]
        new[same] = (new[same] + 1 + rng.integers(0, 19, size=int(same.sum()))) % 20
        out[hit] = new
    return _AA20_BYTES[out]


def make_workload(seed: int = 5, genome_len: int = 500_000_000, n_genes: int = 20_000,
                  n_proteins: int = 200_000, gc: float = 0.4, host_seeding: bool = True) -> GenomeWorkload:
    """The genome, planted genes and proteins; with host_seeding the
    candidate regions of the host stand-in below, otherwise none (to be set
    from the library's seeding and chaining with regions_from_chains)."""
    rng = np.random.default_rng(seed)
    genome = _random_genome(rng, genome_len, gc)
    # ---- planted genes, one per slot of the genome
    slot = genome_len // n_genes
    sources, gs, ge, gstr = [], [], [], []
    for g in range(n_genes):
        plen = int(_lognormal_int(rng, 350, 0.75, 50, 2000))
        plen = min(plen, max(10, (slot - 2200) // 3))
        k = min(int(rng.poisson(3)), 8)
        lens = _lognormal_int(rng, 800, 1.0, 60, 20000, size=k).tolist() if k else []
        while lens and 3 * plen + 8 + sum(lens) > slot - 2200:
            lens.pop(int(np.argmax(lens)))
        prot = random_protein(rng, plen)
        body, _ = plant_gene(rng, prot, float(rng.uniform(0.10, 0.40)), int(rng.integers(0, 4)), lens, 0, 0)
        strand = 1 if rng.random() < 0.5 else -1
        if strand < 0:
            body = revcomp(body)
        start = g * slot + int(rng.integers(1000, max(1001, slot - len(body) - 1000)))
        genome[start:start + len(body)] = np.frombuffer(body.encode(), dtype=np.uint8)
        sources.append(np.frombuffer(prot.encode(), dtype=np.uint8))
        gs.append(start)
        ge.append(start + len(body))
        gstr.append(strand)
    # ---- proteins: sources, paralogs, unrelated, in a shuffled order
    n_src = min(n_genes, n_proteins // 10)
    n_par = (n_proteins - n_src) // 2
    n_unr = n_proteins - n_src - n_par
    prots, kind, gene_of = [], [], []
    for g in range(n_src):
        prots.append(sources[g]); kind.append(0); gene_of.append(g)
    for _ in range(n_par):
        g = int(rng.integers(0, n_genes))
        prots.append(_paralog(rng, sources[g], float(rng.uniform(0.5, 0.7)))); kind.append(1); gene_of.append(g)
    for _ in range(n_unr):
        plen = int(_lognormal_int(rng, 350, 0.75, 50, 2000))
        prots.append(_AA20_BYTES[rng.choice(20, size=plen, p=_FREQ)]); kind.append(2); gene_of.append(-1)
    perm = rng.permutation(len(prots))
    prots = [prots[k] for k in perm]
    kind = np.asarray(kind, np.int8)[perm]
    gene_of = np.asarray(gene_of, np.int64)[perm]
    prot_len = np.array([len(p) for p in prots], dtype=np.int64)
    prot_off = np.concatenate([[0], np.cumsum(prot_len)[:-1]]).astype(np.int64)
    prot_buf = np.concatenate(prots) if prots else np.zeros(0, np.uint8)
    if host_seeding:
        reg = seed_and_chain(genome, prot_buf, prot_off, prot_len)
    else:
        reg = (np.zeros(0, np.int64), np.zeros(0, np.int64), np.zeros(0, np.int64), np.zeros(0, np.int8),
               np.zeros(0, np.int64))
    return GenomeWorkload(genome, prot_buf, prot_off, prot_len, kind, gene_of, np.asarray(gs, np.int64),
                          np.asarray(ge, np.int64), np.asarray(gstr, np.int8), *reg)


# ------------------------------------------------------------- seed + chain
def _kmer_codes(aa: np.ndarray):
    """Base-20 codes of the K-mers starting at each position of an amino-acid
    code array (20 = stop), and whether the K-mer is stop-free."""
    n = len(aa) - K + 1
    if n <= 0:
        return np.zeros(0, np.int64), np.zeros(0, bool)
    code = np.zeros(n, dtype=np.int64)
    for t in range(K):
        code = code * 20 + np.minimum(aa[t:t + n], 19)
    stops = np.concatenate([[0], np.cumsum(aa == 20, dtype=np.int64)])
    return code, (stops[K:K + n] - stops[:n]) == 0


def _kept(code: np.ndarray) -> np.ndarray:
    """The sampling rule shared by genome and protein k-mers: bit 40 of a
    multiplicative hash is 0 (half of the k-mers)."""
    return ((code.astype(np.uint64) * _GOLD) >> np.uint64(40)) & np.uint64(1) == 0


_BIN_BITS = 22           # bins of a strand (< 2^22 for genomes up to ~1 Gb) below the k-mer code


def _index_frame(b: np.ndarray, f: int) -> np.ndarray:
    """Kept k-mers of reading frame f of one strand (base codes b), sorted:
    code << _BIN_BITS | bin of the k-mer's first base in this strand's
    coordinates."""
    n = (len(b) - f) // 3
    if n < K:
        return np.zeros(0, np.int64)
    cod = 16 * b[f:f + 3 * n:3].astype(np.int16) + 4 * b[f + 1:f + 3 * n:3] + b[f + 2:f + 3 * n:3]
    aa = _AA_OF_CODON[cod]
    del cod
    code, ok = _kmer_codes(aa)
    # open reading frames of at least MIN_ORF amino acids
    run = np.cumsum(aa == 20, dtype=np.int32)
    runlen = np.bincount(run[aa != 20], minlength=int(run[-1]) + 1)
    ok &= runlen[run[:len(code)]] >= MIN_ORF
    del run, runlen, aa
    ok &= _kept(code)
    pos = np.nonzero(ok)[0]
    key = (code[pos] << _BIN_BITS) | ((f + 3 * pos) // BIN)
    key.sort()
    return key


def seed_and_chain(genome: np.ndarray, prot_buf: np.ndarray, prot_off: np.ndarray, prot_len: np.ndarray,
                   threads: int = 3):
    from concurrent.futures import ThreadPoolExecutor

    G = len(genome)
    if (G // BIN) >= (1 << _BIN_BITS):
        raise ValueError("genome too long for the bin field")
    b = _NT_LUT[genome]
    if (b == 255).any():
        raise ValueError("genome holds letters other than ACGT")
    rb = (3 - b)[::-1]
    jobs = [(b, f) for f in range(3)] + [(rb, f) for f in range(3)]
    with ThreadPoolExecutor(max_workers=threads) as ex:        # numpy releases the GIL on large arrays
        index = list(ex.map(lambda j: _index_frame(*j), jobs))
    del b, rb
    # protein k-mers (a stop code between proteins keeps k-mers inside one protein)
    n_p = len(prot_len)
    sep = np.full(len(prot_buf) + n_p, 20, dtype=np.uint8)
    at = prot_off + np.arange(n_p)
    idx = np.repeat(at - prot_off, prot_len) + np.arange(len(prot_buf))
    sep[idx] = _AA_LUT[prot_buf]
    qcode, ok = _kmer_codes(sep)
    ok &= _kept(qcode)
    qpos = np.nonzero(ok)[0]
    qprot = np.searchsorted(at, qpos, side="right") - 1
    qy = qpos - at[qprot]
    qcode = qcode[qpos]
    # look the protein k-mers up in each frame's index; k-mers occurring more
    # than MAX_OCC times over the whole index are skipped
    qlo, qhi = qcode << _BIN_BITS, (qcode + 1) << _BIN_BITS
    with ThreadPoolExecutor(max_workers=threads) as ex:
        ranges = list(ex.map(lambda ix: (np.searchsorted(ix, qlo), np.searchsorted(ix, qhi)), index))
    total = sum(hi - lo for lo, hi in ranges)
    skip = total > MAX_OCC
    a_prot, a_y, a_str, a_bin = [], [], [], []
    for j, (ix, (lo, hi)) in enumerate(zip(index, ranges)):
        cnt = np.where(skip, 0, hi - lo)
        tot = int(cnt.sum())
        q = np.repeat(np.arange(len(qcode)), cnt)
        first = np.repeat(np.cumsum(cnt) - cnt, cnt)
        a_bin.append(ix[lo[q] + (np.arange(tot) - first)] & ((1 << _BIN_BITS) - 1))
        a_prot.append(qprot[q])
        a_y.append(qy[q])
        a_str.append(np.full(tot, 1 if j >= 3 else 0, dtype=np.int64))
    del index
    a_prot, a_y, a_str, a_bin = (np.concatenate(v) for v in (a_prot, a_y, a_str, a_bin))
    tot = len(a_prot)
    # exon clusters: anchors of one protein and strand on one diagonal
    # (genome position minus 3 nt per residue, within two bins)
    diag = a_bin * BIN - 3 * a_y
    srt = np.lexsort((a_y, diag, a_str, a_prot))
    a_prot, a_str, a_bin, a_y, diag = a_prot[srt], a_str[srt], a_bin[srt], a_y[srt], diag[srt]
    new = np.ones(tot, dtype=bool)
    if tot > 1:
        new[1:] = (a_prot[1:] != a_prot[:-1]) | (a_str[1:] != a_str[:-1]) | (np.diff(diag) > 2 * BIN)
    head = np.nonzero(new)[0]
    k_n = np.diff(np.append(head, tot))
    k_prot, k_str = a_prot[head], a_str[head]
    k_bin0 = np.minimum.reduceat(a_bin, head) if tot else np.zeros(0, np.int64)
    k_bin1 = np.maximum.reduceat(a_bin, head) if tot else np.zeros(0, np.int64)
    k_y0 = np.minimum.reduceat(a_y, head) if tot else np.zeros(0, np.int64)
    k_y1 = np.maximum.reduceat(a_y, head) if tot else np.zeros(0, np.int64)
    # chains: clusters of >= 2 anchors, consecutive in genome order, with the
    # protein advancing and an intron-sized gap (< MAX_GAP) between them
    o = np.lexsort((k_bin0, k_str, k_prot))
    k_n, k_prot, k_str, k_bin0, k_bin1, k_y0, k_y1 = (v[o] for v in (k_n, k_prot, k_str, k_bin0, k_bin1, k_y0, k_y1))
    nk = len(k_n)
    link = np.zeros(nk, dtype=bool)
    if nk > 1:
        gap = (k_bin0[1:] - k_bin1[:-1]) * BIN - 3 * (k_y0[1:] - k_y1[:-1])
        link[1:] = ((k_prot[1:] == k_prot[:-1]) & (k_str[1:] == k_str[:-1]) & (k_n[1:] >= 2) & (k_n[:-1] >= 2) &
                    (k_y0[1:] > k_y1[:-1] - 2) & (gap > -2 * BIN) & (gap < MAX_GAP))
    chead = np.nonzero(~link)[0]
    n_ch = len(chead)
    c_n = np.add.reduceat(k_n, chead) if nk else np.zeros(0, np.int64)
    c_prot, c_str = k_prot[chead], k_str[chead]
    c_bin0 = np.minimum.reduceat(k_bin0, chead) if nk else np.zeros(0, np.int64)
    c_bin1 = np.maximum.reduceat(k_bin1, chead) if nk else np.zeros(0, np.int64)
    c_y0 = np.minimum.reduceat(k_y0, chead) if nk else np.zeros(0, np.int64)
    c_y1 = np.maximum.reduceat(k_y1, chead) if nk else np.zeros(0, np.int64)
    # the TOP chains of each protein by anchor count (earlier chains first on ties)
    pick = np.lexsort((np.arange(n_ch), -c_n, c_prot))
    rank = np.arange(n_ch) - np.searchsorted(c_prot[pick], c_prot[pick], side="left")
    pick = pick[rank < TOP]
    pick = pick[np.argsort(c_prot[pick], kind="stable")]
    m = prot_len[c_prot[pick]]
    s = c_bin0[pick] * BIN - 3 * c_y0[pick] - FLANK
    e = (c_bin1[pick] + 1) * BIN + 3 * (m - c_y1[pick]) + FLANK
    s = np.clip(s, 0, G)
    e = np.clip(e, 0, G)
    rev = c_str[pick] == 1
    fs = np.where(rev, G - e, s)
    fe = np.where(rev, G - s, e)
    keep = fe > fs
    return (c_prot[pick][keep].astype(np.int64), fs[keep].astype(np.int64), fe[keep].astype(np.int64),
            np.where(rev, -1, 1)[keep].astype(np.int8), c_n[pick][keep].astype(np.int64))


def config5(seed: int = 5, scale: float = 1.0, host_seeding: bool = True) -> GenomeWorkload:
    """The genome-scale workload; scale < 1 shrinks the genome, the gene
    count and the protein count together (tests)."""
    return make_workload(seed, genome_len=int(500_000_000 * scale), n_genes=max(1, int(20_000 * scale)),
                         n_proteins=max(10, int(200_000 * scale)), host_seeding=host_seeding)


def regions_from_chains(w: GenomeWorkload, chains, n_chains) -> GenomeWorkload:
    """Candidate regions from chains (the library's seeding and chaining:
    per protein up to `top` chains of (strand, n_anchors, score, x_first,
    x_last, y_first, y_last), x in 256-bp bins on the chain's strand, y
    residues): each chain's span extended by 3 nt per residue the chain
    leaves unaligned on either side and FLANK bp, clipped to the genome,
    on the forward strand's coordinates (strand -1 for the reverse
    complement).  Returns the workload with these regions."""
    G = len(w.genome)
    n_p, top = chains.shape
    k = np.arange(top)[None, :] < np.asarray(n_chains)[:, None]
    prot = np.broadcast_to(np.arange(n_p)[:, None], (n_p, top))[k].astype(np.int64)
    c = chains[k]
    m = w.prot_len[prot]
    s = c["x_first"] * BIN - 3 * c["y_first"] - FLANK
    e = (c["x_last"] + 1) * BIN + 3 * (m - c["y_last"]) + FLANK
    s, e = np.clip(s, 0, G), np.clip(e, 0, G)
    rev = c["strand"] == 1
    fs, fe = np.where(rev, G - e, s), np.where(rev, G - s, e)
    keep = fe > fs
    w.reg_prot, w.reg_start, w.reg_end = prot[keep], fs[keep].astype(np.int64), fe[keep].astype(np.int64)
    w.reg_strand = np.where(rev, -1, 1)[keep].astype(np.int8)
    w.reg_anchors = c["n_anchors"][keep].astype(np.int64)
    return w
