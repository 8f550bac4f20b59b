/*
 * chain.c -- plain CPU oracle of the seeding and chaining stage (Li 2022,
 * Methods: "Reduced alphabet", "Indexing the genome", "Chaining").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * benchmark's CPU legs may load it.  It shares no code, table or constant
 * with the CUDA library: the reduced alphabet, the genetic code and the hash
 * are written out here on their own.
 *
 * What it computes:
 *   - phi: the reduced 16-letter amino-acid alphabet ("Reduced alphabet").
 *   - psi: an invertible integer hash of a k-mer's 4k-bit code ("Indexing the
 *     genome" cites Li 2016 for it); here Thomas Wang's 64-bit integer mix
 *     with every step taken modulo 2^(4k), the form minimap (Li 2016) uses.
 *   - The index: both strands as independent sequences, all three frames of
 *     each, every open reading frame (a maximal run of codons without a stop
 *     codon) of at least 30 amino acids; every k-mer inside one, whose hash
 *     has lowest bit 0, is stored as (hash, floor(x / 256)) with x the
 *     position of its first base on its strand.  The table is a CSR array
 *     over all 2^(4k) hash values, each value's positions in ascending order
 *     of (strand << 31 | bin).
 *   - Anchors of a protein: each of its k-mers looked up in the table, as
 *     (strand, x = bin, y = residue position of the k-mer's first residue).
 *   - Chaining, Eq. 1-3 of "Chaining": per strand, anchors sorted by (x, y);
 *     f(j) = max(k, max_{i<j, x_i <= x_j, y_i < y_j} f(i) + alpha(i,j) -
 *     gamma(g(i,j))) with g of Eq. 1 (bins of 256 bp), gamma of Eq. 3
 *     (G = 200,000, beta = 0.75) and alpha = min(y_j - y_i, k).
 *
 * Readings (the paper leaves them open):
 *   - Scores are fixed point with 16 fractional bits: each gamma term is
 *     floored to a multiple of 2^-16 (g/3 and beta log2(|g|+1) separately,
 *     the smaller of the two for g < 0), so the sums are exact integers and
 *     ties are exact.
 *   - f(j) keeps the first predecessor (in the sorted order) that reaches
 *     the maximum, and starts a new chain (f = k) unless a predecessor is
 *     strictly better.
 *   - Chains are taken in order of decreasing f of their last anchor (ties:
 *     the earlier anchor), each by following predecessors until an anchor
 *     already used or the start; the chain's score is f of its last anchor
 *     less f of the used anchor it stopped at (if any).  Chains of one
 *     anchor are dropped; the first `top` chains are reported.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define CH_BIN 256
#define CH_G 200000
#define CH_MIN_ORF 30
#define CH_SCALE 65536

/* ---------------------------------------------------------------- phi */

/* Reduced alphabet: A 0, ST 1, RK 2, H 3, ND 4, EQ 5, C 6, P 7, G 8,
 * IV 10, LM 11, FY 12, W 13, stop 14, anything else (X) 15. */
int orc_phi(int ch)
{
    switch (ch >= 'a' && ch <= 'z' ? ch - 32 : ch) {
    case 'A': return 0;
    case 'S': case 'T': return 1;
    case 'R': case 'K': return 2;
    case 'H': return 3;
    case 'N': case 'D': return 4;
    case 'E': case 'Q': return 5;
    case 'C': return 6;
    case 'P': return 7;
    case 'G': return 8;
    case 'I': case 'V': return 10;
    case 'L': case 'M': return 11;
    case 'F': case 'Y': return 12;
    case 'W': return 13;
    case '*': return 14;
    default: return 15;
    }
}

/* ---------------------------------------------------------------- psi */

/* Thomas Wang's integer mix, every step modulo 2^bits (each step is a
 * bijection of [0, 2^bits), so psi is invertible there). */
uint64_t orc_psi(uint64_t key, int bits)
{
    const uint64_t mask = bits >= 64 ? ~0ull : ((1ull << bits) - 1);
    key &= mask;
    key = (~key + (key << 21)) & mask;
    key = key ^ key >> 24;
    key = (key + (key << 3) + (key << 8)) & mask;
    key = key ^ key >> 14;
    key = (key + (key << 2) + (key << 4)) & mask;
    key = key ^ key >> 28;
    key = (key + (key << 31)) & mask;
    return key;
}

/* ---------------------------------------------------------- translation */

/* Standard genetic code (NCBI table 1), codons in T, C, A, G order. */
static const char CH_CODE_TCAG[] = "FFLLSSSSYY**CC*WLLLLPPPPHHQQRRRRIIIMTTTTNNKKSSRRVVVVAAAADDEEGGGG";

static int ch_tcag(int ch)
{
    switch (ch) {
    case 'T': case 't': return 0;
    case 'C': case 'c': return 1;
    case 'A': case 'a': return 2;
    case 'G': case 'g': return 3;
    default: return -1;
    }
}

static char ch_complement(char c)
{
    switch (c) {
    case 'A': case 'a': return 'T';
    case 'C': case 'c': return 'G';
    case 'G': case 'g': return 'C';
    case 'T': case 't': return 'A';
    default: return 'N';
    }
}

/* amino acid letter of the codon at s[0..2]; 'X' if a base is not ACGT */
static char ch_translate(const char *s)
{
    int a = ch_tcag(s[0]), b = ch_tcag(s[1]), c = ch_tcag(s[2]);
    if (a < 0 || b < 0 || c < 0) return 'X';
    return CH_CODE_TCAG[16 * a + 4 * b + c];
}

/* ---------------------------------------------------------------- index */

typedef struct {
    uint64_t hash;
    uint32_t pos;
} ch_entry;

static int ch_cmp_entry(const void *a, const void *b)
{
    const ch_entry *x = (const ch_entry *)a, *y = (const ch_entry *)b;
    if (x->hash != y->hash) return x->hash < y->hash ? -1 : 1;
    return x->pos < y->pos ? -1 : x->pos > y->pos;
}

/* Count (offsets == NULL) or build the index of genome[0..n).  offsets has
 * 2^(4k) + 1 entries, positions offsets[2^(4k)] entries.  Returns the
 * number of entries, or -1 on failure. */
int64_t orc_index(const char *genome, int64_t n, int k, uint64_t *offsets, uint32_t *positions)
{
    char *seq = (char *)malloc((size_t)n + 1);
    char *aa = (char *)malloc((size_t)n / 3 + 2);
    size_t cap = 1024, cnt = 0;
    ch_entry *e = (ch_entry *)malloc(cap * sizeof(ch_entry));
    if (!seq || !aa || !e) { free(seq); free(aa); free(e); return -1; }
    for (int strand = 0; strand < 2; ++strand) {
        for (int64_t t = 0; t < n; ++t) seq[t] = strand == 0 ? genome[t] : ch_complement(genome[n - 1 - t]);
        for (int frame = 0; frame < 3; ++frame) {
            int64_t L = (n - frame) / 3;
            if (L < 0) L = 0;
            for (int64_t t = 0; t < L; ++t) aa[t] = ch_translate(seq + frame + 3 * t);
            /* each maximal run of non-stop codons [a, b) */
            int64_t a = 0;
            while (a < L) {
                while (a < L && aa[a] == '*') ++a;
                int64_t b = a;
                while (b < L && aa[b] != '*') ++b;
                if (b - a >= CH_MIN_ORF) {
                    for (int64_t t = a; t + k <= b; ++t) {
                        uint64_t key = 0;
                        for (int u = 0; u < k; ++u) key = key * 16 + (uint64_t)orc_phi(aa[t + u]);
                        const uint64_t h = orc_psi(key, 4 * k);
                        if (h & 1) continue;
                        if (cnt == cap) {
                            cap *= 2;
                            ch_entry *ne = (ch_entry *)realloc(e, cap * sizeof(ch_entry));
                            if (!ne) { free(seq); free(aa); free(e); return -1; }
                            e = ne;
                        }
                        const int64_t x = frame + 3 * t;
                        e[cnt].hash = h;
                        e[cnt].pos = ((uint32_t)strand << 31) | (uint32_t)(x / CH_BIN);
                        ++cnt;
                    }
                }
                a = b;
            }
        }
    }
    if (offsets) {
        qsort(e, cnt, sizeof(ch_entry), ch_cmp_entry);
        const uint64_t nkeys = 1ull << (4 * k);
        memset(offsets, 0, (nkeys + 1) * sizeof(uint64_t));
        for (size_t t = 0; t < cnt; ++t) offsets[e[t].hash + 1]++;
        for (uint64_t h = 0; h < nkeys; ++h) offsets[h + 1] += offsets[h];
        for (size_t t = 0; t < cnt; ++t) positions[t] = e[t].pos;
    }
    free(seq);
    free(aa);
    free(e);
    return (int64_t)cnt;
}

/* ------------------------------------------------------------- chaining */

/* Eq. 1: the least gap size in bp between anchors i and j (x in bins). */
int64_t orc_gap(int64_t dx, int64_t dy)
{
    const int64_t py = 3 * dy;
    if (py < CH_BIN * (dx - 1)) return py - CH_BIN * (dx - 1);
    if (py > CH_BIN * (dx + 1)) return py - CH_BIN * (dx + 1);
    return 0;
}

/* Eq. 3 in units of 2^-16; -1 for an infinite penalty (|g| >= G). */
int64_t orc_gap_penalty(int64_t g)
{
    if (g == 0) return 0;
    const int64_t a = g < 0 ? -g : g;
    if (a >= CH_G) return -1;
    const int64_t lin = (a * CH_SCALE) / 3;                                   /* floor(S |g| / 3) */
    /* floor(S beta log2(|g|+1)): exact for a power of two (an integer
     * log2), from the double log2 otherwise (every such value lies at least
     * 6.8e-6 from an integer for |g| < G, far beyond the double's error) */
    const int64_t v = a + 1;
    int64_t lg;
    if ((v & (v - 1)) == 0) {
        int e = 0;
        while ((1ll << e) < v) ++e;
        lg = (int64_t)e * (3 * CH_SCALE / 4);
    } else {
        lg = (int64_t)floor(0.75 * CH_SCALE * log2((double)v));
    }
    if (g > 0) return lin + lg;
    return lin < lg ? lin : lg;
}

typedef struct {
    int32_t strand;
    int64_t x, y;
    int64_t f;
    int64_t pred;
    int used;
} ch_anchor;

static int ch_cmp_anchor(const void *a, const void *b)
{
    const ch_anchor *p = (const ch_anchor *)a, *q = (const ch_anchor *)b;
    if (p->strand != q->strand) return p->strand < q->strand ? -1 : 1;
    if (p->x != q->x) return p->x < q->x ? -1 : 1;
    return p->y < q->y ? -1 : p->y > q->y;
}

/* One chain of a protein. */
typedef struct {
    int32_t strand, n_anchors;
    int64_t score;              /* in units of 2^-16 */
    int64_t x_first, x_last;    /* bins on the chain's strand */
    int64_t y_first, y_last;    /* residue positions of the first and last anchor's k-mer */
} orc_chain_t;

/* The anchors of protein prot[0..m) against an index (CSR of orc_index):
 * writes up to cap (strand, x, y) triples, sorted; returns their count
 * (which may exceed cap), or -1. */
int64_t orc_anchors(const uint64_t *offsets, const uint32_t *positions, int k, const char *prot, int64_t m,
                    int64_t *out, int64_t cap)
{
    int64_t cnt = 0;
    for (int64_t t = 0; t + k <= m; ++t) {
        uint64_t key = 0;
        for (int u = 0; u < k; ++u) key = key * 16 + (uint64_t)orc_phi((unsigned char)prot[t + u]);
        const uint64_t h = orc_psi(key, 4 * k);
        for (uint64_t e = offsets[h]; e < offsets[h + 1]; ++e) {
            if (cnt < cap) {
                out[3 * cnt] = positions[e] >> 31;
                out[3 * cnt + 1] = positions[e] & 0x7fffffffu;
                out[3 * cnt + 2] = t;
            }
            ++cnt;
        }
    }
    return cnt;
}

/* Chain anchors (n triples (strand, x, y), any order): the chaining score
 * of every anchor after sorting (f_out[n], may be NULL) and the first `top`
 * chains of at least two anchors.  Returns the number of chains written. */
int orc_chain_anchors(const int64_t *anc, int64_t n, int k, int top, orc_chain_t *chains, int64_t *f_out)
{
    ch_anchor *a = (ch_anchor *)malloc(sizeof(ch_anchor) * (size_t)(n > 0 ? n : 1));
    if (!a) return -1;
    for (int64_t t = 0; t < n; ++t) {
        a[t].strand = (int32_t)anc[3 * t];
        a[t].x = anc[3 * t + 1];
        a[t].y = anc[3 * t + 2];
        a[t].used = 0;
    }
    qsort(a, (size_t)n, sizeof(ch_anchor), ch_cmp_anchor);
    const int64_t S = CH_SCALE;
    for (int64_t j = 0; j < n; ++j) {
        a[j].f = (int64_t)k * S;
        a[j].pred = -1;
        for (int64_t i = 0; i < j; ++i) {
            if (a[i].strand != a[j].strand || a[i].x > a[j].x || a[i].y >= a[j].y) continue;
            const int64_t dy = a[j].y - a[i].y;
            const int64_t pen = orc_gap_penalty(orc_gap(a[j].x - a[i].x, dy));
            if (pen < 0) continue;
            const int64_t cand = a[i].f + (dy < k ? dy : k) * S - pen;
            if (cand > a[j].f) { a[j].f = cand; a[j].pred = i; }
        }
        if (f_out) f_out[j] = a[j].f;
    }
    int nc = 0;
    for (;;) {
        if (nc >= top) break;
        int64_t best = -1;
        for (int64_t j = 0; j < n; ++j)
            if (!a[j].used && (best < 0 || a[j].f > a[best].f)) best = j;
        if (best < 0) break;
        int64_t cnt = 0, cur = best, first = best, stop = -1;
        while (cur >= 0 && !a[cur].used) {
            a[cur].used = 1;
            first = cur;
            ++cnt;
            cur = a[cur].pred;
        }
        if (cur >= 0) stop = cur;
        if (cnt < 2) continue;
        orc_chain_t *c = &chains[nc++];
        c->strand = a[best].strand;
        c->n_anchors = (int32_t)cnt;
        c->score = a[best].f - (stop >= 0 ? a[stop].f : 0);
        c->x_first = a[first].x;
        c->x_last = a[best].x;
        c->y_first = a[first].y;
        c->y_last = a[best].y;
    }
    free(a);
    return nc;
}

/* ------------------------------------------------- second chaining round */

/*
 * "Chaining", last paragraph: around each of a protein's top chains,
 * every 5-mer of the protein is matched against every 5-mer of the local
 * genome region (no sampling, no binning), and the anchors are chained
 * with the gap g' = 3 dy - dx (dx in bases) and the same penalty, Eq. 3.
 *
 * Readings:
 *   - The local region is given by the caller as a (protein, region,
 *     strand) pair, the same pairs the DP aligns: the region's aligned
 *     strand (its reverse complement for strand -1) is read in all three
 *     frames, a 5-mer starting at every base position x with a full five
 *     codons.  k-mers use the reduced alphabet of the first round (phi),
 *     stop codons and codons with a base outside ACGT included (phi 14 and
 *     15), as are X residues of the protein.
 *   - Anchors (x, y): x the base of the 5-mer's first codon on the aligned
 *     strand, y the residue of its first residue.  Sorted by (x, y); f and
 *     the predecessor rule as in the first round (x_i <= x_j, y_i < y_j,
 *     alpha = min(dy, k), the first best predecessor, f >= k).
 *   - The pair's result is its best chain: the anchor with the largest f
 *     (the earliest on ties) and its predecessors; none if it has a single
 *     anchor.  Its score is that f.
 */
typedef struct {
    int32_t n_anchors, reserved;
    int64_t score;
    int64_t x_first, x_last, y_first, y_last;
} orc_chain2_t;

static int ch_cmp_xy(const void *a, const void *b)
{
    const int64_t *p = (const int64_t *)a, *q = (const int64_t *)b;
    if (p[0] != q[0]) return p[0] < q[0] ? -1 : 1;
    return p[1] < q[1] ? -1 : p[1] > q[1];
}

/* Anchors of the pair as (x, y) pairs in out[2 * cap], sorted; returns the
 * count (which may exceed cap), or -1. */
int64_t orc_refine_anchors(const char *prot, int64_t m, const char *nt, int64_t n, int strand, int k,
                           int64_t *out, int64_t cap)
{
    char *seq = (char *)malloc((size_t)n + 1);
    if (!seq) return -1;
    for (int64_t t = 0; t < n; ++t) seq[t] = strand >= 0 ? nt[t] : ch_complement(nt[n - 1 - t]);
    int64_t cnt = 0;
    for (int64_t x = 0; x + 3 * k <= n; ++x) {
        uint64_t gk = 0;
        for (int u = 0; u < k; ++u) gk = gk * 16 + (uint64_t)orc_phi(ch_translate(seq + x + 3 * u));
        for (int64_t y = 0; y + k <= m; ++y) {
            uint64_t pk = 0;
            for (int u = 0; u < k; ++u) pk = pk * 16 + (uint64_t)orc_phi((unsigned char)prot[y + u]);
            if (pk != gk) continue;
            if (cnt < cap) { out[2 * cnt] = x; out[2 * cnt + 1] = y; }
            ++cnt;
        }
    }
    free(seq);
    if (cnt <= cap) qsort(out, (size_t)cnt, 2 * sizeof(int64_t), ch_cmp_xy);
    return cnt;
}

/* Chain n sorted (x, y) anchors with g' = 3 dy - dx: f of every anchor in
 * f_out (may be NULL) and the best chain in *c.  Returns 0, or -1. */
int orc_refine_chain(const int64_t *anc, int64_t n, int k, orc_chain2_t *c, int64_t *f_out)
{
    int64_t *f = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int64_t *pred = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    if (!f || !pred) { free(f); free(pred); return -1; }
    const int64_t S = CH_SCALE;
    int64_t best = -1;
    for (int64_t j = 0; j < n; ++j) {
        f[j] = (int64_t)k * S;
        pred[j] = -1;
        for (int64_t i = 0; i < j; ++i) {
            const int64_t dx = anc[2 * j] - anc[2 * i], dy = anc[2 * j + 1] - anc[2 * i + 1];
            if (dx < 0 || dy <= 0) continue;
            const int64_t pen = orc_gap_penalty(3 * dy - dx);
            if (pen < 0) continue;
            const int64_t cand = f[i] + (dy < k ? dy : k) * S - pen;
            if (cand > f[j]) { f[j] = cand; pred[j] = i; }
        }
        if (f_out) f_out[j] = f[j];
        if (best < 0 || f[j] > f[best]) best = j;
    }
    memset(c, 0, sizeof(*c));
    if (best >= 0 && pred[best] >= 0) {
        int64_t cnt = 0, cur = best, first = best;
        while (cur >= 0) { first = cur; ++cnt; cur = pred[cur]; }
        c->n_anchors = (int32_t)cnt;
        c->score = f[best];
        c->x_first = anc[2 * first];
        c->x_last = anc[2 * best];
        c->y_first = anc[2 * first + 1];
        c->y_last = anc[2 * best + 1];
    }
    free(f);
    free(pred);
    return 0;
}
