/*
 * oracle.c -- plain CPU oracle for the spliced protein-to-genome DP.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * statement of what the GPU path must compute.  Only the tests, the smoke
 * check and the CPU-baseline leg of the benchmark may load it.  It shares no
 * code, header, table or constant with the CUDA library: every table below
 * (genetic code, splice signals, alphabet) is written out here on its own.
 *
 * What it computes (Li 2022, "Protein-to-genome alignment with miniprot"):
 *   - Eq. 7 (Methods, "DP for protein-to-genome alignment"): states I, D,
 *     A, B, C and H over genome position i (1..|T|) and residue j (1..|P|),
 *     with the match term read as H[i-3][j-1] + s(i,j) (the printed
 *     H[i-3][j] cannot advance j; the worked example and Eq. 5 both consume
 *     one residue per codon).
 *   - The final splice model d(i), a(i) (Methods, "Splice models"), or the
 *     simple GT-AG model with cost p defined right after Eq. 7.
 *   - Local mode: H restarts at 0; the best cell is the largest H, ties to
 *     the smallest i and then the smallest j.
 *   - Ties inside every max go to the earliest term in the printed order of
 *     Eq. 7 (open before extend; M, I, D, F1, F2, G1, G2, A, B, C for H);
 *     the restart to 0 wins a tie at 0.
 *   - Split codons of phase-1/2 introns are not scored (Methods, after
 *     Eq. 7).
 *   - Profile queries (Discussion: position-specific substitution and gap
 *     costs): with orc_params.prof set, s(i,j) is the profile's score of the
 *     codon's translation at residue position j, and the I and D states of
 *     column j use that column's gap open and extension costs.
 *
 * Everything is int32 with full (|T|+1) x (|P|+1) matrices for all six
 * states; the traceback re-evaluates the recurrence at each cell, so no
 * direction codes are stored.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_NEG_INF (INT32_MIN / 4)

/* Protein / translated amino-acid alphabet: BLOSUM order, then stop, then X. */
static const char ORC_AA[] = "ARNDCQEGHILKMFPSTWYV*X";
#define ORC_AA_STOP 20
#define ORC_AA_X 21

/* Standard genetic code (NCBI table 1) in the customary T, C, A, G order of
 * first, second and third codon base. */
static const char ORC_CODE_TCAG[] =
    "FFLLSSSSYY**CC*WLLLLPPPPHHQQRRRRIIIMTTTTNNKKSSRRVVVVAAAADDEEGGGG";

typedef struct {
    int32_t q, e, f, r, stop;   /* gap open, gap extend, frameshift, intron, stop codon */
    int32_t mat[22][22];        /* [translated aa][protein residue], ORC_AA order */
    int32_t splice_model;       /* 0: the final model; 1: the simple GT-AG model */
    int32_t splice_p;           /* simple model: cost p of a donor without GT / acceptor without AG */
    int32_t mode;               /* 0 local; 1 global (from cell (0,0) to (|T|,|P|)); 2 extension
                                   (from (0,0), ending anywhere) */
    const int32_t *prof;        /* NULL, or the position-specific costs of a profile query
                                   (Discussion: position-specific substitution and gap costs):
                                   for residue position j = 1..|P|, prof[ORC_PW*j + c] is the score
                                   of a codon translating to c (ORC_AA order, 20 = stop codon)
                                   against position j, in place of mat[c][P[j]] and -stop; for
                                   j = 0..|P|, prof[ORC_PW*j + 21] and prof[ORC_PW*j + 22] are the
                                   gap open and extension costs of column j: an I step consuming
                                   residue j, a D step adding a codon after residue j (j = 0:
                                   before the first residue) */
} orc_params;

#define ORC_PW 23               /* ints per position of a profile */

typedef struct {
    int32_t score;
    int32_t status;             /* 0 ok, 1 cigar capacity, 2 degenerate intron, 3 bad input */
    int32_t prot_st, prot_en;   /* 0-based half-open on the protein */
    int32_t nt_st, nt_en;       /* 0-based half-open on the INPUT's forward strand */
    int32_t n_cigar;
} orc_result;

/* CIGAR op codes: len << 4 | code. */
enum { OP_M = 0, OP_I = 1, OP_D = 2, OP_F = 3, OP_G = 4, OP_N = 5, OP_U = 6, OP_V = 7 };

/* ---------------------------------------------------------------- encoding */

/* Nucleotide letter -> 0..3 (A, C, G, T); anything else -> -1. */
int orc_nt_code(int ch)
{
    switch (ch) {
    case 'A': case 'a': return 0;
    case 'C': case 'c': return 1;
    case 'G': case 'g': return 2;
    case 'T': case 't': return 3;
    default: return -1;
    }
}

/* Amino-acid letter -> index in ORC_AA; letters outside the 20 map to X. */
int orc_aa_code(int ch)
{
    int c = (ch >= 'a' && ch <= 'z') ? ch - 32 : ch;
    for (int k = 0; k < 21; ++k)
        if (ORC_AA[k] == c) return k;
    return ORC_AA_X;
}

static int tcag_index(int base_acgt)
{
    /* A C G T -> position in the T C A G ordering */
    static const int m[4] = {2, 1, 3, 0};
    return m[base_acgt];
}

/* Translate the codon b1 b2 b3 (0..3 each, ACGT) to an ORC_AA index. */
int orc_translate(int b1, int b2, int b3)
{
    char aa = ORC_CODE_TCAG[16 * tcag_index(b1) + 4 * tcag_index(b2) + tcag_index(b3)];
    return orc_aa_code(aa == '*' ? '*' : aa);
}

/* ------------------------------------------------------- splice signals */

/* Base at 1-based position x of T, or -1 outside 1..n. */
static int base_at(const int8_t *T, int n, int x)
{
    return (x >= 1 && x <= n) ? T[x] : -1;
}

enum { A_ = 0, C_ = 1, G_ = 2, T_ = 3 };

/* Donor score d(x) of the final splice model (Methods, "Splice models"):
 * looks at T[x+1..x+3]; bases outside T match nothing. */
int orc_donor(const int8_t *T, int n, int x)
{
    int b1 = base_at(T, n, x + 1), b2 = base_at(T, n, x + 2), b3 = base_at(T, n, x + 3);
    if (b1 == G_ && b2 == T_ && (b3 == A_ || b3 == G_)) return 0;   /* GTA, GTG */
    if (b1 == G_ && b2 == T_ && (b3 == C_ || b3 == T_)) return 8;   /* GTC, GTT */
    if (b1 == G_ && b2 == C_) return 15;                            /* GC */
    if (b1 == A_ && b2 == T_) return 21;                            /* AT */
    return 30;
}

/* Acceptor score a(x) of the final splice model: looks at T[x-2..x]. */
int orc_acceptor(const int8_t *T, int n, int x)
{
    int b1 = base_at(T, n, x - 2), b2 = base_at(T, n, x - 1), b3 = base_at(T, n, x);
    if ((b1 == C_ || b1 == T_) && b2 == A_ && b3 == G_) return 0;   /* CAG, TAG */
    if ((b1 == A_ || b1 == G_) && b2 == A_ && b3 == G_) return 8;   /* AAG, GAG */
    if (b2 == A_ && b3 == C_) return 21;                            /* AC */
    return 30;
}

/* Simple model (Methods, "DP for protein-to-genome alignment", the
 * definitions right after Eq. 7): d(x) = 0 if T[x+1..x+2] is GT, else p;
 * a(x) = 0 if T[x-1..x] is AG, else p.  Bases outside T match nothing. */
int orc_donor_simple(const int8_t *T, int n, int x, int p)
{
    return (base_at(T, n, x + 1) == G_ && base_at(T, n, x + 2) == T_) ? 0 : p;
}

int orc_acceptor_simple(const int8_t *T, int n, int x, int p)
{
    return (base_at(T, n, x - 1) == A_ && base_at(T, n, x) == G_) ? 0 : p;
}

/* d(x) and a(x) under the model the parameters select. */
static int32_t splice_d(const orc_params *p, const int8_t *T, int n, int x)
{
    return p->splice_model == 1 ? orc_donor_simple(T, n, x, p->splice_p) : orc_donor(T, n, x);
}

static int32_t splice_a(const orc_params *p, const int8_t *T, int n, int x)
{
    return p->splice_model == 1 ? orc_acceptor_simple(T, n, x, p->splice_p) : orc_acceptor(T, n, x);
}

/* ------------------------------------------------------------- the DP */

typedef struct {
    int n, m;                  /* |T|, |P| */
    int8_t *T;                 /* T[1..n] base codes */
    int8_t *P;                 /* P[1..m] residue codes */
    int32_t *H, *I, *D, *A, *B, *C;
    const orc_params *p;
} dp_t;

#define IDX(dp, i, j) ((size_t)(i) * (size_t)((dp)->m + 1) + (size_t)(j))

static int32_t getH(const dp_t *dp, int i, int j)
{
    if (i < 0 || j < 0) return ORC_NEG_INF;
    return dp->H[IDX(dp, i, j)];
}
static int32_t getS(const dp_t *dp, const int32_t *X, int i, int j)
{
    (void)dp;
    if (i < 0 || j < 0) return ORC_NEG_INF;
    return X[IDX(dp, i, j)];
}

static int32_t max2(int32_t a, int32_t b) { return a >= b ? a : b; }

/* s(i,j): the codon ending at i against residue j (Eq. 6 / Eq. 7).  A stop
 * codon scores -stop against any residue; i < 3 has no codon. */
static int32_t subst(const dp_t *dp, int i, int j)
{
    if (i < 3) return ORC_NEG_INF;
    int aa = orc_translate(dp->T[i - 2], dp->T[i - 1], dp->T[i]);
    if (dp->p->prof) return dp->p->prof[ORC_PW * j + aa];
    if (aa == ORC_AA_STOP) return -dp->p->stop;
    return dp->p->mat[aa][dp->P[j]];
}

/* Gap open and extension costs of column j (Eq. 7's q and e, or the
 * profile's costs of position j). */
static int32_t gap_q(const orc_params *p, int j) { return p->prof ? p->prof[ORC_PW * j + 21] : p->q; }
static int32_t gap_e(const orc_params *p, int j) { return p->prof ? p->prof[ORC_PW * j + 22] : p->e; }

static int32_t dfun(const dp_t *dp, int x) { return splice_d(dp->p, dp->T, dp->n, x); }
static int32_t afun(const dp_t *dp, int x) { return splice_a(dp->p, dp->T, dp->n, x); }

/* The ten H terms of Eq. 7 at (i, j) in printed order:
 * 0 M, 1 I, 2 D, 3 F1, 4 F2, 5 G1, 6 G2, 7 A, 8 B, 9 C. */
static void h_terms(const dp_t *dp, int i, int j, int32_t t[10])
{
    const orc_params *p = dp->p;
    t[0] = (i >= 3 && j >= 1) ? getH(dp, i - 3, j - 1) + subst(dp, i, j) : ORC_NEG_INF;
    t[1] = dp->I[IDX(dp, i, j)];
    t[2] = dp->D[IDX(dp, i, j)];
    t[3] = getH(dp, i - 1, j - 1) - p->f;
    t[4] = getH(dp, i - 2, j - 1) - p->f;
    t[5] = getH(dp, i - 1, j) - p->f;
    t[6] = getH(dp, i - 2, j) - p->f;
    t[7] = dp->A[IDX(dp, i, j)] - afun(dp, i);
    t[8] = dp->B[IDX(dp, i, j)] - afun(dp, i - 2);
    t[9] = dp->C[IDX(dp, i, j)] - afun(dp, i - 1);
}

/* Fill all six matrices by Eq. 7 in global or extension mode: the path
 * starts at cell (0, 0) (H = 0, every other state -inf there), so row 0 and
 * column 0 follow the recurrence too (row 0 only through I, column 0
 * through D, G and the phase-0 intron state A), and H has no restart. */
static void fill_anchored(dp_t *dp)
{
    const orc_params *p = dp->p;
    int n = dp->n, m = dp->m;
    for (int i = 0; i <= n; ++i) {
        for (int j = 0; j <= m; ++j) {
            size_t c = IDX(dp, i, j);
            if (i == 0 && j == 0) {
                dp->H[c] = 0;
                dp->I[c] = dp->D[c] = dp->A[c] = dp->B[c] = dp->C[c] = ORC_NEG_INF;
                continue;
            }
            dp->I[c] = j >= 1 ? max2(getH(dp, i, j - 1) - gap_q(p, j), getS(dp, dp->I, i, j - 1)) - gap_e(p, j)
                              : ORC_NEG_INF;
            dp->D[c] = max2(getH(dp, i - 3, j) - gap_q(p, j), getS(dp, dp->D, i - 3, j)) - gap_e(p, j);
            dp->A[c] = max2(getH(dp, i - 1, j) - p->r - dfun(dp, i - 1), getS(dp, dp->A, i - 1, j));
            dp->B[c] = max2(getH(dp, i - 1, j - 1) - p->r - dfun(dp, i), getS(dp, dp->B, i - 1, j));
            dp->C[c] = max2(getH(dp, i - 1, j - 1) - p->r - dfun(dp, i + 1), getS(dp, dp->C, i - 1, j));
            int32_t t[10];
            h_terms(dp, i, j, t);
            int32_t h = t[0];
            for (int k = 1; k < 10; ++k) h = max2(h, t[k]);
            dp->H[c] = h;
        }
    }
}

/* Fill all six matrices by Eq. 7 (local mode). */
static void fill(dp_t *dp)
{
    const orc_params *p = dp->p;
    int n = dp->n, m = dp->m;
    if (p->mode != 0) {
        fill_anchored(dp);
        return;
    }
    for (int j = 0; j <= m; ++j) {
        dp->H[IDX(dp, 0, j)] = 0;
        dp->I[IDX(dp, 0, j)] = dp->D[IDX(dp, 0, j)] = ORC_NEG_INF;
        dp->A[IDX(dp, 0, j)] = dp->B[IDX(dp, 0, j)] = dp->C[IDX(dp, 0, j)] = ORC_NEG_INF;
    }
    for (int i = 1; i <= n; ++i) {
        dp->H[IDX(dp, i, 0)] = 0;
        dp->I[IDX(dp, i, 0)] = dp->D[IDX(dp, i, 0)] = ORC_NEG_INF;
        dp->A[IDX(dp, i, 0)] = dp->B[IDX(dp, i, 0)] = dp->C[IDX(dp, i, 0)] = ORC_NEG_INF;
        for (int j = 1; j <= m; ++j) {
            size_t c = IDX(dp, i, j);
            dp->I[c] = max2(getH(dp, i, j - 1) - gap_q(p, j), getS(dp, dp->I, i, j - 1)) - gap_e(p, j);
            dp->D[c] = max2(getH(dp, i - 3, j) - gap_q(p, j), getS(dp, dp->D, i - 3, j)) - gap_e(p, j);
            dp->A[c] = max2(getH(dp, i - 1, j) - p->r - dfun(dp, i - 1), getS(dp, dp->A, i - 1, j));
            dp->B[c] = max2(getH(dp, i - 1, j - 1) - p->r - dfun(dp, i), getS(dp, dp->B, i - 1, j));
            dp->C[c] = max2(getH(dp, i - 1, j - 1) - p->r - dfun(dp, i + 1), getS(dp, dp->C, i - 1, j));
            int32_t t[10];
            h_terms(dp, i, j, t);
            int32_t h = t[0];
            for (int k = 1; k < 10; ++k) h = max2(h, t[k]);
            dp->H[c] = h > 0 ? h : 0;
        }
    }
}

/* Emit an op into a reversed op list, merging consecutive M. */
typedef struct {
    uint32_t *ops;
    int n, cap, overflow;
} oplist;

static void push_op(oplist *L, int code, int len)
{
    if (code == OP_M && L->n > 0 && (L->ops[L->n - 1] & 0xf) == OP_M) {
        L->ops[L->n - 1] += (uint32_t)len << 4;
        return;
    }
    if (L->n >= L->cap) { L->overflow = 1; return; }
    L->ops[L->n++] = ((uint32_t)len << 4) | (uint32_t)code;
}

/* Trace back from (bi, bj) to the restart cell, re-evaluating Eq. 7 at each
 * step with the same tie order as the fill.  Returns the start cell. */
static int traceback(const dp_t *dp, int bi, int bj, oplist *L, int *si, int *sj)
{
    const orc_params *p = dp->p;
    int i = bi, j = bj, degenerate = 0;
    const int anchored = p->mode != 0;               /* global / extension: the path ends at (0, 0) */
    for (;;) {
        if (anchored ? (i == 0 && j == 0) : (i <= 0 || j <= 0)) break;   /* local: row/column 0 hold H = 0 */
        int32_t h = dp->H[IDX(dp, i, j)];
        if (!anchored && h == 0) break;              /* restart wins ties at 0 */
        int32_t t[10];
        h_terms(dp, i, j, t);
        int src = -1;
        for (int k = 0; k < 10; ++k)
            if (t[k] == h) { src = k; break; }
        if (src < 0) return -1;                      /* cannot happen */
        if (src == 0) { push_op(L, OP_M, 1); i -= 3; j -= 1; }
        else if (src == 3) { push_op(L, OP_F, 1); i -= 1; j -= 1; }
        else if (src == 4) { push_op(L, OP_F, 2); i -= 2; j -= 1; }
        else if (src == 5) { push_op(L, OP_G, 1); i -= 1; }
        else if (src == 6) { push_op(L, OP_G, 2); i -= 2; }
        else if (src == 1) {                         /* I run: residues, no nt */
            int k = 0;
            for (;;) {
                ++k;
                int32_t open = getH(dp, i, j - 1) - gap_q(p, j) - gap_e(p, j);
                int32_t ext = getS(dp, dp->I, i, j - 1) - gap_e(p, j);
                j -= 1;
                if (open >= ext) break;
            }
            push_op(L, OP_I, k);
        } else if (src == 2) {                       /* D run: codons, no residue */
            int k = 0;
            for (;;) {
                ++k;
                int32_t open = getH(dp, i - 3, j) - gap_q(p, j) - gap_e(p, j);
                int32_t ext = getS(dp, dp->D, i - 3, j) - gap_e(p, j);
                i -= 3;
                if (open >= ext) break;
            }
            push_op(L, OP_D, k);
        } else if (src == 7) {                       /* phase-0 intron */
            int iexit = i;
            for (;;) {
                int32_t open = getH(dp, i - 1, j) - p->r - dfun(dp, i - 1);
                int32_t ext = getS(dp, dp->A, i - 1, j);
                if (open >= ext) break;
                i -= 1;
            }
            /* opened at i: intron T[i..iexit] */
            push_op(L, OP_N, iexit - i + 1);
            i -= 1;
        } else {                                     /* phase-1 (B) or phase-2 (C) intron */
            int iexit = i;
            int32_t *X = (src == 8) ? dp->B : dp->C;
            for (;;) {
                int32_t open = getH(dp, i - 1, j - 1) - p->r - dfun(dp, src == 8 ? i : i + 1);
                int32_t ext = getS(dp, X, i - 1, j);
                if (open >= ext) break;
                i -= 1;
            }
            int len = iexit - i - 2;                 /* intron length */
            if (len < 1) degenerate = 1;
            push_op(L, src == 8 ? OP_U : OP_V, len > 0 ? len : 0);
            i -= 1; j -= 1;
        }
    }
    *si = i < 0 ? 0 : i;
    *sj = j < 0 ? 0 : j;
    return degenerate;
}

/* Align protein `prot` (ASCII, plen) to genome `nt` (ASCII ACGT, tlen) on
 * the given strand (+1, or -1 = reverse complement of nt).  Writes the CIGAR
 * (forward op order) to cigar[0..cap).  Returns 0 on success. */
int orc_align(const orc_params *p, const char *prot, int32_t plen, const char *nt, int32_t tlen,
              int32_t strand, orc_result *res, uint32_t *cigar, int32_t cap)
{
    memset(res, 0, sizeof(*res));
    dp_t dp;
    memset(&dp, 0, sizeof(dp));
    dp.n = tlen;
    dp.m = plen;
    dp.p = p;
    dp.T = (int8_t *)malloc((size_t)tlen + 1);
    dp.P = (int8_t *)malloc((size_t)plen + 1);
    if (!dp.T || !dp.P) { free(dp.T); free(dp.P); res->status = 3; return -1; }
    for (int i = 1; i <= tlen; ++i) {
        int b = orc_nt_code(nt[strand < 0 ? tlen - i : i - 1]);
        if (b < 0) { free(dp.T); free(dp.P); res->status = 3; return -1; }
        dp.T[i] = (int8_t)(strand < 0 ? 3 - b : b);
    }
    for (int j = 1; j <= plen; ++j) dp.P[j] = (int8_t)orc_aa_code(prot[j - 1]);

    size_t cells = (size_t)(tlen + 1) * (size_t)(plen + 1);
    int32_t *buf = (int32_t *)malloc(cells * 6 * sizeof(int32_t));
    if (!buf) { free(dp.T); free(dp.P); res->status = 3; return -1; }
    dp.H = buf; dp.I = buf + cells; dp.D = buf + 2 * cells;
    dp.A = buf + 3 * cells; dp.B = buf + 4 * cells; dp.C = buf + 5 * cells;
    fill(&dp);

    /* best cell: largest H, then smallest i, then smallest j (local: over
     * cells after a residue and a base; extension: over every cell, (0, 0)
     * with H = 0 included); global: the cell (|T|, |P|) */
    int32_t best = 0;
    int bi = 0, bj = 0;
    if (p->mode == 1) {
        bi = tlen; bj = plen;
        best = dp.H[IDX(&dp, tlen, plen)];
    } else {
        for (int i = p->mode == 2 ? 0 : 1; i <= tlen; ++i)
            for (int j = p->mode == 2 ? 0 : 1; j <= plen; ++j)
                if (dp.H[IDX(&dp, i, j)] > best) { best = dp.H[IDX(&dp, i, j)]; bi = i; bj = j; }
    }

    res->score = best;
    if (best > 0 || p->mode == 1) {
        uint32_t *rev = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(cap > 0 ? cap : 1));
        oplist L = {rev, 0, cap, 0};
        int si = 0, sj = 0;
        int deg = traceback(&dp, bi, bj, &L, &si, &sj);
        for (int k = 0; k < L.n; ++k) cigar[k] = rev[L.n - 1 - k];
        free(rev);
        res->n_cigar = L.n;
        res->prot_st = sj;
        res->prot_en = bj;
        if (strand < 0) { res->nt_st = tlen - bi; res->nt_en = tlen - si; }
        else { res->nt_st = si; res->nt_en = bi; }
        if (L.overflow) res->status = 1;
        else if (deg) res->status = 2;
    }
    free(buf);
    free(dp.T);
    free(dp.P);
    return 0;
}

/* The filled H matrix ((tlen+1) x (plen+1), row-major, aligned
 * orientation) for tests that inspect the DP values themselves. */
int orc_fill_h(const orc_params *p, const char *prot, int32_t plen, const char *nt, int32_t tlen, int32_t strand,
               int32_t *h_out)
{
    dp_t dp;
    memset(&dp, 0, sizeof(dp));
    dp.n = tlen;
    dp.m = plen;
    dp.p = p;
    dp.T = (int8_t *)malloc((size_t)tlen + 1);
    dp.P = (int8_t *)malloc((size_t)plen + 1);
    if (!dp.T || !dp.P) { free(dp.T); free(dp.P); return -1; }
    for (int i = 1; i <= tlen; ++i) {
        int b = orc_nt_code(nt[strand < 0 ? tlen - i : i - 1]);
        if (b < 0) { free(dp.T); free(dp.P); return -1; }
        dp.T[i] = (int8_t)(strand < 0 ? 3 - b : b);
    }
    for (int j = 1; j <= plen; ++j) dp.P[j] = (int8_t)orc_aa_code(prot[j - 1]);
    size_t cells = (size_t)(tlen + 1) * (size_t)(plen + 1);
    int32_t *buf = (int32_t *)malloc(cells * 6 * sizeof(int32_t));
    if (!buf) { free(dp.T); free(dp.P); return -1; }
    dp.H = buf; dp.I = buf + cells; dp.D = buf + 2 * cells;
    dp.A = buf + 3 * cells; dp.B = buf + 4 * cells; dp.C = buf + 5 * cells;
    fill(&dp);
    memcpy(h_out, dp.H, cells * sizeof(int32_t));
    free(buf);
    free(dp.T);
    free(dp.P);
    return 0;
}

/* Score only: the same fill, returning the best H (for large cases). */
int32_t orc_score(const orc_params *p, const char *prot, int32_t plen, const char *nt, int32_t tlen,
                  int32_t strand)
{
    orc_result r;
    uint32_t dummy[1];
    if (orc_align(p, prot, plen, nt, tlen, strand, &r, dummy, 0) != 0) return -1;
    return r.score;
}

/* Score and end cell only, for pairs whose six full matrices would not fit
 * in memory: the same recurrence (Eq. 7), the same modes and the same
 * best-cell rule as orc_align, with each state kept for the last four rows
 * (the deepest look-back of Eq. 7 is H and D at i-3).  Every splice term
 * and the codon of row i depend on i alone, so they are evaluated once per
 * row.  Writes score, prot_en and the genome end of the best cell (nt_en on
 * strand +1, nt_st on strand -1, both on the input's forward strand); the
 * start coordinates are not computed (-1).  Returns 0, or -1 on bad input. */
int orc_score_end(const orc_params *p, const char *prot, int32_t plen, const char *nt, int32_t tlen,
                  int32_t strand, orc_result *res)
{
    memset(res, 0, sizeof(*res));
    const int n = tlen, m = plen;
    const int anchored = p->mode != 0;
    int8_t *T = (int8_t *)malloc((size_t)n + 1);
    int8_t *P = (int8_t *)malloc((size_t)m + 1);
    int32_t *buf = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m + 1) * 14);
    if (!T || !P || !buf) { free(T); free(P); free(buf); res->status = 3; return -1; }
    for (int i = 1; i <= n; ++i) {
        int b = orc_nt_code(nt[strand < 0 ? n - i : i - 1]);
        if (b < 0) { free(T); free(P); free(buf); res->status = 3; return -1; }
        T[i] = (int8_t)(strand < 0 ? 3 - b : b);
    }
    for (int j = 1; j <= m; ++j) P[j] = (int8_t)orc_aa_code(prot[j - 1]);
    /* rows i mod 4 of H and D; rows i mod 2 of A, B, C */
    int32_t *Hr[4], *Dr[4], *Ar[2], *Br[2], *Cr[2];
    for (int k = 0; k < 4; ++k) { Hr[k] = buf + (size_t)k * (m + 1); Dr[k] = buf + (size_t)(4 + k) * (m + 1); }
    for (int k = 0; k < 2; ++k) {
        Ar[k] = buf + (size_t)(8 + k) * (m + 1);
        Br[k] = buf + (size_t)(10 + k) * (m + 1);
        Cr[k] = buf + (size_t)(12 + k) * (m + 1);
    }
    int32_t best = 0;
    int bi = 0, bj = 0;
    for (int i = 0; i <= n; ++i) {
        int32_t *H = Hr[i & 3], *D = Dr[i & 3], *A = Ar[i & 1], *B = Br[i & 1], *C = Cr[i & 1];
        /* rows above 0 are outside the matrix (-inf) */
        const int32_t *H1 = i >= 1 ? Hr[(i - 1) & 3] : NULL, *H2 = i >= 2 ? Hr[(i - 2) & 3] : NULL;
        const int32_t *H3 = i >= 3 ? Hr[(i - 3) & 3] : NULL, *D3 = i >= 3 ? Dr[(i - 3) & 3] : NULL;
        const int32_t *A1 = i >= 1 ? Ar[(i - 1) & 1] : NULL, *B1 = i >= 1 ? Br[(i - 1) & 1] : NULL;
        const int32_t *C1 = i >= 1 ? Cr[(i - 1) & 1] : NULL;
        /* terms of row i that depend on i only */
        const int32_t rd_im1 = p->r + splice_d(p, T, n, i - 1), rd_i = p->r + splice_d(p, T, n, i);
        const int32_t rd_ip1 = p->r + splice_d(p, T, n, i + 1);
        const int32_t a_i = splice_a(p, T, n, i), a_im2 = splice_a(p, T, n, i - 2), a_im1 = splice_a(p, T, n, i - 1);
        int aa = -1;
        if (i >= 3) aa = orc_translate(T[i - 2], T[i - 1], T[i]);
        int32_t Ij = ORC_NEG_INF;                   /* I[i][j-1] */
        for (int j = 0; j <= m; ++j) {
            const int32_t h1j = H1 ? H1[j] : ORC_NEG_INF, h2j = H2 ? H2[j] : ORC_NEG_INF;
            const int32_t h1jm = (H1 && j >= 1) ? H1[j - 1] : ORC_NEG_INF;
            const int32_t h2jm = (H2 && j >= 1) ? H2[j - 1] : ORC_NEG_INF;
            if (anchored ? (i == 0 && j == 0) : (i == 0 || j == 0)) {
                /* local: row and column 0 hold H = 0; anchored: cell (0, 0) */
                H[j] = 0;
                D[j] = A[j] = B[j] = C[j] = ORC_NEG_INF;
                Ij = ORC_NEG_INF;
                continue;
            }
            const int32_t qj = gap_q(p, j), ej = gap_e(p, j);
            const int32_t I = j >= 1 ? max2(H[j - 1] - qj, Ij) - ej : ORC_NEG_INF;
            const int32_t Dv = max2((H3 ? H3[j] : ORC_NEG_INF) - qj, D3 ? D3[j] : ORC_NEG_INF) - ej;
            const int32_t Av = max2(h1j - rd_im1, A1 ? A1[j] : ORC_NEG_INF);
            const int32_t Bv = max2(h1jm - rd_i, B1 ? B1[j] : ORC_NEG_INF);
            const int32_t Cv = max2(h1jm - rd_ip1, C1 ? C1[j] : ORC_NEG_INF);
            int32_t h = ORC_NEG_INF;
            if (i >= 3 && j >= 1)
                h = H3[j - 1] + (p->prof ? p->prof[ORC_PW * j + aa] : aa == ORC_AA_STOP ? -p->stop : p->mat[aa][P[j]]);
            h = max2(h, I);
            h = max2(h, Dv);
            h = max2(h, h1jm - p->f);
            h = max2(h, h2jm - p->f);
            h = max2(h, h1j - p->f);
            h = max2(h, h2j - p->f);
            h = max2(h, Av - a_i);
            h = max2(h, Bv - a_im2);
            h = max2(h, Cv - a_im1);
            if (!anchored && h < 0) h = 0;
            H[j] = h;
            D[j] = Dv;
            A[j] = Av;
            B[j] = Bv;
            C[j] = Cv;
            Ij = I;
            /* best cell: largest H, then smallest i, then smallest j (local:
             * cells after a residue and a base; extension: every cell) */
            if (p->mode != 1 && h > best && (anchored || (i >= 1 && j >= 1))) { best = h; bi = i; bj = j; }
        }
    }
    if (p->mode == 1) { best = Hr[n & 3][m]; bi = n; bj = m; }
    res->score = best;
    res->prot_st = res->nt_st = res->nt_en = -1;
    res->prot_en = bj;
    if (strand < 0) res->nt_st = n - bi;
    else res->nt_en = bi;
    free(T);
    free(P);
    free(buf);
    return 0;
}

/* Op-sum rescoring of a CIGAR (no DP): walks the ops from the aligned start
 * (prot_st, nt position in the aligned orientation) and adds each op's cost
 * as defined by the transitions of Eq. 7.  Returns the score and writes the
 * end coordinates; returns ORC_NEG_INF if the path leaves the sequences. */
int32_t orc_rescore(const orc_params *p, const char *prot, int32_t plen, const char *nt, int32_t tlen,
                    int32_t strand, int32_t prot_st, int32_t nt_st_aligned, const uint32_t *cigar,
                    int32_t n_cigar, int32_t *prot_en, int32_t *nt_en_aligned)
{
    int8_t *T = (int8_t *)malloc((size_t)tlen + 1);
    for (int i = 1; i <= tlen; ++i) {
        int b = orc_nt_code(nt[strand < 0 ? tlen - i : i - 1]);
        T[i] = (int8_t)(strand < 0 ? 3 - b : b);
    }
    int i = nt_st_aligned, j = prot_st;   /* consumed so far */
    int64_t sc = 0;
    int bad = 0;
    for (int k = 0; k < n_cigar && !bad; ++k) {
        int op = (int)(cigar[k] & 0xf);
        int len = (int)(cigar[k] >> 4);
        switch (op) {
        case OP_M:
            for (int c = 0; c < len; ++c) {
                if (i + 3 > tlen || j + 1 > plen) { bad = 1; break; }
                int aa = orc_translate(T[i + 1], T[i + 2], T[i + 3]);
                int pc = orc_aa_code(prot[j]);
                sc += p->prof ? p->prof[ORC_PW * (j + 1) + aa] : (aa == ORC_AA_STOP) ? -p->stop : p->mat[aa][pc];
                i += 3; j += 1;
            }
            break;
        case OP_I:
            /* residues j+1 .. j+len: open at the first, extension at each */
            if (j + len > plen) { bad = 1; break; }
            sc -= gap_q(p, j + 1);
            for (int c = 1; c <= len; ++c) sc -= gap_e(p, j + c);
            j += len;
            break;
        case OP_D: sc -= gap_q(p, j) + (int64_t)gap_e(p, j) * len; i += 3 * len; break;
        case OP_F: sc -= p->f; i += len; j += 1; break;
        case OP_G: sc -= p->f; i += len; break;
        case OP_N: sc -= p->r + splice_d(p, T, tlen, i) + splice_a(p, T, tlen, i + len); i += len; break;
        case OP_U: sc -= p->r + splice_d(p, T, tlen, i + 1) + splice_a(p, T, tlen, i + len + 1);
                   i += len + 3; j += 1; break;
        case OP_V: sc -= p->r + splice_d(p, T, tlen, i + 2) + splice_a(p, T, tlen, i + len + 2);
                   i += len + 3; j += 1; break;
        default: bad = 1;
        }
        if (i > tlen || j > plen) bad = 1;
    }
    free(T);
    *prot_en = j;
    *nt_en_aligned = i;
    return bad ? ORC_NEG_INF : (int32_t)sc;
}

/* Reverse complement of an ASCII ACGT string (helper for tests). */
void orc_revcomp(const char *in, int32_t n, char *out)
{
    static const char comp[4] = {'T', 'G', 'C', 'A'};
    for (int k = 0; k < n; ++k) {
        int b = orc_nt_code(in[n - 1 - k]);
        out[k] = b < 0 ? 'N' : comp[b];
    }
}
