// Traceback of one pair from the H values its DP stored (Li 2022, Eq. 7,
// Methods, "DP for protein-to-genome alignment"): at each H cell the source
// is the first term of Eq. 7, in printed order, whose value equals H.  Used
// by the traceback kernel (a launch after the DP) and by the DP kernel itself
// for a pair whose last strip it has just finished; the latter reads the
// stream written in the same launch, so its loads bypass L1 (Coherent).
#pragma once
#include "mp_device.cuh"
#include "mp_internal.cuh"

namespace mpdp {
namespace {

constexpr int kNeg = -(1 << 28);
constexpr unsigned kTbFull = 0xffffffffu;

template <bool Coherent, typename T>
__device__ __forceinline__ T ld_tb(const T *p)
{
    if (Coherent) return __ldcg(p);
    return __ldg(p);
}


// Read access to one pair: its traceback stream (H of every cell), genome
// and protein.  Cells are 1-based (i, j) as in Eq. 7; row 0 and column 0
// hold H = 0 and rows above 0 are outside the matrix.
template <bool Coherent>
struct PairView {
    const uint8_t *base;
    size_t strip_bytes;
    bool wide;               // int32 stream (4 B per cell)
    const uint8_t *colmax;   // per strip, chunk and lane: the chunk's maximum H of the lane's cells
    int nchunks;
    bool w128;               // 128-residue strips (four cells per lane) instead of 64 (two)
    const uint32_t *g;       // packed genome
    const uint8_t *P;        // residue codes
    int n, m;
    const ScoreParams *sp;
    const int8_t *mat;       // shared-memory copy of sp->mat
    const int32_t *c0;       // anchored modes: column 0 (H[i][0]); null in local mode
    const ProfPos *pf;       // profile queries: positions 0..m; null otherwise
    const int32_t *ep;       // profile queries: gap-extension prefix sums per position

    // cost of an I run over residues j-k+1 .. j (open at the first, extension at each)
    __device__ __forceinline__ int gap_i(int j, int k) const
    {
        if (pf) return pf[j - k + 1].q + (__ldg(ep + j) - __ldg(ep + j - k));
        return sp->q + sp->e * k;
    }
    // cost of a D run of k codons in column j
    __device__ __forceinline__ int gap_d(int j, int k) const
    {
        if (pf) return pf[j].q + pf[j].e * k;
        return sp->q + sp->e * k;
    }

    __device__ __forceinline__ int H(int i, int j) const
    {
        if (i < 0 || j < 0) return kNeg;
        if (c0) {
            // anchored modes: row 0 is an I run from (0, 0); column 0 precomputed
            if (i == 0) return j == 0 ? 0 : -gap_i(j, j);
            if (j == 0) return __ldg(c0 + i);
        } else if (i == 0 || j == 0) {
            return 0;
        }
        const int ii = i - 1, jj = j - 1;
        if (w128) {
            // lane r/4 stores 16 B every two steps: [a(t), b(t), a(t+1), b(t+1)],
            // a = residues 4l, 4l+1 and b = 4l+2, 4l+3 as biased 16-bit halves
            const int s = jj >> 7, r = jj & 127, t = ii + r;
            const uint32_t w = ld_tb<Coherent>(reinterpret_cast<const uint32_t *>(
                base + static_cast<size_t>(s) * strip_bytes + static_cast<size_t>(t >> 1) * 512 + (r >> 2) * 16 +
                (t & 1) * 8 + ((r >> 1) & 1) * 4));
            return static_cast<int>((r & 1) ? (w >> 16) : (w & 0xffffu)) - 32768;
        }
        const int s = jj >> 6, r = jj & 63, t = ii + r;
        if (wide) {
            return ld_tb<Coherent>(reinterpret_cast<const int *>(base + static_cast<size_t>(s) * strip_bytes +
                                                                 static_cast<size_t>(t >> 2) * 1024 + (r >> 1) * 32 +
                                                                 (t & 3) * 8 + (r & 1) * 4));
        }
        const uint32_t w = ld_tb<Coherent>(reinterpret_cast<const uint32_t *>(
            base + static_cast<size_t>(s) * strip_bytes + static_cast<size_t>(t >> 2) * 512 + (r >> 1) * 16 +
            (t & 3) * 4));
        return static_cast<int>((r & 1) ? (w >> 16) : (w & 0xffffu)) - 32768;
    }
    // maximum H over chunk c of residue j (steps c*kChunk .. c*kChunk+kChunk-1)
    __device__ __forceinline__ int cmax(int c, int j) const
    {
        if (w128) {
            // one [a, b] pair of words per strip, chunk and lane
            const int jj = j - 1, s = jj >> 7, r = jj & 127;
            const size_t e = (static_cast<size_t>(s) * nchunks + c) * 32 + (r >> 2);
            const uint32_t w = ld_tb<Coherent>(reinterpret_cast<const uint32_t *>(colmax) + 2 * e + ((r >> 1) & 1));
            return static_cast<int>((r & 1) ? (w >> 16) : (w & 0xffffu)) - 32768;
        }
        const int jj = j - 1, s = jj >> 6, r = jj & 63;
        const size_t e = (static_cast<size_t>(s) * nchunks + c) * 32 + (r >> 1);
        if (wide) return ld_tb<Coherent>(reinterpret_cast<const int *>(colmax) + 2 * e + (r & 1));
        const uint32_t w = ld_tb<Coherent>(reinterpret_cast<const uint32_t *>(colmax) + e);
        return static_cast<int>((r & 1) ? (w >> 16) : (w & 0xffffu)) - 32768;
    }
    // base at 1-based position x (0..3), valid iff 1 <= x <= n
    __device__ __forceinline__ int b(int x) const
    {
        return (__ldg(g + ((x - 1) >> 4)) >> (2 * ((x - 1) & 15))) & 3;
    }
    __device__ __forceinline__ bool in(int x) const { return x >= 1 && x <= n; }
    // splice model: d(x) looks at T[x+1..x+3], a(x) at T[x-2..x]
    __device__ __forceinline__ int d(int x) const
    {
        const bool v1 = in(x + 1), v2 = in(x + 2), v3 = in(x + 3);
        return splice_donor(*sp, v1 ? b(x + 1) : 0, v2 ? b(x + 2) : 0, v3 ? b(x + 3) : 0, v1, v2, v3);
    }
    __device__ __forceinline__ int a(int x) const
    {
        const bool v1 = in(x - 2), v2 = in(x - 1), v3 = in(x);
        return splice_acceptor(*sp, v1 ? b(x - 2) : 0, v2 ? b(x - 1) : 0, v3 ? b(x) : 0, v1, v2, v3);
    }
    // s(i, j): codon T[i-2..i] against residue P[j]
    __device__ __forceinline__ int s(int i, int j) const
    {
        if (i < 3 || i > n) return kNeg;
        const int aa = c_code.v[b(i - 2) * 16 + b(i - 1) * 4 + b(i)];
        if (pf) return pf[j].s[aa];
        if (aa == 20) return -sp->stop;
        return mat[aa * 22 + P[j - 1]];
    }
};

struct OpWriter {
    uint32_t *ops;
    uint32_t cap, n;
    uint32_t pend_code, pend_len;
    bool overflow;

    __device__ void push(uint32_t code, uint32_t len)
    {
        if (pend_len && pend_code == MP_OP_M && code == MP_OP_M) {
            pend_len += len;
            return;
        }
        flush();
        pend_code = code;
        pend_len = len;
    }
    __device__ void flush()
    {
        if (!pend_len) return;
        if (n < cap) ops[n] = (pend_len << 4) | pend_code;
        else overflow = true;
        ++n;
        pend_len = 0;
    }
};

// First k in [1, kmax] (warp-parallel, 32 candidates per round) for which
// pred(k) holds; 0 if none.
template <typename Pred>
__device__ __forceinline__ int first_hit(int kmax, int lane, Pred pred)
{
    for (int k0 = 1; k0 <= kmax; k0 += 32) {
        const int k = k0 + lane;
        const unsigned bal = __ballot_sync(kTbFull, k <= kmax && pred(k));
        if (bal) return k0 + __ffs(bal) - 1;
    }
    return 0;
}

// Largest row x in [1, xhi] of residue column jc with pred(x), 0 if none.
// pred(x) may only hold where H(x, jc) >= thr: chunks whose stored maximum
// is below thr are skipped without reading their cells.
template <bool Coherent, typename Pred>
__device__ __forceinline__ int scan_column(const PairView<Coherent> &v, int jc, int xhi, int thr, int lane, Pred pred)
{
    if (xhi < 1 || jc < 1) return 0;
    const int r = (jc - 1) & (v.w128 ? 127 : 63);
    const int c_lo = r / kChunk, c_hi = (xhi - 1 + r) / kChunk;
    for (int cb = c_hi; cb >= c_lo; cb -= 32) {
        const int c = cb - lane;
        unsigned bal = __ballot_sync(kTbFull, c >= c_lo && v.cmax(c, jc) >= thr);
        while (bal) {
            const int cc = cb - (__ffs(bal) - 1);       // highest flagged chunk first
            bal &= bal - 1;
            const int xa = max(1, cc * kChunk - r + 1), xb = min(xhi, cc * kChunk - r + kChunk);
            for (int x0 = xb; x0 >= xa; x0 -= 32) {
                const int x = x0 - lane;
                const unsigned hit = __ballot_sync(kTbFull, x >= xa && pred(x));
                if (hit) return x0 - (__ffs(hit) - 1);
            }
        }
    }
    return 0;
}

// Walk back from the best cell to the restart.  At an H cell the source is
// the first term of Eq. 7 (M, I, D, F1, F2, G1, G2, A, B, C) whose value
// equals H, the restart when H = 0.  The gap and intron terms use the
// closed forms of their recurrences,
//   I[i][j] = max_k H[i][j-k] - q - e k,      D[i][j] = max_k H[i-3k][j] - q - e k,
//   A[i][j] = max_{i'<=i} H[i'-1][j] - r - d(i'-1),
//   B[i][j] = max_{i'<=i} H[i'-1][j-1] - r - d(i'),  C: the same with d(i'+1),
// each bounded above by H[i][j]; the run length the tie rule picks (open
// before extend) is the shortest one reaching H.
// The view of pair pd whose DP has run (o holds its stream width).
template <bool Coherent>
__device__ __forceinline__ PairView<Coherent> make_view(const TBArgs &a, const PairDesc &pd, const PairOut &o,
                                              const int8_t *mat_s)
{
    const int n = static_cast<int>(pd.nt_len);
    const int W = strip_w_of(pd.flags);
    const int nchunks = (n + W - 1 + kChunk - 1) / kChunk;
    const bool wide = (o.status & kStInt32Stream) != 0;
    // 2 bytes per cell (4 for the int32 stream), W cells per step
    const size_t strip_bytes = static_cast<size_t>(nchunks) * kChunk * W * 2 * (wide ? 2 : 1);
    const bool anchored = a.sp.mode != MP_MODE_LOCAL;
    return PairView<Coherent>{a.codes + pd.code_off, strip_bytes, wide,
                    a.codes + pd.code_off + static_cast<size_t>(pd.n_strips) * strip_bytes, nchunks, W == kStripWMax,
                    a.nt2 + pd.nt_word_off, a.prot + pd.prot_off, n, static_cast<int>(pd.prot_len),
                    &a.sp, mat_s, anchored ? a.col0 + pd.col0_off : nullptr,
                    (pd.flags & PF_PROF) ? a.prof + pd.prof_off : nullptr,
                    (pd.flags & PF_PROF) ? a.epre + pd.prof_off : nullptr};
}

template <bool Coherent>
__device__ void trace_pair(const TBArgs &a, const int8_t *mat_s, uint32_t p, int lane)
{
    const PairDesc pd = a.pairs[p];
    PairOut &o = a.out[p];
    const int n = static_cast<int>(pd.nt_len);
    const int m = static_cast<int>(pd.prot_len);
    // anchored modes: the path ends at cell (0, 0), whose row and column
    // follow the recurrence (PairView returns them) and H has no restart
    const bool anchored = a.sp.mode != MP_MODE_LOCAL;
    const PairView<Coherent> v = make_view<Coherent>(a, pd, o, mat_s);
    const int q = a.sp.q, e = a.sp.e, f = a.sp.f, r = a.sp.r;
    const int hmax = o.score > 0 ? o.score : 0;             // no H exceeds it (H[0][0] = 0 included)
    int i = o.best_ii + 1, j = o.best_jj + 1;
    if (a.sp.mode == MP_MODE_GLOBAL) {
        // global: the alignment ends at (|T|, |P|)
        i = n;
        j = m;
        const int hend = v.H(n, m);
        __syncwarp();
        if (lane == 0) {
            o.score = hend;
            o.best_ii = n - 1;
            o.best_jj = m - 1;
        }
    }
    // the opening row x of an intron in column jc at or above xhi, or -1:
    // rows from 1 by the pruned scan, then column 0 / row 0 in the anchored modes
    auto find_open = [&](int jc, int xhi, int thr, auto pred) -> int {
        if (xhi < 0 || jc < 0) return -1;
        if (jc >= 1) {
            const int x = scan_column(v, jc, xhi, thr, lane, pred);
            if (x) return x;
        } else if (anchored) {
            // column 0 (no stored maxima): a plain scan
            for (int x0 = xhi; x0 >= 1; x0 -= 32) {
                const int x = x0 - lane;
                const unsigned hit = __ballot_sync(kTbFull, x >= 1 && pred(x));
                if (hit) return x0 - (__ffs(hit) - 1);
            }
        }
        return (anchored && pred(0)) ? 0 : -1;
    };
    OpWriter w{a.ops + pd.cig_off, pd.cig_cap, 0, 0, 0, false};
    bool error = false;
    for (;;) {
        if (anchored) {
            if (i == 0 && j == 0) break;
            if (i < 0 || j < 0) { error = true; break; }
        } else if (i <= 0 || j <= 0) {
            break;
        }
        // M runs: cells (i - 3k, j - k) along the codon diagonal
        const int ik = i - 3 * lane, jk = j - lane;
        const bool inside = ik >= 1 && jk >= 1;
        const int hk = (inside || (anchored && ik >= 0 && jk >= 0)) ? v.H(ik, jk) : 0;
        int hn = __shfl_down_sync(kTbFull, hk, 1);
        if (lane == 31) hn = (ik >= 3 && jk >= 1) ? v.H(ik - 3, jk - 1) : kNeg;
        const bool is_m = inside && (anchored || hk > 0) && ik >= 3 && hk == hn + v.s(ik, jk);
        const unsigned nonm = __ballot_sync(kTbFull, !is_m);
        const int cnt = nonm ? __ffs(nonm) - 1 : 32;
        if (cnt > 0) {
            if (lane == 0) w.push(MP_OP_M, cnt);
            i -= 3 * cnt;
            j -= cnt;
        }
        if (cnt == 32) continue;
        const int h = __shfl_sync(kTbFull, hk, cnt);
        if (anchored) {
            if (i == 0 && j == 0) break;
        } else if (i <= 0 || j <= 0 || h <= 0) {
            break;                                           // restart wins a tie at 0
        }
        // I: residues against no genome (runs longer than kgap cannot reach
        // h from an H of at most hmax: every step costs at least e, or 1 in a
        // profile)
        const int kgap = v.pf ? hmax - h : (hmax - q - h) / e;
        int k = kgap >= 1 ? first_hit(j < kgap ? j : kgap, lane,
                                      [&](int kk) { return v.H(i, j - kk) - v.gap_i(j, kk) == h; })
                          : 0;
        if (k) { if (lane == 0) w.push(MP_OP_I, k); j -= k; continue; }
        // D: codons against no residue
        const int kgd = v.pf ? (hmax - v.pf[j].q - h) / v.pf[j].e : kgap;
        k = kgd >= 1 ? first_hit(i / 3 < kgd ? i / 3 : kgd, lane,
                                 [&](int kk) { return v.H(i - 3 * kk, j) - v.gap_d(j, kk) == h; })
                     : 0;
        if (k) { if (lane == 0) w.push(MP_OP_D, k); i -= 3 * k; continue; }
        // frameshifts
        if (v.H(i - 1, j - 1) - f == h) { if (lane == 0) w.push(MP_OP_F, 1); i -= 1; j -= 1; continue; }
        if (v.H(i - 2, j - 1) - f == h) { if (lane == 0) w.push(MP_OP_F, 2); i -= 2; j -= 1; continue; }
        if (v.H(i - 1, j) - f == h) { if (lane == 0) w.push(MP_OP_G, 1); i -= 1; continue; }
        if (v.H(i - 2, j) - f == h) { if (lane == 0) w.push(MP_OP_G, 2); i -= 2; continue; }
        // introns: the opening i' nearest to the exit i; the H cell before it is
        // x = i' - 1 (in local mode row 0 never matches since h > 0)
        const int va = h + v.a(i);
        int x = find_open(j, i - 1, va + r, [&](int xx) { return v.H(xx, j) - r - v.d(xx) == va; });
        if (x >= 0) {
            if (lane == 0) w.push(MP_OP_N, i - x);          // intron T[x+1..i]
            i = x;
            continue;
        }
        const int vb = h + v.a(i - 2), vc = h + v.a(i - 1);
        int op = MP_OP_U;
        x = find_open(j - 1, i - 1, vb + r, [&](int xx) { return v.H(xx, j - 1) - r - v.d(xx + 1) == vb; });
        if (x < 0) {
            op = MP_OP_V;
            x = find_open(j - 1, i - 1, vc + r, [&](int xx) { return v.H(xx, j - 1) - r - v.d(xx + 2) == vc; });
        }
        if (x < 0) { error = true; break; }
        const int L = i - x - 3;                              // intron length i - i' - 2
        if (L < 1) { error = true; break; }
        if (lane == 0) w.push(op, L);
        i = x;
        j -= 1;
    }
    if (lane == 0) {
        w.flush();
        o.n_ops = w.overflow ? 0 : w.n;
        o.st_ii = i > 0 ? i : 0;
        o.st_jj = j > 0 ? j : 0;
        if (error || w.overflow) o.status |= MP_ST_TRACE;
    }
}

}  // namespace
}  // namespace mpdp
