// Input packing, traceback and CIGAR compaction kernels.
//
// Traceback walks from the best cell back to the restart over the H values
// the DP kernel stored, following the paths of Li 2022 Eq. 7 (Methods, "DP
// for protein-to-genome alignment"): M, I, D, the four frameshift terms and
// the three intron states, with the intron coordinates of the phase-1/2
// states as the paper places them (after Eq. 7).  One warp per pair: codons
// of an M run, gap rows and intron columns are scanned 32 cells at a time.
#include "mp_device.cuh"
#include "mp_internal.cuh"
#include "traceback.cuh"

namespace mpdp {
namespace {

constexpr unsigned kFull = 0xffffffffu;

// ------------------------------------------------------------------ pack
__device__ __forceinline__ int nt_code(unsigned char c)
{
    switch (c) {
    case 'A': case 'a': return 0;
    case 'C': case 'c': return 1;
    case 'G': case 'g': return 2;
    case 'T': case 't': return 3;
    default: return -1;
    }
}

__device__ __forceinline__ uint8_t aa_code(unsigned char c)
{
    // ARNDCQEGHILKMFPSTWYV -> 0..19, '*' -> 20, anything else -> X (21)
    switch (c | 0x20) {
    case 'a': return 0;  case 'r': return 1;  case 'n': return 2;  case 'd': return 3;
    case 'c': return 4;  case 'q': return 5;  case 'e': return 6;  case 'g': return 7;
    case 'h': return 8;  case 'i': return 9;  case 'l': return 10; case 'k': return 11;
    case 'm': return 12; case 'f': return 13; case 'p': return 14; case 's': return 15;
    case 't': return 16; case 'w': return 17; case 'y': return 18; case 'v': return 19;
    default: return c == '*' ? 20 : 21;
    }
}

// One CTA per pair: residue codes, and the genome in the alignment
// orientation (reverse complement for strand -1) at 2 bits per base.
__global__ void pack_kernel(const PairDesc *pairs, uint32_t n, const char *ascii, uint8_t *prot,
                            uint32_t *nt2, PairOut *out)
{
    for (uint32_t p = blockIdx.x; p < n; p += gridDim.x) {
        const PairDesc pd = pairs[p];
        __shared__ int bad;
        if (threadIdx.x == 0) bad = 0;
        __syncthreads();
        const unsigned char *pa = reinterpret_cast<const unsigned char *>(ascii) + pd.asc_prot_off;
        for (uint32_t k = threadIdx.x; k < pd.prot_len; k += blockDim.x) prot[pd.prot_off + k] = aa_code(pa[k]);
        const unsigned char *ta = reinterpret_cast<const unsigned char *>(ascii) + pd.asc_nt_off;
        const int n_nt = static_cast<int>(pd.nt_len);
        const int nwords = (n_nt + 15) / 16;
        uint32_t *g = nt2 + pd.nt_word_off;
        for (int w = -kNtPadWords + static_cast<int>(threadIdx.x); w < nwords + kNtPadWords;
             w += blockDim.x) {
            uint32_t word = 0;
            if (w >= 0 && w < nwords) {
                for (int k = 0; k < 16; ++k) {
                    const int pos = w * 16 + k;
                    if (pos >= n_nt) break;
                    int b;
                    if (pd.strand >= 0) {
                        b = nt_code(ta[pos]);
                    } else {
                        b = nt_code(ta[n_nt - 1 - pos]);
                        b = b < 0 ? b : 3 - b;
                    }
                    if (b < 0) { bad = 1; b = 0; }
                    word |= static_cast<uint32_t>(b) << (2 * k);
                }
            }
            g[w] = word;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            PairOut o;
            o.score = 0;
            o.status = bad ? MP_ST_BADSEQ : ((pd.flags & PF_BUDGET) ? MP_ST_BUDGET : 0);
            o.best_ii = o.best_jj = -1;
            o.st_ii = o.st_jj = 0;
            o.n_ops = 0;
            o.cig_out = 0;
            out[p] = o;
        }
        __syncthreads();
    }
}

__global__ void tb_kernel(const TBArgs a)
{
    __shared__ int8_t mat_s[22 * 22];
    for (int k = threadIdx.x; k < 22 * 22; k += blockDim.x) mat_s[k] = a.sp.mat[k / 22][k % 22];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t k = warp; k < a.n_work; k += nwarps) {
        const uint32_t p = a.work[k];
        const PairDesc &pd = a.pairs[p];
        const PairOut &o = a.out[p];
        if ((pd.flags & (PF_SCORE_ONLY | PF_SKIP | PF_BUDGET)) || (o.status & (MP_ST_ERRMASK | kStTraced)) ||
            (o.score <= 0 && a.sp.mode != MP_MODE_GLOBAL))
            continue;
        trace_pair<false>(a, mat_s, p, lane);
    }
}

// Test hook: H of every cell (i, j), 0 <= i <= |T|, 0 <= j <= |P|, of pair
// p, row-major, read through the traceback's own view of the stream.
__global__ void dump_h_kernel(const TBArgs a, uint32_t p, int32_t *h)
{
    __shared__ int8_t mat_s[22 * 22];
    for (int k = threadIdx.x; k < 22 * 22; k += blockDim.x) mat_s[k] = a.sp.mat[k / 22][k % 22];
    __syncthreads();
    const PairDesc pd = a.pairs[p];
    const PairView<false> v = make_view<false>(a, pd, a.out[p], mat_s);
    const size_t cols = static_cast<size_t>(pd.prot_len) + 1;
    const size_t cells = (static_cast<size_t>(pd.nt_len) + 1) * cols;
    for (size_t k = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; k < cells;
         k += static_cast<size_t>(gridDim.x) * blockDim.x)
        h[k] = v.H(static_cast<int>(k / cols), static_cast<int>(k % cols));
}

// ------------------------------------------------------------ compaction
// Exclusive scan of per-pair op counts (one CTA), then a reversed copy of
// each pair's ops into the compact array.
__global__ void scan_kernel(PairOut *out, uint32_t n, uint32_t *total)
{
    __shared__ uint32_t warp_sums[32];
    __shared__ uint32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (uint32_t base = 0; base < n; base += blockDim.x) {
        const uint32_t k = base + threadIdx.x;
        const uint32_t v = k < n ? out[k].n_ops : 0;
        uint32_t x = v;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t y = __shfl_up_sync(kFull, x, off);
            if (lane >= off) x += y;
        }
        if (lane == 31) warp_sums[warp] = x;
        __syncthreads();
        if (warp == 0) {
            uint32_t s = lane < static_cast<int>(blockDim.x >> 5) ? warp_sums[lane] : 0;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const uint32_t y = __shfl_up_sync(kFull, s, off);
                if (lane >= off) s += y;
            }
            warp_sums[lane] = s;
        }
        __syncthreads();
        const uint32_t excl = carry + (warp ? warp_sums[warp - 1] : 0) + x - v;
        if (k < n) out[k].cig_out = excl;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = excl + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = carry;
}

__global__ void copy_ops_kernel(const PairDesc *pairs, const PairOut *out, uint32_t n, const uint32_t *ops,
                                uint32_t *cig)
{
    const int lane = threadIdx.x & 31;
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t p = warp; p < n; p += nwarps) {
        const uint32_t cnt = out[p].n_ops, dst = out[p].cig_out;
        const uint32_t *src = ops + pairs[p].cig_off;
        for (uint32_t k = lane; k < cnt; k += 32) cig[dst + cnt - 1 - k] = src[k];
    }
}

}  // namespace

namespace {
// Column 0 in the anchored modes, where the path starts at cell (0, 0):
// H[0][0] = 0 and, for i >= 1, Eq. 7 with no residue consumed -- a codon
// deletion run (D), the frameshift insertions G1, G2 and the phase-0 intron
// state A (M, I, F1, F2, B and C need column -1):
//   D[i] = max(H[i-3] - q - e, D[i-3] - e)
//   A[i] = max(H[i-1] - r - d(i-1), A[i-1])
//   H[i] = max(D[i], H[i-1] - f, H[i-2] - f, A[i] - a(i)).
// Each row is a (max, +)-linear map of the state
//   s = (H[i], H[i-1], H[i-2], D[i], D[i-1], D[i-2], A[i]),
// so one warp per pair splits the rows into 32 segments: each lane composes
// the 7x7 transfer matrix of its segment, the segments' incoming states are
// then chained across the lanes (32 matrix-vector products), and each lane
// re-runs its segment from its incoming state, writing H.  The critical
// path is |T|/32 rows instead of |T|.  Rows past |T| hold -inf.
constexpr int kCol0Warps = 4;
constexpr int kS = 7;   // state size

struct Col0Ctx {
    const uint32_t *g;
    int n;
    int qe, e, f, r;
};

// base at 1-based position x (1 <= x <= n)
__device__ __forceinline__ int col0_base(const uint32_t *g, int x)
{
    return static_cast<int>((__ldg(g + ((x - 1) >> 4)) >> (2 * ((x - 1) & 15))) & 3);
}

// Splice terms as table lookups: a base is coded 0..3, a position outside
// the region 4; d(i-1) is kDon[T[i]][T[i+1]][T[i+2]] and a(i) is
// kAcc[T[i-2]][T[i-1]][T[i]], both 5 x 5 x 5, filled at launch from the
// splice model's own functions (so no data-dependent branch per row).
constexpr int kOut = 4;

// Sliding window of the codes of T[i-2..i+2] around row i.  The packed words
// ahead of the window are held in registers, the next one loaded 16 rows
// before its first base is needed (reads past the region fall in its zero
// padding).
struct SpliceWindow {
    int b[5];          // codes of T[i-2], T[i-1], T[i], T[i+1], T[i+2]
    int i;
    uint32_t w0, w1;   // the word holding T[i+3] and the one after it
    __device__ __forceinline__ void start(const Col0Ctx &c, int i0)
    {
        i = i0;
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            const int x = i0 - 2 + k;
            b[k] = (x >= 1 && x <= c.n) ? col0_base(c.g, x) : kOut;
        }
        const int wi = (i0 + 2) >> 4;                  // word of position i0 + 3
        w0 = __ldg(c.g + wi);
        w1 = __ldg(c.g + wi + 1);
    }
    __device__ __forceinline__ void advance(const Col0Ctx &c)
    {
        ++i;
#pragma unroll
        for (int k = 0; k < 4; ++k) b[k] = b[k + 1];
        const int x = i + 2;                           // the base entering the window
        b[4] = x <= c.n ? static_cast<int>((w0 >> (2 * ((x - 1) & 15))) & 3) : kOut;
        if (((x - 1) & 15) == 15) {                   // x ends its word: the next word comes in
            w0 = w1;
            w1 = __ldg(c.g + ((x - 1) >> 4) + 2);
        }
    }
    // r + d(i-1) and a(i) of the current row
    __device__ __forceinline__ void terms(const int16_t *don, const int16_t *acc, int r, int &rd, int &aa) const
    {
        rd = r + don[(b[2] * 5 + b[3]) * 5 + b[4]];
        aa = acc[(b[0] * 5 + b[1]) * 5 + b[2]];
    }
};

// One row on a state vector v = (H[i], H[i-1], H[i-2], D[i], D[i-1], D[i-2],
// A[i]) in place; rd = r + d(i), aa = a(i+1).  With clamp, every value stays
// >= NEG; without, values below NEG only drift further down (by at most a few
// thousand per row), which the 32-bit matrix phase absorbs.
template <typename T, bool CLAMP>
__device__ __forceinline__ void col0_row(T *v, const Col0Ctx &c, int rd, int aa)
{
    const T neg = static_cast<T>(kNeg);
    T dn = max(v[2] - c.qe, v[5] - c.e);
    T an = max(v[0] - rd, v[6]);
    T hn = max(max(dn, max(v[0], v[1]) - c.f), an - aa);
    if (CLAMP) {
        dn = max(dn, neg);
        an = max(an, neg);
        hn = max(hn, neg);
    }
    v[5] = v[4]; v[4] = v[3]; v[3] = dn;
    v[2] = v[1]; v[1] = v[0]; v[0] = hn;
    v[6] = an;
}

__global__ void __launch_bounds__(kCol0Warps * 32) col0_kernel(const PairDesc *pairs, uint32_t n_pairs,
                                                                 const uint32_t *nt2, const ScoreParams sp,
                                                                 const ProfPos *prof, int32_t *col0)
{
    __shared__ int16_t s_don[125], s_acc[125];
    for (int k = threadIdx.x; k < 125; k += blockDim.x) {
        const int c1 = k / 25, c2 = (k / 5) % 5, c3 = k % 5;
        const bool v1 = c1 != kOut, v2 = c2 != kOut, v3 = c3 != kOut;
        const int b1 = v1 ? c1 : 0, b2 = v2 ? c2 : 0, b3 = v3 ? c3 : 0;
        s_don[k] = static_cast<int16_t>(splice_donor(sp, b1, b2, b3, v1, v2, v3));
        s_acc[k] = static_cast<int16_t>(splice_acceptor(sp, b1, b2, b3, v1, v2, v3));
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const uint32_t nwarps = gridDim.x * kCol0Warps;
    for (uint32_t p = blockIdx.x * kCol0Warps + (threadIdx.x >> 5); p < n_pairs; p += nwarps) {
        const PairDesc pd = pairs[p];
        if (pd.flags & PF_SKIP) continue;
        const int n = static_cast<int>(pd.nt_len);
        // column 0's D runs take the gap costs of column 0 (a profile's position 0)
        const bool pq = (pd.flags & PF_PROF) != 0;
        const int q0 = pq ? prof[pd.prof_off].q : sp.q, e0 = pq ? prof[pd.prof_off].e : sp.e;
        const Col0Ctx c{nt2 + pd.nt_word_off, n, q0 + e0, e0, sp.f, sp.r};
        int32_t *h = col0 + pd.col0_off;
        const int L = (n + 31) / 32;
        const int r0 = lane * L + 1, r1 = min(n, (lane + 1) * L);     // this lane's rows (none if r0 > r1)
        const int cnt = r1 >= r0 ? r1 - r0 + 1 : 0;

        // 1. transfer matrix of the segment: column k is the state reached
        //    from the k-th unit state (0 at k, -inf elsewhere); the last
        //    segment's matrix is never used
        int32_t t[kS][kS];
#pragma unroll
        for (int k = 0; k < kS; ++k) {
#pragma unroll
            for (int j = 0; j < kS; ++j) t[k][j] = j == k ? 0 : kNeg;
        }
        // (one row per step: ptxas 13.0 at -O1 and above gave wrong matrices
        // for a three-rows-per-step form of this loop, correct at -O0 and in
        // 64 bits; the column-0 tests compare every value with the oracle)
        SpliceWindow w;
        if (cnt > 0 && lane < 31) {
            w.start(c, r0);
            for (int done = 0; done < cnt; ++done) {
                int rd, aa;
                w.terms(s_don, s_acc, c.r, rd, aa);
                if (done + 1 < cnt) w.advance(c);
#pragma unroll
                for (int k = 0; k < kS; ++k) col0_row<int32_t, false>(t[k], c, rd, aa);
            }
        }
        // 2. incoming state of every segment, chained across the lanes from
        //    s_0 = (0, -inf, ...); matrix entries are >= NEG less the drift of
        //    one segment and s is clamped, so the sums stay inside 32 bits
        int32_t s[kS], sin[kS];
#pragma unroll
        for (int k = 0; k < kS; ++k) s[k] = sin[k] = k == 0 ? 0 : kNeg;
        for (int l = 0; l < 31; ++l) {
            if (lane == l) {
#pragma unroll
                for (int k = 0; k < kS; ++k) sin[k] = s[k];
            }
            int32_t ns[kS];
#pragma unroll
            for (int j = 0; j < kS; ++j) ns[j] = kNeg;
#pragma unroll
            for (int k = 0; k < kS; ++k) {
#pragma unroll
                for (int j = 0; j < kS; ++j) ns[j] = max(ns[j], __shfl_sync(kFull, t[k][j], l) + s[k]);
            }
#pragma unroll
            for (int j = 0; j < kS; ++j) s[j] = max(ns[j], kNeg);
        }
        if (lane == 31) {
#pragma unroll
            for (int k = 0; k < kS; ++k) sin[k] = s[k];
        }
        // 3. re-run the segment from its incoming state (64-bit state: ptxas
        //    13.0 at -O1 and above turned an earlier 32-bit form of this
        //    recurrence into code returning +f for H[1][0]; correct at -O0)
        if (lane == 0) h[0] = 0;
        if (cnt > 0) {
            int64_t v[kS];
#pragma unroll
            for (int k = 0; k < kS; ++k) v[k] = sin[k];
            w.start(c, r0);
            for (int done = 0; done < cnt; ++done) {
                int rd, aa;
                w.terms(s_don, s_acc, c.r, rd, aa);
                if (done + 1 < cnt) w.advance(c);
                col0_row<int64_t, true>(v, c, rd, aa);
                h[r0 + done] = static_cast<int32_t>(v[0]);
            }
        }
        for (int i = n + 1 + lane; i <= n + kCol0Pad; i += 32) h[i] = kNeg;
    }
}
}  // namespace

cudaError_t launch_col0(const PairDesc *pairs, uint32_t n, const uint32_t *nt2, const ScoreParams &sp,
                        const ProfPos *prof, int32_t *col0, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    const uint32_t blocks = (n + kCol0Warps - 1) / kCol0Warps;
    col0_kernel<<<blocks < 4096 ? blocks : 4096, kCol0Warps * 32, 0, st>>>(pairs, n, nt2, sp, prof, col0);
    return cudaGetLastError();
}

namespace {
// Complement of one ASCII base (either case); anything else becomes N,
// which the pack step reports as a bad sequence.
__device__ __forceinline__ char complement_base(char ch)
{
    switch (ch | 0x20) {
    case 'a': return 'T';
    case 'c': return 'G';
    case 'g': return 'C';
    case 't': return 'A';
    default: return 'N';
    }
}

// One warp per rescoring pair: the protein, then the bases the alignment
// keeps (codons of M and D, the bases of F and G, the split codon around a
// U or V intron; an N intron and the intron of U or V are skipped), in the
// aligned orientation (reverse complement of the caller's region on strand
// -1).  Every copy is bounded by both the source region and the
// destination length.
__global__ void exon_gather_kernel(const ExonJob *jobs, uint32_t n, const PairDesc *aux, const char *src,
                                   const uint32_t *ops, char *dst)
{
    const int lane = threadIdx.x & 31;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; j < n; j += nwarps) {
        const ExonJob J = jobs[j];
        const PairDesc d = aux[j];
        for (uint32_t k = lane; k < d.prot_len; k += 32) dst[d.asc_prot_off + k] = src[J.src_prot_off + k];
        const int64_t nl = J.src_nt_len, out_len = d.nt_len;
        int64_t i = J.i0, o = 0;
        auto copy = [&](int64_t len) {
            for (int64_t t = lane; t < len; t += 32) {
                const int64_t a = i + t;
                if (a < 0 || a >= nl || o + t >= out_len) continue;
                dst[d.asc_nt_off + o + t] =
                    J.strand > 0 ? src[J.src_nt_off + a] : complement_base(src[J.src_nt_off + nl - 1 - a]);
            }
            i += len;
            o += len;
        };
        for (uint32_t u = 0; u < J.n_ops; ++u) {
            const uint32_t w = ops[J.op_off + u];
            const int64_t len = w >> 4;
            switch (w & 0xf) {
            case MP_OP_M: case MP_OP_D: copy(3 * len); break;
            case MP_OP_F: case MP_OP_G: copy(len); break;
            case MP_OP_N: i += len; break;
            case MP_OP_U: copy(1); i += len; copy(2); break;
            case MP_OP_V: copy(2); i += len; copy(1); break;
            default: break;                                   // I: residues only
            }
        }
    }
}
}  // namespace

cudaError_t launch_exon_gather(const ExonJob *jobs, uint32_t n, const PairDesc *aux, const char *src,
                               const uint32_t *ops, char *dst, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    const uint32_t blocks = (n + 7) / 8;
    exon_gather_kernel<<<blocks < 4096 ? blocks : 4096, 256, 0, st>>>(jobs, n, aux, src, ops, dst);
    return cudaGetLastError();
}

cudaError_t launch_pack(const PairDesc *pairs, uint32_t n, const char *ascii, uint8_t *prot, uint32_t *nt2,
                        PairOut *out, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    const uint32_t grid = n < 8192 ? n : 8192;
    pack_kernel<<<grid, 256, 0, st>>>(pairs, n, ascii, prot, nt2, out);
    return cudaGetLastError();
}

cudaError_t launch_dump_h(const TBArgs &a, uint32_t p, size_t cells, int32_t *h, cudaStream_t st)
{
    const size_t blocks = (cells + 255) / 256;
    dump_h_kernel<<<static_cast<unsigned>(blocks < 1024 ? (blocks ? blocks : 1) : 1024), 256, 0, st>>>(a, p, h);
    return cudaGetLastError();
}

cudaError_t launch_tb(const TBArgs &a, int grid, cudaStream_t st)
{
    if (a.n_work == 0) return cudaSuccess;
    tb_kernel<<<grid, 256, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_compact(const PairDesc *pairs, PairOut *out, uint32_t n, const uint32_t *ops, uint32_t *cig,
                           uint32_t *total, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    scan_kernel<<<1, 1024, 0, st>>>(out, n, total);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const uint32_t grid = (n + 7) / 8 < 4096 ? (n + 7) / 8 : 4096;
    copy_ops_kernel<<<grid, 256, 0, st>>>(pairs, out, n, ops, cig);
    return cudaGetLastError();
}

}  // namespace mpdp
