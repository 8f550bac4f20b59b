// Input packing, traceback and CIGAR compaction kernels.
//
// Traceback walks the direction codes written by the DP kernel from the best
// cell back to the restart, following the paths of Li 2022 Eq. 7 (Methods,
// "DP for protein-to-genome alignment"): M, I, D, the four frameshift terms
// and the three intron states, with the intron coordinates of the phase-1/2
// states as the paper places them (after Eq. 7).  One warp per pair: codons
// of an M run, gap runs and intron runs are scanned 32 cells at a time.
#include "mp_internal.cuh"

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

// ------------------------------------------------------------- traceback
struct CodeView {
    const uint8_t *base;
    size_t strip_bytes;

    // 16-bit code of the 1-based cell (i, j)
    __device__ __forceinline__ uint32_t at(int i, int j) const
    {
        const int ii = i - 1, jj = j - 1;
        const int s = jj >> 6, r = jj & 63, t = ii + r;
        const uint32_t w = __ldg(reinterpret_cast<const uint32_t *>(
            base + static_cast<size_t>(s) * strip_bytes + static_cast<size_t>(t >> 2) * 512 +
            (r >> 1) * 16 + (t & 3) * 4));
        // bytes of w: [lo bits 0-7, hi bits 0-7, lo bits 8-15, hi bits 8-15]
        const uint32_t v = w >> (8 * (r & 1));
        return (v & 0xffu) | ((v >> 8) & 0xff00u);
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

enum { ST_H = 0, ST_I, ST_D, ST_A, ST_B, ST_C };

__device__ void trace_pair(const TBArgs &a, uint32_t p, int lane)
{
    const PairDesc pd = a.pairs[p];
    PairOut &o = a.out[p];
    const int n = static_cast<int>(pd.nt_len);
    const int nchunks = (n + kStripW - 1 + kChunk - 1) / kChunk;
    const CodeView cv{a.codes + pd.code_off, static_cast<size_t>(nchunks) * kChunk * kStepBytes};
    int i = o.best_ii + 1, j = o.best_jj + 1;
    OpWriter w{a.ops + pd.cig_off, pd.cig_cap, 0, 0, 0, false};
    bool error = false;
    int state = ST_H, iexit = 0;
    for (;;) {
        if (state == ST_H) {
            if (i <= 0 || j <= 0) break;
            // codes along the codon diagonal: cells (i - 3k, j - k)
            const int ik = i - 3 * lane, jk = j - lane;
            const bool in = ik >= 1 && jk >= 1;
            const uint32_t c = in ? cv.at(ik, jk) : CB_STOP;
            const bool is_m = in && !(c & CB_STOP) && (c & CB_M);
            const unsigned nonm = __ballot_sync(kFull, !is_m);
            const int cnt = nonm ? __ffs(nonm) - 1 : 32;
            if (cnt > 0) {
                if (lane == 0) w.push(MP_OP_M, cnt);
                i -= 3 * cnt;
                j -= cnt;
            }
            if (cnt == 32) continue;
            const uint32_t cf = __shfl_sync(kFull, c, cnt);
            if (i <= 0 || j <= 0 || (cf & CB_STOP)) break;
            const uint32_t terms = cf & 0x7feu;
            if (!terms) { error = true; break; }
            const int src = __ffs(terms) - 1;   // 2 I, 3 D, 4 F1, 5 F2, 6 G1, 7 G2, 8 A, 9 B, 10 C
            switch (src) {
            case 2: state = ST_I; break;
            case 3: state = ST_D; break;
            case 4: if (lane == 0) w.push(MP_OP_F, 1); i -= 1; j -= 1; break;
            case 5: if (lane == 0) w.push(MP_OP_F, 2); i -= 2; j -= 1; break;
            case 6: if (lane == 0) w.push(MP_OP_G, 1); i -= 1; break;
            case 7: if (lane == 0) w.push(MP_OP_G, 2); i -= 2; break;
            case 8: state = ST_A; iexit = i; break;
            case 9: state = ST_B; iexit = i; break;
            case 10: state = ST_C; iexit = i; break;
            default: error = true; break;
            }
            if (error) break;
        } else {
            // a run: find the first cell (walking back) whose open flag is set
            uint32_t bit;
            int di, dj;
            switch (state) {
            case ST_I: bit = CB_IO; di = 0; dj = 1; break;
            case ST_D: bit = CB_DO; di = 3; dj = 0; break;
            case ST_A: bit = CB_AO; di = 1; dj = 0; break;
            case ST_B: bit = CB_BO; di = 1; dj = 0; break;
            default: bit = CB_CO; di = 1; dj = 0; break;
            }
            int k0 = 0, found = -1;
            for (;;) {
                const int ik = i - di * (k0 + lane), jk = j - dj * (k0 + lane);
                const bool in = ik >= 1 && jk >= 1;
                const bool open = in && (cv.at(ik, jk) & bit);
                const unsigned bal = __ballot_sync(kFull, open || !in);
                if (bal) {
                    const int f = __ffs(bal) - 1;
                    const bool f_in = __shfl_sync(kFull, in ? 1 : 0, f);
                    if (!f_in) error = true;
                    found = k0 + f;
                    break;
                }
                k0 += 32;
            }
            if (error) break;
            const int io = i - di * found, jo = j - dj * found;   // cell where the run opened
            switch (state) {
            case ST_I: if (lane == 0) w.push(MP_OP_I, found + 1); j = jo - 1; break;
            case ST_D: if (lane == 0) w.push(MP_OP_D, found + 1); i = io - 3; break;
            case ST_A: if (lane == 0) w.push(MP_OP_N, iexit - io + 1); i = io - 1; break;
            case ST_B:
            case ST_C: {
                const int L = iexit - io - 2;
                if (L < 1) error = true;
                if (lane == 0) w.push(state == ST_B ? MP_OP_U : MP_OP_V, L > 0 ? L : 0);
                i = io - 1;
                j = jo - 1;
                break;
            }
            }
            if (error) break;
            state = ST_H;
        }
    }
    if (lane == 0) {
        w.flush();
        o.n_ops = w.overflow ? 0 : w.n;
        o.st_ii = i > 0 ? i : 0;
        o.st_jj = j > 0 ? j : 0;
        if (error || w.overflow) o.status |= MP_ST_TRACE;
    }
}

__global__ void tb_kernel(const TBArgs a)
{
    const int lane = threadIdx.x & 31;
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t k = warp; k < a.n_work; k += nwarps) {
        const uint32_t p = a.work[k];
        const PairDesc &pd = a.pairs[p];
        const PairOut &o = a.out[p];
        if ((pd.flags & (PF_SCORE_ONLY | PF_SKIP | PF_BUDGET)) || (o.status & MP_ST_ERRMASK) || o.score <= 0)
            continue;
        trace_pair(a, p, lane);
    }
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

cudaError_t launch_pack(const PairDesc *pairs, uint32_t n, const char *ascii, uint8_t *prot, uint32_t *nt2,
                        PairOut *out, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    const uint32_t grid = n < 8192 ? n : 8192;
    pack_kernel<<<grid, 256, 0, st>>>(pairs, n, ascii, prot, nt2, out);
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
