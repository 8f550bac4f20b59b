// Measured integer ceilings for the DP kernel's roofline.
//
// The recurrence of Eq. 7 is a max-plus scan: it runs on the integer ALU,
// not on the tensor cores, and its traceback stream is far below the HBM
// bound.  The nominal ceiling is N_SM x 128 lanes x 2 int16 halves x f_SM
// simple operations per second; this file measures what this GPU actually
// sustains for the operations the int16 step is made of:
//
//   - the throughput of each packed 16-bit operation alone (warp
//     instructions per clock per SM, eight independent chains per thread,
//     every warp slot of every SM occupied);
//   - the throughput of the step's arithmetic itself: Eq. 7's eleven
//     penalised terms as fused add-max, the three-way maxima, the [H, I]
//     hand-over to the next lane by shuffle and byte permute, the chunk
//     maximum, on register state only (no shared-memory records, no stream
//     stores), at full occupancy.  Reported as cells per clock per SM.
//
// Clocks are counted on the SM (clock64) over each block's run, so the
// rates do not depend on the clock the GPU chose.
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "mp_dp.h"

namespace mpdp {
namespace {

constexpr int kThreads = 256;
constexpr int kChains = 8;

__device__ __forceinline__ uint32_t op_max(uint32_t a, uint32_t b)
{
    uint32_t r;
    asm volatile("max.u16x2 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
    return r;
}
__device__ __forceinline__ uint32_t op_prmt(uint32_t a, uint32_t b)
{
    uint32_t r;
    asm volatile("prmt.b32 %0, %1, %2, 0x5410;" : "=r"(r) : "r"(a), "r"(b));
    return r;
}
__device__ __forceinline__ uint32_t op_lop3(uint32_t a, uint32_t b, uint32_t c)
{
    uint32_t r;
    asm volatile("lop3.b32 %0, %1, %2, %3, 0xE8;" : "=r"(r) : "r"(a), "r"(b), "r"(c));
    return r;
}
__device__ __forceinline__ uint32_t op_imad(uint32_t a, uint32_t b, uint32_t c)
{
    uint32_t r;
    asm volatile("mad.lo.u32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(c));
    return r;
}

// OP: 0 max.u16x2, 1 fused add-max, 2 three-way max, 3 byte permute,
// 4 three-input logic, 5 integer multiply-add
template <int OP>
__global__ void __launch_bounds__(kThreads) op_rate_kernel(uint32_t seed, int iters, uint32_t *sink,
                                                           unsigned long long *cycles)
{
    uint32_t x[kChains], y[kChains];
#pragma unroll
    for (int u = 0; u < kChains; ++u) {
        x[u] = (seed ^ threadIdx.x) * (2u * u + 3u);
        y[u] = x[u] * 0x9e3779b9u + u;
    }
    __syncthreads();
    const long long c0 = clock64();
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int rep = 0; rep < 8; ++rep) {
#pragma unroll
            for (int u = 0; u < kChains; ++u) {
                if (OP == 0) x[u] = op_max(x[u], y[u]);
                if (OP == 1) x[u] = __viaddmax_u16x2(x[u], y[u], x[u]);
                if (OP == 2) x[u] = __vimax3_u16x2(x[u], y[u], seed);
                if (OP == 3) x[u] = op_prmt(x[u], y[u]);
                if (OP == 4) x[u] = op_lop3(x[u], y[u], seed);
                if (OP == 5) x[u] = op_imad(x[u], y[u], seed);
            }
        }
#pragma unroll
        for (int u = 0; u < kChains; ++u) y[u] += x[u];
    }
    __syncthreads();
    const long long c1 = clock64();
    uint32_t r = 0;
#pragma unroll
    for (int u = 0; u < kChains; ++u) r ^= x[u];
    sink[blockIdx.x * kThreads + threadIdx.x] = r;
    if (threadIdx.x == 0) cycles[blockIdx.x] = static_cast<unsigned long long>(c1 - c0);
}

// The int16 step's arithmetic on register state: every warp runs one
// 64-residue strip (two cells per lane, packed biased 16-bit halves) over
// `iters` anti-diagonal steps.  Penalties and substitution scores come from
// a small per-thread rotation of runtime values, so nothing folds.
__global__ void __launch_bounds__(kThreads) step_rate_kernel(const uint32_t *tab, int iters, uint32_t *sink,
                                                             unsigned long long *cycles)
{
    const int lane = threadIdx.x & 31;
    const uint32_t NQE = tab[0], E = tab[1], NF = tab[2], FLOOR = tab[3], BIN = tab[4];
    uint32_t rv[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) rv[k] = tab[8 + ((lane + k) & 7)];
    uint32_t H1 = tab[5], H2 = tab[5], H3 = tab[5], L0 = tab[5], L1 = tab[5], L2 = tab[5], L3 = tab[5];
    uint32_t IL = tab[6], D1 = tab[6], D2 = tab[6], D3 = tab[6], A1 = tab[6], B1 = tab[6], C1 = tab[6];
    uint32_t VD1 = rv[0], VD2 = rv[1], VA1 = rv[2], VA2 = rv[3], X1 = rv[0], cm = 0;
    __syncthreads();
    const long long c0 = clock64();
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const uint32_t VD0 = rv[k], VA0 = rv[(k + 1) & 3], X0 = rv[(k + 2) & 3];
            const uint32_t S = (X0 & 0x0000ffffu) | (X1 & 0xffff0000u);
            const uint32_t I0 = __viaddmax_u16x2(L0, NQE, IL - E);
            const uint32_t D0 = __viaddmax_u16x2(H3, NQE, D3 - E);
            const uint32_t A0 = __viaddmax_u16x2(H1, VD2, A1);
            const uint32_t B0 = __viaddmax_u16x2(L1, VD1, B1);
            const uint32_t C0 = __viaddmax_u16x2(L1, VD0, C1);
            uint32_t Y = __viaddmax_u16x2(H2, NF, FLOOR);
            Y = __viaddmax_u16x2(__vimax3_u16x2(L1, L2, H1), NF, Y);
            Y = __viaddmax_u16x2(C0, VA1, Y);
            Y = __viaddmax_u16x2(B0, VA2, Y);
            Y = __viaddmax_u16x2(A0, VA0, Y);
            const uint32_t H0 = __vimax3_u16x2(__viaddmax_u16x2(L3, S, I0), D0, Y);
            const uint32_t Wd = __byte_perm(H0, I0, 0x7632);
            uint32_t R = __shfl_up_sync(0xffffffffu, Wd, 1);
            if (lane == 0) R = BIN;
            L3 = L2; L2 = L1; L1 = L0;
            L0 = __byte_perm(R, H0, 0x5410);
            IL = __byte_perm(R, I0, 0x5432);
            H3 = H2; H2 = H1; H1 = H0;
            D3 = D2; D2 = D1; D1 = D0;
            A1 = A0; B1 = B0; C1 = C0;
            VD2 = VD1; VD1 = VD0;
            VA2 = VA1; VA1 = VA0;
            X1 = X0;
            cm = op_max(cm, H0);
        }
    }
    __syncthreads();
    const long long c1 = clock64();
    sink[blockIdx.x * kThreads + threadIdx.x] = cm ^ H1 ^ IL;
    if (threadIdx.x == 0) cycles[blockIdx.x] = static_cast<unsigned long long>(c1 - c0);
}

// Longest block run, in SM clocks: every block of a launch runs at once
// (blocks = SMs x resident blocks per SM), so this is the launch's span.
template <typename F>
int timed(F launch, int nblocks, unsigned long long *d_cycles, double *span)
{
    launch();
    if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) return MP_ECUDA;
    std::vector<unsigned long long> c(nblocks);
    if (cudaMemcpy(c.data(), d_cycles, nblocks * sizeof(unsigned long long), cudaMemcpyDeviceToHost) !=
        cudaSuccess)
        return MP_ECUDA;
    unsigned long long mx = 0;
    for (unsigned long long v : c) mx = v > mx ? v : mx;
    *span = static_cast<double>(mx);
    return MP_OK;
}

}  // namespace
}  // namespace mpdp

extern "C" int mp_dp_op_rates(int device, mp_op_rates *out)
{
    using namespace mpdp;
    if (!out) return MP_EINVAL;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return MP_EINVAL;
    int prev = 0;
    cudaGetDevice(&prev);
    if (cudaSetDevice(device) != cudaSuccess) return MP_ECUDA;
    int nsm = 0, per_sm_op = 0, per_sm_step = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_op, op_rate_kernel<1>, kThreads, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_step, step_rate_kernel, kThreads, 0);
    const int nb_op = nsm * (per_sm_op > 0 ? per_sm_op : 1);
    const int nb_step = nsm * (per_sm_step > 0 ? per_sm_step : 1);
    const int nb = nb_op > nb_step ? nb_op : nb_step;
    uint32_t *sink = nullptr, *tab = nullptr;
    unsigned long long *cyc = nullptr;
    int rc = MP_OK;
    if (cudaMalloc(&sink, static_cast<size_t>(nb) * kThreads * sizeof(uint32_t)) != cudaSuccess ||
        cudaMalloc(&cyc, static_cast<size_t>(nb) * sizeof(unsigned long long)) != cudaSuccess ||
        cudaMalloc(&tab, 16 * sizeof(uint32_t)) != cudaSuccess) {
        rc = MP_ENOMEM;
    }
    if (rc == MP_OK) {
        // biased int16 pairs: -(q+e) = -12, e = 1, -f = -23 negated per half,
        // local floor (biased 0), a boundary word, start values, penalties
        auto neg2 = [](uint32_t v) { return ((0x10000u - v) & 0xffffu) * 0x10001u; };
        uint32_t h[16] = {neg2(12), 0x00010001u, neg2(23), 0x80008000u, 0x40008000u, 0x80008000u, 0x40004000u,
                          0, neg2(29), neg2(37), neg2(44), neg2(50), neg2(29), neg2(59), neg2(37), neg2(29)};
        if (cudaMemcpy(tab, h, sizeof(h), cudaMemcpyHostToDevice) != cudaSuccess) rc = MP_ECUDA;
    }
    const int op_iters = 4096, step_iters = 8192;
    double span = 0;
    double *fields[6] = {&out->max_u16x2, &out->viaddmax_u16x2, &out->vimax3_u16x2, &out->prmt, &out->lop3,
                         &out->imad};
    // warp instructions of the timed operation per block
    const double op_insts = static_cast<double>(kThreads / 32) * op_iters * 8 * kChains;
    for (int op = 0; op < 6 && rc == MP_OK; ++op) {
        auto launch = [&]() {
            switch (op) {
            case 0: op_rate_kernel<0><<<nb_op, kThreads>>>(7u, op_iters, sink, cyc); break;
            case 1: op_rate_kernel<1><<<nb_op, kThreads>>>(7u, op_iters, sink, cyc); break;
            case 2: op_rate_kernel<2><<<nb_op, kThreads>>>(7u, op_iters, sink, cyc); break;
            case 3: op_rate_kernel<3><<<nb_op, kThreads>>>(7u, op_iters, sink, cyc); break;
            case 4: op_rate_kernel<4><<<nb_op, kThreads>>>(7u, op_iters, sink, cyc); break;
            default: op_rate_kernel<5><<<nb_op, kThreads>>>(7u, op_iters, sink, cyc); break;
            }
        };
        rc = timed(launch, nb_op, cyc, &span);          // warm-up
        if (rc == MP_OK) rc = timed(launch, nb_op, cyc, &span);
        if (rc == MP_OK) *fields[op] = op_insts * (nb_op / static_cast<double>(nsm)) / span;
    }
    if (rc == MP_OK) {
        auto launch = [&]() { step_rate_kernel<<<nb_step, kThreads>>>(tab, step_iters, sink, cyc); };
        rc = timed(launch, nb_step, cyc, &span);
        if (rc == MP_OK) rc = timed(launch, nb_step, cyc, &span);
        // 64 cells per warp and step
        if (rc == MP_OK)
            out->step_cells_per_clk_sm =
                static_cast<double>(kThreads / 32) * step_iters * 4 * 64 * (nb_step / static_cast<double>(nsm)) / span;
        out->warps_per_sm_step = per_sm_step * (kThreads / 32);
    }
    if (sink) cudaFree(sink);
    if (cyc) cudaFree(cyc);
    if (tab) cudaFree(tab);
    cudaSetDevice(prev);
    return rc;
}
