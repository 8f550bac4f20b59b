// Host runtime of the spliced-DP library: contexts, batch planning into
// traceback-budgeted waves, the device pipeline (captured once per batch as
// a CUDA graph and replayed), result download, and the serving loop.
#include <algorithm>
#include <cstdint>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <functional>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <set>
#include <string>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "mp_internal.cuh"

using namespace mpdp;

namespace {

// ------------------------------------------------------------ defaults
// BLOSUM62 (Henikoff & Henikoff 1992) in ARNDCQEGHILKMFPSTWYV order.
const int8_t kBlosum62[20][20] = {
    {4, -1, -2, -2, 0, -1, -1, 0, -2, -1, -1, -1, -1, -2, -1, 1, 0, -3, -2, 0},
    {-1, 5, 0, -2, -3, 1, 0, -2, 0, -3, -2, 2, -1, -3, -2, -1, -1, -3, -2, -3},
    {-2, 0, 6, 1, -3, 0, 0, 0, 1, -3, -3, 0, -2, -3, -2, 1, 0, -4, -2, -3},
    {-2, -2, 1, 6, -3, 0, 2, -1, -1, -3, -4, -1, -3, -3, -1, 0, -1, -4, -3, -3},
    {0, -3, -3, -3, 9, -3, -4, -3, -3, -1, -1, -3, -1, -2, -3, -1, -1, -2, -2, -1},
    {-1, 1, 0, 0, -3, 5, 2, -2, 0, -3, -2, 1, 0, -3, -1, 0, -1, -2, -1, -2},
    {-1, 0, 0, 2, -4, 2, 5, -2, 0, -3, -3, 1, -2, -3, -1, 0, -1, -3, -2, -2},
    {0, -2, 0, -1, -3, -2, -2, 6, -2, -4, -4, -2, -3, -3, -2, 0, -2, -2, -3, -3},
    {-2, 0, 1, -1, -3, 0, 0, -2, 8, -3, -3, -1, -2, -1, -2, -1, -2, -2, 2, -3},
    {-1, -3, -3, -3, -1, -3, -3, -4, -3, 4, 2, -3, 1, 0, -3, -2, -1, -3, -1, 3},
    {-1, -2, -3, -4, -1, -2, -3, -4, -3, 2, 4, -2, 2, 0, -3, -2, -1, -2, -1, 1},
    {-1, 2, 0, -1, -3, 1, 1, -2, -1, -3, -2, 5, -1, -3, -1, 0, -1, -3, -2, -2},
    {-1, -1, -2, -3, -1, 0, -2, -3, -2, 1, 2, -1, 5, 0, -2, -1, -1, -1, -1, 1},
    {-2, -3, -3, -3, -2, -3, -3, -3, -1, 0, 0, -3, 0, 6, -4, -2, -2, 1, 3, -1},
    {-1, -2, -2, -1, -3, -1, -1, -2, -2, -3, -3, -1, -2, -4, 7, -1, -1, -4, -3, -2},
    {1, -1, 1, 0, -1, 0, 0, 0, -1, -2, -2, 0, -1, -2, -1, 4, 1, -3, -2, -2},
    {0, -1, 0, -1, -1, -1, -1, -2, -2, -1, -1, -1, -1, -2, -1, 1, 5, -2, -2, 0},
    {-3, -3, -4, -4, -2, -2, -3, -2, -2, -3, -2, -3, -1, 1, -4, -3, -2, 11, 2, -3},
    {-2, -2, -2, -3, -2, -1, -2, -3, 2, -1, -1, -2, -1, 3, -3, -2, -2, 2, 7, -1},
    {0, -3, -3, -3, -1, -2, -2, -3, -3, 3, 1, -2, 1, -1, -2, -2, 0, -3, -1, 4},
};

constexpr uint64_t kDefaultBudget = 40ull << 30;

inline uint64_t div_up(uint64_t a, uint64_t b) { return (a + b - 1) / b; }

// Traceback bytes of one pair: strips x padded steps x 2 B per cell plus the
// column maxima (2 B per cell and chunk) of every strip and chunk (x 2 when
// the pair may need the int32 re-run, whose stream holds 4 B per cell);
// w128: 128-residue strips.
inline uint64_t code_bytes(uint32_t m, uint32_t n, bool wide = false, bool w128 = false)
{
    const uint64_t W = w128 ? kStripWMax : kStripW;
    const uint64_t nchunks = div_up(static_cast<uint64_t>(n) + W - 1, kChunk);
    const uint64_t strips = div_up(m, W);
    // H stream, then the per-chunk column maxima
    return strips * nchunks * (kChunk * W * 2 + W * 2) * (wide ? 2 : 1);
}

// Whether a pair runs in 128-residue strips when the configuration asks for
// them: only int16 pairs (never PF_WIDE), and only where the wider strips do
// not add much padding (an odd number of 64-residue strips would pad one
// more 64-residue half strip).
inline bool use_w128(const PairDesc &d)
{
    if (d.flags & (PF_WIDE | PF_SKIP | PF_PROF)) return false;
    const uint64_t k64 = div_up(d.prot_len, kStripW);
    return k64 % 2 == 0 || k64 >= 9;
}

// Residue letter -> code (ARNDCQEGHILKMFPSTWYV 0..19, '*' 20, else X 21).
struct AACodeTable {
    uint8_t v[256];
    AACodeTable()
    {
        static const char order[] = "ARNDCQEGHILKMFPSTWYV";
        for (int c = 0; c < 256; ++c) v[c] = 21;
        for (int k = 0; k < 20; ++k) {
            v[static_cast<unsigned char>(order[k])] = static_cast<uint8_t>(k);
            v[static_cast<unsigned char>(order[k] | 0x20)] = static_cast<uint8_t>(k);
        }
        v[static_cast<unsigned char>('*')] = 20;
    }
};
const AACodeTable kAACode;

inline int host_aa_code(unsigned char c) { return kAACode.v[c]; }

// Upper bound of any H of the pair: every residue scores at most its best
// substitution and every other term of Eq. 7 is a penalty.
// Per residue code, the best score any codon can earn against it (at least
// 0), and the largest of these: the table behind score_bound.
struct BoundTable {
    int best[22];
    int top;
    explicit BoundTable(const ScoreParams &sp)
    {
        top = 0;
        for (int pc = 0; pc < 22; ++pc) {
            int b = -sp.stop;
            for (int t = 0; t < 20; ++t) b = std::max<int>(b, sp.mat[t][pc]);
            best[pc] = std::max(b, 0);
            top = std::max(top, best[pc]);
        }
    }
};

// An upper bound of the pair's local score: the sum over residues of their
// best codon score.  Proteins too short to reach `limit` even at the
// largest per-residue score are not scanned (the returned bound is then
// m * top, below the limit).
inline int64_t score_bound(const BoundTable &bt, const char *prot, uint32_t m, int64_t limit)
{
    if (static_cast<int64_t>(m) * bt.top < limit) return static_cast<int64_t>(m) * bt.top;
    int64_t s = 0;
    for (uint32_t k = 0; k < m; ++k) s += bt.best[host_aa_code(static_cast<unsigned char>(prot[k]))];
    return s;
}

// boundary entries of a pair (for either strip form)
inline uint64_t bnd_entries(uint32_t n)
{
    const uint64_t nchunks = div_up(static_cast<uint64_t>(n) + kStripWMax - 1, kChunk);
    return nchunks * kChunk + 2 * kBndPad + 32;
}

#define CK(x)                                                                         \
    do {                                                                              \
        cudaError_t e_ = (x);                                                         \
        if (e_ != cudaSuccess) {                                                      \
            if (getenv("MP_DP_DEBUG"))                                                \
                fprintf(stderr, "mp_dp: %s failed: %s\n", #x, cudaGetErrorString(e_)); \
            return MP_ECUDA;                                                          \
        }                                                                             \
    } while (0)

template <typename T>
struct DevBuf {
    T *p = nullptr;
    size_t cap = 0;   // elements
    cudaError_t reserve(size_t n)
    {
        if (n <= cap) return cudaSuccess;
        if (p) cudaFree(p);
        p = nullptr;
        cap = 0;
        cudaError_t e = cudaMalloc(&p, std::max<size_t>(n, 1) * sizeof(T));
        if (e == cudaSuccess) cap = n;
        return e;
    }
    void release()
    {
        if (p) cudaFree(p);
        p = nullptr;
        cap = 0;
    }
};

template <typename T>
struct HostBuf {
    T *p = nullptr;
    size_t cap = 0;
    cudaError_t reserve(size_t n)
    {
        if (n <= cap) return cudaSuccess;
        if (p) cudaFreeHost(p);
        p = nullptr;
        cap = 0;
        cudaError_t e = cudaMallocHost(&p, std::max<size_t>(n, 1) * sizeof(T));
        if (e == cudaSuccess) cap = n;
        return e;
    }
    void release()
    {
        if (p) cudaFreeHost(p);
        p = nullptr;
        cap = 0;
    }
};

struct Wave {
    uint32_t begin, end;    // range of the pair order
    uint32_t ibegin, iend;  // range of the strip-item order
    uint64_t code_bytes;
    uint32_t nwide_items;   // items of PF_WIDE pairs, first in the wave's range
};

// timing events: [0] start, [1] after packing; per wave [start, DP, re-run,
// traceback]; then [before compaction, end]
enum { EV_PER_WAVE = 4 };

}  // namespace

struct mp_dp_batch {
    size_t n = 0;
    std::vector<PairDesc> desc;
    std::vector<uint32_t> order;
    std::vector<Wave> waves;
    std::vector<uint32_t> nt_len;
    std::vector<int8_t> strand;
    uint64_t ascii_bytes = 0, prot_total = 0, nt_words = 0, bnd_total = 0, ops_total = 0;
    double cells = 0;
    uint64_t code_bytes_total = 0;
    // bytes moved by construction (planned, per run): records written and
    // read by the strips, boundary rows handed between strips
    uint64_t record_bytes_total = 0, record_read_total = 0, bnd_bytes_total = 0;
    // device
    DevBuf<char> ascii;
    DevBuf<PairDesc> d_desc;
    DevBuf<uint8_t> prot;
    DevBuf<uint32_t> nt2;
    DevBuf<PairOut> out;
    DevBuf<uint32_t> ops, cig, work;
    DevBuf<uint2> items, rerun_items;   // strip items in processing order; re-run list
    DevBuf<uint4> recs;                 // per-nt records of every pair
    DevBuf<int32_t> col0;               // anchored modes: column 0 of every pair
    DevBuf<ProfPos> prof;               // profile queries: positions 0..|P| of each
    DevBuf<int32_t> epre;               // and their gap-extension prefix sums
    std::vector<ProfPos> h_prof;
    std::vector<int32_t> h_epre;
    DevBuf<uint64_t> bnd;
    // per-run state, zeroed by one memset: counters | strips_done | progress | best_key
    DevBuf<unsigned long long> state;
    size_t state_bytes = 0, off_done = 0, off_progress = 0, off_key = 0;
    std::vector<uint2> h_items;
    std::vector<uint32_t> item_off;     // first item of each pair in the order (by order index)
    DevBuf<uint32_t> wave_nwide;        // Wave::nwide_items of each wave, on the device
    uint64_t shape_key = 0;             // shape class for the tuned table
    bool overlap = false;               // waves alternate between two streams and two arena halves
    uint64_t arena_half = 0;            // bytes of one arena half (overlap only)
    bool needs_waves = false;           // the traceback bytes exceed the budget
    int planned = -1;                   // plan_key() the current plan was made for, -1 before planning
    uint64_t strips_total = 0;
    cudaGraphExec_t graph = nullptr;
    uint64_t graph_sig = 0;             // timing flag and configuration the graph was captured with
    int runs = 0;
    std::vector<cudaEvent_t> events;
    // host results
    std::vector<PairOut> h_out;
    std::vector<uint32_t> h_cig;
    int n_launches = 0, n_dp_launches = 0;
};

struct Request {
    uint64_t ticket;
    std::string prot, nt;
    int8_t strand;
    uint32_t flags;
    std::vector<mp_profile_pos> profile;    // a profile query's positions (empty otherwise)
    std::chrono::steady_clock::time_point t_submit;
};

struct Done {
    mp_result r;
    std::vector<uint32_t> cigar;
    bool delivered = false;
};

struct Slot;

// A few host threads kept for the life of a context, so that gathering a
// large batch's sequences does not start threads on every call.  run()
// hands out job indices 0..n-1 to the workers and returns at once; wait()
// returns when every job has finished.
struct WorkerPool {
    std::vector<std::thread> th;
    std::mutex mu;
    std::condition_variable cv, done_cv;
    std::function<void(unsigned)> job;
    unsigned njobs = 0, next = 0, finished = 0;
    uint64_t gen = 0;
    bool stop = false;

    void start(unsigned n)
    {
        for (unsigned k = 0; k < n; ++k) th.emplace_back([this] { loop(); });
    }
    void loop()
    {
        uint64_t seen = 0;
        std::unique_lock<std::mutex> lk(mu);
        for (;;) {
            cv.wait(lk, [&] { return stop || gen != seen; });
            if (stop) return;
            seen = gen;
            while (next < njobs) {
                const unsigned i = next++;
                lk.unlock();
                job(i);
                lk.lock();
                if (++finished == njobs) done_cv.notify_all();
            }
        }
    }
    void run(unsigned n, std::function<void(unsigned)> f)
    {
        std::lock_guard<std::mutex> lk(mu);
        job = std::move(f);
        njobs = n;
        next = 0;
        finished = 0;
        ++gen;
        cv.notify_all();
    }
    void wait()
    {
        std::unique_lock<std::mutex> lk(mu);
        done_cv.wait(lk, [&] { return finished == njobs; });
    }
    ~WorkerPool()
    {
        {
            std::lock_guard<std::mutex> lk(mu);
            stop = true;
        }
        cv.notify_all();
        for (auto &t : th) t.join();
    }
};

struct mp_dp_ctx {
    int device = 0;
    int num_sms = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t stream2 = nullptr;     // second stream: odd waves of an overlapped batch
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    cudaEvent_t ev_staging = nullptr;   // recorded after the last copy out of the staging buffer
    bool staging_busy = false;          // ev_staging is pending
    mp_dp_params params{};
    ScoreParams sp{};
    uint64_t budget = 0;
    DevBuf<uint8_t> codes;      // traceback arena (shared by the waves of a batch)
    // serving slots: a range of the serving loop's shared arena used instead
    // of `codes` (null: the context's own arena)
    uint8_t *codes_ext = nullptr;
    uint64_t codes_ext_cap = 0;
    HostBuf<char> staging;
    HostBuf<char> pstaging;        // a plan's descriptors, order, items and wave counts on their way to the device
    std::unique_ptr<WorkerPool> pool;  // gather threads (started by the first large upload)
    bool timing = false;
    mp_dp_stats stats{};
    mp_dp_batch *last = nullptr;   // batch of the last run (for its counters)
    mp_dp_batch *own = nullptr;    // buffers reused by mp_dp_align_batch from call to call
    mp_dp_batch *aux = nullptr;    // score-only batch of mp_dp_exon_rescore
    DevBuf<uint8_t> exbuf;         // rescoring jobs (and, for earlier results, their regions and ops)
    DevBuf<int8_t> d_mat;          // the substitution matrix for the DP kernel's own tracebacks
    std::vector<uint32_t> host_cig;
    // launch configuration: fixed by mp_dp_set_tuning, else tuned per shape class
    bool has_fixed = false;
    mp_dp_tuning fixed{};
    std::map<uint64_t, mp_dp_tuning> tuned;
    std::string dev_name;

    // serving
    std::mutex mu;
    std::condition_variable cv_req, cv_done;
    std::deque<Request> queue;
    std::unordered_map<uint64_t, Done> done;
    std::unordered_set<uint64_t> inflight;
    std::deque<uint64_t> completed;       // completion order, for mp_dp_wait_any
    std::atomic<uint64_t> next_ticket{1};
    std::thread server;
    bool server_running = false, stopping = false;
    size_t ring_cap = 1 << 20;
    int n_slots = 3;                      // micro-batches in flight on the device
    uint64_t slot_budget = 0;
    uint64_t served_batches = 0, served_pairs = 0;
    std::vector<float> latencies_ms;      // submit -> result available, per completed request
};

namespace mpdp {
int ctx_device(const mp_dp_ctx *c) { return c->device; }
cudaStream_t ctx_stream(const mp_dp_ctx *c) { return c->stream; }
}  // namespace mpdp

// ====================================================================== API
extern "C" {

void mp_dp_default_params(mp_dp_params *p)
{
    if (!p) return;
    memset(p, 0, sizeof(*p));
    p->q = 11; p->e = 1; p->f = 23; p->r = 29; p->stop = 23;
    for (int a = 0; a < 22; ++a)
        for (int b = 0; b < 22; ++b) p->mat[a][b] = -1;        // X against anything
    for (int a = 0; a < 20; ++a) {
        for (int b = 0; b < 20; ++b) p->mat[a][b] = kBlosum62[a][b];
        p->mat[a][20] = -4;                                    // BLOSUM62 stop column
        p->mat[20][a] = -4;
    }
    p->mat[20][20] = 1;
    p->splice_model = MP_SPLICE_FINAL;
    p->splice_p = 30;
    p->mode = MP_MODE_LOCAL;
    p->tb_budget_bytes = kDefaultBudget;
}

const char *mp_dp_strerror(int code)
{
    switch (code) {
    case MP_OK: return "ok";
    case MP_EINVAL: return "invalid argument";
    case MP_ENOMEM: return "out of memory";
    case MP_EBUDGET: return "request exceeds the traceback budget";
    case MP_ETIMEOUT: return "timed out";
    case MP_ECUDA: return "CUDA error";
    case MP_EPENDING: return "result pending";
    case MP_EAGAIN: return "request ring full";
    case MP_ETICKET: return "unknown ticket";
    case MP_ESTATE: return "invalid state";
    case MP_ETOOLARGE: return "input exceeds the fixed scratch of the allocation-free entry point";
    default: return "unknown error";
    }
}

static int validate_params(const mp_dp_params *p)
{
    if (p->q < 0 || p->e < 1 || p->f < 0 || p->r < 0 || p->stop < 0) return MP_EINVAL;
    if (p->q + p->e > 1000 || p->f > 1000 || p->r > 1000 || p->stop > 512) return MP_EINVAL;
    int mn = 0;
    for (int a = 0; a < 20; ++a)
        for (int b = 0; b < 22; ++b) mn = std::min<int>(mn, p->mat[a][b]);
    // an intron of length <= 0 must lose to a frameshift or a match from the same cell
    if (!(p->r > p->f && p->r > p->stop && p->r > -mn)) return MP_EINVAL;
    if ((p->splice_model != MP_SPLICE_FINAL && p->splice_model != MP_SPLICE_SIMPLE) ||
        (p->mode != MP_MODE_LOCAL && p->mode != MP_MODE_GLOBAL && p->mode != MP_MODE_EXTEND))
        return MP_EINVAL;
    if (p->splice_p < 0 || p->splice_p > 1000) return MP_EINVAL;
    if (p->max_pairs_per_launch < 0 || p->wait_limit < 0) return MP_EINVAL;
    return MP_OK;
}

int mp_dp_init(mp_dp_ctx **out, const mp_dp_params *p, int device)
{
    if (!out) return MP_EINVAL;
    *out = nullptr;
    mp_dp_params prm;
    if (p) prm = *p;
    else mp_dp_default_params(&prm);
    if (validate_params(&prm) != MP_OK) return MP_EINVAL;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return MP_ECUDA;
    mp_dp_ctx *c = new (std::nothrow) mp_dp_ctx();
    if (!c) return MP_ENOMEM;
    c->device = device;
    c->params = prm;
    if (cudaSetDevice(device) != cudaSuccess) { delete c; return MP_ECUDA; }
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) { delete c; return MP_ECUDA; }
    c->num_sms = prop.multiProcessorCount;
    c->dev_name = prop.name;
    for (char &ch : c->dev_name)
        if (ch == ' ' || ch == '\t') ch = '_';
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) { delete c; return MP_ECUDA; }
    if (cudaStreamCreateWithFlags(&c->stream2, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_staging, cudaEventDisableTiming) != cudaSuccess) {
        mp_dp_destroy(c);
        return MP_ECUDA;
    }
    c->sp.q = prm.q; c->sp.e = prm.e; c->sp.f = prm.f; c->sp.r = prm.r; c->sp.stop = prm.stop;
    memcpy(c->sp.mat, prm.mat, sizeof(c->sp.mat));
    c->sp.splice_model = prm.splice_model;
    c->sp.splice_p = prm.splice_p;
    c->sp.mode = prm.mode;
    if (c->d_mat.reserve(sizeof(c->sp.mat)) != cudaSuccess ||
        cudaMemcpy(c->d_mat.p, c->sp.mat, sizeof(c->sp.mat), cudaMemcpyHostToDevice) != cudaSuccess) {
        mp_dp_destroy(c);
        return MP_ECUDA;
    }
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    uint64_t budget = prm.tb_budget_bytes ? prm.tb_budget_bytes : kDefaultBudget;
    budget = std::min<uint64_t>(budget, static_cast<uint64_t>(free_b * 0.6));
    c->budget = budget;
    *out = c;
    return MP_OK;
}

int mp_dp_num_sms(mp_dp_ctx *c) { return c ? c->num_sms : 0; }

int mp_dp_debug_h(mp_dp_ctx *c, mp_dp_batch *b, size_t k, int32_t *h)
{
    if (!c || !b || !h || k >= b->n) return MP_EINVAL;
    const PairDesc &d = b->desc[k];
    if (d.flags & (PF_SCORE_ONLY | PF_SKIP | PF_BUDGET)) return MP_EINVAL;      // no stream kept
    // the arena holds the stream of the context's last run, whole only in one wave
    if (c->last != b || b->waves.size() != 1) return MP_ESTATE;
    if (cudaSetDevice(c->device) != cudaSuccess) return MP_ECUDA;
    CK(cudaStreamSynchronize(c->stream));
    const size_t cells = (static_cast<size_t>(d.nt_len) + 1) * (static_cast<size_t>(d.prot_len) + 1);
    DevBuf<int32_t> tmp;
    if (tmp.reserve(cells) != cudaSuccess) return MP_ENOMEM;
    TBArgs t{};
    t.pairs = b->d_desc.p;
    t.codes = c->codes_ext ? c->codes_ext : c->codes.p;
    t.prot = b->prot.p;
    t.nt2 = b->nt2.p;
    t.out = b->out.p;
    t.col0 = c->params.mode != MP_MODE_LOCAL ? b->col0.p : nullptr;
    t.sp = c->sp;
    t.prof = b->prof.p;
    t.epre = b->epre.p;
    cudaError_t e = launch_dump_h(t, static_cast<uint32_t>(k), cells, tmp.p, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h, tmp.p, cells * sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    tmp.release();
    return e == cudaSuccess ? MP_OK : MP_ECUDA;
}

int mp_dp_set_timing(mp_dp_ctx *c, int enable)
{
    if (!c) return MP_EINVAL;
    c->timing = enable != 0;
    return MP_OK;
}

int mp_dp_get_stats(mp_dp_ctx *c, mp_dp_stats *s)
{
    if (!c || !s) return MP_EINVAL;
    *s = c->stats;
    return MP_OK;
}

static void free_batch_device(mp_dp_batch *b)
{
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
    for (cudaEvent_t e : b->events) cudaEventDestroy(e);
    b->events.clear();
    b->ascii.release(); b->d_desc.release(); b->prot.release(); b->nt2.release(); b->out.release();
    b->ops.release(); b->cig.release(); b->work.release(); b->items.release(); b->rerun_items.release();
    b->bnd.release(); b->state.release(); b->recs.release(); b->wave_nwide.release(); b->col0.release();
    b->prof.release(); b->epre.release();
}

void mp_dp_batch_free(mp_dp_ctx *c, mp_dp_batch *b)
{
    if (!b) return;
    if (c) cudaSetDevice(c->device);
    free_batch_device(b);
    delete b;
}

// index of the compacted-CIGAR length among the state counters (after the
// 8 counters of every wave)
static size_t cig_total_index(const mp_dp_batch *b) { return 8 * b->waves.size(); }

static uint32_t log2_bucket(double v)
{
    uint32_t k = 0;
    while (v >= 2.0 && k < 63) { v *= 0.5; ++k; }
    return k;
}

// Shape class of a planned batch: pair count, mean cells per pair, the
// longest critical path (chunks of the region plus the lag of its strips)
// on log2 scales, whether some pair needs int32, and whether the batch needs
// several waves.  Batches of one class take the same tuned configuration.
static uint64_t shape_key_of(const mp_dp_batch &b)
{
    double crit = 0;
    uint32_t any_wide = 0;
    for (const PairDesc &d : b.desc) {
        if (d.flags & PF_SKIP) continue;
        crit = std::max(crit, static_cast<double>(d.nt_len) / kChunk + 2.0 * d.n_strips);
        if (d.flags & PF_WIDE) any_wide = 1;
    }
    const uint64_t nb = log2_bucket(static_cast<double>(b.n) + 1);
    const uint64_t cb = log2_bucket(b.n ? b.cells / b.n + 1 : 1);
    const uint64_t kb = log2_bucket(crit + 1);
    const uint64_t wb = b.needs_waves ? 1 : 0;
    return nb | (cb << 8) | (kb << 16) | (static_cast<uint64_t>(any_wide) << 24) | (wb << 28);
}

static mp_dp_tuning default_tuning()
{
    mp_dp_tuning t{};
    t.dp16_variant = 1;
    t.overlap_waves = 1;
    t.item_order = 1;
    // int16 kernel built for 2 CTAs/SM (no spill; with the tracebacks in the
    // kernel it is the faster build on the 4,096-pair workload), all CTAs that
    // fit, int16 first for wide pairs, overlapped waves, interleaved items
    return t;
}

static mp_dp_tuning tuning_for(const mp_dp_ctx *c, const mp_dp_batch *b)
{
    if (c->has_fixed) return c->fixed;
    auto it = c->tuned.find(b->shape_key);
    return it != c->tuned.end() ? it->second : default_tuning();
}

// What a plan depends on in a configuration: the wave policy (only for a
// batch that needs several waves) and the item order.
static int plan_key(const mp_dp_batch *b, const mp_dp_tuning &t)
{
    return (b->needs_waves && t.overlap_waves ? 1 : 0) | (t.item_order ? 2 : 0) | (t.strip_width << 2);
}

static int plan_waves(mp_dp_ctx *c, mp_dp_batch *b, const mp_dp_tuning &t, bool stream_idle = false);

// Re-plan the batch if its plan was made for another configuration.
static int ensure_plan(mp_dp_ctx *c, mp_dp_batch *b, const mp_dp_tuning &t)
{
    return b->planned == plan_key(b, t) ? MP_OK : plan_waves(c, b, t);
}

// Traceback bytes of the batch's pairs that keep a stream (pairs larger than
// the whole budget are scored without one).
static uint64_t plan_code_bytes(const mp_dp_ctx *c, const mp_dp_batch *b)
{
    uint64_t total = 0;
    for (const PairDesc &d : b->desc) {
        if (d.flags & (PF_SKIP | PF_SCORE_ONLY)) continue;
        const uint64_t cb = div_up(code_bytes(d.prot_len, d.nt_len, (d.flags & PF_WIDE) != 0), 256) * 256;
        if (cb <= c->budget) total += cb;
    }
    return total;
}

// Order each wave's strip items so that a warp rarely takes a strip whose
// predecessor has not yet published the boundary rows it starts with: pairs
// in order (largest first), strip s+1 of a pair placed after strip s by
// about as many items as the warps pop while the predecessor runs kLag = 2
// chunks (the strips of a pair still run close together, so its per-nt
// records and boundary rows are read from L2).  PF_WIDE pairs' items stay a
// prefix of the wave (the int32 queue may take them as a block).
static void interleave_items(const mp_dp_ctx *c, mp_dp_batch *b)
{
    const double warps = static_cast<double>(c->num_sms) * 2 * kWarpsPerCta;
    std::vector<uint32_t> key, count;
    std::vector<uint2> out;
    auto segment = [&](uint32_t lo, uint32_t hi) {
        if (hi - lo < 2) return;
        double chunks = 0;
        for (uint32_t k = lo; k < hi; ++k)
        {
            const PairDesc &d = b->desc[b->h_items[k].x];
            chunks += static_cast<double>((d.nt_len + strip_w_of(d.flags) - 1 + kChunk - 1) / kChunk);
        }
        const uint32_t D = static_cast<uint32_t>(std::max(1.0, std::round(2.0 * warps / (chunks / (hi - lo)))));
        // key = rank of the pair + D * strip; a stable counting sort by key
        key.resize(hi - lo);
        uint32_t rank = 0, top = 0;
        for (uint32_t k = lo; k < hi; ++k) {
            const uint2 it = b->h_items[k];
            if (k > lo && it.x != b->h_items[k - 1].x) ++rank;
            key[k - lo] = rank + it.y * D;
            top = std::max(top, key[k - lo]);
        }
        count.assign(static_cast<size_t>(top) + 2, 0);
        for (uint32_t k = 0; k < hi - lo; ++k) ++count[key[k] + 1];
        for (size_t v = 1; v < count.size(); ++v) count[v] += count[v - 1];
        out.resize(hi - lo);
        for (uint32_t k = 0; k < hi - lo; ++k) out[count[key[k]]++] = b->h_items[lo + k];
        std::copy(out.begin(), out.end(), b->h_items.begin() + lo);
    };
    for (const Wave &w : b->waves) {
        segment(w.ibegin, w.ibegin + w.nwide_items);
        segment(w.ibegin + w.nwide_items, w.iend);
    }
}

// Plan the batch's pair order, waves, strip items and per-run state for the
// wave policy `overlap`, grow the buffers that depend on the plan, and copy
// the plan to the device.  Called by the upload, and again when a
// configuration with the other policy runs the batch.
// stream_idle: the caller has synchronized the stream since the batch's
// buffers were last used (copies the caller enqueued since then are fine)
static int plan_waves(mp_dp_ctx *c, mp_dp_batch *b, const mp_dp_tuning &t, bool stream_idle)
{
    const bool overlap = t.overlap_waves != 0;
    const size_t n = b->n;
    const uint64_t strips = b->strips_total;
    b->waves.clear();
    b->code_bytes_total = 0;
    b->record_bytes_total = b->record_read_total = b->bnd_bytes_total = 0;
    // ---- pair order: largest first (longest-processing-time first), ties
    // in input order
    std::vector<uint64_t> pcells(n);
    for (size_t k = 0; k < n; ++k) pcells[k] = static_cast<uint64_t>(b->desc[k].prot_len) * b->desc[k].nt_len;
    b->order.resize(n);
    for (size_t k = 0; k < n; ++k) b->order[k] = static_cast<uint32_t>(k);
    std::sort(b->order.begin(), b->order.end(), [&](uint32_t x, uint32_t y) {
        return pcells[x] != pcells[y] ? pcells[x] > pcells[y] : x < y;
    });
    // ---- waves under the traceback budget
    // Every wave gets a share of large and small pairs: pairs are taken
    // largest first and placed in the wave with the least work (cells) whose
    // traceback bytes still fit; a wave made only of the largest pairs would
    // have too few strips to keep every SM busy.
    const uint64_t cap = c->budget;
    std::vector<uint64_t> cbytes(n, 0);
    uint64_t total_bytes = 0;
    // strip form of each pair under this configuration.  A 128-residue strip
    // takes about twice as long per step as a 64-residue one and lags its
    // predecessor by three chunks instead of two, so a pair's critical path
    // is longer in the wide form: pairs whose wide critical path would exceed
    // the batch's longest one in 64-residue strips stay in 64-residue strips.
    uint64_t crit64 = 0;
    for (uint32_t k = 0; k < n; ++k) {
        const PairDesc &d = b->desc[k];
        if (d.flags & PF_SKIP) continue;
        crit64 = std::max<uint64_t>(crit64, div_up(d.nt_len + kStripW - 1, kChunk) + 2 * div_up(d.prot_len, kStripW));
    }
    for (uint32_t k = 0; k < n; ++k) {
        PairDesc &d = b->desc[k];
        d.flags &= ~PF_W128;
        const uint64_t crit128 =
            div_up(d.nt_len + kStripWMax - 1, kChunk) + 3 * div_up(d.prot_len, kStripWMax);
        if (t.strip_width && !c->params.force_int32 && use_w128(d) && (t.strip_width == 2 || 2 * crit128 <= crit64))
            d.flags |= PF_W128;
        d.n_strips = static_cast<uint32_t>(div_up(d.prot_len, strip_w_of(d.flags)));
    }
    for (uint32_t k = 0; k < n; ++k) {
        PairDesc &d = b->desc[k];
        if (d.flags & (PF_SKIP | PF_SCORE_ONLY)) continue;
        uint64_t cb = div_up(code_bytes(d.prot_len, d.nt_len, (d.flags & PF_WIDE) != 0, (d.flags & PF_W128) != 0),
                             256) * 256;
        if (cb > cap) {
            d.flags |= PF_BUDGET | PF_SCORE_ONLY;
            cb = 0;
        }
        cbytes[k] = cb;
        total_bytes += cb;
    }
    // With the overlapped-wave policy, a batch that needs several waves plans
    // them at half the budget and runs them alternately on two streams over
    // two halves of the arena, so one wave's tail (its longest pairs) overlaps
    // the next wave's start and its traceback; a pair larger than half the
    // budget keeps one wave per budget.
    uint64_t maxcb = 0;
    for (uint32_t k = 0; k < n; ++k) maxcb = std::max(maxcb, cbytes[k]);
    b->overlap = overlap && c->params.max_pairs_per_launch == 0 && total_bytes > cap && maxcb <= cap / 2;
    const uint64_t wcap = b->overlap ? cap / 2 : cap;
    std::vector<uint32_t> wave_of(n, 0);
    std::vector<uint64_t> wbytes, wcells;
    const size_t nw0 = static_cast<size_t>(std::max<uint64_t>(1, div_up(total_bytes, wcap)));
    wbytes.assign(nw0, 0);
    wcells.assign(nw0, 0);
    // waves by (work, index): the first one with room is the least-loaded
    // wave that fits, the lowest index among equals
    std::set<std::pair<uint64_t, uint32_t>> by_load;
    for (uint32_t w = 0; w < nw0; ++w) by_load.insert({0, w});
    for (uint32_t k = 0; k < n; ++k) {
        const uint32_t p = b->order[k];
        uint32_t best = UINT32_MAX;
        for (auto it = by_load.begin(); it != by_load.end(); ++it) {
            if (wbytes[it->second] + cbytes[p] <= wcap) {
                best = it->second;
                by_load.erase(it);
                break;
            }
        }
        if (best == UINT32_MAX) {
            best = static_cast<uint32_t>(wbytes.size());
            wbytes.push_back(0);
            wcells.push_back(0);
        }
        wave_of[p] = best;
        wbytes[best] += cbytes[p];
        wcells[best] += pcells[p];
        by_load.insert({wcells[best], best});
    }
    // group the largest-first order by wave, PF_WIDE pairs first within a wave
    // (so that their items form a prefix the int32 kernel can take directly),
    // otherwise still largest first
    auto wide = [&](uint32_t x) { return (b->desc[x].flags & PF_WIDE) && !(b->desc[x].flags & PF_SKIP) ? 0 : 1; };
    {
        // stable counting sort by key = 2 * wave + (not wide)
        std::vector<uint32_t> start(2 * wbytes.size() + 1, 0), sorted(n);
        for (uint32_t x : b->order) ++start[2 * wave_of[x] + wide(x) + 1];
        for (size_t v = 1; v < start.size(); ++v) start[v] += start[v - 1];
        for (uint32_t x : b->order) sorted[start[2 * wave_of[x] + wide(x)]++] = x;
        b->order.swap(sorted);
    }
    // strip items in pair order; each wave is a contiguous range
    uint64_t cur = 0, maxw = 0;
    uint32_t wbeg = 0, ibeg = 0, wcur = 0, nwide = 0;
    b->h_items.clear();
    b->h_items.reserve(strips);
    b->item_off.assign(n + 1, 0);
    for (uint32_t k = 0; k < n; ++k) {
        const uint32_t p = b->order[k];
        PairDesc &d = b->desc[p];
        if (wave_of[p] != wcur) {
            b->waves.push_back(Wave{wbeg, k, ibeg, static_cast<uint32_t>(b->h_items.size()), cur, nwide});
            maxw = std::max(maxw, cur);
            wbeg = k;
            ibeg = static_cast<uint32_t>(b->h_items.size());
            cur = 0;
            nwide = 0;
            wcur = wave_of[p];
        }
        b->item_off[k] = static_cast<uint32_t>(b->h_items.size());
        if (d.flags & PF_SKIP) continue;
        d.code_off = cur;
        cur += cbytes[p];
        if (cbytes[p])
            b->code_bytes_total += code_bytes(d.prot_len, d.nt_len, (d.flags & PF_WIDE) != 0, (d.flags & PF_W128) != 0);
        {
            const uint64_t W = (d.flags & PF_W128) ? kStripWMax : kStripW;
            const uint64_t nch = div_up(static_cast<uint64_t>(d.nt_len) + W - 1, kChunk);
            b->record_bytes_total += records_of(d.nt_len) * sizeof(uint4);
            // each strip queues one chunk of records ahead of its first
            b->record_read_total += static_cast<uint64_t>(d.n_strips) * (nch + 1) * kChunk * sizeof(uint4);
            b->bnd_bytes_total += static_cast<uint64_t>(d.n_strips > 0 ? d.n_strips - 1 : 0) * nch * kChunk *
                                  ((d.flags & PF_WIDE) ? 8 : 4);
        }
        for (uint32_t s = 0; s < d.n_strips; ++s) b->h_items.push_back(make_uint2(p, s));
        if (wide(p) == 0) nwide += d.n_strips;
    }
    b->item_off[n] = static_cast<uint32_t>(b->h_items.size());
    b->waves.push_back(Wave{wbeg, static_cast<uint32_t>(n), ibeg, static_cast<uint32_t>(b->h_items.size()), cur, nwide});
    if (c->params.max_pairs_per_launch == 0 && t.item_order) interleave_items(c, b);
    maxw = std::max(maxw, cur);
    if (b->waves.size() < 2) b->overlap = false;
    b->arena_half = std::max<uint64_t>(div_up(maxw, 256) * 256, 256);
    // per-run state block
    // counters: 8 per wave ([0] main-pass head, [4] re-run head, [5] re-run
    // count), the compaction total, and a head per pair group for the
    // one-launch-per-group form
    const size_t ncnt = 8 * b->waves.size() + 8 + 4 * n;
    b->off_done = div_up(ncnt * 4, 8) * 8;
    b->off_progress = b->off_done + div_up(n * 4, 8) * 8;
    b->off_key = b->off_progress + div_up(strips * 4, 8) * 8;
    b->state_bytes = b->off_key + n * 8 + 8;

    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
    b->runs = 0;
    b->planned = plan_key(b, t);
    cudaError_t e = cudaSuccess;
    const uint64_t arena_need = b->overlap ? 2 * b->arena_half : std::max<uint64_t>(maxw, 256);
    if (c->codes_ext && arena_need > c->codes_ext_cap) return MP_ENOMEM;
    if ((e = b->state.reserve(b->state_bytes / 8 + 1)) != cudaSuccess ||
        (e = b->wave_nwide.reserve(b->waves.size())) != cudaSuccess ||
        (!c->codes_ext && (e = c->codes.reserve(arena_need)) != cudaSuccess))
        return e == cudaErrorMemoryAllocation ? MP_ENOMEM : MP_ECUDA;
    cudaStream_t st = c->stream;
    // no run of an earlier plan still reads these buffers, and the pinned
    // plan staging buffer is free again
    if (!stream_idle) CK(cudaStreamSynchronize(st));
    // descriptors, order, items and wave counts go out of pinned memory, so
    // the copies do not wait for sequence copies already on the stream
    const size_t o_desc = 0, o_work = div_up(n * sizeof(PairDesc), 16) * 16;
    const size_t o_items = o_work + div_up(n * sizeof(uint32_t), 16) * 16;
    const size_t o_nw = o_items + div_up(b->h_items.size() * sizeof(uint2), 16) * 16;
    const size_t total = o_nw + b->waves.size() * sizeof(uint32_t);
    if (c->pstaging.reserve(total + 16) != cudaSuccess) return MP_ENOMEM;
    char *h = c->pstaging.p;
    memcpy(h + o_desc, b->desc.data(), n * sizeof(PairDesc));
    memcpy(h + o_work, b->order.data(), n * sizeof(uint32_t));
    memcpy(h + o_items, b->h_items.data(), b->h_items.size() * sizeof(uint2));
    uint32_t *nw = reinterpret_cast<uint32_t *>(h + o_nw);
    for (size_t w = 0; w < b->waves.size(); ++w) nw[w] = b->waves[w].nwide_items;
    CK(cudaMemcpyAsync(b->d_desc.p, h + o_desc, n * sizeof(PairDesc), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(b->work.p, h + o_work, n * sizeof(uint32_t), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(b->items.p, h + o_items, b->h_items.size() * sizeof(uint2), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(b->wave_nwide.p, nw, b->waves.size() * sizeof(uint32_t), cudaMemcpyHostToDevice, st));
    return MP_OK;
}

// (Re)fill batch b with n pairs: plan strips, waves and offsets on the host,
// grow the device buffers when needed, and copy the inputs to the device.
// Wait until the last copy out of the staging buffer has left it.
static cudaError_t staging_wait(mp_dp_ctx *c)
{
    if (!c->staging_busy) return cudaSuccess;
    c->staging_busy = false;
    return cudaEventSynchronize(c->ev_staging);
}

// ascii_on_device: the caller writes the batch's ASCII into b->ascii on the
// context's stream itself (the pairs' nt pointers are unused and may be null;
// the protein pointers still serve the score bound).
// A profile query's positions are within range and keep the degenerate
// intron paths losing (r above every negated score, as mp_dp_init requires
// of the matrix).
static bool profile_valid(const mp_dp_ctx *c, const mp_profile_pos *pf, uint32_t m)
{
    for (uint32_t j = 0; j <= m; ++j) {
        const mp_profile_pos &x = pf[j];
        if (x.gap_open < 0 || x.gap_ext < 1 || x.gap_open + x.gap_ext > 1000) return false;
        if (j == 0) continue;
        for (int a = 0; a < 21; ++a)
            if (x.subst[a] < -500 || x.subst[a] > 500 || !(c->params.r > -x.subst[a])) return false;
    }
    return true;
}

// An upper bound of a profile query's local score: the sum over positions
// of their best score (at least 0).
static int64_t profile_score_bound(const mp_profile_pos *pf, uint32_t m)
{
    int64_t s = 0;
    for (uint32_t j = 1; j <= m; ++j) {
        int b = 0;
        for (int a = 0; a < 21; ++a) b = std::max<int>(b, pf[j].subst[a]);
        s += b;
    }
    return s;
}

static int upload_impl(mp_dp_ctx *c, mp_dp_batch *b, const mp_pair *pairs, size_t n, bool ascii_on_device = false)
{
    for (size_t k = 0; k < n; ++k) {
        const mp_pair &q = pairs[k];
        if ((q.prot_len && !q.prot) || (q.nt_len && !q.nt && !ascii_on_device)) return MP_EINVAL;
        if (q.strand != 1 && q.strand != -1) return MP_EINVAL;
        if (q.prot_len >= (1u << 20) || q.nt_len >= (1u << 20) - 1024) return MP_EINVAL;
    }
    if (cudaSetDevice(c->device) != cudaSuccess) return MP_ECUDA;
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
    b->runs = 0;
    b->n = n;
    b->desc.assign(n, PairDesc{});
    b->nt_len.resize(n);
    b->strand.resize(n);
    b->waves.clear();
    b->cells = 0;
    b->code_bytes_total = 0;
    b->record_bytes_total = b->record_read_total = b->bnd_bytes_total = 0;
    // ---- shared host ranges: when every pair's region lies in one host
    // range no longer than the regions' total length (windows of one genome),
    // and the same holds for the proteins (one protein, several regions),
    // the two ranges are sent once and the pairs point into them
    uintptr_t nlo = UINTPTR_MAX, nhi = 0, plo = UINTPTR_MAX, phi = 0;
    uint64_t nsum = 0, psum = 0;
    for (size_t k = 0; k < n; ++k) {
        const mp_pair &q = pairs[k];
        if (q.nt_len) {
            const uintptr_t x = reinterpret_cast<uintptr_t>(q.nt);
            nlo = std::min(nlo, x);
            nhi = std::max(nhi, x + q.nt_len);
            nsum += q.nt_len;
        }
        if (q.prot_len) {
            const uintptr_t x = reinterpret_cast<uintptr_t>(q.prot);
            plo = std::min(plo, x);
            phi = std::max(phi, x + q.prot_len);
            psum += q.prot_len;
        }
    }
    const uint64_t nspan = nsum ? nhi - nlo : 0, pspan = psum ? phi - plo : 0;
    const uint64_t prot_base = div_up(nspan, 16) * 16;
    const bool span = !ascii_on_device && nsum && psum && nspan <= nsum && pspan <= psum &&
                      nspan + psum > 0 && prot_base + pspan < (uint64_t{1} << 32) && nspan + pspan < nsum + psum;
    // ---- layout
    const BoundTable bt(c->sp);
    uint64_t asc = 0, pro = 0, ntw = 0, bnd = 0, ops = 0, strips = 0, nrec = 0, nc0 = 0, npf = 0;
    const bool anchored = c->params.mode != MP_MODE_LOCAL;
    b->h_prof.clear();
    b->h_epre.clear();
    for (size_t k = 0; k < n; ++k) {
        const mp_pair &q = pairs[k];
        PairDesc &d = b->desc[k];
        if (q.profile) {
            // a profile query: its positions go to the device with the
            // prefix sums of their gap extensions
            if (!profile_valid(c, q.profile, q.prot_len)) return MP_EINVAL;
            d.flags |= PF_PROF;
            d.prof_off = npf;
            npf += static_cast<uint64_t>(q.prot_len) + 1;
            int32_t acc = 0;
            for (uint32_t j = 0; j <= q.prot_len; ++j) {
                ProfPos x;
                memcpy(&x, &q.profile[j], sizeof(x));
                b->h_prof.push_back(x);
                if (j > 0) acc += q.profile[j].gap_ext;
                b->h_epre.push_back(acc);
            }
        }
        d.prot_len = q.prot_len;
        d.nt_len = q.nt_len;
        d.strand = q.strand;
        if (span) {
            d.asc_prot_off = static_cast<uint32_t>(
                prot_base + (q.prot_len ? reinterpret_cast<uintptr_t>(q.prot) - plo : 0));
            d.asc_nt_off = q.nt_len ? reinterpret_cast<uintptr_t>(q.nt) - nlo : 0;
        } else {
            d.asc_prot_off = static_cast<uint32_t>(asc);
            asc += q.prot_len;
            d.asc_nt_off = asc;
            asc += q.nt_len;
            asc = div_up(asc, 16) * 16;
        }
        d.prot_off = static_cast<uint32_t>(pro);
        pro += q.prot_len;
        d.nt_word_off = static_cast<uint32_t>(ntw + kNtPadWords);
        ntw += div_up(q.nt_len, 16) + 2 * kNtPadWords;
        d.bnd_off = bnd;
        bnd += bnd_entries(q.nt_len);
        d.rec_off = nrec;
        nrec += records_of(q.nt_len);
        d.col0_off = nc0;
        if (anchored) nc0 += static_cast<uint64_t>(q.nt_len) + 1 + kCol0Pad;
        d.cig_off = ops;
        d.cig_cap = q.prot_len + q.nt_len + 2;
        ops += d.cig_cap;
        d.n_strips = static_cast<uint32_t>(div_up(q.prot_len, kStripW));
        d.strip_base = static_cast<uint32_t>(strips);
        strips += d.n_strips;
        // global mode reads its score at the end cell from the traceback stream
        if ((q.flags & MP_PAIR_SCORE_ONLY) && c->params.mode != MP_MODE_GLOBAL) d.flags |= PF_SCORE_ONLY;
        if (q.prot_len == 0 || q.nt_len == 0) d.flags |= PF_SKIP;
        const int64_t bound = q.profile ? profile_score_bound(q.profile, q.prot_len)
                                        : score_bound(bt, q.prot, q.prot_len, kOverflowT);
        if (c->params.force_int32 || (q.prot_len && bound >= kOverflowT)) d.flags |= PF_WIDE;
        // anchored modes: H may go negative; a path through row 0 and one
        // column (I run, D run, a frameshift) bounds it from below.  Pairs whose
        // bound leaves the int16 range safely run in int32 (PF_WIDE pairs of
        // these modes skip the int16 pass).
        if (anchored) {
            int64_t gq = c->params.q, ge = c->params.e;
            if (q.profile)
                for (uint32_t j = 0; j <= q.prot_len; ++j) {
                    gq = std::max<int64_t>(gq, q.profile[j].gap_open);
                    ge = std::max<int64_t>(ge, q.profile[j].gap_ext);
                }
            const int64_t lower = 2 * gq + c->params.f + ge * (q.prot_len + q.nt_len / 3 + 2);
            if (lower >= 12000) d.flags |= PF_WIDE;
            // the int32 path represents -inf by -2^28; with half of that as
            // margin, a pair whose H could fall lower is refused
            if (lower >= (int64_t{1} << 27)) return MP_EINVAL;
        }
        b->nt_len[k] = q.nt_len;
        b->strand[k] = q.strand;
        b->cells += static_cast<double>(q.prot_len) * q.nt_len;
    }
    if (span) asc = prot_base + pspan;
    if (asc > 0xffffffffull || pro > 0xffffffffull || ntw > 0xffffffffull || strips > 0xffffffffull)
        return MP_EINVAL;
    b->ascii_bytes = asc; b->prot_total = pro; b->nt_words = ntw; b->bnd_total = bnd; b->ops_total = ops;

    b->strips_total = strips;

    // ---- device buffers (grown, never shrunk)
    cudaError_t e = cudaSuccess;
    if ((e = b->ascii.reserve(asc + 16)) != cudaSuccess || (e = b->d_desc.reserve(n + 1)) != cudaSuccess ||
        (e = b->prot.reserve(pro + 16)) != cudaSuccess || (e = b->nt2.reserve(ntw + 32)) != cudaSuccess ||
        (e = b->out.reserve(n + 1)) != cudaSuccess || (e = b->ops.reserve(ops + 1)) != cudaSuccess ||
        (e = b->cig.reserve(ops + 1)) != cudaSuccess || (e = b->work.reserve(n + 1)) != cudaSuccess ||
        (e = b->items.reserve(strips + 1)) != cudaSuccess ||
        (e = b->rerun_items.reserve(strips + 1)) != cudaSuccess || (e = b->bnd.reserve(bnd + 1)) != cudaSuccess ||
        (anchored && (e = b->col0.reserve(nc0 + 1)) != cudaSuccess) ||
        (npf && (e = b->prof.reserve(npf)) != cudaSuccess) || (npf && (e = b->epre.reserve(npf)) != cudaSuccess) ||
        (e = b->recs.reserve(nrec + 1)) != cudaSuccess) {
        return e == cudaErrorMemoryAllocation ? MP_ENOMEM : MP_ECUDA;
    }
    cudaStream_t st = c->stream;
    // no earlier run still uses this batch's buffers or the context's
    // arenas, and the staging buffers are free
    CK(cudaStreamSynchronize(st));
    c->staging_busy = false;
    if (npf) {
        // profile queries' positions (pageable host memory: the copies
        // return once the data is staged)
        CK(cudaMemcpyAsync(b->prof.p, b->h_prof.data(), npf * sizeof(ProfPos), cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(b->epre.p, b->h_epre.data(), npf * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    }
    b->needs_waves = plan_code_bytes(c, b) > c->budget;
    b->shape_key = shape_key_of(*b);
    b->planned = -1;
    if (ascii_on_device) return plan_waves(c, b, tuning_for(c, b), true);
    // ---- host -> device: worker threads gather the sequences into the
    // pinned staging buffer and send each ~2 MB range as soon as it is
    // gathered, while this thread plans the waves; nothing waits for the
    // copies here: the pipeline follows them on the stream, and the next
    // user of the staging buffer waits for ev_staging
    if (c->staging.reserve(asc + 16) != cudaSuccess) return MP_ENOMEM;
    std::atomic<int> copy_err{0};
    auto gather_send = [&](size_t k0, size_t k1) {
        // (a worker thread issues copies on the context's stream: its device first)
        if (cudaSetDevice(c->device) != cudaSuccess) copy_err = 1;
        size_t from = k0;
        uint64_t acc = 0;
        for (size_t k = k0; k < k1; ++k) {
            const mp_pair &q = pairs[k];
            if (q.prot_len) memcpy(c->staging.p + b->desc[k].asc_prot_off, q.prot, q.prot_len);
            if (q.nt_len) memcpy(c->staging.p + b->desc[k].asc_nt_off, q.nt, q.nt_len);
            acc += q.prot_len + q.nt_len;
            if (acc >= (2u << 20) || k + 1 == k1) {
                const uint64_t lo = b->desc[from].asc_prot_off;
                const uint64_t hi = k + 1 < n ? b->desc[k + 1].asc_prot_off : asc;
                if (hi > lo && cudaMemcpyAsync(b->ascii.p + lo, c->staging.p + lo, hi - lo, cudaMemcpyHostToDevice,
                                               st) != cudaSuccess)
                    copy_err = 1;
                from = k + 1;
                acc = 0;
            }
        }
    };
    // shared ranges: staging [0, nspan) is the regions' host range,
    // [prot_base, prot_base + pspan) the proteins'; sent in ~2 MB pieces
    auto span_send = [&](uint64_t lo, uint64_t hi) {
        if (cudaSetDevice(c->device) != cudaSuccess) copy_err = 1;
        for (uint64_t a = lo; a < hi;) {
            const uint64_t e = std::min<uint64_t>(hi, a + (2u << 20));
            const uint64_t n0 = a, n1 = std::min(e, nspan);
            if (n1 > n0) memcpy(c->staging.p + n0, reinterpret_cast<const char *>(nlo) + n0, n1 - n0);
            const uint64_t p0 = std::max(a, prot_base), p1 = std::min(e, prot_base + pspan);
            if (p1 > p0) memcpy(c->staging.p + p0, reinterpret_cast<const char *>(plo) + (p0 - prot_base), p1 - p0);
            if (cudaMemcpyAsync(b->ascii.p + a, c->staging.p + a, e - a, cudaMemcpyHostToDevice, st) != cudaSuccess)
                copy_err = 1;
            a = e;
        }
    };
    const unsigned nthr = asc > (16u << 20) ? std::min(16u, std::max(1u, std::thread::hardware_concurrency())) : 0u;
    if (nthr && !c->pool) {
        c->pool.reset(new (std::nothrow) WorkerPool());
        if (c->pool) c->pool->start(nthr);
    }
    const bool pooled = nthr && c->pool;
    if (pooled) {
        const unsigned nj = static_cast<unsigned>(c->pool->th.size());
        if (span)
            c->pool->run(nj, [&, nj](unsigned t) { span_send(asc * t / nj, asc * (t + 1) / nj); });
        else
            c->pool->run(nj, [&, nj](unsigned t) { gather_send(n * t / nj, n * (t + 1) / nj); });
    }
    // the plan reads the layout fields of the descriptors the workers read
    // and writes others (code offsets), and copies out of its own buffer
    const int rc = plan_waves(c, b, tuning_for(c, b), true);
    if (pooled) c->pool->wait();
    else if (span) span_send(0, asc);
    else gather_send(0, n);
    if (rc != MP_OK) return rc;
    if (copy_err) return MP_ECUDA;
    CK(cudaEventRecord(c->ev_staging, st));
    c->staging_busy = true;
    return MP_OK;
}

int mp_dp_batch_upload(mp_dp_ctx *c, const mp_pair *pairs, size_t n, mp_dp_batch **out)
{
    if (!c || !out || (n && !pairs)) return MP_EINVAL;
    *out = nullptr;
    mp_dp_batch *b = new (std::nothrow) mp_dp_batch();
    if (!b) return MP_ENOMEM;
    const int rc = upload_impl(c, b, pairs, n);
    if (rc != MP_OK) {
        mp_dp_batch_free(c, b);
        return rc;
    }
    *out = b;
    return MP_OK;
}

// Enqueue the device pipeline of a batch on stream st with configuration t.
static int enqueue_pipeline(mp_dp_ctx *c, mp_dp_batch *b, cudaStream_t st, bool timed, bool capturing,
                            const mp_dp_tuning &t)
{
    const uint32_t n = static_cast<uint32_t>(b->n);
    int launches = 0, dp_launches = 0;
    auto rec_on = [&](int idx, cudaStream_t s_) -> cudaError_t {
        // inside a stream capture only an External record becomes an event-record node
        if (!timed) return cudaSuccess;
        return capturing ? cudaEventRecordWithFlags(b->events[idx], s_, cudaEventRecordExternal)
                         : cudaEventRecord(b->events[idx], s_);
    };
    auto rec = [&](int idx) { return rec_on(idx, st); };
    char *state = reinterpret_cast<char *>(b->state.p);
    uint32_t *counters = reinterpret_cast<uint32_t *>(state);
    const size_t W = b->waves.size();
    CK(rec(0));
    CK(cudaMemsetAsync(state, 0, b->state_bytes, st));
    CK(launch_pack(b->d_desc.p, n, b->ascii.p, b->prot.p, b->nt2.p, b->out.p, st));
    CK(launch_records(b->d_desc.p, n, b->nt2.p, c->sp, b->recs.p, st));
    launches += 2;
    const bool anchored = c->params.mode != MP_MODE_LOCAL;
    if (anchored) {
        CK(launch_col0(b->d_desc.p, n, b->nt2.p, c->sp, b->prof.p, b->col0.p, st));
        ++launches;
    }
    CK(rec(1));
    const int variant = t.dp16_variant == 1 ? 1 : 0;
    const bool wide4 = t.strip_width != 0 && !c->params.force_int32;
    const int fit16 = dp16_blocks_per_sm(variant, wide4), fit32 = dp32_blocks_per_sm();
    const int g16 = c->num_sms * (t.dp16_ctas_per_sm > 0 ? std::min(t.dp16_ctas_per_sm, fit16) : fit16);
    const int g32 = c->num_sms * (t.dp32_ctas_per_sm > 0 ? std::min(t.dp32_ctas_per_sm, fit32) : fit32);
    // in the anchored modes PF_WIDE pairs never take the int16 pass
    const bool direct = (t.wide_direct != 0 || anchored) && !c->params.force_int32;
    const int per_launch = c->params.max_pairs_per_launch;
    const bool overlap = b->overlap && W > 1;
    if (overlap) {
        // the second stream joins after packing (and, under capture, joins the graph)
        CK(cudaEventRecord(c->ev_fork, st));
        CK(cudaStreamWaitEvent(c->stream2, c->ev_fork, 0));
    }
    const cudaStream_t main_st = st;
    for (size_t w = 0; w < W; ++w) {
        const Wave &wv = b->waves[w];
        // odd waves of an overlapped batch: second stream, second arena half
        // (this `st` shadows the main stream for the wave's launches)
        const cudaStream_t st = overlap && (w & 1) ? c->stream2 : main_st;
        uint8_t *arena = (c->codes_ext ? c->codes_ext : c->codes.p) + (overlap && (w & 1) ? b->arena_half : 0);
        CK(rec_on(static_cast<int>(2 + EV_PER_WAVE * w), st));
        DPArgs a{};
        a.pairs = b->d_desc.p;
        a.recs = b->recs.p;
        a.prot = b->prot.p;
        a.nt2 = b->nt2.p;
        a.codes = arena;
        a.bnd = b->bnd.p;
        a.col0 = anchored ? b->col0.p : nullptr;
        a.out = b->out.p;
        a.progress = reinterpret_cast<uint32_t *>(state + b->off_progress);
        a.best_key = reinterpret_cast<unsigned long long *>(state + b->off_key);
        a.strips_done = reinterpret_cast<uint32_t *>(state + b->off_done);
        a.rerun_items = b->rerun_items.p + wv.ibegin;
        a.rerun_count = counters + 8 * w + 5;
        a.sp = c->sp;
        a.spin_limit = c->params.wait_limit > 0 ? static_cast<uint32_t>(c->params.wait_limit) : 0u;
        a.no_publish = (c->params.debug_flags & MP_DEBUG_NO_PUBLISH) ? 1u : 0u;
        a.ops = b->ops.p;
        a.mat = c->d_mat.p;
        a.prof = b->prof.p;
        a.epre = b->epre.p;
        const uint32_t nitems = wv.iend - wv.ibegin;
        if (per_launch > 0) {
            // plain form: one kernel launch per group of pairs
            for (uint32_t k = wv.begin; k < wv.end; k += per_launch) {
                const uint32_t k2 = std::min<uint32_t>(wv.end, k + per_launch);
                DPArgs a1 = a;
                a1.items = b->items.p + b->item_off[k];
                a1.n_items = b->item_off[k2] - b->item_off[k];
                if (!a1.n_items) continue;
                a1.head = counters + 8 * W + 8 + 4 * k;
                const int grid = std::max(1, std::min<int>(c->num_sms, static_cast<int>((a1.n_items + kWarpsPerCta - 1) / kWarpsPerCta)));
                if (c->params.force_int32) CK(launch_dp32(a1, grid, false, st));
                else CK(launch_dp16(a1, grid, variant, wide4, st));
                ++launches;
                ++dp_launches;
            }
        } else {
            // with wide_direct the PF_WIDE pairs' items (a prefix of the wave's
            // range) go straight to the int32 kernel's queue
            const uint32_t skip = direct ? wv.nwide_items : 0;
            if (skip) {
                CK(cudaMemcpyAsync(b->rerun_items.p + wv.ibegin, b->items.p + wv.ibegin, skip * sizeof(uint2),
                                   cudaMemcpyDeviceToDevice, st));
                CK(cudaMemcpyAsync(a.rerun_count, b->wave_nwide.p + w, sizeof(uint32_t), cudaMemcpyDeviceToDevice, st));
            }
            // the wave's interleaved strip items (the wide prefix, if handed
            // to the int32 queue, is skipped)
            a.items = b->items.p + wv.ibegin + skip;
            a.n_items = nitems - skip;
            a.head = counters + 8 * w;
            const int want = static_cast<int>((a.n_items + kWarpsPerCta - 1) / kWarpsPerCta);
            const int grid16 = std::max(1, std::min<int>(g16, want));
            const int grid32 = std::max(1, std::min<int>(g32, want));
            if (c->params.force_int32) CK(launch_dp32(a, grid32, false, st));
            else CK(launch_dp16(a, grid16, variant, wide4, st));
            ++launches;
            ++dp_launches;
        }
        CK(rec_on(static_cast<int>(3 + EV_PER_WAVE * w), st));
        // only PF_WIDE pairs can saturate int16 (others are marked MP_ST_TRACE
        // if they ever did): a wave without them needs no re-run launch
        if (!c->params.force_int32 && wv.nwide_items > 0) {
            a.head = counters + 8 * w + 4;
            a.items = nullptr;
            a.n_items = 0;
            CK(launch_dp32(a, g32, true, st));
            ++launches;
            ++dp_launches;
        }
        CK(rec_on(static_cast<int>(4 + EV_PER_WAVE * w), st));
        TBArgs t{};
        t.pairs = b->d_desc.p;
        t.work = b->work.p + wv.begin;
        t.n_work = wv.end - wv.begin;
        t.codes = arena;
        t.prot = b->prot.p;
        t.nt2 = b->nt2.p;
        t.out = b->out.p;
        t.ops = b->ops.p;
        t.col0 = anchored ? b->col0.p : nullptr;
        t.sp = c->sp;
        t.prof = b->prof.p;
        t.epre = b->epre.p;
        const int tgrid = std::max(1, std::min<int>(c->num_sms * 8, static_cast<int>((t.n_work + 7) / 8)));
        CK(launch_tb(t, tgrid, st));
        ++launches;
        CK(rec_on(static_cast<int>(5 + EV_PER_WAVE * w), st));
    }
    if (overlap) {
        CK(cudaEventRecord(c->ev_join, c->stream2));
        CK(cudaStreamWaitEvent(st, c->ev_join, 0));
    }
    CK(rec(static_cast<int>(2 + EV_PER_WAVE * W)));
    CK(launch_compact(b->d_desc.p, b->out.p, n, b->ops.p, b->cig.p, counters + cig_total_index(b), st));
    launches += 2;
    CK(rec(static_cast<int>(3 + EV_PER_WAVE * W)));
    b->n_launches = launches;
    b->n_dp_launches = dp_launches;
    return MP_OK;
}

static uint64_t tuning_sig(const mp_dp_tuning &t, bool timed)
{
    return (static_cast<uint64_t>(t.dp16_variant & 0xff)) | (static_cast<uint64_t>(t.dp16_ctas_per_sm & 0xff) << 8) |
           (static_cast<uint64_t>(t.dp32_ctas_per_sm & 0xff) << 16) | (static_cast<uint64_t>(t.wide_direct & 1) << 24) |
           (static_cast<uint64_t>(timed) << 25) | (static_cast<uint64_t>(t.overlap_waves & 1) << 26) |
           (static_cast<uint64_t>(t.item_order & 1) << 27) | (1ull << 28) | (static_cast<uint64_t>(t.strip_width & 3) << 29);
}

static int autotune_impl(mp_dp_ctx *c, mp_dp_batch *b, mp_dp_tuning *best, mp_dp_tuning *tried, int max_tried,
                         int *n_tried);

int mp_dp_batch_run(mp_dp_ctx *c, mp_dp_batch *b)
{
    if (!c || !b) return MP_EINVAL;
    if (cudaSetDevice(c->device) != cudaSuccess) return MP_ECUDA;
    cudaStream_t st = c->stream;
    const bool timed = c->timing;
    if (c->params.autotune && !c->has_fixed && c->params.max_pairs_per_launch == 0 && b->n &&
        !c->tuned.count(b->shape_key)) {
        const int rc = autotune_impl(c, b, nullptr, nullptr, 0, nullptr);
        if (rc != MP_OK) return rc;
    }
    const mp_dp_tuning t = tuning_for(c, b);
    {
        const int rc = ensure_plan(c, b, t);
        if (rc != MP_OK) return rc;
    }
    const size_t nev = 4 + EV_PER_WAVE * b->waves.size();
    if (timed && b->events.size() < nev) {
        for (size_t k = b->events.size(); k < nev; ++k) {
            cudaEvent_t e;
            CK(cudaEventCreate(&e));
            b->events.push_back(e);
        }
    }
    // a batch run once is launched directly; from its second run on, the
    // pipeline is captured once as a CUDA graph and replayed (captured again
    // when the timing flag or the configuration changed)
    const bool use_graph = c->params.max_pairs_per_launch == 0 && ++b->runs >= 2;
    const uint64_t sig = tuning_sig(t, timed);
    if (use_graph && b->graph && b->graph_sig != sig) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    if (use_graph && !b->graph) {
        cudaGraph_t g;
        CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        int rc = enqueue_pipeline(c, b, st, timed, true, t);
        cudaError_t e = cudaStreamEndCapture(st, &g);
        if (rc != MP_OK) {
            if (e == cudaSuccess) cudaGraphDestroy(g);
            return rc;
        }
        CK(e);
        e = cudaGraphInstantiate(&b->graph, g, 0);
        cudaGraphDestroy(g);
        CK(e);
        b->graph_sig = sig;
    }
    if (use_graph) CK(cudaGraphLaunch(b->graph, st));
    else {
        int rc = enqueue_pipeline(c, b, st, timed, false, t);
        if (rc != MP_OK) return rc;
    }
    c->last = b;
    return MP_OK;
}

// ------------------------------------------------------------ autotuner
// Kernel candidates: both int16 builds at all CTAs per SM that fit and one
// fewer, and, when the batch has pairs that may need int32, both policies
// for them; each with the default plan (overlapped waves, interleaved items).
static std::vector<mp_dp_tuning> kernel_candidates(mp_dp_ctx *c, const mp_dp_batch *b)
{
    bool any_wide = false;
    for (const PairDesc &d : b->desc) any_wide |= (d.flags & PF_WIDE) && !(d.flags & (PF_SKIP | PF_SCORE_ONLY));
    std::vector<mp_dp_tuning> v;
    const int fit32 = dp32_blocks_per_sm();
    if (c->params.force_int32) {
        for (int k = fit32; k >= std::max(1, fit32 - 1); --k) {
            mp_dp_tuning t = default_tuning();
            t.dp32_ctas_per_sm = k;
            v.push_back(t);
        }
        return v;
    }
    for (int var = 0; var < kDp16Variants; ++var) {
        const int fit = dp16_blocks_per_sm(var);
        for (int k = fit; k >= std::max(1, fit - 1); --k)
            for (int wd = 0; wd <= (any_wide ? 1 : 0); ++wd) {
                mp_dp_tuning t = default_tuning();
                t.dp16_variant = var;
                t.dp16_ctas_per_sm = k;
                t.dp32_ctas_per_sm = fit32;
                t.wide_direct = wd;
                t.strip_width = 0;
                v.push_back(t);
            }
    }
    // 128-residue strips (the 2-CTA build that runs both strip forms), for
    // the pairs whose critical path allows it or for every eligible pair
    const int fitw = dp16_blocks_per_sm(1, true);
    for (int sw = 1; sw <= 2; ++sw)
        for (int wd = 0; wd <= (any_wide ? 1 : 0); ++wd) {
            mp_dp_tuning t = default_tuning();
            t.dp16_variant = 1;
            t.dp16_ctas_per_sm = fitw;
            t.dp32_ctas_per_sm = fit32;
            t.wide_direct = wd;
            t.strip_width = sw;
            v.push_back(t);
        }
    return v;
}

// Plan candidates around a kernel configuration: the other item order and,
// for a batch that needs several waves, the other wave policy.
static std::vector<mp_dp_tuning> plan_candidates(const mp_dp_batch *b, const mp_dp_tuning &k)
{
    std::vector<mp_dp_tuning> v;
    for (int ord = 0; ord <= 1; ++ord)
        for (int ov = 0; ov <= (b->needs_waves ? 1 : 0); ++ov) {
            mp_dp_tuning t = k;
            t.item_order = ord;
            t.overlap_waves = b->needs_waves ? ov : k.overlap_waves;
            if (t.item_order == k.item_order && t.overlap_waves == k.overlap_waves) continue;
            v.push_back(t);
        }
    return v;
}

static int time_run(mp_dp_ctx *c, mp_dp_batch *b, const mp_dp_tuning &t, cudaEvent_t e0, cudaEvent_t e1, float *ms)
{
    {
        const int rc = ensure_plan(c, b, t);        // outside the timed interval
        if (rc != MP_OK) return rc;
    }
    cudaStream_t st = c->stream;
    CK(cudaEventRecord(e0, st));
    const int rc = enqueue_pipeline(c, b, st, false, false, t);
    if (rc != MP_OK) return rc;
    CK(cudaEventRecord(e1, st));
    CK(cudaEventSynchronize(e1));
    CK(cudaEventElapsedTime(ms, e0, e1));
    return MP_OK;
}

static int autotune_impl(mp_dp_ctx *c, mp_dp_batch *b, mp_dp_tuning *best, mp_dp_tuning *tried, int max_tried,
                         int *n_tried)
{
    // two stages: the kernel configurations under the default plan, then the
    // plan options (item order, wave policy) under the fastest of those
    std::vector<mp_dp_tuning> cand = kernel_candidates(c, b);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return MP_ECUDA;
    }
    int rc = MP_OK;
    float ms = 0;
    // warm-up: first launches of each kernel build, pages of the buffers
    for (int var = 0; var < (c->params.force_int32 ? 1 : kDp16Variants) && rc == MP_OK; ++var) {
        mp_dp_tuning t = cand[0];
        t.dp16_variant = var;
        rc = time_run(c, b, t, e0, e1, &ms);
    }
    for (size_t k = 0; k < cand.size() && rc == MP_OK; ++k) rc = time_run(c, b, cand[k], e0, e1, &cand[k].ms);
    if (rc == MP_OK) {
        size_t k1 = 0;
        for (size_t k = 1; k < cand.size(); ++k)
            if (cand[k].ms < cand[k1].ms) k1 = k;
        for (const mp_dp_tuning &t : plan_candidates(b, cand[k1])) {
            cand.push_back(t);
            if ((rc = time_run(c, b, cand.back(), e0, e1, &cand.back().ms)) != MP_OK) break;
        }
    }
    if (rc == MP_OK && cand.size() > 1) {
        // the two fastest once more; each keeps its lower time
        std::vector<size_t> idx(cand.size());
        for (size_t k = 0; k < idx.size(); ++k) idx[k] = k;
        std::stable_sort(idx.begin(), idx.end(), [&](size_t x, size_t y) { return cand[x].ms < cand[y].ms; });
        for (int r = 0; r < 2 && rc == MP_OK; ++r) {
            rc = time_run(c, b, cand[idx[r]], e0, e1, &ms);
            cand[idx[r]].ms = std::min(cand[idx[r]].ms, ms);
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != MP_OK) return rc;
    size_t bi = 0;
    for (size_t k = 1; k < cand.size(); ++k)
        if (cand[k].ms < cand[bi].ms) bi = k;
    c->tuned[b->shape_key] = cand[bi];
    if (b->planned != plan_key(b, cand[bi])) {
        // re-plan for the choice and run once more, so that the batch's
        // results (whose counters sit where the plan puts them) match its plan
        int rc = plan_waves(c, b, cand[bi]);
        if (rc == MP_OK) rc = enqueue_pipeline(c, b, c->stream, false, false, cand[bi]);
        if (rc != MP_OK) return rc;
        CK(cudaStreamSynchronize(c->stream));
    }
    c->last = b;
    if (best) *best = cand[bi];
    if (tried)
        for (size_t k = 0; k < cand.size() && static_cast<int>(k) < max_tried; ++k) tried[k] = cand[k];
    if (n_tried) *n_tried = static_cast<int>(cand.size());
    return MP_OK;
}

int mp_dp_autotune(mp_dp_ctx *c, mp_dp_batch *b, mp_dp_tuning *best, mp_dp_tuning *tried, int max_tried,
                   int *n_tried)
{
    if (!c || !b || (tried && max_tried < 0)) return MP_EINVAL;
    if (c->params.max_pairs_per_launch > 0) return MP_EINVAL;
    if (c->server_running) return MP_ESTATE;
    if (cudaSetDevice(c->device) != cudaSuccess) return MP_ECUDA;
    if (b->n == 0) {
        if (best) *best = tuning_for(c, b);
        if (n_tried) *n_tried = 0;
        return MP_OK;
    }
    return autotune_impl(c, b, best, tried, max_tried, n_tried);
}

int mp_dp_set_tuning(mp_dp_ctx *c, const mp_dp_tuning *t)
{
    if (!c) return MP_EINVAL;
    if (c->server_running) return MP_ESTATE;
    if (!t) {
        c->has_fixed = false;
        return MP_OK;
    }
    if (t->dp16_variant < 0 || t->dp16_variant >= kDp16Variants || t->dp16_ctas_per_sm < 0 ||
        t->dp32_ctas_per_sm < 0 || t->wide_direct < 0 || t->wide_direct > 1 || t->overlap_waves < 0 ||
        t->overlap_waves > 1 || t->item_order < 0 || t->item_order > 1 || t->strip_width < 0 || t->strip_width > 2)
        return MP_EINVAL;
    c->fixed = *t;
    c->has_fixed = true;
    return MP_OK;
}

int mp_dp_get_tuning(mp_dp_ctx *c, const mp_dp_batch *b, mp_dp_tuning *t)
{
    if (!c || !b || !t) return MP_EINVAL;
    *t = tuning_for(c, b);
    return MP_OK;
}

int mp_dp_tuning_save(mp_dp_ctx *c, const char *path)
{
    if (!c || !path) return MP_EINVAL;
    FILE *f = fopen(path, "w");
    if (!f) return MP_EINVAL;
    bool ok = fprintf(f, "mp_dp_tuning 4 %s %d\n", c->dev_name.c_str(), c->num_sms) > 0;
    for (const auto &kv : c->tuned) {
        const mp_dp_tuning &t = kv.second;
        ok = ok && fprintf(f, "%016llx %d %d %d %d %d %d %d %.4f\n", static_cast<unsigned long long>(kv.first),
                           t.dp16_variant, t.dp16_ctas_per_sm, t.dp32_ctas_per_sm, t.wide_direct, t.overlap_waves,
                           t.item_order, t.strip_width, static_cast<double>(t.ms)) > 0;
    }
    ok = (fclose(f) == 0) && ok;
    return ok ? MP_OK : MP_EINVAL;
}

int mp_dp_tuning_load(mp_dp_ctx *c, const char *path)
{
    if (!c || !path) return MP_EINVAL;
    if (c->server_running) return MP_ESTATE;
    FILE *f = fopen(path, "r");
    if (!f) return MP_EINVAL;
    char name[256] = {0};
    int version = 0, sms = 0;
    if (fscanf(f, "mp_dp_tuning %d %255s %d", &version, name, &sms) != 3 || version != 4 ||
        c->dev_name != name || sms != c->num_sms) {
        fclose(f);
        return MP_EINVAL;
    }
    std::map<uint64_t, mp_dp_tuning> got;
    for (;;) {
        unsigned long long key = 0;
        mp_dp_tuning t{};
        double ms = 0;
        const int k = fscanf(f, "%llx %d %d %d %d %d %d %d %lf", &key, &t.dp16_variant, &t.dp16_ctas_per_sm,
                             &t.dp32_ctas_per_sm, &t.wide_direct, &t.overlap_waves, &t.item_order, &t.strip_width, &ms);
        if (k == EOF) break;
        if (k != 9 || t.item_order < 0 || t.item_order > 1 || t.dp16_variant < 0 || t.dp16_variant >= kDp16Variants ||
            t.dp16_ctas_per_sm < 0 || t.dp32_ctas_per_sm < 0 || t.wide_direct < 0 || t.wide_direct > 1 ||
            t.overlap_waves < 0 || t.overlap_waves > 1 || t.strip_width < 0 || t.strip_width > 2) {
            fclose(f);
            return MP_EINVAL;
        }
        t.ms = static_cast<float>(ms);
        got[key] = t;
    }
    fclose(f);
    for (const auto &kv : got) c->tuned[kv.first] = kv.second;
    return MP_OK;
}

static int collect_stats(mp_dp_ctx *c, mp_dp_batch *b)
{
    mp_dp_stats &s = c->stats;
    memset(&s, 0, sizeof(s));
    s.cells = b->cells;
    s.n_waves = static_cast<int32_t>(b->waves.size());
    s.n_launches = b->n_launches;
    s.n_dp_launches = b->n_dp_launches;
    s.code_bytes = b->code_bytes_total;
    s.record_bytes = b->record_bytes_total;
    s.record_read_bytes = b->record_read_total;
    s.boundary_bytes = b->bnd_bytes_total;
    if (c->timing && !b->events.empty()) {
        float ms = 0;
        CK(cudaEventElapsedTime(&ms, b->events[0], b->events[1]));
        s.pack_ms = ms;
        // per wave on its own stream (overlapped waves: the sums exceed the wall time)
        for (size_t w = 0; w < b->waves.size(); ++w) {
            const size_t base = 2 + EV_PER_WAVE * w;
            CK(cudaEventElapsedTime(&ms, b->events[base], b->events[base + 1])); s.dp_ms += ms;
            CK(cudaEventElapsedTime(&ms, b->events[base + 1], b->events[base + 2])); s.rerun_ms += ms;
            CK(cudaEventElapsedTime(&ms, b->events[base + 2], b->events[base + 3])); s.tb_ms += ms;
        }
        const size_t end = 2 + EV_PER_WAVE * b->waves.size();
        CK(cudaEventElapsedTime(&ms, b->events[end], b->events[end + 1]));
        s.tb_ms += ms;
        CK(cudaEventElapsedTime(&ms, b->events[0], b->events[end + 1]));
        s.total_ms = ms;
    }
    return MP_OK;
}

int mp_dp_batch_sync(mp_dp_ctx *c)
{
    if (!c) return MP_EINVAL;
    if (cudaSetDevice(c->device) != cudaSuccess) return MP_ECUDA;
    CK(cudaStreamSynchronize(c->stream));
    if (c->last) return collect_stats(c, c->last);
    return MP_OK;
}

int mp_dp_batch_download(mp_dp_ctx *c, mp_dp_batch *b, mp_result *out)
{
    if (!c || !b || (b->n && !out)) return MP_EINVAL;
    if (cudaSetDevice(c->device) != cudaSuccess) return MP_ECUDA;
    cudaStream_t st = c->stream;
    const size_t n = b->n;
    b->h_out.resize(n);
    uint32_t total = 0;
    CK(cudaMemcpyAsync(b->h_out.data(), b->out.p, n * sizeof(PairOut), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(&total, reinterpret_cast<uint32_t *>(b->state.p) + cig_total_index(b), sizeof(uint32_t),
                       cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    c->host_cig.resize(std::max<size_t>(total, 1));
    if (total) {
        CK(cudaMemcpyAsync(c->host_cig.data(), b->cig.p, total * sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
    }
    int32_t nrerun = 0;
    for (size_t k = 0; k < n; ++k) {
        const PairOut &o = b->h_out[k];
        const PairDesc &d = b->desc[k];
        mp_result &r = out[k];
        memset(&r, 0, sizeof(r));
        r.status = o.status & 0xff;
        if (o.status & MP_ST_RERUN) ++nrerun;
        if ((o.status & MP_ST_ERRMASK) & ~MP_ST_BUDGET) continue;
        const bool global = c->params.mode == MP_MODE_GLOBAL;
        if (global && (d.flags & PF_BUDGET)) continue;                // no stream: no end-cell score
        r.score = global ? o.score : (o.score > 0 ? o.score : 0);    // global scores may be negative
        r.exon_score = r.score;
        const int32_t tn = static_cast<int32_t>(d.nt_len);
        if (!global && r.score <= 0) continue;
        const bool score_only = (d.flags & (PF_SCORE_ONLY | PF_BUDGET)) != 0;
        const int32_t en_al = o.best_ii + 1;
        r.prot_en = o.best_jj + 1;
        if (score_only) {
            r.prot_st = -1;
            if (d.strand > 0) { r.nt_st = -1; r.nt_en = en_al; }
            else { r.nt_st = tn - en_al; r.nt_en = -1; }
            continue;
        }
        r.prot_st = o.st_jj;
        if (d.strand > 0) { r.nt_st = o.st_ii; r.nt_en = en_al; }
        else { r.nt_st = tn - en_al; r.nt_en = tn - o.st_ii; }
        r.n_cigar = o.n_ops;
        r.cigar = o.n_ops ? c->host_cig.data() + o.cig_out : nullptr;
    }
    c->stats.n_rerun = nrerun;
    return MP_OK;
}

static int exon_rescore_impl(mp_dp_ctx *c, const mp_pair *pairs, size_t n, mp_result *res, const mp_dp_batch *src);

int mp_dp_align_batch(mp_dp_ctx *c, const mp_pair *pairs, size_t n, mp_result *out)
{
    if (!c || (n && (!pairs || !out))) return MP_EINVAL;
    // the context keeps one batch whose device buffers only grow, so repeated
    // calls allocate nothing once the largest batch has been seen
    if (!c->own) c->own = new (std::nothrow) mp_dp_batch();
    if (!c->own) return MP_ENOMEM;
    mp_dp_batch *b = c->own;
    int rc = upload_impl(c, b, pairs, n);
    if (rc != MP_OK) return rc;
    rc = mp_dp_batch_run(c, b);
    if (rc == MP_OK) rc = mp_dp_batch_sync(c);
    if (rc == MP_OK) rc = mp_dp_batch_download(c, b, out);
    if (rc == MP_OK && c->params.exon_rescore) rc = exon_rescore_impl(c, pairs, n, out, b);
    c->last = nullptr;
    return rc;
}

// The genome an alignment covers with its introns cut out, in the aligned
// orientation: codons and frameshift bases kept, an N intron dropped, a U or
// V intron dropped with the 3 bases of its split codon kept.  The host only
// walks the ops for the region's length (and checks that the walk stays in
// the region); the bases are gathered on the device (exon_gather_kernel).
static bool exon_walk(const mp_result &r, int64_t n, int64_t i0, uint64_t &len, bool &has_intron)
{
    int64_t i = i0;
    len = 0;
    has_intron = false;
    if (i < 0 || i > n) return false;
    auto take = [&](int64_t l) { i += l; len += static_cast<uint64_t>(l); return i <= n; };
    for (uint32_t k = 0; k < r.n_cigar; ++k) {
        const int64_t l = r.cigar[k] >> 4;
        bool ok = true;
        switch (r.cigar[k] & 0xf) {
        case MP_OP_M: case MP_OP_D: ok = take(3 * l); break;
        case MP_OP_I: break;
        case MP_OP_F: case MP_OP_G: ok = take(l); break;
        case MP_OP_N: i += l; has_intron = true; ok = i <= n; break;
        case MP_OP_U: ok = take(1); i += l; ok = ok && take(2); has_intron = true; break;
        case MP_OP_V: ok = take(2); i += l; ok = ok && take(1); has_intron = true; break;
        default: ok = false;
        }
        if (!ok) return false;
    }
    return true;
}

// src: the batch whose run produced res (its ASCII and compacted ops are
// still on the device), or null for results from elsewhere (their regions,
// proteins and ops are uploaded).
static int exon_rescore_impl(mp_dp_ctx *c, const mp_pair *pairs, size_t n, mp_result *res, const mp_dp_batch *src)
{
    if (c->server_running) return MP_ESTATE;
    std::vector<size_t> idx;
    std::vector<char> intron;
    std::vector<ExonJob> jobs;
    std::vector<mp_pair> sub;
    const uint32_t *hc = c->host_cig.data();
    const size_t hc_n = c->host_cig.size();
    for (size_t k = 0; k < n; ++k) {
        const mp_result &r = res[k];
        if (r.score <= 0 || !r.n_cigar || !r.cigar || (r.status & MP_ST_ERRMASK)) continue;
        const mp_pair &q = pairs[k];
        if (q.strand != 1 && q.strand != -1) continue;
        const int64_t nl = q.nt_len;
        const int64_t i0 = q.strand > 0 ? r.nt_st : nl - r.nt_en;
        uint64_t len = 0;
        bool has_intron = false;
        if (!exon_walk(r, nl, i0, len, has_intron) || len >= (1u << 20) - 1024) continue;
        ExonJob j{};
        j.src_nt_len = q.nt_len;
        j.n_ops = r.n_cigar;
        j.strand = q.strand;
        j.i0 = static_cast<int32_t>(i0);
        jobs.push_back(j);
        sub.push_back(mp_pair{q.prot, q.prot_len, nullptr, static_cast<uint32_t>(len), 1, MP_PAIR_SCORE_ONLY,
                              q.profile});
        idx.push_back(k);
        intron.push_back(has_intron ? 1 : 0);
    }
    if (idx.empty()) return MP_OK;
    // a source batch serves only if every result's ops lie in the context's
    // copy of that batch's compacted CIGARs
    bool resident = src != nullptr && src->n == n;
    for (size_t i = 0; resident && i < idx.size(); ++i) {
        const mp_result &r = res[idx[i]];
        resident = r.cigar >= hc && r.cigar + r.n_cigar <= hc + hc_n;
    }
    if (!c->aux) c->aux = new (std::nothrow) mp_dp_batch();
    if (!c->aux) return MP_ENOMEM;
    mp_dp_batch *b = c->aux;
    int rc = upload_impl(c, b, sub.data(), sub.size(), true);
    if (rc != MP_OK) return rc;
    // device buffer: [jobs][ops][ASCII of the source pairs] (the last two only
    // without a resident source), each part 16-byte aligned
    const size_t nj = jobs.size();
    const size_t jobs_bytes = div_up(nj * sizeof(ExonJob), 16) * 16;
    size_t ops_bytes = 0, asc_bytes = 0;
    if (resident) {
        for (size_t i = 0; i < nj; ++i) {
            const size_t k = idx[i];
            jobs[i].src_nt_off = src->desc[k].asc_nt_off;
            jobs[i].src_prot_off = src->desc[k].asc_prot_off;
            jobs[i].op_off = static_cast<uint64_t>(res[k].cigar - hc);
        }
    } else {
        uint64_t ops = 0, asc = 0;
        for (size_t i = 0; i < nj; ++i) {
            const size_t k = idx[i];
            jobs[i].op_off = ops;
            ops += res[k].n_cigar;
            jobs[i].src_prot_off = static_cast<uint32_t>(asc);
            asc += pairs[k].prot_len;
            jobs[i].src_nt_off = asc;
            asc += pairs[k].nt_len;
            asc = div_up(asc, 16) * 16;
        }
        if (asc > 0xffffffffull) return MP_EINVAL;
        ops_bytes = div_up(ops * sizeof(uint32_t), 16) * 16;
        asc_bytes = asc;
    }
    const size_t total = jobs_bytes + ops_bytes + asc_bytes;
    CK(staging_wait(c));
    if (c->staging.reserve(total + 16) != cudaSuccess || c->exbuf.reserve(total + 16) != cudaSuccess)
        return MP_ENOMEM;
    char *h = c->staging.p;
    memcpy(h, jobs.data(), nj * sizeof(ExonJob));
    if (!resident) {
        uint32_t *hops = reinterpret_cast<uint32_t *>(h + jobs_bytes);
        char *hasc = h + jobs_bytes + ops_bytes;
        for (size_t i = 0; i < nj; ++i) {
            const size_t k = idx[i];
            memcpy(hops + jobs[i].op_off, res[k].cigar, res[k].n_cigar * sizeof(uint32_t));
            const mp_pair &q = pairs[k];
            if (q.prot_len) memcpy(hasc + jobs[i].src_prot_off, q.prot, q.prot_len);
            if (q.nt_len) memcpy(hasc + jobs[i].src_nt_off, q.nt, q.nt_len);
        }
    }
    cudaStream_t st = c->stream;
    CK(cudaMemcpyAsync(c->exbuf.p, h, total, cudaMemcpyHostToDevice, st));
    const ExonJob *d_jobs = reinterpret_cast<const ExonJob *>(c->exbuf.p);
    const uint32_t *d_ops = resident ? src->cig.p : reinterpret_cast<const uint32_t *>(c->exbuf.p + jobs_bytes);
    const char *d_src = resident ? src->ascii.p : reinterpret_cast<const char *>(c->exbuf.p + jobs_bytes + ops_bytes);
    CK(launch_exon_gather(d_jobs, static_cast<uint32_t>(nj), b->d_desc.p, d_src, d_ops, b->ascii.p, st));
    rc = mp_dp_batch_run(c, b);
    if (rc != MP_OK) return rc;
    b->h_out.resize(nj);
    CK(cudaMemcpyAsync(b->h_out.data(), b->out.p, nj * sizeof(PairOut), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    for (size_t i = 0; i < nj; ++i) {
        const PairOut &o = b->h_out[i];
        if (o.status & MP_ST_ERRMASK) continue;
        const int32_t s2 = o.score > 0 ? o.score : 0;
        res[idx[i]].exon_score = s2 - (intron[i] ? 0 : c->params.r);
    }
    return MP_OK;
}

int mp_dp_exon_rescore(mp_dp_ctx *c, const mp_pair *pairs, size_t n, mp_result *res)
{
    if (!c || (n && (!pairs || !res))) return MP_EINVAL;
    return exon_rescore_impl(c, pairs, n, res, nullptr);
}

}  // extern "C"

// ================================================================ serving
// A serving thread turns submitted requests into micro-batches.  Each of
// n_slots slots owns a private context (stream, batch buffers) and, while
// busy, a range of one traceback arena of the whole budget: requests are
// admitted in arrival order into the next free slot, up to a slot's share
// of the budget (a larger request alone, once a range that large is free),
// and the slot's pipeline is enqueued at once, so batches formed while
// others are still on the device run concurrently with them (continuous
// batching).  The request queue is host memory: admission is a host
// decision taken as ranges free up, and everything a batch runs on (its
// arena range, sequences, plan and results) is on the device.
struct Slot {
    mp_dp_ctx *ctx = nullptr;
    mp_dp_batch *batch = nullptr;
    std::vector<uint64_t> tickets;
    std::vector<std::chrono::steady_clock::time_point> t_submit;
    std::vector<mp_result> res;
    bool busy = false;
    uint64_t off = 0, len = 0;          // the slot's range of the shared traceback arena while busy
};

// Traceback bytes a request may need, whichever strip form its run takes
// (0 for score-only requests).
static uint64_t request_bytes(const BoundTable &bt, const Request &r)
{
    if (r.flags & MP_PAIR_SCORE_ONLY) return 0;
    const uint32_t m = static_cast<uint32_t>(r.prot.size()), n = static_cast<uint32_t>(r.nt.size());
    const bool wide = (r.profile.empty() ? score_bound(bt, r.prot.data(), m, kOverflowT)
                                         : profile_score_bound(r.profile.data(), m)) >= kOverflowT;
    return div_up(std::max(code_bytes(m, n, wide, false), code_bytes(m, n, wide, !wide)), 256) * 256;
}

// Lowest offset of a free range of `len` bytes in [0, cap) beside the busy
// slots' ranges, or UINT64_MAX.
static uint64_t arena_fit(const std::vector<Slot> &slots, uint64_t cap, uint64_t len)
{
    std::vector<std::pair<uint64_t, uint64_t>> used;
    for (const Slot &s : slots)
        if (s.busy && s.len) used.push_back({s.off, s.off + s.len});
    std::sort(used.begin(), used.end());
    uint64_t at = 0;
    for (const auto &u : used) {
        if (u.first >= at + len) return at;
        at = std::max(at, u.second);
    }
    return at + len <= cap ? at : UINT64_MAX;
}

// Largest free range beside the busy slots' ranges.
static uint64_t arena_largest_gap(const std::vector<Slot> &slots, uint64_t cap)
{
    std::vector<std::pair<uint64_t, uint64_t>> used;
    for (const Slot &s : slots)
        if (s.busy && s.len) used.push_back({s.off, s.off + s.len});
    std::sort(used.begin(), used.end());
    uint64_t at = 0, best = 0;
    for (const auto &u : used) {
        if (u.first > at) best = std::max(best, u.first - at);
        at = std::max(at, u.second);
    }
    return std::max(best, cap > at ? cap - at : 0);
}

static void finish_slot(mp_dp_ctx *c, Slot &s, bool ok)
{
    if (ok && mp_dp_batch_download(s.ctx, s.batch, s.res.data()) != MP_OK) ok = false;
    {
        const auto now = std::chrono::steady_clock::now();
        std::lock_guard<std::mutex> lk(c->mu);
        for (size_t k = 0; k < s.tickets.size(); ++k) {
            c->latencies_ms.push_back(std::chrono::duration<float, std::milli>(now - s.t_submit[k]).count());
            Done d;
            if (ok) {
                d.r = s.res[k];
                d.cigar.assign(s.res[k].cigar, s.res[k].cigar + s.res[k].n_cigar);
            } else {
                memset(&d.r, 0, sizeof(d.r));
                d.r.status = MP_ST_TRACE;
            }
            d.r.cigar = nullptr;
            c->inflight.erase(s.tickets[k]);
            c->done.emplace(s.tickets[k], std::move(d));
            c->completed.push_back(s.tickets[k]);
        }
        c->served_batches += 1;
        c->served_pairs += s.tickets.size();
    }
    c->cv_done.notify_all();
    s.busy = false;
    s.len = 0;
    s.tickets.clear();
}

static void serve_loop(mp_dp_ctx *c)
{
    cudaSetDevice(c->device);
    std::vector<Slot> slots(c->n_slots);
    bool init_ok = true;
    for (auto &s : slots) {
        mp_dp_params p = c->params;
        p.tb_budget_bytes = c->budget;
        p.max_pairs_per_launch = 0;
        p.autotune = 0;
        if (mp_dp_init(&s.ctx, &p, c->device) != MP_OK) {
            init_ok = false;
            continue;
        }
        s.ctx->has_fixed = c->has_fixed;
        s.ctx->fixed = c->fixed;
        s.ctx->tuned = c->tuned;
    }
    // One traceback arena of the whole budget shared by the slots: a
    // micro-batch is admitted into a free range of it, so the slots' batches
    // together never hold more than the budget, and one request may take up
    // to all of it (it then waits until the other slots have drained).
    DevBuf<uint8_t> arena;
    if (init_ok && arena.reserve(std::max<uint64_t>(c->budget, 256)) != cudaSuccess) init_ok = false;
    std::vector<Request> take;
    for (;;) {
        bool progressed = false;
        // retire finished slots
        for (auto &s : slots) {
            if (s.busy && cudaStreamQuery(s.ctx->stream) != cudaErrorNotReady) {
                finish_slot(c, s, cudaStreamQuery(s.ctx->stream) == cudaSuccess);
                progressed = true;
            }
        }
        // admit queued requests into free slots
        const BoundTable bt(c->sp);
        for (auto &s : slots) {
            if (s.busy) continue;
            take.clear();
            uint64_t bytes = 0;
            {
                std::lock_guard<std::mutex> lk(c->mu);
                // requests in arrival order, up to a slot's share of the budget
                // (or the first request alone, if larger), within the largest
                // free range of the arena; the head of the queue waits while
                // it does not fit
                const uint64_t room = arena_largest_gap(slots, c->budget);
                while (!c->queue.empty()) {
                    const Request &r = c->queue.front();
                    const uint64_t cb = request_bytes(bt, r);
                    const uint64_t cap = std::min(room, take.empty() ? std::max(cb, c->slot_budget) : c->slot_budget);
                    if (bytes + cb > cap) break;
                    bytes += cb;
                    take.push_back(std::move(c->queue.front()));
                    c->queue.pop_front();
                }
            }
            if (take.empty()) break;
            s.len = std::max<uint64_t>(bytes, 256);
            s.off = arena_fit(slots, c->budget, s.len);
            std::vector<mp_pair> pairs(take.size());
            for (size_t k = 0; k < take.size(); ++k) {
                pairs[k].prot = take[k].prot.data();
                pairs[k].prot_len = static_cast<uint32_t>(take[k].prot.size());
                pairs[k].nt = take[k].nt.data();
                pairs[k].nt_len = static_cast<uint32_t>(take[k].nt.size());
                pairs[k].strand = take[k].strand;
                pairs[k].flags = take[k].flags;
                pairs[k].profile = take[k].profile.empty() ? nullptr : take[k].profile.data();
            }
            s.tickets.clear();
            s.t_submit.clear();
            for (auto &r : take) {
                s.tickets.push_back(r.ticket);
                s.t_submit.push_back(r.t_submit);
            }
            s.res.assign(take.size(), mp_result{});
            // the slot's batch keeps its device buffers from one micro-batch to the next
            if (!s.batch) s.batch = new (std::nothrow) mp_dp_batch();
            bool ok = init_ok && s.off != UINT64_MAX;
            if (ok) {
                s.ctx->codes_ext = arena.p + s.off;
                s.ctx->codes_ext_cap = s.len;
                s.ctx->budget = s.len;
            }
            ok = ok && s.batch && upload_impl(s.ctx, s.batch, pairs.data(), pairs.size()) == MP_OK;
            if (ok) ok = mp_dp_batch_run(s.ctx, s.batch) == MP_OK;
            s.busy = true;
            if (!ok) finish_slot(c, s, false);
            progressed = true;
        }
        if (!progressed) {
            std::unique_lock<std::mutex> lk(c->mu);
            bool any_busy = false;
            for (auto &s : slots) any_busy |= s.busy;
            if (c->stopping && !any_busy && c->queue.empty()) break;
            if (any_busy) {
                lk.unlock();
                std::this_thread::sleep_for(std::chrono::microseconds(20));
            } else {
                c->cv_req.wait_for(lk, std::chrono::milliseconds(5),
                                   [&] { return !c->queue.empty() || c->stopping; });
            }
        }
    }
    for (auto &s : slots) {
        if (s.batch) mp_dp_batch_free(s.ctx, s.batch);
        if (s.ctx) mp_dp_destroy(s.ctx);
    }
    arena.release();
}

extern "C" int mp_dp_submit(mp_dp_ctx *c, const mp_pair *q, uint64_t *ticket)
{
    if (!c || !q || !ticket) return MP_EINVAL;
    if ((q->prot_len && !q->prot) || (q->nt_len && !q->nt) || (q->strand != 1 && q->strand != -1))
        return MP_EINVAL;
    std::unique_lock<std::mutex> lk(c->mu);
    if (c->slot_budget == 0) c->slot_budget = c->budget / static_cast<uint64_t>(c->n_slots);
    const BoundTable bt(c->sp);
    Request r;
    r.prot.assign(q->prot, q->prot_len);
    r.nt.assign(q->nt, q->nt_len);
    r.flags = q->flags;
    if (q->profile) r.profile.assign(q->profile, q->profile + q->prot_len + 1);
    // a request is served if its traceback fits the whole budget
    if (request_bytes(bt, r) > c->budget) return MP_EBUDGET;
    if (c->stopping) return MP_ESTATE;
    if (c->queue.size() >= c->ring_cap) return MP_EAGAIN;
    r.ticket = c->next_ticket++;
    r.strand = q->strand;
    r.t_submit = std::chrono::steady_clock::now();
    *ticket = r.ticket;
    c->inflight.insert(r.ticket);
    c->queue.push_back(std::move(r));
    if (!c->server_running) {
        c->server_running = true;
        c->server = std::thread(serve_loop, c);
    }
    lk.unlock();
    c->cv_req.notify_one();
    return MP_OK;
}

// Hand out a finished result; the caller holds c->mu.
static int deliver(mp_dp_ctx *c, uint64_t ticket, mp_result *out)
{
    auto it = c->done.find(ticket);
    if (it == c->done.end()) return MP_ETICKET;
    Done &d = it->second;
    if (d.delivered) {
        c->done.erase(it);
        return MP_ETICKET;
    }
    d.delivered = true;
    *out = d.r;
    out->cigar = d.cigar.empty() ? nullptr : d.cigar.data();
    return MP_OK;
}

extern "C" int mp_dp_poll(mp_dp_ctx *c, uint64_t ticket, mp_result *out, int64_t timeout_us)
{
    if (!c || !out) return MP_EINVAL;
    std::unique_lock<std::mutex> lk(c->mu);
    if (c->done.count(ticket)) return deliver(c, ticket, out);
    if (!c->inflight.count(ticket)) return MP_ETICKET;
    if (timeout_us == 0) return MP_EPENDING;
    auto ready = [&] { return c->done.count(ticket) > 0 || c->stopping; };
    if (timeout_us < 0) c->cv_done.wait(lk, ready);
    else c->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), ready);
    if (!c->done.count(ticket)) return MP_ETIMEOUT;
    return deliver(c, ticket, out);
}

extern "C" int mp_dp_wait_any(mp_dp_ctx *c, uint64_t *ticket, mp_result *out, int64_t timeout_us)
{
    if (!c || !ticket || !out) return MP_EINVAL;
    std::unique_lock<std::mutex> lk(c->mu);
    auto pick = [&]() -> bool {
        while (!c->completed.empty()) {
            const uint64_t t = c->completed.front();
            c->completed.pop_front();
            auto it = c->done.find(t);
            if (it != c->done.end() && !it->second.delivered) {
                *ticket = t;
                return true;
            }
        }
        return false;
    };
    if (pick()) return deliver(c, *ticket, out);
    if (timeout_us == 0) return MP_EPENDING;
    auto ready = [&] { return !c->completed.empty() || c->stopping; };
    if (timeout_us < 0) c->cv_done.wait(lk, ready);
    else c->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), ready);
    if (pick()) return deliver(c, *ticket, out);
    return MP_ETIMEOUT;
}

extern "C" int mp_dp_get_serve_stats(mp_dp_ctx *c, mp_dp_serve_stats *out, int reset)
{
    if (!c || !out) return MP_EINVAL;
    std::lock_guard<std::mutex> lk(c->mu);
    memset(out, 0, sizeof(*out));
    std::vector<float> v = c->latencies_ms;
    out->completed = v.size();
    out->batches = c->served_batches;
    out->mean_batch_pairs = c->served_batches ? static_cast<double>(c->served_pairs) / c->served_batches : 0.0;
    if (!v.empty()) {
        std::sort(v.begin(), v.end());
        auto q = [&](double f) { return static_cast<double>(v[std::min(v.size() - 1, static_cast<size_t>(f * v.size()))]); };
        out->p50_ms = q(0.50);
        out->p99_ms = q(0.99);
        out->max_ms = v.back();
    }
    if (reset) {
        c->latencies_ms.clear();
        c->served_batches = 0;
        c->served_pairs = 0;
    }
    return MP_OK;
}

extern "C" void mp_dp_destroy(mp_dp_ctx *c)
{
    if (!c) return;
    {
        std::lock_guard<std::mutex> lk(c->mu);
        c->stopping = true;
    }
    c->cv_req.notify_all();
    c->cv_done.notify_all();
    if (c->server.joinable()) c->server.join();
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    if (c->own) mp_dp_batch_free(c, c->own);
    if (c->aux) mp_dp_batch_free(c, c->aux);
    c->aux = nullptr;
    c->own = nullptr;
    c->codes.release();
    c->staging.release();
    c->pstaging.release();
    c->exbuf.release();
    c->d_mat.release();
    if (c->stream2) cudaStreamSynchronize(c->stream2);
    if (c->ev_staging) cudaEventDestroy(c->ev_staging);
    if (c->stream) cudaStreamDestroy(c->stream);
    if (c->stream2) cudaStreamDestroy(c->stream2);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    delete c;
}
