// lbm_api.cu -- host side of the C ABI declared in include/lbm.h.
//
// Owns the device state of one chip (see lbm_internal.h for the layout),
// validates every argument before touching the device, builds the wall-link
// table, the per-row port table and the list of fluid tiles, and issues the
// kernels on the handle's stream.  No call here computes any part of the
// time step on the host.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "lbm.h"
#include "lbm_internal.h"

namespace {

thread_local std::string g_create_error = "no error";

constexpr uint32_t kStateMagic = 0x4C424D31u;  // "LBM1"
constexpr int kMaxPorts = 64;
constexpr int kMaxSchedule = 4096;
constexpr int kMaxInstances = 4096;
constexpr int kMaxBlocksPerSM = 32;  // resident blocks per SM, an upper bound for every launch shape
constexpr int kMaxGraphs = 16;       // cached CUDA graphs per handle
constexpr int kMaxGraphSteps = 4096;
// Bulk-copy pipeline shape measured fastest on GB300 for the 4096 x 2048 chip:
// three computing warps with one stage each, four blocks per SM.
constexpr int kDefaultConsumers = 3;
constexpr int kDefaultStagesPerConsumer = 1;
constexpr int kDefaultStagesPerConsumer16 = 2;  // 16-bit stages are half as large
constexpr int kDefaultPipeWarps = 4;
constexpr int kDefaultRegsBlock = 128;
constexpr int kScalarConsumers = 3;   // scalar-only step: computing warps per block
constexpr int kScalarStagesPer = 3;   // and shared-memory stages per computing warp
constexpr int kScalarRegsBlock = 128; // scalar-only step, register variant: threads per block
constexpr int kMaxMultiStep = 65536;  // steps per cooperative launch

struct Alloc {
    void* ptr = nullptr;
    size_t bytes = 0;
};

}  // namespace

struct lbm_ctx {
    int nx = 0, ny = 0, pitch = 0, segs = 0;
    long long plane = 0;
    double tau = 0, tau_c = 0, w0 = 0, rho0 = 1, C0 = 0;
    float wg0 = 0, wg1 = 0, inv_cs2g = 0;
    int device = 0;
    cudaStream_t stream = nullptr;
    lbm_alloc_fn alloc_fn = nullptr;
    lbm_free_fn free_fn = nullptr;
    void* alloc_user = nullptr;

    std::vector<Alloc> allocs;
    // The two state buffers.  They hold elements of `precision` (FP32, or
    // 16-bit for FP16 / BF16 storage); the float type serves FP32 paths.
    float* pop[2] = {nullptr, nullptr};
    int precision = lbm::kFP32;
    size_t elem = sizeof(float);
    int cur = 0;   // buffer holding the current state
    int gbuf = 0;  // buffer holding the current scalar planes: cur, except after
                   // an odd number of scalar-only steps (joined lazily)
    uint8_t* links = nullptr;
    lbm::RowBC* rowbc = nullptr;
    uint2* tiles = nullptr;
    uint2* tiles64 = nullptr;  // the same row segments in 64-node halves (variant 5)
    float2* partials = nullptr;  // per-block diagnostics partials, double-float pairs
    double* diag = nullptr;       // 4 totals formed by lbm_get_diagnostics
    unsigned int* err = nullptr;
    float* fields_tmp = nullptr;  // 4 * nx * ny floats

    int n_tiles = 0;
    int n_tiles64 = 0;
    int n_plain = 0;  // 16-bit storage: tiles without a port node, listed first in the tile table
    // both tile tables in row order (port tiles flagged), from which the
    // device tables are ordered for the launch shape (arrange_tiles)
    std::vector<uint2> tiles_rows, tiles64_rows;
    std::vector<uint2> tiles_order, tiles64_order;  // the orders last copied to the device
    int sms = 0;
    int partials_cap = 0;  // blocks the partials buffer holds (any launch shape fits)
    int diag_grid = 0;     // blocks whose partials the last step wrote
    int scalar_grid = 0;  // one wave of the scalar-only step kernel (set on first use)
    bool scalar_regs = true;  // scalar-only step: register variant (else the bulk-copy pipeline)
    int multi_step = 0;           // lbm_step: steps per cooperative launch (0 = one launch per step)
    int coop_grid = 0;            // blocks of that launch (all resident)
    unsigned* bar = nullptr;      // its grid-barrier count
    unsigned barrier_extra = 0;   // test hook (lbm_debug_barrier_extra)
    lbm::StepLaunch launch{lbm::kVariantBulk, 0, 0, 0};
    long long fluid = 0;
    long long device_bytes = 0;

    int64_t step = 0;
    uint32_t fixed_mask = 0;
    int64_t period = 0;
    std::vector<uint32_t> schedule;

    // Batches of chips (lbm_create_batch): instance k occupies rows
    // [row0, row0 + ny) and columns [0, nx) of the stacked lattice, with its
    // channels c at lattice channels chan_base + c and its own valve program.
    struct Inst {
        int row0, nx, ny, chan_base, n_chan;
        double tau, tau_c;
        uint32_t fixed_mask;
        int64_t period;
        std::vector<uint32_t> schedule;
        uint32_t word_at(int64_t t) const
        {
            if (!schedule.empty()) return schedule[size_t((t / period) % int64_t(schedule.size()))];
            return fixed_mask;
        }
    };
    std::vector<Inst> inst;  // empty for a single chip
    float4* rates = nullptr; // per-row relaxation rates of a batch

    // CUDA graphs of graph_steps consecutive step launches, one per valve
    // words and starting buffer, captured on a private stream.
    struct Graph {
        uint32_t words[lbm::kMaskWords];
        int parity;
        cudaGraphExec_t exec;
    };
    int graph_steps = 0;
    cudaStream_t cap_stream = nullptr;
    float decay = 0.f;         // k of the reaction term R = -k C
    int wall_scheme = 0;       // LBM_WALL_BOUNCE_BACK or LBM_WALL_EQUILIBRIUM
    void* wallv = nullptr;     // the paper's walls: 8 planes of wall values for the step
    long long* woff = nullptr; // offsets of the fluid nodes with wall links
    int n_wall = 0;
    bool paper_ports = false;  // some port has a rescaling kind (no adjoint)
    std::vector<Graph> graphs;

    // Whether the valve words stay the same over steps [t0, t0 + len).
    bool mask_constant(int64_t t0, int64_t len) const
    {
        auto same = [&](int64_t period, size_t n) {
            return n <= 1 || t0 / period == (t0 + len - 1) / period;
        };
        if (inst.empty()) return schedule.empty() || same(period, schedule.size());
        for (const Inst& k : inst)
            if (!k.schedule.empty() && !same(k.period, k.schedule.size())) return false;
        return true;
    }
    bool numeric = false;  // the device error word was found set (bit 0)
    bool timeout = false;  // a bounded device wait gave up (bit 1)

    std::string last_error = "no error";
    std::vector<uint8_t> solid;  // host copy of the mask (non-zero = solid)
    struct Field {
        uint32_t word;
        float* u;                    // 2 planes (u_x, u_y) of ny x pitch floats
    };
    std::vector<Field> fields;       // stored velocity fields, one per valve word

    // The longest run of steps from t0, at most max_len, over which no valve
    // word changes (mask_constant holds for it).
    int64_t mask_run(int64_t t0, int64_t max_len) const
    {
        int64_t len = max_len;
        auto lim = [&](int64_t per, size_t n) {
            if (n > 1) len = std::min(len, per - t0 % per);
        };
        if (inst.empty()) lim(period, schedule.size());
        for (const Inst& k : inst) lim(k.period, k.schedule.size());
        return len;
    }

    uint32_t mask_at(int64_t t) const
    {
        if (!schedule.empty())
            return schedule[size_t((t / period) % int64_t(schedule.size()))];
        return fixed_mask;
    }

    // Valve bits of every lattice channel at step t.
    void mask_words(int64_t t, uint32_t (&w)[lbm::kMaskWords]) const
    {
        for (int j = 0; j < lbm::kMaskWords; ++j) w[j] = 0;
        if (inst.empty()) {
            w[0] = mask_at(t);
            return;
        }
        for (const Inst& k : inst) {
            const uint64_t bits = uint64_t(k.word_at(t)) & ((k.n_chan >= 32 ? 0xFFFFFFFFull : (1ull << k.n_chan) - 1));
            const uint64_t sh = bits << (k.chan_base & 31);
            w[k.chan_base >> 5] |= uint32_t(sh);
            if ((k.chan_base >> 5) + 1 < lbm::kMaskWords) w[(k.chan_base >> 5) + 1] |= uint32_t(sh >> 32);
        }
    }
};

namespace {

// A named range on the host timeline for the duration of a library call (or
// a phase of one), for profilers that read NVTX; with none attached a range
// costs a test and a branch.
struct Range {
    explicit Range(const char* name) { nvtxRangePushA(name); }
    ~Range() { end(); }
    void end()
    {
        if (open) nvtxRangePop();
        open = false;
    }
    Range(const Range&) = delete;
    Range& operator=(const Range&) = delete;
    bool open = true;
};

lbm_status fail(lbm_ctx* h, lbm_status s, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (h) h->last_error = buf;
    else g_create_error = buf;
    return s;
}

lbm_status cuda_fail(lbm_ctx* h, cudaError_t e, const char* what)
{
    return fail(h, e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA, "%s: %s", what,
                cudaGetErrorString(e));
}

#define LBM_CUDA(h, call)                                       \
    do {                                                        \
        cudaError_t e_ = (call);                                \
        if (e_ != cudaSuccess) return cuda_fail((h), e_, #call); \
    } while (0)

// A caller's allocator must return 256-byte aligned memory (the kernels
// use 16-byte vector accesses); anything else is handed back and counts as
// a failed allocation, so no kernel ever sees a misaligned buffer.
void* hook_alloc(lbm_ctx* h, size_t bytes)
{
    void* p = h->alloc_fn(bytes, h->alloc_user);
    if (p && (reinterpret_cast<uintptr_t>(p) & 255u)) {
        if (h->free_fn) h->free_fn(p, bytes, h->alloc_user);
        p = nullptr;
    }
    return p;
}

void* dev_alloc(lbm_ctx* h, size_t bytes)
{
    bytes = (bytes + 255) & ~size_t(255);
    void* p = nullptr;
    if (h->alloc_fn) {
        p = hook_alloc(h, bytes);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    if (p) {
        h->allocs.push_back({p, bytes});
        h->device_bytes += (long long)bytes;
    }
    return p;
}

void free_all(lbm_ctx* h)
{
    for (auto& g : h->graphs) cudaGraphExecDestroy(g.exec);
    h->graphs.clear();
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    h->cap_stream = nullptr;
    for (auto& a : h->allocs) {
        if (h->free_fn) h->free_fn(a.ptr, a.bytes, h->alloc_user);
        else cudaFree(a.ptr);
    }
    h->allocs.clear();
}

bool is_fluid(const uint8_t* mask, int nx, int ny, int x, int y)
{
    return x >= 0 && x < nx && y >= 0 && y < ny && mask[size_t(y) * nx + x] == 0;
}

// One step: the paper's wall values first (when that wall scheme is on),
// then the step kernel.
cudaError_t launch_full_step(const lbm_ctx* h, const lbm::StepArgs& a, const lbm::StepLaunch& L, cudaStream_t s)
{
    if (h->wallv) {
        cudaError_t e = lbm::launch_wall_values(a.src, h->wallv, h->links, h->woff, h->n_wall, h->plane, h->pitch,
                                                h->precision, s);
        if (e != cudaSuccess) return e;
    }
    return lbm::launch_step(a, L, s);
}

// The cached graph of graph_steps launches for the valve words in
// a.open_mask starting from buffer cur, captured on first use.
lbm_status step_graph(lbm_ctx* h, lbm::StepArgs a, cudaGraphExec_t* out)
{
    for (auto& g : h->graphs)
        if (g.parity == h->cur && std::memcmp(g.words, a.open_mask, sizeof(g.words)) == 0) {
            *out = g.exec;
            return LBM_OK;
        }
    if (int(h->graphs.size()) >= kMaxGraphs) {  // keep the cache small: start over
        LBM_CUDA(h, cudaStreamSynchronize(h->stream));
        for (auto& g : h->graphs) cudaGraphExecDestroy(g.exec);
        h->graphs.clear();
    }
    LBM_CUDA(h, cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    for (int j = 0; j < h->graph_steps && e == cudaSuccess; ++j) {
        a.src = h->pop[(h->cur + j) & 1];
        a.dst = h->pop[(h->cur + j + 1) & 1];
        a.reverse = (h->cur + j) & 1;
        e = launch_full_step(h, a, h->launch, h->cap_stream);
    }
    cudaGraph_t graph = nullptr;
    const cudaError_t e_end = cudaStreamEndCapture(h->cap_stream, &graph);
    if (e == cudaSuccess) e = e_end;
    cudaGraphExec_t exec = nullptr;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(h, e, "step graph capture");
    lbm_ctx::Graph g;
    std::memcpy(g.words, a.open_mask, sizeof(g.words));
    g.parity = h->cur;
    g.exec = exec;
    h->graphs.push_back(g);
    *out = exec;
    return LBM_OK;
}

// A tile list ordered for a kernel whose warps take entries w, w + G,
// w + 2G, ... (counted from either end of the table: the steps alternate).
// With n tiles the warps w < r = n - (k - 1) G take k = ceil(n / G) tiles
// and the others k - 1, and the entries of the first group are the same set
// counted from either end.  The tiles that hold a port node take longer, so
// they go to entries of the warps with fewer tiles; the other tiles keep
// their row order in the remaining entries.
std::vector<uint2> order_for_warps(const std::vector<uint2>& rows, long long G)
{
    const long long n = (long long)rows.size();
    if (G <= 0 || n <= G || n % G == 0) return rows;
    const long long k = (n + G - 1) / G, r = n - (k - 1) * G;
    std::vector<char> longer(static_cast<size_t>(n), 0);  // entry of a warp that takes k tiles
    for (long long w = 0; w < r; ++w)
        for (long long j = 0; j < k; ++j) longer[size_t(w + j * G)] = 1;
    std::vector<uint2> out(static_cast<size_t>(n));
    std::vector<char> used(static_cast<size_t>(n), 0);
    long long p = 0, placed = 0;  // next entry for a port tile (the short warps' first); port tiles placed
    for (const uint2& t : rows) {
        if (!(t.y & lbm::kPortTile)) continue;
        while (p < n && longer[size_t(p)]) ++p;
        if (p >= n) break;  // more port tiles than short entries: the rest go with the plain tiles
        out[size_t(p)] = t;
        used[size_t(p++)] = 1;
        ++placed;
    }
    long long q = 0, skipped = 0;
    for (const uint2& t : rows) {
        if ((t.y & lbm::kPortTile) && skipped < placed) {
            ++skipped;
            continue;
        }
        while (used[size_t(q)]) ++q;
        out[size_t(q)] = t;
        used[size_t(q++)] = 1;
    }
    return out;
}

// Copy both tile tables to the device in the order the launch shape L wants:
// 16-bit storage lists the port tiles last (the register kernels give them
// blocks of their own, n_plain); FP32 register kernels (variants 1, 4) and
// variant 5 put them on the warps with fewer tiles (order_for_warps).
cudaError_t arrange_tiles(lbm_ctx* h, const lbm::StepLaunch& L)
{
    const long long G = (long long)L.grid * (L.block / 32);
    if (h->precision != LBM_FP32) {
        h->tiles_order = h->tiles_rows;
        h->n_plain = int(std::stable_partition(h->tiles_order.begin(), h->tiles_order.end(),
                                               [](const uint2& t) { return !(t.y & lbm::kPortTile); }) -
                         h->tiles_order.begin());
    } else {
        const bool regs = L.variant == lbm::kVariantRegs || L.variant == lbm::kVariantAsync;
        h->tiles_order = regs ? order_for_warps(h->tiles_rows, G) : h->tiles_rows;
        h->n_plain = 0;
    }
    h->tiles64_order = L.variant == lbm::kVariantPairs ? order_for_warps(h->tiles64_rows, G) : h->tiles64_rows;
    cudaError_t e = cudaSuccess;
    if (!h->tiles_order.empty())
        e = cudaMemcpyAsync(h->tiles, h->tiles_order.data(), h->tiles_order.size() * sizeof(uint2),
                            cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess && !h->tiles64_order.empty())
        e = cudaMemcpyAsync(h->tiles64, h->tiles64_order.data(), h->tiles64_order.size() * sizeof(uint2),
                            cudaMemcpyHostToDevice, h->stream);
    return e;
}

// One wave of resident blocks, which then stride over the tile table.
int wave_grid(const lbm_ctx* h, const lbm::StepLaunch& L, int per_sm)
{
    const int tiles_per_block = L.variant == lbm::kVariantBulk ? 1 : L.block / 32;  // tiles in flight at once
    const int tiles = L.variant == lbm::kVariantPairs ? h->n_tiles64 : h->n_tiles;
    const int need = (tiles + tiles_per_block - 1) / tiles_per_block;
    return std::max(1, std::min(need, per_sm * h->sms));
}

// What lbm_create_batch adds to a stacked lattice.
struct BatchSpec {
    std::vector<lbm_ctx::Inst> inst;
    std::vector<float4> rates;  // one per lattice row
};

lbm_status check_ctx(lbm_ctx* h)
{
    if (!h) return LBM_ERR_ARG;
    return LBM_OK;
}

// Bring the scalar planes back next to the fluid planes after scalar-only
// steps left them in the other buffer (one device copy of 5 planes).
lbm_status join_scalar(lbm_ctx* h)
{
    if (h->gbuf == h->cur) return LBM_OK;
    const size_t off = size_t(9) * h->plane * h->elem;
    char* to = reinterpret_cast<char*>(h->pop[h->cur]) + off;
    const char* from = reinterpret_cast<const char*>(h->pop[h->gbuf]) + off;
    LBM_CUDA(h, cudaMemcpyAsync(to, from, size_t(5) * h->plane * h->elem, cudaMemcpyDeviceToDevice, h->stream));
    h->gbuf = h->cur;
    return LBM_OK;
}

lbm_status pending_numeric(lbm_ctx* h)
{
    return h->timeout ? LBM_ERR_TIMEOUT : h->numeric ? LBM_ERR_NUMERIC : LBM_OK;
}

}  // namespace

extern "C" {

void lbm_default_options(lbm_options* opt)
{
    if (!opt) return;
    std::memset(opt, 0, sizeof(*opt));
    opt->struct_size = sizeof(lbm_options);
    opt->device = -1;
    opt->w0 = 1.0 / 3.0;
    opt->rho0 = 1.0;
    opt->C0 = 0.0;
}

const char* lbm_status_string(lbm_status s)
{
    switch (s) {
    case LBM_OK: return "LBM_OK";
    case LBM_ERR_ARG: return "LBM_ERR_ARG";
    case LBM_ERR_CUDA: return "LBM_ERR_CUDA";
    case LBM_ERR_OOM: return "LBM_ERR_OOM";
    case LBM_ERR_NUMERIC: return "LBM_ERR_NUMERIC";
    case LBM_ERR_TIMEOUT: return "LBM_ERR_TIMEOUT";
    case LBM_ERR_STATE: return "LBM_ERR_STATE";
    }
    return "LBM_ERR_UNKNOWN";
}

const char* lbm_last_error(lbm_handle h)
{
    return h ? h->last_error.c_str() : g_create_error.c_str();
}

}  // extern "C"

namespace {
lbm_status create_impl(lbm_handle* out, int32_t nx, int32_t ny, const uint8_t* mask, double tau, double tau_c,
                       int32_t n_ports, const lbm_port* ports, const float* edge_u, const float* edge_C,
                       const lbm_options* opt_in, const BatchSpec* batch)
{
    if (!out) return fail(nullptr, LBM_ERR_ARG, "out is NULL");
    *out = nullptr;
    lbm_options opt;
    lbm_default_options(&opt);
    if (opt_in) {
        if (opt_in->struct_size != sizeof(lbm_options))
            return fail(nullptr, LBM_ERR_ARG, "lbm_options.struct_size is %u, expected %zu",
                        opt_in->struct_size, sizeof(lbm_options));
        opt = *opt_in;
    }
    // ---- argument checks (no device call before they pass) ----
    if (nx < 1 || ny < 1) return fail(nullptr, LBM_ERR_ARG, "grid %d x %d is empty", nx, ny);
    if (ny >= lbm::kMaxRows || nx > lbm::kMaxCols)
        return fail(nullptr, LBM_ERR_ARG, "grid %d x %d is too large", nx, ny);
    if (!mask) return fail(nullptr, LBM_ERR_ARG, "mask is NULL");
    if (!(tau > 0.5) || !std::isfinite(tau))
        return fail(nullptr, LBM_ERR_ARG, "tau = %g: the fluid relaxation time must exceed 1/2", tau);
    if (!(tau_c > 0.5) || !std::isfinite(tau_c))
        return fail(nullptr, LBM_ERR_ARG, "tau_c = %g: the scalar relaxation time must exceed 1/2", tau_c);
    if (!(opt.w0 >= 0.0 && opt.w0 < 1.0))
        return fail(nullptr, LBM_ERR_ARG, "w0 = %g outside [0, 1)", opt.w0);
    if (!(opt.rho0 > 0.0) || !std::isfinite(opt.rho0) || !std::isfinite(opt.C0))
        return fail(nullptr, LBM_ERR_ARG, "initial rho0 = %g, C0 = %g invalid", opt.rho0, opt.C0);
    if (opt.block_threads != 0 &&
        (opt.block_threads < 64 || opt.block_threads > 256 || opt.block_threads % 32 != 0))
        return fail(nullptr, LBM_ERR_ARG, "block_threads = %d: use 0 or a multiple of 32 in [64, 256]",
                    opt.block_threads);
    if (opt.max_blocks < 0) return fail(nullptr, LBM_ERR_ARG, "max_blocks = %d < 0", opt.max_blocks);
    if (opt.variant < 0 || opt.variant > 5)
        return fail(nullptr, LBM_ERR_ARG, "variant = %d: use 0, 1, 2, 3, 4 or 5", opt.variant);
    if (opt.variant == 5 && (opt.precision != LBM_FP32 || opt.wall_scheme != LBM_WALL_BOUNCE_BACK))
        return fail(nullptr, LBM_ERR_ARG, "variant 5 needs FP32 storage and bounce-back walls");
    if (opt.variant == 5 && opt.block_threads > 128)
        return fail(nullptr, LBM_ERR_ARG, "block_threads = %d: variant 5 runs blocks of 64 or 128 threads",
                    opt.block_threads);
    if (opt.precision != LBM_FP32 && opt.precision != LBM_FP16 && opt.precision != LBM_BF16)
        return fail(nullptr, LBM_ERR_ARG, "precision = %d: use LBM_FP32, LBM_FP16 or LBM_BF16", opt.precision);
    if (opt.precision != LBM_FP32 && opt.variant == 3)
        return fail(nullptr, LBM_ERR_ARG, "precision = %d: 16-bit storage runs variants 1, 2 and 4, not 3",
                    opt.precision);
    const int max_cw = opt.variant == 3 ? 8 : 7;
    if (opt.consumer_warps < 0 || opt.consumer_warps > max_cw)
        return fail(nullptr, LBM_ERR_ARG, "consumer_warps = %d: use 0 or 1..%d", opt.consumer_warps, max_cw);
    {
        const int nc = opt.consumer_warps ? opt.consumer_warps
                                          : opt.variant == 3 ? kDefaultPipeWarps : kDefaultConsumers;
        const int per = opt.pipeline_stages                ? opt.pipeline_stages
                        : opt.precision == LBM_FP32 ? kDefaultStagesPerConsumer
                                                    : kDefaultStagesPerConsumer16;
        if (opt.pipeline_stages < 0 || nc * per > lbm::kMaxStages)
            return fail(nullptr, LBM_ERR_ARG,
                        "pipeline_stages = %d per consumer warp with %d consumer warps: the ring holds at most %d stages",
                        opt.pipeline_stages, nc, lbm::kMaxStages);
    }
    if ((opt.alloc == nullptr) != (opt.free == nullptr))
        return fail(nullptr, LBM_ERR_ARG, "alloc and free hooks must be given together");
    if (opt.wall_scheme != LBM_WALL_BOUNCE_BACK && opt.wall_scheme != LBM_WALL_EQUILIBRIUM)
        return fail(nullptr, LBM_ERR_ARG, "wall_scheme = %d: use LBM_WALL_BOUNCE_BACK or LBM_WALL_EQUILIBRIUM",
                    opt.wall_scheme);
    if (opt.wall_scheme == LBM_WALL_EQUILIBRIUM && opt.variant == 4)
        return fail(nullptr, LBM_ERR_ARG, "wall_scheme = LBM_WALL_EQUILIBRIUM runs variants 1 and 2, not 4");
    if (opt.wall_scheme == LBM_WALL_EQUILIBRIUM && opt.variant == 3)
        return fail(nullptr, LBM_ERR_ARG, "wall_scheme = LBM_WALL_EQUILIBRIUM runs variants 1 and 2, not 3");
    if (!(opt.decay >= 0.0 && opt.decay < 1.0))
        return fail(nullptr, LBM_ERR_ARG, "decay = %g outside [0, 1)", opt.decay);
    if (opt.multi_step < 0 || opt.multi_step > kMaxMultiStep)
        return fail(nullptr, LBM_ERR_ARG, "multi_step = %d outside [0, %d]", opt.multi_step, kMaxMultiStep);
    if (opt.multi_step > 0 && (opt.precision != LBM_FP32 || opt.wall_scheme != LBM_WALL_BOUNCE_BACK))
        return fail(nullptr, LBM_ERR_ARG, "multi_step needs FP32 storage and bounce-back walls");
    if (opt.scalar_variant < 0 || opt.scalar_variant > 2)
        return fail(nullptr, LBM_ERR_ARG, "scalar_variant = %d outside [0, 2]", opt.scalar_variant);
    if (opt.graph_steps < 0 || opt.graph_steps % 2 != 0 || opt.graph_steps > kMaxGraphSteps)
        return fail(nullptr, LBM_ERR_ARG, "graph_steps = %d: use 0 or an even number up to %d", opt.graph_steps,
                    kMaxGraphSteps);
    const int max_ports = batch ? kMaxPorts * int(batch->inst.size()) : kMaxPorts;
    const int max_channel = batch ? 32 * lbm::kMaskWords - 1 : 31;
    if (n_ports < 0 || n_ports > max_ports)
        return fail(nullptr, LBM_ERR_ARG, "n_ports = %d outside [0, %d]", n_ports, max_ports);
    if (n_ports > 0 && !ports) return fail(nullptr, LBM_ERR_ARG, "ports is NULL");

    std::vector<lbm::RowBC> rowbc(size_t(2) * ny, lbm::RowBC{-1, 0, 0.f, 0.f});
    bool any_velocity = false, any_inlet = false;
    for (int p = 0; p < n_ports; ++p) {
        const lbm_port& P = ports[p];
        if (P.channel < 0 || P.channel > max_channel)
            return fail(nullptr, LBM_ERR_ARG, "port %d: channel %d outside [0, %d]", p, P.channel, max_channel);
        if (P.side != LBM_WEST && P.side != LBM_EAST)
            return fail(nullptr, LBM_ERR_ARG, "port %d: side %d invalid", p, P.side);
        if (P.kind < LBM_PORT_VELOCITY || P.kind > LBM_PORT_INLET_RESCALE)
            return fail(nullptr, LBM_ERR_ARG, "port %d: kind %d invalid", p, P.kind);
        if (P.x < 0 || P.x >= nx || P.y0 < 0 || P.y1 > ny || P.y0 >= P.y1)
            return fail(nullptr, LBM_ERR_ARG, "port %d: column %d rows [%d, %d) outside the grid", p,
                        P.x, P.y0, P.y1);
        if (P.kind != LBM_PORT_VELOCITY && !(P.rho > 0.0 && std::isfinite(P.rho)))
            return fail(nullptr, LBM_ERR_ARG, "port %d: pressure density %g invalid", p, P.rho);
        const int s = P.side == LBM_WEST ? 1 : -1;
        for (int y = P.y0; y < P.y1; ++y) {
            if (!is_fluid(mask, nx, ny, P.x, y))
                return fail(nullptr, LBM_ERR_ARG, "port %d: node (%d, %d) is solid", p, P.x, y);
            lbm::RowBC& b = rowbc[size_t(P.side) * ny + y];
            if (b.x >= 0) return fail(nullptr, LBM_ERR_ARG, "port %d: row %d already has a port on that side", p, y);
            const lbm::RowBC& o = rowbc[size_t(1 - P.side) * ny + y];
            if (o.x == P.x)
                return fail(nullptr, LBM_ERR_ARG, "port %d: node (%d, %d) is also a port of the other side", p, P.x, y);
            b.x = P.x;
            b.chan_kind = P.channel | (P.kind << 8);
            b.a = P.kind != LBM_PORT_VELOCITY ? float(P.rho - 1.0) : 0.f;
        }
        for (int y = P.y0 - 1; y <= P.y1; ++y)
            if (is_fluid(mask, nx, ny, P.x - s, y))
                return fail(nullptr, LBM_ERR_ARG, "port %d: cell (%d, %d) outside the port is fluid", p,
                            P.x - s, y);
        any_velocity |= P.kind == LBM_PORT_VELOCITY;
        any_inlet |= P.kind == LBM_PORT_INLET_RESCALE;
    }
    if (any_velocity && (!edge_u || !edge_C))
        return fail(nullptr, LBM_ERR_ARG, "velocity ports need edge_u and edge_C");
    if (any_inlet && !edge_C) return fail(nullptr, LBM_ERR_ARG, "INLET_RESCALE ports need edge_C");
    for (int side = 0; side < 2; ++side)
        for (int y = 0; y < ny; ++y) {
            lbm::RowBC& b = rowbc[size_t(side) * ny + y];
            if (b.x < 0) continue;
            const int kind = b.chan_kind >> 8;
            if (kind == LBM_PORT_INLET_RESCALE) {
                const float c = edge_C[size_t(side) * ny + y];
                if (!std::isfinite(c)) return fail(nullptr, LBM_ERR_ARG, "inlet port row %d: C = %g invalid", y, c);
                b.c = c;
            }
            if (kind != LBM_PORT_VELOCITY) continue;
            const float u = edge_u[size_t(side) * ny + y], c = edge_C[size_t(side) * ny + y];
            if (!(std::fabs(u) < 1.f) || !std::isfinite(c))
                return fail(nullptr, LBM_ERR_ARG, "velocity port row %d: u_x = %g, C = %g invalid", y, u, c);
            b.a = u;
            b.c = c;
        }

    // wall-link table; every fluid node needs a fluid neighbour
    const int pitch = (nx + lbm::kTileNodes - 1) / lbm::kTileNodes * lbm::kTileNodes;
    const int segs = pitch / lbm::kTileNodes;
    // link masks, the tile table and the fluid count in one pass, rows split
    // over host threads on large lattices (each thread owns whole rows; its
    // tiles are appended in row order and the first bad node in row order is
    // reported)
    std::vector<uint8_t> links(size_t(pitch) * ny, lbm::kSolid);
    struct RowsOut {
        std::vector<uint2> tiles, tiles64;
        long long fluid = 0;
        int bad_x = -1, bad_y = -1;
    };
    // The 128-node tiles of row y from its link bytes L: each tile starts at
    // the row's first fluid node that no earlier tile covers, on a
    // kTileStart boundary, and its lanes q0 .. q1 are the quads holding
    // fluid.  Tiles never overlap (every kernel takes a tile's fluid lanes
    // from the link bytes alone): a row whose next tile would run past the
    // padded row end is tiled by 128-node segments instead.
    auto row_tiles = [&](const uint8_t* L, int y, std::vector<uint2>& tiles) {
        const size_t first = tiles.size();
        for (int pass = 0; pass < 2; ++pass) {
            const int gran = pass == 0 ? lbm::kTileStart : lbm::kTileNodes;
            bool fits = true;
            int t0 = -1, q0 = 0, q1 = 0;
            auto push = [&]() {
                tiles.push_back(make_uint2((uint32_t(y) << lbm::kColBits) | uint32_t(t0 / lbm::kTileStart),
                                           uint32_t(q0) | (uint32_t(q1) << 8)));
            };
            for (int x = 0; x < nx && fits; ++x) {
                if (L[x] == lbm::kSolid) continue;
                if (t0 < 0 || x >= t0 + lbm::kTileNodes) {
                    if (t0 >= 0) push();
                    t0 = x / gran * gran;
                    if (t0 + lbm::kTileNodes > pitch) fits = false;
                    q0 = (x - t0) / 4;
                }
                q1 = (x - t0) / 4;
            }
            if (fits) {
                if (t0 >= 0) push();
                return;
            }
            tiles.resize(first);
        }
    };
    auto build_rows = [&](int y0, int y1, RowsOut& out) {
        // a row of solid cells stands for the rows outside the grid, one
        // more solid cell on each side of every row for the columns outside
        std::vector<uint8_t> pad(size_t(3) * (nx + 2), 1);
        uint8_t* rows[3] = {pad.data(), pad.data() + (nx + 2), pad.data() + 2 * (nx + 2)};
        auto load = [&](uint8_t* dst, int yy) {
            if (yy < 0 || yy >= ny) {
                std::memset(dst, 1, size_t(nx) + 2);
                return;
            }
            const uint8_t* m = mask + size_t(yy) * nx;
            dst[0] = dst[nx + 1] = 1;
            for (int x = 0; x < nx; ++x) dst[x + 1] = m[x] != 0;
        };
        load(rows[0], y0 - 1);  // row y - 1: sources with e_y = +1
        load(rows[1], y0);
        for (int y = y0; y < y1; ++y) {
            load(rows[2], y + 1);  // row y + 1: sources with e_y = -1
            const uint8_t* S = rows[0] + 1;
            const uint8_t* C = rows[1] + 1;
            const uint8_t* N = rows[2] + 1;
            uint8_t* L = links.data() + size_t(y) * pitch;
            int h_cur = -1, p0 = -1, p1 = -1;  // 64-node segments, their first and last node pair holding fluid
            for (int x = 0; x < nx; ++x) {
                if (C[x]) continue;
                // bit i - 1: the pull source x - e_i is not fluid (directions of Eq. lattice)
                const uint8_t lb = uint8_t(C[x - 1] | (S[x] << 1) | (C[x + 1] << 2) | (N[x] << 3) |
                                           (S[x - 1] << 4) | (S[x + 1] << 5) | (N[x + 1] << 6) |
                                           (N[x - 1] << 7));
                if (lb == lbm::kSolid) {
                    out.bad_x = x;
                    out.bad_y = y;
                    return;
                }
                L[x] = lb;
                ++out.fluid;
                const int hg = x / lbm::kPairTileNodes, pr = (x % lbm::kPairTileNodes) / 2;
                if (hg != h_cur) {
                    if (h_cur >= 0)
                        out.tiles64.push_back(make_uint2((uint32_t(y) << lbm::kSegBits64) | uint32_t(h_cur),
                                                         uint32_t(p0) | (uint32_t(p1) << 8)));
                    h_cur = hg;
                    p0 = pr;
                }
                p1 = pr;
            }
            row_tiles(L, y, out.tiles);
            if (h_cur >= 0)
                out.tiles64.push_back(make_uint2((uint32_t(y) << lbm::kSegBits64) | uint32_t(h_cur),
                                                 uint32_t(p0) | (uint32_t(p1) << 8)));
            std::swap(rows[0], rows[1]);
            std::swap(rows[1], rows[2]);
        }
    };
    const int n_thr = (long long)nx * ny < (1 << 20)
                          ? 1
                          : std::max(1, std::min({16, ny, int(std::thread::hardware_concurrency())}));
    std::vector<RowsOut> parts(n_thr);
    {
        std::vector<std::thread> pool;
        for (int k = 1; k < n_thr; ++k)
            pool.emplace_back(build_rows, int((long long)ny * k / n_thr), int((long long)ny * (k + 1) / n_thr),
                              std::ref(parts[k]));
        build_rows(0, int((long long)ny / n_thr), parts[0]);
        for (auto& t : pool) t.join();
    }
    std::vector<uint2> tiles, tiles64;
    long long fluid = 0;
    for (const RowsOut& r : parts) {
        if (r.bad_y >= 0)
            return fail(nullptr, LBM_ERR_ARG, "fluid node (%d, %d) has no fluid neighbour", r.bad_x, r.bad_y);
        tiles.insert(tiles.end(), r.tiles.begin(), r.tiles.end());
        tiles64.insert(tiles64.end(), r.tiles64.begin(), r.tiles64.end());
        fluid += r.fluid;
    }
    if (fluid == 0) return fail(nullptr, LBM_ERR_ARG, "the mask has no fluid node");
    // tiles whose row segment holds a port node, listed after the others
    for (uint2& t : tiles) {
        const int y = int(t.x >> lbm::kColBits);
        const int x0 = int(t.x & ((1u << lbm::kColBits) - 1)) * lbm::kTileStart;
        for (int side = 0; side < 2; ++side) {
            const int px = rowbc[size_t(side) * ny + y].x;
            if (px >= x0 && px < x0 + lbm::kTileNodes) t.y |= lbm::kPortTile;
        }
    }
    for (uint2& t : tiles64) {
        const int y = int(t.x >> lbm::kSegBits64);
        const int x0 = int(t.x & ((1u << lbm::kSegBits64) - 1)) * lbm::kPairTileNodes;
        for (int side = 0; side < 2; ++side) {
            const int px = rowbc[size_t(side) * ny + y].x;
            if (px >= x0 && px < x0 + lbm::kPairTileNodes) t.y |= lbm::kPortTile;
        }
    }

    // ---- device set-up ----
    lbm_ctx* h = new (std::nothrow) lbm_ctx();
    if (!h) return fail(nullptr, LBM_ERR_OOM, "host allocation failed");
    h->nx = nx;
    h->ny = ny;
    h->pitch = pitch;
    h->segs = segs;
    h->plane = (long long)ny * pitch;
    h->tau = tau;
    h->tau_c = tau_c;
    h->w0 = opt.w0;
    h->rho0 = opt.rho0;
    h->C0 = opt.C0;
    h->wg0 = float(opt.w0);
    h->wg1 = float(0.25 * (1.0 - opt.w0));
    h->inv_cs2g = float(2.0 / (1.0 - opt.w0));
    h->stream = static_cast<cudaStream_t>(opt.stream);
    h->alloc_fn = opt.alloc;
    h->free_fn = opt.free;
    h->alloc_user = opt.alloc_user;
    h->n_tiles = int(tiles.size());
    h->n_tiles64 = int(tiles64.size());
    h->tiles_rows = std::move(tiles);
    h->tiles64_rows = std::move(tiles64);
    h->solid.assign(mask, mask + size_t(nx) * ny);
    h->fluid = fluid;
    h->precision = opt.precision;
    h->elem = opt.precision == LBM_FP32 ? sizeof(float) : sizeof(uint16_t);
    h->graph_steps = opt.graph_steps;
    h->scalar_regs = opt.scalar_variant != 2;
    h->multi_step = opt.multi_step;
    h->decay = float(opt.decay);
    h->wall_scheme = opt.wall_scheme;
    for (int p = 0; p < n_ports; ++p) h->paper_ports |= ports[p].kind >= LBM_PORT_PRESSURE_RESCALE;

    auto bail = [&](lbm_status s) {
        g_create_error = h->last_error;
        free_all(h);
        delete h;
        return s;
    };
    cudaError_t e;
    if (opt.device >= 0) {
        e = cudaSetDevice(opt.device);
        if (e != cudaSuccess) return bail(cuda_fail(h, e, "cudaSetDevice"));
    }
    e = cudaGetDevice(&h->device);
    if (e != cudaSuccess) return bail(cuda_fail(h, e, "cudaGetDevice"));
    int sms = 0, per_sm = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
    if (e != cudaSuccess) return bail(cuda_fail(h, e, "cudaDeviceGetAttribute"));
    h->sms = sms;
    lbm::StepLaunch& L = h->launch;
    // default: the register variant; with 16-bit storage (issue-bound) its
    // form with the next tile prefetched by asynchronous copies (the fastest
    // on each, see profiles)
    const int variant = opt.variant                                                              ? opt.variant
                        : opt.precision != LBM_FP32 && opt.wall_scheme == LBM_WALL_BOUNCE_BACK ? 4
                                                                                                : 1;
    L.variant = variant == 1   ? lbm::kVariantRegs
                : variant == 3 ? lbm::kVariantPipe
                : variant == 4 ? lbm::kVariantAsync
                : variant == 5 ? lbm::kVariantPairs
                               : lbm::kVariantBulk;
    L.precision = opt.precision;
    L.pdl = true;  // consecutive steps overlap launch and set-up with the previous step's tail
    L.walls = opt.wall_scheme == LBM_WALL_EQUILIBRIUM;
    if (L.variant == lbm::kVariantBulk) {
        const int nc = opt.consumer_warps ? opt.consumer_warps : kDefaultConsumers;
        L.stages = nc * (opt.pipeline_stages                ? opt.pipeline_stages
                         : opt.precision == LBM_FP32 ? kDefaultStagesPerConsumer
                                                     : kDefaultStagesPerConsumer16);
        L.block = 32 * (nc + 1);
        e = lbm::prepare_step_kernels();
        if (e != cudaSuccess) return bail(cuda_fail(h, e, "shared-memory attribute"));
    } else if (L.variant == lbm::kVariantPipe) {
        const int nw = opt.consumer_warps ? opt.consumer_warps : kDefaultPipeWarps;
        L.stages = nw * (opt.pipeline_stages ? opt.pipeline_stages : kDefaultStagesPerConsumer);
        L.block = 32 * nw;
        e = lbm::prepare_step_kernels();
        if (e != cudaSuccess) return bail(cuda_fail(h, e, "shared-memory attribute"));
    } else {
        L.stages = 0;
        L.block = opt.block_threads ? opt.block_threads : kDefaultRegsBlock;
        if (L.variant == lbm::kVariantAsync) {
            e = lbm::prepare_step_kernels();
            if (e != cudaSuccess) return bail(cuda_fail(h, e, "shared-memory attribute"));
        }
    }
    e = lbm::step_kernel_occupancy(L, &per_sm);
    if (e != cudaSuccess) return bail(cuda_fail(h, e, "occupancy query"));
    if (per_sm < 1) return bail(fail(h, LBM_ERR_ARG, "the step kernel cannot run with this launch shape"));
    L.grid = wave_grid(h, L, per_sm);
    if (opt.max_blocks > 0) L.grid = std::min(L.grid, opt.max_blocks);

    const size_t pop_bytes = size_t(h->plane) * lbm::kPlanes * h->elem;
    h->pop[0] = static_cast<float*>(dev_alloc(h, pop_bytes));
    h->pop[1] = static_cast<float*>(dev_alloc(h, pop_bytes));
    h->links = static_cast<uint8_t*>(dev_alloc(h, links.size()));
    h->rowbc = static_cast<lbm::RowBC*>(dev_alloc(h, rowbc.size() * sizeof(lbm::RowBC)));
    h->tiles = static_cast<uint2*>(dev_alloc(h, std::max<size_t>(1, h->tiles_rows.size()) * sizeof(uint2)));
    h->tiles64 = static_cast<uint2*>(dev_alloc(h, std::max<size_t>(1, h->tiles64_rows.size()) * sizeof(uint2)));
    h->partials_cap = std::max(h->launch.grid, sms * kMaxBlocksPerSM);
    h->diag_grid = h->launch.grid;
    h->partials = static_cast<float2*>(dev_alloc(h, size_t(h->partials_cap) * 4 * sizeof(float2)));
    // the error word, then the ticket counter of lbm_step_diagnostics
    h->err = static_cast<unsigned*>(dev_alloc(h, 2 * sizeof(unsigned)));
    if (h->multi_step > 0) {
        int coop_per_sm = 0;
        e = lbm::steps_coop_occupancy(kDefaultRegsBlock, &coop_per_sm);
        if (e != cudaSuccess) return bail(cuda_fail(h, e, "occupancy query"));
        const int wpb = kDefaultRegsBlock / 32;
        h->coop_grid = std::max(1, std::min((h->n_tiles + wpb - 1) / wpb, std::max(1, coop_per_sm) * sms));
        h->bar = static_cast<unsigned*>(dev_alloc(h, sizeof(unsigned)));
        if (!h->bar) return bail(fail(h, LBM_ERR_OOM, "device allocation of the barrier word failed"));
    }
    h->diag = static_cast<double*>(dev_alloc(h, 4 * sizeof(double)));
    h->fields_tmp = static_cast<float*>(dev_alloc(h, size_t(4) * nx * ny * sizeof(float)));
    if (batch) h->rates = static_cast<float4*>(dev_alloc(h, size_t(ny) * sizeof(float4)));
    std::vector<long long> woff;
    if (opt.wall_scheme == LBM_WALL_EQUILIBRIUM) {
        for (size_t o = 0; o < links.size(); ++o)
            if (links[o] != 0 && links[o] != lbm::kSolid) woff.push_back((long long)o);
        h->n_wall = int(woff.size());
        h->wallv = dev_alloc(h, size_t(8) * h->plane * h->elem);
        h->woff = static_cast<long long*>(dev_alloc(h, std::max<size_t>(1, woff.size()) * sizeof(long long)));
    }
    if (!h->pop[0] || !h->pop[1] || !h->links || !h->rowbc || !h->tiles || !h->tiles64 || !h->partials ||
        !h->err || !h->diag || !h->fields_tmp || (batch && !h->rates) ||
        (opt.wall_scheme == LBM_WALL_EQUILIBRIUM && (!h->wallv || !h->woff)))
        return bail(fail(h, LBM_ERR_OOM, "device allocation of %zu bytes failed", 2 * pop_bytes));
    if (batch) h->inst = batch->inst;

    cudaStream_t st = h->stream;
    e = cudaMemcpyAsync(h->links, links.data(), links.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h->rowbc, rowbc.data(), rowbc.size() * sizeof(lbm::RowBC),
                            cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = arrange_tiles(h, h->launch);
    if (e == cudaSuccess && batch)
        e = cudaMemcpyAsync(h->rates, batch->rates.data(), size_t(ny) * sizeof(float4), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && !woff.empty())
        e = cudaMemcpyAsync(h->woff, woff.data(), woff.size() * sizeof(long long), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->err, 0, 2 * sizeof(unsigned), st);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(h->partials, 0, size_t(h->partials_cap) * 4 * sizeof(float2), st);
    if (e == cudaSuccess)
        e = lbm::launch_init_rest(h->pop[0], ny, pitch, float(h->rho0), h->wg0, h->wg1, float(h->C0),
                                  h->precision, h->decay, st);
    if (e == cudaSuccess)
        e = lbm::launch_init_rest(h->pop[1], ny, pitch, float(h->rho0), h->wg0, h->wg1, float(h->C0),
                                  h->precision, h->decay, st);
    // the host tables above are pageable: wait so they may go out of scope
    if (e == cudaSuccess && h->graph_steps > 0) e = cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return bail(cuda_fail(h, e, "device initialisation"));
    *out = h;
    g_create_error = "no error";
    return LBM_OK;
}
}  // namespace

extern "C" {

lbm_status lbm_create(lbm_handle* out, int32_t nx, int32_t ny, const uint8_t* mask, double tau,
                      double tau_c, int32_t n_ports, const lbm_port* ports, const float* edge_u,
                      const float* edge_C, const lbm_options* opt_in)
{
    Range range("lbm_create");
    return create_impl(out, nx, ny, mask, tau, tau_c, n_ports, ports, edge_u, edge_C, opt_in, nullptr);
}

lbm_status lbm_create_batch(lbm_handle* out, int32_t n, const lbm_chip_desc* chips, const lbm_options* opt)
{
    Range range("lbm_create_batch");
    if (!out) return fail(nullptr, LBM_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (n < 1 || n > kMaxInstances) return fail(nullptr, LBM_ERR_ARG, "n = %d outside [1, %d]", n, kMaxInstances);
    if (!chips) return fail(nullptr, LBM_ERR_ARG, "chips is NULL");
    // stack the chips along y, one solid row between neighbours, so that no
    // link of one chip reaches another (every link that leaves a chip ends
    // on a solid node, as at the edge of a single chip)
    BatchSpec b;
    int nx = 0, ny = 0, chan = 0;
    for (int k = 0; k < n; ++k) {
        const lbm_chip_desc& c = chips[k];
        if (c.nx < 1 || c.ny < 1) return fail(nullptr, LBM_ERR_ARG, "chip %d: grid %d x %d is empty", k, c.nx, c.ny);
        if (!c.mask) return fail(nullptr, LBM_ERR_ARG, "chip %d: mask is NULL", k);
        if (!(c.tau > 0.5) || !std::isfinite(c.tau) || !(c.tau_c > 0.5) || !std::isfinite(c.tau_c))
            return fail(nullptr, LBM_ERR_ARG, "chip %d: tau = %g, tau_c = %g: relaxation times must exceed 1/2", k,
                        c.tau, c.tau_c);
        if (c.n_ports < 0 || c.n_ports > kMaxPorts || (c.n_ports > 0 && !c.ports))
            return fail(nullptr, LBM_ERR_ARG, "chip %d: n_ports = %d or ports invalid", k, c.n_ports);
        int top = -1;
        for (int p = 0; p < c.n_ports; ++p) {
            if (c.ports[p].channel < 0 || c.ports[p].channel > 31)
                return fail(nullptr, LBM_ERR_ARG, "chip %d port %d: channel %d outside [0, 31]", k, p,
                            c.ports[p].channel);
            top = std::max(top, c.ports[p].channel);
        }
        if (k > 0) ++ny;  // separator row
        lbm_ctx::Inst I{ny, c.nx, c.ny, chan, top + 1, c.tau, c.tau_c, 0u, 0, {}};
        b.inst.push_back(I);
        chan += top + 1;
        nx = std::max(nx, int(c.nx));
        if (int64_t(ny) + c.ny >= (1 << 19)) return fail(nullptr, LBM_ERR_ARG, "the stacked chips are too tall");
        ny += c.ny;
    }
    if (chan > 32 * lbm::kMaskWords)
        return fail(nullptr, LBM_ERR_ARG, "the chips have %d valve channels in all, more than %d", chan,
                    32 * lbm::kMaskWords);
    std::vector<uint8_t> mask(size_t(nx) * ny, 1);
    std::vector<float> eu(size_t(2) * ny, 0.f), ec(size_t(2) * ny, 0.f);
    std::vector<lbm_port> ports;
    b.rates.assign(size_t(ny), make_float4(0.f, 0.f, 0.f, 0.f));
    for (int k = 0; k < n; ++k) {
        const lbm_chip_desc& c = chips[k];
        const lbm_ctx::Inst& I = b.inst[k];
        for (int y = 0; y < c.ny; ++y) {
            std::memcpy(&mask[size_t(I.row0 + y) * nx], c.mask + size_t(y) * c.nx, size_t(c.nx));
            b.rates[I.row0 + y] = make_float4(float(1.0 / c.tau), float(1.0 / c.tau_c), 0.f, 0.f);
            for (int side = 0; side < 2; ++side) {
                if (c.edge_u) eu[size_t(side) * ny + I.row0 + y] = c.edge_u[size_t(side) * c.ny + y];
                if (c.edge_C) ec[size_t(side) * ny + I.row0 + y] = c.edge_C[size_t(side) * c.ny + y];
            }
        }
        for (int p = 0; p < c.n_ports; ++p) {
            lbm_port q = c.ports[p];
            if (q.y0 < 0 || q.y1 > c.ny || q.y0 >= q.y1 || q.x < 0 || q.x >= c.nx)
                return fail(nullptr, LBM_ERR_ARG, "chip %d port %d: column %d rows [%d, %d) outside the chip", k, p,
                            q.x, q.y0, q.y1);
            if (q.kind == LBM_PORT_VELOCITY && (!c.edge_u || !c.edge_C))
                return fail(nullptr, LBM_ERR_ARG, "chip %d: velocity ports need edge_u and edge_C", k);
            q.channel += I.chan_base;
            q.y0 += I.row0;
            q.y1 += I.row0;
            ports.push_back(q);
        }
    }
    lbm_options o;
    lbm_default_options(&o);
    if (opt) {
        if (opt->struct_size != sizeof(lbm_options))
            return fail(nullptr, LBM_ERR_ARG, "lbm_options.struct_size is %u, expected %zu", opt->struct_size,
                        sizeof(lbm_options));
        o = *opt;
    }
    return create_impl(out, nx, ny, mask.data(), chips[0].tau, chips[0].tau_c, int32_t(ports.size()), ports.data(),
                       eu.data(), ec.data(), &o, &b);
}

lbm_status lbm_get_instance(lbm_handle h, int32_t k, lbm_instance* out)
{
    if (check_ctx(h) || !out) return fail(h, LBM_ERR_ARG, "out is NULL");
    const int n = h->inst.empty() ? 1 : int(h->inst.size());
    if (k < 0 || k >= n) return fail(h, LBM_ERR_ARG, "instance %d outside [0, %d)", k, n);
    if (h->inst.empty()) {
        *out = lbm_instance{0, h->nx, h->ny, 0};
    } else {
        const lbm_ctx::Inst& I = h->inst[size_t(k)];
        *out = lbm_instance{I.row0, I.nx, I.ny, I.chan_base};
    }
    return LBM_OK;
}

lbm_status lbm_set_instance_valves(lbm_handle h, int32_t k, uint32_t open_mask)
{
    if (check_ctx(h)) return LBM_ERR_ARG;
    if (h->inst.empty()) {
        if (k != 0) return fail(h, LBM_ERR_ARG, "instance %d of a single chip", k);
        return lbm_set_valves(h, open_mask);
    }
    if (k < 0 || k >= int(h->inst.size())) return fail(h, LBM_ERR_ARG, "instance %d outside [0, %zu)", k, h->inst.size());
    lbm_ctx::Inst& I = h->inst[size_t(k)];
    I.fixed_mask = open_mask;
    I.schedule.clear();
    I.period = 0;
    return LBM_OK;
}

lbm_status lbm_set_instance_schedule(lbm_handle h, int32_t k, int64_t period, int32_t n, const uint32_t* states)
{
    if (check_ctx(h)) return LBM_ERR_ARG;
    if (h->inst.empty()) {
        if (k != 0) return fail(h, LBM_ERR_ARG, "instance %d of a single chip", k);
        return lbm_set_valve_schedule(h, period, n, states);
    }
    if (k < 0 || k >= int(h->inst.size())) return fail(h, LBM_ERR_ARG, "instance %d outside [0, %zu)", k, h->inst.size());
    if (n < 0 || n > kMaxSchedule) return fail(h, LBM_ERR_ARG, "schedule length %d outside [0, %d]", n, kMaxSchedule);
    if (n > 0 && period < 1) return fail(h, LBM_ERR_ARG, "schedule period %lld < 1", (long long)period);
    if (n > 0 && !states) return fail(h, LBM_ERR_ARG, "states is NULL");
    lbm_ctx::Inst& I = h->inst[size_t(k)];
    I.schedule.assign(states, states + n);
    I.period = n > 0 ? period : 0;
    return LBM_OK;
}

void lbm_destroy(lbm_handle h)
{
    if (!h) return;
    cudaStreamSynchronize(h->stream);
    free_all(h);
    delete h;
}

lbm_status lbm_set_valves(lbm_handle h, uint32_t open_mask)
{
    if (check_ctx(h)) return LBM_ERR_ARG;
    h->fixed_mask = open_mask;
    h->schedule.clear();
    h->period = 0;
    for (lbm_ctx::Inst& I : h->inst) {  // every chip of a batch runs this valve word
        I.fixed_mask = open_mask;
        I.schedule.clear();
        I.period = 0;
    }
    return LBM_OK;
}

lbm_status lbm_set_valve_schedule(lbm_handle h, int64_t period, int32_t n, const uint32_t* states)
{
    if (check_ctx(h)) return LBM_ERR_ARG;
    if (n == 0) {
        h->schedule.clear();
        h->period = 0;
        for (lbm_ctx::Inst& I : h->inst) {
            I.schedule.clear();
            I.period = 0;
        }
        return LBM_OK;
    }
    if (n < 0 || n > kMaxSchedule) return fail(h, LBM_ERR_ARG, "schedule length %d outside [0, %d]", n, kMaxSchedule);
    if (period < 1) return fail(h, LBM_ERR_ARG, "schedule period %lld < 1", (long long)period);
    if (!states) return fail(h, LBM_ERR_ARG, "states is NULL");
    h->schedule.assign(states, states + n);
    h->period = period;
    for (lbm_ctx::Inst& I : h->inst) {  // every chip of a batch runs this schedule
        I.schedule.assign(states, states + n);
        I.period = period;
    }
    return LBM_OK;
}

}  // extern "C"

// Arguments of the chip's coupled step that do not change from step to step.
static lbm::StepArgs step_args(const lbm_ctx* h)
{
    lbm::StepArgs a{};
    a.links = h->links;
    a.rowbc = h->rowbc;
    a.tiles = h->tiles;
    a.n_tiles = h->n_tiles;
    a.n_plain = h->n_plain;
    a.tiles64 = h->tiles64;
    a.n_tiles64 = h->n_tiles64;
    a.ny = h->ny;
    a.pitch = h->pitch;
    a.plane = h->plane;
    a.omega_f = float(1.0 / h->tau);
    a.omega_g = float(1.0 / h->tau_c);
    a.wg0 = h->wg0;
    a.wg1 = h->wg1;
    a.inv_cs2g = h->inv_cs2g;
    a.decay = h->decay;
    a.wallv = h->wallv;
    a.partials = h->partials;
    a.err = h->err;
    a.rates = h->rates;
    if (h->precision != LBM_FP32) {
        a.gref0 = h->wg0 * lbm::kCRef;
        a.gref1 = h->wg1 * lbm::kCRef;
    }
    return a;
}

extern "C" {

lbm_status lbm_step(lbm_handle h, int64_t n)
{
    Range range("lbm_step");
    if (check_ctx(h)) return LBM_ERR_ARG;
    if (n < 0) return fail(h, LBM_ERR_ARG, "n = %lld < 0", (long long)n);
    if (lbm_status js = join_scalar(h)) return js;
    lbm::StepArgs a = step_args(h);
    const int G = h->graph_steps;
    for (int64_t k = 0; k < n;) {
        h->mask_words(h->step, a.open_mask);
        if (h->multi_step > 0 && n - k >= 2) {
            const int64_t m = h->mask_run(h->step, std::min<int64_t>(n - k, h->multi_step));
            if (m >= 2) {
                // m steps in one cooperative launch; the state ends in the
                // other buffer when m is odd
                a.src = h->pop[h->cur];
                a.dst = h->pop[1 - h->cur];
                a.reverse = h->cur;
                a.barrier_extra = h->barrier_extra;
                cudaError_t e =
                    lbm::launch_steps_coop(a, int(m), 0, h->bar, h->coop_grid, kDefaultRegsBlock, h->stream);
                if (e != cudaSuccess) return cuda_fail(h, e, "multi-step launch");
                if (m & 1) h->cur = 1 - h->cur;
                h->gbuf = h->cur;
                h->diag_grid = h->coop_grid;
                h->step += m;
                k += m;
                continue;
            }
        }
        if (G > 0 && n - k >= G && h->mask_constant(h->step, G)) {
            // G steps (an even number: the state ends in the buffer it
            // started from) as one graph launch
            cudaGraphExec_t exec = nullptr;
            lbm_status s = step_graph(h, a, &exec);
            if (s != LBM_OK) return s;
            LBM_CUDA(h, cudaGraphLaunch(exec, h->stream));
            h->step += G;
            k += G;
            h->diag_grid = h->launch.grid;
            continue;
        }
        a.src = h->pop[h->cur];
        a.dst = h->pop[1 - h->cur];
        a.reverse = h->cur;  // alternate the tile order from step to step
        cudaError_t e = launch_full_step(h, a, h->launch, h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "coupled step launch");
        h->cur = 1 - h->cur;
        h->gbuf = h->cur;
        h->diag_grid = h->launch.grid;
        ++h->step;
        ++k;
    }
    return pending_numeric(h);
}

// The device address of caller memory the device can write: device memory,
// or page-locked host memory mapped into the device's address space (null
// for anything else).
static double* device_address(double* p)
{
    cudaPointerAttributes pa{};
    if (cudaPointerGetAttributes(&pa, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (pa.type == cudaMemoryTypeDevice || pa.type == cudaMemoryTypeManaged || pa.type == cudaMemoryTypeHost)
        return static_cast<double*>(pa.devicePointer);
    return nullptr;
}

lbm_status lbm_step_diagnostics(lbm_handle h, int64_t n, double* out)
{
    Range range("lbm_step_diagnostics");
    if (check_ctx(h)) return LBM_ERR_ARG;
    if (n < 0) return fail(h, LBM_ERR_ARG, "n = %lld < 0", (long long)n);
    if (n == 0) return LBM_OK;
    if (!out) return fail(h, LBM_ERR_ARG, "out is NULL");
    double* dev = device_address(out);
    if (!dev) return fail(h, LBM_ERR_ARG, "out must be device memory or page-locked host memory");
    if (lbm_status js = join_scalar(h)) return js;
    lbm::StepArgs a = step_args(h);
    a.diag_ticket = h->err + 1;
    // The in-kernel fold: variants 1 and 4 with blocks of at least
    // lbm::kFoldThreads threads and halfway bounce-back; other launch shapes
    // leave it to the reduction kernel, launched after each step (the same
    // order of additions, the same bits).
    const bool fold = lbm::step_folds_totals(h->launch);
    for (int64_t k = 0; k < n; ++k) {
        h->mask_words(h->step, a.open_mask);
        a.src = h->pop[h->cur];
        a.dst = h->pop[1 - h->cur];
        a.reverse = h->cur;
        a.diag_out = fold ? dev + 4 * k : nullptr;  // the step's last block writes the totals here
        cudaError_t e = launch_full_step(h, a, h->launch, h->stream);
        if (e == cudaSuccess && !fold) e = lbm::launch_diag_finish(h->partials, h->launch.grid, dev + 4 * k, h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "coupled step launch");
        h->cur = 1 - h->cur;
        h->gbuf = h->cur;
        h->diag_grid = h->launch.grid;
        ++h->step;
    }
    return pending_numeric(h);
}

static lbm_status read_err_word(lbm_handle h);

lbm_status lbm_synchronize(lbm_handle h)
{
    if (check_ctx(h)) return LBM_ERR_ARG;
    LBM_CUDA(h, cudaStreamSynchronize(h->stream));
    LBM_CUDA(h, cudaGetLastError());
    return read_err_word(h);
}

static lbm_status read_err_word(lbm_handle h)
{
    unsigned err = 0;
    LBM_CUDA(h, cudaMemcpyAsync(&err, h->err, sizeof(unsigned), cudaMemcpyDeviceToHost, h->stream));
    LBM_CUDA(h, cudaStreamSynchronize(h->stream));
    if (err & 2u) h->timeout = true;
    if (err & 1u) h->numeric = true;
    if (err & 2u)
        return fail(h, LBM_ERR_TIMEOUT, "timeout: a bounded wait of the step kernel gave up; results are invalid");
    if (err & 1u)
        return fail(h, LBM_ERR_NUMERIC, "numeric: a fluid node reached a non-finite or non-positive density or a non-finite concentration");
    return pending_numeric(h);
}

lbm_status lbm_debug_barrier_extra(lbm_handle h, int32_t extra)
{
    if (check_ctx(h)) return LBM_ERR_ARG;
    if (extra < 0 || extra > 1024) return fail(h, LBM_ERR_ARG, "extra = %d outside [0, 1024]", extra);
    h->barrier_extra = unsigned(extra);
    return LBM_OK;
}

lbm_status lbm_clear_error(lbm_handle h)
{
    if (check_ctx(h)) return LBM_ERR_ARG;
    LBM_CUDA(h, cudaMemsetAsync(h->err, 0, sizeof(unsigned), h->stream));
    LBM_CUDA(h, cudaStreamSynchronize(h->stream));
    h->numeric = false;
    h->timeout = false;
    h->last_error = "no error";
    return LBM_OK;
}

lbm_status lbm_get_fields_device(lbm_handle h, float* rho, float* ux, float* uy, float* C)
{
    if (check_ctx(h)) return LBM_ERR_ARG;
    if (lbm_status js = join_scalar(h)) return js;
    cudaError_t e = lbm::launch_fields(h->pop[h->cur], h->links, h->nx, h->ny, h->pitch, rho, ux, uy, C, h->wg0,
                                       h->wg1, h->precision, h->decay, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "fields kernel launch");
    return LBM_OK;
}

lbm_status lbm_get_fields(lbm_handle h, float* rho, float* ux, float* uy, float* C)
{
    Range range("lbm_get_fields");
    if (check_ctx(h)) return LBM_ERR_ARG;
    const size_t n = size_t(h->nx) * h->ny;
    float* t = h->fields_tmp;
    lbm_status s = lbm_get_fields_device(h, rho ? t : nullptr, ux ? t + n : nullptr,
                                         uy ? t + 2 * n : nullptr, C ? t + 3 * n : nullptr);
    if (s != LBM_OK) return s;
    float* outs[4] = {rho, ux, uy, C};
    for (int q = 0; q < 4; ++q)
        if (outs[q])
            LBM_CUDA(h, cudaMemcpyAsync(outs[q], t + q * n, n * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
    LBM_CUDA(h, cudaStreamSynchronize(h->stream));
    return LBM_OK;
}

lbm_status lbm_get_diagnostics(lbm_handle h, double out[4])
{
    if (check_ctx(h) || !out) return fail(h, LBM_ERR_ARG, "out is NULL");
    cudaError_t e = lbm::launch_diag_finish(h->partials, h->diag_grid, h->diag, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "diagnostics reduction launch");
    LBM_CUDA(h, cudaMemcpyAsync(out, h->diag, 4 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    return read_err_word(h);
}

lbm_status lbm_get_diagnostics_async(lbm_handle h, double* out)
{
    if (check_ctx(h) || !out) return fail(h, LBM_ERR_ARG, "out is NULL");
    // page-locked host memory mapped into the device's address space takes
    // the totals straight from the reduction kernel (no copy in the stream)
    cudaPointerAttributes pa{};
    double* direct = nullptr;
    if (cudaPointerGetAttributes(&pa, out) == cudaSuccess) {
        if (pa.type == cudaMemoryTypeHost && pa.devicePointer) direct = static_cast<double*>(pa.devicePointer);
    } else {
        cudaGetLastError();
    }
    cudaError_t e = lbm::launch_diag_finish(h->partials, h->diag_grid, direct ? direct : h->diag, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "diagnostics reduction launch");
    if (!direct) LBM_CUDA(h, cudaMemcpyAsync(out, h->diag, 4 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    return pending_numeric(h);
}

}  // extern "C"

namespace {

// D2Q9 weights: the device stores f_i - w_i (see lbm_internal.h).
constexpr float kW9[9] = {4.f / 9.f, 1.f / 9.f, 1.f / 9.f, 1.f / 9.f, 1.f / 9.f,
                          1.f / 36.f, 1.f / 36.f, 1.f / 36.f, 1.f / 36.f};

// Device temporaries of one call, released in reverse order on every exit.
struct Scratch {
    lbm_ctx* h;
    std::vector<Alloc> items;
    explicit Scratch(lbm_ctx* ctx) : h(ctx) {}
    void* get(size_t bytes)
    {
        bytes = (bytes + 255) & ~size_t(255);
        void* p = nullptr;
        if (h->alloc_fn) {
            p = hook_alloc(h, bytes);
        } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
        }
        if (p) items.push_back({p, bytes});
        return p;
    }
    ~Scratch()
    {
        cudaStreamSynchronize(h->stream);
        for (auto it = items.rbegin(); it != items.rend(); ++it) {
            if (h->free_fn) h->free_fn(it->ptr, it->bytes, h->alloc_user);
            else cudaFree(it->ptr);
        }
    }
};

// The state in its FP32 representation (fluid planes f_i - w_i, scalar planes
// g_i), [plane][y][x] on the host; 16-bit storage is converted on the device.
lbm_status raw_out(lbm_ctx* h, float* f, float* g)
{
    if (lbm_status js = join_scalar(h)) return js;
    const float* src = h->pop[h->cur];
    Scratch sc(h);
    if (h->precision != LBM_FP32) {
        void* tmp = sc.get(size_t(h->plane) * lbm::kPlanes * sizeof(float));
        if (!tmp) return fail(h, LBM_ERR_OOM, "no device memory for the FP32 copy of the state");
        cudaError_t e = lbm::launch_convert(src, tmp, h->plane, h->wg0, h->wg1, h->precision, true, h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "conversion kernel launch");
        src = static_cast<const float*>(tmp);
    }
    const size_t row = size_t(h->nx) * sizeof(float), pitch = size_t(h->pitch) * sizeof(float);
    cudaError_t e = cudaSuccess;
    if (f) e = cudaMemcpy2DAsync(f, row, src, pitch, row, size_t(9) * h->ny, cudaMemcpyDeviceToHost, h->stream);
    if (g && e == cudaSuccess)
        e = cudaMemcpy2DAsync(g, row, src + 9 * h->plane, pitch, row, size_t(5) * h->ny, cudaMemcpyDeviceToHost,
                              h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "population read-out");
    return LBM_OK;
}

lbm_status raw_in(lbm_ctx* h, const float* f, const float* g)
{
    if (lbm_status js = join_scalar(h)) return js;
    float* dst = h->pop[h->cur];
    Scratch sc(h);
    void* tmp = nullptr;
    cudaError_t e = cudaSuccess;
    if (h->precision != LBM_FP32) {
        // planes that are not given keep their values: start from the state
        tmp = sc.get(size_t(h->plane) * lbm::kPlanes * sizeof(float));
        if (!tmp) return fail(h, LBM_ERR_OOM, "no device memory for the FP32 copy of the state");
        e = lbm::launch_convert(dst, tmp, h->plane, h->wg0, h->wg1, h->precision, true, h->stream);
        dst = static_cast<float*>(tmp);
    }
    const size_t row = size_t(h->nx) * sizeof(float), pitch = size_t(h->pitch) * sizeof(float);
    if (f && e == cudaSuccess)
        e = cudaMemcpy2DAsync(dst, pitch, f, row, row, size_t(9) * h->ny, cudaMemcpyHostToDevice, h->stream);
    if (g && e == cudaSuccess)
        e = cudaMemcpy2DAsync(dst + 9 * h->plane, pitch, g, row, row, size_t(5) * h->ny, cudaMemcpyHostToDevice,
                              h->stream);
    if (tmp && e == cudaSuccess)
        e = lbm::launch_convert(tmp, h->pop[h->cur], h->plane, h->wg0, h->wg1, h->precision, false, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "population write-in");
    return LBM_OK;
}

// The stored elements as they are (elem bytes each), [plane][y][x].
lbm_status stored_out(lbm_ctx* h, void* out)
{
    if (lbm_status js = join_scalar(h)) return js;
    const size_t row = size_t(h->nx) * h->elem, pitch = size_t(h->pitch) * h->elem;
    LBM_CUDA(h, cudaMemcpy2DAsync(out, row, h->pop[h->cur], pitch, row, size_t(lbm::kPlanes) * h->ny,
                                  cudaMemcpyDeviceToHost, h->stream));
    LBM_CUDA(h, cudaStreamSynchronize(h->stream));
    return LBM_OK;
}

lbm_status stored_in(lbm_ctx* h, const void* in)
{
    if (lbm_status js = join_scalar(h)) return js;
    const size_t row = size_t(h->nx) * h->elem, pitch = size_t(h->pitch) * h->elem;
    LBM_CUDA(h, cudaMemcpy2DAsync(h->pop[h->cur], pitch, in, row, row, size_t(lbm::kPlanes) * h->ny,
                                  cudaMemcpyHostToDevice, h->stream));
    LBM_CUDA(h, cudaStreamSynchronize(h->stream));
    return LBM_OK;
}

}  // namespace

extern "C" {

lbm_status lbm_get_populations(lbm_handle h, float* f, float* g)
{
    if (check_ctx(h)) return LBM_ERR_ARG;
    lbm_status s = raw_out(h, f, g);
    if (s != LBM_OK || !f) return s;
    const size_t n = size_t(h->nx) * h->ny;
    for (int i = 0; i < 9; ++i)
        for (size_t k = 0; k < n; ++k) f[i * n + k] += kW9[i];
    return LBM_OK;
}

lbm_status lbm_set_populations(lbm_handle h, const float* f, const float* g)
{
    if (check_ctx(h)) return LBM_ERR_ARG;
    std::vector<float> fd;
    if (f) {
        const size_t n = size_t(h->nx) * h->ny;
        fd.assign(f, f + 9 * n);
        for (int i = 0; i < 9; ++i)
            for (size_t k = 0; k < n; ++k) fd[i * n + k] -= kW9[i];
    }
    return raw_in(h, f ? fd.data() : nullptr, g);
}

lbm_status lbm_init_equilibrium(lbm_handle h, const float* rho, const float* ux, const float* uy,
                                const float* C)
{
    if (check_ctx(h)) return LBM_ERR_ARG;
    if (!rho || !ux || !uy || !C) return fail(h, LBM_ERR_ARG, "a field pointer is NULL");
    if (lbm_status js = join_scalar(h)) return js;
    const size_t n = size_t(h->nx) * h->ny;
    float* t = h->fields_tmp;
    const float* ins[4] = {rho, ux, uy, C};
    for (int q = 0; q < 4; ++q)
        LBM_CUDA(h, cudaMemcpyAsync(t + q * n, ins[q], n * sizeof(float), cudaMemcpyHostToDevice, h->stream));
    cudaError_t e = lbm::launch_init_fields(h->pop[h->cur], h->links, h->nx, h->ny, h->pitch, t, t + n,
                                            t + 2 * n, t + 3 * n, h->wg0, h->wg1, h->inv_cs2g, h->precision,
                                            h->decay, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "equilibrium kernel launch");
    LBM_CUDA(h, cudaStreamSynchronize(h->stream));
    return LBM_OK;
}

namespace {
struct StateHeader {
    uint32_t magic;
    int32_t nx, ny;
    int32_t n_sched;
    int64_t step;
    int64_t period;
    uint32_t fixed_mask;
    uint32_t precision;
};
}  // namespace

lbm_status lbm_save_state(lbm_handle h, void* buf, size_t* bytes)
{
    Range range("lbm_save_state");
    if (check_ctx(h) || !bytes) return fail(h, LBM_ERR_ARG, "bytes is NULL");
    const size_t pop = size_t(h->nx) * h->ny * lbm::kPlanes * h->elem;
    const size_t need = sizeof(StateHeader) + h->schedule.size() * 4 + pop;
    if (!buf) {
        *bytes = need;
        return LBM_OK;
    }
    if (*bytes < need) return fail(h, LBM_ERR_ARG, "state buffer of %zu bytes, need %zu", *bytes, need);
    StateHeader hd{kStateMagic, h->nx,        h->ny, int32_t(h->schedule.size()), h->step, h->period,
                   h->fixed_mask, uint32_t(h->precision)};
    char* p = static_cast<char*>(buf);
    std::memcpy(p, &hd, sizeof(hd));
    p += sizeof(hd);
    if (!h->schedule.empty()) std::memcpy(p, h->schedule.data(), h->schedule.size() * 4);
    p += h->schedule.size() * 4;
    // the stored representation, bit for bit (the buffer may be unaligned)
    std::vector<uint8_t> stored(pop);
    lbm_status s = stored_out(h, stored.data());
    if (s != LBM_OK) return s;
    std::memcpy(p, stored.data(), stored.size());
    *bytes = need;
    return LBM_OK;
}

lbm_status lbm_load_state(lbm_handle h, const void* buf, size_t bytes)
{
    Range range("lbm_load_state");
    if (check_ctx(h) || !buf) return fail(h, LBM_ERR_ARG, "buf is NULL");
    StateHeader hd;
    if (bytes < sizeof(hd)) return fail(h, LBM_ERR_ARG, "state buffer too short");
    std::memcpy(&hd, buf, sizeof(hd));
    if (hd.magic != kStateMagic || hd.nx != h->nx || hd.ny != h->ny || hd.n_sched < 0 ||
        hd.n_sched > kMaxSchedule || (hd.n_sched > 0 && hd.period < 1) || hd.precision != uint32_t(h->precision))
        return fail(h, LBM_ERR_ARG, "state buffer does not match this chip");
    const size_t n = size_t(h->nx) * h->ny;
    const size_t need = sizeof(hd) + size_t(hd.n_sched) * 4 + n * lbm::kPlanes * h->elem;
    if (bytes < need) return fail(h, LBM_ERR_ARG, "state buffer of %zu bytes, need %zu", bytes, need);
    const char* p = static_cast<const char*>(buf) + sizeof(hd);
    std::vector<uint32_t> sched(size_t(hd.n_sched));
    if (hd.n_sched) std::memcpy(sched.data(), p, sched.size() * 4);
    p += sched.size() * 4;
    // the populations may not be aligned inside a caller's buffer
    std::vector<uint8_t> pop(n * lbm::kPlanes * h->elem);
    std::memcpy(pop.data(), p, pop.size());
    lbm_status s = stored_in(h, pop.data());
    if (s != LBM_OK) return s;
    h->step = hd.step;
    h->period = hd.period;
    h->fixed_mask = hd.fixed_mask;
    h->schedule = std::move(sched);
    return LBM_OK;
}

lbm_status lbm_adjoint(lbm_handle h, const lbm_objective* obj, int64_t n, int32_t K, double* J,
                       double* dJ_dtau_c, double* dJ_du_in, double* dJ_dC_in)
{
    Range range("lbm_adjoint");
    if (check_ctx(h)) return LBM_ERR_ARG;
    if (h->precision != LBM_FP32) return fail(h, LBM_ERR_STATE, "%s needs FP32 storage", "lbm_adjoint");
    if (!h->inst.empty()) return fail(h, LBM_ERR_STATE, "%s works on a single chip, not a batch", "lbm_adjoint");
    if (h->decay != 0.f || h->paper_ports || h->wall_scheme != LBM_WALL_BOUNCE_BACK)
        return fail(h, LBM_ERR_STATE, "lbm_adjoint needs Zou-He ports, bounce-back walls and no decay");
    if (!obj || !J || !dJ_dtau_c) return fail(h, LBM_ERR_ARG, "objective, J or dJ_dtau_c is NULL");
    if (n < 1 || K < 1) return fail(h, LBM_ERR_ARG, "n_steps = %lld and ckpt_every = %d must be >= 1", (long long)n, K);
    if (obj->n < 1 || !obj->x || !obj->y || !obj->target || !obj->weight)
        return fail(h, LBM_ERR_ARG, "the objective needs n >= 1 nodes and all four arrays");
    for (int k = 0; k < obj->n; ++k) {
        const int x = obj->x[k], y = obj->y[k];
        if (x < 0 || x >= h->nx || y < 0 || y >= h->ny || h->solid[size_t(y) * h->nx + x])
            return fail(h, LBM_ERR_ARG, "objective node %d at (%d, %d) is not a fluid node", k, x, y);
        if (!std::isfinite(obj->target[k]) || !std::isfinite(obj->weight[k]))
            return fail(h, LBM_ERR_ARG, "objective node %d has a non-finite target or weight", k);
    }
    const long long n_ck = (n + K - 1) / K;
    const int seg_slots = int(std::min<int64_t>(K, n)) - 1;
    const size_t S = size_t(h->plane) * lbm::kPlanes * sizeof(float);
    cudaStream_t st = h->stream;

    int sms = 0, per_sm = 0;
    LBM_CUDA(h, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device));
    const int ablock = lbm::kAdjointBlock;
    LBM_CUDA(h, lbm::adjoint_occupancy(&per_sm));
    const int agrid = std::max(1, std::min((h->n_tiles + ablock / 32 - 1) / (ablock / 32), std::max(1, per_sm) * sms));

    Scratch tmp(h);
    char* ckpt = static_cast<char*>(tmp.get(size_t(n_ck) * S));
    char* seg = seg_slots > 0 ? static_cast<char*>(tmp.get(size_t(seg_slots) * S)) : nullptr;
    float* adj[3] = {static_cast<float*>(tmp.get(S)), static_cast<float*>(tmp.get(S)), static_cast<float*>(tmp.get(S))};
    float* dn = static_cast<float*>(tmp.get(size_t(2) * h->ny * sizeof(float)));
    double* gw = static_cast<double*>(tmp.get(size_t(agrid) * sizeof(double)));
    double* gu = static_cast<double*>(tmp.get(size_t(2) * h->ny * sizeof(double)));
    double* gc = static_cast<double*>(tmp.get(size_t(2) * h->ny * sizeof(double)));
    double* dJ = static_cast<double*>(tmp.get(2 * sizeof(double)));
    int* ox = static_cast<int*>(tmp.get(size_t(obj->n) * sizeof(int)));
    int* oy = static_cast<int*>(tmp.get(size_t(obj->n) * sizeof(int)));
    float* ot = static_cast<float*>(tmp.get(size_t(obj->n) * sizeof(float)));
    float* ow = static_cast<float*>(tmp.get(size_t(obj->n) * sizeof(float)));
    // multi_step: the valve word of every step t0 .. t0 + n for the reverse kernel
    const bool coop = h->multi_step > 0;
    uint32_t* masks_d = coop ? static_cast<uint32_t*>(tmp.get(size_t(n + 1) * sizeof(uint32_t))) : nullptr;
    int coop_grid = 0;
    if (coop) {
        int cps = 0;
        LBM_CUDA(h, lbm::adjoint_coop_occupancy(&cps));
        coop_grid = std::max(1, std::min(agrid, std::max(1, cps) * sms));
    }
    if (!ckpt || (seg_slots > 0 && !seg) || !adj[0] || !adj[1] || !adj[2] || !dn || !gw || !gu || !gc || !dJ ||
        !ox || !oy || !ot || !ow || (coop && !masks_d))
        return fail(h, LBM_ERR_OOM, "adjoint: device memory for %lld checkpoints and %d recomputed states not available",
                    n_ck, seg_slots);

    // forward sweep with checkpoints (the handle advances as in lbm_step)
    Range forward_range("lbm_adjoint: forward sweep");
    lbm::StepArgs a{};
    a.links = h->links;
    a.rowbc = h->rowbc;
    a.tiles = h->tiles;
    a.n_tiles = h->n_tiles;
    a.n_plain = h->n_plain;
    a.tiles64 = h->tiles64;
    a.n_tiles64 = h->n_tiles64;
    a.ny = h->ny;
    a.pitch = h->pitch;
    a.plane = h->plane;
    a.omega_f = float(1.0 / h->tau);
    a.omega_g = float(1.0 / h->tau_c);
    a.wg0 = h->wg0;
    a.wg1 = h->wg1;
    a.inv_cs2g = h->inv_cs2g;
    // Only the sweep's last step forms diagnostics: the call leaves those of
    // its final state, and nothing reads the others.
    a.partials = nullptr;
    a.err = h->err;
    const int64_t t0 = h->step;
    if (lbm_status js = join_scalar(h)) return js;
    a.barrier_extra = h->barrier_extra;
    // Forward steps t = tstart .. tstart + m - 1 of the run, step t reading
    // slot (t - tstart) of `from` and writing the next slot (every state
    // kept); with multi_step, runs of unchanged valve words go to the
    // cooperative kernel.
    auto forward_slots = [&](lbm::StepArgs& x, float* from, int64_t tstart, int64_t m) -> lbm_status {
        const long long stride = (long long)(S / sizeof(float));
        for (int64_t s = 0; s < m;) {
            const int64_t run = coop ? h->mask_run(t0 + tstart + s, std::min<int64_t>(m - s, h->multi_step)) : 1;
            x.open_mask[0] = h->mask_at(t0 + tstart + s);
            x.reverse = int((tstart + s) & 1);
            x.src = from + s * stride;
            cudaError_t e;
            if (run >= 2) {
                e = lbm::launch_steps_coop(x, int(run), stride, h->bar, h->coop_grid, kDefaultRegsBlock, st);
            } else {
                x.dst = from + (s + 1) * stride;
                e = lbm::launch_step(x, h->launch, st);
            }
            if (e != cudaSuccess) return cuda_fail(h, e, "forward step launch");
            s += std::max<int64_t>(run, 1);
        }
        return LBM_OK;
    };
    if (K == 1 && coop) {
        // every state kept, runs of steps in cooperative launches; the last
        // step writes into the other buffer
        LBM_CUDA(h, cudaMemcpyAsync(ckpt, h->pop[h->cur], S, cudaMemcpyDeviceToDevice, st));
        if (lbm_status fs = forward_slots(a, reinterpret_cast<float*>(ckpt), 0, n - 1)) return fs;
        a.src = reinterpret_cast<float*>(ckpt + size_t(n - 1) * S);
        a.dst = h->pop[1 - h->cur];
        a.reverse = int((n - 1) & 1);
        a.open_mask[0] = h->mask_at(t0 + n - 1);
        a.partials = h->partials;
        cudaError_t e = lbm::launch_step(a, h->launch, st);
        if (e != cudaSuccess) return cuda_fail(h, e, "coupled step launch");
        h->cur = 1 - h->cur;
        h->gbuf = h->cur;
        h->diag_grid = h->launch.grid;
        h->step += n;
    } else if (K == 1) {
        // every state kept: the steps write straight into the state array
        // (no copies, no recomputation), the last one into the other buffer
        LBM_CUDA(h, cudaMemcpyAsync(ckpt, h->pop[h->cur], S, cudaMemcpyDeviceToDevice, st));
        for (int64_t t = 0; t < n; ++t) {
            a.src = t == 0 ? h->pop[h->cur] : reinterpret_cast<float*>(ckpt + size_t(t) * S);
            a.dst = t + 1 < n ? reinterpret_cast<float*>(ckpt + size_t(t + 1) * S) : h->pop[1 - h->cur];
            a.reverse = int(t & 1);
            a.open_mask[0] = h->mask_at(t0 + t);
            a.partials = t + 1 < n ? nullptr : h->partials;
            cudaError_t e = lbm::launch_step(a, h->launch, st);
            if (e != cudaSuccess) return cuda_fail(h, e, "coupled step launch");
        }
        h->cur = 1 - h->cur;
        h->gbuf = h->cur;
        h->diag_grid = h->launch.grid;
        h->step += n;
    } else {
        // a checkpoint every K steps; the states of the last segment go
        // straight into the segment slots (its checkpoint, then slots 1 ..
        // len - 1), where the reverse sweep starts, so that segment is never
        // recomputed
        const int64_t s_last = (n_ck - 1) * K;
        for (int64_t t = 0; t < s_last; ++t) {
            if (t % K == 0)
                LBM_CUDA(h, cudaMemcpyAsync(ckpt + size_t(t / K) * S, h->pop[h->cur], S, cudaMemcpyDeviceToDevice, st));
            a.src = h->pop[h->cur];
            a.dst = h->pop[1 - h->cur];
            a.reverse = h->cur;
            a.open_mask[0] = h->mask_at(t0 + t);
            cudaError_t e = lbm::launch_step(a, h->launch, st);
            if (e != cudaSuccess) return cuda_fail(h, e, "coupled step launch");
            h->cur = 1 - h->cur;
            h->gbuf = h->cur;
            h->diag_grid = h->launch.grid;
            ++h->step;
        }
        float* last = reinterpret_cast<float*>(ckpt + size_t(n_ck - 1) * S);
        LBM_CUDA(h, cudaMemcpyAsync(last, h->pop[h->cur], S, cudaMemcpyDeviceToDevice, st));
        const int64_t len = n - s_last;
        if (len >= 2) {
            float* slot1 = reinterpret_cast<float*>(seg);
            a.src = last;
            a.dst = slot1;
            a.reverse = h->cur;
            a.open_mask[0] = h->mask_at(t0 + s_last);
            cudaError_t e = lbm::launch_step(a, h->launch, st);
            if (e != cudaSuccess) return cuda_fail(h, e, "coupled step launch");
            if (lbm_status fs = forward_slots(a, slot1, s_last + 1, len - 2)) return fs;
            last = reinterpret_cast<float*>(seg + size_t(len - 2) * S);
        }
        a.src = last;
        a.dst = h->pop[1 - h->cur];
        a.reverse = int((h->cur + len - 1) & 1);
        a.open_mask[0] = h->mask_at(t0 + n - 1);
        a.partials = h->partials;
        cudaError_t e = lbm::launch_step(a, h->launch, st);
        if (e != cudaSuccess) return cuda_fail(h, e, "coupled step launch");
        h->cur = 1 - h->cur;
        h->gbuf = h->cur;
        h->diag_grid = h->launch.grid;
        h->step += len;
    }

    forward_range.end();
    // J and dJ/dP(n)
    std::vector<int> hx(obj->x, obj->x + obj->n), hy(obj->y, obj->y + obj->n);
    LBM_CUDA(h, cudaMemcpyAsync(ox, hx.data(), hx.size() * sizeof(int), cudaMemcpyHostToDevice, st));
    LBM_CUDA(h, cudaMemcpyAsync(oy, hy.data(), hy.size() * sizeof(int), cudaMemcpyHostToDevice, st));
    LBM_CUDA(h, cudaMemcpyAsync(ot, obj->target, size_t(obj->n) * sizeof(float), cudaMemcpyHostToDevice, st));
    LBM_CUDA(h, cudaMemcpyAsync(ow, obj->weight, size_t(obj->n) * sizeof(float), cudaMemcpyHostToDevice, st));
    for (float* b : adj) LBM_CUDA(h, cudaMemsetAsync(b, 0, S, st));
    LBM_CUDA(h, cudaMemsetAsync(gw, 0, size_t(agrid) * sizeof(double), st));
    LBM_CUDA(h, cudaMemsetAsync(gu, 0, size_t(2) * h->ny * sizeof(double), st));
    LBM_CUDA(h, cudaMemsetAsync(gc, 0, size_t(2) * h->ny * sizeof(double), st));
    LBM_CUDA(h, cudaMemsetAsync(dn, 0, size_t(2) * h->ny * sizeof(float), st));
    std::vector<uint32_t> masks_h;
    if (coop) {
        masks_h.resize(size_t(n + 1));
        for (int64_t t = 0; t <= n; ++t) masks_h[size_t(t)] = h->mask_at(t0 + t);
        LBM_CUDA(h, cudaMemcpyAsync(masks_d, masks_h.data(), masks_h.size() * sizeof(uint32_t), cudaMemcpyHostToDevice,
                                    st));
    }
    {
        cudaError_t e = lbm::launch_adjoint_seed(h->pop[h->cur], h->plane, h->pitch, ox, oy, ot, ow, obj->n, adj[0],
                                                 dJ, st);
        if (e != cudaSuccess) return cuda_fail(h, e, "adjoint seed launch");
    }

    // backward, segment by segment
    Range reverse_range("lbm_adjoint: recomputation and reverse sweep");
    lbm::AdjointArgs A{};
    A.links = h->links;
    A.rowbc = h->rowbc;
    A.tiles = h->tiles;
    A.n_tiles = h->n_tiles;
    A.ny = h->ny;
    A.pitch = h->pitch;
    A.plane = h->plane;
    A.omega_f = a.omega_f;
    A.omega_g = a.omega_g;
    A.wg0 = h->wg0;
    A.wg1 = h->wg1;
    A.inv_cs2g = h->inv_cs2g;
    A.dn = dn;
    A.grad_w = gw;
    A.grad_u = gu;
    A.grad_c = gc;
    A.err = h->err;
    A.barrier_extra = h->barrier_extra;
    lbm::StepArgs r = a;
    r.partials = nullptr;  // recomputed states only: the diagnostics stay those of the last forward step
    // adj[0] holds A(n); M(t) alternates between adj[1] and adj[2]
    int mid = 0;  // 0 before the first reverse step, else adj[mid] holds M(t+1)
    // One reverse step t (state `state`): the first one reads A(n), the
    // others gather M(t + 1).
    auto reverse_one = [&](int64_t t, const float* state) -> lbm_status {
        A.state = state;
        A.adj_next = adj[0];
        A.mid_next = mid ? adj[mid] : nullptr;
        A.adj_mid = adj[mid == 1 ? 2 : 1];
        A.open_mask = h->mask_at(t0 + t);
        A.open_mask_next = h->mask_at(t0 + t + 1);
        A.reverse = int((n - 1 - t) & 1);
        cudaError_t e = lbm::launch_adjoint_step(A, mid == 0, agrid, st);
        if (e != cudaSuccess) return cuda_fail(h, e, "adjoint step launch");
        mid = mid == 1 ? 2 : 1;
        return LBM_OK;
    };
    // Reverse steps t_hi down to t_lo (all after the first), the state of
    // step t at state_lo + (t - t_lo) slots, in cooperative launches of at
    // most multi_step steps.
    auto reverse_coop = [&](int64_t t_hi, int64_t t_lo, const float* state_lo) -> lbm_status {
        const long long stride = (long long)(S / sizeof(float));
        for (int64_t hi = t_hi; hi >= t_lo;) {
            const int64_t lo = std::max<int64_t>(t_lo, hi - h->multi_step + 1);
            A.reverse = int((n - 1 - hi) & 1);
            cudaError_t e = lbm::launch_adjoint_steps_coop(A, int(hi - lo), 0, state_lo + (lo - t_lo) * stride, stride,
                                                           masks_d + lo, adj[mid], adj[3 - mid], h->bar, coop_grid,
                                                           st);
            if (e != cudaSuccess) return cuda_fail(h, e, "multi-step adjoint launch");
            if ((hi - lo + 1) & 1) mid = 3 - mid;
            hi = lo - 1;
        }
        return LBM_OK;
    };
    if (coop && K == 1) {
        // every state kept: the first reverse step, then all others in
        // cooperative launches
        if (lbm_status rs = reverse_one(n - 1, reinterpret_cast<float*>(ckpt + size_t(n - 1) * S))) return rs;
        if (n >= 2)
            if (lbm_status rs = reverse_coop(n - 2, 0, reinterpret_cast<float*>(ckpt))) return rs;
    }
    for (long long sg = n_ck - 1; sg >= 0 && !(coop && K == 1); --sg) {
        const int64_t s0 = sg * K;
        const int len = int(std::min<int64_t>(K, n - s0));
        auto state = [&](int j) -> float* {
            return reinterpret_cast<float*>(j == 0 ? ckpt + size_t(sg) * S : seg + size_t(j - 1) * S);
        };
        // recompute the segment's states 1 .. len - 1 from its checkpoint
        // (the last segment's are still there from the forward sweep)
        if (len >= 2 && sg != n_ck - 1) {
            r.src = state(0);
            r.dst = state(1);
            r.reverse = 1;
            r.open_mask[0] = h->mask_at(t0 + s0);
            cudaError_t e = lbm::launch_step(r, h->launch, st);
            if (e != cudaSuccess) return cuda_fail(h, e, "recompute step launch");
            if (lbm_status fs = forward_slots(r, state(1), s0 + 1, len - 2)) return fs;
        }
        int j_hi = len - 1;
        if (mid == 0) {  // the first reverse step of the sweep
            if (lbm_status rs = reverse_one(s0 + j_hi, state(j_hi))) return rs;
            --j_hi;
        }
        if (coop && j_hi >= 1) {
            if (lbm_status rs = reverse_coop(s0 + j_hi, s0 + 1, state(1))) return rs;
            j_hi = 0;
        }
        for (int j = j_hi; j >= 0; --j)
            if (lbm_status rs = reverse_one(s0 + j, state(j))) return rs;
    }
    {
        cudaError_t e = lbm::launch_sum_doubles(gw, agrid, dJ + 1, st);
        if (e != cudaSuccess) return cuda_fail(h, e, "gradient reduction launch");
    }
    double host[2];
    LBM_CUDA(h, cudaMemcpyAsync(host, dJ, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    if (dJ_du_in) LBM_CUDA(h, cudaMemcpyAsync(dJ_du_in, gu, size_t(2) * h->ny * sizeof(double), cudaMemcpyDeviceToHost, st));
    if (dJ_dC_in) LBM_CUDA(h, cudaMemcpyAsync(dJ_dC_in, gc, size_t(2) * h->ny * sizeof(double), cudaMemcpyDeviceToHost, st));
    LBM_CUDA(h, cudaStreamSynchronize(st));
    *J = host[0];
    *dJ_dtau_c = -host[1] / (h->tau_c * h->tau_c);  // d(1/tau_c)/dtau_c = -1/tau_c^2
    return read_err_word(h);
}

namespace {
float* field_slot(lbm_ctx* h, uint32_t word)
{
    for (auto& f : h->fields)
        if (f.word == word) return f.u;
    if (int(h->fields.size()) >= LBM_MAX_FIELDS) return nullptr;
    float* u = static_cast<float*>(dev_alloc(h, size_t(2) * h->plane * sizeof(float)));
    if (u) h->fields.push_back({word, u});
    return u;
}
const float* find_field(const lbm_ctx* h, uint32_t word)
{
    for (auto& f : h->fields)
        if (f.word == word) return f.u;
    return nullptr;
}
}  // namespace

lbm_status lbm_store_velocity(lbm_handle h, uint32_t open_mask)
{
    if (check_ctx(h)) return LBM_ERR_ARG;
    if (h->precision != LBM_FP32) return fail(h, LBM_ERR_STATE, "%s needs FP32 storage", "lbm_store_velocity");
    if (!h->inst.empty()) return fail(h, LBM_ERR_STATE, "%s works on a single chip, not a batch", "lbm_store_velocity");
    float* u = field_slot(h, open_mask);
    if (!u) return fail(h, LBM_ERR_OOM, "no room for the velocity field of valve word %u (at most %d fields)",
                        open_mask, LBM_MAX_FIELDS);
    cudaError_t e = lbm::launch_velocity_of_state(h->pop[h->cur], h->links, h->plane, u, u + h->plane, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "velocity kernel launch");
    return LBM_OK;
}

lbm_status lbm_set_velocity_field(lbm_handle h, uint32_t open_mask, const float* ux, const float* uy)
{
    if (check_ctx(h)) return LBM_ERR_ARG;
    if (h->precision != LBM_FP32) return fail(h, LBM_ERR_STATE, "%s needs FP32 storage", "lbm_set_velocity_field");
    if (!h->inst.empty()) return fail(h, LBM_ERR_STATE, "%s works on a single chip, not a batch", "lbm_set_velocity_field");
    if (!ux || !uy) return fail(h, LBM_ERR_ARG, "ux or uy is NULL");
    float* u = field_slot(h, open_mask);
    if (!u) return fail(h, LBM_ERR_OOM, "no room for the velocity field of valve word %u (at most %d fields)",
                        open_mask, LBM_MAX_FIELDS);
    const size_t row = size_t(h->nx) * sizeof(float), pitch = size_t(h->pitch) * sizeof(float);
    LBM_CUDA(h, cudaMemcpy2DAsync(u, pitch, ux, row, row, size_t(h->ny), cudaMemcpyHostToDevice, h->stream));
    LBM_CUDA(h, cudaMemcpy2DAsync(u + h->plane, pitch, uy, row, row, size_t(h->ny), cudaMemcpyHostToDevice, h->stream));
    LBM_CUDA(h, cudaStreamSynchronize(h->stream));
    return LBM_OK;
}

lbm_status lbm_scalar_step(lbm_handle h, int64_t n, double u_scale)
{
    Range range("lbm_scalar_step");
    if (check_ctx(h)) return LBM_ERR_ARG;
    if (h->precision != LBM_FP32) return fail(h, LBM_ERR_STATE, "%s needs FP32 storage", "lbm_scalar_step");
    if (!h->inst.empty()) return fail(h, LBM_ERR_STATE, "%s works on a single chip, not a batch", "lbm_scalar_step");
    if (n < 0) return fail(h, LBM_ERR_ARG, "n = %lld < 0", (long long)n);
    if (!std::isfinite(u_scale)) return fail(h, LBM_ERR_ARG, "u_scale = %g is not finite", u_scale);
    // every valve word the steps use needs a field
    const std::vector<uint32_t> words = h->schedule.empty() ? std::vector<uint32_t>{h->fixed_mask} : h->schedule;
    const int64_t reach = h->schedule.empty() ? 1 : std::min<int64_t>(int64_t(words.size()), (n + h->period - 1) / h->period + 1);
    for (int64_t k = 0; k < reach && n > 0; ++k) {
        const uint32_t w = h->schedule.empty() ? words[0] : h->mask_at(h->step + k * h->period);
        if (!find_field(h, w)) return fail(h, LBM_ERR_STATE, "no stored velocity field for valve word %u", w);
    }
    lbm::ScalarArgs a{};
    a.links = h->links;
    a.rowbc = h->rowbc;
    a.tiles = h->tiles;
    a.n_tiles = h->n_tiles;
    a.ny = h->ny;
    a.pitch = h->pitch;
    a.plane = h->plane;
    a.u_scale = float(u_scale);
    a.omega_g = float(1.0 / h->tau_c);
    a.wg0 = h->wg0;
    a.wg1 = h->wg1;
    a.inv_cs2g = h->inv_cs2g;
    a.decay = h->decay;
    a.partials = h->partials;
    a.fluid_blocks = h->diag_grid;
    a.err = h->err;
    if (h->scalar_grid == 0) {
        // one wave of resident blocks of the scalar kernel
        int per_sm = 0;
        if (h->scalar_regs) LBM_CUDA(h, lbm::scalar_regs_occupancy(kScalarRegsBlock, &per_sm));
        else LBM_CUDA(h, lbm::scalar_bulk_occupancy(kScalarConsumers, kScalarStagesPer, &per_sm));
        const int tiles_per_block = h->scalar_regs ? kScalarRegsBlock / 32 : 1;
        h->scalar_grid = std::max(1, std::min((h->n_tiles + tiles_per_block - 1) / tiles_per_block,
                                              std::max(1, per_sm) * h->sms));
    }
    const int scalar_grid = std::min(h->scalar_grid, h->partials_cap);
    a.n_partials = std::max(h->diag_grid, scalar_grid);
    int g = h->gbuf;  // buffer holding the current scalar planes
    for (int64_t k = 0; k < n; ++k) {
        const uint32_t w = h->mask_at(h->step);
        const float* u = find_field(h, w);
        if (!u) {
            h->gbuf = g;
            return fail(h, LBM_ERR_STATE, "no stored velocity field for valve word %u", w);
        }
        a.src = h->pop[g] + 9 * h->plane;
        a.dst = h->pop[1 - g] + 9 * h->plane;
        a.reverse = g;
        a.ux = u;
        a.uy = u + h->plane;
        a.open_mask = w;
        cudaError_t e = h->scalar_regs
                            ? lbm::launch_scalar_step_regs(a, scalar_grid, kScalarRegsBlock, h->stream)
                            : lbm::launch_scalar_step_bulk(a, scalar_grid, kScalarConsumers, kScalarStagesPer, h->stream);
        if (e != cudaSuccess) {
            h->gbuf = g;
            return cuda_fail(h, e, "scalar step launch");
        }
        g = 1 - g;
        ++h->step;
    }
    h->gbuf = g;  // joined with the fluid planes when a call needs both
    if (n > 0) h->diag_grid = std::max(h->diag_grid, scalar_grid);
    return pending_numeric(h);
}

lbm_status lbm_get_step(lbm_handle h, int64_t* t)
{
    if (check_ctx(h) || !t) return fail(h, LBM_ERR_ARG, "t is NULL");
    *t = h->step;
    return LBM_OK;
}

lbm_status lbm_autotune(lbm_handle h, int32_t trial_steps)
{
    Range range("lbm_autotune");
    if (check_ctx(h)) return LBM_ERR_ARG;
    if (trial_steps < 0 || trial_steps > 10000) return fail(h, LBM_ERR_ARG, "trial_steps = %d outside [0, 10000]", trial_steps);
    // 0: a first timing of 20 steps of the first shape sets a count for
    // which a trial lasts about 2 ms (between 20 and 2000 steps): 20 steps
    // of a chip of a few microseconds per step are too short to tell
    // shapes a few percent apart
    bool size_trials = trial_steps == 0;
    if (size_trials) trial_steps = 20;
    if (lbm_status js = join_scalar(h)) return js;
    // candidate shapes: {variant, block (variant 1) or computing warps, stages per computing warp}
    struct Cand { int variant, warps, per; };
    std::vector<Cand> cands = {{1, 4, 0}, {1, 8, 0}, {4, 2, 0}, {4, 4, 0}, {2, 2, 1}, {2, 3, 1},
                               {2, 4, 1}, {2, 2, 2}, {2, 3, 2}, {2, 4, 2}};
    if (h->precision == LBM_FP32) cands.push_back({3, 4, 1});
    else cands.push_back({2, 3, 3});
    if (h->precision == LBM_FP32 && !h->wallv) cands.push_back({5, 4, 0});
    // trials step between two scratch copies of the state, alternating the
    // tile order like lbm_step (the L2 reuse of consecutive steps is part of
    // what is timed): the state, step count and diagnostics stay as they are
    Scratch sc(h);
    const size_t state_bytes = size_t(h->plane) * lbm::kPlanes * h->elem;
    void* buf0 = sc.get(state_bytes);
    void* buf1 = sc.get(state_bytes);
    float2* part = static_cast<float2*>(sc.get(size_t(h->partials_cap) * 4 * sizeof(float2)));
    unsigned* err = static_cast<unsigned*>(sc.get(sizeof(unsigned)));
    if (!buf0 || !buf1 || !part || !err) return fail(h, LBM_ERR_OOM, "no device memory for the trial steps");
    LBM_CUDA(h, lbm::prepare_step_kernels());
    LBM_CUDA(h, cudaMemcpyAsync(buf0, h->pop[h->cur], state_bytes, cudaMemcpyDeviceToDevice, h->stream));
    float* const bufs[2] = {static_cast<float*>(buf0), static_cast<float*>(buf1)};
    lbm::StepArgs a{};
    a.src = bufs[0];
    a.dst = bufs[1];
    a.links = h->links;
    a.rowbc = h->rowbc;
    a.tiles = h->tiles;
    a.n_tiles = h->n_tiles;
    a.n_plain = h->n_plain;
    a.tiles64 = h->tiles64;
    a.n_tiles64 = h->n_tiles64;
    a.ny = h->ny;
    a.pitch = h->pitch;
    a.plane = h->plane;
    a.omega_f = float(1.0 / h->tau);
    a.omega_g = float(1.0 / h->tau_c);
    a.rates = h->rates;
    a.wg0 = h->wg0;
    a.wg1 = h->wg1;
    a.inv_cs2g = h->inv_cs2g;
    a.decay = h->decay;
    a.wallv = h->wallv;
    a.partials = part;
    a.err = err;
    if (h->precision != LBM_FP32) {
        a.gref0 = h->wg0 * lbm::kCRef;
        a.gref1 = h->wg1 * lbm::kCRef;
    }
    h->mask_words(h->step, a.open_mask);
    if (h->wallv)
        LBM_CUDA(h, lbm::launch_wall_values(a.src, h->wallv, h->links, h->woff, h->n_wall, h->plane, h->pitch,
                                            h->precision, h->stream));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    LBM_CUDA(h, cudaEventCreate(&e0));
    cudaError_t e = cudaEventCreate(&e1);
    lbm::StepLaunch best{};
    float best_ms = 0.f;
    for (const Cand& c : cands) {
        if (e != cudaSuccess) break;
        lbm::StepLaunch L{};
        L.precision = h->precision;
        L.pdl = true;
        L.walls = h->wallv != nullptr;
        if (L.walls && (c.variant == 3 || c.variant == 4)) continue;
        if (c.variant == 1 || c.variant == 4 || c.variant == 5) {
            L.variant = c.variant == 1 ? lbm::kVariantRegs : c.variant == 4 ? lbm::kVariantAsync : lbm::kVariantPairs;
            L.block = 32 * c.warps;
            L.stages = 0;
        } else if (c.variant == 2) {
            L.variant = lbm::kVariantBulk;
            L.block = 32 * (c.warps + 1);
            L.stages = c.warps * c.per;
        } else {
            L.variant = lbm::kVariantPipe;
            L.block = 32 * c.warps;
            L.stages = c.warps * c.per;
        }
        int per_sm = 0;
        if (lbm::step_kernel_occupancy(L, &per_sm) != cudaSuccess || per_sm < 1) {
            cudaGetLastError();
            continue;
        }
        L.grid = std::min(wave_grid(h, L, per_sm), h->partials_cap);
        e = arrange_tiles(h, L);  // each shape is timed with its own tile order
        if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(unsigned), h->stream);
        // the step kernel alone (the wall values, when used, are computed
        // once above from the current state); the better of two trials
        int64_t k = 0;  // launches of this shape so far: buffers and tile order alternate
        auto trial_step = [&]() {
            a.src = bufs[k & 1];
            a.dst = bufs[1 - (k & 1)];
            a.reverse = int(k & 1);
            ++k;
            return lbm::launch_step(a, L, h->stream);
        };
        for (int j = 0; j < 3 && e == cudaSuccess; ++j) e = trial_step();
        float ms = 0.f;
        for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {
            if (e == cudaSuccess) e = cudaEventRecord(e0, h->stream);
            for (int j = 0; j < trial_steps && e == cudaSuccess; ++j) e = trial_step();
            if (e == cudaSuccess) e = cudaEventRecord(e1, h->stream);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float t = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
            if (e == cudaSuccess && size_trials) {
                // once, before any comparison: resize and time this shape again
                const double want = std::ceil(2.0 * trial_steps / std::max(double(t), 1e-3));
                trial_steps = int(std::min(2000.0, std::max(double(trial_steps), want)));
                size_trials = false;
                --rep;
                continue;
            }
            if (rep == 0 || t < ms) ms = t;
        }
        unsigned ew = 0;
        if (e == cudaSuccess) e = cudaMemcpy(&ew, err, sizeof(unsigned), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess && (ew & 2u) == 0 && (best.grid == 0 || ms < best_ms)) {
            best = L;
            best_ms = ms;
        }
    }
    cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_fail(h, e, "autotune trial");
    if (best.grid == 0) return fail(h, LBM_ERR_STATE, "no launch shape completed its trial steps");
    if (best.variant != h->launch.variant || best.block != h->launch.block || best.stages != h->launch.stages ||
        best.grid != h->launch.grid) {
        LBM_CUDA(h, cudaStreamSynchronize(h->stream));
        for (auto& g : h->graphs) cudaGraphExecDestroy(g.exec);  // captured with the old shape
        h->graphs.clear();
        h->launch = best;
    }
    LBM_CUDA(h, arrange_tiles(h, h->launch));  // the order of the shape kept
    return LBM_OK;
}

lbm_status lbm_get_info(lbm_handle h, lbm_info* info)
{
    if (check_ctx(h) || !info) return fail(h, LBM_ERR_ARG, "info is NULL");
    info->nx = h->nx;
    info->ny = h->ny;
    info->pitch = h->pitch;
    info->n_tiles = h->n_tiles;
    info->grid = h->launch.grid;
    info->block = h->launch.block;
    info->variant = h->launch.variant;
    info->stages = h->launch.stages;
    info->fluid_nodes = h->fluid;
    info->algorithmic_bytes_per_step = h->fluid * 28 * (long long)h->elem;
    info->device_bytes = h->device_bytes;
    info->precision = h->precision;
    info->instances = h->inst.empty() ? 1 : int32_t(h->inst.size());
    return LBM_OK;
}

}  // extern "C"
