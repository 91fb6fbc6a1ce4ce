// lbm_noalloc.cu -- lbm_step_noalloc: one coupled time step on caller-owned
// device buffers, allocating nothing.
//
// For callers that cannot allocate device memory through the library (code
// living inside another framework's memory pool, or under a rule that
// forbids cudaMalloc after start-up).  The step kernel is the library's
// ordinary one; its only scratch memory, the per-block diagnostics partial
// sums, lives in the fixed array below instead of a handle's allocation.
#include <cstdarg>
#include <cstddef>
#include <cstdio>
#include <mutex>

#include "lbm.h"
#include "lbm_internal.h"

namespace {

constexpr int kMaxDevices = 64;
// launch shape: the bulk-copy pipeline with its default shape
constexpr int kConsumers = 3;
constexpr int kStagesPerConsumer = 1;

// Per-block partial sums of the four diagnostics, 4 double-float pairs (8
// bytes each) per block of the step kernel.  A fixed 64 KiB that every GPU loading the library keeps until
// the process exits; host code reaches it only through the address returned
// by cudaGetSymbolAddress for the current device.
static __device__ __align__(256) float2 g_step_scratch[LBM_NOALLOC_MAX_BLOCKS * 4];

struct DeviceSetup {
    bool ready;
    float2* scratch;  // device address of g_step_scratch on this device
    int grid_cap;     // one wave of resident blocks, at most LBM_NOALLOC_MAX_BLOCKS
};
DeviceSetup g_setup[kMaxDevices];
std::mutex g_setup_mutex;

static_assert(sizeof(lbm_row_port) == sizeof(lbm::RowBC), "lbm_row_port must match the kernel's port entry");
static_assert(offsetof(lbm_row_port, a) == offsetof(lbm::RowBC, a), "lbm_row_port layout");
static_assert(sizeof(lbm_tile) == sizeof(uint2), "lbm_tile must match the kernel's tile entry");

lbm_status reject(const lbm_noalloc_step* s, lbm_status st, const char* fmt, ...)
{
    if (s && s->message && s->message_len > 0) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(s->message, size_t(s->message_len), fmt, ap);
        va_end(ap);
    }
    return st;
}

bool aligned(const void* p, size_t a)
{
    return (reinterpret_cast<uintptr_t>(p) & (a - 1)) == 0;
}

// Once per device, with that device current: the scratch array's device
// address and the launch shape.  No allocation is made here.
lbm_status setup_device(const lbm_noalloc_step* s, int dev, DeviceSetup* out)
{
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    DeviceSetup& d = g_setup[dev];
    if (!d.ready) {
        float2* ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(reinterpret_cast<void**>(&ptr), g_step_scratch);
        if (e != cudaSuccess)
            return reject(s, LBM_ERR_CUDA, "cudaGetSymbolAddress of the step scratch: %s", cudaGetErrorString(e));
        e = lbm::prepare_step_kernels();
        if (e != cudaSuccess) return reject(s, LBM_ERR_CUDA, "shared-memory attribute: %s", cudaGetErrorString(e));
        int sms = 0, per_sm = 0;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return reject(s, LBM_ERR_CUDA, "SM count: %s", cudaGetErrorString(e));
        const lbm::StepLaunch probe{lbm::kVariantBulk, 1, 32 * (kConsumers + 1), kConsumers * kStagesPerConsumer};
        e = lbm::step_kernel_occupancy(probe, &per_sm);
        if (e != cudaSuccess || per_sm < 1)
            return reject(s, LBM_ERR_CUDA, "occupancy query: %s", cudaGetErrorString(e));
        const int cap = per_sm * sms;
        d.scratch = ptr;
        d.grid_cap = cap < LBM_NOALLOC_MAX_BLOCKS ? cap : LBM_NOALLOC_MAX_BLOCKS;
        d.ready = true;
    }
    *out = d;
    return LBM_OK;
}

}  // namespace

extern "C" lbm_status lbm_step_noalloc(const lbm_noalloc_step* s)
{
    if (!s) return LBM_ERR_ARG;
    if (s->struct_size != sizeof(lbm_noalloc_step))
        return reject(s, LBM_ERR_ARG, "struct_size is %u, expected %zu", s->struct_size, sizeof(lbm_noalloc_step));
    if (s->nx < 1 || s->ny < 1 || s->ny >= lbm::kMaxRows || s->nx > lbm::kMaxCols)
        return reject(s, LBM_ERR_ARG, "grid %d x %d outside the supported range", s->nx, s->ny);
    if (s->pitch < s->nx || s->pitch % lbm::kTileNodes != 0)
        return reject(s, LBM_ERR_ARG, "pitch %d: use a multiple of %d that is at least nx = %d", s->pitch,
                      lbm::kTileNodes, s->nx);
    if (s->n_tiles < 0 || (long long)s->n_tiles > (long long)s->ny * (s->pitch / lbm::kTileNodes))
        return reject(s, LBM_ERR_ARG, "n_tiles = %d outside [0, rows x segments]", s->n_tiles);
    if (s->max_blocks < 0 || s->max_blocks > LBM_NOALLOC_MAX_BLOCKS)
        return reject(s, LBM_ERR_ARG, "max_blocks = %d: the fixed scratch holds at most %d blocks", s->max_blocks,
                      LBM_NOALLOC_MAX_BLOCKS);
    if (!s->src || !s->dst || !s->links || !s->ports || !s->err || (s->n_tiles > 0 && !s->tiles))
        return reject(s, LBM_ERR_ARG, "a required buffer pointer is NULL");
    if (!aligned(s->src, 16) || !aligned(s->dst, 16) || !aligned(s->links, 16) || !aligned(s->ports, 16) ||
        !aligned(s->tiles, 8) || !aligned(s->diag, 8) || !aligned(s->err, 4))
        return reject(s, LBM_ERR_ARG, "a buffer is not aligned (populations, links, ports: 16 bytes)");
    const size_t pop_bytes = size_t(s->ny) * size_t(s->pitch) * lbm::kPlanes * sizeof(float);
    const char* a0 = reinterpret_cast<const char*>(s->src);
    const char* b0 = reinterpret_cast<const char*>(s->dst);
    if (a0 < b0 + pop_bytes && b0 < a0 + pop_bytes) return reject(s, LBM_ERR_ARG, "src and dst overlap");
    if (!(s->tau > 0.5) || !(s->tau_c > 0.5) || !(s->tau < 1e30) || !(s->tau_c < 1e30))
        return reject(s, LBM_ERR_ARG, "tau = %g, tau_c = %g: relaxation times must exceed 1/2", s->tau, s->tau_c);
    if (!(s->w0 >= 0.0 && s->w0 < 1.0)) return reject(s, LBM_ERR_ARG, "w0 = %g outside [0, 1)", s->w0);

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return reject(s, LBM_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return reject(s, LBM_ERR_ARG, "device %d beyond %d", dev, kMaxDevices);
    DeviceSetup d;
    lbm_status st = setup_device(s, dev, &d);
    if (st != LBM_OK) return st;

    lbm::StepLaunch L{lbm::kVariantBulk, 0, 32 * (kConsumers + 1), kConsumers * kStagesPerConsumer};
    int grid = s->n_tiles < d.grid_cap ? s->n_tiles : d.grid_cap;
    if (s->max_blocks > 0 && grid > s->max_blocks) grid = s->max_blocks;
    L.grid = grid > 0 ? grid : 1;

    lbm::StepArgs a{};
    a.src = s->src;
    a.dst = s->dst;
    a.links = s->links;
    a.rowbc = reinterpret_cast<const lbm::RowBC*>(s->ports);
    a.tiles = reinterpret_cast<const uint2*>(s->tiles);
    a.n_tiles = s->n_tiles;
    a.ny = s->ny;
    a.pitch = s->pitch;
    a.plane = (long long)s->ny * s->pitch;
    a.omega_f = float(1.0 / s->tau);
    a.omega_g = float(1.0 / s->tau_c);
    a.wg0 = float(s->w0);
    a.wg1 = float(0.25 * (1.0 - s->w0));
    a.inv_cs2g = float(2.0 / (1.0 - s->w0));
    a.open_mask[0] = s->open_mask;  // channels 0..31; the other words stay 0
    a.partials = d.scratch;
    a.err = s->err;
    cudaStream_t stream = static_cast<cudaStream_t>(s->stream);
    e = lbm::launch_step(a, L, stream);
    if (e != cudaSuccess) return reject(s, LBM_ERR_CUDA, "coupled step launch: %s", cudaGetErrorString(e));
    if (s->diag) {
        e = lbm::launch_diag_finish(d.scratch, L.grid, s->diag, stream);
        if (e != cudaSuccess) return reject(s, LBM_ERR_CUDA, "diagnostics reduction launch: %s", cudaGetErrorString(e));
    }
    return LBM_OK;
}
