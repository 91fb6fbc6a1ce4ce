// lbm_kernels.cu -- sm_103a kernels of the coupled D2Q9 + scalar lattice
// Boltzmann step (Tanaka & Iber, arXiv 1307.4703, "Numerical Methods" and
// "Boundary Conditions").
//
// One launch advances the whole chip by one time step.  It is a pull scheme:
// node x gathers f_i from x - e_i (free flight of Eq. lbequation), replaces
// links that start on a wall by halfway bounce-back, completes open valve
// ports (Zou-He for f, held concentration or do-nothing for g), takes the
// moments of Eq. moments, relaxes f (Eq. lbequation) and then g towards the
// equilibrium of Eq. cdeequilibrium with the velocity just computed at the
// same node, and stores the post-collision populations.  Each element of the
// state is read once and written once per step, so the step is bound by HBM
// bandwidth; it contains no dense contraction and uses no tensor cores.
//
// Work decomposition: a warp owns a 128-node row segment (a "tile"), four
// consecutive nodes per lane, so every population plane is written with one
// aligned 128-bit store per lane.  Only segments that hold fluid are listed in
// the tile table, with the span of lanes that hold fluid.
//
// Two variants read the state:
//   coupled_step_bulk  (default) a producer warp per block streams each tile's
//                      14 plane rows and its wall-link bytes into a ring of
//                      shared-memory stages with cp.async.bulk copies that
//                      complete on mbarriers; consumer warps compute from
//                      shared memory.  The ring keeps far more bytes in flight
//                      per SM than registers could, which is what a
//                      bandwidth-bound stream needs.
//   coupled_step_regs  each lane loads its quads with 128-bit loads into
//                      registers; the +-1 column shifts travel between lanes
//                      by warp shuffle.  Instantiated for FP32 storage and for
//                      FP16 / BF16 storage (64-bit loads of four 16-bit
//                      deviations, FP32 arithmetic); so is the bulk variant.
// All share the per-node arithmetic of lbm_device.cuh; the FP32 variants give
// identical results.
#include <algorithm>

#include "lbm_step.cuh"

namespace lbm {
namespace {
// Totals of the block partials of the last step (finish_partials: the same
// order, and so the same bits, as the step kernels' own in-kernel totals).
// out may be page-locked host memory (written over the interconnect).
__global__ void diag_finish(const float2* partials, int n_blocks, double* out)
{
    grid_dependency_sync();  // the step kernel before it has written the partials
    finish_partials(partials, n_blocks, out);
}

// Many steps in one cooperative launch (every block resident): the register
// variant's tile loop once per step, the two buffers swapping roles (or,
// with seq_stride > 0, step s reading src + s seq_stride and writing the
// next slot), and a grid-wide barrier between steps in place of the launch
// boundary.  Loads go
// through L2 (F32Coherent): each step reads what other blocks wrote in the
// step before.  The valve words are those of a.open_mask for all n steps;
// the diagnostics partials are those of the last step.  A barrier that
// times out stops the kernel with bit 1 of the error word set.
__global__ void __launch_bounds__(256, 2) coupled_steps_coop(const StepArgs a, int n, long long seq_stride,
                                                             unsigned* count)
{
    using T = F32Coherent;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int wpb = blockDim.x >> 5;
    const int stride = gridDim.x * wpb;
    LaneDiag diag;
    bool bad = false;
    for (int s = 0; s < n; ++s) {
        float* const src = const_cast<float*>(a.src);  // both buffers are written
        const T* __restrict__ S = reinterpret_cast<const T*>(seq_stride ? src + s * seq_stride : (s & 1) ? a.dst : src);
        T* __restrict__ D = reinterpret_cast<T*>(seq_stride ? src + (s + 1) * seq_stride : (s & 1) ? src : a.dst);
        const int rev = a.reverse ^ (s & 1);
        diag = LaneDiag();
        for (int t = blockIdx.x * wpb + warp; t < a.n_tiles; t += stride)
            regs_tile<T, false>(a, S, D, a.plane, tile_at(a.tiles, a.n_tiles, t, rev), lane, diag, bad);
        if (s + 1 < n && !grid_barrier(count, unsigned(s + 1) * gridDim.x + a.barrier_extra, a.err)) break;
    }
    if (__any_sync(kFull, bad) && lane == 0) atomicOr(a.err, 1u);
    block_partials(a, diag);
}

// ---------------------------------------------------------------------------
// Variant 3: every warp streams its own tiles
// ---------------------------------------------------------------------------
// Proxy fence: the warp's generic reads of a stage are ordered before the
// asynchronous (bulk-copy) writes that refill it.
__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Refill `sg` with `tile`: lane 0 arms the barrier with the byte count, then
// lanes 0..16 each issue one bulk copy (the 14 plane rows, the wall-link
// bytes and the two port entries), so one warp instruction starts them all.
__device__ __forceinline__ void issue_tile(const StepArgs& a, uint2 tile, Stage& sg, uint64_t* bar, int lane)
{
    const int y = int(tile.x >> kColBits);
    const int x0 = tile_x0(tile);
    const int q0 = int(tile.y & 0xFFu), q1 = int((tile.y >> 8) & 0xFFu);
    // columns of the lanes that hold fluid, and one quad more on each side
    // for the planes that pull from x -+ 1
    const int us = x0 + 4 * q0, ue = x0 + 4 * q1 + 4;
    const int ss = us - 4 > 0 ? us - 4 : 0;
    const int se = ue + 4 < a.pitch ? ue + 4 : a.pitch;
    if (lane == 0) {
        sg.tile = tile;
        const uint32_t bytes = uint32_t(6 * (ue - us) + 8 * (se - ss)) * 4u + kTileNodes + 2 * sizeof(RowBC) +
                               (a.rates ? sizeof(float4) : 0);
        mbar_arrive_expect_tx(bar, bytes);
    }
    __syncwarp();
    const long long rC = (long long)y * a.pitch;
    if (lane < kPlanes) {
        const int p = lane;
        const long long r = src_row(p) == 0 ? rC
                            : src_row(p) == 1 ? (long long)(y > 0 ? y - 1 : y) * a.pitch
                                              : (long long)(y + 1 < a.ny ? y + 1 : y) * a.pitch;
        const int b = src_col(p) == 0 ? us : ss;
        const int e = src_col(p) == 0 ? ue : se;
        bulk_g2s(&sg.pl[p][b - x0 + 4], a.src + p * a.plane + r + b, uint32_t(e - b) * 4u, bar);
    } else if (lane == kPlanes) {
        bulk_g2s(sg.links, a.links + rC + x0, kTileNodes, bar);
    } else if (lane == kPlanes + 1) {
        bulk_g2s(&sg.bc[0], a.rowbc + y, sizeof(RowBC), bar);
    } else if (lane == kPlanes + 2) {
        bulk_g2s(&sg.bc[1], a.rowbc + a.ny + y, sizeof(RowBC), bar);
    } else if (lane == kPlanes + 3 && a.rates) {
        bulk_g2s(&sg.rates, a.rates + y, sizeof(float4), bar);
    }
}

// Warp w of the grid takes tiles w, w + W, w + 2W, ... (W warps in all).
// It owns `per` stages; its k-th tile goes to stage k % per as that stage's
// use k / per, and the warp refills a stage as soon as it has read it, so
// `per` tiles are always on their way while it computes.
__global__ void __launch_bounds__(kBulkMaxThreads, 2) coupled_step_pipe(const StepArgs a, int per)
{
    extern __shared__ __align__(128) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int wpb = blockDim.x >> 5;
    Stage* st = reinterpret_cast<Stage*>(smem) + warp * per;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + size_t(wpb) * per * sizeof(Stage)) + warp * per;
    const long long P = a.plane;
    const float* __restrict__ S = a.src;
    const int gw = int(blockIdx.x) * wpb + warp;
    const int W = int(gridDim.x) * wpb;
    const int n_items = gw < a.n_tiles ? (a.n_tiles - 1 - gw) / W + 1 : 0;

    if (lane == 0) {
        for (int s = 0; s < per; ++s) mbar_init(&full[s], 1);
        mbar_fence_init();
    }
    __syncwarp();
    grid_dependency_sync();

    LaneDiag diag;
    bool bad = false;
    int issued = 0;  // items whose copies were started
    for (; issued < n_items && issued < per; ++issued)
        issue_tile(a, tile_at(a.tiles, a.n_tiles, gw + issued * W, a.reverse), st[issued], &full[issued], lane);
    uint2 pending = issued < n_items ? tile_at(a.tiles, a.n_tiles, gw + issued * W, a.reverse) : make_uint2(0u, 0u);

    int k = 0;
    for (; k < n_items; ++k) {
        const int s = k % per;
        const uint32_t use = uint32_t(k / per);
        if (!__all_sync(kFull, mbar_wait(&full[s], use & 1u))) {
            if (lane == 0) atomicOr(a.err, 2u);
            break;
        }
        const Stage& sg = st[s];
        const uint2 tile = sg.tile;
        const int y = int(tile.x >> kColBits);
        const int x0 = tile_x0(tile) + 4 * lane;
        const long long oC = (long long)y * a.pitch + x0;
        const unsigned lk = sg.links[lane];
        const bool act = lk != 0xFFFFFFFFu;
        const RowBC bw = sg.bc[0], be = sg.bc[1];
        const float2 omega = a.rates ? make_float2(sg.rates.x, sg.rates.y) : make_float2(a.omega_f, a.omega_g);
        // ---- free flight (pull) from the staged rows ----
        float4 v[kPlanes];
        if (act) {
#pragma unroll
            for (int p = 0; p < kPlanes; ++p) {
                const float* row = sg.pl[p] + 4 * lane;
                const float4 c = *reinterpret_cast<const float4*>(row + 4);
                if (src_col(p) == 0) v[p] = c;
                else if (src_col(p) == 1) v[p] = make_float4(row[3], c.x, c.y, c.z);
                else v[p] = make_float4(c.y, c.z, c.w, row[8]);
            }
        }
        // ---- refill the stage with the tile `per` items ahead ----
        fence_proxy_async_smem();
        __syncwarp();
        if (issued < n_items) {
            issue_tile(a, pending, st[s], &full[s], lane);
            ++issued;
            if (issued < n_items) pending = tile_at(a.tiles, a.n_tiles, gw + issued * W, a.reverse);
        }
        if (act) {
            bounce_back<float, false>(v, lk, S, P, oC);
            QuadAcc q;
            collide_quad(v, lk, x0, bw, be, a, S, oC, omega, q);
#pragma unroll
            for (int p = 0; p < kPlanes; ++p) stg4(a.dst + p * P + oC, v[p]);
            bad |= q.bad;
            diag.add(q);
        }
    }
    // after a timeout: no copy may still be writing this block's shared memory at exit
    for (int j = k; j < issued; ++j)
        if (!__all_sync(kFull, mbar_wait(&full[j % per], uint32_t(j / per) & 1u)) && lane == 0)
            atomicOr(a.err, 2u);
    if (__any_sync(kFull, bad) && lane == 0) atomicOr(a.err, 1u);
    block_partials(a, diag);
}

// ---------------------------------------------------------------------------
// Set-up and read-out kernels
// ---------------------------------------------------------------------------
template <typename T>
__global__ void init_rest(T* pop, long long plane, float rho0, float wg0, float wg1, float C0, float gref0,
                          float gref1, float decay)
{
    const long long n = plane * kPlanes;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x) {
        const int p = int(e / plane);
        float w;  // f is stored as f_i - w_i
        if (p < 9) w = (p == 0 ? kWr : p <= 4 ? kWa : kWd) * (rho0 - 1.f);
        else w = (p == 9 ? wg0 : wg1) * C0 - (p == 9 ? wg0 : wg1) * decay * C0;
        Codec<T>::st1(pop + e, w, plane_offset(p, gref0, gref1));
    }
}

template <typename T>
__global__ void init_fields(T* pop, const uint8_t* links, int nx, int ny, int pitch,
                            const float* rho_in, const float* ux_in, const float* uy_in,
                            const float* C_in, float wg0, float wg1, float inv_cs2g, float gref0, float gref1,
                            float decay)
{
    const long long P = (long long)ny * pitch;
    for (int y = blockIdx.y; y < ny; y += gridDim.y) {
        const int x = blockIdx.x * blockDim.x + threadIdx.x;
        if (x >= nx) continue;
        const long long o = (long long)y * pitch + x;
        if (links[o] == kSolid) continue;
        const long long idx = (long long)y * nx + x;
        const float rho = rho_in[idx], ux = ux_in[idx], uy = uy_in[idx], C = C_in[idx];
        const float usq = 1.5f * (ux * ux + uy * uy);
        const float e[9] = {0.f, ux, uy, -ux, -uy, ux + uy, uy - ux, -ux - uy, ux - uy};
#pragma unroll
        for (int i = 0; i < 9; ++i) {  // f_eq_i - w_i
            const float w = i == 0 ? kWr : i <= 4 ? kWa : kWd;
            Codec<T>::st1(pop + i * P + o, w * ((rho - 1.f) + rho * (3.f * e[i] + 4.5f * e[i] * e[i] - usq)), 0.f);
        }
        const float R = -decay * C;  // the collision's reaction term, w_i R
        Codec<T>::st1(pop + 9 * P + o, wg0 * C + wg0 * R, gref0);
#pragma unroll
        for (int i = 1; i <= 4; ++i)
            Codec<T>::st1(pop + (9 + i) * P + o, wg1 * C * (1.f + e[i] * inv_cs2g) + wg1 * R, gref1);
    }
}

template <typename T>
__global__ void fields_kernel(const T* pop, const uint8_t* links, int nx, int ny, int pitch,
                              float* rho_out, float* ux_out, float* uy_out, float* C_out, float gref0, float gref1,
                              float decay)
{
    const long long P = (long long)ny * pitch;
    for (int y = blockIdx.y; y < ny; y += gridDim.y) {
        const int x = blockIdx.x * blockDim.x + threadIdx.x;
        if (x >= nx) continue;
        const long long o = (long long)y * pitch + x;
        float r = 0.f, vx = 0.f, vy = 0.f, c = 0.f;
        if (links[o] != kSolid) {
            float f[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) f[i] = Codec<T>::ld1(pop + i * P + o, 0.f);
            r = 1.f + (((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7])) + f[8]);
            const float jx = (f[1] - f[3]) + (f[5] - f[6]) + (f[8] - f[7]);
            const float jy = (f[2] - f[4]) + (f[5] + f[6]) - (f[7] + f[8]);
            vx = jx / r;
            vy = jy / r;
            float g[5];
#pragma unroll
            for (int i = 0; i < 5; ++i) g[i] = Codec<T>::ld1(pop + (9 + i) * P + o, i == 0 ? gref0 : gref1);
            c = ((g[0] + g[1]) + (g[2] + g[3])) + g[4];
            if (decay != 0.f) c /= 1.f - decay;
        }
        const long long idx = (long long)y * nx + x;
        if (rho_out) rho_out[idx] = r;
        if (ux_out) ux_out[idx] = vx;
        if (uy_out) uy_out[idx] = vy;
        if (C_out) C_out[idx] = c;
    }
}

// 16-bit storage <-> FP32 representation, element by element.
template <typename T>
__global__ void convert_kernel(const void* src, void* dst, long long plane, float gref0, float gref1,
                               bool to_fp32)
{
    const long long n = plane * kPlanes;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x) {
        const float off = plane_offset(int(e / plane), gref0, gref1);
        if (to_fp32) static_cast<float*>(dst)[e] = Codec<T>::ld1(static_cast<const T*>(src) + e, off);
        else Codec<T>::st1(static_cast<T*>(dst) + e, static_cast<const float*>(src)[e], off);
    }
}

int elementwise_grid(long long n)
{
    const long long want = (n + 255) / 256;
    return int(want < 65536 ? want : 65536);
}

// The paper's wall values of one step (see launch_wall_values).
template <typename T>
__global__ void wall_values(const T* S, T* W, const uint8_t* links, const long long* woff, int n, long long P,
                            int pitch)
{
    grid_dependency_sync();
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
        const long long o = woff[e];
        const unsigned lb = links[o];
        for (int i = 1; i < 9; ++i)
            if ((lb >> (i - 1)) & 1u)
                Codec<T>::st1(W + (i - 1) * P + o, equilibrium_wall(i, lb, S, links, P, o, pitch), 0.f);
    }
}

}  // namespace

cudaError_t launch_wall_values(const void* src, void* W, const uint8_t* links, const long long* woff, int n,
                               long long plane, int pitch, int precision, cudaStream_t s)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(unsigned(std::max(1, std::min((n + 255) / 256, 4096))));
    cfg.blockDim = dim3(256);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e;
    if (precision == kFP16)
        e = cudaLaunchKernelEx(&cfg, wall_values<__half>, static_cast<const __half*>(src), static_cast<__half*>(W),
                               links, woff, n, plane, pitch);
    else if (precision == kBF16)
        e = cudaLaunchKernelEx(&cfg, wall_values<__nv_bfloat16>, static_cast<const __nv_bfloat16*>(src),
                               static_cast<__nv_bfloat16*>(W), links, woff, n, plane, pitch);
    else
        e = cudaLaunchKernelEx(&cfg, wall_values<float>, static_cast<const float*>(src), static_cast<float*>(W), links,
                               woff, n, plane, pitch);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

size_t bulk_smem_bytes(int stages, int precision)
{
    const size_t stage = precision == kFP32 ? sizeof(Stage) : sizeof(StageT<__half>);
    return size_t(stages) * (stage + 2 * sizeof(uint64_t));
}

int bulk_stage_bytes(int precision)
{
    return int(precision == kFP32 ? sizeof(Stage) : sizeof(StageT<__half>));
}

cudaError_t prepare_step_kernels()
{
    // The attribute belongs to the kernel, not to a handle: allow the largest
    // ring any handle may ask for, so handles of different shapes coexist.
    cudaError_t e = cudaFuncSetAttribute(coupled_step_bulk<float, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         int(bulk_smem_bytes(kMaxStages)));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(coupled_step_bulk<__half, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 int(bulk_smem_bytes(kMaxStages, kFP16)));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(coupled_step_bulk<__nv_bfloat16, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 int(bulk_smem_bytes(kMaxStages, kBF16)));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(coupled_step_pipe, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 int(bulk_smem_bytes(kMaxStages)));
    const int async_max = int(async_smem_bytes(kBulkMaxThreads, kFP32));  // up to 8 warps per block
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(coupled_step_async<float, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 async_max);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(coupled_step_async<__half, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 async_max);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(coupled_step_async<__nv_bfloat16, false>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, async_max);
    if (e == cudaSuccess) e = prepare_walls_kernels();
    if (e == cudaSuccess) e = prepare_fold_kernels();
    return e;
}

// Blocks of a grid that take the port tiles in the register variants, for
// 16-bit storage: the port tiles' share of the grid with each port tile
// weighted as kPortTileCost plain ones, rounded up, and at least one block
// for the tiles without ports.  0 (every block runs every tile through the
// port loop) when there are no port tiles, for grids of one block, and for
// FP32 storage, whose step is bound by memory and measured slower split.
// The weight is measured on the 4096 x 2048 chip, FP16 storage (one port
// tile in 27): 1 -> 52.1 us, 2 -> 40.3 us, 3 -> 41.0 us, 5 -> 42.6 us per
// step; FP32 split: 69.8, 66.7, 67.0, 69.5 us against 62.3 us unsplit.  With
// the weight 1 the few port warps set the step's length.
constexpr int kPortTileCost = 2;

static int port_blocks(int grid, int n_tiles, int n_plain, int precision)
{
    const long long n_port = n_tiles - n_plain;
    if (precision == kFP32 || n_port <= 0 || n_plain <= 0 || grid < 2) return 0;
    const long long w = n_port * kPortTileCost;
    const long long gp = (grid * w + n_plain + w - 1) / (n_plain + w);
    return int(std::min<long long>(std::max<long long>(gp, 1), grid - 1));
}

cudaError_t launch_step(const StepArgs& a, const StepLaunch& l, cudaStream_t s)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(l.grid);
    cfg.blockDim = dim3(l.block);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = l.pdl ? 1 : 0;
    StepArgs b = a;  // the register variants' port blocks for this grid
    b.port_blocks = port_blocks(l.grid, a.n_tiles, a.n_plain, l.precision);
    if (a.wallv) return launch_step_walls(b, l, s);
    if (a.diag_out != nullptr) return launch_step_fold(b, l, cfg);
    cudaError_t e;
    if (l.variant == kVariantBulk) {
        const int per = l.stages / (l.block / 32 - 1);
        cfg.dynamicSmemBytes = bulk_smem_bytes(l.stages, l.precision);
        if (l.precision == kFP16) e = cudaLaunchKernelEx(&cfg, coupled_step_bulk<__half, false>, a, per);
        else if (l.precision == kBF16) e = cudaLaunchKernelEx(&cfg, coupled_step_bulk<__nv_bfloat16, false>, a, per);
        else e = cudaLaunchKernelEx(&cfg, coupled_step_bulk<float, false>, a, per);
    } else if (l.variant == kVariantPipe) {
        const int per = l.stages / (l.block / 32);
        cfg.dynamicSmemBytes = bulk_smem_bytes(l.stages);
        e = cudaLaunchKernelEx(&cfg, coupled_step_pipe, a, per);
    } else if (l.variant == kVariantAsync) {
        cfg.dynamicSmemBytes = async_smem_bytes(l.block, l.precision);
        if (l.precision == kFP16) e = cudaLaunchKernelEx(&cfg, coupled_step_async<__half, false>, b);
        else if (l.precision == kBF16) e = cudaLaunchKernelEx(&cfg, coupled_step_async<__nv_bfloat16, false>, b);
        else e = cudaLaunchKernelEx(&cfg, coupled_step_async<float, false>, b);
    } else if (l.variant == kVariantPairs) {
        e = cudaLaunchKernelEx(&cfg, coupled_step_pairs, a);  // FP32 storage only
    } else if (l.precision == kFP16) {
        e = cudaLaunchKernelEx(&cfg, coupled_step_regs<__half, false>, b);
    } else if (l.precision == kBF16) {
        e = cudaLaunchKernelEx(&cfg, coupled_step_regs<__nv_bfloat16, false>, b);
    } else {
        e = cudaLaunchKernelEx(&cfg, coupled_step_regs<float, false>, b);
    }
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t launch_steps_coop(const StepArgs& a, int n, long long seq_stride, unsigned* count, int grid, int block,
                              cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(count, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;  // all blocks resident, or the launch fails
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, coupled_steps_coop, a, n, seq_stride, count);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t steps_coop_occupancy(int block, int* blocks_per_sm)
{
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, coupled_steps_coop, block, 0);
}

size_t async_smem_bytes(int block, int precision)
{
    const size_t per_warp = precision == kFP32 ? sizeof(AsyncStage<float>) : sizeof(AsyncStage<__half>);
    return per_warp * size_t(block / 32);
}

cudaError_t launch_diag_finish(const float2* partials, int n_blocks, double* out, cudaStream_t s)
{
    // a programmatic dependent of the step before it, like the steps
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(1);
    cfg.blockDim = dim3(kFoldThreads);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, diag_finish, partials, n_blocks, out);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t step_kernel_occupancy(const StepLaunch& l, int* blocks_per_sm)
{
    if (l.walls) return step_walls_occupancy(l, blocks_per_sm);
    if (l.variant == kVariantBulk) {
        const size_t smem = bulk_smem_bytes(l.stages, l.precision);
        if (l.precision == kFP16)
            return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, coupled_step_bulk<__half, false>, l.block,
                                                                 smem);
        if (l.precision == kBF16)
            return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, coupled_step_bulk<__nv_bfloat16, false>,
                                                                 l.block, smem);
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, coupled_step_bulk<float, false>, l.block, smem);
    }
    if (l.variant == kVariantPipe)
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, coupled_step_pipe, l.block,
                                                             bulk_smem_bytes(l.stages));
    if (l.variant == kVariantAsync) {
        const size_t smem = async_smem_bytes(l.block, l.precision);
        if (l.precision == kFP16)
            return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, coupled_step_async<__half, false>,
                                                                 l.block, smem);
        if (l.precision == kBF16)
            return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm,
                                                                 coupled_step_async<__nv_bfloat16, false>, l.block, smem);
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, coupled_step_async<float, false>, l.block,
                                                             smem);
    }
    if (l.variant == kVariantPairs)
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, coupled_step_pairs, l.block, 0);
    if (l.precision == kFP16)
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, coupled_step_regs<__half, false>, l.block, 0);
    if (l.precision == kBF16)
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, coupled_step_regs<__nv_bfloat16, false>,
                                                             l.block, 0);
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, coupled_step_regs<float, false>, l.block, 0);
}

cudaError_t launch_init_rest(void* pop, int ny, int pitch, float rho0, float wg0, float wg1,
                             float C0, int precision, float decay, cudaStream_t s)
{
    const long long plane = (long long)ny * pitch;
    const int grid = elementwise_grid(plane * kPlanes);
    const float r0 = wg0 * kCRef, r1 = wg1 * kCRef;
    if (precision == kFP16)
        init_rest<<<grid, 256, 0, s>>>(static_cast<__half*>(pop), plane, rho0, wg0, wg1, C0, r0, r1, decay);
    else if (precision == kBF16)
        init_rest<<<grid, 256, 0, s>>>(static_cast<__nv_bfloat16*>(pop), plane, rho0, wg0, wg1, C0, r0, r1,
                                       decay);
    else
        init_rest<<<grid, 256, 0, s>>>(static_cast<float*>(pop), plane, rho0, wg0, wg1, C0, 0.f, 0.f, decay);
    return cudaGetLastError();
}

cudaError_t launch_init_fields(void* pop, const uint8_t* links, int nx, int ny, int pitch,
                               const float* rho, const float* ux, const float* uy, const float* C,
                               float wg0, float wg1, float inv_cs2g, int precision, float decay,
                               cudaStream_t s)
{
    dim3 grid((nx + 255) / 256, ny < 65535 ? ny : 65535);
    const float r0 = wg0 * kCRef, r1 = wg1 * kCRef;
    if (precision == kFP16)
        init_fields<<<grid, 256, 0, s>>>(static_cast<__half*>(pop), links, nx, ny, pitch, rho, ux, uy, C, wg0, wg1,
                                         inv_cs2g, r0, r1, decay);
    else if (precision == kBF16)
        init_fields<<<grid, 256, 0, s>>>(static_cast<__nv_bfloat16*>(pop), links, nx, ny, pitch, rho, ux, uy, C,
                                         wg0, wg1, inv_cs2g, r0, r1, decay);
    else
        init_fields<<<grid, 256, 0, s>>>(static_cast<float*>(pop), links, nx, ny, pitch, rho, ux, uy, C, wg0, wg1,
                                         inv_cs2g, 0.f, 0.f, decay);
    return cudaGetLastError();
}

cudaError_t launch_fields(const void* pop, const uint8_t* links, int nx, int ny, int pitch,
                          float* rho, float* ux, float* uy, float* C, float wg0, float wg1, int precision,
                          float decay, cudaStream_t s)
{
    dim3 grid((nx + 255) / 256, ny < 65535 ? ny : 65535);
    const float r0 = wg0 * kCRef, r1 = wg1 * kCRef;
    if (precision == kFP16)
        fields_kernel<<<grid, 256, 0, s>>>(static_cast<const __half*>(pop), links, nx, ny, pitch, rho, ux, uy, C,
                                           r0, r1, decay);
    else if (precision == kBF16)
        fields_kernel<<<grid, 256, 0, s>>>(static_cast<const __nv_bfloat16*>(pop), links, nx, ny, pitch, rho, ux,
                                           uy, C, r0, r1, decay);
    else
        fields_kernel<<<grid, 256, 0, s>>>(static_cast<const float*>(pop), links, nx, ny, pitch, rho, ux, uy, C,
                                           0.f, 0.f, decay);
    return cudaGetLastError();
}

cudaError_t launch_convert(const void* src, void* dst, long long plane, float wg0, float wg1, int precision,
                           bool to_fp32, cudaStream_t s)
{
    const int grid = elementwise_grid(plane * kPlanes);
    const float r0 = wg0 * kCRef, r1 = wg1 * kCRef;
    if (precision == kFP16)
        convert_kernel<__half><<<grid, 256, 0, s>>>(src, dst, plane, r0, r1, to_fp32);
    else if (precision == kBF16)
        convert_kernel<__nv_bfloat16><<<grid, 256, 0, s>>>(src, dst, plane, r0, r1, to_fp32);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

}  // namespace lbm
