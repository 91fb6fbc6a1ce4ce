// lbm_scalar.cu -- scalar-only step on a stored velocity field.
//
// The paper's own workflow (section "Results"): the flow reaches its steady
// state quickly, so the stationary velocity field of each valve state is
// computed once and the advection-diffusion solver reads it, with a larger
// time step for the scalar (the field is rescaled by the ratio of the time
// steps).  One launch advances the scalar lattice by one step: pull-stream of
// g with bounce-back, held concentration / do-nothing at open ports, and BGK
// relaxation towards the equilibrium of Eq. cdeequilibrium with the stored
// (scaled) velocity.  Per fluid node and step it reads 5 scalar populations
// and the 2 velocity components and writes 5 populations: 48 bytes, against
// 112 for the coupled step.
#include "lbm_device.cuh"

namespace lbm {
namespace {

// Bounce-back, ports, relaxation and stores of one lane's quad.  v: the
// streamed scalar populations; ux4, uy4: the stored field at the quad; sc,
// sq: the lane's scalar and outlet-flux sums.
__device__ __forceinline__ void scalar_quad(float4 (&v)[5], unsigned lk, int x0, const RowBC& bw, const RowBC& be,
                                            float4 ux4, float4 uy4, const ScalarArgs& a, const float* S, long long P,
                                            long long oC, KahanF& sc, KahanF& sq, bool& bad)
{
    // ---- no-flux walls: halfway bounce-back of g ----
    unsigned wall = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const unsigned lb = (lk >> (8 * k)) & 0xFFu;
        if (lb != kSolid) wall |= lb;
    }
#pragma unroll
    for (int i = 1; i <= 4; ++i) {
        if (wall & (1u << (i - 1))) {
            const float4 own = ldg4(S + opp(i) * P + oC);
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if ((lk >> (8 * k + i - 1)) & 1u) at(v[i], k) = at(own, k);
        }
    }
    const bool open_w = bw.x >= 0 && ((a.open_mask >> (bw.chan_kind & 31)) & 1u);
    const bool open_e = be.x >= 0 && ((a.open_mask >> (be.chan_kind & 31)) & 1u);
    float tc = 0.f, tq = 0.f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const bool fluid = ((lk >> (8 * k)) & 0xFFu) != kSolid;
        float g[5];
#pragma unroll
        for (int i = 0; i < 5; ++i) g[i] = fluid ? at(v[i], k) : 0.f;
        const int xk = x0 + k;
        const bool pw = open_w && bw.x == xk;
        const bool pe = !pw && open_e && be.x == xk;
        bool pressure_node = false;
        const float ux = a.u_scale * at(ux4, k), uy = a.u_scale * at(uy4, k);
        if (pw || pe) {
            const RowBC b = pw ? bw : be;
            const int gi = pw ? 1 : 3;
            const int kind = (b.chan_kind >> 8) & 0xFF;
            if (kind == 0) {  // held concentration
                float others = 0.f;
#pragma unroll
                for (int i = 0; i < 5; ++i)
                    if (i != gi) others += g[i];
                g[gi] = b.c - others;
            } else {          // do-nothing
                g[gi] = __ldg(S + gi * P + oC + k);
                pressure_node = kind != 3;
                if (kind == 3) {  // the paper's inlet: scaled to C_in
                    const float Cs = ((g[0] + g[1]) + (g[2] + g[3])) + g[4];
                    if (Cs > 0.f) {
                        const float gc = b.c / Cs;
#pragma unroll
                        for (int i = 0; i < 5; ++i) g[i] *= gc;
                    } else {
                        const float c1 = a.wg1 * b.c, cx = c1 * a.inv_cs2g * ux, cy = c1 * a.inv_cs2g * uy;
                        g[0] = b.c - 4.f * c1;
                        g[1] = c1 + cx;
                        g[3] = c1 - cx;
                        g[2] = c1 + cy;
                        g[4] = c1 - cy;
                    }
                }
            }
        }
        const float C = ((g[0] + g[1]) + (g[2] + g[3])) + g[4];
        const float wg = a.omega_g;
        const float c1 = a.wg1 * C, cx = c1 * a.inv_cs2g * ux, cy = c1 * a.inv_cs2g * uy;
        g[0] += wg * ((C - 4.f * c1) - g[0]);
        g[1] += wg * ((c1 + cx) - g[1]);
        g[3] += wg * ((c1 - cx) - g[3]);
        g[2] += wg * ((c1 + cy) - g[2]);
        g[4] += wg * ((c1 - cy) - g[4]);
        if (a.decay != 0.f) {  // reaction term R = -k C of Eq. cde, as w_i R
            const float R = -a.decay * C;
            g[0] += a.wg0 * R;
#pragma unroll
            for (int i = 1; i < 5; ++i) g[i] += a.wg1 * R;
        }
#pragma unroll
        for (int i = 0; i < 5; ++i) at(v[i], k) = g[i];
        if (fluid) {
            bad |= !(fabsf(C) < INFINITY);
            tc += C;
            if (pressure_node) tq += C * ux;
        }
    }
    sc.add(tc);
    if (tq != 0.f) sq.add(tq);
#pragma unroll
    for (int i = 0; i < 5; ++i) stg4(a.dst + i * P + oC, v[i]);
}

// The block's scalar and outlet-flux sums into slots 1 and 3 of its
// partials (and the bookkeeping of the slots of the coupled step's grid).
__device__ __forceinline__ void scalar_partials(const ScalarArgs& a, const KahanF& sc, const KahanF& sq)
{
    __shared__ DF red[32][2];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const DF s1 = warp_sum(sc.pair()), s3 = warp_sum(sq.pair());
    if (lane == 0) {
        red[warp][0] = s1;
        red[warp][1] = s3;
    }
    __syncthreads();
    if (threadIdx.x < 2) {
        DF sum = red[0][threadIdx.x];
        for (int w = 1; w < int(blockDim.x >> 5); ++w) sum = df_add(sum, red[w][threadIdx.x]);
        a.partials[blockIdx.x * 4 + 1 + 2 * threadIdx.x] = make_float2(sum.hi, sum.lo);
        for (int b = blockIdx.x + gridDim.x; b < a.n_partials; b += gridDim.x)
            a.partials[b * 4 + 1 + 2 * threadIdx.x] = make_float2(0.f, 0.f);
        // blocks beyond the last coupled step's grid hold no fluid partial
        if (int(blockIdx.x) >= a.fluid_blocks) a.partials[blockIdx.x * 4 + 2 * threadIdx.x] = make_float2(0.f, 0.f);
    }
}

// The kernel: a producer warp streams each tile's 5 scalar plane rows
// (with the halos of the shifted directions), its 2 stored velocity rows,
// its wall-link bytes and port entries into a ring of shared-memory stages
// with cp.async.bulk copies completing on mbarriers; consumer warps compute
// from shared memory.  The same stage ring as the coupled step's
// coupled_step_bulk (each consumer owns its stages; bounded waits set bit 1
// of the error word).
struct __align__(16) ScalarStage {
    float pl[5][kRowFloats];
    float u[2][kTileNodes];
    unsigned links[kTileNodes / 4];
    RowBC bc[2];
    uint2 tile;
    uint2 pad;
};
static_assert(sizeof(ScalarStage) % 16 == 0 && offsetof(ScalarStage, u) % 16 == 0 &&
                  offsetof(ScalarStage, links) % 16 == 0 && offsetof(ScalarStage, bc) % 16 == 0,
              "bulk-copy targets");

__global__ void __launch_bounds__(kBulkMaxThreads, 2) scalar_frozen_bulk(const ScalarArgs a, int per)
{
    extern __shared__ __align__(128) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nc = (blockDim.x >> 5) - 1;  // consumer warps; the last warp produces
    const int n_stages = nc * per;
    ScalarStage* st = reinterpret_cast<ScalarStage*>(smem);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + size_t(n_stages) * sizeof(ScalarStage));
    uint64_t* empty = full + n_stages;
    const long long P = a.plane;
    const float* __restrict__ S = a.src;
    const int G = int(gridDim.x);
    const int n_items = int(blockIdx.x) < a.n_tiles ? (a.n_tiles - 1 - int(blockIdx.x)) / G + 1 : 0;

    if (threadIdx.x == 0) {
        for (int s = 0; s < n_stages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_fence_init();
    }
    __syncthreads();
    grid_dependency_sync();

    KahanF sc, sq;
    bool bad = false;
    if (warp == nc) {
        // producer: lane l owns stage (l % nc) * per + l / nc (see coupled_step_bulk)
        const bool mine = lane < n_stages;
        const int s = (lane % nc) * per + lane / nc;
        int last_use = -1;
        for (int batch = 0, base = 0; base < n_items; ++batch, base += n_stages) {
            const int j = base + lane;
            bool good = true;
            if (mine && j < n_items) {
                const uint2 tile = tile_at(a.tiles, a.n_tiles, int(blockIdx.x) + j * G, a.reverse);
                if (batch > 0 && !mbar_wait(&empty[s], uint32_t(batch - 1) & 1u)) {
                    good = false;
                } else {
                    const int y = int(tile.x >> kColBits);
                    const int x0 = tile_x0(tile);
                    const int q0 = int(tile.y & 0xFFu), q1 = int((tile.y >> 8) & 0xFFu);
                    const int us = x0 + 4 * q0, ue = x0 + 4 * q1 + 4;
                    const int ss = us - 4 > 0 ? us - 4 : 0;
                    const int se = ue + 4 < a.pitch ? ue + 4 : a.pitch;
                    const long long rC = (long long)y * a.pitch;
                    const long long rS = (long long)(y > 0 ? y - 1 : y) * a.pitch;
                    const long long rN = (long long)(y + 1 < a.ny ? y + 1 : y) * a.pitch;
                    // directions 0, 2, 4 copy the lanes' span, 1 and 3 one quad more on
                    // each side; the two velocity rows the lanes' span
                    const uint32_t bytes = uint32_t(5 * (ue - us) + 2 * (se - ss)) * 4u + kTileNodes + 2 * sizeof(RowBC);
                    st[s].tile = tile;
                    mbar_arrive_expect_tx(&full[s], bytes);
#pragma unroll
                    for (int i = 0; i < 5; ++i) {
                        const int p = 9 + i;
                        const long long r = src_row(p) == 0 ? rC : src_row(p) == 1 ? rS : rN;
                        const int b = src_col(p) == 0 ? us : ss;
                        const int e = src_col(p) == 0 ? ue : se;
                        bulk_g2s(&st[s].pl[i][b - x0 + 4], S + i * P + r + b, uint32_t(e - b) * 4u, &full[s]);
                    }
                    bulk_g2s(&st[s].u[0][us - x0], a.ux + rC + us, uint32_t(ue - us) * 4u, &full[s]);
                    bulk_g2s(&st[s].u[1][us - x0], a.uy + rC + us, uint32_t(ue - us) * 4u, &full[s]);
                    bulk_g2s(st[s].links, a.links + rC + x0, kTileNodes, &full[s]);
                    bulk_g2s(&st[s].bc[0], a.rowbc + y, sizeof(RowBC), &full[s]);
                    bulk_g2s(&st[s].bc[1], a.rowbc + a.ny + y, sizeof(RowBC), &full[s]);
                    last_use = batch;
                }
            }
            if (!__all_sync(kFull, good)) {
                if (lane == 0) atomicOr(a.err, 2u);
                break;
            }
        }
        if (mine && last_use >= 0 && !mbar_wait(&full[s], uint32_t(last_use) & 1u)) atomicOr(a.err, 2u);
        __syncwarp();
    } else {
        for (int k = 0, j = warp; j < n_items; ++k, j += nc) {
            const int s = warp * per + k % per;
            const uint32_t use = uint32_t(k / per);
            if (!__all_sync(kFull, mbar_wait(&full[s], use & 1u))) {
                if (lane == 0) atomicOr(a.err, 2u);
                break;
            }
            const ScalarStage& sg = st[s];
            const uint2 tile = sg.tile;
            const int y = int(tile.x >> kColBits);
            const int x0 = tile_x0(tile) + 4 * lane;
            const long long oC = (long long)y * a.pitch + x0;
            const unsigned lk = sg.links[lane];
            const bool act = lk != 0xFFFFFFFFu;
            const RowBC bw = sg.bc[0], be = sg.bc[1];
            float4 v[5], ux4 = make_float4(0.f, 0.f, 0.f, 0.f), uy4 = ux4;
            if (act) {
#pragma unroll
                for (int i = 0; i < 5; ++i) {
                    const float* row = sg.pl[i] + 4 * lane;
                    const float4 c = *reinterpret_cast<const float4*>(row + 4);
                    if (src_col(9 + i) == 0) v[i] = c;
                    else if (src_col(9 + i) == 1) v[i] = make_float4(row[3], c.x, c.y, c.z);
                    else v[i] = make_float4(c.y, c.z, c.w, row[8]);
                }
                ux4 = *reinterpret_cast<const float4*>(&sg.u[0][4 * lane]);
                uy4 = *reinterpret_cast<const float4*>(&sg.u[1][4 * lane]);
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[s]);  // the stage may be refilled
            if (act) scalar_quad(v, lk, x0, bw, be, ux4, uy4, a, S, P, oC, sc, sq, bad);
        }
        if (__any_sync(kFull, bad) && lane == 0) atomicOr(a.err, 1u);
    }
    scalar_partials(a, sc, sq);
}

// The register variant: each warp pulls its tile's five scalar planes with
// 128-bit loads and warp shuffles (as coupled_step_regs does for all
// fourteen) and the stored field of its nodes; 20 live floats per lane
// instead of 56 leave room for many warps per SM, which keep the loads in
// flight without a shared-memory pipeline.
__global__ void __launch_bounds__(128) scalar_frozen_regs(const ScalarArgs a)
{
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int wpb = blockDim.x >> 5;
    const long long P = a.plane;
    const float* __restrict__ S = a.src;
    KahanF sc, sq;
    bool bad = false;
    grid_dependency_sync();
    for (int t = blockIdx.x * wpb + warp; t < a.n_tiles; t += gridDim.x * wpb) {
        const uint2 tile = tile_at(a.tiles, a.n_tiles, t, a.reverse);
        const int y = int(tile.x >> kColBits);
        const int x0 = tile_x0(tile) + 4 * lane;
        const long long oC = (long long)y * a.pitch + x0;
        const long long oS = (long long)(y > 0 ? y - 1 : y) * a.pitch + x0;
        const long long oN = (long long)(y + 1 < a.ny ? y + 1 : y) * a.pitch + x0;
        const int halo_w = x0 > 0 ? -1 : 0;
        const int halo_e = x0 + 4 < a.pitch ? 4 : 3;
        const unsigned lk = __ldg(reinterpret_cast<const unsigned*>(a.links + oC));
        // loads from the tile's fluid range, beside the wall-link word (see
        // load_range)
        const LoadRange r = load_range(tile, lane);
        float4 v[5];
        pull_quad<false, float, 9, 5>(v, S, P, oC, oS, oN, halo_w, halo_e, r.own, r.west, r.east, lane);
        const float4 ux4 = r.own ? ldg4(a.ux + oC) : make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 uy4 = r.own ? ldg4(a.uy + oC) : make_float4(0.f, 0.f, 0.f, 0.f);
        const bool act = lk != 0xFFFFFFFFu;
        if (!act) continue;
        const RowBC bw = a.rowbc[y];
        const RowBC be = a.rowbc[a.ny + y];
        scalar_quad(v, lk, x0, bw, be, ux4, uy4, a, S, P, oC, sc, sq, bad);
    }
    if (__any_sync(kFull, bad) && lane == 0) atomicOr(a.err, 1u);
    scalar_partials(a, sc, sq);
}

// Velocity of the stored populations (f as deviations) into two planes.
__global__ void velocity_of_state(const float* pop, const uint8_t* links, long long plane, int n, float* ux,
                                  float* uy)
{
    for (long long o = blockIdx.x * (long long)blockDim.x + threadIdx.x; o < plane;
         o += (long long)gridDim.x * blockDim.x) {
        float vx = 0.f, vy = 0.f;
        if (links[o] != kSolid) {
            float f[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) f[i] = pop[i * plane + o];
            const float rho = 1.f + (((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7])) + f[8]);
            vx = ((f[1] - f[3]) + (f[5] - f[6]) + (f[8] - f[7])) / rho;
            vy = ((f[2] - f[4]) + (f[5] + f[6]) - (f[7] + f[8])) / rho;
        }
        ux[o] = vx;
        uy[o] = vy;
    }
    (void)n;
}

}  // namespace

size_t scalar_bulk_smem_bytes(int stages)
{
    return size_t(stages) * (sizeof(ScalarStage) + 2 * sizeof(uint64_t));
}

cudaError_t launch_scalar_step_bulk(const ScalarArgs& a, int grid, int consumers, int per, cudaStream_t s)
{
    static_assert(kBulkMaxThreads >= 32 * 8, "block of up to 7 consumers and a producer");
    cudaError_t e = cudaFuncSetAttribute(scalar_frozen_bulk, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         int(scalar_bulk_smem_bytes(kMaxStages)));
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(32 * (consumers + 1));
    cfg.dynamicSmemBytes = scalar_bulk_smem_bytes(consumers * per);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, scalar_frozen_bulk, a, per);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t scalar_bulk_occupancy(int consumers, int per, int* blocks_per_sm)
{
    cudaError_t e = cudaFuncSetAttribute(scalar_frozen_bulk, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         int(scalar_bulk_smem_bytes(kMaxStages)));
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, scalar_frozen_bulk, 32 * (consumers + 1),
                                                         scalar_bulk_smem_bytes(consumers * per));
}

cudaError_t launch_scalar_step_regs(const ScalarArgs& a, int grid, int block, cudaStream_t s)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, scalar_frozen_regs, a);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t scalar_regs_occupancy(int block, int* blocks_per_sm)
{
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, scalar_frozen_regs, block, 0);
}

cudaError_t launch_velocity_of_state(const float* pop, const uint8_t* links, long long plane, float* ux, float* uy,
                                     cudaStream_t s)
{
    const int block = 256;
    const long long want = (plane + block - 1) / block;
    velocity_of_state<<<int(want < 65536 ? want : 65536), block, 0, s>>>(pop, links, plane, 0, ux, uy);
    return cudaGetLastError();
}

}  // namespace lbm
