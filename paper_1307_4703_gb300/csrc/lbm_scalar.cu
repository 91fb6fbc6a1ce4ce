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

__global__ void __launch_bounds__(256) scalar_frozen_step(const ScalarArgs a)
{
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int wpb = blockDim.x >> 5;
    const long long P = a.plane;
    const float* __restrict__ S = a.src;  // scalar plane 0 of the source buffer
    KahanF sc, sq;
    bool bad = false;
    grid_dependency_sync();
    for (int t = blockIdx.x * wpb + warp; t < a.n_tiles; t += gridDim.x * wpb) {
        const uint2 tile = a.tiles[t];
        const int y = int(tile.x >> kSegBits);
        const int x0 = int(tile.x & ((1u << kSegBits) - 1)) * kTileNodes + 4 * lane;
        const long long oC = (long long)y * a.pitch + x0;
        const long long oS = (long long)(y > 0 ? y - 1 : y) * a.pitch + x0;
        const long long oN = (long long)(y + 1 < a.ny ? y + 1 : y) * a.pitch + x0;
        const int halo_w = x0 > 0 ? -1 : 0;
        const int halo_e = x0 + 4 < a.pitch ? 4 : 3;
        const unsigned lk = __ldg(reinterpret_cast<const unsigned*>(a.links + oC));
        const bool act = lk != 0xFFFFFFFFu;
        const unsigned ball = __ballot_sync(kFull, act);
        const bool ld_w = ((ball | (ball >> 1)) >> lane) & 1u;
        const bool ld_e = ((ball | (ball << 1)) >> lane) & 1u;
        // ---- free flight of g (directions 0..4 use the shifts of planes 9..13) ----
        float4 v[5];
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            const int p = 9 + i;
            const long long o = i * P + (src_row(p) == 0 ? oC : src_row(p) == 1 ? oS : oN);
            const bool ld = src_col(p) == 0 ? act : src_col(p) == 1 ? ld_w : ld_e;
            float4 r = ld ? ldg4(S + o) : make_float4(0.f, 0.f, 0.f, 0.f);
            if (src_col(p) == 1) {
                float h = 0.f;
                if (act && lane == 0) h = __ldg(S + o + halo_w);
                float w = __shfl_up_sync(kFull, r.w, 1);
                if (lane == 0) w = h;
                r = make_float4(w, r.x, r.y, r.z);
            } else if (src_col(p) == 2) {
                float h = 0.f;
                if (act && lane == 31) h = __ldg(S + o + halo_e);
                float e = __shfl_down_sync(kFull, r.x, 1);
                if (lane == 31) e = h;
                r = make_float4(r.y, r.z, r.w, e);
            }
            v[i] = r;
        }
        if (!act) continue;
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
        const float4 ux4 = ldg4(a.ux + oC), uy4 = ldg4(a.uy + oC);
        const RowBC bw = a.rowbc[y];
        const RowBC be = a.rowbc[a.ny + y];
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
    if (__any_sync(kFull, bad) && lane == 0) atomicOr(a.err, 1u);
    // block partials of the scalar diagnostics (slots 1 and 3); the fluid's
    // slots 0 and 2 keep the values of the last coupled step
    __shared__ double red[32][2];
    double s1 = warp_sum(sc.value()), s3 = warp_sum(sq.value());
    if (lane == 0) {
        red[warp][0] = s1;
        red[warp][1] = s3;
    }
    __syncthreads();
    if (threadIdx.x < 2) {
        double s = 0.0;
        for (int w = 0; w < wpb; ++w) s += red[w][threadIdx.x];
        a.partials[blockIdx.x * 4 + 1 + 2 * threadIdx.x] = s;
        // entries of the coupled step's larger grid hold no scalar partial now
        for (int b = blockIdx.x + gridDim.x; b < a.n_partials; b += gridDim.x)
            a.partials[b * 4 + 1 + 2 * threadIdx.x] = 0.0;
    }
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

cudaError_t launch_scalar_step(const ScalarArgs& a, int grid, int block, cudaStream_t s)
{
    // a programmatic dependent of the previous kernel (see grid_dependency_sync)
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, scalar_frozen_step, a);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t scalar_step_occupancy(int block, int* blocks_per_sm)
{
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, scalar_frozen_step, block, 0);
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
