// lbm_kernels.cu -- sm_103a kernels of the coupled D2Q9 + scalar lattice
// Boltzmann step (Tanaka & Iber, arXiv 1307.4703, "Numerical Methods" and
// "Boundary Conditions").
//
// The hot kernel is `coupled_step`: one launch advances the whole chip by one
// time step.  It is a pull scheme: node x gathers f_i from x - e_i (free
// flight of Eq. lbequation), replaces links that start on a wall by
// halfway bounce-back, completes open valve ports (Zou-He for f, held
// concentration or do-nothing for g), takes the moments of Eq. moments,
// relaxes f (Eq. lbequation) and then g towards the equilibrium of
// Eq. cdeequilibrium with the velocity just computed at the same node, and
// stores the post-collision populations.  Each element of the state is read
// once and written once per step, so the step is bound by HBM bandwidth;
// no tensor-core work exists in it.
//
// Work decomposition: a warp owns a 128-node row segment (a "tile"), four
// consecutive nodes per lane, so every population plane is read and written
// with one aligned 128-bit access per lane.  The +-1 column shifts of the
// pull move between lanes by warp shuffle; lane 0 / lane 31 fetch the one
// value that comes from the neighbouring segment.  Only segments that hold
// fluid are listed in the tile table, and lanes whose four nodes are all
// solid load only the shifted planes a fluid neighbour lane needs and store
// nothing.  The grid is persistent (one wave of
// resident blocks) and strides over the tile table.
#include <cmath>

#include "lbm_internal.h"

namespace lbm {
namespace {

constexpr unsigned kFull = 0xffffffffu;

// D2Q9 weights of the equilibrium (Eq. lbequation / the w_i equation).
constexpr float kWr = 4.0f / 9.0f;   // rest
constexpr float kWa = 1.0f / 9.0f;   // axis
constexpr float kWd = 1.0f / 36.0f;  // diagonal

// Eq. lattice: e_1 = E, e_2 = N, e_3 = W, e_4 = S, e_5 = NE, e_6 = NW,
// e_7 = SW, e_8 = SE.  The opposite of direction i.
__device__ __forceinline__ constexpr int opp(int i)
{
    return i == 0 ? 0 : i <= 4 ? ((i + 1) & 3) + 1 : ((i - 3) & 3) + 5;
}

// Pull source of plane p relative to the node: row 0 = same row, 1 = row
// y - 1 (directions with e_y = +1), 2 = row y + 1 (e_y = -1); column
// 0 = same, 1 = x - 1 (e_x = +1), 2 = x + 1 (e_x = -1).  Planes 9..13 are
// the scalar directions 0..4.
__device__ __forceinline__ constexpr int src_row(int p)
{
    const int i = p < 9 ? p : p - 9;
    return (i == 2 || i == 5 || i == 6) ? 1 : (i == 4 || i == 7 || i == 8) ? 2 : 0;
}
__device__ __forceinline__ constexpr int src_col(int p)
{
    const int i = p < 9 ? p : p - 9;
    return (i == 1 || i == 5 || i == 8) ? 1 : (i == 3 || i == 6 || i == 7) ? 2 : 0;
}

__device__ __forceinline__ float4 ldg4(const float* p)
{
    return __ldg(reinterpret_cast<const float4*>(p));
}
__device__ __forceinline__ void stg4(float* p, const float4& v)
{
    *reinterpret_cast<float4*>(p) = v;
}
__device__ __forceinline__ float& at(float4& v, int k)
{
    return k == 0 ? v.x : k == 1 ? v.y : k == 2 ? v.z : v.w;
}
__device__ __forceinline__ float at(const float4& v, int k)
{
    return k == 0 ? v.x : k == 1 ? v.y : k == 2 ? v.z : v.w;
}

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

template <bool kDiag>
__global__ void __launch_bounds__(256) coupled_step(const StepArgs a)
{
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int wpb = blockDim.x >> 5;
    const long long P = a.plane;
    const float* __restrict__ S = a.src;

    double acc0 = 0.0, acc1 = 0.0, acc2 = 0.0, acc3 = 0.0;
    bool bad = false;

    for (int t = blockIdx.x * wpb + warp; t < a.n_tiles; t += gridDim.x * wpb) {
        const uint32_t tile = __ldg(a.tiles + t);
        const int y = int(tile >> kSegBits);
        const int x0 = int(tile & ((1u << kSegBits) - 1)) * kTileNodes + 4 * lane;
        const long long oC = (long long)y * a.pitch + x0;
        // Rows outside the grid are clamped to a valid row: every link that
        // crosses y = -1/2 or y = ny - 1/2 is a wall link, so the value read
        // there is never used.
        const long long oS = (long long)(y > 0 ? y - 1 : y) * a.pitch + x0;
        const long long oN = (long long)(y + 1 < a.ny ? y + 1 : y) * a.pitch + x0;
        const int halo_w = x0 > 0 ? -1 : 0;
        const int halo_e = x0 + 4 < a.pitch ? 4 : 3;
        const unsigned lk = __ldg(reinterpret_cast<const unsigned*>(a.links + oC));
        const bool act = lk != 0xFFFFFFFFu;  // some node of this lane is fluid
        // A shifted plane's edge value also feeds the neighbouring lane (its
        // pull source may be fluid in row y -+ 1 even where this lane's own
        // nodes are all solid), so a lane loads it when it or that
        // neighbour is active.
        const unsigned ball = __ballot_sync(kFull, act);
        const bool ld_w = ((ball | (ball >> 1)) >> lane) & 1u;  // feeds lane + 1
        const bool ld_e = ((ball | (ball << 1)) >> lane) & 1u;  // feeds lane - 1

        // ---- free flight (pull): v[p] component k = plane p at (x0+k) - e ----
        float4 v[kPlanes];
#pragma unroll
        for (int p = 0; p < kPlanes; ++p) {
            const long long o = p * P + (src_row(p) == 0 ? oC : src_row(p) == 1 ? oS : oN);
            const bool ld = src_col(p) == 0 ? act : src_col(p) == 1 ? ld_w : ld_e;
            float4 r = ld ? ldg4(S + o) : make_float4(0.f, 0.f, 0.f, 0.f);
            if (src_col(p) == 1) {  // from column x - 1
                float h = 0.f;
                if (act && lane == 0) h = __ldg(S + o + halo_w);
                float w = __shfl_up_sync(kFull, r.w, 1);
                if (lane == 0) w = h;
                r = make_float4(w, r.x, r.y, r.z);
            } else if (src_col(p) == 2) {  // from column x + 1
                float h = 0.f;
                if (act && lane == 31) h = __ldg(S + o + halo_e);
                float e = __shfl_down_sync(kFull, r.x, 1);
                if (lane == 31) e = h;
                r = make_float4(r.y, r.z, r.w, e);
            }
            v[p] = r;
        }

        // ---- halfway bounce-back: a link from a wall returns the node's own
        //      post-collision population of the opposite direction ----
        unsigned wall = 0;  // union of the wall links of the fluid nodes
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const unsigned lb = (lk >> (8 * k)) & 0xFFu;
            if (lb != kSolid) wall |= lb;
        }
        if (wall) {
#pragma unroll
            for (int i = 1; i <= 8; ++i) {
                if (wall & (1u << (i - 1))) {
                    const float4 own = ldg4(S + opp(i) * P + oC);
                    const float4 ownc = i <= 4 ? ldg4(S + (9 + opp(i)) * P + oC) : own;
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        if ((lk >> (8 * k + i - 1)) & 1u) {
                            at(v[i], k) = at(own, k);
                            if (i <= 4) at(v[9 + i], k) = at(ownc, k);
                        }
                    }
                }
            }
        }

        const RowBC bw = a.rowbc[y];
        const RowBC be = a.rowbc[a.ny + y];
        const bool open_w = bw.x >= 0 && ((a.open_mask >> (bw.chan_kind & 31)) & 1u);
        const bool open_e = be.x >= 0 && ((a.open_mask >> (be.chan_kind & 31)) & 1u);

        float t_m = 0.f, t_c = 0.f;  // sum of rho - 1 and of C over the fluid nodes
        int t_n = 0;                 // fluid nodes
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const unsigned lb = (lk >> (8 * k)) & 0xFFu;
            const bool fluid = lb != kSolid;
            float f[9], g[5];
#pragma unroll
            for (int i = 0; i < 9; ++i) f[i] = at(v[i], k);
#pragma unroll
            for (int i = 0; i < 5; ++i) g[i] = at(v[9 + i], k);
            if (!fluid) {  // solid node: park it at the rest state rho = 1, C = 0
#pragma unroll
                for (int i = 0; i < 9; ++i) f[i] = 0.f;
#pragma unroll
                for (int i = 0; i < 5; ++i) g[i] = 0.f;
            }

            // ---- open valve ports (Zou-He; held concentration / do-nothing) ----
            const int xk = x0 + k;
            const bool pw = open_w && bw.x == xk;
            const bool pe = !pw && open_e && be.x == xk;
            bool pressure_node = false;
            if (pw || pe) {
                const RowBC b = pw ? bw : be;
                const float s = pw ? 1.f : -1.f;
                const bool velocity = ((b.chan_kind >> 8) & 0xFF) == 0;
                // populations leaving through the port: e = (-s, 0), (-s, -1), (-s, +1)
                const float fo_ax = pw ? f[3] : f[1];
                const float fo_dn = pw ? f[7] : f[8];
                const float fo_up = pw ? f[6] : f[5];
                // rho (1 - s u_x) = f0 + f2 + f4 + 2 (leaving) = 1 + Kd in deviations
                // (the weights of those populations add up to one)
                const float Kd = f[0] + f[2] + f[4] + 2.f * (fo_ax + fo_dn + fo_up);
                float jx;  // rho u_x of the node
                if (velocity) {
                    jx = (1.f + Kd) * b.a / (1.f - s * b.a);
                } else {
                    jx = s * (b.a - Kd);  // b.a = prescribed rho - 1
                }
                const float ht = 0.5f * (f[2] - f[4]);
                const float fi_ax = fo_ax + s * (2.f / 3.f) * jx;
                const float fi_up = fo_dn - ht + s * (1.f / 6.f) * jx;  // e = (s, +1)
                const float fi_dn = fo_up + ht + s * (1.f / 6.f) * jx;  // e = (s, -1)
                if (pw) {
                    f[1] = fi_ax;
                    f[5] = fi_up;
                    f[8] = fi_dn;
                } else {
                    f[3] = fi_ax;
                    f[6] = fi_up;
                    f[7] = fi_dn;
                }
                if (velocity) {
                    if (pw) g[1] = b.c - (g[0] + g[2] + g[3] + g[4]);
                    else    g[3] = b.c - (g[0] + g[1] + g[2] + g[4]);
                } else {
                    // do-nothing: the node keeps its own post-collision value
                    if (pw) g[1] = __ldg(S + 10 * P + oC + k);
                    else    g[3] = __ldg(S + 12 * P + oC + k);
                    pressure_node = true;
                }
            }

            // ---- moments (Eq. moments) and BGK collision of f, in deviations
            //      from the rest state: f'_i = f_i - w_i, rho = 1 + sum f'_i ----
            const float rd = ((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7])) + f[8];
            const float rho = 1.f + rd;
            const float jx = (f[1] - f[3]) + (f[5] - f[6]) + (f[8] - f[7]);
            const float jy = (f[2] - f[4]) + (f[5] + f[6]) - (f[7] + f[8]);
            const float inv = 1.f / rho;
            const float ux = jx * inv, uy = jy * inv;
            const float usq = 1.5f * (ux * ux + uy * uy);
            const float wo = a.omega_f;
            {
                // f_eq_i - w_i = w_i [rho - 1 + rho (3 e.u + 9/2 (e.u)^2 - 3/2 u^2)]
                const float e1 = ux, e2 = uy, e5 = ux + uy, e6 = uy - ux;
                const float q1 = rho * (4.5f * e1 * e1 - usq), q2 = rho * (4.5f * e2 * e2 - usq);
                const float q5 = rho * (4.5f * e5 * e5 - usq), q6 = rho * (4.5f * e6 * e6 - usq);
                const float t1 = 3.f * jx, t2 = 3.f * jy, t5 = t1 + t2, t6 = t2 - t1;
                f[0] += wo * (kWr * (rd - rho * usq) - f[0]);
                f[1] += wo * (kWa * (rd + t1 + q1) - f[1]);
                f[3] += wo * (kWa * (rd - t1 + q1) - f[3]);
                f[2] += wo * (kWa * (rd + t2 + q2) - f[2]);
                f[4] += wo * (kWa * (rd - t2 + q2) - f[4]);
                f[5] += wo * (kWd * (rd + t5 + q5) - f[5]);
                f[7] += wo * (kWd * (rd - t5 + q5) - f[7]);
                f[6] += wo * (kWd * (rd + t6 + q6) - f[6]);
                f[8] += wo * (kWd * (rd - t6 + q6) - f[8]);
            }
            // ---- scalar: C = sum g, relaxation towards g_eq(C, u of this node) ----
            const float C = ((g[0] + g[1]) + (g[2] + g[3])) + g[4];
            {
                const float wg = a.omega_g;
                const float c1 = a.wg1 * C, cx = c1 * a.inv_cs2g * ux, cy = c1 * a.inv_cs2g * uy;
                // rest equilibrium w0 C formed as the remainder, so that the five
                // equilibria add up to C exactly (float(w0) + 4 float(w1) != 1)
                g[0] += wg * ((C - 4.f * c1) - g[0]);
                g[1] += wg * ((c1 + cx) - g[1]);
                g[3] += wg * ((c1 - cx) - g[3]);
                g[2] += wg * ((c1 + cy) - g[2]);
                g[4] += wg * ((c1 - cy) - g[4]);
            }
#pragma unroll
            for (int i = 0; i < 9; ++i) at(v[i], k) = f[i];
#pragma unroll
            for (int i = 0; i < 5; ++i) at(v[9 + i], k) = g[i];

            if (fluid) {
                bad |= !(rho > 0.f && rho < INFINITY) || !(fabsf(C) < INFINITY);
                if (kDiag) {
                    t_m += rd;
                    t_c += C;
                    ++t_n;
                    if (pressure_node) {
                        acc2 += double(rho) * double(ux);
                        acc3 += double(C) * double(ux);
                    }
                }
            }
        }
        if (kDiag) {
            acc0 += double(t_n) + double(t_m);
            acc1 += double(t_c);
        }
        if (act) {
#pragma unroll
            for (int p = 0; p < kPlanes; ++p) stg4(a.dst + p * P + oC, v[p]);
        }
    }

    if (__any_sync(kFull, bad) && lane == 0) atomicOr(a.err, 1u);

    if (kDiag) {
        // block partials, then the last block to finish adds them in block order
        __shared__ double red[32][4];
        __shared__ bool last;
        acc0 = warp_sum(acc0);
        acc1 = warp_sum(acc1);
        acc2 = warp_sum(acc2);
        acc3 = warp_sum(acc3);
        if (lane == 0) {
            red[warp][0] = acc0;
            red[warp][1] = acc1;
            red[warp][2] = acc2;
            red[warp][3] = acc3;
        }
        __syncthreads();
        if (threadIdx.x < 4) {
            double s = 0.0;
            for (int w = 0; w < wpb; ++w) s += red[w][threadIdx.x];
            a.partials[blockIdx.x * 4 + threadIdx.x] = s;
            __threadfence();
        }
        __syncthreads();
        if (threadIdx.x == 0) last = atomicAdd(a.ticket, 1u) == gridDim.x - 1;
        __syncthreads();
        if (last) {
            __threadfence();
            double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
            for (int b = threadIdx.x; b < int(gridDim.x); b += blockDim.x) {
                s0 += __ldcg(a.partials + 4 * b + 0);
                s1 += __ldcg(a.partials + 4 * b + 1);
                s2 += __ldcg(a.partials + 4 * b + 2);
                s3 += __ldcg(a.partials + 4 * b + 3);
            }
            s0 = warp_sum(s0);
            s1 = warp_sum(s1);
            s2 = warp_sum(s2);
            s3 = warp_sum(s3);
            __syncthreads();
            if (lane == 0) {
                red[warp][0] = s0;
                red[warp][1] = s1;
                red[warp][2] = s2;
                red[warp][3] = s3;
            }
            __syncthreads();
            if (threadIdx.x < 4) {
                double s = 0.0;
                for (int w = 0; w < wpb; ++w) s += red[w][threadIdx.x];
                a.diag[threadIdx.x] = s;
            }
            if (threadIdx.x == 0) *a.ticket = 0u;
        }
    }
}

__global__ void init_rest(float* pop, long long plane, float rho0, float wg0, float wg1, float C0)
{
    const long long n = plane * kPlanes;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x) {
        const int p = int(e / plane);
        float w;  // f is stored as f_i - w_i
        if (p < 9) w = (p == 0 ? kWr : p <= 4 ? kWa : kWd) * (rho0 - 1.f);
        else w = (p == 9 ? wg0 : wg1) * C0;
        pop[e] = w;
    }
}

__global__ void init_fields(float* pop, const uint8_t* links, int nx, int ny, int pitch,
                            const float* rho_in, const float* ux_in, const float* uy_in,
                            const float* C_in, float wg0, float wg1, float inv_cs2g)
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
            pop[i * P + o] = w * ((rho - 1.f) + rho * (3.f * e[i] + 4.5f * e[i] * e[i] - usq));
        }
        pop[9 * P + o] = wg0 * C;
#pragma unroll
        for (int i = 1; i <= 4; ++i) pop[(9 + i) * P + o] = wg1 * C * (1.f + e[i] * inv_cs2g);
    }
}

__global__ void fields_kernel(const float* pop, const uint8_t* links, int nx, int ny, int pitch,
                              float* rho_out, float* ux_out, float* uy_out, float* C_out)
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
            for (int i = 0; i < 9; ++i) f[i] = pop[i * P + o];
            r = 1.f + (((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7])) + f[8]);
            const float jx = (f[1] - f[3]) + (f[5] - f[6]) + (f[8] - f[7]);
            const float jy = (f[2] - f[4]) + (f[5] + f[6]) - (f[7] + f[8]);
            vx = jx / r;
            vy = jy / r;
            c = ((pop[9 * P + o] + pop[10 * P + o]) + (pop[11 * P + o] + pop[12 * P + o])) +
                pop[13 * P + o];
        }
        const long long idx = (long long)y * nx + x;
        if (rho_out) rho_out[idx] = r;
        if (ux_out) ux_out[idx] = vx;
        if (uy_out) uy_out[idx] = vy;
        if (C_out) C_out[idx] = c;
    }
}

}  // namespace

cudaError_t launch_step(const StepArgs& a, int grid, int block, bool diag, cudaStream_t s)
{
    if (diag) coupled_step<true><<<grid, block, 0, s>>>(a);
    else coupled_step<false><<<grid, block, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t step_kernel_occupancy(int block, bool diag, int* blocks_per_sm)
{
    return diag ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, coupled_step<true>, block, 0)
                : cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, coupled_step<false>, block, 0);
}

cudaError_t launch_init_rest(float* pop, int ny, int pitch, float rho0, float wg0, float wg1,
                             float C0, cudaStream_t s)
{
    const long long plane = (long long)ny * pitch;
    const long long n = plane * kPlanes;
    const int block = 256;
    const long long want = (n + block - 1) / block;
    const int grid = int(want < 65536 ? want : 65536);
    init_rest<<<grid, block, 0, s>>>(pop, plane, rho0, wg0, wg1, C0);
    return cudaGetLastError();
}

cudaError_t launch_init_fields(float* pop, const uint8_t* links, int nx, int ny, int pitch,
                               const float* rho, const float* ux, const float* uy, const float* C,
                               float wg0, float wg1, float inv_cs2g, cudaStream_t s)
{
    dim3 grid((nx + 255) / 256, ny < 65535 ? ny : 65535);
    init_fields<<<grid, 256, 0, s>>>(pop, links, nx, ny, pitch, rho, ux, uy, C, wg0, wg1, inv_cs2g);
    return cudaGetLastError();
}

cudaError_t launch_fields(const float* pop, const uint8_t* links, int nx, int ny, int pitch,
                          float* rho, float* ux, float* uy, float* C, cudaStream_t s)
{
    dim3 grid((nx + 255) / 256, ny < 65535 ? ny : 65535);
    fields_kernel<<<grid, 256, 0, s>>>(pop, links, nx, ny, pitch, rho, ux, uy, C);
    return cudaGetLastError();
}

}  // namespace lbm
