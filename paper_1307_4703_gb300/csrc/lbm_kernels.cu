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
//                      by warp shuffle.
// Both share the per-node arithmetic below and give identical results.
#include <cmath>
#include <cstddef>

#include "lbm_internal.h"

namespace lbm {
namespace {

constexpr unsigned kFull = 0xffffffffu;

// D2Q9 weights of the equilibrium (Eq. lbequation / the w_i equation).
constexpr float kWr = 4.0f / 9.0f;   // rest
constexpr float kWa = 1.0f / 9.0f;   // axis
constexpr float kWd = 1.0f / 36.0f;  // diagonal

// A bounded wait gives up after this many SM cycles (about one second).
constexpr long long kWaitCycles = 1ll << 31;

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

// ---------------------------------------------------------------------------
// sm_90+ asynchronous bulk copies and mbarriers (inline PTX)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0;
}
// Wait for the phase of the given parity to complete; false after about one
// second (the caller then records LBM_ERR_TIMEOUT and stops).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity)
{
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > kWaitCycles) return false;
    return true;
}
// Global -> shared bulk copy completing on an mbarrier (16-byte aligned
// addresses, size a multiple of 16).
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// ---------------------------------------------------------------------------
// Per-node arithmetic shared by both variants
// ---------------------------------------------------------------------------
struct QuadAcc {
    float m = 0.f;      // sum of rho - 1 over the quad's fluid nodes
    float c = 0.f;      // sum of C over the quad's fluid nodes
    int n = 0;          // fluid nodes of the quad
    float q = 0.f;      // sum of rho u_x at open pressure-port nodes
    float qc = 0.f;     // sum of C u_x at open pressure-port nodes
    bool bad = false;   // a non-finite or non-positive density / non-finite C
};

// Compensated (Kahan) FP32 running sum of one lane.  GB300 has a narrow FP64
// pipe, so a lane sums its tiles in FP32 with compensation and FP64 is used
// only when the block combines its lanes.
struct KahanF {
    float s = 0.f, e = 0.f;
    __device__ __forceinline__ void add(float x)
    {
        const float y = x - e;
        const float t = s + y;
        e = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ double value() const { return double(s) - double(e); }
};

// The lane totals of the four diagnostics.
struct LaneDiag {
    KahanF m, c, q, qc;
    int n = 0;
    __device__ __forceinline__ void add(const QuadAcc& a)
    {
        m.add(a.m);
        c.add(a.c);
        if (a.q != 0.f || a.qc != 0.f) {
            q.add(a.q);
            qc.add(a.qc);
        }
        n += a.n;
    }
};

// Halfway bounce-back: a link from a wall returns the node's own
// post-collision population of the opposite direction (row y of the source
// buffer).  Only lanes next to a wall load anything here.
__device__ __forceinline__ void bounce_back(float4 (&v)[kPlanes], unsigned lk, const float* S, long long P,
                                            long long oC)
{
    unsigned wall = 0;  // union of the wall links of the fluid nodes
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const unsigned lb = (lk >> (8 * k)) & 0xFFu;
        if (lb != kSolid) wall |= lb;
    }
    if (!wall) return;
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

// Open ports, moments and both collisions for the four nodes x0..x0+3 of a
// row whose port entries are bw (west) and be (east); v holds the streamed
// populations on entry and the post-collision populations on exit (fluid
// planes as deviations f_i - w_i).
__device__ __forceinline__ void collide_quad(float4 (&v)[kPlanes], unsigned lk, int x0, const RowBC& bw,
                                             const RowBC& be, const StepArgs& a, const float* S, long long oC,
                                             QuadAcc& acc)
{
    const long long P = a.plane;
    const bool open_w = bw.x >= 0 && ((a.open_mask >> (bw.chan_kind & 31)) & 1u);
    const bool open_e = be.x >= 0 && ((a.open_mask >> (be.chan_kind & 31)) & 1u);

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
            if (velocity) jx = (1.f + Kd) * b.a / (1.f - s * b.a);
            else jx = s * (b.a - Kd);  // b.a = prescribed rho - 1
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
                else g[3] = b.c - (g[0] + g[1] + g[2] + g[4]);
            } else {
                // do-nothing: the node keeps its own post-collision value
                if (pw) g[1] = __ldg(S + 10 * P + oC + k);
                else g[3] = __ldg(S + 12 * P + oC + k);
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
            acc.bad |= !(rho > 0.f && rho < INFINITY) || !(fabsf(C) < INFINITY);
            acc.m += rd;
            acc.c += C;
            ++acc.n;
            if (pressure_node) {
                acc.q += jx;  // rho u_x
                acc.qc += C * ux;
            }
        }
    }
}

// The block's partial sums of the four diagnostics (FP64 from here on).
// The cross-block total is formed on demand by diag_finish.
__device__ __forceinline__ void block_partials(const StepArgs& a, const LaneDiag& d)
{
    __shared__ double red[32][4];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    double s0 = warp_sum(double(d.n) + d.m.value());
    double s1 = warp_sum(d.c.value());
    double s2 = warp_sum(d.q.value());
    double s3 = warp_sum(d.qc.value());
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
        a.partials[blockIdx.x * 4 + threadIdx.x] = s;
    }
}

// Total of the block partials of the last step, in a fixed order (the same
// bits on every run for a given launch shape).
__global__ void diag_finish(const double* partials, int n_blocks, double* out)
{
    __shared__ double red[8][4];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double t[4] = {0.0, 0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < n_blocks; b += blockDim.x)
#pragma unroll
        for (int q = 0; q < 4; ++q) t[q] += partials[4 * b + q];
#pragma unroll
    for (int q = 0; q < 4; ++q) t[q] = warp_sum(t[q]);
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < 4; ++q) red[warp][q] = t[q];
    __syncthreads();
    if (threadIdx.x < 4) {
        double s = 0.0;
        for (int w = 0; w < int(blockDim.x >> 5); ++w) s += red[w][threadIdx.x];
        out[threadIdx.x] = s;
    }
}

// ---------------------------------------------------------------------------
// Variant 1: registers and warp shuffles
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) coupled_step_regs(const StepArgs a)
{
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int wpb = blockDim.x >> 5;
    const long long P = a.plane;
    const float* __restrict__ S = a.src;

    LaneDiag diag;
    bool bad = false;

    const int stride = gridDim.x * wpb;
    int t = blockIdx.x * wpb + warp;
    uint2 next = t < a.n_tiles ? a.tiles[t] : make_uint2(0u, 0u);
    for (; t < a.n_tiles; t += stride) {
        const uint2 tile = next;  // the following entry is fetched one tile ahead
        if (t + stride < a.n_tiles) next = a.tiles[t + stride];
        const int y = int(tile.x >> kSegBits);
        const int x0 = int(tile.x & ((1u << kSegBits) - 1)) * kTileNodes + 4 * lane;
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
        if (act) {
            bounce_back(v, lk, S, P, oC);
            const RowBC bw = a.rowbc[y];
            const RowBC be = a.rowbc[a.ny + y];
            QuadAcc q;
            collide_quad(v, lk, x0, bw, be, a, S, oC, q);
#pragma unroll
            for (int p = 0; p < kPlanes; ++p) stg4(a.dst + p * P + oC, v[p]);
            bad |= q.bad;
            diag.add(q);
        }
    }

    if (__any_sync(kFull, bad) && lane == 0) atomicOr(a.err, 1u);
    block_partials(a, diag);
}

// ---------------------------------------------------------------------------
// Variant 2: bulk-copy pipeline through shared memory
// ---------------------------------------------------------------------------
// One staged tile: the 14 plane rows the tile pulls from, each with a
// 4-float halo on both sides (so that every copy starts on a 16-byte
// boundary), the tile's 128 wall-link bytes, the port entries of its row and
// the tile's table entry.
struct __align__(16) Stage {
    float pl[kPlanes][kRowFloats];
    unsigned links[kTileNodes / 4];
    RowBC bc[2];
    uint2 tile;
    uint2 pad;
};
static_assert(sizeof(Stage) % 16 == 0, "stage size must keep 16-byte alignment");
static_assert(offsetof(Stage, links) % 16 == 0 && offsetof(Stage, bc) % 16 == 0, "bulk-copy targets");

// Stage ring: consumer warp c owns stages [c * per, (c + 1) * per) and takes
// the block's tiles c, c + nc, c + 2 nc, ...; its k-th tile goes to stage
// c * per + k % per as that stage's use k / per.  Every stage is therefore
// filled and drained in order by one producer and one consumer, so the
// parity waits on its two mbarriers never skip a phase.
__global__ void __launch_bounds__(kBulkMaxThreads, 2) coupled_step_bulk(const StepArgs a, int per)
{
    extern __shared__ __align__(128) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nc = (blockDim.x >> 5) - 1;  // consumer warps; the last warp produces
    const int n_stages = nc * per;
    Stage* st = reinterpret_cast<Stage*>(smem);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + size_t(n_stages) * sizeof(Stage));
    uint64_t* empty = full + n_stages;
    const long long P = a.plane;
    const float* __restrict__ S = a.src;
    const int G = int(gridDim.x);
    // this block's tiles: blockIdx.x, blockIdx.x + G, ...
    const int n_items = int(blockIdx.x) < a.n_tiles ? (a.n_tiles - 1 - int(blockIdx.x)) / G + 1 : 0;

    if (threadIdx.x == 0) {
        for (int s = 0; s < n_stages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_fence_init();
    }
    __syncthreads();

    LaneDiag diag;
    bool bad = false;

    if (warp == nc) {
        // ---------------- producer warp: lane l owns stage
        //   s_l = (l % nc) * per + l / nc and fills it with tile base + l of
        //   every batch of n_stages consecutive tiles (that tile is use `batch`
        //   of s_l), so up to n_stages tiles are issued in parallel ----------------
        const bool mine = lane < n_stages;
        const int s = (lane % nc) * per + lane / nc;
        int last_use = -1;
        for (int batch = 0, base = 0; base < n_items; ++batch, base += n_stages) {
            const int j = base + lane;
            bool good = true;
            if (mine && j < n_items) {
                const uint2 tile = a.tiles[blockIdx.x + size_t(j) * G];
                if (batch > 0 && !mbar_wait(&empty[s], uint32_t(batch - 1) & 1u)) {
                    good = false;
                } else {
                    const int y = int(tile.x >> kSegBits);
                    const int x0 = int(tile.x & ((1u << kSegBits) - 1)) * kTileNodes;
                    const int q0 = int(tile.y & 0xFFu), q1 = int((tile.y >> 8) & 0xFFu);
                    // columns of the lanes that hold fluid, and one quad more on
                    // each side for the planes that pull from x -+ 1
                    const int us = x0 + 4 * q0, ue = x0 + 4 * q1 + 4;
                    const int ss = us - 4 > 0 ? us - 4 : 0;
                    const int se = ue + 4 < a.pitch ? ue + 4 : a.pitch;
                    const long long rC = (long long)y * a.pitch;
                    const long long rS = (long long)(y > 0 ? y - 1 : y) * a.pitch;
                    const long long rN = (long long)(y + 1 < a.ny ? y + 1 : y) * a.pitch;
                    const uint32_t bytes =
                        uint32_t(6 * (ue - us) + 8 * (se - ss)) * 4u + kTileNodes + 2 * sizeof(RowBC);
                    st[s].tile = tile;  // ordered before the consumer by the arrive below
                    mbar_arrive_expect_tx(&full[s], bytes);
#pragma unroll
                    for (int p = 0; p < kPlanes; ++p) {
                        const long long r = src_row(p) == 0 ? rC : src_row(p) == 1 ? rS : rN;
                        const int b = src_col(p) == 0 ? us : ss;
                        const int e = src_col(p) == 0 ? ue : se;
                        bulk_g2s(&st[s].pl[p][b - x0 + 4], S + p * P + r + b, uint32_t(e - b) * 4u, &full[s]);
                    }
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
        // no copy may still be writing this block's shared memory at exit
        if (mine && last_use >= 0 && !mbar_wait(&full[s], uint32_t(last_use) & 1u)) atomicOr(a.err, 2u);
        __syncwarp();
    } else {
        // ---------------- consumers ----------------
        for (int k = 0, j = warp; j < n_items; ++k, j += nc) {
            const int s = warp * per + k % per;
            const uint32_t use = uint32_t(k / per);
            if (!__all_sync(kFull, mbar_wait(&full[s], use & 1u))) {
                if (lane == 0) atomicOr(a.err, 2u);
                break;
            }
            const Stage& sg = st[s];
            const uint2 tile = sg.tile;
            const int y = int(tile.x >> kSegBits);
            const int x0 = int(tile.x & ((1u << kSegBits) - 1)) * kTileNodes + 4 * lane;
            const long long oC = (long long)y * a.pitch + x0;
            const unsigned lk = sg.links[lane];
            const bool act = lk != 0xFFFFFFFFu;
            const RowBC bw = sg.bc[0], be = sg.bc[1];
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
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[s]);  // the stage may be refilled
            if (act) {
                bounce_back(v, lk, S, P, oC);
                QuadAcc q;
                collide_quad(v, lk, x0, bw, be, a, S, oC, q);
#pragma unroll
                for (int p = 0; p < kPlanes; ++p) stg4(a.dst + p * P + oC, v[p]);
                bad |= q.bad;
                diag.add(q);
            }
        }
        if (__any_sync(kFull, bad) && lane == 0) atomicOr(a.err, 1u);
    }
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
    const int y = int(tile.x >> kSegBits);
    const int x0 = int(tile.x & ((1u << kSegBits) - 1)) * kTileNodes;
    const int q0 = int(tile.y & 0xFFu), q1 = int((tile.y >> 8) & 0xFFu);
    // columns of the lanes that hold fluid, and one quad more on each side
    // for the planes that pull from x -+ 1
    const int us = x0 + 4 * q0, ue = x0 + 4 * q1 + 4;
    const int ss = us - 4 > 0 ? us - 4 : 0;
    const int se = ue + 4 < a.pitch ? ue + 4 : a.pitch;
    if (lane == 0) {
        sg.tile = tile;
        const uint32_t bytes = uint32_t(6 * (ue - us) + 8 * (se - ss)) * 4u + kTileNodes + 2 * sizeof(RowBC);
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

    LaneDiag diag;
    bool bad = false;
    int issued = 0;  // items whose copies were started
    for (; issued < n_items && issued < per; ++issued)
        issue_tile(a, a.tiles[gw + size_t(issued) * W], st[issued], &full[issued], lane);
    uint2 pending = issued < n_items ? a.tiles[gw + size_t(issued) * W] : make_uint2(0u, 0u);

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
        const int y = int(tile.x >> kSegBits);
        const int x0 = int(tile.x & ((1u << kSegBits) - 1)) * kTileNodes + 4 * lane;
        const long long oC = (long long)y * a.pitch + x0;
        const unsigned lk = sg.links[lane];
        const bool act = lk != 0xFFFFFFFFu;
        const RowBC bw = sg.bc[0], be = sg.bc[1];
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
            if (issued < n_items) pending = a.tiles[gw + size_t(issued) * W];
        }
        if (act) {
            bounce_back(v, lk, S, P, oC);
            QuadAcc q;
            collide_quad(v, lk, x0, bw, be, a, S, oC, q);
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

size_t bulk_smem_bytes(int stages)
{
    return size_t(stages) * (sizeof(Stage) + 2 * sizeof(uint64_t));
}

int bulk_stage_bytes()
{
    return int(sizeof(Stage));
}

cudaError_t prepare_step_kernels()
{
    // The attribute belongs to the kernel, not to a handle: allow the largest
    // ring any handle may ask for, so handles of different shapes coexist.
    cudaError_t e = cudaFuncSetAttribute(coupled_step_bulk, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         int(bulk_smem_bytes(kMaxStages)));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(coupled_step_pipe, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 int(bulk_smem_bytes(kMaxStages)));
    return e;
}

cudaError_t launch_step(const StepArgs& a, const StepLaunch& l, cudaStream_t s)
{
    if (l.variant == kVariantBulk) {
        const int per = l.stages / (l.block / 32 - 1);
        coupled_step_bulk<<<l.grid, l.block, bulk_smem_bytes(l.stages), s>>>(a, per);
    } else if (l.variant == kVariantPipe) {
        const int per = l.stages / (l.block / 32);
        coupled_step_pipe<<<l.grid, l.block, bulk_smem_bytes(l.stages), s>>>(a, per);
    } else {
        coupled_step_regs<<<l.grid, l.block, 0, s>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t launch_diag_finish(const double* partials, int n_blocks, double* out, cudaStream_t s)
{
    diag_finish<<<1, 256, 0, s>>>(partials, n_blocks, out);
    return cudaGetLastError();
}

cudaError_t step_kernel_occupancy(const StepLaunch& l, int* blocks_per_sm)
{
    if (l.variant == kVariantBulk)
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, coupled_step_bulk, l.block,
                                                             bulk_smem_bytes(l.stages));
    if (l.variant == kVariantPipe)
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, coupled_step_pipe, l.block,
                                                             bulk_smem_bytes(l.stages));
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, coupled_step_regs, l.block, 0);
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
