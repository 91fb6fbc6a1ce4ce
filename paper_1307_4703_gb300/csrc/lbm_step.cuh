// lbm_step.cuh -- the coupled step kernels (register variant and bulk-copy
// pipeline), templated on the storage type and on the fluid wall scheme
// (kWalls: the paper's wall values precomputed into a buffer, see
// launch_wall_values; otherwise halfway bounce-back).  Included by
// lbm_kernels.cu (bounce-back instantiations) and lbm_walls.cu (the paper's
// walls), so the two sets compile in parallel.
#pragma once

#include "lbm_device.cuh"

namespace lbm {
namespace {

// ---------------------------------------------------------------------------
// Tiles with and without ports (the register kernels, variants 1 and 4)
// ---------------------------------------------------------------------------
// The tile table lists the tiles whose row segment holds no port node first
// (a.n_plain of them) and the port tiles (kPortTile) after them.  The port
// code, present in a tile loop, costs that loop time even where it never
// runs (the 16-bit step on the 4096 x 2048 chip: 48.0 us with it in the
// loop, 44.0 us when only a separate loop has it), so the register kernels
// have two loops: the grid's last a.port_blocks blocks take the port tiles
// with the port code, the other blocks the rest without any (16-bit
// storage; see port_blocks for the share; split_tiles).  Both collide each
// node the same way (collide_quad's forms give the same bits).
__device__ __forceinline__ TileRange warp_tiles(const StepArgs& a, int warp, int wpb, bool& port_loop)
{
    return split_tiles(a.tiles, a.n_tiles, a.n_plain, a.port_blocks, warp, wpb, port_loop);
}

// ---------------------------------------------------------------------------
// Variant 1: registers and warp shuffles
// ---------------------------------------------------------------------------
// kWhole: every tile of the table with the grid's stride, read from the
// kernel parameters (the FP32 kernel sits at its register limit, where the
// range held in registers makes it spill).
template <typename T, bool kWalls, bool kPortCode, bool kWhole = false>
__device__ __forceinline__ void regs_loop(const StepArgs& a, TileRange r, int lane, LaneDiag& diag, bool& bad)
{
    if constexpr (kWhole) {
        r.tiles = a.tiles;
        r.n = a.n_tiles;
        r.stride = int(gridDim.x) * int(blockDim.x >> 5);
    }
    const long long P = a.plane;
    const T* __restrict__ S = reinterpret_cast<const T*>(a.src);
    T* __restrict__ D = reinterpret_cast<T*>(a.dst);
    int t = r.t;
    uint2 next = t < r.n ? tile_at(r.tiles, r.n, t, a.reverse) : make_uint2(0u, 0u);
    grid_dependency_sync();
    for (; t < r.n; t += r.stride) {
        const uint2 tile = next;  // the following entry is fetched one tile ahead
        if (t + r.stride < r.n) next = tile_at(r.tiles, r.n, t + r.stride, a.reverse);
        const int y = int(tile.x >> kColBits);
        const int x0 = tile_x0(tile) + 4 * lane;
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
        pull_quad<false>(v, S, P, oC, oS, oN, halo_w, halo_e, act, ld_w, ld_e, lane);
        if (act) {
            bounce_back<T, kWalls>(v, lk, S, P, oC, static_cast<const T*>(a.wallv));
            QuadAcc q;
            if constexpr (kPortCode) {
                const RowBC bw = a.rowbc[y];
                const RowBC be = a.rowbc[a.ny + y];
                collide_quad<T, !kStoresF32<T>, true>(v, lk, x0, bw, be, a, S, oC, row_rates(a, y), q);
            } else {
                collide_quad<T, !kStoresF32<T>, false>(v, lk, x0, RowBC{}, RowBC{}, a, S, oC, row_rates(a, y), q);
            }
#pragma unroll
            for (int p = 0; p < kPlanes; ++p)
                Codec<T>::st4(D + p * P + oC, v[p], 0.f);
            bad |= q.bad;
            diag.add(q);
        }
    }
}

template <typename T, bool kWalls, bool kFold = false>
__global__ void __launch_bounds__(256, 2) coupled_step_regs(const StepArgs a)
{
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int wpb = blockDim.x >> 5;
    LaneDiag diag;
    bool bad = false;
    if constexpr (kStoresF32<T>) {  // one loop over every tile (port_blocks is 0 for FP32)
        regs_loop<T, kWalls, true, true>(a, TileRange{nullptr, 0, int(blockIdx.x) * wpb + warp, 0}, lane, diag, bad);
    } else {
        bool port_loop;
        const TileRange r = warp_tiles(a, warp, wpb, port_loop);
        if (port_loop) regs_loop<T, kWalls, true>(a, r, lane, diag, bad);
        else regs_loop<T, kWalls, false>(a, r, lane, diag, bad);
    }
    if (__any_sync(kFull, bad) && lane == 0) atomicOr(a.err, 1u);
    block_partials<kFold>(a, diag);
}

// ---------------------------------------------------------------------------
// Variant 4: register variant with the next tile prefetched into shared
// memory by per-lane asynchronous copies (cp.async)
// ---------------------------------------------------------------------------
// Each warp owns one stage: the 14 plane rows of a tile, 128 values each
// with 4 on both sides for the shifted planes' edge values.  A warp copies
// its next tile's rows into the stage as soon as it has read the current one
// into registers, so those loads are in flight while it computes; the copies
// take no registers, so the 128-register budget and 16 warps per SM stay.
// Lane l copies its own 4 values of each row it needs (lanes q0 .. q1 of the
// tile's fluid range, one lane more on each side for the shifted planes);
// lanes 0 and 31 also copy the neighbouring segments' 4 edge values.
template <typename T>
struct AsyncStage {
    static constexpr int kRow = kTileNodes + 8;  // [4 halo | 128 | 4 halo]
    T pl[kPlanes][kRow];
    unsigned links[32];  // the lanes' wall-link words (lanes q0 .. q1)
};

template <typename T>
__device__ __forceinline__ void cp_async_quad(T* dst, const T* src)
{
    if constexpr (sizeof(T) == 4)
        cp_async16(dst, src);
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}

template <typename T>
__device__ __forceinline__ void issue_tile_async(const StepArgs& a, const T* S, long long P, uint2 tile,
                                                 AsyncStage<T>& st, int lane)
{
    const int y = int(tile.x >> kColBits);
    const int xs = tile_x0(tile);
    const int q0 = int(tile.y & 0xFFu), q1 = int((tile.y >> 8) & 0xFFu);
    const long long rC = (long long)y * a.pitch + xs;
    const long long rS = (long long)(y > 0 ? y - 1 : y) * a.pitch + xs;
    const long long rN = (long long)(y + 1 < a.ny ? y + 1 : y) * a.pitch + xs;
    const bool own = lane >= q0 && lane <= q1;
    const bool wide = lane >= q0 - 1 && lane <= q1 + 1;
    if (own)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(&st.links[lane])),
                     "l"(a.links + rC + 4 * lane)
                     : "memory");
#pragma unroll
    for (int p = 0; p < kPlanes; ++p) {
        const int sr = src_row(p), sc = src_col(p);
        const T* row = S + p * P + (sr == 0 ? rC : sr == 1 ? rS : rN);
        if (sc == 0 ? own : wide) cp_async_quad(&st.pl[p][4 + 4 * lane], row + 4 * lane);
        if (sc == 1 && lane == 0 && q0 == 0 && xs > 0) cp_async_quad(&st.pl[p][0], row - 4);
        if (sc == 2 && lane == 31 && q1 == 31 && xs + kTileNodes < a.pitch)
            cp_async_quad(&st.pl[p][4 + kTileNodes], row + kTileNodes);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}

template <typename T, bool kWalls, bool kPortCode>
__device__ __forceinline__ void async_loop(const StepArgs& a, TileRange r, AsyncStage<T>& st, int lane,
                                           LaneDiag& diag, bool& bad)
{
    const long long P = a.plane;
    const T* __restrict__ S = reinterpret_cast<const T*>(a.src);
    T* __restrict__ D = reinterpret_cast<T*>(a.dst);
    int t = r.t;
    grid_dependency_sync();
    uint2 tile = t < r.n ? tile_at(r.tiles, r.n, t, a.reverse) : make_uint2(0u, 0u);
    if (t < r.n) issue_tile_async(a, S, P, tile, st, lane);
    for (; t < r.n; t += r.stride) {
        const bool more = t + r.stride < r.n;
        const uint2 next = more ? tile_at(r.tiles, r.n, t + r.stride, a.reverse) : make_uint2(0u, 0u);
        const int y = int(tile.x >> kColBits);
        const int x0 = tile_x0(tile) + 4 * lane;
        const long long oC = (long long)y * a.pitch + x0;
        // ---- free flight (pull) from the stage: the current tile's copies,
        //      the wall-link words with them (lanes outside the tile's fluid
        //      range q0 .. q1 hold no fluid) ----
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        __syncwarp();
        const int q0 = int(tile.y & 0xFFu), q1 = int((tile.y >> 8) & 0xFFu);
        const unsigned lk = lane >= q0 && lane <= q1 ? st.links[lane] : 0xFFFFFFFFu;
        const bool act = lk != 0xFFFFFFFFu;
        float4 v[kPlanes];
        if (act) {
#pragma unroll
            for (int p = 0; p < kPlanes; ++p) {
                const T* row = &st.pl[p][4 + 4 * lane];
                const float4 c = Codec<T>::lds4(row, 0.f);
                if (src_col(p) == 0) v[p] = c;
                else if (src_col(p) == 1) v[p] = make_float4(Codec<T>::lds1(row - 1, 0.f), c.x, c.y, c.z);
                else v[p] = make_float4(c.y, c.z, c.w, Codec<T>::lds1(row + 4, 0.f));
            }
        }
        __syncwarp();
        if (more) issue_tile_async(a, S, P, next, st, lane);  // the stage is free again
        if (act) {
            bounce_back<T, kWalls>(v, lk, S, P, oC, static_cast<const T*>(a.wallv));
            QuadAcc q;
            if constexpr (kPortCode) {
                const RowBC bw = a.rowbc[y];
                const RowBC be = a.rowbc[a.ny + y];
                collide_quad<T, !kStoresF32<T>, true>(v, lk, x0, bw, be, a, S, oC, row_rates(a, y), q);
            } else {
                collide_quad<T, !kStoresF32<T>, false>(v, lk, x0, RowBC{}, RowBC{}, a, S, oC, row_rates(a, y), q);
            }
#pragma unroll
            for (int p = 0; p < kPlanes; ++p)
                Codec<T>::st4(D + p * P + oC, v[p], 0.f);
            bad |= q.bad;
            diag.add(q);
        }
        tile = next;
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");  // nothing in flight at exit
}

template <typename T, bool kWalls, bool kFold = false>
__global__ void __launch_bounds__(256, 2) coupled_step_async(const StepArgs a)
{
    // named apart from the bulk kernels' 128-byte aligned smem (one symbol per name)
    extern __shared__ __align__(16) unsigned char stage_smem[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int wpb = blockDim.x >> 5;
    AsyncStage<T>& st = reinterpret_cast<AsyncStage<T>*>(stage_smem)[warp];
    LaneDiag diag;
    bool bad = false;
    if constexpr (kStoresF32<T>) {  // one loop over every tile (port_blocks is 0 for FP32)
        async_loop<T, kWalls, true>(a, TileRange{a.tiles, a.n_tiles, int(blockIdx.x) * wpb + warp,
                                                 int(gridDim.x) * wpb},
                                    st, lane, diag, bad);
    } else {
        bool port_loop;
        const TileRange r = warp_tiles(a, warp, wpb, port_loop);
        if (port_loop) async_loop<T, kWalls, true>(a, r, st, lane, diag, bad);
        else async_loop<T, kWalls, false>(a, r, st, lane, diag, bad);
    }
    if (__any_sync(kFull, bad) && lane == 0) atomicOr(a.err, 1u);
    block_partials<kFold>(a, diag);
}

// ---------------------------------------------------------------------------
// Variant 5: registers and warp shuffles, two nodes per lane (FP32 storage,
// halfway bounce-back)
// ---------------------------------------------------------------------------
// The register variant on 64-node warp tiles: a lane holds two nodes, so a
// tile's populations take 28 registers instead of 56 and more warps fit on
// an SM, and a lattice has twice as many (half-size) tiles to spread over
// them.  Meant for small chips, whose steps give each warp about one
// 128-node tile: the warps that draw a second one set the step's length.
// The per-node arithmetic is collide_node, as in every other variant, so the
// results are the same bits.

// Free flight (pull) of one lane's two nodes x0, x0 + 1 (64-bit loads; the
// +-1 column shifts move between lanes by shuffle, lanes 0 and 31 load the
// value that comes from the neighbouring segment).  act / ld_w / ld_e as
// in pull_quad.
__device__ __forceinline__ void pull_pair(float2 (&v)[kPlanes], const float* __restrict__ S, long long P,
                                          long long oC, long long oS, long long oN, int halo_w, int halo_e,
                                          bool act, bool ld_w, bool ld_e, int lane)
{
#pragma unroll
    for (int p = 0; p < kPlanes; ++p) {
        const int sr = src_row(p), sc = src_col(p);
        const long long o = p * P + (sr == 0 ? oC : sr == 1 ? oS : oN);
        const bool ld = sc == 0 ? act : sc == 1 ? ld_w : ld_e;
        float2 r = ld ? ldg2(S + o) : make_float2(0.f, 0.f);
        if (sc == 1) {  // from column x - 1
            float h = 0.f;
            if (act && lane == 0) h = __ldg(S + o + halo_w);
            float w = __shfl_up_sync(kFull, r.y, 1);
            if (lane == 0) w = h;
            r = make_float2(w, r.x);
        } else if (sc == 2) {  // from column x + 1
            float h = 0.f;
            if (act && lane == 31) h = __ldg(S + o + halo_e);
            float e = __shfl_down_sync(kFull, r.x, 1);
            if (lane == 31) e = h;
            r = make_float2(r.y, e);
        }
        v[p] = r;
    }
}

// Halfway bounce-back of the two nodes (wall-link bytes in the low 16 bits
// of lk2), as bounce_back.
__device__ __forceinline__ void bounce_back_pair(float2 (&v)[kPlanes], unsigned lk2, const float* S, long long P,
                                                 long long oC)
{
    unsigned wall = 0;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const unsigned lb = (lk2 >> (8 * k)) & 0xFFu;
        if (lb != kSolid) wall |= lb;
    }
    if (!wall) return;
#pragma unroll
    for (int i = 1; i <= 8; ++i) {
        if (wall & (1u << (i - 1))) {
            const float2 own = ldg2(S + opp(i) * P + oC);
            const float2 ownc = i <= 4 ? ldg2(S + (9 + opp(i)) * P + oC) : own;
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                if ((lk2 >> (8 * k + i - 1)) & 1u) {
                    at(v[i], k) = at(own, k);
                    if (i <= 4) at(v[9 + i], k) = at(ownc, k);
                }
            }
        }
    }
}

// Open ports, moments and both collisions of the two nodes, the port and
// solid-node handling inside the node loop as for FP32 quads.
__device__ __forceinline__ void collide_pair(float2 (&v)[kPlanes], unsigned lk2, int x0, const RowBC& bw,
                                             const RowBC& be, const StepArgs& a, const float* S, long long oC,
                                             float2 omega, QuadAcc& acc)
{
    bool open_w = false, open_e = false;
    if (bw.x >= 0) open_w = valve_open(a, bw.chan_kind);
    if (be.x >= 0) open_e = valve_open(a, be.chan_kind);
    const float dfac = a.decay != 0.f ? 1.f - a.decay / omega.y : 1.f;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const unsigned lb = (lk2 >> (8 * k)) & 0xFFu;
        const bool fluid = lb != kSolid;
        float f[9], g[5];
#pragma unroll
        for (int i = 0; i < 9; ++i) f[i] = fluid ? at(v[i], k) : 0.f;  // solid: parked at rho = 1, C = 0
#pragma unroll
        for (int i = 0; i < 5; ++i) g[i] = fluid ? at(v[9 + i], k) : 0.f;
        bool outlet_k = false;
        const int xk = x0 + k;
        const bool pw = open_w && bw.x == xk;
        const bool pe = !pw && open_e && be.x == xk;
        if (pw || pe) outlet_k = port_node(f, g, pw, pw ? bw : be, a, S, oC + k);
        const NodeMoments nm = collide_node<false>(f, g, omega, dfac, a);
#pragma unroll
        for (int i = 0; i < 9; ++i) at(v[i], k) = f[i];
#pragma unroll
        for (int i = 0; i < 5; ++i) at(v[9 + i], k) = g[i];
        if (fluid) {
            acc.bad |= !(nm.rho > 0.f && nm.rho < INFINITY) || !(fabsf(nm.C) < INFINITY);
            ++acc.n;
            acc.m += nm.rd;
            acc.c += nm.C;
            if (outlet_k) {
                acc.q += nm.jx;  // rho u_x
                acc.qc += nm.C * nm.ux;
            }
        }
    }
}

__global__ void __launch_bounds__(128, 5) coupled_step_pairs(const StepArgs a)
{
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int wpb = blockDim.x >> 5;
    const long long P = a.plane;
    const float* __restrict__ S = a.src;
    float* __restrict__ D = a.dst;

    LaneDiag diag;
    bool bad = false;

    const int n = a.n_tiles64;
    const int stride = gridDim.x * wpb;
    int t = blockIdx.x * wpb + warp;
    uint2 next = t < n ? tile_at(a.tiles64, n, t, a.reverse) : make_uint2(0u, 0u);
    grid_dependency_sync();
    for (; t < n; t += stride) {
        const uint2 tile = next;  // the following entry is fetched one tile ahead
        if (t + stride < n) next = tile_at(a.tiles64, n, t + stride, a.reverse);
        const int y = int(tile.x >> kSegBits64);
        const int x0 = int(tile.x & ((1u << kSegBits64) - 1)) * kPairTileNodes + 2 * lane;
        const long long oC = (long long)y * a.pitch + x0;
        const long long oS = (long long)(y > 0 ? y - 1 : y) * a.pitch + x0;  // rows outside: as coupled_step_regs
        const long long oN = (long long)(y + 1 < a.ny ? y + 1 : y) * a.pitch + x0;
        const int halo_w = x0 > 0 ? -1 : 0;
        const int halo_e = x0 + 2 < a.pitch ? 2 : 1;
        const unsigned lk2 = __ldg(reinterpret_cast<const unsigned short*>(a.links + oC));
        const bool act = lk2 != 0xFFFFu;  // some node of this lane is fluid
        const unsigned ball = __ballot_sync(kFull, act);
        const bool ld_w = ((ball | (ball >> 1)) >> lane) & 1u;  // feeds lane + 1
        const bool ld_e = ((ball | (ball << 1)) >> lane) & 1u;  // feeds lane - 1
        float2 v[kPlanes];
        pull_pair(v, S, P, oC, oS, oN, halo_w, halo_e, act, ld_w, ld_e, lane);
        if (act) {
            bounce_back_pair(v, lk2, S, P, oC);
            const RowBC bw = a.rowbc[y];
            const RowBC be = a.rowbc[a.ny + y];
            QuadAcc q;
            collide_pair(v, lk2, x0, bw, be, a, S, oC, row_rates(a, y), q);
#pragma unroll
            for (int p = 0; p < kPlanes; ++p) stg2(D + p * P + oC, v[p]);
            bad |= q.bad;
            diag.add(q);
        }
    }

    if (__any_sync(kFull, bad) && lane == 0) atomicOr(a.err, 1u);
    block_partials(a, diag);
}

// One warp tile of the register variant as a function (the multi-step
// kernel's body; coupled_step_regs keeps the same code written out, which
// the register allocator handles without spills): pull, walls, ports,
// collisions and stores of the lane's four nodes (S holds time t, D
// receives t + 1).
template <typename T, bool kWalls>
__device__ __forceinline__ void regs_tile(const StepArgs& a, const T* __restrict__ S, T* __restrict__ D,
                                          long long P, uint2 tile, int lane, LaneDiag& diag, bool& bad)
{
    const int y = int(tile.x >> kColBits);
    const int x0 = tile_x0(tile) + 4 * lane;
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
    float4 v[kPlanes];
    pull_quad<false>(v, S, P, oC, oS, oN, halo_w, halo_e, act, ld_w, ld_e, lane);
    if (act) {
        bounce_back<T, kWalls>(v, lk, S, P, oC, static_cast<const T*>(a.wallv));
        const RowBC bw = a.rowbc[y];
        const RowBC be = a.rowbc[a.ny + y];
        QuadAcc q;
        collide_quad<T, true>(v, lk, x0, bw, be, a, S, oC, row_rates(a, y), q);
#pragma unroll
        for (int p = 0; p < kPlanes; ++p)
            Codec<T>::st4(D + p * P + oC, v[p], 0.f);
        bad |= q.bad;
        diag.add(q);
    }
}

// ---------------------------------------------------------------------------
// Variant 2: bulk-copy pipeline through shared memory
// ---------------------------------------------------------------------------
// One staged tile: the 14 plane rows the tile pulls from, each with a
// 16-byte halo on both sides (4 FP32 or 8 16-bit elements, so that every copy
// starts on a 16-byte boundary), the tile's 128 wall-link bytes, the port
// entries of its row and the tile's table entry.
template <typename T>
struct __align__(16) StageT {
    static constexpr int kHalo = 16 / int(sizeof(T));  // elements per 16 bytes
    T pl[kPlanes][kTileNodes + 2 * kHalo];
    unsigned links[kTileNodes / 4];
    RowBC bc[2];
    float4 rates;  // the row's relaxation rates (copied only for batches of chips)
    uint2 tile;
    uint2 pad;
};
using Stage = StageT<float>;
static_assert(sizeof(Stage) % 16 == 0 && sizeof(StageT<__half>) % 16 == 0,
              "stage size must keep 16-byte alignment");
static_assert(offsetof(Stage, links) % 16 == 0 && offsetof(Stage, bc) % 16 == 0 &&
                  offsetof(Stage, rates) % 16 == 0,
              "bulk-copy targets");
static_assert(offsetof(StageT<__half>, links) % 16 == 0 && offsetof(StageT<__half>, bc) % 16 == 0 &&
                  offsetof(StageT<__half>, rates) % 16 == 0,
              "bulk-copy targets");
static_assert(sizeof(StageT<__half>) == sizeof(StageT<__nv_bfloat16>), "16-bit stages");

// Stage ring: consumer warp c owns stages [c * per, (c + 1) * per) and takes
// the block's tiles c, c + nc, c + 2 nc, ...; its k-th tile goes to stage
// c * per + k % per as that stage's use k / per.  Every stage is therefore
// filled and drained in order by one producer and one consumer, so the
// parity waits on its two mbarriers never skip a phase.
//
// Copies must start and end on 16-byte boundaries: a row's copied span is
// widened to whole multiples of Q = 16 / sizeof(T) elements (4 FP32 or 8
// 16-bit), and the shifted planes take Q more on each side.
template <typename T, bool kWalls>
__global__ void __launch_bounds__(kBulkMaxThreads, 2) coupled_step_bulk(const StepArgs a, int per)
{
    using StageX = StageT<T>;
    constexpr int Q = StageX::kHalo;
    extern __shared__ __align__(128) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nc = (blockDim.x >> 5) - 1;  // consumer warps; the last warp produces
    const int n_stages = nc * per;
    StageX* st = reinterpret_cast<StageX*>(smem);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + size_t(n_stages) * sizeof(StageX));
    uint64_t* empty = full + n_stages;
    const long long P = a.plane;
    const T* __restrict__ S = reinterpret_cast<const T*>(a.src);
    T* __restrict__ D = reinterpret_cast<T*>(a.dst);
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
    grid_dependency_sync();

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
                const uint2 tile = tile_at(a.tiles, a.n_tiles, int(blockIdx.x) + j * G, a.reverse);
                if (batch > 0 && !mbar_wait(&empty[s], uint32_t(batch - 1) & 1u)) {
                    good = false;
                } else {
                    const int y = int(tile.x >> kColBits);
                    const int x0 = tile_x0(tile);
                    const int q0 = int(tile.y & 0xFFu), q1 = int((tile.y >> 8) & 0xFFu);
                    // columns of the lanes that hold fluid (widened to whole
                    // 16-byte units), and one unit more on each side for the
                    // planes that pull from x -+ 1
                    const int us = x0 + ((4 * q0) & ~(Q - 1));
                    const int ue = x0 + ((4 * q1 + 4 + Q - 1) & ~(Q - 1));
                    const int ss = us - Q > 0 ? us - Q : 0;
                    const int se = ue + Q < a.pitch ? ue + Q : a.pitch;
                    const long long rC = (long long)y * a.pitch;
                    const long long rS = (long long)(y > 0 ? y - 1 : y) * a.pitch;
                    const long long rN = (long long)(y + 1 < a.ny ? y + 1 : y) * a.pitch;
                    const uint32_t bytes = uint32_t(6 * (ue - us) + 8 * (se - ss)) * uint32_t(sizeof(T)) +
                                           kTileNodes + 2 * sizeof(RowBC) + (a.rates ? sizeof(float4) : 0);
                    st[s].tile = tile;  // ordered before the consumer by the arrive below
                    mbar_arrive_expect_tx(&full[s], bytes);
#pragma unroll
                    for (int p = 0; p < kPlanes; ++p) {
                        const long long r = src_row(p) == 0 ? rC : src_row(p) == 1 ? rS : rN;
                        const int b = src_col(p) == 0 ? us : ss;
                        const int e = src_col(p) == 0 ? ue : se;
                        bulk_g2s(&st[s].pl[p][b - x0 + Q], S + p * P + r + b, uint32_t(e - b) * uint32_t(sizeof(T)),
                                 &full[s]);
                    }
                    bulk_g2s(st[s].links, a.links + rC + x0, kTileNodes, &full[s]);
                    bulk_g2s(&st[s].bc[0], a.rowbc + y, sizeof(RowBC), &full[s]);
                    bulk_g2s(&st[s].bc[1], a.rowbc + a.ny + y, sizeof(RowBC), &full[s]);
                    if (a.rates) bulk_g2s(&st[s].rates, a.rates + y, sizeof(float4), &full[s]);
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
            const StageX& sg = st[s];
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
                    const T* row = sg.pl[p] + 4 * lane;
                    const float4 c = Codec<T>::lds4(row + Q, 0.f);
                    if (src_col(p) == 0) v[p] = c;
                    else if (src_col(p) == 1) v[p] = make_float4(Codec<T>::lds1(row + Q - 1, 0.f), c.x, c.y, c.z);
                    else v[p] = make_float4(c.y, c.z, c.w, Codec<T>::lds1(row + Q + 4, 0.f));
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[s]);  // the stage may be refilled
            if (act) {
                bounce_back<T, kWalls>(v, lk, S, P, oC, static_cast<const T*>(a.wallv));
                QuadAcc q;
                collide_quad(v, lk, x0, bw, be, a, S, oC, omega, q);
#pragma unroll
                for (int p = 0; p < kPlanes; ++p)
                    Codec<T>::st4(D + p * P + oC, v[p], 0.f);
                bad |= q.bad;
                diag.add(q);
            }
        }
        if (__any_sync(kFull, bad) && lane == 0) atomicOr(a.err, 1u);
    }
    block_partials(a, diag);
}

}  // namespace
}  // namespace lbm
