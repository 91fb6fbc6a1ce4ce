// lbm_adjoint.cu -- reverse-mode derivative (adjoint) of the coupled step.
//
// The forward step maps the stored post-collision state P(t) to P(t+1) =
// K(B(F(P(t)))): F the free flight with bounce-back, B the completion of open
// port nodes, K the collision of f and of g (whose equilibrium reads the
// velocity of the same node, Eq. cdeequilibrium).  Given A(t+1) = dJ/dP(t+1)
// the adjoint step is A(t) = F^T M(t) with M(t) = B^T K'^T A(t+1).  The
// reverse sweep carries M instead of A, so that each reverse step is one
// launch that reads its neighbours' M(t+1) once:
//   adjoint_collide  the first reverse step (t = n - 1): A(n) comes from the
//                    objective; recomputes X = B(F(P(t))) exactly as the step
//                    kernel does, applies K'(X)^T and B^T, stores M(t);
//   adjoint_fused    every other step: A(t+1) = F^T M(t+1) per node, a pull
//                    from x + e_i (bounce-back links return the node's own
//                    opposite entry) plus the do-nothing outlet term, kept
//                    in shared memory, then the same work as adjoint_collide.
// A(0) itself is not formed: the parameter derivatives are complete once
// M(0) is.  They accumulate in FP64: d/d(1/tau_g) per block, d/du_in and
// d/dC_in per port row.
#include "lbm_device.cuh"

namespace lbm {
namespace {

// A(t+1) of a lane's four nodes in global memory (the first reverse step).
struct NextGlobal {
    const float* p;  // entry (plane 0, node x0)
    long long P;
    __device__ __forceinline__ float operator()(int i, int k) const { return __ldg(p + i * P + k); }
};

// Per-warp stage of M(t+1) for a fused reverse step: plane p holds the row
// that the transposed free flight pulls plane p from (y + e_y of p), columns
// xs - 4 .. xs + 131 of the tile's segment starting at xs.
struct MidStage {
    float pl[kPlanes][kTileNodes + 8];
};

// Row (0 centre, 1 y - 1, 2 y + 1) and column (0 own, 1 x - 1, 2 x + 1) of
// the transposed free flight's source for plane p: x + e_p.
__device__ __forceinline__ constexpr int rev_row(int p) { return src_row(p) == 0 ? 0 : 3 - src_row(p); }
__device__ __forceinline__ constexpr int rev_col(int p) { return src_col(p) == 0 ? 0 : 3 - src_col(p); }
__device__ __forceinline__ constexpr int col_shift(int c) { return c == 1 ? -1 : c == 2 ? 1 : 0; }

// A(t+1) of a lane's four nodes from the stage: entry (i, k) sits at column
// 4 + 4 lane + k + (shift of plane i).  Each entry is the source of exactly
// one (plane, node), so a lane may overwrite its own entries (bounce-back
// links, do-nothing terms) without affecting any other lane.
struct NextStage {
    MidStage* st;
    int lane;
    __device__ __forceinline__ float& operator()(int i, int k) const
    {
        return st->pl[i][4 + 4 * lane + k + col_shift(rev_col(i))];
    }
};

// Transpose of the collision and of the port completion for the four nodes
// of one lane.  x holds X (fluid planes as deviations); A(t+1) is read and
// M(t) formed one node at a time (fewer live registers than whole quads):
// node k's entries of M(t) replace its entries of X in x as soon as X of
// the node has been read, and the quad is stored with 128-bit stores at the
// end.
template <typename Next>
__device__ __forceinline__ void collide_adjoint_quad(float4 (&x)[kPlanes], unsigned lk, int x0, int y,
                                                     long long oC, const RowBC& bw, const RowBC& be,
                                                     const AdjointArgs& A, const Next& next, KahanF& dwg)
{
    const long long P = A.plane;
    const bool open_w = bw.x >= 0 && ((A.open_mask >> (bw.chan_kind & 31)) & 1u);
    const bool open_e = be.x >= 0 && ((A.open_mask >> (be.chan_kind & 31)) & 1u);
    const float w = A.omega_f, wgr = A.omega_g;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const unsigned lb = (lk >> (8 * k)) & 0xFFu;
        float af[9], ag[5];
        if (lb == kSolid) {
#pragma unroll
            for (int i = 0; i < kPlanes; ++i) at(x[i], k) = 0.f;
            continue;
        }
        float f[9], g[5];
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            f[i] = at(x[i], k);
            af[i] = next(i, k);
        }
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            g[i] = at(x[9 + i], k);
            ag[i] = next(9 + i, k);
        }
        const int xk = x0 + k;
        const bool pw = open_w && bw.x == xk;
        const bool pe = !pw && open_e && be.x == xk;
        float Kd = 0.f;
        if (pw || pe) {
            const float fo_ax = pw ? f[3] : f[1];
            const float fo_dn = pw ? f[7] : f[8];
            const float fo_up = pw ? f[6] : f[5];
            Kd = f[0] + f[2] + f[4] + 2.f * (fo_ax + fo_dn + fo_up);
        }
        // ---- K'^T: the collision's Jacobian at X, transposed ----
        // f_eq_q = w_q rho [1 + 3 e.u + 9/2 (e.u)^2 - 3/2 u^2] with u = j / rho:
        //   d f_eq_q / d rho  = w_q (1 - 9/2 (e.u)^2 + 3/2 u^2)
        //   d f_eq_q / d j    = w_q (e (3 + 9 e.u) - 3 u)
        // and d rho / d f_i = 1, d j / d f_i = e_i.  The sums over q are
        // written out per direction pair (e.u of q and of opp(q) differ in sign).
        const float rd = ((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7])) + f[8];
        const float rho = 1.f + rd;
        const float jx = (f[1] - f[3]) + (f[5] - f[6]) + (f[8] - f[7]);
        const float jy = (f[2] - f[4]) + (f[5] + f[6]) - (f[7] + f[8]);
        const float irho = __fdividef(1.f, rho);  // fast reciprocal (2 ulp): rho stays near 1
        const float ux = jx * irho, uy = jy * irho;
        const float uu15 = 1.5f * (ux * ux + uy * uy);
        const float C = ((g[0] + g[1]) + (g[2] + g[3])) + g[4];
        const float e1 = ux, e2 = uy, e5 = ux + uy, e6 = uy - ux;  // e.u of q = 1, 2, 5, 6
        const float b0 = kWr * af[0];
        const float b1 = kWa * af[1], b2 = kWa * af[2], b3 = kWa * af[3], b4 = kWa * af[4];
        const float b5 = kWd * af[5], b6 = kWd * af[6], b7 = kWd * af[7], b8 = kWd * af[8];
        const float s13 = b1 + b3, s24 = b2 + b4, s57 = b5 + b7, s68 = b6 + b8;
        const float sb = b0 + (s13 + s24) + (s57 + s68);
        const float Ar = b0 * (1.f + uu15) + s13 * (1.f + uu15 - 4.5f * e1 * e1) + s24 * (1.f + uu15 - 4.5f * e2 * e2) +
                         s57 * (1.f + uu15 - 4.5f * e5 * e5) + s68 * (1.f + uu15 - 4.5f * e6 * e6);
        const float Ax = -3.f * ux * sb + 3.f * ((b1 - b3) + (b5 - b7) + (b8 - b6)) +
                         9.f * (e1 * s13 + e5 * s57 - e6 * s68);
        const float Ay = -3.f * uy * sb + 3.f * ((b2 - b4) + (b5 - b7) + (b6 - b8)) +
                         9.f * (e2 * s24 + e5 * s57 + e6 * s68);
        // g_eq_q = w_1 C (1 + e.u / c_s^2) for q = 1..4, the rest entry C - 4 w_1 C:
        //   d/dC = w_1 (1 + e.u / c_s^2) (1 - 4 w_1 at rest), d/d rho = -w_1 C e.u / (c_s^2 rho),
        //   d/dj = w_1 C e / (c_s^2 rho)
        const float c1 = A.wg1 * C;
        const float d13 = ag[1] - ag[3], d24 = ag[2] - ag[4];
        const float seu = ux * d13 + uy * d24;  // sum_q ag_q e.u
        const float sag = (ag[1] + ag[2]) + (ag[3] + ag[4]);
        const float Bc = ag[0] * (1.f - 4.f * A.wg1) + A.wg1 * (sag + A.inv_cs2g * seu);
        const float cr = c1 * A.inv_cs2g * irho;
        const float Br = -cr * seu, Bx = cr * d13, By = cr * d24;
        const float dw = ag[0] * ((C - 4.f * c1) - g[0]) + c1 * (sag + A.inv_cs2g * seu) -
                         ((ag[1] * g[1] + ag[2] * g[2]) + (ag[3] * g[3] + ag[4] * g[4]));
        dwg.add(dw);
        float nf[9], ng[5];
        {
            const float R = w * Ar + wgr * Br, X = w * Ax + wgr * Bx, Y = w * Ay + wgr * By;
            const float w1 = 1.f - w;
            nf[0] = w1 * af[0] + R;
            nf[1] = w1 * af[1] + (R + X);
            nf[3] = w1 * af[3] + (R - X);
            nf[2] = w1 * af[2] + (R + Y);
            nf[4] = w1 * af[4] + (R - Y);
            nf[5] = w1 * af[5] + (R + (X + Y));
            nf[7] = w1 * af[7] + (R - (X + Y));
            nf[6] = w1 * af[6] + (R + (Y - X));
            nf[8] = w1 * af[8] + (R - (Y - X));
        }
#pragma unroll
        for (int q = 0; q < 5; ++q) ng[q] = (1.f - wgr) * ag[q] + wgr * Bc;

        // ---- B^T: fold the completed populations into their sources ----
        if (pw || pe) {
            const RowBC b = pw ? bw : be;
            const int side = pw ? 0 : 1;
            const float s = pw ? 1.f : -1.f;
            const bool velocity = ((b.chan_kind >> 8) & 0xFF) == 0;
            const int ia = pw ? 1 : 3, iu = pw ? 5 : 6, idn = pw ? 8 : 7;      // unknown: (s,0), (s,+1), (s,-1)
            const int oa = pw ? 3 : 1, odn = pw ? 7 : 8, oup = pw ? 6 : 5;     // known: (-s,0), (-s,-1), (-s,+1)
            const float a_ax = nf[ia], a_up = nf[iu], a_dn = nf[idn];
            nf[ia] = nf[iu] = nf[idn] = 0.f;
            nf[oa] += a_ax;
            nf[odn] += a_up;
            nf[oup] += a_dn;
            nf[2] += -0.5f * a_up + 0.5f * a_dn;
            nf[4] += 0.5f * a_up - 0.5f * a_dn;
            const float G = s * (2.f / 3.f) * a_ax + s * (1.f / 6.f) * (a_up + a_dn);  // dJ/d(rho u_x)
            float dK;
            if (velocity) {
                const float den = 1.f - s * b.a;
                dK = G * b.a / den;
                atomicAdd(A.grad_u + side * A.ny + y, double(G) * double(1.f + Kd) / (double(den) * double(den)));
            } else {
                dK = -s * G;
            }
            nf[0] += dK;
            nf[2] += dK;
            nf[4] += dK;
            nf[oa] += 2.f * dK;
            nf[odn] += 2.f * dK;
            nf[oup] += 2.f * dK;
            const int gi = pw ? 1 : 3;
            const float ain = ng[gi];
            ng[gi] = 0.f;
            if (velocity) {  // g_in = C_in - (the other four)
#pragma unroll
                for (int q = 0; q < 5; ++q)
                    if (q != gi) ng[q] -= ain;
                atomicAdd(A.grad_c + side * A.ny + y, double(ain));
            } else {         // g_in = its own post-collision value of step t
                A.dn[side * A.ny + y] = ain;
            }
        }
#pragma unroll
        for (int q = 0; q < 9; ++q) at(x[q], k) = nf[q];
#pragma unroll
        for (int q = 0; q < 5; ++q) at(x[9 + q], k) = ng[q];
    }
#pragma unroll
    for (int i = 0; i < kPlanes; ++i) stg4(A.adj_mid + i * P + oC, x[i]);
}

// Per-block running sum of dJ/d(1/tau_g), one FP64 slot per block: the
// block's lanes are combined as double-float pairs (every warp gets here at
// the same moment, and the FP64 pipe is narrow), then one thread adds the
// block's sum to its slot in FP64.
__device__ __forceinline__ void block_add(double* slot, const KahanF& k)
{
    __shared__ DF red[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    const DF v = warp_sum(k.pair());
    if (lane == 0) red[warp] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        DF s = red[0];
        for (int i = 1; i < wpb; ++i) s = df_add(s, red[i]);
        slot[blockIdx.x] += df_value(s);
    }
}

// Where a lane's four nodes sit and which neighbouring quads hold fluid
// (every lane of the warp calls this: it votes).
struct QuadPos {
    int y, x0, halo_w, halo_e;
    long long oC, oS, oN;
    unsigned lk;
    bool act, ld_w, ld_e;
};

__device__ __forceinline__ QuadPos quad_pos(const AdjointArgs& A, uint2 tile, int lane)
{
    QuadPos q;
    q.y = int(tile.x >> kColBits);
    q.x0 = tile_x0(tile) + 4 * lane;
    q.oC = (long long)q.y * A.pitch + q.x0;
    q.oS = (long long)(q.y > 0 ? q.y - 1 : q.y) * A.pitch + q.x0;
    q.oN = (long long)(q.y + 1 < A.ny ? q.y + 1 : q.y) * A.pitch + q.x0;
    q.halo_w = q.x0 > 0 ? -1 : 0;
    q.halo_e = q.x0 + 4 < A.pitch ? 4 : 3;
    q.lk = __ldg(reinterpret_cast<const unsigned*>(A.links + q.oC));
    q.act = q.lk != 0xFFFFFFFFu;
    const unsigned ball = __ballot_sync(kFull, q.act);
    q.ld_w = ((ball | (ball >> 1)) >> lane) & 1u;
    q.ld_e = ((ball | (ball << 1)) >> lane) & 1u;
    return q;
}

// X = B(F(P(t))) for an active lane: bounce-back, then the forward's port
// completion, so that x is exactly the pre-collision state of the step.
__device__ __forceinline__ void complete_quad(float4 (&x)[kPlanes], const QuadPos& q, const RowBC& bw,
                                              const RowBC& be, const AdjointArgs& A)
{
    const long long P = A.plane;
    bounce_back(x, q.lk, A.state, P, q.oC);
    const bool open_w = bw.x >= 0 && ((A.open_mask >> (bw.chan_kind & 31)) & 1u);
    const bool open_e = be.x >= 0 && ((A.open_mask >> (be.chan_kind & 31)) & 1u);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const bool pw = open_w && bw.x == q.x0 + k;
        const bool pe = !pw && open_e && be.x == q.x0 + k;
        if ((pw || pe) && ((q.lk >> (8 * k)) & 0xFFu) != kSolid) {
            float f[9], g[5];
#pragma unroll
            for (int i = 0; i < 9; ++i) f[i] = at(x[i], k);
#pragma unroll
            for (int i = 0; i < 5; ++i) g[i] = at(x[9 + i], k);
            complete_port(f, g, pw, pw ? bw : be, A.state, P, q.oC + k);
#pragma unroll
            for (int i = 0; i < 9; ++i) at(x[i], k) = f[i];
#pragma unroll
            for (int i = 0; i < 5; ++i) at(x[9 + i], k) = g[i];
        }
    }
}

// Copies of M(t+1) for the tile into the warp's stage (cp.async, 16 bytes a
// lane and row, through L2): lane l copies its own 4 values of each row it
// needs (lanes q0 .. q1 of the tile's fluid range, one more on each side for
// the shifted planes), lanes 0 and 31 the neighbouring segments' 4 edge
// values.  Only values that some fluid node of the tile pulls are used.
__device__ __forceinline__ void issue_mid(const AdjointArgs& A, const QuadPos& q, uint2 tile, MidStage& st, int lane)
{
    const long long P = A.plane;
    const int xs = q.x0 - 4 * lane;
    const int q0 = int(tile.y & 0xFFu), q1 = int((tile.y >> 8) & 0xFFu);
    const bool own = lane >= q0 && lane <= q1;
    const bool wide = lane >= q0 - 1 && lane <= q1 + 1;
#pragma unroll
    for (int p = 0; p < kPlanes; ++p) {
        const int sr = rev_row(p), sc = rev_col(p);
        const float* row = A.mid_next + p * P + (sr == 0 ? q.oC : sr == 1 ? q.oS : q.oN) - 4 * lane;
        if (sc == 0 ? own : wide) cp_async16(&st.pl[p][4 + 4 * lane], row + 4 * lane);
        if (sc == 1 && lane == 0 && q0 == 0 && xs > 0) cp_async16(&st.pl[p][0], row - 4);
        if (sc == 2 && lane == 31 && q1 == 31 && xs + kTileNodes < A.pitch)
            cp_async16(&st.pl[p][4 + kTileNodes], row + kTileNodes);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}

// A(t+1) = F^T M(t+1) in the stage, once its copies have landed: a
// bounce-back link of direction i (the pull source of opp(i) is not fluid)
// takes the node's own opposite entry of M(t+1) (from global memory, only
// next to walls); at an open pressure-port node the scalar population with
// e_x = s gets the do-nothing term of step t+1.  kCoherent: M(t+1) and dn
// were written by other blocks of the same launch (the multi-step kernel),
// so they are read through L2.
template <bool kCoherent>
__device__ __forceinline__ float4 ld4_mid(const float* p)
{
    if constexpr (kCoherent) return __ldcg(reinterpret_cast<const float4*>(p));
    else return ldg4(p);
}

template <bool kCoherent>
__device__ __forceinline__ void transposed_flight(const NextStage& next, const QuadPos& q, const RowBC& bw,
                                                  const RowBC& be, const AdjointArgs& A)
{
    const long long P = A.plane;
    const float* __restrict__ M = A.mid_next;
    unsigned wall = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const unsigned lb = (q.lk >> (8 * k)) & 0xFFu;
        if (lb != kSolid) wall |= lb;
    }
    if (wall) {
#pragma unroll
        for (int i = 1; i <= 8; ++i) {
            const int o = opp(i);
            if (wall & (1u << (o - 1))) {
                const float4 own = ld4_mid<kCoherent>(M + o * P + q.oC);
                const float4 ownc = i <= 4 ? ld4_mid<kCoherent>(M + (9 + o) * P + q.oC) : own;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const unsigned lb = (q.lk >> (8 * k)) & 0xFFu;
                    if (lb != kSolid && ((lb >> (o - 1)) & 1u)) {
                        next(i, k) = at(own, k);
                        if (i <= 4) next(9 + i, k) = at(ownc, k);
                    }
                }
            }
        }
    }
    const uint32_t m = A.open_mask_next;
    const bool dn_w = bw.x >= 0 && ((m >> (bw.chan_kind & 31)) & 1u) && (bw.chan_kind >> 8) == 1;
    const bool dn_e = be.x >= 0 && ((m >> (be.chan_kind & 31)) & 1u) && (be.chan_kind >> 8) == 1;
    if (dn_w || dn_e) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (((q.lk >> (8 * k)) & 0xFFu) == kSolid) continue;
            if (dn_w && bw.x == q.x0 + k) next(10, k) += kCoherent ? __ldcg(A.dn + q.y) : A.dn[q.y];
            else if (dn_e && be.x == q.x0 + k) next(12, k) += kCoherent ? __ldcg(A.dn + A.ny + q.y) : A.dn[A.ny + q.y];
        }
    }
}

// The first reverse step: A(t+1) = A(n) is read from global memory.
__global__ void __launch_bounds__(kAdjointBlock, 4) adjoint_collide(const AdjointArgs A)
{
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int wpb = blockDim.x >> 5;
    const long long P = A.plane;
    KahanF dwg;
    grid_dependency_sync();
    for (int t = blockIdx.x * wpb + warp; t < A.n_tiles; t += gridDim.x * wpb) {
        const QuadPos q = quad_pos(A, tile_at(A.tiles, A.n_tiles, t, A.reverse), lane);
        float4 x[kPlanes];
        pull_quad<false>(x, A.state, P, q.oC, q.oS, q.oN, q.halo_w, q.halo_e, q.act, q.ld_w, q.ld_e, lane);
        if (!q.act) continue;
        const RowBC bw = A.rowbc[q.y];
        const RowBC be = A.rowbc[A.ny + q.y];
        complete_quad(x, q, bw, be, A);
        collide_adjoint_quad(x, q.lk, q.x0, q.y, q.oC, bw, be, A, NextGlobal{A.adj_next + q.oC, P}, dwg);
    }
    block_add(A.grad_w, dwg);
}

// Every later reverse step: A(t+1) = F^T M(t+1) gathered into shared memory
// (each thread reads back only its own entries, so no barrier), then X,
// K'^T and B^T as in adjoint_collide.  dn carries the do-nothing terms from
// one step to the next: the node that reads the entry of step t+1 is the
// node that then writes the one of step t.
// One tile of a fused reverse step (the body of adjoint_fused and of the
// multi-step kernel): the copies of M(t+1) into the warp's stage and the
// loads of P(t) into registers are in flight together; then X, A(t+1) in
// the stage, K'^T and B^T.
template <bool kCoherent>
__device__ __forceinline__ void fused_tile(const AdjointArgs& A, uint2 tile, int lane, MidStage& st, KahanF& dwg)
{
    const long long P = A.plane;
    const QuadPos q = quad_pos(A, tile, lane);
    issue_mid(A, q, tile, st, lane);
    float4 x[kPlanes];
    pull_quad<false>(x, A.state, P, q.oC, q.oS, q.oN, q.halo_w, q.halo_e, q.act, q.ld_w, q.ld_e, lane);
    const RowBC bw = A.rowbc[q.y];
    const RowBC be = A.rowbc[A.ny + q.y];
    if (q.act) complete_quad(x, q, bw, be, A);
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncwarp();
    const NextStage next{&st, lane};
    if (q.act) {
        transposed_flight<kCoherent>(next, q, bw, be, A);
        collide_adjoint_quad(x, q.lk, q.x0, q.y, q.oC, bw, be, A, next, dwg);
    }
    __syncwarp();  // the stage is read before the next tile's copies overwrite it
}

__global__ void __launch_bounds__(kAdjointBlock, 4) adjoint_fused(const AdjointArgs A)
{
    extern __shared__ __align__(16) unsigned char next_smem[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int wpb = blockDim.x >> 5;
    MidStage& st = reinterpret_cast<MidStage*>(next_smem)[warp];
    KahanF dwg;
    grid_dependency_sync();
    for (int t = blockIdx.x * wpb + warp; t < A.n_tiles; t += gridDim.x * wpb)
        fused_tile<false>(A, tile_at(A.tiles, A.n_tiles, t, A.reverse), lane, st, dwg);
    block_add(A.grad_w, dwg);
}

// Reverse steps j = j_hi down to j_lo in one cooperative launch (every block
// resident), a grid-wide barrier between them: step j reads the state
// state_lo + (j - j_lo) stride and the valve words masks[j - j_lo],
// masks[j - j_lo + 1]; M alternates between mid_a (M(j_hi + 1) on entry)
// and mid_b.  The step's own reads of M and dn go through L2.  A barrier
// that times out stops the kernel with bit 1 of the error word set.
__global__ void __launch_bounds__(kAdjointBlock, 4)
    adjoint_steps_coop(const AdjointArgs A0, int j_hi, int j_lo, const float* state_lo, long long stride,
                       const uint32_t* masks, float* mid_a, float* mid_b, unsigned* count)
{
    extern __shared__ __align__(16) unsigned char next_smem[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int wpb = blockDim.x >> 5;
    MidStage& st = reinterpret_cast<MidStage*>(next_smem)[warp];
    KahanF dwg;
    for (int j = j_hi, s = 0; j >= j_lo; --j, ++s) {
        AdjointArgs A = A0;
        A.state = state_lo + (j - j_lo) * stride;
        A.open_mask = __ldg(masks + (j - j_lo));
        A.open_mask_next = __ldg(masks + (j - j_lo) + 1);
        A.mid_next = (s & 1) ? mid_b : mid_a;
        A.adj_mid = (s & 1) ? mid_a : mid_b;
        A.reverse = A0.reverse ^ (s & 1);
        for (int t = blockIdx.x * wpb + warp; t < A.n_tiles; t += gridDim.x * wpb)
            fused_tile<true>(A, tile_at(A.tiles, A.n_tiles, t, A.reverse), lane, st, dwg);
        if (j > j_lo && !grid_barrier(count, unsigned(s + 1) * gridDim.x + A0.barrier_extra, A0.err)) break;
    }
    block_add(A0.grad_w, dwg);
}

// J = sum w (C - target)^2 at the final state, and its derivative with
// respect to the stored populations (A must be zero on entry).
__global__ void adjoint_seed(const float* state, long long plane, int pitch, const int* ox, const int* oy,
                             const float* target, const float* weight, int n, float* adj, double* J)
{
    __shared__ double red[32];
    double part = 0.0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        const long long o = (long long)oy[k] * pitch + ox[k];
        const float C = ((state[9 * plane + o] + state[10 * plane + o]) + (state[11 * plane + o] + state[12 * plane + o])) +
                        state[13 * plane + o];
        const double d = double(C) - double(target[k]);
        part += double(weight[k]) * d * d;
        const float gC = float(2.0 * double(weight[k]) * d);
#pragma unroll
        for (int i = 0; i < 5; ++i) atomicAdd(adj + (9 + i) * plane + o, gC);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    part = warp_sum(part);
    if (lane == 0) red[warp] = part;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < int(blockDim.x >> 5); ++i) s += red[i];
        *J = s;
    }
}

__global__ void sum_doubles(const double* v, int n, double* out)
{
    __shared__ double red[32];
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += v[i];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    s = warp_sum(s);
    if (lane == 0) red[warp] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < int(blockDim.x >> 5); ++i) t += red[i];
        *out = t;
    }
}

}  // namespace

cudaError_t adjoint_occupancy(int* blocks_per_sm)
{
    const size_t smem = adjoint_fused_smem(kAdjointBlock);
    cudaError_t e = cudaFuncSetAttribute(adjoint_fused, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    int a = 0, b = 0;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, adjoint_collide, kAdjointBlock, 0);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, adjoint_fused, kAdjointBlock, smem);
    *blocks_per_sm = a < b ? a : b;
    return e;
}

cudaError_t adjoint_coop_occupancy(int* blocks_per_sm)
{
    const size_t smem = adjoint_fused_smem(kAdjointBlock);
    cudaError_t e = cudaFuncSetAttribute(adjoint_steps_coop, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, adjoint_steps_coop,
                                                                           kAdjointBlock, smem);
    return e;
}

cudaError_t launch_adjoint_steps_coop(const AdjointArgs& a, int j_hi, int j_lo, const float* state_lo,
                                      long long stride, const uint32_t* masks, float* mid_a, float* mid_b,
                                      unsigned* count, int grid, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(count, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kAdjointBlock);
    cfg.dynamicSmemBytes = adjoint_fused_smem(kAdjointBlock);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;  // all blocks resident, or the launch fails
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, adjoint_steps_coop, a, j_hi, j_lo, state_lo, stride, masks, mid_a, mid_b, count);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t launch_adjoint_step(const AdjointArgs& a, bool first, int grid, cudaStream_t s)
{
    // a programmatic dependent of the kernel before it (waits for it in
    // grid_dependency_sync before touching any buffer)
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kAdjointBlock);
    cfg.dynamicSmemBytes = first ? 0 : adjoint_fused_smem(kAdjointBlock);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e = first ? cudaLaunchKernelEx(&cfg, adjoint_collide, a) : cudaLaunchKernelEx(&cfg, adjoint_fused, a);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t launch_adjoint_seed(const float* state, long long plane, int pitch, const int* ox, const int* oy,
                                const float* target, const float* weight, int n, float* adj, double* J,
                                cudaStream_t s)
{
    adjoint_seed<<<1, 256, 0, s>>>(state, plane, pitch, ox, oy, target, weight, n, adj, J);
    return cudaGetLastError();
}

cudaError_t launch_sum_doubles(const double* v, int n, double* out, cudaStream_t s)
{
    sum_doubles<<<1, 256, 0, s>>>(v, n, out);
    return cudaGetLastError();
}

}  // namespace lbm
