// lbm_adjoint.cu -- reverse-mode derivative (adjoint) of the coupled step.
//
// The forward step maps the stored post-collision state P(t) to P(t+1) =
// K(B(F(P(t)))): F the free flight with bounce-back, B the completion of open
// port nodes, K the collision of f and of g (whose equilibrium reads the
// velocity of the same node, Eq. cdeequilibrium).  Given A(t+1) = dJ/dP(t+1)
// the adjoint step forms A(t) = F^T B^T K'^T A(t+1) in two launches:
//   adjoint_collide  per node: recomputes X = B(F(P(t))) exactly as the step
//                    kernel does, applies K'(X)^T to A(t+1) and the transpose
//                    of the port completion, and stores the result A*;
//   adjoint_stream   per node: the transposed free flight, which is a pull
//                    from x + e_i (bounce-back links return the node's own
//                    opposite entry), plus the do-nothing outlet term.
// Derivatives with respect to the parameters accumulate in FP64: d/d(1/tau_g)
// per block, d/du_in and d/dC_in per port row.
#include "lbm_device.cuh"

namespace lbm {
namespace {

// Transpose of the collision and of the port completion for the four nodes
// of one lane.  x holds X (fluid planes as deviations); A(t+1) is read and
// A* written one node at a time (fewer live registers than whole quads).
__device__ __forceinline__ void collide_adjoint_quad(const float4 (&x)[kPlanes], unsigned lk, int x0, int y,
                                                     long long oC, const RowBC& bw, const RowBC& be,
                                                     const AdjointArgs& A, KahanF& dwg)
{
    const long long P = A.plane;
    const bool open_w = bw.x >= 0 && ((A.open_mask >> (bw.chan_kind & 31)) & 1u);
    const bool open_e = be.x >= 0 && ((A.open_mask >> (be.chan_kind & 31)) & 1u);
    const float w = A.omega_f, wgr = A.omega_g;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const unsigned lb = (lk >> (8 * k)) & 0xFFu;
        float af[9], ag[5];
        const long long o = oC + k;
        if (lb == kSolid) {
#pragma unroll
            for (int i = 0; i < kPlanes; ++i) A.adj_mid[i * P + o] = 0.f;
            continue;
        }
        float f[9], g[5];
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            f[i] = at(x[i], k);
            af[i] = __ldg(A.adj_next + i * P + o);
        }
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            g[i] = at(x[9 + i], k);
            ag[i] = __ldg(A.adj_next + (9 + i) * P + o);
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
        const float rd = ((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7])) + f[8];
        const float rho = 1.f + rd;
        const float jx = (f[1] - f[3]) + (f[5] - f[6]) + (f[8] - f[7]);
        const float jy = (f[2] - f[4]) + (f[5] + f[6]) - (f[7] + f[8]);
        const float ux = jx / rho, uy = jy / rho;
        const float uu = ux * ux + uy * uy;
        const float C = ((g[0] + g[1]) + (g[2] + g[3])) + g[4];
        // f_eq_k = w_k [rho + 3 e.j + 9/2 (e.j)^2 / rho - 3/2 j^2 / rho]
        float Ar = 0.f, Ax = 0.f, Ay = 0.f;
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            const float ex = float(q == 1 || q == 5 || q == 8) - float(q == 3 || q == 6 || q == 7);
            const float ey = float(q == 2 || q == 5 || q == 6) - float(q == 4 || q == 7 || q == 8);
            const float wq = q == 0 ? kWr : q <= 4 ? kWa : kWd;
            const float eu = ex * ux + ey * uy;
            Ar += af[q] * wq * (1.f - 4.5f * eu * eu + 1.5f * uu);
            Ax += af[q] * wq * (3.f * ex + 9.f * eu * ex - 3.f * ux);
            Ay += af[q] * wq * (3.f * ey + 9.f * eu * ey - 3.f * uy);
        }
        // g_eq_k = w_k C [1 + e.j / (rho c_s^2)]; the rest entry is C - 4 w_1 C
        float Bc = ag[0] * (1.f - 4.f * A.wg1), Br = 0.f, Bx = 0.f, By = 0.f;
        float dw = ag[0] * ((C - 4.f * A.wg1 * C) - g[0]);
        {
            const float c1 = A.wg1 * C;
            const float e4[4][2] = {{1.f, 0.f}, {0.f, 1.f}, {-1.f, 0.f}, {0.f, -1.f}};
#pragma unroll
            for (int q = 1; q <= 4; ++q) {
                const float ex = e4[q - 1][0], ey = e4[q - 1][1];
                const float eu = ex * ux + ey * uy;
                Bc += ag[q] * A.wg1 * (1.f + eu * A.inv_cs2g);
                Br += ag[q] * c1 * (-eu * A.inv_cs2g / rho);
                Bx += ag[q] * c1 * ex * A.inv_cs2g / rho;
                By += ag[q] * c1 * ey * A.inv_cs2g / rho;
                dw += ag[q] * (c1 * (1.f + eu * A.inv_cs2g) - g[q]);
            }
        }
        dwg.add(dw);
        float nf[9], ng[5];
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            const float ex = float(q == 1 || q == 5 || q == 8) - float(q == 3 || q == 6 || q == 7);
            const float ey = float(q == 2 || q == 5 || q == 6) - float(q == 4 || q == 7 || q == 8);
            nf[q] = (1.f - w) * af[q] + w * (Ar + Ax * ex + Ay * ey) + wgr * (Br + Bx * ex + By * ey);
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
        for (int q = 0; q < 9; ++q) A.adj_mid[q * P + o] = nf[q];
#pragma unroll
        for (int q = 0; q < 5; ++q) A.adj_mid[(9 + q) * P + o] = ng[q];
    }
}

// Per-block running sum of dJ/d(1/tau_g), one slot per block.
__device__ __forceinline__ void block_add(double* slot, double v)
{
    __shared__ double red[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    v = warp_sum(v);
    if (lane == 0) red[warp] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < wpb; ++i) s += red[i];
        slot[blockIdx.x] += s;
    }
}

__global__ void __launch_bounds__(256) adjoint_collide(const AdjointArgs A)
{
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int wpb = blockDim.x >> 5;
    const long long P = A.plane;
    const float* __restrict__ S = A.state;
    KahanF dwg;
    grid_dependency_sync();
    for (int t = blockIdx.x * wpb + warp; t < A.n_tiles; t += gridDim.x * wpb) {
        const uint2 tile = A.tiles[t];
        const int y = int(tile.x >> kSegBits);
        const int x0 = int(tile.x & ((1u << kSegBits) - 1)) * kTileNodes + 4 * lane;
        const long long oC = (long long)y * A.pitch + x0;
        const long long oS = (long long)(y > 0 ? y - 1 : y) * A.pitch + x0;
        const long long oN = (long long)(y + 1 < A.ny ? y + 1 : y) * A.pitch + x0;
        const int halo_w = x0 > 0 ? -1 : 0;
        const int halo_e = x0 + 4 < A.pitch ? 4 : 3;
        const unsigned lk = __ldg(reinterpret_cast<const unsigned*>(A.links + oC));
        const bool act = lk != 0xFFFFFFFFu;
        const unsigned ball = __ballot_sync(kFull, act);
        const bool ld_w = ((ball | (ball >> 1)) >> lane) & 1u;
        const bool ld_e = ((ball | (ball << 1)) >> lane) & 1u;
        float4 x[kPlanes];
        pull_quad<false>(x, S, P, oC, oS, oN, halo_w, halo_e, act, ld_w, ld_e, lane);
        if (!act) continue;
        bounce_back(x, lk, S, P, oC);
        const RowBC bw = A.rowbc[y];
        const RowBC be = A.rowbc[A.ny + y];
        // the forward's port completion, so that x is exactly X
        {
            const bool open_w = bw.x >= 0 && ((A.open_mask >> (bw.chan_kind & 31)) & 1u);
            const bool open_e = be.x >= 0 && ((A.open_mask >> (be.chan_kind & 31)) & 1u);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const bool pw = open_w && bw.x == x0 + k;
                const bool pe = !pw && open_e && be.x == x0 + k;
                if ((pw || pe) && ((lk >> (8 * k)) & 0xFFu) != kSolid) {
                    float f[9], g[5];
#pragma unroll
                    for (int i = 0; i < 9; ++i) f[i] = at(x[i], k);
#pragma unroll
                    for (int i = 0; i < 5; ++i) g[i] = at(x[9 + i], k);
                    complete_port(f, g, pw, pw ? bw : be, S, P, oC + k);
#pragma unroll
                    for (int i = 0; i < 9; ++i) at(x[i], k) = f[i];
#pragma unroll
                    for (int i = 0; i < 5; ++i) at(x[9 + i], k) = g[i];
                }
            }
        }
        collide_adjoint_quad(x, lk, x0, y, oC, bw, be, A, dwg);
    }
    block_add(A.grad_w, dwg.value());
}

// Transposed free flight: A(t)_i(y) = A*_i(y + e_i) when y + e_i is fluid,
// else A*_opp(i)(y) (the bounce-back link), plus, at an open pressure-port
// node, the do-nothing term of the scalar population with e_x = s.
__global__ void __launch_bounds__(256) adjoint_stream(const AdjointArgs A)
{
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int wpb = blockDim.x >> 5;
    const long long P = A.plane;
    const float* __restrict__ S = A.adj_mid;
    grid_dependency_sync();
    for (int t = blockIdx.x * wpb + warp; t < A.n_tiles; t += gridDim.x * wpb) {
        // the reverse of adjoint_collide's order: start where it ended (in L2)
        const uint2 tile = tile_at(A.tiles, A.n_tiles, t, 1);
        const int y = int(tile.x >> kSegBits);
        const int x0 = int(tile.x & ((1u << kSegBits) - 1)) * kTileNodes + 4 * lane;
        const long long oC = (long long)y * A.pitch + x0;
        const long long oS = (long long)(y > 0 ? y - 1 : y) * A.pitch + x0;
        const long long oN = (long long)(y + 1 < A.ny ? y + 1 : y) * A.pitch + x0;
        const int halo_w = x0 > 0 ? -1 : 0;
        const int halo_e = x0 + 4 < A.pitch ? 4 : 3;
        const unsigned lk = __ldg(reinterpret_cast<const unsigned*>(A.links + oC));
        const bool act = lk != 0xFFFFFFFFu;
        const unsigned ball = __ballot_sync(kFull, act);
        const bool ld_w = ((ball | (ball >> 1)) >> lane) & 1u;
        const bool ld_e = ((ball | (ball << 1)) >> lane) & 1u;
        float4 v[kPlanes];
        pull_quad<true>(v, S, P, oC, oS, oN, halo_w, halo_e, act, ld_w, ld_e, lane);
        if (!act) continue;
        // bounce-back links: the link of direction i from y is a wall when
        // the pull source of direction opp(i) at y is not fluid
        unsigned wall = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const unsigned lb = (lk >> (8 * k)) & 0xFFu;
            if (lb != kSolid) wall |= lb;
        }
        if (wall) {
#pragma unroll
            for (int i = 1; i <= 8; ++i) {
                const int o = opp(i);
                if (wall & (1u << (o - 1))) {
                    const float4 own = ldg4(S + o * P + oC);
                    const float4 ownc = i <= 4 ? ldg4(S + (9 + o) * P + oC) : own;
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        if ((lk >> (8 * k + o - 1)) & 1u) {
                            at(v[i], k) = at(own, k);
                            if (i <= 4) at(v[9 + i], k) = at(ownc, k);
                        }
                    }
                }
            }
        }
        const RowBC bw = A.rowbc[y];
        const RowBC be = A.rowbc[A.ny + y];
        const bool dn_w = bw.x >= 0 && ((A.open_mask >> (bw.chan_kind & 31)) & 1u) && (bw.chan_kind >> 8) == 1;
        const bool dn_e = be.x >= 0 && ((A.open_mask >> (be.chan_kind & 31)) & 1u) && (be.chan_kind >> 8) == 1;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const unsigned lb = (lk >> (8 * k)) & 0xFFu;
            if (lb == kSolid) {
#pragma unroll
                for (int p = 0; p < kPlanes; ++p) at(v[p], k) = 0.f;
                continue;
            }
            if (dn_w && bw.x == x0 + k) at(v[10], k) += A.dn[y];
            else if (dn_e && be.x == x0 + k) at(v[12], k) += A.dn[A.ny + y];
        }
#pragma unroll
        for (int p = 0; p < kPlanes; ++p) stg4(A.adj_out + p * P + oC, v[p]);
    }
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

cudaError_t adjoint_occupancy(int block, int* blocks_per_sm)
{
    int a = 0, b = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, adjoint_collide, block, 0);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, adjoint_stream, block, 0);
    *blocks_per_sm = a < b ? a : b;
    return e;
}

cudaError_t launch_adjoint_step(const AdjointArgs& a, int grid, int block, cudaStream_t s)
{
    // both as programmatic dependents of the kernel before them (each waits
    // for it in grid_dependency_sync before touching any buffer)
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, adjoint_collide, a);
    if (e == cudaSuccess) e = cudaLaunchKernelEx(&cfg, adjoint_stream, a);
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
