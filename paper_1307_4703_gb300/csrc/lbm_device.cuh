// lbm_device.cuh -- device code shared by the step kernels (lbm_kernels.cu)
// and the adjoint kernels (lbm_adjoint.cu): lattice tables, the inline-PTX
// bulk-copy and mbarrier helpers, and the per-node arithmetic of the coupled
// step (Tanaka & Iber, arXiv 1307.4703, "Numerical Methods" and "Boundary
// Conditions").  Everything here has internal linkage.
#pragma once

#include <cmath>
#include <cstddef>
#include <type_traits>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

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
__device__ __forceinline__ float2 ldg2(const float* p)
{
    return __ldg(reinterpret_cast<const float2*>(p));
}
__device__ __forceinline__ void stg2(float* p, const float2& v)
{
    *reinterpret_cast<float2*>(p) = v;
}
__device__ __forceinline__ float& at(float2& v, int k) { return k == 0 ? v.x : v.y; }
__device__ __forceinline__ float at(const float2& v, int k) { return k == 0 ? v.x : v.y; }
__device__ __forceinline__ float& at(float4& v, int k)
{
    return k == 0 ? v.x : k == 1 ? v.y : k == 2 ? v.z : v.w;
}
__device__ __forceinline__ float at(const float4& v, int k)
{
    return k == 0 ? v.x : k == 1 ? v.y : k == 2 ? v.z : v.w;
}

// Programmatic dependent launch: wait until the previous kernel of the
// stream has completed and its writes are visible (a no-op for a launch
// without that dependency), then allow the next kernel to launch, so that its
// blocks are placed and set up while this grid's last blocks finish.  Every
// thread calls it before its first access to data that another kernel writes.
__device__ __forceinline__ void grid_dependency_sync()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Entry t of the tile table, counted from its end when `reverse` is set.
// Consecutive steps alternate the direction, so a step starts on the rows
// the previous step wrote last, which are still in L2.
__device__ __forceinline__ uint2 tile_at(const uint2* tiles, int n, int t, int reverse)
{
    return tiles[reverse ? n - 1 - t : t];
}

// First node (column) of a 128-node tile and its row.
__device__ __forceinline__ int tile_x0(uint2 tile)
{
    return int(tile.x & ((1u << kColBits) - 1)) * kTileStart;
}


// Storage of the populations.  FP32 keeps them as they are (fluid planes as
// f_i - w_i, scalar planes as g_i).  FP16 and BF16 hold deviations from a
// reference: the fluid planes the same f_i - w_i, the scalar planes
// g_i - w_i C_ref.  All arithmetic is FP32.  The step kernels move the
// stored deviations as they are (their collision is written for deviations);
// the codec's offset argument, added on loading and subtracted on storing,
// serves the kernels and the port rules that need g_i itself.
// x + off, skipped when off is zero: the fluid planes have no offset, and
// x + 0.0f cannot be folded away (it turns -0 into +0), while this test
// folds when off is a constant after inlining.
__device__ __forceinline__ float add_offset(float x, float off) { return off != 0.f ? x + off : x; }
__device__ __forceinline__ float4 add_offset(float4 v, float off)
{
    return off != 0.f ? make_float4(v.x + off, v.y + off, v.z + off, v.w + off) : v;
}

template <typename T>
struct Codec;

template <>
struct Codec<float> {
    static __device__ __forceinline__ float4 ld4(const float* p, float) { return ldg4(p); }
    static __device__ __forceinline__ float ld1(const float* p, float) { return __ldg(p); }
    static __device__ __forceinline__ void st4(float* p, const float4& v, float) { stg4(p, v); }
    static __device__ __forceinline__ void st1(float* p, float v, float) { *p = v; }
    static __device__ __forceinline__ float4 lds4(const float* p, float) { return *reinterpret_cast<const float4*>(p); }
    static __device__ __forceinline__ float lds1(const float* p, float) { return *p; }
};

// FP32 storage read coherently at L2 (ld.global.cg), for a kernel that
// reads in one time step what other blocks of the same launch wrote in the
// step before (the multi-step kernel): the read-only path of __ldg may not
// be used for such data.
struct F32Coherent {
    float v;
};

template <>
struct Codec<F32Coherent> {
    static __device__ __forceinline__ const float* f(const F32Coherent* p) { return reinterpret_cast<const float*>(p); }
    static __device__ __forceinline__ float* f(F32Coherent* p) { return reinterpret_cast<float*>(p); }
    static __device__ __forceinline__ float4 ld4(const F32Coherent* p, float)
    {
        return __ldcg(reinterpret_cast<const float4*>(p));
    }
    static __device__ __forceinline__ float ld1(const F32Coherent* p, float) { return __ldcg(f(p)); }
    static __device__ __forceinline__ void st4(F32Coherent* p, const float4& v, float) { stg4(f(p), v); }
    static __device__ __forceinline__ void st1(F32Coherent* p, float v, float) { *f(p) = v; }
};

// Storage types that hold FP32 values as they are (no deviation offsets).
template <typename T>
constexpr bool kStoresF32 = std::is_same<T, float>::value || std::is_same<T, F32Coherent>::value;

template <>
struct Codec<__half> {
    static __device__ __forceinline__ float4 ld4(const __half* p, float off)
    {
        const uint2 r = __ldg(reinterpret_cast<const uint2*>(p));
        const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&r.x));
        const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&r.y));
        return add_offset(make_float4(a.x, a.y, b.x, b.y), off);
    }
    static __device__ __forceinline__ float ld1(const __half* p, float off) { return add_offset(__half2float(__ldg(p)), off); }
    static __device__ __forceinline__ void st4(__half* p, const float4& v, float off)
    {
        const __half2 a = __floats2half2_rn(v.x - off, v.y - off);
        const __half2 b = __floats2half2_rn(v.z - off, v.w - off);
        uint2 r;
        r.x = *reinterpret_cast<const unsigned*>(&a);
        r.y = *reinterpret_cast<const unsigned*>(&b);
        *reinterpret_cast<uint2*>(p) = r;
    }
    static __device__ __forceinline__ void st1(__half* p, float v, float off) { *p = __float2half_rn(v - off); }
    static __device__ __forceinline__ float4 lds4(const __half* p, float off)
    {
        const uint2 r = *reinterpret_cast<const uint2*>(p);
        const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&r.x));
        const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&r.y));
        return add_offset(make_float4(a.x, a.y, b.x, b.y), off);
    }
    static __device__ __forceinline__ float lds1(const __half* p, float off) { return add_offset(__half2float(*p), off); }
};

template <>
struct Codec<__nv_bfloat16> {
    static __device__ __forceinline__ float4 ld4(const __nv_bfloat16* p, float off)
    {
        const uint2 r = __ldg(reinterpret_cast<const uint2*>(p));
        const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&r.x));
        const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&r.y));
        return add_offset(make_float4(a.x, a.y, b.x, b.y), off);
    }
    static __device__ __forceinline__ float ld1(const __nv_bfloat16* p, float off)
    {
        return add_offset(__bfloat162float(__ldg(p)), off);
    }
    static __device__ __forceinline__ void st4(__nv_bfloat16* p, const float4& v, float off)
    {
        const __nv_bfloat162 a = __floats2bfloat162_rn(v.x - off, v.y - off);
        const __nv_bfloat162 b = __floats2bfloat162_rn(v.z - off, v.w - off);
        uint2 r;
        r.x = *reinterpret_cast<const unsigned*>(&a);
        r.y = *reinterpret_cast<const unsigned*>(&b);
        *reinterpret_cast<uint2*>(p) = r;
    }
    static __device__ __forceinline__ void st1(__nv_bfloat16* p, float v, float off)
    {
        *p = __float2bfloat16_rn(v - off);
    }
    static __device__ __forceinline__ float4 lds4(const __nv_bfloat16* p, float off)
    {
        const uint2 r = *reinterpret_cast<const uint2*>(p);
        const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&r.x));
        const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&r.y));
        return add_offset(make_float4(a.x, a.y, b.x, b.y), off);
    }
    static __device__ __forceinline__ float lds1(const __nv_bfloat16* p, float off)
    {
        return add_offset(__bfloat162float(*p), off);
    }
};

// Offset of plane p in 16-bit storage (0 for the fluid planes).
__device__ __forceinline__ float plane_offset(int p, float gref0, float gref1)
{
    return p < 9 ? 0.f : p == 9 ? gref0 : gref1;
}

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// A double-float value hi + lo (the unevaluated sum of two floats).  GB300
// issues FP64 arithmetic at a small fraction of its FP32 rate, and every warp
// of a step kernel reduces its diagnostics at the same moment, at the end of
// the kernel, so a reduction of doubles there leaves the SMs waiting on the
// FP64 pipe.  The step kernels' reductions add pairs of floats instead, with
// Knuth's error-free TwoSum on the high parts (about 44 significant bits),
// and form a double only for each block's final sum.
struct DF {
    float hi, lo;
};

__device__ __forceinline__ DF df_add(DF a, DF b)
{
    const float s = a.hi + b.hi;
    const float bv = s - a.hi;
    const float e = (a.hi - (s - bv)) + (b.hi - bv);  // s + e = a.hi + b.hi exactly
    const float lo = e + (a.lo + b.lo);
    const float hi = s + lo;
    return {hi, lo - (hi - s)};
}

__device__ __forceinline__ DF warp_sum(DF v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v = df_add(v, DF{__shfl_xor_sync(kFull, v.hi, o), __shfl_xor_sync(kFull, v.lo, o)});
    return v;
}

__device__ __forceinline__ double df_value(DF v) { return double(v.hi) + double(v.lo); }

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
// Per-lane asynchronous global -> shared copy of 16 bytes through L2
// (cp.async.cg, 16-byte aligned addresses); the lane waits for its copies
// with cp.async.wait_group, and the warp then syncs to see each other's.
__device__ __forceinline__ void cp_async16(void* dst, const void* src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
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

// Grid-wide barrier of a cooperative launch (every block resident): thread 0
// of each block adds one to *count and waits until it reaches target.  The
// wait is bounded like the mbarrier waits (kWaitCycles, about a second); a
// block that gives up, or sees that another one did (bit 1 of the error
// word), sets that bit and returns false, and the kernel stops.  The fences
// around the count make each block's writes before the barrier visible to
// every block after it.
__device__ __forceinline__ bool grid_barrier(unsigned* count, unsigned target, unsigned* err)
{
    __shared__ int go;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        __threadfence();
        atomicAdd(count, 1u);
        const long long t0 = clock64();
        for (;;) {
            unsigned c, e;
            asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(c) : "l"(count) : "memory");
            if (c >= target) break;
            asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(e) : "l"(err) : "memory");
            if ((e & 2u) || clock64() - t0 > kWaitCycles) {
                atomicOr(err, 2u);
                ok = 0;
                break;
            }
            __nanosleep(100);
        }
        __threadfence();
        go = ok;
    }
    __syncthreads();
    return go != 0;
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
    __device__ __forceinline__ DF pair() const { return DF{s, -e}; }
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
// kWalls: the fluid planes take the paper's wall values that
// launch_wall_values left in plane i - 1 of Wb instead (the scalar keeps
// bounce-back).
template <typename T, bool kWalls = false>
__device__ __forceinline__ void bounce_back(float4 (&v)[kPlanes], unsigned lk, const T* S, long long P,
                                            long long oC, const T* Wb = nullptr)
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
            const T* src = S + opp(i) * P;  // the node's own opposite population
            if constexpr (kWalls) src = Wb + (i - 1) * P;
            const float4 own = Codec<T>::ld4(src + oC, 0.f);
            const float4 ownc = i <= 4 ? Codec<T>::ld4(S + (9 + opp(i)) * P + oC, 0.f) : own;
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

// Completion of an open port node (fluid populations as deviations
// f_i - w_i).  west: the port receives from -x, so the populations with
// e_x = +1 are unknown (s = +1); otherwise e_x = -1 (s = -1).  The port kind
// (bits 8..15 of chan_kind):
//   0 velocity  Zou-He with u = (u_x, 0); the scalar's unknown population
//               makes the node's concentration C_in.
//   1 pressure  Zou-He with the prescribed density and zero tangential
//               velocity; the scalar's unknown population keeps its own
//               post-collision value of the previous step (do-nothing).
//   2, 3        the paper's port (section "Boundary Conditions"): the
//               unknown f keep their own post-collision values, then all
//               nine are scaled by gamma = rho_port / rho, which leaves u as
//               it is.  Kind 2 (outlet): do-nothing for the scalar.  Kind 3
//               (inlet): do-nothing for the unknown g, then all five scaled to
//               C_in; a node without compound takes g_eq(C_in, u) instead.
// Post-collision values of the previous step are read from the source
// buffer at index own.  Returns true for an outlet node (kinds 1, 2).
struct PortNode {
    float f[9];
    float g[5];
};

// Kinds 2 and 3 of complete_port, kept out of line: they are rare, and
// inlined into every node of the step kernels' unrolled loops they would
// crowd the instruction cache of the hot path.
template <typename T>
__device__ __noinline__ bool rescaling_port(PortNode& n, bool west, const RowBC& b, const T* S, long long P,
                                            long long own, float gref1, float wg1, float inv_cs2g)
{
    float* f = n.f;
    float* g = n.g;
    const int kind = (b.chan_kind >> 8) & 0xFF;
    if (west) {
        f[1] = Codec<T>::ld1(S + 1 * P + own, 0.f);
        f[5] = Codec<T>::ld1(S + 5 * P + own, 0.f);
        f[8] = Codec<T>::ld1(S + 8 * P + own, 0.f);
    } else {
        f[3] = Codec<T>::ld1(S + 3 * P + own, 0.f);
        f[6] = Codec<T>::ld1(S + 6 * P + own, 0.f);
        f[7] = Codec<T>::ld1(S + 7 * P + own, 0.f);
    }
    const float rd = ((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7])) + f[8];
    // gamma - 1 = (rho_port - rho) / rho; f_i' <- f_i' + (gamma - 1) (w_i + f_i')
    const float gm1 = (b.a - rd) / (1.f + rd);
    for (int i = 0; i < 9; ++i) f[i] += gm1 * ((i == 0 ? kWr : i <= 4 ? kWa : kWd) + f[i]);
    // do-nothing for the scalar's unknown population
    if (west) g[1] = Codec<T>::ld1(S + 10 * P + own, gref1);
    else g[3] = Codec<T>::ld1(S + 12 * P + own, gref1);
    if (kind != 3) return true;
    const float Cs = ((g[0] + g[1]) + (g[2] + g[3])) + g[4];
    if (Cs > 0.f) {
        const float gc = b.c / Cs;
        for (int i = 0; i < 5; ++i) g[i] *= gc;
    } else {
        const float rho = 1.f + (((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7])) + f[8]);
        const float ux = ((f[1] - f[3]) + (f[5] - f[6]) + (f[8] - f[7])) / rho;
        const float uy = ((f[2] - f[4]) + (f[5] + f[6]) - (f[7] + f[8])) / rho;
        const float c1 = wg1 * b.c, cx = c1 * inv_cs2g * ux, cy = c1 * inv_cs2g * uy;
        g[0] = b.c - 4.f * c1;
        g[1] = c1 + cx;
        g[3] = c1 - cx;
        g[2] = c1 + cy;
        g[4] = c1 - cy;
    }
    return false;
}

// Lattice direction components (Eq. lattice).
__device__ __forceinline__ constexpr int dir_x(int i)
{
    return (i == 1 || i == 5 || i == 8) ? 1 : (i == 3 || i == 6 || i == 7) ? -1 : 0;
}
__device__ __forceinline__ constexpr int dir_y(int i)
{
    return (i == 2 || i == 5 || i == 6) ? 1 : (i == 4 || i == 7 || i == 8) ? -1 : 0;
}

// rho - 1 and the momentum of the stored populations (deviations) of one node.
template <typename T>
__device__ __forceinline__ void node_moments(const T* S, long long P, long long o, float& rd, float& jx, float& jy)
{
    float f[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) f[i] = Codec<T>::ld1(S + i * P + o, 0.f);
    rd = ((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7])) + f[8];
    jx = (f[1] - f[3]) + (f[5] - f[6]) + (f[8] - f[7]);
    jy = (f[2] - f[4]) + (f[5] + f[6]) - (f[7] + f[8]);
}

// The paper's wall ("Boundary Conditions") for population i of the fluid
// node at offset own, whose source x - e_i is not fluid (lb: the node's
// wall-link byte, bit j-1 set = the source x - e_j is not fluid): the
// equilibrium, as a deviation f_eq - w_i, of a density extrapolated to first
// order from the fluid along e_i, 2 rho(x + e_i) - rho(x + 2 e_i), and the
// momentum interpolated between zero at the wall, half a link behind the
// node, and x + e_i, one and a half links from it: j(x + e_i) / 3.  Moments
// of the stored state S (the start of the step).  Where x + 2 e_i is not
// fluid the density is that of x + e_i; where x + e_i is not fluid either,
// the node's own density with zero momentum.
template <typename T>
__device__ __forceinline__ float equilibrium_wall(int i, unsigned lb, const T* S, const uint8_t* links, long long P,
                                                  long long own, int pitch)
{
    const int back = opp(i) - 1;  // bit of "x + e_i is not fluid"
    float rd, jx = 0.f, jy = 0.f;
    if (!((lb >> back) & 1u)) {
        const long long o1 = own + dir_x(i) + (long long)dir_y(i) * pitch;
        float r1, x1, y1;
        node_moments(S, P, o1, r1, x1, y1);
        if (!((links[o1] >> back) & 1u)) {
            float r2, x2, y2;
            node_moments(S, P, o1 + dir_x(i) + (long long)dir_y(i) * pitch, r2, x2, y2);
            rd = 2.f * r1 - r2;  // 2 rho1 - rho2 - 1
        } else {
            rd = r1;
        }
        jx = x1 * (1.f / 3.f);
        jy = y1 * (1.f / 3.f);
    } else {
        float ox, oy;
        node_moments(S, P, own, rd, ox, oy);
    }
    const float rho = 1.f + rd;
    const float ux = jx / rho, uy = jy / rho;
    const float eu = float(dir_x(i)) * ux + float(dir_y(i)) * uy;
    const float w = i <= 4 ? kWa : kWd;
    return w * (rd + rho * (3.f * eu + 4.5f * eu * eu - 1.5f * (ux * ux + uy * uy)));
}

template <typename T>
__device__ __forceinline__ bool complete_port(float (&f)[9], float (&g)[5], bool west, const RowBC& b,
                                              const T* S, long long P, long long own, float gref1 = 0.f,
                                              float wg1 = 0.f, float inv_cs2g = 0.f)
{
    const int kind = (b.chan_kind >> 8) & 0xFF;
    if (kind >= 2) {
        PortNode n;
#pragma unroll
        for (int i = 0; i < 9; ++i) n.f[i] = f[i];
#pragma unroll
        for (int i = 0; i < 5; ++i) n.g[i] = g[i];
        const bool outlet = rescaling_port(n, west, b, S, P, own, gref1, wg1, inv_cs2g);
#pragma unroll
        for (int i = 0; i < 9; ++i) f[i] = n.f[i];
#pragma unroll
        for (int i = 0; i < 5; ++i) g[i] = n.g[i];
        return outlet;
    }
    {
        const float s = west ? 1.f : -1.f;
        // populations leaving through the port: e = (-s, 0), (-s, -1), (-s, +1)
        const float fo_ax = west ? f[3] : f[1];
        const float fo_dn = west ? f[7] : f[8];
        const float fo_up = west ? f[6] : f[5];
        // rho (1 - s u_x) = f0 + f2 + f4 + 2 (leaving) = 1 + Kd in deviations
        // (the weights of those populations add up to one)
        const float Kd = f[0] + f[2] + f[4] + 2.f * (fo_ax + fo_dn + fo_up);
        float jx;  // rho u_x of the node
        if (kind == 0) jx = (1.f + Kd) * b.a / (1.f - s * b.a);
        else jx = s * (b.a - Kd);  // b.a = prescribed rho - 1
        const float ht = 0.5f * (f[2] - f[4]);
        const float fi_ax = fo_ax + s * (2.f / 3.f) * jx;
        const float fi_up = fo_dn - ht + s * (1.f / 6.f) * jx;  // e = (s, +1)
        const float fi_dn = fo_up + ht + s * (1.f / 6.f) * jx;  // e = (s, -1)
        if (west) {
            f[1] = fi_ax;
            f[5] = fi_up;
            f[8] = fi_dn;
        } else {
            f[3] = fi_ax;
            f[6] = fi_up;
            f[7] = fi_dn;
        }
    }
    if (kind == 0) {
        if (west) g[1] = b.c - (g[0] + g[2] + g[3] + g[4]);
        else g[3] = b.c - (g[0] + g[1] + g[2] + g[4]);
        return false;
    }
    // do-nothing: the node keeps its own post-collision value
    if (west) g[1] = Codec<T>::ld1(S + 10 * P + own, gref1);
    else g[3] = Codec<T>::ld1(S + 12 * P + own, gref1);
    return true;
}

// Free flight (pull) of one lane's four nodes x0..x0+3 with 128-bit loads:
// v[p] component k = plane p at (x0 + k) - e_i.  The +-1 column shifts move
// between lanes by shuffle; lane 0 / lane 31 load the one value that comes
// from the neighbouring segment.  act: this lane holds fluid; ld_w / ld_e:
// this lane's edge value feeds a fluid neighbour lane.  reverse: pull from
// (x0 + k) + e_i instead (the transposed free flight of the adjoint).
// kP0, kN: the planes kP0 .. kP0 + kN - 1 only (S then points at plane kP0,
// v[j] holds plane kP0 + j).
template <bool kReverse, typename T, int kP0 = 0, int kN = kPlanes>
__device__ __forceinline__ void pull_quad(float4 (&v)[kN], const T* __restrict__ S, long long P,
                                          long long oC, long long oS, long long oN, int halo_w, int halo_e,
                                          bool act, bool ld_w, bool ld_e, int lane)
{
#pragma unroll
    for (int j = 0; j < kN; ++j) {
        const int p = kP0 + j;
        const int sr = kReverse ? (src_row(p) == 0 ? 0 : 3 - src_row(p)) : src_row(p);
        const int sc = kReverse ? (src_col(p) == 0 ? 0 : 3 - src_col(p)) : src_col(p);
        const long long o = j * P + (sr == 0 ? oC : sr == 1 ? oS : oN);
        const bool ld = sc == 0 ? act : sc == 1 ? ld_w : ld_e;
        float4 r = ld ? Codec<T>::ld4(S + o, 0.f) : make_float4(0.f, 0.f, 0.f, 0.f);
        if (sc == 1) {  // from column x - 1
            float h = 0.f;
            if (act && lane == 0) h = Codec<T>::ld1(S + o + halo_w, 0.f);
            float w = __shfl_up_sync(kFull, r.w, 1);
            if (lane == 0) w = h;
            r = make_float4(w, r.x, r.y, r.z);
        } else if (sc == 2) {  // from column x + 1
            float h = 0.f;
            if (act && lane == 31) h = Codec<T>::ld1(S + o + halo_e, 0.f);
            float e = __shfl_down_sync(kFull, r.x, 1);
            if (lane == 31) e = h;
            r = make_float4(r.y, r.z, r.w, e);
        }
        v[j] = r;
    }
}

// Which lanes of a warp tile load plane values, from the tile's table entry
// alone: own = the lane lies in the quad range [q0, q1] that holds the
// tile's fluid; west / east = its edge value feeds a lane of that range
// through the x - 1 / x + 1 shift.  Every lane holding fluid is in the
// range, so the loads can go out before the lane's wall-link word arrives.
struct LoadRange {
    bool own, west, east;
};
__device__ __forceinline__ LoadRange load_range(uint2 tile, int lane)
{
    const int q0 = int(tile.y & 0xFFu), q1 = int((tile.y >> 8) & 0xFFu);
    return LoadRange{lane >= q0 && lane <= q1, lane >= q0 - 1 && lane <= q1, lane >= q0 && lane <= q1 + 1};
}

// A warp's share of a tile table: entries t, t + stride, ... below n of
// tiles.
struct TileRange {
    const uint2* tiles;
    int n, t, stride;
};

// Tile tables list the tiles whose row segment holds no port node first
// (n_plain of them) and the port tiles (kPortTile) after them.  The grid's
// last port_blocks blocks take the port tiles and run them with the port
// code (port_loop), the other blocks the rest with a loop without any.
// port_blocks = 0 with port tiles present sends every block through the
// port loop over every tile; n_plain = 0 (nothing known about the tiles)
// does the same.
__device__ __forceinline__ TileRange split_tiles(const uint2* tiles, int n_tiles, int n_plain, int port_blocks,
                                                 int warp, int wpb, bool& port_loop)
{
    const int gp = port_blocks;
    const int n_port = n_tiles - n_plain;
    const int first_port_block = int(gridDim.x) - gp;
    if (n_port > 0 && (gp == 0 || int(blockIdx.x) >= first_port_block)) {
        port_loop = true;
        if (gp == 0) return TileRange{tiles, n_tiles, int(blockIdx.x) * wpb + warp, int(gridDim.x) * wpb};
        return TileRange{tiles + n_plain, n_port, (int(blockIdx.x) - first_port_block) * wpb + warp, gp * wpb};
    }
    port_loop = false;
    return TileRange{tiles, n_plain, int(blockIdx.x) * wpb + warp, first_port_block * wpb};
}

// Open ports, moments and both collisions for the four nodes x0..x0+3 of a
// row whose port entries are bw (west) and be (east); v holds the streamed
// populations on entry and the post-collision populations on exit (fluid
// planes as deviations f_i - w_i).
// Valve bit of the channel in a port entry's chan_kind (channel in the low
// byte), selected without indexing the parameter array.
__device__ __forceinline__ bool valve_open(const StepArgs& a, int chan_kind)
{
    const int ch = chan_kind & 0xFF;
    if (ch < 32) return (a.open_mask[0] >> ch) & 1u;  // a single chip's channels
    uint32_t w = a.open_mask[0];
#pragma unroll
    for (int j = 1; j < kMaskWords; ++j)
        if ((ch >> 5) == j) w = a.open_mask[j];
    return (w >> (ch & 31)) & 1u;
}

// Relaxation rates {1 / tau_f, 1 / tau_g} of a row.
__device__ __forceinline__ float2 row_rates(const StepArgs& a, int y)
{
    if (a.rates == nullptr) return make_float2(a.omega_f, a.omega_g);
    const float4 r = __ldg(a.rates + y);
    return make_float2(r.x, r.y);
}

// Port completion of node k of the quad (the port rules work on g_i itself,
// so 16-bit deviations are shifted to g_i around them).  Returns true for an
// outlet node.
template <typename T>
__device__ __forceinline__ bool port_node(float (&f)[9], float (&g)[5], bool west, const RowBC& b,
                                          const StepArgs& a, const T* S, long long own)
{
    constexpr bool kDev = !kStoresF32<T>;
    if constexpr (kDev) {
        g[0] += a.gref0;
#pragma unroll
        for (int i = 1; i < 5; ++i) g[i] += a.gref1;
    }
    const bool outlet = complete_port(f, g, west, b, S, a.plane, own, a.gref1, a.wg1, a.inv_cs2g);
    if constexpr (kDev) {
        g[0] -= a.gref0;
#pragma unroll
        for (int i = 1; i < 5; ++i) g[i] -= a.gref1;
    }
    return outlet;
}

// Moments (Eq. moments) and both BGK collisions of one node, in place: f as
// deviations f_i - w_i from the rest state, g as stored (FP32: g_i; kDev:
// g_i - w_i C_ref).  omega = {1 / tau_f, 1 / tau_g}; dfac = 1 - k / omega_g
// with decay rate k (1 without decay).  Returns the moments the diagnostics
// need.
//
// Two evaluations of the same update, chosen by storage type so that every
// kernel of one storage type gives the same bits.  FP32 storage (kernels
// bound by memory latency at their 128-register limit) keeps the direct
// form f_i + omega (f_eq_i - f_i), which holds the fewest constants.  The
// 16-bit kernels are bound by instruction issue and take the factored form
// (1 - omega) f_i + omega f_eq_i with the equilibrium built from shared
// terms: about a third fewer FP32 instructions per node.
struct NodeMoments {
    float rd, rho, jx, ux, C;
};

template <bool kDev>
__device__ __forceinline__ NodeMoments collide_node(float (&f)[9], float (&g)[5], float2 omega, float dfac,
                                                    const StepArgs& a)
{
    if constexpr (kDev) {
        // ---- moments of the deviations f'_i = f_i - w_i:
        //      rho = 1 + sum f'_i, j = sum e_i f'_i ----
        const float s56 = f[5] + f[6], s78 = f[7] + f[8];
        const float rd = ((f[0] + (f[1] + f[3])) + (f[2] + f[4])) + (s56 + s78);
        const float rho = 1.f + rd;
        const float jx = (f[1] - f[3]) + (f[5] - f[6]) + (f[8] - f[7]);
        const float jy = (f[2] - f[4]) + (s56 - s78);
        const float inv = __fdividef(1.f, rho);  // fast reciprocal (2 ulp): rho stays near 1
        const float ux = jx * inv, uy = jy * inv;
        // ---- BGK collision of f.  With j = rho u the equilibrium deviation
        //      is f_eq_i - w_i = w_i [B + 3 e_i.j + 9/2 (e_i.j)(e_i.u)],
        //      B = rho - 1 - 3/2 rho u^2 = (rho - 1) - 3/2 j.u; directions
        //      +-e share B + 9/2 (e.j)(e.u) and differ in the sign of 3 e.j.
        //      The weights are 4/9, 1/9 and 1/36, so omega w_rest = 4 wa and
        //      omega w_diag = wa / 4 with wa = omega w_axis, exactly (a power
        //      of two commutes with rounding): the diagonal terms are formed
        //      a quarter of the size and share wa ----
        {
            const float om = 1.f - omega.x, wa = omega.x * kWa;
            const float p1 = jx * ux, p2 = jy * uy;
            const float B = fmaf(-1.5f, p1 + p2, rd);
            const float j5 = jx + jy, j6 = jy - jx;  // e.j along (1, 1) and (-1, 1)
            const float y1 = fmaf(4.5f, p1, B), y2 = fmaf(4.5f, p2, B);
            const float Bq = 0.25f * B;
            const float y5 = fmaf(1.125f * j5, ux + uy, Bq), y6 = fmaf(1.125f * j6, uy - ux, Bq);
            f[0] = fmaf(wa, 4.f * B, om * f[0]);
            f[1] = fmaf(wa, fmaf(3.f, jx, y1), om * f[1]);
            f[3] = fmaf(wa, fmaf(-3.f, jx, y1), om * f[3]);
            f[2] = fmaf(wa, fmaf(3.f, jy, y2), om * f[2]);
            f[4] = fmaf(wa, fmaf(-3.f, jy, y2), om * f[4]);
            f[5] = fmaf(wa, fmaf(0.75f, j5, y5), om * f[5]);
            f[7] = fmaf(wa, fmaf(-0.75f, j5, y5), om * f[7]);
            f[6] = fmaf(wa, fmaf(0.75f, j6, y6), om * f[6]);
            f[8] = fmaf(wa, fmaf(-0.75f, j6, y6), om * f[8]);
        }
        // ---- scalar: C = sum g + C_ref (the weights add up to one) ----
        const float C = (((g[0] + g[1]) + (g[2] + g[3])) + g[4]) + kCRef;
        {
            // omega_g (g_eq_i - w_i C_ref) = w_i wC + omega_g w_i C e_i.u / c_s^2,
            // wC = omega_g (C dfac - C_ref): the reaction term R = -k C of
            // Eq. cde enters as w_i R = omega_g (w_i R / omega_g), the
            // isotropic part scaled by dfac = 1 - k / omega_g
            const float wg = omega.y, om = 1.f - wg;
            const float wC = fmaf(C, wg * dfac, -(wg * kCRef));
            const float w1C = a.wg1 * wC;
            const float ck = ((wg * a.wg1) * a.inv_cs2g) * C;
            const float cx = ck * ux, cy = ck * uy;
            // rest direction as the remainder wC - 4 w_1 wC (float(w0) + 4 float(w1) != 1)
            g[0] = fmaf(om, g[0], fmaf(-4.f, w1C, wC));
            g[1] = fmaf(om, g[1], w1C + cx);
            g[3] = fmaf(om, g[3], w1C - cx);
            g[2] = fmaf(om, g[2], w1C + cy);
            g[4] = fmaf(om, g[4], w1C - cy);
        }
        return NodeMoments{rd, rho, jx, ux, C};
    } else {
        // ---- moments (Eq. moments) and BGK collision of f, in deviations
        //      from the rest state: f'_i = f_i - w_i, rho = 1 + sum f'_i ----
        const float rd = ((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7])) + f[8];
        const float rho = 1.f + rd;
        const float jx = (f[1] - f[3]) + (f[5] - f[6]) + (f[8] - f[7]);
        const float jy = (f[2] - f[4]) + (f[5] + f[6]) - (f[7] + f[8]);
        const float inv = __fdividef(1.f, rho);  // fast reciprocal (2 ulp): rho stays near 1
        const float ux = jx * inv, uy = jy * inv;
        const float usq = 1.5f * (ux * ux + uy * uy);
        const float wo = omega.x;
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
            const float wg = omega.y;
            // the reaction term R = -k C of Eq. cde enters as w_i R, which is
            // omega (w_i R / omega): the equilibrium's isotropic part scaled by
            // dfac = 1 - k / omega (exactly 1 without decay)
            const float Cd = C * dfac;
            const float c1 = a.wg1 * C, cx = c1 * a.inv_cs2g * ux, cy = c1 * a.inv_cs2g * uy;
            const float c1d = a.wg1 * Cd;
            // rest equilibrium w0 C formed as the remainder, so that the five
            // equilibria add up to C exactly (float(w0) + 4 float(w1) != 1)
            g[0] += wg * ((Cd - 4.f * c1d) - g[0]);
            g[1] += wg * ((c1d + cx) - g[1]);
            g[3] += wg * ((c1d - cx) - g[3]);
            g[2] += wg * ((c1d + cy) - g[2]);
            g[4] += wg * ((c1d - cy) - g[4]);
        }
        return NodeMoments{rd, rho, jx, ux, C};
    }
}

// Open ports, moments and both collisions of the quad.  Where the rare work
// goes depends on the storage type, by measurement: the FP32 kernel waits on
// its loads and is fastest with the port and solid-node handling inside the
// per-node loop (63.7 us per step on the 4096 x 2048 chip, against 64.9 us
// with passes); the 16-bit kernels are bound by instruction issue and are
// fastest with that work in passes over the quad that only quads holding a
// port or a solid node enter (FP16 50.1 us, against 52.3 us inside the loop).
// kPasses selects the passes (the multi-step kernel takes them for FP32 too:
// there they keep its registers from spilling).  Both forms give the same
// bits.  kPorts = false leaves the port code out, for tiles whose row
// segment holds no port node (kPortTile): present in the node loop, it costs
// the step even where it never runs (a timing copy without it: FP16 44.1 us
// against 48.0 us on the 4096 x 2048 chip).  The register kernels take the
// port-free form for those tiles and the pass form for the few others.
template <typename T, bool kPasses = !kStoresF32<T>, bool kPorts = true>
__device__ __forceinline__ void collide_quad(float4 (&v)[kPlanes], unsigned lk, int x0, const RowBC& bw,
                                             const RowBC& be, const StepArgs& a, const T* S, long long oC,
                                             float2 omega, QuadAcc& acc)
{
    // a port entry exists on a few rows only (the entries are the same for
    // the whole warp, so the tests below branch uniformly)
    bool open_w = false, open_e = false;
    if constexpr (kPorts) {
        if (bw.x >= 0) open_w = valve_open(a, bw.chan_kind);
        if (be.x >= 0) open_e = valve_open(a, be.chan_kind);
    }
    const float dfac = a.decay != 0.f ? 1.f - a.decay / omega.y : 1.f;
    // With 16-bit storage the scalar populations stay in their stored form
    // g_i - w_i C_ref here (C_ref = kCRef), as the fluid ones stay f_i - w_i:
    // the collision below is written for deviations, so no offset is added
    // on loading or subtracted on storing.  FP32 storage holds g_i itself.
    constexpr bool kDev = !kStoresF32<T>;

    unsigned outlet = 0;  // passes: bit k = node x0 + k is an open outlet (flux diagnostics)
    if constexpr (kPasses && kPorts) {
        // ---- open valve ports (Zou-He; held concentration / do-nothing):
        //      only the first and last quads of a channel row hold a port
        //      node (ports are fluid, and never on both sides of a row) ----
        const int kw = open_w ? bw.x - x0 : -1;
        const int ke = open_e ? be.x - x0 : -1;
        if (unsigned(kw) < 4u || unsigned(ke) < 4u) {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const bool pw = k == kw;
                if (!pw && k != ke) continue;
                float f[9], g[5];
#pragma unroll
                for (int i = 0; i < 9; ++i) f[i] = at(v[i], k);
#pragma unroll
                for (int i = 0; i < 5; ++i) g[i] = at(v[9 + i], k);
                if (port_node(f, g, pw, pw ? bw : be, a, S, oC + k)) outlet |= 1u << k;
#pragma unroll
                for (int i = 0; i < 9; ++i) at(v[i], k) = f[i];
#pragma unroll
                for (int i = 0; i < 5; ++i) at(v[9 + i], k) = g[i];
            }
        }
    }

    float rmin = 1.f;  // smallest density of the quad's fluid nodes (passes)
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const unsigned lb = (lk >> (8 * k)) & 0xFFu;
        const bool fluid = lb != kSolid;
        float f[9], g[5];
#pragma unroll
        for (int i = 0; i < 9; ++i) f[i] = at(v[i], k);
#pragma unroll
        for (int i = 0; i < 5; ++i) g[i] = at(v[9 + i], k);
        bool outlet_k = (outlet >> k) & 1u;
        if constexpr (!kPasses) {
            if (!fluid) {  // solid node: park it at the rest state rho = 1, C = 0
#pragma unroll
                for (int i = 0; i < 9; ++i) f[i] = 0.f;
#pragma unroll
                for (int i = 0; i < 5; ++i) g[i] = 0.f;
            }
            // ---- open valve ports ----
            if constexpr (kPorts) {
                const int xk = x0 + k;
                const bool pw = open_w && bw.x == xk;
                const bool pe = !pw && open_e && be.x == xk;
                if (pw || pe) outlet_k = port_node(f, g, pw, pw ? bw : be, a, S, oC + k);
            }
        }

        const NodeMoments nm = collide_node<kDev>(f, g, omega, dfac, a);
        const float rd = nm.rd, rho = nm.rho, jx = nm.jx, ux = nm.ux, C = nm.C;
#pragma unroll
        for (int i = 0; i < 9; ++i) at(v[i], k) = f[i];
#pragma unroll
        for (int i = 0; i < 5; ++i) at(v[9 + i], k) = g[i];

        if (fluid) {
            if constexpr (kPasses) {
                rmin = fminf(rmin, rho);
            } else {
                acc.bad |= !(rho > 0.f && rho < INFINITY) || !(fabsf(C) < INFINITY);
                ++acc.n;
            }
            acc.m += rd;
            acc.c += C;
            if (outlet_k) {
                acc.q += jx;  // rho u_x
                acc.qc += C * ux;
            }
        }
    }

    if constexpr (kPasses) {
        // a non-finite density or concentration makes its quad sum non-finite
        acc.bad = !(rmin > 0.f) || !(fabsf(acc.m) < INFINITY) || !(fabsf(acc.c) < INFINITY);
        // ---- solid nodes: parked at the rest state rho = 1, C = 0 (what
        //      they computed above from their pulled values is dropped) ----
        const unsigned sb = ~lk;  // a zero byte marks a solid node
        // the top bit of each byte of sb that is zero (no carry between bytes)
        const unsigned solid = ~(((sb & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | sb) & 0x80808080u;
        acc.n = 4 - __popc(solid);
        if (solid) {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                if (((lk >> (8 * k)) & 0xFFu) != kSolid) continue;
#pragma unroll
                for (int i = 0; i < 9; ++i) at(v[i], k) = 0.f;
                at(v[9], k) = kDev ? -a.gref0 : 0.f;
#pragma unroll
                for (int i = 10; i < 14; ++i) at(v[i], k) = kDev ? -a.gref1 : 0.f;
            }
        }
    }
}

// Totals of the four diagnostics from the partials of n blocks (4
// double-float pairs each), in one fixed order whatever block runs it: the
// block's first kFoldThreads threads, thread i taking blocks i + kFoldThreads
// j for j = 0, 1, ... in rounds of eight (one round for grids of up to 1024
// blocks), the eight of a round added as a pairwise tree (absent blocks count
// as zero) and the rounds in turn; then the lanes of each warp by shuffles,
// then the four warps pairwise; one double per diagnostic written.  Every
// addition is a double-float one on the FP32 pipes, and the loads are one
// round: it is the tail of the step that forms its own totals, and GB300
// issues FP64 arithmetic at a small fraction of its FP32 rate.  Partials
// written by other blocks of a running grid are read through L2
// (ld.global.cg).  Every thread of the block calls this (it has a barrier);
// the block has at least kFoldThreads threads.
__device__ __forceinline__ DF df_tree8(const DF (&x)[8])
{
    return df_add(df_add(df_add(x[0], x[1]), df_add(x[2], x[3])), df_add(df_add(x[4], x[5]), df_add(x[6], x[7])));
}

__device__ __forceinline__ void finish_partials(const float2* partials, int n, double* out)
{
    static_assert(kFoldThreads == 128, "the final combination below adds four warps' sums");
    __shared__ DF red[kFoldThreads / 32][4];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x < kFoldThreads) {
        DF t[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) t[q] = DF{0.f, 0.f};
        constexpr int kRound = 8;
        for (int b0 = threadIdx.x; b0 < n; b0 += kRound * kFoldThreads) {
            float4 v[kRound][2];  // diagnostics 0, 1 and 2, 3 of a block, (hi, lo) each
#pragma unroll
            for (int j = 0; j < kRound; ++j) {
                const int b = b0 + kFoldThreads * j;
                if (b < n) {
                    v[j][0] = __ldcg(reinterpret_cast<const float4*>(partials + 4 * b));
                    v[j][1] = __ldcg(reinterpret_cast<const float4*>(partials + 4 * b + 2));
                } else {
                    v[j][0] = make_float4(0.f, 0.f, 0.f, 0.f);
                    v[j][1] = make_float4(0.f, 0.f, 0.f, 0.f);
                }
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                DF x[kRound];
#pragma unroll
                for (int j = 0; j < kRound; ++j) {
                    const float4& w = v[j][q >> 1];
                    x[j] = (q & 1) ? DF{w.z, w.w} : DF{w.x, w.y};
                }
                t[q] = df_add(t[q], df_tree8(x));
            }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) t[q] = warp_sum(t[q]);
        if (lane == 0)
#pragma unroll
            for (int q = 0; q < 4; ++q) red[warp][q] = t[q];
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        const int q = threadIdx.x;
        out[q] = df_value(df_add(df_add(red[0][q], red[1][q]), df_add(red[2][q], red[3][q])));
    }
}

// The totals of a step formed inside it: the last block to finish adds up
// every block's partials (threadfence reduction: the partials are made
// visible before the ticket is taken, and the block that draws the last
// ticket reads them all after it).  Out of line, so that the step kernels
// carry no more than a call when it is not asked for.
__device__ __noinline__ void fold_totals(const float2* partials, unsigned* ticket, double* out)
{
    __shared__ bool last;
    if (threadIdx.x < 4) __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    finish_partials(partials, gridDim.x, out);
    if (threadIdx.x == 0) *ticket = 0u;  // every block of this step has taken its ticket
}

// The block's partial sums of the four diagnostics: lanes and warps combined
// as double-float pairs, the fluid node count as an integer (added to the
// first as an exact pair), and one double-float pair per diagnostic written.
// Null partials: a step whose diagnostics nothing reads (the forward steps
// inside the adjoint but the last) forms none.  The cross-block total is
// formed on demand by diag_finish, or, in the kernels instantiated with
// kFold, by the step's last block when a.diag_out is set.  Only those
// kernels carry the call: its mere presence made the BF16 kernels' steps
// 0.8-1.5 us longer.
template <bool kFold = false>
__device__ __forceinline__ void block_partials(const StepArgs& a, const LaneDiag& d)
{
    if (a.partials == nullptr) return;  // uniform over the grid
    __shared__ DF red[32][4];
    __shared__ int red_n[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    const DF s0 = warp_sum(d.m.pair()), s1 = warp_sum(d.c.pair());
    DF s2{0.f, 0.f}, s3{0.f, 0.f};
    if (__any_sync(kFull, (d.q.s != 0.f || d.q.e != 0.f) || (d.qc.s != 0.f || d.qc.e != 0.f))) {  // outlet lanes
        s2 = warp_sum(d.q.pair());
        s3 = warp_sum(d.qc.pair());
    }
    const int n = __reduce_add_sync(kFull, d.n);
    if (lane == 0) {
        red[warp][0] = s0;
        red[warp][1] = s1;
        red[warp][2] = s2;
        red[warp][3] = s3;
        red_n[warp] = n;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        DF s = red[0][threadIdx.x];
        int nb = red_n[0];
        for (int w = 1; w < wpb; ++w) {
            s = df_add(s, red[w][threadIdx.x]);
            nb += red_n[w];
        }
        if (threadIdx.x == 0) {
            const float hi = float(nb);  // nb = hi + lo exactly (|lo| <= 64 for any int)
            s = df_add(DF{hi, float(static_cast<long long>(nb) - static_cast<long long>(hi))}, s);
        }
        a.partials[blockIdx.x * 4 + threadIdx.x] = make_float2(s.hi, s.lo);
    }
    if constexpr (kFold) {
        if (a.diag_out != nullptr) fold_totals(a.partials, a.diag_ticket, a.diag_out);
    }
}

}  // namespace
}  // namespace lbm
