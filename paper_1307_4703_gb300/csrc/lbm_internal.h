// lbm_internal.h -- device data layout and kernel launchers shared by the
// host ABI (lbm_api.cu) and the kernels (lbm_kernels.cu).
//
// Layout in device memory (one chip):
//   populations  two buffers (ping-pong), each kPlanes planes of ny rows of
//                `pitch` floats: planes 0..8 hold f_0..f_8, planes 9..13 hold
//                g_0..g_4.  pitch is a multiple of kTileNodes, so every row
//                starts on a 512-byte boundary and a warp tile never leaves
//                its row.  The stored values are POST-collision populations;
//                the fluid planes hold the deviation f_i - w_i from the rest
//                state rho = 1 (the bits of an FP32 word then resolve the
//                small pressure differences that drive the flow), the
//                scalar planes hold g_i itself.
//   links        ny*pitch bytes: bit (i-1) set when the pull source x - e_i
//                of direction i = 1..8 is not a fluid node (solid, outside the
//                grid, or outside a port).  0xFF marks a solid node.
//   rowbc        2*ny entries (west side then east side): the port node of
//                that side and row, if any.
//   tiles        list of the 128-node warp tiles that hold fluid, disjoint:
//                x = (y << 15) | (first column / 16), y = first | (last << 8),
//                the first and last lane (4-node quad) holding fluid.
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

namespace lbm {

constexpr int kTileNodes = 128;  // nodes per warp tile: 32 lanes x 4 nodes
constexpr int kPlanes = 14;      // f_0..f_8, g_0..g_4
// A 128-node tile starts at its row's first fluid node not yet covered, on a
// kTileStart-node boundary (every staged copy stays 16-byte aligned), rather
// than at a 128-node segment boundary: x = (y << kColBits) | first column /
// kTileStart.  Tiles never overlap, so a lane's nodes are its tile's to
// update exactly when they are fluid.
constexpr int kColBits = 15;
constexpr int kTileStart = 16;
constexpr int kMaxRows = 1 << (32 - kColBits);                         // rows a tile entry can name
constexpr int kMaxCols = (1 << kColBits) * kTileStart - kTileNodes;    // columns, ditto
constexpr uint8_t kSolid = 0xFF;
constexpr int kRowFloats = kTileNodes + 8;  // staged plane row: 4-float halo on each side
constexpr int kBulkMaxThreads = 256;        // bulk variant: at most 7 consumer warps + 1 producer
constexpr int kMaxStages = 24;             // bulk variant: largest shared-memory ring
constexpr int kMaskWords = 8;              // valve channels per lattice: 32 * kMaskWords

enum StepVariant { kVariantRegs = 1, kVariantBulk = 2, kVariantPipe = 3, kVariantAsync = 4, kVariantPairs = 5 };
constexpr int kPairTileNodes = 64;  // nodes per warp tile of variant 5: 32 lanes x 2 nodes
// Bit of a tile table entry's .y: the tile's row segment holds a port node
// (of either side; whether its valve is open is decided per step).  Tiles
// without one run a step without any port code.
constexpr uint32_t kPortTile = 1u << 16;
constexpr int kSegBits64 = 13;      // 64-node tile encoding: segment in the low 13 bits
enum Precision { kFP32 = 0, kFP16 = 1, kBF16 = 2 };
constexpr float kCRef = 0.5f;  // reference concentration of 16-bit scalar storage
constexpr int kFoldThreads = 128;  // threads that add up the block partials of the diagnostics

struct StepLaunch {
    int variant;  // kVariantRegs, kVariantBulk, kVariantPipe, kVariantAsync or kVariantPairs
    int grid;
    int block;
    int stages;   // shared-memory stages per block (computing warps x stages per warp)
    int precision = kFP32;  // storage of the populations
    bool pdl = false;       // launch as a programmatic dependent of the previous kernel
    bool walls = false;     // the paper's walls (variants 1 and 2; see StepArgs::wallv)
};

struct RowBC {
    int32_t x;          // port node column, -1 = no port on this side and row
    int32_t chan_kind;  // valve channel | (kind << 8); kind 0 velocity, 1 pressure,
                        // 2 rescaling outlet, 3 rescaling inlet (the paper's ports)
    float a;            // velocity port: u_x; other kinds: rho - 1
    float c;            // kinds 0 and 3: the prescribed concentration
};

struct StepArgs {
    const float* src;       // post-collision populations at time t
    float* dst;             // post-collision populations at time t + 1
    const uint8_t* links;
    const RowBC* rowbc;
    const uint2* tiles;     // x = (y << 15) | first column / 16, y = first | (last << 8) lane (quad) holding
                            // fluid | kPortTile; the n_plain tiles without a port node come first
    int n_tiles;
    int n_plain;            // 0: every tile is treated as a port tile
    int port_blocks;        // variants 1, 4: the grid's last port_blocks blocks take the port tiles
                            // (launch_step sets it from the grid)
    const uint2* tiles64;   // the same lattice in 64-node row segments (variant 5):
                            // x = (y << 13) | segment, y = first | (last << 8) lane (node pair) holding fluid
    int n_tiles64;
    int reverse;            // 1: take the tiles from the end of the table (see tile_at)
    int ny;
    int pitch;
    long long plane;        // ny * pitch
    float omega_f;          // 1 / tau_f
    float omega_g;          // 1 / tau_g
    const float4* rates;    // per row {1 / tau_f, 1 / tau_g, 0, 0} (batches of chips), or null:
                            // omega_f and omega_g hold everywhere
    float wg0;              // scalar rest weight
    float wg1;              // scalar axis weight (1 - wg0) / 4
    float inv_cs2g;         // 1 / c_s^2 of the scalar lattice
    float decay;            // k of the reaction term R = -k C (0: none)
    const void* wallv;      // the paper's walls: 8 planes (population i in plane i - 1, storage type) of
                            // the wall values launch_wall_values computed for this step; null: halfway
                            // bounce-back
    uint32_t open_mask[kMaskWords];  // valve bits of this step: channel c is bit c % 32 of word c / 32
    float2* partials;       // 4 diagnostics partial sums per block, double-float pairs (hi, lo) (scratch);
                            // null: the step forms no diagnostics
    unsigned int* err;      // sticky error word: bit 0 numeric, bit 1 timeout
    float gref0, gref1;     // 16-bit storage: offsets w_0 C_ref and w_1 C_ref of the scalar planes
    unsigned barrier_extra; // multi-step kernel: arrivals its barriers wait for beyond the grid's
                            // (0; a test hook sets 1 so that the bounded wait runs out)
    double* diag_out;       // non-null: the step's last block to finish also forms the four
                            // totals of the partials and writes them here (device-addressable;
                            // the kernels of launch_step_fold)
    unsigned int* diag_ticket;  // blocks of the step that have written their partials (zero
                                // between steps: the last block resets it)
};

// One adjoint step (lbm_adjoint.cu): A(t) from A(t+1) and the state P(t).
struct AdjointArgs {
    const float* state;     // P(t), post-collision populations (fluid planes as deviations)
    const float* adj_next;  // A(t+1) = dJ/dP(t+1), same layout (first reverse step only)
    const float* mid_next;  // M(t+1), the adjoint of the completed pre-collision values of step t+1
    float* adj_mid;         // M(t), written
    const uint8_t* links;
    const RowBC* rowbc;
    const uint2* tiles;
    int n_tiles;
    int ny;
    int pitch;
    long long plane;
    float omega_f, omega_g, wg0, wg1, inv_cs2g;
    uint32_t open_mask;       // valve word of step t
    uint32_t open_mask_next;  // valve word of step t+1
    int reverse;              // take the tile table from its end (alternates from launch to launch)
    float* dn;              // 2*ny: do-nothing terms passed from step t+1 to step t
    double* grad_w;         // one running sum of dJ/d(1/tau_g) per block
    double* grad_u;         // 2*ny running sums of dJ/du_in
    double* grad_c;         // 2*ny running sums of dJ/dC_in
    unsigned* err;          // error word: bit 1 set when a grid barrier of the multi-step kernel timed out
    unsigned barrier_extra; // test hook (see StepArgs)
};

// Threads per block of the reverse-step kernels; the fused one stages
// M(t+1) of each warp's tile in shared memory (14 rows of 136 floats a warp).
constexpr int kAdjointBlock = 128;
inline size_t adjoint_fused_smem(int block)
{
    return size_t(kPlanes) * (kTileNodes + 8) * sizeof(float) * size_t(block / 32);
}

cudaError_t adjoint_occupancy(int* blocks_per_sm);
// first: the first reverse step (A(n) from adj_next); else the fused step
// (A(t+1) gathered from mid_next)
cudaError_t launch_adjoint_step(const AdjointArgs& a, bool first, int grid, cudaStream_t s);
// Reverse steps j_hi .. j_lo (descending, all fused) in one cooperative
// launch of `grid` blocks (<= the occupancy times the SMs): state of step j
// at state_lo + (j - j_lo) stride, valve words masks[0 .. j_hi - j_lo + 1],
// M(j_hi + 1) in mid_a on entry; M(j_lo) ends in mid_a if the step count is
// even, else in mid_b.  count: a device word for the barrier (zeroed here).
cudaError_t launch_adjoint_steps_coop(const AdjointArgs& a, int j_hi, int j_lo, const float* state_lo,
                                      long long stride, const uint32_t* masks, float* mid_a, float* mid_b,
                                      unsigned* count, int grid, cudaStream_t s);
cudaError_t adjoint_coop_occupancy(int* blocks_per_sm);
cudaError_t launch_adjoint_seed(const float* state, long long plane, int pitch, const int* ox, const int* oy,
                                const float* target, const float* weight, int n, float* adj, double* J,
                                cudaStream_t s);
cudaError_t launch_sum_doubles(const double* v, int n, double* out, cudaStream_t s);

// One scalar-only step on a stored velocity field (lbm_scalar.cu).
struct ScalarArgs {
    const float* src;       // scalar plane 0 (g_0) of the source buffer; planes 1..4 follow
    float* dst;             // scalar plane 0 of the destination buffer
    const uint8_t* links;
    const RowBC* rowbc;
    const uint2* tiles;
    int n_tiles;
    int reverse;            // 1: take the tiles from the end of the table (see tile_at)
    int ny;
    int pitch;
    long long plane;
    const float* ux;        // stored field of this step's valve word, ny x pitch
    const float* uy;
    float u_scale;          // ratio of the scalar's time step to the fluid's
    float omega_g, wg0, wg1, inv_cs2g;
    float decay;            // k of the reaction term R = -k C (0: none)
    uint32_t open_mask;
    float2* partials;       // writes slots 1 and 3 of each block's four (double-float pairs)
    int n_partials;         // entries of `partials` (>= grid); those beyond the grid get 0
    int fluid_blocks;       // entries holding the last coupled step's fluid partials (slots 0, 2);
                            // blocks at or beyond it zero their slots 0 and 2
    unsigned int* err;
};

// The scalar-only step (bulk-copy pipeline): blocks of `consumers` computing
// warps and a producer warp, `per` shared-memory stages per computing warp.
cudaError_t launch_scalar_step_bulk(const ScalarArgs& a, int grid, int consumers, int per, cudaStream_t s);
cudaError_t scalar_bulk_occupancy(int consumers, int per, int* blocks_per_sm);
// The register variant of the same step (blocks of `block` threads).
cudaError_t launch_scalar_step_regs(const ScalarArgs& a, int grid, int block, cudaStream_t s);
cudaError_t scalar_regs_occupancy(int block, int* blocks_per_sm);
cudaError_t launch_velocity_of_state(const float* pop, const uint8_t* links, long long plane, float* ux, float* uy,
                                     cudaStream_t s);

// Dynamic shared memory of the bulk variant, and the attribute it needs.
size_t bulk_smem_bytes(int stages, int precision = 0);
// Dynamic shared memory of the cp.async variant (one stage per warp).
size_t async_smem_bytes(int block, int precision);
int bulk_stage_bytes(int precision = 0);
cudaError_t prepare_step_kernels();
cudaError_t launch_step(const StepArgs& a, const StepLaunch& l, cudaStream_t s);
// out[0..3] = sum of the n_blocks x 4 block partials, in a fixed order.
// The paper's wall values for the step that reads src (lbm_device.cuh,
// equilibrium_wall): for every fluid node with wall links (offsets
// woff[0..n)), the value of each population i whose source is not fluid
// goes to plane i - 1 of W (8 planes of the storage type), which the step
// kernels' kWalls instantiations read instead of bounce-back.  A
// programmatic dependent of the previous kernel.
cudaError_t launch_wall_values(const void* src, void* W, const uint8_t* links, const long long* woff, int n,
                               long long plane, int pitch, int precision, cudaStream_t s);

// The step kernels with the paper's walls (lbm_walls.cu): variants 1 and 2.
cudaError_t launch_step_walls(const StepArgs& a, const StepLaunch& l, cudaStream_t s);
cudaError_t step_walls_occupancy(const StepLaunch& l, int* blocks_per_sm);
cudaError_t prepare_walls_kernels();

cudaError_t launch_diag_finish(const float2* partials, int n_blocks, double* out, cudaStream_t s);
// A step that also forms its totals in its last block (a.diag_out set):
// variants 1 and 4 without the paper's walls (lbm_fold_steps.cu); cfg is the
// step's launch configuration.  Other launch shapes return
// cudaErrorNotSupported.
bool step_folds_totals(const StepLaunch& l);
cudaError_t launch_step_fold(const StepArgs& a, const StepLaunch& l, cudaLaunchConfig_t cfg);
cudaError_t prepare_fold_kernels();
// n coupled steps (FP32 storage, halfway bounce-back) in one cooperative
// launch of `grid` blocks of `block` threads, all resident (grid <= the
// occupancy times the SMs): src holds time t; with seq_stride = 0 the result
// of t + n ends in src if n is even, else in dst; with seq_stride > 0 (in
// floats) step s writes src + (s + 1) seq_stride (every state kept, dst
// unused).  count: a device word for the grid barrier (zeroed here).  The
// valve words of a.open_mask hold for all n steps.
cudaError_t launch_steps_coop(const StepArgs& a, int n, long long seq_stride, unsigned* count, int grid, int block,
                              cudaStream_t s);
cudaError_t steps_coop_occupancy(int block, int* blocks_per_sm);
cudaError_t step_kernel_occupancy(const StepLaunch& l, int* blocks_per_sm);

// Every node (fluid and solid, padding included) to the rest equilibrium
// of rho0 and C0.  `pop` holds elements of the given precision.  The stored
// state is post-collision: with decay rate k the equilibrium loses
// w_i k C (the collision of an equilibrium state).
cudaError_t launch_init_rest(void* pop, int ny, int pitch, float rho0, float wg0, float wg1,
                             float C0, int precision, float decay, cudaStream_t s);

// Fluid nodes to the equilibrium of fields given row-major [y][x] (nx per
// row), collided as above.
cudaError_t launch_init_fields(void* pop, const uint8_t* links, int nx, int ny, int pitch,
                               const float* rho, const float* ux, const float* uy, const float* C,
                               float wg0, float wg1, float inv_cs2g, int precision, float decay,
                               cudaStream_t s);

// Moments of the stored populations into row-major [y][x] arrays (any may be
// null); solid nodes give 0.  The stored populations are post-collision:
// with decay rate k the collision removed k C, so C is reported as
// sum g / (1 - k), the concentration before the collision (the moments of f
// are the same before and after it).
cudaError_t launch_fields(const void* pop, const uint8_t* links, int nx, int ny, int pitch,
                          float* rho, float* ux, float* uy, float* C, float wg0, float wg1, int precision,
                          float decay, cudaStream_t s);

// 16-bit storage <-> the FP32 representation (fluid planes f_i - w_i, scalar
// planes g_i), element by element over n_elems = 14 * ny * pitch.
cudaError_t launch_convert(const void* src, void* dst, long long plane, float wg0, float wg1, int precision,
                           bool to_fp32, cudaStream_t s);

}  // namespace lbm
