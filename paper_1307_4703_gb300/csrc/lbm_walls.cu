// lbm_walls.cu -- the coupled step kernels with the paper's wall scheme
// (section "Boundary Conditions": equilibrium interpolation), the kWalls
// instantiations of lbm_step.cuh.  Each step first runs wall_values
// (lbm_kernels.cu), which writes the value of every population whose source
// is not fluid into an 8-plane buffer; these kernels read it where the
// default ones bounce back.  Variants 1 and 2, every storage precision.
#include "lbm_step.cuh"

namespace lbm {

cudaError_t prepare_walls_kernels()
{
    cudaError_t e = cudaFuncSetAttribute(coupled_step_bulk<float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         int(bulk_smem_bytes(kMaxStages)));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(coupled_step_bulk<__half, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 int(bulk_smem_bytes(kMaxStages, kFP16)));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(coupled_step_bulk<__nv_bfloat16, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 int(bulk_smem_bytes(kMaxStages, kBF16)));
    return e;
}

cudaError_t launch_step_walls(const StepArgs& a, const StepLaunch& l, cudaStream_t s)
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
    cudaError_t e;
    if (l.variant == kVariantBulk) {
        const int per = l.stages / (l.block / 32 - 1);
        cfg.dynamicSmemBytes = bulk_smem_bytes(l.stages, l.precision);
        if (l.precision == kFP16) e = cudaLaunchKernelEx(&cfg, coupled_step_bulk<__half, true>, a, per);
        else if (l.precision == kBF16) e = cudaLaunchKernelEx(&cfg, coupled_step_bulk<__nv_bfloat16, true>, a, per);
        else e = cudaLaunchKernelEx(&cfg, coupled_step_bulk<float, true>, a, per);
    } else if (l.variant == kVariantRegs) {
        if (l.precision == kFP16) e = cudaLaunchKernelEx(&cfg, coupled_step_regs<__half, true>, a);
        else if (l.precision == kBF16) e = cudaLaunchKernelEx(&cfg, coupled_step_regs<__nv_bfloat16, true>, a);
        else e = cudaLaunchKernelEx(&cfg, coupled_step_regs<float, true>, a);
    } else {
        return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t step_walls_occupancy(const StepLaunch& l, int* blocks_per_sm)
{
    if (l.variant == kVariantBulk) {
        const size_t smem = bulk_smem_bytes(l.stages, l.precision);
        if (l.precision == kFP16)
            return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, coupled_step_bulk<__half, true>, l.block,
                                                                 smem);
        if (l.precision == kBF16)
            return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, coupled_step_bulk<__nv_bfloat16, true>,
                                                                 l.block, smem);
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, coupled_step_bulk<float, true>, l.block, smem);
    }
    if (l.variant != kVariantRegs) return cudaErrorInvalidValue;
    if (l.precision == kFP16)
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, coupled_step_regs<__half, true>, l.block, 0);
    if (l.precision == kBF16)
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, coupled_step_regs<__nv_bfloat16, true>,
                                                             l.block, 0);
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, coupled_step_regs<float, true>, l.block, 0);
}

}  // namespace lbm
