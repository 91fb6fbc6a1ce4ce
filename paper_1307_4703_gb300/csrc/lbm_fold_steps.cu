// lbm_fold_steps.cu -- the coupled step kernels of variants 1 and 4 (halfway
// bounce-back walls) instantiated with kFold: besides the step, the last
// block to finish adds up every block's diagnostics partials and writes the
// four totals (fold_totals).  lbm_step_diagnostics launches these, so that a
// step hands its totals to the host without a reduction launch; lbm_step
// launches the kernels without the fold, which carry no call to it.
#include "lbm_step.cuh"

namespace lbm {

bool step_folds_totals(const StepLaunch& l)
{
    return !l.walls && l.block >= kFoldThreads && (l.variant == kVariantRegs || l.variant == kVariantAsync);
}

cudaError_t prepare_fold_kernels()
{
    const int async_max = int(async_smem_bytes(kBulkMaxThreads, kFP32));  // up to 8 warps per block
    cudaError_t e = cudaFuncSetAttribute(coupled_step_async<float, false, true>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, async_max);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(coupled_step_async<__half, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 async_max);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(coupled_step_async<__nv_bfloat16, false, true>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, async_max);
    return e;
}

cudaError_t launch_step_fold(const StepArgs& a, const StepLaunch& l, cudaLaunchConfig_t cfg)
{
    if (!step_folds_totals(l)) return cudaErrorNotSupported;
    cudaError_t e;
    if (l.variant == kVariantAsync) {
        cfg.dynamicSmemBytes = async_smem_bytes(l.block, l.precision);
        if (l.precision == kFP16) e = cudaLaunchKernelEx(&cfg, coupled_step_async<__half, false, true>, a);
        else if (l.precision == kBF16) e = cudaLaunchKernelEx(&cfg, coupled_step_async<__nv_bfloat16, false, true>, a);
        else e = cudaLaunchKernelEx(&cfg, coupled_step_async<float, false, true>, a);
    } else if (l.precision == kFP16) {
        e = cudaLaunchKernelEx(&cfg, coupled_step_regs<__half, false, true>, a);
    } else if (l.precision == kBF16) {
        e = cudaLaunchKernelEx(&cfg, coupled_step_regs<__nv_bfloat16, false, true>, a);
    } else {
        e = cudaLaunchKernelEx(&cfg, coupled_step_regs<float, false, true>, a);
    }
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace lbm
