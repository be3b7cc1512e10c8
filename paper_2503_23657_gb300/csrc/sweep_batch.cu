// Batched general-kernel sweeps of 2D instances that the row-pipeline kernel
// does not take (masks, several regions): one launch per class of instances
// with the same warps along y, forward only, 4 or 8 directions per lane.
#include "sweep.cuh"

namespace bte {

template <typename real, int DW>
cudaError_t launch_sweep_batch_t(const SweepBatch<real> &bt, cudaStream_t st) {
    const int threads = bt.WY * 32;
    if (bt.n_inst < 1 || threads > SweepTile<DW, 1, false>::kMaxThreads) return cudaErrorInvalidConfiguration;
    // no staged boundary values (instances differ in face count)
    const size_t smem = sweep_smem_bytes<real, DW, 1, false>(bt.R_max, bt.WY, 0, 0);
    auto kern = sweep_batch_kernel<real, DW>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    kern<<<dim3(bt.chunks, bt.B, bt.n_inst), threads, smem, st>>>(bt.params, bt.inst);
    return cudaGetLastError();
}

template <>
cudaError_t launch_sweep_batch<float>(const SweepBatch<float> &bt, int dw, cudaStream_t st) {
    if (dw == 4) return launch_sweep_batch_t<float, 4>(bt, st);
    if (dw == 8) return launch_sweep_batch_t<float, 8>(bt, st);
    return cudaErrorInvalidConfiguration;
}

template <>
cudaError_t launch_sweep_batch<double>(const SweepBatch<double> &bt, int dw, cudaStream_t st) {
    if (dw == 4) return launch_sweep_batch_t<double, 4>(bt, st);
    if (dw == 8) return launch_sweep_batch_t<double, 8>(bt, st);
    return cudaErrorInvalidConfiguration;
}

}  // namespace bte
