// Instantiations of the row-pipeline 2D sweep: float.
#include "sweep2dp.cuh"

namespace bte {
template <>
cudaError_t launch_sweep2dp<float>(const Sweep2DParams<float> &p, int dw, cudaStream_t st) {
    if (dw == 1) return launch_sweep2dp_t<float, 1, 8>(p, st);
    if (dw == 2) return launch_sweep2dp_t<float, 2, 8>(p, st);
    if (dw == 4) return launch_sweep2dp_t<float, 4, 8>(p, st);
    if (dw == 8) return launch_sweep2dp_t<float, 8, 8>(p, st);
    return cudaErrorInvalidConfiguration;
}

template <>
cudaError_t launch_sweep2dp_batch<float>(const Sweep2DBatch<float> &bt, int dw, cudaStream_t st) {
    if (dw == 1) return launch_sweep2dp_batch_t<float, 1, 8>(bt, st);
    if (dw == 2) return launch_sweep2dp_batch_t<float, 2, 8>(bt, st);
    if (dw == 4) return launch_sweep2dp_batch_t<float, 4, 8>(bt, st);
    if (dw == 8) return launch_sweep2dp_batch_t<float, 8, 8>(bt, st);
    return cudaErrorInvalidConfiguration;
}

size_t sweep2dp_smem(int nx, int ny, int with_phi, int groups, int dw, int stage, int real_bytes) {
    return real_bytes == 4 ? sweep2dp_smem_bytes<float>(nx, ny, with_phi, groups, dw, stage)
                           : sweep2dp_smem_bytes<double>(nx, ny, with_phi, groups, dw, stage);
}
}  // namespace bte
