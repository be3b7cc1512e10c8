// Instantiations of the row-pipeline 2D sweep: double.
#include "sweep2dp.cuh"

namespace bte {
template <>
cudaError_t launch_sweep2dp<double>(const Sweep2DParams<double> &p, int dw, cudaStream_t st) {
    if (dw == 1) return launch_sweep2dp_t<double, 1, 8>(p, st);
    if (dw == 2) return launch_sweep2dp_t<double, 2, 8>(p, st);
    if (dw == 4) return launch_sweep2dp_t<double, 4, 8>(p, st);
    if (dw == 8) return launch_sweep2dp_t<double, 8, 8>(p, st);
    return cudaErrorInvalidConfiguration;
}

template <>
cudaError_t launch_sweep2dp_batch<double>(const Sweep2DBatch<double> &bt, int dw, cudaStream_t st) {
    if (dw == 1) return launch_sweep2dp_batch_t<double, 1, 8>(bt, st);
    if (dw == 2) return launch_sweep2dp_batch_t<double, 2, 8>(bt, st);
    if (dw == 4) return launch_sweep2dp_batch_t<double, 4, 8>(bt, st);
    if (dw == 8) return launch_sweep2dp_batch_t<double, 8, 8>(bt, st);
    return cudaErrorInvalidConfiguration;
}
}  // namespace bte
