// Instantiations of the plane-pipeline 3D sweep: double (two or four
// directions per lane; eight do not fit the register budget in FP64).
#include "sweep3dp.cuh"

namespace bte {
template <>
cudaError_t launch_sweep3dp<double>(const Sweep3DParams<double> &p, int dw, cudaStream_t st) {
    if (dw == 2) return launch_sweep3dp_t<double, 2>(p, st);
    if (dw == 4) return launch_sweep3dp_t<double, 4>(p, st);
    return cudaErrorInvalidConfiguration;
}
}  // namespace bte
