// Instantiations of the plane-pipeline 3D sweep with specular faces: double
// (two or four directions per lane).
#include "sweep3dp.cuh"

namespace bte {
cudaError_t launch_sweep3dp_spec_f64(const Sweep3DParams<double> &p, int dw, cudaStream_t st) {
    if (dw == 2) return launch_sweep3dp_t<double, 2, 1>(p, st);
    if (dw == 4) return launch_sweep3dp_t<double, 4, 1>(p, st);
    return cudaErrorInvalidConfiguration;
}
}  // namespace bte
