// Instantiations of the plane-pipeline 3D sweep with specular faces: float
// (a translation unit of its own, compiled in parallel with the others).
#include "sweep3dp.cuh"

namespace bte {
cudaError_t launch_sweep3dp_spec_f32(const Sweep3DParams<float> &p, int dw, cudaStream_t st) {
    if (dw == 2) return launch_sweep3dp_t<float, 2, 1>(p, st);
    if (dw == 4) return launch_sweep3dp_t<float, 4, 1>(p, st);
    if (dw == 8) return launch_sweep3dp_t<float, 8, 1>(p, st);
    return cudaErrorInvalidConfiguration;
}
}  // namespace bte
