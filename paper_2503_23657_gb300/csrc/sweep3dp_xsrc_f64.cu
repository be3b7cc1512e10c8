// Instantiations of the plane-pipeline 3D sweep with an extra source
// (implicit-Euler time steps), with and without specular faces: double.
#include "sweep3dp.cuh"

namespace bte {
cudaError_t launch_sweep3dp_xsrc_f64(const Sweep3DParams<double> &p, int dw, cudaStream_t st) {
    const bool spec = p.Fs > 0;
    if (dw == 2) return spec ? launch_sweep3dp_t<double, 2, 3>(p, st) : launch_sweep3dp_t<double, 2, 2>(p, st);
    if (dw == 4) return spec ? launch_sweep3dp_t<double, 4, 3>(p, st) : launch_sweep3dp_t<double, 4, 2>(p, st);
    return cudaErrorInvalidConfiguration;
}
}  // namespace bte
