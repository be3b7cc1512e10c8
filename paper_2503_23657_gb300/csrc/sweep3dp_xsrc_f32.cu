// Instantiations of the plane-pipeline 3D sweep with an extra source
// (implicit-Euler time steps, the extension the paper's Conclusion
// announces), with and without specular faces: float.  The forward sweeps of
// a time step add xscale * xsrc[c][b][d] (e of the previous step over dt) to
// every direction's right-hand side; the kernel copies the next step's row of
// DW values into shared memory a step ahead.
#include "sweep3dp.cuh"

namespace bte {
cudaError_t launch_sweep3dp_xsrc_f32(const Sweep3DParams<float> &p, int dw, cudaStream_t st) {
    const bool spec = p.Fs > 0;
    if (dw == 2) return spec ? launch_sweep3dp_t<float, 2, 3>(p, st) : launch_sweep3dp_t<float, 2, 2>(p, st);
    if (dw == 4) return spec ? launch_sweep3dp_t<float, 4, 3>(p, st) : launch_sweep3dp_t<float, 4, 2>(p, st);
    if (dw == 8) return spec ? launch_sweep3dp_t<float, 8, 3>(p, st) : launch_sweep3dp_t<float, 8, 2>(p, st);
    return cudaErrorInvalidConfiguration;
}
}  // namespace bte
