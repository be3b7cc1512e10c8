// Instantiations of the plane-pipeline 3D sweep: double (two or four
// directions per lane; eight do not fit the register budget in FP64).
#include "sweep3dp.cuh"

namespace bte {
// problems with specular faces (sweep3dp_spec_f64.cu), sweeps with an extra
// source (sweep3dp_xsrc_f64.cu)
cudaError_t launch_sweep3dp_spec_f64(const Sweep3DParams<double> &p, int dw, cudaStream_t st);
cudaError_t launch_sweep3dp_xsrc_f64(const Sweep3DParams<double> &p, int dw, cudaStream_t st);

template <>
cudaError_t launch_sweep3dp<double>(const Sweep3DParams<double> &p, int dw, cudaStream_t st) {
    if (p.xsrc != nullptr) return launch_sweep3dp_xsrc_f64(p, dw, st);
    if (p.Fs > 0) return launch_sweep3dp_spec_f64(p, dw, st);
    if (dw == 2) return launch_sweep3dp_t<double, 2, 0>(p, st);
    if (dw == 4) return launch_sweep3dp_t<double, 4, 0>(p, st);
    return cudaErrorInvalidConfiguration;
}
}  // namespace bte
