// Instantiations of the plane-pipeline 3D sweep: float.
#include "sweep3dp.cuh"

namespace bte {
// problems with specular faces (sweep3dp_spec_f32.cu), sweeps with an extra
// source (sweep3dp_xsrc_f32.cu)
cudaError_t launch_sweep3dp_spec_f32(const Sweep3DParams<float> &p, int dw, cudaStream_t st);
cudaError_t launch_sweep3dp_xsrc_f32(const Sweep3DParams<float> &p, int dw, cudaStream_t st);

template <>
cudaError_t launch_sweep3dp<float>(const Sweep3DParams<float> &p, int dw, cudaStream_t st) {
    if (p.xsrc != nullptr) return launch_sweep3dp_xsrc_f32(p, dw, st);
    if (p.Fs > 0) return launch_sweep3dp_spec_f32(p, dw, st);
    if (dw == 2) return launch_sweep3dp_t<float, 2, 0>(p, st);
    if (dw == 4) return launch_sweep3dp_t<float, 4, 0>(p, st);
    if (dw == 8) return launch_sweep3dp_t<float, 8, 0>(p, st);
    return cudaErrorInvalidConfiguration;
}

size_t sweep3dp_smem(int R, int WY, int H, int dw, int real_bytes, int variant) {
    return real_bytes == 4 ? sweep3dp_smem_bytes<float>(R, WY, H, dw, variant)
                           : sweep3dp_smem_bytes<double>(R, WY, H, dw, variant);
}
}  // namespace bte
