// Instantiations of the plane-pipeline 3D sweep: float.
#include "sweep3dp.cuh"

namespace bte {
// problems with specular faces (sweep3dp_spec_f32.cu)
cudaError_t launch_sweep3dp_spec_f32(const Sweep3DParams<float> &p, int dw, cudaStream_t st);

template <>
cudaError_t launch_sweep3dp<float>(const Sweep3DParams<float> &p, int dw, cudaStream_t st) {
    if (p.Fs > 0) return launch_sweep3dp_spec_f32(p, dw, st);
    if (dw == 2) return launch_sweep3dp_t<float, 2, false>(p, st);
    if (dw == 4) return launch_sweep3dp_t<float, 4, false>(p, st);
    if (dw == 8) return launch_sweep3dp_t<float, 8, false>(p, st);
    return cudaErrorInvalidConfiguration;
}

size_t sweep3dp_smem(int R, int WY, int H, int dw, int real_bytes, bool spec) {
    return real_bytes == 4 ? sweep3dp_smem_bytes<float>(R, WY, H, dw, spec)
                           : sweep3dp_smem_bytes<double>(R, WY, H, dw, spec);
}
}  // namespace bte
