// Instantiations of the row-block 2D sweep: float.
#include "sweep2d.cuh"

namespace bte {
cudaError_t launch_sweep2d_float(const Sweep2DParams<float> &p, int dw, int rb, bool adj, cudaStream_t st) {
    if (dw == 1 && rb == 1) return adj ? launch_sweep2d_t<float, 1, 1, true>(p, st) : launch_sweep2d_t<float, 1, 1, false>(p, st);
    if (dw == 1 && rb == 2) return adj ? launch_sweep2d_t<float, 1, 2, true>(p, st) : launch_sweep2d_t<float, 1, 2, false>(p, st);
    if (dw == 1 && rb == 3) return adj ? launch_sweep2d_t<float, 1, 3, true>(p, st) : launch_sweep2d_t<float, 1, 3, false>(p, st);
    if (dw == 1 && rb == 4) return adj ? launch_sweep2d_t<float, 1, 4, true>(p, st) : launch_sweep2d_t<float, 1, 4, false>(p, st);
    if (dw == 1 && rb == 5) return adj ? launch_sweep2d_t<float, 1, 5, true>(p, st) : launch_sweep2d_t<float, 1, 5, false>(p, st);
    if (dw == 2 && rb == 1) return adj ? launch_sweep2d_t<float, 2, 1, true>(p, st) : launch_sweep2d_t<float, 2, 1, false>(p, st);
    if (dw == 2 && rb == 2) return adj ? launch_sweep2d_t<float, 2, 2, true>(p, st) : launch_sweep2d_t<float, 2, 2, false>(p, st);
    if (dw == 2 && rb == 3) return adj ? launch_sweep2d_t<float, 2, 3, true>(p, st) : launch_sweep2d_t<float, 2, 3, false>(p, st);
    if (dw == 2 && rb == 4) return adj ? launch_sweep2d_t<float, 2, 4, true>(p, st) : launch_sweep2d_t<float, 2, 4, false>(p, st);
    if (dw == 2 && rb == 5) return adj ? launch_sweep2d_t<float, 2, 5, true>(p, st) : launch_sweep2d_t<float, 2, 5, false>(p, st);
    if (dw == 4 && rb == 1) return adj ? launch_sweep2d_t<float, 4, 1, true>(p, st) : launch_sweep2d_t<float, 4, 1, false>(p, st);
    if (dw == 4 && rb == 2) return adj ? launch_sweep2d_t<float, 4, 2, true>(p, st) : launch_sweep2d_t<float, 4, 2, false>(p, st);
    if (dw == 4 && rb == 3) return adj ? launch_sweep2d_t<float, 4, 3, true>(p, st) : launch_sweep2d_t<float, 4, 3, false>(p, st);
    if (dw == 4 && rb == 4) return adj ? launch_sweep2d_t<float, 4, 4, true>(p, st) : launch_sweep2d_t<float, 4, 4, false>(p, st);
    if (dw == 4 && rb == 5) return adj ? launch_sweep2d_t<float, 4, 5, true>(p, st) : launch_sweep2d_t<float, 4, 5, false>(p, st);
    return cudaErrorInvalidConfiguration;
}

template <>
cudaError_t launch_sweep2d<float>(const Sweep2DParams<float> &p, int dw, int rb, bool adj, cudaStream_t st) {
    return launch_sweep2d_float(p, dw, rb, adj, st);
}

size_t sweep2d_smem(int nx, int ny, int stage, int with_phi, int warps, int rb, int ring, int real_bytes) {
    return real_bytes == 4 ? sweep2d_smem_bytes<float>(nx, ny, stage, with_phi, warps, rb, ring)
                           : sweep2d_smem_bytes<double>(nx, ny, stage, with_phi, warps, rb, ring);
}
}  // namespace bte
