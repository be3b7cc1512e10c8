// Instantiations of the general sweep kernel's extended variant (specularly
// reflecting faces, extra per-direction source, cell-size gradient
// partials): kSpecDW directions per lane, forward and adjoint, both
// precisions.
#include "sweep.cuh"

namespace bte {

template <typename real, bool ADJ>
cudaError_t launch_sweep_spec_t(const SweepParams<real> &p, int lz, bool z, cudaStream_t st) {
    constexpr int W = kSpecDW;
    if (!z) return lz == 1 ? launch_sweep_t<real, W, 1, false, ADJ, true>(p, st) : cudaErrorInvalidConfiguration;
    if (lz == 1) return launch_sweep_t<real, W, 1, true, ADJ, true>(p, st);
    if (lz == 2) return launch_sweep_t<real, W, 2, true, ADJ, true>(p, st);
    if (lz == 4) return launch_sweep_t<real, W, 4, true, ADJ, true>(p, st);
    if (lz == 8) return launch_sweep_t<real, W, 8, true, ADJ, true>(p, st);
    return cudaErrorInvalidConfiguration;
}

cudaError_t launch_sweep_spec_float(const SweepParams<float> &p, int lz, bool z, bool adj, cudaStream_t st) {
    return adj ? launch_sweep_spec_t<float, true>(p, lz, z, st) : launch_sweep_spec_t<float, false>(p, lz, z, st);
}

cudaError_t launch_sweep_spec_double(const SweepParams<double> &p, int lz, bool z, bool adj, cudaStream_t st) {
    return adj ? launch_sweep_spec_t<double, true>(p, lz, z, st) : launch_sweep_spec_t<double, false>(p, lz, z, st);
}

}  // namespace bte
