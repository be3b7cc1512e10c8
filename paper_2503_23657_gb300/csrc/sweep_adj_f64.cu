// Instantiations of the sweep kernel: transposed (adjoint) sweeps in double.
#include "sweep.cuh"

namespace bte {
cudaError_t launch_sweep_adj_double(const SweepParams<double> &p, int dw, int lz, bool z, cudaStream_t st) {
    if (!z) {
        if (dw == 4 && lz == 1) return launch_sweep_t<double, 4, 1, false, true>(p, st);
        if (dw == 8 && lz == 1) return launch_sweep_t<double, 8, 1, false, true>(p, st);
        if (dw == 16 && lz == 1) return launch_sweep_t<double, 16, 1, false, true>(p, st);
    } else {
        if (dw == 4 && lz == 1) return launch_sweep_t<double, 4, 1, true, true>(p, st);
        if (dw == 4 && lz == 2) return launch_sweep_t<double, 4, 2, true, true>(p, st);
        if (dw == 4 && lz == 4) return launch_sweep_t<double, 4, 4, true, true>(p, st);
        if (dw == 4 && lz == 8) return launch_sweep_t<double, 4, 8, true, true>(p, st);
        if (dw == 8 && lz == 1) return launch_sweep_t<double, 8, 1, true, true>(p, st);
        if (dw == 8 && lz == 2) return launch_sweep_t<double, 8, 2, true, true>(p, st);
        if (dw == 8 && lz == 4) return launch_sweep_t<double, 8, 4, true, true>(p, st);
    }
    return cudaErrorInvalidConfiguration;
}
}  // namespace bte
