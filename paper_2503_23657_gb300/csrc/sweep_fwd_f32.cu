// Instantiations of the sweep kernel: forward sweeps in float.
#include "sweep.cuh"

namespace bte {
cudaError_t launch_sweep_fwd_float(const SweepParams<float> &p, int dw, int lz, bool z, cudaStream_t st) {
    if (!z) {
        if (dw == 4 && lz == 1) return launch_sweep_t<float, 4, 1, false, false>(p, st);
        if (dw == 8 && lz == 1) return launch_sweep_t<float, 8, 1, false, false>(p, st);
        if (dw == 16 && lz == 1) return launch_sweep_t<float, 16, 1, false, false>(p, st);
    } else {
        if (dw == 4 && lz == 1) return launch_sweep_t<float, 4, 1, true, false>(p, st);
        if (dw == 4 && lz == 2) return launch_sweep_t<float, 4, 2, true, false>(p, st);
        if (dw == 4 && lz == 4) return launch_sweep_t<float, 4, 4, true, false>(p, st);
        if (dw == 4 && lz == 8) return launch_sweep_t<float, 4, 8, true, false>(p, st);
        if (dw == 8 && lz == 1) return launch_sweep_t<float, 8, 1, true, false>(p, st);
        if (dw == 8 && lz == 2) return launch_sweep_t<float, 8, 2, true, false>(p, st);
        if (dw == 8 && lz == 4) return launch_sweep_t<float, 8, 4, true, false>(p, st);
    }
    return cudaErrorInvalidConfiguration;
}
}  // namespace bte
