// Dispatch of sweep launches to the instantiated tiles.
#include "sweep.cuh"

namespace bte {

cudaError_t launch_sweep_fwd_float(const SweepParams<float> &p, int dw, int lz, bool z, cudaStream_t st);
cudaError_t launch_sweep_adj_float(const SweepParams<float> &p, int dw, int lz, bool z, cudaStream_t st);
cudaError_t launch_sweep_fwd_double(const SweepParams<double> &p, int dw, int lz, bool z, cudaStream_t st);
cudaError_t launch_sweep_adj_double(const SweepParams<double> &p, int dw, int lz, bool z, cudaStream_t st);
cudaError_t launch_sweep_spec_float(const SweepParams<float> &p, int lz, bool z, bool adj, cudaStream_t st);
cudaError_t launch_sweep_spec_double(const SweepParams<double> &p, int lz, bool z, bool adj, cudaStream_t st);

int sweep_max_threads(int dw, int lz, bool z) {
    if (!z) {
        if (dw == 4 && lz == 1) return SweepTile<4, 1, false>::kMaxThreads;
        if (dw == 8 && lz == 1) return SweepTile<8, 1, false>::kMaxThreads;
        if (dw == 16 && lz == 1) return SweepTile<16, 1, false>::kMaxThreads;
    } else {
        if (dw == 4 && lz == 1) return SweepTile<4, 1, true>::kMaxThreads;
        if (dw == 4 && lz == 2) return SweepTile<4, 2, true>::kMaxThreads;
        if (dw == 4 && lz == 4) return SweepTile<4, 4, true>::kMaxThreads;
        if (dw == 4 && lz == 8) return SweepTile<4, 8, true>::kMaxThreads;
        if (dw == 8 && lz == 1) return SweepTile<8, 1, true>::kMaxThreads;
        if (dw == 8 && lz == 2) return SweepTile<8, 2, true>::kMaxThreads;
        if (dw == 8 && lz == 4) return SweepTile<8, 4, true>::kMaxThreads;
    }
    return 0;
}

// specular faces, an extra source or cell-size gradient partials: the EXT
// variant (kSpecDW directions per lane)
template <>
cudaError_t launch_sweep<float>(const SweepParams<float> &p, int dw, int lz, bool z, bool adj, cudaStream_t st) {
    if (p.sidx || p.xsrc || p.glpart)
        return dw == kSpecDW ? launch_sweep_spec_float(p, lz, z, adj, st) : cudaErrorInvalidConfiguration;
    return adj ? launch_sweep_adj_float(p, dw, lz, z, st) : launch_sweep_fwd_float(p, dw, lz, z, st);
}

template <>
cudaError_t launch_sweep<double>(const SweepParams<double> &p, int dw, int lz, bool z, bool adj, cudaStream_t st) {
    if (p.sidx || p.xsrc || p.glpart)
        return dw == kSpecDW ? launch_sweep_spec_double(p, lz, z, adj, st) : cudaErrorInvalidConfiguration;
    return adj ? launch_sweep_adj_double(p, dw, lz, z, st) : launch_sweep_fwd_double(p, dw, lz, z, st);
}

}  // namespace bte
