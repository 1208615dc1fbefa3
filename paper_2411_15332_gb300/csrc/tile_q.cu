// Tile-kernel variants of one engine, instantiated in their own
// translation unit so that the library's objects compile in parallel.
#include "tile_fns.cuh"

namespace mera {

const void* tile_fn_dpass(int wide) {
    return wide ? (const void*)k_dpass<4, unsigned long long> : (const void*)k_dpass<4, uint32_t>;
}

template <typename IX>
static const void* amp_fn(int qin, int qout) {
    if (qin) return qout ? (const void*)k_amp<1, 1, IX> : (const void*)k_amp<1, 0, IX>;
    return qout ? (const void*)k_amp<0, 1, IX> : (const void*)k_amp<0, 0, IX>;
}
const void* tile_fn_amp(int qin, int qout, int wide) {
    return wide ? amp_fn<unsigned long long>(qin, qout) : amp_fn<uint32_t>(qin, qout);
}
const void* tile_fn_amp_readout(int qin, int wide) {
    if (wide) return qin ? (const void*)k_amp<1, 0, unsigned long long, 1> : (const void*)k_amp<0, 0, unsigned long long, 1>;
    return qin ? (const void*)k_amp<1, 0, uint32_t, 1> : (const void*)k_amp<0, 0, uint32_t, 1>;
}

const void* tile_fn_q(int feat, int qin) {
    if (qin) {
        switch (feat) {
        case FEAT_DIAG: return (const void*)k_tile<double2, ENG_Q, FEAT_DIAG, 1>;
        case FEAT_GATES: return (const void*)k_tile<double2, ENG_Q, FEAT_GATES, 1>;
        case FEAT_GATES | FEAT_DIAG: return (const void*)k_tile<double2, ENG_Q, FEAT_GATES | FEAT_DIAG, 1>;
        default: return (const void*)k_tile<double2, ENG_Q, FEAT_ALL, 1>;
        }
    }
    switch (feat) {
    case FEAT_DIAG: return (const void*)k_tile<double2, ENG_Q, FEAT_DIAG>;
    case FEAT_GATES: return (const void*)k_tile<double2, ENG_Q, FEAT_GATES>;
    case FEAT_GATES | FEAT_DIAG: return (const void*)k_tile<double2, ENG_Q, FEAT_GATES | FEAT_DIAG>;
    default: return (const void*)k_tile<double2, ENG_Q, FEAT_ALL>;
    }
}

}  // namespace mera
