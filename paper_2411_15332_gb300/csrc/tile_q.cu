// Tile-kernel variants of one engine, instantiated in their own
// translation unit so that the library's objects compile in parallel.
#include "tile_fns.cuh"

namespace mera {

const void* tile_fn_dpass(int wide) {
    return wide ? (const void*)k_dpass<4, unsigned long long> : (const void*)k_dpass<4, uint32_t>;
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
