// Tile-kernel variants of one engine, instantiated in their own
// translation unit so that the library's objects compile in parallel.
#include "tile_fns.cuh"

namespace mera {

const void* tile_fn_fp(int feat, int qin) {
    (void)qin;
    switch (feat) {
    case FEAT_DIAG: return (const void*)k_tile<double2, ENG_FP, FEAT_DIAG>;
    case FEAT_GATES: return (const void*)k_tile<double2, ENG_FP, FEAT_GATES>;
    case FEAT_GATES | FEAT_DIAG: return (const void*)k_tile<double2, ENG_FP, FEAT_GATES | FEAT_DIAG>;
    default: return (const void*)k_tile<double2, ENG_FP, FEAT_ALL>;
    }
}

const void* tile_fn_c64() { return (const void*)k_tile<float2, ENG_FP, FEAT_ALL>; }

}  // namespace mera
