// Tile-kernel variants of one engine, instantiated in their own
// translation unit so that the library's objects compile in parallel.
#include "tile_fns.cuh"

namespace mera {

const void* tile_fn_i64(int feat, int qin) {
    (void)qin;
    switch (feat) {
    case FEAT_DIAG: return (const void*)k_tile<double2, ENG_I64, FEAT_DIAG>;
    case FEAT_GATES: return (const void*)k_tile<double2, ENG_I64, FEAT_GATES>;
    case FEAT_GATES | FEAT_DIAG: return (const void*)k_tile<double2, ENG_I64, FEAT_GATES | FEAT_DIAG>;
    default: return (const void*)k_tile<double2, ENG_I64, FEAT_ALL>;
    }
}

}  // namespace mera
