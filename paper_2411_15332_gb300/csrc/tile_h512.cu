// The 512-thread variants of the Hadamard-pass kernel (per-tile int64
// engine, 2^13-amplitude tiles), in their own translation unit so that the
// library's objects compile in parallel.
#include "tile_fns.cuh"

namespace mera {

const void* tile_fn_hpass_wide(int qin, int qout, int odd) {
    if (qin) {
        if (qout) return odd ? (const void*)k_hpass<ENG_I64, 1, 1, 1, 512> : (const void*)k_hpass<ENG_I64, 1, 1, 0, 512>;
        return odd ? (const void*)k_hpass<ENG_I64, 1, 0, 1, 512> : (const void*)k_hpass<ENG_I64, 1, 0, 0, 512>;
    }
    if (qout) return odd ? (const void*)k_hpass<ENG_I64, 0, 1, 1, 512> : (const void*)k_hpass<ENG_I64, 0, 1, 0, 512>;
    return odd ? (const void*)k_hpass<ENG_I64, 0, 0, 1, 512> : (const void*)k_hpass<ENG_I64, 0, 0, 0, 512>;
}

}  // namespace mera
