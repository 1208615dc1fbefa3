// Variants of the Hadamard-pass kernel (k_hpass), in their own translation
// unit so that the library's objects compile in parallel.
#include "tile_fns.cuh"

namespace mera {

template <int QIN, int QOUT>
static const void* hpass_q(int odd) {
    return odd ? (const void*)k_hpass<ENG_Q, QIN, QOUT, 1> : (const void*)k_hpass<ENG_Q, QIN, QOUT, 0>;
}

static const void* hpass_i64_256(int qin, int qout, int odd) {
    if (qin) {
        if (qout) return odd ? (const void*)k_hpass<ENG_I64, 1, 1, 1> : (const void*)k_hpass<ENG_I64, 1, 1, 0>;
        return odd ? (const void*)k_hpass<ENG_I64, 1, 0, 1> : (const void*)k_hpass<ENG_I64, 1, 0, 0>;
    }
    if (qout) return odd ? (const void*)k_hpass<ENG_I64, 0, 1, 1> : (const void*)k_hpass<ENG_I64, 0, 1, 0>;
    return odd ? (const void*)k_hpass<ENG_I64, 0, 0, 1> : (const void*)k_hpass<ENG_I64, 0, 0, 0>;
}

const void* tile_fn_hpass(int eng, int qin, int qout, int odd, int wide) {
    if (eng == ENG_Q) {
        if (qin) return qout ? hpass_q<1, 1>(odd) : hpass_q<1, 0>(odd);
        return qout ? hpass_q<0, 1>(odd) : hpass_q<0, 0>(odd);
    }
    return wide ? tile_fn_hpass_wide(qin, qout, odd) : hpass_i64_256(qin, qout, odd);
}

}  // namespace mera
