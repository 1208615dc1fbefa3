// Entry points of the tile-kernel variants (one translation unit per
// engine: tile_q.cu, tile_i64.cu, tile_fp.cu; the Hadamard-pass kernel in
// tile_h.cu).
#pragma once

#include "tile.cuh"

namespace mera {

// complex128 kernels by engine and feature set; qin = 1 selects the
// fixed-point variant that converts its input from doubles
const void* tile_fn_q(int feat, int qin);
// the streaming kernel of single-phase table passes (resident engine);
// wide = 1: 64-bit indices (states of more than 2^32 amplitudes)
const void* tile_fn_dpass(int wide);
// affine monomial run pass: qin / qout = 1 for the resident format (0: doubles)
const void* tile_fn_amp(int qin, int qout, int wide);
// the same pass writing doubles and summing the readout (AmpArgs::rd_*)
const void* tile_fn_amp_readout(int qin, int wide);
const void* tile_fn_i64(int feat, int qin);
// the Hadamard-pass kernel (ENG_I64 or ENG_Q): qin = 1 when the pass reads
// doubles, qout = 1 when it writes the engine's own format (ENG_Q: global
// fixed point; ENG_I64: per-amplitude exponents), odd = 1 when its level
// count to scale away may be odd, wide = 1 for 512 threads (2^13-amplitude
// tiles, ENG_I64 only)
const void* tile_fn_hpass(int eng, int qin, int qout, int odd, int wide);
const void* tile_fn_hpass_wide(int qin, int qout, int odd);
const void* tile_fn_fp(int feat, int qin);
// the complex64 kernel
const void* tile_fn_c64();

}  // namespace mera
