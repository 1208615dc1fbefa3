// Fused tile passes as reusable plans (fused.cu): build once, launch over a
// single state or over a batch of states.
#pragma once

#include <vector>

#include "common.cuh"
#include "tile.cuh"

namespace mera {

template <typename V>
struct FusedPlan {
    int n = 0, K = 0;
    std::vector<PassArgs<V>> args;        // psi / tab / batch fields filled by the caller
    std::vector<unsigned char> eng, feat;
    std::vector<int> single;              // >= 0: this pass is a per-gate op
    std::vector<V> tabs;                  // diagonal tables to upload (PassArgs::tab)
    std::vector<unsigned char> dpass;     // 1: single-phase table pass for the streaming kernel
    std::vector<DPassArgs> dargs;         // its arguments (state / table pointers set at launch)
    std::vector<unsigned char> hpass;     // 1: Hadamard / sign-term pass for the pipelined kernel
    std::vector<unsigned char> amp;       // 1: affine monomial run (k_amp, out of place)
    std::vector<AmpArgs> aargs;           // its arguments (state / table pointers set at launch)
    bool resident = false;                // complex128 state kept as int64 fixed point (ENG_Q)
    int qguard = 0;                       // ENG_Q: headroom bits above the state norm
    bool efmt = false;                    // ENG_I64 Hadamard runs keep per-amplitude exponents between passes
    bool bulk = false;                    // some Hadamard pass stages its tiles with bulk copies
    int* wait_flag = nullptr;             // device int the bulk-copy waits set when they run out (set at launch)
    // readout summed by the last pass (set at launch; rd_nb receives the
    // number of partial triples written, 0 if the last pass cannot)
    double* rd_partial = nullptr;
    int rd_q = 0;
    mutable int rd_nb = 0;
};

// fp_only: every pass in the float engine (coefficients as plain values).
// amp_ok: runs of affine monomial gates of a resident plan may become single
// out-of-place passes (the caller provides a second state-sized buffer).
// resident_ok: a complex128 circuit of unitary gates whose mixing gates all
// precede a monomial body may keep the state in int64 fixed point across
// its passes, and runs of Hadamard passes of any unitary circuit may keep
// per-amplitude exponents between them (the caller then launches
// qscale_launch before the first pass and sets PassArgs::qS).  kforce > 0
// fixes the tile bits.
template <typename V>
int fused_build(int n, const std::vector<PrepOp>& ops, FusedPlan<V>& plan, bool fp_only = false,
                bool resident_ok = false, int kforce = 0, bool amp_ok = false);
// S = 59 - floor(log2 of a bound of the norm of the complex128 state psi
// (2^n amplitudes)); a pass with g headroom bits stores value * 2^(S - g).
// Uses 16 KiB of scratch; S is written to scratch + 8192.
int qscale_launch(const void* psi, int n, void* scratch, cudaStream_t st);
template <typename V>
int fused_launch(const FusedPlan<V>& plan, size_t i, PassArgs<V>& A, unsigned ny, cudaStream_t st);

}  // namespace mera
