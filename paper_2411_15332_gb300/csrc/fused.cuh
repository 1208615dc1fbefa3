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
};

// fp_only: every pass in the float engine (coefficients as plain values).
template <typename V>
int fused_build(int n, const std::vector<PrepOp>& ops, FusedPlan<V>& plan, bool fp_only = false);
template <typename V>
int fused_launch(const FusedPlan<V>& plan, size_t i, PassArgs<V>& A, unsigned ny, cudaStream_t st);

}  // namespace mera
