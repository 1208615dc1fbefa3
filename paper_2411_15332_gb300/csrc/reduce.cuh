// Readout launchers (reduce.cu).
#pragma once
#include "common.cuh"

namespace mera {
int reduce_blocks(uint64_t N);
int observables_device(mera_state* s, int q, double* partial, double* out_dev);
// The last step of observables_device for nb partial triples already in
// device memory (a pass that summed them while writing the state).
int observables_finish(mera_state* s, const double* partial, int nb, double* out_dev);
int observables(mera_state* s, int q, double out[3]);
int argmax(mera_state* s, uint64_t* idx, double* prob);
int measure(mera_state* s, const double* u, size_t k, uint64_t* out);
int gather(mera_state* s, const uint64_t* idx, size_t k, double* out);
}  // namespace mera
