// Shared definitions of the GB300 state-vector library (C ABI in mera.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <complex>
#include <string>
#include <vector>

#include "mera.h"

namespace mera {

using cplx = std::complex<double>;

// ---------------------------------------------------------------- errors --
// Thread-local message of the last failure; entry points return a status.
void set_error(const char* fmt, ...);
const char* last_error();

struct Error {
    int code;
};

#define MERA_CHECK_CUDA(expr)                                                   \
    do {                                                                        \
        cudaError_t _e = (expr);                                                \
        if (_e != cudaSuccess) {                                                \
            ::mera::set_error("%s failed: %s (%s:%d)", #expr,                   \
                              cudaGetErrorString(_e), __FILE__, __LINE__);      \
            return MERA_ECUDA;                                                  \
        }                                                                       \
    } while (0)

#define MERA_RETURN_IF(cond, code, ...)      \
    do {                                     \
        if (cond) {                          \
            ::mera::set_error(__VA_ARGS__);  \
            return (code);                   \
        }                                    \
    } while (0)

#define MERA_TRY(expr)                  \
    do {                                \
        int _st = (expr);               \
        if (_st != MERA_OK) return _st; \
    } while (0)

// ------------------------------------------------------ launch accounting --
// Every kernel launch goes through launch_begin / launch_end so that the
// library can count launches and, when profiling is on, time each launch
// with CUDA events on its stream.
void launch_begin(cudaStream_t st, int kclass, double algorithmic_bytes);
int launch_end(cudaStream_t st);   // checks cudaGetLastError

// ----------------------------------------------------------------- state --
}  // namespace mera

struct mera_state {
    void* data = nullptr;       // 2^n amplitudes
    int n = 0;
    int dtype = MERA_C128;
    bool owns = false;
    cudaStream_t stream = nullptr;
    int device = 0;
    // small device scratch for reductions and gathers (owned)
    void* scratch = nullptr;
    size_t scratch_bytes = 0;
    // pinned host mirror of reduction results
    double* host_out = nullptr;
    // device buffer for fused-pass programs (grown on demand)
    void* prog = nullptr;
    size_t prog_bytes = 0;
    void* prog_host = nullptr;  // pinned staging of programs
    size_t prog_host_bytes = 0;
    // last fused circuit: its key (the raw ops) and its built passes, whose
    // diagonal tables are resident in `prog`
    void* fused_cache = nullptr;
    // second state-sized buffer: resident fixed-point runs alternate between
    // it and `data` (out-of-place passes), ending in `data`
    void* pong = nullptr;
    size_t pong_bytes = 0;
    bool pong_failed = false;
    // status of the bounded waits in fused passes: a device int the kernels
    // set when a wait runs out, and its pinned host copy (read after each
    // synchronisation)
    int* wait_flag = nullptr;
    int* wait_host = nullptr;
};

namespace mera {

inline size_t elem_bytes(int dtype) { return dtype == MERA_C128 ? 16 : 8; }
inline uint64_t num_amps(const mera_state* s) { return 1ull << s->n; }

int state_ensure_scratch(mera_state* s, size_t bytes);
// After a stream synchronisation: MERA_ETIMEOUT (once) if a bounded device
// wait of a fused pass ran out since the last check, else MERA_OK.
int state_check_waits(mera_state* s);
// The wait-status flag (allocated on first use).
int state_wait_flag(mera_state* s, int** flag);

// ------------------------------------------------------------ gate model --
enum GateKind { KIND_IDENTITY = 0, KIND_DIAG = 1, KIND_MONO = 2, KIND_DENSE = 3 };

// A gate reduced to its compressed index map: the DAX of its 2^k x 2^k
// matrix (entries row-major) plus the classification the kernels use.
struct PrepOp {
    int kind = KIND_DENSE;
    int k = 0;                 // targets
    int t[3] = {0, 0, 0};      // target qubits, t[0] most significant
    uint64_t cmask = 0;        // control qubits
    uint64_t cvals = 0;        // control values
    cplx m[64];                // dense 2^k x 2^k, row-major
    // monomial / diagonal view: row s reads column perm[s] with value v[s]
    int perm[8] = {0, 1, 2, 3, 4, 5, 6, 7};
    cplx v[8];
    int nact = 0;              // rows that change something
    int act[8] = {0};
    bool is_h = false;         // plain Hadamard (the RH / butterfly path)
    int bslot = -1;            // >= 0: 2x2 matrix differs per state of a batch,
                               //       coefficients at bslot * 4 of the state's table
};

// Validates and builds a PrepOp.  Returns MERA_OK or an error code.
int prepare_op(const mera_op& op, int n, PrepOp* out);
int gate_matrix(int gate, const double* params, int* nt, cplx* out);

// ------------------------------------------------------- kernel launchers --
// Per-gate path (gates.cu).
int apply_prepared(mera_state* s, const PrepOp& op);
// Fused path (fused.cu).
int apply_fused(mera_state* s, const std::vector<PrepOp>& ops);
// Fused path for a raw op list: a circuit identical to the previous fused
// circuit of the state reuses its passes and device tables.
int apply_fused_circuit(mera_state* s, const mera_op* ops, size_t nops);
// The same, then the readouts of observables() for qubit q into out[3]
// (host): summed by the circuit's last pass where it is a monomial run
// pass writing doubles, else by the readout reduction afterwards.
int apply_fused_circuit_observe(mera_state* s, const mera_op* ops, size_t nops, int q, double out[3]);
void fused_cache_free(mera_state* s);
void fused_set_bulk_shortfall(unsigned bytes);
int plan_summary(int n, int dtype, const std::vector<PrepOp>& ops, std::string* out, int* npasses);

}  // namespace mera
