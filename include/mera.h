/*
 * mera.h -- C ABI of the GB300 state-vector library for the Mera method
 * (Song et al., "Mera: Memory Reduction and Acceleration for Quantum
 * Circuit Simulation via Redundancy Exploration", arXiv 2411.15332).
 *
 * The library applies quantum gates to a 2^n-amplitude state vector on one
 * GPU without forming the 2^n x 2^n operation matrix of Eq. 6: sparse gates
 * go through their compressed index map (the DAX / DAS structures of
 * Sec. III-A, applied on the fly), Hadamard layers through the RH structure
 * of Sec. III-B (its on-demand signs realised as in-place butterflies).
 *
 * Conventions
 *   - Qubit q is bit q of the basis index (qubit 0 = least significant).
 *     The paper's Eq. 6 numbers qubits from the most significant end; its
 *     qubit k is bit n-k here.
 *   - A state is N = 2^n contiguous complex amplitudes: MERA_C128 is
 *     interleaved (re, im) float64 (16 B, the paper's precision, Sec.
 *     III-A.1), MERA_C64 interleaved float32 (8 B).
 *   - A gate on k targets is a 2^k x 2^k matrix in the basis |t_0 .. t_{k-1}>,
 *     targets[0] the most significant bit of the sub-index.  Controls are
 *     given as a bit mask with the bit values they must hold.
 *   - Pointers are host pointers unless the name says dev_ptr.  The caller
 *     keeps ownership of everything it passes in; objects returned through
 *     an out-parameter are owned by the caller and released with the
 *     matching *_destroy call.
 *
 * Errors: every call returns an int status (MERA_OK = 0).  On failure,
 * mera_last_error() gives a message for the calling host thread.  No C++
 * exception or abort crosses this boundary.  Errors detected before any
 * launch leave the state unchanged.  Calls on one state are asynchronous
 * on the state's stream unless documented as synchronous (readouts).
 */
#ifndef MERA_H
#define MERA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define MERA_OK 0
#define MERA_EINVAL 1        /* bad argument: n, qubit >= n, duplicate qubit, NaN ... */
#define MERA_ENOMEM 2        /* device or host allocation failed */
#define MERA_EUNSUPPORTED 3  /* dtype / gate arity not supported */
#define MERA_ECUDA 4         /* a CUDA runtime call failed */
#define MERA_ETIMEOUT 5      /* a bounded device wait ran out */

/* ---- element types ----------------------------------------------------- */
#define MERA_C64 0           /* complex64: float32 re, im */
#define MERA_C128 1          /* complex128: float64 re, im */

#define MERA_MAX_QUBITS 36

/* ---- gate catalogue (Table I of the paper; controls added by mask) ------ */
enum mera_gate {
    MERA_GATE_I = 0,
    MERA_GATE_X, MERA_GATE_Y, MERA_GATE_Z, MERA_GATE_H,
    MERA_GATE_S, MERA_GATE_SDG, MERA_GATE_T, MERA_GATE_TDG,
    MERA_GATE_SX, MERA_GATE_SXDG,
    MERA_GATE_P,      /* params: lambda; diag(1, e^{i lambda}) (Phase, U1) */
    MERA_GATE_RX, MERA_GATE_RY, MERA_GATE_RZ,   /* params: theta; exp(-i theta P/2) */
    MERA_GATE_R,      /* params: theta, phi; rotation about cos(phi) X + sin(phi) Y */
    MERA_GATE_U2,     /* params: phi, lambda = U(pi/2, phi, lambda) */
    MERA_GATE_U,      /* params: theta, phi, lambda, gamma (4 values; gamma = global phase, 0 for U3) */
    MERA_GATE_SWAP, MERA_GATE_ISWAP, MERA_GATE_DCX, MERA_GATE_ECR,
    MERA_GATE_RXX, MERA_GATE_RYY, MERA_GATE_RZZ, MERA_GATE_RZX, /* params: theta */
    MERA_GATE_FLIP,   /* no targets: multiply the controlled sub-space by -1 */
    MERA_GATE_MATRIX, /* explicit 2^k x 2^k matrix, mera_op.matrix */
    MERA_GATE_COUNT
};

/* One circuit operation. */
typedef struct mera_op {
    int32_t gate;          /* enum mera_gate */
    int32_t nt;            /* number of targets, 0..3 */
    int32_t targets[3];    /* targets[0] is the most significant sub-index bit */
    int32_t reserved;      /* must be 0 */
    uint64_t cmask;        /* control qubits (bit q set = qubit q controls) */
    uint64_t cvals;        /* required control values (bits inside cmask) */
    double params[4];      /* angles, see enum mera_gate */
    const double* matrix;  /* MERA_GATE_MATRIX only: host, 2^nt x 2^nt
                              interleaved complex128, row-major; copied */
} mera_op;

/* apply modes of mera_apply_circuit */
#define MERA_MODE_PER_GATE 0   /* one kernel launch per gate (Eq. 7 per gate) */
#define MERA_MODE_FUSED 1      /* shared-memory tile passes, gates fused */

typedef struct mera_state mera_state;

/* ---- library ----------------------------------------------------------- */

/* Message of the last failed call on this host thread ("" if none).
 * The string stays valid until the next failing call on the thread. */
const char* mera_last_error(void);

/* Library version string (static storage). */
const char* mera_version(void);

/* Number of kernels this library has launched in the process so far
 * (all devices, all states).  Synchronous, host only. */
uint64_t mera_launch_count(void);

/* ---- state lifetime (Sec. II-A, Eq. 3: the 2^n-amplitude state vector) -- */

/* Allocate a state of n qubits (1 <= n <= MERA_MAX_QUBITS) on the current
 * device with cudaMalloc, initialised to |0...0>, bound to the legacy
 * default stream.  *out receives the new state (owned by the caller). */
int mera_state_create(int n, int dtype, mera_state** out);

/* Borrow caller-owned device memory of 2^n amplitudes of `dtype` (e.g. a
 * torch tensor's storage; 16-byte aligned).  The contents are left as
 * they are.  The caller keeps the memory alive until mera_state_destroy.
 * `stream` is a cudaStream_t (NULL = legacy default stream). */
int mera_state_wrap(void* dev_ptr, int n, int dtype, void* stream, mera_state** out);

/* Release the state: frees the amplitudes only if mera_state_create made
 * them, plus the state's small internal scratch buffers.  NULL is a no-op. */
int mera_state_destroy(mera_state* s);

/* Rebind the state to another stream (a cudaStream_t). */
int mera_state_set_stream(mera_state* s, void* stream);

/* Device pointer of the amplitudes, qubit count and dtype. */
int mera_state_info(const mera_state* s, void** dev_ptr, int* n, int* dtype);

/* Set the state to the basis state |index>.  Asynchronous. */
int mera_state_set_basis(mera_state* s, uint64_t index);

/* Copy 2^n amplitudes from / to host memory (pinned memory gives full
 * bandwidth).  Synchronous: returns after the copy completed. */
int mera_state_copy_from_host(mera_state* s, const void* host);
/* As mera_state_copy_from_host, but only enqueued on the state's stream:
 * the call returns at once and the copy overlaps work on other streams
 * (truly asynchronous for page-locked host memory).  The host buffer must
 * stay valid and unchanged until the state's stream has passed the copy
 * (mera_state_synchronize or any later synchronising call on the state). */
int mera_state_copy_from_host_async(mera_state* s, const void* host);
int mera_state_copy_to_host(mera_state* s, void* host);

/* Read k amplitudes at basis indices idx[0..k-1] (host array) into
 * out[2k] as float64 (re, im) pairs, whatever the dtype.  Synchronous. */
int mera_state_get_amplitudes(mera_state* s, const uint64_t* idx, size_t k, double* out);

/* Wait for all work queued on the state's stream. */
int mera_state_synchronize(mera_state* s);

/* ---- gates (Sec. II-A Eq. 6-7 without the operation matrix; Sec. III-A.2
 *      MVM on the gate's compressed index map) ------------------------- */

/* 2^k x 2^k matrix of a catalogue gate, k = number of targets it takes
 * (returned in *nt), written to out[2 * 4^k] as interleaved complex128,
 * row-major.  out must hold 128 doubles.  Host only. */
int mera_gate_matrix(int gate, const double* params, int* nt, double* out);

/* Apply one gate.  targets[nt] and controls[nc] are qubit indices; every
 * qubit may appear once.  params: as enum mera_gate (NULL if none). */
int mera_apply_gate(mera_state* s, int gate, const int* targets, int nt,
                    const int* controls, int nc, const double* params);

/* Apply an explicit 2^nt x 2^nt matrix (interleaved complex128 row-major,
 * host memory, copied) to targets, under controls (all must be 1). */
int mera_apply_matrix(mera_state* s, const double* matrix, const int* targets, int nt,
                      const int* controls, int nc);

/* Apply ops[0..nops-1] in order.  MERA_MODE_PER_GATE launches one kernel per
 * op; MERA_MODE_FUSED plans shared-memory tile passes that apply runs of
 * gates (and Hadamard butterflies) per HBM read/write.  All ops are
 * validated before anything is launched.  Launches are asynchronous: a
 * fused pass that stages its tiles with bulk copies waits for them with a
 * bounded wait (about a second); one that ran out is reported as
 * MERA_ETIMEOUT, once, by the next call that synchronises the state's
 * stream (mera_state_synchronize, mera_state_copy_to_host, the readouts),
 * and the amplitudes are then not valid. */
int mera_apply_circuit(mera_state* s, const mera_op* ops, size_t nops, int mode);

/* mera_apply_circuit followed by mera_observables(s, q, out): the circuit,
 * then out[0] = norm^2, out[1] = <Z_q>, out[2] = sum over qubits of <Z_q>
 * (Eq. 4-5), summed in float64.  In MERA_MODE_FUSED, when the circuit's
 * last pass is a monomial run pass that writes the state as doubles, that
 * pass sums the readout while it stores the amplitudes (no further read of
 * the state); otherwise the readout reduction runs after the circuit.
 * Synchronises the state's stream; q out of range is MERA_EINVAL. */
int mera_apply_circuit_observe(mera_state* s, const mera_op* ops, size_t nops, int mode, int q, double out[3]);

/* Describe how MERA_MODE_FUSED would run ops[0..nops-1] on n qubits of
 * `dtype`, without touching a GPU: a header line (tile bits, passes,
 * whether the complex128 state stays int64 fixed point across passes),
 * then one line per tile pass (tile
 * bits, arithmetic engine, Hadamard levels, register phases, op kinds,
 * the kernel that runs it: "stream" / "pipelined" (Hadamard-pass kernel) /
 * "amp" (a run of affine permutation gates then diagonal gates as one
 * monomial operator, gathered from the whole state; its index-map offsets,
 * table selection bits and sign terms follow) / neither (general tile
 * kernel), permutation runs on its loads / stores
 * ("gather" / "scatter"), "bulk" where the Hadamard-pass kernel stages its
 * tiles with bulk copies of 128-byte chunks, and for the resident engine its scaling: levels
 * scaled at the end and at phase exits, headroom bits), written as a
 * NUL-terminated string into out[cap] (truncated if longer).  Host only;
 * *npasses (may be NULL) receives the number of passes. */
int mera_plan_summary(int n, int dtype, const mera_op* ops, size_t nops, char* out, size_t cap, int* npasses);

/* H on every qubit q with bit q of `mask` set: the RH structure of Sec.
 * III-B (H^{(x)m} stored as its magnitude 2^{-m/2}, element signs
 * (-1)^popcount(r & c), Fig. 3), applied in place as butterflies; same
 * result as the RH-MVM of Algorithm 1 for mask = all qubits. */
int mera_hadamard_layer(mera_state* s, uint64_t mask);

/* The paper's own RH-MVM of H^{(x)n} (Sec. III-B.2, Table II, Algorithm 1):
 * out = H^{(x)n} in, out of place, with the signs of the matrix elements
 * parsed on demand by the quadrant recursion of Fig. 3 (O(n) each) under one
 * of four sign-computation methods:
 *   MERA_RH_NONOPT   every element's sign             (2^n * 2^n signs)
 *   MERA_RH_QUARTER  Method 1, the upper-left quarter  (2^(n-1) * 2^(n-1))
 *   MERA_RH_BLOCK    Method 2, first block + one sign per other block of
 *                    `block` columns (0 = sqrt(2^(n-1)) rounded down to a
 *                    power of two, Theorem 3)     (2^(n-1) (2^(n-1)/b + b - 1))
 *   MERA_RH_LOG      Method 3 / Algorithm 1, signs at columns 2^p only
 *                                                   (2^(n-1) * (n - 1))
 * in and out: distinct complex128 states of the same n, 2 <= n <= 18 (the
 * method keeps a row's signs as bits in shared memory); `block` must be a
 * power of two <= min(256, 2^(n-1)) with 2^(n-1)/block <= 512.  Uses the
 * scratch memory of `out` (16 * 2^n + 256 bytes).  The MVM is O(4^n) work:
 * H^{(x)n} on a state is mera_hadamard_layer (butterflies, O(n 2^n)); these
 * calls exist to run the paper's methods as written.  Runs on out's stream
 * after in's queued work; with sign_count non-NULL, waits for the result
 * and stores the number of compute_sign evaluations (Table II). */
#define MERA_RH_NONOPT 0
#define MERA_RH_QUARTER 1
#define MERA_RH_BLOCK 2
#define MERA_RH_LOG 3
int mera_rh_mvm(mera_state* in, mera_state* out, int method, int block, uint64_t* sign_count);

/* ---- readouts (Sec. II-A Eq. 4-5); synchronous, float64 accumulation -- */

/* sum_i |a_i|^2 */
int mera_norm2(mera_state* s, double* out);
/* <Z_q> = sum_i (1 - 2 bit_q(i)) |a_i|^2 */
int mera_expect_z(mera_state* s, int q, double* out);
/* sum_q <Z_q> = sum_i (n - 2 popcount(i)) |a_i|^2 */
int mera_expect_z_sum(mera_state* s, double* out);
/* All three in one pass over the state: out[0] = norm^2, out[1] = <Z_q>,
 * out[2] = sum_q <Z_q>. */
int mera_observables(mera_state* s, int q, double out[3]);
/* Most probable index (|a|^2 = re*re + im*im, float64, no fused multiply-
 * add); ties go to the lowest index.  *prob may be NULL. */
int mera_argmax(mera_state* s, uint64_t* idx, double* prob);
/* Inverse-CDF sampling: for each u[j] in [0, 1) the smallest i with
 * C_i > u[j] * C_{N-1}, C the running sum of |a_i|^2.  u and idx_out are
 * host arrays of k elements. */
int mera_measure(mera_state* s, const double* u, size_t k, uint64_t* idx_out);

/* The same three sums as mera_observables, for callers that cannot let a
 * library allocate device memory: code whose framework's caching allocator
 * owns all device memory, or latency-critical loops that cannot afford the
 * device synchronisation cudaMalloc / cudaFree may cause.  The paper has no
 * counterpart; this is an interface convenience.
 *   dev_psi : device pointer to 2^n amplitudes of `dtype` (16-byte aligned),
 *             not modified; stream : cudaStream_t to run on (NULL = legacy
 *             default); out : host array of 3 doubles (norm^2, <Z_q>,
 *             sum_q <Z_q>).  Synchronous.
 * Nothing is allocated: the partial sums live in one fixed device array of
 * 3 * 1024 + 8 doubles (24.6 KB) that every GPU loading the library holds
 * until the process exits; n is limited to 1..MERA_MAX_QUBITS (larger n is
 * rejected with MERA_EINVAL).  The first call on a device looks up the
 * array's device address (make that first call before any stream capture).
 * All calls share the array and it keeps the last call's contents (each
 * call overwrites every partial it reads, so nothing needs clearing); calls
 * that overlap on the GPU, e.g. on two streams at once, race on it. */
int mera_observables_noalloc(const void* dev_psi, int n, int dtype, int q, void* stream, double out[3]);

/* ---- DAX / DAS compressed operation matrices (Sec. III-A) ---------------
 *
 * Device-resident, materialised forms of a 2^nq x 2^nq operation matrix:
 *   DAX (Sec. III-A.1, Fig. 1a): per non-zero a float64 (re, im) value and
 *       its row-major linear index row * 2^nq + col (uint64); entries in
 *       ascending index order.  24 bytes per entry (plus a derived row
 *       pointer of 2^nq + 1 uint64 used by the kernels).
 *   DAS (Sec. III-A.1, Fig. 1b): per non-zero a value and a uint64 distance
 *       word: bits 0..62 count the zeros since the previous non-zero of the
 *       same row (or the row start), bit 63 marks the last non-zero of its
 *       row.  Rows in order; every row needs at least one non-zero.
 * nq <= 32 (indices need 2 nq bits).  `stream` is a cudaStream_t (NULL =
 * legacy default); calls are asynchronous on it except the export and info
 * calls.
 * Objects are owned by the caller and freed with *_destroy. */
typedef struct mera_dax mera_dax;
typedef struct mera_das mera_das;

/* Encode a host dense matrix (interleaved complex128, row-major, 2^nq x
 * 2^nq, nq <= 12) by scanning it row by row. */
int mera_dax_from_dense(const double* m, int nq, void* stream, mera_dax** out);
int mera_das_from_dense(const double* m, int nq, void* stream, mera_das** out);
/* Upload host arrays as given (indices ascending / distance words in row
 * order; validated on the host). */
int mera_dax_from_host(int nq, uint64_t nnz, const uint64_t* index, const double* vals, void* stream,
                       mera_dax** out);
int mera_das_from_host(int nq, uint64_t nnz, const uint64_t* dist, const double* vals, void* stream,
                       mera_das** out);
/* MTP (Sec. III-A.2, Fig. 2): *out = a (x) b computed on the device.  DAX:
 * index = concatenated row bits * dim + concatenated column bits, value =
 * product; DAS: the paper's three-case distance equation.  The result has
 * nnz(a) * nnz(b) entries in row-major order. */
int mera_dax_kron(const mera_dax* a, const mera_dax* b, void* stream, mera_dax** out);
int mera_das_kron(const mera_das* a, const mera_das* b, void* stream, mera_das** out);
/* MVM (Sec. III-A.2): out = M in, out of place (in and out distinct states
 * of n = nq qubits, same dtype); runs on out's stream after in's work. */
int mera_dax_mvm(const mera_dax* d, mera_state* in, mera_state* out);
int mera_das_mvm(const mera_das* d, mera_state* in, mera_state* out);
/* Size queries (synchronous). */
int mera_dax_info(const mera_dax* d, int* nq, uint64_t* nnz);
int mera_das_info(const mera_das* d, int* nq, uint64_t* nnz);
/* Copy the entries to host arrays of nnz elements (vals: 2 nnz doubles).
 * Synchronous. */
int mera_dax_export(const mera_dax* d, uint64_t* index, double* vals);
int mera_das_export(const mera_das* d, uint64_t* dist, double* vals);
int mera_dax_destroy(mera_dax* d);
int mera_das_destroy(mera_das* d);

/* ---- batched QNN ansatz and adjoint gradients ----------------------------
 *
 * The hardware-efficient ansatz stands in for the paper's QNN neuron
 * (Sec. IV-D, Table III; its circuit figure is not reproducible): L layers,
 * each RY(theta[l][0][q]) then RZ(theta[l][1][q]) on every qubit q, then the
 * ring CNOT(q -> q+1 mod n) for q = 0..n-1.  A batch owns `capacity` states
 * ("slots") of n qubits (5 <= n <= 26), plus as many adjoint work states.
 * Rows of one call are independent: a slot's result does not depend on the
 * other slots of the call.  Angles are host arrays of float64; calls are
 * asynchronous on the batch's stream except *_observables and the
 * gradient.  Objects are freed with mera_batch_destroy. */
typedef struct mera_batch mera_batch;

int mera_batch_create(int n, int capacity, int dtype, void* stream, mera_batch** out);
int mera_batch_destroy(mera_batch* b);
/* Device pointer of the 2 * capacity states (slot s at s * 2^n; the
 * adjoint state of slot s at (capacity + s) * 2^n). */
int mera_batch_info(const mera_batch* b, void** dev_states, int* n, int* capacity, int* dtype);
int mera_batch_set_stream(mera_batch* b, void* stream);
/* Copy the state of slot `slot` (0 <= slot < 2 * capacity; adjoint states
 * from capacity on) to host memory of 2^n amplitudes.  Synchronous. */
int mera_batch_copy_to_host(mera_batch* b, int slot, void* host);
/* Set the listed slots (slots[nslots], NULL = 0..nslots-1) to |0...0>. */
int mera_batch_reset(mera_batch* b, const int* slots, int nslots);
/* One ansatz layer on each listed slot with its own angles:
 * theta[nslots][2][n] (row j: RY angles then RZ angles of slot slots[j]). */
int mera_batch_layer(mera_batch* b, const int* slots, int nslots, const double* theta);
/* Slots 0..nslots-1: reset, then L layers; theta[nslots][L][2][n]. */
int mera_batch_forward(mera_batch* b, int nslots, int L, const double* theta);
/* out[nslots][3] = (norm^2, <Z_q>, sum_q <Z_q>) per listed slot, float64
 * accumulation in the fixed order of mera_observables.  Synchronous. */
int mera_batch_observables(mera_batch* b, const int* slots, int nslots, int q, double* out);
/* Adjoint differentiation (reverse sweep with inverse gates) of
 * loss_b = sum_q <Z_q> of the ansatz on slots 0..nslots-1:
 * loss[nslots], grad[nslots][L][2][n] = d loss_b / d theta[b][l][g][q].
 * Runs the forward pass itself.  Synchronous. */
int mera_adjoint_grad(mera_batch* b, int nslots, int L, const double* theta, double* loss, double* grad);

/* ---- kernel timing ------------------------------------------------------ */

/* Kernel classes timed when profiling is on (one class per kernel family,
 * so that a workload's dominant kernel can be told apart). */
#define MERA_KCLASS_GATE 0      /* per-gate kernels not listed below (two- and three-target) */
#define MERA_KCLASS_TILE 1      /* general fused tile-pass kernel */
#define MERA_KCLASS_REDUCE 2    /* reductions */
#define MERA_KCLASS_DAX 3       /* DAX / DAS MTP and MVM kernels */
#define MERA_KCLASS_QNN 4       /* batched QNN / adjoint kernels */
#define MERA_KCLASS_HPASS 5     /* Hadamard-pass kernel (butterflies and sign terms) */
#define MERA_KCLASS_DPASS 6     /* streaming single-phase table-pass kernel */
#define MERA_KCLASS_GATE_DIAG 7 /* per-gate diagonal kernels (phases, sign flips) */
#define MERA_KCLASS_GATE_1Q 8   /* per-gate one-target kernels (2x2 and swaps with phases) */
#define MERA_KCLASS_RH 9        /* the paper's RH sign-method MVM kernels */
#define MERA_KCLASS_AMP 10      /* monomial run pass (permutation gather and diagonal tables) */
#define MERA_KCLASS_COUNT 11

/* Turn CUDA-event timing of every launch on/off (process-wide) and clear
 * the accumulated figures. */
int mera_profile_enable(int on);
/* Synchronise the recorded events and return, per kernel class, the number
 * of launches and their summed device time in ms (arrays of
 * MERA_KCLASS_COUNT; either may be NULL).  Also returns the summed
 * algorithmic bytes the timed launches moved (bytes may be NULL). */
int mera_profile_read(uint64_t* launches, double* ms, double* bytes);

/* Test hook for the bounded waits: every bulk-staged tile of later fused
 * launches expects `bytes` more than its copies deliver (a multiple of 16,
 * at most 4096), so that its wait runs out and the pass reports
 * MERA_ETIMEOUT.  0 (the default) restores normal operation.  Process-wide;
 * MERA_EINVAL for other values. */
int mera_test_bulk_shortfall(unsigned bytes);

#ifdef __cplusplus
}
#endif

#endif /* MERA_H */
