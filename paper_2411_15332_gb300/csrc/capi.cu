// C ABI entry points (mera.h), error reporting, launch accounting and the
// state object's lifetime.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"
#include "reduce.cuh"

namespace mera {

// ---------------------------------------------------------------- errors --
static thread_local std::string g_err;

void set_error(const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
}
const char* last_error() { return g_err.c_str(); }

// ------------------------------------------------------ launch accounting --
static std::atomic<uint64_t> g_launches{0};
static std::atomic<bool> g_prof{false};
static std::mutex g_prof_mu;
struct ProfRec {
    cudaEvent_t a, b;
    int kclass;
    double bytes;
};
static std::vector<ProfRec> g_pending;
static std::vector<cudaEvent_t> g_pool;
static uint64_t g_cnt[MERA_KCLASS_COUNT];
static double g_ms[MERA_KCLASS_COUNT];
static double g_bytes[MERA_KCLASS_COUNT];
static thread_local ProfRec t_cur;
static thread_local bool t_open = false;

static cudaEvent_t pool_get() {
    if (!g_pool.empty()) {
        cudaEvent_t e = g_pool.back();
        g_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

void launch_begin(cudaStream_t st, int kclass, double bytes) {
    g_launches.fetch_add(1, std::memory_order_relaxed);
    t_open = false;
    if (!g_prof.load(std::memory_order_relaxed)) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    t_cur.a = pool_get();
    t_cur.b = pool_get();
    t_cur.kclass = kclass;
    t_cur.bytes = bytes;
    if (t_cur.a && t_cur.b && cudaEventRecord(t_cur.a, st) == cudaSuccess) t_open = true;
}

int launch_end(cudaStream_t st) {
    cudaError_t e = cudaGetLastError();
    if (t_open) {
        t_open = false;
        std::lock_guard<std::mutex> lk(g_prof_mu);
        cudaEventRecord(t_cur.b, st);
        g_pending.push_back(t_cur);
    }
    if (e != cudaSuccess) {
        set_error("kernel launch failed: %s", cudaGetErrorString(e));
        return MERA_ECUDA;
    }
    return MERA_OK;
}

static int profile_collect() {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    for (auto& r : g_pending) {
        cudaError_t e = cudaEventSynchronize(r.b);
        if (e != cudaSuccess) {
            set_error("cudaEventSynchronize: %s", cudaGetErrorString(e));
            return MERA_ECUDA;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, r.a, r.b);
        g_cnt[r.kclass] += 1;
        g_ms[r.kclass] += ms;
        g_bytes[r.kclass] += r.bytes;
        g_pool.push_back(r.a);
        g_pool.push_back(r.b);
    }
    g_pending.clear();
    return MERA_OK;
}

// ----------------------------------------------------------------- state --
int state_ensure_scratch(mera_state* s, size_t bytes) {
    if (s->scratch_bytes >= bytes) return MERA_OK;
    size_t want = 64 * 1024;
    while (want < bytes) want *= 2;
    if (s->scratch) {
        // the stream may still use the old buffer
        MERA_CHECK_CUDA(cudaStreamSynchronize(s->stream));
        cudaFree(s->scratch);
        s->scratch = nullptr;
        s->scratch_bytes = 0;
    }
    cudaError_t e = cudaMalloc(&s->scratch, want);
    if (e != cudaSuccess) {
        set_error("cudaMalloc(%zu) for scratch: %s", want, cudaGetErrorString(e));
        return MERA_ENOMEM;
    }
    s->scratch_bytes = want;
    return MERA_OK;
}

int state_wait_flag(mera_state* s, int** flag) {
    if (!s->wait_flag) {
        MERA_CHECK_CUDA(cudaMalloc(&s->wait_flag, 256));
        MERA_CHECK_CUDA(cudaMemsetAsync(s->wait_flag, 0, sizeof(int), s->stream));
        MERA_CHECK_CUDA(cudaHostAlloc(&s->wait_host, sizeof(int), cudaHostAllocDefault));
        *s->wait_host = 0;
    }
    *flag = s->wait_flag;
    return MERA_OK;
}

int state_check_waits(mera_state* s) {
    if (!s->wait_host || *s->wait_host == 0) return MERA_OK;
    *s->wait_host = 0;
    MERA_CHECK_CUDA(cudaMemsetAsync(s->wait_flag, 0, sizeof(int), s->stream));
    set_error("a bounded wait for a staged tile copy ran out; the state's amplitudes are not valid");
    return MERA_ETIMEOUT;
}

template <typename V>
__global__ void k_set_one(V* psi, uint64_t i) {
    V one;
    one.x = 1;
    one.y = 0;
    psi[i] = one;
}

static int set_basis(mera_state* s, uint64_t index) {
    MERA_RETURN_IF(index >= num_amps(s), MERA_EINVAL, "basis index out of range");
    const size_t bytes = num_amps(s) * elem_bytes(s->dtype);
    MERA_CHECK_CUDA(cudaMemsetAsync(s->data, 0, bytes, s->stream));
    launch_begin(s->stream, MERA_KCLASS_GATE, (double)elem_bytes(s->dtype));
    if (s->dtype == MERA_C128) k_set_one<double2><<<1, 1, 0, s->stream>>>((double2*)s->data, index);
    else k_set_one<float2><<<1, 1, 0, s->stream>>>((float2*)s->data, index);
    return launch_end(s->stream);
}

static int check_state(const mera_state* s) {
    MERA_RETURN_IF(s == nullptr || s->data == nullptr, MERA_EINVAL, "state is NULL");
    return MERA_OK;
}

static int to_mask(const int* qs, int nq, int n, uint64_t* mask) {
    *mask = 0;
    MERA_RETURN_IF(nq < 0 || nq > n, MERA_EINVAL, "bad qubit count %d", nq);
    MERA_RETURN_IF(nq > 0 && qs == nullptr, MERA_EINVAL, "qubit list is NULL");
    for (int j = 0; j < nq; ++j) {
        MERA_RETURN_IF(qs[j] < 0 || qs[j] >= n, MERA_EINVAL, "qubit %d out of range for n=%d", qs[j], n);
        MERA_RETURN_IF((*mask >> qs[j]) & 1ull, MERA_EINVAL, "qubit %d listed twice", qs[j]);
        *mask |= 1ull << qs[j];
    }
    return MERA_OK;
}

}  // namespace mera

using namespace mera;

#define API_BEGIN try {
#define API_END                                                   \
    }                                                             \
    catch (const std::bad_alloc&) {                               \
        set_error("host allocation failed");                      \
        return MERA_ENOMEM;                                       \
    }                                                             \
    catch (...) {                                                 \
        set_error("unexpected C++ exception");                    \
        return MERA_EINVAL;                                       \
    }

extern "C" {

const char* mera_last_error(void) { return last_error(); }
const char* mera_version(void) { return "mera-gb300 0.1 (sm_103a)"; }
uint64_t mera_launch_count(void) { return g_launches.load(); }

int mera_state_create(int n, int dtype, mera_state** out) {
    API_BEGIN
    MERA_RETURN_IF(out == nullptr, MERA_EINVAL, "out is NULL");
    *out = nullptr;
    MERA_RETURN_IF(n < 1 || n > MERA_MAX_QUBITS, MERA_EINVAL, "n=%d outside [1, %d]", n, MERA_MAX_QUBITS);
    MERA_RETURN_IF(dtype != MERA_C64 && dtype != MERA_C128, MERA_EUNSUPPORTED, "unknown dtype %d", dtype);
    mera_state* s = new mera_state();
    s->n = n;
    s->dtype = dtype;
    s->owns = true;
    cudaGetDevice(&s->device);
    const size_t bytes = (1ull << n) * elem_bytes(dtype);
    cudaError_t e = cudaMalloc(&s->data, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete s;
        set_error("cudaMalloc(%zu) for the state: %s", bytes, cudaGetErrorString(e));
        return MERA_ENOMEM;
    }
    int st = set_basis(s, 0);
    if (st == MERA_OK) st = state_ensure_scratch(s, 64 * 1024);
    if (st != MERA_OK) {
        cudaFree(s->data);
        delete s;
        return st;
    }
    *out = s;
    return MERA_OK;
    API_END
}

int mera_state_wrap(void* dev_ptr, int n, int dtype, void* stream, mera_state** out) {
    API_BEGIN
    MERA_RETURN_IF(out == nullptr, MERA_EINVAL, "out is NULL");
    *out = nullptr;
    MERA_RETURN_IF(dev_ptr == nullptr, MERA_EINVAL, "dev_ptr is NULL");
    MERA_RETURN_IF(((uintptr_t)dev_ptr & 15) != 0, MERA_EINVAL, "dev_ptr must be 16-byte aligned");
    MERA_RETURN_IF(n < 1 || n > MERA_MAX_QUBITS, MERA_EINVAL, "n=%d outside [1, %d]", n, MERA_MAX_QUBITS);
    MERA_RETURN_IF(dtype != MERA_C64 && dtype != MERA_C128, MERA_EUNSUPPORTED, "unknown dtype %d", dtype);
    mera_state* s = new mera_state();
    s->data = dev_ptr;
    s->n = n;
    s->dtype = dtype;
    s->owns = false;
    s->stream = (cudaStream_t)stream;
    cudaGetDevice(&s->device);
    int st = state_ensure_scratch(s, 64 * 1024);
    if (st != MERA_OK) {
        delete s;
        return st;
    }
    *out = s;
    return MERA_OK;
    API_END
}

int mera_state_destroy(mera_state* s) {
    API_BEGIN
    if (!s) return MERA_OK;
    cudaStreamSynchronize(s->stream);
    if (s->owns && s->data) cudaFree(s->data);
    if (s->scratch) cudaFree(s->scratch);
    if (s->prog) cudaFree(s->prog);
    if (s->prog_host) cudaFreeHost(s->prog_host);
    fused_cache_free(s);
    if (s->pong) cudaFree(s->pong);
    if (s->wait_flag) cudaFree(s->wait_flag);
    if (s->wait_host) cudaFreeHost(s->wait_host);
    delete s;
    return MERA_OK;
    API_END
}

int mera_state_set_stream(mera_state* s, void* stream) {
    MERA_TRY(check_state(s));
    s->stream = (cudaStream_t)stream;
    return MERA_OK;
}

int mera_state_info(const mera_state* s, void** dev_ptr, int* n, int* dtype) {
    MERA_TRY(check_state(s));
    if (dev_ptr) *dev_ptr = s->data;
    if (n) *n = s->n;
    if (dtype) *dtype = s->dtype;
    return MERA_OK;
}

int mera_state_set_basis(mera_state* s, uint64_t index) {
    API_BEGIN
    MERA_TRY(check_state(s));
    return set_basis(s, index);
    API_END
}

int mera_state_copy_from_host(mera_state* s, const void* host) {
    API_BEGIN
    MERA_TRY(check_state(s));
    MERA_RETURN_IF(host == nullptr, MERA_EINVAL, "host is NULL");
    MERA_CHECK_CUDA(cudaMemcpyAsync(s->data, host, num_amps(s) * elem_bytes(s->dtype), cudaMemcpyHostToDevice, s->stream));
    MERA_CHECK_CUDA(cudaStreamSynchronize(s->stream));
    return MERA_OK;
    API_END
}

int mera_state_copy_from_host_async(mera_state* s, const void* host) {
    API_BEGIN
    MERA_TRY(check_state(s));
    MERA_RETURN_IF(host == nullptr, MERA_EINVAL, "host is NULL");
    MERA_CHECK_CUDA(cudaMemcpyAsync(s->data, host, num_amps(s) * elem_bytes(s->dtype), cudaMemcpyHostToDevice, s->stream));
    return MERA_OK;
    API_END
}

int mera_state_copy_to_host(mera_state* s, void* host) {
    API_BEGIN
    MERA_TRY(check_state(s));
    MERA_RETURN_IF(host == nullptr, MERA_EINVAL, "host is NULL");
    MERA_CHECK_CUDA(cudaMemcpyAsync(host, s->data, num_amps(s) * elem_bytes(s->dtype), cudaMemcpyDeviceToHost, s->stream));
    MERA_CHECK_CUDA(cudaStreamSynchronize(s->stream));
    return state_check_waits(s);
    API_END
}

int mera_state_get_amplitudes(mera_state* s, const uint64_t* idx, size_t k, double* out) {
    API_BEGIN
    MERA_TRY(check_state(s));
    MERA_RETURN_IF(k > 0 && (idx == nullptr || out == nullptr), MERA_EINVAL, "NULL array");
    return gather(s, idx, k, out);
    API_END
}

int mera_state_synchronize(mera_state* s) {
    MERA_TRY(check_state(s));
    MERA_CHECK_CUDA(cudaStreamSynchronize(s->stream));
    return state_check_waits(s);
}

int mera_gate_matrix(int gate, const double* params, int* nt, double* out) {
    API_BEGIN
    MERA_RETURN_IF(nt == nullptr || out == nullptr, MERA_EINVAL, "NULL argument");
    MERA_RETURN_IF(gate == MERA_GATE_MATRIX, MERA_EINVAL, "MERA_GATE_MATRIX has no catalogue matrix");
    cplx m[64];
    MERA_TRY(gate_matrix(gate, params, nt, m));
    const int d = 1 << *nt;
    for (int j = 0; j < d * d; ++j) {
        out[2 * j] = m[j].real();
        out[2 * j + 1] = m[j].imag();
    }
    return MERA_OK;
    API_END
}

int mera_apply_gate(mera_state* s, int gate, const int* targets, int nt, const int* controls, int nc,
                    const double* params) {
    API_BEGIN
    MERA_TRY(check_state(s));
    MERA_RETURN_IF(nt < 0 || nt > 3, MERA_EUNSUPPORTED, "nt=%d not in 0..3", nt);
    MERA_RETURN_IF(nt > 0 && targets == nullptr, MERA_EINVAL, "targets is NULL");
    mera_op op;
    memset(&op, 0, sizeof(op));
    op.gate = gate;
    op.nt = nt;
    for (int j = 0; j < nt; ++j) op.targets[j] = targets[j];
    MERA_TRY(to_mask(controls, nc, s->n, &op.cmask));
    op.cvals = op.cmask;
    if (gate != MERA_GATE_MATRIX && gate >= 0 && gate < MERA_GATE_COUNT) {
        // copy exactly the parameters the gate takes
        static const int npar[MERA_GATE_COUNT] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, 1, 1, 1, 2, 2, 4,
                                                  0, 0, 0, 0, 1, 1, 1, 1, 0, 0};
        MERA_RETURN_IF(npar[gate] > 0 && params == nullptr, MERA_EINVAL, "gate %d needs params", gate);
        for (int j = 0; j < npar[gate]; ++j) op.params[j] = params[j];
    }
    PrepOp P;
    MERA_TRY(prepare_op(op, s->n, &P));
    return apply_prepared(s, P);
    API_END
}

int mera_apply_matrix(mera_state* s, const double* matrix, const int* targets, int nt, const int* controls, int nc) {
    API_BEGIN
    MERA_TRY(check_state(s));
    MERA_RETURN_IF(nt < 1 || nt > 3, MERA_EUNSUPPORTED, "nt=%d not in 1..3", nt);
    MERA_RETURN_IF(targets == nullptr || matrix == nullptr, MERA_EINVAL, "NULL argument");
    mera_op op;
    memset(&op, 0, sizeof(op));
    op.gate = MERA_GATE_MATRIX;
    op.nt = nt;
    for (int j = 0; j < nt; ++j) op.targets[j] = targets[j];
    op.matrix = matrix;
    MERA_TRY(to_mask(controls, nc, s->n, &op.cmask));
    op.cvals = op.cmask;
    PrepOp P;
    MERA_TRY(prepare_op(op, s->n, &P));
    return apply_prepared(s, P);
    API_END
}

int mera_apply_circuit(mera_state* s, const mera_op* ops, size_t nops, int mode) {
    API_BEGIN
    MERA_TRY(check_state(s));
    MERA_RETURN_IF(nops > 0 && ops == nullptr, MERA_EINVAL, "ops is NULL");
    MERA_RETURN_IF(mode != MERA_MODE_PER_GATE && mode != MERA_MODE_FUSED, MERA_EINVAL, "unknown mode %d", mode);
    if (mode == MERA_MODE_FUSED) return apply_fused_circuit(s, ops, nops);
    std::vector<PrepOp> prep(nops);
    for (size_t j = 0; j < nops; ++j) {
        int st = prepare_op(ops[j], s->n, &prep[j]);
        if (st != MERA_OK) {
            std::string msg = last_error();
            set_error("op %zu: %s", j, msg.c_str());
            return st;
        }
    }
    for (const PrepOp& P : prep) MERA_TRY(apply_prepared(s, P));
    return MERA_OK;
    API_END
}

int mera_apply_circuit_observe(mera_state* s, const mera_op* ops, size_t nops, int mode, int q, double out[3]) {
    API_BEGIN
    MERA_TRY(check_state(s));
    MERA_RETURN_IF(nops > 0 && ops == nullptr, MERA_EINVAL, "ops is NULL");
    MERA_RETURN_IF(out == nullptr, MERA_EINVAL, "out is NULL");
    MERA_RETURN_IF(q < 0 || q >= s->n, MERA_EINVAL, "qubit %d out of range", q);
    MERA_RETURN_IF(mode != MERA_MODE_PER_GATE && mode != MERA_MODE_FUSED, MERA_EINVAL, "unknown mode %d", mode);
    if (mode == MERA_MODE_FUSED) return apply_fused_circuit_observe(s, ops, nops, q, out);
    MERA_TRY(mera_apply_circuit(s, ops, nops, mode));
    return observables(s, q, out);
    API_END
}

int mera_plan_summary(int n, int dtype, const mera_op* ops, size_t nops, char* out, size_t cap, int* npasses) {
    API_BEGIN
    MERA_RETURN_IF(n < 5 || n > MERA_MAX_QUBITS, MERA_EINVAL, "n=%d outside [5, %d] for the fused path", n,
                   MERA_MAX_QUBITS);
    MERA_RETURN_IF(dtype != MERA_C64 && dtype != MERA_C128, MERA_EUNSUPPORTED, "unknown dtype %d", dtype);
    MERA_RETURN_IF(nops > 0 && ops == nullptr, MERA_EINVAL, "ops is NULL");
    std::vector<PrepOp> prep(nops);
    for (size_t j = 0; j < nops; ++j) MERA_TRY(prepare_op(ops[j], n, &prep[j]));
    std::string s;
    MERA_TRY(plan_summary(n, dtype, prep, &s, npasses));
    if (out && cap > 0) {
        const size_t m = std::min(cap - 1, s.size());
        memcpy(out, s.data(), m);
        out[m] = 0;
    }
    return MERA_OK;
    API_END
}

int mera_hadamard_layer(mera_state* s, uint64_t mask) {
    API_BEGIN
    MERA_TRY(check_state(s));
    MERA_RETURN_IF(s->n < 64 && (mask >> s->n) != 0, MERA_EINVAL, "mask names a qubit >= n");
    std::vector<PrepOp> prep;
    for (int q = 0; q < s->n; ++q) {
        if (!((mask >> q) & 1ull)) continue;
        mera_op op;
        memset(&op, 0, sizeof(op));
        op.gate = MERA_GATE_H;
        op.nt = 1;
        op.targets[0] = q;
        prep.emplace_back();
        MERA_TRY(prepare_op(op, s->n, &prep.back()));
    }
    return apply_fused(s, prep);
    API_END
}

int mera_norm2(mera_state* s, double* out) {
    API_BEGIN
    MERA_TRY(check_state(s));
    MERA_RETURN_IF(out == nullptr, MERA_EINVAL, "out is NULL");
    double r[3];
    MERA_TRY(observables(s, 0, r));
    *out = r[0];
    return MERA_OK;
    API_END
}

int mera_expect_z(mera_state* s, int q, double* out) {
    API_BEGIN
    MERA_TRY(check_state(s));
    MERA_RETURN_IF(out == nullptr, MERA_EINVAL, "out is NULL");
    MERA_RETURN_IF(q < 0 || q >= s->n, MERA_EINVAL, "qubit %d out of range", q);
    double r[3];
    MERA_TRY(observables(s, q, r));
    *out = r[1];
    return MERA_OK;
    API_END
}

int mera_expect_z_sum(mera_state* s, double* out) {
    API_BEGIN
    MERA_TRY(check_state(s));
    MERA_RETURN_IF(out == nullptr, MERA_EINVAL, "out is NULL");
    double r[3];
    MERA_TRY(observables(s, 0, r));
    *out = r[2];
    return MERA_OK;
    API_END
}

int mera_observables(mera_state* s, int q, double out[3]) {
    API_BEGIN
    MERA_TRY(check_state(s));
    MERA_RETURN_IF(out == nullptr, MERA_EINVAL, "out is NULL");
    MERA_RETURN_IF(q < 0 || q >= s->n, MERA_EINVAL, "qubit %d out of range", q);
    return observables(s, q, out);
    API_END
}

int mera_argmax(mera_state* s, uint64_t* idx, double* prob) {
    API_BEGIN
    MERA_TRY(check_state(s));
    MERA_RETURN_IF(idx == nullptr, MERA_EINVAL, "idx is NULL");
    return argmax(s, idx, prob);
    API_END
}

int mera_measure(mera_state* s, const double* u, size_t k, uint64_t* idx_out) {
    API_BEGIN
    MERA_TRY(check_state(s));
    MERA_RETURN_IF(k > 0 && (u == nullptr || idx_out == nullptr), MERA_EINVAL, "NULL array");
    return measure(s, u, k, idx_out);
    API_END
}

int mera_test_bulk_shortfall(unsigned bytes) {
    API_BEGIN
    MERA_RETURN_IF(bytes % 16 != 0 || bytes > 4096, MERA_EINVAL, "shortfall %u: a multiple of 16 up to 4096", bytes);
    fused_set_bulk_shortfall(bytes);
    return MERA_OK;
    API_END
}

int mera_profile_enable(int on) {
    API_BEGIN
    MERA_TRY(profile_collect());
    std::lock_guard<std::mutex> lk(g_prof_mu);
    for (int c = 0; c < MERA_KCLASS_COUNT; ++c) {
        g_cnt[c] = 0;
        g_ms[c] = 0;
        g_bytes[c] = 0;
    }
    g_prof.store(on != 0);
    return MERA_OK;
    API_END
}

int mera_profile_read(uint64_t* launches, double* ms, double* bytes) {
    API_BEGIN
    MERA_TRY(profile_collect());
    std::lock_guard<std::mutex> lk(g_prof_mu);
    for (int c = 0; c < MERA_KCLASS_COUNT; ++c) {
        if (launches) launches[c] = g_cnt[c];
        if (ms) ms[c] = g_ms[c];
        if (bytes) bytes[c] = g_bytes[c];
    }
    return MERA_OK;
    API_END
}

}  // extern "C"
