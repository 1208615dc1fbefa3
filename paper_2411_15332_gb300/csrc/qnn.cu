// Batched QNN ansatz states, their expectations and adjoint gradients.
//
// Ansatz (the QNN workload): L layers, each RY(theta[l][0][q]) then
// RZ(theta[l][1][q]) on every qubit q, then the ring CNOT(q -> q+1 mod n)
// for q = 0..n-1.  A batch holds `capacity` states ("slots") of n qubits,
// contiguous; a second block of `capacity` states holds the adjoint states.
//
// Forward: per qubit the two rotations are one 2x2 matrix RZ(b) RY(a); one
// layer for a list of slots is the fused tile plan of
// [n per-slot 2x2 gates, CNOT ring] launched with one batch row per slot,
// so slots at different layers of different circuits advance together.
//
// Adjoint differentiation (reverse sweep with inverse gates): with
// psi = U|0>, lambda = O psi (O = sum_q Z_q) and, for gates g = G..1,
//   grad_g = 2 Re <lambda| dU_g/dtheta |psi_{g-1}>,
// the rotations RZ, RY have dU/dtheta = (-i/2) P U (P = Z, Y), so
//   grad_g = Im <lambda_g| P_q |psi_g>
// with both states taken after gate g, before it is undone.  Each rotation
// step evaluates that inner product and undoes the gate on both states in
// one pass; block partial sums are reduced in a fixed order per slot, so a
// slot's result does not depend on the other slots in the batch.
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "fused.cuh"
#include "kernels.cuh"
#include "reduce.cuh"

struct mera_batch {
    int n = 0, cap = 0, dtype = MERA_C64;
    cudaStream_t stream = nullptr;
    void* states = nullptr;        // 2 * cap states: slots, then adjoint slots
    void* coef = nullptr;          // per-row coefficients of one launch
    size_t coef_bytes = 0;
    int* dslots = nullptr;         // slot lists of one launch (3 * cap)
    double* dang = nullptr;        // per-row rotation cosines / sines (adjoint)
    size_t dang_bytes = 0;
    double* partial = nullptr;     // reduction partials
    size_t partial_bytes = 0;
    double* dres = nullptr;        // reduction results
    size_t dres_bytes = 0;
    void* layer_plan = nullptr;    // FusedPlan<V>* of one layer
    void* ring_inv_plan = nullptr; // FusedPlan<V>* of the inverse CNOT ring
};

namespace mera {

static constexpr int ADJ_BLOCKS = 16;   // blocks per state in the adjoint steps

template <typename T>
static int grow(T** p, size_t* have, size_t need) {
    if (*have >= need) return MERA_OK;
    if (*p) cudaFree(*p);
    *p = nullptr;
    *have = 0;
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), need);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error("cudaMalloc(%zu): %s", need, cudaGetErrorString(e));
        return MERA_ENOMEM;
    }
    *have = need;
    return MERA_OK;
}

static int prep(int gate, int target, uint64_t cmask, int n, PrepOp* out) {
    mera_op op;
    memset(&op, 0, sizeof(op));
    op.gate = gate;
    op.nt = 1;
    op.targets[0] = target;
    op.cmask = cmask;
    op.cvals = cmask;
    return prepare_op(op, n, out);
}

// One layer: n per-slot 2x2 gates then the CNOT ring.
static int layer_ops(int n, std::vector<PrepOp>& ops) {
    ops.clear();
    for (int q = 0; q < n; ++q) {
        PrepOp P;
        MERA_TRY(prep(MERA_GATE_H, q, 0, n, &P));   // placeholder matrix, replaced per slot
        P.kind = KIND_DENSE;
        P.is_h = false;
        P.bslot = q;
        ops.push_back(P);
    }
    for (int q = 0; q < n; ++q) {
        PrepOp P;
        MERA_TRY(prep(MERA_GATE_X, (q + 1) % n, 1ull << q, n, &P));
        ops.push_back(P);
    }
    return MERA_OK;
}

// Inverse of the ring: the same CNOTs in reverse order.
static int ring_inverse_ops(int n, std::vector<PrepOp>& ops) {
    ops.clear();
    for (int q = n - 1; q >= 0; --q) {
        PrepOp P;
        MERA_TRY(prep(MERA_GATE_X, (q + 1) % n, 1ull << q, n, &P));
        ops.push_back(P);
    }
    return MERA_OK;
}

template <typename V>
static V mk(double re, double im) {
    V r;
    r.x = (decltype(r.x))re;
    r.y = (decltype(r.y))im;
    return r;
}

// A coefficient for the tile passes: plain values, or for the int64 engine
// each part as round(value * 2^61) split into 31-bit limbs h * 2^31 + l
// (int32 h, l for the real part, then for the imaginary part; the same 16
// bytes).
template <typename V>
static V mkq(double re, double im, bool q61) {
    if (!q61 || sizeof(V) != 16) return mk<V>(re, im);
    const double sc = 2305843009213693952.0;   // 2^61
    const long long r = std::llround(re * sc), i = std::llround(im * sc);
    const int32_t w[4] = {(int32_t)(r >> 31), (int32_t)(r & 0x7FFFFFFF), (int32_t)(i >> 31),
                          (int32_t)(i & 0x7FFFFFFF)};
    V v;
    memcpy(&v, w, sizeof(v));
    return v;
}

// ---------------------------------------------------------------- kernels --
template <typename V>
__global__ void k_batch_zero(V* states, const int* slots, uint64_t N) {
    V* psi = states + (uint64_t)slots[blockIdx.y] * N;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (uint64_t)gridDim.x * blockDim.x) {
        V z;
        z.x = (i == 0) ? 1 : 0;
        z.y = 0;
        psi[i] = z;
    }
}

__device__ __forceinline__ double bwarp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Fixed-order block sum of k values (k <= 3), result in thread 0.
template <int KV>
__device__ __forceinline__ void bsum(double (&v)[KV]) {
    __shared__ double sh[KV][8];
#pragma unroll
    for (int j = 0; j < KV; ++j) v[j] = bwarp_sum(v[j]);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0)
#pragma unroll
        for (int j = 0; j < KV; ++j) sh[j][w] = v[j];
    __syncthreads();
    if (w == 0) {
#pragma unroll
        for (int j = 0; j < KV; ++j) {
            v[j] = l < (int)(blockDim.x >> 5) ? sh[j][l] : 0.0;
            v[j] = bwarp_sum(v[j]);
        }
    }
}

__device__ __forceinline__ double prob_d(double2 a) { return __dadd_rn(__dmul_rn(a.x, a.x), __dmul_rn(a.y, a.y)); }
__device__ __forceinline__ double prob_d(float2 a) {
    const double x = a.x, y = a.y;
    return __dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y));
}

// Same partition and order as the single-state reduction (reduce.cu).
template <typename V>
__global__ void __launch_bounds__(256) k_batch_obs(const V* __restrict__ states, const int* __restrict__ slots, int n,
                                                   uint64_t chunk, int q, double* __restrict__ partial) {
    const uint64_t N = 1ull << n;
    const V* psi = states + (uint64_t)slots[blockIdx.y] * N;
    const uint64_t lo = (uint64_t)blockIdx.x * chunk;
    double s[3] = {0.0, 0.0, 0.0};
    for (uint64_t i = lo + threadIdx.x; i < lo + chunk; i += blockDim.x) {
        const double p = prob_d(psi[i]);
        s[0] += p;
        s[1] += ((i >> q) & 1ull) ? -p : p;
        s[2] += (double)(n - 2 * __popcll(i)) * p;
    }
    bsum<3>(s);
    if (threadIdx.x == 0) {
        double* o = partial + ((size_t)blockIdx.y * gridDim.x + blockIdx.x) * 3;
        o[0] = s[0];
        o[1] = s[1];
        o[2] = s[2];
    }
}

__global__ void __launch_bounds__(256) k_batch_obs_finish(const double* __restrict__ partial, int nb,
                                                          double* __restrict__ out) {
    const double* p = partial + (size_t)blockIdx.x * nb * 3;
    double s[3] = {0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
        s[0] += p[3 * b + 0];
        s[1] += p[3 * b + 1];
        s[2] += p[3 * b + 2];
    }
    bsum<3>(s);
    if (threadIdx.x == 0) {
        out[3 * blockIdx.x + 0] = s[0];
        out[3 * blockIdx.x + 1] = s[1];
        out[3 * blockIdx.x + 2] = s[2];
    }
}

// lambda = (sum_q Z_q) psi: lambda_i = (n - 2 popcount(i)) psi_i.
template <typename V>
__global__ void k_adj_init(V* states, const int* slots, int nrows, int cap, int n) {
    const uint64_t N = 1ull << n;
    const V* psi = states + (uint64_t)slots[blockIdx.y] * N;
    V* lam = states + (uint64_t)(slots[blockIdx.y] + cap) * N;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (uint64_t)gridDim.x * blockDim.x) {
        const V a = psi[i];
        const float w = (float)(n - 2 * __popcll(i));
        V r;
        r.x = (decltype(r.x))(w * a.x);
        r.y = (decltype(r.y))(w * a.y);
        lam[i] = r;
    }
}

// Gradient of RZ_q at the current point, then undo RZ_q on both states.
// ang[row][q] = (cos(b/2), sin(b/2)); RZ^dagger = diag(e^{ib/2}, e^{-ib/2}).
template <typename V>
__global__ void __launch_bounds__(256) k_adj_rz(V* states, const int* slots, int cap, int n, int q,
                                                const double* __restrict__ ang, double* __restrict__ partial) {
    const uint64_t N = 1ull << n;
    const int row = blockIdx.y;
    V* psi = states + (uint64_t)slots[row] * N;
    V* lam = states + (uint64_t)(slots[row] + cap) * N;
    const double c = ang[((size_t)row * n + q) * 2 + 0], s = ang[((size_t)row * n + q) * 2 + 1];
    const uint64_t chunk = N / gridDim.x;
    const uint64_t lo = (uint64_t)blockIdx.x * chunk;
    double acc[1] = {0.0};
    for (uint64_t i = lo + threadIdx.x; i < lo + chunk; i += blockDim.x) {
        const V a = psi[i], l = lam[i];
        const double im = (double)l.x * (double)a.y - (double)l.y * (double)a.x;
        const bool one = (i >> q) & 1ull;
        acc[0] += one ? -im : im;
        // multiply by e^{+ib/2} (bit 0) or e^{-ib/2} (bit 1)
        const double sg = one ? -s : s;
        V a2, l2;
        a2.x = (decltype(a2.x))(c * a.x - sg * a.y);
        a2.y = (decltype(a2.y))(c * a.y + sg * a.x);
        l2.x = (decltype(l2.x))(c * l.x - sg * l.y);
        l2.y = (decltype(l2.y))(c * l.y + sg * l.x);
        psi[i] = a2;
        lam[i] = l2;
    }
    bsum<1>(acc);
    if (threadIdx.x == 0) partial[(size_t)row * gridDim.x + blockIdx.x] = acc[0];
}

// Gradient of RY_q, then undo RY_q: RY^dagger = [[c, s], [-s, c]].
template <typename V>
__global__ void __launch_bounds__(256) k_adj_ry(V* states, const int* slots, int cap, int n, int q,
                                                const double* __restrict__ ang, double* __restrict__ partial) {
    const uint64_t N = 1ull << n, half = N >> 1;
    const int row = blockIdx.y;
    V* psi = states + (uint64_t)slots[row] * N;
    V* lam = states + (uint64_t)(slots[row] + cap) * N;
    const double c = ang[((size_t)row * n + q) * 2 + 0], s = ang[((size_t)row * n + q) * 2 + 1];
    const uint64_t chunk = half / gridDim.x;
    const uint64_t lo = (uint64_t)blockIdx.x * chunk;
    const uint64_t low = (1ull << q) - 1ull;
    double acc[1] = {0.0};
    for (uint64_t t = lo + threadIdx.x; t < lo + chunk; t += blockDim.x) {
        const uint64_t i0 = ((t & ~low) << 1) | (t & low), i1 = i0 | (1ull << q);
        const V a0 = psi[i0], a1 = psi[i1], l0 = lam[i0], l1 = lam[i1];
        acc[0] += ((double)l1.x * a0.x + (double)l1.y * a0.y) - ((double)l0.x * a1.x + (double)l0.y * a1.y);
        V b0, b1, m0, m1;
        b0.x = (decltype(b0.x))(c * a0.x + s * a1.x);
        b0.y = (decltype(b0.y))(c * a0.y + s * a1.y);
        b1.x = (decltype(b1.x))(c * a1.x - s * a0.x);
        b1.y = (decltype(b1.y))(c * a1.y - s * a0.y);
        m0.x = (decltype(m0.x))(c * l0.x + s * l1.x);
        m0.y = (decltype(m0.y))(c * l0.y + s * l1.y);
        m1.x = (decltype(m1.x))(c * l1.x - s * l0.x);
        m1.y = (decltype(m1.y))(c * l1.y - s * l0.y);
        psi[i0] = b0;
        psi[i1] = b1;
        lam[i0] = m0;
        lam[i1] = m1;
    }
    bsum<1>(acc);
    if (threadIdx.x == 0) partial[(size_t)row * gridDim.x + blockIdx.x] = acc[0];
}

// grad[row][p] = sum over the blocks of partial[p][row][*] (fixed order).
__global__ void k_adj_finish(const double* __restrict__ partial, int nrows, int nparams, int nb, double* __restrict__ grad) {
    const int row = blockIdx.x;
    for (int p = threadIdx.x; p < nparams; p += blockDim.x) {
        const double* src = partial + ((size_t)p * nrows + row) * nb;
        double s = 0.0;
        for (int b = 0; b < nb; ++b) s += src[b];
        grad[(size_t)row * nparams + p] = s;
    }
}

// ------------------------------------------------------------- host side --
static int upload_slots(mera_batch* b, const int* slots, int nslots, int offset) {
    MERA_RETURN_IF(nslots < 1 || nslots > b->cap, MERA_EINVAL, "%d slots for a batch of %d", nslots, b->cap);
    std::vector<int> tmp(nslots);
    for (int j = 0; j < nslots; ++j) {
        const int s = slots ? slots[j] : j;
        MERA_RETURN_IF(s < 0 || s >= b->cap, MERA_EINVAL, "slot %d out of range", s);
        tmp[j] = s;
    }
    MERA_CHECK_CUDA(cudaMemcpyAsync(b->dslots + offset, tmp.data(), nslots * sizeof(int), cudaMemcpyHostToDevice,
                                    b->stream));
    return MERA_OK;
}

template <typename V>
static int batch_layer_t(mera_batch* b, const int* slots, int nslots, const double* theta) {
    const int n = b->n;
    FusedPlan<V>* plan = reinterpret_cast<FusedPlan<V>*>(b->layer_plan);
    if (!plan) {
        plan = new FusedPlan<V>();
        std::vector<PrepOp> ops;
        int st = layer_ops(n, ops);
        if (st == MERA_OK) st = fused_build<V>(n, ops, *plan);
        // one coefficient encoding serves every pass: a plan that mixes the
        // int64 and float engines is rebuilt in the float engine
        bool mixed = false;
        for (size_t i = 1; st == MERA_OK && i < plan->eng.size(); ++i) mixed = mixed || plan->eng[i] != plan->eng[0];
        if (st == MERA_OK && mixed) {
            *plan = FusedPlan<V>();
            st = fused_build<V>(n, ops, *plan, true);
        }
        if (st != MERA_OK) {
            delete plan;
            return st;
        }
        MERA_RETURN_IF(!plan->tabs.empty(), MERA_EUNSUPPORTED, "unexpected diagonal tables in the layer plan");
        b->layer_plan = plan;
    }
    const bool q61 = !plan->eng.empty() && plan->eng[0] == 1;
    // per-row coefficients: RZ(b) RY(a) for every qubit
    std::vector<V> cf((size_t)nslots * n * 4);
    for (int r = 0; r < nslots; ++r)
        for (int q = 0; q < n; ++q) {
            const double a = theta[((size_t)r * 2 + 0) * n + q], bb = theta[((size_t)r * 2 + 1) * n + q];
            MERA_RETURN_IF(!std::isfinite(a) || !std::isfinite(bb), MERA_EINVAL, "non-finite angle");
            const double c = std::cos(a / 2), s = std::sin(a / 2);
            const double er = std::cos(bb / 2), ei = std::sin(bb / 2);   // e^{ib/2}
            V* m = &cf[((size_t)r * n + q) * 4];
            m[0] = mkq<V>(er * c, -ei * c, q61);      // e^{-ib/2} c
            m[1] = mkq<V>(-er * s, ei * s, q61);      // -e^{-ib/2} s
            m[2] = mkq<V>(er * s, ei * s, q61);       // e^{ib/2} s
            m[3] = mkq<V>(er * c, ei * c, q61);       // e^{ib/2} c
        }
    MERA_TRY(grow(&b->coef, &b->coef_bytes, cf.size() * sizeof(V)));
    MERA_CHECK_CUDA(cudaMemcpyAsync(b->coef, cf.data(), cf.size() * sizeof(V), cudaMemcpyHostToDevice, b->stream));
    MERA_TRY(upload_slots(b, slots, nslots, 0));
    for (size_t i = 0; i < plan->args.size(); ++i) {
        MERA_RETURN_IF(plan->single[i] >= 0, MERA_EUNSUPPORTED, "unexpected per-gate op in the layer plan");
        PassArgs<V> A = plan->args[i];
        A.psi = reinterpret_cast<V*>(b->states);
        A.slots = b->dslots;
        A.bstride = 1ull << n;
        A.bcoef = reinterpret_cast<const V*>(b->coef);
        A.bcstride = 4 * n;
        MERA_TRY(fused_launch<V>(*plan, i, A, (unsigned)nslots, b->stream));
    }
    return MERA_OK;
}

static int batch_layer(mera_batch* b, const int* slots, int nslots, const double* theta) {
    if (b->dtype == MERA_C128) return batch_layer_t<double2>(b, slots, nslots, theta);
    return batch_layer_t<float2>(b, slots, nslots, theta);
}

template <typename V>
static int batch_reset_t(mera_batch* b, int nslots, int offset) {
    const uint64_t N = 1ull << b->n;
    const unsigned bx = (unsigned)std::min<uint64_t>((N + 255) / 256, 64);
    launch_begin(b->stream, MERA_KCLASS_QNN, (double)N * sizeof(V) * nslots);
    k_batch_zero<V><<<dim3(bx, nslots), 256, 0, b->stream>>>(reinterpret_cast<V*>(b->states), b->dslots + offset, N);
    return launch_end(b->stream);
}

static int batch_reset(mera_batch* b, const int* slots, int nslots) {
    MERA_TRY(upload_slots(b, slots, nslots, 0));
    if (b->dtype == MERA_C128) return batch_reset_t<double2>(b, nslots, 0);
    return batch_reset_t<float2>(b, nslots, 0);
}

template <typename V>
static int batch_obs_t(mera_batch* b, int nslots, int q, double* out) {
    const uint64_t N = 1ull << b->n;
    const int nb = reduce_blocks(N);
    MERA_TRY(grow(&b->partial, &b->partial_bytes, (size_t)nslots * nb * 3 * sizeof(double)));
    MERA_TRY(grow(&b->dres, &b->dres_bytes, (size_t)nslots * 3 * sizeof(double)));
    launch_begin(b->stream, MERA_KCLASS_QNN, (double)N * sizeof(V) * nslots);
    k_batch_obs<V><<<dim3(nb, nslots), 256, 0, b->stream>>>(reinterpret_cast<const V*>(b->states), b->dslots, b->n,
                                                             N / nb, q, b->partial);
    MERA_TRY(launch_end(b->stream));
    launch_begin(b->stream, MERA_KCLASS_QNN, 24.0 * nb * nslots);
    k_batch_obs_finish<<<nslots, 256, 0, b->stream>>>(b->partial, nb, b->dres);
    MERA_TRY(launch_end(b->stream));
    MERA_CHECK_CUDA(cudaMemcpyAsync(out, b->dres, (size_t)nslots * 3 * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
    MERA_CHECK_CUDA(cudaStreamSynchronize(b->stream));
    return MERA_OK;
}

static int batch_obs(mera_batch* b, const int* slots, int nslots, int q, double* out) {
    MERA_TRY(upload_slots(b, slots, nslots, 0));
    if (b->dtype == MERA_C128) return batch_obs_t<double2>(b, nslots, q, out);
    return batch_obs_t<float2>(b, nslots, q, out);
}

template <typename V>
static int adjoint_t(mera_batch* b, int nslots, int L, const double* theta, double* loss, double* grad) {
    const int n = b->n;
    const uint64_t N = 1ull << n;
    const int P = L * 2 * n;
    // forward: |0>, L layers
    std::vector<int> ids(nslots);
    for (int j = 0; j < nslots; ++j) ids[j] = j;
    MERA_TRY(batch_reset(b, ids.data(), nslots));
    for (int l = 0; l < L; ++l) {
        std::vector<double> th((size_t)nslots * 2 * n);
        for (int r = 0; r < nslots; ++r)
            memcpy(&th[(size_t)r * 2 * n], &theta[((size_t)r * L + l) * 2 * n], 2 * n * sizeof(double));
        MERA_TRY(batch_layer(b, ids.data(), nslots, th.data()));
    }
    // loss = sum_q <Z_q>
    std::vector<double> obs((size_t)nslots * 3);
    MERA_TRY(batch_obs(b, ids.data(), nslots, 0, obs.data()));
    for (int r = 0; r < nslots; ++r) loss[r] = obs[(size_t)r * 3 + 2];
    // lambda = O psi  (slot list rows 0..nslots-1: psi slots; adjoint states at + cap)
    MERA_TRY(upload_slots(b, ids.data(), nslots, 0));
    const unsigned bx = (unsigned)std::min<uint64_t>((N + 255) / 256, 64);
    launch_begin(b->stream, MERA_KCLASS_QNN, 2.0 * N * sizeof(V) * nslots);
    k_adj_init<V><<<dim3(bx, nslots), 256, 0, b->stream>>>(reinterpret_cast<V*>(b->states), b->dslots, nslots, b->cap, n);
    MERA_TRY(launch_end(b->stream));
    // inverse ring plan over 2 * nslots rows (psi slots and adjoint slots)
    FusedPlan<V>* rplan = reinterpret_cast<FusedPlan<V>*>(b->ring_inv_plan);
    if (!rplan) {
        rplan = new FusedPlan<V>();
        std::vector<PrepOp> ops;
        int st = ring_inverse_ops(n, ops);
        if (st == MERA_OK) st = fused_build<V>(n, ops, *rplan);
        if (st != MERA_OK) {
            delete rplan;
            return st;
        }
        b->ring_inv_plan = rplan;
    }
    std::vector<int> rows(2 * (size_t)nslots);
    for (int j = 0; j < nslots; ++j) {
        rows[j] = j;
        rows[nslots + j] = b->cap + j;
    }
    // the slot buffer holds 2 * cap ints: rows for the ring at offset cap
    MERA_CHECK_CUDA(cudaMemcpyAsync(b->dslots + b->cap, rows.data(), rows.size() * sizeof(int), cudaMemcpyHostToDevice,
                                    b->stream));
    // blocks per state (power of two dividing both N and N/2)
    const int nbz = (int)std::min<uint64_t>(ADJ_BLOCKS, std::max<uint64_t>(1, (N / 2) / 256));
    const int nby = nbz;
    MERA_TRY(grow(&b->partial, &b->partial_bytes, (size_t)P * nslots * nbz * sizeof(double)));
    MERA_TRY(grow(&b->dang, &b->dang_bytes, (size_t)nslots * n * 2 * 2 * sizeof(double)));
    MERA_TRY(grow(&b->dres, &b->dres_bytes, (size_t)nslots * P * sizeof(double)));
    std::vector<double> ang((size_t)nslots * n * 2 * 2);
    for (int l = L - 1; l >= 0; --l) {
        // undo the ring on both states
        for (size_t i = 0; i < rplan->args.size(); ++i) {
            PassArgs<V> A = rplan->args[i];
            A.psi = reinterpret_cast<V*>(b->states);
            A.slots = b->dslots + b->cap;
            A.bstride = N;
            MERA_TRY(fused_launch<V>(*rplan, i, A, (unsigned)(2 * nslots), b->stream));
        }
        // rotation angles of this layer: [row][g][q] -> (cos, sin) of half angles
        for (int r = 0; r < nslots; ++r)
            for (int g = 0; g < 2; ++g)
                for (int q = 0; q < n; ++q) {
                    const double t = theta[(((size_t)r * L + l) * 2 + g) * n + q];
                    double* d = &ang[(((size_t)g * nslots + r) * n + q) * 2];
                    d[0] = std::cos(t / 2);
                    d[1] = std::sin(t / 2);
                }
        MERA_CHECK_CUDA(cudaMemcpyAsync(b->dang, ang.data(), ang.size() * sizeof(double), cudaMemcpyHostToDevice,
                                        b->stream));
        const double* ang_ry = b->dang;
        const double* ang_rz = b->dang + (size_t)nslots * n * 2;
        // RZ gates (forward order RZ_0..RZ_{n-1}), undone last first
        for (int q = n - 1; q >= 0; --q) {
            const int p = (l * 2 + 1) * n + q;
            launch_begin(b->stream, MERA_KCLASS_QNN, 4.0 * N * sizeof(V) * nslots);
            k_adj_rz<V><<<dim3(nbz, nslots), 256, 0, b->stream>>>(reinterpret_cast<V*>(b->states), b->dslots, b->cap, n,
                                                                  q, ang_rz, b->partial + (size_t)p * nslots * nbz);
            MERA_TRY(launch_end(b->stream));
        }
        for (int q = n - 1; q >= 0; --q) {
            const int p = (l * 2 + 0) * n + q;
            launch_begin(b->stream, MERA_KCLASS_QNN, 4.0 * N * sizeof(V) * nslots);
            k_adj_ry<V><<<dim3(nby, nslots), 256, 0, b->stream>>>(reinterpret_cast<V*>(b->states), b->dslots, b->cap, n,
                                                                  q, ang_ry, b->partial + (size_t)p * nslots * nby);
            MERA_TRY(launch_end(b->stream));
        }
    }
    launch_begin(b->stream, MERA_KCLASS_QNN, 8.0 * P * nslots * nbz);
    k_adj_finish<<<nslots, 256, 0, b->stream>>>(b->partial, nslots, P, nbz, b->dres);
    MERA_TRY(launch_end(b->stream));
    MERA_CHECK_CUDA(cudaMemcpyAsync(grad, b->dres, (size_t)nslots * P * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
    MERA_CHECK_CUDA(cudaStreamSynchronize(b->stream));
    return MERA_OK;
}

}  // namespace mera

using namespace mera;

#define QAPI_TRY try {
#define QAPI_CATCH                                  \
    }                                               \
    catch (const std::bad_alloc&) {                 \
        set_error("host allocation failed");        \
        return MERA_ENOMEM;                         \
    }                                               \
    catch (...) {                                   \
        set_error("unexpected C++ exception");      \
        return MERA_EINVAL;                         \
    }

static int check_batch(const mera_batch* b) {
    MERA_RETURN_IF(b == nullptr || b->states == nullptr, MERA_EINVAL, "batch is NULL");
    return MERA_OK;
}

extern "C" {

int mera_batch_create(int n, int capacity, int dtype, void* stream, mera_batch** out) {
    QAPI_TRY
    MERA_RETURN_IF(out == nullptr, MERA_EINVAL, "out is NULL");
    *out = nullptr;
    MERA_RETURN_IF(n < 5 || n > 26, MERA_EINVAL, "batched ansatz supports 5 <= n <= 26, got %d", n);
    MERA_RETURN_IF(capacity < 1 || capacity > 65535, MERA_EINVAL, "capacity %d outside [1, 65535]", capacity);
    MERA_RETURN_IF(dtype != MERA_C64 && dtype != MERA_C128, MERA_EUNSUPPORTED, "unknown dtype %d", dtype);
    mera_batch* b = new mera_batch();
    b->n = n;
    b->cap = capacity;
    b->dtype = dtype;
    b->stream = (cudaStream_t)stream;
    const size_t bytes = 2ull * capacity * (1ull << n) * elem_bytes(dtype);
    cudaError_t e = cudaMalloc(&b->states, bytes);
    // slot lists: one launch's rows at 0, the adjoint ring's 2 * nslots rows at cap
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&b->dslots), 3ull * capacity * sizeof(int));
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (b->states) cudaFree(b->states);
        delete b;
        set_error("cudaMalloc for a batch of %d states of n=%d: %s", capacity, n, cudaGetErrorString(e));
        return MERA_ENOMEM;
    }
    *out = b;
    return MERA_OK;
    QAPI_CATCH
}

int mera_batch_destroy(mera_batch* b) {
    if (!b) return MERA_OK;
    cudaStreamSynchronize(b->stream);
    cudaFree(b->states);
    cudaFree(b->dslots);
    if (b->coef) cudaFree(b->coef);
    if (b->dang) cudaFree(b->dang);
    if (b->partial) cudaFree(b->partial);
    if (b->dres) cudaFree(b->dres);
    if (b->dtype == MERA_C128) {
        delete reinterpret_cast<FusedPlan<double2>*>(b->layer_plan);
        delete reinterpret_cast<FusedPlan<double2>*>(b->ring_inv_plan);
    } else {
        delete reinterpret_cast<FusedPlan<float2>*>(b->layer_plan);
        delete reinterpret_cast<FusedPlan<float2>*>(b->ring_inv_plan);
    }
    delete b;
    return MERA_OK;
}

int mera_batch_info(const mera_batch* b, void** dev_states, int* n, int* capacity, int* dtype) {
    MERA_TRY(check_batch(b));
    if (dev_states) *dev_states = b->states;
    if (n) *n = b->n;
    if (capacity) *capacity = b->cap;
    if (dtype) *dtype = b->dtype;
    return MERA_OK;
}

int mera_batch_copy_to_host(mera_batch* b, int slot, void* host) {
    MERA_TRY(check_batch(b));
    MERA_RETURN_IF(host == nullptr, MERA_EINVAL, "host is NULL");
    MERA_RETURN_IF(slot < 0 || slot >= 2 * b->cap, MERA_EINVAL, "slot %d out of range", slot);
    const size_t bytes = (1ull << b->n) * elem_bytes(b->dtype);
    MERA_CHECK_CUDA(cudaMemcpyAsync(host, static_cast<char*>(b->states) + (size_t)slot * bytes, bytes,
                                    cudaMemcpyDeviceToHost, b->stream));
    MERA_CHECK_CUDA(cudaStreamSynchronize(b->stream));
    return MERA_OK;
}

int mera_batch_set_stream(mera_batch* b, void* stream) {
    MERA_TRY(check_batch(b));
    b->stream = (cudaStream_t)stream;
    return MERA_OK;
}

int mera_batch_reset(mera_batch* b, const int* slots, int nslots) {
    QAPI_TRY
    MERA_TRY(check_batch(b));
    return batch_reset(b, slots, nslots);
    QAPI_CATCH
}

int mera_batch_layer(mera_batch* b, const int* slots, int nslots, const double* theta) {
    QAPI_TRY
    MERA_TRY(check_batch(b));
    MERA_RETURN_IF(theta == nullptr, MERA_EINVAL, "theta is NULL");
    return batch_layer(b, slots, nslots, theta);
    QAPI_CATCH
}

int mera_batch_forward(mera_batch* b, int nslots, int L, const double* theta) {
    QAPI_TRY
    MERA_TRY(check_batch(b));
    MERA_RETURN_IF(theta == nullptr || L < 0, MERA_EINVAL, "bad theta / L");
    std::vector<int> ids(nslots > 0 ? nslots : 1);
    for (int j = 0; j < nslots; ++j) ids[j] = j;
    MERA_TRY(batch_reset(b, ids.data(), nslots));
    std::vector<double> th((size_t)std::max(nslots, 1) * 2 * b->n);
    for (int l = 0; l < L; ++l) {
        for (int r = 0; r < nslots; ++r)
            memcpy(&th[(size_t)r * 2 * b->n], &theta[((size_t)r * L + l) * 2 * b->n], 2 * b->n * sizeof(double));
        MERA_TRY(batch_layer(b, ids.data(), nslots, th.data()));
    }
    return MERA_OK;
    QAPI_CATCH
}

int mera_batch_observables(mera_batch* b, const int* slots, int nslots, int q, double* out) {
    QAPI_TRY
    MERA_TRY(check_batch(b));
    MERA_RETURN_IF(out == nullptr, MERA_EINVAL, "out is NULL");
    MERA_RETURN_IF(q < 0 || q >= b->n, MERA_EINVAL, "qubit %d out of range", q);
    return batch_obs(b, slots, nslots, q, out);
    QAPI_CATCH
}

int mera_adjoint_grad(mera_batch* b, int nslots, int L, const double* theta, double* loss, double* grad) {
    QAPI_TRY
    MERA_TRY(check_batch(b));
    MERA_RETURN_IF(theta == nullptr || loss == nullptr || grad == nullptr, MERA_EINVAL, "NULL argument");
    MERA_RETURN_IF(L < 1, MERA_EINVAL, "L=%d", L);
    MERA_RETURN_IF(nslots < 1 || nslots > b->cap, MERA_EINVAL, "%d slots for a batch of %d", nslots, b->cap);
    if (b->dtype == MERA_C128) return adjoint_t<double2>(b, nslots, L, theta, loss, grad);
    return adjoint_t<float2>(b, nslots, L, theta, loss, grad);
    QAPI_CATCH
}

}  // extern "C"
