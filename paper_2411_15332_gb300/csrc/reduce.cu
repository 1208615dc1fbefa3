// Readouts of Eq. 4-5: squared magnitudes summed in float64.
//
// Every reduction uses the same fixed partition: RB = min(1024, N/256)
// blocks, block b owns the contiguous chunk [b*N/RB, (b+1)*N/RB); its 256
// threads stride through the chunk accumulating in float64, then a fixed
// shuffle tree gives one partial per block, and one block reduces the
// partials in index order.  The result is therefore the same on every run.
#include <algorithm>
#include <cstring>
#include <cmath>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"
#include "reduce.cuh"

namespace mera {

// |a|^2 as re*re + im*im with each operation rounded separately (no fused
// multiply-add), so integer decisions (argmax) match a plain float64 CPU.
__device__ __forceinline__ double prob_rn(double2 a) {
    return __dadd_rn(__dmul_rn(a.x, a.x), __dmul_rn(a.y, a.y));
}
__device__ __forceinline__ double prob_rn(float2 a) {
    const double x = a.x, y = a.y;
    return __dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y));
}

// |a|^2 for sums (one fused multiply-add).
__device__ __forceinline__ double prob_fma(double2 a) { return fma(a.x, a.x, a.y * a.y); }
__device__ __forceinline__ double prob_fma(float2 a) {
    const double x = a.x, y = a.y;
    return fma(x, x, y * y);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide sum of three values (fixed order); result valid in thread 0.
__device__ __forceinline__ void block_sum3(double& a, double& b, double& c) {
    __shared__ double sh[3][8];
    a = warp_sum(a);
    b = warp_sum(b);
    c = warp_sum(c);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) {
        sh[0][w] = a;
        sh[1][w] = b;
        sh[2][w] = c;
    }
    __syncthreads();
    if (w == 0) {
        a = l < (int)(blockDim.x >> 5) ? sh[0][l] : 0.0;
        b = l < (int)(blockDim.x >> 5) ? sh[1][l] : 0.0;
        c = l < (int)(blockDim.x >> 5) ? sh[2][l] : 0.0;
        a = warp_sum(a);
        b = warp_sum(b);
        c = warp_sum(c);
    }
}

// Per-block partial sums of |a|^2, (1 - 2 bit_q) |a|^2, (n - 2 popcount) |a|^2.
template <typename V>
__global__ void __launch_bounds__(256) k_observables(const V* __restrict__ psi, uint64_t chunk, int n, int q,
                                                     double* __restrict__ partial) {
    const uint64_t lo = (uint64_t)blockIdx.x * chunk;
    // five FP64 operations per amplitude (FP64 issues at 1/57 of FP32 on
    // this GPU): |a|^2 with one fused multiply-add, the norm, the mass on
    // bit q = 1, and the popcount-weighted mass
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (uint64_t i = lo + threadIdx.x; i < lo + chunk; i += blockDim.x) {
        const double p = prob_fma(psi[i]);
        s0 += p;
        if ((i >> q) & 1ull) s1 += p;
        s2 = fma((double)__popcll(i), p, s2);
    }
    block_sum3(s0, s1, s2);
    if (threadIdx.x == 0) {
        // <Z_q> = norm - 2 * mass(bit q = 1); sum_q <Z_q> = n norm - 2 sum popcount |a|^2
        partial[3 * blockIdx.x + 0] = s0;
        partial[3 * blockIdx.x + 1] = s0 - 2.0 * s1;
        partial[3 * blockIdx.x + 2] = (double)n * s0 - 2.0 * s2;
    }
}

__global__ void __launch_bounds__(256) k_finish3(const double* __restrict__ partial, int nb, double* __restrict__ out) {
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
        s0 += partial[3 * b + 0];
        s1 += partial[3 * b + 1];
        s2 += partial[3 * b + 2];
    }
    block_sum3(s0, s1, s2);
    if (threadIdx.x == 0) {
        out[0] = s0;
        out[1] = s1;
        out[2] = s2;
    }
}

// ---- argmax: largest |a|^2, lowest index on ties (a total order) --------
struct PI {
    double p;
    unsigned long long i;
};
__device__ __forceinline__ PI better(PI a, PI b) {
    if (b.p > a.p || (b.p == a.p && b.i < a.i)) return b;
    return a;
}
__device__ __forceinline__ PI warp_best(PI v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        PI w;
        w.p = __shfl_down_sync(0xffffffffu, v.p, o);
        w.i = __shfl_down_sync(0xffffffffu, v.i, o);
        v = better(v, w);
    }
    return v;
}
__device__ __forceinline__ PI block_best(PI v) {
    __shared__ double sp[8];
    __shared__ unsigned long long si[8];
    v = warp_best(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) {
        sp[w] = v.p;
        si[w] = v.i;
    }
    __syncthreads();
    if (w == 0) {
        PI x;
        x.p = l < (int)(blockDim.x >> 5) ? sp[l] : -1.0;
        x.i = l < (int)(blockDim.x >> 5) ? si[l] : ~0ull;
        v = warp_best(x);
    }
    return v;
}

template <typename V>
__global__ void __launch_bounds__(256) k_argmax(const V* __restrict__ psi, uint64_t chunk, double* __restrict__ pp,
                                                unsigned long long* __restrict__ pi) {
    const uint64_t lo = (uint64_t)blockIdx.x * chunk;
    PI best{-1.0, ~0ull};
    for (uint64_t i = lo + threadIdx.x; i < lo + chunk; i += blockDim.x) {
        PI c{prob_rn(psi[i]), (unsigned long long)i};
        best = better(best, c);
    }
    best = block_best(best);
    if (threadIdx.x == 0) {
        pp[blockIdx.x] = best.p;
        pi[blockIdx.x] = best.i;
    }
}

__global__ void __launch_bounds__(256) k_argmax_finish(const double* __restrict__ pp, const unsigned long long* __restrict__ pi,
                                                       int nb, double* __restrict__ out_p, unsigned long long* __restrict__ out_i) {
    PI best{-1.0, ~0ull};
    for (int b = threadIdx.x; b < nb; b += blockDim.x) best = better(best, PI{pp[b], pi[b]});
    best = block_best(best);
    if (threadIdx.x == 0) {
        *out_p = best.p;
        *out_i = best.i;
    }
}

// ---- measurement: locate target inside one chunk ------------------------
// Thread j of block s scans the contiguous slice j of chunk cb[s] after an
// exclusive scan of the slice sums, and the first index whose running sum
// exceeds tgt[s] wins.
template <typename V>
__global__ void __launch_bounds__(256) k_measure(const V* __restrict__ psi, uint64_t chunk, const int* __restrict__ cb,
                                                 const double* __restrict__ cbase, const double* __restrict__ tgt,
                                                 unsigned long long* __restrict__ out) {
    __shared__ double sums[256];
    __shared__ unsigned long long found;
    const int s = blockIdx.x;
    const uint64_t lo = (uint64_t)cb[s] * chunk;
    const uint64_t per = chunk / blockDim.x;
    const uint64_t a = lo + per * threadIdx.x;
    double acc = 0.0;
    for (uint64_t i = a; i < a + per; ++i) acc += prob_rn(psi[i]);
    sums[threadIdx.x] = acc;
    if (threadIdx.x == 0) found = ~0ull;
    __syncthreads();
    if (threadIdx.x == 0) {
        double run = cbase[s];
        for (int j = 0; j < (int)blockDim.x; ++j) {
            const double x = sums[j];
            sums[j] = run;
            run += x;
        }
    }
    __syncthreads();
    double run = sums[threadIdx.x];
    const double t = tgt[s];
    if (run + acc > t || threadIdx.x == blockDim.x - 1) {
        for (uint64_t i = a; i < a + per; ++i) {
            run += prob_rn(psi[i]);
            if (run > t) {
                atomicMin(&found, (unsigned long long)i);
                break;
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) out[s] = found == ~0ull ? (unsigned long long)(lo + chunk - 1) : found;
}

// ---- gather of sampled amplitudes, widened to float64 -------------------
template <typename V>
__global__ void k_gather(const V* __restrict__ psi, const unsigned long long* __restrict__ idx, size_t k,
                         double2* __restrict__ out) {
    const size_t j = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < k) {
        const V a = psi[idx[j]];
        out[j] = make_double2((double)a.x, (double)a.y);
    }
}

// ------------------------------------------------------------- launchers --
int reduce_blocks(uint64_t N) {
    uint64_t b = N / 256;
    if (b > 1024) b = 1024;
    if (b < 1) b = 1;
    return (int)b;
}

template <typename V>
static int observables_t(mera_state* s, int q, double* partial, double* out_dev) {
    const uint64_t N = num_amps(s);
    const int nb = reduce_blocks(N);
    const uint64_t chunk = N / nb;
    launch_begin(s->stream, MERA_KCLASS_REDUCE, (double)N * sizeof(V));
    k_observables<V><<<nb, 256, 0, s->stream>>>(reinterpret_cast<const V*>(s->data), chunk, s->n, q, partial);
    MERA_TRY(launch_end(s->stream));
    launch_begin(s->stream, MERA_KCLASS_REDUCE, 24.0 * nb);
    k_finish3<<<1, 256, 0, s->stream>>>(partial, nb, out_dev);
    return launch_end(s->stream);
}

int observables_finish(mera_state* s, const double* partial, int nb, double* out_dev) {
    launch_begin(s->stream, MERA_KCLASS_REDUCE, 24.0 * nb);
    k_finish3<<<1, 256, 0, s->stream>>>(partial, nb, out_dev);
    return launch_end(s->stream);
}

int observables_device(mera_state* s, int q, double* partial, double* out_dev) {
    if (s->dtype == MERA_C128) return observables_t<double2>(s, q, partial, out_dev);
    return observables_t<float2>(s, q, partial, out_dev);
}

int observables(mera_state* s, int q, double out[3]) {
    const uint64_t N = num_amps(s);
    const int nb = reduce_blocks(N);
    MERA_TRY(state_ensure_scratch(s, (size_t)(3 * nb + 8) * sizeof(double)));
    double* partial = reinterpret_cast<double*>(s->scratch);
    double* out_dev = partial + 3 * nb;
    MERA_TRY(observables_device(s, q, partial, out_dev));
    MERA_CHECK_CUDA(cudaMemcpyAsync(out, out_dev, 3 * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    MERA_CHECK_CUDA(cudaStreamSynchronize(s->stream));
    MERA_TRY(state_check_waits(s));
    return MERA_OK;
}

template <typename V>
static int argmax_t(mera_state* s, uint64_t* idx, double* prob) {
    const uint64_t N = num_amps(s);
    const int nb = reduce_blocks(N);
    MERA_TRY(state_ensure_scratch(s, (size_t)(2 * nb + 4) * sizeof(double)));
    double* pp = reinterpret_cast<double*>(s->scratch);
    unsigned long long* pi = reinterpret_cast<unsigned long long*>(pp + nb);
    double* op = pp + 2 * nb;
    unsigned long long* oi = reinterpret_cast<unsigned long long*>(pp + 2 * nb + 1);
    launch_begin(s->stream, MERA_KCLASS_REDUCE, (double)N * sizeof(V));
    k_argmax<V><<<nb, 256, 0, s->stream>>>(reinterpret_cast<const V*>(s->data), N / nb, pp, pi);
    MERA_TRY(launch_end(s->stream));
    launch_begin(s->stream, MERA_KCLASS_REDUCE, 16.0 * nb);
    k_argmax_finish<<<1, 256, 0, s->stream>>>(pp, pi, nb, op, oi);
    MERA_TRY(launch_end(s->stream));
    double res[2];
    MERA_CHECK_CUDA(cudaMemcpyAsync(res, op, 2 * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    MERA_CHECK_CUDA(cudaStreamSynchronize(s->stream));
    MERA_TRY(state_check_waits(s));
    unsigned long long i;
    memcpy(&i, &res[1], sizeof(i));
    *idx = i;
    if (prob) *prob = res[0];
    return MERA_OK;
}

int argmax(mera_state* s, uint64_t* idx, double* prob) {
    if (s->dtype == MERA_C128) return argmax_t<double2>(s, idx, prob);
    return argmax_t<float2>(s, idx, prob);
}

template <typename V>
static int measure_t(mera_state* s, const double* u, size_t k, uint64_t* out) {
    const uint64_t N = num_amps(s);
    const int nb = reduce_blocks(N);
    const uint64_t chunk = N / nb;
    // pass 1: per-chunk sums (the partition of k_observables)
    const size_t need = (size_t)(3 * nb + 8) * sizeof(double) + k * (sizeof(int) + 3 * sizeof(double)) + 64;
    MERA_TRY(state_ensure_scratch(s, need));
    double* partial = reinterpret_cast<double*>(s->scratch);
    double* out3 = partial + 3 * nb;
    MERA_TRY(observables_device(s, 0, partial, out3));
    std::vector<double> hp(3 * nb);
    MERA_CHECK_CUDA(cudaMemcpyAsync(hp.data(), partial, hp.size() * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    MERA_CHECK_CUDA(cudaStreamSynchronize(s->stream));
    MERA_TRY(state_check_waits(s));
    std::vector<double> cum(nb + 1, 0.0);
    for (int b = 0; b < nb; ++b) cum[b + 1] = cum[b] + hp[3 * b];
    const double total = cum[nb];
    MERA_RETURN_IF(!(total > 0.0), MERA_EINVAL, "state has zero norm; cannot sample");
    std::vector<int> cb(k);
    std::vector<double> base(k), tgt(k);
    for (size_t j = 0; j < k; ++j) {
        MERA_RETURN_IF(!(u[j] >= 0.0 && u[j] < 1.0), MERA_EINVAL, "u[%zu] = %g not in [0, 1)", j, u[j]);
        const double t = u[j] * total;
        int b = (int)(std::upper_bound(cum.begin() + 1, cum.end(), t) - (cum.begin() + 1));
        if (b >= nb) {   // rounding at the very top: last chunk with weight
            b = nb - 1;
            while (b > 0 && hp[3 * b] == 0.0) --b;
        }
        cb[j] = b;
        base[j] = cum[b];
        tgt[j] = t;
    }
    char* p = reinterpret_cast<char*>(out3 + 8);
    int* d_cb = reinterpret_cast<int*>(p);
    p += ((k * sizeof(int) + 15) / 16) * 16;
    double* d_base = reinterpret_cast<double*>(p);
    double* d_tgt = d_base + k;
    unsigned long long* d_out = reinterpret_cast<unsigned long long*>(d_tgt + k);
    MERA_CHECK_CUDA(cudaMemcpyAsync(d_cb, cb.data(), k * sizeof(int), cudaMemcpyHostToDevice, s->stream));
    MERA_CHECK_CUDA(cudaMemcpyAsync(d_base, base.data(), k * sizeof(double), cudaMemcpyHostToDevice, s->stream));
    MERA_CHECK_CUDA(cudaMemcpyAsync(d_tgt, tgt.data(), k * sizeof(double), cudaMemcpyHostToDevice, s->stream));
    const int threads = chunk >= 256 ? 256 : (int)chunk;
    launch_begin(s->stream, MERA_KCLASS_REDUCE, (double)k * chunk * sizeof(V));
    k_measure<V><<<(unsigned)k, threads, 0, s->stream>>>(reinterpret_cast<const V*>(s->data), chunk, d_cb, d_base, d_tgt,
                                                          d_out);
    MERA_TRY(launch_end(s->stream));
    std::vector<unsigned long long> res(k);
    MERA_CHECK_CUDA(cudaMemcpyAsync(res.data(), d_out, k * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s->stream));
    MERA_CHECK_CUDA(cudaStreamSynchronize(s->stream));
    MERA_TRY(state_check_waits(s));
    for (size_t j = 0; j < k; ++j) out[j] = res[j];
    return MERA_OK;
}

int measure(mera_state* s, const double* u, size_t k, uint64_t* out) {
    if (k == 0) return MERA_OK;
    if (s->dtype == MERA_C128) return measure_t<double2>(s, u, k, out);
    return measure_t<float2>(s, u, k, out);
}

template <typename V>
static int gather_t(mera_state* s, const uint64_t* idx, size_t k, double* out) {
    const size_t need = k * (sizeof(unsigned long long) + sizeof(double2)) + 64;
    MERA_TRY(state_ensure_scratch(s, need));
    unsigned long long* d_idx = reinterpret_cast<unsigned long long*>(s->scratch);
    double2* d_out = reinterpret_cast<double2*>(d_idx + ((k + 1) & ~size_t(1)));
    MERA_CHECK_CUDA(cudaMemcpyAsync(d_idx, idx, k * sizeof(uint64_t), cudaMemcpyHostToDevice, s->stream));
    launch_begin(s->stream, MERA_KCLASS_REDUCE, (double)k * sizeof(V));
    k_gather<V><<<(unsigned)((k + 255) / 256), 256, 0, s->stream>>>(reinterpret_cast<const V*>(s->data), d_idx, k, d_out);
    MERA_TRY(launch_end(s->stream));
    MERA_CHECK_CUDA(cudaMemcpyAsync(out, d_out, k * sizeof(double2), cudaMemcpyDeviceToHost, s->stream));
    MERA_CHECK_CUDA(cudaStreamSynchronize(s->stream));
    MERA_TRY(state_check_waits(s));
    return MERA_OK;
}

int gather(mera_state* s, const uint64_t* idx, size_t k, double* out) {
    if (k == 0) return MERA_OK;
    const uint64_t N = num_amps(s);
    for (size_t j = 0; j < k; ++j) MERA_RETURN_IF(idx[j] >= N, MERA_EINVAL, "index %llu >= 2^n", (unsigned long long)idx[j]);
    if (s->dtype == MERA_C128) return gather_t<double2>(s, idx, k, out);
    return gather_t<float2>(s, idx, k, out);
}

}  // namespace mera
