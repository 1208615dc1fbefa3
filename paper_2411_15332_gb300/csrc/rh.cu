// The paper's RH-MVM of H^{(x)n} with its four sign-computation methods
// (Sec. III-B.2, Table II, Algorithm 1), as device kernels.
//
// RH stores H^{(x)n} as one number, the common magnitude 1/sqrt(N); the sign
// of element (r, c) is parsed on demand by the quadrant recursion of Fig. 3
// (split the matrix into four quarters, the lower-right one negative, and
// recurse into the quarter holding (r, c)), O(n) per sign.  The MVM first
// scales S by that magnitude (Algorithm 1, first step) and is out of place.
// The methods differ in how many signs they compute per row:
//   non-optimised  every (r, c):                          2^n * 2^n
//   quarter-based  upper-left quarter (r, c < 2^(n-1));
//                  each sign updates four outputs:        2^(n-1) * 2^(n-1)
//   block-based    per quarter row, the b signs of the first block and the
//                  first sign of every other block (b = sqrt(2^(n-1)),
//                  Theorem 3):                            2^(n-1) * (2^(n-1)/b + b - 1)
//   logarithm      per quarter row, the signs at columns 2^0 .. 2^(n-2);
//                  any other column c takes sign[2^p] * sign[c - 2^p], 2^p
//                  the largest power of two <= c (Algorithm 1):
//                                                         2^(n-1) * (n - 1)
// Every kernel counts its compute_sign calls; the host returns the total,
// which equals Table II.
//
// Device layout: a CTA takes RH_ROWS rows at a time.  Its sign phase fills
// a shared-memory bit array per row (bit c = 1 where sign(r, c) = -1; this
// is Algorithm 1's temporary sign[] array) by the method's own rule; its
// accumulate phase then sweeps the columns with all threads, each column's
// scaled amplitudes read once for the CTA's rows, and the four quarter
// updates of Algorithm 1 (two for the non-optimised method's full rows) in
// float64, followed by a block reduction per output.
#include <algorithm>
#include <cmath>

#include "common.cuh"

namespace mera {

enum RhMethod { RH_NONOPT = 0, RH_QUARTER = 1, RH_BLOCK = 2, RH_LOG = 3 };
constexpr int RH_MAX_N = 18;
constexpr int RH_THREADS = 256;
constexpr int RH_ROWS = 4;
constexpr int RH_AUX = 768;       // block: b <= 256 first-block signs + h/b <= 512 block signs

// Fig. 3: the quarter holding (r, c) at each level; the lower-right quarter
// flips the sign.  Returns 1 for -1, 0 for +1.
__device__ __forceinline__ uint32_t rh_compute_sign(uint32_t r, uint32_t c, int n) {
    uint32_t neg = 0;
    for (uint32_t size = 1u << n; size > 1; size >>= 1) {
        const uint32_t half = size >> 1;
        if (r >= half && c >= half) neg ^= 1u;
        r &= half - 1;
        c &= half - 1;
    }
    return neg;
}

__global__ void k_rh_scale(const double2* __restrict__ s, double2* __restrict__ ss, uint32_t N, double value) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        const double2 v = s[i];
        ss[i] = make_double2(value * v.x, value * v.y);
    }
}

__device__ __forceinline__ double2 sgn_apply(double2 a, uint32_t neg) {
    return neg ? make_double2(-a.x, -a.y) : a;
}

template <int M>
__global__ void __launch_bounds__(RH_THREADS) k_rh_mvm(const double2* __restrict__ ss, double2* __restrict__ out,
                                                       int n, uint32_t b, unsigned long long* __restrict__ count) {
    extern __shared__ uint32_t sbits[];                 // RH_ROWS x W words
    __shared__ unsigned char s_aux[RH_ROWS][RH_AUX];    // computed signs (1 = negative)
    __shared__ double s_red[RH_THREADS / 32][RH_ROWS * 4];
    __shared__ unsigned long long s_cnt;
    const uint32_t N = 1u << n, h = N >> 1;
    const uint32_t width = M == RH_NONOPT ? N : h;
    const uint32_t nrows = M == RH_NONOPT ? N : h;
    const uint32_t W = (width + 31u) >> 5;
    const uint32_t tid = threadIdx.x, T = blockDim.x;
    const uint32_t lane = tid & 31u, warp = tid >> 5;
    unsigned long long cnt = 0;
    if (tid == 0) s_cnt = 0;
    __syncthreads();
    for (uint32_t r0 = blockIdx.x * RH_ROWS; r0 < nrows; r0 += gridDim.x * RH_ROWS) {
        const uint32_t R = min((uint32_t)RH_ROWS, nrows - r0);
        // ---------------------------------------------------- signs ----
        if (M == RH_NONOPT || M == RH_QUARTER) {
            for (uint32_t wi = tid; wi < R * W; wi += T) {
                const uint32_t rr = wi / W, w = wi - rr * W;
                const uint32_t cend = min(32u, width - 32u * w);
                uint32_t word = 0;
                for (uint32_t j = 0; j < cend; ++j) word |= rh_compute_sign(r0 + rr, 32u * w + j, n) << j;
                cnt += cend;
                sbits[rr * W + w] = word;
            }
        } else if (M == RH_BLOCK) {
            const uint32_t nb = h / b, per = b + nb - 1;
            for (uint32_t t = tid; t < R * per; t += T) {
                const uint32_t rr = t / per, k = t - rr * per;
                if (k < b) {
                    s_aux[rr][k] = (unsigned char)rh_compute_sign(r0 + rr, k, n);      // first block
                } else {
                    const uint32_t blk = k - b + 1;                                    // 1 .. nb - 1
                    s_aux[rr][256 + blk] = (unsigned char)rh_compute_sign(r0 + rr, blk * b, n);
                }
                ++cnt;
            }
            __syncthreads();
            // a block's signs are the first block's, negated where the
            // block's first sign is negative
            for (uint32_t wi = tid; wi < R * W; wi += T) {
                const uint32_t rr = wi / W, w = wi - rr * W;
                const uint32_t cend = min(32u, width - 32u * w);
                uint32_t word = 0;
                for (uint32_t j = 0; j < cend; ++j) {
                    const uint32_t c = 32u * w + j, blk = c / b, jj = c - blk * b;
                    const uint32_t neg = s_aux[rr][jj] ^ (blk ? s_aux[rr][256 + blk] : 0u);
                    word |= neg << j;
                }
                sbits[rr * W + w] = word;
            }
        } else {
            for (uint32_t t = tid; t < R * (uint32_t)(n - 1); t += T) {
                const uint32_t rr = t / (uint32_t)(n - 1), p = t - rr * (uint32_t)(n - 1);
                s_aux[rr][p] = (unsigned char)rh_compute_sign(r0 + rr, 1u << p, n);   // columns 2^p
                ++cnt;
            }
            __syncthreads();
            // Algorithm 1: sign[0] = 1; a power of two takes its computed
            // sign; any other c takes sign[2^p] * sign[c - 2^p].  Columns
            // below 32 one by one; above, a whole word of 32 columns
            // 2^p + j at once from the word of the columns j
            if (tid < R) {
                const uint32_t cend = min(32u, width);
                uint32_t word = 0;
                for (uint32_t c = 1; c < cend; ++c) {
                    const uint32_t p = 31u - __clz(c), pw = 1u << p;
                    const uint32_t neg = c == pw ? s_aux[tid][p] : (((word >> pw) ^ (word >> (c - pw))) & 1u);
                    word |= neg << c;
                }
                sbits[tid * W] = word;
            }
            __syncthreads();
            for (int p = 5; p < n - 1; ++p) {
                const uint32_t w0 = 1u << (p - 5);
                for (uint32_t wi = tid; wi < R * w0; wi += T) {
                    const uint32_t rr = wi / w0, k = wi - rr * w0;
                    sbits[rr * W + w0 + k] = sbits[rr * W + k] ^ (s_aux[rr][p] ? 0xFFFFFFFFu : 0u);
                }
                __syncthreads();
            }
        }
        __syncthreads();
        // ------------------------------------------------- accumulate ----
        double2 acc0[RH_ROWS], acc1[RH_ROWS];
#pragma unroll
        for (int rr = 0; rr < RH_ROWS; ++rr) acc0[rr] = acc1[rr] = make_double2(0.0, 0.0);
        if (M == RH_NONOPT) {
            for (uint32_t c = tid; c < N; c += T) {
                const double2 a = __ldg(ss + c);
#pragma unroll
                for (int rr = 0; rr < RH_ROWS; ++rr) {
                    if ((uint32_t)rr >= R) break;
                    const double2 sa = sgn_apply(a, (sbits[rr * W + (c >> 5)] >> (c & 31u)) & 1u);
                    acc0[rr].x += sa.x;
                    acc0[rr].y += sa.y;
                }
            }
        } else {
            for (uint32_t c = tid; c < h; c += T) {
                const double2 a = __ldg(ss + c), d = __ldg(ss + c + h);
#pragma unroll
                for (int rr = 0; rr < RH_ROWS; ++rr) {
                    if ((uint32_t)rr >= R) break;
                    const uint32_t neg = (sbits[rr * W + (c >> 5)] >> (c & 31u)) & 1u;
                    const double2 sa = sgn_apply(a, neg), sd = sgn_apply(d, neg);
                    // the four updates of one upper-left sign
                    acc0[rr].x += sa.x;
                    acc0[rr].y += sa.y;
                    acc0[rr].x += sd.x;
                    acc0[rr].y += sd.y;
                    acc1[rr].x += sa.x;
                    acc1[rr].y += sa.y;
                    acc1[rr].x -= sd.x;
                    acc1[rr].y -= sd.y;
                }
            }
        }
        // block reduction: warp shuffles, then one partial per warp
#pragma unroll
        for (int rr = 0; rr < RH_ROWS; ++rr) {
            double v[4] = {acc0[rr].x, acc0[rr].y, acc1[rr].x, acc1[rr].y};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                for (int off = 16; off > 0; off >>= 1) v[q] += __shfl_down_sync(0xffffffffu, v[q], off);
                if (lane == 0) s_red[warp][rr * 4 + q] = v[q];
            }
        }
        __syncthreads();
        if (tid < R * 4) {
            double s = 0.0;
            for (uint32_t w = 0; w < T / 32; ++w) s += s_red[w][tid];
            s_red[0][tid] = s;
        }
        __syncthreads();
        if (tid < R) {
            out[r0 + tid] = make_double2(s_red[0][tid * 4 + 0], s_red[0][tid * 4 + 1]);
            if (M != RH_NONOPT) out[r0 + tid + h] = make_double2(s_red[0][tid * 4 + 2], s_red[0][tid * 4 + 3]);
        }
        __syncthreads();   // sbits and s_red are rewritten by the next rows
    }
    atomicAdd(&s_cnt, cnt);
    __syncthreads();
    if (tid == 0) atomicAdd(count, s_cnt);
}

template <int M>
static int launch_rh(const double2* ss, double2* out, int n, uint32_t b, unsigned long long* cnt, cudaStream_t st) {
    const uint32_t N = 1u << n, h = N >> 1;
    const uint32_t width = M == RH_NONOPT ? N : h;
    const uint32_t nrows = width;
    const size_t smem = (size_t)RH_ROWS * ((width + 31u) >> 5) * sizeof(uint32_t);
    static size_t opted = 0;
    if (smem > 48 * 1024 && smem > opted) {
        MERA_CHECK_CUDA(cudaFuncSetAttribute((const void*)k_rh_mvm<M>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem));
        opted = smem;
    }
    int dev = 0, sms = 0;
    MERA_CHECK_CUDA(cudaGetDevice(&dev));
    MERA_CHECK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const uint32_t groups = (nrows + RH_ROWS - 1) / RH_ROWS;
    const uint32_t grid = std::max(1u, std::min(groups, (uint32_t)sms * 8u));
    k_rh_mvm<M><<<grid, RH_THREADS, smem, st>>>(ss, out, n, b, cnt);
    return MERA_OK;
}

}  // namespace mera

using namespace mera;

extern "C" int mera_rh_mvm(mera_state* in, mera_state* out, int method, int block, uint64_t* sign_count) {
    MERA_RETURN_IF(in == nullptr || out == nullptr, MERA_EINVAL, "NULL state");
    MERA_RETURN_IF(in->n != out->n, MERA_EINVAL, "in and out must have the same n");
    MERA_RETURN_IF(in->dtype != MERA_C128 || out->dtype != MERA_C128, MERA_EUNSUPPORTED,
                   "the RH methods run on complex128 states");
    MERA_RETURN_IF(in->data == out->data, MERA_EINVAL, "the RH-MVM is out of place: in and out must differ");
    const int n = in->n;
    MERA_RETURN_IF(n < 2 || n > RH_MAX_N, MERA_EINVAL, "the RH methods take 2 <= n <= %d (n = %d)", RH_MAX_N, n);
    MERA_RETURN_IF(method < RH_NONOPT || method > RH_LOG, MERA_EINVAL, "unknown RH method %d", method);
    const uint32_t N = 1u << n, h = N >> 1;
    uint32_t b = 0;
    if (method == RH_BLOCK) {
        b = block > 0 ? (uint32_t)block : 1u << ((n - 1) / 2);   // Theorem 3: sqrt(2^(n-1))
        MERA_RETURN_IF((b & (b - 1)) != 0 || b > h || b > 256 || h / b > 512, MERA_EINVAL,
                       "block size %u: a power of two <= min(256, 2^(n-1)) with 2^(n-1)/b <= 512", b);
    }
    // order out's stream after in's queued work
    if (in->stream != out->stream) {
        cudaEvent_t ev;
        MERA_CHECK_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        cudaEventRecord(ev, in->stream);
        cudaStreamWaitEvent(out->stream, ev, 0);
        cudaEventDestroy(ev);
    }
    // scratch of `out`: the scaled state (Algorithm 1, first step) and the counter
    MERA_TRY(state_ensure_scratch(out, (size_t)N * sizeof(double2) + 256));
    double2* ss = reinterpret_cast<double2*>(out->scratch);
    unsigned long long* cnt =
        reinterpret_cast<unsigned long long*>(reinterpret_cast<char*>(out->scratch) + (size_t)N * sizeof(double2));
    cudaStream_t st = out->stream;
    MERA_CHECK_CUDA(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), st));
    launch_begin(st, MERA_KCLASS_RH, 32.0 * N);
    k_rh_scale<<<std::max(1u, std::min(N / 256u, 1024u)), 256, 0, st>>>(reinterpret_cast<const double2*>(in->data), ss,
                                                                      N, 1.0 / std::sqrt((double)N));
    MERA_TRY(launch_end(st));
    launch_begin(st, MERA_KCLASS_RH, 32.0 * N);
    double2* o = reinterpret_cast<double2*>(out->data);
    switch (method) {
    case RH_NONOPT: MERA_TRY(launch_rh<RH_NONOPT>(ss, o, n, b, cnt, st)); break;
    case RH_QUARTER: MERA_TRY(launch_rh<RH_QUARTER>(ss, o, n, b, cnt, st)); break;
    case RH_BLOCK: MERA_TRY(launch_rh<RH_BLOCK>(ss, o, n, b, cnt, st)); break;
    default: MERA_TRY(launch_rh<RH_LOG>(ss, o, n, b, cnt, st)); break;
    }
    MERA_TRY(launch_end(st));
    if (sign_count) {
        unsigned long long v = 0;
        MERA_CHECK_CUDA(cudaMemcpyAsync(&v, cnt, sizeof(v), cudaMemcpyDeviceToHost, st));
        MERA_CHECK_CUDA(cudaStreamSynchronize(st));
        *sign_count = v;
    }
    return MERA_OK;
}
