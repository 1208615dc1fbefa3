// Device helpers and per-gate kernels (the launchers live in gates.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "mera.h"

namespace mera {

// --------------------------------------------------------- complex math --
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(fma(a.x, b.x, -(a.y * b.y)), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -(a.y * b.y)), fmaf(a.x, b.y, a.y * b.x));
}
// acc + a * b
__device__ __forceinline__ double2 cfma(double2 a, double2 b, double2 acc) {
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(a.y, b.x, acc.y);
    return acc;
}
__device__ __forceinline__ float2 cfma(float2 a, float2 b, float2 acc) {
    acc.x = fmaf(a.x, b.x, acc.x);
    acc.x = fmaf(-a.y, b.y, acc.x);
    acc.y = fmaf(a.x, b.y, acc.y);
    acc.y = fmaf(a.y, b.x, acc.y);
    return acc;
}
__device__ __forceinline__ double2 czero(double2) { return make_double2(0.0, 0.0); }
__device__ __forceinline__ float2 czero(float2) { return make_float2(0.f, 0.f); }

// m0 * x0 + m1 * x1
template <typename V>
__device__ __forceinline__ V cdot2(V m0, V x0, V m1, V x1) {
    V acc = cmul(m0, x0);
    return cfma(m1, x1, acc);
}
template <typename V>
__device__ __forceinline__ V vsum(V a, V b) {
    a.x += b.x;
    a.y += b.y;
    return a;
}
template <typename V>
__device__ __forceinline__ V vdiff(V a, V b) {
    a.x -= b.x;
    a.y -= b.y;
    return a;
}
template <typename V, typename R>
__device__ __forceinline__ V vscale(V a, R r) {
    a.x *= r;
    a.y *= r;
    return a;
}

// int64 fixed-point complex (block floating point inside a fused tile).
// Coefficients are Q62: value * 2^62 as int64 (|value| < 2).
struct __align__(16) I2 {
    long long x, y;
};

// (a * c) >> 62 with the full 128-bit product (truncating).
__device__ __forceinline__ long long mulq62(long long a, long long c) {
    const long long hi = __mul64hi(a, c);
    const unsigned long long lo = (unsigned long long)a * (unsigned long long)c;
    return (long long)(((unsigned long long)hi << 2) | (lo >> 62));
}
// c * a for a Q62 coefficient c
__device__ __forceinline__ I2 cmul(I2 c, I2 a) {
    I2 r;
    r.x = mulq62(c.x, a.x) - mulq62(c.y, a.y);
    r.y = mulq62(c.x, a.y) + mulq62(c.y, a.x);
    return r;
}
__device__ __forceinline__ I2 cfma(I2 c, I2 a, I2 acc) {
    acc.x += mulq62(c.x, a.x) - mulq62(c.y, a.y);
    acc.y += mulq62(c.x, a.y) + mulq62(c.y, a.x);
    return acc;
}
// v * 2^-S rounded to nearest even (values below the normal range flush to 0).
__device__ __forceinline__ double fix2d(long long v, int S) {
    if (v == 0) return 0.0;
    const unsigned long long sgn = v < 0 ? (1ull << 63) : 0ull;
    const unsigned long long a = v < 0 ? (unsigned long long)(-v) : (unsigned long long)v;
    int lz = __clzll((long long)a);
    const unsigned long long m = a << lz;
    unsigned long long r = m >> 11;
    const unsigned long long rem = m & 0x7FFull;
    if (rem > 0x400ull || (rem == 0x400ull && (r & 1ull))) {
        r += 1;
        if (r >> 53) {
            r >>= 1;
            lz -= 1;
        }
    }
    const int e = (63 - lz) - S + 1023;
    if (e <= 0) return __longlong_as_double((long long)sgn);
    return __longlong_as_double((long long)(sgn | ((unsigned long long)e << 52) | (r & 0xFFFFFFFFFFFFFull)));
}


// Resident fixed point: a table entry d (|d| <= 1) in Q61, each part split
// as h * 2^31 + l with 0 <= l < 2^31 (stored as int32 rh, rl, ih, il).
// For |x| < 2^59 split the same way, x * d / 2^61 is
// 2 xh dh + (xh dl + xl dh + xl dl / 2^31) / 2^30: six 32x32->64
// multiply-adds and two 32-bit high products per component, rounded to
// nearest (error <= 1/2 unit plus 2^-30; zero stays zero, so amplitudes
// that must vanish do not feed later butterflies).
__device__ __forceinline__ void qsplit(long long x, int& h, int& l) {
    h = (int)(x >> 31);
    l = (int)((unsigned)x & 0x7FFFFFFFu);
}
// (a * b) >> 31 for 0 <= a, b < 2^31, to within one unit
__device__ __forceinline__ long long qlow(int a, int b) { return (long long)(__umulhi((unsigned)a, (unsigned)b) << 1); }
__device__ __forceinline__ long long qcombine(long long m1, long long m2) {
    return 2 * m1 + ((m2 + (1ll << 29)) >> 30);
}
// x * c / 2^61 for |x| < 2^60 and a Q61 value c with |c| < 2^61.5, both
// split into 31-bit limbs, rounded to nearest
__device__ __forceinline__ long long qmul_q(long long x, int ch, int cl) {
    int h, l;
    qsplit(x, h, l);
    return qcombine((long long)h * ch, (long long)h * cl + (long long)l * ch + qlow(l, cl));
}
// Complex product with three real products (c + id)(a + ib):
// k1 = c (a + b), k2 = a (d - c), k3 = b (c + d); re = k1 - k3, im = k1 + k2
// (each k rounded to nearest: error <= 1 unit per part, unbiased, 0 stays 0).
__device__ __forceinline__ I2 qcmul(int4 d, I2 x) {
    const long long c = ((long long)d.x << 31) + (long long)(unsigned)d.y;
    const long long e = ((long long)d.z << 31) + (long long)(unsigned)d.w;
    const long long dmc = e - c, cpd = c + e;
    const long long k1 = qmul_q(x.x + x.y, d.x, d.y);
    const long long k2 = qmul_q(x.x, (int)(dmc >> 31), (int)((unsigned)dmc & 0x7FFFFFFFu));
    const long long k3 = qmul_q(x.y, (int)(cpd >> 31), (int)((unsigned)cpd & 0x7FFFFFFFu));
    I2 r;
    r.x = k1 - k3;
    r.y = k1 + k2;
    return r;
}
// Complex product for a table entry c + is (split Q61 limbs as stored)
// with four real products and without the low-by-low limb terms: each
// component accumulates its middle terms in one 64-bit sum (below 2^63 for
// |x| < 2^59) and rounds once; the dropped terms are replaced by their mean
// over uniform low limbs (0 for the real part, one unit for the imaginary
// part), which bounds the error by about two units per component.  Fewer
// ALU instructions than the three-product form; measured faster in the
// monomial run pass.
__device__ __forceinline__ I2 qcmul4_fast(int4 d, I2 x) {
    int xh, xl, yh, yl;
    qsplit(x.x, xh, xl);
    qsplit(x.y, yh, yl);
    const long long m1r = (long long)xh * d.x - (long long)yh * d.z;
    const long long m2r = (long long)xh * d.y + (long long)xl * d.x - (long long)yh * d.w - (long long)yl * d.z;
    const long long m1i = (long long)xh * d.z + (long long)yh * d.x;
    const long long m2i = (long long)xh * d.w + (long long)xl * d.z + (long long)yh * d.y + (long long)yl * d.x;
    I2 r;
    r.x = 2 * m1r + ((m2r + (1ll << 29)) >> 30);
    r.y = 2 * m1i + ((m2i + (3ll << 29)) >> 30);
    return r;
}
__device__ __forceinline__ long long sneg(long long v) { return -v; }
__device__ __forceinline__ I2 neg_v(I2 x) {
    x.x = -x.x;
    x.y = -x.y;
    return x;
}

// Multiply by a phase given as a code: 0 -> 1, 1 -> i, 2 -> -1, 3 -> -i
// (exact: only moves and sign flips), 4 -> the general value v.
// Sign flips as integer operations on the sign bit.  The XOR is inline PTX
// so that the compiler cannot turn it back into a floating-point negation
// (which would occupy the FP64 pipe, ~57x scarcer than the integer ALUs).
__device__ __forceinline__ int xor_sign(int h) {
    int r;
    asm("xor.b32 %0, %1, 0x80000000;" : "=r"(r) : "r"(h));
    return r;
}
__device__ __forceinline__ double dneg(double v) {
    return __hiloint2double(xor_sign(__double2hiint(v)), __double2loint(v));
}
__device__ __forceinline__ float fneg(float v) { return __int_as_float(xor_sign(__float_as_int(v))); }
// v with its sign bit XORed with bit 31 of m (m is 0 or 0x80000000)
__device__ __forceinline__ int xor_reg(int h, int m) {
    int r;
    asm("xor.b32 %0, %1, %2;" : "=r"(r) : "r"(h), "r"(m));
    return r;
}
__device__ __forceinline__ double flip_sign(double v, int m) {
    return __hiloint2double(xor_reg(__double2hiint(v), m), __double2loint(v));
}
__device__ __forceinline__ float flip_sign(float v, int m) { return __int_as_float(xor_reg(__float_as_int(v), m)); }
__device__ __forceinline__ long long flip_sign(long long v, int m) {
    const long long s = (long long)(m >> 31);   // 0 or -1 (arithmetic shift)
    return (v ^ s) - s;
}
__device__ __forceinline__ double sneg(double v) { return dneg(v); }
__device__ __forceinline__ float sneg(float v) { return fneg(v); }
__device__ __forceinline__ double2 neg_v(double2 x) { return make_double2(dneg(x.x), dneg(x.y)); }
__device__ __forceinline__ float2 neg_v(float2 x) { return make_float2(fneg(x.x), fneg(x.y)); }
template <typename V>
__device__ __forceinline__ V apply_phase(int code, V v, V x) {
    V r;
    switch (code) {
    case 0: return x;
    case 1: r = x; r.x = sneg(x.y); r.y = x.x; return r;
    case 2: return neg_v(x);
    case 3: r = x; r.x = x.y; r.y = sneg(x.x); return r;
    default: return cmul(v, x);
    }
}

// Insert a zero bit at each position ins[0] < ins[1] < ... of t.
__device__ __forceinline__ uint64_t insert_zeros(uint64_t t, const int* ins, int nins) {
    for (int j = 0; j < nins; ++j) {
        const uint64_t lo = t & ((1ull << ins[j]) - 1ull);
        t = ((t - lo) << 1) | lo;
    }
    return t;
}

// ------------------------------------------------------ per-gate kernels --
template <typename V>
struct GateArgs {
    V* psi;
    uint64_t count;              // groups (or elements) to visit
    uint64_t cbits;              // control values at their bit positions
    uint64_t off[8];             // offset of sub-index s inside a group
    int nins;                    // zero bits inserted into the group counter
    int ins[MERA_MAX_QUBITS];    // their positions, ascending
    int k;                       // targets
    int qc;                      // shuffle kernel: target among non-control bits
    int nt;                      // diag kernel: targets
    int tq[3];                   // diag kernel: target qubits, tq[0] most significant
    int nact;                    // monomial: rows that change
    int act[8];                  // monomial: those rows
    int perm[8];                 // monomial: source sub-index of act[j]
    int flag[8];                 // diag: value != 1 for sub-index s
    int code[8];                 // phase code of v[] (see apply_phase)
    int hmode;                   // one target: 1 = the real butterfly r [[1, 1], [1, -1]] (r = m[0].x)
    V v[8];                      // monomial / diag values
    V m[64];                     // dense matrix, row-major
};

// Multiply one sub-space (controls = cbits) by a scalar; four amplitudes a
// grid stride apart per thread and iteration, loads first.
template <typename V>
__global__ void __launch_bounds__(256) k_phase(const __grid_constant__ GateArgs<V> a) {
    constexpr int U = 4;
    const V v = a.v[0];
    const int code = a.code[0];
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t t0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t0 < a.count; t0 += stride * U) {
        uint64_t idx[U];
        V x[U];
#pragma unroll
        for (int u = 0; u < U; ++u) idx[u] = insert_zeros(t0 + (uint64_t)u * stride, a.ins, a.nins) | a.cbits;
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (t0 + (uint64_t)u * stride < a.count) x[u] = __ldcs(a.psi + idx[u]);
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (t0 + (uint64_t)u * stride < a.count) __stcs(a.psi + idx[u], apply_phase(code, v, x[u]));
    }
}

// Diagonal gate: amplitude i (controls holding) times v[sub(i)] where v != 1;
// four amplitudes a grid stride apart per thread and iteration, loads
// first.  For complex128 with general phases the complex multiply (four
// FP64 operations) bounds it on GB300, ~2 SM clocks per amplitude against
// an HBM budget of ~1.5; an integer product of 31-bit limbs on a share of
// the warps was measured slower (its wide multiplies compete for the same
// issue budget).
template <typename V>
__global__ void __launch_bounds__(256) k_diag(const __grid_constant__ GateArgs<V> a) {
    constexpr int U = 4;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t t0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t0 < a.count; t0 += stride * U) {
        uint64_t idx[U];
        int sub[U];
        bool on[U];
        V x[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint64_t t = t0 + (uint64_t)u * stride;
            idx[u] = insert_zeros(t, a.ins, a.nins) | a.cbits;
            int sb = 0;
            for (int j = 0; j < a.nt; ++j) sb = (sb << 1) | (int)((idx[u] >> a.tq[j]) & 1ull);
            sub[u] = sb;
            on[u] = t < a.count && a.flag[sb];
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (on[u]) x[u] = a.psi[idx[u]];
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (on[u]) a.psi[idx[u]] = apply_phase(a.code[sub[u]], a.v[sub[u]], x[u]);
    }
}

// One target, high bit: each thread owns the pair (i0, i0 | off[1]).
// MONO: the gate swaps the pair and multiplies by phases (X, Y and their
// controlled forms): no arithmetic for unit phases.
template <typename V, bool MONO>
__device__ __forceinline__ void pair_update(const GateArgs<V>& a, V& x0, V& x1) {
    if (MONO) {
        const V n0 = apply_phase(a.code[0], a.v[0], x1);
        const V n1 = apply_phase(a.code[1], a.v[1], x0);
        x0 = n0;
        x1 = n1;
    } else if (a.hmode) {
        // Hadamard-type: two adds and two multiplies per component pair
        // instead of a general complex 2x2 product
        const auto r = a.m[0].x;
        const V n0 = vsum(x0, x1), n1 = vdiff(x0, x1);
        x0 = vscale(n0, r);
        x1 = vscale(n1, r);
    } else {
        const V n0 = cdot2(a.m[0], x0, a.m[1], x1);
        const V n1 = cdot2(a.m[2], x0, a.m[3], x1);
        x0 = n0;
        x1 = n1;
    }
}

template <typename V, bool MONO>
__global__ void __launch_bounds__(256) k_dense1_pair(const __grid_constant__ GateArgs<V> a) {
    const uint64_t o = a.off[1];
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    // two groups in flight per thread
    for (; t + stride < a.count; t += 2 * stride) {
        const uint64_t i0 = insert_zeros(t, a.ins, a.nins) | a.cbits;
        const uint64_t j0 = insert_zeros(t + stride, a.ins, a.nins) | a.cbits;
        V x0 = a.psi[i0], x1 = a.psi[i0 | o];
        V y0 = a.psi[j0], y1 = a.psi[j0 | o];
        pair_update<V, MONO>(a, x0, x1);
        pair_update<V, MONO>(a, y0, y1);
        a.psi[i0] = x0;
        a.psi[i0 | o] = x1;
        a.psi[j0] = y0;
        a.psi[j0 | o] = y1;
    }
    if (t < a.count) {
        const uint64_t i0 = insert_zeros(t, a.ins, a.nins) | a.cbits;
        V x0 = a.psi[i0], x1 = a.psi[i0 | o];
        pair_update<V, MONO>(a, x0, x1);
        a.psi[i0] = x0;
        a.psi[i0 | o] = x1;
    }
}

// One target, low bit: one amplitude per thread, the partner comes from the
// lane 1 << qc away (consecutive threads hold consecutive non-control
// indices, so every load and store is fully coalesced).
template <typename V>
__device__ __forceinline__ V shfl_xor_v(V x, int m);
template <>
__device__ __forceinline__ double2 shfl_xor_v<double2>(double2 x, int m) {
    return make_double2(__shfl_xor_sync(0xffffffffu, x.x, m), __shfl_xor_sync(0xffffffffu, x.y, m));
}
template <>
__device__ __forceinline__ float2 shfl_xor_v<float2>(float2 x, int m) {
    return make_float2(__shfl_xor_sync(0xffffffffu, x.x, m), __shfl_xor_sync(0xffffffffu, x.y, m));
}

template <typename V, bool MONO>
__global__ void __launch_bounds__(256) k_dense1_shfl(const __grid_constant__ GateArgs<V> a) {
    const V m0 = a.m[0], m1 = a.m[1], m2 = a.m[2], m3 = a.m[3];
    const int lm = 1 << a.qc;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;   // multiple of 32
    for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < a.count; t += stride) {
        const uint64_t i = insert_zeros(t, a.ins, a.nins) | a.cbits;
        const V x = a.psi[i];
        const V y = shfl_xor_v(x, lm);
        const int hi = (int)((t >> a.qc) & 1ull);
        if (MONO) a.psi[i] = apply_phase(a.code[hi], a.v[hi], y);
        else if (a.hmode) a.psi[i] = vscale(hi ? vdiff(y, x) : vsum(x, y), m0.x);
        else a.psi[i] = hi ? cdot2(m2, y, m3, x) : cdot2(m0, x, m1, y);
    }
}

// Monomial gate on 2-3 targets: row act[j] takes v[j] * amplitude perm[j].
template <typename V>
__global__ void __launch_bounds__(256) k_mono(const __grid_constant__ GateArgs<V> a) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < a.count; t += stride) {
        const uint64_t base = insert_zeros(t, a.ins, a.nins) | a.cbits;
        V in[8];
#pragma unroll
        for (int j = 0; j < 8; ++j)
            if (j < a.nact) in[j] = a.psi[base | a.off[a.perm[j]]];
#pragma unroll
        for (int j = 0; j < 8; ++j)
            if (j < a.nact) a.psi[base | a.off[a.act[j]]] = apply_phase(a.code[j], a.v[j], in[j]);
    }
}

// Dense gate on K targets.
template <typename V, int K>
__global__ void __launch_bounds__(256) k_dense_k(const __grid_constant__ GateArgs<V> a) {
    constexpr int D = 1 << K;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < a.count; t += stride) {
        const uint64_t base = insert_zeros(t, a.ins, a.nins) | a.cbits;
        V in[D];
#pragma unroll
        for (int s = 0; s < D; ++s) in[s] = a.psi[base | a.off[s]];
#pragma unroll
        for (int r = 0; r < D; ++r) {
            V acc = cmul(a.m[r * D], in[0]);
#pragma unroll
            for (int c = 1; c < D; ++c) acc = cfma(a.m[r * D + c], in[c], acc);
            a.psi[base | a.off[r]] = acc;
        }
    }
}

}  // namespace mera
