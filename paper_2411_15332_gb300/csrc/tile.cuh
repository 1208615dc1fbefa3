// Fused tile-pass kernel.
//
// A pass owns K "tile bits" (global bit positions tpos[0..K-1], always
// including the lowest bits so that every tile is a set of contiguous
// 128-byte runs).  Each CTA loads one tile -- the 2^K amplitudes whose other
// bits are fixed -- and applies a run of gates whose targets are tile bits
// (controls and diagonal gates may sit on any bit).  Inside the tile the
// work is split into phases: in a phase each thread holds 2^FR amplitudes
// in registers that differ in FR chosen "register bits"; gates on those
// bits are applied in registers; between phases the tile is exchanged
// through shared memory.  High qubits enter the tile by being named in
// tpos: the tile is gathered from HBM with those qubits as local bits,
// which is the qubit-index swap done on the fly.
//
// Arithmetic engines.  GB300 issues about two FP64 FMAs per clock per SM
// against ~114 FP32 FMAs and ~80 integer adds, so complex128 work avoids
// FP64 where it can:
//  * ENG_FP  : float32 arithmetic for complex64 states.
//  * ENG_Q   : complex128 states held in HBM as int64 fixed point for the
//              whole run of passes of one circuit (value * 2^(S - g), S
//              from a bound of the state norm computed on the device, which
//              unitary passes preserve; g the headroom a pass needs).  Only
//              the first pass of a run converts from doubles and only the
//              last converts back; butterflies, moves and sign flips are
//              exact; table and gate multiplies are 32x32->64 integer
//              products of 31-bit limbs rounded to nearest; the 2^{-m/2}
//              Hadamard scale is a shift (times 1/sqrt(2) for odd m).  The
//              planner uses it for circuits whose mixing gates all precede
//              a monomial body (phases and permutations keep every
//              amplitude's magnitude, so a global scale loses nothing).
//  * ENG_I64 : complex128 states kept as float64 in HBM.  The tile is
//              converted once to int64 block floating point (one exponent
//              per tile, from the tile maximum): butterflies are exact
//              integer adds, permutations and {1, i, -1, -i} phases are moves
//              and sign flips, and every multiplication is the same rounded
//              product of 31-bit limbs as in ENG_Q; the pass's 2^{-m/2}
//              Hadamard scale is applied at phase exits (in the Hadamard-
//              pass kernel) and on the way out.
// In both engines a run of diagonal gates folds into exact sign / i terms
// (TOP_Z4) and one table lookup plus one complex multiply per amplitude
// (TOP_DSEP).
#pragma once

#include <cuda.h>   // CUtensorMap (the type only; maps are encoded on the host)
#include <type_traits>

#include "kernels.cuh"

namespace mera {

constexpr int FR = 4;              // register bits per thread
constexpr int FRA = 1 << FR;       // amplitudes per thread
constexpr int TILE_MAX_PHASES = 32;
constexpr int TILE_MAX_OPS = 160;
constexpr int TILE_MAX_COEF = 448;
constexpr int TILE_MAX_Z4 = 96;
constexpr int TILE_MAX_NT = 48;    // non-tile factors of separable diagonals

enum TileEngine { ENG_FP = 0, ENG_I64 = 1, ENG_Q = 2 };

// Kernel variants by the op kinds a pass holds (Z4 terms are always
// compiled in; FEAT_GATES: Hadamard butterflies and one-target monomials):
// fewer op bodies, fewer live registers, less instruction cache.
enum TileFeature { FEAT_DIAG = 1, FEAT_DENSE1 = 2, FEAT_G2 = 4, FEAT_GATES = 8, FEAT_ALL = 15 };

enum TileOpType : int8_t {
    TOP_G1 = 0,       // dense 2x2 on one register bit (coef[0..3])
    TOP_G1MONO = 1,   // swap of the pair with phases (codes / coef[0..1])
    TOP_H = 2,        // unscaled Hadamard butterfly (pass scale at the end)
    TOP_G2 = 3,       // dense 4x4 on register bits a > b
    TOP_G2MONO = 4,   // monomial 4x4: row s takes phase(s) * amp perm(s)
    TOP_G1SWAP = 5,   // swap of the pair (X, CNOT, Toffoli): moves only
    // 6: unused (three-target gates run as per-gate kernels between passes)
    TOP_DIAG = 7,     // diagonal on any bits: amp *= v[sub] where flagged
    TOP_DSEP = 8,     // separable diagonal: amp *= tab[local index] * prod(non-tile factors)
    TOP_Z4 = 9,       // product of exact phases i^e over pattern terms
};

// TOP_G1 flags: bit s (s = 0..3) set when matrix entry s is imaginary;
// G1_RI when every entry is real or imaginary
constexpr uint32_t G1_RI = 16u;

struct TileOp {
    int8_t type;
    int8_t a, b, c;      // register bits (a is the most significant sub-index bit); c: 1 = per-state
                         // coefficients; sign terms: 2 = matched on the scattered store index
    int8_t nt;           // diag: number of targets; dsep: non-tile factors
    int8_t tq[3];        // diag: global target positions (tq[0] most significant)
    int32_t coef;        // first coefficient in PassArgs::coef
    uint32_t flags;      // diag: bit s set when sub-index s changes; g1: see G1_RI
    uint32_t codes;      // phase codes, 3 bits per row / sub-index
    uint32_t perm;       // monomial: source sub-index of row s, 3 bits per row
    int32_t aux;         // dsep: table offset (elements); z4: first term
    int32_t aux2;        // dsep: first non-tile position; z4: number of terms
    uint64_t cmask;      // control qubits (global positions)
    uint64_t cvals;      // their required values
};

struct Z4Term {
    uint64_t mask, vals;  // amplitude gets i^e when (index & mask) == vals
    int32_t e;
    int32_t pad;
};

// Shared-memory slot map of one side of an exchange: the slot of a
// thread's register slot j is the XOR of tc[t] over the set bits t of the
// thread index and of rc[r] over the set bits r of j.  The maps are linear
// over GF(2): a swizzle Z (bank spreading) composed, on the writing side,
// with the affine index permutation the exchange applies.
constexpr int TILE_MAX_XOFF = 6;
struct XSide {
    int16_t tc[12];
    int16_t rc[FR];
};

// Writing side of an exchange: the slot map plus a block-dependent offset
// (XOR of offv[i] where the tile's bit at global position offq[i] is set).
struct XOut {
    XSide s;
    int16_t off0;
    int8_t noff;
    int8_t offq[TILE_MAX_XOFF];
    int16_t offv[TILE_MAX_XOFF];
};

// Global-index map of a load or store with a permutation folded in: the
// thread's register slot j sits at tile base XOR c XOR (XOR of tc[t] over
// the set bits t of the thread index) XOR (XOR of rc[r] over the set bits
// r of j) XOR (XOR of w[i] where the tile's global bit q[i] is set).
struct GMap {
    unsigned long long tc[12];
    unsigned long long rc[FR];
    unsigned long long c;
    unsigned long long w[TILE_MAX_XOFF];
    int8_t q[TILE_MAX_XOFF];
    int8_t nq;
};

struct TilePhase {
    int8_t rb[FR];       // local tile bits held in registers, ascending
    int16_t op_begin, op_end;
    int8_t permuted;     // 1: the exit map differs from the entry map (all reads finish first)
    int8_t qsh;          // int64 engines: rounded right shift at the exit (part of the 2^(-nh/2) scale)
    XSide in;            // slots this phase reads (from the previous exchange or the load staging)
    XOut out;            // slots this phase writes (next exchange or the store staging)
};

template <typename V>
struct PassArgs {
    V* psi;
    V* psi_out;          // null: in place; else the pass writes here (same layout)
    const V* tab;        // separable-diagonal tables (device), 2^K entries each
    // batches of states (blockIdx.y): state = psi + slot * bstride with
    // slot = slots[blockIdx.y] (or blockIdx.y when slots is NULL); ops with
    // c == 1 read their coefficients from bcoef + blockIdx.y * bcstride
    const int* slots;
    unsigned long long bstride;
    const V* bcoef;
    int bcstride;
    int K;               // tile bits
    int nph;             // phases
    int load_smem;       // 1: stage the first phase's load through shared memory
    int store_smem;      // 1: stage the last phase's store through shared memory
    double scale;        // ENG_FP: applied at the end of the pass
    int nh;              // Hadamard butterflies in the pass (ENG_I64 / ENG_Q scale by 2^-nh/2)
    int q_in, q_out;     // ENG_Q: 1 = the state is read / written as fixed point, 0 = as doubles
    int qgi, qgo;        // ENG_Q: headroom bits of the input / output format (value * 2^(*qS - g))
    int qend;            // int64 engines: Hadamard levels scaled at the end of the pass (the rest
                         // went at phase exits, qsh; ENG_I64 may carry one level to another pass)
    const int* qS;       // ENG_Q: device address of S = 59 - floor(log2 of a norm bound)
    int guard;           // ENG_I64: headroom bits of the fixed-point format
    int tpos[16];        // global bit of local bit j, ascending
    XSide ld;            // load staging: slot of element tid + i * 2^(K-FR)
    XSide st;            // store staging: the same for the final copy out
    int gather, scatter; // 1: phase 0 loads through gin / the last phase stores through gout
    int bulk;            // Hadamard-pass kernel: 1 = the load staging is in natural chunk order (bulk copies)
    GMap gin, gout;      // (a permutation at the start / end of the pass rides on the addresses)
    int8_t ntq[TILE_MAX_NT];   // global positions of separable non-tile factors
    TilePhase ph[TILE_MAX_PHASES];
    TileOp ops[TILE_MAX_OPS];
    Z4Term z4[TILE_MAX_Z4];
    V coef[TILE_MAX_COEF];
};

template <typename V>
struct IsFP {
    static constexpr bool value = true;
};
template <>
struct IsFP<I2> {
    static constexpr bool value = false;
};

// ----------------------------------------------------------- bit helpers --
// Deposit the bits of local index l at the global positions tpos[].
__device__ __forceinline__ uint64_t spread_bits(uint32_t l, const int* tpos, int K) {
    uint64_t g = 0;
    for (int j = 0; j < K; ++j)
        if ((l >> j) & 1u) g |= 1ull << tpos[j];
    return g;
}

// Insert zeros at the FR register positions (ascending) into t.
__device__ __forceinline__ uint32_t insert_reg_zeros(uint32_t t, const int8_t* rb) {
#pragma unroll
    for (int r = 0; r < FR; ++r) {
        const uint32_t lo = t & ((1u << rb[r]) - 1u);
        t = ((t - lo) << 1) | lo;
    }
    return t;
}

// Offset of register slot j: OR of the masks of its set bits (j is a
// compile-time constant after unrolling).
template <typename T>
__device__ __forceinline__ T dep4(int j, const T* m) {
    T r = 0;
    if (j & 1) r |= m[0];
    if (j & 2) r |= m[1];
    if (j & 4) r |= m[2];
    if (j & 8) r |= m[3];
    return r;
}

__device__ __forceinline__ int code_at(uint32_t codes, int s) { return (int)((codes >> (3 * s)) & 7u); }

// XOR of the masks of the set bits of j (slot offsets under the linear
// swizzle).
__device__ __forceinline__ int dep4x(int j, const int* m) {
    int r = 0;
    if (j & 1) r ^= m[0];
    if (j & 2) r ^= m[1];
    if (j & 4) r ^= m[2];
    if (j & 8) r ^= m[3];
    return r;
}

// Slot base of a thread on one side of an exchange.
__device__ __forceinline__ int xbase(const XSide& s, uint32_t tid) {
    int v = 0;
#pragma unroll
    for (int t = 0; t < 12; ++t) v ^= (-(int)((tid >> t) & 1u)) & (int)s.tc[t];
    return v;
}

__device__ __forceinline__ int xbase_out(const XOut& o, uint32_t tid, uint64_t gb) {
    int v = xbase(o.s, tid) ^ (int)o.off0;
    for (int i = 0; i < o.noff; ++i)
        if ((gb >> o.offq[i]) & 1ull) v ^= (int)o.offv[i];
    return v;
}

__device__ __forceinline__ uint64_t gbase(const GMap& g, uint32_t tid, uint64_t tb) {
    uint64_t v = tb ^ g.c;
#pragma unroll
    for (int t = 0; t < 12; ++t) v ^= (0ull - (uint64_t)((tid >> t) & 1u)) & g.tc[t];
    for (int i = 0; i < g.nq; ++i)
        if ((tb >> g.q[i]) & 1ull) v ^= g.w[i];
    return v;
}
template <typename T>
__device__ __forceinline__ T dep4xl(int j, const T* m) {
    T r = 0;
    if (j & 1) r ^= m[0];
    if (j & 2) r ^= m[1];
    if (j & 4) r ^= m[2];
    if (j & 8) r ^= m[3];
    return r;
}

// 16-bit mask of this thread's register slots whose controls hold: the
// non-register control bits are fixed for the thread, the register ones
// select slots.
__device__ __forceinline__ uint32_t active16(uint64_t cmask, uint64_t cvals, uint64_t gb, const uint64_t* gm) {
    if (cmask == 0) return 0xFFFFu;
    const uint64_t regm = gm[0] | gm[1] | gm[2] | gm[3];
    if ((gb & cmask & ~regm) != (cvals & ~regm)) return 0u;
    uint32_t pat = 0xFFFFu;
    const uint32_t b1[4] = {0xAAAAu, 0xCCCCu, 0xF0F0u, 0xFF00u};
#pragma unroll
    for (int r = 0; r < FR; ++r)
        if (cmask & gm[r]) pat &= (cvals & gm[r]) ? b1[r] : ~b1[r];
    return pat & 0xFFFFu;
}

// x * i^k, branch free (k in 0..3).
template <typename V>
__device__ __forceinline__ V mul_ik(V x, int k) {
    V r = x;
    if (k & 1) {
        r.x = x.y;
        r.y = x.x;
    }
    // sign masks: re negated for k = 1, 2; im for k = 2, 3
    const int mx = (int)((unsigned)(((k + 1) >> 1) & 1) << 31), my = (int)((unsigned)((k >> 1) & 1) << 31);
    r.x = flip_sign(r.x, mx);
    r.y = flip_sign(r.y, my);
    return r;
}

// --------------------------------------------------- engine primitives --
template <typename V>
__device__ __forceinline__ V vadd(V a, V b) {
    a.x += b.x;
    a.y += b.y;
    return a;
}
template <typename V>
__device__ __forceinline__ V vsub(V a, V b) {
    a.x -= b.x;
    a.y -= b.y;
    return a;
}

// Exact phase codes 0..3 (moves and sign flips); code 4 multiplies by v
// (FP, or Q62 fixed point in the int64 engine).
template <typename V>
__device__ __forceinline__ V phase_any(int code, V v, V x) {
    return apply_phase(code, v, x);
}

// Read-only table entry.
__device__ __forceinline__ double2 tab_ld(const double2* p) { return __ldg(p); }
__device__ __forceinline__ float2 tab_ld(const float2* p) { return __ldg(p); }
__device__ __forceinline__ I2 tab_ld(const I2* p) {
    const longlong2 v = __ldg(reinterpret_cast<const longlong2*>(p));
    I2 r;
    r.x = v.x;
    r.y = v.y;
    return r;
}

// ------------------------------------------- int64 block floating point --
// Biased exponent field of a double (0 for zero / subnormal).
__device__ __forceinline__ int dexp(double v) {
    return (int)((__double_as_longlong(v) >> 52) & 0x7FF);
}

// round(v * 2^S) as int64, for |v| * 2^S < 2^62 (subnormals read as 0).
__device__ __forceinline__ long long d2fix(double v, int S) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const int e = (int)((b >> 52) & 0x7FF);
    if (e == 0) return 0;
    const unsigned long long m = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    const int sh = S + e - 1075;
    unsigned long long a;
    if (sh >= 0) a = m << sh;
    else if (sh > -64) a = (m + (1ull << (-sh - 1))) >> (-sh);
    else a = 0;
    return (b >> 63) ? -(long long)a : (long long)a;
}

// x * d for a complex128 amplitude held as doubles and a Q62 table entry d
// (|d| <= 1) without FP64 instructions: both parts of x are aligned to the
// larger of their exponents as 62-bit integers, multiplied with full
// 128-bit products (Q62) and rounded back to double (nearest even).  Zero
// and subnormal parts read as 0.  Error: about one unit in the last place
// of max(|Re x|, |Im x|).
__device__ __forceinline__ long long align62(long long b, int eb, int e) {
    if (eb == 0 || e - eb > 61) return 0;
    const long long m = (long long)((((unsigned long long)b & 0xFFFFFFFFFFFFFull) | (1ull << 52)) << 9) >> (e - eb);
    return b < 0 ? -m : m;
}
__device__ __forceinline__ double2 icmul(I2 d, double2 x) {
    const long long br = __double_as_longlong(x.x), bi = __double_as_longlong(x.y);
    const int er = (int)((br >> 52) & 0x7FF), ei = (int)((bi >> 52) & 0x7FF);
    const int e = max(er, ei);
    if (e == 0) return make_double2(0.0, 0.0);
    const long long xr = align62(br, er, e), xi = align62(bi, ei, e);
    const long long pr = mulq62(d.x, xr) - mulq62(d.y, xi);
    const long long pi = mulq62(d.x, xi) + mulq62(d.y, xr);
    const int S = 1084 - e;   // the products carry the scale 2^(e - 1075 - 9)
    return make_double2(fix2d(pr, S), fix2d(pi, S));
}

// d * x for a coefficient d that is real (imag == 0: limbs d.x, d.y of its
// real part) or imaginary (limbs d.z, d.w of its imaginary part): two real
// products instead of the three of a general complex product
__device__ __forceinline__ I2 qrimul(int4 d, uint32_t imag, I2 x) {
    I2 r;
    if (!imag) {
        r.x = qmul_q(x.x, d.x, d.y);
        r.y = qmul_q(x.y, d.x, d.y);
    } else {
        r.x = -qmul_q(x.y, d.z, d.w);
        r.y = qmul_q(x.x, d.z, d.w);
    }
    return r;
}
// x * c for a real Q61 constant c = ch * 2^31 + cl
__device__ __forceinline__ long long qmul_real(long long x, int ch, int cl) {
    int h, l;
    qsplit(x, h, l);
    return qcombine((long long)h * ch, (long long)h * cl + (long long)l * ch + qlow(l, cl));
}

// ------------------------------------------------------------ op bodies --
// Coefficient slot i as split Q61 limbs (ENG_Q coefficient format).
template <typename V>
__device__ __forceinline__ int4 qcoef(const V* cf, int i) {
    return *reinterpret_cast<const int4*>(cf + i);
}

template <typename V, int B, int ENG>
__device__ __forceinline__ void op_g1(V (&x)[FRA], const TileOp& o, const V* cf, uint64_t gb, const uint64_t* gm) {
    const uint32_t act = active16(o.cmask, o.cvals, gb, gm);
    if (act == 0) return;
    if constexpr (ENG == ENG_Q || ENG == ENG_I64) {
        const int4 q0 = qcoef(cf, 0), q1 = qcoef(cf, 1), q2 = qcoef(cf, 2), q3 = qcoef(cf, 3);
        if (o.flags & G1_RI) {
            // every entry real or imaginary (RX, RY, ...): two real products each
            const uint32_t im = o.flags;
#pragma unroll
            for (int j = 0; j < FRA; ++j) {
                if (j & (1 << B)) continue;
                const int j1 = j | (1 << B);
                if (!(act & (1u << j))) continue;
                const V a0 = x[j], a1 = x[j1];
                x[j] = vadd(qrimul(q0, im & 1u, a0), qrimul(q1, im & 2u, a1));
                x[j1] = vadd(qrimul(q2, im & 4u, a0), qrimul(q3, im & 8u, a1));
            }
            return;
        }
#pragma unroll
        for (int j = 0; j < FRA; ++j) {
            if (j & (1 << B)) continue;
            const int j1 = j | (1 << B);
            if (!(act & (1u << j))) continue;
            const V a0 = x[j], a1 = x[j1];
            x[j] = vadd(qcmul(q0, a0), qcmul(q1, a1));
            x[j1] = vadd(qcmul(q2, a0), qcmul(q3, a1));
        }
    } else {
        const V m0 = cf[0], m1 = cf[1], m2 = cf[2], m3 = cf[3];
#pragma unroll
        for (int j = 0; j < FRA; ++j) {
            if (j & (1 << B)) continue;
            const int j1 = j | (1 << B);
            if (!(act & (1u << j))) continue;
            const V a0 = x[j], a1 = x[j1];
            x[j] = cdot2(m0, a0, m1, a1);
            x[j1] = cdot2(m2, a0, m3, a1);
        }
    }
}

template <typename V, int B>
__device__ __forceinline__ void op_g1mono(V (&x)[FRA], const TileOp& o, const V* cf, uint64_t gb, const uint64_t* gm) {
    const uint32_t act = active16(o.cmask, o.cvals, gb, gm);
    if (act == 0) return;
    // phases are unit codes here (the planner sends other monomials to G1)
    const int c0 = code_at(o.codes, 0) & 3, c1 = code_at(o.codes, 1) & 3;
#pragma unroll
    for (int j = 0; j < FRA; ++j) {
        if (j & (1 << B)) continue;
        const int j1 = j | (1 << B);
        if (!(act & (1u << j))) continue;
        const V a0 = x[j], a1 = x[j1];
        x[j] = mul_ik(a1, c0);
        x[j1] = mul_ik(a0, c1);
    }
}

template <typename V, int B>
__device__ __forceinline__ void op_g1swap(V (&x)[FRA], const TileOp& o, uint64_t gb, const uint64_t* gm) {
    const uint32_t act = active16(o.cmask, o.cvals, gb, gm);
    if (act == 0) return;
#pragma unroll
    for (int j = 0; j < FRA; ++j) {
        if (j & (1 << B)) continue;
        const int j1 = j | (1 << B);
        if (!(act & (1u << j))) continue;
        const V t = x[j];
        x[j] = x[j1];
        x[j1] = t;
    }
}

template <typename V, int B>
__device__ __forceinline__ void op_h(V (&x)[FRA]) {
#pragma unroll
    for (int j = 0; j < FRA; ++j) {
        if (j & (1 << B)) continue;
        const int j1 = j | (1 << B);
        if constexpr (IsFP<V>::value) {
            const V a0 = x[j], a1 = x[j1];
            x[j] = vadd(a0, a1);
            x[j1] = vsub(a0, a1);
        } else {
            // integers: a - b = (a + b) - b - b exactly, so both results
            // overwrite their operands without a temporary
            x[j].x += x[j1].x;
            x[j].y += x[j1].y;
            x[j1].x = x[j].x - x[j1].x - x[j1].x;
            x[j1].y = x[j].y - x[j1].y - x[j1].y;
        }
    }
}

template <typename V, int A, int B, int ENG>
__device__ __forceinline__ void op_g2(V (&x)[FRA], const TileOp& o, const V* cf, uint64_t gb, const uint64_t* gm,
                                      bool mono) {
    const uint32_t act = active16(o.cmask, o.cvals, gb, gm);
    if (act == 0) return;
#pragma unroll
    for (int j = 0; j < FRA; ++j) {
        if (j & ((1 << A) | (1 << B))) continue;
        if (!(act & (1u << j))) continue;
        const int id[4] = {j, j | (1 << B), j | (1 << A), j | (1 << A) | (1 << B)};
        V in[4];
#pragma unroll
        for (int s = 0; s < 4; ++s) in[s] = x[id[s]];
        if (mono) {
#pragma unroll
            for (int s = 0; s < 4; ++s) {
                const int src = (int)((o.perm >> (3 * s)) & 7u);
                V v = in[0];
#pragma unroll
                for (int u = 1; u < 4; ++u)
                    if (src == u) v = in[u];
                x[id[s]] = mul_ik(v, code_at(o.codes, s) & 3);
            }
        } else if constexpr (ENG == ENG_Q || ENG == ENG_I64) {
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                V acc = qcmul(qcoef(cf, r * 4), in[0]);
#pragma unroll
                for (int c = 1; c < 4; ++c) acc = vadd(acc, qcmul(qcoef(cf, r * 4 + c), in[c]));
                x[id[r]] = acc;
            }
        } else {
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                V acc = cmul(cf[r * 4], in[0]);
#pragma unroll
                for (int c = 1; c < 4; ++c) acc = cfma(cf[r * 4 + c], in[c], acc);
                x[id[r]] = acc;
            }
        }
    }
}

template <typename V, int ENG>
__device__ __forceinline__ void op_diag(V (&x)[FRA], const TileOp& o, const V* cf, uint64_t gb, const uint64_t* gm) {
    const uint32_t act = active16(o.cmask, o.cvals, gb, gm);
    if (act == 0) return;
#pragma unroll
    for (int j = 0; j < FRA; ++j) {
        if (!(act & (1u << j))) continue;
        const uint64_t g = gb | dep4(j, gm);
        int sub = 0;
        for (int t = 0; t < o.nt; ++t) sub = (sub << 1) | (int)((g >> o.tq[t]) & 1ull);
        if (!((o.flags >> sub) & 1u)) continue;
        const int code = code_at(o.codes, sub);
        if constexpr (ENG == ENG_Q || ENG == ENG_I64) {
            x[j] = code < 4 ? mul_ik(x[j], code) : qcmul(qcoef(cf, sub), x[j]);
        } else {
            x[j] = phase_any(code, cf[sub], x[j]);
        }
    }
}

// Exact phase i^(sum of matching terms' exponents).  The 16 exponents are
// kept mod 4 as two 16-bit planes; each term adds its exponent to the
// slots its pattern selects.
template <typename V>
__device__ __forceinline__ void op_z4(V (&x)[FRA], const TileOp& o, const Z4Term* z4, uint64_t gb, const uint64_t* gm) {
    uint32_t p0 = 0, p1 = 0;
    for (int t = 0; t < o.aux2; ++t) {
        const Z4Term z = z4[o.aux + t];
        const uint32_t act = active16(z.mask, z.vals, gb, gm);
        if (z.e & 1) {
            const uint32_t c = p0 & act;
            p0 ^= act;
            p1 ^= c;
        }
        if (z.e & 2) p1 ^= act;
    }
    if ((p0 | p1) == 0) return;
#pragma unroll
    for (int j = 0; j < FRA; ++j) x[j] = mul_ik(x[j], (int)(((p0 >> j) & 1u) | (((p1 >> j) & 1u) << 1)));
}

// Separable diagonal: the product over tile-local qubits comes from a table
// indexed by the local index.  Up to DSEP_SEL_BITS non-tile qubits select
// one of 2^m pre-multiplied tables (the tile's bits are fixed); beyond that
// the remaining non-tile factors multiply in per tile.
constexpr int DSEP_SEL_BITS = 5;

template <typename V, int ENG>
__device__ __forceinline__ void op_dsep(V (&x)[FRA], const TileOp& o, const V* cf, const V* tab, const int8_t* ntq,
                                        uint32_t lb, const int* lm, uint64_t gb, int K) {
    const int nsel = o.nt < DSEP_SEL_BITS ? o.nt : DSEP_SEL_BITS;
    uint32_t sel = 0;
    for (int f = 0; f < nsel; ++f) sel |= (uint32_t)((gb >> ntq[o.aux2 + f]) & 1ull) << f;
    if constexpr (ENG == ENG_Q || ENG == ENG_I64) {
        // split-Q61 tables; per-tile factors multiply separately
        const int4* t = reinterpret_cast<const int4*>(tab) + o.aux + ((size_t)sel << K);
        // groups of four entries in flight (an empty asm with a memory
        // clobber keeps the compiler from hoisting all sixteen loads)
#pragma unroll
        for (int g = 0; g < FRA; g += 4) {
            int4 d[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) d[u] = __ldg(t + (lb | dep4(g + u, lm)));
#pragma unroll
            for (int u = 0; u < 4; ++u) x[g + u] = qcmul(d[u], x[g + u]);
            asm volatile("" ::: "memory");
        }
        // per-tile factors: each multiplies every amplitude in turn
        for (int f = nsel; f < o.nt; ++f) {
            if (!((gb >> ntq[o.aux2 + f]) & 1ull)) continue;
            const int4 c = qcoef(cf, f - nsel);
#pragma unroll
            for (int j = 0; j < FRA; ++j) x[j] = qcmul(c, x[j]);
        }
    } else if constexpr (std::is_same<V, double2>::value) {
        // complex128 in the float engine: Q62 tables and factors, integer
        // multiplies (no FP64 instruction)
        const I2* t = reinterpret_cast<const I2*>(tab) + o.aux + ((size_t)sel << K);
        const I2* cq = reinterpret_cast<const I2*>(cf);
        bool have_c = false;
        I2 c = cq[0];
        for (int f = nsel; f < o.nt; ++f) {
            if ((gb >> ntq[o.aux2 + f]) & 1ull) {
                c = have_c ? cmul(c, cq[f - nsel]) : cq[f - nsel];
                have_c = true;
            }
        }
        if (have_c) {
#pragma unroll
            for (int j = 0; j < FRA; ++j) x[j] = icmul(cmul(c, tab_ld(t + (lb | dep4(j, lm)))), x[j]);
        } else {
#pragma unroll
            for (int j = 0; j < FRA; ++j) x[j] = icmul(tab_ld(t + (lb | dep4(j, lm))), x[j]);
        }
    } else {
        const V* t = tab + o.aux + ((size_t)sel << K);
        bool have_c = false;
        V c = cf[0];
        for (int f = nsel; f < o.nt; ++f) {
            if ((gb >> ntq[o.aux2 + f]) & 1ull) {
                c = have_c ? cmul(c, cf[f - nsel]) : cf[f - nsel];
                have_c = true;
            }
        }
#pragma unroll
        for (int j = 0; j < FRA; ++j) {
            V d = tab_ld(t + (lb | dep4(j, lm)));
            if (have_c) d = cmul(c, d);
            x[j] = cmul(d, x[j]);
        }
    }
}

template <typename V, typename SV, int ENG, int FEAT>
__device__ __forceinline__ void apply_tile_op(V (&x)[FRA], const TileOp& o, const PassArgs<SV>& a, const V* cf,
                                              uint64_t gb, const uint64_t* gm, uint32_t lb, const int* lm) {
    switch (o.type) {
    case TOP_G1:
        if constexpr ((FEAT & FEAT_DENSE1) != 0) switch (o.a) {
        case 0: op_g1<V, 0, ENG>(x, o, cf, gb, gm); break;
        case 1: op_g1<V, 1, ENG>(x, o, cf, gb, gm); break;
        case 2: op_g1<V, 2, ENG>(x, o, cf, gb, gm); break;
        default: op_g1<V, 3, ENG>(x, o, cf, gb, gm); break;
        }
        break;
    case TOP_G1MONO:
        if constexpr ((FEAT & FEAT_GATES) != 0) switch (o.a) {
        case 0: op_g1mono<V, 0>(x, o, cf, gb, gm); break;
        case 1: op_g1mono<V, 1>(x, o, cf, gb, gm); break;
        case 2: op_g1mono<V, 2>(x, o, cf, gb, gm); break;
        default: op_g1mono<V, 3>(x, o, cf, gb, gm); break;
        }
        break;
    case TOP_G1SWAP:
        if constexpr ((FEAT & FEAT_GATES) != 0) switch (o.a) {
        case 0: op_g1swap<V, 0>(x, o, gb, gm); break;
        case 1: op_g1swap<V, 1>(x, o, gb, gm); break;
        case 2: op_g1swap<V, 2>(x, o, gb, gm); break;
        default: op_g1swap<V, 3>(x, o, gb, gm); break;
        }
        break;
    case TOP_H:
        if constexpr ((FEAT & FEAT_GATES) != 0) switch (o.a) {
        case 0: op_h<V, 0>(x); break;
        case 1: op_h<V, 1>(x); break;
        case 2: op_h<V, 2>(x); break;
        default: op_h<V, 3>(x); break;
        }
        break;
    case TOP_G2:
    case TOP_G2MONO: {
        const bool mono = o.type == TOP_G2MONO;
        if constexpr ((FEAT & FEAT_G2) != 0) switch (o.a * 4 + o.b) {
        case 1 * 4 + 0: op_g2<V, 1, 0, ENG>(x, o, cf, gb, gm, mono); break;
        case 2 * 4 + 0: op_g2<V, 2, 0, ENG>(x, o, cf, gb, gm, mono); break;
        case 2 * 4 + 1: op_g2<V, 2, 1, ENG>(x, o, cf, gb, gm, mono); break;
        case 3 * 4 + 0: op_g2<V, 3, 0, ENG>(x, o, cf, gb, gm, mono); break;
        case 3 * 4 + 1: op_g2<V, 3, 1, ENG>(x, o, cf, gb, gm, mono); break;
        default: op_g2<V, 3, 2, ENG>(x, o, cf, gb, gm, mono); break;
        }
        break;
    }
    case TOP_DIAG:
        if constexpr ((FEAT & FEAT_DIAG) != 0) op_diag<V, ENG>(x, o, cf, gb, gm);
        break;
    case TOP_Z4: op_z4<V>(x, o, a.z4, gb, gm); break;
    default:
        if constexpr ((FEAT & FEAT_DIAG) != 0)
            op_dsep<V, ENG>(x, o, cf, reinterpret_cast<const V*>(a.tab), a.ntq, lb, lm, gb, a.K);
        break;
    }
}

// ---------------------------------------------------------------- kernel --
// Raw bits of a stored value, held in the int64 engine's registers until the
// tile exponent is known.
template <typename SV, typename V>
__device__ __forceinline__ V raw_load(const SV v) {
    if constexpr (IsFP<V>::value) {
        return v;
    } else {
        V r;
        r.x = __double_as_longlong(v.x);
        r.y = __double_as_longlong(v.y);
        return r;
    }
}

// SV: storage type (double2 / float2); ENG selects the arithmetic, FEAT the
// op kinds compiled in.
// complex128: two CTAs per SM for the lightest variant, one (with up to 255
// registers, no spills) when multiplying op bodies are compiled in.
// QIN (ENG_Q only): 1 = this pass converts its input from doubles (the
// first pass of a fixed-point run); a separate instantiation keeps the
// conversion's registers out of the other passes.
template <typename SV, int ENG, int FEAT, int QIN = 0>
__global__ void __launch_bounds__(sizeof(SV) == 16 ? 256 : 512,
                                  (sizeof(SV) == 16 && (FEAT == FEAT_GATES || FEAT == FEAT_DIAG ||
                                                        (ENG != ENG_I64 && FEAT == (FEAT_GATES | FEAT_DIAG)))) ? 2 : 1)
    k_tile(const __grid_constant__ PassArgs<SV> a) {
    using V = typename std::conditional<ENG == ENG_FP, SV, I2>::type;
    extern __shared__ __align__(16) unsigned char smraw[];
    SV* sms = reinterpret_cast<SV*>(smraw);     // staging of stored values
    V* sm = reinterpret_cast<V*>(smraw);        // exchange between phases
    __shared__ int s_emax[16];
    const int K = a.K;
    const uint32_t T = 1u << (K - FR);
    const uint32_t tid = threadIdx.x;
    const uint64_t tile = blockIdx.x;
    const uint64_t tb = insert_zeros(tile, a.tpos, K);    // global index of local 0
    SV* const psi = a.psi + (a.slots ? (unsigned long long)a.slots[blockIdx.y] : (unsigned long long)blockIdx.y) * a.bstride;
    SV* const pso = a.psi_out ? a.psi_out : psi;   // (out of place only for single-state launches)
    const V* const bcf = reinterpret_cast<const V*>(a.bcoef) + (size_t)blockIdx.y * a.bcstride;
    V x[FRA];
    int S = 0;   // ENG_I64 / ENG_Q: fixed-point exponent
    if constexpr (ENG == ENG_Q) S = *a.qS - a.qgi;

    if (a.load_smem) {
        // coalesced copy: element tid + i*T, its top FR local bits come from i
        const uint64_t gt = tb | spread_bits(tid, a.tpos, K - FR);
        uint64_t gtop[FR];
#pragma unroll
        for (int r = 0; r < FR; ++r) gtop[r] = 1ull << a.tpos[K - FR + r];
        int st[FR];
#pragma unroll
        for (int r = 0; r < FR; ++r) st[r] = a.ld.rc[r];
        const int s0 = xbase(a.ld, tid);
#pragma unroll
        for (int i = 0; i < FRA; ++i) sms[s0 ^ dep4x(i, st)] = __ldcs(psi + (gt | dep4(i, gtop)));
        __syncthreads();
    }

    for (int p = 0; p < a.nph; ++p) {
        const TilePhase& ph = a.ph[p];
        const uint32_t lb = insert_reg_zeros(tid, ph.rb);
        const uint64_t gb = tb | spread_bits(lb, a.tpos, K);
        uint64_t gm[FR];
        int lm[FR], sr[FR];
#pragma unroll
        for (int r = 0; r < FR; ++r) {
            gm[r] = 1ull << a.tpos[ph.rb[r]];
            lm[r] = 1 << ph.rb[r];
            sr[r] = ph.in.rc[r];
        }
        const bool read_sm = p > 0 || a.load_smem;
        const int sb = read_sm ? xbase(ph.in, tid) : 0;   // slot maps are XOR-linear: slot = sb ^ xor of sr
        if (p == 0) {
            if (ENG == ENG_Q && a.gather) {
                const uint64_t g0 = gbase(a.gin, tid, tb);
                uint64_t rc[FR];
#pragma unroll
                for (int r = 0; r < FR; ++r) rc[r] = a.gin.rc[r];
#pragma unroll
                for (int j = 0; j < FRA; ++j) x[j] = raw_load<SV, V>(__ldcs(psi + (g0 ^ dep4xl(j, rc))));
            } else if (!a.load_smem) {
#pragma unroll
                for (int j = 0; j < FRA; ++j) x[j] = raw_load<SV, V>(__ldcs(psi + (gb | dep4(j, gm))));
            } else {
#pragma unroll
                for (int j = 0; j < FRA; ++j) x[j] = raw_load<SV, V>(sms[sb ^ dep4x(j, sr)]);
            }
            if constexpr (ENG == ENG_Q && QIN == 1) {
#pragma unroll
                for (int j = 0; j < FRA; ++j) {
                    x[j].x = d2fix(__longlong_as_double(x[j].x), S);
                    x[j].y = d2fix(__longlong_as_double(x[j].y), S);
                }
            }
            if constexpr (ENG == ENG_I64) {
                // tile exponent: max over the tile of both components
                int e = 0;
#pragma unroll
                for (int j = 0; j < FRA; ++j)
                    e = max(e, max((int)((x[j].x >> 52) & 0x7FF), (int)((x[j].y >> 52) & 0x7FF)));
                const unsigned amask = T >= 32 ? 0xffffffffu : ((1u << T) - 1u);
                e = (int)__reduce_max_sync(amask, (unsigned)e);
                if ((tid & 31) == 0) s_emax[tid >> 5] = e;
                __syncthreads();
                int emax = 0;
                for (int w = 0; w < (int)((blockDim.x + 31) >> 5); ++w) emax = max(emax, s_emax[w]);
                // |v| < 2^(emax-1022); the pass grows it by at most 2^(guard-1)
                S = emax == 0 ? 0 : 62 - a.guard - (emax - 1022);
#pragma unroll
                for (int j = 0; j < FRA; ++j) {
                    x[j].x = d2fix(__longlong_as_double(x[j].x), S);
                    x[j].y = d2fix(__longlong_as_double(x[j].y), S);
                }
            }
        } else {
#pragma unroll
            for (int j = 0; j < FRA; ++j) x[j] = sm[sb ^ dep4x(j, sr)];
        }
        for (int o = ph.op_begin; o < ph.op_end; ++o) {
            const TileOp& op = a.ops[o];
            if constexpr (ENG == ENG_Q) {
            if (op.type == TOP_Z4 && op.c == 2) {
                // sign terms after the closing permutation: on the store index
                const uint64_t g0 = gbase(a.gout, tid, tb);
                int e[FRA];
#pragma unroll
                for (int j = 0; j < FRA; ++j) e[j] = 0;
                for (int t = 0; t < op.aux2; ++t) {
                    const Z4Term z = a.z4[op.aux + t];
#pragma unroll
                    for (int j = 0; j < FRA; ++j)
                        if (((g0 ^ dep4xl(j, a.gout.rc)) & z.mask) == z.vals) e[j] += z.e;
                }
#pragma unroll
                for (int j = 0; j < FRA; ++j) x[j] = mul_ik(x[j], e[j] & 3);
                continue;
            }
            }
            const V* cf = (op.c == 1 ? bcf : reinterpret_cast<const V*>(a.coef)) + op.coef;
            apply_tile_op<V, SV, ENG, FEAT>(x, op, a, cf, gb, gm, lb, lm);
        }
        // exit slots: the same as the entry slots unless the exchange
        // permutes the tile index, in which case every read of this phase
        // must finish before any write
        int ob = sb, orr[FR];
        if (ph.permuted) {
            if (read_sm) __syncthreads();
            ob = xbase_out(ph.out, tid, gb);
#pragma unroll
            for (int r = 0; r < FR; ++r) orr[r] = ph.out.s.rc[r];
        } else {
#pragma unroll
            for (int r = 0; r < FR; ++r) orr[r] = sr[r];
        }
        if (p != a.nph - 1) {
            if constexpr (ENG == ENG_Q) {
                if (ph.qsh > 0) {
                    const int k = ph.qsh;
                    const long long half = 1ll << (k - 1);
#pragma unroll
                    for (int j = 0; j < FRA; ++j) {
                        x[j].x = (x[j].x + half) >> k;
                        x[j].y = (x[j].y + half) >> k;
                    }
                }
            }
#pragma unroll
            for (int j = 0; j < FRA; ++j) sm[ob ^ dep4x(j, orr)] = x[j];
            __syncthreads();
            continue;
        }
        // last phase: back to the storage type, then out
        SV* out = reinterpret_cast<SV*>(x);
        if constexpr (ENG == ENG_Q) {
            // the pass's 2^(-nh/2) and the change to the next pass's format
            // (S_out - S_in = qgi - qgo): one rounded shift, times 1/sqrt(2)
            // for odd nh; then doubles unless the state stays fixed point
            const int k = (a.qend >> 1) + (a.q_out ? a.qgo - a.qgi : 0);
            const bool odd = a.qend & 1;
            const long long half = k > 0 ? (1ll << (k - 1)) : 0ll;
            const int r2h = 759250124, r2l = 2134625280;   // round(2^61 / sqrt(2)) = r2h * 2^31 + r2l
#pragma unroll
            for (int j = 0; j < FRA; ++j) {
                long long vx = x[j].x, vy = x[j].y;
                if (odd) {
                    vx = qmul_real(vx, r2h, r2l);
                    vy = qmul_real(vy, r2h, r2l);
                }
                if (k > 0) {
                    vx = (vx + half) >> k;
                    vy = (vy + half) >> k;
                } else if (k < 0) {
                    vx = (long long)((unsigned long long)vx << (-k));
                    vy = (long long)((unsigned long long)vy << (-k));
                }
                if (a.q_out) {
                    x[j].x = vx;
                    x[j].y = vy;
                } else {
                    x[j].x = __double_as_longlong(fix2d(vx, S));
                    x[j].y = __double_as_longlong(fix2d(vy, S));
                }
            }
        } else if constexpr (ENG == ENG_I64) {
            // undo the fixed-point scale and apply 2^(-qend/2) (the pass's
            // levels, with a level carried in from or left to another pass)
            const int So = S + (a.qend >> 1);
            const bool odd = a.qend & 1;
            const int r2h = 759250124, r2l = 2134625280;   // round(2^61 / sqrt(2)) = r2h * 2^31 + r2l
#pragma unroll
            for (int j = 0; j < FRA; ++j) {
                long long vx = x[j].x, vy = x[j].y;
                if (odd) {
                    vx = qmul_real(vx, r2h, r2l);
                    vy = qmul_real(vy, r2h, r2l);
                }
                x[j].x = __double_as_longlong(fix2d(vx, So));
                x[j].y = __double_as_longlong(fix2d(vy, So));
            }
        } else {
            if (a.scale != 1.0) {
#pragma unroll
                for (int j = 0; j < FRA; ++j) {
                    x[j].x = (decltype(x[j].x))(x[j].x * a.scale);
                    x[j].y = (decltype(x[j].y))(x[j].y * a.scale);
                }
            }
        }
        // a permuted load or store moves amplitudes between threads of the
        // tile in place: every load must precede every store
        if (ENG == ENG_Q && a.nph == 1 && (a.gather || a.scatter) && !a.psi_out) __syncthreads();
        if (ENG == ENG_Q && a.scatter) {
            const uint64_t g0 = gbase(a.gout, tid, tb);
            uint64_t rc[FR];
#pragma unroll
            for (int r = 0; r < FR; ++r) rc[r] = a.gout.rc[r];
#pragma unroll
            for (int j = 0; j < FRA; ++j) __stcs(pso + (g0 ^ dep4xl(j, rc)), out[j]);
        } else if (!a.store_smem) {
#pragma unroll
            for (int j = 0; j < FRA; ++j) __stcs(pso + (gb | dep4(j, gm)), out[j]);
        } else {
            // unpermuted: a thread rewrites only the slots it read itself
#pragma unroll
            for (int j = 0; j < FRA; ++j) sms[ob ^ dep4x(j, orr)] = out[j];
            __syncthreads();
            const uint64_t gt = tb | spread_bits(tid, a.tpos, K - FR);
            uint64_t gtop[FR];
#pragma unroll
            for (int r = 0; r < FR; ++r) gtop[r] = 1ull << a.tpos[K - FR + r];
            int st[FR];
#pragma unroll
            for (int r = 0; r < FR; ++r) st[r] = a.st.rc[r];
            const int s0 = xbase(a.st, tid);
#pragma unroll
            for (int i = 0; i < FRA; ++i) __stcs(pso + (gt | dep4(i, gtop)), sms[s0 ^ dep4x(i, st)]);
        }
    }
}

// --------------------------------------------------- Hadamard passes --
// Passes of butterflies and exact sign terms only (the Hadamard layers of
// Sec. III-B's RH path), int64 engines, one state.  Persistent: two CTAs
// per SM walk the tiles blockIdx.x, blockIdx.x + gridDim.x, ...; each
// reads its tiles through one shared-memory buffer, and as soon as the last
// phase of a tile has read the buffer the next tile's asynchronous copy
// (cp.async) starts into it, overlapping that phase's arithmetic and
// stores (the other CTA covers the rest).  Per-phase slot bases and
// offsets are computed once per CTA; the tile base advances by a masked
// add of the deposited grid stride ((tb | ~M) + dG) & M over the non-tile
// mask M.  Every pass reads through the load staging map (the planner
// stages the loads of these passes).
constexpr int HP_MAXPH = 8;
// Two shapes: 256 threads (tiles of up to 2^12 amplitudes, two CTAs per SM)
// and, for the per-tile engine, 512 threads (2^13-amplitude tiles, 128 KiB,
// one CTA per SM: one more butterfly level per pass).
// Tiled tensor copies of a tile (PassArgs::bulk): the state as a tensor
// of float64 words of at most 5 dimensions in ascending global bit order,
// each dimension a run of tile bits (the box spans it) or of non-tile bits
// (box 1, coordinate from the tile base); the first holds re/im and the
// tile's lowest bits.  The tile's top `tm` local bits may be taken as
// non-tile bits, one copy per value (2^tm copies of 2^(K-tm) amplitudes).
// Smem then holds the tile in natural local order.
constexpr int TMA_DIMS = 5;
struct HPassArgs {
    CUtensorMap tmap;              // encoded per launch on the host (input buffer of the pass)
    int* err;                      // set to 1 when a bounded wait for a tile copy ran out
    unsigned extra_tx;             // bytes expected per tile beyond the tile (0; a test makes waits run out)
    unsigned char tsh[TMA_DIMS];   // coordinate i = (copy base >> tsh[i]) & tmk[i]
    unsigned tmk[TMA_DIMS];
    int tm;                        // copies per tile: 2^tm
    unsigned long long tit[2];     // global bits of the copies' local bits K-tm, K-tm+1
    unsigned long long ntmask;     // non-tile global bits (below n)
    unsigned long long dstride;    // gridDim.x deposited into the non-tile bits
    unsigned ntiles;
    unsigned long long gm[HP_MAXPH][FR];   // per phase: global bit of each register bit
    // per op: a run of butterflies on distinct register bits starting here
    // (bits 0..3: the bits, bits 4..7: the run's length in ops), else 0
    unsigned char hrun[TILE_MAX_OPS];
    // sign terms on the scattered store index: bit j of P(q) is the parity
    // of the register bits of slot j that reach index bit q through the
    // scatter map; the first two pattern bits' P in the low / high halves
    unsigned pz[TILE_MAX_Z4];
};

__device__ __forceinline__ void cp_async16(void* sdst, const void* gsrc) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(__cvta_generic_to_global(gsrc))
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Tensor-memory-access copies, completed in bytes on an mbarrier.
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
__device__ __forceinline__ void tma_load5(void* sdst, const CUtensorMap* map, const int (&c)[5], unsigned long long* bar) {
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5, "
        "%6}], [%7];\n" ::"r"(smem_u32(sdst)),
        "l"(reinterpret_cast<unsigned long long>(map)), "r"(c[0]), "r"(c[1]), "r"(c[2]), "r"(c[3]), "r"(c[4]),
        "r"(smem_u32(bar))
        : "memory");
}
// Bounded wait for an mbarrier phase: false if it did not complete within
// about a second of SM clock.
constexpr long long MBAR_WAIT_CYCLES = 1ll << 31;
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > MBAR_WAIT_CYCLES) return false;
    return true;
}

// (hi:lo) >> k for 0 <= k < 32 (arithmetic): two funnel shifts
__device__ __forceinline__ long long shr_lt32(long long v, int k) {
    const unsigned lo = (unsigned)v, hi = (unsigned)(v >> 32);
    const unsigned nlo = __funnelshift_r(lo, hi, k);
    const int nhi = (int)hi >> k;
    return (long long)(((unsigned long long)(unsigned)nhi << 32) | nlo);
}
// (hi:lo) << k for 0 <= k < 32: a funnel shift and a shift
__device__ __forceinline__ long long shl_lt32(long long v, int k) {
    const unsigned lo = (unsigned)v, hi = (unsigned)(v >> 32);
    return (long long)(((unsigned long long)__funnelshift_l(lo, hi, k) << 32) | (lo << k));
}
// Per-amplitude exponent format of the int64 engine between Hadamard passes
// (EF).  A complex128 amplitude is two int64 words: bits 6..63 of the real
// word hold its signed real mantissa and bits 0..5 the amplitude's
// exponent code e (0..63); the imaginary word is the signed imaginary
// mantissa; value = mantissa * 2^-(e + B), B a bias fixed per circuit from
// the state's norm bound.  A stored amplitude has max(|re|, |im|) in
// [2^52, 2^53] (53 significant bits, as in a double) unless it is below
// the normal range, where e = 63 keeps it unnormalised (zero included).
// The mantissa sits where a pass with 9 headroom bits wants the tile's
// largest amplitude, so most amplitudes load with a shift by a few bits to
// the left (exact) and only those below the tile's largest exponent round.
constexpr int EF_LZ = 11;         // leading zeros of a normalised mantissa (top bit at 52)
constexpr int EF_TOP = 53;        // |mantissa| <= 2^EF_TOP

// round(v / 2^s), s >= 1 (0 for s >= 63)
__device__ __forceinline__ long long ef_rshift(long long v, int s) {
    if (s >= 63) return 0;
    return (v + (1ll << (s - 1))) >> s;
}
// v * 2^-s rounded to nearest (ties up) for -32 < s < 32
__device__ __forceinline__ long long shift_round_lt32(long long v, int s) {
    if (s <= 0) return shl_lt32(v, -s);
    return shr_lt32(v + (long long)(1u << (s - 1)), s);
}
// amplitude (vx, vy) = value * 2^T into the two EF words
__device__ __forceinline__ double2 ef_store(long long vx, long long vy, int T, int B) {
    if ((vx | vy) == 0) return make_double2(__longlong_as_double(63ll), 0.0);
    // ones' complement magnitudes: |v| - 1 for v < 0, which moves the top
    // bit only for powers of two, whose shifted mantissa is then 2^53
    const unsigned long long a = (unsigned long long)((vx ^ (vx >> 63)) | (vy ^ (vy >> 63)));
    int sl = __clzll((long long)a) - EF_LZ;     // shift that puts the top bit at 52 (a = 0: v in {0, -1})
    int e = T + sl - B;
    if (e > 63) {                               // below the normal range
        sl -= e - 63;
        e = 63;
    }
    long long mx, my;
    if (sl > -32 && sl < 32) {
        mx = shift_round_lt32(vx, -sl);
        my = shift_round_lt32(vy, -sl);
    } else {
        mx = sl >= 0 ? (long long)((unsigned long long)vx << sl) : ef_rshift(vx, -sl);
        my = sl >= 0 ? (long long)((unsigned long long)vy << sl) : ef_rshift(vy, -sl);
    }
    return make_double2(__longlong_as_double((long long)(((unsigned long long)mx << 6) | (unsigned)e)),
                        __longlong_as_double(my));
}

// Integer butterflies on register bit B that also add h to every result
// (the rounding term of a shift that follows): a + b + h, a - b + h.
template <int B>
__device__ __forceinline__ void op_h_add(I2 (&x)[FRA], long long h) {
#pragma unroll
    for (int j = 0; j < FRA; ++j) {
        if (j & (1 << B)) continue;
        const int j1 = j | (1 << B);
        x[j].x += x[j1].x + h;
        x[j].y += x[j1].y + h;
        x[j1].x = x[j].x - x[j1].x - x[j1].x;
        x[j1].y = x[j].y - x[j1].y - x[j1].y;
    }
}
// Integer butterflies on register bits B0 and B0 + 1 at once (two levels):
// for a, b, c, d on slots j, j|1<<B0, j|2<<B0, j|3<<B0 the results
// a+b+c+d, a-b+c-d, a+b-c-d, a-b-c+d from S = c + d and D = c - d in six
// three-operand sums instead of eight two-operand ones.
template <int B0>
__device__ __forceinline__ void op_h4(I2 (&x)[FRA]) {
#pragma unroll
    for (int j = 0; j < FRA; ++j) {
        if (j & (3 << B0)) continue;
        const int j1 = j | (1 << B0), j2 = j | (2 << B0), j3 = j | (3 << B0);
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            long long& a = c ? x[j].y : x[j].x;
            long long& b = c ? x[j1].y : x[j1].x;
            long long& cc = c ? x[j2].y : x[j2].x;
            long long& d = c ? x[j3].y : x[j3].x;
            const long long S = cc + d, D = S - d - d;
            const long long y0 = a + b + S, y1 = a - b + D;
            a = y0;
            b = y1;
            cc = y0 - S - S;
            d = y1 - D - D;
        }
    }
}
// Butterflies on the register bits set in m: a full phase (all four bits)
// as one straight block, otherwise bit by bit.  Integer engines: pairs of
// levels as radix-4 blocks; h != 0 adds h to every result of the last
// level (the rounding term of the phase's exit shift).
template <typename V>
__device__ __forceinline__ void op_hmask(V (&x)[FRA], int m, long long h = 0) {
    if constexpr (IsFP<V>::value) {
        if (m == 15) {
            op_h<V, 0>(x);
            op_h<V, 1>(x);
            op_h<V, 2>(x);
            op_h<V, 3>(x);
            return;
        }
        if (m & 1) op_h<V, 0>(x);
        if (m & 2) op_h<V, 1>(x);
        if (m & 4) op_h<V, 2>(x);
        if (m & 8) op_h<V, 3>(x);
    } else {
        if (m == 15) {
            op_h4<0>(x);
            if (h != 0) {
                op_h<V, 2>(x);
                op_h_add<3>(x, h);
            } else {
                op_h4<2>(x);
            }
            return;
        }
        const int top = 31 - __clz(m | 1);   // the last level applied
        if (m & 1) {
            if (h != 0 && top == 0) op_h_add<0>(x, h);
            else op_h<V, 0>(x);
        }
        if (m & 2) {
            if (h != 0 && top == 1) op_h_add<1>(x, h);
            else op_h<V, 1>(x);
        }
        if (m & 4) {
            if (h != 0 && top == 2) op_h_add<2>(x, h);
            else op_h<V, 2>(x);
        }
        if (m & 8) {
            if (h != 0 && top == 3) op_h_add<3>(x, h);
            else op_h<V, 3>(x);
        }
    }
}

// QIN: 1 = the pass converts its input from doubles, 0 = it reads the
// engine's format (ENG_Q: global fixed point; ENG_I64: EF); QOUT: 1 = the
// pass writes that format, 0 = doubles (the last pass of a run); ODD: 0 =
// the pass's level count to scale away is even (no 1/sqrt(2) product).  Separate instantiations keep
// code a pass never runs out of its instruction stream.
template <int ENG, int QIN, int QOUT, int ODD, int NT = 256>
__global__ void __launch_bounds__(NT, NT == 256 ? 2 : 1)
    k_hpass(const __grid_constant__ PassArgs<double2> a, const __grid_constant__ HPassArgs h) {
    static_assert(ENG == ENG_I64 || ENG == ENG_Q, "int64 engines only");
    using V = I2;
    extern __shared__ __align__(128) unsigned char smraw_h[];   // a tensor copy's destination: 128-byte aligned
    unsigned char* const smraw = smraw_h;
    __shared__ int s_emax[NT / 32];
    __shared__ unsigned long long s_gloc[HP_MAXPH][NT];
    __shared__ short s_sb[HP_MAXPH][NT], s_ob[HP_MAXPH][NT];
    const int K = a.K;
    const uint32_t T = 1u << (K - FR);
    const uint32_t tid = threadIdx.x;
    double2* const psi = a.psi;
    double2* const pso = a.psi_out ? a.psi_out : a.psi;   // tiles are disjoint: out of place is free
    int Sq = 0, B = 0;
    if constexpr (ENG == ENG_Q) Sq = *a.qS - a.qgi;
    // EF bias: amplitudes are below 2^(60 - *qS); code 0 holds up to 16x that
    if constexpr (ENG == ENG_I64 && (QIN == 0 || QOUT == 1)) B = *a.qS - 11;
    // per phase and thread (tile-independent): global offset of register
    // slot 0, and the entry / exit slot bases in shared memory
    for (int p = 0; p < a.nph; ++p) {
        s_gloc[p][tid] = spread_bits(insert_reg_zeros(tid, a.ph[p].rb), a.tpos, K);
        const int sb = xbase(a.ph[p].in, tid);
        s_sb[p][tid] = (short)sb;
        s_ob[p][tid] = (short)(a.ph[p].permuted ? (xbase(a.ph[p].out.s, tid) ^ (int)a.ph[p].out.off0) : sb);
    }
    // staged copy: element tid + i*T of the tile, its top FR local bits from i
    const uint64_t gt = spread_bits(tid, a.tpos, K - FR);
    uint64_t gtop[FR];
    int lst[FR];
#pragma unroll
    for (int r = 0; r < FR; ++r) {
        gtop[r] = 1ull << a.tpos[K - FR + r];
        lst[r] = a.ld.rc[r];
    }
    const int ls0 = xbase(a.ld, tid);
    // scattered store (a closing permutation run): the thread's part of
    // the map; the tile's part is added per tile
    uint64_t gsc = 0;
    if constexpr (ENG == ENG_Q) {
        gsc = a.gout.c;
#pragma unroll
        for (int t = 0; t < 12; ++t) gsc ^= (0ull - (uint64_t)((tid >> t) & 1u)) & a.gout.tc[t];
    }
    auto scatter_base = [&](uint64_t tb) {
        uint64_t v = tb ^ gsc;
        for (int i = 0; i < a.gout.nq; ++i)
            if ((tb >> a.gout.q[i]) & 1ull) v ^= a.gout.w[i];
        return v;
    };
    const unsigned G = gridDim.x;
    auto madd = [&](uint64_t tb) { return ((tb | ~h.ntmask) + h.dstride) & h.ntmask; };
    double2* const sms = reinterpret_cast<double2*>(smraw);
    V* const sm = reinterpret_cast<V*>(smraw);
    // Bulk staging (a.bulk: the load staging is the natural local order):
    // one tiled tensor copy per tile, issued by thread 0 and counted in
    // bytes on an mbarrier whose phase flips per tile.  Otherwise 16-byte
    // asynchronous copies per element into the swizzled staging layout.
    __shared__ unsigned long long s_bar;
    const bool bulk = a.bulk != 0;
    if (bulk) {
        if (tid == 0) {
            mbar_init(&s_bar, 1);
            mbar_fence_init();
        }
    }
    unsigned bpar = 0;
    auto prefetch = [&](uint64_t t, uint64_t tb) {
        if (bulk) {
            if (t < h.ntiles && tid == 0) {
                fence_proxy_async_smem();   // the buffer's earlier reads (ordered by the barrier) come first
                mbar_expect_tx(&s_bar, (T << 8) + h.extra_tx);
                for (int j = 0; j < (1 << h.tm); ++j) {
                    const uint64_t cb = tb | ((j & 1) ? h.tit[0] : 0ull) | ((j & 2) ? h.tit[1] : 0ull);
                    int c[TMA_DIMS];
#pragma unroll
                    for (int i = 0; i < TMA_DIMS; ++i) c[i] = (int)((unsigned)(cb >> h.tsh[i]) & h.tmk[i]);
                    tma_load5(sms + ((size_t)j << (K - h.tm)), &h.tmap, c, &s_bar);
                }
            }
            return;
        }
        if (t < h.ntiles) {
            const uint64_t g0 = tb | gt;
#pragma unroll
            for (int i = 0; i < FRA; ++i) cp_async16(sms + (ls0 ^ dep4x(i, lst)), psi + (g0 | dep4(i, gtop)));
        }
        cp_async_commit();
    };
    uint64_t tb = insert_zeros(blockIdx.x, a.tpos, K);   // base of the tile being worked on
    __syncthreads();
    prefetch(blockIdx.x, tb);
    for (uint64_t tile = blockIdx.x; tile < h.ntiles; tile += G) {
        if (bulk) {
            // every thread waits for the tile's bytes (bounded); a wait that
            // runs out anywhere makes the whole CTA report it and return
            const bool ok = mbar_wait(&s_bar, bpar);
            bpar ^= 1u;
            if (__syncthreads_or(ok ? 0 : 1)) {
                if (tid == 0) atomicExch(h.err, 1);
                mbar_wait(&s_bar, bpar ^ 1u);   // give copies still in flight a bounded time to land
                return;
            }
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();   // this tile is in the buffer
        const uint64_t tbn = madd(tb);
        V x[FRA];
        int S = Sq;
        for (int p = 0; p < a.nph; ++p) {
            const TilePhase& ph = a.ph[p];
            const uint64_t gb = tb | s_gloc[p][tid];
            uint64_t gm[FR];
            int sr[FR];
#pragma unroll
            for (int r = 0; r < FR; ++r) {
                gm[r] = h.gm[p][r];
                sr[r] = ph.in.rc[r];
            }
            const int sb = s_sb[p][tid];
            if (p == 0) {
#pragma unroll
                for (int j = 0; j < FRA; ++j) x[j] = raw_load<double2, V>(sms[sb ^ dep4x(j, sr)]);
                if constexpr (ENG == ENG_Q && QIN == 1) {
#pragma unroll
                    for (int j = 0; j < FRA; ++j) {
                        x[j].x = d2fix(__longlong_as_double(x[j].x), S);
                        x[j].y = d2fix(__longlong_as_double(x[j].y), S);
                    }
                }
                if constexpr (ENG == ENG_I64 && QIN == 1) {
                    int e = 0;
#pragma unroll
                    for (int j = 0; j < FRA; ++j)
                        e = max(e, max((int)((x[j].x >> 52) & 0x7FF), (int)((x[j].y >> 52) & 0x7FF)));
                    const unsigned amask = T >= 32 ? 0xffffffffu : ((1u << T) - 1u);
                    e = (int)__reduce_max_sync(amask, (unsigned)e);
                    if ((tid & 31) == 0) s_emax[tid >> 5] = e;
                    __syncthreads();
                    int emax = 0;
                    for (int w = 0; w < (int)((T + 31) >> 5); ++w) emax = max(emax, s_emax[w]);
                    S = emax == 0 ? 0 : 62 - a.guard - (emax - 1022);
#pragma unroll
                    for (int j = 0; j < FRA; ++j) {
                        x[j].x = d2fix(__longlong_as_double(x[j].x), S);
                        x[j].y = d2fix(__longlong_as_double(x[j].y), S);
                    }
                } else if constexpr (ENG == ENG_I64) {
                    // EF input: the tile takes the scale of its largest
                    // amplitude (smallest code, zeros hold 63) with the
                    // pass's headroom; each mantissa is aligned to it by a
                    // rounded shift
                    int e = 63;
#pragma unroll
                    for (int j = 0; j < FRA; ++j) e = min(e, (int)(x[j].x & 63));
                    const unsigned amask = T >= 32 ? 0xffffffffu : ((1u << T) - 1u);
                    e = (int)__reduce_min_sync(amask, (unsigned)e);
                    if ((tid & 31) == 0) s_emax[tid >> 5] = e;
                    __syncthreads();
                    int emin = 63;
                    for (int w = 0; w < (int)((T + 31) >> 5); ++w) emin = min(emin, s_emax[w]);
                    // |mantissa| <= 2^EF_TOP at code emin becomes <= 2^(62 - guard)
                    const int sh0 = a.guard - (62 - EF_TOP) - emin;
                    S = emin + B + (62 - EF_TOP) - a.guard;
#pragma unroll
                    for (int j = 0; j < FRA; ++j) {
                        const int sh = (int)(x[j].x & 63) + sh0;
                        const long long mx = x[j].x >> 6, my = x[j].y;
                        if (sh < 32) {   // sh > -32: codes are >= emin, guard >= 0
                            x[j].x = shift_round_lt32(mx, sh);
                            x[j].y = shift_round_lt32(my, sh);
                        } else {
                            x[j].x = ef_rshift(mx, sh);
                            x[j].y = ef_rshift(my, sh);
                        }
                    }
                }
            } else {
#pragma unroll
                for (int j = 0; j < FRA; ++j) x[j] = sm[sb ^ dep4x(j, sr)];
            }
            if (p == a.nph - 1 && !a.store_smem) {
                // the buffer is read: the next tile streams in under this phase
                __syncthreads();
                prefetch(tile + G, tbn);
            }
            bool rounded = false;   // the exit's rounding term was added by the last butterflies
            for (int o = ph.op_begin; o < ph.op_end;) {
                const TileOp& op = a.ops[o];
                if (op.type == TOP_H) {
                    const int r = h.hrun[o];
                    o += max(r >> 4, 1);   // (a run covers at least this op)
                    // a run that ends a phase with a rounded exit shift adds
                    // the rounding term in its last level
                    const bool fuse = o >= ph.op_end && p != a.nph - 1 && ph.qsh > 0;
                    op_hmask<V>(x, r & 15, fuse ? (1ll << (ph.qsh - 1)) : 0ll);
                    rounded = rounded || fuse;
                    continue;
                }
                ++o;
                if (ENG == ENG_Q && op.c == 2) {
                    // sign terms after the closing permutation, on the store
                    // index: bit q of slot j's index is bit q of the thread's
                    // base XOR the parity P(q) of j, so the slots a term
                    // selects form one 16-bit mask per thread
                    const uint64_t g0 = scatter_base(tb);
                    uint32_t p0 = 0, p1 = 0;
                    for (int t = 0; t < op.aux2; ++t) {
                        const Z4Term z = a.z4[op.aux + t];
                        const uint32_t pm = h.pz[op.aux + t];
                        const uint64_t tv = z.vals ^ g0;
                        uint64_t m = z.mask;
                        uint32_t act = 0xFFFFu;
                        for (int k = 0; m; ++k) {
                            const int q = __ffsll((long long)m) - 1;
                            m &= m - 1;
                            uint32_t pq = 0;
                            if (k < 2) {
                                pq = (pm >> (16 * k)) & 0xFFFFu;
                            } else {
                                const uint32_t b1[4] = {0xAAAAu, 0xCCCCu, 0xF0F0u, 0xFF00u};
#pragma unroll
                                for (int r = 0; r < FR; ++r)
                                    if ((a.gout.rc[r] >> q) & 1ull) pq ^= b1[r];
                            }
                            act &= ((tv >> q) & 1ull) ? pq : (~pq & 0xFFFFu);
                        }
                        if (z.e & 1) {
                            const uint32_t c = p0 & act;
                            p0 ^= act;
                            p1 ^= c;
                        }
                        if (z.e & 2) p1 ^= act;
                    }
                    if ((p0 | p1) != 0) {
#pragma unroll
                        for (int j = 0; j < FRA; ++j)
                            x[j] = mul_ik(x[j], (int)(((p0 >> j) & 1u) | (((p1 >> j) & 1u) << 1)));
                    }
                } else {
                    op_z4<V>(x, op, a.z4, gb, gm);
                }
            }
            int orr[FR];
#pragma unroll
            for (int r = 0; r < FR; ++r) orr[r] = ph.permuted ? ph.out.s.rc[r] : sr[r];
            if (ph.permuted) __syncthreads();
            int ob = s_ob[p][tid];
            for (int i = 0; i < ph.out.noff; ++i)
                if ((gb >> ph.out.offq[i]) & 1ull) ob ^= (int)ph.out.offv[i];
            if (p != a.nph - 1) {
                // part of the 2^(-nh/2) scale at the phase exit: a right
                // shift rounded to nearest (ties up), both engines
                if (ph.qsh > 0) {
                    const int k = ph.qsh;
                    const long long half = rounded ? 0ll : (1ll << (k - 1));
#pragma unroll
                    for (int j = 0; j < FRA; ++j) {
                        x[j].x = shr_lt32(x[j].x + half, k);
                        x[j].y = shr_lt32(x[j].y + half, k);
                    }
                }
#pragma unroll
                for (int j = 0; j < FRA; ++j) sm[ob ^ dep4x(j, orr)] = x[j];
                __syncthreads();
                continue;
            }
            double2* out = reinterpret_cast<double2*>(x);
            if constexpr (ENG == ENG_Q) {
                // the pass's 2^(-qend/2) and the change to the next pass's
                // format: one shift rounded to nearest, times 1/sqrt(2)
                // for odd qend; then doubles unless the state stays fixed point
                const int k = (a.qend >> 1) + (a.q_out ? a.qgo - a.qgi : 0);
                const bool odd = ODD && (a.qend & 1);
                const int r2h = 759250124, r2l = 2134625280;   // round(2^61 / sqrt(2)) = r2h * 2^31 + r2l
                const long long half = k > 0 ? (1ll << (k - 1)) : 0ll;
#pragma unroll
                for (int j = 0; j < FRA; ++j) {
                    long long vx = x[j].x, vy = x[j].y;
                    if constexpr (ODD == 1) {
                        if (odd) {
                            vx = qmul_real(vx, r2h, r2l);
                            vy = qmul_real(vy, r2h, r2l);
                        }
                    }
                    if (k > 0) {
                        vx = shr_lt32(vx + half, k);
                        vy = shr_lt32(vy + half, k);
                    } else if (k < 0) {
                        vx = (long long)((unsigned long long)vx << (-k));
                        vy = (long long)((unsigned long long)vy << (-k));
                    }
                    if constexpr (QOUT == 1) {
                        x[j].x = vx;
                        x[j].y = vy;
                    } else {
                        x[j].x = __double_as_longlong(fix2d(vx, S));
                        x[j].y = __double_as_longlong(fix2d(vy, S));
                    }
                }
            } else {
                // levels left unscaled by the phase exits: 2^(-qend/2), a
                // change of scale (doubles) or of exponent code (EF)
                const int So = S + (a.qend >> 1);
                const bool odd = ODD && (a.qend & 1);
                const int r2h = 759250124, r2l = 2134625280;   // round(2^61 / sqrt(2)) = r2h * 2^31 + r2l
#pragma unroll
                for (int j = 0; j < FRA; ++j) {
                    long long vx = x[j].x, vy = x[j].y;
                    if (odd) {
                        vx = qmul_real(vx, r2h, r2l);
                        vy = qmul_real(vy, r2h, r2l);
                    }
                    if constexpr (QOUT == 1) {
                        const double2 w = ef_store(vx, vy, So, B);
                        x[j].x = __double_as_longlong(w.x);
                        x[j].y = __double_as_longlong(w.y);
                    } else {
                        x[j].x = __double_as_longlong(fix2d(vx, So));
                        x[j].y = __double_as_longlong(fix2d(vy, So));
                    }
                }
            }
            if (ENG == ENG_Q && a.scatter) {
                const uint64_t g0 = scatter_base(tb);
                uint64_t rc[FR];
#pragma unroll
                for (int r = 0; r < FR; ++r) rc[r] = a.gout.rc[r];
#pragma unroll
                for (int j = 0; j < FRA; ++j) __stcs(pso + (g0 ^ dep4xl(j, rc)), out[j]);
            } else if (!a.store_smem) {
#pragma unroll
                for (int j = 0; j < FRA; ++j) __stcs(pso + (gb | dep4(j, gm)), out[j]);
            } else {
#pragma unroll
                for (int j = 0; j < FRA; ++j) sms[ob ^ dep4x(j, orr)] = out[j];
                __syncthreads();
                int st[FR];
#pragma unroll
                for (int r = 0; r < FR; ++r) st[r] = a.st.rc[r];
                const int s0 = xbase(a.st, tid);
                const uint64_t g0 = tb | gt;
#pragma unroll
                for (int i = 0; i < FRA; ++i) __stcs(pso + (g0 | dep4(i, gtop)), sms[s0 ^ dep4x(i, st)]);
                __syncthreads();
                prefetch(tile + G, tbn);
            }
        }
        tb = tbn;
    }
    if (!bulk) cp_async_wait<0>();
}

// ------------------------------------------------ single-phase tables --
// A resident-engine pass whose only work is one phase of diagonal tables and
// sign terms (its permutations ride on the gathered loads and scattered
// stores).  512 threads per tile, eight amplitudes each; every address is an
// XOR of masks the host precomputes per thread-index bit and register bit,
// so a thread's setup is a few XORs and an access is one XOR and one address
// add.  IX is the index type: 32-bit arithmetic for states of at most 2^32
// amplitudes, 64-bit above.  No shared memory; with a permuted load or
// store every load precedes every store (block barrier), since amplitudes
// move between threads of the tile in place.
constexpr int DPASS_MAX_TABS = 2;
constexpr int DPASS_TBITS = 9;     // thread-index bits (512 threads)
constexpr int DPASS_RBITS = 3;     // register bits (8 amplitudes)
struct DMap {                      // global index = tile base ^ c ^ thread part ^ register part ^ tile terms
    unsigned long long t[DPASS_TBITS];
    unsigned long long r[DPASS_RBITS];
    unsigned long long c;
    unsigned long long w[TILE_MAX_XOFF];
    int8_t q[TILE_MAX_XOFF];
    int8_t nq;
};
struct DZ4 {
    unsigned long long mask, vals;
    int16_t e;
    int16_t post;                  // 1: matched on the stored (permuted) index
};
struct DPassArgs {
    double2* psi;
    double2* psi_out;              // the pass writes here (may equal psi)
    const int4* tab;
    int K;
    int nruns;                     // tile index -> tile base: runs of non-tile positions
    uint32_t run_src[32], run_w[32], run_dst[32];
    DMap in, out, nat;             // load map, store map, natural (unpermuted) positions
    uint32_t tloc[DPASS_TBITS], rloc[DPASS_RBITS];   // local index (table offset)
    int ntab;
    int tab_off[DPASS_MAX_TABS], tab_nt[DPASS_MAX_TABS];
    int8_t tab_q[DPASS_MAX_TABS][8];
    int shift;                     // right shift into the next pass's format (negative: left)
    int permuted;                  // 1: the load or the store map is a permutation
    uint32_t ntiles;               // tiles of the pass (the grid may be smaller)
    int nz;
    DZ4 z4[TILE_MAX_Z4];
};

template <typename IX>
__device__ __forceinline__ IX dbase(const DMap& m, uint32_t tid, IX tb) {
    IX v = tb ^ (IX)m.c;
#pragma unroll
    for (int t = 0; t < DPASS_TBITS; ++t) v ^= ((IX)0 - (IX)((tid >> t) & 1u)) & (IX)m.t[t];
    for (int i = 0; i < m.nq; ++i)
        if ((tb >> m.q[i]) & 1u) v ^= (IX)m.w[i];
    return v;
}
template <typename IX>
__device__ __forceinline__ IX dreg(int j, const IX* r) {
    IX v = 0;
    if (j & 1) v ^= r[0];
    if (j & 2) v ^= r[1];
    if (j & 4) v ^= r[2];
    return v;
}
__device__ __forceinline__ uint32_t dreg32(int j, const uint32_t* r) {
    uint32_t v = 0;
    if (j & 1) v ^= r[0];
    if (j & 2) v ^= r[1];
    if (j & 4) v ^= r[2];
    return v;
}

template <int GROUP, typename IX>
__global__ void __launch_bounds__(512, 2) k_dpass(const __grid_constant__ DPassArgs a) {
    constexpr int NA = 1 << DPASS_RBITS;
    const uint32_t tid = threadIdx.x;
    // the thread's parts of the maps are the same in every tile
    const IX ti = dbase<IX>(a.in, tid, 0), to = dbase<IX>(a.out, tid, 0), tn = dbase<IX>(a.nat, tid, 0);
    uint32_t lb = 0;
#pragma unroll
    for (int t = 0; t < DPASS_TBITS; ++t) lb ^= (0u - ((tid >> t) & 1u)) & a.tloc[t];
    IX rin[DPASS_RBITS], rout[DPASS_RBITS], rnat[DPASS_RBITS];
    uint32_t rloc[DPASS_RBITS];
#pragma unroll
    for (int r = 0; r < DPASS_RBITS; ++r) {
        rin[r] = (IX)a.in.r[r];
        rout[r] = (IX)a.out.r[r];
        rnat[r] = (IX)a.nat.r[r];
        rloc[r] = a.rloc[r];
    }
    // several tiles per CTA (grid-stride), each as in a one-tile launch
    for (uint32_t tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
    IX tb = 0;
    for (int i = 0; i < a.nruns; ++i) tb |= (IX)((tile >> a.run_src[i]) & ((1u << a.run_w[i]) - 1u)) << a.run_dst[i];
    IX gi0 = tb ^ ti, go0 = tb ^ to;
    const IX gn0 = tb ^ tn;
    for (int i = 0; i < a.in.nq; ++i)
        if ((tb >> a.in.q[i]) & 1u) gi0 ^= (IX)a.in.w[i];
    for (int i = 0; i < a.out.nq; ++i)
        if ((tb >> a.out.q[i]) & 1u) go0 ^= (IX)a.out.w[i];
    const int4* tabs[DPASS_MAX_TABS];
    for (int t = 0; t < a.ntab; ++t) {
        uint32_t sel = 0;
        for (int f = 0; f < a.tab_nt[t]; ++f) sel |= (uint32_t)((tb >> a.tab_q[t][f]) & 1u) << f;
        tabs[t] = a.tab + a.tab_off[t] + ((size_t)sel << a.K);
    }
    I2 x[NA];
#pragma unroll
    for (int j = 0; j < NA; ++j) {
        const longlong2 v = __ldcs(reinterpret_cast<const longlong2*>(a.psi + (gi0 ^ dreg<IX>(j, rin))));
        x[j].x = v.x;
        x[j].y = v.y;
    }
    if (a.permuted && a.psi_out == a.psi) __syncthreads();
    const int k = a.shift;
    const long long half = k > 0 ? (1ll << (k - 1)) : 0ll;
#pragma unroll
    for (int g = 0; g < NA; g += GROUP) {
        for (int t = 0; t < a.ntab; ++t) {
            int4 d[GROUP];
#pragma unroll
            for (int u = 0; u < GROUP; ++u) d[u] = __ldg(tabs[t] + (lb ^ dreg32(g + u, rloc)));
#pragma unroll
            for (int u = 0; u < GROUP; ++u) x[g + u] = qcmul(d[u], x[g + u]);
        }
        if (a.nz) {
            int e[GROUP];
#pragma unroll
            for (int u = 0; u < GROUP; ++u) e[u] = 0;
            for (int z = 0; z < a.nz; ++z) {
                const DZ4 tz = a.z4[z];
#pragma unroll
                for (int u = 0; u < GROUP; ++u) {
                    const IX gi = tz.post ? (go0 ^ dreg<IX>(g + u, rout)) : (gn0 ^ dreg<IX>(g + u, rnat));
                    if ((gi & (IX)tz.mask) == (IX)tz.vals) e[u] += tz.e;
                }
            }
#pragma unroll
            for (int u = 0; u < GROUP; ++u) x[g + u] = mul_ik(x[g + u], e[u] & 3);
        }
#pragma unroll
        for (int u = 0; u < GROUP; ++u) {
            long long vx = x[g + u].x, vy = x[g + u].y;
            if (k > 0) {
                vx = (vx + half) >> k;
                vy = (vy + half) >> k;
            } else if (k < 0) {
                vx = (long long)((unsigned long long)vx << (-k));
                vy = (long long)((unsigned long long)vy << (-k));
            }
            __stcs(reinterpret_cast<longlong2*>(a.psi_out + (go0 ^ dreg<IX>(g + u, rout))), make_longlong2(vx, vy));
        }
    }
    }   // tiles (disjoint index sets: no ordering between them is needed)
}

// ------------------------------------------------- affine monomial run --
// One pass for a run of monomial gates whose index maps are affine over
// GF(2) (X, CNOT, SWAP, any permutation of two or three qubits) followed by
// diagonal gates: the run's product is one monomial operator (a DAX: one
// nonzero per row), out[i] = D(i) in[F^-1(i)], with F the composed affine
// index map and D the product of the diagonals on the output index.  The
// output is walked in tiles of its 12 low bits (thread bits 0..8, register
// bits 9..11: every store is a coalesced row); each amplitude is gathered
// from F^-1(i), whose 128-byte rows the low bits keep together.  D is two
// table lookups: table A over the 12 local bits and up to 8 selected tile
// bits, and a per-tile factor from table T over the remaining tile bits
// (with exact sign terms on tile bits); sign terms with local bits outside
// A's selection apply per amplitude.  Out of place only (tiles read other
// tiles' amplitudes).  Resident int64 fixed point, as the table pass; QIN /
// QOUT = 0 convert from / to doubles at the run's ends.
constexpr int AMP_MAX_XOFF = 48;
constexpr int AMP_MAX_Z4 = 16;
constexpr int AMP_MAX_TZ4 = 32;
constexpr int AMP_A_SEL = 8;
constexpr int AMP_T_BITS = 16;
struct AmpArgs {
    const double2* psi;
    double2* psi_out;              // must differ from psi
    const int4* tab;
    const int* qS;                 // resident scale exponent (device)
    unsigned long long in_t[DPASS_TBITS], in_r[DPASS_RBITS], in_c;   // F^-1 of thread / register bits, of 0
    unsigned long long in_w[AMP_MAX_XOFF];   // F^-1(e_q) ^ e_q for tile bit q = in_q[i]
    int8_t in_q[AMP_MAX_XOFF];
    int in_nq;
    int a_off, a_nt;               // table A: 2^(12 + a_nt) entries at tab + a_off
    int8_t a_q[AMP_A_SEL];
    int t_off, t_nt;               // table T: 2^t_nt entries (t_off < 0: none)
    int8_t t_q[AMP_T_BITS];
    int ntz;                       // sign terms on tile bits (per tile)
    DZ4 tz[AMP_MAX_TZ4];
    int nz;                        // sign terms with local bits: match on the output index outside
    DZ4 z4[AMP_MAX_Z4];            // register bits 9..11 (mask, vals), e = i^e ...
    uint8_t z4j[AMP_MAX_Z4];       // ... on the registers j whose bits 9..11 match (bit j)
    int qgi;                       // input format: value * 2^(*qS - qgi)
    int shift;                     // right shift into the next pass's format
    uint32_t ntiles;
    // Tile groups: the output tiles whose amplitudes come from the same
    // input rows (the images of row bits 0..2 under F, above bit 11) run
    // one after another in one CTA, so that a row read in halves is read
    // from DRAM once.  Tile (g, u) = base(g) ^ hv[u], base(g) deposits g
    // into the tile-index bits outside the group's pivots (runs).
    uint32_t ngroups;
    int h;                         // 2^h tiles per group (h <= 3)
    uint32_t hv[8];
    unsigned long long dgi[8];     // F^-1(hv[u] << 12)
    uint32_t dasel[8], dtsel[8];   // selection bits of hv[u] << 12 for tables A and T
    int g_nruns;
    uint32_t g_src[8], g_w[8], g_dst[8];
    int nperm, ndiag;              // the run's gates (description only)
    // readout in the pass that writes doubles (RD variant): per CTA the
    // partial sums of |a|^2, (1 - 2 bit_q) |a|^2 and (n - 2 popcount) |a|^2
    // of the amplitudes it stores, in float64
    double* rd_partial;
    int rd_q, rd_n;
};

__device__ __forceinline__ uint32_t amp_sel(unsigned long long v, const int8_t* q, int nt) {
    uint32_t s = 0;
    for (int f = 0; f < nt; ++f) s |= (uint32_t)((v >> q[f]) & 1ull) << f;
    return s;
}
__device__ __forceinline__ int4 q61_split(long long re, long long im) {
    return make_int4((int)(re >> 31), (int)((unsigned)re & 0x7FFFFFFFu), (int)(im >> 31),
                     (int)((unsigned)im & 0x7FFFFFFFu));
}

template <int QIN, int QOUT, typename IX, int RD = 0>
__global__ void __launch_bounds__(512, 2) k_amp(const __grid_constant__ AmpArgs a) {
    static_assert(RD == 0 || QOUT == 0, "the readout variant writes doubles");
    constexpr int NA = 1 << DPASS_RBITS;
    const uint32_t tid = threadIdx.x;
    double r0 = 0.0, r1 = 0.0, r2 = 0.0;   // readout sums (RD)
    IX ti = (IX)a.in_c;
#pragma unroll
    for (int t = 0; t < DPASS_TBITS; ++t) ti ^= ((IX)0 - (IX)((tid >> t) & 1u)) & (IX)a.in_t[t];
    IX rin[DPASS_RBITS];
#pragma unroll
    for (int r = 0; r < DPASS_RBITS; ++r) rin[r] = (IX)a.in_r[r];
    const int S = *a.qS - a.qgi;
    for (uint32_t grp = blockIdx.x; grp < a.ngroups; grp += gridDim.x) {
    uint32_t base = 0;
    for (int i = 0; i < a.g_nruns; ++i) base |= ((grp >> a.g_src[i]) & ((1u << a.g_w[i]) - 1u)) << a.g_dst[i];
    const IX tb0 = (IX)base << 12;
    IX gib = tb0 ^ ti;
    for (int i = 0; i < a.in_nq; ++i)
        if ((tb0 >> a.in_q[i]) & 1u) gib ^= (IX)a.in_w[i];
    const uint32_t asel0 = amp_sel(tb0, a.a_q, a.a_nt);
    const uint32_t tsel0 = a.t_off >= 0 ? amp_sel(tb0, a.t_q, a.t_nt) : 0u;
    for (int u = 0; u < (1 << a.h); ++u) {
        const IX tb = tb0 ^ ((IX)a.hv[u] << 12);
        const IX gi0 = gib ^ (IX)a.dgi[u];
        const IX go0 = tb | (IX)tid;
        const int4* A = a.tab + a.a_off + ((size_t)(asel0 ^ a.dasel[u]) << 12);
        // per-tile factor: table T and the sign terms on tile bits
        int et = 0;
        for (int z = 0; z < a.ntz; ++z)
            if ((tb & (IX)a.tz[z].mask) == (IX)a.tz[z].vals) et += a.tz[z].e;
        const bool tf = a.t_off >= 0 || (et & 3) != 0;
        int4 f = make_int4(1 << 30, 0, 0, 0);   // 1 in split Q61
        if (a.t_off >= 0) f = __ldg(a.tab + a.t_off + (tsel0 ^ a.dtsel[u]));
        if (et & 3) {
            I2 v;
            v.x = ((long long)f.x << 31) + (long long)(unsigned)f.y;
            v.y = ((long long)f.z << 31) + (long long)(unsigned)f.w;
            v = mul_ik(v, et & 3);
            f = q61_split(v.x, v.y);
        }
        // sign-term exponents of the thread's amplitudes (mod 4, as two
        // bit planes over the registers)
        uint32_t e0 = 0, e1 = 0;
        for (int z = 0; z < a.nz; ++z)
            if ((go0 & (IX)a.z4[z].mask) == (IX)a.z4[z].vals) {
                const uint32_t J = a.z4j[z];
                if (a.z4[z].e & 1) {
                    e1 ^= e0 & J;
                    e0 ^= J;
                }
                if (a.z4[z].e & 2) e1 ^= J;
            }
        // streaming loads (cached loads halve the DRAM re-reads of half
        // rows but run slower: the pass is bound by its products)
        I2 x[NA];
#pragma unroll
        for (int j = 0; j < NA; ++j) {
            const longlong2 v = __ldcs(reinterpret_cast<const longlong2*>(a.psi + (gi0 ^ dreg<IX>(j, rin))));
            if constexpr (QIN == 0) {
                x[j].x = d2fix(__longlong_as_double(v.x), S);
                x[j].y = d2fix(__longlong_as_double(v.y), S);
            } else {
                x[j].x = v.x;
                x[j].y = v.y;
            }
        }
        const int k = a.shift;
        const long long half = k > 0 ? (1ll << (k - 1)) : 0ll;
#pragma unroll
        for (int j = 0; j < NA; ++j) {
            const uint32_t l = tid | ((uint32_t)j << 9);
            x[j] = qcmul4_fast(__ldg(A + l), x[j]);
            if (tf) x[j] = qcmul4_fast(f, x[j]);
            if (a.nz) x[j] = mul_ik(x[j], (int)(((e0 >> j) & 1u) | (((e1 >> j) & 1u) << 1)));
            long long vx = x[j].x, vy = x[j].y;
            if constexpr (QOUT == 0) {
                const double dx = fix2d(vx, S), dy = fix2d(vy, S);
                const IX go = go0 | ((IX)j << 9);
                __stcs(a.psi_out + go, make_double2(dx, dy));
                if constexpr (RD == 1) {
                    const double p = fma(dx, dx, dy * dy);
                    r0 += p;
                    if (((unsigned long long)go >> a.rd_q) & 1ull) r1 += p;
                    r2 = fma((double)__popcll((unsigned long long)go), p, r2);
                }
            } else {
                if (k > 0) {
                    vx = (vx + half) >> k;
                    vy = (vy + half) >> k;
                } else if (k < 0) {
                    vx = (long long)((unsigned long long)vx << (-k));
                    vy = (long long)((unsigned long long)vy << (-k));
                }
                __stcs(reinterpret_cast<longlong2*>(a.psi_out + (go0 | ((IX)j << 9))), make_longlong2(vx, vy));
            }
        }
    }   // tiles of the group
    }   // groups
    if constexpr (RD == 1) {
        // fixed-order block sums: warps by shuffles, then warp 0
        __shared__ double sh[3][16];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            r0 += __shfl_down_sync(0xffffffffu, r0, o);
            r1 += __shfl_down_sync(0xffffffffu, r1, o);
            r2 += __shfl_down_sync(0xffffffffu, r2, o);
        }
        const int w = (int)(tid >> 5), l = (int)(tid & 31u);
        if (l == 0) {
            sh[0][w] = r0;
            sh[1][w] = r1;
            sh[2][w] = r2;
        }
        __syncthreads();
        if (w == 0) {
            r0 = l < 16 ? sh[0][l] : 0.0;
            r1 = l < 16 ? sh[1][l] : 0.0;
            r2 = l < 16 ? sh[2][l] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                r0 += __shfl_down_sync(0xffffffffu, r0, o);
                r1 += __shfl_down_sync(0xffffffffu, r1, o);
                r2 += __shfl_down_sync(0xffffffffu, r2, o);
            }
            if (l == 0) {
                // <Z_q> = norm - 2 mass(bit q = 1); sum_q <Z_q> = n norm - 2 sum popcount |a|^2
                a.rd_partial[3 * blockIdx.x + 0] = r0;
                a.rd_partial[3 * blockIdx.x + 1] = r0 - 2.0 * r1;
                a.rd_partial[3 * blockIdx.x + 2] = (double)a.rd_n * r0 - 2.0 * r2;
            }
        }
    }
}

}  // namespace mera
