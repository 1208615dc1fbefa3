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
#pragma once

#include "kernels.cuh"

namespace mera {

constexpr int FR = 4;              // register bits per thread
constexpr int FRA = 1 << FR;       // amplitudes per thread
constexpr int TILE_MAX_PHASES = 32;
constexpr int TILE_MAX_OPS = 192;
constexpr int TILE_MAX_COEF = 448;

enum TileOpType : int8_t {
    TOP_G1 = 0,       // dense 2x2 on one register bit (coef[0..3])
    TOP_G1MONO = 1,   // swap of the pair with phases (codes / coef[0..1])
    TOP_H = 2,        // unscaled Hadamard butterfly (pass scale at the end)
    TOP_G2 = 3,       // dense 4x4 on register bits a > b
    TOP_G2MONO = 4,   // monomial 4x4: row s takes phase(s) * amp perm(s)
    TOP_G3 = 5,       // dense 8x8 on register bits a > b > c
    TOP_G3MONO = 6,
    TOP_DIAG = 7,     // diagonal on any bits: amp *= v[sub] where flagged
};

struct TileOp {
    int8_t type;
    int8_t a, b, c;      // register bits (a is the most significant sub-index bit)
    int8_t nt;           // diag: number of targets
    int8_t tq[3];        // diag: global target positions (tq[0] most significant)
    int32_t coef;        // first coefficient in PassArgs::coef
    uint32_t flags;      // diag: bit s set when sub-index s changes
    uint32_t codes;      // phase codes, 3 bits per row / sub-index
    uint32_t perm;       // monomial: source sub-index of row s, 3 bits per row
    uint64_t cmask;      // control qubits (global positions)
    uint64_t cvals;      // their required values
};

struct TilePhase {
    int8_t rb[FR];       // local tile bits held in registers, ascending
    int16_t op_begin, op_end;
};

template <typename V>
struct PassArgs {
    V* psi;
    int K;               // tile bits
    int nph;             // phases
    int load_smem;       // 1: stage the first phase's load through shared memory
    int store_smem;      // 1: stage the last phase's store through shared memory
    double scale;        // applied to every amplitude at the end of the pass
    int tpos[16];        // global bit of local bit j, ascending
    TilePhase ph[TILE_MAX_PHASES];
    TileOp ops[TILE_MAX_OPS];
    V coef[TILE_MAX_COEF];
};

// ----------------------------------------------------------- bit helpers --
// Shared-memory slot of local index l: XOR-fold the higher bit groups into
// the lowest S bits (S = log2 of amplitudes per 128-byte row) so that the
// strided register gathers hit distinct banks.
template <typename V>
__device__ __forceinline__ int swz(int l) {
    constexpr int S = sizeof(V) == 16 ? 3 : 4;
    constexpr int M = (1 << S) - 1;
    const int h = l >> S;
    return l ^ ((h ^ (h >> S) ^ (h >> (2 * S)) ^ (h >> (3 * S)) ^ (h >> (4 * S))) & M);
}

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

// ------------------------------------------------------------ op bodies --
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
template <typename V>
__device__ __forceinline__ V vscale(V a, double s) {
    a.x = (decltype(a.x))(a.x * s);
    a.y = (decltype(a.y))(a.y * s);
    return a;
}

template <typename V, int B>
__device__ __forceinline__ void op_g1(V (&x)[FRA], const TileOp& o, const V* cf, uint64_t gb, const uint64_t* gm) {
#pragma unroll
    for (int j = 0; j < FRA; ++j) {
        if (j & (1 << B)) continue;
        const int j1 = j | (1 << B);
        if (((gb | dep4(j, gm)) & o.cmask) != o.cvals) continue;
        const V a0 = x[j], a1 = x[j1];
        x[j] = cdot2(cf[0], a0, cf[1], a1);
        x[j1] = cdot2(cf[2], a0, cf[3], a1);
    }
}

template <typename V, int B>
__device__ __forceinline__ void op_g1mono(V (&x)[FRA], const TileOp& o, const V* cf, uint64_t gb, const uint64_t* gm) {
    const int c0 = code_at(o.codes, 0), c1 = code_at(o.codes, 1);
#pragma unroll
    for (int j = 0; j < FRA; ++j) {
        if (j & (1 << B)) continue;
        const int j1 = j | (1 << B);
        if (((gb | dep4(j, gm)) & o.cmask) != o.cvals) continue;
        const V a0 = x[j], a1 = x[j1];
        x[j] = apply_phase(c0, cf[0], a1);
        x[j1] = apply_phase(c1, cf[1], a0);
    }
}

template <typename V, int B>
__device__ __forceinline__ void op_h(V (&x)[FRA]) {
#pragma unroll
    for (int j = 0; j < FRA; ++j) {
        if (j & (1 << B)) continue;
        const int j1 = j | (1 << B);
        const V a0 = x[j], a1 = x[j1];
        x[j] = vadd(a0, a1);
        x[j1] = vsub(a0, a1);
    }
}

template <typename V, int A, int B>
__device__ __forceinline__ void op_g2(V (&x)[FRA], const TileOp& o, const V* cf, uint64_t gb, const uint64_t* gm,
                                      bool mono) {
#pragma unroll
    for (int j = 0; j < FRA; ++j) {
        if (j & ((1 << A) | (1 << B))) continue;
        if (((gb | dep4(j, gm)) & o.cmask) != o.cvals) continue;
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
                x[id[s]] = apply_phase(code_at(o.codes, s), cf[s], v);
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

template <typename V, int A, int B, int C>
__device__ __forceinline__ void op_g3(V (&x)[FRA], const TileOp& o, const V* cf, uint64_t gb, const uint64_t* gm,
                                      bool mono) {
#pragma unroll
    for (int j = 0; j < FRA; ++j) {
        if (j & ((1 << A) | (1 << B) | (1 << C))) continue;
        if (((gb | dep4(j, gm)) & o.cmask) != o.cvals) continue;
        int id[8];
#pragma unroll
        for (int s = 0; s < 8; ++s)
            id[s] = j | ((s & 4) ? (1 << A) : 0) | ((s & 2) ? (1 << B) : 0) | ((s & 1) ? (1 << C) : 0);
        V in[8];
#pragma unroll
        for (int s = 0; s < 8; ++s) in[s] = x[id[s]];
        if (mono) {
#pragma unroll
            for (int s = 0; s < 8; ++s) {
                const int src = (int)((o.perm >> (3 * s)) & 7u);
                V v = in[0];
#pragma unroll
                for (int u = 1; u < 8; ++u)
                    if (src == u) v = in[u];
                x[id[s]] = apply_phase(code_at(o.codes, s), cf[s], v);
            }
        } else {
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                V acc = cmul(cf[r * 8], in[0]);
#pragma unroll
                for (int c = 1; c < 8; ++c) acc = cfma(cf[r * 8 + c], in[c], acc);
                x[id[r]] = acc;
            }
        }
    }
}

template <typename V>
__device__ __forceinline__ void op_diag(V (&x)[FRA], const TileOp& o, const V* cf, uint64_t gb, const uint64_t* gm) {
#pragma unroll
    for (int j = 0; j < FRA; ++j) {
        const uint64_t g = gb | dep4(j, gm);
        if ((g & o.cmask) != o.cvals) continue;
        int sub = 0;
        for (int t = 0; t < o.nt; ++t) sub = (sub << 1) | (int)((g >> o.tq[t]) & 1ull);
        if ((o.flags >> sub) & 1u) x[j] = apply_phase(code_at(o.codes, sub), cf[sub], x[j]);
    }
}

template <typename V>
__device__ __forceinline__ void apply_tile_op(V (&x)[FRA], const TileOp& o, const V* cf, uint64_t gb,
                                              const uint64_t* gm) {
    switch (o.type) {
    case TOP_G1:
        switch (o.a) {
        case 0: op_g1<V, 0>(x, o, cf, gb, gm); break;
        case 1: op_g1<V, 1>(x, o, cf, gb, gm); break;
        case 2: op_g1<V, 2>(x, o, cf, gb, gm); break;
        default: op_g1<V, 3>(x, o, cf, gb, gm); break;
        }
        break;
    case TOP_G1MONO:
        switch (o.a) {
        case 0: op_g1mono<V, 0>(x, o, cf, gb, gm); break;
        case 1: op_g1mono<V, 1>(x, o, cf, gb, gm); break;
        case 2: op_g1mono<V, 2>(x, o, cf, gb, gm); break;
        default: op_g1mono<V, 3>(x, o, cf, gb, gm); break;
        }
        break;
    case TOP_H:
        switch (o.a) {
        case 0: op_h<V, 0>(x); break;
        case 1: op_h<V, 1>(x); break;
        case 2: op_h<V, 2>(x); break;
        default: op_h<V, 3>(x); break;
        }
        break;
    case TOP_G2:
    case TOP_G2MONO: {
        const bool mono = o.type == TOP_G2MONO;
        switch (o.a * 4 + o.b) {
        case 1: op_g2<V, 1, 0>(x, o, cf, gb, gm, mono); break;
        case 2 * 4 + 0: op_g2<V, 2, 0>(x, o, cf, gb, gm, mono); break;
        case 2 * 4 + 1: op_g2<V, 2, 1>(x, o, cf, gb, gm, mono); break;
        case 3 * 4 + 0: op_g2<V, 3, 0>(x, o, cf, gb, gm, mono); break;
        case 3 * 4 + 1: op_g2<V, 3, 1>(x, o, cf, gb, gm, mono); break;
        default: op_g2<V, 3, 2>(x, o, cf, gb, gm, mono); break;
        }
        break;
    }
    case TOP_G3:
    case TOP_G3MONO: {
        const bool mono = o.type == TOP_G3MONO;
        switch (6 - o.a - o.b - o.c) {   // a > b > c in 0..3: the missing bit names the triple
        case 3: op_g3<V, 2, 1, 0>(x, o, cf, gb, gm, mono); break;
        case 2: op_g3<V, 3, 1, 0>(x, o, cf, gb, gm, mono); break;
        case 1: op_g3<V, 3, 2, 0>(x, o, cf, gb, gm, mono); break;
        default: op_g3<V, 3, 2, 1>(x, o, cf, gb, gm, mono); break;
        }
        break;
    }
    default: op_diag<V>(x, o, cf, gb, gm); break;
    }
}

// ---------------------------------------------------------------- kernel --
template <typename V>
__global__ void __launch_bounds__(512) k_tile(const __grid_constant__ PassArgs<V> a) {
    extern __shared__ __align__(16) unsigned char smraw[];
    V* sm = reinterpret_cast<V*>(smraw);
    const int K = a.K;
    const uint32_t T = 1u << (K - FR);
    const uint32_t tid = threadIdx.x;
    const uint64_t tile = blockIdx.x;
    const uint64_t tb = insert_zeros(tile, a.tpos, K);    // global index of local 0
    V x[FRA];

    if (a.load_smem) {
        // coalesced copy: element tid + i*T, its top FR local bits come from i
        const uint64_t gt = tb | spread_bits(tid, a.tpos, K - FR);
        uint64_t gtop[FR];
#pragma unroll
        for (int r = 0; r < FR; ++r) gtop[r] = 1ull << a.tpos[K - FR + r];
#pragma unroll
        for (int i = 0; i < FRA; ++i) x[i] = a.psi[gt | dep4(i, gtop)];
#pragma unroll
        for (int i = 0; i < FRA; ++i) sm[swz<V>((int)(tid + i * T))] = x[i];
        __syncthreads();
    }

    for (int p = 0; p < a.nph; ++p) {
        const TilePhase& ph = a.ph[p];
        const uint32_t lb = insert_reg_zeros(tid, ph.rb);
        const uint64_t gb = tb | spread_bits(lb, a.tpos, K);
        uint64_t gm[FR];
        int lm[FR];
#pragma unroll
        for (int r = 0; r < FR; ++r) {
            gm[r] = 1ull << a.tpos[ph.rb[r]];
            lm[r] = 1 << ph.rb[r];
        }
        if (p == 0 && !a.load_smem) {
#pragma unroll
            for (int j = 0; j < FRA; ++j) x[j] = a.psi[gb | dep4(j, gm)];
        } else {
#pragma unroll
            for (int j = 0; j < FRA; ++j) x[j] = sm[swz<V>((int)(lb | dep4(j, lm)))];
        }
        for (int o = ph.op_begin; o < ph.op_end; ++o) {
            const TileOp& op = a.ops[o];
            apply_tile_op<V>(x, op, a.coef + op.coef, gb, gm);
        }
        const bool last = (p == a.nph - 1);
        if (last && a.scale != 1.0) {
#pragma unroll
            for (int j = 0; j < FRA; ++j) x[j] = vscale(x[j], a.scale);
        }
        if (last && !a.store_smem) {
#pragma unroll
            for (int j = 0; j < FRA; ++j) a.psi[gb | dep4(j, gm)] = x[j];
        } else {
            // each slot is read and written by its owner only within a phase
#pragma unroll
            for (int j = 0; j < FRA; ++j) sm[swz<V>((int)(lb | dep4(j, lm)))] = x[j];
            __syncthreads();
        }
    }

    if (a.store_smem) {
        const uint64_t gt = tb | spread_bits(tid, a.tpos, K - FR);
        uint64_t gtop[FR];
#pragma unroll
        for (int r = 0; r < FR; ++r) gtop[r] = 1ull << a.tpos[K - FR + r];
#pragma unroll
        for (int i = 0; i < FRA; ++i) a.psi[gt | dep4(i, gtop)] = sm[swz<V>((int)(tid + i * T))];
    }
}

}  // namespace mera
