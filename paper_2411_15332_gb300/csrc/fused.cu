// Fused path: plan tile passes over a gate list and launch the tile kernel.
//
// Planning (host, per circuit):
//  1. Passes.  Gates are taken in circuit order.  A gate joins the current
//     pass if its target qubits fit in the pass's K tile bits (the L lowest
//     bits are always tile bits, so tiles are runs of 128 contiguous bytes);
//     diagonal gates and controls need no tile bits.  A gate that does not
//     fit is deferred, and every later gate sharing a qubit with a deferred
//     gate is deferred too, so only gates on disjoint qubits (which commute)
//     change order.  Deferred gates start the next pass.
//  2. Phases.  Inside a pass, consecutive gates are grouped while the union
//     of their targets fits in FR register bits.
// Each pass reads and writes the state once: 2 x 2^n x element bytes of HBM
// traffic whatever the number of gates it carries.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include <cuda.h>

#include "common.cuh"
#include "fused.cuh"
#include "reduce.cuh"
#include "tile_fns.cuh"

namespace mera {

static int popc(uint64_t x) { return __builtin_popcountll(x); }

// Partial triples a readout summed by the last pass may write (its CTAs).
static constexpr int RD_MAX_PARTIALS = 4096;

int fused_tile_bits(int dtype, int n) {
    int K = dtype == MERA_C128 ? 12 : 13;
    if (const char* e = getenv("MERA_TILE_BITS")) {
        const int v = atoi(e);
        if (v >= FR + 1 && v <= 14) K = v;
    }
    if (K > n) K = n;
    return K;
}

// MERA_BULK=0 stages Hadamard-pass tiles with 16-byte asynchronous copies
// only (no bulk copies).
static bool bulk_enabled() {
    static int v = -1;
    if (v < 0) {
        const char* e = getenv("MERA_BULK");
        v = (e && atoi(e) == 0) ? 0 : 1;
    }
    return v == 1;
}

// Test hook: bytes each bulk-staged tile expects beyond what is copied, so
// that its bounded waits run out (0 in normal use).
static unsigned g_bulk_shortfall = 0;
void fused_set_bulk_shortfall(unsigned bytes) { g_bulk_shortfall = bytes; }

// The tensor-map dimensions of a tile for tiled tensor copies (see
// HPassArgs): the state's amplitude bits 0..n-1 split into runs of tile
// and non-tile bits, ascending; dimension 0 holds re/im and the tile run
// from bit 0 (which must cover bits 0..2: rows of at least 128 bytes).
// Box sizes are at most 256 words per dimension, so long tile runs take
// several dimensions.  The tile's top `m` local bits may count as non-tile
// bits: the tile is then 2^m copies, one per value of those bits.  False if
// more than TMA_DIMS dimensions are needed.
struct TmaDims {
    int m;                      // top local bits iterated by separate copies (0..2)
    uint64_t gdim[TMA_DIMS];    // extent in float64 words (dimension 0) / in steps of its lowest bit
    uint64_t gstride[TMA_DIMS]; // bytes between consecutive coordinates (dimension 0: 8)
    uint32_t box[TMA_DIMS];
    unsigned char sh[TMA_DIMS];
    unsigned mk[TMA_DIMS];
};
static bool tma_dims_m(const int* tpos, int K, int n, int m, TmaDims& d) {
    bool tile[64] = {};
    for (int b = 0; b < K - m; ++b) tile[tpos[b]] = true;
    if (n > 40 || K - m < 3 || !tile[0] || !tile[1] || !tile[2]) return false;
    d.m = m;
    int nd = 0;
    auto add = [&](int lo, int len, bool t) {
        if (nd == TMA_DIMS) return false;
        const uint64_t ext = (nd == 0 ? 2ull : 1ull) << len;
        d.gdim[nd] = ext;
        d.gstride[nd] = nd == 0 ? 8ull : (16ull << lo);
        d.box[nd] = t ? (uint32_t)ext : 1u;
        d.sh[nd] = (unsigned char)(t ? 0 : lo);
        d.mk[nd] = t ? 0u : (unsigned)((1ull << len) - 1ull);
        ++nd;
        return true;
    };
    for (int q = 0; q < n;) {
        int e = q;
        while (e < n && tile[e] == tile[q]) ++e;
        if (tile[q]) {
            for (int lo = q; lo < e;) {
                const int len = std::min(e - lo, nd == 0 ? 7 : 8);
                if (!add(lo, len, true)) return false;
                lo += len;
            }
        } else {
            if (e - q > 31 || !add(q, e - q, false)) return false;   // coordinates are signed 32-bit
        }
        q = e;
    }
    for (; nd < TMA_DIMS; ++nd) {
        d.gdim[nd] = 1;
        d.gstride[nd] = 16ull << n;
        d.box[nd] = 1;
        d.sh[nd] = 0;
        d.mk[nd] = 0;
    }
    return true;
}
static bool tma_dims(const int* tpos, int K, int n, TmaDims& d) {
    for (int m = 0; m <= 2; ++m)
        if (tma_dims_m(tpos, K, n, m, d)) return true;
    return false;
}

// Encode the tensor map of `d` over the state at `base` (the driver's
// encoder, found through the runtime).
static int encode_tile_map(CUtensorMap* m, const void* base, const TmaDims& d) {
    using Encode = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    static Encode fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<Encode>(p);
        cudaGetLastError();
    });
    MERA_RETURN_IF(!fn, MERA_ECUDA, "the driver's tensor-map encoder is not available");
    cuuint64_t gdim[TMA_DIMS], gstr[TMA_DIMS - 1];
    cuuint32_t box[TMA_DIMS], es[TMA_DIMS];
    for (int i = 0; i < TMA_DIMS; ++i) {
        gdim[i] = d.gdim[i];
        box[i] = d.box[i];
        es[i] = 1;
        if (i > 0) gstr[i - 1] = d.gstride[i];
    }
    const CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, TMA_DIMS, const_cast<void*>(base), gdim, gstr, box, es,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    MERA_RETURN_IF(r != CUDA_SUCCESS, MERA_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return MERA_OK;
}

static int low_bits_for(int dtype, int K) {
    int L = dtype == MERA_C128 ? 3 : 4;   // 128 contiguous bytes
    if (const char* e = getenv("MERA_TILE_LOW")) {
        const int v = atoi(e);
        if (v >= 0 && v <= 8) L = v;
    }
    if (L > K - 3) L = K - 3;
    if (L < 0) L = 0;
    return L;
}

struct Pass {
    uint64_t tile_mask = 0;
    std::vector<int> ops;
    int single = -1;     // >= 0: run this op with the per-gate kernel instead
    bool amp = false;    // an affine monomial run (one streaming pass, see AmpRun)
};

// Three-target non-diagonal gates are not fused: they split the circuit and
// run as per-gate kernels.
static bool is_barrier(const PrepOp& P) { return P.k == 3 && P.kind != KIND_DIAG; }

static uint64_t op_qubits(const PrepOp& P) {
    uint64_t m = P.cmask;
    for (int j = 0; j < P.k; ++j) m |= 1ull << P.t[j];
    return m;
}
static uint64_t op_targets(const PrepOp& P) {
    uint64_t m = 0;
    for (int j = 0; j < P.k; ++j) m |= 1ull << P.t[j];
    return m;
}
// Exact in int64 block floating point: butterflies, moves, {1, i, -1, -i}.
static bool op_is_exact(const PrepOp& P) {
    if (P.is_h) return true;
    if (P.kind != KIND_MONO && P.kind != KIND_DIAG) return false;
    for (int s = 0; s < (1 << P.k); ++s) {
        const cplx v = P.v[s];
        if (!(v == cplx(1, 0) || v == cplx(-1, 0) || v == cplx(0, 1) || v == cplx(0, -1))) return false;
    }
    return true;
}


// Passes with at least this many Hadamard levels take exact gates only;
// other gates wait for the next pass.
static constexpr int H_HEAVY = 3;
// At most this many Hadamard levels per pass (growth 2^(H_MAX_PASS / 2)
// before the pass scale).
static constexpr int H_MAX_PASS = 16;

static int coef_need(const PrepOp& P) {
    if (P.bslot >= 0) return 0;
    if (P.kind == KIND_DIAG) return 1 << P.k;
    if (P.is_h) return 0;
    if (P.kind == KIND_MONO) return 1 << P.k;
    return 1 << (2 * P.k);
}

static void plan_segment(const std::vector<PrepOp>& ops, std::vector<int> remaining, int n, int K, int L,
                         std::vector<Pass>& passes);

// A single-qubit diagonal gate (phase on one qubit) -- the kind folded into
// a separable table.
static int diag_qubit(const PrepOp& P) {
    if (P.kind != KIND_DIAG || P.bslot >= 0) return -1;
    if (P.k == 1 && P.cmask == 0) return P.t[0];
    if (P.k == 0 && __builtin_popcountll(P.cmask) == 1) return __builtin_ctzll(P.cmask);
    return -1;
}

// Move single-qubit diagonal gates whose qubit is not a tile bit of their
// pass to the first later pass where it is, when no gate targeting that
// qubit (non-diagonal) runs in between: the diagonal commutes with every
// gate that does not target its qubit, and in a pass where the qubit is a
// tile bit its factor comes from the pass's table instead of a per-tile
// product.
static void sink_diagonals(const std::vector<PrepOp>& ops, std::vector<Pass>& passes) {
    const int np = (int)passes.size();
    for (int i = 0; i < np; ++i) {
        if (passes[i].single >= 0 || passes[i].amp) continue;
        std::vector<int> keep;
        std::vector<std::pair<int, int>> moved;   // (op, target pass)
        for (size_t k = 0; k < passes[i].ops.size(); ++k) {
            const int idx = passes[i].ops[k];
            const int q = diag_qubit(ops[idx]);
            if (q < 0 || ((passes[i].tile_mask >> q) & 1ull)) {
                keep.push_back(idx);
                continue;
            }
            const uint64_t bit = 1ull << q;
            bool blocked = false;
            // later ops of this pass
            for (size_t m = k + 1; m < passes[i].ops.size() && !blocked; ++m) {
                const PrepOp& G = ops[passes[i].ops[m]];
                if (G.kind != KIND_DIAG && (op_targets(G) & bit)) blocked = true;
            }
            int dest = -1;
            for (int j = i + 1; j < np && !blocked; ++j) {
                if (passes[j].amp) {   // its permutations move qubits: stop here
                    blocked = true;
                    break;
                }
                if (passes[j].single >= 0) {
                    const PrepOp& G = ops[passes[j].single];
                    if (op_targets(G) & bit) blocked = true;
                    continue;
                }
                if ((passes[j].tile_mask >> q) & 1ull) {
                    dest = j;
                    break;
                }
                for (int m : passes[j].ops) {
                    const PrepOp& G = ops[m];
                    if (G.kind != KIND_DIAG && (op_targets(G) & bit)) {
                        blocked = true;
                        break;
                    }
                }
            }
            if (dest < 0 || blocked) {
                keep.push_back(idx);
                continue;
            }
            moved.push_back(std::make_pair(idx, dest));
        }
        passes[i].ops.swap(keep);
        // insert at the front of the destination (before every op there)
        for (auto it = moved.rbegin(); it != moved.rend(); ++it)
            passes[it->second].ops.insert(passes[it->second].ops.begin(), it->first);
    }
}

// ------------------------------------------------ affine monomial runs --
// DAX products (Sec. III-A): the product of monomial matrices is monomial,
// so a run of permutation gates followed by diagonal gates is one operator
// with one nonzero per row, out[i] = D(i) in[F^-1(i)].  For permutations
// that are affine maps of the index bits over GF(2) (X, CNOT, SWAP, and any
// permutation of two qubits), F(j) = M j ^ c; D collects the diagonals,
// which no permutation of the run follows, as a function of the output
// index: per-qubit factors lam[q][bit] and patterns on several qubits.

// The new index of old index x under a monomial gate's permutation (row s
// of the gate reads column perm[s]: old pattern perm[s] moves to s).
static uint64_t mono_apply(const PrepOp& P, uint64_t x) {
    if ((x & P.cmask) != P.cvals) return x;
    int s = 0;
    for (int m = 0; m < P.k; ++m) s = (s << 1) | (int)((x >> P.t[m]) & 1ull);
    int sn = s;
    for (int r = 0; r < (1 << P.k); ++r)
        if (P.perm[r] == s) {
            sn = r;
            break;
        }
    for (int m = 0; m < P.k; ++m) {
        const uint64_t bit = (uint64_t)((sn >> (P.k - 1 - m)) & 1);
        x = (x & ~(1ull << P.t[m])) | (bit << P.t[m]);
    }
    return x;
}
// A pure permutation gate (every value 1) whose index map is affine.
static bool mono_affine(const PrepOp& P) {
    if (P.kind != KIND_MONO || P.bslot >= 0) return false;
    for (int s = 0; s < (1 << P.k); ++s)
        if (P.v[s] != cplx(1, 0)) return false;
    int sup[64], m = 0;
    for (int j = 0; j < P.k; ++j) sup[m++] = P.t[j];
    for (int q = 0; q < 64; ++q)
        if ((P.cmask >> q) & 1ull) sup[m++] = q;
    if (m > 6) return false;
    auto vec = [&](int u) {
        uint64_t x = 0;
        for (int b = 0; b < m; ++b)
            if ((u >> b) & 1) x |= 1ull << sup[b];
        return x;
    };
    const uint64_t g0 = mono_apply(P, 0);
    for (int u = 0; u < (1 << m); ++u)
        for (int w = u + 1; w < (1 << m); ++w)
            if ((mono_apply(P, vec(u) ^ vec(w)) ^ g0) != (mono_apply(P, vec(u)) ^ mono_apply(P, vec(w))))
                return false;
    return true;
}

static int phase_code_f(cplx v);
static uint32_t unit_exp(cplx v);

struct AmpTerm {
    uint64_t mask, vals;   // applies where (i & mask) == vals
    cplx v;
};
struct AmpRun {
    int n = 0;
    uint64_t col[64];      // M e_b
    uint64_t c = 0;
    cplx lam[64][2];
    cplx konst = 1;
    std::vector<AmpTerm> terms;
    std::vector<int> ops;
    bool diag = false;     // a diagonal was taken: no permutation may follow
    uint64_t touched = 0;
    explicit AmpRun(int nn) : n(nn) {
        for (int b = 0; b < 64; ++b) {
            col[b] = 1ull << b;
            lam[b][0] = lam[b][1] = 1;
        }
    }
    // take gate idx if the run stays one affine monomial operator
    bool take(const std::vector<PrepOp>& all, int idx) {
        const PrepOp& P = all[idx];
        if (P.kind == KIND_MONO) {
            if (diag || !mono_affine(P)) return false;
            const uint64_t g0 = mono_apply(P, 0);
            for (int b = 0; b < n; ++b) col[b] = mono_apply(P, col[b]) ^ g0;
            c = mono_apply(P, c);
        } else if (P.kind == KIND_DIAG && P.bslot < 0) {
            diag = true;
            uint64_t tm = 0;
            for (int j = 0; j < P.k; ++j) tm |= 1ull << P.t[j];
            for (int sp = 0; sp < (1 << P.k); ++sp) {
                const cplx v = P.v[sp];
                if (v == cplx(1, 0)) continue;
                uint64_t vals = P.cvals;
                for (int j = 0; j < P.k; ++j)
                    if ((sp >> (P.k - 1 - j)) & 1) vals |= 1ull << P.t[j];
                const uint64_t mask = P.cmask | tm;
                if (mask == 0) konst *= v;
                else if (popc(mask) == 1) lam[__builtin_ctzll(mask)][vals ? 1 : 0] *= v;
                else terms.push_back(AmpTerm{mask, vals, v});
            }
        } else {
            return false;
        }
        ops.push_back(idx);
        touched |= op_qubits(P);
        return true;
    }
};

// Placement of a run's diagonal: local bits 0..11 (table A, with up to
// AMP_A_SEL selected tile bits), table T over other tile bits (one factor
// per tile), exact sign terms per tile or per amplitude.  False if the run
// does not fit (then it is shortened).
struct AmpLayout {
    uint64_t selA = 0, tdom = 0;
    std::vector<int> inA, inT, tileZ, elemZ;   // term indices
};
static bool amp_layout(const AmpRun& r, AmpLayout& L) {
    const uint64_t LOC = 0xFFFull;
    L = AmpLayout();
    auto z4 = [](cplx v) { return phase_code_f(v) <= 3; };
    // tile bits of mixed (local and tile) terms: general phases must be
    // selected by table A; exact ones preferably, else per amplitude
    uint64_t must = 0;
    int freq[64] = {0};
    for (const AmpTerm& t : r.terms) {
        const uint64_t tm = t.mask & ~LOC;
        if ((t.mask & LOC) && tm) {
            if (!z4(t.v)) must |= tm;
            else
                for (int q = 0; q < 64; ++q)
                    if ((tm >> q) & 1ull) ++freq[q];
        }
    }
    if (popc(must) > AMP_A_SEL) return false;
    L.selA = must;
    while (popc(L.selA) < AMP_A_SEL) {
        int best = -1;
        for (int q = 12; q < r.n; ++q)
            if (!((L.selA >> q) & 1ull) && freq[q] > 0 && (best < 0 || freq[q] > freq[best])) best = q;
        if (best < 0) break;
        L.selA |= 1ull << best;
    }
    for (int q = 12; q < r.n; ++q)
        if (!((L.selA >> q) & 1ull) && (r.lam[q][0] != cplx(1, 0) || r.lam[q][1] != cplx(1, 0))) L.tdom |= 1ull << q;
    for (size_t i = 0; i < r.terms.size(); ++i) {
        const AmpTerm& t = r.terms[i];
        const uint64_t tm = t.mask & ~LOC;
        if (!(tm & ~L.selA)) L.inA.push_back((int)i);
        else if (t.mask & LOC) {
            if (!z4(t.v)) return false;
            L.elemZ.push_back((int)i);
        } else if (!z4(t.v)) {
            L.tdom |= tm;
            L.inT.push_back((int)i);
        }
    }
    // exact tile-only terms: in T when its bits are there, else per tile
    for (size_t i = 0; i < r.terms.size(); ++i) {
        const AmpTerm& t = r.terms[i];
        const uint64_t tm = t.mask & ~LOC;
        if ((t.mask & LOC) || !(tm & ~L.selA) || !z4(t.v)) continue;
        if (!(tm & ~L.tdom)) L.inT.push_back((int)i);
        else L.tileZ.push_back((int)i);
    }
    return popc(L.tdom) <= AMP_T_BITS && (int)L.elemZ.size() <= AMP_MAX_Z4 && (int)L.tileZ.size() <= AMP_MAX_TZ4;
}

// The longest affine monomial run starting at ops[pos], shortened until
// its diagonal fits the layout.
static constexpr size_t AMP_MAX_RUN = 2048;   // gates per run (bounds the planning work)
static AmpRun amp_grow(const std::vector<PrepOp>& ops, const std::vector<int>& order, size_t pos, int n) {
    AmpRun r(n);
    for (size_t k = pos; k < order.size() && r.ops.size() < AMP_MAX_RUN; ++k) {
        AmpRun next = r;
        if (!next.take(ops, order[k])) break;
        // a new term or a factor on another tile qubit may overflow the tables
        AmpLayout L;
        if (!amp_layout(next, L)) break;
        r = std::move(next);
    }
    return r;
}
// Worth a pass of its own: the run reaches more qubits than a tile pass
// holds beside its row bits, with a few gates at least.
static bool amp_worth(const AmpRun& r, int K) { return r.ops.size() >= 4 && popc(r.touched) > K - 3; }

static std::vector<Pass> plan_passes(const std::vector<PrepOp>& ops, int n, int K, int L, bool amp_ok) {
    std::vector<Pass> passes;
    std::vector<int> seg;
    std::vector<int> order;
    for (int i = 0; i < (int)ops.size(); ++i)
        if (ops[i].kind != KIND_IDENTITY) order.push_back(i);
    for (size_t k = 0; k < order.size(); ++k) {
        const int i = order[k];
        if (amp_ok && (ops[i].kind == KIND_MONO || ops[i].kind == KIND_DIAG)) {
            AmpRun r = amp_grow(ops, order, k, n);
            if (amp_worth(r, K)) {
                plan_segment(ops, seg, n, K, L, passes);
                seg.clear();
                Pass a;
                a.amp = true;
                a.ops = r.ops;
                passes.push_back(a);
                k += r.ops.size() - 1;
                continue;
            }
        }
        if (is_barrier(ops[i])) {
            plan_segment(ops, seg, n, K, L, passes);
            seg.clear();
            Pass b;
            b.single = i;
            passes.push_back(b);
            continue;
        }
        seg.push_back(i);
    }
    plan_segment(ops, seg, n, K, L, passes);
    sink_diagonals(ops, passes);
    return passes;
}

static void plan_segment(const std::vector<PrepOp>& ops, std::vector<int> remaining, int n, int K, int L,
                         std::vector<Pass>& passes) {
    const uint64_t low = (L >= 64) ? ~0ull : ((1ull << L) - 1ull);
    while (!remaining.empty()) {
        Pass p;
        p.tile_mask = low;
        uint64_t blocked = 0;
        int nops = 0, ncoef = 0;
        // register phases as build_pass will form them (same order, same rule)
        uint64_t ph_need = 0;
        int nph = 1;
        int nh = 0;
        std::vector<int> deferred;
        for (int idx : remaining) {
            const PrepOp& P = ops[idx];
            const uint64_t q = op_qubits(P);
            bool take = !(q & blocked);
            // Hadamard-heavy passes keep to exact gates (butterflies, moves,
            // unit phases): their kernel variant stays lean
            if (take && !op_is_exact(P) && nh >= H_HEAVY) take = false;
            // the pass scale 2^(-nh/2) applies at its end: cap the growth of
            // the unnormalised butterflies (fixed-point headroom)
            if (take && P.is_h && nh >= H_MAX_PASS) take = false;
            if (take && (nops + 1 > TILE_MAX_OPS || ncoef + coef_need(P) > TILE_MAX_COEF)) take = false;
            if (take && P.kind != KIND_DIAG) {
                const uint64_t t = op_targets(P);
                const uint64_t m = p.tile_mask | t;
                const bool new_phase = popc(ph_need | t) > FR;
                if (popc(m) > K || (new_phase && nph + 1 > TILE_MAX_PHASES)) {
                    take = false;
                } else {
                    p.tile_mask = m;
                    if (new_phase) {
                        ++nph;
                        ph_need = t;
                    } else {
                        ph_need |= t;
                    }
                }
            }
            if (take) {
                p.ops.push_back(idx);
                ++nops;
                ncoef += coef_need(P);
                if (P.is_h) ++nh;
            } else {
                deferred.push_back(idx);
                blocked |= q;
            }
        }
        // fill the remaining tile bits with the lowest free positions
        for (int b = 0; b < n && popc(p.tile_mask) < K; ++b) p.tile_mask |= 1ull << b;
        passes.push_back(std::move(p));
        remaining.swap(deferred);
    }
}

template <typename V>
static V to_v(cplx c) {
    V r;
    r.x = (decltype(r.x))c.real();
    r.y = (decltype(r.y))c.imag();
    return r;
}

// Coefficient slot of the pass: float2 for complex64 (FP engine); for
// complex128 the int64 engine reads Q62 fixed point (value * 2^62, |value|
// < 2) from the same 16 bytes.
template <typename V>
static V enc(cplx c, bool q62);
template <>
float2 enc<float2>(cplx c, bool) {
    return to_v<float2>(c);
}
template <>
double2 enc<double2>(cplx c, bool q62) {
    if (!q62) return to_v<double2>(c);
    const double s = 4611686018427387904.0;   // 2^62
    long long q[2] = {std::llround(c.real() * s), std::llround(c.imag() * s)};
    double2 r;
    memcpy(&r, q, sizeof(r));
    return r;
}

// Max absolute row sum of a 2^k x 2^k matrix (bounds the growth of one
// application in the max norm) and whether it is unitary.
static void op_gain(const PrepOp& P, double* rowsum, bool* unitary) {
    if (P.bslot >= 0) {   // per-state unitary 2x2
        *rowsum = std::sqrt(2.0);
        *unitary = true;
        return;
    }
    const int d = 1 << P.k;
    double best = 0.0;
    for (int r = 0; r < d; ++r) {
        double s = 0.0;
        for (int c = 0; c < d; ++c) s += std::abs(P.m[r * d + c]);
        best = std::max(best, s);
    }
    bool u = true;
    for (int r = 0; r < d && u; ++r)
        for (int c = 0; c < d && u; ++c) {
            cplx acc = 0;
            for (int j = 0; j < d; ++j) acc += std::conj(P.m[j * d + r]) * P.m[j * d + c];
            if (std::abs(acc - (r == c ? cplx(1, 0) : cplx(0, 0))) > 1e-9) u = false;
        }
    *rowsum = best;
    *unitary = u;
}

static int phase_code_f(cplx v) {
    if (v == cplx(1, 0)) return 0;
    if (v == cplx(0, 1)) return 1;
    if (v == cplx(-1, 0)) return 2;
    if (v == cplx(0, -1)) return 3;
    return 4;
}

static uint32_t unit_exp(cplx v) { return (uint32_t)phase_code_f(v); }

// Host-side builder of one pass: kernel arguments plus the separable
// diagonal tables (appended to `tabs`, offsets relative to its start).
template <typename V>
struct PassBuilder {
    PassArgs<V>& A;
    std::vector<V>& tabs;
    const std::vector<PrepOp>& ops;
    int K, n;
    int local_of[64];
    int nop = 0, ncoef = 0, nz4 = 0, nnt = 0;
    bool i64 = false;       // coefficients in Q62 fixed point (int64 engines)
    int engine = ENG_FP;
    bool fp_only = false;   // keep every pass in the float engine
    bool qres = false;      // resident fixed point: every pass in ENG_Q
    bool stage_load = false;  // stage the first load through shared memory (pipelined kernel)

    // The open separable-diagonal op: later diagonal runs fold into its
    // table while only pure index permutations (X, CNOT, SWAP, Toffoli:
    // monomials with all values 1) run in between -- D_B applied after a
    // permutation P equals D_B(P(l)) applied before it.  Non-tile control
    // bits of those permutations and non-tile diagonal qubits select one
    // of at most 2^DSEP_SEL_BITS tables.
    struct Factor {
        int q;
        cplx lam[2];
    };
    struct Run {
        std::vector<Factor> fac;
        std::vector<int> perms;   // permutation ops between the table op and this run
        std::vector<Z4Term> z4;   // unit-phase patterns folded into the table
    };
    struct OpenTable {
        bool open = false;
        int opi = -1;
        std::vector<int> selq;    // selection qubits (non-tile)
        std::vector<Run> runs;
        std::vector<int> perms;   // permutation ops since the table op
    } ot;

    PassBuilder(PassArgs<V>& a, std::vector<V>& t, const std::vector<PrepOp>& o, int k, int nn)
        : A(a), tabs(t), ops(o), K(k), n(nn) {}

    static bool pure_perm(const PrepOp& P) {
        if (P.kind != KIND_MONO || P.bslot >= 0 || P.k > 2) return false;
        for (int s = 0; s < (1 << P.k); ++s)
            if (P.v[s] != cplx(1, 0)) return false;
        return true;
    }

    // A non-diagonal gate joins the pass: the open table stays open only
    // across pure permutations.
    void note_gate(int idx) {
        if (!ot.open) return;
        if (pure_perm(ops[idx])) ot.perms.push_back(idx);
        else ot.open = false;
    }

    // Bit of qubit q at local index l (local qubits) or from the selection
    // index (selection qubits).
    int bit_at(int q, uint32_t l, uint32_t sel, const std::vector<int>& selq) const {
        if (local_of[q] >= 0) return (int)((l >> local_of[q]) & 1u);
        for (size_t f = 0; f < selq.size(); ++f)
            if (selq[f] == q) return (int)((sel >> f) & 1u);
        return 0;
    }

    // Where the amplitude at local index l (tile selection sel) sits after
    // the permutations perms.
    uint32_t permute(uint32_t l, uint32_t sel, const std::vector<int>& perms, const std::vector<int>& selq) const {
        for (int idx : perms) {
            const PrepOp& P = ops[idx];
            bool on = true;
            for (int q = 0; q < n && on; ++q)
                if ((P.cmask >> q) & 1ull) on = bit_at(q, l, sel, selq) == (int)((P.cvals >> q) & 1ull);
            if (!on) continue;
            int s = 0;
            for (int j = 0; j < P.k; ++j) s = (s << 1) | (int)((l >> local_of[P.t[j]]) & 1u);
            int r = 0;   // the row that reads column s
            for (int rr = 0; rr < (1 << P.k); ++rr)
                if (P.perm[rr] == s) r = rr;
            for (int j = 0; j < P.k; ++j) {
                const uint32_t b = 1u << local_of[P.t[j]];
                l = ((r >> (P.k - 1 - j)) & 1) ? (l | b) : (l & ~b);
            }
        }
        return l;
    }

    // (Re)write the open table: T[sel][l] = prod over runs and their factors.
    int write_table() {
        TileOp& o = A.ops[ot.opi];
        const size_t T = (size_t)1 << K;
        const int nsel = (int)ot.selq.size();
        MERA_RETURN_IF(nnt + nsel > TILE_MAX_NT, MERA_EUNSUPPORTED, "too many table selection qubits");
        o.aux2 = nnt;
        for (int q : ot.selq) A.ntq[nnt++] = (int8_t)q;
        o.nt = (int8_t)nsel;
        o.aux = (int)tabs.size();
        tabs.resize(tabs.size() + (T << nsel));
        // folded patterns as (local mask, local values, selection mask, selection values)
        struct Pat {
            uint32_t lm, lv, sm, sv;
            int e;
        };
        std::vector<std::vector<Pat>> pats(ot.runs.size());
        for (size_t ri = 0; ri < ot.runs.size(); ++ri)
            for (const Z4Term& z : ot.runs[ri].z4) {
                Pat pt{0, 0, 0, 0, z.e};
                for (int q = 0; q < n; ++q) {
                    if (!((z.mask >> q) & 1ull)) continue;
                    const uint32_t v = (uint32_t)((z.vals >> q) & 1ull);
                    if (local_of[q] >= 0) {
                        pt.lm |= 1u << local_of[q];
                        pt.lv |= v << local_of[q];
                    } else {
                        const int f = (int)(std::find(ot.selq.begin(), ot.selq.end(), q) - ot.selq.begin());
                        pt.sm |= 1u << f;
                        pt.sv |= v << f;
                    }
                }
                pats[ri].push_back(pt);
            }
        static const cplx ipow[4] = {cplx(1, 0), cplx(0, 1), cplx(-1, 0), cplx(0, -1)};
        for (uint32_t sel = 0; sel < (1u << nsel); ++sel)
            for (uint32_t l = 0; l < T; ++l) {
                cplx d = 1;
                int e = 0;
                for (size_t ri = 0; ri < ot.runs.size(); ++ri) {
                    const Run& r = ot.runs[ri];
                    const uint32_t pl = r.perms.empty() ? l : permute(l, sel, r.perms, ot.selq);
                    for (const Factor& fc : r.fac) d *= fc.lam[bit_at(fc.q, pl, sel, ot.selq)];
                    for (const Pat& pt : pats[ri])
                        if ((pl & pt.lm) == pt.lv && (sel & pt.sm) == pt.sv) e += pt.e;
                }
                tabs[o.aux + ((size_t)sel << K) + l] = enc_tab(d * ipow[e & 3]);
            }
        return MERA_OK;
    }

    // An identity separable table op, open for later diagonal runs.
    int open_empty_table() {
        TileOp* o;
        MERA_TRY(add_op(&o));
        o->type = TOP_DSEP;
        ot = OpenTable();
        ot.open = true;
        ot.opi = (int)(o - A.ops);
        ot.runs.push_back(Run{{}, {}, {}});
        return write_table();
    }

    int add_op(TileOp** out) {
        MERA_RETURN_IF(nop >= TILE_MAX_OPS, MERA_EUNSUPPORTED, "tile pass op table full");
        *out = &A.ops[nop++];
        **out = TileOp();
        (*out)->coef = ncoef;
        return MERA_OK;
    }
    int add_coef(cplx c) { return add_coef(c, i64); }
    int add_coef(cplx c, bool q62) {
        MERA_RETURN_IF(ncoef >= TILE_MAX_COEF, MERA_EUNSUPPORTED, "tile pass coefficient table full");
        A.coef[ncoef++] = (engine == ENG_Q || engine == ENG_I64) ? enc_split(c) : enc<V>(c, q62);
        return MERA_OK;
    }
    // split Q61 limbs (int64-engine coefficients and tables), |re|, |im| <= 1
    static V enc_split(cplx d) {
        const double sc = 2305843009213693952.0;   // 2^61
        const long long r = std::llround(d.real() * sc), i = std::llround(d.imag() * sc);
        const int32_t w[4] = {(int32_t)(r >> 31), (int32_t)(r & 0x7FFFFFFF), (int32_t)(i >> 31),
                              (int32_t)(i & 0x7FFFFFFF)};
        V v;
        memcpy(&v, w, sizeof(V) < sizeof(w) ? sizeof(V) : sizeof(w));
        return v;
    }
    // complex128 separable-diagonal tables and their per-tile factors are
    // Q62 fixed point in every engine (integer multiplies)
    bool tq62() const { return sizeof(V) == 16; }
    // a table entry: the int64 engines split each Q61 part into 31-bit limbs
    V enc_tab(cplx d) const { return (engine == ENG_Q || engine == ENG_I64) ? enc_split(d) : enc<V>(d, tq62()); }

    // A run of diagonal gates (they commute): single-qubit factors become one
    // separable diagonal (or exact Z4 terms when all are unit phases), unit-
    // phase multi-qubit patterns become Z4 terms, the rest stay as they are.
    int flush_diag(const std::vector<int>& run) {
        if (run.empty()) return MERA_OK;
        cplx lam[64][2];
        bool has[64] = {false};
        std::vector<Z4Term> terms;
        std::vector<int> others;
        for (int idx : run) {
            const PrepOp& P = ops[idx];
            int q = -1;
            cplx v0, v1;
            if (P.k == 1 && P.cmask == 0) {
                q = P.t[0];
                v0 = P.v[0];
                v1 = P.v[1];
            } else if (P.k == 0 && popc(P.cmask) == 1) {
                q = __builtin_ctzll(P.cmask);
                if (P.cvals) { v0 = 1; v1 = P.v[0]; }
                else { v0 = P.v[0]; v1 = 1; }
            }
            if (q >= 0) {
                if (!has[q]) { lam[q][0] = 1; lam[q][1] = 1; has[q] = true; }
                lam[q][0] *= v0;
                lam[q][1] *= v1;
                continue;
            }
            if (P.k == 0 && phase_code_f(P.v[0]) <= 3) {
                Z4Term z{};
                z.mask = P.cmask;
                z.vals = P.cvals;
                z.e = (int)unit_exp(P.v[0]);
                terms.push_back(z);
                continue;
            }
            others.push_back(idx);
        }
        bool general = false;
        for (int q = 0; q < n; ++q)
            if (has[q] && (phase_code_f(lam[q][0]) > 3 || phase_code_f(lam[q][1]) > 3)) general = true;
        std::vector<Factor> fac;
        std::vector<int> nontile;
        for (int q = 0; q < n; ++q) {
            if (!has[q]) continue;
            fac.push_back(Factor{q, {lam[q][0], lam[q][1]}});
            if (local_of[q] < 0) nontile.push_back(q);
        }
        // unit-phase patterns whose non-tile qubits fit the selection bits
        // fold into the table as well (the table multiply happens anyway)
        auto fold_terms = [&](std::vector<int>& sel, std::vector<Z4Term>& keep) {
            std::vector<Z4Term> folded;
            for (const Z4Term& z : terms) {
                std::vector<int> s2 = sel;
                bool ok = true;
                for (int q = 0; q < n && ok; ++q) {
                    if (!((z.mask >> q) & 1ull) || local_of[q] >= 0) continue;
                    if (std::find(s2.begin(), s2.end(), q) != s2.end()) continue;
                    if ((int)s2.size() >= DSEP_SEL_BITS) ok = false;
                    else s2.push_back(q);
                }
                if (ok) {
                    sel = s2;
                    folded.push_back(z);
                } else {
                    keep.push_back(z);
                }
            }
            return folded;
        };
        std::vector<Z4Term> rest = terms;
        bool folded = false;
        if (ot.open && (!fac.empty() || !terms.empty())) {
            std::vector<int> sel = ot.selq;
            auto add_sel = [&](int q) {
                if (local_of[q] < 0 && std::find(sel.begin(), sel.end(), q) == sel.end()) sel.push_back(q);
            };
            for (int q : nontile) add_sel(q);
            for (int idx : ot.perms)
                for (int q = 0; q < n; ++q)
                    if ((ops[idx].cmask >> q) & 1ull) add_sel(q);
            if ((int)sel.size() <= DSEP_SEL_BITS) {
                std::vector<Z4Term> keep;
                std::vector<Z4Term> ft = fold_terms(sel, keep);
                ot.selq = sel;
                ot.runs.push_back(Run{fac, ot.perms, ft});
                MERA_TRY(write_table());
                rest = keep;
                folded = true;
            }
        }
        if (!folded && general) {
            TileOp* o;
            MERA_TRY(add_op(&o));
            o->type = TOP_DSEP;
            folded = true;
            if ((int)nontile.size() <= DSEP_SEL_BITS) {
                ot = OpenTable();
                ot.open = true;
                ot.opi = (int)(o - A.ops);
                ot.selq = nontile;
                std::vector<Z4Term> keep;
                std::vector<Z4Term> ft = fold_terms(ot.selq, keep);
                ot.runs.push_back(Run{fac, {}, ft});
                MERA_TRY(write_table());
                rest = keep;
            } else {
                // more non-tile qubits than selection bits: the first
                // DSEP_SEL_BITS select a table, the rest multiply per tile
                ot.open = false;
                o->aux = (int)tabs.size();
                o->aux2 = nnt;
                cplx base = 1;
                std::vector<cplx> rho;
                for (int q : nontile) {
                    base *= lam[q][0];
                    MERA_RETURN_IF(nnt >= TILE_MAX_NT, MERA_EUNSUPPORTED, "too many non-tile diagonal factors");
                    A.ntq[nnt++] = (int8_t)q;
                    rho.push_back(lam[q][1] / lam[q][0]);
                }
                const int nf = (int)rho.size();
                const int nsel = std::min(nf, DSEP_SEL_BITS);
                o->coef = ncoef;
                for (int f2 = nsel; f2 < nf; ++f2) MERA_TRY(add_coef(rho[f2], tq62()));
                o->nt = (int8_t)nf;
                const size_t T = (size_t)1 << K;
                const size_t off = tabs.size();
                tabs.resize(off + (T << nsel));
                for (size_t sel = 0; sel < ((size_t)1 << nsel); ++sel) {
                    cplx b = base;
                    for (int f2 = 0; f2 < nsel; ++f2)
                        if ((sel >> f2) & 1) b *= rho[f2];
                    for (size_t l = 0; l < T; ++l) {
                        cplx d = b;
                        for (int j = 0; j < K; ++j) {
                            const int q = A.tpos[j];
                            if (has[q]) d *= lam[q][(l >> j) & 1];
                        }
                        tabs[off + (sel << K) + l] = enc_tab(d);
                    }
                }
            }
        }
        if (!folded) {
            // unit phases only and no table to join: exact sign / i terms
            for (int q = 0; q < n; ++q) {
                if (!has[q]) continue;
                for (int b = 0; b < 2; ++b) {
                    const uint32_t e = unit_exp(lam[q][b]);
                    if (e == 0) continue;
                    Z4Term z{};
                    z.mask = 1ull << q;
                    z.vals = b ? (1ull << q) : 0ull;
                    z.e = (int)e;
                    rest.push_back(z);
                }
            }
        }
        if (!rest.empty()) {
            MERA_RETURN_IF(nz4 + (int)rest.size() > TILE_MAX_Z4, MERA_EUNSUPPORTED, "too many sign terms");
            TileOp* o;
            MERA_TRY(add_op(&o));
            o->type = TOP_Z4;
            o->aux = nz4;
            o->aux2 = (int)rest.size();
            for (const Z4Term& z : rest) A.z4[nz4++] = z;
        }
        for (int idx : others) {
            const PrepOp& P = ops[idx];
            TileOp* o;
            MERA_TRY(add_op(&o));
            o->type = TOP_DIAG;
            o->cmask = P.cmask;
            o->cvals = P.cvals;
            o->nt = (int8_t)P.k;
            for (int t = 0; t < P.k; ++t) o->tq[t] = (int8_t)P.t[t];
            for (int s2 = 0; s2 < (1 << P.k); ++s2) {
                MERA_TRY(add_coef(P.v[s2]));
                if (P.v[s2] != cplx(1, 0)) o->flags |= 1u << s2;
                o->codes |= (uint32_t)phase_code_f(P.v[s2]) << (3 * s2);
            }
        }
        return MERA_OK;
    }

    int add_gate(const PrepOp& P, const int* reg_of) {
        TileOp* o;
        MERA_TRY(add_op(&o));
        o->cmask = P.cmask;
        o->cvals = P.cvals;
        int rr[3] = {0, 0, 0};
        for (int t = 0; t < P.k; ++t) rr[t] = reg_of[local_of[P.t[t]]];
        if (P.k == 1) {
            o->a = (int8_t)rr[0];
            if (P.bslot >= 0) {
                o->type = TOP_G1;
                o->c = 1;                 // per-state coefficients
                o->coef = P.bslot * 4;
            } else if (P.is_h) {
                o->type = TOP_H;
            } else if (P.kind == KIND_MONO && P.v[0] == cplx(1, 0) && P.v[1] == cplx(1, 0)) {
                o->type = TOP_G1SWAP;
            } else if (P.kind == KIND_MONO && phase_code_f(P.v[0]) <= 3 && phase_code_f(P.v[1]) <= 3) {
                o->type = TOP_G1MONO;
                for (int s2 = 0; s2 < 2; ++s2) o->codes |= (uint32_t)phase_code_f(P.v[s2]) << (3 * s2);
            } else {
                o->type = TOP_G1;
                bool ri = true;
                for (int s2 = 0; s2 < 4; ++s2) {
                    MERA_TRY(add_coef(P.m[s2]));
                    if (P.m[s2].imag() != 0.0) {
                        if (P.m[s2].real() != 0.0) ri = false;
                        else o->flags |= 1u << s2;   // imaginary entry
                    }
                }
                if (ri) o->flags |= G1_RI;
                else o->flags = 0;
            }
            return MERA_OK;
        }
        // k = 2: register bits in descending order; conv maps the register
        // sub-index to the gate's sub-index
        const int k = P.k;
        int order[3] = {0, 1, 2};
        std::sort(order, order + k, [&](int x, int y) { return rr[x] > rr[y]; });
        o->a = (int8_t)rr[order[0]];
        o->b = (int8_t)rr[order[1]];
        auto conv = [&](int sr) {
            int sg = 0;
            for (int pos = 0; pos < k; ++pos) {
                const int bit = (sr >> (k - 1 - pos)) & 1;   // register slot pos (0 = most significant)
                sg |= bit << (k - 1 - order[pos]);
            }
            return sg;
        };
        int inv[8];
        for (int sr = 0; sr < (1 << k); ++sr) inv[conv(sr)] = sr;
        const int d = 1 << k;
        bool unit = P.kind == KIND_MONO;
        for (int s2 = 0; unit && s2 < d; ++s2) unit = phase_code_f(P.v[s2]) <= 3;
        if (unit) {
            o->type = TOP_G2MONO;
            for (int sr = 0; sr < d; ++sr) {
                const int sg = conv(sr);
                MERA_TRY(add_coef(P.v[sg]));
                o->codes |= (uint32_t)phase_code_f(P.v[sg]) << (3 * sr);
                o->perm |= (uint32_t)inv[P.perm[sg]] << (3 * sr);
            }
        } else {
            o->type = TOP_G2;
            for (int sr = 0; sr < d; ++sr)
                for (int cr = 0; cr < d; ++cr) MERA_TRY(add_coef(P.m[conv(sr) * d + conv(cr)]));
        }
        return MERA_OK;
    }

    // op kinds present in the built pass
    int features() const {
        int f = 0;
        for (int i = 0; i < nop; ++i) {
            switch (A.ops[i].type) {
            case TOP_G1: f |= FEAT_DENSE1; break;
            case TOP_G2:
            case TOP_G2MONO: f |= FEAT_G2; break;
            case TOP_DIAG:
            case TOP_DSEP: f |= FEAT_DIAG; break;
            case TOP_H:
            case TOP_G1MONO:
            case TOP_G1SWAP: f |= FEAT_GATES; break;
            default: break;
            }
        }
        return f;
    }

    int build(const Pass& p, bool allow_i64) {
        memset(&A, 0, sizeof(A));
        A.K = K;
        for (int q = 0; q < 64; ++q) local_of[q] = -1;
        int j = 0;
        for (int q = 0; q < n; ++q)
            if ((p.tile_mask >> q) & 1ull) {
                A.tpos[j] = q;
                local_of[q] = j++;
            }
        int nh = 0;
        bool all_unitary = true;
        double gain_bits = 0.0;
        for (int idx : p.ops) {
            const PrepOp& P = ops[idx];
            if (P.is_h) {
                ++nh;
                continue;
            }
            double rs;
            bool u;
            op_gain(P, &rs, &u);
            all_unitary = all_unitary && u;
            if (rs > 1.0) gain_bits += std::log2(rs);
        }
        A.nh = nh;
        bool exact = true;
        for (int idx : p.ops) exact = exact && op_is_exact(ops[idx]);
        // FP64 issues about two operations per clock per SM on GB300, so
        // complex128 passes with butterflies or any multiply run the int64
        // engine (block floating point per tile, 31-bit-limb products); a
        // pass of moves and sign flips only stays in float64, where they are
        // exact
        i64 = allow_i64 && !fp_only && (nh > 0 || !exact);
        engine = i64 ? ENG_I64 : ENG_FP;
        if (qres) {
            i64 = true;
            engine = ENG_Q;
        }
        A.scale = std::pow(0.5, nh / 2) * ((nh & 1) ? (1.0 / std::sqrt(2.0)) : 1.0);
        // fixed-point headroom: the max-norm bound (every op's row sum), or
        // for unitary passes the tile 2-norm bound 2^((nh + K) / 2)
        double g = nh + gain_bits;
        if (all_unitary) g = std::min(g, std::ceil((nh + K) / 2.0));
        A.guard = (int)std::ceil(g) + 1;
        if (A.guard > 28 && engine == ENG_I64) {   // too little fixed-point precision left: float64
            i64 = false;
            engine = ENG_FP;
        }
        // Merge diagonal runs: a diagonal gate moves past the non-diagonal
        // gates it commutes with (no shared target: a diagonal commutes with
        // gates that only use its qubits as controls), but only when that
        // brings it next to another diagonal run, first looking forward,
        // then backward.  Non-commuting pairs keep their order.
        std::vector<int> order(p.ops.begin(), p.ops.end());
        auto is_diag = [&](int pos) { return ops[order[pos]].kind == KIND_DIAG; };
        for (int i = (int)order.size() - 1; i >= 0; --i) {
            if (!is_diag(i)) continue;
            const uint64_t dq = op_qubits(ops[order[i]]);
            if (i + 1 < (int)order.size() && !is_diag(i + 1)) {
                int j = i + 1;
                while (j < (int)order.size() && !is_diag(j) && !(op_targets(ops[order[j]]) & dq)) ++j;
                if (j < (int)order.size() && is_diag(j)) {
                    const int d = order[i];
                    order.erase(order.begin() + i);
                    order.insert(order.begin() + (j - 1), d);
                    continue;
                }
            }
        }
        for (int i = 0; i < (int)order.size(); ++i) {
            if (!is_diag(i) || i == 0 || is_diag(i - 1)) continue;
            const uint64_t dq = op_qubits(ops[order[i]]);
            int j = i - 1;
            while (j >= 0 && !is_diag(j) && !(op_targets(ops[order[j]]) & dq)) --j;
            if (j >= 0 && is_diag(j)) {
                const int d = order[i];
                order.erase(order.begin() + i);
                order.insert(order.begin() + (j + 1), d);
            }
        }
        Pass q = p;
        q.ops = order;
        return build_phases(q);
    }

    // ---- permutations absorbed into exchanges --------------------------
    // X, CNOT / anti-CNOT (one target, at most one control) and two-target
    // permutations without controls that are affine on the target bits
    // (SWAP) map the local index l to an affine function of l: an exchange
    // writes amplitude l to the slot of that image instead of running a
    // register op.
    static int sigma(const PrepOp& P, int s) {   // input sub-index s -> output row
        for (int r = 0; r < (1 << P.k); ++r)
            if (P.perm[r] == s) return r;
        return s;
    }
    bool absorbable(const PrepOp& P) const {
        if (P.kind != KIND_MONO || P.bslot >= 0 || P.k < 1 || P.k > 2) return false;
        for (int s = 0; s < (1 << P.k); ++s)
            if (P.v[s] != cplx(1, 0)) return false;
        for (int j = 0; j < P.k; ++j)
            if (local_of[P.t[j]] < 0) return false;
        if (P.k == 1) return popc(P.cmask) <= 1;
        if (P.cmask != 0) return false;
        const int s0 = sigma(P, 0);
        return (sigma(P, 3) ^ s0) == ((sigma(P, 1) ^ s0) ^ (sigma(P, 2) ^ s0));
    }

    // Affine map of the local index: l -> XOR of col[b] over set bits b of l,
    // XOR c, XOR w[i].second where the tile's global bit w[i].first is set.
    struct Affine {
        uint32_t col[16];
        uint32_t c = 0;
        std::vector<std::pair<int, uint32_t>> w;
        explicit Affine(int K) {
            for (int b = 0; b < 16; ++b) col[b] = b < K ? (1u << b) : 0u;
        }
    };

    // Linear part of an absorbable op applied to a local index vector.
    uint32_t op_linear(const PrepOp& P, uint32_t u) const {
        if (P.k == 1) {
            if (P.cmask == 0) return u;
            const int lc = local_of[__builtin_ctzll(P.cmask)];
            if (lc < 0) return u;
            return u ^ (((u >> lc) & 1u) << local_of[P.t[0]]);
        }
        const int l0 = local_of[P.t[0]], l1 = local_of[P.t[1]];   // t[0]: most significant sub-index bit
        const int s = (int)((((u >> l0) & 1u) << 1) | ((u >> l1) & 1u));
        const int r = sigma(P, s) ^ sigma(P, 0);
        u &= ~((1u << l0) | (1u << l1));
        return u | ((uint32_t)((r >> 1) & 1) << l0) | ((uint32_t)(r & 1) << l1);
    }

    // f <- op o f
    void compose(Affine& f, const PrepOp& P) const {
        for (int b = 0; b < K; ++b) f.col[b] = op_linear(P, f.col[b]);
        f.c = op_linear(P, f.c);
        for (auto& t : f.w) t.second = op_linear(P, t.second);
        if (P.k == 2) {
            const int s0 = sigma(P, 0);
            if (s0 & 2) f.c ^= 1u << local_of[P.t[0]];
            if (s0 & 1) f.c ^= 1u << local_of[P.t[1]];
            return;
        }
        const uint32_t et = 1u << local_of[P.t[0]];
        if (P.cmask == 0) {
            f.c ^= et;
            return;
        }
        const int q = __builtin_ctzll(P.cmask);
        const bool cv = (P.cvals >> q) & 1ull;
        if (!cv) f.c ^= et;                       // fires when the control bit is 0: 1 ^ bit
        if (local_of[q] >= 0) return;             // in-tile control: in the linear part
        for (auto& t : f.w)
            if (t.first == q) {
                t.second ^= et;
                return;
            }
        f.w.push_back(std::make_pair(q, et));
    }

    // ---- shared-memory swizzles ---------------------------------------------
    // Z maps a local index to its slot: the default XOR-folds the higher bit
    // groups into the lowest S bits (S = log2 of amplitudes per 128-byte
    // row) so that strided register gathers hit distinct banks.  An exchange
    // whose writer permutes the index searches for another Z of the same
    // form (an invertible map of the low S bits plus a fold of each higher
    // bit into them) under which the lanes of every 128-byte wavefront of
    // both the writer and the reader still land in distinct banks.
    int Sbits() const { return sizeof(V) == 16 ? 3 : 4; }
    void default_z(uint32_t* z) const {
        const int S = Sbits();
        const uint32_t M = (1u << S) - 1u;
        for (int b = 0; b < 16; ++b) {
            const uint32_t l = 1u << b;
            const uint32_t h = l >> S;
            z[b] = b < K ? (l ^ ((h ^ (h >> S) ^ (h >> (2 * S)) ^ (h >> (3 * S)) ^ (h >> (4 * S))) & M)) : 0u;
        }
    }
    static uint32_t zapply(const uint32_t* z, uint32_t u) {
        uint32_t r = 0;
        for (int b = 0; b < 16; ++b)
            if ((u >> b) & 1u) r ^= z[b];
        return r;
    }
    // S minus the rank of the low-S-bit slot projections of S lane vectors
    // (0: conflict free; d: 2^d-way conflicts).
    // (lanes: the first min(S, K - FR) thread-index bits)
    int nlanes() const { return std::min(Sbits(), K - FR); }
    int deficiency(const uint32_t* z, const uint32_t* u) const {
        const int S = Sbits(), m = nlanes();
        uint32_t rows[8];
        for (int i = 0; i < m; ++i) rows[i] = zapply(z, u[i]) & ((1u << S) - 1u);
        return m - rank_of(rows, m, S);
    }
    static int rank_of(uint32_t* rows, int m, int S) {
        int rank = 0;
        for (int bit = S - 1; bit >= 0; --bit) {
            int piv = -1;
            for (int i = rank; i < m; ++i)
                if ((rows[i] >> bit) & 1u) {
                    piv = i;
                    break;
                }
            if (piv < 0) continue;
            std::swap(rows[rank], rows[piv]);
            for (int i = 0; i < m; ++i)
                if (i != rank && ((rows[i] >> bit) & 1u)) rows[i] ^= rows[rank];
            ++rank;
        }
        return rank;
    }
    void choose_z(uint32_t* z, const uint32_t* wl, const uint32_t* rl, uint32_t seed) const {
        default_z(z);
        int best = deficiency(z, wl) + deficiency(z, rl);
        if (best == 0) return;
        const int S = Sbits();
        uint32_t cand[16], keep[16];
        memcpy(keep, z, sizeof(keep));
        uint32_t st = 0x9E3779B9u ^ (seed * 0x85EBCA6Bu);
        auto rnd = [&]() {
            st ^= st << 13;
            st ^= st >> 17;
            st ^= st << 5;
            return st;
        };
        for (int trial = 0; trial < 4096 && best > 0; ++trial) {
            for (int b = 0; b < S; ++b) cand[b] = rnd() & ((1u << S) - 1u);
            uint32_t low[8];
            for (int b = 0; b < S; ++b) low[b] = cand[b];
            if (rank_of(low, S, S) != S) continue;   // the low block must be invertible
            for (int b = S; b < 16; ++b) cand[b] = b < K ? ((1u << b) | (rnd() & ((1u << S) - 1u))) : 0u;
            const int d = deficiency(cand, wl) + deficiency(cand, rl);
            if (d < best) {
                best = d;
                memcpy(keep, cand, sizeof(keep));
            }
        }
        memcpy(z, keep, sizeof(keep));
    }
    struct Ph {
        uint32_t need = 0;
        int begin = 0, end = 0;
        std::vector<int> exitp;   // permutation ops absorbed at the exit
    };

    int build_phases(const Pass& p) {
        const int save_nop = nop, save_ncoef = ncoef, save_nz4 = nz4, save_nnt = nnt;
        const size_t save_tabs = tabs.size();
        const OpenTable save_ot = ot;
        auto restore = [&]() {
            nop = save_nop;
            ncoef = save_ncoef;
            nz4 = save_nz4;
            nnt = save_nnt;
            tabs.resize(save_tabs);
            ot = save_ot;
            A.gather = A.scatter = 0;
        };
        // permutation runs at the ends of the pass on the load / store
        // addresses, the others on exchanges; then exchanges only; then
        // register ops (too many phases or exchange offsets)
        // (load / store address maps exist in the resident engine only)
        int r = MERA_EUNSUPPORTED;
        if (engine == ENG_Q) {
            r = build_phases_with(p, true, true);
            if (r == MERA_OK) return r;
            restore();
        }
        r = build_phases_with(p, true, false);
        if (r == MERA_OK) return r;
        restore();
        return build_phases_with(p, false, false);
    }

    int build_phases_with(const Pass& p, bool absorb, bool gs) {
        // phases: consecutive gates while their targets fit FR register
        // bits; a run of absorbable permutations ends the phase and becomes
        // its exit map (runs of one gate only at a phase start or the end);
        // with gs, a run that opens the pass is applied by the loads and
        // one that closes it by the stores
        std::vector<Ph> phs;
        std::vector<int> entryp, scatterp;
        int scatter_at = -1;
        Ph cur;
        const int nops = (int)p.ops.size();
        for (int i = 0; i < nops; ++i) {
            const PrepOp& P = ops[p.ops[i]];
            if (P.kind == KIND_DIAG) continue;
            if (absorb && absorbable(P)) {
                int j = i;
                while (j < nops && ops[p.ops[j]].kind != KIND_DIAG && absorbable(ops[p.ops[j]])) ++j;
                if (gs && i == 0) {
                    for (int m = i; m < j; ++m) entryp.push_back(p.ops[m]);
                    cur.begin = j;
                    i = j - 1;
                    continue;
                }
                // a closing region: from here on only absorbable permutations
                // and diagonal gates; the permutations are applied by the
                // stores, the diagonals must fold into the pass's table
                // through them, or be sign terms after the last of them
                // (checked when the ops are emitted)
                bool closing = gs;
                for (int m = i; closing && m < nops; ++m) {
                    const PrepOp& Q = ops[p.ops[m]];
                    closing = Q.kind == KIND_DIAG || absorbable(Q);
                }
                if (closing) {
                    for (int m = i; m < nops; ++m)
                        if (ops[p.ops[m]].kind != KIND_DIAG) scatterp.push_back(p.ops[m]);
                    scatter_at = i;
                    i = nops;
                    break;
                }
                if (j - i >= 2 || cur.need == 0 || j == nops) {
                    cur.end = i;
                    for (int m = i; m < j; ++m) cur.exitp.push_back(p.ops[m]);
                    phs.push_back(cur);
                    cur = Ph();
                    cur.begin = j;
                    i = j - 1;
                    continue;
                }
            }
            uint32_t need = 0;
            for (int t = 0; t < P.k; ++t) need |= 1u << local_of[P.t[t]];
            if (popc(cur.need | need) > FR) {
                cur.end = i;
                phs.push_back(cur);
                cur = Ph();
                cur.begin = i;
                cur.need = need;
            } else {
                cur.need |= need;
            }
        }
        cur.end = nops;
        phs.push_back(cur);
        MERA_RETURN_IF((int)phs.size() > TILE_MAX_PHASES, MERA_EUNSUPPORTED, "tile pass with %zu phases", phs.size());
        A.nph = (int)phs.size();
        for (int idx : entryp) note_gate(idx);
        std::vector<std::vector<int>> nonreg(A.nph);
        for (int ph = 0; ph < A.nph; ++ph) {
            uint32_t rbm = phs[ph].need;
            for (int b = K - 1; b >= 0 && popc(rbm) < FR; --b)
                if (!((rbm >> b) & 1u)) rbm |= 1u << b;
            int reg_of[16];
            int r = 0;
            for (int b = 0; b < K; ++b) {
                reg_of[b] = -1;
                if ((rbm >> b) & 1u) {
                    A.ph[ph].rb[r] = (int8_t)b;
                    reg_of[b] = r++;
                } else {
                    nonreg[ph].push_back(b);
                }
            }
            A.ph[ph].op_begin = (int16_t)nop;
            std::vector<int> run;
            int nop_at_scatter = -1;
            for (int i = phs[ph].begin; i < phs[ph].end; ++i) {
                const PrepOp& P = ops[p.ops[i]];
                if (scatter_at >= 0 && i >= scatter_at && P.kind != KIND_DIAG) {
                    // a permutation of the closing region: applied by the stores
                    MERA_TRY(flush_diag(run));
                    run.clear();
                    if (i == scatter_at) {
                        // diagonals with general phases after it fold,
                        // through it, into a table applied before it: open
                        // one if none is (exact sign patterns need none:
                        // they apply at the scattered index)
                        bool general = false;
                        for (int m = i + 1; m < phs[ph].end; ++m) {
                            const PrepOp& Q = ops[p.ops[m]];
                            general = general || (Q.kind == KIND_DIAG && !op_is_exact(Q));
                        }
                        if (!ot.open && general) MERA_TRY(open_empty_table());
                        nop_at_scatter = nop;
                    }
                    MERA_RETURN_IF(nop != nop_at_scatter, MERA_EUNSUPPORTED,
                                   "diagonal between closing permutations did not fold into the table");
                    note_gate(p.ops[i]);
                    continue;
                }
                if (P.kind == KIND_DIAG) {
                    run.push_back(p.ops[i]);
                    continue;
                }
                MERA_TRY(flush_diag(run));
                run.clear();
                note_gate(p.ops[i]);
                MERA_TRY(add_gate(P, reg_of));
            }
            MERA_TRY(flush_diag(run));
            // after the closing run only sign terms may remain: they apply at
            // the scattered (permuted) index
            for (int o = nop_at_scatter; nop_at_scatter >= 0 && o < nop; ++o) {
                MERA_RETURN_IF(A.ops[o].type != TOP_Z4, MERA_EUNSUPPORTED,
                               "diagonal after the closing permutation did not fold into the table");
                A.ops[o].c = 2;
            }
            A.ph[ph].op_end = (int16_t)nop;
            for (int idx : phs[ph].exitp) note_gate(idx);
        }
        // stage the first load / last store through shared memory unless the
        // lanes cover whole 128-byte rows in global memory
        const int S = Sbits();
        auto low_reg = [&](int ph) {
            for (int r = 0; r < FR; ++r)
                if (A.ph[ph].rb[r] < S) return true;
            return false;
        };
        A.load_smem = (stage_load || low_reg(0)) ? 1 : 0;
        A.store_smem = low_reg(A.nph - 1) ? 1 : 0;
        // address maps need direct (unstaged) loads / stores
        MERA_RETURN_IF(!entryp.empty() && A.load_smem, MERA_EUNSUPPORTED, "gathered load needs direct loads");
        MERA_RETURN_IF(!scatterp.empty() && A.store_smem, MERA_EUNSUPPORTED, "scattered store needs direct stores");
        if (!entryp.empty()) {
            Affine f(K);
            for (int idx : entryp) compose(f, ops[idx]);
            MERA_RETURN_IF((int)f.w.size() > TILE_MAX_XOFF, MERA_EUNSUPPORTED, "gather with %zu offsets", f.w.size());
            invert(f);
            fill_gmap(A.gin, f, nonreg[0], A.ph[0].rb);
            A.gather = 1;
        }
        if (!scatterp.empty()) {
            Affine f(K);
            for (int idx : scatterp) compose(f, ops[idx]);
            MERA_RETURN_IF((int)f.w.size() > TILE_MAX_XOFF, MERA_EUNSUPPORTED, "scatter with %zu offsets", f.w.size());
            fill_gmap(A.gout, f, nonreg[A.nph - 1], A.ph[A.nph - 1].rb);
            A.scatter = 1;
        }
        return build_maps(phs, nonreg);
    }

    // f <- f^-1 (Gauss-Jordan over GF(2) on the K x K linear part)
    void invert(Affine& f) const {
        uint32_t rows[16], inv[16];
        for (int r = 0; r < K; ++r) {
            rows[r] = 0;
            for (int b = 0; b < K; ++b)
                if ((f.col[b] >> r) & 1u) rows[r] |= 1u << b;
            inv[r] = 1u << r;
        }
        for (int c = 0; c < K; ++c) {
            int piv = c;
            while (piv < K && !((rows[piv] >> c) & 1u)) ++piv;
            std::swap(rows[c], rows[piv]);
            std::swap(inv[c], inv[piv]);
            for (int r = 0; r < K; ++r)
                if (r != c && ((rows[r] >> c) & 1u)) {
                    rows[r] ^= rows[c];
                    inv[r] ^= inv[c];
                }
        }
        Affine g(K);
        for (int b = 0; b < K; ++b) {
            g.col[b] = 0;
            for (int r = 0; r < K; ++r)
                if ((inv[r] >> b) & 1u) g.col[b] |= 1u << r;
        }
        auto apply = [&](uint32_t u) {
            uint32_t v = 0;
            for (int b = 0; b < K; ++b)
                if ((u >> b) & 1u) v ^= g.col[b];
            return v;
        };
        g.c = apply(f.c);
        for (auto& t : f.w) g.w.push_back(std::make_pair(t.first, apply(t.second)));
        f = g;
    }

    // local-bit vector -> its global positions
    unsigned long long to_global(uint32_t u) const {
        unsigned long long g = 0;
        for (int b = 0; b < K; ++b)
            if ((u >> b) & 1u) g |= 1ull << A.tpos[b];
        return g;
    }
    void fill_gmap(GMap& g, const Affine& f, const std::vector<int>& nr, const int8_t* rb) const {
        memset(&g, 0, sizeof(g));
        for (size_t t = 0; t < nr.size() && t < 12; ++t) g.tc[t] = to_global(f.col[nr[t]]);
        for (int r = 0; r < FR; ++r) g.rc[r] = to_global(f.col[rb[r]]);
        g.c = to_global(f.c);
        g.nq = (int8_t)f.w.size();
        for (size_t i = 0; i < f.w.size(); ++i) {
            g.q[i] = (int8_t)f.w[i].first;
            g.w[i] = to_global(f.w[i].second);
        }
    }

    void fill_side(XSide& x, const uint32_t* z, const std::vector<int>& nr, const int8_t* rb,
                   const Affine* f) const {
        memset(&x, 0, sizeof(x));
        auto img = [&](int b) { return zapply(z, f ? f->col[b] : (1u << b)); };
        for (size_t t = 0; t < nr.size() && t < 12; ++t) x.tc[t] = (int16_t)img(nr[t]);
        for (int r = 0; r < FR; ++r) x.rc[r] = (int16_t)img(rb[r]);
    }

    // Slot maps of every exchange: the load staging, the exchanges between
    // phases (with their absorbed permutations) and the store staging.
    int build_maps(const std::vector<Ph>& phs, const std::vector<std::vector<int>>& nonreg) {
        const int np = A.nph;
        std::vector<int> stage_bits;   // staging copy: lanes on local bits 0..K-FR-1
        for (int b = 0; b < K - FR; ++b) stage_bits.push_back(b);
        int8_t stage_rb[FR];
        for (int r = 0; r < FR; ++r) stage_rb[r] = (int8_t)(K - FR + r);
        uint32_t zin[16];
        // load staging -> phase 0
        {
            uint32_t wl[8], rl[8];
            for (int i = 0; i < nlanes(); ++i) {
                wl[i] = 1u << i;
                rl[i] = 1u << nonreg[0][i];
            }
            // natural order (identity slot map) when it costs no bank
            // conflicts and the tile is one tiled tensor copy (rows of
            // 128 bytes or more, at most 5 dimensions)
            uint32_t zid[16];
            for (int b = 0; b < 16; ++b) zid[b] = b < K ? 1u << b : 0u;
            TmaDims td;
            const bool tma = sizeof(V) == 16 && K >= 4 && tma_dims(A.tpos, K, n, td);
            if (A.load_smem && tma && bulk_enabled() && deficiency(zid, wl) == 0 && deficiency(zid, rl) == 0) {
                memcpy(zin, zid, sizeof(zin));
                A.bulk = 1;
            } else {
                choose_z(zin, wl, rl, 1u);
            }
            fill_side(A.ld, zin, stage_bits, stage_rb, nullptr);
        }
        for (int ph = 0; ph < np; ++ph) {
            TilePhase& T = A.ph[ph];
            const bool read_sm = ph > 0 || A.load_smem;
            fill_side(T.in, zin, nonreg[ph], T.rb, nullptr);
            const bool last = ph == np - 1;
            if (last && !A.store_smem) {
                T.permuted = 0;
                break;
            }
            Affine f(K);
            for (int idx : phs[ph].exitp) compose(f, ops[idx]);
            MERA_RETURN_IF((int)f.w.size() > TILE_MAX_XOFF, MERA_EUNSUPPORTED, "exchange with %zu tile-dependent offsets",
                           f.w.size());
            uint32_t zout[16], wl[8], rl[8];
            for (int i = 0; i < nlanes(); ++i) {
                wl[i] = f.col[nonreg[ph][i]];
                rl[i] = last ? (1u << i) : (1u << nonreg[ph + 1][i]);
            }
            choose_z(zout, wl, rl, 2u + (uint32_t)ph);
            fill_side(T.out.s, zout, nonreg[ph], T.rb, &f);
            T.out.off0 = (int16_t)zapply(zout, f.c);
            T.out.noff = (int8_t)f.w.size();
            for (size_t i = 0; i < f.w.size(); ++i) {
                T.out.offq[i] = (int8_t)f.w[i].first;
                T.out.offv[i] = (int16_t)zapply(zout, f.w[i].second);
            }
            const bool same = memcmp(&T.out.s, &T.in, sizeof(XSide)) == 0 && T.out.off0 == 0 && T.out.noff == 0;
            T.permuted = (!read_sm || !same) ? 1 : 0;
            if (last) fill_side(A.st, zout, stage_bits, stage_rb, nullptr);
            memcpy(zin, zout, sizeof(zin));
        }
        return MERA_OK;
    }
};

// Kernel variants: complex128 has the int64 engine and feature-trimmed
// instantiations (register pressure); complex64 has one full FP variant.
using TileFn = void (*)(PassArgs<double2>);
template <typename V>
struct TileVariant {
    const void* fn;
    int eng, feat;
};

static const void* tile_fn_c128(int eng, int feat, int qin) {
    if (eng == ENG_Q) return tile_fn_q(feat, qin);
    if (eng == ENG_I64) return tile_fn_i64(feat, 0);
    return tile_fn_fp(feat, 0);
}

// Smallest compiled variant that covers the requested features.
static int round_feat(int, int feat, bool c128) {
    if (!c128) return FEAT_ALL;
    if (feat == 0 || feat == FEAT_DIAG) return FEAT_DIAG;   // sign terms only: the leanest body
    if (feat == FEAT_GATES) return FEAT_GATES;
    if (feat == (FEAT_GATES | FEAT_DIAG)) return FEAT_GATES | FEAT_DIAG;
    return FEAT_ALL;
}

// Raise a kernel's dynamic shared-memory limit to at least `bytes` (the
// 48 KiB default covers static plus dynamic shared memory, so a kernel with
// static arrays needs the opt-in below 48 KiB of dynamic memory too).  The
// limit only ever grows: a smaller tile of the same kernel must not lower
// it under a larger one launched earlier.
static int opt_in_smem(const void* fn, size_t bytes) {
    static std::mutex mu;
    static std::vector<std::pair<const void*, size_t>> limit;
    std::lock_guard<std::mutex> lock(mu);
    auto it = std::find_if(limit.begin(), limit.end(), [&](const std::pair<const void*, size_t>& e) { return e.first == fn; });
    if (it != limit.end() && it->second >= bytes) return MERA_OK;
    MERA_CHECK_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    if (it != limit.end()) it->second = bytes;
    else limit.push_back(std::make_pair(fn, bytes));
    return MERA_OK;
}

template <typename V>
static int launch_tile(int eng, int feat, dim3 grid, unsigned block, size_t smem, cudaStream_t st,
                       const PassArgs<V>& A);
template <>
int launch_tile<double2>(int eng, int feat, dim3 grid, unsigned block, size_t smem, cudaStream_t st,
                         const PassArgs<double2>& A) {
    const void* fn = tile_fn_c128(eng, feat, eng == ENG_Q && !A.q_in ? 1 : 0);
    // opt in to the tile's dynamic shared memory (once per variant and size)
    MERA_TRY(opt_in_smem(fn, smem));
    void* args[] = {const_cast<PassArgs<double2>*>(&A)};
    MERA_CHECK_CUDA(cudaLaunchKernel(fn, grid, dim3(block), args, smem, st));
    return MERA_OK;
}
template <>
int launch_tile<float2>(int, int, dim3 grid, unsigned block, size_t smem, cudaStream_t st,
                        const PassArgs<float2>& A) {
    static size_t opted = 0;
    if (smem > 48 * 1024 && smem > opted) {
        MERA_CHECK_CUDA(cudaFuncSetAttribute(tile_fn_c64(), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        opted = smem;
    }
    void* args[] = {const_cast<PassArgs<float2>*>(&A)};
    MERA_CHECK_CUDA(cudaLaunchKernel(tile_fn_c64(), grid, dim3(block), args, smem, st));
    return MERA_OK;
}

// Build every pass of a circuit: kernel arguments (without state pointers),
// engine and kernel variant per pass, and the diagonal tables.  Passes with
// `single` >= 0 are per-gate ops (returned in `singles`, -1 otherwise).
// Arguments of the streaming kernel from a single-phase pass (K = 12):
// per thread-index bit and register bit the global index masks
// of the load, the store and the natural positions, and the local masks.
// Thread bits 0..7 are the phase's non-register bits, thread bit 8 its top
// register bit; register bits 0..2 its lower register bits.
template <typename V>
static void dpass_args(const PassArgs<V>& A, int n, DPassArgs& d) {
    memset(&d, 0, sizeof(d));
    d.K = A.K;
    const int K = A.K;
    const TilePhase& ph = A.ph[0];
    bool reg[16] = {false};
    for (int r = 0; r < FR; ++r) reg[ph.rb[r]] = true;
    int nr[16], nnr = 0;
    for (int b = 0; b < K; ++b)
        if (!reg[b]) nr[nnr++] = b;
    // tile index -> non-tile positions, as runs.  The qubits that select a
    // table slice take the most significant tile-index bits: the tiles a SM
    // runs one after another (block indices a grid-width apart) then read
    // the same 64 KiB slice, which stays in L1.
    bool tilebit[64] = {false}, selbit[64] = {false};
    for (int b = 0; b < K; ++b) tilebit[A.tpos[b]] = true;
    for (int o = ph.op_begin; o < ph.op_end; ++o)
        if (A.ops[o].type == TOP_DSEP)
            for (int f = 0; f < A.ops[o].nt; ++f) selbit[A.ntq[A.ops[o].aux2 + f]] = true;
    int order[64], norder = 0;
    for (int q = 0; q < n; ++q)
        if (!tilebit[q] && !selbit[q]) order[norder++] = q;
    for (int q = 0; q < n; ++q)
        if (!tilebit[q] && selbit[q]) order[norder++] = q;
    for (int i = 0; i < norder;) {
        int w = 1;
        while (i + w < norder && order[i + w] == order[i] + w) ++w;
        d.run_src[d.nruns] = (uint32_t)i;
        d.run_w[d.nruns] = (uint32_t)w;
        d.run_dst[d.nruns] = (uint32_t)order[i];
        ++d.nruns;
        i += w;
    }
    auto g32 = [&](int local) { return 1ull << A.tpos[local]; };
    for (int t = 0; t < 8; ++t) {
        d.nat.t[t] = g32(nr[t]);
        d.tloc[t] = 1u << nr[t];
    }
    d.nat.t[8] = g32(ph.rb[3]);
    d.tloc[8] = 1u << ph.rb[3];
    for (int r = 0; r < 3; ++r) {
        d.nat.r[r] = g32(ph.rb[r]);
        d.rloc[r] = 1u << ph.rb[r];
    }
    auto from_g = [&](const GMap& g, DMap& m) {
        for (int t = 0; t < 8; ++t) m.t[t] = g.tc[t];
        m.t[8] = g.rc[3];
        for (int r = 0; r < 3; ++r) m.r[r] = g.rc[r];
        m.c = g.c;
        m.nq = g.nq;
        for (int i = 0; i < g.nq; ++i) {
            m.q[i] = g.q[i];
            m.w[i] = g.w[i];
        }
    };
    d.in = d.nat;
    d.out = d.nat;
    if (A.gather) from_g(A.gin, d.in);
    if (A.scatter) from_g(A.gout, d.out);
    d.permuted = (A.gather || A.scatter) ? 1 : 0;
    for (int o = ph.op_begin; o < ph.op_end; ++o) {
        const TileOp& op = A.ops[o];
        if (op.type == TOP_DSEP) {
            d.tab_off[d.ntab] = op.aux;
            d.tab_nt[d.ntab] = op.nt;
            for (int f = 0; f < op.nt; ++f) d.tab_q[d.ntab][f] = A.ntq[op.aux2 + f];
            ++d.ntab;
        } else if (op.type == TOP_Z4) {
            for (int z = 0; z < op.aux2; ++z) {
                const Z4Term& t = A.z4[op.aux + z];
                d.z4[d.nz].mask = t.mask;
                d.z4[d.nz].vals = t.vals;
                d.z4[d.nz].e = t.e;
                d.z4[d.nz].post = op.c == 2 ? 1 : 0;
                ++d.nz;
            }
        }
    }
    d.shift = A.q_out ? A.qgo - A.qgi : 0;
}

// The streaming pass of an affine monomial run: the inverse index map
// F^-1 (over GF(2), Gauss-Jordan), the diagonal's tables (appended to tabs,
// split Q61 limbs) and its sign terms.
template <typename V>
static int amp_build(const std::vector<PrepOp>& ops, const std::vector<int>& run_ops, int n, std::vector<V>& tabs,
                     AmpArgs& a) {
    AmpRun r(n);
    for (int idx : run_ops) MERA_RETURN_IF(!r.take(ops, idx), MERA_EUNSUPPORTED, "op %d left its monomial run", idx);
    AmpLayout L;
    MERA_RETURN_IF(!amp_layout(r, L), MERA_EUNSUPPORTED, "monomial run's diagonal does not fit its tables");
    memset(&a, 0, sizeof(a));
    // M^-1: rows of M, augmented with the identity
    uint64_t row[64], inv[64];
    for (int i = 0; i < n; ++i) {
        row[i] = 0;
        for (int b = 0; b < n; ++b)
            if ((r.col[b] >> i) & 1ull) row[i] |= 1ull << b;
        inv[i] = 1ull << i;
    }
    for (int b = 0; b < n; ++b) {
        int piv = -1;
        for (int i = b; i < n; ++i)
            if ((row[i] >> b) & 1ull) {
                piv = i;
                break;
            }
        MERA_RETURN_IF(piv < 0, MERA_EINVAL, "monomial run's index map is not invertible");
        std::swap(row[b], row[piv]);
        std::swap(inv[b], inv[piv]);
        for (int i = 0; i < n; ++i)
            if (i != b && ((row[i] >> b) & 1ull)) {
                row[i] ^= row[b];
                inv[i] ^= inv[b];
            }
    }
    // inv[i] is row i of M^-1
    auto minv = [&](uint64_t v) {
        uint64_t y = 0;
        for (int i = 0; i < n; ++i)
            if (popc(inv[i] & v) & 1) y |= 1ull << i;
        return y;
    };
    a.in_c = minv(r.c);
    for (int t = 0; t < DPASS_TBITS; ++t) a.in_t[t] = minv(1ull << t);
    for (int q = 0; q < DPASS_RBITS; ++q) a.in_r[q] = minv(1ull << (DPASS_TBITS + q));
    for (int q = 12; q < n; ++q) {
        const uint64_t w = minv(1ull << q) ^ (1ull << q);
        if (!w) continue;
        MERA_RETURN_IF(a.in_nq >= AMP_MAX_XOFF, MERA_EUNSUPPORTED, "monomial run map too wide");
        a.in_q[a.in_nq] = (int8_t)q;
        a.in_w[a.in_nq] = w;
        ++a.in_nq;
    }
    // table A: local bits 0..11 and the selected tile bits
    int sq[AMP_A_SEL], ns = 0;
    for (int q = 12; q < n; ++q)
        if ((L.selA >> q) & 1ull) sq[ns++] = q;
    a.a_nt = ns;
    for (int f = 0; f < ns; ++f) a.a_q[f] = (int8_t)sq[f];
    auto sel_of = [&](uint64_t idx, const int* qs, int nq) {
        uint32_t v = 0;
        for (int f = 0; f < nq; ++f) v |= (uint32_t)((idx >> qs[f]) & 1ull) << f;
        return v;
    };
    auto spread = [&](uint32_t v, const int* qs, int nq) {
        uint64_t x = 0;
        for (int f = 0; f < nq; ++f)
            if ((v >> f) & 1u) x |= 1ull << qs[f];
        return x;
    };
    const bool hasT = L.tdom != 0;
    std::vector<cplx> aloc(4096), asel((size_t)1 << ns);
    for (uint32_t l = 0; l < 4096; ++l) {
        cplx d = hasT ? cplx(1, 0) : r.konst;
        for (int b = 0; b < 12; ++b) d *= r.lam[b][(l >> b) & 1];
        aloc[l] = d;
    }
    for (uint32_t v = 0; v < (1u << ns); ++v) {
        cplx d = 1;
        for (int f = 0; f < ns; ++f) d *= r.lam[sq[f]][(v >> f) & 1];
        asel[v] = d;
    }
    std::vector<int> mixed;
    for (int ti : L.inA) {
        const AmpTerm& t = r.terms[ti];
        if (!(t.mask & ~0xFFFull)) {
            for (uint32_t l = 0; l < 4096; ++l)
                if ((l & t.mask) == t.vals) aloc[l] *= t.v;
        } else if (!(t.mask & 0xFFFull)) {
            for (uint32_t v = 0; v < (1u << ns); ++v)
                if ((spread(v, sq, ns) & t.mask) == t.vals) asel[v] *= t.v;
        } else {
            mixed.push_back(ti);
        }
    }
    a.a_off = (int)tabs.size();
    tabs.resize(tabs.size() + ((size_t)4096 << ns));
    for (uint32_t v = 0; v < (1u << ns); ++v) {
        const uint64_t hi = spread(v, sq, ns);
        for (uint32_t l = 0; l < 4096; ++l) {
            cplx d = aloc[l] * asel[v];
            for (int ti : mixed) {
                const AmpTerm& t = r.terms[ti];
                if (((hi | l) & t.mask) == t.vals) d *= t.v;
            }
            tabs[a.a_off + ((size_t)v << 12) + l] = PassBuilder<V>::enc_split(d);
        }
    }
    // table T: the other tile bits with factors (one value per tile)
    a.t_off = -1;
    if (hasT) {
        int tq[AMP_T_BITS], nt = 0;
        for (int q = 12; q < n; ++q)
            if ((L.tdom >> q) & 1ull) tq[nt++] = q;
        a.t_nt = nt;
        for (int f = 0; f < nt; ++f) a.t_q[f] = (int8_t)tq[f];
        a.t_off = (int)tabs.size();
        tabs.resize(tabs.size() + ((size_t)1 << nt));
        for (uint32_t v = 0; v < (1u << nt); ++v) {
            const uint64_t x = spread(v, tq, nt);
            cplx d = r.konst;
            for (int f = 0; f < nt; ++f) d *= r.lam[tq[f]][(v >> f) & 1];
            for (int ti : L.inT) {
                const AmpTerm& t = r.terms[ti];
                if ((x & t.mask) == t.vals) d *= t.v;
            }
            tabs[a.t_off + v] = PassBuilder<V>::enc_split(d);
        }
    }
    for (int ti : L.tileZ) {
        const AmpTerm& t = r.terms[ti];
        a.tz[a.ntz].mask = t.mask;
        a.tz[a.ntz].vals = t.vals;
        a.tz[a.ntz].e = (int16_t)unit_exp(t.v);
        ++a.ntz;
    }
    for (int ti : L.elemZ) {
        const AmpTerm& t = r.terms[ti];
        const uint64_t RB = 7ull << DPASS_TBITS;   // register bits 9..11
        a.z4[a.nz].mask = t.mask & ~RB;
        a.z4[a.nz].vals = t.vals & ~RB;
        a.z4[a.nz].e = (int16_t)unit_exp(t.v);
        uint8_t J = 0;
        for (int j = 0; j < (1 << DPASS_RBITS); ++j)
            if ((((uint64_t)j << DPASS_TBITS) & t.mask) == (t.vals & RB)) J |= (uint8_t)(1u << j);
        a.z4j[a.nz] = J;
        ++a.nz;
    }
    a.ntiles = (uint32_t)(1ull << (n - 12));
    // tile groups: H = span of the tile parts of F(e_0), F(e_1), F(e_2) in
    // echelon form (distinct pivot bits); groups enumerate the other bits
    const int nt = n - 12;
    uint32_t hb[3];
    int h = 0, piv[3];
    for (int k = 0; k < 3; ++k) {
        uint32_t v = (uint32_t)(r.col[k] >> 12);
        for (int u = 0; u < h; ++u)
            if ((v >> piv[u]) & 1u) v ^= hb[u];
        if (!v) continue;
        const int p = 31 - __builtin_clz(v);
        for (int u = 0; u < h; ++u)
            if ((hb[u] >> p) & 1u) hb[u] ^= v;
        hb[h] = v;
        piv[h++] = p;
    }
    a.h = h;
    for (int u = 0; u < (1 << h); ++u) {
        uint32_t v = 0;
        for (int b = 0; b < h; ++b)
            if ((u >> b) & 1) v ^= hb[b];
        a.hv[u] = v;
        a.dgi[u] = minv((uint64_t)v << 12);
        a.dasel[u] = sel_of((uint64_t)v << 12, sq, ns);
        uint32_t ts = 0;
        for (int f = 0; f < a.t_nt; ++f) ts |= (uint32_t)(((uint64_t)v << 12 >> a.t_q[f]) & 1ull) << f;
        a.dtsel[u] = ts;
    }
    a.ngroups = (uint32_t)(1ull << (nt - h));
    int src = 0;
    for (int b = 0; b < nt;) {
        bool pv = false;
        for (int u = 0; u < h; ++u) pv = pv || piv[u] == b;
        if (pv) {
            ++b;
            continue;
        }
        int w = 1;
        auto isp = [&](int q) {
            for (int u = 0; u < h; ++u)
                if (piv[u] == q) return true;
            return false;
        };
        while (b + w < nt && !isp(b + w)) ++w;
        MERA_RETURN_IF(a.g_nruns >= 8, MERA_EUNSUPPORTED, "tile group runs");
        a.g_src[a.g_nruns] = (uint32_t)src;
        a.g_w[a.g_nruns] = (uint32_t)w;
        a.g_dst[a.g_nruns] = (uint32_t)b;
        ++a.g_nruns;
        src += w;
        b += w;
    }
    for (int idx : run_ops) (ops[idx].kind == KIND_MONO ? a.nperm : a.ndiag) += 1;
    return MERA_OK;
}

// A complex128 int64-engine pass of butterflies and sign terms only (a
// closing permutation run may ride on its stores; none on its loads): the
// Hadamard-pass kernel.
template <typename V>
static bool hpass_ok(const PassArgs<V>& A, int eng, int K) {
    if (sizeof(V) != 16 || (eng != ENG_I64 && eng != ENG_Q)) return false;
    // 256 threads for tiles of up to 2^12 amplitudes; 512 (2^13) in the per-tile engine
    if (A.gather || A.nph > HP_MAXPH || (1 << (K - FR)) > (eng == ENG_I64 ? 512 : 256)) return false;
    for (int p = 0; p < A.nph; ++p)
        for (int o = A.ph[p].op_begin; o < A.ph[p].op_end; ++o) {
            const TileOp& op = A.ops[o];
            if (!(op.type == TOP_H || (op.type == TOP_Z4 && (op.c == 0 || (op.c == 2 && A.scatter))))) return false;
        }
    return true;
}

// Per-tile int64 in the Hadamard-pass kernel (butterflies and exact sign
// terms): a rounded right shift by half the pending levels at every phase
// exit, so that the headroom above the tile maximum covers the growth
// between two exits instead of the whole pass.  Bounds of the growth in
// bits: the max norm at most doubles per unscaled level and halves per
// shifted bit; the 2-norm of the tile (at most 2^(K/2) times its maximum
// element) grows by sqrt(2) per unscaled level and halves per shifted bit,
// and bounds every element.  The headroom is the smaller bound plus one.
// cin: a level left unscaled by the previous int64 pass (the stored values
// carry a factor sqrt(2)); cout: one level to leave for the next.
template <typename V>
static void hpass_i64_scaling(PassArgs<V>& A, int cin, int cout) {
    int pending = cin, grow = 0, peak = 0, l2peak = 0;
    for (int ph = 0; ph < A.nph; ++ph) {
        int lv = 0;
        for (int o = A.ph[ph].op_begin; o < A.ph[ph].op_end; ++o) lv += A.ops[o].type == TOP_H;
        pending += lv;
        grow += lv;
        peak = std::max(peak, grow);
        // 2-norm growth in half bits: the levels applied here less the bits
        // shifted away (a carried-in level is already in the tile maximum)
        l2peak = std::max(l2peak, pending - cin);
        A.ph[ph].qsh = 0;
        if (ph + 1 < A.nph && pending >= 2) {
            const int q = pending / 2;
            A.ph[ph].qsh = (int8_t)q;
            pending -= 2 * q;
            grow -= q;
        }
    }
    A.qend = pending - cout;
    const int l2 = (l2peak + A.K + 1) / 2;
    A.guard = std::min(peak, l2) + 1;
}

template <typename V>
int fused_build(int n, const std::vector<PrepOp>& ops, FusedPlan<V>& plan, bool fp_only, bool resident_ok, int kforce,
                bool amp_ok) {
    plan.K = kforce > 0 ? kforce : fused_tile_bits(sizeof(V) == 16 ? MERA_C128 : MERA_C64, n);
    plan.n = n;
    const int L = low_bits_for(sizeof(V) == 16 ? MERA_C128 : MERA_C64, plan.K);
    const size_t tile_bytes = ((size_t)1 << plan.K) * sizeof(V);
    MERA_RETURN_IF(tile_bytes > 227 * 1024, MERA_EUNSUPPORTED, "tile of %zu bytes exceeds shared memory", tile_bytes);
    plan.tabs.clear();
    // resident fixed point: complex128, unitary gates only (the norm bounds
    // every amplitude), some arithmetic to gain from it, and every mixing
    // (non-monomial) gate before the first monomial one.  The monomial body
    // keeps each amplitude's magnitude, so a global scale costs it no
    // precision and nothing later concentrates rounding errors.  Circuits
    // with mixing gates after the body (Hadamard layers between sign flips,
    // as in Grover) keep float64 storage: with one global scale a small
    // amplitude keeps fewer bits, and a later Hadamard layer sums the
    // errors of 2^(n/2) of them into one amplitude
    plan.resident = false;
    plan.qguard = 0;
    // MERA_RESIDENT=0 keeps every complex128 state in float64 between passes
    if (const char* e = getenv("MERA_RESIDENT"))
        if (atoi(e) == 0) resident_ok = false;
    if (sizeof(V) == 16 && !fp_only && resident_ok) {
        bool unit = true, arith = false, body = false, mixed_after = false;
        for (const PrepOp& P : ops) {
            if (P.kind == KIND_IDENTITY) continue;
            double rs;
            bool u;
            op_gain(P, &rs, &u);
            unit = unit && u && P.bslot < 0;
            arith = arith || P.is_h || !op_is_exact(P);
            const bool monomial = P.kind == KIND_MONO || P.kind == KIND_DIAG;
            if (monomial) body = true;
            else if (body) mixed_after = true;
        }
        plan.resident = unit && arith && !mixed_after;
    }
    // affine monomial runs as single streaming passes: resident complex128
    // plans with 12-bit tiles, out of place (MERA_AMP=0 turns them off)
    bool amp_on = amp_ok && plan.resident && plan.K == 12 && n > 12 && n <= 40;
    if (const char* e = getenv("MERA_AMP"))
        if (atoi(e) == 0) amp_on = false;
    std::vector<Pass> passes = plan_passes(ops, n, plan.K, L, amp_on);
    plan.args.assign(passes.size(), PassArgs<V>());
    plan.eng.assign(passes.size(), 0);
    plan.feat.assign(passes.size(), 0);
    plan.single.assign(passes.size(), -1);
    plan.hpass.assign(passes.size(), 0);
    plan.amp.assign(passes.size(), 0);
    plan.aargs.assign(passes.size(), AmpArgs());
    for (size_t i = 0; i < passes.size(); ++i) {
        if (passes[i].single >= 0) {
            plan.single[i] = passes[i].single;
            continue;
        }
        if (passes[i].amp) {
            PassArgs<V>& A = plan.args[i];
            memset(&A, 0, sizeof(A));
            A.K = plan.K;
            A.nph = 1;
            A.qgi = 2;   // unit-modulus products: no growth
            for (int b = 0; b < plan.K; ++b) A.tpos[b] = b;
            plan.eng[i] = ENG_Q;
            plan.amp[i] = 1;
            MERA_TRY(amp_build<V>(ops, passes[i].ops, n, plan.tabs, plan.aargs[i]));
            plan.qguard = std::max(plan.qguard, A.qgi);
            continue;
        }
        const size_t ntab0 = plan.tabs.size();
        auto make = [&](bool stage) {
            std::unique_ptr<PassBuilder<V>> r(new PassBuilder<V>(plan.args[i], plan.tabs, ops, plan.K, n));
            r->fp_only = fp_only;
            r->qres = plan.resident;
            r->stage_load = stage;
            return r;
        };
        std::unique_ptr<PassBuilder<V>> bp = make(false);
        MERA_TRY(bp->build(passes[i], sizeof(V) == 16));
        // Hadamard / sign-term passes of the int64 engines run in the
        // pipelined kernel, which reads every tile through the load staging
        if (hpass_ok(plan.args[i], bp->engine, plan.K) && !plan.args[i].load_smem) {
            plan.tabs.resize(ntab0);
            bp = make(true);
            MERA_TRY(bp->build(passes[i], sizeof(V) == 16));
            MERA_RETURN_IF(!hpass_ok(plan.args[i], bp->engine, plan.K) || !plan.args[i].load_smem,
                           MERA_EUNSUPPORTED, "staged rebuild of a Hadamard pass changed its form");
        }
        PassBuilder<V>& b = *bp;
        plan.eng[i] = (unsigned char)b.engine;
        if (plan.eng[i] == ENG_Q) {
            // Headroom over the state norm: unnormalised butterflies grow an
            // amplitude by at most 2^(h/2) for h levels not yet scaled (the
            // scale is applied at exits once 8 levels are pending, the rest
            // at the end of the pass); two more bits of slack
            PassArgs<V>& A = plan.args[i];
            int pending = 0, most = 0;
            for (int ph = 0; ph < A.nph; ++ph) {
                for (int o = A.ph[ph].op_begin; o < A.ph[ph].op_end; ++o) pending += A.ops[o].type == TOP_H;
                most = std::max(most, pending);
                A.ph[ph].qsh = 0;
                if (ph + 1 < A.nph && pending >= 8) {
                    A.ph[ph].qsh = (int8_t)(pending / 2);
                    pending -= 2 * (pending / 2);
                }
            }
            A.qend = pending;
            A.qgi = (most + 1) / 2 + 2;
            plan.qguard = std::max(plan.qguard, A.qgi);
        }
        plan.feat[i] = (unsigned char)round_feat(plan.eng[i], b.features(), sizeof(V) == 16);
        plan.hpass[i] = hpass_ok(plan.args[i], plan.eng[i], plan.K) ? 1 : 0;
        if (!plan.hpass[i]) plan.args[i].bulk = 0;   // only the pipelined kernel stages with bulk copies
        plan.bulk = plan.bulk || plan.args[i].bulk;
    }
    // int64 passes on float64 storage scale their levels by 2^(-qend/2).  The
    // scale is linear, so a pass with an odd level count leaves one level (a
    // factor sqrt(2) on the stored state) to the next int64 pass, whatever
    // runs in between; only the circuit's last int64 pass multiplies by
    // 1/sqrt(2)
    if (!plan.resident && sizeof(V) == 16) {
        int last = -1;
        for (size_t i = 0; i < passes.size(); ++i)
            if (plan.single[i] < 0 && plan.eng[i] == ENG_I64) last = (int)i;
        int carry = 0;
        for (size_t i = 0; i < passes.size(); ++i) {
            if (plan.single[i] >= 0 || plan.eng[i] != ENG_I64) continue;
            PassArgs<V>& A = plan.args[i];
            const int tot = A.nh + carry;
            const int cout = (int)i == last ? 0 : (tot & 1);
            for (int ph = 0; ph < A.nph; ++ph) A.ph[ph].qsh = 0;
            if (plan.hpass[i]) hpass_i64_scaling(A, carry, cout);
            else A.qend = tot - cout;
            carry = cout;
        }
    }
    // A run of consecutive Hadamard passes in the per-tile int64 engine of a
    // unitary circuit keeps the state between them in the per-amplitude
    // exponent format (no conversion to doubles and back; its bias comes
    // from the norm bound, which unitary passes keep): the run's first pass
    // reads doubles, its last writes doubles
    plan.efmt = false;
    if (!plan.resident && sizeof(V) == 16 && !fp_only && resident_ok) {
        bool unit = true;
        for (const PrepOp& P : ops) {
            if (P.kind == KIND_IDENTITY) continue;
            double rs;
            bool u;
            op_gain(P, &rs, &u);
            unit = unit && u && P.bslot < 0;
        }
        auto hp = [&](size_t k) { return plan.single[k] < 0 && plan.eng[k] == ENG_I64 && plan.hpass[k]; };
        for (size_t i = 0; unit && i < passes.size(); ++i) {
            if (!hp(i)) continue;
            PassArgs<V>& A = plan.args[i];
            A.q_in = (i > 0 && hp(i - 1)) ? 1 : 0;
            A.q_out = (i + 1 < passes.size() && hp(i + 1)) ? 1 : 0;
            if (A.q_in || A.q_out) plan.efmt = true;
        }
    }
    // resident segments: runs of tile passes between per-gate ops; the first
    // reads doubles, the last writes doubles
    plan.dpass.assign(passes.size(), 0);
    plan.dargs.assign(plan.resident ? passes.size() : 0, DPassArgs());
    if (plan.resident) {
        const size_t np = passes.size();
        for (size_t i = 0; i < np; ++i) {
            if (plan.single[i] >= 0) continue;
            PassArgs<V>& A = plan.args[i];
            A.q_in = (i > 0 && plan.single[i - 1] < 0) ? 1 : 0;
            A.q_out = (i + 1 < np && plan.single[i + 1] < 0) ? 1 : 0;
            A.qgo = A.q_out ? plan.args[i + 1].qgi : A.qgi;
            if (plan.amp[i]) {
                AmpArgs& g = plan.aargs[i];
                g.qgi = A.qgi;
                g.shift = A.q_out ? A.qgo - A.qgi : 0;
                continue;
            }
            // single phase of tables and sign terms between fixed-point
            // passes: the streaming kernel
            bool ok = A.nph == 1 && A.q_in && A.q_out && A.qend == 0 && !A.load_smem && !A.store_smem && plan.K == 12;
            int ntab = 0, nz = 0;
            for (int o = A.ph[0].op_begin; ok && o < A.ph[0].op_end; ++o) {
                const TileOp& op = A.ops[o];
                if (op.type == TOP_DSEP) ok = ++ntab <= DPASS_MAX_TABS && op.nt <= DSEP_SEL_BITS;
                else if (op.type == TOP_Z4) ok = ++nz <= 1;
                else ok = false;
            }
            plan.dpass[i] = ok ? 1 : 0;
            if (ok) dpass_args(A, n, plan.dargs[i]);
        }
    }
    return MERA_OK;
}

// ------------------------------------------------- resident fixed point --
// Bound of the squared norm as (E, s): sum of squares < 2^(E - 2046) * s,
// E = twice the largest exponent field, s accumulated in float32 relative
// to 2^(E - 2046).  A normal double with exponent field e and mantissa
// bits m satisfies |x| < (1 + (top 23 bits of m + 1) / 2^23) 2^(e - 1023).
__device__ __forceinline__ float p2neg(int k) { return k > 126 ? 0.f : __int_as_float((127 - k) << 23); }
__device__ __forceinline__ void nb_merge(int& E, float& s, int E2, float s2) {
    if (E2 > E) {
        s = s * p2neg(E2 - E) + s2;
        E = E2;
    } else {
        s += s2 * p2neg(E - E2);
    }
}
__device__ __forceinline__ void nb_reduce_warp(int& E, float& s) {
    for (int off = 16; off > 0; off >>= 1) {
        const int E2 = __shfl_down_sync(0xffffffffu, E, off);
        const float s2 = __shfl_down_sync(0xffffffffu, s, off);
        nb_merge(E, s, E2, s2);
    }
}
__global__ void __launch_bounds__(256) k_normbound(const double2* psi, uint64_t N, int* pE, float* pS) {
    int E = 0;
    float s = 0.f;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (uint64_t)gridDim.x * blockDim.x) {
        const double2 v = __ldcs(psi + i);
        const long long bx = __double_as_longlong(v.x), by = __double_as_longlong(v.y);
        const int ex = (int)((bx >> 52) & 0x7FF), ey = (int)((by >> 52) & 0x7FF);
        // mantissa factor in [1, 2], rounded up
        const float fx = __int_as_float(0x3F800000 | (int)((bx >> 29) & 0x7FFFFF)) + 1.1920929e-7f;
        const float fy = __int_as_float(0x3F800000 | (int)((by >> 29) & 0x7FFFFF)) + 1.1920929e-7f;
        if (ex) nb_merge(E, s, 2 * ex, fx * fx);
        if (ey) nb_merge(E, s, 2 * ey, fy * fy);
    }
    nb_reduce_warp(E, s);
    __shared__ int sE[8];
    __shared__ float sS[8];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) {
        sE[w] = E;
        sS[w] = s;
    }
    __syncthreads();
    if (w == 0) {
        E = lane < 8 ? sE[lane] : 0;
        s = lane < 8 ? sS[lane] : 0.f;
        nb_reduce_warp(E, s);
        if (lane == 0) {
            pE[blockIdx.x] = E;
            pS[blockIdx.x] = s;
        }
    }
}
__global__ void k_qscale(const int* pE, const float* pS, int nb, int* outS) {
    int E = 0;
    float s = 0.f;
    for (int b = threadIdx.x; b < nb; b += 32) nb_merge(E, s, pE[b], pS[b]);
    nb_reduce_warp(E, s);
    if (threadIdx.x == 0) {
        int S = 59;
        if (s > 0.f) {
            // log2 of the norm bound, with room for float rounding; a pass
            // with g headroom bits then keeps |component| * 2^(S - g)
            // below 2^(60 - g)
            const double l2 = 0.5 * ((double)(E - 2046) + log2((double)s * 1.001));
            S = 59 - (int)floor(l2);
        }
        *outS = S;
    }
}

int qscale_launch(const void* psi, int n, void* scratch, cudaStream_t st) {
    const uint64_t N = 1ull << n;
    const int nb = (int)std::min<uint64_t>(1024, std::max<uint64_t>(1, N / 1024));
    char* base = reinterpret_cast<char*>(scratch);
    launch_begin(st, MERA_KCLASS_REDUCE, (double)N * 16.0);
    k_normbound<<<nb, 256, 0, st>>>(reinterpret_cast<const double2*>(psi), N, reinterpret_cast<int*>(base),
                                     reinterpret_cast<float*>(base + 4096));
    MERA_TRY(launch_end(st));
    launch_begin(st, MERA_KCLASS_REDUCE, 0.0);
    k_qscale<<<1, 32, 0, st>>>(reinterpret_cast<const int*>(base), reinterpret_cast<const float*>(base + 4096), nb,
                               reinterpret_cast<int*>(base + 8192));
    return launch_end(st);
}

// Launch pass i of a plan over `ny` states (batch rows).
template <typename V>
int fused_launch(const FusedPlan<V>& plan, size_t i, PassArgs<V>& A, unsigned ny, cudaStream_t st) {
    const int K = plan.K;
    const bool need_sm = A.nph > 1 || A.load_smem || A.store_smem;
    const size_t smem = need_sm ? ((size_t)1 << K) * sizeof(V) : 0;
    const uint64_t tiles = 1ull << (plan.n - K);
    MERA_RETURN_IF(tiles > 0x7fffffffull, MERA_EUNSUPPORTED, "too many tiles");
    MERA_RETURN_IF(ny == 0 || ny > 65535, MERA_EUNSUPPORTED, "batch of %u states per launch", ny);
    const double pass_bytes = 2.0 * (double)(1ull << plan.n) * sizeof(V) * ny;
    if (!plan.amp.empty() && plan.amp[i]) {
        MERA_RETURN_IF(sizeof(V) != 16 || ny != 1, MERA_EUNSUPPORTED, "monomial run pass on a batch");
        MERA_RETURN_IF(!A.psi_out || A.psi_out == A.psi, MERA_EUNSUPPORTED, "monomial run pass needs a second buffer");
        AmpArgs g = plan.aargs[i];
        g.psi = reinterpret_cast<const double2*>(A.psi);
        g.psi_out = reinterpret_cast<double2*>(A.psi_out);
        g.tab = reinterpret_cast<const int4*>(A.tab);
        g.qS = A.qS;
        MERA_RETURN_IF(!g.qS, MERA_EINVAL, "monomial run pass without the resident scale");
        static int sms = 0;
        if (!sms) MERA_CHECK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0));
        const uint64_t ctas = std::max<uint64_t>(1, std::min<uint64_t>(g.ngroups, 16ull * (uint64_t)sms));
        void* args[] = {&g};
        launch_begin(st, MERA_KCLASS_AMP, pass_bytes);
        // 64-bit index arithmetic above 2^32 amplitudes (MERA_AMP_IX64=1
        // forces it, to test that variant on small states)
        static int ix64 = -1;
        if (ix64 < 0) {
            const char* e = getenv("MERA_AMP_IX64");
            ix64 = (e && atoi(e) == 1) ? 1 : 0;
        }
        const int wide = (plan.n > 32 || ix64) ? 1 : 0;
        // the circuit's last pass, writing doubles, may sum the readout
        const bool rd = plan.rd_partial && !A.q_out && i + 1 == plan.args.size() && ctas <= RD_MAX_PARTIALS;
        if (rd) {
            g.rd_partial = plan.rd_partial;
            g.rd_q = plan.rd_q;
            g.rd_n = plan.n;
            plan.rd_nb = (int)ctas;
        }
        MERA_CHECK_CUDA(cudaLaunchKernel(rd ? tile_fn_amp_readout(A.q_in, wide) : tile_fn_amp(A.q_in, A.q_out, wide),
                                         dim3((unsigned)ctas, 1), dim3(512), args, 0, st));
        return launch_end(st);
    }
    if (sizeof(V) == 16 && ny == 1 && plan.dpass[i]) {
        DPassArgs d = plan.dargs[i];
        d.psi = reinterpret_cast<double2*>(A.psi);
        d.psi_out = reinterpret_cast<double2*>(A.psi_out ? A.psi_out : A.psi);
        d.tab = reinterpret_cast<const int4*>(A.tab);
        d.ntiles = (uint32_t)tiles;
        // a few tiles per CTA: the thread's address setup is shared
        static int sms = 0;
        if (!sms) MERA_CHECK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0));
        const uint64_t ctas = std::max<uint64_t>(1, std::min<uint64_t>(tiles, 16ull * (uint64_t)sms));
        void* args[] = {&d};
        launch_begin(st, MERA_KCLASS_DPASS, pass_bytes);
        MERA_CHECK_CUDA(cudaLaunchKernel(tile_fn_dpass(plan.n > 32 ? 1 : 0), dim3((unsigned)ctas, 1), dim3(2u << (K - FR)),
                                         args, 0, st));
        return launch_end(st);
    }
    if (sizeof(V) == 16 && ny == 1 && plan.hpass[i]) {
        static int sms = 0;
        if (!sms) MERA_CHECK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0));
        const bool wide = K > 12;   // 512 threads, one CTA per SM
        const unsigned ctas =
            (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(tiles, (uint64_t)(wide ? 1 : 2) * (uint64_t)sms));
        HPassArgs h;
        uint64_t tilemask = 0;
        for (int b = 0; b < K; ++b) tilemask |= 1ull << A.tpos[b];
        h.ntmask = (plan.n >= 64 ? ~0ull : ((1ull << plan.n) - 1ull)) & ~tilemask;
        h.dstride = 0;
        uint64_t g = ctas;
        for (int q = 0; q < 64 && g; ++q)
            if ((h.ntmask >> q) & 1ull) {
                if (g & 1ull) h.dstride |= 1ull << q;
                g >>= 1;
            }
        h.ntiles = (unsigned)tiles;
        h.err = plan.wait_flag;
        h.extra_tx = g_bulk_shortfall;
        memset(h.tsh, 0, sizeof(h.tsh));
        memset(h.tmk, 0, sizeof(h.tmk));
        if (A.bulk) {
            MERA_RETURN_IF(!h.err, MERA_EINVAL, "bulk-staged pass launched without a wait-status flag");
            TmaDims td;
            MERA_RETURN_IF(!tma_dims(A.tpos, K, plan.n, td), MERA_EINVAL, "bulk-staged pass without a tensor map");
            MERA_TRY(encode_tile_map(&h.tmap, A.psi, td));
            for (int d = 0; d < TMA_DIMS; ++d) {
                h.tsh[d] = td.sh[d];
                h.tmk[d] = td.mk[d];
            }
            h.tm = td.m;
            for (int j = 0; j < 2; ++j) h.tit[j] = j < td.m ? 1ull << A.tpos[K - td.m + j] : 0ull;
        }
        for (int ph = 0; ph < A.nph; ++ph)
            for (int r = 0; r < FR; ++r) h.gm[ph][r] = 1ull << A.tpos[A.ph[ph].rb[r]];
        // parity masks of the sign terms on the scattered store index
        memset(h.pz, 0, sizeof(h.pz));
        for (int ph = 0; ph < A.nph; ++ph)
            for (int o = A.ph[ph].op_begin; o < A.ph[ph].op_end; ++o) {
                const TileOp& op = A.ops[o];
                if (op.type != TOP_Z4 || op.c != 2) continue;
                for (int t = 0; t < op.aux2; ++t) {
                    uint64_t m = A.z4[op.aux + t].mask;
                    for (int k = 0; k < 2 && m; ++k) {
                        const int q = __builtin_ctzll(m);
                        m &= m - 1;
                        static const unsigned b1[4] = {0xAAAAu, 0xCCCCu, 0xF0F0u, 0xFF00u};
                        unsigned pq = 0;
                        for (int r = 0; r < FR; ++r)
                            if ((A.gout.rc[r] >> q) & 1ull) pq ^= b1[r];
                        h.pz[op.aux + t] |= pq << (16 * k);
                    }
                }
            }
        // runs of butterflies on distinct register bits (they commute: one block)
        memset(h.hrun, 0, sizeof(h.hrun));
        for (int ph = 0; ph < A.nph; ++ph)
            for (int o = A.ph[ph].op_begin; o < A.ph[ph].op_end;) {
                if (A.ops[o].type != TOP_H) {
                    ++o;
                    continue;
                }
                int m = 0, len = 0;
                while (o + len < A.ph[ph].op_end && A.ops[o + len].type == TOP_H && !((m >> A.ops[o + len].a) & 1)) {
                    m |= 1 << A.ops[o + len].a;
                    ++len;
                }
                h.hrun[o] = (unsigned char)(m | (len << 4));
                o += len;
            }
        const void* fn = tile_fn_hpass(plan.eng[i], A.q_in ? 0 : 1, A.q_out ? 1 : 0, A.qend & 1, wide ? 1 : 0);
        const size_t hsm = ((size_t)1 << K) * sizeof(V);
        MERA_TRY(opt_in_smem(fn, hsm));
        void* args[] = {reinterpret_cast<void*>(&A), &h};
        launch_begin(st, MERA_KCLASS_HPASS, pass_bytes);
        MERA_CHECK_CUDA(cudaLaunchKernel(fn, dim3(ctas), dim3(1u << (K - FR)), args, hsm, st));
        return launch_end(st);
    }
    launch_begin(st, MERA_KCLASS_TILE, pass_bytes);
    MERA_TRY(launch_tile<V>(plan.eng[i], plan.feat[i], dim3((unsigned)tiles, ny), 1u << (K - FR), smem, st, A));
    return launch_end(st);
}

template int fused_build<double2>(int, const std::vector<PrepOp>&, FusedPlan<double2>&, bool, bool, int, bool);
template int fused_build<float2>(int, const std::vector<PrepOp>&, FusedPlan<float2>&, bool, bool, int, bool);
template int fused_launch<double2>(const FusedPlan<double2>&, size_t, PassArgs<double2>&, unsigned, cudaStream_t);
template int fused_launch<float2>(const FusedPlan<float2>&, size_t, PassArgs<float2>&, unsigned, cudaStream_t);

struct FusedCache {
    std::vector<unsigned char> key;
    std::vector<PrepOp> ops;
    FusedPlan<double2> p128;
    FusedPlan<float2> p64;
};

void fused_cache_free(mera_state* s) {
    delete reinterpret_cast<FusedCache*>(s->fused_cache);
    s->fused_cache = nullptr;
}

// Upload a plan's diagonal tables into the state's program buffer (grown on
// demand) and point every pass at the state and the tables.
template <typename V>
static int upload_plan(mera_state* s, FusedPlan<V>& plan) {
    const V* dtab = nullptr;
    if (!plan.tabs.empty()) {
        const size_t bytes = plan.tabs.size() * sizeof(V);
        if (s->prog_bytes < bytes) {
            MERA_CHECK_CUDA(cudaStreamSynchronize(s->stream));   // earlier passes may read the old tables
            if (s->prog) cudaFree(s->prog);
            s->prog = nullptr;
            s->prog_bytes = 0;
            cudaError_t e = cudaMalloc(&s->prog, bytes);
            if (e != cudaSuccess) {
                set_error("cudaMalloc(%zu) for diagonal tables: %s", bytes, cudaGetErrorString(e));
                return MERA_ENOMEM;
            }
            s->prog_bytes = bytes;
        }
        // pageable source: the call returns once the host buffer was consumed
        MERA_CHECK_CUDA(cudaMemcpyAsync(s->prog, plan.tabs.data(), bytes, cudaMemcpyHostToDevice, s->stream));
        dtab = reinterpret_cast<const V*>(s->prog);
    }
    for (PassArgs<V>& A : plan.args) {
        A.psi = reinterpret_cast<V*>(s->data);
        A.tab = dtab;
    }
    return MERA_OK;
}

// The state's second buffer (allocated on first use); false once an
// allocation failed (resident runs then go in place).
static bool ensure_pong(mera_state* s) {
    if (s->pong_failed) return false;
    const size_t bytes = num_amps(s) * elem_bytes(s->dtype);
    if (s->pong_bytes >= bytes) return true;
    if (s->pong) {
        if (cudaStreamSynchronize(s->stream) != cudaSuccess) return false;
        cudaFree(s->pong);
    }
    s->pong = nullptr;
    s->pong_bytes = 0;
    if (cudaMalloc(&s->pong, bytes) == cudaSuccess) {
        s->pong_bytes = bytes;
        return true;
    }
    cudaGetLastError();
    s->pong_failed = true;
    return false;
}

// The plan of a circuit for this state: monomial run passes only when the
// second buffer they write into is there.
template <typename V>
static int build_for_state(mera_state* s, const std::vector<PrepOp>& ops, FusedPlan<V>& plan) {
    // monomial run passes only if a second state buffer exists or fits
    bool room = !s->pong_failed;
    if (room && s->pong_bytes < num_amps(s) * elem_bytes(s->dtype)) {
        size_t fr = 0, tot = 0;
        room = cudaMemGetInfo(&fr, &tot) == cudaSuccess && fr > num_amps(s) * elem_bytes(s->dtype) + (1ull << 30);
        cudaGetLastError();
    }
    MERA_TRY(fused_build<V>(s->n, ops, plan, false, true, 0, room));
    bool any = false;
    for (unsigned char a : plan.amp) any = any || a;
    if (any && !ensure_pong(s)) {
        plan = FusedPlan<V>();
        MERA_TRY(fused_build<V>(s->n, ops, plan, false, true, 0, false));
    }
    return MERA_OK;
}

template <typename V>
static int launch_plan_passes(mera_state* s, FusedPlan<V>& plan, const std::vector<PrepOp>& ops);

template <typename V>
static int launch_plan(mera_state* s, FusedPlan<V>& plan, const std::vector<PrepOp>& ops, double* rd_partial = nullptr,
                       int rd_q = 0, int* rd_nb = nullptr) {
    // a requested readout rides on the last pass where it can (plan.rd_nb > 0)
    plan.rd_partial = rd_partial;
    plan.rd_q = rd_q;
    plan.rd_nb = 0;
    const int st = launch_plan_passes<V>(s, plan, ops);
    plan.rd_partial = nullptr;
    if (rd_nb) *rd_nb = plan.rd_nb;
    return st;
}

template <typename V>
static int launch_plan_passes(mera_state* s, FusedPlan<V>& plan, const std::vector<PrepOp>& ops) {
    if (plan.resident || plan.efmt) {
        MERA_TRY(state_ensure_scratch(s, 16384));
        MERA_TRY(qscale_launch(s->data, s->n, s->scratch, s->stream));
        const int* qS = reinterpret_cast<const int*>(reinterpret_cast<char*>(s->scratch) + 8192);
        for (PassArgs<V>& A : plan.args) A.qS = qS;
    }
    if (plan.bulk) MERA_TRY(state_wait_flag(s, &plan.wait_flag));
    // resident runs alternate between the state and a second buffer (passes
    // out of place need no load-before-store ordering); the buffers are
    // assigned so that every run ends in the state
    void* other = nullptr;
    if (plan.resident && ensure_pong(s)) other = s->pong;
    const size_t np = plan.args.size();
    for (size_t i = 0; i < np;) {
        if (plan.single[i] >= 0) {
            MERA_TRY(apply_prepared(s, ops[plan.single[i]]));
            ++i;
            continue;
        }
        size_t e = i;   // the run of tile passes [i, e)
        while (e < np && plan.single[e] < 0) ++e;
        V* bufs[2] = {reinterpret_cast<V*>(s->data), reinterpret_cast<V*>(other)};
        // every pass writes the other buffer, except, in a run of odd
        // length, its first pass that may run in place (monomial run passes
        // may not); without one the run ends with a copy into the state
        size_t stay = e;
        if (other && (e - i) % 2 == 1)
            for (size_t k = i; k < e; ++k)
                if (!plan.amp[k]) {
                    stay = k;
                    break;
                }
        int cur = 0;    // buffer holding the input
        for (size_t k = i; k < e; ++k) {
            PassArgs<V>& A = plan.args[k];
            const int dst = !other ? 0 : (k == stay ? cur : cur ^ 1);
            A.psi = bufs[cur];
            A.psi_out = dst == cur ? nullptr : bufs[dst];
            MERA_TRY(fused_launch<V>(plan, k, A, 1, s->stream));
            cur = dst;
        }
        if (cur != 0)
            MERA_CHECK_CUDA(cudaMemcpyAsync(s->data, other, num_amps(s) * elem_bytes(s->dtype), cudaMemcpyDeviceToDevice,
                                            s->stream));
        i = e;
    }
    // the wait status, read by the next synchronising call
    if (plan.bulk)
        MERA_CHECK_CUDA(cudaMemcpyAsync(s->wait_host, s->wait_flag, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
    return MERA_OK;
}

template <typename V>
static int run_fused(mera_state* s, const std::vector<PrepOp>& ops) {
    fused_cache_free(s);   // the program buffer is about to hold other tables
    FusedPlan<V> plan;
    MERA_TRY(build_for_state<V>(s, ops, plan));
    MERA_TRY(upload_plan<V>(s, plan));
    return launch_plan<V>(s, plan, ops);
}

// The key of a circuit: qubit count, dtype, tile geometry and every op's
// bytes (explicit matrices by value).
static std::vector<unsigned char> circuit_key(const mera_state* s, const mera_op* ops, size_t nops) {
    std::vector<unsigned char> k;
    const int K = fused_tile_bits(s->dtype, s->n);
    const int head[4] = {s->n, s->dtype, K, low_bits_for(s->dtype, K)};
    k.insert(k.end(), (const unsigned char*)head, (const unsigned char*)(head + 4));
    for (size_t j = 0; j < nops; ++j) {
        mera_op o = ops[j];
        const double* m = o.matrix;
        o.matrix = nullptr;
        k.insert(k.end(), (const unsigned char*)&o, (const unsigned char*)(&o + 1));
        if (o.gate == MERA_GATE_MATRIX && m && o.nt >= 0 && o.nt <= 3) {
            const size_t d = (size_t)1 << o.nt;
            k.insert(k.end(), (const unsigned char*)m, (const unsigned char*)(m + 2 * d * d));
        }
    }
    return k;
}

// Scratch layout of a readout requested with a fused circuit: above the
// norm-bound partials and the resident scale (bytes 0..16 KiB).
static constexpr size_t RD_SCRATCH_OFF = 16384;

static int apply_fused_circuit_rd(mera_state* s, const mera_op* ops, size_t nops, double* rd_partial, int rd_q,
                                  int* rd_nb) {
    FusedCache* c = reinterpret_cast<FusedCache*>(s->fused_cache);
    std::vector<unsigned char> key = circuit_key(s, ops, nops);
    if (c && c->key == key) {
        if (s->dtype == MERA_C128) return launch_plan<double2>(s, c->p128, c->ops, rd_partial, rd_q, rd_nb);
        return launch_plan<float2>(s, c->p64, c->ops, rd_partial, rd_q, rd_nb);
    }
    std::vector<PrepOp> prep(nops);
    for (size_t j = 0; j < nops; ++j) {
        int st = prepare_op(ops[j], s->n, &prep[j]);
        if (st != MERA_OK) {
            std::string msg = last_error();
            set_error("op %zu: %s", j, msg.c_str());
            return st;
        }
    }
    if (s->n < FR + 1) return apply_fused(s, prep);
    fused_cache_free(s);
    c = new FusedCache();
    c->ops.swap(prep);
    int st;
    if (s->dtype == MERA_C128) {
        st = build_for_state<double2>(s, c->ops, c->p128);
        if (st == MERA_OK) st = upload_plan<double2>(s, c->p128);
    } else {
        st = fused_build<float2>(s->n, c->ops, c->p64);
        if (st == MERA_OK) st = upload_plan<float2>(s, c->p64);
    }
    if (st != MERA_OK) {
        delete c;
        return st;
    }
    c->key.swap(key);
    s->fused_cache = c;
    if (s->dtype == MERA_C128) return launch_plan<double2>(s, c->p128, c->ops, rd_partial, rd_q, rd_nb);
    return launch_plan<float2>(s, c->p64, c->ops, rd_partial, rd_q, rd_nb);
}

int apply_fused_circuit(mera_state* s, const mera_op* ops, size_t nops) {
    return apply_fused_circuit_rd(s, ops, nops, nullptr, 0, nullptr);
}

int apply_fused_circuit_observe(mera_state* s, const mera_op* ops, size_t nops, int q, double out[3]) {
    const size_t np = 3 * (size_t)std::max(RD_MAX_PARTIALS, reduce_blocks(num_amps(s)));
    MERA_TRY(state_ensure_scratch(s, RD_SCRATCH_OFF + (np + 8) * sizeof(double)));
    double* partial = reinterpret_cast<double*>(reinterpret_cast<char*>(s->scratch) + RD_SCRATCH_OFF);
    double* out_dev = partial + np;
    int nb = 0;
    MERA_TRY(apply_fused_circuit_rd(s, ops, nops, partial, q, &nb));
    if (nb > 0) MERA_TRY(observables_finish(s, partial, nb, out_dev));
    else MERA_TRY(observables_device(s, q, partial, out_dev));
    MERA_CHECK_CUDA(cudaMemcpyAsync(out, out_dev, 3 * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    MERA_CHECK_CUDA(cudaStreamSynchronize(s->stream));
    return state_check_waits(s);
}

// Host-only description of the plan (no device work).
template <typename V>
static int describe_fused(int n, int dtype, const std::vector<PrepOp>& ops, std::string* out, int* npasses) {
    FusedPlan<V> plan;
    MERA_TRY(fused_build<V>(n, ops, plan, false, true, 0, true));
    const int K = plan.K;
    char line[640];
    snprintf(line, sizeof(line), "K=%d L=%d passes=%zu resident=%d efmt=%d qguard=%d table_bytes=%zu\n", K,
             low_bits_for(dtype, K), plan.args.size(), plan.resident ? 1 : 0, plan.efmt ? 1 : 0, plan.qguard,
             plan.tabs.size() * sizeof(V));
    *out += line;
    static const char* eng_name[3] = {"fp", "i64", "q"};
    for (size_t i = 0; i < plan.args.size(); ++i) {
        if (plan.single[i] >= 0) {
            snprintf(line, sizeof(line), "pass %zu: per-gate op %d\n", i, plan.single[i]);
            *out += line;
            continue;
        }
        const PassArgs<V>& A = plan.args[i];
        if (plan.amp[i]) {
            const AmpArgs& g = plan.aargs[i];
            std::string bits;
            for (int j = 0; j < K; ++j) bits += std::to_string(A.tpos[j]) + (j + 1 < K ? "," : "");
            snprintf(line, sizeof(line),
                     "pass %zu: eng=q feat=0 nh=0 phases=1 ops=%d [g1=0 mono=%d h=0 g2=0 diag=%d dsep=0 z4=0] guard=0 "
                     "load_smem=0 store_smem=0 q_in=%d q_out=%d tile={%s} amp gather offsets=%d sel_a=%d tile_tab=%d "
                     "z4_tile=%d z4_elem=%d group=%d qend=0 qexit=0 qgi=%d phase_ops=[%d]\n",
                     i, g.nperm + g.ndiag, g.nperm, g.ndiag, A.q_in, A.q_out, bits.c_str(), g.in_nq, g.a_nt,
                     g.t_off >= 0 ? g.t_nt : 0, g.ntz, g.nz, 1 << g.h, A.qgi, g.nperm + g.ndiag);
            *out += line;
            continue;
        }
        const int nop = A.nph > 0 ? A.ph[A.nph - 1].op_end : 0;
        int cnt[16] = {0};
        for (int o = 0; o < nop; ++o) cnt[A.ops[o].type]++;
        std::string bits;
        for (int j = 0; j < K; ++j) bits += std::to_string(A.tpos[j]) + (j + 1 < K ? "," : "");
        std::string dsep;
        for (int o = 0; o < nop; ++o)
            if (A.ops[o].type == TOP_DSEP) dsep += " dsep_nontile=" + std::to_string((int)A.ops[o].nt);
        int nterms = 0;
        for (int o = 0; o < nop; ++o)
            if (A.ops[o].type == TOP_Z4) nterms += A.ops[o].aux2;
        dsep += " z4_terms=" + std::to_string(nterms) + (plan.dpass[i] ? " stream" : "") +
                (plan.hpass[i] ? " pipelined" : "") + (A.bulk ? " bulk" : "") + (A.gather ? " gather" : "") + (A.scatter ? " scatter" : "");
        if (plan.eng[i] == ENG_Q || (plan.eng[i] == ENG_I64 && plan.hpass[i])) {
            // int64 scaling: levels scaled at phase exits (2 * shift) and at the end
            int exits = 0;
            for (int ph = 0; ph < A.nph; ++ph) exits += 2 * A.ph[ph].qsh;
            dsep += " qend=" + std::to_string(A.qend) + " qexit=" + std::to_string(exits) + " qgi=" +
                    std::to_string(A.qgi);
        }
        dsep += " phase_ops=[";
        for (int ph = 0; ph < A.nph; ++ph)
            dsep += std::to_string(A.ph[ph].op_end - A.ph[ph].op_begin) + (A.ph[ph].permuted ? "p" : "") +
                    (ph + 1 < A.nph ? "," : "]");
        snprintf(line, sizeof(line),
                 "pass %zu: eng=%s feat=%d nh=%d phases=%d ops=%d [g1=%d mono=%d h=%d g2=%d diag=%d dsep=%d z4=%d] "
                 "guard=%d load_smem=%d store_smem=%d q_in=%d q_out=%d tile={%s}%s\n",
                 i, eng_name[plan.eng[i] % 3], plan.feat[i], A.nh, A.nph, nop, cnt[TOP_G1],
                 cnt[TOP_G1MONO] + cnt[TOP_G2MONO] + cnt[TOP_G1SWAP], cnt[TOP_H], cnt[TOP_G2], cnt[TOP_DIAG],
                 cnt[TOP_DSEP], cnt[TOP_Z4], A.guard, A.load_smem, A.store_smem, A.q_in, A.q_out, bits.c_str(),
                 dsep.c_str());
        *out += line;
    }
    if (npasses) *npasses = (int)plan.args.size();
    return MERA_OK;
}

int plan_summary(int n, int dtype, const std::vector<PrepOp>& ops, std::string* out, int* npasses) {
    if (dtype == MERA_C128) return describe_fused<double2>(n, dtype, ops, out, npasses);
    return describe_fused<float2>(n, dtype, ops, out, npasses);
}

int apply_fused(mera_state* s, const std::vector<PrepOp>& ops) {
    if (s->n < FR + 1) {
        // too few qubits for a tile: the per-gate kernels
        for (const PrepOp& P : ops) MERA_TRY(apply_prepared(s, P));
        return MERA_OK;
    }
    if (s->dtype == MERA_C128) return run_fused<double2>(s, ops);
    return run_fused<float2>(s, ops);
}

}  // namespace mera
