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
#include <cstring>
#include <vector>

#include "common.cuh"
#include "tile.cuh"

namespace mera {

static int popc(uint64_t x) { return __builtin_popcountll(x); }

int fused_tile_bits(int dtype, int n) {
    int K = dtype == MERA_C128 ? 12 : 13;
    if (const char* e = getenv("MERA_TILE_BITS")) {
        const int v = atoi(e);
        if (v >= FR + 1 && v <= 14) K = v;
    }
    if (K > n) K = n;
    return K;
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
};

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
static int coef_need(const PrepOp& P) {
    if (P.kind == KIND_DIAG) return 1 << P.k;
    if (P.is_h) return 0;
    if (P.kind == KIND_MONO) return 1 << P.k;
    return 1 << (2 * P.k);
}

static std::vector<Pass> plan_passes(const std::vector<PrepOp>& ops, int n, int K, int L) {
    std::vector<int> remaining;
    for (int i = 0; i < (int)ops.size(); ++i)
        if (ops[i].kind != KIND_IDENTITY) remaining.push_back(i);
    std::vector<Pass> passes;
    const uint64_t low = (L >= 64) ? ~0ull : ((1ull << L) - 1ull);
    while (!remaining.empty()) {
        Pass p;
        p.tile_mask = low;
        uint64_t blocked = 0;
        int nops = 0, ncoef = 0;
        // register phases as build_pass will form them (same order, same rule)
        uint64_t ph_need = 0;
        int nph = 1;
        std::vector<int> deferred;
        for (int idx : remaining) {
            const PrepOp& P = ops[idx];
            const uint64_t q = op_qubits(P);
            bool take = !(q & blocked);
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
    return passes;
}

template <typename V>
static V to_v(cplx c) {
    V r;
    r.x = (decltype(r.x))c.real();
    r.y = (decltype(r.y))c.imag();
    return r;
}

static int phase_code_f(cplx v) {
    if (v == cplx(1, 0)) return 0;
    if (v == cplx(0, 1)) return 1;
    if (v == cplx(-1, 0)) return 2;
    if (v == cplx(0, -1)) return 3;
    return 4;
}

// Build the kernel arguments of one pass; returns false if the pass had to
// be cut (too many phases) -- the caller then re-plans with smaller passes.
template <typename V>
static int build_pass(const std::vector<PrepOp>& ops, const Pass& p, int K, PassArgs<V>& A, int n) {
    memset(&A, 0, sizeof(A));
    A.K = K;
    int local_of[64];
    for (int q = 0; q < 64; ++q) local_of[q] = -1;
    int j = 0;
    for (int q = 0; q < n; ++q)
        if ((p.tile_mask >> q) & 1ull) {
            A.tpos[j] = q;
            local_of[q] = j++;
        }
    // phases
    struct Ph {
        uint32_t need = 0;
        int begin = 0, end = 0;
    };
    std::vector<Ph> phs;
    Ph cur;
    cur.begin = 0;
    int nh = 0;
    for (int i = 0; i < (int)p.ops.size(); ++i) {
        const PrepOp& P = ops[p.ops[i]];
        if (P.is_h) ++nh;
        if (P.kind != KIND_DIAG) {
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
    }
    cur.end = (int)p.ops.size();
    phs.push_back(cur);
    MERA_RETURN_IF((int)phs.size() > TILE_MAX_PHASES, MERA_EUNSUPPORTED, "tile pass with %zu phases", phs.size());
    A.nph = (int)phs.size();
    A.scale = std::pow(0.5, nh / 2) * ((nh & 1) ? (1.0 / std::sqrt(2.0)) : 1.0);
    int ncoef = 0, nop = 0;
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
            }
        }
        A.ph[ph].op_begin = (int16_t)nop;
        for (int i = phs[ph].begin; i < phs[ph].end; ++i) {
            const PrepOp& P = ops[p.ops[i]];
            TileOp& o = A.ops[nop++];
            o.cmask = P.cmask;
            o.cvals = P.cvals;
            o.coef = ncoef;
            if (P.kind == KIND_DIAG) {
                o.type = TOP_DIAG;
                o.nt = (int8_t)P.k;
                for (int t = 0; t < P.k; ++t) o.tq[t] = (int8_t)P.t[t];
                for (int s = 0; s < (1 << P.k); ++s) {
                    A.coef[ncoef++] = to_v<V>(P.v[s]);
                    if (P.v[s] != cplx(1, 0)) o.flags |= 1u << s;
                    o.codes |= (uint32_t)phase_code_f(P.v[s]) << (3 * s);
                }
                continue;
            }
            int rr[3];
            for (int t = 0; t < P.k; ++t) rr[t] = reg_of[local_of[P.t[t]]];
            if (P.k == 1) {
                o.a = (int8_t)rr[0];
                if (P.is_h) {
                    o.type = TOP_H;
                } else if (P.kind == KIND_MONO) {
                    o.type = TOP_G1MONO;
                    for (int s = 0; s < 2; ++s) {
                        A.coef[ncoef++] = to_v<V>(P.v[s]);
                        o.codes |= (uint32_t)phase_code_f(P.v[s]) << (3 * s);
                    }
                } else {
                    o.type = TOP_G1;
                    for (int s = 0; s < 4; ++s) A.coef[ncoef++] = to_v<V>(P.m[s]);
                }
                continue;
            }
            // k = 2, 3: order the register bits descending; conv maps the
            // register sub-index to the gate's sub-index
            const int k = P.k;
            int order[3] = {0, 1, 2};
            std::sort(order, order + k, [&](int x, int y) { return rr[x] > rr[y]; });
            o.a = (int8_t)rr[order[0]];
            o.b = (int8_t)rr[order[1]];
            if (k == 3) o.c = (int8_t)rr[order[2]];
            auto conv = [&](int sr) {
                int sg = 0;
                for (int pos = 0; pos < k; ++pos) {
                    const int bit = (sr >> (k - 1 - pos)) & 1;   // register slot pos (0 = most significant)
                    const int t = order[pos];                     // gate target in that slot
                    sg |= bit << (k - 1 - t);
                }
                return sg;
            };
            int inv[8];
            for (int sr = 0; sr < (1 << k); ++sr) inv[conv(sr)] = sr;
            const int d = 1 << k;
            if (P.kind == KIND_MONO) {
                o.type = k == 2 ? TOP_G2MONO : TOP_G3MONO;
                for (int sr = 0; sr < d; ++sr) {
                    const int sg = conv(sr);
                    A.coef[ncoef++] = to_v<V>(P.v[sg]);
                    o.codes |= (uint32_t)phase_code_f(P.v[sg]) << (3 * sr);
                    o.perm |= (uint32_t)inv[P.perm[sg]] << (3 * sr);
                }
            } else {
                o.type = k == 2 ? TOP_G2 : TOP_G3;
                for (int sr = 0; sr < d; ++sr)
                    for (int cr = 0; cr < d; ++cr) A.coef[ncoef++] = to_v<V>(P.m[conv(sr) * d + conv(cr)]);
            }
        }
        A.ph[ph].op_end = (int16_t)nop;
    }
    // stage the first load / last store through shared memory unless the
    // lanes cover whole 128-byte rows in global memory
    const int S = sizeof(V) == 16 ? 3 : 4;
    auto low_reg = [&](int ph) {
        for (int r = 0; r < FR; ++r)
            if (A.ph[ph].rb[r] < S) return true;
        return false;
    };
    A.load_smem = low_reg(0) ? 1 : 0;
    A.store_smem = low_reg(A.nph - 1) ? 1 : 0;
    return MERA_OK;
}

template <typename V>
static int run_fused(mera_state* s, const std::vector<PrepOp>& ops) {
    const int n = s->n;
    const int K = fused_tile_bits(s->dtype, n);
    const int L = low_bits_for(s->dtype, K);
    std::vector<Pass> passes = plan_passes(ops, n, K, L);
    // opt in to the dynamic shared memory of a full tile (2^K elements)
    const size_t tile_bytes = ((size_t)1 << K) * sizeof(V);
    MERA_RETURN_IF(tile_bytes > 227 * 1024, MERA_EUNSUPPORTED, "tile of %zu bytes exceeds shared memory", tile_bytes);
    static int attr_set[2] = {0, 0};
    const int slot = sizeof(V) == 16 ? 1 : 0;
    if (attr_set[slot] < (int)tile_bytes) {
        MERA_CHECK_CUDA(cudaFuncSetAttribute(k_tile<V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tile_bytes));
        attr_set[slot] = (int)tile_bytes;
    }
    std::vector<unsigned char> buf(sizeof(PassArgs<V>));
    PassArgs<V>& A = *reinterpret_cast<PassArgs<V>*>(buf.data());
    for (const Pass& p : passes) {
        MERA_TRY(build_pass<V>(ops, p, K, A, n));
        A.psi = reinterpret_cast<V*>(s->data);
        const bool need_sm = A.nph > 1 || A.load_smem || A.store_smem;
        const size_t smem = need_sm ? ((size_t)1 << K) * sizeof(V) : 0;
        const uint64_t tiles = 1ull << (n - K);
        MERA_RETURN_IF(tiles > 0x7fffffffull, MERA_EUNSUPPORTED, "too many tiles");
        launch_begin(s->stream, MERA_KCLASS_TILE, 2.0 * (double)num_amps(s) * sizeof(V));
        k_tile<V><<<(unsigned)tiles, 1u << (K - FR), smem, s->stream>>>(A);
        MERA_TRY(launch_end(s->stream));
    }
    return MERA_OK;
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
