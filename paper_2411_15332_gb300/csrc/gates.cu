// Gate catalogue, gate preparation and the per-gate kernels.
//
// Per-gate application is Eq. 7 of the paper (S_next = U S) for
// U = I (x) .. (x) G (x) .. (x) I of Eq. 6, computed without U: the gate's
// 2^k x 2^k matrix is kept as its compressed index map (the DAX of Sec.
// III-A: non-zeros with their row/column), and for every group of 2^k
// amplitudes that differ only in the target bits (with the controls
// holding their values) the kernel reads the amplitudes the map names and
// writes the rows it changes.  Three classes fall out of the map:
//   diagonal  (one non-zero per row, on the diagonal: Z, S, T, RZ, CZ ...)
//   monomial  (one non-zero per row: X, Y, CNOT, SWAP, Toffoli ...)
//   dense     (H, RX, RY, U ...).
// Rows that the map leaves unchanged (value 1 on the diagonal) are neither
// read nor written, so CZ touches N/4 amplitudes and SWAP N/2.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <type_traits>

#include "common.cuh"
#include "kernels.cuh"

namespace mera {

// ------------------------------------------------------------ catalogue --
static void rot_pauli(cplx* out, int dim, const cplx* P, double theta) {
    // exp(-i theta P / 2) = cos(theta/2) I - i sin(theta/2) P, P^2 = I
    const double c = std::cos(theta / 2), s = std::sin(theta / 2);
    for (int r = 0; r < dim; ++r)
        for (int col = 0; col < dim; ++col)
            out[r * dim + col] = (r == col ? cplx(c, 0) : cplx(0, 0)) + cplx(0, -s) * P[r * dim + col];
}

static void kron2(const cplx* A, const cplx* B, cplx* out) {
    for (int ra = 0; ra < 2; ++ra)
        for (int ca = 0; ca < 2; ++ca)
            for (int rb = 0; rb < 2; ++rb)
                for (int cb = 0; cb < 2; ++cb)
                    out[(ra * 2 + rb) * 4 + ca * 2 + cb] = A[ra * 2 + ca] * B[rb * 2 + cb];
}

int gate_matrix(int gate, const double* p, int* nt, cplx* out) {
    static const cplx I2[4] = {1, 0, 0, 1};
    static const cplx PX[4] = {0, 1, 1, 0};
    static const cplx PY[4] = {0, cplx(0, -1), cplx(0, 1), 0};
    static const cplx PZ[4] = {1, 0, 0, -1};
    const double r2 = 1.0 / std::sqrt(2.0);
    auto need = [&](int k) -> int {
        if (k > 0 && p == nullptr) {
            set_error("gate %d needs %d parameter(s), params is NULL", gate, k);
            return MERA_EINVAL;
        }
        for (int j = 0; j < k; ++j)
            if (!std::isfinite(p[j])) {
                set_error("gate %d: parameter %d is not finite", gate, j);
                return MERA_EINVAL;
            }
        return MERA_OK;
    };
    auto set1 = [&](cplx a, cplx b, cplx c, cplx d) {
        *nt = 1;
        out[0] = a; out[1] = b; out[2] = c; out[3] = d;
    };
    switch (gate) {
    case MERA_GATE_I: set1(1, 0, 0, 1); return MERA_OK;
    case MERA_GATE_X: set1(0, 1, 1, 0); return MERA_OK;
    case MERA_GATE_Y: set1(0, cplx(0, -1), cplx(0, 1), 0); return MERA_OK;
    case MERA_GATE_Z: set1(1, 0, 0, -1); return MERA_OK;
    case MERA_GATE_H: set1(r2, r2, r2, -r2); return MERA_OK;
    case MERA_GATE_S: set1(1, 0, 0, cplx(0, 1)); return MERA_OK;
    case MERA_GATE_SDG: set1(1, 0, 0, cplx(0, -1)); return MERA_OK;
    case MERA_GATE_T: set1(1, 0, 0, cplx(r2, r2)); return MERA_OK;
    case MERA_GATE_TDG: set1(1, 0, 0, cplx(r2, -r2)); return MERA_OK;
    case MERA_GATE_SX: set1(cplx(0.5, 0.5), cplx(0.5, -0.5), cplx(0.5, -0.5), cplx(0.5, 0.5)); return MERA_OK;
    case MERA_GATE_SXDG: set1(cplx(0.5, -0.5), cplx(0.5, 0.5), cplx(0.5, 0.5), cplx(0.5, -0.5)); return MERA_OK;
    case MERA_GATE_P:
        MERA_TRY(need(1));
        set1(1, 0, 0, std::polar(1.0, p[0]));
        return MERA_OK;
    case MERA_GATE_RX: MERA_TRY(need(1)); *nt = 1; rot_pauli(out, 2, PX, p[0]); return MERA_OK;
    case MERA_GATE_RY: MERA_TRY(need(1)); *nt = 1; rot_pauli(out, 2, PY, p[0]); return MERA_OK;
    case MERA_GATE_RZ: MERA_TRY(need(1)); *nt = 1; rot_pauli(out, 2, PZ, p[0]); return MERA_OK;
    case MERA_GATE_R: {
        MERA_TRY(need(2));
        cplx P[4];
        for (int j = 0; j < 4; ++j) P[j] = std::cos(p[1]) * PX[j] + std::sin(p[1]) * PY[j];
        *nt = 1;
        rot_pauli(out, 2, P, p[0]);
        return MERA_OK;
    }
    case MERA_GATE_U2:
    case MERA_GATE_U: {
        double th, ph, la, ga = 0.0;
        if (gate == MERA_GATE_U2) {
            MERA_TRY(need(2));
            th = M_PI / 2; ph = p[0]; la = p[1];
        } else {
            MERA_TRY(need(4));
            th = p[0]; ph = p[1]; la = p[2]; ga = p[3];
        }
        const double c = std::cos(th / 2), s = std::sin(th / 2);
        const cplx g = std::polar(1.0, ga);
        set1(g * c, -g * std::polar(s, la), g * std::polar(s, ph), g * std::polar(c, ph + la));
        return MERA_OK;
    }
    case MERA_GATE_SWAP:
    case MERA_GATE_ISWAP: {
        *nt = 2;
        for (int j = 0; j < 16; ++j) out[j] = 0;
        const cplx off = gate == MERA_GATE_ISWAP ? cplx(0, 1) : cplx(1, 0);
        out[0] = 1; out[15] = 1; out[1 * 4 + 2] = off; out[2 * 4 + 1] = off;
        return MERA_OK;
    }
    case MERA_GATE_DCX: {
        // CNOT(t0 -> t1) then CNOT(t1 -> t0): |a b> -> |b, a xor b>
        *nt = 2;
        for (int j = 0; j < 16; ++j) out[j] = 0;
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) out[(b * 2 + (a ^ b)) * 4 + a * 2 + b] = 1;
        return MERA_OK;
    }
    case MERA_GATE_ECR: {
        // (I (x) X - X (x) Y) / sqrt(2)
        cplx a[16], b[16];
        kron2(I2, PX, a);
        kron2(PX, PY, b);
        *nt = 2;
        for (int j = 0; j < 16; ++j) out[j] = (a[j] - b[j]) * r2;
        return MERA_OK;
    }
    case MERA_GATE_RXX:
    case MERA_GATE_RYY:
    case MERA_GATE_RZZ:
    case MERA_GATE_RZX: {
        MERA_TRY(need(1));
        cplx P[16];
        if (gate == MERA_GATE_RXX) kron2(PX, PX, P);
        else if (gate == MERA_GATE_RYY) kron2(PY, PY, P);
        else if (gate == MERA_GATE_RZZ) kron2(PZ, PZ, P);
        else kron2(PZ, PX, P);
        *nt = 2;
        rot_pauli(out, 4, P, p[0]);
        return MERA_OK;
    }
    case MERA_GATE_FLIP:
        *nt = 0;
        out[0] = -1;
        return MERA_OK;
    default:
        set_error("unknown gate %d", gate);
        return MERA_EINVAL;
    }
}

// ---------------------------------------------------------- preparation --
int prepare_op(const mera_op& op, int n, PrepOp* out) {
    PrepOp& P = *out;
    P = PrepOp();
    int k = 0;
    if (op.gate == MERA_GATE_MATRIX) {
        MERA_RETURN_IF(op.nt < 1 || op.nt > 3, MERA_EUNSUPPORTED, "matrix gate needs 1..3 targets, got %d", op.nt);
        MERA_RETURN_IF(op.matrix == nullptr, MERA_EINVAL, "matrix gate without matrix");
        k = op.nt;
        const int d = 1 << k;
        for (int j = 0; j < d * d; ++j) {
            double re = op.matrix[2 * j], im = op.matrix[2 * j + 1];
            MERA_RETURN_IF(!std::isfinite(re) || !std::isfinite(im), MERA_EINVAL, "matrix entry %d not finite", j);
            P.m[j] = cplx(re, im);
        }
    } else {
        MERA_TRY(gate_matrix(op.gate, op.params, &k, P.m));
        MERA_RETURN_IF(op.nt != k, MERA_EINVAL, "gate %d takes %d target(s), got %d", op.gate, k, op.nt);
    }
    P.k = k;
    MERA_RETURN_IF(op.reserved != 0, MERA_EINVAL, "mera_op.reserved must be 0");
    MERA_RETURN_IF(n < 64 && (op.cmask >> n) != 0, MERA_EINVAL, "control mask names a qubit >= n=%d", n);
    MERA_RETURN_IF((op.cvals & ~op.cmask) != 0, MERA_EINVAL, "control values outside the control mask");
    uint64_t used = op.cmask;
    for (int j = 0; j < k; ++j) {
        const int q = op.targets[j];
        MERA_RETURN_IF(q < 0 || q >= n, MERA_EINVAL, "target %d out of range for n=%d", q, n);
        MERA_RETURN_IF((used >> q) & 1ull, MERA_EINVAL, "qubit %d used twice", q);
        used |= 1ull << q;
        P.t[j] = q;
    }
    P.cmask = op.cmask;
    P.cvals = op.cvals;
    P.is_h = (op.gate == MERA_GATE_H && op.cmask == 0);

    // the compressed index map: one non-zero per row?
    const int d = 1 << k;
    bool mono = true, diag = true;
    for (int r = 0; r < d; ++r) {
        int nz = 0, col = -1;
        for (int c = 0; c < d; ++c)
            if (P.m[r * d + c] != cplx(0, 0)) { ++nz; col = c; }
        if (nz != 1) { mono = false; diag = false; break; }
        P.perm[r] = col;
        P.v[r] = P.m[r * d + col];
        if (col != r) diag = false;
    }
    if (mono) {
        P.nact = 0;
        for (int r = 0; r < d; ++r)
            if (P.perm[r] != r || P.v[r] != cplx(1, 0)) P.act[P.nact++] = r;
        if (P.nact == 0) {
            P.kind = KIND_IDENTITY;
            return MERA_OK;
        }
        P.kind = diag ? KIND_DIAG : KIND_MONO;
        if (diag && P.nact == 1 && k > 0) {
            // a phase on one sub-index only: fold the targets into the controls
            const int r = P.act[0];
            const cplx v = P.v[r];
            for (int j = 0; j < k; ++j) {
                const uint64_t b = 1ull << P.t[j];
                P.cmask |= b;
                if ((r >> (k - 1 - j)) & 1) P.cvals |= b;
            }
            P.k = 0;
            P.m[0] = v;
            P.v[0] = v;
            P.perm[0] = 0;
            P.nact = 1;
            P.act[0] = 0;
        }
    } else {
        P.kind = KIND_DENSE;
    }
    return MERA_OK;
}

// ----------------------------------------------------------- host setup --
static int popc64(uint64_t x) { return __builtin_popcountll(x); }

// Positions of the bits to insert (targets and controls), ascending.
template <typename V>
static void fill_common(const mera_state* s, const PrepOp& P, bool include_targets, GateArgs<V>& a) {
    uint64_t mask = P.cmask;
    if (include_targets)
        for (int j = 0; j < P.k; ++j) mask |= 1ull << P.t[j];
    a.nins = 0;
    for (int q = 0; q < s->n; ++q)
        if ((mask >> q) & 1ull) a.ins[a.nins++] = q;
    a.cbits = P.cvals;
    a.count = num_amps(s) >> a.nins;
    a.k = P.k;
    for (int sidx = 0; sidx < (1 << P.k); ++sidx) {
        uint64_t o = 0;
        for (int j = 0; j < P.k; ++j)
            if ((sidx >> (P.k - 1 - j)) & 1) o |= 1ull << P.t[j];
        a.off[sidx] = o;
    }
}

template <typename V>
static V to_v(cplx c) {
    V r;
    r.x = (decltype(r.x))c.real();
    r.y = (decltype(r.y))c.imag();
    return r;
}

// Exact unit phases become moves and sign flips in the kernels.
static int phase_code(cplx v) {
    if (v == cplx(1, 0)) return 0;
    if (v == cplx(0, 1)) return 1;
    if (v == cplx(-1, 0)) return 2;
    if (v == cplx(0, -1)) return 3;
    return 4;
}

static int grid_for(uint64_t work, int threads) {
    uint64_t blocks = (work + threads - 1) / threads;
    const uint64_t cap = 152ull * 16;   // a few waves of resident blocks; grid-stride beyond
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    return (int)blocks;
}

template <typename V>
static int launch_prepared(mera_state* s, const PrepOp& P) {
    const int threads = 256;
    const double eb = (double)sizeof(V);
    GateArgs<V> a;
    memset(&a, 0, sizeof(a));
    a.psi = reinterpret_cast<V*>(s->data);
    if (P.kind == KIND_IDENTITY) return MERA_OK;
    if (P.kind == KIND_DIAG) {
        if (P.k == 0) {
            // scalar phase on one sub-space: one thread per touched amplitude
            fill_common(s, P, false, a);
            a.v[0] = to_v<V>(P.v[0]);
            a.code[0] = phase_code(P.v[0]);
            launch_begin(s->stream, MERA_KCLASS_GATE_DIAG, 2.0 * eb * (double)a.count);
            k_phase<V><<<grid_for(a.count, threads), threads, 0, s->stream>>>(a);
            return launch_end(s->stream);
        }
        // element per thread over the controlled sub-space
        fill_common(s, P, false, a);
        a.nt = P.k;
        for (int j = 0; j < P.k; ++j) a.tq[j] = P.t[j];
        for (int r = 0; r < (1 << P.k); ++r) {
            a.v[r] = to_v<V>(P.v[r]);
            a.code[r] = phase_code(P.v[r]);
            a.flag[r] = (P.v[r] != cplx(1, 0));
        }
        int nact = 0;
        for (int r = 0; r < (1 << P.k); ++r) nact += a.flag[r];
        launch_begin(s->stream, MERA_KCLASS_GATE_DIAG,
                     2.0 * eb * (double)a.count * nact / (double)(1 << P.k));
        k_diag<V><<<grid_for(a.count, threads), threads, 0, s->stream>>>(a);
        return launch_end(s->stream);
    }
    if (P.k == 1) {
        // one target: a dense 2x2, or a swap with phases (X, Y, CNOT ...)
        const bool mono = P.kind == KIND_MONO;
        for (int j = 0; j < 4; ++j) a.m[j] = to_v<V>(P.m[j]);
        a.hmode = !mono && P.m[0].imag() == 0.0 && P.m[1] == P.m[0] && P.m[2] == P.m[0] && P.m[3] == -P.m[0];
        for (int r = 0; r < 2; ++r) {
            a.v[r] = to_v<V>(P.v[r]);
            a.code[r] = phase_code(P.v[r]);
        }
        const int q = P.t[0];
        const int below = popc64(P.cmask & ((1ull << q) - 1));
        const int qc = q - below;     // target position among the non-control bits
        const uint64_t ncnt = num_amps(s) >> popc64(P.cmask);
        if (qc < 5 && ncnt >= 32) {
            fill_common(s, P, false, a);
            a.qc = qc;
            launch_begin(s->stream, MERA_KCLASS_GATE_1Q, 2.0 * eb * (double)a.count);
            if (mono) k_dense1_shfl<V, true><<<grid_for(a.count, threads), threads, 0, s->stream>>>(a);
            else k_dense1_shfl<V, false><<<grid_for(a.count, threads), threads, 0, s->stream>>>(a);
            return launch_end(s->stream);
        }
        fill_common(s, P, true, a);
        launch_begin(s->stream, MERA_KCLASS_GATE_1Q, 4.0 * eb * (double)a.count);
        if (mono) k_dense1_pair<V, true><<<grid_for(a.count, threads), threads, 0, s->stream>>>(a);
        else k_dense1_pair<V, false><<<grid_for(a.count, threads), threads, 0, s->stream>>>(a);
        return launch_end(s->stream);
    }
    // two or three targets
    fill_common(s, P, true, a);
    const int d = 1 << P.k;
    if (P.kind == KIND_MONO) {
        a.nact = P.nact;
        for (int j = 0; j < P.nact; ++j) {
            const int r = P.act[j];
            a.act[j] = r;
            a.perm[j] = P.perm[r];
            a.v[j] = to_v<V>(P.v[r]);
            a.code[j] = phase_code(P.v[r]);
        }
        launch_begin(s->stream, MERA_KCLASS_GATE, 2.0 * eb * (double)a.count * P.nact);
        k_mono<V><<<grid_for(a.count, threads), threads, 0, s->stream>>>(a);
        return launch_end(s->stream);
    }
    for (int j = 0; j < d * d; ++j) a.m[j] = to_v<V>(P.m[j]);
    launch_begin(s->stream, MERA_KCLASS_GATE, 2.0 * eb * (double)a.count * d);
    if (P.k == 2) k_dense_k<V, 2><<<grid_for(a.count, threads), threads, 0, s->stream>>>(a);
    else k_dense_k<V, 3><<<grid_for(a.count, threads), threads, 0, s->stream>>>(a);
    return launch_end(s->stream);
}

int apply_prepared(mera_state* s, const PrepOp& P) {
    if (s->dtype == MERA_C128) return launch_prepared<double2>(s, P);
    return launch_prepared<float2>(s, P);
}

}  // namespace mera
