// qf_gates.cu -- gate entries (FP64, host) and the pass planner.
//
// Gate entries follow Appendix B of the paper:
//   Fourier            H_ab = w^(a b) / sqrt(d),  w = exp(2 pi i / d)
//   generalised NOT    X_s |x> = |x + s mod d>
//   phase-shift        P = diag(w^l), applied to a power p
//   rotations          R = exp(-i theta S / 2) with S a generalised Gell-Mann
//                      matrix: on levels (j, k)
//                        x: [[c, -i s], [-i s, c]]   y: [[c, -s], [s, c]]
//                      c = cos(theta/2), s = sin(theta/2); the level-pair
//                      diagonal 'z' phases j by exp(-i theta/2), k by
//                      exp(+i theta/2); the Gell-Mann diagonal 'g' (index j)
//                      phases level l by exp(-i theta v_l / 2), v_l =
//                      sqrt(2/(j(j+1))) for l < j, -j sqrt(2/(j(j+1))) for l = j
//   controlled rot.    sum_m |m><m|_c (x) R(m theta)_t
//   generalised CNOT   |c>|t> -> |c>|t + c mod d>
//   SWAP               |x>|y> -> |y>|x>
#include <algorithm>
#include <cmath>
#include <cstring>

#include "qf_host.h"

namespace qf {

long long ipow_ll(int d, int e) {
    long long r = 1;
    for (int i = 0; i < e; ++i) r *= d;
    return r;
}

static cd omega_pow(int d, long long m) {
    long long r = m % d;
    if (r < 0) r += d;
    double a = 2.0 * M_PI * (double)r / (double)d;
    return cd(std::cos(a), std::sin(a));
}

// Multi-controlled gates: 1..5 controls then the target; dq[i] = dimension
// of g.q[i].
static qf_status check_mc(const HGate &g, const int *dq) {
    auto bad = [&](const std::string &m) { return set_error(QF_ERR_ARG, m); };
    if (g.nq < 2 || g.nq > 6) return bad("multi-controlled gate needs 1..5 controls and a target");
    const int dt = dq[g.nq - 1];
    if (g.kind == G_MCU) {
        for (int i = 0; i + 1 < g.nq; ++i)
            if (g.lv[i] < 0 || g.lv[i] >= dq[i]) return bad("control level out of range [0, d_c)");
        if ((int)g.U.size() != dt * dt) return bad("controlled matrix must be d_t x d_t");
    }
    return QF_OK;
}

qf_status check_gate(const HGate &g, int d, int n) {
    auto bad = [&](const std::string &m) { return set_error(QF_ERR_ARG, m); };
    if (g.nq < 1 || g.nq > 6) return bad("gate needs 1..6 qudits");
    for (int i = 0; i < g.nq; ++i) {
        if (g.q[i] < 0 || g.q[i] >= n) return bad("qudit index out of range [0, n)");
        for (int k = 0; k < i; ++k)
            if (g.q[k] == g.q[i]) return bad("qudits of a gate must be distinct");
    }
    switch (g.kind) {
    case G_DENSE: {
        long long K = ipow_ll(d, g.nq);
        if (K > kMaxDenseK) return set_error(QF_ERR_UNSUPPORTED, "custom gate: d^k must be <= 64");
        if ((long long)g.U.size() != K * K) return bad("custom gate matrix has the wrong size");
        return QF_OK;
    }
    case G_ROT:
    case G_CROT:
        if ((g.kind == G_ROT) != (g.nq == 1)) return bad("rotation arity");
        if (g.axis == 'g') {
            if (g.j < 1 || g.j > d - 1) return bad("Gell-Mann diagonal index j must be in [1, d-1]");
        } else if (g.axis == 'x' || g.axis == 'y' || g.axis == 'z') {
            if (!(0 <= g.j && g.j < g.k && g.k < d)) return bad("levels must satisfy 0 <= j < k < d");
        } else {
            return bad("axis must be 'x', 'y', 'z' or 'g'");
        }
        if (!std::isfinite(g.theta)) return bad("angle is not finite");
        return QF_OK;
    case G_SUM:
    case G_SWAP:
        if (g.nq != 2) return bad("two-qudit gate needs two distinct qudits");
        return QF_OK;
    case G_X:
    case G_Z:
    case G_H:
        if (g.nq != 1) return bad("single-qudit gate arity");
        return QF_OK;
    case G_MCX:
    case G_MCU: {
        int dims[6];
        for (int i = 0; i < 6; ++i) dims[i] = d;
        return check_mc(g, dims);
    }
    default:
        return bad("unknown gate kind");
    }
}

qf_status check_gate_dims(const HGate &g, const int *dims, int n) {
    auto bad = [&](const std::string &m) { return set_error(QF_ERR_ARG, m); };
    if (g.nq < 1 || g.nq > 6) return bad("gate needs 1..6 qudits");
    for (int i = 0; i < g.nq; ++i)
        if (g.q[i] < 0 || g.q[i] >= n) return bad("qudit index out of range [0, n)");
    if (g.kind == G_DENSE) {
        long long K = 1;
        for (int i = 0; i < g.nq; ++i) K *= dims[g.q[i]];
        if (K > kMaxDenseK) return set_error(QF_ERR_UNSUPPORTED, "custom gate: the product of the targets' dims must be <= 64");
        for (int i = 0; i < g.nq; ++i)
            for (int k = 0; k < i; ++k)
                if (g.q[k] == g.q[i]) return bad("qudits of a gate must be distinct");
        if ((long long)g.U.size() != K * K) return bad("custom gate matrix has the wrong size");
        return QF_OK;
    }
    if (g.kind == G_SWAP && g.nq == 2 && dims[g.q[0]] != dims[g.q[1]])
        return bad("SWAP needs two qudits of the same dimension");
    if (is_mc_gate(g)) {
        for (int i = 0; i < g.nq; ++i)
            for (int k = 0; k < i; ++k)
                if (g.q[k] == g.q[i]) return bad("qudits of a gate must be distinct");
        int dq[6];
        for (int i = 0; i < g.nq; ++i) dq[i] = dims[g.q[i]];
        return check_mc(g, dq);
    }
    // everything else is bounded by the target's dimension
    return check_gate(g, dims[gate_target(g)], n);
}

bool gate_is_param(const HGate &g) { return (g.kind == G_ROT || g.kind == G_CROT) && g.slot >= 0; }

double gate_angle(const HGate &g, const double *params) {
    if (g.slot >= 0 && params) return params[g.slot];
    return g.theta;
}

// Rotation entries: PAIR layout (jj, jk, kj, kk) for x/y, diagonal (d) for z/g.
static void rot_entries(int d, int j, int k, char axis, double th, cd *out, int *mask) {
    const double c = std::cos(0.5 * th), s = std::sin(0.5 * th);
    if (axis == 'x') {
        out[0] = cd(c, 0); out[1] = cd(0, -s); out[2] = cd(0, -s); out[3] = cd(c, 0);
        *mask = 0;
        return;
    }
    if (axis == 'y') {
        out[0] = cd(c, 0); out[1] = cd(-s, 0); out[2] = cd(s, 0); out[3] = cd(c, 0);
        *mask = 0;
        return;
    }
    for (int l = 0; l < d; ++l) out[l] = cd(1, 0);
    if (axis == 'z') {
        out[j] = cd(c, -s);
        out[k] = cd(c, s);
        *mask = (1 << j) | (1 << k);
        return;
    }
    // 'g': Gell-Mann diagonal S_z^j
    const double gam = std::sqrt(2.0 / ((double)j * (double)(j + 1)));
    int msk = 0;
    for (int l = 0; l <= j; ++l) {
        const double v = (l < j) ? gam : -(double)j * gam;
        const double a = -0.5 * th * v;
        out[l] = cd(std::cos(a), std::sin(a));
        msk |= 1 << l;
    }
    *mask = msk;
}

// d: the target's dimension; dc: the control's (controlled rotations).
static ROp resolve_impl(const HGate &g, int d, int dc, double th) {
    ROp r;
    std::memset(&r.op, 0, sizeof(TOp));
    TOp &o = r.op;
    o.a = g.q[0];
    switch (g.kind) {
    case G_H:
        o.kind = OP_DENSE;
        r.m.resize((size_t)d * d);
        for (int a = 0; a < d; ++a)
            for (int b = 0; b < d; ++b) r.m[a * d + b] = omega_pow(d, (long long)a * b) / std::sqrt((double)d);
        break;
    case G_X: {
        o.kind = OP_SHIFT;
        int s = g.power % d;
        if (s < 0) s += d;
        o.s = s;
        break;
    }
    case G_Z: {
        o.kind = OP_DIAG;
        r.m.resize(d);
        int msk = 0;
        for (int l = 0; l < d; ++l) {
            long long e = ((long long)g.power * l) % d;
            if (e < 0) e += d;
            r.m[l] = omega_pow(d, e);
            if (e != 0) msk |= 1 << l;
        }
        o.mask = msk;
        break;
    }
    case G_ROT: {
        o.j = g.j;
        o.k = g.k;
        if (g.axis == 'x' || g.axis == 'y') {
            o.kind = OP_PAIR;
            o.s = g.axis == 'y' ? 1 : 0;   // 1: real 2x2 block
            r.m.resize(4);
        } else {
            o.kind = OP_DIAG;
            r.m.resize(d);
        }
        rot_entries(d, g.j, g.k, g.axis, th, r.m.data(), &o.mask);
        break;
    }
    case G_CROT: {
        o.c = g.q[0];
        o.a = g.q[1];
        o.j = g.j;
        o.k = g.k;
        const bool pair = g.axis == 'x' || g.axis == 'y';
        o.kind = pair ? OP_CPAIR : OP_CDIAG;
        o.s = g.axis == 'y' ? 1 : 0;       // 1: real 2x2 blocks
        const int per = pair ? 4 : d;
        r.m.resize((size_t)per * dc);
        for (int m = 0; m < dc; ++m) rot_entries(d, g.j, g.k, g.axis, m * th, r.m.data() + per * m, &o.mask);
        break;
    }
    case G_SUM:
        o.kind = OP_CSHIFT;
        o.c = g.q[0];
        o.a = g.q[1];
        o.s = 1;
        break;
    case G_SWAP:
        o.kind = OP_SWAP;
        o.a = g.q[0];
        o.c = g.q[1];
        break;
    case G_MCX:
    case G_MCU: {
        o.a = g.q[g.nq - 1];
        o.nq = g.nq - 1;
        for (int i = 0; i < o.nq; ++i) o.q[i] = g.q[i];
        if (g.kind == G_MCX) {
            o.kind = OP_MCSHIFT;
            int sh = g.power % d;
            if (sh < 0) sh += d;
            o.s = sh;
        } else {
            o.kind = OP_MCDENSE;
            int msk = 0;
            for (int i = 0; i < o.nq; ++i) msk |= g.lv[i] << (4 * i);
            o.mask = msk;
            r.m = g.U;
        }
        break;
    }
    case G_DENSE:
        if (g.nq == 1) {
            o.kind = OP_DENSE;
        } else {
            o.kind = OP_DENSEK;
            o.nq = g.nq;
            for (int i = 0; i < g.nq; ++i) o.q[i] = g.q[i];
        }
        r.m = g.U;
        break;
    }
    return r;
}

ROp resolve_gate(const HGate &g, int d, double th) { return resolve_impl(g, d, d, th); }

ROp resolve_gate_dims(const HGate &g, const int *dims, double th) {
    const int t = gate_target(g);
    const int dc = (g.kind == G_CROT || g.kind == G_SUM) ? dims[g.q[0]] : dims[t];
    return resolve_impl(g, dims[t], dc, th);
}

std::vector<cd> dense_of(const ROp &r, int d) {
    std::vector<cd> M((size_t)d * d, cd(0, 0));
    const TOp &o = r.op;
    switch (o.kind) {
    case OP_DENSE:
        M = r.m;
        break;
    case OP_PAIR:
        for (int l = 0; l < d; ++l) M[l * d + l] = 1;
        M[o.j * d + o.j] = r.m[0];
        M[o.j * d + o.k] = r.m[1];
        M[o.k * d + o.j] = r.m[2];
        M[o.k * d + o.k] = r.m[3];
        break;
    case OP_DIAG:
        for (int l = 0; l < d; ++l) M[l * d + l] = ((o.mask >> l) & 1) ? r.m[l] : cd(1, 0);
        break;
    case OP_SHIFT:
        for (int x = 0; x < d; ++x) M[((x + o.s) % d) * d + x] = 1;
        break;
    }
    return M;
}

// U^+ of a resolved op, in the same op layout.
ROp dagger(const ROp &r, int d) {
    ROp o = r;
    auto cj = [](const cd &z) { return std::conj(z); };
    switch (r.op.kind) {
    case OP_DENSE:
        for (int a = 0; a < d; ++a)
            for (int b = 0; b < d; ++b) o.m[a * d + b] = cj(r.m[b * d + a]);
        break;
    case OP_PAIR:
        o.m[0] = cj(r.m[0]); o.m[1] = cj(r.m[2]); o.m[2] = cj(r.m[1]); o.m[3] = cj(r.m[3]);
        break;
    case OP_CPAIR:
        for (size_t m = 0; m < r.m.size() / 4; ++m) {
            const cd *src = r.m.data() + 4 * m;
            cd *dst = o.m.data() + 4 * m;
            dst[0] = cj(src[0]); dst[1] = cj(src[2]); dst[2] = cj(src[1]); dst[3] = cj(src[3]);
        }
        break;
    case OP_DIAG:
    case OP_CDIAG:
        for (auto &z : o.m) z = cj(z);
        break;
    case OP_SHIFT:
    case OP_CSHIFT:
    case OP_MCSHIFT:
        o.op.s = (d - r.op.s % d) % d;
        break;
    case OP_MCDENSE:
        for (int a = 0; a < d; ++a)
            for (int b = 0; b < d; ++b) o.m[a * d + b] = cj(r.m[b * d + a]);
        break;
    case OP_DENSEK: {
        int K = (int)std::lround(std::sqrt((double)r.m.size()));
        for (int a = 0; a < K; ++a)
            for (int b = 0; b < K; ++b) o.m[a * K + b] = cj(r.m[b * K + a]);
        break;
    }
    default:  // SWAP is its own inverse
        break;
    }
    return o;
}

// Generator G = S/2 of a parametrised gate (dU/dtheta = -i G U), in the layout
// of the op's matrix: PAIR kinds (jj, jk, kj, kk), DIAG kinds d real entries.
std::vector<cd> generator_entries(const HGate &g, int d) {
    std::vector<cd> G;
    if (g.axis == 'x') {
        G = {cd(0, 0), cd(0.5, 0), cd(0.5, 0), cd(0, 0)};
    } else if (g.axis == 'y') {
        G = {cd(0, 0), cd(0, -0.5), cd(0, 0.5), cd(0, 0)};
    } else if (g.axis == 'z') {
        G.assign(d, cd(0, 0));
        G[g.j] = cd(0.5, 0);
        G[g.k] = cd(-0.5, 0);
    } else {  // 'g'
        G.assign(d, cd(0, 0));
        const double gam = std::sqrt(2.0 / ((double)g.j * (double)(g.j + 1)));
        for (int l = 0; l < g.j; ++l) G[l] = cd(0.5 * gam, 0);
        G[g.j] = cd(-0.5 * g.j * gam, 0);
    }
    return G;
}

// --------------------------------------------------------------- planning
int default_tile_qudits(int d, bool c128) {
    // largest nt with d^nt amplitudes <= 8192 (complex64) / 4096 (complex128)
    const long long cap = c128 ? 4096 : 8192;
    int nt = 0;
    long long t = 1;
    while (t * d <= cap) {
        t *= d;
        ++nt;
    }
    return nt;
}

// Largest tile an explicit override may ask for: d^nt amplitudes of at most
// 160 KiB, leaving room in the 227 KiB of shared memory a CTA can hold.
int max_tile_qudits(int d, bool c128) {
    const long long cap = (160 * 1024) / (c128 ? 16 : 8);
    int nt = 0;
    long long t = 1;
    while (t * d <= cap) {
        t *= d;
        ++nt;
    }
    return nt < kMaxTileQ ? nt : kMaxTileQ;
}

// Lowest qudits always kept in a tile, so every run a tile reads from HBM
// is d^r contiguous amplitudes.  Longer runs read HBM more efficiently, shorter
// ones leave room for more active qudits (more gates per pass).  Measured on
// GB300 with 200-gate random circuits: d=2 keeps 32-amplitude runs, d=3 27 or
// 81 (equal), d=4 is 13% faster with 16-amplitude runs than with 64, d=5 15%
// faster with 5-amplitude runs (14 passes instead of 31) than with 125.
int min_low_qudits(int d) {
    switch (d) {
    case 2: return 5;
    case 3: return 3;
    case 4: return 2;
    case 5: return 1;
    default: {
        int r = 0;
        long long t = 1;
        while (t < 32) {
            t *= d;
            ++r;
        }
        return r;
    }
    }
}

TileGeom make_geom(int d, int n, const std::vector<int> &active, int rL) {
    TileGeom g;
    std::memset(&g, 0, sizeof(g));
    g.kA = (int)active.size();
    g.rL = rL;
    g.nt = g.kA + rL;
    g.T = (int)ipow_ll(d, g.nt);
    g.SEG = (int)ipow_ll(d, rL);
    g.ntiles = ipow_ll(d, n) / g.T;
    for (int i = 0; i < g.kA; ++i) g.strideA[i] = ipow_ll(d, n - 1 - active[i]);
    // outer runs from the least significant qudit (n - rL - 1) upwards
    std::vector<bool> is_act(n, false);
    for (int q : active) is_act[q] = true;
    int nr = 0;
    int q = n - rL - 1;
    while (q >= 0) {
        if (is_act[q]) { --q; continue; }
        int hi = q;
        while (q >= 0 && !is_act[q]) --q;
        int len = hi - q;  // qudits q+1 .. hi
        g.runM[nr] = ipow_ll(d, len);
        g.runS[nr] = ipow_ll(d, n - 1 - hi);
        ++nr;
    }
    g.nruns = nr;
    g.divSEG = FastDiv((uint32_t)g.SEG);
    return g;
}

int local_pos(const TileGeom &g, const std::vector<int> &active, int n, int q) {
    if (q >= n - g.rL) return g.kA + (q - (n - g.rL));
    for (int i = 0; i < (int)active.size(); ++i)
        if (active[i] == q) return i;
    return -1;
}

TOp localize(const TOp &op, const TileGeom &g, const std::vector<int> &active, int n, int d) {
    TOp o = op;
    auto lstride = [&](int p) { return (int)ipow_ll(d, g.nt - 1 - p); };
    o.a = local_pos(g, active, n, op.a);
    o.lsa = lstride(o.a);
    o.fa = FastDiv((uint32_t)o.lsa);
    if (is_controlled(op) || op.kind == OP_SWAP) {
        o.c = local_pos(g, active, n, op.c);
        o.lsc = lstride(o.c);
        o.fc = FastDiv((uint32_t)o.lsc);
    }
    if (op.kind == OP_DENSEK)
        for (int i = 0; i < op.nq; ++i) o.q[i] = local_pos(g, active, n, op.q[i]);
    return o;
}

static void gate_qudits(const HGate &g, std::vector<int> &out) {
    out.clear();
    for (int i = 0; i < g.nq; ++i) out.push_back(g.q[i]);
}

static bool single_qudit_gate(const HGate &g) {
    return g.nq == 1 && (g.kind == G_H || g.kind == G_X || g.kind == G_Z || g.kind == G_ROT || g.kind == G_DENSE);
}

static bool gate_is_diagonal(const HGate &g) {
    return g.kind == G_Z || (g.kind == G_ROT && (g.axis == 'z' || g.axis == 'g'));
}

// Levels a diagonal gate changes (bit l set: level l gets a phase != 1 in
// general).
static int diag_levels(const HGate &g, int d) {
    int m = 0;
    if (g.kind == G_Z) {
        for (int l = 0; l < d; ++l)
            if (((long long)g.power * l) % d != 0) m |= 1 << l;
    } else if (g.axis == 'z') {
        m = (1 << g.j) | (1 << g.k);
    } else {   // Gell-Mann diagonal j: levels 0..j
        m = (1 << (g.j + 1)) - 1;
    }
    return m;
}

static int popcount_i(int x) {
    int c = 0;
    for (; x; x &= x - 1) ++c;
    return c;
}

// Arithmetic of a single-qudit gate applied alone, per fibre of d
// amplitudes, in paired-FMA issue slots: a complex multiply(-add) is two, a
// real one is one.  Dense: d outputs of d complex terms; RX pair: two outputs
// of two complex terms; RY pair: real entries; diagonal: one complex
// multiply per changed level; shift: a permutation, free.
static int gate_cost(const HGate &g, int d) {
    switch (g.kind) {
    case G_H:
    case G_DENSE: return 2 * d * d;
    case G_X: return 0;
    case G_Z: return 2 * popcount_i(diag_levels(g, d));
    case G_ROT:
        if (g.axis == 'x') return 8;
        if (g.axis == 'y') return 4;
        return 2 * popcount_i(diag_levels(g, d));
    default: return 2 * d * d;
    }
}

// Cost of a group of diagonal gates merged into one diagonal.
static int diag_cost(const std::vector<HGate> &gates, const std::vector<int> &grp, int d) {
    int m = 0;
    for (int gi : grp) m |= diag_levels(gates[gi], d);
    return 2 * popcount_i(m);
}

// Which rL (largest) lets the qudit set fit nt_max local qudits; -1 if none.
static int fit_rl(const std::vector<bool> &inset, int n, int nt_max, int rl_min) {
    int top = std::min(nt_max, n);
    for (int rL = top; rL >= std::min(rl_min, top); --rL) {
        int kA = 0;
        for (int q = 0; q < n - rL; ++q) kA += inset[q] ? 1 : 0;
        if (kA + rL <= nt_max && kA <= kMaxActive) return rL;
    }
    return -1;
}

std::vector<PassPlan> plan_passes(const std::vector<HGate> &gates, int d, int n, bool c128, bool fuse, bool for_adjoint,
                                  int nt_override, int max_ops, int rl_override) {
    std::vector<PassPlan> plan;
    int nt_max = std::min(default_tile_qudits(d, c128), kMaxTileQ);
    // Forward passes of qubits (complex64) measured faster on GB300 with
    // 4096-amplitude tiles and 16-amplitude runs than with 8192 and 32
    // (200-gate random circuit, n=28: 6.58 -> 5.92 ms with five-qubit
    // register stages); the adjoint and batched sweeps keep the defaults.
    const bool qubit_fwd = !for_adjoint && d == 2 && !c128;
    if (qubit_fwd) nt_max = std::min(nt_max, 12);
    // an override may exceed the default tile only in the forward (the
    // adjoint holds two tiles, psi and lambda)
    if (nt_override > 0) nt_max = std::min(nt_override, for_adjoint ? nt_max : max_tile_qudits(d, c128));
    const int op_cap = (max_ops > 0 && max_ops < kMaxTileOps) ? max_ops : kMaxTileOps;
    const int rl_min = std::min(rl_override > 0 ? rl_override : qubit_fwd ? 4 : min_low_qudits(d), nt_max);
    std::vector<int> remaining(gates.size());
    for (size_t i = 0; i < gates.size(); ++i) remaining[i] = (int)i;
    std::vector<int> qs;

    auto finish = [&](std::vector<int> &members, std::vector<bool> &inset) {
        PassPlan p;
        // a multi-controlled gate runs alone through its own kernel
        if (members.size() == 1 && is_mc_gate(gates[members[0]])) {
            p.groups = {{members[0]}};
            p.mc = true;
            plan.push_back(p);
            return;
        }
        int rL = fit_rl(inset, n, nt_max, rl_min);
        if (rL < 0) rL = fit_rl(inset, n, nt_max, 0);   // a lone wide gate may need SEG < 32
        std::vector<int> active;
        for (int q = 0; q < n - rL; ++q)
            if (inset[q]) active.push_back(q);
        // Group single-qudit gates on the same qudit.  A qudit's run of
        // consecutive single-qudit gates (no multi-qudit gate on it in
        // between; gates on other qudits commute with them) becomes one op
        // where that costs no more arithmetic: diagonal gates merge into one
        // diagonal, and the run becomes one dense d x d product once it holds
        // a dense gate or once its ops applied one by one would cost at least
        // a dense product (gate_cost); otherwise its gates stay separate ops.
        // Qubit runs always merge: a 2 x 2 product costs at most two cheap
        // ops, and the separate ops measured 10 % slower (an extra register
        // stage in the heaviest pass of the n=28 program).
        std::vector<int> last_op_on(n, -1);            // op index touching qudit last
        std::vector<std::vector<int>> chain(n);        // the qudit's open single-qudit ops
        std::vector<char> gdense, gdiag;               // per op: dense product / diagonal
        std::vector<int> gcost;                        // per op: cost applied alone
        const int dense_cost = d == 2 ? 0 : 2 * d * d;
        auto new_group = [&](int gi, bool dense, bool diag, int cost) {
            p.groups.push_back({gi});
            gdense.push_back(dense);
            gdiag.push_back(diag);
            gcost.push_back(cost);
            return (int)p.groups.size() - 1;
        };
        for (int gi : members) {
            const HGate &g = gates[gi];
            // the adjoint needs every parametrised gate as an op of its own
            const bool mergeable = fuse && single_qudit_gate(g) && (!for_adjoint || !gate_is_param(g));
            if (!mergeable) {
                const int ix = new_group(gi, false, false, 0);
                for (int i = 0; i < g.nq; ++i) {
                    last_op_on[g.q[i]] = ix;
                    chain[g.q[i]].clear();
                }
                continue;
            }
            const int q = g.q[0];
            std::vector<int> &ch = chain[q];
            const bool g_dense = g.kind == G_H || g.kind == G_DENSE;
            const bool g_diag = gate_is_diagonal(g);
            const int g_cost = gate_cost(g, d);
            const int last = ch.empty() ? -1 : ch.back();
            if (last >= 0 && (gdense[last] || (g_diag && gdiag[last]))) {
                p.groups[last].push_back(gi);   // into a dense product, or diagonal into diagonal
                if (!gdense[last]) gcost[last] = diag_cost(gates, p.groups[last], d);
                continue;
            }
            const int ix = new_group(gi, g_dense, g_diag, g_dense ? dense_cost : g_cost);
            last_op_on[q] = ix;
            ch.push_back(ix);
            int total = 0;
            for (int c : ch) total += gcost[c];
            if (ch.size() > 1 && (g_dense || total >= dense_cost)) {
                // one dense product at the chain's first op (the gates in
                // between touch other qudits only)
                const int first = ch[0];
                for (size_t i = 1; i < ch.size(); ++i) {
                    for (int m : p.groups[ch[i]]) p.groups[first].push_back(m);
                    p.groups[ch[i]].clear();
                }
                gdense[first] = 1;
                gdiag[first] = 0;
                gcost[first] = dense_cost;
                ch.assign(1, first);
                last_op_on[q] = first;
            }
        }
        p.groups.erase(std::remove_if(p.groups.begin(), p.groups.end(),
                                      [](const std::vector<int> &x) { return x.empty(); }),
                       p.groups.end());
        // a lone gate on one wide target goes through the strided kernel
        if (!for_adjoint && p.groups.size() == 1 && p.groups[0].size() == 1) {
            const HGate &g = gates[p.groups[0][0]];
            int target = (g.kind == G_CROT || g.kind == G_SUM) ? g.q[1] : g.q[0];
            bool strided_ok = (single_qudit_gate(g) && !(g.kind == G_DENSE && g.nq != 1)) || g.kind == G_CROT ||
                              g.kind == G_SUM;
            if (strided_ok && ipow_ll(d, n - 1 - target) >= kWideMin && ipow_ll(d, n - 1 - target) < (1ll << 31)) {
                p.strided = true;
                plan.push_back(p);
                return;
            }
        }
        p.active = active;
        p.geom = make_geom(d, n, active, rL);
        plan.push_back(p);
    };

    while (!remaining.empty()) {
        std::vector<bool> inset(n, false), blocked(n, false);
        std::vector<int> members, deferred;
        int nparam = 0;
        size_t scan = 0;
        for (; scan < remaining.size(); ++scan) {
            const int gi = remaining[scan];
            gate_qudits(gates[gi], qs);
            bool is_blocked = false;
            for (int q : qs) is_blocked |= blocked[q];
            bool take = false;
            // adjoint passes keep at most kMaxGrad gradient columns (register accumulators)
            const bool param_full = for_adjoint && gate_is_param(gates[gi]) && nparam >= kMaxGrad;
            // a multi-controlled gate is a pass of its own: it starts one, or waits
            const bool mc = is_mc_gate(gates[gi]);
            if (mc && !is_blocked && members.empty()) {
                members.push_back(gi);
                for (int q : qs) inset[q] = true;
                ++scan;
                break;
            }
            if (!is_blocked && !param_full && !mc && (int)members.size() < op_cap && (fuse || members.empty())) {
                std::vector<bool> trial = inset;
                for (int q : qs) trial[q] = true;
                if (fit_rl(trial, n, nt_max, rl_min) >= 0) {
                    inset = trial;
                    take = true;
                }
            }
            if (take) {
                members.push_back(gi);
                if (gate_is_param(gates[gi])) ++nparam;
            } else {
                deferred.push_back(gi);
                for (int q : qs) blocked[q] = true;
                if (!fuse) { ++scan; break; }
                // stop scanning once every qudit is blocked
                bool all = true;
                for (int q = 0; q < n && all; ++q) all = blocked[q];
                if (all) { ++scan; break; }
            }
        }
        for (; scan < remaining.size(); ++scan) deferred.push_back(remaining[scan]);
        if (members.empty()) {
            // cannot happen for valid gates (any gate fits an empty tile)
            members.push_back(deferred.front());
            deferred.erase(deferred.begin());
            gate_qudits(gates[members[0]], qs);
            for (int q : qs) inset[q] = true;
        }
        finish(members, inset);
        remaining.swap(deferred);
    }
    return plan;
}

// Groups a pass's ops (already in tile-local form, in application order)
// into register stages of up to stage_k(d) local qudits.  An op joins the
// current stage if the union of the stage's qudits and the qudits the op must
// hold in registers (its target; none for a diagonal op, which can use a
// block-constant digit) stays within K.  SWAP and custom k-qudit gates are
// shared-memory ops of their own.  Leftover slots take diagonal targets and
// controls of the stage's ops, then the most significant free positions
// (which keeps consecutive threads on consecutive shared-memory words).
std::vector<TStage> build_stages(std::vector<TOp> &ops, const TileGeom &g, int d, int K) {
    std::vector<TStage> st;
    const int nt = g.nt;
    // a tile narrower than K runs every op through shared memory (the kernels
    // treat an empty stage list that way, gradients included)
    if (K == 0 || nt < K || K > kMaxStageK) return st;
    auto legacy_kind = [](const TOp &o) { return o.kind == OP_SWAP || o.kind == OP_DENSEK; };
    auto has = [](const std::vector<int> &v, int x) { return std::find(v.begin(), v.end(), x) != v.end(); };
    size_t i = 0;
    while (i < ops.size()) {
        if (legacy_kind(ops[i])) {
            TStage t;
            std::memset(&t, 0, sizeof(t));
            t.legacy = 1;
            t.first = (int)i;
            t.nops = 1;
            st.push_back(t);
            ++i;
            continue;
        }
        std::vector<int> Q;
        size_t j = i;
        while (j < ops.size() && !legacy_kind(ops[j])) {
            std::vector<int> nq = Q;
            if (ops[j].kind != OP_DIAG && !has(nq, ops[j].a)) nq.push_back(ops[j].a);
            if ((int)nq.size() > K) break;
            Q.swap(nq);
            ++j;
        }
        for (size_t k = i; k < j && (int)Q.size() < K; ++k)
            if (ops[k].kind == OP_DIAG && !has(Q, ops[k].a)) Q.push_back(ops[k].a);
        for (size_t k = i; k < j && (int)Q.size() < K; ++k)
            if (is_controlled(ops[k]) && !has(Q, ops[k].c)) Q.push_back(ops[k].c);
        for (int p = 0; p < nt && (int)Q.size() < K; ++p)
            if (!has(Q, p)) Q.push_back(p);
        std::sort(Q.begin(), Q.end());
        TStage t;
        std::memset(&t, 0, sizeof(t));
        t.legacy = 0;
        t.first = (int)i;
        t.nops = (int)(j - i);
        std::vector<int> asc;
        for (int x = 0; x < K; ++x) {
            t.ls[x] = (int)ipow_ll(d, nt - 1 - Q[x]);
            asc.push_back(t.ls[x]);
        }
        std::sort(asc.begin(), asc.end());
        for (int x = 0; x < K; ++x) {
            t.lsa[x] = asc[x];
            t.fa[x] = FastDiv((uint32_t)asc[x]);
        }
        auto slot_of = [&](int pos) {
            for (int x = 0; x < K; ++x)
                if (Q[x] == pos) return x;
            return -1;
        };
        for (size_t k = i; k < j; ++k) {
            ops[k].q[4] = slot_of(ops[k].a);
            ops[k].q[5] = is_controlled(ops[k]) ? slot_of(ops[k].c) : -1;
        }
        st.push_back(t);
        i = j;
    }
    return st;
}

}  // namespace qf
