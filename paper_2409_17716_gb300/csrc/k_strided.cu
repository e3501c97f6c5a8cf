// k_strided.cu -- gates on one target qudit whose stride S >= 32 amplitudes.
//
// A fibre is the set {hi*(d*S) + l*S + lo : l = 0..d-1} of amplitudes that a
// single-qudit gate couples (Appendix B: every single-qudit gate acts as a
// d x d block on each fibre).  One thread owns UNR fibres; consecutive threads
// own consecutive lo, so each level row is read and written as a coalesced
// stream of 256-byte (complex64) warp transactions.  Only the rows a gate
// touches are loaded: a level-pair rotation reads and writes rows j and k
// (2/d of the state), a diagonal gate only its non-unit rows, a controlled
// gate skips fibres whose control level is 0.
//
// Controlled gates (Appendix B, "Controlled Rotation Gate" and "Generalized
// CNOT gate") use the same fibres over the target; the control level is a
// digit of the fibre's base index: for a control above the target it is a
// digit of hi, below the target a digit of lo.
//
// Registers that mix dimensions (section "Code style") have the same fibre
// structure with the target's own dimension and stride, and a control digit
// taken modulo the control's dimension; the launcher takes that geometry
// explicitly, and any stride works (below 32 the fibres of a warp interleave
// and L1 merges their sectors).
//
// k_strided_adj is one reverse step of the adjoint sweep for such a gate:
// with psi and lambda the states after the gate, it adds 2 Im <lambda|G|psi>
// (G the generator, dU/dtheta = -i G U, scaled by the control level for a
// controlled rotation) to a per-CTA gradient row, then applies U^+ to both.
#include "qf_internal.cuh"
#include "qf_host.h"

namespace qf {

template <int D>
__device__ __forceinline__ int mod_d(uint32_t x, int d_rt) {
    if (D > 0) return (int)(x % (uint32_t)D);
    return (int)(x % (uint32_t)d_rt);
}

template <typename R>
struct StridedArgs {
    cplx<R> *psi;
    long long base0;        // element offset of the first hi block in this launch
    long long hi0;          // global hi index of the first block
    uint32_t nfib;          // fibres in this launch (nh * S)
    uint32_t S;             // target stride
    FastDiv divS;           // divide by S
    FastDiv divC;           // control: divide hi (control above) or lo (below) by this
    int ctrl_above;         // 1: control digit from hi, 0: from lo
    int dc;                 // control dimension (mixed registers; = d otherwise)
    int wide_hi;            // hi index may exceed 32 bits: 64-bit control digit
    long long divC64;       // the control divisor for wide_hi
    TOp op;
    cplx<R> m[kInlineMat];
};

// Control level of a fibre: digit of (hi0 + h) above the target, of lo below.
template <int D, typename A_t>
__device__ __forceinline__ int control_level(const A_t &A, uint32_t h, uint32_t lo, int d) {
    if (A.ctrl_above) {
        if (A.wide_hi) return (int)(((unsigned long long)A.hi0 + h) / (unsigned long long)A.divC64 % (unsigned long long)A.dc);
        const uint32_t x = A.divC.div((uint32_t)(A.hi0 + h));
        return A.dc == d ? mod_d<D>(x, d) : (int)(x % (uint32_t)A.dc);
    }
    const uint32_t x = A.divC.div(lo);
    return A.dc == d ? mod_d<D>(x, d) : (int)(x % (uint32_t)A.dc);
}

constexpr int kStridedBlock = 256;
constexpr int kStridedUnroll = 2;

template <typename R, int D>
__global__ void __launch_bounds__(kStridedBlock) k_strided(const __grid_constant__ StridedArgs<R> A, int d_rt) {
    using C = cplx<R>;
    constexpr int DM = D > 0 ? D : kMaxD;
    const int d = D > 0 ? D : d_rt;
    const TOp &op = A.op;
    const long long S = A.S;
    const long long DS = (long long)d * S;

    long long idx[kStridedUnroll];
    int ctl[kStridedUnroll];
    bool ok[kStridedUnroll];
    const uint32_t f0 = blockIdx.x * (kStridedBlock * kStridedUnroll) + threadIdx.x;
#pragma unroll
    for (int u = 0; u < kStridedUnroll; ++u) {
        uint32_t f = f0 + u * kStridedBlock;
        ok[u] = f < A.nfib;
        uint32_t h = A.divS.div(f);
        uint32_t lo = f - h * A.S;
        idx[u] = A.base0 + (long long)h * DS + lo;
        ctl[u] = control_level<D>(A, h, lo, d);
    }
    C *psi = A.psi;

    switch (op.kind) {
    case OP_DENSE: {
        C v[kStridedUnroll][DM];
#pragma unroll
        for (int u = 0; u < kStridedUnroll; ++u)
            if (ok[u]) {
#pragma unroll
                for (int m = 0; m < DM; ++m)
                    if (m < d) v[u][m] = psi[idx[u] + m * S];
            }
#pragma unroll
        for (int u = 0; u < kStridedUnroll; ++u)
            if (ok[u]) {
#pragma unroll
                for (int l = 0; l < DM; ++l) {
                    if (l >= d) break;
                    C acc = mk<R>(0, 0);
#pragma unroll
                    for (int m = 0; m < DM; ++m)
                        if (m < d) acc = cfma(A.m[l * d + m], v[u][m], acc);
                    psi[idx[u] + l * S] = acc;
                }
            }
        break;
    }
    case OP_PAIR:
    case OP_CPAIR: {
        C a[kStridedUnroll], b[kStridedUnroll];
        const bool ctrl = op.kind == OP_CPAIR;
#pragma unroll
        for (int u = 0; u < kStridedUnroll; ++u) {
            if (ctrl && ctl[u] == 0) ok[u] = false;
            if (ok[u]) {
                a[u] = psi[idx[u] + op.j * S];
                b[u] = psi[idx[u] + op.k * S];
            }
        }
#pragma unroll
        for (int u = 0; u < kStridedUnroll; ++u)
            if (ok[u]) {
                const C *M = A.m + (ctrl ? 4 * ctl[u] : 0);
                C x = cfma(M[1], b[u], cmul(M[0], a[u]));
                C y = cfma(M[3], b[u], cmul(M[2], a[u]));
                psi[idx[u] + op.j * S] = x;
                psi[idx[u] + op.k * S] = y;
            }
        break;
    }
    case OP_DIAG:
    case OP_CDIAG: {
        const bool ctrl = op.kind == OP_CDIAG;
        C v[kStridedUnroll][DM];
#pragma unroll
        for (int u = 0; u < kStridedUnroll; ++u) {
            if (ctrl && ctl[u] == 0) ok[u] = false;
            if (ok[u]) {
#pragma unroll
                for (int l = 0; l < DM; ++l)
                    if (l < d && ((op.mask >> l) & 1)) v[u][l] = psi[idx[u] + l * S];
            }
        }
#pragma unroll
        for (int u = 0; u < kStridedUnroll; ++u)
            if (ok[u]) {
                const C *M = A.m + (ctrl ? d * ctl[u] : 0);
#pragma unroll
                for (int l = 0; l < DM; ++l)
                    if (l < d && ((op.mask >> l) & 1)) psi[idx[u] + l * S] = cmul(M[l], v[u][l]);
            }
        break;
    }
    case OP_SHIFT:
    case OP_CSHIFT: {
        const bool ctrl = op.kind == OP_CSHIFT;
        C v[kStridedUnroll][DM];
        int sh[kStridedUnroll];
#pragma unroll
        for (int u = 0; u < kStridedUnroll; ++u) {
            sh[u] = ctrl ? (int)((op.s * ctl[u]) % d) : op.s;
            if (sh[u] == 0) ok[u] = false;
            if (ok[u]) {
#pragma unroll
                for (int m = 0; m < DM; ++m)
                    if (m < d) v[u][m] = psi[idx[u] + m * S];
            }
        }
#pragma unroll
        for (int u = 0; u < kStridedUnroll; ++u)
            if (ok[u]) {
#pragma unroll
                for (int m = 0; m < DM; ++m)
                    if (m < d) {
                        int dst = m + sh[u];
                        if (dst >= d) dst -= d;
                        psi[idx[u] + dst * S] = v[u][m];
                    }
            }
        break;
    }
    default:
        break;
    }
}

// Fills the geometry-dependent fields of the kernel arguments; returns false
// if the geometry is not supported.
template <typename A_t>
static bool strided_setup(A_t &A, const StridedGeom &g, const TOp &op) {
    const bool ctrl = op.kind == OP_CPAIR || op.kind == OP_CDIAG || op.kind == OP_CSHIFT;
    if (g.S < 1 || g.S >= (1ll << 31) || g.d < 2 || g.d > kMaxD) return false;
    A.ctrl_above = ctrl && g.c_above;
    A.dc = ctrl ? g.dc : g.d;
    A.wide_hi = 0;
    A.divC64 = 1;
    if (ctrl) {
        if (A.ctrl_above) {
            const long long q = g.Sc / (g.d * g.S);   // hi digit divisor
            A.divC64 = q;
            A.wide_hi = (g.H >= (1ll << 32) || q >= (1ll << 32)) ? 1 : 0;
            A.divC = FastDiv(A.wide_hi ? 1u : (uint32_t)q);
        } else {
            A.divC = FastDiv((uint32_t)g.Sc);       // lo digit
        }
    } else {
        A.divC = FastDiv(1);
    }
    A.S = (uint32_t)g.S;
    A.divS = FastDiv((uint32_t)g.S);
    return true;
}

// Host launcher on an explicit geometry.  `op` refers to global qudits: op.a
// is the target, op.c the control for controlled kinds.  `mat` holds the op's
// matrix entries already rounded to R.
template <typename R>
cudaError_t launch_strided_g(const Launch &L, cplx<R> *psi, const StridedGeom &g, const TOp &op, const cplx<R> *mat,
                             int nmat) {
    if (nmat > kInlineMat) return cudaErrorInvalidValue;
    StridedArgs<R> A;
    A.psi = psi;
    A.op = op;
    for (int i = 0; i < nmat; ++i) A.m[i] = mat[i];
    if (!strided_setup(A, g, op)) return cudaErrorInvalidValue;
    const int d = g.d;
    const long long S = g.S, H = g.H;
    // split into launches whose fibre count fits 32 bits
    const long long max_fib = 1ll << 30;
    long long hper = max_fib / S;
    if (hper < 1) hper = 1;
    for (long long h0 = 0; h0 < H; h0 += hper) {
        long long nh = H - h0 < hper ? H - h0 : hper;
        A.hi0 = h0;
        A.base0 = h0 * d * S;
        A.nfib = (uint32_t)(nh * S);
        long long per_block = (long long)kStridedBlock * kStridedUnroll;
        unsigned grid = (unsigned)((A.nfib + per_block - 1) / per_block);
        switch (d) {
#define QF_CASE(DD) case DD: k_strided<R, DD><<<grid, kStridedBlock, 0, L.stream>>>(A, d); break;
            QF_CASE(2) QF_CASE(3) QF_CASE(4) QF_CASE(5) QF_CASE(6) QF_CASE(7) QF_CASE(8)
#undef QF_CASE
        default: k_strided<R, 0><<<grid, kStridedBlock, 0, L.stream>>>(A, d); break;
        }
    }
    return cudaGetLastError();
}

StridedGeom uniform_geom(int d, int n, const TOp &op) {
    StridedGeom g;
    g.d = d;
    g.S = ipow_ll(d, n - 1 - op.a);
    g.H = ipow_ll(d, op.a);
    const bool ctrl = op.kind == OP_CPAIR || op.kind == OP_CDIAG || op.kind == OP_CSHIFT;
    g.dc = d;
    g.Sc = ctrl ? ipow_ll(d, n - 1 - op.c) : 1;
    g.c_above = ctrl && op.c < op.a;
    return g;
}

// Uniform registers: every qudit has dimension d, so S = d^(n-1-a).
template <typename R>
cudaError_t launch_strided(const Launch &L, cplx<R> *psi, int d, int n, const TOp &op, const cplx<R> *mat, int nmat) {
    return launch_strided_g<R>(L, psi, uniform_geom(d, n, op), op, mat, nmat);
}

// ------------------------------------------------------------------ adjoint step
template <typename R>
struct StridedAdjArgs {
    cplx<R> *psi, *lam;
    long long base0, hi0;
    uint32_t nfib, S;
    FastDiv divS, divC;
    int ctrl_above, dc, wide_hi;
    long long divC64;
    int grad;               // 1: accumulate the gradient term of this gate
    double *rows;           // one gradient partial per CTA (this launch's first CTA at rows[0])
    TOp op;                 // U^+ in the op's layout
    cplx<R> m[kInlineMat];
    cplx<R> gen[kMaxD];     // generator: PAIR kinds (jj, jk, kj, kk), DIAG kinds d entries
};

__device__ __forceinline__ double adj_block_sum(double v, double *red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) red[wid] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    return s;
}

// Im(conj(a) * b), in the precision of the amplitudes (FP64 is far slower
// than FP32 on this GPU; each thread's sum is widened at the block reduction)
template <typename C>
__device__ __forceinline__ auto im_conj_mul(C a, C b) -> decltype(a.x) {
    return a.x * b.y - a.y * b.x;
}

template <typename R, int D>
__global__ void __launch_bounds__(kStridedBlock) k_strided_adj(const __grid_constant__ StridedAdjArgs<R> A, int d_rt) {
    using C = cplx<R>;
    constexpr int DM = D > 0 ? D : kMaxD;
    __shared__ double red[kStridedBlock / 32];
    const int d = D > 0 ? D : d_rt;
    const TOp &op = A.op;
    const long long S = A.S;
    C *psi = A.psi, *lam = A.lam;
    R g = 0;
    // grid-stride over fibres: the grid is capped so each gate leaves a few
    // hundred gradient rows, not one per 256 fibres
    for (uint32_t f = blockIdx.x * kStridedBlock + threadIdx.x; f < A.nfib; f += gridDim.x * kStridedBlock) {
        const uint32_t h = A.divS.div(f);
        const uint32_t lo = f - h * A.S;
        const long long idx = A.base0 + (long long)h * d * S + lo;
        const int ctl = control_level<D>(A, h, lo, d);
        switch (op.kind) {
        case OP_DENSE: {
            C v[DM], w[DM];
#pragma unroll
            for (int m = 0; m < DM; ++m)
                if (m < d) { v[m] = psi[idx + m * S]; w[m] = lam[idx + m * S]; }
#pragma unroll
            for (int l = 0; l < DM; ++l) {
                if (l >= d) break;
                C a = mk<R>(0, 0), b = mk<R>(0, 0);
#pragma unroll
                for (int m = 0; m < DM; ++m)
                    if (m < d) { a = cfma(A.m[l * d + m], v[m], a); b = cfma(A.m[l * d + m], w[m], b); }
                psi[idx + l * S] = a;
                lam[idx + l * S] = b;
            }
            break;
        }
        case OP_PAIR:
        case OP_CPAIR: {
            const bool ctrl = op.kind == OP_CPAIR;
            if (ctrl && ctl == 0) break;
            const C a = psi[idx + op.j * S], b = psi[idx + op.k * S];
            const C la = lam[idx + op.j * S], lb = lam[idx + op.k * S];
            if (A.grad) {
                const C ga = cfma(A.gen[1], b, cmul(A.gen[0], a));
                const C gb = cfma(A.gen[3], b, cmul(A.gen[2], a));
                g += (im_conj_mul(la, ga) + im_conj_mul(lb, gb)) * (ctrl ? (R)ctl : (R)1);
            }
            const C *M = A.m + (ctrl ? 4 * ctl : 0);
            psi[idx + op.j * S] = cfma(M[1], b, cmul(M[0], a));
            psi[idx + op.k * S] = cfma(M[3], b, cmul(M[2], a));
            lam[idx + op.j * S] = cfma(M[1], lb, cmul(M[0], la));
            lam[idx + op.k * S] = cfma(M[3], lb, cmul(M[2], la));
            break;
        }
        case OP_DIAG:
        case OP_CDIAG: {
            const bool ctrl = op.kind == OP_CDIAG;
            if (ctrl && ctl == 0) break;
            const C *M = A.m + (ctrl ? d * ctl : 0);
            R t = 0;
#pragma unroll
            for (int l = 0; l < DM; ++l)
                if (l < d && ((op.mask >> l) & 1)) {
                    const C v = psi[idx + l * S], w = lam[idx + l * S];
                    if (A.grad) t += A.gen[l].x * im_conj_mul(w, v);
                    psi[idx + l * S] = cmul(M[l], v);
                    lam[idx + l * S] = cmul(M[l], w);
                }
            g += t * (ctrl ? (R)ctl : (R)1);
            break;
        }
        case OP_SHIFT:
        case OP_CSHIFT: {
            const bool ctrl = op.kind == OP_CSHIFT;
            const int sh = ctrl ? (int)((op.s * ctl) % d) : op.s;
            if (sh == 0) break;
            C v[DM], w[DM];
#pragma unroll
            for (int m = 0; m < DM; ++m)
                if (m < d) { v[m] = psi[idx + m * S]; w[m] = lam[idx + m * S]; }
#pragma unroll
            for (int m = 0; m < DM; ++m)
                if (m < d) {
                    int dst = m + sh;
                    if (dst >= d) dst -= d;
                    psi[idx + dst * S] = v[m];
                    lam[idx + dst * S] = w[m];
                }
            break;
        }
        default:
            break;
        }
    }
    if (A.grad) {
        const double s = adj_block_sum((double)g, red);
        if (threadIdx.x == 0) A.rows[blockIdx.x] = 2.0 * s;
    }
}

constexpr int kAdjBlocksPerSM = 8;

static unsigned adj_grid_of(uint32_t nfib, int num_sms) {
    long long b = ((long long)nfib + kStridedBlock - 1) / kStridedBlock;
    const long long cap = (long long)(num_sms > 0 ? num_sms : 1) * kAdjBlocksPerSM;
    return (unsigned)(b < cap ? b : cap);
}

// CTAs one adjoint step launches (gradient rows it writes).
long long strided_adj_blocks(const StridedGeom &g, int num_sms) {
    const long long max_fib = 1ll << 30;
    long long hper = max_fib / g.S;
    if (hper < 1) hper = 1;
    long long total = 0;
    for (long long h0 = 0; h0 < g.H; h0 += hper) {
        long long nh = g.H - h0 < hper ? g.H - h0 : hper;
        total += adj_grid_of((uint32_t)(nh * g.S), num_sms);
    }
    return total;
}

// One reverse step: `op`/`mat` are U^+; `gen` (nullptr: no gradient) the
// generator entries; rows receives strided_adj_blocks(g) partials.
template <typename R>
cudaError_t launch_strided_adj(const Launch &L, cplx<R> *psi, cplx<R> *lam, const StridedGeom &g, const TOp &op,
                               const cplx<R> *mat, int nmat, const cplx<R> *gen, int ngen, double *rows) {
    if (nmat > kInlineMat || ngen > kMaxD) return cudaErrorInvalidValue;
    StridedAdjArgs<R> A;
    A.psi = psi;
    A.lam = lam;
    A.op = op;
    for (int i = 0; i < nmat; ++i) A.m[i] = mat[i];
    A.grad = gen ? 1 : 0;
    for (int i = 0; i < kMaxD; ++i) A.gen[i] = (gen && i < ngen) ? gen[i] : mk<R>(0, 0);
    if (!strided_setup(A, g, op)) return cudaErrorInvalidValue;
    const int d = g.d;
    const long long S = g.S, H = g.H;
    const long long max_fib = 1ll << 30;
    long long hper = max_fib / S;
    if (hper < 1) hper = 1;
    long long row = 0;
    for (long long h0 = 0; h0 < H; h0 += hper) {
        long long nh = H - h0 < hper ? H - h0 : hper;
        A.hi0 = h0;
        A.base0 = h0 * d * S;
        A.nfib = (uint32_t)(nh * S);
        A.rows = rows ? rows + row : nullptr;
        const unsigned grid = adj_grid_of(A.nfib, L.num_sms);
        row += grid;
        switch (d) {
#define QF_CASE(DD) case DD: k_strided_adj<R, DD><<<grid, kStridedBlock, 0, L.stream>>>(A, d); break;
            QF_CASE(2) QF_CASE(3) QF_CASE(4) QF_CASE(5)
#undef QF_CASE
        default: k_strided_adj<R, 0><<<grid, kStridedBlock, 0, L.stream>>>(A, d); break;
        }
    }
    return cudaGetLastError();
}

template cudaError_t launch_strided_g<float>(const Launch &, cplx<float> *, const StridedGeom &, const TOp &,
                                             const cplx<float> *, int);
template cudaError_t launch_strided_g<double>(const Launch &, cplx<double> *, const StridedGeom &, const TOp &,
                                              const cplx<double> *, int);
template cudaError_t launch_strided_adj<float>(const Launch &, cplx<float> *, cplx<float> *, const StridedGeom &,
                                               const TOp &, const cplx<float> *, int, const cplx<float> *, int, double *);
template cudaError_t launch_strided_adj<double>(const Launch &, cplx<double> *, cplx<double> *, const StridedGeom &,
                                                const TOp &, const cplx<double> *, int, const cplx<double> *, int,
                                                double *);
template cudaError_t launch_strided<float>(const Launch &, cplx<float> *, int, int, const TOp &, const cplx<float> *, int);
template cudaError_t launch_strided<double>(const Launch &, cplx<double> *, int, int, const TOp &, const cplx<double> *, int);

}  // namespace qf
