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
#include "qf_internal.cuh"

namespace qf {

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
    TOp op;
    cplx<R> m[kInlineMat];
};

constexpr int kStridedBlock = 256;
constexpr int kStridedUnroll = 2;

template <int D>
__device__ __forceinline__ int mod_d(uint32_t x, int d_rt) {
    if (D > 0) return (int)(x % (uint32_t)D);
    return (int)(x % (uint32_t)d_rt);
}

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
        if (A.ctrl_above) {
            ctl[u] = mod_d<D>((uint32_t)A.divC.div((uint32_t)(A.hi0 + h)), d);
        } else {
            ctl[u] = mod_d<D>(A.divC.div(lo), d);
        }
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

// Host launcher.  `op` refers to global qudits: op.a is the target (stride
// S = d^(n-1-a)), op.c the control for controlled kinds.  `mat` holds the
// op's matrix entries already rounded to R.
template <typename R>
cudaError_t launch_strided(const Launch &L, cplx<R> *psi, int d, int n, const TOp &op, const cplx<R> *mat, int nmat) {
    if (nmat > kInlineMat) return cudaErrorInvalidValue;
    StridedArgs<R> A;
    A.psi = psi;
    A.op = op;
    for (int i = 0; i < nmat; ++i) A.m[i] = mat[i];
    long long S = 1;
    for (int i = 0; i < n - 1 - op.a; ++i) S *= d;
    long long N = S;
    for (int i = 0; i < op.a + 1; ++i) N *= d;
    long long H = N / (d * S);
    bool ctrl = op.kind == OP_CPAIR || op.kind == OP_CDIAG || op.kind == OP_CSHIFT;
    long long Sc = 1;
    if (ctrl)
        for (int i = 0; i < n - 1 - op.c; ++i) Sc *= d;
    A.ctrl_above = ctrl && op.c < op.a;
    if (ctrl) {
        if (A.ctrl_above) A.divC = FastDiv((uint32_t)(Sc / (d * S)));   // hi digit
        else A.divC = FastDiv((uint32_t)Sc);                           // lo digit
    } else {
        A.divC = FastDiv(1);
    }
    A.S = (uint32_t)S;
    A.divS = FastDiv((uint32_t)S);
    // split into launches whose fibre count and global hi index fit 32 bits
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

template cudaError_t launch_strided<float>(const Launch &, cplx<float> *, int, int, const TOp &, const cplx<float> *, int);
template cudaError_t launch_strided<double>(const Launch &, cplx<double> *, int, int, const TOp &, const cplx<double> *, int);

}  // namespace qf
