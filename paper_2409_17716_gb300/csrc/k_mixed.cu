// k_mixed.cu -- kernels for registers that mix qudit dimensions (section
// "Code style": Circuit(dim=[2,3,4])).
//
// Basis index of a mixed register: i = sum_q i_q S_q, S_q = prod_{p>q} dims[p]
// (mixed radix, qudit 0 most significant).  Single-qudit and controlled gates
// keep the fibre structure {hi*(d_a S_a) + l*S_a + lo} and run through the
// strided kernel with the target's own dimension and stride.  This file adds:
//
//   k_group             multi-qudit dense gate (gather the K = prod d_t
//                       amplitudes a group couples, multiply, scatter) and
//                       SWAP of two equal-dimension qudits; one thread a group
//   k_expect_mixed      <N_q> for every q and the norm in one pass
//   k_number_obs_mixed  lambda = O psi for O = sum_q w_q N_q, and the loss
//
// The reductions view the state as H rows of B contiguous amplitudes, B the
// product of the dims of the lowest qudits (B <= 512).  Row h spells the high
// digits, column c the low digits, so with p_i = |psi_i|^2
//   sum_i i_q p_i = sum_h digit_q(h) P_h      (q high, P_h = row sums)
//                 = sum_c digit_q(c) Q_c      (q low,  Q_c = column sums).
// A warp owns a row at a time: lane l reads columns l, l + 32, ... (coalesced),
// keeps its column sums in registers (FP32 over at most 32 rows, then FP64),
// and the warp sum of the row is weighted by the row's digits, one qudit per
// lane.  Digit extraction is therefore per row and per column, not per
// amplitude.  CTA partials are summed in a fixed order (deterministic).
#include <cstring>

#include "qf_host.h"

namespace qf {

// ------------------------------------------------------------------ groups
struct GroupArgs {
    int K;                          // amplitudes a group couples (dense)
    int swap;                       // 1: SWAP of two qudits of dimension sd
    int sd;
    long long sa, sb;               // SWAP: strides of the two qudits
    long long off[kMaxDenseK];      // dense: offset of group member r
    int nruns;                      // runs of consecutive non-target qudits, least significant first
    long long runM[kMaxQudits];     // radix of a run (product of its dims)
    long long runS[kMaxQudits];     // stride of its least significant qudit
    long long G;                    // groups
};

template <typename R>
__global__ void __launch_bounds__(256) k_group(cplx<R> *__restrict__ psi, const __grid_constant__ GroupArgs A,
                                               const cplx<R> *__restrict__ mat) {
    using C = cplx<R>;
    for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < A.G; g += (long long)gridDim.x * blockDim.x) {
        long long rem = g, base = 0;
        for (int r = 0; r < A.nruns; ++r) {
            const long long nx = rem / A.runM[r];
            base += (rem - nx * A.runM[r]) * A.runS[r];
            rem = nx;
        }
        if (A.swap) {
            for (int x = 0; x < A.sd; ++x)
                for (int y = x + 1; y < A.sd; ++y) {
                    const long long i = base + x * A.sa + y * A.sb, j = base + y * A.sa + x * A.sb;
                    const C u = psi[i], v = psi[j];
                    psi[i] = v;
                    psi[j] = u;
                }
            continue;
        }
        C v[kMaxDenseK];
        for (int m = 0; m < A.K; ++m) v[m] = psi[base + A.off[m]];
        for (int r = 0; r < A.K; ++r) {
            C acc = mk<R>(0, 0);
            for (int m = 0; m < A.K; ++m) acc = cfma(mat[r * A.K + m], v[m], acc);
            psi[base + A.off[r]] = acc;
        }
    }
}

template <typename R>
cudaError_t launch_group(const Launch &L, cplx<R> *psi, const MixedShape &m, const TOp &op, const cplx<R> *mat_dev) {
    GroupArgs A;
    std::memset(&A, 0, sizeof(A));
    bool is_t[kMaxQudits] = {};
    long long K = 1;
    if (op.kind == OP_SWAP) {
        if (m.dims[op.a] != m.dims[op.c]) return cudaErrorInvalidValue;
        A.swap = 1;
        A.sd = m.dims[op.a];
        A.sa = m.S[op.a];
        A.sb = m.S[op.c];
        is_t[op.a] = is_t[op.c] = true;
        K = (long long)A.sd * A.sd;
    } else if (op.kind == OP_DENSEK || op.kind == OP_DENSE) {
        const int nq = op.kind == OP_DENSE ? 1 : op.nq;
        int q[6];
        for (int i = 0; i < nq; ++i) q[i] = op.kind == OP_DENSE ? op.a : op.q[i];
        for (int i = 0; i < nq; ++i) {
            is_t[q[i]] = true;
            K *= m.dims[q[i]];
        }
        if (K > kMaxDenseK || !mat_dev) return cudaErrorInvalidValue;
        A.K = (int)K;
        for (long long r = 0; r < K; ++r) {
            long long rem = r, o = 0;
            for (int i = nq - 1; i >= 0; --i) {
                o += (rem % m.dims[q[i]]) * m.S[q[i]];
                rem /= m.dims[q[i]];
            }
            A.off[r] = o;
        }
    } else {
        return cudaErrorInvalidValue;
    }
    // runs of consecutive non-target qudits, from the least significant
    A.nruns = 0;
    for (int q = m.n - 1; q >= 0;) {
        if (is_t[q]) { --q; continue; }
        long long M = 1;
        const long long S = m.S[q];
        while (q >= 0 && !is_t[q]) { M *= m.dims[q]; --q; }
        A.runM[A.nruns] = M;
        A.runS[A.nruns] = S;
        ++A.nruns;
    }
    A.G = m.N / K;
    long long blocks = (A.G + 255) / 256;
    const long long cap = (long long)L.num_sms * 16;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    k_group<R><<<(unsigned)blocks, 256, 0, L.stream>>>(psi, A, mat_dev);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ multi-controlled gates
// One thread per fibre {hi*(d S) + l*S + lo} of the target (coalesced along lo
// for S >= 32); the control levels are digits of the fibre's base index.
// MCSHIFT moves the target by s * (product of the control levels) mod d and
// skips fibres where that is 0; MCDENSE applies the d x d matrix only where
// every control sits at its level.
template <typename R>
struct MCArgs {
    int kind, d, nc, s;
    long long S, nfib;
    long long cS[6];
    int cd[6], lv[6];
    cplx<R> V[kMaxD * kMaxD];
};

template <typename R>
__global__ void __launch_bounds__(256) k_mc(cplx<R> *__restrict__ psi, const __grid_constant__ MCArgs<R> A) {
    using C = cplx<R>;
    const int d = A.d;
    for (long long f = (long long)blockIdx.x * blockDim.x + threadIdx.x; f < A.nfib;
         f += (long long)gridDim.x * blockDim.x) {
        const long long h = f / A.S, lo = f - h * A.S;
        const long long base = h * d * A.S + lo;
        long long prod = 1;
        bool match = true;
        for (int i = 0; i < A.nc; ++i) {
            const int dig = (int)((base / A.cS[i]) % A.cd[i]);
            prod *= dig;
            match &= dig == A.lv[i];
        }
        C v[kMaxD];
        if (A.kind == OP_MCSHIFT) {
            const int sh = (int)(((long long)A.s * (prod % d)) % d);
            if (sh == 0) continue;
            for (int m = 0; m < d; ++m) v[m] = psi[base + m * A.S];
            for (int m = 0; m < d; ++m) {
                int dst = m + sh;
                if (dst >= d) dst -= d;
                psi[base + dst * A.S] = v[m];
            }
        } else {
            if (!match) continue;
            for (int m = 0; m < d; ++m) v[m] = psi[base + m * A.S];
            for (int l = 0; l < d; ++l) {
                C acc = mk<R>(0, 0);
                for (int m = 0; m < d; ++m) acc = cfma(A.V[l * d + m], v[m], acc);
                psi[base + l * A.S] = acc;
            }
        }
    }
}

template <typename R>
cudaError_t launch_mc(const Launch &L, cplx<R> *psi, const MixedShape &m, const TOp &op, const cplx<R> *mat, int nmat) {
    MCArgs<R> A;
    std::memset(&A, 0, sizeof(A));
    A.kind = op.kind;
    A.d = m.dims[op.a];
    A.S = m.S[op.a];
    A.nfib = m.N / A.d;
    A.nc = op.nq;
    A.s = op.s;
    if (A.nc < 1 || A.nc > 6 || (op.kind != OP_MCSHIFT && op.kind != OP_MCDENSE)) return cudaErrorInvalidValue;
    for (int i = 0; i < A.nc; ++i) {
        A.cS[i] = m.S[op.q[i]];
        A.cd[i] = m.dims[op.q[i]];
        A.lv[i] = (op.mask >> (4 * i)) & 15;
    }
    if (op.kind == OP_MCDENSE) {
        if (nmat != A.d * A.d || !mat) return cudaErrorInvalidValue;
        for (int i = 0; i < nmat; ++i) A.V[i] = mat[i];
    }
    long long blocks = (A.nfib + 255) / 256;
    const long long cap = (long long)L.num_sms * 16;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    k_mc<R><<<(unsigned)blocks, 256, 0, L.stream>>>(psi, A);
    return cudaGetLastError();
}

MixedShape uniform_shape(int d, int n) {
    int dims[kMaxQudits];
    for (int q = 0; q < n; ++q) dims[q] = d;
    return mixed_shape(dims, n);
}

template cudaError_t launch_mc<float>(const Launch &, cplx<float> *, const MixedShape &, const TOp &, const cplx<float> *,
                                      int);
template cudaError_t launch_mc<double>(const Launch &, cplx<double> *, const MixedShape &, const TOp &,
                                       const cplx<double> *, int);

// ------------------------------------------------------------------ row / column reductions
constexpr int kRowMax = 512;                 // B <= 512: at most 16 columns per lane
constexpr int kColSlots = kRowMax / 32;
constexpr int kMixedBlock = 256;
constexpr int kFlushRows = 32;               // FP32 column sums cover at most this many rows

struct RowCol {
    int n, nh;                       // qudits; high qudits (spelled by the row index)
    int B;                           // row length
    long long H;                     // rows
    int wide;                        // H >= 2^32: 64-bit row digits
    int dims[kMaxQudits];
    long long hdiv[kMaxQudits];      // high qudit q: digit = (h / hdiv[q]) % dims[q]
    FastDiv hfd[kMaxQudits];
    int cdiv[kMaxQudits];            // low qudit q: digit = (c / cdiv[q]) % dims[q]
    double w[kMaxQudits];            // observable weights (k_number_obs_mixed)
};

__device__ __forceinline__ int row_digit(const RowCol &M, long long h, int q) {
    if (M.wide) return (int)((unsigned long long)h / (unsigned long long)M.hdiv[q] % (unsigned long long)M.dims[q]);
    return (int)(M.hfd[q].div((uint32_t)h) % (uint32_t)M.dims[q]);
}

__device__ __forceinline__ double warp_sum_m(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// partials: one row of n + 1 doubles per CTA (<N_q> for q < n, then the norm).
template <typename R>
__global__ void __launch_bounds__(kMixedBlock) k_expect_mixed(const cplx<R> *__restrict__ psi,
                                                               const __grid_constant__ RowCol M, double *partials) {
    __shared__ double wacc[kMixedBlock / 32][kMaxQudits + 1];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const long long gw = (long long)blockIdx.x * (kMixedBlock / 32) + wid;
    const long long nw = (long long)gridDim.x * (kMixedBlock / 32);
    R colf[kColSlots];
    double cold[kColSlots];
#pragma unroll
    for (int k = 0; k < kColSlots; ++k) { colf[k] = 0; cold[k] = 0.0; }
    double hacc0 = 0.0, hacc1 = 0.0;   // high qudits lane and lane + 32
    int batch = 0;
    for (long long h = gw; h < M.H; h += nw) {
        const cplx<R> *row = psi + h * M.B;
        R rp = 0;
#pragma unroll
        for (int k = 0; k < kColSlots; ++k) {
            const int c = lane + 32 * k;
            if (c < M.B) {
                const cplx<R> v = row[c];
                const R p = v.x * v.x + v.y * v.y;
                colf[k] += p;
                rp += p;
            }
        }
        const double P = warp_sum_m((double)rp);
        if (lane < M.nh) hacc0 += (double)row_digit(M, h, lane) * P;
        if (lane + 32 < M.nh) hacc1 += (double)row_digit(M, h, lane + 32) * P;
        if (++batch == kFlushRows) {
#pragma unroll
            for (int k = 0; k < kColSlots; ++k) { cold[k] += (double)colf[k]; colf[k] = 0; }
            batch = 0;
        }
    }
#pragma unroll
    for (int k = 0; k < kColSlots; ++k) cold[k] += (double)colf[k];
    // low qudits: sum over this lane's columns of digit_q(c) * Q_c
    for (int q = M.nh; q <= M.n; ++q) {
        double s = 0.0;
#pragma unroll
        for (int k = 0; k < kColSlots; ++k) {
            const int c = lane + 32 * k;
            if (c < M.B) s += (q == M.n ? 1.0 : (double)((c / M.cdiv[q]) % M.dims[q])) * cold[k];
        }
        s = warp_sum_m(s);
        if (lane == 0) wacc[wid][q] = s;
    }
    if (lane < M.nh) wacc[wid][lane] = hacc0;
    if (lane + 32 < M.nh) wacc[wid][lane + 32] = hacc1;
    __syncthreads();
    for (int q = threadIdx.x; q <= M.n; q += blockDim.x) {
        double s = 0.0;
        for (int w = 0; w < kMixedBlock / 32; ++w) s += wacc[w][q];
        partials[(long long)blockIdx.x * (M.n + 1) + q] = s;
    }
}

// lambda_i = (sum_q w_q i_q) psi_i; partials: one loss partial per CTA.
template <typename R>
__global__ void __launch_bounds__(kMixedBlock) k_number_obs_mixed(const cplx<R> *__restrict__ psi, cplx<R> *__restrict__ lam,
                                                                   const __grid_constant__ RowCol M, double *partials) {
    __shared__ double wl[kMixedBlock / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const long long gw = (long long)blockIdx.x * (kMixedBlock / 32) + wid;
    const long long nw = (long long)gridDim.x * (kMixedBlock / 32);
    // weight of each of this lane's columns (low digits)
    R wc[kColSlots];
#pragma unroll
    for (int k = 0; k < kColSlots; ++k) {
        const int c = lane + 32 * k;
        double s = 0.0;
        if (c < M.B)
            for (int q = M.nh; q < M.n; ++q) s += M.w[q] * (double)((c / M.cdiv[q]) % M.dims[q]);
        wc[k] = (R)s;
    }
    double loss = 0.0;
    for (long long h = gw; h < M.H; h += nw) {
        double wh = 0.0;
        if (lane < M.nh) wh += M.w[lane] * (double)row_digit(M, h, lane);
        if (lane + 32 < M.nh) wh += M.w[lane + 32] * (double)row_digit(M, h, lane + 32);
        wh = warp_sum_m(wh);
        const cplx<R> *row = psi + h * M.B;
        cplx<R> *lrow = lam + h * M.B;
        R lr = 0;
#pragma unroll
        for (int k = 0; k < kColSlots; ++k) {
            const int c = lane + 32 * k;
            if (c < M.B) {
                const cplx<R> v = row[c];
                const R wt = (R)wh + wc[k];
                lrow[c] = mk<R>(wt * v.x, wt * v.y);
                lr += wt * (v.x * v.x + v.y * v.y);
            }
        }
        loss += (double)lr;
    }
    loss = warp_sum_m(loss);
    if (lane == 0) wl[wid] = loss;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < kMixedBlock / 32; ++w) s += wl[w];
        partials[blockIdx.x] = s;
    }
}

__global__ void k_sum_rows_mixed(const double *partials, int rows, int cols, double *out) {
    for (int c = threadIdx.x; c < cols; c += blockDim.x) {
        double s = 0.0;
        for (int r = 0; r < rows; ++r) s += partials[(long long)r * cols + c];
        out[c] = s;
    }
}

static RowCol row_col(const MixedShape &m) {
    RowCol M;
    std::memset(&M, 0, sizeof(M));
    M.n = m.n;
    // lowest qudits whose dims multiply to at most kRowMax
    int nl = 0;
    long long B = 1;
    while (nl < m.n && B * m.dims[m.n - 1 - nl] <= kRowMax) {
        B *= m.dims[m.n - 1 - nl];
        ++nl;
    }
    M.nh = m.n - nl;
    M.B = (int)B;
    M.H = m.N / B;
    M.wide = M.H >= (1ll << 32) ? 1 : 0;
    for (int q = 0; q < m.n; ++q) {
        M.dims[q] = m.dims[q];
        if (q < M.nh) {
            M.hdiv[q] = m.S[q] / B;
            M.hfd[q] = FastDiv(M.wide ? 1u : (uint32_t)M.hdiv[q]);
        } else {
            M.cdiv[q] = (int)m.S[q];
        }
    }
    return M;
}

static int rows_grid(const Launch &L, long long H) {
    const long long warps = kMixedBlock / 32;
    long long b = (H + warps - 1) / warps;
    const long long cap = reduce_max_blocks(L.num_sms);
    if (b > cap) b = cap;
    return (int)(b < 1 ? 1 : b);
}

template <typename R>
cudaError_t launch_expect_mixed(const Launch &L, const cplx<R> *psi, const MixedShape &m, double *partials,
                                double *out_dev) {
    const RowCol M = row_col(m);
    const int blocks = rows_grid(L, M.H);
    k_expect_mixed<R><<<blocks, kMixedBlock, 0, L.stream>>>(psi, M, partials);
    k_sum_rows_mixed<<<1, 64, 0, L.stream>>>(partials, blocks, m.n + 1, out_dev);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_number_obs_mixed(const Launch &L, const cplx<R> *psi, cplx<R> *lam, const MixedShape &m,
                                    const double *w, double *partials, double *loss_dev) {
    RowCol M = row_col(m);
    for (int q = 0; q < m.n; ++q) M.w[q] = w[q];
    const int blocks = rows_grid(L, M.H);
    k_number_obs_mixed<R><<<blocks, kMixedBlock, 0, L.stream>>>(psi, lam, M, partials);
    k_sum_rows_mixed<<<1, 32, 0, L.stream>>>(partials, blocks, 1, loss_dev);
    return cudaGetLastError();
}

MixedShape mixed_shape(const int *dims, int n) {
    MixedShape m;
    m.n = n;
    long long N = 1;
    for (int q = n - 1; q >= 0; --q) {
        m.dims[q] = dims[q];
        m.S[q] = N;
        N *= dims[q];
    }
    m.N = N;
    return m;
}

StridedGeom mixed_geom(const MixedShape &m, const TOp &op) {
    StridedGeom g;
    g.d = m.dims[op.a];
    g.S = m.S[op.a];
    g.H = m.N / (g.d * g.S);
    const bool ctrl = op.kind == OP_CPAIR || op.kind == OP_CDIAG || op.kind == OP_CSHIFT;
    g.dc = ctrl ? m.dims[op.c] : g.d;
    g.Sc = ctrl ? m.S[op.c] : 1;
    g.c_above = ctrl && op.c < op.a;
    return g;
}

// One resolved op on a mixed state: strided kinds with their entries inline
// (`mat`, rounded to R), group kinds from the device copy `mat_dev`.
template <typename R>
cudaError_t mixed_launch(const Launch &L, cplx<R> *psi, const MixedShape &m, const TOp &o, const cplx<R> *mat, int nmat,
                         const cplx<R> *mat_dev) {
    if ((o.kind == OP_SHIFT && o.s == 0) || (o.kind == OP_DIAG && o.mask == 0)) return cudaSuccess;   // identity
    if (is_single(o) || is_controlled(o)) return launch_strided_g<R>(L, psi, mixed_geom(m, o), o, mat, nmat);
    if (is_mc(o)) return o.kind == OP_MCSHIFT && o.s == 0 ? cudaSuccess : launch_mc<R>(L, psi, m, o, mat, nmat);
    return launch_group<R>(L, psi, m, o, mat_dev);
}

// One reverse step of the adjoint sweep on a mixed state: `o`, `mat`,
// `mat_dev` describe U^+; `gen` (nullptr: not parametrised) the generator;
// rows receives mixed_adj_rows() gradient partials.
template <typename R>
cudaError_t mixed_adj_launch(const Launch &L, cplx<R> *psi, cplx<R> *lam, const MixedShape &m, const TOp &o,
                             const cplx<R> *mat, int nmat, const cplx<R> *mat_dev, const cplx<R> *gen, int ngen,
                             double *rows) {
    if (is_single(o) || is_controlled(o))
        return launch_strided_adj<R>(L, psi, lam, mixed_geom(m, o), o, mat, nmat, gen, ngen, rows);
    if (is_mc(o)) {
        if (o.kind == OP_MCSHIFT && o.s == 0) return cudaSuccess;
        cudaError_t e = launch_mc<R>(L, psi, m, o, mat, nmat);
        if (e != cudaSuccess) return e;
        return launch_mc<R>(L, lam, m, o, mat, nmat);
    }
    cudaError_t e = launch_group<R>(L, psi, m, o, mat_dev);
    if (e != cudaSuccess) return e;
    return launch_group<R>(L, lam, m, o, mat_dev);
}

long long mixed_adj_rows(const MixedShape &m, const TOp &o, int num_sms) {
    if (is_single(o) || is_controlled(o)) return strided_adj_blocks(mixed_geom(m, o), num_sms);
    return 0;
}

template cudaError_t mixed_launch<float>(const Launch &, cplx<float> *, const MixedShape &, const TOp &,
                                         const cplx<float> *, int, const cplx<float> *);
template cudaError_t mixed_launch<double>(const Launch &, cplx<double> *, const MixedShape &, const TOp &,
                                          const cplx<double> *, int, const cplx<double> *);
template cudaError_t mixed_adj_launch<float>(const Launch &, cplx<float> *, cplx<float> *, const MixedShape &,
                                             const TOp &, const cplx<float> *, int, const cplx<float> *,
                                             const cplx<float> *, int, double *);
template cudaError_t mixed_adj_launch<double>(const Launch &, cplx<double> *, cplx<double> *, const MixedShape &,
                                              const TOp &, const cplx<double> *, int, const cplx<double> *,
                                              const cplx<double> *, int, double *);
template cudaError_t launch_group<float>(const Launch &, cplx<float> *, const MixedShape &, const TOp &,
                                         const cplx<float> *);
template cudaError_t launch_group<double>(const Launch &, cplx<double> *, const MixedShape &, const TOp &,
                                          const cplx<double> *);
template cudaError_t launch_expect_mixed<float>(const Launch &, const cplx<float> *, const MixedShape &, double *, double *);
template cudaError_t launch_expect_mixed<double>(const Launch &, const cplx<double> *, const MixedShape &, double *,
                                                 double *);
template cudaError_t launch_number_obs_mixed<float>(const Launch &, const cplx<float> *, cplx<float> *,
                                                    const MixedShape &, const double *, double *, double *);
template cudaError_t launch_number_obs_mixed<double>(const Launch &, const cplx<double> *, cplx<double> *,
                                                     const MixedShape &, const double *, double *, double *);

}  // namespace qf
