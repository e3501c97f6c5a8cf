// k_adjoint.cu -- adjoint (reverse-mode) gradient of L = sum_q w_q <N_q>.
//
// With psi_l the state after gate l and U_l = exp(-i theta_l G_l), the costate
// lambda_L = O psi_L (O = sum_q w_q N_q, diagonal) is carried backwards with the
// state: for l = L .. 1
//     g_l        = 2 Im <lambda_l | G_l | psi_l>      (dU/dtheta = -i G U)
//     psi_{l-1}  = U_l^+ psi_l,   lambda_{l-1} = U_l^+ lambda_l
// so the state is uncomputed by unitarity instead of being stored per layer.
// G is S/2 for a rotation exp(-i theta S / 2) (Appendix B, "Generalized
// rotation gate") and sum_m |m><m| (x) m S/2 for the controlled rotation
// ("Controlled Rotation Gate"), whose angle is scaled by the control level.
//
// Kernels:
//   k_number_obs     lambda = O psi and the loss <psi|O|psi> in one pass
//   k_tile_adj       one reverse pass: psi and lambda tiles in shared memory,
//                    each gate of the pass (in reverse) adds its gradient
//                    term, then U^+ is applied to both tiles
//   k_grad_gather    per parameter slot, sums its terms over passes and CTAs
//                    in a fixed order (deterministic)
#include "stage_device.cuh"

namespace qf {

// ------------------------------------------------------------------ lambda = O psi
template <int D> struct ObsCfg;
template <> struct ObsCfg<2> { static constexpr int A = 8, B = 4; };
template <> struct ObsCfg<3> { static constexpr int A = 5, B = 2; };
template <> struct ObsCfg<4> { static constexpr int A = 4, B = 2; };
template <> struct ObsCfg<5> { static constexpr int A = 3, B = 2; };
template <> struct ObsCfg<6> { static constexpr int A = 3, B = 1; };
template <> struct ObsCfg<7> { static constexpr int A = 3, B = 1; };
template <> struct ObsCfg<8> { static constexpr int A = 3, B = 1; };

constexpr int ipow_k(int d, int e) { return e == 0 ? 1 : d * ipow_k(d, e - 1); }

struct ObsArgs {
    double w[kMaxQudits + 1];   // weights of N_q
};

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ double block_sum_d(double v, double *red) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
    v = warp_sum_d(v);
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    if (wid == 0) {
        double s = lane < nw ? red[lane] : 0.0;
        s = warp_sum_d(s);
        if (lane == 0) red[32] = s;
    }
    __syncthreads();
    return red[32];
}

// Chunks of d^(A+B) amplitudes; a CTA of d^A threads; thread t reads t + d^A u.
// The weight sum of an amplitude's digits splits into a per-thread part (low A
// digits), a per-u part (next B digits, compile-time digits) and a per-chunk
// part (the remaining high digits).
template <typename R, int D>
__global__ void __launch_bounds__(ipow_k(D, ObsCfg<D>::A)) k_number_obs(const cplx<R> *__restrict__ psi,
                                                                       cplx<R> *__restrict__ lam, int n,
                                                                       long long nchunks, const __grid_constant__ ObsArgs W,
                                                                       double *partials) {
    constexpr int A = ObsCfg<D>::A, B = ObsCfg<D>::B;
    constexpr int BLK = ipow_k(D, A), U = ipow_k(D, B), CH = BLK * U;
    __shared__ double red[33];
    const int tid = threadIdx.x;
    const int nh = n - A - B;
    R sl = 0;
    {
        int t = tid;
        for (int r = 0; r < A; ++r) {
            sl += (R)(t % D) * (R)W.w[n - 1 - r];
            t /= D;
        }
    }
    R wb[B];
#pragma unroll
    for (int r = 0; r < B; ++r) wb[r] = (R)W.w[n - 1 - A - r];
    double loss = 0.0;
    for (long long c = blockIdx.x; c < nchunks; c += gridDim.x) {
        R sh = 0;
        long long cc = c;
        for (int q = nh - 1; q >= 0; --q) {
            sh += (R)(cc % D) * (R)W.w[q];
            cc /= D;
        }
        const R base = sl + sh;
        const long long off = c * CH + tid;
        R lc = 0;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            R o = base;
#pragma unroll
            for (int r = 0; r < B; ++r) {
                int pw = 1;
#pragma unroll
                for (int s = 0; s < r; ++s) pw *= D;
                const int dig = (u / pw) % D;
                if (dig) o += (R)dig * wb[r];
            }
            cplx<R> v = psi[off + u * BLK];
            lc += o * (v.x * v.x + v.y * v.y);
            lam[off + u * BLK] = mk<R>(o * v.x, o * v.y);
        }
        loss += (double)lc;
    }
    double s = block_sum_d(loss, red);
    if (tid == 0) partials[blockIdx.x] = s;
}

template <typename R>
__global__ void __launch_bounds__(256) k_number_obs_generic(const cplx<R> *__restrict__ psi, cplx<R> *__restrict__ lam,
                                                             int d, int n, long long N, const __grid_constant__ ObsArgs W,
                                                             double *partials) {
    __shared__ double red[33];
    double loss = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        double o = 0.0;
        long long rem = i;
        for (int q = n - 1; q >= 0; --q) {
            long long nx = rem / d;
            o += (double)(rem - nx * d) * W.w[q];
            rem = nx;
        }
        cplx<R> v = psi[i];
        loss += o * ((double)v.x * v.x + (double)v.y * v.y);
        lam[i] = mk<R>((R)(o * v.x), (R)(o * v.y));
    }
    double s = block_sum_d(loss, red);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

__global__ void k_sum_rows(const double *partials, int rows, double *out) {
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int r = 0; r < rows; ++r) s += partials[r];
        *out = s;
    }
}

// lambda = O psi, loss -> *loss_dev.  partials holds >= 2*SMs doubles.
template <typename R>
cudaError_t launch_number_obs(const Launch &L, const cplx<R> *psi, cplx<R> *lam, int d, int n, const double *w,
                              double *partials, double *loss_dev) {
    ObsArgs W;
    for (int q = 0; q <= kMaxQudits; ++q) W.w[q] = q < n ? w[q] : 0.0;
    long long N = 1;
    for (int i = 0; i < n; ++i) N *= d;
    const int maxb = 2 * L.num_sms;
    int blocks = 0;
    switch (d) {
#define QF_CASE(DD)                                                                                   \
    case DD: {                                                                                        \
        constexpr int CH = ipow_k(DD, ObsCfg<DD>::A + ObsCfg<DD>::B);                                 \
        if (n >= ObsCfg<DD>::A + ObsCfg<DD>::B) {                                                     \
            long long nch = N / CH;                                                                   \
            blocks = (int)(nch < maxb ? nch : maxb);                                                  \
            k_number_obs<R, DD><<<blocks, ipow_k(DD, ObsCfg<DD>::A), 0, L.stream>>>(psi, lam, n, nch, W, \
                                                                                   partials);         \
        }                                                                                             \
        break;                                                                                        \
    }
        QF_CASE(2) QF_CASE(3) QF_CASE(4) QF_CASE(5) QF_CASE(6) QF_CASE(7) QF_CASE(8)
#undef QF_CASE
    default:
        break;
    }
    if (blocks == 0) {
        long long b = (N + 255) / 256;
        blocks = (int)(b < maxb ? b : maxb);
        k_number_obs_generic<R><<<blocks, 256, 0, L.stream>>>(psi, lam, d, n, N, W, partials);
    }
    k_sum_rows<<<1, 32, 0, L.stream>>>(partials, blocks, loss_dev);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ reverse tile pass
template <typename R>
struct AdjArgs {
    cplx<R> *psi;
    cplx<R> *lam;
    TileGeom g;
    int nops;          // ops in application order (already reversed by the host, with U^+ entries)
    int nmat;
    const TOp *ops;
    const cplx<R> *mats;
    const TStage *stages;   // register stages (nstages > 0), else one op per shared-memory sweep
    int nstages;
    double *rows;      // gradient rows: gridDim.x rows of ncols doubles
    int ncols;
};

constexpr int kAdjWarps = kTileBlock / 32;

// Gradient term Im <lambda_f | G | psi_f> of one fibre (before U^+ is applied).
template <typename R, int D>
__device__ __forceinline__ R fibre_grad(const cplx<R> *p, const cplx<R> *q, int ls, const TOp &op, const cplx<R> *G,
                                        int ctl, int d) {
    constexpr int DM = D > 0 ? D : kMaxD;
    R acc = 0;
    const bool ctrl = op.kind == OP_CPAIR || op.kind == OP_CDIAG;
    if (ctrl && ctl == 0) return 0;
    if (op.kind == OP_PAIR || op.kind == OP_CPAIR) {
        const cplx<R> a = p[op.j * ls], b = p[op.k * ls];
        const cplx<R> la = q[op.j * ls], lb = q[op.k * ls];
        // G a-column products
        cplx<R> ga = cfma(G[1], b, cmul(G[0], a));
        cplx<R> gb = cfma(G[3], b, cmul(G[2], a));
        // Im(conj(la) ga + conj(lb) gb)
        acc = la.x * ga.y - la.y * ga.x + lb.x * gb.y - lb.y * gb.x;
    } else {
#pragma unroll
        for (int l = 0; l < DM; ++l)
            if (l < d && ((op.mask >> l) & 1)) {
                const cplx<R> a = p[l * ls], la = q[l * ls];
                // G diagonal entries are real
                acc += G[l].x * (la.x * a.y - la.y * a.x);
            }
    }
    return ctrl ? acc * (R)ctl : acc;
}

template <typename R, int D>
__global__ void __launch_bounds__(kTileBlock) k_tile_adj(const __grid_constant__ AdjArgs<R> A, int d_rt) {
    using C = cplx<R>;
    extern __shared__ __align__(16) unsigned char smem[];
    const int d = D > 0 ? D : d_rt;
    const TileGeom &g = A.g;
    const int T = g.T;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int nA = T / g.SEG;

    // layout: psi tile | lambda tile | pool | ops | stages | pad 16 | gacc | offA | base
    C *tp = reinterpret_cast<C *>(smem);
    C *tl = tp + T;
    C *mats = tl + T;
    TOp *ops = reinterpret_cast<TOp *>(mats + A.nmat);
    TStage *stages = reinterpret_cast<TStage *>(ops + A.nops);
    size_t off = (size_t)2 * T * sizeof(C) + (size_t)A.nmat * sizeof(C) + (size_t)A.nops * sizeof(TOp) +
                 (size_t)A.nstages * sizeof(TStage);
    off = (off + 15) & ~(size_t)15;
    double *gacc = reinterpret_cast<double *>(smem + off);
    long long *offA = reinterpret_cast<long long *>(gacc + (size_t)A.nops * kAdjWarps);
    long long *sbase = offA + nA;
    float4 *prep = reinterpret_cast<float4 *>(
        smem + ((off + (size_t)A.nops * kAdjWarps * sizeof(double) + (size_t)(nA + 1) * sizeof(long long) + 15) &
                ~(size_t)15));

    for (int i = tid; i < A.nmat; i += kTileBlock) mats[i] = A.mats[i];
    {
        const int *src = reinterpret_cast<const int *>(A.ops);
        int *dst = reinterpret_cast<int *>(ops);
        const int words = A.nops * (int)(sizeof(TOp) / sizeof(int));
        for (int i = tid; i < words; i += kTileBlock) dst[i] = src[i];
    }
    if (A.nstages > 0) {
        const int *src = reinterpret_cast<const int *>(A.stages);
        int *dst = reinterpret_cast<int *>(stages);
        const int words = A.nstages * (int)(sizeof(TStage) / sizeof(int));
        for (int i = tid; i < words; i += kTileBlock) dst[i] = src[i];
    }
    for (int i = tid; i < A.nops * kAdjWarps; i += kTileBlock) gacc[i] = 0.0;
    R gsum[kMaxGrad];   // register-stage gradient accumulators, by gradient column
#pragma unroll
    for (int c = 0; c < kMaxGrad; ++c) gsum[c] = 0;
    for (int a = tid; a < nA; a += kTileBlock) {
        long long o = 0;
        int rem = a;
        for (int i = g.kA - 1; i >= 0; --i) {
            o += (long long)(rem % d) * g.strideA[i];
            rem /= d;
        }
        offA[a] = o;
    }
    if (tid == 0) sbase[0] = tile_base(g, blockIdx.x);
    __syncthreads();
    if (A.nstages > 0) prepare_pool<R>(mats, prep, A.nmat);
    const int a0 = (int)g.divSEG.div((uint32_t)tid), lo0 = tid - a0 * g.SEG;
    const int da = (int)g.divSEG.div((uint32_t)kTileBlock), dl = kTileBlock - da * g.SEG;

    for (long long t = blockIdx.x; t < g.ntiles; t += gridDim.x) {
        const long long base = sbase[0];
        for (int e = tid, a = a0, lo = lo0; e < T; e += kTileBlock) {
            const long long gi = base + offA[a] + lo;
            cp_async_amp<R>(tp + e, A.psi + gi);
            cp_async_amp<R>(tl + e, A.lam + gi);
            lo += dl;
            a += da;
            if (lo >= g.SEG) { lo -= g.SEG; ++a; }
        }
        cp_async_wait_all();
        __syncthreads();
        if constexpr (StageK<R, D, true>::K > 0) {
            if (A.nstages > 0) {
                for (int si = 0; si < A.nstages; ++si) {
                    const TStage &st = stages[si];
                    if (!st.legacy) {
                        stage_run<R, D, StageK<R, D, true>::K, true>(st, ops, mats, prep, tp, tl, T, gsum);
                    } else {
                        // SWAP / custom gates: no angle
                        tile_apply<R, D>(ops[st.first], tp, mats, T, g.nt, d);
                        tile_apply<R, D>(ops[st.first], tl, mats, T, g.nt, d);
                    }
                    __syncthreads();
                }
                goto store;
            }
        }
        for (int o = 0; o < A.nops; ++o) {
            const TOp &op = ops[o];
            const C *M = mats + op.mat;
            if (op.gcol >= 0) {
                // gradient term of this gate, from psi_l and lambda_l
                const C *G = mats + op.gmat;
                const int ls = op.lsa;
                const int F = T / d;
                const bool ctrl = op.kind == OP_CPAIR || op.kind == OP_CDIAG;
                R part = 0;
                for (int f = tid; f < F; f += kTileBlock) {
                    int hi = (int)op.fa.div((uint32_t)f);
                    int b = hi * d * ls + (f - hi * ls);
                    int ctl = ctrl ? dmod<D>(op.fc.div((uint32_t)b), d) : 0;
                    part += fibre_grad<R, D>(tp + b, tl + b, ls, op, G, ctl, d);
                }
                double v = warp_sum_d((double)part);
                if (lane == 0) gacc[o * kAdjWarps + wid] += v;
                // no barrier: U^+ below updates, in each thread, exactly the
                // fibres this thread has just read
            }
            tile_apply<R, D>(op, tp, mats, T, g.nt, d);
            tile_apply<R, D>(op, tl, mats, T, g.nt, d);
            __syncthreads();
            (void)M;
        }
    store:
        for (int e = tid, a = a0, lo = lo0; e < T; e += kTileBlock) {
            const long long gi = base + offA[a] + lo;
            A.psi[gi] = tp[e];
            A.lam[gi] = tl[e];
            lo += dl;
            a += da;
            if (lo >= g.SEG) { lo -= g.SEG; ++a; }
        }
        if (tid == 0 && t + gridDim.x < g.ntiles) sbase[0] = tile_base(g, t + gridDim.x);
        __syncthreads();
    }
    // register-stage accumulators: reduce per column into gacc[col * warps + warp]
    if (A.nstages > 0 && StageK<R, D, true>::K > 0) {
        __syncthreads();
        for (int i = tid; i < A.nops * kAdjWarps; i += kTileBlock) gacc[i] = 0.0;
        __syncthreads();
#pragma unroll
        for (int c = 0; c < kMaxGrad; ++c) {
            if (c >= A.ncols) break;
            const double v = warp_sum_d((double)gsum[c]);
            if (lane == 0) gacc[c * kAdjWarps + wid] = v;
        }
        __syncthreads();
        for (int c = tid; c < A.ncols; c += kTileBlock) {
            double s2 = 0.0;
            for (int w = 0; w < kAdjWarps; ++w) s2 += gacc[c * kAdjWarps + w];
            A.rows[(long long)blockIdx.x * A.ncols + c] = 2.0 * s2;
        }
        return;
    }
    // this CTA's gradient row
    for (int o = tid; o < A.nops; o += kTileBlock) {
        const TOp &op = ops[o];
        if (op.gcol < 0) continue;
        double s = 0.0;
        for (int w = 0; w < kAdjWarps; ++w) s += gacc[o * kAdjWarps + w];
        A.rows[(long long)blockIdx.x * A.ncols + op.gcol] = 2.0 * s;
    }
}

template <typename R>
size_t adj_smem_bytes(const TileGeom &g, int nops, int nmat, int nstages) {
    size_t b = (size_t)2 * g.T * sizeof(cplx<R>) + (size_t)nmat * sizeof(cplx<R>) + (size_t)nops * sizeof(TOp) +
               (size_t)nstages * sizeof(TStage);
    b = (b + 15) & ~(size_t)15;
    b += (size_t)nops * kAdjWarps * sizeof(double);
    b += (size_t)(g.T / g.SEG + 1) * sizeof(long long);
    b = (b + 15) & ~(size_t)15;
    b += (size_t)nmat * sizeof(float4);   // prepared entries (complex64 register stages)
    return b;
}

template <typename R, int D>
static cudaError_t adj_grid_d(int num_sms, const TileGeom &g, size_t smem, int *grid) {
    static int configured = 0;
    if ((int)smem > configured) {
        cudaError_t e = cudaFuncSetAttribute(k_tile_adj<R, D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured = (int)smem;
    }
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tile_adj<R, D>, kTileBlock, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    long long gr = (long long)per_sm * num_sms;
    if (gr > g.ntiles) gr = g.ntiles;
    *grid = (int)gr;
    return cudaSuccess;
}

// Grid the reverse pass will use (the host sizes gradient rows with it).
template <typename R>
cudaError_t adj_grid(int num_sms, int d, const TileGeom &g, int nops, int nmat, int nstages, int *grid) {
    size_t smem = adj_smem_bytes<R>(g, nops, nmat, nstages);
    switch (d) {
#define QF_CASE(DD) case DD: return adj_grid_d<R, DD>(num_sms, g, smem, grid);
        QF_CASE(2) QF_CASE(3) QF_CASE(4) QF_CASE(5) QF_CASE(6) QF_CASE(7) QF_CASE(8)
#undef QF_CASE
    default: return adj_grid_d<R, 0>(num_sms, g, smem, grid);
    }
}

template <typename R>
cudaError_t launch_tile_adj(const Launch &L, cplx<R> *psi, cplx<R> *lam, int d, const TileGeom &g, int nops,
                            const TOp *ops_dev, const cplx<R> *mat_dev, int nmat, const TStage *stages_dev,
                            int nstages, double *rows, int ncols, int grid) {
    AdjArgs<R> A;
    A.psi = psi;
    A.lam = lam;
    A.g = g;
    A.nops = nops;
    A.nmat = nmat;
    A.ops = ops_dev;
    A.mats = mat_dev;
    A.rows = rows;
    A.ncols = ncols;
    A.stages = stages_dev;
    A.nstages = stages_dev ? nstages : 0;
    size_t smem = adj_smem_bytes<R>(g, nops, nmat, A.nstages);
    switch (d) {
#define QF_CASE(DD) case DD: k_tile_adj<R, DD><<<grid, kTileBlock, smem, L.stream>>>(A, d); break;
        QF_CASE(2) QF_CASE(3) QF_CASE(4) QF_CASE(5) QF_CASE(6) QF_CASE(7) QF_CASE(8)
#undef QF_CASE
    default: k_tile_adj<R, 0><<<grid, kTileBlock, smem, L.stream>>>(A, d); break;
    }
    return cudaGetLastError();
}

// ------------------------------------------------------------------ gather
// Term c of slot s is rows[base[c] + b * ncols[c] + col[c]] for b < nrows[c];
// slot s owns terms first[s] .. first[s+1]-1.
struct GatherTerm {
    long long base;
    int nrows, ncols, col, pad;
};

__global__ void k_grad_gather(const double *rows, const GatherTerm *terms, const int *first, int nslots, double *grad) {
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < nslots; s += gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int c = first[s]; c < first[s + 1]; ++c) {
            const GatherTerm t = terms[c];
            for (int b = 0; b < t.nrows; ++b) acc += rows[t.base + (long long)b * t.ncols + t.col];
        }
        grad[s] = acc;
    }
}

cudaError_t launch_grad_gather(const Launch &L, const double *rows, const void *terms, const int *first, int nslots,
                               double *grad) {
    if (nslots <= 0) return cudaSuccess;
    int blocks = (nslots + 127) / 128;
    k_grad_gather<<<blocks, 128, 0, L.stream>>>(rows, reinterpret_cast<const GatherTerm *>(terms), first, nslots, grad);
    return cudaGetLastError();
}

size_t gather_term_bytes() { return sizeof(GatherTerm); }

template cudaError_t launch_number_obs<float>(const Launch &, const cplx<float> *, cplx<float> *, int, int,
                                              const double *, double *, double *);
template cudaError_t launch_number_obs<double>(const Launch &, const cplx<double> *, cplx<double> *, int, int,
                                               const double *, double *, double *);
template cudaError_t adj_grid<float>(int, int, const TileGeom &, int, int, int, int *);
template cudaError_t adj_grid<double>(int, int, const TileGeom &, int, int, int, int *);
template cudaError_t launch_tile_adj<float>(const Launch &, cplx<float> *, cplx<float> *, int, const TileGeom &, int,
                                            const TOp *, const cplx<float> *, int, const TStage *, int, double *, int,
                                            int);
template cudaError_t launch_tile_adj<double>(const Launch &, cplx<double> *, cplx<double> *, int, const TileGeom &, int,
                                             const TOp *, const cplx<double> *, int, const TStage *, int, double *, int,
                                             int);

}  // namespace qf
