// k_batch.cu -- many independent circuits of uneven size in each launch.
//
// The circuits of one qudit dimension d share launches: launch k runs the k-th
// pass of every circuit that has one.  Its work items are (circuit pass, chunk
// of consecutive tiles); a persistent CTA walks the items, stages the pass's
// op list and matrix pool into shared memory when the item belongs to a new
// pass, and runs each tile as the single-circuit kernels do (load with
// cp.async, apply every op, store).  Rotation entries of parametrised gates
// are computed on the device from the parameter vector by one kernel at the
// start of each run (Appendix B, "Generalized rotation gate": R = exp(-i theta
// S / 2); the controlled rotation uses R(m theta) for control level m), so a
// launch sequence captured once in a CUDA graph serves every parameter update.
// The
// adjoint variant carries psi and lambda tiles and writes one gradient row per
// work item (the per-gate terms 2 Im <lambda|G|psi> of its tiles).
#include "stage_device.cuh"

namespace qf {

struct BPass {
    long long psi_off, lam_off;   // element offsets of the circuit's states
    TileGeom g;
    int ops_off, nops;            // op table slice
    int mat_off, nmat;            // pool slice
    int ncols;                    // adjoint gradient columns
    int chunks;                   // work items of this pass
    long long rows_base;          // adjoint gradient rows (chunks rows of ncols)
    int stages_off, nstages;      // register stages (nstages = 0: one op per shared-memory sweep)
};

template <typename R>
struct BatchArgs {
    cplx<R> *states;
    const BPass *passes;
    const long long *prefix;      // npasses + 1 item prefix sums
    int npasses;
    const TOp *ops;
    const cplx<R> *pool;
    const TStage *stages;
    const double *params;
    double *rows;
    int chunk_tiles;
    int max_T, max_nmat, max_nops, max_nA, max_nstages;
};

constexpr int kBatchWarps = kTileBlock / 32;

// Rotation entries at angle th: PAIR layout (jj, jk, kj, kk) for x/y, d
// diagonal entries for z (level pair) and g (Gell-Mann S_z^j).
template <typename R>
__device__ void rot_entries_dev(int d, int j, int k, int axis, double th, cplx<R> *out) {
    double s, c;
    sincos(0.5 * th, &s, &c);
    if (axis == 'x') {
        out[0] = mk<R>((R)c, 0); out[1] = mk<R>(0, (R)-s); out[2] = mk<R>(0, (R)-s); out[3] = mk<R>((R)c, 0);
        return;
    }
    if (axis == 'y') {
        out[0] = mk<R>((R)c, 0); out[1] = mk<R>((R)-s, 0); out[2] = mk<R>((R)s, 0); out[3] = mk<R>((R)c, 0);
        return;
    }
    for (int l = 0; l < d; ++l) out[l] = mk<R>(1, 0);
    if (axis == 'z') {
        out[j] = mk<R>((R)c, (R)-s);
        out[k] = mk<R>((R)c, (R)s);
        return;
    }
    const double gam = sqrt(2.0 / ((double)j * (double)(j + 1)));
    for (int l = 0; l <= j; ++l) {
        const double v = (l < j) ? gam : -(double)j * gam;
        double sv, cv;
        sincos(-0.5 * th * v, &sv, &cv);
        out[l] = mk<R>((R)cv, (R)sv);
    }
}

template <typename R>
__device__ void resolve_param_op(const TOp &op, const double *params, int d, cplx<R> *mats) {
    const double th = (double)op.psign * params[op.pslot];
    cplx<R> *M = mats + op.mat;
    if (op.kind == OP_CPAIR || op.kind == OP_CDIAG) {
        const int per = op.kind == OP_CPAIR ? 4 : d;
        for (int m = 0; m < d; ++m) rot_entries_dev<R>(d, op.j, op.k, op.paxis, m * th, M + per * m);
    } else {
        rot_entries_dev<R>(d, op.j, op.k, op.paxis, th, M);
    }
}

__device__ __forceinline__ double warp_sum_b(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <typename R, int D>
__device__ __forceinline__ R fibre_grad_b(const cplx<R> *p, const cplx<R> *q, int ls, const TOp &op, const cplx<R> *G,
                                          int ctl, int d) {
    constexpr int DM = D > 0 ? D : kMaxD;
    const bool ctrl = op.kind == OP_CPAIR || op.kind == OP_CDIAG;
    if (ctrl && ctl == 0) return 0;
    R acc = 0;
    if (op.kind == OP_PAIR || op.kind == OP_CPAIR) {
        const cplx<R> a = p[op.j * ls], b = p[op.k * ls];
        const cplx<R> la = q[op.j * ls], lb = q[op.k * ls];
        cplx<R> ga = cfma(G[1], b, cmul(G[0], a));
        cplx<R> gb = cfma(G[3], b, cmul(G[2], a));
        acc = la.x * ga.y - la.y * ga.x + lb.x * gb.y - lb.y * gb.x;
    } else {
#pragma unroll
        for (int l = 0; l < DM; ++l)
            if (l < d && ((op.mask >> l) & 1)) {
                const cplx<R> a = p[l * ls], la = q[l * ls];
                acc += G[l].x * (la.x * a.y - la.y * a.x);
            }
    }
    return ctrl ? acc * (R)ctl : acc;
}

template <typename R, int D, bool ADJ>
__global__ void __launch_bounds__(kTileBlock) k_batch(const __grid_constant__ BatchArgs<R> A, int d_rt) {
    using C = cplx<R>;
    extern __shared__ __align__(16) unsigned char smem[];
    const int d = D > 0 ? D : d_rt;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;

    C *tp = reinterpret_cast<C *>(smem);
    C *tl = tp + A.max_T;                              // adjoint only
    C *mats = tl + (ADJ ? A.max_T : 0);
    TOp *ops = reinterpret_cast<TOp *>(mats + A.max_nmat);
    TStage *stages = reinterpret_cast<TStage *>(ops + A.max_nops);
    size_t off = (size_t)(ADJ ? 2 : 1) * A.max_T * sizeof(C) + (size_t)A.max_nmat * sizeof(C) +
                 (size_t)A.max_nops * sizeof(TOp) + (size_t)A.max_nstages * sizeof(TStage);
    off = (off + 15) & ~(size_t)15;
    double *gacc = reinterpret_cast<double *>(smem + off);
    long long *offA = reinterpret_cast<long long *>(gacc + (ADJ ? (size_t)A.max_nops * kBatchWarps : 0));
    long long *sbase = offA + A.max_nA;
    float4 *prep = reinterpret_cast<float4 *>(
        smem + ((off + (ADJ ? (size_t)A.max_nops * kBatchWarps * sizeof(double) : 0) +
                 (size_t)(A.max_nA + 1) * sizeof(long long) + 15) &
                ~(size_t)15));

    const long long total = A.prefix[A.npasses];
    int cur = -1;
    for (long long item = blockIdx.x; item < total; item += gridDim.x) {
        // pass of this item: largest k with prefix[k] <= item
        int lo = 0, hi = A.npasses - 1;
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (A.prefix[mid] <= item) lo = mid;
            else hi = mid - 1;
        }
        const int k = lo;
        const BPass &P = A.passes[k];
        const TileGeom &g = P.g;
        const int T = g.T;
        const int nA = T / g.SEG;
        if (k != cur) {
            // stage the pass (every thread is past the previous tile's barrier)
            for (int i = tid; i < P.nmat; i += kTileBlock) mats[i] = A.pool[P.mat_off + i];
            const int *src = reinterpret_cast<const int *>(A.ops + P.ops_off);
            int *dst = reinterpret_cast<int *>(ops);
            const int words = P.nops * (int)(sizeof(TOp) / sizeof(int));
            for (int i = tid; i < words; i += kTileBlock) dst[i] = src[i];
            const int *ssrc = reinterpret_cast<const int *>(A.stages + P.stages_off);
            int *sdst = reinterpret_cast<int *>(stages);
            const int swords = P.nstages * (int)(sizeof(TStage) / sizeof(int));
            for (int i = tid; i < swords; i += kTileBlock) sdst[i] = ssrc[i];
            for (int a = tid; a < nA; a += kTileBlock) {
                long long o = 0;
                int rem = a;
                for (int i = g.kA - 1; i >= 0; --i) {
                    o += (long long)(rem % d) * g.strideA[i];
                    rem /= d;
                }
                offA[a] = o;
            }
            if (P.nstages > 0) {
                __syncthreads();   // pool staged before it is prepared
                prepare_pool<R>(mats, prep, P.nmat);
            }
            cur = k;
        }
        if (ADJ)
            for (int i = tid; i < P.nops * kBatchWarps; i += kTileBlock) gacc[i] = 0.0;
        constexpr int KS = StageK<R, D, ADJ>::K;
        R gsum[ADJ ? kMaxGrad : 1];
#pragma unroll
        for (int c = 0; c < (ADJ ? kMaxGrad : 1); ++c) gsum[c] = 0;
        const bool staged = KS > 0 && P.nstages > 0;
        const long long chunk = item - A.prefix[k];
        const long long t0 = chunk * A.chunk_tiles;
        long long t1 = t0 + A.chunk_tiles;
        if (t1 > g.ntiles) t1 = g.ntiles;
        C *psi = A.states + P.psi_off;
        C *lam = A.states + P.lam_off;
        if (tid == 0) sbase[0] = tile_base(g, t0);
        __syncthreads();
        for (long long t = t0; t < t1; ++t) {
            const long long base = sbase[0];
            for (int e = tid; e < T; e += kTileBlock) {
                int a = (int)g.divSEG.div((uint32_t)e);
                int l2 = e - a * g.SEG;
                const long long gi = base + offA[a] + l2;
                cp_async_amp<R>(tp + e, psi + gi);
                if (ADJ) cp_async_amp<R>(tl + e, lam + gi);
            }
            cp_async_wait_all();
            __syncthreads();
            if constexpr (KS > 0) {
                if (staged) {
                    for (int si = 0; si < P.nstages; ++si) {
                        const TStage &st = stages[si];
                        if (!st.legacy) {
                            stage_run<R, D, KS, ADJ>(st, ops, mats, prep, tp, tl, T, gsum);
                        } else {
                            tile_apply<R, D>(ops[st.first], tp, mats, T, g.nt, d);
                            if (ADJ) tile_apply<R, D>(ops[st.first], tl, mats, T, g.nt, d);
                        }
                        __syncthreads();
                    }
                }
            }
            for (int o = 0; o < (staged ? 0 : P.nops); ++o) {
                const TOp &op = ops[o];
                if (ADJ && op.gcol >= 0) {
                    const C *G = mats + op.gmat;
                    const int ls = op.lsa;
                    const int F = T / d;
                    const bool ctrl = op.kind == OP_CPAIR || op.kind == OP_CDIAG;
                    R part = 0;
                    for (int f = tid; f < F; f += kTileBlock) {
                        int hi2 = (int)op.fa.div((uint32_t)f);
                        int b = hi2 * d * ls + (f - hi2 * ls);
                        int ctl = ctrl ? dmod<D>(op.fc.div((uint32_t)b), d) : 0;
                        part += fibre_grad_b<R, D>(tp + b, tl + b, ls, op, G, ctl, d);
                    }
                    double v = warp_sum_b((double)part);
                    if (lane == 0) gacc[o * kBatchWarps + wid] += v;
                }
                tile_apply<R, D>(op, tp, mats, T, g.nt, d);
                if (ADJ) tile_apply<R, D>(op, tl, mats, T, g.nt, d);
                __syncthreads();
            }
            for (int e = tid; e < T; e += kTileBlock) {
                int a = (int)g.divSEG.div((uint32_t)e);
                int l2 = e - a * g.SEG;
                const long long gi = base + offA[a] + l2;
                psi[gi] = tp[e];
                if (ADJ) lam[gi] = tl[e];
            }
            if (tid == 0 && t + 1 < t1) sbase[0] = tile_base(g, t + 1);
            __syncthreads();
        }
        if (ADJ) {
            if (staged) {
                // register accumulators -> gacc[col * warps + warp]
#pragma unroll
                for (int c = 0; c < (ADJ ? kMaxGrad : 1); ++c) {
                    if (c >= P.ncols) break;
                    const double v = warp_sum_b((double)gsum[c]);
                    if (lane == 0) gacc[c * kBatchWarps + wid] = v;
                }
                __syncthreads();
                for (int c = tid; c < P.ncols; c += kTileBlock) {
                    double s = 0.0;
                    for (int w = 0; w < kBatchWarps; ++w) s += gacc[c * kBatchWarps + w];
                    A.rows[P.rows_base + chunk * P.ncols + c] = 2.0 * s;
                }
            } else {
                for (int o = tid; o < P.nops; o += kTileBlock) {
                    const TOp &op = ops[o];
                    if (op.gcol < 0) continue;
                    double s = 0.0;
                    for (int w = 0; w < kBatchWarps; ++w) s += gacc[o * kBatchWarps + w];
                    A.rows[P.rows_base + chunk * P.ncols + op.gcol] = 2.0 * s;
                }
            }
            __syncthreads();
        }
    }
}

template <typename R>
size_t batch_smem_bytes(bool adj, int max_T, int max_nmat, int max_nops, int max_nA, int max_nstages) {
    size_t b = (size_t)(adj ? 2 : 1) * max_T * sizeof(cplx<R>) + (size_t)max_nmat * sizeof(cplx<R>) +
               (size_t)max_nops * sizeof(TOp) + (size_t)max_nstages * sizeof(TStage);
    b = (b + 15) & ~(size_t)15;
    if (adj) b += (size_t)max_nops * kBatchWarps * sizeof(double);
    b += (size_t)(max_nA + 1) * sizeof(long long);
    b = (b + 15) & ~(size_t)15;
    b += (size_t)max_nmat * sizeof(float4);   // prepared entries (complex64 register stages)
    return b;
}

template <typename R, int D, bool ADJ>
static cudaError_t batch_prepare_d(size_t smem, int *per_sm) {
    cudaError_t e = cudaFuncSetAttribute(k_batch<R, D, ADJ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_batch<R, D, ADJ>, kTileBlock, smem);
}

// Sets the kernel's shared-memory limit and returns resident CTAs per SM.
template <typename R>
cudaError_t batch_prepare(int d, bool adj, size_t smem, int *per_sm) {
    switch (d) {
#define QF_CASE(DD)                                                                              \
    case DD:                                                                                     \
        return adj ? batch_prepare_d<R, DD, true>(smem, per_sm) : batch_prepare_d<R, DD, false>(smem, per_sm);
        QF_CASE(2) QF_CASE(3) QF_CASE(4) QF_CASE(5) QF_CASE(6) QF_CASE(7) QF_CASE(8) QF_CASE(10)
#undef QF_CASE
    default:
        return adj ? batch_prepare_d<R, 0, true>(smem, per_sm) : batch_prepare_d<R, 0, false>(smem, per_sm);
    }
}

template <typename R>
cudaError_t launch_batch(cudaStream_t stream, int d, bool adj, int grid, size_t smem, cplx<R> *states, const BPass *passes,
                         const long long *prefix, int npasses, const TOp *ops, const cplx<R> *pool,
                         const TStage *stages, const double *params, double *rows, int chunk_tiles, int max_T,
                         int max_nmat, int max_nops, int max_nA, int max_nstages) {
    BatchArgs<R> A;
    A.states = states;
    A.passes = passes;
    A.prefix = prefix;
    A.npasses = npasses;
    A.ops = ops;
    A.pool = pool;
    A.params = params;
    A.rows = rows;
    A.chunk_tiles = chunk_tiles;
    A.max_T = max_T;
    A.max_nmat = max_nmat;
    A.max_nops = max_nops;
    A.max_nA = max_nA;
    A.stages = stages;
    A.max_nstages = max_nstages;
    switch (d) {
#define QF_CASE(DD)                                                                            \
    case DD:                                                                                   \
        if (adj) k_batch<R, DD, true><<<grid, kTileBlock, smem, stream>>>(A, d);               \
        else k_batch<R, DD, false><<<grid, kTileBlock, smem, stream>>>(A, d);                  \
        break;
        QF_CASE(2) QF_CASE(3) QF_CASE(4) QF_CASE(5) QF_CASE(6) QF_CASE(7) QF_CASE(8) QF_CASE(10)
#undef QF_CASE
    default:
        if (adj) k_batch<R, 0, true><<<grid, kTileBlock, smem, stream>>>(A, d);
        else k_batch<R, 0, false><<<grid, kTileBlock, smem, stream>>>(A, d);
        break;
    }
    return cudaGetLastError();
}

// ------------------------------------------------------------------ rotation entries
// One record per parametrised op of the batch tables: its entries are written
// into the pool once per run, before any pass reads them.
struct BParam {
    int pool_off;     // absolute pool offset of the op's entries
    int kind, d, j, k, axis, slot, sign;
};

template <typename R>
__global__ void k_batch_resolve(cplx<R> *pool, const BParam *recs, int count, const double *params) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
        const BParam r = recs[i];
        TOp op;
        op.kind = r.kind;
        op.j = r.j;
        op.k = r.k;
        op.paxis = r.axis;
        op.pslot = r.slot;
        op.psign = r.sign;
        op.mat = r.pool_off;
        resolve_param_op<R>(op, params, r.d, pool);
    }
}

template <typename R>
cudaError_t launch_batch_resolve(cudaStream_t stream, int sms, cplx<R> *pool, const void *recs, int count,
                                 const double *params) {
    if (count <= 0) return cudaSuccess;
    int blocks = (count + 127) / 128;
    if (blocks > 8 * sms) blocks = 8 * sms;
    k_batch_resolve<R><<<blocks, 128, 0, stream>>>(pool, reinterpret_cast<const BParam *>(recs), count, params);
    return cudaGetLastError();
}

size_t bparam_bytes() { return sizeof(BParam); }

// ------------------------------------------------------------------ batched |0..0>, lambda = O psi, loss
struct BObs {
    long long psi_off, lam_off;
    long long N;
    int d, n;
    int w_off;          // weights of this circuit in the weight table
    int items;          // chunks of kObsChunk amplitudes
};

constexpr int kObsChunk = 4096;

__global__ void k_batch_zero(float4 *p, long long n16) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += (long long)gridDim.x * blockDim.x)
        p[i] = make_float4(0.f, 0.f, 0.f, 0.f);
}

template <typename R>
__global__ void k_batch_one(cplx<R> *states, const long long *offs, int count) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < count; c += gridDim.x * blockDim.x)
        states[offs[c]] = mk<R>(1, 0);
}

template <typename R>
__global__ void __launch_bounds__(256) k_batch_obs(cplx<R> *states, const BObs *circ, const long long *prefix, int ncirc,
                                                    const double *weights, double *loss_rows) {
    __shared__ double red[33];
    const long long total = prefix[ncirc];
    for (long long item = blockIdx.x; item < total; item += gridDim.x) {
        int lo = 0, hi = ncirc - 1;
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (prefix[mid] <= item) lo = mid;
            else hi = mid - 1;
        }
        const BObs &B = circ[lo];
        const long long i0 = (item - prefix[lo]) * kObsChunk;
        long long i1 = i0 + kObsChunk;
        if (i1 > B.N) i1 = B.N;
        const cplx<R> *psi = states + B.psi_off;
        cplx<R> *lam = states + B.lam_off;
        const double *w = weights + B.w_off;
        double loss = 0.0;
        for (long long i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
            double o = 0.0;
            long long rem = i;
            for (int q = B.n - 1; q >= 0; --q) {
                long long nx = rem / B.d;
                o += (double)(rem - nx * B.d) * w[q];
                rem = nx;
            }
            cplx<R> v = psi[i];
            loss += o * ((double)v.x * v.x + (double)v.y * v.y);
            lam[i] = mk<R>((R)(o * v.x), (R)(o * v.y));
        }
        // block sum
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        loss = warp_sum_b(loss);
        __syncthreads();
        if (lane == 0) red[wid] = loss;
        __syncthreads();
        if (threadIdx.x == 0) {
            double s = 0.0;
            for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += red[k];
            loss_rows[item] = s;
        }
    }
}

template <typename R>
cudaError_t launch_batch_init(cudaStream_t stream, int sms, cplx<R> *states, long long psi_elems, const long long *offs,
                              int count) {
    const long long n16 = psi_elems * (long long)sizeof(cplx<R>) / 16;
    long long b = (n16 + 255) / 256;
    if (b > 8LL * sms) b = 8LL * sms;
    if (b < 1) b = 1;
    k_batch_zero<<<(unsigned)b, 256, 0, stream>>>(reinterpret_cast<float4 *>(states), n16);
    k_batch_one<R><<<(count + 255) / 256, 256, 0, stream>>>(states, offs, count);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_batch_obs(cudaStream_t stream, int sms, cplx<R> *states, const BObs *circ, const long long *prefix,
                             int ncirc, const double *weights, double *loss_rows) {
    k_batch_obs<R><<<4 * sms, 256, 0, stream>>>(states, circ, prefix, ncirc, weights, loss_rows);
    return cudaGetLastError();
}

size_t bpass_bytes() { return sizeof(BPass); }
size_t bobs_bytes() { return sizeof(BObs); }

template cudaError_t batch_prepare<float>(int, bool, size_t, int *);
template cudaError_t batch_prepare<double>(int, bool, size_t, int *);
template size_t batch_smem_bytes<float>(bool, int, int, int, int, int);
template size_t batch_smem_bytes<double>(bool, int, int, int, int, int);
template cudaError_t launch_batch<float>(cudaStream_t, int, bool, int, size_t, cplx<float> *, const BPass *,
                                         const long long *, int, const TOp *, const cplx<float> *, const TStage *,
                                         const double *, double *, int, int, int, int, int, int);
template cudaError_t launch_batch<double>(cudaStream_t, int, bool, int, size_t, cplx<double> *, const BPass *,
                                          const long long *, int, const TOp *, const cplx<double> *, const TStage *,
                                          const double *, double *, int, int, int, int, int, int);
template cudaError_t launch_batch_resolve<float>(cudaStream_t, int, cplx<float> *, const void *, int, const double *);
template cudaError_t launch_batch_resolve<double>(cudaStream_t, int, cplx<double> *, const void *, int, const double *);
template cudaError_t launch_batch_init<float>(cudaStream_t, int, cplx<float> *, long long, const long long *, int);
template cudaError_t launch_batch_init<double>(cudaStream_t, int, cplx<double> *, long long, const long long *, int);
template cudaError_t launch_batch_obs<float>(cudaStream_t, int, cplx<float> *, const BObs *, const long long *, int,
                                             const double *, double *);
template cudaError_t launch_batch_obs<double>(cudaStream_t, int, cplx<double> *, const BObs *, const long long *, int,
                                              const double *, double *);

}  // namespace qf
