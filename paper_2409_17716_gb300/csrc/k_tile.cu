// k_tile.cu -- fused passes over shared-memory tiles.
//
// A pass names kA "active" high qudits A[0] < ... < A[kA-1] and the rL lowest
// qudits; a tile fixes the digits of every other ("outer") qudit, so it holds
// T = d^(kA + rL) amplitudes: d^kA contiguous runs of SEG = d^rL amplitudes.
// Inside the tile these form a small register of nt = kA + rL local qudits in
// the same significance order (A first, then the low qudits), so every gate of
// the pass that acts only on those qudits is applied to the tile as to a tiny
// state vector (Appendix B definitions, local strides d^(nt-1-p)).  One CTA
// loads a tile with cp.async (8 or 16 bytes per thread, coalesced along each
// run), applies the pass's gate list with a barrier between gates, and writes
// the tile back: each pass costs one read and one write of the state in HBM
// however many gates it holds.  CTAs are persistent over tiles.
#include "qf_internal.cuh"

namespace qf {

template <typename R>
struct TileArgs {
    cplx<R> *psi;
    TileGeom g;
    int nops;
    int nmat;
    const TOp *ops_g;          // device op list, or nullptr -> op_i
    const cplx<R> *mat_g;      // device matrix pool, or nullptr -> mat_i
    TOp op_i;
    cplx<R> mat_i[kInlineMat];
};

constexpr int kTileBlock = 256;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

template <typename R>
__device__ __forceinline__ void cp_async_amp(cplx<R> *dst, const cplx<R> *src);

template <>
__device__ __forceinline__ void cp_async_amp<float>(float2 *dst, const float2 *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
template <>
__device__ __forceinline__ void cp_async_amp<double>(double2 *dst, const double2 *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

template <int D>
__device__ __forceinline__ int dmod(uint32_t x, int d) { return D > 0 ? (int)(x % (uint32_t)D) : (int)(x % (uint32_t)d); }

// One fibre (d amplitudes at p[0], p[ls], ..., p[(d-1) ls]) under a
// single-target op.  ctl = control level (controlled kinds only).
template <typename R, int D>
__device__ __forceinline__ void fibre_apply(cplx<R> *p, int ls, const TOp &op, const cplx<R> *M, int ctl, int d) {
    using C = cplx<R>;
    constexpr int DM = D > 0 ? D : kMaxD;
    switch (op.kind) {
    case OP_DENSE: {
        C v[DM];
#pragma unroll
        for (int m = 0; m < DM; ++m)
            if (m < d) v[m] = p[m * ls];
#pragma unroll
        for (int l = 0; l < DM; ++l) {
            if (l >= d) break;
            C acc = mk<R>(0, 0);
#pragma unroll
            for (int m = 0; m < DM; ++m)
                if (m < d) acc = cfma(M[l * d + m], v[m], acc);
            p[l * ls] = acc;
        }
        break;
    }
    case OP_PAIR:
    case OP_CPAIR: {
        if (op.kind == OP_CPAIR) {
            if (ctl == 0) break;
            M += 4 * ctl;
        }
        C a = p[op.j * ls], b = p[op.k * ls];
        p[op.j * ls] = cfma(M[1], b, cmul(M[0], a));
        p[op.k * ls] = cfma(M[3], b, cmul(M[2], a));
        break;
    }
    case OP_DIAG:
    case OP_CDIAG: {
        if (op.kind == OP_CDIAG) {
            if (ctl == 0) break;
            M += d * ctl;
        }
#pragma unroll
        for (int l = 0; l < DM; ++l)
            if (l < d && ((op.mask >> l) & 1)) p[l * ls] = cmul(M[l], p[l * ls]);
        break;
    }
    case OP_SHIFT:
    case OP_CSHIFT: {
        int sh = op.s;
        if (op.kind == OP_CSHIFT) sh = (op.s * ctl) % d;
        if (sh == 0) break;
        C v[DM];
#pragma unroll
        for (int m = 0; m < DM; ++m)
            if (m < d) v[m] = p[m * ls];
#pragma unroll
        for (int m = 0; m < DM; ++m)
            if (m < d) {
                int dst = m + sh;
                if (dst >= d) dst -= d;
                p[dst * ls] = v[m];
            }
        break;
    }
    default:
        break;
    }
}

// Applies one op to the whole tile (all threads of the CTA cooperate).
template <typename R, int D>
__device__ void tile_apply(const TOp &op, cplx<R> *tile, const cplx<R> *mats, int T, int nt, int d) {
    using C = cplx<R>;
    const int tid = threadIdx.x;
    const C *M = mats + op.mat;
    switch (op.kind) {
    case OP_SWAP: {
        // exchange the digits of local qudits a (stride lsa) and c (stride lsc)
        const int la = op.lsa, lc = op.lsc;
        for (int e = tid; e < T; e += kTileBlock) {
            int x = dmod<D>(op.fa.div((uint32_t)e), d);
            int y = dmod<D>(op.fc.div((uint32_t)e), d);
            if (x < y) {
                int e2 = e + (y - x) * la - (y - x) * lc;
                C t0 = tile[e];
                tile[e] = tile[e2];
                tile[e2] = t0;
            }
        }
        return;
    }
    case OP_DENSEK: {
        const int K = op.nq;
        int ls[6];
        int DK = 1;
        for (int i = 0; i < K; ++i) {
            int s = 1;
            for (int r = 0; r < nt - 1 - op.q[i]; ++r) s *= d;
            ls[i] = s;
            DK *= d;
        }
        int asc[6];
        for (int i = 0; i < K; ++i) asc[i] = ls[i];
        for (int i = 1; i < K; ++i)
            for (int m = i; m > 0 && asc[m - 1] > asc[m]; --m) {
                int t = asc[m]; asc[m] = asc[m - 1]; asc[m - 1] = t;
            }
        const int G = T / DK;
        for (int g = tid; g < G; g += kTileBlock) {
            // insert a zero digit at every target stride (ascending)
            int b = g;
            for (int i = 0; i < K; ++i) b = (b / asc[i]) * (asc[i] * d) + b % asc[i];
            C v[kMaxDenseK];
            for (int r = 0; r < DK; ++r) {
                int off = 0, rr = r;
                for (int i = K - 1; i >= 0; --i) { off += (rr % d) * ls[i]; rr /= d; }
                v[r] = tile[b + off];
            }
            for (int r = 0; r < DK; ++r) {
                C acc = mk<R>(0, 0);
                for (int m = 0; m < DK; ++m) acc = cfma(M[r * DK + m], v[m], acc);
                int off = 0, rr = r;
                for (int i = K - 1; i >= 0; --i) { off += (rr % d) * ls[i]; rr /= d; }
                tile[b + off] = acc;
            }
        }
        return;
    }
    default: {
        // single-target kinds: fibres over local qudit a
        const int ls = op.lsa;
        const int F = T / d;
        const bool ctrl = op.kind == OP_CPAIR || op.kind == OP_CDIAG || op.kind == OP_CSHIFT;
        for (int f = tid; f < F; f += kTileBlock) {
            int hi = (int)op.fa.div((uint32_t)f);
            int b = hi * d * ls + (f - hi * ls);
            int ctl = ctrl ? dmod<D>(op.fc.div((uint32_t)b), d) : 0;
            fibre_apply<R, D>(tile + b, ls, op, M, ctl, d);
        }
        return;
    }
    }
}

__device__ __forceinline__ long long tile_base(const TileGeom &g, long long t) {
    long long base = 0;
    for (int r = 0; r < g.nruns; ++r) {
        long long q = t / g.runM[r];
        base += (t - q * g.runM[r]) * g.runS[r];
        t = q;
    }
    return base;
}

template <typename R, int D>
__global__ void __launch_bounds__(kTileBlock) k_tile(const __grid_constant__ TileArgs<R> A, int d_rt) {
    using C = cplx<R>;
    extern __shared__ __align__(16) unsigned char smem[];
    const int d = D > 0 ? D : d_rt;
    const TileGeom &g = A.g;
    const int T = g.T;
    const int tid = threadIdx.x;
    const int nA = T / g.SEG;   // d^kA runs per tile

    // layout (must match tile_smem_bytes): tile | pool | ops | pad to 16 | offA | base
    C *tile = reinterpret_cast<C *>(smem);
    C *mats = tile + T;
    TOp *ops = reinterpret_cast<TOp *>(mats + A.nmat);
    size_t off = (size_t)T * sizeof(C) + (size_t)A.nmat * sizeof(C) + (size_t)A.nops * sizeof(TOp);
    off = (off + 15) & ~(size_t)15;
    long long *offA = reinterpret_cast<long long *>(smem + off);
    long long *sbase = offA + nA;

    // stage the gate list, matrix pool and run offsets
    const C *msrc = A.mat_g ? A.mat_g : A.mat_i;
    for (int i = tid; i < A.nmat; i += kTileBlock) mats[i] = msrc[i];
    if (A.ops_g) {
        const int *src = reinterpret_cast<const int *>(A.ops_g);
        int *dst = reinterpret_cast<int *>(ops);
        const int words = A.nops * (int)(sizeof(TOp) / sizeof(int));
        for (int i = tid; i < words; i += kTileBlock) dst[i] = src[i];
    } else if (tid == 0) {
        ops[0] = A.op_i;
    }
    for (int a = tid; a < nA; a += kTileBlock) {
        long long off = 0;
        int rem = a;
        for (int i = g.kA - 1; i >= 0; --i) {
            off += (long long)(rem % d) * g.strideA[i];
            rem /= d;
        }
        offA[a] = off;
    }
    if (tid == 0) sbase[0] = tile_base(g, blockIdx.x);
    __syncthreads();

    for (long long t = blockIdx.x; t < g.ntiles; t += gridDim.x) {
        const long long base = sbase[0];
        const C *src = A.psi + base;
        for (int e = tid; e < T; e += kTileBlock) {
            int a = (int)g.divSEG.div((uint32_t)e);
            int lo = e - a * g.SEG;
            cp_async_amp<R>(tile + e, src + offA[a] + lo);
        }
        cp_async_wait_all();
        __syncthreads();
        for (int o = 0; o < A.nops; ++o) {
            tile_apply<R, D>(ops[o], tile, mats, T, g.nt, d);
            __syncthreads();
        }
        C *dst = A.psi + base;
        for (int e = tid; e < T; e += kTileBlock) {
            int a = (int)g.divSEG.div((uint32_t)e);
            int lo = e - a * g.SEG;
            dst[offA[a] + lo] = tile[e];
        }
        if (tid == 0 && t + gridDim.x < g.ntiles) sbase[0] = tile_base(g, t + gridDim.x);
        __syncthreads();
    }
}

template <typename R>
size_t tile_smem_bytes(const TileGeom &g, int nops, int nmat) {
    size_t b = (size_t)g.T * sizeof(cplx<R>) + (size_t)nmat * sizeof(cplx<R>) + (size_t)nops * sizeof(TOp);
    b = (b + 15) & ~(size_t)15;
    b += (size_t)(g.T / g.SEG) * sizeof(long long) + 16;
    return b;
}

template <typename R, int D>
static cudaError_t launch_tile_d(const Launch &L, const TileArgs<R> &A, int d, size_t smem) {
    static int configured_bytes = 0;
    if ((int)smem > configured_bytes) {
        cudaError_t e = cudaFuncSetAttribute(k_tile<R, D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured_bytes = (int)smem;
    }
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tile<R, D>, kTileBlock, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    long long grid = (long long)per_sm * L.num_sms;
    if (grid > A.g.ntiles) grid = A.g.ntiles;
    k_tile<R, D><<<(unsigned)grid, kTileBlock, smem, L.stream>>>(A, d);
    return cudaGetLastError();
}

// Launches one pass.  ops/mat point to device memory (program passes) or are
// nullptr, in which case the single op `op_i` with `nmat` inline entries
// `mat_i` is used.
template <typename R>
cudaError_t launch_tile(const Launch &L, cplx<R> *psi, int d, const TileGeom &g, int nops, const TOp *ops_dev,
                        const cplx<R> *mat_dev, int nmat, const TOp *op_i, const cplx<R> *mat_i) {
    TileArgs<R> A;
    A.psi = psi;
    A.g = g;
    A.nops = nops;
    A.nmat = nmat;
    A.ops_g = ops_dev;
    A.mat_g = mat_dev;
    if (!ops_dev) {
        if (nops != 1 || nmat > kInlineMat) return cudaErrorInvalidValue;
        A.op_i = *op_i;
        for (int i = 0; i < nmat; ++i) A.mat_i[i] = mat_i[i];
    }
    size_t smem = tile_smem_bytes<R>(g, nops, nmat);
    switch (d) {
#define QF_CASE(DD) case DD: return launch_tile_d<R, DD>(L, A, d, smem);
        QF_CASE(2) QF_CASE(3) QF_CASE(4) QF_CASE(5) QF_CASE(6) QF_CASE(7) QF_CASE(8)
#undef QF_CASE
    default: return launch_tile_d<R, 0>(L, A, d, smem);
    }
}

template size_t tile_smem_bytes<float>(const TileGeom &, int, int);
template size_t tile_smem_bytes<double>(const TileGeom &, int, int);
template cudaError_t launch_tile<float>(const Launch &, cplx<float> *, int, const TileGeom &, int, const TOp *,
                                        const cplx<float> *, int, const TOp *, const cplx<float> *);
template cudaError_t launch_tile<double>(const Launch &, cplx<double> *, int, const TileGeom &, int, const TOp *,
                                         const cplx<double> *, int, const TOp *, const cplx<double> *);

}  // namespace qf
