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
#include "stage_device.cuh"

namespace qf {

template <typename R>
struct TileArgs {
    cplx<R> *psi;
    TileGeom g;
    int nops;
    int nmat;
    const TOp *ops_g;          // device op list, or nullptr -> op_i
    const cplx<R> *mat_g;      // device matrix pool, or nullptr -> mat_i
    const TStage *stages_g;    // register stages, or nullptr: every op through shared memory
    int nstages;
    TOp op_i;
    cplx<R> mat_i[kInlineMat];
};

template <typename R, int D>
__global__ void __launch_bounds__(kTileBlock) k_tile(const __grid_constant__ TileArgs<R> A, int d_rt) {
    using C = cplx<R>;
    extern __shared__ __align__(16) unsigned char smem[];
    const int d = D > 0 ? D : d_rt;
    const TileGeom &g = A.g;
    const int T = g.T;
    const int tid = threadIdx.x;
    const int nA = T / g.SEG;   // d^kA runs per tile

    // layout (must match tile_smem_bytes): tile | pool | ops | stages | pad to 16 | offA | base
    C *tile = reinterpret_cast<C *>(smem);
    C *mats = tile + T;
    TOp *ops = reinterpret_cast<TOp *>(mats + A.nmat);
    TStage *stages = reinterpret_cast<TStage *>(ops + A.nops);
    size_t off = (size_t)T * sizeof(C) + (size_t)A.nmat * sizeof(C) + (size_t)A.nops * sizeof(TOp) +
                 (size_t)A.nstages * sizeof(TStage);
    off = (off + 15) & ~(size_t)15;
    long long *offA = reinterpret_cast<long long *>(smem + off);
    long long *sbase = offA + nA;
    float4 *prep = reinterpret_cast<float4 *>(smem + ((off + (size_t)(nA + 1) * sizeof(long long) + 15) & ~(size_t)15));

    // stage the gate list, matrix pool and run offsets
    const C *msrc = A.mat_g ? A.mat_g : A.mat_i;
    for (int i = tid; i < A.nmat; i += blockDim.x) mats[i] = msrc[i];
    if (A.ops_g) {
        const int *src = reinterpret_cast<const int *>(A.ops_g);
        int *dst = reinterpret_cast<int *>(ops);
        const int words = A.nops * (int)(sizeof(TOp) / sizeof(int));
        for (int i = tid; i < words; i += blockDim.x) dst[i] = src[i];
    } else if (tid == 0) {
        ops[0] = A.op_i;
    }
    if (A.nstages > 0) {
        const int *src = reinterpret_cast<const int *>(A.stages_g);
        int *dst = reinterpret_cast<int *>(stages);
        const int words = A.nstages * (int)(sizeof(TStage) / sizeof(int));
        for (int i = tid; i < words; i += blockDim.x) dst[i] = src[i];
    }
    for (int a = tid; a < nA; a += blockDim.x) {
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
    if (A.nstages > 0) prepare_pool<R>(mats, prep, A.nmat);
    // element e = a * SEG + lo of the tile; each thread steps by blockDim.x
    const int a0 = (int)g.divSEG.div((uint32_t)tid), lo0 = tid - a0 * g.SEG;
    const int da = (int)g.divSEG.div((uint32_t)blockDim.x), dl = (int)blockDim.x - da * g.SEG;

    for (long long t = blockIdx.x; t < g.ntiles; t += gridDim.x) {
        const long long base = sbase[0];
        const C *src = A.psi + base;
        for (int e = tid, a = a0, lo = lo0; e < T; e += blockDim.x) {
            cp_async_amp<R>(tile + e, src + offA[a] + lo);
            lo += dl;
            a += da;
            if (lo >= g.SEG) { lo -= g.SEG; ++a; }
        }
        cp_async_wait_all();
        __syncthreads();
        if (A.nstages > 0) {
            for (int si = 0; si < A.nstages; ++si) {
                const TStage &st = stages[si];
                if constexpr (StageK<R, D, false>::K > 0) {
                    if (!st.legacy)
                        stage_run<R, D, StageK<R, D, false>::K, false>(st, ops, mats, prep, tile, nullptr, T, nullptr);
                    else tile_apply<R, D>(ops[st.first], tile, mats, T, g.nt, d);
                } else {
                    tile_apply<R, D>(ops[st.first], tile, mats, T, g.nt, d);
                }
                __syncthreads();
            }
        } else {
            for (int o = 0; o < A.nops; ++o) {
                tile_apply<R, D>(ops[o], tile, mats, T, g.nt, d);
                __syncthreads();
            }
        }
        C *dst = A.psi + base;
        for (int e = tid, a = a0, lo = lo0; e < T; e += blockDim.x) {
            dst[offA[a] + lo] = tile[e];
            lo += dl;
            a += da;
            if (lo >= g.SEG) { lo -= g.SEG; ++a; }
        }
        if (tid == 0 && t + gridDim.x < g.ntiles) sbase[0] = tile_base(g, t + gridDim.x);
        __syncthreads();
    }
}

template <typename R>
size_t tile_smem_bytes(const TileGeom &g, int nops, int nmat, int nstages) {
    size_t b = (size_t)g.T * sizeof(cplx<R>) + (size_t)nmat * sizeof(cplx<R>) + (size_t)nops * sizeof(TOp) +
               (size_t)nstages * sizeof(TStage);
    b = (b + 15) & ~(size_t)15;
    b += (size_t)(g.T / g.SEG + 1) * sizeof(long long);
    b = (b + 15) & ~(size_t)15;
    b += (size_t)nmat * sizeof(float4);   // prepared entries (complex64 register stages)
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
    // a tile with fewer register blocks than a 256-thread CTA runs on 128
    // threads (every loop of the kernel strides by blockDim.x)
    int threads = kTileBlock;
    const int K = stage_k(d, false, sizeof(R) == 8);
    if (A.nstages > 0 && K > 0) {
        int dk = 1;
        for (int i = 0; i < K; ++i) dk *= d;
        if (A.g.T / dk <= kTileBlock / 2) threads = kTileBlock / 2;
    }
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tile<R, D>, threads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    long long grid = (long long)per_sm * L.num_sms;
    if (grid > A.g.ntiles) grid = A.g.ntiles;
    k_tile<R, D><<<(unsigned)grid, threads, smem, L.stream>>>(A, d);
    return cudaGetLastError();
}

// Launches one pass.  ops/mat point to device memory (program passes) or are
// nullptr, in which case the single op `op_i` with `nmat` inline entries
// `mat_i` is used.
template <typename R>
cudaError_t launch_tile(const Launch &L, cplx<R> *psi, int d, const TileGeom &g, int nops, const TOp *ops_dev,
                        const cplx<R> *mat_dev, int nmat, const TOp *op_i, const cplx<R> *mat_i,
                        const TStage *stages_dev, int nstages) {
    TileArgs<R> A;
    A.psi = psi;
    A.g = g;
    A.nops = nops;
    A.nmat = nmat;
    A.ops_g = ops_dev;
    A.mat_g = mat_dev;
    A.stages_g = stages_dev;
    A.nstages = stages_dev ? nstages : 0;
    if (!ops_dev) {
        if (nops != 1 || nmat > kInlineMat) return cudaErrorInvalidValue;
        A.op_i = *op_i;
        for (int i = 0; i < nmat; ++i) A.mat_i[i] = mat_i[i];
    }
    size_t smem = tile_smem_bytes<R>(g, nops, nmat, A.nstages);
    switch (d) {
#define QF_CASE(DD) case DD: return launch_tile_d<R, DD>(L, A, d, smem);
        QF_CASE(2) QF_CASE(3) QF_CASE(4) QF_CASE(5) QF_CASE(6) QF_CASE(7) QF_CASE(8)
#undef QF_CASE
    default: return launch_tile_d<R, 0>(L, A, d, smem);
    }
}

template size_t tile_smem_bytes<float>(const TileGeom &, int, int, int);
template size_t tile_smem_bytes<double>(const TileGeom &, int, int, int);
template cudaError_t launch_tile<float>(const Launch &, cplx<float> *, int, const TileGeom &, int, const TOp *,
                                        const cplx<float> *, int, const TOp *, const cplx<float> *, const TStage *, int);
template cudaError_t launch_tile<double>(const Launch &, cplx<double> *, int, const TileGeom &, int, const TOp *,
                                         const cplx<double> *, int, const TOp *, const cplx<double> *, const TStage *,
                                         int);

}  // namespace qf
