// k_reduce.cu -- state initialisation and FP64 reductions.
//
// Expectation of the level-number observable on every qudit in one pass:
//   <N_q> = sum_i i_q |psi_i|^2,   i = sum_q i_q d^(n-1-q)
// (the measure utility of section "Code style" returns the marginals
// P_q(m) this is built from: <N_q> = sum_m m P_q(m)).
//
// The state is cut into chunks of d^rc contiguous amplitudes, rc = a + B.  A
// CTA has exactly d^a threads and thread t reads amplitudes t + d^a u of a
// chunk (coalesced), so
//   * the lowest a digits of every amplitude a thread reads are the digits of
//     t: their contribution is digit_r(t) * (thread mass), taken once at the
//     end;
//   * the next B digits are the digits of the unrolled loop counter u: their
//     weights are compile-time constants;
//   * the digits above rc are constant over a chunk: the CTA reduces the chunk
//     mass once and adds digit_q(chunk) * mass to an FP64 accumulator per q.
// Per amplitude this costs |psi|^2, one add and at most B fused multiply-adds
// (complex64 states accumulate a chunk in FP32, ~d^B terms per thread, then
// everything is summed in FP64).  CTA partials go to a scratch array that a
// second one-CTA kernel sums in a fixed order, so results are deterministic.
#include "qf_internal.cuh"

namespace qf {

// ------------------------------------------------------------------ init
template <typename R>
__global__ void k_fill_basis(cplx<R> *psi, long long N, long long index) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (; i < N; i += stride) psi[i] = mk<R>(i == index ? (R)1 : (R)0, (R)0);
}

template <typename R>
cudaError_t launch_basis(const Launch &L, cplx<R> *psi, long long N, long long index) {
    long long blocks = (N + 255) / 256;
    long long cap = (long long)L.num_sms * 8;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    k_fill_basis<R><<<(unsigned)blocks, 256, 0, L.stream>>>(psi, N, index);
    return cudaGetLastError();
}
template cudaError_t launch_basis<float>(const Launch &, cplx<float> *, long long, long long);
template cudaError_t launch_basis<double>(const Launch &, cplx<double> *, long long, long long);

// ------------------------------------------------------------------ helpers
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide FP64 sum; result valid in every thread.  `red` has >= 33 slots.
__device__ double block_sum(double v, double *red) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    double s = 0.0;
    if (wid == 0) {
        s = lane < nw ? red[lane] : 0.0;
        s = warp_sum(s);
        if (lane == 0) red[32] = s;
    }
    __syncthreads();
    return red[32];
}

template <int D> struct NumCfg;
template <> struct NumCfg<2> { static constexpr int A = 8, B = 5; };
template <> struct NumCfg<3> { static constexpr int A = 5, B = 3; };
template <> struct NumCfg<4> { static constexpr int A = 4, B = 2; };
template <> struct NumCfg<5> { static constexpr int A = 3, B = 2; };
template <> struct NumCfg<6> { static constexpr int A = 3, B = 2; };
template <> struct NumCfg<7> { static constexpr int A = 3, B = 1; };
template <> struct NumCfg<8> { static constexpr int A = 3, B = 1; };

constexpr int ipow_c(int d, int e) { return e == 0 ? 1 : d * ipow_c(d, e - 1); }

// partials: gridDim.x rows of (n + 1) doubles: <N_q> for q < n, then norm.
template <typename R, int D>
__global__ void __launch_bounds__(ipow_c(D, NumCfg<D>::A)) k_expect_number(const cplx<R> *__restrict__ psi, int n,
                                                                          long long nchunks, double *partials) {
    constexpr int A = NumCfg<D>::A, B = NumCfg<D>::B;
    constexpr int BLK = ipow_c(D, A);
    constexpr int U = ipow_c(D, B);
    constexpr int CH = BLK * U;
    using Acc = R;  // FP32 within a chunk for complex64, FP64 for complex128
    __shared__ double red[33];
    __shared__ double hacc[kMaxQudits + 1];
    const int tid = threadIdx.x;
    const int nh = n - A - B;  // digits constant over a chunk
    for (int q = tid; q <= kMaxQudits; q += BLK) hacc[q] = 0.0;

    double mass = 0.0;
    double w[B];
#pragma unroll
    for (int r = 0; r < B; ++r) w[r] = 0.0;

    for (long long c = blockIdx.x; c < nchunks; c += gridDim.x) {
        const cplx<R> *p = psi + c * CH + tid;
        Acc m = 0, wl[B];
#pragma unroll
        for (int r = 0; r < B; ++r) wl[r] = 0;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            cplx<R> v = p[u * BLK];
            Acc pr = v.x * v.x + v.y * v.y;
            m += pr;
#pragma unroll
            for (int r = 0; r < B; ++r) {
                int pw = 1;
#pragma unroll
                for (int s = 0; s < r; ++s) pw *= D;
                const int dig = (u / pw) % D;
                if (dig) wl[r] += (Acc)dig * pr;
            }
        }
        mass += (double)m;
#pragma unroll
        for (int r = 0; r < B; ++r) w[r] += (double)wl[r];
        if (nh > 0) {
            double cm = block_sum((double)m, red);
            // digits of the chunk index are the digits of qudits nh-1 ... 0
            if (tid < nh) {
                // qudit tid's digit of the chunk index: divide by d^(nh-1-tid)
                long long div = 1;
                for (int s = 0; s < nh - 1 - tid; ++s) div *= D;
                const int dig = (int)((c / div) % D);
                hacc[tid] += (double)dig * cm;
            }
        }
    }
    __syncthreads();
    // per-qudit totals of this CTA
    double *out = partials + (long long)blockIdx.x * (n + 1);
    // thread-constant digits: qudit n-1-r for r < A
    int t = tid;
    for (int r = 0; r < A; ++r) {
        const int dig = t % D;
        t /= D;
        double s = block_sum((double)dig * mass, red);
        if (tid == 0 && n - 1 - r >= 0) out[n - 1 - r] = s;
    }
#pragma unroll
    for (int r = 0; r < B; ++r) {
        double s = block_sum(w[r], red);
        if (tid == 0) out[n - 1 - A - r] = s;
    }
    double s = block_sum(mass, red);
    if (tid == 0) out[n] = s;
    for (int q = tid; q < nh; q += BLK) out[q] = hacc[q];
}

// Generic path (runtime d, or registers too small for the chunked kernel):
// each thread extracts every digit of every amplitude.  FP64 throughout.
template <typename R>
__global__ void __launch_bounds__(256) k_expect_number_generic(const cplx<R> *__restrict__ psi, int d, int n, long long N,
                                                                double *partials) {
    __shared__ double red[33];
    double acc[kMaxQudits + 1];
    for (int q = 0; q <= n; ++q) acc[q] = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        cplx<R> v = psi[i];
        double p = (double)v.x * v.x + (double)v.y * v.y;
        acc[n] += p;
        long long rem = i;
        for (int q = n - 1; q >= 0; --q) {
            long long nx = rem / d;
            acc[q] += (double)(rem - nx * d) * p;
            rem = nx;
        }
    }
    double *out = partials + (long long)blockIdx.x * (n + 1);
    for (int q = 0; q <= n; ++q) {
        double s = block_sum(acc[q], red);
        if (threadIdx.x == 0) out[q] = s;
    }
}

// Sums `rows` rows of `cols` partials: one warp per column, lane l adding
// rows l, l + 32, ... in order, then a fixed shuffle tree, so the result is
// the same on every run (launched with 32 threads per column, at most 1024).
__global__ void k_sum_partials(const double *partials, int rows, int cols, double *out) {
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int c = threadIdx.x >> 5; c < cols; c += nw) {
        double s = 0.0;
        for (int r = lane; r < rows; r += 32) s += partials[(long long)r * cols + c];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) out[c] = s;
    }
}

static unsigned sum_threads(int cols) { return 32u * (unsigned)(cols < 1 ? 1 : cols > 32 ? 32 : cols); }

cudaError_t launch_sum_rows(cudaStream_t stream, const double *rows, int nrows, int cols, double *out) {
    k_sum_partials<<<1, sum_threads(cols), 0, stream>>>(rows, nrows, cols, out);
    return cudaGetLastError();
}

// Fibre reduction over target qudit q (stride S): kind 0 = marginal P_q(m)
// (d outputs), kind 1 = <psi|O_q|psi> (2 outputs: re, im) with O in `obs`.
template <typename R>
__global__ void __launch_bounds__(256) k_fibre_reduce(const cplx<R> *__restrict__ psi, int d, long long nfib, long long S,
                                                        int kind, const double2 *obs, double *partials) {
    __shared__ double red[33];
    double acc[kMaxD];
    for (int m = 0; m < d; ++m) acc[m] = 0.0;
    double are = 0.0, aim = 0.0;
    for (long long f = (long long)blockIdx.x * blockDim.x + threadIdx.x; f < nfib; f += (long long)gridDim.x * blockDim.x) {
        long long h = f / S, lo = f - h * S;
        const cplx<R> *p = psi + h * d * S + lo;
        if (kind == 0) {
            for (int m = 0; m < d; ++m) {
                cplx<R> v = p[m * S];
                acc[m] += (double)v.x * v.x + (double)v.y * v.y;
            }
        } else {
            double vr[kMaxD], vi[kMaxD];
            for (int m = 0; m < d; ++m) { cplx<R> v = p[m * S]; vr[m] = v.x; vi[m] = v.y; }
            for (int l = 0; l < d; ++l) {
                double rr = 0.0, ri = 0.0;
                for (int m = 0; m < d; ++m) {
                    double2 o = obs[l * d + m];
                    rr += o.x * vr[m] - o.y * vi[m];
                    ri += o.x * vi[m] + o.y * vr[m];
                }
                // conj(v_l) * (O v)_l
                are += vr[l] * rr + vi[l] * ri;
                aim += vr[l] * ri - vi[l] * rr;
            }
        }
    }
    const int cols = kind == 0 ? d : 2;
    double *out = partials + (long long)blockIdx.x * cols;
    if (kind == 0) {
        for (int m = 0; m < d; ++m) {
            double s = block_sum(acc[m], red);
            if (threadIdx.x == 0) out[m] = s;
        }
    } else {
        double s0 = block_sum(are, red);
        double s1 = block_sum(aim, red);
        if (threadIdx.x == 0) { out[0] = s0; out[1] = s1; }
    }
}

// Upper bound on the CTAs the reductions use (scratch rows).
// (8 per SM: the per-chunk block sums leave one CTA latency-bound; measured
// 1.6x faster than 2 per SM at these sizes, 16 per SM no better)
int reduce_max_blocks(int num_sms) { return 8 * num_sms; }

// <N_q> for every q plus the norm -> out_dev[0..n].  `partials` must hold
// reduce_max_blocks() * (n + 1) doubles.
template <typename R>
cudaError_t launch_expect_number(const Launch &L, const cplx<R> *psi, int d, int n, double *partials, double *out_dev) {
    long long N = 1;
    for (int i = 0; i < n; ++i) N *= d;
    int maxb = reduce_max_blocks(L.num_sms);
    int blocks = 0;
    switch (d) {
#define QF_CASE(DD)                                                                                  \
    case DD: {                                                                                       \
        constexpr int CH = ipow_c(DD, NumCfg<DD>::A + NumCfg<DD>::B);                                \
        if (n >= NumCfg<DD>::A + NumCfg<DD>::B) {                                                    \
            long long nch = N / CH;                                                                  \
            blocks = (int)(nch < maxb ? nch : maxb);                                                 \
            k_expect_number<R, DD><<<blocks, ipow_c(DD, NumCfg<DD>::A), 0, L.stream>>>(psi, n, nch, partials); \
        }                                                                                            \
        break;                                                                                       \
    }
        QF_CASE(2) QF_CASE(3) QF_CASE(4) QF_CASE(5) QF_CASE(6) QF_CASE(7) QF_CASE(8)
#undef QF_CASE
    default:
        break;
    }
    if (blocks == 0) {
        long long b = (N + 255) / 256;
        blocks = (int)(b < maxb ? b : maxb);
        k_expect_number_generic<R><<<blocks, 256, 0, L.stream>>>(psi, d, n, N, partials);
    }
    k_sum_partials<<<1, sum_threads(n + 1), 0, L.stream>>>(partials, blocks, n + 1, out_dev);
    return cudaGetLastError();
}

// kind 0: marginal of qudit q (d outputs); kind 1: <O_q> (re, im); obs_dev
// holds the d x d FP64 matrix for kind 1.
template <typename R>
cudaError_t launch_fibre_reduce_g(const Launch &L, const cplx<R> *psi, int d, long long S, long long N, int kind,
                                  const double2 *obs_dev, double *partials, double *out_dev);

template <typename R>
cudaError_t launch_fibre_reduce(const Launch &L, const cplx<R> *psi, int d, int n, int q, int kind, const double2 *obs_dev,
                                double *partials, double *out_dev) {
    long long S = 1, N = 1;
    for (int i = 0; i < n - 1 - q; ++i) S *= d;
    for (int i = 0; i < n; ++i) N *= d;
    return launch_fibre_reduce_g<R>(L, psi, d, S, N, kind, obs_dev, partials, out_dev);
}

// The same on an explicit geometry: target of dimension d at stride S in a
// state of N amplitudes (mixed registers use the target's own d and S).
template <typename R>
cudaError_t launch_fibre_reduce_g(const Launch &L, const cplx<R> *psi, int d, long long S, long long N, int kind,
                                  const double2 *obs_dev, double *partials, double *out_dev) {
    long long nfib = N / d;
    int maxb = reduce_max_blocks(L.num_sms);
    long long b = (nfib + 255) / 256;
    int blocks = (int)(b < maxb ? b : maxb);
    k_fibre_reduce<R><<<blocks, 256, 0, L.stream>>>(psi, d, nfib, S, kind, obs_dev, partials);
    k_sum_partials<<<1, sum_threads(kind == 0 ? d : 2), 0, L.stream>>>(partials, blocks, kind == 0 ? d : 2, out_dev);
    return cudaGetLastError();
}

template cudaError_t launch_expect_number<float>(const Launch &, const cplx<float> *, int, int, double *, double *);
template cudaError_t launch_expect_number<double>(const Launch &, const cplx<double> *, int, int, double *, double *);
template cudaError_t launch_fibre_reduce<float>(const Launch &, const cplx<float> *, int, int, int, int, const double2 *,
                                                double *, double *);
template cudaError_t launch_fibre_reduce<double>(const Launch &, const cplx<double> *, int, int, int, int, const double2 *,
                                                 double *, double *);
template cudaError_t launch_fibre_reduce_g<float>(const Launch &, const cplx<float> *, int, long long, long long, int,
                                                  const double2 *, double *, double *);
template cudaError_t launch_fibre_reduce_g<double>(const Launch &, const cplx<double> *, int, long long, long long, int,
                                                   const double2 *, double *, double *);

}  // namespace qf

// ---------------------------------------------------------------------------
// Allocation-free <N_q> entry point.
//
// Some callers cannot allocate device memory when they need a measurement:
// host callbacks and latency-critical loops that must not trigger the
// implicit device synchronisation cudaMalloc/cudaFree can cause, and hosts whose framework owns the whole device heap through its own
// pool and leaves nothing for a library to take.  For them this entry point
// reduces a caller-owned state into a caller-owned output and keeps the
// per-CTA partial sums in a fixed file-scope device array instead of the
// scratch a qf_state allocates.
#include <mutex>
#include <string>

#include "qf_host.h"

namespace qf {

constexpr int kNoAllocRows = 512;              // CTA partial rows
constexpr int kNoAllocCols = 64;               // doubles per row: n + 1 <= 64
constexpr int kNoAllocMaxDevices = 64;

// 512 x 64 doubles = 256 KiB, resident on every device that loads the library
// until the process exits.
static __device__ __align__(256) double g_noalloc_partials[kNoAllocRows * kNoAllocCols];

static std::mutex g_noalloc_mu;
static double *g_noalloc_ptr[kNoAllocMaxDevices];   // device address of the array, per device
static int g_noalloc_sms[kNoAllocMaxDevices];

// Same kernels and CTA partial layout as launch_expect_number, with the CTA
// count capped by the fixed scratch.
template <typename R>
static cudaError_t noalloc_launch(cudaStream_t stream, int sms, const cplx<R> *psi, int d, int n, double *partials,
                                  double *out_dev) {
    long long N = 1;
    for (int i = 0; i < n; ++i) N *= d;
    int maxb = 2 * sms;
    if (maxb > kNoAllocRows) maxb = kNoAllocRows;
    int blocks = 0;
    switch (d) {
#define QF_CASE(DD)                                                                                            \
    case DD: {                                                                                                 \
        constexpr int CH = ipow_c(DD, NumCfg<DD>::A + NumCfg<DD>::B);                                          \
        if (n >= NumCfg<DD>::A + NumCfg<DD>::B) {                                                              \
            long long nch = N / CH;                                                                            \
            blocks = (int)(nch < maxb ? nch : maxb);                                                           \
            k_expect_number<R, DD><<<blocks, ipow_c(DD, NumCfg<DD>::A), 0, stream>>>(psi, n, nch, partials); \
        }                                                                                                      \
        break;                                                                                                 \
    }
        QF_CASE(2) QF_CASE(3) QF_CASE(4) QF_CASE(5) QF_CASE(6) QF_CASE(7) QF_CASE(8)
#undef QF_CASE
    default:
        break;
    }
    if (blocks == 0) {
        long long b = (N + 255) / 256;
        blocks = (int)(b < maxb ? b : maxb);
        k_expect_number_generic<R><<<blocks, 256, 0, stream>>>(psi, d, n, N, partials);
    }
    k_sum_partials<<<1, sum_threads(n + 1), 0, stream>>>(partials, blocks, n + 1, out_dev);
    return cudaGetLastError();
}

}  // namespace qf

extern "C" qf_status qf_expect_number_noalloc(const void *psi_dev, int d, int n, qf_dtype dt, void *cuda_stream,
                                              double *out_dev) {
    using namespace qf;
    if (!psi_dev || ((uintptr_t)psi_dev & 15) != 0)
        return set_error(QF_ERR_ARG, "qf_expect_number_noalloc: amplitudes must be a non-NULL 16-byte aligned device pointer");
    if (!out_dev || ((uintptr_t)out_dev & 7) != 0)
        return set_error(QF_ERR_ARG, "qf_expect_number_noalloc: output must be a non-NULL 8-byte aligned device pointer");
    if (d < 2 || d > kMaxD) return set_error(QF_ERR_ARG, "qf_expect_number_noalloc: d must be in [2, 16]");
    if (dt != QF_C64 && dt != QF_C128) return set_error(QF_ERR_ARG, "qf_expect_number_noalloc: unknown dtype");
    if (n < 1) return set_error(QF_ERR_ARG, "qf_expect_number_noalloc: n must be >= 1");
    // d^n <= 9e15 is the binding limit: it implies n <= 52, so every CTA row
    // of n + 1 outputs fits the scratch's 64 columns
    long double Nf = 1;
    for (int i = 0; i < n && Nf <= 9.0e15L; ++i) Nf *= d;
    if (Nf > 9.0e15L)
        return set_error(QF_ERR_ARG, "qf_expect_number_noalloc: d^n too large (at most 9e15 amplitudes)");
    static_assert(kNoAllocCols >= 53, "the scratch rows must hold n + 1 outputs for every d^n <= 9e15");

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_error(e, "qf_expect_number_noalloc: cudaGetDevice");
    {
        // the scratch address looked up below belongs to the current device,
        // so the stream must too
        int sdev = dev;
        e = cudaStreamGetDevice((cudaStream_t)cuda_stream, &sdev);
        if (e != cudaSuccess) return cuda_error(e, "qf_expect_number_noalloc: cudaStreamGetDevice");
        if (sdev != dev)
            return set_error(QF_ERR_ARG, "qf_expect_number_noalloc: cuda_stream belongs to device " +
                                             std::to_string(sdev) + ", not the current device " + std::to_string(dev));
    }
    if (dev < 0 || dev >= kNoAllocMaxDevices)
        return set_error(QF_ERR_UNSUPPORTED, "qf_expect_number_noalloc: device ordinal beyond 63");
    double *partials = nullptr;
    int sms = 0;
    {
        // one-time set-up per device, with that device current: the host-side
        // name of the array is not a device address, so look the address up
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        if (!g_noalloc_ptr[dev]) {
            double *p = nullptr;
            e = cudaGetSymbolAddress((void **)&p, g_noalloc_partials);
            if (e != cudaSuccess) return cuda_error(e, "qf_expect_number_noalloc: cudaGetSymbolAddress");
            int s = 0;
            e = cudaDeviceGetAttribute(&s, cudaDevAttrMultiProcessorCount, dev);
            if (e != cudaSuccess) return cuda_error(e, "qf_expect_number_noalloc: SM count");
            g_noalloc_sms[dev] = s > 0 ? s : 1;
            g_noalloc_ptr[dev] = p;
        }
        partials = g_noalloc_ptr[dev];
        sms = g_noalloc_sms[dev];
    }
    cudaStream_t stream = (cudaStream_t)cuda_stream;
    e = dt == QF_C64 ? noalloc_launch<float>(stream, sms, (const float2 *)psi_dev, d, n, partials, out_dev)
                     : noalloc_launch<double>(stream, sms, (const double2 *)psi_dev, d, n, partials, out_dev);
    if (e != cudaSuccess) return cuda_error(e, "qf_expect_number_noalloc: reduction kernels");
    return QF_OK;
}

// ---------------------------------------------------------------------------
// Measurement ("Code style": measure(state, index, ..., shots) returns the
// marginal probabilities of the `index` qudits and a histogram of shots).
namespace qf {

struct MargArgs {
    int k;                        // measured qudits
    long long stride[kMaxQudits];  // global strides of the measured qudits, most significant first
    int dim[kMaxQudits];          // their dimensions
    int bins;                     // product of their dimensions
};

// Per-CTA bins in shared memory (FP64 atomics, so the order of additions within
// a CTA -- and the last bits of a bin -- may vary between runs), one row of
// partials per CTA, summed in CTA order.
template <typename R>
__global__ void __launch_bounds__(256) k_marginal(const cplx<R> *__restrict__ psi, long long N,
                                                   const __grid_constant__ MargArgs M, double *partials) {
    extern __shared__ double bins[];
    for (int b = threadIdx.x; b < M.bins; b += blockDim.x) bins[b] = 0.0;
    __syncthreads();
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        const cplx<R> v = psi[i];
        const double p = (double)v.x * v.x + (double)v.y * v.y;
        int r = 0;
        for (int a = 0; a < M.k; ++a) r = r * M.dim[a] + (int)((i / M.stride[a]) % M.dim[a]);
        atomicAdd(&bins[r], p);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < M.bins; b += blockDim.x) partials[(long long)blockIdx.x * M.bins + b] = bins[b];
}

// Shots: shot s lands in the first bin whose cumulative probability exceeds
// u_s (inverse CDF of the marginal; u_s uniform in [0, 1), supplied).
__global__ void k_sample(const double *cdf, int bins, const double *u, long long shots, unsigned long long *counts) {
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < shots; s += (long long)gridDim.x * blockDim.x) {
        const double x = u[s] * cdf[bins - 1];
        int lo = 0, hi = bins - 1;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (cdf[mid] > x) hi = mid;
            else lo = mid + 1;
        }
        atomicAdd(&counts[lo], 1ull);
    }
}

// Inclusive prefix sum of the marginal, one thread, in bin order.
__global__ void k_cdf(const double *marg, int bins, double *cdf) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int b = 0; b < bins; ++b) {
            s += marg[b];
            cdf[b] = s;
        }
    }
}

constexpr int kMargBlocks = 64;

template <typename R>
cudaError_t launch_marginal_dims(const Launch &L, const cplx<R> *psi, const int *dims, int n, const int *idx, int k,
                                 double *partials, double *out_dev) {
    MargArgs M;
    M.k = k;
    M.bins = 1;
    for (int a = 0; a < k; ++a) {
        long long s = 1;
        for (int i = idx[a] + 1; i < n; ++i) s *= dims[i];
        M.stride[a] = s;
        M.dim[a] = dims[idx[a]];
        M.bins *= dims[idx[a]];
    }
    long long N = 1;
    for (int i = 0; i < n; ++i) N *= dims[i];
    long long b = (N + 255) / 256;
    int blocks = (int)(b < kMargBlocks ? b : kMargBlocks);
    const size_t smem = (size_t)M.bins * sizeof(double);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_marginal<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k_marginal<R><<<blocks, 256, smem, L.stream>>>(psi, N, M, partials);
    k_sum_partials<<<1, sum_threads(M.bins), 0, L.stream>>>(partials, blocks, M.bins, out_dev);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_marginal(const Launch &L, const cplx<R> *psi, int d, int n, const int *idx, int k, double *partials,
                            double *out_dev) {
    int dims[kMaxQudits];
    for (int i = 0; i < n; ++i) dims[i] = d;
    return launch_marginal_dims<R>(L, psi, dims, n, idx, k, partials, out_dev);
}

int marginal_max_blocks() { return kMargBlocks; }

cudaError_t launch_sample(const Launch &L, const double *marg, int bins, double *cdf, const double *u, long long shots,
                          unsigned long long *counts) {
    cudaError_t e = cudaMemsetAsync(counts, 0, (size_t)bins * sizeof(unsigned long long), L.stream);
    if (e != cudaSuccess) return e;
    k_cdf<<<1, 32, 0, L.stream>>>(marg, bins, cdf);
    if (shots > 0) {
        long long b = (shots + 255) / 256;
        int blocks = (int)(b < 4LL * L.num_sms ? b : 4LL * L.num_sms);
        k_sample<<<blocks, 256, 0, L.stream>>>(cdf, bins, u, shots, counts);
    }
    return cudaGetLastError();
}

template cudaError_t launch_marginal<float>(const Launch &, const cplx<float> *, int, int, const int *, int, double *,
                                            double *);
template cudaError_t launch_marginal<double>(const Launch &, const cplx<double> *, int, int, const int *, int, double *,
                                             double *);
template cudaError_t launch_marginal_dims<float>(const Launch &, const cplx<float> *, const int *, int, const int *, int,
                                                 double *, double *);
template cudaError_t launch_marginal_dims<double>(const Launch &, const cplx<double> *, const int *, int, const int *,
                                                  int, double *, double *);

}  // namespace qf
