// qf_internal.cuh -- shared declarations of the libqf CUDA implementation.
//
// Layout of a state: N = d^n amplitudes, interleaved (re, im), float2 for
// complex64 and double2 for complex128.  Basis index i = sum_q i_q d^(n-1-q)
// (Appendix B, "Generalized CNOT gate"), so qudit q has stride d^(n-1-q) and
// i = hi * (d * S) + l * S + lo with l the level of qudit q and S its stride.
//
// Two kernel families apply gates:
//   * the strided kernel (k_strided.cu): one thread per fibre {hi, ., lo} of
//     a single target whose stride S >= kWideMin, loads only the levels the
//     gate touches straight from HBM (coalesced along lo);
//   * the tile kernel (k_tile.cu): a CTA stages a tile of T = d^(kA + rL)
//     amplitudes in shared memory -- d^kA contiguous runs of d^rL amplitudes,
//     one per assignment of the kA "active" high qudits -- applies a whole
//     list of gates to it, and writes it back: one HBM round trip per pass.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/qf.h"

namespace qf {

constexpr int kMaxD = 16;          // largest qudit dimension supported
constexpr int kMaxQudits = 62;     // d^n must fit in int64 anyway
constexpr int kWideMin = 32;       // strided kernel needs S >= one warp
constexpr int kMaxTileOps = 96;    // gates per fused pass
constexpr int kMaxTileQ = 16;      // local qudits per tile
constexpr int kMaxActive = 10;     // active high qudits per tile
constexpr int kMaxDenseK = 64;     // d^k limit of the custom k-qudit gate
constexpr int kInlineMat = 256;    // complex entries passed by value

template <typename R> struct CT;
template <> struct CT<float> { using T = float2; };
template <> struct CT<double> { using T = double2; };

template <typename R> using cplx = typename CT<R>::T;

template <typename R> __host__ __device__ __forceinline__ cplx<R> mk(R x, R y) { cplx<R> c; c.x = x; c.y = y; return c; }
template <typename T> __host__ __device__ __forceinline__ T cadd(T a, T b) { T c; c.x = a.x + b.x; c.y = a.y + b.y; return c; }
template <typename T> __host__ __device__ __forceinline__ T cmul(T a, T b) {
    T c; c.x = a.x * b.x - a.y * b.y; c.y = a.x * b.y + a.y * b.x; return c;
}
// acc + a * b
template <typename T> __host__ __device__ __forceinline__ T cfma(T a, T b, T acc) {
    acc.x = fma(a.x, b.x, acc.x); acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y); acc.y = fma(a.y, b.x, acc.y);
    return acc;
}
__device__ __forceinline__ float2 cfma(float2 a, float2 b, float2 acc) {
    acc.x = fmaf(a.x, b.x, acc.x); acc.x = fmaf(-a.y, b.y, acc.x);
    acc.y = fmaf(a.x, b.y, acc.y); acc.y = fmaf(a.y, b.x, acc.y);
    return acc;
}

// Unsigned 32-bit division by a runtime constant via one multiply-high
// (Granlund & Montgomery, "Division by invariant integers using
// multiplication", PLDI 1994, the round-up variant with a 33-bit multiplier
// split as m' + 2^32).  Valid for every 32-bit dividend and divisor >= 1.
struct FastDiv {
    uint32_t d, m, s1, s2;
    __host__ __device__ FastDiv() : d(1), m(0), s1(0), s2(0) {}
    __host__ explicit FastDiv(uint32_t div) {
        d = div;
        uint32_t l = 0;
        while ((1ull << l) < div) ++l;           // l = ceil(log2 d)
        uint64_t mm = ((1ull << 32) * ((1ull << l) - div)) / div + 1;
        m = (uint32_t)mm;
        s1 = l > 0 ? 1 : 0;
        s2 = l > 0 ? l - 1 : 0;
    }
    __host__ __device__ __forceinline__ uint32_t div(uint32_t n) const {
#ifdef __CUDA_ARCH__
        uint32_t t = __umulhi(m, n);
#else
        uint32_t t = (uint32_t)(((uint64_t)m * n) >> 32);
#endif
        return (t + ((n - t) >> s1)) >> s2;
    }
};

// Gate kinds understood by both kernel families.
enum OpKind : int {
    OP_DENSE = 0,   // d x d matrix on qudit a                          mat: d*d
    OP_PAIR = 1,    // 2 x 2 on levels (j, k) of qudit a, rest untouched mat: 4 (jj, jk, kj, kk)
    OP_DIAG = 2,    // diagonal on qudit a; `mask` = levels != 1         mat: d
    OP_SHIFT = 3,   // |x> -> |x + s mod d> on qudit a                   mat: -
    OP_CPAIR = 4,   // control c level m: 2x2 (j,k) on a; m = 0 identity mat: 4*d
    OP_CDIAG = 5,   // control c level m: diagonal on a; m = 0 identity  mat: d*d
    OP_CSHIFT = 6,  // control c level m: shift a by (s * m) mod d        mat: -
    OP_SWAP = 7,    // exchange qudits a and c                          mat: -
    OP_DENSEK = 8,  // d^k x d^k on qudits q[0..k-1] (q[0] most significant) mat: d^(2k)
    OP_MCSHIFT = 9, // controls q[0..nq-1]: shift a by s * (product of their levels) mod d
    OP_MCDENSE = 10,// controls q[0..nq-1] at levels (4 bits each in mask): d x d on a   mat: d*d
};

// One gate, in qudit positions (global for the strided kernel, local tile
// positions for the tile kernel).
struct TOp {
    int kind;
    int a;          // target
    int c;          // control / second qudit
    int j, k;       // levels for PAIR kinds
    int s;          // shift amount / multiplier
    int mask;       // DIAG: bitmask of levels whose phase is not 1
    int mat;        // offset of the matrix in the pool (complex entries)
    int nq;         // DENSEK: number of targets
    int q[6];       // DENSEK targets
    // tile kernel only (filled by the planner): local strides of a and c and
    // divisors by them
    int lsa, lsc;
    FastDiv fa, fc;
    // adjoint only: column of this op in the pass's gradient row (-1: no
    // angle) and pool offset of its generator G (dU/dtheta = -i G U), laid out
    // like the op's matrix (PAIR kinds: 4 entries; DIAG kinds: d entries)
    int gcol, gmat;
    // batched programs only: rotation angle taken on the device from the
    // parameter vector (pslot >= 0), entries written into the pool at `mat`;
    // paxis = 'x','y','z','g'; psign = +1 forward, -1 adjoint (R(theta)^+ =
    // R(-theta))
    int pslot, paxis, psign;
};

static_assert(sizeof(TOp) % sizeof(int) == 0, "TOp is copied as ints");
static_assert(alignof(TOp) == 4, "TOp packs into shared memory after the matrix pool");

// A register stage of a tile pass (see stage_device.cuh): ops[first ..
// first+nops) applied to blocks of d^K amplitudes spanning K local qudits
// ("slots", strides ls, most significant first).  legacy = 1: the single op
// ops[first] is applied through shared memory instead.  The slot of an op's
// target and control within the stage are stored in TOp::q[4] and q[5]
// (-1: not a slot).
constexpr int kMaxStageK = 6;   // compiled passes; the generic kernels use at most 4
constexpr int kMaxGrad = 16;   // parametrised ops per adjoint pass (register accumulators)

struct TStage {
    int legacy;
    int first, nops;
    int ls[kMaxStageK];        // local strides of the slots, most significant first
    int lsa[kMaxStageK];       // the same strides ascending
    FastDiv fa[kMaxStageK];    // divisors by lsa
};

// Slots per register stage (0: shared-memory ops only), chosen so the
// register blocks (psi, and lambda for the adjoint) fit without spilling.
__host__ __device__ constexpr int stage_k(int d, bool adj, bool c128) {
    return d == 2   ? (adj ? (c128 ? 2 : 3) : (c128 ? 3 : 4))
           : d == 3 ? ((adj && c128) ? 1 : (adj || c128) ? 2 : 3)
           : (d == 4 || d == 5) ? ((adj || c128) ? 1 : 2)
                                : 0;
}

// Geometry of a tile pass.
struct TileGeom {
    int nt;                 // local qudits = kA + rL
    int rL;                 // low qudits stored contiguously
    int kA;                 // active high qudits
    int T;                  // amplitudes per tile = d^nt
    int SEG;                // d^rL
    long long ntiles;       // N / T
    long long strideA[kMaxActive];   // global strides of the active qudits, most significant first
    // tile index -> base offset: the outer (non-tile) qudits form nruns runs
    // of consecutive qudits; run r has radix M[r] = d^len and stride S[r];
    // runs are listed from least significant.
    int nruns;
    long long runM[kMaxActive + 1];
    long long runS[kMaxActive + 1];
    FastDiv divSEG;
};

// Host-side launch context.
struct Launch {
    cudaStream_t stream;
    int num_sms;
};

int device_sms();

}  // namespace qf
