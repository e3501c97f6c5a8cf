// stage_device.cuh -- register-blocked application of a run of gates.
//
// A stage names K local qudits of a tile ("stage slots", most significant
// first).  Each thread takes blocks of d^K amplitudes -- all digit
// combinations of the K slots, every other local digit fixed -- loads a block
// from the shared-memory tile into registers, applies every op of the stage
// to it with compile-time register indices, and stores it back: one shared
// memory round trip for the whole run of gates instead of one per gate.
//
// Ops of a stage and where their qudits sit:
//   DENSE / PAIR / SHIFT        target in a slot
//   DIAG                        target in a slot, or outside: then its digit
//                               is constant over the block and the op is one
//                               phase on all d^K amplitudes
//   CPAIR / CDIAG / CSHIFT      target in a slot; control in another slot
//                               (digit fixed per fibre at compile time) or
//                               outside (digit constant over the block)
// Level pairs (j, k) are dispatched to compile-time cases, so d <= 5.
// SWAP and custom k-qudit gates run as their own shared-memory op.
#pragma once
#include "tile_device.cuh"

namespace qf {

__host__ __device__ __forceinline__ constexpr int cpow(int d, int e) {
    int r = 1;
    for (int i = 0; i < e; ++i) r *= d;
    return r;
}

// slots per stage of a kernel (0: no register stages); see stage_k
template <typename R, int D, bool ADJ> struct StageK {
    static constexpr int K = D > 0 ? stage_k(D, ADJ, sizeof(R) == 8) : 0;
};

// Stage-slot fields reuse TOp: sa = slot of the target, sc = slot of the
// control (-1: outside the stage).  They are packed into TOp::q[4], q[5].
__device__ __forceinline__ int op_sa(const TOp &o) { return o.q[4]; }
__device__ __forceinline__ int op_sc(const TOp &o) { return o.q[5]; }

// ---------------------------------------------------------------- fibre kernels on registers
// Fibre f of slot S: base index b = (f / RS) * RS * D + f % RS, elements b + m RS.
template <int D, int K, int S>
struct Fib {
    static constexpr int RS = cpow(D, K - 1 - S);
    static constexpr int DK = cpow(D, K);
    static constexpr int NF = DK / D;
    __host__ __device__ static constexpr int base(int f) { return (f / RS) * RS * D + f % RS; }
};

// Complex64 arithmetic on paired FP32 lanes: with a matrix entry prepared as
// P = (re, re | -im, im), P.lo * a + P.hi * (a.y, a.x) is the complex product.
__device__ __forceinline__ float2 pc_mul(const float4 &P, float2 a) {
    const float2 r = __fmul2_rn(make_float2(P.x, P.y), a);
    return __ffma2_rn(make_float2(P.z, P.w), make_float2(a.y, a.x), r);
}
__device__ __forceinline__ float2 pc_mac(const float4 &P, float2 a, float2 as, float2 acc) {
    acc = __ffma2_rn(make_float2(P.x, P.y), a, acc);
    return __ffma2_rn(make_float2(P.z, P.w), as, acc);
}

template <typename R, int D, int K, int S>
__device__ __forceinline__ void reg_dense(cplx<R> *v, const cplx<R> *M, const float4 *P) {
    using F = Fib<D, K, S>;
#pragma unroll
    for (int f = 0; f < F::NF; ++f) {
        const int b = F::base(f);
        cplx<R> x[D];
#pragma unroll
        for (int m = 0; m < D; ++m) x[m] = v[b + m * F::RS];
        if constexpr (sizeof(R) == 4) {
            float2 xs[D];
#pragma unroll
            for (int m = 0; m < D; ++m) xs[m] = make_float2(x[m].y, x[m].x);
#pragma unroll
            for (int l = 0; l < D; ++l) {
                float2 acc = pc_mul(P[l * D], x[0]);
#pragma unroll
                for (int m = 1; m < D; ++m) acc = pc_mac(P[l * D + m], x[m], xs[m], acc);
                v[b + l * F::RS] = acc;
            }
        } else {
#pragma unroll
            for (int l = 0; l < D; ++l) {
                cplx<R> acc = cmul(M[l * D], x[0]);
#pragma unroll
                for (int m = 1; m < D; ++m) acc = cfma(M[l * D + m], x[m], acc);
                v[b + l * F::RS] = acc;
            }
        }
    }
}

// 2x2 on levels (J, L) of slot S; control: CI = in-stage control slot or -1
// (then ctl is the block's control level); controlled ops use M + 4 ctl and
// skip ctl = 0.
// real = true: the 2x2 block is real (RY-type; entries' imaginary parts
// zero), so each output is two paired real scalings in complex64.
template <typename R, int D, int K, int S, int J, int L, int CI>
__device__ __forceinline__ void reg_pair(cplx<R> *v, const cplx<R> *M, bool ctrl, int ctl_block, bool real) {
    using F = Fib<D, K, S>;
#pragma unroll
    for (int f = 0; f < F::NF; ++f) {
        const int b = F::base(f);
        int ctl = 0;
        if (ctrl) {
            if (CI >= 0) ctl = (b / cpow(D, K - 1 - (CI < 0 ? 0 : CI))) % D;
            else ctl = ctl_block;
            if (ctl == 0) continue;
        }
        const cplx<R> *Mc = ctrl ? M + 4 * ctl : M;
        const cplx<R> a = v[b + J * F::RS], c = v[b + L * F::RS];
        if constexpr (sizeof(R) == 4) {
            if (real) {
                const float m0 = Mc[0].x, m1 = Mc[1].x, m2 = Mc[2].x, m3 = Mc[3].x;
                v[b + J * F::RS] = __ffma2_rn(make_float2(m1, m1), c, __fmul2_rn(make_float2(m0, m0), a));
                v[b + L * F::RS] = __ffma2_rn(make_float2(m3, m3), c, __fmul2_rn(make_float2(m2, m2), a));
                continue;
            }
        }
        v[b + J * F::RS] = cfma(Mc[1], c, cmul(Mc[0], a));
        v[b + L * F::RS] = cfma(Mc[3], c, cmul(Mc[2], a));
    }
}

template <typename R, int D, int K, int S, int CI>
__device__ __forceinline__ void reg_diag(cplx<R> *v, const cplx<R> *M, int mask, bool ctrl, int ctl_block) {
    using F = Fib<D, K, S>;
#pragma unroll
    for (int f = 0; f < F::NF; ++f) {
        const int b = F::base(f);
        int ctl = 0;
        if (ctrl) {
            if (CI >= 0) ctl = (b / cpow(D, K - 1 - (CI < 0 ? 0 : CI))) % D;
            else ctl = ctl_block;
            if (ctl == 0) continue;
        }
        const cplx<R> *Mc = ctrl ? M + D * ctl : M;
#pragma unroll
        for (int l = 0; l < D; ++l)
            if ((mask >> l) & 1) v[b + l * F::RS] = cmul(Mc[l], v[b + l * F::RS]);
    }
}

template <typename R, int D, int K, int S, int CI>
__device__ __forceinline__ void reg_shift(cplx<R> *v, int s, bool ctrl, int ctl_block) {
    using F = Fib<D, K, S>;
#pragma unroll
    for (int f = 0; f < F::NF; ++f) {
        const int b = F::base(f);
        int sh = s;
        if (ctrl) {
            int ctl = CI >= 0 ? (b / cpow(D, K - 1 - (CI < 0 ? 0 : CI))) % D : ctl_block;
            sh = (s * ctl) % D;
        }
        if (sh == 0) continue;
        cplx<R> x[D];
#pragma unroll
        for (int m = 0; m < D; ++m) x[m] = v[b + m * F::RS];
        // out[(m + sh) mod D] = x[m]: select the source for every destination
#pragma unroll
        for (int t = 0; t < D; ++t) {
            cplx<R> y = x[0];
#pragma unroll
            for (int m = 1; m < D; ++m)
                if ((m + sh) % D == t) y = x[m];   // exactly one source m maps to t
            v[b + t * F::RS] = y;
        }
    }
}

// Gradient term of a parametrised op: sum over the fibres of the block of
// Im <lambda|G|psi> (times the control level for controlled ops).
template <typename R, int D, int K, int S, int J, int L, int CI>
__device__ __forceinline__ R reg_grad_pair(const cplx<R> *v, const cplx<R> *w, const cplx<R> *G, bool ctrl, int ctl_block) {
    using F = Fib<D, K, S>;
    R acc = 0;
#pragma unroll
    for (int f = 0; f < F::NF; ++f) {
        const int b = F::base(f);
        int ctl = 1;
        if (ctrl) {
            ctl = CI >= 0 ? (b / cpow(D, K - 1 - (CI < 0 ? 0 : CI))) % D : ctl_block;
            if (ctl == 0) continue;
        }
        const cplx<R> a = v[b + J * F::RS], c = v[b + L * F::RS];
        const cplx<R> la = w[b + J * F::RS], lc = w[b + L * F::RS];
        const cplx<R> ga = cfma(G[1], c, cmul(G[0], a));
        const cplx<R> gc = cfma(G[3], c, cmul(G[2], a));
        const R t = la.x * ga.y - la.y * ga.x + lc.x * gc.y - lc.y * gc.x;
        acc += ctrl ? t * (R)ctl : t;
    }
    return acc;
}

template <typename R, int D, int K, int S, int CI>
__device__ __forceinline__ R reg_grad_diag(const cplx<R> *v, const cplx<R> *w, const cplx<R> *G, int mask, bool ctrl,
                                           int ctl_block) {
    using F = Fib<D, K, S>;
    R acc = 0;
#pragma unroll
    for (int f = 0; f < F::NF; ++f) {
        const int b = F::base(f);
        int ctl = 1;
        if (ctrl) {
            ctl = CI >= 0 ? (b / cpow(D, K - 1 - (CI < 0 ? 0 : CI))) % D : ctl_block;
            if (ctl == 0) continue;
        }
        R t = 0;
#pragma unroll
        for (int l = 0; l < D; ++l)
            if ((mask >> l) & 1) {
                const cplx<R> a = v[b + l * F::RS], la = w[b + l * F::RS];
                t += G[l].x * (la.x * a.y - la.y * a.x);
            }
        acc += ctrl ? t * (R)ctl : t;
    }
    return acc;
}

// ---------------------------------------------------------------- dispatch
// pair index p of (j, k), j < k, in lexicographic order
template <int D>
__device__ __forceinline__ int pair_index(int j, int k) { return j * (2 * D - j - 1) / 2 + (k - j - 1); }

template <int D, int P, int J = 0, int L = 1>
struct PairOf {
    // walk (J, L) lexicographically P steps
    static constexpr int Jn = (L + 1 < D) ? J : J + 1;
    static constexpr int Ln = (L + 1 < D) ? L + 1 : J + 2;
    static constexpr int j = PairOf<D, P - 1, Jn, Ln>::j;
    static constexpr int k = PairOf<D, P - 1, Jn, Ln>::k;
};
template <int D, int J, int L>
struct PairOf<D, 0, J, L> {
    static constexpr int j = J;
    static constexpr int k = L;
};

// Calls f(integral S, integral P, integral CI) for the op's slot, pair and
// control slot; returns false if the combination is not compiled.
#define QF_FOR_SLOT(S_, ...)         \
    switch (S_) {                    \
    case 0: { constexpr int S = 0; __VA_ARGS__; } break; \
    case 1: if constexpr (K > 1) { constexpr int S = 1; __VA_ARGS__; } break; \
    case 2: if constexpr (K > 2) { constexpr int S = 2; __VA_ARGS__; } break; \
    case 3: if constexpr (K > 3) { constexpr int S = 3; __VA_ARGS__; } break; \
    default: break;                  \
    }

#define QF_FOR_CI(C_, ...)           \
    switch (C_) {                    \
    case -1: { constexpr int CI = -1; __VA_ARGS__; } break; \
    case 0: { constexpr int CI = 0; __VA_ARGS__; } break; \
    case 1: if constexpr (K > 1) { constexpr int CI = 1; __VA_ARGS__; } break; \
    case 2: if constexpr (K > 2) { constexpr int CI = 2; __VA_ARGS__; } break; \
    case 3: if constexpr (K > 3) { constexpr int CI = 3; __VA_ARGS__; } break; \
    default: break;                  \
    }

#define QF_FOR_PAIR(P_, ...)                                                               \
    switch (P_) {                                                                          \
    case 0: { constexpr int PJ = PairOf<D, 0>::j, PK = PairOf<D, 0>::k; __VA_ARGS__; } break; \
    case 1: if constexpr (D * (D - 1) / 2 > 1) { constexpr int PJ = PairOf<D, 1>::j, PK = PairOf<D, 1>::k; __VA_ARGS__; } break; \
    case 2: if constexpr (D * (D - 1) / 2 > 2) { constexpr int PJ = PairOf<D, 2>::j, PK = PairOf<D, 2>::k; __VA_ARGS__; } break; \
    case 3: if constexpr (D * (D - 1) / 2 > 3) { constexpr int PJ = PairOf<D, 3>::j, PK = PairOf<D, 3>::k; __VA_ARGS__; } break; \
    case 4: if constexpr (D * (D - 1) / 2 > 4) { constexpr int PJ = PairOf<D, 4>::j, PK = PairOf<D, 4>::k; __VA_ARGS__; } break; \
    case 5: if constexpr (D * (D - 1) / 2 > 5) { constexpr int PJ = PairOf<D, 5>::j, PK = PairOf<D, 5>::k; __VA_ARGS__; } break; \
    case 6: if constexpr (D * (D - 1) / 2 > 6) { constexpr int PJ = PairOf<D, 6>::j, PK = PairOf<D, 6>::k; __VA_ARGS__; } break; \
    case 7: if constexpr (D * (D - 1) / 2 > 7) { constexpr int PJ = PairOf<D, 7>::j, PK = PairOf<D, 7>::k; __VA_ARGS__; } break; \
    case 8: if constexpr (D * (D - 1) / 2 > 8) { constexpr int PJ = PairOf<D, 8>::j, PK = PairOf<D, 8>::k; __VA_ARGS__; } break; \
    case 9: if constexpr (D * (D - 1) / 2 > 9) { constexpr int PJ = PairOf<D, 9>::j, PK = PairOf<D, 9>::k; __VA_ARGS__; } break; \
    default: break;                                                                        \
    }

// Block-constant digit of local position `ls` (stride) in base index b.
template <int D>
__device__ __forceinline__ int block_digit(const FastDiv &f, int b) { return (int)(f.div((uint32_t)b) % (uint32_t)D); }

// Applies op to the register block v (psi) and, with ADJ, to w (lambda); with
// ADJ and a parametrised op, returns its gradient term (before U^+ is applied).
template <typename R, int D, int K, bool ADJ>
__device__ __forceinline__ R reg_apply(const TOp &op, cplx<R> *v, cplx<R> *w, const cplx<R> *mats, const float4 *prep,
                                       int base) {
    const cplx<R> *M = mats + op.mat;
    const float4 *PM = prep + op.mat;
    const int sa = op_sa(op), sc = op_sc(op);
    R g = 0;
    switch (op.kind) {
    case OP_DENSE:
        QF_FOR_SLOT(sa, { reg_dense<R, D, K, S>(v, M, PM); if (ADJ) reg_dense<R, D, K, S>(w, M, PM); })
        break;
    case OP_PAIR:
    case OP_CPAIR: {
        const bool ctrl = op.kind == OP_CPAIR;
        const int cb = (ctrl && sc < 0) ? block_digit<D>(op.fc, base) : 0;
        if (ctrl && sc < 0 && cb == 0) break;
        const int p = pair_index<D>(op.j, op.k);
        QF_FOR_SLOT(sa, QF_FOR_CI((ctrl ? sc : -1), QF_FOR_PAIR(p, {
            if (ADJ && op.gcol >= 0)
                g = reg_grad_pair<R, D, K, S, PJ, PK, CI>(v, w, mats + op.gmat, ctrl, cb);
            reg_pair<R, D, K, S, PJ, PK, CI>(v, M, ctrl, cb, op.s == 1);
            if (ADJ) reg_pair<R, D, K, S, PJ, PK, CI>(w, M, ctrl, cb, op.s == 1);
        })))
        break;
    }
    case OP_DIAG:
    case OP_CDIAG: {
        const bool ctrl = op.kind == OP_CDIAG;
        const int cb = (ctrl && sc < 0) ? block_digit<D>(op.fc, base) : 0;
        if (ctrl && sc < 0 && cb == 0) break;
        if (sa < 0) {
            // target outside the stage: one phase for the whole block
            const int dg = block_digit<D>(op.fa, base);
            if (!((op.mask >> dg) & 1)) break;
            constexpr int DK = cpow(D, K);
            const cplx<R> ph = M[dg];
            if (ADJ && op.gcol >= 0) {
                const R gl = mats[op.gmat + dg].x;
                R t = 0;
#pragma unroll
                for (int r = 0; r < DK; ++r) t += w[r].x * v[r].y - w[r].y * v[r].x;
                g = gl * t;
            }
#pragma unroll
            for (int r = 0; r < DK; ++r) {
                v[r] = cmul(ph, v[r]);
                if (ADJ) w[r] = cmul(ph, w[r]);
            }
            break;
        }
        QF_FOR_SLOT(sa, QF_FOR_CI((ctrl ? sc : -1), {
            if (ADJ && op.gcol >= 0) g = reg_grad_diag<R, D, K, S, CI>(v, w, mats + op.gmat, op.mask, ctrl, cb);
            reg_diag<R, D, K, S, CI>(v, M, op.mask, ctrl, cb);
            if (ADJ) reg_diag<R, D, K, S, CI>(w, M, op.mask, ctrl, cb);
        }))
        break;
    }
    case OP_SHIFT:
    case OP_CSHIFT: {
        const bool ctrl = op.kind == OP_CSHIFT;
        const int cb = (ctrl && sc < 0) ? block_digit<D>(op.fc, base) : 0;
        QF_FOR_SLOT(sa, QF_FOR_CI((ctrl ? sc : -1), {
            reg_shift<R, D, K, S, CI>(v, op.s, ctrl, cb);
            if (ADJ) reg_shift<R, D, K, S, CI>(w, op.s, ctrl, cb);
        }))
        break;
    }
    default:
        break;
    }
    return g;
}

// Runs one register stage over the tile(s).  gsum: per-thread gradient
// accumulators indexed by op.gcol (ADJ only; summed in FP64 afterwards).
// prep: complex64 pool entries prepared for paired FP32 arithmetic
// (prepare_pool), unused for complex128.
template <typename R, int D, int K, bool ADJ>
__device__ __forceinline__ void stage_run(const TStage &st, const TOp *ops, const cplx<R> *mats, const float4 *prep,
                                          cplx<R> *tp, cplx<R> *tl, int T, R *gsum) {
    constexpr int DK = cpow(D, K);
    const int nblk = T / DK;
    for (int blk = threadIdx.x; blk < nblk; blk += blockDim.x) {
        // insert a zero digit at every slot stride (ascending)
        int base = blk;
#pragma unroll
        for (int i = 0; i < K; ++i) {
            const int q = (int)st.fa[i].div((uint32_t)base);
            base = q * st.lsa[i] * D + (base - q * st.lsa[i]);
        }
        cplx<R> v[DK], w[ADJ ? DK : 1];
#pragma unroll
        for (int r = 0; r < DK; ++r) {
            int o = 0;
#pragma unroll
            for (int i = 0; i < K; ++i) o += ((r / cpow(D, K - 1 - i)) % D) * st.ls[i];
            v[r] = tp[base + o];
            if (ADJ) w[r] = tl[base + o];
        }
        for (int oi = 0; oi < st.nops; ++oi) {
            const TOp &op = ops[st.first + oi];
            const R g = reg_apply<R, D, K, ADJ>(op, v, w, mats, prep, base);
            if (ADJ && op.gcol >= 0) {
                // register accumulators: compile-time indices
#pragma unroll
                for (int c = 0; c < kMaxGrad; ++c)
                    if (c == op.gcol) gsum[c] += g;
            }
        }
#pragma unroll
        for (int r = 0; r < DK; ++r) {
            int o = 0;
#pragma unroll
            for (int i = 0; i < K; ++i) o += ((r / cpow(D, K - 1 - i)) % D) * st.ls[i];
            tp[base + o] = v[r];
            if (ADJ) tl[base + o] = w[r];
        }
    }
}

// Pool entries (re, im) -> (re, re, -im, im) for paired FP32 arithmetic.
template <typename R>
__device__ __forceinline__ void prepare_pool(const cplx<R> *mats, float4 *prep, int nmat) {
    if constexpr (sizeof(R) == 4)
        for (int i = threadIdx.x; i < nmat; i += blockDim.x) {
            const cplx<R> m = mats[i];
            prep[i] = make_float4(m.x, m.x, -m.y, m.y);
        }
}

}  // namespace qf
