// tile_device.cuh -- device helpers shared by the forward tile kernel
// (k_tile.cu) and the adjoint tile kernel (k_adjoint.cu): cp.async staging,
// the per-fibre action of every single-target gate kind, the cooperative
// application of one gate to a shared-memory tile, and tile base offsets.
#pragma once
#include "qf_internal.cuh"

namespace qf {

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
        for (int e = tid; e < T; e += blockDim.x) {
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
        for (int g = tid; g < G; g += blockDim.x) {
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
        for (int f = tid; f < F; f += blockDim.x) {
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

}  // namespace qf
