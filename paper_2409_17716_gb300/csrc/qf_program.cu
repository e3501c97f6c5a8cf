// qf_program.cu -- recorded circuits (the Circuit class of the paper's
// "Library Architecture") executed as planned passes.
//
// Running a program resolves every gate at the run's parameters (FP64 on the
// host), multiplies runs of single-qudit gates on the same qudit inside a
// pass into one d x d matrix, rounds entries to the state precision, uploads
// the op lists and matrix pools of all passes in one copy, and launches the
// passes in order on the state's stream.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>

#include "qf_host.h"

using namespace qf;

struct qf_program {
    int d = 0, n = 0;                  // d = 0: the qudits mix dimensions
    bool mixed = false;
    int dims[kMaxQudits] = {};         // per-qudit dimensions
    std::vector<HGate> gates;
    int num_params = 0;
    bool fuse = true;
    bool stages = true;                // register stages in tile passes
    bool jit = true;                   // tile passes compiled at plan time (qf_jit.cu)
    int jit_k = 0;                     // register slots per compiled stage (0: default per d)
    JitProgram *jitp = nullptr;        // compiled passes of `plan` (nullptr: not built)
    bool jit_c128 = false;
    bool jit_df = false;               // jitp holds double-float complex128 passes
    bool fp64 = false;                 // complex128 compiled passes in FP64 (default: double-float)
    JitProgram *jitadj = nullptr;      // compiled reverse passes of `adj_plan`
    bool jitadj_c128 = false;
    bool jitadj_df = false;
    int tile_qudits = 0, min_run_qudits = 0, max_ops = 0;   // planner overrides (0: default)
    bool plan_valid = false;
    bool plan_c128 = false;
    std::vector<PassPlan> plan;
    void *h_buf = nullptr;
    void *d_buf = nullptr;
    size_t cap = 0;
    cudaEvent_t up_ev = nullptr;
    bool up_pending = false;
    cudaEvent_t done_ev = nullptr;
    bool ran = false;
    int last_passes = -1;
    // per-pass timing (tracing): events accumulate over runs until read
    bool timing = false;
    std::vector<cudaEvent_t> tev;      // event pool
    int tused = 0;                     // events recorded since the last read
    std::vector<int> tbefore, tafter;  // event indices around each timed pass
    std::vector<int> tkind;            // 0 tile pass, 1 strided pass
    std::vector<double> tbytes;        // algorithmic HBM bytes of each pass
    // adjoint
    bool adj_valid = false;
    bool adj_c128 = false;
    std::vector<PassPlan> adj_plan;
    double *d_rows = nullptr;          // per-CTA gradient rows
    size_t rows_cap = 0;               // doubles
    double *d_res = nullptr;           // loss + gradient for the host-result entry point
    double *h_res = nullptr;
    size_t res_cap = 0;                // doubles
};

namespace qf {

#define QF_CUDA(call)                                        \
    do {                                                     \
        cudaError_t e_ = (call);                             \
        if (e_ != cudaSuccess) return cuda_error(e_, #call); \
    } while (0)

// Resolves one op of a pass: a single gate, or the product of a group of
// single-qudit gates (applied first to last).
static ROp resolve_group(const std::vector<HGate> &gates, const std::vector<int> &grp, int d, const double *params) {
    if (grp.size() == 1) {
        const HGate &g = gates[grp[0]];
        return resolve_gate(g, d, gate_angle(g, params));
    }
    std::vector<ROp> parts;
    bool all_diag = true;
    for (int gi : grp) {
        const HGate &g = gates[gi];
        parts.push_back(resolve_gate(g, d, gate_angle(g, params)));
        all_diag &= parts.back().op.kind == OP_DIAG;
    }
    ROp out;
    out.op = parts[0].op;
    if (all_diag) {
        out.op.kind = OP_DIAG;
        out.m.assign(d, cd(1, 0));
        int mask = 0;
        for (const ROp &p : parts)
            for (int l = 0; l < d; ++l)
                if ((p.op.mask >> l) & 1) {
                    out.m[l] *= p.m[l];
                    mask |= 1 << l;
                }
        out.op.mask = mask;
        return out;
    }
    std::vector<cd> M = dense_of(parts[0], d);
    for (size_t i = 1; i < parts.size(); ++i) {
        std::vector<cd> G = dense_of(parts[i], d), P((size_t)d * d, cd(0, 0));
        for (int r = 0; r < d; ++r)
            for (int c = 0; c < d; ++c) {
                cd acc(0, 0);
                for (int t = 0; t < d; ++t) acc += G[r * d + t] * M[t * d + c];
                P[r * d + c] = acc;
            }
        M.swap(P);
    }
    out.op.kind = OP_DENSE;
    out.m = M;
    return out;
}

static size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

static int popcount32(int x) {
    int c = 0;
    for (; x; x &= x - 1) ++c;
    return c;
}

// Algorithmic HBM bytes of one strided pass: the amplitudes the op reads and
// writes (touched rows of every fibre whose control level is not 0).
static double strided_bytes(const TOp &o, int d, long long N, int b) {
    const double fib = (double)N / d;
    double rows = d, frac = 1.0;
    switch (o.kind) {
    case OP_PAIR: rows = 2; break;
    case OP_DIAG: rows = popcount32(o.mask); break;
    case OP_CPAIR: rows = 2; frac = (double)(d - 1) / d; break;
    case OP_CDIAG: rows = popcount32(o.mask); frac = (double)(d - 1) / d; break;
    case OP_CSHIFT: frac = (double)(d - 1) / d; break;
    default: break;
    }
    return 2.0 * b * fib * rows * frac;
}

// Copies `host` into the program's device buffer on the state's stream (after
// every earlier use of the buffer by this program on any stream).
static qf_status upload(qf_program *p, qf_state *s, const std::vector<unsigned char> &host) {
    if (p->up_pending) {
        QF_CUDA(cudaEventSynchronize(p->up_ev));
        p->up_pending = false;
    }
    if (p->ran) QF_CUDA(cudaStreamWaitEvent(s->stream, p->done_ev, 0));
    if (host.size() > p->cap) {
        if (p->ran) QF_CUDA(cudaEventSynchronize(p->done_ev));
        if (p->h_buf) cudaFreeHost(p->h_buf);
        if (p->d_buf) cudaFree(p->d_buf);
        p->h_buf = p->d_buf = nullptr;
        p->cap = 0;
        size_t cap = align16(host.size() + host.size() / 2 + 1024);
        if (cudaMallocHost(&p->h_buf, cap) != cudaSuccess || cudaMalloc(&p->d_buf, cap) != cudaSuccess) {
            cudaGetLastError();
            return set_error(QF_ERR_OOM, "program buffer allocation failed");
        }
        p->cap = cap;
    }
    if (!host.empty()) {
        std::memcpy(p->h_buf, host.data(), host.size());
        QF_CUDA(cudaMemcpyAsync(p->d_buf, p->h_buf, host.size(), cudaMemcpyHostToDevice, s->stream));
        QF_CUDA(cudaEventRecord(p->up_ev, s->stream));
        p->up_pending = true;
    }
    return QF_OK;
}

// Prepared entries of a resolved op for a compiled tile pass: complex64 as
// (re, re, -im, im), complex128 as (re, im); 16 bytes each.
template <typename R>
static void append_prepared(const ROp &r, std::vector<unsigned char> &out) {
    for (const cd &z : r.m) {
        if (sizeof(R) == 4) {
            const float v[4] = {(float)z.real(), (float)z.real(), -(float)z.imag(), (float)z.imag()};
            out.insert(out.end(), (const unsigned char *)v, (const unsigned char *)v + 16);
        } else {
            const double v[2] = {z.real(), z.imag()};
            out.insert(out.end(), (const unsigned char *)v, (const unsigned char *)v + 16);
        }
    }
}

// Double-float entries of a resolved op for a complex128 pass in
// double-float arithmetic: each FP64 entry split as hi = nearest float,
// lo = nearest float to the remainder; 32 bytes (urh, urh, -uih, uih, url,
// url, -uil, uil).
static void append_prepared_df(const ROp &r, std::vector<unsigned char> &out) {
    for (const cd &z : r.m) {
        const float rh = (float)z.real(), ih = (float)z.imag();
        const float rl = (float)(z.real() - (double)rh), il = (float)(z.imag() - (double)ih);
        const float v[8] = {rh, rh, -ih, ih, rl, rl, -il, il};
        out.insert(out.end(), (const unsigned char *)v, (const unsigned char *)v + 32);
    }
}

static void drop_jit(qf_program *p) {
    if (p->jitp) {
        jit_free(p->jitp);
        p->jitp = nullptr;
    }
    if (p->jitadj) {
        jit_free(p->jitadj);
        p->jitadj = nullptr;
    }
}

// Localized ops of every tile pass in pool order (entries at `params`).
static std::vector<std::vector<TOp>> jit_ops(const qf_program *p, const double *params) {
    std::vector<std::vector<TOp>> ops(p->plan.size());
    for (size_t pi = 0; pi < p->plan.size(); ++pi) {
        const PassPlan &pp = p->plan[pi];
        if (pp.strided || pp.mc) continue;
        int off = 0;
        for (const auto &grp : pp.groups) {
            ROp r = resolve_group(p->gates, grp, p->d, params);
            TOp o = localize(r.op, pp.geom, pp.active, p->n, p->d);
            o.mat = off;
            off += (int)r.m.size();
            ops[pi].push_back(o);
        }
    }
    return ops;
}

// Forward run with the passes compiled for this plan.
// expect_out (device, n + 1 doubles, or nullptr): <N_q> and the norm of the
// final state, reduced inside the last pass where that pass can (a compiled
// complex64 tile pass), else by the separate reduction after it.
template <typename R>
static qf_status run_program_jit(qf_program *p, qf_state *s, const double *params, double *expect_out = nullptr) {
    using C = cplx<R>;
    const int d = p->d, n = p->n;
    const bool c128 = sizeof(R) == 8;
    const bool df = c128 && !p->fp64;
    if (!p->jitp || p->jit_c128 != c128 || p->jit_df != df) {
        drop_jit(p);
        std::vector<std::vector<TOp>> ops = jit_ops(p, params);
        qf_status st = jit_build(p->plan, ops, d, c128, p->jit_k, false, s->num_sms, &p->jitp, df);
        if (st != QF_OK) return st;
        p->jit_c128 = c128;
        p->jit_df = df;
    }
    // entries of every pass at these parameters; passes reading them from
    // global memory get a copy in the program's upload buffer
    const size_t np = p->plan.size();
    std::vector<std::vector<unsigned char>> prep(np);
    std::vector<ROp> single(np);
    std::vector<size_t> goff(np, 0);
    std::vector<unsigned char> host;
    for (size_t pi = 0; pi < np; ++pi) {
        const PassPlan &pp = p->plan[pi];
        if (pp.strided || pp.mc) {
            single[pi] = resolve_group(p->gates, pp.groups[0], d, params);
            continue;
        }
        for (const auto &grp : pp.groups) {
            const ROp r = resolve_group(p->gates, grp, d, params);
            if (df) append_prepared_df(r, prep[pi]);
            else append_prepared<R>(r, prep[pi]);
        }
        if (jit_pass_global_pool(p->jitp, pi)) {
            goff[pi] = align16(host.size());
            host.resize(goff[pi] + prep[pi].size());
            std::memcpy(host.data() + goff[pi], prep[pi].data(), prep[pi].size());
        }
    }
    qf_status ust = upload(p, s, host);
    if (ust != QF_OK) return ust;
    Launch L;
    L.stream = s->stream;
    L.num_sms = s->num_sms;
    C *psi = reinterpret_cast<C *>(s->data);
    int launched = 0;
    int prev_ev = -1;
    if (p->timing) {
        const size_t need = p->tused + np + 1;
        while (p->tev.size() < need) {
            cudaEvent_t ev;
            QF_CUDA(cudaEventCreate(&ev));
            p->tev.push_back(ev);
        }
        prev_ev = p->tused++;
        QF_CUDA(cudaEventRecord(p->tev[prev_ev], s->stream));
    }
    const long long N = ipow_ll(d, n);
    // double-float passes work on the state converted in place; strided and
    // multi-controlled passes (FP64 kernels) and the caller see double2
    bool packed = false;
    auto convert = [&](bool pack) -> qf_status {
        cudaError_t e = launch_df_convert(s->stream, s->num_sms, s->data, N, pack);
        if (e != cudaSuccess) return cuda_error(e, "double-float conversion");
        packed = pack;
        return QF_OK;
    };
    for (size_t pi = 0; pi < np; ++pi) {
        const PassPlan &pp = p->plan[pi];
        if (pp.strided || pp.mc) {
            const TOp &o = single[pi].op;
            if ((o.kind == OP_SHIFT && o.s == 0) || (o.kind == OP_DIAG && o.mask == 0) ||
                (o.kind == OP_MCSHIFT && o.s == 0))
                continue;
            if (packed) {
                qf_status cst = convert(false);
                if (cst != QF_OK) return cst;
            }
            std::vector<C> m(single[pi].m.size());
            for (size_t i = 0; i < m.size(); ++i) m[i] = mk<R>((R)single[pi].m[i].real(), (R)single[pi].m[i].imag());
            if (p->timing) {
                p->tkind.push_back(1);
                p->tbytes.push_back(pp.mc ? 2.0 * sizeof(C) * (double)N : strided_bytes(o, d, N, (int)sizeof(C)));
            }
            cudaError_t e = pp.mc ? launch_mc<R>(L, psi, uniform_shape(d, n), o, m.data(), (int)m.size())
                                  : launch_strided<R>(L, psi, d, n, o, m.data(), (int)m.size());
            if (e != cudaSuccess) return cuda_error(e, "program pass");
        } else {
            if (df && !packed) {
                qf_status cst = convert(true);
                if (cst != QF_OK) return cst;
            }
            if (p->timing) {
                p->tkind.push_back(0);
                p->tbytes.push_back(2.0 * sizeof(C) * (double)N);
            }
            const void *gp = jit_pass_global_pool(p->jitp, pi)
                                 ? (const void *)(reinterpret_cast<const unsigned char *>(p->d_buf) + goff[pi])
                                 : nullptr;
            double *rows = nullptr;
            if (expect_out && pi + 1 == np && jit_pass_reduces(p->jitp, pi) &&
                (size_t)jit_pass_grid(p->jitp, pi) * (n + 1) <=
                    (size_t)reduce_max_blocks(s->num_sms) * (kMaxQudits + 1 + kMaxD))
                rows = s->d_partials;
            qf_status st = jit_launch(p->jitp, pi, s->stream, psi, pp.geom, prep[pi].data(),
                                      (int)(prep[pi].size() / 16), gp, rows);
            if (st != QF_OK) return st;
        }
        ++launched;
        if (p->timing) {
            const int cur = p->tused++;
            QF_CUDA(cudaEventRecord(p->tev[cur], s->stream));
            p->tbefore.push_back(prev_ev);
            p->tafter.push_back(cur);
            prev_ev = cur;
        }
        if (expect_out && pi + 1 == np && !pp.strided && !pp.mc && jit_pass_reduces(p->jitp, pi) &&
            (size_t)jit_pass_grid(p->jitp, pi) * (n + 1) <=
                (size_t)reduce_max_blocks(s->num_sms) * (kMaxQudits + 1 + kMaxD)) {
            // the pass's per-CTA rows -> <N_q> and the norm (outside the pass timing)
            cudaError_t e = launch_sum_rows(s->stream, s->d_partials, jit_pass_grid(p->jitp, pi), n + 1, expect_out);
            if (e != cudaSuccess) return cuda_error(e, "fused <N_q> row sums");
            expect_out = nullptr;   // done
        }
    }
    if (packed) {
        qf_status cst = convert(false);
        if (cst != QF_OK) return cst;
    }
    if (expect_out) {   // not fused into the last pass
        cudaError_t e = launch_expect_number<R>(L, psi, d, n, s->d_partials, expect_out);
        if (e != cudaSuccess) return cuda_error(e, "<N_q> reduction");
    }
    QF_CUDA(cudaEventRecord(p->done_ev, s->stream));
    p->ran = true;
    p->last_passes = launched;
    return QF_OK;
}

template <typename R>
static qf_status run_program_t(qf_program *p, qf_state *s, const double *params, double *expect_out = nullptr) {
    using C = cplx<R>;
    const int d = p->d, n = p->n;
    const bool c128 = sizeof(R) == 8;
    if (!p->plan_valid || p->plan_c128 != c128) {
        p->plan = plan_passes(p->gates, d, n, c128, p->fuse, false, p->tile_qudits, p->max_ops, p->min_run_qudits);
        p->plan_valid = true;
        p->plan_c128 = c128;
        drop_jit(p);
    }
    if (p->jit) return run_program_jit<R>(p, s, params, expect_out);
    // resolve every pass; tile passes get their op list + pool in one buffer
    struct Built {
        bool strided = false, mc = false;
        ROp rop;
        size_t off = 0;
        int nops = 0, nmat = 0, nstages = 0;
    };
    std::vector<Built> built(p->plan.size());
    std::vector<unsigned char> host;
    for (size_t pi = 0; pi < p->plan.size(); ++pi) {
        const PassPlan &pp = p->plan[pi];
        Built &b = built[pi];
        b.strided = pp.strided;
        b.mc = pp.mc;
        if (pp.strided || pp.mc) {
            b.rop = resolve_group(p->gates, pp.groups[0], d, params);
            continue;
        }
        std::vector<TOp> ops;
        std::vector<C> pool;
        for (const auto &grp : pp.groups) {
            ROp r = resolve_group(p->gates, grp, d, params);
            TOp o = localize(r.op, pp.geom, pp.active, n, d);
            o.mat = (int)pool.size();
            for (const cd &z : r.m) pool.push_back(mk<R>((R)z.real(), (R)z.imag()));
            ops.push_back(o);
        }
        std::vector<TStage> stages = build_stages(ops, pp.geom, d, stage_k(d, false, c128));
        b.nops = (int)ops.size();
        b.nmat = (int)pool.size();
        b.nstages = (int)stages.size();
        b.off = align16(host.size());
        const size_t ops_at = b.off + align16(pool.size() * sizeof(C));
        const size_t st_at = ops_at + ops.size() * sizeof(TOp);
        host.resize(st_at + stages.size() * sizeof(TStage));
        std::memcpy(host.data() + b.off, pool.data(), pool.size() * sizeof(C));
        std::memcpy(host.data() + ops_at, ops.data(), ops.size() * sizeof(TOp));
        std::memcpy(host.data() + st_at, stages.data(), stages.size() * sizeof(TStage));
    }
    qf_status ust = upload(p, s, host);
    if (ust != QF_OK) return ust;
    Launch L;
    L.stream = s->stream;
    L.num_sms = s->num_sms;
    C *psi = reinterpret_cast<C *>(s->data);
    int launched = 0;
    int prev_ev = -1;
    if (p->timing) {
        const size_t need = p->tused + p->plan.size() + 1;
        while (p->tev.size() < need) {
            cudaEvent_t ev;
            QF_CUDA(cudaEventCreate(&ev));
            p->tev.push_back(ev);
        }
        prev_ev = p->tused++;
        QF_CUDA(cudaEventRecord(p->tev[prev_ev], s->stream));
    }
    const long long N = ipow_ll(d, n);
    for (size_t pi = 0; pi < p->plan.size(); ++pi) {
        const PassPlan &pp = p->plan[pi];
        const Built &b = built[pi];
        cudaError_t e;
        if (b.mc) {
            const TOp &o = b.rop.op;
            if (o.kind == OP_MCSHIFT && o.s == 0) continue;
            if (p->timing) {
                p->tkind.push_back(1);
                p->tbytes.push_back(2.0 * sizeof(C) * (double)N);
            }
            std::vector<C> m(b.rop.m.size());
            for (size_t i = 0; i < m.size(); ++i) m[i] = mk<R>((R)b.rop.m[i].real(), (R)b.rop.m[i].imag());
            e = launch_mc<R>(L, psi, uniform_shape(d, n), o, m.data(), (int)m.size());
        } else if (b.strided) {
            const TOp &o = b.rop.op;
            if ((o.kind == OP_SHIFT && o.s == 0) || (o.kind == OP_DIAG && o.mask == 0)) continue;
            if (p->timing) {
                p->tkind.push_back(1);
                p->tbytes.push_back(strided_bytes(o, d, N, (int)sizeof(C)));
            }
            std::vector<C> m(b.rop.m.size());
            for (size_t i = 0; i < m.size(); ++i) m[i] = mk<R>((R)b.rop.m[i].real(), (R)b.rop.m[i].imag());
            e = launch_strided<R>(L, psi, d, n, o, m.data(), (int)m.size());
        } else {
            if (p->timing) {
                p->tkind.push_back(0);
                p->tbytes.push_back(2.0 * sizeof(C) * (double)N);
            }
            const unsigned char *base = reinterpret_cast<const unsigned char *>(p->d_buf) + b.off;
            const C *pool = reinterpret_cast<const C *>(base);
            const TOp *ops = reinterpret_cast<const TOp *>(base + align16(b.nmat * sizeof(C)));
            const TStage *stg = reinterpret_cast<const TStage *>(ops + b.nops);
            e = launch_tile<R>(L, psi, d, pp.geom, b.nops, ops, pool, b.nmat, nullptr, nullptr,
                               p->stages ? stg : nullptr, b.nstages);
        }
        if (e != cudaSuccess) return cuda_error(e, "program pass");
        ++launched;
        if (p->timing) {
            const int cur = p->tused++;
            QF_CUDA(cudaEventRecord(p->tev[cur], s->stream));
            p->tbefore.push_back(prev_ev);
            p->tafter.push_back(cur);
            prev_ev = cur;
        }
    }
    QF_CUDA(cudaEventRecord(p->done_ev, s->stream));
    p->ran = true;
    p->last_passes = launched;
    return QF_OK;
}

// Reverse passes in execution order (last planned pass first) and, per
// tile pass, its ops in application order: U^+ entries at op.mat and, for a
// parametrised op, its generator entries at op.gmat with gradient column
// op.gcol.  With `prep`, also the prepared entries of every pass.
template <typename R>
static std::vector<std::vector<TOp>> adj_jit_ops(const qf_program *p, const std::vector<PassPlan> &exec,
                                                 const double *params, std::vector<std::vector<unsigned char>> *prep,
                                                 bool df = false) {
    std::vector<std::vector<TOp>> ops(exec.size());
    if (prep) prep->assign(exec.size(), std::vector<unsigned char>());
    for (size_t k = 0; k < exec.size(); ++k) {
        const PassPlan &pp = exec[k];
        if (pp.strided || pp.mc) continue;
        int off = 0, ncols = 0;
        for (int gi = (int)pp.groups.size() - 1; gi >= 0; --gi) {
            const auto &grp = pp.groups[gi];
            ROp r = dagger(resolve_group(p->gates, grp, p->d, params), p->d);
            TOp o = localize(r.op, pp.geom, pp.active, p->n, p->d);
            o.mat = off;
            off += (int)r.m.size();
            if (prep) {
                if (df) append_prepared_df(r, (*prep)[k]);
                else append_prepared<R>(r, (*prep)[k]);
            }
            o.gcol = -1;
            o.gmat = 0;
            const HGate &g0 = p->gates[grp[0]];
            if (grp.size() == 1 && gate_is_param(g0)) {
                o.gcol = ncols++;
                o.gmat = off;
                ROp gen;
                gen.m = generator_entries(g0, p->d);
                off += (int)gen.m.size();
                if (prep) {
                    if (df) append_prepared_df(gen, (*prep)[k]);
                    else append_prepared<R>(gen, (*prep)[k]);
                }
            }
            ops[k].push_back(o);
        }
    }
    return ops;
}

// Adjoint sweep with compiled reverse passes (same plan, gradient rows and
// gather as the generic sweep below).
template <typename R>
static qf_status run_adjoint_jit(qf_program *p, qf_state *psi, qf_state *lam, const double *params,
                                 const double *weights, double *loss_dev, double *grad_dev) {
    using C = cplx<R>;
    const int d = p->d, n = p->n;
    const bool c128 = sizeof(R) == 8;
    const int np = (int)p->adj_plan.size();
    const bool df = c128 && !p->fp64;   // double-float reverse passes (see run_program_jit)
    std::vector<PassPlan> exec(p->adj_plan.rbegin(), p->adj_plan.rend());
    if (!p->jitadj || p->jitadj_c128 != c128 || p->jitadj_df != df) {
        if (p->jitadj) {
            jit_free(p->jitadj);
            p->jitadj = nullptr;
        }
        std::vector<std::vector<TOp>> ops = adj_jit_ops<R>(p, exec, params, nullptr, df);
        qf_status st = jit_build(exec, ops, d, c128, p->jit_k, true, psi->num_sms, &p->jitadj, df);
        if (st != QF_OK) return st;
        p->jitadj_c128 = c128;
        p->jitadj_df = df;
    }
    std::vector<std::vector<unsigned char>> prep;
    adj_jit_ops<R>(p, exec, params, &prep, df);
    // gradient rows and terms: (rows base, CTAs, columns, column) per slot, in execution order
    std::vector<long long> rows_base(np, 0);
    std::vector<std::vector<std::array<long long, 4>>> terms(p->num_params);
    long long rows_total = 0;
    std::vector<ROp> single(np);
    for (int k = 0; k < np; ++k) {
        const PassPlan &pp = exec[k];
        if (pp.strided || pp.mc) {
            single[k] = dagger(resolve_group(p->gates, pp.groups[0], d, params), d);
            continue;
        }
        const int grid = jit_pass_grid(p->jitadj, k), nc = jit_pass_ncols(p->jitadj, k);
        rows_base[k] = rows_total;
        rows_total += (long long)grid * nc;
        int col = 0;
        for (int gi = (int)pp.groups.size() - 1; gi >= 0; --gi) {
            const auto &grp = pp.groups[gi];
            const HGate &g0 = p->gates[grp[0]];
            if (grp.size() == 1 && gate_is_param(g0)) terms[g0.slot].push_back({rows_base[k], grid, nc, col++});
        }
    }
    std::vector<unsigned char> host;
    std::vector<size_t> goff(np, 0);
    for (int k = 0; k < np; ++k)
        if (!exec[k].strided && !exec[k].mc && jit_pass_global_pool(p->jitadj, k)) {
            goff[k] = align16(host.size());
            host.resize(goff[k] + prep[k].size());
            std::memcpy(host.data() + goff[k], prep[k].data(), prep[k].size());
        }
    const size_t tb = gather_term_bytes();
    const size_t terms_off = align16(host.size());
    std::vector<int> first(p->num_params + 1, 0);
    host.resize(terms_off);
    for (int sl = 0; sl < p->num_params; ++sl) {
        first[sl + 1] = first[sl] + (int)terms[sl].size();
        for (auto &t : terms[sl]) {
            struct {
                long long base;
                int nrows, ncols, col, pad;
            } rec = {t[0], (int)t[1], (int)t[2], (int)t[3], 0};
            static_assert(sizeof(rec) == 24, "gather term layout");
            const size_t at = host.size();
            host.resize(at + tb);
            std::memcpy(host.data() + at, &rec, sizeof(rec));
        }
    }
    const size_t first_off = align16(host.size());
    host.resize(first_off + first.size() * sizeof(int));
    std::memcpy(host.data() + first_off, first.data(), first.size() * sizeof(int));
    if ((size_t)rows_total > p->rows_cap) {
        if (p->ran) QF_CUDA(cudaEventSynchronize(p->done_ev));
        if (p->d_rows) cudaFree(p->d_rows);
        p->d_rows = nullptr;
        p->rows_cap = 0;
        size_t cap = (size_t)rows_total + 1024;
        if (cudaMalloc(&p->d_rows, cap * sizeof(double)) != cudaSuccess) {
            cudaGetLastError();
            return set_error(QF_ERR_OOM, "gradient scratch allocation failed");
        }
        p->rows_cap = cap;
    }
    qf_status st = upload(p, psi, host);
    if (st != QF_OK) return st;
    Launch L;
    L.stream = psi->stream;
    L.num_sms = psi->num_sms;
    C *ps = reinterpret_cast<C *>(psi->data);
    C *ls = reinterpret_cast<C *>(lam->data);
    cudaError_t e = launch_number_obs<R>(L, ps, ls, d, n, weights, psi->d_partials, loss_dev);
    if (e != cudaSuccess) return cuda_error(e, "lambda = O psi");
    const unsigned char *dev = reinterpret_cast<const unsigned char *>(p->d_buf);
    const MixedShape ushape = uniform_shape(d, n);
    const long long N = ipow_ll(d, n);
    bool packed = false;
    auto convert = [&](bool pack) -> cudaError_t {
        cudaError_t ce = launch_df_convert(psi->stream, psi->num_sms, psi->data, N, pack);
        if (ce == cudaSuccess) ce = launch_df_convert(psi->stream, psi->num_sms, lam->data, N, pack);
        packed = pack;
        return ce;
    };
    for (int k = 0; k < np; ++k) {
        const PassPlan &pp = exec[k];
        if (df && packed != !pp.mc) {
            e = convert(!pp.mc);
            if (e != cudaSuccess) return cuda_error(e, "double-float conversion");
        }
        if (pp.mc) {
            const ROp &r = single[k];
            std::vector<C> m(r.m.size());
            for (size_t i = 0; i < m.size(); ++i) m[i] = mk<R>((R)r.m[i].real(), (R)r.m[i].imag());
            if (!(r.op.kind == OP_MCSHIFT && r.op.s == 0)) {
                e = launch_mc<R>(L, ps, ushape, r.op, m.data(), (int)m.size());
                if (e == cudaSuccess) e = launch_mc<R>(L, ls, ushape, r.op, m.data(), (int)m.size());
                if (e != cudaSuccess) return cuda_error(e, "adjoint multi-controlled gate");
            }
            continue;
        }
        const void *gp = jit_pass_global_pool(p->jitadj, k) ? (const void *)(dev + goff[k]) : nullptr;
        st = jit_launch_adj(p->jitadj, k, psi->stream, ps, ls, p->d_rows + rows_base[k], pp.geom, prep[k].data(),
                            (int)(prep[k].size() / 16), gp);
        if (st != QF_OK) return st;
    }
    if (packed) {
        e = convert(false);
        if (e != cudaSuccess) return cuda_error(e, "double-float conversion");
    }
    e = launch_grad_gather(L, p->d_rows, dev + terms_off, reinterpret_cast<const int *>(dev + first_off), p->num_params,
                           grad_dev);
    if (e != cudaSuccess) return cuda_error(e, "gradient gather");
    QF_CUDA(cudaEventRecord(p->done_ev, psi->stream));
    p->ran = true;
    p->last_passes = np;
    return QF_OK;
}

template <typename R>
static qf_status run_adjoint_t(qf_program *p, qf_state *psi, qf_state *lam, const double *params, const double *weights,
                               double *loss_dev, double *grad_dev) {
    using C = cplx<R>;
    const int d = p->d, n = p->n;
    const bool c128 = sizeof(R) == 8;
    if (!p->adj_valid || p->adj_c128 != c128) {
        p->adj_plan = plan_passes(p->gates, d, n, c128, p->fuse, true, p->tile_qudits, p->max_ops, p->min_run_qudits);
        p->adj_valid = true;
        p->adj_c128 = c128;
        if (p->jitadj) {
            jit_free(p->jitadj);
            p->jitadj = nullptr;
        }
    }
    if (p->jit) return run_adjoint_jit<R>(p, psi, lam, params, weights, loss_dev, grad_dev);
    const auto &plan = p->adj_plan;
    const int np = (int)plan.size();
    struct Built {
        size_t off = 0;
        int nops = 0, nmat = 0, ncols = 0, grid = 0, nstages = 0;
        long long rows_base = 0;
        bool mc = false;
        ROp rop;                                // mc passes: U^+
    };
    std::vector<Built> built(np);
    std::vector<unsigned char> host;
    // gradient terms per slot: (pass in execution order, column)
    std::vector<std::vector<std::pair<int, int>>> terms(p->num_params);
    long long rows_total = 0;
    for (int k = 0; k < np; ++k) {
        const PassPlan &pp = plan[np - 1 - k];   // execution order: last pass first
        Built &b = built[k];
        if (pp.mc) {                             // no angle: U^+ on psi and lambda
            b.mc = true;
            b.rop = dagger(resolve_group(p->gates, pp.groups[0], d, params), d);
            b.rows_base = rows_total;
            continue;
        }
        std::vector<TOp> ops;
        std::vector<C> pool;
        int ncols = 0;
        for (int gi = (int)pp.groups.size() - 1; gi >= 0; --gi) {
            const auto &grp = pp.groups[gi];
            ROp r = dagger(resolve_group(p->gates, grp, d, params), d);
            TOp o = localize(r.op, pp.geom, pp.active, n, d);
            o.mat = (int)pool.size();
            for (const cd &z : r.m) pool.push_back(mk<R>((R)z.real(), (R)z.imag()));
            o.gcol = -1;
            o.gmat = 0;
            const HGate &g0 = p->gates[grp[0]];
            if (grp.size() == 1 && gate_is_param(g0)) {
                o.gcol = ncols++;
                o.gmat = (int)pool.size();
                for (const cd &z : generator_entries(g0, d)) pool.push_back(mk<R>((R)z.real(), (R)z.imag()));
                terms[g0.slot].push_back({k, o.gcol});
            }
            ops.push_back(o);
        }
        std::vector<TStage> stages;
        if (p->stages && stage_k(d, true, c128) > 0) stages = build_stages(ops, pp.geom, d, stage_k(d, true, c128));
        b.nops = (int)ops.size();
        b.nmat = (int)pool.size();
        b.ncols = ncols;
        b.nstages = (int)stages.size();
        cudaError_t e = adj_grid<R>(psi->num_sms, d, pp.geom, b.nops, b.nmat, b.nstages, &b.grid);
        if (e != cudaSuccess) return cuda_error(e, "adjoint pass occupancy");
        b.rows_base = rows_total;
        rows_total += (long long)b.grid * ncols;
        b.off = align16(host.size());
        const size_t ops_at = b.off + align16(pool.size() * sizeof(C));
        const size_t st_at = ops_at + ops.size() * sizeof(TOp);
        host.resize(st_at + stages.size() * sizeof(TStage));
        std::memcpy(host.data() + b.off, pool.data(), pool.size() * sizeof(C));
        std::memcpy(host.data() + ops_at, ops.data(), ops.size() * sizeof(TOp));
        std::memcpy(host.data() + st_at, stages.data(), stages.size() * sizeof(TStage));
    }
    // gather table
    const size_t tb = gather_term_bytes();
    std::vector<unsigned char> tbuf;
    std::vector<int> first(p->num_params + 1, 0);
    for (int sl = 0; sl < p->num_params; ++sl) {
        first[sl + 1] = first[sl] + (int)terms[sl].size();
        for (auto &t : terms[sl]) {
            const Built &b = built[t.first];
            struct {
                long long base;
                int nrows, ncols, col, pad;
            } rec = {b.rows_base, b.grid, b.ncols, t.second, 0};
            static_assert(sizeof(rec) == 24, "gather term layout");
            size_t at = tbuf.size();
            tbuf.resize(at + tb);
            std::memcpy(tbuf.data() + at, &rec, sizeof(rec));
        }
    }
    const size_t terms_off = align16(host.size());
    host.resize(terms_off + tbuf.size());
    if (!tbuf.empty()) std::memcpy(host.data() + terms_off, tbuf.data(), tbuf.size());
    const size_t first_off = align16(host.size());
    host.resize(first_off + first.size() * sizeof(int));
    std::memcpy(host.data() + first_off, first.data(), first.size() * sizeof(int));

    // gradient rows scratch
    if ((size_t)rows_total > p->rows_cap) {
        if (p->ran) QF_CUDA(cudaEventSynchronize(p->done_ev));
        if (p->d_rows) cudaFree(p->d_rows);
        p->d_rows = nullptr;
        p->rows_cap = 0;
        size_t cap = (size_t)rows_total + 1024;
        if (cudaMalloc(&p->d_rows, cap * sizeof(double)) != cudaSuccess) {
            cudaGetLastError();
            return set_error(QF_ERR_OOM, "gradient scratch allocation failed");
        }
        p->rows_cap = cap;
    }
    qf_status st = upload(p, psi, host);
    if (st != QF_OK) return st;
    if (lam->stream != psi->stream) return set_error(QF_ERR_ARG, "psi and lambda must share a stream");

    Launch L;
    L.stream = psi->stream;
    L.num_sms = psi->num_sms;
    C *ps = reinterpret_cast<C *>(psi->data);
    C *ls = reinterpret_cast<C *>(lam->data);
    cudaError_t e = launch_number_obs<R>(L, ps, ls, d, n, weights, psi->d_partials, loss_dev);
    if (e != cudaSuccess) return cuda_error(e, "lambda = O psi");
    const unsigned char *dev = reinterpret_cast<const unsigned char *>(p->d_buf);
    const MixedShape ushape = uniform_shape(d, n);
    for (int k = 0; k < np; ++k) {
        const PassPlan &pp = plan[np - 1 - k];
        const Built &b = built[k];
        if (b.mc) {
            std::vector<C> m(b.rop.m.size());
            for (size_t i = 0; i < m.size(); ++i) m[i] = mk<R>((R)b.rop.m[i].real(), (R)b.rop.m[i].imag());
            if (!(b.rop.op.kind == OP_MCSHIFT && b.rop.op.s == 0)) {
                e = launch_mc<R>(L, ps, ushape, b.rop.op, m.data(), (int)m.size());
                if (e == cudaSuccess) e = launch_mc<R>(L, ls, ushape, b.rop.op, m.data(), (int)m.size());
                if (e != cudaSuccess) return cuda_error(e, "adjoint multi-controlled gate");
            }
            continue;
        }
        const C *pool = reinterpret_cast<const C *>(dev + b.off);
        const TOp *ops = reinterpret_cast<const TOp *>(dev + b.off + align16(b.nmat * sizeof(C)));
        const TStage *stg = b.nstages > 0 ? reinterpret_cast<const TStage *>(ops + b.nops) : nullptr;
        e = launch_tile_adj<R>(L, ps, ls, d, pp.geom, b.nops, ops, pool, b.nmat, stg, b.nstages, p->d_rows + b.rows_base,
                               b.ncols, b.grid);
        if (e != cudaSuccess) return cuda_error(e, "adjoint pass");
    }
    e = launch_grad_gather(L, p->d_rows, dev + terms_off, reinterpret_cast<const int *>(dev + first_off), p->num_params,
                           grad_dev);
    if (e != cudaSuccess) return cuda_error(e, "gradient gather");
    QF_CUDA(cudaEventRecord(p->done_ev, psi->stream));
    p->ran = true;
    p->last_passes = np;
    return QF_OK;
}

// ---------------------------------------------------------------- mixed registers
// Programs on registers that mix dimensions run gate by gate: single-qudit and
// controlled gates through the strided kernel on the target's own (d, S),
// multi-qudit dense gates and SWAPs through the group kernel.  Matrices of
// group gates are uploaded with the program's buffer in one copy.
template <typename R>
static qf_status mixed_run_t(qf_program *p, qf_state *s, const double *params) {
    using C = cplx<R>;
    const MixedShape shape = mixed_shape(p->dims, p->n);
    std::vector<ROp> ops;
    std::vector<std::vector<C>> ent;
    std::vector<size_t> dev_off;
    std::vector<unsigned char> host;
    for (const HGate &g : p->gates) {
        ops.push_back(resolve_gate_dims(g, p->dims, gate_angle(g, params)));
        const ROp &r = ops.back();
        std::vector<C> m(r.m.size());
        for (size_t i = 0; i < r.m.size(); ++i) m[i] = mk<R>((R)r.m[i].real(), (R)r.m[i].imag());
        size_t off = 0;
        if (!(is_single(r.op) || is_controlled(r.op)) && !m.empty()) {
            off = align16(host.size());
            host.resize(off + m.size() * sizeof(C));
            std::memcpy(host.data() + off, m.data(), m.size() * sizeof(C));
        } else if ((int)m.size() > kInlineMat) {
            return set_error(QF_ERR_UNSUPPORTED, "gate table too large for a mixed register");
        }
        ent.push_back(std::move(m));
        dev_off.push_back(off);
    }
    qf_status st = upload(p, s, host);
    if (st != QF_OK) return st;
    Launch L;
    L.stream = s->stream;
    L.num_sms = s->num_sms;
    C *psi = reinterpret_cast<C *>(s->data);
    const unsigned char *dev = reinterpret_cast<const unsigned char *>(p->d_buf);
    for (size_t i = 0; i < ops.size(); ++i) {
        const C *md = reinterpret_cast<const C *>(dev + dev_off[i]);
        cudaError_t e = mixed_launch<R>(L, psi, shape, ops[i].op, ent[i].data(), (int)ent[i].size(), md);
        if (e != cudaSuccess) return cuda_error(e, "mixed-register gate kernel");
    }
    QF_CUDA(cudaEventRecord(p->done_ev, s->stream));
    p->ran = true;
    p->last_passes = (int)ops.size();
    return QF_OK;
}

// Adjoint sweep of a mixed-register program: lambda = O psi, then for every
// gate from the last: gradient term of a parametrised gate and U^+ on psi and
// lambda in one kernel (k_strided_adj), or U^+ on both through the group
// kernel; per slot, the terms are summed in a fixed order.
template <typename R>
static qf_status mixed_adjoint_t(qf_program *p, qf_state *psi, qf_state *lam, const double *params,
                                 const double *weights, double *loss_dev, double *grad_dev) {
    using C = cplx<R>;
    const MixedShape shape = mixed_shape(p->dims, p->n);
    const int G = (int)p->gates.size();
    struct Step {
        ROp r;
        std::vector<C> m, gen;
        size_t off = 0;
        long long rows = 0, nrows = 0;
    };
    std::vector<Step> steps(G);
    std::vector<unsigned char> host;
    std::vector<std::vector<std::pair<long long, long long>>> terms(p->num_params);
    long long rows_total = 0;
    for (int k = 0; k < G; ++k) {
        const HGate &g = p->gates[G - 1 - k];   // execution order: last gate first
        Step &st = steps[k];
        const int dt = p->dims[gate_target(g)];
        st.r = dagger(resolve_gate_dims(g, p->dims, gate_angle(g, params)), dt);
        st.m.resize(st.r.m.size());
        for (size_t i = 0; i < st.r.m.size(); ++i) st.m[i] = mk<R>((R)st.r.m[i].real(), (R)st.r.m[i].imag());
        const bool strided = is_single(st.r.op) || is_controlled(st.r.op);
        if (!strided && !st.m.empty()) {
            st.off = align16(host.size());
            host.resize(st.off + st.m.size() * sizeof(C));
            std::memcpy(host.data() + st.off, st.m.data(), st.m.size() * sizeof(C));
        } else if ((int)st.m.size() > kInlineMat) {
            return set_error(QF_ERR_UNSUPPORTED, "gate table too large for a mixed register");
        }
        if (gate_is_param(g)) {
            for (const cd &z : generator_entries(g, dt)) st.gen.push_back(mk<R>((R)z.real(), (R)z.imag()));
            st.nrows = mixed_adj_rows(shape, st.r.op, psi->num_sms);
            st.rows = rows_total;
            rows_total += st.nrows;
            terms[g.slot].push_back({st.rows, st.nrows});
        }
    }
    // gather table: (base, nrows, ncols = 1, col = 0) per term, slot order
    const size_t tb = gather_term_bytes();
    std::vector<int> first(p->num_params + 1, 0);
    const size_t terms_off = align16(host.size());
    for (int sl = 0; sl < p->num_params; ++sl) {
        first[sl + 1] = first[sl] + (int)terms[sl].size();
        for (auto &t : terms[sl]) {
            struct {
                long long base;
                int nrows, ncols, col, pad;
            } rec = {t.first, (int)t.second, 1, 0, 0};
            static_assert(sizeof(rec) == 24, "gather term layout");
            const size_t at = host.size() < terms_off ? terms_off : host.size();
            host.resize(at + tb);
            std::memcpy(host.data() + at, &rec, sizeof(rec));
        }
    }
    const size_t first_off = align16(host.size());
    host.resize(first_off + first.size() * sizeof(int));
    std::memcpy(host.data() + first_off, first.data(), first.size() * sizeof(int));
    if ((size_t)rows_total > p->rows_cap) {
        if (p->ran) QF_CUDA(cudaEventSynchronize(p->done_ev));
        if (p->d_rows) cudaFree(p->d_rows);
        p->d_rows = nullptr;
        p->rows_cap = 0;
        size_t cap = (size_t)rows_total + 1024;
        if (cudaMalloc(&p->d_rows, cap * sizeof(double)) != cudaSuccess) {
            cudaGetLastError();
            return set_error(QF_ERR_OOM, "gradient scratch allocation failed");
        }
        p->rows_cap = cap;
    }
    qf_status stt = upload(p, psi, host);
    if (stt != QF_OK) return stt;
    Launch L;
    L.stream = psi->stream;
    L.num_sms = psi->num_sms;
    C *ps = reinterpret_cast<C *>(psi->data);
    C *ls = reinterpret_cast<C *>(lam->data);
    cudaError_t e = launch_number_obs_mixed<R>(L, ps, ls, shape, weights, psi->d_partials, loss_dev);
    if (e != cudaSuccess) return cuda_error(e, "lambda = O psi");
    const unsigned char *dev = reinterpret_cast<const unsigned char *>(p->d_buf);
    for (int k = 0; k < G; ++k) {
        const Step &st = steps[k];
        const C *md = reinterpret_cast<const C *>(dev + st.off);
        e = mixed_adj_launch<R>(L, ps, ls, shape, st.r.op, st.m.data(), (int)st.m.size(), md,
                                st.gen.empty() ? nullptr : st.gen.data(), (int)st.gen.size(),
                                st.gen.empty() ? nullptr : p->d_rows + st.rows);
        if (e != cudaSuccess) return cuda_error(e, "mixed-register adjoint step");
    }
    e = launch_grad_gather(L, p->d_rows, dev + terms_off, reinterpret_cast<const int *>(dev + first_off), p->num_params,
                           grad_dev);
    if (e != cudaSuccess) return cuda_error(e, "gradient gather");
    QF_CUDA(cudaEventRecord(p->done_ev, psi->stream));
    p->ran = true;
    p->last_passes = G;
    return QF_OK;
}

qf_status mixed_program_run(qf_program *p, qf_state *s, const double *params) {
    return s->dt == QF_C64 ? mixed_run_t<float>(p, s, params) : mixed_run_t<double>(p, s, params);
}

qf_status mixed_program_adjoint(qf_program *p, qf_state *psi, qf_state *lam, const double *params,
                                const double *weights, double *loss_dev, double *grad_dev) {
    return psi->dt == QF_C64 ? mixed_adjoint_t<float>(p, psi, lam, params, weights, loss_dev, grad_dev)
                             : mixed_adjoint_t<double>(p, psi, lam, params, weights, loss_dev, grad_dev);
}

qf_status program_shape(const qf_program *p, int *d, int *n) {
    if (!p) return set_error(QF_ERR_ARG, "program is NULL");
    *d = p->d;
    *n = p->n;
    return QF_OK;
}

qf_status program_gates(const qf_program *p, std::vector<HGate> *out) {
    if (!p) return set_error(QF_ERR_ARG, "program is NULL");
    *out = p->gates;
    return QF_OK;
}

}  // namespace qf

extern "C" {

qf_status qf_program_create(int d, int n, qf_program **out) {
    if (!out) return set_error(QF_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (d < 2 || d > kMaxD || n < 1 || n > kMaxQudits) return set_error(QF_ERR_ARG, "d or n out of range");
    qf_program *p = new qf_program();
    p->d = d;
    p->n = n;
    for (int q = 0; q < n; ++q) p->dims[q] = d;
    *out = p;
    return QF_OK;
}

qf_status qf_program_create_dims(const int *dims, int n, qf_program **out) {
    if (!out) return set_error(QF_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!dims || n < 1 || n > kMaxQudits) return set_error(QF_ERR_ARG, "dims NULL or n out of range");
    int d = dims[0];
    for (int q = 0; q < n; ++q) {
        if (dims[q] < 2 || dims[q] > kMaxD) return set_error(QF_ERR_ARG, "every dimension must be in [2, 16]");
        if (dims[q] != d) d = 0;
    }
    qf_program *p = new qf_program();
    p->d = d;
    p->n = n;
    p->mixed = d == 0;
    for (int q = 0; q < n; ++q) p->dims[q] = dims[q];
    *out = p;
    return QF_OK;
}

static bool same_dims(const qf_program *p, const qf_state *s) {
    if (p->n != s->n || p->d != s->d) return false;
    for (int q = 0; q < p->n; ++q)
        if (p->dims[q] != s->dims[q]) return false;
    return true;
}

qf_status qf_program_free(qf_program *p) {
    if (!p) return QF_OK;
    if (p->ran && p->done_ev) cudaEventSynchronize(p->done_ev);
    if (p->up_pending && p->up_ev) cudaEventSynchronize(p->up_ev);
    if (p->h_buf) cudaFreeHost(p->h_buf);
    if (p->d_buf) cudaFree(p->d_buf);
    for (cudaEvent_t ev : p->tev) cudaEventDestroy(ev);
    if (p->d_rows) cudaFree(p->d_rows);
    if (p->d_res) cudaFree(p->d_res);
    drop_jit(p);
    if (p->h_res) cudaFreeHost(p->h_res);
    if (p->up_ev) cudaEventDestroy(p->up_ev);
    if (p->done_ev) cudaEventDestroy(p->done_ev);
    delete p;
    return QF_OK;
}

qf_status qf_program_info(const qf_program *p, int *num_gates, int *num_params) {
    if (!p) return set_error(QF_ERR_ARG, "program is NULL");
    if (num_gates) *num_gates = (int)p->gates.size();
    if (num_params) *num_params = p->num_params;
    return QF_OK;
}

static qf_status add(qf_program *p, HGate g) {
    if (!p) return set_error(QF_ERR_ARG, "program is NULL");
    qf_status st = p->mixed ? check_gate_dims(g, p->dims, p->n) : check_gate(g, p->d, p->n);
    if (st != QF_OK) return st;
    if (g.slot >= 0 && g.slot + 1 > p->num_params) p->num_params = g.slot + 1;
    p->gates.push_back(std::move(g));
    p->plan_valid = false;
    p->adj_valid = false;
    drop_jit(p);
    return QF_OK;
}

qf_status qf_program_add_gate(qf_program *p, const int *targets, int k, const double *U) {
    if (!p || !targets || !U || k < 1 || k > 6) return set_error(QF_ERR_ARG, "bad custom gate arguments");
    HGate g;
    g.kind = G_DENSE;
    g.nq = k;
    for (int i = 0; i < k; ++i) g.q[i] = targets[i];
    long long K = 1;
    for (int i = 0; i < k; ++i) {
        if (targets[i] < 0 || targets[i] >= p->n) return set_error(QF_ERR_ARG, "qudit index out of range [0, n)");
        K *= p->dims[targets[i]];
    }
    if (K > kMaxDenseK) return set_error(QF_ERR_UNSUPPORTED, "custom gate: the product of the targets' dims must be <= 64");
    g.U.resize((size_t)K * K);
    for (long long i = 0; i < K * K; ++i) g.U[i] = cd(U[2 * i], U[2 * i + 1]);
    return add(p, std::move(g));
}

qf_status qf_program_add_rot(qf_program *p, int q, int j, int k, char axis, int param_slot, double theta) {
    HGate g;
    g.kind = G_ROT; g.nq = 1; g.q[0] = q; g.j = j; g.k = k; g.axis = axis;
    g.slot = param_slot < 0 ? -1 : param_slot;
    g.theta = param_slot < 0 ? theta : 0.0;
    return add(p, g);
}

qf_status qf_program_add_crot(qf_program *p, int c, int t, int j, int k, char axis, int param_slot, double theta) {
    HGate g;
    g.kind = G_CROT; g.nq = 2; g.q[0] = c; g.q[1] = t; g.j = j; g.k = k; g.axis = axis;
    g.slot = param_slot < 0 ? -1 : param_slot;
    g.theta = param_slot < 0 ? theta : 0.0;
    return add(p, g);
}

static qf_status mc_gate(HGate *g, int kind, const int *controls, const int *levels, int k, int target) {
    if (!controls || k < 1 || k > 5) return set_error(QF_ERR_ARG, "need 1..5 controls");
    if (kind == G_MCU && !levels) return set_error(QF_ERR_ARG, "levels are NULL");
    g->kind = kind;
    g->nq = k + 1;
    for (int i = 0; i < k; ++i) {
        g->q[i] = controls[i];
        g->lv[i] = levels ? levels[i] : 0;
    }
    g->q[k] = target;
    return QF_OK;
}

qf_status qf_program_add_mcx(qf_program *p, const int *controls, int k, int target, int shift) {
    HGate g;
    qf_status st = mc_gate(&g, G_MCX, controls, nullptr, k, target);
    if (st != QF_OK) return st;
    g.power = shift;
    return add(p, g);
}

qf_status qf_program_add_mcu(qf_program *p, const int *controls, const int *levels, int k, int target, const double *U) {
    if (!p) return set_error(QF_ERR_ARG, "program is NULL");
    HGate g;
    qf_status st = mc_gate(&g, G_MCU, controls, levels, k, target);
    if (st != QF_OK) return st;
    if (!U) return set_error(QF_ERR_ARG, "U is NULL");
    if (target < 0 || target >= p->n) return set_error(QF_ERR_ARG, "qudit index out of range [0, n)");
    const int dt = p->dims[target];
    g.U.resize((size_t)dt * dt);
    for (int i = 0; i < dt * dt; ++i) g.U[i] = cd(U[2 * i], U[2 * i + 1]);
    return add(p, g);
}

qf_status qf_program_add_sum(qf_program *p, int c, int t) {
    HGate g; g.kind = G_SUM; g.nq = 2; g.q[0] = c; g.q[1] = t;
    return add(p, g);
}

qf_status qf_program_add_swap(qf_program *p, int a, int b) {
    HGate g; g.kind = G_SWAP; g.nq = 2; g.q[0] = a; g.q[1] = b;
    return add(p, g);
}

qf_status qf_program_add_x(qf_program *p, int q, int shift) {
    HGate g; g.kind = G_X; g.nq = 1; g.q[0] = q; g.power = shift;
    return add(p, g);
}

qf_status qf_program_add_z(qf_program *p, int q, int power) {
    HGate g; g.kind = G_Z; g.nq = 1; g.q[0] = q; g.power = power;
    return add(p, g);
}

qf_status qf_program_add_h(qf_program *p, int q) {
    HGate g; g.kind = G_H; g.nq = 1; g.q[0] = q;
    return add(p, g);
}

qf_status qf_program_set_tiling(qf_program *p, int tile_qudits, int min_run_qudits, int max_ops) {
    if (!p) return set_error(QF_ERR_ARG, "program is NULL");
    if (tile_qudits < 0 || min_run_qudits < 0 || max_ops < 0) return set_error(QF_ERR_ARG, "negative tiling value");
    p->tile_qudits = tile_qudits;
    p->min_run_qudits = min_run_qudits;
    p->max_ops = max_ops;
    p->plan_valid = false;
    p->adj_valid = false;
    drop_jit(p);
    return QF_OK;
}

qf_status qf_program_jit_source(qf_program *p, qf_dtype dt, int adjoint, char *buf, size_t cap, size_t *len) {
    if (!p) return set_error(QF_ERR_ARG, "program is NULL");
    if (p->mixed) return set_error(QF_ERR_UNSUPPORTED, "mixed-dimension programs run gate by gate");
    const bool c128 = dt == QF_C128;
    std::vector<double> zeros((size_t)std::max(1, p->num_params), 0.0);
    std::string src;
    qf_status st;
    if (adjoint) {
        if (!p->adj_valid || p->adj_c128 != c128) {
            p->adj_plan = plan_passes(p->gates, p->d, p->n, c128, p->fuse, true, p->tile_qudits, p->max_ops,
                                      p->min_run_qudits);
            p->adj_valid = true;
            p->adj_c128 = c128;
            if (p->jitadj) {
                jit_free(p->jitadj);
                p->jitadj = nullptr;
            }
        }
        std::vector<PassPlan> exec(p->adj_plan.rbegin(), p->adj_plan.rend());
        std::vector<std::vector<TOp>> ops = c128 ? adj_jit_ops<double>(p, exec, zeros.data(), nullptr)
                                                 : adj_jit_ops<float>(p, exec, zeros.data(), nullptr);
        st = jit_source(exec, ops, p->d, c128, p->jit_k, true, &src, c128 && !p->fp64);
    } else {
        if (!p->plan_valid || p->plan_c128 != c128) {
            p->plan = plan_passes(p->gates, p->d, p->n, c128, p->fuse, false, p->tile_qudits, p->max_ops,
                                  p->min_run_qudits);
            p->plan_valid = true;
            p->plan_c128 = c128;
            drop_jit(p);
        }
        std::vector<std::vector<TOp>> ops = jit_ops(p, zeros.data());
        st = jit_source(p->plan, ops, p->d, c128, p->jit_k, false, &src, c128 && !p->fp64);
    }
    if (st != QF_OK) return st;
    if (len) *len = src.size() + 1;
    if (buf && cap > 0) {
        const size_t nb = std::min(cap - 1, src.size());
        std::memcpy(buf, src.data(), nb);
        buf[nb] = 0;
    }
    return QF_OK;
}

qf_status qf_program_set_jit(qf_program *p, int enable) {
    if (!p) return set_error(QF_ERR_ARG, "program is NULL");
    p->jit = enable != 0;
    drop_jit(p);
    return QF_OK;
}

qf_status qf_program_set_stage_slots(qf_program *p, int slots) {
    if (!p) return set_error(QF_ERR_ARG, "program is NULL");
    if (slots < 0 || slots > kMaxStageK) return set_error(QF_ERR_ARG, "stage slots must be in [0, 6]");
    p->jit_k = slots;
    drop_jit(p);
    return QF_OK;
}

qf_status qf_program_set_fp64(qf_program *p, int exact) {
    if (!p) return set_error(QF_ERR_ARG, "program is NULL");
    if (p->fp64 != (exact != 0)) {
        p->fp64 = exact != 0;
        if (p->jit_c128) drop_jit(p);
    }
    return QF_OK;
}

qf_status qf_program_set_fusion(qf_program *p, int enable) {
    if (!p) return set_error(QF_ERR_ARG, "program is NULL");
    p->fuse = enable != 0;
    p->plan_valid = false;
    p->adj_valid = false;
    drop_jit(p);
    return QF_OK;
}

qf_status qf_program_run(qf_program *p, qf_state *s, const double *params) {
    if (!p || !s) return set_error(QF_ERR_ARG, "program or state is NULL");
    if (!same_dims(p, s)) return set_error(QF_ERR_ARG, "program and state sizes differ");
    if (p->num_params > 0 && !params) return set_error(QF_ERR_ARG, "program needs parameters");
    if (p->gates.empty()) {
        p->last_passes = 0;
        return QF_OK;
    }
    if (!p->up_ev) {
        if (cudaEventCreateWithFlags(&p->up_ev, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&p->done_ev, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            return set_error(QF_ERR_CUDA, "event creation failed");
        }
    }
    if (p->mixed) return mixed_program_run(p, s, params);
    return s->dt == QF_C64 ? run_program_t<float>(p, s, params) : run_program_t<double>(p, s, params);
}

qf_status qf_program_run_expect(qf_program *p, qf_state *s, const double *params, double *out_dev) {
    if (!out_dev || ((uintptr_t)out_dev & 7) != 0)
        return set_error(QF_ERR_ARG, "qf_program_run_expect: output must be a non-NULL 8-byte aligned device pointer");
    if (!p || !s) return set_error(QF_ERR_ARG, "program or state is NULL");
    if (!same_dims(p, s)) return set_error(QF_ERR_ARG, "program and state sizes differ");
    if (p->num_params > 0 && !params) return set_error(QF_ERR_ARG, "program needs parameters");
    if (p->mixed || p->gates.empty() || !p->jit) {
        qf_status st = qf_program_run(p, s, params);
        if (st != QF_OK) return st;
        qf_obs obs = {QF_OBS_NUMBER_ALL, 0, nullptr};
        return qf_expect_device(s, &obs, out_dev);
    }
    if (!p->up_ev) {
        if (cudaEventCreateWithFlags(&p->up_ev, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&p->done_ev, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            return set_error(QF_ERR_CUDA, "event creation failed");
        }
    }
    return s->dt == QF_C64 ? run_program_t<float>(p, s, params, out_dev) : run_program_t<double>(p, s, params, out_dev);
}

qf_status qf_program_plan(qf_program *p, qf_dtype dt, int *num_passes, int *num_strided, int *max_ops) {
    if (!p) return set_error(QF_ERR_ARG, "program is NULL");
    if (p->mixed) {   // one launch per gate
        if (num_passes) *num_passes = (int)p->gates.size();
        if (num_strided) *num_strided = (int)p->gates.size();
        if (max_ops) *max_ops = p->gates.empty() ? 0 : 1;
        return QF_OK;
    }
    const bool c128 = dt == QF_C128;
    if (!p->plan_valid || p->plan_c128 != c128) {
        p->plan = plan_passes(p->gates, p->d, p->n, c128, p->fuse, false, p->tile_qudits, p->max_ops, p->min_run_qudits);
        p->plan_valid = true;
        p->plan_c128 = c128;
        drop_jit(p);
    }
    int ns = 0, mo = 0;
    for (const PassPlan &pp : p->plan) {
        ns += pp.strided ? 1 : 0;
        mo = std::max(mo, (int)pp.groups.size());
    }
    if (num_passes) *num_passes = (int)p->plan.size();
    if (num_strided) *num_strided = ns;
    if (max_ops) *max_ops = mo;
    return QF_OK;
}

// Complex multiply-adds per amplitude of one resolved op (a real entry
// counts half): what the arithmetic units execute, independent of HBM.
static double op_cmacs(const TOp &o, int d) {
    const double ctrl = (double)(d - 1) / d;   // control level 0 is the identity
    int pc = 0;
    for (int m = o.mask; m; m &= m - 1) ++pc;
    switch (o.kind) {
    case OP_DENSE: return d;
    case OP_PAIR: return (o.s == 1 ? 2.0 : 4.0) / d;
    case OP_DIAG: return (double)pc / d;
    case OP_CPAIR: return ctrl * (o.s == 1 ? 2.0 : 4.0) / d;
    case OP_CDIAG: return ctrl * (double)pc / d;
    case OP_DENSEK: {
        double k = 1;
        for (int i = 0; i < o.nq; ++i) k *= d;
        return k;
    }
    default: return 0.0;   // permutations (shift, SUM, SWAP, multi-controlled shift)
    }
}

qf_status qf_program_cmacs(qf_program *p, qf_dtype dt, double *cmacs_per_amplitude) {
    if (!p || !cmacs_per_amplitude) return set_error(QF_ERR_ARG, "program or output is NULL");
    if (p->mixed) return set_error(QF_ERR_UNSUPPORTED, "qf_program_cmacs: mixed-dimension programs");
    qf_status st = qf_program_plan(p, dt, nullptr, nullptr, nullptr);
    if (st != QF_OK) return st;
    std::vector<double> zeros((size_t)std::max(p->num_params, 1), 0.0);
    double total = 0.0;
    for (const PassPlan &pp : p->plan)
        for (const auto &grp : pp.groups) {
            const ROp r = resolve_group(p->gates, grp, p->d, zeros.data());
            if (r.op.kind == OP_MCDENSE) {
                // changes the fibres whose controls sit at their levels
                total += p->d / std::pow((double)p->d, (double)r.op.nq);
            } else {
                total += op_cmacs(r.op, p->d);
            }
        }
    *cmacs_per_amplitude = total;
    return QF_OK;
}

qf_status qf_program_stages(qf_program *p, qf_dtype dt, int *num_tile_passes, int *num_stages, int *num_ops) {
    if (!p) return set_error(QF_ERR_ARG, "program is NULL");
    if (p->mixed) {
        if (num_tile_passes) *num_tile_passes = 0;
        if (num_stages) *num_stages = 0;
        if (num_ops) *num_ops = (int)p->gates.size();
        return QF_OK;
    }
    const bool c128 = dt == QF_C128;
    if (!p->plan_valid || p->plan_c128 != c128) {
        p->plan = plan_passes(p->gates, p->d, p->n, c128, p->fuse, false, p->tile_qudits, p->max_ops, p->min_run_qudits);
        p->plan_valid = true;
        p->plan_c128 = c128;
        drop_jit(p);
    }
    int tp = 0, ns = 0, no = 0;
    for (const PassPlan &pp : p->plan) {
        if (pp.strided || pp.mc) continue;
        std::vector<TOp> ops;
        for (const auto &grp : pp.groups) {
            ROp r = resolve_group(p->gates, grp, p->d, nullptr);
            ops.push_back(localize(r.op, pp.geom, pp.active, p->n, p->d));
        }
        std::vector<TStage> stages = build_stages(ops, pp.geom, p->d, stage_k(p->d, false, c128));
        ++tp;
        ns += stages.empty() ? (int)ops.size() : (int)stages.size();
        no += (int)ops.size();
    }
    if (num_tile_passes) *num_tile_passes = tp;
    if (num_stages) *num_stages = ns;
    if (num_ops) *num_ops = no;
    return QF_OK;
}

static qf_status ensure_events(qf_program *p) {
    if (!p->up_ev) {
        if (cudaEventCreateWithFlags(&p->up_ev, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&p->done_ev, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            return set_error(QF_ERR_CUDA, "event creation failed");
        }
    }
    return QF_OK;
}

qf_status qf_program_adjoint(qf_program *p, qf_state *psi, qf_state *lam, const double *params, const double *weights,
                             double *loss_dev, double *grad_dev) {
    if (!p || !psi || !lam) return set_error(QF_ERR_ARG, "program or state is NULL");
    if (psi == lam || psi->data == lam->data) return set_error(QF_ERR_ARG, "psi and lambda must be different states");
    if (!same_dims(p, psi) || !same_dims(p, lam) || lam->dt != psi->dt)
        return set_error(QF_ERR_ARG, "program and state sizes differ");
    if (!weights) return set_error(QF_ERR_ARG, "weights are NULL");
    if (!loss_dev || !grad_dev) return set_error(QF_ERR_ARG, "outputs are NULL");
    if (p->num_params > 0 && !params) return set_error(QF_ERR_ARG, "program needs parameters");
    qf_status st = ensure_events(p);
    if (st != QF_OK) return st;
    if (lam->stream != psi->stream) return set_error(QF_ERR_ARG, "psi and lambda must share a stream");
    if (p->mixed) return mixed_program_adjoint(p, psi, lam, params, weights, loss_dev, grad_dev);
    return psi->dt == QF_C64 ? run_adjoint_t<float>(p, psi, lam, params, weights, loss_dev, grad_dev)
                             : run_adjoint_t<double>(p, psi, lam, params, weights, loss_dev, grad_dev);
}

qf_status qf_program_gradient(qf_program *p, qf_state *psi, qf_state *lam, const double *params, const double *weights,
                              double *loss_host, double *grad_host) {
    if (!p || !psi || !lam) return set_error(QF_ERR_ARG, "program or state is NULL");
    if (!loss_host || (p->num_params > 0 && !grad_host)) return set_error(QF_ERR_ARG, "outputs are NULL");
    const size_t need = (size_t)p->num_params + 1;
    if (need > p->res_cap) {
        if (p->d_res) { cudaStreamSynchronize(psi->stream); cudaFree(p->d_res); }
        if (p->h_res) cudaFreeHost(p->h_res);
        p->d_res = nullptr;
        p->h_res = nullptr;
        p->res_cap = 0;
        if (cudaMalloc(&p->d_res, need * sizeof(double)) != cudaSuccess ||
            cudaMallocHost(&p->h_res, need * sizeof(double)) != cudaSuccess) {
            cudaGetLastError();
            return set_error(QF_ERR_OOM, "gradient result allocation failed");
        }
        p->res_cap = need;
    }
    qf_status st = qf_program_run(p, psi, params);
    if (st != QF_OK) return st;
    st = qf_program_adjoint(p, psi, lam, params, weights, p->d_res, p->d_res + 1);
    if (st != QF_OK) return st;
    QF_CUDA(cudaMemcpyAsync(p->h_res, p->d_res, need * sizeof(double), cudaMemcpyDeviceToHost, psi->stream));
    QF_CUDA(cudaStreamSynchronize(psi->stream));
    *loss_host = p->h_res[0];
    if (p->num_params > 0) std::memcpy(grad_host, p->h_res + 1, p->num_params * sizeof(double));
    return QF_OK;
}

int qf_program_last_passes(const qf_program *p) { return p ? p->last_passes : -1; }

static void timing_reset(qf_program *p) {
    p->tused = 0;
    p->tbefore.clear();
    p->tafter.clear();
    p->tkind.clear();
    p->tbytes.clear();
}

qf_status qf_program_set_timing(qf_program *p, int enable) {
    if (!p) return set_error(QF_ERR_ARG, "program is NULL");
    if (p->ran && p->done_ev) cudaEventSynchronize(p->done_ev);
    p->timing = enable != 0;
    timing_reset(p);
    return QF_OK;
}

qf_status qf_program_pass_times(qf_program *p, int max, float *ms, int *kind, double *bytes, int *count) {
    if (!p) return set_error(QF_ERR_ARG, "program is NULL");
    const int cnt = (int)p->tafter.size();
    if (count) *count = cnt;
    if (cnt > 0) {
        QF_CUDA(cudaEventSynchronize(p->tev[p->tafter[cnt - 1]]));
        for (int i = 0; i < cnt && i < max; ++i) {
            if (ms) QF_CUDA(cudaEventElapsedTime(ms + i, p->tev[p->tbefore[i]], p->tev[p->tafter[i]]));
            if (kind) kind[i] = p->tkind[i];
            if (bytes) bytes[i] = p->tbytes[i];
        }
    }
    timing_reset(p);
    return QF_OK;
}

}  // extern "C"
