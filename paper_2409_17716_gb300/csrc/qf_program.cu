// qf_program.cu -- recorded circuits (the Circuit class of the paper's
// "Library Architecture") executed as planned passes.
//
// Running a program resolves every gate at the run's parameters (FP64 on the
// host), multiplies runs of single-qudit gates on the same qudit inside a
// pass into one d x d matrix, rounds entries to the state precision, uploads
// the op lists and matrix pools of all passes in one copy, and launches the
// passes in order on the state's stream.
#include <algorithm>
#include <cstring>

#include "qf_host.h"

using namespace qf;

struct qf_program {
    int d = 0, n = 0;
    std::vector<HGate> gates;
    int num_params = 0;
    bool fuse = true;
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

template <typename R>
static qf_status run_program_t(qf_program *p, qf_state *s, const double *params) {
    using C = cplx<R>;
    const int d = p->d, n = p->n;
    const bool c128 = sizeof(R) == 8;
    if (!p->plan_valid || p->plan_c128 != c128) {
        p->plan = plan_passes(p->gates, d, n, c128, p->fuse);
        p->plan_valid = true;
        p->plan_c128 = c128;
    }
    // resolve every pass; tile passes get their op list + pool in one buffer
    struct Built {
        bool strided;
        ROp rop;
        size_t off = 0;
        int nops = 0, nmat = 0;
    };
    std::vector<Built> built(p->plan.size());
    std::vector<unsigned char> host;
    for (size_t pi = 0; pi < p->plan.size(); ++pi) {
        const PassPlan &pp = p->plan[pi];
        Built &b = built[pi];
        b.strided = pp.strided;
        if (pp.strided) {
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
        b.nops = (int)ops.size();
        b.nmat = (int)pool.size();
        b.off = align16(host.size());
        size_t need = b.off + align16(pool.size() * sizeof(C)) + ops.size() * sizeof(TOp);
        host.resize(need);
        std::memcpy(host.data() + b.off, pool.data(), pool.size() * sizeof(C));
        std::memcpy(host.data() + b.off + align16(pool.size() * sizeof(C)), ops.data(), ops.size() * sizeof(TOp));
    }
    // upload
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
        if (b.strided) {
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
            e = launch_tile<R>(L, psi, d, pp.geom, b.nops, ops, pool, b.nmat, nullptr, nullptr);
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

}  // namespace qf

extern "C" {

qf_status qf_program_create(int d, int n, qf_program **out) {
    if (!out) return set_error(QF_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (d < 2 || d > kMaxD || n < 1 || n > kMaxQudits) return set_error(QF_ERR_ARG, "d or n out of range");
    qf_program *p = new qf_program();
    p->d = d;
    p->n = n;
    *out = p;
    return QF_OK;
}

qf_status qf_program_free(qf_program *p) {
    if (!p) return QF_OK;
    if (p->ran && p->done_ev) cudaEventSynchronize(p->done_ev);
    if (p->up_pending && p->up_ev) cudaEventSynchronize(p->up_ev);
    if (p->h_buf) cudaFreeHost(p->h_buf);
    if (p->d_buf) cudaFree(p->d_buf);
    for (cudaEvent_t ev : p->tev) cudaEventDestroy(ev);
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
    qf_status st = check_gate(g, p->d, p->n);
    if (st != QF_OK) return st;
    if (g.slot >= 0 && g.slot + 1 > p->num_params) p->num_params = g.slot + 1;
    p->gates.push_back(std::move(g));
    p->plan_valid = false;
    return QF_OK;
}

qf_status qf_program_add_gate(qf_program *p, const int *targets, int k, const double *U) {
    if (!p || !targets || !U || k < 1 || k > 6) return set_error(QF_ERR_ARG, "bad custom gate arguments");
    HGate g;
    g.kind = G_DENSE;
    g.nq = k;
    for (int i = 0; i < k; ++i) g.q[i] = targets[i];
    long long K = ipow_ll(p->d, k);
    if (K > kMaxDenseK) return set_error(QF_ERR_UNSUPPORTED, "custom gate: d^k must be <= 64");
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

qf_status qf_program_set_fusion(qf_program *p, int enable) {
    if (!p) return set_error(QF_ERR_ARG, "program is NULL");
    p->fuse = enable != 0;
    p->plan_valid = false;
    return QF_OK;
}

qf_status qf_program_run(qf_program *p, qf_state *s, const double *params) {
    if (!p || !s) return set_error(QF_ERR_ARG, "program or state is NULL");
    if (p->d != s->d || p->n != s->n) return set_error(QF_ERR_ARG, "program and state sizes differ");
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
    return s->dt == QF_C64 ? run_program_t<float>(p, s, params) : run_program_t<double>(p, s, params);
}

qf_status qf_program_plan(qf_program *p, qf_dtype dt, int *num_passes, int *num_strided, int *max_ops) {
    if (!p) return set_error(QF_ERR_ARG, "program is NULL");
    const bool c128 = dt == QF_C128;
    if (!p->plan_valid || p->plan_c128 != c128) {
        p->plan = plan_passes(p->gates, p->d, p->n, c128, p->fuse);
        p->plan_valid = true;
        p->plan_c128 = c128;
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
