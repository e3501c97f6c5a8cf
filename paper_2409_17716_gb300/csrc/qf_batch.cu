// qf_batch.cu -- batched forward and adjoint of many independent circuits.
//
// Every circuit (a recorded program, its loss weights) gets a psi and a lambda
// state in one device allocation.  Circuits are planned into tile passes
// (parametrised gates kept as ops of their own); circuits with the same gate
// structure share one plan.  For each qudit dimension d present, launch k of
// the forward runs pass k of every circuit of that d, and launch k of the
// adjoint runs each circuit's passes in reverse.  The whole sequence --
// the rotation entries of every parametrised op, |0...0> initialisation,
// forward passes, lambda = O psi with
// the per-circuit loss, reverse passes and the gradient gathers -- is captured
// once into a CUDA graph and replayed by qf_batch_run after the parameter
// upload.  Rotation entries are
// computed on the device from the uploaded parameter vector, so the graph
// stays valid when parameters change.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <string>

#include "qf_host.h"

namespace qf {

struct BPassHost {  // mirrors BPass in k_batch.cu
    long long psi_off, lam_off;
    TileGeom g;
    int ops_off, nops;
    int mat_off, nmat;
    int ncols;
    int chunks;
    long long rows_base;
    int stages_off, nstages;
};
struct BObsHost {  // mirrors BObs in k_batch.cu
    long long psi_off, lam_off;
    long long N;
    int d, n;
    int w_off;
    int items;
};
size_t bpass_bytes();
size_t bobs_bytes();
template <typename R>
cudaError_t batch_prepare(int d, bool adj, size_t smem, int *per_sm);
template <typename R>
size_t batch_smem_bytes(bool adj, int max_T, int max_nmat, int max_nops, int max_nA, int max_nstages);
struct BPass;
template <typename R>
cudaError_t launch_batch(cudaStream_t stream, int d, bool adj, int grid, size_t smem, cplx<R> *states,
                         const BPass *passes, const long long *prefix, int npasses, const TOp *ops, const cplx<R> *pool,
                         const TStage *stages, const double *params, double *rows, int chunk_tiles, int max_T,
                         int max_nmat, int max_nops, int max_nA, int max_nstages);
struct BParamHost {  // mirrors BParam in k_batch.cu
    int pool_off;
    int kind, d, j, k, axis, slot, sign;
};
size_t bparam_bytes();
template <typename R>
cudaError_t launch_batch_resolve(cudaStream_t stream, int sms, cplx<R> *pool, const void *recs, int count,
                                 const double *params);
struct BObs;
template <typename R>
cudaError_t launch_batch_init(cudaStream_t stream, int sms, cplx<R> *states, long long psi_elems, const long long *offs,
                              int count);
template <typename R>
cudaError_t launch_batch_obs(cudaStream_t stream, int sms, cplx<R> *states, const BObs *circ, const long long *prefix,
                             int ncirc, const double *weights, double *loss_rows);

constexpr int kObsChunkHost = 4096;   // = kObsChunk in k_batch.cu
constexpr int kChunkTiles = 4;        // tiles per work item

}  // namespace qf

using namespace qf;

struct qf_batch {
    qf_dtype dt = QF_C64;
    cudaStream_t user_stream = nullptr;
    cudaStream_t bstream = nullptr;
    int sms = 1;
    struct Circ {
        std::vector<HGate> gates;
        int d = 0, n = 0;
        std::vector<double> w;
        long long N = 0, psi_off = 0, lam_off = 0, grad_off = 0;
        std::vector<int> slots;     // distinct parameter slots, ascending
        int plan = -1;
    };
    std::vector<Circ> circ;
    int tune_nt[kMaxD + 1] = {0};
    int tune_ops[kMaxD + 1] = {0};
    int num_params = 0;
    bool built = false;
    std::vector<std::vector<PassPlan>> plans;
    // device
    void *d_states = nullptr;
    void *d_tab = nullptr;
    double *d_params = nullptr, *h_params = nullptr;
    double *d_rows = nullptr, *d_loss = nullptr, *d_grad_local = nullptr, *d_grad_sum = nullptr;
    long long grad_local_len = 0;
    cudaGraphExec_t g_fb = nullptr, g_f = nullptr;
    cudaEvent_t ev_in = nullptr, ev_done = nullptr, ev_params = nullptr;
    bool params_pending = false;
    int launches_fb = 0, launches_f = 0;
    long long amps = 0;
    double gate_amps = 0.0;   // sum over circuits of N x gates
};

namespace qf {

#define QF_CUDA(call)                                        \
    do {                                                     \
        cudaError_t e_ = (call);                             \
        if (e_ != cudaSuccess) return cuda_error(e_, #call); \
    } while (0)

static std::string structure_key(const qf_batch::Circ &c) {
    std::string k = std::to_string(c.d) + "/" + std::to_string(c.n) + ":";
    for (const HGate &g : c.gates) {
        k += std::to_string(g.kind) + "," + std::to_string(g.nq);
        for (int i = 0; i < g.nq; ++i) k += "," + std::to_string(g.q[i]);
        k += "," + std::to_string(g.j) + "," + std::to_string(g.k) + "," + g.axis + "," + (g.slot >= 0 ? "p" : "f") +
             "," + std::to_string(g.power) + ";";
    }
    return k;
}

// Entries reserved for a device-resolved rotation op of this kind.
static int param_entries(const TOp &o, int d) {
    switch (o.kind) {
    case OP_PAIR: return 4;
    case OP_DIAG: return d;
    case OP_CPAIR: return 4 * d;
    case OP_CDIAG: return d * d;
    default: return 0;
    }
}

static ROp dagger_op(const ROp &r, int d) {
    ROp o = r;
    auto cj = [](const cd &z) { return std::conj(z); };
    switch (r.op.kind) {
    case OP_DENSE:
        for (int a = 0; a < d; ++a)
            for (int b = 0; b < d; ++b) o.m[a * d + b] = cj(r.m[b * d + a]);
        break;
    case OP_PAIR:
        o.m[0] = cj(r.m[0]); o.m[1] = cj(r.m[2]); o.m[2] = cj(r.m[1]); o.m[3] = cj(r.m[3]);
        break;
    case OP_CPAIR:
        for (int m = 0; m < d; ++m) {
            const cd *s = r.m.data() + 4 * m;
            cd *t = o.m.data() + 4 * m;
            t[0] = cj(s[0]); t[1] = cj(s[2]); t[2] = cj(s[1]); t[3] = cj(s[3]);
        }
        break;
    case OP_DIAG:
    case OP_CDIAG:
        for (auto &z : o.m) z = cj(z);
        break;
    case OP_SHIFT:
    case OP_CSHIFT:
        o.op.s = (d - r.op.s % d) % d;
        break;
    case OP_DENSEK: {
        int K = (int)std::lround(std::sqrt((double)r.m.size()));
        for (int a = 0; a < K; ++a)
            for (int b = 0; b < K; ++b) o.m[a * K + b] = cj(r.m[b * K + a]);
        break;
    }
    default:
        break;
    }
    return o;
}

static std::vector<cd> gen_entries(const HGate &g, int d) {
    std::vector<cd> G;
    if (g.axis == 'x') G = {cd(0, 0), cd(0.5, 0), cd(0.5, 0), cd(0, 0)};
    else if (g.axis == 'y') G = {cd(0, 0), cd(0, -0.5), cd(0, 0.5), cd(0, 0)};
    else if (g.axis == 'z') {
        G.assign(d, cd(0, 0));
        G[g.j] = cd(0.5, 0);
        G[g.k] = cd(-0.5, 0);
    } else {
        G.assign(d, cd(0, 0));
        const double gam = std::sqrt(2.0 / ((double)g.j * (double)(g.j + 1)));
        for (int l = 0; l < g.j; ++l) G[l] = cd(0.5 * gam, 0);
        G[g.j] = cd(-0.5 * g.j * gam, 0);
    }
    return G;
}

struct LaunchRec {
    int d = 0;
    bool adj = false;
    int first = 0, count = 0;   // BPass range
    long long prefix_off = 0;   // into the prefix table
    int max_T = 0, max_nmat = 0, max_nops = 0, max_nA = 0, max_nstages = 0;
    size_t smem = 0;
    int grid = 0;
};

static size_t al16(size_t x) { return (x + 15) & ~(size_t)15; }

template <typename R>
static qf_status build_t(qf_batch *b) {
    using C = cplx<R>;
    const bool c128 = sizeof(R) == 8;
    const int nc = (int)b->circ.size();
    // ---- state layout: all psi, then all lambda (offsets even, 16-byte aligned)
    long long off = 0;
    for (auto &c : b->circ) {
        c.psi_off = off;
        off += (c.N + 1) & ~1LL;
    }
    const long long psi_elems = off;
    for (auto &c : b->circ) {
        c.lam_off = off;
        off += (c.N + 1) & ~1LL;
    }
    const long long total_elems = off;
    // ---- per-circuit parameter slots and local gradient offsets
    long long goff = 0;
    for (auto &c : b->circ) {
        std::vector<int> sl;
        for (const HGate &g : c.gates)
            if (gate_is_param(g)) sl.push_back(g.slot);
        std::sort(sl.begin(), sl.end());
        sl.erase(std::unique(sl.begin(), sl.end()), sl.end());
        c.slots = sl;
        c.grad_off = goff;
        goff += (long long)sl.size();
    }
    b->grad_local_len = goff;
    // ---- plans per structure
    std::map<std::string, int> cache;
    b->plans.clear();
    for (auto &c : b->circ) {
        std::string key = structure_key(c);
        auto it = cache.find(key);
        if (it != cache.end()) {
            c.plan = it->second;
            continue;
        }
        c.plan = (int)b->plans.size();
        cache[key] = c.plan;
        b->plans.push_back(plan_passes(c.gates, c.d, c.n, c128, true, true, b->tune_nt[c.d], b->tune_ops[c.d]));
    }
    // ---- tables
    std::vector<BPassHost> passes;
    std::vector<long long> prefix;
    std::vector<TOp> ops;
    std::vector<C> pool;
    std::vector<TStage> stages;
    std::vector<BParamHost> precs;   // parametrised ops whose entries the device writes
    std::vector<LaunchRec> fwd, adj;
    long long rows_total = 0;
    // gradient terms: for local index (grad_off + k): list of (rows_base, chunks, ncols, col)
    struct Term {
        long long base;
        int nrows, ncols, col, pad;
    };
    std::vector<std::vector<Term>> lterms((size_t)goff);
    std::vector<int> ds;
    for (auto &c : b->circ) ds.push_back(c.d);
    std::sort(ds.begin(), ds.end());
    ds.erase(std::unique(ds.begin(), ds.end()), ds.end());

    auto add_pass = [&](const qf_batch::Circ &c, const PassPlan &pp, bool is_adj, LaunchRec &L) {
        BPassHost bp;
        std::memset(&bp, 0, sizeof(bp));
        bp.psi_off = c.psi_off;
        bp.lam_off = c.lam_off;
        bp.g = pp.geom;
        bp.ops_off = (int)ops.size();
        bp.mat_off = (int)pool.size();
        int ncols = 0;
        const int ng = (int)pp.groups.size();
        for (int oi = 0; oi < ng; ++oi) {
            const auto &grp = pp.groups[is_adj ? ng - 1 - oi : oi];
            const HGate &g0 = c.gates[grp[0]];
            const bool param = grp.size() == 1 && gate_is_param(g0);
            // fixed entries (or the op layout of a parametrised rotation)
            std::vector<cd> m;
            TOp o;
            if (grp.size() == 1) {
                ROp r = resolve_gate(g0, c.d, param ? 0.0 : g0.theta);
                if (is_adj && !param) r = dagger_op(r, c.d);
                o = localize(r.op, pp.geom, pp.active, c.n, c.d);
                m = r.m;
            } else {
                // product of fixed single-qudit gates on one qudit
                std::vector<cd> M;
                ROp first = resolve_gate(g0, c.d, g0.theta);
                M = dense_of(first, c.d);
                for (size_t i = 1; i < grp.size(); ++i) {
                    ROp ri = resolve_gate(c.gates[grp[i]], c.d, c.gates[grp[i]].theta);
                    std::vector<cd> G = dense_of(ri, c.d), P((size_t)c.d * c.d, cd(0, 0));
                    for (int rr = 0; rr < c.d; ++rr)
                        for (int cc = 0; cc < c.d; ++cc) {
                            cd acc(0, 0);
                            for (int t = 0; t < c.d; ++t) acc += G[rr * c.d + t] * M[t * c.d + cc];
                            P[rr * c.d + cc] = acc;
                        }
                    M.swap(P);
                }
                ROp r = first;
                r.op.kind = OP_DENSE;
                r.m = M;
                if (is_adj) r = dagger_op(r, c.d);
                o = localize(r.op, pp.geom, pp.active, c.n, c.d);
                m = r.m;
            }
            o.mat = (int)pool.size() - bp.mat_off;
            o.gcol = -1;
            o.gmat = 0;
            o.pslot = -1;
            o.paxis = 0;
            o.psign = 1;
            if (param) {
                o.pslot = g0.slot;
                o.paxis = g0.axis;
                o.psign = is_adj ? -1 : 1;
                const int ne = param_entries(o, c.d);
                precs.push_back({(int)pool.size(), o.kind, c.d, o.j, o.k, o.paxis, o.pslot, o.psign});
                for (int i = 0; i < ne; ++i) pool.push_back(mk<R>(0, 0));   // written on the device
            } else {
                for (const cd &z : m) pool.push_back(mk<R>((R)z.real(), (R)z.imag()));
            }
            if (is_adj && param) {
                o.gcol = ncols++;
                o.gmat = (int)pool.size() - bp.mat_off;
                for (const cd &z : gen_entries(g0, c.d)) pool.push_back(mk<R>((R)z.real(), (R)z.imag()));
            }
            ops.push_back(o);
        }
        bp.nops = (int)ops.size() - bp.ops_off;
        bp.nmat = (int)pool.size() - bp.mat_off;
        bp.ncols = ncols;
        {
            const int K = stage_k(c.d, is_adj, c128);
            bp.stages_off = (int)stages.size();
            bp.nstages = 0;
            if (K > 0) {
                std::vector<TOp> pops(ops.begin() + bp.ops_off, ops.end());
                std::vector<TStage> ps = build_stages(pops, pp.geom, c.d, K);
                std::copy(pops.begin(), pops.end(), ops.begin() + bp.ops_off);
                stages.insert(stages.end(), ps.begin(), ps.end());
                bp.nstages = (int)ps.size();
            }
        }
        bp.chunks = (int)((pp.geom.ntiles + kChunkTiles - 1) / kChunkTiles);
        bp.rows_base = rows_total;
        if (is_adj) {
            rows_total += (long long)bp.chunks * ncols;
            // gradient terms of this pass
            int col = 0;
            for (int oi = 0; oi < ng; ++oi) {
                const auto &grp = pp.groups[ng - 1 - oi];
                const HGate &g0 = c.gates[grp[0]];
                if (grp.size() == 1 && gate_is_param(g0)) {
                    int k = (int)(std::lower_bound(c.slots.begin(), c.slots.end(), g0.slot) - c.slots.begin());
                    lterms[c.grad_off + k].push_back({bp.rows_base, bp.chunks, ncols, col, 0});
                    ++col;
                }
            }
        }
        L.max_T = std::max(L.max_T, pp.geom.T);
        L.max_nmat = std::max(L.max_nmat, bp.nmat);
        L.max_nops = std::max(L.max_nops, bp.nops);
        L.max_nA = std::max(L.max_nA, pp.geom.T / pp.geom.SEG);
        L.max_nstages = std::max(L.max_nstages, bp.nstages);
        prefix.push_back(prefix.back() + bp.chunks);
        passes.push_back(bp);
    };

    for (int d : ds) {
        int maxp = 0;
        for (auto &c : b->circ)
            if (c.d == d) maxp = std::max(maxp, (int)b->plans[c.plan].size());
        for (int dir = 0; dir < 2; ++dir) {
            for (int k = 0; k < maxp; ++k) {
                LaunchRec L;
                L.d = d;
                L.adj = dir == 1;
                L.first = (int)passes.size();
                L.prefix_off = (long long)prefix.size();
                prefix.push_back(0);
                for (auto &c : b->circ) {
                    if (c.d != d) continue;
                    const auto &plan = b->plans[c.plan];
                    const int np = (int)plan.size();
                    if (k >= np) continue;
                    add_pass(c, plan[L.adj ? np - 1 - k : k], L.adj, L);
                }
                L.count = (int)passes.size() - L.first;
                if (L.count == 0) {
                    prefix.pop_back();
                    continue;
                }
                (L.adj ? adj : fwd).push_back(L);
            }
        }
    }
    // ---- observable / loss items
    std::vector<BObsHost> obs(nc);
    std::vector<long long> oprefix(nc + 1, 0);
    std::vector<double> wts;
    for (int i = 0; i < nc; ++i) {
        const auto &c = b->circ[i];
        BObsHost &o = obs[i];
        std::memset(&o, 0, sizeof(o));
        o.psi_off = c.psi_off;
        o.lam_off = c.lam_off;
        o.N = c.N;
        o.d = c.d;
        o.n = c.n;
        o.w_off = (int)wts.size();
        for (double x : c.w) wts.push_back(x);
        o.items = (int)((c.N + kObsChunkHost - 1) / kObsChunkHost);
        oprefix[i + 1] = oprefix[i] + o.items;
    }
    const long long loss_rows_base = rows_total;
    rows_total += oprefix[nc];
    // ---- gather tables: loss (nc), local gradient (goff), summed gradient (num_params)
    std::vector<Term> terms;
    std::vector<int> f_loss(nc + 1, 0), f_local(goff + 1, 0), f_sum(b->num_params + 1, 0);
    for (int i = 0; i < nc; ++i) {
        terms.push_back({loss_rows_base + oprefix[i], obs[i].items, 1, 0, 0});
        f_loss[i + 1] = (int)terms.size();
    }
    const int local_first = (int)terms.size();
    for (long long k = 0; k < goff; ++k) {
        for (const Term &t : lterms[k]) terms.push_back(t);
        f_local[k + 1] = (int)terms.size() - local_first;
    }
    std::vector<std::vector<long long>> uses(b->num_params);
    for (const auto &c : b->circ)
        for (size_t k = 0; k < c.slots.size(); ++k) uses[c.slots[k]].push_back(c.grad_off + (long long)k);
    const int sum_first = (int)terms.size();
    for (int s = 0; s < b->num_params; ++s) {
        for (long long li : uses[s]) terms.push_back({li, 1, 1, 0, 0});
        f_sum[s + 1] = (int)terms.size() - sum_first;
    }
    std::vector<long long> one_offs(nc);
    for (int i = 0; i < nc; ++i) one_offs[i] = b->circ[i].psi_off;

    // ---- one device table buffer
    size_t o_pass = 0, sz = al16(passes.size() * bpass_bytes());
    size_t o_pref = sz;  sz = al16(sz + prefix.size() * sizeof(long long));
    size_t o_ops = sz;   sz = al16(sz + ops.size() * sizeof(TOp));
    size_t o_pool = sz;  sz = al16(sz + pool.size() * sizeof(C));
    size_t o_stg = sz;   sz = al16(sz + std::max<size_t>(stages.size(), 1) * sizeof(TStage));
    size_t o_prec = sz;  sz = al16(sz + std::max<size_t>(precs.size(), 1) * sizeof(BParamHost));
    size_t o_obs = sz;   sz = al16(sz + obs.size() * bobs_bytes());
    size_t o_opref = sz; sz = al16(sz + oprefix.size() * sizeof(long long));
    size_t o_w = sz;     sz = al16(sz + wts.size() * sizeof(double));
    size_t o_terms = sz; sz = al16(sz + terms.size() * sizeof(Term));
    size_t o_fl = sz;    sz = al16(sz + f_loss.size() * sizeof(int));
    size_t o_fg = sz;    sz = al16(sz + f_local.size() * sizeof(int));
    size_t o_fs = sz;    sz = al16(sz + f_sum.size() * sizeof(int));
    size_t o_one = sz;   sz = al16(sz + one_offs.size() * sizeof(long long));
    if (bpass_bytes() != sizeof(BPassHost) || bobs_bytes() != sizeof(BObsHost) || gather_term_bytes() != sizeof(Term) ||
        bparam_bytes() != sizeof(BParamHost))
        return set_error(QF_ERR_CUDA, "batch table layout mismatch");
    std::vector<unsigned char> host(sz, 0);
    auto put = [&](size_t at, const void *src, size_t n) {
        if (n) std::memcpy(host.data() + at, src, n);
    };
    put(o_pass, passes.data(), passes.size() * sizeof(BPassHost));
    put(o_pref, prefix.data(), prefix.size() * sizeof(long long));
    put(o_ops, ops.data(), ops.size() * sizeof(TOp));
    put(o_pool, pool.data(), pool.size() * sizeof(C));
    put(o_stg, stages.data(), stages.size() * sizeof(TStage));
    put(o_prec, precs.data(), precs.size() * sizeof(BParamHost));
    put(o_obs, obs.data(), obs.size() * sizeof(BObsHost));
    put(o_opref, oprefix.data(), oprefix.size() * sizeof(long long));
    put(o_w, wts.data(), wts.size() * sizeof(double));
    put(o_terms, terms.data(), terms.size() * sizeof(Term));
    put(o_fl, f_loss.data(), f_loss.size() * sizeof(int));
    put(o_fg, f_local.data(), f_local.size() * sizeof(int));
    put(o_fs, f_sum.data(), f_sum.size() * sizeof(int));
    put(o_one, one_offs.data(), one_offs.size() * sizeof(long long));

    const size_t state_bytes = (size_t)total_elems * sizeof(C);
    if (cudaMalloc(&b->d_states, state_bytes) != cudaSuccess || cudaMalloc(&b->d_tab, sz) != cudaSuccess ||
        cudaMalloc(&b->d_rows, (size_t)std::max<long long>(rows_total, 1) * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&b->d_loss, (size_t)std::max(nc, 1) * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&b->d_grad_local, (size_t)std::max<long long>(goff, 1) * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&b->d_grad_sum, (size_t)std::max(b->num_params, 1) * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&b->d_params, (size_t)std::max(b->num_params, 1) * sizeof(double)) != cudaSuccess ||
        cudaMallocHost(&b->h_params, (size_t)std::max(b->num_params, 1) * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        return set_error(QF_ERR_OOM, "batch allocation of " + std::to_string(state_bytes) + " state bytes failed");
    }
    std::memset(b->h_params, 0, (size_t)std::max(b->num_params, 1) * sizeof(double));
    QF_CUDA(cudaMemcpy(b->d_tab, host.data(), sz, cudaMemcpyHostToDevice));

    // ---- launch configuration (outside capture).  The shared-memory limit is
    // an attribute of the kernel instantiation, so each (d, direction) gets
    // one value: the largest any of its launches needs.
    std::map<std::pair<int, int>, size_t> group_smem;
    for (auto *list : {&fwd, &adj})
        for (LaunchRec &L : *list) {
            L.smem = batch_smem_bytes<R>(L.adj, L.max_T, L.max_nmat, L.max_nops, L.max_nA, L.max_nstages);
            size_t &gs = group_smem[{L.d, L.adj ? 1 : 0}];
            gs = std::max(gs, L.smem);
        }
    std::map<std::pair<int, int>, int> group_per_sm;
    for (auto &kv : group_smem) {
        int per_sm = 0;
        cudaError_t e = batch_prepare<R>(kv.first.first, kv.first.second == 1, kv.second, &per_sm);
        if (e != cudaSuccess) return cuda_error(e, "batch kernel configuration");
        if (per_sm < 1) return set_error(QF_ERR_UNSUPPORTED, "batch tile does not fit shared memory");
        group_per_sm[kv.first] = per_sm;
    }
    for (auto *list : {&fwd, &adj})
        for (LaunchRec &L : *list) {
            const int per_sm = group_per_sm[{L.d, L.adj ? 1 : 0}];
            long long items = prefix[L.prefix_off + L.count];
            long long gr = (long long)per_sm * b->sms;
            L.grid = (int)std::min<long long>(gr, items);
        }

    // ---- capture
    unsigned char *tab = reinterpret_cast<unsigned char *>(b->d_tab);
    C *states = reinterpret_cast<C *>(b->d_states);
    auto record = [&](bool backward, cudaGraphExec_t *out, int *nlaunch) -> qf_status {
        int nl = 0;
        QF_CUDA(cudaStreamBeginCapture(b->bstream, cudaStreamCaptureModeThreadLocal));
        cudaError_t e = cudaSuccess;
        {
            e = launch_batch_resolve<R>(b->bstream, b->sms, reinterpret_cast<C *>(tab + o_pool), tab + o_prec,
                                        (int)precs.size(), b->d_params);
            nl += precs.empty() ? 0 : 1;
            if (e == cudaSuccess)
                e = launch_batch_init<R>(b->bstream, b->sms, states, psi_elems,
                                         reinterpret_cast<const long long *>(tab + o_one), nc);
            nl += 2;
        }
        for (const LaunchRec &L : fwd) {
            if (e != cudaSuccess) break;
            e = launch_batch<R>(b->bstream, L.d, false, L.grid, L.smem, states,
                                reinterpret_cast<const BPass *>(tab + o_pass + (size_t)L.first * sizeof(BPassHost)),
                                reinterpret_cast<const long long *>(tab + o_pref) + L.prefix_off, L.count,
                                reinterpret_cast<const TOp *>(tab + o_ops), reinterpret_cast<const C *>(tab + o_pool),
                                reinterpret_cast<const TStage *>(tab + o_stg), b->d_params, b->d_rows, kChunkTiles,
                                L.max_T, L.max_nmat, L.max_nops, L.max_nA, L.max_nstages);
            ++nl;
        }
        if (e == cudaSuccess) {
            e = launch_batch_obs<R>(b->bstream, b->sms, states, reinterpret_cast<const BObs *>(tab + o_obs),
                                    reinterpret_cast<const long long *>(tab + o_opref), nc,
                                    reinterpret_cast<const double *>(tab + o_w), b->d_rows + loss_rows_base);
            ++nl;
        }
        if (e == cudaSuccess) {
            e = launch_grad_gather(Launch{b->bstream, b->sms}, b->d_rows, tab + o_terms,
                                   reinterpret_cast<const int *>(tab + o_fl), nc, b->d_loss);
            ++nl;
        }
        if (backward) {
            for (const LaunchRec &L : adj) {
                if (e != cudaSuccess) break;
                e = launch_batch<R>(b->bstream, L.d, true, L.grid, L.smem, states,
                                    reinterpret_cast<const BPass *>(tab + o_pass + (size_t)L.first * sizeof(BPassHost)),
                                    reinterpret_cast<const long long *>(tab + o_pref) + L.prefix_off, L.count,
                                    reinterpret_cast<const TOp *>(tab + o_ops),
                                    reinterpret_cast<const C *>(tab + o_pool),
                                    reinterpret_cast<const TStage *>(tab + o_stg), b->d_params, b->d_rows, kChunkTiles,
                                    L.max_T, L.max_nmat, L.max_nops, L.max_nA, L.max_nstages);
                ++nl;
            }
            if (e == cudaSuccess && goff > 0) {
                e = launch_grad_gather(Launch{b->bstream, b->sms}, b->d_rows, tab + o_terms + local_first * sizeof(Term),
                                       reinterpret_cast<const int *>(tab + o_fg), (int)goff, b->d_grad_local);
                ++nl;
            }
            if (e == cudaSuccess && b->num_params > 0) {
                e = launch_grad_gather(Launch{b->bstream, b->sms}, b->d_grad_local,
                                       tab + o_terms + sum_first * sizeof(Term), reinterpret_cast<const int *>(tab + o_fs),
                                       b->num_params, b->d_grad_sum);
                ++nl;
            }
        }
        cudaGraph_t graph = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(b->bstream, &graph);
        if (e != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return cuda_error(e, "batch capture");
        }
        if (e2 != cudaSuccess) return cuda_error(e2, "cudaStreamEndCapture");
        e = cudaGraphInstantiate(out, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return cuda_error(e, "cudaGraphInstantiate");
        *nlaunch = nl;
        return QF_OK;
    };
    qf_status st = record(true, &b->g_fb, &b->launches_fb);
    if (st != QF_OK) return st;
    st = record(false, &b->g_f, &b->launches_f);
    if (st != QF_OK) return st;
    b->built = true;
    return QF_OK;
}

}  // namespace qf

extern "C" {

qf_status qf_batch_create(qf_dtype dt, void *cuda_stream, qf_batch **out) {
    if (!out) return set_error(QF_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (dt != QF_C64 && dt != QF_C128) return set_error(QF_ERR_ARG, "unknown dtype");
    qf_batch *b = new qf_batch();
    b->dt = dt;
    b->user_stream = (cudaStream_t)cuda_stream;
    *out = b;
    return QF_OK;
}

qf_status qf_batch_free(qf_batch *b) {
    if (!b) return QF_OK;
    if (b->bstream) cudaStreamSynchronize(b->bstream);
    if (b->g_fb) cudaGraphExecDestroy(b->g_fb);
    if (b->g_f) cudaGraphExecDestroy(b->g_f);
    for (void *p : {(void *)b->d_states, b->d_tab, (void *)b->d_params, (void *)b->d_rows, (void *)b->d_loss,
                    (void *)b->d_grad_local, (void *)b->d_grad_sum})
        if (p) cudaFree(p);
    if (b->h_params) cudaFreeHost(b->h_params);
    if (b->ev_in) cudaEventDestroy(b->ev_in);
    if (b->ev_done) cudaEventDestroy(b->ev_done);
    if (b->ev_params) cudaEventDestroy(b->ev_params);
    if (b->bstream) cudaStreamDestroy(b->bstream);
    delete b;
    return QF_OK;
}

qf_status qf_batch_add(qf_batch *b, const qf_program *p, const double *weights, int *index) {
    if (!b || !p || !weights) return set_error(QF_ERR_ARG, "batch, program or weights is NULL");
    if (b->built) return set_error(QF_ERR_ARG, "batch already built");
    qf_batch::Circ c;
    int d = 0, n = 0;
    qf_status st = program_shape(p, &d, &n);
    if (st != QF_OK) return st;
    if (d == 0) return set_error(QF_ERR_UNSUPPORTED, "mixed-dimension programs cannot be batched");
    c.d = d;
    c.n = n;
    c.N = ipow_ll(d, n);
    if (c.N > (1ll << 31)) return set_error(QF_ERR_UNSUPPORTED, "batched circuits must have d^n < 2^31");
    st = program_gates(p, &c.gates);
    if (st != QF_OK) return st;
    for (const HGate &g : c.gates)
        if (is_mc_gate(g)) return set_error(QF_ERR_UNSUPPORTED, "multi-controlled gates cannot be batched");
    c.w.assign(weights, weights + n);
    if (index) *index = (int)b->circ.size();
    b->amps += c.N;
    b->gate_amps += (double)c.N * (double)c.gates.size();
    b->circ.push_back(std::move(c));
    return QF_OK;
}

qf_status qf_batch_tune(qf_batch *b, int d, int tile_qudits, int max_ops) {
    if (!b) return set_error(QF_ERR_ARG, "batch is NULL");
    if (d < 2 || d > kMaxD) return set_error(QF_ERR_ARG, "d out of range");
    if (b->built) return set_error(QF_ERR_ARG, "batch already built");
    b->tune_nt[d] = tile_qudits > 0 ? tile_qudits : 0;
    b->tune_ops[d] = max_ops > 0 ? max_ops : 0;
    return QF_OK;
}

qf_status qf_batch_build(qf_batch *b, int num_params) {
    if (!b) return set_error(QF_ERR_ARG, "batch is NULL");
    if (b->built) return set_error(QF_ERR_ARG, "batch already built");
    if (b->circ.empty()) return set_error(QF_ERR_ARG, "batch has no circuits");
    for (const auto &c : b->circ)
        for (const HGate &g : c.gates)
            if (g.slot >= num_params) return set_error(QF_ERR_ARG, "a gate uses a parameter slot >= num_params");
    b->num_params = num_params;
    b->sms = device_sms();
    if (cudaStreamCreateWithFlags(&b->bstream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev_done, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev_params, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        return set_error(QF_ERR_CUDA, "stream/event creation failed");
    }
    return b->dt == QF_C64 ? build_t<float>(b) : build_t<double>(b);
}

qf_status qf_batch_run(qf_batch *b, const double *params, int backward) {
    if (!b || !b->built) return set_error(QF_ERR_ARG, "batch is NULL or not built");
    if (b->num_params > 0 && !params) return set_error(QF_ERR_ARG, "batch needs parameters");
    if (b->params_pending) {
        QF_CUDA(cudaEventSynchronize(b->ev_params));
        b->params_pending = false;
    }
    if (b->num_params > 0) std::memcpy(b->h_params, params, (size_t)b->num_params * sizeof(double));
    QF_CUDA(cudaEventRecord(b->ev_in, b->user_stream));
    QF_CUDA(cudaStreamWaitEvent(b->bstream, b->ev_in, 0));
    // the parameter upload precedes the graph on the batch stream; the pinned
    // copy may be overwritten once ev_params has passed
    QF_CUDA(cudaMemcpyAsync(b->d_params, b->h_params, (size_t)std::max(b->num_params, 1) * sizeof(double),
                            cudaMemcpyHostToDevice, b->bstream));
    QF_CUDA(cudaEventRecord(b->ev_params, b->bstream));
    QF_CUDA(cudaGraphLaunch(backward ? b->g_fb : b->g_f, b->bstream));
    QF_CUDA(cudaEventRecord(b->ev_done, b->bstream));
    QF_CUDA(cudaStreamWaitEvent(b->user_stream, b->ev_done, 0));
    b->params_pending = true;
    return QF_OK;
}

qf_status qf_batch_outputs(qf_batch *b, double **loss_dev, double **grad_local_dev, double **grad_sum_dev) {
    if (!b || !b->built) return set_error(QF_ERR_ARG, "batch is NULL or not built");
    if (loss_dev) *loss_dev = b->d_loss;
    if (grad_local_dev) *grad_local_dev = b->d_grad_local;
    if (grad_sum_dev) *grad_sum_dev = b->d_grad_sum;
    return QF_OK;
}

qf_status qf_batch_read(qf_batch *b, double *loss_host, double *grad_local_host, double *grad_sum_host) {
    if (!b || !b->built) return set_error(QF_ERR_ARG, "batch is NULL or not built");
    QF_CUDA(cudaStreamSynchronize(b->bstream));
    if (loss_host) QF_CUDA(cudaMemcpy(loss_host, b->d_loss, b->circ.size() * sizeof(double), cudaMemcpyDeviceToHost));
    if (grad_local_host && b->grad_local_len > 0)
        QF_CUDA(cudaMemcpy(grad_local_host, b->d_grad_local, (size_t)b->grad_local_len * sizeof(double),
                           cudaMemcpyDeviceToHost));
    if (grad_sum_host && b->num_params > 0)
        QF_CUDA(cudaMemcpy(grad_sum_host, b->d_grad_sum, (size_t)b->num_params * sizeof(double),
                           cudaMemcpyDeviceToHost));
    return QF_OK;
}

qf_status qf_batch_circuit_params(const qf_batch *b, int index, int *slots, int max, int *count, long long *grad_offset) {
    if (!b || !b->built) return set_error(QF_ERR_ARG, "batch is NULL or not built");
    if (index < 0 || index >= (int)b->circ.size()) return set_error(QF_ERR_ARG, "circuit index out of range");
    const auto &c = b->circ[index];
    if (count) *count = (int)c.slots.size();
    if (grad_offset) *grad_offset = c.grad_off;
    if (slots)
        for (int i = 0; i < (int)c.slots.size() && i < max; ++i) slots[i] = c.slots[i];
    return QF_OK;
}

qf_status qf_batch_info(const qf_batch *b, int *circuits, long long *amplitudes, double *gate_amplitudes,
                        int *launches_forward, int *launches_backward, long long *grad_local_len, int *num_params) {
    if (!b) return set_error(QF_ERR_ARG, "batch is NULL");
    if (num_params) *num_params = b->num_params;
    if (grad_local_len) *grad_local_len = b->grad_local_len;
    if (circuits) *circuits = (int)b->circ.size();
    if (amplitudes) *amplitudes = b->amps;
    if (gate_amplitudes) *gate_amplitudes = b->gate_amps;
    if (launches_forward) *launches_forward = b->launches_f;
    if (launches_backward) *launches_backward = b->launches_fb;
    return QF_OK;
}

}  // extern "C"
