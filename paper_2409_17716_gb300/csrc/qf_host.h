// qf_host.h -- host-side internals of libqf: recorded gates, gate entries,
// pass planning and the launchers the kernels export.
#pragma once
#include <complex>
#include <string>
#include <vector>

#include "qf_internal.cuh"

namespace qf {

using cd = std::complex<double>;

// ---- kernel launchers (defined next to their kernels)
// Geometry of a gate on one target: dimension d at stride S with H blocks of
// d*S amplitudes; for controlled kinds the control's dimension and stride.
struct StridedGeom {
    int d = 2;
    long long S = 1, H = 1;
    int dc = 2;
    long long Sc = 1;
    bool c_above = false;
};
StridedGeom uniform_geom(int d, int n, const TOp &op);
// In-place conversion of a complex128 state between double2 and its
// double-float form (k_df.cu): pack = double2 -> (hi.re, hi.im, lo.re, lo.im).
cudaError_t launch_df_convert(cudaStream_t stream, int num_sms, void *psi, long long N, bool pack);

template <typename R>
cudaError_t launch_strided(const Launch &L, cplx<R> *psi, int d, int n, const TOp &op, const cplx<R> *mat, int nmat);
template <typename R>
cudaError_t launch_strided_g(const Launch &L, cplx<R> *psi, const StridedGeom &g, const TOp &op, const cplx<R> *mat,
                             int nmat);
long long strided_adj_blocks(const StridedGeom &g, int num_sms);
template <typename R>
cudaError_t launch_strided_adj(const Launch &L, cplx<R> *psi, cplx<R> *lam, const StridedGeom &g, const TOp &op,
                               const cplx<R> *mat, int nmat, const cplx<R> *gen, int ngen, double *rows);

// Mixed-radix register: dims[q] per qudit, stride S[q] = prod_{p>q} dims[p].
struct MixedShape {
    int n = 0;
    int dims[kMaxQudits] = {};
    long long S[kMaxQudits] = {};
    long long N = 1;
};
MixedShape mixed_shape(const int *dims, int n);
StridedGeom mixed_geom(const MixedShape &m, const TOp &op);
// Multi-qudit dense gate (matrix on the device, K x K, K = prod of the
// targets' dims <= kMaxDenseK) or SWAP of two equal-dimension qudits.
template <typename R>
cudaError_t launch_group(const Launch &L, cplx<R> *psi, const MixedShape &m, const TOp &op, const cplx<R> *mat_dev);
template <typename R>
cudaError_t mixed_launch(const Launch &L, cplx<R> *psi, const MixedShape &m, const TOp &o, const cplx<R> *mat, int nmat,
                         const cplx<R> *mat_dev);
template <typename R>
cudaError_t mixed_adj_launch(const Launch &L, cplx<R> *psi, cplx<R> *lam, const MixedShape &m, const TOp &o,
                             const cplx<R> *mat, int nmat, const cplx<R> *mat_dev, const cplx<R> *gen, int ngen,
                             double *rows);
long long mixed_adj_rows(const MixedShape &m, const TOp &o, int num_sms);
// Multi-controlled gate (OP_MCSHIFT / OP_MCDENSE, `mat` = the target's d x d
// entries rounded to R) on any register shape.
template <typename R>
cudaError_t launch_mc(const Launch &L, cplx<R> *psi, const MixedShape &m, const TOp &op, const cplx<R> *mat, int nmat);
MixedShape uniform_shape(int d, int n);
template <typename R>
cudaError_t launch_expect_mixed(const Launch &L, const cplx<R> *psi, const MixedShape &m, double *partials,
                                double *out_dev);
template <typename R>
cudaError_t launch_number_obs_mixed(const Launch &L, const cplx<R> *psi, cplx<R> *lam, const MixedShape &m,
                                    const double *w, double *partials, double *loss_dev);
template <typename R>
cudaError_t launch_fibre_reduce_g(const Launch &L, const cplx<R> *psi, int d, long long S, long long N, int kind,
                                  const double2 *obs_dev, double *partials, double *out_dev);
template <typename R>
cudaError_t launch_marginal_dims(const Launch &L, const cplx<R> *psi, const int *dims, int n, const int *idx, int k,
                                 double *partials, double *out_dev);
template <typename R>
cudaError_t launch_tile(const Launch &L, cplx<R> *psi, int d, const TileGeom &g, int nops, const TOp *ops_dev,
                        const cplx<R> *mat_dev, int nmat, const TOp *op_i, const cplx<R> *mat_i,
                        const TStage *stages_dev = nullptr, int nstages = 0);
template <typename R>
size_t tile_smem_bytes(const TileGeom &g, int nops, int nmat, int nstages = 0);
template <typename R>
cudaError_t launch_basis(const Launch &L, cplx<R> *psi, long long N, long long index);
template <typename R>
cudaError_t launch_expect_number(const Launch &L, const cplx<R> *psi, int d, int n, double *partials, double *out_dev);
template <typename R>
cudaError_t launch_fibre_reduce(const Launch &L, const cplx<R> *psi, int d, int n, int q, int kind, const double2 *obs_dev,
                                double *partials, double *out_dev);
int reduce_max_blocks(int num_sms);
template <typename R>
cudaError_t launch_marginal(const Launch &L, const cplx<R> *psi, int d, int n, const int *idx, int k, double *partials,
                            double *out_dev);
int marginal_max_blocks();
cudaError_t launch_sample(const Launch &L, const double *marg, int bins, double *cdf, const double *u, long long shots,
                          unsigned long long *counts);
template <typename R>
cudaError_t launch_number_obs(const Launch &L, const cplx<R> *psi, cplx<R> *lam, int d, int n, const double *w,
                              double *partials, double *loss_dev);
template <typename R>
cudaError_t adj_grid(int num_sms, int d, const TileGeom &g, int nops, int nmat, int nstages, int *grid);
template <typename R>
cudaError_t launch_tile_adj(const Launch &L, cplx<R> *psi, cplx<R> *lam, int d, const TileGeom &g, int nops,
                            const TOp *ops_dev, const cplx<R> *mat_dev, int nmat, const TStage *stages_dev,
                            int nstages, double *rows, int ncols, int grid);
cudaError_t launch_grad_gather(const Launch &L, const double *rows, const void *terms, const int *first, int nslots,
                               double *grad);
size_t gather_term_bytes();

// ---- errors
qf_status set_error(qf_status s, const std::string &msg);
qf_status cuda_error(cudaError_t e, const char *where);

// ---- recorded gates (program entries and immediate calls share this form)
enum GateKind { G_DENSE = 0, G_ROT, G_CROT, G_SUM, G_SWAP, G_X, G_Z, G_H, G_MCX, G_MCU };

struct HGate {
    int kind = G_DENSE;
    int nq = 0;
    int q[6] = {0, 0, 0, 0, 0, 0};   // targets; crot/sum: (c, t); swap: (a, b)
    int j = 0, k = 0;
    char axis = 'x';
    int slot = -1;                   // parameter slot, -1 = fixed theta
    double theta = 0.0;
    int power = 0;                   // X shift / Z power / MCX shift
    int lv[6] = {0, 0, 0, 0, 0, 0};  // G_MCU: control levels
    std::vector<cd> U;               // G_DENSE: d^nq x d^nq row-major; G_MCU: target d x d
};

// Validates a gate against (d, n); returns QF_OK or QF_ERR_ARG with message.
qf_status check_gate(const HGate &g, int d, int n);
// The same against per-qudit dimensions (levels bounded by the target's d).
qf_status check_gate_dims(const HGate &g, const int *dims, int n);

// A resolved op: kind (OpKind) on global qudits plus FP64 entries.
struct ROp {
    TOp op;                 // a/c/q[] are GLOBAL qudit indices here
    std::vector<cd> m;      // matrix entries in the layout of op.kind
};

// Entries of a gate at angle theta (theta ignored for fixed gates).
ROp resolve_gate(const HGate &g, int d, double theta);
// The same on a mixed register: target and control take their own dims.
ROp resolve_gate_dims(const HGate &g, const int *dims, double theta);
// U^+ of a resolved op in the same layout; d = the target's dimension.
ROp dagger(const ROp &r, int d);
// Generator G (dU/dtheta = -i G U) of a parametrised gate in the layout of
// its op: PAIR kinds (jj, jk, kj, kk), DIAG kinds d entries; d = target's dim.
std::vector<cd> generator_entries(const HGate &g, int d);
// Target qudit of a gate (the second qudit of crot / sum, the last of a
// multi-controlled gate).
inline int gate_target(const HGate &g) {
    if (g.kind == G_MCX || g.kind == G_MCU) return g.q[g.nq - 1];
    return (g.kind == G_CROT || g.kind == G_SUM) ? g.q[1] : g.q[0];
}
inline bool is_mc_gate(const HGate &g) { return g.kind == G_MCX || g.kind == G_MCU; }
// theta of a gate given the parameter vector.
double gate_angle(const HGate &g, const double *params);
// Generator-scaled derivative support: returns false if the gate has no angle.
bool gate_is_param(const HGate &g);

// True if the op only moves the qudit it targets (a d x d action).
inline bool is_single(const TOp &o) {
    return o.kind == OP_DENSE || o.kind == OP_PAIR || o.kind == OP_DIAG || o.kind == OP_SHIFT;
}
inline bool is_controlled(const TOp &o) { return o.kind == OP_CPAIR || o.kind == OP_CDIAG || o.kind == OP_CSHIFT; }
inline bool is_mc(const TOp &o) { return o.kind == OP_MCSHIFT || o.kind == OP_MCDENSE; }

// d x d matrix of a single-qudit resolved op.
std::vector<cd> dense_of(const ROp &r, int d);

// ---- planning
struct PassPlan {
    bool strided = false;               // one op through the strided kernel
    bool mc = false;                    // one multi-controlled gate through its own kernel
    TileGeom geom;                      // tile passes
    std::vector<std::vector<int>> groups;  // per op of the pass: gate indices merged (in order)
    std::vector<int> active;            // active qudits (sorted)
};

int default_tile_qudits(int d, bool c128);   // nt_max
int max_tile_qudits(int d, bool c128);       // largest explicit override
int min_low_qudits(int d);                   // rL_min (SEG >= 32)
long long ipow_ll(int d, int e);

// Plans passes over `gates` (indices into the gate list).  fuse = false gives
// one pass per gate.  for_adjoint: tile passes only, and parametrised gates
// are never multiplied into a group (each needs its own gradient).
std::vector<PassPlan> plan_passes(const std::vector<HGate> &gates, int d, int n, bool c128, bool fuse,
                                  bool for_adjoint = false, int nt_override = 0, int max_ops = 0, int rl_override = 0);

// Tile geometry for the given active qudits and low-qudit count.
TileGeom make_geom(int d, int n, const std::vector<int> &active, int rL);
// Register stages of K slots over a pass's localized ops (sets the ops'
// stage slots); K = stage_k(d, adjoint, complex128) of the kernel that runs them.
std::vector<TStage> build_stages(std::vector<TOp> &ops, const TileGeom &g, int d, int K);
// Local position of global qudit q in a tile geometry (-1 if not in the tile).
int local_pos(const TileGeom &g, const std::vector<int> &active, int n, int q);
// Converts a resolved op on global qudits into tile-local form.
TOp localize(const TOp &op, const TileGeom &g, const std::vector<int> &active, int n, int d);

// Shape and recorded gates of a program (for batches).
qf_status program_shape(const qf_program *p, int *d, int *n);
qf_status program_gates(const qf_program *p, std::vector<HGate> *out);

// Tile passes of a program compiled at plan time (qf_jit.cu).
struct JitProgram;
// df: complex128 forward passes in double-float arithmetic (k_df.cu); their
// prepared entries are 32 bytes, (urh, urh, -uih, uih, url, url, -uil, uil).
qf_status jit_build(const std::vector<PassPlan> &plan, std::vector<std::vector<TOp>> &ops, int d, bool c128,
                    int k_override, bool adj, int num_sms, JitProgram **out, bool df = false);
qf_status jit_launch_adj(const JitProgram *jp, size_t pi, cudaStream_t stream, void *psi, void *lam, double *rows,
                         const TileGeom &g, const void *prepared, int npool, const void *gpool);
int jit_pass_grid(const JitProgram *jp, size_t pi);
int jit_pass_ncols(const JitProgram *jp, size_t pi);
void jit_free(JitProgram *jp);
qf_status jit_source(const std::vector<PassPlan> &plan, std::vector<std::vector<TOp>> &ops, int d, bool c128,
                     int k_override, bool adj, std::string *out, bool df = false);
bool jit_pass_ready(const JitProgram *jp, size_t pi);
// Whether pass pi reduces <N_q> into per-CTA rows (jit_launch's rows, n + 1
// doubles per CTA of jit_pass_grid) when given them.
bool jit_pass_reduces(const JitProgram *jp, size_t pi);
// out[c] = sum over `rows` rows of rows[r * cols + c] (k_reduce.cu).
cudaError_t launch_sum_rows(cudaStream_t stream, const double *rows, int nrows, int cols, double *out);
bool jit_pass_global_pool(const JitProgram *jp, size_t pi);
qf_status jit_launch(const JitProgram *jp, size_t pi, cudaStream_t stream, void *psi, const TileGeom &g,
                     const void *prepared, int npool, const void *gpool, double *rows = nullptr);

// Immediate application of one resolved op on a mixed-dimension state.
qf_status run_op_mixed(qf_state *s, const ROp &r);
// Mixed-dimension programs: gate by gate forward, and the per-gate adjoint
// sweep (loss and gradient to device buffers).
qf_status mixed_program_run(qf_program *p, qf_state *s, const double *params);
qf_status mixed_program_adjoint(qf_program *p, qf_state *psi, qf_state *lam, const double *params,
                                const double *weights, double *loss_dev, double *grad_dev);
// <N_q> and the norm of a mixed state into out_dev[0..n].
qf_status mixed_expect_number(qf_state *s, double *out_dev);

}  // namespace qf

// The opaque handle of include/qf.h.
struct qf_state {
    int d = 0, n = 0;               // d = 0 when the qudits mix dimensions
    bool mixed = false;
    int dims[qf::kMaxQudits] = {};  // per-qudit dimensions (all d when uniform)
    qf_dtype dt = QF_C64;
    long long N = 0;
    void *data = nullptr;
    bool owned = false;
    cudaStream_t stream = nullptr;
    int device = 0;
    int num_sms = 0;
    double *d_partials = nullptr;    // reduction scratch
    double *d_out = nullptr;         // reduction results
    double *h_out = nullptr;         // pinned copy of results
    // uploads of large matrices (custom gates, observables)
    void *h_up = nullptr;
    void *d_up = nullptr;
    size_t up_cap = 0;
    cudaEvent_t up_ev = nullptr;
    bool up_pending = false;
    // measurement scratch (marginal partials, probabilities, CDF, counts, uniforms)
    void *d_meas = nullptr;
    size_t meas_cap = 0;
};
