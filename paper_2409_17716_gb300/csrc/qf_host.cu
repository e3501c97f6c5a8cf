// qf_host.cu -- the C ABI of include/qf.h: states, immediate gates and
// measurements.  Every call validates on the host, then launches on the
// state's stream.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>

#include <sys/mman.h>

#include <map>
#include <mutex>

#include "qf_host.h"

namespace qf {

static thread_local std::string g_err = "no error";

qf_status set_error(qf_status s, const std::string &msg) {
    g_err = msg;
    return s;
}

qf_status cuda_error(cudaError_t e, const char *where) {
    g_err = std::string(where) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return QF_ERR_CUDA;
}

#define QF_CUDA(call)                                    \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return cuda_error(e_, #call); \
    } while (0)

static Launch launch_of(const qf_state *s) {
    Launch L;
    L.stream = s->stream;
    L.num_sms = s->num_sms;
    return L;
}

static qf_status check_state(const qf_state *s) {
    if (!s) return set_error(QF_ERR_ARG, "state handle is NULL");
    return QF_OK;
}

// Ensures the upload staging of a state holds `bytes`; waits for the previous
// upload to have left the pinned buffer.
static qf_status up_reserve(qf_state *s, size_t bytes) {
    if (s->up_pending) {
        QF_CUDA(cudaEventSynchronize(s->up_ev));
        s->up_pending = false;
    }
    if (bytes <= s->up_cap) return QF_OK;
    // the device buffer may still be read by queued kernels
    QF_CUDA(cudaStreamSynchronize(s->stream));
    if (s->h_up) cudaFreeHost(s->h_up);
    if (s->d_up) cudaFree(s->d_up);
    s->h_up = s->d_up = nullptr;
    s->up_cap = 0;
    size_t cap = bytes < 65536 ? 65536 : bytes;
    if (cudaMallocHost(&s->h_up, cap) != cudaSuccess) return set_error(QF_ERR_OOM, "pinned staging allocation failed");
    if (cudaMalloc(&s->d_up, cap) != cudaSuccess) return set_error(QF_ERR_OOM, "device staging allocation failed");
    s->up_cap = cap;
    return QF_OK;
}

static qf_status up_send(qf_state *s, size_t bytes) {
    QF_CUDA(cudaMemcpyAsync(s->d_up, s->h_up, bytes, cudaMemcpyHostToDevice, s->stream));
    QF_CUDA(cudaEventRecord(s->up_ev, s->stream));
    s->up_pending = true;
    return QF_OK;
}

// Runs one resolved op on the state (immediate mode).
template <typename R>
static qf_status run_op_t(qf_state *s, const ROp &r) {
    const int d = s->d, n = s->n;
    const Launch L = launch_of(s);
    cplx<R> *psi = reinterpret_cast<cplx<R> *>(s->data);
    std::vector<cplx<R>> m(r.m.size());
    for (size_t i = 0; i < r.m.size(); ++i) m[i] = mk<R>((R)r.m[i].real(), (R)r.m[i].imag());
    const TOp &o = r.op;
    if ((o.kind == OP_SHIFT && o.s == 0) || ((o.kind == OP_DIAG) && o.mask == 0)) return QF_OK;  // identity
    if (is_mc(o)) {
        if (o.kind == OP_MCSHIFT && o.s == 0) return QF_OK;
        cudaError_t e = launch_mc<R>(L, psi, uniform_shape(d, n), o, m.data(), (int)m.size());
        if (e != cudaSuccess) return cuda_error(e, "multi-controlled gate kernel");
        return QF_OK;
    }
    const bool single_target = is_single(o) || is_controlled(o);
    const long long S = ipow_ll(d, n - 1 - o.a);
    // the strided kernel at every stride: below one warp its fibres
    // interleave and L1 merges their sectors (measured on GB300 for strides
    // 1-27: 0.66-1.05 of HBM against 0.53-0.77 through a one-op tile pass)
    if (single_target && S < (1ll << 31) && (int)m.size() <= kInlineMat) {
        cudaError_t e = launch_strided<R>(L, psi, d, n, o, m.data(), (int)m.size());
        if (e != cudaSuccess) return cuda_error(e, "strided gate kernel");
        return QF_OK;
    }
    // tile pass holding this op alone
    std::vector<bool> inset(n, false);
    inset[o.a] = true;
    if (is_controlled(o) || o.kind == OP_SWAP) inset[o.c] = true;
    if (o.kind == OP_DENSEK)
        for (int i = 0; i < o.nq; ++i) inset[o.q[i]] = true;
    const int nt_max = default_tile_qudits(d, sizeof(R) == 8);
    int rL = -1;
    for (int cand = std::min(nt_max, n); cand >= 0 && rL < 0; --cand) {
        int kA = 0;
        for (int q = 0; q < n - cand; ++q) kA += inset[q];
        if (kA + cand <= std::max(nt_max, kA) && kA <= kMaxActive) rL = cand;
    }
    if (rL < 0) return set_error(QF_ERR_UNSUPPORTED, "gate qudits do not fit a tile");
    std::vector<int> active;
    for (int q = 0; q < n - rL; ++q)
        if (inset[q]) active.push_back(q);
    TileGeom g = make_geom(d, n, active, rL);
    TOp lo = localize(o, g, active, n, d);
    lo.mat = 0;
    cudaError_t e;
    if ((int)m.size() <= kInlineMat) {
        e = launch_tile<R>(L, psi, d, g, 1, nullptr, nullptr, (int)m.size(), &lo, m.data());
    } else {
        size_t mb = m.size() * sizeof(cplx<R>);
        size_t bytes = mb + sizeof(TOp);
        qf_status st = up_reserve(s, bytes);
        if (st != QF_OK) return st;
        std::memcpy(s->h_up, m.data(), mb);
        std::memcpy((char *)s->h_up + mb, &lo, sizeof(TOp));
        st = up_send(s, bytes);
        if (st != QF_OK) return st;
        e = launch_tile<R>(L, psi, d, g, 1, reinterpret_cast<const TOp *>((char *)s->d_up + mb),
                           reinterpret_cast<const cplx<R> *>(s->d_up), (int)m.size(), nullptr, nullptr);
    }
    if (e != cudaSuccess) return cuda_error(e, "tile gate kernel");
    return QF_OK;
}

// Mixed-dimension state: strided kinds carry their entries inline; a
// multi-qudit dense gate's matrix goes through the state's upload staging.
template <typename R>
static qf_status run_op_mixed_t(qf_state *s, const ROp &r) {
    const Launch L = launch_of(s);
    cplx<R> *psi = reinterpret_cast<cplx<R> *>(s->data);
    std::vector<cplx<R>> m(r.m.size());
    for (size_t i = 0; i < r.m.size(); ++i) m[i] = mk<R>((R)r.m[i].real(), (R)r.m[i].imag());
    const MixedShape shape = mixed_shape(s->dims, s->n);
    const TOp &o = r.op;
    const cplx<R> *mat_dev = nullptr;
    if (!(is_single(o) || is_controlled(o)) && !m.empty()) {
        const size_t bytes = m.size() * sizeof(cplx<R>);
        qf_status st = up_reserve(s, bytes);
        if (st != QF_OK) return st;
        std::memcpy(s->h_up, m.data(), bytes);
        st = up_send(s, bytes);
        if (st != QF_OK) return st;
        mat_dev = reinterpret_cast<const cplx<R> *>(s->d_up);
    }
    if ((is_single(o) || is_controlled(o)) && (int)m.size() > kInlineMat)
        return set_error(QF_ERR_UNSUPPORTED, "gate table too large for a mixed register");
    cudaError_t e = mixed_launch<R>(L, psi, shape, o, m.data(), (int)m.size(), mat_dev);
    if (e != cudaSuccess) return cuda_error(e, "mixed-register gate kernel");
    return QF_OK;
}

qf_status run_op_mixed(qf_state *s, const ROp &r) {
    return s->dt == QF_C64 ? run_op_mixed_t<float>(s, r) : run_op_mixed_t<double>(s, r);
}

qf_status mixed_expect_number(qf_state *s, double *out_dev) {
    const Launch L = launch_of(s);
    const MixedShape shape = mixed_shape(s->dims, s->n);
    cudaError_t e = s->dt == QF_C64
                        ? launch_expect_mixed<float>(L, (const float2 *)s->data, shape, s->d_partials, out_dev)
                        : launch_expect_mixed<double>(L, (const double2 *)s->data, shape, s->d_partials, out_dev);
    if (e != cudaSuccess) return cuda_error(e, "mixed-register reduction kernels");
    return QF_OK;
}

static qf_status apply_gate(qf_state *s, const HGate &g) {
    qf_status st = check_state(s);
    if (st != QF_OK) return st;
    if (s->mixed) {
        st = check_gate_dims(g, s->dims, s->n);
        if (st != QF_OK) return st;
        return run_op_mixed(s, resolve_gate_dims(g, s->dims, g.theta));
    }
    st = check_gate(g, s->d, s->n);
    if (st != QF_OK) return st;
    ROp r = resolve_gate(g, s->d, g.theta);
    return s->dt == QF_C64 ? run_op_t<float>(s, r) : run_op_t<double>(s, r);
}

int device_sms() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

}  // namespace qf

using namespace qf;

extern "C" {

const char *qf_last_error(void) { return g_err.c_str(); }

int qf_expect_size(int d, int n, const qf_obs *obs) {
    if (!obs) return -1;
    switch (obs->kind) {
    case QF_OBS_NUMBER_ALL: return n + 1;
    case QF_OBS_NORM: return 1;
    case QF_OBS_HERMITIAN: return 2;
    case QF_OBS_MARGINAL: return d;
    default: return -1;
    }
}

// dims == nullptr: every qudit has dimension d.
static qf_status make_state(int d, const int *dims, int n, qf_dtype dt, void *ptr, void *stream, qf_state **out) {
    if (!out) return set_error(QF_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (n < 1 || n > kMaxQudits) return set_error(QF_ERR_ARG, "n must be in [1, 62]");
    if (dims) {
        d = dims[0];
        for (int q = 0; q < n; ++q) {
            if (dims[q] < 2 || dims[q] > kMaxD) return set_error(QF_ERR_ARG, "every dimension must be in [2, 16]");
            if (dims[q] != d) d = 0;
        }
    } else if (d < 2 || d > kMaxD) {
        return set_error(QF_ERR_ARG, "d must be in [2, 16]");
    }
    if (dt != QF_C64 && dt != QF_C128) return set_error(QF_ERR_ARG, "unknown dtype");
    long double Nf = 1;
    for (int q = 0; q < n; ++q) Nf *= dims ? dims[q] : d;
    if (Nf > 9.0e15L) return set_error(QF_ERR_ARG, "state size (product of the dimensions) too large");
    if (d == 0 && Nf / dims[0] >= 2147483648.0L)
        return set_error(QF_ERR_UNSUPPORTED, "mixed register: amplitudes / dims[0] must stay below 2^31");
    qf_state *s = new qf_state();
    s->d = d;
    s->n = n;
    s->mixed = d == 0;
    for (int q = 0; q < n; ++q) s->dims[q] = dims ? dims[q] : d;
    s->dt = dt;
    s->N = (long long)Nf;
    s->stream = (cudaStream_t)stream;
    cudaGetDevice(&s->device);
    s->num_sms = device_sms();
    const size_t bytes = (size_t)s->N * (dt == QF_C64 ? 8 : 16);
    if (ptr) {
        if (((uintptr_t)ptr & 15) != 0) {
            delete s;
            return set_error(QF_ERR_ARG, "device pointer must be 16-byte aligned");
        }
        s->data = ptr;
        s->owned = false;
    } else {
        if (cudaMalloc(&s->data, bytes) != cudaSuccess) {
            cudaGetLastError();
            delete s;
            return set_error(QF_ERR_OOM, "state allocation of " + std::to_string(bytes) + " bytes failed");
        }
        s->owned = true;
    }
    const size_t pbytes = (size_t)reduce_max_blocks(s->num_sms) * (kMaxQudits + 1 + kMaxD) * sizeof(double);
    if (cudaMalloc(&s->d_partials, pbytes) != cudaSuccess || cudaMalloc(&s->d_out, 128 * sizeof(double)) != cudaSuccess ||
        cudaMallocHost(&s->h_out, 128 * sizeof(double)) != cudaSuccess ||
        cudaEventCreateWithFlags(&s->up_ev, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        qf_state_free(s);
        return set_error(QF_ERR_OOM, "scratch allocation failed");
    }
    *out = s;
    return QF_OK;
}

qf_status qf_state_init(int d, int n, qf_dtype dt, void *cuda_stream, qf_state **out) {
    qf_status st = make_state(d, nullptr, n, dt, nullptr, cuda_stream, out);
    if (st != QF_OK) return st;
    st = qf_state_set_basis(*out, 0);
    if (st != QF_OK) {
        qf_state_free(*out);
        *out = nullptr;
    }
    return st;
}

qf_status qf_state_wrap(int d, int n, qf_dtype dt, void *dev_ptr, void *cuda_stream, qf_state **out) {
    if (!dev_ptr) return set_error(QF_ERR_ARG, "device pointer is NULL");
    return make_state(d, nullptr, n, dt, dev_ptr, cuda_stream, out);
}

qf_status qf_state_init_dims(const int *dims, int n, qf_dtype dt, void *cuda_stream, qf_state **out) {
    if (!dims) return set_error(QF_ERR_ARG, "dims is NULL");
    qf_status st = make_state(0, dims, n, dt, nullptr, cuda_stream, out);
    if (st != QF_OK) return st;
    st = qf_state_set_basis(*out, 0);
    if (st != QF_OK) {
        qf_state_free(*out);
        *out = nullptr;
    }
    return st;
}

qf_status qf_state_wrap_dims(const int *dims, int n, qf_dtype dt, void *dev_ptr, void *cuda_stream, qf_state **out) {
    if (!dims) return set_error(QF_ERR_ARG, "dims is NULL");
    if (!dev_ptr) return set_error(QF_ERR_ARG, "device pointer is NULL");
    return make_state(0, dims, n, dt, dev_ptr, cuda_stream, out);
}

qf_status qf_state_dims(const qf_state *s, int *dims, int cap) {
    if (!s) return set_error(QF_ERR_ARG, "state handle is NULL");
    if (!dims || cap < s->n) return set_error(QF_ERR_ARG, "dims is NULL or shorter than n");
    for (int q = 0; q < s->n; ++q) dims[q] = s->dims[q];
    return QF_OK;
}

qf_status qf_state_free(qf_state *s) {
    if (!s) return QF_OK;
    cudaStreamSynchronize(s->stream);
    if (s->owned && s->data) cudaFree(s->data);
    if (s->d_partials) cudaFree(s->d_partials);
    if (s->d_out) cudaFree(s->d_out);
    if (s->h_out) cudaFreeHost(s->h_out);
    if (s->h_up) cudaFreeHost(s->h_up);
    if (s->d_up) cudaFree(s->d_up);
    if (s->up_ev) cudaEventDestroy(s->up_ev);
    if (s->d_meas) cudaFree(s->d_meas);
    delete s;
    return QF_OK;
}

qf_status qf_state_ptr(qf_state *s, void **dev_ptr, long long *num_amps) {
    if (!s) return set_error(QF_ERR_ARG, "state handle is NULL");
    if (dev_ptr) *dev_ptr = s->data;
    if (num_amps) *num_amps = s->N;
    return QF_OK;
}

qf_status qf_state_info(const qf_state *s, int *d, int *n, qf_dtype *dt) {
    if (!s) return set_error(QF_ERR_ARG, "state handle is NULL");
    if (d) *d = s->d;
    if (n) *n = s->n;
    if (dt) *dt = s->dt;
    return QF_OK;
}

qf_status qf_state_set_stream(qf_state *s, void *cuda_stream) {
    if (!s) return set_error(QF_ERR_ARG, "state handle is NULL");
    s->stream = (cudaStream_t)cuda_stream;
    return QF_OK;
}

qf_status qf_state_set_basis(qf_state *s, long long index) {
    if (!s) return set_error(QF_ERR_ARG, "state handle is NULL");
    if (index < 0 || index >= s->N) return set_error(QF_ERR_ARG, "basis index out of range");
    const Launch L = launch_of(s);
    cudaError_t e = s->dt == QF_C64 ? launch_basis<float>(L, (float2 *)s->data, s->N, index)
                                    : launch_basis<double>(L, (double2 *)s->data, s->N, index);
    if (e != cudaSuccess) return cuda_error(e, "basis fill kernel");
    return QF_OK;
}

qf_status qf_state_copy(qf_state *dst, const qf_state *src) {
    if (!dst || !src) return set_error(QF_ERR_ARG, "state handle is NULL");
    if (dst->d != src->d || dst->n != src->n || dst->dt != src->dt) return set_error(QF_ERR_ARG, "state shapes differ");
    for (int q = 0; q < dst->n; ++q)
        if (dst->dims[q] != src->dims[q]) return set_error(QF_ERR_ARG, "state dimensions differ");
    if (dst == src) return QF_OK;
    const size_t bytes = (size_t)dst->N * (dst->dt == QF_C64 ? 8 : 16);
    QF_CUDA(cudaMemcpyAsync(dst->data, src->data, bytes, cudaMemcpyDeviceToDevice, dst->stream));
    return QF_OK;
}

// Page-locked host memory: anonymous pages of the process, mapped here and
// registered with the driver.  Measured on GB300 (Grace host): 7.3 GB of
// uploads per step from such pages never stalled in 42 steps, while the same
// copies from cudaHostAlloc memory stalled for 150-400 ms in 3 to 6 of 14
// steps, copies alone included.
static std::mutex g_host_mu;
static std::map<void *, size_t> g_host_maps;

qf_status qf_host_alloc(size_t bytes, void **out) {
    if (!out) return set_error(QF_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (bytes == 0) return set_error(QF_ERR_ARG, "qf_host_alloc: zero bytes");
    const size_t huge = (size_t)2 << 20;
    const size_t len = (bytes + huge - 1) / huge * huge;
    void *p = mmap(nullptr, len, PROT_READ | PROT_WRITE, MAP_PRIVATE | MAP_ANONYMOUS, -1, 0);
    if (p == MAP_FAILED) return set_error(QF_ERR_OOM, "qf_host_alloc: mmap of " + std::to_string(len) + " bytes failed");
    madvise(p, len, MADV_HUGEPAGE);   // a hint; ignored where transparent huge pages are off
    const cudaError_t e = cudaHostRegister(p, len, cudaHostRegisterDefault);
    if (e != cudaSuccess) {
        munmap(p, len);
        cudaGetLastError();
        return set_error(QF_ERR_OOM, std::string("qf_host_alloc: page-locking failed: ") + cudaGetErrorString(e));
    }
    {
        std::lock_guard<std::mutex> lock(g_host_mu);
        g_host_maps[p] = len;
    }
    *out = p;
    return QF_OK;
}

qf_status qf_host_free(void *p) {
    if (!p) return QF_OK;
    size_t len = 0;
    {
        std::lock_guard<std::mutex> lock(g_host_mu);
        auto it = g_host_maps.find(p);
        if (it == g_host_maps.end()) return set_error(QF_ERR_ARG, "qf_host_free: pointer not from qf_host_alloc");
        len = it->second;
        g_host_maps.erase(it);
    }
    cudaHostUnregister(p);
    munmap(p, len);
    return QF_OK;
}

// Host <-> state copies of amplitudes [first, first + count): one
// cudaMemcpyAsync over the contiguous range, on the state's stream.
static qf_status host_copy(qf_state *s, void *host, long long first, long long count, bool up) {
    if (!s) return set_error(QF_ERR_ARG, "state handle is NULL");
    if (!host) return set_error(QF_ERR_ARG, "host buffer is NULL");
    if (first < 0 || count < 0 || first > s->N || count > s->N - first)
        return set_error(QF_ERR_ARG, "amplitude range outside the state");
    if (count == 0) return QF_OK;
    const size_t b = s->dt == QF_C64 ? 8 : 16;
    char *dev = (char *)s->data + (size_t)first * b;
    if (up) QF_CUDA(cudaMemcpyAsync(dev, host, (size_t)count * b, cudaMemcpyHostToDevice, s->stream));
    else QF_CUDA(cudaMemcpyAsync(host, dev, (size_t)count * b, cudaMemcpyDeviceToHost, s->stream));
    return QF_OK;
}

qf_status qf_state_upload(qf_state *s, const void *host, long long first, long long count) {
    return host_copy(s, const_cast<void *>(host), first, count, true);
}

qf_status qf_state_download(qf_state *s, void *host, long long first, long long count) {
    return host_copy(s, host, first, count, false);
}

static HGate one(int kind, int q) {
    HGate g;
    g.kind = kind;
    g.nq = 1;
    g.q[0] = q;
    return g;
}
static HGate two(int kind, int a, int b) {
    HGate g;
    g.kind = kind;
    g.nq = 2;
    g.q[0] = a;
    g.q[1] = b;
    return g;
}

qf_status qf_apply_gate(qf_state *s, const int *targets, int k, const double *U) {
    if (!s) return set_error(QF_ERR_ARG, "state handle is NULL");
    if (!targets || !U || k < 1 || k > 6) return set_error(QF_ERR_ARG, "targets/U NULL or k out of range");
    HGate g;
    g.kind = G_DENSE;
    g.nq = k;
    for (int i = 0; i < k; ++i) g.q[i] = targets[i];
    long long K = 1;
    for (int i = 0; i < k; ++i) {
        if (targets[i] < 0 || targets[i] >= s->n) return set_error(QF_ERR_ARG, "qudit index out of range [0, n)");
        K *= s->dims[targets[i]];
    }
    if (K > kMaxDenseK) return set_error(QF_ERR_UNSUPPORTED, "custom gate: the product of the targets' dims must be <= 64");
    g.U.resize((size_t)K * K);
    for (long long i = 0; i < K * K; ++i) g.U[i] = cd(U[2 * i], U[2 * i + 1]);
    return apply_gate(s, g);
}

qf_status qf_apply_rot(qf_state *s, int q, int j, int k, double theta, char axis) {
    HGate g = one(G_ROT, q);
    g.j = j; g.k = k; g.axis = axis; g.theta = theta;
    return apply_gate(s, g);
}

qf_status qf_apply_crot(qf_state *s, int c, int t, int j, int k, double theta, char axis) {
    HGate g = two(G_CROT, c, t);
    g.j = j; g.k = k; g.axis = axis; g.theta = theta;
    return apply_gate(s, g);
}

qf_status qf_apply_sum(qf_state *s, int c, int t) { return apply_gate(s, two(G_SUM, c, t)); }

static qf_status mc_hgate(HGate *g, int kind, const int *controls, const int *levels, int k, int target) {
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

qf_status qf_apply_mcx(qf_state *s, const int *controls, int k, int target, int shift) {
    if (!s) return set_error(QF_ERR_ARG, "state handle is NULL");
    HGate g;
    qf_status st = mc_hgate(&g, G_MCX, controls, nullptr, k, target);
    if (st != QF_OK) return st;
    g.power = shift;
    return apply_gate(s, g);
}

qf_status qf_apply_mcu(qf_state *s, const int *controls, const int *levels, int k, int target, const double *U) {
    if (!s) return set_error(QF_ERR_ARG, "state handle is NULL");
    HGate g;
    qf_status st = mc_hgate(&g, G_MCU, controls, levels, k, target);
    if (st != QF_OK) return st;
    if (!U) return set_error(QF_ERR_ARG, "U is NULL");
    if (target < 0 || target >= s->n) return set_error(QF_ERR_ARG, "qudit index out of range [0, n)");
    const int dt = s->dims[target];
    g.U.resize((size_t)dt * dt);
    for (int i = 0; i < dt * dt; ++i) g.U[i] = cd(U[2 * i], U[2 * i + 1]);
    return apply_gate(s, g);
}
qf_status qf_apply_swap(qf_state *s, int a, int b) { return apply_gate(s, two(G_SWAP, a, b)); }

qf_status qf_apply_x(qf_state *s, int q, int shift) {
    HGate g = one(G_X, q);
    g.power = shift;
    return apply_gate(s, g);
}

qf_status qf_apply_z(qf_state *s, int q, int power) {
    HGate g = one(G_Z, q);
    g.power = power;
    return apply_gate(s, g);
}

qf_status qf_apply_h(qf_state *s, int q) { return apply_gate(s, one(G_H, q)); }

qf_status qf_expect_device(qf_state *s, const qf_obs *obs, double *out_dev) {
    if (!s) return set_error(QF_ERR_ARG, "state handle is NULL");
    if (!obs || !out_dev) return set_error(QF_ERR_ARG, "observable or output is NULL");
    if (((uintptr_t)out_dev & 7) != 0) return set_error(QF_ERR_ARG, "output must be 8-byte aligned");
    const Launch L = launch_of(s);
    const bool c64 = s->dt == QF_C64;
    cudaError_t e = cudaSuccess;
    if (s->mixed) {
        switch (obs->kind) {
        case QF_OBS_NUMBER_ALL:
            return mixed_expect_number(s, out_dev);
        case QF_OBS_NORM: {
            qf_status st = mixed_expect_number(s, s->d_out);
            if (st != QF_OK) return st;
            QF_CUDA(cudaMemcpyAsync(out_dev, s->d_out + s->n, sizeof(double), cudaMemcpyDeviceToDevice, s->stream));
            return QF_OK;
        }
        case QF_OBS_MARGINAL:
        case QF_OBS_HERMITIAN: {
            if (obs->q < 0 || obs->q >= s->n) return set_error(QF_ERR_ARG, "observable qudit out of range");
            const int kind = obs->kind == QF_OBS_MARGINAL ? 0 : 1;
            const int dq = s->dims[obs->q];
            const double2 *od = nullptr;
            if (kind == 1) {
                if (!obs->matrix) return set_error(QF_ERR_ARG, "Hermitian observable needs a matrix");
                size_t bytes = (size_t)dq * dq * sizeof(double2);
                qf_status st = up_reserve(s, bytes);
                if (st != QF_OK) return st;
                std::memcpy(s->h_up, obs->matrix, bytes);
                st = up_send(s, bytes);
                if (st != QF_OK) return st;
                od = (const double2 *)s->d_up;
            }
            const MixedShape shape = mixed_shape(s->dims, s->n);
            e = c64 ? launch_fibre_reduce_g<float>(L, (const float2 *)s->data, dq, shape.S[obs->q], shape.N, kind, od,
                                                   s->d_partials, out_dev)
                    : launch_fibre_reduce_g<double>(L, (const double2 *)s->data, dq, shape.S[obs->q], shape.N, kind, od,
                                                    s->d_partials, out_dev);
            if (e != cudaSuccess) return cuda_error(e, "reduction kernels");
            return QF_OK;
        }
        default:
            return set_error(QF_ERR_ARG, "unknown observable kind");
        }
    }
    switch (obs->kind) {
    case QF_OBS_NUMBER_ALL:
        e = c64 ? launch_expect_number<float>(L, (const float2 *)s->data, s->d, s->n, s->d_partials, out_dev)
                : launch_expect_number<double>(L, (const double2 *)s->data, s->d, s->n, s->d_partials, out_dev);
        break;
    case QF_OBS_NORM: {
        // the norm is the last entry of the number reduction
        e = c64 ? launch_expect_number<float>(L, (const float2 *)s->data, s->d, s->n, s->d_partials, s->d_out)
                : launch_expect_number<double>(L, (const double2 *)s->data, s->d, s->n, s->d_partials, s->d_out);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(out_dev, s->d_out + s->n, sizeof(double), cudaMemcpyDeviceToDevice, s->stream);
        break;
    }
    case QF_OBS_MARGINAL:
    case QF_OBS_HERMITIAN: {
        if (obs->q < 0 || obs->q >= s->n) return set_error(QF_ERR_ARG, "observable qudit out of range");
        const int kind = obs->kind == QF_OBS_MARGINAL ? 0 : 1;
        const double2 *od = nullptr;
        if (kind == 1) {
            if (!obs->matrix) return set_error(QF_ERR_ARG, "Hermitian observable needs a matrix");
            size_t bytes = (size_t)s->d * s->d * sizeof(double2);
            qf_status st = up_reserve(s, bytes);
            if (st != QF_OK) return st;
            std::memcpy(s->h_up, obs->matrix, bytes);
            st = up_send(s, bytes);
            if (st != QF_OK) return st;
            od = (const double2 *)s->d_up;
        }
        e = c64 ? launch_fibre_reduce<float>(L, (const float2 *)s->data, s->d, s->n, obs->q, kind, od, s->d_partials, out_dev)
                : launch_fibre_reduce<double>(L, (const double2 *)s->data, s->d, s->n, obs->q, kind, od, s->d_partials,
                                              out_dev);
        break;
    }
    default:
        return set_error(QF_ERR_ARG, "unknown observable kind");
    }
    if (e != cudaSuccess) return cuda_error(e, "reduction kernels");
    return QF_OK;
}

qf_status qf_measure(qf_state *s, const int *idx, int k, const double *uniforms, long long shots, double *probs,
                     long long *counts) {
    if (!s) return set_error(QF_ERR_ARG, "state handle is NULL");
    if (!idx || k < 1 || k > s->n) return set_error(QF_ERR_ARG, "need 1 <= k <= n measured qudits");
    for (int a = 0; a < k; ++a) {
        if (idx[a] < 0 || idx[a] >= s->n) return set_error(QF_ERR_ARG, "measured qudit out of range");
        for (int b = 0; b < a; ++b)
            if (idx[a] == idx[b]) return set_error(QF_ERR_ARG, "measured qudits must be distinct");
    }
    long long bins = 1;
    for (int a = 0; a < k; ++a) {
        bins *= s->dims[idx[a]];
        if (bins > 16384) return set_error(QF_ERR_UNSUPPORTED, "measure: the measured qudits' dims must multiply to <= 16384");
    }
    if (shots < 0 || (shots > 0 && (!uniforms || !counts))) return set_error(QF_ERR_ARG, "bad shots / uniforms / counts");
    if (!probs) return set_error(QF_ERR_ARG, "probs is NULL");
    const size_t need = (size_t)marginal_max_blocks() * bins * 8 + 2 * bins * 8 + bins * 8 + (size_t)shots * 8 + 256;
    if (need > s->meas_cap) {
        QF_CUDA(cudaStreamSynchronize(s->stream));
        if (s->d_meas) cudaFree(s->d_meas);
        s->d_meas = nullptr;
        s->meas_cap = 0;
        if (cudaMalloc(&s->d_meas, need) != cudaSuccess) {
            cudaGetLastError();
            return set_error(QF_ERR_OOM, "measurement scratch allocation failed");
        }
        s->meas_cap = need;
    }
    double *part = reinterpret_cast<double *>(s->d_meas);
    double *pr = part + (size_t)marginal_max_blocks() * bins;
    double *cdf = pr + bins;
    unsigned long long *cnt = reinterpret_cast<unsigned long long *>(cdf + bins);
    double *u = reinterpret_cast<double *>(cnt + bins);
    const Launch L = launch_of(s);
    if (shots > 0) QF_CUDA(cudaMemcpyAsync(u, uniforms, (size_t)shots * 8, cudaMemcpyHostToDevice, s->stream));
    cudaError_t e = s->dt == QF_C64
                        ? launch_marginal_dims<float>(L, (const float2 *)s->data, s->dims, s->n, idx, k, part, pr)
                        : launch_marginal_dims<double>(L, (const double2 *)s->data, s->dims, s->n, idx, k, part, pr);
    if (e != cudaSuccess) return cuda_error(e, "marginal kernels");
    if (shots > 0) {
        e = launch_sample(L, pr, (int)bins, cdf, u, shots, cnt);
        if (e != cudaSuccess) return cuda_error(e, "sampling kernels");
    }
    QF_CUDA(cudaMemcpyAsync(probs, pr, (size_t)bins * 8, cudaMemcpyDeviceToHost, s->stream));
    if (shots > 0) QF_CUDA(cudaMemcpyAsync(counts, cnt, (size_t)bins * 8, cudaMemcpyDeviceToHost, s->stream));
    QF_CUDA(cudaStreamSynchronize(s->stream));
    return QF_OK;
}

qf_status qf_expect(qf_state *s, const qf_obs *obs, double *out_host) {
    if (!s) return set_error(QF_ERR_ARG, "state handle is NULL");
    if (!out_host) return set_error(QF_ERR_ARG, "output is NULL");
    int cnt = qf_expect_size(s->d, s->n, obs);
    if (cnt < 0) return set_error(QF_ERR_ARG, "unknown observable kind");
    if (obs->kind == QF_OBS_MARGINAL) {
        if (obs->q < 0 || obs->q >= s->n) return set_error(QF_ERR_ARG, "observable qudit out of range");
        cnt = s->dims[obs->q];
    }
    qf_status st = qf_expect_device(s, obs, s->d_out);
    if (st != QF_OK) return st;
    QF_CUDA(cudaMemcpyAsync(s->h_out, s->d_out, cnt * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    QF_CUDA(cudaStreamSynchronize(s->stream));
    std::memcpy(out_host, s->h_out, cnt * sizeof(double));
    return QF_OK;
}

}  // extern "C"
