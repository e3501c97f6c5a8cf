// qf_jit.cu -- tile passes of recorded programs specialised at plan time.
//
// The generic tile kernel (k_tile.cu) interprets a pass: for every register
// block of every tile it reads each op's kind, slots, levels and matrix
// entries from shared memory and branches on them.  A program's passes are
// fixed once it is planned, so each tile pass is instead emitted as CUDA C++
// with everything structural written as literals -- the register slots and
// element offsets of every stage, the level pairs, control slots, diagonal
// masks, shift amounts and the tile geometry -- and compiled at run time with
// NVRTC for the current GPU.  Only the numbers that change between runs (the
// gate entries, which depend on the rotation angles) are passed, as kernel
// parameters indexed by literals, so they reach the FMAs straight from the
// constant bank.  Per amplitude a pass then costs its loads and stores, one
// shared-memory round trip per register stage and the gates' own arithmetic.
//
// The arithmetic is that of the generic kernel (stage_device.cuh): complex64
// entries prepared as (re, re, -im, im) for paired FP32 FMAs, complex128 in
// FP64 FMAs.  NVRTC is loaded with dlopen and the driver entry points through
// the runtime, so the library itself links against neither.
#include <cuda.h>
#include <dlfcn.h>
#include <nvrtc.h>

#include <sys/stat.h>
#include <unistd.h>

#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <thread>
#include <functional>
#include <map>
#include <mutex>
#include <sstream>
#include <string>
#include <vector>

#include "qf_host.h"

namespace qf {

// ------------------------------------------------------------------ NVRTC and driver entry points
namespace {

struct Nvrtc {
    nvrtcResult (*create)(nvrtcProgram *, const char *, const char *, int, const char *const *, const char *const *);
    nvrtcResult (*compile)(nvrtcProgram, int, const char *const *);
    nvrtcResult (*log_size)(nvrtcProgram, size_t *);
    nvrtcResult (*log)(nvrtcProgram, char *);
    nvrtcResult (*cubin_size)(nvrtcProgram, size_t *);
    nvrtcResult (*cubin)(nvrtcProgram, char *);
    nvrtcResult (*destroy)(nvrtcProgram *);
    nvrtcResult (*version)(int *, int *);
};

struct Driver {
    CUresult (*module_load)(CUmodule *, const void *);
    CUresult (*get_function)(CUfunction *, CUmodule, const char *);
    CUresult (*launch)(CUfunction, unsigned, unsigned, unsigned, unsigned, unsigned, unsigned, unsigned, CUstream,
                       void **, void **);
    CUresult (*set_attribute)(CUfunction, CUfunction_attribute, int);
    CUresult (*occupancy)(int *, CUfunction, int, size_t);
};

std::mutex g_mu;
bool g_loaded = false;
std::string g_load_err;
Nvrtc g_nv;
Driver g_drv;
// (device ordinal, generated source) -> loaded module: a module belongs to the
// context it was loaded in, so each device loads its own
std::map<std::pair<int, std::string>, CUmodule> g_modules;
std::string g_tool_tag;   // NVRTC and driver versions: part of every cached cubin's key

bool load_apis() {
    if (g_loaded) return true;
    if (!g_load_err.empty()) return false;
    void *h = nullptr;
    for (const char *name : {"libnvrtc.so.13", "libnvrtc.so", "libnvrtc.so.12"}) {
        h = dlopen(name, RTLD_NOW | RTLD_LOCAL);
        if (h) break;
    }
    if (!h) {
        g_load_err = "NVRTC (libnvrtc.so) not found; it compiles the program's tile passes";
        return false;
    }
    auto sym = [&](const char *s) { return dlsym(h, s); };
    g_nv.create = (decltype(g_nv.create))sym("nvrtcCreateProgram");
    g_nv.compile = (decltype(g_nv.compile))sym("nvrtcCompileProgram");
    g_nv.log_size = (decltype(g_nv.log_size))sym("nvrtcGetProgramLogSize");
    g_nv.log = (decltype(g_nv.log))sym("nvrtcGetProgramLog");
    g_nv.cubin_size = (decltype(g_nv.cubin_size))sym("nvrtcGetCUBINSize");
    g_nv.cubin = (decltype(g_nv.cubin))sym("nvrtcGetCUBIN");
    g_nv.destroy = (decltype(g_nv.destroy))sym("nvrtcDestroyProgram");
    g_nv.version = (decltype(g_nv.version))sym("nvrtcVersion");
    if (!g_nv.create || !g_nv.compile || !g_nv.log_size || !g_nv.log || !g_nv.cubin_size || !g_nv.cubin ||
        !g_nv.destroy || !g_nv.version) {
        g_load_err = "NVRTC symbols missing";
        return false;
    }
    auto drv = [&](const char *s, void **fp) {
        cudaDriverEntryPointQueryResult q;
        return cudaGetDriverEntryPointByVersion(s, fp, 13000, cudaEnableDefault, &q) == cudaSuccess &&
               q == cudaDriverEntryPointSuccess && *fp;
    };
    if (!drv("cuModuleLoadData", (void **)&g_drv.module_load) ||
        !drv("cuModuleGetFunction", (void **)&g_drv.get_function) || !drv("cuLaunchKernel", (void **)&g_drv.launch) ||
        !drv("cuFuncSetAttribute", (void **)&g_drv.set_attribute) ||
        !drv("cuOccupancyMaxActiveBlocksPerMultiprocessor", (void **)&g_drv.occupancy)) {
        cudaGetLastError();
        g_load_err = "CUDA driver entry points for module loading are unavailable";
        return false;
    }
    int vmaj = 0, vmin = 0, drv_ver = 0;
    g_nv.version(&vmaj, &vmin);
    cudaDriverGetVersion(&drv_ver);
    g_tool_tag = "nvrtc" + std::to_string(vmaj) + "." + std::to_string(vmin) + "|driver" + std::to_string(drv_ver);
    g_loaded = true;
    return true;
}

// Device helpers every generated kernel starts with.
const char *kPrelude = R"(
#if QJ_C64
typedef float2 C;
typedef float4 P;
__device__ __forceinline__ C jm(const P p, C a) {
    const C r = __fmul2_rn(make_float2(p.x, p.y), a);
    return __ffma2_rn(make_float2(p.z, p.w), make_float2(a.y, a.x), r);
}
__device__ __forceinline__ C jma(const P p, C a, C acc) {
    acc = __ffma2_rn(make_float2(p.x, p.y), a, acc);
    return __ffma2_rn(make_float2(p.z, p.w), make_float2(a.y, a.x), acc);
}
__device__ __forceinline__ C jrm(const P p, C a) { return __fmul2_rn(make_float2(p.x, p.x), a); }
__device__ __forceinline__ C jrma(const P p, C a, C acc) { return __ffma2_rn(make_float2(p.x, p.x), a, acc); }
__device__ __forceinline__ C jn(C a) { return a; }
#define QJ_CP_BYTES "8"
#define QJ_CP_KIND "ca"
#elif QJ_DF
// Double-float complex128 (values hi + lo of two floats; C = (hi.re, hi.im,
// lo.re, lo.im)).  An entry u = ur + i ui holds (urh, urh, -uih, uih) and
// (url, url, -uil, uil), so one complex product is two paired products:
// (ur, ur) * (xr, xi) + (-ui, ui) * (xi, xr).  Each paired product a * b of
// hi/lo pairs is ph = ah * bh rounded plus pe = the exact error of ah * bh
// (one FMA, Dekker's TwoProduct) + ah * bl + al * bh; sums keep their rounding
// error exactly (Knuth's TwoSum) in the low part; jn renormalizes.
typedef float4 C;
struct __align__(16) P { float4 h, l; };
__device__ __forceinline__ float2 qf2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 qng(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ void qts(float2 a, float2 b, float2 &s, float2 &e) {
    s = __fadd2_rn(a, b);
    const float2 bb = __fadd2_rn(s, qng(a));
    e = __fadd2_rn(__fadd2_rn(a, qng(__fadd2_rn(s, qng(bb)))), __fadd2_rn(b, qng(bb)));
}
__device__ __forceinline__ void qtp(float2 ah, float2 al, float2 bh, float2 bl, float2 &p, float2 &e) {
    p = __fmul2_rn(ah, bh);
    e = __ffma2_rn(ah, bh, qng(p));
    e = __ffma2_rn(ah, bl, e);
    e = __ffma2_rn(al, bh, e);
}
__device__ __forceinline__ C jm(const P p, C a) {
    float2 p1, e1, p2, e2, s, t;
    qtp(qf2(p.h.x, p.h.y), qf2(p.l.x, p.l.y), qf2(a.x, a.y), qf2(a.z, a.w), p1, e1);
    qtp(qf2(p.h.z, p.h.w), qf2(p.l.z, p.l.w), qf2(a.y, a.x), qf2(a.w, a.z), p2, e2);
    qts(p1, p2, s, t);
    const float2 l = __fadd2_rn(__fadd2_rn(e1, e2), t);
    return make_float4(s.x, s.y, l.x, l.y);
}
__device__ __forceinline__ C jma(const P p, C a, C acc) {
    float2 p1, e1, p2, e2, s, t1, t2;
    qtp(qf2(p.h.x, p.h.y), qf2(p.l.x, p.l.y), qf2(a.x, a.y), qf2(a.z, a.w), p1, e1);
    qtp(qf2(p.h.z, p.h.w), qf2(p.l.z, p.l.w), qf2(a.y, a.x), qf2(a.w, a.z), p2, e2);
    qts(qf2(acc.x, acc.y), p1, s, t1);
    qts(s, p2, s, t2);
    const float2 l = __fadd2_rn(__fadd2_rn(qf2(acc.z, acc.w), __fadd2_rn(e1, e2)), __fadd2_rn(t1, t2));
    return make_float4(s.x, s.y, l.x, l.y);
}
__device__ __forceinline__ C jrm(const P p, C a) {
    float2 q, e;
    qtp(qf2(p.h.x, p.h.x), qf2(p.l.x, p.l.x), qf2(a.x, a.y), qf2(a.z, a.w), q, e);
    return make_float4(q.x, q.y, e.x, e.y);
}
__device__ __forceinline__ C jrma(const P p, C a, C acc) {
    float2 q, e, s, t;
    qtp(qf2(p.h.x, p.h.x), qf2(p.l.x, p.l.x), qf2(a.x, a.y), qf2(a.z, a.w), q, e);
    qts(qf2(acc.x, acc.y), q, s, t);
    const float2 l = __fadd2_rn(qf2(acc.z, acc.w), __fadd2_rn(e, t));
    return make_float4(s.x, s.y, l.x, l.y);
}
__device__ __forceinline__ C jn(C a) {
    float2 s, t;
    qts(qf2(a.x, a.y), qf2(a.z, a.w), s, t);
    return make_float4(s.x, s.y, t.x, t.y);
}
// Gradient terms of the adjoint sweep as double-float reals (hi, lo):
// Im(conj(l) g) = lr gi - li gr from one paired TwoProduct and a TwoSum.
__device__ __forceinline__ void qts1(float a, float b, float &s, float &e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ float2 qim(C l, C g) {
    float2 p, e;
    qtp(qf2(l.x, l.y), qf2(l.z, l.w), qf2(g.y, g.x), qf2(g.w, g.z), p, e);
    float s, t;
    qts1(p.x, -p.y, s, t);
    return qf2(s, t + (e.x - e.y));
}
__device__ __forceinline__ float2 qad(float2 a, float2 b) {
    float s, t;
    qts1(a.x, b.x, s, t);
    return qf2(s, a.y + b.y + t);
}
// a * (mh + ml): a double-float real times a double-float entry
__device__ __forceinline__ float2 qmu(float2 a, float mh, float ml) {
    const float p = a.x * mh;
    const float e = fmaf(a.x, mh, -p) + fmaf(a.x, ml, a.y * mh);
    return qf2(p, e);
}
__device__ __forceinline__ double qdd(float2 a) { return (double)a.x + (double)a.y; }
#define QJ_CP_BYTES "16"
#define QJ_CP_KIND "cg"
#else
typedef double2 C;
typedef double2 P;
__device__ __forceinline__ C jm(const P p, C a) {
    return make_double2(fma(p.x, a.x, -p.y * a.y), fma(p.x, a.y, p.y * a.x));
}
__device__ __forceinline__ C jma(const P p, C a, C acc) {
    acc.x = fma(p.x, a.x, acc.x); acc.x = fma(-p.y, a.y, acc.x);
    acc.y = fma(p.x, a.y, acc.y); acc.y = fma(p.y, a.x, acc.y);
    return acc;
}
__device__ __forceinline__ C jrm(const P p, C a) { return make_double2(p.x * a.x, p.x * a.y); }
__device__ __forceinline__ C jrma(const P p, C a, C acc) { return make_double2(fma(p.x, a.x, acc.x), fma(p.x, a.y, acc.y)); }
__device__ __forceinline__ C jn(C a) { return a; }
#define QJ_CP_BYTES "16"
#define QJ_CP_KIND "cg"
#endif
__device__ __forceinline__ unsigned qj_smem(const void *p) {
    unsigned r;
    asm("{ .reg .u64 t; cvta.to.shared.u64 t, %1; cvt.u32.u64 %0, t; }" : "=r"(r) : "l"(p));
    return r;
}
__device__ __forceinline__ void qj_cp(C *dst, const C *src) {
    asm volatile("cp.async." QJ_CP_KIND ".shared.global [%0], [%1], " QJ_CP_BYTES ";\n" ::"r"(qj_smem(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void qj_wait() { asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory"); }
__device__ __forceinline__ void qj_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void qj_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void qj_wait0() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }
// two complex64 amplitudes (16 bytes, both addresses 16-byte aligned)
__device__ __forceinline__ void qj_cp2(C *dst, const C *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(qj_smem(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void qj_st2(C *dst, const C *src) {
    *reinterpret_cast<float4 *>(dst) = *reinterpret_cast<const float4 *>(src);
}
)";

constexpr int kParamPoolMax = 1800;   // pool entries passed as kernel parameters (16 bytes each)

int ipow_i(int d, int e) {
    int r = 1;
    for (int i = 0; i < e; ++i) r *= d;
    return r;
}

// Source of one tile pass.  `ops` are tile-local with their stage slots; the
// pool offsets op.mat index the pass's prepared entries.
struct PassSrc {
    int d, T, SEG, nt, kA, nruns, K, threads;
    bool c128, params;   // params: entries in the kernel parameters, else global
    bool df = false;     // complex128 in double-float arithmetic (32-byte entries)
    int npool;
    bool adj = false;    // reverse pass of the adjoint sweep (psi and lambda, gradient columns)
    long long ntiles = 0;                        // tiles of the pass
    std::vector<long long> runM, runS, strideA;  // tile geometry (literals in the source)
    int ncols = 0;       // gradient columns (parametrised ops, op.gcol) of an adjoint pass
    std::vector<TOp> ops;
    std::vector<TStage> stages;
    // Padded tile layout (forward complex64 passes at odd d, runs of >= 3
    // amplitudes): every run of SEG amplitudes sits in a slot of SEG + 1,
    // shifted by one where it starts at an odd amplitude, so that each run
    // moves between HBM and shared memory as 16-byte amplitude pairs.  A run
    // of an odd-d state starts at an odd index exactly when its run number
    // plus the tile base is odd (every stride is odd).
    bool pad = false;
    int slots() const { return pad ? (T / SEG) * (SEG + 1) : T; }   // amplitudes of one tile buffer
    // <N_q> and the norm reduced in this pass (the last pass of a complex64
    // program, when the caller asks for them): global qudit of each local
    // position, and for each outer qudit x the divisor D_x of the tile index
    // (digit = (t / D_x) mod d)
    bool red = false;
    int n = 0;
    std::vector<int> local_q;
    // Direct stages (forward complex64): the first register stage loads its
    // blocks from HBM (din) and the last stores them to HBM (dout) instead of
    // going through the shared-memory tile, where every slot of that stage is
    // an active qudit (its registers then sit in whole runs: consecutive
    // threads read consecutive amplitudes of a run).
    bool din = false, dout = false;
    bool pf = false;   // L2 prefetch of the next tile (forward complex64 passes at odd d)
    std::vector<std::pair<int, long long>> outer_div;
};

// Whether a forward pass of this geometry uses the padded tile layout: runs
// of at least 9 amplitudes (measured on GB300: d=3 passes 3.5 % faster; at
// d=5 with 5-amplitude runs the 20 % larger tile costs the second buffer and
// the passes ran 17 % slower).
static bool use_pad(int d, bool c128, bool adj, int SEG) { return !c128 && !adj && d % 2 == 1 && SEG >= 9; }

class Gen {
  public:
    Gen(const PassSrc &p, std::ostringstream &o) : p_(p), o_(o), D_(p.d) {}

    // Forward pass.  With A.mode != 0 tiles are double-buffered: while a CTA
    // applies the gates to one tile, the copy of its next tile is in flight,
    // so the barrier after a tile's load rarely waits on HBM; the host picks
    // that mode only where the second buffer costs no CTAs per SM.  A pass
    // with a direct first stage has no tile load (its first stage reads HBM),
    // one with a direct last stage no tile store; single-buffered passes with
    // long runs prefetch their next tile into L2 instead.  The tile geometry
    // is literal (tile bases by division by constants in every thread).
    // Shared memory: run offsets, then one or two tiles.
    void kernel(const std::string &name) {
        const int NG = std::max(1, 2 * p_.nruns + p_.kA);
        const int NP = std::max(1, p_.params ? p_.npool : 1);
        const int NA = p_.T / p_.SEG;
        const size_t boff = ((size_t)NA * 8 + 15) & ~(size_t)15;
        o_ << "struct __align__(16) A_" << name << " { C *psi; const P *gp; long long mode; double *rows; long long geo["
           << NG << "]; P pool[" << NP << "]; };\n";
        o_ << "extern \"C\" __global__ void __launch_bounds__(" << p_.threads << ") " << name
           << "(const __grid_constant__ A_" << name << " A) {\n";
        o_ << "  extern __shared__ __align__(16) unsigned char qj_sm[];\n";
        o_ << "  long long *offA = reinterpret_cast<long long *>(qj_sm);\n";
        o_ << "  C *buf0 = reinterpret_cast<C *>(qj_sm + " << boff << ");\n";
        o_ << "  C *buf1 = buf0 + " << p_.slots() << ";   // tile of " << p_.T << " amplitudes\n";
        o_ << "  const int tid = threadIdx.x;\n";
        emit_lanes();
        if (p_.red) {
            o_ << "  double qr_acc0 = 0.0, qr_acc1 = 0.0;\n";
            reduce_roles();
        }
        o_ << "  const bool db = A.mode != 0;\n";
        emit_offA(NA);
        o_ << "  __syncthreads();\n";
        o_ << "  // register stages: " << p_.stages.size() << (p_.din ? ", first from HBM" : "")
           << (p_.dout ? ", last to HBM" : "") << "\n";
        o_ << "  long long t = blockIdx.x;\n";
        if (p_.din) {
            // the first stage reads the tile from HBM: no tile copy, no prefetch
            o_ << "  for (; t < " << p_.ntiles << "; t += gridDim.x) {\n";
            o_ << "    C *tile = buf0;\n";
            o_ << "    const long long base = qj_tb_" << name << "(t);\n";
        } else {
            o_ << "  if (db && t < " << p_.ntiles << ") { C *tile = buf0; const long long base = qj_tb_" << name
               << "(t);\n";
            transfer(true, {{"tile", "A.psi"}});
            o_ << "    qj_commit();\n  }\n";
            o_ << "  for (int it = 0; t < " << p_.ntiles << "; ++it, t += gridDim.x) {\n";
            o_ << "    C *tile = (db && (it & 1)) ? buf1 : buf0;\n";
            o_ << "    const long long base = qj_tb_" << name << "(t);\n";
            o_ << "    if (db) {\n      const long long tn = t + gridDim.x;\n      if (tn < " << p_.ntiles
               << ") { C *tile = (it & 1) ? buf0 : buf1; const long long base = qj_tb_" << name << "(tn);\n";
            transfer(true, {{"tile", "A.psi"}});
            o_ << "      }\n      qj_commit();\n      qj_wait1();\n    } else {\n";
            transfer(true, {{"tile", "A.psi"}});
            o_ << "      qj_commit();\n      qj_wait0();\n    }\n";
            o_ << "    __syncthreads();\n";
        }
        // the prefetch goes between the first two stages (barriers keep its
        // registers apart from the stages'), before the only stage otherwise
        const bool pf_first = p_.pf && p_.stages.size() < 2;
        if (pf_first) prefetch_next(name);
        if (p_.pad) o_ << "    const int tp = (int)(base & 1);\n";
        for (size_t si = 0; si < p_.stages.size(); ++si) {
            const TStage &st = p_.stages[si];
            const bool last = si + 1 == p_.stages.size();
            if (st.legacy) legacy(p_.ops[st.first]);
            else stage(st, si == 0 && p_.din, last && p_.dout);
            if (!(last && p_.dout)) o_ << "    __syncthreads();\n";
            if (si == 0 && p_.pf && !pf_first) prefetch_next(name);
        }
        if (p_.red) reduce_tile();
        if (!p_.dout) transfer(false, {{"tile", "A.psi"}});
        o_ << "    __syncthreads();\n  }\n  qj_wait0();\n";
        if (p_.red) reduce_finish();
        o_ << "}\n";
    }

    // Without a double buffer, the CTA's next tile is fetched into L2 while
    // this one is processed: every 128-byte line of each of its runs (the
    // run's last byte too, for runs that start inside a line), so its tile
    // copy or direct loads find the lines in L2 instead of waiting on HBM.
    void prefetch_next(const std::string &name) {
        const int NA = p_.T / p_.SEG;
        const long long RB = (long long)p_.SEG * (long long)elt();   // bytes of a run
        const long long LPR = (RB + 127) / 128 + 1;
        o_ << "    if (!db) { const long long tn = t + gridDim.x;\n      if (tn < " << p_.ntiles
           << ") { const long long bn = qj_tb_" << name << "(tn);\n";
        o_ << "        for (int k = tid; k < " << NA * LPR << "; k += " << p_.threads << ") { const int a = k / " << LPR
           << "; const long long l = (long long)(k - a * " << LPR << ") * 128; "
           << "const char *pl = reinterpret_cast<const char *>(A.psi + bn + offA[a]) + (l < " << RB << " ? l : " << RB - 1
           << "); asm volatile(\"prefetch.L2 [%0];\" :: \"l\"(pl)); }\n      }\n    }\n";
    }

    // <N_q> for every qudit and the norm of the finished tile (complex64),
    // when A.rows is set.  Blocks of DK consecutive tile elements (the K2
    // lowest local qudits, all in one run) give p = |psi|^2 sums in FP32 per
    // thread: the norm, the K2 low qudits' digit-weighted sums (literal
    // digits) and the other local qudits' sums (digit of the block); a warp's
    // sums are added across lanes (shuffles), and lane c of each warp adds
    // output c (and c + 32) of the tile to its FP64 accumulator: a local
    // qudit's sum, an outer qudit's digit (from the tile index) times the
    // norm, or the norm.
    void reduce_tile() {
        const int nt = p_.nt, rL = p_.T == p_.SEG ? nt : ipow_log(p_.SEG);
        const int K2 = std::min(rL, D_ == 2 ? 4 : D_ == 3 ? 3 : 2);
        const int DK = ipow_i(D_, K2), NB = p_.T / DK;
        o_ << "    if (A.rows) {\n      float qr_P = 0.f";
        for (int i = 0; i < nt; ++i) o_ << ", qr_S" << i << " = 0.f";
        o_ << ";\n";
        o_ << "      for (int blk = tid; blk < " << NB << "; blk += " << p_.threads << ") {\n";
        o_ << "        const int e0 = blk * " << DK << ";\n";
        if (p_.pad) {
            o_ << "        const int ra = e0 / " << p_.SEG << ";\n";
            o_ << "        const C *q = tile + e0 + ra + ((tp ^ ra) & 1);\n";
        } else {
            o_ << "        const C *q = tile + e0;\n";
        }
        o_ << "        float pb = 0.f";
        for (int k = 0; k < K2; ++k) o_ << ", pk" << k << " = 0.f";
        o_ << ";\n";
        for (int r = 0; r < DK; ++r) {
            o_ << "        { const C v = q[" << r << "]; const float pr = fmaf(v.x, v.x, v.y * v.y); pb += pr;";
            for (int k = 0; k < K2; ++k) {
                const int dig = (r / ipow_i(D_, K2 - 1 - k)) % D_;   // slot k = local position nt - K2 + k
                if (dig == 1) o_ << " pk" << k << " += pr;";
                else if (dig > 1) o_ << " pk" << k << " = fmaf(" << dig << ".f, pr, pk" << k << ");";
            }
            o_ << " }\n";
        }
        o_ << "        qr_P += pb;";
        for (int k = 0; k < K2; ++k) o_ << " qr_S" << (nt - K2 + k) << " += pk" << k << ";";
        o_ << "\n";
        for (int i = 0; i < nt - K2; ++i) {
            const int div = ipow_i(D_, nt - 1 - i) / DK;   // local stride / DK
            o_ << "        qr_S" << i << " = fmaf((float)((blk / " << div << ") % " << D_ << "), pb, qr_S" << i << ");\n";
        }
        o_ << "      }\n";
        // warp sums
        o_ << "      for (int o = 16; o > 0; o >>= 1) { qr_P += __shfl_xor_sync(0xffffffffu, qr_P, o);";
        for (int i = 0; i < nt; ++i) o_ << " qr_S" << i << " += __shfl_xor_sync(0xffffffffu, qr_S" << i << ", o);";
        o_ << " }\n";
        // each lane adds its outputs c = lane, lane + 32: a local qudit's sum
        // (selected by literal compares), an outer qudit's digit of the tile
        // index (the lane's divisor, set once per kernel) times the norm, or
        // the norm -- formed in FP32, one conversion to FP64 per output
        o_ << "      const unsigned tt = (unsigned)t;\n";
        for (int half = 0; half < 2; ++half) {
            if (half == 1 && p_.n + 1 <= 32) break;
            const std::string acc = half ? "qr_acc1" : "qr_acc0";
            const std::string dv = half ? "qr_div1" : "qr_div0";
            const int off = half * 32;
            o_ << "      { float ad = 0.f; const int c = (tid & 31) + " << off << ";\n";
            for (int i = 0; i < nt; ++i) o_ << "        if (c == " << p_.local_q[i] << ") ad = qr_S" << i << ";\n";
            o_ << "        if (" << dv << ") ad = qr_P * (float)((tt / " << dv << ") % " << D_ << "u);\n";
            o_ << "        if (c == " << p_.n << ") ad = qr_P;\n";
            o_ << "        " << acc << " += (double)ad; }\n";
        }
        o_ << "    }\n";
    }

    // Once per kernel: the tile-index divisor of each lane's outer-qudit
    // outputs (0 for local qudits and the norm).
    void reduce_roles() {
        for (int half = 0; half < 2; ++half) {
            const std::string dv = half ? "qr_div1" : "qr_div0";
            o_ << "  unsigned " << dv << " = 0u;\n";
            if (half == 1 && p_.n + 1 <= 32) continue;
            o_ << "  { const int c = (threadIdx.x & 31) + " << half * 32 << ";";
            for (const auto &od : p_.outer_div) o_ << " if (c == " << od.first << ") " << dv << " = " << od.second << "u;";
            o_ << " }\n";
        }
    }

    // Per-CTA rows: the warps' accumulators summed in warp order.
    void reduce_finish() {
        const int W = p_.threads / 32, C1 = p_.n + 1;
        o_ << "  if (A.rows) {\n    double *qr_w = reinterpret_cast<double *>(qj_sm);\n    __syncthreads();\n";
        o_ << "    if ((tid & 31) < " << std::min(C1, 32) << ") qr_w[(tid >> 5) * 64 + (tid & 31)] = qr_acc0;\n";
        if (C1 > 32) o_ << "    if ((tid & 31) + 32 < " << C1 << ") qr_w[(tid >> 5) * 64 + 32 + (tid & 31)] = qr_acc1;\n";
        o_ << "    __syncthreads();\n";
        o_ << "    for (int c = tid; c < " << C1 << "; c += " << p_.threads << ") { double s = 0.0; for (int w = 0; w < "
           << W << "; ++w) s += qr_w[w * 64 + c]; A.rows[(long long)blockIdx.x * " << C1 << " + c] = s; }\n  }\n";
    }

    int ipow_log(int x) const {
        int e = 0;
        for (int v = 1; v < x; v *= D_) ++e;
        return e;
    }

    // Padded layout: run a of the tile fills the 16-byte aligned window of
    // SEG + 1 amplitudes that starts at (base + offA[a]) rounded down to an
    // even index, i.e. chunk k = a * CH + c of CH = (SEG + 1) / 2 amplitude
    // pairs lands at slot 2k.  The chunk holding only the run's first (odd
    // start) or last (even start) amplitude moves that amplitude alone, so
    // nothing outside the run is read or written.
    void transfer_pad(bool load) {
        const int NA = p_.T / p_.SEG, CH = (p_.SEG + 1) / 2;
        auto body = [&](const std::string &a, const std::string &c, const std::string &k) {
            o_ << "const long long rs = base + offA[" << a << "]; const int sh = (int)(rs & 1); "
               << "const long long g = rs - sh + 2 * " << c << "; C *dst = tile + 2 * (" << k << "); ";
            if (load)
                o_ << "if (" << c << " == 0 && sh) qj_cp(dst + 1, A.psi + g + 1); else if (" << c << " == " << CH - 1
                   << " && !sh) qj_cp(dst, A.psi + g); else qj_cp2(dst, A.psi + g); ";
            else
                o_ << "if (" << c << " == 0 && sh) A.psi[g + 1] = dst[1]; else if (" << c << " == " << CH - 1
                   << " && !sh) A.psi[g] = dst[0]; else qj_st2(A.psi + g, dst); ";
        };
        if (lanes()) {
            const int R = p_.threads / CH;
            o_ << "    if (qj_tr < " << R << ") for (int a = qj_tr; a < " << NA << "; a += " << R << ") { ";
            body("a", "qj_tu", "a * " + std::to_string(CH) + " + qj_tu");
            o_ << "}\n";
        } else if (CH >= 64) {
            o_ << "    for (int a = 0; a < " << NA << "; ++a) {\n      for (int c = tid; c < " << CH << "; c += "
               << p_.threads << ") { ";
            body("a", "c", "a * " + std::to_string(CH) + " + c");
            o_ << "}\n    }\n";
        } else {
            o_ << "    for (int k = tid; k < " << NA * CH << "; k += " << p_.threads << ") { const int a = k / " << CH
               << "; const int c = k - a * " << CH << "; ";
            body("a", "c", "k");
            o_ << "}\n";
        }
    }

    // offA[a] = offset of run a: digits of a on the active qudits (literal strides).
    void emit_offA(int NA) {
        o_ << "  for (int a = tid; a < " << NA << "; a += " << p_.threads << ") {\n    long long o = 0; int rem = a;\n";
        for (int i = p_.kA - 1; i >= 0; --i)
            o_ << "    o += (long long)(rem % " << D_ << ") * " << p_.strideA[i] << "LL; rem /= " << D_ << ";\n";
        o_ << "    offA[a] = o;\n  }\n";
    }

    // Base offset of tile t: the outer qudits' digits, runs from the least
    // significant (literal radices and strides).
    void tile_base_lit(const std::string &name) {
        const bool narrow = p_.ntiles < (1ll << 32);
        o_ << "__device__ __forceinline__ long long qj_tb_" << name << "(long long tl) {\n  long long base = 0;\n";
        if (narrow) o_ << "  unsigned t = (unsigned)tl;\n";
        else o_ << "  unsigned long long t = (unsigned long long)tl;\n";
        for (int r = 0; r < p_.nruns; ++r) {
            const std::string M = std::to_string(p_.runM[r]) + (narrow ? "u" : "ull");
            o_ << "  { const auto q = t / " << M << "; base += (long long)(t - q * " << M << ") * " << p_.runS[r]
               << "LL; t = q; }\n";
        }
        o_ << "  return base;\n}\n";
    }

    // Reverse pass of the adjoint sweep: psi and lambda tiles; every op is
    // U^+ (entries at op.mat); a parametrised op first adds Im <lambda|G|psi>
    // of the block (generator entries at op.gmat) to its column; each CTA
    // writes one row of 2 x column sums.
    void kernel_adj(const std::string &name) {
        const int NG = std::max(1, 2 * p_.nruns + p_.kA);
        const int NP = std::max(1, p_.params ? p_.npool : 1);
        const int NA = p_.T / p_.SEG;
        const int WARPS = p_.threads / 32;
        const int NC = p_.ncols;
        o_ << "struct __align__(16) A_" << name << " { C *psi; C *lam; const P *gp; double *rows; long long ntiles; "
           << "long long geo[" << NG << "]; P pool[" << NP << "]; };\n";
        o_ << "extern \"C\" __global__ void __launch_bounds__(" << p_.threads << ") " << name
           << "(const __grid_constant__ A_" << name << " A) {\n";
        o_ << "  extern __shared__ __align__(16) unsigned char qj_sm[];\n";
        o_ << "  __shared__ double qj_red[" << std::max(1, NC * WARPS) << "];\n";
        o_ << "  C *tile = reinterpret_cast<C *>(qj_sm);\n";
        o_ << "  C *ltile = tile + " << p_.T << ";\n";
        o_ << "  long long *offA = reinterpret_cast<long long *>(qj_sm + " << (size_t)2 * p_.T * elt() << ");\n";
        o_ << "  const int tid = threadIdx.x;\n";
        emit_lanes();
        for (int c = 0; c < NC; ++c) o_ << "  double g" << c << " = 0.0;\n";
        o_ << "  for (int a = tid; a < " << NA << "; a += " << p_.threads << ") {\n    long long o = 0; int rem = a;\n";
        for (int i = p_.kA - 1; i >= 0; --i)
            o_ << "    o += (long long)(rem % " << D_ << ") * A.geo[" << 2 * p_.nruns + i << "]; rem /= " << D_ << ";\n";
        o_ << "    offA[a] = o;\n  }\n";
        o_ << "  __syncthreads();\n";
        o_ << "  // register stages: " << p_.stages.size() << (p_.din ? ", first from HBM" : "")
           << (p_.dout ? ", last to HBM" : "") << "\n";
        o_ << "  for (long long t = blockIdx.x; t < " << p_.ntiles << "; t += gridDim.x) {\n";
        o_ << "    const long long base = qj_tb_" << name << "(t);\n";
        if (!p_.din) {
            transfer(true, {{"tile", "A.psi"}, {"ltile", "A.lam"}});
            o_ << "    qj_wait();\n    __syncthreads();\n";
        }
        for (size_t si = 0; si < p_.stages.size(); ++si) {
            const TStage &st = p_.stages[si];
            const bool last = si + 1 == p_.stages.size();
            if (st.legacy) {
                tn_ = "tile";
                legacy(p_.ops[st.first]);
                tn_ = "ltile";
                legacy(p_.ops[st.first]);
                tn_ = "tile";
            } else {
                stage_adj(st, si == 0 && p_.din, last && p_.dout);
            }
            if (!(last && p_.dout)) o_ << "    __syncthreads();\n";
        }
        if (!p_.dout) transfer(false, {{"tile", "A.psi"}, {"ltile", "A.lam"}});
        o_ << "    __syncthreads();\n  }\n";
        if (NC > 0) {
            o_ << "  const int lane = tid & 31, wid = tid >> 5;\n";
            for (int c = 0; c < NC; ++c)
                o_ << "  { double x = g" << c << "; for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);"
                   << " if (lane == 0) qj_red[" << c * WARPS << " + wid] = x; }\n";
            o_ << "  __syncthreads();\n";
            o_ << "  for (int c = tid; c < " << NC << "; c += " << p_.threads << ") { double s = 0.0; for (int w = 0; w < "
               << WARPS << "; ++w) s += qj_red[c * " << WARPS << " + w]; A.rows[(long long)blockIdx.x * " << NC
               << " + c] = 2.0 * s; }\n";
        }
        o_ << "}\n";
    }

    // Tile load (cp.async) or store between shared memory and the d^kA runs
    // of SEG amplitudes at base + offA[a].  Complex64 at even d moves
    // amplitude pairs (every run start is even, so 16-byte aligned); runs of
    // at least 64 transfers are walked run by run without index division.
    void transfer(bool load, const std::vector<std::pair<std::string, std::string>> &bufs) {
        if (p_.pad) {
            transfer_pad(load);
            return;
        }
        const int pf = (!p_.c128 && D_ % 2 == 0 && p_.SEG % 2 == 0) ? 2 : 1;
        const int per_run = p_.SEG / pf, NA = p_.T / p_.SEG;
        auto one = [&](const std::string &sm, const std::string &g, const std::string &e, const std::string &gi) {
            if (load) o_ << (pf == 2 ? "qj_cp2(" : "qj_cp(") << sm << " + " << e << ", " << g << " + " << gi << "); ";
            else if (pf == 2) o_ << "qj_st2(" << g << " + " << gi << ", " << sm << " + " << e << "); ";
            else o_ << g << "[" << gi << "] = " << sm << "[" << e << "]; ";
        };
        if (lanes()) {
            const int R = p_.threads / per_run;
            o_ << "    if (qj_tr < " << R << ") for (int a = qj_tr; a < " << NA << "; a += " << R
               << ") { const long long ro = base + offA[a]; const int l = qj_tu * " << pf << "; ";
            for (auto &b : bufs) one(b.first, b.second, "a * " + std::to_string(p_.SEG) + " + l", "ro + l");
            o_ << "}\n";
        } else if (per_run >= 64) {
            o_ << "    for (int a = 0; a < " << NA << "; ++a) { const long long ro = base + offA[a];\n";
            o_ << "      for (int l = tid * " << pf << "; l < " << p_.SEG << "; l += " << p_.threads * pf << ") { ";
            for (auto &b : bufs) one(b.first, b.second, "a * " + std::to_string(p_.SEG) + " + l", "ro + l");
            o_ << "}\n    }\n";
        } else {
            o_ << "    for (int e = tid * " << pf << "; e < " << p_.T << "; e += " << p_.threads * pf
               << ") { const int a = e / " << p_.SEG << "; const long long gi = base + offA[a] + (e - a * " << p_.SEG
               << "); ";
            for (auto &b : bufs) one(b.first, b.second, "e", "gi");
            o_ << "}\n";
        }
    }


    size_t elt() const { return p_.c128 ? 16 : 8; }

    // Copy units of one run: amplitude pairs (complex64, even d), padded
    // pairs, or amplitudes.
    int run_units() const {
        if (p_.pad) return (p_.SEG + 1) / 2;
        const int pf = (!p_.c128 && D_ % 2 == 0 && p_.SEG % 2 == 0) ? 2 : 1;
        return p_.SEG / pf;
    }

    // At odd d, runs of at most 32 units move with a fixed lane layout:
    // thread tid copies unit qj_tu of runs qj_tr, qj_tr + R, ... (R =
    // threads / units), so no index is divided per element and a run's offset
    // is read once (measured on GB300: d=5 passes 4 % faster; at even d the
    // division is a shift and the layout lost 5 % at d=2).
    bool lanes() const { return D_ % 2 == 1 && run_units() <= 32; }
    void emit_lanes() {
        const int U = run_units();
        if (lanes()) o_ << "  const int qj_tr = tid / " << U << ", qj_tu = tid - qj_tr * " << U << ";\n";
    }

  private:
    const PassSrc &p_;
    std::ostringstream &o_;
    int D_;

    std::string vp_ = "v";       // register block the ops write (v: psi, w: lambda)
    std::string tn_ = "tile";    // shared-memory tile of legacy ops

    std::string E(int k) const { return (p_.params ? "A.pool[" : "A.gp[") + std::to_string(k) + "]"; }
    std::string Edyn(const std::string &expr) const { return (p_.params ? "A.pool[" : "A.gp[") + expr + "]"; }
    std::string V(int r) const { return vp_ + std::to_string(r); }
    static std::string W(int r) { return "w" + std::to_string(r); }
    static std::string Pv(int r) { return "v" + std::to_string(r); }

    // ---------------------------------------------------------------- register stage
    // din / dout: the block's registers come from / go to HBM (every slot of
    // the stage is an active qudit, so register r sits Da_r runs further:
    // global offset G_r from the active strides, same position in the run).
    void stage(const TStage &st, bool din = false, bool dout = false) {
        const int K = p_.K, DK = ipow_i(D_, K), NBLK = p_.T / DK;
        o_ << "    for (int blk = tid; blk < " << NBLK << "; blk += " << p_.threads << ") {\n      int b = blk;\n";
        for (int i = 0; i < K; ++i)
            o_ << "      { const int q = b / " << st.lsa[i] << "; b = q * " << st.lsa[i] * D_ << " + (b - q * "
               << st.lsa[i] << "); }\n";
        std::vector<int> off(DK);
        for (int r = 0; r < DK; ++r) {
            int o = 0;
            for (int i = 0; i < K; ++i) o += ((r / ipow_i(D_, K - 1 - i)) % D_) * st.ls[i];
            off[r] = o;
        }
        std::vector<std::string> at(DK);
        if (p_.pad) {
            // b = a_b * SEG + l_b; register r sits Da runs and Dl amplitudes
            // further (off[r] = Da * SEG + Dl, the stage's digits are zero in
            // b), at slot (a_b + Da) * (SEG + 1) + l_b + Dl + shift, and the
            // shift of run a_b + Da is the block's shift flipped when Da is odd
            const int SEG = p_.SEG;
            o_ << "      const int ab = b / " << SEG << "; const int sb = (tp ^ ab) & 1;\n";
            o_ << "      C *P0 = tile + b + ab + sb; C *P1 = tile + b + ab + 1 - sb;\n";
            for (int r = 0; r < DK; ++r) {
                const int da = off[r] / SEG, dl = off[r] % SEG;
                at[r] = std::string(da & 1 ? "P1[" : "P0[") + std::to_string(da * (SEG + 1) + dl) + "]";
            }
        } else {
            for (int r = 0; r < DK; ++r) at[r] = "tile[b + " + std::to_string(off[r]) + "]";
        }
        std::vector<std::string> gat(DK);
        if (din || dout) {
            const int SEG = p_.SEG;
            o_ << "      const int gab = b / " << SEG << ";\n";
            o_ << "      C *gq = A.psi + (base + offA[gab] + (b - gab * " << SEG << "));\n";
            for (int r = 0; r < DK; ++r) gat[r] = "gq[" + std::to_string(global_offset(off[r])) + "LL]";
        }
        for (int r = 0; r < DK; ++r) o_ << "      C " << V(r) << " = " << (din ? gat[r] : at[r]) << ";\n";
        for (int i = 0; i < st.nops; ++i) op(p_.ops[st.first + i]);
        for (int r = 0; r < DK; ++r) o_ << "      " << (dout ? gat[r] : at[r]) << " = " << V(r) << ";\n";
        o_ << "    }\n";
    }

    // Shared-memory element of standard tile index e (legacy ops).
    std::string sx(const std::string &e) const {
        if (!p_.pad) return e;
        const std::string S = std::to_string(p_.SEG);
        return "(" + e + " + " + e + " / " + S + " + ((tp ^ (" + e + " / " + S + ")) & 1))";
    }

    void stage_adj(const TStage &st, bool din = false, bool dout = false) {
        const int K = p_.K, DK = ipow_i(D_, K), NBLK = p_.T / DK;
        o_ << "    for (int blk = tid; blk < " << NBLK << "; blk += " << p_.threads << ") {\n      int b = blk;\n";
        for (int i = 0; i < K; ++i)
            o_ << "      { const int q = b / " << st.lsa[i] << "; b = q * " << st.lsa[i] * D_ << " + (b - q * "
               << st.lsa[i] << "); }\n";
        std::vector<int> off(DK);
        for (int r = 0; r < DK; ++r) {
            int o = 0;
            for (int i = 0; i < K; ++i) o += ((r / ipow_i(D_, K - 1 - i)) % D_) * st.ls[i];
            off[r] = o;
        }
        std::vector<std::string> G(DK);
        if (din || dout) {
            const int SEG = p_.SEG;
            o_ << "      const int gab = b / " << SEG << ";\n";
            o_ << "      const long long go = base + offA[gab] + (b - gab * " << SEG << ");\n";
            o_ << "      C *gq = A.psi + go; C *gl = A.lam + go;\n";
            for (int r = 0; r < DK; ++r) G[r] = std::to_string(global_offset(off[r])) + "LL";
        }
        for (int r = 0; r < DK; ++r) {
            if (din)
                o_ << "      C " << Pv(r) << " = gq[" << G[r] << "]; C " << W(r) << " = gl[" << G[r] << "];\n";
            else
                o_ << "      C " << Pv(r) << " = tile[b + " << off[r] << "]; C " << W(r) << " = ltile[b + " << off[r]
                   << "];\n";
        }
        for (int i = 0; i < st.nops; ++i) {
            const TOp &o = p_.ops[st.first + i];
            if (o.gcol >= 0) grad(o);
            vp_ = "v";
            op(o);
            vp_ = "w";
            op(o);
            vp_ = "v";
        }
        for (int r = 0; r < DK; ++r) {
            if (dout)
                o_ << "      gq[" << G[r] << "] = " << Pv(r) << "; gl[" << G[r] << "] = " << W(r) << ";\n";
            else
                o_ << "      tile[b + " << off[r] << "] = " << Pv(r) << "; ltile[b + " << off[r] << "] = " << W(r)
                   << ";\n";
        }
        o_ << "    }\n";
    }

    // Global offset of a register whose tile offset (a multiple of SEG: the
    // stage's slots are active qudits) is off: its run-number digits times
    // the active strides, digit 0 first as the offA table composes them.
    long long global_offset(int off) const {
        long long G = 0;
        int da = off / p_.SEG;
        for (int pos = 0; pos < p_.kA; ++pos, da /= D_) G += (long long)(da % D_) * p_.strideA[p_.kA - 1 - pos];
        return G;
    }

    // Im(conj(lambda) * x) for register names.
    static std::string imc(const std::string &l, const std::string &x) {
        return "(" + l + ".x * " + x + ".y - " + l + ".y * " + x + ".x)";
    }

    // Adds the block's Im <lambda|G|psi> of a parametrised op to g<gcol>.
    // Double-float form of grad(): the block's terms summed as double-float
    // reals (qim / qad / qmu), added to the FP64 column once per op and block.
    void grad_df(const TOp &o) {
        const int sa = o.q[4], sc = o.q[5];
        const int gm = o.gmat;
        const bool ctrl = is_controlled(o);
        const std::string gv = "g" + std::to_string(o.gcol);
        auto scaled = [&](const std::string &x, int cl) {
            return cl == 1 ? x : "qmu(" + x + ", " + std::to_string(cl) + ".f, 0.f)";
        };
        if (o.kind == OP_PAIR || o.kind == OP_CPAIR) {
            const int RS = rs(sa);
            auto fib = [&](int b0, int cl) {
                const std::string a = Pv(b0 + o.j * RS), c = Pv(b0 + o.k * RS);
                const std::string la = W(b0 + o.j * RS), lc = W(b0 + o.k * RS);
                o_ << "      { const C ga = jma(" << E(gm + 1) << ", " << c << ", jm(" << E(gm) << ", " << a
                   << ")); const C gc = jma(" << E(gm + 3) << ", " << c << ", jm(" << E(gm + 2) << ", " << a << ")); "
                   << "qt = qad(qt, " << scaled("qad(qim(" + la + ", ga), qim(" + lc + ", gc))", cl) << "); }\n";
            };
            if (ctrl && sc < 0) {
                o_ << "      { const int cl = " << outside_digit(o.lsc) << "; if (cl) { float2 qt = qf2(0.f, 0.f);\n";
                for (int b0 : fibres(sa)) fib(b0, 1);
                o_ << "      " << gv << " += qdd(qmu(qt, (float)cl, 0.f)); } }\n";
                return;
            }
            o_ << "      { float2 qt = qf2(0.f, 0.f);\n";
            for (int b0 : fibres(sa)) {
                const int cl = ctrl ? slot_digit(b0, sc) : 1;
                if (cl == 0) continue;
                fib(b0, cl);
            }
            o_ << "      " << gv << " += qdd(qt); }\n";
            return;
        }
        if (o.kind == OP_DIAG || o.kind == OP_CDIAG) {
            if (sa < 0) {
                const int DK = ipow_i(D_, p_.K);
                o_ << "      { const int dg = " << outside_digit(o.lsa) << "; if ((" << o.mask
                   << " >> dg) & 1) { float2 qt = qf2(0.f, 0.f);";
                for (int r = 0; r < DK; ++r) o_ << " qt = qad(qt, qim(" << W(r) << ", " << Pv(r) << "));";
                o_ << " const P ge = " << Edyn(std::to_string(gm) + " + dg") << "; " << gv
                   << " += qdd(qmu(qt, ge.h.x, ge.l.x)); } }\n";
                return;
            }
            const int RS = rs(sa);
            auto fib = [&](int b0) {
                for (int l = 0; l < D_; ++l)
                    if ((o.mask >> l) & 1)
                        o_ << "      qt = qad(qt, qmu(qim(" << W(b0 + l * RS) << ", " << Pv(b0 + l * RS) << "), " << E(gm + l)
                           << ".h.x, " << E(gm + l) << ".l.x));\n";
            };
            if (ctrl && sc < 0) {
                o_ << "      { const int cl = " << outside_digit(o.lsc) << "; if (cl) { float2 qt = qf2(0.f, 0.f);\n";
                for (int b0 : fibres(sa)) fib(b0);
                o_ << "      " << gv << " += qdd(qmu(qt, (float)cl, 0.f)); } }\n";
                return;
            }
            o_ << "      { float2 qt = qf2(0.f, 0.f);\n";
            for (int b0 : fibres(sa)) {
                const int cl = ctrl ? slot_digit(b0, sc) : 1;
                if (cl == 0) continue;
                if (cl == 1) {
                    fib(b0);
                } else {
                    o_ << "      { float2 qs = qt; qt = qf2(0.f, 0.f);\n";
                    fib(b0);
                    o_ << "      qt = qad(qs, qmu(qt, " << cl << ".f, 0.f)); }\n";
                }
            }
            o_ << "      " << gv << " += qdd(qt); }\n";
        }
    }

    void grad(const TOp &o) {
        if (p_.df) {
            grad_df(o);
            return;
        }
        const int sa = o.q[4], sc = o.q[5];
        const int gm = o.gmat;
        const bool ctrl = is_controlled(o);
        const std::string gv = "g" + std::to_string(o.gcol);
        if (o.kind == OP_PAIR || o.kind == OP_CPAIR) {
            const int RS = rs(sa);
            auto fib = [&](int b0, const std::string &scale) {
                const std::string a = Pv(b0 + o.j * RS), c = Pv(b0 + o.k * RS);
                const std::string la = W(b0 + o.j * RS), lc = W(b0 + o.k * RS);
                o_ << "      { const C ga = jma(" << E(gm + 1) << ", " << c << ", jm(" << E(gm) << ", " << a
                   << ")); const C gc = jma(" << E(gm + 3) << ", " << c << ", jm(" << E(gm + 2) << ", " << a << ")); "
                   << "qt += " << scale << "(" << imc(la, "ga") << " + " << imc(lc, "gc") << "); }\n";
            };
            if (ctrl && sc < 0) {
                o_ << "      { const int cl = " << outside_digit(o.lsc) << "; if (cl) { decltype(C().x) qt = 0;\n";
                for (int b0 : fibres(sa)) fib(b0, "");
                o_ << "      " << gv << " += (double)qt * cl; } }\n";
                return;
            }
            o_ << "      { decltype(C().x) qt = 0;\n";
            for (int b0 : fibres(sa)) {
                if (ctrl) {
                    const int cl = slot_digit(b0, sc);
                    if (cl == 0) continue;
                    fib(b0, std::to_string(cl) + " * ");
                } else {
                    fib(b0, "");
                }
            }
            o_ << "      " << gv << " += (double)qt; }\n";
            return;
        }
        if (o.kind == OP_DIAG || o.kind == OP_CDIAG) {
            if (sa < 0) {
                const int DK = ipow_i(D_, p_.K);
                o_ << "      { const int dg = " << outside_digit(o.lsa) << "; if ((" << o.mask
                   << " >> dg) & 1) { decltype(C().x) qt = 0;";
                for (int r = 0; r < DK; ++r) o_ << " qt += " << imc(W(r), Pv(r)) << ";";
                o_ << " " << gv << " += (double)(" << Edyn(std::to_string(gm) + " + dg") << ".x * qt); } }\n";
                return;
            }
            const int RS = rs(sa);
            auto fib = [&](int b0, const std::string &scale) {
                o_ << "      qt += " << scale << "(";
                bool first = true;
                for (int l = 0; l < D_; ++l)
                    if ((o.mask >> l) & 1) {
                        o_ << (first ? "" : " + ") << E(gm + l) << ".x * " << imc(W(b0 + l * RS), Pv(b0 + l * RS));
                        first = false;
                    }
                if (first) o_ << "0";
                o_ << ");\n";
            };
            if (ctrl && sc < 0) {
                o_ << "      { const int cl = " << outside_digit(o.lsc) << "; if (cl) { decltype(C().x) qt = 0;\n";
                for (int b0 : fibres(sa)) fib(b0, "");
                o_ << "      " << gv << " += (double)qt * cl; } }\n";
                return;
            }
            o_ << "      { decltype(C().x) qt = 0;\n";
            for (int b0 : fibres(sa)) {
                if (ctrl) {
                    const int cl = slot_digit(b0, sc);
                    if (cl == 0) continue;
                    fib(b0, std::to_string(cl) + " * ");
                } else {
                    fib(b0, "");
                }
            }
            o_ << "      " << gv << " += (double)qt; }\n";
        }
    }

    int rs(int S) const { return ipow_i(D_, p_.K - 1 - S); }
    std::vector<int> fibres(int S) const {
        const int RS = rs(S), DK = ipow_i(D_, p_.K);
        std::vector<int> b;
        for (int f = 0; f < DK / D_; ++f) b.push_back((f / RS) * RS * D_ + f % RS);
        return b;
    }
    int slot_digit(int r, int slot) const { return (r / ipow_i(D_, p_.K - 1 - slot)) % D_; }

    void pair_fibre(int b0, int RS, int J, int L, const std::string &e0, const std::string &e1, const std::string &e2,
                    const std::string &e3, bool real) {
        const std::string a = V(b0 + J * RS), c = V(b0 + L * RS);
        o_ << "      { const C qa = " << a << ", qc = " << c << ";\n";
        if (real) {
            o_ << "        " << a << " = jn(jrma(" << e1 << ", qc, jrm(" << e0 << ", qa)));\n";
            o_ << "        " << c << " = jn(jrma(" << e3 << ", qc, jrm(" << e2 << ", qa))); }\n";
        } else {
            o_ << "        " << a << " = jn(jma(" << e1 << ", qc, jm(" << e0 << ", qa)));\n";
            o_ << "        " << c << " = jn(jma(" << e3 << ", qc, jm(" << e2 << ", qa))); }\n";
        }
    }

    void shift_fibre(int b0, int RS, int sh) {
        if (sh == 0) return;
        o_ << "      {";
        for (int m = 0; m < D_; ++m) o_ << " const C t" << m << " = " << V(b0 + m * RS) << ";";
        for (int m = 0; m < D_; ++m) o_ << " " << V(b0 + ((m + sh) % D_) * RS) << " = t" << m << ";";
        o_ << " }\n";
    }

    std::string outside_digit(int ls) const {
        return "((b / " + std::to_string(ls) + ") % " + std::to_string(D_) + ")";
    }

    void op(const TOp &o) {
        const int sa = o.q[4], sc = o.q[5];
        const int m = o.mat;
        const bool ctrl = is_controlled(o);
        switch (o.kind) {
        case OP_DENSE: {
            const int RS = rs(sa);
            for (int b0 : fibres(sa)) {
                o_ << "      {";
                for (int x = 0; x < D_; ++x) o_ << " const C x" << x << " = " << V(b0 + x * RS) << ";";
                o_ << "\n";
                for (int l = 0; l < D_; ++l) {
                    std::string acc = "jm(" + E(m + l * D_) + ", x0)";
                    for (int x = 1; x < D_; ++x) acc = "jma(" + E(m + l * D_ + x) + ", x" + std::to_string(x) + ", " + acc + ")";
                    o_ << "        " << V(b0 + l * RS) << " = jn(" << acc << ");\n";
                }
                o_ << "      }\n";
            }
            break;
        }
        case OP_PAIR:
        case OP_CPAIR: {
            const int RS = rs(sa);
            const bool real = o.s == 1;
            if (ctrl && sc < 0) {
                o_ << "      { const int cl = " << outside_digit(o.lsc) << "; if (cl) { const int mb = " << m
                   << " + 4 * cl;\n";
                for (int b0 : fibres(sa))
                    pair_fibre(b0, RS, o.j, o.k, Edyn("mb"), Edyn("mb + 1"), Edyn("mb + 2"), Edyn("mb + 3"), real);
                o_ << "      } }\n";
                break;
            }
            for (int b0 : fibres(sa)) {
                int mb = m;
                if (ctrl) {
                    const int cl = slot_digit(b0, sc);
                    if (cl == 0) continue;
                    mb = m + 4 * cl;
                }
                pair_fibre(b0, RS, o.j, o.k, E(mb), E(mb + 1), E(mb + 2), E(mb + 3), real);
            }
            break;
        }
        case OP_DIAG:
        case OP_CDIAG: {
            if (sa < 0) {   // target outside the stage: one phase for the block
                o_ << "      { const int dg = " << outside_digit(o.lsa) << "; if ((" << o.mask
                   << " >> dg) & 1) { const P ph = " << Edyn(std::to_string(m) + " + dg") << ";";
                const int DK = ipow_i(D_, p_.K);
                for (int r = 0; r < DK; ++r) o_ << " " << V(r) << " = jn(jm(ph, " << V(r) << "));";
                o_ << " } }\n";
                break;
            }
            const int RS = rs(sa);
            if (ctrl && sc < 0) {
                o_ << "      { const int cl = " << outside_digit(o.lsc) << "; if (cl) { const int mb = " << m << " + "
                   << D_ << " * cl;";
                for (int b0 : fibres(sa))
                    for (int l = 0; l < D_; ++l)
                        if ((o.mask >> l) & 1)
                            o_ << " " << V(b0 + l * RS) << " = jn(jm(" << Edyn("mb + " + std::to_string(l)) << ", "
                               << V(b0 + l * RS) << "));";
                o_ << " } }\n";
                break;
            }
            for (int b0 : fibres(sa)) {
                int mb = m;
                if (ctrl) {
                    const int cl = slot_digit(b0, sc);
                    if (cl == 0) continue;
                    mb = m + D_ * cl;
                }
                o_ << "     ";
                for (int l = 0; l < D_; ++l)
                    if ((o.mask >> l) & 1)
                        o_ << " " << V(b0 + l * RS) << " = jn(jm(" << E(mb + l) << ", " << V(b0 + l * RS) << "));";
                o_ << "\n";
            }
            break;
        }
        case OP_SHIFT:
        case OP_CSHIFT: {
            const int RS = rs(sa);
            if (ctrl && sc < 0) {
                o_ << "      { const int sh = (" << o.s << " * " << outside_digit(o.lsc) << ") % " << D_ << ";\n";
                for (int sh = 1; sh < D_; ++sh) {
                    o_ << "      if (sh == " << sh << ") {\n";
                    for (int b0 : fibres(sa)) shift_fibre(b0, RS, sh);
                    o_ << "      }\n";
                }
                o_ << "      }\n";
                break;
            }
            for (int b0 : fibres(sa)) {
                const int sh = ctrl ? (o.s * slot_digit(b0, sc)) % D_ : o.s % D_;
                shift_fibre(b0, RS, sh);
            }
            break;
        }
        default:
            break;
        }
    }

    // ---------------------------------------------------------------- shared-memory ops
    void legacy(const TOp &o) {
        if (o.kind == OP_SWAP) {
            const int la = o.lsa, lc = o.lsc;
            o_ << "    for (int e = tid; e < " << p_.T << "; e += " << p_.threads << ") {\n";
            o_ << "      const int x = (e / " << la << ") % " << D_ << ", y = (e / " << lc << ") % " << D_ << ";\n";
            o_ << "      if (x < y) { const int e2 = e + (y - x) * " << (la - lc) << "; const C t0 = " << tn_ << "["
               << sx("e") << "]; " << tn_ << "[" << sx("e") << "] = " << tn_ << "[" << sx("e2") << "]; " << tn_ << "["
               << sx("e2") << "] = t0; }\n    }\n";
            return;
        }
        // OP_DENSEK: entries always in global memory (up to 64 x 64)
        const int K = o.nq;
        std::vector<int> ls(K);
        int DK = 1;
        for (int i = 0; i < K; ++i) {
            ls[i] = ipow_i(D_, p_.nt - 1 - o.q[i]);
            DK *= D_;
        }
        std::vector<int> asc = ls;
        std::sort(asc.begin(), asc.end());
        o_ << "    for (int g = tid; g < " << p_.T / DK << "; g += " << p_.threads << ") {\n      int b = g;\n";
        for (int s : asc) o_ << "      { const int q = b / " << s << "; b = q * " << s * D_ << " + (b - q * " << s << "); }\n";
        o_ << "      const int offs[" << DK << "] = {";
        for (int r = 0; r < DK; ++r) {
            int off = 0, rr = r;
            for (int i = K - 1; i >= 0; --i) { off += (rr % D_) * ls[i]; rr /= D_; }
            o_ << (r ? ", " : "") << off;
        }
        o_ << "};\n      C xs[" << DK << "];\n";
        o_ << "      for (int r = 0; r < " << DK << "; ++r) xs[r] = " << tn_ << "[" << sx("(b + offs[r])") << "];\n";
        o_ << "      for (int r = 0; r < " << DK << "; ++r) { C acc = jm(A.gp[" << o.mat << " + r * " << DK
           << "], xs[0]); for (int x = 1; x < " << DK << "; ++x) acc = jma(A.gp[" << o.mat << " + r * " << DK
           << " + x], xs[x], acc); " << tn_ << "[" << sx("(b + offs[r])") << "] = jn(acc); }\n    }\n";
    }
};

std::string cuda_err(CUresult r) { return "CUresult " + std::to_string((int)r); }

}  // namespace

// Register slots of a generated register stage.
// Register slots of a generated reverse (adjoint) stage: psi and lambda
// blocks both live in registers.
int jit_stage_k_adj(int d, bool c128) {
    if (c128) return d == 2 ? 2 : 1;
    return d == 2 ? 3 : d <= 4 ? 2 : 1;
}

// Double-float complex128 passes at d = 4 take one slot: their 16-amplitude
// two-slot blocks need 170-240 registers, and one slot measured 19 % faster
// on the 200-gate d=4 n=14 program (61.5 vs 75.7 ms on GB300).
int jit_stage_k(int d, bool c128, bool df = false) {
    if (c128 && df && d == 4) return 1;
    if (c128) return d == 2 ? 3 : (d == 3 || d == 4) ? 2 : 1;
    return d == 2 ? 5 : d <= 5 ? 2 : 1;
}

struct JitPassInfo {
    size_t smem2 = 0;       // forward passes: shared memory with a double buffer (0: not offered)
    bool dbuf = false;      // forward passes: double-buffered tiles chosen
    bool l1_copies = false; // tile copies of 8 bytes through L1 (complex64 at odd d or odd runs)
    int ncols = 0;          // gradient columns (adjoint passes)
    size_t header = 24;     // bytes of pointers and tile count before geo[]
    CUfunction fn = nullptr;
    int threads = 256;
    size_t smem = 0;
    int grid = 1;
    bool params = true;     // pool in the kernel parameters
    bool red = false;       // reduces <N_q> when given rows (the program's last pass, complex64)
    int npool = 0;
    size_t arg_bytes = 0, pool_off = 0;
    int NG = 1;
};

struct JitProgram {
    std::vector<JitPassInfo> passes;   // per plan pass (fn == nullptr for strided / mc passes)
};

// CUDA source of every tile pass of a plan (one translation unit per pass,
// empty for strided / multi-controlled passes), and the launch shape of each.
// `ops` are the passes' localized ops in pool order (op.mat already set), one
// vector per pass; k_override > 0 sets the register slots per stage.
static std::vector<std::string> gen_sources(const std::vector<PassPlan> &plan, std::vector<std::vector<TOp>> &ops,
                                            int d, bool c128, int k_override, bool adj, JitProgram *jp,
                                            std::vector<std::string> &names, bool df) {
    jp->passes.resize(plan.size());
    names.assign(plan.size(), std::string());
    std::vector<std::string> out(plan.size());
    std::vector<PassSrc> specs(plan.size());
    for (size_t pi = 0; pi < plan.size(); ++pi) {
        const PassPlan &pp = plan[pi];
        if (pp.strided || pp.mc) continue;
        PassSrc &ps = specs[pi];
        ps.d = d;
        ps.c128 = c128;
        ps.df = df && c128;
        ps.T = pp.geom.T;
        ps.SEG = pp.geom.SEG;
        ps.nt = pp.geom.nt;
        ps.kA = pp.geom.kA;
        ps.nruns = pp.geom.nruns;
        ps.ntiles = pp.geom.ntiles;
        ps.runM.assign(pp.geom.runM, pp.geom.runM + pp.geom.nruns);
        ps.runS.assign(pp.geom.runS, pp.geom.runS + pp.geom.nruns);
        ps.strideA.assign(pp.geom.strideA, pp.geom.strideA + pp.geom.kA);
        ps.adj = adj;
        ps.pad = use_pad(d, c128, adj, ps.SEG);
        ps.n = 0;
        for (long long N = 1; N < (long long)ps.ntiles * ps.T; N *= d) ++ps.n;
        // the last pass of a complex64 forward program can reduce <N_q> too
        if (!adj && !c128 && pi + 1 == plan.size() && ps.ntiles < (1ll << 32) && ps.n + 1 <= 64) {
            ps.red = true;
            const int n = ps.n;
            for (int i = 0; i < ps.nt; ++i)
                ps.local_q.push_back(i < ps.kA ? pp.active[i] : n - pp.geom.rL + (i - ps.kA));
            long long prefix = 1;
            for (int r = 0; r < ps.nruns; ++r) {
                int hi = n - 1, len = 0;
                for (long long v = ps.runS[r]; v > 1; v /= d) --hi;
                for (long long v = ps.runM[r]; v > 1; v /= d) ++len;
                long long dx = prefix;
                for (int x = hi; x > hi - len; --x) {
                    ps.outer_div.push_back({x, dx});
                    dx *= d;
                }
                prefix *= ps.runM[r];
            }
        }
        ps.K = std::min(k_override > 0 ? k_override : (adj ? jit_stage_k_adj(d, c128) : jit_stage_k(d, c128, ps.df)),
                        pp.geom.nt);
        ps.ops = ops[pi];
        ps.stages = build_stages(ps.ops, pp.geom, d, ps.K);
        ops[pi] = ps.ops;   // the stage slots written by build_stages
        // Direct stages (forward and adjoint passes, not the reducing pass,
        // whose tile goes through shared memory for the reduction): the last
        // stage stores to HBM at every d and precision; the first stage loads
        // from HBM for complex64 at odd d.  Measured on GB300 (200-gate
        // programs, program time): complex64 d=2 6.01 -> 5.94 ms, d=3 6.71 ->
        // 6.26, d=4 9.52 -> 9.39, d=5 18.82 -> 17.45; complex128 (double-
        // float) 2 % faster; adjoint gradients (d=3 ansatz) 4.50 -> 4.31 ms
        // at n=14, 1559 -> 1485 ms at n=20 (complex64), 16.6 -> 16.3 ms
        // (complex128).  Direct loads at even d lose the double-buffered
        // prefetch (d=2 2 %, d=4 4 % slower), and in double-float passes they
        // measured 1.3 % slower than direct stores alone.
        if (!ps.red && !ps.stages.empty() && ps.T > ps.SEG) {
            auto direct = [&](const TStage &s) {
                if (s.legacy) return false;
                for (int x = 0; x < ps.K; ++x)
                    if (s.ls[x] < ps.SEG) return false;   // a run qudit
                return true;
            };
            ps.din = !c128 && d % 2 == 1 && direct(ps.stages.front());
            ps.dout = direct(ps.stages.back());
        }
        // L2 prefetch of the next tile: complex64 forward passes at odd d
        // (never double-buffered) whose runs are at least a cache line.
        // Measured per pass on GB300: runs of 27-729 amplitudes up to 12 %
        // faster (d=3 program 6.27 -> 5.97 ms), 25-amplitude runs 0-6 %;
        // 5-amplitude (40-byte) runs 4-51 % slower (two prefetches and an
        // index per 40 bytes, and up to 17 more registers).
        ps.pf = !adj && !c128 && d % 2 == 1 && (long long)ps.SEG * 8 >= 128;
        int npool = 0;
        bool dense_k = false;
        for (const TOp &o : ps.ops) dense_k |= o.kind == OP_DENSEK;
        // pool size: one past the largest entry any op uses
        for (const TOp &o : ps.ops) {
            int cnt = 0;
            switch (o.kind) {
            case OP_DENSE: cnt = d * d; break;
            case OP_PAIR: cnt = 4; break;
            case OP_DIAG: cnt = d; break;
            case OP_CPAIR: cnt = 4 * d; break;
            case OP_CDIAG: cnt = d * d; break;
            case OP_DENSEK: { int K = 1; for (int i = 0; i < o.nq; ++i) K *= d; cnt = K * K; break; }
            default: cnt = 0;
            }
            npool = std::max(npool, o.mat + cnt);
            if (adj && o.gcol >= 0) {
                const int gcnt = (o.kind == OP_PAIR || o.kind == OP_CPAIR) ? 4 : d;
                npool = std::max(npool, o.gmat + gcnt);
                ps.ncols = std::max(ps.ncols, o.gcol + 1);
            }
        }
        ps.npool = npool;
        const int units = ps.df ? 2 : 1;   // 16-byte units per entry
        ps.params = npool * units <= kParamPoolMax && !dense_k;
        const int DK = ipow_i(d, ps.K);
        // one register block per thread and stage where 128 threads cover
        // them; forward complex64 passes with up to 256 blocks also run 128
        // threads (two blocks each: 3 % faster at d=4 on GB300, more CTAs
        // per SM)
        const int nblk = ps.T / DK;
        ps.threads = (nblk <= 128 || (!adj && !c128 && nblk <= 256)) ? 128 : 256;
        std::ostringstream nm;
        nm << (adj ? "k_tile_adj_jit_d" : "k_tile_jit_d") << d << (ps.df ? "_c128df_" : c128 ? "_c128_" : "_c64_") << pi;
        names[pi] = nm.str();
        std::ostringstream src;
        src << "#define QJ_C64 " << (c128 ? 0 : 1) << "\n#define QJ_DF " << (ps.df ? 1 : 0) << "\n" << kPrelude;
        Gen g(ps, src);
        g.tile_base_lit(names[pi]);
        if (adj) g.kernel_adj(names[pi]);
        else g.kernel(names[pi]);
        out[pi] = src.str();
        JitPassInfo &ji = jp->passes[pi];
        ji.threads = ps.threads;
        if (adj) {
            ji.smem = (size_t)2 * ps.T * (c128 ? 16 : 8) + (size_t)(ps.T / ps.SEG) * 8;   // psi and lambda tiles
        } else {
            const size_t boff = ((size_t)(ps.T / ps.SEG) * 8 + 15) & ~(size_t)15;
            ji.smem = boff + (size_t)ps.slots() * (c128 ? 16 : 8);         // single buffer
            ji.smem2 = boff + (size_t)2 * ps.slots() * (c128 ? 16 : 8);    // double buffer
            ji.l1_copies = !c128 && !ps.pad && !(d % 2 == 0 && ps.SEG % 2 == 0);
            if (ps.din) ji.smem2 = 0;   // nothing to prefetch
            if (ps.din && ps.dout && ps.stages.size() == 1) ji.smem = boff;   // no tile in shared memory
        }
        ji.ncols = ps.ncols;
        ji.header = adj ? 40 : 32;
        ji.red = ps.red;
        ji.params = ps.params;
        ji.npool = npool;
        ji.NG = std::max(1, 2 * ps.nruns + ps.kA);
        ji.pool_off = (ji.header + 8 * (size_t)ji.NG + 15) & ~(size_t)15;
        ji.arg_bytes = ji.pool_off + 16 * (size_t)units * std::max(1, ps.params ? npool : 1);
    }
    return out;
}

qf_status jit_source(const std::vector<PassPlan> &plan, std::vector<std::vector<TOp>> &ops, int d, bool c128,
                     int k_override, bool adj, std::string *out, bool df) {
    JitProgram jp;
    std::vector<std::string> names;
    std::vector<std::string> srcs = gen_sources(plan, ops, d, c128, k_override, adj, &jp, names, df);
    out->clear();
    for (const std::string &x : srcs)
        if (!x.empty()) *out += "// ---- translation unit\n" + x;
    return QF_OK;
}

namespace {

// FNV-1a over the source, the target and the NVRTC / driver versions: the
// name of a cached cubin (a cubin from another toolkit gets another name).
std::string source_key(const std::string &src, const std::string &arch) {
    uint64_t h = 1469598103934665603ull;
    for (unsigned char c : src + "|" + arch + "|" + g_tool_tag) {
        h ^= c;
        h *= 1099511628211ull;
    }
    char buf[32];
    snprintf(buf, sizeof(buf), "%016llx", (unsigned long long)h);
    return std::string(buf) + "_" + std::to_string(src.size());
}

// Cubin cache directory next to the library (created on first use).
std::string cache_dir() {
    Dl_info info;
    std::string dir;
    if (dladdr((void *)&cache_dir, &info) && info.dli_fname) {
        dir = info.dli_fname;
        const size_t k = dir.rfind('/');
        dir = (k == std::string::npos ? std::string(".") : dir.substr(0, k)) + "/jit_cache";
    }
    return dir;
}

bool read_file(const std::string &path, std::vector<char> &out) {
    FILE *f = fopen(path.c_str(), "rb");
    if (!f) return false;
    fseek(f, 0, SEEK_END);
    const long n = ftell(f);
    fseek(f, 0, SEEK_SET);
    out.resize(n > 0 ? (size_t)n : 0);
    const bool ok = n > 0 && fread(out.data(), 1, (size_t)n, f) == (size_t)n;
    fclose(f);
    return ok;
}

void write_file(const std::string &path, const std::vector<char> &data) {
    const std::string tmp = path + ".tmp" + std::to_string((long)getpid());
    FILE *f = fopen(tmp.c_str(), "wb");
    if (!f) return;
    const bool ok = fwrite(data.data(), 1, data.size(), f) == data.size();
    fclose(f);
    if (ok) rename(tmp.c_str(), path.c_str());
    else remove(tmp.c_str());
}

// Compiles one translation unit; returns false with the log on failure.
bool nvrtc_compile(const std::string &code, const std::string &arch, std::vector<char> &cubin, std::string &log) {
    nvrtcProgram prog;
    if (g_nv.create(&prog, code.c_str(), "qf_tile_pass.cu", 0, nullptr, nullptr) != NVRTC_SUCCESS) {
        log = "program creation failed";
        return false;
    }
    const char *opts[] = {arch.c_str(), "-std=c++17", "-default-device"};
    const nvrtcResult cr = g_nv.compile(prog, 3, opts);
    if (cr != NVRTC_SUCCESS) {
        size_t ls = 0;
        g_nv.log_size(prog, &ls);
        log.assign(ls, '\0');
        if (ls) g_nv.log(prog, &log[0]);
        g_nv.destroy(&prog);
        return false;
    }
    size_t cs = 0;
    g_nv.cubin_size(prog, &cs);
    cubin.resize(cs);
    g_nv.cubin(prog, cubin.data());
    g_nv.destroy(&prog);
    return true;
}

}  // namespace

// Builds (or reuses) the kernels of every tile pass of a plan: cached modules
// of this process first, then cubins cached on disk, then NVRTC (passes
// compiled in parallel threads).
qf_status jit_build(const std::vector<PassPlan> &plan, std::vector<std::vector<TOp>> &ops, int d, bool c128,
                    int k_override, bool adj, int num_sms, JitProgram **out, bool df) {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!load_apis()) return set_error(QF_ERR_UNSUPPORTED, g_load_err);
    JitProgram *jp = new JitProgram();
    std::vector<std::string> names;
    const std::vector<std::string> srcs = gen_sources(plan, ops, d, c128, k_override, adj, jp, names, df);
    int major = 10, minor = 3, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
    const std::string arch = "--gpu-architecture=sm_" + std::to_string(major) + std::to_string(minor) + "a";
    int smem_optin = 0;   // largest dynamic shared memory a CTA may opt in to
    cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const std::string dir = cache_dir();
    if (!dir.empty()) mkdir(dir.c_str(), 0755);
    const size_t np = plan.size();
    std::vector<std::vector<char>> cubins(np);
    std::vector<std::string> keys(np), logs(np);
    std::vector<char> need(np, 0);
    for (size_t pi = 0; pi < np; ++pi) {
        if (srcs[pi].empty() || g_modules.count({dev, srcs[pi]})) continue;
        keys[pi] = source_key(srcs[pi], arch);
        if (!dir.empty() && read_file(dir + "/" + keys[pi] + ".cubin", cubins[pi])) continue;
        need[pi] = 1;
    }
    std::vector<std::thread> pool;
    std::vector<char> ok(np, 1);
    std::atomic<size_t> next(0);
    const unsigned nthreads = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
    for (unsigned w = 0; w < nthreads; ++w)
        pool.emplace_back([&]() {
            for (size_t pi = next++; pi < np; pi = next++)
                if (need[pi]) ok[pi] = nvrtc_compile(srcs[pi], arch, cubins[pi], logs[pi]) ? 1 : 0;
        });
    for (auto &t : pool) t.join();
    cudaFree(0);   // the runtime's primary context is current
    for (size_t pi = 0; pi < np; ++pi) {
        if (srcs[pi].empty()) continue;
        if (!ok[pi]) {
            delete jp;
            return set_error(QF_ERR_CUDA, "NVRTC compile of a tile pass failed: " + logs[pi].substr(0, 2000));
        }
        CUmodule mod = nullptr;
        auto it = g_modules.find({dev, srcs[pi]});
        if (it != g_modules.end()) {
            mod = it->second;
        } else {
            CUresult lr = g_drv.module_load(&mod, cubins[pi].data());
            if (lr != CUDA_SUCCESS && !need[pi]) {
                // a cached cubin this driver rejects: compile afresh and
                // replace the cache entry
                if (!nvrtc_compile(srcs[pi], arch, cubins[pi], logs[pi])) {
                    delete jp;
                    return set_error(QF_ERR_CUDA, "NVRTC compile of a tile pass failed: " + logs[pi].substr(0, 2000));
                }
                need[pi] = 1;
                lr = g_drv.module_load(&mod, cubins[pi].data());
            }
            if (lr != CUDA_SUCCESS) {
                delete jp;
                return set_error(QF_ERR_CUDA, "loading a compiled tile pass failed: " + cuda_err(lr));
            }
            g_modules[{dev, srcs[pi]}] = mod;
            if (need[pi] && !dir.empty()) write_file(dir + "/" + keys[pi] + ".cubin", cubins[pi]);
        }
        JitPassInfo &ji = jp->passes[pi];
        if (ji.smem > (size_t)smem_optin) {
            delete jp;
            return set_error(QF_ERR_ARG, "a tile pass needs " + std::to_string(ji.smem) +
                                             " bytes of shared memory, above the " + std::to_string(smem_optin) +
                                             " a CTA may hold");
        }
        if (ji.smem2 > (size_t)smem_optin) ji.smem2 = 0;   // a second tile does not fit: single buffer
        CUresult r = g_drv.get_function(&ji.fn, mod, names[pi].c_str());
        const size_t smax = std::max(ji.smem, ji.smem2);
        if (r == CUDA_SUCCESS && smax > 48 * 1024)
            r = g_drv.set_attribute(ji.fn, CU_FUNC_ATTRIBUTE_MAX_DYNAMIC_SHARED_SIZE_BYTES, (int)smax);
        int per_sm = 0;
        if (r == CUDA_SUCCESS) r = g_drv.occupancy(&per_sm, ji.fn, ji.threads, ji.smem);
        if (r == CUDA_SUCCESS && ji.smem2 > 0 && per_sm > 0) {
            // double-buffer only where the second tile costs no CTAs per SM
            // and, for passes whose 8-byte copies go through L1, leaves the
            // SM at least ~67 KB of it
            int per_sm2 = 0;
            r = g_drv.occupancy(&per_sm2, ji.fn, ji.threads, ji.smem2);
            if (r == CUDA_SUCCESS && per_sm2 >= per_sm && (!ji.l1_copies || (size_t)per_sm * ji.smem2 <= 160 * 1024)) {
                ji.dbuf = true;
                ji.smem = ji.smem2;
            }
        }
        if (r != CUDA_SUCCESS || per_sm < 1) {
            delete jp;
            return set_error(QF_ERR_CUDA, "tile pass kernel setup failed: " + cuda_err(r));
        }
        long long grid = (long long)per_sm * num_sms;
        if (grid > plan[pi].geom.ntiles) grid = plan[pi].geom.ntiles;
        ji.grid = (int)grid;
    }
    *out = jp;
    return QF_OK;
}

void jit_free(JitProgram *jp) { delete jp; }

bool jit_pass_ready(const JitProgram *jp, size_t pi) { return jp && pi < jp->passes.size() && jp->passes[pi].fn; }

// Whether pass pi takes its entries from a global pool (the caller uploads
// the prepared entries and passes their device address).
bool jit_pass_global_pool(const JitProgram *jp, size_t pi) { return !jp->passes[pi].params; }

// Launches pass pi.  `prepared` holds the pass's entries in kernel form
// (complex64: (re, re, -im, im) as float4; complex128: (re, im) as double2),
// 16 bytes each; gpool is their device copy when the pass reads them globally.
qf_status jit_launch(const JitProgram *jp, size_t pi, cudaStream_t stream, void *psi, const TileGeom &g,
                     const void *prepared, int npool, const void *gpool, double *rows) {
    const JitPassInfo &ji = jp->passes[pi];
    std::vector<unsigned char> args(ji.arg_bytes, 0);
    std::memcpy(args.data(), &psi, 8);
    std::memcpy(args.data() + 8, &gpool, 8);
    const long long mode = ji.dbuf ? 1 : 0;
    std::memcpy(args.data() + 16, &mode, 8);
    if (!ji.red) rows = nullptr;
    std::memcpy(args.data() + 24, &rows, 8);
    long long geo[2 * (kMaxActive + 1) + kMaxActive] = {};
    for (int r = 0; r < g.nruns; ++r) {
        geo[r] = g.runM[r];
        geo[g.nruns + r] = g.runS[r];
    }
    for (int i = 0; i < g.kA; ++i) geo[2 * g.nruns + i] = g.strideA[i];
    std::memcpy(args.data() + 32, geo, 8 * (size_t)(2 * g.nruns + g.kA));
    if (ji.params && npool > 0) std::memcpy(args.data() + ji.pool_off, prepared, 16 * (size_t)npool);
    void *kp[] = {args.data()};
    const CUresult r = g_drv.launch(ji.fn, (unsigned)ji.grid, 1, 1, (unsigned)ji.threads, 1, 1, (unsigned)ji.smem,
                                    (CUstream)stream, kp, nullptr);
    if (r != CUDA_SUCCESS) return set_error(QF_ERR_CUDA, "tile pass launch failed: " + cuda_err(r));
    return QF_OK;
}

bool jit_pass_reduces(const JitProgram *jp, size_t pi) { return jp && pi < jp->passes.size() && jp->passes[pi].red; }

// Launches reverse pass pi of the adjoint sweep; rows receives grid x ncols
// doubles (jit_pass_grid, jit_pass_ncols).
qf_status jit_launch_adj(const JitProgram *jp, size_t pi, cudaStream_t stream, void *psi, void *lam, double *rows,
                         const TileGeom &g, const void *prepared, int npool, const void *gpool) {
    const JitPassInfo &ji = jp->passes[pi];
    std::vector<unsigned char> args(ji.arg_bytes, 0);
    std::memcpy(args.data(), &psi, 8);
    std::memcpy(args.data() + 8, &lam, 8);
    std::memcpy(args.data() + 16, &gpool, 8);
    std::memcpy(args.data() + 24, &rows, 8);
    std::memcpy(args.data() + 32, &g.ntiles, 8);
    long long geo[2 * (kMaxActive + 1) + kMaxActive] = {};
    for (int r = 0; r < g.nruns; ++r) {
        geo[r] = g.runM[r];
        geo[g.nruns + r] = g.runS[r];
    }
    for (int i = 0; i < g.kA; ++i) geo[2 * g.nruns + i] = g.strideA[i];
    std::memcpy(args.data() + 40, geo, 8 * (size_t)(2 * g.nruns + g.kA));
    if (ji.params && npool > 0) std::memcpy(args.data() + ji.pool_off, prepared, 16 * (size_t)npool);
    void *kp[] = {args.data()};
    const CUresult r = g_drv.launch(ji.fn, (unsigned)ji.grid, 1, 1, (unsigned)ji.threads, 1, 1, (unsigned)ji.smem,
                                    (CUstream)stream, kp, nullptr);
    if (r != CUDA_SUCCESS) return set_error(QF_ERR_CUDA, "adjoint tile pass launch failed: " + cuda_err(r));
    return QF_OK;
}

int jit_pass_grid(const JitProgram *jp, size_t pi) { return jp->passes[pi].grid; }
int jit_pass_ncols(const JitProgram *jp, size_t pi) { return jp->passes[pi].ncols; }

}  // namespace qf
