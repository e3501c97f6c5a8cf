/*
 * qf.h -- C ABI of libqf, a GB300 (sm_103a) qudit state-vector engine.
 *
 * The operations follow QuForge (arXiv 2409.17716): a register of n qudits of
 * dimension d is a dense complex vector of d^n amplitudes (section "Library
 * Architecture"; the State class), gates from Appendix B "Matrix form of the
 * quantum gates" are applied to it in circuit order (the Circuit class), and
 * the result is reduced to expectation values (the measure utility of
 * section "Code style" returns the marginal probabilities they are built from).
 *
 * Conventions shared by every entry point
 *   - Basis index i = sum_q i_q d^(n-1-q) (Appendix B, "Generalized CNOT
 *     gate", decimal representation): qudit 0 is the most significant digit,
 *     qudit q has stride d^(n-1-q).  Levels are 0-based.
 *   - Amplitudes are stored contiguously, real and imaginary parts
 *     interleaved: QF_C64 = two floats per amplitude, QF_C128 = two doubles.
 *     Device buffers must be 16-byte aligned.
 *   - Every call is asynchronous on the state's CUDA stream, except the ones
 *     documented as returning host results (they synchronise that stream).
 *   - Arguments are validated on the host before any launch; an invalid call
 *     returns QF_ERR_ARG and leaves the state untouched.  qf_last_error()
 *     returns a thread-local message describing the most recent failure.
 *   - Angles and matrices are passed in FP64 on the host.  Gate entries are
 *     computed in FP64 once per gate and rounded to the state's precision.
 *   - Supported sizes: 2 <= d <= 16, n >= 1, d^n amplitudes must fit in
 *     device memory (QF_ERR_OOM otherwise).
 */
#ifndef QF_H
#define QF_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    QF_OK = 0,
    QF_ERR_ARG = 1,         /* invalid argument; nothing was launched */
    QF_ERR_OOM = 2,         /* device or pinned-host allocation failed */
    QF_ERR_CUDA = 3,        /* a CUDA runtime call failed (message in qf_last_error) */
    QF_ERR_TIMEOUT = 4,     /* a bounded device-side wait gave up */
    QF_ERR_UNSUPPORTED = 5  /* valid request outside this build's limits */
} qf_status;

typedef enum { QF_C64 = 0, QF_C128 = 1 } qf_dtype;

typedef struct qf_state qf_state;
typedef struct qf_program qf_program;

/* Observables for qf_expect (section "Code style": measure returns the
 * probabilities of the measured qudits; <N_q> = sum_m m P_q(m)).
 *   QF_OBS_NUMBER_ALL : out[0..n-1] = <N_q> for N = diag(0, 1, ..., d-1) on
 *                       every qudit q, out[n] = sum_i |psi_i|^2.  (n+1 values)
 *   QF_OBS_NORM       : out[0] = sum_i |psi_i|^2.                  (1 value)
 *   QF_OBS_HERMITIAN  : out[0] = Re <psi| O_q |psi>, out[1] = Im, for the
 *                       d x d row-major complex matrix `matrix` (interleaved
 *                       re, im, FP64, host memory) on qudit `q`. (2 values)
 *   QF_OBS_MARGINAL   : out[r] = probability that qudit `q` is at level r,
 *                       r = 0..d-1.                                 (d values)
 * All sums are accumulated in FP64 on the device. */
typedef enum { QF_OBS_NUMBER_ALL = 0, QF_OBS_NORM = 1, QF_OBS_HERMITIAN = 2, QF_OBS_MARGINAL = 3 } qf_obs_kind;

typedef struct {
    int kind;              /* qf_obs_kind */
    int q;                 /* qudit for QF_OBS_HERMITIAN / QF_OBS_MARGINAL */
    const double *matrix;  /* QF_OBS_HERMITIAN: host FP64 interleaved d x d */
} qf_obs;

/* Thread-local description of the last error (never NULL). */
const char *qf_last_error(void);

/* Number of output doubles qf_expect writes for `obs` on a (d, n) register,
 * or -1 for an invalid observable. */
int qf_expect_size(int d, int n, const qf_obs *obs);

/* ---------------------------------------------------------------- states */

/* Allocates a state of d^n amplitudes on the current CUDA device, owned by the
 * library, and sets it to |0...0> (the State class with an all-zero string).
 * `cuda_stream` is a cudaStream_t (NULL = legacy default stream).  The handle
 * is written to *out.  Errors: QF_ERR_ARG (d, n out of range, out NULL),
 * QF_ERR_OOM, QF_ERR_CUDA. */
qf_status qf_state_init(int d, int n, qf_dtype dt, void *cuda_stream, qf_state **out);

/* Wraps caller-owned device memory (e.g. a torch tensor's data pointer) of
 * d^n amplitudes of type dt.  The memory is borrowed: qf_state_free does not
 * free it, and it must outlive the handle.  Contents are left unchanged.
 * Errors: QF_ERR_ARG (NULL or misaligned pointer, bad sizes). */
qf_status qf_state_wrap(int d, int n, qf_dtype dt, void *dev_ptr, void *cuda_stream, qf_state **out);

/* Registers that mix qudit dimensions (section "Code style":
 * Circuit(dim=[2,3,4]) and State('0-1-3', dim=[2,3,4])).  dims[q] in [2, 16]
 * is the dimension of qudit q; the state holds prod_q dims[q] amplitudes with
 * the mixed-radix index i = sum_q i_q S_q, S_q = prod_{p>q} dims[p] (qudit 0
 * most significant).  dims is copied.  Every gate and measurement entry point
 * accepts such a state: levels and angles are bounded by the target's own
 * dimension; SUM(c, t) maps |c>|t> to |c>|(t + c) mod d_t> and a controlled
 * rotation runs over the control's d_c levels; SWAP needs two qudits of equal
 * dimension; a custom gate's matrix has prod_i dims[targets[i]] (<= 64) rows.
 * Gates run one launch each (no fusion).  If every entry of dims is equal the
 * state is an ordinary d^n register.  Limits: prod_q dims[q] / dims[0] < 2^31
 * (QF_ERR_UNSUPPORTED otherwise).  qf_state_info reports d = 0 for a mixed
 * register.  Errors as qf_state_init / qf_state_wrap, plus QF_ERR_ARG for
 * dims NULL or an entry out of range. */
qf_status qf_state_init_dims(const int *dims, int n, qf_dtype dt, void *cuda_stream, qf_state **out);
qf_status qf_state_wrap_dims(const int *dims, int n, qf_dtype dt, void *dev_ptr, void *cuda_stream, qf_state **out);
/* Copies the n per-qudit dimensions into dims[0..n-1] (cap >= n). */
qf_status qf_state_dims(const qf_state *s, int *dims, int cap);

/* Releases the handle, its scratch buffers and, if owned, the amplitudes.
 * Synchronises the state's stream first.  NULL is accepted. */
qf_status qf_state_free(qf_state *s);

/* Device pointer of the amplitudes and their count d^n. */
qf_status qf_state_ptr(qf_state *s, void **dev_ptr, long long *num_amps);

/* Shape of a state: qudit dimension, qudit count and dtype (any output
 * pointer may be NULL). */
qf_status qf_state_info(const qf_state *s, int *d, int *n, qf_dtype *dt);

/* Changes the stream subsequent calls on this state are issued on. */
qf_status qf_state_set_stream(qf_state *s, void *cuda_stream);

/* psi = |index> for 0 <= index < d^n (State('i_0-i_1-...') of "Code style"
 * with the digits of `index`).  Writes every amplitude. */
qf_status qf_state_set_basis(qf_state *s, long long index);

/* dst <- src (same d, n, dtype); both on dst's stream. */
qf_status qf_state_copy(qf_state *dst, const qf_state *src);

/* Host buffers <-> amplitudes [first, first + count) of the state (the
 * State class of "Library Architecture" holds the amplitude vector; these
 * move it between host and device).  `host` holds count amplitudes in the
 * state's layout (interleaved re, im; float for QF_C64, double for
 * QF_C128).  One cudaMemcpyAsync on the state's stream: asynchronous for
 * page-locked host memory (the buffer must stay valid and, for upload,
 * unchanged until the stream reaches the copy), synchronous for pageable
 * memory.  QF_ERR_ARG for a NULL buffer or a range outside the state. */
qf_status qf_state_upload(qf_state *s, const void *host, long long first, long long count);
qf_status qf_state_download(qf_state *s, void *host, long long first, long long count);

/* Page-locked host memory for the copies above (no counterpart in the
 * paper): `bytes` rounded up to 2 MiB of anonymous pages, registered with
 * the CUDA driver; *out receives the address.  On GB300 with a Grace host,
 * uploads from this memory ran without the 150-400 ms stalls measured for
 * cudaHostAlloc memory.  Free with qf_host_free (QF_ERR_ARG for any other
 * pointer).  QF_ERR_OOM if mapping or page-locking fails. */
qf_status qf_host_alloc(size_t bytes, void **out);
qf_status qf_host_free(void *p);

/* ---------------------------------------------------------------- gates */

/* Custom gate (section "Quantum Gates": users may supply a matrix; the
 * Grover example applies 9 x 9 matrices on two qutrits).  U is a host
 * row-major d^k x d^k complex matrix (interleaved re, im, FP64), copied at
 * the call; targets[0] is the most significant factor.  Targets must be
 * distinct and in [0, n); 1 <= k and d^k <= 64.  U is not checked for
 * unitarity.  One pass over the touched amplitudes. */
qf_status qf_apply_gate(qf_state *s, const int *targets, int k, const double *U);

/* Rotation R(theta) = exp(-i theta S / 2) on qudit q (Appendix B,
 * "Generalized rotation gate"), with S chosen by axis:
 *   'x' : S_x^{jk} = |j><k| + |k><j|        (0 <= j < k < d)
 *   'y' : S_y^{jk} = -i|j><k| + i|k><j|     (0 <= j < k < d)
 *   'z' : |j><j| - |k><k|, the level-pair RZ that phases only j and k
 *         (0 <= j < k < d; equals the paper's S_z^1 for (j, k) = (0, 1))
 *   'g' : Gell-Mann diagonal S_z^j, 1 <= j <= d-1, k ignored
 *         (sqrt(2/(j(j+1))) on levels 0..j-1, -j sqrt(2/(j(j+1))) on level j).
 * Only the levels the rotation moves are read and written. */
qf_status qf_apply_rot(qf_state *s, int q, int j, int k, double theta, char axis);

/* Controlled rotation (Appendix B, "Controlled Rotation Gate"):
 * sum_m |m><m|_c (x) R^{jk}_axis(m theta)_t; control level m scales the angle,
 * m = 0 is the identity.  c != t, axis and levels as in qf_apply_rot. */
qf_status qf_apply_crot(qf_state *s, int c, int t, int j, int k, double theta, char axis);

/* Generalised CNOT / SUM (Appendix B, "Generalized CNOT gate"):
 * |..i_c..i_t..> -> |..i_c..(i_t + i_c) mod d..>, for c < t and c > t. */
qf_status qf_apply_sum(qf_state *s, int c, int t);

/* Generalised SWAP (Appendix B, "Generalized SWAP Gate") of qudits a != b. */
qf_status qf_apply_swap(qf_state *s, int a, int b);

/* Generalised NOT X_s (Appendix B, "Generalized NOT gate"):
 * |x> -> |x + shift mod d> on qudit q (any integer shift). */
qf_status qf_apply_x(qf_state *s, int q, int shift);

/* Phase-shift / clock gate to a power (Appendix B, "Generalized phase-shift
 * gate"): |x> -> w^(power x) |x>, w = exp(2 pi i / d). */
qf_status qf_apply_z(qf_state *s, int q, int power);

/* Fourier / generalised Hadamard (Appendix B, "Fourier gate"):
 * H_ab = w^(a b) / sqrt(d). */
qf_status qf_apply_h(qf_state *s, int q);

/* Multi-controlled gates (section "Quantum Gates" lists a Toffoli and a
 * multi-controlled NOT gate; the paper gives no qudit definition, so this
 * library reads them as follows).  controls[0..k-1] (1 <= k <= 5, distinct,
 * different from target):
 *   qf_apply_mcx: |c_1..c_k>|t> -> |c_1..c_k>|(t + shift * c_1 c_2 ... c_k) mod d_t>
 *                 (k = 1 is SUM; d = 2 and shift = 1 is the qubit Toffoli /
 *                 multi-controlled NOT);
 *   qf_apply_mcu: the d_t x d_t matrix U (host, row-major, interleaved FP64)
 *                 on the target where every control c_i is at levels[i]
 *                 (0 <= levels[i] < d_{c_i}), the identity elsewhere.
 * One launch, one thread per target fibre; fibres the gate leaves unchanged
 * are neither read nor written.  Programs run such a gate as a pass of its
 * own (qf_program_add_mcx / qf_program_add_mcu); batches reject them
 * (QF_ERR_UNSUPPORTED). */
qf_status qf_apply_mcx(qf_state *s, const int *controls, int k, int target, int shift);
qf_status qf_apply_mcu(qf_state *s, const int *controls, const int *levels, int k, int target, const double *U);

/* ---------------------------------------------------------------- measurement */

/* Evaluates `obs` (see qf_obs) and writes qf_expect_size() doubles to host
 * memory out_host.  Synchronises the state's stream. */
qf_status qf_expect(qf_state *s, const qf_obs *obs, double *out_host);

/* Measurement (section "Code style": measure(state, index, ..., shots)
 * returns a histogram and the probabilities of the measured qudits).
 * probs (host, d^k doubles): marginal probability of every joint level r of
 * the k qudits idx[0..k-1] (idx[0] most significant digit of r), summed in
 * FP64.  With shots > 0, counts (host, d^k int64) is the histogram of `shots`
 * samples: sample s falls in the first r whose cumulative probability exceeds
 * uniforms[s] times the total (uniforms: host, shots values in [0, 1), drawn
 * by the caller).  Requires d^k <= 16384.  Synchronises the state's stream. */
qf_status qf_measure(qf_state *s, const int *idx, int k, const double *uniforms, long long shots, double *probs,
                     long long *counts);

/* As qf_expect, but writes the FP64 results to device memory out_dev
 * (8-byte aligned) asynchronously on the state's stream. */
qf_status qf_expect_device(qf_state *s, const qf_obs *obs, double *out_dev);

/* Allocation-free <N_q> (no counterpart in the paper; a deployment aid).
 * For callers that cannot allocate device memory at the point of measurement
 * -- host callbacks and latency-bound loops that must not trigger the
 * device-wide synchronisation an allocation or free can cause, and hosts
 * whose own memory pool holds the whole device heap.  Computes what qf_expect with QF_OBS_NUMBER_ALL computes:
 * out_dev[q] = <N_q> for q < n and out_dev[n] = sum_i |psi_i|^2 (n + 1 FP64
 * values, device memory, 8-byte aligned), from the caller's d^n amplitudes at
 * psi_dev (device, 16-byte aligned, interleaved as dt), asynchronously on
 * cuda_stream (a cudaStream_t, NULL = legacy default stream).  No qf_state is
 * needed and nothing is allocated or freed: the per-CTA partial sums live in
 * one fixed 256 KiB device array (512 rows of 64 doubles) that every device
 * loading the library holds until the process exits.  Sizes: 2 <= d <= 16,
 * n >= 1 and d^n <= 9e15 (which keeps n + 1 within the array's 64 columns);
 * anything larger is rejected with QF_ERR_ARG and a message.  cuda_stream
 * must belong to the current device (QF_ERR_ARG otherwise), since the array
 * address used is the current device's.  The first call on each device looks up the array's device
 * address with that device current; make that first call before any stream
 * capture begins.  All calls share the array and it keeps the last call's
 * contents (every value a call reads is written by that call first, so
 * nothing needs clearing); calls whose kernels overlap on the GPU -- e.g. on
 * two streams at once -- race on it and must be serialised by the caller. */
qf_status qf_expect_number_noalloc(const void *psi_dev, int d, int n, qf_dtype dt, void *cuda_stream, double *out_dev);

/* ---------------------------------------------------------------- programs
 * A program is a circuit recorded once (the Circuit class of "Library
 * Architecture") and executed many times.  Running it plans passes: runs of
 * gates whose qudits fit one on-chip tile are applied in a single read and
 * write of the state (gates on disjoint qudits are moved past each other only
 * where they commute).  Rotations may take their angle from a parameter
 * vector supplied at run time (param_slot >= 0) or keep a fixed angle
 * (param_slot < 0, angle = theta). */

qf_status qf_program_create(int d, int n, qf_program **out);
/* A program on a mixed-dimension register (see qf_state_init_dims); it runs on
 * states of the same dims, one launch per gate, and its adjoint sweep
 * (qf_program_adjoint / qf_program_gradient) takes one launch per gate that
 * updates psi and lambda together and adds the gate's gradient term.  Mixed
 * programs cannot be added to a batch (QF_ERR_UNSUPPORTED). */
qf_status qf_program_create_dims(const int *dims, int n, qf_program **out);
qf_status qf_program_free(qf_program *p);
/* Number of gates recorded, and the number of parameter slots referenced
 * (1 + largest slot, 0 if none). */
qf_status qf_program_info(const qf_program *p, int *num_gates, int *num_params);

qf_status qf_program_add_gate(qf_program *p, const int *targets, int k, const double *U);
qf_status qf_program_add_rot(qf_program *p, int q, int j, int k, char axis, int param_slot, double theta);
qf_status qf_program_add_crot(qf_program *p, int c, int t, int j, int k, char axis, int param_slot, double theta);
qf_status qf_program_add_sum(qf_program *p, int c, int t);
qf_status qf_program_add_swap(qf_program *p, int a, int b);
qf_status qf_program_add_x(qf_program *p, int q, int shift);
qf_status qf_program_add_z(qf_program *p, int q, int power);
qf_status qf_program_add_h(qf_program *p, int q);
qf_status qf_program_add_mcx(qf_program *p, const int *controls, int k, int target, int shift);
qf_status qf_program_add_mcu(qf_program *p, const int *controls, const int *levels, int k, int target, const double *U);

/* Fusion control: enable != 0 (the default) plans fused passes; enable = 0
 * gives one pass per gate, in recorded order (the per-gate kernels).  Takes
 * effect at the next run. */
/* Tile passes of a program are compiled for the current GPU when the program
 * is first run after planning (NVRTC, about a second per program; compiled
 * passes are shared by identical programs in the process): gate structure,
 * register slots and offsets become literals and only the gate entries are
 * passed per run.  enable = 0 runs the same passes through the library's
 * generic tile kernel instead (no compilation).  Default 1.  Errors at run
 * time: QF_ERR_UNSUPPORTED if NVRTC cannot be loaded, QF_ERR_CUDA (with the
 * compiler log) if a pass fails to compile. */
qf_status qf_program_set_jit(qf_program *p, int enable);
/* Qudits held in registers per stage of a compiled tile pass (1..6; 0 = the
 * default for d, 5 for d = 2 and 2 for d = 3..5 in complex64): more slots
 * mean fewer shared-memory round trips and more registers per thread. */
qf_status qf_program_set_stage_slots(qf_program *p, int slots);
/* The CUDA source the program's tile passes compile from (for dtype dt; the
 * forward passes, or with adjoint != 0 the reverse passes of the adjoint
 * sweep), as a NUL-terminated string of *len bytes; buf (capacity cap) may be
 * NULL to query the length.  Host only; nothing is compiled or launched. */
qf_status qf_program_jit_source(qf_program *p, qf_dtype dt, int adjoint, char *buf, size_t cap, size_t *len);
qf_status qf_program_set_fusion(qf_program *p, int enable);
/* Arithmetic of the compiled forward passes on complex128 states.  The
 * state is complex128 either way ("Library Architecture": a state of complex
 * amplitudes); exact = 0 (the default) computes the gates in double-float
 * arithmetic on FP32 units -- each real an unevaluated sum of two floats,
 * products split exactly by a fused multiply-add (Dekker's TwoProduct), sums
 * by Knuth's TwoSum, about 48 significant bits, within 1e-12 max-abs of the
 * exact result after the 200-gate benchmark circuits -- converting the state
 * in place to that form before the first compiled pass and back after the
 * last (the caller never sees the intermediate form; the stream is the
 * state's).  exact = 1 computes in FP64 (on GB300 about 1/70 of the FP32
 * rate).  In the double-float form amplitudes must stay below 2^128 in
 * magnitude; parts of magnitude 2^-74 .. 2^-126 keep an absolute precision of
 * 2^-96 and smaller ones become 0.  The same choice applies to the compiled
 * reverse passes of the adjoint sweep (psi and lambda converted around them;
 * gradient terms summed in double-float per block, then in FP64); lambda =
 * O psi, the loss and the immediate-mode gates use FP64. */
qf_status qf_program_set_fp64(qf_program *p, int exact);
/* qf_program_run followed by <N_q> of every qudit and the norm ("Code
 * style": measure returns the marginals; <N_q> = sum_m m P_q(m)) into out_dev
 * (device, n + 1 FP64 values, 8-byte aligned), asynchronously on the state's
 * stream: what qf_program_run and qf_expect_device with QF_OBS_NUMBER_ALL
 * compute, in one pass fewer where the program's last pass is a compiled
 * complex64 tile pass -- it sums |psi|^2 weighted by every qudit's level
 * while its final tile is in shared memory (FP32 within a tile, FP64 across
 * tiles, the same order on every run).  Otherwise the separate reduction
 * runs after the program.  Errors as qf_program_run; QF_ERR_ARG for a NULL or
 * misaligned out_dev. */
qf_status qf_program_run_expect(qf_program *p, qf_state *s, const double *params, double *out_dev);
/* Arithmetic of the program as planned for dtype dt: complex multiply-adds
 * per amplitude summed over its fused ops (a multiply-add with a real entry
 * counts one half; permutations count zero).  Host only; no counterpart in
 * the paper (a measurement aid: with the device rates below it gives the
 * rate the arithmetic units alone would allow).  QF_ERR_UNSUPPORTED for
 * programs on mixed-dimension registers. */
qf_status qf_program_cmacs(qf_program *p, qf_dtype dt, double *cmacs_per_amplitude);
/* FP64 and FP32 fused multiply-add throughput of the current device (FMA/s),
 * measured on cuda_stream (synchronised) with eight independent FMA chains
 * per thread on 8 CTAs of 256 threads per SM, best of five timed launches
 * (CUDA events), at the clocks the GPU runs.  No counterpart in the paper:
 * it states which arithmetic unit bounds a pass.  Allocates and frees a
 * small device buffer; QF_ERR_OOM if that fails. */
qf_status qf_device_fma_rates(void *cuda_stream, double *fp64_fma_per_s, double *fp32_fma_per_s);

/* Tiling of fused passes (0 = default for each): tile_qudits = local qudits
 * per shared-memory tile (default: the largest t with d^t amplitudes <= 8192
 * for complex64 / 4096 for complex128, and 12 for forward passes of qubits in
 * complex64; a forward-pass override may go up to 160 KiB of amplitudes per
 * tile, single-buffered where two tiles exceed a CTA's shared memory);
 * min_run_qudits = lowest qudits always in the tile, so every contiguous run
 * read from HBM has d^r amplitudes (default 5, 3, 2, 1 for d = 2, 3, 4, 5 and
 * 4 for forward passes of qubits in complex64, chosen by measurement;
 * otherwise the smallest r with d^r >= 32); max_ops = gates per pass (<= 96).
 * Takes effect at the next run.  QF_ERR_ARG at run time if a pass would need
 * more shared memory than a CTA may hold. */
qf_status qf_program_set_tiling(qf_program *p, int tile_qudits, int min_run_qudits, int max_ops);

/* Applies the program to s (same d and n).  params: host FP64 vector of
 * at least num_params entries (may be NULL if num_params == 0).  Async. */
qf_status qf_program_run(qf_program *p, qf_state *s, const double *params);

/* Adjoint gradient (the paper differentiates through stored gate matrices
 * with autograd, "Sparsity to lower memory consumption"; here the "Generalized rotation
 * gate" and "Controlled Rotation Gate" definitions U = exp(-i theta G) give
 * dU/dtheta = -i G U with G = S/2, or sum_m |m><m| (x) m S/2 for the
 * controlled rotation).  Loss L = sum_q weights[q] <N_q> (weights: n host
 * doubles).  On entry psi holds the program's output psi_L for `params` (a
 * qf_program_run of this program on psi_0); lam is a second state of the same
 * shape and stream used as the costate and overwritten.  The sweep sets
 * lambda = O psi, then for every gate in reverse adds 2 Im<lambda|G|psi> to
 * its parameter slot and applies U^+ to psi and lambda; on return psi holds
 * psi_0 again up to rounding.  Writes L to loss_dev[0] and dL/dparams to
 * grad_dev[0 .. num_params-1] (device FP64, every slot written, 0 for unused
 * slots; shared slots sum their gates' terms).  Asynchronous on psi's stream.
 * Errors: QF_ERR_ARG for mismatched shapes, psi == lam, NULL outputs. */
qf_status qf_program_adjoint(qf_program *p, qf_state *psi, qf_state *lam, const double *params, const double *weights,
                             double *loss_dev, double *grad_dev);

/* Forward run of p on psi (holding psi_0 on entry) followed by
 * qf_program_adjoint; writes the loss and the num_params gradient entries to
 * host memory and synchronises psi's stream.  psi holds psi_0 again (up to
 * rounding) on return. */
qf_status qf_program_gradient(qf_program *p, qf_state *psi, qf_state *lam, const double *params, const double *weights,
                              double *loss_host, double *grad_host);

/* Number of kernel passes the last run or adjoint launched (for throughput
 * accounting), or -1 before the first run. */
int qf_program_last_passes(const qf_program *p);

/* Per-pass timing (tracing).  With timing enabled, every run records a CUDA
 * event on the state's stream before its first pass and after each pass;
 * the records accumulate over runs until qf_program_pass_times reads them.
 * Enabling or disabling clears them. */
qf_status qf_program_set_timing(qf_program *p, int enable);

/* Waits for the last timed run, then writes, for each of the first `max`
 * passes timed since the last read (all runs, in launch order), the elapsed
 * milliseconds between its events, its kernel (0 = tile pass, 1 = strided
 * single-gate pass) and its algorithmic HBM bytes (amplitudes read plus
 * written: 2 N b for a tile pass, the touched rows for a strided pass);
 * *count = number of passes timed.  Clears the records.  Any output pointer
 * may be NULL. */
qf_status qf_program_pass_times(qf_program *p, int max, float *ms, int *kind, double *bytes, int *count);

/* Plans the program for states of dtype dt without running it (host only):
 * number of passes, how many of them are single gates on the strided kernel,
 * and the largest number of ops in one pass.  Output pointers may be NULL. */
qf_status qf_program_plan(qf_program *p, qf_dtype dt, int *num_passes, int *num_strided, int *max_ops);

/* Register-stage statistics of the plan for dtype dt: tile passes, register
 * stages over all tile passes (one shared-memory round trip and one barrier
 * each) and ops (single-qudit runs already multiplied together).  Host-only
 * planning; nothing is launched. */
qf_status qf_program_stages(qf_program *p, qf_dtype dt, int *num_tile_passes, int *num_stages, int *num_ops);

/* ---------------------------------------------------------------- batches
 * Many independent circuits of uneven qudit dimension and size (the
 * data-encoding VQA circuits of the paper's "Variational quantum algorithm"
 * section, one per sample), run forward and backward together.  Each circuit
 * is a recorded program whose parametrised gates index one global parameter
 * vector (shared trainable angles and per-sample encoding angles alike) and a
 * loss L_c = sum_q weights_c[q] <N_q> on its own output.  Every circuit starts
 * from |0...0>.  Building plans each distinct circuit structure once, lays out
 * a psi and a lambda state per circuit in one device allocation, and captures
 * the whole run -- initialisation, one batched tile launch
 * per (qudit dimension, pass index), lambda = O psi with the losses, the
 * reverse passes and the gradient gathers -- into a CUDA graph; qf_batch_run
 * uploads the parameters and replays it.  Rotation entries are computed on the device from the
 * parameters, so the graph is valid for every parameter vector. */
typedef struct qf_batch qf_batch;

qf_status qf_batch_create(qf_dtype dt, void *cuda_stream, qf_batch **out);
qf_status qf_batch_free(qf_batch *b);

/* Copies the program's gates and n loss weights into the batch (before
 * qf_batch_build).  *index receives the circuit's index.  Circuits need
 * d^n < 2^31. */
qf_status qf_batch_add(qf_batch *b, const qf_program *p, const double *weights, int *index);

/* Tile size (local qudits, 0 = default) and fusion depth (gates per pass,
 * 0 = default) for the circuits of qudit dimension d; before building. */
qf_status qf_batch_tune(qf_batch *b, int d, int tile_qudits, int max_ops);

/* Plans, allocates (2 states per circuit plus tables) and captures the
 * graphs.  num_params = length of the global parameter vector; every slot a
 * circuit uses must be below it. */
qf_status qf_batch_build(qf_batch *b, int num_params);

/* Runs the batch for the host parameter vector (copied at the call, so the
 * caller may reuse it at once).  backward = 0: losses only; backward = 1:
 * losses and gradients.  Asynchronous with respect to the stream given at
 * creation (the batch runs on its own stream ordered after it). */
qf_status qf_batch_run(qf_batch *b, const double *params, int backward);

/* Device FP64 outputs of the last run, owned by the batch: loss[c] per
 * circuit; grad_local: for circuit c, at its grad_offset, dL_c/dparam for
 * each slot it uses (ascending slot order, see qf_batch_circuit_params);
 * grad_sum[s] = sum over circuits of dL_c/dparam_s. */
qf_status qf_batch_outputs(qf_batch *b, double **loss_dev, double **grad_local_dev, double **grad_sum_dev);

/* Copies the last run's outputs to host memory after waiting for it: loss
 * (one per circuit), grad_local and grad_sum with the lengths qf_batch_info
 * reports.  Any pointer may be NULL. */
qf_status qf_batch_read(qf_batch *b, double *loss_host, double *grad_local_host, double *grad_sum_host);

/* Parameter slots circuit `index` uses (ascending, up to max written), their
 * count and the offset of its entries in grad_local. */
qf_status qf_batch_circuit_params(const qf_batch *b, int index, int *slots, int max, int *count, long long *grad_offset);

/* Circuits, total amplitudes, sum over circuits of amplitudes x gates, the
 * kernel launches one forward-only / forward+backward graph replay makes, the
 * length of grad_local and of the parameter vector (grad_sum).  Any output
 * pointer may be NULL. */
qf_status qf_batch_info(const qf_batch *b, int *circuits, long long *amplitudes, double *gate_amplitudes,
                        int *launches_forward, int *launches_backward, long long *grad_local_len, int *num_params);

#ifdef __cplusplus
}
#endif

#endif /* QF_H */
