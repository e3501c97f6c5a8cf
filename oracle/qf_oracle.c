/*
 * qf_oracle.c -- plain CPU complex128 qudit state-vector simulator.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the correctness oracle for the GPU
 * library: only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark may load it.  It shares no code, header, table or helper with the
 * CUDA path, and the CUDA path never calls it.
 *
 * Everything here is written straight from the definitions in the paper
 * (QuForge, arXiv 2409.17716, Appendix B "Matrix form of the quantum gates"):
 * every gate is built entry by entry from its formula, and every gate is applied
 * by the same explicit gather / multiply / scatter loop over the groups of
 * amplitudes it couples.  No blocking, fusion or reordering.
 *
 * Conventions (Appendix B, "Generalized CNOT gate", decimal representation):
 *   basis index  j = sum_k j_k d^(n-1-k),  so qudit 0 is the most significant
 *   digit and qudit q has stride d^(n-1-q).  Levels are 0-based, as the paper's
 *   code uses them (end of "Generalized rotation gate").
 *   A k-qudit matrix U acting on targets (t_0, ..., t_{k-1}) is indexed by the
 *   row/column number r = sum_i r_i d^(k-1-i), r_i being the level of qudit t_i,
 *   so t_0 is the most significant factor (the left factor of the Kronecker
 *   product).  Matrices are row-major, complex128.
 *   Registers may mix dimensions (section "Code style": Circuit(dim=[2,3,4])):
 *   with dims[q] the dimension of qudit q the index is mixed-radix,
 *   j = sum_q j_q S_q with S_q = prod_{p>q} dims[p], and a k-qudit matrix on
 *   (t_0..t_{k-1}) has prod_i dims[t_i] rows indexed in the same mixed radix.
 *   The functions taking a single d are the equal-dimension case of the *_dims
 *   functions.
 *
 * Arithmetic is IEEE double, compiled with -ffp-contract=off so the x86 and Arm
 * builds round identically.  Gate application is parallelised with OpenMP over
 * independent groups only; every output amplitude is computed by the same
 * sequence of operations as in a serial run.  Reductions are serial.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <omp.h>

typedef double complex cplx;

#define OR_PI 3.14159265358979323846264338327950288

static long long or_ipow(int d, int e)
{
    long long r = 1;
    for (int i = 0; i < e; ++i) r *= d;
    return r;
}

/* omega^m with omega = exp(2 pi i / d)  ("Generalized phase-shift gate").
 * The exponent is reduced mod d first, which changes nothing mathematically. */
static cplx or_omega_pow(int d, long long m)
{
    long long r = m % d;
    if (r < 0) r += d;
    double a = 2.0 * OR_PI * (double)r / (double)d;
    return cos(a) + I * sin(a);
}

/* ------------------------------------------------------------------------- */
/* Single-qudit gate matrices (d x d, row-major).                            */
/* ------------------------------------------------------------------------- */

/* Identity. */
void or_gate_identity(int d, cplx *U)
{
    for (int a = 0; a < d; ++a)
        for (int b = 0; b < d; ++b) U[a * d + b] = (a == b) ? 1.0 : 0.0;
}

/* Fourier / generalised Hadamard ("Fourier gate"): H_ab = omega^(a b) / sqrt(d). */
void or_gate_fourier(int d, cplx *U)
{
    double s = 1.0 / sqrt((double)d);
    for (int a = 0; a < d; ++a)
        for (int b = 0; b < d; ++b) U[a * d + b] = s * or_omega_pow(d, (long long)a * b);
}

/* Generalised NOT ("Generalized NOT gate"): X_s |x> = |x + s mod d>.
 * Column x has its single 1 in row (x + s) mod d. */
void or_gate_shift(int d, int s, cplx *U)
{
    for (int a = 0; a < d * d; ++a) U[a] = 0.0;
    for (int x = 0; x < d; ++x) {
        int y = (int)(((long long)x + s) % d);
        if (y < 0) y += d;
        U[y * d + x] = 1.0;
    }
}

/* Phase-shift / clock ("Generalized phase-shift gate"): P = diag(1, w, ..., w^(d-1));
 * this returns P^p = diag(w^(p k)). */
void or_gate_clock(int d, int p, cplx *U)
{
    for (int a = 0; a < d * d; ++a) U[a] = 0.0;
    for (int k = 0; k < d; ++k) U[k * d + k] = or_omega_pow(d, (long long)p * k);
}

/* Generators S of the rotations ("Generalized Gell-Mann matrices"), 0-based:
 *   'x': S_x^{jk} = |j><k| + |k><j|
 *   'y': S_y^{jk} = -i|j><k| + i|k><j|
 *   'z': two-level diagonal |j><j| - |k><k|  (the level-pair RZ^{jk}; equals
 *        S_z^1 of the paper when (j,k) = (0,1))
 *   'g': Gell-Mann diagonal S_z^j, j = 1..d-1:
 *        sqrt(2/(j(j+1))) (sum_{l<j} |l><l| - j |j><j|)   (0-based levels)
 * Returns 0 on success, -1 on an invalid (axis, j, k). */
int or_generator(int d, int j, int k, char axis, cplx *S)
{
    for (int a = 0; a < d * d; ++a) S[a] = 0.0;
    if (axis == 'g') {
        if (j < 1 || j > d - 1) return -1;
        double c = sqrt(2.0 / ((double)j * (double)(j + 1)));
        for (int l = 0; l < j; ++l) S[l * d + l] = c;
        S[j * d + j] = -(double)j * c;
        return 0;
    }
    if (j < 0 || k <= j || k >= d) return -1;
    if (axis == 'x') {
        S[j * d + k] = 1.0;
        S[k * d + j] = 1.0;
    } else if (axis == 'y') {
        S[j * d + k] = -I;
        S[k * d + j] = I;
    } else if (axis == 'z') {
        S[j * d + j] = 1.0;
        S[k * d + k] = -1.0;
    } else {
        return -1;
    }
    return 0;
}

/* Rotation R(theta) = exp(-i theta S / 2) ("Generalized rotation gate").
 * The non-zero elements are the ones the paper lists:
 *   x: <j|R|j> = <k|R|k> = cos(theta/2), <j|R|k> = <k|R|j> = -i sin(theta/2)
 *   y: <j|R|j> = <k|R|k> = cos(theta/2), <j|R|k> = -sin(theta/2), <k|R|j> = +sin(theta/2)
 *   z/g: diagonal, <l|R|l> = exp(-i theta v_l / 2) with v_l the diagonal of S
 *   all other levels: 1.
 * Returns 0 on success, -1 on invalid arguments. */
int or_gate_rot(int d, int j, int k, double theta, char axis, cplx *U)
{
    cplx *S = (cplx *)malloc(sizeof(cplx) * (size_t)d * d);
    if (!S) return -1;
    if (or_generator(d, j, k, axis, S) != 0) { free(S); return -1; }
    or_gate_identity(d, U);
    double c = cos(0.5 * theta), s = sin(0.5 * theta);
    if (axis == 'x') {
        U[j * d + j] = c;
        U[k * d + k] = c;
        U[j * d + k] = -I * s;
        U[k * d + j] = -I * s;
    } else if (axis == 'y') {
        U[j * d + j] = c;
        U[k * d + k] = c;
        U[j * d + k] = -s;
        U[k * d + j] = s;
    } else { /* diagonal generators: 'z', 'g' */
        for (int l = 0; l < d; ++l) {
            double v = creal(S[l * d + l]);
            double a = -0.5 * theta * v;
            U[l * d + l] = cos(a) + I * sin(a);
        }
    }
    free(S);
    return 0;
}

/* Plain row-major complex matrix product C = A B (m x m). */
static void or_matmul(int m, const cplx *A, const cplx *B, cplx *C)
{
    for (int r = 0; r < m; ++r)
        for (int c = 0; c < m; ++c) {
            cplx acc = 0.0;
            for (int t = 0; t < m; ++t) acc += A[r * m + t] * B[t * m + c];
            C[r * m + c] = acc;
        }
}

/* dR/dtheta for R = exp(-i theta S/2): (-i S / 2) R(theta). */
int or_gate_rot_deriv(int d, int j, int k, double theta, char axis, cplx *dU)
{
    size_t sz = sizeof(cplx) * (size_t)d * d;
    cplx *S = (cplx *)malloc(sz), *R = (cplx *)malloc(sz);
    if (!S || !R) { free(S); free(R); return -1; }
    if (or_generator(d, j, k, axis, S) != 0 || or_gate_rot(d, j, k, theta, axis, R) != 0) {
        free(S); free(R); return -1;
    }
    for (int a = 0; a < d * d; ++a) S[a] *= -0.5 * I;
    or_matmul(d, S, R, dU);
    free(S); free(R);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Two-qudit gate matrices (d^2 x d^2, row-major, control = first factor).   */
/* ------------------------------------------------------------------------- */

/* Generalised CNOT = SUM ("Generalized CNOT gate"): |c>|t> -> |c>|t + c mod d>,
 * i.e. <c, t (+) c| C_x |c, t> = 1.  The index rule of the paper is used; the
 * displayed case equation there is garbled and is not followed.  With a
 * control of dimension dc and a target of dimension dt the control level is
 * added modulo the target's dimension: |c>|t> -> |c>|(t + c) mod dt>
 * (dc*dt x dc*dt, control = first factor). */
void or_gate_sum2(int dc, int dt, cplx *U)
{
    int D2 = dc * dt;
    for (int a = 0; a < D2 * D2; ++a) U[a] = 0.0;
    for (int c = 0; c < dc; ++c)
        for (int t = 0; t < dt; ++t) {
            int col = c * dt + t;
            int row = c * dt + (t + c) % dt;
            U[row * D2 + col] = 1.0;
        }
}

void or_gate_sum(int d, cplx *U)
{
    or_gate_sum2(d, d, U);
}

/* Generalised SWAP ("Generalized SWAP Gate"): |x>|y> -> |y>|x>. */
void or_gate_swap(int d, cplx *U)
{
    int D2 = d * d;
    for (int a = 0; a < D2 * D2; ++a) U[a] = 0.0;
    for (int x = 0; x < d; ++x)
        for (int y = 0; y < d; ++y) U[(y * d + x) * D2 + (x * d + y)] = 1.0;
}

/* Controlled rotation ("Controlled Rotation Gate"):
 *   C = sum_{m=0}^{dc-1} |m><m| (x) R^{jk}_alpha(m theta),
 * control of dimension dc, rotation on a target of dimension dt
 * (dc*dt x dc*dt).  deriv != 0 returns dC/dtheta = sum_m |m><m| (x) m R'(m theta). */
static int or_gate_crot_impl(int dc, int dt, int j, int k, double theta, char axis, int deriv, cplx *U)
{
    int D2 = dc * dt;
    cplx *R = (cplx *)malloc(sizeof(cplx) * (size_t)dt * dt);
    if (!R) return -1;
    for (int a = 0; a < D2 * D2; ++a) U[a] = 0.0;
    for (int m = 0; m < dc; ++m) {
        int rc = deriv ? or_gate_rot_deriv(dt, j, k, m * theta, axis, R)
                       : or_gate_rot(dt, j, k, m * theta, axis, R);
        if (rc != 0) { free(R); return -1; }
        for (int a = 0; a < dt; ++a)
            for (int b = 0; b < dt; ++b) {
                cplx v = R[a * dt + b];
                if (deriv) v *= (double)m;
                U[(m * dt + a) * D2 + (m * dt + b)] = v;
            }
    }
    free(R);
    return 0;
}

int or_gate_crot2(int dc, int dt, int j, int k, double theta, char axis, cplx *U)
{
    return or_gate_crot_impl(dc, dt, j, k, theta, axis, 0, U);
}

int or_gate_crot2_deriv(int dc, int dt, int j, int k, double theta, char axis, cplx *U)
{
    return or_gate_crot_impl(dc, dt, j, k, theta, axis, 1, U);
}

int or_gate_crot(int d, int j, int k, double theta, char axis, cplx *U)
{
    return or_gate_crot_impl(d, d, j, k, theta, axis, 0, U);
}

int or_gate_crot_deriv(int d, int j, int k, double theta, char axis, cplx *U)
{
    return or_gate_crot_impl(d, d, j, k, theta, axis, 1, U);
}

/* Multi-controlled gates.  The paper lists a Toffoli and a multi-controlled
 * NOT gate among its gates (section "Quantum Gates") without writing them out
 * for qudits.  Reading taken here, which reduces to SUM for one control and to
 * the qubit Toffoli / multi-controlled NOT for d = 2:
 *   MCX^s:  |c_1 .. c_k>|t> -> |c_1 .. c_k>|(t + s c_1 c_2 ... c_k) mod dt>
 * and, for a fixed single-qudit matrix V on the target,
 *   MCU:    V applied to the target when every control c_i is at level l_i,
 *           the identity otherwise.
 * Controls are the most significant factors, in the order given, then the
 * target; the matrices have (prod_i dc_i) * dt rows. */
int or_gate_mcx(const int *dc, int k, int dt, int s, cplx *U)
{
    long long C = 1;
    for (int i = 0; i < k; ++i) {
        if (dc[i] < 2) return -1;
        C *= dc[i];
    }
    long long D = C * dt;
    for (long long a = 0; a < D * D; ++a) U[a] = 0.0;
    for (long long c = 0; c < C; ++c) {
        /* product of the control levels spelled by c (first control most significant) */
        long long rem = c, prod = 1;
        for (int i = k - 1; i >= 0; --i) {
            prod *= rem % dc[i];
            rem /= dc[i];
        }
        long long sh = ((long long)s * prod) % dt;
        if (sh < 0) sh += dt;
        for (int t = 0; t < dt; ++t) {
            long long col = c * dt + t;
            long long row = c * dt + (t + sh) % dt;
            U[row * D + col] = 1.0;
        }
    }
    return 0;
}

int or_gate_mcu(const int *dc, const int *levels, int k, int dt, const cplx *V, cplx *U)
{
    long long C = 1;
    for (int i = 0; i < k; ++i) {
        if (dc[i] < 2 || levels[i] < 0 || levels[i] >= dc[i]) return -1;
        C *= dc[i];
    }
    long long D = C * dt;
    for (long long a = 0; a < D * D; ++a) U[a] = 0.0;
    for (long long c = 0; c < C; ++c) {
        long long rem = c;
        int match = 1;
        for (int i = k - 1; i >= 0; --i) {
            if (rem % dc[i] != levels[i]) match = 0;
            rem /= dc[i];
        }
        for (int a = 0; a < dt; ++a)
            for (int b = 0; b < dt; ++b)
                U[(c * dt + a) * D + (c * dt + b)] = match ? V[a * dt + b] : (a == b ? 1.0 : 0.0);
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Gate application.                                                          */
/* ------------------------------------------------------------------------- */

/* Fills stride[q] = prod_{p>q} dims[p] and returns the state length
 * prod_q dims[q], or -1 on an invalid dimension. */
static long long or_strides(const int *dims, int n, long long *stride)
{
    long long N = 1;
    for (int q = n - 1; q >= 0; --q) {
        if (dims[q] < 2) return -1;
        stride[q] = N;
        N *= dims[q];
    }
    return N;
}

/* Applies the K x K matrix U (K = prod_i dims[targets[i]]) to the target
 * qudits of psi (length prod_q dims[q]):
 *   psi'[.., r, ..] = sum_m U[r, m] psi[.., m, ..]
 * for every assignment of the non-target digits.  Targets must be distinct
 * and in [0, n).  Returns 0, or -1 on invalid arguments. */
int or_apply_dims(cplx *psi, const int *dims, int n, const int *targets, int k, const cplx *U)
{
    if (n < 1 || k < 1 || k > n || n > 64) return -1;
    int is_target[64];
    memset(is_target, 0, sizeof(is_target));
    for (int i = 0; i < k; ++i) {
        if (targets[i] < 0 || targets[i] >= n || is_target[targets[i]]) return -1;
        is_target[targets[i]] = 1;
    }
    long long *stride = (long long *)malloc(sizeof(long long) * n);
    if (!stride) return -1;
    long long N = or_strides(dims, n, stride);
    if (N < 0) { free(stride); return -1; }
    long long K = 1;
    for (int i = 0; i < k; ++i) K *= dims[targets[i]];
    long long G = N / K;
    long long *off = (long long *)malloc(sizeof(long long) * K);
    if (!off) { free(stride); return -1; }
    /* offset of row/column r inside a group: its digits r_i sit on qudit t_i */
    for (long long r = 0; r < K; ++r) {
        long long rem = r, o = 0;
        for (int i = k - 1; i >= 0; --i) {
            int dt = dims[targets[i]];
            o += (rem % dt) * stride[targets[i]];
            rem /= dt;
        }
        off[r] = o;
    }
    int fail = 0;
#pragma omp parallel
    {
        cplx *v = (cplx *)malloc(sizeof(cplx) * K);
        if (!v) {
#pragma omp atomic write
            fail = 1;
        } else {
#pragma omp for schedule(static)
            for (long long g = 0; g < G; ++g) {
                /* base index: the digits of g fill the non-target qudits,
                 * least significant qudit first */
                long long rem = g, base = 0;
                for (int q = n - 1; q >= 0; --q) {
                    if (is_target[q]) continue;
                    base += (rem % dims[q]) * stride[q];
                    rem /= dims[q];
                }
                for (long long m = 0; m < K; ++m) v[m] = psi[base + off[m]];
                for (long long r = 0; r < K; ++r) {
                    cplx acc = 0.0;
                    for (long long m = 0; m < K; ++m) acc += U[r * K + m] * v[m];
                    psi[base + off[r]] = acc;
                }
            }
            free(v);
        }
    }
    free(stride);
    free(off);
    return fail ? -1 : 0;
}

/* Equal dimensions: every qudit has dimension d. */
int or_apply(cplx *psi, int d, int n, const int *targets, int k, const cplx *U)
{
    if (d < 2 || n < 1 || n > 64) return -1;
    int dims[64];
    for (int q = 0; q < n; ++q) dims[q] = d;
    return or_apply_dims(psi, dims, n, targets, k, U);
}

/* ------------------------------------------------------------------------- */
/* Reductions (serial, plain summation in index order).                      */
/* ------------------------------------------------------------------------- */

/* Squared norm sum_i |psi_i|^2. */
double or_norm2(const cplx *psi, long long N)
{
    double s = 0.0;
    for (long long i = 0; i < N; ++i) s += creal(psi[i]) * creal(psi[i]) + cimag(psi[i]) * cimag(psi[i]);
    return s;
}

/* <N_q> = sum_i i_q |psi_i|^2 for every qudit q, with N = diag(0, 1, ..., d_q-1)
 * the level-number observable and i_q the q-th (mixed-radix) digit of i
 * ("Generalized CNOT gate", decimal representation).  out has n entries. */
void or_expect_number_dims(const cplx *psi, const int *dims, int n, double *out)
{
    long long N = 1;
    for (int q = 0; q < n; ++q) N *= dims[q];
    for (int q = 0; q < n; ++q) out[q] = 0.0;
    for (long long i = 0; i < N; ++i) {
        double p = creal(psi[i]) * creal(psi[i]) + cimag(psi[i]) * cimag(psi[i]);
        long long rem = i;
        for (int q = n - 1; q >= 0; --q) {
            out[q] += (double)(rem % dims[q]) * p;
            rem /= dims[q];
        }
    }
}

void or_expect_number(const cplx *psi, int d, int n, double *out)
{
    int dims[64];
    for (int q = 0; q < n && q < 64; ++q) dims[q] = d;
    or_expect_number_dims(psi, dims, n, out);
}

/* <psi| O_q |psi> for a dims[q] x dims[q] matrix O on qudit q (complex
 * result; real for Hermitian O). */
void or_expect_obs_dims(const cplx *psi, const int *dims, int n, int q, const cplx *O, double *out_re, double *out_im)
{
    long long N = 1, S = 1;
    for (int p = 0; p < n; ++p) N *= dims[p];
    for (int p = q + 1; p < n; ++p) S *= dims[p];
    int d = dims[q];
    cplx acc = 0.0;
    for (long long i = 0; i < N; ++i) {
        long long l = (i / S) % d;
        long long base = i - l * S;
        cplx row = 0.0;
        for (int m = 0; m < d; ++m) row += O[l * d + m] * psi[base + m * S];
        acc += conj(psi[i]) * row;
    }
    *out_re = creal(acc);
    *out_im = cimag(acc);
}

void or_expect_obs(const cplx *psi, int d, int n, int q, const cplx *O, double *out_re, double *out_im)
{
    int dims[64];
    for (int p = 0; p < n && p < 64; ++p) dims[p] = d;
    or_expect_obs_dims(psi, dims, n, q, O, out_re, out_im);
}

/* Marginal probabilities of the qudits listed in idx (k of them):
 * out[r] = sum over i whose digits on idx[0..k-1] spell r (idx[0] most
 * significant, mixed radix over dims[idx[a]]) of |psi_i|^2.  out has
 * prod_a dims[idx[a]] entries. */
void or_marginal_dims(const cplx *psi, const int *dims, int n, const int *idx, int k, double *out)
{
    long long N = 1, K = 1;
    long long stride[64];
    for (int q = n - 1; q >= 0; --q) {
        stride[q] = N;
        N *= dims[q];
    }
    for (int a = 0; a < k; ++a) K *= dims[idx[a]];
    for (long long r = 0; r < K; ++r) out[r] = 0.0;
    for (long long i = 0; i < N; ++i) {
        double p = creal(psi[i]) * creal(psi[i]) + cimag(psi[i]) * cimag(psi[i]);
        long long r = 0;
        for (int a = 0; a < k; ++a) r = r * dims[idx[a]] + (i / stride[idx[a]]) % dims[idx[a]];
        out[r] += p;
    }
}

void or_marginal(const cplx *psi, int d, int n, const int *idx, int k, double *out)
{
    int dims[64];
    for (int q = 0; q < n && q < 64; ++q) dims[q] = d;
    or_marginal_dims(psi, dims, n, idx, k, out);
}

/* <a|b> = sum_i conj(a_i) b_i. */
void or_inner(const cplx *a, const cplx *b, long long N, double *out_re, double *out_im)
{
    cplx acc = 0.0;
    for (long long i = 0; i < N; ++i) acc += conj(a[i]) * b[i];
    *out_re = creal(acc);
    *out_im = cimag(acc);
}

/* psi = |index>  (the basis state whose decimal representation is index). */
void or_basis_state(cplx *psi, long long N, long long index)
{
    for (long long i = 0; i < N; ++i) psi[i] = 0.0;
    psi[index] = 1.0;
}

/* Host threads the OpenMP loops use (the CPU baseline times the oracle on
 * all host cores and on one); no arithmetic changes with the count. */
void or_set_threads(int t)
{
    omp_set_num_threads(t > 0 ? t : 1);
}

int or_get_threads(void)
{
    return omp_get_max_threads();
}
