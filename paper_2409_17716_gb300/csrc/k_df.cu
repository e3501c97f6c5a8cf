// k_df.cu -- complex128 states in double-float form for the compiled passes.
//
// GB300 runs FP64 at about 1/73 of its FP32 rate (measured: 1.05 TFLOP/s of
// FP64 FMA against 76.8 TFLOP/s of FP32 FMA), and the complex128 gate
// arithmetic of a fused pass is bound by it.  The compiled passes therefore
// compute complex128 programs in double-float arithmetic: every real number
// is an unevaluated sum hi + lo of two floats (T. J. Dekker, "A
// floating-point technique for extending the available precision", Numer.
// Math. 18, 1971), with products split exactly by a fused multiply-add and
// sums by Knuth's TwoSum (D. E. Knuth, TAOCP vol. 2, sec. 4.2.2), about 48
// significant bits.  A double2 amplitude (16 bytes) and its double-float form
// (hi.re, hi.im, lo.re, lo.im as float4, 16 bytes) occupy the same bytes, so a
// program run converts the state in place once before its first compiled pass
// and back after its last one.  The conversions use integer operations only:
// conversions between FP32 and FP64 run at the FP64 rate on this GPU, and
// these kernels stay bound by HBM.
//
// Range: |x| must be below 2^128 (every amplitude of a state of norm <= 2^64
// is); finite magnitudes below 2^-126 become 0 (an absolute error below 1.2e-38).
#include "qf_host.h"

namespace qf {

// hi + lo for one double: hi = x with its mantissa cut to 24 bits, lo = the
// remaining 29 bits rounded to a float (so hi + lo = x within 2^-48 |x|).
__device__ __forceinline__ float2 df_split(double x) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(x);
    const unsigned sign = (unsigned)(u >> 32) & 0x80000000u;
    const int E = (int)((u >> 52) & 0x7ff) - 1023;
    const unsigned long long m = u & 0xfffffffffffffull;
    if (E < -126) return make_float2(0.0f, 0.0f);
    if (E > 127) return make_float2(__uint_as_float(sign | 0x7f800000u), 0.0f);   // beyond float: infinite
    const float hi = __uint_as_float(sign | ((unsigned)(E + 127) << 23) | (unsigned)(m >> 29));
    float lo = 0.0f;
    if (E >= -74) lo = __uint2float_rn((unsigned)(m & 0x1fffffffull)) * __uint_as_float((unsigned)(E - 52 + 127) << 23);
    return make_float2(hi, sign ? -lo : lo);
}

// The double nearest to hi + lo (|lo| below one float ulp of hi, as every
// renormalized pair is): both significands as integers in units of 2^-52 of
// hi's binade, one integer add, one normalization step, round to nearest.
__device__ __forceinline__ double df_join(float hi, float lo) {
    const unsigned hb = __float_as_uint(hi), lb = __float_as_uint(lo);
    const int eh = (int)((hb >> 23) & 0xff), el = (int)((lb >> 23) & 0xff);
    if (eh == 0) {   // hi is zero: lo alone (zero too when hi was)
        if (el == 0) return 0.0;
        const unsigned long long bits = ((unsigned long long)(lb >> 31) << 63) |
                                        ((unsigned long long)(el - 127 + 1023) << 52) |
                                        ((unsigned long long)(lb & 0x7fffffu) << 29);
        return __longlong_as_double((long long)bits);
    }
    long long S = (long long)((hb & 0x7fffffu) | 0x800000u) << 29;   // 2^52 <= S < 2^53
    if (hb >> 31) S = -S;
    if (el != 0) {
        const long long ml = (long long)((lb & 0x7fffffu) | 0x800000u);
        const int sh = el - eh + 29;
        long long Ml = 0;
        if (sh >= 0) Ml = ml << (sh < 30 ? sh : 30);
        else if (sh > -40) Ml = (ml + (1ll << (-sh - 1))) >> (-sh);
        S += (lb >> 31) ? -Ml : Ml;
    }
    unsigned long long sign = 0;
    if (S < 0) {
        sign = 1ull << 63;
        S = -S;
    }
    if (S == 0) return 0.0;
    int e = eh - 127 + 1023;
    while (S >= (1ll << 53)) {
        S = (S + 1) >> 1;
        ++e;
    }
    while (S < (1ll << 52)) {
        S <<= 1;
        --e;
    }
    return __longlong_as_double((long long)(sign | ((unsigned long long)e << 52) | ((unsigned long long)S & 0xfffffffffffffull)));
}

__global__ void __launch_bounds__(256) k_df_pack(double2 *psi, long long N) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        const double2 v = psi[i];
        const float2 r = df_split(v.x), m = df_split(v.y);
        reinterpret_cast<float4 *>(psi)[i] = make_float4(r.x, m.x, r.y, m.y);
    }
}

__global__ void __launch_bounds__(256) k_df_unpack(double2 *psi, long long N) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        const float4 v = reinterpret_cast<const float4 *>(psi)[i];
        psi[i] = make_double2(df_join(v.x, v.z), df_join(v.y, v.w));
    }
}

cudaError_t launch_df_convert(cudaStream_t stream, int num_sms, void *psi, long long N, bool pack) {
    long long blocks = (N + 255) / 256;
    const long long cap = (long long)num_sms * 8;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    if (pack) k_df_pack<<<(unsigned)blocks, 256, 0, stream>>>(reinterpret_cast<double2 *>(psi), N);
    else k_df_unpack<<<(unsigned)blocks, 256, 0, stream>>>(reinterpret_cast<double2 *>(psi), N);
    return cudaGetLastError();
}

}  // namespace qf
