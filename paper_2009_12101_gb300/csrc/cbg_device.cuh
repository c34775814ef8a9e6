// cbg_device.cuh -- device building blocks of the compressed-basis GMRES kernels.
//
// * double-float ("DF32") arithmetic: a value is an unevaluated pair hi + lo of FP32
//   numbers; products use the FMA error-free product, sums use Knuth's TwoSum.  Every
//   operation that must be rounded exactly once is written with the _rn intrinsics so
//   the compiler cannot contract it into an FMA.
// * the basis accessor (Section 4.2): encode an FP64 value into the storage format and
//   decode 16 bytes of codes into values that are exact in FP32 (or an exact FP32 pair
//   for f64 and int32 codes).
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace cbg {

enum Format { F64 = 0, F32 = 1, F16 = 2, BF16 = 3, E4M3 = 4, I32 = 5, I16 = 6 };

template <int FMT> struct FmtInfo;
template <> struct FmtInfo<F64> { static constexpr int bytes = 8; };
template <> struct FmtInfo<F32> { static constexpr int bytes = 4; };
template <> struct FmtInfo<F16> { static constexpr int bytes = 2; };
template <> struct FmtInfo<BF16> { static constexpr int bytes = 2; };
template <> struct FmtInfo<E4M3> { static constexpr int bytes = 1; };
template <> struct FmtInfo<I32> { static constexpr int bytes = 4; };
template <> struct FmtInfo<I16> { static constexpr int bytes = 2; };

// formats whose decoded code is exact in a single FP32 (else an exact FP32 pair)
template <int FMT> struct SingleFloat { static constexpr bool value = !(FMT == F64 || FMT == I32); };

// ------------------------------------------------------------------ double-float (DF32)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e)
{
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e)
{  // requires |a| >= |b| (or a == 0)
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}

// acc (S + C) += v * (wh + wl), v exact FP32.  p + pe equals v*(wh+wl) up to the
// rounding of v*wl (relative 2^-24 of a term already 2^-24 smaller than the product).
__device__ __forceinline__ void df_mac(float& S, float& C, float v, float wh, float wl)
{
    float p = __fmul_rn(v, wh);
    float pe = __fmaf_rn(v, wh, -p);
    pe = __fmaf_rn(v, wl, pe);
    float s, e;
    two_sum(S, p, s, e);
    C = __fadd_rn(C, __fadd_rn(e, pe));
    S = s;
}

// acc += (vh + vl) * (wh + wl) for a value that needs an FP32 pair (f64, int32 codes)
__device__ __forceinline__ void df_mac2(float& S, float& C, float vh, float vl, float wh,
                                        float wl)
{
    float p = __fmul_rn(vh, wh);
    float pe = __fmaf_rn(vh, wh, -p);
    pe = __fmaf_rn(vh, wl, pe);
    pe = __fmaf_rn(vl, wh, pe);
    float s, e;
    two_sum(S, p, s, e);
    C = __fadd_rn(C, __fadd_rn(e, pe));
    S = s;
}

__device__ __forceinline__ void df_renorm(float& S, float& C)
{
    float s, e;
    fast_two_sum(S, C, s, e);
    S = s;
    C = e;
}

// ---- the same operations on two independent accumulations at once, on the packed
// FP32x2 pipe of sm_100-class GPUs (one instruction per pair).  Subtractions are written
// as FMAs with a -1 multiplier, which round exactly like the subtraction, so every
// component is bitwise identical to the scalar routine above.
__device__ __forceinline__ float2 f2_neg1() { return make_float2(-1.f, -1.f); }

// (S + C) += v * (wh + wl) per component; nwh = -wh, v exact FP32
__device__ __forceinline__ void df2_mac(float2& S, float2& C, float2 v, float2 wh, float2 nwh, float2 wl)
{
    const float2 m1 = f2_neg1();
    const float2 np = __fmul2_rn(v, nwh);           // -p, p = RN(v*wh)
    float2 pe = __ffma2_rn(v, wh, np);              // v*wh - p, exact
    pe = __ffma2_rn(v, wl, pe);
    const float2 s = __ffma2_rn(np, m1, S);         // TwoSum(S, p): s = S + p
    const float2 bb = __ffma2_rn(S, m1, s);         // s - S
    const float2 t1 = __ffma2_rn(bb, m1, s);        // s - bb
    const float2 t2 = __ffma2_rn(t1, m1, S);        // S - (s - bb)
    const float2 u = __fadd2_rn(np, bb);            // -(p - bb)
    const float2 e = __ffma2_rn(u, m1, t2);         // t2 + (p - bb)
    C = __fadd2_rn(C, __fadd2_rn(e, pe));
    S = s;
}

// (S + C) += (vh + vl) * (wh + wl) per component, for codes that need an FP32 pair
__device__ __forceinline__ void df2_mac2(float2& S, float2& C, float2 vh, float2 vl, float2 wh, float2 nwh,
                                         float2 wl)
{
    const float2 m1 = f2_neg1();
    const float2 np = __fmul2_rn(vh, nwh);
    float2 pe = __ffma2_rn(vh, wh, np);
    pe = __ffma2_rn(vh, wl, pe);
    pe = __ffma2_rn(vl, wh, pe);
    const float2 s = __ffma2_rn(np, m1, S);
    const float2 bb = __ffma2_rn(S, m1, s);
    const float2 t1 = __ffma2_rn(bb, m1, s);
    const float2 t2 = __ffma2_rn(t1, m1, S);
    const float2 u = __fadd2_rn(np, bb);
    const float2 e = __ffma2_rn(u, m1, t2);
    C = __fadd2_rn(C, __fadd2_rn(e, pe));
    S = s;
}

__device__ __forceinline__ void df2_renorm(float2& S, float2& C)
{
    const float2 m1 = f2_neg1();
    const float2 s = __fadd2_rn(S, C);
    const float2 d = __ffma2_rn(S, m1, s);          // s - S
    C = __ffma2_rn(d, m1, C);                       // C - (s - S)
    S = s;
}

// (aS + aC) += (bS + bC)
__device__ __forceinline__ void df_add(float& aS, float& aC, float bS, float bC)
{
    float s, e;
    two_sum(aS, bS, s, e);
    e = __fadd_rn(e, __fadd_rn(aC, bC));
    fast_two_sum(s, e, aS, aC);
}

// The hardware conversions between FP32 and FP64 run on GB300's narrow FP64 pipe.  The
// helpers below convert in integer operations and keep the hardware instruction only
// for rare inputs, behind a call that the compiler cannot turn into predicated code
// (a predicated-off FP64-pipe instruction still occupies the pipe).
static __device__ __noinline__ float f64_to_f32_hw(double x) { return __double2float_rn(x); }

// Split an FP64 value into hi + lo FP32 with integer operations only (the FP64 pipe of
// GB300 is ~70x slower than FP32).  hi = x truncated to 24 significant bits (exact),
// lo = the remaining 29 significand bits rounded to 24 bits, so hi + lo = x with a
// relative error below 2^-48.  |x| < 2^-74 keeps only hi (absolute error < 2^-98);
// |x| < 2^-126, |x| >= 2^128, Inf and NaN go through the exact FP64->FP32 conversion.
__device__ __forceinline__ void split_f64(double x, float& hi, float& lo)
{
    unsigned long long u = (unsigned long long)__double_as_longlong(x);
    unsigned int uh = (unsigned int)(u >> 32), ul = (unsigned int)u;
    unsigned int e = (uh >> 20) & 0x7FFu;
    unsigned int sign = uh & 0x80000000u;
    if (e - 897u <= 253u) {  // 897 <= e <= 1150: hi is a normal float
        unsigned int hb = __funnelshift_l(ul, uh, 3);              // low 9 exponent bits + 23 mantissa bits
        hb = ((hb - (384u << 23)) & 0x7FFFFFFFu) | sign;            // rebias 1023 -> 127
        hi = __uint_as_float(hb);
        unsigned int r = ul & 0x1FFFFFFFu;                          // remaining 29 bits
        if (e >= 949u && r != 0u) {
            float rf = __uint2float_rn(r);                          // <= 2^-24 relative
            float sc = __uint_as_float((e - 948u) << 23);           // 2^(e - 1075)
            lo = __uint_as_float(__float_as_uint(__fmul_rn(rf, sc)) | sign);
        } else {
            lo = 0.0f;
        }
    } else if (e == 0u) {
        hi = __uint_as_float(sign);
        lo = 0.0f;
    } else {
        hi = f64_to_f32_hw(x);
        lo = 0.0f;
    }
}

// Exact FP32 -> FP64 conversion, every input in integer operations (normal numbers,
// zeros, subnormals normalised with a leading-zero count, infinities and NaNs).
__device__ __forceinline__ double f32_to_f64_exact(float f)
{
    const unsigned int u = __float_as_uint(f);
    const unsigned int sign = u & 0x80000000u, e = (u >> 23) & 0xFFu, m = u & 0x7FFFFFu;
    unsigned int hi, lo;
    if (e - 1u < 254u) {                       // normal
        hi = sign | ((e + 896u) << 20) | (m >> 3);
        lo = (m & 7u) << 29;
    } else if (e == 255u) {                    // infinity, NaN (payload kept)
        hi = sign | 0x7FF00000u | (m >> 3);
        lo = (m & 7u) << 29;
    } else if (m == 0u) {                      // zero
        hi = sign;
        lo = 0u;
    } else {                                   // subnormal m * 2^-149: leading one to bit 23
        const unsigned int sh = (unsigned int)__clz(m) - 8u;
        const unsigned int mn = (m << sh) & 0x7FFFFFu;
        hi = sign | ((897u - sh) << 20) | (mn >> 3);
        lo = (mn & 7u) << 29;
    }
    return __hiloint2double((int)hi, (int)lo);
}

// FP64 -> FP32 with round-to-nearest-even, in integer operations when the result is a
// normal float or zero (the FP64->FP32 conversion instruction runs on GB300's narrow FP64
// pipe); subnormal results, overflow, Inf and NaN take the hardware conversion.  A carry
// out of the rounded significand moves into the exponent, as IEEE rounding does.
__device__ __forceinline__ float f64_to_f32_rn(double x)
{
    const unsigned long long u = (unsigned long long)__double_as_longlong(x);
    const unsigned int sign = (unsigned int)(u >> 32) & 0x80000000u;
    const unsigned int e = (unsigned int)(u >> 52) & 0x7FFu;
    if (e - 897u <= 253u) {                                    // 897 <= e <= 1150
        const unsigned long long m = u & 0xFFFFFFFFFFFFFull;   // 52 fraction bits
        unsigned int b = ((e - 896u) << 23) | (unsigned int)(m >> 29);
        const unsigned int rem = (unsigned int)m & 0x1FFFFFFFu, half = 0x10000000u;
        b += (rem > half || (rem == half && (b & 1u))) ? 1u : 0u;
        return __uint_as_float(b | sign);
    }
    if ((u << 1) == 0ull) return __uint_as_float(sign);       // +-0
    return f64_to_f32_hw(x);
}

// hi + lo rounded once to FP64: both widened exactly with integer operations, then one
// FP64 addition
__device__ __forceinline__ double df_to_double(float hi, float lo)
{
    return __dadd_rn(f32_to_f64_exact(hi), f32_to_f64_exact(lo));
}

// ------------------------------------------------------------------------- decoding
// Exact conversions of codes to FP32.  The per-vector scale is applied by the caller
// (once per column in a dot product, folded into the coefficient in an axpy).
__device__ __forceinline__ float dec_f16(unsigned int h16)
{
    return __half2float(__ushort_as_half((unsigned short)h16));
}
__device__ __forceinline__ float dec_bf16(unsigned int b16) { return __uint_as_float(b16 << 16); }
__device__ __forceinline__ float dec_i16(int q)
{   // exact for |q| < 2^22: the code lands in the mantissa of 1.5 * 2^23
    return __fsub_rn(__int_as_float(0x4B400000 + q), 12582912.0f);
}
__device__ __forceinline__ void dec_i32(int q, float& hi, float& lo)
{   // hi = q truncated to its top 24 significant bits (exact float), lo = q - hi
    // (an integer below 2^7 in magnitude, exact), so |lo| < 2^-23 |hi|
    hi = __int2float_rz(q);
    lo = dec_i16(q - __float2int_rz(hi));
}

// decode two e4m3 codes (low 16 bits of `pair`) into FP32 via the exact e4m3 -> f16 path
__device__ __forceinline__ void dec_e4m3x2(unsigned int pair, float& a, float& b)
{
    __half2_raw h2 = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(pair & 0xFFFFu), __NV_E4M3);
    __half2 hv = *reinterpret_cast<__half2*>(&h2);
    float2 f = __half22float2(hv);
    a = f.x;
    b = f.y;
}

// Decoded element of a 16-byte chunk.  For single-float formats vh is the exact value
// (without the per-vector scale) and vl = 0.
template <int FMT> struct Chunk {
    static constexpr int E = 16 / FmtInfo<FMT>::bytes;
    float vh[E];
    float vl[SingleFloat<FMT>::value ? 1 : E];
};

template <int FMT> __device__ __forceinline__ void decode_chunk(const uint4& raw, Chunk<FMT>& c)
{
    const unsigned int w[4] = {raw.x, raw.y, raw.z, raw.w};
    if constexpr (FMT == F64) {
        double d0 = __hiloint2double((int)w[1], (int)w[0]);
        double d1 = __hiloint2double((int)w[3], (int)w[2]);
        split_f64(d0, c.vh[0], c.vl[0]);
        split_f64(d1, c.vh[1], c.vl[1]);
    } else if constexpr (FMT == F32) {
#pragma unroll
        for (int k = 0; k < 4; k++) c.vh[k] = __uint_as_float(w[k]);
    } else if constexpr (FMT == F16) {
#pragma unroll
        for (int k = 0; k < 4; k++) {
            c.vh[2 * k] = dec_f16(w[k] & 0xFFFFu);
            c.vh[2 * k + 1] = dec_f16(w[k] >> 16);
        }
    } else if constexpr (FMT == BF16) {
#pragma unroll
        for (int k = 0; k < 4; k++) {
            c.vh[2 * k] = __uint_as_float(w[k] << 16);
            c.vh[2 * k + 1] = __uint_as_float(w[k] & 0xFFFF0000u);
        }
    } else if constexpr (FMT == E4M3) {
#pragma unroll
        for (int k = 0; k < 4; k++) {
            dec_e4m3x2(w[k] & 0xFFFFu, c.vh[4 * k], c.vh[4 * k + 1]);
            dec_e4m3x2(w[k] >> 16, c.vh[4 * k + 2], c.vh[4 * k + 3]);
        }
    } else if constexpr (FMT == I32) {
#pragma unroll
        for (int k = 0; k < 4; k++) dec_i32((int)w[k], c.vh[k], c.vl[k]);
    } else if constexpr (FMT == I16) {
#pragma unroll
        for (int k = 0; k < 4; k++) {
            c.vh[2 * k] = dec_i16((int)(short)(w[k] & 0xFFFFu));
            c.vh[2 * k + 1] = dec_i16((int)w[k] >> 16);
        }
    }
}

// Exact FP64 value of one code (scale not applied); used by the FP64 arithmetic mode,
// the SpMV and the decode kernel.
template <int FMT> __device__ __forceinline__ double code_value(const void* base, int64_t i)
{
    if constexpr (FMT == F64) return reinterpret_cast<const double*>(base)[i];
    else if constexpr (FMT == F32) return f32_to_f64_exact(reinterpret_cast<const float*>(base)[i]);
    else if constexpr (FMT == F16) return f32_to_f64_exact(__half2float(reinterpret_cast<const __half*>(base)[i]));
    else if constexpr (FMT == BF16)
        return f32_to_f64_exact(__uint_as_float(((unsigned int)reinterpret_cast<const unsigned short*>(base)[i]) << 16));
    else if constexpr (FMT == E4M3) {
        unsigned int c = reinterpret_cast<const unsigned char*>(base)[i];
        float a, b;
        dec_e4m3x2(c, a, b);
        return f32_to_f64_exact(a);
    } else if constexpr (FMT == I32) {
        float hi, lo;
        dec_i32(reinterpret_cast<const int*>(base)[i], hi, lo);   // both parts exact
        return __dadd_rn(f32_to_f64_exact(hi), f32_to_f64_exact(lo));
    } else return f32_to_f64_exact(dec_i16((int)reinterpret_cast<const short*>(base)[i]));
}

// One code (or FP64 vector entry) as an FP32 pair with x = xh + xl: exact for every
// format except FP64 vectors and f64 codes (relative error below 2^-48 there).
template <int XFMT> __device__ __forceinline__ void xval_df(const void* x, int c, float& xh, float& xl)
{
    if constexpr (XFMT < 0 || XFMT == F64) {
        split_f64(reinterpret_cast<const double*>(x)[c], xh, xl);
    } else if constexpr (XFMT == I32) {
        dec_i32(reinterpret_cast<const int*>(x)[c], xh, xl);
    } else {
        if constexpr (XFMT == F32) xh = reinterpret_cast<const float*>(x)[c];
        else if constexpr (XFMT == F16) xh = __half2float(reinterpret_cast<const __half*>(x)[c]);
        else if constexpr (XFMT == BF16)
            xh = __uint_as_float(((unsigned int)reinterpret_cast<const unsigned short*>(x)[c]) << 16);
        else if constexpr (XFMT == E4M3) {
            float b;
            dec_e4m3x2(reinterpret_cast<const unsigned char*>(x)[c], xh, b);
        } else xh = dec_i16((int)reinterpret_cast<const short*>(x)[c]);
        xl = 0.f;
    }
}

// ------------------------------------------------------------------------- encoding
// Per-vector encode parameters, computed once from vmax = max_i |v_i| (Section 4.2 and
// the bf16/e4m3 power-of-two scale).  `scale` is what decoding multiplies by.
struct EncParams {
    double scale;     // sigma (int), 2^e (bf16/e4m3), 1 otherwise
    double inv;       // 1/sigma (int) or 2^-e (bf16/e4m3)
};

// 2^e as an FP64 value built from its bits, for |e| <= 1022
__device__ __forceinline__ double pow2d(int e) { return __longlong_as_double((long long)(1023 + e) << 52); }

__host__ __device__ inline int pow2_exponent_for(double vmax, double fmax)
{   // smallest integer e with vmax <= fmax * 2^e, at least -126
    int e2;
    (void)frexp(vmax, &e2);
    int e = e2 - 12;
    while (vmax > ldexp(fmax, e)) e += 1;
    if (e < -126) e = -126;
    return e;
}

__host__ __device__ inline EncParams enc_params(int fmt, double vmax)
{
    EncParams p{1.0, 1.0};
    if (!(vmax > 0.0)) vmax = 1.0;
    if (fmt == I32 || fmt == I16) {
        double mx = fmt == I32 ? 2147483647.0 : 32767.0;
        p.scale = vmax / mx;
        p.inv = 1.0 / p.scale;
    } else if (fmt == BF16 || fmt == E4M3) {
        int e = pow2_exponent_for(vmax, fmt == BF16 ? 1.0 : 448.0);
        p.scale = ldexp(1.0, e);
        p.inv = ldexp(1.0, -e);
    }
    return p;
}

// Store v (normalised FP64 value) at position i of the code array.
template <int FMT> __device__ __forceinline__ void encode_store(void* base, int64_t i, double v,
                                                               const EncParams& p)
{
    if constexpr (FMT == F64) {
        reinterpret_cast<double*>(base)[i] = v;
    } else if constexpr (FMT == F32) {
        reinterpret_cast<float*>(base)[i] = f64_to_f32_rn(v);
    } else if constexpr (FMT == F16) {
        reinterpret_cast<__half*>(base)[i] = __double2half(v);
    } else if constexpr (FMT == I32 || FMT == I16) {
        const int mx = FMT == I32 ? 2147483647 : 32767;
        double t = __dmul_rn(v, p.inv);
        double mxd = (double)mx;
        t = t > mxd ? mxd : (t < -mxd ? -mxd : t);
        int q = __double2int_rn(t);
        if constexpr (FMT == I32) reinterpret_cast<int*>(base)[i] = q;
        else reinterpret_cast<short*>(base)[i] = (short)q;
    } else if constexpr (FMT == BF16) {
        float f = f64_to_f32_rn(__dmul_rn(v, p.inv));
        __nv_bfloat16 b = __float2bfloat16_rn(f);
        reinterpret_cast<__nv_bfloat16*>(base)[i] = b;
    } else if constexpr (FMT == E4M3) {
        float f = f64_to_f32_rn(__dmul_rn(v, p.inv));
        reinterpret_cast<unsigned char*>(base)[i] =
            (unsigned char)__nv_cvt_float_to_fp8(f, __NV_SATFINITE, __NV_E4M3);
    }
}

// ------------------------------------------------------------------- memory helpers
__device__ __forceinline__ uint4 ldg_stream(const void* p)
{   // read-only streaming load, do not keep in L1
    uint4 r;
    asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
                 : "l"(p));
    return r;
}

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    return v;
}

__device__ __forceinline__ double warp_max(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xFFFFFFFFu, v, o));
    return v;
}

// maximum of non-negative doubles over the warp, compared as bit patterns with 32-bit
// integer operations (no FP64 instruction: GB300's FP64 pipe is narrow and slow)
__device__ __forceinline__ double warp_max_nonneg(double v)
{
    unsigned int hi = (unsigned int)__double2hiint(v), lo = (unsigned int)__double2loint(v);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned int h2 = __shfl_xor_sync(0xFFFFFFFFu, hi, o), l2 = __shfl_xor_sync(0xFFFFFFFFu, lo, o);
        if (h2 > hi || (h2 == hi && l2 > lo)) {
            hi = h2;
            lo = l2;
        }
    }
    return __hiloint2double((int)hi, (int)lo);
}

// The block's sum of the threads' ss and maximum of their mx (mx >= 0): a shuffle tree in
// every warp, then warp 0 folds the warps' results with a second tree (five dependent
// FP64 additions instead of one per warp).  red_s, red_m: shared, blockDim.x / 32 entries.
// All threads call it; the totals are valid in warp 0.
__device__ __forceinline__ void block_sum_max(double ss, double mx, double* red_s, double* red_m, double& s,
                                              double& m)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    ss = warp_sum(ss);
    mx = warp_max_nonneg(mx);
    if (lane == 0) {
        red_s[warp] = ss;
        red_m[warp] = mx;
    }
    __syncthreads();
    s = 0.0;
    m = 0.0;
    if (warp == 0) {                 // a tree over the first pow2 >= nw lanes only
        s = lane < nw ? red_s[lane] : 0.0;
        m = lane < nw ? red_m[lane] : 0.0;
        unsigned int hi = (unsigned int)__double2hiint(m), lo = (unsigned int)__double2loint(m);
        for (int o = 16; o > 0; o >>= 1) {
            if (o >= nw) continue;   // lanes >= nw hold zeros: nothing to fold from there
            s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
            const unsigned int h2 = __shfl_xor_sync(0xFFFFFFFFu, hi, o), l2 = __shfl_xor_sync(0xFFFFFFFFu, lo, o);
            if (h2 > hi || (h2 == hi && l2 > lo)) {
                hi = h2;
                lo = l2;
            }
        }
        m = __hiloint2double((int)hi, (int)lo);
    }
}

}  // namespace cbg
