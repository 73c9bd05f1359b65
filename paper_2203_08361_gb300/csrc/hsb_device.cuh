// hsb_device.cuh -- device helpers shared by the kernels of libhsb: the
// counter-based initial-state generator, the FP8 sign encoding and the fused
// spin update of the Methods section.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "hsb_internal.cuh"

namespace hsb {

// FP8 e4m3 encodings of +1 and -1 (sign 0/1, biased exponent 7, mantissa 0).
constexpr uint8_t kFp8PlusOne = 0x38;
constexpr uint8_t kFp8MinusOne = 0xB8;

// SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): output number n (n >= 1) of
// the generator started from `state` is the finaliser of state + n * GAMMA.
__device__ __forceinline__ uint64_t splitmix64_out(uint64_t state, uint64_t n)
{
    uint64_t z = state + n * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

// Uniform value in (-L, L): draw u = output (1 + r*2^32 + 2i + comp) of the
// instance stream, m = top 24 bits, value = fl32((2m + 1 - 2^24) * scale)
// with scale = fl32(L * 2^-24).  2m + 1 - 2^24 is an odd integer below 2^24
// in magnitude, exact in binary32, so the value takes one rounding.
__device__ __forceinline__ float init_uniform(uint64_t s_inst, uint32_t r, uint32_t i, int comp,
                                              float scale)
{
    const uint64_t n = 1u + ((uint64_t)r << 32) + 2u * (uint64_t)i + (uint64_t)comp;
    const uint64_t u = splitmix64_out(s_inst, n);
    const int m = (int)(u >> 40);
    const float v = (float)(2 * m + 1 - 16777216);
    return __fmul_rn(v, scale);
}

// e2m1 (FP4) codes of +1 and -1 (sign 0/1, exponent 01, mantissa 0), packed
// two per byte with the even index in the low nibble; 0 is 0x0.
constexpr uint32_t kFp4PlusOne = 0x2;
constexpr uint32_t kFp4MinusOne = 0xA;

// sgn(x) as an FP8 byte; +1 for x >= 0 (including -0.0).
__device__ __forceinline__ uint8_t fp8_sign(float x)
{
    return x >= 0.f ? kFp8PlusOne : kFp8MinusOne;
}

// ---- bit spreading for the sign codes (host and device) --------------------
// bit k of b (k < 4) to bit 8k: one bit per byte (the four partial products
// of the multiplication occupy distinct bits, so nothing carries)
__host__ __device__ __forceinline__ uint32_t spread4_bytes(uint32_t b)
{
    return ((b & 0xFu) * 0x00204081u) & 0x01010101u;
}

// bit k of b (k < 8) to bit 4k: one bit per nibble
__host__ __device__ __forceinline__ uint32_t spread8_nibbles(uint32_t b)
{
    uint32_t x = b & 0xFFu;
    x = (x | (x << 12)) & 0x000F000Fu;
    x = (x | (x << 6)) & 0x03030303u;
    return (x | (x << 3)) & 0x11111111u;
}

// 0xFF in byte i of the result for each set bit i (i < 4) of b, else 0x00
__host__ __device__ __forceinline__ uint32_t byte_mask4(uint32_t b)
{
    return spread4_bytes(b) * 0xFFu;
}

// 0xF in nibble i of the result for each set bit i (i < 8) of b, else 0x0
__host__ __device__ __forceinline__ uint32_t nibble_mask8(uint32_t b)
{
    return spread8_nibbles(b) * 0xFu;
}

// One spin update (Methods):
//   y~  = y + {-(a0 - a(t_k)) x + c0 f} dt        Eq. (eq_SyEuY)
//   x~  = x + a0 y~ dt                             Eq. (eq_SyEuX)
//   x'  = g(x~), y~~ = h(x~, y~)                   Eqs. (eq_WallX), (eq_WallY)
//   y'  = y~~ + gamma y(t_k) dt                    Eq. (eq_EuHeat)
// Every operation is one binary32 rounding in this fixed order (no fused
// multiply-add): u = c0 f; v = p_k x; w = u - v; yt = y + w dt; xt = x + q yt;
// walls (strict |x~| > 1); y' = ytt + g y(t_k).
__device__ __forceinline__ void sb_update(float f, float x0, float y0, float pk,
                                          const StepConsts &c, float &xn, float &yn)
{
    const float u = __fmul_rn(c.c0, f);
    const float v = __fmul_rn(pk, x0);
    const float w = __fsub_rn(u, v);
    const float wd = __fmul_rn(w, c.dt);
    const float yt = __fadd_rn(y0, wd);
    const float qy = __fmul_rn(c.q, yt);
    const float xt = __fadd_rn(x0, qy);
    float ytt = yt;
    xn = xt;
    if (xt > 1.f) {
        xn = 1.f;
        ytt = 0.f;
    } else if (xt < -1.f) {
        xn = -1.f;
        ytt = 0.f;
    }
    const float gy = __fmul_rn(c.g, y0);
    yn = __fadd_rn(ytt, gy);
}

// ---- two updates at once on packed binary32 pairs (lo, hi) -----------------
// The arithmetic uses add/sub/fma.rn.f32x2 and gives the same bits as two
// sb_update calls.  Each product a*b is computed as fma(a, b, z) with z = -0.0
// supplied at run time (StepConsts::nz): the sum is exactly a*b for every
// product (a zero product keeps its sign), rounded once, and because z is not
// a compile-time constant the compiler cannot turn the product back into a
// multiply and fuse it into the following add, which it does for plain
// mul/add.rn.f32x2 pairs.

__device__ __forceinline__ uint64_t f2_pack(float lo, float hi)
{
    return ((uint64_t)__float_as_uint(hi) << 32) | __float_as_uint(lo);
}
__device__ __forceinline__ uint64_t f2_pack_bits(uint32_t lo, uint32_t hi)
{
    return ((uint64_t)hi << 32) | lo;
}
__device__ __forceinline__ float f2_lo(uint64_t v) { return __uint_as_float((uint32_t)v); }
__device__ __forceinline__ float f2_hi(uint64_t v) { return __uint_as_float((uint32_t)(v >> 32)); }

__device__ __forceinline__ uint64_t f2_fma(uint64_t a, uint64_t b, uint64_t c)
{
    uint64_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ uint64_t f2_add(uint64_t a, uint64_t b)
{
    uint64_t d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ uint64_t f2_sub(uint64_t a, uint64_t b)
{
    uint64_t d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// StepConsts broadcast to both halves of a pair.
struct StepConsts2 {
    uint64_t c0, dt, q, g, z;
};

__device__ __forceinline__ StepConsts2 step_consts2(const StepConsts &c)
{
    StepConsts2 k;
    k.c0 = f2_pack(c.c0, c.c0);
    k.dt = f2_pack(c.dt, c.dt);
    k.q = f2_pack(c.q, c.q);
    k.g = f2_pack(c.g, c.g);
    k.z = f2_pack(c.nz, c.nz);
    return k;
}

// x~ of a pair (Eqs. eq_SyEuY, eq_SyEuX), by the same operations as
// sb_update2.  The walls keep the sign of x~, so sgn(x') = sgn(x~).
__device__ __forceinline__ uint64_t sb_position2(uint64_t f, uint64_t x0, uint64_t y0, uint64_t pk2,
                                                 const StepConsts2 &k)
{
    const uint64_t u = f2_fma(k.c0, f, k.z);
    const uint64_t v = f2_fma(pk2, x0, k.z);
    const uint64_t w = f2_sub(u, v);
    const uint64_t wd = f2_fma(w, k.dt, k.z);
    const uint64_t yt = f2_add(y0, wd);
    const uint64_t qy = f2_fma(k.q, yt, k.z);
    return f2_add(x0, qy);
}

// sb_update on the pairs (f, x0, y0) with p_k broadcast in pk2; the walls
// are applied per element.  Returns x' per element and y' as a pair.
__device__ __forceinline__ void sb_update2(uint64_t f, uint64_t x0, uint64_t y0, uint64_t pk2,
                                           const StepConsts2 &k, float &xn_lo, float &xn_hi,
                                           uint64_t &yn)
{
    const uint64_t u = f2_fma(k.c0, f, k.z);
    const uint64_t v = f2_fma(pk2, x0, k.z);
    const uint64_t w = f2_sub(u, v);
    const uint64_t wd = f2_fma(w, k.dt, k.z);
    const uint64_t yt = f2_add(y0, wd);
    const uint64_t qy = f2_fma(k.q, yt, k.z);
    const uint64_t xt = f2_add(x0, qy);
    const float xt0 = f2_lo(xt), xt1 = f2_hi(xt);
    // walls: |x~| > 1 -> x' = sgn(x~), y~~ = 0 (Eqs. eq_WallX, eq_WallY)
    xn_lo = fminf(fmaxf(xt0, -1.f), 1.f);
    xn_hi = fminf(fmaxf(xt1, -1.f), 1.f);
    const float ytt0 = fabsf(xt0) > 1.f ? 0.f : f2_lo(yt);
    const float ytt1 = fabsf(xt1) > 1.f ? 0.f : f2_hi(yt);
    const uint64_t gy = f2_fma(k.g, y0, k.z);
    yn = f2_add(f2_pack(ytt0, ytt1), gy);
}

}  // namespace hsb
