// Canonical Fibonacci launch directions (Sec. II-F), shared by the specular and
// the diffuse tracers so that both launch bit-identical FP32 rays.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

// sin and cos of the angle 2 pi k / 2^32, evaluated with IEEE FP32 operations
// that are never contracted (so any IEEE implementation gets the same bits):
// the top three bits of k pick the octant; inside it the angle theta in
// [0, pi/4] goes through the Taylor series of sin (to theta^11) and cos (to
// theta^12) in Horner form, and the octant symmetries give the final pair.
static __device__ __forceinline__ void sincos_turn(uint32_t k, float& s_out, float& c_out) {
    const uint32_t oct = k >> 29;
    const float y = __fmul_rn(__uint2float_rn(k & 0x1fffffffu), 1.0f / 536870912.0f);   // 2^-29
    const float t = (oct & 1u) ? __fsub_rn(1.0f, y) : y;
    const float th = __fmul_rn(t, 0.785398185253143310546875f);   // pi/4 rounded to FP32
    const float x = __fmul_rn(th, th);
    float ps = -2.50521083854417187751e-08f;   // -1/11!
    ps = __fadd_rn(__fmul_rn(ps, x), 2.75573192239858906526e-06f);    // 1/9!
    ps = __fadd_rn(__fmul_rn(ps, x), -1.98412698412698412698e-04f);   // -1/7!
    ps = __fadd_rn(__fmul_rn(ps, x), 8.33333333333333333333e-03f);    // 1/5!
    ps = __fadd_rn(__fmul_rn(ps, x), -1.66666666666666666667e-01f);   // -1/3!
    ps = __fadd_rn(__fmul_rn(ps, x), 1.0f);
    const float sn = __fmul_rn(ps, th);
    float pc = 2.08767569878680989792e-09f;    // 1/12!
    pc = __fadd_rn(__fmul_rn(pc, x), -2.75573192239858906526e-07f);   // -1/10!
    pc = __fadd_rn(__fmul_rn(pc, x), 2.48015873015873015873e-05f);    // 1/8!
    pc = __fadd_rn(__fmul_rn(pc, x), -1.38888888888888888889e-03f);   // -1/6!
    pc = __fadd_rn(__fmul_rn(pc, x), 4.16666666666666666667e-02f);    // 1/4!
    pc = __fadd_rn(__fmul_rn(pc, x), -0.5f);                          // -1/2!
    pc = __fadd_rn(__fmul_rn(pc, x), 1.0f);
    const float cs = pc;
    // angle = m pi/2 + sigma theta, m = (oct + 1) / 2, sigma = +1 (even oct) / -1 (odd)
    const uint32_t m = ((oct + 1u) >> 1) & 3u;
    const float ss = (oct & 1u) ? -sn : sn;   // sin(sigma theta)
    if (m == 0) {
        s_out = ss;
        c_out = cs;
    } else if (m == 1) {
        s_out = cs;
        c_out = -ss;
    } else if (m == 2) {
        s_out = -ss;
        c_out = -cs;
    } else {
        s_out = -cs;
        c_out = ss;
    }
}

// Fibonacci-lattice launch direction i of N: z = 1 - (2i+1)/N (one correctly
// rounded FP64 division and subtraction, rounded to FP32; the kernels read it
// from a per-N table made on the host, see ray_schedule), r = sqrt(1 - z^2) and
// azimuth fraction frac(i g) of the golden-ratio Weyl sequence in 32-bit fixed
// point, (i * 0x9E3779B9) mod 2^32; every FP32 step is an uncontracted IEEE
// operation, so both implementations produce the same bits.
static __device__ __forceinline__ float3 launch_dir(int64_t i, float z) {
    const float r = __fsqrt_rn(__fsub_rn(1.0f, __fmul_rn(z, z)));
    float s, c;
    sincos_turn((uint32_t)((uint64_t)i * 0x9E3779B9ull), s, c);
    return make_float3(__fmul_rn(r, c), __fmul_rn(r, s), z);
}

