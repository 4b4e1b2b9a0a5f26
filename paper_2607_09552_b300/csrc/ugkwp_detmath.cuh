// Device-side counter-based RNG and deterministic elementary functions.
//
// Every transcendental value that decides an integer of the method (a cell index after transport, the
// number of sampled particles, a fixed-point tally) goes through these functions. They use only IEEE
// round-to-nearest +, -, *, / (explicit __f*_rn / __d*_rn intrinsics, so that no multiply-add is ever
// contracted, whatever the compilation flags) and exact bit manipulation, so their results are fixed bit
// patterns defined by the recipe below.
//
//  Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): 10 rounds of two 32x32->64 multiplications by the
//    Philox constants with xor-mixing of the high halves, key bumped by the two Weyl constants.
//  log: x = 2^e m with m in [sqrt(1/2), sqrt(2)], ln m = 2 atanh(s), s = (m-1)/(m+1), odd series of atanh
//    in Horner form; ln 2 split into a short high part (exact products with e) and a low part
//    (Cody & Waite, 1980).
//  exp: k = rint(x / ln 2), r = (x - k ln2_hi) - k ln2_lo, Taylor series of e^r to r^17, times 2^k built
//    from exponent bits; results below 2^-1021 are flushed to zero.
//  sincos(2 pi u): exact reduction in turns u = q/4 + r (|r| <= 1/8), Taylor series of sin and cos of
//    2 pi r, quadrant from q mod 4.
#pragma once
#include <cstdint>

namespace ugk {

struct u32x4 { uint32_t x, y, z, w; };

__device__ __forceinline__ u32x4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                                               uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        // one 32 x 32 -> 64-bit product per multiplier gives both halves
        const uint64_t p0 = (uint64_t)0xD2511F53u * c0, p1 = (uint64_t)0xCD9E8D57u * c2;
        const uint32_t lo0 = (uint32_t)p0, hi0 = (uint32_t)(p0 >> 32);
        const uint32_t lo1 = (uint32_t)p1, hi1 = (uint32_t)(p1 >> 32);
        const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    }
    return {c0, c1, c2, c3};
}

// stream layout: key = (seed_lo ^ case_id, seed_hi), counter = (pid_lo, pid_hi, step, draw)
struct Rng {
    uint32_t k0, k1, step;
    __device__ __forceinline__ u32x4 draw(uint64_t pid, uint32_t d) const
    {
        return philox4x32_10((uint32_t)pid, (uint32_t)(pid >> 32), step, d, k0, k1);
    }
};

// draw groups (first counter word)
constexpr uint32_t DRAW_POS = 0u, DRAW_VEL = 2u, DRAW_TF = 5u;
__device__ __forceinline__ uint32_t draw_wall(int h) { return 8u + 2u * (uint32_t)h; }
// Shakhov acceptance-rejection attempt a: proposal draws +0 (+1 in FP64), acceptance draw +2
__device__ __forceinline__ uint32_t draw_ar(int a) { return 1024u + 4u * (uint32_t)a; }
constexpr int kArAttempts = 64;

__device__ __forceinline__ float u01(uint32_t w)
{
    return __fmul_rn(__fadd_rn(__uint2float_rn(w >> 9), 0.5f), 0x1p-23f);
}
__device__ __forceinline__ double u01d(uint32_t lo, uint32_t hi)
{
    const uint64_t b = ((uint64_t)hi << 32) | (uint64_t)lo;
    return __dmul_rn(__dadd_rn(__ull2double_rn(b >> 12), 0.5), 0x1p-52);
}

// n uniforms of a draw group in precision T (float: one Philox call holds four; double: two per call)
template <typename T> struct Unif;
template <> struct Unif<float> {
    __device__ __forceinline__ static void get(const Rng& g, uint64_t pid, uint32_t base, int n, float* u)
    {
        const u32x4 w = g.draw(pid, base);
        u[0] = u01(w.x);
        if (n > 1) u[1] = u01(w.y);
        if (n > 2) u[2] = u01(w.z);
        if (n > 3) u[3] = u01(w.w);
    }
};
template <> struct Unif<double> {
    __device__ __forceinline__ static void get(const Rng& g, uint64_t pid, uint32_t base, int n, double* u)
    {
        const u32x4 a = g.draw(pid, base);
        u[0] = u01d(a.x, a.y);
        if (n > 1) u[1] = u01d(a.z, a.w);
        if (n > 2) {
            const u32x4 b = g.draw(pid, base + 1u);
            u[2] = u01d(b.x, b.y);
            if (n > 3) u[3] = u01d(b.z, b.w);
        }
    }
};

// ------------------------------------------------------------------------------------------- float
__device__ __forceinline__ float dlog(float x)
{
    const uint32_t b = __float_as_uint(x);
    int e = (int)((b >> 23) & 0xffu) - 127;
    uint32_t mb = (b & 0x7fffffu) | 0x3f800000u;
    if (mb > 0x3fb504f3u) { mb -= 0x00800000u; e += 1; }
    const float m = __uint_as_float(mb);
    const float f = __fsub_rn(m, 1.0f);
    const float s = __fdiv_rn(f, __fadd_rn(2.0f, f));
    const float z = __fmul_rn(s, s);
    float p = __fmul_rn(z, 0x1.c71c72p-4f);          // 1/9
    p = __fmul_rn(z, __fadd_rn(0x1.24924ap-3f, p));  // 1/7
    p = __fmul_rn(z, __fadd_rn(0x1.99999ap-3f, p));  // 1/5
    p = __fadd_rn(0x1.555556p-2f, p);                // 1/3
    const float lm = __fadd_rn(__fmul_rn(2.0f, s), __fmul_rn(2.0f, __fmul_rn(s, __fmul_rn(z, p))));
    const float fe = (float)e;
    return __fadd_rn(__fmul_rn(fe, 0x1.62e4p-1f), __fadd_rn(lm, __fmul_rn(fe, 0x1.7f7d1cp-20f)));
}

__device__ __forceinline__ void dsincos2pi(float u, float* s, float* c)
{
    const float q = rintf(__fmul_rn(4.0f, u));
    const float r = __fsub_rn(u, __fmul_rn(0.25f, q));
    const int k = ((int)q) & 3;
    const float t = __fmul_rn(r, 0x1.921fb6p+2f);
    const float z = __fmul_rn(t, t);
    float ps = __fmul_rn(z, 0x1.71de3ap-19f);         // 1/9!
    ps = __fmul_rn(z, __fadd_rn(-0x1.a01a02p-13f, ps)); // -1/7!
    ps = __fmul_rn(z, __fadd_rn(0x1.111112p-7f, ps));   // 1/5!
    ps = __fadd_rn(-0x1.555556p-3f, ps);                // -1/3!
    const float sp = __fadd_rn(t, __fmul_rn(t, __fmul_rn(z, ps)));
    float pc = __fmul_rn(z, -0x1.27e4fcp-22f);         // -1/10!
    pc = __fmul_rn(z, __fadd_rn(0x1.a01a02p-16f, pc));  // 1/8!
    pc = __fmul_rn(z, __fadd_rn(-0x1.6c16c2p-10f, pc)); // -1/6!
    pc = __fmul_rn(z, __fadd_rn(0x1.555556p-5f, pc));   // 1/4!
    pc = __fadd_rn(-0.5f, pc);
    const float cp = __fadd_rn(1.0f, __fmul_rn(z, pc));
    switch (k) {
    case 0: *s = sp; *c = cp; break;
    case 1: *s = cp; *c = -sp; break;
    case 2: *s = -sp; *c = -cp; break;
    default: *s = -cp; *c = sp; break;
    }
}

// ------------------------------------------------------------------------------------------ double
__device__ __forceinline__ double dlog(double x)
{
    const uint64_t b = (uint64_t)__double_as_longlong(x);
    int e = (int)((b >> 52) & 0x7ffu) - 1023;
    uint64_t mb = (b & 0xfffffffffffffULL) | 0x3ff0000000000000ULL;
    if (mb > 0x3ff6a09e667f3bcdULL) { mb -= 0x0010000000000000ULL; e += 1; }
    const double m = __longlong_as_double((long long)mb);
    const double f = __dsub_rn(m, 1.0);
    const double s = __ddiv_rn(f, __dadd_rn(2.0, f));
    const double z = __dmul_rn(s, s);
    const double c[11] = {0x1.5555555555555p-2, 0x1.999999999999ap-3, 0x1.2492492492492p-3, 0x1.c71c71c71c71cp-4,
                          0x1.745d1745d1746p-4, 0x1.3b13b13b13b14p-4, 0x1.1111111111111p-4, 0x1.e1e1e1e1e1e1ep-5,
                          0x1.af286bca1af28p-5, 0x1.8618618618618p-5, 0x1.642c8590b2164p-5};  // 1/3 .. 1/23
    double p = c[10];
#pragma unroll
    for (int k = 9; k >= 0; --k) p = __dadd_rn(c[k], __dmul_rn(z, p));
    const double lm = __dadd_rn(__dmul_rn(2.0, s), __dmul_rn(2.0, __dmul_rn(s, __dmul_rn(z, p))));
    const double fe = (double)e;
    return __dadd_rn(__dmul_rn(fe, 0x1.62e42feep-1), __dadd_rn(lm, __dmul_rn(fe, 0x1.a39ef35793c76p-33)));
}

__device__ __forceinline__ double dexp(double x)
{
    if (x < -708.0) return 0.0;
    if (x > 709.0) return __longlong_as_double(0x7ff0000000000000LL);
    const double kf = rint(__dmul_rn(x, 0x1.71547652b82fep+0));
    const int k = (int)kf;
    const double r = __dsub_rn(__dsub_rn(x, __dmul_rn(kf, 0x1.62e42feep-1)), __dmul_rn(kf, 0x1.a39ef35793c76p-33));
    // 1/k! for k = 17 .. 2
    const double c[16] = {0x1.952c77030ad4ap-49, 0x1.ae7f3e733b81fp-45, 0x1.ae7f3e733b81fp-41, 0x1.93974a8c07c9dp-37,
                          0x1.6124613a86d09p-33, 0x1.1eed8eff8d898p-29, 0x1.ae64567f544e4p-26, 0x1.27e4fb7789f5cp-22,
                          0x1.71de3a556c734p-19, 0x1.a01a01a01a01ap-16, 0x1.a01a01a01a01ap-13, 0x1.6c16c16c16c17p-10,
                          0x1.1111111111111p-7,  0x1.5555555555555p-5,  0x1.5555555555555p-3,  0.5};
    double p = c[0];
#pragma unroll
    for (int k = 1; k < 16; ++k) p = __dadd_rn(c[k], __dmul_rn(r, p));
    p = __dadd_rn(1.0, __dmul_rn(r, p));
    p = __dadd_rn(1.0, __dmul_rn(r, p));
    const double sc = __longlong_as_double((long long)((uint64_t)(k + 1023) << 52));
    return __dmul_rn(p, sc);
}

__device__ __forceinline__ double dpow(double x, double y) { return dexp(__dmul_rn(y, dlog(x))); }

// erfc in FP64 (the half-range moments of the wave flux in the all-FP64 mode): for |x| < 3/2, 1 - erf(x) with
// erf(x) = (2 / sqrt(pi)) e^{-x^2} sum_n 2^n x^(2n+1) / (1 * 3 * ... * (2n+1)), a series of positive terms
// (Abramowitz & Stegun 7.1.6) summed until a term falls below 2^-56 of the partial sum; for x >= 3/2 Laplace's
// continued fraction erfc(x) = (e^{-x^2} / sqrt(pi)) / (x + (1/2) / (x + 1 / (x + (3/2) / (x + ...))))
// (A&S 7.1.14) evaluated from the bottom at depth 8 + floor(240 / x^2); erfc(-x) = 2 - erfc(x). About 1e-16
// relative where the continued fraction is used, 5e-15 next to 3/2 from the subtraction 1 - erf.
__device__ __forceinline__ double derfc(double x)
{
    if (x != x) return x;
    const double a = fabs(x);
    const double rsqrt_pi = 0x1.20dd750429b6dp-1;
    double r;
    if (a < 1.5) {
        const double x2 = __dmul_rn(2.0, __dmul_rn(a, a));
        double t = a, s = a;
        for (int n = 0; n < 200; ++n) {
            t = __ddiv_rn(__dmul_rn(t, x2), (double)(2 * n + 3));
            if (!(t > __dmul_rn(0x1p-56, s))) break;
            s = __dadd_rn(s, t);
        }
        r = __dsub_rn(1.0, __dmul_rn(__dmul_rn(2.0 * rsqrt_pi, dexp(-__dmul_rn(a, a))), s));
    } else {
        const int depth = 8 + (int)__ddiv_rn(240.0, __dmul_rn(a, a));
        double k = 0.0;
        for (int j = depth; j > 0; --j) k = __ddiv_rn(__dmul_rn(0.5, (double)j), __dadd_rn(a, k));
        r = __ddiv_rn(__dmul_rn(dexp(-__dmul_rn(a, a)), rsqrt_pi), __dadd_rn(a, k));
    }
    return x < 0.0 ? __dsub_rn(2.0, r) : r;
}

__device__ __forceinline__ void dsincos2pi(double u, double* s, double* c)
{
    const double q = rint(__dmul_rn(4.0, u));
    const double r = __dsub_rn(u, __dmul_rn(0.25, q));
    const int k = ((int)q) & 3;
    const double t = __dmul_rn(r, 0x1.921fb54442d18p+2);
    const double z = __dmul_rn(t, t);
    // sin: -1/19!, 1/17!, ..., -1/3!
    const double cs[9] = {-0x1.2f49b46814157p-57, 0x1.952c77030ad4ap-49, -0x1.ae7f3e733b81fp-41,
                          0x1.6124613a86d09p-33, -0x1.ae64567f544e4p-26, 0x1.71de3a556c734p-19,
                          -0x1.a01a01a01a01ap-13, 0x1.1111111111111p-7, -0x1.5555555555555p-3};
    double ps = cs[0];
#pragma unroll
    for (int j = 1; j < 9; ++j) ps = __dadd_rn(cs[j], __dmul_rn(z, ps));
    const double sp = __dadd_rn(t, __dmul_rn(t, __dmul_rn(z, ps)));
    // cos: 1/20!, -1/18!, ..., 1/4!, -1/2
    const double cc[10] = {0x1.e542ba4020225p-62, -0x1.6827863b97d97p-53, 0x1.ae7f3e733b81fp-45,
                           -0x1.93974a8c07c9dp-37, 0x1.1eed8eff8d898p-29, -0x1.27e4fb7789f5cp-22,
                           0x1.a01a01a01a01ap-16, -0x1.6c16c16c16c17p-10, 0x1.5555555555555p-5, -0.5};
    double pc = cc[0];
#pragma unroll
    for (int j = 1; j < 10; ++j) pc = __dadd_rn(cc[j], __dmul_rn(z, pc));
    const double cp = __dadd_rn(1.0, __dmul_rn(z, pc));
    switch (k) {
    case 0: *s = sp; *c = cp; break;
    case 1: *s = cp; *c = -sp; break;
    case 2: *s = -sp; *c = -cp; break;
    default: *s = -cp; *c = sp; break;
    }
}

}  // namespace ugk
