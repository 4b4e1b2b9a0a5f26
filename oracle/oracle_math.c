/* ORACLE (test infrastructure only; never linked into the product path).
 *
 * Deterministic elementary functions built from IEEE +, -, *, / and exact bit manipulation only, so that
 * two independent implementations that follow the same published recipe produce identical bits. The
 * particle path needs them wherever a transcendental value decides an integer (a cell index after
 * transport, the number of sampled particles, a fixed-point tally).
 *
 *  log : range reduction x = 2^e m, m in [sqrt(1/2), sqrt(2)], then ln m = 2 atanh(s), s = (m-1)/(m+1),
 *        summed as the odd power series of atanh; ln 2 split Cody-Waite style into a short high part
 *        (exact products e * hi) and a low part. [Cody & Waite, "Software Manual for the Elementary
 *        Functions", 1980, ch. 5.]
 *  exp : x = k ln2 + r, |r| <= ln2/2 with the same split, Taylor series of e^r (Horner), scaled by 2^k
 *        built from the exponent bits. Double: results below 2^-1021 are flushed to 0; float (Taylor to
 *        r^7): arguments below -87 give 0.
 *  erfc (double; the wave flux's half-range moments): for |x| < 3/2, 1 - erf(x) with
 *        erf(x) = (2/sqrt(pi)) e^{-x^2} sum_n 2^n x^(2n+1) / (1 * 3 * ... * (2n+1)), a series of positive terms
 *        [Abramowitz & Stegun 7.1.6], summed until a term falls below 2^-56 of the partial sum; for x >= 3/2
 *        Laplace's continued fraction erfc(x) = (e^{-x^2}/sqrt(pi)) / (x + (1/2)/(x + 1/(x + (3/2)/(x + ...))))
 *        [A&S 7.1.14], evaluated from the bottom at depth 8 + floor(240/x^2) (converged to about 1e-16);
 *        erfc(-x) = 2 - erfc(x).
 *  sincos(2 pi u): reduction in turns, u = q/4 + r exactly, |r| <= 1/8, Taylor series of sin and cos of
 *        2 pi r, quadrant by q mod 4.
 * Coefficients are reciprocal factorials and reciprocal odd integers, written as exact divisions.
 * The file is compiled with -ffp-contract=off so no multiply-add is fused.
 */
#include "oracle_internal.h"
#include <string.h>

#define OR_LN2_HI_F 0x1.62e4p-1f
#define OR_LN2_LO_F 0x1.7f7d1cp-20f
#define OR_LN2_HI_D 0x1.62e42feep-1
#define OR_LN2_LO_D 0x1.a39ef35793c76p-33
#define OR_INV_LN2_D 0x1.71547652b82fep+0
#define OR_INV_LN2_F 0x1.715476p+0f
#define OR_TWO_PI_F 0x1.921fb6p+2f
#define OR_TWO_PI_D 0x1.921fb54442d18p+2

float or_logf(float x)
{
    uint32_t b;
    memcpy(&b, &x, 4);
    int e = (int)((b >> 23) & 0xffu) - 127;
    uint32_t mb = (b & 0x7fffffu) | 0x3f800000u;
    if (mb > 0x3fb504f3u) { mb -= 0x00800000u; e += 1; }
    float m;
    memcpy(&m, &mb, 4);
    const float f = m - 1.0f;
    const float s = f / (2.0f + f);
    const float z = s * s;
    const float p = (1.0f / 3.0f) + z * ((1.0f / 5.0f) + z * ((1.0f / 7.0f) + z * (1.0f / 9.0f)));
    const float lm = 2.0f * s + 2.0f * (s * (z * p));
    const float fe = (float)e;
    return fe * OR_LN2_HI_F + (lm + fe * OR_LN2_LO_F);
}

double or_logd(double x)
{
    uint64_t b;
    memcpy(&b, &x, 8);
    int e = (int)((b >> 52) & 0x7ffu) - 1023;
    uint64_t mb = (b & 0xfffffffffffffULL) | 0x3ff0000000000000ULL;
    if (mb > 0x3ff6a09e667f3bcdULL) { mb -= 0x0010000000000000ULL; e += 1; }
    double m;
    memcpy(&m, &mb, 8);
    const double f = m - 1.0;
    const double s = f / (2.0 + f);
    const double z = s * s;
    double p = 1.0 / 23.0;
    p = 1.0 / 21.0 + z * p;
    p = 1.0 / 19.0 + z * p;
    p = 1.0 / 17.0 + z * p;
    p = 1.0 / 15.0 + z * p;
    p = 1.0 / 13.0 + z * p;
    p = 1.0 / 11.0 + z * p;
    p = 1.0 / 9.0 + z * p;
    p = 1.0 / 7.0 + z * p;
    p = 1.0 / 5.0 + z * p;
    p = 1.0 / 3.0 + z * p;
    const double lm = 2.0 * s + 2.0 * (s * (z * p));
    const double fe = (double)e;
    return fe * OR_LN2_HI_D + (lm + fe * OR_LN2_LO_D);
}

double or_expd(double x)
{
    if (x < -708.0) return 0.0;
    if (x > 709.0) return 1.0 / 0.0;
    const double kf = rint(x * OR_INV_LN2_D);
    const int k = (int)kf;
    const double r = (x - kf * OR_LN2_HI_D) - kf * OR_LN2_LO_D;
    double p = 1.0 / 355687428096000.0;            /* 1/17! */
    p = 1.0 / 20922789888000.0 + r * p;            /* 1/16! */
    p = 1.0 / 1307674368000.0 + r * p;
    p = 1.0 / 87178291200.0 + r * p;
    p = 1.0 / 6227020800.0 + r * p;
    p = 1.0 / 479001600.0 + r * p;
    p = 1.0 / 39916800.0 + r * p;
    p = 1.0 / 3628800.0 + r * p;
    p = 1.0 / 362880.0 + r * p;
    p = 1.0 / 40320.0 + r * p;
    p = 1.0 / 5040.0 + r * p;
    p = 1.0 / 720.0 + r * p;
    p = 1.0 / 120.0 + r * p;
    p = 1.0 / 24.0 + r * p;
    p = 1.0 / 6.0 + r * p;
    p = 0.5 + r * p;
    p = 1.0 + r * p;
    p = 1.0 + r * p;
    const uint64_t sb = (uint64_t)(k + 1023) << 52;
    double sc;
    memcpy(&sc, &sb, 8);
    return p * sc;
}

double or_erfcd(double x)
{
    if (x != x) return x;
    const double a = x < 0.0 ? -x : x;
    const double rsqrt_pi = 0x1.20dd750429b6dp-1;   /* 1/sqrt(pi) */
    double r;
    if (a < 1.5) {
        const double x2 = 2.0 * (a * a);
        double t = a, s = a;
        for (int n = 0; n < 200; ++n) {
            t = (t * x2) / (double)(2 * n + 3);
            if (!(t > 0x1p-56 * s)) break;
            s = s + t;
        }
        r = 1.0 - ((2.0 * rsqrt_pi) * or_expd(-(a * a))) * s;
    } else {
        const int depth = 8 + (int)(240.0 / (a * a));
        double k = 0.0;
        for (int j = depth; j > 0; --j) k = (0.5 * (double)j) / (a + k);
        r = (or_expd(-(a * a)) * rsqrt_pi) / (a + k);
    }
    return x < 0.0 ? 2.0 - r : r;
}

float or_expf(float x)
{
    if (x < -87.0f) return 0.0f;
    if (x > 88.0f) return 1.0f / 0.0f;
    const float kf = rintf(x * OR_INV_LN2_F);
    const int k = (int)kf;
    const float r = (x - kf * OR_LN2_HI_F) - kf * OR_LN2_LO_F;
    float p = 1.0f / 5040.0f;                      /* 1/7! */
    p = 1.0f / 720.0f + r * p;
    p = 1.0f / 120.0f + r * p;
    p = 1.0f / 24.0f + r * p;
    p = 1.0f / 6.0f + r * p;
    p = 0.5f + r * p;
    p = 1.0f + r * p;
    p = 1.0f + r * p;
    const uint32_t sb = (uint32_t)(k + 127) << 23;
    float sc;
    memcpy(&sc, &sb, 4);
    return p * sc;
}

double or_powd(double x, double y)
{
    return or_expd(y * or_logd(x));
}

void or_sincos2pif(float u, float* s, float* c)
{
    const float q = rintf(4.0f * u);
    const float r = u - 0.25f * q;
    const int k = ((int)q) & 3;
    const float t = r * OR_TWO_PI_F;
    const float z = t * t;
    const float sp = t + t * (z * (-1.0f / 6.0f + z * (1.0f / 120.0f + z * (-1.0f / 5040.0f + z * (1.0f / 362880.0f)))));
    const float cp = 1.0f + z * (-0.5f + z * (1.0f / 24.0f + z * (-1.0f / 720.0f + z * (1.0f / 40320.0f
                     + z * (-1.0f / 3628800.0f)))));
    switch (k) {
    case 0: *s = sp; *c = cp; break;
    case 1: *s = cp; *c = -sp; break;
    case 2: *s = -sp; *c = -cp; break;
    default: *s = -cp; *c = sp; break;
    }
}

void or_sincos2pid(double u, double* s, double* c)
{
    const double q = rint(4.0 * u);
    const double r = u - 0.25 * q;
    const int k = ((int)q) & 3;
    const double t = r * OR_TWO_PI_D;
    const double z = t * t;
    double ps = -1.0 / 121645100408832000.0;       /* -1/19! */
    ps = 1.0 / 355687428096000.0 + z * ps;         /* 1/17! */
    ps = -1.0 / 1307674368000.0 + z * ps;          /* -1/15! */
    ps = 1.0 / 6227020800.0 + z * ps;              /* 1/13! */
    ps = -1.0 / 39916800.0 + z * ps;               /* -1/11! */
    ps = 1.0 / 362880.0 + z * ps;                  /* 1/9! */
    ps = -1.0 / 5040.0 + z * ps;
    ps = 1.0 / 120.0 + z * ps;
    ps = -1.0 / 6.0 + z * ps;
    const double sp = t + t * (z * ps);
    double pc = 1.0 / 2432902008176640000.0;       /* 1/20! */
    pc = -1.0 / 6402373705728000.0 + z * pc;       /* -1/18! */
    pc = 1.0 / 20922789888000.0 + z * pc;          /* 1/16! */
    pc = -1.0 / 87178291200.0 + z * pc;            /* -1/14! */
    pc = 1.0 / 479001600.0 + z * pc;               /* 1/12! */
    pc = -1.0 / 3628800.0 + z * pc;                /* -1/10! */
    pc = 1.0 / 40320.0 + z * pc;
    pc = -1.0 / 720.0 + z * pc;
    pc = 1.0 / 24.0 + z * pc;
    pc = -0.5 + z * pc;
    const double cp = 1.0 + z * pc;
    switch (k) {
    case 0: *s = sp; *c = cp; break;
    case 1: *s = cp; *c = -sp; break;
    case 2: *s = -sp; *c = -cp; break;
    default: *s = -cp; *c = sp; break;
    }
}

/* exported for the accuracy pins */
float oracle_logf(float x) { return or_logf(x); }
double oracle_logd(double x) { return or_logd(x); }
double oracle_expd(double x) { return or_expd(x); }
double oracle_erfcd(double x) { return or_erfcd(x); }
float oracle_expf(float x) { return or_expf(x); }
void oracle_sincos2pif(float u, float* s, float* c) { or_sincos2pif(u, s, c); }
void oracle_sincos2pid(double u, double* s, double* c) { or_sincos2pid(u, s, c); }
