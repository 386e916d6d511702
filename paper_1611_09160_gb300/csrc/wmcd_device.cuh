// Device (and host-callable) building blocks of the WMCD kernels for sm_103a.
//
// Every quantity that moves a bead is formed with explicitly rounded IEEE operations
// (__dmul_rn, __dadd_rn, ... and __fma_rn where a fused step is intended) in a fixed order,
// so the compiler cannot contract or reorder them; the same arithmetic is stated in the
// comments so that an independent implementation can reproduce positions bit for bit.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace wmcd {

#define WMCD_HD __host__ __device__ __forceinline__

constexpr double kPi = 3.141592653589793;
constexpr double kTwoPi = 6.283185307179586;
constexpr double kLn2 = 0.6931471805599453;
constexpr double kWcaCut = 1.122462048309373;   // 2^(1/6), WCA cutoff in units of sigma (Eq. 2)

// ---- explicitly rounded arithmetic (host: plain IEEE ops in a TU built without contraction) ----
#if defined(__CUDA_ARCH__)
WMCD_HD double mul(double a, double b) { return __dmul_rn(a, b); }
WMCD_HD double add(double a, double b) { return __dadd_rn(a, b); }
WMCD_HD double sub(double a, double b) { return __dsub_rn(a, b); }
WMCD_HD double dvd(double a, double b) { return __ddiv_rn(a, b); }
WMCD_HD double sqr_t(double a) { return __dsqrt_rn(a); }
WMCD_HD double fma_(double a, double b, double c) { return __fma_rn(a, b, c); }
WMCD_HD float mulf(float a, float b) { return __fmul_rn(a, b); }
WMCD_HD float addf(float a, float b) { return __fadd_rn(a, b); }
WMCD_HD float subf(float a, float b) { return __fsub_rn(a, b); }
WMCD_HD float dvdf(float a, float b) { return __fdiv_rn(a, b); }
WMCD_HD float sqrtf_(float a) { return __fsqrt_rn(a); }
WMCD_HD float fmaf_(float a, float b, float c) { return __fmaf_rn(a, b, c); }
#else
WMCD_HD double mul(double a, double b) { return a * b; }
WMCD_HD double add(double a, double b) { return a + b; }
WMCD_HD double sub(double a, double b) { return a - b; }
WMCD_HD double dvd(double a, double b) { return a / b; }
WMCD_HD double sqr_t(double a) { return __builtin_sqrt(a); }
WMCD_HD double fma_(double a, double b, double c) { return __builtin_fma(a, b, c); }
WMCD_HD float mulf(float a, float b) { return a * b; }
WMCD_HD float addf(float a, float b) { return a + b; }
WMCD_HD float subf(float a, float b) { return a - b; }
WMCD_HD float dvdf(float a, float b) { return a / b; }
WMCD_HD float sqrtf_(float a) { return __builtin_sqrtf(a); }
WMCD_HD float fmaf_(float a, float b, float c) { return __builtin_fmaf(a, b, c); }
#endif

// ---- Philox4x32-10 (Salmon et al., SC'11): counter-based random numbers ----
struct u4 { uint32_t x, y, z, w; };

WMCD_HD uint32_t mulhi32(uint32_t a, uint32_t b) {
#if defined(__CUDA_ARCH__)
    return __umulhi(a, b);
#else
    return (uint32_t)(((uint64_t)a * b) >> 32);
#endif
}

WMCD_HD u4 philox4x32_10(u4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; r++) {
        const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
        uint32_t hi0 = mulhi32(M0, c.x), lo0 = M0 * c.x;
        uint32_t hi1 = mulhi32(M1, c.z), lo1 = M1 * c.z;
        u4 n{hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0};
        c = n;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// Stream kinds, placed in bits 24..31 of counter word 2.
enum Kind : uint32_t {
    K_COUNT = 1, K_SLOT = 2, K_VB = 3, K_VP = 4, K_ACC = 5, K_PWCOUNT = 6, K_PWMODE = 7, K_PWDIR = 8,
    K_PWACC = 9, K_DPWMODE = 10, K_DPWDIR = 11, K_DPWACC = 12, K_PWSHELL = 14, K_PWKDIR = 15, K_DPWSHELL = 16,
    K_DPWKDIR = 17, K_BUNI = 18
};

// counter = (index, sweep lo, kind << 24 | layer << 16 | attempt, sweep hi); key = (k0, k1)
WMCD_HD u4 draw(uint32_t k0, uint32_t k1, uint32_t kind, int layer, uint64_t sweep, uint32_t index,
                uint32_t attempt) {
    u4 c{index, (uint32_t)sweep, (kind << 24) | ((uint32_t)(layer & 0xFF) << 16) | (attempt & 0xFFFFu),
         (uint32_t)(sweep >> 32)};
    return philox4x32_10(c, k0, k1);
}
// uniform in [0, 1) with 53 random bits (exact conversion)
WMCD_HD double u53(uint32_t hi, uint32_t lo) {
    uint64_t m = ((uint64_t)(hi >> 5) << 26) | (uint64_t)(lo >> 6);
    return (double)m * (1.0 / 9007199254740992.0);
}
// uniform in (0, 1): the same 53 bits with the lowest set, so neither end is reached
WMCD_HD double u_open(uint32_t hi, uint32_t lo) {
    uint64_t m = ((uint64_t)(hi >> 5) << 26) | (uint64_t)(lo >> 6);
    return (double)(m | 1u) * (1.0 / 9007199254740992.0);
}
// uniform integer in [0, n): high word of the 64 x 64 product
WMCD_HD int64_t pick(uint32_t hi, uint32_t lo, int64_t n) {
    uint64_t x = ((uint64_t)hi << 32) | lo;
#if defined(__CUDA_ARCH__)
    return (int64_t)__umul64hi(x, (uint64_t)n);
#else
    return (int64_t)(((unsigned __int128)x * (uint64_t)n) >> 64);
#endif
}
// coordinate of a point of [-1, 1)^3 (exact)
WMCD_HD double sym(uint32_t w) { return (double)w * (1.0 / 2147483648.0) - 1.0; }

// ---- own elementary functions ----
// w^(-1/3) for w in [hi^-3, lo^-3] with hi <= 2 lo: 8 Newton steps y <- y (4 - w y^3) / 3 from y = lo
WMCD_HD double inv_cbrt_band(double w, double lo) {
    double y = lo;
#pragma unroll
    for (int it = 0; it < 8; it++) {
        double t = mul(w, mul(mul(y, y), y));
        y = dvd(mul(y, sub(4.0, t)), 3.0);
    }
    return y;
}
// Taylor polynomials of cos and sin on [0, pi/4], Horner in t^2 with fused steps
WMCD_HD double cos_poly(double t) {
    double z = mul(t, t), nz = -z;
    double c = 1.0 / 6402373705728000.0;       // 1/18!
    c = fma_(c, nz, 1.0 / 20922789888000.0);   // 1/16!
    c = fma_(c, nz, 1.0 / 87178291200.0);      // 1/14!
    c = fma_(c, nz, 1.0 / 479001600.0);        // 1/12!
    c = fma_(c, nz, 1.0 / 3628800.0);          // 1/10!
    c = fma_(c, nz, 1.0 / 40320.0);
    c = fma_(c, nz, 1.0 / 720.0);
    c = fma_(c, nz, 1.0 / 24.0);
    c = fma_(c, nz, 0.5);
    c = fma_(c, nz, 1.0);
    return c;
}
WMCD_HD double sin_poly(double t) {
    double z = mul(t, t), nz = -z;
    double c = 1.0 / 121645100408832000.0;     // 1/19!
    c = fma_(c, nz, 1.0 / 355687428096000.0);  // 1/17!
    c = fma_(c, nz, 1.0 / 1307674368000.0);    // 1/15!
    c = fma_(c, nz, 1.0 / 6227020800.0);       // 1/13!
    c = fma_(c, nz, 1.0 / 39916800.0);         // 1/11!
    c = fma_(c, nz, 1.0 / 362880.0);
    c = fma_(c, nz, 1.0 / 5040.0);
    c = fma_(c, nz, 1.0 / 120.0);
    c = fma_(c, nz, 1.0 / 6.0);
    c = fma_(c, nz, 1.0);
    return mul(c, t);
}
// cos(2 pi t), sin(2 pi t) for t in turns; the reductions are exact
WMCD_HD double cos2pi(double t) {
    double x = sub(t, floor(t));
    if (x > 0.5) x = sub(1.0, x);
    if (x <= 0.125) return cos_poly(mul(kTwoPi, x));
    if (x <= 0.375) return sin_poly(mul(kTwoPi, sub(0.25, x)));
    return -cos_poly(mul(kTwoPi, sub(0.5, x)));
}
WMCD_HD double sin2pi(double t) {
    double x = sub(t, floor(t)), sgn = 1.0;
    if (x >= 0.5) { x = sub(x, 0.5); sgn = -1.0; }
    if (x > 0.25) x = sub(0.5, x);
    double r = (x <= 0.125) ? sin_poly(mul(kTwoPi, x)) : cos_poly(mul(kTwoPi, sub(0.25, x)));
    return sgn * r;
}
WMCD_HD float cos_poly_f(float t) {
    float z = mulf(t, t), nz = -z;
    float c = 1.0f / 3628800.0f;
    c = fmaf_(c, nz, 1.0f / 40320.0f);
    c = fmaf_(c, nz, 1.0f / 720.0f);
    c = fmaf_(c, nz, 1.0f / 24.0f);
    c = fmaf_(c, nz, 0.5f);
    c = fmaf_(c, nz, 1.0f);
    return c;
}
WMCD_HD float sin_poly_f(float t) {
    float z = mulf(t, t), nz = -z;
    float c = 1.0f / 39916800.0f;
    c = fmaf_(c, nz, 1.0f / 362880.0f);
    c = fmaf_(c, nz, 1.0f / 5040.0f);
    c = fmaf_(c, nz, 1.0f / 120.0f);
    c = fmaf_(c, nz, 1.0f / 6.0f);
    c = fmaf_(c, nz, 1.0f);
    return mulf(c, t);
}
WMCD_HD float cos2pi_f(double t) {
    double x = sub(t, floor(t));
    if (x > 0.5) x = sub(1.0, x);
    if (x <= 0.125) return cos_poly_f((float)mul(kTwoPi, x));
    if (x <= 0.375) return sin_poly_f((float)mul(kTwoPi, sub(0.25, x)));
    return -cos_poly_f((float)mul(kTwoPi, sub(0.5, x)));
}

// ---- periodic box ----
// On the device the comparisons below are taken on the bit patterns: for IEEE doubles and a
// positive bound, the order of the patterns as signed integers is the order of the values for
// every input but a NaN, so the results are those of the binary64 comparisons, without using
// the binary64 pipe (slow on this part) for them.
#ifdef __CUDA_ARCH__
__device__ __forceinline__ bool ge_pos(double x, double b) {      // x >= b, b > 0 finite
    return __double_as_longlong(x) >= __double_as_longlong(b);
}
__device__ __forceinline__ bool lt_zero(double x) {               // x < 0
    const long long xb = __double_as_longlong(x);
    return xb < 0 && (xb & 0x7fffffffffffffffLL) != 0;
}
__device__ __forceinline__ bool gt_pos(double x, double b) {      // x > b, b > 0 finite
    return __double_as_longlong(x) > __double_as_longlong(b);
}
__device__ __forceinline__ bool lt_neg(double x, double b) {      // x < -b, b > 0 finite
    const long long xb = __double_as_longlong(x);
    return xb < 0 && (xb & 0x7fffffffffffffffLL) > __double_as_longlong(b);
}
#else
inline bool ge_pos(double x, double b) { return x >= b; }
inline bool lt_zero(double x) { return x < 0.0; }
inline bool gt_pos(double x, double b) { return x > b; }
inline bool lt_neg(double x, double b) { return x < -b; }
#endif
// wrap into [0, L); image counter change returned through *im (may be null)
WMCD_HD double wrap(double x, double L, int* im) {
    if (ge_pos(x, L)) { x = sub(x, L); if (im) *im += 1; }
    else if (lt_zero(x)) { x = add(x, L); if (im) *im -= 1; }
    if (ge_pos(x, L)) x = 0.0;
    return x;
}
// minimum image of a difference of two wrapped coordinates
WMCD_HD double mi(double d, double L, double h) {
    if (gt_pos(d, h)) return sub(d, L);
    if (lt_neg(d, h)) return add(d, L);
    return d;
}
WMCD_HD double norm2(double x, double y, double z) { return add(add(mul(x, x), mul(y, y)), mul(z, z)); }

// fine cell index floor(x G_f / L), clamped to [0, G_f - 1] (a NaN maps to 0)
WMCD_HD int fine_cell(double x, double invf, int Gf) {
    double f = floor(mul(x, invf));
    if (!(f >= 0.0)) return 0;
    if (f >= (double)(Gf - 1)) return Gf - 1;
    return (int)f;
}
WMCD_HD int64_t floordiv(int64_t a, int64_t b) { int64_t q = a / b; if ((a % b != 0) && ((a < 0) != (b < 0))) q--; return q; }
WMCD_HD int64_t ceildiv(int64_t a, int64_t b) { return -floordiv(-a, b); }
WMCD_HD bool range_inside(int64_t t0, int64_t t1, int64_t lo, int64_t hi, int64_t Gf) {
    return (t0 - Gf >= lo && t1 - Gf <= hi) || (t0 >= lo && t1 <= hi) || (t0 + Gf >= lo && t1 + Gf <= hi);
}

// ---- displacement of a bead at offset d from the wavelet centre (Sec. V.A, Eq. 21/23) ----
// delta = s (p x d) with s = (A_w (1 - sqrt(d2)/lambda)) / lambda
WMCD_HD void wavelet_disp64(const double d[3], double d2, double lam, double Aw, const double p[3], double out[3]) {
    double rho = dvd(sqr_t(d2), lam);
    double sc = dvd(mul(Aw, sub(1.0, rho)), lam);
    double cx = sub(mul(p[1], d[2]), mul(p[2], d[1]));
    double cy = sub(mul(p[2], d[0]), mul(p[0], d[2]));
    double cz = sub(mul(p[0], d[1]), mul(p[1], d[0]));
    out[0] = mul(sc, cx); out[1] = mul(sc, cy); out[2] = mul(sc, cz);
}
// mixed precision: the same expression in binary32 on inputs rounded once
// the same with lam, A_w and p already rounded to binary32 (once per move, not per member),
// returning the binary32 displacement
WMCD_HD void wavelet_disp32ff(const double d[3], float lf, float af, const float pf[3], float out[3]) {
    float dx = (float)d[0], dy = (float)d[1], dz = (float)d[2];
    float d2f = addf(addf(mulf(dx, dx), mulf(dy, dy)), mulf(dz, dz));
    float px = pf[0], py = pf[1], pz = pf[2];
    float rho = dvdf(sqrtf_(d2f), lf);
    float sc = dvdf(mulf(af, subf(1.0f, rho)), lf);
    float cx = subf(mulf(py, dz), mulf(pz, dy));
    float cy = subf(mulf(pz, dx), mulf(px, dz));
    float cz = subf(mulf(px, dy), mulf(py, dx));
    out[0] = mulf(sc, cx); out[1] = mulf(sc, cy); out[2] = mulf(sc, cz);
}
WMCD_HD void wavelet_disp32f(const double d[3], float lf, float af, const float pf[3], double out[3]) {
    float dx = (float)d[0], dy = (float)d[1], dz = (float)d[2];
    float d2f = addf(addf(mulf(dx, dx), mulf(dy, dy)), mulf(dz, dz));
    float px = pf[0], py = pf[1], pz = pf[2];
    float rho = dvdf(sqrtf_(d2f), lf);
    float sc = dvdf(mulf(af, subf(1.0f, rho)), lf);
    float cx = subf(mulf(py, dz), mulf(pz, dy));
    float cy = subf(mulf(pz, dx), mulf(px, dz));
    float cz = subf(mulf(px, dy), mulf(py, dx));
    out[0] = (double)mulf(sc, cx); out[1] = (double)mulf(sc, cy); out[2] = (double)mulf(sc, cz);
}
WMCD_HD void wavelet_disp32(const double d[3], double lam, double Aw, const double p[3], double out[3]) {
    float dx = (float)d[0], dy = (float)d[1], dz = (float)d[2];
    float d2f = addf(addf(mulf(dx, dx), mulf(dy, dy)), mulf(dz, dz));
    float lf = (float)lam, af = (float)Aw, px = (float)p[0], py = (float)p[1], pz = (float)p[2];
    float rho = dvdf(sqrtf_(d2f), lf);
    float sc = dvdf(mulf(af, subf(1.0f, rho)), lf);
    float cx = subf(mulf(py, dz), mulf(pz, dy));
    float cy = subf(mulf(pz, dx), mulf(px, dz));
    float cz = subf(mulf(px, dy), mulf(py, dx));
    out[0] = (double)mulf(sc, cx); out[1] = (double)mulf(sc, cy); out[2] = (double)mulf(sc, cz);
}

// ---- energies (Eqs. 1, 2; harmonic bond; external well) ----
struct Pot {
    double sig2, eps, rc2;          // WCA; eps = 0: off
    int bond;                        // 0 none, 1 harmonic, 2 FENE
    double bk, br0, R02;
    double kappa, halfL, L;          // external well at the box centre
};
WMCD_HD double U_wca(const Pot& P, double r2) {
    if (P.eps == 0.0 || !(r2 < P.rc2)) return 0.0;
    double s2 = P.sig2 / r2, s6 = s2 * s2 * s2;
    return 4.0 * P.eps * (s6 * s6 - s6) + P.eps;
}
WMCD_HD double U_bond(const Pot& P, double r2) {
    if (P.bond == 1) { double d = sqrt(r2) - P.br0; return 0.5 * P.bk * d * d; }
    if (P.bond == 2) {
        double x = r2 / P.R02;
        if (!(x < 1.0)) return __builtin_inf();
        return -0.5 * P.bk * P.R02 * log(1.0 - x);
    }
    return 0.0;
}
WMCD_HD double U_ext(const Pot& P, double x, double y, double z) {
    if (P.kappa == 0.0) return 0.0;
    double dx = mi(x - P.halfL, P.L, P.halfL), dy = mi(y - P.halfL, P.L, P.halfL), dz = mi(z - P.halfL, P.L, P.halfL);
    return 0.5 * P.kappa * (dx * dx + dy * dy + dz * dz);
}

}  // namespace wmcd
