/*
 * CPU oracle for Wavelet Monte Carlo dynamics (Dyer & Ball, arXiv:1611.09160).
 *
 * TEST INFRASTRUCTURE ONLY. This file is a plain, slow, sequential FP64 statement of
 * what the WMCD sweep computes. It is loaded only by the test-suite, by the smoke check
 * and by the benchmark's CPU-baseline leg; the product library never links, loads or
 * calls it, and it shares no code, header, table or constant generator with the CUDA
 * library. The only thing both sides share is the seeded input generator (initial bead
 * positions), which contains none of the method's arithmetic.
 *
 * What it follows (sections and equations of the paper):
 *   - potentials: FENE (Eq. 1), WCA (Eq. 2), harmonic theta-solvent bond (Sec. VI.B);
 *   - the move loop and Metropolis test (Sec. V, Eq. 20); no Jacobian (divergence-free);
 *   - tapered wavelet, w = p x grad(phi), phi = r^2/2 - r^3/3 - 1/6 (Sec. V.A, Eqs. 21-25),
 *     which gives the displacement  d = A_w (1 - |x|) (p x x),  x = (r - b)/lambda;
 *   - P_b (Eq. 26), A_w = A0 lambda / sqrt(n) (Eq. 29), P_lambda ~ lambda^-4 (Eq. 32);
 *   - time per accepted move (Eq. 34 wavelet-only, Eq. 57 wavelet + plane wave);
 *   - lambda_a = (2/pi) M4/M3 (Eq. 42) with the moments M_m of Eq. 22;
 *   - plane-wave moves (Sec. VI, Eqs. 47, 48, 51, 55, 56) and
 *   - the generation procedures of Appendix D (choice of move type, lambda by inverse
 *     transform, bead pick, uniform point in a ball by rejection, polarisation, n counted
 *     with one image, periodic k, phase and polarisation of a plane wave, recycling of
 *     lambda and |k| after a rejection, time advanced only on acceptance).
 *
 * Readings where the paper leaves a choice (a "sweep", the layered lambda schedule, the
 * colouring and deferral rule that define the order of moves, recycling per queue, the
 * random-number stream, the truncated periodic k set) are stated where they are used.
 *
 * Arithmetic contract: every quantity that changes a position is formed from IEEE
 * +, -, *, /, sqrt and explicit fma in a fixed order (see the comments at each step);
 * cube roots and cos/sin are evaluated by our own Newton iteration and Taylor polynomials
 * for that reason. Compile with -ffp-contract=off.
 */
#include <cmath>
#include <cstdint>
#include <cstring>
#include <cstdio>
#include <vector>
#include <algorithm>

namespace orc {

static const double PI = 3.141592653589793;
static const double TWO_PI = 6.283185307179586;
static const double LN2 = 0.6931471805599453;
static const double WCA_CUT = 1.122462048309373;   // 2^(1/6): WCA cutoff in units of sigma (Eq. 2)

/* ------------------------------------------------------------------------------------
 * Fourier transform of the scalar wavelet (Sec. V.A, Eq. 25) and its moments (Eq. 22).
 * ------------------------------------------------------------------------------------ */

// phi~(k) = 4 pi k^-6 (5 k sin k - (k^2 - 8) cos k - 8).  For small k the bracket cancels
// catastrophically, so there we use the power series of the same transform, obtained by
// expanding sin(kr)/(kr) inside  phi~(k) = 4 pi Int_0^1 phi(r) sin(kr)/(kr) r^2 dr  with
// phi(r) = r^2/2 - r^3/3 - 1/6 (Eq. 24):
//   phi~(k) = 4 pi Sum_j (-1)^j k^{2j}/(2j+1)! [1/(2(2j+5)) - 1/(3(2j+6)) - 1/(6(2j+3))].
double phitilde(double k) {
    k = std::fabs(k);
    if (k < 2.0) {
        double sum = 0.0, kp = 1.0, fact = 1.0;   // kp = k^{2j}, fact = (2j+1)!
        for (int j = 0; j < 30; j++) {
            if (j > 0) { kp *= k * k; fact *= (double)(2 * j) * (double)(2 * j + 1); }
            double c = 1.0 / (2.0 * (2 * j + 5)) - 1.0 / (3.0 * (2 * j + 6)) - 1.0 / (6.0 * (2 * j + 3));
            double term = kp / fact * c;
            sum += (j % 2 == 0) ? term : -term;
        }
        return 4.0 * PI * sum;
    }
    double k2 = k * k, k6 = k2 * k2 * k2;
    return 4.0 * PI * (5.0 * k * std::sin(k) - (k2 - 8.0) * std::cos(k) - 8.0) / k6;
}

// Gauss-Legendre nodes on [-1, 1] by Newton iteration on P_n.
static void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
    x.assign(n, 0.0); w.assign(n, 0.0);
    for (int i = 0; i < n; i++) {
        double z = std::cos(PI * (i + 0.75) / (n + 0.5)), pp = 0.0;
        for (int it = 0; it < 100; it++) {
            double p1 = 1.0, p2 = 0.0;
            for (int j = 1; j <= n; j++) { double p3 = p2; p2 = p1; p1 = ((2.0 * j - 1.0) * z * p2 - (j - 1.0) * p3) / j; }
            pp = n * (z * p1 - p2) / (z * z - 1.0);
            double dz = p1 / pp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        x[i] = z; w[i] = 2.0 / ((1.0 - z * z) * pp * pp);
    }
}

// Cut-off of the numerical k integrals: an even multiple of pi/2, so that the leading
// oscillatory part of the tail (~ sin 2K) vanishes; the smooth part of the tail is added
// in closed form from the large-k expansion of phi~^2 (Eq. 25 squared):
//   k^m phi~^2 = 16 pi^2 k^{m-12} [k^4/2 + 9/2 k^2 + 96 + (oscillating terms)].
static const int TAIL_PANELS = 20000;              // panels of width pi/8 up to K = 2500 pi
static double KMAX() { return TAIL_PANELS * (PI / 8.0); }

static double smooth_tail(int m, double K) {
    // Int_K^inf 16 pi^2 k^{m-12} (k^4/2 + 4.5 k^2 + 96) dk,  valid for m <= 6
    double c = 16.0 * PI * PI, s = 0.0;
    int p1 = m - 8, p2 = m - 10, p3 = m - 12;        // exponents
    s += 0.5 * std::pow(K, p1 + 1) / (-(p1 + 1));
    s += 4.5 * std::pow(K, p2 + 1) / (-(p2 + 1));
    s += 96.0 * std::pow(K, p3 + 1) / (-(p3 + 1));
    return c * s;
}

// M_m = Int_0^inf k^m phi~(k)^2 dk  (Eq. 22).
double moment(int m) {
    std::vector<double> gx, gw;
    gauss_legendre(16, gx, gw);
    double h = PI / 8.0, sum = 0.0;
    for (int p = 0; p < TAIL_PANELS; p++) {
        double a = p * h, c = a + 0.5 * h;
        for (int i = 0; i < 16; i++) {
            double k = c + 0.5 * h * gx[i], f = phitilde(k);
            sum += 0.5 * h * gw[i] * std::pow(k, m) * f * f;
        }
    }
    return sum + smooth_tail(m, KMAX());
}

// G(Q) = Int_Q^inf q^3 phi~(q)^2 dq, the weight of a plane-wave mode (Eqs. 49, 51).
// Evaluated for many Q at once: integrate panel by panel from K downwards.
void G_many(const std::vector<double>& Q, std::vector<double>& out) {
    std::vector<double> gx, gw;
    gauss_legendre(16, gx, gw);
    double h = PI / 8.0;
    auto seg = [&](double a, double b) {
        double s = 0.0, c = 0.5 * (a + b), hh = 0.5 * (b - a);
        for (int i = 0; i < 16; i++) { double k = c + hh * gx[i], f = phitilde(k); s += hh * gw[i] * k * k * k * f * f; }
        return s;
    };
    // cumulative integral from K down to each panel edge
    std::vector<double> from_edge(TAIL_PANELS + 1, 0.0);
    from_edge[TAIL_PANELS] = smooth_tail(3, KMAX());
    for (int p = TAIL_PANELS - 1; p >= 0; p--) from_edge[p] = from_edge[p + 1] + seg(p * h, (p + 1) * h);
    out.resize(Q.size());
    for (size_t i = 0; i < Q.size(); i++) {
        double q = Q[i];
        if (q >= KMAX()) { out[i] = smooth_tail(3, q); continue; }
        int p = (int)std::floor(q / h);
        double hi = (p + 1) * h;
        out[i] = from_edge[p + 1] + (hi > q ? seg(q, hi) : 0.0);
    }
}

/* ------------------------------------------------------------------------------------
 * Distribution of |k| for the infinite system and the quasi-continuous shell (Sec. VI.B,
 * Eqs. 52-53; Appendix D, choosing k). With Q = k lambda_max, P_k^inf is proportional to
 * Q^2 G(Q) with integral M6/3 (Eq. 53). Integrating by parts (G' = -Q^3 phi~^2),
 *     F(Q) = [Q^3 G(Q) + Int_0^Q q^6 phi~(q)^2 dq] / M6,
 * which is tabulated on Q_i = i KT_H up to Q_max = KT_N KT_H. The paper converts a uniform
 * number to k through a pre-computed table with interpolation; here: linear interpolation of
 * F^(1/3) between the grid points (exact for the leading F ~ Q^3 G(0)/M6 at small Q, where
 * the amplitude A_F ~ 1/k is largest), and beyond Q_max the Q^-1 tail of 1 - F that
 * G ~ 2 pi^2 Q^-4 gives, matched at Q_max.
 * ------------------------------------------------------------------------------------ */
static const int KT_N = 8192;
static const double KT_H = PI / 128.0;
static const double M6_EXACT = 8.0 * PI * PI * PI / 5.0;   // (2 pi)^3 / 5, pinned against quadrature

static void k_cdf_table(std::vector<double>& F) {
    std::vector<double> Q(KT_N + 1), Gv, gx, gw;
    for (int i = 0; i <= KT_N; i++) Q[i] = i * KT_H;
    G_many(Q, Gv);
    gauss_legendre(16, gx, gw);
    F.assign(KT_N + 1, 0.0);
    double cum = 0.0, comp = 0.0;             // compensated (Kahan) running sum over the panels
    for (int i = 1; i <= KT_N; i++) {
        double a = Q[i - 1], c = a + 0.5 * KT_H, panel = 0.0;
        for (int k = 0; k < 16; k++) {
            double q = c + 0.5 * KT_H * gx[k], f = phitilde(q);
            double q3 = q * q * q;
            panel += 0.5 * KT_H * gw[k] * (q3 * q3) * f * f;
        }
        double y = panel - comp, t = cum + y;
        comp = (t - cum) - y;
        cum = t;
        F[i] = (Q[i] * Q[i] * Q[i] * Gv[i] + cum) / M6_EXACT;
    }
}
// F(Q) by direct quadrature (no table): the normalisation of the shell uses it
static double k_cdf_exact(double Q) {
    std::vector<double> gx, gw, Gv;
    gauss_legendre(16, gx, gw);
    int panels = (int)std::ceil(Q / KT_H);
    double cum = 0.0, comp = 0.0;
    for (int p = 0; p < panels; p++) {
        double a = p * KT_H, b = std::min(Q, (p + 1) * KT_H), c = 0.5 * (a + b), hh = 0.5 * (b - a), panel = 0.0;
        for (int k = 0; k < 16; k++) {
            double q = c + hh * gx[k], f = phitilde(q), q3 = q * q * q;
            panel += hh * gw[k] * (q3 * q3) * f * f;
        }
        double y = panel - comp, t = cum + y;
        comp = (t - cum) - y;
        cum = t;
    }
    G_many(std::vector<double>{Q}, Gv);
    return (Q * Q * Q * Gv[0] + cum) / M6_EXACT;
}
// F of the table (F^(1/3) linear between grid points; the Q^-1 tail beyond Q_max)
static double k_cdf_interp(const std::vector<double>& F, double Q) {
    if (Q >= KT_N * KT_H) return 1.0 - (1.0 - F[KT_N]) * (KT_N * KT_H) / Q;
    int i = (int)(Q / KT_H);
    if (i >= KT_N) i = KT_N - 1;
    double a = std::cbrt(F[i]), b = std::cbrt(F[i + 1]);
    double t = a + (b - a) * ((Q - i * KT_H) / KT_H);
    return (t * t) * t;
}
// inverse of the tabulated F for u in (0, 1): the largest i with F_i <= u, then
// Q = Q_i + KT_H (u^(1/3) - F_i^(1/3)) / (F_{i+1}^(1/3) - F_i^(1/3))
static double k_inverse(const std::vector<double>& F, double u) {
    if (u >= F[KT_N]) return (KT_N * KT_H) * ((1.0 - F[KT_N]) / (1.0 - u));
    int i = (int)(std::upper_bound(F.begin(), F.end(), u) - F.begin()) - 1;
    if (i < 0) i = 0;
    if (i >= KT_N) i = KT_N - 1;
    double a = std::cbrt(F[i]), b = std::cbrt(F[i + 1]);
    return i * KT_H + KT_H * ((std::cbrt(u) - a) / (b - a));
}

// Solid angle of the directions n with |n_x|, |n_y|, |n_z| <= t (t <= 1). For t >= 1/sqrt(2)
// the sphere loses six caps that do not overlap, each of solid angle 2 pi (1 - t):
// 4 pi - 12 pi (1 - t). Below, by Archimedes the area is uniform in n_z; at height n_z the
// circle of radius rho = sqrt(1 - n_z^2) keeps the angle 2 pi - 8 arccos(t / rho) inside the
// square |n_x|, |n_y| <= t while rho <= t sqrt 2 (none beyond), and rho > t on all of
// |n_z| <= t: a smooth integrand from n_z = sqrt(1 - 2 t^2) to t.
static double solid_angle_in_cube(double t) {
    if (2.0 * t * t >= 1.0) return 4.0 * PI - 12.0 * PI * (1.0 - std::min(t, 1.0));
    if (3.0 * t * t <= 1.0) return 0.0;
    std::vector<double> gx, gw;
    gauss_legendre(16, gx, gw);
    double a = std::sqrt(1.0 - 2.0 * t * t), b = t, sum = 0.0;
    for (int p = 0; p < 16; p++) {
        double pa = a + (b - a) * p / 16.0, pb = a + (b - a) * (p + 1) / 16.0, c = 0.5 * (pa + pb), hh = 0.5 * (pb - pa);
        for (int k = 0; k < 16; k++) {
            double z = c + hh * gx[k], rho = std::sqrt(1.0 - z * z);
            sum += hh * gw[k] * (TWO_PI - 8.0 * std::acos(t / rho));
        }
    }
    return 2.0 * sum;                                                     // n_z and -n_z
}

/* ------------------------------------------------------------------------------------
 * Random numbers. The paper only says "a pseudo random number generator" (App. D).
 * Reading: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), counter-based, so that
 * every draw is a pure function of (seed, simulation, sweep, layer, slot, attempt).
 * ------------------------------------------------------------------------------------ */
struct U4 { uint32_t v[4]; };

U4 philox(U4 c, uint32_t k0, uint32_t k1) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    for (int r = 0; r < 10; r++) {
        uint64_t p0 = (uint64_t)M0 * c.v[0], p1 = (uint64_t)M1 * c.v[2];
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0, hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        U4 n;
        n.v[0] = hi1 ^ c.v[1] ^ k0;
        n.v[1] = lo1;
        n.v[2] = hi0 ^ c.v[3] ^ k1;
        n.v[3] = lo0;
        c = n;
        k0 += W0; k1 += W1;
    }
    return c;
}

// stream kinds (bits 24..31 of counter word 2)
enum { K_COUNT = 1, K_SLOT = 2, K_VB = 3, K_VP = 4, K_ACC = 5, K_PWCOUNT = 6, K_PWMODE = 7, K_PWDIR = 8,
       K_PWACC = 9, K_DPWMODE = 10, K_DPWDIR = 11, K_DPWACC = 12, K_PROPOSE = 13,
       K_PWSHELL = 14, K_PWKDIR = 15, K_DPWSHELL = 16, K_DPWKDIR = 17, K_BUNI = 18 };

struct Stream {
    uint32_t k0, k1;
    // counter = (index, sweep lo, kind<<24 | layer<<16 | attempt, sweep hi)
    U4 draw(int kind, int layer, uint64_t sweep, uint32_t index, uint32_t attempt) const {
        U4 c;
        c.v[0] = index;
        c.v[1] = (uint32_t)sweep;
        c.v[2] = ((uint32_t)kind << 24) | ((uint32_t)(layer & 0xFF) << 16) | (attempt & 0xFFFFu);
        c.v[3] = (uint32_t)(sweep >> 32);
        return philox(c, k0, k1);
    }
};
static Stream make_stream(uint64_t seed, uint64_t sim_id) {
    Stream s;
    s.k0 = (uint32_t)seed;
    s.k1 = (uint32_t)(seed >> 32) ^ (uint32_t)sim_id;
    return s;
}
// uniform in [0, 1) with 53 random bits
static double u53(uint32_t hi, uint32_t lo) {
    uint64_t m = ((uint64_t)(hi >> 5) << 26) | (uint64_t)(lo >> 6);
    return (double)m * (1.0 / 9007199254740992.0);
}
// uniform in (0, 1): the same 53 bits with the lowest forced to 1 (never 0, never 1)
static double u_open(uint32_t hi, uint32_t lo) {
    uint64_t m = ((uint64_t)(hi >> 5) << 26) | (uint64_t)(lo >> 6);
    return (double)(m | 1u) * (1.0 / 9007199254740992.0);
}
// uniform integer in [0, n): high 64 bits of (64-bit draw) * n
static int64_t pick(uint32_t hi, uint32_t lo, int64_t n) {
    uint64_t x = ((uint64_t)hi << 32) | lo;
    return (int64_t)(((unsigned __int128)x * (unsigned __int128)(uint64_t)n) >> 64);
}
// component of a point of [-1, 1)^3
static double sym(uint32_t w) { return (double)w * (1.0 / 2147483648.0) - 1.0; }

/* ------------------------------------------------------------------------------------
 * Own elementary functions (fixed operation order, explicit fma).
 * ------------------------------------------------------------------------------------ */
// lambda = w^(-1/3) by 8 Newton steps on f(y) = y^-3 - w from the lower edge `lo` of the
// band that contains the root (the band spans at most a factor 2, Newton from below is
// monotone): y <- y (4 - w y^3) / 3.
static double inv_cbrt_from(double w, double lo) {
    double y = lo;
    for (int it = 0; it < 8; it++) {
        double t = w * ((y * y) * y);
        y = (y * (4.0 - t)) / 3.0;
    }
    return y;
}
// Taylor coefficients of cos and sin about 0, evaluated on [0, pi/4]
static double cos_poly(double t) {
    double z = t * t;
    double c = 1.0 / 6402373705728000.0;                             // 1/18!
    c = std::fma(c, -z, 1.0 / 20922789888000.0);                      // 1/16!
    c = std::fma(c, -z, 1.0 / 87178291200.0);                         // 1/14!
    c = std::fma(c, -z, 1.0 / 479001600.0);                           // 1/12!
    c = std::fma(c, -z, 1.0 / 3628800.0);                             // 1/10!
    c = std::fma(c, -z, 1.0 / 40320.0);                               // 1/8!
    c = std::fma(c, -z, 1.0 / 720.0);
    c = std::fma(c, -z, 1.0 / 24.0);
    c = std::fma(c, -z, 0.5);
    c = std::fma(c, -z, 1.0);
    return c;
}
static double sin_poly(double t) {
    double z = t * t;
    double c = 1.0 / 121645100408832000.0;                           // 1/19!
    c = std::fma(c, -z, 1.0 / 355687428096000.0);                     // 1/17!
    c = std::fma(c, -z, 1.0 / 1307674368000.0);                       // 1/15!
    c = std::fma(c, -z, 1.0 / 6227020800.0);                          // 1/13!
    c = std::fma(c, -z, 1.0 / 39916800.0);                            // 1/11!
    c = std::fma(c, -z, 1.0 / 362880.0);                              // 1/9!
    c = std::fma(c, -z, 1.0 / 5040.0);
    c = std::fma(c, -z, 1.0 / 120.0);
    c = std::fma(c, -z, 1.0 / 6.0);
    c = std::fma(c, -z, 1.0);
    return c * t;
}
// cos(2 pi t) and sin(2 pi t) for t in turns: reduce to [0, 1/2] by symmetry, then to an
// octant (all reductions are exact by Sterbenz), then one Taylor polynomial.
static double cos2pi(double t) {
    double x = t - std::floor(t);                 // [0, 1)
    if (x > 0.5) x = 1.0 - x;                      // cos symmetric about 1/2
    if (x <= 0.125) return cos_poly(TWO_PI * x);
    if (x <= 0.375) return sin_poly(TWO_PI * (0.25 - x));
    return -cos_poly(TWO_PI * (0.5 - x));
}
static double sin2pi(double t) {
    double x = t - std::floor(t);                 // [0, 1)
    double sgn = 1.0;
    if (x >= 0.5) { x = x - 0.5; sgn = -1.0; }     // sin(2pi(x+1/2)) = -sin(2pi x)
    if (x > 0.25) x = 0.5 - x;                     // symmetric about 1/4
    double r = (x <= 0.125) ? sin_poly(TWO_PI * x) : cos_poly(TWO_PI * (0.25 - x));
    return sgn * r;
}
// single-precision variants for the mixed-precision displacement (reduction in FP64)
static float cos_poly_f(float t) {
    float z = t * t;
    float c = 1.0f / 3628800.0f;                   // 1/10!
    c = std::fma(c, -z, 1.0f / 40320.0f);
    c = std::fma(c, -z, 1.0f / 720.0f);
    c = std::fma(c, -z, 1.0f / 24.0f);
    c = std::fma(c, -z, 0.5f);
    c = std::fma(c, -z, 1.0f);
    return c;
}
static float sin_poly_f(float t) {
    float z = t * t;
    float c = 1.0f / 39916800.0f;                  // 1/11!
    c = std::fma(c, -z, 1.0f / 362880.0f);
    c = std::fma(c, -z, 1.0f / 5040.0f);
    c = std::fma(c, -z, 1.0f / 120.0f);
    c = std::fma(c, -z, 1.0f / 6.0f);
    c = std::fma(c, -z, 1.0f);
    return c * t;
}
static float cos2pi_f(double t) {
    double x = t - std::floor(t);
    if (x > 0.5) x = 1.0 - x;
    if (x <= 0.125) return cos_poly_f((float)(TWO_PI * x));
    if (x <= 0.375) return sin_poly_f((float)(TWO_PI * (0.25 - x)));
    return -cos_poly_f((float)(TWO_PI * (0.5 - x)));
}

}  // namespace orc

/* ====================================================================================
 * Simulation state
 * ==================================================================================== */
extern "C" {
// Parameters of one simulation (lengths in units of the bead radius a, energies in kT units
// when kT = 1). Mirrors the product's parameter block field by field but is declared here
// on its own.
typedef struct OParams {
    int64_t n_beads;
    double box_L;
    double lambda_min, lambda_max, A0, kT;
    int32_t bond_type;            // 0 none, 1 harmonic (k/2)(r - r0)^2, 2 FENE (Eq. 1)
    double bond_k, bond_r0, fene_R0;
    double wca_sigma, wca_eps;    // WCA (Eq. 2); eps = 0 disables it
    double ext_kappa;             // external well (kappa/2)|r - centre|^2, 0 disables it
    int32_t planewave_mode;       // 0 off (wavelets only), 1 periodic plane waves
    int32_t lcut;                 // plane-wave modes |l| <= lcut
    int32_t precision;            // 0 FP64, 1 mixed (FP32 displacement, FP64 decision)
    uint64_t seed, sim_id;
    int32_t colour_K;             // colours per axis of the concurrent schedule (2..4)
    int32_t grid_f;               // fine cells per axis
    int32_t n_cap;                // largest support handled by a concurrent move
    int32_t grid_layer[16];       // coarse cells per axis per layer, 0 = serial layer
    int32_t big_support;          // a launch choice of the GPU library; no meaning here
    int32_t acceptance;           // 0 Metropolis (Eq. 20), 1 Glauber
    int32_t centring;             // 0 centre near a picked bead (Eq. 26), 1 uniform in the box (Sec. V.D)
    int32_t level2;               // bit l: layer l's deferred slots get a second colouring on a grid half as fine
} OParams;

typedef struct OStats {
    int64_t attempts[16], accepts[16], deferred[16];
    int64_t pw_attempts, pw_accepts;
    int64_t bead_updates;
    int64_t accepted_total;
    double sim_time;
    int64_t sweeps;
    int64_t n_layers;
    double dt_move, p_fourier;
    int64_t moved_beads;          // beads moved by accepted moves (support sizes; N per plane wave)
} OStats;
}

namespace orc {

enum { ACCEPT = 1, REJECT = 2, DEFER = 3 };

struct Layer {
    double lo, hi;        // band [lo, hi) of lambda
    double ilo3, ihi3;    // lo^-3, hi^-3
    double mass;          // p_l: probability of the band under P_lambda (Eq. 32)
    double expect;        // expected slots per sweep, N (1 - P_F) p_l
    int G;                // coarse cells per axis, 0 = serial
};

struct Sim {
    OParams P;
    int64_t N;
    double L, halfL, invf;
    std::vector<double> pos;      // 3N, wrapped into [0, L)
    std::vector<int32_t> img;     // 3N image counters
    std::vector<uint8_t> bnext;   // bead i bonded to i+1
    std::vector<Layer> layers;
    Stream rng;
    uint64_t sweep = 0;
    uint64_t pw_calls = 0;
    double rc2 = 0.0, rc = 0.0;   // WCA cutoff
    double r_reach = 0.0;         // spatial reach of interactions used by the region rule
    double dt_move = 0.0;         // simulated time per accepted move (units of tau)
    double p_fourier = 0.0;
    // carries of lambda after a rejection (Appendix D, parameter recycling)
    std::vector<std::vector<double>> carry_q;   // per layer, per coarse cell (0 = none)
    std::vector<std::vector<double>> carry_q2;  // per layer, per cell of the second-level grid
    std::vector<double> carry_serial;           // per layer
    int pw_carry = -1;                          // carried plane-wave mode (index), -1 none
    int pw_carry_l[3] = {0, 0, 0};
    double pw_carry_Q = 0.0;                    // infinite system: carried |k| lambda_max
    // full periodic scheme (discrete cube + quasi-continuous shell) and infinite system
    std::vector<double> kF;                     // tabulated F(Q), Q = |k| lambda_max
    double kF0 = 0.0;                           // F at the shell's inner edge (periodic full)
    double p_disc = 1.0;                        // probability of the discrete cube (periodic full)
    double z_cube = 0.0, z_shell = 0.0;         // the two parts of the mode normalisation
    std::vector<double> tr_pw_k;                // 3 per traced plane wave, in units of 2 pi / L
    // plane-wave tables
    std::vector<int> modes;                     // 3 per mode
    std::vector<double> mode_prob, mode_cdf;
    double R = 1.0;
    // statistics and per-slot trace of the last sweep
    OStats st;
    std::vector<std::vector<uint8_t>> tr_out;
    std::vector<std::vector<int32_t>> tr_n;
    std::vector<std::vector<double>> tr_du;
    std::vector<std::vector<double>> tr_lam;    // the lambda each slot's attempt used (its own or a carry)
    double last_du = 0.0, last_lam = 0.0;
    std::vector<uint8_t> tr_pw_out;
    std::vector<int32_t> tr_pw_mode;
    // scratch
    std::vector<uint8_t> inS;
    // wavelet attempts left before the current sweep is cut short (-1: no limit); only for
    // timing a bounded sample of a sweep, never set by the tests of the method
    int64_t move_budget = -1;
};

static inline double wrap(double x, double L, int32_t* im) {
    if (x >= L) { x = x - L; if (im) *im += 1; }
    else if (x < 0.0) { x = x + L; if (im) *im -= 1; }
    if (x >= L) x = 0.0;          // a tiny negative value rounded up to L
    return x;
}
static inline double mi(double d, double L, double h) {
    if (d > h) d = d - L;
    else if (d < -h) d = d + L;
    return d;
}

/* ---- energies (Eqs. 1, 2; harmonic bond of Sec. VII.B; external well for tests) ---- */
static double U_wca(const Sim& s, double r2) {
    if (s.P.wca_eps == 0.0 || !(r2 < s.rc2)) return 0.0;
    double s2 = (s.P.wca_sigma * s.P.wca_sigma) / r2;
    double s6 = (s2 * s2) * s2;
    return 4.0 * s.P.wca_eps * (s6 * s6 - s6) + s.P.wca_eps;
}
static double U_bond(const Sim& s, double r2) {
    if (s.P.bond_type == 1) {
        double r = std::sqrt(r2), d = r - s.P.bond_r0;
        return 0.5 * s.P.bond_k * d * d;
    }
    if (s.P.bond_type == 2) {
        double R02 = s.P.fene_R0 * s.P.fene_R0, x = r2 / R02;
        if (!(x < 1.0)) return INFINITY;
        return -0.5 * s.P.bond_k * R02 * std::log(1.0 - x);
    }
    return 0.0;
}
static double U_ext(const Sim& s, const double* p) {
    if (s.P.ext_kappa == 0.0) return 0.0;
    double r2 = 0.0;
    for (int a = 0; a < 3; a++) { double d = mi(p[a] - s.halfL, s.L, s.halfL); r2 += d * d; }
    return 0.5 * s.P.ext_kappa * r2;
}
static inline double dist2(const Sim& s, const double* p, const double* q) {
    double dx = mi(p[0] - q[0], s.L, s.halfL), dy = mi(p[1] - q[1], s.L, s.halfL), dz = mi(p[2] - q[2], s.L, s.halfL);
    return (dx * dx + dy * dy) + dz * dz;
}
static inline bool bonded(const Sim& s, int64_t i, int64_t j) {
    if (j == i + 1) return s.bnext[i];
    if (i == j + 1) return s.bnext[j];
    return false;
}
static double U_pair(const Sim& s, int64_t i, int64_t j, const double* p, const double* q) {
    double r2 = dist2(s, p, q);
    double u = U_wca(s, r2);
    if (bonded(s, i, j)) u += U_bond(s, r2);
    return u;
}

// Energy change when the beads in `S` move from `pos` to `newp` (3 per entry of S).
// Brute force over all partners: every pair with at least one moved bead, counted once.
static double delta_U(Sim& s, const std::vector<int64_t>& S, const std::vector<double>& newp) {
    for (size_t k = 0; k < S.size(); k++) s.inS[S[k]] = 1;
    // map from bead to its index in S (only for moved beads)
    std::vector<std::pair<int64_t, size_t>> idx(S.size());
    for (size_t k = 0; k < S.size(); k++) idx[k] = {S[k], k};
    std::sort(idx.begin(), idx.end());
    auto where = [&](int64_t b) {
        auto it = std::lower_bound(idx.begin(), idx.end(), std::make_pair(b, (size_t)0));
        return it->second;
    };
    double dU = 0.0;
    for (size_t k = 0; k < S.size(); k++) {
        int64_t m = S[k];
        const double* om = &s.pos[3 * m];
        const double* nm = &newp[3 * k];
        dU += U_ext(s, nm) - U_ext(s, om);
        for (int64_t q = 0; q < s.N; q++) {
            if (q == m) continue;
            const double* oq = &s.pos[3 * q];
            if (s.inS[q]) {
                if (q < m) continue;                 // pair of two moved beads: counted once
                const double* nq = &newp[3 * where(q)];
                dU += U_pair(s, m, q, nm, nq) - U_pair(s, m, q, om, oq);
            } else {
                dU += U_pair(s, m, q, nm, oq) - U_pair(s, m, q, om, oq);
            }
        }
    }
    for (size_t k = 0; k < S.size(); k++) s.inS[S[k]] = 0;
    return dU;
}

// Acceptance test on the draw w. Metropolis (Eq. 20): accept with probability
// min(1, exp(-dU/kT)), i.e. iff dU <= -kT ln(1 - u) with u uniform in [0, 1). Glauber (the
// paper's proposed alternative, Secs. V.C and VIII): accept with probability
// 1 / (1 + exp(dU/kT)), i.e. iff dU <= kT (ln(1 - u) - ln u) with u uniform in (0, 1).
// An infinite or undefined dU rejects.
static double accept_threshold(const Sim& s, const U4& w) {
    if (s.P.acceptance == 1) {
        double u = u_open(w.v[0], w.v[1]);
        return s.P.kT * (std::log(1.0 - u) - std::log(u));
    }
    return -s.P.kT * std::log(1.0 - u53(w.v[0], w.v[1]));
}
static bool metropolis(const Sim& s, double dU, const U4& w) {
    return dU <= accept_threshold(s, w);
}

/* ---- proposal parameters (Appendix D) ---- */
// Uniform point of the closed unit ball by rejection from [-1, 1)^3 (Appendix D, choosing b).
// Attempts are counter-indexed; after 64 failed attempts (probability 0.48^64) the centre
// is used.
static void ball_point(const Sim& s, int kind, int layer, uint64_t sweep, uint32_t j, double V[3], bool nonzero) {
    for (uint32_t a = 0; a < 64; a++) {
        U4 w = s.rng.draw(kind, layer, sweep, j, a);
        double x = sym(w.v[0]), y = sym(w.v[1]), z = sym(w.v[2]);
        double q = (x * x + y * y) + z * z;
        if (q <= 1.0 && (!nonzero || q > 0.0)) { V[0] = x; V[1] = y; V[2] = z; return; }
    }
    V[0] = 0.0; V[1] = 0.0; V[2] = nonzero ? 1.0 : 0.0;
}
// Isotropic polarisation p = V / |V| (Appendix D, choosing p).
static void polarisation(const Sim& s, int layer, uint64_t sweep, uint32_t j, double p[3]) {
    double V[3];
    ball_point(s, K_VP, layer, sweep, j, V, true);
    double q = (V[0] * V[0] + V[1] * V[1]) + V[2] * V[2];
    double r = std::sqrt(q);
    p[0] = V[0] / r; p[1] = V[1] / r; p[2] = V[2] / r;
}

// Centre uniform in the box (Sec. V.D, the homogeneous alternative with P_b = 1/L^3): each
// coordinate L times a 32-bit uniform of the slot's own draw.
static void uniform_centre(const Sim& s, int l, uint64_t sweep, uint32_t j, double b[3]) {
    U4 w = s.rng.draw(K_BUNI, l, sweep, j, 0);
    for (int a = 0; a < 3; a++) b[a] = s.L * ((double)w.v[a] * (1.0 / 4294967296.0));
}
// Amplitude of a wavelet move: A_w = A0 lam / sqrt(n) (Eq. 29) for a bead-centred move; with a
// uniform centre n is replaced by its mean at the global density, N (4 pi / 3) lam^3 / L^3
// (Sec. V.D: the mean count; this reading gives P_b A_w^2 = 3 A0^2 / (4 pi N lam) as Eq. 29 does).
static double wavelet_amplitude(const Sim& s, double lam, int n) {
    if (s.P.centring == 1) {
        double nbar = ((double)s.N * ((4.0 * PI / 3.0) * ((lam * lam) * lam))) / ((s.L * s.L) * s.L);
        return (s.P.A0 * lam) / std::sqrt(nbar);
    }
    return (s.P.A0 * lam) / std::sqrt((double)n);
}

// Displacement of a bead at minimum-image offset d from the centre (Sec. V.A):
//   delta = A_w (1 - |x|) (p x x),  x = d / lambda,
// evaluated as  s = (A_w (1 - sqrt(d2)/lambda)) / lambda,  delta = s (p x d).
static void wavelet_disp(const Sim& s, const double d[3], double d2, double lam, double Aw, const double p[3],
                         double out[3]) {
    if (s.P.precision == 0) {
        double rho = std::sqrt(d2) / lam;
        double sc = (Aw * (1.0 - rho)) / lam;
        double cx = p[1] * d[2] - p[2] * d[1];
        double cy = p[2] * d[0] - p[0] * d[2];
        double cz = p[0] * d[1] - p[1] * d[0];
        out[0] = sc * cx; out[1] = sc * cy; out[2] = sc * cz;
    } else {
        // mixed precision: the same expression in binary32 on FP64 inputs rounded once
        float dx = (float)d[0], dy = (float)d[1], dz = (float)d[2];
        float d2f = (dx * dx + dy * dy) + dz * dz;
        float lf = (float)lam, af = (float)Aw, px = (float)p[0], py = (float)p[1], pz = (float)p[2];
        float rho = std::sqrt(d2f) / lf;
        float sc = (af * (1.0f - rho)) / lf;
        float cx = py * dz - pz * dy;
        float cy = pz * dx - px * dz;
        float cz = px * dy - py * dx;
        out[0] = (double)(sc * cx); out[1] = (double)(sc * cy); out[2] = (double)(sc * cz);
    }
}

/* ---- the concurrency region of a coarse cell (our schedule; the paper runs moves one
 *      after another and names parallel non-overlapping moves as future work, Sec. VIII) ----
 * A coloured layer splits the box into G^3 coarse cells, coloured by (cx mod K, cy mod K,
 * cz mod K). The region of a cell is the cell widened by (K-1)/2 cells on every side; the
 * regions of one colour tile the box. A move of the queue of cell C may run concurrently
 * with the other queues of its colour only if everything it reads or writes lies in fine
 * cells wholly inside C's region; otherwise it is deferred to the serial phase. */
static inline int64_t floordiv(int64_t a, int64_t b) { int64_t q = a / b; if ((a % b != 0) && ((a < 0) != (b < 0))) q--; return q; }
static inline int64_t ceildiv(int64_t a, int64_t b) { return -floordiv(-a, b); }

struct Region { int64_t lo[3], hi[3]; };   // inclusive fine-cell index ranges (may exceed [0, Gf))

static Region region_of(const Sim& s, int G, const int c[3]) {
    Region R;
    int64_t K = s.P.colour_K, Gf = s.P.grid_f;
    for (int a = 0; a < 3; a++) {
        R.lo[a] = ceildiv((2 * (int64_t)c[a] - (K - 1)) * Gf, 2 * (int64_t)G);
        R.hi[a] = floordiv((2 * (int64_t)c[a] + 2 + (K - 1)) * Gf, 2 * (int64_t)G) - 1;
    }
    return R;
}
static inline bool range_inside(int64_t t0, int64_t t1, int64_t lo, int64_t hi, int64_t Gf) {
    for (int64_t sh = -Gf; sh <= Gf; sh += Gf)
        if (t0 + sh >= lo && t1 + sh <= hi) return true;
    return false;
}
static inline int64_t fine_cell(const Sim& s, double x) {
    int64_t c = (int64_t)std::floor(x * s.invf);
    if (c < 0) c = 0;
    if (c >= s.P.grid_f) c = s.P.grid_f - 1;
    return c;
}
// The influence ball of a move centred at b with scale lam: everything read or written is
// within R = lam + A0 lam / 4 + r_reach of b (|delta| <= A_w / 4 <= A0 lam / 4).
static bool ball_inside(const Sim& s, const Region& Rg, const double b[3], double lam) {
    double R = (lam + (0.25 * s.P.A0) * lam) + s.r_reach;
    for (int a = 0; a < 3; a++) {
        int64_t t0 = (int64_t)std::floor((b[a] - R) * s.invf);
        int64_t t1 = (int64_t)std::floor((b[a] + R) * s.invf);
        if (!range_inside(t0, t1, Rg.lo[a], Rg.hi[a], s.P.grid_f)) return false;
    }
    return true;
}
static bool point_inside(const Sim& s, const Region& Rg, const double* p) {
    for (int a = 0; a < 3; a++) {
        int64_t c = fine_cell(s, p[a]);
        if (!range_inside(c, c, Rg.lo[a], Rg.hi[a], s.P.grid_f)) return false;
    }
    return true;
}

// One wavelet move (Sec. V and Appendix D): slot j of layer l in the current sweep, with
// scale lam (own draw or the carried scale of a rejected move). `Rg` is the concurrency
// region when the move runs in a coloured phase, null in the serial phase.
// Returns ACCEPT, REJECT or DEFER; n receives the number of beads in the support.
static int wavelet_attempt(Sim& s, int l, uint32_t j, int64_t i, double lam, const Region* Rg, int* n_out,
                           int ncap) {
    const uint64_t sw = s.sweep;
    s.last_du = 0.0;
    s.last_lam = lam;
    // centre: b = r_i + lam V, V uniform in the unit ball (wrapped into the box); or uniform in
    // the box
    double V[3], b[3];
    if (s.P.centring == 1) uniform_centre(s, l, sw, j, b);
    else {
        ball_point(s, K_VB, l, sw, j, V, false);
        for (int a = 0; a < 3; a++) b[a] = wrap(s.pos[3 * i + a] + lam * V[a], s.L, nullptr);
    }
    if (Rg && !ball_inside(s, *Rg, b, lam)) return DEFER;
    // support: beads strictly inside the ball, one image each (lam <= L/2)
    std::vector<int64_t> S;
    std::vector<double> D;   // offsets d = mi(r - b), 4 per member (d, d2)
    double lam2 = lam * lam;
    for (int64_t m = 0; m < s.N; m++) {
        double d[3];
        for (int a = 0; a < 3; a++) d[a] = mi(s.pos[3 * m + a] - b[a], s.L, s.halfL);
        double d2 = (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2];
        if (d2 < lam2) { S.push_back(m); D.insert(D.end(), {d[0], d[1], d[2], d2}); }
    }
    int n = (int)S.size();
    *n_out = n;
    if (Rg && n > ncap) return DEFER;
    double p[3];
    polarisation(s, l, sw, j, p);
    // amplitude A_w = A0 lam / sqrt(n)  (Eq. 29) and the new positions
    std::vector<double> newp(3 * (size_t)n);
    std::vector<int32_t> newimg(3 * (size_t)n);
    if (n > 0) {
        double Aw = wavelet_amplitude(s, lam, n);
        for (int k = 0; k < n; k++) {
            double dl[3];
            wavelet_disp(s, &D[4 * k], D[4 * k + 3], lam, Aw, p, dl);
            for (int a = 0; a < 3; a++) {
                int32_t im = s.img[3 * S[k] + a];
                newp[3 * k + a] = wrap(s.pos[3 * S[k] + a] + dl[a], s.L, &im);
                newimg[3 * k + a] = im;
            }
        }
    }
    // bonded partners outside the support must lie in the region too
    if (Rg) {
        for (int k = 0; k < n; k++) {
            int64_t m = S[k];
            for (int e = 0; e < 2; e++) {
                int64_t q = (e == 0) ? m - 1 : m + 1;
                if (q < 0 || q >= s.N || !bonded(s, m, q)) continue;
                bool in = std::find(S.begin(), S.end(), q) != S.end();
                if (!in && !point_inside(s, *Rg, &s.pos[3 * q])) return DEFER;
            }
        }
    }
    double dU = n > 0 ? delta_U(s, S, newp) : 0.0;
    s.last_du = dU;
    U4 w = s.rng.draw(K_ACC, l, sw, j, 0);
    bool acc = metropolis(s, dU, w);
    if (acc) {
        for (int k = 0; k < n; k++)
            for (int a = 0; a < 3; a++) { s.pos[3 * S[k] + a] = newp[3 * k + a]; s.img[3 * S[k] + a] = newimg[3 * k + a]; }
    }
    return acc ? ACCEPT : REJECT;
}

}  // namespace orc

namespace orc {

/* ---- slot parameters: scale within the layer's band and the picked bead ----
 * Eq. 32 restricted to the band [lo, hi):  lambda = (lo^-3 - u (lo^-3 - hi^-3))^(-1/3),
 * the inverse transform of Appendix D applied to one octave; the bead is uniform. */
static void slot_draw(const Sim& s, int l, uint64_t sweep, uint32_t j, double* lam, int64_t* bead) {
    const Layer& L = s.layers[l];
    U4 w = s.rng.draw(K_SLOT, l, sweep, j, 0);
    double u = u53(w.v[0], w.v[1]);
    double wv = L.ilo3 - u * (L.ilo3 - L.ihi3);
    *lam = inv_cbrt_from(wv, L.lo);
    *bead = pick(w.v[2], w.v[3], s.N);
}
// Number of slots: floor(x) plus one more with probability frac(x) (stratified count).
static int64_t slot_count(const Sim& s, int kind, int l, uint64_t ctr, double x) {
    U4 w = s.rng.draw(kind, l, ctr, 0, 0);
    double u = u53(w.v[0], w.v[1]);
    double f = std::floor(x);
    return (int64_t)f + ((u < x - f) ? 1 : 0);
}

/* ---- second-level grid of coloured layer l: K floor(G / 2K) coarse cells per axis when that
 *      leaves at least two per colour and axis and the run asks for it, else none ---- */
static const int SECOND_NCAP = 256;
static int level2_grid(const Sim& s, int l, int G) {
    if (!((s.P.level2 >> l) & 1) || G <= 0) return 0;
    const int K = s.P.colour_K, G2 = K * (G / (2 * K));
    return G2 >= 2 * K ? G2 : 0;
}

/* ---- one layer: coloured phases then the serial phase ---- */
static void run_layer(Sim& s, int l) {
    const Layer& Ly = s.layers[l];
    const uint64_t sw = s.sweep;
    int64_t M = slot_count(s, K_COUNT, l, sw, Ly.expect);
    std::vector<double> lam(M);
    std::vector<int64_t> bead(M);
    for (int64_t j = 0; j < M; j++) slot_draw(s, l, sw, (uint32_t)j, &lam[j], &bead[j]);
    s.tr_out[l].assign(M, 0);
    s.tr_n[l].assign(M, 0);
    s.tr_du[l].assign(M, 0.0);
    s.tr_lam[l].assign(M, 0.0);
    std::vector<int64_t> serial;
    // flags: 4 = deferred from the first colouring, 8 = deferred from the second as well
    bool second = false;
    auto record = [&](int64_t j, int r, int n, int flags) {
        s.tr_out[l][j] = (uint8_t)((r == ACCEPT ? 1 : 2) | flags);
        s.tr_n[l][j] = n;
        s.tr_du[l][j] = s.last_du;
        s.tr_lam[l][j] = s.last_lam;
        s.st.attempts[l]++;
        s.st.bead_updates += n;
        if (r == ACCEPT) { s.st.accepts[l]++; s.st.accepted_total++; s.st.moved_beads += n; }
    };
    const int G = Ly.G;
    if (G > 0) {
        // bucket the slots by the coarse cell of their bead at the start of the layer;
        // order: colour, then cell (ascending linear index within the colour), then slot
        const int K = s.P.colour_K, Q = G / K;
        const int64_t nq3 = (int64_t)Q * Q * Q;
        const double invG = (double)G / s.L;
        std::vector<std::pair<int64_t, int64_t>> keyed(M);
        for (int64_t j = 0; j < M; j++) {
            int c[3];
            double bc[3];
            if (s.P.centring == 1) uniform_centre(s, l, sw, (uint32_t)j, bc);     // bucket by the centre
            for (int a = 0; a < 3; a++) {
                int64_t v = (int64_t)std::floor((s.P.centring == 1 ? bc[a] : s.pos[3 * bead[j] + a]) * invG);
                if (v < 0) v = 0;
                if (v >= G) v = G - 1;
                c[a] = (int)v;
            }
            int64_t colour = (c[0] % K) + K * ((c[1] % K) + K * (c[2] % K));
            int64_t q = (c[0] / K) + (int64_t)Q * ((c[1] / K) + (int64_t)Q * (c[2] / K));
            keyed[j] = {colour * nq3 + q, j};
        }
        std::sort(keyed.begin(), keyed.end());
        int64_t a = 0;
        while (a < M) {
            int64_t key = keyed[a].first, e = a;
            while (e < M && keyed[e].first == key) e++;
            int64_t colour = key / nq3, q = key % nq3;
            int c[3] = {(int)(K * (q % Q) + colour % K), (int)(K * ((q / Q) % Q) + (colour / K) % K),
                        (int)(K * (q / ((int64_t)Q * Q)) + colour / (K * K))};
            Region Rg = region_of(s, G, c);
            int64_t cell = c[0] + (int64_t)G * (c[1] + (int64_t)G * c[2]);
            double carry = s.carry_q[l][cell];
            for (int64_t t = a; t < e; t++) {
                if (s.move_budget == 0) return;
                if (s.move_budget > 0) s.move_budget--;
                int64_t j = keyed[t].second;
                double lam_eff = carry > 0.0 ? carry : lam[j];
                int n = 0;
                int r = wavelet_attempt(s, l, (uint32_t)j, bead[j], lam_eff, &Rg, &n, s.P.n_cap);
                if (r == DEFER) { serial.push_back(j); s.st.deferred[l]++; continue; }
                record(j, r, n, 0);
                carry = (r == ACCEPT) ? 0.0 : lam_eff;
            }
            s.carry_q[l][cell] = carry;
            a = e;
        }
        // second level (our schedule, as the first): the deferred slots are bucketed again on the
        // grid G2 = K floor(G / 2K), by the coarse cell of their bead (or centre) now, and run in
        // its colour phases, regions twice as wide and supports up to SECOND_NCAP beads; a slot
        // deferred again runs in the serial phase, in this second schedule's order
        const int G2 = level2_grid(s, l, G);
        if (G2 > 0) {
            const int Q2 = G2 / K;
            const int64_t nq2 = (int64_t)Q2 * Q2 * Q2;
            const double invG2 = (double)G2 / s.L;
            std::vector<std::pair<int64_t, int64_t>> keyed2(serial.size());
            for (size_t t = 0; t < serial.size(); t++) {
                int64_t j = serial[t];
                int c[3];
                double bc[3];
                if (s.P.centring == 1) uniform_centre(s, l, sw, (uint32_t)j, bc);
                for (int a2 = 0; a2 < 3; a2++) {
                    int64_t v = (int64_t)std::floor((s.P.centring == 1 ? bc[a2] : s.pos[3 * bead[j] + a2]) * invG2);
                    if (v < 0) v = 0;
                    if (v >= G2) v = G2 - 1;
                    c[a2] = (int)v;
                }
                int64_t colour = (c[0] % K) + K * ((c[1] % K) + K * (c[2] % K));
                int64_t q = (c[0] / K) + (int64_t)Q2 * ((c[1] / K) + (int64_t)Q2 * (c[2] / K));
                keyed2[t] = {colour * nq2 + q, (int64_t)t};
            }
            std::sort(keyed2.begin(), keyed2.end());
            std::vector<int64_t> serial2;
            size_t a2 = 0;
            while (a2 < keyed2.size()) {
                int64_t key = keyed2[a2].first;
                size_t e = a2;
                while (e < keyed2.size() && keyed2[e].first == key) e++;
                int64_t colour = key / nq2, q = key % nq2;
                int c[3] = {(int)(K * (q % Q2) + colour % K), (int)(K * ((q / Q2) % Q2) + (colour / K) % K),
                            (int)(K * (q / ((int64_t)Q2 * Q2)) + colour / (K * K))};
                Region Rg = region_of(s, G2, c);
                int64_t cell = c[0] + (int64_t)G2 * (c[1] + (int64_t)G2 * c[2]);
                double carry = s.carry_q2[l][cell];
                for (size_t t = a2; t < e; t++) {
                    if (s.move_budget == 0) return;
                    if (s.move_budget > 0) s.move_budget--;
                    int64_t j = serial[keyed2[t].second];
                    double lam_eff = carry > 0.0 ? carry : lam[j];
                    int n = 0;
                    int r = wavelet_attempt(s, l, (uint32_t)j, bead[j], lam_eff, &Rg, &n, SECOND_NCAP);
                    if (r == DEFER) { serial2.push_back(j); continue; }
                    record(j, r, n, 4);
                    carry = (r == ACCEPT) ? 0.0 : lam_eff;
                }
                s.carry_q2[l][cell] = carry;
                a2 = e;
            }
            serial.swap(serial2);
            second = true;
        }
    } else {
        for (int64_t j = 0; j < M; j++) serial.push_back(j);
    }
    // serial phase: deferred slots in schedule order (or all slots of a serial layer)
    double carry = s.carry_serial[l];
    for (int64_t j : serial) {
        if (s.move_budget == 0) return;
        if (s.move_budget > 0) s.move_budget--;
        double lam_eff = carry > 0.0 ? carry : lam[j];
        int n = 0;
        int r = wavelet_attempt(s, l, (uint32_t)j, bead[j], lam_eff, nullptr, &n, s.P.n_cap);
        record(j, r, n, G > 0 ? (second ? 12 : 4) : 0);
        carry = (r == ACCEPT) ? 0.0 : lam_eff;
    }
    s.carry_serial[l] = carry;
}

/* ---- plane-wave moves (Sec. VI; Appendix D, periodic system) ---- */
static const int PERM[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};

// Polarisation of a periodic plane wave with integer wave vector l != 0 and angle psi (in
// turns), Appendix D (choosing e): the unit vector at angle 2 pi psi about k in the plane
// perpendicular to k, from the basis u1 = normalise(k x z) (x when k is along z), u2 = k^ x u1.
static void pw_polarisation(const int lv[3], double psi, double e[3]) {
    int l2 = lv[0] * lv[0] + lv[1] * lv[1] + lv[2] * lv[2];
    double lm = std::sqrt((double)l2);
    double kh[3] = {lv[0] / lm, lv[1] / lm, lv[2] / lm}, u1[3], u2[3];
    if (lv[0] == 0 && lv[1] == 0) { u1[0] = 1.0; u1[1] = 0.0; u1[2] = 0.0; }
    else {
        double nr = std::sqrt((double)(lv[0] * lv[0] + lv[1] * lv[1]));
        u1[0] = lv[1] / nr; u1[1] = -lv[0] / nr; u1[2] = 0.0;
    }
    u2[0] = kh[1] * u1[2] - kh[2] * u1[1];
    u2[1] = kh[2] * u1[0] - kh[0] * u1[2];
    u2[2] = kh[0] * u1[1] - kh[1] * u1[0];
    double cp = cos2pi(psi), sp = sin2pi(psi);
    for (int a = 0; a < 3; a++) e[a] = cp * u1[a] + sp * u2[a];
}
// Amplitude A_F = (2/k) sqrt(dU_est/(mu N)) with dU_est/mu = M6 A0^2/(2 pi)^3 = A0^2/5 (Eq. 48),
// k = 2 pi |l| / L.
static double pw_amplitude(const Sim& s, const int lv[3]) {
    int l2 = lv[0] * lv[0] + lv[1] * lv[1] + lv[2] * lv[2];
    double lm = std::sqrt((double)l2);
    double kmag = (TWO_PI * lm) / s.L;
    return (2.0 * s.P.A0) / (kmag * std::sqrt(5.0 * (double)s.N));
}
// Displacement A_F cos(k.r + Phi) e of a bead at r (Eq. 47), phase in turns.
static void pw_displacement(const Sim& s, const int lv[3], double phi, double AF, const double e[3], const double* r,
                            double dl[3]) {
    double t = ((lv[0] * r[0] + lv[1] * r[1]) + lv[2] * r[2]) / s.L + phi;
    if (s.P.precision == 0) {
        double amp = AF * cos2pi(t);
        for (int a = 0; a < 3; a++) dl[a] = amp * e[a];
    } else {
        float amp = (float)AF * cos2pi_f(t);
        for (int a = 0; a < 3; a++) dl[a] = (double)(amp * (float)e[a]);
    }
}

// Polarisation for a continuous unit wave vector kh (infinite system): the same construction
// as pw_polarisation, u1 = normalise(kh x z) (x when kh is along z), u2 = kh x u1.
static void pw_polarisation_k(const double kh[3], double psi, double e[3]) {
    double u1[3], u2[3];
    if (kh[0] == 0.0 && kh[1] == 0.0) { u1[0] = 1.0; u1[1] = 0.0; u1[2] = 0.0; }
    else {
        double nr = std::sqrt(kh[0] * kh[0] + kh[1] * kh[1]);
        u1[0] = kh[1] / nr; u1[1] = -kh[0] / nr; u1[2] = 0.0;
    }
    u2[0] = kh[1] * u1[2] - kh[2] * u1[1];
    u2[1] = kh[2] * u1[0] - kh[0] * u1[2];
    u2[2] = kh[0] * u1[1] - kh[1] * u1[0];
    double cp = cos2pi(psi), sp = sin2pi(psi);
    for (int a = 0; a < 3; a++) e[a] = cp * u1[a] + sp * u2[a];
}

// A mode of the quasi-continuous shell (Appendix D): |k| from the distribution restricted to
// Q >= Q0 (the shell's inner edge, |l| = N_layers + 1/2), a direction as for p, the point
// snapped to the nearest lattice mode; a mode inside the discrete cube is drawn again (up to
// 64 attempts, after which the last one stands).
static void shell_mode(const Sim& s, int kshell, int kkdir, uint64_t ctr, uint32_t m, int lv[3]) {
    const int Nl = s.P.lcut;
    for (uint32_t a = 0; a < 64; a++) {
        U4 w = s.rng.draw(kshell, 0, ctr, m, a);
        double us = u_open(w.v[0], w.v[1]);
        double Q = k_inverse(s.kF, s.kF0 + us * (1.0 - s.kF0));
        double V[3] = {0.0, 0.0, 1.0};
        for (uint32_t b = 0; b < 64; b++) {
            U4 d = s.rng.draw(kkdir, 0, ctr, m, 64u * a + b);
            double x = sym(d.v[0]), y = sym(d.v[1]), z = sym(d.v[2]), q = (x * x + y * y) + z * z;
            if (q <= 1.0 && q > 0.0) { V[0] = x; V[1] = y; V[2] = z; break; }
        }
        double r = std::sqrt((V[0] * V[0] + V[1] * V[1]) + V[2] * V[2]);
        double sc = (Q * s.L) / (TWO_PI * s.P.lambda_max);    // |k| in units of 2 pi / L
        int inside = 1;
        for (int c = 0; c < 3; c++) {
            lv[c] = (int)std::floor(sc * (V[c] / r) + 0.5);
            if (std::abs(lv[c]) > Nl) inside = 0;
        }
        if (!inside) return;
    }
}

// Wave vector of a fresh (not recycled) plane wave. Periodic modes (1, 2) set lv; the infinite
// system (3) sets the unit direction kh and Q = |k| lambda_max.
static void pw_fresh_k(const Sim& s, int kshell, int kkdir, uint64_t ctr, uint32_t m, const U4& w1, int lv[3],
                       double kh[3], double* Q) {
    const int pwm = s.P.planewave_mode;
    double u_mode = u53(w1.v[0], w1.v[1]);
    if (pwm == 3) {
        *Q = k_inverse(s.kF, u_open(w1.v[0], w1.v[1]));
        double V[3];
        ball_point(s, kkdir, 0, ctr, m, V, true);
        double r = std::sqrt((V[0] * V[0] + V[1] * V[1]) + V[2] * V[2]);
        for (int a = 0; a < 3; a++) kh[a] = V[a] / r;
        return;
    }
    if (pwm == 2 && !(u_mode < s.p_disc)) { shell_mode(s, kshell, kkdir, ctr, m, lv); return; }
    size_t nm = s.mode_prob.size(), idx = nm - 1;
    for (size_t i = 0; i < nm; i++) if (u_mode < s.mode_cdf[i]) { idx = i; break; }
    for (int a = 0; a < 3; a++) lv[a] = s.modes[3 * idx + a];
}

// Returns ACCEPT or REJECT; mode receives the packed wave vector index (-1 when a component is
// beyond 127 or the wave vector is not a lattice mode).
static int planewave_attempt(Sim& s, int kmode, int kdir, int kacc, uint64_t ctr, uint32_t m, int32_t* mode_out) {
    const bool direct = kmode == K_DPWMODE;
    const int kshell = direct ? K_DPWSHELL : K_PWSHELL, kkdir = direct ? K_DPWKDIR : K_PWKDIR;
    const bool cont = s.P.planewave_mode == 3;
    U4 w1 = s.rng.draw(kmode, 0, ctr, m, 0);
    U4 w2 = s.rng.draw(kdir, 0, ctr, m, 0);
    double phi = u53(w1.v[2], w1.v[3]);                                     // phase in turns
    double psi = u53(w2.v[0], w2.v[1]);                                     // polarisation angle in turns
    int perm = (int)(((uint64_t)w2.v[2] * 6u) >> 32);
    uint32_t signs = w2.v[3] & 7u;
    int lv[3] = {0, 0, 0};
    double kh[3] = {0.0, 0.0, 1.0}, Q = 0.0;
    if (s.pw_carry >= 0 && !cont) {
        // recycle |k| after a rejection: permute the components, flip each sign with prob 1/2
        for (int a = 0; a < 3; a++) {
            int v = s.pw_carry_l[PERM[perm][a]];
            lv[a] = ((signs >> a) & 1u) ? -v : v;
        }
    } else if (s.pw_carry >= 0 && cont) {
        // infinite system: the same |k| with a new direction (Appendix D, parameter recycling)
        double dummyQ;
        pw_fresh_k(s, kshell, kkdir, ctr, m, w1, lv, kh, &dummyQ);
        Q = s.pw_carry_Q;
    } else {
        pw_fresh_k(s, kshell, kkdir, ctr, m, w1, lv, kh, &Q);
    }
    if (cont) {
        *mode_out = -1;
        double sc = (Q * s.L) / (TWO_PI * s.P.lambda_max);
        s.tr_pw_k.insert(s.tr_pw_k.end(), {sc * kh[0], sc * kh[1], sc * kh[2]});
    } else {
        bool fits = std::abs(lv[0]) <= 127 && std::abs(lv[1]) <= 127 && std::abs(lv[2]) <= 127;
        *mode_out = fits ? (lv[0] + 128) | ((lv[1] + 128) << 8) | ((lv[2] + 128) << 16) : -1;
        s.tr_pw_k.insert(s.tr_pw_k.end(), {(double)lv[0], (double)lv[1], (double)lv[2]});
    }
    s.st.pw_attempts++;
    if (!cont && lv[0] == 0 && lv[1] == 0 && lv[2] == 0) {
        // the k = 0 mode moves nothing and is accepted (Sec. VI.A)
        s.pw_carry = -1;
        s.st.pw_accepts++;
        s.st.accepted_total++;
        return ACCEPT;
    }
    s.st.bead_updates += s.N;
    double AF, e[3], kappa = 0.0;
    if (cont) {
        // A_F = (2/k) sqrt(dU_est/(mu N)) with k = Q / lambda_max (Eq. 48); the field is applied at
        // the unwrapped positions (an infinite system: the box only organises the neighbours)
        double kmag = Q / s.P.lambda_max;
        AF = (2.0 * s.P.A0) / (kmag * std::sqrt(5.0 * (double)s.N));
        pw_polarisation_k(kh, psi, e);
        kappa = Q / (TWO_PI * s.P.lambda_max);                              // turns per unit length
    } else {
        AF = pw_amplitude(s, lv);
        pw_polarisation(lv, psi, e);
    }
    // displacement A_F cos(k.r + Phi) e of every bead (Eq. 47)
    std::vector<double> newp(3 * (size_t)s.N);
    std::vector<int32_t> newimg(3 * (size_t)s.N);
    for (int64_t i = 0; i < s.N; i++) {
        const double* r = &s.pos[3 * i];
        double dl[3];
        if (cont) {
            double X[3];
            for (int a = 0; a < 3; a++) X[a] = r[a] + (double)s.img[3 * i + a] * s.L;
            double t = kappa * ((kh[0] * X[0] + kh[1] * X[1]) + kh[2] * X[2]) + phi;
            if (s.P.precision == 0) {
                double amp = AF * cos2pi(t);
                for (int a = 0; a < 3; a++) dl[a] = amp * e[a];
            } else {
                float amp = (float)AF * cos2pi_f(t);
                for (int a = 0; a < 3; a++) dl[a] = (double)(amp * (float)e[a]);
            }
        } else {
            pw_displacement(s, lv, phi, AF, e, r, dl);
        }
        for (int a = 0; a < 3; a++) {
            int32_t im = s.img[3 * i + a];
            newp[3 * i + a] = wrap(r[a] + dl[a], s.L, &im);
            newimg[3 * i + a] = im;
        }
    }
    // energy change over all pairs and the external term
    double dU = 0.0;
    for (int64_t i = 0; i < s.N; i++) {
        dU += U_ext(s, &newp[3 * i]) - U_ext(s, &s.pos[3 * i]);
        for (int64_t j = i + 1; j < s.N; j++)
            dU += U_pair(s, i, j, &newp[3 * i], &newp[3 * j]) - U_pair(s, i, j, &s.pos[3 * i], &s.pos[3 * j]);
    }
    U4 w3 = s.rng.draw(kacc, 0, ctr, m, 0);
    bool acc = metropolis(s, dU, w3);
    if (acc) {
        s.pos.swap(newp);
        s.img.swap(newimg);
        s.pw_carry = -1;
        s.st.pw_accepts++;
        s.st.accepted_total++;
        s.st.moved_beads += s.N;
    } else {
        s.pw_carry = 1;
        for (int a = 0; a < 3; a++) s.pw_carry_l[a] = lv[a];
        s.pw_carry_Q = Q;
    }
    return acc ? ACCEPT : REJECT;
}

static void sweep_once(Sim& s) {
    for (int l = 0; l < (int)s.layers.size(); l++) run_layer(s, l);
    s.tr_pw_out.clear();
    s.tr_pw_mode.clear();
    s.tr_pw_k.clear();
    if (s.P.planewave_mode != 0) {
        int64_t MF = slot_count(s, K_PWCOUNT, 0, s.sweep, (double)s.N * s.p_fourier);
        for (int64_t m = 0; m < MF; m++) {
            int32_t mode = 0;
            int r = planewave_attempt(s, K_PWMODE, K_PWDIR, K_PWACC, s.sweep, (uint32_t)m, &mode);
            s.tr_pw_out.push_back((uint8_t)(r == ACCEPT ? 1 : 2));
            s.tr_pw_mode.push_back(mode);
        }
    }
    s.sweep++;
    s.st.sweeps++;
    s.st.sim_time = (double)s.st.accepted_total * s.dt_move;
}

}  // namespace orc

namespace orc {

static const double LAMBDA_A = 1.0 / (1.125 - LN2);   // Eq. 42 for the tapered wavelet

static int setup(Sim& s, const OParams* p, const double* pos, const int32_t* chain_len, int64_t n_chains) {
    s.P = *p;
    const OParams& P = s.P;
    if (P.n_beads < 1 || !(P.box_L > 0) || !(P.lambda_min > 0) || !(P.lambda_max > P.lambda_min) ||
        P.lambda_max > 0.5 * P.box_L || !(P.A0 > 0) || !(P.kT > 0) || P.colour_K < 2 || P.colour_K > 4 ||
        P.grid_f < 1 || P.n_cap < 1 || P.bond_type < 0 || P.bond_type > 2 || P.acceptance < 0 || P.acceptance > 1 ||
        P.centring < 0 || P.centring > 1 || P.level2 < 0 || P.level2 > 0xffff)
        return -1;
    s.N = P.n_beads;
    s.L = P.box_L;
    s.halfL = 0.5 * P.box_L;
    s.invf = (double)P.grid_f / P.box_L;
    s.pos.assign(pos, pos + 3 * s.N);
    for (int64_t i = 0; i < 3 * s.N; i++)
        if (!(pos[i] >= 0.0 && pos[i] < s.L)) return -1;
    s.img.assign(3 * s.N, 0);
    s.bnext.assign(s.N, 0);
    int64_t b = 0;
    for (int64_t c = 0; c < n_chains; c++) {
        for (int32_t k = 0; k + 1 < chain_len[c]; k++) s.bnext[b + k] = 1;
        b += chain_len[c];
    }
    if (b != s.N) return -1;
    s.inS.assign(s.N, 0);
    s.rng = make_stream(P.seed, P.sim_id);
    s.rc = WCA_CUT * P.wca_sigma;
    s.rc2 = s.rc * s.rc;
    s.r_reach = (P.wca_eps != 0.0 ? s.rc : 0.0) + 1e-6;
    // plane-wave tables and the probability of a plane-wave move (Eqs. 51, 55, 56)
    s.p_fourier = 0.0;
    if (P.planewave_mode < 0 || P.planewave_mode > 3) return -1;
    const double M6 = 8.0 * PI * PI * PI / 5.0;
    const double rl = P.lambda_max / P.lambda_min;
    if (P.planewave_mode == 1 || P.planewave_mode == 2) {
        // mode 1: the sphere |l| <= lcut, normalised over itself (a truncated set);
        // mode 2: the cube |l_i| <= lcut (= N_layers) of Appendix D plus the quasi-continuous
        // shell outside it, normalised over all modes
        if (P.lcut < 0 || P.lcut > (P.planewave_mode == 1 ? 120 : 40)) return -1;
        std::vector<double> Q;
        for (int lx = -P.lcut; lx <= P.lcut; lx++)
            for (int ly = -P.lcut; ly <= P.lcut; ly++)
                for (int lz = -P.lcut; lz <= P.lcut; lz++)
                    if (P.planewave_mode == 2 || lx * lx + ly * ly + lz * lz <= P.lcut * P.lcut) {
                        s.modes.insert(s.modes.end(), {lx, ly, lz});
                        Q.push_back(TWO_PI * std::sqrt((double)(lx * lx + ly * ly + lz * lz)) / s.L * P.lambda_max);
                    }
        std::vector<double> Gv;
        G_many(Q, Gv);
        double tot = 0.0;
        for (double g : Gv) tot += g;
        s.z_cube = tot;
        double Z = tot;
        s.p_disc = 1.0;
        if (P.planewave_mode == 2) {
            // shell normalisation in mode-index units u = k L / (2 pi): the integral of
            // G(2 pi |u| lambda_max / L) over all u outside the cube C = [-c, c]^3, c = N_layers + 1/2,
            // = (the integral outside the ball |u| = c) - (the part of C outside that ball)
            const double c = P.lcut + 0.5, scale = TWO_PI * P.lambda_max / s.L;
            s.kF.clear();
            k_cdf_table(s.kF);
            const double Q0 = scale * c;
            s.kF0 = k_cdf_interp(s.kF, Q0);
            const double ball_out = 4.0 * PI * (M6 / 3.0) * (1.0 - k_cdf_exact(Q0)) / (scale * scale * scale);
            std::vector<double> gx, gw, U, W;
            gauss_legendre(16, gx, gw);
            const double ub = c * std::sqrt(3.0);
            for (int p = 0; p < 256; p++) {
                double a = c + (ub - c) * p / 256.0, b = c + (ub - c) * (p + 1) / 256.0, m = 0.5 * (a + b), hh = 0.5 * (b - a);
                for (int k = 0; k < 16; k++) { double u = m + hh * gx[k]; U.push_back(u); W.push_back(hh * gw[k]); }
            }
            std::vector<double> QU(U.size()), GU;
            for (size_t i = 0; i < U.size(); i++) QU[i] = scale * U[i];
            G_many(QU, GU);
            double corner = 0.0;
            for (size_t i = 0; i < U.size(); i++) corner += W[i] * U[i] * U[i] * solid_angle_in_cube(c / U[i]) * GU[i];
            s.z_shell = ball_out - corner;
            Z = tot + s.z_shell;
            s.p_disc = tot / Z;
        }
        s.mode_prob.resize(Gv.size());
        s.mode_cdf.resize(Gv.size());
        double acc = 0.0;
        for (size_t i = 0; i < Gv.size(); i++) {
            s.mode_prob[i] = Gv[i] / Z;
            acc += Gv[i];
            s.mode_cdf[i] = s.p_disc * (acc / tot);
        }
        double ratio = s.L / P.lambda_max;
        s.R = (1.0 / (6.0 * PI * PI)) * (ratio * ratio * ratio) * M6 / Z;
        s.p_fourier = 1.0 / (1.0 + s.R * (rl * rl * rl - 1.0));
    } else if (P.planewave_mode == 3) {
        // infinite system: |k| from P_k^inf (Eq. 52), P_F^inf = (lambda_min / lambda_max)^3 (Eq. 54)
        k_cdf_table(s.kF);
        s.R = 1.0;
        s.p_fourier = 1.0 / (rl * rl * rl);
    }
    // octave layers of P_lambda (Eq. 32): [lmin 2^l, lmin 2^(l+1)), the last one ending at lmax
    int nL = 1;
    while (P.lambda_min * std::ldexp(1.0, nL) < P.lambda_max) nL++;
    if (nL > 16) return -1;
    double imin3 = 1.0 / ((P.lambda_min * P.lambda_min) * P.lambda_min);
    double imax3 = 1.0 / ((P.lambda_max * P.lambda_max) * P.lambda_max);
    s.layers.resize(nL);
    for (int l = 0; l < nL; l++) {
        Layer& Ly = s.layers[l];
        Ly.lo = P.lambda_min * std::ldexp(1.0, l);
        Ly.hi = (l + 1 == nL) ? P.lambda_max : P.lambda_min * std::ldexp(1.0, l + 1);
        Ly.ilo3 = 1.0 / ((Ly.lo * Ly.lo) * Ly.lo);
        Ly.ihi3 = 1.0 / ((Ly.hi * Ly.hi) * Ly.hi);
        Ly.mass = (Ly.ilo3 - Ly.ihi3) / (imin3 - imax3);
        Ly.expect = ((double)s.N * (1.0 - s.p_fourier)) * Ly.mass;
        Ly.G = P.grid_layer[l];
        if (Ly.G < 0 || (Ly.G > 0 && (Ly.G % P.colour_K != 0 || Ly.G < P.colour_K))) return -1;
    }
    s.carry_q.resize(nL);
    for (int l = 0; l < nL; l++) s.carry_q[l].assign(s.layers[l].G > 0 ? (size_t)s.layers[l].G * s.layers[l].G * s.layers[l].G : 0, 0.0);
    s.carry_serial.assign(nL, 0.0);
    s.carry_q2.resize(nL);
    for (int l = 0; l < nL; l++) {
        int G2 = level2_grid(s, l, s.layers[l].G);
        s.carry_q2[l].assign((size_t)G2 * G2 * G2, 0.0);
    }
    s.tr_out.resize(nL);
    s.tr_n.resize(nL);
    s.tr_du.resize(nL);
    s.tr_lam.resize(nL);
    // time per accepted move: Eq. 57 with plane waves, Eq. 34 without (M4/(2pi)^3 = 1/105)
    double A02 = P.A0 * P.A0, la2 = LAMBDA_A * LAMBDA_A;
    if (P.planewave_mode != 0) s.dt_move = (6.0 * A02 * la2) / (105.0 * (double)s.N);
    else {
        double Nl = 3.0 / (imin3 - imax3);
        s.dt_move = ((2.0 * A02 * la2) / (105.0 * (double)s.N)) * (Nl * imin3) * (1.0 - P.lambda_min / P.lambda_max);
    }
    std::memset(&s.st, 0, sizeof s.st);
    s.st.n_layers = nL;
    s.st.dt_move = s.dt_move;
    s.st.p_fourier = s.p_fourier;
    return 0;
}

static double total_energy(const Sim& s) {
    double E = 0.0;
    for (int64_t i = 0; i < s.N; i++) {
        E += U_ext(s, &s.pos[3 * i]);
        for (int64_t j = i + 1; j < s.N; j++) E += U_pair(s, i, j, &s.pos[3 * i], &s.pos[3 * j]);
    }
    return E;
}

}  // namespace orc

using namespace orc;

extern "C" {

void* oracle_create(const OParams* p, const double* pos, const int32_t* chain_len, int64_t n_chains, int* err) {
    Sim* s = new Sim();
    int rc = setup(*s, p, pos, chain_len, n_chains);
    if (err) *err = rc;
    if (rc != 0) { delete s; return nullptr; }
    return s;
}
void oracle_destroy(void* h) { delete (Sim*)h; }

int oracle_sweep(void* h, int64_t n) {
    Sim& s = *(Sim*)h;
    for (int64_t k = 0; k < n; k++) sweep_once(s);
    return 0;
}
// n plane-wave moves outside the sweep schedule (their own counter stream)
int oracle_planewave(void* h, int64_t n) {
    Sim& s = *(Sim*)h;
    if (s.P.planewave_mode == 0) return -1;
    s.tr_pw_out.clear();
    s.tr_pw_mode.clear();
    s.tr_pw_k.clear();
    for (int64_t m = 0; m < n; m++) {
        int32_t mode = 0;
        int r = planewave_attempt(s, K_DPWMODE, K_DPWDIR, K_DPWACC, s.pw_calls, (uint32_t)m, &mode);
        s.tr_pw_out.push_back((uint8_t)(r == ACCEPT ? 1 : 2));
        s.tr_pw_mode.push_back(mode);
    }
    s.pw_calls++;
    s.st.sim_time = (double)s.st.accepted_total * s.dt_move;
    return 0;
}
int oracle_positions(void* h, double* out, int unwrapped) {
    Sim& s = *(Sim*)h;
    for (int64_t i = 0; i < 3 * s.N; i++) out[i] = unwrapped ? s.pos[i] + (double)s.img[i] * s.L : s.pos[i];
    return 0;
}
int oracle_stats(void* h, OStats* out) { *out = ((Sim*)h)->st; return 0; }

int64_t oracle_trace_layer(void* h, int l, uint8_t* out, int32_t* n, int64_t cap) {
    Sim& s = *(Sim*)h;
    if (l < 0 || l >= (int)s.layers.size()) return -1;
    int64_t M = (int64_t)s.tr_out[l].size();
    for (int64_t j = 0; j < M && j < cap; j++) { out[j] = s.tr_out[l][j]; n[j] = s.tr_n[l][j]; }
    return M;
}
// energy change of each wavelet slot of the last sweep (0 when nothing moved)
int64_t oracle_trace_du(void* h, int l, double* out, int64_t cap) {
    Sim& s = *(Sim*)h;
    if (l < 0 || l >= (int)s.layers.size()) return -1;
    int64_t M = (int64_t)s.tr_du[l].size();
    for (int64_t j = 0; j < M && j < cap; j++) out[j] = s.tr_du[l][j];
    return M;
}
// lambda used by each wavelet slot's attempt in the last sweep (a carried one after a rejection,
// Appendix D parameter recycling); 0 for a slot not attempted
int64_t oracle_trace_lam(void* h, int l, double* out, int64_t cap) {
    Sim& s = *(Sim*)h;
    if (l < 0 || l >= (int)s.layers.size()) return -1;
    int64_t M = (int64_t)s.tr_lam[l].size();
    for (int64_t j = 0; j < M && j < cap; j++) out[j] = s.tr_lam[l][j];
    return M;
}
int64_t oracle_trace_pw(void* h, uint8_t* out, int32_t* mode, int64_t cap) {
    Sim& s = *(Sim*)h;
    int64_t M = (int64_t)s.tr_pw_out.size();
    for (int64_t j = 0; j < M && j < cap; j++) { out[j] = s.tr_pw_out[j]; mode[j] = s.tr_pw_mode[j]; }
    return M;
}

/* ---- entry points used by the pins ---- */
void oracle_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out) {
    U4 c;
    for (int a = 0; a < 4; a++) c.v[a] = ctr[a];
    U4 r = philox(c, key[0], key[1]);
    for (int a = 0; a < 4; a++) out[a] = r.v[a];
}
double oracle_phitilde(double k) { return phitilde(k); }
double oracle_moment(int m) { return moment(m); }
void oracle_G(const double* Q, int64_t n, double* out) {
    std::vector<double> q(Q, Q + n), o;
    G_many(q, o);
    for (int64_t i = 0; i < n; i++) out[i] = o[i];
}
double oracle_cos2pi(double t) { return cos2pi(t); }
double oracle_sin2pi(double t) { return sin2pi(t); }
float oracle_cos2pi_f(double t) { return cos2pi_f(t); }
double oracle_inv_cbrt(double w, double lo) { return inv_cbrt_from(w, lo); }
double oracle_lambda_a(void) { return LAMBDA_A; }

int oracle_layers(void* h, double* lo, double* hi, double* mass, double* expect, int cap) {
    Sim& s = *(Sim*)h;
    int nL = (int)s.layers.size();
    for (int l = 0; l < nL && l < cap; l++) { lo[l] = s.layers[l].lo; hi[l] = s.layers[l].hi; mass[l] = s.layers[l].mass; expect[l] = s.layers[l].expect; }
    return nL;
}
// slot counts of sweep `sw`: out[l] for the wavelet layers, out[16] for the plane waves
int oracle_slot_counts(void* h, uint64_t sw, int64_t* out) {
    Sim& s = *(Sim*)h;
    int nL = (int)s.layers.size();
    for (int l = 0; l < 16; l++) out[l] = l < nL ? slot_count(s, K_COUNT, l, sw, s.layers[l].expect) : 0;
    out[16] = s.P.planewave_mode != 0 ? slot_count(s, K_PWCOUNT, 0, sw, (double)s.N * s.p_fourier) : 0;
    return nL;
}
// scales and beads of slots 0..n-1 of layer l in the current sweep
int64_t oracle_sample_slots(void* h, int l, int64_t n, double* lam, int64_t* bead) {
    Sim& s = *(Sim*)h;
    if (l < 0 || l >= (int)s.layers.size()) return -1;
    for (int64_t j = 0; j < n; j++) slot_draw(s, l, s.sweep, (uint32_t)j, &lam[j], &bead[j]);
    return n;
}
// n uniform points of the unit ball from the centre stream of layer 0, sweep `sw`
int64_t oracle_sample_ball(void* h, uint64_t sw, int64_t n, double* out) {
    Sim& s = *(Sim*)h;
    for (int64_t j = 0; j < n; j++) ball_point(s, K_VB, 0, sw, (uint32_t)j, &out[3 * j], false);
    return n;
}
int64_t oracle_sample_polarisation(void* h, uint64_t sw, int64_t n, double* out) {
    Sim& s = *(Sim*)h;
    for (int64_t j = 0; j < n; j++) polarisation(s, 0, sw, (uint32_t)j, &out[3 * j]);
    return n;
}
// displacement of a bead at `pt` by a wavelet (b, lam, p, A_w): zero outside the support
void oracle_wavelet_field(void* h, const double* b, double lam, const double* p, double Aw, const double* pt, double* out) {
    Sim& s = *(Sim*)h;
    double d[3];
    for (int a = 0; a < 3; a++) d[a] = mi(pt[a] - b[a], s.L, s.halfL);
    double d2 = (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2];
    if (!(d2 < lam * lam)) { out[0] = out[1] = out[2] = 0.0; return; }
    wavelet_disp(s, d, d2, lam, Aw, p, out);
}
double oracle_delta_u(void* h, int64_t n, const int64_t* ids, const double* newpos) {
    Sim& s = *(Sim*)h;
    std::vector<int64_t> S(ids, ids + n);
    std::vector<double> np(newpos, newpos + 3 * n);
    return delta_U(s, S, np);
}
double oracle_total_energy(void* h) { return total_energy(*(Sim*)h); }

// polarisation of the periodic plane wave with wave vector l (three ints) at angle psi (turns)
void oracle_pw_polarisation(const int32_t* l, double psi, double* e) {
    int lv[3] = {l[0], l[1], l[2]};
    pw_polarisation(lv, psi, e);
}
// displacement of a bead at `pt` by the periodic plane wave (l, phase phi, angle psi) of this
// simulation, as a move applies it (amplitude of Eq. 48, field of Eq. 47)
void oracle_planewave_field(void* h, const int32_t* l, double phi, double psi, const double* pt, double* out) {
    Sim& s = *(Sim*)h;
    int lv[3] = {l[0], l[1], l[2]};
    double e[3];
    pw_polarisation(lv, psi, e);
    pw_displacement(s, lv, phi, pw_amplitude(s, lv), e, pt, out);
}

int64_t oracle_pw_modes(void* h, int32_t* modes, double* prob, int64_t cap, double* R, double* PF) {
    Sim& s = *(Sim*)h;
    int64_t nm = (int64_t)s.mode_prob.size();
    for (int64_t i = 0; i < nm && i < cap; i++) {
        for (int a = 0; a < 3; a++) modes[3 * i + a] = s.modes[3 * i + a];
        prob[i] = s.mode_prob[i];
    }
    *R = s.R;
    *PF = s.p_fourier;
    return nm;
}

// Moments of proposed wavelet displacements of beads 0 and 1 on the frozen configuration:
// out[0..8] = <d0 (x) d1>, out[9..17] = <d0 (x) d0>, out[18..26] = <d1 (x) d1>, per proposal.
// Proposals use the move generation of Appendix D with the layered P_lambda; nothing is
// accepted or moved.
int oracle_propose_moments(void* h, int64_t n_props, uint64_t offset, double* out) {
    Sim& s = *(Sim*)h;
    if (s.N < 2) return -1;
    double acc[27] = {0};
    int nL = (int)s.layers.size();
    std::vector<double> cum(nL);
    double c = 0.0;
    for (int l = 0; l < nL; l++) { c += s.layers[l].mass; cum[l] = c; }
    for (int64_t t = 0; t < n_props; t++) {
        uint64_t sw = (1ull << 40) + offset + (uint64_t)t;
        U4 w = s.rng.draw(K_PROPOSE, 0, sw, 0, 0);
        double ul = u53(w.v[0], w.v[1]) * c;
        int l = nL - 1;
        for (int k = 0; k < nL; k++) if (ul < cum[k]) { l = k; break; }
        double lam;
        int64_t i;
        slot_draw(s, l, sw, 0, &lam, &i);
        double V[3], b[3], p[3];
        if (s.P.centring == 1) uniform_centre(s, l, sw, 0, b);
        else {
            ball_point(s, K_VB, l, sw, 0, V, false);
            for (int a = 0; a < 3; a++) b[a] = wrap(s.pos[3 * i + a] + lam * V[a], s.L, nullptr);
        }
        polarisation(s, l, sw, 0, p);
        int n = 0;
        double dd[2][4];
        bool in01[2] = {false, false};
        for (int64_t m = 0; m < s.N; m++) {
            double d[3];
            for (int a = 0; a < 3; a++) d[a] = mi(s.pos[3 * m + a] - b[a], s.L, s.halfL);
            double d2 = (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2];
            if (d2 < lam * lam) {
                n++;
                if (m < 2) { in01[m] = true; dd[m][0] = d[0]; dd[m][1] = d[1]; dd[m][2] = d[2]; dd[m][3] = d2; }
            }
        }
        if (n == 0) continue;
        double Aw = wavelet_amplitude(s, lam, n), dl[2][3] = {{0, 0, 0}, {0, 0, 0}};
        for (int m = 0; m < 2; m++) if (in01[m]) wavelet_disp(s, dd[m], dd[m][3], lam, Aw, p, dl[m]);
        for (int a = 0; a < 3; a++)
            for (int bb = 0; bb < 3; bb++) {
                acc[3 * a + bb] += dl[0][a] * dl[1][bb];
                acc[9 + 3 * a + bb] += dl[0][a] * dl[0][bb];
                acc[18 + 3 * a + bb] += dl[1][a] * dl[1][bb];
            }
    }
    for (int k = 0; k < 27; k++) out[k] = acc[k] / (double)n_props;
    return 0;
}

// The first `max_moves` wavelet attempts of the next sweep, in schedule order; the rest of that
// sweep is skipped (its counter still advances). For timing a bounded sample of a large
// system's sweep; returns the attempts made.
int64_t oracle_sweep_sample(void* h, int64_t max_moves) {
    Sim& s = *(Sim*)h;
    int64_t before = 0, after = 0;
    for (int l = 0; l < 16; l++) before += s.st.attempts[l] + s.st.deferred[l];
    s.move_budget = max_moves < 0 ? 0 : max_moves;
    sweep_once(s);
    s.move_budget = -1;
    for (int l = 0; l < 16; l++) after += s.st.attempts[l] + s.st.deferred[l];
    return after - before;
}

// normalisation parts of the plane-wave scheme: [p_disc, z_cube, z_shell, F(Q0) of the table]
void oracle_pw_tables(void* h, double* out) {
    Sim& s = *(Sim*)h;
    out[0] = s.p_disc; out[1] = s.z_cube; out[2] = s.z_shell; out[3] = s.kF0;
}
// tabulated F(Q) and its inverse (Q = |k| lambda_max), and the direct quadrature of F
double oracle_k_cdf_exact(double Q) { return k_cdf_exact(Q); }
double oracle_k_inverse(void* h, double u) { return k_inverse(((Sim*)h)->kF, u); }
double oracle_solid_angle_in_cube(double t) { return solid_angle_in_cube(t); }
// n fresh wave vectors as plane waves draw them (direct-call streams at counter ctr, no
// recycling), in units of 2 pi / L, 3 per draw
int64_t oracle_sample_pw_k(void* h, uint64_t ctr, int64_t n, double* out) {
    Sim& s = *(Sim*)h;
    if (s.P.planewave_mode == 0) return -1;
    for (int64_t j = 0; j < n; j++) {
        U4 w1 = s.rng.draw(K_DPWMODE, 0, ctr, (uint32_t)j, 0);
        int lv[3] = {0, 0, 0};
        double kh[3] = {0.0, 0.0, 1.0}, Q = 0.0;
        pw_fresh_k(s, K_DPWSHELL, K_DPWKDIR, ctr, (uint32_t)j, w1, lv, kh, &Q);
        if (s.P.planewave_mode == 3) {
            double sc = (Q * s.L) / (TWO_PI * s.P.lambda_max);
            for (int a = 0; a < 3; a++) out[3 * j + a] = sc * kh[a];
        } else {
            for (int a = 0; a < 3; a++) out[3 * j + a] = (double)lv[a];
        }
    }
    return n;
}
// wave vectors (units of 2 pi / L) of the last sweep's or call's plane waves
int64_t oracle_trace_pw_k(void* h, double* out, int64_t cap) {
    Sim& s = *(Sim*)h;
    int64_t M = (int64_t)s.tr_pw_k.size() / 3;
    for (int64_t j = 0; j < M && j < cap; j++)
        for (int a = 0; a < 3; a++) out[3 * j + a] = s.tr_pw_k[3 * j + a];
    return M;
}

// acceptance thresholds of n wavelet slots of layer 0 in sweep `sw` (accept iff dU <= threshold)
int64_t oracle_sample_threshold(void* h, uint64_t sw, int64_t n, double* out) {
    Sim& s = *(Sim*)h;
    for (int64_t j = 0; j < n; j++) out[j] = accept_threshold(s, s.rng.draw(K_ACC, 0, sw, (uint32_t)j, 0));
    return n;
}

// run n sweeps, recording the unwrapped position of bead 0 after each
int oracle_sweep_record(void* h, int64_t n, double* out) {
    Sim& s = *(Sim*)h;
    for (int64_t k = 0; k < n; k++) {
        sweep_once(s);
        for (int a = 0; a < 3; a++) out[3 * k + a] = s.pos[a] + (double)s.img[a] * s.L;
    }
    return 0;
}

}  // extern "C"
