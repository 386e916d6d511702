// Host side of the WMCD library: per-simulation constants and tables, device allocation,
// the order of launches in a sweep, and the C ABI declared in include/wmcd.h.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>
#include "../../include/wmcd.h"
#include "wmcd_host.h"

namespace wmcd {

// ---------------------------------------------------------------------------------------
// Plane-wave weights G(Q) = Int_Q^inf q^3 phi~(q)^2 dq (Eqs. 49, 51) for the tapered
// wavelet, phi~(k) = 4 pi k^-6 (5 k sin k - (k^2 - 8) cos k - 8) (Eq. 25).
// Near k = 0 the bracket is replaced by its Taylor series, whose coefficients follow from
// those of sin and cos:  bracket = sum_{p>=3} c_p k^{2p},
//   c_p = (-1)^{p-1} [5/(2p-1)! - 1/(2p-2)! - 8/(2p)!].
// ---------------------------------------------------------------------------------------
static double phit(double k) {
    k = std::fabs(k);
    if (k < 1.5) {
        double s = 0.0;
        double f2m2 = 24.0;                   // (2p-2)! at p = 3
        for (int p = 3; p < 24; p++) {
            double f2m1 = f2m2 * (2 * p - 1), f2 = f2m1 * (2 * p);
            double c = 5.0 / f2m1 - 1.0 / f2m2 - 8.0 / f2;
            double term = c * std::pow(k, 2 * p - 6);
            s += (p % 2 == 1) ? term : -term;
            f2m2 = f2;
        }
        return 4.0 * kPi * s;
    }
    double k2 = k * k;
    return 4.0 * kPi * (5.0 * k * std::sin(k) - (k2 - 8.0) * std::cos(k) - 8.0) / (k2 * k2 * k2);
}
// 10-point Gauss-Legendre nodes and weights on [-1, 1]
static const double GL10_X[5] = {0.1488743389816312, 0.4333953941292472, 0.6794095682990244, 0.8650633666889845,
                                 0.9739065285171717};
static const double GL10_W[5] = {0.2955242247147529, 0.2692667193099963, 0.2190863625159820, 0.1494513491505806,
                                 0.0666713443086881};
static double gl10(double a, double b) {
    double c = 0.5 * (a + b), h = 0.5 * (b - a), s = 0.0;
    for (int i = 0; i < 5; i++) {
        for (int sg = -1; sg <= 1; sg += 2) {
            double q = c + sg * h * GL10_X[i], f = phit(q);
            s += GL10_W[i] * q * q * q * f * f;
        }
    }
    return s * h;
}
// Smooth part of the tail beyond Kc: the non-oscillating terms of q^3 phi~^2 at large q,
// 16 pi^2 (q^-5/2 + 9/2 q^-7 + 96 q^-9), integrated exactly.
static double tail3(double Kc) {
    return 16.0 * kPi * kPi * (0.125 * std::pow(Kc, -4) + 0.75 * std::pow(Kc, -6) + 12.0 * std::pow(Kc, -8));
}
static const std::vector<double>& G_panels() {
    // acc[p] = G(p h), summed from the tail inwards once per process
    static const std::vector<double> acc = [] {
        const double h = kPi / 20.0;
        const int panels = 40000;             // up to Kc = 2000 pi (a multiple of pi)
        std::vector<double> a(panels + 1);
        a[panels] = tail3(panels * h);
        for (int p = panels - 1; p >= 0; p--) a[p] = a[p + 1] + gl10(p * h, (p + 1) * h);
        return a;
    }();
    return acc;
}
static void G_table(const std::vector<double>& Q, std::vector<double>& out) {
    const double h = kPi / 20.0;
    const int panels = 40000;
    const std::vector<double>& acc = G_panels();
    out.resize(Q.size());
    for (size_t i = 0; i < Q.size(); i++) {
        double q = Q[i];
        if (q >= panels * h) { out[i] = tail3(q); continue; }
        int p = (int)(q / h);
        double top = (p + 1) * h;
        out[i] = acc[p + 1] + (top > q ? gl10(q, top) : 0.0);
    }
}

// ---------------------------------------------------------------------------------------
// Distribution of |k| for the infinite system and the quasi-continuous shell (Sec. VI.B,
// Eqs. 52-53): in Q = k lambda_max, P_k^inf ~ Q^2 G(Q) with integral M6/3, whose CDF is,
// after an integration by parts (dG/dQ = -Q^3 phi~^2),
//     F(Q) = [Q^3 G(Q) + Int_0^Q q^6 phi~(q)^2 dq] / M6.
// Tabulated on Q_i = i kKtH (i = 0..kKtN); moves invert it by interpolation (the paper's
// conversion table), F^(1/3) linear between grid points.
// ---------------------------------------------------------------------------------------
static double gl10_q6(double a, double b) {
    double c = 0.5 * (a + b), h = 0.5 * (b - a), s = 0.0;
    for (int i = 0; i < 5; i++) {
        for (int sg = -1; sg <= 1; sg += 2) {
            const double q = c + sg * h * GL10_X[i], f = phit(q), q3 = q * q * q;
            s += GL10_W[i] * q3 * q3 * f * f;
        }
    }
    return s * h;
}
static const double kM6 = 8.0 * kPi * kPi * kPi / 5.0;
static const std::vector<double>& k_cdf_table() {
    static const std::vector<double> F = [] {
        std::vector<double> Q(kKtN + 1), g;
        for (int i = 0; i <= kKtN; i++) Q[i] = i * kKtH;
        G_table(Q, g);
        std::vector<double> t(kKtN + 1, 0.0);
        double cum = 0.0, comp = 0.0;         // compensated running sum
        for (int i = 1; i <= kKtN; i++) {
            // two 10-point panels per grid step
            const double y = (gl10_q6(Q[i - 1], Q[i - 1] + 0.5 * kKtH) + gl10_q6(Q[i - 1] + 0.5 * kKtH, Q[i])) - comp;
            const double tt = cum + y;
            comp = (tt - cum) - y;
            cum = tt;
            t[i] = (Q[i] * Q[i] * Q[i] * g[i] + cum) / kM6;
        }
        return t;
    }();
    return F;
}
// F(Q) directly (the shell's normalisation) and through the table (where the shell starts)
static double k_cdf_direct(double Q) {
    const double step = 0.5 * kKtH;
    double cum = 0.0, comp = 0.0, a = 0.0;
    while (a < Q) {
        const double b = std::min(Q, a + step), y = gl10_q6(a, b) - comp, t = cum + y;
        comp = (t - cum) - y;
        cum = t;
        a = b;
    }
    std::vector<double> g;
    G_table(std::vector<double>{Q}, g);
    return (Q * Q * Q * g[0] + cum) / kM6;
}
static double k_cdf_tabled(const std::vector<double>& F, double Q) {
    if (Q >= kKtN * kKtH) return 1.0 - (1.0 - F[kKtN]) * (kKtN * kKtH) / Q;
    int i = std::min((int)(Q / kKtH), kKtN - 1);
    const double a = std::cbrt(F[i]), b = std::cbrt(F[i + 1]);
    const double t = a + (b - a) * ((Q - i * kKtH) / kKtH);
    return t * t * t;
}
// Solid angle of the unit vectors with every |component| <= t. With 2 t^2 >= 1 the six caps
// n_i > t (or < -t) are disjoint, 2 pi (1 - t) each. Otherwise the area, uniform in n_z, is
// taken height by height: for |n_z| <= t the circle of radius rho = sqrt(1 - n_z^2) > t keeps
// 2 pi - 8 arccos(t / rho) inside the square |n_x|, |n_y| <= t when rho <= t sqrt(2), nothing
// beyond, which leaves a smooth integral over n_z in [sqrt(1 - 2 t^2), t].
static double cube_solid_angle(double t) {
    if (2.0 * t * t >= 1.0) return 4.0 * kPi * (3.0 * std::min(t, 1.0) - 2.0);
    if (3.0 * t * t <= 1.0) return 0.0;
    const double a = std::sqrt(1.0 - 2.0 * t * t), b = t;
    double sum = 0.0;
    const int sub = 24;
    for (int p = 0; p < sub; p++) {
        const double pa = a + (b - a) * p / sub, pb = a + (b - a) * (p + 1) / sub;
        const double c = 0.5 * (pa + pb), h = 0.5 * (pb - pa);
        for (int i = 0; i < 5; i++)
            for (int sg = -1; sg <= 1; sg += 2) {
                const double z = c + sg * h * GL10_X[i], rho = std::sqrt(1.0 - z * z);
                sum += h * GL10_W[i] * (kTwoPi - 8.0 * std::acos(t / rho));
            }
    }
    return 2.0 * sum;
}
// Weight of the quasi-continuous shell, in mode-index units u = k L / (2 pi): the integral of
// G(2 pi |u| lambda_max / L) over the u outside the cube [-c, c]^3, c = N_layers + 1/2; that is
// the integral outside the ball |u| = c less the part of the cube outside that ball.
static double shell_weight(int nl, double L, double lmax) {
    const double c = nl + 0.5, scale = kTwoPi * lmax / L;
    const double ball = 4.0 * kPi * (kM6 / 3.0) * (1.0 - k_cdf_direct(scale * c)) / (scale * scale * scale);
    const double ub = c * std::sqrt(3.0);
    std::vector<double> U, W, QU, g;
    const int panels = 512;
    for (int p = 0; p < panels; p++) {
        const double a = c + (ub - c) * p / panels, b = c + (ub - c) * (p + 1) / panels, m = 0.5 * (a + b), h = 0.5 * (b - a);
        for (int i = 0; i < 5; i++)
            for (int sg = -1; sg <= 1; sg += 2) { U.push_back(m + sg * h * GL10_X[i]); W.push_back(h * GL10_W[i]); }
    }
    for (double u : U) QU.push_back(scale * u);
    G_table(QU, g);
    double corner = 0.0;
    for (size_t i = 0; i < U.size(); i++) corner += W[i] * U[i] * U[i] * cube_solid_angle(c / U[i]) * g[i];
    return ball - corner;
}

int last_cuda_status() {
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? WMCD_OK : WMCD_ECUDA;
}

template <class T>
static int dalloc(Handle* h, T** p, size_t count) {
    size_t nb = std::max<size_t>(count, 1) * sizeof(T);
    if (h->arena) {
        Arena& a = *h->arena;
        const size_t off = (a.used + 255) & ~(size_t)255;
        a.used = off + nb;
        h->bytes += nb;
        if (a.count_only) { *p = nullptr; return WMCD_OK; }
        if (a.used > a.size) return WMCD_ENOMEM;
        *p = (T*)(a.base + off);
        return WMCD_OK;
    }
    void* q = nullptr;
    if (cudaMalloc(&q, nb) != cudaSuccess) { cudaGetLastError(); return WMCD_ENOMEM; }
    h->allocs.push_back(q);
    h->bytes += nb;
    *p = (T*)q;
    return WMCD_OK;
}

static bool is_device_ptr(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) { cudaGetLastError(); return false; }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

static cudaEvent_t get_event(Handle* h) {
    if (!h->ev_pool.empty()) { cudaEvent_t e = h->ev_pool.back(); h->ev_pool.pop_back(); return e; }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
}
void prof_harvest(Handle* h) {
    for (auto& u : h->ev_used) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, u.second.first, u.second.second) == cudaSuccess) {
            h->prof_ms[u.first] += ms;
            h->prof_launches[u.first]++;
        } else {
            cudaGetLastError();
        }
        h->ev_pool.push_back(u.second.first);
        h->ev_pool.push_back(u.second.second);
    }
    h->ev_used.clear();
}
struct ProfScope {
    Handle* h; int cls; cudaStream_t s; cudaEvent_t a{}, b{};
    ProfScope(Handle* h_, int c, cudaStream_t s_) : h(h_), cls(c), s(s_) {
        if (h && h->prof) { a = get_event(h); cudaEventRecord(a, s); }
    }
    ~ProfScope() {
        if (h && h->prof) {
            b = get_event(h);
            cudaEventRecord(b, s);
            h->ev_used.push_back({cls, {a, b}});
            if (h->ev_used.size() > 20000) { cudaEventSynchronize(b); prof_harvest(h); }
        }
    }
};

// stratified slot count: floor(x) plus one more with probability frac(x)
int64_t slot_count(const Handle* h, uint32_t kind, int l, uint64_t ctr, double x) {
    u4 w = draw(h->v.k0, h->v.k1, kind, l, ctr, 0u, 0u);
    double u = u53(w.x, w.y), f = std::floor(x);
    return (int64_t)f + ((u < x - f) ? 1 : 0);
}

__global__ void k_fill_beads(Bead* bead, BeadF* bf, const double* pos, int64_t N) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        put_bead(bead, bf, i, pos[3 * i], pos[3 * i + 1], pos[3 * i + 2]);
        bead[i].mark = 0u;
    }
}
__global__ void k_read_beads(const Bead* bead, const int* img, double L, int unwrapped, double* out, int64_t N) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        Bead b = bead[i];
        double x[3] = {b.x, b.y, b.z};
        for (int a = 0; a < 3; a++) out[3 * i + a] = unwrapped ? add(x[a], mul((double)img[3 * i + a], L)) : x[a];
    }
}
static int grid_for(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 16)); }

}  // namespace wmcd

using namespace wmcd;


int wmcd::validate_params(const wmcd_params* p) {
    if (!p || p->n_beads < 1 || p->n_beads > (int64_t)1 << 30) return WMCD_EINVAL;
    if (!(p->box_L > 0.0) || !(p->lambda_min > 0.0) || !(p->lambda_max > p->lambda_min) ||
        p->lambda_max > 0.5 * p->box_L || !(p->A0 > 0.0) || !(p->kT > 0.0))
        return WMCD_EINVAL;
    if (p->bond_type < 0 || p->bond_type > 2 || p->colour_K < 2 || p->colour_K > 4 || p->grid_f < 1 ||
        p->n_cap < 1 || p->n_cap > kNCapMax || p->precision < 0 || p->precision > 1)
        return WMCD_EINVAL;
    if (p->planewave_mode < 0 || p->planewave_mode > 3) return WMCD_EINVAL;
    if (p->acceptance < 0 || p->acceptance > 1 || p->centring < 0 || p->centring > 1) return WMCD_EINVAL;
    if (p->level2 < 0 || p->level2 > 0xffff) return WMCD_EINVAL;
    if (p->planewave_mode == 1 && (p->lcut < 0 || p->lcut > 120)) return WMCD_EINVAL;
    if (p->planewave_mode == 2 && (p->lcut < 0 || p->lcut > 40)) return WMCD_EINVAL;
    if ((int64_t)p->grid_f * p->grid_f * p->grid_f > ((int64_t)1 << 31) - 1) return WMCD_EINVAL;
    if (p->wca_eps != 0.0 && p->box_L / p->grid_f < kWcaCut * p->wca_sigma * (1.0 - 1e-12)) return WMCD_EINVAL;
    if (p->bond_type == 2 && !(p->fene_R0 > 0.0)) return WMCD_EINVAL;
    return WMCD_OK;
}

int wmcd::create_handle(wmcd_handle* H, const wmcd_params* params, const double* pos, const int32_t* chain_len,
                        int64_t n_chains, cudaStream_t s, Arena* arena) {
    const bool counting = arena && arena->count_only;
    int rc = validate_params(params);
    if (rc) return rc;
    const wmcd_params& P = *params;
    if (!counting) {
        if (!pos || !chain_len || n_chains < 1) return WMCD_EINVAL;
        int64_t tot = 0;
        for (int64_t c = 0; c < n_chains; c++) { if (chain_len[c] < 1) return WMCD_EINVAL; tot += chain_len[c]; }
        if (tot != P.n_beads) return WMCD_EINVAL;
    }
    Handle* h = &H->h;
    h->arena = arena;
    h->P = P;
    h->N = P.n_beads;
    cudaGetDevice(&h->dev);
    SimView& v = h->v;
    std::memset(&v, 0, sizeof v);
    v.N = P.n_beads;
    v.L = P.box_L;
    v.halfL = 0.5 * P.box_L;
    v.Gf = P.grid_f;
    v.invf = (double)P.grid_f / P.box_L;
    v.K = P.colour_K;
    v.n_cap = P.n_cap;
    v.precision = P.precision;
    v.A0 = P.A0;
    v.kT = P.kT;
    v.rc = kWcaCut * P.wca_sigma;
    v.r_reach = (P.wca_eps != 0.0 ? v.rc : 0.0) + 1e-6;
    v.pot.sig2 = P.wca_sigma * P.wca_sigma;
    v.pot.eps = P.wca_eps;
    v.pot.rc2 = v.rc * v.rc;
    v.pot.bond = P.bond_type;
    v.pot.bk = P.bond_k;
    v.pot.br0 = P.bond_r0;
    v.pot.R02 = P.fene_R0 * P.fene_R0;
    v.pot.kappa = P.ext_kappa;
    v.pot.halfL = v.halfL;
    v.pot.L = v.L;
    v.k0 = (uint32_t)P.seed;
    v.k1 = (uint32_t)(P.seed >> 32) ^ (uint32_t)P.sim_id;
    v.acceptance = P.acceptance;
    v.centring = P.centring;

    // plane-wave tables and P_F (Eqs. 51, 55, 56): mode 1 the sphere |l| <= lcut normalised over
    // itself; mode 2 the cube |l_i| <= lcut (N_layers) plus the quasi-continuous shell, normalised
    // over all modes (Appendix D); mode 3 the infinite system, P_F = (lambda_min/lambda_max)^3 (Eq. 54)
    std::vector<int> modes;
    std::vector<double> cdf;
    h->p_fourier = 0.0;
    double p_disc = 1.0, kF0 = 0.0;
    const double rl = P.lambda_max / P.lambda_min;
    if (P.planewave_mode == 1 || P.planewave_mode == 2) {
        std::vector<double> Q;
        for (int lx = -P.lcut; lx <= P.lcut; lx++)
            for (int ly = -P.lcut; ly <= P.lcut; ly++)
                for (int lz = -P.lcut; lz <= P.lcut; lz++) {
                    int l2 = lx * lx + ly * ly + lz * lz;
                    if (P.planewave_mode == 1 && l2 > P.lcut * P.lcut) continue;
                    modes.push_back(lx); modes.push_back(ly); modes.push_back(lz);
                    Q.push_back(kTwoPi * std::sqrt((double)l2) / P.box_L * P.lambda_max);
                }
        std::vector<double> g;
        G_table(Q, g);
        double tot_w = 0.0;
        for (double x : g) tot_w += x;
        double Z = tot_w;
        if (P.planewave_mode == 2) {
            const double zs = shell_weight(P.lcut, P.box_L, P.lambda_max);
            Z = tot_w + zs;
            p_disc = tot_w / Z;
            kF0 = k_cdf_tabled(k_cdf_table(), kTwoPi * P.lambda_max / P.box_L * (P.lcut + 0.5));
        }
        cdf.resize(g.size());
        double acc = 0.0;
        for (size_t i = 0; i < g.size(); i++) { acc += g[i]; cdf[i] = p_disc * (acc / tot_w); }
        const double M6 = 8.0 * kPi * kPi * kPi / 5.0;
        const double ratio = P.box_L / P.lambda_max;
        h->R = (1.0 / (6.0 * kPi * kPi)) * (ratio * ratio * ratio) * M6 / Z;
        h->p_fourier = 1.0 / (1.0 + h->R * (rl * rl * rl - 1.0));
    } else if (P.planewave_mode == 3) {
        h->R = 1.0;
        h->p_fourier = 1.0 / (rl * rl * rl);
    }
    // octave layers of P_lambda (Eq. 32)
    int nL = 1;
    while (P.lambda_min * std::ldexp(1.0, nL) < P.lambda_max) nL++;
    if (nL > kMaxLayers) return WMCD_EINVAL;
    h->nL = v.nL = nL;
    const double imin3 = 1.0 / ((P.lambda_min * P.lambda_min) * P.lambda_min);
    const double imax3 = 1.0 / ((P.lambda_max * P.lambda_max) * P.lambda_max);
    int64_t tr_total = 0, carry_total = 0, keys_max = 1, Mall = 1;
    for (int l = 0; l < nL; l++) {
        LayerDev& Ly = v.layer[l];
        Ly.lo = P.lambda_min * std::ldexp(1.0, l);
        Ly.hi = (l + 1 == nL) ? P.lambda_max : P.lambda_min * std::ldexp(1.0, l + 1);
        Ly.ilo3 = 1.0 / ((Ly.lo * Ly.lo) * Ly.lo);
        Ly.ihi3 = 1.0 / ((Ly.hi * Ly.hi) * Ly.hi);
        const double mass = (Ly.ilo3 - Ly.ihi3) / (imin3 - imax3);
        h->expect[l] = ((double)h->N * (1.0 - h->p_fourier)) * mass;
        h->Mmax[l] = (int)std::floor(h->expect[l]) + 1;
        Ly.expect = h->expect[l];
        Ly.Mmax = h->Mmax[l];
        Mall = std::max<int64_t>(Mall, h->Mmax[l]);
        Ly.G = P.grid_layer[l];
        if (Ly.G < 0 || (Ly.G > 0 && (Ly.G % P.colour_K != 0 || Ly.G < P.colour_K)) || Ly.G > 256) {
            return WMCD_EINVAL;
        }
        Ly.invG = Ly.G > 0 ? (double)Ly.G / P.box_L : 0.0;
        Ly.carry_off = (int)carry_total;
        carry_total += (int64_t)Ly.G * Ly.G * Ly.G;
        keys_max = std::max<int64_t>(keys_max, (int64_t)Ly.G * Ly.G * Ly.G);
        Ly.tr_off = tr_total;
        tr_total += h->Mmax[l];
    }
    // second colourings: K floor(G / 2K) cells per axis where that leaves at least 2K (their
    // carries after all first-colouring ones)
    for (int l = 0; l < nL; l++) {
        LayerDev& Ly = v.layer[l];
        const int K = P.colour_K, G2 = K * (Ly.G / (2 * K));
        Ly.G2 = (((P.level2 >> l) & 1) && Ly.G > 0 && G2 >= 2 * K) ? G2 : 0;
        Ly.invG2 = Ly.G2 > 0 ? (double)Ly.G2 / P.box_L : 0.0;
        Ly.carry_off2 = (int)carry_total;
        carry_total += (int64_t)Ly.G2 * Ly.G2 * Ly.G2;
    }
    // time per accepted move: Eq. 57 with plane waves, Eq. 34 without (M4/(2 pi)^3 = 1/105)
    {
        const double la = 1.0 / (1.125 - kLn2), A02 = P.A0 * P.A0, la2 = la * la;
        if (P.planewave_mode != 0) h->dt_move = (6.0 * A02 * la2) / (105.0 * (double)h->N);
        else {
            double Nl = 3.0 / (imin3 - imax3);
            h->dt_move = ((2.0 * A02 * la2) / (105.0 * (double)h->N)) * (Nl * imin3) * (1.0 - P.lambda_min / P.lambda_max);
        }
    }
    // device state
    const int64_t N = h->N;
    const int64_t ncell = (int64_t)P.grid_f * P.grid_f * P.grid_f;
    int pw_cap = (int)std::min<double>(1e6, 4.0 * h->p_fourier * (double)N + 64.0);
    v.pw_blocks = (int)((N + 255) / 256);
    bool ok = true;
    ok = ok && !dalloc(h, &v.bead, N) && !dalloc(h, &v.bf, N) && !dalloc(h, &v.prev, N) && !dalloc(h, &v.img, 3 * N) &&
         !dalloc(h, &v.bnext, N) && !dalloc(h, &v.head, ncell);
    v.occ_w = (P.grid_f + 31) / 32;
    ok = ok && !dalloc(h, &v.occ, (size_t)P.grid_f * P.grid_f * v.occ_w);
    ok = ok && !dalloc(h, &v.slot_V, 3 * Mall) && !dalloc(h, &v.slot_p, 3 * Mall) && !dalloc(h, &v.slot_thr, Mall);
    ok = ok && !dalloc(h, &v.slot_lam, Mall) && !dalloc(h, &v.slot_bead, Mall) && !dalloc(h, &v.slot_key, Mall) &&
         !dalloc(h, &v.q_slots, Mall) && !dalloc(h, &v.defer, Mall) && !dalloc(h, &v.serial_list, Mall);
    ok = ok && !dalloc(h, &v.q_count, keys_max) && !dalloc(h, &v.q_start, keys_max) && !dalloc(h, &v.q_fill, keys_max);
    ok = ok && !dalloc(h, &v.serial_count, 4) && !dalloc(h, &v.carry_q, carry_total) &&
         !dalloc(h, &v.carry_serial, kMaxLayers);
    ok = ok && !dalloc(h, &v.tr_out, tr_total) && !dalloc(h, &v.tr_n, tr_total) && !dalloc(h, &v.tr_du, tr_total) && !dalloc(h, &v.tr_pw_out, pw_cap) &&
         !dalloc(h, &v.tr_pw_mode, pw_cap) && !dalloc(h, &v.tr_pw_count, 1) && !dalloc(h, &v.tr_pw_k, 3 * (size_t)pw_cap);
    double* d_kF = nullptr;
    if (P.planewave_mode >= 2) ok = ok && !dalloc(h, &d_kF, kKtN + 1);
    ok = ok && !dalloc(h, &v.ctr, C_NCTR) && !dalloc(h, &v.err, 1);
    ok = ok && !dalloc(h, &v.s_ids, N) && !dalloc(h, &v.s_d, 4 * N) && !dalloc(h, &v.s_new, 3 * N) &&
         !dalloc(h, &v.s_img, N) && !dalloc(h, &v.s_slot, N) && !dalloc(h, &v.s_changed, 3 * N) &&
         !dalloc(h, &v.s_box, 6 * N) && !dalloc(h, &v.s_pre, N + 1) &&
         !dalloc(h, &v.serial_tag, 1);
    ok = ok && !dalloc(h, &v.pw, 1) && !dalloc(h, &v.pw_new, 3 * N) && !dalloc(h, &v.pw_imgd, N) &&
         !dalloc(h, &v.pw_part, v.pw_blocks) && !dalloc(h, &v.pw_rebuild, 1) && !dalloc(h, &v.cl_stale, 1) &&
         !dalloc(h, &v.big, 1);
    ok = ok && !dalloc(h, &v.step, 2) && !dalloc(h, &v.counts, kMaxLayers + 1) && !dalloc(h, &h->dview, 1);
    int* d_modes = nullptr;
    double* d_cdf = nullptr;
    ok = ok && !dalloc(h, &d_modes, modes.size() + 3) && !dalloc(h, &d_cdf, cdf.size() + 1);
    ok = ok && !dalloc(h, &h->staging, 3 * N);
    // region assignment for staging: per-axis tables fine cell -> queue coordinate (-1 = the
    // cell straddles two regions of the colour), per layer and colour offset
    // (a second colouring's tables at schedule index kLevel2 + l)
    const bool any2 = [&] { for (int l = 0; l < nL; l++) if (v.layer[l].G2 > 0) return true; return false; }();
    const int n_tab = any2 ? kLevel2 + nL : nL;
    std::vector<int> tab((size_t)n_tab * P.colour_K * P.grid_f, -1);
    int64_t nq_max = 1;
    double expect_region = 0.0;
    for (int i = 0; i < n_tab; i++) {
        const int l = i;
        if (i >= nL && i < kLevel2) continue;
        const int G = i < kLevel2 ? v.layer[l].G : v.layer[l - kLevel2].G2, K = P.colour_K, Gf = P.grid_f;
        if (G == 0) continue;
        nq_max = std::max<int64_t>(nq_max, (int64_t)(G / K) * (G / K) * (G / K));
        if (expect_region == 0.0 && i < kLevel2) expect_region = (double)N * std::pow((double)K / G, 3.0);
        for (int c = 0; c < G; c++) {
            const int64_t lo = ceildiv((2 * (int64_t)c - (K - 1)) * Gf, 2 * (int64_t)G);
            const int64_t hi = floordiv((2 * (int64_t)c + 2 + (K - 1)) * Gf, 2 * (int64_t)G) - 1;
            for (int64_t u = lo; u <= hi; u++) {
                const int64_t f = ((u % Gf) + Gf) % Gf;
                tab[((size_t)l * K + c % K) * Gf + f] = c / K;
            }
        }
    }
    int* d_tab = nullptr;
    ok = ok && !dalloc(h, &v.rkey, N) && !dalloc(h, &v.rlist, N) && !dalloc(h, &v.rcount, nq_max) &&
         !dalloc(h, &v.rstart, nq_max) && !dalloc(h, &v.rfill, nq_max) && !dalloc(h, &d_tab, tab.size()) &&
         !dalloc(h, &v.hq_list, nq_max) && !dalloc(h, &v.hq_ctl, 4);
    if (!ok) return WMCD_ENOMEM;
    if (counting) return WMCD_OK;
    v.axis_tab = d_tab;
    {
        // staging capacity per warp: room for 16x the average bead count of a layer-0 region
        int cap = 256;
        while (cap < 1024 && cap < 16.0 * expect_region) cap *= 2;
        v.stage_cap = cap;
    }
    cudaMemcpyAsync(d_tab, tab.data(), tab.size() * sizeof(int), cudaMemcpyHostToDevice, s);
    v.tr_pw_cap = pw_cap;
    v.modes = d_modes;
    v.mode_cdf = d_cdf;
    v.n_modes = (int)cdf.size();
    v.expect_F = (double)N * h->p_fourier;
    v.pw_on = P.planewave_mode != 0;
    v.pw_mode = P.planewave_mode;
    v.pw_nl = P.lcut;
    v.p_disc = p_disc;
    v.kF0 = kF0;
    v.kF = d_kF;
    if (d_kF) cudaMemcpyAsync(d_kF, k_cdf_table().data(), (kKtN + 1) * sizeof(double), cudaMemcpyHostToDevice, s);
    {
        // shared-memory serial phase: small simulations without coloured layers, for the layers
        // of small scale (a support of a few beads; the large scales keep the cell lists)
        bool all_serial = true;
        for (int l = 0; l < nL; l++) all_serial = all_serial && v.layer[l].G == 0;
        v.smem_layers = 0;
        if (all_serial && N <= kSmemSerialMaxN)
            for (int l = 0; l < nL; l++)
                if (v.layer[l].hi <= 4.0 * P.lambda_min) v.smem_layers |= 1 << l;
        // whole-GPU moves: serial layers whose expected support (N times the volume fraction of
        // a ball of the band's geometric-mean scale) reaches big_support beads
        v.big_layers = 0;
        const double bs = P.big_support == 0 ? 2048.0 : (double)P.big_support;
        if (P.big_support >= 0)
            for (int l = 0; l < nL; l++) {
                if (v.layer[l].G != 0 || ((v.smem_layers >> l) & 1)) continue;
                const double lm = std::sqrt(v.layer[l].lo * v.layer[l].hi);
                const double ns = (double)N * (4.0 / 3.0) * kPi * lm * lm * lm / (P.box_L * P.box_L * P.box_L);
                if (ns >= bs) v.big_layers |= 1 << l;
            }
    }
    // launch bounds of this simulation
    {
        GroupDims& g = h->g;
        int dev = 0, n_sm = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) n_sm = 0;
        g.S = 1;
        g.ncap = P.n_cap;
        g.maxN = N;
        g.maxCells = std::max<int64_t>(ncell, 1);
        g.maxL = nL;
        g.maxK3 = P.colour_K * P.colour_K * P.colour_K;
        g.pw = v.pw_on != 0;
        g.maxMF = g.pw ? (int)std::floor(v.expect_F) + 1 : 0;
        g.stage_cap = v.stage_cap;
        g.pw_blocks = v.pw_blocks;
        g.prec_mask = 1 << P.precision;
        g.smem_maxN = v.smem_layers ? N : 0;
        for (int c = 0; c < 3; c++)
            if (v.smem_layers && N <= kSmemClassHi[c] && (c == 0 || N > kSmemClassHi[c - 1])) g.smem_cls[c] = N;
        g.any_global_serial = (v.smem_layers | v.big_layers) != (1 << nL) - 1;
        for (int l = 0; l < nL; l++) {
            const int G = v.layer[l].G, Q = G / P.colour_K;
            g.Mmax[l] = h->Mmax[l];
            g.keys[l] = std::max(G * G * G, 1);
            g.nq[l] = std::max(Q * Q * Q, 1);
            g.coloured[l] = G > 0;
            g.bigM[l] = ((v.big_layers >> l) & 1) ? h->Mmax[l] : 0;
            // a layer whose regions mostly overflow the base capacity but fit one block's shared
            // memory, and whose queues of one colour are no more than the SMs, stages each
            // region in a block of its own (a coarse layer of a dilute system): no queue waits
            // for an SM, and moves avoid the global cell walks
            const double region = G > 0 ? (double)N * std::pow((double)P.colour_K / G, 3.0) : 0.0;
            const int cmax = staged_cap_max(P.n_cap);
            g.cap_l[l] = (G > 0 && Q * Q * Q <= n_sm && region > 0.8 * v.stage_cap && region <= 0.8 * cmax) ? cmax : 0;
            const int G2 = v.layer[l].G2, Q2 = G2 / P.colour_K, l2 = kLevel2 + l;
            g.Mmax[l2] = h->Mmax[l];
            g.keys[l2] = std::max(G2 * G2 * G2, 1);
            g.nq[l2] = std::max(Q2 * Q2 * Q2, 1);
            g.coloured[l2] = G2 > 0;
        }
    }
    cudaMemsetAsync(v.step, 0, 2 * sizeof(uint64_t), s);
    cudaMemsetAsync(v.counts, 0, (kMaxLayers + 1) * sizeof(int), s);
    cudaMemsetAsync(v.cl_stale, 0, sizeof(int), s);
    cudaMemcpyAsync(h->dview, &v, sizeof(SimView), cudaMemcpyHostToDevice, s);
    // host -> device
    std::vector<uint8_t> bn(N, 0);
    {
        int64_t b = 0;
        for (int64_t c = 0; c < n_chains; c++) {
            for (int32_t k = 0; k + 1 < chain_len[c]; k++) bn[b + k] = 1;
            b += chain_len[c];
        }
    }
    cudaMemcpyAsync(v.bnext, bn.data(), N, cudaMemcpyHostToDevice, s);
    if (!modes.empty()) {
        cudaMemcpyAsync(d_modes, modes.data(), modes.size() * sizeof(int), cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(d_cdf, cdf.data(), cdf.size() * sizeof(double), cudaMemcpyHostToDevice, s);
    }
    cudaMemcpyAsync(h->staging, pos, 3 * N * sizeof(double), is_device_ptr(pos) ? cudaMemcpyDeviceToDevice
                                                                                 : cudaMemcpyHostToDevice, s);
    cudaMemsetAsync(v.img, 0, 3 * N * sizeof(int), s);
    cudaMemsetAsync(v.carry_q, 0, std::max<int64_t>(carry_total, 1) * sizeof(double), s);
    cudaMemsetAsync(v.carry_serial, 0, kMaxLayers * sizeof(double), s);
    cudaMemsetAsync(v.ctr, 0, C_NCTR * sizeof(unsigned long long), s);
    cudaMemsetAsync(v.err, 0, sizeof(int), s);
    cudaMemsetAsync(v.serial_tag, 0, sizeof(uint32_t), s);
    cudaMemsetAsync(v.pw, 0, sizeof(PWDev), s);
    cudaMemsetAsync(v.tr_out, 0, std::max<int64_t>(tr_total, 1), s);
    cudaMemsetAsync(v.tr_n, 0, std::max<int64_t>(tr_total, 1) * sizeof(int), s);
    k_fill_beads<<<grid_for(N), 256, 0, s>>>(v.bead, v.bf, h->staging, N);
    launch_cl_rebuild(h->dview, h->g, s, 0);
    if (cudaStreamSynchronize(s) != cudaSuccess || last_cuda_status()) { cudaGetLastError(); return WMCD_ECUDA; }
    int err = 0;
    cudaMemcpyAsync(&err, v.err, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) { cudaGetLastError(); return WMCD_ECUDA; }
    if (err) return WMCD_EINVAL;   // a coordinate outside [0, L) or not finite
    if (!arena) {
        // a lone simulation's side streams: the dense regions of a colour phase run on them
        // beside the ordinary ones (a batch brings its own)
        if (cudaStreamCreateWithFlags(&h->fj.side[0], cudaStreamNonBlocking) != cudaSuccess ||
            cudaStreamCreateWithFlags(&h->fj.side[1], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&h->fj.fork, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&h->fj.join[0], cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&h->fj.join[1], cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            return WMCD_ECUDA;
        }
    }
    h->arena = nullptr;            // later allocations (trace growth) are the handle's own
    return WMCD_OK;
}

extern "C" int wmcd_create(const wmcd_params* params, const double* pos, const int32_t* chain_len, int64_t n_chains,
                           void* stream, wmcd_handle** out) {
    if (!out || !pos || !chain_len || n_chains < 1) return WMCD_EINVAL;
    *out = nullptr;
    wmcd_handle* H = new (std::nothrow) wmcd_handle();
    if (!H) return WMCD_ENOMEM;
    const int rc = create_handle(H, params, pos, chain_len, n_chains, (cudaStream_t)stream, nullptr);
    if (rc) { destroy_handle(H); return rc; }
    *out = H;
    return WMCD_OK;
}

static int popcount3(int m) { return (m & 1) + ((m >> 1) & 1); }

// The launches of one sweep for every simulation of a group (Sec. V-VIII order: octave layers
// in ascending order, each in its colour phases then its serial phase, then the plane-wave
// slots), ending with the advance of the sweep counter. `hc` (a lone simulation only) holds
// this sweep's exact slot counts, used to leave out launches with no work; a batch launches
// every phase up to its bounds and the kernels return early where a simulation has none.
// Returns the number of kernels launched.
int64_t wmcd::enqueue_sweep(const SimView* d, const GroupDims& g, const int64_t* hc, Handle* prof, cudaStream_t s,
                            const ForkJoin* fj) {
    const int np = popcount3(g.prec_mask);
    int64_t launches = 0;
    { ProfScope ps(prof, 4, s); launch_counts(d, g, s); }
    launches += 1;
    for (int l = 0; l < g.maxL; l++) {
        if (hc && hc[l] <= 0) continue;
        { ProfScope ps(prof, 4, s); launch_slots(d, g, l, s); }
        launches += 1;
        // a coloured layer's phases, then those of its second colouring (schedule index
        // kLevel2 + l) over the slots the first deferred
        for (int ls = l; ls < 2 * kMaxLayers; ls += kLevel2) {
            if (!g.coloured[ls]) continue;
            { ProfScope ps(prof, 4, s); launch_bucket(d, g, ls, s); }
            for (int c = 0; c < g.maxK3; c++) { ProfScope ps(prof, 0, s); launches += launch_colour_staged(d, g, ls, c, s, fj); }
            { ProfScope ps(prof, 4, s); launch_defer_compact(d, g, ls, s); }
            launches += 5 + 1;
        }
        { ProfScope ps(prof, 1, s); launches += launch_serial(d, g, l, s, fj); }
        if (g.bigM[l] > 0) {
            const int64_t M = hc ? hc[l] : g.bigM[l];
            ProfScope ps(prof, 5, s);
            for (int64_t t = 0; t < M; t++) launches += launch_big(d, g, l, (int)t, s);
        }
    }
    if (g.pw) {
        const int64_t MF = hc ? hc[kMaxLayers] : g.maxMF;
        for (int64_t m = 0; m < MF; m++) {
            ProfScope ps(prof, 2, s);
            launches += launch_planewave(d, g, 0, (int)m, s);
        }
    }
    launch_advance(d, g, 0, s);
    return launches + 1;
}

static void run_sweep(Handle* h, cudaStream_t s) {
    int64_t hc[kMaxLayers + 1] = {0};
    for (int l = 0; l < h->nL; l++) hc[l] = slot_count(h, K_COUNT, l, h->sweep, h->expect[l]);
    hc[kMaxLayers] = h->g.pw ? slot_count(h, K_PWCOUNT, 0, h->sweep, h->v.expect_F) : 0;
    h->launches += enqueue_sweep(h->dview, h->g, hc, h, s, &h->fj);
    h->tr_pw_count = hc[kMaxLayers];
    h->sweep++;
}

extern "C" int wmcd_sweep(wmcd_handle* H, int64_t n_sweeps, void* stream) {
    if (!H || n_sweeps < 0) return WMCD_EINVAL;
    Handle* h = &H->h;
    cudaStream_t s = (cudaStream_t)stream;
    for (int64_t k = 0; k < n_sweeps; k++) run_sweep(h, s);
    return last_cuda_status();
}

extern "C" int wmcd_planewave(wmcd_handle* H, int64_t n_moves, void* stream) {
    if (!H || n_moves < 0) return WMCD_EINVAL;
    Handle* h = &H->h;
    if (h->P.planewave_mode == 0) return WMCD_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    if (n_moves > h->v.tr_pw_cap) {
        // grow the trace so every move of this call is recorded
        cudaStreamSynchronize(s);
        uint8_t* o = nullptr;
        int* md = nullptr;
        double* kk = nullptr;
        if (dalloc(h, &o, n_moves) || dalloc(h, &md, n_moves) || dalloc(h, &kk, 3 * n_moves)) return WMCD_ENOMEM;
        h->v.tr_pw_out = o;
        h->v.tr_pw_mode = md;
        h->v.tr_pw_k = kk;
        h->v.tr_pw_cap = (int)std::min<int64_t>(n_moves, 1 << 30);
        cudaMemcpyAsync(h->dview, &h->v, sizeof(SimView), cudaMemcpyHostToDevice, s);
        if (h->batch) batch_view_changed(h->batch);
    }
    for (int64_t m = 0; m < n_moves; m++) {
        ProfScope ps(h, 2, s);
        h->launches += launch_planewave(h->dview, h->g, 1, (int)m, s);
    }
    launch_advance(h->dview, h->g, 1, s);
    h->launches += 1;
    h->tr_pw_count = n_moves;
    h->pw_calls++;
    return last_cuda_status();
}

extern "C" int wmcd_positions(wmcd_handle* H, double* out, int unwrapped, void* stream) {
    if (!H || !out) return WMCD_EINVAL;
    Handle* h = &H->h;
    cudaStream_t s = (cudaStream_t)stream;
    const bool dev = is_device_ptr(out);
    double* dst = dev ? out : h->staging;
    k_read_beads<<<grid_for(h->N), 256, 0, s>>>(h->v.bead, h->v.img, h->v.L, unwrapped, dst, h->N);
    if (!dev) {
        cudaMemcpyAsync(out, h->staging, 3 * h->N * sizeof(double), cudaMemcpyDeviceToHost, s);
        if (cudaStreamSynchronize(s) != cudaSuccess) return WMCD_ECUDA;
    }
    return last_cuda_status();
}

extern "C" int wmcd_set_positions(wmcd_handle* H, const double* pos, void* stream) {
    if (!H || !pos) return WMCD_EINVAL;
    Handle* h = &H->h;
    cudaStream_t s = (cudaStream_t)stream;
    const bool dev = is_device_ptr(pos);
    cudaMemcpyAsync(h->staging, pos, 3 * h->N * sizeof(double), dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s);
    if (!dev && cudaStreamSynchronize(s) != cudaSuccess) return WMCD_ECUDA;
    cudaMemsetAsync(h->v.img, 0, 3 * h->N * sizeof(int), s);
    k_fill_beads<<<grid_for(h->N), 256, 0, s>>>(h->v.bead, h->v.bf, h->staging, h->N);
    launch_cl_rebuild(h->dview, h->g, s, 0);
    return last_cuda_status();
}

extern "C" int wmcd_stats(wmcd_handle* H, wmcd_stats_t* out, void* stream) {
    if (!H || !out) return WMCD_EINVAL;
    Handle* h = &H->h;
    cudaStream_t s = (cudaStream_t)stream;
    unsigned long long c[C_NCTR];
    int err = 0;
    cudaMemcpyAsync(c, h->v.ctr, sizeof c, cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(&err, h->v.err, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) return WMCD_ECUDA;
    std::memset(out, 0, sizeof *out);
    for (int l = 0; l < kMaxLayers; l++) {
        out->attempts[l] = (int64_t)c[C_ATT + l];
        out->accepts[l] = (int64_t)c[C_ACC + l];
        out->deferred[l] = (int64_t)c[C_DEF + l];
    }
    out->pw_attempts = (int64_t)c[C_PWATT];
    out->pw_accepts = (int64_t)c[C_PWACC];
    out->bead_updates = (int64_t)c[C_BU];
    out->accepted_total = (int64_t)c[C_ACCTOT];
    out->rechecks = (int64_t)c[C_RECHECK];
    out->partner_evals = (int64_t)c[C_PARTNER];
    out->sim_time = (double)out->accepted_total * h->dt_move;
    out->sweeps = (int64_t)h->sweep;
    out->n_layers = h->nL;
    out->dt_move = h->dt_move;
    out->p_fourier = h->p_fourier;
    out->error_flags = err;
    out->kernel_launches = h->launches;
    out->conc_bead_updates = (int64_t)c[C_CBU];
    out->conc_moved_beads = (int64_t)c[C_CMOVED];
    out->conc_partner_evals = (int64_t)c[C_CPE];
    out->moved_beads = (int64_t)c[C_MOVED];
    if (err & E_WALK) return WMCD_ETIMEOUT;
    if (err & E_NONFINITE) return WMCD_ESTATE;
    return WMCD_OK;
}

extern "C" int wmcd_trace(wmcd_handle* H, int layer, uint8_t* out, int32_t* n, int64_t cap, int64_t* count,
                          void* stream) {
    if (!H || !out || !n || !count || cap < 0) return WMCD_EINVAL;
    Handle* h = &H->h;
    cudaStream_t s = (cudaStream_t)stream;
    if (layer == -1) {
        int64_t m = std::min<int64_t>(std::min<int64_t>(h->tr_pw_count, cap), h->v.tr_pw_cap);
        if (m > 0) {
            cudaMemcpyAsync(out, h->v.tr_pw_out, m, cudaMemcpyDeviceToHost, s);
            cudaMemcpyAsync(n, h->v.tr_pw_mode, m * sizeof(int), cudaMemcpyDeviceToHost, s);
        }
        *count = h->tr_pw_count;
        return cudaStreamSynchronize(s) == cudaSuccess ? WMCD_OK : WMCD_ECUDA;
    }
    if (layer < 0 || layer >= h->nL) return WMCD_EINVAL;
    // the number of slots of the last sweep follows from the counter stream
    const int64_t M = h->sweep == 0 ? 0 : slot_count(h, K_COUNT, layer, h->sweep - 1, h->expect[layer]);
    const int64_t m = std::min<int64_t>(M, cap);
    if (m > 0) {
        cudaMemcpyAsync(out, h->v.tr_out + h->v.layer[layer].tr_off, m, cudaMemcpyDeviceToHost, s);
        cudaMemcpyAsync(n, h->v.tr_n + h->v.layer[layer].tr_off, m * sizeof(int), cudaMemcpyDeviceToHost, s);
    }
    *count = M;
    return cudaStreamSynchronize(s) == cudaSuccess ? WMCD_OK : WMCD_ECUDA;
}

extern "C" int wmcd_trace_du(wmcd_handle* H, int layer, double* out, int64_t cap, int64_t* count, void* stream) {
    if (!H || !out || !count || cap < 0) return WMCD_EINVAL;
    Handle* h = &H->h;
    if (layer < 0 || layer >= h->nL) return WMCD_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t M = h->sweep == 0 ? 0 : slot_count(h, K_COUNT, layer, h->sweep - 1, h->expect[layer]);
    const int64_t m = std::min<int64_t>(M, cap);
    if (m > 0) cudaMemcpyAsync(out, h->v.tr_du + h->v.layer[layer].tr_off, m * sizeof(double), cudaMemcpyDeviceToHost, s);
    *count = M;
    return cudaStreamSynchronize(s) == cudaSuccess ? WMCD_OK : WMCD_ECUDA;
}

// ---- checkpoint ----
struct StateHeader {
    uint64_t magic, n_beads, n_carry, sweep, pw_calls;
};
static const uint64_t kStateMagic = 0x574D434453543031ull;   // "WMCDST01"

static int64_t carry_count(const Handle* h) {
    int64_t c = 0;
    for (int l = 0; l < h->nL; l++) {
        const LayerDev& Ly = h->v.layer[l];
        c += (int64_t)Ly.G * Ly.G * Ly.G + (int64_t)Ly.G2 * Ly.G2 * Ly.G2;
    }
    return c;
}
static int64_t state_bytes(const Handle* h) {
    return (int64_t)sizeof(StateHeader) + 3 * h->N * (int64_t)(sizeof(double) + sizeof(int)) +
           carry_count(h) * (int64_t)sizeof(double) + kMaxLayers * (int64_t)sizeof(double) + (int64_t)sizeof(PWDev) +
           C_NCTR * (int64_t)sizeof(unsigned long long) + (int64_t)sizeof(uint32_t);
}

extern "C" int wmcd_trace_pw_k(wmcd_handle* H, double* out, int64_t cap, int64_t* count, void* stream) {
    if (!H || !count || cap < 0 || (cap > 0 && !out)) return WMCD_EINVAL;
    Handle* h = &H->h;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t m = std::min<int64_t>(std::min<int64_t>(h->tr_pw_count, cap), h->v.tr_pw_cap);
    if (m > 0) cudaMemcpyAsync(out, h->v.tr_pw_k, 3 * sizeof(double) * (size_t)m, cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) { cudaGetLastError(); return WMCD_ECUDA; }
    *count = h->tr_pw_count;
    return last_cuda_status();
}

extern "C" int wmcd_state_size(wmcd_handle* H, int64_t* bytes) {
    if (!H || !bytes) return WMCD_EINVAL;
    *bytes = state_bytes(&H->h);
    return WMCD_OK;
}

extern "C" int wmcd_get_state(wmcd_handle* H, void* buf, int64_t bytes, void* stream) {
    if (!H || !buf) return WMCD_EINVAL;
    Handle* h = &H->h;
    if (bytes < state_bytes(h)) return WMCD_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    char* p = (char*)buf;
    StateHeader hd{kStateMagic, (uint64_t)h->N, (uint64_t)carry_count(h), h->sweep, h->pw_calls};
    std::memcpy(p, &hd, sizeof hd);
    p += sizeof hd;
    k_read_beads<<<grid_for(h->N), 256, 0, s>>>(h->v.bead, h->v.img, h->v.L, 0, h->staging, h->N);
    cudaMemcpyAsync(p, h->staging, 3 * h->N * sizeof(double), cudaMemcpyDeviceToHost, s);
    p += 3 * h->N * sizeof(double);
    cudaMemcpyAsync(p, h->v.img, 3 * h->N * sizeof(int), cudaMemcpyDeviceToHost, s);
    p += 3 * h->N * sizeof(int);
    const int64_t nc = carry_count(h);
    if (nc) cudaMemcpyAsync(p, h->v.carry_q, nc * sizeof(double), cudaMemcpyDeviceToHost, s);
    p += nc * sizeof(double);
    cudaMemcpyAsync(p, h->v.carry_serial, kMaxLayers * sizeof(double), cudaMemcpyDeviceToHost, s);
    p += kMaxLayers * sizeof(double);
    cudaMemcpyAsync(p, h->v.pw, sizeof(PWDev), cudaMemcpyDeviceToHost, s);
    p += sizeof(PWDev);
    cudaMemcpyAsync(p, h->v.ctr, C_NCTR * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s);
    p += C_NCTR * sizeof(unsigned long long);
    cudaMemcpyAsync(p, h->v.serial_tag, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
    return cudaStreamSynchronize(s) == cudaSuccess ? last_cuda_status() : WMCD_ECUDA;
}

extern "C" int wmcd_set_state(wmcd_handle* H, const void* buf, int64_t bytes, void* stream) {
    if (!H || !buf) return WMCD_EINVAL;
    Handle* h = &H->h;
    if (bytes < state_bytes(h)) return WMCD_EINVAL;
    StateHeader hd;
    std::memcpy(&hd, buf, sizeof hd);
    if (hd.magic != kStateMagic || hd.n_beads != (uint64_t)h->N || hd.n_carry != (uint64_t)carry_count(h))
        return WMCD_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const char* p = (const char*)buf + sizeof hd;
    cudaMemcpyAsync(h->staging, p, 3 * h->N * sizeof(double), cudaMemcpyHostToDevice, s);
    p += 3 * h->N * sizeof(double);
    cudaMemcpyAsync(h->v.img, p, 3 * h->N * sizeof(int), cudaMemcpyHostToDevice, s);
    p += 3 * h->N * sizeof(int);
    const int64_t nc = carry_count(h);
    if (nc) cudaMemcpyAsync(h->v.carry_q, p, nc * sizeof(double), cudaMemcpyHostToDevice, s);
    p += nc * sizeof(double);
    cudaMemcpyAsync(h->v.carry_serial, p, kMaxLayers * sizeof(double), cudaMemcpyHostToDevice, s);
    p += kMaxLayers * sizeof(double);
    cudaMemcpyAsync(h->v.pw, p, sizeof(PWDev), cudaMemcpyHostToDevice, s);
    p += sizeof(PWDev);
    cudaMemcpyAsync(h->v.ctr, p, C_NCTR * sizeof(unsigned long long), cudaMemcpyHostToDevice, s);
    p += C_NCTR * sizeof(unsigned long long);
    cudaMemcpyAsync(h->v.serial_tag, p, sizeof(uint32_t), cudaMemcpyHostToDevice, s);
    k_fill_beads<<<grid_for(h->N), 256, 0, s>>>(h->v.bead, h->v.bf, h->staging, h->N);
    launch_cl_rebuild(h->dview, h->g, s, 0);
    cudaMemsetAsync(h->v.err, 0, sizeof(int), s);
    h->sweep = hd.sweep;
    h->pw_calls = hd.pw_calls;
    {
        static thread_local uint64_t st[2];
        st[0] = hd.sweep;
        st[1] = hd.pw_calls;
        cudaMemcpyAsync(h->v.step, st, sizeof st, cudaMemcpyHostToDevice, s);
    }
    return cudaStreamSynchronize(s) == cudaSuccess ? last_cuda_status() : WMCD_ECUDA;
}

extern "C" int wmcd_profile(wmcd_handle* H, int enable) {
    if (!H) return WMCD_EINVAL;
    H->h.prof = enable != 0;
    return WMCD_OK;
}

int wmcd::take_kernel_times(Handle* h, int64_t* launches, double* ms, int n_classes) {
    prof_harvest(h);
    for (int c = 0; c < n_classes && c < 8; c++) {
        if (launches) launches[c] = h->prof_launches[c];
        if (ms) ms[c] = h->prof_ms[c];
        h->prof_launches[c] = 0;
        h->prof_ms[c] = 0.0;
    }
    return WMCD_OK;
}

extern "C" int wmcd_kernel_times(wmcd_handle* H, int64_t* launches, double* ms, int n_classes, void* stream) {
    if (!H || n_classes < 0) return WMCD_EINVAL;
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return WMCD_ECUDA;
    return take_kernel_times(&H->h, launches, ms, n_classes);
}

extern "C" int wmcd_audit(wmcd_handle* H, int64_t capacity, void* stream) {
    if (!H) return WMCD_EINVAL;
    Handle* h = &H->h;
    cudaStream_t s = (cudaStream_t)stream;
    if (capacity < 0) {
        h->v.audit = nullptr;
    } else {
        if (cudaStreamSynchronize(s) != cudaSuccess) { cudaGetLastError(); return WMCD_ECUDA; }
        AuditDev* a = nullptr;
        double* rec = nullptr;
        if (dalloc(h, &a, 1) || dalloc(h, &rec, 4 * (size_t)std::max<int64_t>(capacity, 1))) return WMCD_ENOMEM;
        AuditDev init;
        std::memset(&init, 0, sizeof init);
        init.rec = rec;
        init.cap = capacity;
        cudaMemcpyAsync(a, &init, sizeof init, cudaMemcpyHostToDevice, s);
        h->v.audit = a;
    }
    cudaMemcpyAsync(h->dview, &h->v, sizeof(SimView), cudaMemcpyHostToDevice, s);
    if (h->batch) batch_view_changed(h->batch);
    return cudaStreamSynchronize(s) == cudaSuccess ? last_cuda_status() : WMCD_ECUDA;
}

extern "C" int wmcd_audit_read(wmcd_handle* H, wmcd_audit_t* out, double* rec, int64_t cap, void* stream) {
    if (!H || !out || cap < 0 || (cap > 0 && !rec)) return WMCD_EINVAL;
    Handle* h = &H->h;
    if (!h->v.audit) return WMCD_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    AuditDev a;
    cudaMemcpyAsync(&a, h->v.audit, sizeof a, cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) { cudaGetLastError(); return WMCD_ECUDA; }
    float mr;
    std::memcpy(&mr, &a.max_ratio, sizeof mr);
    out->decisions = (int64_t)a.n;
    out->outside = (int64_t)a.outside;
    out->violations = (int64_t)a.viol;
    out->flips = (int64_t)a.flip;
    out->max_ratio = (double)mr;
    out->records = (int64_t)std::min<unsigned long long>(a.n, (unsigned long long)a.cap);
    const int64_t k = std::min<int64_t>(cap, out->records);
    if (k > 0) {
        cudaMemcpyAsync(rec, a.rec, 4 * sizeof(double) * (size_t)k, cudaMemcpyDeviceToHost, s);
        if (cudaStreamSynchronize(s) != cudaSuccess) { cudaGetLastError(); return WMCD_ECUDA; }
    }
    return last_cuda_status();
}

extern "C" int wmcd_device_bytes(wmcd_handle* H, int64_t* bytes) {
    if (!H || !bytes) return WMCD_EINVAL;
    *bytes = (int64_t)H->h.bytes;
    return WMCD_OK;
}

void wmcd::destroy_handle(wmcd_handle* H) {
    Handle* h = &H->h;
    cudaDeviceSynchronize();
    for (auto& u : h->ev_used) { cudaEventDestroy(u.second.first); cudaEventDestroy(u.second.second); }
    for (auto e : h->ev_pool) cudaEventDestroy(e);
    for (void* p : h->allocs) cudaFree(p);
    for (int c = 0; c < 2; c++) {
        if (h->fj.side[c]) cudaStreamDestroy(h->fj.side[c]);
        if (h->fj.join[c]) cudaEventDestroy(h->fj.join[c]);
    }
    if (h->fj.fork) cudaEventDestroy(h->fj.fork);
    cudaGetLastError();
    delete H;
}

extern "C" int wmcd_set_block(wmcd_handle* H, int stage_warps, int serial_threads) {
    if (!H || stage_warps < 1 || stage_warps > kMaxStageWarps) return WMCD_EINVAL;
    if (serial_threads != 32 && serial_threads != 128 && serial_threads != 512) return WMCD_EINVAL;
    H->h.g.block_warps = stage_warps;
    H->h.g.serial_threads = serial_threads;
    return WMCD_OK;
}

extern "C" int wmcd_destroy(wmcd_handle* H) {
    if (!H) return WMCD_EINVAL;
    if (H->h.batch) return WMCD_EINVAL;   // owned by a batch: wmcd_batch_retire releases it
    destroy_handle(H);
    return WMCD_OK;
}

extern "C" const char* wmcd_strerror(int status) {
    switch (status) {
        case WMCD_OK: return "ok";
        case WMCD_EINVAL: return "invalid argument or parameter";
        case WMCD_ENOMEM: return "out of memory";
        case WMCD_ECUDA: return "CUDA runtime error";
        case WMCD_ETIMEOUT: return "a bounded device-side wait or list walk gave up";
        case WMCD_ESTATE: return "non-finite or out-of-box positions detected";
        case WMCD_EFULL: return "the batch has no free slot or pool room for the simulation";
        default: return "unknown status";
    }
}

namespace wmcd {
// Plane-wave mode table written into caller buffers, using only static storage (for the
// allocation-free entry point): modes |l| <= lcut in the enumeration order of wmcd_create
// and their cumulative probabilities. Returns the number of modes, or -1 if cap is too small.
// Not thread-safe (one static work array).
int mode_table_static(double L, double lmax, int lcut, int* modes, double* cdf, int cap) {
    static double acc[40001];
    static double gq[((2 * 8 + 1) * (2 * 8 + 1) * (2 * 8 + 1))];
    const double h = kPi / 20.0;
    const int panels = 40000;
    acc[panels] = tail3(panels * h);
    for (int p = panels - 1; p >= 0; p--) acc[p] = acc[p + 1] + gl10(p * h, (p + 1) * h);
    int n = 0;
    double tot = 0.0;
    for (int lx = -lcut; lx <= lcut; lx++)
        for (int ly = -lcut; ly <= lcut; ly++)
            for (int lz = -lcut; lz <= lcut; lz++) {
                const int l2 = lx * lx + ly * ly + lz * lz;
                if (l2 > lcut * lcut) continue;
                if (n >= cap || n >= (int)(sizeof gq / sizeof gq[0])) return -1;
                modes[3 * n] = lx; modes[3 * n + 1] = ly; modes[3 * n + 2] = lz;
                const double q = kTwoPi * std::sqrt((double)l2) / L * lmax;
                double g;
                if (q >= panels * h) g = tail3(q);
                else {
                    const int p = (int)(q / h);
                    const double top = (p + 1) * h;
                    g = acc[p + 1] + (top > q ? gl10(q, top) : 0.0);
                }
                gq[n++] = g;
                tot += g;
            }
    double a = 0.0;
    for (int i = 0; i < n; i++) { a += gq[i]; cdf[i] = a / tot; }
    return n;
}
}  // namespace wmcd
