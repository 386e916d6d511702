/*
 * Seeded synthetic initial configurations for bead-spring systems in a periodic cube.
 *
 * This module holds none of the simulation method's arithmetic: it only places beads.
 * It is shared by the CUDA path and the CPU oracle as their common input source.
 *
 *  - chains: each chain starts at a uniform random point of the box and grows as a
 *    random walk of fixed step length with isotropic steps; a step that lands closer
 *    than `min_dist` (minimum image) to any bead already placed is redrawn, up to
 *    100 tries, after which the whole chain is restarted.
 *  - spheres: random sequential addition with the same minimum distance.
 *
 * Only +, -, *, / and sqrt are used on floating point values, so the output is
 * bit-identical on every IEEE-754 machine (x86-64 and aarch64 alike).
 * The generator is xoshiro256** seeded by splitmix64.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

typedef struct { uint64_t s[4]; } rng_t;

static uint64_t splitmix64(uint64_t* x) {
    uint64_t z = (*x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
static uint64_t rotl(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }
static uint64_t next_u64(rng_t* r) {
    uint64_t* s = r->s;
    uint64_t res = rotl(s[1] * 5, 7) * 9;
    uint64_t t = s[1] << 17;
    s[2] ^= s[0]; s[3] ^= s[1]; s[1] ^= s[2]; s[0] ^= s[3];
    s[2] ^= t; s[3] = rotl(s[3], 45);
    return res;
}
static double uni(rng_t* r) { return (double)(next_u64(r) >> 11) * (1.0 / 9007199254740992.0); }
static void rng_seed(rng_t* r, uint64_t seed) {
    uint64_t x = seed;
    for (int i = 0; i < 4; i++) r->s[i] = splitmix64(&x);
}
/* isotropic unit vector by rejection from the cube (no transcendental functions) */
static void unit_vec(rng_t* r, double v[3]) {
    for (;;) {
        double x = 2.0 * uni(r) - 1.0, y = 2.0 * uni(r) - 1.0, z = 2.0 * uni(r) - 1.0;
        double q = x * x + y * y + z * z;
        if (q > 1e-6 && q <= 1.0) {
            double s = 1.0 / sqrt(q);
            v[0] = x * s; v[1] = y * s; v[2] = z * s;
            return;
        }
    }
}

/* ---- spatial hash of placed beads (cell side >= min_dist), open addressing ---- */
typedef struct {
    int64_t* key;   /* packed cell id, -1 = empty */
    int64_t* head;  /* first bead in the cell */
    int64_t* next;  /* per bead */
    uint64_t mask;
    int64_t G;      /* cells per axis */
    double L, inv_h;
} grid_t;

static uint64_t hmix(uint64_t k) {
    k ^= k >> 33; k *= 0xff51afd7ed558ccdull; k ^= k >> 33; k *= 0xc4ceb9fe1a85ec53ull; k ^= k >> 33;
    return k;
}
static int grid_init(grid_t* g, int64_t nmax, double L, double min_dist) {
    g->L = L;
    g->G = (int64_t)floor(L / min_dist);
    if (g->G < 1) g->G = 1;
    if (g->G > 2000000) g->G = 2000000;
    g->inv_h = (double)g->G / L;
    uint64_t cap = 1024;
    while (cap < (uint64_t)(2 * nmax + 16)) cap <<= 1;
    g->mask = cap - 1;
    g->key = (int64_t*)malloc(cap * sizeof(int64_t));
    g->head = (int64_t*)malloc(cap * sizeof(int64_t));
    g->next = (int64_t*)malloc((size_t)(nmax > 0 ? nmax : 1) * sizeof(int64_t));
    if (!g->key || !g->head || !g->next) return -1;
    for (uint64_t i = 0; i < cap; i++) { g->key[i] = -1; g->head[i] = -1; }
    return 0;
}
static void grid_free(grid_t* g) { free(g->key); free(g->head); free(g->next); }
static int64_t cell_of(const grid_t* g, double x) {
    int64_t c = (int64_t)floor(x * g->inv_h);
    if (c < 0) c = 0;
    if (c >= g->G) c = g->G - 1;
    return c;
}
static int64_t pack(const grid_t* g, int64_t cx, int64_t cy, int64_t cz) {
    cx = ((cx % g->G) + g->G) % g->G; cy = ((cy % g->G) + g->G) % g->G; cz = ((cz % g->G) + g->G) % g->G;
    return (cx * g->G + cy) * g->G + cz;
}
static uint64_t slot_find(const grid_t* g, int64_t k) {
    uint64_t h = hmix((uint64_t)k) & g->mask;
    while (g->key[h] != -1 && g->key[h] != k) h = (h + 1) & g->mask;
    return h;
}
static void grid_insert(grid_t* g, int64_t id, const double* p) {
    int64_t k = pack(g, cell_of(g, p[0]), cell_of(g, p[1]), cell_of(g, p[2]));
    uint64_t h = slot_find(g, k);
    if (g->key[h] == -1) { g->key[h] = k; g->head[h] = -1; }
    g->next[id] = g->head[h];
    g->head[h] = id;
}
static void grid_remove_last(grid_t* g, int64_t id, const double* p) {
    /* remove bead `id`, which must be the most recent insertion into its cell */
    int64_t k = pack(g, cell_of(g, p[0]), cell_of(g, p[1]), cell_of(g, p[2]));
    uint64_t h = slot_find(g, k);
    if (g->key[h] == k && g->head[h] == id) g->head[h] = g->next[id];
}
static double wrapd(double x, double L) {
    if (x >= L) x -= L;
    else if (x < 0.0) x += L;
    if (x >= L || x < 0.0) x = 0.0;
    return x;
}
static double mind(double d, double L) {
    if (d > 0.5 * L) d -= L;
    else if (d < -0.5 * L) d += L;
    return d;
}
static int clashes(const grid_t* g, const double* pos, const double* p, double min_d2) {
    int64_t cx = cell_of(g, p[0]), cy = cell_of(g, p[1]), cz = cell_of(g, p[2]);
    int64_t r = g->G >= 3 ? 1 : 0;
    for (int64_t dx = -r; dx <= r; dx++)
        for (int64_t dy = -r; dy <= r; dy++)
            for (int64_t dz = -r; dz <= r; dz++) {
                int64_t k = pack(g, cx + dx, cy + dy, cz + dz);
                uint64_t h = slot_find(g, k);
                if (g->key[h] != k) continue;
                for (int64_t b = g->head[h]; b >= 0; b = g->next[b]) {
                    double ex = mind(pos[3 * b] - p[0], g->L), ey = mind(pos[3 * b + 1] - p[1], g->L),
                           ez = mind(pos[3 * b + 2] - p[2], g->L);
                    if (ex * ex + ey * ey + ez * ez < min_d2) return 1;
                }
            }
    return 0;
}
static int clashes_all(const double* pos, int64_t n, const double* p, double min_d2, double L) {
    for (int64_t b = 0; b < n; b++) {
        double ex = mind(pos[3 * b] - p[0], L), ey = mind(pos[3 * b + 1] - p[1], L), ez = mind(pos[3 * b + 2] - p[2], L);
        if (ex * ex + ey * ey + ez * ez < min_d2) return 1;
    }
    return 0;
}

/*
 * Place `n_chains` chains of the given lengths followed by `n_spheres` free spheres.
 * out: (sum(chain_len) + n_spheres) * 3 doubles, positions wrapped into [0, L).
 * Returns 0 on success, -1 on allocation failure, -2 if placement failed.
 */
int wmcd_gen_system(int64_t n_chains, const int32_t* chain_len, int64_t n_spheres, double L,
                    double bond, double min_dist, uint64_t seed, double* out) {
    int64_t nb = 0;
    for (int64_t c = 0; c < n_chains; c++) nb += chain_len[c];
    int64_t ntot = nb + n_spheres;
    grid_t g;
    if (grid_init(&g, ntot, L, min_dist) != 0) return -1;
    /* brute force only when the box is too small for a 3x3x3 stencil */
    int brute = g.G < 3;
    rng_t r;
    rng_seed(&r, seed);
    double md2 = min_dist * min_dist;
    int64_t placed = 0;
    for (int64_t c = 0; c < n_chains; c++) {
        int64_t len = chain_len[c];
        int restarts = 0;
    restart_chain:
        if (restarts > 1000) { grid_free(&g); return -2; }
        {
            int64_t start = placed;
            int64_t k = 0;
            while (k < len) {
                double p[3];
                int ok = 0;
                for (int t = 0; t < 100 && !ok; t++) {
                    if (k == 0) {
                        p[0] = uni(&r) * L; p[1] = uni(&r) * L; p[2] = uni(&r) * L;
                    } else {
                        double v[3];
                        unit_vec(&r, v);
                        const double* q = out + 3 * (start + k - 1);
                        p[0] = q[0] + bond * v[0]; p[1] = q[1] + bond * v[1]; p[2] = q[2] + bond * v[2];
                    }
                    p[0] = wrapd(p[0], L); p[1] = wrapd(p[1], L); p[2] = wrapd(p[2], L);
                    ok = brute ? !clashes_all(out, start + k, p, md2, L) : !clashes(&g, out, p, md2);
                }
                if (!ok) {
                    /* undo this chain and start it again */
                    for (int64_t j = start + k - 1; j >= start; j--) grid_remove_last(&g, j, out + 3 * j);
                    placed = start;
                    restarts++;
                    goto restart_chain;
                }
                memcpy(out + 3 * (start + k), p, sizeof p);
                if (!brute) grid_insert(&g, start + k, p);
                k++;
            }
            placed = start + len;
        }
    }
    for (int64_t s = 0; s < n_spheres; s++) {
        double p[3];
        int ok = 0;
        for (int t = 0; t < 100000 && !ok; t++) {
            p[0] = uni(&r) * L; p[1] = uni(&r) * L; p[2] = uni(&r) * L;
            ok = brute ? !clashes_all(out, placed, p, md2, L) : !clashes(&g, out, p, md2);
        }
        if (!ok) { grid_free(&g); return -2; }
        memcpy(out + 3 * placed, p, sizeof p);
        if (!brute) grid_insert(&g, placed, p);
        placed++;
    }
    grid_free(&g);
    return 0;
}

/* log-uniform integer draws in [lo, hi] (used for ensembles of uneven chain lengths).
 * Uses libm log/exp, so a length can differ between machines when a draw lands
 * within rounding of a half-integer; ensembles are regenerated per machine. */
int wmcd_gen_loguniform_lengths(int64_t n, int32_t lo, int32_t hi, uint64_t seed, int32_t* out) {
    rng_t r;
    rng_seed(&r, seed ^ 0x5DEECE66Dull);
    double a = log((double)lo), b = log((double)hi);
    for (int64_t i = 0; i < n; i++) {
        double v = exp(a + (b - a) * uni(&r));
        int32_t k = (int32_t)floor(v + 0.5);
        if (k < lo) k = lo;
        if (k > hi) k = hi;
        out[i] = k;
    }
    return 0;
}
