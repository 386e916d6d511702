// WMCD kernels for sm_103a: cell list, slot generation and bucketing, the concurrent
// (one warp per queue) wavelet kernel, the serial wavelet kernel and the plane-wave kernels.
//
// Nothing here is a dense contraction, so there are no tensor-core paths: the work is
// gathers of 32-byte bead records through per-cell linked lists, pair energies and
// warp / block reductions. See the host file for the order of launches in a sweep.
#include <algorithm>
#include <cfloat>
#include "wmcd_internal.h"

namespace wmcd {

__device__ __forceinline__ void set_err(const SimView& v, int bit) { atomicOr(v.err, bit); }

// Acceptance threshold of a move on its draw w (accept iff dU <= threshold): Metropolis
// (Eq. 20), -kT ln(1 - u) with u in [0, 1); Glauber (Secs. V.C, VIII), accept with probability
// 1 / (1 + exp(dU / kT)), i.e. kT (ln(1 - u) - ln u) with u in (0, 1).
// Centre uniform in the box (Sec. V.D, the homogeneous scheme, P_b = 1/L^3): each coordinate L
// times a 32-bit uniform of the slot's own draw.
__device__ __forceinline__ void uniform_centre(const SimView& v, int l, uint64_t sweep, uint32_t j, double b[3]) {
    const u4 w = draw(v.k0, v.k1, K_BUNI, l, sweep, j, 0);
    b[0] = mul(v.L, (double)w.x * (1.0 / 4294967296.0));
    b[1] = mul(v.L, (double)w.y * (1.0 / 4294967296.0));
    b[2] = mul(v.L, (double)w.z * (1.0 / 4294967296.0));
}
// Amplitude with a uniform centre: A0 lam / sqrt(nbar), nbar = N (4 pi / 3) lam^3 / L^3 the mean
// support at the global density (Eq. 29 with the mean count)
__device__ __forceinline__ double uniform_aw(const SimView& v, double lam) {
    const double nbar = dvd(mul((double)v.N, mul(4.0 * kPi / 3.0, mul(mul(lam, lam), lam))), mul(mul(v.L, v.L), v.L));
    return dvd(mul(v.A0, lam), sqr_t(nbar));
}
__device__ __forceinline__ double accept_threshold(const SimView& v, const u4& w) {
    if (v.acceptance == 1) {
        const double u = u_open(w.x, w.y);
        return v.kT * (log(1.0 - u) - log(u));
    }
    return -v.kT * log(1.0 - u53(w.x, w.y));
}

// One audited mixed-precision decision: d32 and band as the decision used them, thr_cmp the
// threshold d32 was compared with, d64 the binary64 energy change and thr64 its threshold.
__device__ void audit_record(const SimView& v, double d32, double band, double thr_cmp, double d64, double thr64) {
    AuditDev* A = v.audit;
    const unsigned long long k = atomicAdd(&A->n, 1ull);
    const bool outside = isfinite(d32) && isfinite(band) && fabs(d32 - thr_cmp) > band;
    double ratio = 0.0;
    if (isfinite(d32) && isfinite(d64) && isfinite(band) && band > 0.0) ratio = fabs(d32 - d64) / band;
    if (outside) atomicAdd(&A->outside, 1ull);
    if (ratio >= 1.0) atomicAdd(&A->viol, 1ull);
    if (outside && ((d32 <= thr_cmp) != (d64 <= thr64))) atomicAdd(&A->flip, 1ull);
    atomicMax(&A->max_ratio, __float_as_uint((float)ratio));
    if ((long long)k < A->cap) {
        A->rec[4 * k] = d32; A->rec[4 * k + 1] = d64; A->rec[4 * k + 2] = band; A->rec[4 * k + 3] = thr64;
    }
}

// wrap and minimum image with the rare correction behind a branch that the lanes of `mask` take
// together: written plainly, the correction's binary64 add is predicated and, on this part,
// occupies the binary64 pipe even when no lane needs it
__device__ __forceinline__ double wrap_u(double x, double L, unsigned mask, int* im) {
    if (__any_sync(mask, ge_pos(x, L) || lt_zero(x))) x = wrap(x, L, im);
    return x;
}
__device__ __forceinline__ double mi_u(double d, double L, double h, unsigned mask) {
    if (__any_sync(mask, gt_pos(d, h) || lt_neg(d, h))) d = mi(d, L, h);
    return d;
}
// the same for the three components of a vector, with one vote for all three
__device__ __forceinline__ void wrap3_u(double x[3], double L, unsigned mask, int* im) {
    const bool need = ge_pos(x[0], L) || lt_zero(x[0]) || ge_pos(x[1], L) || lt_zero(x[1]) || ge_pos(x[2], L) ||
                      lt_zero(x[2]);
    if (__any_sync(mask, need))
        for (int a = 0; a < 3; a++) x[a] = wrap(x[a], L, im ? &im[a] : nullptr);
}
__device__ __forceinline__ void mi3_u(double d[3], double L, double h, unsigned mask) {
    const bool need = gt_pos(d[0], h) || lt_neg(d[0], h) || gt_pos(d[1], h) || lt_neg(d[1], h) || gt_pos(d[2], h) ||
                      lt_neg(d[2], h);
    if (__any_sync(mask, need))
        for (int a = 0; a < 3; a++) d[a] = mi(d[a], L, h);
}

// Every kernel serves a group of simulations: blockIdx.y selects one, whose view is copied
// into shared memory once per block. SIM_EXIT_IF tests a condition on the view in global
// memory first, so blocks of a simulation with no work in this launch leave without the copy.
#define SIM_EXIT_IF(cond)                                                                     \
    {                                                                                         \
        const SimView& gv = vs[blockIdx.y];                                                   \
        if (cond) return;                                                                     \
    }
#define SIM_PROLOGUE                                                                          \
    __shared__ SimView sv_;                                                                   \
    {                                                                                         \
        const int* src_ = (const int*)(vs + blockIdx.y);                                      \
        int* dst_ = (int*)&sv_;                                                               \
        for (int w_ = threadIdx.x; w_ < (int)(sizeof(SimView) / 4); w_ += blockDim.x)        \
            dst_[w_] = src_[w_];                                                              \
    }                                                                                         \
    __syncthreads();                                                                          \
    const SimView& v = sv_;

__device__ __forceinline__ int cell_lin(const SimView& v, double x, double y, double z) {
    return fine_cell(x, v.invf, v.Gf) + v.Gf * (fine_cell(y, v.invf, v.Gf) + v.Gf * fine_cell(z, v.invf, v.Gf));
}
__device__ __forceinline__ int wrapi(int c, int G) { c %= G; return c < 0 ? c + G : c; }

// occupancy bit of fine cell c (atomic: cells of neighbouring regions share a word)
__device__ __forceinline__ void occ_bit(const SimView& v, int c, bool on) {
    if (!v.occ) return;
    const int x = c % v.Gf, yz = c / v.Gf;
    uint32_t* w = &v.occ[(size_t)yz * v.occ_w + (x >> 5)];
    if (on) atomicOr(w, 1u << (x & 31));
    else atomicAnd(w, ~(1u << (x & 31)));
}
// the bits of occupancy word wi of a row that lie in the cell range [a, b) of the row
__device__ __forceinline__ uint32_t occ_masked(uint32_t word, int a, int b, int wi) {
    const int lo = max(a - (wi << 5), 0), hi = min(b - (wi << 5), 32);
    if (hi <= lo) return 0u;
    return word & (hi >= 32 ? 0xffffffffu : ((1u << hi) - 1u)) & ~((1u << lo) - 1u);
}
// Move bead m from the list of fine cell oc to the head of the list of ncl (lists doubly linked
// through Bead::next and prev[]), keeping both cells' occupancy bits.
__device__ __forceinline__ void relink(const SimView& v, int m, int oc, int ncl) {
    const int pr = v.prev[m], nx = v.bead[m].next;
    if (pr >= 0) v.bead[pr].next = nx; else v.head[oc] = nx;
    if (nx >= 0) v.prev[nx] = pr;
    if (pr < 0 && nx < 0) occ_bit(v, oc, false);
    const int hd = v.head[ncl];
    v.bead[m].next = hd;
    v.prev[m] = -1;
    if (hd >= 0) v.prev[hd] = m;
    v.head[ncl] = m;
    occ_bit(v, ncl, true);
}

// The cell changes of one accepted move, (bead, old cell, new cell) in cm/co/cn, applied by the
// nt threads of a block together: one thread per old cell unlinks that cell's leaving beads,
// then one thread per new cell pushes its arriving beads in entry order, so the lists end as
// the one-at-a-time relinks leave them. Every thread of the block calls it (two barriers).
__device__ void grouped_relink(const SimView& v, const int* cm, const int* co, const int* cn, int nch, int tid, int nt) {
    for (int c = tid; c < nch; c += nt) {
        const int oc = co[c];
        bool first = true;
        for (int e = 0; e < c && first; e++) first = co[e] != oc;
        if (!first) continue;
        for (int e = c; e < nch; e++) {
            if (co[e] != oc) continue;
            const int m = cm[e], pr = v.prev[m], nx = v.bead[m].next;
            if (pr >= 0) v.bead[pr].next = nx; else v.head[oc] = nx;
            if (nx >= 0) v.prev[nx] = pr;
            if (pr < 0 && nx < 0) occ_bit(v, oc, false);
        }
    }
    __syncthreads();
    for (int c = tid; c < nch; c += nt) {
        const int ncl = cn[c];
        bool first = true;
        for (int e = 0; e < c && first; e++) first = cn[e] != ncl;
        if (!first) continue;
        for (int e = c; e < nch; e++) {
            if (cn[e] != ncl) continue;
            const int m = cm[e], hd = v.head[ncl];
            v.bead[m].next = hd;
            v.prev[m] = -1;
            if (hd >= 0) v.prev[hd] = m;
            v.head[ncl] = m;
        }
        occ_bit(v, ncl, true);
    }
    __syncthreads();
}

// ======================================================================================
// Cell list: per fine cell a singly linked list through Bead::next plus prev[] for O(1)
// removal. Built in canonical order (ascending bead id within a cell) so runs repeat.
// use_flag 0: always rebuilt; 1: after an accepted plane wave moved the beads; 2: before an
// active plane-wave move if the shared-memory serial phase left the lists stale; 3 + l: before
// the global-memory serial phase of layer l if they are stale.
// ======================================================================================
__device__ __forceinline__ bool cl_skip(const SimView& v, int use_flag) {
    if (use_flag == 1) return !*v.pw_rebuild;
    if (use_flag == 2) return !(v.pw->active && !v.pw->null_move && *v.cl_stale);
    if (use_flag >= 3) return !(*v.cl_stale && !((v.smem_layers >> (use_flag - 3)) & 1));
    return false;
}
__global__ void k_cl_clear(const SimView* __restrict__ vs, int use_flag) {
    SIM_EXIT_IF(cl_skip(gv, use_flag))
    SIM_PROLOGUE
    if (v.occ && use_flag != 0) {
        // lists and bits agree since the last full rebuild: empty only the occupied cells
        const int64_t nw = (int64_t)v.Gf * v.Gf * v.occ_w;
        for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < nw; w += (int64_t)gridDim.x * blockDim.x) {
            const uint32_t bits0 = v.occ[w];
            if (!bits0) continue;
            const int64_t base = (w % v.occ_w) * 32 + (int64_t)v.Gf * (w / v.occ_w);
            for (uint32_t bits = bits0; bits; bits &= bits - 1u) v.head[base + __ffs(bits) - 1] = -1;
            v.occ[w] = 0u;
        }
        return;
    }
    // full rebuild (creation, new positions or state): every cell and every bit
    int64_t nc = (int64_t)v.Gf * v.Gf * v.Gf;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nc; c += (int64_t)gridDim.x * blockDim.x)
        v.head[c] = -1;
    if (v.occ) {
        const int64_t nw = (int64_t)v.Gf * v.Gf * v.occ_w;
        for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < nw; w += (int64_t)gridDim.x * blockDim.x)
            v.occ[w] = 0u;
    }
}
__global__ void k_cl_insert(const SimView* __restrict__ vs, int use_flag) {
    SIM_EXIT_IF(cl_skip(gv, use_flag))
    SIM_PROLOGUE
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < v.N; i += (int64_t)gridDim.x * blockDim.x) {
        Bead b = v.bead[i];
        if (!(b.x >= 0.0 && b.x < v.L && b.y >= 0.0 && b.y < v.L && b.z >= 0.0 && b.z < v.L)) set_err(v, E_NONFINITE);
        int c = cell_lin(v, b.x, b.y, b.z);
        int old = atomicExch(&v.head[c], (int)i);
        v.bead[i].next = old;
        if (old < 0) occ_bit(v, c, true);
    }
}
// put the list of fine cell c in ascending bead-id order and set prev[]
__device__ void canon_cell(const SimView& v, int64_t c) {
    int ids[32];
    int n = 0, p = v.head[c];
    bool small = true;
    while (p >= 0) {
        if (n < 32) ids[n] = p;
        n++;
        if (n > 32) small = false;
        if (n > kMaxWalk) { set_err(v, E_WALK); break; }
        p = v.bead[p].next;
    }
    if (n == 0) return;
    if (small) {
        for (int a = 1; a < n; a++) {      // insertion sort by bead id
            int x = ids[a], b = a - 1;
            while (b >= 0 && ids[b] > x) { ids[b + 1] = ids[b]; b--; }
            ids[b + 1] = x;
        }
        v.head[c] = ids[0];
        for (int a = 0; a < n; a++) {
            v.bead[ids[a]].next = (a + 1 < n) ? ids[a + 1] : -1;
            v.prev[ids[a]] = (a > 0) ? ids[a - 1] : -1;
        }
    } else {
        int pr = -1;
        for (int q = v.head[c]; q >= 0; q = v.bead[q].next) { v.prev[q] = pr; pr = q; }
    }
}
__global__ void k_cl_canon(const SimView* __restrict__ vs, int use_flag) {
    SIM_EXIT_IF(cl_skip(gv, use_flag))
    SIM_PROLOGUE
    if (v.occ) {
        // only the occupied cells (the bits were set by the insert pass just before)
        const int64_t nw = (int64_t)v.Gf * v.Gf * v.occ_w;
        for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < nw; w += (int64_t)gridDim.x * blockDim.x) {
            const int64_t yz = w / v.occ_w;
            const int xb = (int)(w % v.occ_w) << 5;
            for (uint32_t bits = v.occ[w]; bits; bits &= bits - 1u)
                canon_cell(v, (int64_t)(xb + __ffs(bits) - 1) + (int64_t)v.Gf * yz);
        }
        return;
    }
    int64_t nc = (int64_t)v.Gf * v.Gf * v.Gf;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nc; c += (int64_t)gridDim.x * blockDim.x)
        canon_cell(v, c);
}
// blocks per simulation for a grid-stride kernel: what the largest simulation needs, but no
// more than keeps about 8k blocks over the whole group
static unsigned gx(int64_t needed_blocks, int S) {
    const int64_t cap = std::max<int64_t>(1, 8192 / std::max(S, 1));
    return (unsigned)std::max<int64_t>(1, std::min(needed_blocks, cap));
}
void launch_cl_rebuild(const SimView* d, const GroupDims& g, cudaStream_t s, int use_flag) {
    const dim3 bc(gx((g.maxCells + 255) / 256, g.S), g.S);
    const dim3 bb(gx((g.maxN + 255) / 256, g.S), g.S);
    k_cl_clear<<<bc, 256, 0, s>>>(d, use_flag);
    k_cl_insert<<<bb, 256, 0, s>>>(d, use_flag);
    k_cl_canon<<<bc, 256, 0, s>>>(d, use_flag);
}

// Slot counts of the sweep about to run, from the counter stream: floor(x) plus one more
// with probability frac(x), per layer and for the plane waves.
__global__ void k_counts(const SimView* __restrict__ vs) {
    SIM_PROLOGUE
    if (threadIdx.x != 0) return;
    const uint64_t sw = v.step[0];
    for (int l = 0; l < v.nL; l++) {
        const u4 w = draw(v.k0, v.k1, K_COUNT, l, sw, 0u, 0u);
        const double x = v.layer[l].expect, f = floor(x);
        v.counts[l] = (int)f + ((u53(w.x, w.y) < x - f) ? 1 : 0);
    }
    int mf = 0;
    if (v.pw_on) {
        const u4 w = draw(v.k0, v.k1, K_PWCOUNT, 0, sw, 0u, 0u);
        const double x = v.expect_F, f = floor(x);
        mf = (int)f + ((u53(w.x, w.y) < x - f) ? 1 : 0);
    }
    v.counts[kMaxLayers] = mf;
}
__global__ void k_advance(const SimView* __restrict__ vs, int which) {
    SIM_PROLOGUE
    if (threadIdx.x == 0) v.step[which] += 1;
}
void launch_counts(const SimView* d, const GroupDims& g, cudaStream_t s) {
    k_counts<<<dim3(1, g.S), 32, 0, s>>>(d);
}
void launch_advance(const SimView* d, const GroupDims& g, int which, cudaStream_t s) {
    k_advance<<<dim3(1, g.S), 32, 0, s>>>(d, which);
}

// ======================================================================================
// Slots of a layer: scale in the band (Eq. 32 restricted to [lo, hi), inverse transform of
// Appendix D) and the picked bead; then bucketing by coarse cell in colour-major order.
// ======================================================================================
__global__ void k_slots(const SimView* __restrict__ vs, int l) {
    SIM_EXIT_IF(l >= gv.nL || (int)(blockIdx.x * blockDim.x) >= gv.counts[l])
    SIM_PROLOGUE
    if (l >= v.nL) return;
    const int M = v.counts[l];
    const uint64_t sweep = v.step[0];
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= M) return;
    const LayerDev& Ly = v.layer[l];
    u4 w = draw(v.k0, v.k1, K_SLOT, l, sweep, (uint32_t)j, 0);
    double u = u53(w.x, w.y);
    double wv = sub(Ly.ilo3, mul(u, sub(Ly.ilo3, Ly.ihi3)));
    v.slot_lam[j] = inv_cbrt_band(wv, Ly.lo);
    v.slot_bead[j] = (int)pick(w.z, w.w, v.N);
    v.tr_out[Ly.tr_off + j] = 0;
    v.tr_n[Ly.tr_off + j] = 0;
    v.tr_du[Ly.tr_off + j] = 0.0;
    // the rest of the slot's draws, whichever phase runs it: centre offset V in the unit ball
    // (or the centre itself, uniform in the box), unit polarisation p by rejection (Appendix D),
    // and the acceptance threshold (Eq. 20); one slot per thread, so full warps share the
    // binary64 work
    double V[3] = {0.0, 0.0, 0.0}, p[3] = {0.0, 0.0, 1.0};
    for (uint32_t a = 0; a < 64; a++) {
        const u4 wb = draw(v.k0, v.k1, K_VB, l, sweep, (uint32_t)j, a);
        const double x = sym(wb.x), y = sym(wb.y), z = sym(wb.z);
        if (norm2(x, y, z) <= 1.0) { V[0] = x; V[1] = y; V[2] = z; break; }
    }
    for (uint32_t a = 0; a < 64; a++) {
        const u4 wp = draw(v.k0, v.k1, K_VP, l, sweep, (uint32_t)j, a);
        const double x = sym(wp.x), y = sym(wp.y), z = sym(wp.z), q = norm2(x, y, z);
        if (q <= 1.0 && q > 0.0) { p[0] = x; p[1] = y; p[2] = z; break; }
    }
    const double r = sqr_t(norm2(p[0], p[1], p[2]));
    if (v.centring == 1) uniform_centre(v, l, sweep, (uint32_t)j, V);   // slot_V holds the centre itself
    for (int a = 0; a < 3; a++) {
        v.slot_V[3 * j + a] = V[a];
        v.slot_p[3 * j + a] = dvd(p[a], r);
    }
    const u4 wa = draw(v.k0, v.k1, K_ACC, l, sweep, (uint32_t)j, 0);
    v.slot_thr[j] = accept_threshold(v, wa);
}
void launch_slots(const SimView* d, const GroupDims& g, int l, cudaStream_t s) {
    k_slots<<<dim3((g.Mmax[l] + 255) / 256, g.S), 256, 0, s>>>(d, l);
}

// The layer record of schedule index l: layer l itself, or (l >= kLevel2) the second colouring
// of layer l - kLevel2, with its grid and carries in place of the layer's own.
__device__ __forceinline__ LayerDev sched_layer(const SimView& v, int l) {
    if (l < kLevel2) return v.layer[l];
    LayerDev y = v.layer[l - kLevel2];
    y.G = y.G2;
    y.invG = y.invG2;
    y.carry_off = y.carry_off2;
    return y;
}
__device__ __forceinline__ bool sched_on(const SimView& v, int l) {
    return layer_real(l) < v.nL && (l < kLevel2 ? v.layer[l].G : v.layer[l - kLevel2].G2) > 0;
}
// slots a schedule index buckets: the layer's slots, or the ones its first colouring deferred
__device__ __forceinline__ int sched_count(const SimView& v, int l) { return l < kLevel2 ? v.counts[l] : *v.serial_count; }
// largest support a concurrent move of the index takes
__device__ __forceinline__ int sched_ncap(const SimView& v, int l) { return l < kLevel2 ? v.n_cap : kNCapMax; }

// The slots of schedule index l by coarse cell (of the picked bead now, or of the centre):
// entry t is slot t of the layer, or for a second colouring the t-th slot its first deferred.
__global__ void k_bucket_count(const SimView* __restrict__ vs, int l) {
    SIM_EXIT_IF(!sched_on(gv, l) || (int)(blockIdx.x * blockDim.x) >= sched_count(gv, l))
    SIM_PROLOGUE
    if (!sched_on(v, l)) return;
    const int M = sched_count(v, l);
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= M) return;
    const int j = l < kLevel2 ? t : v.serial_list[t];
    const LayerDev Ly = sched_layer(v, l);
    const int G = Ly.G, K = v.K, Q = G / K;
    double xs[3];
    if (v.centring == 1) uniform_centre(v, layer_real(l), v.step[0], (uint32_t)j, xs);      // bucket by the centre
    else {
        const Bead b = v.bead[v.slot_bead[j]];
        xs[0] = b.x; xs[1] = b.y; xs[2] = b.z;
    }
    int c[3];
    for (int a = 0; a < 3; a++) {
        double f = floor(mul(xs[a], Ly.invG));
        int ci = (int)f;
        if (f < 0.0) ci = 0;
        if (ci >= G) ci = G - 1;
        c[a] = ci;
    }
    int colour = (c[0] % K) + K * ((c[1] % K) + K * (c[2] % K));
    int q = (c[0] / K) + Q * ((c[1] / K) + Q * (c[2] / K));
    int key = colour * Q * Q * Q + q;
    v.slot_key[t] = key;
    atomicAdd(&v.q_count[key], 1);
}
// Exclusive prefix of one value per thread over a block of 1,024 threads (32 warps): a shuffle
// scan per warp, the warp totals scanned by warp 0; two block barriers. *total receives the sum.
__device__ __forceinline__ int block_excl_scan(int x, int* s_w, int* total) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int incl = x;
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(FULL, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) s_w[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        const int c = s_w[lane];
        int ci = c;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(FULL, ci, o);
            if (lane >= o) ci += y;
        }
        s_w[lane] = ci - c;
        if (lane == 31) s_w[32] = ci;
    }
    __syncthreads();
    *total = s_w[32];
    return s_w[wid] + incl - x;
}
constexpr int kScanPer = 8;   // consecutive entries per thread in the single-block scans

// exclusive scan of n ints by one block of 1,024 threads per simulation: mode 0 = bucket counts
// of layer l (G^3 keys), mode 1 = region counts of layer l (Q^3 queues); each thread takes
// kScanPer consecutive entries of a chunk. With heavy_lo >= 0 (mode 1) it also lists the queues
// of the colour phase that have slots and more than heavy_lo beads in their region, in no
// particular order: those with at most heavy_mid beads from the front of hq_list, the others
// from its back, and resets the two lists' work counters.
__global__ void k_scan(const SimView* __restrict__ vs, int mode, int l, int colour, int heavy_lo, int heavy_mid) {
    SIM_EXIT_IF(!sched_on(gv, l))
    SIM_PROLOGUE
    if (!sched_on(v, l)) return;
    const int G = sched_layer(v, l).G, Q = G / v.K;
    const int n = mode == 0 ? G * G * G : Q * Q * Q;
    const int* in = mode == 0 ? v.q_count : v.rcount;
    int* out = mode == 0 ? v.q_start : v.rstart;
    __shared__ int s_w[33];
    int carry = 0;
    for (int base = 0; base < n; base += kScanPer * 1024) {
        const int i0 = base + kScanPer * (int)threadIdx.x;
        int x[kScanPer], sum = 0;
#pragma unroll
        for (int u = 0; u < kScanPer; u++) { x[u] = i0 + u < n ? in[i0 + u] : 0; sum += x[u]; }
        int total;
        int pre = carry + block_excl_scan(sum, s_w, &total);
#pragma unroll
        for (int u = 0; u < kScanPer; u++) {
            if (i0 + u < n) out[i0 + u] = pre;
            pre += x[u];
        }
        carry += total;
        __syncthreads();                          // s_w is rewritten by the next chunk
    }
    if (mode == 1 && heavy_lo >= 0) {
        __shared__ int hc[2];
        if (threadIdx.x < 2) hc[threadIdx.x] = 0;
        __syncthreads();
        for (int q = threadIdx.x; q < n; q += blockDim.x)
            if (in[q] > heavy_lo && v.q_count[colour * n + q] > 0) {
                if (in[q] <= heavy_mid) v.hq_list[atomicAdd(&hc[0], 1)] = q;
                else v.hq_list[n - 1 - atomicAdd(&hc[1], 1)] = q;
            }
        __syncthreads();
        if (threadIdx.x == 0) { v.hq_ctl[0] = hc[0]; v.hq_ctl[1] = 0; v.hq_ctl[2] = hc[1]; v.hq_ctl[3] = 0; }
    }
}
// zero the per-phase counters: mode 0 = bucket counts, fills and deferral flags of layer l,
// mode 1 = region counts and fills
__global__ void k_zero(const SimView* __restrict__ vs, int mode, int l) {
    SIM_EXIT_IF(!sched_on(gv, l))
    SIM_PROLOGUE
    if (!sched_on(v, l)) return;
    const int G = sched_layer(v, l).G, Q = G / v.K;
    const int n = mode == 0 ? G * G * G : Q * Q * Q;
    int* a = mode == 0 ? v.q_count : v.rcount;
    int* b = mode == 0 ? v.q_fill : v.rfill;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) { a[i] = 0; b[i] = 0; }
    if (mode == 0) {
        const int M = v.layer[layer_real(l)].Mmax;
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < M; i += gridDim.x * blockDim.x) v.defer[i] = 0;
    }
}
__global__ void k_bucket_scatter(const SimView* __restrict__ vs, int l) {
    SIM_EXIT_IF(!sched_on(gv, l) || (int)(blockIdx.x * blockDim.x) >= sched_count(gv, l))
    SIM_PROLOGUE
    if (!sched_on(v, l)) return;
    const int M = sched_count(v, l);
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= M) return;
    int key = v.slot_key[t];
    int pos = v.q_start[key] + atomicAdd(&v.q_fill[key], 1);
    v.q_slots[pos] = t;
}
// slots of one queue in ascending slot id (the order of the sequential schedule); a second
// colouring sorts its entries in first-schedule order and then names their slots
__global__ void k_bucket_sort(const SimView* __restrict__ vs, int l) {
    SIM_EXIT_IF(!sched_on(gv, l))
    SIM_PROLOGUE
    if (!sched_on(v, l)) return;
    const int G = sched_layer(v, l).G, nkeys = G * G * G;
    int key = blockIdx.x * blockDim.x + threadIdx.x;
    if (key >= nkeys) return;
    int s = v.q_start[key], n = v.q_count[key];
    int* a = v.q_slots + s;
    for (int i = 1; i < n; i++) {
        int x = a[i], b = i - 1;
        while (b >= 0 && a[b] > x) { a[b + 1] = a[b]; b--; }
        a[b + 1] = x;
    }
    if (l >= kLevel2)
        for (int i = 0; i < n; i++) a[i] = v.serial_list[a[i]];
}
void launch_bucket(const SimView* d, const GroupDims& g, int l, cudaStream_t s) {
    const int keys = g.keys[l], M = g.Mmax[l];
    k_zero<<<dim3(gx((std::max(keys, M) + 255) / 256, g.S), g.S), 256, 0, s>>>(d, 0, l);
    k_bucket_count<<<dim3((M + 255) / 256, g.S), 256, 0, s>>>(d, l);
    k_scan<<<dim3(1, g.S), 1024, 0, s>>>(d, 0, l, 0, -1, 0);
    k_bucket_scatter<<<dim3((M + 255) / 256, g.S), 256, 0, s>>>(d, l);
    k_bucket_sort<<<dim3((keys + 127) / 128, g.S), 128, 0, s>>>(d, l);
}

// deferred slots in schedule order -> serial list
__global__ void k_defer_compact(const SimView* __restrict__ vs, int l) {
    SIM_EXIT_IF(!sched_on(gv, l))
    SIM_PROLOGUE
    if (!sched_on(v, l)) return;
    // (a second colouring's entries are the first one's deferred slots: read before the barriers
    // below, ahead of the new count written at the end)
    const int M = sched_count(v, l);
    // the deferred slots in schedule order: each thread takes kScanPer consecutive entries of a
    // chunk, a block prefix of the per-thread counts places them; chunks without a deferred slot
    // (nearly all) cost one block vote
    __shared__ int s_w[33];
    int carry = 0;
    for (int base = 0; base < M; base += kScanPer * 1024) {
        const int i0 = base + kScanPer * (int)threadIdx.x;
        unsigned f = 0u;
#pragma unroll
        for (int u = 0; u < kScanPer; u++)
            if (i0 + u < M && v.defer[i0 + u]) f |= 1u << u;
        if (!__syncthreads_or(f != 0u)) continue;
        int total;
        int pos = carry + block_excl_scan(__popc(f), s_w, &total);
        for (; f; f &= f - 1u) v.serial_list[pos++] = v.q_slots[i0 + __ffs(f) - 1];
        carry += total;
        __syncthreads();                          // s_w is rewritten by the next chunk
    }
    if (threadIdx.x == 0) *v.serial_count = carry;
}
void launch_defer_compact(const SimView* d, const GroupDims& g, int l, cudaStream_t s) {
    k_defer_compact<<<dim3(1, g.S), 1024, 0, s>>>(d, l);
}

}  // namespace wmcd

namespace wmcd {

// ======================================================================================
// Concurrent wavelet moves: one warp per queue (coarse cell) of one colour.
// ======================================================================================
struct WarpSmem {
    int ids[kNCapMax];          // support, in gather order
    double d[kNCapMax][4];      // exact minimum-image offset from the centre, and its square
    double op[kNCapMax][3];     // old positions
    double np[kNCapMax][3];     // new (wrapped) positions
    double nu[kNCapMax][3];     // new unwrapped positions (old + delta)
    int dimg[kNCapMax];         // packed image change
    int sid[kNCapMax];          // support ids ascending
    int cpre[kNCapMax + 1];     // prefix of partner-search columns per member
    int cbox[kNCapMax][6];      // partner-search box per member: first cell c0[3], cells nc[3]
};

__device__ __forceinline__ double warp_sum(double x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}
__device__ __forceinline__ int warp_sum_i(int x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}
__device__ __forceinline__ bool sorted_has(const int* a, int n, int x) {
    int lo = 0, hi = n - 1;
    while (lo <= hi) {
        int m = (lo + hi) >> 1;
        if (a[m] == x) return true;
        if (a[m] < x) lo = m + 1; else hi = m - 1;
    }
    return false;
}

// Uniform point of the unit ball by rejection (Appendix D): attempt a uses counter attempt a;
// the warp tries 32 attempts at once and takes the first accepted one, which is what a
// sequential loop over the attempts would return.
__device__ void warp_ball_point(const SimView& v, uint32_t kind, int l, uint64_t sweep, uint32_t j, bool nonzero,
                                int lane, double V[3]) {
    for (int base = 0; base < 64; base += 32) {
        u4 w = draw(v.k0, v.k1, kind, l, sweep, j, (uint32_t)(base + lane));
        double x = sym(w.x), y = sym(w.y), z = sym(w.z);
        double q = norm2(x, y, z);
        unsigned ok = __ballot_sync(0xffffffffu, q <= 1.0 && (!nonzero || q > 0.0));
        if (ok) {
            int src = __ffs(ok) - 1;
            V[0] = __shfl_sync(0xffffffffu, x, src);
            V[1] = __shfl_sync(0xffffffffu, y, src);
            V[2] = __shfl_sync(0xffffffffu, z, src);
            return;
        }
    }
    V[0] = 0.0; V[1] = 0.0; V[2] = nonzero ? 1.0 : 0.0;
}

// cell box [floor((lo) invf), floor((hi) invf)] per axis, at most Gf cells
__device__ __forceinline__ void cell_box(const SimView& v, const double lo[3], const double hi[3], int c0[3], int nc[3]) {
    for (int a = 0; a < 3; a++) {
        int t0 = (int)floor(mul(lo[a], v.invf));
        int t1 = (int)floor(mul(hi[a], v.invf));
        c0[a] = t0;
        nc[a] = min(t1 - t0 + 1, v.Gf);
    }
}
__device__ __forceinline__ int box_cell(const SimView& v, const int c0[3], const int nc[3], int k) {
    int kx = k % nc[0], ky = (k / nc[0]) % nc[1], kz = k / (nc[0] * nc[1]);
    return wrapi(c0[0] + kx, v.Gf) + v.Gf * (wrapi(c0[1] + ky, v.Gf) + v.Gf * wrapi(c0[2] + kz, v.Gf));
}

// cell index modulo G: one add or subtract in the common case, a remainder otherwise
__device__ __forceinline__ int wrapc(int c, int G) {
    if (c < 0) c += G;
    else if (c >= G) c -= G;
    if ((unsigned)c >= (unsigned)G) { c %= G; if (c < 0) c += G; }
    return c;
}

// difference a - b of two wrapped coordinates in binary32, minimum image applied
__device__ __forceinline__ float dif32(double a, double b, double L, float hLf) {
    const double d = sub(a, b);
    float f = (float)d;
    if (fabsf(f) > hLf) f = (float)(d > 0.0 ? sub(d, L) : add(d, L));
    return f;
}
__device__ __forceinline__ float norm2f(float x, float y, float z) { return x * x + y * y + z * z; }

// binary32 pair energies with a magnitude m such that |error| <= 64 u m  (u = 2^-24)
struct Pot32 {
    float sig2, eps, rc2, bk, br0, br02, R02, kappa, hL;
    int bond;
};
__device__ __forceinline__ Pot32 pot32(const Pot& P) {
    Pot32 q;
    q.sig2 = (float)P.sig2; q.eps = (float)P.eps; q.rc2 = (float)P.rc2; q.bk = (float)P.bk; q.br0 = (float)P.br0;
    q.br02 = q.br0 * q.br0; q.R02 = (float)P.R02; q.kappa = (float)P.kappa; q.hL = (float)P.halfL; q.bond = P.bond;
    return q;
}
__device__ __forceinline__ void wca32(const Pot32& P, float r2, float& u, float& m) {
    if (P.eps == 0.0f || !(r2 < P.rc2)) { u = 0.0f; m = 0.0f; return; }
    const float s2 = __fdiv_rn(P.sig2, r2), s6 = s2 * s2 * s2, s12 = s6 * s6;
    u = 4.0f * P.eps * (s12 - s6) + P.eps;
    m = 4.0f * P.eps * (s12 + s6) + P.eps;
}
__device__ __forceinline__ void bond32(const Pot32& P, float r2, float& u, float& m) {
    if (P.bond == 1) {
        // |error| <= 5 ulp * k (|d| r + d^2): r2 carries ~7 ulp, sqrt halves it, one more for
        // the subtraction and two for the products (scaled by 80 ulp in the band: ample)
        const float r = __fsqrt_rn(r2), d = r - P.br0;
        u = 0.5f * P.bk * d * d;
        m = P.bk * (fabsf(d) * r + d * d + 1e-6f * P.br02);
    } else if (P.bond == 2) {
        const float x = __fdiv_rn(r2, P.R02);
        if (!(x < 0.98f)) { u = 0.0f; m = __int_as_float(0x7f800000); return; }   // near R0: decide in FP64
        const float lg = log1pf(-x);
        u = -0.5f * P.bk * P.R02 * lg;
        m = 0.5f * P.bk * P.R02 * (fabsf(lg) + 8.0f * x / (1.0f - x) + 1.0f);
    } else {
        u = 0.0f; m = 0.0f;
    }
}

// Partner-search boxes of the support: [min(old, new) - rc, max(old, new) + rc] per member;
// columns (x, y) are spread over lanes, z is looped. Returns the column count and max z extent.
__device__ void partner_boxes(const SimView& v, WarpSmem& sm, int n, int lane, int* ncols, int* nzmax) {
    int nz = 0;
    for (int k = lane; k < n; k += 32) {
        int c0[3], nc[3];
        for (int a = 0; a < 3; a++) {
            const double o = sm.op[k][a], u = sm.nu[k][a];
            c0[a] = (int)floor(mul(sub(fmin(o, u), v.rc + 1e-9), v.invf));
            const int t1 = (int)floor(mul(add(fmax(o, u), v.rc + 1e-9), v.invf));
            nc[a] = min(t1 - c0[a] + 1, v.Gf);
        }
        for (int a = 0; a < 3; a++) { sm.cbox[k][a] = c0[a]; sm.cbox[k][3 + a] = nc[a]; }
        sm.cpre[k + 1] = nc[0] * nc[1];
        nz = max(nz, nc[2]);
    }
    __syncwarp();
    if (lane == 0) { sm.cpre[0] = 0; for (int k = 0; k < n; k++) sm.cpre[k + 1] += sm.cpre[k]; }
    for (int o = 16; o > 0; o >>= 1) nz = max(nz, __shfl_xor_sync(0xffffffffu, nz, o));
    __syncwarp();
    *ncols = sm.cpre[n];
    *nzmax = nz;
}

// Energy change of the move (Eqs. 1, 2; external well): support-support pairs, bonds to beads
// outside the support, WCA to beads outside the support (cell lists). F32: binary32 terms,
// returns the sum, the magnitude sum and the term count; otherwise binary64.
template <bool F32>
__device__ void energy(const SimView& v, WarpSmem& sm, int n, int lane, int ncols, int nzmax, double* dU64,
                       float* dU32, float* mag32, int* terms, int* pe_out) {
    const double L = v.L, hL = v.halfL;
    const Pot& P = v.pot;
    const Pot32 P32 = pot32(P);
    const float hLf = (float)hL;
    double a64 = 0.0;
    float a32 = 0.0f, m32 = 0.0f;
    int T = 0, pe = 0;
    // external well and bonds to partners outside the support
    for (int k = lane; k < n; k += 32) {
        if (P.kappa != 0.0) {
            if (F32) {
                float x = dif32(sm.np[k][0], hL, L, hLf), y = dif32(sm.np[k][1], hL, L, hLf), z = dif32(sm.np[k][2], hL, L, hLf);
                float un = 0.5f * P32.kappa * norm2f(x, y, z);
                x = dif32(sm.op[k][0], hL, L, hLf); y = dif32(sm.op[k][1], hL, L, hLf); z = dif32(sm.op[k][2], hL, L, hLf);
                float uo = 0.5f * P32.kappa * norm2f(x, y, z);
                a32 += un - uo; m32 += un + uo; T += 2;
            } else {
                a64 += U_ext(P, sm.np[k][0], sm.np[k][1], sm.np[k][2]) - U_ext(P, sm.op[k][0], sm.op[k][1], sm.op[k][2]);
            }
        }
        const int m = sm.ids[k];
        for (int e = 0; e < 2; e++) {
            const int q = e ? m + 1 : m - 1;
            if (q < 0 || q >= v.N || !(e ? v.bnext[m] : v.bnext[q]) || sorted_has(sm.sid, n, q)) continue;
            const Bead bq = v.bead[q];
            if (F32) {
                float r2n = norm2f(dif32(sm.np[k][0], bq.x, L, hLf), dif32(sm.np[k][1], bq.y, L, hLf), dif32(sm.np[k][2], bq.z, L, hLf));
                float r2o = norm2f(dif32(sm.op[k][0], bq.x, L, hLf), dif32(sm.op[k][1], bq.y, L, hLf), dif32(sm.op[k][2], bq.z, L, hLf));
                float un, mn, uo, mo;
                bond32(P32, r2n, un, mn);
                bond32(P32, r2o, uo, mo);
                a32 += un - uo; m32 += mn + mo; T += 2;
            } else {
                double r2n = norm2(mi(sm.np[k][0] - bq.x, L, hL), mi(sm.np[k][1] - bq.y, L, hL), mi(sm.np[k][2] - bq.z, L, hL));
                double r2o = norm2(mi(sm.op[k][0] - bq.x, L, hL), mi(sm.op[k][1] - bq.y, L, hL), mi(sm.op[k][2] - bq.z, L, hL));
                a64 += U_bond(P, r2n) - U_bond(P, r2o);
            }
        }
    }
    // pairs inside the support
    const int npairs = n * (n - 1) / 2;
    for (int t = lane; t < npairs; t += 32) {
        int a = (int)((sqrtf(8.0f * t + 1.0f) - 1.0f) * 0.5f);
        while (a * (a + 1) / 2 > t) a--;
        while ((a + 1) * (a + 2) / 2 <= t) a++;
        const int k1 = t - a * (a + 1) / 2, k2 = a + 1;
        const int m1 = sm.ids[k1], m2 = sm.ids[k2];
        const int lo_ = min(m1, m2), hi_ = max(m1, m2);
        const bool bonded = hi_ == lo_ + 1 && v.bnext[lo_];
        if (F32) {
            float r2n = norm2f(dif32(sm.np[k1][0], sm.np[k2][0], L, hLf), dif32(sm.np[k1][1], sm.np[k2][1], L, hLf),
                               dif32(sm.np[k1][2], sm.np[k2][2], L, hLf));
            float r2o = norm2f(dif32(sm.op[k1][0], sm.op[k2][0], L, hLf), dif32(sm.op[k1][1], sm.op[k2][1], L, hLf),
                               dif32(sm.op[k1][2], sm.op[k2][2], L, hLf));
            float un, mn, uo, mo;
            wca32(P32, r2n, un, mn);
            wca32(P32, r2o, uo, mo);
            a32 += un - uo; m32 += mn + mo; T += 2;
            if (bonded) { bond32(P32, r2n, un, mn); bond32(P32, r2o, uo, mo); a32 += un - uo; m32 += mn + mo; T += 2; }
        } else {
            double r2n = norm2(mi(sm.np[k1][0] - sm.np[k2][0], L, hL), mi(sm.np[k1][1] - sm.np[k2][1], L, hL),
                               mi(sm.np[k1][2] - sm.np[k2][2], L, hL));
            double r2o = norm2(mi(sm.op[k1][0] - sm.op[k2][0], L, hL), mi(sm.op[k1][1] - sm.op[k2][1], L, hL),
                               mi(sm.op[k1][2] - sm.op[k2][2], L, hL));
            double u = U_wca(P, r2n) - U_wca(P, r2o);
            if (bonded) u += U_bond(P, r2n) - U_bond(P, r2o);
            a64 += u;
        }
    }
    // WCA with beads outside the support, through the cell lists
    if (P.eps != 0.0) {
        const int Gf = v.Gf;
        for (int base = 0; base < ncols; base += 32) {
            const int w = base + lane;
            int k = 0, cx = 0, cy = 0, c0z = 0, nz = 0;
            const bool valid = w < ncols;
            if (valid) {
                while (sm.cpre[k + 1] <= w) k++;
                const int col = w - sm.cpre[k], nx = sm.cbox[k][3];
                cx = wrapc(sm.cbox[k][0] + col % nx, Gf);
                cy = wrapc(sm.cbox[k][1] + col / nx, Gf);
                c0z = sm.cbox[k][2];
                nz = sm.cbox[k][5];
            }
            const int m = sm.ids[k];
            const int colbase = cx + Gf * cy;
            for (int kz = 0; kz < nzmax; kz++) {
                int q = (valid && kz < nz) ? v.head[colbase + Gf * Gf * wrapc(c0z + kz, Gf)] : -1;
                int guard = 0;
                while (q >= 0) {
                    const Bead bq = v.bead[q];
                    if (q != m && !sorted_has(sm.sid, n, q)) {
                        if (F32) {
                            float r2n = norm2f(dif32(sm.np[k][0], bq.x, L, hLf), dif32(sm.np[k][1], bq.y, L, hLf),
                                               dif32(sm.np[k][2], bq.z, L, hLf));
                            float r2o = norm2f(dif32(sm.op[k][0], bq.x, L, hLf), dif32(sm.op[k][1], bq.y, L, hLf),
                                               dif32(sm.op[k][2], bq.z, L, hLf));
                            if (r2n < P32.rc2 || r2o < P32.rc2) {
                                float un, mn, uo, mo;
                                wca32(P32, r2n, un, mn);
                                wca32(P32, r2o, uo, mo);
                                a32 += un - uo; m32 += mn + mo; T += 2; pe++;
                            }
                        } else {
                            double r2n = norm2(mi(sm.np[k][0] - bq.x, L, hL), mi(sm.np[k][1] - bq.y, L, hL),
                                               mi(sm.np[k][2] - bq.z, L, hL));
                            double r2o = norm2(mi(sm.op[k][0] - bq.x, L, hL), mi(sm.op[k][1] - bq.y, L, hL),
                                               mi(sm.op[k][2] - bq.z, L, hL));
                            if (r2n < P.rc2 || r2o < P.rc2) { a64 += U_wca(P, r2n) - U_wca(P, r2o); pe++; }
                        }
                    }
                    q = bq.next;
                    if (++guard > kMaxWalk) { set_err(v, E_WALK); break; }
                }
            }
        }
    }
    // lane 0's sums for every lane (a butterfly leaves lanes with differently rounded totals)
    const unsigned FULL = 0xffffffffu;
    if (F32) {
        float s = a32, mm = m32;
        int tt = T;
        for (int o = 16; o > 0; o >>= 1) {
            s += __shfl_xor_sync(FULL, s, o);
            mm += __shfl_xor_sync(FULL, mm, o);
            tt = max(tt, __shfl_xor_sync(FULL, tt, o));
        }
        *dU32 = __shfl_sync(FULL, s, 0);
        *mag32 = __shfl_sync(FULL, mm, 0);
        *terms = __shfl_sync(FULL, tt, 0) + 5;   // summation depth: one lane's terms, then the butterfly
    } else {
        *dU64 = __shfl_sync(FULL, warp_sum(a64), 0);
    }
    *pe_out = warp_sum_i(pe);
}

template <int PREC>
__device__ int warp_attempt(const SimView& v, WarpSmem& sm, int ls, int j, int i, double lam, uint64_t sweep,
                            const int64_t rlo[3], const int64_t rhi[3], int lane, int* n_out, int* pe_out,
                            int* recheck_out, double* du_out) {
    const unsigned FULL = 0xffffffffu;
    const int l = layer_real(ls), ncap = sched_ncap(v, ls);   // draws are the layer's own
    const double L = v.L, hL = v.halfL;
    const float hLf = (float)hL;
    *du_out = 0.0;
    const int Gf = v.Gf;
    // centre b = r_i + lam V (Appendix D), wrapped into the box; or uniform in the box
    double V[3], b[3];
    if (v.centring == 1) uniform_centre(v, l, sweep, (uint32_t)j, b);
    else {
        const double ri[3] = {v.bead[i].x, v.bead[i].y, v.bead[i].z};
        warp_ball_point(v, K_VB, l, sweep, (uint32_t)j, false, lane, V);
        for (int a = 0; a < 3; a++) b[a] = wrap(add(ri[a], mul(lam, V[a])), L, nullptr);
    }
    // the influence ball must lie in fine cells wholly inside the queue's region
    const double R = add(add(lam, mul(mul(0.25, v.A0), lam)), v.r_reach);
    for (int a = 0; a < 3; a++) {
        const int64_t t0 = (int64_t)floor(mul(sub(b[a], R), v.invf));
        const int64_t t1 = (int64_t)floor(mul(add(b[a], R), v.invf));
        if (!range_inside(t0, t1, rlo[a], rhi[a], Gf)) return DEFER;
    }
    // gather the support: beads strictly inside the ball (one image each, lambda <= L/2);
    // binary32 prefilter, exact binary64 test within 1e-6 of the sphere
    const double lam2 = mul(lam, lam);
    const float lam2f = (float)lam2, lin = lam2f * (1.0f - 1e-6f), lout = lam2f * (1.0f + 1e-6f);
    int c0[3], nc[3];
    for (int a = 0; a < 3; a++) {
        c0[a] = (int)floor(mul(sub(b[a], lam + 1e-9), v.invf));
        const int t1 = (int)floor(mul(add(b[a], lam + 1e-9), v.invf));
        nc[a] = min(t1 - c0[a] + 1, Gf);
    }
    int n = 0;
    // one bead per lane per step: test it, vote, append the members in vote order; a support
    // above n_cap means the move is deferred, so the walk stops there
    auto step = [&](int& ptr) {
        bool in = false;
        int nxt = -1;
        Bead bb;
        if (ptr >= 0) {
            bb = v.bead[ptr];
            nxt = bb.next;
            const float d2f = norm2f(dif32(bb.x, b[0], L, hLf), dif32(bb.y, b[1], L, hLf), dif32(bb.z, b[2], L, hLf));
            if (d2f < lin) in = true;
            else if (d2f <= lout) {
                const double e2 = norm2(mi(sub(bb.x, b[0]), L, hL), mi(sub(bb.y, b[1]), L, hL), mi(sub(bb.z, b[2]), L, hL));
                in = e2 < lam2;
            }
        }
        const unsigned msk = __ballot_sync(FULL, in);
        const int slot = n + __popc(msk & ((1u << lane) - 1u));
        if (in && slot < kNCapMax) {
            sm.ids[slot] = ptr;
            sm.op[slot][0] = bb.x; sm.op[slot][1] = bb.y; sm.op[slot][2] = bb.z;
        }
        n += __popc(msk);
        ptr = nxt;
    };
    if (v.occ) {
        // rows (y, z) of the ball's cell box over the lanes; each lane takes the occupied cells of
        // its row's x range from the occupancy words, one list at a time
        const int rows = nc[1] * nc[2], x0 = wrapi(c0[0], Gf);
        int guard = 0;
        for (int base = 0; base < rows; base += 32) {
            const int r = base + lane;
            bool live = r < rows;
            const uint32_t* row = nullptr;
            int rowcell = 0, piece = 0, a = x0, bnd = min(x0 + nc[0], Gf), wi = x0 >> 5;
            uint32_t bits = 0u;
            if (live) {
                const int y = wrapi(c0[1] + r % nc[1], Gf), z = wrapi(c0[2] + r / nc[1], Gf);
                row = v.occ + ((size_t)y + (size_t)Gf * z) * v.occ_w;
                rowcell = Gf * (y + Gf * z);
                bits = occ_masked(row[wi], a, bnd, wi);
            }
            int ptr = -1;
            while (true) {
                while (live && ptr < 0) {
                    if (bits) { ptr = v.head[rowcell + (wi << 5) + __ffs(bits) - 1]; bits &= bits - 1u; continue; }
                    if (wi < ((bnd - 1) >> 5)) { wi++; bits = occ_masked(row[wi], a, bnd, wi); continue; }
                    if (piece == 0 && x0 + nc[0] > Gf) {
                        piece = 1; a = 0; bnd = x0 + nc[0] - Gf; wi = 0;
                        bits = occ_masked(row[0], a, bnd, 0);
                        continue;
                    }
                    live = false;
                }
                if (!__any_sync(FULL, ptr >= 0)) break;
                step(ptr);
                if (n > ncap) { *n_out = n; return DEFER; }
                if (++guard > kMaxWalk) { if (lane == 0) set_err(v, E_WALK); return DEFER; }
            }
        }
    } else {
        const int nxy = nc[0] * nc[1];
        int guard = 0;
        for (int base = 0; base < nxy; base += 32) {
            const int w = base + lane;
            const bool col = w < nxy;
            const int colbase = col ? wrapc(c0[0] + w % nc[0], Gf) + Gf * wrapc(c0[1] + w / nc[0], Gf) : 0;
            for (int kz = 0; kz < nc[2]; kz++) {
                int ptr = col ? v.head[colbase + Gf * Gf * wrapc(c0[2] + kz, Gf)] : -1;
                while (__any_sync(FULL, ptr >= 0)) {
                    step(ptr);
                    if (n > ncap) { *n_out = n; return DEFER; }
                    if (++guard > kMaxWalk) { if (lane == 0) set_err(v, E_WALK); return DEFER; }
                }
            }
        }
    }
    *n_out = n;
    if (n > ncap) return DEFER;
    __syncwarp();
    if (n == 0) {                        // no bead moves: dU = 0 against the threshold
        const u4 w0 = draw(v.k0, v.k1, K_ACC, l, sweep, (uint32_t)j, 0);
        return 0.0 <= accept_threshold(v, w0) ? ACCEPT : REJECT;
    }
    // polarisation and amplitude A_w = A0 lam / sqrt(n) (Eq. 29)
    double p[3];
    warp_ball_point(v, K_VP, l, sweep, (uint32_t)j, true, lane, p);
    {
        const double r = sqr_t(norm2(p[0], p[1], p[2]));
        p[0] = dvd(p[0], r); p[1] = dvd(p[1], r); p[2] = dvd(p[2], r);
    }
    const double Aw = v.centring == 1 ? uniform_aw(v, lam) : dvd(mul(v.A0, lam), sqr_t((double)n));
    for (int k = lane; k < n; k += 32) {
        double d[3];
        for (int a = 0; a < 3; a++) d[a] = mi(sub(sm.op[k][a], b[a]), L, hL);
        const double d2 = norm2(d[0], d[1], d[2]);
        double dl[3];
        if (PREC == 0) wavelet_disp64(d, d2, lam, Aw, p, dl);
        else wavelet_disp32(d, lam, Aw, p, dl);
        int im[3] = {0, 0, 0};
        for (int a = 0; a < 3; a++) {
            const double u = add(sm.op[k][a], dl[a]);
            sm.nu[k][a] = u;
            sm.np[k][a] = wrap(u, L, &im[a]);
        }
        sm.dimg[k] = pack_img(im[0], im[1], im[2]);
        const int me = sm.ids[k];
        int r = 0;
        for (int t = 0; t < n; t++) r += sm.ids[t] < me;
        sm.sid[r] = me;
    }
    __syncwarp();
    // bonded partners outside the support must lie in the region
    bool bad = false;
    for (int k = lane; k < n; k += 32) {
        const int m = sm.ids[k];
        for (int e = 0; e < 2; e++) {
            const int q = e ? m + 1 : m - 1;
            if (q < 0 || q >= v.N || !(e ? v.bnext[m] : v.bnext[q]) || sorted_has(sm.sid, n, q)) continue;
            const Bead bq = v.bead[q];
            const int64_t cq[3] = {fine_cell(bq.x, v.invf, Gf), fine_cell(bq.y, v.invf, Gf), fine_cell(bq.z, v.invf, Gf)};
            for (int a = 0; a < 3; a++) if (!range_inside(cq[a], cq[a], rlo[a], rhi[a], Gf)) bad = true;
        }
    }
    if (__any_sync(FULL, bad)) return DEFER;
    int ncols = 0, nzmax = 0;
    partner_boxes(v, sm, n, lane, &ncols, &nzmax);
    // Metropolis threshold (Eq. 20): accept iff dU <= -kT ln(1 - u)
    const u4 w = draw(v.k0, v.k1, K_ACC, l, sweep, (uint32_t)j, 0);
    const double thr = accept_threshold(v, w);
    bool acc;
    int pe = 0;
    if (PREC == 1) {
        // binary32 energy change; decided in binary64 only within the rigorous error band
        float d32 = 0.0f, m32 = 0.0f;
        int T = 0;
        energy<true>(v, sm, n, lane, ncols, nzmax, nullptr, &d32, &m32, &T, &pe);
        const double band = 2.0 * (double)(80 + T + 6) * 5.9604644775390625e-08 * (double)m32 + 1e-9 * v.kT;
        if (isfinite(d32) && isfinite(m32) && fabs((double)d32 - thr) > band) {
            acc = (double)d32 <= thr;
            *du_out = (double)d32;
            if (v.audit) {
                double d64 = 0.0;
                int pe2 = 0;
                energy<false>(v, sm, n, lane, ncols, nzmax, &d64, nullptr, nullptr, nullptr, &pe2);
                if (lane == 0) audit_record(v, (double)d32, band, thr, d64, thr);
            }
        } else {
            double d64 = 0.0;
            int pe2 = 0;
            energy<false>(v, sm, n, lane, ncols, nzmax, &d64, nullptr, nullptr, nullptr, &pe2);
            acc = d64 <= thr;
            *du_out = d64;
            (*recheck_out)++;
            if (v.audit && lane == 0) audit_record(v, (double)d32, isfinite(m32) ? band : (double)INFINITY, thr, d64, thr);
        }
    } else {
        double d64 = 0.0;
        energy<false>(v, sm, n, lane, ncols, nzmax, &d64, nullptr, nullptr, nullptr, &pe);
        acc = d64 <= thr;
        *du_out = d64;
    }
    *pe_out += pe;
    if (!acc) return REJECT;
    // commit: positions, image counters, then cell-list moves (lane 0, in support order)
    for (int k = lane; k < n; k += 32) {
        const int m = sm.ids[k];
        put_bead(v.bead, v.bf, m, sm.np[k][0], sm.np[k][1], sm.np[k][2]);
        if (sm.dimg[k] != pack_img(0, 0, 0)) {
            int dd[3];
            unpack_img(sm.dimg[k], dd);
            v.img[3 * m] += dd[0]; v.img[3 * m + 1] += dd[1]; v.img[3 * m + 2] += dd[2];
        }
    }
    __syncwarp();
    if (lane == 0) {
        for (int k = 0; k < n; k++) {
            const int m = sm.ids[k];
            const int oc = cell_lin(v, sm.op[k][0], sm.op[k][1], sm.op[k][2]);
            const int ncl = cell_lin(v, sm.np[k][0], sm.np[k][1], sm.np[k][2]);
            if (oc == ncl) continue;
            relink(v, m, oc, ncl);
        }
    }
    __syncwarp();
    return ACCEPT;
}

}  // namespace wmcd

namespace wmcd {

// ======================================================================================
// Serial wavelet moves: one block runs the layer's deferred slots (schedule order), or
// every slot of a serial layer, one move after another. Supports of any size.
// ======================================================================================
// Slot parameters of the serial phase, one thread per slot, ahead of the sequential loop:
// the centre offset V and the polarisation by rejection from the unit ball (Appendix D), p
// normalised, and the Metropolis threshold -kT ln(1 - u) (Eq. 20). They depend only on the
// slot's counter, not on the state, so computing them early changes nothing.

// pairs a serial move keeps for its binary64 recheck (dynamic shared memory of the serial kernel
// in its mixed-precision 512-thread form, the one lone simulations use; other forms walk again)
constexpr int kSerialPairCap = 8192;
template <int PREC, int NT> __host__ __device__ constexpr int serial_pair_cap() { return (PREC == 1 && NT >= 512) ? kSerialPairCap : 0; }
// support members the gather keeps in shared memory (the 512-thread forms): written there by the
// few lanes that find a member, then to the global arrays in whole warps by the displacement
// pass; single-lane global stores from the gather held the block's memory pipe ~37k cycles a move
constexpr int kSerialMemCap = 2048;
template <int NT> __host__ __device__ constexpr int serial_mem_cap() { return NT >= 512 ? kSerialMemCap : 0; }
// (member, occupied partner cell) entries of a move's pair search, walked one per thread
constexpr int kSerialEntCap = 4096;
template <int NT> __host__ __device__ constexpr int serial_ent_cap() { return NT >= 512 ? kSerialEntCap : 0; }
template <int PREC, int NT> __host__ __device__ constexpr size_t serial_dyn_bytes() {
    return (size_t)serial_mem_cap<NT>() * (4 * sizeof(double) + sizeof(int)) + (size_t)serial_pair_cap<PREC, NT>() * sizeof(int2) +
           (size_t)serial_ent_cap<NT>() * 2 * sizeof(int);
}
template <int PREC, int NT>
__global__ void __launch_bounds__(NT, 1) k_serial(const SimView* __restrict__ vs, int l) {
    SIM_EXIT_IF(l >= gv.nL || gv.precision != PREC || (((gv.smem_layers | gv.big_layers) >> l) & 1))
    SIM_PROLOGUE
    if (l >= v.nL || v.precision != PREC || (((v.smem_layers | v.big_layers) >> l) & 1)) return;
    if (threadIdx.x == 0) *v.cl_stale = 0;      // rebuilt just before this launch if it was stale
    const int M = v.counts[l];
    const int use_list = v.layer[l].G > 0;
    __shared__ double sh_b[3], sh_p[3], sh_carry, sh_awx[2];
    // dynamic shared memory: support offsets (4 per member) and ids of the first members, then
    // the pairs within the WCA cutoff (old or new) found by the binary32 pass, for a binary64
    // pass that then visits only those (more than the capacity: the full walk again)
    extern __shared__ __align__(16) double sh_dyn[];
    // occupied cells of the ball found by the row pass, walked one per thread afterwards (a row
    // of a dense region holds tens of beads: one thread walking it is the search's longest chain)
    constexpr int kCellCap = NT >= 512 ? 4096 : 1;
    __shared__ int sh_cells[kCellCap];
    __shared__ int sh_ncell;
    double* const sm_d = sh_dyn;
    int2* const sh_pairs = (int2*)(sh_dyn + 4 * serial_mem_cap<NT>());
    int* const sm_ids = (int*)(sh_pairs + serial_pair_cap<PREC, NT>());
    int* const ent_k = sm_ids + serial_mem_cap<NT>();
    int* const ent_c = ent_k + serial_ent_cap<NT>();
    __shared__ int sh_nent;
    // beads of an accepted move that change fine cell: (bead, old cell, new cell), relinked by
    // one thread per old cell and then one per new cell (a cell's beads in list order)
    constexpr int kChCap = NT >= 512 ? 1024 : 1;
    __shared__ int sc_m[kChCap], sc_oc[kChCap], sc_nc[kChCap];
    __shared__ int sh_np;
    __shared__ double sh_red[NT / 32];
    __shared__ int sh_n, sh_nch, sh_acc, sh_brute, sh_c0[3], sh_nc[3], sh_total, sh_need64;
    __shared__ float sh_a32[3];                   // binary32 energy change, band, threshold (audit)
    __shared__ float sh_f32[NT / 32], sh_m32[NT / 32];
    __shared__ int sh_T[NT / 32];
    __shared__ int sh_scan[NT];
    __shared__ uint32_t sh_tag;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const LayerDev& Ly = v.layer[l];
    const double L = v.L, hL = v.halfL;
    const Pot& P = v.pot;
    const int count = use_list ? *v.serial_count : M;
    // trace flags of a serial move: 4 deferred by the colouring, 8 by its second colouring too
    const int dflag = use_list ? (v.layer[l].G2 > 0 ? 12 : 4) : 0;
    if (tid == 0) sh_carry = v.carry_serial[l];
    __syncthreads();
    long long att = 0, acc_n = 0, bu = 0, pe = 0, rechecks = 0, moved_n = 0;
    const float hLf = (float)hL, Lf = (float)L;
    const bool kappa_on = P.kappa != 0.0, eps_on = P.eps != 0.0;
    __shared__ double sh_lam, sh_lam2;
    __shared__ float sh_bf[3], sh_rl2f;
    // the binary64 values the whole block needs for a move are formed once, by thread 0, and
    // shared: on this part each binary64 instruction of every warp would occupy the pipe
    for (int t = 0; t < count; t++) {
        const int j = use_list ? v.serial_list[t] : t;
        const int i = v.slot_bead[j];
        if (tid == 0) {
            const double lam = sh_carry > 0.0 ? sh_carry : v.slot_lam[j];
            sh_lam = lam;
            sh_lam2 = mul(lam, lam);
            const float rlf = (float)lam + (float)(8.0 * L * 5.9604644775390625e-8 + 1e-6);
            sh_rl2f = rlf * rlf * (1.0f + 9.5367431640625e-7f);
            const double ri[3] = {v.bead[i].x, v.bead[i].y, v.bead[i].z};
            for (int a = 0; a < 3; a++) {
                sh_b[a] = v.centring == 1 ? v.slot_V[3 * j + a] : wrap(add(ri[a], mul(lam, v.slot_V[3 * j + a])), L, nullptr);
                sh_p[a] = v.slot_p[3 * j + a];
                sh_bf[a] = (float)sh_b[a];
            }
            const double eps = 1e-9;
            int64_t ncell = 1;
            for (int a = 0; a < 3; a++) {
                int t0 = (int)floor(mul(sub(sh_b[a], lam + eps), v.invf));
                int t1 = (int)floor(mul(add(sh_b[a], lam + eps), v.invf));
                sh_c0[a] = t0;
                sh_nc[a] = min(t1 - t0 + 1, v.Gf);
                ncell *= sh_nc[a];
            }
            sh_brute = ncell > v.N;
            sh_n = 0;
            sh_total = 0;
            sh_nch = 0;
            sh_np = 0;
            sh_ncell = 0;
            sh_nent = 0;
            uint32_t tag = *v.serial_tag + 1u;
            if (tag == 0u) tag = 1u;
            *v.serial_tag = tag;
            sh_tag = tag;
        }
        __syncthreads();
        const double lam = sh_lam, lam2 = sh_lam2;
        const double b[3] = {sh_b[0], sh_b[1], sh_b[2]};
        // gather the support
        // binary32 screen on the shadow (margin 8 L 2^-24 + 1e-6 on the distance covers the rounding
        // of the shadow, of b and of the difference), then the binary64 test
        const float bxf = sh_bf[0], byf = sh_bf[1], bzf = sh_bf[2];
        const float rl2f = sh_rl2f;
        auto wrapg = [&](float f) { return fabsf(f) > hLf ? f - copysignf(Lf, f) : f; };
        auto screened = [&](const BeadF& f) {
            const float sx = wrapg(f.hx - bxf), sy = wrapg(f.hy - byf), sz = wrapg(f.hz - bzf);
            return sx * sx + sy * sy + sz * sz <= rl2f;
        };
        auto consider_exact = [&](int m, const Bead& bb) {
            double d0 = mi(sub(bb.x, b[0]), L, hL), d1 = mi(sub(bb.y, b[1]), L, hL), d2c = mi(sub(bb.z, b[2]), L, hL);
            double d2 = norm2(d0, d1, d2c);
            if (d2 < lam2) {
                int idx = atomicAdd(&sh_n, 1);
                int* ids = v.s_ids;
                double* dd = v.s_d;
                if (idx < serial_mem_cap<NT>()) { ids = sm_ids; dd = sm_d; }
                ids[idx] = m;
                dd[4 * idx] = d0; dd[4 * idx + 1] = d1; dd[4 * idx + 2] = d2c; dd[4 * idx + 3] = d2;
            }
        };
        // four independent loads in flight per thread (the shadows of four beads, or the heads
        // of four cells) before any is used
        if (sh_brute) {
            for (int64_t m0 = tid; m0 < v.N; m0 += 4 * (int64_t)NT) {
                BeadF f[4];
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    const int64_t m = m0 + (int64_t)u * NT;
                    if (m < v.N) f[u] = v.bf[m];
                }
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    const int64_t m = m0 + (int64_t)u * NT;
                    if (m < v.N && screened(f[u])) consider_exact((int)m, v.bead[m]);
                }
            }
        } else if (v.occ) {
            // rows (y, z) of the ball's cell box over the threads; each row's x range read as
            // occupancy words, and only the lists of occupied cells walked
            const int c0[3] = {sh_c0[0], sh_c0[1], sh_c0[2]}, nc[3] = {sh_nc[0], sh_nc[1], sh_nc[2]};
            const int Gf = v.Gf, rows = nc[1] * nc[2];
            const int x0 = wrapi(c0[0], Gf);
            for (int r = tid; r < rows; r += NT) {
                const int y = wrapi(c0[1] + r % nc[1], Gf), z = wrapi(c0[2] + r / nc[1], Gf);
                const uint32_t* row = v.occ + ((size_t)y + (size_t)Gf * z) * v.occ_w;
                const int rowcell = Gf * (y + Gf * z);
                // the x range [x0, x0 + nc[0]) as at most two pieces inside [0, Gf)
                for (int piece = 0; piece < 2; piece++) {
                    const int a = piece == 0 ? x0 : 0;
                    const int b = piece == 0 ? min(x0 + nc[0], Gf) : x0 + nc[0] - Gf;
                    for (int wi = a >> 5; a < b && wi <= (b - 1) >> 5; wi++) {
                        uint32_t bits = row[wi];
                        const int lo = max(a - (wi << 5), 0), hi = min(b - (wi << 5), 32);
                        bits &= (hi >= 32 ? 0xffffffffu : ((1u << hi) - 1u)) & ~((1u << lo) - 1u);
                        for (; bits; bits &= bits - 1u) {
                            const int cell = rowcell + (wi << 5) + __ffs(bits) - 1;
                            const int slot = NT >= 512 ? atomicAdd(&sh_ncell, 1) : kCellCap;
                            if (slot < kCellCap) { sh_cells[slot] = cell; continue; }
                            int guard = 0;             // list full: walked here
                            for (int q = v.head[cell]; q >= 0;) {
                                const Bead bb = v.bead[q];
                                if (screened(v.bf[q])) consider_exact(q, bb);
                                q = bb.next;
                                if (++guard > kMaxWalk) { set_err(v, E_WALK); break; }
                            }
                        }
                    }
                }
            }
            if (NT >= 512) {
                __syncthreads();
                const int nlist = min(sh_ncell, kCellCap);
                for (int i = tid; i < nlist; i += NT) {
                    int guard = 0;
                    for (int q = v.head[sh_cells[i]]; q >= 0;) {
                        const Bead bb = v.bead[q];
                        if (screened(v.bf[q])) consider_exact(q, bb);
                        q = bb.next;
                        if (++guard > kMaxWalk) { set_err(v, E_WALK); break; }
                    }
                }
            }
        } else {
            const int c0[3] = {sh_c0[0], sh_c0[1], sh_c0[2]}, nc[3] = {sh_nc[0], sh_nc[1], sh_nc[2]};
            const int ncell = nc[0] * nc[1] * nc[2];
            for (int k0 = tid; k0 < ncell; k0 += 4 * NT) {
                int hd[4];
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    const int k = k0 + u * NT;
                    hd[u] = -1;
                    if (k < ncell) {
                        const int kx = k % nc[0], ky = (k / nc[0]) % nc[1], kz = k / (nc[0] * nc[1]);
                        hd[u] = v.head[wrapi(c0[0] + kx, v.Gf) + v.Gf * (wrapi(c0[1] + ky, v.Gf) + v.Gf * wrapi(c0[2] + kz, v.Gf))];
                    }
                }
                for (int u = 0; u < 4; u++) {
                    int guard = 0;
                    for (int q = hd[u]; q >= 0;) {
                        const Bead bb = v.bead[q];
                        if (screened(v.bf[q])) consider_exact(q, bb);
                        q = bb.next;
                        if (++guard > kMaxWalk) { set_err(v, E_WALK); break; }
                    }
                }
            }
        }
        __syncthreads();
        const int n = sh_n;
        if (n == 0) {      // nothing inside: no motion, dU = 0 against the threshold
            if (tid == 0) {
                const bool acc0 = 0.0 <= v.slot_thr[j];
                att++;
                if (acc0) acc_n++;
                v.tr_out[Ly.tr_off + j] = (uint8_t)((acc0 ? 1 : 2) | dflag);
                v.tr_n[Ly.tr_off + j] = 0;
                v.tr_du[Ly.tr_off + j] = 0.0;
                sh_carry = acc0 ? 0.0 : lam;
            }
            __syncthreads();
            continue;
        }
        const uint32_t tag = sh_tag;
        // A_w (Eq. 29) and the partner-box reach, formed once by thread 0: on this part every
        // binary64 instruction of a warp holds the unit for tens of cycles, so the division and
        // square root are not repeated in every warp that holds a member
        if (tid == 0) {
            const double aw = v.centring == 1 ? uniform_aw(v, lam) : dvd(mul(v.A0, lam), sqr_t((double)n));
            sh_awx[0] = aw;
            sh_awx[1] = add(v.rc, mul(0.25, aw)) + 1e-9;
        }
        __syncthreads();
        const double Aw = sh_awx[0];
        const double p[3] = {sh_p[0], sh_p[1], sh_p[2]};
        for (int k = tid; k < n; k += NT) {
            const bool in_sm = k < serial_mem_cap<NT>();
            const double* dd = in_sm ? sm_d : v.s_d;
            const int m = in_sm ? sm_ids[k] : v.s_ids[k];
            if (in_sm) v.s_ids[k] = m;           // the later passes read the global arrays
            v.bead[m].mark = tag;
            v.s_slot[m] = k;
            double d[3] = {dd[4 * k], dd[4 * k + 1], dd[4 * k + 2]}, dl[3];
            if (PREC == 0) wavelet_disp64(d, dd[4 * k + 3], lam, Aw, p, dl);
            else wavelet_disp32(d, lam, Aw, p, dl);
            const double o[3] = {v.bead[m].x, v.bead[m].y, v.bead[m].z};
            int im[3] = {0, 0, 0};
            const unsigned am = __activemask();
            double nx[3] = {add(o[0], dl[0]), add(o[1], dl[1]), add(o[2], dl[2])};
            wrap3_u(nx, L, am, im);
            for (int a = 0; a < 3; a++) {
                v.s_new[3 * k + a] = nx[a];
                v.s_d[4 * k + a] = dl[a];        // keep the displacement for the partner boxes
            }
            v.s_img[k] = pack_img(im[0], im[1], im[2]);
        }
        __syncthreads();
        // energy change: bonds and the external well per member; pair terms by one thread per
        // (member, fine cell of its partner box) item, so a small support still spreads its list
        // walks over the block. Mixed precision: a binary32 pass first (each difference of
        // binary64 positions rounded once, the new one formed from the old one and the binary32
        // displacements), deciding outside the rigorous error band; the binary64 pass decides
        // inside it and in binary64 mode.
        const double ext = sh_awx[1];
        const double thr = v.slot_thr[j];
        // old-position difference a - b, minimum image, rounded once to binary32
        auto d32 = [&](double a, double b) {
            const double e = sub(a, b);
            float f = (float)e;
            if (fabsf(f) > hLf) f = (float)(e > 0.0 ? sub(e, L) : add(e, L));
            return f;
        };
        auto wrapf = [&](float f) { return fabsf(f) > hLf ? f - copysignf(Lf, f) : f; };
        // the same difference from the binary32 shadows (hi, lo): no binary64 arithmetic unless
        // the pair straddles a face, where it is wrapped in binary64
        auto dsh = [&](float ha, float la, float hb, float lb, double a, double b) {
            const float dh = ha - hb;
            if (fabsf(dh) <= hLf) return dh + (la - lb);
            return d32(a, b);
        };
        // partner boxes and their exclusive prefix (items), shared by both passes
        for (int k = tid; k < n; k += NT) {
            int cnt = 0;
            if (eps_on) {
                const int m = v.s_ids[k];
                const Bead bm = v.bead[m];
                const double o[3] = {bm.x, bm.y, bm.z};
                double lo[3], hi[3];
                for (int a = 0; a < 3; a++) {
                    double u = add(o[a], v.s_d[4 * k + a]);
                    lo[a] = sub(fmin(o[a], u), ext);
                    hi[a] = add(fmax(o[a], u), ext);
                }
                int c0[3], nc[3];
                cell_box(v, lo, hi, c0, nc);
                for (int a = 0; a < 3; a++) { v.s_box[6 * k + a] = c0[a]; v.s_box[6 * k + 3 + a] = nc[a]; }
                cnt = v.occ ? nc[1] * nc[2] : nc[0] * nc[1] * nc[2];   // rows (y, z), or cells
            }
            v.s_pre[k] = cnt;
        }
        __syncthreads();
        int W = 0;
        if (eps_on) {
            // exclusive prefix of the box sizes, NT members per pass
            for (int base = 0; base < n; base += NT) {
                const int k = base + tid;
                const int x = k < n ? v.s_pre[k] : 0;
                sh_scan[tid] = x;
                __syncthreads();
                for (int off = 1; off < NT; off <<= 1) {
                    const int y = tid >= off ? sh_scan[tid - off] : 0;
                    __syncthreads();
                    sh_scan[tid] += y;
                    __syncthreads();
                }
                if (k < n) v.s_pre[k] = sh_total + sh_scan[tid] - x;
                __syncthreads();
                if (tid == NT - 1) sh_total += sh_scan[NT - 1];
                __syncthreads();
            }
            W = sh_total;
            if (tid == 0) v.s_pre[n] = W;
            __syncthreads();
        }
        // each thread takes a contiguous run of items, with one search for its first member and
        // member data reloaded only when the run crosses to the next member
        auto run_items = [&](auto&& item) {
            const int t0 = (int)((int64_t)tid * W / NT), t1 = (int)((int64_t)(tid + 1) * W / NT);
            if (t0 >= t1) return;
            int lo_k = 0, hi_k = n - 1;                 // last member with s_pre <= t0
            while (lo_k < hi_k) {
                const int mid = (lo_k + hi_k + 1) >> 1;
                if (v.s_pre[mid] <= t0) lo_k = mid; else hi_k = mid - 1;
            }
            int kn = lo_k, kn_start = v.s_pre[kn], kn_end = v.s_pre[kn + 1];
            int c0n[3] = {v.s_box[6 * kn], v.s_box[6 * kn + 1], v.s_box[6 * kn + 2]};
            int ncn[3] = {v.s_box[6 * kn + 3], v.s_box[6 * kn + 4], v.s_box[6 * kn + 5]};
            auto advance = [&](int t) {
                while (t >= kn_end) {
                    kn++;
                    kn_start = kn_end;
                    kn_end = v.s_pre[kn + 1];
                    for (int a = 0; a < 3; a++) { c0n[a] = v.s_box[6 * kn + a]; ncn[a] = v.s_box[6 * kn + 3 + a]; }
                }
            };
            item(t0, t1, advance, kn, kn_start, c0n, ncn);
        };
        auto walk = [&](auto&& visit, int h, int k, int m) {
            int guard = 0;
            for (int q = h; q >= 0;) {
                const Bead bq = v.bead[q];
                const int nx = bq.next;
                if (q != m) visit(k, m, q, bq);
                q = nx;
                if (++guard > kMaxWalk) { set_err(v, E_WALK); break; }
            }
        };
        // with occupancy bits an item is a row (y, z) of a member's partner box, whose x range is
        // read as occupancy words: cellfn(k, m, cell) for each occupied cell
        auto for_cells = [&](auto&& cellfn) {
            run_items([&](int t0, int t1, auto& advance, int& kn, int& kn_start, int* c0n, int* ncn) {
                const int Gf = v.Gf;
                for (int t = t0; t < t1; t++) {
                    advance(t);
                    const int r = t - kn_start, m = v.s_ids[kn];
                    const int y = wrapi(c0n[1] + r % ncn[1], Gf), z = wrapi(c0n[2] + r / ncn[1], Gf);
                    const uint32_t* row = v.occ + ((size_t)y + (size_t)Gf * z) * v.occ_w;
                    const int rowcell = Gf * (y + Gf * z), x0 = wrapi(c0n[0], Gf);
                    // the x range [x0, x0 + nc) as at most two pieces inside [0, Gf)
                    for (int piece = 0; piece < 2; piece++) {
                        const int xa = piece == 0 ? x0 : 0;
                        const int xb = piece == 0 ? min(x0 + ncn[0], Gf) : x0 + ncn[0] - Gf;
                        for (int wi = xa >> 5; xa < xb && wi <= (xb - 1) >> 5; wi++)
                            for (uint32_t bits = occ_masked(row[wi], xa, xb, wi); bits; bits &= bits - 1u)
                                cellfn(kn, m, rowcell + (wi << 5) + __ffs(bits) - 1);
                    }
                }
            });
        };
        // the (member, occupied cell) entries listed once, then walked one per thread: a run of
        // items in a dense region walked by one thread was the pass's longest chain
        int nent = 0;
        bool listed = false;
        if (eps_on && v.occ && serial_ent_cap<NT>() > 0) {
            for_cells([&](int k, int m, int cell) {
                const int i = atomicAdd(&sh_nent, 1);
                if (i < serial_ent_cap<NT>()) { ent_k[i] = k; ent_c[i] = cell; }
            });
            __syncthreads();
            nent = sh_nent;
            listed = nent <= serial_ent_cap<NT>();
        }
        // every (member, bead) pair of the partner boxes: visit(k, m, q, bead q)
        auto for_pairs = [&](auto&& visit) {
            if (listed) {
                for (int i = tid; i < nent; i += NT) {
                    const int k = ent_k[i];
                    walk(visit, v.head[ent_c[i]], k, v.s_ids[k]);
                }
                return;
            }
            if (v.occ) {
                for_cells([&](int k, int m, int cell) { walk(visit, v.head[cell], k, m); });
                return;
            }
            // an item is a cell; the head of the next item's cell is loaded before the current
            // cell is walked
            run_items([&](int t0, int t1, auto& advance, int& kn, int& kn_start, int* c0n, int* ncn) {
                advance(t0);
                int h = v.head[box_cell(v, c0n, ncn, t0 - kn_start)];
                int cur_k = kn;
                for (int t = t0; t < t1; t++) {
                    int hn = -1, nk = cur_k;
                    if (t + 1 < t1) { advance(t + 1); hn = v.head[box_cell(v, c0n, ncn, t + 1 - kn_start)]; nk = kn; }
                    walk(visit, h, cur_k, v.s_ids[cur_k]);
                    h = hn;
                    cur_k = nk;
                }
            });
        };
        bool need64 = PREC == 0;
        if (PREC == 1) {
            const Pot32 P32 = pot32(P);
            float a32 = 0.0f, m32 = 0.0f;
            int T = 0;
            for (int k = tid; k < n; k += NT) {
                const int m = v.s_ids[k];
                const Bead bm = v.bead[m];
                const double o[3] = {bm.x, bm.y, bm.z};
                const float dlm[3] = {(float)v.s_d[4 * k], (float)v.s_d[4 * k + 1], (float)v.s_d[4 * k + 2]};
                const BeadF fm = v.bf[m];
                const float mh[3] = {fm.hx, fm.hy, fm.hz}, ml[3] = {fm.lx, fm.ly, fm.lz};
                if (kappa_on) {
                    float ro = 0.0f, rn = 0.0f;
                    for (int a = 0; a < 3; a++) {
                        const float c = d32(o[a], hL);
                        ro += c * c;
                        const float cn = wrapf(c + dlm[a]);
                        rn += cn * cn;
                    }
                    const float un = 0.5f * P32.kappa * rn, uo = 0.5f * P32.kappa * ro;
                    a32 += un - uo; m32 += un + uo; T += 2;
                }
                for (int e = 0; e < 2; e++) {
                    const int q = e ? m + 1 : m - 1;
                    if (q < 0 || q >= v.N || !(e ? v.bnext[m] : v.bnext[q])) continue;
                    const Bead bq = v.bead[q];
                    float dlq[3] = {0.0f, 0.0f, 0.0f};
                    if (bq.mark == tag) {
                        if (q < m) continue;
                        const int sq = v.s_slot[q];
                        for (int a = 0; a < 3; a++) dlq[a] = (float)v.s_d[4 * sq + a];
                    }
                    const double qo[3] = {bq.x, bq.y, bq.z};
                    const BeadF fq = v.bf[q];
                    const float qh[3] = {fq.hx, fq.hy, fq.hz}, ql[3] = {fq.lx, fq.ly, fq.lz};
                    float ro = 0.0f, rn = 0.0f;
                    for (int a = 0; a < 3; a++) {
                        const float c = dsh(mh[a], ml[a], qh[a], ql[a], o[a], qo[a]);
                        ro += c * c;
                        const float cn = wrapf(c + dlm[a] - dlq[a]);
                        rn += cn * cn;
                    }
                    float un, mn, uo, mo;
                    bond32(P32, rn, un, mn);
                    bond32(P32, ro, uo, mo);
                    a32 += un - uo; m32 += mn + mo; T += 2;
                }
            }
            if (eps_on) {
                const float rc2p = P32.rc2 * 1.0001f;
                int mk = -1;
                double o[3] = {0.0, 0.0, 0.0};
                float dlm[3] = {0.0f, 0.0f, 0.0f}, mh[3] = {0.0f, 0.0f, 0.0f}, ml[3] = {0.0f, 0.0f, 0.0f};
                for_pairs([&](int k, int m, int q, const Bead& bq) {
                    const bool member = bq.mark == tag;
                    if (member && q < m) return;
                    if (k != mk) {
                        mk = k;
                        const Bead bm = v.bead[m];
                        o[0] = bm.x; o[1] = bm.y; o[2] = bm.z;
                        const BeadF fm = v.bf[m];
                        mh[0] = fm.hx; mh[1] = fm.hy; mh[2] = fm.hz; ml[0] = fm.lx; ml[1] = fm.ly; ml[2] = fm.lz;
                        for (int a = 0; a < 3; a++) dlm[a] = (float)v.s_d[4 * k + a];
                    }
                    float dlq[3] = {0.0f, 0.0f, 0.0f};
                    if (member) {
                        const int sq = v.s_slot[q];
                        for (int a = 0; a < 3; a++) dlq[a] = (float)v.s_d[4 * sq + a];
                    }
                    const double qo[3] = {bq.x, bq.y, bq.z};
                    const BeadF fq = v.bf[q];
                    const float qh[3] = {fq.hx, fq.hy, fq.hz}, ql[3] = {fq.lx, fq.ly, fq.lz};
                    float ro = 0.0f, rn = 0.0f;
                    for (int a = 0; a < 3; a++) {
                        const float c = dsh(mh[a], ml[a], qh[a], ql[a], o[a], qo[a]);
                        ro += c * c;
                        const float cn = wrapf(c + dlm[a] - dlq[a]);
                        rn += cn * cn;
                    }
                    float un, mn, uo, mo;
                    wca32(P32, rn, un, mn);
                    wca32(P32, ro, uo, mo);
                    if (un != 0.0f || uo != 0.0f || mn != 0.0f || mo != 0.0f) {
                        a32 += un - uo; m32 += mn + mo; T += 2;
                        if (!member) pe++;
                    }
                    // within the cutoff with a margin far above the binary32 error of r^2
                    if (rn < rc2p || ro < rc2p) {
                        const int ip = atomicAdd(&sh_np, 1);
                        if (ip < serial_pair_cap<PREC, NT>()) sh_pairs[ip] = make_int2(k, q);
                    }
                });
            }
            for (int sft = 16; sft > 0; sft >>= 1) {
                a32 += __shfl_xor_sync(0xffffffffu, a32, sft);
                m32 += __shfl_xor_sync(0xffffffffu, m32, sft);
                T = max(T, __shfl_xor_sync(0xffffffffu, T, sft));
            }
            if (lane == 0) { sh_f32[wid] = a32; sh_m32[wid] = m32; sh_T[wid] = T; }
            __syncthreads();
            if (tid == 0) {
                float du = 0.0f, mm = 0.0f;
                int tt = 0;
                for (int w = 0; w < NT / 32; w++) { du += sh_f32[w]; mm += sh_m32[w]; tt = max(tt, sh_T[w]); }
                tt += 5 + NT / 32;     // summation depth: one thread's terms, the butterfly, the warp totals
                const float thr32 = (float)thr;
                const float band = 2.0f * (float)(80 + tt + 6) * 5.9604645e-08f * mm + 1e-9f * (float)v.kT +
                                   2.4e-7f * fabsf(thr32);
                sh_a32[0] = du; sh_a32[1] = band; sh_a32[2] = thr32;
                if (isfinite(du) && isfinite(band) && fabsf(du - thr32) > band) {
                    sh_acc = du <= thr32;
                    sh_need64 = v.audit ? 2 : 0;     // 2: the binary64 pass runs for the audit only
                    v.tr_du[Ly.tr_off + j] = (double)du;
                } else {
                    sh_need64 = 1;
                    rechecks++;
                }
            }
            __syncthreads();
            need64 = sh_need64;
        }
        if (need64) {
            double dU = 0.0;
            for (int k = tid; k < n; k += NT) {
                const int m = v.s_ids[k];
                const Bead bm = v.bead[m];
                const double o[3] = {bm.x, bm.y, bm.z};
                const double nw[3] = {v.s_new[3 * k], v.s_new[3 * k + 1], v.s_new[3 * k + 2]};
                dU += U_ext(P, nw[0], nw[1], nw[2]) - U_ext(P, o[0], o[1], o[2]);
                for (int e = 0; e < 2; e++) {
                    int q = e ? m + 1 : m - 1;
                    if (q < 0 || q >= v.N || !(e ? v.bnext[m] : v.bnext[q])) continue;
                    Bead bq = v.bead[q];
                    double qn[3] = {bq.x, bq.y, bq.z};
                    if (bq.mark == tag) {
                        if (q < m) continue;
                        int sq = v.s_slot[q];
                        qn[0] = v.s_new[3 * sq]; qn[1] = v.s_new[3 * sq + 1]; qn[2] = v.s_new[3 * sq + 2];
                    }
                    double r2n = norm2(mi(nw[0] - qn[0], L, hL), mi(nw[1] - qn[1], L, hL), mi(nw[2] - qn[2], L, hL));
                    double r2o = norm2(mi(o[0] - bq.x, L, hL), mi(o[1] - bq.y, L, hL), mi(o[2] - bq.z, L, hL));
                    dU += U_bond(P, r2n) - U_bond(P, r2o);
                }
            }
            // the pairs the binary32 pass listed (mixed precision, list complete), else all pairs
            const int npairs = serial_pair_cap<PREC, NT>() > 0 ? sh_np : 1;
            if (eps_on && npairs <= serial_pair_cap<PREC, NT>()) {
                for (int ip = tid; ip < npairs; ip += NT) {
                    const int2 pr = sh_pairs[ip];
                    const int k = pr.x, m = v.s_ids[k], q = pr.y;
                    const Bead bm = v.bead[m], bq = v.bead[q];
                    const double nw[3] = {v.s_new[3 * k], v.s_new[3 * k + 1], v.s_new[3 * k + 2]};
                    double qn[3] = {bq.x, bq.y, bq.z};
                    if (bq.mark == tag) {
                        const int sq = v.s_slot[q];
                        qn[0] = v.s_new[3 * sq]; qn[1] = v.s_new[3 * sq + 1]; qn[2] = v.s_new[3 * sq + 2];
                    }
                    const double r2n = norm2(mi(nw[0] - qn[0], L, hL), mi(nw[1] - qn[1], L, hL), mi(nw[2] - qn[2], L, hL));
                    const double r2o = norm2(mi(bm.x - bq.x, L, hL), mi(bm.y - bq.y, L, hL), mi(bm.z - bq.z, L, hL));
                    if (r2n < P.rc2 || r2o < P.rc2) dU += U_wca(P, r2n) - U_wca(P, r2o);
                }
            } else if (eps_on) {
                int mk = -1;
                double o[3] = {0.0, 0.0, 0.0}, nw[3] = {0.0, 0.0, 0.0};
                for_pairs([&](int k, int m, int q, const Bead& bq) {
                    const bool member = bq.mark == tag;
                    if (member && q < m) return;
                    if (k != mk) {
                        mk = k;
                        const Bead bm = v.bead[m];
                        o[0] = bm.x; o[1] = bm.y; o[2] = bm.z;
                        nw[0] = v.s_new[3 * k]; nw[1] = v.s_new[3 * k + 1]; nw[2] = v.s_new[3 * k + 2];
                    }
                    double qn[3] = {bq.x, bq.y, bq.z};
                    if (member) {
                        const int sq = v.s_slot[q];
                        qn[0] = v.s_new[3 * sq]; qn[1] = v.s_new[3 * sq + 1]; qn[2] = v.s_new[3 * sq + 2];
                    }
                    const double r2n = norm2(mi(nw[0] - qn[0], L, hL), mi(nw[1] - qn[1], L, hL), mi(nw[2] - qn[2], L, hL));
                    const double r2o = norm2(mi(o[0] - bq.x, L, hL), mi(o[1] - bq.y, L, hL), mi(o[2] - bq.z, L, hL));
                    if (r2n < P.rc2 || r2o < P.rc2) {
                        dU += U_wca(P, r2n) - U_wca(P, r2o);
                        if (!member && PREC == 0) pe++;
                    }
                });
            }
            dU = warp_sum(dU);
            if (lane == 0) sh_red[wid] = dU;
            __syncthreads();
            if (tid == 0) {
                double su = 0.0;
                for (int w = 0; w < NT / 32; w++) su += sh_red[w];
                if (PREC == 1 && v.audit) audit_record(v, (double)sh_a32[0], (double)sh_a32[1], (double)sh_a32[2], su, thr);
                if (PREC == 0 || sh_need64 != 2) {
                    sh_acc = su <= thr;
                    v.tr_du[Ly.tr_off + j] = su;
                }
            }
            __syncthreads();
        }
        const bool acc = sh_acc;
        if (acc) {
            for (int k = tid; k < n; k += NT) {
                const int m = v.s_ids[k];
                const Bead bm = v.bead[m];
                const int oc = cell_lin(v, bm.x, bm.y, bm.z);
                const double nw[3] = {v.s_new[3 * k], v.s_new[3 * k + 1], v.s_new[3 * k + 2]};
                const int ncl = cell_lin(v, nw[0], nw[1], nw[2]);
                put_bead(v.bead, v.bf, m, nw[0], nw[1], nw[2]);
                if (v.s_img[k] != pack_img(0, 0, 0)) {
                    int dd[3];
                    unpack_img(v.s_img[k], dd);
                    v.img[3 * m] += dd[0]; v.img[3 * m + 1] += dd[1]; v.img[3 * m + 2] += dd[2];
                }
                if (oc != ncl) {
                    int idx = atomicAdd(&sh_nch, 1);
                    v.s_changed[3 * idx] = m; v.s_changed[3 * idx + 1] = oc; v.s_changed[3 * idx + 2] = ncl;
                    if (idx < kChCap) { sc_m[idx] = m; sc_oc[idx] = oc; sc_nc[idx] = ncl; }
                }
            }
        }
        __syncthreads();
        const int nch = sh_nch;
        if (NT >= 512 && nch > 1 && nch <= kChCap) {
            grouped_relink(v, sc_m, sc_oc, sc_nc, nch, tid, NT);
        } else if (tid == 0) {
            for (int c = 0; c < nch; c++) {
                int m = v.s_changed[3 * c], oc = v.s_changed[3 * c + 1], ncl = v.s_changed[3 * c + 2];
                relink(v, m, oc, ncl);
            }
        }
        if (tid == 0) {
            att++;
            bu += n;
            if (acc) { acc_n++; moved_n += n; }
            v.tr_out[Ly.tr_off + j] = (uint8_t)((acc ? 1 : 2) | dflag);
            v.tr_n[Ly.tr_off + j] = n;
            sh_carry = acc ? 0.0 : lam;
        }
        __syncthreads();
    }
    // partner counts are per thread
    unsigned long long pe_all = (unsigned long long)pe;
    if (pe_all) atomicAdd(&v.ctr[C_PARTNER], pe_all);
    if (tid == 0) {
        v.carry_serial[l] = sh_carry;
        atomicAdd(&v.ctr[C_ATT + l], (unsigned long long)att);
        atomicAdd(&v.ctr[C_ACC + l], (unsigned long long)acc_n);
        atomicAdd(&v.ctr[C_ACCTOT], (unsigned long long)acc_n);
        atomicAdd(&v.ctr[C_BU], (unsigned long long)bu);
        if (moved_n) atomicAdd(&v.ctr[C_MOVED], (unsigned long long)moved_n);
        if (rechecks) atomicAdd(&v.ctr[C_RECHECK], (unsigned long long)rechecks);
    }
}
// Serial phase of a small simulation whose layers are all serial: the whole simulation is
// staged in shared memory for the launch (positions in binary64 and a binary32 copy), every
// slot of the layer runs on-chip, and the beads are written back at the end. Supports and
// pair partners are found by a binary32 pass over all staged beads with a margin that covers
// the rounding of the copy, then decided in binary64 exactly as the global-memory kernel
// does, so the two kernels take the same decisions. The global cell lists are not updated
// here; they are marked stale and rebuilt before the next plane-wave move that needs them.
// Shared bytes per bead: see smem_serial_bytes.
template <int PREC, int NT>
__global__ void __launch_bounds__(NT, 65536 / (NT * 128)) k_serial_smem(const SimView* __restrict__ vs, int l, int64_t nlo, int64_t nhi) {
    SIM_EXIT_IF(l >= gv.nL || gv.precision != PREC || !((gv.smem_layers >> l) & 1) || gv.counts[l] == 0 ||
                gv.N <= nlo || gv.N > nhi)
    SIM_PROLOGUE
    extern __shared__ __align__(16) char dsm[];
    if (l >= v.nL || v.precision != PREC || !((v.smem_layers >> l) & 1)) return;
    const int count = v.counts[l];
    if (count == 0) return;
    const int N = (int)v.N;
    // 8-byte arrays first, then 4-, 2- and 1-byte ones, so every array is aligned for any N
    double* px = (double*)dsm;
    double* py = px + N;
    double* pz = py + N;
    double* mnew = pz + N;                       // 3 per support member
    float* fx = (float*)(mnew + 3 * (size_t)N);  // binary32 pairs (hi, lo) of the positions
    float* fy = fx + N;
    float* fz = fy + N;
    float* lx = fz + N;
    float* ly = lx + N;
    float* lz = ly + N;
    float* mnf = lz + N;                         // 3 per member: new position, hi ...
    float* mnl = mnf + 3 * (size_t)N;            // ... and lo
    int* mid = (int*)(mnl + 3 * (size_t)N);      // support, in gather order
    short* sslot = (short*)(mid + N);            // per bead: index in the support or -1
    short* dimg = sslot + N;                     // 3 per bead: image change over the launch
    uint8_t* mimg = (uint8_t*)(dimg + 3 * (size_t)N);   // per member: packed image change of the move
    uint8_t* bn = mimg + N;                      // bond to the next bead
    __shared__ int s_cand[kSmemCand];            // beads within reach of the move, not in the support
    __shared__ int sh_nc;
    __shared__ float sh_rR2;
    __shared__ double sh_aw[33];                 // A_w for supports of 1..32 beads
    __shared__ float sh_awf[33], sh_lamf, sh_pf[3];
    __shared__ double sh_b[3], sh_p[3], sh_carry;
    __shared__ double sh_red[NT / 32];
    __shared__ float sh_f32[NT / 32], sh_m32[NT / 32];
    __shared__ int sh_T[NT / 32];
    __shared__ int sh_n, sh_acc, sh_stale, sh_need64;
    __shared__ float sh_a32[3];                   // binary32 energy change, band, threshold (audit)
    __shared__ double sh_lam, sh_lam2;
    __shared__ float sh_bf[3], sh_rl2;
    __shared__ double s_sqrt[kNCap + 1];         // sqrt(n), correctly rounded, for small supports
    for (int i2 = threadIdx.x; i2 <= kNCap; i2 += NT) s_sqrt[i2] = sqr_t((double)i2);
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const LayerDev& Ly = v.layer[l];
    const double L = v.L, hL = v.halfL;
    const float Lf = (float)L, hLf = (float)hL;
    const Pot& P = v.pot;
    // binary32 screens: a distance error of the copies below 8 L 2^-24 (rounding of the copies,
    // of the difference and of the image shift), so screening at r + 8 L 2^-24 + 1e-6 and a
    // relative 2^-20 on the square keeps every bead the binary64 test accepts
    const float marg = (float)(8.0 * L * 5.9604644775390625e-8 + 1e-6);
    for (int m = tid; m < N; m += NT) {
        const Bead b = v.bead[m];
        px[m] = b.x; py[m] = b.y; pz[m] = b.z;
        fx[m] = (float)b.x; fy[m] = (float)b.y; fz[m] = (float)b.z;
        lx[m] = (float)(b.x - (double)fx[m]); ly[m] = (float)(b.y - (double)fy[m]); lz[m] = (float)(b.z - (double)fz[m]);
        sslot[m] = -1;
        dimg[3 * m] = 0; dimg[3 * m + 1] = 0; dimg[3 * m + 2] = 0;
        bn[m] = v.bnext[m];
    }
    if (tid == 0) { sh_carry = v.carry_serial[l]; sh_stale = 0; }
    __syncthreads();
    const Pot32 P32 = pot32(P);
    const bool kappa_on = P.kappa != 0.0, eps_on = P.eps != 0.0;
    const float rcf = (float)v.rc + marg;
    const float rc2f = rcf * rcf * (1.0f + 9.5367431640625e-7f);
    long long att = 0, acc_n = 0, bu = 0, pe = 0, rechecks = 0, moved_n = 0;
    const float A0f = (float)v.A0, rcr = (float)v.rc;
    // every binary64 value the whole block needs for a move is formed once, by threads 0-2 (one
    // axis each) and shared: on this part each binary64 instruction of every warp would occupy
    // the pipe
    for (int j = 0; j < count; j++) {
        const int i = v.slot_bead[j];
        if (tid < 3) {
            const int a = tid;
            const double lam0 = __double_as_longlong(sh_carry) > 0 ? sh_carry : v.slot_lam[j];
            const double ri = a == 0 ? px[i] : (a == 1 ? py[i] : pz[i]);
            const double ba = v.centring == 1 ? v.slot_V[3 * j + a] : wrap_u(add(ri, mul(lam0, v.slot_V[3 * j + a])), L, 7u, nullptr);
            sh_b[a] = ba;
            sh_p[a] = v.slot_p[3 * j + a];
            sh_bf[a] = (float)ba;
            if (a == 0) {
                sh_lam = lam0;
                sh_lam2 = mul(lam0, lam0);
                const float lf = (float)lam0;
                const float rl = lf + marg;
                sh_rl2 = rl * rl * (1.0f + 9.5367431640625e-7f);
                // every WCA partner of a member, old or new position, lies within lam + A0 lam / 4 +
                // r_c of the centre (|displacement| <= A_w / 4 <= A0 lam / 4); three margins cover
                // the rounding of this screen and of the energy pass's own
                const float rR = lf + 0.25f * A0f * lf + rcr + 3.0f * marg;
                sh_rR2 = rR * rR * (1.0f + 9.5367431640625e-7f);
                sh_n = 0;
                sh_nc = 0;
            }
        } else if (tid >= 32 && tid < 64) {
            // beside thread 0 (another scheduler): A_w = A0 lam / sqrt(n) (Eq. 29) for n = 1..32
            // and the move's binary32 constants
            const double lam0 = __double_as_longlong(sh_carry) > 0 ? sh_carry : v.slot_lam[j];
            const int nn = tid - 31;
            const double aw = v.centring == 1 ? uniform_aw(v, lam0) : dvd(mul(v.A0, lam0), s_sqrt[nn]);
            sh_aw[nn] = aw;
            sh_awf[nn] = (float)aw;
            if (tid == 32) {
                sh_lamf = (float)lam0;
                for (int a = 0; a < 3; a++) sh_pf[a] = (float)v.slot_p[3 * j + a];
            }
        }
        __syncthreads();
        const double lam = sh_lam, lam2 = sh_lam2;
        const double b[3] = {sh_b[0], sh_b[1], sh_b[2]};
        {
            const float bx = sh_bf[0], by = sh_bf[1], bz = sh_bf[2];
            const float rl2 = sh_rl2, rR2 = sh_rR2;
            for (int m = tid; m < N; m += NT) {
                float dx = fx[m] - bx, dy = fy[m] - by, dz = fz[m] - bz;
                dx = fabsf(dx) > hLf ? dx - copysignf(Lf, dx) : dx;
                dy = fabsf(dy) > hLf ? dy - copysignf(Lf, dy) : dy;
                dz = fabsf(dz) > hLf ? dz - copysignf(Lf, dz) : dz;
                const float d2f = dx * dx + dy * dy + dz * dz;
                if (d2f > rR2) continue;
                bool in = false;
                if (d2f <= rl2) {
                    const unsigned am = __activemask();
                    double dd[3] = {sub(px[m], b[0]), sub(py[m], b[1]), sub(pz[m], b[2])};
                    mi3_u(dd, L, hL, am);
                    in = norm2(dd[0], dd[1], dd[2]) < lam2;
                }
                if (in) mid[atomicAdd(&sh_n, 1)] = m;
                else {
                    const int c = atomicAdd(&sh_nc, 1);
                    if (c < kSmemCand) s_cand[c] = m;
                }
            }
        }
        __syncthreads();
        const int n = sh_n;
        if (n == 0) {      // nothing inside: no motion, dU = 0 against the threshold
            if (tid == 0) {
                const bool acc0 = 0.0 <= v.slot_thr[j];
                att++;
                if (acc0) acc_n++;
                v.tr_out[Ly.tr_off + j] = (uint8_t)(acc0 ? 1 : 2);
                v.tr_n[Ly.tr_off + j] = 0;
                v.tr_du[Ly.tr_off + j] = 0.0;
                sh_carry = acc0 ? 0.0 : lam;
            }
            __syncthreads();
            continue;
        }
        // A_w and the binary32 constants: only in warps that hold a member
        double Aw = 0.0;
        float lamf = 0.0f, af = 0.0f, pf[3] = {0.0f, 0.0f, 0.0f};
        const double p[3] = {sh_p[0], sh_p[1], sh_p[2]};
        if ((tid & ~31) < n) {
            if (n <= 32) {
                Aw = sh_aw[n];
                af = sh_awf[n];
            } else {
                Aw = v.centring == 1 ? uniform_aw(v, lam) : dvd(mul(v.A0, lam), n <= kNCap ? s_sqrt[n] : sqr_t((double)n));
                af = (float)Aw;
            }
            lamf = sh_lamf; pf[0] = sh_pf[0]; pf[1] = sh_pf[1]; pf[2] = sh_pf[2];
        }
        for (int k = tid; k < n; k += NT) {
            const unsigned am = __activemask();
            const int m = mid[k];
            const double o[3] = {px[m], py[m], pz[m]};
            double d[3] = {sub(o[0], b[0]), sub(o[1], b[1]), sub(o[2], b[2])}, dl[3];
            mi3_u(d, L, hL, am);
            if (PREC == 0) wavelet_disp64(d, norm2(d[0], d[1], d[2]), lam, Aw, p, dl);
            else wavelet_disp32f(d, lamf, af, pf, dl);
            int im[3] = {0, 0, 0};
            const float oh[3] = {fx[m], fy[m], fz[m]}, ol[3] = {lx[m], ly[m], lz[m]};
            double nx[3] = {add(o[0], dl[0]), add(o[1], dl[1]), add(o[2], dl[2])};
            wrap3_u(nx, L, am, im);
            for (int a = 0; a < 3; a++) {
                mnew[3 * k + a] = nx[a];
                if (im[a] == 0) {
                    // old (hi, lo) plus the displacement by a binary32 two-sum, renormalised
                    const float dlf = (float)dl[a];
                    const float s1 = oh[a] + dlf, bb = s1 - oh[a];
                    const float l1 = ol[a] + ((oh[a] - (s1 - bb)) + (dlf - bb));
                    const float h2 = s1 + l1;
                    mnf[3 * k + a] = h2;
                    mnl[3 * k + a] = l1 - (h2 - s1);
                } else {                       // wrapped across a face: split the binary64 value
                    mnf[3 * k + a] = (float)mnew[3 * k + a];
                    mnl[3 * k + a] = (float)(mnew[3 * k + a] - (double)mnf[3 * k + a]);
                }
            }
            mimg[k] = (uint8_t)pack_img(im[0], im[1], im[2]);
            sslot[m] = (short)k;
        }
        __syncthreads();
        // the (member, bead) pairs of the WCA sums: each member against the candidates within
        // reach of the move and against the later members, or against every staged bead when
        // the candidate list overflowed; the same pairs pass the energy screens either way
        const int ncand = sh_nc;
        auto for_wca_pairs = [&](auto&& f) {
            if (ncand <= kSmemCand) {
                const int nl = ncand + n, total = n * nl;
                for (int t = tid; t < total; t += NT) {
                    const int k = t / nl, u = t - k * nl;
                    const int q = u < ncand ? s_cand[u] : mid[u - ncand];
                    const int m = mid[k];
                    const int sq = sslot[q];
                    if (q != m && !(sq >= 0 && q < m)) f(k, m, q, sq);
                }
            } else {
                const int total = n * N;
                int k = tid / N, q = tid - k * N;
                const int kstep = NT / N, qstep = NT - kstep * N;
                for (int t = tid; t < total; t += NT) {
                    const int m = mid[k];
                    const int sq = sslot[q];
                    if (q != m && !(sq >= 0 && q < m)) f(k, m, q, sq);
                    k += kstep;
                    q += qstep;
                    if (q >= N) { q -= N; k++; }
                }
            }
        };
        // energy change. Mixed precision: a binary32 pass (differences of the binary64
        // positions rounded once, then binary32 terms with their magnitudes) decides outside
        // the rigorous error band; inside it, and in binary64 mode, the binary64 pass decides.
        const double thr = v.slot_thr[j];
        bool need64 = PREC == 0;
        if (PREC == 1) {
            float a32 = 0.0f, m32 = 0.0f;
            int T = 0;
            auto r2f = [&](double ax, double ay, double az, double bx, double by, double bz) {
                const double e[3] = {sub(ax, bx), sub(ay, by), sub(az, bz)};
                float r2 = 0.0f;
                for (int a = 0; a < 3; a++) {
                    float f = (float)e[a];
                    if (fabsf(f) > hLf) f = (float)(e[a] > 0.0 ? sub(e[a], L) : add(e[a], L));
                    r2 += f * f;
                }
                return r2;
            };

            // squared distance between two staged points given as (hi, lo) binary32 pairs: the hi
            // difference is rounded once relative to the result and the lo parts add the rest, so
            // the difference carries about one ulp; a component across a face (the hi difference
            // beyond L/2, rare for pairs in range) is wrapped in binary64 from the positions
            auto comp = [&](float ha, float la, float hb, float lb, double xa, double xb) {
                const float dh = ha - hb;
                if (fabsf(dh) <= hLf) return dh + (la - lb);
                const double e = sub(xa, xb);
                return (float)(e > 0.0 ? sub(e, L) : add(e, L));
            };
            for (int k = tid; k < n; k += NT) {
                const int m = mid[k];
                const double o[3] = {px[m], py[m], pz[m]};
                const double nw[3] = {mnew[3 * k], mnew[3 * k + 1], mnew[3 * k + 2]};
                if (kappa_on) {
                    const float un = 0.5f * P32.kappa * r2f(nw[0], nw[1], nw[2], hL, hL, hL);
                    const float uo = 0.5f * P32.kappa * r2f(o[0], o[1], o[2], hL, hL, hL);
                    a32 += un - uo; m32 += un + uo; T += 2;
                }
                for (int e = 0; e < 2; e++) {
                    const int q = e ? m + 1 : m - 1;
                    if (q < 0 || q >= N || !(e ? bn[m] : bn[q])) continue;
                    const int sq = sslot[q];
                    if (sq >= 0 && q < m) continue;
                    const double qo[3] = {px[q], py[q], pz[q]};
                    const double qn[3] = {sq >= 0 ? mnew[3 * sq] : qo[0], sq >= 0 ? mnew[3 * sq + 1] : qo[1],
                                          sq >= 0 ? mnew[3 * sq + 2] : qo[2]};
                    const float qnh[3] = {sq >= 0 ? mnf[3 * sq] : fx[q], sq >= 0 ? mnf[3 * sq + 1] : fy[q],
                                          sq >= 0 ? mnf[3 * sq + 2] : fz[q]};
                    const float qnl[3] = {sq >= 0 ? mnl[3 * sq] : lx[q], sq >= 0 ? mnl[3 * sq + 1] : ly[q],
                                          sq >= 0 ? mnl[3 * sq + 2] : lz[q]};
                    const float ex = comp(mnf[3 * k], mnl[3 * k], qnh[0], qnl[0], nw[0], qn[0]);
                    const float ey = comp(mnf[3 * k + 1], mnl[3 * k + 1], qnh[1], qnl[1], nw[1], qn[1]);
                    const float ez = comp(mnf[3 * k + 2], mnl[3 * k + 2], qnh[2], qnl[2], nw[2], qn[2]);
                    const float gx_ = comp(fx[m], lx[m], fx[q], lx[q], o[0], qo[0]);
                    const float gy_ = comp(fy[m], ly[m], fy[q], ly[q], o[1], qo[1]);
                    const float gz_ = comp(fz[m], lz[m], fz[q], lz[q], o[2], qo[2]);
                    float un, mn, uo, mo;
                    bond32(P32, ex * ex + ey * ey + ez * ez, un, mn);
                    bond32(P32, gx_ * gx_ + gy_ * gy_ + gz_ * gz_, uo, mo);
                    a32 += un - uo; m32 += mn + mo; T += 2;
                }
            }
            if (eps_on) {
                for_wca_pairs([&](int k, int m, int q, int sq) {
                        const float qfx = fx[q], qfy = fy[q], qfz = fz[q];
                        float ax = fx[m] - qfx, ay = fy[m] - qfy, az = fz[m] - qfz;
                        ax = fabsf(ax) > hLf ? ax - copysignf(Lf, ax) : ax;
                        ay = fabsf(ay) > hLf ? ay - copysignf(Lf, ay) : ay;
                        az = fabsf(az) > hLf ? az - copysignf(Lf, az) : az;
                        const float qnx = sq >= 0 ? mnf[3 * sq] : qfx, qny = sq >= 0 ? mnf[3 * sq + 1] : qfy,
                                    qnz = sq >= 0 ? mnf[3 * sq + 2] : qfz;
                        float cx = mnf[3 * k] - qnx, cy = mnf[3 * k + 1] - qny, cz = mnf[3 * k + 2] - qnz;
                        cx = fabsf(cx) > hLf ? cx - copysignf(Lf, cx) : cx;
                        cy = fabsf(cy) > hLf ? cy - copysignf(Lf, cy) : cy;
                        cz = fabsf(cz) > hLf ? cz - copysignf(Lf, cz) : cz;
                        if (ax * ax + ay * ay + az * az <= rc2f || cx * cx + cy * cy + cz * cz <= rc2f) {
                            const double qo[3] = {px[q], py[q], pz[q]};
                            const double qn[3] = {sq >= 0 ? mnew[3 * sq] : qo[0], sq >= 0 ? mnew[3 * sq + 1] : qo[1],
                                                  sq >= 0 ? mnew[3 * sq + 2] : qo[2]};
                            const float qnl[3] = {sq >= 0 ? mnl[3 * sq] : lx[q], sq >= 0 ? mnl[3 * sq + 1] : ly[q],
                                                  sq >= 0 ? mnl[3 * sq + 2] : lz[q]};
                            const float ex = comp(mnf[3 * k], mnl[3 * k], qnx, qnl[0], mnew[3 * k], qn[0]);
                            const float ey = comp(mnf[3 * k + 1], mnl[3 * k + 1], qny, qnl[1], mnew[3 * k + 1], qn[1]);
                            const float ez = comp(mnf[3 * k + 2], mnl[3 * k + 2], qnz, qnl[2], mnew[3 * k + 2], qn[2]);
                            const float gx_ = comp(fx[m], lx[m], qfx, lx[q], px[m], qo[0]);
                            const float gy_ = comp(fy[m], ly[m], qfy, ly[q], py[m], qo[1]);
                            const float gz_ = comp(fz[m], lz[m], qfz, lz[q], pz[m], qo[2]);
                            float un, mn, uo, mo;
                            wca32(P32, ex * ex + ey * ey + ez * ez, un, mn);
                            wca32(P32, gx_ * gx_ + gy_ * gy_ + gz_ * gz_, uo, mo);
                            a32 += un - uo; m32 += mn + mo; T += 2;
                            if (sq < 0 && (un != 0.0f || uo != 0.0f)) pe++;
                        }
                });
            }
            for (int o = 16; o > 0; o >>= 1) {
                a32 += __shfl_xor_sync(0xffffffffu, a32, o);
                m32 += __shfl_xor_sync(0xffffffffu, m32, o);
                T = max(T, __shfl_xor_sync(0xffffffffu, T, o));
            }
            if (lane == 0) { sh_f32[wid] = a32; sh_m32[wid] = m32; sh_T[wid] = T; }
            __syncthreads();
            if (tid == 0) {
                float d32 = 0.0f, mm = 0.0f;
                int tt = 0;
                for (int w = 0; w < NT / 32; w++) { d32 += sh_f32[w]; mm += sh_m32[w]; tt = max(tt, sh_T[w]); }
                tt += 5 + NT / 32;     // summation depth: one thread's terms, the butterfly, the warp totals
                const float thr32 = (float)thr;
                const float band = 2.0f * (float)(80 + tt + 6) * 5.9604645e-08f * mm + 1e-9f * (float)v.kT +
                                   2.4e-7f * fabsf(thr32);
                sh_a32[0] = d32; sh_a32[1] = band; sh_a32[2] = thr32;
                if (isfinite(d32) && isfinite(band) && fabsf(d32 - thr32) > band) {
                    sh_acc = d32 <= thr32;
                    sh_need64 = v.audit ? 2 : 0;     // 2: the binary64 pass runs for the audit only
                    v.tr_du[Ly.tr_off + j] = (double)d32;
                } else {
                    sh_need64 = 1;
                    rechecks++;
                }
            }
            __syncthreads();
            need64 = sh_need64;
        }
        if (need64) {
            double dU = 0.0;
            for (int k = tid; k < n; k += NT) {
                const int m = mid[k];
                const double o[3] = {px[m], py[m], pz[m]};
                const double nw[3] = {mnew[3 * k], mnew[3 * k + 1], mnew[3 * k + 2]};
                dU += U_ext(P, nw[0], nw[1], nw[2]) - U_ext(P, o[0], o[1], o[2]);
                for (int e = 0; e < 2; e++) {
                    const int q = e ? m + 1 : m - 1;
                    if (q < 0 || q >= N || !(e ? bn[m] : bn[q])) continue;
                    const int sq = sslot[q];
                    if (sq >= 0 && q < m) continue;
                    const double qo[3] = {px[q], py[q], pz[q]};
                    const double qn[3] = {sq >= 0 ? mnew[3 * sq] : qo[0], sq >= 0 ? mnew[3 * sq + 1] : qo[1],
                                          sq >= 0 ? mnew[3 * sq + 2] : qo[2]};
                    const double r2n = norm2(mi(nw[0] - qn[0], L, hL), mi(nw[1] - qn[1], L, hL), mi(nw[2] - qn[2], L, hL));
                    const double r2o = norm2(mi(o[0] - qo[0], L, hL), mi(o[1] - qo[1], L, hL), mi(o[2] - qo[2], L, hL));
                    dU += U_bond(P, r2n) - U_bond(P, r2o);
                }
            }
            if (eps_on) {
                // one (member, bead) pair per thread and step, all members at once
                for_wca_pairs([&](int k, int m, int q, int sq) {
                        const float qfx = fx[q], qfy = fy[q], qfz = fz[q];
                        float ax = fx[m] - qfx, ay = fy[m] - qfy, az = fz[m] - qfz;
                        ax = fabsf(ax) > hLf ? ax - copysignf(Lf, ax) : ax;
                        ay = fabsf(ay) > hLf ? ay - copysignf(Lf, ay) : ay;
                        az = fabsf(az) > hLf ? az - copysignf(Lf, az) : az;
                        const float qnx = sq >= 0 ? mnf[3 * sq] : qfx, qny = sq >= 0 ? mnf[3 * sq + 1] : qfy,
                                    qnz = sq >= 0 ? mnf[3 * sq + 2] : qfz;
                        float cx = mnf[3 * k] - qnx, cy = mnf[3 * k + 1] - qny, cz = mnf[3 * k + 2] - qnz;
                        cx = fabsf(cx) > hLf ? cx - copysignf(Lf, cx) : cx;
                        cy = fabsf(cy) > hLf ? cy - copysignf(Lf, cy) : cy;
                        cz = fabsf(cz) > hLf ? cz - copysignf(Lf, cz) : cz;
                        if (ax * ax + ay * ay + az * az <= rc2f || cx * cx + cy * cy + cz * cz <= rc2f) {
                            const double o[3] = {px[m], py[m], pz[m]};
                            const double nw[3] = {mnew[3 * k], mnew[3 * k + 1], mnew[3 * k + 2]};
                            const double qo[3] = {px[q], py[q], pz[q]};
                            const double qn[3] = {sq >= 0 ? mnew[3 * sq] : qo[0], sq >= 0 ? mnew[3 * sq + 1] : qo[1],
                                                  sq >= 0 ? mnew[3 * sq + 2] : qo[2]};
                            const double r2n = norm2(mi(nw[0] - qn[0], L, hL), mi(nw[1] - qn[1], L, hL), mi(nw[2] - qn[2], L, hL));
                            const double r2o = norm2(mi(o[0] - qo[0], L, hL), mi(o[1] - qo[1], L, hL), mi(o[2] - qo[2], L, hL));
                            if (r2n < P.rc2 || r2o < P.rc2) {
                                dU += U_wca(P, r2n) - U_wca(P, r2o);
                                if (sq < 0 && PREC == 0) pe++;
                            }
                        }
                });
            }
            dU = warp_sum(dU);
            if (lane == 0) sh_red[wid] = dU;
            __syncthreads();
            if (tid == 0) {
                double su = 0.0;
                for (int w = 0; w < NT / 32; w++) su += sh_red[w];
                if (PREC == 1 && v.audit) audit_record(v, (double)sh_a32[0], (double)sh_a32[1], (double)sh_a32[2], su, thr);
                if (PREC == 0 || sh_need64 != 2) {
                    sh_acc = su <= thr;
                    v.tr_du[Ly.tr_off + j] = su;
                }
            }
            __syncthreads();
        }
        const bool acc = sh_acc;
        for (int k = tid; k < n; k += NT) {
            const int m = mid[k];
            if (acc) {
                px[m] = mnew[3 * k]; py[m] = mnew[3 * k + 1]; pz[m] = mnew[3 * k + 2];
                fx[m] = mnf[3 * k]; fy[m] = mnf[3 * k + 1]; fz[m] = mnf[3 * k + 2];
                lx[m] = mnl[3 * k]; ly[m] = mnl[3 * k + 1]; lz[m] = mnl[3 * k + 2];
                int dd[3];
                unpack_img(mimg[k], dd);
                dimg[3 * m] += (short)dd[0]; dimg[3 * m + 1] += (short)dd[1]; dimg[3 * m + 2] += (short)dd[2];
            }
            sslot[m] = -1;
        }
        if (tid == 0) {
            att++;
            bu += n;
            if (acc) { acc_n++; moved_n += n; }
            v.tr_out[Ly.tr_off + j] = (uint8_t)(acc ? 1 : 2);
            v.tr_n[Ly.tr_off + j] = n;
            sh_carry = acc ? 0.0 : lam;
        }
        __syncthreads();
    }
    // write back what moved; the cell lists go stale if a bead changed fine cell
    for (int m = tid; m < N; m += NT) {
        const Bead ob = v.bead[m];
        if (ob.x == px[m] && ob.y == py[m] && ob.z == pz[m]) continue;
        put_bead(v.bead, v.bf, m, px[m], py[m], pz[m]);
        if (dimg[3 * m] | dimg[3 * m + 1] | dimg[3 * m + 2]) {
            v.img[3 * m] += dimg[3 * m]; v.img[3 * m + 1] += dimg[3 * m + 1]; v.img[3 * m + 2] += dimg[3 * m + 2];
        }
        if (cell_lin(v, ob.x, ob.y, ob.z) != cell_lin(v, px[m], py[m], pz[m])) sh_stale = 1;
    }
    unsigned long long pe_all = (unsigned long long)pe;
    if (pe_all) atomicAdd(&v.ctr[C_PARTNER], pe_all);
    __syncthreads();
    if (tid == 0) {
        if (sh_stale) *v.cl_stale = 1;
        if (rechecks) atomicAdd(&v.ctr[C_RECHECK], (unsigned long long)rechecks);
        v.carry_serial[l] = sh_carry;
        atomicAdd(&v.ctr[C_ATT + l], (unsigned long long)att);
        atomicAdd(&v.ctr[C_ACC + l], (unsigned long long)acc_n);
        atomicAdd(&v.ctr[C_ACCTOT], (unsigned long long)acc_n);
        atomicAdd(&v.ctr[C_BU], (unsigned long long)bu);
        if (moved_n) atomicAdd(&v.ctr[C_MOVED], (unsigned long long)moved_n);
    }
}

size_t smem_serial_bytes(int64_t n) { return (size_t)n * (3 * 8 + 3 * 8 + 6 * 4 + 6 * 4 + 4 + 2 + 3 * 2 + 1 + 1) + 64; }

int launch_serial(const SimView* d, const GroupDims& g, int l, cudaStream_t s, const ForkJoin* fj) {
    const int np = (g.prec_mask & 1) + ((g.prec_mask >> 1) & 1);
    int launched = g.any_global_serial ? np : 0;
    prepare_staged(g);
    // one launch per precision; each returns at once for simulations of the other precision
    const dim3 grid(1, g.S);
    if (g.smem_maxN > 0) {
        // one launch per size class, each with the shared memory of its largest simulation, so
        // small simulations pack many blocks per SM; with side streams the classes run side by side
        int ncls = 0;
        for (int c = 0; c < 3; c++) ncls += g.smem_cls[c] > 0;
        const bool fork = fj && fj->side[0] && ncls > 1;
        if (fork) {
            cudaEventRecord(fj->fork, s);
            cudaStreamWaitEvent(fj->side[0], fj->fork, 0);
            cudaStreamWaitEvent(fj->side[1], fj->fork, 0);
        }
        for (int c = 2; c >= 0; c--) {
            if (!g.smem_cls[c]) continue;
            cudaStream_t cs = fork ? (c == 2 ? s : fj->side[c]) : s;
            const size_t sm = smem_serial_bytes(g.smem_cls[c]);
            const int64_t lo = c ? kSmemClassHi[c - 1] : 0, hi = kSmemClassHi[c];
            // threads per class: few for small simulations (several blocks share an SM), many
            // for large ones (one block per SM, whose warps must hide the latency of the scans)
            if (c == 0) {
                if (g.prec_mask & 1) k_serial_smem<0, 128><<<grid, 128, sm, cs>>>(d, l, lo, hi);
                if (g.prec_mask & 2) k_serial_smem<1, 128><<<grid, 128, sm, cs>>>(d, l, lo, hi);
            } else if (c == 1) {
                if (g.prec_mask & 1) k_serial_smem<0, 256><<<grid, 256, sm, cs>>>(d, l, lo, hi);
                if (g.prec_mask & 2) k_serial_smem<1, 256><<<grid, 256, sm, cs>>>(d, l, lo, hi);
            } else {
                if (g.prec_mask & 1) k_serial_smem<0, 512><<<grid, 512, sm, cs>>>(d, l, lo, hi);
                if (g.prec_mask & 2) k_serial_smem<1, 512><<<grid, 512, sm, cs>>>(d, l, lo, hi);
            }
            launched += np;
        }
        if (fork) {
            for (int c = 0; c < 2; c++) {
                cudaEventRecord(fj->join[c], fj->side[c]);
                cudaStreamWaitEvent(s, fj->join[c], 0);
            }
        }
    }
    if (!g.any_global_serial) return launched;
    if (g.smem_maxN > 0) {
        launch_cl_rebuild(d, g, s, 3 + l);
        launched += 3;
    }
    if (g.serial_threads <= 32) {
        if (g.prec_mask & 1) k_serial<0, 32><<<grid, 32, serial_dyn_bytes<0, 32>(), s>>>(d, l);
        if (g.prec_mask & 2) k_serial<1, 32><<<grid, 32, serial_dyn_bytes<1, 32>(), s>>>(d, l);
    } else if (g.serial_threads <= 128) {
        if (g.prec_mask & 1) k_serial<0, 128><<<grid, 128, serial_dyn_bytes<0, 128>(), s>>>(d, l);
        if (g.prec_mask & 2) k_serial<1, 128><<<grid, 128, serial_dyn_bytes<1, 128>(), s>>>(d, l);
    } else {
        if (g.prec_mask & 1) k_serial<0, 512><<<grid, 512, serial_dyn_bytes<0, 512>(), s>>>(d, l);
        if (g.prec_mask & 2) k_serial<1, 512><<<grid, 512, serial_dyn_bytes<1, 512>(), s>>>(d, l);
    }
    return launched;
}

}  // namespace wmcd

namespace wmcd {

// ======================================================================================
// Plane-wave moves (Sec. VI, Appendix D): every bead moves by A_F cos(k.r + Phi) e.
// setup (1 thread) -> displacements (grid) -> energy change (grid, per-block partials)
// -> decision (1 block, fixed-order sum) -> commit (grid) -> cell-list rebuild if moved.
// ======================================================================================
// direct = 0: the m-th plane-wave slot of the current sweep (active if m < the sweep's count);
// direct = 1: the m-th move of a direct call. The counter is the sweep or the call index.
// inverse of the tabulated |k| CDF for u in (0, 1): the largest i with F_i <= u, then F^(1/3)
// linear between Q_i and Q_{i+1}; beyond the table the Q^-1 tail of 1 - F
__device__ double k_inverse(const double* F, double u) {
    if (u >= F[kKtN]) return mul((double)kKtN * kKtH, dvd(sub(1.0, F[kKtN]), sub(1.0, u)));
    int lo = 0, hi = kKtN;                 // F[lo] <= u < F[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (F[mid] <= u) lo = mid; else hi = mid;
    }
    const double a = cbrt(F[lo]), b = cbrt(F[lo + 1]);
    return add(mul((double)lo, kKtH), mul(kKtH, dvd(sub(cbrt(u), a), sub(b, a))));
}
// a nonzero point of the unit ball by rejection (kind, counter and first attempt as given); the
// unit vector along it
__device__ void unit_by_rejection(const SimView& v, uint32_t kind, uint64_t ctr, uint32_t m, uint32_t a0,
                                  double kh[3]) {
    double V[3] = {0.0, 0.0, 1.0};
    for (uint32_t b = 0; b < 64; b++) {
        const u4 d = draw(v.k0, v.k1, kind, 0, ctr, m, a0 + b);
        const double x = sym(d.x), y = sym(d.y), z = sym(d.z), q = norm2(x, y, z);
        if (q <= 1.0 && q > 0.0) { V[0] = x; V[1] = y; V[2] = z; break; }
    }
    const double r = sqr_t(norm2(V[0], V[1], V[2]));
    for (int c = 0; c < 3; c++) kh[c] = dvd(V[c], r);
}
// Fresh wave vector (Appendix D): the infinite system's |k| from the table and an isotropic
// direction; the quasi-continuous shell's snapped mode outside the discrete cube (up to 64
// attempts, the last standing); otherwise a mode of the table by its cumulative probability.
__device__ void pw_fresh_k(const SimView& v, uint32_t kshell, uint32_t kkdir, uint64_t ctr, uint32_t m, const u4& w1,
                           int lv[3], double kh[3], double* Q) {
    const double u_mode = u53(w1.x, w1.y);
    if (v.pw_mode == 3) {
        *Q = k_inverse(v.kF, u_open(w1.x, w1.y));
        unit_by_rejection(v, kkdir, ctr, m, 0u, kh);
        return;
    }
    if (v.pw_mode == 2 && !(u_mode < v.p_disc)) {
        const double lmax = v.layer[v.nL - 1].hi;
        for (uint32_t a = 0; a < 64; a++) {
            const u4 w = draw(v.k0, v.k1, kshell, 0, ctr, m, a);
            const double us = u_open(w.x, w.y);
            const double q = k_inverse(v.kF, add(v.kF0, mul(us, sub(1.0, v.kF0))));
            double d[3];
            unit_by_rejection(v, kkdir, ctr, m, 64u * a, d);
            const double sc = dvd(mul(q, v.L), mul(kTwoPi, lmax));
            int inside = 1;
            for (int c = 0; c < 3; c++) {
                lv[c] = (int)floor(add(mul(sc, d[c]), 0.5));
                if (abs(lv[c]) > v.pw_nl) inside = 0;
            }
            if (!inside) return;
        }
        return;
    }
    int lo = 0, hi = v.n_modes - 1;           // first mode with u < cdf
    while (lo < hi) { int mid = (lo + hi) >> 1; if (u_mode < v.mode_cdf[mid]) hi = mid; else lo = mid + 1; }
    for (int a = 0; a < 3; a++) lv[a] = v.modes[3 * lo + a];
}

__global__ void k_pw_setup(const SimView* __restrict__ vs, int direct, int m) {
    SIM_PROLOGUE
    if (threadIdx.x != 0) return;
    PWDev& P = *v.pw;
    *v.pw_rebuild = 0;
    P.active = direct ? 1 : (v.pw_on && m < v.counts[kMaxLayers]);
    if (!P.active) return;
    const uint64_t ctr = v.step[direct ? 1 : 0];
    const int kmode = direct ? K_DPWMODE : K_PWMODE, kdir = direct ? K_DPWDIR : K_PWDIR;
    const uint32_t kshell = direct ? K_DPWSHELL : K_PWSHELL, kkdir = direct ? K_DPWKDIR : K_PWKDIR;
    const bool cont = v.pw_mode == 3;
    const int trace_index = m;
    u4 w1 = draw(v.k0, v.k1, (uint32_t)kmode, 0, ctr, (uint32_t)m, 0);
    u4 w2 = draw(v.k0, v.k1, (uint32_t)kdir, 0, ctr, (uint32_t)m, 0);
    const double phi = u53(w1.z, w1.w), psi = u53(w2.x, w2.y);
    const int perm = (int)(((uint64_t)w2.z * 6u) >> 32);
    const uint32_t signs = w2.w & 7u;
    const int PERM[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
    int lv[3] = {0, 0, 0};
    double kh[3] = {0.0, 0.0, 1.0}, Q = 0.0;
    if (P.carry && !cont) {
        // recycle |k| after a rejection: permute the components, flip each sign with prob 1/2
        for (int a = 0; a < 3; a++) {
            int x = P.carry_l[PERM[perm][a]];
            lv[a] = ((signs >> a) & 1u) ? -x : x;
        }
    } else {
        pw_fresh_k(v, kshell, kkdir, ctr, (uint32_t)m, w1, lv, kh, &Q);
        if (P.carry && cont) Q = P.carry_Q;     // the same |k|, a new direction
    }
    const double lmax = v.layer[v.nL - 1].hi;
    for (int a = 0; a < 3; a++) P.lv[a] = lv[a];
    P.cont = cont;
    P.Q = Q;
    const bool fits = abs(lv[0]) <= 127 && abs(lv[1]) <= 127 && abs(lv[2]) <= 127;
    P.mode_packed = (cont || !fits) ? -1 : (lv[0] + 128) | ((lv[1] + 128) << 8) | ((lv[2] + 128) << 16);
    P.phi = phi;
    P.null_move = !cont && (lv[0] == 0 && lv[1] == 0 && lv[2] == 0);
    P.accept = 0;
    atomicAdd(&v.ctr[C_PWATT], 1ull);
    if (trace_index >= 0 && trace_index < v.tr_pw_cap) {
        v.tr_pw_mode[trace_index] = P.mode_packed;
        const double sc = cont ? dvd(mul(Q, v.L), mul(kTwoPi, lmax)) : 0.0;
        for (int a = 0; a < 3; a++) v.tr_pw_k[3 * trace_index + a] = cont ? mul(sc, kh[a]) : (double)lv[a];
    }
    if (P.null_move) {
        // k = 0 moves nothing and is accepted (Sec. VI.A)
        P.accept = 1;
        P.carry = 0;
        atomicAdd(&v.ctr[C_PWACC], 1ull);
        atomicAdd(&v.ctr[C_ACCTOT], 1ull);
        if (trace_index >= 0 && trace_index < v.tr_pw_cap) v.tr_pw_out[trace_index] = 1;
        return;
    }
    double u1[3], u2[3];
    if (cont) {
        // infinite system: A_F = (2/k) sqrt(dU_est/(mu N)) with k = Q / lambda_max (Eq. 48), the
        // polarisation about the continuous direction kh, the phase in turns per unit length
        const double kmag = dvd(Q, lmax);
        P.AF = dvd(mul(2.0, v.A0), mul(kmag, sqr_t(mul(5.0, (double)v.N))));
        P.kappa = dvd(Q, mul(kTwoPi, lmax));
        for (int a = 0; a < 3; a++) P.kh[a] = kh[a];
        if (kh[0] == 0.0 && kh[1] == 0.0) { u1[0] = 1.0; u1[1] = 0.0; u1[2] = 0.0; }
        else {
            const double nr = sqr_t(add(mul(kh[0], kh[0]), mul(kh[1], kh[1])));
            u1[0] = dvd(kh[1], nr); u1[1] = dvd(-kh[0], nr); u1[2] = 0.0;
        }
    } else {
        // A_F = (2/k) sqrt(dU_est/(mu N)), dU_est/mu = M6 A0^2/(2 pi)^3 = A0^2/5 (Eq. 48)
        const int l2 = lv[0] * lv[0] + lv[1] * lv[1] + lv[2] * lv[2];
        const double lm = sqr_t((double)l2);
        const double kmag = dvd(mul(kTwoPi, lm), v.L);
        P.AF = dvd(mul(2.0, v.A0), mul(kmag, sqr_t(mul(5.0, (double)v.N))));
        // polarisation e perpendicular to k: e = cos(psi) u1 + sin(psi) u2, u1 = k x z / |k x z|
        kh[0] = dvd((double)lv[0], lm); kh[1] = dvd((double)lv[1], lm); kh[2] = dvd((double)lv[2], lm);
        if (lv[0] == 0 && lv[1] == 0) { u1[0] = 1.0; u1[1] = 0.0; u1[2] = 0.0; }
        else {
            double nr = sqr_t((double)(lv[0] * lv[0] + lv[1] * lv[1]));
            u1[0] = dvd((double)lv[1], nr); u1[1] = dvd((double)(-lv[0]), nr); u1[2] = 0.0;
        }
    }
    u2[0] = sub(mul(kh[1], u1[2]), mul(kh[2], u1[1]));
    u2[1] = sub(mul(kh[2], u1[0]), mul(kh[0], u1[2]));
    u2[2] = sub(mul(kh[0], u1[1]), mul(kh[1], u1[0]));
    const double cp = cos2pi(psi), sp = sin2pi(psi);
    for (int a = 0; a < 3; a++) P.e[a] = add(mul(cp, u1[a]), mul(sp, u2[a]));
    P.reach = v.rc + 2.0 * fabs(P.AF) + 1e-9;
}

__global__ void k_pw_disp(const SimView* __restrict__ vs) {
    SIM_EXIT_IF(!gv.pw->active || gv.pw->null_move)
    SIM_PROLOGUE
    const PWDev& P = *v.pw;
    if (!P.active || P.null_move) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) *v.cl_stale = 0;   // rebuilt just before, if it was stale
    const double lx = (double)P.lv[0], ly = (double)P.lv[1], lz = (double)P.lv[2];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < v.N; i += (int64_t)gridDim.x * blockDim.x) {
        const Bead b = v.bead[i];
        const double r[3] = {b.x, b.y, b.z};
        double t;
        if (P.cont) {
            // infinite system: the field at the unwrapped position
            double X[3];
            for (int a = 0; a < 3; a++) X[a] = add(r[a], mul((double)v.img[3 * i + a], v.L));
            t = add(mul(P.kappa, add(add(mul(P.kh[0], X[0]), mul(P.kh[1], X[1])), mul(P.kh[2], X[2]))), P.phi);
        } else {
            t = add(dvd(add(add(mul(lx, r[0]), mul(ly, r[1])), mul(lz, r[2])), v.L), P.phi);
        }
        double dl[3];
        if (v.precision == 0) {
            const double amp = mul(P.AF, cos2pi(t));
            for (int a = 0; a < 3; a++) dl[a] = mul(amp, P.e[a]);
        } else {
            const float amp = mulf((float)P.AF, cos2pi_f(t));
            for (int a = 0; a < 3; a++) dl[a] = (double)mulf(amp, (float)P.e[a]);
        }
        int im[3] = {0, 0, 0};
        for (int a = 0; a < 3; a++) v.pw_new[3 * i + a] = wrap(add(r[a], dl[a]), v.L, &im[a]);
        v.pw_imgd[i] = pack_img(im[0], im[1], im[2]);
    }
}

__global__ void __launch_bounds__(256) k_pw_energy(const SimView* __restrict__ vs) {
    SIM_EXIT_IF(!gv.pw->active || (int)blockIdx.x >= gv.pw_blocks)
    SIM_PROLOGUE
    __shared__ double red[8];
    const PWDev& P = *v.pw;
    if (!P.active || blockIdx.x >= v.pw_blocks) return;
    double dU = 0.0;
    long long pe = 0;
    if (!P.null_move) {
        const double L = v.L, hL = v.halfL;
        const Pot& Po = v.pot;
        const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
        if (i < v.N) {
            const Bead b = v.bead[i];
            const double o[3] = {b.x, b.y, b.z};
            const double nw[3] = {v.pw_new[3 * i], v.pw_new[3 * i + 1], v.pw_new[3 * i + 2]};
            dU += U_ext(Po, nw[0], nw[1], nw[2]) - U_ext(Po, o[0], o[1], o[2]);
            if (i + 1 < v.N && v.bnext[i]) {
                const Bead c = v.bead[i + 1];
                const double* cn = &v.pw_new[3 * (i + 1)];
                double r2n = norm2(mi(nw[0] - cn[0], L, hL), mi(nw[1] - cn[1], L, hL), mi(nw[2] - cn[2], L, hL));
                double r2o = norm2(mi(o[0] - c.x, L, hL), mi(o[1] - c.y, L, hL), mi(o[2] - c.z, L, hL));
                dU += U_bond(Po, r2n) - U_bond(Po, r2o);
            }
            if (Po.eps != 0.0) {
                double lo[3], hi[3];
                for (int a = 0; a < 3; a++) { lo[a] = sub(o[a], P.reach); hi[a] = add(o[a], P.reach); }
                int c0[3], nc[3];
                cell_box(v, lo, hi, c0, nc);
                const int ncell = nc[0] * nc[1] * nc[2];
                for (int k = 0; k < ncell; k++) {
                    int guard = 0;
                    for (int q = v.head[box_cell(v, c0, nc, k)]; q >= 0;) {
                        const Bead bq = v.bead[q];
                        if (q > i) {
                            const double* qn = &v.pw_new[3 * (int64_t)q];
                            double r2n = norm2(mi(nw[0] - qn[0], L, hL), mi(nw[1] - qn[1], L, hL), mi(nw[2] - qn[2], L, hL));
                            double r2o = norm2(mi(o[0] - bq.x, L, hL), mi(o[1] - bq.y, L, hL), mi(o[2] - bq.z, L, hL));
                            if (r2n < Po.rc2 || r2o < Po.rc2) { dU += U_wca(Po, r2n) - U_wca(Po, r2o); pe++; }
                        }
                        q = bq.next;
                        if (++guard > kMaxWalk) { set_err(v, E_WALK); break; }
                    }
                }
            }
        }
    }
    dU = warp_sum(dU);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = dU;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < 8; w++) s += red[w];
        v.pw_part[blockIdx.x] = s;
    }
    if (pe) atomicAdd(&v.ctr[C_PARTNER], (unsigned long long)pe);
}

__global__ void __launch_bounds__(256) k_pw_decide(const SimView* __restrict__ vs, int direct, int m) {
    SIM_EXIT_IF(!gv.pw->active || gv.pw->null_move)
    SIM_PROLOGUE
    __shared__ double red[8];
    PWDev& P = *v.pw;
    if (!P.active || P.null_move) return;
    const uint64_t ctr = v.step[direct ? 1 : 0];
    const int kacc = direct ? K_DPWACC : K_PWACC;
    const int trace_index = m;
    double s = 0.0;
    for (int b = threadIdx.x; b < v.pw_blocks; b += 256) s += v.pw_part[b];
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x != 0) return;
    double dU = 0.0;
    for (int w = 0; w < 8; w++) dU += red[w];
    u4 w = draw(v.k0, v.k1, (uint32_t)kacc, 0, ctr, (uint32_t)m, 0);
    const double thr = accept_threshold(v, w);
    const bool acc = dU <= thr;
    P.accept = acc;
    atomicAdd(&v.ctr[C_BU], (unsigned long long)v.N);
    if (acc) {
        P.carry = 0;
        atomicAdd(&v.ctr[C_PWACC], 1ull);
        atomicAdd(&v.ctr[C_ACCTOT], 1ull);
        atomicAdd(&v.ctr[C_MOVED], (unsigned long long)v.N);
    } else {
        P.carry = 1;
        for (int a = 0; a < 3; a++) P.carry_l[a] = P.lv[a];
        P.carry_Q = P.Q;
    }
    if (trace_index >= 0 && trace_index < v.tr_pw_cap) v.tr_pw_out[trace_index] = (uint8_t)(acc ? 1 : 2);
}

__global__ void k_pw_commit(const SimView* __restrict__ vs) {
    SIM_EXIT_IF(!(gv.pw->active && gv.pw->accept && !gv.pw->null_move))
    SIM_PROLOGUE
    const PWDev& P = *v.pw;
    const bool moved = P.active && P.accept && !P.null_move;
    if (blockIdx.x == 0 && threadIdx.x == 0) *v.pw_rebuild = moved;
    if (!moved) return;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < v.N; i += (int64_t)gridDim.x * blockDim.x) {
        put_bead(v.bead, v.bf, i, v.pw_new[3 * i], v.pw_new[3 * i + 1], v.pw_new[3 * i + 2]);
        const int pk = v.pw_imgd[i];
        if (pk != pack_img(0, 0, 0)) {
            int dd[3];
            unpack_img(pk, dd);
            v.img[3 * i] += dd[0]; v.img[3 * i + 1] += dd[1]; v.img[3 * i + 2] += dd[2];
        }
    }
}

int launch_planewave(const SimView* d, const GroupDims& g, int direct, int m, cudaStream_t s) {
    const int nb = g.pw_blocks;
    const int gb = (int)gx(nb, g.S);
    k_pw_setup<<<dim3(1, g.S), 32, 0, s>>>(d, direct, m);
    launch_cl_rebuild(d, g, s, 2);
    k_pw_disp<<<dim3(gb, g.S), 256, 0, s>>>(d);
    k_pw_energy<<<dim3(nb, g.S), 256, 0, s>>>(d);
    k_pw_decide<<<dim3(1, g.S), 256, 0, s>>>(d, direct, m);
    k_pw_commit<<<dim3(gb, g.S), 256, 0, s>>>(d);
    launch_cl_rebuild(d, g, s, 1);
    return 11;
}

}  // namespace wmcd

namespace wmcd {

// ======================================================================================
// Serial moves of a large-scale layer on the whole GPU (Sec. VIII: a single large wavelet
// move executed in parallel). One move is a short sequence of launches over all beads or
// all support members: centre and slot parameters (one thread), support by a scan of all
// beads, displacements, energy change with per-block partial sums, the decision (fixed-order
// sum of the partials), the commit, and a cell-list rebuild if the move was accepted. The
// arithmetic of every step is that of the one-block serial kernel, so decisions agree.
// ======================================================================================
__global__ void k_big_setup(const SimView* __restrict__ vs, int l, int t) {
    SIM_PROLOGUE
    if (threadIdx.x != 0) return;
    *v.pw_rebuild = 0;                          // every simulation: the rebuild below is only for this move
    if (l >= v.nL || !((v.big_layers >> l) & 1)) return;
    BigMove& B = *v.big;
    B.active = t < v.counts[l];
    if (!B.active) return;
    const int j = t;
    const double carry = v.carry_serial[l];
    const double lam = carry > 0.0 ? carry : v.slot_lam[j];
    const Bead bi = v.bead[v.slot_bead[j]];
    const double ri[3] = {bi.x, bi.y, bi.z};
    for (int a = 0; a < 3; a++) {
        B.b[a] = v.centring == 1 ? v.slot_V[3 * j + a] : wrap(add(ri[a], mul(lam, v.slot_V[3 * j + a])), v.L, nullptr);
        B.p[a] = v.slot_p[3 * j + a];
    }
    B.lam = lam;
    B.j = j;
    B.thr = v.slot_thr[j];
    B.n = 0;
    B.acc = 0;
    B.nch = 0;
    uint32_t tag = *v.serial_tag + 1u;
    if (tag == 0u) tag = 1u;
    *v.serial_tag = tag;
    B.tag = tag;
}

// support: every bead strictly inside the ball (minimum image), in no particular order
__global__ void k_big_gather(const SimView* __restrict__ vs, int l) {
    SIM_EXIT_IF(l >= gv.nL || !((gv.big_layers >> l) & 1) || !gv.big->active)
    SIM_PROLOGUE
    BigMove* B = v.big;
    const double b[3] = {B->b[0], B->b[1], B->b[2]};
    const double lam = B->lam, lam2 = mul(lam, lam);
    const double L = v.L, hL = v.halfL;
    for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < v.N; m += (int64_t)gridDim.x * blockDim.x) {
        const Bead bb = v.bead[m];
        const double d0 = mi(sub(bb.x, b[0]), L, hL), d1 = mi(sub(bb.y, b[1]), L, hL), d2c = mi(sub(bb.z, b[2]), L, hL);
        const double d2 = norm2(d0, d1, d2c);
        if (d2 < lam2) {
            const int idx = atomicAdd(&B->n, 1);
            v.s_ids[idx] = (int)m;
            v.s_d[4 * idx] = d0; v.s_d[4 * idx + 1] = d1; v.s_d[4 * idx + 2] = d2c; v.s_d[4 * idx + 3] = d2;
        }
    }
}

__global__ void k_big_disp(const SimView* __restrict__ vs, int l) {
    SIM_EXIT_IF(l >= gv.nL || !((gv.big_layers >> l) & 1) || !gv.big->active || gv.big->n == 0)
    SIM_PROLOGUE
    const BigMove& B = *v.big;
    const int n = B.n;
    const double lam = B.lam;
    const double Aw = v.centring == 1 ? uniform_aw(v, lam) : dvd(mul(v.A0, lam), sqr_t((double)n));
    const double p[3] = {B.p[0], B.p[1], B.p[2]};
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const int m = v.s_ids[k];
        v.bead[m].mark = B.tag;
        v.s_slot[m] = k;
        double d[3] = {v.s_d[4 * k], v.s_d[4 * k + 1], v.s_d[4 * k + 2]}, dl[3];
        if (v.precision == 0) wavelet_disp64(d, v.s_d[4 * k + 3], lam, Aw, p, dl);
        else wavelet_disp32(d, lam, Aw, p, dl);
        const Bead bm = v.bead[m];
        const double o[3] = {bm.x, bm.y, bm.z};
        int im[3] = {0, 0, 0};
        for (int a = 0; a < 3; a++) {
            v.s_new[3 * k + a] = wrap(add(o[a], dl[a]), v.L, &im[a]);
            v.s_d[4 * k + a] = dl[a];          // the displacement, for the partner box
        }
        v.s_img[k] = pack_img(im[0], im[1], im[2]);
    }
}

// energy change, one thread per member: external well, bonds, WCA with every bead in the
// member's partner box; per-block partial sums in pw_part
__global__ void __launch_bounds__(256) k_big_energy(const SimView* __restrict__ vs, int l) {
    SIM_EXIT_IF(l >= gv.nL || !((gv.big_layers >> l) & 1) || !gv.big->active ||
                (int)(blockIdx.x * blockDim.x) >= gv.big->n)
    SIM_PROLOGUE
    __shared__ double red[8];
    const BigMove& B = *v.big;
    const int n = B.n;
    const uint32_t tag = B.tag;
    const double L = v.L, hL = v.halfL;
    const Pot& P = v.pot;
    const double Aw = v.centring == 1 ? uniform_aw(v, B.lam) : dvd(mul(v.A0, B.lam), sqr_t((double)n));
    const double ext = add(v.rc, mul(0.25, Aw)) + 1e-9;
    double dU = 0.0;
    long long pe = 0;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) {
        const int m = v.s_ids[k];
        const Bead bm = v.bead[m];
        const double o[3] = {bm.x, bm.y, bm.z};
        const double nw[3] = {v.s_new[3 * k], v.s_new[3 * k + 1], v.s_new[3 * k + 2]};
        dU += U_ext(P, nw[0], nw[1], nw[2]) - U_ext(P, o[0], o[1], o[2]);
        for (int e = 0; e < 2; e++) {
            const int q = e ? m + 1 : m - 1;
            if (q < 0 || q >= v.N || !(e ? v.bnext[m] : v.bnext[q])) continue;
            const Bead bq = v.bead[q];
            double qn[3] = {bq.x, bq.y, bq.z};
            if (bq.mark == tag) {
                if (q < m) continue;
                const int sq = v.s_slot[q];
                qn[0] = v.s_new[3 * sq]; qn[1] = v.s_new[3 * sq + 1]; qn[2] = v.s_new[3 * sq + 2];
            }
            const double r2n = norm2(mi(nw[0] - qn[0], L, hL), mi(nw[1] - qn[1], L, hL), mi(nw[2] - qn[2], L, hL));
            const double r2o = norm2(mi(o[0] - bq.x, L, hL), mi(o[1] - bq.y, L, hL), mi(o[2] - bq.z, L, hL));
            dU += U_bond(P, r2n) - U_bond(P, r2o);
        }
        if (P.eps != 0.0) {
            double lo[3], hi[3];
            for (int a = 0; a < 3; a++) {
                const double u = add(o[a], v.s_d[4 * k + a]);
                lo[a] = sub(fmin(o[a], u), ext);
                hi[a] = add(fmax(o[a], u), ext);
            }
            int c0[3], nc[3];
            cell_box(v, lo, hi, c0, nc);
            const int ncell = nc[0] * nc[1] * nc[2];
            for (int kk = 0; kk < ncell; kk++) {
                int guard = 0;
                for (int q = v.head[box_cell(v, c0, nc, kk)]; q >= 0;) {
                    const Bead bq = v.bead[q];
                    const int nx = bq.next;
                    if (q != m) {
                        const bool member = bq.mark == tag;
                        if (!(member && q < m)) {
                            double qn[3] = {bq.x, bq.y, bq.z};
                            if (member) {
                                const int sq = v.s_slot[q];
                                qn[0] = v.s_new[3 * sq]; qn[1] = v.s_new[3 * sq + 1]; qn[2] = v.s_new[3 * sq + 2];
                            }
                            const double r2n = norm2(mi(nw[0] - qn[0], L, hL), mi(nw[1] - qn[1], L, hL), mi(nw[2] - qn[2], L, hL));
                            const double r2o = norm2(mi(o[0] - bq.x, L, hL), mi(o[1] - bq.y, L, hL), mi(o[2] - bq.z, L, hL));
                            if (r2n < P.rc2 || r2o < P.rc2) { dU += U_wca(P, r2n) - U_wca(P, r2o); if (!member) pe++; }
                        }
                    }
                    q = nx;
                    if (++guard > kMaxWalk) { set_err(v, E_WALK); break; }
                }
            }
        }
    }
    dU = warp_sum(dU);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = dU;
    __syncthreads();
    if (threadIdx.x == 0) {
        double su = 0.0;
        for (int w = 0; w < 8; w++) su += red[w];
        v.pw_part[blockIdx.x] = su;
    }
    if (pe) atomicAdd(&v.ctr[C_PARTNER], (unsigned long long)pe);
}

// decision: the partials of the blocks that held members, summed in a fixed order
__global__ void __launch_bounds__(256) k_big_decide(const SimView* __restrict__ vs, int l) {
    SIM_EXIT_IF(l >= gv.nL || !((gv.big_layers >> l) & 1) || !gv.big->active)
    SIM_PROLOGUE
    __shared__ double red[8];
    BigMove& B = *v.big;
    const int n = B.n;
    const int nb = (n + 255) / 256;
    double su = 0.0;
    for (int b = threadIdx.x; b < nb; b += 256) su += v.pw_part[b];
    su = warp_sum(su);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = su;
    __syncthreads();
    if (threadIdx.x != 0) return;
    double dU = 0.0;
    for (int w = 0; w < 8; w++) dU += red[w];
    const LayerDev& Ly = v.layer[l];
    const bool acc = (n == 0 ? 0.0 : dU) <= B.thr;   // an empty support moves nothing: dU = 0
    B.acc = acc;
    v.tr_out[Ly.tr_off + B.j] = (uint8_t)(acc ? 1 : 2);
    v.tr_n[Ly.tr_off + B.j] = n;
    v.tr_du[Ly.tr_off + B.j] = n == 0 ? 0.0 : dU;
    v.carry_serial[l] = acc ? 0.0 : B.lam;
    atomicAdd(&v.ctr[C_ATT + l], 1ull);
    atomicAdd(&v.ctr[C_BU], (unsigned long long)n);
    if (acc) {
        atomicAdd(&v.ctr[C_ACC + l], 1ull);
        atomicAdd(&v.ctr[C_ACCTOT], 1ull);
        if (n) atomicAdd(&v.ctr[C_MOVED], (unsigned long long)n);
    }
}

__global__ void k_big_commit(const SimView* __restrict__ vs, int l) {
    SIM_EXIT_IF(l >= gv.nL || !((gv.big_layers >> l) & 1) || !gv.big->active || !gv.big->acc || gv.big->n == 0)
    SIM_PROLOGUE
    const int n = v.big->n;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const int m = v.s_ids[k];
        const Bead ob = v.bead[m];
        const int oc = cell_lin(v, ob.x, ob.y, ob.z), ncl = cell_lin(v, v.s_new[3 * k], v.s_new[3 * k + 1], v.s_new[3 * k + 2]);
        if (oc != ncl) {
            // the cell changes, relinked next (or, beyond what one block relinks, a rebuild)
            const int idx = atomicAdd(&v.big->nch, 1);
            v.s_changed[3 * idx] = m; v.s_changed[3 * idx + 1] = oc; v.s_changed[3 * idx + 2] = ncl;
        }
        put_bead(v.bead, v.bf, m, v.s_new[3 * k], v.s_new[3 * k + 1], v.s_new[3 * k + 2]);
        const int pk = v.s_img[k];
        if (pk != pack_img(0, 0, 0)) {
            int dd[3];
            unpack_img(pk, dd);
            v.img[3 * m] += dd[0]; v.img[3 * m + 1] += dd[1]; v.img[3 * m + 2] += dd[2];
        }
    }
}

// the cell changes of an accepted whole-GPU move relinked by one block, or (more than it holds,
// or lists left stale) the cell lists rebuilt by the launches after it
constexpr int kBigRelinkCap = 3072;
__global__ void __launch_bounds__(1024) k_big_relink(const SimView* __restrict__ vs, int l) {
    SIM_EXIT_IF(l >= gv.nL || !((gv.big_layers >> l) & 1) || !gv.big->active || !gv.big->acc || gv.big->n == 0)
    SIM_PROLOGUE
    const int nch = v.big->nch;
    // lists a shared-memory serial phase left stale cannot be relinked: rebuilt instead
    if (nch > kBigRelinkCap || *v.cl_stale) {
        if (threadIdx.x == 0) *v.pw_rebuild = 1;
        return;
    }
    __shared__ int cm[kBigRelinkCap], co[kBigRelinkCap], cn[kBigRelinkCap];
    for (int c = threadIdx.x; c < nch; c += blockDim.x) {
        cm[c] = v.s_changed[3 * c]; co[c] = v.s_changed[3 * c + 1]; cn[c] = v.s_changed[3 * c + 2];
    }
    __syncthreads();
    grouped_relink(v, cm, co, cn, nch, threadIdx.x, blockDim.x);
}
int launch_big(const SimView* d, const GroupDims& g, int l, int t, cudaStream_t s) {
    const int gb = (int)gx((g.maxN + 255) / 256, g.S);
    k_big_setup<<<dim3(1, g.S), 32, 0, s>>>(d, l, t);
    k_big_gather<<<dim3(gb, g.S), 256, 0, s>>>(d, l);
    k_big_disp<<<dim3(gb, g.S), 256, 0, s>>>(d, l);
    k_big_energy<<<dim3(g.pw_blocks, g.S), 256, 0, s>>>(d, l);
    k_big_decide<<<dim3(1, g.S), 256, 0, s>>>(d, l);
    k_big_commit<<<dim3(gb, g.S), 256, 0, s>>>(d, l);
    k_big_relink<<<dim3(1, g.S), 1024, 0, s>>>(d, l);
    launch_cl_rebuild(d, g, s, 1);
    return 10;
}

}  // namespace wmcd

namespace wmcd {

// ======================================================================================
// Staged concurrent wavelet moves. In a colour phase every queue owns the beads in the fine
// cells wholly inside its region (no other queue reads or writes them), so its warp copies
// them into shared memory once, runs all its moves there and writes them back at the end.
// Beads are assigned to regions by a counting sort over all beads before each colour phase.
// ======================================================================================
// With at most kRegionPriv queues per colour (coarse layers, whose regions hold thousands of
// beads each) the counts are kept per block in shared memory and added to the global ones once
// per block and queue: one global counter per queue would otherwise take an atomic per bead.
constexpr int kRegionPriv = 8192;
__global__ void k_region_count(const SimView* __restrict__ vs, int l, int colour) {
    SIM_EXIT_IF(!sched_on(gv, l) || colour >= gv.K * gv.K * gv.K)
    SIM_PROLOGUE
    if (!sched_on(v, l) || colour >= v.K * v.K * v.K) return;
    const int K = v.K, Gf = v.Gf, Q = sched_layer(v, l).G / K, nq = Q * Q * Q;
    const int ox = colour % K, oy = (colour / K) % K, oz = colour / (K * K);
    const int* tab = v.axis_tab + (size_t)l * K * Gf;
    __shared__ int sh[kRegionPriv];
    const bool priv = nq <= kRegionPriv;
    if (priv) {
        for (int i = threadIdx.x; i < nq; i += blockDim.x) sh[i] = 0;
        __syncthreads();
    }
    for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < v.N; m += (int64_t)gridDim.x * blockDim.x) {
        const Bead b = v.bead[m];
        const int qx = tab[ox * Gf + fine_cell(b.x, v.invf, Gf)];
        const int qy = tab[oy * Gf + fine_cell(b.y, v.invf, Gf)];
        const int qz = tab[oz * Gf + fine_cell(b.z, v.invf, Gf)];
        const int key = (qx < 0 || qy < 0 || qz < 0) ? -1 : qx + Q * (qy + Q * qz);
        v.rkey[m] = key;
        if (key >= 0) atomicAdd(priv ? &sh[key] : &v.rcount[key], 1);
    }
    if (priv) {
        __syncthreads();
        for (int i = threadIdx.x; i < nq; i += blockDim.x)
            if (sh[i]) atomicAdd(&v.rcount[i], sh[i]);
    }
}
// Bead ids grouped by queue (the order within a queue is immaterial: a staged region is
// searched as a set). Per-block shared counts as above: each bead's rank within its block and
// queue (kept in s_slot, free between moves), one reservation per block and queue, then the
// placement.
__global__ void k_region_scatter(const SimView* __restrict__ vs, int l, int colour) {
    SIM_EXIT_IF(!sched_on(gv, l) || colour >= gv.K * gv.K * gv.K)
    SIM_PROLOGUE
    if (!sched_on(v, l) || colour >= v.K * v.K * v.K) return;
    const int Q = sched_layer(v, l).G / v.K, nq = Q * Q * Q;
    const int64_t m0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, ms = (int64_t)gridDim.x * blockDim.x;
    if (nq > kRegionPriv) {
        for (int64_t m = m0; m < v.N; m += ms) {
            const int key = v.rkey[m];
            if (key >= 0) v.rlist[v.rstart[key] + atomicAdd(&v.rfill[key], 1)] = (int)m;
        }
        return;
    }
    __shared__ int sh[kRegionPriv];
    for (int i = threadIdx.x; i < nq; i += blockDim.x) sh[i] = 0;
    __syncthreads();
    for (int64_t m = m0; m < v.N; m += ms) {
        const int key = v.rkey[m];
        if (key >= 0) v.s_slot[m] = atomicAdd(&sh[key], 1);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nq; i += blockDim.x)
        if (sh[i]) sh[i] = v.rstart[i] + atomicAdd(&v.rfill[i], sh[i]);
    __syncthreads();
    for (int64_t m = m0; m < v.N; m += ms) {
        const int key = v.rkey[m];
        if (key >= 0) v.rlist[sh[key] + v.s_slot[m]] = (int)m;
    }
}

// pointers into one warp's share of the dynamic shared memory
struct Stage {
    double *sx, *sy, *sz;            // staged positions (binary64, wrapped)
    float *hx, *hy, *hz;             // position relative to the region origin: hi part ...
    float *lx, *ly, *lz;             // ... and lo part (hi + lo carries the binary64 value)
    int *sid, *sdim, *stag;          // bead id, image change | dirty, support tag
    int *hkey, *hval;                // bead id -> staged index (open addressing)
    int *mem, *mimg, *mpart, *cand;  // support (staged indices), image change, bonded partners, candidates
    double *mnp;                     // new positions of the support (binary64, wrapped)
    float *mnh, *mnl;                // the same relative to the origin, hi and lo
    int *cj, *ci;                    // slot chunk: slot id, bead
    double *clam, *cV, *cp, *cthr;   // slot chunk: scale, centre offset, polarisation, threshold
    double *cR, *clamV, *cA0l;       // ... influence radius, lam V and A0 lam for the slot's own scale
    float *clamf, *cRf, *cVf, *cpf;  // ... binary32 forms of lam, R, V and p
    float* cthrf;                    // ... and of the threshold
    int* cti;                        // ... staged index of the picked bead (-1: not staged)
    int cap, hbits, ncap;            // staged beads, hash bits, support capacity
};
__host__ __device__ inline size_t stage_bytes(int cap, int ncap) {
    return (size_t)cap * (3 * 8 + 6 * 4 + 3 * 4 + 2 * 2 * 4) + (size_t)ncap * (4 + 4 + 2 * 4 + 3 * 8 + 6 * 4) +
           (size_t)kCandCap * 4 + (size_t)kSlotChunk * (4 + 4 + 8 + 24 + 24 + 8 + 8 + 24 + 8 + 4 + 4 + 4 + 12 + 12 + 4) + 160;
}
__host__ __device__ inline size_t warp_stride(int cap, int ncap) {
    size_t per = stage_bytes(cap, ncap) > sizeof(WarpSmem) ? stage_bytes(cap, ncap) : sizeof(WarpSmem);
    return (per + 15) & ~(size_t)15;
}
// per-warp bytes of a launch whose regions all fit `cap` (no global-memory path, so no room for
// its scratch)
__host__ __device__ inline size_t warp_stride_staged(int cap, int ncap) {
    return (stage_bytes(cap, ncap) + 15) & ~(size_t)15;
}
__device__ inline Stage stage_carve(char* base, int cap, int ncap) {
    Stage S;
    S.cap = cap;
    S.ncap = ncap;
    // hash table: the largest power of two that fits its 2 cap entries (load factor <= 1/2 for
    // power-of-two capacities, < 1 for any other)
    S.hbits = 1;
    while ((2 << S.hbits) <= 2 * cap) S.hbits++;
    char* p = base;
    auto take = [&](size_t bytes) { char* q = p; p += (bytes + 7) & ~(size_t)7; return q; };
    S.sx = (double*)take(8 * cap); S.sy = (double*)take(8 * cap); S.sz = (double*)take(8 * cap);
    S.mnp = (double*)take(8 * 3 * ncap);
    S.clam = (double*)take(8 * kSlotChunk); S.cV = (double*)take(8 * 3 * kSlotChunk);
    S.cp = (double*)take(8 * 3 * kSlotChunk); S.cthr = (double*)take(8 * kSlotChunk);
    S.hx = (float*)take(4 * cap); S.hy = (float*)take(4 * cap); S.hz = (float*)take(4 * cap);
    S.lx = (float*)take(4 * cap); S.ly = (float*)take(4 * cap); S.lz = (float*)take(4 * cap);
    S.mnh = (float*)take(4 * 3 * ncap); S.mnl = (float*)take(4 * 3 * ncap);
    S.sid = (int*)take(4 * cap); S.sdim = (int*)take(4 * cap); S.stag = (int*)take(4 * cap);
    S.hkey = (int*)take(4 * 2 * cap); S.hval = (int*)take(4 * 2 * cap);
    S.mem = (int*)take(4 * ncap); S.mimg = (int*)take(4 * ncap); S.mpart = (int*)take(4 * 2 * ncap);
    S.cand = (int*)take(4 * kCandCap);
    S.cj = (int*)take(4 * kSlotChunk); S.ci = (int*)take(4 * kSlotChunk);
    S.cR = (double*)take(8 * kSlotChunk); S.clamV = (double*)take(8 * 3 * kSlotChunk);
    S.cA0l = (double*)take(8 * kSlotChunk);
    S.clamf = (float*)take(4 * kSlotChunk); S.cRf = (float*)take(4 * kSlotChunk);
    S.cVf = (float*)take(4 * 3 * kSlotChunk); S.cpf = (float*)take(4 * 3 * kSlotChunk);
    S.cthrf = (float*)take(4 * kSlotChunk);
    S.cti = (int*)take(4 * kSlotChunk);
    return S;
}
__device__ __forceinline__ uint32_t hslot(int id, int bits) { return ((uint32_t)id * 2654435761u) >> (32 - bits); }
__device__ __forceinline__ int stage_find(const Stage& S, int id) {
    const uint32_t mask = (1u << S.hbits) - 1u;
    uint32_t h = hslot(id, S.hbits);
    for (int probe = 0; probe <= (int)mask; probe++) {
        const int k = S.hkey[h];
        if (k == id) return S.hval[h];
        if (k == -1) return -1;
        h = (h + 1u) & mask;
    }
    return -1;
}
// coordinate relative to the region origin o, brought into [0, L), as a binary32 pair hi + lo
__device__ __forceinline__ void local_split(double x, double o, double L, float& hi, float& lo) {
    double t = sub(x, o);
    if (lt_zero(t)) t = add(t, L);
    else if (ge_pos(t, L)) t = sub(t, L);
    hi = (float)t;
    lo = (float)sub(t, (double)hi);
}
// difference of two such coordinates: relative error about 2 ulp of binary32, no binary64 work
__device__ __forceinline__ float dfd(float ha, float la, float hb, float lb) { return (ha - hb) + (la - lb); }

// binary32 constants of a launch, converted once
struct Stage32 {
    Pot32 P32;
    float hLf, rcs2;
    const double* sqrt_n;            // sqrt(n) for n <= kNCap, correctly rounded (as sqr_t)
    float side[3];                   // region side per axis
    int kappa_on, eps_on;            // external well, WCA
    float kT9;                       // 1e-9 kT, the band's absolute floor
};
__device__ inline Stage32 stage32(const SimView& v) {
    Stage32 c;
    c.P32 = pot32(v.pot);
    c.hLf = (float)v.halfL;
    const float rcs = (float)(v.rc * (1.0 + 1e-6) + 1e-6);
    c.rcs2 = rcs * rcs;
    c.kappa_on = v.pot.kappa != 0.0;
    c.eps_on = v.pot.eps != 0.0;
    c.kT9 = 1e-9f * (float)v.kT;
    return c;
}

// Energy change of a staged move in binary64 (Eqs. 2, 5): bonds to beads outside the support,
// pairs inside it, WCA with the interaction candidates; fixed order per lane, warp sum.
__device__ void stage_energy64(const SimView& v, const Stage& S, const Stage32& C, int n, int nc, bool all_cand, int ns,
                               int tag, int lane, double* dU64, int* pe_out) {
    const double L = v.L, hL = v.halfL;
    const Pot& P = v.pot;
    const float rcs2 = C.rcs2;
    double a64 = 0.0;
    int pe = 0;
    auto pos64 = [&](int k, double* x) {
        if (k >= 0) { x[0] = S.mnp[3 * k]; x[1] = S.mnp[3 * k + 1]; x[2] = S.mnp[3 * k + 2]; }
        else { const int t = -1 - k; x[0] = S.sx[t]; x[1] = S.sy[t]; x[2] = S.sz[t]; }
    };
    auto r2_64 = [&](int ka, int kb) {
        double x[3], y[3];
        pos64(ka, x);
        pos64(kb, y);
        return norm2(mi(x[0] - y[0], L, hL), mi(x[1] - y[1], L, hL), mi(x[2] - y[2], L, hL));
    };
    // the binary32 distance of the candidate screen (the same screen as the binary32 pass)
    auto r2_32 = [&](int ka, int kb) {
        float h[2][3], lo[2][3];
        const int ks[2] = {ka, kb};
        for (int u = 0; u < 2; u++) {
            const int k = ks[u];
            if (k >= 0) {
                for (int a = 0; a < 3; a++) { h[u][a] = S.mnh[3 * k + a]; lo[u][a] = S.mnl[3 * k + a]; }
            } else {
                const int t = -1 - k;
                h[u][0] = S.hx[t]; h[u][1] = S.hy[t]; h[u][2] = S.hz[t];
                lo[u][0] = S.lx[t]; lo[u][1] = S.ly[t]; lo[u][2] = S.lz[t];
            }
        }
        const float dx = dfd(h[0][0], lo[0][0], h[1][0], lo[1][0]), dy = dfd(h[0][1], lo[0][1], h[1][1], lo[1][1]),
                    dz = dfd(h[0][2], lo[0][2], h[1][2], lo[1][2]);
        return dx * dx + dy * dy + dz * dz;
    };
    auto term = [&](int na, int nb, int oa, int ob, bool bonded, bool wca) {
        const double r2n = r2_64(na, nb), r2o = r2_64(oa, ob);
        double u = 0.0;
        if (wca) u += U_wca(P, r2n) - U_wca(P, r2o);
        if (bonded) u += U_bond(P, r2n) - U_bond(P, r2o);
        a64 += u;
    };
    // external well and bonds to beads outside the support
    for (int k = lane; k < n; k += 32) {
        const int t = S.mem[k];
        if (C.kappa_on) {
            const double* nw = &S.mnp[3 * k];
            a64 += U_ext(P, nw[0], nw[1], nw[2]) - U_ext(P, S.sx[t], S.sy[t], S.sz[t]);
        }
        for (int e = 0; e < 2; e++) {
            const int tq = S.mpart[2 * k + e];
            if (tq < 0) continue;                     // no bond, or the partner moves too
            term(k, -1 - tq, -1 - t, -1 - tq, true, false);
        }
    }
    // pairs inside the support
    const int npairs = n * (n - 1) / 2;
    for (int w = lane; w < npairs; w += 32) {
        int a = (int)((sqrtf(8.0f * w + 1.0f) - 1.0f) * 0.5f);
        while (a * (a + 1) / 2 > w) a--;
        while ((a + 1) * (a + 2) / 2 <= w) a++;
        const int k1 = w - a * (a + 1) / 2, k2 = a + 1;
        const int t1 = S.mem[k1], t2 = S.mem[k2];
        const int m1 = S.sid[t1], m2 = S.sid[t2];
        // bonded members: the lower one's partner above moves with the support (partner table)
        const int klo = m1 < m2 ? k1 : k2;
        const bool bonded = max(m1, m2) == min(m1, m2) + 1 && S.mpart[2 * klo + 1] == -2;
        term(k1, k2, -1 - t1, -1 - t2, bonded, true);
    }
    // WCA with the interaction candidates outside the support
    if (C.eps_on) {
        const int nsrc = all_cand ? ns : nc;
        const int total = n * nsrc;
        for (int w = lane; w < total; w += 32) {
            const int k = w / nsrc;
            const int c = all_cand ? (w - k * nsrc) : S.cand[w - k * nsrc];
            if (S.stag[c] == tag) continue;           // a support member (only when scanning everything)
            const int t = S.mem[k];
            if (!(r2_32(k, -1 - c) < rcs2) && !(r2_32(-1 - t, -1 - c) < rcs2)) continue;
            term(k, -1 - c, -1 - t, -1 - c, false, true);
            pe++;
        }
    }
    *dU64 = __shfl_sync(0xffffffffu, warp_sum(a64), 0);
    *pe_out = __reduce_add_sync(0xffffffffu, (unsigned)pe);
}

// The same energy change in binary32 from the staged hi + lo local coordinates, with the
// magnitude sum and summation depth its error band needs. All terms (bonds to outside beads,
// pairs inside the support, candidates) form one list dealt to the lanes, so a lane resolves
// its item and then every lane evaluates the same potentials together.
// This thread's share of the items (item w for w = i0, i0 + stride, ...): partial sums of the
// change and of the magnitudes, terms added, candidates within reach.
__device__ void stage_energy32_items(const SimView& v, const Stage& S, const Stage32& C, int n, int nc, bool all_cand,
                                     int ns, int tag, int i0, int stride, float& a32, float& m32, int& T, int& pe) {
    const double L = v.L, hL = v.halfL;
    const Pot32& P32 = C.P32;
    const float hLf = C.hLf;
    const float rcs2 = C.rcs2;
    a32 = 0.0f; m32 = 0.0f;
    T = 0; pe = 0;
    // external well (rare: only with kappa != 0), from the binary64 positions
    if (C.kappa_on) {
        for (int k = i0; k < n; k += stride) {
            const int t = S.mem[k];
            const double* nw = &S.mnp[3 * k];
            float un = 0.5f * P32.kappa * norm2f(dif32(nw[0], hL, L, hLf), dif32(nw[1], hL, L, hLf), dif32(nw[2], hL, L, hLf));
            float uo = 0.5f * P32.kappa * norm2f(dif32(S.sx[t], hL, L, hLf), dif32(S.sy[t], hL, L, hLf), dif32(S.sz[t], hL, L, hLf));
            a32 += un - uo; m32 += un + uo; T += 2;
        }
    }
    const int nB = 2 * n, nP = n * (n - 1) / 2;
    const int nsrc = all_cand ? ns : nc;
    const int nD = C.eps_on ? n * nsrc : 0;
    const int total = nB + nP + nD;
    for (int w = i0; w < total; w += stride) {
        // the item: new positions (na, nb), old positions (oa, ob); k >= 0 is a support member
        // (new position), k < 0 the staged bead -1 - k
        int na = 0, nb = 0, oa = 0, ob = 0;
        bool use = true, wca = false, bnd = false, screen = false;
        if (w < nB) {
            const int k = w >> 1, tq = S.mpart[w];
            use = tq >= 0;                            // no bond, or the partner moves too
            na = k; nb = -1 - tq; oa = -1 - S.mem[k]; ob = nb;
            bnd = true;
        } else if (w < nB + nP) {
            const int u = w - nB;
            int a = (int)((sqrtf(8.0f * u + 1.0f) - 1.0f) * 0.5f);
            while (a * (a + 1) / 2 > u) a--;
            while ((a + 1) * (a + 2) / 2 <= u) a++;
            const int k1 = u - a * (a + 1) / 2, k2 = a + 1;
            const int t1 = S.mem[k1], t2 = S.mem[k2];
            const int m1 = S.sid[t1], m2 = S.sid[t2];
            // bonded members: the lower one's partner above moves with the support
            const int klo = m1 < m2 ? k1 : k2;
            bnd = max(m1, m2) == min(m1, m2) + 1 && S.mpart[2 * klo + 1] == -2;
            wca = true;
            na = k1; nb = k2; oa = -1 - t1; ob = -1 - t2;
        } else {
            const int u = w - nB - nP;
            const int k = u / nsrc;
            const int c = all_cand ? (u - k * nsrc) : S.cand[u - k * nsrc];
            use = S.stag[c] != tag;                   // a support member (only when scanning everything)
            na = k; nb = -1 - c; oa = -1 - S.mem[k]; ob = nb;
            wca = true; screen = true;
        }
        if (!use) continue;
        float hn[2][3], ln[2][3];
        const int ks[4] = {na, nb, oa, ob};
        float r2[2];
        for (int pr = 0; pr < 2; pr++) {
            for (int u = 0; u < 2; u++) {
                const int k = ks[2 * pr + u];
                if (k >= 0) {
                    hn[u][0] = S.mnh[3 * k]; hn[u][1] = S.mnh[3 * k + 1]; hn[u][2] = S.mnh[3 * k + 2];
                    ln[u][0] = S.mnl[3 * k]; ln[u][1] = S.mnl[3 * k + 1]; ln[u][2] = S.mnl[3 * k + 2];
                } else {
                    const int t = -1 - k;
                    hn[u][0] = S.hx[t]; hn[u][1] = S.hy[t]; hn[u][2] = S.hz[t];
                    ln[u][0] = S.lx[t]; ln[u][1] = S.ly[t]; ln[u][2] = S.lz[t];
                }
            }
            const float dx = dfd(hn[0][0], ln[0][0], hn[1][0], ln[1][0]), dy = dfd(hn[0][1], ln[0][1], hn[1][1], ln[1][1]),
                        dz = dfd(hn[0][2], ln[0][2], hn[1][2], ln[1][2]);
            r2[pr] = dx * dx + dy * dy + dz * dz;
        }
        // a candidate counts only within the interaction reach, new or old (the screen's
        // distances are the term's distances)
        if (screen && !(r2[0] < rcs2) && !(r2[1] < rcs2)) continue;
        if (screen) pe++;
        float un, mn, uo, mo;
        if (wca) { wca32(P32, r2[0], un, mn); wca32(P32, r2[1], uo, mo); a32 += un - uo; m32 += mn + mo; T += 2; }
        if (bnd) { bond32(P32, r2[0], un, mn); bond32(P32, r2[1], uo, mo); a32 += un - uo; m32 += mn + mo; T += 2; }
    }
}
__device__ void stage_energy32(const SimView& v, const Stage& S, const Stage32& C, int n, int nc, bool all_cand, int ns,
                               int tag, int lane, float* dU32, float* mag32, int* terms, int* pe_out) {
    float a32, m32;
    int T, pe;
    stage_energy32_items(v, S, C, n, nc, all_cand, ns, tag, lane, 32, a32, m32, T, pe);
    const unsigned FULL = 0xffffffffu;
    float sm = a32, mm = m32;
    for (int o = 16; o > 0; o >>= 1) {
        sm += __shfl_xor_sync(FULL, sm, o);
        mm += __shfl_xor_sync(FULL, mm, o);
    }
    *dU32 = __shfl_sync(FULL, sm, 0);
    *mag32 = __shfl_sync(FULL, mm, 0);
    // summation depth: the most terms one lane added, then the five butterfly levels
    *terms = (int)__reduce_max_sync(FULL, (unsigned)T) + 5;
    *pe_out = (int)__reduce_add_sync(FULL, (unsigned)pe);
}

// What the warps of a block that serves one queue together share during a move.
struct CoopSh {
    int memw[kMaxStageWarps][kNCapMax];  // per warp: members found in its share of the scan
    int candw[kMaxStageWarps][kCandCap]; // ... and candidates
    int cnt[kMaxStageWarps][2];          // ... and their counts
    float part[kMaxStageWarps][2];       // per warp: binary32 change and magnitude sums
    int partT[kMaxStageWarps], partPE[kMaxStageWarps];
    int bad;                             // a bonded partner is not staged: the move is deferred
    int r[2];                            // outcome of the move, by parity of the move's tag
};

// One move of a staged queue. The slot's centre offset V, polarisation p and Metropolis
// threshold were prepared in the chunk arrays at index c. COOP: all H warps of the block call
// this together (role = warp index); each scans a contiguous share of the staged beads and takes
// a share of the binary32 energy items, warp 0 does the rest. Every branch around a block
// barrier depends only on values every warp computed alike or read after a barrier, so all
// warps meet every barrier. Warps other than 0 return 0 once their part is done.
template <int PREC, bool COOP>
__device__ int stage_attempt(const SimView& v, const Stage& S, const Stage32& C, int ns, const double org[3], float sidef,
                             int l, int c, double lam, const int64_t rlo[3], const int64_t rhi[3], int lane, int tag,
                             int* n_out, int* pe_out, int* recheck_out, double* du_out, int H, int role, CoopSh* X) {
    const unsigned FULL = 0xffffffffu;
    const double L = v.L, hL = v.halfL;
    const int Gf = v.Gf;
    *du_out = 0.0;
    const bool uni = v.centring == 1;             // centre uniform in the box: the chunk holds it in cV
    const int ti = S.cti[c];
    if (ti < 0 && !uni) return DEFER;             // the picked bead lies outside the region interior
    // centre b = r_i + lam V (Appendix D), wrapped; binary64 because the region rule and the
    // support must match the sequential definition exactly. For the slot's own scale lam V and
    // the influence radius R were formed ahead (same operations, same values); a carried scale
    // forms them here.
    const bool own = __double_as_longlong(lam) == __double_as_longlong(S.clam[c]);
    double b[3], lv[3];
    if (uni) {
        for (int a = 0; a < 3; a++) b[a] = S.cV[3 * c + a];
    } else {
        for (int a = 0; a < 3; a++) lv[a] = own ? S.clamV[3 * c + a] : mul(lam, S.cV[3 * c + a]);
        b[0] = add(S.sx[ti], lv[0]);
        b[1] = add(S.sy[ti], lv[1]);
        b[2] = add(S.sz[ti], lv[2]);
        wrap3_u(b, L, FULL, nullptr);
    }
    const double R = own ? S.cR[c] : add(add(lam, mul(mul(0.25, v.A0), lam)), v.r_reach);
    const float lamf = own ? S.clamf[c] : (float)lam;
    // A_w = A0 lam / sqrt(n) (Eq. 29) for every support size up to 32, one per lane, formed
    // while the scan below runs; the scan's n picks one
    const double a0l = own ? S.cA0l[c] : mul(v.A0, lam);
    const double aw_lane = uni ? uniform_aw(v, lam) : dvd(a0l, C.sqrt_n[lane + 1]);
    // the centre relative to the region origin in binary32 (from the picked bead's staged local
    // coordinates): its error, a few 1e-7 of the region side plus lam, is far inside the margins
    // of the screens below
    float bh[3];
    if (uni) {
        for (int a = 0; a < 3; a++) {
            float hi_, lo_;
            local_split(b[a], org[a], L, hi_, lo_);
            bh[a] = hi_ + lo_;
        }
    } else {
        bh[0] = (S.hx[ti] + S.lx[ti]) + lamf * S.cVf[3 * c];
        bh[1] = (S.hy[ti] + S.ly[ti]) + lamf * S.cVf[3 * c + 1];
        bh[2] = (S.hz[ti] + S.lz[ti]) + lamf * S.cVf[3 * c + 2];
    }
    // region rule: a binary32 screen proves most balls well inside the region's interior; the
    // others take the binary64 cell indices of the definition
    const float Rf = own ? S.cRf[c] : (float)R;
    bool surely_inside = true;
    for (int a = 0; a < 3; a++) {
        const float dm = 1e-6f * (C.side[a] + Rf) + 1e-6f;
        surely_inside = surely_inside && (bh[a] - Rf >= dm) && (bh[a] + Rf <= C.side[a] - dm);
    }
    if (!surely_inside) {
        bool inside = true;
        for (int a = 0; a < 3; a++) {
            const int64_t t0 = (int64_t)floor(mul(sub(b[a], R), v.invf));
            const int64_t t1 = (int64_t)floor(mul(add(b[a], R), v.invf));
            inside = inside && range_inside(t0, t1, rlo[a], rhi[a], Gf);
        }
        if (!inside) return DEFER;
    }
    // support and candidates in one binary32 pass over the staged beads (hi parts, with a
    // margin eps for their rounding); ties within eps of the sphere decided in binary64
    const float eps = 1e-6f * (sidef + lamf) + 1e-9f;
    const float lin = (lamf - eps) * (lamf - eps), lout = (lamf + eps) * (lamf + eps);
    const float Rc = Rf + eps;
    const float rcand = Rc * Rc;
    int n = 0, nc = 0;
    // the scan's share: all staged beads, or (COOP) a contiguous range, so that the warps' lists
    // concatenated in warp order are the single scan's lists
    const int qs = COOP ? ((ns + 32 * H - 1) / (32 * H)) * 32 : ns;
    const int t_lo = COOP ? min(ns, role * qs) : 0, t_hi = COOP ? min(ns, t_lo + qs) : ns;
    int* const lmem = COOP ? X->memw[role] : S.mem;
    int* const lcand = COOP ? X->candw[role] : S.cand;
    for (int base = t_lo; base < t_hi; base += 32) {
        const int t = base + lane;
        bool in = false, cd = false, tie = false;
        float d2 = 0.0f;
        if (t < t_hi) {
            const float dx = S.hx[t] - bh[0], dy = S.hy[t] - bh[1], dz = S.hz[t] - bh[2];
            d2 = dx * dx + dy * dy + dz * dz;
            in = d2 < lin;
            tie = !in && d2 <= lout;
        }
        // the binary64 test only in the rare passes that hold a tie (a branch the whole warp takes)
        if (__any_sync(FULL, tie)) {
            if (tie) {
                const double e2 = norm2(mi(sub(S.sx[t], b[0]), L, hL), mi(sub(S.sy[t], b[1]), L, hL), mi(sub(S.sz[t], b[2]), L, hL));
                in = e2 < mul(lam, lam);
            }
        }
        cd = t < t_hi && !in && d2 < rcand;
        const unsigned mi_ = __ballot_sync(FULL, in), mc = __ballot_sync(FULL, cd);
        const unsigned below = (1u << lane) - 1u;
        if (in) { const int s = n + __popc(mi_ & below); if (s < S.ncap) lmem[s] = t; }
        if (cd) { const int s = nc + __popc(mc & below); if (s < kCandCap) lcand[s] = t; }
        n += __popc(mi_);
        nc += __popc(mc);
    }
    if (COOP) {
        if (lane == 0) { X->cnt[role][0] = n; X->cnt[role][1] = nc; }
        __syncthreads();
        const int nw = n, ncw = nc;
        int om = 0, oc = 0;
        n = 0; nc = 0;
        for (int w = 0; w < H; w++) {
            if (w == role) { om = n; oc = nc; }
            n += X->cnt[w][0];
            nc += X->cnt[w][1];
        }
        // in place only when the whole list fits (otherwise the move is deferred, or the
        // candidates are taken from all staged beads)
        if (n <= sched_ncap(v, l))
            for (int k = lane; k < nw; k += 32) S.mem[om + k] = X->memw[role][k];
        if (nc <= kCandCap)
            for (int k = lane; k < ncw; k += 32) S.cand[oc + k] = X->candw[role][k];
        __syncthreads();
    }
    __syncwarp();                                 // support and candidate lists are read by every lane
    *n_out = n;
    if (n > sched_ncap(v, l)) return DEFER;
    if (n == 0) return 0.0 <= S.cthr[c] ? ACCEPT : REJECT;   // no bead moves: dU = 0 against the threshold
    const bool all_cand = nc > kCandCap;
    // displacement (Sec. V.A) with A_w = A0 lam / sqrt(n) (Eq. 29)
    const double Aw = uni ? aw_lane
                          : (n <= 32 ? __shfl_sync(FULL, aw_lane, n - 1) : dvd(a0l, n <= kNCap ? C.sqrt_n[n] : sqr_t((double)n)));
    const double p[3] = {S.cp[3 * c], S.cp[3 * c + 1], S.cp[3 * c + 2]};
    const float af = (float)Aw, pf[3] = {S.cpf[3 * c], S.cpf[3 * c + 1], S.cpf[3 * c + 2]};
    bool bad = false;
    if (!COOP || role == 0) {
    for (int k = lane; k < n; k += 32) {
        const unsigned am = __activemask();
        const int t = S.mem[k];
        S.stag[t] = tag;
        const double o[3] = {S.sx[t], S.sy[t], S.sz[t]};
        double d[3] = {sub(o[0], b[0]), sub(o[1], b[1]), sub(o[2], b[2])};
        mi3_u(d, L, hL, am);
        double dl[3];
        float dlf3[3];
        if (PREC == 0) {
            wavelet_disp64(d, norm2(d[0], d[1], d[2]), lam, Aw, p, dl);
            for (int a = 0; a < 3; a++) dlf3[a] = (float)dl[a];
        } else {
            wavelet_disp32ff(d, lamf, af, pf, dlf3);
            for (int a = 0; a < 3; a++) dl[a] = (double)dlf3[a];
        }
        int im[3] = {0, 0, 0};
        const float oh[3] = {S.hx[t], S.hy[t], S.hz[t]}, ol[3] = {S.lx[t], S.ly[t], S.lz[t]};
        double nx[3] = {add(o[0], dl[0]), add(o[1], dl[1]), add(o[2], dl[2])};
        wrap3_u(nx, L, am, im);
        for (int a = 0; a < 3; a++) {
            S.mnp[3 * k + a] = nx[a];
            // new local coordinate = old + displacement, in binary32 pairs (two-sum, then
            // renormalised); local coordinates are continuous inside the region, no wrap
            const float dlf = dlf3[a];
            const float s1 = oh[a] + dlf, bb = s1 - oh[a];
            const float err = (oh[a] - (s1 - bb)) + (dlf - bb);
            const float l1 = ol[a] + err;
            const float h2 = s1 + l1;
            S.mnh[3 * k + a] = h2;
            S.mnl[3 * k + a] = l1 - (h2 - s1);
        }
        S.mimg[k] = pack_img(im[0], im[1], im[2]);
    }
    __syncwarp();
    // bonded partners: staged (inside the region) or the move is deferred
    for (int k = lane; k < n; k += 32) {
        const int tk = S.mem[k];
        const int m = S.sid[tk], fl = S.sdim[tk] >> 25;   // staged bond flags: 1 up, 2 down
        for (int e = 0; e < 2; e++) {
            const int q = e ? m + 1 : m - 1;
            int tq = -1;
            if (q >= 0 && q < v.N && ((fl >> (1 - e)) & 1)) {
                tq = stage_find(S, q);
                if (tq < 0) bad = true;
                else if (S.stag[tq] == tag) tq = -2;   // moves with the support
            }
            S.mpart[2 * k + e] = tq;
        }
    }
    bad = __any_sync(FULL, bad);
    }
    if (COOP) {
        if (role == 0 && lane == 0) X->bad = bad;
        __syncthreads();
        bad = X->bad != 0;
    }
    if (bad) return DEFER;
    __syncwarp();
    const double thr = S.cthr[c];
    bool acc;
    int pe = 0;
    if (PREC == 1) {
        // binary32 energy change; the decision is taken in binary32 outside the rigorous error
        // band (per term 80 ulp of its magnitude, plus the summation) and in binary64 inside it
        float d32 = 0.0f, m32 = 0.0f;
        int T = 0;
        if (COOP) {
            // the items over every thread of the block; warp totals added by warp 0 in warp order
            float a, m;
            int Tt, pt;
            stage_energy32_items(v, S, C, n, nc, all_cand, ns, tag, role * 32 + lane, 32 * H, a, m, Tt, pt);
            for (int o = 16; o > 0; o >>= 1) {
                a += __shfl_xor_sync(FULL, a, o);
                m += __shfl_xor_sync(FULL, m, o);
            }
            Tt = (int)__reduce_max_sync(FULL, (unsigned)Tt);
            pt = (int)__reduce_add_sync(FULL, (unsigned)pt);
            if (lane == 0) { X->part[role][0] = a; X->part[role][1] = m; X->partT[role] = Tt; X->partPE[role] = pt; }
            __syncthreads();
            if (role != 0) return 0;
            for (int w = 0; w < H; w++) {
                d32 += X->part[w][0];
                m32 += X->part[w][1];
                T = max(T, X->partT[w]);
                pe += X->partPE[w];
            }
            T += 5 + H;      // summation depth: a thread's terms, the butterfly, the warp totals
        } else {
            stage_energy32(v, S, C, n, nc, all_cand, ns, tag, lane, &d32, &m32, &T, &pe);
        }
        const float thr32 = S.cthrf[c];
        const float band = 2.0f * (float)(80 + T + 6) * 5.9604645e-08f * m32 + C.kT9 + 2.4e-7f * fabsf(thr32);
        if (isfinite(d32) && isfinite(band) && fabsf(d32 - thr32) > band) {
            acc = d32 <= thr32;
            *du_out = (double)d32;
            if (v.audit) {
                double d64 = 0.0;
                int pe2 = 0;
                stage_energy64(v, S, C, n, nc, all_cand, ns, tag, lane, &d64, &pe2);
                if (lane == 0) audit_record(v, (double)d32, (double)band, (double)thr32, d64, thr);
            }
        } else {
            double d64 = 0.0;
            int pe2 = 0;
            stage_energy64(v, S, C, n, nc, all_cand, ns, tag, lane, &d64, &pe2);
            acc = d64 <= thr;
            *du_out = d64;
            (*recheck_out)++;
            if (v.audit && lane == 0) audit_record(v, (double)d32, (double)band, (double)thr32, d64, thr);
        }
    } else {
        if (COOP && role != 0) return 0;
        double d64 = 0.0;
        stage_energy64(v, S, C, n, nc, all_cand, ns, tag, lane, &d64, &pe);
        acc = d64 <= thr;
        *du_out = d64;
    }
    *pe_out += pe;
    if (!acc) return REJECT;
    for (int k = lane; k < n; k += 32) {
        const int t = S.mem[k];
        S.sx[t] = S.mnp[3 * k]; S.sy[t] = S.mnp[3 * k + 1]; S.sz[t] = S.mnp[3 * k + 2];
        S.hx[t] = S.mnh[3 * k]; S.hy[t] = S.mnh[3 * k + 1]; S.hz[t] = S.mnh[3 * k + 2];
        S.lx[t] = S.mnl[3 * k]; S.ly[t] = S.mnl[3 * k + 1]; S.lz[t] = S.mnl[3 * k + 2];
        // accumulate the image change (3 fields of 8 bits, offset 128) and mark dirty (bit 24)
        int dd[3], cur = S.sdim[t];
        unpack_img(S.mimg[k], dd);
        const int ax = ((cur & 0xff) - 128) + dd[0], ay = (((cur >> 8) & 0xff) - 128) + dd[1],
                  az = (((cur >> 16) & 0xff) - 128) + dd[2];
        S.sdim[t] = (ax + 128) | ((ay + 128) << 8) | ((az + 128) << 16) | (1 << 24) | (cur & (3 << 25));
    }
    __syncwarp();
    return ACCEPT;
}

// Whether a block of the staged kernel has a queue to run: a slot in it and a region whose bead
// count lies in [ns_lo, ns_hi] (read from global memory before the block copies anything).
__device__ __forceinline__ bool staged_block_has_work(const SimView& g, int l, int colour, int qpb, int ns_lo,
                                                      int ns_hi) {
    const int Q = sched_layer(g, l).G / g.K, nq = Q * Q * Q;
    for (int w = 0; w < qpb; w++) {
        const int q = (int)blockIdx.x * qpb + w;
        if (q >= nq) break;
        if (g.q_count[colour * nq + q] == 0) continue;
        const int ns = g.rcount[q];
        if (ns >= ns_lo && ns <= ns_hi) return true;
    }
    return false;
}

// The cooperative scratch of a block whose warps serve one queue together (none for the light
// variant, whose blocks serve one queue per warp).
template <bool USE>
__device__ __forceinline__ CoopSh* coop_scratch() {
    if constexpr (USE) {
        __shared__ CoopSh s_coop;
        return &s_coop;
    } else {
        return nullptr;
    }
}
// A block serves qpb queues with one warp each, or (qpb = 1) one queue with all its warps: then
// every warp stages a share of the region (the binary64 work of staging spreads over the SM's
// four schedulers) and warp 0 alone runs the moves. cap = staged beads per queue; stride =
// shared bytes per queue. Only queues whose region holds ns_lo..ns_hi beads run: a colour phase
// is split between a launch for ordinary regions (small staging, more warps per SM) and launches
// for the dense ones, which take disjoint queues, so the split changes nothing in the results.
// list = 0: queue blockIdx.x * qpb + warp; list = 1 or 2: the block takes queues from that list
// of dense regions (built by the region scan) until it is done.
// VAR 0: every path. VAR 1 (light): a launch whose regions all fit its staging, one warp per
// queue: no global-memory path and no cooperating warps are compiled in. VAR 2 (middle dense
// tier): cooperating warps, regions that always fit, no global-memory path. The narrower
// variants leave fewer registers per thread, so three blocks fit an SM.
template <int PREC, int VAR>
__global__ void __launch_bounds__(kMaxStageWarps * 32, VAR == 0 ? 1 : 3) k_colour_staged(const SimView* __restrict__ vs, int l, int colour,
                                                                        int cap, int qpb, int ncap, int stride,
                                                                        int ns_lo, int ns_hi, int list) {
    SIM_EXIT_IF(!sched_on(gv, l) || gv.precision != PREC || colour >= gv.K * gv.K * gv.K ||
                (list ? (int)blockIdx.x >= gv.hq_ctl[list == 2 ? 2 : 0]
                      : ((int)(blockIdx.x * qpb) >= (sched_layer(gv, l).G / gv.K) * (sched_layer(gv, l).G / gv.K) * (sched_layer(gv, l).G / gv.K) ||
                         !staged_block_has_work(gv, l, colour, qpb, ns_lo, ns_hi))))
    SIM_PROLOGUE
    extern __shared__ __align__(16) char dsm[];
    if (!sched_on(v, l) || v.precision != PREC || colour >= v.K * v.K * v.K) return;
    // sqrt(n) for the amplitude A_w = A0 lam / sqrt(n) (Eq. 29), once per block
    __shared__ double s_sqrt[kNCap + 1];
    constexpr bool LIGHT = VAR == 1, STAGED_ONLY = VAR != 0;
    CoopSh* const X = coop_scratch<!LIGHT>();
    for (int i = threadIdx.x; i <= kNCap; i += blockDim.x) s_sqrt[i] = sqr_t((double)i);
    __syncthreads();
    const uint64_t sweep = v.step[0];
    const int H = LIGHT ? 1 : (int)(blockDim.x >> 5) / qpb;     // warps per queue: 1, or all of the block
    const int wib = (int)(threadIdx.x >> 5) / H, role = (int)(threadIdx.x >> 5) % H, lane = threadIdx.x & 31;
    const unsigned FULL = 0xffffffffu;
    const LayerDev Ly = sched_layer(v, l);
    // random draws, counters and trace are the layer's own; a second colouring's moves carry flag 4
    const int lr = layer_real(l);
    const uint8_t tflag = l >= kLevel2 ? 4 : 0;
    const int G = Ly.G, K = v.K, Q = G / K, nq = Q * Q * Q;
    // one queue per warp (or per block), or (list) the block takes queues of the phase's list of
    // dense regions one after another until the list is done; "continue" ends a queue
    __shared__ int s_item;
    for (int it = 0;; it++) {
        int q;
        if (list) {
            // list 1: the front of hq_list (regions up to the middle size), list 2: its back
            const int lc = list == 2 ? 2 : 0;
            if (threadIdx.x == 0) s_item = atomicAdd(&v.hq_ctl[lc + 1], 1);
            __syncthreads();
            const int i = s_item;
            __syncthreads();                          // read by all before the next item is taken
            if (i >= v.hq_ctl[lc]) break;
            q = v.hq_list[list == 2 ? nq - 1 - i : i];
        } else {
            if (it > 0) break;
            q = blockIdx.x * qpb + wib;
        }
        if (q >= nq) continue;                        // uniform over the warps of a queue
        const int key = colour * nq + q;
        const int start = v.q_start[key], cnt = v.q_count[key];
        if (cnt == 0) continue;
        {
            const int ns0 = v.rcount[q];
            if (ns0 < ns_lo || ns0 > ns_hi) continue; // another launch of this phase runs the queue
        }
        char* base = dsm + (size_t)wib * (size_t)stride;
        const int c[3] = {K * (q % Q) + colour % K, K * ((q / Q) % Q) + (colour / K) % K, K * (q / (Q * Q)) + colour / (K * K)};
        int64_t rlo[3], rhi[3];
        for (int a = 0; a < 3; a++) {
            rlo[a] = ceildiv((2 * (int64_t)c[a] - (K - 1)) * v.Gf, 2 * (int64_t)G);
            rhi[a] = floordiv((2 * (int64_t)c[a] + 2 + (K - 1)) * v.Gf, 2 * (int64_t)G) - 1;
        }
        const int cell = c[0] + G * (c[1] + G * c[2]);
        double carry = v.carry_q[Ly.carry_off + cell];
        int att = 0, acc = 0, def = 0, pe = 0, rechecks = 0;
        long long bu = 0, moved = 0;
        const int rs = v.rstart[q], ns = v.rcount[q];
        if (!STAGED_ONLY && ns > cap) {
            // region too full for shared memory: the global-memory path
            if (role != 0) continue;
            WarpSmem& sm = *(WarpSmem*)base;
            for (int t = 0; t < cnt; t++) {
                const int j = v.q_slots[start + t];
                const double lam = carry > 0.0 ? carry : v.slot_lam[j];
                int n = 0;
                double du = 0.0;
                int r = warp_attempt<PREC>(v, sm, l, j, v.slot_bead[j], lam, sweep, rlo, rhi, lane, &n, &pe, &rechecks, &du);
                __syncwarp();
                if (r == DEFER) { if (lane == 0) v.defer[start + t] = 1; def++; continue; }
                att++; bu += n;
                if (r == ACCEPT) { acc++; moved += n; }
                if (lane == 0) {
                    v.tr_out[Ly.tr_off + j] = (uint8_t)((r == ACCEPT ? 1 : 2) | tflag);
                    v.tr_n[Ly.tr_off + j] = n;
                    v.tr_du[Ly.tr_off + j] = du;
                }
                carry = (r == ACCEPT) ? 0.0 : lam;
            }
        } else {
            Stage S = stage_carve(base, cap, ncap);
            Stage32 C32 = stage32(v);
            C32.sqrt_n = s_sqrt;
            for (int a = 0; a < 3; a++) C32.side[a] = (float)((double)(rhi[a] - rlo[a] + 1) * (v.L / v.Gf));
            const int HT = 1 << S.hbits;
            const int ql = role * 32 + lane, qstride = 32 * H;   // this thread among the queue's warps
            for (int h = ql; h < HT; h += qstride) S.hkey[h] = -1;
            if (H > 1) __syncthreads(); else __syncwarp();
            const double hf = v.L / v.Gf;
            const double org[3] = {(double)rlo[0] * hf, (double)rlo[1] * hf, (double)rlo[2] * hf};
            const float sidef = (float)((double)(rhi[0] - rlo[0] + 1) * hf);
            for (int t = ql; t < ns; t += qstride) {
                const int m = v.rlist[rs + t];
                const Bead bb = v.bead[m];
                S.sx[t] = bb.x; S.sy[t] = bb.y; S.sz[t] = bb.z;
                local_split(bb.x, org[0], v.L, S.hx[t], S.lx[t]);
                local_split(bb.y, org[1], v.L, S.hy[t], S.ly[t]);
                local_split(bb.z, org[2], v.L, S.hz[t], S.lz[t]);
                S.sid[t] = m;
                const int bflag = (v.bnext[m] ? 1 : 0) | (m > 0 && v.bnext[m - 1] ? 2 : 0);
                S.sdim[t] = 128 | (128 << 8) | (128 << 16) | (bflag << 25);
                S.stag[t] = 0;
                const uint32_t mask = (uint32_t)HT - 1u;
                uint32_t h = hslot(m, S.hbits);
                for (int probe = 0; probe < HT; probe++) {
                    const int prev = atomicCAS(&S.hkey[h], -1, m);
                    if (prev == -1) { S.hval[h] = t; break; }
                    h = (h + 1u) & mask;
                }
            }
            if (H > 1) __syncthreads(); else __syncwarp();
            int tag = 0;
            for (int c0 = 0; c0 < cnt; c0 += kSlotChunk) {
                // slot parameters of the chunk, one lane of warp 0 per slot: V, p and the acceptance
                // threshold as the slot kernel drew them (Appendix D, Eq. 20)
                const int t = c0 + lane;
                if (role == 0 && t < cnt) {
                    const int j = v.q_slots[start + t];
                    S.cj[lane] = j;
                    S.ci[lane] = v.slot_bead[j];
                    S.clam[lane] = v.slot_lam[j];
                    double V[3];
                    for (int a = 0; a < 3; a++) {
                        V[a] = v.slot_V[3 * j + a];             // with uniform centres: the centre itself
                        S.cV[3 * lane + a] = V[a];
                        S.cp[3 * lane + a] = v.slot_p[3 * j + a];
                    }
                    S.cthr[lane] = v.slot_thr[j];
                    S.cthrf[lane] = (float)S.cthr[lane];
                    // what the move needs from its own scale, ahead of the sequential loop
                    const double lam_s = S.clam[lane];
                    const double R_s = add(add(lam_s, mul(mul(0.25, v.A0), lam_s)), v.r_reach);
                    S.cR[lane] = R_s;
                    S.cRf[lane] = (float)R_s;
                    S.clamf[lane] = (float)lam_s;
                    S.cA0l[lane] = mul(v.A0, lam_s);
                    for (int a = 0; a < 3; a++) {
                        S.clamV[3 * lane + a] = mul(lam_s, V[a]);
                        S.cVf[3 * lane + a] = (float)V[a];
                        S.cpf[3 * lane + a] = (float)S.cp[3 * lane + a];
                    }
                    S.cti[lane] = stage_find(S, S.ci[lane]);
                }
                if (H > 1) __syncthreads(); else __syncwarp();
                const int cend = min(kSlotChunk, cnt - c0);
                for (int cc = 0; cc < cend; cc++) {
                    const int j = S.cj[cc];
                    const double lam = __double_as_longlong(carry) > 0 ? carry : S.clam[cc];
                    int n = 0;
                    double du = 0.0;
                    tag++;
                    int r;
                    if (H > 1) {
                        r = stage_attempt<PREC, true>(v, S, C32, ns, org, sidef, l, cc, lam, rlo, rhi, lane, tag, &n, &pe,
                                                      &rechecks, &du, H, role, X);
                        __syncwarp();
                        // warp 0's outcome (and its commit) reach every warp before the next move
                        if (role == 0 && lane == 0) X->r[tag & 1] = r;
                        __syncthreads();
                        r = X->r[tag & 1];
                    } else {
                        r = stage_attempt<PREC, false>(v, S, C32, ns, org, sidef, l, cc, lam, rlo, rhi, lane, tag, &n, &pe,
                                                       &rechecks, &du, 1, 0, nullptr);
                        __syncwarp();
                    }
                    if (r == DEFER) { if (role == 0 && lane == 0) v.defer[start + c0 + cc] = 1; def++; continue; }
                    att++; bu += n;
                    if (r == ACCEPT) { acc++; moved += n; }
                    if (role == 0 && lane == 0) {
                        v.tr_out[Ly.tr_off + j] = (uint8_t)((r == ACCEPT ? 1 : 2) | tflag);
                        v.tr_n[Ly.tr_off + j] = n;
                        v.tr_du[Ly.tr_off + j] = du;
                    }
                    carry = (r == ACCEPT) ? 0.0 : lam;
                }
                // the chunk arrays are refilled only after every warp has finished this chunk
                if (H > 1) __syncthreads(); else __syncwarp();
            }
            if (role != 0) continue;                    // the write-back runs on warp 0
            // write back the moved beads (lanes in parallel); cell-list moves by lane 0, in
            // staged order, for the beads whose fine cell changed (the old cell from the bead's
            // record, which nothing else writes during the phase)
            for (int base2 = 0; base2 < ns; base2 += 32) {
                const int t = base2 + lane;
                int newcell = -1, oldcell = -1;
                if (t < ns && (S.sdim[t] & (1 << 24))) {
                    const int dm = S.sdim[t];
                    const int m = S.sid[t];
                    const Bead ob = v.bead[m];
                    oldcell = cell_lin(v, ob.x, ob.y, ob.z);
                    put_bead(v.bead, v.bf, m, S.sx[t], S.sy[t], S.sz[t]);
                    const int ax = (dm & 0xff) - 128, ay = ((dm >> 8) & 0xff) - 128, az = ((dm >> 16) & 0xff) - 128;
                    if (ax | ay | az) { v.img[3 * m] += ax; v.img[3 * m + 1] += ay; v.img[3 * m + 2] += az; }
                    const int nc2 = cell_lin(v, S.sx[t], S.sy[t], S.sz[t]);
                    if (nc2 != oldcell) newcell = nc2;
                }
                const unsigned ch = __ballot_sync(FULL, newcell >= 0);
                S.cand[lane] = newcell;
                S.cand[32 + lane] = oldcell;
                __syncwarp();
                if (lane == 0) {
                    for (unsigned bits = ch; bits; bits &= bits - 1u) {
                        const int ln = __ffs(bits) - 1, tt = base2 + ln;
                        const int m = S.sid[tt], oc = S.cand[32 + ln], ncl = S.cand[ln];
                        relink(v, m, oc, ncl);
                    }
                }
                __syncwarp();
            }
        }
        if (lane == 0) {
            v.carry_q[Ly.carry_off + cell] = carry;
            atomicAdd(&v.ctr[C_ATT + lr], (unsigned long long)att);
            atomicAdd(&v.ctr[C_ACC + lr], (unsigned long long)acc);
            if (l < kLevel2) atomicAdd(&v.ctr[C_DEF + lr], (unsigned long long)def);   // first deferrals only
            atomicAdd(&v.ctr[C_ACCTOT], (unsigned long long)acc);
            atomicAdd(&v.ctr[C_BU], (unsigned long long)bu);
            atomicAdd(&v.ctr[C_PARTNER], (unsigned long long)pe);
            atomicAdd(&v.ctr[C_CBU], (unsigned long long)bu);
            atomicAdd(&v.ctr[C_CMOVED], (unsigned long long)moved);
            atomicAdd(&v.ctr[C_MOVED], (unsigned long long)moved);
            atomicAdd(&v.ctr[C_CPE], (unsigned long long)pe);
            if (rechecks) atomicAdd(&v.ctr[C_RECHECK], (unsigned long long)rechecks);
        }
    }   // queues
}

size_t staged_smem_bytes(int cap, int warps, int ncap) { return (size_t)warps * warp_stride(cap, ncap); }
// the launch of ordinary regions: regions of at most kLightCap beads, kMaxStageWarps queues per block
constexpr int kLightCap = 80;
// the dense regions of a split phase: up to kMidCap beads staged by blocks small enough for three
// per SM, the larger ones by blocks with the most shared memory
constexpr int kMidCap = 512;
// (its supports are at most its regions' kLightCap beads, so its support arrays need no more)
static int light_ncap(int ncap) { return ncap < kLightCap ? ncap : kLightCap; }
static size_t light_smem_bytes(int ncap) {
    return (size_t)kMaxStageWarps * warp_stride_staged(kLightCap, light_ncap(ncap));
}
// largest support of schedule index l's concurrent moves over the group
static int sched_ncap_g(const GroupDims& g, int l) { return l >= kLevel2 ? kNCapMax : g.ncap; }
static bool split_layer(const GroupDims& g, int l, int cap) {
    return g.cap_l[l] == 0 && cap > kLightCap &&
           light_smem_bytes(sched_ncap_g(g, l)) + sizeof(SimView) + sizeof(CoopSh) + 1024 <= 227u * 1024u;
}
static bool staged_fits(int cap, int queues, int ncap) {
    // dynamic shared memory + the static view copy, sqrt table and cooperative scratch within the
    // 227 KB of a block
    return staged_smem_bytes(cap, queues, ncap) + sizeof(SimView) + sizeof(CoopSh) + 1024 <= 227u * 1024u;
}
int staged_cap_max(int ncap) {
    int cap = 256;
    while (staged_fits(cap + 32, 1, ncap)) cap += 32;
    return cap;
}
// staging capacity of layer l's launches (the largest over the group, within one block's shared
// memory: a region above it takes the global-memory path)
static int layer_cap(const GroupDims& g, int l) {
    return std::min(std::max(g.stage_cap, g.cap_l[l]), staged_cap_max(sched_ncap_g(g, l)));
}
// queues per block actually used: the requested count, lowered until the block's shared memory
// fits; a block of one queue with a region larger than 1,024 beads gets kMaxStageWarps warps,
// which share the staging
static void staged_shape(const GroupDims& g, int cap, int ncap, int* qpb, int* warps) {
    int nw = std::max(1, std::min(g.block_warps, kMaxStageWarps));
    while (nw > 1 && !staged_fits(cap, nw, ncap)) nw--;
    *qpb = nw;
    *warps = (nw == 1 && cap > 1024) ? kMaxStageWarps : nw;
}

// The largest dynamic shared memory each staged kernel was opened for, per device: raised
// before a launch needs more, so that launches recorded into a graph set nothing.
static int g_staged_smem[64][2][3];
static int g_serial_smem[64][2];
void prepare_staged(const GroupDims& g) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    static bool serial_opened[64] = {false};
    if (!serial_opened[dev]) {
        cudaFuncSetAttribute(k_serial<1, 512>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)serial_dyn_bytes<1, 512>());
        cudaFuncSetAttribute(k_serial<0, 512>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)serial_dyn_bytes<0, 512>());
        serial_opened[dev] = true;
    }
    if (g.smem_maxN > 0) {
        const int sm = (int)smem_serial_bytes(g.smem_maxN);
        if ((g.prec_mask & 1) && sm > g_serial_smem[dev][0]) {
            cudaFuncSetAttribute(k_serial_smem<0, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
            cudaFuncSetAttribute(k_serial_smem<0, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
            cudaFuncSetAttribute(k_serial_smem<0, 512>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
            g_serial_smem[dev][0] = sm;
        }
        if ((g.prec_mask & 2) && sm > g_serial_smem[dev][1]) {
            cudaFuncSetAttribute(k_serial_smem<1, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
            cudaFuncSetAttribute(k_serial_smem<1, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
            cudaFuncSetAttribute(k_serial_smem<1, 512>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
            g_serial_smem[dev][1] = sm;
        }
    }
    int smem = 0, smemL = 0, smemM = 0;
    for (int i = 0; i < 2 * g.maxL; i++) {
        const int l = i < g.maxL ? i : kLevel2 + i - g.maxL;
        if (!g.coloured[l]) continue;
        const int cap = layer_cap(g, l), ncap = sched_ncap_g(g, l);
        int qpb = 1, warps = 1;
        staged_shape(g, cap, ncap, &qpb, &warps);
        smem = std::max(smem, (int)staged_smem_bytes(cap, qpb, ncap));
        if (split_layer(g, l, cap)) {
            smemL = std::max(smemL, (int)light_smem_bytes(ncap));
            smemM = std::max(smemM, (int)warp_stride_staged(kMidCap, ncap));
            smem = std::max(smem, (int)staged_smem_bytes(staged_cap_max(ncap), 1, ncap));
        }
    }
    if ((g.prec_mask & 1) && smem > g_staged_smem[dev][0][0]) {
        cudaFuncSetAttribute(k_colour_staged<0, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        g_staged_smem[dev][0][0] = smem;
    }
    if ((g.prec_mask & 2) && smem > g_staged_smem[dev][1][0]) {
        cudaFuncSetAttribute(k_colour_staged<1, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        g_staged_smem[dev][1][0] = smem;
    }
    if ((g.prec_mask & 1) && smemL > g_staged_smem[dev][0][1]) {
        cudaFuncSetAttribute(k_colour_staged<0, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smemL);
        g_staged_smem[dev][0][1] = smemL;
    }
    if ((g.prec_mask & 2) && smemL > g_staged_smem[dev][1][1]) {
        cudaFuncSetAttribute(k_colour_staged<1, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smemL);
        g_staged_smem[dev][1][1] = smemL;
    }
    if ((g.prec_mask & 1) && smemM > g_staged_smem[dev][0][2]) {
        cudaFuncSetAttribute(k_colour_staged<0, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, smemM);
        g_staged_smem[dev][0][2] = smemM;
    }
    if ((g.prec_mask & 2) && smemM > g_staged_smem[dev][1][2]) {
        cudaFuncSetAttribute(k_colour_staged<1, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, smemM);
        g_staged_smem[dev][1][2] = smemM;
    }
}

// multiprocessors of the current device (cached per device)
static int sm_count() {
    static int cache[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    if (cache[dev] == 0) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) n = 1;
        cache[dev] = n;
    }
    return cache[dev];
}

int launch_colour_staged(const SimView* d, const GroupDims& g, int l, int colour, cudaStream_t s, const ForkJoin* fj) {
    const int nq = g.nq[l];
    const int gb = (int)gx((g.maxN + 255) / 256, g.S);
    const int cap = layer_cap(g, l), ncap = sched_ncap_g(g, l);
    const bool split = split_layer(g, l, cap) && fj && fj->side[0];
    k_zero<<<dim3(gx((nq + 255) / 256, g.S), g.S), 256, 0, s>>>(d, 1, l);
    k_region_count<<<dim3(gb, g.S), 256, 0, s>>>(d, l, colour);
    k_scan<<<dim3(1, g.S), 1024, 0, s>>>(d, 1, l, colour, split ? kLightCap : -1, kMidCap);
    k_region_scatter<<<dim3(gb, g.S), 256, 0, s>>>(d, l, colour);
    int qpb = 1, warps = 1;
    staged_shape(g, cap, ncap, &qpb, &warps);
    const size_t smem = staged_smem_bytes(cap, qpb, ncap);
    const dim3 grid((nq + qpb - 1) / qpb, g.S);
    prepare_staged(g);
    const int stride = (int)warp_stride(cap, ncap);
    const int np = (g.prec_mask & 1) + ((g.prec_mask >> 1) & 1);
    if (split) {
        // Ordinary regions (at most kLightCap beads) on the stream, one warp per queue and small
        // staging; the dense regions (a chain's worth of beads, the longest queues of the phase)
        // at the same time on side streams, one block of cooperating warps per queue: those up to
        // kMidCap beads by a variant without the global-memory path (three blocks per SM), the
        // rest with room for the largest region. The launches take disjoint queues of one colour; the dense ones run
        // persistently over the lists the region scan made.
        const int qL = kMaxStageWarps;
        const dim3 gridL((nq + qL - 1) / qL, g.S);
        const size_t smemL = light_smem_bytes(ncap);
        const int strideL = (int)warp_stride_staged(kLightCap, light_ncap(ncap));
        const int capH = staged_cap_max(ncap);
        const size_t smemH = staged_smem_bytes(capH, 1, ncap);
        const int strideH = (int)warp_stride(capH, ncap);
        const int strideM = (int)warp_stride_staged(kMidCap, ncap);   // its regions always fit
        const dim3 gridH(std::min(nq, sm_count()), g.S), gridM(std::min(nq, 3 * sm_count()), g.S);
        cudaStream_t sm_ = fj->side[0], sh_ = fj->side[1] ? fj->side[1] : fj->side[0];
        cudaEventRecord(fj->fork, s);
        cudaStreamWaitEvent(sm_, fj->fork, 0);
        if (sh_ != sm_) cudaStreamWaitEvent(sh_, fj->fork, 0);
        if (g.prec_mask & 1) {
            k_colour_staged<0, 2><<<gridM, kMaxStageWarps * 32, strideM, sm_>>>(d, l, colour, kMidCap, 1, ncap, strideM, kLightCap + 1, kMidCap, 1);
            k_colour_staged<0, 0><<<gridH, kMaxStageWarps * 32, smemH, sh_>>>(d, l, colour, capH, 1, ncap, strideH, kMidCap + 1, 1 << 30, 2);
        }
        if (g.prec_mask & 2) {
            k_colour_staged<1, 2><<<gridM, kMaxStageWarps * 32, strideM, sm_>>>(d, l, colour, kMidCap, 1, ncap, strideM, kLightCap + 1, kMidCap, 1);
            k_colour_staged<1, 0><<<gridH, kMaxStageWarps * 32, smemH, sh_>>>(d, l, colour, capH, 1, ncap, strideH, kMidCap + 1, 1 << 30, 2);
        }
        const int ncL = light_ncap(ncap);
        if (g.prec_mask & 1) k_colour_staged<0, 1><<<gridL, qL * 32, smemL, s>>>(d, l, colour, kLightCap, qL, ncL, strideL, 0, kLightCap, 0);
        if (g.prec_mask & 2) k_colour_staged<1, 1><<<gridL, qL * 32, smemL, s>>>(d, l, colour, kLightCap, qL, ncL, strideL, 0, kLightCap, 0);
        cudaEventRecord(fj->join[0], sm_);
        cudaStreamWaitEvent(s, fj->join[0], 0);
        if (sh_ != sm_) {
            cudaEventRecord(fj->join[1], sh_);
            cudaStreamWaitEvent(s, fj->join[1], 0);
        }
        return 4 + 3 * np;
    }
    // one launch per precision; each returns at once for simulations of the other precision
    if (g.prec_mask & 1) k_colour_staged<0, 0><<<grid, warps * 32, smem, s>>>(d, l, colour, cap, qpb, ncap, stride, 0, 1 << 30, 0);
    if (g.prec_mask & 2) k_colour_staged<1, 0><<<grid, warps * 32, smem, s>>>(d, l, colour, cap, qpb, ncap, stride, 0, 1 << 30, 0);
    return 4 + np;

}

}  // namespace wmcd
