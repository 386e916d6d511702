// Plane-wave moves without any device allocation (wmcd_planewave_noalloc in include/wmcd.h).
//
// Some callers cannot call cudaMalloc: code that runs while another framework owns the
// device memory pool, real-time loops that must not allocate after start-up, and hosts that
// forbid allocation inside their own callbacks. For them this file keeps every scratch buffer
// the plane-wave kernels need in one file-scope device array of fixed size, which the driver
// reserves when the library is loaded and keeps on every GPU that loads it until exit.
#include <cuda.h>
#include <cstring>
#include "../../include/wmcd.h"
#include "wmcd_host.h"

namespace wmcd {

int mode_table_static(double L, double lmax, int lcut, int* modes, double* cdf, int cap);

constexpr int64_t kNaBeads = 16384;              // largest N
constexpr int64_t kNaCells = 48 * 48 * 48;       // largest grid_f^3
constexpr int kNaLcut = 8;                       // largest lcut
constexpr int kNaModes = (2 * kNaLcut + 1) * (2 * kNaLcut + 1) * (2 * kNaLcut + 1);
constexpr int64_t kNaBlocks = (kNaBeads + 255) / 256;

// byte offsets of the pieces inside the scratch array (each 256-byte aligned)
constexpr int64_t al(int64_t x) { return (x + 255) & ~(int64_t)255; }
constexpr int64_t oBead = 0;
constexpr int64_t oPrev = oBead + al(sizeof(Bead) * kNaBeads);
constexpr int64_t oImg = oPrev + al(4 * kNaBeads);
constexpr int64_t oBnext = oImg + al(12 * kNaBeads);
constexpr int64_t oHead = oBnext + al(kNaBeads);
constexpr int64_t oPwNew = oHead + al(4 * kNaCells);
constexpr int64_t oPwImg = oPwNew + al(24 * kNaBeads);
constexpr int64_t oPart = oPwImg + al(4 * kNaBeads);
constexpr int64_t oPw = oPart + al(8 * kNaBlocks);
constexpr int64_t oCtr = oPw + al(sizeof(PWDev));
constexpr int64_t oErr = oCtr + al(8 * C_NCTR);
constexpr int64_t oRebuild = oErr + al(4);
constexpr int64_t oModes = oRebuild + al(4);
constexpr int64_t oCdf = oModes + al(12 * kNaModes);
constexpr int64_t oView = oCdf + al(8 * kNaModes);
constexpr int64_t oStep = oView + al(sizeof(SimView));
constexpr int64_t oCounts = oStep + al(16);
constexpr int64_t oClStale = oCounts + al(4 * (kMaxLayers + 1));
constexpr int64_t kNaBytes = oClStale + al(4);   // about 1.9 MB

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaBytes];

static __global__ void k_na_fill(Bead* bead, const double* pos, int64_t N) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        bead[i].x = pos[3 * i]; bead[i].y = pos[3 * i + 1]; bead[i].z = pos[3 * i + 2];
        bead[i].mark = 0u;
    }
}
// copies the moved beads back into the caller's buffer unless an error was flagged, so that
// on any error return the caller's positions are left as they were
static __global__ void k_na_read(const Bead* bead, double* pos, int64_t N, const int* err) {
    if (*err) return;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        pos[3 * i] = bead[i].x; pos[3 * i + 1] = bead[i].y; pos[3 * i + 2] = bead[i].z;
    }
}
static __global__ void k_na_carry(PWDev* pw, const int* carry_in) {
    pw->carry = carry_in[0];
    pw->carry_l[0] = carry_in[1]; pw->carry_l[1] = carry_in[2]; pw->carry_l[2] = carry_in[3];
}
static __global__ void k_na_check(const double* pos, int64_t N, double L, int* err) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < 3 * N; i += (int64_t)gridDim.x * blockDim.x)
        if (!(pos[i] >= 0.0 && pos[i] < L)) atomicOr(err, E_NONFINITE);
}

// Identifier of the calling thread's current context (0 if it cannot be read): a device reset
// or any other teardown of the primary context gives the next context a new identifier. The
// driver functions are reached through the runtime's entry-point query, so nothing links the
// driver library directly.
static unsigned long long current_context_id() {
    typedef CUresult (*CtxCur)(CUcontext*);
    typedef CUresult (*CtxId)(CUcontext, unsigned long long*);
    static CtxCur f_cur = nullptr;
    static CtxId f_id = nullptr;
    static bool looked = false;
    if (!looked) {
        looked = true;
        void* a = nullptr;
        void* b = nullptr;
        cudaDriverEntryPointQueryResult qa, qb;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &a, 12000, cudaEnableDefault, &qa) == cudaSuccess &&
            qa == cudaDriverEntryPointSuccess)
            f_cur = (CtxCur)a;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &b, 12000, cudaEnableDefault, &qb) == cudaSuccess &&
            qb == cudaDriverEntryPointSuccess)
            f_id = (CtxId)b;
        cudaGetLastError();
    }
    CUcontext c = nullptr;
    unsigned long long id = 0;
    if (f_cur && f_id && f_cur(&c) == CUDA_SUCCESS && c && f_id(c, &id) == CUDA_SUCCESS) return id;
    return 0;
}

// Device address of the scratch array, looked up with the device current when a device is
// first used, and again whenever its context has changed since (host code may not use the
// symbol itself: in host code it names a host-side stand-in, not device memory).
static void* g_na_ptr[64];
static unsigned long long g_na_ctx[64];
static int na_scratch(int dev, unsigned char** out) {
    if (dev < 0 || dev >= 64) return WMCD_ECUDA;
    const unsigned long long ctx = current_context_id();
    if (!g_na_ptr[dev] || ctx != g_na_ctx[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) { cudaGetLastError(); return WMCD_ECUDA; }
        g_na_ptr[dev] = p;
        g_na_ctx[dev] = ctx;
    }
    *out = (unsigned char*)g_na_ptr[dev];
    return WMCD_OK;
}

// cached mode table of the last (L, lambda_max, lcut)
static int h_modes[3 * kNaModes];
static double h_cdf[kNaModes];
static int h_nmodes = 0;
static double h_key[3] = {-1.0, -1.0, -1.0};
// host staging of the call's small inputs (copied to the device before the call returns)
static uint8_t h_bnext[kNaBeads];
static int h_carry[4];
static SimView h_view;
static uint64_t h_step[2];

}  // namespace wmcd

using namespace wmcd;

extern "C" int wmcd_planewave_noalloc(const wmcd_params* params, double* pos, const int32_t* chain_len,
                                      int64_t n_chains, int64_t call_index, int32_t* carry, int64_t n_moves,
                                      void* stream) {
    if (!params || !pos || !chain_len || !carry || n_chains < 1 || n_moves < 0 || call_index < 0) return WMCD_EINVAL;
    // the checks of wmcd_create, then the limits of the static scratch
    if (validate_params(params)) return WMCD_EINVAL;
    const wmcd_params& P = *params;
    if (P.n_beads > kNaBeads) return WMCD_EINVAL;
    if ((int64_t)P.grid_f * P.grid_f * P.grid_f > kNaCells) return WMCD_EINVAL;
    if (P.planewave_mode != WMCD_PLANEWAVE_PERIODIC || P.lcut > kNaLcut) return WMCD_EINVAL;
    // the carried wave vector must be one of the mode table's (|l| <= lcut, not zero)
    if (carry[0] != 0 && carry[0] != 1) return WMCD_EINVAL;
    if (carry[0] == 1) {
        const int64_t c2 = (int64_t)carry[1] * carry[1] + (int64_t)carry[2] * carry[2] + (int64_t)carry[3] * carry[3];
        if (c2 == 0 || c2 > (int64_t)P.lcut * P.lcut) return WMCD_EINVAL;
    }
    // positions: device memory of the current device (or managed memory); another GPU's
    // memory is refused rather than read without peer access
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return WMCD_ECUDA; }
    cudaPointerAttributes pa;
    if (cudaPointerGetAttributes(&pa, pos) != cudaSuccess) { cudaGetLastError(); return WMCD_EINVAL; }
    if (pa.type != cudaMemoryTypeDevice && pa.type != cudaMemoryTypeManaged) return WMCD_EINVAL;
    if (pa.type == cudaMemoryTypeDevice && pa.device != dev) return WMCD_EINVAL;
    const int64_t N = P.n_beads;
    {
        int64_t tot = 0, b = 0;
        for (int64_t c = 0; c < n_chains; c++) if (chain_len[c] < 1) return WMCD_EINVAL; else tot += chain_len[c];
        if (tot != N) return WMCD_EINVAL;
        std::memset(h_bnext, 0, (size_t)N);
        for (int64_t c = 0; c < n_chains; c++) {
            for (int32_t k = 0; k + 1 < chain_len[c]; k++) h_bnext[b + k] = 1;
            b += chain_len[c];
        }
    }
    if (h_key[0] != P.box_L || h_key[1] != P.lambda_max || h_key[2] != (double)P.lcut) {
        h_nmodes = mode_table_static(P.box_L, P.lambda_max, P.lcut, h_modes, h_cdf, kNaModes);
        if (h_nmodes <= 0) return WMCD_EINVAL;
        h_key[0] = P.box_L; h_key[1] = P.lambda_max; h_key[2] = (double)P.lcut;
    }
    unsigned char* base = nullptr;
    int rc = na_scratch(dev, &base);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    SimView& v = h_view;
    std::memset(&v, 0, sizeof v);
    v.bead = (Bead*)(base + oBead);
    v.prev = (int*)(base + oPrev);
    v.img = (int*)(base + oImg);
    v.bnext = base + oBnext;
    v.head = (int*)(base + oHead);
    v.pw_new = (double*)(base + oPwNew);
    v.pw_imgd = (int*)(base + oPwImg);
    v.pw_part = (double*)(base + oPart);
    v.pw = (PWDev*)(base + oPw);
    v.ctr = (unsigned long long*)(base + oCtr);
    v.err = (int*)(base + oErr);
    v.pw_rebuild = (int*)(base + oRebuild);
    v.modes = (const int*)(base + oModes);
    v.mode_cdf = (const double*)(base + oCdf);
    v.n_modes = h_nmodes;
    v.tr_pw_cap = 0;                                      // no trace
    v.N = N;
    v.L = P.box_L;
    v.halfL = 0.5 * P.box_L;
    v.Gf = P.grid_f;
    v.invf = (double)P.grid_f / P.box_L;
    v.precision = P.precision;
    v.A0 = P.A0;
    v.kT = P.kT;
    v.rc = kWcaCut * P.wca_sigma;
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
    v.pw_blocks = (int)((N + 255) / 256);
    v.step = (uint64_t*)(base + oStep);
    v.counts = (int*)(base + oCounts);
    v.cl_stale = (int*)(base + oClStale);
    v.pw_on = 1;
    v.pw_mode = WMCD_PLANEWAVE_PERIODIC;
    v.pw_nl = P.lcut;
    SimView* dview = (SimView*)(base + oView);
    GroupDims g;
    g.S = 1;
    g.maxN = N;
    g.maxCells = (int64_t)P.grid_f * P.grid_f * P.grid_f;
    g.pw = true;
    g.pw_blocks = v.pw_blocks;
    g.prec_mask = 1 << P.precision;
    h_step[0] = 0;
    h_step[1] = (uint64_t)call_index;
    // inputs: bond flags, mode table, carry; zero what must start at zero
    h_carry[0] = carry[0]; h_carry[1] = carry[1]; h_carry[2] = carry[2]; h_carry[3] = carry[3];
    cudaMemcpyAsync(v.bnext, h_bnext, (size_t)N, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(base + oModes, h_modes, sizeof(int) * 3 * h_nmodes, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(base + oCdf, h_cdf, sizeof(double) * h_nmodes, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(dview, &v, sizeof(SimView), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(v.step, h_step, sizeof h_step, cudaMemcpyHostToDevice, s);
    cudaMemsetAsync(v.counts, 0, 4 * (kMaxLayers + 1), s);
    cudaMemsetAsync(v.cl_stale, 0, 4, s);
    cudaMemsetAsync(v.pw, 0, sizeof(PWDev), s);
    cudaMemcpyAsync(v.ctr, h_carry, sizeof h_carry, cudaMemcpyHostToDevice, s);   // carry staged in ctr[0..1]
    k_na_carry<<<1, 1, 0, s>>>(v.pw, (const int*)v.ctr);
    cudaMemsetAsync(v.ctr, 0, 8 * C_NCTR, s);
    cudaMemsetAsync(v.err, 0, sizeof(int), s);
    cudaMemsetAsync(v.img, 0, 12 * N, s);
    const int gb = (int)std::min<int64_t>((N + 255) / 256, 152 * 16);
    // refuse non-finite or out-of-box coordinates before anything runs on them
    k_na_check<<<gb, 256, 0, s>>>(pos, N, v.L, v.err);
    {
        int e0 = 0;
        cudaMemcpyAsync(&e0, v.err, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (cudaStreamSynchronize(s) != cudaSuccess) { cudaGetLastError(); return WMCD_ECUDA; }
        if (e0) return WMCD_ESTATE;
    }
    k_na_fill<<<gb, 256, 0, s>>>(v.bead, pos, N);
    launch_cl_rebuild(dview, g, s, 0);
    for (int64_t m = 0; m < n_moves; m++) launch_planewave(dview, g, 1, (int)m, s);
    k_na_read<<<gb, 256, 0, s>>>(v.bead, pos, N, v.err);
    // outputs: the carried wave vector, and the error flags
    int out[5] = {0, 0, 0, 0, 0};
    cudaMemcpyAsync(out, &v.pw->carry, sizeof(int) * 4, cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(out + 4, v.err, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) { cudaGetLastError(); return WMCD_ECUDA; }
    if (cudaGetLastError() != cudaSuccess) return WMCD_ECUDA;
    if (out[4] & E_NONFINITE) return WMCD_ESTATE;
    if (out[4] & E_WALK) return WMCD_ETIMEOUT;
    carry[0] = out[0]; carry[1] = out[1]; carry[2] = out[2]; carry[3] = out[3];
    return WMCD_OK;
}
