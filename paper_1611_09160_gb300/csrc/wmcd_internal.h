// Internal layout of a simulation's device state and the kernel launchers.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include "wmcd_device.cuh"

namespace wmcd {

// One bead record: 32 bytes, so a gather of a bead is one sector. `next` links the bead into
// the list of its fine cell; `mark` tags membership of the support of the current serial move.
struct __align__(32) Bead {
    double x, y, z;
    int next;
    uint32_t mark;
};
static_assert(sizeof(Bead) == 32, "bead record must be 32 bytes");

// binary32 shadow of a bead's position: hi = the binary64 coordinate rounded, lo = the rounded
// remainder, so hi + lo carries it to ~48 bits. Differences of nearby beads formed from the
// pairs carry about one binary32 ulp, with no binary64 arithmetic (slow on this part). Written
// with every position; read by the binary32 screens and energies.
struct __align__(32) BeadF {
    float hx, hy, hz, lx, ly, lz, pad0, pad1;
};
static_assert(sizeof(BeadF) == 32, "shadow record must be 32 bytes");

// write a bead's binary64 position and its binary32 shadow (if the view has one)
__device__ __forceinline__ void put_bead(Bead* bead, BeadF* bf, int64_t m, double x, double y, double z) {
    bead[m].x = x; bead[m].y = y; bead[m].z = z;
    if (bf) {
        BeadF f;
        f.hx = (float)x; f.hy = (float)y; f.hz = (float)z;
        f.lx = (float)(x - (double)f.hx); f.ly = (float)(y - (double)f.hy); f.lz = (float)(z - (double)f.hz);
        f.pad0 = 0.0f; f.pad1 = 0.0f;
        bf[m] = f;
    }
}

constexpr int kMaxLayers = 16;
constexpr int kNCap = 64;          // supports up to this size take sqrt(n) from a table
constexpr int kNCapMax = 256;      // largest n_cap: support of a concurrent move
constexpr int kWarpsPerBlock = 4;  // concurrent kernel: one warp per queue
constexpr int kSerialThreads = 512;
constexpr int kMaxWalk = 1 << 22;  // bound on list-walk iterations inside one move
constexpr int kStageWarps = 2;     // staged concurrent kernel: default warps per block
constexpr int kMaxStageWarps = 4;  // ... and the most a block may have
constexpr int kCandCap = 256;      // interaction candidates of one staged move held in shared memory
constexpr int kSlotChunk = 32;     // slot parameters prepared per chunk
constexpr int kSmemSerialMaxN = 2048;
constexpr int kSmemCand = 1024;    // interaction candidates of one shared-memory serial move
constexpr int kSmemThreads = 512;  // threads of the shared-memory serial block (many warps hide the
                                   // latency of the scans over all staged beads)  // largest simulation whose serial phase runs in shared memory

enum Outcome { ACCEPT = 1, REJECT = 2, DEFER = 3 };

// device counters
enum Ctr {
    C_ATT = 0, C_ACC = 16, C_DEF = 32, C_PWATT = 48, C_PWACC = 49, C_BU = 50, C_ACCTOT = 51, C_RECHECK = 52,
    C_PARTNER = 53, C_CBU = 54, C_CMOVED = 55, C_CPE = 56, C_MOVED = 57, C_NCTR = 64
};
// device error bits
enum Err { E_WALK = 1, E_SCRATCH = 2, E_NONFINITE = 4 };

struct LayerDev {
    double lo, hi, ilo3, ihi3;   // band [lo, hi) and its inverse cubes
    double invG;                 // G / L
    double expect;               // expected slots per sweep, N (1 - P_F) p_l
    int Mmax;                    // floor(expect) + 1: bound on the slots of one sweep
    int G;                       // coarse cells per axis, 0 = serial layer
    int carry_off;               // offset of this layer's per-cell carries
    int64_t tr_off;              // offset of this layer's trace
    // second colouring of the slots the layer defers: G2 = K floor(G / 2K) cells per axis
    // (0 = none), their carries at carry_off2
    int G2, carry_off2;
    double invG2;
};
// The schedule index of a layer's second colouring: its phases run kernels written for a layer
// with the index kMaxLayers + l (grid G2, carries at carry_off2, supports up to kNCapMax beads;
// random draws, counters and trace those of layer l).
constexpr int kLevel2 = kMaxLayers;
WMCD_HD int layer_real(int l) { return l >= kLevel2 ? l - kLevel2 : l; }

// The serial move of a large-scale layer that runs on the whole GPU, one kernel per step.
struct BigMove {
    int active;                  // this slot exists in the current sweep
    int j, n, acc;               // slot, support size (gathered), decision
    int nch;                     // members of the accepted move that change fine cell
    uint32_t tag;                // support mark of this move
    double lam, thr, b[3], p[3];
};

// Audit of the mixed-precision decisions (a checking switch, off by default): with it on, every
// binary32 decision also evaluates the binary64 energy change, and the pair (with the band and
// the threshold) is counted and recorded. The decision itself is taken exactly as without it.
struct AuditDev {
    unsigned long long n;        // mixed-precision decisions audited
    unsigned long long outside;  // of which taken in binary32 (|dU32 - thr| above the band)
    unsigned long long viol;     // |dU32 - dU64| at or above the band
    unsigned long long flip;     // taken in binary32 with an outcome the binary64 value would not give
    unsigned int max_ratio;      // bits of the largest |dU32 - dU64| / band (a non-negative float)
    unsigned int pad;
    double* rec;                 // 4 per record: dU32, dU64, band, threshold (the first `cap` decisions)
    long long cap;
};

// |k| table of the infinite system and the quasi-continuous shell: F(Q), Q = |k| lambda_max,
// on Q_i = i kKtH, i = 0..kKtN
constexpr int kKtN = 8192;
constexpr double kKtH = 3.141592653589793 / 128.0;

struct PWDev {
    int lv[3];
    int cont;                    // continuous wave vector (infinite system)
    double kh[3], Q, kappa;      // ... its unit direction, |k| lambda_max, turns per unit length
    double carry_Q;              // recycled |k| lambda_max (infinite system)
    int null_move;               // k = 0
    int accept;
    int mode_packed;
    double AF, phi, e[3];
    double reach;                // partner search reach rc + 2 |A_F|
    int carry, carry_l[3];       // recycled |k| after a rejection
    int active;                  // this plane-wave slot exists in the current sweep / call
};

struct SimView {
    // beads and cell list
    Bead* bead;
    BeadF* bf;                   // binary32 shadow of the positions (null: none)
    int* prev;
    int* img;                    // 3 per bead
    uint8_t* bnext;              // bead i bonded to i + 1
    int* head;                   // Gf^3 fine cells, -1 = empty
    uint32_t* occ;               // occupancy bits of the fine cells: row (y, z) holds occ_w words,
                                 // bit x of the row set iff head[x + Gf (y + Gf z)] != -1 (null: none)
    int occ_w;                   // words per row, ceil(Gf / 32)
    int64_t N;
    double L, halfL, invf;
    int Gf, K, n_cap, precision;
    double A0, kT, r_reach, rc;
    Pot pot;
    uint32_t k0, k1;
    int nL;
    LayerDev layer[kMaxLayers];
    uint64_t* step;              // [0] sweep counter, [1] direct plane-wave call counter
    int* counts;                 // slots of the current sweep: [l] layer l, [kMaxLayers] plane waves
    double expect_F;             // expected plane-wave slots per sweep, N P_F
    int pw_on;                   // plane waves enabled
    int pw_mode;                 // 1 sphere |l| <= lcut, 2 cube + quasi-continuous shell, 3 infinite system
    int pw_nl;                   // cube half-width N_layers (mode 2)
    double p_disc;               // probability of the discrete cube (mode 2)
    double kF0;                  // F at the shell's inner edge (mode 2)
    const double* kF;            // the |k| table (modes 2, 3)
    double* tr_pw_k;             // 3 per traced plane wave: wave vector in units of 2 pi / L
    // schedule scratch (sized for the largest layer)
    double* slot_lam;
    int* slot_bead;
    double* slot_V;              // serial phase: 3 per slot, centre offset in the unit ball
    double* slot_p;              // 3 per slot, unit polarisation
    double* slot_thr;            // per slot, Metropolis threshold -kT ln(1 - u)
    int* slot_key;
    int* q_count;
    int* q_start;
    int* q_fill;
    int* q_slots;
    uint8_t* defer;
    int* serial_list;
    int* serial_count;
    double* carry_q;
    double* carry_serial;
    // trace of the last sweep
    uint8_t* tr_out;
    int* tr_n;
    double* tr_du;               // energy change used for each decision
    uint8_t* tr_pw_out;
    int* tr_pw_mode;
    int* tr_pw_count;
    int tr_pw_cap;
    // counters and errors
    unsigned long long* ctr;
    int* err;
    // staging of the beads of each region of one colour (concurrent kernel)
    int* rkey;                   // per bead: queue whose region interior holds it, -1 = none
    int* rcount;                 // per queue
    int* rstart;
    int* rfill;
    int* rlist;                  // bead ids grouped by queue
    const int* axis_tab;         // per layer, per colour offset, per fine cell: queue coordinate or -1
    int* hq_list;                // queues of the current colour phase with dense regions
    int* hq_ctl;                 // [0] how many up to the middle size (front of the list), [1] their work
                                 // counter, [2] how many larger (back of the list), [3] their counter
    int stage_cap;               // beads a warp can stage in shared memory
    // serial-phase scratch (n up to N)
    int* s_ids;
    double* s_d;                 // 4 per member: offset from the centre and its square
    double* s_new;               // 3 per member: new wrapped position
    int* s_img;                  // per member: packed image change
    int* s_slot;                 // per bead: index in the support of the current serial move
                                 // (between moves: ranks of the region scatter)
    int* s_changed;              // members whose fine cell changes
    int* s_box;                  // 6 per member: partner cell box (first cell, cells per axis)
    int* s_pre;                  // n + 1: prefix of the partner-box sizes
    uint32_t* serial_tag;
    // plane waves
    PWDev* pw;
    double* pw_new;              // 3 per bead
    int* pw_imgd;                // per bead packed image change
    double* pw_part;             // per-block partial sums
    int* pw_rebuild;             // set by the commit when beads moved: the cell list is rebuilt
    int* cl_stale;               // set by the shared-memory serial phase when beads changed fine cell
    BigMove* big;
    int big_layers;              // bit l: layer l's moves run one at a time on the whole GPU
    int smem_layers;             // bit l: layer l's serial phase runs in shared memory (small N, no
                                 // coloured layer, small scales)
    int pw_blocks;
    const int* modes;            // 3 per mode
    const double* mode_cdf;
    int n_modes;
    AuditDev* audit;             // null: no audit of mixed-precision decisions
    int acceptance;              // 0 Metropolis, 1 Glauber
    int centring;                // 0 centre near a picked bead, 1 uniform in the box
};

// packed image change: three 2-bit fields holding -1, 0, +1 (as 0, 1, 2)
WMCD_HD int pack_img(int dx, int dy, int dz) { return (dx + 1) | ((dy + 1) << 2) | ((dz + 1) << 4); }
WMCD_HD void unpack_img(int p, int* d) { d[0] = (p & 3) - 1; d[1] = ((p >> 2) & 3) - 1; d[2] = ((p >> 4) & 3) - 1; }

// Launch bounds over the simulations of a group (one simulation, or a batch): every launch
// covers all of them (blockIdx.y = simulation) and kernels return early where a simulation has
// no work, so the launch sequence of a sweep is static and can be captured in a CUDA graph.
struct GroupDims {
    int S = 1;
    int64_t maxN = 1, maxCells = 1;
    int maxL = 0, maxK3 = 1, maxMF = 0, stage_cap = 256, pw_blocks = 1;
    // per schedule index: layer l, and kLevel2 + l for layer l's second colouring
    int cap_l[2 * kMaxLayers] = {0};  // staging capacity of a coloured layer when above stage_cap
    int ncap = kNCap;            // largest n_cap of the group (sizes the staged support arrays)
    int Mmax[2 * kMaxLayers] = {0}, keys[2 * kMaxLayers] = {0}, nq[2 * kMaxLayers] = {0};
    bool coloured[2 * kMaxLayers] = {false};
    bool pw = false;
    int prec_mask = 3;           // bit 0: some simulation runs in binary64, bit 1: some in mixed precision
    int block_warps = kStageWarps;  // warps (queues) per block of the staged concurrent kernel, 1..4
    int serial_threads = kSerialThreads;  // threads of the serial-phase block: 32, 128 or 512
    int64_t smem_maxN = 0;       // largest N among simulations with the shared-memory serial phase
    int64_t smem_cls[3] = {0, 0, 0};  // ... per size class (N <= 320, <= 1024, larger), 0 = none
    int bigM[kMaxLayers] = {0};  // slots of a whole-GPU layer (largest over the group), 0 = none
    bool any_global_serial = true;  // some simulation runs its serial phase through global memory
};

// ---- launchers (wmcd_kernels.cu) ----
void launch_cl_rebuild(const SimView* d, const GroupDims& g, cudaStream_t s, int use_flag);
void launch_counts(const SimView* d, const GroupDims& g, cudaStream_t s);
void launch_advance(const SimView* d, const GroupDims& g, int which, cudaStream_t s);
void launch_slots(const SimView* d, const GroupDims& g, int l, cudaStream_t s);
void launch_bucket(const SimView* d, const GroupDims& g, int l, cudaStream_t s);

void launch_defer_compact(const SimView* d, const GroupDims& g, int l, cudaStream_t s);
// Side streams and events to run independent launches of a phase side by side (recorded as
// parallel branches of a graph); null members mean one stream.
struct ForkJoin {
    cudaStream_t side[2] = {nullptr, nullptr};
    cudaEvent_t fork = nullptr, join[2] = {nullptr, nullptr};
};
constexpr int64_t kSmemClassHi[3] = {320, 1024, 1 << 30};
// kernels launched; with side streams in fj the dense regions of the phase run beside the rest
int launch_colour_staged(const SimView* d, const GroupDims& g, int l, int colour, cudaStream_t s, const ForkJoin* fj);
int launch_serial(const SimView* d, const GroupDims& g, int l, cudaStream_t s, const ForkJoin* fj);  // kernels launched
int launch_planewave(const SimView* d, const GroupDims& g, int direct, int m, cudaStream_t s);
int launch_big(const SimView* d, const GroupDims& g, int l, int t, cudaStream_t s);     // kernels launched
size_t staged_smem_bytes(int cap, int warps, int ncap);
int staged_cap_max(int ncap);    // most beads one queue can stage (a block of one queue)
size_t smem_serial_bytes(int64_t n);
// open the kernels that take large dynamic shared memory for the sizes of g (before a graph
// capture: a recorded launch sets nothing)
void prepare_staged(const GroupDims& g);

}  // namespace wmcd
