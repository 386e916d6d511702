/*
 * wmcd.h — C ABI of the GB300 (sm_103a) Wavelet Monte Carlo dynamics library.
 *
 * Wavelet Monte Carlo dynamics (Dyer & Ball, arXiv:1611.09160) evolves N interacting
 * Brownian beads by Metropolis-accepted, spatially correlated moves: divergence-free
 * tapered-wavelet moves of scale lambda drawn from P_lambda ~ lambda^-4 (Secs. IV-V,
 * Eqs. 21-34, Appendix D) and, for a periodic box, plane-wave moves that carry the
 * longest-range correlations (Sec. VI, Eqs. 47-57). Their accumulated displacements
 * reproduce Oseen / Rotne-Prager hydrodynamics.
 *
 * Conventions for every entry point:
 *  - lengths are in units of the bead radius a, energies in the same units as kT;
 *  - positions are double[3 * n_beads], row-major (x, y, z per bead);
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream); all
 *    work is enqueued on it and is asynchronous unless stated otherwise;
 *  - a pointer argument documented "host or device" is classified with
 *    cudaPointerGetAttributes; host memory may be pageable or pinned;
 *  - the handle owns all device state; caller buffers are only borrowed for the call;
 *  - a handle is not thread-safe; different handles are independent;
 *  - every function returns 0 (WMCD_OK) or a negative wmcd_status; no C++ exception or
 *    CUDA error crosses the ABI. wmcd_strerror() turns a status into text.
 */
#ifndef WMCD_H
#define WMCD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum wmcd_status {
    WMCD_OK = 0,
    WMCD_EINVAL = -1,     /* bad argument or parameter (see wmcd_create) */
    WMCD_ENOMEM = -2,     /* device or host allocation failed */
    WMCD_ECUDA = -3,      /* a CUDA runtime call failed */
    WMCD_ETIMEOUT = -4,   /* a bounded device-side wait or list walk gave up */
    WMCD_ESTATE = -5,     /* non-finite positions or a corrupted cell list were detected */
    WMCD_EFULL = -6       /* a batch has no free slot, or its pool no room, for the simulation */
} wmcd_status;

enum { WMCD_BOND_NONE = 0, WMCD_BOND_HARMONIC = 1, WMCD_BOND_FENE = 2 };
/* Plane-wave moves (Sec. VI): OFF; PERIODIC, the modes |l| <= lcut of the periodic box,
 * normalised over that sphere; PERIODIC_FULL, the paper's periodic scheme (Appendix D): a
 * discrete cube |l_i| <= lcut (its N_layers, 15 in the paper) and the quasi-continuous region
 * outside it (|k| from P_k^inf restricted to the shell, snapped to the nearest mode, drawn again
 * inside the cube), normalised over all modes; INFINITE, the infinite system (Sec. VI.B): |k|
 * from P_k^inf (Eq. 52) by a tabulated inverse, k^ isotropic, P_F = (lambda_min/lambda_max)^3
 * (Eq. 54), the field applied at the unwrapped positions. */
enum { WMCD_PLANEWAVE_OFF = 0, WMCD_PLANEWAVE_PERIODIC = 1, WMCD_PLANEWAVE_PERIODIC_FULL = 2,
       WMCD_PLANEWAVE_INFINITE = 3 };
enum { WMCD_FP64 = 0, WMCD_MIXED = 1 };
enum { WMCD_ACCEPT_METROPOLIS = 0, WMCD_ACCEPT_GLAUBER = 1 };
enum { WMCD_CENTRE_BEAD = 0, WMCD_CENTRE_UNIFORM = 1 };
#define WMCD_MAX_LAYERS 16

/* Parameters of one simulation. */
typedef struct wmcd_params {
    int64_t n_beads;          /* N >= 1 */
    double box_L;             /* side of the periodic cube */
    double lambda_min;        /* smallest wavelet scale (sets the hydrodynamic radius, Eq. 42) */
    double lambda_max;        /* largest scale, lambda_min < lambda_max <= L/2 (Sec. V.C) */
    double A0;                /* move amplitude parameter A_w = A0 lambda / sqrt(n) (Eq. 29) */
    double kT;                /* thermal energy of the Metropolis test (Eq. 20) */
    int32_t bond_type;        /* WMCD_BOND_*: chain neighbours i, i+1 of one chain are bonded */
    double bond_k;            /* harmonic: U = (k/2)(r - r0)^2; FENE: Eq. 1 with k and R0 */
    double bond_r0;
    double fene_R0;
    double wca_sigma;         /* WCA repulsion (Eq. 2) between all pairs; eps = 0 disables */
    double wca_eps;
    double ext_kappa;         /* external well (kappa/2)|r - box centre|^2; 0 disables */
    int32_t planewave_mode;   /* WMCD_PLANEWAVE_*: plane-wave moves (Sec. VI) */
    int32_t lcut;             /* PERIODIC: modes k = (2 pi / L) l with |l| <= lcut (0..120);
                                 PERIODIC_FULL: N_layers of the discrete cube (0..40) */
    int32_t precision;        /* WMCD_FP64, or WMCD_MIXED: FP32 displacements and pair
                                 energies, FP64 positions, FP64 recheck near the threshold */
    uint64_t seed;            /* Philox key, with sim_id */
    uint64_t sim_id;
    /* concurrent schedule: moves of one layer run concurrently in K^3 colour phases over
       G^3 coarse cells; a move that does not fit its cell's region is deferred to a serial
       phase, so results do not depend on these values except through that order */
    int32_t colour_K;         /* colours per axis, 2..4 */
    int32_t grid_f;           /* fine (cell-list) cells per axis, L / grid_f >= WCA cutoff */
    int32_t n_cap;            /* largest support a concurrent move handles (1..256) */
    int32_t grid_layer[WMCD_MAX_LAYERS];  /* coarse cells per axis per layer; 0 = serial;
                                             otherwise a multiple of colour_K, at most 256 */
    int32_t big_support;      /* a serial layer whose expected support (N times the volume of a
                                 ball of the layer's middle scale over L^3) reaches this many
                                 beads runs each of its moves on the whole GPU (Sec. VIII: large
                                 moves in parallel); 0 = 2048, negative = never. A launch choice:
                                 decisions do not depend on it */
    int32_t acceptance;       /* WMCD_ACCEPT_METROPOLIS (Eq. 20) or WMCD_ACCEPT_GLAUBER (Secs. V.C,
                                 VIII: accept with probability 1 / (1 + exp(dU / kT))) */
    int32_t centring;         /* WMCD_CENTRE_BEAD: b within lambda of a picked bead (Eq. 26,
                                 A_w of Eq. 29); WMCD_CENTRE_UNIFORM: b uniform in the box, A_w from
                                 the mean support at the global density (Sec. V.D) */
    int32_t level2;           /* bit l set: the slots coloured layer l defers get a second
                                 colouring on K floor(G / 2K) coarse cells per axis (regions twice
                                 as wide, supports up to 256 beads) before the serial phase, where
                                 that leaves at least 2K cells; 0 = none (0..0xffff). Part of the
                                 schedule: it changes the order of moves as the grid does */
} wmcd_params;

/* Counters since creation (or the last wmcd_set_state). */
typedef struct wmcd_stats_t {
    int64_t attempts[WMCD_MAX_LAYERS];   /* wavelet moves attempted, per layer */
    int64_t accepts[WMCD_MAX_LAYERS];
    int64_t deferred[WMCD_MAX_LAYERS];   /* concurrent attempts sent to the serial phase */
    int64_t pw_attempts, pw_accepts;     /* plane-wave moves (k = 0 counts as accepted) */
    int64_t bead_updates;                /* sum of support sizes n, plus N per k != 0 plane wave */
    int64_t accepted_total;              /* all accepted moves: simulated time = this * dt_move */
    int64_t rechecks;                    /* mixed precision: moves re-decided in FP64 */
    int64_t partner_evals;               /* pair evaluations with beads outside the support */
    double sim_time;                     /* in units of tau = pi eta a^3 / kT (Eq. 3) */
    int64_t sweeps;
    int64_t n_layers;
    double dt_move;                      /* Eq. 57 with plane waves, Eq. 34 without */
    double p_fourier;                    /* probability of a plane-wave move (Eq. 56) */
    int32_t error_flags;                 /* device-side error bits, 0 = none */
    int64_t kernel_launches;             /* kernels this library has launched */
    int64_t conc_bead_updates;           /* bead updates done by the concurrent wavelet kernel */
    int64_t conc_moved_beads;            /* beads written back by accepted concurrent moves */
    int64_t conc_partner_evals;          /* its pair evaluations with beads outside the support */
    int64_t moved_beads;                 /* beads moved by accepted moves of every kind (support
                                            sizes of accepted wavelets, N per accepted plane wave) */
} wmcd_stats_t;

typedef struct wmcd_handle wmcd_handle;

/* Create a simulation. pos: N*3 doubles (host or device), each coordinate in [0, L).
 * chain_len: n_chains int32 (host), the lengths of consecutive runs of bead ids that form
 * chains (free beads are chains of length 1); the lengths must sum to N.
 * Validates: N >= 1; 0 < lambda_min < lambda_max <= L/2; A0 > 0; kT > 0; colour_K in 2..4;
 * grid_f >= 1 with L/grid_f >= the WCA cutoff 2^(1/6) sigma (when WCA is on);
 * 1 <= n_cap <= 256; each grid_layer[l] is 0 or a multiple of colour_K in [colour_K, 256];
 * at most 16 octave layers; level2 in 0..0xffff; planewave_mode 0..3, lcut in 0..120 (PERIODIC) or 0..40
 * (PERIODIC_FULL). Returns WMCD_EINVAL otherwise.
 * Synchronises `stream` before returning. *out receives the handle. */
int wmcd_create(const wmcd_params* params, const double* pos, const int32_t* chain_len, int64_t n_chains,
                void* stream, wmcd_handle** out);

/* Advance by n_sweeps sweeps. A sweep = the octave layers of P_lambda (Eq. 32) in ascending
 * order, each with floor(N (1 - P_F) p_l) slots plus one more with probability of the
 * fraction (P_F of Eq. 56), run as colour phases then a serial phase; then the sweep's
 * plane-wave slots (Sec. VI). Each slot is one move generated as in Appendix D (scale by
 * inverse transform within the band, bead, centre, polarisation; lambda recycled after a
 * rejection) and decided by the Metropolis test of Eq. 20. Asynchronous. */
int wmcd_sweep(wmcd_handle* h, int64_t n_sweeps, void* stream);

/* n_moves plane-wave moves (Sec. VI) outside the sweep schedule, one after another, with
 * their own random stream. Needs planewave_mode = PERIODIC. Asynchronous. */
int wmcd_planewave(wmcd_handle* h, int64_t n_moves, void* stream);

/* Copy positions to `out` (N*3 doubles, host or device); unwrapped != 0 adds the periodic
 * image counters times L. Synchronises `stream` when `out` is host memory. */
int wmcd_positions(wmcd_handle* h, double* out, int unwrapped, void* stream);

/* Replace the positions (N*3 doubles in [0, L), host or device) and zero the image counters;
 * rebuilds the cell list. Carries, counters and the sweep index are kept. Asynchronous for
 * device input; host input is copied before return. */
int wmcd_set_positions(wmcd_handle* h, const double* pos, void* stream);

/* Synchronises `stream`, then fills *out. */
int wmcd_stats(wmcd_handle* h, wmcd_stats_t* out, void* stream);

/* Per-slot outcome of the last sweep, for layer `layer` (wavelet moves) or layer = -1
 * (that sweep's plane-wave moves): out[j] = 1 accepted / 2 rejected, +4 when a concurrent
 * attempt was deferred and ran in the serial phase; n[j] = support size (plane waves: the
 * wave vector packed as (lx+128) | (ly+128) << 8 | (lz+128) << 16, or -1 when a component is
 * beyond 127 or the system is infinite: see wmcd_trace_pw_k). Buffers are host memory of `cap`
 * entries; *count receives the number of slots. Synchronises `stream`. */
int wmcd_trace(wmcd_handle* h, int layer, uint8_t* out, int32_t* n, int64_t cap, int64_t* count, void* stream);

/* Energy change behind each wavelet decision of the last sweep, layer `layer` (host buffer of
 * `cap` doubles, *count receives the number of slots; 0 where the support was empty). A
 * deferred slot records the value of its serial attempt. In mixed precision the value is the
 * binary32 sum when that decided, the binary64 recheck otherwise. Synchronises `stream`. */
int wmcd_trace_du(wmcd_handle* h, int layer, double* out, int64_t cap, int64_t* count, void* stream);

/* Wave vectors of the plane waves of the last sweep (or of the last wmcd_planewave call), in
 * units of 2 pi / L: the integer mode l for the periodic schemes, the continuous k L / (2 pi)
 * for the infinite system. out: host, 3 doubles per move, `cap` moves; *count receives the
 * number of moves. Synchronises `stream`. */
int wmcd_trace_pw_k(wmcd_handle* h, double* out, int64_t cap, int64_t* count, void* stream);

/* Checkpoint: the state is positions, image counters, carries, the sweep and plane-wave
 * call counters and the statistics. wmcd_state_size gives the byte size; get writes it to
 * a host buffer, set restores it. With the counter-based random stream a restored run
 * continues bit-identically. Both synchronise `stream`. */
int wmcd_state_size(wmcd_handle* h, int64_t* bytes);
int wmcd_get_state(wmcd_handle* h, void* buf, int64_t bytes, void* stream);
int wmcd_set_state(wmcd_handle* h, const void* buf, int64_t bytes, void* stream);

/* Per-kernel timing: when enabled, the library records CUDA events around every launch of
 * its concurrent wavelet kernel, serial kernel and plane-wave kernels on `stream`;
 * wmcd_kernel_times synchronises and returns (launches, total milliseconds) for the
 * kernel classes 0 = concurrent wavelet, 1 = serial wavelet, 2 = plane wave, 3 = cell list,
 * 4 = schedule (slots and bucketing), 5 = serial moves of large scale run on the whole GPU. */
int wmcd_profile(wmcd_handle* h, int enable);
int wmcd_kernel_times(wmcd_handle* h, int64_t* launches, double* ms, int n_classes, void* stream);

/* Audit of the mixed-precision decisions (a checking switch; the paper has no counterpart:
 * it checks this library's precision scheme). With the audit on, every move decided in mixed
 * precision also evaluates its binary64 energy change dU64 beside the binary32 one dU32, and
 * the library counts: decisions; those taken in binary32 (|dU32 - threshold| above the error
 * band); violations, |dU32 - dU64| at or above the band; flips, binary32 decisions whose
 * outcome dU64 would not give. The decisions themselves, and so the trajectory, are exactly
 * those without the audit; only the binary64 work is added. wmcd_audit(h, capacity) turns it
 * on with counters reset and room for the first `capacity` records (allocates; capacity >= 0)
 * or off (capacity < 0); synchronises `stream`. wmcd_audit_read fills *out and copies up to
 * `cap` records (4 doubles each: dU32, dU64, band, binary64 threshold -kT ln(1 - u)) to the
 * host buffer `rec`; WMCD_EINVAL if the audit was never turned on. Synchronises `stream`. */
typedef struct wmcd_audit_t {
    int64_t decisions, outside, violations, flips;
    double max_ratio;                    /* largest |dU32 - dU64| / band over the decisions */
    int64_t records;                     /* records kept: min(decisions, capacity) */
} wmcd_audit_t;
int wmcd_audit(wmcd_handle* h, int64_t capacity, void* stream);
int wmcd_audit_read(wmcd_handle* h, wmcd_audit_t* out, double* rec, int64_t cap, void* stream);

/* Device bytes held by the handle. */
int wmcd_device_bytes(wmcd_handle* h, int64_t* bytes);

/* Plane-wave moves on caller-owned device positions without allocating anything (the paper
 * has no counterpart: this is a deployment variant of wmcd_planewave). For callers that may not
 * call cudaMalloc, e.g. code running while another framework owns the device memory, real-time
 * loops that must not allocate after start-up, or hosts that forbid allocation in callbacks.
 * params: checked as by wmcd_create, plus the limits below. pos: N*3 doubles in device memory
 * of the current device (or managed memory), coordinates in [0, L), replaced in place by the
 * positions after n_moves moves (wrapped; no image counters). chain_len: host, as for
 * wmcd_create. call_index: the plane-wave call counter (0 for the first call, then 1, 2, ...);
 * carry: host int32[4], the recycled wave vector (carry[0] = 1 means carry[1..3] is carried,
 * 0 means none), read and updated; a carried vector must be nonzero with |l| <= lcut. With the
 * same params, positions, call_index and carry the result equals n_moves moves of
 * wmcd_planewave on a handle whose plane-wave call counter is call_index.
 * Errors: WMCD_EINVAL for parameters, carry or a pointer that is not memory of the current
 * device; WMCD_ESTATE for a non-finite or out-of-box coordinate (found before anything runs);
 * WMCD_ETIMEOUT when a bounded cell-list walk gave up. On any error `pos` and `carry` are left
 * unchanged.
 * Scratch: one file-scope device array of about 1.9 MB that every GPU loading the library
 * holds until exit; limits N <= 16384, grid_f^3 <= 48^3, lcut <= 8, plane waves periodic,
 * else WMCD_EINVAL. The first call on a device (and the first after its context was torn
 * down, e.g. by cudaDeviceReset) looks the array up (cudaGetSymbolAddress): make that call
 * before any stream capture. All calls share the array, so calls that overlap on the GPU
 * (other streams or threads) race; the function is not thread-safe. No cudaMalloc, cudaFree
 * or allocating library call is made. Synchronises `stream`. */
int wmcd_planewave_noalloc(const wmcd_params* params, double* pos, const int32_t* chain_len, int64_t n_chains,
                           int64_t call_index, int32_t* carry, int64_t n_moves, void* stream);

/* Launch shapes: warps per block of the concurrent wavelet kernel (one coarse-cell queue per
 * warp), 1..4, lowered where the block's shared memory would exceed 227 KB (default 2; a layer
 * whose regions need a block each runs one queue per block on 4 cooperating warps whatever this
 * is); and threads of the serial-phase block, 32, 128 or 512 (default 512). Choices of launch
 * shape only: decisions and positions do not depend on them (an energy change is summed in
 * another order, which moves it by rounding). WMCD_EINVAL for other values. */
int wmcd_set_block(wmcd_handle* h, int stage_warps, int serial_threads);

/* Releases the handle and its device state. WMCD_EINVAL for a handle a batch owns. */
int wmcd_destroy(wmcd_handle* h);
const char* wmcd_strerror(int status);

/* ---- batches (many simulations, one launch per phase) and serving --------------------
 * A batch keeps up to `capacity` independent simulations (any N, box, parameters, precision)
 * resident on the current device and advances all of them together: every phase of a sweep
 * (slot generation, bucketing, each colour, the serial phase, each plane-wave slot) is one
 * kernel launch over all resident simulations, and the whole sweep is recorded once as a CUDA
 * graph, which wmcd_batch_step replays. Each simulation's random stream, schedule and
 * reduction order are its own, so a simulation follows exactly the trajectory it follows
 * alone under wmcd_sweep, whatever else is in the batch (Sec. V-VIII order per simulation).
 *
 * Device memory: the batch reserves one pool of `pool_bytes` at creation and places each
 * admitted simulation's whole state in one block of it (first fit, blocks merged on release);
 * admission fails with WMCD_EFULL when no slot is free or no free block is large enough.
 *
 * Streams: admission runs on a stream of the batch's own, so it overlaps with steps already
 * queued on the caller's stream, and returns when the new state is on the device. Steps are
 * asynchronous on `stream`. Retiring synchronises `stream` before the memory is reused.
 * Not thread-safe. */
typedef struct wmcd_batch wmcd_batch;
int wmcd_batch_create(int capacity, int64_t pool_bytes, wmcd_batch** out);
/* pool bytes a simulation with these parameters takes (its state placed in one block) */
int wmcd_batch_need(const wmcd_params* params, int64_t* bytes);
/* admit a simulation (arguments as wmcd_create); *slot receives its slot id, 0..capacity-1 */
int wmcd_batch_admit(wmcd_batch* b, const wmcd_params* params, const double* pos, const int32_t* chain_len,
                     int64_t n_chains, int* slot);
/* n_sweeps sweeps of every resident simulation, one graph launch per sweep */
int wmcd_batch_step(wmcd_batch* b, int64_t n_sweeps, void* stream);
/* the handle of a resident simulation (borrowed, valid until retired): positions, stats,
 * trace and checkpoint calls work on it as on a lone simulation */
int wmcd_batch_handle(wmcd_batch* b, int slot, wmcd_handle** h);
/* release a simulation's slot and pool block (synchronises `stream` first) */
int wmcd_batch_retire(wmcd_batch* b, int slot, void* stream);
/* launch shapes for the whole batch (as wmcd_set_block); the graph is recorded again */
int wmcd_batch_set_block(wmcd_batch* b, int stage_warps, int serial_threads);
/* resident simulations, free pool bytes, largest free block, and kernel launches (graph
 * nodes) per batched sweep (0 before the first step after a change) */
int wmcd_batch_info(wmcd_batch* b, int64_t* resident, int64_t* pool_free, int64_t* largest_free,
                    int64_t* launches_per_sweep);
/* per-kernel timing of batched sweeps (as wmcd_profile / wmcd_kernel_times): while enabled,
 * steps launch the sweep kernel by kernel with CUDA events around each class instead of
 * replaying the graph */
int wmcd_batch_profile(wmcd_batch* b, int enable);
int wmcd_batch_kernel_times(wmcd_batch* b, int64_t* launches, double* ms, int n_classes, void* stream);
/* releases every resident simulation and the pool */
int wmcd_batch_destroy(wmcd_batch* b);

#ifdef __cplusplus
}
#endif
#endif /* WMCD_H */
