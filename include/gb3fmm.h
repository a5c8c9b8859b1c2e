/*
 * gb3fmm.h -- C ABI of the GB300 fast multipole method for unsoftened gravity
 * (Dehnen, "A fast multipole method for stellar dynamics", arXiv 1405.2255).
 *
 * The library computes, for N particles with positions x_b and masses mu_b,
 * the (negative) potential and the acceleration of eq. (1):
 *
 *     psi_b = sum_{a != b} G mu_a / |x_b - x_a|,      acc_b = grad psi_b
 *           = sum_{a != b} G mu_a (x_a - x_b) / |x_a - x_b|^3,
 *
 * approximated by the FMM of Sec. 2 (P2M, M2M, dual tree walk with M2L and P2P,
 * L2L, L2P) under the error-balanced multipole-acceptance criteria of
 * eqs. (18a,b).  The free parameters are the expansion order p and the accuracy
 * parameter eps (Sec. 6).  psi is the paper's Psi: it is POSITIVE, the physical
 * potential is -psi.
 *
 * Conventions for every call:
 *   - Return 0 on success or a negative FMM_E_* code.  No C++ exception crosses
 *     the ABI.  fmm_last_error(ctx) gives a one-line description of the last
 *     failure on that context.
 *   - Particle arrays are array-of-structures FP64: x[n][3] (x, y, z of particle i
 *     at x[3i..3i+2]), mu[n], psi[n], acc[n][3], in the caller's particle order.
 *   - Pointers documented as "device" must point to memory of the context's
 *     device (cudaMalloc'd, or torch tensors' data_ptr()).  Pointers documented as
 *     "host" are ordinary CPU memory.  The caller owns all input and output
 *     buffers; the context owns its workspace (tree, expansions, lists).
 *   - `stream` is a cudaStream_t (NULL: the legacy default stream).  Device
 *     calls are asynchronous with respect to the host unless stated otherwise;
 *     inputs must stay valid until the stream has reached the call's end.  An
 *     evaluation forks independent parts of its work onto three streams of the
 *     context (the upward pass beside the scale estimate, whose own M2L and P2P
 *     branches run side by side; later the P2P beside the M2L and downward pass)
 *     and joins them back into `stream` with events before
 *     it goes on, so everything the call does is ordered before work queued later
 *     on `stream`.
 *   - A context is not thread-safe: one host thread at a time per context.
 */
#ifndef GB3FMM_H
#define GB3FMM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* error codes */
#define FMM_OK            0
#define FMM_E_INVALID    -1   /* NaN/Inf position, mu < 0, p outside [1,20], eps <= 0, bad sizes */
#define FMM_E_OOM        -2   /* device allocation failed */
#define FMM_E_ADMISSION  -3   /* serving: footprint above the context's memory budget */
#define FMM_E_CUDA       -4   /* a CUDA runtime call failed */
#define FMM_E_TIMEOUT    -5   /* a bounded device or host wait ran out */
#define FMM_E_OVERFLOW   -6   /* an internal capacity could not be grown */
#define FMM_E_NOTFOUND   -7   /* unknown system id or ticket */
#define FMM_E_BUSY       -8   /* not finished yet (fmm_poll), or a request already in flight */

/* multipole-acceptance criteria */
#define FMM_MAC_A      0  /* eq. (18a): theta<1 and E~ M_A/r^2 < eps min_{b in B} a_b  */
#define FMM_MAC_F      1  /* eq. (18b): theta<1 and E~ M_A/r^2 < eps min_{b in B} f_b  */
#define FMM_MAC_THETA  2  /* eq. (9):   theta < theta_crit (geometric, for tests)       */

/* arithmetic of the path */
#define FMM_PREC_FP64   0  /* every step in IEEE FP64                                   */
#define FMM_PREC_MIXED  1  /* P2P in FP32 on two-float positions with compensated
                              accumulation; expansion terms of order > 2 (> 1 in the
                              rotated M2L) in FP32 on radius-scaled harmonics
                              (m2l_split, m2l_rot); the acceleration estimate's M2L in
                              FP32; everything else FP64.  Computed in units in which
                              the extent and the largest mass are of order one (exact
                              powers of two), so the results do not depend on the
                              caller's units                                          */

/* source of the acceleration scale used by (18a)/(18b) */
#define FMM_SCALE_ESTIMATE 0  /* low-order FMM estimate (Sec. 5.3.2)                  */
#define FMM_SCALE_CALLER   1  /* per-particle scale array passed to fmm_evaluate      */

typedef struct {
    int    p;           /* expansion order, 1..20 (Sec. 2.1)                          */
    double eps;         /* accuracy parameter of eqs. (18a,b), > 0                     */
    int    mac;         /* FMM_MAC_*                                                   */
    double theta_crit;  /* opening angle for FMM_MAC_THETA, in (0,1)                   */
    int    leaf_size;   /* a cell holding more particles is split (1..4096)            */
    double p2p_c;       /* a pair (A,B) is summed directly when N_A N_B < p2p_c p^3     */
    int    precision;   /* FMM_PREC_*                                                  */
    int    scale_src;   /* FMM_SCALE_*                                                 */
    int    p2p_two_float; /* mixed P2P, how dx = x_a - x_b is formed in FP32:
                             1 = per source cell A of sink leaf B: if A may hold a source
                             closer than rho_B to a sink (|s_A - s_B| < rho_A + 2 rho_B),
                             dx = (h_a - h_b) + (l_a - l_b) from the two-float positions
                             (hi + lo); otherwise from FP32 offsets to B's centre c,
                             (h - c_h) + (l - c_l), formed once per staged tile (default);
                             2 = offsets for every source; 3 = two-float for every source;
                             0 = from the FP32 high parts only                           */
    int    m2l_split;   /* mixed mode M2L: 1 = terms of order n+k <= 2 in FP64 and the others
                           in FP32 on scaled harmonics; 0 = every term in FP64        */
    int    m2l_rot;     /* mixed mode M2L with m2l_split, 3 <= p <= 16: 1 = the terms of order
                           n+k >= 2 in FP32 through rotations into the frame of the
                           interaction axis, the z-axis kernel eq. (A31) and the swap
                           matrices of App. A.5 (O(p^3) per pair), n+k <= 1 in FP64;
                           0 = eq. (3b) term by term (O(p^4)).  Same result up to FP32
                           rounding.                                                    */
    int    adaptive_p;  /* 1: every accepted M2L interaction takes the lowest order q in
                           [min(3, p), p] whose error estimate E~ (eq. 17 with order q)
                           meets the criterion (18a,b) (Sec. 7, opening); its M2L computes
                           F_n for n <= q from M_k, k <= q - n.  0: every interaction at p.
                           Only with FMM_MAC_A / FMM_MAC_F; fmm_evaluate_noalloc ignores it. */
} fmm_params;

typedef struct {
    /* counts of the last evaluation */
    int64_t n, ncells, nleaves, n_m2l, n_p2p, p2p_interactions, coincident;
    int64_t est_m2l, est_p2p;
    int     depth, p;
    double  eps;
    int     leaf_size;
    /* device time per phase in milliseconds (CUDA events).  Two pairs of phases run side by
       side on the context's streams: t_estimate and t_up both start at the end of the tree
       phase; t_walk starts once both are done; t_m2l and t_p2p both start at the end of the
       walk, t_down where t_m2l ends (on the M2L's stream); t_total spans the whole evaluation
       (the phases overlap, so they add up to more than it). */
    float   t_tree, t_estimate, t_up, t_walk, t_m2l, t_p2p, t_down, t_total;
    /* number of kernels the library launched for the evaluation */
    int64_t launches;
    /* device time in milliseconds of the main M2L kernel(s) of the rotated precision-split
       path and of the main mixed-precision P2P kernel alone (CUDA events recorded right
       before and after the launch; the phases above also hold their list sorts, work
       plans and reductions); 0 where that kernel did not run */
    float   t_m2l_kernel, t_p2p_kernel;
} fmm_stats;

typedef struct fmm_ctx fmm_ctx;

/* Default parameters: p = 8, eps = 1e-7, (18a) with the low-order estimate,
 * leaf_size = 64, p2p_c = 8, mixed precision with two-float P2P positions and
 * the precision-split, rotation-accelerated M2L.  Host pointer, filled in. */
void fmm_default_params(fmm_params* out);

/* Create a context on CUDA device `device` (the device becomes current for the
 * calling thread).  `params` (host, may be NULL for defaults) is copied.  The
 * context allocates its workspace lazily and keeps it for later calls. */
int fmm_create(fmm_ctx** out, const fmm_params* params, int device);

/* Replace the parameters of an existing context (host pointer, copied). */
int fmm_set_params(fmm_ctx* ctx, const fmm_params* params);

/* One force evaluation (Sec. 2.2.2; the phases of Table 2): tree build, scale
 * estimate, upward pass, dual tree walk, M2L, P2P, downward pass.
 *   n      number of particles, 0 <= n < 2^31 (0 is a no-op)
 *   x      device, [n][3] FP64 positions
 *   mu     device, [n] FP64 masses, >= 0
 *   G      gravitational constant (psi and acc scale with it)
 *   scale  device, [n] FP64 per-particle a_b (MAC_A) or f_b (MAC_F) when
 *          params.scale_src == FMM_SCALE_CALLER, else ignored (may be NULL)
 *   psi    device, [n] FP64 out: potential (positive, eq. 1)
 *   acc    device, [n][3] FP64 out: acceleration
 *   stream cudaStream_t or NULL
 *   stats  host, may be NULL: counts and phase times (filling it synchronises
 *          the stream)
 * The call returns once the work is queued, or after the stream is synchronised
 * when stats != NULL.  The tree build reads a handful of counts back to the
 * host, so the call always waits for the tree phase of its own stream.
 * Pairs at distance 0 contribute nothing and are counted in stats->coincident.
 * FMM_E_INVALID is returned for NaN/Inf positions or negative masses (checked on
 * the device; outputs are left unspecified in that case). */
int fmm_evaluate(fmm_ctx* ctx, int64_t n, const double* x, const double* mu, double G,
                 const double* scale, double* psi, double* acc, void* stream, fmm_stats* stats);

/* As fmm_evaluate, but x, mu, psi and acc are HOST pointers; the context copies
 * the inputs to its own device buffers and the outputs back, and synchronises
 * the stream before returning (the end-to-end call). */
int fmm_evaluate_host(fmm_ctx* ctx, int64_t n, const double* x, const double* mu, double G,
                      double* psi, double* acc, void* stream, fmm_stats* stats);

/* Direct summation of eq. (1) (and f_b of eq. (6) if f != NULL) on the GPU in
 * FP64 for the sinks listed in `sinks` (device int64 [nsinks] indices into the
 * n sources; NULL means all n particles are sinks, nsinks ignored).  Outputs
 * psi [nsinks], acc [nsinks][3], f [nsinks] (device; f may be NULL) in the
 * order of `sinks`.  Coincident pairs are skipped. */
int fmm_direct(fmm_ctx* ctx, int64_t n, const double* x, const double* mu, double G,
               int64_t nsinks, const int64_t* sinks, double* psi, double* acc, double* f,
               void* stream);

/* The general evaluation: forces for a subset of the particles, individual accuracy
 * parameters and a re-cycled tree, each optional.
 * Subset (Sec. 7.1: block time steps).  All n particles act as sources; active (DEVICE,
 * n bytes, caller order, NULL = all) marks the sinks: psi[i] and acc[i] are written for
 * active[i] != 0 only and left untouched otherwise.  The tree and
 * the upward pass cover all particles; the walk drops every cell pair whose sink cell
 * holds no active particle, so M2L, P2P, L2L and L2P run for the active part of the tree
 * only.  The MAC scale of a sink cell (eqs. 18a,b) is the minimum over its ACTIVE
 * particles, and the low-order estimate of Sec. 5.3.2 is evaluated for the active sinks:
 * the error criterion concerns the forces being computed.  With every particle active
 * the result equals fmm_evaluate's bit for bit.
 * Individual accuracy (Sec. 7, opening): eps_b (DEVICE, n doubles > 0, caller order, NULL = the
 * global eps) replaces eps min_{b in B} a_b in (18a) (f_b in 18b) by min_{b in B} eps_b a_b;
 * ignored by the geometric criterion.  eps_b[i] = eps for all i gives the global result.
 * reuse_tree = 1 re-cycles the tree of the previous evaluation on ctx (the other
 * measure Sec. 7.1 names): it must have been a completed single-system evaluation
 * (fmm_evaluate, fmm_evaluate_host or fmm_evaluate_active) of the same n particles in the
 * same caller order.  The particle order, the cells and their expansion centres are
 * kept; the positions and masses are gathered in that order and the radii, masses and
 * centres of mass are recomputed exactly, so the MAC holds for the new positions (cells
 * need not be the key cubes of the new positions); multipoles, walk and everything after
 * them are recomputed.  With unchanged positions the result equals a fresh evaluation's
 * bit for bit.  reuse_tree = 0 builds the tree anew.  Other arguments and errors as for
 * fmm_evaluate; FMM_E_INVALID also for a non-positive or non-finite eps_b or for
 * reuse_tree = 1 without such a previous evaluation.
 * Tidal tensor (Sec. 7.4): tidal (DEVICE, [n][6] doubles, caller order, NULL = not computed)
 * receives T = grad grad Psi as (xx, xy, xz, yy, yz, zz), G applied, for the active particles:
 * the far part from the local expansion's Psi_2^m at the particle (T_xy = +Im Psi_2^2 / 2
 * with this library's harmonics; the paper prints the opposite sign), the near part as the
 * direct Hessian over the same sources as the particle's P2P (mixed mode: FP32 terms on
 * two-float positions with two-float sums; FP64 mode: FP64).  T is one order of the
 * expansion less accurate than a. */
int fmm_evaluate_active(fmm_ctx* ctx, int64_t n, const double* x, const double* mu, double G,
                        const double* scale, const unsigned char* active, const double* eps_b, int reuse_tree,
                        double* psi, double* acc, double* tidal, void* stream, fmm_stats* stats);

/* Many independent systems in one call (the batched ensemble).  System s holds
 * particles [offsets[s], offsets[s+1]) of x/mu/psi/acc (device arrays laid out as
 * for fmm_evaluate); offsets is a HOST int64 array of nsys+1 non-decreasing entries
 * starting at 0 (empty systems allowed, at most 2^31-1 particles in all); G is a
 * HOST array of nsys finite constants.  Systems share no interactions.  All systems
 * are evaluated together as one forest (one root per non-empty system, one set of
 * launches per phase); each system's tree, lists and results are those it gets
 * alone in fmm_evaluate with the same parameters (bit for bit).  The scale source
 * must be FMM_SCALE_ESTIMATE (or the MAC geometric).  Returns after the stream has
 * completed; stats (HOST, may be NULL) cover the whole forest.  Errors as for
 * fmm_evaluate, plus FMM_E_INVALID for bad offsets or G. */
int fmm_evaluate_batch(fmm_ctx* ctx, int nsys, const int64_t* offsets, const double* x,
                       const double* mu, const double* G, double* psi, double* acc,
                       void* stream, fmm_stats* stats);

/* ---------------------------------------------------------------- serving
 * A request loop for many independent systems (concurrent cluster simulations)
 * whose force requests arrive over time.  The paper has no counterpart: this is
 * the batching and admission around its evaluation.
 *
 * The context runs `slots` workers, each with its own stream and workspace.  A
 * free slot takes every queued request (in arrival order) whose summed footprints
 * fit its share budget/slots and evaluates them as one forest
 * (fmm_evaluate_batch), so results are bit for bit those of each system alone;
 * slots run concurrently on the device.  Requests arriving while others run wait
 * in the queue for the next free slot.
 *
 * fmm_serve_config: optional, before the first fmm_system_register (else
 *   FMM_E_BUSY).  budget_bytes = device memory the slots' workspaces may hold
 *   (0: 80 % of the device's free memory at the first registration); slots in
 *   [0, 16] (0: 2).
 * fmm_footprint_bytes: the workspace bound used for admission, for n particles
 *   and the given parameters (NULL: defaults); -1 for invalid arguments.
 * fmm_system_register: a system of n particles (fixed for its lifetime);
 *   FMM_E_ADMISSION if its footprint exceeds one slot's share.  *sys_id >= 0.
 * fmm_submit: one force request: x [n][3], mu [n] DEVICE arrays that must hold
 *   their values when the call is made (synchronise the stream that wrote them);
 *   psi [n], acc [n][3] DEVICE outputs, written before fmm_poll reports completion
 *   and not to be touched until then.  G finite.  At most one request per system
 *   in flight (else FMM_E_BUSY); unknown sys_id: FMM_E_NOTFOUND.  *ticket > 0.
 * fmm_poll: wait up to timeout_ms (0: do not wait, < 0: no limit) for a ticket.
 *   Returns FMM_E_BUSY if it has not completed, else the request's result code
 *   (0 or an FMM_E_* of its evaluation); a completed ticket is retired, and
 *   *latency_s (may be NULL) is the time from fmm_submit to completion.
 * fmm_system_release: forget a system (FMM_E_BUSY while it has a request in flight).
 * fmm_workspace_bytes: device bytes currently held by the context and its slots.
 * fmm_destroy waits for the queued requests to finish before stopping the slots.
 * The serving calls are thread-safe among themselves. */
int fmm_serve_config(fmm_ctx* ctx, uint64_t budget_bytes, int slots);
int64_t fmm_footprint_bytes(const fmm_params* params, int64_t n);
int fmm_system_register(fmm_ctx* ctx, int64_t n, int* sys_id);
int fmm_submit(fmm_ctx* ctx, int sys_id, const double* x, const double* mu, double G, double* psi,
               double* acc, uint64_t* ticket);
int fmm_poll(fmm_ctx* ctx, uint64_t ticket, int timeout_ms, double* latency_s);
int fmm_system_release(fmm_ctx* ctx, int sys_id);
uint64_t fmm_workspace_bytes(fmm_ctx* ctx);

/* Copy the context's view of the last evaluation to HOST buffers, for tests:
 * cells (ncells x 5 int64: level, leaf, first, count, nchild; ncells x 6 double:
 * centre x,y,z, rho, mass, minscale), the M2L and P2P lists as (source cell,
 * sink cell) int64 pairs, and perm[n] (sorted position -> caller index).  Any
 * pointer may be NULL; counts are in the last stats. */
int fmm_debug_dump(fmm_ctx* ctx, int64_t* cells_int, double* cells_dbl, int64_t* m2l,
                   int64_t* p2p, int64_t* perm, double* scale_sorted);

/* The expansion order of every M2L interaction of the last evaluation, in the order of
 * fmm_debug_dump's m2l list (HOST out, n_m2l ints): the pair's q with adaptive_p, else p. */
int fmm_debug_m2l_orders(fmm_ctx* ctx, int32_t* q);

/* Counts and phase times of the last evaluation on ctx (HOST out).  Phase events
 * are recorded on every evaluation; this call waits for the last one to finish. */
int fmm_last_stats(fmm_ctx* ctx, fmm_stats* out);

/* The swap matrix B_n (App. A.5.1: Theta_n^m(z, y, x) = sum_l B_n^{ml} Theta_n^l(x, y, z))
 * that the rotation-accelerated M2L is built from, for 0 <= n <= 16: (2n+1)^2 doubles,
 * row m = -n..n, column l = -n..n, row-major, into the HOST array B.  No device work.
 * FMM_E_INVALID for n outside that range or B == NULL. */
int fmm_swap_matrix(int n, double* B);

/* Measure the device's FP64 (DFMA) and FP32 (FFMA) throughput in TFLOP/s with
 * two short register-only loops on the current device (HOST outs; about 50 ms).
 * These are the roofline denominators of the ALU-bound kernels. */
int fmm_alu_peaks(double* fp64_tflops, double* fp32_tflops);

/* The rate of the mixed P2P's pair arithmetic alone (eq. 1 in its far form: dx from FP32
 * offsets, packed FP32 operations, the hardware rsqrt approximation), sources from shared
 * memory, two sinks per lane, no staging, list walking or idle lanes, with warps_per_sm warps
 * per SM (4..32) on the current device: the ceiling the P2P kernel's arithmetic is measured
 * against.  *gpairs_s (HOST out): 10^9 particle pairs per second.  About 10 ms; allocates and
 * frees a small device buffer. */
int fmm_pair_peak(int warps_per_sm, double* gpairs_s);

/* Measurement behind a design choice of the rotation-accelerated M2L (App. A.5; no
 * counterpart in the paper's method): the swap stage (the matrices of App. A.5.1 applied to
 * one vector per interaction pair, orders 0..14) timed on the current device for npairs
 * random vectors, `reps` applications each (reps even, > 0), once as the FMA-immediate code
 * the M2L kernel uses and once on the tensor cores (TF32 mma.sync, three products per entry
 * for FP32 accuracy).  ms[0], ms[1] (HOST out): best kernel times of the two; *maxdiff
 * (HOST out): the largest difference of their results after one more application.  Allocates
 * and frees its own device buffers; FMM_E_INVALID for bad arguments. */
int fmm_swap_probe(int npairs, int reps, double* ms, double* maxdiff);

/* fmm_evaluate for small systems without allocating any device memory.
 * (The paper has no counterpart: this is a service of the library.)  Some callers
 * cannot allocate: simulation codes whose device memory belongs to their own pool
 * allocator (a cudaMalloc behind the pool's back breaks its accounting and can
 * fail once the pool holds the memory), and plugins that may not grow the host
 * process's device footprint.  They evaluate systems of up to 8192 particles
 * here.  All scratch memory comes from one fixed 32 MiB array in device global
 * memory that every GPU loading the library holds until the process exits;
 * nothing calls cudaMalloc, cudaFree or any other device allocator.  On its first
 * call on a device the entry point looks up that array's device address
 * (cudaGetSymbolAddress, with the device current); make that first call before
 * any stream capture.  All calls share the array and it keeps the last call's
 * contents (what must start at zero is cleared on every call); calls whose work
 * overlaps on the GPU race on it and give wrong results, so serialise them.  The
 * call waits for its stream several times (the tree's level sizes and the walk's
 * frontier lengths are read on the host).
 *   n       0 <= n <= 8192, else FMM_E_INVALID
 *   x, mu   device, [n][3] and [n] FP64 (as fmm_evaluate)
 *   params  host; p <= 10, 24 <= leaf_size <= 4096, scale_src = FMM_SCALE_ESTIMATE
 *   psi/acc device outputs (as fmm_evaluate)
 *   stream  cudaStream_t or NULL
 *   errbuf  host, may be NULL: receives a one-line description of a failure
 * The M2L and P2P lists hold at most 196,608 cell pairs each: parameters that need
 * longer lists (at n near 8192: eps below ~1e-8, or p2p_c below ~2 with eps near
 * 1e-7) return FMM_E_OVERFLOW.
 * Returns 0, FMM_E_INVALID, FMM_E_OVERFLOW (an interaction list or the tree does
 * not fit in the array) or FMM_E_CUDA. */
int fmm_evaluate_noalloc(int64_t n, const double* x, const double* mu, double G, const fmm_params* params,
                         double* psi, double* acc, void* stream, char* errbuf, int errlen);

/* Release the context and all of its device memory. */
int fmm_destroy(fmm_ctx* ctx);

/* Static description of an error code. */
const char* fmm_strerror(int code);

/* Description of the last failure on ctx (empty string if none). */
const char* fmm_last_error(fmm_ctx* ctx);

/* Version string of the library. */
const char* fmm_version(void);

#ifdef __cplusplus
}
#endif
#endif /* GB3FMM_H */
