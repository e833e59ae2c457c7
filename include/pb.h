/*
 * pb.h — C ABI of the GB300 electron-phonon collision-integral library (libpb.so).
 *
 * What it computes (arXiv:2511.03683, "Efficient GPU Parallelization of
 * Electronic Transport and Nonequilibrium Dynamics from Electron-Phonon
 * Interactions in the Perturbo Code"):
 *
 *   Eq. 2 (collision integral of state s = (n,k)):
 *     I_s = -(2 pi/hbar)(1/N_q) sum_{m q nu} |g_{mn nu}(k,q)|^2
 *           [ delta(eps_s - eps_p + hbar w) F_abs + delta(eps_s - eps_p - hbar w) F_em ]
 *   with p = (m, k+q), w = omega_{nu q}, delta a normalised Gaussian of width sigma and
 *     F_abs = f_s (1-f_p) N - (1-f_s) f_p (N+1),
 *     F_em  = f_s (1-f_p)(N+1) - (1-f_s) f_p N,       N = 1/(exp(hbar w / k_B T) - 1).
 *   (The paper names F_abs and F_em without writing them out; these are the Fermi
 *   golden-rule forms, under which each channel adds equal and opposite amounts to
 *   I(nk) and I(mk+q), as the paper states in Sec. "Optimized GPU algorithm", step 1.)
 *
 * A scattering channel is the tuple (k, q, n, m, nu) (Sec. "Collision integral, e-ph
 * coupling matrix, and scattering channels").  The library keeps every channel whose
 * two states lie inside the energy window and whose phonon energy is positive, in a
 * state-segmented CSR list that holds each channel under both of its states, so the
 * per-state sums need no atomic updates (the paper's aim in its "target layer",
 * Fig. 2) and no second "sc_col" pass (Fig. 2b-c): contribution and reduction are fused.
 *
 * Units: eV, fs, K; hbar = 0.6582119569 eV fs, k_B = 8.617333262e-5 eV/K.  Rates are 1/fs.
 *
 * Conventions shared by every call:
 *  - Full-grid state id: id = ik * nbands + n,  ik = (j1 * N2 + j2) * N3 + j3,
 *    k_i = 2 pi j_i / N_i.  The q grid equals the k grid (commensurate grids, N_q = N1 N2 N3).
 *  - Window states are numbered 0..nstate-1 in ascending full-grid id.  Every device
 *    vector (f, dfdt, inv_tau, F) is indexed by that number.
 *  - Status: every int-returning call returns PB_OK (0) or one of the PB_E* codes below;
 *    pb_last_error() then gives a message (thread-local; valid until the thread's next call).
 *    No C++ exception crosses the ABI.
 *  - Streams: `stream` is a cudaStream_t passed as void*; NULL is the legacy default stream.
 *    Device calls are asynchronous on that stream unless stated.
 *  - Concurrency: the device calls on one pb_dev (or pb_batch) share that handle's scratch
 *    regions, so they must not overlap on the GPU: issue them on one stream, or order the
 *    streams.  A handle also keeps host state (its call-graph cache and the launch settings
 *    a call records), so calls on one handle from several host threads must be serialised by
 *    the caller.  Separate handles are independent.
 *  - Ownership: the library owns only its opaque host handles (pb_channels, pb_dev).  All
 *    device memory is the caller's: pb_dev_create carves its arrays out of one caller-
 *    allocated device arena and never frees it; vectors passed to the compute calls are
 *    caller-owned device pointers.
 */
#ifndef PB_H
#define PB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  PB_OK = 0,
  PB_EINVAL = 1,      /* bad argument (null pointer, size, dimension, non-finite input) */
  PB_ENOMEM = 2,      /* host allocation failed, or the device arena is too small */
  PB_ECUDA = 3,       /* a CUDA runtime call failed; message holds cudaGetErrorString */
  PB_ENOTCLOSED = 4,  /* a channel's reverse channel is missing or has a different |g|^2 */
  PB_ENOCONV = 5,     /* pb_iter_transport reached maxit above tol */
  PB_ETIMEOUT = 6,    /* a bounded device-side wait gave up (reported by pb_dev_check) */
  PB_ECALLBACK = 7,   /* the |g|^2 callback returned non-zero or a negative/non-finite value */
  PB_EDEVICE = 8      /* no usable CUDA device, or it is not an sm_103 part */
};

/* ---------------------------------------------------------------- host model */

/* One e-ph system on commensurate k/q grids (Eq. 2; Sec. "Collision integral ...").
 * All pointers are HOST memory owned by the caller and only read during
 * pb_build_channels (the library copies what it keeps). */
typedef struct pb_model {
  int32_t nk[3];        /* grid N1, N2, N3 (>= 1 each); N_q = N1*N2*N3 */
  int32_t nbands;       /* bands per k point (1..255) */
  int32_t nmodes;       /* phonon branches (1..255) */
  const double *eps;    /* [N_q][nbands] band energies, eV */
  const double *vel;    /* [N_q][nbands][3] band velocities (any length unit per fs), or NULL */
  const double *omega;  /* [N_q][nmodes] phonon energies hbar*omega_{nu q}, eV; must be even in q */
  const double *win;    /* [nbands][2] per-band energy window [lo, hi] (inclusive), or NULL = all states */
  double T;             /* phonon temperature, K (> 0) */
  double sigma;         /* Gaussian width of the delta function, eV (> 0) */
} pb_model;

/* |g|^2 (eV^2) of n channels.  s[i], p[i] are FULL-GRID ids of the two states and
 * nu[i] the branch; write g2[i].  Must be symmetric: g2(s,p,nu) == g2(p,s,nu).
 * Return 0 on success.  Called from one thread unless pb_build_opts.callback_threadsafe. */
typedef int (*pb_g2_fn)(int64_t n, const int32_t *s, const int32_t *p, const int32_t *nu, double *g2,
                        void *user);

typedef struct pb_build_opts {
  int32_t nthreads;             /* host threads (0 = all available) */
  int32_t callback_threadsafe;  /* nonzero: g2 callback may run on several threads at once */
  int32_t check_closure;        /* nonzero: verify every channel's reverse exists with equal g2 */
  int32_t reserved;
  double g2_min;                /* drop channels with g2 < g2_min (the paper's |g| cutoff); 0 keeps all */
  double delta_nsigma;          /* drop channels with min(|x+w|, |x-w|) > delta_nsigma * sigma, x = eps_s -
                                   eps_p (the paper's approximate energy conservation); 0 keeps all */
} pb_build_opts;

typedef struct pb_channels pb_channels; /* opaque host CSR, library-owned */

typedef struct pb_channels_info {
  int64_t nstate;      /* window states (CSR rows) */
  int64_t nchannels;   /* stored channels (each physical channel appears under both its states) */
  int64_t nq;          /* N_q */
  int32_t nk[3];
  int32_t nbands;
  int32_t nmodes;
  int32_t reserved;
  double T, sigma;
  int64_t max_row;     /* longest row */
} pb_channels_info;

/* Step 1 of the paper's GPU scheme ("create the target layer", done once on the CPU):
 * select window states, enumerate every channel (s, p, nu) with s and p in the window,
 * q = k_p - k_s folded onto the grid and hbar*omega_{nu q} > 0, fetch |g|^2 through the
 * callback, and store the list in CSR order: rows = window states ascending, channels
 * within a row sorted by (partner, nu).  With check_closure, fails with PB_ENOTCLOSED
 * unless the list is closed under s <-> p with equal |g|^2 (which makes sum_s I_s = 0).
 * On success *out is a new handle (free with pb_channels_free). */
int pb_build_channels(const pb_model *model, pb_g2_fn g2, void *user, const pb_build_opts *opts,
                      pb_channels **out);

int pb_channels_get_info(const pb_channels *ch, pb_channels_info *info);

/* Copy the CSR to caller HOST arrays (any pointer may be NULL to skip it):
 * row_ptr[nstate+1], col[nchannels] (partner window index), nu[nchannels],
 * g2[nchannels], state_ids[nstate] (full-grid id of each window state). */
int pb_channels_export(const pb_channels *ch, int64_t *row_ptr, int32_t *col, int32_t *nu, double *g2,
                       int32_t *state_ids);

void pb_channels_free(pb_channels *ch);

/* ---------------------------------------------------------------- device */

/* Hot-path variants.  Each evaluates the same Eq. 2 and meets the same FP64 oracle.
 *  PB_VARIANT_FF      (default) per-channel rate coefficients, precomputed once in FP64
 *                     and streamed as float-float (hi,lo) pairs with float-float
 *                     accumulation: FP64-level accuracy at FP32 issue rate.
 *  PB_VARIANT_F64     the same coefficients as doubles with native FP64 FMAs.
 *  PB_VARIANT_LITERAL streams |g|^2 and the packed (partner, nu) index and evaluates the
 *                     Gaussians and Bose factors per channel in FP64 registers.
 *  PB_VARIANT_G32     |g|^2 stored FP32, per-channel arithmetic in FP32, compensated
 *                     (Kahan) accumulation, FP64 state.
 *  PB_VARIANT_G16     as G32 with |g|^2 stored BF16.
 *  PB_VARIANT_H16     as G32 with |g|^2 stored FP16 times a power of two chosen at creation (the
 *                     largest value maps into [2^9, 2^10)): the same 2 bytes as BF16 with 11
 *                     significand bits instead of 8.  Values from 2^-23 of the largest value at
 *                     creation up to 63 times it are normal FP16 numbers; a value above that range
 *                     (overflow) or a nonzero value below it (fewer significand bits) makes
 *                     pb_dev_check return PB_EINVAL.
 *  PB_VARIANT_PAPER   the paper's own layout (Sec. "Optimized GPU algorithm", Fig. 2), for
 *                     comparison: every channel stored once, per-channel contributions written
 *                     to sc_col (step 2), then gathered with signs by each state's target list
 *                     (step 3).  Collision integral and RK4 only (no scattering rates).
 *  PB_VARIANT_C32     the FF device whose collision, rate and RK4 sweeps stream the symmetric
 *                     tiles (dense_rows 3) of the branch-merged coefficients in FP32: 8 bytes per
 *                     state pair, half the float-float tiles.  Each (P_in, P_out) pair is rounded
 *                     with its ratio kept; every tile entry forms its net term
 *                     P_in f_p (1-f_s) - P_out f_s (1-f_p) in FP32 with the larger product made
 *                     exact by an FMA, plus first-order terms in the low part of the float-float
 *                     f; FP64 for the per-state combination and the RK4 update.  df/dt within
 *                     about 1e-6 of Eq. 2 (normwise).  Needs the symmetric tiles (a list built with
 *                     check_closure whose rows are complete, or miss few partners, or dense_rows
 *                     3), branch merging and tile_sweep 0 or 2..8 (PB_EINVAL otherwise).  Transport, the
 *                     no-allocation call and, after pb_dev_set_g2, every sweep run the FF rows;
 *                     the adjoint calls return PB_EINVAL. */
enum { PB_VARIANT_FF = 0, PB_VARIANT_F64 = 1, PB_VARIANT_LITERAL = 2, PB_VARIANT_G32 = 3, PB_VARIANT_G16 = 4,
       PB_VARIANT_PAPER = 5, PB_VARIANT_H16 = 6, PB_VARIANT_C32 = 7 };

typedef struct pb_dev_opts {
  int32_t variant;           /* PB_VARIANT_* */
  int32_t item_channels;     /* channels per work item (multiple of 64; 0 = automatic, 256..4096) */
  int32_t ctas_per_sm;       /* resident CTAs per SM for the coefficient sweeps (0 = 3) */
  int32_t transport;         /* nonzero: reserve transport buffers (weights and F) */
  int32_t transport_gather;  /* transport F gather: 0 automatic (= 4), 1 shared memory, 2 through L1 with
                                4-channel groups per lane, 3 through L1 with one channel per lane;
                                one channel per lane with lazily renormalised float-float sums: 4 one
                                1024-thread CTA per SM with F in shared memory (5 if F does not fit) and
                                the next trip in registers, 5 the same through L1, 6 = 3 with lazy sums;
                                7 row blocks on complete branch-merged float-float rows: a warp takes
                                four rows and one segment of their partners, each partner's F (shared
                                memory) read once for the four rows, the weights through a per-warp
                                ring of asynchronous copies, one 768-thread CTA per SM (PB_EINVAL where
                                the rows do not qualify or F and the rings exceed shared memory) */
  int32_t transport_ctas;    /* resident 256-thread transport CTAs per SM, 1..8 (0 = 8 with L1 gathers) */
  int32_t channel_per_lane;  /* FP32/BF16/FP16 sweep shape: 0 automatic (= 5 when the channel list fills at
                                least 85% of the (state, branch, partner) slots, else 4); one channel per
                                lane in 512-thread CTAs, three per SM: 1 plain, 3 with an L2 prefetch of the
                                stream two 128-channel trips ahead; 2 four-channel groups per lane; 4 one
                                channel per lane in one 1024-thread CTA per SM, next trip's stream in
                                registers; 5 dense pair-major: |g|^2 in one slot per (state, branch,
                                partner), zero where no channel exists, no index streamed, one partner per
                                lane with its branches in turn (the forward sweeps; the adjoint keeps the
                                channel list) */
  int32_t stream_mode;       /* FF collision sweep: 0 automatic (= 1), 1 vector loads from global memory,
                                2 TMA bulk copies (cp.async.bulk) into a shared-memory ring (FF variant,
                                nstate <= 65536); its bounded waits report through pb_dev_check */
  int32_t merge_branches;    /* FF and F64: 0 automatic (= 1); 1 sum the coefficients of the branches nu of
                                every state pair (s, p) once at setup and stream one entry per pair (Eq. 2
                                depends on nu only through |g|^2, N and the deltas, all fixed with eps,
                                omega, sigma and T); 2 stream one entry per channel */
  int32_t dense_rows;        /* FF, branch-merged: 0 automatic (= 3 when every row holds every window state
                                in order, i.e. no cutoffs, or when the tiles below stream at most 0.7 of the
                                rows' bytes; else 2); 1 (complete rows only) the collision, rate and
                                transport sweeps take each entry's partner from its position and stream no
                                index (16 instead of 18 bytes per entry); 3 as 1 where the rows are complete,
                                and the collision and rate sweeps stream the upper block triangle of the pair
                                matrix as 64 x 64 tiles of (P_in, P_out), zero where a pair has no channel,
                                adding each tile to its rows and, through the reverse channels (P_in(p,s) =
                                P_out(s,p)), to its columns: about 8 bytes per state pair (only for a list
                                built with check_closure, which guarantees those reverse channels; 1 or 2
                                otherwise); 2 always stream the index */
  int32_t tile_sweep;        /* the symmetric tile sweep (dense_rows 3): 0 automatic (= 3); 1 each thread
                                loads its 4 x 4 entries of a tile from global memory (3 CTAs per SM);
                                2 one persistent CTA per SM with 256 threads keeps three tiles in flight in
                                shared memory through TMA bulk copies (cp.async.bulk, mbarrier-counted),
                                its bounded waits reporting through pb_dev_check; 3 the same ring in
                                half-tiles (32 x 64 entries, 32 KB), the column sums of a tile carried in
                                registers across its two halves: two stages per CTA and three CTAs per SM
                                (ctas_per_sm 2: three stages, two CTAs).  PB_VARIANT_C32: 0 or 2 its
                                default launch shape (two stages, three CTAs per SM), 3..6 other shapes
                                (3 x 2, 2 x 2, 4 x 1, 6 x 1 stages x CTAs), 7 and 8 half-tiles
                                (3 x 4, 4 x 3) */
  int32_t adjoint;           /* 1: reserve the accumulators of the deferred |g|^2 gradient
                                (pb_rtbte_rk4_vjp_defer): FF with branch merging, one float-float
                                (u, v) per stored state pair (16 bytes); G32/G16/H16, three doubles per
                                (state, partner) pair (24 nstate^2 bytes); ignored otherwise */
} pb_dev_opts;

typedef struct pb_dev pb_dev; /* opaque host handle describing device-resident data */

/* Bytes of device arena pb_dev_create needs for this channel list and options. */
int pb_dev_arena_bytes(const pb_channels *ch, const pb_dev_opts *opts, size_t *bytes);

/* Upload the CSR and tables into `arena` (caller-owned device memory of at least
 * pb_dev_arena_bytes, 256-byte aligned) and precompute per-channel coefficients on the
 * GPU.  Synchronises `stream` before returning.  The arena must outlive the handle. */
int pb_dev_create(const pb_channels *ch, const pb_dev_opts *opts, void *arena, size_t arena_bytes, void *stream,
                  pb_dev **out);

void pb_dev_destroy(pb_dev *dev);

/* Synchronise `stream` and report PB_ETIMEOUT if a bounded device-side wait of an earlier
 * launch gave up (the TMA bulk-copy sweeps), or PB_EINVAL if a |g|^2 value fell outside the
 * normal range of the scaled FP16 storage of a PB_VARIANT_H16 device; PB_OK otherwise.  The report clears the
 * handle's error word, so the next check sees only later launches. */
int pb_dev_check(pb_dev *dev, void *stream);

/* Test of the bounded-wait machinery itself (the paper has no counterpart): one CTA issues a
 * 1 KB bulk copy from the handle's arena into shared memory, then waits on an mbarrier that
 * nothing ever completes, giving up after wait_us microseconds (1..2000000; the sweeps' own
 * waits give up after 2 s); on the give-up it records the failure in the error word and waits
 * (bounded) for its own copy before returning, as the sweeps do.  No fault and no hang: the
 * next pb_dev_check reports PB_ETIMEOUT and the handle stays usable. */
int pb_dev_selftest_wait(pb_dev *dev, int32_t wait_us, void *stream);

typedef struct pb_dev_info {
  int64_t nstate, nchannels, nchannels_padded, nitems;
  int32_t variant, sm_count;
  double bytes_per_channel;  /* algorithmic bytes streamed per channel by pb_collision */
  double c;                  /* (2 pi / hbar) / N_q, 1/(eV fs) */
} pb_dev_info;

int pb_dev_get_info(const pb_dev *dev, pb_dev_info *info);

/* Eq. 2: dfdt[s] = I_s[f] for every window state.  f, dfdt: device double[nstate].
 * The call's launches are replayed from a CUDA graph kept per argument set (captured on first
 * use; the handle keeps its twelve most recent call graphs, shared with pb_scatter_rates,
 * pb_transport_iterate, the host-buffer calls, the RK4 adjoint steps and the transport solver's
 * passes); when `stream` is itself being captured, the launches are recorded into the caller's
 * capture. */
int pb_collision(pb_dev *dev, const double *f, double *dfdt, void *stream);

/* Measurement aid (the paper has no counterpart): the average device duration of the
 * collision sweep kernel alone, from CUDA events recorded on `stream` around `nlaunch`
 * back-to-back launches of it on f (device double[nstate]); the stage-input conversion runs
 * once before the first event and no finaliser runs.  order 0: every launch takes the tile
 * list in its stored order; 1: the launches alternate between that order and the reverse, as
 * the RK4 stages of the symmetric-tile sweeps do (each then starts on the tiles the launch before
 * it left in L2).  Leaves the partial sums of the last launch in the handle's scratch;
 * synchronises `stream`.  nlaunch in 1..10000. */
int pb_dev_time_sweep(pb_dev *dev, const double *f, int32_t nlaunch, int32_t order, float *avg_ms,
                      void *stream);

/* Scattering rates 1/tau_s = -dI_s/df_s
 *   = (2pi/hbar)(1/N_q) sum |g|^2 [G(x+w)(N+f_p) + G(x-w)(N+1-f_p)],  x = eps_s - eps_p.
 * f, inv_tau: device double[nstate]. */
int pb_scatter_rates(pb_dev *dev, const double *f, double *inv_tau, void *stream);

/* nsteps classic RK4 steps of the field-free rt-BTE df/dt = I[f] (Eq. 1 with F = 0),
 * step dt (fs), in place on the device vector f.  Steps are replayed from CUDA graphs captured
 * on first use per (f, dt) (the capture uses an internal stream): the call's first step from a
 * graph that also converts f into the sweeps' stage input, the others from one that takes it
 * from the step before. */
int pb_rtbte_rk4_step(pb_dev *dev, double *f, double dt, int32_t nsteps, void *stream);

/* Same as pb_rtbte_rk4_step with HOST buffers: copies f_host_in (double[nstate]) to the
 * device, runs nsteps steps, copies the result to f_host_out, and synchronises `stream`.
 * The host buffers should be pinned for asynchronous copies; pageable memory works.  With
 * nsteps = 1 and page-locked buffers, both copies and the step's launches are one CUDA graph,
 * replayed per (f_host_in, f_host_out, dt) from the handle's call-graph cache. */
int pb_rtbte_rk4_host(pb_dev *dev, const double *f_host_in, double *f_host_out, double dt, int32_t nsteps,
                      void *stream);

/* Iterative linearised transport for the three field directions at once
 * (Sec. "Optimized GPU algorithm": sc_col gains a field-direction dimension):
 *   F^{i+1}_{s a} = tau_s ( v_{s a} + sum_c W_c F^i_{p a} ),  a = x, y, z,
 *   W_c = (2pi/hbar)(1/N_q)|g|^2 [G(x+w)(N+f0_p) + G(x-w)(N+1-f0_p)],  1/tau_s = sum_c W_c,
 * from F^0 = tau v until max|F^{i+1}-F^i| <= tol * max|F^{i+1}|.
 * f0: device double[nstate]; vel3, F3: device double[nstate][3].  On return (stream
 * synchronised) *iters holds the iterations done and *resid the last relative change;
 * PB_ENOCONV if maxit was reached first (F3 then holds the last iterate).  Each pass is
 * replayed from a CUDA graph, and the next pass is queued before the host reads the previous
 * pass's residual (one extra pass runs after the converged one; it changes neither F3 nor the
 * result); the residual numbers go through 48 bytes of page-locked host memory that the
 * handle allocates on its first solve and frees in pb_dev_destroy.
 * Needs a pb_dev created with opts.transport != 0. */
int pb_iter_transport(pb_dev *dev, const double *f0, const double *vel3, double tol, int32_t maxit, double *F3,
                      int32_t *iters, double *resid, void *stream);

/* Compute and keep the transport weights W_c and tau_s at f0 (device double[nstate])
 * for later pb_transport_iterate calls.  pb_iter_transport and pb_transport_map call
 * it themselves. */
int pb_transport_setup(pb_dev *dev, const double *f0, void *stream);

/* One pass of the transport map with the weights of the last pb_transport_setup:
 * F3out = tau (v + W F3in), all device double[nstate][3], without any host
 * synchronisation.  If resid3 (device double[3]) is not NULL it receives
 * (max|F3out-F3in| / max|F3out|, max|F3out-F3in|, max|F3out|).  The pass's four launches are
 * replayed from a CUDA graph kept per set of pointers, as for pb_collision (an iteration that
 * alternates between two buffers replays two graphs). */
int pb_transport_iterate(pb_dev *dev, const double *vel3, const double *F3in, double *F3out, double *resid3,
                         void *stream);

/* Same as pb_transport_iterate with the iterates in HOST buffers: copies F3in_host
 * (double[nstate][3]) to the device, runs one pass with the weights of the last
 * pb_transport_setup, copies the new iterate to F3out_host (which may equal F3in_host) and, if
 * resid3_host is not NULL, the three residual numbers of pb_transport_iterate to it, then
 * synchronises `stream`.  vel3 is a device vector as there.  The host buffers should be pinned
 * for asynchronous copies; pageable memory works (page-locked buffers: the copies and the pass
 * are one CUDA graph, replayed per buffer set from the handle's call-graph cache).  Needs
 * opts.transport != 0 (the copies use the handle's own iterate buffers). */
int pb_transport_iterate_host(pb_dev *dev, const double *vel3, const double *F3in_host, double *F3out_host,
                              double *resid3_host, void *stream);

/* One transport map application without the convergence loop: F3out = tau (v + W F3in)
 * with W, tau at f0 (pb_transport_setup followed by pb_transport_iterate). */
int pb_transport_map(pb_dev *dev, const double *f0, const double *vel3, const double *F3in, double *F3out,
                     void *stream);

/* ---------------------------------------------------------------- adjoint (reverse mode) */

/* Vector-Jacobian product of the collision integral (Eq. 2) at f:
 *   grad_f[x] = sum_s lam[s] dI_s/df_x                       (device double[nstate], overwritten)
 *   grad_g2[c] += lam[s_c] dI_{s_c}/dg2_c for every stored channel c in the CSR order of
 *                 pb_channels_export (device double[nchannels], accumulated; may be NULL).
 * Each stored channel's |g|^2 is its own variable here; the derivative with respect to the
 * shared |g|^2 of a channel and its reverse is the sum of the two entries.  The transposed
 * sum is evaluated as a gather over each state's own row (the list is closed under
 * s <-> p), so no atomic updates are needed.  Needs a PB_VARIANT_FF device (FP64-accurate) or a
 * PB_VARIANT_G32 / G16 / H16 device (FP32 per-channel terms, FP64 accumulation). */
int pb_collision_vjp(pb_dev *dev, const double *f, const double *lam, double *grad_f, double *grad_g2,
                     void *stream);

/* Discrete adjoint of one classic RK4 step from f (device double[nstate]): on entry lam holds
 * dL/df_{n+1}, on return dL/df_n; grad_g2 (or NULL) accumulates dL/dg2 as above.  The four
 * stage inputs are recomputed from f.  f is first copied into the handle; the step's launches
 * are then replayed from a CUDA graph kept per (lam, dt, grad_g2) in the handle's call-graph
 * cache (as is pb_rtbte_rk4_vjp_defer's, per (lam, dt)), so a backward pass that keeps one lam
 * vector replays one graph whatever its f. */
int pb_rtbte_rk4_vjp(pb_dev *dev, const double *f, double *lam, double dt, double *grad_g2, void *stream);

/* The same RK4 adjoint step with the |g|^2 gradient deferred.  Eq. 2 is linear in each
 * |g|^2, and the derivative of a channel's term depends on f only through two sums per state
 * pair (shared by the pair's branches and modes) and on the channel only through fixed
 * coefficients; so instead of updating every stored channel, the step adds its stage sums into
 * the handle's per-pair accumulators and pb_dev_g2grad_flush applies them later, once.  f, lam:
 * device double[nstate] as in pb_rtbte_rk4_vjp (lam in/out; dL/df_n on return).  Needs a device
 * created with pb_dev_opts.adjoint = 1 on the FF variant with branch merging or on G32/G16/H16:
 * PB_EINVAL otherwise, and for a null pointer or a non-finite dt.  Asynchronous on `stream`;
 * the accumulators belong to the handle (in its arena). */
int pb_rtbte_rk4_vjp_defer(pb_dev *dev, const double *f, double *lam, double dt, void *stream);

/* grad_g2 (caller's device double[nchannels], CSR order of pb_channels_export) += the |g|^2
 * gradient accumulated by pb_rtbte_rk4_vjp_defer since the last flush; the accumulators are
 * cleared.  PB_EINVAL for a null pointer or a device without accumulators.  Asynchronous on
 * `stream`. */
int pb_dev_g2grad_flush(pb_dev *dev, double *grad_g2, void *stream);

/* Replace the device |g|^2 (device double[nchannels], CSR order of pb_channels_export) and
 * recompute the per-channel coefficients.  The two stored copies of a channel (under each of
 * its states) may be given different values, so the device stops using the symmetric tiles
 * (dense_rows 3) and streams rows from then on.  Transport weights are not refreshed: call
 * pb_transport_setup again before iterating. */
int pb_dev_set_g2(pb_dev *dev, const double *g2, void *stream);

/* ---------------------------------------------------------------- batched rt-BTE */

/* Many independent systems (different grids, bands, modes, temperatures) advanced together:
 * one persistent launch per RK4 stage sweeps every instance, followed by one epilogue
 * launch; a CUDA graph replays the eight launches of a step.  Precision 0 (default): the
 * literal per-channel form of Eq. 2 with |g|^2 stored in FP32 (rounded on the host), FP32
 * per-channel arithmetic with Kahan lane sums and FP64 states.  Precision 1: the
 * FP64-accurate branch-merged coefficient stream of the FF variant, each instance's
 * prefactor folded into its coefficients.  Precision 2: those coefficients as FP32 pairs
 * (the PB_VARIANT_C32 arithmetic on rows).  Device vectors are the instances' state vectors
 * concatenated in instance order (offsets from pb_batch_get_info). */
typedef struct pb_batch pb_batch;

typedef struct pb_batch_opts {
  int32_t item_channels;  /* sweep entries per work item (0 = 2048; else a multiple of 64, >= 1024) */
  int32_t ctas_per_sm;    /* resident CTAs per SM: 512-thread (precision 0, default 2) or 256-thread
                             (precision 1, default 4); 0..4 */
  int32_t precision;      /* 0: |g|^2 in FP32, the literal per-channel form of Eq. 2 in FP32 (one entry per
                             channel); 1: FP64-accurate: each instance's coefficients computed in FP64,
                             summed over the branches of every state pair, stored float-float (one entry
                             per state pair); 2: the coefficients of 1 rounded once to FP32 pairs
                             (P_in, P_out) with their ratio kept (8 bytes per state pair), each entry's
                             net term in FP32 with an exact leading product and first-order terms in the
                             low part of f, as PB_VARIANT_C32 (df/dt within about 1e-6) */
  int32_t layout;         /* precision 0: 0 automatic (the dense pair-major form when the stored channels
                             fill at least 85% of the instances' (state, partner, branch) slots: |g|^2 in
                             one FP32 slot each, zero where no channel exists, no index streamed; work
                             items of item_channels / 4 partners); 1 one entry per channel.
                             precision 1 and 2: 0 automatic (symmetric tiles when every instance's list
                             was built with check_closure and the tiles stream at most 0.7 of the rows'
                             bytes: each instance's states in 64-state blocks of one padded state space,
                             the upper block triangle of each instance stored as 64 x 64 tiles, one
                             unordered state pair per entry for both directions, zero where a pair has
                             no channel); 1 rows (one entry per directed state pair); 2 symmetric tiles
                             whatever their bytes (PB_EINVAL for a list built without check_closure) */
} pb_batch_opts;

int pb_batch_arena_bytes(const pb_channels *const *chs, int32_t n, const pb_batch_opts *opts, size_t *bytes);

/* Upload n channel lists into `arena` (caller-owned device memory, 256-byte aligned, of at
 * least pb_batch_arena_bytes).  Synchronises `stream`.  The channel lists may be freed after. */
int pb_batch_create(const pb_channels *const *chs, int32_t n, const pb_batch_opts *opts, void *arena,
                    size_t arena_bytes, void *stream, pb_batch **out);

void pb_batch_destroy(pb_batch *batch);

/* Total states and channels, state_offsets[n+1] (may be NULL), current launch shape:
 * item_channels is 0 when the batch streams symmetric tiles (ctas_per_sm then gives the tile
 * ring's resident CTAs per SM). */
int pb_batch_get_info(const pb_batch *batch, int64_t *nstate, int64_t *nchannels, int64_t *state_offsets,
                      int32_t *item_channels, int32_t *ctas_per_sm);

/* Reads (and clears) the batch's device error word: PB_ETIMEOUT when a bounded wait of the
 * tile sweep gave up since the last check (its results are then invalid).  Synchronises
 * `stream`. */
int pb_batch_check(pb_batch *batch, void *stream);

/* dfdt = I[f] for every state of every instance (device double[nstate total]). */
int pb_batch_collision(pb_batch *batch, const double *f, double *dfdt, void *stream);

/* nsteps classic RK4 steps of every instance, in place on f (device double[nstate total]). */
int pb_batch_rk4_step(pb_batch *batch, double *f, double dt, int32_t nsteps, void *stream);

/* Time candidate launch shapes (rows: work-item sizes 1024/2048/4096 entries x 2/3/4 CTAs
 * per SM; symmetric tiles: the tile ring's stages x CTAs per SM, item size reported as 0) on
 * collision sweeps at f and keep the fastest; reports it (any pointer may be NULL).
 * Synchronises `stream`. */
int pb_batch_autotune(pb_batch *batch, const double *f, void *stream, int32_t *best_item_channels,
                      int32_t *best_ctas_per_sm, double *best_ms);

/* Observables of a distribution: out[0] = sum_s f_s (carriers), out[1] = sum_s eps_s f_s (eV),
 * out[2] = sum_s I_s[f] (conservation check, 1/fs).  out: device double[3]. */
int pb_observables(pb_dev *dev, const double *f, double *out3, void *stream);

/* No-allocation form of pb_collision.  It is for callers that cannot allocate device
 * memory at all: code embedded in a host application whose device memory belongs to
 * another allocator (a framework's caching pool, or a fixed budget carved out at
 * start-up), so that neither the caller nor a library it calls may use cudaMalloc.
 * The caller passes the same inputs and outputs as to pb_collision (a pb_dev, f and
 * dfdt, device double[nstate]).  The per-call scratch (the float-float copy of f and
 * one partial sum per work item) lives in a file-scope device array of
 * PB_STATIC_SCRATCH_BYTES inside libpb.so, which every GPU that loads the library
 * keeps until the process exits.  A problem needs 8*nstate (rounded up to 256) +
 * 32*nitems bytes of it; larger ones fail with PB_EINVAL and say so (pb_collision
 * has no such limit).  The call itself allocates nothing.
 * The first call on each device looks up the array's device address with that
 * device current (cudaGetSymbolAddress); make that first call before any stream
 * capture.  All calls share the one array and it keeps the last call's contents:
 * calls that overlap on the GPU (other streams or threads) race, so the caller must
 * serialise them.  Each call writes every scratch byte it reads before reading it,
 * so nothing needs clearing.  The paper has no counterpart of this entry point. */
#define PB_STATIC_SCRATCH_BYTES (4u << 20)
int pb_collision_static(pb_dev *dev, const double *f, double *dfdt, void *stream);

const char *pb_last_error(void);

/* Library version string, e.g. "pb 0.1 sm_103a". */
const char *pb_version(void);

#ifdef __cplusplus
}
#endif

#endif /* PB_H */
