/*
 * mlb.h -- C ABI of the GB300 (sm_103a) multispecies Enskog/RPA lattice
 * Boltzmann step of Marini Bettolo Marconi & Melchionna, "Multicomponent
 * Diffusion in Nanosystems" (arXiv:1105.3634).
 *
 * One time step advances the D3Q19 populations f^a_i of every species a by
 *   moments      n^a = sum_i f^a_i, n^a u^a = sum_i c_i f^a_i        (Sec. II, Eq. colonna)
 *   contact g    g_ab = BMCSL contact value of the densities smoothed over
 *                a ball of radius kappa sigma_c                    (Sec. II, "smoothing procedure")
 *   field        Phi^a = F^hc + G + F^drag + F^visc                (Sec. III, Eqs. splitforce,
 *                                                                   potmeanforce, gammaab, viscousforce)
 *   collide      f - omega (f - psi_perp) + forcing                (Sec. II, Eqs. evolution, prefactor)
 *   stream       f_i(r + c_i, t + 1), periodic or halfway bounce-back walls
 * in FP32 on the GPU.  The contact-sphere integrals are sums over the lattice
 * shell sigma_ab - 1/2 <= |d| < sigma_ab + 1/2 with weight 4 pi/|shell|; the
 * attraction is U_ab = -eps_ab (sigma_ab/r)^6 on sigma_ab <= r <= lambda_c sigma_ab.
 * The force enters with a semi-implicit half-force shift (psi_perp and the
 * forcing evaluated at u + a/2, forcing scaled by 1 - omega/2) unless
 * MLB_FORCE_EXPLICIT is set.
 *
 * Conventions
 *   - Units: lattice spacing = time step = 1; every mass must be 1 and kT = 1/3
 *     (the D3Q19 sound speed squared).
 *   - Site index: x + nx * (y + ny * z)  (x fastest).
 *   - Host arrays are owned by the caller and only read or written during the
 *     call.  All device memory is owned by the context; it is obtained once in
 *     mlb_create from desc->dev_alloc (or cudaMalloc when NULL) and released by
 *     mlb_destroy.
 *   - Every function returns an mlb_status and never aborts.  After
 *     MLB_ECUDA, MLB_ENUMERIC or MLB_ETIMEOUT the context is failed: later
 *     calls return MLB_ESTATE until mlb_destroy.  mlb_last_error() gives a
 *     one-line reason.
 *   - mlb_step is asynchronous on the context's stream; the mlb_get_* and
 *     mlb_conservation calls synchronise that stream.
 *   - One context per host thread at a time.
 */
#ifndef MLB_H
#define MLB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MLB_Q 19                 /* D3Q19 velocities */
#define MLB_MAX_SPECIES 4

typedef struct mlb_ctx mlb_ctx;

typedef enum {
    MLB_OK = 0,
    MLB_EINVAL = 1,    /* invalid argument or state (message says which) */
    MLB_ENOMEM = 2,    /* device allocation failed */
    MLB_ECUDA = 3,     /* a CUDA call failed */
    MLB_ENUMERIC = 4,  /* NaN/Inf met, or packing xi3 >= 1 somewhere */
    MLB_ETIMEOUT = 5,  /* a bounded device wait gave up */
    MLB_ESTATE = 6     /* context failed earlier, or call made out of order */
} mlb_status;

/* flags */
#define MLB_DRAG_ONLY       1u   /* partner velocity at r: Eq. gammaab alone, no viscous part */
#define MLB_FORCE_EXPLICIT  2u   /* forward-Euler forcing at u (no half-force shift) */
#define MLB_SPLIT_COLLIDE   4u   /* launch pass 2 and the collision separately (the acceleration
                                    field is stored every step); default: one fused launch.
                                    Both give bitwise-identical populations. */
#define MLB_MEANFIELD_BF16  8u   /* the attractive mean field G (Sec. III, Eq. potmeanforce) as a
                                    band-matrix product along z on the tensor cores: BF16 operands
                                    split hi + lo (densities and kernel), FP32 accumulation, the
                                    compensated product hi*hi + hi*lo + lo*hi (relative error of G
                                    about 1e-5).  Needs 1 or 2 species, an attraction reach of 1..8,
                                    nz % 8 == 0 and no walls normal to z (mlb_set_interactions
                                    returns MLB_EINVAL otherwise).  Default: FP32 column sums. */
#define MLB_MEANFIELD_BF16_1PASS 16u  /* with MLB_MEANFIELD_BF16: the single product hi*hi only
                                    (about a third of the tensor work; relative error of G of
                                    order 1e-3) */

typedef struct {
    int32_t nx, ny, nz;          /* lattice extents, each >= 1 */
    int32_t nspecies;            /* 1 .. MLB_MAX_SPECIES */
    int32_t wall_axis;           /* -1: periodic; 0/1/2: halfway bounce-back walls normal to that
                                    axis at coordinates -1/2 and n-1/2 */
    uint32_t flags;              /* MLB_* flags */
    double wall_u_lo[3];         /* velocity of the wall at coordinate -1/2 (tangential) */
    double wall_u_hi[3];         /* velocity of the wall at coordinate n-1/2 (tangential) */
    double tau;                  /* BGK relaxation time (omega = 1/tau), > 1/2 */
    double kT;                   /* must be 1/3 */
    double kappa;                /* smoothing-ball radius / sigma_cc (0.5 by default if 0) */
    /* device allocator: returns a device pointer aligned to 256 bytes, or NULL.
       NULL function pointers select cudaMalloc/cudaFree. */
    void *(*dev_alloc)(size_t bytes, void *user);
    void (*dev_free)(void *ptr, void *user);
    void *alloc_user;
    void *stream;                /* cudaStream_t the context launches on; NULL = a stream the
                                    context creates and owns */
} mlb_lattice_desc;

/* Create a context for one lattice of the method of Sec. II: the D3Q19
 * populations f^a_i of Eq. (evolution) for nspecies species on an
 * nx x ny x nz lattice, with relaxation time tau (omega = 1/tau of
 * Eq. evolution) and k_B T of Eq. (prefactor).  Validates desc, allocates
 * every device buffer (ownership: the context, through desc->dev_alloc).
 * The context then needs mlb_set_species, optionally mlb_set_interactions,
 * and mlb_set_fields (or mlb_set_populations) before mlb_step.
 * Errors: MLB_EINVAL (bad extents, tau <= 1/2, kT != 1/3, wall velocity with a
 * normal component), MLB_ENOMEM, MLB_ECUDA. */
mlb_status mlb_create(const mlb_lattice_desc *desc, mlb_ctx **out);

/* Hard-sphere diameters sigma_aa (Sec. III: sigma_ab = (sigma_aa + sigma_bb)/2)
 * and masses, each array of nspecies doubles.  Requires sigma >= 1 and every
 * mass == 1.  Builds the contact shells and smoothing balls.
 * Errors: MLB_EINVAL, also when a stencil offset reaches a full periodic
 * extent (every periodic extent must exceed the largest offset component). */
mlb_status mlb_set_species(mlb_ctx *ctx, const double *sigma, const double *mass);

/* Attractive tails (Sec. III, G term of Eq. potmeanforce; RPA, g = 1 inside):
 * eps[a*S+b] = eps_ab >= 0 (symmetric), lambda_c[a*S+b] = cutoff / sigma_ab
 * (symmetric, >= 1).  eps = NULL switches the attraction off.
 * Errors: MLB_EINVAL (asymmetric, negative, non-finite, table too large). */
mlb_status mlb_set_interactions(mlb_ctx *ctx, const double *eps, const double *lambda_c);

/* Initial state f := psi_perp(n, u) (Eq. prefactor at the given fields).
 * n: [S][N] number densities (>= 0, finite);  u: [S][3][N] species velocities
 * or NULL for rest.  Also fixes the per-species reference density n_ref^a
 * (the mean of n^a) that the FP32 populations are stored relative to.  The
 * fields are copied to the device first and checked and summed there (FP64);
 * a rejected field leaves the state unchanged.  Synchronises the stream.
 * Errors: MLB_EINVAL (negative or non-finite n, |u| >= 1, packing xi3 >= 1;
 * the message names the first offending entry). */
mlb_status mlb_set_fields(mlb_ctx *ctx, const double *n, const double *u);

/* Per-site external body force F^a (Eq. evolution) in lattice units:
 * fext: [S][3][N], or NULL to remove it. */
mlb_status mlb_set_external_force(mlb_ctx *ctx, const double *fext);

/* Number of Jacobi sweeps of the half step of the semi-implicit forcing (the
 * force term of Eq. (evolution) entering at u + a/2): u* = u + a(u*)/2 is
 * solved at every site by (I + Gamma/2) du = (F^hc + G + F^a + F^v)/2, with
 * Gamma the local friction matrix and F^v the velocity exchange of
 * Eqs. (gammaab), (viscousforce).  The first sweep takes the partners'
 * velocities at u (the default, one sweep); each further sweep repeats the
 * exchange and friction sums with the partners at the previous sweep's u*
 * (one more pass over the contact shells, one more launch per step).  More
 * sweeps approach the exactly solved half step: for unequal diameters the
 * lattice mutual diffusion coefficient with one sweep lies about 0.6 %
 * (sigma 1/1.5) above that of the exactly solved half step, with two about
 * 0.02 %; the uniform sigma 1/1.5 mixture stays linearly stable to packing
 * 0.3 with three sweeps (one sweep: about 0.2).  sweeps: 1..8.  The first
 * request of more than one sweep allocates S x N float4 on the device
 * (desc->dev_alloc), released by mlb_destroy.
 * Errors: MLB_EINVAL (out of range, or MLB_FORCE_EXPLICIT set), MLB_ENOMEM. */
mlb_status mlb_set_predictor_sweeps(mlb_ctx *ctx, int32_t sweeps);

/* Advance nsteps >= 0 time steps of Eq. (evolution), Sec. II: per step the
 * moments (Eq. colonna), the contact values, the effective field
 * Phi = F^hc + G + F^v of Eqs. (splitforce), (potmeanforce), (gammaab) and
 * (viscousforce), the collision toward psi_perp of Eq. (prefactor) with the
 * forcing term, and streaming.  Asynchronous on the context's stream; numeric
 * faults found on the way are reported by the next synchronising call.
 * Errors: MLB_EINVAL (nsteps < 0), MLB_ESTATE (no species or state yet, or a
 * failed context), MLB_ECUDA (a launch failed). */
mlb_status mlb_step(mlb_ctx *ctx, int64_t nsteps);

/* One step that also reports the FP64 conservation sums of the state it
 * starts from (Eqs. continuity, momentcomponent), without stalling: the sums
 * are reduced from the FP32 site moments n^a - n_ref^a and j^a the step
 * computes anyway (FP32 sums over 8 sites of a thread, accumulated in FP64)
 * and copied to sums[S + 3] (mass[S] then mom[3], as in mlb_conservation)
 * asynchronously on the context's stream.  sums is host
 * memory owned by the caller that must stay valid until the stream has passed
 * the step (pinned memory makes the copy truly asynchronous); it is written
 * when the stream reaches it, so read it after mlb_synchronize or after an
 * event recorded behind the call.  NaN/Inf in the moments is reported by the
 * next synchronising call.  The step launches one kernel more than
 * mlb_launches_per_step says (the final sum).  The sums differ from
 * mlb_conservation's (FP64 sums of the populations themselves) by the FP32
 * rounding of the site moments and of the 8-site groups: at most
 * 8 x 2^-24 x sum_r |n^a - n_ref^a| for mass[a] and 8 x 2^-24 x
 * sum_a sum_r |j^a| for each momentum component.  Errors: MLB_EINVAL (sums NULL), MLB_ESTATE,
 * MLB_ECUDA. */
mlb_status mlb_step_monitored(mlb_ctx *ctx, double *sums);

/* Wait for the context's stream; reports numeric faults found by the steps. */
mlb_status mlb_synchronize(mlb_ctx *ctx);

/* Moments of the current populations (Sec. II, Eq. colonna: n^a = sum_i f^a_i,
 * n^a u^a = sum_i c_i f^a_i): n [S][N] and u [S][3][N] as FP64 host arrays
 * owned by the caller (u^a = j^a/n^a, or the barycentric velocity of
 * Eq. massdensity where n^a is below 1e-12).  Either may be NULL.
 * Synchronous.  Errors: MLB_ESTATE, MLB_ECUDA, MLB_ENUMERIC (NaN/Inf met). */
mlb_status mlb_get_moments(mlb_ctx *ctx, double *n, double *u);

/* Acceleration a^a = (Phi^a + F^a)/m^a the next step applies to the current
 * state, Phi^a the effective field of Sec. III, Eqs. (splitforce) and
 * (potmeanforce) with the velocity exchange of Eqs. (gammaab) and
 * (viscousforce): acc [S][3][N], an FP64 host array owned by the caller.
 * With the half-force shift it is F^hc + G + F^a plus the velocity-exchange
 * force at u*, the last of the Jacobi sweeps of u* = u + a(u*)/2 (see
 * mlb_set_predictor_sweeps; the first solves (I + Gamma/2) du =
 * (F^hc + G + F^a + F^v(u))/2 at each site, Gamma the local friction
 * matrix).  Synchronous; errors MLB_EINVAL (acc NULL), MLB_ESTATE, MLB_ECUDA. */
mlb_status mlb_get_acceleration(mlb_ctx *ctx, double *acc);

/* FP64 global sums of the current state, the quantities the continuity
 * equations conserve (Sec. II, Eqs. continuity and momentcomponent):
 * mass[a] = sum_r n^a (S doubles), mom[3] = sum_a m^a sum_r j^a, with
 * n^a = sum_i f^a_i and j^a = sum_i c_i f^a_i taken from the stored FP32
 * populations, every population converted to FP64 before it is added
 * (no FP32 rounding beyond the storage).  Host outputs owned by the caller;
 * any may be NULL.  Synchronous.  Returns MLB_ENUMERIC if a sum is NaN/Inf. */
mlb_status mlb_conservation(mlb_ctx *ctx, double *mass, double *mom);

/* Raw FP32 populations as stored (checkpoint and resume): f_host[a][i][r] =
 * f^a_i(r) - w_i n_ref^a, a HOST array of S x 19 x N floats owned by the
 * caller, in the velocity order of mlb_velocity_set, plus n_ref [S] (host)
 * and the step counter.  Any output pointer may be NULL.  set restores them
 * bit for bit (f_host and nref required; nref must be FP32-representable).
 * Synchronous.  Errors: MLB_EINVAL, MLB_ESTATE, MLB_ECUDA. */
mlb_status mlb_get_populations(mlb_ctx *ctx, float *f_host, double *nref, int64_t *step);
mlb_status mlb_set_populations(mlb_ctx *ctx, const float *f_host, const double *nref, int64_t step);

/* The D3Q19 velocity set the populations use: c[19][3] and weights w[19]. */
mlb_status mlb_velocity_set(int32_t *c, double *w);

/* Number of kernel launches one mlb_step(1) issues with the current settings. */
int32_t mlb_launches_per_step(const mlb_ctx *ctx);

/* Instrumentation (no counterpart in the paper).  While enabled, mlb_step
 * records a CUDA event pair around every kernel launch on the context's
 * stream.  mlb_profile_read synchronises, then returns per kernel kind k
 * (0 .. count-1, named by mlb_kernel_name) the summed device time in
 * milliseconds and the number of launches since the last read, and resets
 * them.  Arrays hold max_kernels entries; returns the number of kinds. */
mlb_status mlb_profile_enable(mlb_ctx *ctx, int32_t enable);
int32_t mlb_profile_read(mlb_ctx *ctx, double *ms, int64_t *launches, int32_t max_kernels);
const char *mlb_kernel_name(int32_t k);

/* Work decomposition tuner (no counterpart in the paper; the physics is
 * unchanged: every site's arithmetic is the same under every candidate, so
 * results are bitwise identical whatever it picks).  Times `trials` force +
 * collision passes from the current state for each candidate number of z
 * planes per block of the stencil kernels (4, 8, 12, 16, 32, not above nz) and,
 * where both exist, the fused and the split pass-2 + collision launches, and
 * keeps the fastest.  The state is untouched: a trial reads f[cur] and writes
 * the other population buffer, and cur is not advanced.  Synchronises the
 * context's stream.  zchunk_out / fused_out (may be NULL) receive the choice.
 * Errors: MLB_EINVAL for trials < 1, MLB_ESTATE before fields are set. */
mlb_status mlb_autotune(mlb_ctx *ctx, int32_t trials, int32_t *zchunk_out, int32_t *fused_out);

/* Batched ensemble (no counterpart in the paper): independent contexts of any
 * sizes and settings stepped together, captured into a CUDA graph and
 * replayed; two steps are captured per graph so that the ping-pong population
 * buffers return to their parity.  Members that take the same kernels (one or
 * two species, site-local contact values, contact shells of reach 1 or 2,
 * one predictor sweep, the fused pass 2 + collision on bulk tensor copies,
 * no active surrogate) form groups by species count, shell reach and drag
 * mode; a group of two or more steps by one launch per stage and lane
 * (mlb_batch_set_grouping; moments, pass 1, fused pass 2 + collision) over
 * all the lane's members, each block reading
 * its member and tile from a table, with bitwise the arithmetic of the
 * members' own launches.  A grouped member's column attraction, if any, runs
 * on its own stream between the moments and pass 1.  Every other member's
 * launches run on its own stream, forked from and joined back to the batch
 * stream, concurrently with the rest.  The graph and the group tables are
 * rebuilt when a member's settings or buffer parity changed since the capture.
 *   members  n >= 1 distinct contexts on the current device, each with its own
 *            stream (the default NULL stream of mlb_lattice_desc gives one);
 *            the batch does not own them and they must outlive it.
 *   stream   cudaStream_t the batch launches on; NULL = a stream it creates.
 * mlb_batch_step(nsteps) advances every member by nsteps (an odd last step
 * runs through mlb_step on the members' streams); work already queued on a
 * member's stream runs first, and later work on it runs after.  It returns
 * without waiting; mlb_batch_synchronize waits for the batch and checks every
 * member's numeric flags.  Errors: MLB_EINVAL for bad arguments, MLB_ESTATE if
 * a member has no fields or failed; a capture or launch error puts the batch
 * in a failed state (every call returns MLB_ESTATE); mlb_batch_last_error
 * gives the message. */
typedef struct mlb_batch mlb_batch;
mlb_status mlb_batch_create(mlb_ctx *const *members, int32_t n, void *stream, mlb_batch **out);
mlb_status mlb_batch_step(mlb_batch *batch, int64_t nsteps);
mlb_status mlb_batch_synchronize(mlb_batch *batch);
/* Which members are grouped and how (defaults: lanes 1, max_sites 131072).
 * Only members of at most max_sites sites join groups: a grouped block reads
 * its member's parameters from shared memory instead of the constant bank,
 * which costs a few percent in the arithmetic-bound passes, while a small
 * member's own launches leave most of the GPU idle (measured on ensembles of
 * equal members, all grouped: 16^3 members 1.7x faster, 32^3 1.2x, 64^3
 * 0.97x).  lanes 0: every member by its own launches; lanes >= 1: each group
 * is dealt into `lanes` lanes of similar work (members in order of size),
 * each lane one launch per stage on its own stream (the stream of its first
 * member), the lanes concurrently.  Takes effect at the next capture.
 * Errors: MLB_EINVAL for lanes outside 0..64 or max_sites < 1, MLB_ESTATE
 * for a failed batch. */
mlb_status mlb_batch_set_grouping(mlb_batch *batch, int32_t lanes, int64_t max_sites);
/* members stepped by grouped launches in the current capture (0 before the first) */
int32_t mlb_batch_grouped_members(const mlb_batch *batch);
const char *mlb_batch_last_error(const mlb_batch *batch);
void mlb_batch_destroy(mlb_batch *batch);

/* The rest force of pass 1 at the current state, F^hc + G + F_ext per
 * particle (Eq. potmeanforce without the velocity exchange), as FP64
 * force[S][3][N] on the host.  Synchronous.  Without tails and external
 * force it is the hard-core force alone: the training target of the
 * surrogate below. */
mlb_status mlb_get_rest_force(mlb_ctx *ctx, double *force);

/* Learned surrogate of the hard-core force (no counterpart in the paper; the
 * exact force stays as the reference).  A 3-layer 3D convolutional network
 * for binary mixtures on a periodic lattice: input (n^a - n_ref^a) in_scale_a
 * (2 channels), 3^3 convolutions to 32 and 32 channels with tanh, a 1^3
 * convolution to 6 outputs = F^a_i out_scale_a (a 5^3 receptive field).
 * The biases are part of the layout but training keeps them at zero (the
 * network is odd in its input, as the hard-core force is at linear order).
 * FP32 input, BF16 hidden activations, FP32 accumulation; the 32 -> 32 layer on the tensor
 * cores.  Parameters: mlb_net_param_count() FP32 values, layout
 * W1[27][32][2] b1[32] W2[27][32][32] b2[32] W3[6][32] b3[6] with
 * W[tap][out][in], tap = (dz+1)*9 + (dy+1)*3 + (dx+1).  The net owns its
 * device memory and stream; host arrays are the caller's and are copied.
 *   create: dims = (nx, ny, nz) of the lattices it will serve, each >= 3;
 *           parameters start at zero.
 *   forward: dn [2][N] -> force [2][3][N] (FP64 host arrays).
 *   gradient: loss = sum (net - t)^2 / sum t^2 over the 6N entries, with
 *           t = force out_scale (the squared relative force error; force must
 *           not vanish everywhere), and its gradient grad[param_count]
 *           (either output may be NULL).
 *   train:  `iters` Adam steps (beta 0.9 / 0.999) on one frame; loss of the
 *           last step.  Only the weights move: the biases keep the values
 *           last set (zero keeps the network odd in its input).
 * Errors: MLB_EINVAL (bad arguments, non-finite parameters or scales),
 * MLB_ENOMEM, MLB_ECUDA (mlb_net_last_error gives the message). */
typedef struct mlb_net mlb_net;
int64_t mlb_net_param_count(void);
mlb_status mlb_net_create(const int32_t *dims, mlb_net **out);
mlb_status mlb_net_set_params(mlb_net *net, const float *params);
mlb_status mlb_net_get_params(mlb_net *net, float *params);
mlb_status mlb_net_set_scales(mlb_net *net, const double *in_scale, const double *out_scale);
mlb_status mlb_net_forward(mlb_net *net, const double *dn, double *force);
mlb_status mlb_net_gradient(mlb_net *net, const double *dn, const double *force, float *grad, double *loss);
mlb_status mlb_net_train(mlb_net *net, const double *dn, const double *force, int32_t iters, double lr,
                         double *loss);
const char *mlb_net_last_error(const mlb_net *net);
void mlb_net_destroy(mlb_net *net);

/* Use the surrogate for the hard-core force in mlb_step (net = NULL detaches
 * it).  Binary, periodic, no tails, no drag-only mode, contact shells of
 * reach <= 2, the net's dims equal to the lattice's.  While it is active,
 * pass 1 skips the hard-core sums and takes the network's force; every
 * `recheck_every` >= 1 steps the step runs with the exact force instead and
 * compares: if the relative 2-norm error of the network's force exceeds
 * `bound` the surrogate is switched off for good (the exact force is the
 * fallback).  The net must outlive the attachment.  mlb_surrogate_status
 * reports whether it is active, the last measured error (-1 before the first
 * recheck), and the numbers of rechecks and rejections (any pointer may be
 * NULL). */
mlb_status mlb_attach_surrogate(mlb_ctx *ctx, mlb_net *net, int32_t recheck_every, double bound);
mlb_status mlb_surrogate_status(mlb_ctx *ctx, int32_t *active, double *last_error, int64_t *rechecks,
                                int64_t *rejections);

/* Device-to-device copy bandwidth in GB/s (bytes read + written per second):
 * a grid-stride float4 copy between two fresh buffers of `bytes` each
 * (>= 1 MiB; use more than the 129 MB L2), `reps` >= 1 launches timed with
 * CUDA events after two untimed ones, on the current device.  The memory is
 * allocated and released inside the call.  Errors: MLB_EINVAL, MLB_ENOMEM,
 * MLB_ECUDA.  (No counterpart in the paper: the HBM peak the kernels'
 * roofline fractions are quoted against.) */
mlb_status mlb_copy_bandwidth(int64_t bytes, int32_t reps, double *gbs);

/* FP32 FMA throughput in TFLOP/s (2 flops per FMA): 2048 threads per SM,
 * each `iters` rounds of 16 independent FMA chains (as packed FP32 pairs),
 * `reps` >= 1 launches timed with CUDA events after one untimed one, on the
 * current device.  Errors: MLB_EINVAL, MLB_ENOMEM, MLB_ECUDA.  (No
 * counterpart in the paper: the arithmetic peak the arithmetic-bound
 * kernels are quoted against.) */
mlb_status mlb_fma_throughput(int32_t iters, int32_t reps, double *tflops);

/* Conservation sums without any allocation (the paper has no counterpart:
 * this serves callers that cannot let the library allocate).  A caller whose
 * device memory is all owned by its own memory manager (a framework pool, a
 * stream-ordered allocator that must not be mixed with cudaMalloc), or that
 * must not allocate once a run is under way, cannot create a context, since
 * mlb_create obtains all of a context's device memory.  This entry point
 * computes the FP64 sums of mlb_conservation from populations the caller
 * holds on the device, and allocates nothing: no cudaMalloc or cudaFree, no
 * allocating library call.  It runs the same two kernels as mlb_conservation
 * (every population converted to FP64 before it is added), so on the same
 * populations the two give the same sums bit for bit.  Its reduction keeps its block partial sums in a
 * fixed 28 KiB array (512 blocks x (MLB_MAX_SPECIES + 3) doubles) that every
 * GPU which loads this library holds until the process exits.
 *   fdev    device pointer, [nspecies][19][nsites] FP32 populations minus
 *           w_i n_ref, in the mlb_velocity_set order (as mlb_get_populations
 *           returns them); read only
 *   nref    host array of nspecies reference densities
 *   out     device pointer to nspecies + 3 doubles: mass[a] = sum_r n^a,
 *           then sum_a sum_r j^a (masses 1); written by the call
 *   stream  cudaStream_t the two kernels are launched on (asynchronous)
 * Returns MLB_EINVAL for NULL pointers, nspecies outside 1..MLB_MAX_SPECIES
 * (more species than the fixed array holds), nsites outside 1..2^34 or a
 * non-finite nref; MLB_ECUDA if the lookup or a launch fails (no context, so
 * no message).  Every call looks up the array's device address on the
 * current device (cudaGetSymbolAddress, a host-side query that allocates
 * nothing), so a device reset between calls leaves nothing stale; the first
 * call on a device also loads the library's kernels there, so make that first
 * call before any stream capture.  All calls share the one array, which keeps
 * the last call's contents: every call overwrites each partial it reads, so
 * nothing needs clearing, but calls that overlap on the GPU (other streams,
 * other host threads) race on it and must be serialised by the caller. */
mlb_status mlb_conservation_noalloc(const float *fdev, const double *nref, int32_t nspecies, int64_t nsites,
                                    double *out, void *stream);

const char *mlb_last_error(const mlb_ctx *ctx);
const char *mlb_status_string(mlb_status s);
void mlb_destroy(mlb_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* MLB_H */
