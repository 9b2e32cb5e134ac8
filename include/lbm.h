/*
 * liblbm: GPU (sm_103a) implementation of the double-distribution-function
 * D2Q9 lattice Boltzmann model of the liquid-vapor phase transition of
 * Huang, Wu & Adams (PRL 2021), "Mesoscopic lattice Boltzmann modeling of
 * the liquid-vapor phase transition".
 *
 * The library advances the density DF f (mass, momentum) and the total-
 * kinetic-energy DF g (energy) by the fused per-step update of Eq. 12a-c:
 * pair force (Eq. 13) on the density field, moments (Eq. 14), dense-gas EOS
 * (Eq. 17), collision of f and g in moment space with the force, source,
 * compensation and viscous-dissipation terms of Supplemental Material (SM)
 * Eq. S3-S6, and pull streaming, with the conservation sums reduced in the
 * same pass.
 *
 * Conventions used by every call:
 *   - status: every function returns 0 (LBM_OK) or a negative LBM_ERR_*.
 *     lbm_last_error() returns a message for the calling thread's last
 *     failure. No call aborts the process.
 *   - NULL: a NULL handle or required pointer returns LBM_ERR_ARG before any
 *     device work; the *_destroy calls take NULL as a no-op (LBM_OK); the
 *     queries return -1 (lbm_step_count) or 0 (the node, byte and parameter
 *     counts) for a NULL handle; lbm_default_config(NULL, ...) does nothing.
 *   - units: lattice spacing dx = 1 and R, a~, b~ as configured; the lattice
 *     speed is c = sqrt(3) c_s with c_s from Eq. 19, so the time step is
 *     dt = 1 / c (not 1).
 *   - fields: row-major [ny][nx] arrays of double, index y * nx + x.
 *   - populations: [9][ny][nx] double, direction i as in SM Eq. S1:
 *     (0,0),(1,0),(0,1),(-1,0),(0,-1),(1,1),(-1,1),(-1,-1),(1,-1); they are
 *     the post-streaming (pre-collision) populations whose moments Eq. 14
 *     defines.
 *   - memory: the handle owns all device memory it allocates in lbm_init and
 *     frees it in lbm_destroy. Pointers passed in are never retained past
 *     the call. "on_device" arguments say whether a field pointer is device
 *     memory (1) or host memory (0).
 *   - streams: work is issued on cfg.stream (a cudaStream_t, or NULL for a
 *     stream the handle creates). lbm_step is asynchronous; errors detected
 *     on the device (non-finite density, a timed-out wait) are reported by
 *     the next synchronising call (lbm_synchronize, lbm_moments,
 *     lbm_conservation, lbm_step_stats, lbm_get_populations).
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LBM_OK 0
#define LBM_ERR_ARG (-1)      /* invalid argument or configuration */
#define LBM_ERR_CUDA (-2)     /* a CUDA runtime or driver call failed */
#define LBM_ERR_OOM (-3)      /* device or host allocation failed */
#define LBM_ERR_DIVERGED (-4) /* non-finite or non-positive density or temperature seen */
#define LBM_ERR_TIMEOUT (-5)  /* a device-side wait ran out its bound */
#define LBM_ERR_STATE (-6)    /* call not valid in the handle's state */
#define LBM_ERR_IO (-7)       /* checkpoint file could not be read/written */

/* Population storage precision. Collision arithmetic is FP64 for LBM_F64
 * and FP32 otherwise. The shifted formats store l_i - l_i^rest, with
 * l^rest the rest equilibrium at (rho_ref, T_ref, u = 0). */
#define LBM_F64 0
#define LBM_F32 1
#define LBM_F16S 2
#define LBM_BF16S 3

/* Case description. lbm_default_config() fills the paper's simulation
 * parameters (paragraph after Eq. 19): varpi = 1/6, gamma1 = -2,
 * gamma2 = 2, a~ = 1, b~ = 4, R = 1, Tr0 = 0.8, K_EOS = 0.479820,
 * K_INT = 2.294922, and for the rates the paper leaves open: s_p = 1,
 * s_eps = 1, sigma_e = sigma_eps = sigma_p = 1, tau_j = 0.25 (vapour) and
 * 2.5 (liquid) so that lambda_l = 10 lambda_v, c_v = 3/2 R, C_ref =
 * rho_v c_v. */
typedef struct lbm_config {
    int32_t nx, ny;        /* lattice size; nx >= 8, ny >= 8 */
    int32_t precision;     /* LBM_F64, LBM_F32, LBM_F16S, LBM_BF16S */
    int32_t walls;         /* 0: periodic box; 1: half-way bounce-back walls
                              at y = -1/2 and y = ny - 1/2, periodic in x */
    double a_t, b_t, R;    /* a~, b~ of Eq. 17 and the gas constant */
    double K_EOS, K_INT;   /* scaling factors of Eq. 17-19 */
    double Tr0;            /* reference reduced temperature: c_s (Eq. 19) is
                              taken at rho_l(Tr0); also T_ref of the shift */
    double varpi, gamma1, gamma2; /* model coefficients (SM Eq. S3-S5) */
    double s_p, s_eps;     /* f relaxation rates; s_e, s_q follow from the
                              constraint tau_p tau_q = (k+1) tau_e tau_q = 1/12 */
    double sig_e, sig_eps, sig_p; /* g relaxation rates (SM Eq. S5b) */
    double tau_j_v, tau_j_l;      /* tau_j = 1/sigma_j - 1/2, linear in rho
                                     between rho_v and rho_l (clamped);
                                     sigma_q = sigma_j */
    double c_v;            /* specific heat in units of R */
    double C_ref;          /* reference volumetric heat capacity; <= 0 means
                              rho_v(Tr0) c_v */
    double accel_x, accel_y;      /* body acceleration a (Eq. 14: F = F_pair + rho a) */
    double Tr_bottom, Tr_top;     /* fixed wall reduced temperatures; <= 0: adiabatic */
    double Tr_hot;                /* reduced temperature of a hot segment of the bottom wall */
    int32_t hot_x0, hot_len;      /* hot segment: x in [hot_x0, hot_x0 + hot_len) mod nx */
    double rho_ref;        /* shifted storage reference density; <= 0: rho_v(Tr0) */
    void* stream;          /* cudaStream_t to issue work on; NULL: own stream */
    int32_t device;        /* CUDA device ordinal */
    int32_t rounding;      /* 16-bit storage only: 0 rounds each stored value
                              to nearest; 1 (default) rounds stochastically,
                              up with probability equal to the discarded
                              fraction, from a counter-based dither of (node,
                              step, population), so that increments below
                              half a 16-bit step still act on average and
                              runs stay deterministic; other values:
                              LBM_ERR_ARG. */
    int32_t open_sides;    /* open, heated sides at constant pressure, for the
                              Stefan problem and the evaporating droplet
                              (paragraph after Eq. 19, where the outflow and
                              constant-pressure condition drives the phase
                              change; its scheme is in another paper, so
                              this one is the library's): a ghost node beyond
                              an open side carries the post-collision
                              populations of its nearest fluid node with
                              their equilibrium part moved to (rho_open,
                              T_open) at that node's velocity (non-
                              equilibrium extrapolation); populations that
                              leave through it are lost, and the pair force
                              sees rho_open beyond it. Bits: 1 bottom, 2 top
                              (both need walls = 1; they replace that wall),
                              4 left, 8 right (only as 15: all four sides).
                              0: none. Other combinations: LBM_ERR_ARG */
    double Tr_open;        /* reduced temperature of the open sides (> 0 when
                              open_sides != 0) */
    double rho_open;       /* density of the open sides; <= 0: the vapour
                              branch of Eq. 17 at Tr_open and the saturation
                              pressure at Tr0 */
    int32_t cubic;         /* 1: eliminate the cubic velocity terms of the
                              viscous stress (paragraph after Eq. 16; its
                              details are in another paper, so this is the
                              library's reading): the q_x, q_y equilibria
                              gain 3 rho u_x u_y^2 and 3 rho u_y u_x^2 (u over
                              c), and a source -c (d_x(rho u_x^3) -
                              d_y(rho u_y^3)) enters the p_xx row of the f
                              collision as dt (1 - s_p/2) R, from central
                              differences of rho u^3 that a pass before each
                              step computes. Periodic boxes only (walls = 0,
                              no open sides), single cases only; 0 (default):
                              the model as SM Eq. S3-S6 state it */
} lbm_config;

/* Quantities derived in lbm_init (Eq. 16-19, SM Eq. S3-S5 constants). */
typedef struct lbm_params {
    double Tc, pc;          /* critical point of Eq. 17 */
    double T0;              /* Tr0 * Tc */
    double rho_v, rho_l;    /* Maxwell coexistence densities at T0 */
    double p_s;             /* saturation pressure at T0 (times K_EOS) */
    double cs, c, dt;       /* Eq. 19; c = sqrt(3) c_s; dt = 1 / c */
    double G2, a, kappa;    /* Eq. 18, Eq. 16 */
    double cv, Cref;
    double beta, kS, hS, bS; /* SM: beta, k, h, b */
    double se, sq;          /* from the relaxation constraint */
    double rho_open, T_open; /* state of the open sides (0 without them) */
} lbm_params;

typedef struct lbm_handle lbm_handle;

/* Message for the calling thread's last failed call ("" if none). */
const char* lbm_last_error(void);

/* Fill *cfg with the defaults described above for an nx x ny box. */
void lbm_default_config(lbm_config* cfg, int32_t nx, int32_t ny);

/* Create a case: validates cfg (LBM_ERR_ARG on e.g. s outside (0,2),
 * non-positive K, Tr0 >= 1, nx or ny < 8), derives lbm_params (Maxwell
 * coexistence at Tr0, Eq. 16-19), allocates two device copies of the
 * f and g planes plus reduction scratch. Populations start at zero; call
 * lbm_set_fields or lbm_set_populations next. */
int lbm_init(const lbm_config* cfg, lbm_handle** out);

int lbm_get_params(const lbm_handle* h, lbm_params* out);

/* Maxwell coexistence of the EOS of cfg (Eq. 17: a~, b~, R, K_EOS) at
 * reduced temperature Tr: out[0] rho_v, out[1] rho_l, out[2] saturation
 * pressure. Host only; LBM_ERR_ARG if Tr is not in (0.3, 1). */
int lbm_maxwell(const lbm_config* cfg, double Tr, double out[3]);

/* Coexistence across a curved interface at reduced temperature Tr (host
 * only): the densities with equal chemical potential whose pressures
 * (Eq. 17 with K_EOS) differ by dp, the liquid's above the vapour's --
 * Laplace's law for a droplet of radius R in 2-D takes dp = sigma / R.
 * out[0] rho_v, out[1] rho_l, out[2] the vapour's pressure; dp = 0 gives
 * lbm_maxwell's values. LBM_ERR_ARG if Tr is not in (0.3, 1) or no such
 * pair exists. */
int lbm_coexistence(const lbm_config* cfg, double Tr, double dp, double out[3]);

/* Surface tension of a planar interface at reduced temperature Tr from the
 * square-gradient theory of the model's pressure tensor (Eq. 11, kappa of
 * Eq. 16 with G of Eq. 18): sigma = int sqrt(2 kappa K_EOS Omega) drho
 * over [rho_v, rho_l], Omega the grand-potential excess of Eq. 17's free
 * energy. With the paper's K_EOS, K_INT it is 0.01 at Tr = 0.8 (the value
 * the paper prescribes). Host only. */
int lbm_surface_tension(const lbm_config* cfg, double Tr, double* sigma);

/* The full EOS of cfg (Eq. 17: p = K_EOS (p_CS - a~ rho^2), p_CS the
 * Carnahan-Starling term) at density rho and temperature T, both in the
 * units lbm_moments reports (T absolute, not reduced). Host only;
 * LBM_ERR_ARG for a null pointer or rho outside (0, 4 / b~). */
int lbm_eos_pressure(const lbm_config* cfg, double rho, double T, double* p);

/* Initial populations from macroscopic fields (rho, u_x, u_y, T), each
 * [ny][nx] double: m = m^eq - dt/2 F_m and n = n^eq - dt/2 q_m at every
 * node (SM Eq. S3, S4), so that Eq. 14 returns the given fields to the
 * storage's precision (per-node arithmetic in FP64 for LBM_F64 storage, in
 * FP32 for the others). Synchronous. */
int lbm_set_fields(lbm_handle* h, const double* rho, const double* ux,
                   const double* uy, const double* T, int on_device);

/* Advance n >= 0 time steps (Eq. 12a-c), asynchronously on the stream. */
int lbm_step(lbm_handle* h, int n);

/* Macroscopic fields of the current state (Eq. 13, 14), [ny][nx] double
 * each; any pointer may be NULL. Per-node arithmetic in FP64 for LBM_F64
 * storage, in FP32 for the others. Synchronous. */
int lbm_moments(lbm_handle* h, double* rho, double* ux, double* uy,
                double* T, int on_device);

/* Conservation record of the current state, FP64 sums over all nodes:
 * out[0] mass, out[1..2] momentum sum rho u (Eq. 14), out[3] sum rho e_k,
 * out[4] total energy sum (rho e_k + rho eps_p), rho eps_p = rho V_mean / 2
 * with V_mean = -2 a rho - kappa lap rho (Eq. 8, isotropic 9-point
 * Laplacian), out[5] max |u|. Synchronous. */
int lbm_conservation(lbm_handle* h, double out[6]);

/* The same record, as reduced inside the most recent time step for the
 * state that step started from; out[6] = number of nodes in it with a
 * non-finite or non-positive density or temperature or a non-finite
 * velocity (any such node makes the step's synchronising call return
 * LBM_ERR_DIVERGED), out[7] = number of time steps the handle has
 * executed. Synchronous. */
int lbm_step_stats(lbm_handle* h, double out[8]);

/* Read / write the post-streaming populations, host arrays [9][ny][nx]
 * double each. Synchronous. Shifted formats round on write. */
int lbm_get_populations(lbm_handle* h, double* f, double* g);
int lbm_set_populations(lbm_handle* h, const double* f, const double* g);

/* Checkpoint: the raw stored state (both DFs, storage precision), the step
 * counter and a hash of the configuration (every lbm_config field but the
 * stream and the device), to a binary file; lbm_load refuses, with
 * LBM_ERR_ARG and the handle unchanged, a file whose lattice or
 * configuration differs from the handle's. Resume is bitwise. */
int lbm_save(lbm_handle* h, const char* path);
int lbm_load(lbm_handle* h, const char* path);

/* Wait for queued work; reports device-side errors (LBM_ERR_DIVERGED,
 * LBM_ERR_TIMEOUT). */
int lbm_synchronize(lbm_handle* h);

/* Steps taken since init (or restored by lbm_load). */
int64_t lbm_step_count(const lbm_handle* h);

/* Default bound on each wait of the step kernel for a tile's copies: 2 s. */
#define LBM_TILE_WAIT_DEFAULT_NS 2000000000LL

/* Bound, in nanoseconds, on each wait of the step kernel for the copies of
 * a tile into shared memory (failure detection; not a parameter of the
 * paper's method). A wait that runs out ends the launch early in every
 * block that met it, sets the handle's status, and the next synchronising
 * call returns LBM_ERR_TIMEOUT; the state is then undefined until the next
 * lbm_set_fields, lbm_set_populations or lbm_load. 0 means no waiting: a
 * tile whose copies have not landed when its turn comes times out, which a
 * step from a fresh state always meets (its first copies were issued just
 * before). The kernel never exits with a copy in flight: after a timeout it
 * still waits, within the default bound, for the copies it has issued.
 * ns < 0: LBM_ERR_ARG. Takes effect from the next lbm_step. */
int lbm_set_tile_wait(lbm_handle* h, int64_t ns);

/* Bytes of population traffic one time step moves at the algorithmic
 * minimum (one read and one write of 18 populations per node). */
double lbm_bytes_per_step(const lbm_handle* h);

int lbm_destroy(lbm_handle* h);

/* ---- Batched cases -------------------------------------------------------
 * Many independent cases (each its own lattice size, temperature and
 * droplet) advanced together: one persistent launch per time step walks a
 * work list of (case, tile) items, with the cases' tensor maps and constants
 * in device tables. The rows are the same model as lbm_step; a case in a
 * batch gives the same populations as that case on its own handle with the
 * same precision, up to floating-point rounding (the two kernels are
 * compiled separately). With 16-bit storage the batch rounds its stores
 * as lbm_config.rounding says, stochastically by default, with the dither
 * of a single handle keyed by (node, batch step count), which the device
 * keeps. Extension of the paper's method for parameter sweeps (the paper
 * runs single cases). Requirements: every cfgs[i] periodic (walls = 0, no
 * open sides), one precision for all (LBM_F32, LBM_F16S or LBM_BF16S), one
 * rounding for all; the stream and device of cfgs[0] are used. */
typedef struct lbm_batch lbm_batch;

int lbm_batch_init(const lbm_config* cfgs, int32_t ncases, lbm_batch** out);
/* As lbm_set_fields, for case i. */
int lbm_batch_set_fields(lbm_batch* b, int32_t i, const double* rho, const double* ux,
                         const double* uy, const double* T, int on_device);
/* Advance every case n steps (CUDA-graph replay), asynchronously. */
int lbm_batch_step(lbm_batch* b, int n);
/* As lbm_moments / lbm_conservation / lbm_get_populations, for case i. */
int lbm_batch_moments(lbm_batch* b, int32_t i, double* rho, double* ux, double* uy,
                      double* T, int on_device);
int lbm_batch_conservation(lbm_batch* b, int32_t i, double out[6]);
int lbm_batch_get_populations(lbm_batch* b, int32_t i, double* f, double* g);
/* Case i's conservation record as reduced inside the most recent step
 * (per-tile FP32 partial sums, summed per case in FP64): layout of
 * lbm_step_stats out[0..6]; out[7] = the steps the batch has executed, as
 * counted on the device (the count that keys stochastic rounding).
 * Synchronous. */
int lbm_batch_step_stats(lbm_batch* b, int32_t i, double out[8]);
/* Steps the batch has executed (host count; includes autotuner trials). */
int64_t lbm_batch_step_count(const lbm_batch* b);
/* As lbm_set_tile_wait, for the batch's step kernel: the bound on each wait
 * for an item's copies (0: no waiting); a wait that runs out is reported as
 * LBM_ERR_TIMEOUT by the next synchronising call, and the cases' states are
 * undefined until set again. ns < 0: LBM_ERR_ARG. */
int lbm_batch_set_tile_wait(lbm_batch* b, int64_t ns);
/* Autotuner: times every candidate (tile shape x work-list order) for
 * trial_steps steps on the current state and keeps the fastest; the trial
 * steps are real steps of every case (the state advances). choice[0] =
 * tile shape index, choice[1] = order index (0 case-major, 1 largest case
 * first, 2 round-robin over cases); ms[k] (may be NULL, >= 6 entries) =
 * the time per step of candidate k = 3 * shape + order. Synchronous. */
int lbm_batch_autotune(lbm_batch* b, int trial_steps, int32_t choice[2], double* ms);
/* Select a candidate directly (tile shape, order). */
int lbm_batch_select(lbm_batch* b, int32_t shape, int32_t order);
int lbm_batch_get_params(const lbm_batch* b, int32_t i, lbm_params* out);
int lbm_batch_synchronize(lbm_batch* b);
int64_t lbm_batch_nodes(const lbm_batch* b);
double lbm_batch_bytes_per_step(const lbm_batch* b);
int lbm_batch_destroy(lbm_batch* b);

/* ---- Learned surrogate ---------------------------------------------------
 * A convolutional neural operator that advances the macroscopic fields
 * (rho, u_x, u_y, T) of a periodic case by K lattice steps in one jump, with
 * the LB step as its fallback and arbiter. Not in the paper: an extension of
 * the method for faster time-to-solution. Network (3x3 convolutions,
 * periodic padding, bias; BF16 tensor-core kernels, FP32 accumulation):
 *   h0 = lift(x); h_{b+1} = h_b + conv_b2(relu(conv_b1(relu(h_b))));
 *   y  = x + proj(relu(h_B)),
 * on normalised fields x_c = (field_c - off[c]) / scale[c]; with
 * conserve_mass, an output layer then sets y_rho -= mean over the image of
 * (y_rho - x_rho), so that every jump keeps each image's mass (the LB
 * conserves it exactly on a periodic box). Parameters in
 * lbm_surrogate_set_params order: lift weight [9][C][4], lift bias [C], for
 * each block w1 [9][C][C], b1 [C], w2 [9][C][C], b2 [C], proj weight
 * [9][4][C], proj bias [4] (weight index [tap][out][in], tap = 3 (dy + 1) +
 * (dx + 1) reading input pixel (y + dy, x + dx)). Field arrays: device
 * double, 4 planes [4][N][H][W] (rho, u_x, u_y, T); W a multiple of 16. */
typedef struct lbm_surrogate lbm_surrogate;

typedef struct lbm_surrogate_config {
    int32_t channels;    /* C: 64 */
    int32_t blocks;      /* B: 6 */
    int32_t K;           /* lattice steps per jump */
    int32_t conv_path;   /* 3x3 convolutions (forward and input gradient):
                            0 tcgen05 MMAs with tensor-memory accumulators,
                            1 warp-level mma.sync; weight gradients use
                            mma.sync either way */
    double norm_off[4];  /* normalisation offsets of rho, u_x, u_y, T */
    double norm_scale[4];
    void* stream;        /* cudaStream_t; NULL: own stream */
    int32_t device;
    int32_t conserve_mass;  /* nonzero: the mass-conserving output layer */
} lbm_surrogate_config;

int lbm_surrogate_create(const lbm_surrogate_config* cfg, lbm_surrogate** out);
int64_t lbm_surrogate_num_params(const lbm_surrogate* s);
/* Host FP32 arrays of lbm_surrogate_num_params values, in the order above. */
int lbm_surrogate_set_params(lbm_surrogate* s, const float* params);
int lbm_surrogate_get_params(lbm_surrogate* s, float* params);
/* One jump for N fields: out = network(in) (device arrays). Synchronous. */
int lbm_surrogate_forward(lbm_surrogate* s, const double* in, int32_t N, int32_t H, int32_t W, double* out);
/* Loss (mean squared error of the normalised fields) and, if grads is not
 * NULL, its gradient in parameter order (host FP32). Synchronous. */
int lbm_surrogate_loss_grad(lbm_surrogate* s, const double* in, const double* target, int32_t N, int32_t H,
                            int32_t W, double* loss, float* grads);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) on a minibatch;
 * returns the minibatch loss before the step. Synchronous. */
int lbm_surrogate_train_step(lbm_surrogate* s, const double* in, const double* target, int32_t N, int32_t H,
                             int32_t W, double lr, double* loss);
/* Rollout on a periodic FP32/FP64 case: njumps times, snapshot the state,
 * predict K steps ahead, re-initialise the populations from the predicted
 * fields, and let the LB run verify_steps steps from that surrogate state
 * (the LB as arbiter: a state it cannot advance counts as a rejected jump);
 * then compare before and after the two quantities the model conserves, mass and total
 * energy (lbm_conservation out[0] and out[4]; sum rho e_k is not one of
 * them, it exchanges latent heat with the pair potential as liquid
 * evaporates), and the position of the interface: its mean displacement
 * D / L in lattice units, with D the number of nodes whose phase (liquid:
 * rho above (rho_v + rho_l) / 2) the jump changed and L = (pi / 4) E the
 * interface length before the jump from its E liquid-vapour edges between
 * lattice neighbours; and, node by node, what the verification steps did
 * to the prediction: the largest change of a node's density and of its
 * temperature between the predicted state and the verified one, each over
 * that field's largest value in the prediction (a local defect that the
 * global sums cannot see, such as a one-node temperature spike, is what
 * the LB moves most). An unphysical prediction (non-finite, rho <= 0 or
 * T <= 0), a relative mass or energy change above drift_tol, a
 * displacement above iface_tol, or a local change above field_tol restores
 * the snapshot and runs K + verify_steps LB steps instead. Every jump thus
 * advances the lattice by K + verify_steps steps, and the handle's step
 * count (lbm_step_count, and the device copy that keys stochastic
 * rounding) by the same. LBM_ERR_DIVERGED is
 * returned only if those fallback LB steps diverge.
 * stats (may be NULL, >= 17): [0] jumps accepted, [1] fallbacks,
 * [2] ms in surrogate jumps (prediction, checks, re-initialisation and
 * verification: [12] + [13] + [14]), [3] ms in fallback LB steps, [4]
 * largest accepted mass drift, [5] largest accepted energy drift, [6..7]
 * largest mass and energy drift over all jumps, [8] largest interface
 * displacement over all jumps, [9] jumps with an unphysical prediction,
 * [10] jumps whose verification steps diverged, [11] ms reading the state
 * before each jump (fields, conservation record, checks, snapshot), [12] ms
 * in the network, [13] ms in the checks of the prediction, the
 * re-initialisation of the populations and the conservation record, [14]
 * ms in the verification steps, [15] and [16] the largest local change of
 * density and of temperature over all verified jumps. Synchronous. */
int lbm_surrogate_rollout(lbm_surrogate* s, lbm_handle* h, int32_t njumps, int32_t verify_steps, double drift_tol,
                          double iface_tol, double field_tol, double* stats);
int lbm_surrogate_destroy(lbm_surrogate* s);

/* Largest lattice (nx * ny) lbm_conservation_noalloc accepts. */
#define LBM_NOALLOC_MAX_NODES (1 << 20)

/* The conservation record of lbm_conservation, for populations that live in
 * caller-owned device memory, computed without allocating any memory and
 * without a handle. It is for callers that cannot call cudaMalloc -- for
 * example code running while another framework owns the device memory
 * pool, or code on a path where an allocation is not allowed -- since
 * lbm_init allocates. The paper has no counterpart: this is an interface
 * of this library only.
 *   cfg    case description as for lbm_init (nx, ny, walls, EOS and model
 *          parameters, body force); its stream, device and precision
 *          fields are ignored. nx * ny above LBM_NOALLOC_MAX_NODES returns
 *          LBM_ERR_ARG with a message naming the limit.
 *   f, g   device arrays [9][ny][nx] of double: post-streaming populations
 *          (the layout of lbm_get_populations), read only.
 *   out    device array of at least 7 doubles, written asynchronously:
 *          out[0..5] as lbm_conservation, out[6] the number of nodes with a
 *          non-finite or non-positive density or temperature or a
 *          non-finite velocity.
 *   stream cudaStream_t to run on (NULL: the legacy default stream); the
 *          work runs on the calling thread's current device.
 * Scratch: a fixed device array inside the library (about 8.3 MiB on every
 * GPU that loads it, held until the process exits) replaces allocations.
 * The first call on each device looks up that array's device address, so
 * make it before any stream capture. All calls share the array and it keeps
 * the previous call's contents (the completion counter is cleared at the
 * start of each call): calls that can overlap on the GPU -- on different
 * streams, or from several threads -- race on it and must be serialised by
 * the caller. */
int lbm_conservation_noalloc(const lbm_config* cfg, const double* f, const double* g,
                             double* out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H */
