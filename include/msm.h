/*
 * msm.h -- C ABI of libmsm, the GB300 (sm_103a) engine for the DPD-CGMD
 * multiscale blood-clot model with multiple time stepping (arXiv 2205.14121).
 *
 * The model: DPD plasma (Eq. 1), CGMD platelets -- harmonic bonds, LJ 12-6
 * and Morse (Eq. 2) --, the fluid-platelet interface (Eq. 3), inter-platelet
 * Morse + receptor term (Eq. 4), integrated by the multi-level RESPA loop of
 * Table 1, with the per-platelet step ratio chosen by the learned controller
 * of Table 2 (Sec. 3.3).
 *
 * Conventions for every entry point
 *  - Return value: MD_OK (0) or a negative MD_E* code; md_last_error() gives
 *    a message.  Nothing aborts, traps or exits.
 *  - Device work is ordered on the CUDA stream given to md_init(); entry
 *    points that return host data synchronise that stream first.
 *  - Particle ids are the row numbers of the arrays given to
 *    md_set_particles(); storage is re-sorted internally by cell, but every
 *    array read back is in id order.
 *  - One md_system per host thread; calls on one system are not reentrant.
 *  - Units are reduced DPD units (m = kT = rc = 1).
 */
#ifndef MSM_H
#define MSM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define MD_OK             0
#define MD_EINVAL        (-1)   /* bad argument or configuration            */
#define MD_ENOMEM        (-2)   /* workspace smaller than md_workspace_size */
#define MD_ECUDA         (-3)   /* a CUDA runtime call failed               */
#define MD_ENBR_OVERFLOW (-4)   /* a neighbour list exceeded its capacity   */
#define MD_EUNSTABLE     (-5)   /* NaN/Inf state or a particle left the box */
#define MD_ETIMEOUT      (-6)   /* a bounded device wait gave up            */
#define MD_ENOTRAINED    (-7)   /* the controller has no weights loaded     */
#define MD_ETOOLARGE     (-8)   /* n beyond a fixed static scratch capacity */

/* ---- force levels (Table 1 component splitting) ------------------------- */
#define MD_LEVEL_FLUID 1u  /* plasma-plasma and plasma-wall DPD + body force */
#define MD_LEVEL_IFACE 2u  /* DPD between platelet and plasma/wall (Eq. 3)   */
#define MD_LEVEL_PLT   4u  /* bonds, LJ (Eq. 2), receptor Morse (Eq. 4)      */
#define MD_LEVEL_ALL   7u

/* ---- configuration flags ----------------------------------------------- */
#define MD_CFG_WALLS        1  /* frozen wall layers outside y in [0,Ly], bounce-back */
#define MD_CFG_LEES_EDWARDS 2  /* sliding periodic images in y at shear_rate       */
#define MD_CFG_MORSE_STANDARD 4 /* morse_alpha is the standard form's range a, U =
                                   D [e^(-2a(r-r0)) - 2 e^(-a(r-r0))]: the printed
                                   form of Eq. 2 with alpha = 2 a r0 (default: the
                                   printed form's alpha)                             */
#define MD_CFG_IFACE_LJ     8  /* Eq. 3 with an LJ conservative term: the plasma-
                                   platelet conservative force is the LJ (lj_eps,
                                   lj_sigma) cut at its minimum 2^(1/6) lj_sigma
                                   instead of a_fp (1 - r/rc); dissipative and random
                                   parts as Eq. 1                                     */
#define MD_CFG_UNIFORM_NOISE 16 /* zeta_ij of Eq. 1 / Eq. 3 as a uniform variate of
                                   zero mean and unit variance, sqrt(3) (2u - 1) with
                                   u = (b + 1/2) 2^-24 from the top 24 bits b of the
                                   pair's first Philox word, instead of the normal
                                   variate the paper names (a speed option: the
                                   fluctuation-dissipation balance needs only the
                                   first two moments)                                 */

/* ---- neighbour-list kinds ---------------------------------------------- */
#define MD_LIST_FLUID 0  /* plasma-plasma, plasma-wall (half list)             */
#define MD_LIST_IFACE 1  /* platelet rows -> plasma/wall partners              */
#define MD_LIST_LJ    2  /* platelet-platelet LJ pairs (half list)             */
#define MD_LIST_MORSE 3  /* receptor pairs of different platelets (half list)  */

/*
 * Particle tag (int32): -1 plasma, -2 wall, p >= 0 platelet id p; bit 30 set
 * on receptor sites.  Rest positions X0 are used only for the same-platelet
 * LJ exclusion (pairs closer than lj_excl at rest feel no LJ).
 */
#define MD_TAG_FLUID    (-1)
#define MD_TAG_WALL     (-2)
#define MD_RECEPTOR_BIT (1 << 30)

/*
 * System configuration.  Defaults follow the paper's model as read for the
 * synthetic systems: Eq. 1 a = 25 (plasma-plasma, plasma-wall), gamma = 4.5,
 * sigma = 3, rc = 1; Eq. 3 interface DPD a_fp = 50; Eq. 2 LJ eps = 1,
 * sigma = 0.8, cut-off 2.5 sigma, between particles of different platelets
 * (lj_excl = 1e30: a same-platelet pair feels LJ only when its rest distance
 * is at least lj_excl), k_b = 100, angle constant k_theta = 5 on the bending
 * triplets given to md_set_angles; Eq. 2/4 Morse D = 2, alpha = 2, r0 = 1 with
 * cut-off 5.
 */
typedef struct md_config {
    int64_t  n;               /* particles (plasma + wall + platelet), 1 .. 2^27  */
    int64_t  n_bonds;         /* harmonic bonds                                   */
    int64_t  n_plt_particles; /* particles with tag >= 0                          */
    int64_t  n_receptors;     /* platelet particles with the receptor bit         */
    int32_t  n_platelets;     /* platelets (largest platelet id + 1)              */
    int32_t  flags;           /* MD_CFG_*                                         */
    double   box[3];          /* fluid region [0,Lx) x [0,Ly) x [0,Lz)            */
    double   wall;            /* wall layer thickness (MD_CFG_WALLS)              */
    double   shear_rate;      /* Lees-Edwards rate (MD_CFG_LEES_EDWARDS)          */
    double   body_force;      /* g along +x on every non-wall particle            */
    double   dt;              /* fluid step dt_f                                  */
    double   skin;            /* Verlet skin added to every list cut-off          */
    double   rc, a_ff, a_fw, a_fp, gamma, sigma;          /* Eq. 1 / Eq. 3       */
    double   lj_eps, lj_sigma, lj_rc, lj_excl;            /* Eq. 2 LJ            */
    double   morse_D, morse_alpha, morse_r0, morse_rc, f_A; /* Eq. 2 / Eq. 4     */
    double   k_bond;                                       /* Eq. 2 bonds        */
    uint64_t seed;            /* key of the Philox4x32-10 pair noise              */
    int32_t  cap_fluid, cap_iface, cap_lj, cap_morse; /* list capacities per row;
                                                   0: 96, 96, 1024, 256        */
    double   skin_plt;        /* skin of the platelet particles (0: skin): the
                                 LJ and Morse lists reach cut-off + skin_plt, the
                                 interface list rc + (skin + skin_plt) / 2, and a
                                 platelet particle trips a rebuild at skin_plt/2 */
    int64_t  n_angles;        /* angle triplets of the Eq. 2 angle term          */
    double   k_angle;         /* its constant k_theta in U = k_theta (theta -
                                 theta0)^2 (as printed, no 1/2); default 5       */
} md_config;

/* Fill *cfg with the defaults above for n particles in box (no platelets). */
int md_config_defaults(md_config *cfg);

/*
 * Bytes of device workspace md_init needs for cfg (256-byte aligned start).
 * The workspace holds every per-particle array, the neighbour lists and the
 * scratch of the sort, list build and reductions.
 */
int md_workspace_size(const md_config *cfg, size_t *bytes);

typedef struct md_buffers {
    void  *workspace;       /* device memory, caller-owned, >= md_workspace_size */
    size_t workspace_bytes;
} md_buffers;

typedef struct md_system md_system;

/*
 * Create a system on the current CUDA device.  cuda_stream: a cudaStream_t
 * (NULL = legacy default stream).  The library never frees bufs->workspace;
 * it owns only its host-side state and a few bytes of pinned host memory,
 * released by md_destroy().
 * Errors: MD_EINVAL (inconsistent cfg, a periodic dimension shorter than three
 * list cells), MD_ENOMEM (workspace too small), MD_ECUDA.
 */
int md_init(const md_config *cfg, const md_buffers *bufs, void *cuda_stream, md_system **out);

/* Release host-side state; the workspace stays the caller's. */
void md_destroy(md_system *sys);

/* Message for the last error on sys (static string when sys is NULL). */
const char *md_last_error(const md_system *sys);

/*
 * Load the particle state from HOST arrays in id order:
 * x[n*3] positions (FP64, fluid region coordinates; walls outside y in [0,Ly]),
 * v[n*3] velocities, tag[n] tags, X0[n*3] rest positions (may be NULL: X0 = x).
 * Resets the step counter to step0 and the time to step0*dt; marks the
 * neighbour lists and forces stale (rebuilt and recomputed on the next call
 * that needs them).  Errors: MD_EINVAL, MD_ECUDA.
 */
int md_set_particles(md_system *sys, const double *x, const double *v, const int32_t *tag,
                     const double *X0, int64_t step0);

/*
 * Load a new state of the particle set last given to md_set_particles():
 * x[n*3] positions and v[n*3] velocities as HOST arrays in id order; tags,
 * rest positions and bonds are kept on the device (nothing but x and v
 * crosses to the GPU).  Resets the step counter to step0 and marks forces
 * stale.  When neighbour lists are built, the state goes into their particle
 * order and they are kept if it passes the rebuild check of a step (every
 * particle within its skin threshold of the last build, plasma beyond skin/2
 * listed for the fast-particle pass); otherwise the next call rebuilds them.
 * Synchronises the stream.  Errors: MD_EINVAL (null argument, or no earlier
 * md_set_particles), MD_EUNSTABLE (non-finite or escaped position), MD_ECUDA.
 */
int md_set_xv(md_system *sys, const double *x, const double *v, int64_t step0);

/*
 * Harmonic bonds (Eq. 2) as HOST arrays: ij[nb*2] particle ids, r0[nb] rest
 * lengths.  nb must equal cfg.n_bonds.  Errors: MD_EINVAL, MD_ECUDA.
 */
int md_set_bonds(md_system *sys, const int32_t *ij, const double *r0, int64_t nb);

/*
 * Angle term of Eq. 2, U = k_angle (theta - theta0)^2 summed over triplets,
 * as HOST arrays: ijk[na*3] particle ids (i, vertex j, k) of one platelet,
 * theta0[na] rest angles in radians.  theta is the angle at j between the
 * minimum images of x_i - x_j and x_k - x_j; the force on i is
 * 2 k (theta - theta0) / sin(theta) (e_kj - cos(theta) e_ij) / |x_i - x_j|
 * (sin theta held at 1e-3 at least), on k likewise, on j minus their sum.
 * The term belongs to the platelet level (MD_LEVEL_PLT) and, under AI-MTS,
 * to its platelet's step ratio.  na must equal cfg.n_angles.
 * Errors: MD_EINVAL (count, an id out of range, a triplet spanning
 * platelets), MD_ECUDA.
 */
int md_set_angles(md_system *sys, const int32_t *ijk, const double *theta0, int64_t na);

/*
 * Verlet-skin neighbour lists (Table 1, "neighbor lists construction"):
 * cell binning and counting sort of every particle array (K1), then every
 * list (K2).  force = 0 rebuilds only when some particle moved more than
 * skin/2 (minus a safety margin) since the last build.  list_mask: bit per
 * MD_LIST_* kind (all kinds are rebuilt together; the mask is validated only).
 * Errors: MD_ENBR_OVERFLOW (a row exceeded its capacity; raise cap_*),
 * MD_ECUDA.
 */
int md_neighbor_build(md_system *sys, uint32_t list_mask, int force);

/* flags of md_forces */
#define MD_FORCE_VIRIAL 1u  /* also accumulate the FP64 pair virial */
/* Deterministic forces: every pair and bond term, evaluated with the particle
 * of lower id first, is rounded to a multiple of 2^-32 and summed as a 64-bit
 * integer per particle and level.  The result does not depend on the order of
 * the atomic updates (bit-identical from run to run and whatever the particle
 * order), and the pair terms cancel exactly: without walls and body force the
 * forces read back by md_read_forces (which takes these sums exactly while no
 * step, rebuild or new state intervened) add up to exactly zero.  The FP32
 * level buffers the integrator uses are the sums rounded to FP32.  The virial
 * is not covered.  Slower than the default. */
#define MD_FORCE_DETERMINISTIC 2u

/*
 * Forces of the levels in level_mask at the current state (Eq. 1-4),
 * written to each level's force buffer.  The pair noise zeta_ij is drawn
 * from Philox4x32-10 with counter (min id, max id, n, c) and key seed, where
 * (n, c) is the time index of the current state (n = completed fluid steps,
 * c = completed interface substeps); F^R = sigma w zeta / sqrt(dt_level).
 * Rebuilds stale lists first.  Errors: MD_ENBR_OVERFLOW, MD_ECUDA.
 */
int md_forces(md_system *sys, uint32_t level_mask, uint32_t flags);

/*
 * Copy the sum of the level forces in level_mask to HOST f[n*3] (FP64, id
 * order); stale forces (new particles, or after an AI-MTS call) are
 * recomputed first.  Synchronises the stream.  Errors: MD_EINVAL, MD_ECUDA.
 */
int md_read_forces(md_system *sys, uint32_t level_mask, double *f);

/*
 * Copy the state to HOST arrays in id order: x[n*3] FP64 master positions,
 * v[n*3] velocities (FP32 widened), x32[n*3] the FP32 position copy the
 * force kernels read (any pointer may be NULL).  Synchronises the stream.
 */
int md_read_particles(md_system *sys, double *x, double *v, float *x32);

/* ---- multiple time stepping (Table 1) ----------------------------------- */
#define MD_MODE_STS   0  /* single time step: every force every dt_f           */
#define MD_MODE_RESPA 1  /* k_m interface substeps, k_p platelet substeps each  */
#define MD_MODE_AI    2  /* per-platelet k (md_set_platelet_levels), Table 2    */

#define MD_SCHED_DIRECT 1  /* launch every kernel from the host (no CUDA graph) */
#define MD_SCHED_RECORD 2  /* append the per-platelet measurements after every
                              outer step to the feature ring (md_record_features) */
#define MD_SCHED_DETERMINISTIC 4  /* every force of the call summed as with
                              MD_FORCE_DETERMINISTIC (64-bit fixed point, lower
                              id first), so that a trajectory does not depend
                              on the order of the atomic updates: two runs from
                              the same state, or a run resumed from md_get_state,
                              agree bit for bit.  STS and RESPA only (MD_EINVAL
                              with MD_MODE_AI); slower than the default */

typedef struct md_mts_schedule {
    int32_t mode;        /* MD_MODE_*                                            */
    int32_t k_m;         /* interface substeps per fluid step (>= 1)             */
    int32_t k_p;         /* platelet substeps per interface step (RESPA)         */
    int32_t flags;       /* MD_SCHED_* bits                                      */
} md_mts_schedule;

/*
 * Advance n_outer fluid steps.  STS: velocity-Verlet with dt_f for every
 * force.  RESPA: Table 1 read symmetrically -- half-kick with the fluid
 * forces, k_m interface substeps (half-kick, k_p platelet kick-drift-force-
 * kick substeps, interface forces, half-kick), fluid forces, half-kick.
 * Positions are FP64 masters; the lists are rebuilt on device when the
 * displacement check trips (no host round trip per step).  After the first
 * step, the remaining n_outer - 1 steps replay one captured CUDA graph
 * (a WHILE node over the outer step, IF nodes around the rebuild chain)
 * unless sched->flags has MD_SCHED_DIRECT or kernel profiling is on.
 * Errors: MD_ENBR_OVERFLOW, MD_EUNSTABLE, MD_ECUDA (checked once at the end).
 */
int md_mts_step(md_system *sys, int64_t n_outer, const md_mts_schedule *sched);

/*
 * AI-MTS step ratios (Sec. 3.3, Table 2): k[P] (HOST, P = cfg.n_platelets)
 * platelet substeps per interface step for each platelet, as the controller
 * predicts them (classes {1, 2, 5, 10, 20}).  MD_MODE_AI then cuts each
 * interface step into K = lcm(k) substeps of dt_m / K in which every
 * platelet particle drifts.  Each platelet-level term -- a bond, an LJ or a
 * Morse pair -- lives on the grid of the finer of its two platelets,
 * c = max(k_i, k_j), and is integrated there by velocity-Verlet with step
 * dt_m / c: half kicks at the ends of the interface step, full kicks at its
 * interior points K/c, 2K/c, ...  Both ends of a pair get the same impulse at
 * the same time, so momentum is conserved, and with all k_p equal this is
 * MD_MODE_RESPA with that k_p.  During an AI-MTS call the platelet force
 * buffer holds impulses; the call ends by evaluating the plain platelet
 * forces of the final state.  Each k_p >= 1 and K <= MD_AI_K_LCM_MAX.  Copies synchronously;
 * the ratios may change between md_mts_step calls (a new K recaptures the
 * step graph).  Errors: MD_EINVAL (no platelets, k out of range), MD_ECUDA.
 */
#define MD_AI_K_LCM_MAX 64
int md_set_platelet_levels(md_system *sys, const int32_t *k);

/* Observables (Sec. 4.2), FP64, reduced on the device. */
typedef struct md_observables_t {
    int64_t step;            /* completed fluid steps                          */
    double  time;            /* step * dt_f                                    */
    double  momentum[3];     /* total momentum of mobile particles             */
    double  kinetic;         /* 1/2 sum m v^2 (mobile)                         */
    double  temperature;     /* sum m|v-u|^2 / N_dof; u: the Lees-Edwards profile,
                                or with walls the mean v_x of the mobile particles
                                in each of 20 slabs of y (N_dof = 3N - 3, 3N with walls) */
    double  kin_tensor[9];   /* sum m (v-u)_a (v-u)_b                          */
    double  virial_c[9];     /* sum over pairs r_a F^C_b (conservative), last forces with MD_FORCE_VIRIAL */
    double  pressure;        /* (trace kin_tensor + trace virial_c) / (3V)     */
    int64_t n_builds;        /* neighbour-list builds so far                   */
    int64_t max_rows[4];     /* longest list row of each MD_LIST_* kind        */
} md_observables_t;

/*
 * Reduce the observables of the current state into *out (host).  The virial
 * is that of the last force evaluation made with MD_FORCE_VIRIAL (md_forces)
 * -- call md_forces(sys, MD_LEVEL_ALL, MD_FORCE_VIRIAL) first for a current
 * pressure.  Synchronises the stream.
 */
int md_observables(md_system *sys, md_observables_t *out);

/*
 * Flow profile across the channel (Sec. 4.2, Fig. 4): nbins equal slabs of y
 * in [0, Ly) (positions below 0 or above Ly count in the edge slabs); HOST
 * out[2*nbins] = mean v_x of the plasma particles of each slab (out[b], 0 for
 * an empty slab), then their number density (out[nbins + b], particles per
 * unit volume).  FP64 sums on the device; velocities as stored (synchronised
 * after md_mts_step).  Errors: MD_EINVAL (nbins outside [1, 256]), MD_ECUDA.
 */
int md_flow_profile(md_system *sys, int32_t nbins, double *out);

/*
 * Per-platelet measurements of the current state (the time series the
 * controller reads, Sec. 3.3 / Table 1 "compute and dump platelet physical
 * properties"), reduced in FP64 on the device, written to HOST
 * out[n_platelets][12]:
 *   0-2 centre-of-mass velocity; 3-5 angular velocity I^-1 L about the
 *   centre of mass; 6-8 principal values (ascending) of the force-moment
 *   stress -1/2 sum (r F^T + F r^T); 9 largest bond strain |r - r0|/r0;
 *   10 receptor contacts with other platelets closer than 1.5 morse_r0;
 *   11 mean speed of the plasma within 2 of the centre of mass.
 * Errors: MD_EINVAL (no platelets), MD_ECUDA.
 */
int md_platelet_features(md_system *sys, double *out);

/*
 * Append the current measurements to the device ring of the last 128
 * records per platelet (no host copy), and read that ring back: HOST
 * out[n_platelets][128][12], oldest retained record first (out = NULL: only
 * the count); *count gets the number of records appended so far (records
 * beyond 128 overwrite the oldest).
 */
int md_record_features(md_system *sys);
int md_read_feature_ring(md_system *sys, float *out, int64_t *count);

/*
 * Neighbour pairs of list kind `kind` as particle ids (a < b), written to
 * HOST pairs[2*cap]; *count gets the total (pairs = NULL: the count alone,
 * from the row counts).  For parity checks of K2.  Synchronises the stream.
 */
int md_neighbor_pairs(md_system *sys, int32_t kind, int32_t *pairs, int64_t cap, int64_t *count);

/* ---- learned step-size controller (Sec. 3.3, Table 2) --------------------- */
/*
 * Inference pipeline of Table 2 on the device: raw windows [B][T][F] of the
 * per-platelet measurements -> denoise (causal moving average over 5 steps,
 * one-level Haar transform with the soft threshold median|d|/0.6745 *
 * sqrt(2 ln T), inverse) -> per-feature normalisation -> GRU autoencoder
 * (2-layer encoder, hidden 64; latent = linear map of the last hidden state;
 * 2-layer decoder fed the repeated latent; linear read-out) -> two FCN heads
 * on the latent (ReLU hidden layers head_hidden[0..2]): logits over the step
 * ratios k in {1, 2, 5, 10, 20} and log of the hold length.
 * GRU cell: r = s(W_ir x + b_ir + W_hr h + b_hr), z = s(W_iz x + b_iz + W_hz h
 * + b_hz), n = tanh(W_in x + b_in + r (W_hn h + b_hn)), h' = (1-z) n + z h.
 * Matrix products run on the tensor cores in BF16 with FP32 accumulation;
 * parameters, activations and optimiser state are FP32.
 *
 * Flat FP32 parameter layout (md_ai_param_count entries), in order:
 *   enc1 {W_ih[3H][F], W_hh[3H][H], b_ih[3H], b_hh[3H]}, enc2 {W_ih[3H][H], ...},
 *   lat {W[L][H], b[L]}, dec1 {W_ih[3H][L], ...}, dec2 {W_ih[3H][H], ...},
 *   out {W[F][H], b[F]}, k-head {W0[h0][L], b0, W1[h1][h0], b1, W2[h2][h1], b2,
 *   W3[C][h2], b3}, hold head {same with 1 output}.
 */
#define MD_AI_HOST   0   /* argument arrays live in host memory   */
#define MD_AI_DEVICE 1   /* ... in device memory                  */
#define MD_AI_TRAIN_AE    1
#define MD_AI_TRAIN_HEADS 2

typedef struct md_ai_config {
    int32_t T;              /* window length (even, <= 256)              */
    int32_t F;              /* measurements per step                     */
    int32_t hidden;         /* GRU hidden size (64)                      */
    int32_t latent;         /* latent size                               */
    int32_t n_classes;      /* step-ratio classes                        */
    int32_t head_hidden[3]; /* FCN hidden widths                         */
    int32_t batch_max;      /* largest batch of windows                  */
} md_ai_config;

typedef struct md_ai md_ai;

int md_ai_config_defaults(md_ai_config *cfg);          /* T 128, F 12, H 64, L 16, C 5, (32,16,8), B 256 */
int md_ai_param_count(const md_ai_config *cfg, int64_t *n);
int md_ai_workspace_size(const md_ai_config *cfg, size_t *bytes);
/* Create over a caller-owned device workspace (>= md_ai_workspace_size). */
int md_ai_init(const md_ai_config *cfg, void *workspace, size_t bytes, void *cuda_stream, md_ai **out);
void md_ai_destroy(md_ai *ai);
const char *md_ai_last_error(const md_ai *ai);
/* Parameters (HOST, flat layout above); setting them resets the Adam state. */
int md_ai_set_params(md_ai *ai, const float *params, int64_t n);
int md_ai_get_params(md_ai *ai, float *params, int64_t n);
/* Per-feature normalisation applied after denoising (HOST mean[F], std[F]). */
int md_ai_set_norm(md_ai *ai, const float *mean, const float *stdv);
/*
 * Table 2 steps 1-4 for B raw windows (raw in host or device memory per
 * `where`): out (HOST) [B][C + 2] = class probabilities, predicted log hold,
 * reconstruction error (mean square over the window).  Errors: MD_EINVAL,
 * MD_ENOTRAINED (no parameters), MD_ECUDA.
 */
int md_ai_predict(md_ai *ai, const float *raw, int32_t B, int32_t where, float *out);
/*
 * Table 2 steps 1-2 only: raw windows (host or device per `where`) ->
 * denoised, normalised HOST windows out[B][T][F], the input of md_ai_encode,
 * md_ai_grads and md_ai_train_step (no parameters needed; the identity
 * normalisation until md_ai_set_norm).  Errors: MD_EINVAL, MD_ECUDA.
 */
int md_ai_prepare(md_ai *ai, const float *raw, int32_t B, int32_t where, float *out);
/*
 * Autoencoder on already denoised, normalised HOST windows x[B][T][F]:
 * latent (HOST [B][L], may be NULL) and reconstruction (HOST, time-major
 * [T][B][F], may be NULL).
 */
int md_ai_encode(md_ai *ai, const float *x, int32_t B, float *latent, float *recon);
/*
 * Loss and gradient (HOST grads[n_params], may be NULL; flat layout) on a
 * batch of denoised, normalised HOST windows: what = MD_AI_TRAIN_AE
 * (reconstruction MSE over B*T*F; head gradients are zero) or
 * MD_AI_TRAIN_HEADS (mean over the batch of the softmax cross-entropy of
 * k_class[B] plus the squared error of log_hold[B]; autoencoder gradients are
 * zero).  md_ai_train_step also applies one Adam step (b1 0.9, b2 0.999,
 * eps 1e-8) with learning rate lr to that part.
 */
int md_ai_grads(md_ai *ai, const float *x, const int32_t *k_class, const float *log_hold, int32_t B, int32_t what,
                float *grads, float *loss);
int md_ai_train_step(md_ai *ai, const float *x, const int32_t *k_class, const float *log_hold, int32_t B,
                     int32_t what, float lr, float *loss);

/*
 * Table 2 steps 5-6 on the device: the trust bound and the step-ratio map.
 * A window whose top class probability is below p_min, whose reconstruction
 * error (mean square over the denoised, normalised window) is above rec_max,
 * or whose raw measurement column strain_col (the largest bond strain; -1:
 * no strain test) exceeds strain_max at any step is "unsure" and gets
 * fallback_k (fixed-k RESPA); every other window gets the ratio of its most
 * probable class.  The hold length is exp(predicted log hold) clipped to
 * [hold_min, hold_max] steps, truncated to an integer.  NaN fails every test.
 */
typedef struct md_ai_trust {
    float   p_min;        /* smallest accepted top class probability         */
    float   rec_max;      /* largest accepted reconstruction error           */
    float   strain_max;   /* largest accepted value of column strain_col     */
    int32_t strain_col;   /* raw-window column of the bond strain, -1: none  */
    int32_t fallback_k;   /* ratio of an unsure window                       */
    float   hold_min, hold_max;
} md_ai_trust;

#define MD_AI_UNSURE_PROB   1   /* reason bits of an unsure window */
#define MD_AI_UNSURE_REC    2
#define MD_AI_UNSURE_STRAIN 4

/*
 * Table 2 steps 1-6 for B raw windows [B][T][F] (host or device memory per
 * `where`): the md_ai_predict pipeline, then the trust bound and ratio map
 * above on the device.  k_values[n_classes] (HOST): the step ratio of each
 * class ({1, 2, 5, 10, 20}).  HOST outputs: k_out[B] ratio, hold_out[B] hold
 * length in steps (may be NULL), why_out[B] MD_AI_UNSURE_* bits, 0 for a
 * trusted window (may be NULL).  Errors: MD_EINVAL, MD_ENOTRAINED, MD_ECUDA.
 */
int md_ai_decide(md_ai *ai, const float *raw, int32_t B, int32_t where, const md_ai_trust *trust,
                 const int32_t *k_values, int32_t *k_out, int32_t *hold_out, int32_t *why_out);

/*
 * md_ai_decide on the system's own feature ring (md_record_features; Table 1
 * "compute and dump platelet physical properties"): the last T records of
 * every platelet are gathered in time order on the device and decided there,
 * one window per platelet (B = n_platelets), so that only the P decisions
 * cross to the host.  Drains the system's stream first.  Errors: MD_EINVAL
 * (no platelets, fewer than T records, or a controller whose batch, window
 * or measurement count does not fit the system), MD_ENOTRAINED, MD_ECUDA.
 */
int md_ai_decide_system(md_ai *ai, md_system *sys, const md_ai_trust *trust, const int32_t *k_values,
                        int32_t *k_out, int32_t *hold_out, int32_t *why_out);

/* ---- the paper's own controller variant (Sec. 3.3) ------------------------ */
/*
 * The last T = 50 steps of F = 6 per-platelet measurements, denoised and
 * normalised as in md_ai_predict (Table 2 step 2), through a two-layer LSTM
 * autoencoder of H1 = 16 and H2 = 4 units; the latent is the second layer's
 * final hidden and cell state (2 H2 = 8 features); a mirrored decoder (LSTM
 * 2 H2 -> H2, LSTM H2 -> H1, linear H1 -> F at every step, fed the repeated
 * latent) reconstructs the window; a four-layer FCN (fcn[0..2] = 32, 16, 8
 * ReLU units, one linear output) gives log k, the ratio of the fluid step to
 * the platelet step (Table 2 step 4).
 * LSTM cell, gates stacked (i, f, g, o) along the rows of W_ih [4H][in] and
 * W_hh [4H][H]: i = s(W_ii x + b_ii + W_hi h + b_hi), f, o alike, g = tanh(..),
 * c' = f c + i g, h' = o tanh(c'); zero initial state.  FP32 throughout
 * (the layers are a few units wide).
 *
 * Flat FP32 parameter layout (md_lstm_param_count entries), in order:
 *   enc1 {W_ih[4 H1][F], W_hh[4 H1][H1], b_ih[4 H1], b_hh[4 H1]},
 *   enc2 {W_ih[4 H2][H1], W_hh[4 H2][H2], b_ih, b_hh},
 *   dec1 {W_ih[4 H2][2 H2], W_hh[4 H2][H2], b_ih, b_hh},
 *   dec2 {W_ih[4 H1][H2], W_hh[4 H1][H1], b_ih, b_hh}, out {W[F][H1], b[F]},
 *   fcn {W0[fcn0][2 H2], b0, W1[fcn1][fcn0], b1, W2[fcn2][fcn1], b2, W3[1][fcn2], b3}.
 */
typedef struct md_lstm_config {
    int32_t T, F;           /* window length (even, <= 256), measurements      */
    int32_t H1, H2;         /* LSTM widths (16, 4)                             */
    int32_t fcn[3];         /* FCN hidden widths (32, 16, 8)                   */
    int32_t batch_max;      /* largest batch of windows                        */
} md_lstm_config;

typedef struct md_lstm md_lstm;

int md_lstm_config_defaults(md_lstm_config *cfg);      /* T 50, F 6, H 16/4, FCN 32/16/8, B 256 */
int md_lstm_param_count(const md_lstm_config *cfg, int64_t *n);
int md_lstm_workspace_size(const md_lstm_config *cfg, size_t *bytes);
/* Create over a caller-owned device workspace (>= md_lstm_workspace_size). */
int md_lstm_init(const md_lstm_config *cfg, void *workspace, size_t bytes, void *cuda_stream, md_lstm **out);
void md_lstm_destroy(md_lstm *m);
const char *md_lstm_last_error(const md_lstm *m);
int md_lstm_set_params(md_lstm *m, const float *params, int64_t n);   /* HOST; resets Adam */
int md_lstm_get_params(md_lstm *m, float *params, int64_t n);
int md_lstm_set_norm(md_lstm *m, const float *mean, const float *stdv);
/* B raw windows [B][T][F] (host or device per `where`) -> HOST out[B][2]:
 * predicted log k, reconstruction error (mean square over the window). */
int md_lstm_predict(md_lstm *m, const float *raw, int32_t B, int32_t where, float *out);
/* Table 2 steps 1-2 only: raw windows -> denoised, normalised HOST out[B][T][F]. */
int md_lstm_prepare(md_lstm *m, const float *raw, int32_t B, int32_t where, float *out);
/*
 * Loss and gradient (HOST grads[n_params], may be NULL) on denoised,
 * normalised HOST windows x[B][T][F]: what = MD_AI_TRAIN_AE (reconstruction
 * MSE over B T F) or MD_AI_TRAIN_HEADS (mean squared error of the FCN's
 * log k against log_k[B]); the other part's gradient is zero.
 * md_lstm_train_step also takes one Adam step (b1 0.9, b2 0.999, eps 1e-8,
 * learning rate lr) on that part.  Errors: MD_EINVAL, MD_ENOTRAINED, MD_ECUDA.
 */
int md_lstm_grads(md_lstm *m, const float *x, const float *log_k, int32_t B, int32_t what, float *grads, float *loss);
int md_lstm_train_step(md_lstm *m, const float *x, const float *log_k, int32_t B, int32_t what, float lr,
                       float *loss);

/* ---- diagnostics ---------------------------------------------------------- */
#define MD_PROF_FLUID   0  /* K3 plasma-plasma / plasma-wall DPD pass          */
#define MD_PROF_IFACE   1  /* K3 interface DPD pass                            */
#define MD_PROF_PLT     2  /* K4 + K5 platelet forces                          */
#define MD_PROF_INTEG   3  /* K7 kick / drift / rebuild check                  */
#define MD_PROF_BUILD   4  /* K1 + K2 rebuild chain (gated: mostly empty)      */
#define MD_PROF_OTHER   5  /* time-index updates, reductions                   */
#define MD_PROF_CLASSES 6

typedef struct md_profile_t {
    int64_t launches[MD_PROF_CLASSES];  /* kernel launches per class          */
    double  ms[MD_PROF_CLASSES];        /* summed CUDA-event time per class   */
    int64_t total_launches;             /* every kernel libmsm launched       */
} md_profile_t;

/*
 * Kernel accounting: with enable = 1, md_mts_step brackets each kernel class
 * it launches with CUDA events on the system's stream (a small perturbation;
 * launch counting is always on).  md_profile_read synchronises, sums and
 * (reset = 1) clears the counters.  Errors: MD_EINVAL, MD_ECUDA.
 */
int md_profile_enable(md_system *sys, int enable);
int md_profile_read(md_system *sys, md_profile_t *out, int reset);

/*
 * Philox4x32-10 on the device, as used for the pair noise: out[4k..4k+3] =
 * Philox4x32-10(ctr[4k..4k+3], key) for k < n.  HOST arrays in and out.  With
 * use_library = 1 the same blocks come from cuRAND's device Philox4_32_10
 * generator (counter mapped to its subsequence/offset), for cross-checking.
 * Errors: MD_EINVAL (n < 0, or a counter the library mapping cannot reach),
 * MD_ECUDA.
 */
int md_philox(const uint32_t *ctr, const uint32_t key[2], int64_t n, uint32_t *out, int use_library);

/*
 * md_philox without any allocation.  The paper has no counterpart: this is a
 * service entry point of the library, for callers that cannot allocate device
 * memory -- a process whose device memory is held by a caching pool
 * allocator (a cudaMalloc there fails or forces the pool to give memory
 * back), or a caller working beside other streams, for which cudaFree's
 * implicit device-wide synchronisation would stall the work in flight.
 * Same arguments, blocks and errors as md_philox; the device staging
 * buffers are a file-scope static __device__ array of 2 * MD_PHILOX_STATIC_MAX
 * uint4 (512 KiB, 256-byte aligned, part of the library's module image)
 * instead of cudaMalloc'd scratch.  No cudaMalloc, cudaFree or allocating
 * library routine is called.
 *  - n > MD_PHILOX_STATIC_MAX returns MD_ETOOLARGE before any CUDA call.
 *  - The array's device address is looked up (cudaGetSymbolAddress, which
 *    does not allocate) in the current context on every call, so a context
 *    rebuilt after a cudaDeviceReset is served like a new one.  The first
 *    call on a device may load the library's module: make it before any
 *    stream capture begins on that device.
 *  - The array keeps the last call's counters and outputs.  Nothing in it
 *    has to start at zero: a call copies its n counters in before the kernel
 *    reads them, and the kernel writes the n outputs before they are copied
 *    out.
 *  - Every call on a device shares the one array, so overlapping calls (from
 *    several host threads) race on it: the caller serialises them.
 * Runs on the legacy default stream with synchronous copies, as md_philox.
 */
#define MD_PHILOX_STATIC_MAX 16384
int md_philox_static(const uint32_t *ctr, const uint32_t key[2], int64_t n, uint32_t *out, int use_library);

/*
 * Checkpoint: md_get_state writes the full dynamical state (positions,
 * velocities, level forces, step counters, Lees-Edwards offset) in id order
 * to the HOST blob (pass blob = NULL to get the size in *n); md_set_state
 * restores it.  The counter-based noise makes a resumed run identical to an
 * uninterrupted one.
 */
int md_get_state(md_system *sys, void *blob, size_t *n);
int md_set_state(md_system *sys, const void *blob, size_t n);

#ifdef __cplusplus
}
#endif

#endif /* MSM_H */
