/*
 * pdq.h -- C ABI of libpdq, the GB300 (sm_103a) particle-deposition library.
 *
 * libpdq advances the Lagrangian particle phase of the high-fidelity model of
 * Yao, Huan & Capecelatro, "Multi-fidelity uncertainty quantification of
 * particle deposition in turbulent pipe flow" (App. A.2, Eq. newtonlaw with
 * the drag law Eq. part_source, the Coulomb force Eq. coulomb, the van der
 * Waals force Eq. vdw and the rebound model of Sec. 4.3) for many Monte Carlo
 * samples of the uncertain inputs (charge scale xi, Hamaker ratio zeta,
 * temperature theta; Secs. 2.1 and 4.3), tallies the deposition velocity
 * V_dep+ (Sec. 2.1), evaluates the 1-D Eulerian low-fidelity deposition
 * model of App. B for the same samples, and evaluates the multi-fidelity Monte
 * Carlo estimators of Sec. 3.  The carrier phase is a frozen synthetic pipe
 * field (log-law mean plus divergence-free random Fourier modes) standing in
 * for the paper's DNS.
 *
 * Conventions (every entry point):
 *   - Returns an int status: PDQ_OK (0) or a negative PDQ_ERR_* code.  No
 *     exception or abort crosses the ABI; pdq_strerror() names the code.
 *   - Device pointers are caller-owned CUDA global memory on the current
 *     device; host pointers are caller-owned host memory.  The library owns
 *     only the opaque pdq_field handle.
 *   - Work is enqueued on the caller's stream `stream` (a cudaStream_t; NULL
 *     is the legacy default stream) and returns without synchronising, unless
 *     stated otherwise.  Calls that read device values on the host say so.
 *   - Units are wall units (+): length nu/u*, velocity u*, time nu/u*^2.
 *   - Invalid sizes or NULL pointers return PDQ_ERR_INVALID_ARG before any
 *     work is enqueued; CUDA failures return PDQ_ERR_CUDA.
 */
#ifndef PDQ_H
#define PDQ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef void* pdq_stream_t; /* cudaStream_t */

/* ---------------------------------------------------------------- status */
enum {
    PDQ_OK = 0,
    PDQ_ERR_INVALID_ARG = -1, /* bad size, NULL pointer, unknown enum value        */
    PDQ_ERR_CUDA = -2,        /* a CUDA runtime call failed                        */
    PDQ_ERR_OOM = -3,         /* device allocation failed (pdq_field, pdq_p3m)      */
    PDQ_ERR_NAN = -4,         /* a kernel saw a non-finite particle state          */
    PDQ_ERR_TIMEOUT = -5,     /* a bounded device wait gave up                     */
    PDQ_ERR_PRECOND = -6,     /* MFMC precondition (Eq. mf-precond) violated       */
    PDQ_ERR_UNSUPPORTED = -7, /* valid request the library does not implement      */
    PDQ_ERR_WORKSPACE = -8    /* caller workspace smaller than required            */
};
const char* pdq_strerror(int status);
int pdq_version(void); /* major*10000 + minor*100 + patch */

/* ------------------------------------------------------ physical constants
 * Sec. 2.1: D = 20 mm, nu = 1.5e-5 m^2/s, Re_tau = 180, U_b = 4 m/s,
 * rho_p = 2650 kg/m^3, q_max = 500 e (d/1um)^2, A0 = 1e-18 J; Sec. 2.2:
 * eps0 = 8.854e-12 F/m, delta_min = 1e-9 m; Sec. 4.3: E = 70 GPa,
 * delta_c = 0.165 nm, sigma_y0 = 200 MPa.  rho_f (gas density) is not printed;
 * 1.2 kg/m^3 reproduces the printed tau_p+ of the three particle sizes.      */
typedef struct pdq_phys {
    double nu;        /* kinematic viscosity, m^2/s                 */
    double radius;    /* pipe radius D/2, m                         */
    double re_tau;    /* friction Reynolds number u* R / nu         */
    double u_bulk;    /* bulk velocity, m/s (capture efficiency)    */
    double rho_p;     /* particle material density, kg/m^3          */
    double rho_f;     /* gas density, kg/m^3                        */
    double eps0;      /* vacuum permittivity, F/m                   */
    double q_unit;    /* q_max / (d/1um)^2 = 500 e, C               */
    double hamaker0;  /* A0, J                                      */
    double delta_min; /* vdW saturation gap, m                      */
    double young;     /* Young's modulus E, Pa                      */
    double delta_c;   /* cohesion length delta_c, m                 */
    double sigma_y0;  /* yield stress at theta = 0, Pa              */
    double g;         /* gravitational acceleration, m/s^2          */
    double restitution;     /* soft-sphere collisions: coefficient of restitution e (0.9, App. A.2) */
    double tau_col_steps;   /* collision time tau_col in steps (15, App. A.2)                       */
    double neg_charge_frac; /* seeding: share of particles with a negative charge (0: like-signed,   */
                            /* as in the paper; the sign draws Philox counter word 2)               */
    double contact_scale;   /* Coulomb distance clamp d_c = contact_scale x the largest class       */
                            /* diameter (1 by default; > 0): a smaller value tests how much the     */
                            /* clamp matters (d_min/d_max puts it at the smallest class diameter)   */
} pdq_phys;
void pdq_phys_default(pdq_phys* out);

/* ------------------------------------------------- synthetic carrier field
 * Mean U+(y+) = y+ below the sublayer/log-law crossing, ln(y+)/kappa + B above
 * (the paper's DNS field is not available); fluctuation
 *   u' = curl( (1 - r^2/R^2)^2 sum_n b_n cos(k_n . x + phi_n) ),
 * divergence-free and zero at the wall, modes drawn from Philox4x32-10 with
 * key = seed: |k| log-uniform in [k_min, k_max], isotropic direction, k_z
 * rounded to the lattice 2 pi m / L, b_n perpendicular to k_n with
 * |b_n| = u_rms sqrt(6/n_modes) / |k_n|, phi_n uniform.  Stored at the nodes
 * r_i = R tanh(beta i/(n_r-1))/tanh(beta), theta_j = 2 pi j/n_th,
 * z_k = L k/n_z as Cartesian (u_x, u_y, u_z): FP64 and FP32 copies.          */
typedef struct pdq_field_desc {
    int32_t n_r, n_th, n_z; /* grid nodes in r (incl. axis and wall), theta, z: n_r >= 2, n_th >= 1, n_z >= 1 */
    int32_t n_modes;        /* random Fourier modes, 0..4096            */
    double r_plus;          /* pipe radius R+ (= Re_tau)                */
    double l_plus;          /* periodic length L+                      */
    double u_rms;           /* per-component rms of u' on the axis      */
    double beta;            /* radial stretching (> 0)                  */
    double kappa, b_log;    /* log-law constants                        */
    double k_min, k_max;    /* wavenumber shell, 0 < k_min <= k_max     */
} pdq_field_desc;

typedef struct pdq_field pdq_field; /* opaque, owns its device memory */

/* Build the field on the current device.  Allocates ~44 B per node plus the
 * mode table, launches the mode and grid kernels on `stream` and waits for
 * them.  *out receives the handle; destroy it with pdq_destroy_pipe_field.
 * Errors: INVALID_ARG (desc out of range), OOM, CUDA.                        */
int pdq_create_pipe_field(const pdq_field_desc* desc, uint64_t seed, pdq_stream_t stream, pdq_field** out);
int pdq_destroy_pipe_field(pdq_field* field);
/* Device views of the field: grid64 = double4 [n_z][n_th][n_r] (w unused),
 * grid32 = float4 [n_z][n_th][n_r], modes = double [n_modes][7]
 * (kx, ky, kz, bx, by, bz, phi).  Any output pointer may be NULL.            */
int pdq_field_views(const pdq_field* field, pdq_field_desc* desc, const void** grid64, const void** grid32,
                    const double** modes);
/* Copy the field into caller buffers (device or host; NULL skips a part):
 * grid64 = n_z*n_th*n_r*32 bytes, grid32 = n_z*n_th*n_r*16 bytes,
 * modes = n_modes*56 bytes.  Enqueued on `stream` (cudaMemcpyAsync,
 * direction inferred from the pointers).                                     */
int pdq_field_copy(const pdq_field* field, void* grid64, void* grid32, void* modes, pdq_stream_t stream);

/* ------------------------------------------------------------ particles */
#define PDQ_MAX_CLASSES 16
enum { PDQ_FP64 = 0, PDQ_MIXED = 1 };

/* Caller-owned particle state of S samples.  Sample s owns the slots
 * [offset[s], offset[s+1]); its first count[s] slots hold its particles
 * (live ones and those deposited since the last compaction).  Arrays marked
 * [2] are double-buffered: half `cur` holds the current state; a step writes
 * the other half and flips `cur`.  Element types by precision:
 *   pos[2]: FP64 double4 (x+, y+, z+, q_eff); MIXED float4 (x+, y+, z+, q_eff)
 *           where MIXED x+, y+ are FP32 copies of xy; q_eff = charge in units
 *           of q_unit (= xi (d/1um)^2 times the per-particle factor), 0 once
 *           deposited.
 *   vel[2]: FP64 double4 / MIXED float4 (vx+, vy+, vz+, alive: 1 or 0).
 *   xy[2] : MIXED only, double2 (x+, y+), the authoritative wall-normal
 *           position; NULL for FP64.
 *   tag   : int2 (particle id within its sample, size class), not
 *           double-buffered; compaction permutes it with the current half.
 *   ctl   : int64 [8] control block the library owns the contents of (step
 *           counter, work-queue counters, error word); zeroed by seeding.
 * All arrays need 32-byte alignment.                                         */
typedef struct pdq_state {
    int32_t precision;                    /* PDQ_FP64 or PDQ_MIXED                        */
    int32_t cur;                          /* 0 or 1, maintained by the library            */
    int32_t n_samples;                    /* S >= 1                                       */
    int32_t n_classes;                    /* C in 1..PDQ_MAX_CLASSES                      */
    double st_plus[PDQ_MAX_CLASSES];      /* Stokes number tau_p+ of each size class      */
    int64_t capacity;                     /* offset[S]                                    */
    int64_t step;                         /* global step index (host mirror)              */
    const int64_t* offset;                /* device [S+1], offset[0] = 0, non-decreasing  */
    int32_t* count;                       /* device [S]                                   */
    void* pos[2];
    void* vel[2];
    void* xy[2];
    int32_t* tag;
    int64_t* ctl;
} pdq_state;

/* Per-sample uncertain inputs (device array [S]): xi scales the charge
 * q = xi q_max (Sec. 2.1), zeta = A/A0 (Sec. 2.1), theta the yield-stress
 * drop sigma_y = sigma_y0 (1 - theta) (Sec. 4.3).                            */
typedef struct pdq_sample_params {
    double xi, zeta, theta, pad;
} pdq_sample_params;

/* Seed every sample (Sec. 2.1: particles at rest, uniformly distributed in
 * the pipe, q = xi q_max): local particle j uses Philox4x32-10 counter
 * (j, 0, 0, 0), key = seed, for (r, theta, z) = ((R - d/2) sqrt(u0), 2 pi u1,
 * L u2) with u = (word + 1/2) 2^-32, and counter (j, 1, 0, 0) for the
 * lognormal charge factor exp(sigma sqrt(-2 ln u0) cos(2 pi u1)) when
 * charge_sigma > 0.  Class = j mod C, so all samples share their first
 * particles (common random numbers).  Writes half 0 of every array, sets
 * count[s] = offset[s+1] - offset[s], cur = 0, step = 0, zeroes ctl.
 * Errors: INVALID_ARG (precision, classes, NULL arrays), CUDA.               */
int pdq_seed_particles(const pdq_field* field, const pdq_phys* phys, double charge_sigma, uint64_t seed,
                       const pdq_sample_params* params, pdq_state* state, pdq_stream_t stream);

/* pdq_seed_particles with a random stream per sample: sample s draws with
 * counter word 3 = s + 1, i.e. counters (j, 0, 0, s+1), (j, 1, 0, s+1) and
 * (j, 2, 0, s+1), so its particles are independent of the other samples'
 * (the common-random-numbers default uses word 3 = 0).  For studies that
 * need many distinct trajectories, such as validating V_dep+ statistics,
 * rather than the paired comparisons common random numbers serve.        */
int pdq_seed_particles_independent(const pdq_field* field, const pdq_phys* phys, double charge_sigma, uint64_t seed,
                                   const pdq_sample_params* params, pdq_state* state, pdq_stream_t stream);

/* ------------------------------------------------------------------ step */
enum { PDQ_STICK = 0, PDQ_REBOUND = 1 };
/* PDQ_F_ALL: the forces of the batched model (drag, gravity, Coulomb, image
 * charge, wall vdW).  PDQ_F_COLLIDE / PDQ_F_VDW_PP add particle-particle
 * contact (App. A.2 collision force and Eq. vdw between particles):
 *  - collisions: linear spring-dashpot along the line of centres while the
 *    spheres overlap, K = (pi^2 + ln^2 e)/tau_col^2, H = -2 ln e / tau_col per
 *    unit effective mass, so a contact lasts tau_col = tau_col_steps dt and
 *    returns e times the approach speed; normal direction only;
 *  - vdW: Eq. vdw with the effective diameter 2 d_i d_j / (d_i + d_j), gap
 *    saturated at delta_min (also while overlapping), zero beyond a quarter of
 *    that diameter, Hamaker constant zeta A0;
 *  - both are evaluated at the mid-step predicted positions x + v dt/2.
 * Contact runs use 4 particles per thread (MIXED), no FP64 j-split, and ignore
 * cfg->variant; pdq_adjoint_run rejects them.                                */
enum { PDQ_F_DRAG = 1, PDQ_F_GRAVITY = 2, PDQ_F_COULOMB = 4, PDQ_F_IMAGE = 8, PDQ_F_VDW = 16, PDQ_F_ALL = 31,
       PDQ_F_COLLIDE = 32, PDQ_F_VDW_PP = 64, PDQ_F_CONTACT = 96 };

typedef struct pdq_step_cfg {
    double dt;            /* time step dt+ > 0                                              */
    double gravity[3];    /* direction of gravity (scaled by g nu/u*^3); zero = none        */
    int32_t mode;         /* PDQ_STICK (removal on wall contact, App. A) or PDQ_REBOUND      */
    int32_t forces;       /* PDQ_F_* mask                                                    */
    int64_t window_start; /* first global step index counted in the tallies (t+ >= t_w)      */
    int32_t compact_every;/* compact deposited particles out every this many steps (done     */
                          /* with the z-binning pass, so at least every 10 steps); 0 never   */
    int32_t block;        /* threads per CTA of the step kernel: 0 (auto), 64, 128, 256      */
                          /* (and 32 for PDQ_FP64)                                           */
    int32_t use_graph;    /* 1: capture the call as a CUDA graph (first call with a given      */
                          /*    argument set) and replay it afterwards; needs a created        */
                          /*    (non-default) stream; see pdq_release_graphs.                  */
                          /* 2: capture and instantiate that graph without running it: the    */
                          /*    state, tallies and host fields are left as they were, and a    */
                          /*    later call with use_graph = 1 and the same arguments replays it */
    int32_t variant;      /* MIXED pair math: 0 packed f32x2 (4 particles per thread),      */
                          /* 1 packed with scalar sums, 2 packed with 8 particles per thread, */
                          /* 3 Newton pairs: each pair evaluated once for both particles     */
                          /*   (Eq. coulomb is odd in x_i - x_j), summed through atomics     */
                          /*   (float for MIXED, double for PDQ_FP64; not bit-reproducible   */
                          /*   from run to run), then the local update; block 64 or 128      */
                          /*   only.  MIXED contact runs take the Coulomb sums this way and  */
                          /*   keep the contact forces one-sided; PDQ_FP64 contact runs      */
                          /*   ignore it.  For PDQ_FP64 the only other value read is 0       */
} pdq_step_cfg;

/* Caller-owned tallies, device int64 [S][C], accumulated across calls:
 * n_dep = particles deposited during counted steps, n_alive = sum over counted
 * steps of the particles alive at the start of the step.                     */
typedef struct pdq_tally {
    int64_t* n_dep;
    int64_t* n_alive;
} pdq_tally;

/* Workspace bytes pdq_step_particles needs for this state and configuration
 * (the work-item table; MIXED: the z-binning sort's scratch; pair variant 3:
 * 16 B (MIXED) or 24 B (PDQ_FP64) x capacity of sums; PDQ_FP64 with few
 * i-tiles, one-sided: per-chunk partial pair sums, 24 B x particles x chunks,
 * chunks <= 64, chosen from the capacity, the tile and the device's SM
 * count).                                                                    */
int pdq_step_workspace_size(const pdq_state* state, const pdq_step_cfg* cfg, size_t* bytes);

/* Advance all samples n_steps steps (App. A.2).  One step of particle i:
 *   a_i = sum_{j != i, same sample} k q_i q_j (x_i - x_j) / (m_i max(|x_i - x_j|, d_c)^3)
 *         (Eq. coulomb; minimum image in z; d_c = phys->contact_scale x the largest
 *         class diameter)
 *       + image charge q_i^2 / (4 pi eps0 (2 y)^2 m_i) toward the wall (Sec. 2.2)
 *       + 2 F_vw(delta)/m_i toward the wall (Eq. vdw; delta saturated at
 *         delta_min, zero beyond d/4)  + gravity;
 *   u = trilinear interpolation of the field in (s(r), theta, z);
 *   drag (f / tau_p+)(u - v), f = 1 + 0.15 Re_p^0.687 (Eq. part_source);
 *   exponential integrator with u, f, a frozen over the step;
 *   wall contact when R - r - d/2 <= 0: STICK removes the particle,
 *   REBOUND applies CoR_n of Sec. 4.3 (sticking when it is 0).
 * FP64 runs everything in double; MIXED keeps x, y, the wall gap, the vdW
 * term and the tallies in double and runs the pair sum, interpolation, drag
 * and velocities in float.  `workspace` (>= pdq_step_workspace_size bytes,
 * device, 256-byte aligned) holds the work queue.  The particles of each
 * sample are grouped by z (a stable binning; `tag` moves with them, so
 * identify particles by tag, not by row) at the start of the call and every
 * min(compact_every, 10) steps (every 10 when compact_every = 0); when
 * compact_every > 0 the same pass compacts deposited particles out, updating
 * count[].  All work is enqueued on `stream`; the call does not wait for it
 * (except graph mode's first call for an argument set, which instantiates a
 * graph).
 * Errors: INVALID_ARG, WORKSPACE, CUDA.  Non-finite states set the error word
 * read by pdq_check_state.                                                   */
int pdq_step_particles(const pdq_field* field, const pdq_phys* phys, pdq_state* state,
                       const pdq_sample_params* params, const pdq_step_cfg* cfg, int64_t n_steps,
                       pdq_tally* tally, void* workspace, size_t workspace_bytes, pdq_stream_t stream);

/* Built-in scratch size of pdq_step_particles_noalloc, bytes. */
#define PDQ_NOALLOC_SCRATCH_BYTES (1u << 20)

/* pdq_step_particles for callers that cannot allocate device memory: for
 * example a host program whose device memory is owned by another allocator or
 * held under a hard cap, or a latency-critical loop that must not call
 * cudaMalloc (which can synchronise the device).  The paper has no
 * counterpart; this is a deployment variant of the step above, with the same
 * arguments and results except that the work queue lives in a 1 MiB array
 * compiled into libpdq (PDQ_NOALLOC_SCRATCH_BYTES), which every GPU that
 * loads the library keeps until the process exits.  The call allocates
 * nothing (no cudaMalloc, cudaFree or allocating library routine).
 * Limits: the step's whole workspace must fit the scratch, else the call
 * returns PDQ_ERR_WORKSPACE before any device work.  It holds the work-item
 * table (8 B per (sample, i-tile) item, times the j-chunks of FP64 runs), 4 B
 * per sample, the z-binning sort's tag scratch (8 B per slot of capacity),
 * with pair variant 3 the Newton-pair sums (16 B per slot MIXED, 24 B FP64),
 * and for FP64 one-sided runs whose few i-tiles are split over JS > 1
 * j-chunks (JS <= 64) partial sums of 24 JS B per slot.  Approximate largest
 * capacity: MIXED pair variants 0-2 130,000 slots, variant 3 43,000; FP64
 * variant 3 30,000; FP64 one-sided 9,900, and again from 32,768 to 128,000
 * (above 32,768 slots JS = 1).  pdq_step_workspace_size() <=
 * PDQ_NOALLOC_SCRATCH_BYTES is a sufficient test (it sizes the item table
 * for the narrower tile the P3M driver also uses); the call itself checks
 * the exact need.  cfg->use_graph must be 0 (PDQ_ERR_INVALID_ARG otherwise).
 * Set-up: the first call on each device resolves the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.
 * Sharing: all calls share the one array and it keeps the last call's
 * contents; each call rebuilds the work queue and zeroes the sums before
 * using them, so nothing needs clearing, but calls whose GPU work overlaps
 * (different streams, or host threads, without ordering between them) race
 * on it.                                                                    */
int pdq_step_particles_noalloc(const pdq_field* field, const pdq_phys* phys, pdq_state* state,
                               const pdq_sample_params* params, const pdq_step_cfg* cfg, int64_t n_steps,
                               pdq_tally* tally, pdq_stream_t stream);

/* Autotuner: times one step of each candidate tile shape (threads per CTA 64,
 * 128, 256, and 32 for PDQ_FP64) and, for PDQ_MIXED, each pair-math variant
 * on this state, and
 * writes the fastest into cfg->block / cfg->variant.  The timed steps write
 * the scratch half and a scratch tally; the current half, state->cur,
 * state->step and the device step counter are restored.  With PDQ_MIXED and
 * cfg->compact_every > 0 the state is z-binned first (live particles
 * reordered and compacted, as pdq_step_particles does at the start of a call).
 * Results are cached per (precision, log2 capacity, log2 samples, forces);
 * a cached entry costs no device work.  Synchronises `stream`.
 * Errors: INVALID_ARG, WORKSPACE, CUDA.                                      */
int pdq_autotune_workspace_size(const pdq_state* state, size_t* bytes);
int pdq_autotune(const pdq_field* field, const pdq_phys* phys, pdq_state* state, const pdq_sample_params* params,
                 pdq_step_cfg* cfg, void* workspace, size_t workspace_bytes, pdq_stream_t stream);

/* Destroy every cached step graph (use_graph = 1).  A cached graph bakes in
 * the device pointers of its call: release the graphs before freeing or
 * reusing those buffers for another purpose.                                 */
int pdq_release_graphs(void);

/* Stream compaction of deposited particles (alive == 0) of every sample, in
 * place and order-preserving on the current half; updates count[].          */
int pdq_compact(pdq_state* state, pdq_stream_t stream);

/* Synchronise `stream` and read the device error word: PDQ_OK, PDQ_ERR_NAN
 * (a non-finite state appeared) or PDQ_ERR_TIMEOUT.  Clears the word.        */
int pdq_check_state(pdq_state* state, pdq_stream_t stream);

/* ---------------------------------------------------------- deposition
 * V_dep+ = (R+/2) n_dep / (dt+ n_alive) per (sample, class): the definition
 * J_w / (rho_pm u*) of Sec. 2.1 with J_w = (dN_dep/dt) m_p / (2 pi R L) and
 * rho_pm = N m_p / (pi R^2 L), N integrated over the counted window.  Also
 * the Monte Carlo mean over samples and its standard error
 * sd / sqrt(S) per class (sd with divisor S-1; 0 when S = 1).  Outputs are
 * device arrays: vdep [S][C], mean [C], se [C] (mean/se may be NULL).       */
int pdq_deposition_tally(const pdq_tally* tally, int32_t n_samples, int32_t n_classes, double dt,
                         double r_plus, double* vdep, double* mean, double* se, pdq_stream_t stream);

/* Capture efficiency (Sec. 4.3): ce[k] = (4 L / D) (u* / U_b) vdep[k] for n
 * device values, L = the field's periodic length, D = 2R, u* = Re_tau nu / R,
 * U_b = phys->u_bulk.  With rebound-mode tallies (only sticking particles
 * counted) vdep is V_dep+|stick and ce the capture efficiency; under all-stick
 * it is the upper bound the paper states.  Errors: INVALID_ARG, CUDA.        */
int pdq_capture_efficiency(const pdq_field* field, const pdq_phys* phys, const double* vdep, int64_t n, double* ce,
                           pdq_stream_t stream);

/* ---------------------------------------------------------------- adjoint
 * Batch description for the adjoint's workspace layout and for its
 * self-seeding form: offset is a device array [S+1] as in pdq_state; st_plus
 * the class Stokes numbers.                                                  */
typedef struct pdq_batch {
    int32_t precision;                 /* PDQ_FP64 or PDQ_MIXED             */
    int32_t n_samples;                 /* S >= 1                            */
    int32_t n_classes;                 /* 1..PDQ_MAX_CLASSES                */
    int32_t pad;
    double st_plus[PDQ_MAX_CLASSES];
    int64_t capacity;                  /* offset[S]                         */
    const int64_t* offset;             /* device [S+1]                      */
} pdq_batch;

/* Workspace bytes of the adjoint: FP64 storage of 8 arrays per particle
 * and 2 int32 ones per checkpoint (ceil(n_steps/K) of them: the state
 * z-binned, its charges, classes and binning permutation), 10 per step of one
 * segment (K + 1 levels), 19 for cotangents and charges, 16 B per particle of
 * float sums (the MIXED Newton-pair kernels), plus 4 [S][C] tallies.  The
 * layout depends only on (capacity, S, C, n_steps, K).
 * pdq_adjoint_state_workspace_size sizes it for a pdq_state (its batch is
 * {precision, S, C, st_plus, capacity, offset} of the state).                */
int pdq_adjoint_workspace_size(const pdq_batch* batch, int64_t n_steps, int32_t K, size_t* bytes);
int pdq_adjoint_state_workspace_size(const pdq_state* init, int64_t n_steps, int32_t K, size_t* bytes);

/* Extra workspace bytes that let PDQ_MIXED adjoints with Coulomb forces keep
 * the forward sweep's Newton-pair sums (App. A.2 Coulomb sum, one float4 per
 * particle per step: 16 B x capacity x n_steps, plus a 256-byte marker).
 * When the workspace passed to pdq_adjoint_run(_seeded) holds at least the
 * layout size plus these bytes, the forward sweep accumulates each step's sums
 * in this region and the reverse sweep's recompute of each segment reuses them
 * instead of summing the pairs again (the recomputed states then equal the
 * forward sweep's exactly); J and pbar are the same functional and gradient.
 * pdq_adjoint_reverse decides the same way from its workspace_bytes, so pass
 * it the size the forward call had; with the extra bytes it returns
 * INVALID_ARG unless the region holds the sums of a forward sweep with the
 * same n_steps, K and capacity.  FP64 or Coulomb-free runs ignore the region.
 * Errors: INVALID_ARG (capacity < 0, n_steps < 1, bytes NULL).              */
int pdq_adjoint_stored_sums_size(int64_t capacity, int64_t n_steps, size_t* bytes);

/* Smoothed deposition functional and its hand-written reverse-mode adjoint,
 * starting from the caller's particle state `init` (e.g. one that
 * pdq_step_particles has advanced through a transient).
 * Forward (App. A.2 step of pdq_step_particles) with the wall removal
 * replaced by a weight update w' = w (1 - sigma(-gap'/eps)),
 * sigma(a) = 1/(1+e^-a), gap' = R - r' - d/2, and the Coulomb sum taken over
 * weighted charges w_j q_j; per (sample, class) over the counted steps
 * J = (R+/2) sum_n sum_p (w_n - w_{n+1}) / (dt+ sum_n sum_p w_n), which tends
 * to V_dep+ (Sec. 2.1) as eps -> 0.
 * Initial state: init's current half.  Particle p of sample s starts with its
 * position, velocity, class (tag), weight w = its alive flag (0 for a particle
 * deposited but not yet compacted out) and charge q = xi_s qhat_p with
 * qhat_p = q_eff / xi_s, so xi_s must be non-zero and finite for every sample
 * (params is read to the host to check this).  Slots [count[s], offset[s+1])
 * become weightless, uncharged particles at rest on the axis.  The adjoint
 * runs in init->precision; init is not modified.  Steps are numbered from 0
 * at the start of this call: cfg->window_start counts from there.
 * Reverse: checkpoints every K steps; each of the n_vec cotangent vectors
 * gbar[v] (device [S][C]) gives pbar[v] (device [S][3]) = sum_c gbar[v][s][c]
 * dJ[s][c]/d(xi_s, zeta_s, theta_s).  Under PDQ_STICK theta does not enter
 * and its component is exactly 0.  With cfg->mode = PDQ_REBOUND (Sec. 4.3) the
 * weight loss is multiplied by the smoothed sticking probability
 * sigma(-arg/eps_stick), arg = sigma_y0^2 (1-theta)^2/(rho_p E)
 * - 2 A_cont gamma_c/m (m^2/s^2; eps_stick > 0 required), and the rest of the
 * particle rebounds with CoR_n (0 when arg <= 0, capped at 1), mirrored into
 * the pipe.  J (device [S][C]) is always written; n_vec = 0 runs the forward
 * sweep alone and leaves its checkpoints in the workspace for
 * pdq_adjoint_reverse.  Reads offset[] to the host (synchronises `stream`).
 * PDQ_MIXED with Coulomb forces evaluates each particle pair once for both
 * particles (float sums through atomics, so not bit-reproducible from run to
 * run) and takes at most 33,553,920 particles per sample.  Contact forces
 * (PDQ_F_CONTACT) are not differentiated: cfg->forces must lie in PDQ_F_ALL.
 * workspace: device, 256-byte aligned, >= pdq_adjoint_state_workspace_size
 * (plus pdq_adjoint_stored_sums_size to keep the forward sweep's pair sums).
 * Errors: INVALID_ARG, WORKSPACE, UNSUPPORTED (sample too large), CUDA.     */
int pdq_adjoint_run(const pdq_field* field, const pdq_phys* phys, const pdq_state* init,
                    const pdq_sample_params* params, const pdq_step_cfg* cfg, int64_t n_steps, int32_t K,
                    double eps, double eps_stick, int32_t n_vec, const double* gbar, double* J, double* pbar,
                    void* workspace, size_t workspace_bytes, pdq_stream_t stream);

/* pdq_adjoint_run on particles it seeds itself, as
 * pdq_seed_particles(seed, charge_sigma) would (common random numbers), in
 * batch->precision: the same functional, sweeps, outputs and errors.        */
int pdq_adjoint_run_seeded(const pdq_field* field, const pdq_phys* phys, const pdq_batch* batch,
                           const pdq_sample_params* params, double charge_sigma, uint64_t seed,
                           const pdq_step_cfg* cfg, int64_t n_steps, int32_t K, double eps, double eps_stick,
                           int32_t n_vec, const double* gbar, double* J, double* pbar, void* workspace,
                           size_t workspace_bytes, pdq_stream_t stream);

/* The reverse sweeps alone (n_vec >= 1 cotangent vectors), on the forward
 * sweep that an earlier pdq_adjoint_run or pdq_adjoint_run_seeded call left in
 * `workspace`: pass the same batch layout (for pdq_adjoint_run, the state's:
 * see pdq_adjoint_state_workspace_size), params, cfg, n_steps, K, eps and
 * eps_stick, and the workspace unchanged since.  pbar as above.  Lets a
 * caller (the autograd function of the binding) take J first and gradients
 * later without a second forward sweep.
 * Errors: INVALID_ARG, WORKSPACE, UNSUPPORTED, CUDA.                         */
int pdq_adjoint_reverse(const pdq_field* field, const pdq_phys* phys, const pdq_batch* batch,
                        const pdq_sample_params* params, const pdq_step_cfg* cfg, int64_t n_steps, int32_t K,
                        double eps, double eps_stick, int32_t n_vec, const double* gbar, double* pbar,
                        void* workspace, size_t workspace_bytes, pdq_stream_t stream);

/* ---------------------------------------------------- multi-fidelity MC
 * Optimal MFMC allocation (Sec. 3.2, Eqs. opt1-opt3 and mf-precond) for k
 * models sorted by decreasing correlation with model 1 (host arrays [k]:
 * rho[0] = 1, sigma > 0, unit costs w > 0).  budget = p; with d_inputs > 0 the
 * Sobol' effective budget p/(d+2) of Sec. 4 is used.  rho_{1,k+1} is read as 0.
 * Outputs (host): m_out = floor(m_i*) made non-decreasing, alpha_out
 * (alpha_1 = 1), optional m_real_out = m_i*, optional gamma_out = MSE of the
 * MFMC mean over the MSE of plain MC at the same budget (equals
 * (sqrt(1 - rho^2) + rho sqrt(w2/w1))^2 for k = 2, Sec. 4.1).
 * Errors: INVALID_ARG, PRECOND (precondition violated or rho not decreasing).
 * Host-only; touches no device.                                              */
int pdq_mfmc_allocate(int32_t k, const double* rho, const double* sigma, const double* w, double budget,
                      int32_t d_inputs, int64_t* m_out, double* alpha_out, double* m_real_out, double* gamma_out);

/* Workspace bytes of pdq_mfmc_sobol: 8 (1 + n_boot) k 2 C (4 + 2d).          */
int pdq_mfmc_workspace_size(int32_t k, int32_t d, int32_t C, int32_t n_boot, size_t* bytes);

/* MFMC mean, variance and Sobol' main / total indices (Sec. 3.3: Owen's
 * main-effect and Jansen's total-effect estimators inside the control-variate
 * form of Eq. MFMC_mean, same alpha and m for all statistics; Var(Y) is the
 * MFMC variance estimate).  y[i] is a device array [n_i >= m_i][d+2][C] of
 * model i's pick-freeze groups: column 0 = f(x), 1 = f(x'), 2+j = f(z^(j))
 * with z^(j) = x' except input j taken from x; the first m_{i-1} groups of
 * every model are the samples shared with model i-1 (host arrays y[k],
 * m[k] (2 <= m_1 <= ... <= m_k < 2^32), alpha[k]).  1 <= d <= 16, C >= 1
 * outputs.  n_boot > 0 adds percentile bootstrap intervals (2.5 %, 97.5 %):
 * replicate b maps group position t in the nesting block [m_{l-1}, m_l)
 * (m_0 = 0) to m_{l-1} + ((philox(t, b, 0, 2).x * (m_l - m_{l-1})) >> 32)
 * (Philox4x32-10, key = seed); model i reads positions t < m_i, so it never
 * reads beyond its own m_i groups.
 * FP64 sums on the device (one deterministic CTA reduction per model,
 * prefix, output and replicate), assembly on the host.  Host outputs: mean[C],
 * var[C], s_main[d][C], s_total[d][C], s_main_ci / s_total_ci [d][C][2]
 * (may be NULL when n_boot = 0).  Synchronises `stream`.
 * Errors: INVALID_ARG, WORKSPACE, CUDA.                                      */
int pdq_mfmc_sobol(int32_t k, const double* const* y, const int64_t* m, const double* alpha, int32_t d, int32_t C,
                   int32_t n_boot, uint64_t seed, double* mean, double* var, double* s_main, double* s_total,
                   double* s_main_ci, double* s_total_ci, void* workspace, size_t workspace_bytes,
                   pdq_stream_t stream);

/* Derivative-based upper bounds on the total Sobol' indices (Sobol' and
 * Kucherenko, for inputs uniform on [a_j, b_j]):
 *   s_j^t <= (b_j - a_j)^2 nu_j / (pi^2 Var f),  nu_j = E[(df/dx_j)^2],
 * from S >= 2 Monte Carlo samples: grad device [S][C][d] (e.g. from
 * pdq_adjoint_run with one-hot cotangents), y device [S][C] the outputs,
 * width host [d] = b_j - a_j.  Host outputs nu [d][C], bound [d][C] (NaN
 * where Var f = 0).  FP64 fixed-order reductions on the device into the
 * caller's workspace (device, 8-byte aligned, >= pdq_dgsm_workspace_size =
 * 8 (d+1) C bytes); synchronises `stream`.
 * Errors: INVALID_ARG, WORKSPACE, CUDA.                                      */
int pdq_dgsm_workspace_size(int32_t C, int32_t d, size_t* bytes);
int pdq_dgsm_bounds(int32_t S, int32_t C, int32_t d, const double* grad, const double* y, const double* width,
                    double* nu, double* bound, void* workspace, size_t workspace_bytes, pdq_stream_t stream);

/* ------------------------------------ 1-D Eulerian low-fidelity model
 * The low-fidelity model of App. B (the unified advection-diffusion deposition
 * model with the kinetic wall condition, Eqs. momentum/mom_modified and
 * continuity, F_elec and F_vdw as printed), evaluated for every (sample, size
 * class) item, as model 2 of the multi-fidelity estimators (Sec. 3).  App. B
 * cites its closures without printing them; this library reads them as:
 *   v_f'^2(y)  the variance over (theta, z) of the carrier field's radial
 *              velocity at r = R - y (pdq_lf_fluid_variance), linear in the
 *              field's stretched radial coordinate between its nodes;
 *   R_ratio    T_L/(T_L + tau_p);  eps/nu = v_f'^2 T_L;  tau_1 = tau_p;
 *   D_B        k_B T tau_p / m_p;  D_T term 0 (isothermal gas);
 *   M_r        -V_w/(sqrt(2) sigma), sigma^2 = R_ratio v_f'^2 + k_B T/m_p at
 *              contact, i.e. the one-way flux of a Gaussian wall-normal
 *              velocity into an absorbing wall.
 * Charge q = xi q_max of the class, Hamaker constant A = zeta A0; theta does
 * not enter (the isothermal STICK model).  Grid: n_y nodes from contact
 * y = d/2 to the axis, y_k = d/2 + (R - d/2) expm1(gamma k/(n_y-1))/expm1(gamma);
 * the momentum equation in energy form with the drag implicit, marched from
 * V = 0 on the axis (V = 0 wherever the net force would drive particles away
 * from the wall); the continuity equation solved exactly on each cell with V
 * and D at their cell means.  The result converges at first order in the node
 * spacing (about 1 % at 2,048 nodes for St+ = 10).                           */
#define PDQ_LF_MAX_NODES 4096
typedef struct pdq_lf_desc {
    int32_t n_y;          /* wall-normal nodes, 3..PDQ_LF_MAX_NODES (default 2048)          */
    int32_t precision;    /* PDQ_FP64 (default): the march in FP64; PDQ_MIXED: the cell     */
                          /* table and the march in FP32 (Q summed with compensation), the  */
                          /* wall condition and the final ratio in FP64: within ~1e-5 of    */
                          /* the FP64 result, dozens of times faster on the FP32 pipe       */
    double stretch;       /* near-wall refinement gamma, 0 < gamma <= 700 (default 8)      */
    double t_lagr;        /* fluid Lagrangian integral time T_L+ > 0 (default 10)          */
    double temperature;   /* gas temperature, K > 0 (default 293.15)                       */
    double vdw_cutoff;    /* gap below which F_vdw is held constant, m > 0 (1e-12, App. B) */
} pdq_lf_desc;
void pdq_lf_desc_default(pdq_lf_desc* out);

/* v_f'^2 at the field's radial nodes r_i: var device [n_r] (caller-owned),
 * the population variance over the n_th x n_z nodes of u_r = cos(theta_j) u_x
 * + sin(theta_j) u_y of the FP64 grid (mean removed; fixed-order reductions,
 * deterministic).  Enqueued on `stream`.  Errors: INVALID_ARG, CUDA.          */
int pdq_lf_fluid_variance(const pdq_field* field, double* var, pdq_stream_t stream);

/* V_dep+ of the low-fidelity model for n_samples >= 0 samples and n_classes
 * size classes (host st_plus [C], 1 <= C <= 16): params device [S] (xi and
 * zeta used), var device [n_r] any v_f'^2 profile at `field`'s radial nodes
 * (normally pdq_lf_fluid_variance's), vdep device [S][C] (row = sample, the
 * deposition velocity over the centreline particle density; caller-owned).
 * One thread per item, 5 (n_y - 1) doubles (PDQ_MIXED: floats) of shared
 * memory per CTA of 256 samples.  Enqueued on `stream`; no allocation, no synchronisation.
 * Errors: INVALID_ARG (sizes, desc out of range, field radius != phys
 * Re_tau, NULL pointers), CUDA.                                              */
int pdq_lf_vdep(const pdq_field* field, const pdq_phys* phys, const pdq_lf_desc* lf, const double* var,
                int32_t n_classes, const double* st_plus, int64_t n_samples, const pdq_sample_params* params,
                double* vdep, pdq_stream_t stream);

/* ------------------------------------------------------------------ P3M
 * Electrostatics by P3M (App. A.2: the particle-particle particle-mesh method
 * the paper uses for ~1e6 particles per sample), for the periodic pipe:
 * periodic along z with period L, isolated across (no images through the
 * wall).  It approximates, for every live particle i of a sample,
 *   s_i = sum_j sum_k q_j d / max(|d|, d_c)^3,  d = x_i - x_j - k L e_z,
 * over all images k (the all-pairs path uses the nearest image only), d_c the
 * largest class diameter.  Splitting d/r^3 = K_L + K_S with the Gaussian
 * screening erf(alpha r)/r: K_L on a mesh of M cells across the diameter
 * (h = 2R/M; M + 5 nodes from -R - 2h, doubled to Nx = 2(M + 5) so that the
 * FFT convolution is the open one) and Nz nodes along z; charges assigned and
 * sums interpolated with TSC weights; the image-summed kernel's transform
 * divided by the squared TSC window; K_S = d/max(r, d_c)^3 - K_L summed
 * directly over pairs closer than r_cut via a cell list.  FP64 throughout;
 * cuFFT for the transforms.  With alpha h = 0.5 and r_cut = 3.3/alpha the
 * RMS relative error against the exact periodic sum is ~1.4e-4.
 * A plan owns its device memory (kernel transforms, meshes, cell list; about
 * 40 Nx^2 Nz bytes, plus a [capacity][3] FP64 buffer that
 * pdq_step_particles_p3m allocates the first time it meets a state that large).  Pick M with 2(M + 5) a product of small primes (123,
 * 251) for fast transforms.                                                  */
typedef struct pdq_p3m_desc {
    int32_t M;        /* mesh cells across the diameter, >= 4                          */
    int32_t Nz;       /* mesh nodes along the period L, >= 4                           */
    double alpha;     /* screening, 1/wall units; 0 = 0.5/h                             */
    double r_cut;     /* short-range cut-off, wall units, < L/2; 0 = 3.3/alpha          */
    int32_t n_img;    /* kernel images each way along z before the far-field tail; 0=200 */
    int32_t pad;
} pdq_p3m_desc;
typedef struct pdq_p3m pdq_p3m;

/* Build a plan for `field`'s pipe (R = r_plus, L = l_plus) and up to
 * max_particles particles per call (the largest sample).  Synchronises
 * `stream`.  Errors: INVALID_ARG, OOM, CUDA.                                 */
int pdq_p3m_create(const pdq_field* field, const pdq_p3m_desc* desc, int64_t max_particles, pdq_stream_t stream,
                   pdq_p3m** out);
int pdq_p3m_destroy(pdq_p3m* plan);
/* The effective alpha, r_cut, n_img and the transform size Nx of a plan.   */
int pdq_p3m_params(const pdq_p3m* plan, double* alpha, double* r_cut, int32_t* n_img, int32_t* nx);

/* P3M Coulomb sums of the current half of `state`: sums device [capacity][3]
 * (row g = particle g; zero for removed particles and unused rows), in the
 * units of the all-pairs sum (q in q_unit, lengths in wall units); the
 * acceleration is coul q_i s_i.  Samples are solved one after another on
 * `stream`; every sample must have <= max_particles particles.  Reads
 * count[] to the host (synchronises `stream`).
 * Errors: INVALID_ARG (state, plan, sizes), CUDA.                            */
int pdq_p3m_coulomb(pdq_p3m* plan, const pdq_phys* phys, const pdq_state* state, double* sums,
                    pdq_stream_t stream);

/* pdq_step_particles with the Coulomb acceleration from P3M: each step runs
 * pdq_p3m_coulomb on the current state, then the step kernel with those sums
 * in place of its all-pairs loop.  cfg as for pdq_step_particles except:
 * use_graph = 0, no contact forces (PDQ_F_CONTACT); compaction every
 * cfg->compact_every steps (unsorted).  workspace as sized by
 * pdq_step_workspace_size for (state, cfg).  Synchronises `stream` once per
 * step (sample sizes).  Errors: as pdq_step_particles and pdq_p3m_coulomb.   */
int pdq_step_particles_p3m(const pdq_field* field, const pdq_phys* phys, pdq_state* state,
                           const pdq_sample_params* params, const pdq_step_cfg* cfg, int64_t n_steps,
                           pdq_tally* tally, pdq_p3m* plan, void* workspace, size_t workspace_bytes,
                           pdq_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* PDQ_H */
