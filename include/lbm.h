/*
 * lbm.h - C ABI of the GB300 (sm_103a) lattice Boltzmann / DEM library for
 * slurries of spheres, after Mutabaruka & Kamrin, "A simulation technique for
 * slurries interacting with moving parts and deformable solids with
 * applications" (arXiv 1703.05158).
 *
 * One handle is one simulation on one GPU:
 *   - a D3Q19 lattice (Sect. 2.2, Table 1) of nx*ny*nz nodes, periodic in x
 *     and y, with plane walls at z = -1/2 and z = nz - 1/2 (halfway, i.e.
 *     link fraction q = 1/2) that may slide tangentially;
 *   - BGK collision (Eq. 12) towards the second-order equilibrium (Eq. 9)
 *     with the Smagorinsky relaxation time tau* = tau0 + tau_t (Eq. 18) and a
 *     body acceleration g (force density rho*g on fluid nodes);
 *   - spheres coupled to the fluid by interpolated bounce-back on cut links
 *     (Eqs. 19, 21), momentum-exchange force and torque (Eqs. 25, 26) and
 *     equilibrium refill of nodes a sphere uncovers;
 *   - a linear spring-dashpot normal contact (Eq. 1) between spheres and
 *     with the walls, integrated by velocity Verlet (Sect. 2.1) in
 *     dem_substeps sub-steps per lattice step.
 * Everything is in lattice units (Sect. 2.2): dx = dt = 1, fluid reference
 * density 1, c_s^2 = 1/3.
 *
 * Conventions
 *   Node index   n = x + nx*(y + ny*z).
 *   Populations  [19][N] with N = nx*ny*nz, direction order of Table 1.
 *   Vectors      per sphere, 3 consecutive doubles (x, y, z): array [n][3].
 *   where        LBM_HOST (any host memory) or LBM_DEVICE (device memory on
 *                the handle's device).  Output copies are complete when the
 *                call returns (the call synchronises the handle's stream).
 *   Ownership    the caller owns every buffer it passes; the library copies
 *                inputs during the call and keeps no caller pointer.
 *   Errors       0 on success, a negative LBM_ERR_* code otherwise.  Argument
 *                errors leave the state untouched.  Errors the device detects
 *                while stepping (capacity, divergence, a particle moving a
 *                quarter of a node or more in one step, a wait that ran
 *                out) are sticky: lbm_step returns at once and lbm_sync,
 *                lbm_forces, lbm_fields, ... report them until the handle
 *                is destroyed.
 *   Threads      a handle is not thread-safe; all its work goes to its
 *                stream in call order.
 */
#ifndef GB300_LBM_H
#define GB300_LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_s *lbm_handle;

/* Return codes. */
#define LBM_OK 0
#define LBM_ERR_ARG (-1)          /* invalid argument */
#define LBM_ERR_CUDA (-2)         /* a CUDA runtime call failed */
#define LBM_ERR_NOMEM (-3)        /* device allocation failed */
#define LBM_ERR_CAPACITY (-4)     /* more spheres, neighbours or links than sized */
#define LBM_ERR_DIVERGED (-5)     /* non-positive or non-finite density found */
#define LBM_ERR_UNSUPPORTED (-6)  /* valid request this build does not implement */
#define LBM_ERR_TIMEOUT (-7)      /* a device-side wait gave up */
#define LBM_ERR_GEOMETRY (-8)     /* a sphere moved >= 1/4 node in one step or left the box */

/* Storage of the populations (arithmetic is FP32 in every case). */
#define LBM_FP32 0       /* f_i - w_i stored as FP32 */
#define LBM_BF16_DEV 1   /* f_i - w_i stored as bfloat16 */
#define LBM_FP16_DEV 2   /* f_i - w_i stored as binary16 */

/* Order of the work inside lbm_step when spheres are present.  Both give
 * bitwise the same results.  SERIAL (the default) runs every kernel on the
 * handle's stream, one after the other.  OVERLAP collides the nodes of
 * 32-byte groups far from every sphere on a second, low-priority stream
 * while the link, DEM and geometry work of the neighbouring steps runs on a
 * high-priority one; the near groups are collided from a compacted list.
 * On a dense suspension (256^3, 2000 spheres of radius 4) OVERLAP is the
 * slower of the two: a quarter of the groups are near, and splitting the
 * collide costs more memory time than the overlap hides. */
#define LBM_SCHEDULE_SERIAL 0
#define LBM_SCHEDULE_OVERLAP 1

/* Execution of the DEM sub-steps. */
#define LBM_DEM_AUTO 0
#define LBM_DEM_CLUSTER 1
#define LBM_DEM_GRID 2

/* Momentum exchange on sphere links. */
#define LBM_MEA_PAPER 0
#define LBM_MEA_GALILEAN 1

/* Memory space of a caller buffer. */
#define LBM_HOST 0
#define LBM_DEVICE 1

typedef struct {
    int32_t nx, ny, nz;        /* lattice nodes; each >= 1 */
    int32_t periodic_z;        /* must be 0: walls at z = -1/2 and nz - 1/2 */
    double tau0;               /* relaxation time, > 1/2 (Eq. 15) */
    double cs_smag;            /* Smagorinsky constant C >= 0 (Eq. 18); 0 = BGK */
    double body_accel[3];      /* g; force density rho*g on fluid nodes */
    double wall_vel_lo[3];     /* velocity of the z = -1/2 wall; z component must be 0 */
    double wall_vel_hi[3];     /* velocity of the z = nz-1/2 wall; z component must be 0 */
    double rho_particle;       /* sphere density / fluid density, > 0 */
    double kn;                 /* normal contact stiffness (Eq. 1), >= 0 */
    double restitution;        /* normal restitution coefficient, in (0, 1] */
    int32_t dem_substeps;      /* DEM sub-steps per lattice step, >= 1 */
    int32_t precision;         /* LBM_FP32, LBM_BF16_DEV or LBM_FP16_DEV */
    int32_t max_particles;     /* capacity for spheres, >= 0 */
    double max_radius;         /* largest radius lbm_set_particles accepts, <= 16 */
    void *cuda_stream;         /* cudaStream_t to run on; NULL: the library makes one */
    int32_t device;            /* CUDA device ordinal */
    int32_t schedule;          /* LBM_SCHEDULE_SERIAL (0) or LBM_SCHEDULE_OVERLAP */
    int32_t momentum_correction; /* 1: a node a sphere covers hands its fluid momentum (and torque)
                                    to the sphere, a refilled node takes its momentum from it
                                    (Aidun, Lu & Ding 1998; not in the paper); 0: off;
                                    other values: LBM_ERR_ARG */
    double kt;                 /* tangential contact stiffness (Eq. 2), >= 0 */
    double mu;                 /* Coulomb friction coefficient mu_s (Eq. 2), >= 0; friction acts
                                  between spheres and against the walls when kt > 0 and mu > 0 */
    double restitution_t;      /* tangential restitution in (0, 1], sets the dashpot gamma_t of
                                  Eq. 2 like restitution sets gamma_n; 1: no tangential damping */
    int32_t zieb;              /* 1: the plane z = 0 is a ZIEB face (Sect. 2.6) onto a virtual
                                  piston cylinder below it, in place of the wall z = -1/2 for the
                                  fluid (spheres still touch that plane); needs
                                  LBM_SCHEDULE_SERIAL and no batch (else LBM_ERR_UNSUPPORTED);
                                  0: off; other values: LBM_ERR_ARG */
    double zieb_area;          /* piston / cylinder cross-section A_p > 0 (lattice units) */
    double zieb_volume;        /* cylinder volume V_0 > zieb_area * (piston travel); a step at which
                                  V_0 - A_p H_p <= 0 sets LBM_ERR_DIVERGED (sticky) */
    double zieb_piston_velocity; /* v_p: the piston displacement H_p grows by v_p per step */
    int32_t mea;               /* momentum exchange: LBM_MEA_PAPER (Eqs. 25, 26) or LBM_MEA_GALILEAN
                                  (populations carry c - u_b, Wen, Zhang & Fang 2014; not in the
                                  paper); other values: LBM_ERR_ARG */
    int32_t dem_mode;          /* how the DEM sub-steps run: LBM_DEM_AUTO (one thread-block
                                  cluster up to 4096 spheres, else a cooperative grid),
                                  LBM_DEM_CLUSTER or LBM_DEM_GRID; the same arithmetic either way;
                                  other values: LBM_ERR_ARG */
} lbm_params;

typedef struct {
    int64_t nodes;             /* nx*ny*nz */
    int64_t fluid_nodes;       /* fluid nodes of the current geometry */
    int64_t links;             /* sphere cut links treated in the last step */
    int64_t refilled;          /* nodes refilled in the last step */
    int64_t steps;             /* lattice steps taken since lbm_set_particles */
    int32_t particles;         /* spheres */
    int32_t precision;         /* as created */
    int64_t device_bytes;      /* device memory the handle holds */
} lbm_info_t;

/* Allocate a simulation and set the fluid to rest (f = w, rho = 1, u = 0)
 * with no spheres.  *out receives the handle.  LBM_ERR_ARG on an invalid
 * parameter (tau0 <= 1/2, a wall velocity with a z component, with spheres
 * an nx or ny below 2 (ceil(max_radius) + 3) + 1, so that a sphere's link
 * tile does not wrap onto itself, ...), LBM_ERR_UNSUPPORTED for
 * periodic_z != 0, LBM_ERR_NOMEM / LBM_ERR_CUDA on device failure. */
int lbm_create(const lbm_params *params, lbm_handle *out);

/* ZIEB face (Sect. 2.6, Eqs. 8, 9): after each step the cylinder density
 * rho follows rho <- rho exp[(v_p A_p - v_f A_p) / (V_0 - A_p H_p)], with v_f
 * the mean inflow velocity u_z over the face's fluid nodes, and every fluid
 * node of the face takes the equilibrium at density rho and at the velocity
 * left once the population normal to the face has restored that density.
 * out[3] (host) receives rho, H_p and v_f after the last step (synchronises).
 * LBM_ERR_ARG when the handle has no ZIEB face. */
int lbm_zieb_state(lbm_handle h, double *out);

/* Piston velocity v_p for the following steps (synchronises).  LBM_ERR_ARG
 * when the handle has no ZIEB face or vp is not finite. */
int lbm_zieb_set_piston(lbm_handle h, double vp);

/* Self-test of the failure path of the device-side waits (no compute):
 * runs the bounded grid barrier of the cooperative DEM with a partner block
 * that never arrives.  The wait gives up after its poll limit (about a
 * second), the kernel returns, and the call returns LBM_ERR_TIMEOUT, which
 * stays the handle's sticky status; the device context stays usable for
 * other handles. */
int lbm_selftest_wait(lbm_handle h);

/* Free everything the handle holds (synchronises its stream first). */
int lbm_destroy(lbm_handle h);

/* Place n spheres (host arrays): centres pos[n][3] (x in [0, nx), y in
 * [0, ny): the caller wraps periodic coordinates; z in (-1/2, nz - 1/2);
 * else LBM_ERR_ARG), velocities vel[n][3], angular velocities
 * omega[n][3], radii radius[n] in (0, max_radius], and fixed[n] (NULL = none
 * fixed; 1 = prescribed motion: the centre moves with the given constant
 * velocity, velocity and spin never change).  Resets the fluid to rest, the
 * step counter to 0, the external load to 0, the tangential contact state
 * (Eq. 2) and a ZIEB cylinder (density 1, H_p = 0, the piston velocity kept),
 * and computes the node geometry (Sect. 2.3).  LBM_ERR_CAPACITY if
 * n > max_particles. */
int lbm_set_particles(lbm_handle h, int32_t n, const double *pos, const double *vel,
                      const double *omega, const double *radius, const uint8_t *fixed);

/* External force and torque on every sphere ([n][3] each, NULL = zero), added
 * to the hydrodynamic load during the DEM sub-steps of every following step
 * until set again (e.g. the load of another solver coupled to the spheres).
 * Host values are copied into the library's pinned staging buffers before the
 * call returns (the caller may reuse its arrays at once) and reach the device
 * in stream order, without waiting for the stream.  Non-finite host values:
 * LBM_ERR_ARG; LBM_ERR_NOMEM if the staging buffers cannot be allocated. */
int lbm_set_particle_load(lbm_handle h, const double *force, const double *torque, int32_t where);

/* Overwrite the populations of the fluid nodes with f[19][N] (FP64, the
 * pre-collision state of the current time); solid nodes are ignored. */
int lbm_set_populations(lbm_handle h, const double *f, int32_t where);

/* Advance nsteps >= 0 lattice steps (asynchronous on the handle's stream).
 * One step, Sect. 2.5 in the order of Sect. 2.3: geometry at the current
 * sphere positions, refill of uncovered nodes, collision, streaming with
 * interpolated bounce-back, momentum exchange, DEM sub-steps. */
int lbm_step(lbm_handle h, int32_t nsteps);

/* Hydrodynamic force F[n][3] and torque T[n][3] (about the centre) of the
 * last step (Eqs. 25, 26, or their Galilean-invariant form under
 * LBM_MEA_GALILEAN, plus the covered / uncovered-node momentum under
 * momentum_correction); zero before the first step. */
int lbm_forces(lbm_handle h, double *F, double *T, int32_t where);

/* Current sphere centres, velocities and angular velocities ([n][3] each;
 * any pointer may be NULL to skip it). */
int lbm_particles(lbm_handle h, double *pos, double *vel, double *omega, int32_t where);

/* lbm_forces and lbm_particles in one call with one stream synchronisation
 * (a coupling loop reads both after every step): F, T the hydrodynamic load
 * of the last step, pos, vel, omega the current state ([n][3] each; any
 * pointer may be NULL to skip it). */
int lbm_particle_state(lbm_handle h, double *F, double *T, double *pos, double *vel, double *omega,
                       int32_t where);

/* Density rho[N] and velocity u[3][N] of the current state (Eqs. 5, 6 with
 * the half-force shift); solid nodes give rho = 0 and u = 0.  Either pointer
 * may be NULL. */
int lbm_fields(lbm_handle h, float *rho, float *u, int32_t where);

/* Pre-collision populations f[19][N] of the current state in FP64
 * (w_i + stored deviation); solid nodes give 0. */
int lbm_populations(lbm_handle h, double *f, int32_t where);

/* Owner of every node for the current geometry: sphere index, -1 = fluid. */
int lbm_geometry(lbm_handle h, int32_t *owner, int32_t where);

/* Counters and sizes (synchronises the stream). */
int lbm_info(lbm_handle h, lbm_info_t *info);

/* Phases of a step timed by the profiler.  Under LBM_SCHEDULE_OVERLAP with
 * spheres, the collisions of nodes far from every sphere run on a second
 * stream (LBM_PHASE_COLLIDE_FAR), overlapped with the link / DEM / geometry
 * work of the previous step and the near-node collisions of this one;
 * LBM_PHASE_COLLIDE then times the near nodes only.  Otherwise
 * LBM_PHASE_COLLIDE times the whole lattice and the two far phases are 0. */
#define LBM_PHASE_GEOMETRY 0     /* node geometry and refill */
#define LBM_PHASE_COLLIDE 1      /* fused collide-stream kernel (near nodes) */
#define LBM_PHASE_LINKS 2        /* bounce-back on sphere links and momentum exchange */
#define LBM_PHASE_DEM 3          /* neighbour lists and DEM sub-steps */
#define LBM_PHASE_COLLIDE_FAR 4  /* fused collide-stream kernel, far nodes (second stream) */
#define LBM_PHASE_WAIT_FAR 5     /* near tags of the next step, then the wait for the far collisions */
#define LBM_PHASES 6

/* enable != 0: from now on record CUDA events on the handle's stream around
 * each phase of every step and reset the totals; enable == 0: stop.  Adds no
 * work on the device, only event records between kernels. */
int lbm_profile(lbm_handle h, int32_t enable);

/* Device time per phase, summed over the steps since profiling was enabled:
 * ms[LBM_PHASES] in milliseconds, *steps the number of steps (either pointer
 * may be NULL).  Synchronises the stream. */
int lbm_profile_read(lbm_handle h, double *ms, int64_t *steps);

/* Largest lattice (nodes) lbm_fields_noalloc accepts. */
#define LBM_NOALLOC_MAX_NODES (1 << 20)

/* lbm_fields to host memory without allocating device memory.  lbm_fields
 * with host outputs stages the data through a stream-ordered temporary
 * (cudaMallocAsync); some callers cannot allow that: an application whose
 * framework allocator already holds the device's memory, or a step loop
 * that must not allocate (a real-time loop).  This entry point stages
 * through a fixed 16 MiB array built into the library instead; it calls no
 * device allocation routine.  The paper has no counterpart: this is a
 * service of the library.
 *   rho[N], u[3][N]: host buffers (either may be NULL), as lbm_fields.
 *   LBM_ERR_CAPACITY if nx*ny*nz > LBM_NOALLOC_MAX_NODES.
 * The first call on a device looks up the array's device address there.
 * With lazy module loading (the CUDA default) the driver commits the
 * array's 16 MiB on that device at this first call, not when the library
 * loads, and holds it until the process exits: make the first call at
 * start-up, before a framework allocator takes the device's memory (if the
 * driver cannot commit it, the call returns LBM_ERR_NOMEM).  Synchronises the
 * handle's stream, like lbm_fields to host memory.  All calls on a device
 * share the array; calls whose work overlaps on the same GPU (handles on
 * different streams used from different threads) race on it. */
int lbm_fields_noalloc(lbm_handle h, float *rho, float *u);

/* Wait for the handle's stream and return its sticky device status. */
int lbm_sync(lbm_handle h);

/* Static description of a return code. */
const char *lbm_error_string(int code);

/* ---- Batched form: many independent simulations stepped together --------
 *
 * Not in the paper, which runs its parameter sweeps (particle size, packing
 * fraction, polydispersity) as separate simulations.  A batch holds `count`
 * members, each an lbm_handle created from params[i] (its own box, tau0,
 * Cs, body force, capacities), all on one device, one precision and one
 * stream (params[0].cuda_stream, or a stream the batch makes).  One batched
 * step is six launches for all members together: marks, refill, one
 * persistent collide launch over a table of 256-ish-node chunks of every
 * member, links, neighbour lists, and the DEM with one thread-block cluster
 * per member.  The six are captured once per step parity in a CUDA graph
 * and replayed; the collide's block size and grid come from an autotuner
 * that times the candidates on the members' own state (which it restores).
 * Results are bitwise those of stepping each member alone with lbm_step. */
typedef struct lbm_batch_s *lbm_batch;

/* Create count >= 1 members.  Members run the serial order with one DEM
 * cluster each: their schedule and dem_mode fields are not used.  LBM_ERR_ARG
 * if the params differ in device, precision or stream or one is invalid (as
 * lbm_create, whose box rule each member meets for its own max_radius),
 * LBM_ERR_UNSUPPORTED if the DEM cluster cannot hold the largest
 * max_particles or a member has a ZIEB face. */
int lbm_batch_create(const lbm_params *params, int32_t count, lbm_batch *out);

/* Destroy the batch and its members (synchronises the stream first). */
int lbm_batch_destroy(lbm_batch b);

/* Member i (0 <= i < count): use it with lbm_set_particles,
 * lbm_set_particle_load, lbm_set_populations, lbm_forces, lbm_particles,
 * lbm_fields, lbm_populations, lbm_geometry, lbm_info and lbm_sync.  The
 * batch owns it: lbm_step and lbm_destroy on a member return LBM_ERR_ARG. */
int lbm_batch_handle(lbm_batch b, int32_t i, lbm_handle *out);

/* Run the collide autotuner now (lbm_batch_step runs it on first use):
 * block sizes 128, 256, 512, each with a register budget of 64 or 85 per
 * thread, x grids of half and all resident blocks and one block per chunk,
 * three timed launches each on the members' state, which
 * is copied aside and restored (needs that much free device memory, else
 * LBM_ERR_NOMEM).  Outputs (each may be NULL): threads per block, blocks,
 * mean ms per launch of the choice. */
int lbm_batch_tune(lbm_batch b, int32_t *threads, int32_t *blocks, float *ms);

/* Advance every member by nsteps (asynchronous on the batch stream).
 * LBM_ERR_ARG if the members are not at the same step parity (a member's
 * lbm_set_particles resets its step count); a member's sticky error is
 * returned as is. */
int lbm_batch_step(lbm_batch b, int32_t nsteps);

/* Wait for the batch stream; the first member's sticky error, if any. */
int lbm_batch_sync(lbm_batch b);

/* ---- Differentiation form: plate drag of a channel flow and its gradient --
 *
 * Not in the paper.  A D3Q19 channel: an inlet plane x = 0 where the
 * populations are the equilibrium (Eq. 9) at the density of plane x = 1 and
 * the velocity u_peak 4 zh (1 - zh) x^, zh = (z + 1/2)/nz; an outlet plane
 * x = nx - 1 at the equilibrium with density 1 and the velocity of plane
 * nx - 2; y periodic; halfway walls at z = -1/2 and nz - 1/2; a fixed plate
 * (node box, halfway bounce-back) and fixed spheres (interpolated
 * bounce-back, Eq. 19).  The collision is the production one (Sect. 2.2:
 * BGK, Smagorinsky tau of Eq. 18, body force g_x).  J is the plate drag
 * (x component of the momentum exchange, Eq. 25) averaged over steps
 * avg_from .. steps.  lbm_channel_backward returns dJ/dtheta,
 * theta = (inlet_peak, body_accel_x, cs_smag), by a hand-written adjoint of
 * the step, recomputing the states between checkpoints taken every
 * checkpoint_every steps of the forward run. */
typedef struct lbm_channel_s *lbm_channel;

typedef struct {
    int32_t nx, ny, nz;        /* nx >= 8, nz >= 2 */
    double tau0;               /* > 1/2 */
    double cs_smag;            /* theta[2], >= 0 */
    double body_accel_x;       /* theta[1] */
    double inlet_peak;         /* theta[0] */
    int32_t plate_lo[3];       /* plate node box, inclusive (empty if lo > hi); 2 <= x <= nx - 3 */
    int32_t plate_hi[3];
    int32_t steps;             /* >= 1 */
    int32_t avg_from;          /* first step of the drag average, 1 .. steps */
    int32_t checkpoint_every;  /* K >= 1: device memory holds K + steps/K + 5 lattice states */
    int32_t device;
    void *cuda_stream;         /* NULL: the channel makes its own */
} lbm_channel_params;

/* Create; n fixed spheres (host arrays pos[n][3], radius[n]; x - R > 1 and
 * x + R < nx - 2).  Decides the node classes and link fractions once.
 * LBM_ERR_UNSUPPORTED when 19 nx ny nz >= 2^31, ny > 65535 or nz > 64000
 * (the kernels index in 32 bits and run one block row per (y, z)). */
int lbm_channel_create(const lbm_channel_params *params, int32_t n, const double *pos, const double *radius,
                       lbm_channel *out);
int lbm_channel_destroy(lbm_channel c);

/* Replace theta = (inlet_peak, body_accel_x, cs_smag); drops the checkpoints. */
int lbm_channel_set_theta(lbm_channel c, const double *theta);

/* Run steps from rest, keep the checkpoints, *J = the mean plate drag. */
int lbm_channel_forward(lbm_channel c, double *J);

/* grad[3] = dJ/dtheta at the theta of the last lbm_channel_forward
 * (LBM_ERR_ARG if there was none since the last set_theta). */
int lbm_channel_backward(lbm_channel c, double *grad);

/* After a forward: per-step plate drag drag[steps]; the final populations
 * f[19][nx*ny*nz] (f = w + stored deviation); node classes type[nx*ny*nz]
 * (0 fluid, 1 sphere, 2 inlet, 3 outlet, 4 plate; geometry needs no forward). */
int lbm_channel_drag(lbm_channel c, double *drag);
int lbm_channel_populations(lbm_channel c, double *f);
int lbm_channel_geometry(lbm_channel c, uint8_t *type);

#ifdef __cplusplus
}
#endif

#endif /* GB300_LBM_H */
