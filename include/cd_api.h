/*
 * cd_api.h -- C ABI of the GB300 (sm_103a) Contact Dynamics hot path.
 *
 * The library computes one time step of the non-smooth Contact Dynamics (CD)
 * method of Shojaaee et al., "An Adaptive Hierarchical Domain Decomposition
 * Method for Parallel Contact Dynamics Simulations of Granular Materials"
 * (arXiv:1104.3516), for rigid frictional discs (2D) or spheres (3D):
 *
 *   1. contact detection with a cell list (Sec. 3.2), margin delta (Eq. 12,
 *      Sec. 3.1: cell side l = 2 r_max + delta),
 *   2. the iterative contact-impulse solve: every contact re-solved from its
 *      two bodies' current velocities against the Signorini (Eqs. 3-5) and
 *      Coulomb (Eqs. 6-11) conditions, nonlinear Gauss-Seidel until the
 *      convergence test of Sec. 2.1 passes (Fig. 2, Sec. 2.1),
 *   3. the first-order Euler update of velocities and positions (Eqs. 1-2).
 *
 * The Gauss-Seidel order is a colour order: contacts are coloured so that no
 * two contacts of one colour share a particle, and each colour is updated in
 * parallel.  This is an admissible sequential order of the paper's scheme
 * (each freshly computed force is used immediately by later contacts).
 *
 * Conventions used by every entry point:
 *   - Arrays passed as pointers are DEVICE pointers on the current CUDA
 *     device unless the parameter name ends in `_host`.  They are owned by
 *     the caller and must stay valid for the life of the system; the library
 *     never frees them.
 *   - Layouts: pos, vel: n*dim doubles interleaved per particle
 *     (x0,y0[,z0],x1,...); omega: n doubles (2D, about z) or n*3 (3D);
 *     theta: n doubles (2D orientation) or NULL.
 *   - Walls are axis-aligned planes with index k = 2*axis + side (side 0:
 *     low plane, side 1: high plane), infinite mass and prescribed velocity.
 *     A wall acts as body number n + k in contact keys.
 *   - Contacts are identified by key (a, b), a < b; the normal points from
 *     body a to body b; impulses are P = R dt.  2D impulses are stored as
 *     (P_n, P_t) with t = (-n_y, n_x); 3D as (P_n, P_tx, P_ty, P_tz).
 *   - All work is enqueued on the stream given at creation; calls that
 *     return statistics synchronise that stream.  A system is not
 *     thread-safe; use one system per stream.
 *   - Every function returns a cd_status and never aborts or traps; the
 *     message of the last failure is available from cd_last_error().
 */
#ifndef CD_API_H
#define CD_API_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CD_OK = 0,
    CD_ERR_INVALID_ARG = 1,   /* bad size, NaN or non-positive radius, bad params */
    CD_ERR_CUDA = 2,          /* a CUDA runtime call failed (message has details) */
    CD_ERR_OOM = 3,           /* workspace missing or too small */
    CD_ERR_CAPACITY = 4,      /* more contacts (or colours) than the capacity */
    CD_ERR_NOT_CONVERGED = 5, /* informational: sweep cap reached, step still taken */
    CD_ERR_TIMEOUT = 6,       /* a bounded device-side wait ran out */
    CD_ERR_STATE = 7          /* call out of order (e.g. solve before detection) */
} cd_status;

enum { CD_FP64 = 0, CD_FP32 = 1 };
/* Convergence tests of Sec. 2.1.  GLOBAL_REL: |R^j - R^{j-1}| / (R^j + R^{j-1})
 * < alpha with R = mean |P| (the default); GLOBAL_SQ: the paper's squared form
 * (II); LOCAL: test (I) (90% of contacts below alpha relative, the rest below
 * alpha R_avg^2 absolute); NONE: run exactly max_sweeps. */
enum { CD_CONV_NONE = -1, CD_CONV_GLOBAL_REL = 0, CD_CONV_GLOBAL_SQ = 1, CD_CONV_LOCAL = 2 };

typedef struct {
    int64_t dim;            /* 2 or 3 */
    int64_t precision;      /* CD_FP64 or CD_FP32 (sweep arithmetic; detection,
                               residual and integration stay FP64) */
    double dt;              /* time step */
    double mu;              /* Coulomb friction coefficient (Eq. 8) */
    double gravity[3];      /* external acceleration, applied explicitly (Eq. 1) */
    double box_lo[3];       /* box spanned by the cell grid; periodic extent */
    double box_hi[3];
    int64_t periodic[3];    /* 1: periodic along that axis */
    int64_t wall_mask;      /* bit k set: wall k present */
    double wall_pos[6];     /* initial plane position of each wall */
    double wall_vel[18];    /* velocity of each wall (3 per wall) */
    double delta;           /* detection margin: contact iff surface gap < delta */
    double alpha;           /* convergence threshold */
    int64_t criterion;      /* CD_CONV_* */
    int64_t max_sweeps;     /* iteration cap N_I per time step */
    int64_t warm_start;     /* 1: start each solve from the previous step's
                               impulses matched by contact key; 0: from zero */
    int64_t rotations;      /* 0: rotational degrees of freedom frozen */
    uint64_t seed;          /* seeds the colouring priorities */
    int64_t max_contacts;   /* contact capacity of the workspace */
    int64_t timing;         /* 1: record CUDA events around the phases of each
                               step on the system's stream (see cd_step_stats) */
    double parallel_p;      /* mixed update of Sec. 2.3: the contacts whose key
                               hashes below p (splitmix64(key ^ seed *
                               0xD1B54A32D192ED03) / 2^64 < p) are updated in
                               parallel within each sweep (from the velocities
                               at the sweep start, applied at its end), the
                               rest sequentially.  0: pure Gauss-Seidel.
                               Plain (not batched) systems only. */
    int64_t tape_steps;     /* 0: no adjoint.  T > 0: every cd_step records the
                               data cd_adjoint_step needs (colour-order contact
                               records with their converged impulses, and the
                               velocities the step produced) into a ring of T
                               slots in the workspace (about 64 B per contact of
                               capacity and 32 B per particle each); plain 2D
                               FP64 systems only. */
    double adjoint_compliance; /* 0: the reverse pass solves the rigid
                               frozen-state system exactly (derivative of
                               the method as it stands).  eps > 0: each
                               retained row gets a relative compliance eps
                               (rows Phi^T (H Gamma + q) - eps diag(w) Y = 0,
                               w = 1/m_n, 1/m_t), so that hyperstatic contact
                               networks, where the rigid multipliers are not
                               unique and the Gauss-Seidel iteration can
                               drift, give the bounded derivative of slightly
                               compliant contacts.  Not in the paper. */
    int64_t use_graph;      /* 1: cd_step captures the launches of one time
                               step into a CUDA graph on first use and replays
                               it for every step (fewer launch overheads for
                               small systems); same results.  Needs a
                               non-default stream and timing 0; the graph is
                               dropped by cd_set_workspace. */
    int64_t sweep_threads;  /* block shape of the persistent sweep grid: threads
                               per block, 128, 256 or 512 (0: 512) ... */
    int64_t sweep_blocks_per_sm; /* ... and blocks per SM, 1, 2 or 4 (0: 1), at
                               most 1024 threads per SM.  The colour classes are
                               spread over all blocks; results do not depend on
                               the shape except for the summation order of the
                               residual.  Chosen by the autotuner of the
                               Python package, or left at 512 x 1. */
    double wall_push[6];    /* force-controlled walls (the pressure walls of the
                               Fig. 10 setup): wall k with wall_mass[k] > 0 is a
                               rigid body of that mass moving along its normal
                               only, pushed along its inward normal by the force
                               wall_push[k] (applied explicitly, Eq. 1) and
                               taking part in the impulse solve like a particle:
                               its inverse mass enters the normal row of its
                               contacts, and its contacts conflict in the
                               colouring.  wall_vel holds its velocity, which
                               the steps update.  Plain systems with the global
                               colour order, no mixed update, no tape. */
    double wall_mass[6];    /* 0: wall k kinematic (prescribed velocity) */
    int64_t domains[3];     /* domain-wise update of the parallel algorithm
                               (Sec. 3.1): the box [box_lo, box_hi] is cut
                               into domains[k] equal slabs along axis k (0 or
                               1: not cut); a contact belongs to the domain
                               holding the middle of its gap, x_a + n (r_a +
                               g / 2) (wrapped on a periodic axis).  In every
                               sweep each domain updates its own contacts in
                               the colour order, seeing the velocities of the
                               sweep start changed by its own updates only
                               (the other domains' contacts keep the impulses
                               of the previous sweep), and the domains'
                               velocity changes are summed at the end of the
                               sweep: what a multi-processor run of the paper
                               computes, on one GPU.  The workspace grows by
                               2 velocity records (and their start copies) per
                               contact of capacity.  Plain systems with the
                               colour-barrier schedule, kinematic walls, no
                               mixed update, no tape.  All 1: Gauss-Seidel. */
    int64_t parallel_redraw; /* mixed update (parallel_p): 0 the parallel subset
                               is fixed per contact key; 1 it is drawn afresh
                               in every iteration step (the step's number
                               mixed into the hash of the key), the way the
                               paper draws its random sequential order anew
                               each step (Sec. 2.1) */
    int64_t merge_last_colour; /* colour-barrier schedule of a plain system:
                               a step may run its M last colours in one
                               phase when the last class is small (at most a
                               quarter of the first merged one): the contacts
                               of the M colours are grouped into the chains
                               that share particles (each at most 64
                               contacts), every chain goes whole to one block,
                               which updates the chains' contacts of colour
                               K-M, synchronises its threads, then those of
                               colour K-M+1, and so on.  The order is the
                               colour order, so results equal those without
                               merging; M - 1 grid barriers per sweep fewer.
                               1 or 3: M = 3 if that is taken, else M = 2;
                               2: M = 2 only; 4: as 1, but a step merges only
                               if the system's previous solve took at least
                               64 sweeps (or there was none): the grouping
                               costs about as much as ~60 sweeps' saving;
                               0: every colour its own phase. */
} cd_params;

typedef struct cd_system cd_system;

typedef struct {
    int64_t sweeps;           /* sweeps done in the last solve */
    int64_t converged;        /* 1 if the convergence test passed */
    double residual;          /* value of the convergence test at the last sweep */
    double r_avg;             /* mean |P| after the last sweep */
    int64_t n_contacts;
    int64_t n_colours;
    double wall_force[6];     /* sum of normal impulses on each wall / dt */
    int64_t n_phases;         /* grid-barrier phases per sweep: n_colours, or
                                 M - 1 fewer when the M last colours ran as
                                 one phase (params.merge_last_colour) */
} cd_solve_stats;

typedef struct {
    int64_t steps_done;
    int64_t total_sweeps;         /* summed over the steps of the call */
    int64_t total_contact_updates;/* sum over steps of sweeps * contacts */
    int64_t max_sweeps_in_step;
    int64_t n_not_converged;      /* steps that hit the sweep cap */
    int64_t kernel_launches;      /* kernels this library launched in the call */
    double phase_ms[4];           /* with params.timing: device time of [0]
                                     detection, [1] colouring, ordering and the
                                     free-flight velocities, [2] the persistent
                                     sweep kernel (the impulse solve), [3] the
                                     integration, summed over the steps of the
                                     call (CUDA events on the system's stream) */
    cd_solve_stats last;          /* statistics of the last step */
} cd_step_stats;

/* Creates a system over caller-owned device arrays (layouts above).
 * inv_mass / inv_inertia: 1/m and 1/I per particle (0 for an immovable
 * particle).  f_ext: n*dim explicit external forces, or NULL.  cuda_stream:
 * a cudaStream_t (NULL = legacy default stream).  Validates the parameters,
 * and the radii, inverse masses, positions and velocities (copied to the host
 * once), and returns CD_ERR_INVALID_ARG for a non-positive or NaN radius, a
 * negative or NaN inverse mass, a non-finite position or velocity, or a
 * box/cell grid the periodic wrap cannot handle.  The system needs a
 * workspace before use. */
cd_status cd_create_system(const cd_params* params, int64_t n, double* pos, double* vel, double* omega,
                           double* theta, const double* radius, const double* inv_mass,
                           const double* inv_inertia, const double* f_ext, void* cuda_stream,
                           cd_system** out);

/* A batch of independent packings stepped together (hundreds of packings of
 * uneven size).  Particles of all packings are concatenated: packing b owns
 * particles offsets_host[b] .. offsets_host[b+1]-1 (offsets_host[0] = 0,
 * offsets_host[n_packings] = n; host array of n_packings + 1).  params is a
 * host array of n_packings cd_params: per packing mu, gravity, box, periodic
 * axes, walls (mask, positions, velocities) are taken from its own entry;
 * dim, precision, dt, delta, alpha, criterion, max_sweeps, warm_start,
 * rotations, seed, timing and max_contacts (total over the batch) from
 * entry 0.  State arrays as in cd_create_system over
 * all n particles.  Each packing keeps its own cell grid and walls (wall k of
 * packing b is body n + 6 b + k), contacts never join two packings, and each
 * packing has its own convergence test (Sec. 2.1): the colour phases are
 * shared, and a packing whose test passed is not updated in later sweeps, so
 * every packing gets exactly the result of solving it alone.  cd_step,
 * cd_detect_contacts, cd_solve_contacts, cd_get_contacts work on the whole
 * batch; per-packing results come from cd_get_packing_stats. */
cd_status cd_create_batch(const cd_params* params, int64_t n_packings, const int64_t* offsets_host, double* pos,
                          double* vel, double* omega, double* theta, const double* radius, const double* inv_mass,
                          const double* inv_inertia, const double* f_ext, void* cuda_stream, cd_system** out);

/* Bytes of device workspace the system needs (cell grid, contact arrays in
 * key and colour order, colouring and reduction buffers). */
cd_status cd_workspace_size(const cd_system* sys, size_t* bytes);

/* Hands the system a caller-allocated device buffer of at least
 * cd_workspace_size() bytes, 256-byte aligned.  The library never calls
 * cudaMalloc; the buffer stays owned by the caller. */
cd_status cd_set_workspace(cd_system* sys, void* dev_ptr, size_t bytes);

/* Contact detection for the current positions (Sec. 3.2), followed by the
 * contact geometry, the warm-start match by key, the colouring and the colour
 * ordering.  Returns the number of contacts in *n_contacts (synchronises).
 * If they exceed max_contacts, returns CD_ERR_CAPACITY with the number
 * needed in *n_contacts and leaves the previous contact set unchanged. */
cd_status cd_detect_contacts(cd_system* sys, int64_t* n_contacts);

/* Replaces the contact set by the caller's list (device arrays, nc keys
 * (a, b) with a < b in ascending key order; impulses may be NULL for zero,
 * else nc*2 (2D) or nc*4 (3D) doubles).  Geometry, colouring and ordering are
 * computed as after detection.  Used to feed an externally chosen contact
 * set (for instance to compare solvers on the same contacts). */
cd_status cd_set_contacts(cd_system* sys, int64_t nc, const int32_t* pairs, const double* impulses);

/* The iterative impulse solve of Sec. 2.1 on the current contact set.  The
 * current particle velocities are taken as the free velocities (no contact
 * impulses); the solve applies the starting impulses, sweeps the colours
 * until the convergence test passes or max_sweeps is reached, and writes the
 * final velocities back into vel/omega and the impulses into the contact
 * store.  Positions are not moved.  out may be NULL (then nothing is
 * synchronised).  Returns CD_ERR_NOT_CONVERGED (informational) when the
 * sweep cap was hit and out was given. */
cd_status cd_solve_contacts(cd_system* sys, cd_solve_stats* out);

/* n_steps full time steps (Fig. 3): detection (as cd_detect_contacts), the
 * explicit external forces (Eq. 1 with F = m g + f_ext), the impulse solve
 * (as cd_solve_contacts), the position update (Eq. 2, periodic wrap) and the
 * wall motion.  Nothing is synchronised between steps.  out may be NULL.  On
 * contact overflow the failing step and all later ones are skipped on the
 * device, the state stays as it was before that step, and CD_ERR_CAPACITY is
 * returned once out is read (needs out != NULL or a later call). */
cd_status cd_step(cd_system* sys, int64_t n_steps, cd_step_stats* out);

/* Copies the current contact set in key order into caller DEVICE arrays
 * (any pointer may be NULL): pairs nc*2 int32, normal nc*3, gap nc,
 * impulse nc*2 (2D) / nc*4 (3D), colour nc int32.  *n_contacts receives nc.
 * Synchronises. */
cd_status cd_get_contacts(cd_system* sys, int64_t* n_contacts, int32_t* pairs, double* normal, double* gap,
                          double* impulse, int32_t* colour);

typedef struct {
    int64_t sweeps;          /* sweeps of the last solve of this packing */
    int64_t converged;
    double residual;
    double r_avg;
    int64_t n_contacts;
    double wall_force[6];    /* normal impulses on each wall / dt, last solve */
    double wall_pos[6];      /* current wall planes */
} cd_packing_stats;

/* Statistics of packings first .. first+count-1 of a batch (a plain system is
 * packing 0) into a host array of count entries.  Synchronises. */
cd_status cd_get_packing_stats(cd_system* sys, int64_t first, int64_t count, cd_packing_stats* out_host);

/* Distribution of contact-force orientations (Sec. 4.4, Fig. 14), 2D: over
 * the contacts with a nonzero impulse, phi = arctan(R_y / R_x) folded into
 * [0, pi) is counted in nbins equal bins (host array of nbins).  Uses the
 * current contact set and impulses.  Synchronises. */
cd_status cd_force_orientation(cd_system* sys, int64_t nbins, int64_t* counts_host);

/* Stress profile (Sec. 4.4, Fig. 15): for stripes [lo + i w, lo + (i+1) w)
 * along axis (i < nstripes), sigma_{axis,axis} = (1/V) sum R_axis l_axis over
 * the contacts whose contact point (middle of the gap, Sec. 3.1) lies in the
 * stripe, R = P / dt the contact force on body b, l the branch vector from
 * body a's centre to body b's centre (minimum image) or to the wall surface,
 * V = w times the box extents of the other axes (compression positive).  Host
 * array of nstripes.  Plain systems.  Synchronises. */
cd_status cd_stress_profile(cd_system* sys, int64_t axis, double lo, double width, int64_t nstripes,
                            double* sigma_host);

/* Current wall plane positions (6 doubles, host memory; packing 0 of a
 * batch).  Synchronises. */
cd_status cd_get_walls(cd_system* sys, double* wall_pos_host);

/* Host <-> device copies of the particle state (pos, vel, omega; theta if
 * the system has it) from/to pinned or pageable host memory, enqueued on the
 * system's stream (download synchronises). */
cd_status cd_upload_state(cd_system* sys, const double* pos_host, const double* vel_host,
                          const double* omega_host);
cd_status cd_download_state(cd_system* sys, double* pos_host, double* vel_host, double* omega_host);

/* Contact detection that allocates nothing, for callers that cannot call
 * cudaMalloc (code running inside a framework that owns all device memory, a
 * plug-in that may only use buffers it is given, a run with a frozen memory
 * budget).  There is no counterpart in the paper: it is the detection of
 * cd_detect_contacts (same contact set, normals and gaps, key order, walls
 * as bodies n + k) without a system object or a workspace.
 *
 * Inputs (device): pos, radius, inv_mass, inv_inertia as in
 * cd_create_system; params as there (wall planes from params->wall_pos).
 * Outputs (device, caller-owned): pairs max_contacts*2 int32, normal
 * max_contacts*3 doubles, gap max_contacts doubles (may be NULL when
 * max_contacts is 0: a size query); *n_contacts (host) the number found.
 * Work is enqueued on cuda_stream, and every call synchronises that stream
 * (it reads the largest radius and the contact count back to the host).
 *
 * Scratch lives in a fixed device array of about 4.1 MB inside the library,
 * held by every GPU that loads it until the process exits; limits: n <= 16384
 * particles, at most 65536 cells of side 2 r_max + delta, max_contacts <=
 * 65536.  Larger sizes return CD_ERR_INVALID_ARG (message via
 * cd_last_error(NULL)); more contacts than max_contacts return
 * CD_ERR_CAPACITY with the number needed in *n_contacts and nothing written
 * past max_contacts.  The first call on each device looks up the array's
 * device address (cudaGetSymbolAddress) with that device current, so make
 * that first call before any stream capture; the address is then kept for
 * the life of the process, so the entry point must not be used on a device
 * after a cudaDeviceReset of it.  All calls share the array:
 * each call clears what must start at zero, and calls that overlap on the
 * GPU (different streams or threads) race with each other. */
cd_status cd_detect_contacts_noalloc(const cd_params* params, int64_t n, const double* pos, const double* radius,
                                     const double* inv_mass, const double* inv_inertia, int64_t max_contacts,
                                     int32_t* pairs, double* normal, double* gap, int64_t* n_contacts,
                                     void* cuda_stream);

/* ---- Reverse-mode derivatives of time steps --------------------------------
 * The paper has no derivative of its method.  These calls differentiate the
 * time step map (x, v, omega, mu) -> (x', v', omega') of Eqs. 1-2 with the
 * converged impulses of the iteration (Sec. 2.1, Fig. 2, Eqs. 3-11), for
 * gradient-based calibration of friction and initial conditions.  The
 * derivative is taken at fixed contact set and fixed contact states, read off
 * the converged impulses: open (P_n at most 1e-9 times the step's largest
 * P_n: Eq. 3, or bodies left touching with no force), sliding (|P_t| equal to
 * the rounded product mu P_n: Eqs. 9-11) or sticking (Eq. 5).  Where a small
 * change of the inputs changes a state or the contact set the map has a kink
 * and this is the derivative of the side with the recorded states.  2D, FP64,
 * plain systems with params.tape_steps > 0. */
typedef struct {
    int64_t sweeps;           /* Gauss-Seidel sweeps of the transposed system */
    int64_t converged;        /* 1 if the last sweep changed the multipliers Y by
                                 sum |dY| <= alpha max(sum |Y|, sum m_n |W lambda|
                                 at the contact's two bodies) */
    double residual;          /* that ratio after the last sweep */
    int64_t n_contacts;
    int64_t n_open;
    int64_t n_stick;
    int64_t n_slide;
    double dL_dmu;            /* this step's contribution to dL/dmu */
    int64_t kernel_launches;
    int64_t n_rows;           /* equations of the frozen-state system: 2 per sticking,
                                 1 per sliding contact */
    int64_t n_dof;            /* degrees of freedom of the particles those contacts
                                 touch (3 each in 2D, 2 with rotations frozen);
                                 n_rows > n_dof means a hyperstatic network,
                                 where the impulses are not unique and the
                                 multipliers Y are the Gauss-Seidel ones from
                                 zero (the derivative of the positions is then
                                 not unique either) */
    int64_t diverged;         /* 1 if sum |Y| grew past 1e30 times its scale or
                                 stopped being finite (sweeps stopped; outputs
                                 are not meaningful) */
} cd_adjoint_stats;

/* Back-propagates through the most recent step recorded on the tape and
 * removes it from the tape (call once per step, newest first).  Inputs
 * (device): dL_dpos, dL_dvel n*2, dL_domega n -- the gradient of a loss L with
 * respect to that step's output positions, velocities and angular
 * velocities; dL_dwall_force_host (host, 6 doubles, or NULL for zeros) -- its
 * gradient with respect to that step's wall forces (the sum of the normal
 * impulses on wall k divided by dt, as cd_solve_stats.wall_force reports;
 * a wall pressure is that force over the wall's length or area).
 * Outputs (device, n*2, n*2, n): the gradient with respect to
 * the step's input state (positions before the step, velocities before the
 * external forces of Eq. 1).  Outputs may alias the inputs.  The transposed
 * system is solved by Gauss-Seidel in the forward colour order from zero
 * until a sweep changes the multipliers by less than alpha relative (see
 * cd_adjoint_stats) or max_sweeps;
 * returns CD_ERR_NOT_CONVERGED (outputs written) if the cap was hit.
 * CD_ERR_STATE if the tape is empty or the recorded step had failed.
 * out_host may be NULL.  Synchronises. */
cd_status cd_adjoint_step(cd_system* sys, const double* dL_dpos, const double* dL_dvel, const double* dL_domega,
                          const double* dL_dwall_force_host, double* dL_dpos_prev, double* dL_dvel_prev,
                          double* dL_domega_prev, double alpha, int64_t max_sweeps, cd_adjoint_stats* out_host);

/* Checkpoints of the full stepping state: positions, velocities, angular
 * velocities, orientations (if the system has them), wall planes, and the
 * contact set with its impulses (the warm start of the next step), so that
 * stepping on from a loaded checkpoint repeats the original steps bit for
 * bit.  The buffer is caller-owned device memory of cd_checkpoint_size()
 * bytes, 256-byte aligned; copies are enqueued on the system's stream.
 * Loading also empties the tape. */
cd_status cd_checkpoint_size(const cd_system* sys, size_t* bytes);
cd_status cd_save_checkpoint(cd_system* sys, void* dev_buf, size_t bytes);
cd_status cd_load_checkpoint(cd_system* sys, const void* dev_buf, size_t bytes);

/* Self-check of the bounded device-side waits (no counterpart in the paper):
 * launches the library's grid barrier as a cooperative grid (one small block
 * per SM) in which one block never arrives.  The others must give up after
 * the bound (2 s), flag the timeout and return, leaving the context usable.
 * dev_scratch: caller-owned device memory of at least 1024 bytes, 256-byte
 * aligned.  Returns
 * CD_OK when the withheld barrier ended by its bound with the timeout
 * flagged (*elapsed_ms_host: the kernel's duration), CD_ERR_STATE if the
 * barrier completed or no timeout was flagged.  Synchronises the stream. */
cd_status cd_selfcheck_wait_bound(void* dev_scratch, size_t bytes, void* cuda_stream, double* elapsed_ms_host);

/* Releases the host-side system object (not the caller's arrays or
 * workspace).  Safe on NULL. */
void cd_destroy_system(cd_system* sys);

/* Message of the last failure on this system ("" if none); NULL system gives
 * the last failure of cd_create_system or cd_detect_contacts_noalloc on this
 * thread. */
const char* cd_last_error(const cd_system* sys);

#ifdef __cplusplus
}
#endif

#endif /* CD_API_H */
