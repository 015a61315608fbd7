/*
 * lbib.h -- C ABI of the GB300 lattice-Boltzmann / immersed-boundary step.
 *
 * One simulation = one D3Q19 fluid box plus elastic triangulated objects
 * coupled to it (Cimrak, Gusenbauer, Jancigova, "An ESPResSo implementation
 * of elastic objects immersed in a fluid", arXiv:1312.3426).  The calls
 * follow the paper's statement of a simulation: create a template (Sec. 5,
 * template creation), add objects from it (Sec. 5, adding of the object),
 * initialise the fluid (Sec. 6, fluid initialisation), integrate (Sec. 6,
 * main loop) and read out node positions, object measures and the velocity
 * field (Sec. 5, output and object analysis).
 *
 * Conventions shared by every call:
 *   - Lattice units: spacing 1, time step 1.  Lattice node (i,j,k) sits at
 *     (i+1/2, j+1/2, k+1/2); the box is [0,nx) x [0,ny) x [0,nz).
 *   - With walls_y = 1 the rows j = 0 and j = ny-1 are solid and the
 *     halfway bounce-back planes are y = 1 and y = ny-1; x and z are always
 *     periodic, y is periodic when walls_y = 0.
 *   - All pointers are plain host pointers unless stated otherwise.  Input
 *     arrays are owned by the caller and copied before the call returns.
 *     Output arrays are caller-allocated; their capacity (in elements) is
 *     passed in and LBIB_ERR_ARG is returned when it is too small.
 *   - The library owns all device memory of a simulation; lbib_destroy
 *     releases it.
 *   - Every call returns a status.  lbib_last_error() gives a message for
 *     the last failing call on that simulation.  A device-side error (a
 *     CUDA error, an unstable fluid, a bounded device wait that gave up) is
 *     sticky: every later call on the simulation returns it, until
 *     lbib_destroy.
 *   - Work is enqueued on the CUDA stream given to lbib_create (0 = legacy
 *     default stream).  lbib_step returns before the GPU finishes; read-outs
 *     and lbib_sync wait for it.  Inside lbib_step the membrane forces of
 *     the next step are computed on a second, library-owned stream while
 *     the fluid step runs; lbib_step orders that stream behind the given
 *     one with CUDA events and makes the given stream wait for it before
 *     returning, so later work on the given stream sees a finished step.
 *   - The library uses the current CUDA device at lbib_create for all later
 *     calls on that simulation.
 */
#ifndef LBIB_H
#define LBIB_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define LBIB_API __attribute__((visibility("default")))
#else
#define LBIB_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbib_sim lbib_sim;          /* opaque, library-owned */

typedef enum {
    LBIB_OK = 0,
    LBIB_ERR_ARG = -1,       /* bad argument, capacity too small, NULL pointer */
    LBIB_ERR_ID = -2,        /* template/object ids must run 0,1,2,... (Sec. 5) */
    LBIB_ERR_MESH = -3,      /* not a closed, consistently inward-ordered 2-manifold */
    LBIB_ERR_NOMEM = -4,     /* device allocation failed */
    LBIB_ERR_UNSTABLE = -5,  /* NaN or |u| > 0.3 in the fluid, or a NaN node */
    LBIB_ERR_TIMEOUT = -6,   /* a bounded device-side wait gave up */
    LBIB_ERR_CUDA = -7,      /* any other CUDA error */
    LBIB_ERR_STATE = -8      /* call out of order (e.g. step before fluid_init) */
} lbib_status;

/* Storage of the 19 populations.  All forms store h_i = f_i - w_i rho0 (the
 * deviation from the rest equilibrium) and collide in FP32.  F16S/BF16S
 * store h_i * 2^pop_scale_log2 rounded to nearest-even in FP16/BF16. */
typedef enum {
    LBIB_POP_F32 = 0,
    LBIB_POP_F16S = 1,
    LBIB_POP_BF16S = 2
} lbib_precision;

/* Fluid parameters (Sec. 6, fluid initialisation; Sec. 2, LB method).
 * tau: BGK relaxation time (> 0.5; kinematic viscosity (tau - 1/2)/3).
 * rho0: rest density.  body_force: uniform force density on every fluid
 * cell.  friction: the drag coefficient xi of Eq. dragforce. */
typedef struct {
    int nx, ny, nz;
    int walls_y;
    double tau;
    double rho0;
    double body_force[3];
    double friction;
    int precision;           /* lbib_precision */
    int pop_scale_log2;      /* F16S/BF16S only; 0..30 */
} lbib_fluid_params;

/* Creates a simulation: allocates the fluid on the current device (state
 * undefined until lbib_fluid_init).  cuda_stream is a cudaStream_t or NULL.
 * Limits: nx, nz >= 1; ny >= 3 with walls; fluid cells < 2^31. */
LBIB_API lbib_status lbib_create(const lbib_fluid_params *params, void *cuda_stream, lbib_sim **out);

/* Releases every device and host resource of the simulation. NULL is a no-op. */
LBIB_API void lbib_destroy(lbib_sim *sim);

/* Message of the last failing call (never NULL; "" when none). */
LBIB_API const char *lbib_last_error(const lbib_sim *sim);

/* Template (Sec. 5, template creation).  tid must equal the number of
 * templates created so far.  nodes_xyz: [n_nodes][3] FP64; tris: [n_tris][3]
 * node ids, each triangle ordered so that AB x AC points inside the object.
 * stretch: per-axis scale of the coordinates (NULL = 1,1,1).  Moduli of
 * Sec. 4: ks stretching, kb bending, kal local area, kag global area, kv
 * volume; nonlinear_ks selects the neo-Hookean kappa of the stretching force
 * (else kappa = 1).  Relaxed lengths, angles, areas, total area and volume
 * are measured on the stretched geometry.  Errors: LBIB_ERR_ID,
 * LBIB_ERR_MESH (open, non-manifold, inconsistent or outward-ordered),
 * LBIB_ERR_ARG (n_nodes > 5120 or < 4). */
LBIB_API lbib_status lbib_template_create(lbib_sim *sim, int tid, const double *nodes_xyz, int n_nodes,
                                 const int32_t *tris, int n_tris, const double stretch[3],
                                 double ks, double kb, double kal, double kag, double kv,
                                 int nonlinear_ks);

/* Topology and relaxed state the library built for a template.  Each output
 * may be NULL.  edges: [ne][2] with i < j, lexicographic order.  quads:
 * [ne][4] (a,b,c,d) for edge (b,c) = edges[e]; (a,b,c) is a cyclic order of
 * the triangle that runs b->c and (d,c,b) of the triangle that runs c->b.
 * L0, theta0: [ne]; S0: [n_tris]; globals: {S_g0, V0}.  *n_edges receives ne. */
LBIB_API lbib_status lbib_template_topology(const lbib_sim *sim, int tid, int32_t *edges, int32_t *quads,
                                   double *L0, double *theta0, double *S0, double *globals,
                                   int *n_edges);

/* Host-only mesh check (Sec. 5, mesh analysis and the template rules):
 * validates a mesh exactly as lbib_template_create does and, when it is
 * valid, returns the same topology and relaxed measures (outputs as for
 * lbib_template_topology; each may be NULL; edges/quads/L0/theta0 need
 * 3*n_tris/2 entries).  Needs no GPU.  On LBIB_ERR_MESH/LBIB_ERR_ARG the
 * reason is written to msg (NUL-terminated, at most msg_cap bytes). */
LBIB_API lbib_status lbib_mesh_check(const double *nodes_xyz, int n_nodes, const int32_t *tris, int n_tris,
                                     const double stretch[3], int32_t *edges, int32_t *quads, double *L0,
                                     double *theta0, double *S0, double *globals, int *n_edges, char *msg,
                                     int msg_cap);

/* Mesh orientation (Sec. 5, mesh analysis: orientation check, repair,
 * flip).  mode 0 reports in *changed how many triangles a repair would
 * turn (0: the mesh is consistently ordered with AB x AC pointing inside);
 * mode 1 repairs: the orientation is made consistent across shared edges
 * and then chosen so that the triangles point inside (positive enclosed
 * volume), which holds for concave meshes too; mode 2 flips every
 * triangle.  out [n_tris][3] receives the resulting triangles (NULL:
 * none).  Needs no GPU.  LBIB_ERR_MESH for a mesh that is not a closed
 * orientable 2-manifold, LBIB_ERR_ARG for bad arguments. */
LBIB_API lbib_status lbib_mesh_orient(const double *nodes_xyz, int n_nodes, const int32_t *tris, int n_tris, int mode,
                                      int32_t *out, int *changed);

/* Object (Sec. 5, adding of the object).  oid must equal the number of
 * objects added so far.  The template geometry is rotated by rotate[0]
 * about x, then rotate[1] about y, then rotate[2] about z (NULL = none),
 * then translated by origin.  mass: mass of every node (> 0).  Node
 * velocities start at 0. */
LBIB_API lbib_status lbib_object_add(lbib_sim *sim, int oid, int tid, const double origin[3],
                            const double rotate[3], double mass);

/* Soft-sphere repulsion between objects and against the walls (the
 * object-object and object-wall "soft-sphere" interactions of the example
 * in Sec. 6; the paper names the potential and its parameters only).
 * object[3] = (a, n, cutoff) for pairs of nodes of different objects:
 * nodes at distance r < cutoff push each other apart with a force of
 * magnitude a n r^-(n+1) (the potential a r^-n, offset 0).  wall[3] =
 * (a, n, cutoff) for a node at distance d < cutoff from a wall plane
 * (y = 1 or y = ny-1): pushed away with a n max(d, 1e-3)^-(n+1).  a = 0
 * switches a term off (the default).  Separations use the nearest periodic
 * image; the object cutoff must be below half of every periodic box length
 * (LBIB_ERR_ARG otherwise, and for a < 0, n <= 0 with a > 0, cutoff < 0).
 * Evaluated with the membrane forces, on the node positions of the step.
 * At most 32 close object pairs per object (sticky LBIB_ERR_NOMEM beyond). */
LBIB_API lbib_status lbib_set_repulsion(lbib_sim *sim, const double object[3], const double wall[3]);

/* Direction of the local-area force of template tid (Sec. 4 discusses two):
 * altitude = 0 (default) from the triangle's centroid to the vertex, 1
 * along the vertex's altitude (from the foot on the opposite edge to the
 * vertex).  The global-area force keeps the centroid direction.
 * LBIB_ERR_ID for an unknown template. */
LBIB_API lbib_status lbib_template_set_kal_direction(lbib_sim *sim, int tid, int altitude);

/* Obstacle cells (the rhomboid obstacles of the Sec. 6 channel): mask
 * [nz][ny][nx] bytes, non-zero = solid; n must be nx*ny*nz.  Entries in the
 * wall rows are ignored.  Obstacle cells hold no fluid and are treated like
 * the wall rows: a population streaming into one is reflected back into
 * its own cell (halfway bounce-back), velocity interpolation sees u = 0
 * there and force spread there is dropped (lbib_dropped_momentum).
 * Read-outs give u = 0 and rho = 0 at obstacle cells, and populations with
 * zero deviation; lbib_fluid_mass counts fluid cells only.  NULL removes
 * every obstacle.  Must precede lbib_fluid_init (LBIB_ERR_STATE). */
LBIB_API lbib_status lbib_set_solid(lbib_sim *sim, const uint8_t *mask, int64_t n);

/* Velocity inlet (the inflow of the Sec. 6 example, which sets the fluid
 * velocity of a plane of nodes before every step): at the start of every
 * step the populations of the cells x in [box[0], box[1]), y in
 * [box[2], box[3]) (lattice rows, wall rows included and skipped), z in
 * [box[4], box[5]) are replaced by the equilibrium at the cell's own
 * density and velocity u[3], then collide as usual.  The box is clipped to
 * the lattice; an empty box switches the inlet off (the default).
 * LBIB_ERR_ARG for |u| >= 0.3. */
LBIB_API lbib_status lbib_set_inlet(lbib_sim *sim, const int32_t box[6], const double u[3]);

/* External force on every node of an object (Sec. 5, object customization). */
LBIB_API lbib_status lbib_object_set_force(lbib_sim *sim, int oid, const double f[3]);

/* Replaces the node positions [n][3] of an object (Sec. 5, mesh-nodes; the
 * restart path).  n must equal the template's node count. */
LBIB_API lbib_status lbib_object_set_nodes(lbib_sim *sim, int oid, const double *xyz, int n);

/* Replaces the node velocities [n][3] of an object. */
LBIB_API lbib_status lbib_object_set_velocities(lbib_sim *sim, int oid, const double *v, int n);

/* Fluid at rest: h_i = 0 (f_i = w_i rho0), u = 0; clears the coupling force
 * field.  Required once before lbib_step. */
LBIB_API lbib_status lbib_fluid_init(lbib_sim *sim);

/* Advances n_steps full steps (Eq. lbequation, Eq. newton, Eq. dragforce,
 * Sec. 4): object measures and membrane forces, interpolation, drag,
 * spreading and node update, then fluid stream + collide with the body
 * force plus the spread force.  The membrane forces of step t+1 depend on
 * the node positions only and are computed while the fluid part of step t
 * runs.  Asynchronous on the simulation's stream; device-side errors
 * surface at the next synchronising call. */
LBIB_API lbib_status lbib_step(lbib_sim *sim, int n_steps);

/* Waits for the simulation's stream and returns the sticky device status. */
LBIB_API lbib_status lbib_sync(lbib_sim *sim);

/* Node positions and/or velocities ([n][3] FP64; either may be NULL) of
 * object oid, or of all objects in id order when oid = -1 (Sec. 5,
 * mesh-nodes output).  cap: capacity of each array in nodes. */
LBIB_API lbib_status lbib_read_nodes(lbib_sim *sim, int oid, double *xyz, double *v, int64_t cap);

/* Fluid velocity of the last collision, [3][nz][ny][nx] FP32, 0 on solid
 * rows (the velocity of Sec. 2 including half the applied force). */
LBIB_API lbib_status lbib_read_velocity(lbib_sim *sim, float *u, int64_t cap);

/* Fluid density [nz][ny][nx] FP32 (rho0 on solid rows). */
LBIB_API lbib_status lbib_read_density(lbib_sim *sim, float *rho, int64_t cap);

/* Force density the objects spread onto the fluid in the last step
 * (Sec. 2, the opposite drag distributed to the grid), [3][nz][ny][nx]
 * FP32, 0 where nothing was spread and on solid rows. */
LBIB_API lbib_status lbib_read_coupling_force(lbib_sim *sim, float *g, int64_t cap);

/* Restores the force field of lbib_read_coupling_force as the force spread
 * in the last step (part of a checkpoint: the velocity of the last
 * collision includes half of it).  Call after lbib_set_populations. */
LBIB_API lbib_status lbib_set_coupling_force(lbib_sim *sim, const float *g, int64_t n);

/* Populations as deviations h_i = f_i - w_i rho0, [19][nz][ny][nx] FP64 in
 * the direction order of lbib_lattice, 0 on solid rows.  Together with
 * lbib_set_populations this is the fluid checkpoint; for every storage
 * precision the round trip is exact. */
LBIB_API lbib_status lbib_read_populations(lbib_sim *sim, double *h, int64_t cap);
LBIB_API lbib_status lbib_set_populations(lbib_sim *sim, const double *h, int64_t n);

/* Object analysis (Sec. 5): out[14] = origin (mean of nodes) [3], bounds
 * xmin,xmax,ymin,ymax,zmin,zmax [6], volume, surface area, mean node
 * velocity [3].  Sums are error-free FP32 pairs on the GPU over positions
 * relative to the first node, finished in FP64. */
LBIB_API lbib_status lbib_object_analyze(lbib_sim *sim, int oid, double out[14]);

/* Batched forms for a per-step host loop (the paper's main loop sets inputs
 * and reads object properties every iteration, Sec. 6): set the external
 * force of every object from f [n_obj][3] (one host-to-device copy), and
 * analyse every object into out [n_obj][14] (one kernel, one copy back;
 * layout as lbib_object_analyze).  cap: capacity of out in objects. */
LBIB_API lbib_status lbib_objects_set_force(lbib_sim *sim, const double *f, int n_obj);
LBIB_API lbib_status lbib_objects_analyze(lbib_sim *sim, double *out, int64_t cap);

/* The same object analysis (Sec. 5) without waiting, for host loops that
 * keep the device busy (the result of step t is read while step t+1 runs;
 * the paper's main loop reads object properties every iteration, Sec. 6).
 * lbib_objects_analyze_async enqueues the analysis of the state after the
 * steps enqueued so far, and its copy with the status word into slot `slot`
 * (0 or 1) of a page-locked buffer the library owns, and returns at once.
 * lbib_objects_analyze_wait waits for that slot and writes it to out
 * [n_obj][14] (layout as lbib_object_analyze; cap: capacity in objects),
 * then reports the status word it carried as lbib_sync does.  A slot must be
 * waited for before it is enqueued again, and a wait needs an enqueued slot:
 * LBIB_ERR_STATE otherwise; LBIB_ERR_ARG for a slot other than 0 or 1. */
LBIB_API lbib_status lbib_objects_analyze_async(lbib_sim *sim, int slot);
LBIB_API lbib_status lbib_objects_analyze_wait(lbib_sim *sim, int slot, double *out, int64_t cap);

/* Per-phase timing with CUDA events on the streams the kernels run on.
 * While enabled (on != 0), lbib_step records events around each kernel of
 * every on-th step (on = 1: every step; the events themselves add a few
 * microseconds to a timed step, so a sampling period keeps the run close
 * to an untimed one).
 * lbib_profile_read waits for both streams and returns, since the last
 * enable: out[0] total ms and out[1] launches of the fluid kernel, out[2]
 * total ms and out[3] launches of the node-update kernel, out[4] total ms
 * and out[5] launches of the membrane-force kernel (which overlaps the
 * fluid kernel). */
LBIB_API lbib_status lbib_profile_enable(lbib_sim *sim, int on);
LBIB_API lbib_status lbib_profile_read(lbib_sim *sim, double out[6]);

/* Check of the device-side bounded waits (the warp-specialised fluid
 * kernel's pipeline waits give up after about 2 s, set the status the next
 * call reports as LBIB_ERR_TIMEOUT, and leave the context usable instead
 * of hanging).  Runs one such wait on the current device, on a barrier that
 * nothing completes (arrive = 0) or that its own thread completes first
 * (arrive = 1), bounded by `seconds`; *timed_out = 1 when the wait gave up.
 * Returns after the wait.  LBIB_ERR_ARG for a null output or seconds outside
 * (0, 10]; LBIB_ERR_CUDA when the device calls fail. */
LBIB_API lbib_status lbib_check_bounded_wait(double seconds, int arrive, int *timed_out);

/* Total fluid mass sum_cells sum_i f_i, an FP64 reduction on the GPU. */
LBIB_API lbib_status lbib_fluid_mass(lbib_sim *sim, double *mass);

/* The same total as lbib_fluid_mass without allocating anything (the paper
 * has no counterpart: its mass check is not part of the method).  For
 * callers that cannot allocate device memory: a serving process that has
 * admitted simulations up to its device-memory budget (an allocation there
 * can fail or evict), and host loops that must not call into the allocator
 * between steps.  Each thread block writes its FP64 partial to its own slot
 * of a static 1024-double scratch array of the library (one per device per
 * process); the host adds the slots in block order, so the result is
 * deterministic.  Limit: the reduction grid (4 blocks per SM) must fit the
 * 1024 slots, i.e. devices with up to 256 SMs; otherwise LBIB_ERR_ARG.
 * Calls that overlap in time on the same device (other threads, other
 * streams) race on the one scratch array and must be serialised by the
 * caller; the call waits for the simulation's stream before returning, so
 * calls made one after another are safe. */
LBIB_API lbib_status lbib_fluid_mass_noalloc(lbib_sim *sim, double *mass);

/* Counts (oif_info, Sec. 5).  out[8] = n_templates, n_objects, n_nodes,
 * fluid cells, steps taken, device bytes held, precision, and the fluid
 * kernel the step uses: 0 one cell per thread; 1 two x-adjacent cells per
 * thread (16-bit storage, even nx, no obstacles, no inlet); 2 the
 * warp-specialised two-cells kernel (see LBIB_TUNE_FLUID_KERNEL). */
LBIB_API lbib_status lbib_info(const lbib_sim *sim, int64_t out[8]);

/* Momentum the nodes would have given to solid corners (Sec. 2 spreading
 * restricted to fluid nodes), summed since lbib_fluid_init. */
LBIB_API lbib_status lbib_dropped_momentum(lbib_sim *sim, double out[3]);

/* The library's D3Q19 set: e [19][3], w [19] (NULL allowed).  Returns 19. */
LBIB_API int lbib_lattice(int32_t *e, double *w);

/* Device bytes a simulation of this size would hold (fluid + coupling
 * fields + n_nodes nodes + n_tri_total template triangles), for admission
 * control. */
LBIB_API int64_t lbib_footprint_bytes(const lbib_fluid_params *params, int64_t n_nodes, int64_t n_tri_total);

/* Advances n simulations (same device) by n_steps each (batching; the
 * paper steps one system at a time).  Each kernel of the step is launched
 * once for all n simulations over a flat work list, and chunks of steps are
 * replayed from a captured CUDA graph; the work is ordered on the stream of
 * sims[0] (the others' pending work is waited for first).  Each
 * simulation's result equals that of lbib_step on it alone up to the order
 * of floating-point atomics.  Returns after the steps have completed. */
LBIB_API lbib_status lbib_batch_step(lbib_sim *const *sims, int n, int n_steps);

/* Continuous-batching scheduler for many simulations on one device (no
 * counterpart in the paper, which runs one system per process: a serving
 * layer above lbib_batch_step).
 *   lbib_server_create: budget_bytes caps the device bytes the resident
 *     simulations hold together (lbib_info out[5]); max_resident caps their
 *     number; chunk_steps (>= 1) caps the steps of one advance.
 *   lbib_server_admit: makes sim resident to run n_steps (>= 1) more
 *     steps; tag is returned when it finishes.  LBIB_ERR_NOMEM when it does
 *     not fit the budget or no slot is free now (nothing changes; admit it
 *     after a retirement); LBIB_ERR_ARG for a sim already resident.  The
 *     caller keeps ownership of sim and must neither step nor destroy it
 *     while it is resident.
 *   lbib_server_advance: advances every resident simulation by
 *     min(chunk_steps, fewest remaining steps) steps in one lbib_batch_step
 *     and retires those that have no steps left, writing their tags to
 *     done[0 .. *n_done - 1] (at most cap; the rest retire on the next
 *     call, which then advances nothing).  *n_done = 0 with nothing resident.
 *     A simulation whose step fails (its sticky status, see lbib_sync) is
 *     retired at once with its tag in done; the others are unaffected.
 *   lbib_server_stats: out[4] = resident simulations, resident bytes,
 *     advances made, lattice updates done (sum of cells x steps).
 * The scheduler holds no device memory. */
typedef struct lbib_server lbib_server;
LBIB_API lbib_status lbib_server_create(int64_t budget_bytes, int max_resident, int chunk_steps, lbib_server **out);
LBIB_API void lbib_server_destroy(lbib_server *srv);
LBIB_API lbib_status lbib_server_admit(lbib_server *srv, lbib_sim *sim, int64_t n_steps, int64_t tag);
LBIB_API lbib_status lbib_server_advance(lbib_server *srv, int64_t *done, int cap, int *n_done);
LBIB_API lbib_status lbib_server_stats(const lbib_server *srv, int64_t out[4]);

/* Launch-shape knobs, chosen by the autotuner of the Python package or set
 * by hand.  LBIB_TUNE_IB_CLUSTER: thread blocks per object in the
 * membrane-force kernel (1..8, default 1).  LBIB_TUNE_OVERLAP: 1 (default)
 * computes the membrane forces of step t+1 on the library's second stream
 * while the fluid part of step t runs; 0 computes them on the simulation's
 * stream at the start of each step.  LBIB_TUNE_MEMBRANE_CLUSTERS: number of
 * clusters of the membrane-force kernel, each looping over the objects
 * (0, default: one cluster per object; a small grid leaves most SMs to the
 * fluid kernel running beside it).  LBIB_TUNE_MEMBRANE_THREADS: threads per
 * block of the membrane-force kernel (a multiple of 32 in [32, 256],
 * default 192: fewer threads leave more of each SM to the fluid kernel
 * running beside it).  LBIB_TUNE_FLUID_KERNEL (16-bit storage): 0
 * (default) and 1 the two-cells-per-thread kernel (where nx is even and
 * there are no obstacles or inlet), 2 the warp-specialised two-cells kernel
 * (a producer warp streams the populations through shared memory with bulk
 * asynchronous copies; needs nx a multiple of 8 with a row segment of at
 * least 64 cells, and no obstacles or inlet, else the step uses value 1;
 * slower than value 1 on a GB300, kept for comparison; lbib_batch_step runs
 * value 1 instead), 3 one cell per thread; FP32 storage ignores it.
 * LBIB_TUNE_NODE_THREADS: nodes per block of the node-update kernel (32,
 * 64, 128 or 256, default 256; lbib_batch_step takes the first
 * simulation's).  LBIB_TUNE_MEMBRANE_GROUP: objects per block of the
 * membrane-force kernel (1..15, default 1); above 1 each object gets
 * LBIB_TUNE_MEMBRANE_THREADS threads of a block of group x threads threads
 * (at most 1024) and the cluster knobs do not apply; the step takes as
 * many objects per block as fit (threads and shared memory for the largest
 * template), at most the knob's value.
 * lbib_batch_step takes the first simulation's; it runs the objects within
 * a factor 2 of the largest in one launch and the others beside it in a
 * second (each with shared-memory slices sized for its own largest
 * object), with as many objects per block as fit, and keeps one object per
 * cluster when a single size class does not fit more than one.  LBIB_TUNE_EARLY_LAUNCH: 1 lets each node-update and
 * fluid kernel of lbib_step after the first start while the kernel before
 * it finishes (programmatic dependent launch: the early part reads only data
 * that kernel does not write, and waits for it before the rest), 0 (default)
 * launches them one after the other; lbib_batch_step ignores it.
 * Results do not depend on the knobs beyond the order of
 * floating-point atomics (the three 16-bit kernels give identical
 * populations).  LBIB_ERR_ARG for an unknown key or an out-of-range value. */
typedef enum {
    LBIB_TUNE_IB_CLUSTER = 0,
    LBIB_TUNE_OVERLAP = 1,
    LBIB_TUNE_MEMBRANE_CLUSTERS = 2,
    LBIB_TUNE_MEMBRANE_THREADS = 3,
    LBIB_TUNE_FLUID_KERNEL = 4,
    LBIB_TUNE_NODE_THREADS = 5,
    LBIB_TUNE_MEMBRANE_GROUP = 6,
    LBIB_TUNE_EARLY_LAUNCH = 7
} lbib_tune_key;
LBIB_API lbib_status lbib_set_tuning(lbib_sim *sim, int key, int value);
LBIB_API lbib_status lbib_get_tuning(const lbib_sim *sim, int key, int *value);

/* Version of the ABI (incremented on incompatible change). */
LBIB_API int lbib_abi_version(void);

#ifdef __cplusplus
}
#endif

#endif /* LBIB_H */
