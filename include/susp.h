/*
 * susp.h — C ABI of the GB300 (sm_103a) sheared-suspension step.
 *
 * Method: Pradipto & Hayakawa, "Simulation of dense non-Brownian suspensions
 * with the lattice Boltzmann method: shear jammed and fragile states"
 * (arXiv:1904.02929).  One step is
 *   - the D3Q19 lattice-Boltzmann collide-stream update (Appendix A, Eq. 3-5;
 *     BGK, which equals the paper's linear operator when every non-conserved
 *     mode relaxes fully, i.e. tau = 1, or that operator itself with separate
 *     shear and bulk relaxation times and the ghost modes removed),
 *   - moving-particle bounce-back and link momentum exchange (Eq. 6-10),
 *   - a Lees-Edwards sheared boundary in y (x flow, z vorticity), driven by a
 *     constant rate or the oscillatory strain of Eq. 16,
 *   - per particle: frictional contacts with tangential-spring history and
 *     Coulomb slip (Eq. 11, 11t), double-layer repulsion (Eq. 13), the pairwise
 *     lubrication correction (Appendix A) and rigid-body integration (Eq. 1),
 *   - stress sums (Eq. 12, 14, 15, with the lubrication stresslets), angular
 *     contact histograms (Eq. 19-23) for the angular stress of Eq. 26 / 27,
 *     and the storage and loss moduli of Eq. 17, 18.
 * Shear can also be applied as in the paper by bumpy walls: spheres flagged
 * as driven keep their prescribed velocity (Sec. 3).
 *
 * Memory: the caller owns one device workspace of susp_workspace_bytes()
 * bytes (for example a torch uint8 tensor).  The library never allocates
 * device memory.  All work is enqueued on the caller's CUDA stream.
 *
 * Threading: a handle is used from one host thread at a time.  Calls that
 * return host data (susp_stress, susp_get_*, susp_save) synchronise the
 * handle's stream; susp_step is asynchronous.
 *
 * Populations exchanged with the host are FP64, layout [19][nz][ny][nx]
 * (x fastest), in this velocity order (c_x, c_y, c_z):
 *   0 ( 0, 0, 0)   1 ( 1, 0, 0)   2 (-1, 0, 0)   3 ( 0, 1, 0)   4 ( 0,-1, 0)
 *   5 ( 0, 0, 1)   6 ( 0, 0,-1)   7 ( 1, 1, 0)   8 (-1,-1, 0)   9 ( 1,-1, 0)
 *  10 (-1, 1, 0)  11 ( 1, 0, 1)  12 (-1, 0,-1)  13 ( 1, 0,-1)  14 (-1, 0, 1)
 *  15 ( 0, 1, 1)  16 ( 0,-1,-1)  17 ( 0, 1,-1)  18 ( 0,-1, 1)
 * and hold post-collision values n*(r, c_q, t).  Values at solid nodes
 * (inside a particle's mapped radius) are undefined.
 */
#ifndef SUSP_H
#define SUSP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SUSP_OK = 0,
  SUSP_EINVAL = -1,     /* bad argument or parameter                             */
  SUSP_ENOMEM = -2,     /* workspace too small, or a fixed-capacity table full   */
  SUSP_ECUDA = -3,      /* a CUDA call failed (message in susp_last_error)       */
  SUSP_EOVERLAP = -4,   /* two mapped spheres claimed one node (Appendix A (i))  */
  SUSP_EUNSTABLE = -5,  /* non-positive density or a particle faster than 0.5/step */
  SUSP_ETIMEOUT = -6,   /* reserved: a bounded device wait gave up               */
  SUSP_ESTATE = -7      /* call not valid in the handle's state                  */
} susp_status;

typedef enum {
  SUSP_FP64 = 0,        /* populations stored and computed in FP64               */
  SUSP_FP32 = 1,        /* stored and computed in FP32                           */
  SUSP_FP16_DEV = 2,    /* stored as FP16 deviations n - C^q rho0, FP32 compute  */
  SUSP_BF16_DEV = 3     /* stored as BF16 deviations n - C^q rho0, FP32 compute  */
} susp_precision;

typedef struct {
  int nx, ny, nz;           /* lattice; x flow, y gradient (Lees-Edwards), z vorticity; each >= 4,
                               nx, ny <= 2047, nz <= 1023 and nx ny nz < 2^27 per box (element
                               indices stay 32-bit); larger problems run as many boxes           */
  double tau;               /* BGK relaxation time (> 0.5); eta0 = rho0 (tau - 1/2) / 3            */
  double rho0;              /* reference fluid density, used in Eq. 7                             */
  int n;                    /* number of particles (>= 0)                                          */
  const double *radius;     /* [n] contact radii (host; copied)                                     */
  const double *pos;        /* [3n] centres, x y z per particle (host; copied; finite; wrapped into the box) */
  const double *vel;        /* [3n] initial velocities or NULL (host; copied)                       */
  const double *omega;      /* [3n] initial angular velocities or NULL (host; copied)               */
  double rho_p;             /* particle density; m = rho_p 4/3 pi a^3, I = 2/5 m a^2                */
  double mu;                /* Coulomb friction coefficient (Sec. 2)                                */
  double kn;                /* normal spring constant (Sec. 2)                                      */
  double kt_ratio;          /* kt / kn (the paper uses 0.2)                                         */
  double eta_n;             /* normal dashpot; < 0 selects sqrt(m0 kn) with m0 the mean mass         */
  double F0, debye;         /* double-layer force F0 exp(-h / debye) (Eq. 13); F0 = 0 disables      */
  double lub_delta;         /* roughness length delta of the lubrication functions                  */
  double lub_cut;           /* lubrication correction for gaps below lub_cut; 0 disables            */
  double a_map_ratio;       /* mapped radius / contact radius (0.95 in Appendix A)                  */
  int dem_substeps;         /* particle sub-steps per lattice step; 0 = automatic                   */
  int quasi2d;              /* monolayer: U_z = 0, Omega_x = Omega_y = 0 (Sec. 4.1)                 */
  int move_particles;       /* 0 = particles held at their given velocities                         */
  int nbins;                /* angular histogram bins over [0, pi) (Eq. 19-23); <= 0 selects 36    */
  double body_force[3];     /* uniform force density on the fluid (0 for shear runs)                */
  susp_precision prec;      /* population storage                                                   */
  int collision;            /* 0: BGK, every non-conserved mode relaxed by 1/tau; 1: Ladd's linear
                               operator (Eq. 5 by its eigenvalues): the traceless non-equilibrium
                               stress relaxed by -1/tau, its trace by -1/tau_bulk, ghost modes
                               removed.  Both coincide at tau = tau_bulk = 1                      */
  double tau_bulk;          /* Ladd: bulk relaxation time (> 0.5); <= 0 selects tau                */
  const int *driven;        /* [n] or NULL (host; copied): nonzero marks a driven sphere, which keeps
                               its given velocity and spin whatever the forces (the wall spheres of
                               the bumpy walls that shear the suspension in Sec. 3); it still takes
                               part in contacts, lubrication and bounce-back                      */
} susp_params;

typedef struct {
  int kind;                 /* 0: constant rate; 1: oscillatory strain, Eq. 16                     */
  double rate;              /* kind 0: shear rate (lattice units)                                   */
  double gamma0;            /* kind 1: strain amplitude                                             */
  double omega;             /* kind 1: angular frequency (per lattice step)                         */
  double theta;             /* kind 1: initial phase Theta                                          */
} susp_shear;

typedef enum {
  SUSP_STRESS_VISCOUS = 0,  /* fluid viscous stress + particle stresslet (sigma^h, Appendix A)      */
  SUSP_STRESS_CONTACT = 1,  /* contact virial, Eq. 12                                               */
  SUSP_STRESS_REPULSIVE = 2,/* double-layer virial, Eq. 14                                          */
  SUSP_STRESS_TOTAL = 3,    /* Eq. 15, with the lubrication stresslets                              */
  SUSP_STRESS_ANGULAR = 4,  /* Eq. 26 (quasi2d) or Eq. 27 from the contact histogram                */
  SUSP_STRESS_LUBRICATION = 5 /* the pairs' lubrication stresslets (Appendix A, G and H blocks, the
                               correction form of the lubrication forces), sampled with the virials */
} susp_stress_kind;

typedef struct susp susp;

/* Bytes of device workspace needed for these parameters; 0 if they are invalid. */
size_t susp_workspace_bytes(const susp_params *p);

/* Create a box.  dev_workspace: device pointer to >= susp_workspace_bytes(p)
 * bytes, 256-byte aligned, owned by the caller and kept alive until
 * susp_destroy.  cuda_stream: a cudaStream_t (NULL = legacy default stream).
 * Initial fluid at rest (n = C^q rho0); nodes inside a_map_ratio * radius are
 * solid.  Synchronises the stream.  Errors: SUSP_EINVAL, SUSP_ENOMEM,
 * SUSP_EOVERLAP, SUSP_ECUDA; *out is NULL on error. */
susp_status susp_create(const susp_params *p, void *dev_workspace, size_t bytes,
                        void *cuda_stream, susp **out);

/* Advance nsteps lattice steps under the shear protocol *sh.  The step
 * counter t is absolute and continues across calls; the Lees-Edwards offset
 * is the compensated sum of the per-step increments L_y (gamma(t+1) - gamma(t)),
 * so a new protocol (e.g. the amplitude reduction of Sec. 4.1) continues it
 * without a jump.  Asynchronous; device-side errors surface at the next
 * synchronising call.  Errors: SUSP_EINVAL. */
susp_status susp_step(susp *h, int nsteps, const susp_shear *sh);

/* Time-averaged stress since the last reset, row-major out[9].  If hist is
 * non-NULL and nbins equals the handle's bin count, hist[3*nbins] receives
 * (count, sum F_nor, sum F_tan) per angular bin.  Synchronises; returns the
 * device error status (SUSP_EOVERLAP, SUSP_EUNSTABLE, SUSP_ENOMEM) if set. */
susp_status susp_stress(susp *h, susp_stress_kind kind, double out[9], double *hist, int nbins);
/* Storage and loss moduli of the oscillatory protocol (Eq. 17, 18):
 *   G' = -(omega/pi) int_0^{2 pi/omega} sigma_xy(t) cos(omega t + Theta) dt / gamma0,
 *   G'' = (omega/pi) int_0^{2 pi/omega} sigma_xy(t) sin(omega t + Theta) dt / gamma0,
 * from the total shear stress sigma_xy (as SUSP_STRESS_TOTAL) of every step
 * since the last susp_stress_reset, each step's stress taken at the
 * midpoint phase omega (t + 1/2) + Theta (the step shears by
 * gamma(t+1) - gamma(t)); the window should hold a whole number of periods.
 * gamma0, omega and Theta are those of the box's current protocol.
 * Synchronises.  Errors: SUSP_EINVAL (NULL), SUSP_ESTATE (no oscillatory
 * protocol with gamma0 > 0), a device status, SUSP_ECUDA. */
susp_status susp_moduli(susp *h, double *Gp, double *Gpp);

/* Zero the stress and histogram accumulators (asynchronous). */
susp_status susp_stress_reset(susp *h);

/* Particle state to host arrays [3n] (any may be NULL).  Synchronises. */
susp_status susp_get_particles(susp *h, double *pos, double *vel, double *omega);

/* Hydrodynamic link force and torque [3n] that the next step applies. Synchronises. */
susp_status susp_get_hydro(susp *h, double *force, double *torque);

/* A step's results in one transfer (no counterpart in the paper): the device
 * gathers the error word, the stress sums and sample counters, the angular
 * histogram and the particles' centres, velocities and spins into a block of
 * susp_results_bytes(h) bytes in the workspace and copies it to host_buf
 * with one copy on the handle's stream.  async = 0: synchronises and returns
 * the device status as susp_get_particles does.  async = 1: only enqueues
 * the gather and the copy and returns SUSP_OK; host_buf must then be pinned
 * host memory, and holds the block once the stream has passed the copy (the
 * caller waits on an event recorded after the call, or synchronises); a
 * later call may reuse host_buf only after that.  The block's status and
 * contents are read on the host by susp_results_particles and
 * susp_results_stress, which touch no device memory: the centres,
 * velocities and spins (any may be NULL) and the time-averaged stress of
 * one kind with the histogram, exactly as susp_get_particles and
 * susp_stress give them at that point of the stream.  Both return the
 * block's device status (SUSP_EOVERLAP, SUSP_EUNSTABLE, ...).  Errors:
 * SUSP_EINVAL (NULL argument, bytes below susp_results_bytes, async not 0 or
 * 1), SUSP_ECUDA. */
size_t susp_results_bytes(susp *h);
susp_status susp_read_results(susp *h, void *host_buf, size_t bytes, int async);
susp_status susp_results_particles(susp *h, const void *buf, double *pos, double *vel, double *omega);
susp_status susp_results_stress(susp *h, const void *buf, susp_stress_kind kind, double out[9], double *hist,
                                int nbins);

/* Populations to / from FP64 host arrays [19*nx*ny*nz] in the layout above.
 * Set converts to the storage precision and recomputes the link forces.
 * Both synchronise. */
susp_status susp_get_populations(susp *h, double *f);
susp_status susp_set_populations(susp *h, const double *f);

/* Node owner map [nx*ny*nz] (-1 fluid, else particle index). Synchronises. */
susp_status susp_get_owner(susp *h, int32_t *owner);

/* Step counter and Lees-Edwards offset (in [0, nx)).  Synchronises. */
susp_status susp_get_time(susp *h, int64_t *t, double *delta);

/* Run facts: particle sub-steps per lattice step, kernels launched per step,
 * whether the pair search is brute force (small boxes), lattice nodes,
 * workspace bytes, and whether the collide-stream runs beside the particle
 * kernel (overlap, see susp_set_overlap; for a box attached to a batch, the
 * batch's). */
typedef struct {
  int dem_substeps;
  int launches_per_step;
  int brute_force_pairs;
  long long ncell;
  size_t workspace_bytes;
  int overlap;
} susp_info;
susp_status susp_get_info(susp *h, susp_info *info);

/* Checkpoint and resume.  susp_save writes the box's whole state (device
 * workspace plus the shear protocol in force) to host_buf; with host_buf NULL
 * it only sets *bytes to the size needed.  susp_load restores a checkpoint
 * into a handle created with the same parameters (lattice, particle count,
 * precision; otherwise SUSP_EINVAL); stepping then continues exactly where
 * the saved run was.  Both synchronise.  The format is this library's own
 * (a header and the raw workspace, not portable across builds). */
susp_status susp_save(susp *h, void *host_buf, size_t *bytes);
susp_status susp_load(susp *h, const void *host_buf, size_t bytes);

/* Instrumentation (no counterpart in the paper): when enabled, each step
 * records CUDA events on the handle's stream at its stage boundaries (at
 * most 4096 steps per window).  susp_profile_read synchronises and
 * returns the summed launch time in ms and the number of launches, then
 * starts a new window. */
susp_status susp_profile(susp *h, int enable);
susp_status susp_profile_read(susp *h, double *ms_total, int *launches);
/* The same window split by stage: ms[5] receives the summed times of (0) the
 * collide-stream (which also writes the next step's Lees-Edwards plane
 * moments), (1) the particle sub-steps with their cell list, (2) the stress /
 * protocol finalisation (0 when particles move: the particle kernel then
 * ends with it and its time is in (1)), (3) the node-map update (uncover,
 * cover) and (4) the boundary links; *steps the number of profiled steps.
 * With the overlapped step (susp_set_overlap) (0) is the collide-stream's
 * time beside the particle kernel, (1) the particle time not hidden behind
 * it and (2) the separate finalisation; the stages still add up to the
 * step.  Synchronises and
 * starts a new window (it shares the window with susp_profile_read). */
susp_status susp_profile_stages(susp *h, double *ms, int *steps);

/* Allocation-free fluid step.  The paper has no counterpart: this entry point
 * exists for callers that cannot allocate device memory or hand the library a
 * workspace at all, e.g. code running inside a host framework that owns every
 * device allocation, or a loop that must not touch the allocator.  It advances
 * a particle-free FP32 box by one step -- the same collide-stream and
 * Lees-Edwards planes as susp_step -- from f_in to f_out (device pointers,
 * [19][nz][ny][nx] post-collision populations, caller-owned; overlapping
 * f_in and f_out ranges are rejected with SUSP_EINVAL),
 * with Lees-Edwards offset delta and image velocity u_le for this step, and
 * writes the step's viscous stress (3 x 3, row-major, per unit volume) to the
 * device pointer visc_out.  Its scratch (plane moments and block partials)
 * is a fixed static device array of about 2.2 MiB inside the library, held by
 * every GPU that loads the library until the process exits; boxes with
 * nx * nz > 65536 are rejected with SUSP_EINVAL.  The first call on a device
 * looks up that array's address (cudaGetSymbolAddress), so make the first
 * call on each device before any stream capture; the address is kept per
 * device with the ID of the CUDA context it belongs to and looked up again
 * when another context is current (after a device reset, for instance).  All
 * calls share the array:
 * calls that overlap on the GPU race.  Nothing is allocated; asynchronous on
 * cuda_stream.  Errors: SUSP_EINVAL, SUSP_ECUDA. */
susp_status susp_fluid_step_noalloc(int nx, int ny, int nz, double tau, double delta, double u_le,
                                    const float *f_in, float *f_out, double *visc_out,
                                    void *cuda_stream);

/* Replay a captured CUDA graph of the step (default on; no counterpart in the
 * paper).  susp_step captures the step once, on the handle's stream (which
 * must not be the legacy default stream), and replays it every step: the
 * population buffer and spring-table parities follow from the step counter on
 * the device, so one graph serves every step.  If capture fails the step runs
 * as plain launches.  Disabling drops the captured graph.  Synchronises. */
susp_status susp_set_graphs(susp *h, int enable);

/* Launch-shape tuner (no counterpart in the paper; the batched step takes
 * its tile shapes from it).  Times the collide-stream on this machine for each
 * tile height of 4, 8 and 16 rows of 32 nodes and each count of resident
 * blocks per SM that the occupancy allows, and for FP32 / FP16 / BF16
 * storage also the staged kernel (tiles of 128 x 4 nodes whose source rows
 * tensor copies bring into shared memory; see susp_set_launch_shape) at each
 * resident block count (three launches per shape after a
 * warm-up, CUDA events on the handle's stream), keeps the fastest, and
 * reports it: *tile_rows, *blocks_per_sm, and *us, the average launch time
 * of that shape in microseconds (any of the three may be NULL).  Call it
 * between steps: the trial launches only rewrite the population buffer that
 * the next step overwrites, and the current step's viscous-stress sums are
 * cleared after them, so the following steps give the untuned results up to
 * the summation order of the viscous-stress block sums (populations and
 * particles are bitwise the same).  The choice holds for later steps and
 * across susp_save / susp_load.  Synchronises; drops the captured graph.  A
 * box attached to a batch returns SUSP_ESTATE (tune the batch).  Errors:
 * SUSP_EINVAL, SUSP_ESTATE, SUSP_ECUDA. */
susp_status susp_tune(susp *h, int *tile_rows, int *blocks_per_sm, double *us);

/* The collide-stream launch shape in use, or set explicitly (no counterpart
 * in the paper).  tile_rows: 4, 8 or 16 rows of 32 nodes per tile;
 * blocks_per_sm: resident blocks per SM of the persistent grid (capped by
 * the occupancy); staged: 1 for the kernel whose per-tile source rows of the
 * 19 populations are brought into shared memory by tensor copies (FP32,
 * FP16 and BF16 storage; tiles of 128 x 4 nodes, given as tile_rows = 4; a
 * box whose x rows are not a multiple of 16 bytes pulls from global memory
 * in that kernel), 0 for direct pulls.  Both kernels give the same populations bit for bit; the
 * viscous-stress sums differ in summation order only.  Set synchronises and
 * drops the captured graph; a box attached to a batch returns SUSP_ESTATE
 * (set the batch's).  Get reports the shape of the batch a box is attached
 * to.  Errors: SUSP_EINVAL (bad value, NULL handle), SUSP_ESTATE, SUSP_ECUDA. */
susp_status susp_set_launch_shape(susp *h, int tile_rows, int blocks_per_sm, int staged);
susp_status susp_get_launch_shape(susp *h, int *tile_rows, int *blocks_per_sm, int *staged);

/* Overlapped step (no counterpart in the paper): within a lattice step the
 * collide-stream depends neither on the particle sub-steps nor on their
 * results (it reads the compute-type particle copy of step t; the particle
 * kernel then writes the next step's copy into a second buffer, which the
 * finalisation copies over), so it can run on a second stream beside them,
 * with the step's finalisation after both.  enable = 1
 * asks for it and sets the collide-stream grid to one block per SM; it takes
 * effect when the particles move and the particle kernel's grid fits one
 * block per SM beside it (susp_info.overlap tells).  susp_tune does not
 * choose it and turns it off: on the 96^3 suspension (N = 882, FP32) the
 * collide-stream beside the particle kernel took 127 us against 47 us alone
 * and the step 0.232 ms against 0.193 ms in sequence.  Populations,
 * particles and stresses are those of the
 * sequential step up to the summation order of the link forces.  Set
 * synchronises and drops the captured graph.  Errors: SUSP_EINVAL, SUSP_ESTATE
 * (attached to a batch: set the batch's), SUSP_ECUDA. */
susp_status susp_set_overlap(susp *h, int enable);

/* Release the handle (not the caller's workspace). */
void susp_destroy(susp *h);

/* ------------------------------------------------------------------ batches
 * Many independent boxes stepped in lockstep by one launch sequence (no
 * counterpart in the paper, which runs one box at a time; this serves
 * parameter sweeps such as the volume-fraction and amplitude scans of
 * Sec. 4).  Every kernel of the step covers all attached boxes: the
 * collide-stream is one persistent grid over the tiles of every box, the
 * particle sub-steps one cooperative grid over every particle.  Each box keeps
 * its own parameters, protocol, step counter and workspace, and the results
 * of a box are the same whether it is stepped alone or in a batch.
 *
 * Storage: the caller owns a device workspace of
 * susp_batch_workspace_bytes(max_boxes) bytes (256-byte aligned) for the
 * box descriptors, and a stream that is not the legacy default stream.
 * Attach: the box must share the batch's storage precision and have a shear
 * protocol set (susp_step with nsteps = 0); its stream is synchronised and
 * from then on its work runs on the batch's stream.  While attached, susp_step
 * with nsteps > 0 returns SUSP_ESTATE; the read-back calls work as usual.
 * Attach and detach synchronise the batch's stream and drop its captured
 * graph, so continuous batching (boxes joining and leaving between steps)
 * costs one capture per membership change.  susp_destroy of an attached box
 * detaches it first.  Errors: SUSP_EINVAL, SUSP_ENOMEM (batch full),
 * SUSP_ESTATE, SUSP_ECUDA. */
typedef struct susp_batch susp_batch;
size_t susp_batch_workspace_bytes(int max_boxes);
susp_status susp_batch_create(int max_boxes, void *dev_workspace, size_t bytes, void *cuda_stream,
                              susp_batch **out);
susp_status susp_batch_attach(susp_batch *b, susp *h);
susp_status susp_batch_detach(susp_batch *b, susp *h);
int susp_batch_size(const susp_batch *b);
/* Advance every attached box by nsteps steps under its own protocol (asynchronous). */
susp_status susp_batch_step(susp_batch *b, int nsteps);
/* As susp_tune, over every attached box at once (one shape for the batch's
 * persistent collide-stream grid); the choice holds across attach and
 * detach.  SUSP_ESTATE when no box is attached. */
susp_status susp_batch_tune(susp_batch *b, int *tile_rows, int *blocks_per_sm, double *us);
/* As susp_set_launch_shape / susp_get_launch_shape, for the batch. */
susp_status susp_batch_set_launch_shape(susp_batch *b, int tile_rows, int blocks_per_sm, int staged);
susp_status susp_batch_get_launch_shape(susp_batch *b, int *tile_rows, int *blocks_per_sm, int *staged);
/* As susp_set_overlap, for the batch; *overlap (may be NULL) tells whether
 * it is in effect. */
susp_status susp_batch_set_overlap(susp_batch *b, int enable);
susp_status susp_batch_get_overlap(susp_batch *b, int *overlap);
/* As susp_profile / susp_profile_read, for the batch's collide-stream launch. */
susp_status susp_batch_profile(susp_batch *b, int enable);
susp_status susp_batch_profile_read(susp_batch *b, double *ms_total, int *launches);
susp_status susp_batch_profile_stages(susp_batch *b, double *ms, int *steps);
/* Device error status of every attached box, in attach order (the order
 * detaching keeps), into status[0 .. susp_batch_size(b)); n is the array's
 * length.  One gather launch and one copy for the whole batch; synchronises
 * the batch's stream.  A box whose status is not SUSP_OK keeps stepping
 * safely (its kernels stay inside its own buffers) but its results are
 * invalid; a server retires it.  Errors: SUSP_EINVAL, SUSP_ECUDA. */
susp_status susp_batch_errors(susp_batch *b, int *status, int n);
/* Release the batch (detaching its boxes), not the caller's workspace. */
void susp_batch_destroy(susp_batch *b);

/* Message of the last failing call on this thread (never NULL). */
const char *susp_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
