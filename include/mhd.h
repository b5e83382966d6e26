/*
 * mhd.h -- C ABI of the GB300 (sm_103a) recursive regularised lattice
 * Boltzmann solver for 2-D incompressible resistive MHD.
 *
 * Method: De Rosis, "Recursive regularised lattice Boltzmann method for
 * magnetohydrodynamics".  Fluid: D2Q9 populations f_i, fourth-order Hermite
 * equilibrium carrying the Maxwell stress (Eq. feq_4th), recursive regularised
 * collision (Section "Recursive regularised lattice Boltzmann method", tasks
 * 1-5 of "Algorithm of computation").  Magnetic field: D2Q5 vector populations
 * g_j relaxed by BGK towards Dellar's induction equilibrium (Eq. collide_g).
 *
 * Conventions for every call:
 *  - Lattice units.  Node n = y*nx + x, x fastest.  Host arrays are FP64,
 *    caller-owned, read or written only during the call.
 *  - nu = (tau_f - 1/2)/3 and eta = (tau_m - 1/2)/3 (cs^2 = 1/3 on both
 *    lattices; the paper's transport relation prints the bracket without the
 *    cs^2 factor).
 *  - The library owns all device memory of a lattice.  No exception crosses
 *    the ABI; every call returns an mhd_status and, on failure, leaves a
 *    message for mhd_last_error() in the calling thread.  A lattice must not
 *    be used from two host threads at once.
 *  - Work is queued on the CUDA stream given at creation (NULL: the legacy
 *    default stream).  mhd_advance returns without waiting; every mhd_get_*
 *    call waits for the stream.
 *  - The device buffer holds post-collision populations f*(t) (pull scheme:
 *    one kernel per step gathers f*(t-1) from the neighbours, collides, and
 *    writes f*(t)).  rho, rho u and b are collision invariants, so fields read
 *    back are the moments of the state at time t.
 */
#ifndef MHD_LBM_H
#define MHD_LBM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mhd_lattice mhd_lattice; /* opaque single lattice */
typedef struct mhd_batch mhd_batch;     /* opaque ensemble of independent lattices */

typedef enum {
    MHD_OK = 0,
    MHD_EINVAL = 1,    /* bad argument (NULL pointer, size, tau <= 1/2, ...) */
    MHD_ENOMEM = 2,    /* device or host allocation failed */
    MHD_ECUDA = 3,     /* a CUDA runtime call failed; see mhd_last_error() */
    MHD_EUNSTABLE = 4, /* a diagnostic came out non-finite (the run blew up) */
    MHD_ESTATE = 5     /* call not valid in the current state (e.g. no fields set) */
} mhd_status;

typedef enum {
    MHD_FP64 = 0,  /* populations stored as FP64 deviations, FP64 arithmetic */
    MHD_FP32 = 1,  /* FP32 deviations f_i - w_i rho0 (g unshifted), FP32 arithmetic */
    MHD_FP16S = 2  /* IEEE FP16 of 2^12 (f_i - w_i rho0) and 2^12 g, FP32 arithmetic */
} mhd_precision;

/* Boundary of an axis.  MHD_WALL: half-way bounce-back.  MHD_HALO (bc_y
 * only): the lattice is one slab of a periodic lattice split into row slabs
 * (a domain decomposition of the y axis, e.g. one slab per GPU); it keeps
 * one ghost row below row 0 and one above row ny-1, which
 * mhd_slab_exchange fills from the neighbouring slabs after every step.
 * Two-buffer streaming only, no closure. */
typedef enum { MHD_PERIODIC = 0, MHD_WALL = 1, MHD_HALO = 2 } mhd_bc;

typedef enum {
    MHD_RR = 0, /* recursive regularised (the paper's scheme) */
    MHD_BGK = 1 /* plain BGK fluid collision (Eq. collide_f), for comparison */
} mhd_collision;

/* Storage of the state.  MHD_TWO_BUFFERS: the pull scheme reads one buffer
 * and writes the other.  MHD_IN_PLACE: one buffer, updated in place by a
 * pair of alternating kernels (the "AA" access pattern: the first streams
 * and collides and writes each population back into the cell it came from,
 * the second collides locally); half the device memory for the same bytes
 * moved per step, bitwise the same states.  In-place lattices need a
 * periodic x axis, and have no closure and no access to the previous step's
 * state (mhd_closure_filter / mhd_closure_sgs_targets / mhd_set_closure
 * return MHD_EINVAL). */
typedef enum { MHD_TWO_BUFFERS = 0, MHD_IN_PLACE = 1 } mhd_streaming;

/* Collision of the magnetic populations. */
typedef enum {
    MHD_MAG_BGK = 0,         /* Eq. collide_g (the paper's scheme) */
    MHD_MAG_REGULARISED = 1  /* only the first Hermite moment of g - g_eq relaxes:
                                Lambda_ab = sum_j e_{j,a} (g - g_eq)_{j,b},
                                g* = g_eq + (1 - omega_m) psi_j e_{j,a} Lambda_ab / cs^2
                                (the extension the Conclusions name as the next step;
                                same magnetic diffusivity) */
} mhd_mag_collision;

typedef struct {
    double rho0;    /* reference density, > 0 (shift of the stored populations) */
    double tau_f;   /* fluid relaxation time, > 1/2 (omega = 1/tau_f) */
    double tau_m;   /* magnetic relaxation time, > 1/2 (omega_m = 1/tau_m) */
    int bc_x, bc_y; /* mhd_bc */
    int precision;  /* mhd_precision */
    int eq_variant; /* 0: Eq. feq_4th as printed (Maxwell stress at 2nd order
                       only); 1: with the u (x) M terms of Eq. a0_4 at 3rd and
                       4th order */
    int collision;  /* mhd_collision */
    int mag_collision; /* mhd_mag_collision */
    int streaming;     /* mhd_streaming (single lattices; batches use MHD_TWO_BUFFERS) */
} mhd_params;

/* Global diagnostics at the current time (mhd_get_totals).  Sums run over
 * all nodes; means divide by nx*ny.  Gradients use the isotropic lattice
 * stencil of the Orszag-Tang section; on a wall axis, nodes whose 3x3
 * stencil leaves the lattice are left out of divb_*, omega_max. */
typedef struct {
    double mass;      /* sum rho */
    double mom_x;     /* sum rho u_x */
    double mom_y;     /* sum rho u_y */
    double e_kin;     /* mean |u|^2 / 2  (E_k of the Orszag-Tang section) */
    double e_mag;     /* mean |b|^2 / 2  (E_m) */
    double cross_hel; /* mean u . b */
    double bsum_x;    /* sum b_x */
    double bsum_y;    /* sum b_y */
    double divb_max;  /* max |div b| */
    double divb_rms;  /* sqrt(mean (div b)^2) */
    double jz_max;    /* max |j_z|, j_z from the populations by Eq. current */
    double omega_max; /* max |d_x u_y - d_y u_x| */
    long long step;   /* time steps taken since the fields were set */
} mhd_totals;

/* Kernel launch shape of the fused step (chosen by mhd_autotune or the
 * built-in heuristic).  nodes_per_thread: consecutive x nodes one thread
 * updates with vector loads and stores: 1, 2 or 4 (at most 2 for MHD_FP64);
 * it must divide nx and must be 1 when the x axis has walls.
 * rows_per_block: warps per block, one row of 32*nodes_per_thread nodes
 * each: 1..16 (1..8 for MHD_FP64 and for MHD_FP16S with MHD_IN_PLACE).
 * warps_per_sm: the staging depth of the streamed neighbourhood -- how many
 * row tiles (warps) the persistent grid keeps in flight per SM, and with
 * them how many bytes of every plane are being loaded at once
 * (warps_per_sm x 32 x nodes_per_thread elements): 0 for the built-in rule
 * (about 4 KB of every plane per SM for FP32 and FP16S storage, every
 * resident warp for FP64), else 1..64, rounded down to whole blocks and
 * capped by what fits on an SM.  Ignored by the x-wall kernel. */
typedef struct {
    int nodes_per_thread;
    int rows_per_block;
    int warps_per_sm;
} mhd_kernel_config;

/* Create an nx x ny lattice on the current CUDA device.  The populations are
 * undefined until mhd_set_fields or mhd_set_populations.
 * stream: a cudaStream_t (may be NULL).  *out receives the handle (NULL on
 * failure).  MHD_EINVAL if nx or ny < 2, nx*ny > 2^31, tau_f or tau_m <= 1/2,
 * rho0 <= 0, an unknown enum value, or NULL p / out; MHD_ENOMEM if the two
 * population buffers (2 x 19 planes) do not fit in device memory. */
mhd_status mhd_create(int nx, int ny, const mhd_params* p, void* stream, mhd_lattice** out);

/* Set the initial state: f = f_eq(rho, u, b) (Eq. feq_4th), g = g_eq(u, b),
 * i.e. zero non-equilibrium (a1^(2) = 0, so this is both the pre- and the
 * post-collision state at t = 0).  ux, uy, bx, by: host arrays of nx*ny;
 * rho may be NULL (rho = rho0).  Resets the step counter.  Non-finite input,
 * or rho <= 0 -> MHD_EINVAL and the state is left as it was.  The arrays
 * are only read, and not after the call returns; pinned (page-locked)
 * arrays of a two-buffer lattice are read in place by the device in one
 * pass over the host link, other arrays through a device copy. */
mhd_status mhd_set_fields(mhd_lattice* l, const double* ux, const double* uy, const double* bx,
                          const double* by, const double* rho);

/* Queue nsteps fused stream-and-collide steps (tasks 1-6 of "Algorithm of
 * computation") on the lattice's stream; runs of 64 steps go through a CUDA
 * graph captured on first use.  nsteps >= 0. */
mhd_status mhd_advance(mhd_lattice* l, long long nsteps);

/* Read the fields of the current state into host arrays of nx*ny (any of
 * them may be NULL).  Waits for the stream.  Pinned (page-locked) arrays
 * are written in place by the device, others through a device copy. */
mhd_status mhd_get_fields(mhd_lattice* l, double* rho, double* ux, double* uy, double* bx,
                          double* by);

/* FP32 forms of mhd_set_fields and mhd_get_fields, for host data in single
 * precision (half the bytes over the host link).  Same arguments, layout
 * (row-major nx*ny, x fastest), NULL rules, ownership and errors.  Inputs
 * are widened exactly, so mhd_set_fields_f32 sets the state mhd_set_fields
 * sets for the same values held as double; each output is the value
 * mhd_get_fields returns, rounded to float (to nearest even). */
mhd_status mhd_set_fields_f32(mhd_lattice* l, const float* ux, const float* uy, const float* bx,
                              const float* by, const float* rho);
mhd_status mhd_get_fields_f32(mhd_lattice* l, float* rho, float* ux, float* uy, float* bx,
                              float* by);

/* Global diagnostics of the current state (see mhd_totals), reduced on the
 * GPU in FP64 with a fixed order (bitwise reproducible).  Waits for the
 * stream.  MHD_EUNSTABLE (with *out filled) if any total is not finite.
 * j_z needs the pre-collision magnetic populations: after a step they are
 * gathered again from the buffer that step read; right after
 * mhd_set_populations or mhd_autotune they are recovered from the stored
 * post-collision ones as g - g_eq = (g* - g_eq)/(1 - omega_m) (jz_max = 0
 * when tau_m = 1, where that inverse does not exist). */
mhd_status mhd_get_totals(mhd_lattice* l, mhd_totals* out);

/* Advance nsteps >= 1 steps (as mhd_advance) and return the point totals of
 * the pre-collision state the last step gathered -- the quantities of
 * mhd_totals that need no neighbour of a node: mass, momentum, e_kin, e_mag,
 * cross_hel, bsum and jz_max, with the definitions and arithmetic of
 * mhd_get_totals (the task 1 moments, Eq. current, the energies of the
 * Orszag-Tang section; FP64 only in the reductions).  The last step forms
 * them from the populations it holds for its collision, so this sample step
 * costs about what a plain step does (one read and one write of the state,
 * no diagnostics pass).  divb_max, divb_rms and omega_max need the 3 x 3
 * neighbourhood and are set to NaN here (mhd_get_totals gives them).  The
 * populations written are those of mhd_advance, bit for bit.  Two-buffer
 * lattices with a periodic x axis, no closure and no ghost rows; for other
 * lattices the call is mhd_advance followed by mhd_get_totals (all fields
 * filled).  Waits for the stream.  nsteps < 1 -> MHD_EINVAL; a non-finite
 * point total -> MHD_EUNSTABLE (with *out filled). */
mhd_status mhd_advance_totals(mhd_lattice* l, long long nsteps, mhd_totals* out);

/* Checkpoint: the stored post-collision populations as unshifted FP64 values.
 * f: 9*nx*ny doubles, plane i at f + i*nx*ny (i in the paper's D2Q9 order);
 * g: 10*nx*ny doubles, component a of g_j at g + (2*j + a)*nx*ny.
 * Waits for the stream. */
mhd_status mhd_get_populations(mhd_lattice* l, double* f, double* g);

/* Restore populations written by mhd_get_populations (same layout; values are
 * rounded to the storage precision).  The step counter is kept.  The FP64
 * view round-trips exactly for MHD_FP32 and MHD_FP16S storage; for MHD_FP64
 * storage to within one ulp (the shift w_i rho0 is added and removed in
 * FP64) -- use mhd_get_state / mhd_set_state for a bitwise checkpoint. */
mhd_status mhd_set_populations(mhd_lattice* l, const double* f, const double* g);

/* Bitwise checkpoint of the stored state: the 19 planes exactly as stored
 * (storage precision, FP32/FP16S/FP64 deviations f_i - w_i rho0 and g_{j,a},
 * FP16S scaled by 2^12), plane after plane, each nx*ny elements without row
 * padding.  *bytes = 19 * nx * ny * element size.  mhd_get_state waits for
 * the stream; mhd_set_state makes the restored state current (resuming
 * from it is bitwise identical to the run it was saved from).  host must
 * hold exactly mhd_state_bytes bytes (MHD_EINVAL otherwise). */
mhd_status mhd_state_bytes(const mhd_lattice* l, size_t* bytes);
mhd_status mhd_get_state(mhd_lattice* l, void* host, size_t bytes);
mhd_status mhd_set_state(mhd_lattice* l, const void* host, size_t bytes);

/* Halo exchange between two neighbouring slabs of a row-decomposed
 * periodic lattice (the decomposition of the y axis along which the step
 * shards over GPUs; see MHD_HALO).  `lower` holds the rows just below
 * `upper` in the global lattice (for the periodic wrap, the top slab is the
 * lower neighbour of the bottom one; one slab alone is its own neighbour).
 * Pull streaming carries across the boundary exactly the populations whose
 * velocity crosses it: from the top row of `lower` into the ghost row below
 * `upper` those with c_y = +1 (f_1, f_7, f_8 and g_4: 3 fluid populations and
 * one magnetic vector), from the bottom row of `upper` into the ghost row
 * above `lower` those with c_y = -1 (f_3, f_4, f_5 and g_2).  all_planes = 1
 * copies all 19 populations of those rows instead, which mhd_get_totals of a
 * slab needs (the gradient stencil at the slab's edge rows reads the moments
 * of the ghost rows).  Both lattices: bc_y = MHD_HALO, the same nx,
 * precision and bc_x, on devices that can copy to each other.  Usage: after
 * mhd_set_fields / mhd_set_populations / mhd_set_state, and after every
 * mhd_advance(l, 1), exchange every boundary once before the next step.
 * The copies are queued on the receiving lattice's stream after that
 * stream has been made to wait for the sending lattice's stream; nothing
 * waits on the host.  A lattice that has not been exchanged keeps the
 * ghost rows it had (zeros after mhd_create). */
mhd_status mhd_slab_exchange(mhd_lattice* lower, mhd_lattice* upper, int all_planes);

/* The slabs of one row-decomposed periodic lattice stepped together on one
 * device: mhd_slab_group_advance(g, n) does what n rounds of (mhd_advance of
 * every slab by one step, then mhd_slab_exchange of every boundary) do, with
 * every round's exchanges in one kernel and runs of 64 rounds in one CUDA
 * graph (captured on first use).  slabs[0..n-1] in order along y (slab i
 * just below slab i+1, the last just below the first); every slab
 * bc_y = MHD_HALO, the same nx, precision and bc_x, on the current device,
 * created with the same stream.  The group only borrows
 * the lattices (they must outlive it; the caller still destroys them) and
 * holds a small device table of its copies.  MHD_EINVAL for NULL or
 * mismatched slabs; advance: MHD_ESTATE unless every slab has its fields set
 * and all have taken the same number of steps modulo 2 (as they do when
 * stepped through the group).
 * Exchange after setting the fields (mhd_slab_exchange of every boundary)
 * before the first advance, as for slabs stepped one by one. */
typedef struct mhd_slab_group mhd_slab_group;
mhd_status mhd_slab_group_create(mhd_lattice* const* slabs, int n, mhd_slab_group** out);
mhd_status mhd_slab_group_advance(mhd_slab_group* g, long long nsteps);
mhd_status mhd_slab_group_destroy(mhd_slab_group* g);

/* Allocation-free global diagnostics (the paper has no counterpart to this
 * call; it is a service for callers that cannot allocate device memory
 * when they need the totals -- e.g. a host framework that has reserved the
 * whole GPU for its own memory pool and lends out only pointers it owns, or
 * a latency-critical loop that must not call cudaMalloc, which synchronises
 * the device).  It computes what mhd_get_totals computes, without a lattice
 * handle and without allocating: no cudaMalloc, cudaFree or other allocating
 * routine is called.
 *   state       device pointer to a state in the packed layout of
 *               mhd_get_state (19 planes of nx*ny elements of the storage
 *               type of p->precision), caller-owned, read only;
 *   prev_state  device pointer to the state the last step read (same
 *               layout), or NULL: then the pre-collision magnetic
 *               populations are recovered from `state` as
 *               g - g_eq = (g* - g_eq)/(1 - omega_m) (jz_max = 0 for
 *               tau_m = 1);
 *   p           rho0, tau_m, bc_x, bc_y and precision are used;
 *   stream      cudaStream_t (may be NULL); the call waits for it;
 *   out         caller-owned host struct (out->step is set to 0).
 * The per-block partial sums go to one fixed scratch array of about 1.7 MB
 * (room for 16384 blocks) that is compiled into the library: every GPU that
 * loads the library holds it until the process exits.  The diagnostics grid
 * is persistent and capped at the blocks the array holds, so the array
 * limits no lattice size; a lattice whose state (19 * nx * ny elements)
 * would not fit in the device's memory is rejected with MHD_EINVAL ("too
 * large") before anything is launched.  The caller must pass the state's
 * true extent: a smaller wrong size cannot be detected.  The array's device address is looked up on the first call made
 * in each device's current context (with that device current) and again
 * after the context changes (e.g. after cudaDeviceReset).  Every call uses
 * the same array and each call overwrites what it reads, so calls whose
 * work overlaps on a GPU (different streams or host threads at the same
 * time) race and must be serialised by the caller.  Any alignment of the
 * state pointers works (16-byte aligned states take the vector loads).
 * Non-finite totals -> MHD_EUNSTABLE (with *out filled). */
mhd_status mhd_totals_noalloc(const void* state, const void* prev_state, int nx, int ny,
                              const mhd_params* p, void* stream, mhd_totals* out);

/* Current launch shape, or set one explicitly (MHD_EINVAL if the shape is not
 * valid for this lattice). */
mhd_status mhd_get_kernel_config(const mhd_lattice* l, mhd_kernel_config* out);
mhd_status mhd_set_kernel_config(mhd_lattice* l, const mhd_kernel_config* cfg);

/* Autotune the launch shape: time every valid (nodes_per_thread,
 * rows_per_block) for this lattice with CUDA events at the built-in staging
 * depth, then the fastest shape at other depths (warps_per_sm = 1/2, 3/4,
 * 3/2 and 2 times the rule's), and keep the fastest (another depth only if
 * it is at least 1 % faster).
 * The state is not advanced (candidates read the current buffer and write
 * the spare one).  Results are cached per (GPU, precision, nx, ny, bc) in
 * the JSON file named by $MHD_TUNE_CACHE (no caching when unset); a cached
 * entry is reused without timing.  best (may be NULL) receives the choice.
 * With $MHD_TUNE_VERBOSE set, every candidate's time is printed to stderr. */
mhd_status mhd_autotune(mhd_lattice* l, mhd_kernel_config* best);

mhd_status mhd_destroy(mhd_lattice* l);

/* Message of the last failed call in this thread ("" if none). */
const char* mhd_last_error(void);

/* ---------------------------------------------------------------------------
 * Batched ensemble: many independent periodic lattices of uneven sizes and
 * relaxation times advanced by ONE persistent kernel launch per time step
 * (a tile work-list over all lattices, as many blocks as fit on the GPU),
 * the step loop captured in CUDA graphs of 64 steps.  Storage is FP32; each
 * lattice i has its own params[i] (precision must be MHD_FP32 and both axes
 * MHD_PERIODIC).  A lattice advanced in a batch is bitwise identical to the
 * same lattice advanced alone with the same launch shape.  Same conventions
 * as the single-lattice calls; index selects a lattice (0..count-1).
 * ------------------------------------------------------------------------- */
mhd_status mhd_batch_create(int count, const int* nx, const int* ny, const mhd_params* params,
                            void* stream, mhd_batch** out);
mhd_status mhd_batch_set_fields(mhd_batch* b, int index, const double* ux, const double* uy,
                                const double* bx, const double* by, const double* rho);
/* every lattice must have its fields set (MHD_ESTATE otherwise) */
mhd_status mhd_batch_advance(mhd_batch* b, long long nsteps);
/* Advance nsteps >= 1 steps (as mhd_batch_advance) and return the point
 * totals of every lattice's pre-collision state of the last step into
 * out[0 .. count-1]: mass, momentum, e_kin, e_mag, cross_hel, bsum and
 * jz_max (the definitions and arithmetic of mhd_totals), formed by that
 * step from the populations it collides, so the sample step reads and
 * writes the ensemble once; divb_max, divb_rms and omega_max are NaN (they
 * need the neighbourhood: mhd_batch_get_all_totals).  The populations are
 * those of mhd_batch_advance, bit for bit.  Waits for the stream.
 * nsteps < 1 -> MHD_EINVAL; a non-finite point total in any lattice ->
 * MHD_EUNSTABLE, with every entry filled. */
mhd_status mhd_batch_advance_totals(mhd_batch* b, long long nsteps, mhd_totals* out);
mhd_status mhd_batch_get_fields(mhd_batch* b, int index, double* rho, double* ux, double* uy,
                                double* bx, double* by);
mhd_status mhd_batch_get_totals(mhd_batch* b, int index, mhd_totals* out);
/* The totals of every lattice of the batch into out[0 .. count-1]: one
 * diagnostics launch walks the tiles of all the lattices (each tile's sums
 * into a partial of its own, then each lattice's partials added in tile
 * order), one copy back, one wait for the stream.  The values are those of
 * mhd_batch_get_totals of each index up to the order of the FP64 sums (the
 * maxima exactly); where a lattice's rows do not allow the kernel's
 * two-node vector loads, every lattice's own pass is queued instead (then
 * bit for bit those values).  A lattice whose fields were not
 * set -> MHD_ESTATE (nothing written); a non-finite total in any lattice ->
 * MHD_EUNSTABLE, with every entry filled. */
mhd_status mhd_batch_get_all_totals(mhd_batch* b, mhd_totals* out);
/* total number of nodes over all lattices */
mhd_status mhd_batch_nodes(const mhd_batch* b, long long* nodes);
/* launch shape (nodes_per_thread must divide every nx; warps_per_sm 0 keeps
 * every resident block, which the ensemble's many short rows want); autotune
 * times every valid shape over the whole ensemble without advancing it,
 * then the fastest at half and three quarters of the resident warps */
mhd_status mhd_batch_get_kernel_config(const mhd_batch* b, mhd_kernel_config* out);
mhd_status mhd_batch_set_kernel_config(mhd_batch* b, const mhd_kernel_config* cfg);
mhd_status mhd_batch_autotune(mhd_batch* b, mhd_kernel_config* best);
mhd_status mhd_batch_destroy(mhd_batch* b);

/* ---------------------------------------------------------------------------
 * Learned sub-grid closure (an extension; the paper has no closure).  A
 * per-node MLP predicts a correction dA = (xx, xy, yy) of the projected
 * non-equilibrium coefficient a1^(2) (task 3 of "Algorithm of computation")
 * on a coarse lattice; dA is added before the recursion, so mass and
 * momentum stay exact.  The MLP is 24 -> 64 -> 64 -> 3 with ReLU:
 *   y = out_scale * (W3^T h2 + b3), h2 = relu(W2^T h1 + b2),
 *   h1 = relu(W1^T xn + b1), xn = (x - mean) * scale,
 * evaluated and trained on BF16 tensor cores (mma.sync m16n8k16) with FP32
 * accumulation; the master weights are FP32.
 * Features x (24 per node, of the pre-collision state): rho - rho0, u_x,
 * u_y, b_x, b_y, a1^(2)_xx, a1^(2)_xy, a1^(2)_yy, then for each of u_x, u_y,
 * b_x, b_y: d_x, d_y (isotropic lattice gradient), the 9-point lattice
 * Laplacian (4 sum_axes + sum_diagonals - 20 q)/6, and
 * d_xy = (q_NE - q_NW - q_SE + q_SW)/4.
 * Parameter blob (MHD_MLP_PARAMS floats, in order): mean[24], scale[24],
 * out_scale[3], W1[24][64], b1[64], W2[64][64], b2[64], W3[64][3], b3[3]
 * (weights input-major, W[in][out]).
 * Device pointers below are caller-owned CUDA memory; the calls wait for
 * their stream (the MLP's, or the one passed) before returning.
 * ------------------------------------------------------------------------- */
#define MHD_MLP_PARAMS 6006
typedef struct mhd_mlp mhd_mlp;

/* He-normal weights from SplitMix64(seed), zero biases, identity
 * normalisation.  max_batch: the largest number of samples one training
 * batch or gradient call holds (16 .. 2^24). */
mhd_status mhd_mlp_create(unsigned long long seed, int max_batch, void* stream, mhd_mlp** out);
mhd_status mhd_mlp_destroy(mhd_mlp* m);
/* host copy of the FP32 parameter blob (count must be MHD_MLP_PARAMS);
 * set_params also resets the Adam state */
mhd_status mhd_mlp_get_params(const mhd_mlp* m, float* host, size_t count);
mhd_status mhd_mlp_set_params(mhd_mlp* m, const float* host, size_t count);
/* mean / scale = 1/std per feature and out_scale = std per target from a
 * data set X (n x 24), T (n x 3) in device memory (FP64 reductions) */
mhd_status mhd_mlp_fit_normalisation(mhd_mlp* m, const float* X, const float* T, long long n);
/* Loss L = mean over n x 3 entries of (y / out_scale - T / out_scale)^2 and
 * its gradient with respect to the blob (grad_host: MHD_MLP_PARAMS floats,
 * zero for the normalisation entries), one full batch of n <= max_batch. */
mhd_status mhd_mlp_gradients(mhd_mlp* m, const float* X, const float* T, long long n, float* grad_host,
                             double* loss);
/* Mini-batch Adam (beta1 0.9, beta2 0.999, eps 1e-8) over `epochs`
 * passes of the data set, each in a different pseudo-random order (a
 * bijection of the sample indices computed on the GPU, keyed by seed and
 * the Adam step count); *last_epoch_loss (may be NULL) is the mean batch
 * loss of the last pass.  MHD_EUNSTABLE if it is not finite. */
mhd_status mhd_mlp_train(mhd_mlp* m, const float* X, const float* T, long long n, int epochs, int batch,
                         float lr, unsigned long long seed, double* last_epoch_loss);
/* Y (n x 3, device) = dA predicted for the features X (n x 24, device). */
mhd_status mhd_mlp_predict(mhd_mlp* m, const float* X, long long n, float* Y);

/* Box filter (factor x factor block average) of a lattice's pre-collision
 * populations at its current time into a packed coarse state
 * (FP32 deviations f_i - w_i rho0 and g, 19 planes of
 * (nx/factor)*(ny/factor) values, the layout of mhd_get_state for FP32).
 * The lattice must be periodic and have taken at least one step since its
 * state was set (MHD_ESTATE otherwise). */
mhd_status mhd_closure_filter(mhd_lattice* l, int factor, float* coarse_state);
/* Features (n x 24) of a packed FP32 pre-collision state (periodic). */
mhd_status mhd_closure_features(const float* state, int nx, int ny, double rho0, float* X, void* stream);
/* Targets (n x 3): the correction that makes one coarse collide-and-stream
 * step from state_t reproduce state_t1 in its second-order moments:
 * dA = (sum_i H2_i F_i(x + c_i, t+1) - a0^(2)) / (1 - 1/tau_f) - a1^(2)(t),
 * with a0^(2) = rho u u + M (FP64 arithmetic).  Periodic. */
mhd_status mhd_closure_targets(const float* state_t, const float* state_t1, int nx, int ny, double rho0,
                               double tau_f, float* T, void* stream);
/* Sub-grid stress targets (n_coarse x 3, device) from a lattice's
 * pre-collision state at its current time: per coarse node (factor x factor
 * block) tau_sgs = <rho u u + M(b)> - (<rho> u_t u_t + M(<b>)) with
 * u_t = <rho u>/<rho> (xx, xy, yy, FP64 arithmetic), returned as the
 * a1^(2) correction tau_sgs / (1 - 1/tau_coarse) that adds tau_sgs to the
 * coarse post-collision momentum flux.  Periodic lattices with rho0 = 1,
 * after at least one step (MHD_ESTATE otherwise). */
mhd_status mhd_closure_sgs_targets(mhd_lattice* l, int factor, double tau_coarse, float* targets);
/* Make `state` (device, packed FP32 pre-collision populations as written by
 * mhd_closure_filter, of this lattice's size) the pre-collision state of the
 * next step: the stored state becomes S_i(x) = F_i(x + c_i), so the next
 * mhd_advance collides exactly F.  Fields and totals read before that step
 * describe S, not F.  Periodic lattices. */
mhd_status mhd_set_precollision_state(mhd_lattice* l, const float* state);
/* Switch the lattice's step to the closure variant with a copy of the MLP's
 * current parameters (the MLP may be destroyed afterwards), or back to the
 * plain scheme with mlp = NULL.  FP32 storage and periodic axes only. */
mhd_status mhd_set_closure(mhd_lattice* l, const mhd_mlp* mlp);
/* The kernel that evaluates the closure MLP inside the step (an
 * implementation choice with no counterpart in the paper; the results agree
 * to BF16 rounding of the summation order):
 *   MHD_CLOSURE_WARP_MMA: warp-level mma.sync BF16 fragments, activations kept
 *     in registers between layers (the default);
 *   MHD_CLOSURE_TCGEN05: 5th-generation tensor cores, two M = 128 MMAs per
 *     32 x 8-node tile issued by one thread, accumulators in tensor memory.
 * mhd_autotune on a lattice with a closure times both and keeps the faster.
 * A tcgen05 wait that gives up (after ~0.1 s) is reported as MHD_ECUDA by the
 * next read of fields, totals, populations or state. */
typedef enum { MHD_CLOSURE_WARP_MMA = 0, MHD_CLOSURE_TCGEN05 = 1 } mhd_closure_kernel;
mhd_status mhd_set_closure_kernel(mhd_lattice* l, int kind);
mhd_status mhd_get_closure_kernel(const mhd_lattice* l, int* kind);
/* Refresh interval of the closure (an option of this implementation; the
 * closure itself is not in the paper): the features and the MLP are
 * evaluated on every k-th step only -- the steps whose count since the last
 * change of the state, of the closure or of k is a multiple of k -- and the
 * correction they give each node is stored (3 x nx*ny FP32, allocated by
 * this call) and added again on the k - 1 steps between, which then cost a
 * plain step plus 12 bytes per node.  k = 1 (the default) evaluates the MLP
 * on every step.  k must divide 64 (the steps of a captured CUDA graph);
 * k > 1 needs an FP32 periodic two-buffer lattice with nx % 4 == 0
 * (MHD_EINVAL otherwise).  Takes effect on the lattice's next step. */
mhd_status mhd_set_closure_interval(mhd_lattice* l, int k);
mhd_status mhd_get_closure_interval(const mhd_lattice* l, int* k);

#ifdef __cplusplus
}
#endif
#endif /* MHD_LBM_H */
