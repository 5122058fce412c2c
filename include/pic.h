/*
 * pic.h -- C ABI of the GB300 (sm_103a) boosted-frame electromagnetic
 * particle-in-cell library.
 *
 * The library advances a laser-plasma stage in a frame Lorentz-boosted along
 * the laser axis z (Vay et al., arXiv:1011.0917, introduction and section
 * "Effect of the hyperbolic rotation in Minkowski space": the boost contracts
 * the plasma and dilates the laser so that far fewer steps are needed).  One
 * step is: field gather and relativistic Boris push of the electrons,
 * Esirkepov charge-conserving current deposition (electrons and, in a boosted
 * frame, the ions drifting at -beta), the laser antenna current, binomial
 * filtering of the current (section "Mitigation of a numerical instability":
 * filtering of short wavelengths), the Yee update of B and E, and injection
 * of the plasma that enters the box.
 *
 * Units everywhere in this interface: lengths in the laser wavelength lambda0,
 * times in lambda0/c, momenta u = gamma v / c, fields in m c omega0 / e (a laser
 * of normalised amplitude a0 has peak E = a0), densities in the critical
 * density n_c.  Lab-frame inputs are transformed to the simulation frame by
 * the library in FP64.
 *
 * Memory: the CALLER owns all device memory.  pic_query_sizes() reports the
 * byte size of each buffer; the caller allocates them on the device (256-byte
 * aligned) and passes them to pic_bind_buffers().  The library owns only its
 * small host context.  All device work is enqueued on the stream given in
 * pic_grid_params; calls that return data synchronise that stream.
 *
 * Errors: every call returns a pic_status; no exception or longjmp crosses the
 * ABI.  pic_last_error() gives a human-readable detail of the last failure of
 * a context.  A context is not thread-safe; distinct contexts are independent.
 */
#ifndef PIC_H
#define PIC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum pic_status {
    PIC_OK = 0,
    PIC_ERR_ARG = 1,      /* invalid argument or size                          */
    PIC_ERR_STATE = 2,    /* call out of order (e.g. step before bind)         */
    PIC_ERR_CUDA = 3,     /* a CUDA call failed; detail in pic_last_error      */
    PIC_ERR_CAPACITY = 4, /* a tile bucket overflowed; particles were dropped  */
    PIC_ERR_CFL = 5,      /* a particle moved a cell or more in one step       */
    PIC_ERR_NAN = 6,      /* a non-finite momentum or position was produced    */
    PIC_ERR_TIMEOUT = 7   /* reserved for bounded device waits                 */
} pic_status;

enum { PIC_BC_PERIODIC = 0, PIC_BC_MUR = 1 };       /* z boundary (x, y periodic) */
enum { PIC_FP32 = 0, PIC_FP64 = 1 };                /* arithmetic of the path     */
enum { PIC_ELECTRONS = 0, PIC_IONS = 1 };           /* species index              */
enum { PIC_POL_X = 0, PIC_POL_Y = 1 };              /* laser polarisation         */

/* field components, bit i of a component mask selects component i */
enum {
    PIC_EX = 0, PIC_EY = 1, PIC_EZ = 2, PIC_BX = 3, PIC_BY = 4, PIC_BZ = 5,
    PIC_JX = 6, PIC_JY = 7, PIC_JZ = 8, PIC_NCOMP = 9
};

/* Phases of one step, in the order pic_step runs them (a mask of these bits
   selects a subset for pic_step_phases; PIC_PH_ALL is one full step):
     ZERO_J   J = 0
     PUSH     electrons: gather E^n, B^n at x^n, Boris u^{n-1/2} -> u^{n+1/2},
              x^{n+1} = x^n + dt u/gamma, Esirkepov J^{n+1/2}, boundaries,
              re-bucketing by tile
     IONS     ions (boosted frame): constant drift, deposit, boundaries
     ANTENNA  laser current sheet at t^{n+1/2}
     FILTER   filter_passes binomial passes along each axis on Jx, Jy, Jz
     YEE      B -= dt/2 curl E; E += dt (curl B - 2 pi J) (+ Mur); B -= dt/2 curl E
     INJECT   plasma crossing z = Lz during (t, t+dt] appended at x^{n+1}
     TIME     t += dt (FP64 host accumulator)                                  */
#define PIC_PH_ZERO_J 1u
#define PIC_PH_PUSH 2u
#define PIC_PH_IONS 4u
#define PIC_PH_ANTENNA 8u
#define PIC_PH_FILTER 16u
#define PIC_PH_YEE 32u
#define PIC_PH_INJECT 64u
#define PIC_PH_TIME 128u
#define PIC_PH_ALL 255u

typedef struct pic_ctx pic_ctx;

/* Grid and numerics.  Lab-frame cell sizes: the simulation-frame ones are
   hx = dx, hy = dy, hz = dz * gamma * (1 + beta) (same cells per Doppler-
   stretched laser wavelength), dt = cfl / sqrt(sum 1/h_d^2). */
typedef struct pic_grid_params {
    int dim;                /* 2: (x, z) with y ignorable (2D3V); 3: (x, y, z)  */
    int nx, ny, nz;         /* cells; ny must be 1 when dim == 2                */
    double dx, dy, dz;      /* lab-frame cell sizes, lambda0 (dy unused in 2D) */
    double cfl;             /* time step as a fraction of the Courant limit, <1 */
    double gamma_boost;     /* Lorentz factor of the frame, >= 1                */
    int shape_order;        /* 1: linear (CIC), 2: quadratic spline             */
    int filter_passes;      /* binomial passes per axis, >= 0                   */
    int bc_z;               /* PIC_BC_MUR or PIC_BC_PERIODIC                    */
    int precision;          /* PIC_FP32 (production) or PIC_FP64 (debug)        */
    uint64_t seed;          /* SplitMix64 seed of the plasma jitter             */
    double slots_per_cell;  /* particle slots per cell and species, > 0         */
    int tile[3];            /* tile shape in cells: 0 or a compiled shape:      */
                            /* 8x8x8 in 3D (CIC also 8x8x4); 16x1x16 in 2D,     */
                            /* with the CIC shape also 32x1x8, 8x1x32 (others:  */
                            /* PIC_ERR_ARG)                                      */
    int track_ids;          /* 1: carry an int64 lattice id with each particle */
    int explicit_ions;      /* 1: store every drifting ion as its own record    */
                            /* (0: electron-ion pairs, see pic_load_plasma)     */
    int z_relative;         /* electron position storage: 0 automatic (relative */
                            /* when gamma_boost >= 50), 1 relative, 2 absolute; */
                            /* see the note below                               */
    void *stream;           /* cudaStream_t for all device work (NULL: legacy)  */
} pic_grid_params;

/* Relative positions.  In a frame boosted to gamma the plasma (electrons and
   ions, gamma n each) streams through a good part of a cell every step, and
   the wake is the small difference between the two species' currents: about
   1 / (2 gamma^2) of the plasma's response in the lab, i.e. ~3e-8 of either
   species' current at gamma = 130.  Positions rounded to FP32 (6e-8 cell)
   and currents formed in FP32 then leave only rounding noise of the wake.
   With z_relative an electron record holds, per axis, a reference offset --
   along z it moves with exactly the arithmetic of a drifting ion, across z
   it stays where the particle was placed, so it is the path of the
   electron's own ion -- plus the departure from it in its own FP32 word
   (relative precision); the currents of electrons and ions are formed in
   FP64 from these exact positions and accumulated in the same fixed-point
   words.  It costs 8 bytes (2D) or 12 bytes (3D) more per electron record in
   FP32 and FP64 deposit arithmetic; the gather, the push and the fields keep
   the working precision.  The method computed is the same either way. */

/* Sizes of the caller-owned device buffers and derived quantities. */
typedef struct pic_sizes {
    size_t field_bytes;        /* 9 components x (nz+1) x ny x nx elements         */
    size_t species_bytes[2];   /* particle store per species (two bucket sides)    */
    size_t scratch_bytes;      /* tile counters, raw-current / filter buffer,      */
                               /* the second E, B buffer of the Yee update, ...   */
    int64_t slots[2];          /* particle slots per side and species              */
    int64_t ntiles;            /* number of tiles                                  */
    int tile_capacity;         /* slots per tile                                   */
    int tile[3];               /* tile shape in cells                              */
    int elem_bytes;            /* 4 (FP32) or 8 (FP64)                             */
    double dt, hx, hy, hz;     /* simulation-frame step and cell sizes, lambda0    */
    double beta;               /* boost velocity / c                               */
} pic_sizes;

typedef struct pic_buffers {
    void *fields;              /* field_bytes                                      */
    void *species[2];          /* species_bytes[s]; species[1] may be NULL if 0    */
    void *scratch;             /* scratch_bytes                                    */
} pic_buffers;

/* Plasma at rest in the lab frame, loaded on a lattice of ppc points per cell
   and axis with a uniform jitter; in a boosted frame it drifts at -beta and
   is contracted by gamma, and the part beyond z = Lz enters the box later. */
typedef struct pic_plasma_params {
    double ne_over_nc;         /* lab-frame electron density / n_c                 */
    double z_start, z_end;     /* lab-frame extent, lambda0                        */
    double ramp_len;           /* linear up-ramp length from z_start, lambda0      */
    int ppc[3];                /* lattice points per cell and axis (ppc[1] 2D: 1)  */
    double jitter;             /* uniform jitter half width, cells, in [0, 0.5)    */
    int n_profile;             /* number of cosine-profile coefficients, <= 16     */
    const double *profile;     /* c_m: n = n0 (1 + sum_m c_m cos(m pi zeta))      */
    int ions;                  /* 1: ions immobile in the lab frame                */
} pic_plasma_params;

/* Linearly polarised Gaussian laser, lab-frame parameters.  The antenna is a
   current sheet at rest in the simulation frame on the node plane nearest to
   z_antenna (at least 2 nodes from either z end). */
typedef struct pic_laser_params {
    double a0;                 /* peak normalised amplitude                        */
    double waist;              /* 1/e field radius, lambda0                        */
    double fwhm;               /* intensity FWHM duration, lambda0/c               */
    double z_antenna;          /* antenna plane, simulation frame, lambda0         */
    double t_peak;             /* envelope peak (lab time at antenna); <0: 3 tau   */
    int polarization;          /* PIC_POL_X or PIC_POL_Y                           */
    double x_center, y_center; /* transverse centre, lambda0; NaN: box centre      */
} pic_laser_params;

typedef struct pic_diag {
    double t;                  /* simulation-frame time                            */
    int64_t step;              /* steps taken                                      */
    int64_t n_particles[2];    /* live particles per species (ions: stored ions    */
                               /* plus the ions of paired electrons)               */
    int64_t n_paired;          /* electrons still paired with their ion            */
    double field_energy;       /* (1/2) sum (E^2 + B^2) V, Kahan-compensated FP64   */
    double kinetic_energy;     /* sum w (gamma - 1) of the electrons, FP64 Kahan   */
    double charge;             /* sum q w of both species, FP64 Kahan              */
    double z_window;           /* moving window displacement (positions, fields    */
                               /* and rho are relative to it), lambda0             */
} pic_diag;

/* ---------------------------------------------------------------- set-up */

/* Validates the parameters and creates a context.  PIC_ERR_CFL if cfl >= 1,
   PIC_ERR_ARG for any other invalid field.  *out is NULL on failure.
   Paper: the stage is simulated in a frame boosted to gamma_boost along the
   laser axis (introduction: the boost contracts the plasma and dilates the
   laser, so far fewer steps are needed); the cell sizes keep the cells per
   Doppler-stretched laser wavelength. */
pic_status pic_init_grid(const pic_grid_params *p, pic_ctx **out);

/* Buffer sizes and derived quantities of a context (the simulation-frame cell
   sizes and time step of pic_init_grid).  No counterpart in the paper: the
   library's memory contract.  PIC_ERR_ARG for a NULL argument. */
pic_status pic_query_sizes(const pic_ctx *ctx, pic_sizes *out);

/* Binds the caller-owned device buffers and clears them (fields, particle
   counts, error word) on the stream.  Pointers must be 256-byte aligned and
   at least the queried sizes.  May be called once per context.  No
   counterpart in the paper.  PIC_ERR_ARG for a NULL or misaligned buffer,
   PIC_ERR_STATE if buffers are already bound. */
pic_status pic_bind_buffers(pic_ctx *ctx, const pic_buffers *b);

/* Paper: a plasma at rest in the laboratory, seen from the boosted frame
   through the Lorentz transformation (the hyperbolic rotation of section
   "Effect of the hyperbolic rotation in Minkowski space"): density gamma n,
   drift -beta, contracted by gamma, entering the box as the frame moves.
   Generates the plasma on the device: every lattice point whose simulation-
   frame position at the current time lies in the box becomes an electron
   (and, boosted with ions, a drifting ion at the same place); the rest of a
   boosted plasma is injected as it crosses z = Lz.  Lab-frame immobile ions
   are a neutralising background and carry no current.  The lattice id of a
   point with indices (ix, iy, iz) is (iz * NY + iy) * NX + ix, NX = nx*ppc[0],
   NY = ny*ppc[1] (1 in 2D).  PIC_ERR_CAPACITY if a tile overflowed.
   Storage of drifting ions: an electron and its ion start at the same place
   with the same momentum and move identically until a non-zero field reaches
   the electron, so their currents cancel exactly; such a pair is kept as the
   electron record alone ("paired"), and the ion gets its own record, at the
   electron's position, in the step the electron first gathers a non-zero
   field.  pic_get_particles and pic_get_diagnostics report both members. */
pic_status pic_load_plasma(pic_ctx *ctx, const pic_plasma_params *p);

/* Appends n particles given as host FP64 arrays (simulation frame):
   state[a*n + i] for a = 0..6 = x, y, z, ux, uy, uz, w.  Ions take the
   species' drift momentum and ignore ux, uy, uz.  (The device holds electron
   momenta relative to the plasma drift, u - (0, 0, -gamma beta), so that the
   working precision resolves the plasma's response; pic_get_particles adds
   the drift back.)  ids (may be NULL) are kept
   when track_ids is set.  Positions outside the box are rejected
   (PIC_ERR_ARG); PIC_ERR_CAPACITY if a tile overflowed.  No counterpart in
   the paper: explicit particles for tests and restarts (the paper's plasma
   is pic_load_plasma's). */
pic_status pic_load_particles(pic_ctx *ctx, int species, int64_t n, const double *state,
                              const int64_t *ids);

/* Sets the laser; the antenna current is added in every later step.
   Paper: the laser is launched in the boosted frame, its lab-frame pulse
   Doppler-transformed (amplitude and frequency gamma (1 - beta), duration
   gamma (1 + beta); section "Effect of the hyperbolic rotation in Minkowski
   space").  PIC_ERR_ARG for a0 < 0, a waist or duration <= 0, a non-finite
   z_antenna or an unknown polarisation.  A forward run of the adjoint taken
   before this call no longer belongs to the context's run. */
pic_status pic_launch_laser(pic_ctx *ctx, const pic_laser_params *p);

/* ------------------------------------------------------------------ step */

/* Advances nsteps full steps, synchronises the stream and checks the device
   error word (PIC_ERR_CAPACITY / PIC_ERR_CFL / PIC_ERR_NAN / PIC_ERR_TIMEOUT).
   Paper: one step of the particle-in-cell loop the paper's runs use (the
   electromagnetic PIC method named in section "Effect of the hyperbolic
   rotation in Minkowski space"), with the current filtered against short
   wavelengths as in section "Mitigation of a numerical instability". */
pic_status pic_step(pic_ctx *ctx, int nsteps);

/* Same as pic_step without the synchronisation and the error check (read
   the device error word later with pic_step(ctx, 0)).  PIC_ERR_ARG for
   nsteps < 0, PIC_ERR_STATE before pic_bind_buffers. */
pic_status pic_step_async(pic_ctx *ctx, int nsteps);

/* One step restricted to the phases in mask (PIC_PH_* bits), synchronised
   and checked like pic_step.  Used to test each phase on its own (the phases
   are those of pic_step).  PIC_ERR_ARG for unknown bits. */
pic_status pic_step_phases(pic_ctx *ctx, unsigned mask);

/* --------------------------------------------------------------- output */

/* Frames of pic_get_fields. */
enum { PIC_FRAME_BOOST = 0, PIC_FRAME_LAB = 1 };

/* Copies the components selected by mask, in component order, each as
   (nz+1) x ny x nx elements of elem_bytes in [k][j][i] order (the native
   layout; the plane k = nz of Ez, Bx, By, Jz is unused and zero).  dst may be
   host (dst_is_device = 0) or device memory; dst_bytes must hold them all.
   frame PIC_FRAME_BOOST: the simulation-frame fields as stored.
   frame PIC_FRAME_LAB: E and B as the laboratory sees them on the same grid
   nodes at the current simulation time (the inverse of the boost, the
   paper's hyperbolic rotation; section "Effect of the hyperbolic rotation in
   Minkowski space"): Ex = gamma (Ex' + beta By'), Ey = gamma (Ey' - beta Bx'),
   Ez = Ez', Bx = gamma (Bx' - beta Ey'), By = gamma (By' + beta Ex'),
   Bz = Bz', in FP64, each component at its own Yee position and the partner
   it mixes with (half a cell away in z) taken as the mean of its two planes
   around it (the nearer plane alone at an absorbing z end; planes wrap when
   z is periodic).  Only E and B (mask bits 0..5; J bits: PIC_ERR_ARG); a
   device dst must be aligned to elem_bytes.  With gamma_boost = 1 both
   frames are the same.  For snapshots at a fixed lab time use pic_btd_*. */
pic_status pic_get_fields(pic_ctx *ctx, unsigned mask, int frame, void *dst, size_t dst_bytes,
                          int dst_is_device);

/* Overwrites the selected components from src, same layout as pic_get_fields
   (simulation frame).  No counterpart in the paper: initial and test
   conditions.  PIC_ERR_ARG for a NULL src, an empty or unknown mask or too
   small a source, PIC_ERR_STATE before pic_bind_buffers. */
pic_status pic_set_fields(pic_ctx *ctx, unsigned mask, const void *src, size_t src_bytes,
                          int src_is_device);

/* Component c on the line i = nx/2, j = ny/2, k = 0..nz (nz+1 elements of
   elem_bytes): the on-axis field history diagnostic of the paper's Fig. 2.
   PIC_ERR_ARG for a NULL dst, an unknown component or too small a
   destination, PIC_ERR_STATE before pic_bind_buffers. */
pic_status pic_get_axis(pic_ctx *ctx, int component, void *dst, size_t dst_bytes,
                        int dst_is_device);

/* Live particles of a species as host FP64 arrays in the pic_load_particles
   layout (order unspecified); *n_out receives the count.  (Paper: the
   macroparticles of the PIC method; simulation-frame positions and momenta.)  With dst == NULL
   only *n_out is set.  ids (may be NULL) receives the lattice ids when
   track_ids is set.  PIC_ERR_ARG for an unknown species or too small a
   destination, PIC_ERR_STATE before pic_bind_buffers. */
pic_status pic_get_particles(pic_ctx *ctx, int species, double *dst, size_t dst_bytes,
                             int64_t *n_out, int64_t *ids);

/* Nodal charge density (nz+1) x ny x nx of the particles (electrons and
   drifting ions, shape of the grid's order), elem_bytes each, into host or
   device memory.  Lab-frame immobile ions are not included.  A diagnostic of
   the charge that Esirkepov's deposition conserves (the continuity the
   method's current deposition satisfies; no printed formula in the paper).
   PIC_ERR_ARG for a NULL dst or too small a destination, PIC_ERR_STATE before
   pic_bind_buffers. */
pic_status pic_get_rho(pic_ctx *ctx, void *dst, size_t dst_bytes, int dst_is_device);

/* Time, counts and FP64 Kahan-compensated sums (synchronises the stream):
   field energy (1/2) sum (E^2 + B^2) V over each component's valid nodes,
   electron kinetic energy sum w (gamma - 1), charge sum q w (drifting ions
   +1; lab-frame immobile ions are a background), both energies in units of
   n_c m c^2 lambda0^3.  (Paper: no counterpart; the energy budget of the
   stage.)  PIC_ERR_ARG for a NULL out, PIC_ERR_STATE before
   pic_bind_buffers. */
pic_status pic_get_diagnostics(pic_ctx *ctx, pic_diag *out);

/* ------------------------------------------------------------------ batch */

/* Several independent runs stepped together (a scan over stage parameters:
   different boosts, grid lengths, density profiles, laser amplitudes).
   pic_batch_step issues one step of every context in turn before the next
   step; each context's work goes on its own stream (pic_grid_params.stream:
   give every context a distinct stream so that their kernels run
   concurrently), and every context's device error word is checked at the end
   (the first failure is returned; pic_last_error of each context has its
   detail).  The batch holds pointers only: the contexts stay the caller's and
   must outlive it.  PIC_ERR_STATE if a context is not bound, PIC_ERR_ARG for
   n < 1 or a context listed twice.  No counterpart in the paper, which runs
   one stage at a time: the batch is the library's scan over stages. */
typedef struct pic_batch pic_batch;
pic_status pic_batch_create(pic_ctx *const *ctxs, int n, pic_batch **out);
pic_status pic_batch_step(pic_batch *batch, int nsteps);
void pic_batch_destroy(pic_batch *batch);

/* Steps of a batch run as CUDA graphs of steps_per_graph steps of every
   context (even; default 20; 0: streams only): pic_batch_step replays the
   graph nsteps / steps_per_graph times (the remainder, and batches with a
   moving window, lab snapshots, phase timing or a context on the legacy
   default stream, take the stream path).  The graph is captured by the
   first call that needs it and kept by the batch while every context stays
   as the capture left it: a call that changes what a context's step launches
   (binding, plasma or particle load, laser, window, snapshots, state restore,
   phase timing, an adjoint run) or an odd number of steps taken outside the
   graph (the double buffers then start on their other halves) makes the
   next call capture again.  The per-step values (antenna amplitude,
   injection band and times) of all replays of a call are written to pinned
   host memory first, one region per replay, each copied to the device on
   the graph's stream just before its replay, so replays follow each other
   without waiting for the host; the graph's stream is ordered after the work
   already queued on the contexts' streams and before the work queued on them
   later.  PIC_ERR_ARG for a negative or odd count. */
pic_status pic_batch_set_graph(pic_batch *batch, int steps_per_graph);

/* The form of the captured graph.  fused = S >= 1 (default 4): the
   batched form, where every launch of every context's steps has one (all
   do, except the per-pass filter path for more than 4 passes).  The runs are
   spread over min(S, n) launch chains by size; each chain is a stream of its
   own inside the graph (forked from and joined to the graph's stream) on
   which each phase of each step is one launch over the work items of the
   chain's runs (runs whose particle kernels differ in precision, dimension,
   shape order, tile shape or position form get one launch per kind): the
   zeroing of the raw currents, the particle push -- a persistent grid whose
   CTAs take (run, tile) items from a device-wide counter, so runs of uneven
   size share the GPU to the last tile -- the drifting ions, the antenna,
   the filter (3D runs take the plane-load filter instead of the TMA one: a
   tensor map is made per launch), the Yee update and the injection.  Chains
   overlap one chain's field phases with another's push.  Each item is
   processed by the same code and arithmetic as in a single run's launch, so
   the results are those of the per-context graph (up to the order of the
   floating-point additions of tiles into J).  fused = 0: the per-context
   graph (every context's launches on its own stream, forked from and joined
   to the graph's).  A change drops the kept graph.  PIC_ERR_ARG for
   fused < 0. */
pic_status pic_batch_set_fused(pic_batch *batch, int fused);

/* The graph the batch keeps (zeros before the first capture): its launch
   chains if it is the fused form (0: per context), the launches one replay
   issues (kernels and counter resets) and the steps it covers.  Any output
   pointer may be NULL; PIC_ERR_ARG for a null batch.  No counterpart in the
   paper. */
pic_status pic_batch_graph_info(pic_batch *batch, int *fused, int64_t *launches_per_replay, int *steps);

/* ---------------------------------------------------------- moving window */

/* Moving window (in the paper's gamma = 1 and gamma = 5 runs the box
   follows the laser, moving at its group velocity v_g in the plasma; section
   "Effect of the hyperbolic rotation in Minkowski space").  From
   simulation time t0 on the grid moves along +z at velocity v (0 < v <= 1, in
   c): after the TIME phase of a step at which v (t - t0) >= (n + 1) S hz (n
   the moves so far), it moves by shift_cells = S cells at once: every field
   plane k takes plane k + S and the top S planes become zero, particles move
   S cells down in the grid (those below z = 0 leave), the plasma of the newly
   covered layer enters at its position at that time, and the antenna, which
   stays where it was launched, is switched off once it is below plane 2.
   Positions, fields, rho and snapshots are relative to the window; its
   displacement n S hz is pic_diag.z_window.  S must be a positive multiple of
   the tile's z extent (8 in 3D, that of the tile shape in 2D) below nz, and z absorbing
   (PIC_BC_MUR); v = 0 switches the window off (PIC_ERR_ARG otherwise). */
pic_status pic_set_moving_window(pic_ctx *ctx, double v, double t0, int shift_cells);

/* ------------------------------------------------- lab-frame snapshots */

/* Lab-frame ("back-transformed") snapshots of a boosted run: the boosted data
   seen in laboratory coordinates after Lorentz transformation (section
   "Effect of the hyperbolic rotation in Minkowski space", Fig. 2).  Snapshot j
   holds the lab fields at lab time T_j = t0 + j dt on the lab points
   Z_k = z0 + k dz (k < nz): on the axis line (plane 0: the nodes i = nx/2,
   j = ny/2 of each component) or on the (x, z) plane j = ny/2 (plane 1, all
   nx columns).  A point is filled during the step whose interval
   [t'^n, t'^{n+1}) holds its simulation-frame time t' = gamma (T - beta Z),
   from the fields linear in t' between (E^n, B^n) and (E^{n+1}, B^{n+1}) and
   linear in z' = gamma (Z - beta T) between the planes of each component,
   transformed by
     Ex = gamma (Ex' + beta By'), Ey = gamma (Ey' - beta Bx'), Ez = Ez',
     Bx = gamma (Bx' - beta Ey'), By = gamma (By' + beta Ex'), Bz = Bz'.
   A point whose z' does not lie between two planes of every component stays
   unfilled (flag 0, fields 0).  Event times and weights are FP64; the fields
   are in the working precision. */
typedef struct pic_btd_params {
    int n_snapshots;           /* 1..64                                            */
    double t0, dt;             /* lab times of the snapshots, lambda0/c            */
    double z0, dz;             /* lab positions, lambda0 (dz > 0)                  */
    int nz;                    /* lab points per snapshot, >= 1                    */
    int plane;                 /* 0: axis line, 1: (x, z) plane                    */
} pic_btd_params;

/* Bytes of the caller-owned device buffer of the snapshots: n_snapshots
   blocks of [6 components: Ex Ey Ez Bx By Bz][nz][nxs] elements (elem_bytes
   each, nxs = 1 for plane 0, nx for plane 1), then n_snapshots x nz int32
   fill flags starting at a 256-byte boundary.  PIC_ERR_ARG for NULL
   arguments, invalid parameters or an unboosted grid. */
pic_status pic_btd_bytes(const pic_ctx *ctx, const pic_btd_params *p, size_t *bytes);

/* Zeroes buf (device memory of at least pic_btd_bytes, owned by the caller,
   which keeps it alive while snapshots are taken) and fills the snapshots
   from the next step's YEE phase on.  p == NULL stops.  PIC_ERR_ARG for an
   unboosted grid (gamma_boost = 1) or invalid parameters. */
pic_status pic_btd_setup(pic_ctx *ctx, const pic_btd_params *p, void *buf, size_t bytes);

/* Copies snapshot j to host or device memory: its [6][nz][nxs] elements,
   then its nz int32 flags (1: filled).  PIC_ERR_STATE when no snapshots are
   being taken, PIC_ERR_ARG for a NULL dst, j out of range or too small a
   destination. */
pic_status pic_btd_get(pic_ctx *ctx, int j, void *dst, size_t dst_bytes, int dst_is_device);

/* ---------------------------------------------------------------- adjoint */

/* Reverse-mode gradient of a run (2D3V or 3D, either shape, no moving window): the
   library's own extension of the method, built from the transposes of the
   step's maps (Yee with Mur's condition, filter, antenna, Esirkepov deposit,
   gather, Boris rotation, move).  The objective is linear in the final fields,
   L = sum(lambda_E E^N) + sum(lambda_B B^N) with caller-given cotangents; the
   gradient is taken with respect to the plasma profile coefficients c_1..c_M
   of pic_load_plasma (they scale every particle weight), the laser's a0 and
   its waist w0.  The run starts right after pic_load_plasma and
   pic_launch_laser (no step taken): pic_adjoint_forward regenerates the same
   plasma in a fixed-order particle store (slot p is one particle for the whole
   run), runs nsteps steps and keeps a checkpoint every checkpoint_every steps;
   pic_adjoint_backward recomputes each segment from its checkpoint and runs it
   backwards.  The context's own state is not changed. */
typedef struct {
    int nsteps;            /* N >= 1                                          */
    int checkpoint_every;  /* K >= 1: checkpoints at steps 0, K, 2K, ...      */
    int sub_checkpoint_every; /* K2: 0 (or >= K) one level: a segment's K + 1 */
                           /* states are all kept while it is reversed;       */
                           /* 0 < K2 < K: two levels: the segment is first    */
                           /* recomputed once leaving a state every K2 steps, */
                           /* then each K2-step piece is recomputed and       */
                           /* reversed, so K2 + 1 + ceil(K / K2) states are   */
                           /* kept instead of K + 1 (one more forward pass)   */
} pic_adjoint_params;

/* Bytes of the device buffer an adjoint run needs (ceil(N / K) checkpoints,
   one segment of K + 1 states or, with sub-checkpoints, K2 + 1 states and
   ceil(K / K2) sub-checkpoints, the cotangents).  PIC_ERR_ARG for an unsupported run,
   PIC_ERR_STATE if a step has been taken since pic_load_plasma.  (The
   library's adjoint: no counterpart in the paper.) */
pic_status pic_adjoint_bytes(pic_ctx *ctx, const pic_adjoint_params *p, size_t *bytes);

/* The forward run into buf (device memory of at least pic_adjoint_bytes bytes,
   owned by the caller and kept alive until pic_adjoint_backward).  fields_out
   (device, may be NULL) receives E^N, B^N: six components of (nz+1) ny nx
   elements (ny = 1 in 2D), Ex Ey Ez Bx By Bz.  The adjoint calls have no
   counterpart in the paper (see above).  PIC_ERR_ARG for an unsupported run
   (a moving window, invalid parameters) or too small a buffer, PIC_ERR_STATE
   before pic_bind_buffers or once a step has been taken. */
pic_status pic_adjoint_forward(pic_ctx *ctx, const pic_adjoint_params *p, void *buf, size_t bytes,
                               void *fields_out);

/* cot: device cotangents lambda_E, lambda_B of E^N, B^N (the layout of
   fields_out).  grad (host, M + 2 doubles): dL/dc_1 .. dL/dc_M, dL/da0,
   dL/dw0.  PIC_ERR_STATE without a preceding pic_adjoint_forward, or when
   pic_load_plasma or pic_launch_laser has been called since it (the gradient
   would belong to another run).  No counterpart in the paper. */
pic_status pic_adjoint_backward(pic_ctx *ctx, const void *cot, double *grad);

/* The gradients of every run of a batch (the scan's reverse mode): for run
   i, pic_adjoint_forward with p[i] into bufs[i] (bytes[i], from
   pic_adjoint_bytes) and pic_adjoint_backward with the device cotangents
   cots[i], its M_i + 2 sums written to grads + i * grad_stride (host;
   grad_stride >= max M_i + 2).  Every run's forward, then every run's
   reverse sweep is queued on its own stream without waiting for any of
   them, so the runs' adjoint kernels execute concurrently; the call returns
   after one wait per stream, with the first failure (each context's
   pic_last_error has its detail).  PIC_ERR_ARG for null arrays or too small
   a stride.  No counterpart in the paper. */
pic_status pic_batch_adjoint(pic_batch *batch, const pic_adjoint_params *p, void *const *bufs,
                             const size_t *bytes, const void *const *cots, double *grads, int grad_stride);

/* ------------------------------------------------------------ checkpoint */

/* Size of a compact snapshot (fields, live particles, time, laser) now.  The
   snapshot calls have no counterpart in the paper: checkpoint and restart of
   a run.  Each returns PIC_ERR_ARG for NULL arguments or too small a buffer
   and PIC_ERR_STATE before pic_bind_buffers. */
pic_status pic_state_bytes(pic_ctx *ctx, size_t *bytes);

/* Writes the snapshot to host or device memory (PIC_ERR_ARG if dst_bytes is
   smaller than pic_state_bytes). */
pic_status pic_get_state(pic_ctx *ctx, void *dst, size_t dst_bytes, int dst_is_device);

/* Restores a snapshot taken from a context with the same grid parameters.
   PIC_ERR_ARG if it does not match; PIC_ERR_CAPACITY on bucket overflow. */
pic_status pic_set_state(pic_ctx *ctx, const void *src, size_t src_bytes, int src_is_device);

/* ------------------------------------------------------------- cell order */

/* Orders every tile's bucket of each species by cell (the cell's index in its
   tile, x fastest, then y, then z; a counting sort per tile into the other
   half of the double buffer, all of a tile's records then in its bottom
   run).  The push writes the particles that stay in their tile in the order
   it read them, so the order decays only by the particles that cross tiles.
   The results of a step do not depend on the order (the deposit sums in
   exact fixed point).  Synchronises the stream.  PIC_ERR_STATE before
   pic_bind_buffers; the device error word is checked as after a step.  No
   counterpart in the paper: a memory order of the particle store. */
pic_status pic_sort_cells(pic_ctx *ctx);

/* Sort by cell before every `every`-th step (the step count a multiple of
   every; 0, the default: never).  A context that sorts is stepped launch by
   launch (a batch does not capture it in a graph).  PIC_ERR_ARG for
   every < 0.  No counterpart in the paper. */
pic_status pic_set_cell_sort(pic_ctx *ctx, int every);

/* -------------------------------------------------------------- profiling */

/* While enabled, every phase of later steps is bracketed by CUDA events on the
   context's stream and the kernels the library launches are counted.  No
   counterpart in the paper (measurement).  PIC_ERR_ARG for a NULL context. */
pic_status pic_profile(pic_ctx *ctx, int enable);

/* Accumulated device time since the last read: ms[i] milliseconds and calls[i]
   runs of phase bit i (i = 0..6, PIC_PH_ZERO_J .. PIC_PH_INJECT; slot 7, the
   TIME phase's, which launches nothing, holds the cell sorts of
   pic_set_cell_sort), *kernels the number of kernel launches.  Synchronises
   the stream and resets the sums.  Any output pointer may be NULL.  No
   counterpart in the paper.  PIC_ERR_ARG for a NULL context. */
pic_status pic_profile_read(pic_ctx *ctx, double ms[8], int64_t calls[8], int64_t *kernels);

/* --------------------------------------------- allocation-free current filter */

/* Largest field component, in nodes ((nz+1) * ny * nx), that
   pic_filter_current_noalloc accepts. */
#define PIC_NOALLOC_MAX_NODES 4194304

/* The binomial current filter of the FILTER phase, for callers that cannot
   allocate device memory: the rest of this library needs a caller-provided
   scratch buffer (pic_query_sizes / pic_bind_buffers), which a caller cannot
   supply when every byte of device memory is owned by another framework's
   allocator, or when it runs under a fixed device-memory budget or in a
   latency-critical loop that must never allocate.  The paper has no
   counterpart of this entry point; it is a deployment variant of the FILTER
   phase and computes the same thing: `passes` (1/4, 1/2, 1/4) passes along x,
   then y (3D), then z, on each of Jx, Jy, Jz in place, with the same boundary
   rules (x, y periodic; z periodic or zero outside each component's valid z
   range).

   jx, jy, jz: device arrays of (nz+1) * ny * nx elements (float for
   precision PIC_FP32, double for PIC_FP64) in the library's [k][j][i] layout;
   ny must be 1 when dim == 2.  Work is enqueued on `stream` (a cudaStream_t,
   NULL: legacy default stream) and the call returns without synchronising.

   Scratch: one field component lives in a file-scope device array of
   PIC_NOALLOC_MAX_NODES doubles (32 MiB) that every GPU which loads the
   library holds until the process exits.  The call allocates and frees
   nothing.  The first call on a device (the current device at the time of
   the call) looks up that array's device address once (cudaGetSymbolAddress);
   make that first call before any stream capture.  Every call shares the one
   array, which keeps the last call's contents; nothing in it needs to start at
   zero because every pass writes each element before it is read.  Calls whose
   work overlaps on the GPU (different streams, or other threads) race on the
   array: issue them one after another, e.g. on one stream.

   Errors: PIC_ERR_ARG for an invalid dimension, size, boundary, precision or
   null pointer, and when (nz+1) * ny * nx exceeds PIC_NOALLOC_MAX_NODES;
   PIC_ERR_CUDA if a CUDA call fails.  No context is involved, so there is no
   pic_last_error detail. */
pic_status pic_filter_current_noalloc(int dim, int nx, int ny, int nz, int bc_z, int passes, int precision,
                                      void *jx, void *jy, void *jz, void *stream);

/* ------------------------------------------------------- bounded waits */

/* Kernels that stage data with the tensor memory accelerator wait on
   mbarriers; no such wait spins without limit: it gives up after a time
   budget, the kernel stops issuing work, and the step reports
   PIC_ERR_TIMEOUT instead of hanging.  This call checks that path on the
   device: one CTA waits on an mbarrier that expects one arrival, which the
   kernel makes (arrive = 1: PIC_OK) or withholds (arrive = 0: nothing ever
   completes the phase, the wait runs out after budget_ms and the call
   returns PIC_ERR_TIMEOUT).  No fault is raised either way.  budget_ms in
   (0, 10000], else PIC_ERR_ARG; PIC_ERR_CUDA if a CUDA call fails.  The
   paper has no counterpart: this is a check of the library's own waits. */
pic_status pic_wait_check(int arrive, double budget_ms, void *stream);

/* ------------------------------------------------------------------ misc */

const char *pic_last_error(const pic_ctx *ctx);
const char *pic_status_string(pic_status s);
void pic_destroy(pic_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* PIC_H */
