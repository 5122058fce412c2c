/*
 * pic_oracle.h -- FP64 CPU oracle of the boosted-frame electromagnetic PIC step.
 *
 * TEST INFRASTRUCTURE ONLY.  A plain, slow, single-threaded restatement of the
 * method (field gather, relativistic Boris push, Esirkepov charge-conserving
 * deposition, binomial current filter, Yee FDTD update with first-order Mur
 * boundaries, boosted-frame plasma injection and a laser antenna at rest in the
 * simulation frame).  The CUDA library is checked against it; it shares no code,
 * header, table or helper with that library.  Only the tests, the smoke check and
 * the benchmark's CPU-baseline leg load it.
 *
 * Units: lengths in the laser wavelength lambda0, times in lambda0/c, c = 1,
 * fields in m c omega0 / e (a linearly polarised laser has peak E = a0), densities
 * in the critical density n_c, currents in e n_c c.  With these units
 *     du/dt = 2 pi (q/m) (E + v x B),   dE/dt = curl B - 2 pi J,   dB/dt = -curl E,
 *     div E = 2 pi rho.
 *
 * Parity status of each function is stated beside it; every function listed
 * here is pinned by a closed form or an invariant in the oracle's own tests.
 */
#ifndef PIC_ORACLE_H
#define PIC_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* field component order of every field array */
enum { OPIC_EX = 0, OPIC_EY, OPIC_EZ, OPIC_BX, OPIC_BY, OPIC_BZ, OPIC_JX, OPIC_JY, OPIC_JZ, OPIC_NCOMP };

/* phases of one step (a full step is OPIC_PH_ALL) */
#define OPIC_PH_ZERO_J   1u   /* J = 0                                        */
#define OPIC_PH_PUSH     2u   /* electrons: gather, Boris, move, deposit, BCs */
#define OPIC_PH_IONS     4u   /* drifting ions: move, deposit, BCs            */
#define OPIC_PH_ANTENNA  8u   /* laser antenna current at t + dt/2            */
#define OPIC_PH_FILTER  16u   /* binomial passes on Jx, Jy, Jz                */
#define OPIC_PH_YEE     32u   /* B half step, E full step (+Mur), B half step */
#define OPIC_PH_INJECT  64u   /* plasma entering through z = Lz during the step */
#define OPIC_PH_TIME   128u   /* t += dt                                      */
#define OPIC_PH_ALL    255u

/* particle attribute order of opic_particles() */
enum { OPIC_PX = 0, OPIC_PY, OPIC_PZ, OPIC_PUX, OPIC_PUY, OPIC_PUZ, OPIC_PW, OPIC_NATTR };

typedef struct opic opic;

typedef struct opic_grid {
    int dim;                 /* 2: (x, z) with y ignorable; 3: (x, y, z)      */
    int nx, ny, nz;          /* cells; ny is ignored (1) in 2D               */
    double dx, dy, dz;       /* lab-frame cell sizes in lambda0             */
    double cfl;              /* dt = cfl * Courant limit                     */
    double gamma_boost;      /* >= 1                                         */
    int shape;               /* 1: linear (CIC), 2: quadratic spline         */
    int npass;               /* binomial passes per axis                     */
    int bc_z;                /* 0: periodic z, 1: Mur absorbing z            */
    uint64_t seed;           /* SplitMix64 seed of the plasma jitter         */
} opic_grid;

typedef struct opic_plasma {
    double ne;               /* lab-frame electron density / n_c             */
    double z_start, z_end;   /* lab-frame extent of the plasma, lambda0      */
    double ramp;             /* length of the linear up-ramp, lambda0        */
    int ppc[3];              /* lattice points per cell and axis            */
    double jitter;           /* half width of the uniform jitter, in cells   */
    int nprof;               /* number of cosine profile coefficients        */
    const double *prof;      /* c_m, m = 1..nprof                            */
    int ions;                /* 1: ions immobile in the lab frame           */
} opic_plasma;

typedef struct opic_laser {
    double a0;               /* peak normalised vector potential (lab)       */
    double waist;            /* 1/e field radius, lambda0                    */
    double fwhm;             /* intensity FWHM duration, lambda0/c (lab)     */
    double z_antenna;        /* antenna plane position, simulation frame     */
    double t_peak;           /* envelope peak, lab retarded time; <0: 3 tau  */
    int pol;                 /* 0: E along x, 1: E along y                   */
    double xc, yc;           /* transverse centre; NaN: box centre           */
} opic_laser;

/* Lab-frame snapshots of a boosted-frame run (the paper shows its boosted
   results transformed back to laboratory coordinates; section "Effect of the
   hyperbolic rotation in Minkowski space", Fig. 2).  Snapshot j
   holds the lab-frame fields at lab time T_j = t0 + j dt on the lab points
   Z_k = z0 + k dz, k < nz; each is filled during the boosted step whose time
   interval [t'^n, t'^{n+1}) contains the event's boosted time.  Parity
   status: pinned (uniform fields transform exactly; lab-frame and boosted-frame
   runs of one pulse agree). */
typedef struct opic_btd {
    int nsnap;               /* number of lab snapshots, 1..64                */
    double t0, dt;           /* lab times T_j = t0 + j dt, lambda0/c          */
    double z0, dz;           /* lab positions Z_k = z0 + k dz, lambda0        */
    int nz;                  /* lab points per snapshot                       */
    int plane;               /* 0: the axis line (i = nx/2, j = ny/2);        */
                             /* 1: the (x, z) plane j = ny/2 (all i)          */
} opic_btd;

opic *opic_create(const opic_grid *g);
void opic_destroy(opic *s);

/* derived simulation-frame quantities:
   out[0]=dt out[1]=hx out[2]=hy out[3]=hz out[4]=beta out[5]=Lx out[6]=Ly out[7]=Lz */
void opic_info(const opic *s, double out[8]);
double opic_time(const opic *s);
int64_t opic_steps(const opic *s);

/* plasma loading (lattice + jitter, boosted to the simulation frame); returns
   the number of electrons placed in the box, or -1 on bad arguments */
int64_t opic_load_plasma(opic *s, const opic_plasma *p);
int64_t opic_pending(const opic *s);
void opic_set_laser(opic *s, const opic_laser *l);

/* explicit particle states (species 0 electrons, 1 drifting ions) */
int opic_add_particles(opic *s, int sp, int64_t n, const double *x, const double *y,
                       const double *z, const double *ux, const double *uy,
                       const double *uz, const double *w, const int64_t *id);
int64_t opic_num(const opic *s, int sp);
double *opic_particles(opic *s, int sp, int attr);
int64_t *opic_ids(opic *s, int sp);

/* field component c: (nz+1)*ny*nx doubles, index (k*ny + j)*nx + i */
double *opic_field(opic *s, int c);
double *opic_rho_background(opic *s);

void opic_step(opic *s, int nsteps);
void opic_step_phases(opic *s, unsigned mask);

/* Moving window (in the paper's gamma = 1 and 5 runs the box moves with the
   laser at its group velocity v_g; section "Effect of the hyperbolic rotation
   in Minkowski space").  From time t0 on, the window (the grid) moves
   along +z at velocity v (0 < v <= 1); whenever its displacement
   v (t - t0) reaches (n + 1) S hz after the TIME phase, the window moves by S
   cells at once (n counts the moves): every field plane k takes plane k + S,
   the top S planes become zero, particle z decreases by S hz (particles below
   z = 0 are removed), the antenna plane moves S planes down (it stops below
   plane 2), and the plasma of the newly covered layer enters (in the lab
   frame with its immobile ions' background, as at load).  Positions stay
   relative to the window; opic_window() is its displacement n S hz.  Parity
   status: pinned (a pulse in the window matches the same pulse in a long
   fixed box, also while the antenna still emits; a static plasma seen through
   the window is the lattice, a boosted one the long box's, and a lab plasma
   stays neutral; the moves follow the schedule). */
int opic_set_window(opic *s, double v, double t0, int S);   /* 0, or -1 on bad arguments */
double opic_window(const opic *s);

/* back-transformed snapshots: setup (0, or -1 on bad arguments or gamma = 1;
   NULL switches them off), then per snapshot j the fields [6][nz][nxs]
   (Ex Ey Ez Bx By Bz, nxs = 1 or nx) and nz fill flags */
int opic_btd_setup(opic *s, const opic_btd *b);
double *opic_btd_data(opic *s, int j);
unsigned char *opic_btd_filled(opic *s, int j);

/* Diagnostics of the state, FP64 Kahan-compensated sums: out[0] the field
   energy (1/2) sum (E^2 + B^2) V, out[1] the electrons' kinetic energy
   sum w (gamma - 1), out[2] the particles' charge sum q w (electrons -1,
   drifting ions +1), all in n_c m c^2 lambda0^3 (charge in e n_c lambda0^3).
   Parity status: pinned (energy of uniform and single-mode fields from
   discrete orthogonality, kinetic energy and charge of a cold boosted plasma
   from the Lorentz factor and the loaded density, and the conservation of
   field plus kinetic energy through a plasma oscillation). */
void opic_diagnostics(const opic *s, double out[3]);

/* Lab-frame E, B on the simulation grid at the current time (inverse field
   transformation of the boost; each component at its own Yee position, the
   partner it mixes with averaged over its two planes around it):
   out = 6 arrays of (nz+1)*ny*nx doubles, Ex Ey Ez Bx By Bz.  Parity status:
   pinned (uniformly moving charges' fields and the invariants E.B, E^2-B^2). */
void opic_fields_lab(const opic *s, double *out);

/* building blocks exposed for the oracle's own pins */
void opic_gather(const opic *s, int64_t n, const double *x, const double *y,
                 const double *z, double *eb /* n x 6 */);
void opic_boris(double u[3], const double e[3], const double b[3], double q_over_m, double dt);
void opic_deposit_current(opic *s, double qw, const double x0[3], const double x1[3], double vy);
void opic_deposit_rho(const opic *s, double *rho /* (nz+1)*ny*nx */);
void opic_filter(opic *s);
double opic_density(const opic_plasma *p, double z_lab);
double opic_shape(int order, double d);
uint64_t opic_splitmix64(uint64_t seed, uint64_t counter);
double opic_uniform(uint64_t seed, uint64_t counter);

#ifdef __cplusplus
}
#endif
#endif
