/*
 * pic_oracle.c -- FP64 CPU oracle of the boosted-frame electromagnetic PIC step.
 *
 * TEST INFRASTRUCTURE ONLY (see pic_oracle.h).  Plain loops, no blocking, no
 * fusion: each routine follows the textbook definition it names, in the order
 * the step applies them.  The paper (Vay et al., "Effects of hyperbolic rotation
 * in Minkowski space on the modeling of plasma accelerators in a Lorentz boosted
 * frame") names the method -- a PIC code run in a frame boosted along the laser
 * axis (introduction; section "Effect of the hyperbolic rotation in Minkowski
 * space"), with current filtering to keep short wavelengths in check (section
 * "Mitigation of a numerical instability") -- but prints none of the per-step
 * algorithms.  Each one below is the standard published scheme:
 *   gather:   direct interpolation with the same B-spline order on every
 *             staggered component;
 *   push:     relativistic Boris rotation (Boris 1970);
 *   deposit:  Esirkepov's charge-conserving density decomposition (Esirkepov 2001);
 *   filter:   (1/4, 1/2, 1/4) binomial passes along each axis;
 *   fields:   Yee staggered leapfrog (Yee 1966), B split in two half steps so
 *             that E and B live at integer times, Mur first-order absorbing
 *             boundaries in z (Mur 1981);
 *   frame:    Lorentz transform z' = z/gamma - beta t' of a plasma at rest in
 *             the lab, laser Doppler factor gamma (1 - beta) (the hyperbolic
 *             rotation of the paper's second section);
 *   jitter:   SplitMix64 (Steele, Lea, Flood 2014) as a counter-based generator.
 * Parity: every routine is pinned by the oracle's tests (closed forms and
 * invariants); none is "parity unpinned".
 */
#include "pic_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define TWO_PI 6.283185307179586
#define PI_ 3.141592653589793

typedef struct species {
    int64_t n, cap;
    double *a[OPIC_NATTR];
    int64_t *id;
} species;

typedef struct pending_particle {
    double x, y, zlab, w;
    int64_t id;
} pending_particle;

struct opic {
    opic_grid g;
    double hx, hy, hz, dt, beta, gam, Lx, Ly, Lz;
    int ny;               /* 1 in 2D */
    int64_t nn;           /* (nz+1)*ny*nx */
    double *f[OPIC_NCOMP];
    double *rho_bg;
    species sp[2];
    pending_particle *pend;
    int64_t npend, cappend;
    double ion_u[3];
    int has_ions;
    int bg_ions;          /* lab frame: immobile ions as a static background */
    int laser_on;
    opic_laser las;
    int ka;
    double t;
    int64_t step;
    /* moving window */
    int win_on;
    double win_v, win_t0;
    int win_S;
    int64_t win_n;
    /* back-transformed snapshots */
    int btd_on;
    opic_btd btd;
    int btd_nxs;
    double *btd_data;        /* [nsnap][6][nz][nxs] */
    unsigned char *btd_fill; /* [nsnap][nz] */
    double *btd_prev[6];     /* E, B at the start of the step */
};

/* ------------------------------------------------------------------ utils */

static int64_t fidx(const opic *s, int64_t i, int64_t j, int64_t k)
{
    return (k * s->ny + j) * s->g.nx + i;
}

static int64_t wrap_index(int64_t i, int64_t n)
{
    int64_t r = i % n;
    return r < 0 ? r + n : r;
}

/* SplitMix64, the (counter+1)-th output of the sequence whose state starts at
   `seed` and advances by the golden-ratio increment 0x9E3779B97F4A7C15. */
uint64_t opic_splitmix64(uint64_t seed, uint64_t counter)
{
    uint64_t z = seed + (counter + 1u) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* uniform double in [0, 1) from the top 53 bits */
double opic_uniform(uint64_t seed, uint64_t counter)
{
    return (double)(opic_splitmix64(seed, counter) >> 11) * (1.0 / 9007199254740992.0);
}

/* B-spline shape of order 1 (linear) or 2 (quadratic) at distance d (cells). */
double opic_shape(int order, double d)
{
    double a = fabs(d);
    if (order == 1)
        return a < 1.0 ? 1.0 - a : 0.0;
    if (a < 0.5)
        return 0.75 - a * a;
    if (a < 1.5) {
        double b = 1.5 - a;
        return 0.5 * b * b;
    }
    return 0.0;
}

/* ------------------------------------------------------------ life cycle */

opic *opic_create(const opic_grid *g)
{
    if (!g || (g->dim != 2 && g->dim != 3) || g->nx < 1 || g->nz < 2 ||
        (g->dim == 3 && g->ny < 1) || g->shape < 1 || g->shape > 2 ||
        g->gamma_boost < 1.0 || g->cfl <= 0.0 || g->npass < 0)
        return NULL;
    opic *s = (opic *)calloc(1, sizeof(opic));
    s->g = *g;
    s->ny = g->dim == 3 ? g->ny : 1;
    s->gam = g->gamma_boost;
    /* beta from gamma; simulation-frame cell sizes: the transverse ones are
       invariant, the longitudinal one is the lab one times gamma (1 + beta) so
       that the Doppler-stretched laser wavelength keeps its cells per period */
    s->beta = sqrt(1.0 - 1.0 / (s->gam * s->gam));
    s->hx = g->dx;
    s->hy = g->dim == 3 ? g->dy : 1.0;
    s->hz = g->dz * (s->gam * (1.0 + s->beta));
    if (g->dim == 3)
        s->dt = g->cfl / sqrt(1.0 / (s->hx * s->hx) + 1.0 / (s->hy * s->hy) + 1.0 / (s->hz * s->hz));
    else
        s->dt = g->cfl / sqrt(1.0 / (s->hx * s->hx) + 1.0 / (s->hz * s->hz));
    s->Lx = g->nx * s->hx;
    s->Ly = s->ny * s->hy;
    s->Lz = g->nz * s->hz;
    s->nn = (int64_t)(g->nz + 1) * s->ny * g->nx;
    for (int c = 0; c < OPIC_NCOMP; ++c)
        s->f[c] = (double *)calloc((size_t)s->nn, sizeof(double));
    s->rho_bg = (double *)calloc((size_t)s->nn, sizeof(double));
    s->ion_u[0] = 0.0;
    s->ion_u[1] = 0.0;
    s->ion_u[2] = -(s->gam * s->beta);
    return s;
}

void opic_destroy(opic *s)
{
    if (!s)
        return;
    for (int c = 0; c < OPIC_NCOMP; ++c)
        free(s->f[c]);
    free(s->rho_bg);
    for (int sp = 0; sp < 2; ++sp) {
        for (int a = 0; a < OPIC_NATTR; ++a)
            free(s->sp[sp].a[a]);
        free(s->sp[sp].id);
    }
    free(s->pend);
    free(s->btd_data);
    free(s->btd_fill);
    for (int c = 0; c < 6; ++c)
        free(s->btd_prev[c]);
    free(s);
}

void opic_info(const opic *s, double out[8])
{
    out[0] = s->dt;
    out[1] = s->hx;
    out[2] = s->hy;
    out[3] = s->hz;
    out[4] = s->beta;
    out[5] = s->Lx;
    out[6] = s->Ly;
    out[7] = s->Lz;
}

double opic_time(const opic *s) { return s->t; }
int64_t opic_steps(const opic *s) { return s->step; }
double *opic_field(opic *s, int c) { return (c >= 0 && c < OPIC_NCOMP) ? s->f[c] : NULL; }
double *opic_rho_background(opic *s) { return s->rho_bg; }
int64_t opic_num(const opic *s, int sp) { return (sp == 0 || sp == 1) ? s->sp[sp].n : -1; }
int64_t opic_pending(const opic *s) { return s->npend; }

double *opic_particles(opic *s, int sp, int attr)
{
    if ((sp != 0 && sp != 1) || attr < 0 || attr >= OPIC_NATTR)
        return NULL;
    return s->sp[sp].a[attr];
}

int64_t *opic_ids(opic *s, int sp) { return (sp == 0 || sp == 1) ? s->sp[sp].id : NULL; }

/* --------------------------------------------------------- particle store */

static void species_reserve(species *p, int64_t need)
{
    if (need <= p->cap)
        return;
    int64_t cap = p->cap ? p->cap : 1024;
    while (cap < need)
        cap *= 2;
    for (int a = 0; a < OPIC_NATTR; ++a)
        p->a[a] = (double *)realloc(p->a[a], (size_t)cap * sizeof(double));
    p->id = (int64_t *)realloc(p->id, (size_t)cap * sizeof(int64_t));
    p->cap = cap;
}

static void species_push(species *p, double x, double y, double z, double ux, double uy,
                         double uz, double w, int64_t id)
{
    species_reserve(p, p->n + 1);
    int64_t k = p->n++;
    p->a[OPIC_PX][k] = x;
    p->a[OPIC_PY][k] = y;
    p->a[OPIC_PZ][k] = z;
    p->a[OPIC_PUX][k] = ux;
    p->a[OPIC_PUY][k] = uy;
    p->a[OPIC_PUZ][k] = uz;
    p->a[OPIC_PW][k] = w;
    p->id[k] = id;
}

static void species_remove(species *p, int64_t k)
{
    int64_t last = p->n - 1;
    if (k != last) {
        for (int a = 0; a < OPIC_NATTR; ++a)
            p->a[a][k] = p->a[a][last];
        p->id[k] = p->id[last];
    }
    p->n = last;
}

int opic_add_particles(opic *s, int sp, int64_t n, const double *x, const double *y,
                       const double *z, const double *ux, const double *uy,
                       const double *uz, const double *w, const int64_t *id)
{
    if (sp != 0 && sp != 1)
        return -1;
    for (int64_t k = 0; k < n; ++k)
        species_push(&s->sp[sp], x[k], y ? y[k] : 0.0, z[k], ux[k], uy[k], uz[k], w[k],
                     id ? id[k] : k);
    if (sp == 1)
        s->has_ions = 1;
    return 0;
}

/* ------------------------------------------------------------- plasma load */

/* lab-frame density n(z): linear up-ramp from z_start over `ramp`, then the
   cosine-series profile n0 (1 + sum_m c_m cos(m pi zeta)), zeta = (z - z_start)/L */
double opic_density(const opic_plasma *p, double z)
{
    if (z < p->z_start || z >= p->z_end)
        return 0.0;
    double r = 1.0;
    if (p->ramp > 0.0 && z < p->z_start + p->ramp)
        r = (z - p->z_start) / p->ramp;
    double f = 1.0;
    if (p->nprof > 0) {
        double zeta = (z - p->z_start) / (p->z_end - p->z_start);
        for (int m = 1; m <= p->nprof; ++m)
            f += p->prof[m - 1] * cos((double)m * PI_ * zeta);
    }
    return p->ne * r * f;
}

static void deposit_rho_species(const opic *s, const species *p, int64_t from, double q, double *rho);

int64_t opic_load_plasma(opic *s, const opic_plasma *p)
{
    if (!p || p->ppc[0] < 1 || p->ppc[2] < 1 || (s->g.dim == 3 && p->ppc[1] < 1) ||
        p->z_end <= p->z_start || p->ne < 0.0 || p->jitter < 0.0 || p->jitter >= 0.5)
        return -1;
    const int dim3 = s->g.dim == 3;
    const int ppx = p->ppc[0], ppy = dim3 ? p->ppc[1] : 1, ppz = p->ppc[2];
    const int64_t NX = (int64_t)s->g.nx * ppx;
    const int64_t NY = dim3 ? (int64_t)s->g.ny * ppy : 1;
    /* lab-frame length of one simulation cell at fixed simulation time */
    const double hz_lab = s->gam * s->hz;
    const double dzl = hz_lab / (double)ppz;
    const int64_t MZ = (int64_t)ceil((p->z_end - p->z_start) / dzl);
    const double vol = dim3 ? s->hx * s->hy * s->hz : s->hx * s->hz;
    const double wfac = s->gam * vol / (double)(ppx * ppy * ppz);
    const double uz0 = -(s->gam * s->beta);
    const int boosted = s->gam > 1.0;
    const int drift_ions = p->ions && boosted;
    int64_t placed = 0;

    for (int64_t m = 0; m < MZ; ++m) {
        for (int64_t iy = 0; iy < NY; ++iy) {
            for (int64_t ix = 0; ix < NX; ++ix) {
                const int64_t L = (m * NY + iy) * NX + ix;
                const uint64_t c0 = 3u * (uint64_t)L;
                double x = ((double)ix + 0.5) * (s->hx / (double)ppx) +
                           (p->jitter * s->hx) * (2.0 * opic_uniform(s->g.seed, c0) - 1.0);
                if (x < 0.0)
                    x += s->Lx;
                if (x >= s->Lx)
                    x -= s->Lx;
                double y = 0.0;
                if (dim3) {
                    y = ((double)iy + 0.5) * (s->hy / (double)ppy) +
                        (p->jitter * s->hy) * (2.0 * opic_uniform(s->g.seed, c0 + 1u) - 1.0);
                    if (y < 0.0)
                        y += s->Ly;
                    if (y >= s->Ly)
                        y -= s->Ly;
                }
                const double zlab = p->z_start + ((double)m + 0.5) * dzl +
                                    (p->jitter * hz_lab) * (2.0 * opic_uniform(s->g.seed, c0 + 2u) - 1.0);
                const double n = opic_density(p, zlab);
                if (!(n > 0.0))
                    continue;
                const double w = n * wfac;
                /* simulation-frame position at the current time, relative to
                   the window */
                const double zb = zlab / s->gam - s->beta * s->t - opic_window(s);
                if (zb >= 0.0 && zb < s->Lz) {
                    species_push(&s->sp[0], x, y, zb, 0.0, 0.0, uz0, w, L);
                    if (drift_ions)
                        species_push(&s->sp[1], x, y, zb, 0.0, 0.0, uz0, w, L);
                    ++placed;
                } else if (zb >= s->Lz) {
                    /* ahead of the box: enters later (drifting in, or when the
                       window moves over it) */
                    if (s->npend == s->cappend) {
                        s->cappend = s->cappend ? 2 * s->cappend : 1024;
                        s->pend = (pending_particle *)realloc(s->pend, (size_t)s->cappend * sizeof(pending_particle));
                    }
                    pending_particle *q = &s->pend[s->npend++];
                    q->x = x;
                    q->y = y;
                    q->zlab = zlab;
                    q->w = w;
                    q->id = L;
                }
            }
        }
    }
    if (drift_ions)
        s->has_ions = 1;
    if (p->ions && !boosted) {
        /* immobile lab-frame ions: a static background equal and opposite to
           the electron charge at load time */
        memset(s->rho_bg, 0, (size_t)s->nn * sizeof(double));
        deposit_rho_species(s, &s->sp[0], 0, 1.0, s->rho_bg);
        s->bg_ions = 1;
    }
    return placed;
}

/* plasma whose simulation-frame position z/gamma - beta t1, relative to the
   window, is below Lz enters the box there: called for t1 = t + dt (the
   plasma that crossed z = Lz during the step) and after a window move */
static void inject_at(opic *s, double t1)
{
    const double uz0 = -(s->gam * s->beta);
    int64_t k = 0;
    while (k < s->npend) {
        pending_particle *q = &s->pend[k];
        const double zb = q->zlab / s->gam - s->beta * t1 - opic_window(s);
        if (zb < s->Lz) {
            species_push(&s->sp[0], q->x, q->y, zb, 0.0, 0.0, uz0, q->w, q->id);
            if (s->has_ions)
                species_push(&s->sp[1], q->x, q->y, zb, 0.0, 0.0, uz0, q->w, q->id);
            s->pend[k] = s->pend[--s->npend];
        } else {
            ++k;
        }
    }
}

static void inject(opic *s) { inject_at(s, s->t + s->dt); }

/* ------------------------------------------------------------------ laser */

void opic_set_laser(opic *s, const opic_laser *l)
{
    s->las = *l;
    s->laser_on = 1;
    int ka = (int)floor(l->z_antenna / s->hz + 0.5);
    if (ka < 2)
        ka = 2;
    if (ka > s->g.nz - 2)
        ka = s->g.nz - 2;
    s->ka = ka;
    if (isnan(s->las.xc))
        s->las.xc = 0.5 * s->Lx;
    if (isnan(s->las.yc))
        s->las.yc = 0.5 * s->Ly;
}

/* Current sheet on plane k_a.  A sheet current K radiates E = -pi K each way in
   these units, so J = -E_target / (pi hz) puts the target field in the forward
   wave.  In the boosted frame the antenna is at rest; the lab field at its
   position, seen there, is multiplied by D = gamma (1 - beta) and its time
   argument by D (plane-wave Doppler transform along the boost). */
static void antenna(opic *s)
{
    /* the antenna stays where it was launched; the window moves past it */
    const int64_t ka = s->ka - s->win_n * s->win_S;
    if (ka < 2)
        return;
    const opic_laser *l = &s->las;
    const double D = 1.0 / (s->gam * (1.0 + s->beta));
    const double tau = l->fwhm / sqrt(2.0 * log(2.0));
    const double spk = l->t_peak >= 0.0 ? l->t_peak : 3.0 * tau;
    const double th = s->t + 0.5 * s->dt;
    const double sr = D * th - spk;
    const double env = exp(-(sr / tau) * (sr / tau));
    const double amp = l->a0 * D * env * sin(TWO_PI * sr);
    const double j0 = -amp / (PI_ * s->hz);
    const int c = l->pol == 0 ? OPIC_JX : OPIC_JY;
    const double sx = l->pol == 0 ? 0.5 : 0.0;
    const double sy = (l->pol == 1 && s->g.dim == 3) ? 0.5 : 0.0;
    for (int j = 0; j < s->ny; ++j) {
        const double y = ((double)j + sy) * s->hy;
        for (int i = 0; i < s->g.nx; ++i) {
            const double x = ((double)i + sx) * s->hx;
            double r2 = (x - l->xc) * (x - l->xc);
            if (s->g.dim == 3)
                r2 += (y - l->yc) * (y - l->yc);
            s->f[c][fidx(s, i, j, ka)] += j0 * exp(-r2 / (l->waist * l->waist));
        }
    }
}

/* ------------------------------------------------------------------ gather */

/* Highest valid z index of a component: nodes 0..nz for integer-z components,
   half nodes 0..nz-1 for half-integer ones; periodic z wraps over nz. */
static int zmax_of(const opic *s, double sz)
{
    if (s->g.bc_z == 0)
        return s->g.nz - 1;
    return sz > 0.0 ? s->g.nz - 1 : s->g.nz;
}

/* staggering of each component (x, y, z offsets in cells) on the Yee lattice */
static const double STAG[OPIC_NCOMP][3] = {
    {0.5, 0.0, 0.0}, /* Ex (i+1/2, j,     k    ) */
    {0.0, 0.5, 0.0}, /* Ey (i,     j+1/2, k    ) */
    {0.0, 0.0, 0.5}, /* Ez (i,     j,     k+1/2) */
    {0.0, 0.5, 0.5}, /* Bx (i,     j+1/2, k+1/2) */
    {0.5, 0.0, 0.5}, /* By (i+1/2, j,     k+1/2) */
    {0.5, 0.5, 0.0}, /* Bz (i+1/2, j+1/2, k    ) */
    {0.5, 0.0, 0.0}, /* Jx */
    {0.0, 0.5, 0.0}, /* Jy */
    {0.0, 0.0, 0.5}, /* Jz */
};

/* value of component c interpolated with the shape of the grid's order at the
   position (x, y, z): sum over nodes of F * S(x-node) S(y-node) S(z-node) */
static double gather_comp(const opic *s, int c, double x, double y, double z)
{
    const int S = s->g.shape;
    const double xi = x / s->hx - STAG[c][0];
    const double zi = z / s->hz - STAG[c][2];
    const int64_t bx = (int64_t)floor(xi) - 1, bz = (int64_t)floor(zi) - 1;
    const int zmax = zmax_of(s, STAG[c][2]);
    double yi = 0.0;
    int64_t by = 0;
    int ny_loop = 1;
    if (s->g.dim == 3) {
        yi = y / s->hy - STAG[c][1];
        by = (int64_t)floor(yi) - 1;
        ny_loop = 4;
    }
    double sum = 0.0;
    for (int cz = 0; cz < 4; ++cz) {
        int64_t k = bz + cz;
        double wz = opic_shape(S, zi - (double)k);
        if (wz == 0.0)
            continue;
        if (s->g.bc_z == 0)
            k = wrap_index(k, s->g.nz);
        else if (k < 0 || k > zmax)
            continue;
        for (int cy = 0; cy < ny_loop; ++cy) {
            int64_t j = 0;
            double wy = 1.0;
            if (s->g.dim == 3) {
                j = by + cy;
                wy = opic_shape(S, yi - (double)j);
                if (wy == 0.0)
                    continue;
                j = wrap_index(j, s->g.ny);
            }
            for (int cx = 0; cx < 4; ++cx) {
                int64_t i = bx + cx;
                double wx = opic_shape(S, xi - (double)i);
                if (wx == 0.0)
                    continue;
                i = wrap_index(i, s->g.nx);
                sum += s->f[c][fidx(s, i, j, k)] * wx * wy * wz;
            }
        }
    }
    return sum;
}

void opic_gather(const opic *s, int64_t n, const double *x, const double *y, const double *z,
                 double *eb)
{
    for (int64_t p = 0; p < n; ++p)
        for (int c = 0; c < 6; ++c)
            eb[6 * p + c] = gather_comp(s, c, x[p], y ? y[p] : 0.0, z[p]);
}

/* ------------------------------------------------------------------- Boris */

/* relativistic Boris rotation for du/dt = 2 pi (q/m)(E + u x B / gamma) */
void opic_boris(double u[3], const double e[3], const double b[3], double q_over_m, double dt)
{
    const double eps = PI_ * q_over_m * dt; /* (2 pi q/m) dt / 2 */
    double um[3], t[3], sv[3], up[3], upl[3];
    for (int d = 0; d < 3; ++d)
        um[d] = u[d] + eps * e[d];
    const double gm = sqrt(1.0 + um[0] * um[0] + um[1] * um[1] + um[2] * um[2]);
    for (int d = 0; d < 3; ++d)
        t[d] = eps * b[d] / gm;
    const double t2 = t[0] * t[0] + t[1] * t[1] + t[2] * t[2];
    for (int d = 0; d < 3; ++d)
        sv[d] = 2.0 * t[d] / (1.0 + t2);
    up[0] = um[0] + (um[1] * t[2] - um[2] * t[1]);
    up[1] = um[1] + (um[2] * t[0] - um[0] * t[2]);
    up[2] = um[2] + (um[0] * t[1] - um[1] * t[0]);
    upl[0] = um[0] + (up[1] * sv[2] - up[2] * sv[1]);
    upl[1] = um[1] + (up[2] * sv[0] - up[0] * sv[2]);
    upl[2] = um[2] + (up[0] * sv[1] - up[1] * sv[0]);
    for (int d = 0; d < 3; ++d)
        u[d] = upl[d] + eps * e[d];
}

/* ------------------------------------------------------------- Esirkepov */

static void add_j(opic *s, int c, int64_t i, int64_t j, int64_t k, double v)
{
    if (v == 0.0)
        return;
    i = wrap_index(i, s->g.nx);
    if (s->g.dim == 3)
        j = wrap_index(j, s->g.ny);
    else
        j = 0;
    if (s->g.bc_z == 0)
        k = wrap_index(k, s->g.nz);
    else if (k < 0 || k > zmax_of(s, STAG[c][2]))
        return;
    s->f[c][fidx(s, i, j, k)] += v;
}

/* Esirkepov's decomposition of the change of the particle's density into
   currents that satisfy the discrete continuity equation exactly.  For each
   axis, S0 / S1 are the 1D shape weights at the old and new positions and
   DS = S1 - S0 on a common node range; the 3D weights are
     Wx = DSx (S0y S0z + DSy S0z / 2 + S0y DSz / 2 + DSy DSz / 3)  (cyclic),
   and J along an axis is the running sum  J(i+1/2) - J(i-1/2) = -(q w h/(dt V)) W(i).
   In 2D the out-of-plane current is the path average of the shape times q w vy / V.
   x0, x1 are positions in lambda0 (x1 unwrapped: it may leave the periodic box). */
void opic_deposit_current(opic *s, double qw, const double x0[3], const double x1[3], double vy)
{
    const int S = s->g.shape;
    const int dim3 = s->g.dim == 3;
    const double h[3] = {s->hx, s->hy, s->hz};
    double S0[3][5], DS[3][5];
    int64_t lo[3] = {0, 0, 0};
    for (int d = 0; d < 3; ++d) {
        if (d == 1 && !dim3)
            continue;
        const double a = x0[d] / h[d], b = x1[d] / h[d];
        lo[d] = (int64_t)floor(a < b ? a : b) - 1;
        for (int q = 0; q < 5; ++q) {
            const double node = (double)(lo[d] + q);
            S0[d][q] = opic_shape(S, a - node);
            DS[d][q] = opic_shape(S, b - node) - S0[d][q];
        }
    }
    const double vol = dim3 ? s->hx * s->hy * s->hz : s->hx * s->hz;
    const double cx = -qw * s->hx / (s->dt * vol);
    const double cy = -qw * s->hy / (s->dt * vol);
    const double cz = -qw * s->hz / (s->dt * vol);
    if (dim3) {
        for (int b = 0; b < 5; ++b)
            for (int c = 0; c < 5; ++c) {
                double acc = 0.0;
                for (int a = 0; a < 5; ++a) {
                    acc += DS[0][a] * (S0[1][b] * S0[2][c] + 0.5 * DS[1][b] * S0[2][c] +
                                       0.5 * S0[1][b] * DS[2][c] + DS[1][b] * DS[2][c] / 3.0);
                    add_j(s, OPIC_JX, lo[0] + a, lo[1] + b, lo[2] + c, cx * acc);
                }
            }
        for (int a = 0; a < 5; ++a)
            for (int c = 0; c < 5; ++c) {
                double acc = 0.0;
                for (int b = 0; b < 5; ++b) {
                    acc += DS[1][b] * (S0[2][c] * S0[0][a] + 0.5 * DS[2][c] * S0[0][a] +
                                       0.5 * S0[2][c] * DS[0][a] + DS[2][c] * DS[0][a] / 3.0);
                    add_j(s, OPIC_JY, lo[0] + a, lo[1] + b, lo[2] + c, cy * acc);
                }
            }
        for (int a = 0; a < 5; ++a)
            for (int b = 0; b < 5; ++b) {
                double acc = 0.0;
                for (int c = 0; c < 5; ++c) {
                    acc += DS[2][c] * (S0[0][a] * S0[1][b] + 0.5 * DS[0][a] * S0[1][b] +
                                       0.5 * S0[0][a] * DS[1][b] + DS[0][a] * DS[1][b] / 3.0);
                    add_j(s, OPIC_JZ, lo[0] + a, lo[1] + b, lo[2] + c, cz * acc);
                }
            }
    } else {
        for (int c = 0; c < 5; ++c) {
            double acc = 0.0;
            for (int a = 0; a < 5; ++a) {
                acc += DS[0][a] * (S0[2][c] + 0.5 * DS[2][c]);
                add_j(s, OPIC_JX, lo[0] + a, 0, lo[2] + c, cx * acc);
            }
        }
        for (int a = 0; a < 5; ++a) {
            double acc = 0.0;
            for (int c = 0; c < 5; ++c) {
                acc += DS[2][c] * (S0[0][a] + 0.5 * DS[0][a]);
                add_j(s, OPIC_JZ, lo[0] + a, 0, lo[2] + c, cz * acc);
            }
        }
        const double cyv = qw * vy / vol;
        for (int a = 0; a < 5; ++a)
            for (int c = 0; c < 5; ++c) {
                const double wgt = S0[0][a] * S0[2][c] + 0.5 * DS[0][a] * S0[2][c] +
                                   0.5 * S0[0][a] * DS[2][c] + DS[0][a] * DS[2][c] / 3.0;
                add_j(s, OPIC_JY, lo[0] + a, 0, lo[2] + c, cyv * wgt);
            }
    }
}

/* nodal charge density q w S S S / V of the particles from index `from` on of
   one species (diagnostic) */
static void deposit_rho_species(const opic *s, const species *p, int64_t from, double q, double *rho)
{
    const int S = s->g.shape;
    const int dim3 = s->g.dim == 3;
    const double vol = dim3 ? s->hx * s->hy * s->hz : s->hx * s->hz;
    const int zmax = zmax_of(s, 0.0);
    for (int64_t n = from; n < p->n; ++n) {
        const double xi = p->a[OPIC_PX][n] / s->hx, zi = p->a[OPIC_PZ][n] / s->hz;
        const double yi = dim3 ? p->a[OPIC_PY][n] / s->hy : 0.0;
        const double qw = q * p->a[OPIC_PW][n] / vol;
        const int64_t bx = (int64_t)floor(xi) - 1, by = (int64_t)floor(yi) - 1,
                      bz = (int64_t)floor(zi) - 1;
        for (int cz = 0; cz < 4; ++cz) {
            int64_t k = bz + cz;
            const double wz = opic_shape(S, zi - (double)k);
            if (wz == 0.0)
                continue;
            if (s->g.bc_z == 0)
                k = wrap_index(k, s->g.nz);
            else if (k < 0 || k > zmax)
                continue;
            for (int cy = 0; cy < (dim3 ? 4 : 1); ++cy) {
                int64_t j = 0;
                double wy = 1.0;
                if (dim3) {
                    j = by + cy;
                    wy = opic_shape(S, yi - (double)j);
                    if (wy == 0.0)
                        continue;
                    j = wrap_index(j, s->g.ny);
                }
                for (int cx = 0; cx < 4; ++cx) {
                    int64_t i = bx + cx;
                    const double wx = opic_shape(S, xi - (double)i);
                    if (wx == 0.0)
                        continue;
                    i = wrap_index(i, s->g.nx);
                    rho[fidx(s, i, j, k)] += qw * wx * wy * wz;
                }
            }
        }
    }
}

void opic_deposit_rho(const opic *s, double *rho)
{
    for (int64_t n = 0; n < s->nn; ++n)
        rho[n] = s->rho_bg[n];
    deposit_rho_species(s, &s->sp[0], 0, -1.0, rho);
    if (s->sp[1].n > 0)
        deposit_rho_species(s, &s->sp[1], 0, 1.0, rho);
}

/* --------------------------------------------------------------- push */

static void push_electrons(opic *s)
{
    species *p = &s->sp[0];
    const int dim3 = s->g.dim == 3;
    int64_t n = 0;
    while (n < p->n) {
        const double x0[3] = {p->a[OPIC_PX][n], p->a[OPIC_PY][n], p->a[OPIC_PZ][n]};
        double eb[6];
        for (int c = 0; c < 6; ++c)
            eb[c] = gather_comp(s, c, x0[0], x0[1], x0[2]);
        double u[3] = {p->a[OPIC_PUX][n], p->a[OPIC_PUY][n], p->a[OPIC_PUZ][n]};
        opic_boris(u, eb, eb + 3, -1.0, s->dt);
        const double g = sqrt(1.0 + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
        double x1[3];
        x1[0] = x0[0] + s->dt * u[0] / g;
        x1[1] = dim3 ? x0[1] + s->dt * u[1] / g : x0[1];
        x1[2] = x0[2] + s->dt * u[2] / g;
        opic_deposit_current(s, -p->a[OPIC_PW][n], x0, x1, u[1] / g);
        p->a[OPIC_PUX][n] = u[0];
        p->a[OPIC_PUY][n] = u[1];
        p->a[OPIC_PUZ][n] = u[2];
        /* boundaries: periodic x (y); z periodic or absorbing (particle removed) */
        if (x1[0] < 0.0)
            x1[0] += s->Lx;
        else if (x1[0] >= s->Lx)
            x1[0] -= s->Lx;
        if (dim3) {
            if (x1[1] < 0.0)
                x1[1] += s->Ly;
            else if (x1[1] >= s->Ly)
                x1[1] -= s->Ly;
        }
        if (s->g.bc_z == 0) {
            if (x1[2] < 0.0)
                x1[2] += s->Lz;
            else if (x1[2] >= s->Lz)
                x1[2] -= s->Lz;
        } else if (x1[2] < 0.0 || x1[2] >= s->Lz) {
            species_remove(p, n);
            continue;
        }
        p->a[OPIC_PX][n] = x1[0];
        p->a[OPIC_PY][n] = x1[1];
        p->a[OPIC_PZ][n] = x1[2];
        ++n;
    }
}

/* ions immobile in the lab: constant simulation-frame velocity u/gamma(u) */
static void move_ions(opic *s)
{
    species *p = &s->sp[1];
    const int dim3 = s->g.dim == 3;
    int64_t n = 0;
    while (n < p->n) {
        const double u[3] = {p->a[OPIC_PUX][n], p->a[OPIC_PUY][n], p->a[OPIC_PUZ][n]};
        const double g = sqrt(1.0 + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
        const double x0[3] = {p->a[OPIC_PX][n], p->a[OPIC_PY][n], p->a[OPIC_PZ][n]};
        double x1[3];
        x1[0] = x0[0] + s->dt * u[0] / g;
        x1[1] = dim3 ? x0[1] + s->dt * u[1] / g : x0[1];
        x1[2] = x0[2] + s->dt * u[2] / g;
        opic_deposit_current(s, p->a[OPIC_PW][n], x0, x1, u[1] / g);
        if (x1[0] < 0.0)
            x1[0] += s->Lx;
        else if (x1[0] >= s->Lx)
            x1[0] -= s->Lx;
        if (dim3) {
            if (x1[1] < 0.0)
                x1[1] += s->Ly;
            else if (x1[1] >= s->Ly)
                x1[1] -= s->Ly;
        }
        if (s->g.bc_z == 0) {
            if (x1[2] < 0.0)
                x1[2] += s->Lz;
            else if (x1[2] >= s->Lz)
                x1[2] -= s->Lz;
        } else if (x1[2] < 0.0 || x1[2] >= s->Lz) {
            species_remove(p, n);
            continue;
        }
        p->a[OPIC_PX][n] = x1[0];
        p->a[OPIC_PY][n] = x1[1];
        p->a[OPIC_PZ][n] = x1[2];
        ++n;
    }
}

/* ----------------------------------------------------------------- filter */

/* one (1/4, 1/2, 1/4) pass of component c along axis `ax`; periodic axes wrap,
   outside the valid z range of an absorbing-z grid the values are zero */
static void filter_pass(opic *s, int c, int ax, double *tmp)
{
    const int nx = s->g.nx, ny = s->ny, nz = s->g.nz;
    const int zmax = zmax_of(s, STAG[c][2]);
    memcpy(tmp, s->f[c], (size_t)s->nn * sizeof(double));
    for (int k = 0; k <= zmax; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                double lo, hi;
                if (ax == 0) {
                    lo = tmp[fidx(s, wrap_index(i - 1, nx), j, k)];
                    hi = tmp[fidx(s, wrap_index(i + 1, nx), j, k)];
                } else if (ax == 1) {
                    lo = tmp[fidx(s, i, wrap_index(j - 1, ny), k)];
                    hi = tmp[fidx(s, i, wrap_index(j + 1, ny), k)];
                } else if (s->g.bc_z == 0) {
                    lo = tmp[fidx(s, i, j, wrap_index(k - 1, nz))];
                    hi = tmp[fidx(s, i, j, wrap_index(k + 1, nz))];
                } else {
                    lo = k > 0 ? tmp[fidx(s, i, j, k - 1)] : 0.0;
                    hi = k < zmax ? tmp[fidx(s, i, j, k + 1)] : 0.0;
                }
                s->f[c][fidx(s, i, j, k)] = 0.25 * lo + 0.5 * tmp[fidx(s, i, j, k)] + 0.25 * hi;
            }
}

void opic_filter(opic *s)
{
    double *tmp = (double *)malloc((size_t)s->nn * sizeof(double));
    for (int c = OPIC_JX; c <= OPIC_JZ; ++c)
        for (int ax = 0; ax < 3; ++ax) {
            if (ax == 1 && s->g.dim != 3)
                continue;
            for (int p = 0; p < s->g.npass; ++p)
                filter_pass(s, c, ax, tmp);
        }
    free(tmp);
}

/* -------------------------------------------------------------------- Yee */

/* B -= h curl E on the Yee lattice (h = dt/2) */
static void yee_b(opic *s, double h)
{
    const int nx = s->g.nx, ny = s->ny, nz = s->g.nz, dim3 = s->g.dim == 3;
    const int per = s->g.bc_z == 0;
    double *Ex = s->f[OPIC_EX], *Ey = s->f[OPIC_EY], *Ez = s->f[OPIC_EZ];
    double *Bx = s->f[OPIC_BX], *By = s->f[OPIC_BY], *Bz = s->f[OPIC_BZ];
    for (int k = 0; k <= nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                const int ip = (i + 1) % nx, jp = (j + 1) % ny;
                const int64_t o = fidx(s, i, j, k);
                if (k < nz) {
                    const int kp = per ? (k + 1) % nz : k + 1;
                    /* Bx(i, j+1/2, k+1/2) */
                    double dEz_dy = dim3 ? (Ez[fidx(s, i, jp, k)] - Ez[o]) / s->hy : 0.0;
                    double dEy_dz = (Ey[fidx(s, i, j, kp)] - Ey[o]) / s->hz;
                    Bx[o] -= h * (dEz_dy - dEy_dz);
                    /* By(i+1/2, j, k+1/2) */
                    double dEx_dz = (Ex[fidx(s, i, j, kp)] - Ex[o]) / s->hz;
                    double dEz_dx = (Ez[fidx(s, ip, j, k)] - Ez[o]) / s->hx;
                    By[o] -= h * (dEx_dz - dEz_dx);
                }
                if (k < nz || !per) {
                    /* Bz(i+1/2, j+1/2, k) */
                    double dEy_dx = (Ey[fidx(s, ip, j, k)] - Ey[o]) / s->hx;
                    double dEx_dy = dim3 ? (Ex[fidx(s, i, jp, k)] - Ex[o]) / s->hy : 0.0;
                    Bz[o] -= h * (dEy_dx - dEx_dy);
                }
            }
}

/* E += dt (curl B - 2 pi J); with absorbing z the tangential E on the planes
   k = 0 and k = nz follows Mur's first-order condition instead */
static void yee_e(opic *s)
{
    const int nx = s->g.nx, ny = s->ny, nz = s->g.nz, dim3 = s->g.dim == 3;
    const int per = s->g.bc_z == 0;
    const double dt = s->dt;
    double *Ex = s->f[OPIC_EX], *Ey = s->f[OPIC_EY], *Ez = s->f[OPIC_EZ];
    double *Bx = s->f[OPIC_BX], *By = s->f[OPIC_BY], *Bz = s->f[OPIC_BZ];
    double *Jx = s->f[OPIC_JX], *Jy = s->f[OPIC_JY], *Jz = s->f[OPIC_JZ];
    double *old = NULL;
    const int64_t plane = (int64_t)nx * ny;
    if (!per) {
        /* E^n on planes 0, 1, nz-1, nz for the Mur update */
        old = (double *)malloc((size_t)(8 * plane) * sizeof(double));
        const int planes[4] = {0, 1, nz - 1, nz};
        for (int q = 0; q < 4; ++q) {
            memcpy(old + (2 * q) * plane, Ex + planes[q] * plane, (size_t)plane * sizeof(double));
            memcpy(old + (2 * q + 1) * plane, Ey + planes[q] * plane, (size_t)plane * sizeof(double));
        }
    }
    for (int k = 0; k <= nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                const int im = (i + nx - 1) % nx, jm = (j + ny - 1) % ny;
                const int64_t o = fidx(s, i, j, k);
                const int interior = per ? (k < nz) : (k >= 1 && k <= nz - 1);
                if (interior) {
                    const int km = per ? (k + nz - 1) % nz : k - 1;
                    /* Ex(i+1/2, j, k) */
                    double dBz_dy = dim3 ? (Bz[o] - Bz[fidx(s, i, jm, k)]) / s->hy : 0.0;
                    double dBy_dz = (By[o] - By[fidx(s, i, j, km)]) / s->hz;
                    Ex[o] += dt * ((dBz_dy - dBy_dz) - TWO_PI * Jx[o]);
                    /* Ey(i, j+1/2, k) */
                    double dBx_dz = (Bx[o] - Bx[fidx(s, i, j, km)]) / s->hz;
                    double dBz_dx = (Bz[o] - Bz[fidx(s, im, j, k)]) / s->hx;
                    Ey[o] += dt * ((dBx_dz - dBz_dx) - TWO_PI * Jy[o]);
                }
                if (k < nz) {
                    /* Ez(i, j, k+1/2) */
                    double dBy_dx = (By[o] - By[fidx(s, im, j, k)]) / s->hx;
                    double dBx_dy = dim3 ? (Bx[o] - Bx[fidx(s, i, jm, k)]) / s->hy : 0.0;
                    Ez[o] += dt * ((dBy_dx - dBx_dy) - TWO_PI * Jz[o]);
                }
            }
    if (!per) {
        const double cm = (dt - s->hz) / (dt + s->hz);
        for (int64_t q = 0; q < plane; ++q) {
            /* z = 0: wave leaving towards -z */
            const double ex0 = old[0 * plane + q], ey0 = old[1 * plane + q];
            const double ex1 = old[2 * plane + q], ey1 = old[3 * plane + q];
            Ex[q] = ex1 + cm * (Ex[plane + q] - ex0);
            Ey[q] = ey1 + cm * (Ey[plane + q] - ey0);
            /* z = Lz: wave leaving towards +z */
            const double exm = old[4 * plane + q], eym = old[5 * plane + q];
            const double exn = old[6 * plane + q], eyn = old[7 * plane + q];
            Ex[(int64_t)nz * plane + q] = exm + cm * (Ex[(int64_t)(nz - 1) * plane + q] - exn);
            Ey[(int64_t)nz * plane + q] = eym + cm * (Ey[(int64_t)(nz - 1) * plane + q] - eyn);
        }
        free(old);
    }
}

/* ------------------------------------------------------------ moving window */

int opic_set_window(opic *s, double v, double t0, int S)
{
    if (v == 0.0) {
        s->win_on = 0;
        return 0;
    }
    if (!(v > 0.0 && v <= 1.0) || !isfinite(t0) || S < 1 || S >= s->g.nz || s->g.bc_z != 1)
        return -1;
    s->win_on = 1;
    s->win_v = v;
    s->win_t0 = t0;
    s->win_S = S;
    return 0;
}

double opic_window(const opic *s) { return (double)s->win_n * s->win_S * s->hz; }

/* move the window by S cells: fields, particles, then the plasma it now covers */
static void window_move(opic *s)
{
    const int S = s->win_S;
    const int64_t plane = (int64_t)s->ny * s->g.nx;
    double *bufs[OPIC_NCOMP + 1];
    for (int c = 0; c < OPIC_NCOMP; ++c)
        bufs[c] = s->f[c];
    bufs[OPIC_NCOMP] = s->rho_bg;
    for (int c = 0; c <= OPIC_NCOMP; ++c) {
        double *f = bufs[c];
        for (int64_t k = 0; k <= s->g.nz; ++k)
            for (int64_t o = 0; o < plane; ++o)
                f[k * plane + o] = k + S <= s->g.nz ? f[(k + S) * plane + o] : 0.0;
    }
    const double dz = S * s->hz;
    for (int sp = 0; sp < 2; ++sp) {
        species *p = &s->sp[sp];
        int64_t k = 0;
        while (k < p->n) {
            p->a[OPIC_PZ][k] -= dz;
            if (p->a[OPIC_PZ][k] < 0.0)
                species_remove(p, k);
            else
                ++k;
        }
    }
    s->win_n += 1;
    const int64_t n0 = s->sp[0].n;
    inject_at(s, s->t);
    /* the plasma the window now covers brings its immobile ions along: their
       background is that of its electrons, as at load */
    if (s->bg_ions)
        deposit_rho_species(s, &s->sp[0], n0, 1.0, s->rho_bg);
}

/* --------------------------------------------- back-transformed snapshots */

int opic_btd_setup(opic *s, const opic_btd *b)
{
    free(s->btd_data);
    free(s->btd_fill);
    s->btd_data = NULL;
    s->btd_fill = NULL;
    s->btd_on = 0;
    if (!b)
        return 0;
    if (s->gam <= 1.0 || b->nsnap < 1 || b->nsnap > 64 || b->nz < 1 || !(b->dz > 0.0) ||
        (b->plane != 0 && b->plane != 1))
        return -1;
    s->btd = *b;
    s->btd_nxs = b->plane ? s->g.nx : 1;
    s->btd_data = (double *)calloc((size_t)b->nsnap * 6 * b->nz * s->btd_nxs, sizeof(double));
    s->btd_fill = (unsigned char *)calloc((size_t)b->nsnap * b->nz, 1);
    for (int c = 0; c < 6; ++c)
        if (!s->btd_prev[c])
            s->btd_prev[c] = (double *)calloc((size_t)s->nn, sizeof(double));
    s->btd_on = 1;
    return 0;
}

double *opic_btd_data(opic *s, int j)
{
    if (!s->btd_on || j < 0 || j >= s->btd.nsnap)
        return NULL;
    return s->btd_data + (size_t)j * 6 * s->btd.nz * s->btd_nxs;
}

unsigned char *opic_btd_filled(opic *s, int j)
{
    if (!s->btd_on || j < 0 || j >= s->btd.nsnap)
        return NULL;
    return s->btd_fill + (size_t)j * s->btd.nz;
}

/* component c of field array f at transverse node (i, j) and simulation-frame
   height zp, linear in z between the component's own planes; returns 0 where
   zp is not between two of them */
static int btd_zinterp(const opic *s, const double *f, int c, int64_t i, int64_t j, double zp, double *out)
{
    const double sz = STAG[c][2];
    const double u = zp / s->hz - sz;
    const double k0 = floor(u);
    const double fz = u - k0;
    if (k0 < 0.0 || k0 + 1.0 > (double)zmax_of(s, sz))
        return 0;
    const int64_t k = (int64_t)k0;
    *out = (1.0 - fz) * f[fidx(s, i, j, k)] + fz * f[fidx(s, i, j, k + 1)];
    return 1;
}

/* Fill every lab point whose event lies in the boosted step [t0, t0 + dt):
   the event (T, Z) of the lab frame is (t', z') = (gamma (T - beta Z),
   gamma (Z - beta T)) in the simulation frame, which moves at +beta along z.
   The simulation-frame fields at the event are linear in t' between the start
   and the end of the step and linear in z' between planes, and go to the lab
   frame by the inverse field transformation
     Ex = gamma (Ex' + beta By'),  Ey = gamma (Ey' - beta Bx'),  Ez = Ez',
     Bx = gamma (Bx' - beta Ey'),  By = gamma (By' + beta Ex'),  Bz = Bz'. */
static void btd_fill(opic *s, double t0)
{
    const opic_btd *b = &s->btd;
    const double gam = s->gam, beta = s->beta;
    const int64_t jc = s->ny / 2;
    const int nxs = s->btd_nxs;
    for (int js = 0; js < b->nsnap; ++js) {
        const double T = b->t0 + js * b->dt;
        for (int k = 0; k < b->nz; ++k) {
            const double Z = b->z0 + k * b->dz;
            const double tp = gam * (T - beta * Z);
            if (!(tp >= t0 && tp < t0 + s->dt))
                continue;
            const double zp = gam * (Z - beta * T) - opic_window(s);
            const double th = (tp - t0) / s->dt;
            int ok = 1;
            double v[6][2];
            for (int is = 0; is < nxs && ok; ++is) {
                const int64_t i = nxs == 1 ? s->g.nx / 2 : is;
                for (int c = 0; c < 6 && ok; ++c) {
                    double a0, a1;
                    ok = btd_zinterp(s, s->btd_prev[c], c, i, jc, zp, &a0) &&
                         btd_zinterp(s, s->f[c], c, i, jc, zp, &a1);
                    v[c][0] = a0;
                    v[c][1] = a1;
                }
                if (!ok)
                    break;
                double e[6];
                for (int c = 0; c < 6; ++c)
                    e[c] = (1.0 - th) * v[c][0] + th * v[c][1];
                double *d = s->btd_data + (size_t)js * 6 * b->nz * nxs;
                const double lab[6] = {gam * (e[0] + beta * e[4]), gam * (e[1] - beta * e[3]), e[2],
                                       gam * (e[3] - beta * e[1]), gam * (e[4] + beta * e[0]), e[5]};
                for (int c = 0; c < 6; ++c)
                    d[((size_t)c * b->nz + k) * nxs + is] = lab[c];
            }
            if (ok)
                s->btd_fill[(size_t)js * b->nz + k] = 1;
        }
    }
}

/* ------------------------------------------------------------ diagnostics */

/* Kahan-compensated running sum (Kahan 1965): the rounding error of every
   addition is carried into the next one */
typedef struct kahan {
    double s, c;
} kahan;

static void kahan_add(kahan *k, double v)
{
    const double y = v - k->c;
    const double t = k->s + y;
    k->c = (t - k->s) - y;
    k->s = t;
}

/* out[0] field energy (1/2) sum (E^2 + B^2) V over each component's valid
   nodes (E, B in m c omega0 / e: with n_c = eps0 m omega0^2 / e^2 the energy
   density eps0 E^2 / 2 is n_c m c^2 E^2 / 2, so this is in n_c m c^2 lambda0^3);
   out[1] electron kinetic energy sum w (gamma - 1), gamma - 1 formed as
   u^2 / (gamma + 1) (same units: w counts physical electrons per n_c lambda0^3);
   out[2] charge sum q w over the particle species (electrons q = -1, drifting
   ions q = +1; the lab frame's immobile ions are a background, not particles).
   Components in order, nodes and particles in storage order. */
void opic_diagnostics(const opic *s, double out[3])
{
    kahan fe = {0, 0};
    for (int c = 0; c < 6; ++c) {
        const int km = zmax_of(s, STAG[c][2]);
        for (int64_t k = 0; k <= km; ++k)
            for (int64_t j = 0; j < s->ny; ++j)
                for (int64_t i = 0; i < s->g.nx; ++i) {
                    const double v = s->f[c][fidx(s, i, j, k)];
                    kahan_add(&fe, v * v);
                }
    }
    const double vol = s->hx * s->hy * s->hz;
    out[0] = 0.5 * vol * fe.s;
    kahan ke = {0, 0}, q = {0, 0};
    const species *e = &s->sp[0];
    for (int64_t p = 0; p < e->n; ++p) {
        const double ux = e->a[OPIC_PUX][p], uy = e->a[OPIC_PUY][p], uz = e->a[OPIC_PUZ][p];
        const double u2 = ux * ux + uy * uy + uz * uz;
        kahan_add(&ke, e->a[OPIC_PW][p] * (u2 / (sqrt(1.0 + u2) + 1.0)));
        kahan_add(&q, -e->a[OPIC_PW][p]);
    }
    const species *ion = &s->sp[1];
    for (int64_t p = 0; p < ion->n; ++p)
        kahan_add(&q, ion->a[OPIC_PW][p]);
    out[1] = ke.s;
    out[2] = q.s;
}

/* Lab-frame E and B on the simulation grid at the current simulation time
   (the inverse of the boost along z, the hyperbolic rotation of section
   "Effect of the hyperbolic rotation in Minkowski space"):
     Ex = gamma (Ex' + beta By'), Ey = gamma (Ey' - beta Bx'), Ez = Ez',
     Bx = gamma (Bx' - beta Ey'), By = gamma (By' + beta Ex'), Bz = Bz'.
   Every component stays at its own Yee position; the partner it mixes with
   sits half a cell away in z and is taken there as the mean of its two
   neighbouring planes (the nearer plane alone at an absorbing z end; planes
   wrap when z is periodic).  out: 6 arrays of nn values, Ex Ey Ez Bx By Bz. */
static double zmean(const opic *s, const double *f, int c, int64_t i, int64_t j, int64_t k, int up)
{
    /* the partner c at the component's height: planes k-1, k (up = 0) or
       k, k+1 (up = 1) of the partner's own index */
    const int km = zmax_of(s, STAG[c][2]);
    int64_t a = up ? k : k - 1, b = up ? k + 1 : k;
    if (s->g.bc_z == 0) {
        a = wrap_index(a, s->g.nz);
        b = wrap_index(b, s->g.nz);
    } else {
        if (a < 0)
            a = b;
        if (b > km)
            b = a;
        if (a > km)
            a = b = km;
    }
    return 0.5 * (f[fidx(s, i, j, a)] + f[fidx(s, i, j, b)]);
}

void opic_fields_lab(const opic *s, double *out)
{
    const double gam = s->gam, beta = s->beta;
    for (int c = 0; c < 6; ++c) {
        double *d = out + (size_t)c * s->nn;
        const int km = zmax_of(s, STAG[c][2]);
        for (int64_t k = 0; k <= s->g.nz; ++k)
            for (int64_t j = 0; j < s->ny; ++j)
                for (int64_t i = 0; i < s->g.nx; ++i) {
                    const int64_t o = fidx(s, i, j, k);
                    double v = 0.0;
                    if (k <= km) {
                        /* integer-z E components meet half-integer-z B partners
                           (planes k-1, k) and the other way round (k, k+1) */
                        switch (c) {
                        case OPIC_EX: v = gam * (s->f[OPIC_EX][o] + beta * zmean(s, s->f[OPIC_BY], OPIC_BY, i, j, k, 0)); break;
                        case OPIC_EY: v = gam * (s->f[OPIC_EY][o] - beta * zmean(s, s->f[OPIC_BX], OPIC_BX, i, j, k, 0)); break;
                        case OPIC_EZ: v = s->f[OPIC_EZ][o]; break;
                        case OPIC_BX: v = gam * (s->f[OPIC_BX][o] - beta * zmean(s, s->f[OPIC_EY], OPIC_EY, i, j, k, 1)); break;
                        case OPIC_BY: v = gam * (s->f[OPIC_BY][o] + beta * zmean(s, s->f[OPIC_EX], OPIC_EX, i, j, k, 1)); break;
                        default: v = s->f[OPIC_BZ][o]; break;
                        }
                    }
                    d[o] = v;
                }
    }
}

/* ------------------------------------------------------------------- step */

void opic_step_phases(opic *s, unsigned mask)
{
    if (mask & OPIC_PH_ZERO_J)
        for (int c = OPIC_JX; c <= OPIC_JZ; ++c)
            memset(s->f[c], 0, (size_t)s->nn * sizeof(double));
    if (mask & OPIC_PH_PUSH)
        push_electrons(s);
    if ((mask & OPIC_PH_IONS) && s->sp[1].n > 0)
        move_ions(s);
    if ((mask & OPIC_PH_ANTENNA) && s->laser_on)
        antenna(s);
    if ((mask & OPIC_PH_FILTER) && s->g.npass > 0)
        opic_filter(s);
    if (mask & OPIC_PH_YEE) {
        if (s->btd_on)
            for (int c = 0; c < 6; ++c)
                memcpy(s->btd_prev[c], s->f[c], (size_t)s->nn * sizeof(double));
        yee_b(s, 0.5 * s->dt);
        yee_e(s);
        yee_b(s, 0.5 * s->dt);
        if (s->btd_on)
            btd_fill(s, s->t);
    }
    if ((mask & OPIC_PH_INJECT) && s->npend > 0)
        inject(s);
    if (mask & OPIC_PH_TIME) {
        s->t += s->dt;
        s->step += 1;
        if (s->win_on && s->t >= s->win_t0 &&
            s->win_v * (s->t - s->win_t0) >= (double)(s->win_n + 1) * s->win_S * s->hz)
            window_move(s);
    }
}

void opic_step(opic *s, int nsteps)
{
    for (int n = 0; n < nsteps; ++n)
        opic_step_phases(s, OPIC_PH_ALL);
}
