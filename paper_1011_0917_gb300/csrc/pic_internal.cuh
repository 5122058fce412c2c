// pic_internal.cuh -- device-side data layout and helpers of the PIC library.
//
// Layout in HBM (all caller-owned):
//   fields:  9 components (Ex Ey Ez Bx By Bz Jx Jy Jz), each (nz+1) x ny x nx
//            elements in [k][j][i] order.  Yee staggering of component c at
//            array index (i, j, k): Ex (i+1/2, j, k), Ey (i, j+1/2, k),
//            Ez (i, j, k+1/2), Bx (i, j+1/2, k+1/2), By (i+1/2, j, k+1/2),
//            Bz (i+1/2, j+1/2, k); J like E.
//   species: per species two "sides" (double buffer).  A side is a structure
//            of arrays with `slots` entries per attribute; tile t owns slots
//            [t*cap, (t+1)*cap) and keeps its particles in two runs: a bottom
//            run [0, lo) that the tile's own CTA writes (particles that stayed
//            in the tile, counted in shared memory) and a top run
//            [cap - hi, cap) that others append to with global atomics
//            (particles that arrived from a neighbour, were loaded or were
//            injected).  A particle is an int32 packed cell index plus its
//            offsets in [0,1) inside that cell (real), its weight and
//            (electrons) u = gamma v; with drift-relative z (below) an
//            electron also carries its departure from the drift.
//   scratch: per-side tile counters, the filter ping-pong buffer, per-tile
//            offsets for compaction, reduction partials and the error word.
#pragma once

#include <cstdint>
#include <cstring>
#include <cuda_runtime.h>
#include <type_traits>
#include <vector>

namespace pic {

enum : unsigned { ERR_CAPACITY = 1u, ERR_CFL = 2u, ERR_NAN = 4u, ERR_TILE = 8u, ERR_TIMEOUT = 16u };

// Bit 31 of an electron's cell word: the electron is paired with a drifting ion
// at its own position that has moved exactly like it since both were placed
// (the plasma no field has touched).  Such a pair carries no current and is
// stored as the electron record alone; its ion gets a record of its own (at the
// electron's position) the first time the electron gathers a non-zero field.
constexpr uint32_t kPaired = 0x80000000u;

struct Geom {
    int dim;            // 2 or 3
    int nx, ny, nz;     // cells (ny = 1 in 2D)
    int bc_z;           // 0 periodic, 1 Mur
    int shape;          // 1 or 2
    int bx, by;         // bits of i and j in a packed cell index
    int lt[3];          // log2 of the tile shape
    int nt[3];          // tiles per axis
    int cap;            // slots per tile
    int64_t plane;      // nx * ny
    int64_t ncomp;      // (nz + 1) * plane, elements per field component
    int64_t ntiles;
};

// attribute arrays of a species side, in this order: ox oy oz w ux uy uz cell
// id dlx dly dlz (absent ones are null)
constexpr int kAttrs = 12;

template <typename real>
struct Species {
    real *ox, *oy, *oz, *w;     // oy is null in 2D
    real *ux, *uy, *uz;         // null for ions (constant drift)
    int32_t *cell;
    int64_t *id;                // null unless ids are tracked
    real *dlx, *dly, *dlz;      // relative positions only (see rel_actual); dly null in 2D
};

// Relative positions of an electron record.  In a strongly boosted frame the
// plasma (electrons and ions, gamma n each) streams through a good part of a
// cell every step, while the wake is made of the difference between the two
// species' currents: ~1/(2 gamma^2) of the plasma's response in the lab, so
// at gamma = 130 about 3e-8 of either species' current.  Each particle's
// current must then be formed from a position exact far beyond FP32, and in
// FP64 arithmetic, or the difference is rounding noise.  A record in relative
// form holds, per axis, a reference offset o in [0, 1) -- along z it moves
// with exactly the arithmetic of a drifting ion, across it stays where the
// particle was placed, i.e. it is its ion's path -- plus the departure dl
// from it, |dl| <= 1/2 (whole cells move between dl and the reference cell,
// which is exact).  The position is c_ref + o + dl with c_ref = c + r, c the
// stored cell (the one the electron is in, so that tiles and stencils are as
// for any record) and r the shift this function returns; its result is the
// electron's offset in cell c, in [0, 1), for the gather.  The rounding of
// o + dl here does not accumulate: it is redone from the exact pair every
// step, and the current is deposited from the pair itself (in FP64).
template <typename real>
__host__ __device__ inline real rel_actual(real o, real dl, int &r)
{
    const real a = o + dl;
    if (a < real(0)) {
        const real t = a + real(1);
        if (t < real(1)) {
            r = 1;
            return t;
        }
        r = 0;  // within rounding of the cell's lower face
        return real(0);
    }
    if (a >= real(1)) {
        r = -1;
        return a - real(1);
    }
    r = 0;
    return a;
}

__host__ __device__ inline int32_t pack_cell(const Geom &g, int i, int j, int k)
{
    return (int32_t)((uint32_t)i | ((uint32_t)j << g.bx) | ((uint32_t)k << (g.bx + g.by)));
}

__host__ __device__ inline void unpack_cell(const Geom &g, int32_t c, int &i, int &j, int &k)
{
    uint32_t u = (uint32_t)c & ~kPaired;
    i = (int)(u & ((1u << g.bx) - 1u));
    j = g.by ? (int)((u >> g.bx) & ((1u << g.by) - 1u)) : 0;
    k = (int)(u >> (g.bx + g.by));
}

__host__ __device__ inline int64_t tile_of(const Geom &g, int i, int j, int k)
{
    return ((int64_t)(k >> g.lt[2]) * g.nt[1] + (j >> g.lt[1])) * g.nt[0] + (i >> g.lt[0]);
}

__host__ __device__ inline int64_t fidx(const Geom &g, int i, int j, int k)
{
    return ((int64_t)k * g.ny + j) * g.nx + i;
}

// z index range of a component: half-integer-z components (Ez, Bx, By, Jz)
// live on k = 0..nz-1, the others on 0..nz; periodic z wraps over nz.
__host__ __device__ inline int zmax_of(const Geom &g, bool half_z)
{
    if (g.bc_z == 0) return g.nz - 1;
    return half_z ? g.nz - 1 : g.nz;
}

__host__ __device__ inline int wrapi(int i, int n)
{
    i %= n;
    return i < 0 ? i + n : i;
}

// ------------------------------------------------------------- buckets

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

// Reserve one slot per lane in the bucket of `dest` (dest < 0: no slot),
// one atomic per distinct destination in the warp.  All 32 lanes must call.
__device__ __forceinline__ int reserve_slot(int *cnt, int64_t dest)
{
    const unsigned lane = lane_id();
    const unsigned peers = __match_any_sync(0xffffffffu, (unsigned long long)dest);
    const int leader = __ffs(peers) - 1;
    const int rank = __popc(peers & ((1u << lane) - 1u));
    int base = 0;
    if (dest >= 0 && (int)lane == leader) base = atomicAdd(&cnt[dest], __popc(peers));
    base = __shfl_sync(peers, base, leader);
    return base + rank;
}

// slot of the p-th live particle of tile t (bottom run first, then top run)
__device__ __forceinline__ int64_t bucket_slot(int64_t t, int cap, int n_lo, int n_hi, int p)
{
    return t * (int64_t)cap + (p < n_lo ? p : cap - n_hi + (p - n_lo));
}

// run lengths of tile t; runs that overlap mean the bucket overflowed: that is
// reported and the runs are clamped so that no slot is read twice
__device__ __forceinline__ void bucket_counts(const int *lo, const int *hi, int64_t t, int cap, int &n_lo,
                                              int &n_hi, unsigned *err)
{
    n_lo = lo[t];
    n_hi = hi[t];
    if (n_lo > cap) n_lo = cap;
    if (n_hi > cap - n_lo) {
        if (err) atomicOr(err, ERR_CAPACITY);
        n_hi = cap - n_lo;
    }
}

// ---------------------------------------------------------------- shapes

// 1D B-spline weights of order S at a position p measured from node 0 of a
// window; returns the first node of the support and fills S+1 weights.
template <int S, typename real>
__device__ __forceinline__ int spline_weights(real p, real w[S + 1])
{
    if (S == 1) {
        real f = floor(p);
        real d = p - f;
        w[0] = real(1) - d;
        w[1] = d;
        return (int)f;
    } else {
        real c = floor(p + real(0.5));
        real d = p - c;
        real a = real(0.5) - d, b = real(0.5) + d;
        w[0] = real(0.5) * a * a;
        w[1] = real(0.75) - d * d;
        w[2] = real(0.5) * b * b;
        return (int)c - 1;
    }
}

// The same at an in-cell offset o in [0, 1) (the particle's own cell, an
// invariant of the store): for CIC the support starts at the cell's node, so
// the floor is 0 and the weights are those of spline_weights<1>(o) bit for bit.
template <int S, typename real>
__device__ __forceinline__ int offset_weights(real o, real w[S + 1])
{
    if (S == 1) {
        w[0] = real(1) - o;
        w[1] = o;
        return 0;
    }
    return spline_weights<S>(o, w);
}

// And at o - 1/2 (components staggered by half a cell), o in [0, 1): for CIC
// the floor is -1 or 0; the weights are those of spline_weights<1>(o - 1/2)
// bit for bit.
template <int S, typename real>
__device__ __forceinline__ int half_weights(real o, real w[S + 1])
{
    if (S == 1) {
        const real p = o - real(0.5);
        const bool lo = p < real(0);
        const real d = lo ? p + real(1) : p;
        w[0] = real(1) - d;
        w[1] = d;
        return lo ? -1 : 0;
    }
    return spline_weights<S>(o - real(0.5), w);
}

// Esirkepov window along one axis: old offset x0 in [0,1), new position x1 =
// x0 + d (|d| < 1), both relative to the old cell.  Returns the first node of
// a window of S+2 nodes that holds both supports, with S0 and DS = S1 - S0 on
// it, and whether the support moved to another first node.
template <int S, typename real>
__device__ __forceinline__ int esirk_axis_c(real x0, real x1, real S0[S + 2], real DS[S + 2], bool &crossed)
{
    real w0[S + 1], w1[S + 1];
    const int b0 = offset_weights<S>(x0, w0);  // x0: the in-cell offset at the start
    const int b1 = spline_weights<S>(x1, w1);
    const int anchor = b0 < b1 ? b0 : b1;
    const bool s0 = b0 != anchor, s1 = b1 != anchor;
    crossed = b0 != b1;
#pragma unroll
    for (int q = 0; q < S + 2; ++q) {
        const real v0 = s0 ? (q >= 1 ? w0[q - 1 < S ? q - 1 : S] : real(0)) : (q <= S ? w0[q <= S ? q : S] : real(0));
        const real v1 = s1 ? (q >= 1 ? w1[q - 1 < S ? q - 1 : S] : real(0)) : (q <= S ? w1[q <= S ? q : S] : real(0));
        S0[q] = v0;
        DS[q] = v1 - v0;
    }
    return anchor;
}

// The same for a start position x0 that need not lie in [0, 1) (within a
// cell of it): both supports from the spline itself.
template <int S, typename real>
__device__ __forceinline__ int esirk_axis_g(real x0, real x1, real S0[S + 2], real DS[S + 2], bool &crossed)
{
    real w0[S + 1], w1[S + 1];
    const int b0 = spline_weights<S>(x0, w0);
    const int b1 = spline_weights<S>(x1, w1);
    const int anchor = b0 < b1 ? b0 : b1;
    const bool s0 = b0 != anchor, s1 = b1 != anchor;
    crossed = b0 != b1;
#pragma unroll
    for (int q = 0; q < S + 2; ++q) {
        const real v0 = s0 ? (q >= 1 ? w0[q - 1 < S ? q - 1 : S] : real(0)) : (q <= S ? w0[q <= S ? q : S] : real(0));
        const real v1 = s1 ? (q >= 1 ? w1[q - 1 < S ? q - 1 : S] : real(0)) : (q <= S ? w1[q <= S ? q : S] : real(0));
        S0[q] = v0;
        DS[q] = v1 - v0;
    }
    return anchor;
}

// periodic index for i in [-n, 2n)
__device__ __forceinline__ int wrap1(int i, int n)
{
    return i < 0 ? i + n : (i >= n ? i - n : i);
}

// ----------------------------------------------------------------- Boris

// reciprocals used by the push: IEEE in FP64 (the debug path).  In FP32 the
// hardware reciprocal square root refined by one Newton-Raphson step for
// f(y) = 1/y^2 - x, y <- y (3 - x y^2) / 2, which squares its relative error
// (to below the FP32 rounding), so that the systematic error of v = u/gamma
// does not accumulate over many steps of a drifting plasma; and the correctly
// rounded reciprocal intrinsic.
__device__ __forceinline__ double rsqrt_p(double x) { return 1.0 / sqrt(x); }
__device__ __forceinline__ float rsqrt_p(float x)
{
    const float y = rsqrtf(x);
    return y * fmaf(-0.5f * x * y, y, 1.5f);
}
__device__ __forceinline__ double div_p(double a, double b) { return a / b; }
__device__ __forceinline__ float div_p(float a, float b) { return a * __frcp_rn(b); }

// Momenta are stored relative to the plasma drift u_d = (0, 0, U) (U = 0 in
// the lab frame, -gamma beta in the boosted frame): a record holds
// du = u - u_d.  In FP32 a momentum near -gamma beta resolves changes of one
// ulp of gamma beta, and v = u / gamma of it only ~6e-8, while a change du
// moves v_z by du / gamma^3; relative storage and the velocity formula below
// keep the plasma response at the relative precision of du itself.

// relativistic Boris rotation for du/dt = 2 pi (q/m)(E + u x B / gamma) on
// the stored du; eps = pi (q/m) dt is half the impulse factor.  The rotation
// acts on the full u^- = u_d + du^-; its increments are added to du, so zero
// fields leave du unchanged bit for bit.
template <typename real>
__device__ __forceinline__ void boris(real &dux, real &duy, real &duz, real U, real ex, real ey, real ez,
                                      real bx, real by, real bz, real eps)
{
    const real dmx = dux + eps * ex, dmy = duy + eps * ey, dmz = duz + eps * ez;
    const real umx = dmx, umy = dmy, umz = U + dmz;
    real f = eps * rsqrt_p(real(1) + umx * umx + umy * umy + umz * umz);
    real tx = f * bx, ty = f * by, tz = f * bz;
    real t2 = tx * tx + ty * ty + tz * tz;
    real s = div_p(real(2), real(1) + t2);
    real sx = s * tx, sy = s * ty, sz = s * tz;
    real upx = umx + (umy * tz - umz * ty);
    real upy = umy + (umz * tx - umx * tz);
    real upz = umz + (umx * ty - umy * tx);
    dux = dmx + (upy * sz - upz * sy) + eps * ex;
    duy = dmy + (upz * sx - upx * sz) + eps * ey;
    duz = dmz + (upx * sy - upy * sx) + eps * ez;
}

// correctly rounded add and multiply that the compiler may not contract into
// a fused multiply-add (the drift's displacement must round the same way in
// every kernel that applies it)
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }

// gamma_d^2 = 1 + U^2, 1 / gamma_d and the displacement per step dz (in
// cells, dtdh = dt / h_z) of the drift; the drifting ions and the electrons
// take all from here, and move by add_rn(offset, dz), so that a field-free
// electron and its ion move bit-identically
template <typename real>
struct Drift {
    real U, g2, ig, g, dz;
    __device__ __forceinline__ Drift(real u, real dtdh) : U(u)
    {
        g2 = add_rn(real(1), mul_rn(U, U));
        ig = rsqrt_p(g2);
        g = mul_rn(g2, ig);
        dz = mul_rn(mul_rn(U, ig), dtdh);
    }
};

// Velocity of a record with momentum u_d + du: returns v_z - v_d and sets
// vx, vy.  With gamma^2 = gamma_d^2 + D, D = du_z (2U + du_z) + p2,
// p2 = du_x^2 + du_y^2, and s = gamma + gamma_d,
//   v_z - v_d = [du_z (2 + E) - U p2] / (gamma gamma_d s),
//   E = gamma_d (gamma - gamma_d) - U du_z = (gamma_d (du_z^2 + p2) - U du_z D / s) / s,
// an exact rearrangement in which no term cancels the drift (E is of second
// order in du).  du = 0 gives exactly 0.  In the lab frame (U = 0) it is the
// plain du_z / gamma.
template <typename real>
__device__ __forceinline__ real drift_velocity(const Drift<real> &d, real dux, real duy, real duz, real &vx,
                                               real &vy)
{
    const real p2 = dux * dux + duy * duy;
    const real D = duz * (real(2) * d.U + duz) + p2;
    const real ig = rsqrt_p(d.g2 + D);
    vx = dux * ig;
    vy = duy * ig;
    if (d.U == real(0)) return duz * ig;
    const real is = div_p(real(1), (d.g2 + D) * ig + d.g);
    const real E = (d.g * (duz * duz + p2) - d.U * duz * D * is) * is;
    return (duz * (real(2) + E) - d.U * p2) * (ig * d.ig * is);
}

// largest value below one, for offsets that round up to 1
template <typename real> __host__ __device__ inline real below_one();
template <> __host__ __device__ inline float below_one<float>() { return 0.99999994f; }
template <> __host__ __device__ inline double below_one<double>() { return 0.99999999999999989; }

// ---------------------------------------------------- kernel argument packs

template <typename real>
struct IonSide {         // the drifting-ion species of a step
    Species<real> in, out;
    int *in_lo, *in_hi, *out_lo, *out_hi;
    real jfac_z;         // -q h_z / (dt V) of the ions
};

template <typename real>
struct PushArgs {
    Geom g;
    const real *E[3];
    const real *B[3];
    real *J[3];
    Species<real> in, out;
    int *in_lo, *in_hi, *out_lo, *out_hi;   // run lengths per tile (see the layout note)
    real dtdh[3];       // dt / h_d
    real eps;           // pi (q/m) dt
    real jfac[3];       // -q h_d / (dt V): multiplied by w and the running sum
    real jyfac;         // q / V (2D out-of-plane current, times w vy)
    real u_drift;       // U: the plasma's drift momentum (0, 0, U); electron
                        // records store u - (0, 0, U), ions move with it
    // fixed-point current accumulation (FP32; FP64 uses 1): the per-particle
    // factors of Jx, Jy (2D: the out-of-plane factor), Jz are multiplied by
    // fx_scale[c]; a shared-tile node's integer sum times fx_quant[c] =
    // 1 / fx_scale[c] is its current; fx_lo = {2^K, 2^-K} scales the "lo" words
    real fx_scale[3], fx_quant[3], fx_lo[2];
    Species<real> ion_in;  // ion side the IONS phase reads next (released ions go there)
    int *ion_in_hi;        // its top-run lengths
    int fuse_ions;         // 1: the same CTA then moves and deposits the tile's ions
    IonSide<real> ions;    // (with fuse_ions) the ion sides and counters
    int rel;               // 1: electron records in relative form (rel_actual), currents
                           //    of electrons and ions from FP64 arithmetic
    unsigned *err;
};

template <typename real>
struct BucketArgs {      // re-bucket a flat list into tiles
    Geom g;
    Species<real> src, dst;
    int64_t n;
    int *dst_hi;         // top-run lengths of the destination side
    unsigned *err;
};

template <typename real>
struct CompactArgs {     // copy tiles into a flat list
    Geom g;
    Species<real> src, dst;
    const int *lo, *hi;
    const int64_t *offset;
};

template <typename real>
struct SortArgs {        // order every tile's bucket by cell (into the other side)
    Geom g;
    Species<real> in, out;
    int *in_lo, *in_hi, *out_lo;
    unsigned *err;
};

template <typename real>
struct BtdArgs {         // lab-frame snapshots filled during one step
    Geom g;
    const real *E0[3], *B0[3];  // fields at the start of the step
    const real *E1[3], *B1[3];  // and at its end
    real *data;                 // [nsnap][6][nz][nxs]
    int *flags;                 // [nsnap][nz]
    double gam, beta, hz;
    double zwin;                // window displacement (simulation-frame positions are relative to it)
    double t0, dt;              // the step's simulation-frame interval [t0, t0 + dt)
    double T0, dT, Z0, dZ;      // lab times and positions of the snapshots
    int nsnap, nz, nxs;
    int klo[64], kn[64];        // per snapshot, the lab points this step may fill
};

// per-step scalars of a captured step (CUDA graph): the antenna amplitude and
// the injection's times and lattice band, read by the kernels from device
// memory that the host refills before each replay
struct StepScal {
    double j0, t, t1;
    int64_t m_lo, m_hi;
};

struct InjectArgs {      // lattice load / boosted injection, FP64
    Geom g;
    double hx, hy, hz, Lx, Ly, Lz, gam, beta;
    int ppx, ppy, ppz;
    int64_t NX, NY, m_lo, m_hi;
    double z_start, z_end, ramp, ne, jitter, dzl, hz_lab, wfac;
    int nprof;
    double prof[16];
    uint64_t seed;
    int mode;           // 0: in [zmin, Lz) at t; 1: crossing z = Lz during (t, t1]
    double t, t1;
    double zwin;        // window displacement (positions are relative to it)
    double zmin;        // lower end of a mode-0 load (0, or the layer a window move uncovers)
    int drift_ions;     // ions drift with the plasma
    int paired;         // electrons are placed paired with their ion (no ion record)
    int precision;      // 0 float, 1 double
    void *sp_e[kAttrs];  // ox oy oz w ux uy uz cell id dlx dly dlz of the electron side
    void *sp_i[kAttrs];  // same for the ion side (ux..uz, dl* unused)
    int *hi_e, *hi_i;    // top-run lengths of the electron / ion sides
    unsigned *err;
    // fixed-order ("flat") output of an adjoint run (flat_base >= 0, 2D):
    // lattice point q of the band goes to slot flat_base + q, alive or not
    int64_t flat_base;
    int *fe_ci, *fe_cj, *fe_ck;  // electron state (cj, oy in 3D)
    void *fe_ox, *fe_oy, *fe_oz, *fe_ux, *fe_uy, *fe_uz;
    unsigned char *fe_alive;
    int *fi_ck;                  // ion state
    void *fi_oz;
    unsigned char *fi_alive;
    int *f_ion_ci, *f_ion_cj;    // per slot, constant: the ion's transverse cells
    void *f_ion_ox, *f_ion_oy;   // and offsets,
    void *f_w;                   // the weight (shared by the pair)
    double *f_zeta;              // and the lab profile coordinate
    const StepScal *scal;        // non-null: t, t1, m_lo, m_hi from here (a captured
                                 // step; m_lo, m_hi above then bound the launch)
};

// One state of the flat particle store of an adjoint run (slot p is the same
// particle at every step; cj, oy only in 3D)
template <typename real>
struct FlatE {
    int *ci, *cj, *ck;
    real *ox, *oy, *oz, *ux, *uy, *uz;  // offsets; momenta relative to the drift
    unsigned char *alive;
};
template <typename real>
struct FlatI {
    int *ck;
    real *oz;
    unsigned char *alive;
};

template <typename real>
struct AdjArgs {
    Geom g;
    const real *E[3], *B[3];        // E^n, B^n
    real *J[3];                     // forward: current; reverse: its cotangent
    FlatE<real> in, out;            // electron states n and n+1
    FlatI<real> iin, iout;          // ion states n and n+1
    const real *w;                  // weights per slot
    const int *ion_ci, *ion_cj;     // ion transverse cells / offsets per slot
    const real *ion_ox, *ion_oy;
    int64_t n;                      // slots
    real dtdh[3];                   // dt / h_d
    real eps, u_drift;
    real jfac[3], jyfac, jfac_iz;   // electrons' -q h_d / (dt V), 2D q / V; ions' Jz factor
    real *lE[3], *lB[3];            // reverse: field cotangents at n
    real *lx, *ly, *lz, *lux, *luy, *luz;  // reverse: particle cotangents
    double *lw;                     // reverse: weight cotangents per slot
    const unsigned char *lj_plane;  // reverse: 1 for the cells ck within reach of a plane where lJ is not zero
    const unsigned char *f_plane;   // 1 for the cells ck within reach of a plane where E or B is not zero
    int with_ions;                  // the drifting ion of every slot too
};

// ------------------------------------------------- batched launch recording
//
// A batch of independent runs can step together with one launch per phase
// over the work items of all of them.  Such a step is built by running each
// run's own step on the host with a recorder installed on the calling
// thread: every launch function then appends what it would launch -- its
// phase, the batched form of its kernel, its argument struct and its number
// of work items (blocks, or tiles for the persistent particle kernels) --
// instead of launching.  A batched kernel maps its block (or the next item
// of a device-wide queue) to (run, item) through the runs' prefix sums of
// work items, copies that run's argument struct into shared memory and runs
// the same per-block body as the single-run kernel, so both give identical
// results.
//
// BatchLaunch(args, start, n, total, queue, stream): args = n argument
// structs (device), start = n + 1 prefix sums of the runs' work items
// (device), total = start[n], queue = a zeroed device counter (persistent
// kernels) or null.
using BatchLaunch = void (*)(const void *args, const int64_t *start, int n, int64_t total, unsigned *queue,
                             cudaStream_t s);
// phases in the order a step issues them
enum BatchPhase : int { kBPZero = 0, kBPPush, kBPIons, kBPAntenna, kBPFilter, kBPYee, kBPInject, kBPCount };
struct LaunchRecord {
    int chain, step, phase;
    BatchLaunch fn;
    std::vector<unsigned char> args;
    int64_t items;
    bool queue;  // the batched kernel pulls its items from a device counter
};
struct BatchRecorder {
    int chain = 0;             // the launch chain (stream) the current run belongs to
    int step = 0;
    int nctx = 1;              // runs in the batch (field kernels size their z chunks for all of them)
    bool unsupported = false;  // the step asked for something the batched step does not do
    std::vector<LaunchRecord> recs;
};
extern thread_local BatchRecorder *g_rec;

// true (and recorded) while a recorder is installed
template <typename A>
inline bool record_launch(int phase, BatchLaunch fn, const A &a, int64_t items, bool queue = false)
{
    static_assert(std::is_trivially_copyable<A>::value, "argument structs are copied as bytes");
    BatchRecorder *r = g_rec;
    if (!r) return false;
    LaunchRecord L;
    L.chain = r->chain;
    L.step = r->step;
    L.phase = phase;
    L.fn = fn;
    L.args.resize(sizeof(A));
    std::memcpy(L.args.data(), &a, sizeof(A));
    L.items = items;
    L.queue = queue;
    r->recs.push_back(std::move(L));
    return true;
}
// for launches with no batched form: true (the step is then not batched)
// while a recorder is installed
inline bool record_unsupported()
{
    if (!g_rec) return false;
    g_rec->unsupported = true;
    return true;
}
// runs whose field kernels share one launch (z chunks are sized for all)
inline int batch_runs() { return g_rec ? g_rec->nctx : 1; }

#ifdef __CUDACC__
// the run owning work item `item`: the last r with start[r] <= item
__device__ __forceinline__ int batch_run_of(const int64_t *start, int n, int64_t item)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (start[mid] <= item) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// all threads of the CTA copy an argument struct (global -> shared)
template <typename A>
__device__ __forceinline__ void batch_copy_args(A *dst, const A *src)
{
    static_assert(sizeof(A) % 4 == 0, "argument structs are copied as words");
    const int *s = reinterpret_cast<const int *>(src);
    int *d = reinterpret_cast<int *>(dst);
    for (int i = (int)threadIdx.x; i < (int)(sizeof(A) / 4); i += (int)blockDim.x) d[i] = s[i];
}

// block blockIdx.x of a batched launch with one block per work item: its
// run's arguments into *sa (shared), returns the block's index in its run
template <typename A>
__device__ __forceinline__ int64_t batch_block(const A *runs, const int64_t *start, int n, A *sa)
{
    __shared__ int s_r;
    if (threadIdx.x == 0) s_r = batch_run_of(start, n, (int64_t)blockIdx.x);
    __syncthreads();
    const int r = s_r;
    batch_copy_args(sa, runs + r);
    __syncthreads();
    return (int64_t)blockIdx.x - start[r];
}
#endif

// the zeroing of a current buffer as a batchable launch (cudaMemsetAsync
// otherwise)
template <typename real>
struct ZeroArgs {
    real *p;
    int64_t n;
};
template <typename real> void launch_zero(real *p, int64_t n, cudaStream_t s);
// SMs of the current device (cached per device)
int device_sms();

// host launchers (defined in the .cu files)
template <typename real> void launch_push(const PushArgs<real> &a, cudaStream_t s);
template <typename real> void launch_ions(const PushArgs<real> &a, cudaStream_t s);
template <typename real> void launch_bucket(const BucketArgs<real> &a, cudaStream_t s);
template <typename real> void launch_compact(const CompactArgs<real> &a, cudaStream_t s);
template <typename real> void launch_sort_cells(const SortArgs<real> &a, cudaStream_t s);
template <typename real>
void launch_rho(const Geom &g, const Species<real> &sp, const int *lo, const int *hi, real qfac, real *rho,
                cudaStream_t s);
template <typename real>
void launch_particle_sums(const Geom &g, const Species<real> &sp, const int *lo, const int *hi, double q,
                          const real u_drift[3], double *partials, int nblocks, cudaStream_t s);
void launch_inject(const InjectArgs &a, cudaStream_t s);
template <typename real>
void launch_btd(const BtdArgs<real> &a, cudaStream_t s);
// component comp (0..5) of the lab-frame E, B on the grid (F the component,
// P its partner: By, Bx, -, Ey, Ex, -) into out; FP64 transformation
template <typename real>
void launch_lab_fields(const Geom &g, const real *F, const real *P, int comp, real *out, double gam, double beta,
                       int sms, cudaStream_t s);
// moving window: every field plane k of dst takes plane k + S of src (zero
// above), for the nine components
template <typename real>
void launch_window_fields(const Geom &g, real *const src[9], real *const dst[9], int S, cudaStream_t s);
// moving window: the bucket of tile t of the output side takes the bucket of
// tile t + m ntx nty of the input side with every cell index S = m tz lower
template <typename real>
void launch_window_particles(const Geom &g, const Species<real> &in, const Species<real> &out, const int *in_lo,
                             const int *in_hi, int *out_lo, int *out_hi, int m, int S, cudaStream_t s);

template <typename real>
void launch_yee(const Geom &g, real *const F[9], real *const F1[6], double dt, double hx, double hy, double hz,
                cudaStream_t s);
// (err: the device error word for a bounded wait that ran out; may be null)
template <typename real>
void launch_filter(const Geom &g, real *const J[3], real *tmp, int npass, cudaStream_t s, unsigned *err = nullptr);
// all passes from src (3 contiguous components, left unchanged) into J;
// false (nothing launched) where only the per-pass path applies (npass > 4)
template <typename real>
bool launch_filter_from(const Geom &g, const real *src, real *const J[3], int npass, cudaStream_t s,
                        unsigned *err = nullptr);
// j0p non-null: the amplitude is read from device memory (a captured step)
template <typename real>
void launch_antenna(const Geom &g, real *J, int pol, int ka, double j0, double hx, double hy,
                    double xc, double yc, double waist, cudaStream_t s, const double *j0p = nullptr);
template <typename real>
void launch_field_sums(const Geom &g, real *const F[9], double *partials, int nblocks,
                       cudaStream_t s);
// adjoint: flat forward steps (electrons, and the slots' ions) and their transposes
template <typename real> void launch_adj_push(const AdjArgs<real> &a, cudaStream_t s);
template <typename real> void launch_adj_push_vjp(const AdjArgs<real> &a, cudaStream_t s);
template <typename real>
void launch_adj_yee(const Geom &g, real *lE[3], real *lB[3], real *lE0[3], real *pE[3], real *lJ[3], double dt,
                    double hx, double hy, double hz, cudaStream_t s);
template <typename real>
void launch_adj_antenna(const Geom &g, const real *lJ, int pol, int ka, double hx, double hy, double xc, double yc,
                        double waist, double fa, double fw, double *s, cudaStream_t st);
void launch_adj_profile(int64_t n, const double *lw, const void *w, int precision, const double *zeta, int M,
                        const double *coef, double *out, cudaStream_t s);
// planes[k] = 1 where any of the three components of lJ is non-zero on plane k
template <typename real>
void launch_adj_planes(const Geom &g, const real *F, int nc, unsigned char *near, cudaStream_t s);

}  // namespace pic
