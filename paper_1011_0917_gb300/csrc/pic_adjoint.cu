// pic_adjoint.cu -- reverse mode (adjoint) of the step, 2D3V and 3D, CIC and
// quadratic shapes.
//
// The step is differentiated as the composition it is (section "Effect of the
// hyperbolic rotation in Minkowski space" sets up the boosted-frame run; the
// reverse mode is this library's own extension):
//   gather  E_p = G(E^n, B^n; x^n)          Boris  du^{n+1/2} = R(du^{n-1/2}, E_p, B_p)
//   move    x^{n+1} = x^n + dt v(du^{n+1/2}) deposit J = D(x^n, x^{n+1}, w, v_y)
//   antenna J += A(t; a0, w0)                filter J_f = F J
//   Yee     (E, B)^{n+1} = Y(E^n, B^n, J_f) (with Mur's condition on the z ends)
//   inject  new particles at fixed positions with weights w(c_m).
// Every map is transposed by hand: Y and F are linear (F is symmetric), the
// particle maps are differentiated along each trajectory.  Particles live in
// a fixed-order ("flat") store during an adjoint run, so that slot p is the
// same particle at every step; the forward states of a segment of K steps are
// recomputed from a checkpoint and kept while the segment is reversed.
//
// Units and layout are those of the forward path: positions as cell index
// plus an offset in [0, 1) of the working precision, momenta relative to the
// plasma drift, fields (nz+1) x ny x nx per component (ny = 1 in 2D).
// Cotangents of positions are per cell (d/d offset): the shape weights are
// differentiated on their own support (CIC: (1 - d, d) and (-1, +1);
// quadratic: the three B-spline pieces and their slopes).
#include "pic_internal.cuh"

namespace pic {

namespace {

constexpr double kTwoPiD = 6.283185307179586;

unsigned adj_grid(int64_t n, int block)
{
    int64_t b = (n + block - 1) / block;
    const int64_t cap = (int64_t)device_sms() * 32;
    return (unsigned)(b < cap ? (b > 0 ? b : 1) : cap);
}

// (i, j, k) of node o of a component; 32-bit division when the component
// has fewer than 2^31 nodes (every grid that fits a GPU's memory here)
__device__ __forceinline__ void node_ijk(const Geom &g, int64_t o, int &i, int &j, int &k)
{
    if (g.ncomp <= 0x7fffffffLL) {
        const unsigned u = (unsigned)o, pl = (unsigned)g.plane, nx = (unsigned)g.nx;
        const unsigned kk = u / pl, r = u - kk * pl, jj = r / nx;
        k = (int)kk;
        j = (int)jj;
        i = (int)(r - jj * nx);
    } else {
        k = (int)(o / g.plane);
        const int64_t r = o - (int64_t)k * g.plane;
        j = (int)(r / g.nx);
        i = (int)(r - (int64_t)j * g.nx);
    }
}

// Is every node a particle in cell (ci, cj, ck) reads or deposits to (gather
// supports, Esirkepov windows of a move of less than a cell) inside the grid,
// with no wrap and no clipping?  Such a particle addresses its nodes directly.
template <int DIM, int S>
__device__ __forceinline__ bool inner_cell(const Geom &g, int ci, int cj, int ck)
{
    constexpr int M = S + 3;
    return ci >= M && ci <= g.nx - M - 2 && (DIM == 2 || (cj >= M && cj <= g.ny - M - 2)) && ck >= M &&
           ck <= g.nz - M - 2;
}

// field value at node (i, j, k) of a component (x, y periodic; z periodic or
// zero outside the component's valid range; `inner`: the node is known to be
// inside, see inner_cell)
template <typename real>
__device__ __forceinline__ real fval(const Geom &g, const real *F, int i, int j, int k, bool half_z, bool inner)
{
    if (inner) return F[(int64_t)k * g.plane + (j * g.nx + i)];
    i = wrap1(i, g.nx);
    j = g.dim == 3 ? wrap1(j, g.ny) : 0;
    if (g.bc_z == 0) k = wrapi(k, g.nz);
    else if (k < 0 || k > zmax_of(g, half_z)) return real(0);
    return F[((int64_t)k * g.ny + j) * g.nx + i];
}

// atomically add v at node (i, j, k) (dropped outside the valid z range; an
// exact zero, e.g. a window node outside both supports, is not added)
template <typename real>
__device__ __forceinline__ void fadd(const Geom &g, real *F, int i, int j, int k, bool half_z, real v, bool inner)
{
    if (v == real(0)) return;
    if (inner) {
        atomicAdd(F + (int64_t)k * g.plane + (j * g.nx + i), v);
        return;
    }
    i = wrap1(i, g.nx);
    j = g.dim == 3 ? wrap1(j, g.ny) : 0;
    if (g.bc_z == 0) k = wrapi(k, g.nz);
    else if (k < 0 || k > zmax_of(g, half_z)) return;
    atomicAdd(F + ((int64_t)k * g.ny + j) * g.nx + i, v);
}

// shape weights of order S and their first node for one staggered axis:
// integer nodes (half = false) or half-integer nodes (half = true, node index
// i for i + 1/2)
template <int S, typename real>
__device__ __forceinline__ int axis_weights(real o, bool half, real w[S + 1])
{
    return half ? half_weights<S>(o, w) : offset_weights<S>(o, w);
}

// d w / d p of the weights spline_weights<S>(p) gives (the same support):
// CIC (-1, +1); quadratic (-(1/2 - d), -2 d, 1/2 + d), d = p - floor(p + 1/2)
template <int S, typename real>
__device__ __forceinline__ void spline_dw(real p, real dw[S + 1])
{
    if (S == 1) {
        dw[0] = real(-1);
        dw[1] = real(1);
    } else {
        const real d = p - floor(p + real(0.5));
        dw[0] = -(real(0.5) - d);
        dw[1] = real(-2) * d;
        dw[2] = real(0.5) + d;
    }
}

// the staggering of the six E, B components: half-integer along x, y, z?
__device__ __forceinline__ bool hx_of(int c) { return c == 0 || c == 4 || c == 5; }
__device__ __forceinline__ bool hy_of(int c) { return c == 1 || c == 3 || c == 5; }
__device__ __forceinline__ bool hz_of(int c) { return c == 2 || c == 3 || c == 4; }

// T(u, v) = S0u (S0v + DSv / 2) + DSu (S0v / 2 + DSv / 3): the path-averaged
// transverse shape product of Esirkepov's weights
template <typename real>
__device__ __forceinline__ real tshape(real s0u, real dsu, real s0v, real dsv)
{
    return s0u * (s0v + real(0.5) * dsv) + dsu * (real(0.5) * s0v + real(1) / real(3) * dsv);
}

// The Boris rotation of boris() (same expressions, same rounding) with the
// intermediate values its transpose needs
template <typename real>
struct BorisFwd {
    real dm[3], um[3], igm, fb, t[3], s2, s[3], up[3], u[3];
    __device__ __forceinline__ BorisFwd(const real du[3], real U, const real e[3], const real b[3], real eps)
    {
        dm[0] = du[0] + eps * e[0];
        dm[1] = du[1] + eps * e[1];
        dm[2] = du[2] + eps * e[2];
        um[0] = dm[0];
        um[1] = dm[1];
        um[2] = U + dm[2];
        igm = rsqrt_p(real(1) + um[0] * um[0] + um[1] * um[1] + um[2] * um[2]);
        fb = eps * igm;
        t[0] = fb * b[0];
        t[1] = fb * b[1];
        t[2] = fb * b[2];
        const real t2 = t[0] * t[0] + t[1] * t[1] + t[2] * t[2];
        s2 = div_p(real(2), real(1) + t2);
        s[0] = s2 * t[0];
        s[1] = s2 * t[1];
        s[2] = s2 * t[2];
        up[0] = um[0] + (um[1] * t[2] - um[2] * t[1]);
        up[1] = um[1] + (um[2] * t[0] - um[0] * t[2]);
        up[2] = um[2] + (um[0] * t[1] - um[1] * t[0]);
        u[0] = dm[0] + (up[1] * s[2] - up[2] * s[1]) + eps * e[0];
        u[1] = dm[1] + (up[2] * s[0] - up[0] * s[2]) + eps * e[1];
        u[2] = dm[2] + (up[0] * s[1] - up[1] * s[0]) + eps * e[2];
    }
};

// gathered E (0..2) and B (3..5) at a particle, with the weights and first
// nodes of every component (kept for the transpose; y trivial in 2D)
template <typename real, int DIM, int S>
struct GatherFwd {
    real wx[6][S + 1], wy[6][S + 1], wz[6][S + 1], f[6];
    int bx[6], by[6], bz[6];
    template <typename Args>
    __device__ __forceinline__ GatherFwd(const Args &a, int ci, int cj, int ck, real ox, real oy, real oz,
                                         bool inner)
    {
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            bx[c] = ci + axis_weights<S>(ox, hx_of(c), wx[c]);
            if (DIM == 3) {
                by[c] = cj + axis_weights<S>(oy, hy_of(c), wy[c]);
            } else {
                by[c] = 0;
#pragma unroll
                for (int q = 0; q <= S; ++q) wy[c][q] = real(q == 0);
            }
            bz[c] = ck + axis_weights<S>(oz, hz_of(c), wz[c]);
            const real *F = c < 3 ? a.E[c] : a.B[c - 3];
            real sum = 0;
#pragma unroll
            for (int cc = 0; cc <= S; ++cc) {
#pragma unroll
                for (int b = 0; b < (DIM == 3 ? S + 1 : 1); ++b) {
                    real r = 0;
#pragma unroll
                    for (int q = 0; q <= S; ++q)
                        r += wx[c][q] * fval(a.g, F, bx[c] + q, by[c] + b, bz[c] + cc, hz_of(c), inner);
                    sum += wz[c][cc] * wy[c][b] * r;
                }
            }
            f[c] = sum;
        }
    }
};

// The gather of GatherFwd (same weights, same sums) together with the
// gradient of every gathered component with respect to the particle's
// position (d/dx, d/dy, d/dz of sum w F: the weights' slopes in place of the
// weights along one axis), read from the same field values in one pass
template <typename real, int DIM, int S>
struct GatherGrad {
    real wx[6][S + 1], wy[6][S + 1], wz[6][S + 1], f[6], gx[6], gy[6], gz[6];
    int bx[6], by[6], bz[6];
    template <typename Args>
    __device__ __forceinline__ GatherGrad(const Args &a, int ci, int cj, int ck, real ox, real oy, real oz,
                                          bool inner, bool load)
    {
        real dxi[S + 1], dxh[S + 1], dyi[S + 1], dyh[S + 1], dzi[S + 1], dzh[S + 1];
        spline_dw<S>(ox, dxi);
        spline_dw<S>(ox - real(0.5), dxh);
        spline_dw<S>(oz, dzi);
        spline_dw<S>(oz - real(0.5), dzh);
        if (DIM == 3) {
            spline_dw<S>(oy, dyi);
            spline_dw<S>(oy - real(0.5), dyh);
        }
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            bx[c] = ci + axis_weights<S>(ox, hx_of(c), wx[c]);
            if (DIM == 3) {
                by[c] = cj + axis_weights<S>(oy, hy_of(c), wy[c]);
            } else {
                by[c] = 0;
#pragma unroll
                for (int q = 0; q <= S; ++q) wy[c][q] = real(q == 0);
            }
            bz[c] = ck + axis_weights<S>(oz, hz_of(c), wz[c]);
            const real *dwx = hx_of(c) ? dxh : dxi, *dwy = hy_of(c) ? dyh : dyi, *dwz = hz_of(c) ? dzh : dzi;
            const real *F = c < 3 ? a.E[c] : a.B[c - 3];
            real sum = 0, sx = 0, sy = 0, sz = 0;
#pragma unroll
            for (int cc = 0; cc <= S; ++cc) {
#pragma unroll
                for (int b = 0; b < (DIM == 3 ? S + 1 : 1); ++b) {
                    real r = 0, rd = 0;
#pragma unroll
                    for (int q = 0; q <= S; ++q) {
                        const real v = load ? fval(a.g, F, bx[c] + q, by[c] + b, bz[c] + cc, hz_of(c), inner) : real(0);
                        r += wx[c][q] * v;
                        rd += dwx[q] * v;
                    }
                    sum += wz[c][cc] * wy[c][b] * r;
                    sx += wz[c][cc] * wy[c][b] * rd;
                    if (DIM == 3) sy += wz[c][cc] * dwy[b] * r;
                    sz += dwz[cc] * wy[c][b] * r;
                }
            }
            f[c] = sum;
            gx[c] = sx;
            gy[c] = sy;
            gz[c] = sz;
        }
    }
};

}  // namespace

// ------------------------------------------------------------ flat forward

// A slot's drifting-ion state, loaded with the electron's before either is
// used so that the loads of both share one memory round trip.
template <typename real, int DIM>
struct IonSlot {
    bool alive;
    int ci, cj, ck;
    real ox, oy, oz;
    __device__ __forceinline__ IonSlot(const AdjArgs<real> &a, int64_t p)
    {
        alive = a.with_ions && a.iin.alive[p];
        ci = cj = ck = 0;
        ox = oy = oz = real(0);
        if (a.with_ions) {
            ci = a.ion_ci[p];
            ck = a.iin.ck[p];
            ox = a.ion_ox[p];
            oz = a.iin.oz[p];
            if (DIM == 3) {
                cj = a.ion_cj[p];
                oy = a.ion_oy[p];
            }
        }
    }
};

// One step of drifting ion p of the flat store (alive, state i, weight w):
// z move by the drift's displacement and the z-only deposit (the electron
// kernel calls it for the ion of every slot).
template <typename real, int DIM, int S>
__device__ __forceinline__ void adj_ion_step(const AdjArgs<real> &a, const Drift<real> &drift, int64_t p,
                                             const IonSlot<real, DIM> &i, real w, bool deposit)
{
    constexpr int W = S + 2;
    const Geom &g = a.g;
    const int ci = i.ci, cj = i.cj, ck = i.ck;
    const real ox = i.ox, oy = i.oy, oz = i.oz;
    const bool inner = inner_cell<DIM, S>(g, ci, cj, ck);
    const real z1 = add_rn(oz, drift.dz);
    real S0z[W], DSz[W], wx[S + 1], wy[S + 1];
    bool cr;
    const int az = ck + esirk_axis_c<S>(oz, z1, S0z, DSz, cr);
    const int bx = ci + offset_weights<S>(ox, wx);
    int by = 0;
    if (DIM == 3) by = cj + offset_weights<S>(oy, wy);
    else
#pragma unroll
        for (int q = 0; q <= S; ++q) wy[q] = real(q == 0);
    const real fz = a.jfac_iz * w;
    real acc = 0;
    if (deposit) {
#pragma unroll
        for (int c = 0; c < W - 1; ++c) {
            acc += DSz[c];
#pragma unroll
            for (int b = 0; b < (DIM == 3 ? S + 1 : 1); ++b)
#pragma unroll
                for (int q = 0; q <= S; ++q)
                    fadd(g, a.J[2], bx + q, by + b, az + c, true, fz * acc * wx[q] * wy[b], inner);
        }
    }
    int sz = 0;
    real noz = z1;
    if (z1 < real(0)) {
        noz = z1 + real(1);
        sz = -1;
        if (noz >= real(1)) { noz = 0; sz = 0; }
    }
    int nk = ck + sz;
    bool alive = true;
    if (nk < 0) {
        if (g.bc_z == 0) nk += g.nz;
        else alive = false;
    }
    a.iout.alive[p] = alive ? 1 : 0;
    a.iout.ck[p] = nk;
    a.iout.oz[p] = noz;
}

// One step of the electrons of the flat store: gather E^n, B^n at x^n, Boris,
// move, Esirkepov deposit with global atomics, re-cell; state `in` -> `out`.
// Shape order S: supports of S + 1 nodes, Esirkepov windows of W = S + 2.
template <typename real, int DIM, int S>
__global__ void __launch_bounds__(256, 6) adj_push_kernel(AdjArgs<real> a)
{
    constexpr int W = S + 2, WY = DIM == 3 ? W : 1;
    const Geom &g = a.g;
    const Drift<real> drift(a.u_drift, a.dtdh[2]);
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < a.n; p += (int64_t)gridDim.x * blockDim.x) {
        // the slot's whole state first (a dead slot's values are not used)
        const bool alive = a.in.alive[p];
        const int ci = a.in.ci[p], cj = DIM == 3 ? a.in.cj[p] : 0, ck = a.in.ck[p];
        const real ox = a.in.ox[p], oy = DIM == 3 ? a.in.oy[p] : real(0), oz = a.in.oz[p], w = a.w[p];
        const real du[3] = {a.in.ux[p], a.in.uy[p], a.in.uz[p]};
        const IonSlot<real, DIM> ion(a, p);
        // no field within reach: the gather is zero (skipped); an electron
        // at rest relative to the drift then moves with its drifting ion, bit
        // for bit, and if the two share their position their deposits cancel
        // exactly: neither is made
        const bool field = alive && a.f_plane[ck];
        const bool together = alive && ion.alive && !field && du[0] == real(0) && du[1] == real(0) &&
                              du[2] == real(0) && ci == ion.ci && ck == ion.ck && ox == ion.ox && oz == ion.oz &&
                              (DIM == 2 || (cj == ion.cj && oy == ion.oy));
        if (ion.alive) adj_ion_step<real, DIM, S>(a, drift, p, ion, w, !together);
        else if (a.with_ions) a.iout.alive[p] = 0;
        if (!alive) {
            a.out.alive[p] = 0;
            continue;
        }
        const bool inner = inner_cell<DIM, S>(g, ci, cj, ck);
        real fe[6];
        if (field) {
            const GatherFwd<real, DIM, S> gf(a, ci, cj, ck, ox, oy, oz, inner);
#pragma unroll
            for (int c = 0; c < 6; ++c) fe[c] = gf.f[c];
        } else {
#pragma unroll
            for (int c = 0; c < 6; ++c) fe[c] = real(0);
        }
        const BorisFwd<real> bf(du, drift.U, fe, fe + 3, a.eps);
        const real ux = bf.u[0], uy = bf.u[1], uz = bf.u[2];
        real vx, vy;
        const real dvz = drift_velocity(drift, ux, uy, uz, vx, vy);
        const real x1 = ox + vx * a.dtdh[0];
        const real y1 = DIM == 3 ? oy + vy * a.dtdh[1] : real(0);
        const real z1 = add_rn(oz, drift.dz) + dvz * a.dtdh[2];
        real S0x[W], DSx[W], S0y[W], DSy[W], S0z[W], DSz[W];
#pragma unroll
        for (int q = 0; q < W; ++q) {
            S0y[q] = real(q == 0);
            DSy[q] = real(0);
        }
        bool cr;
        const int ax = ci + esirk_axis_c<S>(ox, x1, S0x, DSx, cr);
        const int ay = DIM == 3 ? cj + esirk_axis_c<S>(oy, y1, S0y, DSy, cr) : 0;
        const int az = ck + esirk_axis_c<S>(oz, z1, S0z, DSz, cr);
        real Rx[W], Ry[W], Rz[W];
        {
            real sx_ = 0, sy_ = 0, sz_ = 0;
#pragma unroll
            for (int q = 0; q < W; ++q) {
                sx_ += DSx[q];
                sy_ += DSy[q];
                sz_ += DSz[q];
                Rx[q] = sx_;
                Ry[q] = sy_;
                Rz[q] = sz_;
            }
        }
        const real fx = a.jfac[0] * w, fy = a.jfac[1] * w, fz = a.jfac[2] * w, fyv = a.jyfac * w * vy;
        if (!together) {
#pragma unroll
            for (int q = 0; q < W; ++q)
#pragma unroll
                for (int b = 0; b < WY; ++b)
#pragma unroll
                    for (int c = 0; c < W; ++c) {
                        if (q < W - 1)
                            fadd(g, a.J[0], ax + q, ay + b, az + c, false,
                                 fx * Rx[q] * tshape(S0y[b], DSy[b], S0z[c], DSz[c]), inner);
                        if (DIM == 3) {
                            if (b < W - 1)
                                fadd(g, a.J[1], ax + q, ay + b, az + c, false,
                                     fy * Ry[b] * tshape(S0z[c], DSz[c], S0x[q], DSx[q]), inner);
                        } else {
                            fadd(g, a.J[1], ax + q, 0, az + c, false, fyv * tshape(S0x[q], DSx[q], S0z[c], DSz[c]),
                                 inner);
                        }
                        if (c < W - 1)
                            fadd(g, a.J[2], ax + q, ay + b, az + c, true,
                                 fz * Rz[c] * tshape(S0x[q], DSx[q], S0y[b], DSy[b]), inner);
                    }
        }
        // new cell (an offset that rounds to 1 moves on)
        int sx = (int)floor(x1), sy = DIM == 3 ? (int)floor(y1) : 0, sz = (int)floor(z1);
        real nox = x1 - real(sx), noy = DIM == 3 ? y1 - real(sy) : real(0), noz = z1 - real(sz);
        if (nox >= real(1)) { sx += 1; nox = 0; }
        if (DIM == 3 && noy >= real(1)) { sy += 1; noy = 0; }
        if (noz >= real(1)) { sz += 1; noz = 0; }
        const int ni = wrapi(ci + sx, g.nx), nj = DIM == 3 ? wrapi(cj + sy, g.ny) : 0;
        int nk = ck + sz;
        bool stays = true;
        if (g.bc_z == 0) nk = wrapi(nk, g.nz);
        else if (nk < 0 || nk >= g.nz) stays = false;
        a.out.alive[p] = stays ? 1 : 0;
        a.out.ci[p] = ni;
        a.out.ck[p] = nk;
        a.out.ox[p] = nox;
        a.out.oz[p] = noz;
        if (DIM == 3) {
            a.out.cj[p] = nj;
            a.out.oy[p] = noy;
        }
        a.out.ux[p] = ux;
        a.out.uy[p] = uy;
        a.out.uz[p] = uz;
    }
}

// ------------------------------------------------------------- reverse

// d/dx of the window node q's weight, the support (S + 1 nodes) starting at
// window node r with weight derivatives dw
template <int S, typename real>
__device__ __forceinline__ real dwin(int q, int r, const real dw[S + 1])
{
    real v = 0;
#pragma unroll
    for (int m = 0; m <= S; ++m) v = (q == r + m) ? dw[m] : v;
    return v;
}

// Weight cotangent of a slot's drifting ion (state i, alive) in one step (its
// position does not depend on the parameters); the electron VJP kernel calls
// it for every slot and adds the result to the slot's weight cotangent.
template <typename real, int DIM, int S>
__device__ __forceinline__ real adj_ion_vjp_one(const AdjArgs<real> &a, const Drift<real> &drift,
                                                const IonSlot<real, DIM> &i)
{
    constexpr int W = S + 2;
    const Geom &g = a.g;
    const int ci = i.ci, cj = i.cj, ck = i.ck;
    const bool inner = inner_cell<DIM, S>(g, ci, cj, ck);
    if (!a.lj_plane[ck]) return real(0);  // no current cotangent where this ion deposits
    const real ox = i.ox, oy = i.oy, oz = i.oz;
    const real z1 = add_rn(oz, drift.dz);
    real S0z[W], DSz[W], wx[S + 1], wy[S + 1];
    bool cr;
    const int az = ck + esirk_axis_c<S>(oz, z1, S0z, DSz, cr);
    const int bx = ci + offset_weights<S>(ox, wx);
    int by = 0;
    if (DIM == 3) by = cj + offset_weights<S>(oy, wy);
    else
#pragma unroll
        for (int q = 0; q <= S; ++q) wy[q] = real(q == 0);
    real acc = 0, L = 0;
#pragma unroll
    for (int c = 0; c < W - 1; ++c) {
        acc += DSz[c];
#pragma unroll
        for (int b = 0; b < (DIM == 3 ? S + 1 : 1); ++b)
#pragma unroll
            for (int q = 0; q <= S; ++q)
                L += acc * wx[q] * wy[b] * fval(g, (const real *)a.J[2], bx + q, by + b, az + c, true, inner);
    }
    return a.jfac_iz * L;
}

// Cotangents of one electron step.  Reads the state at n (x^n, du^{n-1/2}),
// E^n, B^n, the filtered-and-transposed current cotangent lJ, and the
// particle's cotangents of x^{n+1}, du^{n+1/2}; writes those of x^n,
// du^{n-1/2} in their place, adds the gather's field cotangents to lE, lB and
// the weight's cotangent to lw.
template <typename real, int DIM, int S>
__global__ void __launch_bounds__(256, 3) adj_push_vjp_kernel(AdjArgs<real> a)
{
    constexpr int W = S + 2, WY = DIM == 3 ? W : 1;
    const Geom &g = a.g;
    const Drift<real> drift(a.u_drift, a.dtdh[2]);
    const real half = real(0.5), third = real(1) / real(3);
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < a.n; p += (int64_t)gridDim.x * blockDim.x) {
        // the slot's whole state and cotangents first (a dead slot's values
        // are not used)
        const bool alive = a.in.alive[p];
        const int ci = a.in.ci[p], cj = DIM == 3 ? a.in.cj[p] : 0, ck = a.in.ck[p];
        const real ox = a.in.ox[p], oy = DIM == 3 ? a.in.oy[p] : real(0), oz = a.in.oz[p], w = a.w[p];
        const real du0[3] = {a.in.ux[p], a.in.uy[p], a.in.uz[p]};
        const real clx = a.lx[p], cly = DIM == 3 ? a.ly[p] : real(0), clz = a.lz[p];
        const real clux = a.lux[p], cluy = a.luy[p], cluz = a.luz[p];
        const double lw0 = a.lw[p];
        const IonSlot<real, DIM> ion(a, p);
        const real Lwi = ion.alive ? adj_ion_vjp_one<real, DIM, S>(a, drift, ion) : real(0);
        if (!alive) {
            if (Lwi != real(0)) a.lw[p] = lw0 + (double)Lwi;
            continue;
        }
        // a particle whose incoming cotangents are zero and whose deposit
        // reaches no node with a current cotangent contributes nothing (its
        // gather cotangents are then zero too): skip it
        if (clx == real(0) && clz == real(0) && cly == real(0) && clux == real(0) && cluy == real(0) &&
            cluz == real(0) && !a.lj_plane[ck]) {
            if (Lwi != real(0)) a.lw[p] = lw0 + (double)Lwi;
            continue;
        }
        // ---- recompute the forward values of this step
        const bool inner = inner_cell<DIM, S>(g, ci, cj, ck);
        const GatherGrad<real, DIM, S> gf(a, ci, cj, ck, ox, oy, oz, inner, a.f_plane[ck] != 0);
        const BorisFwd<real> bf(du0, drift.U, gf.f, gf.f + 3, a.eps);
        const real eps = a.eps, U = drift.U;
        const real ux = bf.u[0], uy = bf.u[1], uz = bf.u[2];
        real vx, vy;
        const real dvz = drift_velocity(drift, ux, uy, uz, vx, vy);
        const real x1 = ox + vx * a.dtdh[0];
        const real y1 = DIM == 3 ? oy + vy * a.dtdh[1] : real(0);
        const real z1 = add_rn(oz, drift.dz) + dvz * a.dtdh[2];
        real S0x[W], DSx[W], S0y[W], DSy[W], S0z[W], DSz[W];
#pragma unroll
        for (int q = 0; q < W; ++q) {
            S0y[q] = real(q == 0);
            DSy[q] = real(0);
        }
        bool cr;
        real wtmp[S + 1], dw0x[S + 1], dw1x[S + 1], dw0y[S + 1], dw1y[S + 1], dw0z[S + 1], dw1z[S + 1];
        const int b0x = offset_weights<S>(ox, wtmp), b1x = spline_weights<S>(x1, wtmp);
        const int b0z = offset_weights<S>(oz, wtmp), b1z = spline_weights<S>(z1, wtmp);
        spline_dw<S>(ox, dw0x);
        spline_dw<S>(x1, dw1x);
        spline_dw<S>(oz, dw0z);
        spline_dw<S>(z1, dw1z);
        const int anx = esirk_axis_c<S>(ox, x1, S0x, DSx, cr);
        const int anz = esirk_axis_c<S>(oz, z1, S0z, DSz, cr);
        int b0y = 0, b1y = 0, any_ = 0;
        if (DIM == 3) {
            b0y = offset_weights<S>(oy, wtmp);
            b1y = spline_weights<S>(y1, wtmp);
            spline_dw<S>(oy, dw0y);
            spline_dw<S>(y1, dw1y);
            any_ = esirk_axis_c<S>(oy, y1, S0y, DSy, cr);
        }
        const int ax = ci + anx, ay = cj + any_, az = ck + anz;
        real Rx[W], Ry[W], Rz[W];
        {
            real sx_ = 0, sy_ = 0, sz_ = 0;
#pragma unroll
            for (int q = 0; q < W; ++q) {
                sx_ += DSx[q];
                sy_ += DSy[q];
                sz_ += DSz[q];
                Rx[q] = sx_;
                Ry[q] = sy_;
                Rz[q] = sz_;
            }
        }
        // ---- deposit transposed: dL/dS0, dL/dDS per window node, dL/dw, dL/dvy
        const real fx = a.jfac[0] * w, fy = a.jfac[1] * w, fz = a.jfac[2] * w;
        const real fy1 = a.jyfac * vy;  // 2D out-of-plane factor over w
        real gS0x[W], gDSx[W], gS0y[W], gDSy[W], gS0z[W], gDSz[W], gRx[W], gRy[W], gRz[W];
#pragma unroll
        for (int q = 0; q < W; ++q)
            gS0x[q] = gDSx[q] = gS0y[q] = gDSy[q] = gS0z[q] = gDSz[q] = gRx[q] = gRy[q] = gRz[q] = real(0);
        real Lw = 0, Ly = 0;
        // derivatives of T(u, v) with respect to S0u, DSu (the same form in v)
        auto dT0 = [&](real s0v, real dsv) { return s0v + half * dsv; };
        auto dT1 = [&](real s0v, real dsv) { return half * s0v + third * dsv; };
#pragma unroll
        for (int q = 0; q < W; ++q)
#pragma unroll
            for (int b = 0; b < WY; ++b)
#pragma unroll
                for (int c = 0; c < W; ++c) {
                    if (q < W - 1) {  // Jx = fx Rx[q] T(y_b, z_c)
                        const real l = fval(g, (const real *)a.J[0], ax + q, ay + b, az + c, false, inner);
                        const real T = tshape(S0y[b], DSy[b], S0z[c], DSz[c]);
                        gRx[q] += fx * T * l;
                        Lw += a.jfac[0] * Rx[q] * T * l;
                        const real k = fx * Rx[q] * l;
                        gS0z[c] += k * dT0(S0y[b], DSy[b]);
                        gDSz[c] += k * dT1(S0y[b], DSy[b]);
                        if (DIM == 3) {
                            gS0y[b] += k * dT0(S0z[c], DSz[c]);
                            gDSy[b] += k * dT1(S0z[c], DSz[c]);
                        }
                    }
                    if (DIM == 3) {
                        if (b < W - 1) {  // Jy = fy Ry[b] T(z_c, x_q)
                            const real l = fval(g, (const real *)a.J[1], ax + q, ay + b, az + c, false, inner);
                            const real T = tshape(S0z[c], DSz[c], S0x[q], DSx[q]);
                            gRy[b] += fy * T * l;
                            Lw += a.jfac[1] * Ry[b] * T * l;
                            const real k = fy * Ry[b] * l;
                            gS0z[c] += k * dT0(S0x[q], DSx[q]);
                            gDSz[c] += k * dT1(S0x[q], DSx[q]);
                            gS0x[q] += k * dT0(S0z[c], DSz[c]);
                            gDSx[q] += k * dT1(S0z[c], DSz[c]);
                        }
                    } else {  // 2D out of plane: Jy = fy1 w T(x_q, z_c)
                        const real l = fval(g, (const real *)a.J[1], ax + q, 0, az + c, false, inner);
                        Ly += tshape(S0x[q], DSx[q], S0z[c], DSz[c]) * l;
                        const real k = fy1 * w * l;
                        gS0x[q] += k * dT0(S0z[c], DSz[c]);
                        gDSx[q] += k * dT1(S0z[c], DSz[c]);
                        gS0z[c] += k * dT0(S0x[q], DSx[q]);
                        gDSz[c] += k * dT1(S0x[q], DSx[q]);
                    }
                    if (c < W - 1) {  // Jz = fz Rz[c] T(x_q, y_b)
                        const real l = fval(g, (const real *)a.J[2], ax + q, ay + b, az + c, true, inner);
                        const real T = tshape(S0x[q], DSx[q], S0y[b], DSy[b]);
                        gRz[c] += fz * T * l;
                        Lw += a.jfac[2] * Rz[c] * T * l;
                        const real k = fz * Rz[c] * l;
                        gS0x[q] += k * dT0(S0y[b], DSy[b]);
                        gDSx[q] += k * dT1(S0y[b], DSy[b]);
                        if (DIM == 3) {
                            gS0y[b] += k * dT0(S0x[q], DSx[q]);
                            gDSy[b] += k * dT1(S0x[q], DSx[q]);
                        }
                    }
                }
        if (DIM == 2) Lw += fy1 * Ly;
        // running sums: R[q] = sum_{q' <= q} DS[q']
        {
            real sx_ = 0, sy_ = 0, sz_ = 0;
#pragma unroll
            for (int q = W - 1; q >= 0; --q) {
                sx_ += gRx[q];
                sy_ += gRy[q];
                sz_ += gRz[q];
                gDSx[q] += sx_;
                gDSy[q] += sy_;
                gDSz[q] += sz_;
            }
        }
        // DS = S1 - S0 on the window: dL/dS1 = gDS, dL/dS0 = gS0 - gDS; the
        // supports of x0 and x1 start at window nodes b0 - an and b1 - an
        real lx1 = 0, ly1 = 0, lz1 = 0, lx0 = 0, ly0 = 0, lz0 = 0;
#pragma unroll
        for (int q = 0; q < W; ++q) {
            lx0 += (gS0x[q] - gDSx[q]) * dwin<S>(q, b0x - anx, dw0x);
            lx1 += gDSx[q] * dwin<S>(q, b1x - anx, dw1x);
            lz0 += (gS0z[q] - gDSz[q]) * dwin<S>(q, b0z - anz, dw0z);
            lz1 += gDSz[q] * dwin<S>(q, b1z - anz, dw1z);
            if (DIM == 3) {
                ly0 += (gS0y[q] - gDSy[q]) * dwin<S>(q, b0y - any_, dw0y);
                ly1 += gDSy[q] * dwin<S>(q, b1y - any_, dw1y);
            }
        }
        // ---- move transposed: x1 = ox + vx dtdh_x (and y), z1 = oz + dz_d + dvz dtdh_z
        lx1 += clx;
        lz1 += clz;
        if (DIM == 3) ly1 += cly;
        const real lvx = a.dtdh[0] * lx1, lvz = a.dtdh[2] * lz1;
        const real lvy = DIM == 3 ? a.dtdh[1] * ly1 : a.jyfac * w * Ly;
        // velocity transposed: v = u / gamma (u the full momentum), d v / d du
        // = (I - v v^T) / gamma; (I - v v^T) l = l / gamma^2 + v x (l x v)
        // (no cancellation when v is nearly along z)
        const real vz = U * drift.ig + dvz;  // full velocity (drift + departure)
        const real ig = rsqrt_p(drift.g2 + (uz * (real(2) * U + uz) + ux * ux + uy * uy));
        const real ig2 = ig * ig;
        const real cx = lvy * vz - lvz * vy, cy = lvz * vx - lvx * vz, cz = lvx * vy - lvy * vx;  // l x v
        const real lux = clux + ig * (lvx * ig2 + (vy * cz - vz * cy));
        const real luy = cluy + ig * (lvy * ig2 + (vz * cx - vx * cz));
        const real luz = cluz + ig * (lvz * ig2 + (vx * cy - vy * cx));
        // ---- Boris transposed
        const real sx = bf.s[0], sy = bf.s[1], sz = bf.s[2], tx = bf.t[0], ty = bf.t[1], tz = bf.t[2];
        const real upx = bf.up[0], upy = bf.up[1], upz = bf.up[2];
        const real umx = bf.um[0], umy = bf.um[1], umz = bf.um[2];
        const real s2 = bf.s2, sden = half * bf.s2, fb = bf.fb, igm = bf.igm;
        real lE[3] = {eps * lux, eps * luy, eps * luz};  // the last half kick
        real ldmx = lux, ldmy = luy, ldmz = luz;
        // u += up x s: lup = s x lu, ls = lu x up
        const real lupx = sy * luz - sz * luy, lupy = sz * lux - sx * luz, lupz = sx * luy - sy * lux;
        const real lsx = luy * upz - luz * upy, lsy = luz * upx - lux * upz, lsz = lux * upy - luy * upx;
        // up = um + um x t: lum += lup + t x lup, lt = lup x um
        real lumx = lupx + (ty * lupz - tz * lupy);
        real lumy = lupy + (tz * lupx - tx * lupz);
        real lumz = lupz + (tx * lupy - ty * lupx);
        real ltx = lupy * umz - lupz * umy, lty = lupz * umx - lupx * umz, ltz = lupx * umy - lupy * umx;
        // s = s2 t, s2 = 2 / (1 + t^2): d s / d t = s2 I - 4 t t^T / (1 + t^2)^2
        const real tl = tx * lsx + ty * lsy + tz * lsz;
        ltx += s2 * lsx - real(2) * s2 * sden * tx * tl;
        lty += s2 * lsy - real(2) * s2 * sden * ty * tl;
        ltz += s2 * lsz - real(2) * s2 * sden * tz * tl;
        // t = fb B, fb = eps / gamma_m
        const real lB[3] = {fb * ltx, fb * lty, fb * ltz};
        const real lfb = gf.f[3] * ltx + gf.f[4] * lty + gf.f[5] * ltz;
        const real kf = -lfb * fb * igm * igm;  // d fb / d um = -fb um / gamma_m^2
        lumx += kf * umx;
        lumy += kf * umy;
        lumz += kf * umz;
        ldmx += lumx;
        ldmy += lumy;
        ldmz += lumz;
        lE[0] += eps * ldmx;
        lE[1] += eps * ldmy;
        lE[2] += eps * ldmz;
        // ---- gather transposed: position cotangents from the gathered
        // gradients; field cotangents scattered with the gather weights
        const real lf[6] = {lE[0], lE[1], lE[2], lB[0], lB[1], lB[2]};
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            real *LF = c < 3 ? a.lE[c] : a.lB[c - 3];
            const real l = lf[c];
            lx0 += l * gf.gx[c];
            if (DIM == 3) ly0 += l * gf.gy[c];
            lz0 += l * gf.gz[c];
#pragma unroll
            for (int cc = 0; cc <= S; ++cc)
#pragma unroll
                for (int b = 0; b < (DIM == 3 ? S + 1 : 1); ++b)
#pragma unroll
                    for (int q = 0; q <= S; ++q)
                        fadd(g, LF, gf.bx[c] + q, gf.by[c] + b, gf.bz[c] + cc, hz_of(c),
                             l * gf.wx[c][q] * gf.wy[c][b] * gf.wz[c][cc], inner);
        }
        // ---- write the cotangents of x^n, du^{n-1/2}; the weight's
        a.lx[p] = lx1 + lx0;
        a.lz[p] = lz1 + lz0;
        if (DIM == 3) a.ly[p] = ly1 + ly0;
        a.lux[p] = ldmx;
        a.luy[p] = ldmy;
        a.luz[p] = ldmz;
        a.lw[p] = lw0 + (double)Lwi + (double)Lw;
    }
}

// lE += (transpose of B -= h curl E) applied to lB: the gather form of the
// scatter of every B update onto the E nodes it read (hy_ unused in 2D).
template <typename real>
__global__ void adj_curl_e_t_kernel(Geom g, real *lEx, real *lEy, real *lEz, const real *lBx, const real *lBy,
                                    const real *lBz, real hz_, real hx_, real hy_)
{
    const bool per = g.bc_z == 0, d3 = g.dim == 3;
    const int nk = per ? g.nz : g.nz + 1;
    const int64_t plane = g.plane;
    for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < (int64_t)nk * plane;
         o += (int64_t)gridDim.x * blockDim.x) {
        int i, j, k;
        node_ijk(g, o, i, j, k);
        const int im = i == 0 ? g.nx - 1 : i - 1, jm = j == 0 ? g.ny - 1 : j - 1;
        // B on half-integer z (Bx, By) exists for k' in [0, nz); Bz on the E planes
        auto bh = [&](const real *B, int ii, int jj, int kk) -> real {
            if (per) kk = wrapi(kk, g.nz);
            else if (kk < 0 || kk >= g.nz) return real(0);
            return B[((int64_t)kk * g.ny + jj) * g.nx + ii];
        };
        auto bi = [&](const real *B, int ii, int jj, int kk) -> real { return B[((int64_t)kk * g.ny + jj) * g.nx + ii]; };
        lEx[o] += hz_ * (bh(lBy, i, j, k) - bh(lBy, i, j, k - 1));
        lEy[o] += hz_ * (bh(lBx, i, j, k - 1) - bh(lBx, i, j, k)) + hx_ * (bi(lBz, i, j, k) - bi(lBz, im, j, k));
        if (d3) lEx[o] += hy_ * (bi(lBz, i, jm, k) - bi(lBz, i, j, k));
        if (k < g.nz) {
            lEz[o] += hx_ * (bi(lBy, im, j, k) - bi(lBy, i, j, k));
            if (d3) lEz[o] += hy_ * (bi(lBx, i, j, k) - bi(lBx, i, jm, k));
        }
    }
}

// The E update transposed.  From lE1 (cotangent of E^{n+1} after the B half
// step has been transposed) it forms the cotangent of the interior update's
// output (Mur's condition transposed first: the boundary values were computed
// from E^n and the new interior values next to them), the current cotangent
// lJ = -2 pi dt lE1' and the cotangent of E^n, lE0.
template <typename real>
__global__ void adj_e_update_t_kernel(Geom g, const real *lE1x, const real *lE1y, const real *lE1z, real *pEx,
                                      real *pEy, real *pEz, real *lE0x, real *lE0y, real *lE0z, real *lJx,
                                      real *lJy, real *lJz, real cm, real m2pidt)
{
    const bool per = g.bc_z == 0;
    const int nk = g.nz + 1;
    const int64_t plane = g.plane;
    for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < (int64_t)nk * plane;
         o += (int64_t)gridDim.x * blockDim.x) {
        int i, j, k;
        node_ijk(g, o, i, j, k);
        const int64_t r = o - (int64_t)k * plane;  // node within the plane
        const int64_t top = (int64_t)g.nz * plane + r;
        for (int c = 0; c < 2; ++c) {
            const real *L1 = c == 0 ? lE1x : lE1y;
            real *P = c == 0 ? pEx : pEy;
            real *L0 = c == 0 ? lE0x : lE0y;
            real *LJ = c == 0 ? lJx : lJy;
            real vp = 0, v0 = 0;
            if (per) {
                if (k < g.nz) vp = v0 = L1[o];
            } else if (k >= 1 && k <= g.nz - 1) {
                vp = L1[o];
                v0 = L1[o];
                if (k == 1) { vp += cm * L1[r]; v0 += cm * L1[r] + L1[r]; }
                if (k == g.nz - 1) { vp += cm * L1[top]; v0 += cm * L1[top] + L1[top]; }
            } else {
                v0 = -cm * L1[o];  // k = 0 or nz: E^n of the boundary node itself
            }
            P[o] = vp;
            L0[o] = v0;
            LJ[o] = m2pidt * vp;
        }
        const real vz = k < g.nz ? lE1z[o] : real(0);
        pEz[o] = vz;
        lE0z[o] = vz;
        lJz[o] = m2pidt * vz;
    }
}

// lB += dt (curl B)^T applied to lE': the gather form of the scatter of the E
// interior updates onto the B nodes they read.
template <typename real>
__global__ void adj_curl_b_t_kernel(Geom g, const real *pEx, const real *pEy, const real *pEz, real *lBx,
                                    real *lBy, real *lBz, real dthz, real dthx, real dthy)
{
    const bool per = g.bc_z == 0, d3 = g.dim == 3;
    const int nk = g.nz + 1;
    const int64_t plane = g.plane;
    for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < (int64_t)nk * plane;
         o += (int64_t)gridDim.x * blockDim.x) {
        int i, j, k;
        node_ijk(g, o, i, j, k);
        const int ip = i + 1 == g.nx ? 0 : i + 1, jp = j + 1 == g.ny ? 0 : j + 1;
        auto pe = [&](const real *P, int ii, int jj, int kk) -> real {  // E' on the integer-z planes
            if (per) kk = wrapi(kk, g.nz);
            else if (kk < 0 || kk > g.nz) return real(0);
            return P[((int64_t)kk * g.ny + jj) * g.nx + ii];
        };
        auto at = [&](const real *P, int ii, int jj) -> real { return P[((int64_t)k * g.ny + jj) * g.nx + ii]; };
        if (k < g.nz) {
            lBy[o] += dthz * (pe(pEx, i, j, k + 1) - pe(pEx, i, j, k)) + dthx * (at(pEz, i, j) - at(pEz, ip, j));
            lBx[o] += dthz * (pe(pEy, i, j, k) - pe(pEy, i, j, k + 1));
            if (d3) lBx[o] += dthy * (at(pEz, i, jp) - at(pEz, i, j));
        }
        if (k < g.nz || !per) {
            lBz[o] += dthx * (at(pEy, ip, j) - at(pEy, i, j));
            if (d3) lBz[o] += dthy * (at(pEx, i, j) - at(pEx, i, jp));
        }
    }
}

// Sums over the antenna plane: s[0] += j0u sum lJ g, s[1] += j0w sum lJ g r^2
// (g = exp(-r^2 / w0^2) at each node's own staggered transverse position, as
// in the forward), for the a0 and w0 cotangents.
template <typename real>
__global__ void adj_antenna_kernel(Geom g, const real *lJ, int pol, int ka, double hx, double hy, double xc,
                                   double yc, double inv_w2, double fa, double fw, double *s)
{
    double s0 = 0, s1 = 0;
    for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < g.plane;
         o += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(o % g.nx), j = (int)(o / g.nx);
        const double x = ((double)i + (pol == 0 ? 0.5 : 0.0)) * hx - xc;
        double r2 = x * x;
        if (g.dim == 3) {
            const double y = ((double)j + (pol == 1 ? 0.5 : 0.0)) * hy - yc;
            r2 += y * y;
        }
        const double gg = exp(-r2 * inv_w2);
        const double l = (double)lJ[(int64_t)ka * g.plane + o];
        s0 += l * gg;
        s1 += l * gg * r2;
    }
    atomicAdd(s, fa * s0);
    atomicAdd(s + 1, fw * s1);
}

// dL/dc_m = sum_p lw_p w_p cos(m pi zeta_p) / (1 + sum_m' c_m' cos(m' pi zeta_p)),
// the cos(m pi zeta) by the recurrence cos((m+1) t) = 2 cos t cos(m t) - cos((m-1) t)
// from one cosine per particle; block partial sums, one atomic per block and
// coefficient
__global__ void adj_profile_kernel(int64_t n, const double *lw, const void *w, int precision, const double *zeta,
                                   int M, const double *coef, double *out)
{
    double acc[16];
    for (int m = 0; m < 16; ++m) acc[m] = 0;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        if (lw[p] == 0.0) continue;  // never alive, or no current
        const double wp = precision ? ((const double *)w)[p] : (double)((const float *)w)[p];
        const double l = lw[p] * wp;
        double cm[16];
        const double c1 = cos(3.141592653589793 * zeta[p]);
        double prev = 1.0, cur = c1;
        double f = 1.0;
        for (int m = 1; m <= M; ++m) {
            cm[m - 1] = cur;
            f += coef[m - 1] * cur;
            const double next = 2.0 * c1 * cur - prev;
            prev = cur;
            cur = next;
        }
        const double lf = l / f;
        for (int m = 0; m < M; ++m) acc[m] += lf * cm[m];
    }
    __shared__ double red[256];
    for (int m = 0; m < M; ++m) {
        red[threadIdx.x] = acc[m];
        __syncthreads();
        for (int off = blockDim.x / 2; off > 0; off >>= 1) {
            if ((int)threadIdx.x < off) red[threadIdx.x] += red[threadIdx.x + off];
            __syncthreads();
        }
        if (threadIdx.x == 0) atomicAdd(out + m, red[0]);
        __syncthreads();
    }
}

// near[k] = 1 for every cell plane k within S + 2 planes of a z plane on which
// one of nc components (consecutive arrays of g.ncomp values) is not zero: a
// particle in cell k reads and deposits only within that reach, so a particle
// with near[k] = 0 sees zero there.
__device__ __forceinline__ void mark_near(const Geom &g, int k, unsigned char *near)
{
    const int R = g.shape + 2;
    for (int d = -R; d <= R; ++d) {
        int kk = k + d;
        if (g.bc_z == 0) kk = wrap1(kk, g.nz);
        else if (kk < 0 || kk > g.nz) continue;
        near[kk] = 1;
    }
}

// wide planes: one CTA reduces one plane at a time
template <typename real>
__global__ void adj_planes_kernel(Geom g, const real *F, int nc, unsigned char *near)
{
    const int nk = g.bc_z == 0 ? g.nz : g.nz + 1;
    for (int k = (int)blockIdx.x; k < nk; k += (int)gridDim.x) {
        int any = 0;
        for (int c = 0; c < nc; ++c) {
            const real *P = F + (int64_t)c * g.ncomp + (int64_t)k * g.plane;
            for (int64_t o = threadIdx.x; o < g.plane; o += blockDim.x) any |= P[o] != real(0);
        }
        if (__syncthreads_or(any) && threadIdx.x == 0) mark_near(g, k, near);
    }
}

// narrow planes (2D, small 3D sections): one warp per plane, every load of
// the plane issued before the vote
template <typename real>
__global__ void adj_planes_warp_kernel(Geom g, const real *F, int nc, unsigned char *near)
{
    const int nk = g.bc_z == 0 ? g.nz : g.nz + 1;
    const int lane = (int)(threadIdx.x & 31u), wpb = (int)(blockDim.x >> 5);
    // k is the same on all lanes of a warp, so every vote has all 32
    for (int k = (int)blockIdx.x * wpb + (int)(threadIdx.x >> 5); k < nk; k += (int)gridDim.x * wpb) {
        int any = 0;
        for (int c = 0; c < nc; ++c) {
            const real *P = F + (int64_t)c * g.ncomp + (int64_t)k * g.plane;
            for (int64_t o = lane; o < g.plane; o += 32) any |= P[o] != real(0);
        }
        if (__any_sync(0xffffffffu, any) && lane == 0) mark_near(g, k, near);
    }
}

template <typename real>
void launch_adj_planes(const Geom &g, const real *F, int nc, unsigned char *near, cudaStream_t s)
{
    cudaMemsetAsync(near, 0, (size_t)g.nz + 1, s);
    const int nk = g.nz + 1;
    const int cap = device_sms() * 16;
    if (g.plane <= 4096) {
        const int blocks = (nk + 7) / 8;
        adj_planes_warp_kernel<real><<<(unsigned)(blocks < cap ? blocks : cap), 256, 0, s>>>(g, F, nc, near);
    } else {
        adj_planes_kernel<real><<<(unsigned)(nk < cap ? nk : cap), 128, 0, s>>>(g, F, nc, near);
    }
}

// --------------------------------------------------------------- launchers

#define PIC_ADJ_LAUNCH(kernel)                                                                  \
    if (a.n <= 0) return;                                                                       \
    const unsigned grid = adj_grid(a.n, 256);                                                   \
    if (a.g.dim == 3) {                                                                         \
        if (a.g.shape == 1) kernel<real, 3, 1><<<grid, 256, 0, s>>>(a);                         \
        else kernel<real, 3, 2><<<grid, 256, 0, s>>>(a);                                        \
    } else {                                                                                    \
        if (a.g.shape == 1) kernel<real, 2, 1><<<grid, 256, 0, s>>>(a);                         \
        else kernel<real, 2, 2><<<grid, 256, 0, s>>>(a);                                        \
    }

template <typename real>
void launch_adj_push(const AdjArgs<real> &a, cudaStream_t s)
{
    PIC_ADJ_LAUNCH(adj_push_kernel)
}

template <typename real>
void launch_adj_push_vjp(const AdjArgs<real> &a, cudaStream_t s)
{
    PIC_ADJ_LAUNCH(adj_push_vjp_kernel)
}

#undef PIC_ADJ_LAUNCH

// the Yee step transposed: (lE, lB) at n+1 -> (lE, lB) at n and lJ (the
// cotangent of the filtered current); lE0 and pE are work components
template <typename real>
void launch_adj_yee(const Geom &g, real *lE[3], real *lB[3], real *lE0[3], real *pE[3], real *lJ[3], double dt,
                    double hx, double hy, double hz, cudaStream_t s)
{
    const unsigned grid = adj_grid((int64_t)(g.nz + 1) * g.plane, 256);
    const real h = (real)(0.5 * dt);
    // B^{n+1} = B' - h curl E^{n+1}
    adj_curl_e_t_kernel<real><<<grid, 256, 0, s>>>(g, lE[0], lE[1], lE[2], lB[0], lB[1], lB[2], (real)(h / hz),
                                                  (real)(h / hx), (real)(h / hy));
    // E^{n+1} = E^n + dt (curl B' - 2 pi J), Mur on the z ends
    adj_e_update_t_kernel<real><<<grid, 256, 0, s>>>(g, lE[0], lE[1], lE[2], pE[0], pE[1], pE[2], lE0[0], lE0[1],
                                                    lE0[2], lJ[0], lJ[1], lJ[2], (real)((dt - hz) / (dt + hz)),
                                                    (real)(-kTwoPiD * dt));
    adj_curl_b_t_kernel<real><<<grid, 256, 0, s>>>(g, pE[0], pE[1], pE[2], lB[0], lB[1], lB[2], (real)(dt / hz),
                                                  (real)(dt / hx), (real)(dt / hy));
    // B' = B^n - h curl E^n
    adj_curl_e_t_kernel<real><<<grid, 256, 0, s>>>(g, lE0[0], lE0[1], lE0[2], lB[0], lB[1], lB[2], (real)(h / hz),
                                                  (real)(h / hx), (real)(h / hy));
}

template <typename real>
void launch_adj_antenna(const Geom &g, const real *lJ, int pol, int ka, double hx, double hy, double xc, double yc,
                        double waist, double fa, double fw, double *s, cudaStream_t st)
{
    adj_antenna_kernel<real><<<adj_grid(g.plane, 256), 256, 0, st>>>(g, lJ, pol, ka, hx, hy, xc, yc,
                                                                      1.0 / (waist * waist), fa, fw, s);
}

void launch_adj_profile(int64_t n, const double *lw, const void *w, int precision, const double *zeta, int M,
                        const double *coef, double *out, cudaStream_t s)
{
    if (n > 0 && M > 0) adj_profile_kernel<<<adj_grid(n, 256), 256, 0, s>>>(n, lw, w, precision, zeta, M, coef, out);
}

#define PIC_ADJ_INSTANTIATE(real)                                                                              \
    template void launch_adj_push<real>(const AdjArgs<real> &, cudaStream_t);                                  \
    template void launch_adj_push_vjp<real>(const AdjArgs<real> &, cudaStream_t);                              \
    template void launch_adj_yee<real>(const Geom &, real *[3], real *[3], real *[3], real *[3], real *[3],     \
                                       double, double, double, double, cudaStream_t);                          \
    template void launch_adj_planes<real>(const Geom &, const real *, int, unsigned char *, cudaStream_t);     \
    template void launch_adj_antenna<real>(const Geom &, const real *, int, int, double, double, double, double, \
                                           double, double, double, double *, cudaStream_t);
PIC_ADJ_INSTANTIATE(float)
PIC_ADJ_INSTANTIATE(double)
#undef PIC_ADJ_INSTANTIATE

}  // namespace pic
