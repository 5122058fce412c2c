// pic_fields.cu -- field kernels: Yee leapfrog with Mur boundaries, binomial
// current filter, laser antenna and the FP64 field-energy reduction.
//
// Yee (1966) on the staggered lattice of pic_internal.cuh, B split in two half
// steps so that E and B both live at integer times:
//   B -= (dt/2) curl E;   E += dt (curl B - 2 pi J);   B -= (dt/2) curl E.
// With absorbing z the tangential E (Ex, Ey) on the end planes k = 0 and
// k = nz follows Mur's first-order condition (Mur 1981)
//   E0^{n+1} = E1^n + (dt - dz)/(dt + dz) (E1^{n+1} - E0^n)
// and the thread that updates plane 1 (nz-1) also updates plane 0 (nz), so no
// thread reads a value another thread of the same launch writes.
#include "pic_internal.cuh"

namespace pic {

template <typename real>
struct YeeArgs {
    Geom g;
    real *E[3], *B[3];
    const real *J[3];
    real h;             // time step of this update (dt/2 for B, dt for E)
    real ihx, ihy, ihz; // 1 / h_d
    real twopi;         // 2 pi
    real mur;           // (dt - hz) / (dt + hz)
};

template <typename real, int DIM>
__global__ void yee_b_kernel(YeeArgs<real> a)
{
    const Geom &g = a.g;
    const int64_t n = a.g.ncomp;
    for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < n; o += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(o % g.nx);
        const int j = (int)((o / g.nx) % g.ny);
        const int k = (int)(o / g.plane);
        const int ip = i + 1 == g.nx ? 0 : i + 1;
        const int jp = j + 1 == g.ny ? 0 : j + 1;
        const real *Ex = a.E[0], *Ey = a.E[1], *Ez = a.E[2];
        const bool per = g.bc_z == 0;
        if (k < g.nz) {
            const int kp = (per && k + 1 == g.nz) ? 0 : k + 1;
            const int64_t okp = fidx(g, i, j, kp);
            real dEz_dy = 0, dEx_dy = 0;
            if (DIM == 3) dEz_dy = (Ez[fidx(g, i, jp, k)] - Ez[o]) * a.ihy;
            const real dEy_dz = (Ey[okp] - Ey[o]) * a.ihz;
            a.B[0][o] -= a.h * (dEz_dy - dEy_dz);
            const real dEx_dz = (Ex[okp] - Ex[o]) * a.ihz;
            const real dEz_dx = (Ez[fidx(g, ip, j, k)] - Ez[o]) * a.ihx;
            a.B[1][o] -= a.h * (dEx_dz - dEz_dx);
            (void)dEx_dy;
        }
        if (k < g.nz || !per) {
            const real dEy_dx = (Ey[fidx(g, ip, j, k)] - Ey[o]) * a.ihx;
            real dEx_dy = 0;
            if (DIM == 3) dEx_dy = (Ex[fidx(g, i, jp, k)] - Ex[o]) * a.ihy;
            a.B[2][o] -= a.h * (dEy_dx - dEx_dy);
        }
    }
}

template <typename real, int DIM>
__device__ __forceinline__ void ampere_exy(const YeeArgs<real> &a, int i, int j, int k, int km, real &ex, real &ey)
{
    const Geom &g = a.g;
    const int im = i == 0 ? g.nx - 1 : i - 1;
    const int jm = j == 0 ? g.ny - 1 : j - 1;
    const int64_t o = fidx(g, i, j, k), okm = fidx(g, i, j, km);
    const real *Bx = a.B[0], *By = a.B[1], *Bz = a.B[2];
    real dBz_dy = 0;
    if (DIM == 3) dBz_dy = (Bz[o] - Bz[fidx(g, i, jm, k)]) * a.ihy;
    const real dBy_dz = (By[o] - By[okm]) * a.ihz;
    ex = a.E[0][o] + a.h * ((dBz_dy - dBy_dz) - a.twopi * a.J[0][o]);
    const real dBx_dz = (Bx[o] - Bx[okm]) * a.ihz;
    const real dBz_dx = (Bz[o] - Bz[fidx(g, im, j, k)]) * a.ihx;
    ey = a.E[1][o] + a.h * ((dBx_dz - dBz_dx) - a.twopi * a.J[1][o]);
}

template <typename real, int DIM>
__global__ void yee_e_kernel(YeeArgs<real> a)
{
    const Geom &g = a.g;
    const int64_t n = a.g.ncomp;
    const bool per = g.bc_z == 0;
    for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < n; o += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(o % g.nx);
        const int j = (int)((o / g.nx) % g.ny);
        const int k = (int)(o / g.plane);
        const int im = i == 0 ? g.nx - 1 : i - 1;
        const int jm = j == 0 ? g.ny - 1 : j - 1;
        if (k < g.nz) {
            const real *Bx = a.B[0], *By = a.B[1];
            const real dBy_dx = (By[o] - By[fidx(g, im, j, k)]) * a.ihx;
            real dBx_dy = 0;
            if (DIM == 3) dBx_dy = (Bx[o] - Bx[fidx(g, i, jm, k)]) * a.ihy;
            a.E[2][o] += a.h * ((dBy_dx - dBx_dy) - a.twopi * a.J[2][o]);
        }
        if (per) {
            if (k < g.nz) {
                real ex, ey;
                ampere_exy<real, DIM>(a, i, j, k, k == 0 ? g.nz - 1 : k - 1, ex, ey);
                a.E[0][o] = ex;
                a.E[1][o] = ey;
            }
        } else if (k >= 1 && k <= g.nz - 1) {
            real ex, ey;
            ampere_exy<real, DIM>(a, i, j, k, k - 1, ex, ey);
            if (k == 1) {  // this thread also owns plane 0
                const int64_t o0 = fidx(g, i, j, 0);
                const real ex1 = a.E[0][o], ey1 = a.E[1][o];
                const real ex0 = a.E[0][o0], ey0 = a.E[1][o0];
                a.E[0][o0] = ex1 + a.mur * (ex - ex0);
                a.E[1][o0] = ey1 + a.mur * (ey - ey0);
            }
            if (k == g.nz - 1) {  // and plane nz
                const int64_t on = fidx(g, i, j, g.nz);
                const real exm = a.E[0][o], eym = a.E[1][o];
                const real exn = a.E[0][on], eyn = a.E[1][on];
                a.E[0][on] = exm + a.mur * (ex - exn);
                a.E[1][on] = eym + a.mur * (ey - eyn);
            }
            a.E[0][o] = ex;
            a.E[1][o] = ey;
        }
    }
}

static unsigned grid_for(int64_t n, int block)
{
    int64_t b = (n + block - 1) / block;
    const int64_t cap = 152LL * 32;
    return (unsigned)(b < cap ? (b > 0 ? b : 1) : cap);
}

template <typename real>
void launch_yee(const Geom &g, real *const F[9], double dt, double hx, double hy, double hz, cudaStream_t s)
{
    YeeArgs<real> a;
    a.g = g;
    for (int c = 0; c < 3; ++c) {
        a.E[c] = F[c];
        a.B[c] = F[3 + c];
        a.J[c] = F[6 + c];
    }
    a.ihx = (real)(1.0 / hx);
    a.ihy = (real)(1.0 / hy);
    a.ihz = (real)(1.0 / hz);
    a.twopi = (real)6.283185307179586;
    a.mur = (real)((dt - hz) / (dt + hz));
    const unsigned grid = grid_for(g.ncomp, 256);
    a.h = (real)(0.5 * dt);
    if (g.dim == 3) yee_b_kernel<real, 3><<<grid, 256, 0, s>>>(a);
    else yee_b_kernel<real, 2><<<grid, 256, 0, s>>>(a);
    a.h = (real)dt;
    if (g.dim == 3) yee_e_kernel<real, 3><<<grid, 256, 0, s>>>(a);
    else yee_e_kernel<real, 2><<<grid, 256, 0, s>>>(a);
    a.h = (real)(0.5 * dt);
    if (g.dim == 3) yee_b_kernel<real, 3><<<grid, 256, 0, s>>>(a);
    else yee_b_kernel<real, 2><<<grid, 256, 0, s>>>(a);
}

// ---------------------------------------------------------------- filter

// One (1/4, 1/2, 1/4) pass of Jx, Jy, Jz along `axis` from `in` to `out`.
// Periodic axes wrap; with absorbing z the values outside a component's valid
// z range are zero (and the unused plane nz of Jz stays zero).
template <typename real>
__global__ void filter_kernel(Geom g, const real *in0, const real *in1, const real *in2, real *out0,
                              real *out1, real *out2, int axis)
{
    const int64_t n = g.ncomp;
    for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < 3 * n; o += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(o / n);
        const int64_t r = o - c * n;
        const real *in = c == 0 ? in0 : (c == 1 ? in1 : in2);
        real *out = c == 0 ? out0 : (c == 1 ? out1 : out2);
        const int i = (int)(r % g.nx);
        const int j = (int)((r / g.nx) % g.ny);
        const int k = (int)(r / g.plane);
        const int zmax = zmax_of(g, c == 2);
        if (k > zmax) {
            out[r] = 0;
            continue;
        }
        real lo, hi;
        if (axis == 0) {
            lo = in[fidx(g, i == 0 ? g.nx - 1 : i - 1, j, k)];
            hi = in[fidx(g, i + 1 == g.nx ? 0 : i + 1, j, k)];
        } else if (axis == 1) {
            lo = in[fidx(g, i, j == 0 ? g.ny - 1 : j - 1, k)];
            hi = in[fidx(g, i, j + 1 == g.ny ? 0 : j + 1, k)];
        } else if (g.bc_z == 0) {
            lo = in[fidx(g, i, j, k == 0 ? g.nz - 1 : k - 1)];
            hi = in[fidx(g, i, j, k + 1 == g.nz ? 0 : k + 1)];
        } else {
            lo = k > 0 ? in[fidx(g, i, j, k - 1)] : real(0);
            hi = k < zmax ? in[fidx(g, i, j, k + 1)] : real(0);
        }
        out[r] = real(0.25) * lo + real(0.5) * in[r] + real(0.25) * hi;
    }
}

// All passes of all axes in one kernel.  A CTA owns blocks of one component:
// BX = 32 - 2H nodes along x (plus a halo of H = npass per side), 8 rows in
// y (3D: BY = 8 consecutive y plus the halo; 2D: 8 independent x sub-blocks
// side by side), BZ along z plus the halo.  x passes: one warp per row, a lane
// per x node, neighbours by warp shuffle, all H passes in registers.  y and z
// passes: a thread per column holds the column in registers.  The arithmetic
// per pass and node is the one of filter_kernel, in the same order (x, then y,
// then z); with absorbing z, nodes outside the component's valid z range are
// zero before every z pass, as filter_kernel treats them.
template <typename real, int DIM, int BZ, int H>
__global__ void __launch_bounds__(256) filter_fused_kernel(Geom g, const real *in0, const real *in1, const real *in2,
                                                           real *out0, real *out1, real *out2)
{
    constexpr int AX = 32, BX = AX - 2 * H;
    constexpr int BY = 8;                                   // y rows (3D) or x sub-blocks (2D)
    constexpr int AY = DIM == 3 ? BY + 2 * H : BY, AZ = BZ + 2 * H;
    constexpr int HY = DIM == 3 ? H : 0;
    constexpr int SPAN = DIM == 3 ? BX : BY * BX;           // x nodes of one CTA's centre
    extern __shared__ __align__(16) unsigned char smem_raw[];
    real *A = reinterpret_cast<real *>(smem_raw);  // [AZ][AY][AX]
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int c = blockIdx.z;
    const real *in = c == 0 ? in0 : (c == 1 ? in1 : in2);
    real *out = c == 0 ? out0 : (c == 1 ? out1 : out2);
    const int zmax = zmax_of(g, c == 2);
    const int nbx = (g.nx + SPAN - 1) / SPAN;
    const int bxi = blockIdx.x % nbx, byi = blockIdx.x / nbx;
    const int x0 = bxi * SPAN, y0 = DIM == 3 ? byi * BY : 0, oz = blockIdx.y * BZ - H;

    // load + x passes: warp per row
    for (int row = warp; row < AY * AZ; row += 8) {
        const int ly = row % AY, lz = row / AY;
        const int gi = wrapi(x0 + (DIM == 3 ? 0 : ly * BX) - H + lane, g.nx);
        const int gj = DIM == 3 ? wrapi(y0 - H + ly, g.ny) : 0;
        const int gk = oz + lz;
        real v = 0;
        if (g.bc_z == 0) v = in[fidx(g, gi, gj, wrapi(gk, g.nz))];
        else if (gk >= 0 && gk <= zmax) v = in[fidx(g, gi, gj, gk)];
#pragma unroll
        for (int p = 0; p < H; ++p) {
            const real lo = __shfl_up_sync(0xffffffffu, v, 1), hi = __shfl_down_sync(0xffffffffu, v, 1);
            if (lane != 0 && lane != 31) v = real(0.25) * lo + real(0.5) * v + real(0.25) * hi;
        }
        A[row * AX + lane] = v;
    }
    __syncthreads();

    // y passes (3D): thread per (x, z) column
    if (DIM == 3) {
        for (int col = threadIdx.x; col < AX * AZ; col += 256) {
            const int lx = col % AX, lz = col / AX;
            real v[AY];
#pragma unroll
            for (int l = 0; l < AY; ++l) v[l] = A[(lz * AY + l) * AX + lx];
#pragma unroll
            for (int p = 0; p < H; ++p) {
                real prev = v[0];
#pragma unroll
                for (int l = 1; l < AY - 1; ++l) {
                    const real cur = v[l];
                    v[l] = real(0.25) * prev + real(0.5) * cur + real(0.25) * v[l + 1];
                    prev = cur;
                }
            }
#pragma unroll
            for (int l = 0; l < AY; ++l) A[(lz * AY + l) * AX + lx] = v[l];
        }
        __syncthreads();
    }

    // z passes and the write of the block centre: thread per (x, row) column
    for (int col = threadIdx.x; col < BX * BY; col += 256) {
        const int lx = col % BX + H, ly = col / BX + HY;
        const int gx = DIM == 3 ? x0 + lx - H : x0 + (ly * BX) + lx - H;
        const int gy = DIM == 3 ? y0 + ly - H : 0;
        real v[AZ];
#pragma unroll
        for (int l = 0; l < AZ; ++l) v[l] = A[(l * AY + ly) * AX + lx];
#pragma unroll
        for (int p = 0; p < H; ++p) {
            real prev = v[0];
#pragma unroll
            for (int l = 1; l < AZ - 1; ++l) {
                const real cur = v[l];
                real nv = real(0.25) * prev + real(0.5) * cur + real(0.25) * v[l + 1];
                if (g.bc_z != 0) {
                    const int gk = oz + l;
                    if (gk < 0 || gk > zmax) nv = 0;
                }
                v[l] = nv;
                prev = cur;
            }
        }
        if (gx >= g.nx || gy >= g.ny) continue;
#pragma unroll
        for (int l = H; l < H + BZ; ++l) {
            const int gk = oz + l;
            if (gk <= g.nz) out[fidx(g, gx, gy, gk)] = gk > zmax ? real(0) : v[l];
        }
    }
}

template <typename real, int DIM, int BZ, int H>
static void launch_fused(const Geom &g, real *const J[3], real *tmp, cudaStream_t s)
{
    constexpr int BX = 32 - 2 * H, BY = 8;
    constexpr int SPAN = DIM == 3 ? BX : BY * BX;
    constexpr int AN = 32 * (DIM == 3 ? BY + 2 * H : BY) * (BZ + 2 * H);
    const size_t smem = sizeof(real) * AN;
    auto k = filter_fused_kernel<real, DIM, BZ, H>;
    if (smem > 48 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const unsigned nbx = (g.nx + SPAN - 1) / SPAN, nby = DIM == 3 ? (g.ny + BY - 1) / BY : 1;
    dim3 grid(nbx * nby, (g.nz + 1 + BZ - 1) / BZ, 3);
    k<<<grid, 256, smem, s>>>(g, J[0], J[1], J[2], tmp, tmp + g.ncomp, tmp + 2 * g.ncomp);
    cudaMemcpyAsync(J[0], tmp, 3 * sizeof(real) * g.ncomp, cudaMemcpyDeviceToDevice, s);
}

template <typename real>
void launch_filter(const Geom &g, real *const J[3], real *tmp, int npass, cudaStream_t s)
{
    if (npass <= 0) return;
    // the three components are contiguous in the field buffer; the fused
    // kernel covers 1..4 passes, more fall back to one launch per pass
    const bool contiguous = J[1] == J[0] + g.ncomp && J[2] == J[1] + g.ncomp;
    if (contiguous && npass <= 4) {
        if (g.dim == 3) {
            switch (npass) {
            case 1: launch_fused<real, 3, 16, 1>(g, J, tmp, s); return;
            case 2: launch_fused<real, 3, 16, 2>(g, J, tmp, s); return;
            case 3: launch_fused<real, 3, 16, 3>(g, J, tmp, s); return;
            default: launch_fused<real, 3, 16, 4>(g, J, tmp, s); return;
            }
        } else {
            switch (npass) {
            case 1: launch_fused<real, 2, 32, 1>(g, J, tmp, s); return;
            case 2: launch_fused<real, 2, 32, 2>(g, J, tmp, s); return;
            case 3: launch_fused<real, 2, 32, 3>(g, J, tmp, s); return;
            default: launch_fused<real, 2, 32, 4>(g, J, tmp, s); return;
            }
        }
    }
    real *src[3] = {J[0], J[1], J[2]};
    real *dst[3] = {tmp, tmp + g.ncomp, tmp + 2 * g.ncomp};
    const unsigned grid = grid_for(3 * g.ncomp, 256);
    int passes = 0;
    for (int axis = 0; axis < 3; ++axis) {
        if (axis == 1 && g.dim != 3) continue;
        for (int p = 0; p < npass; ++p) {
            filter_kernel<real><<<grid, 256, 0, s>>>(g, src[0], src[1], src[2], dst[0], dst[1], dst[2], axis);
            for (int c = 0; c < 3; ++c) {
                real *t = src[c];
                src[c] = dst[c];
                dst[c] = t;
            }
            ++passes;
        }
    }
    if (passes & 1)
        for (int c = 0; c < 3; ++c)
            cudaMemcpyAsync(J[c], src[c], sizeof(real) * g.ncomp, cudaMemcpyDeviceToDevice, s);
}

// ---------------------------------------------------------------- antenna

// Current sheet on plane ka: J_pol += j0 exp(-r^2 / w0^2) at each node of the
// polarisation component (its own staggered transverse position).  One plane
// per step: the profile is evaluated in FP64 and rounded once.
template <typename real>
__global__ void antenna_kernel(Geom g, real *J, int pol, int ka, double j0, double hx, double hy, double xc,
                               double yc, double inv_w2)
{
    const int64_t n = g.plane;
    for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < n; o += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(o % g.nx), j = (int)(o / g.nx);
        const double x = ((double)i + (pol == 0 ? 0.5 : 0.0)) * hx - xc;
        double r2 = x * x;
        if (g.dim == 3) {
            const double y = ((double)j + (pol == 1 ? 0.5 : 0.0)) * hy - yc;
            r2 += y * y;
        }
        J[(int64_t)ka * g.plane + o] += (real)(j0 * exp(-r2 * inv_w2));
    }
}

template <typename real>
void launch_antenna(const Geom &g, real *J, int pol, int ka, double j0, double hx, double hy, double xc,
                    double yc, double waist, cudaStream_t s)
{
    antenna_kernel<real><<<grid_for(g.plane, 256), 256, 0, s>>>(g, J, pol, ka, j0, hx, hy, xc, yc,
                                                               1.0 / (waist * waist));
}

// ------------------------------------------------------------ field sums

// Kahan-compensated FP64 partials of sum (E^2 + B^2) over the valid nodes of
// each component; the host multiplies by V/2 and adds the partials.
template <typename real>
__global__ void field_sums_kernel(Geom g, const real *F0, const real *F1, const real *F2, const real *F3,
                                  const real *F4, const real *F5, double *partials)
{
    double s = 0, c = 0;
    const int64_t n = g.ncomp;
    for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < 6 * n; o += (int64_t)gridDim.x * blockDim.x) {
        const int comp = (int)(o / n);
        const int64_t r = o - comp * n;
        const int k = (int)(r / g.plane);
        const bool halfz = comp == 2 || comp == 3 || comp == 4;
        if (k > zmax_of(g, halfz)) continue;
        const real *F = comp == 0 ? F0 : comp == 1 ? F1 : comp == 2 ? F2 : comp == 3 ? F3 : comp == 4 ? F4 : F5;
        const double v = (double)F[r];
        const double y = v * v - c;
        const double t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __shared__ double red[256];
    red[threadIdx.x] = s - c;
    __syncthreads();
    for (int off = blockDim.x / 2; off > 0; off >>= 1) {
        if ((int)threadIdx.x < off) red[threadIdx.x] += red[threadIdx.x + off];
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[blockIdx.x] = red[0];
}

template <typename real>
void launch_field_sums(const Geom &g, real *const F[9], double *partials, int nblocks, cudaStream_t s)
{
    field_sums_kernel<real><<<nblocks, 256, 0, s>>>(g, F[0], F[1], F[2], F[3], F[4], F[5], partials);
}

#define PIC_FIELDS_INSTANTIATE(real)                                                                    \
    template void launch_yee<real>(const Geom &, real *const[9], double, double, double, double,       \
                                   cudaStream_t);                                                       \
    template void launch_filter<real>(const Geom &, real *const[3], real *, int, cudaStream_t);         \
    template void launch_antenna<real>(const Geom &, real *, int, int, double, double, double, double,  \
                                       double, double, cudaStream_t);                                   \
    template void launch_field_sums<real>(const Geom &, real *const[9], double *, int, cudaStream_t);
PIC_FIELDS_INSTANTIATE(float)
PIC_FIELDS_INSTANTIATE(double)

}  // namespace pic
