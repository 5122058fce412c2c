// pic_btd.cu -- lab-frame ("back-transformed") snapshots of a boosted run.
//
// After the Yee update of step n both (E^n, B^n) and (E^{n+1}, B^{n+1}) are
// in memory (the two field buffers).  Every lab snapshot point (T_j, Z_k)
// whose simulation-frame event time t' = gamma (T - beta Z) lies in
// [t'^n, t'^{n+1}) is filled now: the fields at z' = gamma (Z - beta T),
// linear in z' between the planes of each component and linear in t' between
// the two times, transformed to the lab frame (the simulation frame moves at
// +beta along z):
//   Ex = gamma (Ex' + beta By'),  Ey = gamma (Ey' - beta Bx'),  Ez = Ez',
//   Bx = gamma (Bx' - beta Ey'),  By = gamma (By' + beta Ex'),  Bz = Bz'.
// Event times, heights and weights are FP64 and this file is compiled without
// FMA contraction, so which points a step fills is decided exactly as the
// FP64 reference decides it.
#include "pic_internal.cuh"

namespace pic {

template <typename real>
__global__ void btd_kernel(BtdArgs<real> a)
{
    const int js = (int)blockIdx.y;
    const int idx = (int)(blockIdx.x * blockDim.x + threadIdx.x);
    const int kk = idx / a.nxs, is = idx - kk * a.nxs;
    if (kk >= a.kn[js]) return;
    const int k = a.klo[js] + kk;
    const Geom &g = a.g;
    const double T = a.T0 + js * a.dT;
    const double Z = a.Z0 + k * a.dZ;
    const double tp = a.gam * (T - a.beta * Z);
    if (!(tp >= a.t0 && tp < a.t0 + a.dt)) return;
    const double zp = a.gam * (Z - a.beta * T) - a.zwin;
    const double th = (tp - a.t0) / a.dt;
    const int i = a.nxs == 1 ? g.nx / 2 : is;
    const int jc = g.ny / 2;
    real v[6];
    for (int c = 0; c < 6; ++c) {
        // Ez, Bx, By sit half a cell up in z
        const double sz = (c == 2 || c == 3 || c == 4) ? 0.5 : 0.0;
        const double u = zp / a.hz - sz;
        const double k0 = floor(u);
        const double fz = u - k0;
        const int zmax = g.bc_z == 0 ? g.nz - 1 : (sz > 0.0 ? g.nz - 1 : g.nz);
        if (k0 < 0.0 || k0 + 1.0 > (double)zmax) return;  // the same for every column
        const int64_t o0 = fidx(g, i, jc, (int)k0), o1 = o0 + g.plane;
        const real *F0 = c < 3 ? a.E0[c] : a.B0[c - 3];
        const real *F1 = c < 3 ? a.E1[c] : a.B1[c - 3];
        const real w0 = (real)(1.0 - fz), w1 = (real)fz;
        const real f0 = w0 * F0[o0] + w1 * F0[o1];
        const real f1 = w0 * F1[o0] + w1 * F1[o1];
        v[c] = (real)(1.0 - th) * f0 + (real)th * f1;
    }
    const real gam = (real)a.gam, beta = (real)a.beta;
    const real lab[6] = {gam * (v[0] + beta * v[4]), gam * (v[1] - beta * v[3]), v[2],
                         gam * (v[3] - beta * v[1]), gam * (v[4] + beta * v[0]), v[5]};
    real *d = a.data + (size_t)js * 6 * a.nz * a.nxs;
    for (int c = 0; c < 6; ++c) d[((size_t)c * a.nz + k) * a.nxs + is] = lab[c];
    if (is == 0) a.flags[(size_t)js * a.nz + k] = 1;
}

template <typename real>
void launch_btd(const BtdArgs<real> &a, cudaStream_t s)
{
    int span = 0;
    for (int j = 0; j < a.nsnap; ++j) span = a.kn[j] > span ? a.kn[j] : span;
    if (span == 0) return;
    const int64_t n = (int64_t)span * a.nxs;
    dim3 grid((unsigned)((n + 255) / 256), (unsigned)a.nsnap);
    btd_kernel<real><<<grid, 256, 0, s>>>(a);
}

template void launch_btd<float>(const BtdArgs<float> &, cudaStream_t);
template void launch_btd<double>(const BtdArgs<double> &, cudaStream_t);

// ----------------------------------------------- lab-frame view of the grid

// partner component c at the height of a component of the other z
// staggering: the mean of its planes k - 1, k (up = 0: the component is on
// integer z, the partner on half-integer z) or k, k + 1 (up = 1); the nearer
// plane alone at an absorbing end, planes wrap when z is periodic
template <typename real>
__device__ __forceinline__ double zmean(const Geom &g, const real *P, int i, int j, int k, int up, int km)
{
    int a = up ? k : k - 1, b = up ? k + 1 : k;
    if (g.bc_z == 0) {
        a = wrapi(a, g.nz);
        b = wrapi(b, g.nz);
    } else {
        if (a < 0) a = b;
        if (b > km) b = a;
        if (a > km) a = b = km;
    }
    return 0.5 * ((double)P[fidx(g, i, j, a)] + (double)P[fidx(g, i, j, b)]);
}

// Component comp (0..5: Ex Ey Ez Bx By Bz) of the lab-frame fields on the
// simulation grid at the current time, each at its own Yee position, by the
// inverse field transformation (FP64): F the component, P the partner it
// mixes with (By for Ex, Bx for Ey, Ey for Bx, Ex for By); nodes beyond the
// component's z range are zero.
template <typename real>
__global__ void lab_fields_kernel(Geom g, const real *F, const real *P, int comp, real *out, double gam,
                                  double beta)
{
    const bool half = comp == 2 || comp == 3 || comp == 4;
    const int km = zmax_of(g, half);
    const int kmp = zmax_of(g, !half);  // the partner's range
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < g.ncomp; r += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(r % g.nx);
        const int j = (int)((r / g.nx) % g.ny);
        const int k = (int)(r / g.plane);
        double v = 0.0;
        if (k <= km) {
            const double f = (double)F[r];
            switch (comp) {
            case 0: v = gam * (f + beta * zmean(g, P, i, j, k, 0, kmp)); break;
            case 1: v = gam * (f - beta * zmean(g, P, i, j, k, 0, kmp)); break;
            case 3: v = gam * (f - beta * zmean(g, P, i, j, k, 1, kmp)); break;
            case 4: v = gam * (f + beta * zmean(g, P, i, j, k, 1, kmp)); break;
            default: v = f; break;
            }
        }
        out[r] = (real)v;
    }
}

template <typename real>
void launch_lab_fields(const Geom &g, const real *F, const real *P, int comp, real *out, double gam, double beta,
                       int sms, cudaStream_t s)
{
    int64_t blocks = (g.ncomp + 255) / 256;
    if (blocks > 8LL * sms) blocks = 8LL * sms;
    lab_fields_kernel<real><<<(unsigned)blocks, 256, 0, s>>>(g, F, P, comp, out, gam, beta);
}

template void launch_lab_fields<float>(const Geom &, const float *, const float *, int, float *, double, double, int,
                                       cudaStream_t);
template void launch_lab_fields<double>(const Geom &, const double *, const double *, int, double *, double, double,
                                        int, cudaStream_t);

}  // namespace pic
