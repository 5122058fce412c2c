// pic_inject.cu -- plasma loading and boosted-frame injection (FP64).
//
// A plasma at rest in the lab sits on a lattice of ppc points per cell and
// axis with a seeded uniform jitter; in a frame boosted by gamma it is seen at
// z' = z_lab / gamma - beta t' (the Lorentz transform, the paper's "hyperbolic
// rotation"), with density gamma n and drift u_z = -gamma beta.  One thread
// handles one lattice point: it recomputes the point's lab position from its
// index (SplitMix64 jitter, counter 3 * id + axis), and either places it if it
// lies in the box at time t (load) or appends it if it crosses z = Lz during
// (t, t1] (injection), at its position at t1.  No list of pending plasma is
// kept.
//
// This file is compiled without floating-point contraction so that every
// double operation rounds once, in the order written: the decision "in the
// box" / "crosses now" is then the same as in any other IEEE implementation
// of the same expressions.
#include "pic_internal.cuh"

namespace pic {

__device__ __forceinline__ uint64_t splitmix64(uint64_t seed, uint64_t counter)
{
    uint64_t z = seed + (counter + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ double uniform01(uint64_t seed, uint64_t counter)
{
    return (double)(splitmix64(seed, counter) >> 11) * (1.0 / 9007199254740992.0);
}

// lab-frame density: linear up-ramp, then the cosine-series profile
__device__ double lab_density(const InjectArgs &a, double z)
{
    if (z < a.z_start || z >= a.z_end) return 0.0;
    double r = 1.0;
    if (a.ramp > 0.0 && z < a.z_start + a.ramp) r = (z - a.z_start) / a.ramp;
    double f = 1.0;
    if (a.nprof > 0) {
        // cos(m pi zeta) by the recurrence cos(m t) = 2 cos t cos((m-1) t) -
        // cos((m-2) t): one cosine per point (FP64 is the slow pipe here)
        const double zeta = (z - a.z_start) / (a.z_end - a.z_start);
        const double c1 = cos(3.141592653589793 * zeta);
        double cp = 1.0, cm = c1;
        f += a.prof[0] * c1;
        for (int m = 2; m <= a.nprof; ++m) {
            const double cn = 2.0 * c1 * cm - cp;
            f += a.prof[m - 1] * cn;
            cp = cm;
            cm = cn;
        }
    }
    return a.ne * r * f;
}

// position (one axis) -> cell and offset in [0,1) of the working precision
template <typename real>
__device__ __forceinline__ void to_cell(double x, double h, int n, bool periodic, int &c, real &off)
{
    const double xi = x / h;
    double f = floor(xi);
    c = (int)f;
    double o = xi - f;
    if (c >= n) {  // x just below the box end rounded up
        if (periodic) { c -= n; } else { c = n - 1; o = (double)below_one<real>(); }
    }
    off = (real)o;
    if (off >= real(1)) {
        if (c + 1 < n) { c += 1; off = 0; }
        else if (periodic) { c = 0; off = 0; }
        else off = below_one<real>();
    }
}

template <typename real>
__device__ __forceinline__ void store(void *const sp[kAttrs], int64_t d, real ox, real oy, real oz, real w, int32_t cell,
                                      int64_t id, bool electron, bool dim3)
{
    static_cast<real *>(sp[0])[d] = ox;
    if (dim3) static_cast<real *>(sp[1])[d] = oy;
    static_cast<real *>(sp[2])[d] = oz;
    static_cast<real *>(sp[3])[d] = w;
    if (electron) {  // momenta relative to the drift: the cold plasma has none
        static_cast<real *>(sp[4])[d] = real(0);
        static_cast<real *>(sp[5])[d] = real(0);
        static_cast<real *>(sp[6])[d] = real(0);
    }
    static_cast<int32_t *>(sp[7])[d] = cell;
    if (sp[8]) static_cast<int64_t *>(sp[8])[d] = id;
    if (electron) {  // relative form: on its reference
        for (int q = 9; q < kAttrs; ++q)
            if (sp[q]) static_cast<real *>(sp[q])[d] = real(0);
    }
}

template <typename real>
__device__ __forceinline__ void inject_body(const InjectArgs &a, const int64_t b, const int64_t nb)
{
    const bool dim3 = a.g.dim == 3;
    // the step's times and lattice band (from device memory in a captured step)
    const double t = a.scal ? a.scal->t : a.t, t1 = a.scal ? a.scal->t1 : a.t1;
    const int64_t m_lo = a.scal ? a.scal->m_lo : a.m_lo, m_hi = a.scal ? a.scal->m_hi : a.m_hi;
    const int64_t total = (m_hi - m_lo) * a.NY * a.NX;
    const int64_t nround = (total + 31) / 32 * 32;
    const int64_t stride = nb * blockDim.x;
    for (int64_t q = b * blockDim.x + threadIdx.x; q < nround; q += stride) {
        int64_t dest = -1;
        int ci = 0, cj = 0, ck = 0;
        real ox = 0, oy = 0, oz = 0, wr = 0;
        int64_t L = 0;
        double zeta = 0.0;
        if (q < total) {
            const int64_t ix = q % a.NX;
            const int64_t r = q / a.NX;
            const int64_t iy = r % a.NY;
            const int64_t m = m_lo + r / a.NY;
            L = (m * a.NY + iy) * a.NX + ix;
            const uint64_t c0 = 3ull * (uint64_t)L;
            double x = ((double)ix + 0.5) * (a.hx / (double)a.ppx) +
                       (a.jitter * a.hx) * (2.0 * uniform01(a.seed, c0) - 1.0);
            if (x < 0.0) x += a.Lx;
            if (x >= a.Lx) x -= a.Lx;
            double y = 0.0;
            if (dim3) {
                y = ((double)iy + 0.5) * (a.hy / (double)a.ppy) +
                    (a.jitter * a.hy) * (2.0 * uniform01(a.seed, c0 + 1ull) - 1.0);
                if (y < 0.0) y += a.Ly;
                if (y >= a.Ly) y -= a.Ly;
            }
            const double zlab = a.z_start + ((double)m + 0.5) * a.dzl +
                                (a.jitter * a.hz_lab) * (2.0 * uniform01(a.seed, c0 + 2ull) - 1.0);
            zeta = (zlab - a.z_start) / (a.z_end - a.z_start);
            const double n = lab_density(a, zlab);
            if (n > 0.0) {
                bool take;
                double zb;
                // simulation-frame positions relative to the (moving) window
                if (a.mode == 0) {
                    zb = zlab / a.gam - a.beta * t - a.zwin;
                    take = zb >= a.zmin && zb < a.Lz;
                } else {
                    const double zb0 = zlab / a.gam - a.beta * t - a.zwin;
                    zb = zlab / a.gam - a.beta * t1 - a.zwin;
                    take = zb0 >= a.Lz && zb < a.Lz;
                }
                if (take) {
                    to_cell<real>(x, a.hx, a.g.nx, true, ci, ox);
                    if (dim3) to_cell<real>(y, a.hy, a.g.ny, true, cj, oy);
                    to_cell<real>(zb, a.hz, a.g.nz, a.g.bc_z == 0, ck, oz);
                    wr = (real)(n * a.wfac);
                    dest = tile_of(a.g, ci, cj, ck);
                }
            }
        }
        if (a.flat_base >= 0) {  // the fixed-order store of an adjoint run
            if (q < total) {
                const int64_t sl = a.flat_base + q;
                const bool in = dest >= 0;
                a.fe_alive[sl] = in ? 1 : 0;
                a.fi_alive[sl] = (in && a.drift_ions) ? 1 : 0;
                if (in) {
                    a.fe_ci[sl] = ci;
                    a.fe_ck[sl] = ck;
                    if (dim3) {
                        a.fe_cj[sl] = cj;
                        static_cast<real *>(a.fe_oy)[sl] = oy;
                        a.f_ion_cj[sl] = cj;
                        static_cast<real *>(a.f_ion_oy)[sl] = oy;
                    }
                    static_cast<real *>(a.fe_ox)[sl] = ox;
                    static_cast<real *>(a.fe_oz)[sl] = oz;
                    static_cast<real *>(a.fe_ux)[sl] = real(0);
                    static_cast<real *>(a.fe_uy)[sl] = real(0);
                    static_cast<real *>(a.fe_uz)[sl] = real(0);
                    a.fi_ck[sl] = ck;
                    static_cast<real *>(a.fi_oz)[sl] = oz;
                    a.f_ion_ci[sl] = ci;
                    static_cast<real *>(a.f_ion_ox)[sl] = ox;
                    static_cast<real *>(a.f_w)[sl] = wr;
                    a.f_zeta[sl] = zeta;
                }
            }
            continue;
        }
        // appended to the top run of the destination bucket
        const int re = reserve_slot(a.hi_e, dest);
        int ri = 0;
        if (a.drift_ions && !a.paired) ri = reserve_slot(a.hi_i, dest);
        if (dest < 0) continue;
        // every reserved slot below the capacity is written, so a bucket never
        // holds a stale entry; an overflow drops the particle and is reported.
        // With drifting ions the electron is placed paired with its ion (one
        // record for both until a field reaches them).
        const int32_t cell = pack_cell(a.g, ci, cj, ck);
        const int32_t ecell = (int32_t)((uint32_t)cell | (a.paired ? kPaired : 0u));
        if (re < a.g.cap)
            store<real>(a.sp_e, dest * (int64_t)a.g.cap + (a.g.cap - 1 - re), ox, oy, oz, wr, ecell, L, true, dim3);
        else atomicOr(a.err, ERR_CAPACITY);
        if (a.drift_ions && !a.paired) {
            if (ri < a.g.cap)
                store<real>(a.sp_i, dest * (int64_t)a.g.cap + (a.g.cap - 1 - ri), ox, oy, oz, wr, cell, L, false,
                            dim3);
            else atomicOr(a.err, ERR_CAPACITY);
        }
    }
}

template <typename real>
__global__ void inject_kernel(InjectArgs a)
{
    inject_body<real>(a, (int64_t)blockIdx.x, (int64_t)gridDim.x);
}

template <typename real>
__global__ void inject_batch_kernel(const InjectArgs *__restrict__ runs, const int64_t *__restrict__ start, int n)
{
    __shared__ __align__(16) InjectArgs sa;
    const int64_t b = batch_block(runs, start, n, &sa);
    const int r = batch_run_of(start, n, (int64_t)blockIdx.x);
    inject_body<real>(sa, b, start[r + 1] - start[r]);
}

// the work per point is FP64 arithmetic, whose pipe is narrow: CTAs of two
// warps spread a step's thin band of lattice points over many SMs
constexpr int kInjectThreads = 64;

template <typename real>
static void launch_inject_batch(const void *args, const int64_t *start, int n, int64_t total, unsigned *,
                                cudaStream_t s)
{
    inject_batch_kernel<real>
        <<<(unsigned)total, kInjectThreads, 0, s>>>(static_cast<const InjectArgs *>(args), start, n);
}

void launch_inject(const InjectArgs &a, cudaStream_t s)
{
    const int64_t total = (a.m_hi - a.m_lo) * a.NY * a.NX;
    if (total <= 0) return;
    int64_t blocks = (total + kInjectThreads - 1) / kInjectThreads;
    if (blocks > (int64_t)device_sms() * 128) blocks = (int64_t)device_sms() * 128;
    if (record_launch(kBPInject, a.precision == 0 ? launch_inject_batch<float> : launch_inject_batch<double>, a,
                      blocks))
        return;
    if (a.precision == 0) inject_kernel<float><<<(unsigned)blocks, kInjectThreads, 0, s>>>(a);
    else inject_kernel<double><<<(unsigned)blocks, kInjectThreads, 0, s>>>(a);
}

}  // namespace pic
