// pic_fields.cu -- field kernels: Yee leapfrog with Mur boundaries, binomial
// current filter, laser antenna and the FP64 field-energy reduction.
//
// Yee (1966) on the staggered lattice of pic_internal.cuh, B split in two half
// steps so that E and B both live at integer times:
//   B -= (dt/2) curl E;   E += dt (curl B - 2 pi J);   B -= (dt/2) curl E,
// all three in one kernel that reads E^n, B^n from one field buffer and writes
// E^{n+1}, B^{n+1} to another (yee2d_kernel, yee3d_kernel).  With absorbing z
// the tangential E (Ex, Ey) on the end planes k = 0 and k = nz follows Mur's
// first-order condition (Mur 1981).
#include "pic.h"
#include "pic_internal.cuh"
#include "pic_tma.cuh"

#include <cuda_pipeline.h>
#include <mutex>

namespace pic {

// ----------------------------------------------------------- tensor maps

bool encode_map_4d(CUtensorMap *map, const void *base, int elem, uint64_t n0, uint64_t n1, uint64_t n2,
                   uint64_t count, uint32_t b0, uint32_t b1)
{
    using Encode = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    static Encode fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<Encode>(p);
    });
    if (!fn || (reinterpret_cast<uintptr_t>(base) & 15u) || ((n0 * (uint64_t)elem) & 15u) ||
        ((b0 * (uint32_t)elem) & 15u) || b0 > 256 || b1 > 256 || count > 256)
        return false;
    const cuuint64_t dims[4] = {n0, n1, n2, count};
    const cuuint64_t strides[3] = {n0 * elem, n0 * n1 * elem, n0 * n1 * n2 * elem};
    const cuuint32_t box[4] = {b0, b1, 1, (cuuint32_t)count};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    const CUresult r = fn(map, elem == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4,
                          const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

template <typename real>
struct Ptr9 {
    real *p[9];
};

template <typename real>
struct YeeArgs {
    Geom g;
    const real *E[3], *B[3];  // E^n, B^n
    real *E1[3], *B1[3];      // E^{n+1}, B^{n+1} (another buffer)
    const real *J[3];
    real hb, he;              // dt/2 (B half steps), dt (E step)
    real ihx, ihy, ihz;       // 1 / h_d
    real twopi;               // 2 pi
    real mur;                 // (dt - hz) / (dt + hz)
    int cz, nchunks;          // z planes per chunk, chunks
};

// CTAs of a grid-stride loop over n items: all of them, at most 32 per SM
static unsigned grid_for(int64_t n, int block)
{
    int64_t b = (n + block - 1) / block;
    const int64_t cap = (int64_t)device_sms() * 32;
    return (unsigned)(b < cap ? (b > 0 ? b : 1) : cap);
}

// --------------------------------------------------- 2D Yee, column march

// One Yee step in one pass over the grid, as a march up z with the planes in
// registers: each thread holds one (x, y) column and a chunk of z planes,
// and at plane k of the march computes
//   Bh(k)   = B^n(k) - (dt/2) curl E^n       (E^n at k and k+1)
//   E'(k)   = E^n(k) + dt (curl Bh - 2 pi J)  (Bh at k and k-1)
//   B'(k-1) = Bh(k-1) - (dt/2) curl E'       (E' at k-1 and k)
// and writes E'(k-1), B'(k-1) to the other field buffer, so that no thread
// reads a value another one writes.  Every z neighbour is a register of the
// previous iteration, every x neighbour a warp shuffle (lane l holds column
// x0 + l - 1), and the loads of a plane are issued an iteration ahead of
// their use.  Each curl takes the next neighbour on one side, so the columns
// at a strip's edges are its halo: Bh is exact on lanes 0-30, E' on lanes
// 1-30 and B' on lanes 1-29, the strip's own kColOwn columns.  With absorbing
// z the tangential E (Ex, Ey) of the end planes follows Mur's first-order
// condition
//   E0^{n+1} = E1^n + (dt - dz)/(dt + dz) (E1^{n+1} - E0^n)
// (Mur 1981), evaluated from the registers once E' of the neighbouring plane
// is known.  The chunk [z0, z1) starts two planes early (E' of plane z0 - 1
// for Mur's upper plane when nz - 1 is the plane before the chunk) and ends
// one late.  The arithmetic per node is that of the split-B leapfrog written
// out term by term; planes a component does not have (Ez, Bx, By at k = nz;
// every component at k = nz with periodic z) are neither read nor written.
//
// In 2D (d/dy = 0) a warp is independent of the others: no shared memory
// and no barrier.
constexpr int kColOwn = 29;

template <typename real>
__device__ __forceinline__ void yee2d_body(const YeeArgs<real> &a, const int strip, const int chunk)
{
    const Geom &g = a.g;
    const bool per = g.bc_z == 0;
    const int nzo = per ? g.nz : g.nz + 1;
    const unsigned lane = threadIdx.x & 31u;
    const int x = strip * kColOwn + (int)lane - 1;
    const int gx = x >= 0 && x < g.nx ? x : wrapi(x, g.nx);
    const bool own = lane >= 1u && lane <= (unsigned)kColOwn && x < g.nx;
    const int z0 = chunk * a.cz;
    const int z1 = chunk == a.nchunks - 1 ? nzo : z0 + a.cz;
    // offset of this lane's node of plane k of a component with integer
    // (half = false) or half-integer z, -1 where the component has no plane k
    auto off = [&](int k, bool half) -> int64_t {
        const int kk = per ? wrapi(k, g.nz) : (k >= 0 && k <= zmax_of(g, half) ? k : -1);
        return kk >= 0 ? (int64_t)kk * g.plane + gx : int64_t(-1);
    };
    auto ld = [&](const real *p, int64_t o) { return o >= 0 ? p[o] : real(0); };
    auto dn = [&](real v) { return __shfl_down_sync(0xffffffffu, v, 1); };  // the value at x + 1
    auto up = [&](real v) { return __shfl_up_sync(0xffffffffu, v, 1); };    // the value at x - 1
    const real zero = real(0);
    const int kb = z0 - 2;
    // offsets of planes k and k + 1 (carried along the march)
    int64_t oi0 = off(kb, false), oh0 = off(kb, true), oi1 = off(kb + 1, false), oh1 = off(kb + 1, true);
    // E^n of planes k - 1 (for Mur), k and k + 1; B^n and J of plane k;
    // Bh and E' of plane k - 1
    real emx = 0, emy = 0;
    real ex0 = ld(a.E[0], oi0), ey0 = ld(a.E[1], oi0), ez0 = ld(a.E[2], oh0);
    real ex1 = ld(a.E[0], oi1), ey1 = ld(a.E[1], oi1), ez1 = ld(a.E[2], oh1);
    real bx = ld(a.B[0], oh0), by = ld(a.B[1], oh0), bz = ld(a.B[2], oi0);
    real jx = ld(a.J[0], oi0), jy = ld(a.J[1], oi0), jz = ld(a.J[2], oh0);
    real bmx = 0, bmy = 0, bmz = 0, fpx = 0, fpy = 0, fpz = 0;
    real murx = 0, mury = 0;  // E'(nz) x, y by Mur's condition (from plane nz - 1)
    for (int k = kb; k <= z1; ++k) {
        // the next plane's loads, used one iteration later
        const int64_t oi2 = off(k + 2, false), oh2 = off(k + 2, true);
        const real nex = ld(a.E[0], oi2), ney = ld(a.E[1], oi2), nez = ld(a.E[2], oh2);
        const real nbx = ld(a.B[0], oh1), nby = ld(a.B[1], oh1), nbz = ld(a.B[2], oi1);
        const real njx = ld(a.J[0], oi1), njy = ld(a.J[1], oi1), njz = ld(a.J[2], oh1);
        // ---- Bh(k)
        const bool vxy = oh0 >= 0, vz = oi0 >= 0;
        const real eyr = dn(ey0), ezr = dn(ez0);
        const real dEy_dz = (ey1 - ey0) * a.ihz;
        const real dEx_dz = (ex1 - ex0) * a.ihz;
        const real dEz_dx = (ezr - ez0) * a.ihx;
        const real dEy_dx = (eyr - ey0) * a.ihx;
        const real hx = vxy ? bx - a.hb * (zero - dEy_dz) : real(0);
        const real hy = vxy ? by - a.hb * (dEx_dz - dEz_dx) : real(0);
        const real hz = vz ? bz - a.hb * (dEy_dx - zero) : real(0);
        // ---- E'(k)
        real fx = ex0, fy = ey0, fz = 0;
        {
            const real hyl = up(hy), hzl = up(hz);
            const bool ve = per || (k >= 1 && k <= g.nz - 1), vze = oh0 >= 0;
            if (ve) {
                const real dBy_dz = (hy - bmy) * a.ihz;
                fx = ex0 + a.he * ((zero - dBy_dz) - a.twopi * jx);
                const real dBx_dz = (hx - bmx) * a.ihz;
                const real dBz_dx = (hz - hzl) * a.ihx;
                fy = ey0 + a.he * ((dBx_dz - dBz_dx) - a.twopi * jy);
            }
            const real dBy_dx = (hy - hyl) * a.ihx;
            fz = vze ? ez0 + a.he * ((dBy_dx - zero) - a.twopi * jz) : real(0);
            if (!per) {
                if (k == 1) {  // E'(0) x, y from plane 1
                    fpx = ex0 + a.mur * (fx - emx);
                    fpy = ey0 + a.mur * (fy - emy);
                }
                if (k == g.nz - 1) {  // E'(nz) x, y from plane nz - 1
                    murx = ex0 + a.mur * (fx - ex1);
                    mury = ey0 + a.mur * (fy - ey1);
                }
                if (k == g.nz) {
                    fx = murx;
                    fy = mury;
                }
            }
        }
        // ---- E'(k - 1), B'(k - 1) of the own columns
        {
            const int kw = k - 1;
            const real fpyr = dn(fpy), fpzr = dn(fpz);
            if (kw >= z0 && kw < z1 && own) {
                const int64_t o = (int64_t)kw * g.plane + x;
                const bool wxy = kw <= zmax_of(g, false), wz = kw <= zmax_of(g, true);
                if (wxy) {
                    a.E1[0][o] = fpx;
                    a.E1[1][o] = fpy;
                }
                if (wz) {
                    a.E1[2][o] = fpz;
                    const real dEy_dz1 = (fy - fpy) * a.ihz;
                    a.B1[0][o] = bmx - a.hb * (zero - dEy_dz1);
                    const real dEx_dz1 = (fx - fpx) * a.ihz;
                    const real dEz_dx1 = (fpzr - fpz) * a.ihx;
                    a.B1[1][o] = bmy - a.hb * (dEx_dz1 - dEz_dx1);
                }
                if (wxy) {
                    const real dEy_dx1 = (fpyr - fpy) * a.ihx;
                    a.B1[2][o] = bmz - a.hb * (dEy_dx1 - zero);
                }
            }
        }
        // ---- shift the march by one plane
        oi0 = oi1;
        oh0 = oh1;
        oi1 = oi2;
        oh1 = oh2;
        emx = ex0;
        emy = ey0;
        ex0 = ex1;
        ey0 = ey1;
        ez0 = ez1;
        ex1 = nex;
        ey1 = ney;
        ez1 = nez;
        bx = nbx;
        by = nby;
        bz = nbz;
        jx = njx;
        jy = njy;
        jz = njz;
        bmx = hx;
        bmy = hy;
        bmz = hz;
        fpx = fx;
        fpy = fy;
        fpz = fz;
    }
}

// ------------------------------------------------------ 3D Yee, column march

// The Yee step on 3D grids with the planes in registers: a CTA of 16 warps
// owns kCol3Y x kColOwn (y, x) columns and a chunk of z planes; warp w holds
// row y = y0 + w - 1 and lane l column x = x0 + l - 1 (both wrapped), so that
// the x neighbours are shuffles and the y neighbours come through shared
// memory, two exchanges per plane (E^n(k) and E'(k-1) with the row above;
// Bh(k) with the row below).  Bh is exact on lanes 0-30 and warps 0-14, E' on
// lanes 1-30 and warps 1-14, B' on lanes 1-29 and warps 1-13, the own
// columns.  The march, its chunk ends, Mur's planes and the arithmetic are
// yee2d_body's with the y terms of the curls.
constexpr int kCol3Y = 13, kCol3Warps = 16;

template <typename real>
__device__ __forceinline__ void yee3d_body(const YeeArgs<real> &a, const int sx, const int sy, const int chunk)
{
    __shared__ real xs[2][6][kCol3Warps][32];  // per parity: Ex, Ez, E'x, E'z of each row; Bh x, z
    const Geom &g = a.g;
    const bool per = g.bc_z == 0;
    const int nzo = per ? g.nz : g.nz + 1;
    const unsigned lane = threadIdx.x & 31u;
    const int w = (int)(threadIdx.x >> 5);
    const int x = sx * kColOwn + (int)lane - 1, y = sy * kCol3Y + w - 1;
    const int gx = x >= 0 && x < g.nx ? x : wrapi(x, g.nx);
    const int gy = y >= 0 && y < g.ny ? y : wrapi(y, g.ny);
    const int64_t col = (int64_t)gy * g.nx + gx;
    const bool own = lane >= 1u && lane <= (unsigned)kColOwn && w >= 1 && w <= kCol3Y && x < g.nx && y < g.ny;
    const int wu = w + 1 < kCol3Warps ? w + 1 : w, wd = w >= 1 ? w - 1 : w;  // rows above and below (halo: own)
    const int z0 = chunk * a.cz;
    const int z1 = chunk == a.nchunks - 1 ? nzo : z0 + a.cz;
    auto off = [&](int k, bool half) -> int64_t {
        const int kk = per ? wrapi(k, g.nz) : (k >= 0 && k <= zmax_of(g, half) ? k : -1);
        return kk >= 0 ? (int64_t)kk * g.plane + col : int64_t(-1);
    };
    auto ld = [&](const real *p, int64_t o) { return o >= 0 ? p[o] : real(0); };
    auto dn = [&](real v) { return __shfl_down_sync(0xffffffffu, v, 1); };  // x + 1
    auto up = [&](real v) { return __shfl_up_sync(0xffffffffu, v, 1); };    // x - 1
    const real zero = real(0);
    const int kb = z0 - 2;
    int64_t oi0 = off(kb, false), oh0 = off(kb, true), oi1 = off(kb + 1, false), oh1 = off(kb + 1, true);
    real emx = 0, emy = 0;
    real ex0 = ld(a.E[0], oi0), ey0 = ld(a.E[1], oi0), ez0 = ld(a.E[2], oh0);
    real ex1 = ld(a.E[0], oi1), ey1 = ld(a.E[1], oi1), ez1 = ld(a.E[2], oh1);
    real bx = ld(a.B[0], oh0), by = ld(a.B[1], oh0), bz = ld(a.B[2], oi0);
    real jx = ld(a.J[0], oi0), jy = ld(a.J[1], oi0), jz = ld(a.J[2], oh0);
    real bmx = 0, bmy = 0, bmz = 0, fpx = 0, fpy = 0, fpz = 0;
    real murx = 0, mury = 0;
    for (int k = kb; k <= z1; ++k) {
        const int P = k & 1;
        const int64_t oi2 = off(k + 2, false), oh2 = off(k + 2, true);
        const real nex = ld(a.E[0], oi2), ney = ld(a.E[1], oi2), nez = ld(a.E[2], oh2);
        const real nbx = ld(a.B[0], oh1), nby = ld(a.B[1], oh1), nbz = ld(a.B[2], oi1);
        const real njx = ld(a.J[0], oi1), njy = ld(a.J[1], oi1), njz = ld(a.J[2], oh1);
        // ---- exchange 1: E^n(k) and E'(k - 1) with the row above
        xs[P][0][w][lane] = ex0;
        xs[P][1][w][lane] = ez0;
        xs[P][2][w][lane] = fpx;
        xs[P][3][w][lane] = fpz;
        __syncthreads();
        const real exu = xs[P][0][wu][lane], ezu = xs[P][1][wu][lane];
        const real fpxu = xs[P][2][wu][lane], fpzu = xs[P][3][wu][lane];
        // ---- Bh(k)
        const bool vxy = oh0 >= 0, vz = oi0 >= 0;
        const real eyr = dn(ey0), ezr = dn(ez0);
        const real dEz_dy = (ezu - ez0) * a.ihy;
        const real dEx_dy = (exu - ex0) * a.ihy;
        const real dEy_dz = (ey1 - ey0) * a.ihz;
        const real dEx_dz = (ex1 - ex0) * a.ihz;
        const real dEz_dx = (ezr - ez0) * a.ihx;
        const real dEy_dx = (eyr - ey0) * a.ihx;
        const real hx = vxy ? bx - a.hb * (dEz_dy - dEy_dz) : real(0);
        const real hy = vxy ? by - a.hb * (dEx_dz - dEz_dx) : real(0);
        const real hz = vz ? bz - a.hb * (dEy_dx - dEx_dy) : real(0);
        // ---- exchange 2: Bh(k) with the row below
        xs[P][4][w][lane] = hx;
        xs[P][5][w][lane] = hz;
        __syncthreads();
        const real hxd = xs[P][4][wd][lane], hzd = xs[P][5][wd][lane];
        // ---- E'(k)
        real fx = ex0, fy = ey0, fz = 0;
        {
            const real hyl = up(hy), hzl = up(hz);
            const bool ve = per || (k >= 1 && k <= g.nz - 1), vze = oh0 >= 0;
            if (ve) {
                const real dBz_dy = (hz - hzd) * a.ihy;
                const real dBy_dz = (hy - bmy) * a.ihz;
                fx = ex0 + a.he * ((dBz_dy - dBy_dz) - a.twopi * jx);
                const real dBx_dz = (hx - bmx) * a.ihz;
                const real dBz_dx = (hz - hzl) * a.ihx;
                fy = ey0 + a.he * ((dBx_dz - dBz_dx) - a.twopi * jy);
            }
            const real dBy_dx = (hy - hyl) * a.ihx;
            const real dBx_dy = (hx - hxd) * a.ihy;
            fz = vze ? ez0 + a.he * ((dBy_dx - dBx_dy) - a.twopi * jz) : real(0);
            if (!per) {
                if (k == 1) {
                    fpx = ex0 + a.mur * (fx - emx);
                    fpy = ey0 + a.mur * (fy - emy);
                }
                if (k == g.nz - 1) {
                    murx = ex0 + a.mur * (fx - ex1);
                    mury = ey0 + a.mur * (fy - ey1);
                }
                if (k == g.nz) {
                    fx = murx;
                    fy = mury;
                }
            }
        }
        // ---- E'(k - 1), B'(k - 1) of the own columns.  At k = 1 Mur's
        // condition has just set E'(0) x, y: the row above's E'x(0), which B'z
        // reads, is exchanged again (k is the same for the whole CTA)
        real fpxu2 = fpxu;
        if (!per && k == 1) {
            xs[P][2][w][lane] = fpx;
            __syncthreads();
            fpxu2 = xs[P][2][wu][lane];
        }
        {
            const int kw = k - 1;
            const real fpyr = dn(fpy), fpzr = dn(fpz);
            if (kw >= z0 && kw < z1 && own) {
                const int64_t o = (int64_t)kw * g.plane + col;
                const bool wxy = kw <= zmax_of(g, false), wz = kw <= zmax_of(g, true);
                if (wxy) {
                    a.E1[0][o] = fpx;
                    a.E1[1][o] = fpy;
                }
                if (wz) {
                    a.E1[2][o] = fpz;
                    const real dEz_dy1 = (fpzu - fpz) * a.ihy;
                    const real dEy_dz1 = (fy - fpy) * a.ihz;
                    a.B1[0][o] = bmx - a.hb * (dEz_dy1 - dEy_dz1);
                    const real dEx_dz1 = (fx - fpx) * a.ihz;
                    const real dEz_dx1 = (fpzr - fpz) * a.ihx;
                    a.B1[1][o] = bmy - a.hb * (dEx_dz1 - dEz_dx1);
                }
                if (wxy) {
                    const real dEy_dx1 = (fpyr - fpy) * a.ihx;
                    const real dEx_dy1 = (fpxu2 - fpx) * a.ihy;
                    a.B1[2][o] = bmz - a.hb * (dEy_dx1 - dEx_dy1);
                }
            }
        }
        oi0 = oi1;
        oh0 = oh1;
        oi1 = oi2;
        oh1 = oh2;
        emx = ex0;
        emy = ey0;
        ex0 = ex1;
        ey0 = ey1;
        ez0 = ez1;
        ex1 = nex;
        ey1 = ney;
        ez1 = nez;
        bx = nbx;
        by = nby;
        bz = nbz;
        jx = njx;
        jy = njy;
        jz = njz;
        bmx = hx;
        bmy = hy;
        bmz = hz;
        fpx = fx;
        fpy = fy;
        fpz = fz;
    }
}

template <typename real>
__device__ __forceinline__ void yee3d_item(const YeeArgs<real> &a, int64_t item)
{
    const int nsx = (a.g.nx + kColOwn - 1) / kColOwn, nsy = (a.g.ny + kCol3Y - 1) / kCol3Y;
    const int sx = (int)(item % nsx), sy = (int)((item / nsx) % nsy), ch = (int)(item / ((int64_t)nsx * nsy));
    yee3d_body(a, sx, sy, ch);
}

template <typename real>
__global__ void __launch_bounds__(512, 2) yee3d_kernel(YeeArgs<real> a)
{
    yee3d_item(a, (int64_t)blockIdx.x);
}

template <typename real>
__global__ void __launch_bounds__(512, 2) yee3d_batch_kernel(const YeeArgs<real> *__restrict__ runs,
                                                             const int64_t *__restrict__ start, int n)
{
    __shared__ __align__(16) YeeArgs<real> sa;
    const int64_t b = batch_block(runs, start, n, &sa);
    yee3d_item(sa, b);
}

template <typename real>
static void launch_yee3d_batch(const void *args, const int64_t *start, int n, int64_t total, unsigned *,
                               cudaStream_t s)
{
    yee3d_batch_kernel<real><<<(unsigned)total, 512, 0, s>>>(static_cast<const YeeArgs<real> *>(args), start, n);
}

// one warp per (strip, chunk) item; YeeArgs::cz holds the planes per chunk,
// nchunks the chunks (the strips follow from the grid)
template <typename real>
__device__ __forceinline__ void yee2d_items(const YeeArgs<real> &a, int64_t item, int64_t nitems)
{
    if (item >= nitems) return;
    const int nstrip = (a.g.nx + kColOwn - 1) / kColOwn;
    yee2d_body(a, (int)(item % nstrip), (int)(item / nstrip));
}

template <typename real>
__global__ void __launch_bounds__(256) yee2d_kernel(YeeArgs<real> a, int64_t nitems)
{
    yee2d_items(a, (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5), nitems);
}

template <typename real>
__global__ void __launch_bounds__(256) yee2d_batch_kernel(const YeeArgs<real> *__restrict__ runs,
                                                          const int64_t *__restrict__ start, int n)
{
    __shared__ __align__(16) YeeArgs<real> sa;
    const int64_t b = batch_block(runs, start, n, &sa);
    const int nstrip = (sa.g.nx + kColOwn - 1) / kColOwn;
    yee2d_items(sa, b * 8 + (threadIdx.x >> 5), (int64_t)nstrip * sa.nchunks);
}

template <typename real>
static void launch_yee2d_batch(const void *args, const int64_t *start, int n, int64_t total, unsigned *,
                               cudaStream_t s)
{
    yee2d_batch_kernel<real><<<(unsigned)total, 256, 0, s>>>(static_cast<const YeeArgs<real> *>(args), start, n);
}

template <typename real>
void launch_yee(const Geom &g, real *const F[9], real *const F1[6], double dt, double hx, double hy, double hz,
                cudaStream_t s)
{
    YeeArgs<real> a;
    a.g = g;
    for (int c = 0; c < 3; ++c) {
        a.E[c] = F[c];
        a.B[c] = F[3 + c];
        a.J[c] = F[6 + c];
        a.E1[c] = F1[c];
        a.B1[c] = F1[3 + c];
    }
    a.hb = (real)(0.5 * dt);
    a.he = (real)dt;
    a.ihx = (real)(1.0 / hx);
    a.ihy = (real)(1.0 / hy);
    a.ihz = (real)(1.0 / hz);
    a.twopi = (real)6.283185307179586;
    a.mur = (real)((dt - hz) / (dt + hz));
    const int nzo = g.bc_z == 0 ? g.nz : g.nz + 1;
    const bool is3 = g.dim == 3;
    if (!is3) {
        // chunks of 12..64 planes, as many as leave about 24 warps per SM
        const int nstrip = (g.nx + kColOwn - 1) / kColOwn;
        int64_t czl = (int64_t)nzo * nstrip * batch_runs() / ((int64_t)device_sms() * 24);
        a.cz = (int)(czl < 12 ? 12 : (czl > 64 ? 64 : czl));
        if (a.cz > nzo) a.cz = nzo;
        a.nchunks = (nzo + a.cz - 1) / a.cz;
        const int64_t nitems = (int64_t)nstrip * a.nchunks, nblocks = (nitems + 7) / 8;
        if (record_launch(kBPYee, launch_yee2d_batch<real>, a, nblocks)) return;
        yee2d_kernel<real><<<(unsigned)nblocks, 256, 0, s>>>(a, nitems);
        return;
    }
    {
        // the column march: chunks of 16..64 planes, as many as leave about
        // four CTAs of 16 warps per SM
        const int64_t ncol = (int64_t)((g.nx + kColOwn - 1) / kColOwn) * ((g.ny + kCol3Y - 1) / kCol3Y);
        int64_t czl = (int64_t)nzo * ncol * batch_runs() / ((int64_t)device_sms() * 4);
        a.cz = (int)(czl < 16 ? 16 : (czl > 64 ? 64 : czl));
        if (a.cz > nzo) a.cz = nzo;
        a.nchunks = (nzo + a.cz - 1) / a.cz;
        const int64_t nblocks = ncol * a.nchunks;
        if (record_launch(kBPYee, launch_yee3d_batch<real>, a, nblocks)) return;
        yee3d_kernel<real><<<(unsigned)nblocks, 512, 0, s>>>(a);
    }
}

// ---------------------------------------------------------- moving window

// dst plane k = src plane k + S (zero for k + S > nz), nine components
template <typename real>
__global__ void window_fields_kernel(Geom g, Ptr9<real> src, Ptr9<real> dst, int S)
{
    const int64_t n = 9 * g.ncomp;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(q / g.ncomp);
        const int64_t o = q - c * g.ncomp;
        const int64_t k = o / g.plane;
        dst.p[c][o] = k + S <= g.nz ? src.p[c][o + S * g.plane] : real(0);
    }
}

template <typename real>
void launch_window_fields(const Geom &g, real *const src[9], real *const dst[9], int S, cudaStream_t s)
{
    Ptr9<real> a, b;
    for (int c = 0; c < 9; ++c) {
        a.p[c] = src[c];
        b.p[c] = dst[c];
    }
    window_fields_kernel<real><<<grid_for(9 * g.ncomp, 256), 256, 0, s>>>(g, a, b, S);
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

// All H passes of all axes in one z-marching kernel.  A CTA owns a TX x TY
// column of nodes (32 x 8 in 3D, 256 x 1 in 2D) of the three components and a
// chunk of z planes.  Per plane it loads the column widened by H nodes in x
// and y (periodic) into shared memory; H binomial passes along x and then
// along y are, on a periodic axis, the binomial stencil of width 2H + 1
// (weights C(2H, i) / 4^H, exact in binary), so each thread takes its node's
// x-y filtered value as that stencil sum.  The z passes follow in registers,
// one pass after the other as the march goes up, each on values that are zero
// outside the component's valid z range (absorbing z) or wrapped (periodic).
// The chunk starts H planes early and ends H planes late.
template <typename real, int DIM, int H>
__device__ __forceinline__ void march_body(const Geom &g, const real *in, real *out, const int cz, const int nchunks,
                                           const int bx_, const int by_)
{
    constexpr int TX = DIM == 3 ? 32 : 256, TY = DIM == 3 ? 8 : 1, HY = DIM == 3 ? H : 0;
    constexpr int RX = TX + 2 * H, RY = TY + 2 * HY, RN = RX * RY;
    constexpr int W = 2 * H + 1;
    __shared__ real A[3][RN];
    // binomial weights C(2H, i) / 4^H
    real wb[W];
    {
        double c = 1.0;
        for (int i = 0; i < W; ++i) {
            wb[i] = (real)(c / (double)(1 << (2 * H)));
            c = c * (double)(2 * H - i) / (double)(i + 1);
        }
    }
    const bool per = g.bc_z == 0;
    const int nbx = (g.nx + TX - 1) / TX;
    const int x0 = (bx_ % nbx) * TX, y0 = (bx_ / nbx) * TY;
    const int z0 = by_ * cz;
    const int z1 = by_ == nchunks - 1 ? g.nz + 1 : z0 + cz;
    const int tid = threadIdx.x, tx = tid % TX, ty = tid / TX;
    const bool own = x0 + tx < g.nx && (DIM == 2 || y0 + ty < g.ny);
    const int64_t oown = own ? (int64_t)(y0 + ty) * g.nx + (x0 + tx) : 0;
    // this thread's nodes of the widened plane (at most ceil(RN / 256) of them)
    constexpr int NL = (RN + 255) / 256;
    int off[NL];
#pragma unroll
    for (int m = 0; m < NL; ++m) {
        const int r = tid + 256 * m;
        const int ly = r / RX, lx = r - ly * RX;
        const int gx = wrapi(x0 - H + lx, g.nx);
        const int gy = DIM == 3 ? wrapi(y0 - HY + ly, g.ny) : 0;
        off[m] = r < RN ? gy * g.nx + gx : -1;
    }
    // per component, z windows: lev[c][p][0..2] = the values after p z passes
    // at the last three planes they were computed for
    real lev[3][H + 1][3];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int p = 0; p <= H; ++p) lev[c][p][0] = lev[c][p][1] = lev[c][p][2] = real(0);
    const int zmax_xy = zmax_of(g, false), zmax_z = zmax_of(g, true);
    for (int k = z0 - H; k <= z1 - 1 + H; ++k) {
        const int kk = per ? wrapi(k, g.nz) : k;
        __syncthreads();  // previous plane consumed
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const bool have = per || (k >= 0 && k <= (c == 2 ? zmax_z : zmax_xy));
            const real *src = in + (size_t)c * g.ncomp + (int64_t)kk * g.plane;
#pragma unroll
            for (int m = 0; m < NL; ++m)
                if (off[m] >= 0) A[c][tid + 256 * m] = have ? src[off[m]] : real(0);
        }
        __syncthreads();
        const int ko = k - H;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const int zmax = c == 2 ? zmax_z : zmax_xy;
            // x-y passes: the binomial stencil around this thread's node
            real v = 0;
#pragma unroll
            for (int j = 0; j < (DIM == 3 ? W : 1); ++j) {
                real r = 0;
#pragma unroll
                for (int i = 0; i < W; ++i) r += wb[i] * A[c][(ty + j) * RX + tx + i];
                v += (DIM == 3 ? wb[j] : real(1)) * r;
            }
            // z passes, one level per pass, each centred one plane lower
#pragma unroll
            for (int p = 0; p <= H; ++p) {
                lev[c][p][0] = lev[c][p][1];
                lev[c][p][1] = lev[c][p][2];
                const int kc = k - p;  // plane of the new level-p value
                const bool in_range = per || (kc >= 0 && kc <= zmax);
                const real nv = p == 0 ? v
                                       : real(0.25) * lev[c][p - 1][0] + real(0.5) * lev[c][p - 1][1] +
                                             real(0.25) * lev[c][p - 1][2];
                lev[c][p][2] = in_range ? nv : real(0);
            }
            if (own && ko >= z0 && ko < z1)
                out[(size_t)c * g.ncomp + (int64_t)ko * g.plane + oown] = ko > zmax ? real(0) : lev[c][H][2];
        }
    }
}

template <typename real, int DIM, int H>
__global__ void __launch_bounds__(256) filter_march_kernel(Geom g, const real *in, real *out, int cz, int nchunks)
{
    march_body<real, DIM, H>(g, in, out, cz, nchunks, (int)blockIdx.x, (int)blockIdx.y);
}

template <typename real>
struct MarchArgs {
    Geom g;
    const real *in;
    real *out;
    int cz, nchunks;
};

template <typename real, int DIM, int H>
__global__ void __launch_bounds__(256) filter_march_batch_kernel(const MarchArgs<real> *__restrict__ runs,
                                                                 const int64_t *__restrict__ start, int n)
{
    __shared__ __align__(16) MarchArgs<real> sa;
    const int64_t b = batch_block(runs, start, n, &sa);
    constexpr int TX = DIM == 3 ? 32 : 256, TY = DIM == 3 ? 8 : 1;
    const int ncol = ((sa.g.nx + TX - 1) / TX) * (DIM == 3 ? (sa.g.ny + TY - 1) / TY : 1);
    march_body<real, DIM, H>(sa.g, sa.in, sa.out, sa.cz, sa.nchunks, (int)(b % ncol), (int)(b / ncol));
}

template <typename real, int DIM, int H>
static void launch_march_batch(const void *args, const int64_t *start, int n, int64_t total, unsigned *,
                               cudaStream_t s)
{
    filter_march_batch_kernel<real, DIM, H>
        <<<(unsigned)total, 256, 0, s>>>(static_cast<const MarchArgs<real> *>(args), start, n);
}

// The same filter in 3D with its planes staged by TMA.  A CTA owns a 32 x 8
// (x, y) column and a chunk of z planes; one tiled bulk tensor copy per plane
// brings the three components of the column widened to x0 - 4 .. x0 + 35
// (the copy's x start must be a multiple of 4 elements: the H <= 4 halo
// nodes needed on each side lie inside) and y0 - H .. y0 + 7 + H into shared
// memory, completing on that stage's mbarrier; NS planes are in flight while
// one is filtered.  Nodes outside the grid in x or y arrive as zeros and are
// replaced by their periodic images, loaded into registers one plane ahead
// (only CTAs at a grid edge have any); z beyond the grid is zero (absorbing)
// or wrapped by the copy's z coordinate (periodic).  The x-y passes are the
// binomial stencil of width 2H + 1 taken separably (x over the widened rows
// into shared memory, then y), the z passes are those of
// filter_march_kernel.  The x pass works on 16-byte groups of consecutive
// outputs (their inputs read as 16-byte vectors); the z levels sit in a ring
// of three register slots, the march unrolled by three so that the slot of
// each plane is a compile-time index and no value is moved between planes.
// A stage whose copy does not land within the wait budget stops the CTA and
// records ERR_TIMEOUT.
constexpr int kFilterStages = 4;

template <typename real> struct Vec16;
template <> struct Vec16<float> { using type = float4; };
template <> struct Vec16<double> { using type = double2; };
__device__ __forceinline__ void unpack16(const float4 &t, float *o)
{
    o[0] = t.x;
    o[1] = t.y;
    o[2] = t.z;
    o[3] = t.w;
}
__device__ __forceinline__ void unpack16(const double2 &t, double *o)
{
    o[0] = t.x;
    o[1] = t.y;
}
__device__ __forceinline__ float4 pack16(const float *o) { return make_float4(o[0], o[1], o[2], o[3]); }
__device__ __forceinline__ double2 pack16(const double *o) { return make_double2(o[0], o[1]); }
template <int N> struct Slot { static constexpr int value = N; };

// CTAs per SM the register budget allows without spills
template <typename real, int H> struct FilterTmaBlocks {
    static constexpr int value = sizeof(real) == 4 ? (H <= 2 ? 4 : 3) : (H <= 2 ? 3 : 2);
};

template <typename real, int H>
__global__ void __launch_bounds__(256, (FilterTmaBlocks<real, H>::value)) filter_tma_kernel(const __grid_constant__ CUtensorMap map, Geom g,
                                                         const real *in, real *out, int cz, int nchunks,
                                                         unsigned *err)
{
    constexpr int TX = 32, TY = 8, BX = TX + 8, BY = TY + 2 * H, PN = BX * BY;
    constexpr int NS = kFilterStages, W = 2 * H + 1, XO = 4 - H;
    constexpr uint32_t kBytes = 3u * PN * sizeof(real);
    // a tensor copy's shared-memory destination must sit on a 128-byte
    // boundary: stages are kStride elements apart, the base is rounded up
    constexpr int kStride = (int)(((kBytes + 127u) / 128u) * 128u / sizeof(real));
    constexpr int XR = BY * TX;                  // x-filtered values per component
    // x-pass groups: VW consecutive outputs of one row, from the VW + 8
    // inputs starting at the group's own column (16-byte aligned: stages,
    // components and rows all start on 16-byte boundaries)
    constexpr int VW = 16 / (int)sizeof(real), NV = (VW + 8) / VW, GR = TX / VW;
    constexpr int XG = 3 * BY * GR, NXG = (XG + 255) / 256;
    static_assert(TX % VW == 0 && BX % VW == 0 && H <= 4, "x-pass groups");
    using vec_t = typename Vec16<real>::type;
    constexpr int NP = (3 * PN + 255) / 256;     // box nodes per thread (periodic images)
    extern __shared__ __align__(128) unsigned char smem_tma[];
    real *stage = reinterpret_cast<real *>(smem_tma + ((128u - (smem_addr(smem_tma) & 127u)) & 127u));
    real *xs = stage + (size_t)NS * kStride;     // [3][BY][TX]
    __shared__ __align__(8) uint64_t bar[NS];
    real wb[W];
    {
        double c = 1.0;
        for (int i = 0; i < W; ++i) {
            wb[i] = (real)(c / (double)(1 << (2 * H)));
            c = c * (double)(2 * H - i) / (double)(i + 1);
        }
    }
    const bool per = g.bc_z == 0;
    const int nbx = (g.nx + TX - 1) / TX;
    const int x0 = (int)(blockIdx.x % nbx) * TX, y0 = (int)(blockIdx.x / nbx) * TY;
    const int z0 = (int)blockIdx.y * cz;
    const int z1 = (int)blockIdx.y == nchunks - 1 ? g.nz + 1 : z0 + cz;
    const int kf = z0 - H, np = (z1 - 1 + H) - kf + 1;
    const int tid = threadIdx.x, tx = tid % TX, ty = tid / TX;
    const bool own = x0 + tx < g.nx && y0 + ty < g.ny;
    const int64_t oown = own ? (int64_t)(y0 + ty) * g.nx + (x0 + tx) : 0;
    const bool edge = x0 - 4 < 0 || x0 + TX + 4 > g.nx || y0 - H < 0 || y0 + TY + H > g.ny;
    const int zmax_xy = zmax_of(g, false), zmax_z = zmax_of(g, true);
    // this thread's box nodes outside the grid in x or y: their periodic
    // images' offsets within a plane
    int poff[NP];
    unsigned pmask = 0u;
#pragma unroll
    for (int m = 0; m < NP; ++m) {
        poff[m] = 0;
        const int r = tid + 256 * m;
        if (!edge || r >= 3 * PN) continue;
        const int rr = r % PN, ly = rr / BX, lx = rr - ly * BX;
        const int gx = x0 - 4 + lx, gy = y0 - H + ly;
        if (gx >= 0 && gx < g.nx && gy >= 0 && gy < g.ny) continue;
        poff[m] = wrapi(gy, g.ny) * g.nx + wrapi(gx, g.nx);
        pmask |= 1u << m;
    }
    real pv[NP];
    auto patch_load = [&](int k) {  // plane k's periodic images into registers
        const int kk = per ? wrapi(k, g.nz) : k;
#pragma unroll
        for (int m = 0; m < NP; ++m) {
            if (!(pmask >> m & 1u)) continue;
            const int c = (tid + 256 * m) / PN;
            const bool have = per || (k >= 0 && k <= (c == 2 ? zmax_z : zmax_xy));
            pv[m] = have ? in[(size_t)c * g.ncomp + (int64_t)kk * g.plane + poff[m]] : real(0);
        }
    };
    if (tid == 0) {
        for (int q = 0; q < NS; ++q) mbar_init(&bar[q], 1);
        fence_proxy_async();
    }
    __syncthreads();
    auto issue = [&](int q) {  // plane kf + q into stage q % NS
        const int k = kf + q;
        uint64_t *b = &bar[q % NS];
        mbar_arrive_expect(b, kBytes);
        tma_load_4d(stage + (size_t)(q % NS) * kStride, &map, x0 - 4, y0 - H, per ? wrapi(k, g.nz) : k, 0, b);
    };
    if (tid == 0)
        for (int q = 0; q < NS && q < np; ++q) issue(q);
    if (pmask) patch_load(kf);
    // z levels: level p taken at march plane k (its value belongs to plane
    // k - p) sits in slot (k - kf) % 3
    real lev[3][H + 1][3];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int p = 0; p <= H; ++p) lev[c][p][0] = lev[c][p][1] = lev[c][p][2] = real(0);
    // one plane of the march; false once a copy has not landed (the CTA
    // stops together)
    auto plane = [&](const int q, auto slot) -> bool {
        constexpr int PH = decltype(slot)::value, P1 = (PH + 1) % 3, P2 = (PH + 2) % 3;  // planes q, q-2, q-1
        const int k = kf + q;
        real *S = stage + (size_t)(q % NS) * kStride;
        const bool ok = mbar_wait(&bar[q % NS], (uint32_t)(q / NS) & 1u, global_ns(), kWaitBudgetNs);
        if (ok) {
            // planes a component does not have are zero (Jz at k = nz)
            if (!per && k == g.nz)
                for (int r = tid; r < PN; r += 256) S[2 * PN + r] = real(0);
            if (pmask) {
#pragma unroll
                for (int m = 0; m < NP; ++m)
                    if (pmask >> m & 1u) S[tid + 256 * m] = pv[m];
                if (q + 1 < np) patch_load(k + 1);  // in flight while this plane is filtered
            }
        }
        if (__syncthreads_or(!ok)) return false;
        // x passes over the widened rows
#pragma unroll
        for (int n = 0; n < NXG; ++n) {
            const int gi = tid + 256 * n;
            if (gi < XG) {
                const int c = gi / (BY * GR), rr = gi - c * (BY * GR), row = rr / GR, cv = rr - row * GR;
                const vec_t *A = reinterpret_cast<const vec_t *>(S + c * PN + row * BX + cv * VW);
                real in[NV * VW];
#pragma unroll
                for (int m = 0; m < NV; ++m) unpack16(A[m], in + m * VW);
                real o[VW];
#pragma unroll
                for (int j = 0; j < VW; ++j) {
                    real v = 0;
#pragma unroll
                    for (int i = 0; i < W; ++i) v += wb[i] * in[j + XO + i];
                    o[j] = v;
                }
                *reinterpret_cast<vec_t *>(xs + c * XR + row * TX + cv * VW) = pack16(o);
            }
        }
        __syncthreads();  // the stage is consumed: refill it while the y and z passes run
        if (tid == 0 && q + NS < np) {
            fence_proxy_async();
            issue(q + NS);
        }
        const int ko = k - H;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const int zmax = c == 2 ? zmax_z : zmax_xy;
            const real *X = xs + c * XR + ty * TX + tx;
            real v = 0;
#pragma unroll
            for (int j = 0; j < W; ++j) v += wb[j] * X[j * TX];
#pragma unroll
            for (int p = 0; p <= H; ++p) {
                const int kc = k - p;
                const bool in_range = per || (kc >= 0 && kc <= zmax);
                const real nv = p == 0 ? v
                                       : real(0.25) * lev[c][p - 1][P1] + real(0.5) * lev[c][p - 1][P2] +
                                             real(0.25) * lev[c][p - 1][PH];
                lev[c][p][PH] = in_range ? nv : real(0);
            }
            if (own && ko >= z0 && ko < z1)
                out[(size_t)c * g.ncomp + (int64_t)ko * g.plane + oown] = ko > zmax ? real(0) : lev[c][H][PH];
        }
        return true;
    };
    int q = 0;
    while (q < np) {
        if (!plane(q, Slot<0>())) break;
        if (++q >= np) break;
        if (!plane(q, Slot<1>())) break;
        if (++q >= np) break;
        if (!plane(q, Slot<2>())) break;
        ++q;
    }
    if (q < np) {
        // a copy did not land: record it, then give the copies still in
        // flight a bounded chance to finish before the CTA leaves
        if (tid == 0) {
            if (err) atomicOr(err, ERR_TIMEOUT);
            const int last = np < q + NS ? np : q + NS;
            for (int r = q; r < last; ++r)
                (void)mbar_wait(&bar[r % NS], (uint32_t)(r / NS) & 1u, global_ns(), kWaitBudgetNs / 4);
        }
        __syncthreads();
    }
}

template <typename real, int H>
static bool launch_filter_tma(const Geom &g, const real *in, real *out, unsigned *err, cudaStream_t s)
{
    constexpr int TX = 32, TY = 8, BX = TX + 8, BY = TY + 2 * H;
    // a batch of runs takes the plane-load kernel (one tensor map per launch)
    if (g_rec) return false;
    CUtensorMap map;
    if (!encode_map_4d(&map, in, (int)sizeof(real), (uint64_t)g.nx, (uint64_t)g.ny, (uint64_t)g.nz + 1, 3, BX, BY))
        return false;
    const int nzo = g.nz + 1;
    const unsigned nb = (unsigned)(((g.nx + TX - 1) / TX) * ((g.ny + TY - 1) / TY));
    // z chunks of 8..64 planes, as long as there are about eight CTAs per SM
    int64_t czl = (int64_t)nzo * nb / ((int64_t)device_sms() * 8);
    czl = czl < 8 ? 8 : (czl > 64 ? 64 : czl);
    const int cz = (int)(czl < nzo ? czl : nzo);
    const int nchunks = nzo / cz > 0 ? nzo / cz : 1;
    // stages on 128-byte boundaries, plus room to align the base, then the
    // x-filtered rows
    const size_t stage_bytes = ((size_t)3 * BX * BY * sizeof(real) + 127) / 128 * 128;
    const size_t smem = (size_t)kFilterStages * stage_bytes + 128 + (size_t)3 * BY * TX * sizeof(real);
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(filter_tma_kernel<real, H>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    filter_tma_kernel<real, H><<<dim3(nb, (unsigned)nchunks, 1), 256, smem, s>>>(map, g, in, out, cz, nchunks, err);
    return true;
}

// The same H passes on 2D grids with the planes in registers: a warp owns a
// strip of 32 - 2H x columns and a chunk of z planes (lane l: x = strip
// (32 - 2H) + l - H, wrapped; lanes H .. 31 - H own their column), marches
// up the chunk like filter_march_kernel and takes the x passes (the binomial
// stencil of width 2H + 1) over the lanes l - H .. l + H by shuffles; the z
// passes are the march's register levels.  No shared memory, no barrier; a
// plane's loads are issued an iteration ahead of their use.
template <typename real, int H>
__device__ __forceinline__ void filter2d_body(const Geom &g, const real *in, real *out, const int strip,
                                              const int chunk, const int cz, const int nchunks)
{
    constexpr int OWN = 32 - 2 * H, NW = 2 * H + 1;
    real wb[NW];
    {
        double c = 1.0;
        for (int i = 0; i < NW; ++i) {
            wb[i] = (real)(c / (double)(1 << (2 * H)));
            c = c * (double)(2 * H - i) / (double)(i + 1);
        }
    }
    const bool per = g.bc_z == 0;
    const int lane = (int)(threadIdx.x & 31u);
    const int x = strip * OWN + lane - H;
    const int gx = x >= 0 && x < g.nx ? x : wrapi(x, g.nx);
    const bool own = lane >= H && lane < 32 - H && x < g.nx;
    const int z0 = chunk * cz;
    const int z1 = chunk == nchunks - 1 ? g.nz + 1 : z0 + cz;
    const int zmax_xy = zmax_of(g, false), zmax_z = zmax_of(g, true);
    // the three components of plane k (Jx, Jy on integer z, Jz on half-integer z)
    auto load3 = [&](int k, real v[3]) {
        const int kk = per ? wrapi(k, g.nz) : k;
        const int64_t o = (int64_t)kk * g.plane + gx;
        const bool hxy = per || (k >= 0 && k <= zmax_xy), hz = per || (k >= 0 && k <= zmax_z);
        v[0] = hxy ? in[o] : real(0);
        v[1] = hxy ? in[g.ncomp + o] : real(0);
        v[2] = hz ? in[2 * g.ncomp + o] : real(0);
    };
    real lev[3][H + 1][3];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int p = 0; p <= H; ++p) lev[c][p][0] = lev[c][p][1] = lev[c][p][2] = real(0);
    real cur[3];
    load3(z0 - H, cur);
    for (int k = z0 - H; k <= z1 - 1 + H; ++k) {
        real nxt[3] = {real(0), real(0), real(0)};
        if (k + 1 <= z1 - 1 + H) load3(k + 1, nxt);
        const int ko = k - H;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const int zmax = c == 2 ? zmax_z : zmax_xy;
            // x passes: the binomial stencil around this lane's column
            real r = 0;
#pragma unroll
            for (int i = 0; i < NW; ++i) r += wb[i] * __shfl_sync(0xffffffffu, cur[c], lane - H + i);
            const real v = real(0) + real(1) * r;
            // z passes, one level per pass, each centred one plane lower
#pragma unroll
            for (int p = 0; p <= H; ++p) {
                lev[c][p][0] = lev[c][p][1];
                lev[c][p][1] = lev[c][p][2];
                const int kc = k - p;
                const bool in_range = per || (kc >= 0 && kc <= zmax);
                const real nv = p == 0 ? v
                                       : real(0.25) * lev[c][p - 1][0] + real(0.5) * lev[c][p - 1][1] +
                                             real(0.25) * lev[c][p - 1][2];
                lev[c][p][2] = in_range ? nv : real(0);
            }
            if (own && ko >= z0 && ko < z1)
                out[(size_t)c * g.ncomp + (int64_t)ko * g.plane + x] = ko > zmax ? real(0) : lev[c][H][2];
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) cur[c] = nxt[c];
    }
}

// one warp per (strip, chunk) item
template <typename real, int H>
__device__ __forceinline__ void filter2d_items(const Geom &g, const real *in, real *out, int cz, int nchunks,
                                               int64_t item)
{
    const int nstrip = (g.nx + (32 - 2 * H) - 1) / (32 - 2 * H);
    if (item >= (int64_t)nstrip * nchunks) return;
    filter2d_body<real, H>(g, in, out, (int)(item % nstrip), (int)(item / nstrip), cz, nchunks);
}

template <typename real, int H>
__global__ void __launch_bounds__(256) filter2d_kernel(Geom g, const real *in, real *out, int cz, int nchunks)
{
    filter2d_items<real, H>(g, in, out, cz, nchunks, (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5));
}

template <typename real, int H>
__global__ void __launch_bounds__(256) filter2d_batch_kernel(const MarchArgs<real> *__restrict__ runs,
                                                             const int64_t *__restrict__ start, int n)
{
    __shared__ __align__(16) MarchArgs<real> sa;
    const int64_t b = batch_block(runs, start, n, &sa);
    filter2d_items<real, H>(sa.g, sa.in, sa.out, sa.cz, sa.nchunks, b * 8 + (threadIdx.x >> 5));
}

template <typename real, int H>
static void launch_filter2d_batch(const void *args, const int64_t *start, int n, int64_t total, unsigned *,
                                  cudaStream_t s)
{
    filter2d_batch_kernel<real, H>
        <<<(unsigned)total, 256, 0, s>>>(static_cast<const MarchArgs<real> *>(args), start, n);
}

template <typename real, int DIM, int H>
static void launch_march(const Geom &g, const real *in, real *out, cudaStream_t s)
{
    const int nzo = g.nz + 1;
    if constexpr (DIM == 2) {
        // the register march (2D grids): chunks of 12..64 planes, as many as
        // leave about 24 warps per SM
        constexpr int OWN = 32 - 2 * H;
        const int nstrip = (g.nx + OWN - 1) / OWN;
        int64_t czl = (int64_t)nzo * nstrip * batch_runs() / ((int64_t)device_sms() * 24);
        int cz = (int)(czl < 12 ? 12 : (czl > 64 ? 64 : czl));
        if (cz > nzo) cz = nzo;
        const int nchunks = (nzo + cz - 1) / cz;
        const int64_t nblocks = ((int64_t)nstrip * nchunks + 7) / 8;
        if (record_launch(kBPFilter, launch_filter2d_batch<real, H>, MarchArgs<real>{g, in, out, cz, nchunks},
                          nblocks))
            return;
        filter2d_kernel<real, H><<<(unsigned)nblocks, 256, 0, s>>>(g, in, out, cz, nchunks);
    } else {
        constexpr int TX = 32, TY = 8;
        const unsigned nb = (unsigned)(((g.nx + TX - 1) / TX) * ((g.ny + TY - 1) / TY));
        // z chunks of 8..64 planes, as long as there are about eight CTAs per SM
        int64_t czl = (int64_t)nzo * nb * batch_runs() / ((int64_t)device_sms() * 8);
        czl = czl < 8 ? 8 : (czl > 64 ? 64 : czl);
        const int cz = (int)(czl < nzo ? czl : nzo);
        const int nchunks = nzo / cz > 0 ? nzo / cz : 1;
        if (record_launch(kBPFilter, launch_march_batch<real, DIM, H>, MarchArgs<real>{g, in, out, cz, nchunks},
                          (int64_t)nb * nchunks))
            return;
        filter_march_kernel<real, DIM, H><<<dim3(nb, (unsigned)nchunks, 1), 256, 0, s>>>(g, in, out, cz, nchunks);
    }
}

template <typename real>
static bool fused_passes(const Geom &g, const real *in, real *out, int npass, cudaStream_t s, unsigned *err)
{
    if (npass < 1 || npass > 4) return false;
    if (g.dim == 3) {
        // TMA staging where the tensor map can be made (x extent a multiple
        // of 16 bytes), else the plane loads of filter_march_kernel
        bool done = false;
        switch (npass) {
        case 1: done = launch_filter_tma<real, 1>(g, in, out, err, s); break;
        case 2: done = launch_filter_tma<real, 2>(g, in, out, err, s); break;
        case 3: done = launch_filter_tma<real, 3>(g, in, out, err, s); break;
        default: done = launch_filter_tma<real, 4>(g, in, out, err, s); break;
        }
        if (done) return true;
        switch (npass) {
        case 1: launch_march<real, 3, 1>(g, in, out, s); break;
        case 2: launch_march<real, 3, 2>(g, in, out, s); break;
        case 3: launch_march<real, 3, 3>(g, in, out, s); break;
        default: launch_march<real, 3, 4>(g, in, out, s); break;
        }
    } else {
        switch (npass) {
        case 1: launch_march<real, 2, 1>(g, in, out, s); break;
        case 2: launch_march<real, 2, 2>(g, in, out, s); break;
        case 3: launch_march<real, 2, 3>(g, in, out, s); break;
        default: launch_march<real, 2, 4>(g, in, out, s); break;
        }
    }
    return true;
}

template <typename real>
bool launch_filter_from(const Geom &g, const real *src, real *const J[3], int npass, cudaStream_t s, unsigned *err)
{
    const bool contiguous = J[1] == J[0] + g.ncomp && J[2] == J[1] + g.ncomp;
    return contiguous && fused_passes<real>(g, src, J[0], npass, s, err);
}

template <typename real>
void launch_filter(const Geom &g, real *const J[3], real *tmp, int npass, cudaStream_t s, unsigned *err)
{
    if (npass <= 0) return;
    // the three components are contiguous in the field buffer; the fused
    // kernel covers 1..4 passes, more fall back to one launch per pass
    if (record_unsupported()) return;  // (a copy back, or one launch per pass)
    const bool contiguous = J[1] == J[0] + g.ncomp && J[2] == J[1] + g.ncomp;
    if (contiguous && fused_passes<real>(g, J[0], tmp, npass, s, err)) {
        cudaMemcpyAsync(J[0], tmp, 3 * sizeof(real) * g.ncomp, cudaMemcpyDeviceToDevice, s);
        return;
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
struct AntennaArgs {
    Geom g;
    real *J;
    int pol, ka;
    double j0, hx, hy, xc, yc, inv_w2;
    const double *j0p;
};

template <typename real>
__device__ __forceinline__ void antenna_body(const AntennaArgs<real> &a, int64_t b, int64_t nb)
{
    const Geom &g = a.g;
    const double j0 = a.j0p ? *a.j0p : a.j0;
    const int64_t n = g.plane;
    for (int64_t o = b * blockDim.x + threadIdx.x; o < n; o += nb * blockDim.x) {
        const int i = (int)(o % g.nx), j = (int)(o / g.nx);
        const double x = ((double)i + (a.pol == 0 ? 0.5 : 0.0)) * a.hx - a.xc;
        double r2 = x * x;
        if (g.dim == 3) {
            const double y = ((double)j + (a.pol == 1 ? 0.5 : 0.0)) * a.hy - a.yc;
            r2 += y * y;
        }
        a.J[(int64_t)a.ka * g.plane + o] += (real)(j0 * exp(-r2 * a.inv_w2));
    }
}

template <typename real>
__global__ void antenna_kernel(AntennaArgs<real> a)
{
    antenna_body(a, (int64_t)blockIdx.x, (int64_t)gridDim.x);
}

template <typename real>
__global__ void antenna_batch_kernel(const AntennaArgs<real> *__restrict__ runs, const int64_t *__restrict__ start,
                                     int n)
{
    __shared__ __align__(16) AntennaArgs<real> sa;
    const int64_t b = batch_block(runs, start, n, &sa);
    const int r = batch_run_of(start, n, (int64_t)blockIdx.x);
    antenna_body(sa, b, start[r + 1] - start[r]);
}

template <typename real>
static void launch_antenna_batch(const void *args, const int64_t *start, int n, int64_t total, unsigned *,
                                 cudaStream_t s)
{
    antenna_batch_kernel<real><<<(unsigned)total, 256, 0, s>>>(static_cast<const AntennaArgs<real> *>(args), start, n);
}

template <typename real>
void launch_antenna(const Geom &g, real *J, int pol, int ka, double j0, double hx, double hy, double xc,
                    double yc, double waist, cudaStream_t s, const double *j0p)
{
    const AntennaArgs<real> a{g, J, pol, ka, j0, hx, hy, xc, yc, 1.0 / (waist * waist), j0p};
    const unsigned nb = grid_for(g.plane, 256);
    if (record_launch(kBPAntenna, launch_antenna_batch<real>, a, (int64_t)nb)) return;
    antenna_kernel<real><<<nb, 256, 0, s>>>(a);
}

// ---------------------------------------------------------------- zeroing

// blocks of kZeroChunk elements; the batched form zeroes every run's buffer
constexpr int kZeroChunk = 8192;

template <typename real>
__global__ void __launch_bounds__(256) zero_batch_kernel(const ZeroArgs<real> *__restrict__ runs,
                                                         const int64_t *__restrict__ start, int n)
{
    __shared__ __align__(16) ZeroArgs<real> sa;
    const int64_t b = batch_block(runs, start, n, &sa);
    const int64_t lo = b * kZeroChunk;
    const int64_t hi = lo + kZeroChunk < sa.n ? lo + kZeroChunk : sa.n;
    for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) sa.p[i] = real(0);
}

template <typename real>
static void launch_zero_batch(const void *args, const int64_t *start, int n, int64_t total, unsigned *, cudaStream_t s)
{
    zero_batch_kernel<real><<<(unsigned)total, 256, 0, s>>>(static_cast<const ZeroArgs<real> *>(args), start, n);
}

template <typename real>
void launch_zero(real *p, int64_t n, cudaStream_t s)
{
    if (n <= 0) return;
    if (record_launch(kBPZero, launch_zero_batch<real>, ZeroArgs<real>{p, n}, (n + kZeroChunk - 1) / kZeroChunk))
        return;
    cudaMemsetAsync(p, 0, (size_t)n * sizeof(real), s);
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
    template void launch_yee<real>(const Geom &, real *const[9], real *const[6], double, double, double, \
                                   double, cudaStream_t);                                               \
    template void launch_filter<real>(const Geom &, real *const[3], real *, int, cudaStream_t, unsigned *); \
    template bool launch_filter_from<real>(const Geom &, const real *, real *const[3], int, cudaStream_t,  \
                                           unsigned *);                                                   \
    template void launch_window_fields<real>(const Geom &, real *const[9], real *const[9], int, cudaStream_t); \
    template void launch_antenna<real>(const Geom &, real *, int, int, double, double, double, double,  \
                                       double, double, cudaStream_t, const double *);                   \
    template void launch_field_sums<real>(const Geom &, real *const[9], double *, int, cudaStream_t); \
    template void launch_zero<real>(real *, int64_t, cudaStream_t);
PIC_FIELDS_INSTANTIATE(float)
PIC_FIELDS_INSTANTIATE(double)

// ------------------------------------------------ bounded-wait self-check

namespace {
__device__ unsigned g_wait_result;

// one CTA: an mbarrier expecting one arrival, which this kernel makes or
// withholds; the wait gives up after budget_ns
__global__ void wait_check_kernel(int arrive, uint64_t budget_ns)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_proxy_async();
    }
    __syncthreads();
    if (threadIdx.x == 0 && arrive)
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(&bar)) : "memory");
    const bool ok = mbar_wait(&bar, 0u, global_ns(), budget_ns);
    if (__syncthreads_or(!ok) && threadIdx.x == 0) g_wait_result = 1u;
}
}  // namespace

}  // namespace pic

extern "C" pic_status pic_wait_check(int arrive, double budget_ms, void *stream)
{
    if (!(budget_ms > 0.0) || budget_ms > 10000.0) return PIC_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const unsigned zero = 0u;
    if (cudaMemcpyToSymbolAsync(pic::g_wait_result, &zero, sizeof(zero), 0, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return PIC_ERR_CUDA;
    pic::wait_check_kernel<<<1, 64, 0, s>>>(arrive ? 1 : 0, (uint64_t)(budget_ms * 1e6));
    unsigned r = 0;
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyFromSymbolAsync(&r, pic::g_wait_result, sizeof(r), 0, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return PIC_ERR_CUDA;
    return r ? PIC_ERR_TIMEOUT : PIC_OK;
}
