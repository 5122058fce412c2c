// pic_fields.cu -- field kernels: Yee leapfrog with Mur boundaries, binomial
// current filter, laser antenna and the FP64 field-energy reduction.
//
// Yee (1966) on the staggered lattice of pic_internal.cuh, B split in two half
// steps so that E and B both live at integer times:
//   B -= (dt/2) curl E;   E += dt (curl B - 2 pi J);   B -= (dt/2) curl E,
// all three in one kernel that reads E^n, B^n from one field buffer and writes
// E^{n+1}, B^{n+1} to another (yee_kernel).  With absorbing z the tangential E
// (Ex, Ey) on the end planes k = 0 and k = nz follows Mur's first-order
// condition (Mur 1981).
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

// column shape of a CTA of the marching Yee kernel (3D grids; 2D grids take
// yee2d_kernel): 32 x 8 (x, y)
template <int DIM> struct YeeTile { static constexpr int TX = 32, TY = 8, HY = 1; };

// One Yee step in one pass over the grid.  A CTA owns a column of TX x TY
// nodes in (x, y) and a chunk of z planes; it marches up the chunk keeping a
// few planes of E^n, B^n, J, of the half-step B (Bh) and of E^{n+1} (E') in
// shared memory.  At plane k of the march:
//   Bh(k)   = B^n(k) - (dt/2) curl E^n      (E^n at k and k+1)
//   E'(k)   = E^n(k) + dt (curl Bh - 2 pi J) (Bh at k and k-1)
//   B'(k-1) = Bh(k-1) - (dt/2) curl E'      (E' at k-1 and k)
// while the planes the next step of the march reads (E^n(k+2), B^n(k+1),
// J(k+1)) are copied into shared memory with cp.async.  Each curl takes the
// next (x, y) neighbour on one side, so Bh is updated on the column widened
// by one node on both sides, E' widened by one node above, and neighbouring
// columns recompute the widened nodes; E' and B' of the column's own nodes
// are written to the other field buffer, so no CTA reads a value another one
// writes.  The chunk starts one plane early (the Bh plane below its first E'
// plane) and ends one plane late (the E' plane above its last B' plane).
// With absorbing z the tangential E (Ex, Ey) of the end planes follows Mur's
// first-order condition
//   E0^{n+1} = E1^n + (dt - dz)/(dt + dz) (E1^{n+1} - E0^n)
// (Mur 1981), evaluated once E' of the neighbouring plane is known.  The
// arithmetic per node is that of the split-B leapfrog written out term by
// term.  Planes a component does not have (Ez, Bx, By at k = nz; every
// component at k = nz with periodic z) are neither read nor written.
template <typename real, int DIM>
__device__ __forceinline__ void yee_body(const YeeArgs<real> &a, const int bx_, const int by_)
{
    constexpr int TX = YeeTile<DIM>::TX, TY = YeeTile<DIM>::TY, HY = YeeTile<DIM>::HY;
    constexpr int NT = 256;  // threads; every thread owns at most two nodes of each shared plane
    // shared planes: E^n on x0-1 .. x0+TX+1, y0-HY .. y0+TY-1+2HY; B^n and Bh
    // on x0-1 .. x0+TX, y0-HY .. y0+TY-1+HY; J and E' on x0 .. x0+TX,
    // y0 .. y0+TY-1+HY
    constexpr int NX0 = TX + 3, NY0 = TY + 3 * HY, P0 = NX0 * NY0;
    constexpr int NX1 = TX + 2, NY1 = TY + 2 * HY, P1 = NX1 * NY1;
    constexpr int NX2 = TX + 1, NY2 = TY + HY, P2 = NX2 * NY2;
    static_assert(P0 <= 2 * NT && TX * TY == NT, "plane regions must fit two nodes per thread");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    real *sE = reinterpret_cast<real *>(smem_raw);  // E^n: [4 planes][3 components][P0]
    real *sN = sE + 12 * P0;                         // B^n: [2][3][P1]
    real *sJ = sN + 6 * P1;                          // J:   [2][3][P2]
    real *sB = sJ + 6 * P2;                          // Bh:  [2][3][P1]
    real *sF = sB + 6 * P1;                          // E':  [3][3][P2]
    const Geom &g = a.g;
    const bool per = g.bc_z == 0;
    const int nbx = (g.nx + TX - 1) / TX;
    const int x0 = (bx_ % nbx) * TX, y0 = (bx_ / nbx) * TY;
    const int nzo = per ? g.nz : g.nz + 1;  // planes written
    const int z0 = by_ * a.cz;
    const int z1 = by_ == a.nchunks - 1 ? nzo : z0 + a.cz;
    const int kb = z0 - 1;
    const int tid = (int)threadIdx.x;
    auto r2 = [&](int k) { return (k - kb) & 1; };
    auto r3 = [&](int k) { return (k - kb) % 3; };
    auto r4 = [&](int k) { return (k - kb) & 3; };
    // plane k of a component in memory (-1: the component has no plane k)
    auto mem_plane = [&](int k, bool half) {
        return per ? wrapi(k, g.nz) : (k >= 0 && k <= zmax_of(g, half) ? k : -1);
    };
    // periodic x, y (columns of grids narrower than a CTA wrap more than once)
    auto gxw = [&](int x) { return x >= 0 && x < g.nx ? x : wrapi(x, g.nx); };
    auto gyw = [&](int y) { return DIM == 3 ? (y >= 0 && y < g.ny ? y : wrapi(y, g.ny)) : 0; };
    // this thread's nodes r = tid, tid + NT of a region (nx_ wide, np nodes,
    // origin (xo, yo)): their offsets within a plane in memory (-1: none)
    auto offs = [&](int nx_, int np, int xo, int yo, int o[2]) {
#pragma unroll
        for (int m = 0; m < 2; ++m) {
            const int r = tid + m * NT;
            const int ly = r / nx_, lx = r - ly * nx_;
            o[m] = r < np ? gyw(yo + ly) * g.nx + gxw(xo + lx) : -1;
        }
    };
    int oE[2], oB[2], oJ[2];
    offs(NX0, P0, x0 - 1, y0 - HY, oE);
    offs(NX1, P1, x0 - 1, y0 - HY, oB);
    offs(NX2, P2, x0, y0, oJ);
    // copy plane k of three components into shared memory (this thread's
    // nodes); planes a component does not have are zero
    auto fetch = [&](const real *const src[3], real *dst, int k, int np, const int o[2], bool e_half) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const int kk = mem_plane(k, e_half ? c == 2 : c != 2);
            const real *base = src[c] + (int64_t)kk * g.plane;
#pragma unroll
            for (int m = 0; m < 2; ++m) {
                if (o[m] < 0) continue;
                real *d = dst + c * np + tid + m * NT;
                if (kk >= 0) __pipeline_memcpy_async(d, base + o[m], sizeof(real));
                else *d = real(0);
            }
        }
    };
    auto fetch_all = [&](int ke, int kbj) {
        fetch(a.E, sE + r4(ke) * 3 * P0, ke, P0, oE, true);
        fetch(a.B, sN + r2(kbj) * 3 * P1, kbj, P1, oB, false);
        fetch(a.J, sJ + r2(kbj) * 3 * P2, kbj, P2, oJ, true);
    };

    // Bh(k) on its widened column
    auto half_b = [&](int k) {
        const real *e0 = sE + r4(k) * 3 * P0, *e1 = sE + r4(k + 1) * 3 * P0, *bn = sN + r2(k) * 3 * P1;
        real *dst = sB + r2(k) * 3 * P1;
        const bool vxy = mem_plane(k, true) >= 0, vz = mem_plane(k, false) >= 0;
#pragma unroll
        for (int m = 0; m < 2; ++m) {
            const int r = tid + m * NT;
            if (r >= P1) continue;
            const int ly = r / NX1, lx = r - ly * NX1;
            const int o = ly * NX0 + lx;  // the same node in the E^n plane
            real dEz_dy = 0, dEx_dy = 0;
            if (DIM == 3) {
                dEz_dy = (e0[2 * P0 + o + NX0] - e0[2 * P0 + o]) * a.ihy;
                dEx_dy = (e0[o + NX0] - e0[o]) * a.ihy;
            }
            const real dEy_dz = (e1[P0 + o] - e0[P0 + o]) * a.ihz;
            const real dEx_dz = (e1[o] - e0[o]) * a.ihz;
            const real dEz_dx = (e0[2 * P0 + o + 1] - e0[2 * P0 + o]) * a.ihx;
            const real dEy_dx = (e0[P0 + o + 1] - e0[P0 + o]) * a.ihx;
            dst[r] = vxy ? bn[r] - a.hb * (dEz_dy - dEy_dz) : real(0);
            dst[P1 + r] = vxy ? bn[P1 + r] - a.hb * (dEx_dz - dEz_dx) : real(0);
            dst[2 * P1 + r] = vz ? bn[2 * P1 + r] - a.hb * (dEy_dx - dEx_dy) : real(0);
        }
    };
    // E'(k) on its widened column (Ampere; Ex, Ey of the Mur planes are set
    // apart by the boundary condition)
    auto full_e = [&](int k) {
        const real *e0 = sE + r4(k) * 3 * P0, *jj = sJ + r2(k) * 3 * P2;
        const real *b0 = sB + r2(k) * 3 * P1, *bm = sB + r2(k - 1) * 3 * P1;
        real *dst = sF + r3(k) * 3 * P2;
        const bool vz = mem_plane(k, true) >= 0;
        const bool vxy = per || (k >= 1 && k <= g.nz - 1);
#pragma unroll
        for (int m = 0; m < 2; ++m) {
            const int r = tid + m * NT;
            if (r >= P2) continue;
            const int ly = r / NX2, lx = r - ly * NX2;
            const int ob = (ly + HY) * NX1 + lx + 1;  // the node in the Bh plane
            const int oe = (ly + HY) * NX0 + lx + 1;  // and in the E^n plane
            real dBz_dy = 0, dBx_dy = 0;
            if (DIM == 3) {
                dBz_dy = (b0[2 * P1 + ob] - b0[2 * P1 + ob - NX1]) * a.ihy;
                dBx_dy = (b0[ob] - b0[ob - NX1]) * a.ihy;
            }
            if (vxy) {
                const real dBy_dz = (b0[P1 + ob] - bm[P1 + ob]) * a.ihz;
                dst[r] = e0[oe] + a.he * ((dBz_dy - dBy_dz) - a.twopi * jj[r]);
                const real dBx_dz = (b0[ob] - bm[ob]) * a.ihz;
                const real dBz_dx = (b0[2 * P1 + ob] - b0[2 * P1 + ob - 1]) * a.ihx;
                dst[P2 + r] = e0[P0 + oe] + a.he * ((dBx_dz - dBz_dx) - a.twopi * jj[P2 + r]);
            }
            const real dBy_dx = (b0[P1 + ob] - b0[P1 + ob - 1]) * a.ihx;
            dst[2 * P2 + r] = vz ? e0[2 * P0 + oe] + a.he * ((dBy_dx - dBx_dy) - a.twopi * jj[2 * P2 + r]) : real(0);
        }
    };
    // Mur: Ex, Ey of plane kt from plane kn (its neighbour inside the box)
    auto mur = [&](int kt, int kn) {
        const real *et = sE + r4(kt) * 3 * P0, *en = sE + r4(kn) * 3 * P0;
        const real *fn = sF + r3(kn) * 3 * P2;
        real *ft = sF + r3(kt) * 3 * P2;
#pragma unroll
        for (int m = 0; m < 2; ++m) {
            const int r = tid + m * NT;
            if (r >= P2) continue;
            const int ly = r / NX2, lx = r - ly * NX2;
            const int oe = (ly + HY) * NX0 + lx + 1;
            ft[r] = en[oe] + a.mur * (fn[r] - et[oe]);
            ft[P2 + r] = en[P0 + oe] + a.mur * (fn[P2 + r] - et[P0 + oe]);
        }
    };
    // B'(k) and E'(k) of the column's own node of this thread to memory
    const int lxo = tid % TX, lyo = tid / TX;
    const bool own = x0 + lxo < g.nx && (DIM == 2 || y0 + lyo < g.ny);
    const int64_t oxy = own ? (int64_t)(y0 + lyo) * g.nx + (x0 + lxo) : 0;
    auto write_out = [&](int k) {
        if (!own) return;
        const real *b0 = sB + r2(k) * 3 * P1;
        const real *f0 = sF + r3(k) * 3 * P2, *f1 = sF + r3(k + 1) * 3 * P2;
        const int64_t o = (int64_t)k * g.plane + oxy;
        const int of = lyo * NX2 + lxo;               // the node in the E' plane
        const int ob = (lyo + HY) * NX1 + lxo + 1;    // and in the Bh plane
        const bool vxy = k <= zmax_of(g, false), vz = k <= zmax_of(g, true);
        if (vxy) {
            a.E1[0][o] = f0[of];
            a.E1[1][o] = f0[P2 + of];
        }
        if (vz) {
            a.E1[2][o] = f0[2 * P2 + of];
            real dEz_dy = 0;
            if (DIM == 3) dEz_dy = (f0[2 * P2 + of + NX2] - f0[2 * P2 + of]) * a.ihy;
            const real dEy_dz = (f1[P2 + of] - f0[P2 + of]) * a.ihz;
            a.B1[0][o] = b0[ob] - a.hb * (dEz_dy - dEy_dz);
            const real dEx_dz = (f1[of] - f0[of]) * a.ihz;
            const real dEz_dx = (f0[2 * P2 + of + 1] - f0[2 * P2 + of]) * a.ihx;
            a.B1[1][o] = b0[P1 + ob] - a.hb * (dEx_dz - dEz_dx);
        }
        if (vxy) {
            const real dEy_dx = (f0[P2 + of + 1] - f0[P2 + of]) * a.ihx;
            real dEx_dy = 0;
            if (DIM == 3) dEx_dy = (f0[of + NX2] - f0[of]) * a.ihy;
            a.B1[2][o] = b0[2 * P1 + ob] - a.hb * (dEy_dx - dEx_dy);
        }
    };

    fetch(a.E, sE + r4(kb) * 3 * P0, kb, P0, oE, true);
    fetch_all(kb + 1, kb);
    __pipeline_commit();
    for (int k = kb; k <= z1; ++k) {
        // the planes the next step reads, while this one is computed
        fetch_all(k + 2, k + 1);
        __pipeline_commit();
        __pipeline_wait_prior(1);
        __syncthreads();
        half_b(k);
        __syncthreads();
        if (k >= z0) {
            full_e(k);
            __syncthreads();
            if (!per && (k == 1 || k == g.nz - 1)) {
                if (k == 1) mur(0, 1);
                if (k == g.nz - 1) mur(g.nz, g.nz - 1);
                __syncthreads();
            }
        }
        if (k >= z0 + 1) write_out(k - 1);
    }
    __pipeline_wait_prior(0);
}

template <typename real, int DIM>
__global__ void __launch_bounds__(256) yee_kernel(YeeArgs<real> a)
{
    yee_body<real, DIM>(a, (int)blockIdx.x, (int)blockIdx.y);
}

// CTAs of one z column chunk per run of a batch: block b of run r is column
// b % ncol, chunk b / ncol
template <typename real, int DIM>
__global__ void __launch_bounds__(256) yee_batch_kernel(const YeeArgs<real> *__restrict__ runs,
                                                        const int64_t *__restrict__ start, int n)
{
    __shared__ __align__(16) YeeArgs<real> sa;
    const int64_t b = batch_block(runs, start, n, &sa);
    constexpr int TX = YeeTile<DIM>::TX, TY = YeeTile<DIM>::TY;
    const int ncol = ((sa.g.nx + TX - 1) / TX) * (DIM == 3 ? (sa.g.ny + TY - 1) / TY : 1);
    yee_body<real, DIM>(sa, (int)(b % ncol), (int)(b / ncol));
}

// ------------------------------------------------------- 2D tiled Yee

// Shared rows of the 2D tile kernels: x from x0 - 4 to x0 + 67 of a tile
// whose own columns are x0 .. x0 + 63 (x0 a multiple of 64), kRowPitch
// elements per row, so that every 16-byte chunk of a row is a 16-byte chunk
// of the grid row (where the grid width is a multiple of 16 bytes).
constexpr int kRowX = 64, kRowPitch = 72, kRowOrigin = 4;

// Copies rows zo .. zo + nrows - 1 of one component into dst[row][x - x0 + 4]
// with cp.async: 16-byte copies for the chunks inside the grid, element
// copies (x wrapped) for the chunks across its periodic x edge; a row the
// component does not have (plane(k) < 0) is zero.
template <typename real, typename PlaneFn>
__device__ __forceinline__ void stage_rows(real *dst, const real *src, int nrows, int zo, int x0, const Geom &g,
                                           PlaneFn plane)
{
    constexpr int V = 16 / (int)sizeof(real), NCH = kRowPitch / V;
    const bool vec = g.nx % V == 0 && (reinterpret_cast<uintptr_t>(src) & 15u) == 0;
    for (int q = (int)threadIdx.x; q < nrows * NCH; q += (int)blockDim.x) {
        const int row = q / NCH, ch = q - row * NCH;
        const int kk = plane(zo + row);
        real *d = dst + row * kRowPitch + ch * V;
        const int xs = x0 - kRowOrigin + ch * V;
        if (kk < 0) {
#pragma unroll
            for (int v = 0; v < V; ++v) d[v] = real(0);
            continue;
        }
        const real *srow = src + (int64_t)kk * g.plane;
        if (vec && xs >= 0 && xs + V <= g.nx) {
            __pipeline_memcpy_async(d, srow + xs, 16);
        } else {
#pragma unroll
            for (int v = 0; v < V; ++v) __pipeline_memcpy_async(d + v, srow + wrapi(xs + v, g.nx), sizeof(real));
        }
    }
}

// The same Yee step on 2D grids, without the march: a CTA owns a tile of
// 64 x kY2Z (x, z) nodes and copies, all at once with cp.async (above),
// x0 - 4 .. x0 + 67 of E^n on planes z0 - 2 .. z0 + kY2Z + 1, of B^n on
// z0 - 2 .. z0 + kY2Z and of J on z0 - 1 .. z0 + kY2Z into shared memory
// (planes a component does not have are zero), so that a tile costs one load
// latency however narrow the grid is (the march pays one per plane, which
// dominates on grids a few hundred nodes wide).  Then, in shared memory and
// node by node with the march's arithmetic: Bh in place of B^n on
// x0 - 1 .. x0 + 64, E' in place of E^n on x0 .. x0 + 64, z0 - 1 .. z0 + kY2Z,
// Mur's condition for the end planes (from the saved E^n of their inner
// neighbours), and E', B' of the own nodes to the other buffer.  (d/dy = 0:
// the y derivatives of the 3D formulas are zero terms.)
constexpr int kY2Z = 16;
constexpr int kY2EZ = kY2Z + 4, kY2BZ = kY2Z + 3, kY2JZ = kY2Z + 2;  // rows of E^n, B^n, J

template <typename real>
__device__ __forceinline__ void yee2d_body(const YeeArgs<real> &a, const int bx_, const int bz_)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int W = kRowPitch;
    constexpr int PE = kY2EZ * W, PB = kY2BZ * W, PJ = kY2JZ * W;
    real *sE = reinterpret_cast<real *>(smem_raw);  // [3][kY2EZ][W], E^n then E'
    real *sB = sE + 3 * PE;                          // [3][kY2BZ][W], B^n then Bh
    real *sJ = sB + 3 * PB;                          // [3][kY2JZ][W]
    real *sM = sJ + 3 * PJ;                          // [2 ends][2 comps][W]: E^n x, y of planes 1, nz-1
    const Geom &g = a.g;
    const bool per = g.bc_z == 0;
    const int nzo = per ? g.nz : g.nz + 1;
    const int x0 = bx_ * kRowX, z0 = bz_ * kY2Z;
    const int z1 = z0 + kY2Z < nzo ? z0 + kY2Z : nzo;
    const int tid = (int)threadIdx.x, nt = (int)blockDim.x;
    auto plane_of = [&](bool half) {
        return [&g, per, half](int k) { return per ? wrapi(k, g.nz) : (k >= 0 && k <= zmax_of(g, half) ? k : -1); };
    };
    const auto pint = plane_of(false), phalf = plane_of(true);
    // ---- copy E^n (Ez half-z), B^n (Bx, By half-z), J (Jz half-z)
    stage_rows(sE, a.E[0], kY2EZ, z0 - 2, x0, g, pint);
    stage_rows(sE + PE, a.E[1], kY2EZ, z0 - 2, x0, g, pint);
    stage_rows(sE + 2 * PE, a.E[2], kY2EZ, z0 - 2, x0, g, phalf);
    stage_rows(sB, a.B[0], kY2BZ, z0 - 2, x0, g, phalf);
    stage_rows(sB + PB, a.B[1], kY2BZ, z0 - 2, x0, g, phalf);
    stage_rows(sB + 2 * PB, a.B[2], kY2BZ, z0 - 2, x0, g, pint);
    stage_rows(sJ, a.J[0], kY2JZ, z0 - 1, x0, g, pint);
    stage_rows(sJ + PJ, a.J[1], kY2JZ, z0 - 1, x0, g, pint);
    stage_rows(sJ + 2 * PJ, a.J[2], kY2JZ, z0 - 1, x0, g, phalf);
    __pipeline_commit();
    __pipeline_wait_prior(0);
    __syncthreads();
    // the E^n of the planes Mur's condition reads after E' has replaced them
    const bool mur_lo = !per && z0 - 1 <= 0 && 0 <= z0 + kY2Z - 1;        // plane 0 is computed here
    const bool mur_hi = !per && z0 - 1 <= g.nz - 1 && g.nz <= z0 + kY2Z;  // plane nz too
    if (mur_lo || mur_hi) {
        for (int r = tid; r < 2 * 2 * W; r += nt) {
            const int end = r / (2 * W), c = (r / W) & 1, j = r % W;
            const int pz = (end == 0 ? 1 : g.nz - 1) - (z0 - 2);
            sM[r] = (pz >= 0 && pz < kY2EZ) ? sE[c * PE + pz * W + j] : real(0);
        }
    }
    // ---- Bh(k) = B^n(k) - (dt/2) curl E^n on every B row, x0 - 1 .. x0 + 64
    const real zero = real(0);
    {
        constexpr int NX = kRowX + 2;
        for (int r = tid; r < kY2BZ * NX; r += nt) {
            const int pb = r / NX, j = r - pb * NX + kRowOrigin - 1;
            const int k = z0 - 2 + pb;
            const int o = pb * W + j;  // the same index in the E and B rows
            const bool vxy = phalf(k) >= 0, vz = pint(k) >= 0;
            const real dEy_dz = (sE[PE + o + W] - sE[PE + o]) * a.ihz;
            const real dEx_dz = (sE[o + W] - sE[o]) * a.ihz;
            const real dEz_dx = (sE[2 * PE + o + 1] - sE[2 * PE + o]) * a.ihx;
            const real dEy_dx = (sE[PE + o + 1] - sE[PE + o]) * a.ihx;
            sB[o] = vxy ? sB[o] - a.hb * (zero - dEy_dz) : real(0);
            sB[PB + o] = vxy ? sB[PB + o] - a.hb * (dEx_dz - dEz_dx) : real(0);
            sB[2 * PB + o] = vz ? sB[2 * PB + o] - a.hb * (dEy_dx - zero) : real(0);
        }
    }
    __syncthreads();
    // ---- E'(k) = E^n(k) + dt (curl Bh - 2 pi J) on x0 .. x0 + 64, z0 - 1 .. z0 + kY2Z
    {
        constexpr int NX = kRowX + 1;
        for (int r = tid; r < kY2JZ * NX; r += nt) {
            const int lz = r / NX, j = r - lz * NX + kRowOrigin;
            const int k = z0 - 1 + lz;
            const int o = (lz + 1) * W + j;  // in the E and B rows
            const int oj = lz * W + j;
            const bool vz = phalf(k) >= 0;
            const bool vxy = per || (k >= 1 && k <= g.nz - 1);
            if (vxy) {
                const real dBy_dz = (sB[PB + o] - sB[PB + o - W]) * a.ihz;
                sE[o] = sE[o] + a.he * ((zero - dBy_dz) - a.twopi * sJ[oj]);
                const real dBx_dz = (sB[o] - sB[o - W]) * a.ihz;
                const real dBz_dx = (sB[2 * PB + o] - sB[2 * PB + o - 1]) * a.ihx;
                sE[PE + o] = sE[PE + o] + a.he * ((dBx_dz - dBz_dx) - a.twopi * sJ[PJ + oj]);
            }
            const real dBy_dx = (sB[PB + o] - sB[PB + o - 1]) * a.ihx;
            sE[2 * PE + o] = vz ? sE[2 * PE + o] + a.he * ((dBy_dx - zero) - a.twopi * sJ[2 * PJ + oj]) : real(0);
        }
    }
    __syncthreads();
    // ---- Mur: Ex, Ey of plane kt from plane kn, its neighbour inside the box
    if (mur_lo || mur_hi) {
        for (int r = tid; r < 2 * (kRowX + 1); r += nt) {
            const int end = r / (kRowX + 1), j = r % (kRowX + 1) + kRowOrigin;
            if (end == 0 ? !mur_lo : !mur_hi) continue;
            const int kt = end == 0 ? 0 : g.nz, kn = end == 0 ? 1 : g.nz - 1;
            const int ot = (kt - (z0 - 2)) * W + j, on = (kn - (z0 - 2)) * W + j;
            const real *old = sM + end * 2 * W;  // E^n of plane kn
#pragma unroll
            for (int c = 0; c < 2; ++c)
                sE[c * PE + ot] = old[c * W + j] + a.mur * (sE[c * PE + on] - sE[c * PE + ot]);
        }
        __syncthreads();
    }
    // ---- E', B' of the own nodes
    for (int r = tid; r < kRowX * kY2Z; r += nt) {
        const int lz = r / kRowX, lx = r - lz * kRowX;
        const int k = z0 + lz, x = x0 + lx;
        if (k >= z1 || x >= g.nx) continue;
        const int of = (lz + 2) * W + lx + kRowOrigin;  // in the E and B rows
        const int64_t o = (int64_t)k * g.plane + x;
        const bool vxy = k <= zmax_of(g, false), vz = k <= zmax_of(g, true);
        if (vxy) {
            a.E1[0][o] = sE[of];
            a.E1[1][o] = sE[PE + of];
        }
        if (vz) {
            a.E1[2][o] = sE[2 * PE + of];
            const real dEy_dz = (sE[PE + of + W] - sE[PE + of]) * a.ihz;
            a.B1[0][o] = sB[of] - a.hb * (zero - dEy_dz);
            const real dEx_dz = (sE[of + W] - sE[of]) * a.ihz;
            const real dEz_dx = (sE[2 * PE + of + 1] - sE[2 * PE + of]) * a.ihx;
            a.B1[1][o] = sB[PB + of] - a.hb * (dEx_dz - dEz_dx);
        }
        if (vxy) {
            const real dEy_dx = (sE[PE + of + 1] - sE[PE + of]) * a.ihx;
            a.B1[2][o] = sB[2 * PB + of] - a.hb * (dEy_dx - zero);
        }
    }
}

template <typename real>
__global__ void __launch_bounds__(256) yee2d_kernel(YeeArgs<real> a)
{
    yee2d_body(a, (int)blockIdx.x, (int)blockIdx.y);
}

// (YeeArgs::nchunks holds the tiles along x here)
template <typename real>
__global__ void __launch_bounds__(256) yee2d_batch_kernel(const YeeArgs<real> *__restrict__ runs,
                                                          const int64_t *__restrict__ start, int n)
{
    __shared__ __align__(16) YeeArgs<real> sa;
    const int64_t b = batch_block(runs, start, n, &sa);
    yee2d_body(sa, (int)(b % sa.nchunks), (int)(b / sa.nchunks));
}

template <typename real>
static size_t yee2d_smem()
{
    return sizeof(real) * (size_t)kRowPitch * (3 * (kY2EZ + kY2BZ + kY2JZ) + 4);
}

template <typename real>
static void launch_yee2d_batch(const void *args, const int64_t *start, int n, int64_t total, unsigned *,
                               cudaStream_t s)
{
    const size_t smem = yee2d_smem<real>();
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(yee2d_batch_kernel<real>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    yee2d_batch_kernel<real><<<(unsigned)total, 256, smem, s>>>(static_cast<const YeeArgs<real> *>(args), start, n);
}

template <typename real, int DIM>
static size_t yee_smem()
{
    constexpr int TX = YeeTile<DIM>::TX, TY = YeeTile<DIM>::TY, HY = YeeTile<DIM>::HY;
    // E^n 4 planes, B^n and Bh 2 each, J 2, E' 3 (three components each)
    return sizeof(real) * 3 *
           (4 * (size_t)(TX + 3) * (TY + 3 * HY) + 4 * (size_t)(TX + 2) * (TY + 2 * HY) +
            5 * (size_t)(TX + 1) * (TY + HY));
}

template <typename real, int DIM>
static void launch_yee_batch(const void *args, const int64_t *start, int n, int64_t total, unsigned *, cudaStream_t s)
{
    const size_t smem = yee_smem<real, DIM>();
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(yee_batch_kernel<real, DIM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    yee_batch_kernel<real, DIM><<<(unsigned)total, 256, smem, s>>>(static_cast<const YeeArgs<real> *>(args), start, n);
}

static unsigned grid_for(int64_t n, int block)
{
    int64_t b = (n + block - 1) / block;
    const int64_t cap = 152LL * 32;
    return (unsigned)(b < cap ? (b > 0 ? b : 1) : cap);
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
        const int ntx = (g.nx + kRowX - 1) / kRowX, ntz = (nzo + kY2Z - 1) / kY2Z;
        a.cz = kY2Z;
        a.nchunks = ntx;
        if (record_launch(kBPYee, launch_yee2d_batch<real>, a, (int64_t)ntx * ntz)) return;
        const size_t smem = yee2d_smem<real>();
        if (smem > 48 * 1024)
            cudaFuncSetAttribute(yee2d_kernel<real>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        yee2d_kernel<real><<<dim3((unsigned)ntx, (unsigned)ntz), 256, smem, s>>>(a);
        return;
    }
    constexpr int TX = YeeTile<3>::TX, TY = YeeTile<3>::TY;
    // chunks of 4..32 planes, as long as there are about eight CTAs per SM;
    // the last chunk takes the remainder
    if (nzo < 8) {
        a.cz = nzo;
    } else {
        const int64_t ncol = (int64_t)((g.nx + TX - 1) / TX) * ((g.ny + TY - 1) / TY);
        int64_t czl = (int64_t)nzo * ncol * batch_runs() / ((int64_t)device_sms() * 8);
        a.cz = (int)(czl < 4 ? 4 : (czl > 32 ? 32 : czl));
    }
    a.nchunks = nzo / a.cz;
    if (a.nchunks < 1) a.nchunks = 1;
    const size_t smem = yee_smem<real, 3>();
    const unsigned nb = (unsigned)(((g.nx + TX - 1) / TX) * ((g.ny + TY - 1) / TY));
    if (record_launch(kBPYee, launch_yee_batch<real, 3>, a, (int64_t)nb * a.nchunks)) return;
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(yee_kernel<real, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    yee_kernel<real, 3><<<dim3(nb, (unsigned)a.nchunks), 256, smem, s>>>(a);
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
// filter_march_kernel.  A stage whose copy does not land within the wait
// budget stops the CTA and records ERR_TIMEOUT.
constexpr int kFilterStages = 4;

template <typename real, int H>
__global__ void __launch_bounds__(256) filter_tma_kernel(const __grid_constant__ CUtensorMap map, Geom g,
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
    constexpr int NXP = (3 * XR + 255) / 256;    // of them per thread
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
    real lev[3][H + 1][3];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int p = 0; p <= H; ++p) lev[c][p][0] = lev[c][p][1] = lev[c][p][2] = real(0);
    int q = 0;
    for (; q < np; ++q) {
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
        if (__syncthreads_or(!ok)) break;  // the CTA stops together
        // x passes over the widened rows
#pragma unroll
        for (int n = 0; n < NXP; ++n) {
            const int idx = tid + 256 * n;
            if (idx < 3 * XR) {
                const int c = idx / XR, rr = idx - c * XR, row = rr / TX, col = rr - row * TX;
                const real *A = S + c * PN + row * BX + col + XO;
                real v = 0;
#pragma unroll
                for (int i = 0; i < W; ++i) v += wb[i] * A[i];
                xs[idx] = v;
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
                out[(size_t)c * g.ncomp + (int64_t)ko * g.plane + oown] = ko > zmax ? real(0) : lev[c][H][2];
        }
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
    int64_t czl = (int64_t)nzo * nb / (152 * 8);
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

// The same H passes on 2D grids, without the march: a CTA owns 64 x kF2Z
// (x, z) nodes of the three components and copies, all at once with
// cp.async (stage_rows), x0 - 4 .. x0 + 67 of their input on planes
// z0 - H .. z0 + kF2Z + H - 1 (zero or wrapped beyond the grid); per
// component, the x passes are the binomial stencil of width 2H + 1
// (filter_march_kernel's sum), and the z passes follow one level at a time in
// shared memory, each narrower by a plane on both sides and zero outside the
// component's z range, as in the march.
constexpr int kF2Z = 32;

template <typename real, int H>
__device__ __forceinline__ void filter2d_body(const Geom &g, const real *in, real *out, const int bx_, const int bz_)
{
    static_assert(H <= kRowOrigin, "the halo fits the staged rows");
    constexpr int W = kRowPitch, IZ = kF2Z + 2 * H, PI = IZ * W, PL = kRowX * IZ;
    constexpr int NW = 2 * H + 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    real *sI = reinterpret_cast<real *>(smem_raw);  // [3][IZ][W] input
    real *sL = sI + 3 * PI;                          // [2][IZ][64] levels (ping-pong)
    real wb[NW];
    {
        double c = 1.0;
        for (int i = 0; i < NW; ++i) {
            wb[i] = (real)(c / (double)(1 << (2 * H)));
            c = c * (double)(2 * H - i) / (double)(i + 1);
        }
    }
    const bool per = g.bc_z == 0;
    const int x0 = bx_ * kRowX, z0 = bz_ * kF2Z;
    const int tid = (int)threadIdx.x, nt = (int)blockDim.x;
    const int zmax_xy = zmax_of(g, false), zmax_z = zmax_of(g, true);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const int zmax = c == 2 ? zmax_z : zmax_xy;
        stage_rows(sI + c * PI, in + (size_t)c * g.ncomp, IZ, z0 - H, x0, g,
                   [&g, per, zmax](int k) { return per ? wrapi(k, g.nz) : (k >= 0 && k <= zmax ? k : -1); });
    }
    __pipeline_commit();
    __pipeline_wait_prior(0);
    __syncthreads();
#pragma unroll 1
    for (int c = 0; c < 3; ++c) {
        const int zmax = c == 2 ? zmax_z : zmax_xy;
        const real *I = sI + c * PI;
        real *L0 = sL, *L1 = sL + PL;
        // level 0: the x stencil on every staged plane
        for (int r = tid; r < PL; r += nt) {
            const int pz = r / kRowX, lx = r - pz * kRowX;
            const int k = z0 - H + pz;
            real v = 0;
#pragma unroll
            for (int i = 0; i < NW; ++i) v += wb[i] * I[pz * W + lx + kRowOrigin - H + i];
            L0[r] = (per || (k >= 0 && k <= zmax)) ? v : real(0);
        }
        __syncthreads();
        // level p on planes p .. IZ - 1 - p of the staged range
#pragma unroll
        for (int p = 1; p <= H; ++p) {
            for (int r = tid; r < PL; r += nt) {
                const int pz = r / kRowX;
                if (pz < p || pz >= IZ - p) continue;
                const int k = z0 - H + pz;
                const real nv = real(0.25) * L0[r - kRowX] + real(0.5) * L0[r] + real(0.25) * L0[r + kRowX];
                L1[r] = (per || (k >= 0 && k <= zmax)) ? nv : real(0);
            }
            __syncthreads();
            real *t = L0;
            L0 = L1;
            L1 = t;
        }
        for (int r = tid; r < kRowX * kF2Z; r += nt) {
            const int lz = r / kRowX, lx = r - lz * kRowX;
            const int k = z0 + lz, x = x0 + lx;
            if (k > g.nz || x >= g.nx) continue;
            out[(size_t)c * g.ncomp + (int64_t)k * g.plane + x] = k > zmax ? real(0) : L0[(lz + H) * kRowX + lx];
        }
        __syncthreads();
    }
}

template <typename real, int H>
__global__ void __launch_bounds__(256) filter2d_kernel(Geom g, const real *in, real *out)
{
    filter2d_body<real, H>(g, in, out, (int)blockIdx.x, (int)blockIdx.y);
}

// (MarchArgs::cz holds the tiles along x here)
template <typename real, int H>
__global__ void __launch_bounds__(256) filter2d_batch_kernel(const MarchArgs<real> *__restrict__ runs,
                                                             const int64_t *__restrict__ start, int n)
{
    __shared__ __align__(16) MarchArgs<real> sa;
    const int64_t b = batch_block(runs, start, n, &sa);
    filter2d_body<real, H>(sa.g, sa.in, sa.out, (int)(b % sa.cz), (int)(b / sa.cz));
}

template <typename real, int H>
static size_t filter2d_smem()
{
    return sizeof(real) * (3 * (size_t)kRowPitch * (kF2Z + 2 * H) + 2 * (size_t)kRowX * (kF2Z + 2 * H));
}

template <typename real, int H>
static void launch_filter2d_batch(const void *args, const int64_t *start, int n, int64_t total, unsigned *,
                                  cudaStream_t s)
{
    const size_t smem = filter2d_smem<real, H>();
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(filter2d_batch_kernel<real, H>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    filter2d_batch_kernel<real, H>
        <<<(unsigned)total, 256, smem, s>>>(static_cast<const MarchArgs<real> *>(args), start, n);
}

template <typename real, int DIM, int H>
static void launch_march(const Geom &g, const real *in, real *out, cudaStream_t s)
{
    const int nzo = g.nz + 1;
    if constexpr (DIM == 2) {
        // the tiled kernel (2D grids)
        const int ntx = (g.nx + kRowX - 1) / kRowX, ntz = (nzo + kF2Z - 1) / kF2Z;
        if (record_launch(kBPFilter, launch_filter2d_batch<real, H>, MarchArgs<real>{g, in, out, ntx, ntz},
                          (int64_t)ntx * ntz))
            return;
        const size_t smem = filter2d_smem<real, H>();
        if (smem > 48 * 1024)
            cudaFuncSetAttribute(filter2d_kernel<real, H>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        filter2d_kernel<real, H><<<dim3((unsigned)ntx, (unsigned)ntz), 256, smem, s>>>(g, in, out);
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
