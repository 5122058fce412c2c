// pic_particles.cu -- particle kernels of a single run: fused gather / Boris
// push / Esirkepov deposit / re-bucketing per tile (bodies in pic_push.cuh),
// the drifting-ion deposit, bucketing of flat lists, compaction, charge
// density and particle sums.
#include "pic_push.cuh"

namespace pic {

template <typename real, int DIM, int S, int TX, int TY, int TZ, bool REL>
__global__ void __launch_bounds__(kBlock, MinBlocks<real>::value) push_kernel(PushArgs<real> a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    for (int64_t t = blockIdx.x; t < a.g.ntiles; t += gridDim.x) push_tile<real, DIM, S, TX, TY, TZ, REL>(a, t, smem_raw);
}

// ----------------------------------------------------- drifting-ion kernel

template <typename real, int DIM, int S, int TX, int TY, int TZ, bool REL>
__global__ void __launch_bounds__(kBlock) ion_kernel(PushArgs<real> a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    for (int64_t t = blockIdx.x; t < a.g.ntiles; t += gridDim.x) ion_tile<real, DIM, S, TX, TY, TZ, REL>(a, t, smem_raw);
}

template <typename real, int DIM, int S, int TX, int TY, int TZ, bool REL>
static void launch_push_z(const PushArgs<real> &a, bool ions, cudaStream_t s)
{
    if (ions ? record_launch(kBPIons, launch_push_batch<real, DIM, S, TX, TY, TZ, REL, true>, a, a.g.ntiles, true)
             : record_launch(kBPPush, launch_push_batch<real, DIM, S, TX, TY, TZ, REL, false>, a, a.g.ntiles, true))
        return;
    const size_t smem = push_smem<real, DIM, S, TX, TY, TZ, REL>(ions);
    auto k = ions ? ion_kernel<real, DIM, S, TX, TY, TZ, REL> : push_kernel<real, DIM, S, TX, TY, TZ, REL>;
    if (smem > 48 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const int64_t grid = a.g.ntiles < 2147483647LL ? a.g.ntiles : 2147483647LL;
    k<<<(unsigned)grid, kBlock, smem, s>>>(a);
}

// records in relative form (and their ions) take the REL kernels
template <typename real, int DIM, int S, int TX, int TY, int TZ>
static void launch_push_t(const PushArgs<real> &a, bool ions, cudaStream_t s)
{
    if (a.rel) launch_push_z<real, DIM, S, TX, TY, TZ, true>(a, ions, s);
    else launch_push_z<real, DIM, S, TX, TY, TZ, false>(a, ions, s);
}

template <typename real>
static void dispatch_push(const PushArgs<real> &a, bool ions, cudaStream_t s)
{
    if (a.g.dim == 3) {
        if (a.g.shape == 2) launch_push_t<real, 3, 2, kTile3[0], kTile3[1], kTile3[2]>(a, ions, s);
        else if (a.g.lt[2] == 2) launch_push_t<real, 3, 1, 8, 8, 4>(a, ions, s);  // 8 x 8 x 4
        else launch_push_t<real, 3, 1, kTile3[0], kTile3[1], kTile3[2]>(a, ions, s);
    } else if (a.g.shape == 2) {
        launch_push_t<real, 2, 2, kTile2[0], kTile2[1], kTile2[2]>(a, ions, s);
    } else if (a.g.lt[0] == 5) {  // 32 x 8
        launch_push_t<real, 2, 1, 32, 1, 8>(a, ions, s);
    } else if (a.g.lt[0] == 3) {  // 8 x 32
        launch_push_t<real, 2, 1, 8, 1, 32>(a, ions, s);
    } else {
        launch_push_t<real, 2, 1, kTile2[0], kTile2[1], kTile2[2]>(a, ions, s);
    }
}

template <typename real> void launch_push(const PushArgs<real> &a, cudaStream_t s) { dispatch_push(a, false, s); }
template <typename real> void launch_ions(const PushArgs<real> &a, cudaStream_t s) { dispatch_push(a, true, s); }

// --------------------------------------------------------- moving window

// One CTA per output tile: it copies the bucket of the input tile m layers
// above (same slots, both runs) with the cell index S = m tz lower; the top m
// layers are left empty and the bottom m layers of the input are dropped.
template <typename real>
__global__ void window_particles_kernel(Geom g, Species<real> in, Species<real> out, const int *in_lo,
                                        const int *in_hi, int *out_lo, int *out_hi, int m, int S)
{
    const int64_t ntxy = (int64_t)g.nt[0] * g.nt[1];
    const int64_t t = blockIdx.x;
    const int64_t tz = t / ntxy;
    int n_lo = 0, n_hi = 0;
    if (tz + m < g.nt[2]) bucket_counts(in_lo, in_hi, t + m * ntxy, g.cap, n_lo, n_hi, nullptr);
    if (threadIdx.x == 0) {
        out_lo[t] = n_lo;
        out_hi[t] = n_hi;
    }
    const int n = n_lo + n_hi;
    const uint32_t dk = (uint32_t)S << (g.bx + g.by);
    for (int p = threadIdx.x; p < n; p += blockDim.x) {
        const int64_t d = bucket_slot(t, g.cap, n_lo, n_hi, p);
        const int64_t s = d + m * ntxy * (int64_t)g.cap;
        out.ox[d] = in.ox[s];
        if (g.dim == 3) out.oy[d] = in.oy[s];
        out.oz[d] = in.oz[s];
        out.w[d] = in.w[s];
        if (in.ux) {
            out.ux[d] = in.ux[s];
            out.uy[d] = in.uy[s];
            out.uz[d] = in.uz[s];
        }
        if (in.dlx) {
            out.dlx[d] = in.dlx[s];
            if (in.dly) out.dly[d] = in.dly[s];
            out.dlz[d] = in.dlz[s];
        }
        out.cell[d] = (int32_t)((uint32_t)in.cell[s] - dk);  // keeps the pair bit
        if (in.id) out.id[d] = in.id[s];
    }
}

template <typename real>
void launch_window_particles(const Geom &g, const Species<real> &in, const Species<real> &out, const int *in_lo,
                             const int *in_hi, int *out_lo, int *out_hi, int m, int S, cudaStream_t s)
{
    window_particles_kernel<real><<<(unsigned)g.ntiles, 256, 0, s>>>(g, in, out, in_lo, in_hi, out_lo, out_hi, m, S);
}

// ------------------------------------------------------ bucket / compact

template <typename real>
__global__ void bucket_kernel(BucketArgs<real> a)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t nround = (a.n + 31) / 32 * 32;  // whole warps iterate together
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nround; p += stride) {
        int64_t dest = -1;
        int ci = 0, cj = 0, ck = 0;
        if (p < a.n) {
            unpack_cell(a.g, a.src.cell[p], ci, cj, ck);
            dest = tile_of(a.g, ci, cj, ck);
        }
        const int r = reserve_slot(a.dst_hi, dest);
        if (dest < 0) continue;
        if (r >= a.g.cap) {
            atomicOr(a.err, ERR_CAPACITY);
            continue;
        }
        const int64_t d = dest * (int64_t)a.g.cap + (a.g.cap - 1 - r);
        a.dst.ox[d] = a.src.ox[p];
        if (a.dst.oy) a.dst.oy[d] = a.src.oy[p];
        a.dst.oz[d] = a.src.oz[p];
        a.dst.w[d] = a.src.w[p];
        if (a.dst.ux) {
            a.dst.ux[d] = a.src.ux[p];
            a.dst.uy[d] = a.src.uy[p];
            a.dst.uz[d] = a.src.uz[p];
        }
        if (a.dst.dlx) {
            a.dst.dlx[d] = a.src.dlx[p];
            if (a.dst.dly) a.dst.dly[d] = a.src.dly[p];
            a.dst.dlz[d] = a.src.dlz[p];
        }
        a.dst.cell[d] = a.src.cell[p];
        if (a.dst.id) a.dst.id[d] = a.src.id ? a.src.id[p] : 0;
    }
}

template <typename real>
void launch_bucket(const BucketArgs<real> &a, cudaStream_t s)
{
    if (a.n <= 0) return;
    int64_t blocks = (a.n + 255) / 256;
    if (blocks > (int64_t)device_sms() * 64) blocks = (int64_t)device_sms() * 64;
    bucket_kernel<real><<<(unsigned)blocks, 256, 0, s>>>(a);
}

template <typename real>
__global__ void compact_kernel(CompactArgs<real> a)
{
    for (int64_t t = blockIdx.x; t < a.g.ntiles; t += gridDim.x) {
        int n_lo, n_hi;
        bucket_counts(a.lo, a.hi, t, a.g.cap, n_lo, n_hi, nullptr);
        const int n = n_lo + n_hi;
        const int64_t o = a.offset[t];
        for (int p = threadIdx.x; p < n; p += blockDim.x) {
            const int64_t s = bucket_slot(t, a.g.cap, n_lo, n_hi, p), d = o + p;
            a.dst.ox[d] = a.src.ox[s];
            if (a.src.oy) a.dst.oy[d] = a.src.oy[s];
            a.dst.oz[d] = a.src.oz[s];
            a.dst.w[d] = a.src.w[s];
            if (a.src.ux) {
                a.dst.ux[d] = a.src.ux[s];
                a.dst.uy[d] = a.src.uy[s];
                a.dst.uz[d] = a.src.uz[s];
            }
            if (a.src.dlx) {
                a.dst.dlx[d] = a.src.dlx[s];
                if (a.src.dly) a.dst.dly[d] = a.src.dly[s];
                a.dst.dlz[d] = a.src.dlz[s];
            }
            a.dst.cell[d] = a.src.cell[s];
            if (a.src.id) a.dst.id[d] = a.src.id[s];
        }
    }
}

template <typename real>
void launch_compact(const CompactArgs<real> &a, cudaStream_t s)
{
    const int64_t grid = a.g.ntiles < 1048576 ? a.g.ntiles : 1048576;
    if (grid > 0) compact_kernel<real><<<(unsigned)grid, 256, 0, s>>>(a);
}

// ------------------------------------------------------------ cell order

// Counting sort of every tile's bucket by cell -- the cell's index inside
// its tile, x fastest, then y, then z -- into the bottom run of the same
// tile on the other side of the double buffer.  One CTA per tile: a
// histogram of the cells in shared memory, its exclusive scan, then every
// record copied to its cell's next slot (the order inside a cell is the
// order of the slot claims, which the results of a step do not depend on).
// A bucket of more than kSortKeys records is copied in its own order.
constexpr int kSortKeys = 8192;
constexpr int kSortCells = 512;  // the largest compiled tile (8 x 8 x 8, 16 x 16, 32 x 8)

template <typename real>
__global__ void __launch_bounds__(256) sort_cells_kernel(SortArgs<real> a)
{
    __shared__ int cnt[kSortCells];
    __shared__ unsigned short key[kSortKeys];
    __shared__ int wsum[8];
    const Geom &g = a.g;
    const int ncell = 1 << (g.lt[0] + g.lt[1] + g.lt[2]);
    const int tid = (int)threadIdx.x;
    for (int64_t t = blockIdx.x; t < g.ntiles; t += gridDim.x) {
        int n_lo, n_hi;
        bucket_counts(a.in_lo, a.in_hi, t, g.cap, n_lo, n_hi, a.err);
        const int n = n_lo + n_hi;
        const int tix = (int)(t % g.nt[0]);
        const int tiy = (int)((t / g.nt[0]) % g.nt[1]);
        const int tiz = (int)(t / ((int64_t)g.nt[0] * g.nt[1]));
        const int lox = tix << g.lt[0], loy = tiy << g.lt[1], loz = tiz << g.lt[2];
        const bool sorted = n <= kSortKeys;
        __syncthreads();  // the previous tile is done with shared memory
        for (int q = tid; q < ncell; q += blockDim.x) cnt[q] = 0;
        __syncthreads();
        if (sorted) {
            for (int p = tid; p < n; p += blockDim.x) {
                int ci, cj, ck;
                unpack_cell(g, a.in.cell[bucket_slot(t, g.cap, n_lo, n_hi, p)], ci, cj, ck);
                int li = ci - lox, lj = cj - loy, lk = ck - loz;
                if (li < 0 || li >= (1 << g.lt[0]) || lj < 0 || lj >= (1 << g.lt[1]) || lk < 0 ||
                    lk >= (1 << g.lt[2])) {
                    atomicOr(a.err, ERR_TILE);
                    li = lj = lk = 0;
                }
                const int lc = (((lk << g.lt[1]) | lj) << g.lt[0]) | li;
                key[p] = (unsigned short)lc;
                atomicAdd(&cnt[lc], 1);
            }
            __syncthreads();
            // exclusive scan of the counts: each thread two cells, then the
            // warps' totals
            const int c0 = 2 * tid, v0 = c0 < ncell ? cnt[c0] : 0, v1 = c0 + 1 < ncell ? cnt[c0 + 1] : 0;
            int x = v0 + v1;
            const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, x, o);
                if ((int)lane >= o) x += y;
            }
            if (lane == 31) wsum[warp] = x;
            __syncthreads();
            int before = 0;
            for (unsigned w = 0; w < warp; ++w) before += wsum[w];
            const int excl = before + x - (v0 + v1);
            __syncthreads();  // every count has been read
            if (c0 < ncell) cnt[c0] = excl;
            if (c0 + 1 < ncell) cnt[c0 + 1] = excl + v0;
            __syncthreads();
        }
        for (int p = tid; p < n; p += blockDim.x) {
            const int64_t s = bucket_slot(t, g.cap, n_lo, n_hi, p);
            const int64_t d = t * (int64_t)g.cap + (sorted ? atomicAdd(&cnt[key[p]], 1) : p);
            a.out.ox[d] = a.in.ox[s];
            if (a.in.oy) a.out.oy[d] = a.in.oy[s];
            a.out.oz[d] = a.in.oz[s];
            a.out.w[d] = a.in.w[s];
            if (a.in.ux) {
                a.out.ux[d] = a.in.ux[s];
                a.out.uy[d] = a.in.uy[s];
                a.out.uz[d] = a.in.uz[s];
            }
            if (a.in.dlx) {
                a.out.dlx[d] = a.in.dlx[s];
                if (a.in.dly) a.out.dly[d] = a.in.dly[s];
                a.out.dlz[d] = a.in.dlz[s];
            }
            a.out.cell[d] = a.in.cell[s];
            if (a.in.id) a.out.id[d] = a.in.id[s];
        }
        if (tid == 0) {
            a.out_lo[t] = n;
            a.in_lo[t] = 0;
            a.in_hi[t] = 0;
        }
    }
}

template <typename real>
void launch_sort_cells(const SortArgs<real> &a, cudaStream_t s)
{
    const int64_t grid = a.g.ntiles < 1048576 ? a.g.ntiles : 1048576;
    if (grid > 0) sort_cells_kernel<real><<<(unsigned)grid, 256, 0, s>>>(a);
}

// ------------------------------------------------------- charge density

template <typename real, int DIM, int S>
__global__ void rho_kernel(Geom g, Species<real> sp, const int *lo, const int *hi, real qfac, real *rho)
{
    for (int64_t t = blockIdx.x; t < g.ntiles; t += gridDim.x) {
        int n_lo, n_hi;
        bucket_counts(lo, hi, t, g.cap, n_lo, n_hi, nullptr);
        const int n = n_lo + n_hi;
        for (int p = threadIdx.x; p < n; p += blockDim.x) {
            const int64_t s = bucket_slot(t, g.cap, n_lo, n_hi, p);
            if ((uint32_t)sp.cell[s] & kPaired) continue;  // with its ion: no net charge
            int ci, cj, ck;
            unpack_cell(g, sp.cell[s], ci, cj, ck);
            real wx[S + 1], wy[S + 1], wz[S + 1];
            real ox = sp.ox[s], oy = DIM == 3 ? sp.oy[s] : real(0), oz = sp.oz[s];
            if (sp.dlx) {  // relative form: the offsets in the stored cell
                int r;
                ox = rel_actual(ox, sp.dlx[s], r);
                oz = rel_actual(oz, sp.dlz[s], r);
                if (DIM == 3) oy = rel_actual(oy, sp.dly[s], r);
            }
            const int bx = spline_weights<S>(ox, wx) + ci;
            const int bz = spline_weights<S>(oz, wz) + ck;
            int by = 0;
            if (DIM == 3) by = spline_weights<S>(oy, wy) + cj;
            const real q = qfac * sp.w[s];
            for (int c = 0; c <= S; ++c) {
                int k = bz + c;
                if (g.bc_z == 0) k = wrapi(k, g.nz);
                else if (k < 0 || k > g.nz) continue;
                for (int b = 0; b < (DIM == 3 ? S + 1 : 1); ++b) {
                    const int j = DIM == 3 ? wrapi(by + b, g.ny) : 0;
                    for (int a = 0; a <= S; ++a) {
                        const int i = wrapi(bx + a, g.nx);
                        const real wt = DIM == 3 ? wx[a] * wy[b] * wz[c] : wx[a] * wz[c];
                        atomicAdd(rho + fidx(g, i, j, k), q * wt);
                    }
                }
            }
        }
    }
}

template <typename real>
void launch_rho(const Geom &g, const Species<real> &sp, const int *lo, const int *hi, real qfac, real *rho,
                cudaStream_t s)
{
    const int64_t grid = g.ntiles < 1048576 ? g.ntiles : 1048576;
    if (grid <= 0) return;
    if (g.dim == 3) {
        if (g.shape == 1) rho_kernel<real, 3, 1><<<(unsigned)grid, 128, 0, s>>>(g, sp, lo, hi, qfac, rho);
        else rho_kernel<real, 3, 2><<<(unsigned)grid, 128, 0, s>>>(g, sp, lo, hi, qfac, rho);
    } else {
        if (g.shape == 1) rho_kernel<real, 2, 1><<<(unsigned)grid, 128, 0, s>>>(g, sp, lo, hi, qfac, rho);
        else rho_kernel<real, 2, 2><<<(unsigned)grid, 128, 0, s>>>(g, sp, lo, hi, qfac, rho);
    }
}

// -------------------------------------------------------- particle sums

// Kahan-compensated FP64 partial sums per block: [0] sum w (gamma-1),
// [1] sum q w (a paired electron and its ion carry no net charge), [2] the
// number of paired electrons.  The host adds the block partials, also with
// compensation.
template <typename real>
__global__ void particle_sums_kernel(Geom g, Species<real> sp, const int *lo, const int *hi, double q,
                                     double iux, double iuy, double iuz, double *partials)
{
    double s0 = 0, c0 = 0, s1 = 0, c1 = 0, npair = 0;
    for (int64_t t = blockIdx.x; t < g.ntiles; t += gridDim.x) {
        int n_lo, n_hi;
        bucket_counts(lo, hi, t, g.cap, n_lo, n_hi, nullptr);
        const int n = n_lo + n_hi;
        for (int p = threadIdx.x; p < n; p += blockDim.x) {
            const int64_t s = bucket_slot(t, g.cap, n_lo, n_hi, p);
            const double w = (double)sp.w[s];
            // records hold u - u_drift; ions move with the drift itself
            double ux = iux, uy = iuy, uz = iuz;
            if (sp.ux) {
                ux += (double)sp.ux[s];
                uy += (double)sp.uy[s];
                uz += (double)sp.uz[s];
            }
            const double u2 = ux * ux + uy * uy + uz * uz;
            const double ke = w * (u2 / (sqrt(1.0 + u2) + 1.0));  // gamma - 1 without cancellation
            const bool pair = ((uint32_t)sp.cell[s] & kPaired) != 0u;
            npair += pair ? 1.0 : 0.0;
            double y = ke - c0, tt = s0 + y;
            c0 = (tt - s0) - y;
            s0 = tt;
            y = (pair ? 0.0 : q * w) - c1;
            tt = s1 + y;
            c1 = (tt - s1) - y;
            s1 = tt;
        }
    }
    __shared__ double red[3][256];
    red[0][threadIdx.x] = s0 - c0;
    red[1][threadIdx.x] = s1 - c1;
    red[2][threadIdx.x] = npair;
    __syncthreads();
    for (int off = blockDim.x / 2; off > 0; off >>= 1) {
        if ((int)threadIdx.x < off) {
            red[0][threadIdx.x] += red[0][threadIdx.x + off];
            red[1][threadIdx.x] += red[1][threadIdx.x + off];
            red[2][threadIdx.x] += red[2][threadIdx.x + off];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        partials[3 * blockIdx.x] = red[0][0];
        partials[3 * blockIdx.x + 1] = red[1][0];
        partials[3 * blockIdx.x + 2] = red[2][0];
    }
}

template <typename real>
void launch_particle_sums(const Geom &g, const Species<real> &sp, const int *lo, const int *hi, double q,
                          const real u_drift[3], double *partials, int nblocks, cudaStream_t s)
{
    particle_sums_kernel<real><<<nblocks, 256, 0, s>>>(g, sp, lo, hi, q, (double)u_drift[0], (double)u_drift[1],
                                                       (double)u_drift[2], partials);
}

#define PIC_INSTANTIATE(real)                                                                       \
    template void launch_push<real>(const PushArgs<real> &, cudaStream_t);                          \
    template void launch_window_particles<real>(const Geom &, const Species<real> &, const Species<real> &, \
                                                const int *, const int *, int *, int *, int, int, cudaStream_t); \
    template void launch_ions<real>(const PushArgs<real> &, cudaStream_t);                          \
    template void launch_bucket<real>(const BucketArgs<real> &, cudaStream_t);                      \
    template void launch_compact<real>(const CompactArgs<real> &, cudaStream_t);                    \
    template void launch_sort_cells<real>(const SortArgs<real> &, cudaStream_t);                    \
    template void launch_rho<real>(const Geom &, const Species<real> &, const int *, const int *, real, \
                                   real *, cudaStream_t);                                            \
    template void launch_particle_sums<real>(const Geom &, const Species<real> &, const int *,      \
                                             const int *, double, const real *, double *, int,      \
                                             cudaStream_t);
PIC_INSTANTIATE(float)
PIC_INSTANTIATE(double)

}  // namespace pic
