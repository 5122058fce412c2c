// pic_push.cuh -- the per-tile bodies of the particle kernels and their
// helpers: fused gather / Boris push / Esirkepov deposit / re-bucketing of a
// tile's electrons (with its paired and released ions), and the drifting-ion
// deposit.  The single-run kernels (pic_particles.cu) and the batched ones
// (pic_batch.cu) run the same bodies.
//
// One CTA owns one tile of cells.  It stages E and B of the tile plus guard
// nodes in shared memory, pushes every particle of the tile, accumulates the
// current of all of them in a shared-memory J tile (tile plus the guard nodes
// a one-cell move can reach) and adds that tile to J in HBM once.  Each pushed
// particle is written straight into the bucket of the tile it now lies in, on
// the other side of the double buffer, so the store stays tile-sorted without
// a separate sort pass.
#pragma once

#include "pic_internal.cuh"

#include <cuda_pipeline.h>
#include <type_traits>

namespace pic {

// threads per CTA of the particle kernels; resident CTAs per SM the push
// kernel is compiled for (FP32: 3, which its shared memory allows on a 3D
// tile, i.e. up to 80 registers a thread; the FP64 debug path keeps more
// registers)
constexpr int kBlock = 256;
template <typename real> struct MinBlocks { static constexpr int value = sizeof(real) == 4 ? 3 : 2; };

// ---------------------------------------------------------------- helpers

// Shared-memory current accumulators.  FP32 currents are accumulated exactly,
// in 64-bit fixed point split over two 32-bit integer words per node: a
// contribution p = a*b, already multiplied by the launch's fixed-point scale
// (PushArgs::fx_scale, |p| < 2^21), is split into its nearest integer h and
// the remainder r = p - h (exact, |r| <= 1/2), and h and round(r 2^K) go to
// the "hi" and "lo" words with native integer atomics.  Integer addition is
// exact and associative, so a tile's sums do not depend on the order in which
// its particles are processed, and they carry the contributions to 2^-K.
// The "lo" word of a node sits LOFF words after its "hi" word.  FP64
// accumulates in double.  Zero words (e.g. nodes of a window outside both
// supports) are not added.
template <typename real> struct Acc { using type = double; };
template <> struct Acc<float> { using type = int; };

// adding 1.5 * 2^23 to x (|x| <= 2^22) leaves round(x) in the low mantissa
// bits, which are read back as an integer
constexpr float kRoundMagic = 12582912.0f;
constexpr int kRoundMagicBits = 0x4B400000;

template <int LOFF>
__device__ __forceinline__ void sh_acc(int *p, float a, float b, float lo_scale)
{
    const float v = a * b;
    const float t = v + kRoundMagic;
    const int h = __float_as_int(t) - kRoundMagicBits;
    const float r = v - (t - kRoundMagic);
    const int l = __float_as_int(fmaf(r, lo_scale, kRoundMagic)) - kRoundMagicBits;
    if (h != 0) atomicAdd(p, h);
    if (l != 0) atomicAdd(p + LOFF, l);
}

// FP64 contributions into the same fixed-point words (records in relative
// form): h and the remainder's 2^K multiple rounded from the FP64 product
template <int LOFF>
__device__ __forceinline__ void sh_acc(int *p, double a, double b, double lo_scale)
{
    const double v = a * b;
    const double hd = rint(v);
    const int h = (int)hd;
    const int l = (int)rint((v - hd) * lo_scale);
    if (h != 0) atomicAdd(p, h);
    if (l != 0) atomicAdd(p + LOFF, l);
}

template <int LOFF>
__device__ __forceinline__ void sh_acc(double *p, double a, double b, double)
{
    const double v = a * b;
    if (v != 0.0) atomicAdd(p, v);
}


template <typename real>
struct Ptr6 {
    const real *p0, *p1, *p2, *p3, *p4, *p5;
    __device__ __forceinline__ const real *operator[](int c) const
    {
        return c == 0 ? p0 : c == 1 ? p1 : c == 2 ? p2 : c == 3 ? p3 : c == 4 ? p4 : p5;
    }
};

template <typename real>
struct Ptr3 {
    real *p0, *p1, *p2;
    __device__ __forceinline__ real *operator[](int c) const { return c == 0 ? p0 : c == 1 ? p1 : p2; }
};

// Stage NC field components of the box [lo - L, lo - L + F) (per axis) into
// shared memory.  Element-wise over all threads with compile-time extents, so
// the index decomposition is a few multiply-shifts; consecutive threads read
// consecutive x.  Nodes outside the valid z range of a component (absorbing z)
// are zero; x and y wrap.  Returns whether this thread staged a non-zero value.
template <typename real, int DIM, int NC, int FX, int FY, int FZ, int L>
__device__ __forceinline__ bool stage_tile(const Geom &g, const Ptr6<real> src, unsigned half_z, real *dst, int lox,
                                           int loy, int loz)
{
    constexpr int FN = FX * FY * FZ;
    const bool tiny = g.nx < FX || (DIM == 3 && g.ny < FY);
    bool nonzero = false;
    // each node of the box once, all components of it together
    for (int r = threadIdx.x; r < FN; r += blockDim.x) {
        const int lz = r / (FX * FY), r2 = r - lz * (FX * FY);
        const int ly = r2 / FX, lx = r2 - ly * FX;
        int gk = loz - L + lz;
        const bool inz = g.bc_z == 0 || gk >= 0;
        if (g.bc_z == 0) gk = wrapi(gk, g.nz);
        const int gi = tiny ? wrapi(lox - L + lx, g.nx) : wrap1(lox - L + lx, g.nx);
        const int gj = DIM == 3 ? (tiny ? wrapi(loy - L + ly, g.ny) : wrap1(loy - L + ly, g.ny)) : 0;
        const int64_t o = fidx(g, gi, gj, inz ? gk : 0);
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const bool ok = inz && (g.bc_z == 0 || gk <= zmax_of(g, (half_z >> c) & 1u));
            const real v = ok ? src[c][o] : real(0);
            dst[c * FN + r] = v;
            nonzero = nonzero || v != real(0);
        }
    }
    return nonzero;
}

// Add NC shared-memory tiles (box [lo - L, lo - L + Q) per axis) to the global
// arrays, element-wise over all threads: non-zero nodes only, periodic x and y,
// nodes outside a component's valid z range dropped (absorbing z).  FP32
// tiles hold fixed-point "hi" and "lo" words (see sh_acc): the node's value is
// (hi + lo lo_inv) times the component's quantum q_c.
template <typename real, int DIM, int NC, int QX, int QY, int QZ, int L>
__device__ __forceinline__ void flush_tile(const Geom &g, const Ptr3<real> dstJ, unsigned half_z,
                                           const typename Acc<real>::type *src, real q0, real q1, real q2,
                                           real lo_inv, int lox, int loy, int loz)
{
    constexpr int QN = QX * QY * QZ;
    const bool tiny = g.nx < QX || (DIM == 3 && g.ny < QY);
    // each node of the box once, all components of it together
    for (int r = threadIdx.x; r < QN; r += blockDim.x) {
        real v[NC];
        bool any = false;
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            if constexpr (sizeof(real) == 4) {
                const int h = src[c * QN + r], l = src[NC * QN + c * QN + r];  // "hi" and "lo" words
                v[c] = (h | l) == 0 ? real(0) : fmaf((float)l, lo_inv, (float)h);
            } else {
                v[c] = src[c * QN + r];
            }
            any = any || v[c] != real(0);
        }
        if (!any) continue;
        const int lz = r / (QX * QY), r2 = r - lz * (QX * QY);
        const int ly = r2 / QX, lx = r2 - ly * QX;
        int gk = loz - L + lz;
        if (g.bc_z == 0) gk = wrapi(gk, g.nz);
        else if (gk < 0) continue;
        const int gi = tiny ? wrapi(lox - L + lx, g.nx) : wrap1(lox - L + lx, g.nx);
        const int gj = DIM == 3 ? (tiny ? wrapi(loy - L + ly, g.ny) : wrap1(loy - L + ly, g.ny)) : 0;
        const int64_t o = fidx(g, gi, gj, gk);
#pragma unroll
        for (int c = 0; c < NC; ++c)
            if (v[c] != real(0) && (g.bc_z == 0 || gk <= zmax_of(g, (half_z >> c) & 1u)))
                atomicAdd(dstJ[c] + o, v[c] * (c == 0 ? q0 : c == 1 ? q1 : q2));
    }
}

// Output slot of every lane's particle (dest < 0: none).  Particles that stay
// in tile `own` take the next slots of its bottom run from a shared-memory
// counter (one shared atomic per warp); the others take slots of their
// destination's top run through global atomics (one per destination tile in
// the warp).  Returns the slot index inside the destination bucket, or -1 when
// the bucket is full.
__device__ __forceinline__ int output_slot(int *s_stay, int *out_hi, int64_t dest, int64_t own, int cap)
{
    const unsigned lane = threadIdx.x & 31u;
    const unsigned stay = __ballot_sync(0xffffffffu, dest == own);
    int base = 0;
    if (lane == 0 && stay) base = atomicAdd(s_stay, __popc(stay));
    base = __shfl_sync(0xffffffffu, base, 0);
    const bool leave = dest >= 0 && dest != own;
    const int r = __any_sync(0xffffffffu, leave) ? reserve_slot(out_hi, leave ? dest : -1) : 0;
    if (dest == own) {
        const int slot = base + __popc(stay & ((1u << lane) - 1u));
        return slot < cap ? slot : -1;
    }
    return (leave && r < cap) ? cap - 1 - r : -1;
}

// ---------------------------------------------------------------- gather

// interpolate one component from the shared field tile: node (a, b, c) of the
// support of each axis starts at base + cell-local index (+ guard FL)
template <int DIM, int S, typename real>
__device__ __forceinline__ real gather_comp(const real *F, int FX, int FY, int ix, int iy, int iz,
                                            const real *wx, const real *wy, const real *wz)
{
    real sum = 0;
    if (DIM == 3) {
#pragma unroll
        for (int c = 0; c <= S; ++c) {
#pragma unroll
            for (int b = 0; b <= S; ++b) {
                const real *row = F + ((int64_t)(iz + c) * FY + (iy + b)) * FX + ix;
                real r = 0;
#pragma unroll
                for (int a = 0; a <= S; ++a) r += wx[a] * row[a];
                sum += wz[c] * wy[b] * r;
            }
        }
    } else {
#pragma unroll
        for (int c = 0; c <= S; ++c) {
            const real *row = F + (int64_t)(iz + c) * FX + ix;
            real r = 0;
#pragma unroll
            for (int a = 0; a <= S; ++a) r += wx[a] * row[a];
            sum += wz[c] * r;
        }
    }
    return sum;
}

// --------------------------------------------------------- Esirkepov

// Current of one particle into the shared J tile.  Along an axis the window
// has W nodes: S+1 when no lane of the warp moved its support to another first
// node along that axis (the last node is then outside both supports), else
// S+2.  The running sum along an axis is taken over DS first:
//   Jx(a,b,c) = fx * (sum_{a'<=a} DSx[a']) * T_yz(b,c),
//   T_yz = S0y (S0z + DSz/2) + DSy (S0z/2 + DSz/3)        (and cyclically),
// which is Esirkepov's decomposition rearranged; the last running sum of a
// window is zero and is not added.  In 2D3V the out-of-plane current is the
// path average of the shape times q w vy / V.
template <typename real, typename accT, int DIM, int S, int QX, int QY, int QN, int WX, int WY, int WZ>
__device__ __forceinline__ void deposit_w(accT *sJ, const real *S0x, const real *DSx, const real *S0y,
                                          const real *DSy, const real *S0z, const real *DSz, int ax, int ay, int az,
                                          real fx, real fy, real fz, real fyv, real los)
{
    constexpr int LOFF = 3 * QN;  // "lo" words follow the three components' "hi" words
    constexpr real half = real(0.5), third = real(1) / real(3);
    auto *Jx = sJ, *Jy = sJ + QN, *Jz = sJ + 2 * QN;
    real Px[WX], Pz[WZ];
    real acc = 0;
#pragma unroll
    for (int q = 0; q < WX; ++q) { acc += DSx[q]; Px[q] = fx * acc; }
    acc = 0;
#pragma unroll
    for (int c = 0; c < WZ; ++c) { acc += DSz[c]; Pz[c] = fz * acc; }
    if (DIM == 3) {
        real Py[WY];
        acc = 0;
#pragma unroll
        for (int b = 0; b < WY; ++b) { acc += DSy[b]; Py[b] = fy * acc; }
#pragma unroll
        for (int c = 0; c < WZ; ++c) {
            const real za = S0z[c] + half * DSz[c], zb = half * S0z[c] + third * DSz[c];
#pragma unroll
            for (int b = 0; b < WY; ++b) {
                const real tyz = S0y[b] * za + DSy[b] * zb;
                auto *row = Jx + ((az + c) * QY + (ay + b)) * QX + ax;
#pragma unroll
                for (int q = 0; q < WX - 1; ++q) sh_acc<LOFF>(row + q, Px[q], tyz, los);
            }
#pragma unroll
            for (int q = 0; q < WX; ++q) {
                const real tzx = S0z[c] * (S0x[q] + half * DSx[q]) + DSz[c] * (half * S0x[q] + third * DSx[q]);
                auto *col = Jy + ((az + c) * QY + ay) * QX + ax + q;
#pragma unroll
                for (int b = 0; b < WY - 1; ++b) sh_acc<LOFF>(col + b * QX, Py[b], tzx, los);
            }
        }
#pragma unroll
        for (int b = 0; b < WY; ++b) {
            const real ya = S0y[b] + half * DSy[b], yb = half * S0y[b] + third * DSy[b];
#pragma unroll
            for (int q = 0; q < WX; ++q) {
                const real txy = S0x[q] * ya + DSx[q] * yb;
                auto *col = Jz + (az * QY + (ay + b)) * QX + ax + q;
#pragma unroll
                for (int c = 0; c < WZ - 1; ++c) sh_acc<LOFF>(col + c * QX * QY, Pz[c], txy, los);
            }
        }
    } else {
#pragma unroll
        for (int c = 0; c < WZ; ++c) {
            const real za = S0z[c] + half * DSz[c], zb = half * S0z[c] + third * DSz[c];
            auto *row = Jx + (az + c) * QX + ax;
#pragma unroll
            for (int q = 0; q < WX - 1; ++q) sh_acc<LOFF>(row + q, Px[q], za, los);
#pragma unroll
            for (int q = 0; q < WX; ++q) sh_acc<LOFF>(Jy + (az + c) * QX + ax + q, fyv, S0x[q] * za + DSx[q] * zb, los);
        }
#pragma unroll
        for (int q = 0; q < WX; ++q) {
            const real xa = S0x[q] + half * DSx[q];
#pragma unroll
            for (int c = 0; c < WZ - 1; ++c) sh_acc<LOFF>(Jz + (az + c) * QX + ax + q, Pz[c], xa, los);
        }
    }
}

// The current of particles that did not move across z (3D): Wx = Wy = 0
// exactly, so Jx = Jy = 0 and Jz(q,b,c) = fz (sum_{c'<=c} DSz[c']) S0x[q] S0y[b]
// -- the general formula's values with DSx = DSy = 0.  Windows along x and y
// have S+1 nodes (their supports did not move).
template <typename real, typename accT, int S, int QX, int QY, int QN, int WZ>
__device__ __forceinline__ void deposit_z(accT *sJ, const real *S0x, const real *S0y, const real *S0z,
                                          const real *DSz, int ax, int ay, int az, real fz, real los)
{
    constexpr int LOFF = 3 * QN;
    auto *Jz = sJ + 2 * QN;
    real Pz[WZ];
    real acc = 0;
#pragma unroll
    for (int c = 0; c < WZ; ++c) { acc += DSz[c]; Pz[c] = fz * acc; }
    (void)S0z;
#pragma unroll
    for (int b = 0; b < S + 1; ++b) {
#pragma unroll
        for (int q = 0; q < S + 1; ++q) {
            const real txy = S0x[q] * S0y[b];
            auto *col = Jz + (az * QY + (ay + b)) * QX + ax + q;
#pragma unroll
            for (int c = 0; c < WZ - 1; ++c) sh_acc<LOFF>(col + c * QX * QY, Pz[c], txy, los);
        }
    }
}

// picks the window lengths for the warp: bit 2 x, bit 1 y, bit 0 z crossed
template <typename real, typename accT, int DIM, int S, int QX, int QY, int QN>
__device__ __forceinline__ void deposit_sel(unsigned sel, accT *sJ, const real *S0x, const real *DSx, const real *S0y,
                                            const real *DSy, const real *S0z, const real *DSz, int ax, int ay, int az,
                                            real fx, real fy, real fz, real fyv, real los)
{
    constexpr int A = S + 1, B = S + 2;
#define PIC_DEP(wx, wy, wz) \
    deposit_w<real, accT, DIM, S, QX, QY, QN, wx, wy, wz>(sJ, S0x, DSx, S0y, DSy, S0z, DSz, ax, ay, az, fx, fy, fz, fyv, los)
    if (DIM == 3) {
        switch (sel) {
        case 0: PIC_DEP(A, A, A); break;
        case 1: PIC_DEP(A, A, B); break;
        case 2: PIC_DEP(A, B, A); break;
        case 3: PIC_DEP(A, B, B); break;
        case 4: PIC_DEP(B, A, A); break;
        case 5: PIC_DEP(B, A, B); break;
        case 6: PIC_DEP(B, B, A); break;
        default: PIC_DEP(B, B, B); break;
        }
    } else {
        switch (sel & 5u) {
        case 0: PIC_DEP(A, 1, A); break;
        case 1: PIC_DEP(A, 1, B); break;
        case 4: PIC_DEP(B, 1, A); break;
        default: PIC_DEP(B, 1, B); break;
        }
    }
#undef PIC_DEP
}

// ------------------------------------------------------------- drifting ions

// Ions immobile in the lab move at the species' constant u = (0, 0, -gamma
// beta) in the boosted frame: every ion of a step moves by the same
// dz = u_z dt / (gamma h_z), in (-1, 0) cells, and its transverse position
// never changes.  So only Jz is deposited, Wz = DSz (S0x S0y) (the general
// formula with DSx = DSy = 0, in the arithmetic order of the electrons'
// z-only deposit), and an ion either stays in its tile or moves to the one
// tile below it (the top tile when z wraps, none when it leaves the box):
// one counter per warp reserves the slots of the leavers.
// The ions of tile t (all threads of the CTA call it): their Jz into the
// current tile at Jz (the "hi" words; the "lo" words LOFF further), records
// into the output side.  sP holds kIonStages x 5 x kBlock prefetch slots
// (the copies of two iterations are in flight while one is processed: the
// ion loop moves little data per instruction).  Returns false (nothing done)
// for an empty bucket.
constexpr int kIonStages = 3;

// Jz of one ion moving along z from z0 to z1 (both relative to its cell, z0 in
// [0, 1)), in arithmetic ar, into the current tile Jz (QX x QY rows)
template <typename ar, typename accT, int DIM, int S, int QX, int QY, int LOFF>
__device__ __forceinline__ void ion_deposit(accT *Jz, ar z0, ar z1, ar ox, ar oy, int li, int lj, int lk, ar fz,
                                            ar lo_scale)
{
    constexpr int JL = S;
    ar S0z[S + 2], DSz[S + 2], wx[S + 1], wy[S + 1];
    bool crossed;
    const int az = esirk_axis_c<S>(z0, z1, S0z, DSz, crossed) + lk + JL;
    const int bx = offset_weights<S>(ox, wx) + li + JL;
    int by = 0;
    if (DIM == 3) by = offset_weights<S>(oy, wy) + lj + JL;
    ar Pz[S + 2];
    ar run = 0;
#pragma unroll
    for (int c = 0; c < S + 2; ++c) {
        run += DSz[c];
        Pz[c] = fz * run;
    }
#pragma unroll
    for (int b = 0; b < (DIM == 3 ? S + 1 : 1); ++b) {
#pragma unroll
        for (int q = 0; q < S + 1; ++q) {
            const ar sxy = DIM == 3 ? wx[q] * wy[b] : wx[q];
#pragma unroll
            for (int c = 0; c < S + 1; ++c)
                sh_acc<LOFF>(Jz + ((az + c) * QY + (by + b)) * QX + bx + q, Pz[c], sxy, lo_scale);
        }
    }
}

// REL: the tile's electrons are in relative form; the ions' currents are then
// formed in FP64 from their stored positions (the end of one step's path is
// exactly the start of the next one's)
template <typename real, int DIM, int S, int TX, int TY, int TZ, int LOFF, bool REL>
__device__ __forceinline__ bool ions_of_tile(const Geom &g, const IonSide<real> &is, int64_t t,
                                             typename Acc<real>::type *Jz, real *sP, real dz, real scale_z,
                                             real lo_scale, unsigned *err, int *s_stay)
{
    constexpr int JL = S, JH = S + 1;
    constexpr int QX = TX + JL + JH, QY = DIM == 3 ? TY + JL + JH : 1;
    using acc_t = typename Acc<real>::type;
    const unsigned lane = threadIdx.x & 31u;
    int n_lo, n_hi;
    bucket_counts(is.in_lo, is.in_hi, t, g.cap, n_lo, n_hi, err);
    const int n = n_lo + n_hi;
    if (n == 0) return false;
    auto prefetch = [&](int it) {
        const int p = it * kBlock + (int)threadIdx.x;
        if (p < n) {
            const int64_t s = bucket_slot(t, g.cap, n_lo, n_hi, p);
            real *d = sP + (it % kIonStages) * 5 * kBlock + threadIdx.x;
            __pipeline_memcpy_async(d + 0 * kBlock, is.in.ox + s, sizeof(real));
            if (DIM == 3) __pipeline_memcpy_async(d + 1 * kBlock, is.in.oy + s, sizeof(real));
            __pipeline_memcpy_async(d + 2 * kBlock, is.in.oz + s, sizeof(real));
            __pipeline_memcpy_async(d + 3 * kBlock, is.in.w + s, sizeof(real));
            __pipeline_memcpy_async(d + 4 * kBlock, is.in.cell + s, sizeof(int32_t));
        }
        __pipeline_commit();
    };
    const int64_t ntxy = (int64_t)g.nt[0] * g.nt[1];
    const int tix = (int)(t % g.nt[0]);
    const int tiy = (int)((t / g.nt[0]) % g.nt[1]);
    const int tiz = (int)(t / ntxy);
    const int lox = tix << g.lt[0], loy = tiy << g.lt[1], loz = tiz << g.lt[2];
    // the tile an ion leaving this one through its lower z face enters
    // (-1: it leaves the box)
    const int64_t below = tiz > 0 ? t - ntxy : (g.bc_z == 0 ? t + (int64_t)(g.nt[2] - 1) * ntxy : -1);
    __syncthreads();
    if (threadIdx.x == 0) *s_stay = 0;
    // each thread copies and reads only its own slots: no barrier between
    // the stages
    for (int it = 0; it < kIonStages - 1; ++it) prefetch(it);
    __syncthreads();
    for (int it = 0; it * kBlock < n; ++it) {
        const int p = it * kBlock + threadIdx.x;
        prefetch(it + kIonStages - 1);
        __pipeline_wait_prior(kIonStages - 1);
        bool stay = false, leave = false;
        real ox = 0, oy = 0, oz = 0, w = 0;
        int32_t cell = 0;
        int64_t pid = 0;
        if (p < n) {
            const real *d = sP + (it % kIonStages) * 5 * kBlock + threadIdx.x;
            int ci, cj, ck;
            unpack_cell(g, *reinterpret_cast<const int32_t *>(d + 4 * kBlock), ci, cj, ck);
            const int li = ci - lox, lj = cj - loy, lk = ck - loz;
            if (li < 0 || li >= TX || lj < 0 || lj >= TY || lk < 0 || lk >= TZ) {
                atomicOr(err, ERR_TILE);
            } else {
                ox = d[0 * kBlock];
                oy = DIM == 3 ? d[1 * kBlock] : real(0);
                oz = d[2 * kBlock];
                w = d[3 * kBlock];
                if (is.in.id) pid = is.in.id[bucket_slot(t, g.cap, n_lo, n_hi, p)];
                const real z1 = add_rn(oz, dz);
                if (!REL) {
                    // written out here rather than through ion_deposit: the
                    // inlined call measured more register spills in the
                    // electron kernel that fuses this pass
                    real S0z[S + 2], DSz[S + 2], wx[S + 1], wy[S + 1];
                    bool crossed;
                    const int az = esirk_axis_c<S>(oz, z1, S0z, DSz, crossed) + lk + JL;
                    const int bx = offset_weights<S>(ox, wx) + li + JL;
                    int by = 0;
                    if (DIM == 3) by = offset_weights<S>(oy, wy) + lj + JL;
                    const real fz = is.jfac_z * w * scale_z;
                    real Pz[S + 2];
                    real run = 0;
#pragma unroll
                    for (int c = 0; c < S + 2; ++c) { run += DSz[c]; Pz[c] = fz * run; }
#pragma unroll
                    for (int b = 0; b < (DIM == 3 ? S + 1 : 1); ++b) {
#pragma unroll
                        for (int q = 0; q < S + 1; ++q) {
                            const real sxy = DIM == 3 ? wx[q] * wy[b] : wx[q];
#pragma unroll
                            for (int c = 0; c < S + 1; ++c)
                                sh_acc<LOFF>(Jz + ((az + c) * QY + (by + b)) * QX + bx + q, Pz[c], sxy, lo_scale);
                        }
                    }
                }
                // z1 in (-1, 1): the same cell or the one below; an offset
                // that rounds to 1 stays in the cell with offset 0
                int sz = 0;
                real on = z1;
                if (z1 < real(0)) {
                    on = z1 + real(1);
                    sz = -1;
                    if (on >= real(1)) { on = 0; sz = 0; }
                }
                if (REL)  // from the stored position to the stored position
                    ion_deposit<double, acc_t, DIM, S, QX, QY, LOFF>(
                        Jz, (double)oz, (double)sz + (double)on, (double)ox, (double)oy, li, lj, lk,
                        (double)is.jfac_z * (double)w * (double)scale_z, (double)lo_scale);
                oz = on;
                int nk = ck + sz;
                bool alive = true;
                if (nk < 0) {
                    if (g.bc_z == 0) nk += g.nz;
                    else alive = false;
                }
                if (alive) {
                    cell = pack_cell(g, ci, cj, nk);
                    stay = lk + sz >= 0;
                    leave = !stay;
                }
            }
        }
        // slots: stayers from the shared counter, leavers from the counter
        // of the tile below (one atomic each per warp)
        const unsigned ms = __ballot_sync(0xffffffffu, stay), ml = __ballot_sync(0xffffffffu, leave);
        int bs = 0, bl = 0;
        if (lane == 0) {
            if (ms) bs = atomicAdd(s_stay, __popc(ms));
            if (ml) bl = atomicAdd(&is.out_hi[below], __popc(ml));
        }
        bs = __shfl_sync(0xffffffffu, bs, 0);
        bl = __shfl_sync(0xffffffffu, bl, 0);
        const unsigned below_me = (1u << lane) - 1u;
        int64_t d = -1;
        if (stay) {
            const int r = bs + __popc(ms & below_me);
            if (r < g.cap) d = t * (int64_t)g.cap + r;
            else atomicOr(err, ERR_CAPACITY);
        } else if (leave) {
            const int r = bl + __popc(ml & below_me);
            if (r < g.cap) d = below * (int64_t)g.cap + (g.cap - 1 - r);
            else atomicOr(err, ERR_CAPACITY);
        }
        if (d >= 0) {
            is.out.ox[d] = ox;
            if (DIM == 3) is.out.oy[d] = oy;
            is.out.oz[d] = oz;
            is.out.w[d] = w;
            is.out.cell[d] = cell;
            if (is.out.id) is.out.id[d] = pid;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        is.out_lo[t] = min(*s_stay, g.cap);
        is.in_lo[t] = 0;
        is.in_hi[t] = 0;
    }
    return true;
}

// ------------------------------------------------------------ push kernel

// one axis of a record in relative form: the departure takes the step's
// displacement d; whole cells move to the reference (exact: |dl| <= 3/2)
template <typename real>
__device__ __forceinline__ real rel_step(real dl, real d, int &fold)
{
    real v = dl + d;
    fold = 0;
    if (v > real(0.5)) {
        v = v - real(1);
        fold = 1;
    } else if (v < real(-0.5)) {
        v = v + real(1);
        fold = -1;
    }
    return v;
}

// REL: electron records in relative form (rel_actual): the gather uses the
// offsets in the stored cell, the current is deposited in FP64 from the exact
// positions reference + departure
template <typename real, int DIM, int S, int TX, int TY, int TZ, bool REL>
__device__ __forceinline__ void push_tile(const PushArgs<real> &a, const int64_t t, unsigned char *smem_raw)
{
    const Geom &g = a.g;
    // tile shape and shared-tile extents are compile-time constants, so every
    // stencil offset below folds into an immediate
    constexpr int FL = 1, FH = S;        // field guards below / above the tile
    constexpr int JL = S, JH = S + 1;    // current guards below / above the tile
    constexpr int FX = TX + FL + FH, FY = DIM == 3 ? TY + FL + FH : 1, FZ = TZ + FL + FH;
    constexpr int QX = TX + JL + JH, QY = DIM == 3 ? TY + JL + JH : 1, QZ = TZ + JL + JH;
    constexpr int FN = FX * FY * FZ, QN = QX * QY * QZ;
    using acc_t = typename Acc<real>::type;
    // arithmetic of the deposit: FP64 for records in relative form
    using dep_t = typename std::conditional<REL, double, real>::type;
    real *sF = reinterpret_cast<real *>(smem_raw);
    acc_t *sJ = reinterpret_cast<acc_t *>(sF + 6 * FN);
    // the next iteration's particle records are copied into shared memory
    // with cp.async while the current ones are pushed (two buffers of
    // NA attributes x kBlock particles; each thread copies and reads its own)
    constexpr int NA = REL ? (DIM == 3 ? 11 : 10) : 8;
    real *sP = reinterpret_cast<real *>(sJ + (sizeof(real) == 4 ? 6 : 3) * QN);
    __shared__ int s_stay, s_stay_i;
    // the plasma drift and its displacement per step (the drifting ions')
    const Drift<real> drift(a.u_drift, a.dtdh[2]);
    const real dz_drift = drift.dz;

    {
        int n_lo, n_hi;
        bucket_counts(a.in_lo, a.in_hi, t, g.cap, n_lo, n_hi, a.err);
        const int n = n_lo + n_hi;
        // uniform over the CTA
        if (n == 0 && !(a.fuse_ions && a.ions.in_lo[t] + a.ions.in_hi[t] > 0)) return;
        auto prefetch = [&](int it) {
            const int p = it * kBlock + (int)threadIdx.x;
            if (p < n) {
                const int64_t s = bucket_slot(t, g.cap, n_lo, n_hi, p);
                real *d = sP + (it & 1) * NA * kBlock + threadIdx.x;
                __pipeline_memcpy_async(d + 0 * kBlock, a.in.ox + s, sizeof(real));
                if (DIM == 3) __pipeline_memcpy_async(d + 1 * kBlock, a.in.oy + s, sizeof(real));
                __pipeline_memcpy_async(d + 2 * kBlock, a.in.oz + s, sizeof(real));
                __pipeline_memcpy_async(d + 3 * kBlock, a.in.w + s, sizeof(real));
                __pipeline_memcpy_async(d + 4 * kBlock, a.in.ux + s, sizeof(real));
                __pipeline_memcpy_async(d + 5 * kBlock, a.in.uy + s, sizeof(real));
                __pipeline_memcpy_async(d + 6 * kBlock, a.in.uz + s, sizeof(real));
                __pipeline_memcpy_async(d + 7 * kBlock, a.in.cell + s, sizeof(int32_t));
                if (REL) {
                    __pipeline_memcpy_async(d + 8 * kBlock, a.in.dlx + s, sizeof(real));
                    __pipeline_memcpy_async(d + 9 * kBlock, a.in.dlz + s, sizeof(real));
                    if (DIM == 3) __pipeline_memcpy_async(d + 10 * kBlock, a.in.dly + s, sizeof(real));
                }
            }
            __pipeline_commit();
        };
        const int tix = (int)(t % g.nt[0]);
        const int tiy = (int)((t / g.nt[0]) % g.nt[1]);
        const int tiz = (int)(t / ((int64_t)g.nt[0] * g.nt[1]));
        const int lox = tix << g.lt[0], loy = tiy << g.lt[1], loz = tiz << g.lt[2];

        __syncthreads();  // previous tile finished with shared memory
        if (threadIdx.x == 0) s_stay = 0;
        // Ez, Bx, By live on half-integer z (bits 2, 3, 4)
        const bool staged_nonzero = stage_tile<real, DIM, 6, FX, FY, FZ, FL>(
            g, Ptr6<real>{a.E[0], a.E[1], a.E[2], a.B[0], a.B[1], a.B[2]}, 0x1Cu, sF, lox, loy, loz);
        for (int q = threadIdx.x; q < (sizeof(real) == 4 ? 6 : 3) * QN; q += blockDim.x) sJ[q] = 0;
        prefetch(0);
        const bool field_in_tile = __syncthreads_or(staged_nonzero) != 0;

        for (int it = 0; it * kBlock < n; ++it) {
            const int p = it * kBlock + threadIdx.x;
            bool valid = p < n;
            prefetch(it + 1);
            __pipeline_wait_prior(1);
            real ox = 0, oy = 0, oz = 0, w = 0, ux = 0, uy = 0, uz = 0;
            // relative form: reference offsets, departures and the reference
            // cell's shift from the stored cell, per axis
            real orx = 0, ory = 0, orz = 0, dlx = 0, dly = 0, dlz = 0;
            int rx = 0, ry = 0, rz = 0;
            int ci = 0, cj = 0, ck = 0, li = 0, lj = 0, lk = 0;
            int64_t pid = 0;
            bool paired = false;
            // ---- load (from the prefetched records)
            if (valid) {
                const real *d = sP + (it & 1) * NA * kBlock + threadIdx.x;
                const int32_t word = *reinterpret_cast<const int32_t *>(d + 7 * kBlock);
                paired = ((uint32_t)word & kPaired) != 0u;
                unpack_cell(g, word, ci, cj, ck);
                li = ci - lox;
                lj = cj - loy;
                lk = ck - loz;
                if (li < 0 || li >= TX || lj < 0 || lj >= TY || lk < 0 || lk >= TZ) {
                    atomicOr(a.err, ERR_TILE);
                    valid = false;
                } else {
                    ox = d[0 * kBlock];
                    if (DIM == 3) oy = d[1 * kBlock];
                    oz = d[2 * kBlock];
                    w = d[3 * kBlock];
                    ux = d[4 * kBlock];
                    uy = d[5 * kBlock];
                    uz = d[6 * kBlock];
                    if (REL) {
                        orx = ox;
                        ory = oy;
                        orz = oz;
                        dlx = d[8 * kBlock];
                        dlz = d[9 * kBlock];
                        if (DIM == 3) dly = d[10 * kBlock];
                        ox = rel_actual(orx, dlx, rx);
                        oz = rel_actual(orz, dlz, rz);
                        if (DIM == 3) oy = rel_actual(ory, dly, ry);
                    }
                    if (a.in.id) pid = a.in.id[bucket_slot(t, g.cap, n_lo, n_hi, p)];
                }
            }
            // ---- gather E^n, B^n at x^n, Boris, move
            real x1 = 0, y1 = 0, z1 = 0, vy = 0;
            // relative form: new departures, new z reference, the new cell's
            // shift per axis, and the exact (FP64) start and end of the path
            // relative to the old cell
            real dlx1 = 0, dly1 = 0, dlz1 = 0, orz1 = 0;
            int mx = 0, my = 0, mz = 0;
            double X0 = 0, X1 = 0, Y0 = 0, Y1 = 0, Z0 = 0, Z1 = 0;
            bool release = false;
            if (valid) {
                // a tile whose staged E and B are all zero gathers exactly zero
                // everywhere: Boris is then the identity and no pair is released
                if (field_in_tile) {
                    real wxu[S + 1], wxh[S + 1], wyu[S + 1], wyh[S + 1], wzu[S + 1], wzh[S + 1];
                    const int bxu = offset_weights<S>(ox, wxu) + li + FL;
                    const int bxh = half_weights<S>(ox, wxh) + li + FL;
                    const int bzu = offset_weights<S>(oz, wzu) + lk + FL;
                    const int bzh = half_weights<S>(oz, wzh) + lk + FL;
                    int byu = 0, byh = 0;
                    if (DIM == 3) {
                        byu = offset_weights<S>(oy, wyu) + lj + FL;
                        byh = half_weights<S>(oy, wyh) + lj + FL;
                    } else {
#pragma unroll
                        for (int q = 0; q <= S; ++q) wyu[q] = wyh[q] = real(q == 0);
                    }
                    const real ex = gather_comp<DIM, S>(sF + 0 * FN, FX, FY, bxh, byu, bzu, wxh, wyu, wzu);
                    const real ey = gather_comp<DIM, S>(sF + 1 * FN, FX, FY, bxu, byh, bzu, wxu, wyh, wzu);
                    const real ez = gather_comp<DIM, S>(sF + 2 * FN, FX, FY, bxu, byu, bzh, wxu, wyu, wzh);
                    const real bx = gather_comp<DIM, S>(sF + 3 * FN, FX, FY, bxu, byh, bzh, wxu, wyh, wzh);
                    const real by = gather_comp<DIM, S>(sF + 4 * FN, FX, FY, bxh, byu, bzh, wxh, wyu, wzh);
                    const real bz = gather_comp<DIM, S>(sF + 5 * FN, FX, FY, bxh, byh, bzu, wxh, wyh, wzu);
                    // a paired electron that gathers a non-zero field leaves its
                    // ion behind: the pair's current is no longer zero
                    if (paired && (ex != real(0) || ey != real(0) || ez != real(0) || bx != real(0) ||
                                   by != real(0) || bz != real(0)))
                        release = true;
                    boris(ux, uy, uz, drift.U, ex, ey, ez, bx, by, bz, a.eps);
                }
                real vx;
                const real dvz = drift_velocity(drift, ux, uy, uz, vx, vy);
                const real dx = vx * a.dtdh[0];
                const real dy = DIM == 3 ? vy * a.dtdh[1] : real(0);
                // the drift's displacement (the ions' own) plus the record's
                // departure from it
                const real ddz = dvz * a.dtdh[2];
                const real dz = dz_drift + ddz;
                if (!(fabs(dx) < real(1) && fabs(dy) < real(1) && fabs(dz) < real(1))) {
                    atomicOr(a.err, (dx == dx && dy == dy && dz == dz) ? ERR_CFL : ERR_NAN);
                    valid = false;
                } else if (REL) {
                    // across z the reference stays, the departure moves
                    int fx, r1;
                    dlx1 = rel_step(dlx, dx, fx);
                    (void)rel_actual(orx, dlx1, r1);
                    mx = rx + fx - r1;
                    X0 = (double)rx + ((double)orx + (double)dlx);
                    X1 = (double)(rx + fx) + ((double)orx + (double)dlx1);
                    if (DIM == 3) {
                        int fy;
                        dly1 = rel_step(dly, dy, fy);
                        (void)rel_actual(ory, dly1, r1);
                        my = ry + fy - r1;
                        Y0 = (double)ry + ((double)ory + (double)dly);
                        Y1 = (double)(ry + fy) + ((double)ory + (double)dly1);
                    }
                    // along z the reference moves exactly like a drifting ion
                    // (same rounding, same cell changes)
                    real sref = add_rn(orz, dz_drift);
                    int sr = 0;
                    if (sref < real(0)) {
                        sref = sref + real(1);
                        sr = -1;
                        if (sref >= real(1)) { sref = 0; sr = 0; }
                    } else if (sref >= real(1)) {
                        sref = sref - real(1);
                        sr = 1;
                    }
                    int fz;
                    dlz1 = rel_step(dlz, ddz, fz);
                    (void)rel_actual(sref, dlz1, r1);
                    orz1 = sref;
                    mz = rz + sr + fz - r1;
                    Z0 = (double)rz + ((double)orz + (double)dlz);
                    Z1 = (double)(rz + sr + fz) + ((double)sref + (double)dlz1);
                } else {
                    x1 = ox + dx;
                    y1 = oy + dy;
                    z1 = add_rn(oz, dz_drift) + ddz;
                }
            }
            // ---- released ion: a record at the pair's position x^n, in the ion
            // side the IONS phase of this step reads (it moves and deposits it)
            if (__any_sync(0xffffffffu, release)) {
                const int r = reserve_slot(a.ion_in_hi, release ? t : -1);
                if (release) {
                    if (r >= g.cap) {
                        atomicOr(a.err, ERR_CAPACITY);
                    } else {
                        // (a paired record sits on its reference: orx = ox, ...)
                        const int64_t d = t * (int64_t)g.cap + (g.cap - 1 - r);
                        a.ion_in.ox[d] = REL ? orx : ox;
                        if (DIM == 3) a.ion_in.oy[d] = REL ? ory : oy;
                        a.ion_in.oz[d] = REL ? orz : oz;
                        a.ion_in.w[d] = w;
                        a.ion_in.cell[d] = pack_cell(g, ci, cj, ck);
                        if (a.ion_in.id) a.ion_in.id[d] = pid;
                    }
                }
            }
            const bool keep_pair = valid && paired && !release;  // exactly zero net current
            // ---- Esirkepov windows; the warp agrees on their lengths
            dep_t S0x[S + 2], DSx[S + 2], S0y[S + 2], DSy[S + 2], S0z[S + 2], DSz[S + 2];
            int ax = 0, ay = 0, az = 0;
            bool cx = false, cy = false, cz = false;
            if (valid && !keep_pair) {
                if (REL) {
                    ax = esirk_axis_g<S, dep_t>((dep_t)X0, (dep_t)X1, S0x, DSx, cx) + li + JL;
                    az = esirk_axis_g<S, dep_t>((dep_t)Z0, (dep_t)Z1, S0z, DSz, cz) + lk + JL;
                    if (DIM == 3) ay = esirk_axis_g<S, dep_t>((dep_t)Y0, (dep_t)Y1, S0y, DSy, cy) + lj + JL;
                } else {
                    ax = esirk_axis_c<S, dep_t>(ox, x1, S0x, DSx, cx) + li + JL;
                    az = esirk_axis_c<S, dep_t>(oz, z1, S0z, DSz, cz) + lk + JL;
                    if (DIM == 3) ay = esirk_axis_c<S, dep_t>(oy, y1, S0y, DSy, cy) + lj + JL;
                }
            }
            const unsigned sel = (__any_sync(0xffffffffu, cx) ? 4u : 0u) | (__any_sync(0xffffffffu, cy) ? 2u : 0u) |
                                 (__any_sync(0xffffffffu, cz) ? 1u : 0u);
            // 3D: no lane moved in x or y (e.g. plasma the laser has not reached)
            const bool z_only =
                DIM == 3 && __all_sync(0xffffffffu, !valid || keep_pair ||
                                                        (REL ? (X1 == X0 && Y1 == Y0) : (x1 == ox && y1 == oy)));
            int64_t dest = -1;
            int ni = 0, nj = 0, nk = 0;
            if (valid && keep_pair) {
                // moved exactly like its ion: no deposit
            } else if (valid) {
                // (the fixed-point factors are read from the parameters at each
                // use: held in registers they would cost spills here)
                const dep_t fz = (dep_t)a.jfac[2] * (dep_t)w * (dep_t)a.fx_scale[2];
                if (z_only) {
                    if (sel & 1u)
                        deposit_z<dep_t, acc_t, S, QX, QY, QN, S + 2>(sJ, S0x, S0y, S0z, DSz, ax, ay, az, fz,
                                                                      (dep_t)a.fx_lo[0]);
                    else
                        deposit_z<dep_t, acc_t, S, QX, QY, QN, S + 1>(sJ, S0x, S0y, S0z, DSz, ax, ay, az, fz,
                                                                      (dep_t)a.fx_lo[0]);
                } else {
                    deposit_sel<dep_t, acc_t, DIM, S, QX, QY, QN>(
                        sel, sJ, S0x, DSx, S0y, DSy, S0z, DSz, ax, ay, az,
                        (dep_t)a.jfac[0] * (dep_t)w * (dep_t)a.fx_scale[0],
                        (dep_t)a.jfac[1] * (dep_t)w * (dep_t)a.fx_scale[1], fz,
                        (dep_t)a.jyfac * (dep_t)w * (dep_t)vy * (dep_t)a.fx_scale[1], (dep_t)a.fx_lo[0]);
                }
            }
            if (valid) {
                // new cell and offsets; an offset that rounds to 1 moves on
                int sx, sy = 0, sz;
                if (REL) {
                    sx = mx;
                    sy = my;
                    sz = mz;
                    oz = orz1;  // x, y references do not move
                    ox = orx;
                    oy = ory;
                } else {
                    sx = (int)floor(x1);
                    sy = DIM == 3 ? (int)floor(y1) : 0;
                    sz = (int)floor(z1);
                    ox = x1 - real(sx);
                    if (ox >= real(1)) { sx += 1; ox = 0; }
                    if (DIM == 3) {
                        oy = y1 - real(sy);
                        if (oy >= real(1)) { sy += 1; oy = 0; }
                    }
                    oz = z1 - real(sz);
                    if (oz >= real(1)) { sz += 1; oz = 0; }
                }
                ni = ci + sx;
                if (ni < 0) ni += g.nx; else if (ni >= g.nx) ni -= g.nx;
                nj = cj + sy;
                if (DIM == 3) { if (nj < 0) nj += g.ny; else if (nj >= g.ny) nj -= g.ny; }
                nk = ck + sz;
                bool alive = true;
                if (g.bc_z == 0) {
                    if (nk < 0) nk += g.nz; else if (nk >= g.nz) nk -= g.nz;
                } else if (nk < 0 || nk >= g.nz) {
                    alive = false;
                }
                if (alive) dest = tile_of(g, ni, nj, nk);
            }
            // ---- write into the bucket of the destination tile
            const int r = output_slot(&s_stay, a.out_hi, dest, t, g.cap);
            if (dest >= 0) {
                if (r < 0) {
                    atomicOr(a.err, ERR_CAPACITY);
                } else {
                    const int64_t d = dest * (int64_t)g.cap + r;
                    a.out.ox[d] = ox;
                    if (DIM == 3) a.out.oy[d] = oy;
                    a.out.oz[d] = oz;
                    a.out.w[d] = w;
                    a.out.ux[d] = ux;
                    a.out.uy[d] = uy;
                    a.out.uz[d] = uz;
                    if (REL) {
                        a.out.dlx[d] = dlx1;
                        if (DIM == 3) a.out.dly[d] = dly1;
                        a.out.dlz[d] = dlz1;
                    }
                    a.out.cell[d] = (int32_t)((uint32_t)pack_cell(g, ni, nj, nk) | (keep_pair ? kPaired : 0u));
                    if (a.out.id) a.out.id[d] = pid;
                }
            }
        }
        __syncthreads();
        // the drifting ions of the tile, into the same current tile
        if (a.fuse_ions) {
            ions_of_tile<real, DIM, S, TX, TY, TZ, 3 * QN, REL>(g, a.ions, t, sJ + 2 * QN, sP, dz_drift,
                                                                 a.fx_scale[2], a.fx_lo[0], a.err, &s_stay_i);
        }
        // flush the J tile: one global add per non-zero node
        flush_tile<real, DIM, 3, QX, QY, QZ, JL>(g, Ptr3<real>{a.J[0], a.J[1], a.J[2]}, 0x4u, sJ, a.fx_quant[0],
                                                 a.fx_quant[1], a.fx_quant[2], a.fx_lo[1], lox, loy, loz);
        if (threadIdx.x == 0) {
            a.out_lo[t] = min(s_stay, g.cap);
            a.in_lo[t] = 0;
            a.in_hi[t] = 0;
        }
    }
}

// ------------------------------------------------------ drifting-ion tile

template <typename real, int DIM, int S, int TX, int TY, int TZ, bool REL>
__device__ __forceinline__ void ion_tile(const PushArgs<real> &a, const int64_t t, unsigned char *smem_raw)
{
    const Geom &g = a.g;
    constexpr int JL = S, JH = S + 1;
    constexpr int QX = TX + JL + JH, QY = DIM == 3 ? TY + JL + JH : 1, QZ = TZ + JL + JH;
    constexpr int QN = QX * QY * QZ;
    using acc_t = typename Acc<real>::type;
    acc_t *sJ = reinterpret_cast<acc_t *>(smem_raw);
    // prefetched records after the J tile ("hi" and, in FP32, "lo" words):
    // kIonStages buffers x 5 attributes x kBlock
    real *sP = reinterpret_cast<real *>(sJ + (sizeof(real) == 4 ? 2 : 1) * QN);
    const Drift<real> drift(a.u_drift, a.dtdh[2]);
    const real dz = drift.dz;
    const IonSide<real> &is = a.ions;
    __shared__ int s_stay;

    {
        if (is.in_lo[t] + is.in_hi[t] == 0) return;  // uniform over the CTA
        const int tix = (int)(t % g.nt[0]);
        const int tiy = (int)((t / g.nt[0]) % g.nt[1]);
        const int tiz = (int)(t / ((int64_t)g.nt[0] * g.nt[1]));
        const int lox = tix << g.lt[0], loy = tiy << g.lt[1], loz = tiz << g.lt[2];
        __syncthreads();
        for (int q = threadIdx.x; q < (sizeof(real) == 4 ? 2 : 1) * QN; q += blockDim.x) sJ[q] = 0;
        ions_of_tile<real, DIM, S, TX, TY, TZ, QN, REL>(g, is, t, sJ, sP, dz, a.fx_scale[2], a.fx_lo[0], a.err,
                                                        &s_stay);
        flush_tile<real, DIM, 1, QX, QY, QZ, JL>(g, Ptr3<real>{a.J[2], a.J[2], a.J[2]}, 0x1u, sJ, a.fx_quant[2],
                                                 a.fx_quant[2], a.fx_quant[2], a.fx_lo[1], lox, loy, loz);
    }
}

// the tile shapes the kernels are compiled for (pic_init_grid accepts these):
// 8 x 8 x 8 in 3D, and for CIC also 8 x 8 x 4; 16 x 16 in 2D, and for CIC
// also 32 x 8 and 8 x 32 (x, z)
constexpr int kTile3[3] = {8, 8, 8};
constexpr int kTile2[3] = {16, 1, 16};

template <typename real, int DIM, int S, int TX, int TY, int TZ, bool REL>
static size_t push_smem(bool ions)
{
    const int FN = (TX + 1 + S) * (DIM == 3 ? TY + 1 + S : 1) * (TZ + 1 + S);
    const int QN = (TX + 2 * S + 1) * (DIM == 3 ? TY + 2 * S + 1 : 1) * (TZ + 2 * S + 1);
    // FP32 currents take two words per node ("hi" and "lo"), FP64 one
    const int JW = sizeof(real) == 4 ? 2 : 1;
    static_assert(kIonStages * 5 <= 2 * 8, "the ion stages fit in the electrons' prefetch buffers");
    return ions ? sizeof(real) * (size_t)(JW * QN + kIonStages * 5 * kBlock)
                : sizeof(real) * (size_t)(6 * FN + JW * 3 * QN + 2 * (REL ? (DIM == 3 ? 11 : 10) : 8) * kBlock);
}

// the batched particle launches (pic_batch.cu): a persistent grid over the
// (run, tile) items of all runs; IONS selects the drifting-ion kernel
template <typename real, int DIM, int S, int TX, int TY, int TZ, bool REL, bool IONS>
void launch_push_batch(const void *args, const int64_t *start, int n, int64_t total, unsigned *queue, cudaStream_t s);

}  // namespace pic
