// pic_capi.cu -- host side of the C ABI declared in include/pic.h.
//
// Holds the small host context (parameters, derived simulation-frame
// quantities, the FP64 time accumulator, pointers into the caller's buffers)
// and enqueues the kernels of pic_particles.cu, pic_fields.cu and
// pic_inject.cu on the caller's stream.
#include "pic.h"
#include "pic_internal.cuh"

#include <cmath>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <array>
#include <atomic>
#include <new>
#include <string>
#include <vector>

using namespace pic;

namespace pic {
thread_local BatchRecorder *g_rec = nullptr;

int device_sms()
{
    constexpr int kDevices = 128;
    static std::atomic<int> cache[kDevices];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kDevices) return 1;
    int n = cache[dev].load(std::memory_order_relaxed);
    if (n > 0) return n;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) n = 1;
    cache[dev].store(n, std::memory_order_relaxed);
    return n;
}
}  // namespace pic

namespace {

constexpr double kPi = 3.141592653589793;
constexpr double kTwoPi = 6.283185307179586;
constexpr int kPartialBlocks = 1024;
constexpr size_t kAlign = 256;

size_t align_up(size_t n) { return (n + kAlign - 1) / kAlign * kAlign; }

int ceil_log2(int64_t n)
{
    int b = 0;
    while ((int64_t(1) << b) < n) ++b;
    return b;
}

struct SideLayout {       // byte offsets of the attribute arrays within one side
    size_t off[kAttrs];   // ox oy oz w ux uy uz cell id dz (SIZE_MAX: absent)
    size_t bytes;
};

struct StateHeader {
    char magic[8];
    int32_t dim, nx, ny, nz, precision, track_ids, has_ions, laser_on;
    int64_t n[2];
    double t;
    int64_t step;
    pic_laser_params laser;
    int32_t cur[2];
    double wmax;  // bound of the particle weights (fixed-point current scales)
    double win_v, win_t0;
    int32_t win_on, win_S;
    int64_t win_n;
    int32_t rel, pad0;  // electron records in relative form (their departure columns follow)
    char pad[512 - 8 - 8 * 4 - 16 - 8 - 8 - sizeof(pic_laser_params) - 8 - 8 - 16 - 8 - 8 - 8];
};
static_assert(sizeof(StateHeader) == 512, "state header must be 512 bytes");

}  // namespace

struct pic_ctx {
    pic_grid_params p{};
    Geom g{};
    cudaStream_t stream = nullptr;
    double gam = 1, beta = 0, hx = 1, hy = 1, hz = 1, dt = 0, Lx = 0, Ly = 0, Lz = 0, vol = 1;
    int es = 4;  // element bytes
    bool ions_species = false;
    bool rel = false;  // electron records in relative form (rel_actual)
    int sms = 152;     // multiprocessors of the device the buffers live on (set at binding)

    size_t field_bytes = 0, species_bytes[2] = {0, 0}, scratch_bytes = 0;
    int64_t slots = 0;
    SideLayout side[2]{};
    size_t off_cnt = 0, off_tmp = 0, off_offsets = 0, off_partials = 0, off_err = 0;
    // E and B live in two buffers that the Yee kernel alternates between (it
    // reads one and writes the other): the field buffer (fset 0) and a copy of
    // its first six components in scratch (fset 1)
    size_t off_eb = 0;
    int fset = 0;

    bool bound = false;
    unsigned char *fields = nullptr;
    unsigned char *species[2] = {nullptr, nullptr};
    unsigned char *scratch = nullptr;
    int cur[2] = {0, 0};

    // largest |weight| any particle loaded so far carries (weights never
    // change), the bound of the fixed-point current scales
    double wmax = 0;

    // moving window: from t0 on it moves at v along +z, by S cells at a time
    bool win_on = false;
    double win_v = 0, win_t0 = 0;
    int win_S = 0;
    int64_t win_n = 0;  // moves so far
    double zwin() const { return (double)win_n * win_S * hz; }

    // lab-frame snapshots (caller's device buffer)
    bool btd_on = false;
    pic_btd_params btd{};
    unsigned char *btd_buf = nullptr;
    size_t btd_flags_off = 0;

    bool plasma_loaded = false;
    pic_plasma_params plasma{};
    double prof[16] = {0};

    bool laser_on = false;
    pic_laser_params laser{};
    int ka = 2;

    double t = 0;
    int64_t step = 0;
    int64_t epoch = 0;  // bumped by every call that changes what a step launches
    int sort_every = 0; // order the buckets by cell before every sort_every-th step (0: never)
    std::string err;

    // adjoint run: the flat store's bands (slot base and lattice planes of
    // the load and of every step's injection), the step times, the caller's
    // buffer holding the checkpoints between the forward and reverse calls
    struct {
        bool ready = false;
        bool last_seg_ready = false;  // the forward left its last segment's states in place
        int N = 0, K = 0, K2 = 0;
        int64_t P = 0;
        std::vector<int64_t> base, mlo, mhi;
        std::vector<double> tn;
        unsigned char *buf = nullptr;
        size_t bytes = 0;
        double *hgrad = nullptr;  // pinned: the reverse sweep's sums as they leave the device
    } adj;

    // CUDA-graph capture of steps (batch): step cap_s of the graph being
    // captured takes its per-step scalars from cap_scal[cap_s] (device)
    bool capturing = false;
    const StepScal *cap_scal = nullptr;
    int cap_s = 0;
    int64_t inj_planes_max = 0;  // bound of an injection band (lattice planes)

    // profiling: event pairs recorded around phases, summed on read
    bool profiling = false;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<std::pair<int, size_t>> ev_used;  // (phase bit index, first event of the pair)
    int64_t kernels = 0;

    ~pic_ctx()
    {
        for (cudaEvent_t e : ev_pool) cudaEventDestroy(e);
        if (adj.hgrad) cudaFreeHost(adj.hgrad);
    }
};

// ------------------------------------------------------------------ helpers

static pic_status fail(pic_ctx *c, pic_status s, const std::string &msg)
{
    if (c) c->err = msg;
    return s;
}

#define CUDA_TRY(ctx, call)                                                                      \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess)                                                                   \
            return fail((ctx), PIC_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

// run lengths per tile of one side of one species: which 0 = bottom run (the
// tile's own CTA), 1 = top run (appended by others)
static int *counts(pic_ctx *c, int sp, int sidx, int which)
{
    return reinterpret_cast<int *>(c->scratch + c->off_cnt) +
           ((size_t)((2 * sp + sidx) * 2 + which)) * (size_t)c->g.ntiles;
}

// component comp (0..8: Ex Ey Ez Bx By Bz Jx Jy Jz) of the current fields;
// eb_other: E, B component comp (0..5) of the buffer the next Yee update writes
static void *field_ptr(pic_ctx *c, int comp)
{
    if (comp < 6 && c->fset) return c->scratch + c->off_eb + (size_t)comp * c->g.ncomp * c->es;
    return c->fields + (size_t)comp * c->g.ncomp * c->es;
}
static void *eb_other(pic_ctx *c, int comp)
{
    if (!c->fset) return c->scratch + c->off_eb + (size_t)comp * c->g.ncomp * c->es;
    return c->fields + (size_t)comp * c->g.ncomp * c->es;
}

template <typename real>
static Species<real> species_view(pic_ctx *c, int sp, int sidx)
{
    Species<real> s{};
    unsigned char *base = c->species[sp] + (size_t)sidx * c->side[sp].bytes;
    auto at = [&](int a) -> void * {
        return c->side[sp].off[a] == SIZE_MAX ? nullptr : (void *)(base + c->side[sp].off[a]);
    };
    s.ox = (real *)at(0);
    s.oy = (real *)at(1);
    s.oz = (real *)at(2);
    s.w = (real *)at(3);
    s.ux = (real *)at(4);
    s.uy = (real *)at(5);
    s.uz = (real *)at(6);
    s.cell = (int32_t *)at(7);
    s.id = (int64_t *)at(8);
    s.dlx = (real *)at(9);
    s.dly = (real *)at(10);
    s.dlz = (real *)at(11);
    return s;
}

static void side_raw(pic_ctx *c, int sp, int sidx, void *out[kAttrs])
{
    unsigned char *base = c->species[sp] + (size_t)sidx * c->side[sp].bytes;
    for (int a = 0; a < kAttrs; ++a)
        out[a] = c->side[sp].off[a] == SIZE_MAX ? nullptr : (void *)(base + c->side[sp].off[a]);
}

static cudaMemcpyKind kind_out(int dst_is_device) { return dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost; }
static cudaMemcpyKind kind_in(int src_is_device) { return src_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice; }

static size_t attr_size(const pic_ctx *c, int a) { return a == 7 ? 4 : (a == 8 ? 8 : (size_t)c->es); }

// the plasma's drift momentum U (u = (0, 0, U)) in the working precision:
// -gamma beta in a boosted frame, 0 in the lab frame.  Electron records store
// u - (0, 0, U); the drifting ions move with it.
template <typename real>
static real drift_u(const pic_ctx *c)
{
    return (real)(-(c->gam * c->beta));
}

static pic_status check_device_error(pic_ctx *c)
{
    unsigned h = 0;
    unsigned *d = reinterpret_cast<unsigned *>(c->scratch + c->off_err);
    CUDA_TRY(c, cudaMemcpyAsync(&h, d, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    if (h == 0) return PIC_OK;
    CUDA_TRY(c, cudaMemsetAsync(d, 0, sizeof(unsigned), c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    if (h & ERR_NAN) return fail(c, PIC_ERR_NAN, "a non-finite particle momentum or position was produced");
    if (h & ERR_CFL) return fail(c, PIC_ERR_CFL, "a particle moved one cell or more in one step");
    if (h & ERR_CAPACITY) return fail(c, PIC_ERR_CAPACITY, "a tile bucket overflowed (raise slots_per_cell)");
    if (h & ERR_TIMEOUT) return fail(c, PIC_ERR_TIMEOUT, "a bounded device wait ran out (a staged copy did not land)");
    return fail(c, PIC_ERR_STATE, "a particle was found outside its tile bucket");
}

// ------------------------------------------------------------------- set-up

extern "C" pic_status pic_init_grid(const pic_grid_params *p, pic_ctx **out)
{
    if (!out) return PIC_ERR_ARG;
    *out = nullptr;
    if (!p) return PIC_ERR_ARG;
    if (p->dim != 2 && p->dim != 3) return PIC_ERR_ARG;
    if (p->nx < 1 || p->nz < 4 || (p->dim == 3 && p->ny < 1) || (p->dim == 2 && p->ny != 1)) return PIC_ERR_ARG;
    if (!(p->dx > 0) || !(p->dz > 0) || (p->dim == 3 && !(p->dy > 0))) return PIC_ERR_ARG;
    if (!(p->cfl > 0)) return PIC_ERR_ARG;
    if (!(p->cfl < 1)) return PIC_ERR_CFL;
    if (!(p->gamma_boost >= 1) || !std::isfinite(p->gamma_boost)) return PIC_ERR_ARG;
    if (p->shape_order != 1 && p->shape_order != 2) return PIC_ERR_ARG;
    if (p->filter_passes < 0 || p->filter_passes > 64) return PIC_ERR_ARG;
    if (p->bc_z != PIC_BC_MUR && p->bc_z != PIC_BC_PERIODIC) return PIC_ERR_ARG;
    if (p->precision != PIC_FP32 && p->precision != PIC_FP64) return PIC_ERR_ARG;
    if (!(p->slots_per_cell > 0) || p->slots_per_cell > 4096) return PIC_ERR_ARG;
    if (p->z_relative < 0 || p->z_relative > 2) return PIC_ERR_ARG;
    for (int d = 0; d < 3; ++d)
        if (p->tile[d] < 0 || (p->tile[d] & (p->tile[d] - 1))) return PIC_ERR_ARG;

    pic_ctx *c = new (std::nothrow) pic_ctx();
    if (!c) return PIC_ERR_ARG;
    c->p = *p;
    c->stream = static_cast<cudaStream_t>(p->stream);
    c->es = p->precision == PIC_FP64 ? 8 : 4;

    // simulation-frame quantities (FP64): beta, contracted-grid cell sizes, dt
    c->gam = p->gamma_boost;
    c->beta = std::sqrt(1.0 - 1.0 / (c->gam * c->gam));
    c->hx = p->dx;
    c->hy = p->dim == 3 ? p->dy : 1.0;
    c->hz = p->dz * (c->gam * (1.0 + c->beta));
    if (p->dim == 3)
        c->dt = p->cfl / std::sqrt(1.0 / (c->hx * c->hx) + 1.0 / (c->hy * c->hy) + 1.0 / (c->hz * c->hz));
    else
        c->dt = p->cfl / std::sqrt(1.0 / (c->hx * c->hx) + 1.0 / (c->hz * c->hz));
    c->Lx = p->nx * c->hx;
    c->Ly = (p->dim == 3 ? p->ny : 1) * c->hy;
    c->Lz = p->nz * c->hz;
    c->vol = p->dim == 3 ? c->hx * c->hy * c->hz : c->hx * c->hz;
    c->ions_species = c->gam > 1.0;
    c->rel = p->z_relative == 1 || (p->z_relative == 0 && c->gam >= 50.0);

    Geom &g = c->g;
    g.dim = p->dim;
    g.nx = p->nx;
    g.ny = p->dim == 3 ? p->ny : 1;
    g.nz = p->nz;
    g.bc_z = p->bc_z == PIC_BC_PERIODIC ? 0 : 1;
    g.shape = p->shape_order;
    g.bx = ceil_log2(g.nx) > 0 ? ceil_log2(g.nx) : 1;
    g.by = p->dim == 3 ? ceil_log2(g.ny) : 0;
    const int bz = ceil_log2(g.nz);
    if (g.bx + g.by + bz > 31) {
        delete c;
        return PIC_ERR_ARG;
    }
    // the particle kernels are compiled for two tile shapes in 3D (8 x 8 x 8,
    // and for the CIC shape 8 x 8 x 4) and three in 2D (16 x 16, 32 x 8,
    // 8 x 32 cells along x, z; the last two for the CIC shape only); a zero
    // entry takes the default
    int def2[3] = {16, 1, 16};
    int def3[3] = {8, 8, 8};
    if (p->dim == 3 && p->tile[2] == 4) {
        if (p->shape_order != 1) {
            delete c;
            return PIC_ERR_ARG;
        }
        def3[2] = 4;
    }
    if (p->dim == 2 && (p->tile[0] != 0 || p->tile[2] != 0)) {
        const int tx = p->tile[0] ? p->tile[0] : 16, tz = p->tile[2] ? p->tile[2] : 16;
        const bool ok = (tx == 16 && tz == 16) || (p->shape_order == 1 && ((tx == 32 && tz == 8) || (tx == 8 && tz == 32)));
        if (!ok) {
            delete c;
            return PIC_ERR_ARG;
        }
        def2[0] = tx;
        def2[2] = tz;
    }
    const int ncell[3] = {g.nx, g.ny, g.nz};
    int64_t cells_per_tile = 1;
    for (int d = 0; d < 3; ++d) {
        const int t = p->dim == 3 ? def3[d] : def2[d];
        if (p->tile[d] != 0 && p->tile[d] != t && !(p->dim == 2 && d == 1)) {
            delete c;
            return PIC_ERR_ARG;
        }
        g.lt[d] = ceil_log2(t);
        g.nt[d] = (ncell[d] + t - 1) / t;
        cells_per_tile *= t;
    }
    g.ntiles = (int64_t)g.nt[0] * g.nt[1] * g.nt[2];
    int64_t cap = (int64_t)std::ceil(p->slots_per_cell * (double)cells_per_tile);
    cap = (cap + 31) / 32 * 32;
    if (cap < 32) cap = 32;
    if (cap > (1 << 24)) {
        delete c;
        return PIC_ERR_ARG;
    }
    g.cap = (int)cap;
    g.plane = (int64_t)g.nx * g.ny;
    g.ncomp = (int64_t)(g.nz + 1) * g.plane;
    c->slots = g.ntiles * (int64_t)g.cap;

    // buffer layout
    c->field_bytes = (size_t)PIC_NCOMP * (size_t)g.ncomp * c->es;
    for (int sp = 0; sp < 2; ++sp) {
        SideLayout &L = c->side[sp];
        size_t o = 0;
        for (int a = 0; a < kAttrs; ++a) {
            bool present = true;
            if (a == 1 && p->dim != 3) present = false;
            if (sp == 1 && a >= 4 && a <= 6) present = false;
            if (a == 8 && !p->track_ids) present = false;
            if (a >= 9 && (sp == 1 || !c->rel)) present = false;  // departures dlx dly dlz
            if (a == 10 && p->dim != 3) present = false;
            if (!present) {
                L.off[a] = SIZE_MAX;
                continue;
            }
            L.off[a] = o;
            o += align_up((size_t)c->slots * attr_size(c, a));
        }
        L.bytes = o;
        c->species_bytes[sp] = (sp == 1 && !c->ions_species) ? 0 : 2 * o;
    }
    size_t o = 0;
    c->off_cnt = o;
    o += align_up(sizeof(int) * 8 * (size_t)g.ntiles);
    c->off_tmp = o;
    o += align_up((size_t)3 * g.ncomp * c->es);
    c->off_offsets = o;
    o += align_up(sizeof(int64_t) * (size_t)g.ntiles);
    c->off_partials = o;
    o += align_up(sizeof(double) * 3 * kPartialBlocks);
    c->off_err = o;
    o += kAlign;
    c->off_eb = o;
    o += align_up((size_t)6 * g.ncomp * c->es);
    c->scratch_bytes = o;
    c->plasma.ions = 0;
    *out = c;
    return PIC_OK;
}

extern "C" pic_status pic_query_sizes(const pic_ctx *c, pic_sizes *s)
{
    if (!c || !s) return PIC_ERR_ARG;
    std::memset(s, 0, sizeof(*s));
    s->field_bytes = c->field_bytes;
    s->species_bytes[0] = c->species_bytes[0];
    s->species_bytes[1] = c->species_bytes[1];
    s->scratch_bytes = c->scratch_bytes;
    s->slots[0] = c->slots;
    s->slots[1] = c->ions_species ? c->slots : 0;
    s->ntiles = c->g.ntiles;
    s->tile_capacity = c->g.cap;
    for (int d = 0; d < 3; ++d) s->tile[d] = 1 << c->g.lt[d];
    s->elem_bytes = c->es;
    s->dt = c->dt;
    s->hx = c->hx;
    s->hy = c->hy;
    s->hz = c->hz;
    s->beta = c->beta;
    return PIC_OK;
}

extern "C" pic_status pic_bind_buffers(pic_ctx *c, const pic_buffers *b)
{
    if (!c || !b) return PIC_ERR_ARG;
    c->epoch += 1;
    if (c->bound) return fail(c, PIC_ERR_STATE, "buffers are already bound");
    auto aligned = [](const void *q) { return ((uintptr_t)q % kAlign) == 0; };
    if (!b->fields || !b->species[0] || !b->scratch) return fail(c, PIC_ERR_ARG, "null buffer");
    if (c->species_bytes[1] && !b->species[1]) return fail(c, PIC_ERR_ARG, "null ion buffer");
    if (!aligned(b->fields) || !aligned(b->species[0]) || !aligned(b->scratch) ||
        (c->species_bytes[1] && !aligned(b->species[1])))
        return fail(c, PIC_ERR_ARG, "buffers must be 256-byte aligned");
    c->fields = (unsigned char *)b->fields;
    c->species[0] = (unsigned char *)b->species[0];
    c->species[1] = (unsigned char *)b->species[1];
    c->scratch = (unsigned char *)b->scratch;
    CUDA_TRY(c, cudaMemsetAsync(c->fields, 0, c->field_bytes, c->stream));
    CUDA_TRY(c, cudaMemsetAsync(c->scratch, 0, c->scratch_bytes, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && n > 0)
        c->sms = n;
    c->fset = 0;
    c->bound = true;
    return PIC_OK;
}

// --------------------------------------------------------------- plasma

static void fill_inject_common(pic_ctx *c, InjectArgs &a)
{
    const pic_plasma_params &p = c->plasma;
    a.g = c->g;
    a.hx = c->hx;
    a.hy = c->hy;
    a.hz = c->hz;
    a.Lx = c->Lx;
    a.Ly = c->Ly;
    a.Lz = c->Lz;
    a.gam = c->gam;
    a.beta = c->beta;
    a.ppx = p.ppc[0];
    a.ppy = c->g.dim == 3 ? p.ppc[1] : 1;
    a.ppz = p.ppc[2];
    a.NX = (int64_t)c->g.nx * a.ppx;
    a.NY = c->g.dim == 3 ? (int64_t)c->g.ny * a.ppy : 1;
    a.z_start = p.z_start;
    a.z_end = p.z_end;
    a.ramp = p.ramp_len;
    a.ne = p.ne_over_nc;
    a.jitter = p.jitter;
    a.hz_lab = c->gam * c->hz;
    a.dzl = a.hz_lab / (double)a.ppz;
    a.wfac = c->gam * c->vol / (double)(a.ppx * a.ppy * a.ppz);
    a.nprof = p.n_profile;
    for (int m = 0; m < 16; ++m) a.prof[m] = m < p.n_profile ? c->prof[m] : 0.0;
    a.seed = c->p.seed;
    a.zwin = c->zwin();
    a.zmin = 0.0;
    a.drift_ions = (p.ions && c->ions_species) ? 1 : 0;
    a.paired = (a.drift_ions && !c->p.explicit_ions) ? 1 : 0;
    a.precision = c->p.precision;
    side_raw(c, 0, c->cur[0], a.sp_e);
    a.hi_e = counts(c, 0, c->cur[0], 1);
    if (a.drift_ions) {
        side_raw(c, 1, c->cur[1], a.sp_i);
        a.hi_i = counts(c, 1, c->cur[1], 1);
    } else {
        for (int q = 0; q < kAttrs; ++q) a.sp_i[q] = nullptr;
        a.hi_i = nullptr;
    }
    a.err = reinterpret_cast<unsigned *>(c->scratch + c->off_err);
    a.flat_base = -1;  // into the tile buckets
}

// lattice planes whose lab z may fall in [zlo, zhi) after jitter
static void lattice_band(const InjectArgs &a, double zlo, double zhi, int64_t &m_lo, int64_t &m_hi)
{
    const int64_t MZ = (int64_t)std::ceil((a.z_end - a.z_start) / a.dzl);
    const double jm = a.jitter * a.hz_lab + a.dzl;
    double lo = std::floor((zlo - a.z_start - jm) / a.dzl - 0.5) - 1.0;
    double hi = std::ceil((zhi - a.z_start + jm) / a.dzl - 0.5) + 2.0;
    if (lo < 0) lo = 0;
    if (hi > (double)MZ) hi = (double)MZ;
    m_lo = (int64_t)lo;
    m_hi = (int64_t)hi;
    if (m_hi < m_lo) m_hi = m_lo;
}

extern "C" pic_status pic_load_plasma(pic_ctx *c, const pic_plasma_params *p)
{
    if (!c || !p) return PIC_ERR_ARG;
    c->epoch += 1;
    if (!c->bound) return fail(c, PIC_ERR_STATE, "bind buffers first");
    const bool dim3 = c->g.dim == 3;
    if (!(p->ne_over_nc >= 0) || !(p->z_end > p->z_start) || !(p->ramp_len >= 0) || p->ppc[0] < 1 ||
        p->ppc[2] < 1 || (dim3 && p->ppc[1] < 1) || !(p->jitter >= 0 && p->jitter < 0.5) || p->n_profile < 0 ||
        p->n_profile > 16 || (p->n_profile > 0 && !p->profile))
        return fail(c, PIC_ERR_ARG, "invalid plasma parameters");
    c->plasma = *p;
    c->adj.ready = false;  // an adjoint forward run recorded before this is another run's
    for (int m = 0; m < 16; ++m) c->prof[m] = m < p->n_profile ? p->profile[m] : 0.0;
    c->plasma.profile = c->prof;
    c->plasma_loaded = true;
    InjectArgs a{};
    fill_inject_common(c, a);
    {
        // the lab density is at most ne (1 + sum |c_m|); the margin covers the
        // rounding of the weight to the working precision
        double f = 1.0;
        for (int m = 0; m < p->n_profile; ++m) f += std::fabs(p->profile[m]);
        c->wmax = std::max(c->wmax, std::fabs(p->ne_over_nc) * f * a.wfac * (1.0 + 1e-6));
    }
    a.mode = 0;
    a.t = c->t;
    a.t1 = c->t;
    // every lattice plane whose simulation-frame position lies in [0, Lz)
    lattice_band(a, c->gam * (c->zwin() + c->beta * c->t), c->gam * (c->zwin() + c->Lz + c->beta * c->t), a.m_lo,
                 a.m_hi);
    launch_inject(a, c->stream);
    CUDA_TRY(c, cudaGetLastError());
    return check_device_error(c);
}

// host FP64 position -> cell + offset in the working precision (same rules as
// the device loader: offsets in [0,1), an offset that rounds to 1 moves on)
template <typename real>
static bool host_to_cell(double x, double h, int n, bool periodic, int &cell, real &off)
{
    const double xi = x / h;
    const double f = std::floor(xi);
    if (!(f >= 0) || f > (double)n) return false;
    cell = (int)f;
    double o = xi - f;
    if (cell >= n) {
        if (periodic) cell -= n;
        else { cell = n - 1; o = (double)below_one<real>(); }
    }
    off = (real)o;
    if (off >= real(1)) {
        if (cell + 1 < n) { cell += 1; off = 0; }
        else if (periodic) { cell = 0; off = 0; }
        else off = below_one<real>();
    }
    return true;
}

// bucket slots [0, n) of the inactive (staging) side into the active side
template <typename real>
static pic_status bucket_staged(pic_ctx *c, int sp, int64_t n)
{
    const int stage = c->cur[sp] ^ 1;
    BucketArgs<real> b{};
    b.g = c->g;
    b.src = species_view<real>(c, sp, stage);
    b.dst = species_view<real>(c, sp, c->cur[sp]);
    b.n = n;
    b.dst_hi = counts(c, sp, c->cur[sp], 1);
    b.err = reinterpret_cast<unsigned *>(c->scratch + c->off_err);
    launch_bucket<real>(b, c->stream);
    CUDA_TRY(c, cudaGetLastError());
    return check_device_error(c);
}

// copy flat columns (host or device) into the staging side, then bucket them
template <typename real>
static pic_status upload_flat(pic_ctx *c, int sp, int64_t n, const void *const cols[kAttrs], int src_is_device)
{
    void *dst[kAttrs];
    side_raw(c, sp, c->cur[sp] ^ 1, dst);
    for (int a = 0; a < kAttrs; ++a) {
        if (!dst[a]) continue;
        const size_t bytes = (size_t)n * attr_size(c, a);
        if (bytes == 0) continue;
        CUDA_TRY(c, cudaMemcpyAsync(dst[a], cols[a], bytes, kind_in(src_is_device), c->stream));
    }
    return bucket_staged<real>(c, sp, n);
}

template <typename real>
static pic_status load_particles_t(pic_ctx *c, int sp, int64_t n, const double *state, const int64_t *ids)
{
    const bool dim3 = c->g.dim == 3;
    // (zero-filled: a loaded electron sits on its drift reference, dz = 0)
    std::vector<std::vector<unsigned char>> cols(kAttrs);
    for (int a = 0; a < kAttrs; ++a)
        if (c->side[sp].off[a] != SIZE_MAX) cols[a].resize((size_t)n * attr_size(c, a));
    auto R = [&](int a) { return reinterpret_cast<real *>(cols[a].data()); };
    double wmax = 0;
    for (int64_t i = 0; i < n; ++i) {
        double x = state[0 * n + i], y = state[1 * n + i], z = state[2 * n + i];
        int ci = 0, cj = 0, ck = 0;
        real ox, oy = 0, oz;
        if (!(x >= 0 && x < c->Lx) || !(z >= 0 && z < c->Lz) || (dim3 && !(y >= 0 && y < c->Ly)))
            return fail(c, PIC_ERR_ARG, "particle outside the box");
        if (!std::isfinite(state[6 * n + i])) return fail(c, PIC_ERR_ARG, "non-finite particle weight");
        if (!host_to_cell<real>(x, c->hx, c->g.nx, true, ci, ox) ||
            !host_to_cell<real>(z, c->hz, c->g.nz, c->g.bc_z == 0, ck, oz) ||
            (dim3 && !host_to_cell<real>(y, c->hy, c->g.ny, true, cj, oy)))
            return fail(c, PIC_ERR_ARG, "particle outside the box");
        R(0)[i] = ox;
        if (dim3) R(1)[i] = oy;
        R(2)[i] = oz;
        R(3)[i] = (real)state[6 * n + i];
        wmax = std::max(wmax, std::fabs(state[6 * n + i]) * (1.0 + 1e-6));
        if (sp == 0) {  // stored relative to the plasma drift
            R(4)[i] = (real)state[3 * n + i];
            R(5)[i] = (real)state[4 * n + i];
            R(6)[i] = (real)(state[5 * n + i] - (double)drift_u<real>(c));
        }
        reinterpret_cast<int32_t *>(cols[7].data())[i] = pack_cell(c->g, ci, cj, ck);
        if (c->p.track_ids) reinterpret_cast<int64_t *>(cols[8].data())[i] = ids ? ids[i] : i;
    }
    const void *ptrs[kAttrs];
    for (int a = 0; a < kAttrs; ++a) ptrs[a] = cols[a].empty() ? nullptr : cols[a].data();
    c->wmax = std::max(c->wmax, wmax);
    return upload_flat<real>(c, sp, n, ptrs, 0);
}

extern "C" pic_status pic_load_particles(pic_ctx *c, int sp, int64_t n, const double *state, const int64_t *ids)
{
    if (!c || (sp != 0 && sp != 1) || n < 0 || (n > 0 && !state)) return PIC_ERR_ARG;
    c->epoch += 1;
    if (!c->bound) return fail(c, PIC_ERR_STATE, "bind buffers first");
    if (sp == 1 && !c->ions_species) return fail(c, PIC_ERR_ARG, "drifting ions exist only in a boosted frame");
    if (n > c->slots) return fail(c, PIC_ERR_CAPACITY, "more particles than slots");
    if (n == 0) return PIC_OK;
    return c->es == 4 ? load_particles_t<float>(c, sp, n, state, ids) : load_particles_t<double>(c, sp, n, state, ids);
}

extern "C" pic_status pic_launch_laser(pic_ctx *c, const pic_laser_params *p)
{
    if (!c || !p) return PIC_ERR_ARG;
    c->epoch += 1;
    if (!(p->a0 >= 0) || !(p->waist > 0) || !(p->fwhm > 0) || !std::isfinite(p->z_antenna) ||
        (p->polarization != PIC_POL_X && p->polarization != PIC_POL_Y))
        return fail(c, PIC_ERR_ARG, "invalid laser parameters");
    c->laser = *p;
    c->adj.ready = false;  // as in pic_load_plasma
    int ka = (int)std::floor(p->z_antenna / c->hz + 0.5);
    if (ka < 2) ka = 2;
    if (ka > c->g.nz - 2) ka = c->g.nz - 2;
    c->ka = ka;
    if (std::isnan(c->laser.x_center)) c->laser.x_center = 0.5 * c->Lx;
    if (std::isnan(c->laser.y_center)) c->laser.y_center = 0.5 * c->Ly;
    c->laser_on = true;
    return PIC_OK;
}

// ---------------------------------------------------------------------- step

// Scales of the FP32 fixed-point current accumulation (see sh_acc).  Every
// contribution of one particle to one node of a component is at most
// C_c = |f_c| w_max in magnitude (f_c the component's current factor before
// the weight: the running sums of the shape differences lie in [-1, 1], the
// path-averaged shape products in [0, 1], |v_y| < 1), and a node of a tile
// receives at most one contribution per particle of the tile, at most cap of
// them.  The scale lim / C_c with lim = min(2^30 / cap, 2^21) keeps every
// rounded contribution below 2^21 and every node's "hi" sum below
// 2^30 + cap / 2; the "lo" words take K = min(22, 30 - ceil(log2 cap)) bits
// of the remainders, so their sums stay below cap 2^(K-1) <= 2^29.  The
// scales are the same for electrons and ions, so the contributions of an
// electron and an ion on the same path cancel exactly.
template <typename real>
static void fixed_point_scales(const pic_ctx *c, int nsources, real scale[3], real quant[3], real lo[2])
{
    if (sizeof(real) != 4) {
        for (int q = 0; q < 3; ++q) scale[q] = quant[q] = real(1);
        lo[0] = lo[1] = real(1);
        return;
    }
    // a node of a current tile takes at most one contribution from each of
    // the tile's records: nsources buckets of cap records each
    const int cap = c->g.cap * nsources;
    int lg = 0;
    while ((1LL << lg) < (long long)cap) ++lg;  // ceil(log2 cap)
    const int k = std::min(22, 30 - lg);
    const double lim = std::min(std::ldexp(1.0, 30) / cap, std::ldexp(1.0, 21));
    const double f[3] = {c->hx / (c->dt * c->vol), c->g.dim == 3 ? c->hy / (c->dt * c->vol) : 1.0 / c->vol,
                         c->hz / (c->dt * c->vol)};
    for (int q = 0; q < 3; ++q) {
        const double cb = f[q] * c->wmax;
        scale[q] = cb > 0 ? (real)(lim / cb) : real(0);
        quant[q] = cb > 0 ? (real)(cb / lim) : real(0);
    }
    lo[0] = (real)std::ldexp(1.0, k);
    lo[1] = (real)std::ldexp(1.0, -k);
}

template <typename real>
static PushArgs<real> push_args(pic_ctx *c, int sp)
{
    PushArgs<real> a{};
    a.g = c->g;
    real *F[9];
    for (int q = 0; q < 9; ++q) F[q] = (real *)field_ptr(c, q);
    for (int q = 0; q < 3; ++q) {
        a.E[q] = F[q];
        a.B[q] = F[3 + q];
        a.J[q] = F[6 + q];
    }
    a.in = species_view<real>(c, sp, c->cur[sp]);
    a.out = species_view<real>(c, sp, c->cur[sp] ^ 1);
    a.in_lo = counts(c, sp, c->cur[sp], 0);
    a.in_hi = counts(c, sp, c->cur[sp], 1);
    a.out_lo = counts(c, sp, c->cur[sp] ^ 1, 0);
    a.out_hi = counts(c, sp, c->cur[sp] ^ 1, 1);
    a.dtdh[0] = (real)(c->dt / c->hx);
    a.dtdh[1] = (real)(c->dt / c->hy);
    a.dtdh[2] = (real)(c->dt / c->hz);
    const double q = sp == 0 ? -1.0 : 1.0;
    a.eps = (real)(kPi * -1.0 * c->dt);
    a.jfac[0] = (real)(-q * c->hx / (c->dt * c->vol));
    a.jfac[1] = (real)(-q * c->hy / (c->dt * c->vol));
    a.jfac[2] = (real)(-q * c->hz / (c->dt * c->vol));
    a.jyfac = (real)(q / c->vol);
    a.u_drift = drift_u<real>(c);
    a.rel = c->rel ? 1 : 0;
    fixed_point_scales(c, 1, a.fx_scale, a.fx_quant, a.fx_lo);
    if (c->ions_species) {
        a.ion_in = species_view<real>(c, 1, c->cur[1]);
        a.ion_in_hi = counts(c, 1, c->cur[1], 1);
    }
    a.err = reinterpret_cast<unsigned *>(c->scratch + c->off_err);
    return a;
}

// the drifting-ion species of this step: the side the step reads, the side
// it writes, their bucket counters and the ions' current factor (q = +1)
template <typename real>
static IonSide<real> ion_side(pic_ctx *c)
{
    IonSide<real> s{};
    s.in = species_view<real>(c, 1, c->cur[1]);
    s.out = species_view<real>(c, 1, c->cur[1] ^ 1);
    s.in_lo = counts(c, 1, c->cur[1], 0);
    s.in_hi = counts(c, 1, c->cur[1], 1);
    s.out_lo = counts(c, 1, c->cur[1] ^ 1, 0);
    s.out_hi = counts(c, 1, c->cur[1] ^ 1, 1);
    s.jfac_z = (real)(-1.0 * c->hz / (c->dt * c->vol));
    return s;
}

// records an event pair around one phase when profiling is on
struct PhaseTimer {
    pic_ctx *c;
    int bit;
    size_t first = SIZE_MAX;
    PhaseTimer(pic_ctx *ctx, int b) : c(ctx), bit(b)
    {
        if (!c->profiling) return;
        first = c->ev_used.empty() ? 0 : c->ev_used.back().second + 2;
        while (c->ev_pool.size() < first + 2) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) {
                first = SIZE_MAX;
                return;
            }
            c->ev_pool.push_back(e);
        }
        cudaEventRecord(c->ev_pool[first], c->stream);
    }
    ~PhaseTimer()
    {
        if (first == SIZE_MAX) return;
        cudaEventRecord(c->ev_pool[first + 1], c->stream);
        c->ev_used.push_back({bit, first});
    }
};

// Move the window by S cells: fields (E, B into the other buffer, J through
// the scratch buffer), each species' buckets m = S / tz tile layers down, then
// the plasma of the newly covered layer [Lz - S hz, Lz) (relative to the
// moved window) at the current time.
template <typename real>
static void window_move(pic_ctx *c)
{
    const int S = c->win_S;
    real *src[9], *dst[9];
    for (int q = 0; q < 6; ++q) {
        src[q] = (real *)field_ptr(c, q);
        dst[q] = (real *)eb_other(c, q);
    }
    real *tmp = (real *)(c->scratch + c->off_tmp);
    for (int q = 0; q < 3; ++q) {
        src[6 + q] = (real *)field_ptr(c, 6 + q);
        dst[6 + q] = tmp + (size_t)q * c->g.ncomp;
    }
    launch_window_fields<real>(c->g, src, dst, S, c->stream);
    cudaMemcpyAsync(field_ptr(c, 6), tmp, (size_t)3 * c->g.ncomp * sizeof(real), cudaMemcpyDeviceToDevice,
                    c->stream);
    c->fset ^= 1;
    c->kernels += 1;
    const int m = S >> c->g.lt[2];
    for (int sp = 0; sp < 2; ++sp) {
        if (sp == 1 && !c->ions_species) break;
        launch_window_particles<real>(c->g, species_view<real>(c, sp, c->cur[sp]),
                                      species_view<real>(c, sp, c->cur[sp] ^ 1), counts(c, sp, c->cur[sp], 0),
                                      counts(c, sp, c->cur[sp], 1), counts(c, sp, c->cur[sp] ^ 1, 0),
                                      counts(c, sp, c->cur[sp] ^ 1, 1), m, S, c->stream);
        cudaMemsetAsync(counts(c, sp, c->cur[sp], 0), 0, sizeof(int) * 2 * (size_t)c->g.ntiles, c->stream);
        c->cur[sp] ^= 1;
        c->kernels += 1;
    }
    c->win_n += 1;
    if (c->plasma_loaded) {
        InjectArgs a{};
        fill_inject_common(c, a);
        a.mode = 0;
        a.t = c->t;
        a.t1 = c->t;
        a.zmin = c->Lz - S * c->hz;
        lattice_band(a, c->gam * (c->zwin() + a.zmin + c->beta * c->t), c->gam * (c->zwin() + c->Lz + c->beta * c->t),
                     a.m_lo, a.m_hi);
        launch_inject(a, c->stream);
        if (a.m_hi > a.m_lo) c->kernels += 1;
    }
}

static int btd_nxs(const pic_ctx *c, const pic_btd_params *p) { return p->plane ? c->g.nx : 1; }

// Lab snapshot points whose event falls in this step (E0, B0: the fields at
// its start, E1, B1 at its end): per snapshot a range of lab points that holds
// them all (the kernel decides each point exactly).  Returns the launches.
template <typename real>
static int fill_btd(pic_ctx *c, real *const F0[9], real *const F1[6])
{
    const pic_btd_params &p = c->btd;
    BtdArgs<real> a{};
    a.g = c->g;
    for (int q = 0; q < 3; ++q) {
        a.E0[q] = F0[q];
        a.B0[q] = F0[3 + q];
        a.E1[q] = F1[q];
        a.B1[q] = F1[3 + q];
    }
    a.data = reinterpret_cast<real *>(c->btd_buf);
    a.flags = reinterpret_cast<int *>(c->btd_buf + c->btd_flags_off);
    a.gam = c->gam;
    a.beta = c->beta;
    a.hz = c->hz;
    a.zwin = c->zwin();
    a.t0 = c->t;
    a.dt = c->dt;
    a.T0 = p.t0;
    a.dT = p.dt;
    a.Z0 = p.z0;
    a.dZ = p.dz;
    a.nsnap = p.n_snapshots;
    a.nz = p.nz;
    a.nxs = btd_nxs(c, &p);
    bool any = false;
    for (int j = 0; j < p.n_snapshots; ++j) {
        // t0 <= gamma (T - beta Z) < t0 + dt  <=>  Z in ((T - (t0+dt)/gamma)/beta, (T - t0/gamma)/beta]
        const double T = p.t0 + j * p.dt;
        const double zlo = (T - (c->t + c->dt) / c->gam) / c->beta, zhi = (T - c->t / c->gam) / c->beta;
        double klo = std::floor((zlo - p.z0) / p.dz) - 1.0, khi = std::ceil((zhi - p.z0) / p.dz) + 1.0;
        if (klo < 0.0) klo = 0.0;
        if (khi > (double)(p.nz - 1)) khi = (double)(p.nz - 1);
        a.klo[j] = (int)klo;
        a.kn[j] = khi >= klo ? (int)(khi - klo) + 1 : 0;
        any = any || a.kn[j] > 0;
    }
    if (!any) return 0;
    launch_btd<real>(a, c->stream);
    return 1;
}

// The antenna's sheet current amplitude in the step starting at t: the lab
// laser seen by an antenna at rest in the boosted frame, amplitude and time
// argument scaled by D = gamma (1 - beta); J = -E_target / (pi hz).
static double antenna_j0(const pic_ctx *c, double t, double a0)
{
    const pic_laser_params &l = c->laser;
    const double D = 1.0 / (c->gam * (1.0 + c->beta));
    const double tau = l.fwhm / std::sqrt(2.0 * std::log(2.0));
    const double spk = l.t_peak >= 0.0 ? l.t_peak : 3.0 * tau;
    const double th = t + 0.5 * c->dt;
    const double sr = D * th - spk;
    const double env = std::exp(-(sr / tau) * (sr / tau));
    const double amp = a0 * D * env * std::sin(kTwoPi * sr);
    return -amp / (kPi * c->hz);
}

// Every tile's bucket of each species ordered by cell (sort_cells_kernel),
// into the other side of its double buffer
template <typename real>
static void sort_cells_t(pic_ctx *c)
{
    for (int sp = 0; sp < 2; ++sp) {
        if (sp == 1 && !c->ions_species) break;
        SortArgs<real> a{};
        a.g = c->g;
        a.in = species_view<real>(c, sp, c->cur[sp]);
        a.out = species_view<real>(c, sp, c->cur[sp] ^ 1);
        a.in_lo = counts(c, sp, c->cur[sp], 0);
        a.in_hi = counts(c, sp, c->cur[sp], 1);
        a.out_lo = counts(c, sp, c->cur[sp] ^ 1, 0);
        a.err = reinterpret_cast<unsigned *>(c->scratch + c->off_err);
        launch_sort_cells<real>(a, c->stream);
        c->cur[sp] ^= 1;
        c->kernels += 1;
    }
}

template <typename real>
static void run_phases_t(pic_ctx *c, unsigned mask)
{
    if ((mask & PIC_PH_PUSH) && c->sort_every > 0 && !c->capturing && c->step % c->sort_every == 0) {
        PhaseTimer pt(c, 7);
        sort_cells_t<real>(c);
    }
    real *F[9];
    for (int q = 0; q < 9; ++q) F[q] = (real *)field_ptr(c, q);
    // When one call zeroes, deposits and filters the current, the raw current
    // is accumulated in the scratch buffer and the filter writes its result
    // straight into J (no copy back); otherwise every phase works on J.
    real *tmp = (real *)(c->scratch + c->off_tmp);
    const bool raw_in_tmp = (mask & PIC_PH_ZERO_J) && (mask & PIC_PH_FILTER) && c->p.filter_passes >= 1 &&
                            c->p.filter_passes <= 4;
    real *R[3] = {F[6], F[7], F[8]};
    if (raw_in_tmp)
        for (int q = 0; q < 3; ++q) R[q] = tmp + (size_t)q * c->g.ncomp;
    if (mask & PIC_PH_ZERO_J) {
        PhaseTimer pt(c, 0);
        launch_zero<real>(R[0], (int64_t)3 * c->g.ncomp, c->stream);
    }
    // With ions paired to their electrons, the electron kernel also takes the
    // tile's drifting ion records, so electron and ion currents add in one
    // integer tile: a pair whose electron has not moved away from its ion
    // flushes exactly zero, and no rounding residue of the global adds seeds
    // fields ahead of the laser (such residues release pairs at the stencil's
    // speed of 3 cells per step).  Explicit ions keep their own kernel, which
    // measured faster when every tile holds a full bucket of both species,
    // except with records in relative form: there the two species' currents
    // differ by ~1/(2 gamma^2) and must cancel in the integer tile, not in
    // FP32 global adds.
    const bool fused = (mask & PIC_PH_PUSH) && (mask & PIC_PH_IONS) && c->ions_species &&
                       (!c->p.explicit_ions || c->rel);
    if (mask & PIC_PH_PUSH) {
        PhaseTimer pt(c, 1);
        PushArgs<real> a = push_args<real>(c, 0);
        for (int q = 0; q < 3; ++q) a.J[q] = R[q];
        if (fused) {
            a.fuse_ions = 1;
            a.ions = ion_side<real>(c);
            // electrons and ions add into one integer tile: bound its sums
            // by both species' bucket capacities
            fixed_point_scales(c, 2, a.fx_scale, a.fx_quant, a.fx_lo);
        }
        launch_push<real>(a, c->stream);
        c->cur[0] ^= 1;
        if (fused) c->cur[1] ^= 1;
        c->kernels += 1;
    }
    if ((mask & PIC_PH_IONS) && c->ions_species && !fused) {
        PhaseTimer pt(c, 2);
        PushArgs<real> a = push_args<real>(c, 1);
        for (int q = 0; q < 3; ++q) a.J[q] = R[q];
        a.ions = ion_side<real>(c);
        launch_ions<real>(a, c->stream);
        c->cur[1] ^= 1;
        c->kernels += 1;
    }
    // the antenna stays where it was launched; a moving window leaves it behind
    const int64_t ka_rel = (int64_t)c->ka - c->win_n * c->win_S;
    if ((mask & PIC_PH_ANTENNA) && c->laser_on && ka_rel >= 2) {
        PhaseTimer pt(c, 3);
        const pic_laser_params &l = c->laser;
        const double j0 = c->capturing ? 0.0 : antenna_j0(c, c->t, l.a0);
        const int comp = l.polarization == PIC_POL_X ? 0 : 1;
        launch_antenna<real>(c->g, R[comp], l.polarization, (int)ka_rel, j0, c->hx, c->hy, l.x_center, l.y_center,
                             l.waist, c->stream, c->capturing ? &c->cap_scal[c->cap_s].j0 : nullptr);
        c->kernels += 1;
    }
    if ((mask & PIC_PH_FILTER) && c->p.filter_passes > 0) {
        PhaseTimer pt(c, 4);
        real *J[3] = {F[6], F[7], F[8]};
        unsigned *err = reinterpret_cast<unsigned *>(c->scratch + c->off_err);
        if (!raw_in_tmp) {
            launch_filter<real>(c->g, J, tmp, c->p.filter_passes, c->stream, err);
        } else if (!launch_filter_from<real>(c->g, tmp, J, c->p.filter_passes, c->stream, err) &&
                   !record_unsupported()) {
            cudaMemcpyAsync(J[0], tmp, (size_t)3 * c->g.ncomp * sizeof(real), cudaMemcpyDeviceToDevice, c->stream);
            launch_filter<real>(c->g, J, tmp, c->p.filter_passes, c->stream, err);
        }
        c->kernels += c->p.filter_passes <= 4 ? 1 : (int64_t)(c->g.dim == 3 ? 3 : 2) * c->p.filter_passes;
    }
    if (mask & PIC_PH_YEE) {
        PhaseTimer pt(c, 5);
        real *F1[6];
        for (int q = 0; q < 6; ++q) F1[q] = (real *)eb_other(c, q);
        launch_yee<real>(c->g, F, F1, c->dt, c->hx, c->hy, c->hz, c->stream);
        c->fset ^= 1;
        c->kernels += 1;
        if (c->btd_on) c->kernels += fill_btd<real>(c, F, F1);
    }
    if ((mask & PIC_PH_INJECT) && c->plasma_loaded && c->gam > 1.0) {
        PhaseTimer pt(c, 6);
        InjectArgs a{};
        fill_inject_common(c, a);
        a.mode = 1;
        a.t = c->t;
        a.t1 = c->t + c->dt;
        if (c->capturing) {
            // the band comes from the step's scalars; the launch covers the bound
            a.scal = &c->cap_scal[c->cap_s];
            a.m_lo = 0;
            a.m_hi = c->inj_planes_max;
        } else {
            lattice_band(a, c->gam * (c->zwin() + c->Lz + c->beta * a.t),
                         c->gam * (c->zwin() + c->Lz + c->beta * a.t1), a.m_lo, a.m_hi);
        }
        launch_inject(a, c->stream);
        if (a.m_hi > a.m_lo) c->kernels += 1;
    }
    if ((mask & PIC_PH_TIME) && !c->capturing) {
        c->t += c->dt;
        c->step += 1;
        if (c->win_on && c->t >= c->win_t0 &&
            c->win_v * (c->t - c->win_t0) >= (double)(c->win_n + 1) * c->win_S * c->hz)
            window_move<real>(c);
    }
}

static pic_status run_steps(pic_ctx *c, int nsteps, unsigned mask, bool check)
{
    if (!c) return PIC_ERR_ARG;
    if (!c->bound) return fail(c, PIC_ERR_STATE, "bind buffers first");
    if (nsteps < 0) return fail(c, PIC_ERR_ARG, "negative step count");
    for (int n = 0; n < nsteps; ++n) {
        if (c->es == 4) run_phases_t<float>(c, mask);
        else run_phases_t<double>(c, mask);
    }
    CUDA_TRY(c, cudaGetLastError());
    if (!check) return PIC_OK;
    return check_device_error(c);
}

// ------------------------------------------------------------------ batch

// The captured graph of a batch, kept between calls while the contexts are
// where the capture left them: same configuration (epoch), same halves of
// their double buffers, same window position.
struct BatchGraph {
    int K = 0;
    std::vector<std::array<int64_t, 5>> sig;  // per context: epoch, fset, cur[0], cur[1], win_n
    std::vector<int64_t> kern;                 // per context: kernels one replay launches
    cudaStream_t cs = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    StepScal *dev = nullptr;   // nctx x K scalars the graph's kernels read
    StepScal *host = nullptr;  // pinned: reps x nctx x K, one region per replay
    size_t host_n = 0;
    cudaEvent_t join = nullptr;
    std::vector<cudaEvent_t> ev;  // one per context
    int fused = 0;                // the graph is the batched form with this many launch chains (0: per context)
    void *fargs = nullptr;        // its argument structs, work-item prefix sums and queue counters
    int64_t launches = 0;         // its launches per replay (batched kernels and counter resets)
    std::vector<cudaStream_t> chain_cs;  // the chains' streams (capture only)
    std::vector<cudaEvent_t> chain_ev;
    void drop_graph()
    {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (dev) cudaFree(dev);
        if (fargs) cudaFree(fargs);
        exec = nullptr;
        graph = nullptr;
        dev = nullptr;
        fargs = nullptr;
        fused = 0;
        launches = 0;
        K = 0;
        sig.clear();
    }
    ~BatchGraph()
    {
        if (cs) cudaStreamSynchronize(cs);
        drop_graph();
        if (host) cudaFreeHost(host);
        if (join) cudaEventDestroy(join);
        for (cudaEvent_t e : ev)
            if (e) cudaEventDestroy(e);
        for (cudaEvent_t e : chain_ev)
            if (e) cudaEventDestroy(e);
        for (cudaStream_t x : chain_cs)
            if (x) cudaStreamDestroy(x);
        if (cs) cudaStreamDestroy(cs);
    }
};

struct pic_batch {
    std::vector<pic_ctx *> ctx;
    int graph_steps = 20;  // steps per captured graph (even; 0: streams only)
    int fused = 4;         // launch chains of the batched form of a captured step (0: per-context graph)
    BatchGraph gr;
};

// Whether the contexts' steps can be captured: nothing in them depends on the
// host at run time except the per-step scalars of StepScal (no moving
// window, no lab snapshots, no phase timing), and every context has a stream
// of its own (the legacy default stream cannot be captured).
static bool batch_capturable(const pic_batch *b)
{
    for (const pic_ctx *c : b->ctx)
        if (c->win_on || c->btd_on || c->profiling || c->sort_every > 0 || c->stream == nullptr) return false;
    return true;
}

// Per-step scalars of steps [c->t, c->t + K dt) (times accumulated as the
// step does) into host memory
static void fill_step_scalars(pic_ctx *c, int K, StepScal *h)
{
    InjectArgs a{};
    fill_inject_common(c, a);
    double t = c->t;
    for (int s = 0; s < K; ++s) {
        const double t1 = t + c->dt;
        h[s].j0 = c->laser_on ? antenna_j0(c, t, c->laser.a0) : 0.0;
        h[s].t = t;
        h[s].t1 = t1;
        h[s].m_lo = h[s].m_hi = 0;
        if (c->plasma_loaded && c->gam > 1.0)
            lattice_band(a, c->gam * (c->zwin() + c->Lz + c->beta * t), c->gam * (c->zwin() + c->Lz + c->beta * t1),
                         h[s].m_lo, h[s].m_hi);
        t = t1;
    }
}

static std::array<int64_t, 5> ctx_signature(const pic_ctx *c)
{
    return {c->epoch, c->fset, c->cur[0], c->cur[1], c->win_n};
}

// The batched form of K steps of every context.  Each context's steps run on
// the host with a launch recorder installed (nothing is launched; the
// double buffers flip K times, K even, so every context ends where it
// started).  The records are grouped by step, phase and kernel instance, in
// the order the step issues its phases, and each group becomes one launch
// over the work items of all its runs, captured on the batch's stream; the
// persistent particle kernels take their items from a counter zeroed just
// before them.  ok = false (nothing captured) where some step asked for a
// launch without a batched form.
static pic_status batch_capture_fused(pic_batch *b, int K, bool &ok)
{
    ok = false;
    BatchGraph &G = b->gr;
    const size_t nctx = b->ctx.size();
    pic_ctx *c0 = b->ctx[0];
    auto bad = [&](cudaError_t e) {
        if (e == cudaSuccess) return false;
        c0->err = std::string("batch graph: ") + cudaGetErrorString(e);
        return true;
    };
    // the runs spread over the chains by size (tiles), largest first onto the
    // least loaded chain
    const int S = (int)std::min<size_t>((size_t)b->fused, nctx);
    std::vector<int> chain_of(nctx, 0);
    {
        std::vector<size_t> by(nctx);
        for (size_t i = 0; i < nctx; ++i) by[i] = i;
        std::stable_sort(by.begin(), by.end(),
                         [&](size_t x, size_t y) { return b->ctx[x]->g.ntiles > b->ctx[y]->g.ntiles; });
        std::vector<int64_t> load(S, 0);
        for (size_t i : by) {
            const int m = (int)(std::min_element(load.begin(), load.end()) - load.begin());
            chain_of[i] = m;
            load[m] += b->ctx[i]->g.ntiles;
        }
    }
    BatchRecorder rec;
    rec.nctx = (int)((nctx + S - 1) / S);
    std::vector<int64_t> k0(nctx);
    for (size_t i = 0; i < nctx; ++i) k0[i] = b->ctx[i]->kernels;
    g_rec = &rec;
    for (int s = 0; s < K; ++s)
        for (size_t i = 0; i < nctx; ++i) {
            pic_ctx *c = b->ctx[i];
            rec.chain = chain_of[i];
            rec.step = s;
            c->capturing = true;
            c->cap_scal = G.dev + i * K;
            c->cap_s = s;
            if (c->es == 4) run_phases_t<float>(c, PIC_PH_ALL);
            else run_phases_t<double>(c, PIC_PH_ALL);
            c->capturing = false;
        }
    g_rec = nullptr;
    G.sig.assign(nctx, {});
    G.kern.assign(nctx, 0);
    for (size_t i = 0; i < nctx; ++i) {
        pic_ctx *c = b->ctx[i];
        G.kern[i] = c->kernels - k0[i];
        c->kernels = k0[i];
        G.sig[i] = ctx_signature(c);
    }
    if (rec.unsupported || rec.recs.empty()) return PIC_OK;
    // groups: records of one step and phase with the same kernel instance
    std::vector<size_t> order(rec.recs.size());
    for (size_t j = 0; j < order.size(); ++j) order[j] = j;
    std::stable_sort(order.begin(), order.end(), [&](size_t x, size_t y) {
        const LaunchRecord &X = rec.recs[x], &Y = rec.recs[y];
        if (X.chain != Y.chain) return X.chain < Y.chain;
        return X.step != Y.step ? X.step < Y.step : X.phase < Y.phase;
    });
    struct Group {
        int chain;
        BatchLaunch fn;
        bool queue;
        std::vector<size_t> idx;
        size_t args_off = 0, start_off = 0, q_off = 0;
        int64_t total = 0;
    };
    std::vector<Group> groups;
    for (size_t a = 0; a < order.size();) {
        size_t e = a;
        const LaunchRecord &A = rec.recs[order[a]];
        while (e < order.size() && rec.recs[order[e]].chain == A.chain && rec.recs[order[e]].step == A.step &&
               rec.recs[order[e]].phase == A.phase)
            ++e;
        const size_t first = groups.size();
        for (size_t j = a; j < e; ++j) {
            const LaunchRecord &L = rec.recs[order[j]];
            size_t gi = first;
            while (gi < groups.size() && groups[gi].fn != L.fn) ++gi;
            if (gi == groups.size()) groups.push_back(Group{A.chain, L.fn, L.queue, {}});
            groups[gi].idx.push_back(order[j]);
        }
        a = e;
    }
    auto al = [](size_t x) { return (x + 255) / 256 * 256; };
    size_t off = 0;
    for (Group &g : groups) {
        const size_t bytes = rec.recs[g.idx[0]].args.size();
        g.args_off = off;
        off += al(bytes * g.idx.size());
        g.start_off = off;
        off += al(sizeof(int64_t) * (g.idx.size() + 1));
        if (g.queue) {
            g.q_off = off;
            off += 256;
        }
    }
    std::vector<unsigned char> hb(off, 0);
    for (Group &g : groups) {
        const size_t bytes = rec.recs[g.idx[0]].args.size();
        int64_t *st = reinterpret_cast<int64_t *>(hb.data() + g.start_off);
        st[0] = 0;
        for (size_t j = 0; j < g.idx.size(); ++j) {
            const LaunchRecord &L = rec.recs[g.idx[j]];
            std::memcpy(hb.data() + g.args_off + j * bytes, L.args.data(), bytes);
            st[j + 1] = st[j] + L.items;
        }
        g.total = st[g.idx.size()];
    }
    if (bad(cudaMalloc(&G.fargs, off)) || bad(cudaMemcpy(G.fargs, hb.data(), off, cudaMemcpyHostToDevice)))
        return PIC_ERR_CUDA;
    unsigned char *d = static_cast<unsigned char *>(G.fargs);
    while ((int)G.chain_cs.size() < S) {
        cudaStream_t x = nullptr;
        cudaEvent_t ev = nullptr;
        if (bad(cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking)) ||
            bad(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)))
            return PIC_ERR_CUDA;
        G.chain_cs.push_back(x);
        G.chain_ev.push_back(ev);
    }
    // every chain forks from the batch's stream and joins it at the end
    if (bad(cudaStreamBeginCapture(G.cs, cudaStreamCaptureModeRelaxed))) return PIC_ERR_CUDA;
    cudaEventRecord(G.join, G.cs);
    for (int m = 0; m < S; ++m) cudaStreamWaitEvent(G.chain_cs[m], G.join, 0);
    int64_t launches = 0;
    for (const Group &g : groups) {
        if (g.total <= 0) continue;
        cudaStream_t x = G.chain_cs[g.chain];
        unsigned *q = g.queue ? reinterpret_cast<unsigned *>(d + g.q_off) : nullptr;
        if (q) {
            cudaMemsetAsync(q, 0, sizeof(unsigned), x);
            ++launches;
        }
        g.fn(d + g.args_off, reinterpret_cast<const int64_t *>(d + g.start_off), (int)g.idx.size(), g.total, q, x);
        ++launches;
    }
    for (int m = 0; m < S; ++m) {
        cudaEventRecord(G.chain_ev[m], G.chain_cs[m]);
        cudaStreamWaitEvent(G.cs, G.chain_ev[m], 0);
    }
    const cudaError_t e = cudaStreamEndCapture(G.cs, &G.graph);
    if (bad(e) || bad(cudaGetLastError()) || bad(cudaGraphInstantiate(&G.exec, G.graph, 0))) {
        G.drop_graph();
        return PIC_ERR_CUDA;
    }
    G.fused = S;
    G.launches = launches;
    G.K = K;
    ok = true;
    return PIC_OK;
}

// Capture K steps of every context as one graph on the batch's stream: the
// batched form where it applies, else fork every context's stream from it,
// K steps each, join.  Step s of context i reads its scalars from dev[i K + s].
static pic_status batch_capture(pic_batch *b, int K)
{
    BatchGraph &G = b->gr;
    const size_t nctx = b->ctx.size();
    pic_ctx *c0 = b->ctx[0];
    auto bad = [&](cudaError_t e) {
        if (e == cudaSuccess) return false;
        c0->err = std::string("batch graph: ") + cudaGetErrorString(e);
        return true;
    };
    G.drop_graph();
    if (bad(cudaMalloc(&G.dev, sizeof(StepScal) * nctx * K))) return PIC_ERR_CUDA;
    for (size_t i = 0; i < nctx; ++i) {
        pic_ctx *c = b->ctx[i];
        // a band never spans more lattice planes than this (see lattice_band)
        InjectArgs a{};
        fill_inject_common(c, a);
        const double jm = a.jitter * a.hz_lab + a.dzl;
        c->inj_planes_max = (int64_t)std::ceil((c->gam * c->beta * c->dt + 2.0 * jm) / a.dzl) + 8;
    }
    if (b->fused) {
        bool ok = false;
        const pic_status st = batch_capture_fused(b, K, ok);
        if (st != PIC_OK || ok) return st;
    }
    if (bad(cudaStreamBeginCapture(G.cs, cudaStreamCaptureModeRelaxed))) return PIC_ERR_CUDA;
    cudaEventRecord(G.join, G.cs);
    for (size_t i = 0; i < nctx; ++i) cudaStreamWaitEvent(b->ctx[i]->stream, G.join, 0);
    std::vector<int64_t> k0(nctx);
    for (size_t i = 0; i < nctx; ++i) k0[i] = b->ctx[i]->kernels;
    for (int s = 0; s < K; ++s)
        for (size_t i = 0; i < nctx; ++i) {
            pic_ctx *c = b->ctx[i];
            c->capturing = true;
            c->cap_scal = G.dev + i * K;
            c->cap_s = s;
            if (c->es == 4) run_phases_t<float>(c, PIC_PH_ALL);
            else run_phases_t<double>(c, PIC_PH_ALL);
            c->capturing = false;
        }
    for (size_t i = 0; i < nctx; ++i) {
        cudaEventRecord(G.ev[i], b->ctx[i]->stream);
        cudaStreamWaitEvent(G.cs, G.ev[i], 0);
    }
    const cudaError_t e = cudaStreamEndCapture(G.cs, &G.graph);
    // the capture flipped every double buffer K times (K even: back where it
    // was) and counted the kernels of K steps, which every replay adds
    G.sig.assign(nctx, {});
    G.kern.assign(nctx, 0);
    for (size_t i = 0; i < nctx; ++i) {
        pic_ctx *c = b->ctx[i];
        G.kern[i] = c->kernels - k0[i];
        c->kernels = k0[i];
        G.sig[i] = ctx_signature(c);
    }
    if (bad(e) || bad(cudaGraphInstantiate(&G.exec, G.graph, 0))) {
        G.drop_graph();
        return PIC_ERR_CUDA;
    }
    G.K = K;
    G.launches = 0;
    for (int64_t k : G.kern) G.launches += k;
    return PIC_OK;
}

// K steps of every context as one CUDA graph, replayed nsteps / K times.  The
// graph is captured once and kept while the contexts stay where it left them.
// Each replay is preceded, on the batch's stream, by the copy of its own
// region of per-step scalars from pinned host memory (all regions are filled
// before the first replay), so no replay waits for the host.  Returns the
// number of steps done (a multiple of K).
static pic_status batch_graph_steps(pic_batch *b, int nsteps, int &done)
{
    done = 0;
    BatchGraph &G = b->gr;
    const int K = b->graph_steps;
    const int reps = nsteps / K;
    if (reps < 1) return PIC_OK;
    const size_t nctx = b->ctx.size();
    pic_ctx *c0 = b->ctx[0];
    auto bad = [&](cudaError_t e) {
        if (e == cudaSuccess) return false;
        c0->err = std::string("batch graph: ") + cudaGetErrorString(e);
        return true;
    };
    if (!G.cs) {
        if (bad(cudaStreamCreateWithFlags(&G.cs, cudaStreamNonBlocking))) return PIC_ERR_CUDA;
        if (bad(cudaEventCreateWithFlags(&G.join, cudaEventDisableTiming))) return PIC_ERR_CUDA;
    }
    while (G.ev.size() < nctx) {
        cudaEvent_t e = nullptr;
        if (bad(cudaEventCreateWithFlags(&e, cudaEventDisableTiming))) return PIC_ERR_CUDA;
        G.ev.push_back(e);
    }
    // the previous call's copies out of the host regions are done
    if (bad(cudaStreamSynchronize(G.cs))) return PIC_ERR_CUDA;
    bool same = G.exec && G.K == K && G.sig.size() == nctx;
    for (size_t i = 0; same && i < nctx; ++i) same = G.sig[i] == ctx_signature(b->ctx[i]);
    if (!same) {
        const pic_status st = batch_capture(b, K);
        if (st != PIC_OK) return st;
    }
    const size_t per = nctx * (size_t)K;
    if (G.host_n < per * reps) {
        if (G.host) cudaFreeHost(G.host);
        G.host = nullptr;
        G.host_n = 0;
        if (bad(cudaMallocHost(&G.host, sizeof(StepScal) * per * reps))) return PIC_ERR_CUDA;
        G.host_n = per * reps;
    }
    for (int r = 0; r < reps; ++r)
        for (size_t i = 0; i < nctx; ++i) {
            pic_ctx *c = b->ctx[i];
            fill_step_scalars(c, K, G.host + r * per + i * K);
            for (int s = 0; s < K; ++s) c->t += c->dt;
            c->step += K;
            c->kernels += G.kern[i];
        }
    // order after the work already queued on the contexts' streams
    for (size_t i = 0; i < nctx; ++i) {
        cudaEventRecord(G.ev[i], b->ctx[i]->stream);
        cudaStreamWaitEvent(G.cs, G.ev[i], 0);
    }
    for (int r = 0; r < reps; ++r) {
        if (bad(cudaMemcpyAsync(G.dev, G.host + r * per, sizeof(StepScal) * per, cudaMemcpyHostToDevice, G.cs)) ||
            bad(cudaGraphLaunch(G.exec, G.cs)))
            return PIC_ERR_CUDA;
        done += K;
    }
    // and the contexts' later work after the replays
    cudaEventRecord(G.join, G.cs);
    for (size_t i = 0; i < nctx; ++i) cudaStreamWaitEvent(b->ctx[i]->stream, G.join, 0);
    return PIC_OK;
}

extern "C" pic_status pic_batch_set_graph(pic_batch *b, int steps_per_graph)
{
    if (!b || steps_per_graph < 0 || (steps_per_graph & 1)) return PIC_ERR_ARG;
    b->graph_steps = steps_per_graph;
    return PIC_OK;
}

extern "C" pic_status pic_batch_set_fused(pic_batch *b, int fused)
{
    if (!b || fused < 0) return PIC_ERR_ARG;
    if (b->fused != fused) {
        if (b->gr.cs) cudaStreamSynchronize(b->gr.cs);
        b->gr.drop_graph();
    }
    b->fused = fused;
    return PIC_OK;
}

extern "C" pic_status pic_batch_graph_info(pic_batch *b, int *fused, int64_t *launches_per_replay, int *steps)
{
    if (!b) return PIC_ERR_ARG;
    if (fused) *fused = b->gr.exec ? b->gr.fused : 0;
    if (launches_per_replay) *launches_per_replay = b->gr.exec ? b->gr.launches : 0;
    if (steps) *steps = b->gr.exec ? b->gr.K : 0;
    return PIC_OK;
}

extern "C" pic_status pic_batch_create(pic_ctx *const *ctxs, int n, pic_batch **out)
{
    if (!out) return PIC_ERR_ARG;
    *out = nullptr;
    if (!ctxs || n < 1) return PIC_ERR_ARG;
    for (int i = 0; i < n; ++i) {
        if (!ctxs[i] || !ctxs[i]->bound) return PIC_ERR_STATE;
        for (int k = 0; k < i; ++k)
            if (ctxs[k] == ctxs[i]) return PIC_ERR_ARG;
    }
    pic_batch *b = new (std::nothrow) pic_batch;
    if (!b) return PIC_ERR_ARG;
    b->ctx.assign(ctxs, ctxs + n);
    *out = b;
    return PIC_OK;
}

extern "C" pic_status pic_batch_step(pic_batch *b, int nsteps)
{
    if (!b || nsteps < 0) return PIC_ERR_ARG;
    int done = 0;
    if (b->graph_steps > 0 && nsteps >= b->graph_steps && batch_capturable(b)) {
        pic_status s = batch_graph_steps(b, nsteps, done);
        if (s != PIC_OK) return s;
    }
    // step n of every context before step n + 1 of any: the contexts' streams
    // run concurrently, so the GPU holds the kernels of all of them at once
    for (int n = done; n < nsteps; ++n)
        for (pic_ctx *c : b->ctx) {
            pic_status s = run_steps(c, 1, PIC_PH_ALL, false);
            if (s != PIC_OK) return s;
        }
    pic_status first = PIC_OK;
    for (pic_ctx *c : b->ctx) {
        pic_status s = check_device_error(c);
        if (s != PIC_OK && first == PIC_OK) first = s;
    }
    return first;
}

extern "C" void pic_batch_destroy(pic_batch *b) { delete b; }

extern "C" pic_status pic_sort_cells(pic_ctx *c)
{
    if (!c) return PIC_ERR_ARG;
    if (!c->bound) return fail(c, PIC_ERR_STATE, "bind buffers first");
    if (c->es == 4) sort_cells_t<float>(c);
    else sort_cells_t<double>(c);
    CUDA_TRY(c, cudaGetLastError());
    return check_device_error(c);
}

extern "C" pic_status pic_set_cell_sort(pic_ctx *c, int every)
{
    if (!c || every < 0) return PIC_ERR_ARG;
    c->sort_every = every;
    c->epoch += 1;
    return PIC_OK;
}

extern "C" pic_status pic_step(pic_ctx *c, int nsteps) { return run_steps(c, nsteps, PIC_PH_ALL, true); }
extern "C" pic_status pic_step_async(pic_ctx *c, int nsteps) { return run_steps(c, nsteps, PIC_PH_ALL, false); }
extern "C" pic_status pic_step_phases(pic_ctx *c, unsigned mask)
{
    if (mask & ~PIC_PH_ALL) return fail(c, PIC_ERR_ARG, "unknown phase bits");
    return run_steps(c, 1, mask, true);
}

// ---------------------------------------------------------- moving window

extern "C" pic_status pic_set_moving_window(pic_ctx *c, double v, double t0, int shift_cells)
{
    if (!c) return PIC_ERR_ARG;
    c->epoch += 1;
    if (v == 0.0) {
        c->win_on = false;
        return PIC_OK;
    }
    const int tz = 1 << c->g.lt[2];
    if (!(v > 0.0 && v <= 1.0) || !std::isfinite(t0) || shift_cells < tz || shift_cells % tz != 0 ||
        shift_cells >= c->g.nz || c->g.bc_z != PIC_BC_MUR)
        return fail(c, PIC_ERR_ARG, "moving window: 0 < v <= 1, absorbing z, and moves of a whole number of tile "
                                    "layers smaller than the grid");
    c->win_on = true;
    c->win_v = v;
    c->win_t0 = t0;
    c->win_S = shift_cells;
    return PIC_OK;
}

// ---------------------------------------------------------- lab snapshots

static bool btd_valid(const pic_ctx *c, const pic_btd_params *p)
{
    return c->gam > 1.0 && p->n_snapshots >= 1 && p->n_snapshots <= 64 && p->nz >= 1 && p->dz > 0.0 &&
           std::isfinite(p->t0) && std::isfinite(p->dt) && std::isfinite(p->z0) && std::isfinite(p->dz) &&
           (p->plane == 0 || p->plane == 1) &&
           (double)p->n_snapshots * 6.0 * p->nz * (p->plane ? c->g.nx : 1) < 4e12;
}

static size_t btd_data_bytes(const pic_ctx *c, const pic_btd_params *p)
{
    return align_up((size_t)p->n_snapshots * 6 * p->nz * btd_nxs(c, p) * c->es);
}

extern "C" pic_status pic_btd_bytes(const pic_ctx *c, const pic_btd_params *p, size_t *bytes)
{
    if (!c || !p || !bytes) return PIC_ERR_ARG;
    if (!btd_valid(c, p)) return PIC_ERR_ARG;
    *bytes = btd_data_bytes(c, p) + align_up(sizeof(int) * (size_t)p->n_snapshots * p->nz);
    return PIC_OK;
}

extern "C" pic_status pic_btd_setup(pic_ctx *c, const pic_btd_params *p, void *buf, size_t bytes)
{
    if (!c) return PIC_ERR_ARG;
    c->epoch += 1;
    if (!p) {
        c->btd_on = false;
        c->btd_buf = nullptr;
        return PIC_OK;
    }
    if (!c->bound) return fail(c, PIC_ERR_STATE, "bind buffers first");
    if (!btd_valid(c, p)) return fail(c, PIC_ERR_ARG, "invalid snapshot parameters (a boosted grid is needed)");
    size_t need = 0;
    pic_btd_bytes(c, p, &need);
    if (!buf || bytes < need || ((uintptr_t)buf % kAlign) != 0)
        return fail(c, PIC_ERR_ARG, "snapshot buffer too small or not 256-byte aligned");
    c->btd = *p;
    c->btd_buf = (unsigned char *)buf;
    c->btd_flags_off = btd_data_bytes(c, p);
    CUDA_TRY(c, cudaMemsetAsync(buf, 0, need, c->stream));
    c->btd_on = true;
    return PIC_OK;
}

extern "C" pic_status pic_btd_get(pic_ctx *c, int j, void *dst, size_t dst_bytes, int dst_is_device)
{
    if (!c || !dst) return PIC_ERR_ARG;
    if (!c->btd_on) return fail(c, PIC_ERR_STATE, "no snapshots are being taken");
    const pic_btd_params &p = c->btd;
    if (j < 0 || j >= p.n_snapshots) return fail(c, PIC_ERR_ARG, "snapshot index out of range");
    const size_t nd = (size_t)6 * p.nz * btd_nxs(c, &p) * c->es, nf = sizeof(int) * (size_t)p.nz;
    if (dst_bytes < nd + nf) return fail(c, PIC_ERR_ARG, "destination too small");
    CUDA_TRY(c, cudaMemcpyAsync(dst, c->btd_buf + (size_t)j * nd, nd, kind_out(dst_is_device), c->stream));
    CUDA_TRY(c, cudaMemcpyAsync((unsigned char *)dst + nd, c->btd_buf + c->btd_flags_off + (size_t)j * nf, nf,
                                kind_out(dst_is_device), c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return PIC_OK;
}

// -------------------------------------------------------------------- output


static int popcount9(unsigned m)
{
    int n = 0;
    for (int q = 0; q < PIC_NCOMP; ++q) n += (m >> q) & 1u;
    return n;
}

// lab-frame E, B components of mask (bits 0..5) into dst, one component at a
// time through the scratch current buffer when dst is host memory
template <typename real>
static pic_status get_fields_lab_t(pic_ctx *c, unsigned mask, unsigned char *dst, int dst_is_device)
{
    const size_t per = (size_t)c->g.ncomp * c->es;
    real *tmp = reinterpret_cast<real *>(c->scratch + c->off_tmp);
    static const int partner[6] = {4, 3, -1, 1, 0, -1};  // By, Bx, -, Ey, Ex, -
    size_t o = 0;
    for (int q = 0; q < 6; ++q) {
        if (!(mask >> q & 1u)) continue;
        real *out = dst_is_device ? reinterpret_cast<real *>(dst + o) : tmp;
        const real *F = (const real *)field_ptr(c, q);
        const real *P = partner[q] >= 0 ? (const real *)field_ptr(c, partner[q]) : F;
        launch_lab_fields<real>(c->g, F, P, q, out, c->gam, c->beta, c->sms, c->stream);
        CUDA_TRY(c, cudaGetLastError());
        if (!dst_is_device) CUDA_TRY(c, cudaMemcpyAsync(dst + o, tmp, per, cudaMemcpyDeviceToHost, c->stream));
        o += per;
    }
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return PIC_OK;
}

extern "C" pic_status pic_get_fields(pic_ctx *c, unsigned mask, int frame, void *dst, size_t dst_bytes,
                                     int dst_is_device)
{
    if (!c || !dst || (mask & ~0x1FFu) || mask == 0) return PIC_ERR_ARG;
    if (frame != PIC_FRAME_BOOST && frame != PIC_FRAME_LAB) return fail(c, PIC_ERR_ARG, "unknown frame");
    if (frame == PIC_FRAME_LAB && (mask & 0x1C0u))
        return fail(c, PIC_ERR_ARG, "the lab-frame view holds E and B only");
    if (!c->bound) return fail(c, PIC_ERR_STATE, "bind buffers first");
    const size_t per = (size_t)c->g.ncomp * c->es;
    if (dst_bytes < per * popcount9(mask)) return fail(c, PIC_ERR_ARG, "destination too small");
    if (frame == PIC_FRAME_LAB && c->gam > 1.0) {
        if (dst_is_device && ((uintptr_t)dst % (uintptr_t)c->es) != 0)
            return fail(c, PIC_ERR_ARG, "device destination not aligned to the element size");
        return c->es == 4 ? get_fields_lab_t<float>(c, mask, (unsigned char *)dst, dst_is_device)
                          : get_fields_lab_t<double>(c, mask, (unsigned char *)dst, dst_is_device);
    }
    size_t o = 0;
    for (int q = 0; q < PIC_NCOMP; ++q) {
        if (!(mask >> q & 1u)) continue;
        CUDA_TRY(c, cudaMemcpyAsync((unsigned char *)dst + o, field_ptr(c, q), per, kind_out(dst_is_device), c->stream));
        o += per;
    }
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return PIC_OK;
}

extern "C" pic_status pic_set_fields(pic_ctx *c, unsigned mask, const void *src, size_t src_bytes, int src_is_device)
{
    if (!c || !src || (mask & ~0x1FFu) || mask == 0) return PIC_ERR_ARG;
    if (!c->bound) return fail(c, PIC_ERR_STATE, "bind buffers first");
    const size_t per = (size_t)c->g.ncomp * c->es;
    if (src_bytes < per * popcount9(mask)) return fail(c, PIC_ERR_ARG, "source too small");
    size_t o = 0;
    for (int q = 0; q < PIC_NCOMP; ++q) {
        if (!(mask >> q & 1u)) continue;
        CUDA_TRY(c, cudaMemcpyAsync(field_ptr(c, q), (const unsigned char *)src + o, per, kind_in(src_is_device), c->stream));
        o += per;
    }
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return PIC_OK;
}

extern "C" pic_status pic_get_axis(pic_ctx *c, int comp, void *dst, size_t dst_bytes, int dst_is_device)
{
    if (!c || !dst || comp < 0 || comp >= PIC_NCOMP) return PIC_ERR_ARG;
    if (!c->bound) return fail(c, PIC_ERR_STATE, "bind buffers first");
    const size_t n = (size_t)c->g.nz + 1;
    if (dst_bytes < n * c->es) return fail(c, PIC_ERR_ARG, "destination too small");
    const size_t off = ((size_t)(c->g.ny / 2) * c->g.nx + c->g.nx / 2) * c->es;
    CUDA_TRY(c, cudaMemcpy2DAsync(dst, c->es, (unsigned char *)field_ptr(c, comp) + off, (size_t)c->g.plane * c->es,
                                  c->es, n, kind_out(dst_is_device), c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return PIC_OK;
}

// live count per tile (both runs, clamped to the capacity) and exclusive
// offsets; PIC_ERR_CAPACITY if the runs of a tile overlap (the bucket overflowed)
static pic_status tile_offsets(pic_ctx *c, int sp, std::vector<int64_t> &off, int64_t &total)
{
    const size_t nt = (size_t)c->g.ntiles;
    std::vector<int> lo(nt), hi(nt);
    CUDA_TRY(c, cudaMemcpyAsync(lo.data(), counts(c, sp, c->cur[sp], 0), sizeof(int) * nt, cudaMemcpyDeviceToHost,
                                c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(hi.data(), counts(c, sp, c->cur[sp], 1), sizeof(int) * nt, cudaMemcpyDeviceToHost,
                                c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    off.resize(nt);
    total = 0;
    bool overflow = false;
    for (size_t t = 0; t < nt; ++t) {
        off[t] = total;
        const int l = lo[t] < c->g.cap ? lo[t] : c->g.cap;
        int h = hi[t];
        if (h > c->g.cap - l) {
            overflow = true;
            h = c->g.cap - l;
        }
        total += l + h;
    }
    if (overflow) return fail(c, PIC_ERR_CAPACITY, "a tile bucket overflowed (raise slots_per_cell)");
    return PIC_OK;
}

// compact the live particles of a species into slots [0, n) of its inactive side
template <typename real>
static pic_status compact_t(pic_ctx *c, int sp, int64_t &n)
{
    std::vector<int64_t> off;
    pic_status s = tile_offsets(c, sp, off, n);
    if (s != PIC_OK) return s;
    int64_t *d_off = reinterpret_cast<int64_t *>(c->scratch + c->off_offsets);
    CUDA_TRY(c, cudaMemcpyAsync(d_off, off.data(), sizeof(int64_t) * off.size(), cudaMemcpyHostToDevice, c->stream));
    CompactArgs<real> a{};
    a.g = c->g;
    a.src = species_view<real>(c, sp, c->cur[sp]);
    a.dst = species_view<real>(c, sp, c->cur[sp] ^ 1);
    a.lo = counts(c, sp, c->cur[sp], 0);
    a.hi = counts(c, sp, c->cur[sp], 1);
    a.offset = d_off;
    launch_compact<real>(a, c->stream);
    CUDA_TRY(c, cudaGetLastError());
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return PIC_OK;
}

// compacted records of a species, downloaded: attribute columns as bytes
template <typename real>
static pic_status download_species(pic_ctx *c, int sp, int64_t &n, std::vector<std::vector<unsigned char>> &h)
{
    pic_status s = compact_t<real>(c, sp, n);
    if (s != PIC_OK) return s;
    void *col[kAttrs];
    side_raw(c, sp, c->cur[sp] ^ 1, col);
    h.assign(kAttrs, {});
    for (int a = 0; a < kAttrs; ++a) {
        if (!col[a]) continue;
        h[a].resize((size_t)n * attr_size(c, a));
        if (n) CUDA_TRY(c, cudaMemcpyAsync(h[a].data(), col[a], h[a].size(), cudaMemcpyDeviceToHost, c->stream));
    }
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return PIC_OK;
}

// Live particles as FP64 rows.  Species 1 (drifting ions) is the stored ion
// records plus, for every paired electron, its ion at the electron's position.
template <typename real>
static pic_status get_particles_t(pic_ctx *c, int sp, double *dst, size_t dst_bytes, int64_t *n_out, int64_t *ids)
{
    int64_t ne = 0, ni = 0;
    std::vector<std::vector<unsigned char>> he, hi;
    pic_status s = download_species<real>(c, 0, ne, he);
    if (s != PIC_OK) return s;
    if (sp == 1) {
        s = download_species<real>(c, 1, ni, hi);
        if (s != PIC_OK) return s;
    }
    const int32_t *ecell = reinterpret_cast<const int32_t *>(he[7].data());
    int64_t npaired = 0;
    if (sp == 1)
        for (int64_t p = 0; p < ne; ++p) npaired += ((uint32_t)ecell[p] & kPaired) ? 1 : 0;
    const int64_t n = sp == 0 ? ne : ni + npaired;
    if (n_out) *n_out = n;
    if (!dst) return PIC_OK;
    if (dst_bytes < (size_t)n * 7 * sizeof(double)) return fail(c, PIC_ERR_ARG, "destination too small");
    const double uz_ion = (double)drift_u<real>(c);
    int64_t row = 0;
    auto emit = [&](const std::vector<std::vector<unsigned char>> &h, int64_t p, bool electron) {
        auto R = [&](int a) { return reinterpret_cast<const real *>(h[a].data()); };
        int i, j, k;
        unpack_cell(c->g, reinterpret_cast<const int32_t *>(h[7].data())[p], i, j, k);
        if (electron && !h[9].empty()) {
            // relative form: reference cell + reference offset + departure
            // (the reference cell is the stored one shifted by rel_actual's r)
            auto coord = [&](int cell, int ao, int ad, double h_) {
                int r;
                (void)rel_actual<real>(R(ao)[p], R(ad)[p], r);
                return ((double)(cell + r) + ((double)R(ao)[p] + (double)R(ad)[p])) * h_;
            };
            dst[0 * n + row] = coord(i, 0, 9, c->hx);
            dst[1 * n + row] = c->g.dim == 3 ? coord(j, 1, 10, c->hy) : 0.0;
            dst[2 * n + row] = coord(k, 2, 11, c->hz);
        } else {
            dst[0 * n + row] = ((double)i + (double)R(0)[p]) * c->hx;
            dst[1 * n + row] = c->g.dim == 3 ? ((double)j + (double)R(1)[p]) * c->hy : 0.0;
            dst[2 * n + row] = ((double)k + (double)R(2)[p]) * c->hz;
        }
        if (electron) {
            dst[3 * n + row] = (double)R(4)[p];
            dst[4 * n + row] = (double)R(5)[p];
            dst[5 * n + row] = uz_ion + (double)R(6)[p];
        } else {
            dst[3 * n + row] = 0.0;
            dst[4 * n + row] = 0.0;
            dst[5 * n + row] = uz_ion;
        }
        dst[6 * n + row] = (double)R(3)[p];
        if (ids) ids[row] = c->p.track_ids ? reinterpret_cast<const int64_t *>(h[8].data())[p] : -1;
        ++row;
    };
    if (sp == 0) {
        for (int64_t p = 0; p < ne; ++p) emit(he, p, true);
    } else {
        for (int64_t p = 0; p < ni; ++p) emit(hi, p, false);
        for (int64_t p = 0; p < ne; ++p)
            if ((uint32_t)ecell[p] & kPaired) emit(he, p, false);
    }
    return PIC_OK;
}

extern "C" pic_status pic_get_particles(pic_ctx *c, int sp, double *dst, size_t dst_bytes, int64_t *n_out, int64_t *ids)
{
    if (!c || (sp != 0 && sp != 1)) return PIC_ERR_ARG;
    if (!c->bound) return fail(c, PIC_ERR_STATE, "bind buffers first");
    if (sp == 1 && !c->ions_species) {
        if (n_out) *n_out = 0;
        return PIC_OK;
    }
    return c->es == 4 ? get_particles_t<float>(c, sp, dst, dst_bytes, n_out, ids)
                      : get_particles_t<double>(c, sp, dst, dst_bytes, n_out, ids);
}

template <typename real>
static pic_status get_rho_t(pic_ctx *c, void *dst, size_t dst_bytes, int dst_is_device)
{
    const size_t bytes = (size_t)c->g.ncomp * sizeof(real);
    if (dst_bytes < bytes) return fail(c, PIC_ERR_ARG, "destination too small");
    real *rho = (real *)(c->scratch + c->off_tmp);
    CUDA_TRY(c, cudaMemsetAsync(rho, 0, bytes, c->stream));
    launch_rho<real>(c->g, species_view<real>(c, 0, c->cur[0]), counts(c, 0, c->cur[0], 0), counts(c, 0, c->cur[0], 1),
                     (real)(-1.0 / c->vol), rho, c->stream);
    if (c->ions_species)
        launch_rho<real>(c->g, species_view<real>(c, 1, c->cur[1]), counts(c, 1, c->cur[1], 0),
                         counts(c, 1, c->cur[1], 1), (real)(1.0 / c->vol), rho, c->stream);
    CUDA_TRY(c, cudaGetLastError());
    CUDA_TRY(c, cudaMemcpyAsync(dst, rho, bytes, kind_out(dst_is_device), c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return PIC_OK;
}

extern "C" pic_status pic_get_rho(pic_ctx *c, void *dst, size_t dst_bytes, int dst_is_device)
{
    if (!c || !dst) return PIC_ERR_ARG;
    if (!c->bound) return fail(c, PIC_ERR_STATE, "bind buffers first");
    return c->es == 4 ? get_rho_t<float>(c, dst, dst_bytes, dst_is_device) : get_rho_t<double>(c, dst, dst_bytes, dst_is_device);
}

static double kahan_sum(const double *v, size_t n, size_t stride)
{
    double s = 0, comp = 0;
    for (size_t i = 0; i < n; ++i) {
        const double y = v[i * stride] - comp;
        const double t = s + y;
        comp = (t - s) - y;
        s = t;
    }
    return s;
}

template <typename real>
static pic_status diagnostics_t(pic_ctx *c, pic_diag *out)
{
    double *part = reinterpret_cast<double *>(c->scratch + c->off_partials);
    std::vector<double> h(3 * kPartialBlocks);
    real *F[9];
    for (int q = 0; q < 9; ++q) F[q] = (real *)field_ptr(c, q);
    launch_field_sums<real>(c->g, F, part, kPartialBlocks, c->stream);
    CUDA_TRY(c, cudaGetLastError());
    CUDA_TRY(c, cudaMemcpyAsync(h.data(), part, sizeof(double) * kPartialBlocks, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    out->field_energy = 0.5 * c->vol * kahan_sum(h.data(), kPartialBlocks, 1);
    out->kinetic_energy = 0;
    out->charge = 0;
    const real u_drift[3] = {0, 0, drift_u<real>(c)};
    for (int sp = 0; sp < (c->ions_species ? 2 : 1); ++sp) {
        launch_particle_sums<real>(c->g, species_view<real>(c, sp, c->cur[sp]), counts(c, sp, c->cur[sp], 0),
                                   counts(c, sp, c->cur[sp], 1), sp == 0 ? -1.0 : 1.0, u_drift, part, kPartialBlocks,
                                   c->stream);
        CUDA_TRY(c, cudaGetLastError());
        CUDA_TRY(c, cudaMemcpyAsync(h.data(), part, sizeof(double) * 3 * kPartialBlocks, cudaMemcpyDeviceToHost, c->stream));
        CUDA_TRY(c, cudaStreamSynchronize(c->stream));
        if (sp == 0) {
            out->kinetic_energy = kahan_sum(h.data(), kPartialBlocks, 3);
            double np = 0;
            for (int b = 0; b < kPartialBlocks; ++b) np += h[3 * b + 2];
            out->n_paired = (int64_t)np;
        }
        out->charge += kahan_sum(h.data() + 1, kPartialBlocks, 3);
    }
    return PIC_OK;
}

extern "C" pic_status pic_get_diagnostics(pic_ctx *c, pic_diag *out)
{
    if (!c || !out) return PIC_ERR_ARG;
    if (!c->bound) return fail(c, PIC_ERR_STATE, "bind buffers first");
    std::memset(out, 0, sizeof(*out));
    out->t = c->t;
    out->step = c->step;
    out->z_window = c->zwin();
    for (int sp = 0; sp < 2; ++sp) {
        if (sp == 1 && !c->ions_species) break;
        std::vector<int64_t> off;
        int64_t n = 0;
        pic_status s = tile_offsets(c, sp, off, n);
        if (s != PIC_OK) return s;
        out->n_particles[sp] = n;
    }
    pic_status s = c->es == 4 ? diagnostics_t<float>(c, out) : diagnostics_t<double>(c, out);
    if (s == PIC_OK) out->n_particles[1] += out->n_paired;
    return s;
}

// ---------------------------------------------------------------- checkpoint

static size_t species_state_bytes(const pic_ctx *c, int sp, int64_t n)
{
    size_t b = 0;
    for (int a = 0; a < kAttrs; ++a)
        if (c->side[sp].off[a] != SIZE_MAX) b += (size_t)n * attr_size(c, a);
    return b;
}

extern "C" pic_status pic_state_bytes(pic_ctx *c, size_t *bytes)
{
    if (!c || !bytes) return PIC_ERR_ARG;
    if (!c->bound) return fail(c, PIC_ERR_STATE, "bind buffers first");
    size_t b = sizeof(StateHeader) + c->field_bytes;
    for (int sp = 0; sp < (c->ions_species ? 2 : 1); ++sp) {
        std::vector<int64_t> off;
        int64_t n = 0;
        pic_status s = tile_offsets(c, sp, off, n);
        if (s != PIC_OK) return s;
        b += species_state_bytes(c, sp, n);
    }
    *bytes = b;
    return PIC_OK;
}

template <typename real>
static pic_status get_state_t(pic_ctx *c, unsigned char *dst, size_t dst_bytes, int dst_is_device)
{
    StateHeader h{};
    std::memcpy(h.magic, "PICSTAT4", 8);
    h.rel = c->rel;
    h.dim = c->g.dim;
    h.nx = c->g.nx;
    h.ny = c->g.ny;
    h.nz = c->g.nz;
    h.precision = c->p.precision;
    h.track_ids = c->p.track_ids;
    h.has_ions = c->ions_species;
    h.laser_on = c->laser_on;
    h.t = c->t;
    h.step = c->step;
    h.laser = c->laser;
    h.wmax = c->wmax;
    h.win_on = c->win_on;
    h.win_v = c->win_v;
    h.win_t0 = c->win_t0;
    h.win_S = c->win_S;
    h.win_n = c->win_n;
    int64_t n[2] = {0, 0};
    for (int sp = 0; sp < (c->ions_species ? 2 : 1); ++sp) {
        pic_status s = compact_t<real>(c, sp, n[sp]);
        if (s != PIC_OK) return s;
    }
    h.n[0] = n[0];
    h.n[1] = n[1];
    size_t need = sizeof(StateHeader) + c->field_bytes + species_state_bytes(c, 0, n[0]) +
                  (c->ions_species ? species_state_bytes(c, 1, n[1]) : 0);
    if (dst_bytes < need) return fail(c, PIC_ERR_ARG, "destination too small");
    CUDA_TRY(c, cudaMemcpyAsync(dst, &h, sizeof(h), dst_is_device ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost, c->stream));
    size_t o = sizeof(StateHeader);
    for (int q = 0; q < PIC_NCOMP; ++q) {
        const size_t per = (size_t)c->g.ncomp * c->es;
        CUDA_TRY(c, cudaMemcpyAsync(dst + o, field_ptr(c, q), per, kind_out(dst_is_device), c->stream));
        o += per;
    }
    for (int sp = 0; sp < (c->ions_species ? 2 : 1); ++sp) {
        void *col[kAttrs];
        side_raw(c, sp, c->cur[sp] ^ 1, col);
        for (int a = 0; a < kAttrs; ++a) {
            if (!col[a]) continue;
            const size_t b = (size_t)n[sp] * attr_size(c, a);
            if (b) CUDA_TRY(c, cudaMemcpyAsync(dst + o, col[a], b, kind_out(dst_is_device), c->stream));
            o += b;
        }
    }
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return PIC_OK;
}

extern "C" pic_status pic_get_state(pic_ctx *c, void *dst, size_t dst_bytes, int dst_is_device)
{
    if (!c || !dst) return PIC_ERR_ARG;
    if (!c->bound) return fail(c, PIC_ERR_STATE, "bind buffers first");
    return c->es == 4 ? get_state_t<float>(c, (unsigned char *)dst, dst_bytes, dst_is_device)
                      : get_state_t<double>(c, (unsigned char *)dst, dst_bytes, dst_is_device);
}

template <typename real>
static pic_status set_state_t(pic_ctx *c, const unsigned char *src, size_t src_bytes, int src_is_device)
{
    StateHeader h{};
    if (src_bytes < sizeof(h)) return fail(c, PIC_ERR_ARG, "snapshot too small");
    CUDA_TRY(c, cudaMemcpyAsync(&h, src, sizeof(h), src_is_device ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    if (std::memcmp(h.magic, "PICSTAT4", 8) != 0 || h.rel != (int)c->rel || h.dim != c->g.dim || h.nx != c->g.nx || h.ny != c->g.ny ||
        h.nz != c->g.nz || h.precision != c->p.precision || h.track_ids != c->p.track_ids ||
        h.has_ions != (int)c->ions_species || h.n[0] < 0 || h.n[1] < 0 || h.n[0] > c->slots || h.n[1] > c->slots ||
        !(h.wmax >= 0) || !std::isfinite(h.wmax))
        return fail(c, PIC_ERR_ARG, "snapshot does not match this grid");
    const size_t need = sizeof(StateHeader) + c->field_bytes + species_state_bytes(c, 0, h.n[0]) +
                        (c->ions_species ? species_state_bytes(c, 1, h.n[1]) : 0);
    if (src_bytes < need) return fail(c, PIC_ERR_ARG, "snapshot truncated");
    size_t o = sizeof(StateHeader);
    c->fset = 0;
    CUDA_TRY(c, cudaMemcpyAsync(c->fields, src + o, c->field_bytes, kind_in(src_is_device), c->stream));
    o += c->field_bytes;
    for (int sp = 0; sp < (c->ions_species ? 2 : 1); ++sp) {
        CUDA_TRY(c, cudaMemsetAsync(counts(c, sp, 0, 0), 0, sizeof(int) * 4 * (size_t)c->g.ntiles, c->stream));
        const void *cols[kAttrs] = {nullptr};
        for (int a = 0; a < kAttrs; ++a) {
            if (c->side[sp].off[a] == SIZE_MAX) continue;
            cols[a] = src + o;
            o += (size_t)h.n[sp] * attr_size(c, a);
        }
        if (h.n[sp] == 0) continue;
        pic_status s = upload_flat<real>(c, sp, h.n[sp], cols, src_is_device);
        if (s != PIC_OK) return s;
    }
    c->wmax = h.wmax;
    c->win_on = h.win_on != 0;
    c->win_v = h.win_v;
    c->win_t0 = h.win_t0;
    c->win_S = h.win_S;
    c->win_n = h.win_n;
    c->t = h.t;
    c->step = h.step;
    c->laser_on = h.laser_on != 0;
    c->laser = h.laser;
    if (c->laser_on) {
        int ka = (int)std::floor(c->laser.z_antenna / c->hz + 0.5);
        c->ka = ka < 2 ? 2 : (ka > c->g.nz - 2 ? c->g.nz - 2 : ka);
    }
    return PIC_OK;
}

extern "C" pic_status pic_set_state(pic_ctx *c, const void *src, size_t src_bytes, int src_is_device)
{
    if (!c || !src) return PIC_ERR_ARG;
    c->epoch += 1;
    if (!c->bound) return fail(c, PIC_ERR_STATE, "bind buffers first");
    return c->es == 4 ? set_state_t<float>(c, (const unsigned char *)src, src_bytes, src_is_device)
                      : set_state_t<double>(c, (const unsigned char *)src, src_bytes, src_is_device);
}

// ----------------------------------------------------------------- profiling

extern "C" pic_status pic_profile(pic_ctx *c, int enable)
{
    if (!c) return PIC_ERR_ARG;
    c->epoch += 1;
    c->profiling = enable != 0;
    return PIC_OK;
}

extern "C" pic_status pic_profile_read(pic_ctx *c, double ms[8], int64_t calls[8], int64_t *kernels)
{
    if (!c) return PIC_ERR_ARG;
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    double acc[8] = {0};
    int64_t cnt[8] = {0};
    for (const auto &u : c->ev_used) {
        float e = 0;
        CUDA_TRY(c, cudaEventElapsedTime(&e, c->ev_pool[u.second], c->ev_pool[u.second + 1]));
        acc[u.first] += e;
        cnt[u.first] += 1;
    }
    c->ev_used.clear();
    for (int q = 0; q < 8; ++q) {
        if (ms) ms[q] = acc[q];
        if (calls) calls[q] = cnt[q];
    }
    if (kernels) *kernels = c->kernels;
    c->kernels = 0;
    return PIC_OK;
}


// ------------------------------------------------------------------ adjoint

namespace {

// byte layout of an adjoint run's buffer
struct AdjLayout {
    int64_t P = 0;
    int N = 0, K = 0, C = 0;
    int K2 = 0, CS = 0;  // second level: sub-checkpoints every K2 steps of a segment (CS of them), 0: none
    size_t w = 0, zeta = 0, ion_ci = 0, ion_ox = 0, ion_cj = 0, ion_oy = 0;  // per slot, constant
    size_t st = 0, fl = 0;                           // one particle state, one field state (6 comps)
    size_t ckpt = 0, seg = 0, sub = 0;               // C, KS + 1 and CS (state, fields) pairs
    size_t J = 0, tmp = 0, lE = 0, lB = 0, lE0 = 0, pE = 0, lJ = 0;  // 3 components each
    size_t lx = 0, ly = 0, lz = 0, lux = 0, luy = 0, luz = 0, lw = 0, acc = 0, coef = 0, planes = 0;
    size_t total = 0;
    // inside one particle state
    size_t e_ci = 0, e_cj = 0, e_ck = 0, e_ox = 0, e_oy = 0, e_oz = 0, e_ux = 0, e_uy = 0, e_uz = 0, e_alive = 0;
    size_t i_ck = 0, i_oz = 0, i_alive = 0, fm = 0;
};

// K2 > 0 (and < K): segments are recomputed in two levels, so the segment
// buffer holds K2 + 1 states and ceil(K / K2) sub-checkpoints instead of K + 1
AdjLayout adj_layout(int64_t P, int N, int K, int K2, size_t es, int64_t ncomp, bool dim3, int64_t nz1)
{
    const int64_t P3 = dim3 ? P : 0;  // y arrays only in 3D
    AdjLayout L;
    L.P = P;
    L.N = N;
    L.K = K;
    L.C = (N + K - 1) / K;
    L.K2 = (K2 > 0 && K2 < K) ? K2 : 0;
    L.CS = L.K2 ? (K + L.K2 - 1) / L.K2 : 0;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o += align_up(bytes);
        return at;
    };
    // one particle state
    size_t q = 0;
    auto sub = [&](size_t bytes) {
        const size_t at = q;
        q += align_up(bytes);
        return at;
    };
    L.e_ci = sub(4 * P);
    L.e_cj = sub(4 * P3);
    L.e_ck = sub(4 * P);
    L.e_ox = sub(es * P);
    L.e_oy = sub(es * P3);
    L.e_oz = sub(es * P);
    L.e_ux = sub(es * P);
    L.e_uy = sub(es * P);
    L.e_uz = sub(es * P);
    L.e_alive = sub(P);
    L.i_ck = sub(4 * P);
    L.i_oz = sub(es * P);
    L.i_alive = sub(P);
    L.fm = sub(nz1);  // cells within reach of a nonzero field of the state
    L.st = q;
    L.fl = align_up(6 * es * ncomp);
    L.w = take(es * P);
    L.zeta = take(8 * P);
    L.ion_ci = take(4 * P);
    L.ion_ox = take(es * P);
    L.ion_cj = take(4 * P3);
    L.ion_oy = take(es * P3);
    L.ckpt = take((size_t)L.C * (L.st + L.fl));
    L.seg = take((size_t)((L.K2 ? L.K2 : K) + 1) * (L.st + L.fl));
    L.sub = take((size_t)L.CS * (L.st + L.fl));
    L.J = take(3 * es * ncomp);
    L.tmp = take(3 * es * ncomp);
    L.lE = take(3 * es * ncomp);
    L.lB = take(3 * es * ncomp);
    L.lE0 = take(3 * es * ncomp);
    L.pE = take(3 * es * ncomp);
    L.lJ = take(3 * es * ncomp);
    L.lx = take(es * P);
    L.ly = take(es * P3);
    L.lz = take(es * P);
    L.lux = take(es * P);
    L.luy = take(es * P);
    L.luz = take(es * P);
    L.lw = take(8 * P);
    L.acc = take(8 * 2);
    L.planes = take((size_t)nz1);
    L.coef = take(8 * 32);
    L.total = o;
    return L;
}

template <typename real>
FlatE<real> flat_e(unsigned char *st, const AdjLayout &L)
{
    FlatE<real> e;
    e.ci = (int *)(st + L.e_ci);
    e.cj = (int *)(st + L.e_cj);
    e.ck = (int *)(st + L.e_ck);
    e.ox = (real *)(st + L.e_ox);
    e.oy = (real *)(st + L.e_oy);
    e.oz = (real *)(st + L.e_oz);
    e.ux = (real *)(st + L.e_ux);
    e.uy = (real *)(st + L.e_uy);
    e.uz = (real *)(st + L.e_uz);
    e.alive = st + L.e_alive;
    return e;
}

template <typename real>
FlatI<real> flat_i(unsigned char *st, const AdjLayout &L)
{
    FlatI<real> i;
    i.ck = (int *)(st + L.i_ck);
    i.oz = (real *)(st + L.i_oz);
    i.alive = st + L.i_alive;
    return i;
}

}  // namespace

// lattice bands of the load and of every step's injection, their slot bases,
// and the step times (accumulated as the step does)
static void adj_bands(pic_ctx *c, int N)
{
    auto &A = c->adj;
    A.tn.assign(N + 1, 0.0);
    A.tn[0] = c->t;
    for (int n = 0; n < N; ++n) A.tn[n + 1] = A.tn[n] + c->dt;
    InjectArgs a{};
    fill_inject_common(c, a);
    A.mlo.assign(N + 1, 0);
    A.mhi.assign(N + 1, 0);
    A.base.assign(N + 2, 0);
    lattice_band(a, c->gam * (c->beta * A.tn[0]), c->gam * (c->Lz + c->beta * A.tn[0]), A.mlo[0], A.mhi[0]);
    if (c->gam > 1.0)
        for (int n = 0; n < N; ++n)
            lattice_band(a, c->gam * (c->Lz + c->beta * A.tn[n]), c->gam * (c->Lz + c->beta * A.tn[n + 1]),
                         A.mlo[n + 1], A.mhi[n + 1]);
    for (int b = 0; b <= N; ++b) A.base[b + 1] = A.base[b] + (A.mhi[b] - A.mlo[b]) * a.NY * a.NX;
    A.P = A.base[N + 1];
}

static pic_status adj_check(pic_ctx *c, const pic_adjoint_params *p)
{
    if (!c || !p) return PIC_ERR_ARG;
    if (!c->bound) return fail(c, PIC_ERR_STATE, "bind buffers first");
    if (p->nsteps < 1 || p->checkpoint_every < 1 || p->sub_checkpoint_every < 0)
        return fail(c, PIC_ERR_ARG, "invalid adjoint parameters");
    if (c->win_on) return fail(c, PIC_ERR_ARG, "the adjoint does not cover a moving window");
    if (!c->plasma_loaded || c->step != 0)
        return fail(c, PIC_ERR_STATE, "the adjoint starts right after pic_load_plasma (no step taken)");
    return PIC_OK;
}

extern "C" pic_status pic_adjoint_bytes(pic_ctx *c, const pic_adjoint_params *p, size_t *bytes)
{
    pic_status st = adj_check(c, p);
    if (st != PIC_OK) return st;
    if (!bytes) return PIC_ERR_ARG;
    adj_bands(c, p->nsteps);
    *bytes = adj_layout(c->adj.P, p->nsteps, p->checkpoint_every, p->sub_checkpoint_every, (size_t)c->es,
                        c->g.ncomp, c->g.dim == 3, c->g.nz + 1)
                 .total;
    return PIC_OK;
}

// the arguments every adjoint kernel of a step shares
template <typename real>
static void adj_common(pic_ctx *c, const AdjLayout &L, AdjArgs<real> &a)
{
    unsigned char *B = c->adj.buf;
    a.g = c->g;
    a.w = (const real *)(B + L.w);
    a.ion_ci = (const int *)(B + L.ion_ci);
    a.ion_cj = (const int *)(B + L.ion_cj);
    a.ion_ox = (const real *)(B + L.ion_ox);
    a.ion_oy = (const real *)(B + L.ion_oy);
    a.n = L.P;
    a.dtdh[0] = (real)(c->dt / c->hx);
    a.dtdh[1] = (real)(c->dt / c->hy);
    a.dtdh[2] = (real)(c->dt / c->hz);
    a.eps = (real)(kPi * -1.0 * c->dt);
    a.u_drift = drift_u<real>(c);
    // electrons (q = -1): -q h_d / (dt V); 2D out-of-plane q / V; ions (q = +1)
    a.jfac[0] = (real)(1.0 * c->hx / (c->dt * c->vol));
    a.jfac[1] = (real)(1.0 * c->hy / (c->dt * c->vol));
    a.jfac[2] = (real)(1.0 * c->hz / (c->dt * c->vol));
    a.jyfac = (real)(-1.0 / c->vol);
    a.jfac_iz = (real)(-1.0 * c->hz / (c->dt * c->vol));
    a.with_ions = c->ions_species ? 1 : 0;
}

// the flat-output pointers of an injection into state st
template <typename real>
static void adj_inject_out(pic_ctx *c, const AdjLayout &L, unsigned char *st, InjectArgs &ia)
{
    unsigned char *B = c->adj.buf;
    FlatE<real> e = flat_e<real>(st, L);
    FlatI<real> i = flat_i<real>(st, L);
    ia.fe_ci = e.ci;
    ia.fe_cj = e.cj;
    ia.fe_ck = e.ck;
    ia.fe_ox = e.ox;
    ia.fe_oy = e.oy;
    ia.fe_oz = e.oz;
    ia.fe_ux = e.ux;
    ia.fe_uy = e.uy;
    ia.fe_uz = e.uz;
    ia.fe_alive = e.alive;
    ia.fi_ck = i.ck;
    ia.fi_oz = i.oz;
    ia.fi_alive = i.alive;
    ia.f_ion_ci = (int *)(B + L.ion_ci);
    ia.f_ion_cj = (int *)(B + L.ion_cj);
    ia.f_ion_ox = B + L.ion_ox;
    ia.f_ion_oy = B + L.ion_oy;
    ia.f_w = B + L.w;
    ia.f_zeta = (double *)(B + L.zeta);
}

// one flat step n: state/fields slot a -> slot b
template <typename real>
static void adj_step(pic_ctx *c, const AdjLayout &L, unsigned char *sa, unsigned char *sb, unsigned char *fa,
                     unsigned char *fb, int n)
{
    unsigned char *B = c->adj.buf;
    const int64_t nc = c->g.ncomp;
    // the raw current goes to the filter's input buffer; the filter writes J
    real *J = (real *)(B + L.J), *R = (real *)(B + L.tmp);
    cudaMemsetAsync(R, 0, 3 * sizeof(real) * nc, c->stream);
    AdjArgs<real> a{};
    a.g = c->g;
    for (int q = 0; q < 3; ++q) {
        a.E[q] = (const real *)fa + q * nc;
        a.B[q] = (const real *)fa + (3 + q) * nc;
        a.J[q] = R + q * nc;
    }
    a.in = flat_e<real>(sa, L);
    a.out = flat_e<real>(sb, L);
    a.iin = flat_i<real>(sa, L);
    a.iout = flat_i<real>(sb, L);
    adj_common<real>(c, L, a);
    launch_adj_planes<real>(c->g, (const real *)fa, 6, sa + L.fm, c->stream);
    a.f_plane = sa + L.fm;
    launch_adj_push<real>(a, c->stream);
    real *Rc[3] = {R, R + nc, R + 2 * nc};
    if (c->laser_on && c->ka >= 2) {
        const pic_laser_params &l = c->laser;
        const double j0 = antenna_j0(c, c->adj.tn[n], l.a0);
        launch_antenna<real>(c->g, Rc[l.polarization == PIC_POL_X ? 0 : 1], l.polarization, c->ka, j0, c->hx, c->hy,
                             l.x_center, l.y_center, l.waist, c->stream);
    }
    real *Jc[3] = {J, J + nc, J + 2 * nc};
    if (c->p.filter_passes == 0) {
        for (int q = 0; q < 3; ++q) Jc[q] = Rc[q];
    } else if (!launch_filter_from<real>(c->g, R, Jc, c->p.filter_passes, c->stream)) {
        cudaMemcpyAsync(J, R, 3 * sizeof(real) * nc, cudaMemcpyDeviceToDevice, c->stream);
        launch_filter<real>(c->g, Jc, R, c->p.filter_passes, c->stream);
    }
    real *F[9], *F1[6];
    for (int q = 0; q < 6; ++q) {
        F[q] = (real *)fa + q * nc;
        F1[q] = (real *)fb + q * nc;
    }
    for (int q = 0; q < 3; ++q) F[6 + q] = Jc[q];
    launch_yee<real>(c->g, F, F1, c->dt, c->hx, c->hy, c->hz, c->stream);
    if (c->gam > 1.0 && c->adj.mhi[n + 1] > c->adj.mlo[n + 1]) {
        InjectArgs ia{};
        fill_inject_common(c, ia);
        ia.mode = 1;
        ia.t = c->adj.tn[n];
        ia.t1 = c->adj.tn[n + 1];
        ia.m_lo = c->adj.mlo[n + 1];
        ia.m_hi = c->adj.mhi[n + 1];
        ia.flat_base = c->adj.base[n + 1];
        adj_inject_out<real>(c, L, sb, ia);
        launch_inject(ia, c->stream);
    }
}

template <typename real>
static pic_status adj_forward_t(pic_ctx *c, const pic_adjoint_params *p, void *fields_out, bool defer)
{
    auto &A = c->adj;
    const AdjLayout L =
        adj_layout(A.P, p->nsteps, p->checkpoint_every, p->sub_checkpoint_every, sizeof(real), c->g.ncomp,
                   c->g.dim == 3, c->g.nz + 1);
    unsigned char *B = A.buf;
    unsigned char *seg = B + L.seg;
    auto st = [&](int s) { return seg + (size_t)s * (L.st + L.fl); };
    auto fl = [&](int s) { return seg + (size_t)s * (L.st + L.fl) + L.st; };
    auto ck_st = [&](int q) { return B + L.ckpt + (size_t)q * (L.st + L.fl); };
    const size_t fbytes = 6 * sizeof(real) * c->g.ncomp;
    // state 0: the plasma as loaded (into its fixed slots), the current fields;
    // slots no lattice point takes keep zero weights
    CUDA_TRY(c, cudaMemsetAsync(B + L.w, 0, L.ckpt - L.w, c->stream));
    CUDA_TRY(c, cudaMemsetAsync(st(0), 0, L.st, c->stream));
    CUDA_TRY(c, cudaMemsetAsync(st(1), 0, L.st, c->stream));
    for (int q = 0; q < 6; ++q)
        CUDA_TRY(c, cudaMemcpyAsync(fl(0) + q * sizeof(real) * c->g.ncomp, field_ptr(c, q),
                                    sizeof(real) * c->g.ncomp, cudaMemcpyDeviceToDevice, c->stream));
    {
        InjectArgs ia{};
        fill_inject_common(c, ia);
        ia.mode = 0;
        ia.t = A.tn[0];
        ia.t1 = A.tn[0];
        ia.m_lo = A.mlo[0];
        ia.m_hi = A.mhi[0];
        ia.flat_base = 0;
        adj_inject_out<real>(c, L, st(0), ia);
        launch_inject(ia, c->stream);
    }
    // steps before the last segment alternate between slots 0 and 1; the last
    // segment's states are kept in the slots the reverse sweep reads them
    // from, so that its first segment needs no recomputation (one-level
    // schedule; with sub-checkpoints every step alternates)
    const int nlast = L.K2 ? L.N + 1 : (L.C - 1) * L.K;
    for (int n = 0; n < L.N; ++n) {
        int a = n & 1, b = a ^ 1;
        if (n == nlast && a == 1) {
            CUDA_TRY(c, cudaMemcpyAsync(st(0), st(1), L.st + L.fl, cudaMemcpyDeviceToDevice, c->stream));
        }
        if (n >= nlast) {
            a = n - nlast;
            b = a + 1;
        }
        if (n % L.K == 0)
            CUDA_TRY(c, cudaMemcpyAsync(ck_st(n / L.K), st(a), L.st + L.fl, cudaMemcpyDeviceToDevice, c->stream));
        adj_step<real>(c, L, st(a), st(b), fl(a), fl(b), n);
    }
    CUDA_TRY(c, cudaGetLastError());
    if (fields_out)
        CUDA_TRY(c, cudaMemcpyAsync(fields_out, fl(L.K2 ? (L.N & 1) : L.N - nlast), fbytes, cudaMemcpyDeviceToDevice,
                                    c->stream));
    A.last_seg_ready = L.K2 == 0;
    A.ready = true;
    A.N = L.N;
    A.K = L.K;
    A.K2 = L.K2;
    return defer ? PIC_OK : check_device_error(c);
}

// defer: everything is queued on the context's stream, nothing waits for it
// (a batch checks the device error word after all its runs)
static pic_status adjoint_forward(pic_ctx *c, const pic_adjoint_params *p, void *buf, size_t bytes,
                                  void *fields_out, bool defer)
{
    pic_status s = adj_check(c, p);
    if (s != PIC_OK) return s;
    c->epoch += 1;
    if (!buf) return PIC_ERR_ARG;
    adj_bands(c, p->nsteps);
    if (bytes < adj_layout(c->adj.P, p->nsteps, p->checkpoint_every, p->sub_checkpoint_every, (size_t)c->es,
                           c->g.ncomp, c->g.dim == 3, c->g.nz + 1)
                    .total)
        return fail(c, PIC_ERR_ARG, "adjoint buffer too small");
    c->adj.buf = (unsigned char *)buf;
    c->adj.bytes = bytes;
    c->adj.ready = false;
    return c->es == 4 ? adj_forward_t<float>(c, p, fields_out, defer) : adj_forward_t<double>(c, p, fields_out, defer);
}

extern "C" pic_status pic_adjoint_forward(pic_ctx *c, const pic_adjoint_params *p, void *buf, size_t bytes,
                                          void *fields_out)
{
    return adjoint_forward(c, p, buf, bytes, fields_out, false);
}

// The reverse sweep queued on the context's stream; its sums (dL/da0,
// dL/dw0, then the M profile sums) are copied into the pinned adj.hgrad,
// which the caller reads after synchronising the stream (adj_grad_out).
template <typename real>
static pic_status adj_backward_t(pic_ctx *c, const void *cot)
{
    auto &A = c->adj;
    const AdjLayout L = adj_layout(A.P, A.N, A.K, A.K2, sizeof(real), c->g.ncomp, c->g.dim == 3, c->g.nz + 1);
    unsigned char *B = A.buf;
    const int64_t nc = c->g.ncomp;
    unsigned char *seg = B + L.seg;
    auto st = [&](int s) { return seg + (size_t)s * (L.st + L.fl); };
    auto fl = [&](int s) { return seg + (size_t)s * (L.st + L.fl) + L.st; };
    auto ck_st = [&](int q) { return B + L.ckpt + (size_t)q * (L.st + L.fl); };
    real *lE[3], *lB[3], *lE0[3], *pE[3], *lJ[3], *lJr[3];
    for (int q = 0; q < 3; ++q) {
        lE[q] = (real *)(B + L.lE) + q * nc;
        lB[q] = (real *)(B + L.lB) + q * nc;
        lE0[q] = (real *)(B + L.lE0) + q * nc;
        pE[q] = (real *)(B + L.pE) + q * nc;
        lJ[q] = (real *)(B + L.lJ) + q * nc;
        lJr[q] = (real *)(B + L.tmp) + q * nc;
    }
    const size_t cb = 3 * sizeof(real) * nc;
    CUDA_TRY(c, cudaMemcpyAsync(lE[0], cot, cb, cudaMemcpyDeviceToDevice, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(lB[0], (const unsigned char *)cot + cb, cb, cudaMemcpyDeviceToDevice, c->stream));
    for (size_t off : {L.lx, L.lz, L.lux, L.luy, L.luz})
        CUDA_TRY(c, cudaMemsetAsync(B + off, 0, sizeof(real) * L.P, c->stream));
    if (c->g.dim == 3) CUDA_TRY(c, cudaMemsetAsync(B + L.ly, 0, sizeof(real) * L.P, c->stream));
    CUDA_TRY(c, cudaMemsetAsync(B + L.lw, 0, 8 * L.P, c->stream));
    CUDA_TRY(c, cudaMemsetAsync(B + L.acc, 0, 16, c->stream));
    const pic_laser_params &l = c->laser;
    const int comp = l.polarization == PIC_POL_X ? 0 : 1;
    auto sub_st = [&](int q) { return B + L.sub + (size_t)q * (L.st + L.fl); };
    // the reverse sweep over the states st(0..n1 - n0) of steps n0..n1 - 1
    auto reverse = [&](int n0, int n1) -> pic_status {
        for (int s = n1 - n0 - 1; s >= 0; --s) {
            const int n = n0 + s;
            // the current cotangent before the filter goes to the scratch
            // buffer, the filter (its own transpose) writes lJ
            launch_adj_yee<real>(c->g, lE, lB, lE0, pE, lJr, c->dt, c->hx, c->hy, c->hz, c->stream);
            for (int q = 0; q < 3; ++q) std::swap(lE[q], lE0[q]);
            if (c->p.filter_passes == 0 || !launch_filter_from<real>(c->g, lJr[0], lJ, c->p.filter_passes, c->stream)) {
                CUDA_TRY(c, cudaMemcpyAsync(lJ[0], lJr[0], 3 * sizeof(real) * nc, cudaMemcpyDeviceToDevice, c->stream));
                launch_filter<real>(c->g, lJ, lJr[0], c->p.filter_passes, c->stream);
            }
            launch_adj_planes<real>(c->g, lJ[0], 3, B + L.planes, c->stream);
            if (c->laser_on && c->ka >= 2) {
                const double j0 = antenna_j0(c, A.tn[n], l.a0);
                // j0 is linear in a0; the profile exp(-r^2/w0^2) gives 2 r^2 / w0^3
                const double ja = antenna_j0(c, A.tn[n], 1.0);
                launch_adj_antenna<real>(c->g, lJ[comp], l.polarization, c->ka, c->hx, c->hy, l.x_center,
                                         l.y_center, l.waist, ja, j0 * 2.0 / (l.waist * l.waist * l.waist),
                                         (double *)(B + L.acc), c->stream);
            }
            AdjArgs<real> a{};
            a.g = c->g;
            for (int q = 0; q < 3; ++q) {
                a.E[q] = (const real *)fl(s) + q * nc;
                a.B[q] = (const real *)fl(s) + (3 + q) * nc;
                a.J[q] = lJ[q];
                a.lE[q] = lE[q];
                a.lB[q] = lB[q];
            }
            a.in = flat_e<real>(st(s), L);
            a.iin = flat_i<real>(st(s), L);
            adj_common<real>(c, L, a);
            a.lx = (real *)(B + L.lx);
            a.ly = (real *)(B + L.ly);
            a.lz = (real *)(B + L.lz);
            a.lux = (real *)(B + L.lux);
            a.luy = (real *)(B + L.luy);
            a.luz = (real *)(B + L.luz);
            a.lw = (double *)(B + L.lw);
            a.lj_plane = B + L.planes;
            a.f_plane = st(s) + L.fm;  // made by the forward step from this state
            launch_adj_push_vjp<real>(a, c->stream);
        }
        return PIC_OK;
    };
    for (int sgi = L.C - 1; sgi >= 0; --sgi) {
        const int n0 = sgi * L.K, n1 = std::min(L.N, n0 + L.K);
        if (sgi == L.C - 1 && A.last_seg_ready) {
            A.last_seg_ready = false;  // kept by the forward run, used once
            reverse(n0, n1);
        } else if (!L.K2) {
            CUDA_TRY(c, cudaMemcpyAsync(st(0), ck_st(sgi), L.st + L.fl, cudaMemcpyDeviceToDevice, c->stream));
            for (int s = 0; s < n1 - n0; ++s) adj_step<real>(c, L, st(s), st(s + 1), fl(s), fl(s + 1), n0 + s);
            reverse(n0, n1);
        } else {
            // two levels: the segment once through slots 0 and 1, leaving a
            // sub-checkpoint every K2 steps, then each sub-segment again with
            // all its states, backwards
            CUDA_TRY(c, cudaMemcpyAsync(sub_st(0), ck_st(sgi), L.st + L.fl, cudaMemcpyDeviceToDevice, c->stream));
            CUDA_TRY(c, cudaMemcpyAsync(st(0), ck_st(sgi), L.st + L.fl, cudaMemcpyDeviceToDevice, c->stream));
            for (int s = 0; s + 1 < n1 - n0; ++s) {
                const int a = s & 1, b = a ^ 1;
                adj_step<real>(c, L, st(a), st(b), fl(a), fl(b), n0 + s);
                if ((s + 1) % L.K2 == 0)
                    CUDA_TRY(c, cudaMemcpyAsync(sub_st((s + 1) / L.K2), st(b), L.st + L.fl, cudaMemcpyDeviceToDevice,
                                                c->stream));
            }
            for (int m = (n1 - n0 - 1) / L.K2; m >= 0; --m) {
                const int m0 = n0 + m * L.K2, m1 = std::min(n1, m0 + L.K2);
                CUDA_TRY(c, cudaMemcpyAsync(st(0), sub_st(m), L.st + L.fl, cudaMemcpyDeviceToDevice, c->stream));
                for (int s = 0; s < m1 - m0; ++s) adj_step<real>(c, L, st(s), st(s + 1), fl(s), fl(s + 1), m0 + s);
                reverse(m0, m1);
            }
        }
    }
    // the profile coefficients enter through every weight
    const int M = c->plasma.n_profile;
    if (!A.hgrad) CUDA_TRY(c, cudaMallocHost(&A.hgrad, sizeof(double) * (2 + 16 + 16)));
    double *h = A.hgrad;
    if (M > 0) {
        CUDA_TRY(c, cudaMemcpyAsync(B + L.coef, c->prof, 8 * 16, cudaMemcpyHostToDevice, c->stream));
        CUDA_TRY(c, cudaMemsetAsync(B + L.coef + 8 * 16, 0, 8 * 16, c->stream));
        launch_adj_profile(L.P, (const double *)(B + L.lw), B + L.w, sizeof(real) == 8 ? 1 : 0,
                           (const double *)(B + L.zeta), M, (const double *)(B + L.coef),
                           (double *)(B + L.coef + 8 * 16), c->stream);
        CUDA_TRY(c, cudaMemcpyAsync(h + 2, B + L.coef + 8 * 16, 8 * M, cudaMemcpyDeviceToHost, c->stream));
    }
    CUDA_TRY(c, cudaMemcpyAsync(h, B + L.acc, 16, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaGetLastError());
    return PIC_OK;
}

// after the stream has been synchronised: grad = dL/dc_1..M, dL/da0, dL/dw0
static pic_status adj_grad_out(pic_ctx *c, double *grad)
{
    const int M = c->plasma.n_profile;
    const double *h = c->adj.hgrad;
    for (int m = 0; m < M; ++m) grad[m] = h[2 + m];
    grad[M] = h[0];
    grad[M + 1] = h[1];
    return check_device_error(c);
}

extern "C" pic_status pic_adjoint_backward(pic_ctx *c, const void *cot, double *grad)
{
    if (!c || !cot || !grad) return PIC_ERR_ARG;
    c->epoch += 1;
    if (!c->adj.ready) return fail(c, PIC_ERR_STATE, "run pic_adjoint_forward first");
    const pic_status s = c->es == 4 ? adj_backward_t<float>(c, cot) : adj_backward_t<double>(c, cot);
    if (s != PIC_OK) return s;
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return adj_grad_out(c, grad);
}

// The gradients of all runs of a batch: every run's forward, then every
// run's reverse sweep, each queued on its own stream without waiting, so the
// runs' adjoint kernels execute concurrently; one wait per stream at the end.
extern "C" pic_status pic_batch_adjoint(pic_batch *b, const pic_adjoint_params *p, void *const *bufs,
                                        const size_t *bytes, const void *const *cots, double *grads, int grad_stride)
{
    if (!b || !p || !bufs || !bytes || !cots || !grads || grad_stride < 2) return PIC_ERR_ARG;
    const size_t n = b->ctx.size();
    for (size_t i = 0; i < n; ++i)
        if (b->ctx[i]->plasma.n_profile + 2 > grad_stride || !cots[i]) return PIC_ERR_ARG;
    if (b->gr.cs) cudaStreamSynchronize(b->gr.cs);  // replays of the batch's graph are done
    pic_status first = PIC_OK;
    std::vector<char> ok(n, 0);
    for (size_t i = 0; i < n; ++i) {
        const pic_status s = adjoint_forward(b->ctx[i], &p[i], bufs[i], bytes[i], nullptr, true);
        if (s != PIC_OK && first == PIC_OK) first = s;
        ok[i] = s == PIC_OK;
    }
    for (size_t i = 0; i < n; ++i) {
        if (!ok[i]) continue;
        pic_ctx *c = b->ctx[i];
        c->epoch += 1;
        const pic_status s = c->es == 4 ? adj_backward_t<float>(c, cots[i]) : adj_backward_t<double>(c, cots[i]);
        if (s != PIC_OK && first == PIC_OK) first = s;
        ok[i] = s == PIC_OK;
    }
    for (size_t i = 0; i < n; ++i) {
        if (!ok[i]) continue;
        pic_ctx *c = b->ctx[i];
        const cudaError_t e = cudaStreamSynchronize(c->stream);
        pic_status s = e == cudaSuccess ? adj_grad_out(c, grads + i * (size_t)grad_stride)
                                        : fail(c, PIC_ERR_CUDA, cudaGetErrorString(e));
        if (s != PIC_OK && first == PIC_OK) first = s;
    }
    return first;
}

// ---------------------------------------------------------------------- misc

extern "C" const char *pic_last_error(const pic_ctx *c) { return c ? c->err.c_str() : "null context"; }

extern "C" const char *pic_status_string(pic_status s)
{
    switch (s) {
    case PIC_OK: return "ok";
    case PIC_ERR_ARG: return "invalid argument";
    case PIC_ERR_STATE: return "call out of order";
    case PIC_ERR_CUDA: return "CUDA error";
    case PIC_ERR_CAPACITY: return "tile bucket overflow";
    case PIC_ERR_CFL: return "Courant condition violated";
    case PIC_ERR_NAN: return "non-finite value";
    case PIC_ERR_TIMEOUT: return "device wait timed out";
    }
    return "unknown status";
}

extern "C" void pic_destroy(pic_ctx *c) { delete c; }
