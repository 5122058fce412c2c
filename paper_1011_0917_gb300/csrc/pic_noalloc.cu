// pic_noalloc.cu -- the current filter for callers that cannot allocate
// device memory (pic_filter_current_noalloc in include/pic.h).
//
// The regular FILTER phase ping-pongs Jx, Jy, Jz through a scratch buffer that
// the caller allocates and binds.  Some callers have no such buffer to give:
// an application whose device memory all belongs to another framework's
// allocator, or code under a fixed device-memory budget or in a loop that must
// never allocate.  This file gives them the same filter with its scratch in a
// file-scope device array of fixed size, so nothing is allocated or freed.
// The array's device address is looked up once per device (host code may not
// pass the array's name to a kernel: in host code it is only a stand-in).
#include "pic.h"
#include "pic_internal.cuh"

#include <mutex>

namespace {

// one field component of scratch, the largest precision: 32 MiB per device
static __device__ __align__(256) double g_filter_scratch[PIC_NOALLOC_MAX_NODES];

constexpr int kMaxDevices = 128;
std::mutex g_lock;
void *g_scratch[kMaxDevices] = {nullptr};
int g_sms[kMaxDevices] = {0};

// device address of the scratch array on the current device and that
// device's multiprocessor count (both looked up once per device)
cudaError_t scratch_address(void **out, int *sms)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> guard(g_lock);
    if (!g_scratch[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_filter_scratch);
        if (e != cudaSuccess) return e;
        int n = 0;
        e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        g_sms[dev] = n > 0 ? n : 1;
        g_scratch[dev] = p;
    }
    *out = g_scratch[dev];
    *sms = g_sms[dev];
    return cudaSuccess;
}

// one (1/4, 1/2, 1/4) pass of a single component along `axis`, the same
// arithmetic and boundary rules as the FILTER phase's kernel
template <typename real>
__global__ void filter_one_kernel(pic::Geom g, const real *in, real *out, int axis, bool half_z)
{
    const int64_t n = g.ncomp;
    const int zmax = pic::zmax_of(g, half_z);
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(r % g.nx);
        const int j = (int)((r / g.nx) % g.ny);
        const int k = (int)(r / g.plane);
        if (k > zmax) {
            out[r] = 0;
            continue;
        }
        real lo, hi;
        if (axis == 0) {
            lo = in[pic::fidx(g, i == 0 ? g.nx - 1 : i - 1, j, k)];
            hi = in[pic::fidx(g, i + 1 == g.nx ? 0 : i + 1, j, k)];
        } else if (axis == 1) {
            lo = in[pic::fidx(g, i, j == 0 ? g.ny - 1 : j - 1, k)];
            hi = in[pic::fidx(g, i, j + 1 == g.ny ? 0 : j + 1, k)];
        } else if (g.bc_z == 0) {
            lo = in[pic::fidx(g, i, j, k == 0 ? g.nz - 1 : k - 1)];
            hi = in[pic::fidx(g, i, j, k + 1 == g.nz ? 0 : k + 1)];
        } else {
            lo = k > 0 ? in[pic::fidx(g, i, j, k - 1)] : real(0);
            hi = k < zmax ? in[pic::fidx(g, i, j, k + 1)] : real(0);
        }
        out[r] = real(0.25) * lo + real(0.5) * in[r] + real(0.25) * hi;
    }
}

template <typename real>
cudaError_t filter_all(const pic::Geom &g, int passes, real *const J[3], real *tmp, int sms, cudaStream_t s)
{
    // a grid-stride loop: at most 8 resident CTAs of 256 threads per SM
    int64_t blocks = (g.ncomp + 255) / 256;
    if (blocks > 8LL * sms) blocks = 8LL * sms;
    for (int c = 0; c < 3; ++c) {
        real *src = J[c], *dst = tmp;
        int done = 0;
        for (int axis = 0; axis < 3; ++axis) {
            if (axis == 1 && g.dim != 3) continue;
            for (int p = 0; p < passes; ++p) {
                filter_one_kernel<real><<<(unsigned)blocks, 256, 0, s>>>(g, src, dst, axis, c == 2);
                real *t = src;
                src = dst;
                dst = t;
                ++done;
            }
        }
        if (done & 1) {
            cudaError_t e = cudaMemcpyAsync(J[c], tmp, sizeof(real) * g.ncomp, cudaMemcpyDeviceToDevice, s);
            if (e != cudaSuccess) return e;
        }
    }
    return cudaGetLastError();
}

}  // namespace

extern "C" pic_status pic_filter_current_noalloc(int dim, int nx, int ny, int nz, int bc_z, int passes, int precision,
                                                 void *jx, void *jy, void *jz, void *stream)
{
    if ((dim != 2 && dim != 3) || nx < 1 || ny < 1 || nz < 4 || (dim == 2 && ny != 1)) return PIC_ERR_ARG;
    if ((bc_z != PIC_BC_MUR && bc_z != PIC_BC_PERIODIC) || passes < 0 || passes > 64) return PIC_ERR_ARG;
    if ((precision != PIC_FP32 && precision != PIC_FP64) || !jx || !jy || !jz) return PIC_ERR_ARG;
    const int64_t nodes = (int64_t)(nz + 1) * ny * nx;
    if (nodes > (int64_t)PIC_NOALLOC_MAX_NODES) return PIC_ERR_ARG;
    if (passes == 0) return PIC_OK;
    void *scratch = nullptr;
    int sms = 1;
    if (scratch_address(&scratch, &sms) != cudaSuccess) return PIC_ERR_CUDA;
    pic::Geom g{};
    g.dim = dim;
    g.nx = nx;
    g.ny = ny;
    g.nz = nz;
    g.bc_z = bc_z == PIC_BC_PERIODIC ? 0 : 1;
    g.plane = (int64_t)nx * ny;
    g.ncomp = nodes;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    if (precision == PIC_FP32) {
        float *J[3] = {(float *)jx, (float *)jy, (float *)jz};
        e = filter_all<float>(g, passes, J, (float *)scratch, sms, s);
    } else {
        double *J[3] = {(double *)jx, (double *)jy, (double *)jz};
        e = filter_all<double>(g, passes, J, (double *)scratch, sms, s);
    }
    return e == cudaSuccess ? PIC_OK : PIC_ERR_CUDA;
}
